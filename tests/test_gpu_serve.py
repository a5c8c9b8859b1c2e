"""The serving loop: requests of many systems queued as they arrive, evaluated by
concurrent slots with continuous batching (one forest per batch).  Every result
must be bit for bit the system's result alone; admission follows the footprint."""
import threading

import numpy as np
import pytest

from paper_1405_2255_gb300 import inputs

pytestmark = pytest.mark.gpu

PRM = dict(p=8, eps=1e-6, leaf_size=32, p2p_c=2.0)


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_2255_gb300 import build
    build.build()
    from paper_1405_2255_gb300 import gb3fmm
    gb3fmm.load()
    return gb3fmm


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _systems(k, seed):
    out = []
    for i, n in enumerate(inputs.ensemble_sizes(k, seed, 3.0, 1.5)):
        s = inputs.system_seed(seed, i)
        x, mu = inputs.plummer(int(n), s) if i % 2 == 0 else inputs.dehnen(int(n), s)
        out.append((_dev(x), _dev(mu), 0.5 + i))
    return out


def _alone(g, systems):
    ctx = g.Context(**PRM)
    res = [ctx.fmm_evaluate(x, mu, G) for x, mu, G in systems]
    out = [(p.cpu().numpy(), a.cpu().numpy()) for p, a in res]
    ctx.close()
    return out


def test_served_results_equal_alone(g):
    import torch
    systems = _systems(10, inputs.BASE_SEED + 5)
    ref = _alone(g, systems)
    ctx = g.Context(**PRM)
    ids = [ctx.fmm_system_register(len(mu)) for _, mu, _ in systems]
    outs = [(torch.empty(len(mu), dtype=torch.float64, device="cuda:0"),
             torch.empty((len(mu), 3), dtype=torch.float64, device="cuda:0")) for _, mu, _ in systems]
    torch.cuda.synchronize()
    for rnd in range(2):
        tickets = [ctx.fmm_submit(i, x, mu, G, *o) for i, (x, mu, G), o in zip(ids, systems, outs)]
        lats = [ctx.fmm_poll(t, 60000) for t in tickets]
        assert all(l is not None and l > 0 for l in lats)
        for (p_ref, a_ref), (p, a) in zip(ref, outs):
            assert np.array_equal(p.cpu().numpy(), p_ref)
            assert np.array_equal(a.cpu().numpy(), a_ref)
    for i in ids:
        ctx.fmm_system_release(i)
    ctx.close()


def test_concurrent_submitters(g):
    """Four host threads, each driving two systems through three requests with pauses:
    requests arrive while others run and land in different batches and slots."""
    import time
    import torch
    systems = _systems(8, inputs.BASE_SEED + 55)
    ref = _alone(g, systems)
    ctx = g.Context(**PRM)
    ctx.fmm_serve_config(0, 3)
    ids = [ctx.fmm_system_register(len(mu)) for _, mu, _ in systems]
    outs = [[(torch.empty(len(mu), dtype=torch.float64, device="cuda:0"),
              torch.empty((len(mu), 3), dtype=torch.float64, device="cuda:0")) for _ in range(3)]
            for _, mu, _ in systems]
    torch.cuda.synchronize()
    errors = []

    def client(w):
        try:
            rng = np.random.default_rng(w)
            for r in range(3):
                mine = [2 * w, 2 * w + 1]
                ts = []
                for k in mine:
                    x, mu, G = systems[k]
                    ts.append(ctx.fmm_submit(ids[k], x, mu, G, *outs[k][r]))
                    time.sleep(rng.uniform(0, 0.004))
                for t in ts:
                    assert ctx.fmm_poll(t, 60000) is not None
        except Exception as e:  # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=client, args=(w,)) for w in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join(120)
    assert not errors, errors
    for k, (p_ref, a_ref) in enumerate(ref):
        for p, a in outs[k]:
            assert np.array_equal(p.cpu().numpy(), p_ref)
            assert np.array_equal(a.cpu().numpy(), a_ref)
    ctx.close()


def test_admission_by_footprint(g):
    ctx = g.Context(**PRM)
    share = g.fmm_footprint_bytes(100_000, **PRM)
    ctx.fmm_serve_config(2 * share, 2)
    ctx.fmm_system_register(100_000)
    ctx.fmm_system_register(50_000)
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_system_register(200_000)
    assert e.value.code == g.FMM_E_ADMISSION
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_serve_config(0, 2)  # the loop is already running
    assert e.value.code == g.FMM_E_BUSY
    ctx.close()


def test_busy_release_and_unknown(g):
    import torch
    n = 1_000_000  # tens of milliseconds on the device: the next calls find it in flight
    x, mu = inputs.plummer(n, 8)
    xd, md = _dev(x), _dev(mu)
    psi = torch.empty(n, dtype=torch.float64, device="cuda:0")
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda:0")
    ctx = g.Context(**PRM)
    sid = ctx.fmm_system_register(n)
    torch.cuda.synchronize()
    t = ctx.fmm_submit(sid, xd, md, 1.0, psi, acc)
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_submit(sid, xd, md, 1.0, psi, acc)
    assert e.value.code == g.FMM_E_BUSY
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_system_release(sid)
    assert e.value.code == g.FMM_E_BUSY
    if ctx.fmm_poll(t, 0) is None:  # not waiting: still running (else it just completed)
        assert ctx.fmm_poll(t, 60000) is not None
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_poll(t, 0)  # retired
    assert e.value.code == g.FMM_E_NOTFOUND
    ctx.fmm_system_release(sid)
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_submit(sid, xd, md, 1.0, psi, acc)
    assert e.value.code == g.FMM_E_NOTFOUND
    ctx.close()


@pytest.mark.parametrize("model,n", [("plummer", 200_000), ("dehnen", 200_000), ("plummer", 2_000)])
@pytest.mark.parametrize("prm", [dict(PRM), dict(p=12, eps=2e-7, leaf_size=64, p2p_c=4.0)])
def test_workspace_within_footprint(g, model, n, prm):
    x, mu = (inputs.plummer if model == "plummer" else inputs.dehnen)(n, 77)
    ctx = g.Context(**prm)
    ctx.fmm_evaluate(_dev(x), _dev(mu))
    assert ctx.fmm_workspace_bytes() <= g.fmm_footprint_bytes(n, **prm)
    ctx.close()
