"""The allocation-free entry point fmm_evaluate_noalloc, called through the C ABI.

Callers that cannot allocate device memory (simulation codes whose device memory
belongs to their own pool allocator, plugins that may not grow the process's
footprint) evaluate small systems with it; the library takes all its scratch from
one fixed array in device memory.  This file is collected last so
that a run stopping at the first failure has run every other test first; it also
passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1405_2255_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64-mode parity tolerance of the other GPU tests


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


def _rel(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_evaluate_on_two_calls(g, precision):
    import torch
    prm = dict(p=8, eps=1e-6, leaf_size=32, p2p_c=4.0, precision=precision)
    ctx = g.Context(**prm)
    # two calls in a row with different systems: the second must not see the first's leftovers
    for seed, n in ((inputs.BASE_SEED + 11, 3000), (inputs.BASE_SEED + 12, 5000)):
        x, mu = inputs.plummer(n, seed)
        xd, md = _dev(x), _dev(mu)
        psi_ref, acc_ref = ctx.fmm_evaluate(xd, md, 1.0)
        psi = torch.empty(n, dtype=torch.float64, device="cuda:0")
        acc = torch.empty((n, 3), dtype=torch.float64, device="cuda:0")
        g.fmm_evaluate_noalloc(xd, md, 1.0, psi=psi, acc=acc, **prm)
        torch.cuda.synchronize()
        a, ar = acc.cpu().numpy(), acc_ref.cpu().numpy()
        assert np.max(_rel(a, ar)) <= TOL
        assert np.max(np.abs(psi.cpu().numpy() - psi_ref.cpu().numpy()) / psi_ref.cpu().numpy()) <= TOL
    ctx.close()


def test_noalloc_mixed_any_units(g):
    """The working units of the mixed path here too: positions x 2^70 and masses x 2^100
    give Psi x 2^30 and a x 2^-40, bit for bit."""
    import torch
    prm = dict(p=8, eps=1e-6, leaf_size=32, p2p_c=4.0, precision=1)
    x, mu = inputs.plummer(4000, inputs.BASE_SEED + 13)
    out = []
    for ex, em in ((0, 0), (70, 100)):
        psi = torch.empty(len(mu), dtype=torch.float64, device="cuda:0")
        acc = torch.empty((len(mu), 3), dtype=torch.float64, device="cuda:0")
        g.fmm_evaluate_noalloc(_dev(np.ldexp(x, ex)), _dev(np.ldexp(mu, em)), 1.0, psi=psi, acc=acc, **prm)
        torch.cuda.synchronize()
        out.append((psi.cpu().numpy(), acc.cpu().numpy()))
    assert np.all(np.isfinite(out[0][1]))
    assert np.array_equal(out[1][0], np.ldexp(out[0][0], 30))
    assert np.array_equal(out[1][1], np.ldexp(out[0][1], -40))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("model", ["plummer", "cusp"])
def test_noalloc_at_its_documented_limits(g, precision, model):
    """The largest documented case fits the fixed array: n = 8192, p = 10, leaf_size = 24
    (eps 1e-7, p2p_c 2), both precisions, with the same result as fmm_evaluate."""
    import torch
    prm = dict(p=10, eps=1e-7, leaf_size=24, p2p_c=2.0, precision=precision)
    x, mu = (inputs.plummer if model == "plummer" else inputs.dehnen)(8192, inputs.BASE_SEED + 14)
    xd, md = _dev(x), _dev(mu)
    ctx = g.Context(**prm)
    psi_ref, acc_ref = ctx.fmm_evaluate(xd, md, 1.0)
    psi = torch.empty(8192, dtype=torch.float64, device="cuda:0")
    acc = torch.empty((8192, 3), dtype=torch.float64, device="cuda:0")
    g.fmm_evaluate_noalloc(xd, md, 1.0, psi=psi, acc=acc, **prm)
    torch.cuda.synchronize()
    assert np.max(_rel(acc.cpu().numpy(), acc_ref.cpu().numpy())) <= TOL
    ctx.close()


def test_noalloc_reports_list_overflow(g):
    """Lists longer than the fixed capacity end in FMM_E_OVERFLOW, not in a wrong result."""
    x, mu = inputs.plummer(8192, inputs.BASE_SEED + 15)
    with pytest.raises(g.FMMError) as e:
        g.fmm_evaluate_noalloc(_dev(x), _dev(mu), 1.0, p=10, eps=1e-9, leaf_size=24, p2p_c=0.0)
    assert e.value.code == g.FMM_E_OVERFLOW


def test_noalloc_rejects_too_many_particles(g):
    x, mu = inputs.plummer(8193, 3)
    with pytest.raises(g.FMMError) as e:
        g.fmm_evaluate_noalloc(_dev(x), _dev(mu), 1.0, p=6, leaf_size=32)
    assert e.value.code == g.FMM_E_INVALID
    assert "8192" in str(e.value)
