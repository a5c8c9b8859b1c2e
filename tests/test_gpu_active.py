"""GPU force evaluation for a subset of the particles (Sec. 7.1, fmm_evaluate_active)
against the oracle's subset run and against the library's own full evaluation."""
import numpy as np
import pytest

from paper_1405_2255_gb300 import inputs

pytestmark = pytest.mark.gpu

PARITY_TOL = 1e-10


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
    return np.linalg.norm(a - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


def _subsets(x, seed):
    rng = np.random.default_rng(seed)
    r = np.linalg.norm(x, axis=1)
    return {"central": r < np.median(r) * 0.5, "sparse": rng.random(len(r)) < 0.02,
            "one": np.arange(len(r)) == 17, "none": np.zeros(len(r), bool)}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_all_active_equals_full(g, prec):
    x, mu = inputs.plummer(20000, inputs.BASE_SEED + 111)
    p = g.FMM_PREC_FP64 if prec == "fp64" else g.FMM_PREC_MIXED
    ctx = g.Context(p=8, eps=1e-7, leaf_size=32, p2p_c=2.0, precision=p)
    psi, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    import torch
    psi_a, acc_a = ctx.fmm_evaluate_active(_dev(x), _dev(mu), torch.ones(20000, dtype=torch.uint8, device="cuda:0"))
    assert torch.equal(psi, psi_a) and torch.equal(acc, acc_a)
    ctx.close()


@pytest.mark.parametrize("which", ["central", "sparse", "one"])
def test_fp64_subset_matches_oracle(g, orc, which):
    """FP64 mode: the subset run against the oracle's subset run element by element."""
    x, mu = inputs.plummer(6000, inputs.BASE_SEED + 112)
    act = _subsets(x, 5)[which]
    kw = dict(p=6, eps=1e-7, leaf_size=16, p2p_c=1.0)
    ctx = g.Context(precision=g.FMM_PREC_FP64, **kw)
    psi, acc, st = ctx.fmm_evaluate_active(_dev(x), _dev(mu), _dev(act.astype(np.uint8)), stats=True)
    run = orc.fmm(x, mu, active=act, **kw)
    psi, acc = psi.cpu().numpy(), acc.cpu().numpy()
    assert st["n_m2l"] == run.stats["n_m2l"] and st["n_p2p"] == run.stats["n_p2p"]
    assert np.max(_rel(acc[act], run.acc[act])) <= PARITY_TOL
    assert np.max(np.abs(psi[act] - run.psi[act]) / np.abs(run.psi[act])) <= PARITY_TOL
    # the outputs of inactive particles are not written (NaN from the wrapper stays)
    assert np.isnan(acc[~act]).all() and np.isnan(psi[~act]).all()
    ctx.close()


def test_empty_subset_writes_nothing(g):
    import torch
    x, mu = inputs.plummer(3000, inputs.BASE_SEED + 113)
    ctx = g.Context()
    psi, acc, st = ctx.fmm_evaluate_active(_dev(x), _dev(mu), torch.zeros(3000, dtype=torch.uint8, device="cuda:0"),
                                           stats=True)
    assert torch.isnan(psi).all() and torch.isnan(acc).all()
    assert st["n_m2l"] == 0 and st["n_p2p"] == 0
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_geometric_mac_subset_equals_full(g, prec):
    """With the geometric criterion the active particles get exactly the interactions of the
    full run: identical results bit for bit."""
    x, mu = inputs.plummer(30000, inputs.BASE_SEED + 114)
    act = _subsets(x, 6)["central"] | _subsets(x, 7)["sparse"]
    p = g.FMM_PREC_FP64 if prec == "fp64" else g.FMM_PREC_MIXED
    ctx = g.Context(p=10, mac=g.FMM_MAC_THETA, theta_crit=0.55, leaf_size=32, p2p_c=1.0, precision=p)
    psi, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    psi_a, acc_a, st = ctx.fmm_evaluate_active(_dev(x), _dev(mu), _dev(act.astype(np.uint8)), stats=True)
    a, aa = acc.cpu().numpy(), acc_a.cpu().numpy()
    assert np.array_equal(aa[act], a[act]) and np.array_equal(psi_a.cpu().numpy()[act], psi.cpu().numpy()[act])
    ctx.close()


def test_mixed_subset_accuracy(g):
    """Mixed mode, central subset of a Plummer sphere: accuracy against the FP64 direct sum."""
    import torch
    n = 200000
    x, mu = inputs.plummer(n, inputs.BASE_SEED + 115)
    act = np.linalg.norm(x, axis=1) < 0.3
    ctx = g.Context(p=12, eps=2e-7, leaf_size=48, p2p_c=1.0, precision=g.FMM_PREC_MIXED)
    xt, mt = _dev(x), _dev(mu)
    _, acc_full, st_full = ctx.fmm_evaluate(xt, mt, stats=True)
    _, acc, st = ctx.fmm_evaluate_active(xt, mt, _dev(act.astype(np.uint8)), stats=True)
    idx = np.flatnonzero(act)[::max(1, int(act.sum()) // 2000)]
    _, a_t = ctx.fmm_direct(xt, mt, 1.0, sinks=torch.from_numpy(idx).to("cuda:0"))
    e = _rel(acc.cpu().numpy()[idx], a_t.cpu().numpy())
    ef = _rel(acc_full.cpu().numpy()[idx], a_t.cpu().numpy())
    assert np.sqrt(np.mean(e ** 2)) < 2e-7 and np.sqrt(np.mean(e ** 2)) < 1.5 * np.sqrt(np.mean(ef ** 2)) + 1e-8
    assert st["n_p2p"] < 0.5 * st_full["n_p2p"]
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reused_tree_unchanged_positions_equals_fresh(g, prec):
    import torch
    x, mu = inputs.plummer(20000, inputs.BASE_SEED + 116)
    p = g.FMM_PREC_FP64 if prec == "fp64" else g.FMM_PREC_MIXED
    ctx = g.Context(p=8, eps=1e-7, leaf_size=32, p2p_c=2.0, precision=p)
    xt, mt = _dev(x), _dev(mu)
    psi, acc = ctx.fmm_evaluate(xt, mt)
    ones = torch.ones(20000, dtype=torch.uint8, device="cuda:0")
    psi_r, acc_r = ctx.fmm_evaluate_active(xt, mt, ones, reuse_tree=True)
    assert torch.equal(psi, psi_r) and torch.equal(acc, acc_r)
    ctx.close()


@pytest.mark.parametrize("which", ["all", "central"])
def test_fp64_reused_tree_matches_oracle(g, orc, which):
    """FP64 mode after a drift of the particles: the re-cycled tree against the oracle's."""
    import torch
    x, mu = inputs.plummer(6000, inputs.BASE_SEED + 117)
    rng = np.random.default_rng(9)
    x1 = x + rng.normal(size=x.shape) * 0.02
    act = np.ones(6000, bool) if which == "all" else np.linalg.norm(x1, axis=1) < 0.7
    kw = dict(p=6, eps=1e-7, leaf_size=16, p2p_c=1.0)
    ctx = g.Context(precision=g.FMM_PREC_FP64, **kw)
    ctx.fmm_evaluate(_dev(x), _dev(mu))
    psi, acc, st = ctx.fmm_evaluate_active(_dev(x1), _dev(mu), _dev(act.astype(np.uint8)), reuse_tree=True,
                                           stats=True)
    run = orc.fmm_reused(x, mu, x1, mu, active=act, **kw)
    assert st["n_m2l"] == run.stats["n_m2l"] and st["n_p2p"] == run.stats["n_p2p"]
    acc = acc.cpu().numpy()
    assert np.max(_rel(acc[act], run.acc[act])) <= PARITY_TOL
    ctx.close()


def test_reuse_needs_a_previous_single_system(g):
    import torch
    x, mu = inputs.plummer(3000, inputs.BASE_SEED + 118)
    ones = torch.ones(3000, dtype=torch.uint8, device="cuda:0")
    ctx = g.Context()
    with pytest.raises(g.FMMError):  # nothing evaluated yet
        ctx.fmm_evaluate_active(_dev(x), _dev(mu), ones, reuse_tree=True)
    ctx.fmm_evaluate(_dev(x[:2000]), _dev(mu[:2000]))
    with pytest.raises(g.FMMError):  # another n
        ctx.fmm_evaluate_active(_dev(x), _dev(mu), ones, reuse_tree=True)
    ctx.fmm_evaluate_batch(np.array([0, 1500, 3000]), _dev(x), _dev(mu), np.ones(2))
    with pytest.raises(g.FMMError):  # the last evaluation was a forest
        ctx.fmm_evaluate_active(_dev(x), _dev(mu), ones, reuse_tree=True)
    ctx.fmm_evaluate(_dev(x), _dev(mu))
    ctx.fmm_evaluate_active(_dev(x), _dev(mu), ones, reuse_tree=True)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_individual_eps(g, orc, prec):
    """Sec. 7, opening: eps_b = eps is the global run bit for bit; a tighter eps_b for the inner
    particles matches the oracle (FP64) and lowers their errors (mixed)."""
    import torch
    x, mu = inputs.plummer(8000, inputs.BASE_SEED + 119)
    p = g.FMM_PREC_FP64 if prec == "fp64" else g.FMM_PREC_MIXED
    kw = dict(p=6, eps=1e-5, leaf_size=16, p2p_c=1.0)
    ctx = g.Context(precision=p, **kw)
    xt, mt = _dev(x), _dev(mu)
    _, acc = ctx.fmm_evaluate(xt, mt)
    _, acc_same = ctx.fmm_evaluate_active(xt, mt, eps_b=torch.full((8000,), 1e-5, dtype=torch.float64, device="cuda:0"))
    assert torch.equal(acc, acc_same)
    inner = np.linalg.norm(x, axis=1) < 0.5
    eb = np.where(inner, 1e-8, 1e-5)
    _, acc_t, st = ctx.fmm_evaluate_active(xt, mt, eps_b=_dev(eb), stats=True)
    run = orc.fmm(x, mu, eps_b=eb, **kw)
    if prec == "fp64":
        assert st["n_m2l"] == run.stats["n_m2l"] and st["n_p2p"] == run.stats["n_p2p"]
        assert np.max(_rel(acc_t.cpu().numpy(), run.acc)) <= PARITY_TOL
    _, a_t, _, _ = orc.direct(x, mu)
    e0, e1 = _rel(acc.cpu().numpy(), a_t), _rel(acc_t.cpu().numpy(), a_t)
    assert np.sqrt(np.mean(e1[inner] ** 2)) < 0.2 * np.sqrt(np.mean(e0[inner] ** 2))
    with pytest.raises(g.FMMError):
        ctx.fmm_evaluate_active(xt, mt, eps_b=torch.zeros(8000, dtype=torch.float64, device="cuda:0"))
    ctx.close()


def _frob_rel(T, R):
    return np.linalg.norm(T - R, axis=1) / np.linalg.norm(R, axis=1)


@pytest.mark.parametrize("sub", [False, True])
def test_fp64_tidal_matches_oracle(g, orc, sub):
    """Sec. 7.4 in FP64 mode: the tidal tensor against the oracle's FMM tidal tensor."""
    x, mu = inputs.plummer(6000, inputs.BASE_SEED + 120)
    act = (np.linalg.norm(x, axis=1) < 0.8) if sub else np.ones(6000, bool)
    kw = dict(p=7, eps=1e-7, leaf_size=16, p2p_c=1.0)
    ctx = g.Context(precision=g.FMM_PREC_FP64, **kw)
    psi, acc, T = ctx.fmm_evaluate_active(_dev(x), _dev(mu), _dev(act.astype(np.uint8)), G=1.5, tidal=True)
    run = orc.fmm(x, mu, G=1.5, active=act, tidal=True, **kw)
    T = T.cpu().numpy()
    assert np.max(_frob_rel(T[act], run.tidal[act])) <= PARITY_TOL
    assert np.isnan(T[~act]).all()
    ctx.close()


def test_mixed_tidal_accuracy(g, orc):
    """Mixed mode: the tidal tensor against the direct Hessian; trace-free to rounding."""
    x, mu = inputs.plummer(20000, inputs.BASE_SEED + 121)
    ctx = g.Context(p=10, eps=1e-7, leaf_size=32, p2p_c=1.0, precision=g.FMM_PREC_MIXED)
    _, acc, T = ctx.fmm_evaluate_active(_dev(x), _dev(mu), tidal=True)
    sinks = np.arange(0, 20000, 13)
    Td = orc.direct_tidal(x, mu, sinks=sinks)
    T = T.cpu().numpy()
    e = _frob_rel(T[sinks], Td)
    assert np.sqrt(np.mean(e ** 2)) < 1e-5 and np.percentile(e, 99) < 1e-4
    tr = np.abs(T[:, 0] + T[:, 3] + T[:, 5]) / np.linalg.norm(T, axis=1)
    assert np.percentile(tr, 99) < 1e-4
    ctx.close()


@pytest.mark.parametrize("prec,rot", [("fp64", 1), ("mixed", 1), ("mixed", 0)])
def test_adaptive_order_matches_oracle(g, orc, prec, rot):
    """Sec. 7, opening, on the GPU: the same lists and per-pair orders as the oracle; FP64
    mode to 1e-10, the mixed kernels (rotated: grouped by order; direct: per-pair truncation)
    to the FP32 level against the oracle's FP64 run on those lists."""
    x, mu = inputs.plummer(8000, inputs.BASE_SEED + 122)
    kw = dict(p=11, eps=3e-7, leaf_size=24, p2p_c=1.0)
    p = g.FMM_PREC_FP64 if prec == "fp64" else g.FMM_PREC_MIXED
    ctx = g.Context(precision=p, m2l_rot=rot, adaptive_p=1, **kw)
    _, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    d = ctx.fmm_debug_dump()
    q = ctx.fmm_debug_m2l_orders()
    run = orc.fmm(x, mu, adaptive_p=True, **kw)
    # cells are numbered differently on the two sides: identify them by (first, count, level)
    idg = [tuple(r) for r in d["cells_int"][:, [2, 3, 0]]]
    ido = [tuple(r) for r in run.cells_int[:, [2, 3, 0]]]
    key_g = sorted((idg[a_], idg[b_], int(q_)) for a_, b_, q_ in zip(d["m2l"][:, 0], d["m2l"][:, 1], q))
    key_o = sorted((ido[a_], ido[b_], int(q_)) for a_, b_, q_ in zip(run.m2l[:, 0], run.m2l[:, 1], run.m2l_q))
    assert key_g == key_o
    acc = acc.cpu().numpy()
    e = _rel(acc, run.acc)
    if prec == "fp64":
        assert e.max() <= PARITY_TOL
    else:
        assert np.sqrt(np.mean(e ** 2)) < 1e-7 and e.max() < 2e-6
    ctx.close()
