"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element, on the same seeded inputs.  FP64 mode must match the oracle's FMM to
max |a_gpu - a_orc| / |a_orc| <= 1e-10 (and its tree and interaction lists
exactly); the GPU FP64 direct sum must match the oracle's to 1e-12."""
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


def _cell_ids(ci):
    # identity of a cell: (first, count, level)
    return [tuple(r) for r in ci[:, [2, 3, 0]]]


def _run_both(g, orc, x, mu, G=1.0, **kw):
    prm = dict(p=6, eps=1e-7, mac=0, theta_crit=0.5, leaf_size=16, p2p_c=1.0)
    prm.update(kw)
    ctx = g.Context(precision=g.FMM_PREC_FP64, **{k: v for k, v in prm.items()})
    psi, acc, st = ctx.fmm_evaluate(_dev(x), _dev(mu), G, stats=True)
    dump = ctx.fmm_debug_dump()
    ctx.close()
    run = orc.fmm(x, mu, G=G, **prm)
    return psi.cpu().numpy(), acc.cpu().numpy(), st, dump, run


def _compare_structure(dump, run):
    gi, oi = _cell_ids(dump["cells_int"]), _cell_ids(run.cells_int)
    assert sorted(gi) == sorted(oi), "trees differ"
    # centres and radii per cell
    go = {k: i for i, k in enumerate(gi)}
    idx = np.array([go[k] for k in oi])
    gd, od = dump["cells_dbl"][idx], run.cells_dbl
    scale = np.maximum(od[:, 3], 1e-300)
    assert np.max(np.linalg.norm(gd[:, :3] - od[:, :3], axis=1) / scale) < 1e-12
    assert np.max(np.abs(gd[:, 3] - od[:, 3]) / scale) < 1e-12
    # interaction lists as sets of (source id, sink id)
    def pairs(lst, ids):
        return sorted((ids[a], ids[b]) for a, b in lst)
    assert np.array_equal(dump["perm"], run.perm)
    gm, om = pairs(dump["m2l"], gi), pairs(run.m2l, oi)
    gp, op = pairs(dump["p2p"], gi), pairs(run.p2p, oi)
    flips = len(set(gm) ^ set(om)) + len(set(gp) ^ set(op))
    return flips, len(gm), len(gp)


def test_direct_fp64_matches_oracle(g, orc):
    x, mu = inputs.config_input(1)
    ctx = g.Context()
    psi, acc = ctx.fmm_direct(_dev(x), _dev(mu), 1.0)
    p_o, a_o, f_o, _ = orc.direct(x, mu)
    assert np.max(np.abs(psi.cpu().numpy() - p_o) / p_o) < 1e-12
    assert np.max(_rel(acc.cpu().numpy(), a_o)) < 1e-12
    # sampled sinks with the f scale
    import torch
    sinks = torch.arange(0, len(mu), 37, dtype=torch.int64, device="cuda:0")
    psi, acc, f = ctx.fmm_direct(_dev(x), _dev(mu), 2.0, sinks=sinks, want_f=True)
    s = sinks.cpu().numpy()
    assert np.max(np.abs(f.cpu().numpy() - 2 * f_o[s]) / f_o[s]) < 1e-12
    assert np.max(_rel(acc.cpu().numpy(), 2 * a_o[s])) < 1e-12
    ctx.close()


@pytest.mark.parametrize("case", [
    dict(eps=1e-5), dict(eps=1e-7), dict(mac=2, theta_crit=0.5), dict(mac=1, eps=1e-6),
    dict(eps=1e-6, p=10, leaf_size=32), dict(eps=1e-6, p=3, leaf_size=8, p2p_c=0.0),
])
def test_fmm_fp64_matches_oracle(g, orc, case):
    """Plummer N=4096 (the small configuration): tree, lists and forces vs the oracle."""
    x, mu = inputs.config_input(1)
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, **case)
    flips, nm, npp = _compare_structure(dump, run)
    assert flips == 0
    if case.get("eps", 1) >= 1e-6 or case.get("mac") == 2:
        assert st["n_m2l"] > 0
    assert st["n_m2l"] == run.stats["n_m2l"] and st["n_p2p"] == run.stats["n_p2p"]
    assert st["p2p_interactions"] == run.stats["p2p_interactions"]
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL
    assert np.max(np.abs(psi - run.psi) / run.psi) <= PARITY_TOL


def test_fmm_fp64_matches_oracle_at_benchmark_parameters(g, orc):
    """Plummer N = 2e5 from the benchmark's generator at the benchmark's parameters (p = 14,
    eps = 3e-7, leaf 80, p2p_c 1) in FP64 mode: tree, lists and forces equal the oracle's.
    This reaches the order-14 FP64 M2L, sinks whose lists span many work items and lists
    larger than a fresh context's first capacity."""
    x, mu = inputs.plummer(200000, inputs.BASE_SEED + 2)
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, p=14, eps=3e-7, leaf_size=80, p2p_c=1.0)
    flips, nm, npp = _compare_structure(dump, run)
    assert flips == 0 and nm > 100000 and npp > 100000
    assert st["n_m2l"] == run.stats["n_m2l"] and st["p2p_interactions"] == run.stats["p2p_interactions"]
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL
    assert np.max(np.abs(psi - run.psi) / run.psi) <= PARITY_TOL


@pytest.mark.parametrize("shift,mscale", [(1e5, 1.0), (0.0, 1e-38), (0.0, 1e36), (3e3, 1e-20)])
def test_walk_single_precision_view_extremes(g, orc, shift, mscale):
    """The walk takes its acceptance test in FP32 from a single-precision view of the cells and
    leaves to FP64 every decision within its error margins or outside the FP32 range. Far from
    the origin the two-float centre differences lose their bound for close cells; masses far
    outside the FP32 range put P_0 and eps * minscale out of it. Trees, lists and forces stay
    those of the oracle."""
    x, mu = inputs.config_input(1)
    x = x + shift
    mu = mu * mscale
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, eps=1e-6)
    flips, nm, npp = _compare_structure(dump, run)
    assert flips == 0 and nm > 0 and npp > 0
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL
    assert np.max(np.abs(psi - run.psi) / run.psi) <= PARITY_TOL


@pytest.mark.parametrize("ex,em", [(70, 100), (-60, -90), (0, 0)])
def test_mixed_mode_any_units(g, ex, em):
    """Mixed precision works in units in which the extent and the largest mass are of order
    one (powers of two, exact): a system in other units (here positions x 2^ex and masses
    x 2^em, far outside the FP32 range for |ex|, |em| >= 60) gives Psi x 2^(em - ex) and
    a x 2^(em - 2 ex), bit for bit."""
    x, mu = inputs.plummer(20000, inputs.BASE_SEED + 140)
    ctx = g.Context(p=10, eps=1e-6, leaf_size=32, precision=g.FMM_PREC_MIXED)
    psi0, acc0 = ctx.fmm_evaluate(_dev(x), _dev(mu))
    psi1, acc1 = ctx.fmm_evaluate(_dev(np.ldexp(x, ex)), _dev(np.ldexp(mu, em)))
    p0, a0 = psi0.cpu().numpy(), acc0.cpu().numpy()
    assert np.all(np.isfinite(a0)) and np.all(p0 > 0)
    assert np.array_equal(psi1.cpu().numpy(), np.ldexp(p0, em - ex))
    assert np.array_equal(acc1.cpu().numpy(), np.ldexp(a0, em - 2 * ex))
    ctx.close()


def test_estimate_scale_matches_oracle(g, orc):
    x, mu = inputs.config_input(1)
    for mac in (0, 1):
        _, _, _, dump, run = _run_both(g, orc, x, mu, mac=mac, eps=1e-6)
        assert np.max(np.abs(dump["scale"] - run.scale) / run.scale) < 1e-10


@pytest.mark.parametrize("n,leaf", [(1, 16), (2, 16), (17, 16), (100, 1), (3001, 16), (5000, 64)])
def test_sizes_and_ragged_tails(g, orc, n, leaf):
    x, mu = inputs.plummer(n, 101 + n)
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, G=0.7, leaf_size=leaf, eps=1e-6)
    flips, _, _ = _compare_structure(dump, run)
    assert flips == 0
    if n == 1:
        assert psi[0] == 0 and np.all(acc == 0)
        return
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL


def test_large_leaves_match_oracle(g, orc):
    """Leaves above 128 particles take the enclosing-ball recursion without move-to-front
    (and partly from global memory): tree, centres and forces still match the oracle."""
    x, mu = inputs.plummer(3000, inputs.BASE_SEED + 80)
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, p=6, eps=1e-6, leaf_size=200)
    ci = dump["cells_int"]
    assert ci[ci[:, 1] == 1, 3].max() > 128  # some leaf holds more than 128 particles
    flips, _, _ = _compare_structure(dump, run)
    assert flips == 0
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL


def test_empty_input(g):
    import torch
    ctx = g.Context()
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda:0")
    psi, acc = ctx.fmm_evaluate(e, torch.zeros(0, dtype=torch.float64, device="cuda:0"))
    assert psi.numel() == 0
    ctx.close()


def test_cusp_with_point_mass(g, orc):
    x, mu = inputs.dehnen(6000, inputs.BASE_SEED + 3)
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, p=8, eps=1e-6, leaf_size=16)
    flips, _, _ = _compare_structure(dump, run)
    assert flips == 0
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL


def test_coincident_particles(g, orc):
    x, mu = inputs.plummer(500, 7)
    x[10] = x[11]
    x[20] = x[21] = x[22]
    psi, acc, st, dump, run = _run_both(g, orc, x, mu, leaf_size=4, eps=1e-6)
    assert st["coincident"] == run.stats["coincident"] == 2 + 6
    assert np.all(np.isfinite(acc))
    assert np.max(_rel(acc, run.acc)) <= PARITY_TOL


def test_invalid_input_is_rejected(g):
    x, mu = inputs.plummer(100, 3)
    ctx = g.Context()
    bad = x.copy()
    bad[5, 1] = np.nan
    with pytest.raises(g.FMMError) as e:
        ctx.fmm_evaluate(_dev(bad), _dev(mu))
    assert e.value.code == g.FMM_E_INVALID
    m2 = mu.copy()
    m2[3] = -1
    with pytest.raises(g.FMMError):
        ctx.fmm_evaluate(_dev(x), _dev(m2))
    # the context stays usable
    psi, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    assert np.all(np.isfinite(acc.cpu().numpy()))
    ctx.close()


def test_mixed_precision_accuracy(g, orc):
    """Mixed mode (FP32 compensated P2P): accuracy against FP64 direct summation."""
    x, mu = inputs.config_input(1)
    _, a_t, _, _ = orc.direct(x, mu)
    ctx = g.Context(p=6, eps=1e-7, leaf_size=32, p2p_c=4.0, precision=g.FMM_PREC_MIXED)
    psi, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    e = _rel(acc.cpu().numpy(), a_t)
    assert np.sqrt(np.mean(e ** 2)) < 1e-7
    ctx.close()


@pytest.mark.parametrize("shift", [0.0, 3e4])
def test_mixed_p2p_dx_forms(g, orc, shift):
    """The mixed P2P's forms of dx (p2p_two_float): two-float for near source cells and
    leaf-centre offsets for the far ones (1, default), offsets for all (2), two-float for all
    (3).  Against FP64 direct summation 1 and 3 meet the accuracy target, also far from the
    origin, and 1 stays within FP32 rounding of 3; 2 loses accuracy on close pairs (their
    offsets from the leaf centre are rounded relative to the leaf's size, not to their
    distance) and is only bounded."""
    x, mu = inputs.plummer(20000, inputs.BASE_SEED + 150)
    x = x + shift
    sinks = np.arange(0, 20000, 5)
    _, a_t, _, _ = orc.direct(x, mu, sinks=sinks)
    out, rms = {}, {}
    for mode in (1, 2, 3):
        ctx = g.Context(p=10, eps=1e-7, leaf_size=48, p2p_c=1.0, precision=g.FMM_PREC_MIXED, p2p_two_float=mode)
        _, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
        out[mode] = acc.cpu().numpy()
        e = _rel(out[mode][sinks], a_t)
        rms[mode] = np.sqrt(np.mean(e ** 2))
        assert rms[mode] < (1e-7 if mode != 2 else 3e-7), (mode, rms)
        assert np.all(np.isfinite(out[mode]))
        ctx.close()
    # the split's extra rounding (far dx good to a few 2^-24, like the pair's rsqrt.approx)
    # adds in quadrature to the FMM's own error
    assert rms[1] <= 1.1 * rms[3] + 5e-9, rms
    d = _rel(out[1], out[3])
    assert np.sqrt(np.mean(d ** 2)) < 5e-8 and d.max() < 2e-6, (np.sqrt(np.mean(d ** 2)), d.max())


def test_host_entry_matches_device_entry(g):
    x, mu = inputs.plummer(3000, 9)
    ctx = g.Context(p=5, eps=1e-6, precision=g.FMM_PREC_FP64)
    psi_d, acc_d = ctx.fmm_evaluate(_dev(x), _dev(mu), 1.3)
    psi_h, acc_h = ctx.fmm_evaluate_host(x, mu, 1.3)
    assert np.array_equal(psi_h, psi_d.cpu().numpy())
    assert np.array_equal(acc_h, acc_d.cpu().numpy())
    ctx.close()


def _ensemble_with_gaps(nsys, seed):
    systems = inputs.ensemble(nsys, seed)
    # an empty system and a one-particle system among them
    systems.insert(1, (np.zeros((0, 3)), np.zeros(0)))
    x1, m1 = inputs.plummer(1, seed + 17)
    systems.insert(3, (x1, m1))
    return systems


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_alone(g, prec):
    """The ensemble is evaluated as one forest; every system's result is bit for bit
    the one it gets alone (same tree, same lists in the same order, same kernels)."""
    systems = _ensemble_with_gaps(6, inputs.BASE_SEED + 4)
    xs = np.concatenate([s[0] for s in systems])
    ms = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    Gs = 0.5 + np.arange(len(systems))
    p = g.FMM_PREC_FP64 if prec == "fp64" else g.FMM_PREC_MIXED
    ctx = g.Context(p=6, eps=1e-6, leaf_size=32, p2p_c=2.0, precision=p)
    psi, acc, st = ctx.fmm_evaluate_batch(off, _dev(xs), _dev(ms), Gs, stats=True)
    psi, acc = psi.cpu().numpy(), acc.cpu().numpy()
    n_m2l = n_p2p = inter = 0
    for i, (x, mu) in enumerate(systems):
        if len(mu) == 0:
            continue
        p1, a1, s1 = ctx.fmm_evaluate(_dev(x), _dev(mu), Gs[i], stats=True)
        assert np.array_equal(acc[off[i]:off[i + 1]], a1.cpu().numpy()), i
        assert np.array_equal(psi[off[i]:off[i + 1]], p1.cpu().numpy()), i
        n_m2l += s1["n_m2l"]
        n_p2p += s1["n_p2p"]
        inter += s1["p2p_interactions"]
    assert (st["n_m2l"], st["n_p2p"], st["p2p_interactions"]) == (n_m2l, n_p2p, inter)
    assert st["n"] == len(ms)
    ctx.close()


def test_batch_identical_systems_are_not_coincident(g):
    """Two copies of one system in an ensemble: equal positions in different systems
    are no coincident pairs, and both copies get the same forces."""
    x, mu = inputs.plummer(3000, 99)
    off = np.array([0, 3000, 6000])
    ctx = g.Context(p=5, eps=1e-6, precision=g.FMM_PREC_FP64)
    psi, acc, st = ctx.fmm_evaluate_batch(off, _dev(np.concatenate([x, x])), _dev(np.concatenate([mu, mu])), 1.0,
                                          stats=True)
    acc = acc.cpu().numpy()
    assert st["coincident"] == 0
    assert np.array_equal(acc[:3000], acc[3000:])
    ctx.close()


def test_batch_matches_oracle(g, orc):
    """Each system of a small FP64 ensemble against the oracle run on it alone."""
    systems = _ensemble_with_gaps(3, inputs.BASE_SEED + 40)
    systems = [(x[:2500], mu[:2500]) for x, mu in systems]
    xs = np.concatenate([s[0] for s in systems])
    ms = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    prm = dict(p=6, eps=1e-6, leaf_size=16, p2p_c=1.0)
    ctx = g.Context(precision=g.FMM_PREC_FP64, **prm)
    psi, acc = ctx.fmm_evaluate_batch(off, _dev(xs), _dev(ms), 1.0)
    acc = acc.cpu().numpy()
    for i, (x, mu) in enumerate(systems):
        if len(mu) < 2:
            continue
        run = orc.fmm(x, mu, **prm)
        assert np.max(_rel(acc[off[i]:off[i + 1]], run.acc)) <= PARITY_TOL
    ctx.close()


def test_batch_rejects_bad_offsets(g):
    x, mu = inputs.plummer(100, 3)
    ctx = g.Context()
    for off in ([1, 50, 100], [0, 60, 50, 100]):
        with pytest.raises(g.FMMError):
            ctx.fmm_evaluate_batch(np.array(off), _dev(x), _dev(mu), 1.0)
    with pytest.raises(g.FMMError):
        ctx.fmm_evaluate_batch(np.array([0, 50, 100]), _dev(x), _dev(mu), np.array([1.0, np.inf]))
    ctx.close()


@pytest.mark.parametrize("split", [0, 1])
def test_mixed_m2l_split_accuracy(g, orc, split):
    """Mixed mode with the precision-split M2L (orders > 2 in FP32) keeps the error of
    the FP64-M2L mixed mode: both against FP64 direct summation."""
    x, mu = inputs.plummer(20000, inputs.BASE_SEED + 21)
    ctx = g.Context(p=10, eps=1e-7, leaf_size=32, p2p_c=2.0, precision=g.FMM_PREC_MIXED, m2l_split=split)
    psi, acc, st = ctx.fmm_evaluate(_dev(x), _dev(mu), stats=True)
    assert st["n_m2l"] > 1000
    sinks = np.arange(0, 20000, 7)
    _, a_t, _, _ = orc.direct(x, mu, sinks=sinks)
    e = _rel(acc.cpu().numpy()[sinks], a_t)
    assert np.sqrt(np.mean(e ** 2)) < 1e-7
    assert np.percentile(e, 99.9) < 2e-6
    ctx.close()


def test_autotune_meets_target(g):
    """The tuner's choice reaches the target rms on its own sample and is the fastest
    of the candidates that did."""
    from paper_1405_2255_gb300 import autotune
    x, mu = inputs.plummer(30000, inputs.BASE_SEED + 61)
    r = autotune.tune(_dev(x), _dev(mu), target_rms=1e-6, ps=(6, 8), leaves=(32, 64), cs=(2.0,), nsinks=1024,
                      eps0=1e-6)
    assert r.best.rms <= 1e-6 and r.best.eps > 0
    ok = [c for c in r.tried if c.rms <= 1e-6]
    assert r.best.ms == min(c.ms for c in ok)
    # the chosen parameters reproduce the accuracy on an independent sample of sinks
    ctx = g.Context(precision=g.FMM_PREC_MIXED, **r.params())
    _, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    sinks = np.arange(5, 30000, 29)
    import torch
    _, a_t = ctx.fmm_direct(_dev(x), _dev(mu), 1.0, sinks=torch.from_numpy(sinks).to("cuda:0"))
    e = _rel(acc.cpu().numpy()[sinks], a_t.cpu().numpy())
    assert np.sqrt(np.mean(e ** 2)) < 1.5e-6
    ctx.close()


@pytest.mark.parametrize("leaf", [1, 3, 8, 20, 40, 80, 200])
def test_mixed_small_leaves(g, orc, leaf):
    """Mixed P2P with every item shape the leaves produce (1..200 sinks: one to eight
    replicas, one to four items of up to 64 sinks, two per lane) against the FP64 direct sum."""
    x, mu = inputs.plummer(3000, inputs.BASE_SEED + 70 + leaf)
    ctx = g.Context(p=8, eps=1e-8, leaf_size=leaf, p2p_c=4.0, precision=g.FMM_PREC_MIXED)
    psi, acc = ctx.fmm_evaluate(_dev(x), _dev(mu))
    _, a_t, _, _ = orc.direct(x, mu)
    e = _rel(acc.cpu().numpy(), a_t)
    assert np.all(np.isfinite(e))
    assert np.sqrt(np.mean(e ** 2)) < 1e-7
    ctx.close()


def test_mixed_long_items_split(g, orc):
    """Leaves whose P2P items are long have their source streams cut into pieces whose FP64
    partial sums are added in piece order.  With p2p_c = 512 nearly every pair is P2P, so every
    leaf of 16 sees about N sources (2 N / R > 8192 pair steps per lane at N = 40000): the
    result matches the FP64 direct sum, and in an ensemble each system equals itself alone bit
    for bit (the split depends on the leaf alone)."""
    systems = [inputs.plummer(40000, inputs.BASE_SEED + 90), inputs.plummer(25000, inputs.BASE_SEED + 91)]
    ctx = g.Context(p=8, eps=1e-8, leaf_size=16, p2p_c=512.0, precision=g.FMM_PREC_MIXED)
    alone = []
    for x, mu in systems:
        psi, acc, st = ctx.fmm_evaluate(_dev(x), _dev(mu), stats=True)
        assert st["p2p_interactions"] > 0.9 * len(mu) * (len(mu) - 1)
        alone.append((psi.cpu().numpy(), acc.cpu().numpy()))
    x, mu = systems[0]
    idx = np.random.default_rng(7).choice(len(mu), 2000, replace=False)
    p_t, a_t, _, _ = orc.direct(x, mu, sinks=idx)
    e = _rel(alone[0][1][idx], a_t)
    assert np.sqrt(np.mean(e ** 2)) < 1e-7
    xs = np.concatenate([s[0] for s in systems])
    ms = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    psi_b, acc_b = ctx.fmm_evaluate_batch(off, _dev(xs), _dev(ms), 1.0)
    psi_b, acc_b = psi_b.cpu().numpy(), acc_b.cpu().numpy()
    for i in range(len(systems)):
        assert np.array_equal(acc_b[off[i]:off[i + 1]], alone[i][1]), i
        assert np.array_equal(psi_b[off[i]:off[i + 1]], alone[i][0]), i
    ctx.close()


def test_small_then_large_on_one_context(g):
    """A context first used on a small system keeps working on a much larger ensemble:
    the walk's list capacities follow the tree (regression: they once stayed at the
    small system's size and the walk gave up growing them)."""
    ctx = g.Context(p=14, eps=3.5e-7, leaf_size=80, p2p_c=4.0)
    x, mu = inputs.plummer(2000, 5)
    ctx.fmm_evaluate(_dev(x), _dev(mu))
    systems = inputs.served_systems(8, inputs.BASE_SEED + 5)
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in systems])])
    xs = np.concatenate([s[0] for s in systems])
    ms = np.concatenate([s[1] for s in systems])
    psi, acc, st = ctx.fmm_evaluate_batch(off, _dev(xs), _dev(ms), 1.0, stats=True)
    assert st["n"] == len(ms) and st["n_m2l"] > 0
    assert np.all(np.isfinite(acc.cpu().numpy()))
    ctx.close()


@pytest.mark.parametrize("p,leaf,n", [(3, 24, 6000), (5, 24, 6000), (8, 24, 6000), (12, 24, 6000), (14, 24, 6000),
                                      (16, 24, 6000), (14, 80, 40000)])
def test_m2l_rot_matches_direct(g, orc, p, leaf, n):
    """The rotation-accelerated M2L (App. A.5: z rotations, swap matrices, eq. A31) gives
    the direct eq. (3b) result up to FP32 rounding: same lists, same FP64 low orders, and
    both against the oracle's FP64 FMM on those lists (p = 14 also at the benchmark's leaf
    size 80)."""
    x, mu = inputs.plummer(n, inputs.BASE_SEED + 80 + p + (leaf if leaf != 24 else 0))
    kw = dict(p=p, mac=g.FMM_MAC_THETA, theta_crit=0.6, leaf_size=leaf, p2p_c=0.0, precision=g.FMM_PREC_MIXED)
    c_rot, c_dir = g.Context(m2l_rot=1, **kw), g.Context(m2l_rot=0, **kw)
    _, a_rot, st = c_rot.fmm_evaluate(_dev(x), _dev(mu), stats=True)
    _, a_dir = c_dir.fmm_evaluate(_dev(x), _dev(mu))
    assert st["n_m2l"] > 5000
    a_rot, a_dir = a_rot.cpu().numpy(), a_dir.cpu().numpy()
    d = _rel(a_rot, a_dir)
    assert np.sqrt(np.mean(d ** 2)) < 1e-7 and d.max() < 2e-6
    run = orc.fmm(x, mu, p=p, mac=orc.MAC_THETA, theta_crit=0.6, leaf_size=leaf, p2p_c=0.0)
    e_rot, e_dir = _rel(a_rot, run.acc), _rel(a_dir, run.acc)
    assert np.sqrt(np.mean(e_rot ** 2)) < 1.5 * np.sqrt(np.mean(e_dir ** 2)) + 2e-8
    assert e_rot.max() < 4e-6
    c_rot.close()
    c_dir.close()


def test_m2l_rot_outside_range_falls_back(g):
    """Orders without a rotation kernel (p > 16) take the direct FP32 M2L: identical results."""
    x, mu = inputs.plummer(4000, inputs.BASE_SEED + 99)
    kw = dict(p=17, mac=g.FMM_MAC_THETA, theta_crit=0.5, leaf_size=16, p2p_c=0.0, precision=g.FMM_PREC_MIXED)
    c1, c0 = g.Context(m2l_rot=1, **kw), g.Context(m2l_rot=0, **kw)
    _, a1 = c1.fmm_evaluate(_dev(x), _dev(mu))
    _, a0 = c0.fmm_evaluate(_dev(x), _dev(mu))
    assert np.array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    c1.close()
    c0.close()


def test_library_swap_matrices_match_oracle_and_paper(g, orc):
    """The swap matrices compiled into the rotation-accelerated M2L (host constants of the
    library) equal the oracle's recurrence for every n <= 16 and the matrix printed in
    App. A.5.1 for n = 4."""
    import os
    want4 = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "swap_b4_x16.txt"))
    assert np.array_equal(16.0 * g.fmm_swap_matrix(4), want4)
    for n in range(17):
        assert np.max(np.abs(g.fmm_swap_matrix(n) - orc.swap_matrix(n))) <= 1e-12 * max(1.0, np.abs(orc.swap_matrix(n)).max())
    with pytest.raises(g.FMMError):
        g.fmm_swap_matrix(17)


def test_swap_probe_paths_agree(g):
    """The tensor-core form of the swap stage (3xTF32 mma.sync on the parity blocks of the swap
    matrices) computes what the FMA-immediate form computes, to FP32 rounding."""
    r = g.fmm_swap_probe(4096, 2)
    assert r["fma_ms"] > 0 and r["mma_ms"] > 0
    assert r["maxdiff"] < 1e-4


def test_walk_lists_grow_after_an_overflow(g, orc):
    """A context whose lists were sized by a tiny system meets a large one: the walk overflows,
    grows the lists and is redone; the result equals a fresh context's."""
    import torch
    xs, ms = inputs.plummer(200, inputs.BASE_SEED + 130)
    x, mu = inputs.plummer(60000, inputs.BASE_SEED + 131)
    kw = dict(p=6, eps=1e-6, leaf_size=8, p2p_c=0.5)
    c1 = g.Context(**kw)
    c1.fmm_evaluate(_dev(xs), _dev(ms))
    _, a1 = c1.fmm_evaluate(_dev(x), _dev(mu))
    c2 = g.Context(**kw)
    _, a2 = c2.fmm_evaluate(_dev(x), _dev(mu))
    assert torch.equal(a1, a2)
    c1.close()
    c2.close()
