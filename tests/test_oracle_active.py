"""Pins of the force evaluation for a subset of the particles (Sec. 7.1) in the oracle."""
import numpy as np

from paper_1405_2255_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_all_active_is_the_full_evaluation(orc):
    x, mu = inputs.plummer(2500, 301)
    full = orc.fmm(x, mu, p=6, eps=1e-6, leaf_size=24)
    sub = orc.fmm(x, mu, p=6, eps=1e-6, leaf_size=24, active=np.ones(2500, bool))
    assert np.array_equal(full.acc, sub.acc) and np.array_equal(full.psi, sub.psi)
    assert np.array_equal(full.m2l, sub.m2l) and np.array_equal(full.p2p, sub.p2p)


def test_geometric_mac_subset_equals_full(orc):
    """With the geometric criterion the decisions do not depend on the sinks' scale, so the
    active particles get exactly the interactions, in the same order, as in the full run."""
    x, mu = inputs.plummer(3000, 302)
    act = np.linalg.norm(x, axis=1) < 0.6
    kw = dict(p=5, mac=orc.MAC_THETA, theta_crit=0.5, leaf_size=16, p2p_c=0.0)
    full = orc.fmm(x, mu, **kw)
    sub = orc.fmm(x, mu, active=act, **kw)
    assert np.array_equal(sub.acc[act], full.acc[act]) and np.array_equal(sub.psi[act], full.psi[act])
    assert np.isnan(sub.acc[~act]).all() and np.isnan(sub.psi[~act]).all()
    # every interaction of the subset run has a sink holding an active particle, and the
    # subset run keeps exactly the full run's interactions of those sinks
    ci = sub.cells_int
    sorted_act = act[sub.perm]
    nact = np.array([sorted_act[f:f + c].sum() for f, c in zip(ci[:, 2], ci[:, 3])])
    for lst_s, lst_f in ((sub.m2l, full.m2l), (sub.p2p, full.p2p)):
        assert (nact[lst_s[:, 1]] > 0).all()
        keep = nact[lst_f[:, 1]] > 0
        assert np.array_equal(lst_s, lst_f[keep])


def test_subset_accuracy_and_work(orc):
    """The criterion on the active sinks' own scale keeps their errors at the level of the
    full run, with far fewer interactions when the subset is a central sphere."""
    x, mu = inputs.plummer(4000, 303)
    act = np.linalg.norm(x, axis=1) < 0.4
    full = orc.fmm(x, mu, p=6, eps=1e-6, leaf_size=24)
    sub = orc.fmm(x, mu, p=6, eps=1e-6, leaf_size=24, active=act)
    _, a_t, _, _ = orc.direct(x, mu)
    e_sub, e_full = _rel(sub.acc[act], a_t[act]), _rel(full.acc[act], a_t[act])
    assert np.sqrt(np.mean(e_sub ** 2)) < 2 * np.sqrt(np.mean(e_full ** 2)) + 1e-8
    assert np.sqrt(np.mean(e_sub ** 2)) < 1e-6
    assert sub.stats["n_p2p"] < full.stats["n_p2p"] and sub.stats["n_m2l"] < full.stats["n_m2l"]


def test_reused_tree_with_unchanged_positions_is_the_fresh_run(orc):
    x, mu = inputs.plummer(2500, 304)
    fresh = orc.fmm(x, mu, p=6, eps=1e-6, leaf_size=24)
    reuse = orc.fmm_reused(x, mu, x, mu, p=6, eps=1e-6, leaf_size=24)
    assert np.array_equal(fresh.acc, reuse.acc) and np.array_equal(fresh.m2l, reuse.m2l)
    assert np.array_equal(fresh.cells_dbl, reuse.cells_dbl)


def test_reused_tree_after_a_drift(orc):
    """After the particles moved, the re-cycled tree keeps its cells and centres but its
    radii enclose the new positions exactly, and the forces keep the fresh tree's accuracy."""
    x, mu = inputs.plummer(3000, 305)
    rng = np.random.default_rng(3)
    x1 = x + rng.normal(size=x.shape) * 0.02
    reuse = orc.fmm_reused(x, mu, x1, mu, p=6, eps=1e-6, leaf_size=24)
    fresh = orc.fmm(x1, mu, p=6, eps=1e-6, leaf_size=24)
    xs = x1[reuse.perm]
    for (lev, leaf, f, c, nch), (sx, sy, sz, rho, m, _) in zip(reuse.cells_int, reuse.cells_dbl):
        d = np.linalg.norm(xs[f:f + c] - np.array([sx, sy, sz]), axis=1)
        assert d.max() == rho
        assert np.isclose(m, mu[reuse.perm][f:f + c].sum(), rtol=1e-14)
    _, a_t, _, _ = orc.direct(x1, mu)
    e_r, e_f = _rel(reuse.acc, a_t), _rel(fresh.acc, a_t)
    assert np.sqrt(np.mean(e_r ** 2)) < 2 * np.sqrt(np.mean(e_f ** 2))


def test_individual_eps(orc):
    """Sec. 7, opening: eps_b = eps everywhere is the global run; tightening eps_b for a group of
    particles lowers their errors and keeps the rest as it was."""
    x, mu = inputs.plummer(3000, 306)
    kw = dict(p=5, eps=1e-5, leaf_size=24)
    ref = orc.fmm(x, mu, **kw)
    same = orc.fmm(x, mu, eps_b=np.full(3000, 1e-5), **kw)
    assert np.array_equal(ref.acc, same.acc)
    inner = np.linalg.norm(x, axis=1) < 0.5
    eb = np.where(inner, 1e-8, 1e-5)
    tight = orc.fmm(x, mu, eps_b=eb, **kw)
    _, a_t, _, _ = orc.direct(x, mu)
    e_ref, e_t = _rel(ref.acc, a_t), _rel(tight.acc, a_t)
    assert np.sqrt(np.mean(e_t[inner] ** 2)) < 0.1 * np.sqrt(np.mean(e_ref[inner] ** 2))
    assert tight.stats["n_p2p"] + tight.stats["n_m2l"] > ref.stats["n_p2p"] + ref.stats["n_m2l"]


def test_adaptive_order(orc):
    """Sec. 7, opening: the adaptive walk keeps the lists and gives every accepted pair the
    lowest order in [3, p] that passes; its forces keep the accuracy of the criterion."""
    x, mu = inputs.plummer(4000, 307)
    kw = dict(p=10, eps=3e-7, leaf_size=24, p2p_c=1.0)
    fix = orc.fmm(x, mu, **kw)
    ada = orc.fmm(x, mu, adaptive_p=True, **kw)
    assert np.array_equal(fix.m2l, ada.m2l) and np.array_equal(fix.p2p, ada.p2p)
    assert (fix.m2l_q == 10).all()
    assert ada.m2l_q.min() >= 3 and ada.m2l_q.max() <= 10 and (ada.m2l_q < 10).any()
    _, a_t, _, _ = orc.direct(x, mu)
    e_f, e_a = _rel(fix.acc, a_t), _rel(ada.acc, a_t)
    assert np.sqrt(np.mean(e_a ** 2)) < 2 * np.sqrt(np.mean(e_f ** 2))
    # the geometric criterion has no order to adapt
    geo = orc.fmm(x, mu, p=8, mac=orc.MAC_THETA, theta_crit=0.5, leaf_size=24, adaptive_p=True)
    assert (geo.m2l_q == 8).all()
