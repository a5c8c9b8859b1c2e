"""Pins of the tidal tensor T = grad grad Psi (Sec. 7.4) in the oracle: the direct sum against
finite differences of the direct accelerations and the trace of a harmonic field; the FMM's
T from Psi_2^m (reading: T_xy = +Im Psi_2^2 / 2) against the direct sum as theta -> 0."""
import numpy as np

from paper_1405_2255_gb300 import inputs


def _T3(t):
    xx, xy, xz, yy, yz, zz = t
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def test_direct_tidal_is_the_gradient_of_the_acceleration(orc):
    x, mu = inputs.plummer(1500, 401)
    sinks = np.array([3, 400, 1200])
    T = orc.direct_tidal(x, mu, G=2.0, sinks=sinks)
    h = 1e-5
    for s, t in zip(sinks, T):
        xs, ms = np.delete(x, s, 0), np.delete(mu, s)
        H = np.zeros((3, 3))
        for u in range(3):
            e = np.zeros(3)
            e[u] = h
            ap = orc.direct(np.vstack([xs, x[s] + e]), np.append(ms, 0.0), G=2.0, sinks=np.array([len(ms)]))[1][0]
            am = orc.direct(np.vstack([xs, x[s] - e]), np.append(ms, 0.0), G=2.0, sinks=np.array([len(ms)]))[1][0]
            H[u] = (ap - am) / (2 * h)
        assert np.max(np.abs(_T3(t) - H)) <= 1e-6 * np.max(np.abs(H))


def test_direct_tidal_is_trace_free(orc):
    x, mu = inputs.plummer(1000, 402)
    T = orc.direct_tidal(x, mu)
    assert np.max(np.abs(T[:, 0] + T[:, 3] + T[:, 5])) <= 1e-12 * np.max(np.abs(T))


def test_fmm_tidal_converges_to_the_direct_sum(orc):
    x, mu = inputs.plummer(2000, 403)
    Td = orc.direct_tidal(x, mu)
    errs = []
    for th in (0.4, 0.2, 0.05):
        r = orc.fmm(x, mu, p=8, mac=orc.MAC_THETA, theta_crit=th, leaf_size=16, p2p_c=0.0, tidal=True)
        e = np.linalg.norm(r.tidal - Td, axis=1) / np.linalg.norm(Td, axis=1)
        errs.append(np.sqrt(np.mean(e ** 2)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9 and errs[1] < 1e-5
    # trace free up to the truncation
    assert np.max(np.abs(r.tidal[:, 0] + r.tidal[:, 3] + r.tidal[:, 5])) <= 1e-9 * np.max(np.abs(Td))
