"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the multipole method.  It only draws
particles, so that the GPU library, the CPU oracle, the tests and the
benchmark all see the same bits for the same seed.

Models (the paper measures on Plummer spheres only, Sec. 4 and Sec. 6):
  * ``plummer``  -- equal-mass Plummer sphere, G = 1, total mass 1, scale
    radius 1, radii by inverse CDF, truncated at ``rt`` scale radii,
    isotropic directions.  M(r) = r^3 / (1 + r^2)^{3/2}.
  * ``dehnen``   -- Dehnen gamma-model, M(r) = (r / (r + 1))^{3 - gamma},
    truncated at ``rt``, N - 1 equal-mass stars sharing ``1 - m_bh`` of the
    mass plus one point mass ``m_bh`` at the origin.
  * ``kroupa_masses`` -- dN/dm ~ m^-2.3 on [0.1, 100] by inverse CDF,
    normalised to total mass 1, drawn independently of position.

Random numbers: counter-based SplitMix64 (Steele, Lea & Flood 2014): the
i-th draw of stream s under seed k is splitmix64(k + (s * 2^40 + i + 1) *
0x9E3779B97F4A7C15); the top 53 bits give a double in [0, 1).  Being a pure
function of (seed, stream, index), it vectorises and any subset of draws can
be regenerated independently.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 14052255
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(counter: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = counter * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream ``stream`` of seed ``seed``."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        ctr = (np.uint64(stream) << np.uint64(40)) + np.arange(1, n + 1, dtype=np.uint64)
        # seed enters additively before mixing: state_i = seed + i * gamma
        z = _splitmix64(ctr) + base
        z = _splitmix64(z)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _directions(seed: int, n: int, r: np.ndarray) -> np.ndarray:
    cos_t = 2.0 * uniforms(seed, 1, n) - 1.0
    phi = 2.0 * np.pi * uniforms(seed, 2, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    x = np.empty((n, 3), dtype=np.float64)
    x[:, 0] = r * sin_t * np.cos(phi)
    x[:, 1] = r * sin_t * np.sin(phi)
    x[:, 2] = r * cos_t
    return x


def plummer_mass(r, rt=None):
    r = np.asarray(r, dtype=np.float64)
    return r ** 3 / (1.0 + r * r) ** 1.5


def plummer(n: int, seed: int, rt: float = 30.0):
    """Equal-mass truncated Plummer sphere: positions [n,3] and masses [n] (sum 1)."""
    mt = float(plummer_mass(rt))
    u = mt * uniforms(seed, 0, n)
    with np.errstate(divide="ignore"):
        r = np.where(u > 0, 1.0 / np.sqrt(np.maximum(u, 1e-300) ** (-2.0 / 3.0) - 1.0), 0.0)
    x = _directions(seed, n, r)
    mu = np.full(n, 1.0 / n, dtype=np.float64) if n > 0 else np.zeros(0)
    return x, mu


def dehnen_mass(r, gamma=1.5):
    r = np.asarray(r, dtype=np.float64)
    return (r / (r + 1.0)) ** (3.0 - gamma)


def dehnen(n: int, seed: int, gamma: float = 1.5, rt: float = 30.0, m_bh: float = 0.01):
    """Truncated Dehnen gamma-model of n - 1 stars plus a central point mass m_bh."""
    if n < 1:
        return np.zeros((0, 3)), np.zeros(0)
    ns = n - 1
    mt = float(dehnen_mass(rt, gamma))
    u = mt * uniforms(seed, 0, ns)
    w = u ** (1.0 / (3.0 - gamma))
    r = w / (1.0 - w)
    x = np.zeros((n, 3), dtype=np.float64)
    x[1:] = _directions(seed, ns, r)
    mu = np.empty(n, dtype=np.float64)
    mu[0] = m_bh
    mu[1:] = (1.0 - m_bh) / max(ns, 1)
    return x, mu


def kroupa_masses(n: int, seed: int, slope: float = 2.3, mlo: float = 0.1, mhi: float = 100.0):
    """Masses with dN/dm ~ m^-slope on [mlo, mhi], normalised so that they sum to 1."""
    e = slope - 1.0
    a, b = mlo ** (-e), mhi ** (-e)
    u = uniforms(seed, 3, n)
    m = (a + u * (b - a)) ** (-1.0 / e)
    return m / m.sum()


def system_seed(config_seed: int, index: int) -> int:
    return config_seed + 1000 * (index + 1)


def ensemble_sizes(nsys: int, seed: int, lo_exp: float = 3.0, span: float = 2.0):
    u = uniforms(seed, 7, nsys)
    return np.rint(10.0 ** (lo_exp + span * u)).astype(np.int64)


def ensemble(nsys: int = 256, seed: int = BASE_SEED + 4):
    """Batched-ensemble workload: nsys Plummer spheres with N log-uniform in [1e3, 1e5]
    and Kroupa-like masses.  Returns a list of (x, mu)."""
    out = []
    for i, n in enumerate(ensemble_sizes(nsys, seed)):
        s = system_seed(seed, i)
        x, _ = plummer(int(n), s)
        out.append((x, kroupa_masses(int(n), s)))
    return out


def served_systems(nsys: int = 64, seed: int = BASE_SEED + 5):
    """Served-stream workload: half Plummer, half gamma = 1.5 cusps, N log-uniform in [1e4, 2e6]."""
    out = []
    for i, n in enumerate(ensemble_sizes(nsys, seed, 4.0, np.log10(2e6) - 4.0)):
        s = system_seed(seed, i)
        out.append(plummer(int(n), s) if i % 2 == 0 else dehnen(int(n), s))
    return out


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    u = uniforms(seed, 9, n)
    return np.cumsum(-np.log1p(-u) / rate)


def config_input(k: int, n: int | None = None):
    """Inputs of the paper-shaped configurations: 1 -> Plummer 4096, 2 -> Plummer 1e6,
    3 -> Dehnen cusp 1e7 (n overrides the size)."""
    seed = BASE_SEED + k
    if k == 1:
        return plummer(n or 4096, seed)
    if k == 2:
        return plummer(n or 1_000_000, seed)
    if k == 3:
        return dehnen(n or 10_000_000, seed)
    raise ValueError(k)
