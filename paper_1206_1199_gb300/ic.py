"""Seeded synthetic particle systems (inputs only; no force arithmetic here).

Both the GPU path and the CPU oracle read these arrays.  Positions are FP64
[n][3], masses FP32 [n] (equal masses), G = 1.  Every generator takes an
integer seed and uses NumPy's PCG64.

The paper measures on synthetic models too: a Plummer sphere and a uniform
sphere of N = 8M (Sections III-D and IV-A), a cold-collapse sphere and a white-dwarf
merger (Section V).  The merger's stars are replaced here by n = 1.5
polytropes (gravity only; no equation-of-state tables are involved).
"""
from __future__ import annotations

import functools
import math

import numpy as np

BASE_SEED = 1206_1199


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng, r):
    """Points at radii r with isotropic random directions."""
    n = r.shape[0]
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth], axis=1)


def _equal_masses(n, total=1.0):
    return np.full(n, total / n, dtype=np.float32)


def plummer(n, seed, a=1.0, rmax=100.0, velocities=False):
    """Plummer sphere, M = 1, scale radius a (Aarseth, Henon & Wielen 1974
    inversion r = a (X^(-2/3) - 1)^(-1/2)); radii beyond rmax * a are redrawn.
    With velocities=True the isotropic distribution function is sampled by
    rejection on q^2 (1 - q^2)^(7/2) (escape-speed fraction q)."""
    rng = _rng(seed)
    r = np.empty(0)
    while r.shape[0] < n:
        x = rng.uniform(0.0, 1.0, 2 * (n - r.shape[0]) + 16)
        x = x[x > 0.0]
        rr = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= rmax * a]])
    r = r[:n]
    pos = _isotropic(rng, r)
    mass = _equal_masses(n)
    if not velocities:
        return pos, mass
    q = np.empty(0)
    while q.shape[0] < n:
        x1 = rng.uniform(0.0, 1.0, 2 * n)
        x2 = rng.uniform(0.0, 0.1, 2 * n)
        keep = x2 < x1 * x1 * (1.0 - x1 * x1) ** 3.5
        q = np.concatenate([q, x1[keep]])
    q = q[:n]
    ve = math.sqrt(2.0) * (1.0 + (r / a) ** 2) ** -0.25 / math.sqrt(a)
    vel = _isotropic(rng, q * ve)
    return pos, mass, vel


def hernquist(n, seed, a=1.0, rt=100.0):
    """Hernquist halo truncated at rt (in units of a), total mass 1 inside rt:
    M(r) / M(rt) = [r / (r + a)]^2 / f with f = (rt / (rt + a))^2, inverted as
    r = a sqrt(X f) / (1 - sqrt(X f))."""
    rng = _rng(seed)
    f = (rt / (rt + a)) ** 2
    x = rng.uniform(0.0, 1.0, n)
    s = np.sqrt(x * f)
    r = a * s / (1.0 - s)
    return _isotropic(rng, r), _equal_masses(n)


def uniform_sphere(n, seed, radius=1.0):
    """Uniform-density sphere, M = 1 (the paper's second distribution)."""
    rng = _rng(seed)
    r = radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    return _isotropic(rng, r), _equal_masses(n)


def _rk4(f, y0, x0, h, stop, max_steps=2_000_000):
    """Fixed-step RK4 from x0 until stop(x, y) is true; returns arrays."""
    xs = [x0]
    ys = [np.array(y0, dtype=np.float64)]
    x, y = x0, ys[0]
    for _ in range(max_steps):
        k1 = f(x, y)
        k2 = f(x + 0.5 * h, y + 0.5 * h * k1)
        k3 = f(x + 0.5 * h, y + 0.5 * h * k2)
        k4 = f(x + h, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        x = x + h
        xs.append(x)
        ys.append(y)
        if stop(x, y):
            break
    return np.array(xs), np.array(ys)


def _sample_radii(rng, n, r_grid, m_grid):
    """Inverse-CDF sampling of radii from a tabulated increasing M(r)."""
    cdf = m_grid / m_grid[-1]
    cdf, idx = np.unique(cdf, return_index=True)
    return np.interp(rng.uniform(0.0, 1.0, n), cdf, r_grid[idx])


@functools.lru_cache(maxsize=4)
def king_profile(w0=6.0, h=1e-3):
    """King (1966) model: dimensionless potential W(r), r in King radii r0,
    from (1/r^2) d/dr (r^2 dW/dr) = -9 rho(W) / rho(W0) with
    rho(W) ~ exp(W) erf(sqrt W) - sqrt(4W/pi) (1 + 2W/3), integrated out to the
    tidal radius W = 0.  Returns (r, M(r)) with arbitrary mass units."""
    def rho(w):
        w = max(w, 0.0)
        return math.exp(w) * math.erf(math.sqrt(w)) - math.sqrt(4.0 * w / math.pi) * (1.0 + 2.0 * w / 3.0)

    rho0 = rho(w0)

    def f(r, y):
        w, dw, m = y
        d = rho(w) / rho0
        return np.array([dw, -9.0 * d - 2.0 * dw / r, r * r * d])

    r0 = 1e-6
    xs, ys = _rk4(f, [w0 - 1.5 * r0 * r0, -3.0 * r0, r0 ** 3 / 3.0], r0, h, lambda x, y: y[0] <= 0.0)
    return xs, ys[:, 2]


def king(n, seed, w0=6.0):
    """King W0 = 6 model, M = 1, positions in King radii (scale radius 1)."""
    rng = _rng(seed)
    r_grid, m_grid = king_profile(w0)
    r = _sample_radii(rng, n, r_grid, m_grid)
    return _isotropic(rng, r), _equal_masses(n)


@functools.lru_cache(maxsize=4)
def lane_emden(n_index=1.5, h=2e-4):
    """Lane-Emden theta'' + (2/xi) theta' = -theta^n to the first zero xi1.
    Returns (xi, mass profile -xi^2 theta')."""
    def f(x, y):
        t, dt = y
        return np.array([dt, -max(t, 0.0) ** n_index - 2.0 * dt / x])

    x0 = 1e-6
    xs, ys = _rk4(f, [1.0 - x0 * x0 / 6.0, -x0 / 3.0], x0, h, lambda x, y: y[0] <= 0.0)
    return xs, -xs * xs * ys[:, 1]


def polytrope(n, seed, mass, radius, n_index=1.5):
    """n = 1.5 polytrope of the given mass and radius, centred at the origin."""
    rng = _rng(seed)
    xi, m = lane_emden(n_index)
    r = _sample_radii(rng, n, xi / xi[-1] * radius, m)
    return _isotropic(rng, r)


def polytrope_pair(n, seed, m1=0.6, m2=0.9, r1=0.012, r2=0.008, sep=0.05, velocities=False):
    """Two n = 1.5 polytropes on a circular orbit (the merger-like test):
    star 1 (m1, r1) and star 2 (m2, r2) separated by sep along x around their
    barycentre, N1 = round(n m1 / (m1 + m2)) equal-mass particles in star 1.
    Stars start cold in their own frames; the relative speed is
    sqrt((m1 + m2) / sep) along y."""
    mt = m1 + m2
    n1 = int(round(n * m1 / mt))
    n2 = n - n1
    p1 = polytrope(n1, seed, m1, r1)
    p2 = polytrope(n2, seed + 1, m2, r2)
    p1[:, 0] -= m2 / mt * sep
    p2[:, 0] += m1 / mt * sep
    pos = np.concatenate([p1, p2])
    mass = _equal_masses(n, mt)
    if not velocities:
        return pos, mass
    v = math.sqrt(mt / sep)
    vel = np.zeros_like(pos)
    vel[:n1, 1] = -m2 / mt * v
    vel[n1:, 1] = m1 / mt * v
    return pos, mass, vel


def batch_systems(n_sys=64, seed=BASE_SEED + 3, log2_min=10, log2_max=18):
    """Independent systems of uneven size: even k Plummer, odd k King W0 = 6,
    N_k = round(2^(log2_min + (log2_max - log2_min) u_k)), u_k ~ U(0, 1),
    eps_k = 4 N_k^(-1/3) (scale radius 1).  Returns a list of (pos, mass, eps)."""
    rng = _rng(seed)
    u = rng.uniform(0.0, 1.0, n_sys)
    out = []
    for k in range(n_sys):
        nk = int(round(2.0 ** (log2_min + (log2_max - log2_min) * u[k])))
        sk = seed + 1000 + k
        pos, mass = plummer(nk, sk) if k % 2 == 0 else king(nk, sk)
        out.append((pos, mass, 4.0 * nk ** (-1.0 / 3.0)))
    return out


def subsample(n, k, seed):
    """k distinct indices of range(n), uniform without replacement, sorted."""
    rng = _rng(seed)
    if k >= n:
        return np.arange(n, dtype=np.int64)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


# The five workloads (sizes and parameters of each configuration).
WORKLOADS = {
    "plummer4k": dict(model="plummer", n=4096, eps=0.01, leaf_size=8, n_crit=64, theta=0.5,
                      use_quad=False, seed=BASE_SEED + 1),
    "plummer1m": dict(model="plummer", n=1 << 20, eps=1e-3, leaf_size=8, n_crit=128,
                      theta=0.5, thetas=(0.3, 0.5, 0.75), use_quad=True, seed=BASE_SEED + 2),
    "hernquist8m": dict(model="hernquist", n=1 << 23, eps=5e-4, leaf_size=8, n_crit=64,
                        theta=0.5, use_quad=True, seed=BASE_SEED + 3),
    "batch64": dict(model="batch", n_sys=64, leaf_size=8, n_crit=64, theta=0.5, use_quad=True,
                    seed=BASE_SEED + 4),
    "merger4m": dict(model="polytrope_pair", n=1 << 22, leaf_size=8, n_crit=64, theta=0.5,
                     use_quad=True, eps=1e-4, seed=BASE_SEED + 5),
}


def sph_radii(pos, mass, n_ngb=64, model="plummer", a=1.0):
    """Neighbour radii for the SPH density stage: h_j encloses about n_ngb
    particles at the model's analytic density, (4 pi / 3) h^3 rho(r_j) / m_j
    = n_ngb, with rho(r) = 3 M / (4 pi a^3) (1 + r^2/a^2)^(-5/2) for a
    Plummer sphere and M a / (2 pi r (r + a)^3) for a Hernquist halo (M = 1).
    FP32, caller order."""
    r = np.linalg.norm(np.asarray(pos, np.float64), axis=1)
    if model == "plummer":
        rho = 3.0 / (4.0 * math.pi * a ** 3) * (1.0 + (r / a) ** 2) ** -2.5
    elif model == "hernquist":
        rr = np.maximum(r, 1e-6 * a)
        rho = a / (2.0 * math.pi * rr * (rr + a) ** 3)
    else:
        raise ValueError(model)
    h = (3.0 * n_ngb * np.asarray(mass, np.float64) / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    return h.astype(np.float32)


def make(model, n, seed, **kw):
    """Positions and masses of a named model."""
    if model == "plummer":
        return plummer(n, seed)
    if model == "hernquist":
        return hernquist(n, seed)
    if model == "king":
        return king(n, seed)
    if model == "uniform":
        return uniform_sphere(n, seed)
    if model == "polytrope_pair":
        return polytrope_pair(n, seed)
    raise ValueError("unknown model %r" % model)
