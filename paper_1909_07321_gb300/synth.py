"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

The paper's workloads (inner-region H.DAT data for Ni3+, Fe I, Ge2+; Section
"Test cases") are not available, so these generators stand in for them with
the shapes the paper describes: up to ~10^3 channels with ~15-35 poles per
channel, thousands of incident energies, grids that cross many thresholds so
that half-open/half-closed energies are common (Section "Computational
details").

Every draw uses numpy.random.Generator(PCG64(seed)) with
seed = 190907321 + workload index, in a fixed order (documented per function),
so the oracle and the GPU path receive bit-identical inputs.

A partial wave is a dict with keys
  E_k (N,) float64  pole energies E_k (Ry), sorted ascending
  W   (n, N) float64 surface amplitudes, W[i, k] = w_ik, row-major
  a, b               boundary radius (a0) and log-derivative (Eq. match)
  e_thr (n,) float64 channel thresholds (Ry); l (n,) int32; z ion charge
  level (n,) int32   target level of each channel; n_levels; g statistical weight
"""
import numpy as np

SEED0 = 190907321


def midpoint_grid(lo, hi, n):
    """E_m = lo + (m + 1/2)(hi - lo)/n, m = 0..n-1 (never exactly on lo)."""
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def jittered_poles(rng, n_poles, lo, hi, jitter=0.1):
    """Poles E_k = lo + (k + 1/2 + u_k) (hi - lo)/N, u_k ~ U(-jitter, jitter), sorted."""
    h = (hi - lo) / n_poles
    u = rng.uniform(-jitter, jitter, n_poles)
    return np.sort(lo + (np.arange(n_poles) + 0.5 + u) * h)


def _pw(E_k, W, a, e_thr, l, z, level, n_levels, g, b=0.0):
    return dict(E_k=np.ascontiguousarray(E_k, dtype=np.float64),
                W=np.ascontiguousarray(W, dtype=np.float64), a=float(a), b=float(b),
                e_thr=np.ascontiguousarray(e_thr, dtype=np.float64),
                l=np.ascontiguousarray(l, dtype=np.int32), z=float(z),
                level=np.ascontiguousarray(level, dtype=np.int32),
                n_levels=int(n_levels), g=float(g))


def workload_small(n_energies=2000):
    """4 channels (thresholds 0, 0.5, 1.0, 1.5 Ry; l = 0, 1, 2, 1; z = 1),
    80 poles on [-1, 40] Ry (+-10% spacing jitter), w ~ N(0, 0.1^2), a = 20,
    energies on a midpoint grid over 0.01-3 Ry. Draw order: jitter, W."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 0))
    E_k = jittered_poles(rng, 80, -1.0, 40.0)
    W = rng.normal(0.0, 0.1, (4, 80))
    pw = _pw(E_k, W, 20.0, [0.0, 0.5, 1.0, 1.5], [0, 1, 2, 1], 1.0, [0, 1, 2, 3], 4, 1.0)
    return [pw], midpoint_grid(0.01, 3.0, n_energies)


def workload_64ch(n_energies=20000):
    """64 channels, thresholds uniform over 0-2 Ry, l ~ U{0..8}, z = 2,
    1920 poles (30 per channel) on [-2, 60] Ry, w ~ N(0, 0.05^2), a = 15,
    energies on a midpoint grid over 0.01-2.5 Ry. Draw order: l, jitter, W."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 1))
    n, N = 64, 1920
    l = rng.integers(0, 9, n)
    E_k = jittered_poles(rng, N, -2.0, 60.0)
    W = rng.normal(0.0, 0.05, (n, N))
    pw = _pw(E_k, W, 15.0, np.linspace(0.0, 2.0, n), l, 2.0, np.arange(n), n, 1.0)
    return [pw], midpoint_grid(0.01, 2.5, n_energies)


def _leveled_channels(rng, n, e_levels):
    """4 channels per target level (distinct l in 0..8 within a level)."""
    n_lev = (n + 3) // 4
    level = np.arange(n) // 4
    l = np.concatenate([rng.choice(9, 4, replace=False) for _ in range(n_lev)])[:n]
    return level, l, np.asarray(e_levels)[level]


def workload_batched(n_pw=40, n_energies=10000, n_min=20, n_max=400):
    """Batched partial waves: n_p ~ U{n_min..n_max} channels, 30 poles per
    channel on [-5, 200] Ry, w ~ N(0, 0.05^2), z = 3, a = 20, 100 target
    levels at linspace(0, 4) Ry with 4 channels per level, g_p = (2J+1)/2 with
    J = p + 1/2; energies on a midpoint grid over 0-5 Ry.
    Draw order per pw: n_p, l, jitter, W."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 2))
    n_levels = (n_max + 3) // 4
    e_levels = np.linspace(0.0, 4.0, n_levels)
    pws = []
    for p in range(n_pw):
        n = int(rng.integers(n_min, n_max + 1))
        level, l, e_thr = _leveled_channels(rng, n, e_levels)
        E_k = jittered_poles(rng, 30 * n, -5.0, 200.0)
        W = rng.normal(0.0, 0.05, (n, 30 * n))
        pws.append(_pw(E_k, W, 20.0, e_thr, l, 3.0, level, n_levels, p + 1.0))
    return pws, midpoint_grid(0.0, 5.0, n_energies)


def workload_1000ch(n_energies=5000, n=1000, n_poles=30000):
    """One partial wave with 1000 channels and 30000 poles over [-5, 200] Ry,
    w ~ N(0, 0.02^2), z = 2, a = 20, 250 levels at linspace(0, 8) Ry with
    4 channels each; energies on a midpoint grid over 0-10 Ry.
    Draw order: l, jitter, W."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 3))
    n_levels = (n + 3) // 4
    level, l, e_thr = _leveled_channels(rng, n, np.linspace(0.0, 8.0, n_levels))
    E_k = jittered_poles(rng, n_poles, -5.0, 200.0)
    W = rng.normal(0.0, 0.02, (n, n_poles))
    return [_pw(E_k, W, 20.0, e_thr, l, 2.0, level, n_levels, 1.0)], \
        midpoint_grid(0.0, 10.0, n_energies)


def random_pw(seed, n, n_poles, z=1.0, a=20.0, e_max=1.5, sigma=0.1, pole_lo=-1.0,
              pole_hi=40.0, l_max=4, b=0.0):
    """Small random partial wave for unit tests (one channel per level)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    l = rng.integers(0, l_max + 1, n)
    e_thr = np.sort(rng.uniform(0.0, e_max, n))
    e_thr[0] = 0.0
    E_k = jittered_poles(rng, n_poles, pole_lo, pole_hi)
    W = rng.normal(0.0, sigma, (n, n_poles))
    return _pw(E_k, W, a, e_thr, l, z, np.arange(n), n, 1.0, b)


def serving_pole_set(set_id, n, base_seed=SEED0 + 4):
    """Pole set `set_id` of the serving pool: n channels (4 per level, levels at
    linspace(0, 6) Ry), N = U{25..35} n poles on [-5, 200] Ry, w ~ N(0, 0.03^2),
    z = 2, a = 20. Draw order: N/n, l, jitter, W."""
    rng = np.random.default_rng(np.random.PCG64(base_seed * 1000 + set_id))
    per = int(rng.integers(25, 36))
    n_lev = (n + 3) // 4
    level, l, e_thr = _leveled_channels(rng, n, np.linspace(0.0, 6.0, n_lev))
    E_k = jittered_poles(rng, per * n, -5.0, 200.0)
    W = rng.normal(0.0, 0.03, (n, per * n))
    return _pw(E_k, W, 20.0, e_thr, l, 2.0, level, n_lev, 1.0)


def serving_requests(n_req, rate_hz, n_range=(50, 1500), ne_range=(256, 8192), n_sets=64,
                     mqdt_fraction=0.5, seed=SEED0 + 4):
    """Poisson stream of requests: arrival times (s), pole-set id from a pool of
    n_sets (each set has a fixed channel count drawn from n_range), an energy
    batch of U{ne_range} midpoint energies on [0, 8] Ry with a random offset,
    and the matching mode (MQDT with probability mqdt_fraction).
    Returns a list of dicts; pole sets are built lazily by serving_pole_set."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    set_n = rng.integers(n_range[0], n_range[1] + 1, n_sets)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_req))
    out = []
    for i in range(n_req):
        sid = int(rng.integers(0, n_sets))
        ne = int(rng.integers(ne_range[0], ne_range[1] + 1))
        lo = float(rng.uniform(0.0, 0.5 * 8.0 / ne))
        E = lo + midpoint_grid(0.0, 8.0, ne)
        out.append(dict(id=i, t_arrival=float(t[i]), set_id=sid, n=int(set_n[sid]), E=E,
                        mode=int(rng.random() < mqdt_fraction)))
    return out


def workload_multipole(n_energies=2048, n=32):
    """Outer-region propagation workload: n = 32 channels, 8 levels at
    linspace(0, 1.4) Ry with 4 channels each, z = 2, a = 15, 30 poles per
    channel on [-2, 60] Ry, w ~ N(0, 0.05^2); long-range coefficients
    (Ry a0^(lambda+1)) A^1 ~ N(0, 0.5^2) between channels of different
    levels (dipole) and A^2 ~ N(0, 0.5^2) between all channels (quadrupole),
    symmetrised; propagation to r1 = 35 a0 in 2000 Numerov steps (the
    paper's default outer grid has 3201 points); energies on a
    midpoint grid over 0.01-2.5 Ry. Draw order: l, jitter, W, A^1, A^2.
    Returns (pw, A [2][n][n], r1, n_steps, E)."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 5))
    n_levels = (n + 3) // 4
    level, l, e_thr = _leveled_channels(rng, n, np.linspace(0.0, 1.4, n_levels))
    E_k = jittered_poles(rng, 30 * n, -2.0, 60.0)
    W = rng.normal(0.0, 0.05, (n, 30 * n))
    A = rng.normal(0.0, 0.5, (2, n, n))
    A = 0.5 * (A + A.transpose(0, 2, 1))
    A[0][level[:, None] == level[None, :]] = 0.0
    pw = _pw(E_k, W, 15.0, e_thr, l, 2.0, level, n_levels, 1.0)
    return pw, np.ascontiguousarray(A), 35.0, 2000, midpoint_grid(0.01, 2.5, n_energies)
