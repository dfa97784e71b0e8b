"""Pins of the oracle to things other than itself (CPU only).

Each test checks one oracle function against a closed form, a library
routine evaluated independently (mpmath at 30+ digits, scipy), an invariant
the mathematics fixes, or brute force on a tiny case. A plausible mistake
(dropped term, wrong sign or index, transposed operand) in the oracle makes
at least one of them fail; tests/test_oracle_mutations.py plants such
mistakes and checks exactly that.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import _clib
from paper_1909_07321_gb300 import synth

mp = pytest.importorskip("mpmath")


def _mp_coulomb(l, eta, rho):
    with mp.workdps(40):
        F = mp.coulombf(l, eta, rho)
        G = mp.coulombg(l, eta, rho)
        Fp = mp.diff(lambda r: mp.coulombf(l, eta, r), rho)
        Gp = mp.diff(lambda r: mp.coulombg(l, eta, r), rho)
        return [float(x) for x in (F, Fp, G, Gp)]


# (l, eta, rho) across the workloads: z = 1..3, a = 15..20, eps from 1e-6 to 10 Ry,
# including rho inside the centrifugal barrier (high l, small rho).
OPEN_POINTS = [
    (0, -3000.0, 0.02), (8, -3000.0, 0.02), (0, -300.0, 0.2), (5, -300.0, 0.2),
    (0, -30.0, 2.0), (8, -30.0, 2.0), (2, -9.487, 6.3246), (8, -9.487, 6.3246),
    (0, -3.0, 20.0), (8, -3.0, 20.0), (1, -1.732, 34.641), (8, -0.949, 63.2456),
    (3, -0.632, 47.4342), (8, -20.0, 0.5), (4, -2.0, 1.0), (8, -1.0, 3.0),
    (2, -6.0, 0.05), (7, -0.5, 40.0),
]


@pytest.mark.parametrize("l,eta,rho", OPEN_POINTS)
def test_coulomb_open_vs_mpmath(l, eta, rho):
    out, st = _clib.coulomb_open([l], [eta], [rho])
    assert st[0] == 0
    ref = _mp_coulomb(l, eta, rho)
    amp = math.hypot(ref[0], ref[2])
    ampd = math.hypot(ref[1], ref[3])
    o = out[0]
    err = max(abs(o[0] - ref[0]) / amp, abs(o[2] - ref[2]) / amp,
              abs(o[1] - ref[1]) / ampd, abs(o[3] - ref[3]) / ampd)
    assert err < 1e-13, (o, ref)


def test_coulomb_wronskian():
    rng = np.random.default_rng(7)
    n = 300
    l = rng.integers(0, 9, n)
    k = np.sqrt(10.0 ** rng.uniform(-5, 1, n))
    z = rng.choice([1.0, 2.0, 3.0], n)
    a = rng.uniform(10, 25, n)
    out, st = _clib.coulomb_open(l, -z / k, k * a)
    assert not st.any()
    F, Fp, G, Gp = out.T
    np.testing.assert_allclose(Fp * G - F * Gp, 1.0, rtol=0, atol=1e-13)


def test_coulomb_eta0_riccati_bessel():
    rho = np.linspace(0.3, 40.0, 57)
    o0, _ = _clib.coulomb_open(np.zeros(rho.size, int), np.zeros(rho.size), rho)
    np.testing.assert_allclose(o0[:, 0], np.sin(rho), atol=1e-15)
    np.testing.assert_allclose(o0[:, 1], np.cos(rho), atol=1e-15)
    np.testing.assert_allclose(o0[:, 2], np.cos(rho), atol=1e-15)
    np.testing.assert_allclose(o0[:, 3], -np.sin(rho), atol=1e-15)
    o1, _ = _clib.coulomb_open(np.ones(rho.size, int), np.zeros(rho.size), rho)
    F1 = np.sin(rho) / rho - np.cos(rho)
    G1 = np.cos(rho) / rho + np.sin(rho)
    np.testing.assert_allclose(o1[:, 0], F1, atol=2e-15)
    np.testing.assert_allclose(o1[:, 2], G1, atol=2e-15)
    np.testing.assert_allclose(o1[:, 1], np.cos(rho) / rho - np.sin(rho) / rho**2 + np.sin(rho),
                               atol=2e-15)


CLOSED_POINTS = [  # (l, z, eps, a)
    (0, 1, -1e-6, 20.0), (8, 2, -2.11e-6, 15.0), (5, 2, -3e-3, 15.0), (8, 2, -3e-3, 15.0),
    (8, 1, -3e-3, 20.0), (8, 3, -3e-3, 20.0), (0, 3, -0.05, 20.0), (8, 1, -0.3, 20.0),
    (2, 2, -1.0, 15.0), (5, 3, -3.0, 20.0), (1, 1, -1.5, 20.0), (6, 2, -0.25, 15.0),
    (3, 1, -0.0625, 20.0),
]


@pytest.mark.parametrize("l,z,eps,a", CLOSED_POINTS)
def test_whittaker_vs_mpmath(l, z, eps, a):
    kap = math.sqrt(-eps)
    nu = z / kap
    x = 2 * kap * a
    y, st = _clib.whittaker_logderiv([l], [nu], [x])
    assert st[0] == 0
    # the reference takes the same double-rounded nu and x as the oracle: near
    # threshold L moves by ~1e-13 under a 1-ulp change of nu
    with mp.workdps(40):
        nq = mp.mpf(nu)
        xq = mp.mpf(x)
        w = lambda t: mp.whitw(nq, l + mp.mpf(1) / 2, t)  # noqa: E731
        ref = float(mp.diff(w, xq) / w(xq))
    # compare the direction of (theta, theta') at r = a, which is what K sees
    L = 2 * kap * y[0]
    Lr = 2 * kap * ref
    assert abs(math.atan(a * L) - math.atan(a * Lr)) < 1e-13


@pytest.mark.parametrize("n_,l", [(1, 0), (2, 0), (2, 1), (3, 1), (5, 2), (9, 8), (12, 3)])
def test_whittaker_hydrogenic(n_, l):
    """Integer nu = n > l: W_{n,l+1/2}(x) is proportional to
    exp(-x/2) x^{l+1} L^{(2l+1)}_{n-l-1}(x) (generalised Laguerre)."""
    from scipy.special import eval_genlaguerre
    x = np.linspace(0.5, 60.0, 41)
    m = n_ - l - 1
    al = 2 * l + 1
    Lm = eval_genlaguerre(m, al, x)
    dLm = -eval_genlaguerre(m - 1, al + 1, x) if m > 0 else np.zeros_like(x)
    ref = -0.5 + (l + 1) / x + dLm / Lm
    y, st = _clib.whittaker_logderiv(np.full(x.size, l), np.full(x.size, float(n_)), x)
    assert not st.any()
    # nodes of the polynomial make ref large; compare angles
    np.testing.assert_allclose(np.arctan(y), np.arctan(ref), atol=1e-13)


def test_regular_analytic_gamow_relation():
    """For eps > 0 the energy-normalised s = F/sqrt(k) equals
    [A / (1 - exp(-2 pi z / k))]^{1/2} f with A = prod_{p=1..l} (1 + p^2 eps / z^2)."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        l = int(rng.integers(0, 9))
        z = float(rng.choice([1.0, 2.0, 3.0]))
        eps = float(10 ** rng.uniform(-4, -0.3))
        r = float(rng.uniform(5, 20))
        k = math.sqrt(eps)
        (F, Fp, G, Gp), = _clib.coulomb_open([l], [-z / k], [k * r])[0]
        (f, fp), = _clib.regular_analytic([l], [z], [eps], [r])[0]
        A = np.prod([1 + p * p * eps / z**2 for p in range(1, l + 1)])
        B = math.sqrt(A / (1 - math.exp(-2 * math.pi * z / k)))
        assert abs(F / math.sqrt(k) - B * f) <= 1e-12 * max(1.0, abs(B * f))
        assert abs(Fp * math.sqrt(k) - B * fp) <= 1e-12 * max(1.0, abs(B * fp))


def test_regular_analytic_closed_vs_mpmath():
    """eps < 0: f = N_f (2 kappa)^{-(l+1)} M_{nu,l+1/2}(2 kappa r)."""
    for (l, z, eps, r) in [(0, 1, -0.01, 20.0), (3, 2, -0.3, 15.0), (8, 3, -0.05, 20.0),
                           (2, 2, -1.7, 20.0)]:
        (f, fp), = _clib.regular_analytic([l], [z], [eps], [r])[0]
        with mp.workdps(40):
            kap = mp.sqrt(-mp.mpf(eps))
            nu = z / kap
            Nf = mp.sqrt(2 * mp.pi * z) * (2 * z) ** l / mp.factorial(2 * l + 1)
            c = Nf / (2 * kap) ** (l + 1)
            m = lambda t: c * mp.whitm(nu, l + mp.mpf(1) / 2, 2 * kap * t)  # noqa: E731
            fr = float(m(r))
            fpr = float(mp.diff(m, r))
        assert abs(f - fr) <= 1e-13 * abs(fr)
        assert abs(fp - fpr) <= 1e-13 * abs(fpr)


def test_r_matrix_bruteforce_and_symmetry():
    rng = np.random.default_rng(11)
    n, N, a = 3, 7, 17.0
    E_k = np.sort(rng.uniform(-1, 5, N))
    W = rng.normal(0, 0.3, (n, N))
    E = 1.2345
    R = oracle.r_matrix(E, E_k, W, a)
    assert np.array_equal(R, R.T)
    with mp.workdps(40):
        for i in range(n):
            for j in range(n):
                s = mp.fsum(mp.mpf(W[i, k]) * W[j, k] / (mp.mpf(E_k[k]) - E) for k in range(N))
                ref = float(s / (2 * a))
                assert abs(R[i, j] - ref) <= 1e-14 * max(abs(ref), 1e-3)


def test_r_matrix_single_pole_limit():
    rng = np.random.default_rng(12)
    E_k = np.array([-0.5, 0.7, 2.0])
    W = rng.normal(0, 0.2, (4, 3))
    a = 10.0
    for h in [1e-6, 1e-8]:
        E = 0.7 - h
        R = oracle.r_matrix(E, E_k, W, a)
        lim = np.outer(W[:, 1], W[:, 1]) / (2 * a)
        np.testing.assert_allclose((E_k[1] - E) * R, lim, rtol=0, atol=5 * h)


def _one_channel_K(cf, R, a, b=0.0):
    s, sp, c, cp = cf["s"][0], cf["sp"][0], cf["c"][0], cf["cp"][0]
    r = R[0, 0]
    return -(s - r * (a * sp - b * s)) / (c - r * (a * cp - b * c))


@pytest.mark.parametrize("b", [0.0, 0.37])
def test_k_one_channel_by_hand(b):
    pw = synth.random_pw(5, 1, 30, z=2.0, a=15.0)
    for E in [0.05, 0.8, 2.3]:
        cf = oracle.channel_functions(E, pw["e_thr"], pw["l"], pw["z"], pw["a"])
        R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
        K, oi = oracle.match_direct(R, cf, pw["a"], b)
        ref = _one_channel_K(cf, R, pw["a"], b)
        assert abs(K[0, 0] - ref) <= 1e-13 * max(1.0, abs(ref))


def _square_well_poles(n_basis, a, r_w, V0):
    """Eigen-decomposition of -d^2/dr^2 + V on [0, a], V = -V0 for r < r_w,
    in the basis u_j = sqrt(2/a) sin(alpha_j r), alpha_j = (j - 1/2) pi / a,
    which has u_j'(a) = 0 (no Bloch term). Surface amplitude w_k = sqrt(2) u_k(a)."""
    j = np.arange(1, n_basis + 1)
    al = (j - 0.5) * np.pi / a
    ai, aj = np.meshgrid(al, al, indexing="ij")
    with np.errstate(divide="ignore", invalid="ignore"):
        off = (np.sin((ai - aj) * r_w) / (ai - aj) - np.sin((ai + aj) * r_w) / (ai + aj)) / a
    diag = (r_w - np.sin(2 * al * r_w) / (2 * al)) / a
    O = np.where(np.eye(n_basis, dtype=bool), diag[:, None] * np.ones(n_basis), off)
    H = np.diag(al**2) - V0 * O
    Ek, C = np.linalg.eigh(H)
    u_a = np.sqrt(2 / a) * np.sin(al * a)
    w = math.sqrt(2.0) * (C.T @ u_a)
    return Ek, w


def _square_well_tan_delta(E, r_w, V0):
    k = math.sqrt(E)
    Kin = math.sqrt(E + V0)
    return (k * math.tan(Kin * r_w) - Kin * math.tan(k * r_w)) / \
        (Kin + k * math.tan(k * r_w) * math.tan(Kin * r_w))


def _buttle(E, a, n_basis, v_mean):
    """Completion of the truncated pole sum by the poles a particle in the
    constant potential v_mean would have above n_basis: its exact
    R = tan(qa)/(qa), q^2 = E - v_mean, minus the n_basis-pole expansion
    2 sum_j 1/(((j-1/2)pi)^2 - (qa)^2) (Mittag-Leffler series of tan x / x).
    Exact when the potential fills [0, a]."""
    x = math.sqrt(E - v_mean) * a
    j = np.arange(1, n_basis + 1)
    return math.tan(x) / x - np.sum(2.0 / (((j - 0.5) * np.pi) ** 2 - x**2))


@pytest.mark.parametrize("r_w", [10.0, 6.0])
def test_square_well_tan_delta(r_w):
    """z = 0, l = 0 square well inside r = a: K = tan(delta) from the oracle's
    R-matrix path (finite-basis poles + free-particle completion) against the
    closed form; the error must fall as the basis grows."""
    a, V0 = 10.0, 1.3
    errs = []
    for nb in [100, 400]:
        Ek, w = _square_well_poles(nb, a, r_w, V0)
        errs.append([])
        for E in [0.07, 0.4, 1.1]:
            cf = oracle.channel_functions(E, np.array([0.0]), np.array([0]), 0.0, a)
            R = oracle.r_matrix(E, Ek, w[None, :], a)
            R = R + _buttle(E, a, nb, -V0 * r_w / a)
            K, _ = oracle.match_direct(R, cf, a)
            errs[-1].append(abs(K[0, 0] - _square_well_tan_delta(E, r_w, V0)))
    errs = np.array(errs)
    tol = 1e-10 if r_w == a else 2e-4
    assert errs[-1].max() < tol, errs
    if r_w != a:
        assert np.all(errs[1] < errs[0])


def test_one_open_one_closed_closed_form():
    """R_eff = R_oo + a R_oc^2 L / (1 - a R_cc L), then the one-channel formula."""
    pw = synth.random_pw(21, 2, 40, z=1.0, a=20.0)
    pw["e_thr"] = np.array([0.0, 1.2])
    for E in [0.3, 0.9, 1.15]:
        cf = oracle.channel_functions(E, pw["e_thr"], pw["l"], pw["z"], pw["a"])
        R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
        K, oi = oracle.match_direct(R, cf, pw["a"])
        a = pw["a"]
        L = cf["L"][1]
        Reff = R[0, 0] + a * R[0, 1] ** 2 * L / (1 - a * R[1, 1] * L)
        ref = _one_channel_K(cf, np.array([[Reff]]), a)
        assert abs(K[0, 0] - ref) <= 1e-12 * max(1.0, abs(ref))


def _mixed_pw():
    return synth.random_pw(33, 6, 90, z=2.0, a=15.0, e_max=1.8, l_max=5)


def test_k_symmetric_and_s_unitary():
    pw = _mixed_pw()
    for E in np.linspace(0.05, 2.2, 23):
        st, K, oi, _ = oracle.solve_energy(pw, float(E))
        assert st == oracle.RM_OK
        nK = max(1.0, np.abs(K).max())
        assert np.abs(K - K.T).max() <= 1e-12 * nK
        n = K.shape[0]
        S = (np.eye(n) + 1j * K) @ np.linalg.inv(np.eye(n) - 1j * K)
        assert np.abs(S.conj().T @ S - np.eye(n)).max() < 1e-12
        assert np.abs(S - S.T).max() < 1e-12
        T = oracle.t_matrix(K)
        # optical theorem: sum_b |T_ab|^2 = -2 Re T_aa
        np.testing.assert_allclose((np.abs(T) ** 2).sum(axis=1), -2 * T.real.diagonal(),
                                   atol=1e-12)


def test_k_invariant_under_theta_scaling():
    pw = _mixed_pw()
    E = 0.9
    cf = oracle.channel_functions(E, pw["e_thr"], pw["l"], pw["z"], pw["a"])
    R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
    K, _ = oracle.match_direct(R, cf, pw["a"])
    cl = ~cf["open"]
    cf2 = dict(cf)
    scale = np.where(cl, np.linspace(-3.0, 7.0, cl.size), 1.0)
    cf2["th"] = cf["th"] * scale
    cf2["thp"] = cf["thp"] * scale
    K2, _ = oracle.match_direct(R, cf2, pw["a"])
    np.testing.assert_allclose(K2, K, rtol=0, atol=1e-12 * np.abs(K).max())


def test_mqdt_equals_direct():
    pw = _mixed_pw()
    n_q = 0
    # a coarse grid plus energies just below each threshold (the Rydberg
    # region where closed channels are eliminated by quantum-defect theory)
    below = np.concatenate([t - np.array([0.001, 0.002, 0.005, 0.01, 0.03]) for t in pw["e_thr"][1:]])
    for E in np.concatenate([np.linspace(0.05, 2.2, 31), below]):
        cf = oracle.channel_functions(float(E), pw["e_thr"], pw["l"], pw["z"], pw["a"])
        R = oracle.r_matrix(float(E), pw["E_k"], pw["W"], pw["a"])
        Kd, _ = oracle.match_direct(R, cf, pw["a"])
        Km, Ku, oi, qi = oracle.match_mqdt(R, cf, pw["l"], pw["z"], pw["a"])
        n_q += len(qi)
        np.testing.assert_allclose(Km, Kd, rtol=0, atol=1e-10 * max(1.0, np.abs(Kd).max()))
        assert np.abs(Ku - Ku.T).max() <= 1e-11 * max(1.0, np.abs(Ku).max())
    assert n_q > 20


def test_mqdt_two_channel_vs_mpmath():
    """z = 1, a = 20, E = 0.8 Ry; open channel (l = 1, threshold 0.5), closed
    channel (l = 2, threshold 1.0); fixed R. K from the oracle's direct and
    MQDT routes against a 40-digit mpmath evaluation of the same matching."""
    a, z, E = 20.0, 1.0, 0.8
    R = np.array([[0.013, -0.021], [-0.021, 0.034]])
    e_thr = np.array([0.5, 1.0])
    l = np.array([1, 2])
    cf = oracle.channel_functions(E, e_thr, l, z, a)
    Kd, _ = oracle.match_direct(R, cf, a)
    Km, _, _, qi = oracle.match_mqdt(R, cf, l, z, a, kappa_a_max=10.0)   # kappa a = 8.9 here
    assert len(qi) == 1
    with mp.workdps(40):
        k = mp.sqrt(mp.mpf(E) - mp.mpf("0.5"))
        eta = -z / k
        F = lambda r: mp.coulombf(1, eta, k * r) / mp.sqrt(k)  # noqa: E731
        G = lambda r: mp.coulombg(1, eta, k * r) / mp.sqrt(k)  # noqa: E731
        kap = mp.sqrt(mp.mpf("1.0") - mp.mpf(E))
        nu = z / kap
        th = lambda r: mp.whitw(nu, mp.mpf(5) / 2, 2 * kap * r)  # noqa: E731
        s, sp = F(a), mp.diff(F, a)
        c, cp = G(a), mp.diff(G, a)
        t, tp = th(a), mp.diff(th, a)
        Rm = mp.matrix([[mp.mpf(R[0, 0]), mp.mpf(R[0, 1])], [mp.mpf(R[1, 0]), mp.mpf(R[1, 1])]])
        A = mp.matrix([[c - Rm[0, 0] * a * cp, -Rm[0, 1] * a * tp],
                       [-Rm[1, 0] * a * cp, t - Rm[1, 1] * a * tp]])
        B = mp.matrix([[-(s - Rm[0, 0] * a * sp)], [Rm[1, 0] * a * sp]])
        X = mp.lu_solve(A, B)
        ref = float(X[0])
    assert abs(Kd[0, 0] - ref) <= 1e-12 * abs(ref)
    assert abs(Km[0, 0] - ref) <= 1e-10 * abs(ref)


def test_omega_real_form_and_symmetry():
    """|T|^2 from T = 2iK(1 - iK)^{-1} equals the real form 4(X^2 + Y^2) with
    M = 1 + K^2, X = M^{-1} K, Y = M^{-1} K^2; Omega is built from the upper
    triangle of a symmetric level matrix."""
    pw = _mixed_pw()
    pw["level"] = np.array([0, 0, 1, 1, 2, 2], dtype=np.int32)
    pw["n_levels"] = 3
    pw["e_thr"] = np.repeat(pw["e_thr"][[0, 2, 4]], 2)
    for E in [0.4, 1.3, 2.1]:
        st, K, oi, row = oracle.solve_energy(pw, E)
        n = K.shape[0]
        M = np.eye(n) + K @ K
        X = np.linalg.solve(M, K)
        Y = np.linalg.solve(M, K @ K)
        T2 = 4 * (X**2 + Y**2)
        T = oracle.t_matrix(K)
        np.testing.assert_allclose(np.abs(T) ** 2, T2, atol=1e-13)
        full = np.zeros((3, 3))
        lv = pw["level"][oi]
        for p in range(n):
            for q in range(n):
                full[lv[p], lv[q]] += T2[p, q]
        assert np.allclose(full, full.T, atol=1e-13)
        ref = np.array([full[I, J] for I in range(3) for J in range(I, 3)])
        np.testing.assert_allclose(row, ref, atol=1e-13)


def _level_matrix(row, n_levels):
    """Symmetric level matrix from the row-wise upper triangle: Omega_IJ for
    I <= J and Omega_JI otherwise."""
    full = np.zeros((n_levels, n_levels))
    for I in range(n_levels):
        for J in range(I, n_levels):
            full[I, J] = full[J, I] = row[oracle.tri_index(I, J, n_levels)]
    return full


@pytest.mark.parametrize("seed", [3, 17, 29])
def test_omega_aggregation_from_unitarity(seed):
    """With S unitary and K symmetric, sum_b |T_ab|^2 = -2 Re T_aa (optical
    theorem), so for every target level I the row sum of the symmetric level
    matrix is sum_J Omega_IJ = -2 g sum_{a in I} Re T_aa. This checks
    omega_add's level indexing against an identity of the scattering
    matrix, not against a restatement of the level sum. Channels of a level
    are spread over the open-channel order, and one level has no open
    channel (its row must vanish)."""
    rng = np.random.default_rng(seed)
    n_open, n_levels, g = 9, 5, 2.5
    A = rng.normal(0.0, 1.3, (n_open, n_open))
    K = 0.5 * (A + A.T)
    T = oracle.t_matrix(K)
    level_of_open = rng.permutation(np.array([0, 0, 1, 1, 1, 3, 3, 4, 4]))
    level = np.concatenate([level_of_open, [2, 2]]).astype(np.int32)   # level 2: closed channels only
    open_idx = np.arange(n_open)
    row = oracle.omega_add(np.zeros(n_levels * (n_levels + 1) // 2), T, open_idx, level, n_levels, g)
    full = _level_matrix(row, n_levels)
    for I in range(n_levels):
        ref = -2.0 * g * sum(T[a, a].real for a in range(n_open) if level_of_open[a] == I)
        assert abs(full[I].sum() - ref) <= 1e-12 * max(1.0, abs(ref)), I
    assert np.all(full[2] == 0.0)


def test_omega_two_levels_by_hand():
    """Two channels in two levels, K = [[p, q], [q, r]]: (1 - iK)^{-1} is the
    adjugate over the determinant d = (1 - ip)(1 - ir) + q^2, so
      T_00 = 2i (p (1 - ir) + i q^2) / d,  T_11 = 2i (r (1 - ip) + i q^2) / d,
      T_01 = 2i q / d,
    and Omega = g (|T_00|^2, |T_01|^2, |T_11|^2) in the row-wise upper triangle."""
    p, q, r, g = 0.7, -0.4, 1.9, 1.5
    d = (1 - 1j * p) * (1 - 1j * r) + q * q
    T00 = 2j * (p * (1 - 1j * r) + 1j * q * q) / d
    T11 = 2j * (r * (1 - 1j * p) + 1j * q * q) / d
    T01 = 2j * q / d
    K = np.array([[p, q], [q, r]])
    row = oracle.omega_add(np.zeros(3), oracle.t_matrix(K), np.array([0, 1]), np.array([0, 1]), 2, g)
    np.testing.assert_allclose(row, g * np.abs(np.array([T00, T01, T11])) ** 2, rtol=1e-14)
    # the same two channels with their levels swapped: Omega_01 is unchanged,
    # the elastic entries trade places
    row2 = oracle.omega_add(np.zeros(3), oracle.t_matrix(K), np.array([0, 1]), np.array([1, 0]), 2, g)
    np.testing.assert_allclose(row2, g * np.abs(np.array([T11, T01, T00])) ** 2, rtol=1e-14)


def test_status_codes():
    pw = _mixed_pw()
    st, *_ = oracle.solve_energy(pw, float(pw["e_thr"][2]) + 1e-12)
    assert st == oracle.RM_ETHRESHOLD
    st, *_ = oracle.solve_energy(pw, float(pw["E_k"][40]))
    assert st == oracle.RM_ENEAR_POLE


def _scan_points(seed, n):
    """Random (l, z, eps, a) over the workloads' ranges, log-uniform |eps|."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        l = int(rng.integers(0, 9))
        z = float(rng.choice([1.0, 2.0, 3.0]))
        a = float(rng.choice([15.0, 20.0]))
        mag = float(10 ** rng.uniform(-6, 1))
        out.append((l, z, mag, a))
    return out


@pytest.mark.parametrize("l,z,mag,a", _scan_points(101, 16))
def test_coulomb_open_random_scan(l, z, mag, a):
    k = math.sqrt(mag)
    eta, rho = -z / k, k * a
    out, st = _clib.coulomb_open([l], [eta], [rho])
    assert st[0] == 0
    ref = _mp_coulomb(l, eta, rho)
    amp = math.hypot(ref[0], ref[2])
    ampd = math.hypot(ref[1], ref[3])
    o = out[0]
    err = max(abs(o[0] - ref[0]) / amp, abs(o[2] - ref[2]) / amp,
              abs(o[1] - ref[1]) / ampd, abs(o[3] - ref[3]) / ampd)
    assert err < 1e-13


@pytest.mark.parametrize("l,z,mag,a", _scan_points(202, 16))
def test_whittaker_random_scan(l, z, mag, a):
    test_whittaker_vs_mpmath(l, z, -mag, a)


def test_many_channel_invariants():
    """At 64 channels (the benchmark's partial wave) the oracle's K stays
    symmetric to rounding (every open channel's Wronskian normalisation and
    the closed-channel treatment enter), and MQDT elimination reproduces the
    direct K and Omega (an exact identity) where closed channels are present."""
    from paper_1909_07321_gb300 import synth
    pws, E = synth.workload_64ch(20000)
    pw = pws[0]
    for x in E[[5, 4000, 9000, 13000, 17000, 19990]]:
        st, K, oi, _ = oracle.solve_energy(pw, float(x))
        assert st == oracle.RM_OK
        assert np.abs(K - K.T).max() <= 1e-13 * max(1.0, np.abs(K).max())
    idx = [4000, 9000, 13000]
    d = oracle.solve_energies(pw, E[idx])
    m = oracle.solve_energies(pw, E[idx], mode=oracle.MODE_MQDT)
    for k in range(len(idx)):
        assert d["status"][k] == m["status"][k] == 0
        assert d["n_open"][k] < pw["W"].shape[0]
        np.testing.assert_allclose(m["K"][k], d["K"][k], rtol=0, atol=1e-12 * np.abs(d["K"][k]).max())
        np.testing.assert_allclose(m["omega"][k], d["omega"][k], rtol=0,
                                   atol=1e-12 * np.abs(d["omega"][k]).max())


def _grouped_wave(seed=2027):
    """8 channels in two groups, the even and the odd channels (thresholds
    interleaved), each group coupled only to its own 30 poles."""
    rng = np.random.default_rng(seed)
    n, N = 8, 60
    e_thr = np.linspace(0.0, 1.4, n)
    l = rng.integers(0, 5, n).astype(np.int32)
    E_k = np.sort(rng.uniform(-1.0, 30.0, N))
    pole_group = rng.permutation(np.arange(N) % 2)
    W = rng.normal(0.0, 0.1, (n, N))
    W[(np.arange(n)[:, None] % 2) != pole_group[None, :]] = 0.0
    pw = dict(E_k=E_k, W=W, a=15.0, b=0.0, e_thr=e_thr, l=l, z=2.0,
              level=np.arange(n, dtype=np.int32), n_levels=n, g=1.0)
    return pw, pole_group


def _energies_off_thresholds(e_thr, lo, hi, m):
    E = synth.midpoint_grid(lo, hi, m)
    return E[np.abs(E[:, None] - np.asarray(e_thr)[None, :]).min(axis=1) > 1e-3]


@pytest.mark.parametrize("mode", [oracle.MODE_DIRECT, oracle.MODE_MQDT])
def test_decoupled_channel_groups(mode):
    """Channels that share no poles with another group do not couple to it:
    R is block-diagonal, so K (over the open channels) is block-diagonal and
    each block, and each group's collision strengths, equal those of the
    group solved alone as its own partial wave (its channels and poles). The
    groups interleave in channel order, so an open-position, channel-order or
    level-pair index mixed up anywhere breaks the equality."""
    pw, pole_group = _grouped_wave()
    E = _energies_off_thresholds(pw["e_thr"], 0.05, 1.9, 40)
    full = oracle.solve_energies(pw, E, mode=mode)
    n = pw["W"].shape[0]
    subs = []
    for gidx in (0, 1):
        ch = np.arange(n)[np.arange(n) % 2 == gidx]
        pk = np.nonzero(pole_group == gidx)[0]
        sub = dict(pw, E_k=pw["E_k"][pk], W=pw["W"][np.ix_(ch, pk)], e_thr=pw["e_thr"][ch], l=pw["l"][ch],
                   level=np.arange(ch.size, dtype=np.int32), n_levels=ch.size)
        subs.append((ch, oracle.solve_energies(sub, E, mode=mode)))
    checked = 0
    for m in range(E.size):
        if full["status"][m]:
            continue
        K = full["K"][m]
        oi = np.nonzero(E[m] > pw["e_thr"])[0]
        assert K.shape == (oi.size, oi.size)
        pos = {c: i for i, c in enumerate(oi)}
        for ch, res in subs:
            assert res["status"][m] == 0
            oc = [pos[c] for c in ch if c in pos]
            other = [pos[c] for c in oi if c not in ch]
            if oc:
                np.testing.assert_allclose(K[np.ix_(oc, oc)], res["K"][m], rtol=0,
                                           atol=1e-12 * max(1.0, np.abs(res["K"][m]).max()))
            if oc and other:
                assert np.all(K[np.ix_(oc, other)] == 0.0)
            for I, cI in enumerate(ch):
                for J, cJ in enumerate(ch):
                    if I <= J:
                        a = full["omega"][m][oracle.tri_index(cI, cJ, n)]
                        b = res["omega"][m][oracle.tri_index(I, J, ch.size)]
                        assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), (m, cI, cJ)
        ev, od = np.arange(0, n, 2), np.arange(1, n, 2)
        for cI in ev:
            for cJ in od:
                assert full["omega"][m][oracle.tri_index(min(cI, cJ), max(cI, cJ), n)] == 0.0
        checked += 1
    assert checked > 30


def test_channel_relabelling():
    """Relabelling the channels (thresholds, l, levels and the rows of W
    permuted together) permutes K over the open channels the same way and
    moves each collision strength to the relabelled level pair: nothing in
    the method depends on the order the channels are listed in."""
    pw = synth.random_pw(2029, 7, 140, z=1.0, a=18.0, e_max=1.5, sigma=0.1, l_max=4)
    rng = np.random.default_rng(2030)
    perm = rng.permutation(7)           # new channel i is old channel perm[i]
    inv = np.argsort(perm)
    pp = dict(pw, e_thr=pw["e_thr"][perm], l=pw["l"][perm], W=pw["W"][perm],
              level=inv[pw["level"]][perm].astype(np.int32))
    E = _energies_off_thresholds(pw["e_thr"], 0.05, 1.8, 30)
    a = oracle.solve_energies(pw, E)
    b = oracle.solve_energies(pp, E)
    assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["n_open"], b["n_open"])
    nl = pw["n_levels"]
    checked = 0
    for m in range(E.size):
        if a["status"][m]:
            continue
        oi_a = np.nonzero(E[m] > pw["e_thr"])[0]          # old labels, ascending
        oi_b = np.nonzero(E[m] > pp["e_thr"])[0]          # new labels, ascending
        sel = [int(np.nonzero(oi_a == perm[c])[0][0]) for c in oi_b]
        np.testing.assert_allclose(b["K"][m], a["K"][m][np.ix_(sel, sel)], rtol=0,
                                   atol=1e-12 * max(1.0, np.abs(a["K"][m]).max()))
        for I in range(nl):
            for J in range(I, nl):
                nI, nJ = sorted((int(inv[I]), int(inv[J])))
                x = a["omega"][m][oracle.tri_index(I, J, nl)]
                y = b["omega"][m][oracle.tri_index(nI, nJ, nl)]
                assert abs(x - y) <= 1e-12 * max(1.0, abs(x)), (m, I, J)
        checked += 1
    assert checked > 20
