"""Pins of the oracle's outer-region propagation (oracle/propagate.py).

What fixes it independently of its own code:
  * without coupling (A = 0) propagation changes nothing physical: K matched
    at r1 equals K matched at a (open and closed channels), an identity;
  * a free s-wave (z = 0, l = 0) propagates in closed form,
    Psi(r) = Psi(a) cos k(r - a) + Psi'(a) sin k(r - a) / k;
  * with coupling, propagating a -> r1 -> a returns R(a);
  * a plain RK4 written here converges to it at fourth order.
"""
import numpy as np
import pytest

import oracle
from oracle import propagate as pr
from paper_1909_07321_gb300 import synth


def _pw():
    pw = synth.random_pw(5150, 4, 60, z=1.0, a=12.0, e_max=1.5, sigma=0.1, l_max=3)
    pw["e_thr"] = np.array([0.0, 0.4, 0.8, 1.2])
    return pw


def _coupling(n, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, scale, (2, n, n))
    return 0.5 * (A + A.transpose(0, 2, 1))


def test_no_coupling_leaves_k_unchanged():
    pw = _pw()
    E = np.array([0.15, 0.55, 0.95, 1.37, 1.6])
    A0 = np.zeros((1, 4, 4))
    for r1 in (13.0, 16.5):
        res = pr.solve_energies(pw, E, A0, r1)
        ref = oracle.solve_energies(pw, E)
        assert np.array_equal(res["status"], ref["status"])
        for m in range(E.size):
            if ref["status"][m]:
                continue
            np.testing.assert_allclose(res["K"][m], ref["K"][m], rtol=1e-9,
                                       atol=1e-9 * np.abs(ref["K"][m]).max())
            np.testing.assert_allclose(res["omega"][m], ref["omega"][m], rtol=1e-9,
                                       atol=1e-9 * np.abs(ref["omega"][m]).max())


def test_free_s_wave_closed_form():
    a, r1, k, b = 10.0, 17.3, 0.7, 0.0
    for R_a in (0.37, -2.1, 15.0):
        R1 = pr.propagate_r(np.array([[R_a]]), a, r1, [k * k], [0], 0.0, np.zeros((1, 1, 1)), b)
        psi_a, dpsi_a = R_a, 1.0 / a
        x = k * (r1 - a)
        psi = psi_a * np.cos(x) + dpsi_a * np.sin(x) / k
        dpsi = -psi_a * k * np.sin(x) + dpsi_a * np.cos(x)
        assert abs(R1[0, 0] - psi / (r1 * dpsi)) <= 1e-10 * max(1.0, abs(psi / (r1 * dpsi)))


def test_round_trip_with_coupling():
    pw = _pw()
    A = _coupling(4, 3)
    for E in (0.3, 1.0, 1.45):
        eps = E - pw["e_thr"]
        R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
        R1 = pr.propagate_r(R, pw["a"], 15.0, eps, pw["l"], pw["z"], A)
        Rb = pr.propagate_r(R1, 15.0, pw["a"], eps, pw["l"], pw["z"], A)
        np.testing.assert_allclose(Rb, R, rtol=1e-9, atol=1e-9 * np.abs(R).max())
        assert np.abs(R1 - R).max() > 1e-3 * np.abs(R).max()      # it did move


def _rk4(R_a, a, r1, eps, l, z, A, steps):
    n = R_a.shape[0]
    h = (r1 - a) / steps
    Psi, P = R_a.copy(), np.eye(n) / a

    def W(r):
        return np.diag(l * (l + 1) / r ** 2 - 2.0 * z / r - eps) + pr.coupling(r, A)

    r = a
    for _ in range(steps):
        k1p, k1q = P, W(r) @ Psi
        k2p, k2q = P + 0.5 * h * k1q, W(r + 0.5 * h) @ (Psi + 0.5 * h * k1p)
        k3p, k3q = P + 0.5 * h * k2q, W(r + 0.5 * h) @ (Psi + 0.5 * h * k2p)
        k4p, k4q = P + h * k3q, W(r + h) @ (Psi + h * k3p)
        Psi = Psi + h / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        P = P + h / 6.0 * (k1q + 2 * k2q + 2 * k3q + k4q)
        r = a + (_ + 1) * h
    return Psi @ np.linalg.inv(r1 * P)


def test_independent_rk4_converges_to_it():
    pw = _pw()
    A = _coupling(4, 4)
    E = 0.9
    eps = E - pw["e_thr"]
    l = np.asarray(pw["l"], dtype=np.float64)
    R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
    ref = pr.propagate_r(R, pw["a"], 14.0, eps, l, pw["z"], A)
    errs = [np.abs(_rk4(R, pw["a"], 14.0, eps, l, pw["z"], A, s) - ref).max() for s in (50, 100, 200)]
    assert errs[2] < 1e-7 * np.abs(ref).max()
    assert 10.0 < errs[0] / errs[1] < 22.0 and 10.0 < errs[1] / errs[2] < 22.0, errs


def test_sectors_do_not_change_k():
    """R(r1) does not depend on the basis of solutions carried, so restarting
    from R at sector boundaries (any sector length) gives the same K; with
    strongly closed channels (kappa (r1 - a) ~ 10) the sectored results agree
    with each other to ~1e-12."""
    pw = _pw()
    A = _coupling(4, 4)
    E = 0.05                                     # three closed channels
    eps = E - pw["e_thr"]
    R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
    cf = oracle.channel_functions(E, pw["e_thr"], pw["l"], pw["z"], 22.0)
    Ks = []
    for sector in (None, 2.0, 1.0, 0.3):
        R1 = pr.propagate_r(R, pw["a"], 22.0, eps, pw["l"], pw["z"], A, sector=sector)
        K, _ = oracle.match_direct(R1, cf, 22.0, 0.0)
        Ks.append(K)
    for K in Ks[1:]:
        np.testing.assert_allclose(K, Ks[2], rtol=0, atol=1e-11 * np.abs(Ks[2]).max())


def _fit_and_r1(u, du, a, r1, R_a, b):
    """Closed-form single-channel propagation: the solution u = c1 u1 + c2 u2
    through Psi(a) = R_a, a Psi'(a) - b Psi(a) = 1, then R(r1)."""
    psi_a, dpsi_a = R_a, (1.0 + b * R_a) / a
    M = np.array([[u[0](a), u[1](a)], [du[0](a), du[1](a)]])
    c = np.linalg.solve(M, [psi_a, dpsi_a])
    psi = c[0] * u[0](r1) + c[1] * u[1](r1)
    dpsi = c[0] * du[0](r1) + c[1] * du[1](r1)
    return psi / (r1 * dpsi - b * psi)


def test_dipole_tail_bessel_closed_form():
    """One channel, z = 0, l = 0, U = A/r^2 (lambda = 1): u'' = (A/r^2 - k^2) u
    is solved by sqrt(r) J_nu(k r), sqrt(r) Y_nu(k r) with nu^2 = A + 1/4.
    Fixes the power r^-(lambda+1), the sign of U and of eps, and b."""
    sp = pytest.importorskip("scipy.special")
    a, r1, k = 9.0, 16.0, 0.8
    for A1, b, R_a in ((0.7, 0.0, 0.4), (2.5, 0.6, -1.3), (-0.2, -0.4, 3.0)):
        nu = np.sqrt(A1 + 0.25)
        u = (lambda r: np.sqrt(r) * sp.jv(nu, k * r), lambda r: np.sqrt(r) * sp.yv(nu, k * r))
        du = (lambda r: sp.jv(nu, k * r) / (2 * np.sqrt(r)) + np.sqrt(r) * k * sp.jvp(nu, k * r),
              lambda r: sp.yv(nu, k * r) / (2 * np.sqrt(r)) + np.sqrt(r) * k * sp.yvp(nu, k * r))
        exact = _fit_and_r1(u, du, a, r1, R_a, b)
        R1 = pr.propagate_r(np.array([[R_a]]), a, r1, [k * k], [0], 0.0, np.array([[[A1]]]), b)
        assert abs(R1[0, 0] - exact) <= 1e-10 * max(1.0, abs(exact)), (A1, b, R1[0, 0], exact)


def test_quadrupole_tail_zero_energy_closed_form():
    """One channel, z = 0, l = 0, E = threshold, U = A/r^3 (lambda = 2, A > 0):
    u'' = A r^-3 u is solved by sqrt(r) I_1(x), sqrt(r) K_1(x), x = 2 sqrt(A/r)
    (u' = (Z - x Z'(x)) / (2 sqrt r))."""
    sp = pytest.importorskip("scipy.special")
    a, r1 = 6.0, 14.0
    for A2, b, R_a in ((1.5, 0.0, 0.9), (4.0, 0.3, -0.5)):
        def x(r):
            return 2.0 * np.sqrt(A2 / r)
        u = (lambda r: np.sqrt(r) * sp.iv(1, x(r)), lambda r: np.sqrt(r) * sp.kv(1, x(r)))
        du = (lambda r: (sp.iv(1, x(r)) - x(r) * sp.ivp(1, x(r))) / (2 * np.sqrt(r)),
              lambda r: (sp.kv(1, x(r)) - x(r) * sp.kvp(1, x(r))) / (2 * np.sqrt(r)))
        exact = _fit_and_r1(u, du, a, r1, R_a, b)
        A = np.zeros((2, 1, 1))
        A[1, 0, 0] = A2
        R1 = pr.propagate_r(np.array([[R_a]]), a, r1, [0.0], [0], 0.0, A, b)
        assert abs(R1[0, 0] - exact) <= 1e-10 * max(1.0, abs(exact)), (A2, b, R1[0, 0], exact)


_orig_coupling = pr.coupling
_orig_propagate_r = pr.propagate_r


def _coupling_power(r, A):
    A = np.asarray(A, dtype=np.float64)
    return sum(A[lam - 1] / r ** lam for lam in range(1, A.shape[0] + 1))


def _coupling_sign(r, A):
    return -_orig_coupling(r, A)


def _propagate_eps_sign(R_a, a, r1, eps, l, z, A, b=0.0, **kw):
    return _orig_propagate_r(R_a, a, r1, -np.asarray(eps, dtype=np.float64), l, z, A, b, **kw)


def _propagate_b_sign(R_a, a, r1, eps, l, z, A, b=0.0, **kw):
    return _orig_propagate_r(R_a, a, r1, eps, l, z, A, -b, **kw)


@pytest.mark.parametrize("name,fn", [("coupling", _coupling_power), ("coupling", _coupling_sign),
                                     ("propagate_r", _propagate_eps_sign),
                                     ("propagate_r", _propagate_b_sign)],
                         ids=["power", "u_sign", "eps_sign", "b_sign"])
def test_propagation_mutation_is_caught(monkeypatch, name, fn):
    """Each planted mistake fails at least one of the closed-form pins."""
    monkeypatch.setattr(pr, name, fn)
    caught = 0
    for pin in (test_free_s_wave_closed_form, test_dipole_tail_bessel_closed_form,
                test_quadrupole_tail_zero_energy_closed_form):
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught, name
