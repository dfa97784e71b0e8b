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
