"""The library's propagation scheme (Numerov from r0 = a to r1; Section
"Overview", namelist mzpts), restated here in numpy and checked against the
oracle's independent DOP853 integration on the CPU. This pins the scheme the
CUDA kernel implements (summed-form Numerov, (1 - T)^-1 to second order,
Runge-Kutta start, O(h^4) derivative at r1, basis renormalisation every
1/kappa_max), apart from the CUDA code itself, which tests/test_gpu_propagate.py
compares with the oracle:
  * fourth-order convergence (error ratio 16 per halving of h);
  * the renormalisation changes R by rounding only, and the scheme stays
    within 1e-9 of the oracle in K where closed channels grow by e^23;
  * the second-order series for (1 - T)^-1 keeps the error within a small
    factor of Numerov with the exact inverse.
"""
import numpy as np

import oracle
from oracle import propagate as pr
from paper_1909_07321_gb300 import synth


def numerov_r(R, a, r1, eps, l, z, A, b, steps, renormalise=True, exact_inverse=False):
    n = R.shape[0]
    h = (r1 - a) / steps
    l = np.asarray(l, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)

    def W(r):
        return np.diag(l * (l + 1) / r ** 2 - 2.0 * z / r - eps) + pr.coupling(r, A)

    def T(r):
        return (h * h / 12.0) * W(r)

    # Psi_1 by four Runge-Kutta steps of h/4
    psi, dps = R.copy(), (np.eye(n) + b * R) / a
    hh = h / 4.0
    for s in range(4):
        r0 = a + s * hh
        k1p, k1q = dps, W(r0) @ psi
        k2p, k2q = dps + hh / 2 * k1q, W(r0 + hh / 2) @ (psi + hh / 2 * k1p)
        k3p, k3q = dps + hh / 2 * k2q, W(r0 + hh / 2) @ (psi + hh / 2 * k2p)
        k4p, k4q = dps + hh * k3q, W(r0 + hh) @ (psi + hh * k3p)
        psi = psi + hh / 6 * (k1p + 2 * k2p + 2 * k3p + k4p)
        dps = dps + hh / 6 * (k1q + 2 * k2q + 2 * k3q + k4q)
    tpp, tp, dl = T(a) @ R, T(a + h) @ psi, psi - R
    k2 = max(0.0, float(np.max(l * (l + 1) / a ** 2 - eps)))
    m = 1.0 / (np.sqrt(k2) * h) if k2 > 0 else steps
    sector = steps if m >= steps else max(1, int(m))
    for k in range(1, steps + 1):
        F = psi + dl + 10 * tp + tpp
        Tk = T(a + (k + 1) * h)
        if exact_inverse:
            tn = Tk @ np.linalg.solve(np.eye(n) - Tk, F)
        else:
            g1 = Tk @ F
            tn = g1 + Tk @ g1
        d = dl + tn + 10 * tp + tpp
        if k == steps:
            dpsi = (d + dl) / (2 * h) - (tn - tpp) / h      # Psi'_N; psi is Psi_N
            break
        dl, psi, tpp, tp = d, psi + d, tp, tn
        if renormalise and k % sector == 0 and k + 1 < steps:
            r = a + (k + 1) * h
            Gi = np.linalg.inv(r * dl / h - b * psi)
            psi, dl, tp, tpp = psi @ Gi, dl @ Gi, tp @ Gi, tpp @ Gi
    R1 = np.linalg.solve((r1 * dpsi - b * psi).T, psi.T).T
    return 0.5 * (R1 + R1.T)


def _case(n=4, seed=5150):
    pw = synth.random_pw(seed, n, 15 * n, z=1.0, a=12.0, e_max=1.5, sigma=0.1, l_max=3)
    pw["e_thr"] = np.linspace(0.0, 1.2, n)
    rng = np.random.default_rng(11)
    A = rng.normal(0.0, 0.3, (2, n, n))
    return pw, 0.5 * (A + A.transpose(0, 2, 1))


def test_fourth_order_convergence():
    pw, A = _case()
    for E in (0.3, 1.0, 1.45):
        eps = E - pw["e_thr"]
        R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
        ref = pr.propagate_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A)
        errs = [np.abs(numerov_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A, 0.0, s) - ref).max()
                / np.abs(ref).max() for s in (100, 200, 400)]
        for e1, e2 in zip(errs, errs[1:]):
            assert 14.0 < e1 / e2 < 18.0, (E, errs)
        assert errs[-1] < 1e-8


def test_renormalisation_is_exact():
    """Renormalising the basis changes R by rounding only (an open case), and
    on the 32-channel multipole workload at its lowest energy (28 closed
    channels growing by up to e^23 over 20 a0) the renormalised scheme keeps
    K within 1e-9 of the oracle."""
    pw, A = _case()
    E = 1.45
    eps = E - pw["e_thr"]
    R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
    r_on = numerov_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A, 0.0, 800)
    r_off = numerov_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A, 0.0, 800, renormalise=False)
    assert np.abs(r_on - r_off).max() <= 1e-12 * np.abs(r_on).max()

    pwm, Am, r1, steps, Em = synth.workload_multipole(1024)
    x = float(Em[3])
    epsm = x - pwm["e_thr"]
    Rm = oracle.r_matrix(x, pwm["E_k"], pwm["W"], pwm["a"])
    cf = oracle.channel_functions(x, pwm["e_thr"], pwm["l"], pwm["z"], r1)
    K_ref, _ = oracle.match_direct(pr.propagate_r(Rm, pwm["a"], r1, epsm, pwm["l"], pwm["z"], Am), cf, r1, 0.0)
    K, _ = oracle.match_direct(numerov_r(Rm, pwm["a"], r1, epsm, pwm["l"], pwm["z"], Am, 0.0, 8000), cf, r1, 0.0)
    assert np.abs(K - K_ref).max() <= 1e-9 * np.abs(K_ref).max()


def test_second_order_inverse_is_enough():
    """T (1 - T)^-1 F taken as T F + T^2 F: the dropped T^3 F is O(h^6) per
    step like Numerov's own local error, so the scheme keeps its fourth order
    and its error stays within a small factor of Numerov with the exact
    inverse (measured 0.6-2.3x on these energies)."""
    pw, A = _case()
    for E in (0.3, 1.0, 1.45):
        eps = E - pw["e_thr"]
        R = oracle.r_matrix(E, pw["E_k"], pw["W"], pw["a"])
        ref = pr.propagate_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A)
        scale = np.abs(ref).max()
        for steps in (400, 800):
            e2 = np.abs(numerov_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A, 0.0, steps) - ref).max()
            ex = np.abs(numerov_r(R, pw["a"], 20.0, eps, pw["l"], pw["z"], A, 0.0, steps,
                                  exact_inverse=True) - ref).max()
            assert e2 < 3.0 * ex and ex < 1e-8 * scale, (E, steps, e2 / scale, ex / scale)
