"""Oracle restatement of the outer-region propagation with the long-range
multipole potential (Section "Overview", Eq. radial with U != 0: the coupled
radial functions are propagated from the inner-region boundary r0 = a to the
asymptotic radius r1, where they are matched to the asymptotic functions;
namelist variable ipert).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings (the paper prints the equation garbled and does not give U):
  * In Rydberg units the coupled equations are
        u_i'' + (eps_i + 2z/r - l_i(l_i+1)/r^2) u_i = sum_j U_ij(r) u_j,
        U_ij(r) = sum_{lambda=1..lambda_max} A^lambda_ij / r^(lambda+1),
    with symmetric A^lambda given by the caller (any factor of the
    Rydberg/Hartree conversion absorbed into A, as the amplitudes w absorb
    theirs).
  * The R-matrix at a defines the solution matrix Psi (n x n) by
    Psi(a) = R(a), a Psi'(a) - b Psi(a) = 1; Psi is propagated to r1 and
        R(r1) = Psi(r1) [r1 Psi'(r1) - b Psi(r1)]^{-1},
    which is symmetric (U symmetric). The paper integrates with Numerov's
    method; here the integration restarts from R at sector boundaries (the
    result does not depend on the basis of solutions Psi carries), which keeps
    strongly closed channels from swamping the others. K follows from Eq. match at r = r1 with
    the channel functions (U = 0) at r1; the tail of U beyond r1 (ipert 3, 4)
    is not included.
  * The propagation here is scipy's DOP853 at rtol 1e-13 on the first-order
    system (Psi, Psi'); the GPU integrates the same equation by RK4 with a
    fixed number of steps. (At rtol 1e-12 R over 20 a0 carries ~1e-10 of
    error, which the matching's condition, up to ~5e4, raises to ~5e-10 in
    K: too close to a 1e-9 comparison.)
"""
import numpy as np
from scipy.integrate import solve_ivp

from . import rmatrix as rm


def coupling(r, A):
    """U(r) = sum_lambda A[lambda-1] / r^(lambda+1)."""
    A = np.asarray(A, dtype=np.float64)
    U = np.zeros(A.shape[1:])
    for lam in range(1, A.shape[0] + 1):
        U += A[lam - 1] / r ** (lam + 1)
    return U


def propagate_r(R_a, a, r1, eps, l, z, A, b=0.0, rtol=1e-13, sector=1.0):
    """R(r1) from R(a) (see the module docstring), sector by sector.

    R(r) = Psi (r Psi' - b Psi)^{-1} does not depend on which basis of the
    solution space Psi holds (Psi -> Psi G for any invertible G), so the
    integration restarts from R at the end of each sector of length
    sector / kappa_max, kappa_max^2 = max_i (l_i(l_i+1)/a^2 - eps_i): within a
    sector no closed channel grows by more than ~e^sector against the others
    and the columns of Psi stay independent (sector=None: one sector)."""
    R_a = np.asarray(R_a, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    if r1 == a:
        return R_a.copy()
    kmax = np.sqrt(max(0.0, float(np.max(l * (l + 1) / (a * a) - eps))))
    if sector is None or kmax * abs(r1 - a) <= sector:
        return _propagate_sector(R_a, a, r1, eps, l, z, A, b, rtol)
    m = int(np.ceil(kmax * abs(r1 - a) / sector))
    edges = a + (r1 - a) * np.arange(m + 1) / m
    edges[-1] = r1
    R = R_a
    for x0, x1 in zip(edges[:-1], edges[1:]):
        R = _propagate_sector(R, x0, x1, eps, l, z, A, b, rtol)
        if R is None:
            return None
    return R


def _propagate_sector(R_a, a, r1, eps, l, z, A, b, rtol):
    """One sector: integrate (Psi, Psi') from a to r1 and form R(r1)."""
    n = R_a.shape[0]

    def rhs(r, y):
        Psi = y[: n * n].reshape(n, n)
        Pp = y[n * n:].reshape(n, n)
        W = np.diag(l * (l + 1) / r ** 2 - 2.0 * z / r - eps) + coupling(r, A)
        return np.concatenate([Pp.ravel(), (W @ Psi).ravel()])

    y0 = np.concatenate([R_a.ravel(), ((np.eye(n) + b * R_a) / a).ravel()])
    sol = solve_ivp(rhs, (a, r1), y0, method="DOP853", rtol=rtol, atol=1e-14 * max(1.0, np.abs(y0).max()))
    if not sol.success:
        return None
    Psi = sol.y[: n * n, -1].reshape(n, n)
    Pp = sol.y[n * n:, -1].reshape(n, n)
    try:
        R1 = np.linalg.solve((r1 * Pp - b * Psi).T, Psi.T).T
    except np.linalg.LinAlgError:
        return None                     # r1 Psi' - b Psi singular: RM_ESINGULAR
    return 0.5 * (R1 + R1.T)


def solve_energy(pw, E, A, r1, mode=rm.MODE_DIRECT, eps_thr=1e-10, fnumin=0.0, margin=0.1, rtol=1e-13):
    """One energy: R at a (Eq. rmatrix), propagated to r1, matched there.
    Returns (status, K, open_idx, omega_row)."""
    nlev = int(pw["n_levels"])
    row = np.zeros(nlev * (nlev + 1) // 2)
    E_k = np.asarray(pw["E_k"], dtype=np.float64)
    if np.any(np.abs(E - E_k) < 1e-12 * max(1.0, abs(E))):
        return rm.RM_ENEAR_POLE, None, None, row
    b = pw.get("b", 0.0)
    cf = rm.channel_functions(E, pw["e_thr"], pw["l"], pw["z"], r1, eps_thr)
    if cf["status"] != rm.RM_OK:
        return cf["status"], None, None, row
    R = rm.r_matrix(E, E_k, pw["W"], pw["a"])
    R1 = propagate_r(R, pw["a"], r1, E - np.asarray(pw["e_thr"], dtype=np.float64), pw["l"], pw["z"], A, b,
                     rtol=rtol)
    if R1 is None:
        return rm.RM_ESINGULAR, None, None, row
    if mode == rm.MODE_MQDT:
        K, _, oi, _ = rm.match_mqdt(R1, cf, pw["l"], pw["z"], r1, b, fnumin=fnumin, margin=margin)
    else:
        K, oi = rm.match_direct(R1, cf, r1, b)
    if K is None:
        return rm.RM_ESINGULAR, None, oi, row
    rm.omega_add(row, rm.t_matrix(K), oi, pw["level"], nlev, pw["g"])
    return rm.RM_OK, K, oi, row


def solve_energies(pw, E, A, r1, mode=rm.MODE_DIRECT, **kw):
    """All energies (same layout as rmatrix.solve_energies)."""
    E = np.asarray(E, dtype=np.float64)
    nlev = int(pw["n_levels"])
    om = np.zeros((E.size, nlev * (nlev + 1) // 2))
    st = np.zeros(E.size, dtype=np.int32)
    no = np.zeros(E.size, dtype=np.int32)
    Ks = []
    e_thr = np.asarray(pw["e_thr"], dtype=np.float64)
    for m, Em in enumerate(E):
        s, K, oi, row = solve_energy(pw, float(Em), A, r1, mode, **kw)
        st[m] = s
        no[m] = int(np.sum(Em - e_thr > 0))
        Ks.append(K)
        om[m] = row
    return dict(status=st, n_open=no, K=Ks, omega=om)
