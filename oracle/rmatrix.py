"""Oracle restatement of the per-energy R -> K -> Omega path.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Notation (Rydberg units, r in a0), Section "Overview":
  channel i: threshold e_i, angular momentum l_i; ion charge z; boundary
  radius a (r_0 in the paper); log-derivative b (Eq. match).
  eps_i = E - e_i; channel open iff eps_i > 0, closed iff eps_i < 0.

A partial wave is passed as a plain dict with keys
  E_k (N,), W (n, N) with W[i, k] = w_ik, a, b, e_thr (n,), l (n,), z,
  level (n,), n_levels, g.
"""
import math

import numpy as np

from . import _clib

# Per-energy status codes (same meaning as the library's).
RM_OK = 0
RM_ETHRESHOLD = 1     # |E - e_i| below eps_thr for some channel
RM_ENEAR_POLE = 2     # |E - E_k| below 1e-12 max(1, |E|) for some pole
RM_ESINGULAR = 3      # matching system singular
RM_ECF_NOCONV = 4     # a continued fraction did not settle

MODE_DIRECT = 0
MODE_MQDT = 1


def tri_index(I, J, n_levels):
    """Position of (I, J), I <= J, in the row-wise upper triangle."""
    return I * n_levels - I * (I - 1) // 2 + (J - I)


def channel_functions(E, e_thr, l, z, a, eps_thr=1e-10):
    """Boundary values at r = a of the asymptotic channel functions.

    Open channel (Section "Glossary", oscillatory asymptotic form): the
    energy-normalised pair s = F/sqrt(k), c = G/sqrt(k) with r-derivatives
    s' = sqrt(k) F', c' = sqrt(k) G' (so that s'c - sc' = 1); rho = k a,
    eta = -z/k (attractive Coulomb potential of Eq. radial).
    Closed channel (exponentially decaying form): theta = W_{nu,l+1/2}(2 kappa r),
    kappa = sqrt(-eps), nu = z/kappa; only the direction of (theta, theta')
    at r = a matters, returned as th = 1/sqrt(1 + (aL)^2), thp = L th with
    L = theta'/theta.
    """
    e_thr = np.asarray(e_thr, dtype=np.float64)
    l = np.asarray(l, dtype=np.int32)
    n = e_thr.size
    eps = E - e_thr
    cf = dict(eps=eps, open=eps > 0, s=np.zeros(n), sp=np.zeros(n), c=np.zeros(n),
              cp=np.zeros(n), th=np.zeros(n), thp=np.zeros(n), L=np.zeros(n),
              nu=np.zeros(n), status=RM_OK)
    if np.any(np.abs(eps) < eps_thr):
        cf["status"] = RM_ETHRESHOLD
        return cf
    op = eps > 0
    if op.any():
        k = np.sqrt(eps[op])
        out, st = _clib.coulomb_open(l[op], -z / k, k * a)
        if st.any():
            cf["status"] = RM_ECF_NOCONV
        sk = np.sqrt(k)
        cf["s"][op] = out[:, 0] / sk
        cf["sp"][op] = out[:, 1] * sk
        cf["c"][op] = out[:, 2] / sk
        cf["cp"][op] = out[:, 3] * sk
    cl = ~op
    if cl.any():
        kap = np.sqrt(-eps[cl])
        nu = z / kap
        y, st = _clib.whittaker_logderiv(l[cl], nu, 2 * kap * a)
        if st.any():
            cf["status"] = RM_ECF_NOCONV
        L = 2 * kap * y
        nrm = 1.0 / np.sqrt(1.0 + (a * L) ** 2)
        cf["L"][cl] = L
        cf["nu"][cl] = nu
        cf["th"][cl] = nrm
        cf["thp"][cl] = L * nrm
    return cf


def r_matrix(E, E_k, W, a):
    """Eq. rmatrix: R_ij = (1/2a) sum_k w_ik w_jk / (E_k - E).
    The upper triangle is computed and mirrored, so R is exactly symmetric."""
    d = 1.0 / (np.asarray(E_k, dtype=np.float64) - E)
    R = (W * d[None, :]) @ W.T / (2.0 * a)
    iu = np.triu_indices(R.shape[0], 1)
    R[(iu[1], iu[0])] = R[iu]
    return R


def _solve(A, B):
    try:
        X = np.linalg.solve(A, B)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(X)):
        return None
    return X


def match_direct(R, cf, a, b=0.0):
    """Eq. match with closed channels eliminated by their decaying boundary
    condition. Unknowns X (n x n_o): psi_ij = s_i delta_ij + ghat_i X_ij with
    ghat = c (open i) or theta (closed i). Matching psi = R (a psi' - b psi)
    at r = a gives
      [diag(ghat) - R diag(a ghat' - b ghat)] X = -[diag(s) - R diag(a s' - b s)] P
    with P selecting the open columns; K = X[open rows]. Returns (K, open
    indices) or (None, open indices) if the system is singular."""
    op = cf["open"]
    oi = np.nonzero(op)[0]
    gh = np.where(op, cf["c"], cf["th"])
    ghp = np.where(op, cf["cp"], cf["thp"])
    A = np.diag(gh) - R * (a * ghp - b * gh)[None, :]
    Bfull = np.diag(cf["s"]) - R * (a * cf["sp"] - b * cf["s"])[None, :]
    B = -Bfull[:, oi]
    if oi.size == 0:
        return np.zeros((0, 0)), oi
    X = _solve(A, B)
    if X is None:
        return None, oi
    return X[oi, :], oi


def sincos_pi(nu):
    """sin(pi nu), cos(pi nu) from the fractional part of nu (exact argument
    reduction: pi*nu itself would carry an absolute rounding error ~ nu 1e-16)."""
    m = np.round(nu)
    f = nu - m
    sgn = np.where(np.mod(m, 2) == 0, 1.0, -1.0)
    return sgn * np.sin(np.pi * f), sgn * np.cos(np.pi * f)


def mqdt_set(cf, l, fnumin=0.0, margin=0.1, sin_min=1e-3, kappa_a_max=5.0, a=None):
    """Closed channels treated by quantum-defect elimination: nu >= max(l +
    margin, fnumin) and |sin(pi nu)| >= sin_min (Section "namelist stgf MQDT
    variables": fnumin; iomsw = 1 omits closed channels with nu < l + 0.1),
    and kappa a <= kappa_a_max: at r = a the regular and irregular closed
    functions differ by exp(2 kappa a), which the elimination loses in
    precision (measured: z = 1, a = 20, nu = 1.1 costs 1e-6 in binary64).
    Every other closed channel keeps its decaying boundary condition."""
    l = np.asarray(l)
    cl = ~cf["open"]
    nu = cf["nu"]
    with np.errstate(invalid="ignore", divide="ignore"):
        q = cl & (nu >= np.maximum(l + margin, fnumin)) & (np.abs(sincos_pi(nu)[0]) >= sin_min)
        if a is not None:
            kap = np.sqrt(np.maximum(-cf["eps"], 0.0))
            q &= kap * a <= kappa_a_max
    return q


def match_mqdt(R, cf, l, z, a, b=0.0, Q=None, fnumin=0.0, margin=0.1, kappa_a_max=5.0):
    """Unphysical K_u and physical K by closed-channel elimination.

    For closed channels in Q the pair (f, g) replaces (s, c): f is the
    energy-analytic regular solution, g is fixed by the decaying solution as
    theta ~ f cos(beta) - g sin(beta), beta = pi nu, with f'g - fg' = 1.
    K_u solves the matching system with open and Q channels as 'open'; then
      K = K_oo - K_oc (K_cc + diag(tan pi nu))^{-1} K_co.
    Returns (K, K_u, open indices, Q indices) or (None, None, ...) when singular."""
    if Q is None:
        Q = mqdt_set(cf, l, fnumin, margin, kappa_a_max=kappa_a_max, a=a)
    op = cf["open"]
    n = op.size
    S = cf["s"].copy()
    Sp = cf["sp"].copy()
    gh = np.where(op, cf["c"], cf["th"])
    ghp = np.where(op, cf["cp"], cf["thp"])
    qi = np.nonzero(Q)[0]
    if qi.size:
        fo, st = _clib.regular_analytic(np.asarray(l)[qi], z, cf["eps"][qi], a)
        f, fp = fo[:, 0], fo[:, 1]
        L = cf["L"][qi]
        sb, cb = sincos_pi(cf["nu"][qi])
        th = sb / (f * L - fp)
        thp = L * th
        g = (f * cb - th) / sb
        gp = (fp * cb - thp) / sb
        S[qi], Sp[qi] = f, fp
        gh[qi], ghp[qi] = g, gp
    P = op | Q
    pi_ = np.nonzero(P)[0]
    oi = np.nonzero(op)[0]
    if pi_.size == 0:
        return np.zeros((0, 0)), np.zeros((0, 0)), oi, qi
    A = np.diag(gh) - R * (a * ghp - b * gh)[None, :]
    Bfull = np.diag(S) - R * (a * Sp - b * S)[None, :]
    X = _solve(A, -Bfull[:, pi_])
    if X is None:
        return None, None, oi, qi
    Ku = X[pi_, :]
    po = op[pi_]            # which P-rows are open
    pc = ~po
    Koo = Ku[np.ix_(po, po)]
    if qi.size == 0:
        return Koo, Ku, oi, qi
    Koc = Ku[np.ix_(po, pc)]
    Kco = Ku[np.ix_(pc, po)]
    Kcc = Ku[np.ix_(pc, pc)]
    sb, cb = sincos_pi(cf["nu"][qi])
    Y = _solve(Kcc + np.diag(sb / cb), Kco)
    if Y is None:
        return None, Ku, oi, qi
    return Koo - Koc @ Y, Ku, oi, qi


def t_matrix(K):
    """Section "Glossary": T = S - 1 with S = (1 + iK)(1 - iK)^{-1}, i.e.
    T = 2iK (1 - iK)^{-1}, by complex LU."""
    n = K.shape[0]
    if n == 0:
        return np.zeros((0, 0), dtype=np.complex128)
    M = np.eye(n) - 1j * K
    return 2j * K @ np.linalg.solve(M, np.eye(n, dtype=np.complex128))


def omega_add(row, T, open_idx, level, n_levels, g):
    """Collision strengths (Section "Glossary"): for target levels I <= J,
    Omega_IJ += g sum_{a in I, b in J} |T_ab|^2 over open channels a, b
    (I = J includes the elastic terms). `row` is the row-wise upper triangle."""
    level = np.asarray(level)
    T2 = np.abs(T) ** 2
    lv = level[open_idx]
    for p in range(lv.size):
        I = int(lv[p])
        for q in range(lv.size):
            J = int(lv[q])
            if I <= J:
                row[tri_index(I, J, n_levels)] += g * T2[p, q]
    return row


def solve_energy(pw, E, mode=MODE_DIRECT, eps_thr=1e-10, fnumin=0.0, margin=0.1):
    """One energy of one partial wave. Returns (status, K, open_idx, omega_row)."""
    nlev = int(pw["n_levels"])
    row = np.zeros(nlev * (nlev + 1) // 2)
    E_k = np.asarray(pw["E_k"], dtype=np.float64)
    if np.any(np.abs(E - E_k) < 1e-12 * max(1.0, abs(E))):
        return RM_ENEAR_POLE, None, None, row
    cf = channel_functions(E, pw["e_thr"], pw["l"], pw["z"], pw["a"], eps_thr)
    if cf["status"] != RM_OK:
        return cf["status"], None, None, row
    R = r_matrix(E, E_k, pw["W"], pw["a"])
    if mode == MODE_MQDT:
        K, _, oi, _ = match_mqdt(R, cf, pw["l"], pw["z"], pw["a"], pw.get("b", 0.0),
                                 fnumin=fnumin, margin=margin)
    else:
        K, oi = match_direct(R, cf, pw["a"], pw.get("b", 0.0))
    if K is None:
        return RM_ESINGULAR, None, oi, row
    T = t_matrix(K)
    omega_add(row, T, oi, pw["level"], nlev, pw["g"])
    return RM_OK, K, oi, row


def solve_energies(pw, E, mode=MODE_DIRECT, **kw):
    """All energies of one partial wave. Returns dict with status (n_E,),
    n_open (n_E,) = number of channels with E > e_i (for every energy, failed
    or not), K (list of arrays or None), omega (n_E, n_tri)."""
    E = np.asarray(E, dtype=np.float64)
    nlev = int(pw["n_levels"])
    om = np.zeros((E.size, nlev * (nlev + 1) // 2))
    st = np.zeros(E.size, dtype=np.int32)
    no = np.zeros(E.size, dtype=np.int32)
    Ks = []
    e_thr = np.asarray(pw["e_thr"], dtype=np.float64)
    for m, Em in enumerate(E):
        s, K, oi, row = solve_energy(pw, float(Em), mode, **kw)
        st[m] = s
        no[m] = int(np.sum(Em - e_thr > 0))
        Ks.append(K)
        om[m] = row
    return dict(status=st, n_open=no, K=Ks, omega=om)
