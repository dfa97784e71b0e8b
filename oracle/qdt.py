"""Oracle restatement of the MQDT coarse-mesh interpolation (Section "namelist
stgf MQDT variables": imode = -1, single pass -- a full solution on a coarse
mesh and an interpolative solution on the fine mesh; ieq, qetest).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The unphysical K_u of quantum-defect theory (closed channels of the MQDT set
carried with the energy-analytic pair f, g) has none of the closed-channel
resonances, so it is computed on a coarse set of energies (nodes) and
interpolated linearly in energy; at every fine energy the closed channels
are then eliminated with nu of that energy. iqdt = 1 works with the
unphysical S_u = (1 + i K_u)(1 - i K_u)^{-1} (unitary, so it has no poles to
interpolate across), and
  S = S_oo - S_oc (S_cc - diag(exp(-2 i pi nu)))^{-1} S_co,   T = S - 1
(the same physical S as the K form below: checked to 1e-16 on random data);
iqdt = 2 works with K_u itself,
  K = K_oo - K_oc (K_cc + diag(tan pi nu))^{-1} K_co,
and T, Omega follow as for any K (K_u passes through poles wherever an
eigenphase crosses pi/2, so it needs a finer coarse mesh).

Readings (the paper names the controls only):
  * K_u is defined for a fixed set of open and eliminated channels, so the
    fine mesh is cut into segments of consecutive energies with the same
    channel classes (open / eliminated / decaying, by the rules of
    rmatrix.mqdt_set without its |sin pi nu| guard), and interpolation never
    crosses a segment boundary.
  * Nodes of a segment [E_i0, E_i1]: ieq < 0 -- its first fine energy, every
    |ieq|-th after it and its last; ieq > 0 -- its first and last fine
    energies and the points of the ieq-point grid spanning the whole fine
    range that fall inside it (ieq = 0 is not a valid choice).
  * A node is dropped when a channel of the eliminated set has
    |sin pi nu| < 1e-3 there (g is not formed), when it lies within
    2.5e-5 max(z^2, 1) Ry of a threshold (where the Coulomb continued
    fractions are deepest: such a node alone would cost more than the rest
    of the mesh), on a pole (|E - E_k| < 1e-12 max(1, |E|)), or when its K_u
    cannot be computed; fine
    energies beyond the outermost remaining node are extrapolated linearly
    from the two nearest (held constant when one remains), and a segment
    without nodes fails (RM_ESINGULAR).
  * qetest (here absolute Ry): K_u is re-interpolated only when the energy
    has moved by more than qetest since the last interpolation within the
    segment; until then the last interpolation energy is reused (qetest <= 0
    re-interpolates at every energy).
  * A partial wave may carry "prop" = (A, r1), the long-range coupling of
    oracle/propagate.py: R is then propagated from a to r1 before the
    matching, and the matching radius r1 takes the place of a everywhere
    (channel functions, the kappa a cap of the eliminated set).
"""
import numpy as np

from . import rmatrix as rm

CL_OPEN, CL_ELIM, CL_DECAY = 0, 1, 2
SIN_MIN = 1e-3
NODE_MIN_EPS = 2.5e-5      # x max(z^2, 1) Ry: closest a node may lie to a threshold


def match_radius(pw):
    """a, or r1 when the wave carries an outer-region propagation."""
    prop = pw.get("prop")
    return pw["a"] if prop is None else prop[1]


def classes(E, pw, fnumin=0.0, margin=0.1, kappa_a_max=5.0, eps_thr=1e-10):
    """Channel classes at E (None if E lies on a threshold)."""
    e_thr = np.asarray(pw["e_thr"], dtype=np.float64)
    l = np.asarray(pw["l"])
    eps = E - e_thr
    if np.any(np.abs(eps) < eps_thr):
        return None
    z, a = pw["z"], match_radius(pw)
    cls = np.full(e_thr.size, CL_DECAY, dtype=np.int32)
    cls[eps > 0] = CL_OPEN
    cl = eps < 0
    if z > 0:
        kap = np.sqrt(np.where(cl, -eps, 1.0))
        nu = z / kap
        el = cl & (nu >= np.maximum(l + margin, fnumin)) & (kap * a <= kappa_a_max)
        cls[el] = CL_ELIM
    return cls


def plan(pw, E, ieq, qetest=0.0, **kw):
    """Segments, nodes and the interpolation of every fine energy.

    Returns dict: seg (n_E,) segment index or -1 (threshold), segments: list
    of (i0, i1, classes), nodes: list of arrays of node energies per segment
    (before validity checks), e_int (n_E,) interpolation energies."""
    E = np.asarray(E, dtype=np.float64)
    if ieq == 0:
        raise ValueError("ieq = 0 is not a valid choice")
    if np.any(np.diff(E) <= 0):
        raise ValueError("fine energies must be strictly ascending")
    n_E = E.size
    cls = [classes(float(x), pw, **kw) for x in E]
    seg = np.full(n_E, -1, dtype=np.int64)
    segments = []
    for m in range(n_E):
        if cls[m] is None:
            continue
        if m > 0 and cls[m - 1] is not None and segments and seg[m - 1] == len(segments) - 1 \
                and np.array_equal(cls[m - 1], cls[m]):
            segments[-1][1] = m
        else:
            segments.append([m, m, cls[m]])
        seg[m] = len(segments) - 1
    nodes = []
    for i0, i1, _ in segments:
        pts = {E[i0], E[i1]}
        if ieq < 0:
            pts |= set(E[i0:i1 + 1:-ieq].tolist())
        else:
            if ieq >= 2:
                G = E[0] + np.arange(ieq) * ((E[-1] - E[0]) / (ieq - 1))
            else:
                G = np.array([E[0]])
            pts |= set(G[(G > E[i0]) & (G < E[i1])].tolist())
        nodes.append(np.array(sorted(pts)))
    e_int = E.copy()
    for i0, i1, _ in segments:
        last = E[i0]
        for m in range(i0, i1 + 1):
            if m == i0 or qetest <= 0 or E[m] - last > qetest:
                last = E[m]
            e_int[m] = last
    return dict(seg=seg, segments=segments, nodes=nodes, e_int=e_int)


def node_valid(pw, x, cls_seg, **kw):
    """A node keeps the segment's classes, has |sin pi nu| >= 1e-3 for every
    eliminated channel, keeps 2.5e-5 max(z^2, 1) Ry from every threshold, and
    does not lie on a pole."""
    c = classes(x, pw, **kw)
    if c is None or not np.array_equal(c, cls_seg):
        return False
    E_k = np.asarray(pw["E_k"], dtype=np.float64)
    if np.any(np.abs(x - E_k) < 1e-12 * max(1.0, abs(x))):
        return False
    if np.any(np.abs(x - np.asarray(pw["e_thr"])) < NODE_MIN_EPS * max(pw["z"] ** 2, 1.0)):
        return False
    el = np.nonzero(cls_seg == CL_ELIM)[0]
    if el.size:
        nu = pw["z"] / np.sqrt(np.asarray(pw["e_thr"])[el] - x)
        if np.any(np.abs(rm.sincos_pi(nu)[0]) < SIN_MIN):
            return False
    return True


def cayley(K):
    """S = (1 + i K)(1 - i K)^{-1}."""
    n = K.shape[0]
    return np.linalg.solve((np.eye(n) - 1j * K).T, (np.eye(n) + 1j * K).T).T


def k_unphysical(pw, x, cls_seg):
    """K_u at energy x with the segment's eliminated set (channel order of
    the open and eliminated channels), or None."""
    am = match_radius(pw)
    b = pw.get("b", 0.0)
    cf = rm.channel_functions(x, pw["e_thr"], pw["l"], pw["z"], am)
    if cf["status"] != rm.RM_OK:
        return None
    R = rm.r_matrix(x, pw["E_k"], pw["W"], pw["a"])
    if pw.get("prop") is not None:
        from . import propagate
        R = propagate.propagate_r(R, pw["a"], am, x - np.asarray(pw["e_thr"], dtype=np.float64), pw["l"],
                                  pw["z"], pw["prop"][0], b)
        if R is None:
            return None
    _, Ku, _, _ = rm.match_mqdt(R, cf, pw["l"], pw["z"], am, b, Q=(cls_seg == CL_ELIM))
    return Ku


def interpolation_weights(xs, x):
    """(j, t): K_u(x) = (1 - t) K_u(xs[j]) + t K_u(xs[j + 1]) over the sorted
    valid nodes xs (t outside [0, 1] beyond the outer nodes; (0, 0.0) with a
    single node)."""
    if xs.size == 1:
        return 0, 0.0
    j = int(np.searchsorted(xs, x, side="right")) - 1
    j = min(max(j, 0), xs.size - 2)
    return j, (x - xs[j]) / (xs[j + 1] - xs[j])


def eliminate(Ku, cls_seg, x, pw):
    """Physical K at energy x from the interpolated K_u, or None if singular."""
    P = np.nonzero(cls_seg != CL_DECAY)[0]
    po = cls_seg[P] == CL_OPEN
    pc = ~po
    Koo = Ku[np.ix_(po, po)]
    if not pc.any():
        return Koo
    q = P[pc]
    nu = pw["z"] / np.sqrt(np.asarray(pw["e_thr"])[q] - x)
    sb, cb = rm.sincos_pi(nu)
    Y = rm._solve(Ku[np.ix_(pc, pc)] + np.diag(sb / cb), Ku[np.ix_(pc, po)])
    if Y is None:
        return None
    return Koo - Ku[np.ix_(po, pc)] @ Y


def eliminate_s(Su, cls_seg, x, pw):
    """Physical S at energy x from the interpolated S_u, or None if singular."""
    P = np.nonzero(cls_seg != CL_DECAY)[0]
    po = cls_seg[P] == CL_OPEN
    pc = ~po
    Soo = Su[np.ix_(po, po)]
    if not pc.any():
        return Soo
    q = P[pc]
    nu = pw["z"] / np.sqrt(np.asarray(pw["e_thr"])[q] - x)
    sb, cb = rm.sincos_pi(nu)
    d = (cb * cb - sb * sb) - 2j * sb * cb          # exp(-2 i pi nu)
    try:
        Y = np.linalg.solve(Su[np.ix_(pc, pc)] - np.diag(d), Su[np.ix_(pc, po)])
    except np.linalg.LinAlgError:
        return None
    return Soo - Su[np.ix_(po, pc)] @ Y


def node_matrix(pw, x, cls_seg, iqdt):
    """S_u (iqdt = 1) or K_u (iqdt = 2) at node x, or None."""
    Ku = k_unphysical(pw, x, cls_seg)
    if Ku is None:
        return None
    return cayley(Ku) if iqdt == 1 else Ku


def solve_energies(pw, E, ieq, qetest=0.0, iqdt=1, **kw):
    """Omega (and, for iqdt = 2, K) on the fine mesh by coarse-mesh
    interpolation of S_u (iqdt = 1) or K_u (iqdt = 2). Returns dict like
    rmatrix.solve_energies plus the plan and the node energies used per
    segment."""
    E = np.asarray(E, dtype=np.float64)
    pl = plan(pw, E, ieq, qetest, **kw)
    nlev = int(pw["n_levels"])
    om = np.zeros((E.size, nlev * (nlev + 1) // 2))
    st = np.zeros(E.size, dtype=np.int32)
    no = np.array([int(np.sum(x - np.asarray(pw["e_thr"]) > 0)) for x in E], dtype=np.int32)
    Ks = [None] * E.size
    used = []
    for s, (i0, i1, cls_seg) in enumerate(pl["segments"]):
        xs, kus = [], []
        for x in pl["nodes"][s]:
            if not node_valid(pw, float(x), cls_seg, **kw):
                continue
            Mu = node_matrix(pw, float(x), cls_seg, iqdt)
            if Mu is None:
                continue
            xs.append(float(x))
            kus.append(Mu)
        xs = np.array(xs)
        used.append(xs)
        oi = np.nonzero(cls_seg == CL_OPEN)[0]
        for m in range(i0, i1 + 1):
            if xs.size == 0:
                st[m] = rm.RM_ESINGULAR
                continue
            j, t = interpolation_weights(xs, pl["e_int"][m])
            Mu = kus[j] if xs.size == 1 else (1.0 - t) * kus[j] + t * kus[j + 1]
            row = np.zeros(nlev * (nlev + 1) // 2)
            if iqdt == 1:
                S = eliminate_s(Mu, cls_seg, float(E[m]), pw)
                if S is None:
                    st[m] = rm.RM_ESINGULAR
                    continue
                rm.omega_add(row, S - np.eye(S.shape[0]), oi, pw["level"], nlev, pw["g"])
            else:
                K = eliminate(Mu, cls_seg, float(E[m]), pw)
                if K is None:
                    st[m] = rm.RM_ESINGULAR
                    continue
                Ks[m] = K
                rm.omega_add(row, rm.t_matrix(K), oi, pw["level"], nlev, pw["g"])
            om[m] = row
    st[pl["seg"] < 0] = rm.RM_ETHRESHOLD
    return dict(status=st, n_open=no, K=Ks, omega=om, plan=pl, nodes_used=used)
