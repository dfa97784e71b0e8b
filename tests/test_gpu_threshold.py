"""Channel functions near thresholds on the GPU against the oracle.

With channel tables (the default of mixed-precision contexts, requested
here explicitly) and z > 0 the library evaluates a pair (energy, channel) within THR_ZONE
node spacings h of the channel's threshold by barycentric interpolation of
the channel's node table (16 energies straddling the threshold) instead of
continued fractions, h = min(0.0164 sqrt(z) / a^1.5, 0.05 z^2 / (l + 1)^2);
channels whose table fails its leave-one-out check, and z = 0, keep the
continued fractions (on the side stream). The oracle evaluates every pair by
its binary128 continued fractions. Energies are placed at fixed offsets from
each threshold, inside the zone, on both sides of its edge and just beyond.
"""
import numpy as np
import pytest

import oracle
from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu

THR_ZONE = 4.0


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


def node_spacing(z, a, l):
    return min(0.0164 * np.sqrt(z) / a ** 1.5, 0.05 * z * z / (l + 1.0) ** 2)


# (z, a, l of the four channels). In the last one the power series of f
# cancels by ~1e28 at r = a (sqrt(8 z a) = 64), the tables fail their check
# and every pair keeps its continued fractions; its energies stay at least
# h / 2 from the thresholds (closer ones take the binary128 oracle minutes).
CASES = [(2.0, 15.0, (0, 3, 8, 5)), (1.0, 30.0, (0, 4, 10, 15)), (5.0, 5.0, (1, 2, 6, 12)),
           (12.0, 10.0, (0, 2, 4, 7)), (1.0, 5.0, (15, 0, 10, 2)), (26.0, 20.0, (2, 0, 4, 1))]
REFUSED = len(CASES) - 1


def _pw(z, a, ls, seed):
    pw = synth.random_pw(seed, 4, 80, z=z, a=a, e_max=1.5, sigma=0.1)
    pw["e_thr"] = np.array([0.0, 0.5, 1.0, 1.5])
    pw["l"] = np.array(ls, dtype=np.int32)
    return pw


def _energies(pw, close=True):
    E = []
    for t, l in zip(pw["e_thr"], pw["l"]):
        h = node_spacing(pw["z"], pw["a"], int(l))
        offs = (3e-7, 4e-5) if close else ()
        for off in offs + (0.5 * h, 2.5 * h, 3.95 * h, 4.05 * h):
            for sg in (1.0, -1.0):
                x = t + sg * off
                if x > 0.0:
                    E.append(x)
    return np.array(sorted(E))


def _check_channel_functions(g, Es, pw, tag):
    for m, x in enumerate(Es):
        cf = oracle.channel_functions(float(x), pw["e_thr"], pw["l"], pw["z"], pw["a"])
        op = cf["open"]
        amp = np.hypot(cf["s"], cf["c"])[op]
        ampd = np.hypot(cf["sp"], cf["cp"])[op]
        for j, key in enumerate(["s", "sp", "c", "cp"]):
            sc = amp if key in ("s", "c") else ampd
            err = np.abs(g[m, op, j] - cf[key][op]) / sc
            assert err.max(initial=0) < 1e-11, (tag, x, key, err.max())
        cl = ~op
        assert np.abs(g[m, cl, 0] - cf["th"][cl]).max(initial=0) < 1e-10, (tag, x)
        assert np.abs(pw["a"] * (g[m, cl, 1] - cf["thp"][cl])).max(initial=0) < 1e-10, (tag, x)


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_channel_functions_near_thresholds(rt, ci):
    torch, rmgb = rt
    z, a, ls = CASES[ci]
    pw = _pw(z, a, ls, 900 + ci)
    Es = _energies(pw, close=ci != REFUSED)
    with rmgb.Context(channel_tables=1) as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
        out = torch.zeros((Es.size, 4, 4), dtype=torch.float64, device="cuda")
        st = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        ctx.channel_functions(0, Ed, out, st)
        w = torch.zeros((Es.size, 4, 4), dtype=torch.int32, device="cuda")
        ctx.channel_work(0, Ed, w)
        g = out.cpu().numpy()
        w = w.cpu().numpy()
        assert not st.cpu().numpy().any()
    _check_channel_functions(g, Es, pw, CASES[ci])
    # which pairs took the table: inside the zone unless the table was refused
    eps = Es[:, None] - pw["e_thr"][None, :]
    h = np.array([node_spacing(z, a, int(l)) for l in pw["l"]])
    interp = w[..., 0] == 3
    assert not (interp & (np.abs(eps) >= THR_ZONE * h[None, :])).any()
    if ci != REFUSED:
        assert np.array_equal(interp, np.abs(eps) < THR_ZONE * h[None, :])
    else:
        assert not interp.any()


@pytest.mark.parametrize("mode", [0, 1])
def test_k_omega_near_thresholds(rt, mode):
    """FP64 path (direct and MQDT) at the near-threshold energies against the
    oracle, 1e-9 norm-wise and per element."""
    torch, rmgb = rt
    pw = _pw(2.0, 15.0, (0, 3, 8, 5), 900)
    Es = _energies(pw)
    n = 4
    with rmgb.Context(channel_tables=1) as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
        K = torch.zeros((Es.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, Ed, mode, K, no, st)
        om = ctx.collision_strengths()
        K = K.cpu().numpy().reshape(Es.size, n, n)
        st = st.cpu().numpy()
    ref = oracle.solve_energies(pw, Es, mode=oracle.MODE_MQDT if mode else oracle.MODE_DIRECT)
    assert np.array_equal(st, ref["status"])
    bad = []
    for m in range(Es.size):
        if st[m]:
            continue
        k = ref["n_open"][m]
        for got, exp in ((K[m, :k, :k], ref["K"][m]), (om[m], ref["omega"][m])):
            nrm = np.linalg.norm(exp)
            mx = np.abs(exp).max(initial=0.0)
            if nrm and not (np.linalg.norm(got - exp) <= 1e-9 * nrm and
                            np.all(np.abs(got - exp) <= 1e-9 * np.maximum(np.abs(exp), mx))):
                bad.append(Es[m])
    assert not bad, bad[:10]


@pytest.mark.parametrize("ci", range(len(CASES) - 1))
def test_open_tables_vs_oracle(rt, ci):
    """Open pairs beyond the near-threshold zone come from the channel's
    Chebyshev table (12 terms per k-segment of width 0.9 / a, up to 16 Ry):
    random energies up to 15 Ry above the thresholds against the oracle."""
    torch, rmgb = rt
    z, a, ls = CASES[ci]
    pw = _pw(z, a, ls, 900 + ci)
    rng = np.random.default_rng(77 + ci)
    Es = np.sort(np.concatenate([rng.uniform(0.0, 2.0, 40), rng.uniform(2.0, 16.5, 40)]))
    with rmgb.Context(channel_tables=1) as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
        out = torch.zeros((Es.size, 4, 4), dtype=torch.float64, device="cuda")
        st = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        ctx.channel_functions(0, Ed, out, st)
        w = torch.zeros((Es.size, 4, 4), dtype=torch.int32, device="cuda")
        ctx.channel_work(0, Ed, w)
        g = out.cpu().numpy()
        w = w.cpu().numpy()
        assert not st.cpu().numpy().any()
    _check_channel_functions(g, Es, pw, ("open table",) + CASES[ci])
    eps = Es[:, None] - pw["e_thr"][None, :]
    h = np.array([node_spacing(z, a, int(l)) for l in pw["l"]])
    k0 = np.sqrt(THR_ZONE * h)[None, :]
    nseg = np.ceil(4.0 / (0.9 / a))
    inside = (eps > 0) & (np.sqrt(np.maximum(eps, 0)) - k0 >= 0) & (np.sqrt(np.maximum(eps, 0)) - k0 < nseg * 0.9 / a)
    assert inside.sum() > 100
    assert np.array_equal(w[..., 0] == 4, inside)


@pytest.mark.parametrize("ci", range(len(CASES) - 1))
def test_closed_tables_vs_oracle(rt, ci):
    """Closed pairs beyond the near-threshold zone (direct mode) come from the
    channel's table of the direction (theta, a theta') in nu (cells of 0.25
    split into up to 16 sub-segments of 12 terms) where the cell passed its
    check, else from the continued fractions: thresholds at 0, 5, 10, 15 Ry
    and random energies, so that closed pairs range from 16 Ry below
    threshold to the zone edge. All must match the oracle; deep closed pairs
    (smooth direction) must mostly come from the table."""
    torch, rmgb = rt
    z, a, ls = CASES[ci]
    pw = _pw(z, a, ls, 900 + ci)
    pw["e_thr"] = np.array([0.0, 5.0, 10.0, 15.0])
    rng = np.random.default_rng(99 + ci)
    Es = np.sort(np.concatenate([rng.uniform(0.01, 15.0, 60),
                                 np.array([5.0, 10.0, 15.0]) - rng.uniform(0.005, 0.05, 3)]))
    with rmgb.Context(channel_tables=1) as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
        out = torch.zeros((Es.size, 4, 4), dtype=torch.float64, device="cuda")
        st = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        ctx.channel_functions(0, Ed, out, st)
        w = torch.zeros((Es.size, 4, 4), dtype=torch.int32, device="cuda")
        ctx.channel_work(0, Ed, w)
        g = out.cpu().numpy()
        w = w.cpu().numpy()
        assert not st.cpu().numpy().any()
    _check_channel_functions(g, Es, pw, ("closed table",) + CASES[ci])
    eps = Es[:, None] - pw["e_thr"][None, :]
    h = np.array([node_spacing(z, a, int(l)) for l in pw["l"]])
    closed = (eps < 0) & (-eps >= THR_ZONE * h[None, :]) & (eps >= -16.0)
    assert closed.sum() > 60
    tab = w[..., 0] == 5
    assert not (tab & ~closed).any()
    assert np.isin(w[..., 0][closed], (1, 5)).all()
    deep = closed & (np.sqrt(np.maximum(-eps, 0.0)) * a > 8.0)
    assert tab[deep].mean() > 0.8, tab[deep].mean()
    # tables stop at the cell (0.25 in nu) that reaches kappa a = 6
    nu = z / np.sqrt(np.maximum(-eps, 1e-300))
    assert not (tab & (nu > z * a / 6.0 + 0.25 + 1e-9)).any()
