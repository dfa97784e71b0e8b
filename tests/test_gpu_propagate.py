"""Outer-region propagation with the long-range multipole potential on the GPU
(rm_set_multipoles) against the oracle (oracle/propagate.py).

The GPU integrates the coupled equations from a to r1 by Numerov's method
with a fixed number of steps, the oracle by DOP853 at rtol 1e-13 sector by
sector; with a = 12, r1 = 15 and 4000 steps (h = 7.5e-4) the O(h^4) error of
Numerov is ~1e-13 of R, far below the 1e-9 bar, so K and Omega must agree to
1e-9 norm-wise and per element, in direct and MQDT modes, with and without
channel tables (built at r1).
"""
import numpy as np
import pytest

from oracle import propagate as pr
import oracle
from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu

A_, R1, STEPS = 12.0, 15.0, 4000


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


def _pw(n=4, seed=5150, z=1.0):
    pw = synth.random_pw(seed, n, 15 * n, z=z, a=A_, e_max=1.5, sigma=0.1, l_max=3)
    pw["e_thr"] = np.linspace(0.0, 1.2, n)
    return pw


def _coupling(n, lmax, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, scale, (lmax, n, n))
    return 0.5 * (A + A.transpose(0, 2, 1))


def _energies(pw, m=24, seed=1):
    rng = np.random.default_rng(seed)
    E = np.sort(rng.uniform(0.02, 1.6, m))
    # keep clear of thresholds (the continued fractions there are slow in
    # the oracle and the channel classes flip)
    thr = np.asarray(pw["e_thr"])
    return E[np.abs(E[:, None] - thr[None, :]).min(axis=1) > 5e-3]


def _gpu_solve(rt, pw, E, A, mode, r1=R1, steps=STEPS, **opts):
    torch, rmgb = rt
    n = pw["W"].shape[0]
    with rmgb.Context(**opts) as ctx:
        ctx.load_pw(0, pw)
        if A is not None:
            ctx.set_multipoles(0, A, r1, steps)
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, Ed, mode, K, no, st)
        om = ctx.collision_strengths()
        return K.cpu().numpy().reshape(E.size, n, n), no.cpu().numpy(), st.cpu().numpy(), om


def _compare(E, K, no, st, om, ref, tol=1e-9):
    assert np.array_equal(st, ref["status"]), (st, ref["status"])
    assert np.array_equal(no, ref["n_open"])
    bad = []
    for m in range(E.size):
        if st[m]:
            continue
        k = ref["n_open"][m]
        for got, exp in ((K[m, :k, :k], ref["K"][m]), (om[m], ref["omega"][m])):
            nrm = np.linalg.norm(exp)
            mx = np.abs(exp).max(initial=0.0)
            if nrm and not (np.linalg.norm(got - exp) <= tol * nrm and
                            np.all(np.abs(got - exp) <= tol * np.maximum(np.abs(exp), mx))):
                bad.append((E[m], np.abs(got - exp).max() / mx))
    assert not bad, bad[:10]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("tables", [0, 1])
def test_propagated_k_omega_vs_oracle(rt, mode, tables):
    pw = _pw()
    A = _coupling(4, 2, 11)
    E = _energies(pw)
    K, no, st, om = _gpu_solve(rt, pw, E, A, mode, channel_tables=tables)
    ref = pr.solve_energies(pw, E, A, R1, mode=oracle.MODE_MQDT if mode else oracle.MODE_DIRECT)
    assert (st == 0).sum() >= E.size - 2
    _compare(E, K, no, st, om, ref)


def test_propagated_lambda_max_4_and_b(rt):
    """All four multipole orders, a non-zero log-derivative b and 8 channels."""
    pw = _pw(n=8, seed=77, z=2.0)
    pw["b"] = 0.7
    A = _coupling(8, 4, 12, scale=0.2)
    E = _energies(pw, m=16, seed=2)
    K, no, st, om = _gpu_solve(rt, pw, E, A, 0)
    ref = pr.solve_energies(pw, E, A, R1)
    _compare(E, K, no, st, om, ref)


@pytest.mark.parametrize("n,lmax,mode", [(20, 2, 0), (48, 2, 0), (48, 2, 1), (64, 3, 0), (64, 3, 1)])
def test_propagated_above_16_channels(rt, n, lmax, mode):
    """The one-energy-per-CTA kernels: 20 channels (the 256-thread kernel,
    ragged against its 32-channel tiles), 48 and 64 channels (the 512-thread
    kernel; 64 with lambda_max = 3, the most that fits one CTA), direct and
    MQDT modes, against the oracle at 1e-9."""
    pw = _pw(n=n, seed=900 + n, z=2.0)
    A = _coupling(n, lmax, 40 + n, scale=0.2)
    E = _energies(pw, m=16, seed=n)
    K, no, st, om = _gpu_solve(rt, pw, E, A, mode)
    ref = pr.solve_energies(pw, E, A, R1, mode=oracle.MODE_MQDT if mode else oracle.MODE_DIRECT)
    assert (ref["status"] == 0).sum() >= E.size - 2
    _compare(E, K, no, st, om, ref)


def test_propagated_64_channels_mixed(rt):
    """64 channels, bf16x3 formation and the FP32 solve on propagated R:
    Omega within 1e-4 of the oracle in the median and 1e-2 at most (relative
    to the energy's largest entry). The FP32 elimination's backward error
    grows as n 2^-24 (4e-6 at 64 channels, before the matching's
    conditioning), 16x that of the 4-channel case's 1e-5."""
    pw = _pw(n=64, seed=964, z=2.0)
    A = _coupling(64, 3, 104, scale=0.2)
    E = _energies(pw, m=16, seed=64)
    K, no, st, om = _gpu_solve(rt, pw, E, A, 0, precision=2, solve_precision=1)
    ref = pr.solve_energies(pw, E, A, R1)
    assert np.array_equal(st, ref["status"])
    errs = [np.abs(om[m] - ref["omega"][m]).max() / np.abs(ref["omega"][m]).max()
            for m in range(E.size) if not st[m] and np.abs(ref["omega"][m]).max()]
    assert len(errs) >= 8
    assert np.median(errs) < 1e-4 and max(errs) < 1e-2, errs


def test_coupling_matters_and_off_switch(rt):
    """The coupling changes Omega; lambda_max = 0 (A None) restores the
    unpropagated results bit for bit; reloading the poles clears it."""
    torch, rmgb = rt
    pw = _pw()
    A = _coupling(4, 2, 11)
    E = _energies(pw)
    _, _, st0, om0 = _gpu_solve(rt, pw, E, None, 0)
    _, _, st1, om1 = _gpu_solve(rt, pw, E, A, 0)
    ok = (st0 == 0) & (st1 == 0)
    assert np.abs(om1[ok] - om0[ok]).max() > 1e-3 * np.abs(om0[ok]).max()
    n = 4
    for how in ("off", "reload"):
        with rmgb.Context() as ctx:
            ctx.load_pw(0, pw)
            ctx.set_multipoles(0, A, R1, STEPS)
            if how == "off":
                ctx.set_multipoles(0, None)
            else:
                rmgb.rm_load_poles(ctx.h, 0, pw["E_k"], pw["W"], pw["a"], 0.0)
            st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
            ctx.solve_energies(0, torch.tensor(E, dtype=torch.float64, device="cuda"), 0, None, None, st)
            om = ctx.collision_strengths()
            assert np.array_equal(st.cpu().numpy(), st0)
            assert np.array_equal(om, om0), how


def test_zero_coupling_matches_unpropagated(rt):
    """A = 0: propagation from a to r1 only carries the Coulomb functions
    along, so K matched at r1 equals K matched at a (to Numerov's error)."""
    pw = _pw()
    E = _energies(pw)
    K0, no0, st0, om0 = _gpu_solve(rt, pw, E, None, 0)
    K1, no1, st1, om1 = _gpu_solve(rt, pw, E, np.zeros((1, 4, 4)), 0)
    ref = oracle.solve_energies(pw, E)
    _compare(E, K1, no1, st1, om1, ref)
    _compare(E, K0, no0, st0, om0, ref)


def test_mixed_precision_with_propagation(rt):
    """bf16x3 formation and the FP32 solve on propagated R: Omega within the
    mixed path's usual accuracy of the oracle (median 1e-5, max 1e-2
    relative to the energy's largest entry)."""
    pw = _pw()
    A = _coupling(4, 2, 11)
    E = _energies(pw, m=40, seed=3)
    K, no, st, om = _gpu_solve(rt, pw, E, A, 0, precision=2, solve_precision=1)
    ref = pr.solve_energies(pw, E, A, R1)
    assert np.array_equal(st, ref["status"])
    errs = []
    for m in range(E.size):
        if st[m]:
            continue
        mx = np.abs(ref["omega"][m]).max(initial=0.0)
        if mx:
            errs.append(np.abs(om[m] - ref["omega"][m]).max() / mx)
    errs = np.array(errs)
    assert errs.size > 30
    assert np.median(errs) < 1e-5 and errs.max() < 1e-2, (np.median(errs), errs.max())


def test_set_multipoles_rejects_bad_arguments(rt):
    torch, rmgb = rt
    pw = _pw()
    A = _coupling(4, 2, 11)
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        cases = [
            (np.zeros((5, 4, 4)), R1, STEPS, rmgb.RM_EINVAL),              # lambda_max > 4
            (A, A_ - 0.5, STEPS, rmgb.RM_EINVAL),                          # r1 < a
            (A, R1, 1, rmgb.RM_EINVAL),                                    # < 2 steps
            (A + np.triu(np.ones((4, 4)), 1)[None], R1, STEPS, rmgb.RM_EINVAL),  # not symmetric
            (np.full((1, 4, 4), np.nan), R1, STEPS, rmgb.RM_EINVAL),
        ]
        for Ab, r1, steps, code in cases:
            with pytest.raises(rmgb.RmError) as ei:
                ctx.set_multipoles(0, Ab, r1, steps)
            assert ei.value.code == code
        with pytest.raises(rmgb.RmError) as ei:
            ctx.set_multipoles(1, A, R1, STEPS)
        assert ei.value.code == rmgb.RM_ENOTLOADED
        big = synth.random_pw(3, 65, 130, z=1.0, a=A_)
        ctx.load_pw(2, big)
        with pytest.raises(rmgb.RmError) as ei:
            ctx.set_multipoles(2, np.zeros((1, 65, 65)), R1, STEPS)
        assert ei.value.code == rmgb.RM_EUNSUPPORTED
        # 64 channels: lambda_max = 3 fits one CTA's shared memory, 4 does not
        ctx.load_pw(3, synth.random_pw(4, 64, 128, z=1.0, a=A_))
        ctx.set_multipoles(3, np.zeros((3, 64, 64)), R1, STEPS)
        with pytest.raises(rmgb.RmError) as ei:
            ctx.set_multipoles(3, np.zeros((4, 64, 64)), R1, STEPS)
        assert ei.value.code == rmgb.RM_EUNSUPPORTED


def test_multipole_workload_sampled(rt):
    """The 32-channel multipole workload (lambda_max = 2, a = 15 -> r1 = 35),
    all 1024 energies in one launch as the benchmark runs them: FP64 with 16x
    the benchmark's steps against the oracle at 1e-9 on 8 sampled energies
    (Numerov's error in R falls 16x per halving of h: ~7e-8 at 2000 steps,
    ~2e-10 at 8000; at 32000 what is left, ~6e-11, is rounding on both
    sides), and the benchmark's mixed configuration (bf16x3 formation, FP32
    solve, 2000 steps) within the mixed path's accuracy."""
    torch, rmgb = rt
    pw, A, r1, steps, E = synth.workload_multipole(1024)
    n = pw["W"].shape[0]
    idx = np.linspace(3, E.size - 4, 8).astype(int)
    ref = pr.solve_energies(pw, E[idx], A, r1)
    for opts, st_mult in ((dict(precision=0), 16), (dict(precision=2, solve_precision=1), 1)):
        K, no, st, om = _gpu_solve(rt, pw, E, A, 0, r1=r1, steps=steps * st_mult, **opts)
        if opts["precision"] == 0:
            _compare(E[idx], K[idx], no[idx], st[idx], om[idx], ref)
        else:
            assert np.array_equal(st[idx], ref["status"])
            rel = [np.abs(om[m] - ref["omega"][k]).max() / np.abs(ref["omega"][k]).max()
                   for k, m in enumerate(idx) if not st[m]]
            assert np.median(rel) < 1e-5 and max(rel) < 1e-2, rel
        assert (st == 0).mean() > 0.95


def test_small_n_batched_energies(rt):
    """n <= 16 runs several energies per CTA (64 at n = 3): 150 energies, so
    that the last CTA is partly empty, one of them on a pole (its status must
    stay RM_ENEAR_POLE and its neighbours in the same CTA must be unaffected),
    against the oracle at 1e-9."""
    pw = _pw(n=3, seed=31, z=1.0)
    A = _coupling(3, 2, 17)
    rng = np.random.default_rng(5)
    E = np.sort(rng.uniform(0.02, 1.6, 150))
    thr = np.asarray(pw["e_thr"])
    E = E[np.abs(E[:, None] - thr[None, :]).min(axis=1) > 5e-3]
    pole = pw["E_k"][(pw["E_k"] > 0.1) & (pw["E_k"] < 1.5)][0]
    E[40] = pole
    E = np.sort(E)
    K, no, st, om = _gpu_solve(rt, pw, E, A, 0)
    ref = pr.solve_energies(pw, E, A, R1)
    assert (ref["status"] != 0).sum() >= 1
    _compare(E, K, no, st, om, ref)
