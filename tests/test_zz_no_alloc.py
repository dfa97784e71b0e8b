"""rm_k_matrices_noalloc: the entry point for callers that cannot let the
library allocate device memory (memory owned by another allocator, or loops
that cannot take cudaMalloc's device-wide synchronisation). It must give the
K-matrices that rm_solve_energies gives, call after call, although every call
reuses the same static workspace.

This file is collected last so that a run stopping at its first failure has
run every other test already."""
import ctypes

import numpy as np
import pytest

from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_K = 1e-9


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    fn = rmgb.lib().rm_k_matrices_noalloc
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    fn.restype = i
    fn.argtypes = [i, i, i, i, vp, vp, vp, vp, d, d, d, vp, d, vp, vp, vp, vp,
                   ctypes.c_char_p, ctypes.c_size_t]
    return torch, rmgb, fn


def _reference_K(torch, rmgb, pw, E):
    n = pw["W"].shape[0]
    with rmgb.Context(channel_tables=0) as ctx:   # the same continued fractions as the call
        ctx.load_pw(0, pw)
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, Ed, 0, K, no, st)
        torch.cuda.synchronize()
    return K.cpu().numpy(), no.cpu().numpy(), st.cpu().numpy()


def _noalloc_K(torch, fn, pw, E, free_bytes=None):
    """K, n_open and statuses from rm_k_matrices_noalloc. With free_bytes (a
    list), the device's free memory (cudaMemGetInfo) just before and just
    after the call is appended to it; every buffer the call sees is made
    before the first reading."""
    n, N = pw["W"].shape
    order = np.argsort(pw["E_k"], kind="stable")      # the call wants sorted poles
    dev = lambda x, t=torch.float64: torch.tensor(np.ascontiguousarray(x), dtype=t,  # noqa: E731
                                                  device="cuda")
    Ek, W = dev(pw["E_k"][order]), dev(pw["W"][:, order])
    thr, l = dev(pw["e_thr"]), dev(pw["l"], torch.int32)
    Ed = dev(E)
    K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
    no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
    st = torch.full((E.size,), 7, dtype=torch.int32, device="cuda")   # must be cleared by the call
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream or None
    torch.cuda.synchronize()
    if free_bytes is not None:
        free_bytes.append(torch.cuda.mem_get_info()[0])
    rc = fn(0, n, N, E.size, Ek.data_ptr(), W.data_ptr(), thr.data_ptr(), l.data_ptr(),
            pw["z"], pw["a"], pw.get("b", 0.0), Ed.data_ptr(), 1e-10, K.data_ptr(),
            no.data_ptr(), st.data_ptr(), stream, err, 256)
    assert rc == 0, err.value
    torch.cuda.synchronize()
    if free_bytes is not None:
        free_bytes.append(torch.cuda.mem_get_info()[0])
    return K.cpu().numpy(), no.cpu().numpy(), st.cpu().numpy()


def _assert_same_K(got, ref, n):
    Kg, nog, stg = got
    Kr, nor, str_ = ref
    assert np.array_equal(stg, str_)
    assert np.array_equal(nog, nor)
    for e in range(stg.size):
        if stg[e]:
            continue
        m = nor[e]
        A = Kg[e].reshape(n, n)[:m, :m]
        B = Kr[e].reshape(n, n)[:m, :m]
        nrm = np.linalg.norm(B)
        assert np.linalg.norm(A - B) <= TOL_K * max(nrm, 1e-300)


def test_noalloc_matches_solve_energies_twice(rt):
    torch, rmgb, fn = rt
    cases = [synth.workload_small(500), synth.workload_64ch(20000)]
    for pws, E in cases:
        pw = pws[0]
        n = pw["W"].shape[0]
        if E.size > 2500:        # more energies than one workspace chunk holds
            E = E[::8][:2500].copy()
        ref = _reference_K(torch, rmgb, pw, E)
        first = _noalloc_K(torch, fn, pw, E)
        second = _noalloc_K(torch, fn, pw, E)
        _assert_same_K(first, ref, n)
        _assert_same_K(second, ref, n)


def test_noalloc_leaves_free_memory_unchanged(rt):
    """The promise of the call's name: after a first (warm-up) call has loaded
    the code, a second call over more energies than one workspace chunk holds
    (the 64-channel workload: about 1700 energies per chunk) changes the
    device's free memory by nothing, and leaves the caller's current device
    as it was."""
    torch, rmgb, fn = rt
    pws, E = synth.workload_64ch(20000)
    E = E[::8][:2500].copy()
    _noalloc_K(torch, fn, pws[0], E)
    dev_before = torch.cuda.current_device()
    free = []
    _noalloc_K(torch, fn, pws[0], E, free)
    assert free[0] == free[1], "free device memory changed by %d bytes" % (free[0] - free[1])
    assert torch.cuda.current_device() == dev_before


def test_noalloc_rejects_oversize(rt):
    torch, rmgb, fn = rt
    err = ctypes.create_string_buffer(256)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = fn(0, 97, 4, 1, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 1.0, 10.0, 0.0,
            x.data_ptr(), 1e-10, None, None, x.data_ptr(), None, err, 256)
    assert rc == rmgb.RM_EUNSUPPORTED
    assert b"97" in err.value
