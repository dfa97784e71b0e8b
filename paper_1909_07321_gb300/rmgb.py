"""Python binding of the C ABI in include/rmgb.h (argument marshalling only).

Every function has the name of its C counterpart; arrays may be numpy arrays
(host) or torch tensors (host or CUDA). All arithmetic runs in librmgb.so;
if the library has not been built this module raises on import of any entry
point -- there is no CPU fallback.

A small `Context` class wraps the same calls for convenience.
"""
import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librmgb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rmgb.h")


def _constants():
    """#define RM_* integer constants, read from the header."""
    out = {}
    with open(HEADER) as f:
        for m in re.finditer(r"#define\s+(RM_\w+)\s+(-?\d+)", f.read()):
            out[m.group(1)] = int(m.group(2))
    return out


globals().update(_constants())


class RmOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("delta_pole", ctypes.c_double),
                ("eps_thr", ctypes.c_double), ("fnumin", ctypes.c_double),
                ("nu_margin", ctypes.c_double), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("mem_budget", ctypes.c_size_t),
                ("mqdt_kappa_a_max", ctypes.c_double), ("solver", ctypes.c_int),
                ("formulation", ctypes.c_int), ("solve_precision", ctypes.c_int),
                ("channel_tables", ctypes.c_int), ("lanes", ctypes.c_int), ("autotune", ctypes.c_int),
                ("pair_tile", ctypes.c_int)]


class RmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (rm_strerror(code), code, msg))
        self.code = code


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "rm_default_opts": (None, [ctypes.POINTER(RmOpts)]),
    "rm_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(RmOpts)]),
    "rm_destroy": (None, [_VP]),
    "rm_load_poles": (_I, [_VP, _I, _I, _I, _VP, _VP, _D, _D]),
    "rm_set_channels": (_I, [_VP, _I, _VP, _VP, _D, _VP, _I, _D]),
    "rm_set_multipoles": (_I, [_VP, _I, _I, _VP, _D, _I]),
    "rm_solve_energies": (_I, [_VP, _I, _I, _VP, _I, _VP, _VP, _VP]),
    "rm_collision_strengths": (_I, [_VP, _VP, _I]),
    "rm_collision_strengths_async": (_I, [_VP, _VP, _I]),
    "rm_solve_energies_qdt": (_I, [_VP, _I, _I, _VP, _I, _D, _I, _VP, _VP]),
    "rm_qdt_plan_inspect": (_I, [_I, _VP, _D, _I, _VP, _I, _VP, _VP, _I, _D, _VP, _I, _VP, _VP, _VP, _VP,
                                 _VP, _VP, _VP, _VP]),
    "rm_grid_shape": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rm_channel_functions": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "rm_form_r": (_I, [_VP, _I, _I, _VP, _VP]),
    "rm_channel_work": (_I, [_VP, _I, _I, _VP, _VP]),
    "rm_sync": (_I, [_VP]),
    "rm_reset_omega": (_I, [_VP]),
    "rm_profile_enable": (_I, [_VP, _I]),
    "rm_profile_get": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "rm_launch_count": (ctypes.c_longlong, [_VP]),
    "rm_lane_solve_energies": (_I, [_VP, _I, _I, _I, _VP, _I, _VP, _VP, _VP]),
    "rm_lane_collision_strengths": (_I, [_VP, _I, _VP, _I]),
    "rm_lane_query": (_I, [_VP, _I]),
    "rm_lane_sync": (_I, [_VP, _I]),
    "rm_lane_stream": (_VP, [_VP, _I]),
    "rm_lane_reserve": (_I, [_VP, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "rm_pw_bytes": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "rm_unload_pw": (_I, [_VP, _I]),
    "rm_solve_batch": (_I, [_VP, _I, _VP, _I, _VP, _I, _I]),
    "rm_autotune_info": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), _VP]),
    "rm_set_wait_probe": (_I, [_VP, ctypes.c_ulonglong]),
    "rm_strerror": (ctypes.c_char_p, [_I]),
    "rm_last_error": (ctypes.c_char_p, [_VP]),
}


def lib():
    """Load librmgb.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librmgb.so is not built (run paper_1909_07321_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x, dtype=None):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(x.dtype).split(".")[-1] != np.dtype(dtype).name:
            raise TypeError("tensor dtype %s, expected %s" % (x.dtype, np.dtype(dtype).name))
        return x.data_ptr()
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous):
        raise ValueError("expected a C-contiguous numpy array or a torch tensor")
    if dtype is not None and x.dtype != np.dtype(dtype):
        raise TypeError("array dtype %s, expected %s" % (x.dtype, np.dtype(dtype).name))
    return x.ctypes.data


def _host(x, dtype):
    if hasattr(x, "data_ptr"):
        return x
    return np.ascontiguousarray(x, dtype=dtype)


def rm_strerror(code):
    return lib().rm_strerror(int(code)).decode()


def rm_last_error(ctx):
    return lib().rm_last_error(ctx).decode()


def rm_default_opts():
    o = RmOpts()
    lib().rm_default_opts(ctypes.byref(o))
    return o


def rm_create(opts=None):
    h = _VP()
    rc = lib().rm_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None)
    if rc:
        raise RmError(rc, "rm_create")
    return h


def rm_destroy(ctx):
    lib().rm_destroy(ctx)


def _check(ctx, rc):
    if rc:
        raise RmError(rc, rm_last_error(ctx))
    return rc


def rm_load_poles(ctx, pw, E_k, W, a, b=0.0):
    E_k = _host(E_k, np.float64)
    W = _host(W, np.float64)
    n_ch, n_poles = W.shape
    return _check(ctx, lib().rm_load_poles(ctx, pw, n_ch, n_poles, _ptr(E_k, np.float64),
                                           _ptr(W, np.float64), a, b))


def rm_set_channels(ctx, pw, e_thr, l, z, level, n_levels, g_weight):
    e_thr = _host(e_thr, np.float64)
    l = _host(l, np.int32)
    level = _host(level, np.int32)
    return _check(ctx, lib().rm_set_channels(ctx, pw, _ptr(e_thr, np.float64), _ptr(l, np.int32),
                                             z, _ptr(level, np.int32), n_levels, g_weight))


def rm_set_multipoles(ctx, pw, A, r1, n_steps):
    """A: [lambda_max][n_ch][n_ch] (lambda_max = 0 or A None: propagation off)."""
    if A is None:
        return _check(ctx, lib().rm_set_multipoles(ctx, pw, 0, None, 0.0, 0))
    if hasattr(A, "cpu"):
        A = A.cpu().numpy()
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim != 3:
        raise ValueError("A must be [lambda_max][n_ch][n_ch]")
    return _check(ctx, lib().rm_set_multipoles(ctx, pw, int(A.shape[0]), _ptr(A, np.float64), float(r1),
                                               int(n_steps)))


def rm_solve_energies(ctx, pw, E, mode=0, K_out=None, n_open_out=None, status_out=None):
    E = _host(E, np.float64)
    return _check(ctx, lib().rm_solve_energies(ctx, pw, int(E.shape[0]), _ptr(E, np.float64), mode,
                                               _ptr(K_out, np.float64), _ptr(n_open_out, np.int32),
                                               _ptr(status_out, np.int32)))


def rm_solve_energies_qdt(ctx, pw, E, ieq, qetest=0.0, iqdt=1, n_open_out=None, status_out=None):
    """MQDT coarse-mesh interpolation; E must be a host array (ascending)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    return _check(ctx, lib().rm_solve_energies_qdt(ctx, pw, int(E.shape[0]), _ptr(E, np.float64), int(ieq),
                                                   float(qetest), int(iqdt), _ptr(n_open_out, np.int32),
                                                   _ptr(status_out, np.int32)))


def rm_lane_solve_energies(ctx, lane, pw, E, mode=0, K_out=None, n_open_out=None, status_out=None):
    E = _host(E, np.float64)
    return _check(ctx, lib().rm_lane_solve_energies(ctx, int(lane), pw, int(E.shape[0]), _ptr(E, np.float64),
                                                    mode, _ptr(K_out, np.float64), _ptr(n_open_out, np.int32),
                                                    _ptr(status_out, np.int32)))


def rm_lane_collision_strengths(ctx, lane, omega_out, reset=False):
    """Copies lane `lane`'s Omega into omega_out (host float64 array of the
    lane's grid shape) after synchronising that lane."""
    return _check(ctx, lib().rm_lane_collision_strengths(ctx, int(lane), _ptr(omega_out, np.float64),
                                                         int(bool(reset))))


def rm_lane_query(ctx, lane):
    """True when the lane's enqueued work has completed."""
    rc = lib().rm_lane_query(ctx, int(lane))
    if rc < 0:
        raise RmError(rc, rm_last_error(ctx))
    return bool(rc)


def rm_lane_sync(ctx, lane):
    return _check(ctx, lib().rm_lane_sync(ctx, int(lane)))


def rm_lane_stream(ctx, lane):
    return lib().rm_lane_stream(ctx, int(lane))


def rm_lane_reserve(ctx, lane, pw, n_E):
    """Pre-sizes the lane's workspace for n_E energies of pw; returns the
    lane's device bytes."""
    b = ctypes.c_size_t(0)
    _check(ctx, lib().rm_lane_reserve(ctx, int(lane), int(pw), int(n_E), ctypes.byref(b)))
    return b.value


def rm_pw_bytes(ctx, pw):
    b = ctypes.c_size_t(0)
    _check(ctx, lib().rm_pw_bytes(ctx, int(pw), ctypes.byref(b)))
    return b.value


def rm_unload_pw(ctx, pw):
    return _check(ctx, lib().rm_unload_pw(ctx, int(pw)))


def rm_solve_batch(ctx, pws, E, mode=0, use_graph=True):
    """Solves the partial waves pws (sequence of indices) on the energies E,
    spread over the context's lanes, accumulating into Omega."""
    p = np.ascontiguousarray(pws, dtype=np.int32)
    E = _host(E, np.float64)
    return _check(ctx, lib().rm_solve_batch(ctx, int(p.size), _ptr(p, np.int32), int(E.shape[0]),
                                            _ptr(E, np.float64), int(mode), int(bool(use_graph))))


def rm_autotune_info(ctx, pw):
    """(formulation, tile_n, stages, ms per energy of the 4 candidates)."""
    f, t, st = _I(), _I(), _I()
    ms = np.zeros(4)
    _check(ctx, lib().rm_autotune_info(ctx, int(pw), ctypes.byref(f), ctypes.byref(t), ctypes.byref(st),
                                       _ptr(ms, np.float64)))
    return f.value, t.value, st.value, ms


def rm_grid_shape(ctx):
    a, b = _I(), _I()
    lib().rm_grid_shape(ctx, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def rm_collision_strengths(ctx, omega_out=None, reset=False):
    """Copies Omega into omega_out (numpy, allocated if None) and returns it."""
    nE, ntri = rm_grid_shape(ctx)
    if omega_out is None and nE:
        omega_out = np.empty((nE, ntri), dtype=np.float64)
    _check(ctx, lib().rm_collision_strengths(ctx, _ptr(omega_out, np.float64), int(bool(reset))))
    return omega_out


def rm_collision_strengths_async(ctx, omega_out, reset=False):
    """Enqueues the copy of Omega into omega_out (host, [n_E][n_tri] float64;
    page-locked for overlap, e.g. a pinned torch tensor's numpy view); it is
    written by the time rm_sync returns."""
    nE, ntri = rm_grid_shape(ctx)
    if hasattr(omega_out, "data_ptr"):
        ok = tuple(omega_out.shape) == (nE, ntri) and omega_out.device.type == "cpu"
    else:
        ok = isinstance(omega_out, np.ndarray) and omega_out.shape == (nE, ntri)
    if not ok:
        raise ValueError("omega_out must be a host array of shape (%d, %d)" % (nE, ntri))
    return _check(ctx, lib().rm_collision_strengths_async(ctx, _ptr(omega_out, np.float64),
                                                          int(bool(reset))))


def rm_qdt_plan_inspect(e_thr, z, E_k, E, cls, ieq, qetest=0.0, node_ok=None):
    """Host planning of the coarse-mesh interpolation (no GPU needed): cls is
    [n_E][n_ch] int8 (0 open, 1 eliminated, 2 decaying, 3 on a threshold);
    node_ok (optional, one flag per valid node) marks node solves that
    failed. Returns dict seg, e_int, node_x, node_seg, node_a, node_b, t."""
    e_thr = np.ascontiguousarray(e_thr, dtype=np.float64)
    E_k = np.ascontiguousarray(E_k, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    cls = np.ascontiguousarray(cls, dtype=np.int8)
    n_E, n = E.size, e_thr.size
    if cls.shape != (n_E, n):
        raise ValueError("cls must be [n_E][n_ch]")
    cap = 4 * n_E + (abs(int(ieq)) if ieq > 0 else 0) + 8
    seg = np.empty(n_E, dtype=np.int32)
    e_int = np.empty(n_E)
    nn = ctypes.c_int(0)
    node_x = np.empty(cap)
    node_seg = np.empty(cap, dtype=np.int32)
    na = np.empty(n_E, dtype=np.int32)
    nb = np.empty(n_E, dtype=np.int32)
    t = np.empty(n_E)
    ok = None if node_ok is None else np.ascontiguousarray(node_ok, dtype=np.int32)
    if ok is not None and ok.size < cap:
        ok = np.concatenate([ok, np.ones(cap - ok.size, dtype=np.int32)])
    rc = lib().rm_qdt_plan_inspect(n, _ptr(e_thr), float(z), E_k.size, _ptr(E_k) if E_k.size else None, n_E,
                                   _ptr(E), cls.ctypes.data, int(ieq), float(qetest), _ptr(ok), cap, _ptr(seg),
                                   _ptr(e_int), ctypes.byref(nn), _ptr(node_x), _ptr(node_seg), _ptr(na),
                                   _ptr(nb), _ptr(t))
    if rc:
        raise RmError(rc, "rm_qdt_plan_inspect")
    k = nn.value
    return dict(seg=seg, e_int=e_int, node_x=node_x[:k].copy(), node_seg=node_seg[:k].copy(),
                node_a=na, node_b=nb, t=t)


def rm_channel_functions(ctx, pw, E, out, status=None):
    return _check(ctx, lib().rm_channel_functions(ctx, pw, int(E.shape[0]), _ptr(E, np.float64),
                                                  _ptr(out, np.float64), _ptr(status, np.int32)))


def rm_channel_work(ctx, pw, E, work):
    return _check(ctx, lib().rm_channel_work(ctx, pw, int(E.shape[0]), _ptr(E, np.float64),
                                             _ptr(work, np.int32)))


def rm_form_r(ctx, pw, E, R_out):
    return _check(ctx, lib().rm_form_r(ctx, pw, int(E.shape[0]), _ptr(E, np.float64),
                                       _ptr(R_out, np.float64)))


def rm_sync(ctx):
    return _check(ctx, lib().rm_sync(ctx))


def rm_reset_omega(ctx):
    return _check(ctx, lib().rm_reset_omega(ctx))


def rm_profile_enable(ctx, enable=True):
    return _check(ctx, lib().rm_profile_enable(ctx, int(bool(enable))))


def rm_profile_get(ctx, phase):
    """(launches, milliseconds) of one RM_PH_* phase since rm_profile_enable."""
    n, ms = _I(), _D()
    _check(ctx, lib().rm_profile_get(ctx, phase, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def rm_launch_count(ctx):
    return int(lib().rm_launch_count(ctx))


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def _torch_current_stream(device):
    """Handle of torch's current stream on `device` (legacy default -> cudaStreamLegacy),
    or None when torch/CUDA is unavailable."""
    try:
        import torch
    except ImportError:
        return None
    if not torch.cuda.is_available():
        return None
    h = torch.cuda.current_stream(device).cuda_stream
    return h if h else CUDA_STREAM_LEGACY


class Context:
    """Owns one rm_ctx; methods forward to the rm_* functions above.

    By default the context enqueues on torch's current stream of `device`, so
    its work is ordered with the torch operations that fill its inputs and
    read its outputs."""

    def __init__(self, precision=0, stream=None, mem_budget=0, device=0, **kw):
        o = rm_default_opts()
        o.precision = precision
        o.device = device
        o.mem_budget = mem_budget
        if stream is None:
            stream = _torch_current_stream(device)
        if stream is not None:
            o.stream = stream
        for k, v in kw.items():
            if k not in [f[0] for f in RmOpts._fields_]:
                raise TypeError("unknown rm_opts field %r" % k)
            setattr(o, k, v)
        self._n_ch = {}          # channels of each loaded partial wave
        self.h = rm_create(o)

    def close(self):
        if self.h:
            rm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_pw(self, pw, d):
        """Load one partial wave given as a dict (keys of synth's partial waves)."""
        rm_load_poles(self.h, pw, d["E_k"], d["W"], d["a"], d.get("b", 0.0))
        self._n_ch[pw] = int(d["W"].shape[0]) if hasattr(d["W"], "shape") else len(d["W"])
        rm_set_channels(self.h, pw, d["e_thr"], d["l"], d["z"], d["level"], d["n_levels"], d["g"])

    def set_multipoles(self, pw, A, r1=0.0, n_steps=0):
        """A: [lambda_max][n_ch][n_ch] of the loaded wave (None: propagation off)."""
        n = getattr(self, "_n_ch", {}).get(pw)
        if A is not None and n is not None:
            shape = tuple(A.shape) if hasattr(A, "shape") else np.shape(A)
            if len(shape) != 3 or shape[1:] != (n, n):
                raise ValueError("A must be [lambda_max][%d][%d] for partial wave %d, got %s" % (n, n, pw, shape))
        return rm_set_multipoles(self.h, pw, A, r1, n_steps)

    def solve_energies(self, pw, E, mode=0, K_out=None, n_open_out=None, status_out=None):
        return rm_solve_energies(self.h, pw, E, mode, K_out, n_open_out, status_out)

    def collision_strengths(self, omega_out=None, reset=False):
        return rm_collision_strengths(self.h, omega_out, reset)

    def collision_strengths_async(self, omega_out, reset=False):
        return rm_collision_strengths_async(self.h, omega_out, reset)

    def channel_functions(self, pw, E, out, status=None):
        return rm_channel_functions(self.h, pw, E, out, status)

    def solve_energies_qdt(self, pw, E, ieq, qetest=0.0, iqdt=1, n_open_out=None, status_out=None):
        return rm_solve_energies_qdt(self.h, pw, E, ieq, qetest, iqdt, n_open_out, status_out)

    def form_r(self, pw, E, R_out):
        return rm_form_r(self.h, pw, E, R_out)

    def channel_work(self, pw, E, work):
        return rm_channel_work(self.h, pw, E, work)

    def sync(self):
        return rm_sync(self.h)

    def launch_count(self):
        return rm_launch_count(self.h)

    def reset_omega(self):
        return rm_reset_omega(self.h)

    def profile_enable(self, enable=True):
        return rm_profile_enable(self.h, enable)

    def profile_get(self, phase):
        return rm_profile_get(self.h, phase)

    def lane_solve_energies(self, lane, pw, E, mode=0, K_out=None, n_open_out=None, status_out=None):
        return rm_lane_solve_energies(self.h, lane, pw, E, mode, K_out, n_open_out, status_out)

    def lane_collision_strengths(self, lane, omega_out, reset=False):
        return rm_lane_collision_strengths(self.h, lane, omega_out, reset)

    def lane_query(self, lane):
        return rm_lane_query(self.h, lane)

    def lane_sync(self, lane):
        return rm_lane_sync(self.h, lane)

    def lane_stream(self, lane):
        return rm_lane_stream(self.h, lane)

    def lane_reserve(self, lane, pw, n_E):
        return rm_lane_reserve(self.h, lane, pw, n_E)

    def pw_bytes(self, pw):
        return rm_pw_bytes(self.h, pw)

    def solve_batch(self, pws, E, mode=0, use_graph=True):
        return rm_solve_batch(self.h, pws, E, mode, use_graph)

    def autotune_info(self, pw):
        return rm_autotune_info(self.h, pw)

    def set_wait_probe(self, limit_ns):
        return _check(self.h, lib().rm_set_wait_probe(self.h, int(limit_ns)))

    def unload_pw(self, pw):
        self._n_ch.pop(pw, None)
        return rm_unload_pw(self.h, pw)
