"""GB300 partial-update MACE CT reconstruction (arXiv 1911.09278).

Thin ctypes binding of the C ABI in ``include/mace.h``: argument marshalling
only, every step of the reconstruction runs in the CUDA library
``libmace.so`` built from ``csrc/mace.cu`` for sm_103a.  There is no CPU
fallback: importing works without a GPU, but every call that needs the library
raises if it is not built or cannot run.

Arrays may be numpy (host memory) or torch CUDA tensors (device memory, used
in place on the given stream); all are float32 except where noted.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MACE_DEBUG=1: the build with device-side bounds checks (build(debug=True))
LIB_PATH = os.path.join(HERE, "libmace_debug.so" if os.environ.get("MACE_DEBUG") == "1" else "libmace.so")

MACE_OK = 0
MACE_EINVAL = -1
MACE_ENOMEM = -2
MACE_ECUDA = -3
MACE_ENOTCONVERGED = -4
MACE_ETIMEOUT = -5
MACE_ENUMERIC = -6

DTYPES = {"f32": 0, "bf16": 1, "f16": 2}

# every symbol include/mace.h declares
EXPORTS = [
    "mace_build_sysmatrix", "mace_sysmatrix_get_info", "mace_sysmatrix_column",
    "mace_get_visit_order",
    "mace_init", "mace_iterate", "mace_launch", "mace_poll", "mace_poll_async", "mace_poll_ready",
    "mace_reconstruct", "mace_consensus",
    "mace_set_timing", "mace_get_timing", "mace_wait_selftest", "mace_consensus_noalloc", "mace_state_bytes",
    "mace_get_state", "mace_set_state", "mace_prox_pass", "mace_get_error",
    "mace_error_size", "mace_recompute_error", "mace_get_stats",
    "mace_free_state", "mace_free_sysmatrix", "mace_last_error",
    "mace_group_create", "mace_group_update", "mace_group_launch", "mace_group_free", "mace_get_launch_info",
]


class MaceError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_views", ctypes.c_int32), ("n_channels", ctypes.c_int32),
                ("pixel_pitch", ctypes.c_double), ("channel_pitch", ctypes.c_double),
                ("channel_offset", ctypes.c_double), ("view_angles", ctypes.c_void_p)]


class Partition(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int32), ("view_agent", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("prior", ctypes.c_int32), ("neighbourhood", ctypes.c_int32),
                ("beta", ctypes.c_double), ("sigma_x", ctypes.c_double),
                ("p", ctypes.c_double), ("q", ctypes.c_double), ("T", ctypes.c_double),
                ("sigma", ctypes.c_double), ("sigma_mode", ctypes.c_int32),
                ("rho", ctypes.c_double), ("sweeps_per_iter", ctypes.c_int32),
                ("symmetric", ctypes.c_int32), ("recompute_every", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("concurrency", ctypes.c_int32), ("sv_order", ctypes.c_int32),
                ("chains", ctypes.c_int32), ("pnp", ctypes.c_int32),
                ("forward_geometry", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("warps_per_voxel", ctypes.c_int32)]


class SysmatrixInfo(ctypes.Structure):
    _fields_ = [("n_voxels", ctypes.c_int64), ("n_agents", ctypes.c_int32),
                ("sv_size", ctypes.c_int32), ("n_sv", ctypes.c_int32),
                ("max_views", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("bytes_columns", ctypes.c_int64), ("bytes_meta", ctypes.c_int64),
                ("agent_bytes", ctypes.c_int64 * 64)]


_lib = None


def load(path=LIB_PATH):
    """Load libmace.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmace.so is not built: run paper_1911_09278_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.mace_build_sysmatrix.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Partition), i32, i32, vp, pp]
    L.mace_sysmatrix_get_info.argtypes = [vp, ctypes.POINTER(SysmatrixInfo)]
    L.mace_sysmatrix_column.argtypes = [vp, i32, i32, i32, vp, vp, vp]
    L.mace_get_visit_order.argtypes = [vp, vp]
    L.mace_init.argtypes = [vp, i32, vp, vp, i32, ctypes.POINTER(Params), vp, vp, pp]
    L.mace_iterate.argtypes = [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    L.mace_state_bytes.argtypes = [vp, i32, ctypes.POINTER(Params), i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.mace_state_bytes.restype = ctypes.c_int
    L.mace_launch.argtypes = [vp, i32]
    L.mace_poll.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    L.mace_poll_async.argtypes = [vp]
    L.mace_poll_ready.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.mace_set_timing.argtypes = [vp, i32, i32]
    L.mace_wait_selftest.argtypes = [ctypes.c_uint32, vp]
    L.mace_consensus_noalloc.argtypes = [vp, vp, i32]
    L.mace_get_timing.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    L.mace_reconstruct.argtypes = [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    L.mace_consensus.argtypes = [vp, vp, i32]
    L.mace_get_state.argtypes = [vp, vp, vp, i32]
    L.mace_set_state.argtypes = [vp, vp, vp, i32]
    L.mace_prox_pass.argtypes = [vp, vp, i32, i32]
    L.mace_get_error.argtypes = [vp, vp, i32]
    L.mace_error_size.argtypes = [vp]
    L.mace_error_size.restype = i64
    L.mace_recompute_error.argtypes = [vp]
    L.mace_get_stats.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                 ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.mace_free_state.argtypes = [vp]
    L.mace_free_state.restype = None
    L.mace_free_sysmatrix.argtypes = [vp]
    L.mace_free_sysmatrix.restype = None
    L.mace_last_error.restype = ctypes.c_char_p
    L.mace_group_create.argtypes = [ctypes.POINTER(vp), i32, vp, pp]
    L.mace_group_update.argtypes = [vp, ctypes.POINTER(vp), i32]
    L.mace_get_launch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.mace_group_launch.argtypes = [vp, i32]
    L.mace_group_free.argtypes = [vp]
    for name in ("mace_build_sysmatrix", "mace_sysmatrix_get_info", "mace_sysmatrix_column",
                 "mace_get_visit_order",
                 "mace_init", "mace_iterate", "mace_launch", "mace_poll", "mace_poll_async", "mace_poll_ready",
                 "mace_reconstruct", "mace_consensus",
                 "mace_set_timing", "mace_get_timing",
                 "mace_get_state", "mace_set_state", "mace_prox_pass", "mace_get_error",
                 "mace_recompute_error", "mace_get_stats",
                 "mace_group_create", "mace_group_update", "mace_group_launch", "mace_group_free",
                 "mace_get_launch_info"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc, allow=()):
    if rc != MACE_OK and rc not in allow:
        raise MaceError(rc, load().mace_last_error().decode())
    return rc


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _in_ptr(a, n=None):
    """(pointer, ptr_is_device, keepalive) for a float32 input array."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("torch inputs must be contiguous float32")
        if n is not None and a.numel() != n:
            raise ValueError("expected %d elements, got %d" % (n, a.numel()))
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and arr.size != n:
        raise ValueError("expected %d elements, got %d" % (n, arr.size))
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Sysmatrix:
    """Handle of a stored system matrix (mace_build_sysmatrix)."""

    def __init__(self, handle, nx, ny, n_views, n_channels, n_agents, view_agent, dtype, sv_size):
        self.handle = handle
        self.nx, self.ny, self.n_views, self.n_channels = nx, ny, n_views, n_channels
        self.n_agents, self.view_agent, self.dtype, self.sv_size = n_agents, view_agent, dtype, sv_size

    def info(self):
        inf = SysmatrixInfo()
        _check(load().mace_sysmatrix_get_info(self.handle, ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in SysmatrixInfo._fields_ if k != "agent_bytes"}
        d["agent_bytes"] = list(inf.agent_bytes[:min(64, self.n_agents)])
        return d

    def agent_views(self, g):
        return np.nonzero(self.view_agent == g)[0]

    def column(self, g, i, j):
        """Decoded column of pixel (i, j) for agent g: (c0, len, vals[V, 3])."""
        V = int((self.view_agent == g).sum())
        c0 = np.zeros(V, np.int32)
        ln = np.zeros(V, np.int32)
        vals = np.zeros((V, 3), np.float32)
        _check(load().mace_sysmatrix_column(self.handle, g, i, j, c0.ctypes.data_as(ctypes.c_void_p),
                                            ln.ctypes.data_as(ctypes.c_void_p),
                                            vals.ctypes.data_as(ctypes.c_void_p)))
        return c0, ln, vals

    def close(self):
        if self.handle:
            load().mace_free_sysmatrix(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mace_build_sysmatrix(nx, ny, n_views, n_channels, n_agents, view_agent=None, dtype="f32",
                         sv_size=8, stream=None, pixel_pitch=1.0, channel_pitch=1.0,
                         channel_offset=0.0, view_angles=None, nz=1):
    L = load()
    va = (np.arange(n_views) % n_agents).astype(np.int32) if view_agent is None \
        else np.ascontiguousarray(view_agent, dtype=np.int32)
    ang = None if view_angles is None else np.ascontiguousarray(view_angles, dtype=np.float64)
    geom = Geometry(nx, ny, nz, n_views, n_channels, pixel_pitch, channel_pitch, channel_offset,
                    None if ang is None else ang.ctypes.data_as(ctypes.c_void_p))
    part = Partition(n_agents, va.ctypes.data_as(ctypes.c_void_p))
    h = ctypes.c_void_p()
    _check(L.mace_build_sysmatrix(ctypes.byref(geom), ctypes.byref(part), DTYPES[dtype], sv_size,
                                  _stream_handle(stream), ctypes.byref(h)))
    return Sysmatrix(h, nx, ny, n_views, n_channels, n_agents, va, dtype, sv_size)


def make_params(prior="qggmrf", beta=1.0, sigma_x=1.0, p=2.0, q=1.2, T=1.0, sigma=0.1,
                sigma_mode=1, rho=0.8, sweeps_per_iter=1, symmetric=False, recompute_every=0,
                max_iter=1000, tol=1e-5, concurrency=0, neighbourhood=8, sv_order=0, chains=0, pnp=False,
                forward_geometry=None, deterministic=False, schedule=0, warps_per_voxel=0):
    """forward_geometry: None = the library's default (the geometry-evaluated
    e recompute for BF16/FP16 stored values), True = always from the
    geometry, False = always from the stored values.  schedule: 0 = fixed
    warps per (reconstruction, agent) pair, 1 = a persistent grid fed from
    a work queue.  warps_per_voxel: warps sweeping one super-voxel together
    (schedule 1; 0 = automatic by views per agent)."""
    return Params(0 if prior == "quadratic" else 1, neighbourhood, beta, sigma_x, p, q, T, sigma,
                  sigma_mode, rho, sweeps_per_iter, int(bool(symmetric)), recompute_every,
                  max_iter, tol, concurrency, sv_order, chains, int(bool(pnp)),
                  0 if forward_geometry is None else (1 if forward_geometry else 2), int(bool(deterministic)),
                  int(schedule), int(warps_per_voxel))


class State:
    """Handle of a reconstruction state (mace_init) holding `batch`
    reconstructions that share one system matrix."""

    def __init__(self, handle, sm, params, batch):
        self.handle = handle
        self.sm = sm            # the state borrows the system matrix
        self.params = params
        self.batch = batch
        self.n = sm.nx * sm.ny

    def _img_shape(self):
        return (self.sm.ny, self.sm.nx) if self.batch == 1 else (self.batch, self.sm.ny, self.sm.nx)

    def iterate(self, n_iters):
        r = ctypes.c_double()
        c = ctypes.c_int32()
        _check(load().mace_iterate(self.handle, n_iters, ctypes.byref(r), ctypes.byref(c)))
        return r.value, bool(c.value)

    def launch(self, n_iters):
        """Enqueue n_iters iterations on the state's stream (no wait)."""
        _check(load().mace_launch(self.handle, n_iters))

    def poll(self):
        r = ctypes.c_double()
        c = ctypes.c_int32()
        _check(load().mace_poll(self.handle, ctypes.byref(r), ctypes.byref(c)))
        return r.value, bool(c.value)

    def poll_async(self):
        """Enqueue a copy of the current status (returns at once)."""
        _check(load().mace_poll_async(self.handle))

    def poll_ready(self):
        """(ready, residual, converged) of the last poll_async, without waiting."""
        r = ctypes.c_double()
        c = ctypes.c_int32()
        ok = ctypes.c_int32()
        _check(load().mace_poll_ready(self.handle, ctypes.byref(r), ctypes.byref(c), ctypes.byref(ok)))
        return bool(ok.value), r.value, bool(c.value)

    def set_timing(self, enable=True, max_launches=4096):
        _check(load().mace_set_timing(self.handle, int(bool(enable)), max_launches))

    def get_timing(self):
        """(summed sweep-kernel device ms, launches) since set_timing / last call."""
        ms = ctypes.c_double()
        n = ctypes.c_int32()
        _check(load().mace_get_timing(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def reconstruct(self, out=None):
        """Iterate to tol / max_iter; returns (x, iters, residual, converged)."""
        x = np.empty(self._img_shape(), np.float32) if out is None else out
        ptr, dev, keep = _out_ptr(x, self.batch * self.n)
        it = ctypes.c_int32()
        r = ctypes.c_double()
        rc = _check(load().mace_reconstruct(self.handle, ptr, dev, ctypes.byref(it), ctypes.byref(r)),
                    allow=(MACE_ENOTCONVERGED,))
        return x, it.value, r.value, rc == MACE_OK

    def consensus(self, out=None):
        x = np.empty(self._img_shape(), np.float32) if out is None else out
        ptr, dev, keep = _out_ptr(x, self.batch * self.n)
        _check(load().mace_consensus(self.handle, ptr, dev))
        return x

    def consensus_noalloc(self, out=None):
        """mace_consensus through the library's fixed device array (no
        allocation); see include/mace.h for its limits."""
        x = np.empty(self._img_shape(), np.float32) if out is None else out
        ptr, dev, keep = _out_ptr(x, self.batch * self.n)
        _check(load().mace_consensus_noalloc(self.handle, ptr, dev))
        return x

    def get_state(self):
        N = self.sm.n_agents
        shape = (N, self.n) if self.batch == 1 else (self.batch, N, self.n)
        w = np.empty(shape, np.float32)
        X = np.empty(shape, np.float32)
        _check(load().mace_get_state(self.handle, w.ctypes.data_as(ctypes.c_void_p),
                                     X.ctypes.data_as(ctypes.c_void_p), 0))
        return w, X

    def set_state(self, w, X):
        N = self.sm.n_agents
        pw, dw, kw = _in_ptr(w, self.batch * N * self.n)
        px, dx, kx = _in_ptr(X, self.batch * N * self.n)
        if dw != dx:
            raise ValueError("w and X must both be host or both be device arrays")
        _check(load().mace_set_state(self.handle, pw, px, dw))

    def prox_pass(self, v, backward=False):
        pv, dv, kv = _in_ptr(v, self.batch * self.sm.n_agents * self.n)
        _check(load().mace_prox_pass(self.handle, pv, dv, int(bool(backward))))

    def visit_order(self):
        """Pixel visiting order of a forward ICD pass (raster indices)."""
        o = np.empty(self.n, np.int64)
        _check(load().mace_get_visit_order(self.handle, o.ctypes.data_as(ctypes.c_void_p)))
        return o

    def error(self):
        ne = load().mace_error_size(self.handle)
        e = np.empty(ne, np.float32)
        _check(load().mace_get_error(self.handle, e.ctypes.data_as(ctypes.c_void_p), 0))
        return e

    def recompute_error(self):
        _check(load().mace_recompute_error(self.handle))

    def stats(self):
        it = ctypes.c_int32()
        s = ctypes.c_double()
        r = ctypes.c_double()
        c = ctypes.c_int32()
        k = ctypes.c_int32()
        _check(load().mace_get_stats(self.handle, ctypes.byref(it), ctypes.byref(s), ctypes.byref(r),
                                     ctypes.byref(c), ctypes.byref(k)))
        sc, wpv, nw = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().mace_get_launch_info(self.handle, ctypes.byref(sc), ctypes.byref(wpv), ctypes.byref(nw)))
        return dict(iters=it.value, sigma_abs=s.value, last_residual=r.value, concurrency=c.value,
                    chains=k.value, schedule=sc.value, warps_per_voxel=wpv.value, warps=nw.value)

    def close(self):
        if self.handle:
            load().mace_free_state(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _out_ptr(a, n):
    if _is_torch(a):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n:
            raise ValueError("output tensor must be contiguous float32 with %d elements" % n)
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != n:
        raise ValueError("output array must be contiguous float32 with %d elements" % n)
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def mace_state_bytes(sm, params, batch=1, inputs_on_device=False):
    """(persistent, peak) device bytes of a state mace_init would create."""
    p = ctypes.c_int64()
    q = ctypes.c_int64()
    _check(load().mace_state_bytes(sm.handle, batch, ctypes.byref(params), int(bool(inputs_on_device)),
                                   ctypes.byref(p), ctypes.byref(q)))
    return p.value, q.value


def mace_init(sm, y, weights, params, w0=None, stream=None, batch=None):
    """y, weights: [batch][n_views][n_channels] (or [n_views][n_channels] for
    one reconstruction)."""
    m = sm.n_views * sm.n_channels
    if batch is None:
        size = y.numel() if _is_torch(y) else np.asarray(y).size
        batch = max(1, size // m)
    py, dy, ky = _in_ptr(y, batch * m)
    pl, dl, kl = _in_ptr(weights, batch * m)
    if dy != dl:
        raise ValueError("y and weights must both be host or both be device arrays")
    pw, dw, kw = _in_ptr(w0, batch * sm.n_agents * sm.nx * sm.ny)
    if w0 is not None and dw != dy:
        raise ValueError("w0 must live where y does")
    h = ctypes.c_void_p()
    _check(load().mace_init(sm.handle, batch, py, pl, dy, ctypes.byref(params), pw, _stream_handle(stream),
                            ctypes.byref(h)))
    return State(h, sm, params, batch)


class Group:
    """Several states advanced together (mace_group_create): their ICD
    passes share one queue-fed launch per pass.  The members are borrowed
    and must outlive the group."""

    def __init__(self, states, stream=None):
        self.states = list(states)
        arr = (ctypes.c_void_p * len(self.states))(*[st.handle for st in self.states])
        h = ctypes.c_void_p()
        _check(load().mace_group_create(arr, len(self.states), _stream_handle(stream), ctypes.byref(h)))
        self.handle = h

    def update(self, states):
        """Replace the members (stream-ordered; no wait)."""
        states = list(states)
        arr = (ctypes.c_void_p * len(states))(*[st.handle for st in states])
        _check(load().mace_group_update(self.handle, arr, len(states)))
        self.states = states

    def launch(self, n_iters):
        """Enqueue n_iters Mann iterations of every member (no wait)."""
        _check(load().mace_group_launch(self.handle, n_iters))

    def close(self):
        if self.handle:
            load().mace_group_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mace_group_create(states, stream=None):
    return Group(states, stream=stream)


def mace_wait_selftest(spin_limit=1000, stream=None):
    """Run the bounded-wait self test; returns the MACE code (expect MACE_ETIMEOUT)."""
    rc = load().mace_wait_selftest(spin_limit, _stream_handle(stream))
    return rc


def mace_iterate(state, n_iters):
    return state.iterate(n_iters)


def mace_reconstruct(state, out=None):
    return state.reconstruct(out)
