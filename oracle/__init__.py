"""FP64 CPU oracle for partial-update MACE (arXiv 1911.09278).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this package.  It shares no code with the CUDA library.

What it computes (all in double precision, C in ``mace_oracle.c``):

* ``footprint`` / ``dense_A`` -- the stored system matrix A_k of Sec. II-A,
  read as the parallel-beam strip integral of a square pixel (the paper cites
  but does not define its projector; see the C header).
* ``icd_sweep`` -- one pass of Algorithm 2 (ICD partial update of the proximal
  map F_i of Eq. "prox_F"), any voxel order.
* ``mace`` -- Algorithm 1 (partial-update MACE), or exact MACE when the inner
  loop is run to convergence (Eq. "Mann" with exact F).
* ``central_icd`` -- centralised MAP by ICD (the single-node method, Sec. IV-A).
* ``cost`` / ``gradient`` -- the MAP cost of Eq. "global_obj" and its gradient
  (KKT check of the converged image).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("n_views", ctypes.c_int32), ("n_channels", ctypes.c_int32),
        ("pixel_pitch", ctypes.c_double), ("channel_pitch", ctypes.c_double),
        ("channel_offset", ctypes.c_double),
        ("cos_t", ctypes.c_void_p), ("sin_t", ctypes.c_void_p),
        ("y", ctypes.c_void_p), ("lam", ctypes.c_void_p),
        ("n_agents", ctypes.c_int32), ("view_agent", ctypes.c_void_p),
        ("prior", ctypes.c_int32), ("neighbourhood", ctypes.c_int32),
        ("beta", ctypes.c_double), ("sigma_x", ctypes.c_double),
        ("p", ctypes.c_double), ("q", ctypes.c_double), ("T", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(_Problem)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.or_version.restype = ctypes.c_int
        L.or_angles.argtypes = [i32, vp, vp]
        L.or_footprint.argtypes = [P, i32, i32, i32, vp, vp]
        L.or_footprint.restype = i32
        L.or_dense_A.argtypes = [P, vp]
        L.or_agent_views.argtypes = [P, i32, vp]
        L.or_agent_views.restype = i32
        L.or_error_sinogram.argtypes = [P, i32, vp, vp]
        L.or_theta2.argtypes = [P, i32, vp]
        L.or_icd_sweep.argtypes = [P, i32, i32, dbl, dbl, vp, vp, vp, vp]
        L.or_icd_sweep.restype = dbl
        L.or_cost.argtypes = [P, vp]
        L.or_cost.restype = dbl
        L.or_gradient.argtypes = [P, vp, vp]
        L.or_central_icd.argtypes = [P, vp, i32, dbl, vp, vp]
        L.or_central_icd.restype = i32
        L.or_mace.argtypes = [P, dbl, dbl, i32, i32, dbl, i32, dbl, vp, i32,
                              vp, vp, vp, vp, vp, i32, vp, vp]
        L.or_mace.restype = i32
        L.or_prior_prox.argtypes = [P, dbl, vp, vp, i32, dbl]
        L.or_prior_prox.restype = i32
        L.or_pnp_mace.argtypes = [P, dbl, dbl, i32, i32, i32, dbl, vp, i32, dbl,
                                  vp, vp, vp, vp, vp, i32]
        L.or_pnp_mace.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def angles(n_views):
    """cos/sin of theta_m = m pi / N_theta (views uniform over 180 degrees)."""
    c = np.empty(n_views, np.float64)
    s = np.empty(n_views, np.float64)
    lib().or_angles(n_views, _ptr(c), _ptr(s))
    return c, s


class Problem:
    """The reconstruction problem: geometry, data (y, Lambda), partition J_i
    and prior.  Arrays are kept alive for the lifetime of the object.

    y and lam are [nz][n_views][n_channels]; view_agent[m] is the agent that
    owns view m (interleaved subsets: m mod N)."""

    def __init__(self, nx, ny, n_views, n_channels, y, lam, n_agents=1,
                 view_agent=None, nz=1, prior="quadratic", neighbourhood=None,
                 beta=1.0, sigma_x=1.0, p=2.0, q=1.2, T=1.0,
                 pixel_pitch=1.0, channel_pitch=1.0, channel_offset=0.0,
                 view_angles=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n_views, self.n_channels = int(n_views), int(n_channels)
        self.n = self.nx * self.ny * self.nz
        if view_angles is None:
            self.cos_t, self.sin_t = angles(self.n_views)
        else:
            th = _f64(view_angles)
            self.cos_t, self.sin_t = _f64(np.cos(th)), _f64(np.sin(th))
        shape = (self.nz, self.n_views, self.n_channels)
        self.y = _f64(y).reshape(shape)
        self.lam = _f64(lam).reshape(shape)
        self.n_agents = int(n_agents)
        if view_agent is None:
            view_agent = np.arange(self.n_views) % self.n_agents
        self.view_agent = np.ascontiguousarray(view_agent, dtype=np.int32)
        if neighbourhood is None:
            neighbourhood = 8 if self.nz == 1 else 26
        if float(p) != 2.0:
            raise ValueError("the oracle implements the p = 2 Q-GGMRF only")
        self.prior_name = prior
        self._s = _Problem(
            self.nx, self.ny, self.nz, self.n_views, self.n_channels,
            float(pixel_pitch), float(channel_pitch), float(channel_offset),
            _ptr(self.cos_t), _ptr(self.sin_t), _ptr(self.y), _ptr(self.lam),
            self.n_agents, _ptr(self.view_agent),
            0 if prior == "quadratic" else 1, int(neighbourhood),
            float(beta), float(sigma_x), float(p), float(q), float(T))

    @property
    def ref(self):
        return ctypes.byref(self._s)

    # -- system matrix ----------------------------------------------------
    def footprint(self, m, i, j):
        """(first channel, values) of pixel (row i, col j) in view m."""
        c0 = np.zeros(1, np.int32)
        v = np.zeros(3, np.float64)
        L = lib().or_footprint(self.ref, m, i, j, _ptr(c0), _ptr(v))
        return int(c0[0]), v[:L].copy()

    def dense_A(self):
        """Dense A of one slice: [n_views * n_channels, nx * ny]."""
        out = np.empty((self.n_views * self.n_channels, self.nx * self.ny), np.float64)
        lib().or_dense_A(self.ref, _ptr(out))
        return out

    def agent_views(self, g):
        v = np.empty(self.n_views, np.int32)
        cnt = lib().or_agent_views(self.ref, g, _ptr(v))
        return v[:cnt].copy()

    # -- per-agent quantities ---------------------------------------------
    def error_sinogram(self, g, x):
        V = self.n_views if g < 0 else len(self.agent_views(g))
        e = np.empty((self.nz, V, self.n_channels), np.float64)
        lib().or_error_sinogram(self.ref, g, _ptr(_f64(x)), _ptr(e))
        return e

    def theta2(self, g):
        out = np.empty(self.n, np.float64)
        lib().or_theta2(self.ref, g, _ptr(out))
        return out

    def icd_sweep(self, g, x, e, v=None, sigma=1.0, pscale=None, order=None):
        """One ICD pass (Algorithm 2) in place on x, e; returns sum alpha^2.
        v is None: plain ICD on the cost (no proximal term)."""
        assert x.dtype == np.float64 and x.flags.c_contiguous
        assert e.dtype == np.float64 and e.flags.c_contiguous
        if pscale is None:
            pscale = self._s.beta / (self.n_agents if g >= 0 else 1)
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        vv = None if v is None else _f64(v)
        return lib().or_icd_sweep(self.ref, g, 0 if v is None else 1, float(sigma),
                                  float(pscale), _ptr(o), _ptr(vv), _ptr(x), _ptr(e))

    # -- cost ---------------------------------------------------------------
    def cost(self, x):
        return lib().or_cost(self.ref, _ptr(_f64(x)))

    def gradient(self, x):
        g = np.empty(self.n, np.float64)
        lib().or_gradient(self.ref, _ptr(_f64(x)), _ptr(g))
        return g

    # -- solvers --------------------------------------------------------------
    def central_icd(self, x0=None, max_sweeps=1000, tol=1e-12, order=None):
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        r = np.zeros(1)
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        it = lib().or_central_icd(self.ref, _ptr(x), int(max_sweeps), float(tol), _ptr(o), _ptr(r))
        return x, int(it), float(r[0])

    def mace(self, sigma, rho=0.8, sweeps=1, max_iter=1000, tol=1e-10, w0=None,
             X0=None, order=None, inner_tol=0.0, n_threads=0, symmetric=False,
             xref=None):
        """Algorithm 1.  Returns dict(x, w, X, iters, resid, hist)."""
        N, n = self.n_agents, self.n
        w = np.zeros((N, n)) if w0 is None else _f64(w0).reshape(N, n).copy()
        X = np.zeros((N, n)) if X0 is None else _f64(X0).reshape(N, n).copy()
        xbar = np.empty(n)
        hist = np.zeros(max(int(max_iter), 1))
        r = np.zeros(1)
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        xr = None if xref is None else _f64(xref)
        nh = np.zeros_like(hist)
        it = lib().or_mace(self.ref, float(sigma), float(rho), int(sweeps), int(bool(symmetric)), float(inner_tol),
                           int(max_iter), float(tol), _ptr(o), 1 if X0 is None else 0,
                           _ptr(w), _ptr(X), _ptr(xbar), _ptr(hist), _ptr(r), int(n_threads),
                           _ptr(xr), _ptr(nh))
        if it < 0:
            raise ValueError("or_mace failed: %d" % it)
        return dict(x=xbar, w=w, X=X, iters=int(it), resid=float(r[0]), hist=hist[:it].copy(),
                    nrmse_hist=nh[:it].copy() if xref is not None else None)


    def prior_prox(self, v, sigma, tol=1e-14, max_pass=100000):
        """H(v) = argmin_z beta h(z) + ||z - v||^2 / (2 sigma^2) (Gauss-Seidel to tol)."""
        v = _f64(v).ravel()
        x = np.empty_like(v)
        lib().or_prior_prox(self.ref, float(sigma), _ptr(v), _ptr(x), int(max_pass), float(tol))
        return x

    def pnp_mace(self, sigma, rho=0.8, sweeps=1, max_iter=1000, tol=1e-10, w0=None, X0=None,
                 order=None, n_threads=0, symmetric=False, h_tol=1e-14):
        """Algorithm 3 (partial-update MACE with the prior's proximal map as
        the plug-and-play denoiser).  Returns dict(x, w, X, iters, resid, hist)."""
        N, n = self.n_agents, self.n
        w = np.zeros((N, n)) if w0 is None else _f64(w0).reshape(N, n).copy()
        X = np.zeros((N, n)) if X0 is None else _f64(X0).reshape(N, n).copy()
        xs = np.empty(n)
        hist = np.zeros(max(int(max_iter), 1))
        r = np.zeros(1)
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        it = lib().or_pnp_mace(self.ref, float(sigma), float(rho), int(sweeps), int(bool(symmetric)),
                               int(max_iter), float(tol), _ptr(o), 1 if X0 is None else 0, float(h_tol),
                               _ptr(w), _ptr(X), _ptr(xs), _ptr(hist), _ptr(r), int(n_threads))
        if it < 0:
            raise ValueError("or_pnp_mace failed: %d" % it)
        return dict(x=xs, w=w, X=X, iters=int(it), resid=float(r[0]), hist=hist[:it].copy())


def mean_theta2(problem):
    """Mean over agents and voxels of the data-Hessian diagonal of f_i."""
    return float(np.mean([problem.theta2(g).mean() for g in range(problem.n_agents)]))
