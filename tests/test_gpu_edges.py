"""Edge cases of the CUDA path against the oracle: a ragged, non-square
image with an uneven view partition; a single agent; a detector offset so
that pixels near the centre have empty columns; zero weights (dead
channels and a dropped view); the size limits of the geometry."""
import functools

import numpy as np
import pytest

import oracle
import synth
from helpers import nrmse

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def edge_case(name):
    if name == "ragged":        # 45 x 38 pixels: neither side a multiple of 8
        nx, ny, V, D, N, prior, off = 45, 38, 40, 61, 3, "qggmrf", 0.0
        va = synth.uneven_partition(7, V, N, 10, 16)
    elif name == "one_agent":
        nx, ny, V, D, N, prior, off = 40, 40, 36, 57, 1, "quadratic", 0.0
        va = None
    elif name == "offset":      # detector covers t in [2, 22]: central pixels miss every view
        nx, ny, V, D, N, prior, off = 32, 32, 30, 20, 2, "quadratic", 12.0
        va = None
    else:                       # "dead": zero weights on a channel band and on one view
        nx, ny, V, D, N, prior, off = 48, 48, 40, 69, 4, "qggmrf", 0.0
        va = None
    m = min(nx, ny)
    E = synth.ellipses(31, m, 0.02 * 64 / m)
    p = synth.sinogram(E, V, D, channel_offset=off)
    y, lam = synth.measurements(p, 2e4, synth.CounterRNG(131))
    if name == "dead":
        lam[:, 30:36] = 0.0
        lam[7, :] = 0.0
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    P = oracle.Problem(nx, ny, V, D, y, lam, n_agents=N, view_agent=va, prior=prior, sigma_x=sx,
                       channel_offset=off)
    xs, it, r = P.central_icd(max_sweeps=40000, tol=1e-13)
    g0 = np.linalg.norm(P.gradient(np.zeros(P.n)))
    assert np.linalg.norm(P.gradient(xs)) / g0 < 1e-9
    return dict(nx=nx, ny=ny, V=V, D=D, N=N, prior=prior, off=off, va=va, y=y, lam=lam, sx=sx, P=P, xs=xs)


def _sysmatrix(mace, c):
    return mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], c["N"], view_agent=c["va"],
                                     channel_offset=c["off"], sv_size=8)


@pytest.mark.parametrize("name", ["ragged", "one_agent", "offset", "dead"])
def test_edge_converges_to_map(gpu_lib, name):
    mace = gpu_lib
    c = edge_case(name)
    sm = _sysmatrix(mace, c)
    prm = mace.make_params(prior=c["prior"], sigma_x=c["sx"], sigma=0.5, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, recompute_every=10, tol=2e-8, max_iter=8000, concurrency=1)
    st = mace.mace_init(sm, c["y"], c["lam"], prm)
    x, iters, r, conv = st.reconstruct()
    st.close()
    sm.close()
    err = nrmse(x, c["xs"])
    print("%s: iters=%d r=%.2e nrmse=%.2e" % (name, iters, r, err))
    assert err < 1e-4


@pytest.mark.parametrize("name", ["ragged", "offset"])
def test_edge_one_pass_matches_algorithm2(gpu_lib, name):
    mace = gpu_lib
    c = edge_case(name)
    P, N, n = c["P"], c["N"], c["nx"] * c["ny"]
    sm = _sysmatrix(mace, c)
    rng = np.random.default_rng(2)
    xs = c["xs"]
    X0 = (xs[None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((N, n))).astype(np.float32)
    v = (xs[None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((N, n))).astype(np.float32)
    prm = mace.make_params(prior=c["prior"], sigma_x=c["sx"], sigma=0.5, sigma_mode=1, concurrency=1)
    st = mace.mace_init(sm, c["y"], c["lam"], prm)
    st.set_state(X0.copy(), X0)
    st.prox_pass(v)
    _, Xg = st.get_state()
    sigma = st.stats()["sigma_abs"]
    order = st.visit_order()
    st.close()
    sm.close()
    for g in range(N):
        x = X0[g].astype(np.float64)
        e = P.error_sinogram(g, x)
        P.icd_sweep(g, x, e, v=v[g].astype(np.float64), sigma=sigma, order=order)
        assert nrmse(Xg.reshape(N, n)[g], x) < 2e-5, g


def test_offset_detector_has_empty_columns(gpu_lib):
    """The central pixel misses every view: its stored column is empty."""
    mace = gpu_lib
    c = edge_case("offset")
    sm = _sysmatrix(mace, c)
    for g in range(c["N"]):
        c0, ln, vals = sm.column(g, 16, 16)
        assert int(np.sum(ln)) == 0
        assert sum(len(c["P"].footprint(int(m), 16, 16)[1]) for m in c["P"].agent_views(g)) == 0
    sm.close()


def test_geometry_limits(gpu_lib):
    mace = gpu_lib
    with pytest.raises(mace.MaceError) as ei:
        mace.mace_build_sysmatrix(16, 16, 4097, 23, 1)
    assert ei.value.code == mace.MACE_EINVAL
    with pytest.raises(mace.MaceError) as ei:
        mace.mace_build_sysmatrix(16, 16, 8, 65536, 1)
    assert ei.value.code == mace.MACE_EINVAL
    with pytest.raises(mace.MaceError) as ei:
        mace.mace_build_sysmatrix(16, 16, 0, 23, 1)
    assert ei.value.code == mace.MACE_EINVAL


@pytest.mark.parametrize("chains", [1, 2])
def test_many_views_per_agent(gpu_lib, chains):
    """Agents with more views than four rounds of lanes (here 150 views per
    agent) run the sweep variant that decodes each column as it is used: one
    pass at concurrency 1 equals Algorithm 2 in the library's order, and the
    converged image equals the oracle's MAP image (relative RMSE 1e-4)."""
    mace = gpu_lib
    n, V, D, N = 40, 300, 59, 2
    E = synth.ellipses(37, n, 0.02 * 64 / n)
    p = synth.sinogram(E, V, D)
    y, lam = synth.measurements(p, 2e4, synth.CounterRNG(137))
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=N, prior="qggmrf", sigma_x=sx)
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, sv_size=4)
    batch = chains
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=0.5, sigma_mode=1, concurrency=1, chains=chains)
    st = mace.mace_init(sm, np.stack([y] * batch), np.stack([lam] * batch), prm, batch=batch)
    assert st.stats()["chains"] == chains
    rng = np.random.default_rng(3)
    xs, _, _ = P.central_icd(max_sweeps=20000, tol=1e-13)
    X0 = (xs[None, None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((batch, N, n * n))).astype(np.float32)
    v = (xs[None, None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((batch, N, n * n))).astype(np.float32)
    st.set_state(X0.copy(), X0.copy())
    st.prox_pass(v)
    _, Xg = st.get_state()
    Xg = Xg.reshape(batch, N, n * n)
    sigma = st.stats()["sigma_abs"]
    order = st.visit_order()
    for b in range(batch):
        for g in range(N):
            x = X0[b, g].astype(np.float64)
            e = P.error_sinogram(g, x)
            P.icd_sweep(g, x, e, v=v[b, g].astype(np.float64), sigma=sigma, order=order)
            assert nrmse(Xg[b, g], x) < 2e-5, (b, g)
    st.close()
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=0.5, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, recompute_every=10, max_iter=4000, tol=1e-7, concurrency=4, chains=chains)
    st = mace.mace_init(sm, np.stack([y] * batch), np.stack([lam] * batch), prm, batch=batch)
    x, iters, r, conv = st.reconstruct()
    st.close()
    sm.close()
    assert conv
    for b in range(batch):
        err = nrmse(np.asarray(x).reshape(batch, -1)[b], xs)
        print("150 views per agent, chains %d: iters %d, NRMSE vs oracle %.2e" % (chains, iters, err))
        assert err < 1e-4


def test_state_bytes_matches_device_usage(gpu_lib):
    """mace_state_bytes (the server's admission count) against the device
    memory mace_init actually takes (cudaMemGetInfo around it): the
    persistent bytes, up to the allocator's rounding."""
    import torch
    mace = gpu_lib
    n, V, D, N, B = 256, 360, 363, 16, 2
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, sv_size=4)
    prm = mace.make_params(prior="qggmrf", sigma_x=1.0, sigma=0.1, concurrency=-1, chains=2)
    persistent, peak = mace.mace_state_bytes(sm, prm, batch=B)
    assert peak > persistent > 0
    y = np.ones((B, V, D), np.float32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = mace.mace_init(sm, y, y, prm, batch=B)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    print("state bytes: library %d, measured %d" % (persistent, used))
    assert persistent <= used + (2 << 20)
    assert used <= persistent + (32 << 20)
    st.close()
    sm.close()


@pytest.mark.parametrize("sv", [16, 32])
@pytest.mark.parametrize("schedule", [0, 1])
def test_large_super_voxels_one_pass(gpu_lib, sv, schedule):
    """16 x 16 and 32 x 32 super-voxels (the largest tiles, widest bands):
    one pass at concurrency 1 equals Algorithm 2 for every agent, on the
    fixed grid and on the work queue."""
    mace = gpu_lib
    c = edge_case("ragged")
    P, N, n = c["P"], c["N"], c["nx"] * c["ny"]
    sm = mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], N, view_agent=c["va"], sv_size=sv)
    rng = np.random.default_rng(4)
    xs = c["xs"]
    X0 = (xs[None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((N, n))).astype(np.float32)
    v = (xs[None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((N, n))).astype(np.float32)
    prm = mace.make_params(prior=c["prior"], sigma_x=c["sx"], sigma=0.5, sigma_mode=1, concurrency=1,
                           schedule=schedule)
    st = mace.mace_init(sm, c["y"], c["lam"], prm)
    st.set_state(X0.copy(), X0)
    st.prox_pass(v)
    _, Xg = st.get_state()
    sigma = st.stats()["sigma_abs"]
    order = st.visit_order()
    st.close()
    sm.close()
    for g in range(N):
        x = X0[g].astype(np.float64)
        e = P.error_sinogram(g, x)
        P.icd_sweep(g, x, e, v=v[g].astype(np.float64), sigma=sigma, order=order)
        assert nrmse(Xg.reshape(N, n)[g], x) < 2e-5, g
