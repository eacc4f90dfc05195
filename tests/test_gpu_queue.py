"""The work-queue schedule (params.schedule = 1): a persistent grid of every
resident warp taking (reconstruction, agent, row of super-voxels) items from a
counter.  Checked against the oracle: one pass at concurrency 1 equals
Algorithm 2 for every reconstruction and agent (2D, and a volume whose slices
are swept even ones first, then odd ones); converged images equal the MAP
image (Theorem 1); more pairs than the GPU holds warps still converge."""
import functools

import numpy as np
import pytest

import oracle
import synth
from helpers import nrmse

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def ragged_case(batch):
    """45 x 38 pixels, 40 views over 3 agents of 10-16 views, one scan per
    batch element (different noise draws)."""
    nx, ny, V, D, N = 45, 38, 40, 61, 3
    va = synth.uneven_partition(7, V, N, 10, 16)
    E = synth.ellipses(31, min(nx, ny), 0.02 * 64 / min(nx, ny))
    p = synth.sinogram(E, V, D)
    ys, ls = [], []
    for b in range(batch):
        y, lam = synth.measurements(p, 2e4, synth.CounterRNG(131 + b))
        ys.append(y)
        ls.append(lam)
    y, lam = np.stack(ys), np.stack(ls)
    sx = synth.prior_sigma_x(lam[0], V, frac=1.0)
    probs = [oracle.Problem(nx, ny, V, D, y[b], lam[b], n_agents=N, view_agent=va, prior="qggmrf", sigma_x=sx)
             for b in range(batch)]
    return dict(nx=nx, ny=ny, V=V, D=D, N=N, va=va, y=y, lam=lam, sx=sx, P=probs)


def _map(P):
    xs, _, _ = P.central_icd(max_sweeps=40000, tol=1e-13)
    g0 = np.linalg.norm(P.gradient(np.zeros(P.n)))
    assert np.linalg.norm(P.gradient(xs)) / g0 < 1e-9
    return xs


def test_queue_one_pass_matches_algorithm2(gpu_lib):
    """Concurrency 1: each item is one whole (reconstruction, agent) pair, so
    a pass is Algorithm 2 in the library's order for each of them; an odd
    batch of three different scans checks the item-to-pair mapping."""
    mace = gpu_lib
    B = 3
    c = ragged_case(B)
    N, n = c["N"], c["nx"] * c["ny"]
    sm = mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], N, view_agent=c["va"], sv_size=8)
    rng = np.random.default_rng(5)
    xs = _map(c["P"][0])
    sc = 0.3 * np.abs(xs).mean()
    X0 = (xs[None, None, :] + sc * rng.standard_normal((B, N, n))).astype(np.float32)
    v = (xs[None, None, :] + sc * rng.standard_normal((B, N, n))).astype(np.float32)
    for backward in (0, 1):
        prm = mace.make_params(prior="qggmrf", sigma_x=c["sx"], sigma=0.5, sigma_mode=1, concurrency=1, schedule=1)
        st = mace.mace_init(sm, c["y"], c["lam"], prm, batch=B)
        assert st.stats()["chains"] == 1 and st.stats()["concurrency"] == 1
        st.set_state(X0.copy(), X0)
        st.prox_pass(v, backward=bool(backward))
        _, Xg = st.get_state()
        Xg = Xg.reshape(B, N, n)
        sigma = st.stats()["sigma_abs"]
        order = st.visit_order()
        st.close()
        if backward:
            order = order[::-1].copy()
        for b in range(B):
            P = c["P"][b]
            for g in range(N):
                x = X0[b, g].astype(np.float64)
                e = P.error_sinogram(g, x)
                P.icd_sweep(g, x, e, v=v[b, g].astype(np.float64), sigma=sigma, order=order)
                assert nrmse(Xg[b, g], x) < 2e-5, (backward, b, g)
    sm.close()


def test_queue_converges_to_map_and_agrees_with_fixed(gpu_lib):
    """One item per row of 4x4 super-voxels (concurrency -1): every
    reconstruction of the batch converges to its scan's MAP image, and the
    fixed schedule at the same settings reaches the same image."""
    mace = gpu_lib
    B = 3
    c = ragged_case(B)
    sm = mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], c["N"], view_agent=c["va"], sv_size=4)
    out = {}
    for schedule in (0, 1):
        prm = mace.make_params(prior="qggmrf", sigma_x=c["sx"], sigma=0.2, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                               symmetric=True, recompute_every=10, tol=1e-7, max_iter=8000, concurrency=-1,
                               schedule=schedule)
        st = mace.mace_init(sm, c["y"], c["lam"], prm, batch=B)
        x, iters, r, conv = st.reconstruct()
        stats = st.stats()
        st.close()
        print("schedule %d: converged %s, residual %.2e" % (schedule, conv, r))
        assert conv, schedule
        out[schedule] = np.asarray(x, np.float64).reshape(B, -1)
        print("schedule %d: concurrency %d, iters %d" % (schedule, stats["concurrency"], iters))
    sm.close()
    for b in range(B):
        xs = _map(c["P"][b])
        for schedule in (0, 1):
            assert nrmse(out[schedule][b], xs) < 1e-4, (schedule, b)
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]) < 2e-5


def _volume(nz):
    n, V, D, N = 32, 60, 47, 4
    c = synth.make_volume(n=n, nz=nz, n_views=V, n_channels=D, I0=2e4, mu_max=0.04, seed=4, noise_seed=104)
    va = synth.uneven_partition(204, V, N, 10, 20)
    sx = synth.prior_sigma_x(c["lam"], V, frac=1.0)
    P = oracle.Problem(n, n, V, D, c["y"], c["lam"], n_agents=N, view_agent=va, nz=nz, prior="qggmrf",
                       neighbourhood=26, sigma_x=sx)
    return n, V, D, N, va, sx, c, P


@pytest.mark.parametrize("nz,chains", [(5, 1), (8, 2)])
def test_queue_volume_one_pass_is_zparity_algorithm2(gpu_lib, nz, chains):
    """A volume at concurrency 1: the even slices are swept side by side,
    then the odd ones, each reading neighbour slices that no warp is
    updating, so the pass equals Algorithm 2 over the whole volume in the
    order (even slices, then odd slices, each in the library's in-slice
    order).  With two chains a warp sweeps two slices of one parity (z and
    z + 2) over each column load."""
    mace = gpu_lib
    n, V, D, N, va, sx, c, P = _volume(nz)
    npx = n * n
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, view_agent=va, sv_size=8)
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=0.5, sigma_mode=1, concurrency=1, neighbourhood=26,
                           schedule=1, chains=chains)
    st = mace.mace_init(sm, c["y"], c["lam"], prm, batch=nz)
    assert st.stats()["chains"] == chains
    rng = np.random.default_rng(9)
    xs = _map(P)
    sc = 0.3 * np.abs(xs).mean()
    # state layout [slice][agent][pixel]; the oracle's volume is [slice][pixel]
    X0 = (xs.reshape(nz, 1, npx) + sc * rng.standard_normal((nz, N, npx))).astype(np.float32)
    v = (xs.reshape(nz, 1, npx) + sc * rng.standard_normal((nz, N, npx))).astype(np.float32)
    st.set_state(X0.copy(), X0)
    st.prox_pass(v)
    _, Xg = st.get_state()
    Xg = Xg.reshape(nz, N, npx)
    sigma = st.stats()["sigma_abs"]
    inslice = st.visit_order()
    st.close()
    sm.close()
    order = np.concatenate([z * npx + inslice for z in list(range(0, nz, 2)) + list(range(1, nz, 2))])
    for g in range(N):
        x = np.ascontiguousarray(X0[:, g, :].astype(np.float64).ravel())
        e = P.error_sinogram(g, x)
        P.icd_sweep(g, x, e, v=np.ascontiguousarray(v[:, g, :].astype(np.float64).ravel()), sigma=sigma,
                    order=order)
        assert nrmse(Xg[:, g, :].ravel(), x) < 2e-5, g


@pytest.mark.parametrize("concurrency,nz,chains", [(1, 6, 1), (-1, 6, 1), (-1, 8, 2)])
def test_queue_volume_matches_3d_map(gpu_lib, concurrency, nz, chains):
    mace = gpu_lib
    n, V, D, N, va, sx, c, P = _volume(nz)
    xs = _map(P)
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, view_agent=va, sv_size=8)
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=0.5 if concurrency == 1 else 0.2, sigma_mode=1,
                           rho=0.8, sweeps_per_iter=2, symmetric=True, recompute_every=10,
                           tol=1e-7, max_iter=8000,
                           concurrency=concurrency, neighbourhood=26, schedule=1, chains=chains)
    st = mace.mace_init(sm, c["y"], c["lam"], prm, batch=nz)
    assert st.stats()["chains"] == chains
    x, iters, res, conv = st.reconstruct()
    st.close()
    sm.close()
    err = nrmse(np.asarray(x).ravel(), xs)
    print("queue volume conc=%d: iters=%d r=%.2e nrmse=%.2e" % (concurrency, iters, res, err))
    assert conv and err < 1e-4


def test_queue_more_pairs_than_resident_warps(gpu_lib):
    """512 reconstructions x 8 agents x 2 rows: far more items than the GPU
    holds warps (the fixed schedule refuses this batch).  Two distinct scans
    alternate over the batch; every reconstruction converges to its scan's
    MAP image."""
    mace = gpu_lib
    n, V, D, N, B = 32, 64, 47, 8, 512
    E = synth.ellipses(41, n, 0.02 * 64 / n)
    p = synth.sinogram(E, V, D)
    scans = [synth.measurements(p, 2e4, synth.CounterRNG(151 + k)) for k in range(2)]
    y = np.stack([scans[b % 2][0] for b in range(B)])
    lam = np.stack([scans[b % 2][1] for b in range(B)])
    sx = synth.prior_sigma_x(lam[0], V, frac=1.0)
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, sv_size=8)
    kw = dict(prior="qggmrf", sigma_x=sx, sigma=0.3, sigma_mode=1, rho=0.8, sweeps_per_iter=2, symmetric=True,
              recompute_every=10, tol=2e-7, max_iter=8000, concurrency=2)
    with pytest.raises(mace.MaceError):
        mace.mace_init(sm, y, lam, mace.make_params(**kw, chains=1), batch=B)
    st = mace.mace_init(sm, y, lam, mace.make_params(**kw, schedule=1), batch=B)
    x, iters, res, conv = st.reconstruct()
    st.close()
    sm.close()
    print("%d reconstructions: converged %s after %d iterations, worst residual %.2e" % (B, conv, iters, res))
    assert conv
    x = np.asarray(x, np.float64).reshape(B, -1)
    for k in range(2):
        P = oracle.Problem(n, n, V, D, scans[k][0], scans[k][1], n_agents=N, prior="qggmrf", sigma_x=sx)
        xs = _map(P)
        errs = [nrmse(x[b], xs) for b in range(k, B, 2)]
        print("scan %d: %d reconstructions, worst NRMSE vs oracle %.2e (iters %d)" % (k, len(errs), max(errs), iters))
        assert max(errs) < 1e-4


@functools.lru_cache(maxsize=None)
def wide_case():
    """40 x 40 pixels, 300 views over 2 agents: 150 views per agent."""
    n, V, D, N = 40, 300, 59, 2
    E = synth.ellipses(37, n, 0.02 * 64 / n)
    p = synth.sinogram(E, V, D)
    y, lam = synth.measurements(p, 2e4, synth.CounterRNG(137))
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=N, prior="qggmrf", sigma_x=sx)
    return dict(nx=n, ny=n, V=V, D=D, N=N, va=None, y=y[None], lam=lam[None], sx=sx, P=[P])


@pytest.mark.parametrize("case,W", [("wide", 2), ("wide", 4), ("ragged", 4)])
def test_warp_team_one_pass_matches_algorithm2(gpu_lib, case, W):
    """Teams of W warps per super-voxel (each warp holding a share of the
    agent's views and of the band, theta1 summed across the team): one pass
    at concurrency 1 is still Algorithm 2 for every agent.  The ragged case
    has 10-16 views per agent, so all but one warp of a team of four own no
    view at all."""
    mace = gpu_lib
    c = wide_case() if case == "wide" else ragged_case(1)
    N, n = c["N"], c["nx"] * c["ny"]
    sm = mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], N, view_agent=c["va"], sv_size=4)
    P = c["P"][0]
    xs = _map(P)
    rng = np.random.default_rng(11)
    sc = 0.3 * np.abs(xs).mean()
    X0 = (xs[None, :] + sc * rng.standard_normal((N, n))).astype(np.float32)
    v = (xs[None, :] + sc * rng.standard_normal((N, n))).astype(np.float32)
    for backward in (0, 1):
        prm = mace.make_params(prior="qggmrf", sigma_x=c["sx"], sigma=0.5, sigma_mode=1, concurrency=1, schedule=1,
                               warps_per_voxel=W)
        st = mace.mace_init(sm, c["y"][:1], c["lam"][:1], prm)
        assert st.stats()["warps_per_voxel"] == W
        st.set_state(X0.copy(), X0)
        st.prox_pass(v, backward=bool(backward))
        _, Xg = st.get_state()
        Xg = Xg.reshape(N, n)
        sigma = st.stats()["sigma_abs"]
        order = st.visit_order()
        st.close()
        if backward:
            order = order[::-1].copy()
        for g in range(N):
            x = X0[g].astype(np.float64)
            e = P.error_sinogram(g, x)
            P.icd_sweep(g, x, e, v=v[g].astype(np.float64), sigma=sigma, order=order)
            assert nrmse(Xg[g], x) < 2e-5, (backward, g)
    sm.close()


def test_warp_teams_converge_to_map(gpu_lib):
    """150 views per agent, rows of super-voxels in flight: with teams of
    two and four warps the image converges to the oracle's MAP image, as
    with one warp per super-voxel (the default, 0)."""
    mace = gpu_lib
    c = wide_case()
    sm = mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], c["N"], sv_size=4)
    xs = _map(c["P"][0])
    for W in (0, 2, 4):
        prm = mace.make_params(prior="qggmrf", sigma_x=c["sx"], sigma=0.3, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                               symmetric=True, recompute_every=10, tol=1e-7, max_iter=6000, concurrency=-1,
                               schedule=1, warps_per_voxel=W)
        st = mace.mace_init(sm, c["y"], c["lam"], prm)
        stats = st.stats()
        assert stats["warps_per_voxel"] == max(W, 1)
        x, iters, r, conv = st.reconstruct()
        st.close()
        err = nrmse(np.asarray(x).ravel(), xs)
        print("warps per voxel %d: iters %d, NRMSE vs oracle %.2e" % (stats["warps_per_voxel"], iters, err))
        assert conv and err < 1e-4
    sm.close()


def test_queue_volume_64x64x8_matches_3d_map(gpu_lib):
    """A larger stack: 64^2 x 8 slices, 90 views over 6 uneven agents, the
    work queue with z-parity and two slices per warp (serial order within
    each (slice, agent) pair): the converged volume equals the oracle's 3D
    MAP image.  (One row of super-voxels per item at normalised sigma 0.2
    diverges on this scan of 10-20 views per agent: concurrent super-voxels
    of an agent need a smaller sigma than serial passes do.)"""
    mace = gpu_lib
    n, nz, V, D, N = 64, 8, 90, 95, 6
    c = synth.make_volume(n=n, nz=nz, n_views=V, n_channels=D, I0=2e4, mu_max=0.02, seed=6, noise_seed=106)
    va = synth.uneven_partition(206, V, N, 10, 20)
    sx = synth.prior_sigma_x(c["lam"], V, frac=1.0)
    P = oracle.Problem(n, n, V, D, c["y"], c["lam"], n_agents=N, view_agent=va, nz=nz, prior="qggmrf",
                       neighbourhood=26, sigma_x=sx)
    xs = _map(P)
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, view_agent=va, sv_size=8)
    # FP32 iterates: the Mann residual settles near 1.4e-7 on this scan
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=0.5, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, recompute_every=10, tol=3e-7, max_iter=8000, concurrency=1,
                           neighbourhood=26, schedule=1, chains=2)
    st = mace.mace_init(sm, c["y"], c["lam"], prm, batch=nz)
    assert st.stats()["chains"] == 2
    x, iters, res, conv = st.reconstruct()
    st.close()
    sm.close()
    err = nrmse(np.asarray(x).ravel(), xs)
    print("64^2 x 8 volume: iters=%d r=%.2e nrmse=%.2e" % (iters, res, err))
    assert conv and err < 1e-4
