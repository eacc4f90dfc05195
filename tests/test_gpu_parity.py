"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from helpers import case, central_reference, nrmse

pytestmark = pytest.mark.gpu


def _build(mace, c, dtype="f32", sv=8, view_agent=None):
    return mace.mace_build_sysmatrix(c["n"], c["n"], c["V"], c["D"], c["N"], view_agent=view_agent,
                                     dtype=dtype, sv_size=sv)


@pytest.mark.parametrize("shape", [(64, 90, 95, 4), (37, 30, 53, 3)])
@pytest.mark.parametrize("sv", [8, 4])
def test_sysmatrix_bit_exact(gpu_lib, shape, sv):
    """Stored runs: indices bit-exact, FP32 values equal to the oracle's FP64
    strip integral rounded to nearest (both sides do the same IEEE ops)."""
    mace = gpu_lib
    n, V, D, N = shape
    c = case(n, V, D, N, "quadratic")
    P = c["P"]
    sm = _build(mace, c, sv=sv)
    rng = np.random.default_rng(0)
    pix = [(i, j) for i in range(n) for j in range(n)]
    if len(pix) > 600:
        pix = [pix[k] for k in rng.choice(len(pix), 600, replace=False)]
        pix += [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0)]
    for g in range(N):
        views = P.agent_views(g)
        for (i, j) in pix:
            c0, ln, vals = sm.column(g, i, j)
            for k, m in enumerate(views):
                oc0, ov = P.footprint(int(m), i, j)
                assert ln[k] == len(ov), (g, i, j, m)
                if len(ov):
                    assert c0[k] == oc0, (g, i, j, m)
                    np.testing.assert_array_equal(vals[k, :len(ov)], ov.astype(np.float32))
    info = sm.info()
    assert info["nnz"] == sum(len(P.footprint(int(m), i, j)[1])
                              for m in range(V) for i in range(n) for j in range(n))
    sm.close()


@pytest.mark.parametrize("sv_order,conc", [(0, 1), (0, 3), (1, 2)])
def test_visit_order_is_permutation(gpu_lib, sv_order, conc):
    mace = gpu_lib
    c = case(37, 30, 53, 3, "quadratic")
    sm = _build(mace, c, sv=4)
    st = mace.mace_init(sm, c["y"], c["lam"], mace.make_params(sigma_x=c["sigma_x"], concurrency=conc,
                                                               sv_order=sv_order))
    o = st.visit_order()
    assert sorted(o.tolist()) == list(range(37 * 37))


@pytest.mark.parametrize("prior", ["quadratic", "qggmrf"])
@pytest.mark.parametrize("backward", [False, True])
@pytest.mark.parametrize("batch", [1, 2, 4])
def test_one_pass_matches_algorithm2(gpu_lib, prior, backward, batch):
    """With one super-voxel per agent in flight, a GPU pass is Algorithm 2 in
    the library's visiting order: compare X after one pass from a random state."""
    mace = gpu_lib
    c = case(64, 90, 95, 4, prior)
    P, N, n = c["P"], c["N"], 64 * 64
    sm = _build(mace, c)
    rng = np.random.default_rng(1)
    xs = central_reference(64, 90, 95, 4, prior)
    # the same scan in every batch slot, different starting states
    X0 = (xs[None, None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((batch, N, n))).astype(np.float32)
    w0 = X0.copy()
    v = (xs[None, None, :] + 0.3 * np.abs(xs).mean() * rng.standard_normal((batch, N, n))).astype(np.float32)
    prm = mace.make_params(prior=prior, sigma_x=c["sigma_x"], sigma=0.5, sigma_mode=1, concurrency=1,
                           chains=batch)
    st = mace.mace_init(sm, np.stack([c["y"]] * batch), np.stack([c["lam"]] * batch), prm, batch=batch)
    assert st.stats()["chains"] == (2 if batch % 2 == 0 else 1)
    st.set_state(w0, X0)
    st.prox_pass(v, backward=backward)
    _, Xg = st.get_state()
    Xg = Xg.reshape(batch, N, n)
    sigma = st.stats()["sigma_abs"]
    order = st.visit_order()
    if backward:
        order = order[::-1].copy()
    for b in range(batch):
        for g in range(N):
            x = X0[b, g].astype(np.float64)
            e = P.error_sinogram(g, x)
            P.icd_sweep(g, x, e, v=v[b, g].astype(np.float64), sigma=sigma, order=order)
            err = nrmse(Xg[b, g], x)
            assert err < 2e-5, (b, g, err)
            # the pass moved the state
            assert nrmse(X0[b, g], x) > 1e-3
    st.close()
    sm.close()


def _reconstruct(mace, c, **kw):
    sm = _build(mace, c)
    args = dict(prior=c["prior"], sigma_x=c["sigma_x"], sigma=0.5, sigma_mode=1, rho=0.8,
                sweeps_per_iter=2, symmetric=True, recompute_every=10, max_iter=4000, tol=1e-7)
    args.update(kw)
    prm = mace.make_params(**args)
    st = mace.mace_init(sm, c["y"], c["lam"], prm)
    x, iters, r, conv = st.reconstruct()
    w, X = st.get_state()
    stats = st.stats()
    st.close()
    sm.close()
    return x, iters, r, conv, w, X, stats


@pytest.mark.parametrize("concurrency", [1])
def test_converged_matches_map_cfg1(gpu_lib, concurrency):
    """Config-1 shapes (64^2, 90 views, 95 channels, 4 interleaved agents,
    quadratic prior): the converged consensus equals the oracle's MAP image
    (MACE fixed point = MAP, Sec. II-B) within relative RMSE 1e-4."""
    c = case(64, 90, 95, 4, "quadratic")
    xs = central_reference(64, 90, 95, 4, "quadratic")
    x, iters, r, conv, w, X, stats = _reconstruct(gpu_lib, c, concurrency=concurrency)
    err = nrmse(x, xs)
    print("cfg1 concurrency=%s iters=%d r=%.2e nrmse=%.2e" % (stats["concurrency"], iters, r, err))
    assert conv
    assert err < 1e-4
    # at the fixed point every agent state equals the consensus (Thm 1 proof)
    wbar = w.astype(np.float64).mean(0)
    for g in range(4):
        assert nrmse(X[g], wbar) < 1e-4


@pytest.mark.parametrize("concurrency,sigma", [(1, 0.5), (8, 0.1)])
def test_converged_matches_map_qggmrf(gpu_lib, concurrency, sigma):
    """Q-GGMRF prior (p=2, q=1.2, T=1), 96^2 image, 8 agents: serial passes
    and concurrent super-voxels reach the oracle's MAP image."""
    c = case(96, 144, 137, 8, "qggmrf")
    xs = central_reference(96, 144, 137, 8, "qggmrf")
    x, iters, r, conv, w, X, stats = _reconstruct(gpu_lib, c, concurrency=concurrency, sigma=sigma,
                                                  tol=2e-8, max_iter=8000)
    err = nrmse(x, xs)
    print("qggmrf iters=%d r=%.2e nrmse=%.2e conc=%d" % (iters, r, err, stats["concurrency"]))
    assert err < 1e-4


def test_checkpoint_resume(gpu_lib):
    """(w, X) is the complete state (Eq. PUCEupdate): save, restore into a
    fresh state and continue; the result matches an uninterrupted run."""
    mace = gpu_lib
    c = case(64, 90, 95, 4, "quadratic")
    sm = _build(mace, c)
    prm = mace.make_params(prior="quadratic", sigma_x=c["sigma_x"], sigma=0.5, rho=0.8,
                           sweeps_per_iter=2, symmetric=True, concurrency=1, max_iter=100000)
    a = mace.mace_init(sm, c["y"], c["lam"], prm)
    a.iterate(40)
    w, X = a.get_state()
    a.iterate(40)
    xa = a.consensus()
    b = mace.mace_init(sm, c["y"], c["lam"], prm)
    b.set_state(w, X)
    b.iterate(40)
    xb = b.consensus()
    assert nrmse(xb, xa) < 1e-5
    a.close()
    b.close()
    sm.close()


def test_bad_inputs_rejected(gpu_lib):
    mace = gpu_lib
    c = case(37, 30, 53, 3, "quadratic")
    with pytest.raises(mace.MaceError) as ei:
        mace.mace_build_sysmatrix(37, 37, 30, 53, 3, sv_size=64)
    assert ei.value.code == mace.MACE_EINVAL
    sm = _build(mace, c, sv=4)
    lam = c["lam"].copy()
    lam[3, 7] = -1.0
    with pytest.raises(mace.MaceError) as ei:
        mace.mace_init(sm, c["y"], lam, mace.make_params(sigma_x=c["sigma_x"]))
    assert ei.value.code == mace.MACE_EINVAL
    y = c["y"].copy()
    y[0, 0] = np.nan
    with pytest.raises(mace.MaceError):
        mace.mace_init(sm, y, c["lam"], mace.make_params(sigma_x=c["sigma_x"]))
    with pytest.raises(mace.MaceError):
        mace.mace_init(sm, c["y"], c["lam"], mace.make_params(sigma_x=c["sigma_x"], rho=1.5))
    sm.close()


def test_graph_replay_matches_eager(gpu_lib):
    """On an explicit stream, iterations run as a captured CUDA graph
    replayed once per recompute period; the result equals eager launches on
    the default stream (up to the order of the sweep's atomic additions).
    One super-voxel per agent in flight: a trajectory that does not depend
    on scheduling."""
    import torch
    mace = gpu_lib
    c = case(64, 90, 95, 4, "quadratic")
    sm = _build(mace, c)
    out = {}
    for mode in ("eager", "graph"):
        stream = torch.cuda.Stream() if mode == "graph" else None
        prm = mace.make_params(prior="quadratic", sigma_x=c["sigma_x"], sigma=0.5, sigma_mode=1, rho=0.8,
                               sweeps_per_iter=2, symmetric=True, recompute_every=10, max_iter=4000, tol=1e-7,
                               concurrency=1)
        st = mace.mace_init(sm, c["y"], c["lam"], prm, stream=stream)
        out[mode] = st.reconstruct()
        st.close()
    sm.close()
    xe, ie, re, ce = out["eager"]
    xg, ig, rg, cg = out["graph"]
    assert ce and cg
    assert abs(ie - ig) <= 10
    assert nrmse(xg, xe) < 1e-5
