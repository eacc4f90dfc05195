"""Bit-for-bit reproducibility of the deterministic mode (params.deterministic
= 1) in the benchmark's launch configuration: 4x4 super-voxels, one
super-voxel row per warp (many super-voxels of an agent in flight), two
chains per warp, symmetric ICD passes.  In this mode the warps of an agent
advance in lock-step phases and sum their changes of e in fixed point, so the
iterates of Algorithm 1 are a function of the inputs alone (Eq. PUCEupdate
gives the next state from (w, X) only)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N_PIX, V, D, N = 128, 180, 183, 16


def _inputs(batch, seed0=60):
    ys, ls = [], []
    for b in range(batch):
        c = synth.make_case(n=N_PIX, n_views=V, n_channels=D, I0=2e4, mu_max=0.02 * 64 / N_PIX,
                            seed=seed0 + b, noise_seed=seed0 + 100 + b)
        ys.append(c["y"][0])
        ls.append(c["lam"][0])
    y, lam = np.stack(ys), np.stack(ls)
    return y, lam, synth.prior_sigma_x(lam[0], V, frac=1.0)


def _params(mace, sx, det=True, **kw):
    # sigma 0.1: the 4x4 row-per-warp schedule is stable at this size
    a = dict(prior="qggmrf", sigma_x=sx, sigma=0.1, sigma_mode=1, rho=0.95, sweeps_per_iter=2, symmetric=True,
             recompute_every=10, max_iter=400, tol=8e-7, concurrency=-1, chains=2, deterministic=det)
    a.update(kw)
    return mace.make_params(**a)


@pytest.fixture(scope="module")
def problem(gpu_lib):
    mace = gpu_lib
    y, lam, sx = _inputs(2)
    sm = mace.mace_build_sysmatrix(N_PIX, N_PIX, V, D, N, sv_size=4)
    yield mace, sm, y, lam, sx
    sm.close()


def _run(mace, sm, y, lam, prm, iters, stream=None):
    st = mace.mace_init(sm, y, lam, prm, stream=stream, batch=2)
    st.iterate(iters)
    w, X = st.get_state()
    x = st.consensus()
    stats = st.stats()
    st.close()
    return w, X, x, stats


def test_repeated_runs_bitwise(problem):
    """Two runs from the same inputs give identical bits (w, X and the
    consensus image), with many super-voxels of each agent in flight."""
    mace, sm, y, lam, sx = problem
    w1, X1, x1, s1 = _run(mace, sm, y, lam, _params(mace, sx), 60)
    w2, X2, x2, s2 = _run(mace, sm, y, lam, _params(mace, sx), 60)
    assert s1["concurrency"] == N_PIX // 4 and s1["chains"] == 2
    assert np.array_equal(w1, w2) and np.array_equal(X1, X2) and np.array_equal(x1, x2)


def test_deterministic_mode_converges_to_the_same_image(problem):
    """The lock-step schedule converges to the same fixed point as the free
    one (Theorem 1 does not depend on the order of the updates)."""
    mace, sm, y, lam, sx = problem
    out = {}
    for det in (False, True):
        st = mace.mace_init(sm, y, lam, _params(mace, sx, det=det, max_iter=3000), batch=2)
        x, it, r, conv = st.reconstruct()
        st.close()
        assert conv, det
        out[det] = x.astype(np.float64)
    err = np.linalg.norm(out[True] - out[False]) / np.linalg.norm(out[False])
    print("deterministic vs free schedule: relative difference %.2e" % err)
    assert err < 1e-4


def test_checkpoint_resume_bitwise(problem):
    """Checkpoint (w, X) after 30 iterations (a multiple of the e recompute
    period, where e = y - A X is a function of X), resume into a fresh state
    and run 30 more: the same bits as 60 iterations straight."""
    mace, sm, y, lam, sx = problem
    prm = _params(mace, sx)
    w_ref, X_ref, x_ref, _ = _run(mace, sm, y, lam, prm, 60)
    st = mace.mace_init(sm, y, lam, prm, batch=2)
    st.iterate(30)
    w, X = st.get_state()
    st.close()
    st = mace.mace_init(sm, y, lam, prm, batch=2)
    st.set_state(w, X)
    st.iterate(30)
    w2, X2 = st.get_state()
    x2 = st.consensus()
    st.close()
    assert np.array_equal(w2, w_ref) and np.array_equal(X2, X_ref) and np.array_equal(x2, x_ref)


def test_graph_replay_equals_eager_bitwise(problem):
    """Iterations replayed from the captured CUDA graph (explicit stream)
    give the same bits as eager launches (legacy default stream)."""
    import torch
    mace, sm, y, lam, sx = problem
    prm = _params(mace, sx)
    w_e, X_e, x_e, _ = _run(mace, sm, y, lam, prm, 40, stream=None)
    w_g, X_g, x_g, _ = _run(mace, sm, y, lam, prm, 40, stream=torch.cuda.Stream())
    assert np.array_equal(w_e, w_g) and np.array_equal(X_e, X_g) and np.array_equal(x_e, x_g)


def test_same_alone_and_in_the_mix_bitwise(problem):
    """Two batches iterated at the same time on two streams (their sweeps
    share the GPU) give the same bits as each alone."""
    import torch
    mace, sm, y, lam, sx = problem
    y2, lam2, _ = _inputs(2, seed0=80)
    prm = _params(mace, sx)
    alone_a = _run(mace, sm, y, lam, prm, 40)
    alone_b = _run(mace, sm, y2, lam2, prm, 40)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    sta = mace.mace_init(sm, y, lam, prm, stream=sa, batch=2)
    stb = mace.mace_init(sm, y2, lam2, prm, stream=sb, batch=2)
    for _ in range(4):
        sta.launch(10)
        stb.launch(10)
    sta.poll()
    stb.poll()
    mix = []
    for st in (sta, stb):
        w, X = st.get_state()
        mix.append((w, X, st.consensus()))
        st.close()
    for alone, m in zip((alone_a, alone_b), mix):
        assert np.array_equal(alone[0], m[0]) and np.array_equal(alone[1], m[1]) and np.array_equal(alone[2], m[2])


def test_free_schedule_spread(problem):
    """Without the deterministic mode the float atomics of concurrent
    super-voxels make the trajectories of two runs differ, but both converge
    to the same fixed point (the spread is printed)."""
    mace, sm, y, lam, sx = problem
    prm = _params(mace, sx, det=False)
    _, _, x1, _ = _run(mace, sm, y, lam, prm, 60)
    _, _, x2, _ = _run(mace, sm, y, lam, prm, 60)
    d60 = float(np.linalg.norm(x1.astype(np.float64) - x2) / np.linalg.norm(x2))
    xs = []
    for _ in range(2):
        st = mace.mace_init(sm, y, lam, _params(mace, sx, det=False, max_iter=3000), batch=2)
        x, it, r, conv = st.reconstruct()
        st.close()
        assert conv
        xs.append(x.astype(np.float64))
    dconv = float(np.linalg.norm(xs[0] - xs[1]) / np.linalg.norm(xs[1]))
    print("free schedule, two runs: relative difference %.2e after 60 iterations, %.2e converged" % (d60, dconv))
    assert dconv < 1e-5
