"""The consensus entry point that allocates nothing (mace_consensus_noalloc)
against mace_consensus, for callers that may not allocate device memory.

Collected last on purpose: it runs after every other GPU test, and alone."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _state(mace, n=64, batch=2):
    V, D, N = 90, 95, 4
    c = synth.make_case(n=n, n_views=V, n_channels=D, I0=1e4, mu_max=0.02, seed=1, noise_seed=101)
    y, lam = c["y"][0], c["lam"][0]
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, sv_size=8)
    prm = mace.make_params(prior="quadratic", sigma_x=sx, sigma=0.5, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, concurrency=1, max_iter=1000, tol=0.0)
    st = mace.mace_init(sm, np.stack([y] * batch), np.stack([lam] * batch), prm, batch=batch)
    return sm, st


def test_consensus_noalloc_matches_consensus(gpu_lib):
    """Host output through the library's fixed array, two calls in a row with
    the state moving in between: the same bits as mace_consensus (both run
    the same consensus kernel on the same state)."""
    mace = gpu_lib
    sm, st = _state(mace)
    for _ in range(2):
        st.iterate(7)
        ref = st.consensus()
        got = st.consensus_noalloc()
        assert np.abs(ref).max() > 0
        assert np.array_equal(got, ref)
    st.close()
    sm.close()


def test_consensus_noalloc_device_output(gpu_lib):
    """With a device output the images go straight to the caller's array."""
    import torch
    mace = gpu_lib
    sm, st = _state(mace)
    st.iterate(5)
    ref = st.consensus()
    out = torch.empty((2, 64, 64), device="cuda", dtype=torch.float32)
    st.consensus_noalloc(out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
    st.close()
    sm.close()


def test_consensus_noalloc_rejects_oversize(gpu_lib):
    """A host read-out larger than the fixed array (batch * n > 2^20 floats)
    is rejected with MACE_EINVAL, and the state stays usable."""
    mace = gpu_lib
    sm, st = _state(mace, n=512, batch=5)          # 5 * 512^2 floats > 2^20
    with pytest.raises(mace.MaceError) as ei:
        st.consensus_noalloc()
    assert ei.value.code == mace.MACE_EINVAL
    st.iterate(1)
    st.close()
    sm.close()
