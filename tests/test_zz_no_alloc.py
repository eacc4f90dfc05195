"""The consensus entry point that allocates nothing (mace_consensus_noalloc)
against mace_consensus, for callers that may not allocate device memory.

Collected last on purpose: it runs after every other GPU test, and alone."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_consensus_noalloc_matches_consensus(gpu_lib):
    mace = gpu_lib
    n, V, D, N = 64, 90, 95, 4
    c = synth.make_case(n=n, n_views=V, n_channels=D, I0=1e4, mu_max=0.02, seed=1, noise_seed=101)
    y, lam = c["y"][0], c["lam"][0]
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, sv_size=8)
    prm = mace.make_params(prior="quadratic", sigma_x=sx, sigma=0.5, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, concurrency=1, max_iter=1000, tol=0.0)
    st = mace.mace_init(sm, np.stack([y, y]), np.stack([lam, lam]), prm, batch=2)
    for _ in range(2):            # two calls in a row, the state moving in between
        st.iterate(7)
        ref = st.consensus()
        got = st.consensus_noalloc()
        assert np.abs(ref).max() > 0
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=0)
    st.close()
    sm.close()
