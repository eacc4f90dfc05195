"""3D stacks: slices share the 2D matrix and a 26-neighbourhood Q-GGMRF prior
couples them; agents own uneven view subsets spread over the half circle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import nrmse

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chains", [1, 2])
@pytest.mark.parametrize("concurrency,sigma", [(1, 0.5), (4, 0.1)])
def test_volume_matches_3d_map(gpu_lib, concurrency, sigma, chains):
    mace = gpu_lib
    n, nz, V, D, N = 32, 6, 60, 47, 4
    c = synth.make_volume(n=n, nz=nz, n_views=V, n_channels=D, I0=2e4, mu_max=0.04, seed=4, noise_seed=104)
    y, lam = c["y"], c["lam"]
    va = synth.uneven_partition(204, V, N, 10, 20)
    assert sorted(np.bincount(va).tolist()) == sorted(np.bincount(va).tolist()) and np.bincount(va).min() >= 10
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=N, view_agent=va, nz=nz, prior="qggmrf",
                       neighbourhood=26, sigma_x=sx)
    xs, it, r = P.central_icd(max_sweeps=20000, tol=1e-13)
    g0 = np.linalg.norm(P.gradient(np.zeros(P.n)))
    assert np.linalg.norm(P.gradient(xs)) / g0 < 1e-9
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, view_agent=va, sv_size=8)
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=sigma, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, recompute_every=10, tol=2e-8, max_iter=8000,
                           concurrency=concurrency, neighbourhood=26, chains=chains)
    st = mace.mace_init(sm, y, lam, prm, batch=nz)
    assert st.stats()["chains"] == chains     # two chains: two slices per warp
    x, iters, res, conv = st.reconstruct()
    err = nrmse(x.ravel(), xs)
    print("volume conc=%d chains=%d: iters=%d r=%.2e nrmse=%.2e" % (concurrency, chains, iters, res, err))
    assert err < 1e-4
