"""MACE with a plug-and-play prior (Sec. III, Algorithm 3) on the GPU: the
data agents (sqrt(N) sigma, no prior) with the denoiser H = the quadratic
prior's proximal map in the consensus operator.  Parity with the oracle's
Algorithm 3 step by step, and the converged image equals the MAP image
(Theorem 3 with Lemma 2)."""
import numpy as np
import pytest

from helpers import case, central_reference, nrmse

pytestmark = pytest.mark.gpu

CASE = (64, 90, 95, 4, "quadratic")


def _state(mace, c, **kw):
    sm = mace.mace_build_sysmatrix(c["n"], c["n"], c["V"], c["D"], c["N"], sv_size=8)
    args = dict(prior="quadratic", sigma_x=c["sigma_x"], sigma=0.2, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                symmetric=True, recompute_every=0, max_iter=4000, tol=1e-8, concurrency=1, pnp=True)
    args.update(kw)
    return sm, mace.mace_init(sm, c["y"], c["lam"], mace.make_params(**args))


def test_pnp_iterations_match_algorithm3(gpu_lib):
    """Three Mann iterations from w = 0 with one super-voxel per agent in
    flight follow the oracle's Algorithm 3 in the library's visiting order."""
    mace = gpu_lib
    c = case(*CASE)
    sm, st = _state(mace, c)
    st.iterate(3)
    w, X = st.get_state()
    x = st.consensus()
    sigma = st.stats()["sigma_abs"]
    order = st.visit_order()
    st.close()
    res = c["P"].pnp_mace(sigma, rho=0.8, sweeps=2, symmetric=True, max_iter=3, tol=0.0, order=order)
    assert nrmse(w, res["w"]) < 2e-5
    assert nrmse(X, res["X"]) < 2e-5
    assert nrmse(x, res["x"]) < 2e-5


@pytest.mark.parametrize("concurrency,sigma", [(1, 0.2), (8, 0.1)])
def test_pnp_converges_to_map(gpu_lib, concurrency, sigma):
    """Serial passes, and concurrent super-voxels at a smaller sigma (the
    data-only agents' proximal parameter is sqrt(N) sigma; at sigma 0.2 eight
    concurrent super-voxels per agent diverge on this case)."""
    mace = gpu_lib
    c = case(*CASE)
    xs = central_reference(*CASE)
    # the FP32 state's Mann residual levels off near 1e-7: stop at 2e-7
    sm, st = _state(mace, c, concurrency=concurrency, sigma=sigma, tol=2e-7, max_iter=3000)
    x, iters, r, conv = st.reconstruct()
    w, X = st.get_state()
    st.close()
    err = nrmse(x, xs)
    print("pnp conc=%d: iters=%d r=%.2e nrmse=%.2e" % (concurrency, iters, r, err))
    assert conv
    assert err < 1e-4
    # each agent's state equals the solution at the fixed point
    for g in range(c["N"]):
        assert nrmse(X[g], x.ravel()) < 1e-4


def test_pnp_rejects_qggmrf(gpu_lib):
    mace = gpu_lib
    c = case(*CASE)
    with pytest.raises(mace.MaceError):
        _state(mace, c, prior="qggmrf")
