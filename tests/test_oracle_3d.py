"""Pins of the oracle's 3D stack (slices sharing one 2D matrix, the
26-neighbourhood prior coupling them), of theta2 and of the uneven view
partition, against hand-computed values, finite differences, dense algebra
and stationarity."""
import math

import numpy as np

import oracle
import synth


def _volume(n=6, nz=3, V=10, D=11, N=2, prior="qggmrf", lam_scale=1.0, seed=4):
    c = synth.make_volume(n=n, nz=nz, n_views=V, n_channels=D, I0=2e4, mu_max=0.2, seed=seed,
                          noise_seed=seed + 100)
    y, lam = c["y"].astype(np.float64), c["lam"].astype(np.float64) * lam_scale
    sx = synth.prior_sigma_x(c["lam"], V, frac=1.0)
    return oracle.Problem(n, n, V, D, y, lam, n_agents=N, nz=nz, prior=prior, neighbourhood=26, sigma_x=sx), sx


def test_26_neighbour_pair_weight_by_hand():
    """Two voxels stacked in z with no data: h has one pair, the face
    neighbour of weight 1 / (6 + 12/sqrt2 + 8/sqrt3), rho = D^2 / (2 sx^2);
    a 1 x 2 in-plane pair (8-neighbourhood) has weight 1 / (4 + 4/sqrt2)."""
    sx = 0.7
    zero = np.zeros((2, 3, 5))
    P3 = oracle.Problem(1, 1, 3, 5, zero, zero, n_agents=1, nz=2, prior="quadratic", neighbourhood=26,
                        sigma_x=sx)
    x = np.array([0.3, -0.2])
    b = 1.0 / (6 + 12 / math.sqrt(2) + 8 / math.sqrt(3))
    assert abs(P3.cost(x) - b * 0.5 ** 2 / (2 * sx ** 2)) < 1e-15
    zero2 = np.zeros((1, 3, 5))
    P2 = oracle.Problem(2, 1, 3, 5, zero2, zero2, n_agents=1, prior="quadratic", sigma_x=sx)
    b2 = 1.0 / (4 + 4 / math.sqrt(2))
    assert abs(P2.cost(x) - b2 * 0.5 ** 2 / (2 * sx ** 2)) < 1e-15


def test_3d_gradient_matches_cost():
    P, sx = _volume()
    rng = np.random.default_rng(7)
    x = 0.02 + 0.01 * rng.standard_normal(P.n)
    g = P.gradient(x)
    h = 1e-6
    for s in rng.choice(P.n, 15, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[s] += h
        xm[s] -= h
        fd = (P.cost(xp) - P.cost(xm)) / (2 * h)
        assert abs(fd - g[s]) <= 1e-5 * (abs(g[s]) + 1e-3 * np.abs(g).max())


def test_3d_central_icd_is_stationary():
    P, sx = _volume(n=8, nz=4, V=12, D=13)
    x, it, r = P.central_icd(max_sweeps=20000, tol=1e-14)
    g0 = np.linalg.norm(P.gradient(np.zeros(P.n)))
    assert np.linalg.norm(P.gradient(x)) / g0 < 1e-10


def test_theta2_is_the_data_hessian_diagonal():
    """theta2 of agent g = diag(A_g^T Lambda_g A_g), from the dense matrix."""
    c = synth.make_case(n=10, n_views=14, n_channels=15, I0=1e4, mu_max=0.1, seed=3, noise_seed=103)
    y, lam = c["y"][0].astype(np.float64), c["lam"][0].astype(np.float64)
    P = oracle.Problem(10, 10, 14, 15, y, lam, n_agents=3, prior="quadratic", sigma_x=1.0)
    A = P.dense_A()
    for g in range(3):
        rows = np.concatenate([np.arange(m * 15, (m + 1) * 15) for m in P.agent_views(g)])
        d = np.einsum("ks,k,ks->s", A[rows], lam.reshape(-1)[rows], A[rows])
        np.testing.assert_allclose(P.theta2(g), d, rtol=1e-13, atol=1e-15)


def test_uneven_partition():
    """Counts within [lo, hi] summing to the views; every agent's views
    spread over the half circle (none holds a contiguous block)."""
    V, N, lo, hi = 960, 32, 16, 40
    va = synth.uneven_partition(204, V, N, lo, hi)
    cnt = np.bincount(va, minlength=N)
    assert cnt.sum() == V and cnt.min() >= lo and cnt.max() <= hi
    for g in range(N):
        m = np.flatnonzero(va == g)
        assert m.min() < V // 8 and m.max() > V - V // 8
        assert np.diff(m).max() <= 4 * V // cnt[g]
