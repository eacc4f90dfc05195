"""Pins of the oracle's MACE with a plug-and-play prior (Sec. III,
Algorithm 3, Theorem 3): with H the proximal map of the quadratic prior, H
is the dense solve (I + sigma^2 B)^-1 v, and the fixed point is the MAP
image (A^T Lambda A + B)^-1 A^T Lambda y; at the fixed point each data
agent's proximal map at sigma returns x* from x* + u_i (the equilibrium of
Theorem 3), which pins the sqrt(N) sigma the iteration uses."""
import math

import numpy as np

import oracle
from test_oracle_pins import _agent_system, _prior_B, _tiny


def test_prior_prox_is_dense_solve():
    P, y, lam, sx = _tiny(n=10, V=12, D=15, N=3)
    rng = np.random.default_rng(3)
    v = rng.uniform(0.0, 0.02, P.n)
    B = _prior_B(P.nx, sx)
    for sigma in (0.3 * sx, sx, 4.0 * sx):
        x = P.prior_prox(v, sigma)
        xd = np.linalg.solve(np.eye(P.n) + sigma ** 2 * B, v)
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12


def test_pnp_fixed_point_is_map_and_equilibrium():
    P, y, lam, sx = _tiny(n=12, V=18, D=19, N=3)
    H, b = _agent_system(P, y, lam, -1)
    xmap = np.linalg.solve(H, b)
    t2 = oracle.mean_theta2(P)
    sigma = 0.3 / math.sqrt(t2)
    res = P.pnp_mace(sigma, rho=0.8, sweeps=2, symmetric=True, max_iter=40000, tol=1e-15)
    x = res["x"]
    assert np.linalg.norm(x - xmap) / np.linalg.norm(xmap) < 1e-9
    N = P.n_agents
    w = res["w"]
    # w* = N copies of x* - N u*  (Theorem 3)  ->  u_i = (x* - w_i) / N, and
    # F_i(x* + u_i; sigma) = x* with F_i the data-only proximal map at sigma
    for g in range(N):
        Hi, bi = _agent_system(P, y, lam, g, beta=0.0)
        u = (x - w[g]) / N
        z = np.linalg.solve(Hi + np.eye(P.n) / sigma ** 2, bi + (x + u) / sigma ** 2)
        assert np.linalg.norm(z - x) / np.linalg.norm(x) < 1e-8
        # each agent's state X_i equals x* at the fixed point
        assert np.linalg.norm(res["X"][g] - x) / np.linalg.norm(x) < 1e-9
    # and the denoiser's residual alpha = -sum u_i satisfies H(x* + alpha) = x*
    alpha = -sum((x - w[g]) / N for g in range(N))
    assert np.linalg.norm(P.prior_prox(x + alpha, sigma) - x) / np.linalg.norm(x) < 1e-9


def test_qggmrf_prior_prox_is_stationary():
    """The oracle's prior proximal map for the Q-GGMRF prior (a nonlinear
    map, by coordinate steps to convergence): beta grad h(x) + (x - v) /
    sigma^2 = 0, with grad h from the cost's gradient on a problem without
    data (all weights zero)."""
    n, V, D = 10, 8, 15
    zero = np.zeros((V, D))
    sx = 0.01
    P = oracle.Problem(n, n, V, D, zero, zero, n_agents=1, prior="qggmrf", sigma_x=sx)
    rng = np.random.default_rng(4)
    v = 0.02 + 0.01 * rng.standard_normal(P.n)
    for sigma in (0.3 * sx, 3.0 * sx):
        x = P.prior_prox(v, sigma)
        g = P.gradient(x) + (x - v) / sigma ** 2
        assert np.linalg.norm(g) < 1e-10 * np.linalg.norm((v - v.mean()) / sigma ** 2)
