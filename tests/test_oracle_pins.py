"""Pins of the oracle's ICD and MACE against closed forms from the paper:
Eq. ICDUpdate1 (one ICD pass is a Gauss-Seidel step), Eq. prox_exact,
Lemma B.1, Theorem 1 (MACE fixed point = MAP), Theorem 2 (spectral radius),
the Q-GGMRF gradient against finite differences of the cost, and the
Q-GGMRF potential through its q = p special case (half the quadratic prior)
and its growth exponents (p near zero, q far from it)."""
import math

import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle
import synth


def _tiny(n=12, V=16, D=19, N=3, prior="quadratic", seed=5):
    c = synth.make_case(n=n, n_views=V, n_channels=D, I0=1e4, mu_max=0.02 * 64 / n, seed=seed,
                        noise_seed=seed + 100)
    y, lam = c["y"][0].astype(np.float64), c["lam"][0].astype(np.float64)
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=N, prior=prior, sigma_x=sx)
    return P, y, lam, sx


def _prior_B(n, sx):
    """B with h = 1/2 x^T B x for the quadratic prior: b_sr ~ 1/distance over
    the 8-neighbourhood normalised to sum 1, each pair once, rho = D^2/(2 sx^2)."""
    w = {(0, 1): 1.0, (1, 0): 1.0, (1, 1): 1 / math.sqrt(2), (1, -1): 1 / math.sqrt(2)}
    tot = 4 * 1.0 + 4 / math.sqrt(2)
    B = np.zeros((n * n, n * n))
    for i in range(n):
        for j in range(n):
            for (di, dj), b in w.items():
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    s, r = i * n + j, ii * n + jj
                    c = b / tot / sx ** 2
                    B[s, s] += c
                    B[r, r] += c
                    B[s, r] -= c
                    B[r, s] -= c
    return B


def _agent_system(P, y, lam, g, beta=1.0):
    """H_i = A_i^T Lambda_i A_i + (beta/N) B and b_i = A_i^T Lambda_i y_i (Eq. prox_exact)."""
    A = P.dense_A()
    V, D, N = P.n_views, P.n_channels, P.n_agents
    rows = np.concatenate([np.arange(m * D, (m + 1) * D) for m in range(V)
                           if g < 0 or P.view_agent[m] == g])
    Ai = A[rows]
    li = lam.reshape(-1)[rows]
    yi = y.reshape(-1)[rows]
    B = _prior_B(P.nx, P._s.sigma_x)
    scale = beta if g < 0 else beta / N
    return Ai.T @ (li[:, None] * Ai) + scale * B, Ai.T @ (li * yi)


@pytest.mark.parametrize("order_kind", ["raster", "random"])
def test_one_pass_is_gauss_seidel(order_kind):
    """Eq. ICDUpdate1: F~_i(v; x) = -(L_i + D_i + I/sigma^2)^-1 (L_i^T x - b_i - v/sigma^2),
    with L_i, D_i the strict lower and diagonal parts of H_i in visiting order."""
    P, y, lam, sx = _tiny()
    rng = np.random.default_rng(0)
    n = P.n
    order = np.arange(n) if order_kind == "raster" else rng.permutation(n)
    for g in range(P.n_agents):
        H, b = _agent_system(P, y, lam, g)
        sigma = 0.7 / math.sqrt(np.mean(np.diag(H)))
        x = 0.01 * rng.standard_normal(n)
        v = 0.01 * rng.standard_normal(n)
        # dense reference in the permuted basis
        Hp = H[np.ix_(order, order)]
        Lt = np.tril(Hp) + np.eye(n) / sigma ** 2
        U = np.triu(Hp, 1)
        zp = solve_triangular(Lt, b[order] + v[order] / sigma ** 2 - U @ x[order], lower=True)
        z = np.empty(n)
        z[order] = zp
        # oracle
        xo = x.copy()
        e = P.error_sinogram(g, xo)
        P.icd_sweep(g, xo, e, v=v, sigma=sigma, order=order)
        assert np.linalg.norm(xo - z) / np.linalg.norm(z) < 1e-12
        # e stays the error sinogram of the new state
        np.testing.assert_allclose(e, P.error_sinogram(g, xo), rtol=0, atol=1e-13)


def test_prox_closed_form():
    """Eq. prox_exact: ICD passes with v fixed converge to
    F_i(v) = (H_i + I/sigma^2)^-1 (b_i + v/sigma^2)."""
    P, y, lam, sx = _tiny()
    rng = np.random.default_rng(1)
    g = 1
    H, b = _agent_system(P, y, lam, g)
    sigma = 1.0 / math.sqrt(np.mean(np.diag(H)))
    v = 0.01 * rng.standard_normal(P.n)
    F = np.linalg.solve(H + np.eye(P.n) / sigma ** 2, b + v / sigma ** 2)
    x = np.zeros(P.n)
    e = P.error_sinogram(g, x)
    for _ in range(400):
        P.icd_sweep(g, x, e, v=v, sigma=sigma)
    assert np.linalg.norm(x - F) / np.linalg.norm(F) < 1e-11


def test_lemma_b1_fixed_point_of_partial_update():
    """Lemma B.1: F~_i(v; x) = x exactly when x = F_i(v)."""
    P, y, lam, sx = _tiny()
    rng = np.random.default_rng(2)
    g = 2
    H, b = _agent_system(P, y, lam, g)
    sigma = 0.5 / math.sqrt(np.mean(np.diag(H)))
    v = 0.01 * rng.standard_normal(P.n)
    F = np.linalg.solve(H + np.eye(P.n) / sigma ** 2, b + v / sigma ** 2)
    x = F.copy()
    e = P.error_sinogram(g, x)
    P.icd_sweep(g, x, e, v=v, sigma=sigma, order=rng.permutation(P.n))
    assert np.linalg.norm(x - F) / np.linalg.norm(F) < 1e-12
    # and a state that is not F_i(v) moves
    x2 = F + 1e-3
    e2 = P.error_sinogram(g, x2)
    P.icd_sweep(g, x2, e2, v=v, sigma=sigma)
    assert np.linalg.norm(x2 - (F + 1e-3)) > 1e-6


def test_mace_fixed_point_is_map():
    """Sec. II-B / Theorem 1: the MACE solution is the MAP estimate
    (A^T Lambda A + beta B)^-1 A^T Lambda y; so is centralised ICD."""
    P, y, lam, sx = _tiny(n=16, V=24, D=25, N=4)
    H, b = _agent_system(P, y, lam, -1)
    xmap = np.linalg.solve(H, b)
    xc, it, r = P.central_icd(max_sweeps=5000, tol=1e-14)
    assert np.linalg.norm(xc - xmap) / np.linalg.norm(xmap) < 1e-11
    t2 = oracle.mean_theta2(P)
    res = P.mace(0.5 / math.sqrt(t2), rho=0.8, sweeps=2, symmetric=True, max_iter=20000, tol=1e-14)
    assert np.linalg.norm(res["x"] - xmap) / np.linalg.norm(xmap) < 1e-10
    # at the fixed point X_i = mean_i w_i for every agent (proof of Theorem 1)
    for g in range(4):
        assert np.linalg.norm(res["X"][g] - res["x"]) / np.linalg.norm(xmap) < 1e-10


def test_mace_one_forward_pass_small_sigma():
    """Algorithm 1 exactly as printed (one forward ICD pass per iteration)
    converges to the MAP image for small sigma (Theorem 2 regime)."""
    P, y, lam, sx = _tiny(n=12, V=16, D=19, N=2)
    H, b = _agent_system(P, y, lam, -1)
    xmap = np.linalg.solve(H, b)
    t2 = oracle.mean_theta2(P)
    res = P.mace(0.1 / math.sqrt(t2), rho=0.8, sweeps=1, max_iter=40000, tol=1e-14)
    assert np.linalg.norm(res["x"] - xmap) / np.linalg.norm(xmap) < 1e-9


def test_theorem2_spectral_radius():
    """Theorem 2: for a quadratic prior and small sigma the augmented update
    (w, X) -> M (w, X) + c is a contraction (all |eigenvalues| < 1); M is built
    column by column by running one iteration on unit vectors with y = 0."""
    n, V, D, N = 6, 8, 11, 2
    P0, y, lam, sx = _tiny(n=n, V=V, D=D, N=N)
    P = oracle.Problem(n, n, V, D, np.zeros_like(y), lam, n_agents=N, prior="quadratic", sigma_x=sx)
    t2 = oracle.mean_theta2(P)
    nn = n * n

    def radius(sn, rho=0.8):
        M = np.zeros((2 * N * nn, 2 * N * nn))
        for k in range(2 * N * nn):
            z = np.zeros(2 * N * nn)
            z[k] = 1.0
            r = P.mace(sn / math.sqrt(t2), rho=rho, max_iter=1, tol=0.0,
                       w0=z[:N * nn].reshape(N, nn), X0=z[N * nn:].reshape(N, nn))
            M[:, k] = np.concatenate([r["w"].ravel(), r["X"].ravel()])
        return np.abs(np.linalg.eigvals(M)).max()

    assert radius(0.05) < 1.0
    assert radius(0.2) < 1.0


@pytest.mark.parametrize("prior", ["quadratic", "qggmrf"])
def test_fixed_point_independent_of_N_sigma_rho_order(prior):
    """Theorem 1 with Lemma B.1: x* does not depend on N, sigma, rho or the
    voxel order; all equal the centralised MAP image."""
    P1, y, lam, sx = _tiny(n=12, V=24, D=19, N=1, prior=prior)
    xc, _, _ = P1.central_icd(max_sweeps=20000, tol=1e-14)
    rng = np.random.default_rng(3)
    for N, sn, rho, order in [(2, 0.5, 0.8, None), (4, 1.0, 0.5, rng.permutation(144)),
                              (3, 0.3, 0.8, rng.permutation(144))]:
        P = oracle.Problem(12, 12, 24, 19, y, lam, n_agents=N, prior=prior, sigma_x=sx)
        t2 = oracle.mean_theta2(P)
        res = P.mace(sn / math.sqrt(t2), rho=rho, sweeps=2, symmetric=True, order=order,
                     max_iter=30000, tol=1e-14)
        assert np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc) < 1e-9, (N, sn, rho)


def test_qggmrf_gradient_matches_cost():
    """The oracle's gradient (data term and rho'(D) of the Q-GGMRF) against
    central finite differences of the MAP cost."""
    P, y, lam, sx = _tiny(n=8, V=12, D=13, N=1, prior="qggmrf")
    rng = np.random.default_rng(5)
    x = 0.02 + 0.01 * rng.standard_normal(P.n)
    g = P.gradient(x)
    h = 1e-6
    for s in rng.choice(P.n, 12, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[s] += h
        xm[s] -= h
        fd = (P.cost(xp) - P.cost(xm)) / (2 * h)
        assert abs(fd - g[s]) <= 1e-5 * (abs(g[s]) + 1e-3 * np.abs(g).max())


def test_qggmrf_central_icd_kkt():
    """Centralised ICD with the surrogate prior steps converges to a
    stationary point of the true cost (||grad f|| / ||grad f(0)|| tiny)."""
    P, y, lam, sx = _tiny(n=12, V=16, D=19, N=1, prior="qggmrf")
    x, it, r = P.central_icd(max_sweeps=20000, tol=1e-14)
    g0 = np.linalg.norm(P.gradient(np.zeros(P.n)))
    assert np.linalg.norm(P.gradient(x)) / g0 < 1e-10


def _prior_only(nx, ny, prior, q=1.2, T=1.0, sx=0.7):
    """A problem whose weights are all zero: its cost is beta h(x) alone."""
    V, D = 4, 9
    z = np.zeros((V, D))
    return oracle.Problem(nx, ny, V, D, z, z, n_agents=1, prior=prior, sigma_x=sx, q=q, T=T)


def test_qggmrf_with_q_equal_p_is_half_the_quadratic_prior():
    """With q = p = 2 the Q-GGMRF's edge factor is constant (1/2), so its
    cost and gradient are half those of the quadratic prior (pinned above
    against the dense B), over every neighbour pair of a ragged image."""
    rng = np.random.default_rng(9)
    x = rng.standard_normal(6 * 5)
    Pq = _prior_only(6, 5, "qggmrf", q=2.0, T=0.5)
    Pquad = _prior_only(6, 5, "quadratic")
    assert Pquad.cost(x) > 0
    assert Pq.cost(x) == pytest.approx(0.5 * Pquad.cost(x), rel=1e-13)
    np.testing.assert_allclose(Pq.gradient(x), 0.5 * Pquad.gradient(x), rtol=1e-12, atol=1e-15)


def test_qggmrf_potential_growth_exponents():
    """The Q-GGMRF potential of one neighbour pair grows like |D|^p (p = 2,
    low-contrast detail kept by a quadratic) for |D| << T sigma_x and like
    |D|^q (q = 1.2, edges penalised less) for |D| >> T sigma_x; it is even,
    zero at zero and increasing in |D|."""
    sx, T, q = 0.7, 1.0, 1.2
    P = _prior_only(2, 1, "qggmrf", q=q, T=T, sx=sx)

    def h(d):
        return P.cost(np.array([d, 0.0]))
    assert h(0.0) == 0.0
    assert h(-0.3) == pytest.approx(h(0.3), rel=1e-15)
    small, large = 1e-6 * T * sx, 1e6 * T * sx
    assert h(2 * small) / h(small) == pytest.approx(4.0, rel=1e-3)
    assert h(2 * large) / h(large) == pytest.approx(2.0 ** q, rel=1e-3)
    ds = np.geomspace(1e-3, 1e3, 61) * T * sx
    vals = [h(d) for d in ds]
    assert all(b > a for a, b in zip(vals, vals[1:]))
