"""Why the e recompute evaluates the matrix from the geometry when the stored
values are rounded: dense solves of the quadratic-prior MAP problem on a
small scan, with the oracle's FP64 matrix and prior.  The fixed point with
rounded values in both projections is further from the exact MAP image than
the one with the exact forward projection (what the recompute re-anchors e
to) and rounded back-projection (what theta1 uses)."""
import numpy as np
import pytest

import oracle
import synth


def to_bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5, 0.0])
    # 8-bit significand: 1 + 2^-8 is not representable; the ties go to even
    assert list(to_bf16(x)) == [1.0, 1.0, 1.0, 1.0 + 2 ** -7, -2.5, 0.0]


@pytest.mark.parametrize("rnd,name", [(to_bf16, "bf16"), (lambda a: np.asarray(a, np.float16).astype(np.float64), "f16")])
def test_exact_forward_is_closer_to_the_map(rnd, name):
    n, V, D = 32, 48, 47
    c = synth.make_case(n=n, n_views=V, n_channels=D, I0=2e4, mu_max=0.04, seed=5, noise_seed=55)
    y, lam = c["y"][0], c["lam"][0]
    sx = synth.prior_sigma_x(lam, V, frac=1.0)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=4, prior="quadratic", sigma_x=sx)
    A = P.dense_A()
    W = lam.reshape(-1).astype(np.float64)
    yy = y.reshape(-1).astype(np.float64)
    N = n * n
    AtWA = A.T @ (W[:, None] * A)
    # the prior's Hessian from the oracle's gradient: grad(x) = A^T W (A x - y) + B x
    g0 = P.gradient(np.zeros(N))
    B = np.empty((N, N))
    for j in range(N):
        ej = np.zeros(N)
        ej[j] = 1.0
        B[:, j] = P.gradient(ej) - g0 - AtWA[:, j]
    assert np.allclose(B, B.T, atol=1e-9 * np.abs(B).max())
    x_map = np.linalg.solve(AtWA + B, A.T @ (W * yy))
    # the oracle's own solver reaches the same MAP image
    x_icd, _, _ = P.central_icd(max_sweeps=20000, tol=1e-13)
    assert np.linalg.norm(x_icd - x_map) / np.linalg.norm(x_map) < 1e-8
    Ar = rnd(A)
    x_pair = np.linalg.solve(Ar.T @ (W[:, None] * Ar) + B, Ar.T @ (W * yy))
    x_mixed = np.linalg.solve(Ar.T @ (W[:, None] * A) + B, Ar.T @ (W * yy))
    e_pair = np.linalg.norm(x_pair - x_map) / np.linalg.norm(x_map)
    e_mixed = np.linalg.norm(x_mixed - x_map) / np.linalg.norm(x_map)
    print("%s: rounded pair %.2e, exact forward %.2e" % (name, e_pair, e_mixed))
    assert e_mixed < 0.6 * e_pair
