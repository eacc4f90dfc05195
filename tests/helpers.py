"""Shared test cases: seeded synthetic problems and their oracle references."""
import functools

import numpy as np

import oracle
import synth


@functools.lru_cache(maxsize=None)
def case(n, V, D, N, prior, frac=1.0, I0=2e4, seed=3, noise_seed=103, mu=None):
    mu_max = 0.02 * 64 / n if mu is None else mu
    c = synth.make_case(n=n, n_views=V, n_channels=D, I0=I0, mu_max=mu_max, seed=seed,
                        noise_seed=noise_seed)
    y, lam = c["y"][0], c["lam"][0]
    sx = synth.prior_sigma_x(lam, V, frac=frac)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=N, prior=prior, sigma_x=sx)
    return dict(n=n, V=V, D=D, N=N, y=y, lam=lam, sigma_x=sx, prior=prior, P=P)


@functools.lru_cache(maxsize=None)
def central_reference(n, V, D, N, prior, frac=1.0, tol=1e-12, max_sweeps=20000, **kw):
    c = case(n, V, D, N, prior, frac, **kw)
    x, it, r = c["P"].central_icd(max_sweeps=max_sweeps, tol=tol)
    return x


def nrmse(x, ref):
    x = np.asarray(x, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
