"""Continuous batching: requests of different sizes arrive while others run;
each served image equals the same request reconstructed alone."""
import numpy as np
import pytest

import oracle
import synth
from helpers import nrmse

pytestmark = pytest.mark.gpu


def _requests(serve_mod, specs, rate, seed=5):
    rng = synth.CounterRNG(seed)
    gaps = -np.log(1.0 - rng.uniform(9, np.arange(len(specs)))) / rate
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for k, (n, V, D, N) in enumerate(specs):
        c = synth.make_case(n=n, n_views=V, n_channels=D, I0=2e4, mu_max=0.02 * 64 / n, seed=1000 + k,
                            noise_seed=2000 + k)
        sx = synth.prior_sigma_x(c["lam"][0], V, frac=1.0)
        reqs.append(serve_mod.Request(k, float(t[k]), n, n, V, D, N, c["y"][0], c["lam"][0], sx, None))
    return reqs


PARAMS = dict(prior="qggmrf", sigma=0.5, sigma_mode=1, rho=0.8, sweeps_per_iter=2, symmetric=True,
              recompute_every=10, tol=1e-6, concurrency=1)


def test_served_equals_alone(gpu_lib):
    from paper_1911_09278_gb300 import serve
    specs = [(64, 90, 95, 4), (48, 72, 71, 8), (64, 90, 95, 4), (32, 48, 47, 4), (48, 72, 71, 8), (64, 90, 95, 4)]
    reqs = _requests(serve, specs, rate=200.0)
    srv = serve.Server(PARAMS, dtype="f32", sv_size=8, max_active=4, max_iter=6000)
    mixed = srv.run(reqs)
    alone, alone_iters = {}, {}
    for r in reqs:
        one = srv.run([r._replace(arrival=0.0)], serial=True)
        alone[r.rid] = one["results"][r.rid]["x"]
        alone_iters[r.rid] = one["results"][r.rid]["iters"]
    for r in reqs:
        got = mixed["results"][r.rid]
        assert got["converged"], r.rid
        assert got["iters"] == alone_iters[r.rid], r.rid
        assert nrmse(got["x"], alone[r.rid]) < 1e-6, r.rid
    # and one of them against the oracle's MAP image
    r = reqs[3]
    P = oracle.Problem(r.nx, r.ny, r.n_views, r.n_channels, r.y, r.lam, n_agents=r.n_agents, prior="qggmrf",
                       sigma_x=r.sigma_x)
    xs, _, _ = P.central_icd(max_sweeps=20000, tol=1e-13)
    assert nrmse(mixed["results"][r.rid]["x"], xs) < 1e-4
    print("served: %.2f recons/s, p50 %.3f s, p99 %.3f s" % (mixed["recons_per_s"], mixed["p50"], mixed["p99"]))
    srv.close()


def test_grouped_serving_equals_alone(gpu_lib):
    """Grouped serving (all active requests in one group, their ICD passes
    in one queue-fed launch per pass): every image equals the request
    reconstructed alone in grouped mode, and the iteration counts agree."""
    from paper_1911_09278_gb300 import serve
    specs = [(64, 90, 95, 4), (48, 72, 71, 8), (64, 90, 95, 16), (32, 48, 47, 4), (48, 72, 71, 8), (64, 90, 95, 4)]
    reqs = _requests(serve, specs, rate=200.0)
    srv = serve.Server(PARAMS, dtype="f32", sv_size=8, max_active=4, max_iter=6000)
    mixed = srv.run(reqs, grouped=True)
    assert not mixed["failed"]
    for r in reqs:
        one = srv.run([r._replace(arrival=0.0)], grouped=True)["results"][r.rid]
        got = mixed["results"][r.rid]
        assert got["converged"], r.rid
        assert got["iters"] == one["iters"], (r.rid, got["iters"], one["iters"])
        assert np.array_equal(got["x"], one["x"]), r.rid
    print("grouped: %.2f recons/s, p50 %.3f s, p99 %.3f s" % (mixed["recons_per_s"], mixed["p50"], mixed["p99"]))
    srv.close()


def test_admission_respects_budget(gpu_lib):
    """With a budget that holds one request at a time the server still
    finishes every request, one after another."""
    from paper_1911_09278_gb300 import serve
    specs = [(32, 48, 47, 4)] * 3
    reqs = _requests(serve, specs, rate=1000.0)
    one = serve.state_bytes(32, 32, 48, 47, 4)
    srv = serve.Server(PARAMS, dtype="f32", sv_size=8, max_active=3, budget=0, max_iter=6000)
    out = srv.run(reqs)
    assert len(out["results"]) == 3
    starts = sorted((d["start"], d["finish"]) for d in out["results"].values())
    for (s0, f0), (s1, f1) in zip(starts, starts[1:]):
        assert s1 >= f0 - 1e-9          # never two at once
    assert one > 0
    srv.close()
