"""Host logic of the sweep-configuration autotuner, on the CPU: the
iterations-to-tolerance extrapolation against closed forms, and the choice
among candidates with a fake library whose residuals contract at set rates
and whose iterations cost set times on a fake clock."""
import math

import numpy as np
import pytest

import paper_1911_09278_gb300 as mace
from paper_1911_09278_gb300 import autotune


def test_estimate_matches_the_geometric_closed_form():
    r0, q, tol = 0.1, 0.9, 1e-7
    traj = [(k, r0 * q ** k) for k in range(10, 110, 10)]
    exact = math.log(tol / r0) / math.log(q)
    assert autotune.estimate_iterations(traj, tol) == pytest.approx(exact, rel=1e-9)


def test_estimate_uses_the_tail_of_the_probe():
    # a fast transient, then the asymptotic rate 0.97
    traj = [(k, (0.5 * 0.5 ** k if k < 40 else 0.0) + 1e-2 * 0.97 ** k) for k in range(10, 210, 10)]
    tol = 1e-8
    exact = math.log(tol / 1e-2) / math.log(0.97)
    assert autotune.estimate_iterations(traj, tol) == pytest.approx(exact, rel=1e-3)


def test_estimate_special_cases():
    assert autotune.estimate_iterations([(10, 1e-3), (20, 1e-6), (30, 1e-9)], 1e-5) == 20
    assert autotune.estimate_iterations([(10, 1e-3), (20, 1e-3), (30, 2e-3)], 1e-5) == math.inf
    assert autotune.estimate_iterations([(10, 1e-3)], 1e-5) == math.inf
    assert autotune.estimate_iterations([(10, float("nan")), (20, 1e-3)], 1e-5) == math.inf


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeLib:
    """Per (sv_size, chains used): seconds per iteration and contraction rate.
    sv_size 16 is rejected; chains above what the batch allows are lowered,
    as the library does."""

    def __init__(self, cfg, clock):
        self.cfg = cfg
        self.clock = clock
        self.open_sm = 0
        self.open_st = 0

    def build(self, nx, ny, V, D, N, view_agent=None, dtype="f32", sv_size=8, stream=None):
        if sv_size == 16:
            raise mace.MaceError(mace.MACE_EINVAL, "unsupported super-voxel size")
        self.open_sm += 1
        lib = self

        class SM:
            sv = sv_size

            def close(self):
                lib.open_sm -= 1
        return SM()

    def init(self, sm, y, lam, prm, stream=None, batch=1):
        chains = prm["chains"] if batch % max(1, prm["chains"]) == 0 else 1
        wpv = prm.get("warps_per_voxel", 0) or 1
        key = (sm.sv, chains) if prm.get("schedule", 0) == 0 else (sm.sv, chains, 1, wpv)
        sec, q = self.cfg[key]
        lib = self
        lib.open_st += 1

        class St:
            it = 0

            def stats(self):
                return dict(chains=chains, warps_per_voxel=wpv, concurrency=7)

            def iterate(self, k):
                self.it += k
                lib.clock.t += sec * k
                r = 1e-2 * q ** self.it
                if r > 1e3:
                    raise mace.MaceError(mace.MACE_ENUMERIC, "non-finite Mann residual (divergence)")
                return r, r < prm["tol"]

            def close(self):
                lib.open_st -= 1
        return St()


@pytest.fixture
def fake(monkeypatch):
    def make(cfg):
        clock = Clock()
        lib = FakeLib(cfg, clock)
        monkeypatch.setattr(autotune, "mace_build_sysmatrix", lib.build)
        monkeypatch.setattr(autotune, "mace_init", lib.init)
        monkeypatch.setattr(autotune, "make_params", lambda **kw: kw)
        return lib, clock
    return make


def test_tune_picks_the_least_time_to_tolerance(fake):
    cfg = {(4, 1): (2.0e-3, 0.95), (4, 2): (1.5e-3, 0.95), (8, 1): (1.0e-3, 0.99), (8, 2): (0.8e-3, 1.3)}
    lib, clock = fake(cfg)
    tol = 1e-9
    best, table = autotune.tune(64, 64, 90, 95, 4, None, None, dict(tol=tol), batch=2,
                                probe_iters=100, chunk=10, clock=clock)
    assert (best["sv_size"], best["chains"]) == (4, 2)
    rows = {(r["sv_size"], r["chains_asked"]): r for r in table}
    assert len(table) == len(autotune.DEFAULT_CANDIDATES)
    # time per reconstruction = seconds per iteration x iterations / batch
    k_star = math.log(tol / 1e-2) / math.log(0.95)
    assert rows[(4, 2)]["est_iterations"] == pytest.approx(k_star, rel=1e-6)
    assert rows[(4, 2)]["est_s_per_recon"] == pytest.approx(1.5e-3 * k_star / 2, rel=1e-6)
    assert rows[(4, 2)]["ms_per_iteration"] == pytest.approx(1.5, rel=1e-9)
    assert rows[(8, 2)]["error"].startswith("diverged")
    assert lib.open_sm == 0 and lib.open_st == 0


def test_tune_reports_rejected_candidates(fake):
    lib, clock = fake({(8, 1): (1e-3, 0.9)})
    best, table = autotune.tune(64, 64, 90, 95, 4, None, None, dict(tol=1e-6), batch=1,
                                candidates=[autotune.Candidate(16, 1), autotune.Candidate(8, 1)], clock=clock)
    assert "unsupported" in table[0]["error"]
    assert best is table[1]
    assert lib.open_sm == 0 and lib.open_st == 0


def test_tune_calls_match_the_binding():
    """The calls the tuner makes bind to the real binding's signatures."""
    import inspect
    inspect.signature(mace.mace_build_sysmatrix).bind(64, 64, 90, 95, 4, view_agent=None, dtype="f32",
                                                      sv_size=8, stream=None)
    inspect.signature(mace.mace_init).bind(None, None, None, None, stream=None, batch=2)
    prm = mace.make_params(**dict(dict(prior="quadratic", sigma_x=1.0, sigma=0.5, tol=1e-7), chains=2))
    assert prm.chains == 2
    for name in ("iterate", "stats", "close"):
        assert callable(getattr(mace.State, name))


def test_tune_marks_resolved_duplicates_and_stops_at_convergence(fake):
    cfg = {(4, 1): (1e-3, 0.5), (8, 1): (1e-3, 0.8)}
    lib, clock = fake(cfg)
    best, table = autotune.tune(64, 64, 90, 95, 4, None, None, dict(tol=1e-6), batch=1,
                                candidates=[autotune.Candidate(4, 1), autotune.Candidate(4, 2),
                                            autotune.Candidate(8, 1)], clock=clock)
    assert table[1]["chains"] == 1 and table[1]["duplicate_of"] == 0
    # (4, 1) passes tol within the probe: the first chunk below it counts
    first_below = next(k for k in range(20, 200, 10) if 1e-2 * 0.5 ** k < 1e-6)
    assert table[0]["est_iterations"] == first_below
    assert table[0]["probe_iterations"] == first_below - 10
    assert best is table[0]
    assert lib.open_sm == 0 and lib.open_st == 0


def test_tune_rejects_a_probe_shorter_than_two_chunks(fake):
    fake({})
    with pytest.raises(ValueError):
        autotune.tune(8, 8, 4, 5, 1, None, None, dict(tol=1e-6), probe_iters=10, chunk=10)


def test_tune_ranks_schedules_and_warp_teams(fake):
    """Wide agents: the queue-fed schedule with teams of warps per
    super-voxel competes with the fixed schedule; the fastest to tolerance
    wins and the row records the team size the library used."""
    cands = autotune.candidates_for(180)
    assert autotune.Candidate(4, 1, 1, 4) in cands and autotune.Candidate(8, 1, 1, 2) in cands
    assert autotune.Candidate(4, 1, 1, 4) not in autotune.candidates_for(45)
    cfg = {k[:2] if k.schedule == 0 else (k.sv_size, k.chains, 1, k.warps_per_voxel): (2e-3, 0.9) for k in cands}
    cfg[(4, 1, 1, 4)] = (1e-3, 0.9)
    lib, clock = fake(cfg)
    best, table = autotune.tune(64, 64, 720, 95, 4, None, None, dict(tol=1e-6), batch=1, candidates=cands,
                                clock=clock)
    assert (best["sv_size"], best["schedule"], best["warps_per_voxel"]) == (4, 1, 4)
    assert lib.open_sm == 0 and lib.open_st == 0
