"""Host logic of the continuous-batching server, on the CPU: admission by
slots and memory budget, arrival order, two chunks queued per request,
retirement one chunk after convergence is seen, serial mode.  The library
calls are replaced by a fake state whose residual falls below tol after a
set number of iterations; no GPU work is involved."""
import sys
import types

import numpy as np
import pytest

from paper_1911_09278_gb300 import serve


class FakeState:
    log = []

    def __init__(self, req_id, conv_at):
        self.rid = req_id
        self.conv_at = conv_at
        self.iters = 0
        self.polled_at = None
        self.ready_calls = 0
        self.closed = False

    def launch(self, k):
        assert not self.closed
        self.iters += k
        FakeState.log.append(("launch", self.rid, self.iters))

    def poll_async(self):
        self.polled_at = self.iters

    def poll_ready(self):
        # every other query finds the copy still in flight
        self.ready_calls += 1
        if self.ready_calls % 2:
            return False, 0.0, False
        if self.conv_at == -1:
            raise serve.MaceError(-6, "non-finite Mann residual (divergence)")
        r = 1e-9 if self.polled_at >= self.conv_at else 1.0
        return True, r, r < 1e-6

    def stats(self):
        return dict(iters=self.iters)

    def consensus(self):
        FakeState.log.append(("retire", self.rid, self.iters))
        return np.full((4, 4), float(self.rid), np.float32)

    def close(self):
        self.closed = True


@pytest.fixture
def fake_server(monkeypatch):
    """A Server whose library calls are fakes; mace_init gets the request's
    iterations to convergence from y[0, 0]."""
    FakeState.log = []
    active = {"now": 0, "max": 0}

    def fake_init(sm, y, lam, prm, stream=None):
        if int(y[0, 0]) == -2:
            raise serve.MaceError(-1, "y and weights must be finite and weights >= 0")
        st = FakeState(int(lam[0, 0]), int(y[0, 0]))
        active["now"] += 1
        active["max"] = max(active["max"], active["now"])
        orig_close = st.close

        def close():
            active["now"] -= 1
            orig_close()
        st.close = close
        return st

    monkeypatch.setattr(serve, "mace_init", fake_init)
    monkeypatch.setattr(serve, "make_params", lambda **kw: kw)
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Stream=lambda: None))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)

    def make(max_active=3, budget=1 << 40, chunk=10, max_iter=200):
        srv = serve.Server(dict(prior="quadratic"), max_active=max_active, budget=budget, chunk=chunk,
                           max_iter=max_iter)
        srv._matrix = lambda r: None
        srv.matrix_bytes = {}
        return srv
    return make, active


def _requests(conv_iters, arrivals=None):
    reqs = []
    for k, c in enumerate(conv_iters):
        y = np.full((2, 3), float(c), np.float32)
        lam = np.full((2, 3), float(k), np.float32)
        t = 0.0 if arrivals is None else arrivals[k]
        reqs.append(serve.Request(k, t, 4, 4, 2, 3, 2, y, lam, 1.0, None))
    return reqs


def test_each_request_retires_one_chunk_after_convergence(fake_server):
    make, active = fake_server
    srv = make(max_active=3, chunk=10)
    out = srv.run(_requests([30, 50, 20, 40, 10]))
    assert sorted(out["results"]) == [0, 1, 2, 3, 4]
    for rid, conv in enumerate([30, 50, 20, 40, 10]):
        d = out["results"][rid]
        assert d["converged"]
        # convergence is seen on the status after `conv` iterations; the chunk
        # queued behind it has run when the image is read
        assert d["iters"] == conv + 10
        assert float(d["x"][0, 0]) == rid
    assert active["max"] == 3


def test_slots_and_budget_limit_admission(fake_server):
    make, active = fake_server
    one = serve.state_bytes(4, 4, 2, 3, 2)
    srv = make(max_active=8, budget=2 * one + one // 2)
    srv._matrix_estimate = lambda r: 0
    out = srv.run(_requests([20] * 5))
    assert len(out["results"]) == 5
    assert active["max"] == 2          # the budget holds two states


def test_admission_uses_the_library_footprint(fake_server, monkeypatch):
    """Once a geometry's matrix is resident, admission counts the library's
    own footprint of a state (mace_state_bytes: the peak during mace_init to
    admit, the persistent bytes while active)."""
    make, active = fake_server
    calls = []

    def fake_state_bytes(sm, prm, batch=1, inputs_on_device=False):
        calls.append(batch)
        return 1000, 1500
    monkeypatch.setattr(serve, "mace_state_bytes", fake_state_bytes)
    srv = make(max_active=8, budget=2 * 1000 + 1500 - 1)
    reqs = _requests([20] * 5)
    srv.matrices[srv._key(reqs[0])] = object()
    out = srv.run(reqs)
    assert len(out["results"]) == 5 and calls
    assert active["max"] == 2          # 1000 + 1000 held, a third needs 1500 more


def test_serial_mode_is_one_at_a_time_in_arrival_order(fake_server):
    make, active = fake_server
    srv = make(max_active=4)
    out = srv.run(_requests([20, 10, 30], arrivals=[0.0, 0.001, 0.002]), serial=True)
    assert active["max"] == 1
    order = [rid for kind, rid, _ in FakeState.log if kind == "retire"]
    assert order == [0, 1, 2]
    starts = sorted((d["start"], d["finish"]) for d in out["results"].values())
    for (s0, f0), (s1, f1) in zip(starts, starts[1:]):
        assert s1 >= f0 - 1e-9


def test_max_iter_stops_an_unconverged_request(fake_server):
    make, active = fake_server
    srv = make(max_active=2, chunk=10, max_iter=60)
    out = srv.run(_requests([10 ** 6, 20]))
    d = out["results"][0]
    assert not d["converged"]
    assert d["iters"] == 60
    assert out["results"][1]["converged"]


def test_failed_requests_are_retired_and_the_rest_served(fake_server):
    make, active = fake_server
    srv = make(max_active=3, chunk=10)
    # request 1 is rejected by mace_init, request 3 diverges on the GPU
    out = srv.run(_requests([20, -2, 30, -1, 10]))
    assert sorted(out["results"]) == [0, 2, 4]
    assert sorted(out["failed"]) == [1, 3]
    assert out["failed"][1]["code"] == -1 and out["failed"][3]["code"] == -6
    for rid in (0, 2, 4):
        assert out["results"][rid]["converged"]
    assert active["now"] == 0          # every state that was made is closed


class FakeGroup:
    log = []

    def __init__(self, states, stream=None):
        self.states = list(states)
        self.closed = False
        FakeGroup.log.append(("create", [st.rid for st in self.states]))

    def update(self, states):
        assert not self.closed
        self.states = list(states)
        FakeGroup.log.append(("update", [st.rid for st in self.states]))

    def launch(self, k):
        assert not self.closed
        for st in self.states:
            assert not st.closed, "a retired state is still a member"
            st.launch(k)

    def close(self):
        self.closed = True


@pytest.fixture
def grouped(fake_server, monkeypatch):
    FakeGroup.log = []
    monkeypatch.setattr(serve, "mace_group_create", lambda states, stream=None: FakeGroup(states, stream))
    return fake_server


def test_grouped_mode_retires_one_chunk_after_convergence(grouped):
    """Grouped serving: every request is served, its image read one chunk
    after the status that showed convergence, never more than max_active at
    once, and no retired state stays in the group."""
    make, active = grouped
    srv = make(max_active=3, chunk=10)
    conv = [30, 50, 20, 40, 10, 60]
    out = srv.run(_requests(conv), grouped=True)
    assert sorted(out["results"]) == list(range(len(conv)))
    for rid, c in enumerate(conv):
        d = out["results"][rid]
        assert d["converged"] and d["iters"] == c + 10, (rid, d["iters"])
        assert float(d["x"][0, 0]) == rid
    assert active["max"] == 3
    sizes = [len(m) for kind, m in FakeGroup.log]
    assert max(sizes) <= 3 and FakeGroup.log[0][0] == "create"


def test_grouped_mode_retires_a_diverged_request_alone(grouped):
    make, active = grouped
    srv = make(max_active=4, chunk=10)
    out = srv.run(_requests([20, -1, 30]), grouped=True)
    assert sorted(out["results"]) == [0, 2]
    assert list(out["failed"]) == [1] and out["failed"][1]["code"] == -6
    assert active["now"] == 0
