"""Continuous-batching reconstruction server over the C ABI.

Requests (a scan: geometry, partition, y, Lambda) arrive over time.  Each
admitted request gets its own reconstruction state on its own CUDA stream;
the server enqueues its Mann iterations in short chunks (mace_launch), so the
iterations of every active request run on the GPU at the same time.  Each
request keeps two chunks queued: after one chunk a status copy is enqueued
(mace_poll_async) and the server checks it without waiting
(mace_poll_ready); when it lands, the next chunk is queued behind the one
still running, so no stream waits on the host.  Converged requests are
retired (consensus image copied to the host; they ran one chunk past the
point where convergence was seen) and waiting ones admitted as slots and
device memory free up.  Stored system matrices are shared by every request
with the same geometry and partition and stay resident.

Grouped mode (grouped=True) advances every active request in one group
(mace_group_*): each chunk is one series of launches on one stream whose ICD
passes are single queue-fed launches over the items of all requests, so
small requests share the GPU's warps instead of each holding a fixed grid.
Membership follows admission and retirement (mace_group_update, stream
ordered); one chunk stays queued behind the one whose status is read.  Every
member advances one pass per launch and a pass lasts as long as its longest
item, so on mixes dominated by large requests the per-request mode (the
default) serves faster; measured on a GB300 it does on small requests too.

Admission is by device-memory footprint: the request's state (the library's
own count, mace_state_bytes, once its geometry's matrix is resident) plus,
for a new geometry, its system matrix must fit the budget next to what is
resident.
This module only orchestrates; every step of a reconstruction runs in
libmace.so.
"""
import collections
import time

import numpy as np

from . import (MaceError, Sysmatrix, load, make_params, mace_build_sysmatrix, mace_group_create,  # noqa: F401
               mace_init, mace_state_bytes)

Request = collections.namedtuple(
    "Request", "rid arrival nx ny n_views n_channels n_agents y lam sigma_x view_agent")


def state_bytes(nx, ny, n_views, n_channels, n_agents):
    """Estimated device bytes of one reconstruction state, for a geometry
    whose system matrix is not built yet (then the library's exact count,
    mace_state_bytes, is not available): per measurement (e, Lambda), the
    fixed-point accumulator of changes of e and y; per agent and pixel w, X
    and theta2; the FP64 consensus; the host inputs' staging during
    mace_init; and a margin for the small buffers."""
    m = n_views * n_channels
    n = nx * ny
    return m * (8 + 8 + 4 + 8) + n_agents * n * (4 + 4 + 4) + n * 8 + (1 << 20)


class Server:
    """Host-side scheduler; see the module docstring.

    params: keyword arguments for make_params (sigma_x comes per request).
    sv_size: super-voxel side, or "auto": 4 for agents of more than 64 views
    (more, smaller items in flight: faster for the wide agents of large
    scans with few agents, measured), else 8.  max_active: requests on the
    GPU at once.  budget: device bytes the server may hold (system matrices
    + states).  chunk: iterations enqueued per request between polls."""

    def __init__(self, params, dtype="bf16", sv_size=8, max_active=8, budget=64 << 30,
                 chunk=10, max_iter=4000):
        import torch
        self.torch = torch
        self.params = dict(params)
        self.dtype = dtype
        self.sv_size = sv_size
        self.max_active = max_active
        self.budget = budget
        self.chunk = chunk
        self.max_iter = max_iter
        self.matrices = {}      # geometry key -> Sysmatrix
        self.matrix_bytes = {}

    def _sv(self, r):
        if self.sv_size != "auto":
            return self.sv_size
        return 4 if r.n_views > 64 * r.n_agents else 8

    def _key(self, r):
        va = None if r.view_agent is None else bytes(np.asarray(r.view_agent, np.int32))
        return (r.nx, r.ny, r.n_views, r.n_channels, r.n_agents, va, self._sv(r))

    def _resident(self):
        return sum(self.matrix_bytes.values())

    def _matrix(self, r):
        k = self._key(r)
        if k not in self.matrices:
            sm = mace_build_sysmatrix(r.nx, r.ny, r.n_views, r.n_channels, r.n_agents,
                                      view_agent=r.view_agent, dtype=self.dtype, sv_size=self._sv(r))
            info = sm.info()
            self.matrices[k] = sm
            self.matrix_bytes[k] = info["bytes_columns"] + info["bytes_meta"]
        return self.matrices[k]

    def _matrix_estimate(self, r):
        # per (pixel, view): a header byte and two values, and for about 27 %
        # of them a third value with its 2-byte list entry; 16-byte column
        # padding; offsets and band descriptors
        vb = 4 if self.dtype == "f32" else 2
        n = r.nx * r.ny
        return int(n * r.n_views * (1 + 2 * vb + 0.3 * (2 + vb)) * 1.05 + n * r.n_agents * 12)

    def _params(self, r, grouped=False):
        kw = dict(self.params)
        if grouped:
            kw["schedule"] = 1
        return make_params(sigma_x=r.sigma_x, max_iter=self.max_iter, **kw)

    def _state_need(self, r, grouped=False):
        """(bytes to admit, bytes held while active) of request r's state: the
        library's count when its matrix is resident, else the estimate."""
        k = self._key(r)
        if k in self.matrices:
            persistent, peak = mace_state_bytes(self.matrices[k], self._params(r, grouped), batch=1)
            return peak, persistent
        est = state_bytes(r.nx, r.ny, r.n_views, r.n_channels, r.n_agents)
        return est + self._matrix_estimate(r), est

    def _admit(self, pending, active, t, limit, grouped, failed, now, t0):
        """Admit waiting requests that have arrived while slots and the
        budget allow; returns the new entries (state initialised on its own
        stream).  Requests the library rejects go to `failed`."""
        torch = self.torch
        new = []
        while pending and pending[0].arrival <= t and len(active) + len(new) < limit:
            r = pending[0]
            need, _ = self._state_need(r, grouped)
            held = self._resident() + sum(a["bytes"] for a in active + new)
            if held + need > self.budget and (active or new):
                break
            pending.popleft()
            st = None
            try:
                sm = self._matrix(r)
                stream = torch.cuda.Stream()
                st = mace_init(sm, r.y, r.lam, self._params(r, grouped), stream=stream)
            except MaceError as e:
                failed[r.rid] = dict(error=str(e), code=e.code, finish=now() - t0)
                if st is not None:
                    st.close()
                continue
            new.append(dict(req=r, st=st, stream=stream, start=now() - t0, seen=0,
                            bytes=self._state_need(r, grouped)[1]))
        return new

    def _retire(self, a, r_, conv, done, now, t0):
        st = a["st"]
        x = st.consensus()
        fin = now() - t0
        done[a["req"].rid] = dict(x=x, iters=st.stats()["iters"], residual=r_, converged=conv,
                                  latency=fin - a["req"].arrival, finish=fin, start=a["start"])
        st.close()

    def _run_grouped(self, requests, now):
        """Grouped mode (see the module docstring).  Each cycle waits for
        the status copies enqueued behind chunk k while chunk k+1 runs; then
        it retires the converged members (their image is read after chunk
        k+1), enqueues the status copies of chunk k+1, launches chunk k+2
        for the members left, and admits new requests into the freed slots
        and memory; those join the next launch."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        active, done, failed = [], {}, {}
        stream = torch.cuda.Stream()
        group = None
        polled = []         # members whose status copy of the chunk before last is in flight
        t0 = now()

        def relaunch(members):
            nonlocal group
            sts = [a["st"] for a in members]
            if group is None:
                group = mace_group_create(sts, stream=stream)
            else:
                group.update(sts)
            group.launch(self.chunk)

        while pending or active:
            if not polled:
                # start (or restart) the pipeline: chunk, status copies, chunk
                active += self._admit(pending, active, now() - t0, self.max_active, True, failed, now, t0)
                if not active:
                    if pending:
                        time.sleep(max(0.0, min(0.01, pending[0].arrival - (now() - t0))))
                    continue
                relaunch(active)
                for a in active:
                    a["st"].poll_async()
                    a["seen"] = a["st"].stats()["iters"]
                polled = list(active)
                group.launch(self.chunk)
                continue
            # the status copies, without blocking the host
            got = {}
            while len(got) < len(polled):
                for k, a in enumerate(polled):
                    if k in got:
                        continue
                    try:
                        ready, r_, conv = a["st"].poll_ready()
                    except MaceError as e:
                        got[k] = e
                        continue
                    if ready:
                        got[k] = (r_, conv)
                if len(got) < len(polled):
                    time.sleep(0.0002)
            keep, retire = [], []
            for k, a in enumerate(polled):
                res = got[k]
                if isinstance(res, MaceError):
                    # divergence or a timed-out wait: retire it, serve the rest
                    failed[a["req"].rid] = dict(error=str(res), code=res.code, finish=now() - t0, start=a["start"])
                    retire.append((a, None))
                elif res[1] or a["seen"] >= self.max_iter:
                    retire.append((a, res))
                else:
                    keep.append(a)
            keep += [a for a in active if not any(a is p for p in polled)]    # admitted last cycle
            polled = []
            for a in keep:
                if a["st"].stats()["iters"] > 0:
                    a["st"].poll_async()
                    a["seen"] = a["st"].stats()["iters"]
                    polled.append(a)
            if keep:
                relaunch(keep)
            # retire (the image read waits for the chunk before last; the
            # chunk just launched keeps the GPU busy), then admit into the
            # freed slots and memory: the new requests join the next launch
            for a, res in retire:
                if res is None:
                    a["st"].close()
                else:
                    self._retire(a, res[0], res[1], done, now, t0)
            active = keep + self._admit(pending, keep, now() - t0, self.max_active, True, failed, now, t0)
        if group is not None:
            group.close()
        return self._summary(requests, done, failed)

    def _summary(self, requests, done, failed):
        makespan = max(d["finish"] for d in done.values()) if done else 0.0
        lat = np.array([d["latency"] for d in done.values()])
        first = min(r.arrival for r in requests) if requests else 0.0
        return dict(results=done, failed=failed, recons_per_s=len(done) / max(1e-9, makespan - first),
                    p50=float(np.percentile(lat, 50)) if len(lat) else None,
                    p99=float(np.percentile(lat, 99)) if len(lat) else None,
                    makespan=makespan)

    def run(self, requests, serial=False, grouped=False, now=time.perf_counter):
        """Serve `requests` (arrival times in seconds from the start).  With
        serial=True one request at a time (the plain GPU form); grouped=True
        advances all active requests in one group.  Returns a dict with
        per-request results, `failed` (requests the library rejected or that
        diverged, with the error; the others are served on) and throughput /
        latency figures over the completed requests."""
        if grouped and not serial:
            return self._run_grouped(requests, now)
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        active = []
        done = {}
        failed = {}     # requests the library rejected or that diverged
        t0 = now()
        while pending or active:
            t = now() - t0
            # admission
            limit = 1 if serial else self.max_active
            while pending and pending[0].arrival <= t and len(active) < limit:
                r = pending[0]
                need, _ = self._state_need(r)
                held = self._resident() + sum(a["bytes"] for a in active)
                if held + need > self.budget and active:
                    break
                pending.popleft()
                st = None
                try:
                    sm = self._matrix(r)
                    stream = torch.cuda.Stream()
                    prm = self._params(r)
                    st = mace_init(sm, r.y, r.lam, prm, stream=stream)
                    # first chunk, its status copy, and the next chunk behind it
                    st.launch(self.chunk)
                    st.poll_async()
                    seen = self.chunk
                    if seen < self.max_iter:
                        st.launch(self.chunk)
                except MaceError as e:
                    failed[r.rid] = dict(error=str(e), code=e.code, finish=now() - t0)
                    if st is not None:
                        st.close()
                    continue
                active.append(dict(req=r, st=st, stream=stream, start=now() - t0, seen=seen,
                                   bytes=self._state_need(r)[1]))
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - (now() - t0))))
                continue
            still = []
            progressed = False
            for a in active:
                st = a["st"]
                try:
                    ready, r_, conv = st.poll_ready()
                    if not ready:
                        still.append(a)
                        continue
                    progressed = True
                    if conv or a["seen"] >= self.max_iter:
                        x = st.consensus()
                        fin = now() - t0
                        done[a["req"].rid] = dict(x=x, iters=st.stats()["iters"], residual=r_, converged=conv,
                                                  latency=fin - a["req"].arrival, finish=fin,
                                                  start=a["start"])
                        st.close()
                        continue
                    # status of the chunk queued behind, then one more chunk
                    st.poll_async()
                    a["seen"] = st.stats()["iters"]
                    if a["seen"] < self.max_iter:
                        st.launch(self.chunk)
                    still.append(a)
                except MaceError as e:
                    # divergence (non-finite residual), a timed-out wait or a
                    # CUDA error: retire this request, keep serving the rest
                    progressed = True
                    failed[a["req"].rid] = dict(error=str(e), code=e.code, finish=now() - t0,
                                                start=a["start"])
                    st.close()
            active = still
            if not progressed:
                time.sleep(0.0002)
        return self._summary(requests, done, failed)

    def close(self):
        for sm in self.matrices.values():
            sm.close()
        self.matrices.clear()
        self.matrix_bytes.clear()
