"""Autotuner for the sweep configuration of one scan geometry.

Four settings trade sweep speed against convergence:
- the super-voxel size S, the side of the tile one warp updates. It sets the
  warp's working set and how stale concurrent updates are.
- the chains per warp, the reconstructions of a batch that share each column
  load. With two chains each half-warp serves one reconstruction.
- the schedule (fixed warps per pair, or a persistent grid fed from a work
  queue) and, with the queue, the warps per super-voxel: a team of 2 or 4
  warps splitting an agent's views, for agents with many views.
- the concurrency, the super-voxels of one agent in flight (rows of
  super-voxels by default).

The fixed point depends on none of them (Theorem 1), so they are chosen by
measurement. For each candidate the tuner:
1. builds the system matrix (once per S);
2. runs a short probe of Mann iterations on the caller's scans, timed on the
   host clock (mace_iterate returns once the GPU has finished);
3. extrapolates the iterations to the tolerance from the contraction rate of
   the Mann residual over the probe's second half.

The candidate with the least estimated time per reconstruction wins. A
candidate is reported with its reason instead when the library rejects it (a
size it does not instantiate, a working set that does not fit) or when it
diverges. Every step of the method runs in libmace.so; this module only
orchestrates.
"""
import collections
import math
import time

import numpy as np

from . import MACE_ENUMERIC, MaceError, mace_build_sysmatrix, mace_init, make_params

# schedule, warps_per_voxel: as make_params; concurrency None keeps the
# caller's
Candidate = collections.namedtuple("Candidate", "sv_size chains schedule warps_per_voxel concurrency",
                                   defaults=(0, 0, None))
# the sizes and chain counts the GPU tests cover; 16 x 16 super-voxels (one
# chain) are built by the library and may be passed explicitly
DEFAULT_CANDIDATES = tuple(Candidate(s, k) for s in (4, 8) for k in (1, 2))


def candidates_for(views_per_agent):
    """The default candidates plus the work-queue schedule (one chain), and
    for agents of more than 128 views teams of 2 and 4 warps per
    super-voxel."""
    out = list(DEFAULT_CANDIDATES) + [Candidate(s, 1, 1, 1) for s in (4, 8)]
    if views_per_agent > 128:
        out += [Candidate(s, 1, 1, w) for s in (4, 8) for w in (2, 4)]
    return tuple(out)


def estimate_iterations(traj, tol, tail=0.5):
    """Iterations until the relative Mann residual falls below tol.

    traj is the probe trajectory [(iteration, residual), ...] in increasing
    iteration order. If the probe already reached tol, returns the first
    iteration below it. Otherwise fits log r = a + k log q by least squares
    over the last `tail` fraction of the points (at least two) and
    extrapolates from the last point. Returns math.inf when the fitted rate
    does not contract (q >= 1)."""
    for it, r in traj:
        if r < tol:
            return float(it)
    pts = [(it, r) for it, r in traj if r > 0 and math.isfinite(r)]
    if len(pts) < 2:
        return math.inf
    pts = pts[-max(2, int(math.ceil(len(pts) * tail))):]
    k = np.array([p[0] for p in pts], np.float64)
    slope = float(np.polyfit(k, np.log([p[1] for p in pts]), 1)[0])
    if not slope < 0.0:
        return math.inf
    it_last, r_last = pts[-1]
    return it_last + math.log(tol / r_last) / slope


def tune(nx, ny, n_views, n_channels, n_agents, y, lam, params, batch=1, candidates=DEFAULT_CANDIDATES,
         dtype="f32", view_agent=None, probe_iters=100, chunk=10, stream=None, clock=time.perf_counter):
    """Choose (sv_size, chains) for these scans.

    params: keyword arguments for make_params. Its tol is the target;
    `chains` is set per candidate. y, lam: as for mace_init with `batch`
    reconstructions.

    Returns (best, table). best is the winning table row, or None if no
    candidate contracts. Each table row holds sv_size, chains_asked,
    chains (as used by the library), ms_per_iteration, probe_iterations,
    trajectory, est_iterations and est_s_per_recon, or `error` with the
    reason. A candidate that resolves to the same configuration as an
    earlier one is marked `duplicate_of`."""
    if probe_iters < 2 * chunk:
        raise ValueError("probe_iters must cover at least two chunks")
    tol = params.get("tol", 1e-5)
    table = []
    seen = {}
    matrices = {}
    try:
        for c in candidates:
            row = dict(sv_size=c.sv_size, chains_asked=c.chains, schedule=c.schedule,
                       warps_per_voxel_asked=c.warps_per_voxel)
            if c.concurrency is not None:
                row["concurrency_asked"] = c.concurrency
            table.append(row)
            st = None
            try:
                sm = matrices.get(c.sv_size)
                if sm is None:
                    sm = mace_build_sysmatrix(nx, ny, n_views, n_channels, n_agents, view_agent=view_agent,
                                              dtype=dtype, sv_size=c.sv_size, stream=stream)
                    matrices[c.sv_size] = sm
                kw = dict(params, chains=c.chains, schedule=c.schedule, warps_per_voxel=c.warps_per_voxel)
                if c.concurrency is not None:
                    kw["concurrency"] = c.concurrency
                st = mace_init(sm, y, lam, make_params(**kw), stream=stream, batch=batch)
                info = st.stats()
                row["chains"] = info["chains"]
                row["warps_per_voxel"] = info.get("warps_per_voxel", 1)
                row["concurrency"] = info.get("concurrency")
                key = (c.sv_size, row["chains"], c.schedule, row["warps_per_voxel"], row["concurrency"])
                if key in seen:
                    row["duplicate_of"] = seen[key]
                    continue
                seen[key] = len(table) - 1
                st.iterate(chunk)   # first launch: graph capture, caches
                traj = []
                done = chunk
                t0 = clock()
                while done < chunk + probe_iters:
                    r, conv = st.iterate(chunk)
                    done += chunk
                    traj.append((done, r))
                    if conv:
                        break
                elapsed = clock() - t0
                timed = done - chunk
                row["ms_per_iteration"] = 1e3 * elapsed / timed
                row["probe_iterations"] = timed
                row["trajectory"] = traj
                est = estimate_iterations(traj, tol)
                row["est_iterations"] = est
                row["est_s_per_recon"] = (elapsed / timed) * est / batch
            except MaceError as e:
                row["error"] = ("diverged: " if e.code == MACE_ENUMERIC else "") + str(e)
            finally:
                if st is not None:
                    st.close()
    finally:
        for sm in matrices.values():
            sm.close()
    ok = [r for r in table
          if "error" not in r and "duplicate_of" not in r and math.isfinite(r["est_s_per_recon"])]
    best = min(ok, key=lambda r: r["est_s_per_recon"]) if ok else None
    return best, table
