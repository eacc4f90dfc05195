"""Benchmark: MACE reconstructions per second on the 512^2 / 720-view /
725-channel / 16-agent Q-GGMRF workload, on one or more GB300s.

A step is one complete partial-update MACE reconstruction (Algorithm 1, the
ICD sweeps of Algorithm 2, the FP64 consensus and the Mann update, iterated
to the Mann-residual tolerance) of a batch of B synthetic scans that share
the stored system matrix.  `value` counts reconstructions per second with the
inputs already in HBM; `e2e` repeats the measurement through the same C-ABI
call with host buffers (pinned-host -> device copies of y and Lambda before,
device -> host copy of the images after, inside the timed region).

--impl reference times the FP64 CPU oracle instead (bounded sample, host
cores).  Under torchrun every rank runs its own independent batch (replicas;
no collective on the data path).
"""
import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# the timed launch configuration (the full-size parity test runs the same)
# 4x4 super-voxels, concurrency -1: one super-voxel row per warp (128
# concurrent super-voxels per agent at 512^2); chains 2: each warp updates
# both scans of the batch in two 16-lane halves over one column load; sigma
# (normalised) and rho from the convergence study recorded with the design
# notes
DEFAULTS = dict(batch=2, concurrency=-1, sigma=0.17, rho=0.95, tol=8e-7, max_iter=4000, sv=4, dtype="f32",
                chains=2, recompute_every=10, forward="auto", deterministic=False)

WORKLOAD = dict(name="parallel-beam 2D 512x512, 720 views over 180 deg, 725 channels, "
                     "16 interleaved agents x 45 views, Q-GGMRF (p=2, q=1.2, T=1), FP32",
                n=512, n_views=720, n_channels=725, n_agents=16)


def sweep_source_sha():
    """sha256 of the ICD sweep kernel's source (the traffic counters in
    profiles/ are only used for the kernel they were taken from)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("common.cuh", "sweep.cuh"):
        with open(os.path.join(ROOT, "paper_1911_09278_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(value, dist, device):
    """The largest value over the ranks (a replica job takes as long as its
    slowest rank); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(batch, rank):
    import synth
    ys, ls = [], []
    for b in range(batch):
        c = synth.make_case(n=WORKLOAD["n"], n_views=WORKLOAD["n_views"], n_channels=WORKLOAD["n_channels"],
                            I0=2e4, mu_max=0.02 * 64 / WORKLOAD["n"], seed=2 + 1000 * rank + 7 * b,
                            noise_seed=102 + 1000 * rank + 7 * b)
        ys.append(c["y"][0])
        ls.append(c["lam"][0])
    y = np.stack(ys).astype(np.float32)
    lam = np.stack(ls).astype(np.float32)
    return y, lam


def oracle_match(x, y, lam, dtype="f32", sx=None, name="cfg2"):
    """Relative RMSE of a reconstruction against the oracle's stored MAP image
    of the same scan (tests/golden/<name>_reference.npz, written by
    tests/golden/make_reference.py from the oracle alone), when the stored
    image's input digest and prior scale match."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", "%s_reference.npz" % name)
    if not os.path.exists(path):
        return {"nrmse_vs_oracle": None, "why": "no stored oracle image"}
    d = np.load(path)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(y, np.float32).tobytes())
    h.update(np.ascontiguousarray(lam, np.float32).tobytes())
    if str(d["digest"]) != h.hexdigest():
        return {"nrmse_vs_oracle": None, "why": "stored oracle image is of other inputs"}
    if sx is not None and abs(float(d["sigma_x"]) - sx) > 1e-6 * abs(sx):
        return {"nrmse_vs_oracle": None, "why": "stored oracle image is of another prior scale"}
    ref = d["x"].reshape(x.shape)
    err = float(np.sqrt(np.mean((x.astype(np.float64) - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))
    return {"nrmse_vs_oracle": err, "bound": 1e-4 if dtype == "f32" else 1e-3, "oracle_kkt": float(d["kkt"]),
            "oracle_iters": int(d["iters"])}


def forward_geometry(args):
    """The e recompute evaluates A from the geometry when the stored values
    are rounded (auto), or as asked."""
    return args.forward == "geometry" or (args.forward == "auto" and args.dtype != "f32")


def forward_param(args):
    """The library's forward_geometry argument for --forward (None: its default)."""
    return None if args.forward == "auto" else args.forward == "geometry"


def solver_params(mace, sigma_x, args):
    return mace.make_params(prior="qggmrf", sigma_x=sigma_x, sigma=args.sigma, sigma_mode=1, rho=args.rho,
                            sweeps_per_iter=2, symmetric=True, recompute_every=args.recompute_every,
                            max_iter=args.max_iter, tol=args.tol, concurrency=args.concurrency, sv_order=0, chains=args.chains,
                            forward_geometry=forward_param(args), deterministic=args.deterministic)


def run_mace(args, rank, world):
    import torch
    import synth
    import paper_1911_09278_gb300 as mace
    from paper_1911_09278_gb300 import build as gbuild

    gbuild.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B = args.batch
    y, lam = make_inputs(B, rank)
    sx = synth.prior_sigma_x(lam[0], WORKLOAD["n_views"], frac=args.prior_frac)
    stream = torch.cuda.Stream()
    sm = mace.mace_build_sysmatrix(WORKLOAD["n"], WORKLOAD["n"], WORKLOAD["n_views"], WORKLOAD["n_channels"],
                                   WORKLOAD["n_agents"], sv_size=args.sv, dtype=args.dtype, stream=stream)
    info = sm.info()
    prm = solver_params(mace, sx, args)
    d_y = torch.from_numpy(y).cuda()
    d_l = torch.from_numpy(lam).cuda()
    d_x = torch.empty((B, WORKLOAD["n"], WORKLOAD["n"]), device="cuda", dtype=torch.float32)
    h_y = torch.from_numpy(y).pin_memory()
    h_l = torch.from_numpy(lam).pin_memory()
    h_x = torch.empty((B, WORKLOAD["n"], WORKLOAD["n"]), dtype=torch.float32).pin_memory()

    iters_seen = []
    timing = {"ms": 0.0, "launches": 0}

    def step(device_inputs, record):
        if device_inputs:
            st = mace.mace_init(sm, d_y, d_l, prm, stream=stream, batch=B)
        else:
            dy = torch.empty_like(d_y)
            dl = torch.empty_like(d_l)
            with torch.cuda.stream(stream):
                dy.copy_(h_y, non_blocking=True)
                dl.copy_(h_l, non_blocking=True)
            st = mace.mace_init(sm, dy, dl, prm, stream=stream, batch=B)
        if record:
            st.set_timing(True, max_launches=2 * args.max_iter + 8)
        x, it, r, conv = st.reconstruct(out=d_x)
        if not device_inputs:
            with torch.cuda.stream(stream):
                h_x.copy_(d_x, non_blocking=True)
        if record:
            ms, n = st.get_timing()
            timing["ms"] += ms
            timing["launches"] += n
        iters_seen.append((it, r, conv))
        st.close()

    def timed(device_inputs, record, warmup):
        for _ in range(warmup):
            step(device_inputs, False)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(device_inputs, record)
        ev1.record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ck = clocks.stop()
        dev_s = ev0.elapsed_time(ev1) / 1000.0
        el = reduce_max(max(dev_s, wall), dist, "cuda")
        return el, ck

    el, clocks = timed(True, True, args.warmup)
    iters_main = [it for it, _, _ in iters_seen[-args.steps:]]
    conv_main = all(c for _, _, c in iters_seen[-args.steps:])
    accuracy = oracle_match(d_x[0].cpu().numpy(), y[0], lam[0], args.dtype, sx)
    if B > 1:
        accuracy = {"scan0": accuracy,
                    "scan1": oracle_match(d_x[1].cpu().numpy(), y[1], lam[1], args.dtype, sx, name="cfg2_scan1")}
    el_e2e, _ = timed(False, False, 1)
    recons = B * args.steps * world
    value = recons / el
    e2e = recons / el_e2e
    hbm, peak_kind = peaks()
    # roofline of the ICD sweep kernel: algorithmic bytes per launch = the
    # stored matrix's content read once for the whole batch (its non-zero
    # values, and one 16-bit run header (first channel, length) per (pixel,
    # view)) + per reconstruction the state it reads and writes (X read and
    # written, w and theta2 read per agent and pixel, the FP64 consensus, the
    # error sinogram and weights read and written once)
    n = WORKLOAD["n"] ** 2
    N = WORKLOAD["n_agents"]
    vbytes = 4 if args.dtype == "f32" else 2
    matrix_bytes = info["nnz"] * vbytes + n * WORKLOAD["n_views"] * 2
    per_recon = N * n * (4 + 4 + 4 + 4) + n * 8 + 2 * WORKLOAD["n_views"] * WORKLOAD["n_channels"] * 8
    alg_bytes = matrix_bytes + B * per_recon
    avg_launch_s = (timing["ms"] / 1000.0) / max(1, timing["launches"])
    achieved = alg_bytes / avg_launch_s / 1e9 if timing["launches"] else None
    traffic = None
    tf = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if os.path.exists(tf):
        try:
            with open(tf) as f:
                tt = json.load(f)
            # counters of this exact kernel source and launch configuration only
            if (tt.get("batch") == B and tt.get("sv") == args.sv and tt.get("dtype") == args.dtype
                    and tt.get("chains") == args.chains and tt.get("kernel_source_sha256") == sweep_source_sha()):
                traffic = tt.get("bytes_per_launch")
        except Exception:
            pass
    out = {
        "metric": "recons/sec at oracle-matched RMSE",
        "value": value,
        "unit": "recons/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * el / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.dtype == "f32" else args.dtype + "-A/f32",
        "data": "synthetic (seeded ellipse phantoms, analytic sinograms, Poisson counts)",
        "config": {"workload": WORKLOAD["name"], "batch_per_gpu": B, "sv_size": args.sv, "chains": args.chains,
                   "concurrency_per_agent": args.concurrency, "sigma_normalised": args.sigma, "rho": args.rho,
                   "tol": args.tol, "recompute_every": args.recompute_every, "deterministic": bool(args.deterministic),
                   "e_recompute": "geometry" if forward_geometry(args) else "stored values", "iterations": iters_main, "converged": conv_main,
                   "accuracy": accuracy,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (stored matrix %.2f GB)" % (info["bytes_columns"] / 1e9)},
        "e2e": {"value": e2e, "unit": "recons/s",
                "h2d_bytes_per_step": int(2 * y.nbytes), "d2h_bytes_per_step": int(B * n * 4)},
        "gpu_launches": None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": "icd_sweep_kernel",
                     "alg_bytes_per_launch": alg_bytes, "alg_matrix_bytes": matrix_bytes,
                     "alg_state_bytes_per_recon": per_recon, "stored_matrix_bytes": info["bytes_columns"],
                     "avg_launch_ms": avg_launch_s * 1000.0},
        "clocks": clocks,
    }
    # kernel launches inside one timed step: init (check, pack, consensus,
    # broadcast, reset, forward, theta2) + per iteration (consensus, 2 sweeps,
    # mann, residual) + recompute every few iterations (reset, forward) + output
    its = sum(iters_main)
    out["gpu_launches"] = int(args.steps * 7 + its * 5 + 2 * (its // args.recompute_every) + args.steps)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, y[0], lam[0], sx, int(np.mean(iters_main)),
                                           seconds=args.cpu_seconds)
        try:
            out["cpu_baseline"]["config1_to_tolerance"] = config1_to_tolerance()
        except Exception as e:      # a side-measurement: never fails the benchmark line
            out["cpu_baseline"]["config1_to_tolerance"] = {"error": str(e)}
    if dist:
        dist.destroy_process_group()
    return out


def cpu_baseline(args, y, lam, sx, iters, seconds=20.0):
    """The FP64 oracle (Algorithm 1 with the same solver settings, serial ICD
    order, one OpenMP thread per agent) on the host cores: time a bounded
    number of Mann iterations and scale to the iteration count the GPU run
    needed for the same tolerance (the oracle's serial passes contract at the
    same rate per iteration on this workload)."""
    import oracle
    threads = os.cpu_count() or 1
    P = oracle.Problem(WORKLOAD["n"], WORKLOAD["n"], WORKLOAD["n_views"], WORKLOAD["n_channels"], y, lam,
                       n_agents=WORKLOAD["n_agents"], prior="qggmrf", sigma_x=sx)
    t2 = oracle.mean_theta2(P)
    sigma = args.sigma / math.sqrt(t2)
    t0 = time.perf_counter()
    P.mace(sigma, rho=args.rho, sweeps=2, symmetric=True, max_iter=1, tol=0.0, n_threads=threads)
    one = time.perf_counter() - t0
    k = max(1, min(20, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    P.mace(sigma, rho=args.rho, sweeps=2, symmetric=True, max_iter=k, tol=0.0, n_threads=threads)
    per_iter = (time.perf_counter() - t0) / k
    # the same on one thread (the agents one after another): one iteration
    t0 = time.perf_counter()
    P.mace(sigma, rho=args.rho, sweeps=2, symmetric=True, max_iter=1, tol=0.0, n_threads=1)
    per_iter_1 = time.perf_counter() - t0
    # the paper's single-node method: centralised ICD over all views, one sweep
    t0 = time.perf_counter()
    P.central_icd(max_sweeps=1, tol=0.0)
    central_sweep = time.perf_counter() - t0
    return {"value": 1.0 / (per_iter * iters), "unit": "recons/s", "cores": threads, "kind": "oracle",
            "sample": "%d Mann iterations (2 ICD passes each) of one %dx%d reconstruction, "
                      "%.2f s/iteration, scaled to %d iterations to tolerance"
                      % (k, WORKLOAD["n"], WORKLOAD["n"], per_iter, iters),
            "single_thread": {"value": 1.0 / (per_iter_1 * iters), "unit": "recons/s", "cores": 1,
                              "s_per_iteration": per_iter_1, "sample": "1 Mann iteration on one thread"},
            "central_icd": {"s_per_sweep": central_sweep, "cores": 1,
                            "sample": "1 sweep of the centralised MAP ICD over all views"}}


def config1_to_tolerance(tol=1e-6):
    """Both sides timed to the same tolerance, nothing extrapolated: config 1
    (64^2, 90 views, 95 channels, 4 interleaved agents, quadratic prior,
    rho 0.8, serial voxel order) at the parity tests' solver settings:
    normalised sigma 0.5 and two symmetric ICD passes per Mann iteration (at
    normalised sigma 1 with one pass the partial-update iteration diverges
    on both sides: Theorem 2 asks for a small enough sigma).  The oracle (FP64, one thread per agent) on the host cores
    and the library (one warp per agent) each run Algorithm 1 from w = 0 to
    the Mann residual tol; the images are compared at the end."""
    import torch
    import synth
    import oracle
    import paper_1911_09278_gb300 as mace
    cfg = synth.CONFIGS["cfg1"]
    c = synth.make_case(**{k: cfg[k] for k in ("n", "n_views", "n_channels", "I0", "mu_max", "seed", "noise_seed")})
    y, lam = c["y"][0], c["lam"][0]
    n, V, D, N = cfg["n"], cfg["n_views"], cfg["n_channels"], cfg["n_agents"]
    sx = synth.prior_sigma_x(lam, V, frac=cfg["prior_frac"])
    threads = min(N, os.cpu_count() or 1)
    P = oracle.Problem(n, n, V, D, y, lam, n_agents=N, prior="quadratic", sigma_x=sx)
    sigma = 0.5 / math.sqrt(oracle.mean_theta2(P))
    t0 = time.perf_counter()
    res = P.mace(sigma, rho=0.8, sweeps=2, symmetric=True, max_iter=20000, tol=tol, n_threads=threads)
    t_cpu = time.perf_counter() - t0
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, sv_size=8)
    prm = mace.make_params(prior="quadratic", sigma_x=sx, sigma=0.5, sigma_mode=1, rho=0.8, sweeps_per_iter=2,
                           symmetric=True, recompute_every=10, tol=tol, max_iter=20000, concurrency=1)
    st = mace.mace_init(sm, y, lam, prm)       # warm-up: kernels loaded, graph captured
    st.reconstruct()
    st.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = mace.mace_init(sm, y, lam, prm)
    x, iters, r, conv = st.reconstruct()
    t_gpu = time.perf_counter() - t0
    st.close()
    sm.close()
    xo = np.asarray(res["x"], np.float64)
    return {"tol": tol, "oracle": {"s_per_recon": t_cpu, "iters": int(res["iters"]), "cores": threads},
            "gpu": {"s_per_recon": t_gpu, "iters": int(iters), "converged": bool(conv),
                    "includes": "mace_init (inputs from host memory) + mace_reconstruct + image to host"},
            "gpu_over_oracle": t_cpu / t_gpu,
            "nrmse_gpu_vs_oracle": float(np.linalg.norm(np.asarray(x, np.float64).ravel() - xo)
                                         / np.linalg.norm(xo))}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample of the
    same workload (a few Mann iterations), reported in reconstructions/s."""
    if rank != 0:
        return None
    import synth
    import oracle
    y, lam = make_inputs(1, 0)
    sx = synth.prior_sigma_x(lam[0], WORKLOAD["n_views"], frac=args.prior_frac)
    threads = os.cpu_count() or 1
    P = oracle.Problem(WORKLOAD["n"], WORKLOAD["n"], WORKLOAD["n_views"], WORKLOAD["n_channels"], y[0], lam[0],
                       n_agents=WORKLOAD["n_agents"], prior="qggmrf", sigma_x=sx)
    t2 = oracle.mean_theta2(P)
    sigma = args.sigma / math.sqrt(t2)
    per_step_iters = 2
    for _ in range(args.warmup):
        P.mace(sigma, rho=args.rho, sweeps=2, symmetric=True, max_iter=1, tol=0.0, n_threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.mace(sigma, rho=args.rho, sweeps=2, symmetric=True, max_iter=per_step_iters, tol=0.0, n_threads=threads)
    el = time.perf_counter() - t0
    per_iter = el / (args.steps * per_step_iters)
    value = 1.0 / (per_iter * args.oracle_iters)
    sample = ("%d Mann iterations per step of one 512^2 reconstruction (%.2f s/iteration), "
              "scaled to %d iterations to tolerance" % (per_step_iters, per_iter, args.oracle_iters))
    return {"impl": "reference", "metric": "recons/sec at oracle-matched RMSE", "value": value,
            "unit": "recons/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "batch_per_gpu": 1},
            "cpu_baseline": {"value": value, "unit": "recons/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "recons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


SERVE_SIZES = [(128, 180, 183), (256, 360, 363), (512, 720, 725), (1024, 1440, 1449)]   # (n, views, channels)
SERVE_AGENTS = [4, 8, 16, 32]


def run_serve(args):
    """Serving on one GPU: a seeded stream of 2D requests, sizes and agent
    counts drawn uniformly from SERVE_SIZES and SERVE_AGENTS (BF16 matrices,
    FP32 state, Q-GGMRF 8-neighbour, super-voxel side 4 for agents of more
    than 64 views, else 8, the work-queue sweep).  Every request waits at
    time 0 (a burst) and is served three ways: grouped (all active requests
    in one group, their ICD passes in one queue-fed launch per pass), one
    stream per request (their launches overlap on the GPU), and one at a
    time; recons/s is the capacity of each.  With --serve-poisson the same
    requests then arrive as a Poisson stream at args.serve_load times the
    grouped capacity and are served all three ways again.  Every mode stops
    a request at the same Mann residual (args.serve_tol).  Latency is
    arrival to image in host memory."""
    import torch
    import synth
    from paper_1911_09278_gb300 import build as gbuild
    from paper_1911_09278_gb300 import serve

    def note(msg):
        print("[serve %.0fs] %s" % (time.perf_counter() - t_start, msg), file=sys.stderr, flush=True)
    t_start = time.perf_counter()
    gbuild.build()
    torch.cuda.set_device(0)
    rng = synth.CounterRNG(5)
    u = rng.uniform(11, np.arange(3 * args.requests)).reshape(args.requests, 3)
    reqs = []
    for k in range(args.requests):
        n, V, D = SERVE_SIZES[min(len(SERVE_SIZES) - 1, int(u[k, 0] * len(SERVE_SIZES)))]
        N = SERVE_AGENTS[min(len(SERVE_AGENTS) - 1, int(u[k, 1] * len(SERVE_AGENTS)))]
        c = synth.make_case(n=n, n_views=V, n_channels=D, I0=2e4, mu_max=0.02 * 64 / n, seed=1000 + k,
                            noise_seed=3000 + k)
        sx = synth.prior_sigma_x(c["lam"][0], V, frac=1.0)
        reqs.append(serve.Request(k, 0.0, n, n, V, D, N, c["y"][0], c["lam"][0], sx, None))
    # the work-queue sweep in every mode, so one request's iterates are the
    # same served grouped and alone (up to the order of float additions)
    params = dict(prior="qggmrf", sigma=args.serve_sigma, sigma_mode=1, rho=args.rho, sweeps_per_iter=2,
                  symmetric=True, recompute_every=10, tol=args.serve_tol, concurrency=args.serve_concurrency,
                  schedule=1)
    srv = serve.Server(params, dtype=args.serve_dtype, sv_size="auto", max_active=args.max_active,
                       max_iter=args.max_iter)
    for r in reqs:                      # matrices resident before any timing
        srv._matrix(r)
    note("%d requests, matrices built" % len(reqs))
    small = sorted(reqs, key=lambda r: r.nx)[:2]
    srv.run(small, grouped=True)        # warm-up
    srv.run(small, serial=True)
    torch.cuda.synchronize()
    runs = {}
    runs["grouped"] = srv.run(reqs, grouped=True)
    note("burst, grouped: %.1f s" % runs["grouped"]["makespan"])
    runs["streams"] = srv.run(reqs)
    note("burst, one stream per request: %.1f s" % runs["streams"]["makespan"])
    if not args.no_serial:
        runs["one_at_a_time"] = srv.run(reqs, serial=True)
        note("burst, one at a time: %.1f s" % runs["one_at_a_time"]["makespan"])
    capacity = len(runs["grouped"]["results"]) / max(1e-9, runs["grouped"]["makespan"])
    if args.serve_poisson:
        rate = args.serve_load * capacity
        gaps = -np.log(1.0 - rng.uniform(12, np.arange(len(reqs)))) / rate
        t = np.cumsum(gaps) - gaps[0]
        timed = [r._replace(arrival=float(t[k])) for k, r in enumerate(reqs)]
        runs["poisson_grouped"] = srv.run(timed, grouped=True)
        note("poisson, grouped done")
        if not args.no_serial:
            runs["poisson_one_at_a_time"] = srv.run(timed, serial=True)
            note("poisson, one at a time done")
        runs["poisson_streams"] = srv.run(timed)
    worst = None
    if "one_at_a_time" in runs:
        worst = 0.0
        for r in reqs:
            a, b = runs["grouped"]["results"].get(r.rid), runs["one_at_a_time"]["results"].get(r.rid)
            if a is None or b is None:
                continue      # failed in one of the modes: counted below
            worst = max(worst, float(np.linalg.norm(a["x"] - b["x"]) / max(1e-30, np.linalg.norm(b["x"]))))
    best_name = max(("grouped", "streams"), key=lambda k: runs[k]["recons_per_s"])
    best = g = runs[best_name]
    conv = all(d["converged"] for d in g["results"].values())
    srv.close()
    mix = collections.Counter((r.nx, r.n_agents) for r in reqs)

    def brief(o):
        its = [d["iters"] for d in o["results"].values()]
        return {"value": o["recons_per_s"], "unit": "recons/s", "p50_s": o["p50"], "p99_s": o["p99"],
                "makespan_s": o["makespan"], "completed": len(o["results"]), "failed": len(o["failed"]),
                "converged": sum(d["converged"] for d in o["results"].values()),
                "iters_min_max": [min(its), max(its)] if its else None}
    out = {
        "metric": "served recons/sec (continuous batching, the better of grouped and per-request streams) "
                  "with p50/p99 latency, burst of requests",
        "value": best["recons_per_s"], "best_mode": best_name, "unit": "recons/s", "n_gpus": 1, "higher_is_better": True,
        "p50_s": g["p50"], "p99_s": g["p99"],
        "modes": {k: brief(v) for k, v in runs.items()},
        "max_nrmse_grouped_vs_one_at_a_time": worst,
        "converged": conv, "failed": len(g["failed"]),
        "dtype": args.serve_dtype + "-A/f32", "data": "synthetic",
        "config": {"workload": "%d 2D requests at time 0, sizes %s, agents %s" % (len(reqs), SERVE_SIZES,
                                                                               SERVE_AGENTS),
                   "mix": {"%dx%d/%d agents" % (k[0], k[0], k[1]): v for k, v in sorted(mix.items())},
                   "max_active": args.max_active, "concurrency_per_agent": args.serve_concurrency,
                   "sv_size": "4 above 64 views per agent, else 8", "sigma_normalised": args.serve_sigma,
                   "tol": args.serve_tol, "max_iter": args.max_iter},
    }
    if "one_at_a_time" in runs:
        out["speedup_vs_one_at_a_time"] = g["recons_per_s"] / runs["one_at_a_time"]["recons_per_s"]
    if args.serve_poisson:
        out["poisson_rate_per_s"] = args.serve_load * capacity
    return out


def run_volume(args):
    """A 3D stack: args.slices slices of 512^2 sharing one 2D matrix (960
    views over 180 deg, 725 channels), 32 agents with uneven view subsets
    (16-40 views each, spread over the half circle), 26-neighbourhood
    Q-GGMRF coupling the slices.  Schedule 0 (default): fixed warps per
    (slice pair, agent), all slices at once; schedule 1: a persistent grid
    fed from a work queue of (slice, agent, row of super-voxels) items, even
    slices first, then odd ones; --volume-chains 2: two slices per warp.  Times args.steps Mann iterations (value = Mann iterations
    per second of the whole volume); with --volume-tol > 0 it then runs on
    to that residual (at most args.max_iter iterations) and reports the
    iterations and the time to get there."""
    import torch
    import synth
    import paper_1911_09278_gb300 as mace
    from paper_1911_09278_gb300 import build as gbuild

    gbuild.build()
    torch.cuda.set_device(0)
    n, nz, V, D, N = 512, args.slices, 960, 725, 32
    c = synth.make_volume(n=n, nz=nz, n_views=V, n_channels=D, I0=2e4, mu_max=0.02 * 64 / n, seed=4,
                          noise_seed=104)
    va = synth.uneven_partition(204, V, N, 16, 40)
    sx = synth.prior_sigma_x(c["lam"], V, frac=1.0)
    stream = torch.cuda.Stream()
    sm = mace.mace_build_sysmatrix(n, n, V, D, N, view_agent=va, sv_size=args.volume_sv, dtype=args.dtype,
                                   stream=stream)
    info = sm.info()
    prm = mace.make_params(prior="qggmrf", sigma_x=sx, sigma=args.volume_sigma, sigma_mode=1, rho=args.rho,
                           sweeps_per_iter=2, symmetric=True, recompute_every=10, max_iter=args.max_iter,
                           tol=args.volume_tol, concurrency=args.concurrency, neighbourhood=26,
                           schedule=args.volume_schedule, chains=args.volume_chains)
    st = mace.mace_init(sm, c["y"], c["lam"], prm, stream=stream, batch=nz)
    st.iterate(args.warmup)
    st.set_timing(True, max_launches=4 * args.steps + 8)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st.launch(args.steps)
    ev1.record(stream)
    stream.synchronize()
    el = ev0.elapsed_time(ev1) / 1000.0
    ms, nl = st.get_timing()
    st.set_timing(False)
    stats = st.stats()
    r_now, _ = st.poll()
    out = {
        "metric": "Mann iterations / s of a 3D stack (all slices and agents)", "value": args.steps / el,
        "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True, "dtype": args.dtype,
        "data": "synthetic (seeded ellipsoid phantom, analytic sinograms, Poisson counts)",
        "sweep_ms": ms / max(1, nl), "voxel_updates_per_s": nz * n * n * N / (ms / max(1, nl) / 1000.0),
        "residual_after_timed": r_now,
        "schedule": stats["schedule"], "concurrency_per_agent": stats["concurrency"], "warps": stats["warps"],
        "chains": stats["chains"],
        "config": {"workload": "3D %dx%dx%d, 960 views, 725 channels, 32 agents with 16-40 views, "
                               "26-neighbour Q-GGMRF" % (n, n, nz),
                   "matrix_gb": info["bytes_columns"] / 1e9, "sv_size": args.volume_sv,
                   "sigma_normalised": args.volume_sigma, "rho": args.rho},
    }
    if args.volume_tol > 0:
        t0 = time.perf_counter()
        conv, r = False, r_now
        traj = []
        while not conv and stats["iters"] < args.max_iter:
            st.launch(50)
            r, conv = st.poll()
            stats = st.stats()
            traj.append([stats["iters"], r])
        out["to_tolerance"] = {"tol": args.volume_tol, "converged": conv, "iters": stats["iters"],
                               "residual": r, "trajectory": traj, "seconds_after_timed": time.perf_counter() - t0,
                               "seconds_est_total": stats["iters"] * el / args.steps}
    st.close()
    sm.close()
    return out


def run_autotune(args):
    """The sweep-configuration autotuner on the benchmark's scans (or, with
    --size and --agents, a scan of that size and agent count): for each
    candidate (super-voxel size, chains, schedule, warps per super-voxel) a
    short probe of Mann iterations, timed, and the iterations to tolerance
    extrapolated from the residual's rate."""
    import torch
    import synth
    import paper_1911_09278_gb300 as mace
    from paper_1911_09278_gb300 import autotune
    from paper_1911_09278_gb300 import build as gbuild

    gbuild.build()
    torch.cuda.set_device(0)
    if args.agents:
        WORKLOAD["n_agents"] = args.agents
    y, lam = make_inputs(args.batch, 0)
    sx = synth.prior_sigma_x(lam[0], WORKLOAD["n_views"], frac=args.prior_frac)
    params = dict(prior="qggmrf", sigma_x=sx, sigma=args.sigma, sigma_mode=1, rho=args.rho, sweeps_per_iter=2,
                  symmetric=True, recompute_every=args.recompute_every, max_iter=args.max_iter, tol=args.tol,
                  concurrency=args.concurrency, sv_order=0, forward_geometry=forward_param(args))
    cands = autotune.candidates_for(-(-WORKLOAD["n_views"] // WORKLOAD["n_agents"]))
    best, table = autotune.tune(WORKLOAD["n"], WORKLOAD["n"], WORKLOAD["n_views"], WORKLOAD["n_channels"],
                                WORKLOAD["n_agents"], y, lam, params, batch=args.batch, dtype=args.dtype,
                                candidates=cands, probe_iters=args.probe_iters)
    for row in table:
        row.pop("trajectory", None)
        for k, v in row.items():
            if isinstance(v, float) and not math.isfinite(v):
                row[k] = None     # did not contract within the probe
    pick = None if best is None else {k: best[k] for k in ("sv_size", "chains", "schedule", "warps_per_voxel",
                                                           "concurrency")}
    return {"mode": "autotune", "workload": "%s (%d agents)" % (WORKLOAD["name"], WORKLOAD["n_agents"]),
            "batch": args.batch, "sigma_normalised": args.sigma,
            "rho": args.rho, "tol": args.tol, "probe_iters": args.probe_iters, "best": pick, "candidates": table}


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mace", choices=["mace", "reference"])
    ap.add_argument("--batch", type=int, default=DEFAULTS["batch"])
    ap.add_argument("--concurrency", type=int, default=DEFAULTS["concurrency"])
    ap.add_argument("--sigma", type=float, default=DEFAULTS["sigma"])
    ap.add_argument("--rho", type=float, default=DEFAULTS["rho"])
    ap.add_argument("--tol", type=float, default=DEFAULTS["tol"])
    ap.add_argument("--max-iter", dest="max_iter", type=int, default=DEFAULTS["max_iter"])
    ap.add_argument("--sv", type=int, default=DEFAULTS["sv"])
    ap.add_argument("--chains", type=int, default=DEFAULTS["chains"],
                    help="reconstructions of the batch one warp updates together (1, 2 or 4)")
    ap.add_argument("--dtype", default=DEFAULTS["dtype"], choices=["f32", "bf16", "f16"])
    ap.add_argument("--forward", default=DEFAULTS["forward"], choices=["auto", "stored", "geometry"],
                    help="A for the e recompute: stored values or evaluated from the geometry (auto: geometry "
                         "when the stored values are BF16/FP16)")
    ap.add_argument("--recompute-every", dest="recompute_every", type=int, default=DEFAULTS["recompute_every"],
                    help="Mann iterations between recomputations of e = y - A x")
    ap.add_argument("--deterministic", action="store_true",
                    help="lock-step super-voxel phases and fixed-point sums: bit-identical results run to run")
    ap.add_argument("--oracle-iters", dest="oracle_iters", type=int, default=670,
                    help="Mann iterations to tolerance the reference arm scales its sample to (the GPU path's count at the default settings)")
    ap.add_argument("--cpu-seconds", dest="cpu_seconds", type=float, default=20.0)
    ap.add_argument("--prior-frac", dest="prior_frac", type=float, default=1.0,
                    help="prior curvature as a fraction of the data curvature (1/sigma_x^2 = frac x the median "
                         "pixel data curvature)")
    ap.add_argument("--no-cpu-baseline", dest="no_cpu_baseline", action="store_true")
    ap.add_argument("--size", type=int, default=0,
                    help="profiling only: an n x n image with 1.40625 n views and ceil(sqrt(2) n) channels "
                         "(the same geometry family, smaller), instead of the 512^2 workload")
    ap.add_argument("--serve", action="store_true",
                    help="continuous batching vs one-at-a-time service on a request stream (its own JSON line)")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--max-active", dest="max_active", type=int, default=16)
    ap.add_argument("--serve-concurrency", dest="serve_concurrency", type=int, default=-1)
    ap.add_argument("--serve-dtype", dest="serve_dtype", default="bf16", choices=["f32", "bf16", "f16"])
    # serving runs 8x8 super-voxels, one row per item; sigma 0.1 is stable over
    # the whole size and agent mix (0.13 diverged for 256^2 with 32 agents)
    ap.add_argument("--serve-sigma", dest="serve_sigma", type=float, default=0.1)
    ap.add_argument("--serve-tol", dest="serve_tol", type=float, default=1e-5)
    ap.add_argument("--serve-poisson", dest="serve_poisson", action="store_true",
                    help="serving: after the burst, a Poisson stream at --serve-load times the grouped capacity")
    ap.add_argument("--serve-load", dest="serve_load", type=float, default=0.8,
                    help="arrival rate as a multiple of the grouped server's capacity")
    ap.add_argument("--no-serial", dest="no_serial", action="store_true",
                    help="serving: skip the one-at-a-time run")
    ap.add_argument("--volume", action="store_true",
                    help="time Mann iterations of a 3D stack with uneven agents (its own JSON line)")
    ap.add_argument("--slices", type=int, default=64)
    # the fixed grid (one warp per slice pair and agent: serial order per
    # pair) converges at sigma 0.3; the work queue with a row of super-voxels
    # per item runs as fast per iteration but diverged at 0.13 on this stack
    ap.add_argument("--volume-schedule", dest="volume_schedule", type=int, default=0, choices=[0, 1])
    ap.add_argument("--volume-sv", dest="volume_sv", type=int, default=8)
    ap.add_argument("--volume-chains", dest="volume_chains", type=int, default=1,
                    help="volume: slices one warp sweeps over each column load (1 or 2)")
    ap.add_argument("--volume-sigma", dest="volume_sigma", type=float, default=0.3)
    ap.add_argument("--volume-tol", dest="volume_tol", type=float, default=0.0,
                    help="volume: after the timed iterations, run on to this Mann residual")
    ap.add_argument("--autotune", action="store_true",
                    help="rank super-voxel sizes and chains on the workload by estimated time to tolerance "
                         "(its own JSON line)")
    ap.add_argument("--probe-iters", dest="probe_iters", type=int, default=100)
    ap.add_argument("--agents", type=int, default=0, help="autotune: agents of the scan (default 16)")
    return ap


def main():
    args = build_parser().parse_args()
    if args.autotune:
        if args.size:
            n = args.size
            WORKLOAD.update(n=n, n_views=int(round(1.40625 * n)), n_channels=int(math.ceil(math.sqrt(2.0) * n)),
                            name="parallel-beam 2D %dx%d, %d views, Q-GGMRF" % (n, n, int(round(1.40625 * n))))
        print(json.dumps(run_autotune(args)))
        return
    if args.volume:
        print(json.dumps(run_volume(args)))
        return
    if args.serve:
        print(json.dumps(run_serve(args)))
        return
    if args.size:
        n = args.size
        D = int(math.ceil(math.sqrt(2.0) * n))
        WORKLOAD.update(n=n, n_views=int(round(1.40625 * n)), n_channels=D,
                        name="parallel-beam 2D %dx%d, %d views over 180 deg, %d channels, 16 interleaved agents, "
                             "Q-GGMRF (p=2, q=1.2, T=1), FP32 (profiling size)"
                             % (n, n, int(round(1.40625 * n)), D))
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_mace(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
