#!/usr/bin/env python
"""Benchmark: GWN queries/s of the antipodal method on one GB300 (per rank).

One step = one gwn_classify call over the whole query batch: the exact +z
crossing count (BVH traversal), the boundary-curve sum, the combine into w and
the labels with the FP64 re-evaluation of queries near 1/2.  The mesh and its
acceleration data are built once before timing (the paper excludes
precomputation from its timings, Sec. 5.1); the build time is reported.

Default workload ``soup8``: the level-8 displaced icosphere plus a translated
copy with 2% of the faces deleted (2.57M triangles, ~157k boundary edges),
2M queries (1M uniform in the padded bounding box, 1M near the surface).

Printed: one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (bounded samples of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GWN queries/sec at 1M tris (antipodal vs direct sum, same GPU, |Δw|≤1e-5)"

WORKLOADS = {
    "soup8": "icosphere L8 displaced + translated copy, 2% faces deleted (self-intersecting soup "
             "with holes); 1M uniform-in-padded-bbox + 1M near-surface (sigma 1e-3) queries, seed 4",
    "soup7": "icosphere L7 displaced + translated copy, 2% faces deleted; 1M uniform + 1M "
             "near-surface queries, seed 1",
    "small": "icosphere L3 with the z>0.8 cap removed; 10k uniform queries in [-1.5,1.5]^3, seed 0",
    "precision": "voxel-staircase sphere of radius 40 (60,288 triangles, closed) + open 200x200 integer height "
                 "field (79,202 triangles); 500k queries exactly on vertices, edge midpoints, staircase faces and "
                 "integer grid points, seed 2",
    "surrogate": "icosphere L8 displaced + translated copy, 2% faces deleted; learned surrogate trained on 2M "
                 "samples (1M uniform in the padded bbox, 1M near-surface, labelled by the GPU antipodal path, "
                 "seed 4); classify the 256^3 grid of cell centres over the padded bbox (16,777,216 queries)",
    "surrogate_infer": "network inference alone (gwn_surrogate_predict) over the 256^3 grid of cell centres of the "
                       "padded bbox of the L8 soup (16,777,216 queries), He-normal random weights (seed 6)",
    "gradient": "grad w (Supp. S4, Algorithm 3) of the soup8 queries: icosphere L8 displaced + translated copy, "
                "2% faces deleted; 1M uniform + 1M near-surface queries, seed 4",
    "grid": "256^3 grid of cell centres over the padded bbox, classified with ray reuse (Supp. S3) vs per point: "
            "the closed soup (icosphere L8 displaced + translated copy, no faces deleted: 2,621,440 triangles, w = chi) "
            "and the holed soup8 mesh",
    "param": "100 bicubic Bezier patches, every control point uniform in the unit cube (seed 7); the 32^3 grid "
             "of cell centres over the control points' box padded by 10% (32,768 queries): w and chi by "
             "Algorithm 2 (Sec. 4.4)",
    "peaks": "pipe-throughput microbenchmarks: paired FP32 FMAs (FFMA2) and SFU reciprocal / reciprocal square "
             "root in independent chains on every SM, the denominators of the boundary kernels' ALU rooflines",
    "batched": "256 meshes (superquadrics e1,e2~U[0.3,3], random open height fields, unwelded random soups), "
               "triangles log-uniform in [100, 500k], queries log-uniform in [1k, 1M] (half uniform in the "
               "padded bbox, half near-surface), seed 3",
}

# Algorithmic work per gradient term (one query x one boundary edge) of
# Algorithm 3 with x1 = -z, in FP32 issue slots: per endpoint (shared by the two
# edges of a chained point) 3 sub, 3 FMA (squared lengths), 1 mul (length),
# 3 mul (unit vector), 4 for the cancellation-free h; per edge n 2, d 3,
# n^2 + d^2 2, the factor 2 / (n^2 + d^2) 1, c_n and c_d 2, r0 + r1 3, the
# h1 v0 + h0 v1 corrections 6, l0 + l1 1, assembling c_n g_n + c_d g_d 6,
# accumulating 3 -> 43 slots, plus 3 SFU operations.
GRAD_OPS_PER_TERM = 43.0
# Algorithmic work per boundary edge term (one query x one boundary edge), the
# plain formula of Algorithm 1 with x1 = (0, 0, -1) counted in FP32 issue slots
# (one add, mul or FMA = one slot), endpoint work amortised over the chained
# edges: per endpoint 3 sub + 3 FMA (squared length) + 3 mul (scale by the
# rsqrt); per edge 2 for the numerator, 5 for the denominator, 1 accumulate;
# atan2 about 12 (ratio, polynomial, octant) -> 28 slots, plus 2 SFU ops.
OPS_PER_TERM = 28.0
SFU_OPS_PER_TERM = 2.0
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="soup8")
    ap.add_argument("--n-query", type=int, default=None, help="override the query count")
    ap.add_argument("--direct-sample", type=int, default=65536)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline sample time")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle check of the timed output")
    ap.add_argument("--n-mesh", type=int, default=256, help="batched workload: meshes (smaller for profiling)")
    ap.add_argument("--level", type=int, default=0, help="surrogate workload: icosphere level (0 = 8)")
    ap.add_argument("--res", type=int, default=0, help="surrogate workload: grid resolution (0 = 256)")
    ap.add_argument("--train-steps", type=int, default=3000, help="surrogate workload: Adam steps")
    ap.add_argument("--parity-sample", type=int, default=2000,
                    help="queries of the timed output checked against the oracle (half nearest the boundary)")
    ap.add_argument("--kq", type=int, default=0, help="queries per thread of the boundary kernel (0 = default)")
    ap.add_argument("--tile", type=int, default=0, help="boundary points per shared-memory tile (0 = default)")
    ap.add_argument("--chain", type=int, default=0, help="1 chain boundary edges into loops, -1 do not")
    ap.add_argument("--qbits", type=int, default=0,
                    help="30: predicates on the 30-bit fixed-point snap of the inputs (Supp. S2.1); 0: exact FP32")
    ap.add_argument("--group-test", type=int, default=0, choices=[0, 1, 2],
                    help="boundary group acceptance: 0 auto (by boundary density), 1 per-term pi/8, 2 running")
    ap.add_argument("--fp64-cancel", type=int, default=0, choices=[-1, 0, 1],
                    help="0 (default): boundary terms whose denominator cancels are evaluated in FP64; "
                         "-1: every boundary term in FP32")
    return ap.parse_args()


def _recorded_kernel(args) -> bool:
    """True when the boundary kernel runs in the configuration its committed
    DRAM-traffic capture was taken in (4 queries per thread, 512-point tiles,
    chained points, exact predicates, FP64 for cancelling boundary terms, the
    default group test, the workload's own query count)."""
    return (args.kq in (0, 4) and args.tile in (0, 512) and args.chain != -1 and not args.qbits
            and args.fp64_cancel != -1 and args.group_test == 0 and args.n_query is None)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The slowest rank's step time (every rank gets it); ``dist`` is
    torch.distributed (NCCL with CUDA tensors, gloo with CPU tensors) or None."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world_size: int, step_ms: float) -> float:
    """Whole-job units per second: every rank processes its own replica of the
    workload (queries are independent), timed by the slowest rank."""
    return world_size * units_per_rank / (step_ms / 1e3)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi's start-up (driver initialisation) slows CUDA calls of this
        # process for a moment: let it write its first sample before timing starts
        t0 = time.perf_counter()
        while self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def read_profile(gwn):
    """({step: (runs, ms)}, {step: {"runs", "ms", "kernels"}}, kernels launched in all) since the last enable."""
    p3 = gwn.profile_read(with_kernels=True)
    prof = {k: v[:2] for k, v in p3.items()}
    table = {k: {"runs": v[0], "ms": v[1], "kernels": v[2]} for k, v in p3.items()}
    return prof, table, sum(v[2] for v in p3.values())


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _traffic_record(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu record (profiles/traffic.txt),
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    for rec in lines:
        if len(rec) == 5 and rec[0] == kernel and rec[1] == workload:
            # the kernel's source files and their hashes, comma-separated, in the same order
            files, hashes = rec[3].split(","), rec[4].split(",")
            if len(files) != len(hashes):
                return None
            for f, want in zip(files, hashes):
                try:
                    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2605_01536_gb300", "csrc", f), "rb").read())
                except OSError:
                    return None
                if h.hexdigest()[:16] != want:
                    return None
            return int(rec[2])
    return None


def cpu_baseline(mesh, Q, seconds: float, seed: int = 0):
    """The oracle (FP64 antipodal with exact crossing counts), as it stands, on a
    bounded sample of the workload's queries."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    E = oracle.boundary(mesh.F, mesh.nv)
    probe = Q[rng.choice(len(Q), 256, replace=False)]
    t = time.perf_counter()
    c = oracle.chi(mesh.V, mesh.F, probe)
    oracle.antipodal(mesh.V, E, probe, c)
    per_q = (time.perf_counter() - t) / len(probe)
    n = int(max(256, min(len(Q), seconds / max(per_q, 1e-9))))
    sample = Q[rng.choice(len(Q), n, replace=False)]
    t = time.perf_counter()
    c = oracle.chi(mesh.V, mesh.F, sample)
    oracle.antipodal(mesh.V, E, sample, c)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} seeded random queries of the workload (FP64 antipodal + exact chi), {dt:.1f} s"}


def near_boundary_queries(V, F, Q, k: int):
    """Indices of the k queries closest to the mesh's boundary curve (distance
    to five points along every boundary edge), where FP32 is weakest."""
    import numpy as np
    import oracle
    from scipy.spatial import cKDTree
    E = oracle.boundary(F, len(V))
    if len(E) == 0 or k <= 0:
        return np.zeros(0, np.int64)
    A, B = V[E[:, 0]].astype(np.float64), V[E[:, 1]].astype(np.float64)
    S = np.concatenate([A + (B - A) * t for t in (0.1, 0.3, 0.5, 0.7, 0.9)])
    dist, _ = cKDTree(S).query(np.asarray(Q, np.float64))
    return np.argsort(dist, kind="stable")[:k]


def timed_parity(m, mesh, Q, labels, w, n_sample: int, quantize_bits: int = 0, tol: float = 1e-5):
    """The timed step's output checked against the oracle on a seeded sample:
    half uniform over the batch, half the queries nearest the boundary curve.
    w within tol and labels exact on every query off the boundary curve (where
    w is undefined: excluded and counted); crossing numbers bit-exact, from
    gwn_query_batch on the sampled queries (the same crossing kernel)."""
    import numpy as np
    import oracle
    import torch
    rng = np.random.default_rng(12)
    half = n_sample // 2
    near = near_boundary_queries(mesh.V, mesh.F, Q, half)
    rest = np.setdiff1d(np.arange(len(Q)), near)
    idx = np.concatenate([near, rng.choice(rest, min(n_sample - len(near), len(rest)), replace=False)])
    t0 = time.perf_counter()
    ref = oracle.reference(mesh.V, mesh.F, Q[idx], quantize_bits=quantize_bits)
    oracle_s = time.perf_counter() - t0
    _, chi = m.query(torch.from_numpy(Q[idx]).cuda())
    chi = chi.cpu().numpy()
    ok = ref["flags"] == 0
    dw = np.abs(w[idx].astype(np.float64) - ref["w_antipodal"])[ok]
    want = (ref["w_antipodal"] > 0.5).astype(np.uint8)
    out = {"n": int(len(idx)), "n_near_boundary": int(len(near)), "n_uniform": int(len(idx) - len(near)),
           "max_dw": float(dw.max()) if len(dw) else 0.0,
           "max_dw_near_boundary": float(np.abs(w[near].astype(np.float64) - ref["w_antipodal"][:len(near)])
                                         [ok[:len(near)]].max()) if ok[:len(near)].any() else 0.0,
           "chi_mismatch": int((chi != ref["chi"]).sum()), "label_mismatch": int((labels[idx] != want)[ok].sum()),
           "excluded_on_boundary": int((~ok).sum()), "tolerance": tol, "oracle_s": round(oracle_s, 2),
           "what": "the last timed step's w and labels vs the FP64 oracle (exact crossing numbers)"}
    out["pass"] = out["max_dw"] <= tol and out["chi_mismatch"] == 0 and out["label_mismatch"] == 0
    return out


def run_reference_param(args):
    """The oracle's Algorithm 2 boundary integral (FP64, scipy quad) on bounded
    samples of the parametric workload's cells; the oracle has no ray-patch
    intersection, so chi is not part of the timed work."""
    import numpy as np
    import gen
    from oracle import parametric as par
    P, Q = gen.param_workload()
    curves = par.boundary_curves(P.astype(np.float64))
    rng = np.random.default_rng(1)
    times = []
    n = 2
    for step in range(args.warmup + args.steps):
        s = Q[rng.choice(len(Q), n, replace=False)].astype(np.float64)
        t = time.perf_counter()
        for q in s:
            par.boundary_term(curves, q)
        if step >= args.warmup:
            times.append(time.perf_counter() - t)
    step_s = sum(times) / len(times)
    value = n / step_s
    line = {"impl": "reference", "metric": "parametric GWN queries/sec, 100 random bicubic Bezier patches, 32^3 "
                                           "voxel grid (Sec. 4.4, Algorithm 2)",
            "value": value, "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"param: {WORKLOADS['param']}", "n_queries_per_step": n,
                       "parallelism": "one host core"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} seeded random cells per step: the Algorithm 2 boundary integral over "
                                       f"all {len(curves)} curves (chi not included)"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    if args.workload == "param":
        return run_reference_param(args)
    import numpy as np
    import gen
    import oracle
    mesh, Q = gen.workload(args.workload, n_query=args.n_query)
    E = oracle.boundary(mesh.F, mesh.nv)
    rng = np.random.default_rng(1)
    probe = Q[rng.choice(len(Q), 16, replace=False)]
    t = time.perf_counter()
    oracle.antipodal(mesh.V, E, probe, oracle.chi(mesh.V, mesh.F, probe))
    per_q = (time.perf_counter() - t) / len(probe)
    n = int(max(16, min(len(Q), 4.0 / max(per_q, 1e-9))))   # ~4 s of host work per step
    times = []
    for step in range(args.warmup + args.steps):
        s = Q[rng.choice(len(Q), n, replace=False)]
        t = time.perf_counter()
        oracle.antipodal(mesh.V, E, s, oracle.chi(mesh.V, mesh.F, s))
        if step >= args.warmup:
            times.append(time.perf_counter() - t)
    step_s = sum(times) / len(times)
    value = n / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_tris": mesh.nt,
                       "n_queries_per_step": n, "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{n} seeded random queries of the workload per step"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    mesh, Q = gen.workload(args.workload, n_query=args.n_query)
    n = len(Q)
    q_dev = torch.from_numpy(Q).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = gwn.Mesh(mesh.V, mesh.F, config=dict(queries_per_thread=args.kq, boundary_tile=args.tile,
                                             chain_boundary=args.chain, quantize_bits=args.qbits,
                                             fp64_cancel=args.fp64_cancel, group_test=args.group_test))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = m.info()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        m.classify(q_dev, want_w=True)
    torch.cuda.synchronize()

    m.counters(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    timed_out = None
    for i in range(args.steps):
        flush.fill_(i & 0xff)             # evict the previous step's data from L2 (untimed)
        ev[i][0].record(stream)
        timed_out = m.classify(q_dev, want_w=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    # event counts of the timed steps (per step)
    counters = {k: v / args.steps for k, v in m.counters().items()
                if k in ("cancel_terms", "fp64_reevaluations", "exact_edge", "exact_plane", "exact_branch",
                         "cancel_overflow")}
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # per-kernel times and launch counts from an identical profiled pass: the
    # profiler's events cost host time that would show in short steps above
    gwn.profile_enable(True)
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        m.classify(q_dev, want_w=True)
    torch.cuda.synchronize()
    prof, prof_table, prof_kernels = read_profile(gwn)
    gwn.profile_enable(False)
    step_ms = max_over_ranks(step_ms, dist, dev)
    value = job_throughput(n, ws, step_ms)

    # direct-sum baseline on a sample of the same queries (same GPU)
    nd = min(args.direct_sample, n)
    qd = q_dev[torch.randperm(n, generator=torch.Generator().manual_seed(3))[:nd].to(dev)].contiguous()
    m.direct(qd)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record(stream)
    for _ in range(reps):
        m.direct(qd)
    b.record(stream)
    torch.cuda.synchronize()
    direct_qps = nd * reps / (a.elapsed_time(b) / 1e3)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        q_host = torch.from_numpy(Q).pin_memory()
        m.classify(q_host, want_w=True)
        times = []
        for _ in range(args.steps):
            t1 = time.perf_counter()
            lab, w = m.classify(q_host, want_w=True)     # returns after the D2H copies completed
            times.append(time.perf_counter() - t1)
        e2e_s = sum(times) / len(times)
        e2e = {"value": ws * n / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": int(Q.nbytes),
               "d2h_bytes_per_step": int(n * (1 + 4))}

    # roofline of the dominant kernel (boundary-curve sum): FP32 ALU bound
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 0) or (clk or {}).get("sm_max_mhz", 0) or 2070.0)
    peak_tops = sms * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    launches, bsum_ms = prof.get("boundary_sum", (0, 0.0))
    roof = None
    if launches:
        per_launch_s = bsum_ms / launches / 1e3
        terms = n * info["n_boundary_edges"]
        achieved = terms * OPS_PER_TERM / per_launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Top/s (FP32 issue slots)",
                "frac": achieved / peak_tops,
                "traffic": _traffic_record("boundary_sum", args.workload) if _recorded_kernel(args) else None,
                "kernel": "boundary_sum", "ms_per_launch": per_launch_s * 1e3,
                "edge_terms_per_launch": terms, "ops_per_term": OPS_PER_TERM,
                "edge_terms_per_s": terms / per_launch_s,
                "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                               f"(sm_max_mhz of MEASURED_PEAKS.json)"}
        # the measured pipe rates beside the derived peak: the FP32 and SFU bounds of
        # the same launch (2 SFU operations per term: a reciprocal square root and a
        # reciprocal per chained point)
        mp = pipe_peaks(gwn, float((clk or {}).get("sm_mhz", 0) or sm_max))
        roof["measured_pipes"] = mp
        roof["frac_of_measured_ffma"] = terms * OPS_PER_TERM / per_launch_s / mp["fp32_ffma_slots_per_s"]
        roof["frac_of_measured_ffma2"] = terms * OPS_PER_TERM / per_launch_s / mp["fp32_ffma2_slots_per_s"]
        roof["fp32_bound_ms"] = terms * OPS_PER_TERM / (peak_tops * 1e12) * 1e3
        roof["sfu_bound_ms"] = terms * SFU_OPS_PER_TERM / mp["sfu_ops_per_s"] * 1e3
    # roofline of the traversal (the crossing count): HBM bound.  Algorithmic
    # bytes per query = nodes x 32 B + triangles x 36 B + 12 B query + 4 B count,
    # where nodes and triangles are the query's own visits in this tree (every
    # node whose box the stackless walk of that one query must read: counted by
    # the instrumented per-query walk, untimed), so the count does not depend on
    # the order or grouping the timed kernel uses
    troof = None
    c_launches, chi_ms = prof.get("chi_traversal", (0, 0.0))
    if c_launches and not args.qbits:
        _, nodes_read, tris_tested = m.chi_visits(q_dev)
        tbytes = nodes_read * 32 + tris_tested * 36 + n * 16
        per_s = chi_ms / c_launches / 1e3
        hbm = float(peaks.get("hbm_gbs", 0) or 6800.0)
        troof = {"bound": "hbm", "achieved": tbytes / per_s / 1e9, "peak": hbm, "unit": "GB/s",
                 "frac": tbytes / per_s / 1e9 / hbm,
                 "traffic": _traffic_record("chi_traversal", args.workload) if _recorded_kernel(args) else None,
                 "kernel": "chi_traversal",
                 "ms_per_launch": per_s * 1e3, "bytes_per_launch": int(tbytes),
                 "nodes_per_query": nodes_read / n, "triangles_per_query": tris_tested / n,
                 "peak_source": "hbm_gbs of MEASURED_PEAKS.json" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"}
    kernels = prof_table
    gpu_launches = prof_kernels
    step_roof = step_roofline(roof, troof, step_ms)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mesh, Q, args.cpu_seconds)
    parity = None
    if rank == 0 and not args.no_parity:
        lab_t, w_t = timed_out
        parity = timed_parity(m, mesh, Q, lab_t.cpu().numpy(), w_t.cpu().numpy(), args.parity_sample,
                              quantize_bits=args.qbits)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_tris": mesh.nt,
                           "n_queries_per_rank": n, "n_boundary_edges": info["n_boundary_edges"],
                           "n_boundary_loops": info["n_boundary_loops"], "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{ws} (queries independent, no collective)",
                           "build_s": build_s, "queries_per_thread": args.kq or 4,
                           "predicates": "fixed point, 30 bits" if args.qbits else "exact on FP32 inputs",
                           "fp64_cancel": args.fp64_cancel,
                           "group_test": group_test_name(args.group_test, info["n_boundary_edges"], mesh.nt),
                           "boundary_tile": args.tile or 512},
                "direct_sum": {"value": direct_qps * ws, "unit": "queries/s", "sample_queries": nd,
                               "antipodal_speedup": value / (direct_qps * ws)},
                "roofline": roof, "traversal_roofline": troof, "step_roofline": step_roof,
                "cpu_baseline": cpu, "e2e": e2e,
                "parity": parity, "counters": counters, "gpu_launches": gpu_launches, "kernels": kernels,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    m.close()
    if dist:
        dist.destroy_process_group()
    if parity is not None and not parity["pass"]:
        print(f"parity failed: {parity}", file=sys.stderr, flush=True)
        return 3
    return 0


def batched_parity(items, offs, w, chi, n_sample: int, tol: float = 1e-5):
    """The batched step's output against the oracle: half the sample the
    queries nearest the boundary curve of the five densest meshes, half
    uniform over the whole batch.  w within tol on every query off the boundary
    curve, crossing numbers bit-exact."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(12)
    dens = sorted(range(len(items)), key=lambda i: -len(oracle.boundary(items[i][0].F, items[i][0].nv)))[:5]
    per = max(1, (n_sample // 2) // max(1, len(dens)))
    near = np.concatenate([offs[i] + near_boundary_queries(items[i][0].V, items[i][0].F, items[i][1], per)
                           for i in dens]).astype(np.int64)
    rest = np.setdiff1d(np.arange(int(offs[-1])), near)
    idx = np.concatenate([near, rng.choice(rest, min(n_sample - len(near), len(rest)), replace=False)])
    mesh_of = np.searchsorted(offs, idx, side="right") - 1
    t0 = time.perf_counter()
    dw_all, dw_near, n_chi, excluded = [], [], 0, 0
    for i in np.unique(mesh_of):
        sel = idx[mesh_of == i]
        m = items[i][0]
        ref = oracle.reference(m.V, m.F, items[i][1][sel - offs[i]])
        ok = ref["flags"] == 0
        excluded += int((~ok).sum())
        n_chi += int((chi[sel] != ref["chi"]).sum())
        d = np.abs(w[sel].astype(np.float64) - ref["w_antipodal"])
        dw_all.append(d[ok])
        dw_near.append(d[ok & np.isin(sel, near)])
    dw_all, dw_near = np.concatenate(dw_all), np.concatenate(dw_near)
    out = {"n": int(len(idx)), "n_near_boundary": int(len(near)), "n_uniform": int(len(idx) - len(near)),
           "max_dw": float(dw_all.max()) if len(dw_all) else 0.0,
           "max_dw_near_boundary": float(dw_near.max()) if len(dw_near) else 0.0,
           "chi_mismatch": n_chi, "excluded_on_boundary": excluded, "tolerance": tol,
           "oracle_s": round(time.perf_counter() - t0, 2),
           "what": "the last timed step's w and chi vs the FP64 oracle (exact crossing numbers); near-boundary "
                   "queries from the five meshes with the most boundary edges"}
    out["pass"] = out["max_dw"] <= tol and n_chi == 0
    return out


def run_batched(args):
    """One persistent graph-captured launch over 256 meshes vs one gwn_query_batch per mesh."""
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    items = gen.batched_workload(n_mesh=args.n_mesh, seed=3)
    gen_s = time.perf_counter() - t0
    counts = [len(Q) for _, Q in items]
    t0 = time.perf_counter()
    meshes = [gwn.Mesh(m.V, m.F) for m, _ in items]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    q = torch.from_numpy(np.concatenate([Q for _, Q in items])).to(dev)
    offs = np.concatenate([[0], np.cumsum(counts)])
    n = int(offs[-1])
    stream = torch.cuda.current_stream()
    b = gwn.Batch(meshes, counts)
    t0 = time.perf_counter()
    chosen = b.autotune(q, None)
    tune_s = time.perf_counter() - t0
    w = torch.empty(n, dtype=torch.float32, device=dev)
    chi = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        b.run(q, w, chi)
    torch.cuda.synchronize()
    gwn.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        b.run(q, w, chi)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof, prof_table, prof_kernels = read_profile(gwn)
    gwn.profile_enable(False)
    batch_ms = sum(a.elapsed_time(c) for a, c in ev) / args.steps
    # the same work as one call per mesh
    views = [q[offs[i]:offs[i + 1]] for i in range(len(meshes))]
    w_pm = torch.empty(n, dtype=torch.float32, device=dev)
    def per_mesh():
        for i, m in enumerate(meshes):
            if counts[i]:
                wi, _ = m.query(views[i])
                w_pm[offs[i]:offs[i + 1]] = wi
    per_mesh()
    torch.cuda.synchronize()
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        per_mesh()
    c.record(stream)
    torch.cuda.synchronize()
    pm_ms = a.elapsed_time(c) / args.steps
    max_dw = float(torch.max(torch.abs(w - w_pm)).item())
    parity = None
    if rank == 0 and not args.no_parity:
        b.run(q, w, chi)   # the timed call again: w and chi of one step
        torch.cuda.synchronize()
        parity = batched_parity(items, offs, w.cpu().numpy(), chi.cpu().numpy(), args.parity_sample)
    if rank == 0:
        tris = sum(m.nt for m in meshes)
        medges = [m.info()["n_boundary_edges"] for m in meshes]
        edges = sum(medges)
        # algorithmic FP32 work of the step's boundary terms (the crossing counts
        # are not counted), over the whole persistent launch
        terms = sum(c * e for c, e in zip(counts, medges))
        peaks = _peaks()
        props = torch.cuda.get_device_properties(dev)
        sm_max = float(peaks.get("sm_max_mhz", 0) or (clk or {}).get("sm_max_mhz", 0) or 2070.0)
        peak_tops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
        ach = terms * OPS_PER_TERM / (batch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "Top/s (FP32 issue slots)",
                "frac": ach / peak_tops, "traffic": None, "kernel": "k_batch (whole launch, boundary terms only)",
                "edge_terms_per_step": terms, "ops_per_term": OPS_PER_TERM}
        mp = pipe_peaks(gwn, float((clk or {}).get("sm_mhz", 0) or sm_max))
        roof["fp32_bound_ms"] = terms * OPS_PER_TERM / (peak_tops * 1e12) * 1e3
        roof["sfu_bound_ms"] = terms * SFU_OPS_PER_TERM / mp["sfu_ops_per_s"] * 1e3
        # the crossing counts' algorithmic bytes (each query's own node and
        # triangle reads in its mesh's tree, from the instrumented walk, untimed)
        tbytes = 0
        for i, m in enumerate(meshes):
            if counts[i]:
                _, nodes_read, tris_tested = m.chi_visits(views[i])
                tbytes += nodes_read * 32 + tris_tested * 36 + counts[i] * 16
        hbm = float(peaks.get("hbm_gbs", 0) or 6800.0)
        step_roof = step_roofline(roof, {"bytes_per_launch": tbytes, "peak": hbm}, batch_ms)
        line = {"metric": f"GWN queries/sec, {len(meshes)}-mesh batch in one persistent graph launch",
                "value": ws * n / (batch_ms / 1e3),
                "unit": "queries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"batched: {WORKLOADS['batched']}", "n_mesh": len(meshes), "n_tris": tris,
                           "n_queries": n, "n_boundary_edges": edges, "schedule": chosen, "gen_s": gen_s,
                           "build_s": build_s, "autotune_s": tune_s},
                "per_mesh_launches": {"value": ws * n / (pm_ms / 1e3), "unit": "queries/s", "ms_per_step": pm_ms,
                                      "launches_per_step": 2 * sum(1 for x in counts if x)},
                "batch_speedup": pm_ms / batch_ms, "max_abs_dw_vs_per_mesh": max_dw, "parity": parity,
                "roofline": roof, "step_roofline": step_roof,
                "kernels": prof_table, "gpu_launches": prof_kernels, "clocks": clk}
        line["config"]["l2"] = "flushed between steps (256 MB write)"
        print(json.dumps(line), flush=True)
    b.close()
    for m in meshes:
        m.close()
    if parity is not None and not parity["pass"]:
        print("parity check of the timed output failed", file=sys.stderr, flush=True)
        return 3
    return 0


def run_surrogate(args):
    """Classify a 256^3 grid with the learned surrogate (gate: margin + surface
    band, exact fallback) against plain antipodal classify of the same grid."""
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    mesh, S, G = gen.surrogate_workload(level=args.level or 8, n_train=2_000_000, res=args.res or 256, seed=4)
    gen_s = time.perf_counter() - t0
    n = len(G)
    qg = torch.from_numpy(G).to(dev)
    samples = torch.from_numpy(S).to(dev)
    m = gwn.Mesh(mesh.V, mesh.F)
    info = m.info()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / args.steps

    lab_exact = m.classify(qg)
    plain_ms = timed(lambda: m.classify(qg))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = m.train_surrogate(samples, config={"steps": args.train_steps, "seed": 7})
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    lo, hi = G.min(0), G.max(0)
    held = torch.from_numpy(rng.uniform(lo, hi, size=(1_000_000, 3)).astype(np.float32)).to(dev)
    t0 = time.perf_counter()
    margin, held_err = m.calibrate_surrogate(held, max_error_rate=0.0, min_margin=0.1)
    calib_s = time.perf_counter() - t0

    m.counters(reset=True)
    gwn.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    sur_ms = timed(lambda: m.classify(qg))
    clk = clocks.stop()
    prof, prof_table, prof_kernels = read_profile(gwn)
    gwn.profile_enable(False)
    c = m.counters()
    steps_run = args.warmup + args.steps
    answered = 1.0 - c["surrogate_fallbacks"] / max(c["surrogate_queries"], 1)
    lab = m.classify(qg)
    errors = int((lab != lab_exact).sum().item())

    # end to end with pinned host buffers
    e2e = None
    if not args.no_e2e:
        qh = torch.from_numpy(G).pin_memory()
        m.classify(qh)
        t1 = time.perf_counter()
        m.classify(qh)
        e2e_s = time.perf_counter() - t1
        e2e = {"value": n / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": int(G.nbytes),
               "d2h_bytes_per_step": int(n)}

    # the oracle on a sample of the grid: labels of the surrogate path against FP64 + exact chi
    cpu = None
    oracle_check = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        idx = np.random.default_rng(5).choice(n, 1000, replace=False)
        sub = G[idx]
        E = oracle.boundary(mesh.F, mesh.nv)
        t1 = time.perf_counter()
        chi = oracle.chi(mesh.V, mesh.F, sub)
        w_or, _ = oracle.antipodal(mesh.V, E, sub, chi)
        dt = time.perf_counter() - t1
        lab_or = (np.asarray(w_or) > 0.5).astype(np.uint8)
        lab_np = lab.cpu().numpy()[idx]
        oracle_check = {"sample": len(idx), "label_errors_surrogate_path": int((lab_np != lab_or).sum()),
                        "label_errors_exact_path": int((lab_exact.cpu().numpy()[idx] != lab_or).sum())}
        cpu = {"value": len(idx) / dt, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{len(idx)} seeded random grid queries (FP64 antipodal + exact chi), {dt:.1f} s"}

    # rooflines: the MLP forward on the tensor cores, the boundary sum of the fallback
    peaks = _peaks()
    flop_per_q = 2.0 * (128 * 64 + 3 * 64 * 64)
    mlp_launches, mlp_ms = prof.get("surrogate_forward", (0, 0.0))
    roof_mlp = None
    if mlp_launches:
        per = mlp_ms / mlp_launches / 1e3
        peak = float(peaks.get("bf16_tflops", 0) or 1900.0)
        ach = n * flop_per_q / per / 1e12
        roof_mlp = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": None, "kernel": "surrogate_forward", "ms_per_launch": per * 1e3,
                    "flop_per_query": flop_per_q}
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 0) or (clk or {}).get("sm_max_mhz", 0) or 2070.0)
    peak_tops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    b_l, b_ms = prof.get("boundary_sum", (0, 0.0))
    roof = None
    if b_l:
        per = b_ms / b_l / 1e3
        terms = c["surrogate_fallbacks"] / steps_run * info["n_boundary_edges"]
        ach = terms * OPS_PER_TERM / per / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "Top/s (FP32 issue slots)",
                "frac": ach / peak_tops, "traffic": None, "kernel": "boundary_sum", "ms_per_launch": per * 1e3}
    kernels = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}
    if rank == 0:
        line = {"metric": "GWN classify queries/sec, 256^3 grid, learned surrogate + exact fallback",
                "value": ws * n / (sur_ms / 1e3), "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": sur_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 (network) + f32/f64 (fallback)", "data": "synthetic",
                "config": {"workload": f"surrogate: {WORKLOADS['surrogate']}", "n_tris": mesh.nt,
                           "n_queries": n, "n_boundary_edges": info["n_boundary_edges"],
                           "l2": "flushed between steps (256 MB write)", "gen_s": gen_s,
                           "train_steps": args.train_steps, "train_batch": 16384, "train_s": train_s, "final_loss": loss,
                           "gate": "|w_hat - 1/2| > margin, outside the surface band, |w_hat - chi| <= 0.25 (chi exact, every query)",
                           "calibration": {"samples": 1_000_000, "max_error_rate": 0.0, "margin": margin,
                                           "held_out_errors": held_err, "seconds": calib_s}},
                "plain_antipodal": {"value": ws * n / (plain_ms / 1e3), "unit": "queries/s", "ms_per_step": plain_ms},
                "surrogate_speedup": plain_ms / sur_ms, "answered_by_network": answered,
                "label_errors_vs_exact_path": errors, "oracle_check": oracle_check,
                "roofline": roof, "roofline_mlp": roof_mlp, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": prof_kernels, "kernels": prof_table, "clocks": clk}
        print(json.dumps(line), flush=True)
    m.close()
    return 0


def run_surrogate_infer(args):
    """Throughput of the surrogate network's forward pass on the tensor cores."""
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mesh, _ = gen.displaced_soup(8, 4)
    G = gen.grid_queries(mesh.V, 256)
    n = len(G)
    qg = torch.from_numpy(G).to(dev)
    m = gwn.Mesh(mesh.V, mesh.F, build=False)
    lib = gwn.load()
    rng = np.random.default_rng(6)
    parts = [rng.normal(scale=np.sqrt(2.0 / 128), size=64 * 128), np.zeros(64)]
    for _ in range(3):
        parts += [rng.normal(scale=np.sqrt(2.0 / 64), size=64 * 64), np.zeros(64)]
    parts += [rng.normal(scale=0.2, size=64), np.zeros(1)]
    params = np.concatenate(parts).astype(np.float32)
    assert params.size == lib.gwn_surrogate_num_params()
    m.set_surrogate_params(params, np.concatenate([G.min(0), G.max(0)]).astype(np.float32))
    w = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)

    def step():
        gwn._check(lib.gwn_surrogate_predict(m.handle, ctypes.c_void_p(qg.data_ptr()), n,
                                             ctypes.c_void_p(w.data_ptr()), sp))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    peaks = _peaks()
    flop_per_q = 2.0 * (128 * 64 + 3 * 64 * 64)
    peak = float(peaks.get("bf16_tflops", 0) or 1900.0)
    ach = n * flop_per_q / (ms / 1e3) / 1e12
    if rank == 0:
        line = {"metric": "surrogate network queries/sec (forward on the tensor cores)", "value": ws * n / (ms / 1e3),
                "unit": "queries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": f"surrogate_infer: {WORKLOADS['surrogate_infer']}", "n_queries": n,
                           "l2": "flushed between steps (256 MB write); inputs 201 MB > L2"},
                "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                             "traffic": None, "kernel": "k_mlp_forward", "flop_per_query": flop_per_q,
                             "algorithmic_bytes_per_query": 16},
                "gpu_launches": args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    m.close()
    return 0


def run_gradient(args):
    """Throughput of gwn_query_gradient on the soup8 queries."""
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mesh, Q = gen.workload("soup8", n_query=args.n_query)
    n = len(Q)
    qd = torch.from_numpy(Q).to(dev)
    m = gwn.Mesh(mesh.V, mesh.F)
    info = m.info()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        m.gradient(qd)
    torch.cuda.synchronize()
    gwn.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        m.gradient(qd)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof, prof_table, prof_kernels = read_profile(gwn)
    gwn.profile_enable(False)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    launches, gms = prof.get("gradient", (0, 0.0))
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 0) or (clk or {}).get("sm_max_mhz", 0) or 2070.0)
    peak_tops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    roof = None
    if launches:
        per = gms / launches / 1e3
        terms = n * info["n_boundary_edges"]
        ach = terms * GRAD_OPS_PER_TERM / per / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "Top/s (FP32 issue slots)",
                "frac": ach / peak_tops, "traffic": None, "kernel": "k_gradient", "ms_per_launch": per * 1e3,
                "edge_terms_per_launch": terms, "ops_per_term": GRAD_OPS_PER_TERM}
    e2e = None
    if not args.no_e2e:
        qh = torch.from_numpy(Q).pin_memory()
        m.gradient(qh)
        t1 = time.perf_counter()
        m.gradient(qh)
        dt = time.perf_counter() - t1
        e2e = {"value": n / dt, "unit": "queries/s", "h2d_bytes_per_step": int(Q.nbytes),
               "d2h_bytes_per_step": int(12 * n)}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        idx = np.random.default_rng(5).choice(n, 4000, replace=False)
        E = oracle.boundary(mesh.F, mesh.nv)
        t1 = time.perf_counter()
        oracle.gradient(mesh.V, E, Q[idx])
        dt = time.perf_counter() - t1
        cpu = {"value": len(idx) / dt, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{len(idx)} seeded random queries of the workload (FP64 Algorithm 3), {dt:.1f} s"}
    if rank == 0:
        line = {"metric": "GWN gradient queries/sec at 1M tris (Supp. S4, Algorithm 3)", "value": ws * n / (ms / 1e3),
                "unit": "queries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"gradient: {WORKLOADS['gradient']}", "n_tris": mesh.nt, "n_queries": n,
                           "n_boundary_edges": info["n_boundary_edges"], "l2": "flushed between steps (256 MB write)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": prof_kernels, "kernels": prof_table, "clocks": clk}
        print(json.dumps(line), flush=True)
    m.close()
    return 0


def _grid_axes(V, res, pad=0.1):
    import numpy as np
    V = np.asarray(V, dtype=np.float64)
    lo, hi = V.min(0), V.max(0)
    ext = hi - lo
    lo, hi = lo - pad * ext, hi + pad * ext
    return [(lo[d] + (np.arange(res) + 0.5) * (hi[d] - lo[d]) / res).astype(np.float32) for d in range(3)]


def run_grid(args):
    """Grid classify with ray reuse against per-point classify of the same cells."""
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    gwn.profile_enable(True)
    for name, hole_p in (("closed", 0.0), ("holed", 0.02)):
        mesh, _ = gen.displaced_soup(8, seed=4, hole_p=hole_p)
        x, y, z = _grid_axes(mesh.V, 256)
        Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
        P = torch.from_numpy(np.stack([Xg.ravel(), Yg.ravel(), Zg.ravel()], 1).astype(np.float32)).to(dev)
        del Xg, Yg, Zg
        n = P.shape[0]
        m = gwn.Mesh(mesh.V, mesh.F)
        lab_g = m.classify_grid(x, y, z)
        lab_p = m.classify(P)
        same = bool(torch.equal(lab_g.ravel(), lab_p))
        steps = args.steps if name == "closed" else max(1, min(args.steps, 2))
        warm = args.warmup if name == "closed" else 1
        g_ms = timed(lambda: m.classify_grid(x, y, z), steps, warm)
        p_ms = timed(lambda: m.classify(P), steps, warm)
        out[name] = {"n_tris": mesh.nt, "n_boundary_edges": m.info()["n_boundary_edges"], "n_queries": n,
                     "grid_ms": g_ms, "per_point_ms": p_ms, "grid_qps": n / (g_ms / 1e3),
                     "per_point_qps": n / (p_ms / 1e3), "speedup": p_ms / g_ms, "labels_identical": same}
        if name == "closed":
            # the per-point classify of a closed mesh is its traversal: HBM roofline
            # with nodes x 32 B + triangles x 36 B + 12 B + 4 B per query (instrumented walk)
            _, nodes_read, tris_tested = m.chi_visits(P)
            tbytes = nodes_read * 32 + tris_tested * 36 + n * 16
            hbm = float(_peaks().get("hbm_gbs", 0) or 6800.0)
            out[name]["traversal_roofline"] = {
                "bound": "hbm", "achieved": tbytes / (p_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": tbytes / (p_ms / 1e3) / 1e9 / hbm, "traffic": None,
                "kernel": "chi_traversal (whole per-point classify)", "bytes_per_launch": int(tbytes),
                "nodes_per_query": nodes_read / n, "triangles_per_query": tris_tested / n}
        m.close()
        del P
    prof, prof_table, prof_kernels = read_profile(gwn)
    gwn.profile_enable(False)
    clk = clocks.stop()
    c = out["closed"]
    if rank == 0:
        line = {"metric": "GWN grid classify queries/sec with ray reuse (Supp. S3), 256^3 grid, closed 2.6M-tri mesh",
                "value": ws * c["grid_qps"], "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": c["grid_ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"grid: {WORKLOADS['grid']}", "l2": "flushed between steps (256 MB write)"},
                "closed_mesh": out["closed"], "holed_soup8": out["holed"],
                "kernels": prof_table, "gpu_launches": prof_kernels, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


# FP32 issue slots per quadrature panel of the parametric boundary integral
# (Algorithm 2's integrand in the closed form r x r' / (L (L - r_z)), 15
# Gauss-Kronrod nodes): per node 12 FMA for the point, 8 for the derivative's
# x and y, 2 for the z-cross product, 3 for rho^2 and L^2, 3 for the two
# branches' products, 2 for g and f, 3 accumulations (K15, G7, rounding
# scale) and 2 for the scale's absolute values -> 35 slots and 2 SFU (sqrt,
# reciprocal); per panel 24 for the centre's float-pair difference and 12 for
# the control points -> 15 * 35 + 36 = 561 slots.
PARAM_OPS_PER_PANEL = 15 * 35.0 + 36.0


def run_param(args):
    """Parametric surfaces (Sec. 4.4, Algorithm 2): cells/s of gwn_param_query_grid
    on the random-patch voxel workload (ray reuse per column, FP32 panels);
    per-point queries and FP64 panels timed beside it."""
    import numpy as np
    import torch
    import gen
    import paper_2605_01536_gb300 as gwn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P, Q = gen.param_workload()
    n = len(Q)
    axes = [np.unique(Q[:, d]) for d in range(3)]
    qd = torch.from_numpy(Q).to(dev)
    t0 = time.perf_counter()
    surf = gwn.ParamSurface(P)
    create_s = time.perf_counter() - t0
    surf64 = gwn.ParamSurface(P, fp64=1)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    for _ in range(args.warmup):
        surf.query_grid(*axes)
    torch.cuda.synchronize()
    surf.status(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed(lambda: surf.query_grid(*axes), args.steps, 0)
    clk = clocks.stop()
    status = surf.status(reset=True)
    panels_per_step = status["panels"] / args.steps
    # kernel times from a separate profiled pass (the events the profiler adds
    # cost host time that would show in the step above)
    gwn.profile_enable(True)
    timed(lambda: surf.query_grid(*axes), args.steps, 0)
    prof, prof_table, prof_kernels = read_profile(gwn)
    gwn.profile_enable(False)
    surf.status(reset=True)
    point_ms = timed(lambda: surf.query(qd), max(1, min(args.steps, 3)), 1)
    fp64_ms = timed(lambda: surf64.query_grid(*axes), max(1, min(args.steps, 2)), 1)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 0) or (clk or {}).get("sm_max_mhz", 0) or 2070.0)
    peak_tops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    roof = None
    launches, bms = prof.get("param_boundary", (0, 0.0))
    if launches:
        per = bms / launches / 1e3
        ach = panels_per_step * PARAM_OPS_PER_PANEL / per / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "Top/s (FP32 issue slots)",
                "frac": ach / peak_tops, "traffic": _traffic_record("param_boundary", "param"),
                "kernel": "k_param_boundary<GridPoints>",
                "ms_per_launch": per * 1e3, "panels_per_launch": panels_per_step,
                "ops_per_panel": PARAM_OPS_PER_PANEL}
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        w, chi = surf.query_grid(*axes)
        w.cpu()
        chi.cpu()
        dt = time.perf_counter() - t1
        e2e = {"value": n / dt, "unit": "queries/s", "h2d_bytes_per_step": int(sum(a.nbytes for a in axes)),
               "d2h_bytes_per_step": int(8 * n)}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import parametric as par
        curves = par.boundary_curves(P.astype(np.float64))
        idx = np.random.default_rng(5).choice(n, 3, replace=False)
        t1 = time.perf_counter()
        for k in idx:
            par.boundary_term(curves, Q[k].astype(np.float64))
        dt = time.perf_counter() - t1
        cpu = {"value": len(idx) / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(idx)} seeded random cells: the FP64 Algorithm 2 boundary integral over all "
                         f"{len(curves)} curves (scipy quad), {dt:.1f} s; the oracle has no ray-patch "
                         f"intersection, so chi is not included"}
    if rank == 0:
        nc = int(surf.boundary_curves().shape[0])
        line = {"metric": "parametric GWN queries/sec, 100 random bicubic Bezier patches, 32^3 voxel grid "
                          "(Sec. 4.4, Algorithm 2)",
                "value": ws * n / (ms / 1e3), "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 (FP64 below panel depth 12, for leaf corners and the bilinear solve)",
                "data": "synthetic",
                "config": {"workload": f"param: {WORKLOADS['param']}", "n_patches": int(P.shape[0]),
                           "n_boundary_curves": nc, "n_queries": n, "l2": "flushed between steps (256 MB write)",
                           "create_s": create_s},
                "panels_per_query_curve": panels_per_step / (n * max(nc, 1)),
                "per_point_ms": point_ms, "per_point_qps": n / (point_ms / 1e3),
                "fp64_panels_ms": fp64_ms, "fp64_panels_qps": n / (fp64_ms / 1e3),
                "status": status, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "kernels": prof_table, "gpu_launches": prof_kernels, "clocks": clk}
        print(json.dumps(line), flush=True)
    surf.close()
    surf64.close()
    return 0


def pipe_peaks(gwn, sm_mhz: float):
    """The measured FP32 and SFU rates of this GPU (gwn_measure_pipe_peaks), also
    per SM and clock at the given SM clock."""
    p = gwn.measure_pipe_peaks()
    per = p["sm_count"] * sm_mhz * 1e6
    return {"fp32_ffma_slots_per_s": p["ffma_per_s"], "fp32_ffma2_slots_per_s": 2.0 * p["ffma2_per_s"],
            "sfu_ops_per_s": p["mufu_per_s"], "ffma_per_sm_clock": p["ffma_per_s"] / per,
            "ffma2_slots_per_sm_clock": 2.0 * p["ffma2_per_s"] / per, "sfu_per_sm_clock": p["mufu_per_s"] / per,
            "sm_mhz_assumed": sm_mhz}


def run_peaks(args):
    """Measured FP32 (scalar and paired FMA) and SFU throughputs against the
    peak derived from 128 FP32 lanes per SM at the maximum clock."""
    import torch
    import paper_2605_01536_gb300 as gwn
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    gwn.measure_pipe_peaks()   # warm the clocks up
    p = pipe_peaks(gwn, 1.0)
    clk = clocks.stop()
    sm_mhz = float((clk or {}).get("sm_mhz", 0) or _peaks().get("sm_max_mhz", 0) or 2070.0)
    p = {k: (v / sm_mhz if "per_sm_clock" in k else v) for k, v in p.items()}
    p["sm_mhz_assumed"] = sm_mhz
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * FP32_LANES_PER_SM * float(_peaks().get("sm_max_mhz", 0) or 2070.0) * 1e6
    line = {"metric": "FP32 issue slots/s (scalar FMA) measured, with paired-FMA and SFU rates",
            "value": p["fp32_ffma_slots_per_s"], "unit": "slots/s", "n_gpus": 1, "steps": 3, "warmup": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"peaks: {WORKLOADS['peaks']}", "sm_count": sms},
            "fp32_derived_slots_per_s": derived, **p,
            "ffma_over_derived": p["fp32_ffma_slots_per_s"] / derived,
            "ffma2_over_derived": p["fp32_ffma2_slots_per_s"] / derived, "clocks": clk, "gpu_launches": 24}
    print(json.dumps(line), flush=True)
    return 0


def step_roofline(roof, troof, step_ms):
    """The whole step against its roofline: the boundary sum's bound (the larger
    of its FP32 issue and SFU times) plus the crossing count's byte time at the
    HBM rate, over the measured step time."""
    if not roof or "fp32_bound_ms" not in roof:
        return None
    a5 = max(roof["fp32_bound_ms"], roof.get("sfu_bound_ms", 0.0))
    a4 = troof["bytes_per_launch"] / (troof["peak"] * 1e9) * 1e3 if troof else 0.0
    return {"boundary_bound_ms": a5, "traversal_byte_bound_ms": a4, "roofline_ms": a5 + a4,
            "measured_ms": step_ms, "frac": (a5 + a4) / step_ms,
            "definition": "(max(FP32 issue, SFU) time of the boundary terms + the crossing count's algorithmic "
                          "bytes at the measured HBM rate) / measured step time"}


def group_test_name(flag, nb, nt):
    """The boundary kernel's group acceptance test for a mesh (the library's
    rule for gwn_config.group_test = 0: running where nb >= nt / 2)."""
    running = flag == 2 or (flag == 0 and nb > 0 and 2 * nb >= nt)
    return "running (product keeps a positive real part)" if running else "per term (angle below pi/8)"


def main():
    args = parse()
    if args.workload == "peaks":
        return run_peaks(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "surrogate_infer":
        return run_surrogate_infer(args)
    if args.workload == "gradient":
        return run_gradient(args)
    if args.workload == "grid":
        return run_grid(args)
    if args.workload == "param":
        return run_param(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
