"""Benchmark: seconds per colouring of colour-coding tree counting on the
1M-vertex R-MAT workload, FP32-batched form vs plain FP64 form.

Workload: R-MAT scale 20 (a,b,c,d = .57,.19,.19,.05, ids permuted),
2^24 undirected edges, template tree10 (parent [-1,0,1,1,0,4,5,5,2,6], root
0), k = 10 colours.  One step of the FP32-batched form counts B colourings in
one call; one step of the plain form counts one colouring in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank counts its
own colourings on its own GPU (replicas: colourings are independent), the
step time is the maximum over ranks and `value` covers all ranks' colourings.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sg2v_inputs as si  # noqa: E402

METRIC = "seconds per coloring + HBM GB/s vs peak, FP32-batched vs FP64 plain, RMAT 1M"
UNIT = "s/colouring"
WORKLOAD = "rmat20_16m_tree10_k10"
# plan of the headline template: work-minimising cut order (measured 3.6% faster than cutting the
# last child on this workload; the counts do not depend on it)
PLAN_CUT = "min_work"
TEMPLATE = si.TREE10
K_COLOURS = 10
FULL_SCALE, FULL_EDGES = 20, 1 << 24


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def fp64_peak_ops(torch):
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (4096^3, best of 5,
    CUDA events), in FP64 operations per second counting one fused
    multiply-add as one operation (the unit of the FP64 node kernels' adds
    and FMAs)."""
    nsz = 4096
    a = torch.randn(nsz, nsz, dtype=torch.float64, device="cuda")
    b = torch.randn(nsz, nsz, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return float(nsz) ** 3 / (best * 1e-3)


def fp32_alu_peak_flops(peaks):
    """FP32 FMA throughput from unit counts and clocks: 148 SMs x 128 FP32
    lanes x 2 FLOP per FMA x the maximum SM clock."""
    return 148 * 128 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6


def node_fp64_ops(t, a, p, kc, n, nnz, half_root):
    """FP64 adds and FMAs of one node launch over n rows (one colouring):
    the gather adds one compressed row of C(kc-1, p-1) entries per arc to a
    neighbour of another colour (a colour count for p = 1), Y' sums p
    per-colour terms for each of its C(kc-1, p) sets, and the eMA does
    C(t-1, a-1) products per output set (one per p-set at a one-set root)."""
    from math import comb

    arcs = nnz * (kc - 1) / kc * (0.5 if half_root else 1.0)
    ops = arcs * (1 if p == 1 else comb(kc - 1, p - 1))
    ops += n * comb(kc - 1, p) * p
    if a >= 2:
        ops += n * (comb(kc - 1, p) if t == kc else comb(kc - 1, t - 1) * comb(t - 1, a - 1))
    return ops


def parse_node(name):
    """(t, a, p) from a kernel record name 'node t=T a=A p=P ...'."""
    parts = dict(x.split("=") for x in name.split() if "=" in x)
    return int(parts["t"]), int(parts["a"]), int(parts["p"])


def records_block(records, steps, units):
    """Per-kernel table and step totals of one block's kernel records."""
    table = {}
    step_bytes = step_ms = 0.0
    for r in records:
        per = r["total_ms"] / r["launches"]
        table[r["name"]] = {"launches_per_step": r["launches"] / steps, "ms_per_launch": round(per, 4),
                            "algorithmic_GB_per_launch": round(r["bytes_per_launch"] / 1e9, 4),
                            "GBps": round(r["bytes_per_launch"] / (per * 1e-3) / 1e9, 1) if per > 0 else None}
        step_bytes += r["bytes_per_launch"] * r["launches"] / steps
        step_ms += r["total_ms"] / steps
    return table, step_bytes, step_ms


def hbm_roofline(name, bytes_per_launch, ms_per_launch, peak, peak_kind):
    achieved = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind}


def gather_rate(rec, g, kc, ms):
    """Bytes the dominant node kernel gathers per launch (one compressed row
    of C(kc-1, p-1) FP32 entries per arc to a neighbour of another colour;
    half the arcs at a root whose children are one table) over its time,
    against the L2 bandwidth ncu reports as the GPU's peak (profiles/l2_peak.json)."""
    from math import comb

    t, a, p = parse_node(rec["name"])
    if p < 2:
        return None
    arcs = g.nnz * (kc - 1) / kc * (0.5 if (t == kc and a == p) else 1.0)
    gathered = arcs * comb(kc - 1, p - 1) * 4
    out = {"bytes_per_launch": gathered, "GBps": gathered / (ms * 1e-3) / 1e9}
    try:
        l2 = json.load(open(os.path.join(ROOT, "profiles", "l2_peak.json")))
        out.update({"l2_peak_GBps": l2["l2_peak_GBps"], "frac_of_l2_peak": out["GBps"] / l2["l2_peak_GBps"],
                    "l2_peak_source": l2["source"]})
    except (OSError, KeyError, ValueError):
        pass
    return out


def source_digest() -> str:
    """Digest of the sources that decide what a node launch does (kernels and
    the executor that sets its launch configuration)."""
    h = hashlib.sha256()
    for name in ("kernels.cu", "run_kernel.cu", "device_common.cuh", "kernels.cuh", "api.cu"):
        h.update(open(os.path.join(ROOT, "paper_2009_11665_b300", "csrc", name), "rb").read())
    return h.hexdigest()


def traffic_record():
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except OSError:
        return {}
    if rec.get("source_sha256") != source_digest():
        return {}
    return rec.get("bytes_per_launch", {})


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_seconds_per_colouring(scale: int, threads: int):
    """The exact CPU oracle on an R-MAT sibling of the workload (same R-MAT
    parameters and average degree, 2^scale vertices), one colouring; seconds
    scaled linearly in the edge count to the full workload."""
    import oracle

    g = si.rmat(scale, (1 << scale) * 16, seed=0)
    col = si.colouring(g.n, K_COLOURS, 0)
    t0 = time.perf_counter()
    oracle.count(g.row_ptr, g.col_idx, TEMPLATE.parent, 0, col, per_vertex=False, threads=threads)
    dt = time.perf_counter() - t0
    factor = FULL_EDGES / g.m
    return dt * factor, dt, g


def run_reference(args, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    scale = args.reference_scale
    for _ in range(args.warmup):
        oracle_seconds_per_colouring(scale, threads)
    vals, raw = [], []
    for _ in range(args.steps):
        v, dt, g = oracle_seconds_per_colouring(scale, threads)
        vals.append(v)
        raw.append(dt)
    value = statistics.median(vals)
    sample = (f"exact oracle DP (128-bit integers) on R-MAT scale {scale} ({g.m} edges, same parameters and "
              f"average degree), 1 colouring of tree10 per step; seconds x{FULL_EDGES // g.m} (work is linear "
              f"in the edge count)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.median(raw) * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": "rmat scale 20, 2^24 edges", "template": list(TEMPLATE.parent),
                   "num_colours": K_COLOURS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def physical_gpu_index(local: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p.strip() for p in vis.split(",") if p.strip()]
    if local < len(parts) and parts[local].isdigit():
        return int(parts[local])
    return local


def rank_colourings(n: int, kc: int, batch: int, rank: int, seed: int) -> np.ndarray:
    """Colourings of `rank` (replicas over colourings, Alg. 1's independent
    draws): indices rank*batch .. rank*batch+batch-1 of one seeded stream, so
    the ranks' colourings are disjoint and together the stream's first
    world*batch."""
    return si.colourings(n, kc, batch * (rank + 1), seed=seed)[rank * batch:(rank + 1) * batch]


def max_over_ranks(torch, value: float, dist=None) -> float:
    """The largest of every rank's value (the whole job's step time); the
    reduction runs on the GPU under NCCL and on the host under gloo."""
    if not dist:
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(torch, fn, steps, warmup, stream, dist=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    stop.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(torch, start.elapsed_time(stop), dist)
    if dist:
        dist.barrier()
    return ms / steps


def profile_call(args):
    """One sg2v_count_batched call (B = --batch colourings): tree10 on an
    R-MAT graph with the workload's parameters and average degree 32
    (rmat18, rmat19, rmat20), or tree15 with k = 15 on the large form's scale-17
    sibling (large17: 6.25e6 edges, average degree about 95); chunglu200k_grad
    runs the differentiable form's forward and forward + gradient calls."""
    import torch

    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as sg

    torch.cuda.set_device(0)
    if args.profile_call == "er_degrees":
        # the same 2^24 edges on 2^22 .. 2^18 vertices (average degree 8 .. 128): the
        # run kernels' cost per row, per colour run and per gathered arc
        for scale in (22, 21, 20, 19, 18):
            g = si.erdos_renyi(1 << scale, 1 << 24, seed=1)
            graph = sg.Graph(g.row_ptr, g.col_idx)
            plan = sg.Plan(TEMPLATE.parent, 0, K_COLOURS, cut=PLAN_CUT, avg_degree=32.0)
            cols = si.colourings(g.n, K_COLOURS, 1, seed=0)
            tot = torch.empty((1, 1), dtype=torch.float64, device="cuda")
            sg.sg2v_count_batched(graph.handle, [plan.handle], torch.from_numpy(cols).cuda(), 1, sg.SG2V_FP32, None,
                                  tot)
            torch.cuda.synchronize()
            c = cols[0].astype(np.int64)
            rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
            nc = c[g.col_idx]
            keep = nc != c[rows]
            runs = np.unique(rows[keep] * 16 + nc[keep]).size
            print(json.dumps({"vertices": g.n, "gathered_arcs": int(keep.sum()), "colour_runs": int(runs),
                              "total": float(tot[0, 0])}))
            del graph
        return
    if args.profile_call == "chunglu200k_grad":
        # the differentiable form's workload: one forward call, then one
        # forward + gradient call (stored form), FP32, tree8, k = 8
        g = si.workload_graph("chunglu200k")
        w = si.arc_weights(g, si.edge_weights(g, seed=0))
        graph = sg.Graph(g.row_ptr, g.col_idx, w)
        plan = sg.Plan(si.TREE8.parent, 0, 8)
        col = torch.from_numpy(si.colouring(g.n, 8, 0)).cuda()
        tot = torch.empty((1, 1), dtype=torch.float64, device="cuda")
        grad = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        sg.sg2v_count_batched(graph.handle, [plan.handle], col, 1, sg.SG2V_FP32, None, tot)
        total = sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.SG2V_FP32, grad, None,
                                       flags=sg.SG2V_BACKWARD_STORE)
        torch.cuda.synchronize()
        print(json.dumps({"profile_call": args.profile_call, "total": float(tot[0, 0]), "backward_total": total,
                          "grad_abs_sum": float(grad.abs().sum())}))
        return
    if args.profile_call == "large17":
        g = si.rmat(17, 50_000_000 >> 3, seed=0)
        template, kc = si.TREE15, 15
    else:
        scale = {"rmat18": 18, "rmat19": 19, "rmat20": 20}[args.profile_call]
        g = si.rmat(scale, (1 << scale) * 16, seed=0)
        template, kc = TEMPLATE, K_COLOURS
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(template.parent, 0, kc, cut=PLAN_CUT if template is TEMPLATE else None, avg_degree=32.0)
    cols = torch.from_numpy(si.colourings(g.n, kc, args.batch, seed=0)).cuda()
    tot = torch.empty((1, args.batch), dtype=torch.float64, device="cuda")
    sg.sg2v_count_batched(graph.handle, [plan.handle], cols, args.batch, sg.PRECISIONS[args.precision], None, tot)
    torch.cuda.synchronize()
    print(json.dumps({"profile_call": args.profile_call, "batch": args.batch, "precision": args.precision,
                      "totals": tot.cpu().tolist()}))


def session_headline(sg, torch, graph, plan, B, d_cols, h_cols, tot, est, h_tot, h_est, stream, args, dist):
    """The headline step through an autotuned session: its first run (a
    warm-up step) times the split schedule, wave width and node forms; later
    runs replay a CUDA graph.  Timed from device colourings and, end to end,
    from pinned host colourings with host totals and estimates."""
    ses = sg.Session(graph, [plan], B, "fp32", autotune=True)
    ms = time_steps(torch, lambda: ses.run(d_cols, tot, est, None, stream), args.steps, args.warmup, stream, dist)
    ms_e2e = time_steps(torch, lambda: ses.run(h_cols, h_tot, h_est, None, stream), max(3, args.steps // 2),
                        args.warmup, stream, dist)
    tuning = ses.tuning()
    ses.close()
    return {"s_per_colouring": ms * 1e-3 / B, "e2e_s_per_colouring": ms_e2e * 1e-3 / B, "wave": tuning["wave"],
            "split_chunk": tuning["chunk"], "cuda_graph": True,
            "forms": [f"({n['t']},{n['a']},{n['p']}) {n['kernel']}" for n in tuning["nodes"]]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=int(os.environ.get("SG2V_BENCH_BATCH", "4")))
    ap.add_argument("--impl", default="sg2v", choices=["sg2v", "reference"])
    ap.add_argument("--reference-scale", type=int, default=16)
    ap.add_argument("--cpu-baseline-scale", type=int, default=17)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 3-template x 64-colouring session block")
    ap.add_argument("--no-large", action="store_true", help="skip the tree15 (k = 15) large-form block")
    ap.add_argument("--no-session", action="store_true", help="skip the headline step through an autotuned session")
    ap.add_argument("--profile-call", choices=["rmat18", "rmat19", "rmat20", "large17", "er_degrees",
                                               "chunglu200k_grad"], default=None,
                    help="run exactly one count call (R-MAT scale 18, 19 or 20 with avg degree 32 and tree10, or the "
                         "large form's scale-17 sibling with tree15; chunglu200k_grad: the differentiable form's "
                         "forward call and forward + gradient call) and exit: the cases the committed ncu "
                         "summaries capture")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp32_scaled", "u64", "u128"], default="fp32")
    args = ap.parse_args()
    if args.profile_call:
        profile_call(args)
        return
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and "RANK" in os.environ:
        print(f"warning: WORLD_SIZE {world} != --gpus {args.gpus}", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as sg

    B = args.batch
    g = si.workload_graph("rmat20_16m")
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(TEMPLATE.parent, 0, K_COLOURS, cut=PLAN_CUT, avg_degree=32.0)
    # colourings of this rank: indices rank*B .. rank*B+B-1 (replicas over colourings)
    cols = rank_colourings(g.n, K_COLOURS, B, rank, seed=0)
    d_cols = torch.from_numpy(cols).cuda()
    stream = torch.cuda.current_stream()
    tot32 = torch.empty((1, B), dtype=torch.float64, device="cuda")
    est32 = torch.empty((1, B), dtype=torch.float64, device="cuda")
    tot64 = torch.empty((1, 1), dtype=torch.float64, device="cuda")

    def step_fp32():
        sg.sg2v_count_batched(graph.handle, [plan.handle], d_cols, B, sg.SG2V_FP32, None, tot32, est32, stream)

    def step_fp64():
        sg.sg2v_count_batched(graph.handle, [plan.handle], d_cols[0:1], 1, sg.SG2V_FP64, None, tot64, None, stream)

    # plain FP64 form: event records of its kernels over the timed steps, and
    # the FP64 operation rate of its node kernels against measured DGEMM
    peaks, peak_kind = measured_peaks()
    steps64 = max(3, args.steps // 2)
    for _ in range(args.warmup):
        step_fp64()
    torch.cuda.synchronize()
    sg.sg2v_profile_reset()
    sg.sg2v_profile_enable(True)
    ms64 = time_steps(torch, step_fp64, steps64, 0, stream, dist)
    sg.sg2v_profile_enable(False)
    rec64 = sg.sg2v_profile_read()
    fp64_ops_peak = fp64_peak_ops(torch)
    ops64 = ms_nodes64 = 0.0
    for r in rec64:
        if r["name"].startswith("node"):
            t, a, p = parse_node(r["name"])
            ops64 += node_fp64_ops(t, a, p, K_COLOURS, g.n, g.nnz, half_root=(t == len(TEMPLATE.parent) and a == p)) \
                * r["launches"] / steps64
            ms_nodes64 += r["total_ms"] / steps64

    # FP32-batched form (the headline): kernel records collected over the timed region
    for _ in range(args.warmup):
        step_fp32()
    torch.cuda.synchronize()
    sg.sg2v_profile_reset()
    sg.sg2v_profile_enable(True)
    with ClockSampler(physical_gpu_index(local)) as clocks:
        ms32 = time_steps(torch, step_fp32, args.steps, 0, stream, dist)
    sg.sg2v_profile_enable(False)
    launches = sg.sg2v_launch_count()
    records = sg.sg2v_profile_read()

    # end-to-end through the C ABI with host buffers, copies inside the timed
    # region: the colourings from pinned host memory in, the step's result
    # (totals and estimates) out; then the same with the per-vertex counts
    # too (their root gathers every arc, and 8 bytes per vertex come back)
    h_cols = torch.from_numpy(cols).pin_memory()
    h_pv = torch.empty((1, B, g.n), dtype=torch.float64).pin_memory()
    h_tot = np.zeros((1, B))
    h_est = np.zeros((1, B))

    def step_e2e():
        sg.sg2v_count_batched(graph.handle, [plan.handle], h_cols, B, sg.SG2V_FP32, None, h_tot, h_est, stream)

    def step_e2e_pv():
        sg.sg2v_count_batched(graph.handle, [plan.handle], h_cols, B, sg.SG2V_FP32, h_pv, h_tot, h_est, stream)

    ms_e2e = time_steps(torch, step_e2e, max(3, args.steps // 2), args.warmup, stream, dist)
    ms_e2e_pv = time_steps(torch, step_e2e_pv, max(3, args.steps // 2), args.warmup, stream, dist)

    # the same step through an autotuned session
    session_block = None
    if not args.no_session:
        session_block = session_headline(sg, torch, graph, plan, B, d_cols, h_cols, tot32, est32, h_tot, h_est,
                                         stream, args, dist)

    # batched form: 64 colourings x 3 templates (path7, star7, tree7, k = 7) on
    # R-MAT scale 18 (avg degree 16), one CUDA-graph replay per step, autotuned waves
    batched = None
    if not args.no_batched:
        g3 = si.workload_graph("rmat18_d16")
        graph3 = sg.Graph(g3.row_ptr, g3.col_idx)
        plans3 = [sg.Plan(t.parent, 0, 7) for t in (si.PATH7, si.STAR7, si.TREE7)]
        B3 = 64
        ses = sg.Session(graph3, plans3, B3, "fp32", autotune=True)
        cols3 = torch.from_numpy(rank_colourings(g3.n, 7, B3, rank, seed=1)).cuda()
        tot3 = torch.empty((3, B3), dtype=torch.float64, device="cuda")
        ms3 = time_steps(torch, lambda: ses.run(cols3, tot3, None, None, stream), args.steps, args.warmup, stream,
                         dist)
        ses.sync(stream)
        wave3, graph_on = ses.info()
        tuning3 = ses.tuning()
        # kernel records of separate (profiled) steps: algorithmic bytes per step over the step time
        sg.sg2v_profile_reset()
        sg.sg2v_profile_enable(True)
        for _ in range(3):
            ses.run(cols3, tot3, None, None, stream)
        ses.sync(stream)
        torch.cuda.synchronize()
        sg.sg2v_profile_enable(False)
        tab3, bytes3, kms3 = records_block(sg.sg2v_profile_read(), 3, 1)
        dom3 = max(tab3.items(), key=lambda kv: kv[1]["ms_per_launch"] * kv[1]["launches_per_step"])
        batched = {"workload": "rmat18_d16 (R-MAT scale 18, avg degree 16), path7+star7+tree7, k=7, 64 colourings",
                   "ms_per_step": ms3, "s_per_colouring_template": ms3 * 1e-3 / (B3 * 3 * world),
                   "wave": wave3, "split_chunk": tuning3.get("chunk"), "cuda_graph": graph_on, "dtype": "f32",
                   "autotuned": [f"({n['t']},{n['a']},{n['p']}) {n['kernel']}{', lane groups' if n['lane_groups'] else ''}"
                                 for n in tuning3["nodes"]],
                   "kernel_ms_per_step": kms3, "algorithmic_GB_per_step": bytes3 / 1e9,
                   "roofline": dict(hbm_roofline("whole step", bytes3, ms3, float(peaks["hbm_gbs"]), peak_kind),
                                    dominant_kernel=dom3[0], dominant_GBps=dom3[1]["GBps"]),
                   "kernels": tab3}
        ses.close()

    # differentiable form: Chung-Lu 200k (avg degree 20, gamma 2.3), FP32 weights
    # in [0.5, 1.5), tree8, k = 8: forward count and forward + gradient call
    differentiable = None
    if not args.no_batched:
        g4 = si.workload_graph("chunglu200k")
        w4 = si.arc_weights(g4, si.edge_weights(g4, seed=0))
        graph4 = sg.Graph(g4.row_ptr, g4.col_idx, w4)
        plan4 = sg.Plan(si.TREE8.parent, 0, 8)
        col4 = torch.from_numpy(si.colouring(g4.n, 8, rank)).cuda()
        grad4 = torch.empty(g4.nnz, dtype=torch.float64, device="cuda")
        tot4 = torch.empty((1, 1), dtype=torch.float64, device="cuda")
        reps4 = max(3, args.steps // 2)

        def fwd4():
            sg.sg2v_count_batched(graph4.handle, [plan4.handle], col4, 1, sg.SG2V_FP32, None, tot4, None, stream)

        def bwd4(flag):
            return lambda: sg.sg2v_count_backward(graph4.handle, plan4.handle, col4, sg.SG2V_FP32, grad4, None, stream,
                                                  flags=flag)

        def profiled(fn, reps):
            sg.sg2v_profile_reset()
            sg.sg2v_profile_enable(True)
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            sg.sg2v_profile_enable(False)
            return records_block(sg.sg2v_profile_read(), reps, 1)

        ms_f = time_steps(torch, fwd4, reps4, args.warmup, stream, dist)
        # the same forward through an autotuned session (its warm-up run tunes
        # the split schedule and forms; the timed runs replay a CUDA graph)
        ses4 = sg.Session(graph4, [plan4], 1, "fp32", autotune=True)
        col4b = col4.view(1, -1)
        ms_fs = time_steps(torch, lambda: ses4.run(col4b, tot4, None, None, stream), reps4, args.warmup, stream, dist)
        chunk4 = ses4.tuning()["chunk"]
        ses4.close()
        ms_b = time_steps(torch, bwd4(sg.SG2V_BACKWARD_STORE), reps4, args.warmup, stream, dist)
        peak_store = sg.sg2v_last_call_peak_bytes()
        ms_r = time_steps(torch, bwd4(sg.SG2V_BACKWARD_RECOMPUTE), reps4, args.warmup, stream, dist)
        peak_rec = sg.sg2v_last_call_peak_bytes()
        tab_f, bytes_f, _ = profiled(fwd4, 3)
        tab_b, bytes_b, _ = profiled(bwd4(sg.SG2V_BACKWARD_STORE), 3)
        tab_r, bytes_r, _ = profiled(bwd4(sg.SG2V_BACKWARD_RECOMPUTE), 3)
        hbm = float(peaks["hbm_gbs"])
        differentiable = {"workload": "chunglu200k (200k vertices, 2M edges, gamma 2.3, weights [0.5,1.5)), tree8, "
                                      "k=8, one colouring", "forward_ms": ms_f,
                          "forward_session_ms": ms_fs, "forward_session_split_chunk": chunk4,
                          "forward_and_gradient_ms": ms_b,
                          "forward_and_gradient_recompute_ms": ms_r, "peak_workspace_bytes": peak_store,
                          "peak_workspace_bytes_recompute": peak_rec, "dtype": "f32",
                          "roofline_forward": hbm_roofline("forward step", bytes_f, ms_f, hbm, peak_kind),
                          "roofline_forward_session": hbm_roofline("forward step (session replay)", bytes_f, ms_fs,
                                                                   hbm, peak_kind),
                          "roofline_forward_and_gradient": hbm_roofline("forward+gradient step", bytes_b, ms_b, hbm,
                                                                        peak_kind),
                          "roofline_forward_and_gradient_recompute": hbm_roofline("forward+gradient step (recompute)",
                                                                                  bytes_r, ms_r, hbm, peak_kind),
                          "kernels_forward": tab_f, "kernels_forward_and_gradient": tab_b}

    # exact integer tables: the same Chung-Lu graph unweighted, tree8, k = 8,
    # one colouring per call; its table entries reach 2^61, past the 2^53 up
    # to which FP64 tables are exact (the headline's reach 2^94: no fit)
    exact = None
    if not args.no_batched:
        graph4u = sg.Graph(g4.row_ptr, g4.col_idx)

        def one(prec):
            return lambda: sg.sg2v_count_batched(graph4u.handle, [plan4.handle], col4, 1, prec, None, tot4, None,
                                                 stream)

        reps = max(3, args.steps // 2)
        try:
            ms_u = time_steps(torch, one(sg.SG2V_U64), reps, args.warmup, stream, dist)
            exact_total = float(tot4.item())
        except sg.Sg2vError as e:  # a colouring whose counts pass 2^64
            ms_u, exact_total = None, str(e)
        ms_d = time_steps(torch, one(sg.SG2V_FP64), reps, args.warmup, stream, dist)
        ms_s = time_steps(torch, one(sg.SG2V_FP32), reps, args.warmup, stream, dist)
        # the headline workload (entries up to 2^94) in 128-bit integers, beside its plain FP64 form
        ms_h = time_steps(torch, lambda: sg.sg2v_count_batched(graph.handle, [plan.handle], d_cols[0:1], 1,
                                                               sg.SG2V_U128, None, tot64, None, stream),
                          max(3, args.steps // 2), args.warmup, stream, dist)
        exact = {"workload": "chunglu200k unweighted (200k vertices, 2M edges, gamma 2.3), tree8, k=8, one "
                             "colouring per call; table entries up to 2^61", "u64_ms": ms_u, "fp64_ms": ms_d,
                 "fp32_ms": ms_s, "u64_total": exact_total, "dtype": "u64 (exact), f64, f32",
                 "headline_u128": {"workload": WORKLOAD + ", one colouring per call (entries up to 2^94)",
                                   "ms_per_colouring": ms_h, "fp64_ms_per_colouring": ms64, "dtype": "u128 (exact)"}}
        del graph4u

    # large form: R-MAT scale 20 with 5e7 edges, tree15, k = 15, 8 colourings
    # per call.  Counts reach about 2^155, beyond FP32's range, so the tables
    # carry per-row exponents (plain FP32 would overflow and be rerun).
    large = None
    if not args.no_large:
        g5 = si.workload_graph("rmat20_50m")
        graph5 = sg.Graph(g5.row_ptr, g5.col_idx)
        plan5 = sg.Plan(si.TREE15.parent, 0, 15)
        B5 = 8
        cols5 = torch.from_numpy(rank_colourings(g5.n, 15, B5, rank, seed=0)).cuda()
        tot5 = torch.empty((1, B5), dtype=torch.float64, device="cuda")
        def step5():
            sg.sg2v_count_batched(graph5.handle, [plan5.handle], cols5, B5, sg.SG2V_FP32_SCALED, None, tot5, None,
                                  stream)

        ms5 = time_steps(torch, step5, 2, 1, stream, dist)
        sg.sg2v_profile_reset()
        sg.sg2v_profile_enable(True)
        step5()
        torch.cuda.synchronize()
        sg.sg2v_profile_enable(False)
        tab5, bytes5, _ = records_block(sg.sg2v_profile_read(), 1, 1)
        from math import comb

        # the deferred eMA of the (10,5,5) node: 2 FLOP per product, C(14,9) sets x C(9,4) splits per row
        ema5 = [(k, v) for k, v in tab5.items() if k.startswith("ema t=10 a=5 p=5")]
        ema_roof = None
        if ema5:
            k5, v5 = ema5[0]
            flops = 2.0 * comb(14, 9) * comb(9, 4) * g5.n * B5 / v5["launches_per_step"]
            achieved = flops / (v5["ms_per_launch"] * 1e-3) / 1e12
            alu = fp32_alu_peak_flops(peaks) / 1e12
            ema_roof = {"kernel": k5, "bound": "alu", "achieved": achieved, "peak": alu, "unit": "TFLOP/s",
                        "frac": achieved / alu, "peak_kind": "derived: 148 SMs x 128 FP32 lanes x 2 x max SM clock"}
        large = {"workload": "rmat20_50m (R-MAT scale 20, 5e7 edges), tree15, k=15, 8 colourings per call",
                 "ms_per_call": ms5, "s_per_colouring": ms5 * 1e-3 / B5, "dtype": "f32 with per-row exponents",
                 "max_total": float(tot5.max().item()), "steps": 2, "warmup": 1,
                 "roofline": hbm_roofline("whole step", bytes5, ms5, float(peaks["hbm_gbs"]), peak_kind),
                 "roofline_deferred_ema": ema_roof, "kernels": tab5}
        del graph5, g5

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    total_colourings = B * world
    value = ms32 * 1e-3 / total_colourings
    fp64_s = ms64 * 1e-3 / world
    node_recs = [r for r in records if r["name"].startswith("node")]
    dom = max(node_recs, key=lambda r: r["total_ms"])
    dom_ms = dom["total_ms"] / dom["launches"]
    achieved = dom["bytes_per_launch"] / (dom_ms * 1e-3) / 1e9
    step_bytes = sum(r["bytes_per_launch"] * r["launches"] for r in records) / args.steps
    peak = float(peaks["hbm_gbs"])
    traffic = traffic_record().get(dom["name"])
    kernel_table = {r["name"]: {"launches_per_step": r["launches"] / args.steps,
                                "ms_per_launch": round(r["total_ms"] / r["launches"], 4),
                                "algorithmic_GB_per_launch": round(r["bytes_per_launch"] / 1e9, 4),
                                "GBps": round(r["bytes_per_launch"] / (r["total_ms"] / r["launches"]) / 1e6, 1)}
                    for r in records}
    cpu = None
    if not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, dt, gs = oracle_seconds_per_colouring(args.cpu_baseline_scale, threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": (f"exact oracle DP (128-bit integers) on R-MAT scale {args.cpu_baseline_scale} "
                          f"({gs.m} edges, same parameters and average degree), 1 colouring of tree10, "
                          f"{dt:.2f} s measured, scaled x{FULL_EDGES // gs.m} to 2^24 edges")}
    clk = clocks.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": "rmat scale 20 (.57,.19,.19,.05), 2^24 undirected edges, ids permuted",
                   "template": list(TEMPLATE.parent), "num_colours": K_COLOURS, "batch_colourings_per_step": B,
                   "plan": f"cut {PLAN_CUT} (avg degree 32): nodes {[n[:3] for n in plan.nodes()]}",
                   "parallelism": f"replicas over colourings x{world}",
                   "l2": "inputs larger than L2: count tables of 1-8 GB per step"},
        "fp64_plain": {"s_per_colouring": fp64_s, "ms_per_step": ms64, "dtype": "f64",
                       "roofline": {"kernel": "node kernels of one colouring", "bound": "fp64",
                                    "achieved": ops64 / (ms_nodes64 * 1e-3) / 1e12,
                                    "peak": fp64_ops_peak / 1e12, "unit": "TOP/s (FP64 add or FMA)",
                                    "frac": ops64 / (ms_nodes64 * 1e-3) / fp64_ops_peak,
                                    "peak_kind": "measured: cuBLAS DGEMM 4096^3 on this GPU, FMA = 1 op",
                                    "ops_per_colouring": ops64, "node_ms_per_colouring": ms_nodes64},
                       "kernels": records_block(rec64, steps64, 1)[0]},
        "fp32_batched": {"s_per_colouring": value, "ms_per_step": ms32, "B": B},
        "fp32_batched_session": session_block,
        "speedup_fp32_batched_vs_fp64_plain": fp64_s / value,
        "hbm": {"algorithmic_GB_per_step": step_bytes / 1e9, "GBps_step": step_bytes / (ms32 * 1e-3) / 1e9,
                "frac_of_measured_peak": step_bytes / (ms32 * 1e-3) / 1e9 / peak,
                "frac_of_nameplate_8TBps": step_bytes / (ms32 * 1e-3) / 1e9 / 8000.0},
        "roofline": {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "gather": gather_rate(dom, g, K_COLOURS, dom_ms)},
        "kernels": kernel_table,
        "batched_3_templates": batched,
        "differentiable": differentiable,
        "exact_integer": exact,
        "large_form": large,
        "cpu_baseline": cpu,
        "e2e": {"value": ms_e2e * 1e-3 / total_colourings, "unit": UNIT, "h2d_bytes_per_step": int(B * g.n),
                "d2h_bytes_per_step": int(2 * B * 8), "outputs": "totals and estimates"},
        "e2e_per_vertex": {"value": ms_e2e_pv * 1e-3 / total_colourings, "unit": UNIT,
                           "h2d_bytes_per_step": int(B * g.n), "d2h_bytes_per_step": int(B * g.n * 8 + 2 * B * 8),
                           "outputs": "per-vertex counts, totals and estimates"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
