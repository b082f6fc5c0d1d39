"""Writes the stored expected values used by the full-size GPU parity tests.

Every value here comes from the exact CPU oracle (oracle/), never from the
CUDA path.  The inputs are regenerated from their seeds by sg2v_inputs; the
file also records a fingerprint of the graph so that a test can confirm it
rebuilt the same input before comparing.

    python tests/golden/make_golden.py            # all workloads
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import sg2v_inputs as si  # noqa: E402

SAMPLES = 4096


def fingerprint(g) -> str:
    h = hashlib.sha256()
    h.update(g.row_ptr.tobytes())
    h.update(g.col_idx.tobytes())
    return h.hexdigest()


def large_form(scale: int, colourings: int = 8, samples: int = 512):
    """The large form's scaled sibling: R-MAT scale `scale` with the full
    workload's parameters and edge/vertex ratio (5e7 edges at scale 20),
    tree15, k = 15, colourings 0..7 of seed 0: exact totals and sampled
    per-vertex counts."""
    m = int(round(50_000_000 / (1 << (20 - scale))))
    g = si.rmat(scale, m, seed=0)
    idx = sorted(set(int(i) for i in si.sample_indices(min(samples, g.n), g.n, seed=2)) |
                 set(int(i) for i in g.degrees().argsort()[-16:]))
    out = {"workload": f"rmat{scale}_large_sibling_tree15_k15", "graph": f"rmat scale {scale}, m={m}",
           "scale": scale, "m": m, "n": g.n, "graph_sha256": fingerprint(g), "template": list(si.TREE15.parent),
           "root": 0, "num_colours": 15, "colouring_seed": 0, "sample_vertices": idx, "colourings": [],
           "source": "oracle.count (exact decoupled DP, 384-bit), tests/golden/make_golden.py"}
    for b in range(colourings):
        col = si.colouring(g.n, 15, 0, b)
        t0 = time.time()
        r = oracle.count(g.row_ptr, g.col_idx, si.TREE15.parent, 0, col, 15, min_limbs=6)
        out["colourings"].append({"index": b, "total": str(r.total), "max_table_bits": r.max_bits,
                                  "sample_counts": [str(r.per_vertex[i]) for i in idx],
                                  "oracle_seconds": round(time.time() - t0, 1)})
        print(f"scale {scale} colouring {b}: bits {r.max_bits} ({time.time() - t0:.0f}s)", flush=True)
        with open(os.path.join(HERE, f"rmat{scale}_large_sibling_tree15_k15.json"), "w") as f:
            json.dump(out, f, indent=1)


def one(name, graph_name, template, kc, colouring_seed, colouring_index=0):
    g = si.workload_graph(graph_name)
    col = si.colouring(g.n, kc, colouring_seed, colouring_index)
    t0 = time.time()
    r = oracle.count(g.row_ptr, g.col_idx, template.parent, template.root, col, kc)
    dt = time.time() - t0
    idx = si.sample_indices(SAMPLES, g.n, seed=1)
    # include the vertices with the largest counts and degrees too
    deg = g.degrees()
    extra = sorted(set(int(i) for i in deg.argsort()[-32:]) |
                   set(int(i) for i in sorted(range(g.n), key=lambda v: r.per_vertex[v])[-32:]))
    idx = sorted(set(int(i) for i in idx) | set(extra))
    out = {
        "workload": name,
        "graph": graph_name,
        "n": g.n,
        "m": g.m,
        "graph_sha256": fingerprint(g),
        "template": list(template.parent),
        "root": template.root,
        "num_colours": kc,
        "colouring_seed": colouring_seed,
        "colouring_index": colouring_index,
        "total": str(r.total),
        "max_table_bits": r.max_bits,
        "sample_vertices": idx,
        "sample_counts": [str(r.per_vertex[i]) for i in idx],
        "oracle_seconds": round(dt, 2),
        "source": "oracle.count (exact decoupled DP), tests/golden/make_golden.py",
    }
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"{path}: total={r.total} bits={r.max_bits} ({dt:.1f}s)")


def bench_step(colourings: int = 4):
    """The benchmark's timed step: rmat20_16m, tree10, k = 10, colourings
    0..3 of seed 0 (the first rank's batch): exact totals."""
    g = si.workload_graph("rmat20_16m")
    cols = si.colourings(g.n, 10, colourings, seed=0)
    out = {"workload": "rmat20_16m_tree10_k10_bench_step", "graph": "rmat20_16m", "n": g.n, "m": g.m,
           "graph_sha256": fingerprint(g), "template": list(si.TREE10.parent), "root": 0, "num_colours": 10,
           "colouring_seed": 0, "colourings": [],
           "source": "oracle.count (exact decoupled DP, totals only), tests/golden/make_golden.py"}
    for b in range(colourings):
        t0 = time.time()
        r = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, cols[b], per_vertex=False)
        out["colourings"].append({"index": b, "total": str(r.total), "max_table_bits": r.max_bits,
                                  "oracle_seconds": round(time.time() - t0, 1)})
        print(f"bench step colouring {b}: {r.total} ({time.time() - t0:.0f}s)", flush=True)
        with open(os.path.join(HERE, "rmat20_16m_tree10_k10_bench_step.json"), "w") as f:
            json.dump(out, f, indent=1)


def batched_form(colourings: int = 2):
    """The batched form's workload: rmat18_d16, path7 / star7 / tree7, k = 7,
    colourings 0..1 of seed 1 (the first two of the benchmark's 64): exact
    totals and sampled per-vertex counts."""
    g = si.workload_graph("rmat18_d16")
    cols = si.colourings(g.n, 7, colourings, seed=1)
    deg = g.degrees()
    idx = sorted(set(int(i) for i in si.sample_indices(SAMPLES, g.n, seed=3)) |
                 set(int(i) for i in deg.argsort()[-32:]))
    out = {"workload": "rmat18_d16_k7_batched", "graph": "rmat18_d16", "n": g.n, "m": g.m,
           "graph_sha256": fingerprint(g), "num_colours": 7, "colouring_seed": 1, "sample_vertices": idx,
           "templates": [], "source": "oracle.count (exact decoupled DP), tests/golden/make_golden.py"}
    for t in (si.PATH7, si.STAR7, si.TREE7):
        entry = {"name": t.name, "template": list(t.parent), "root": t.root, "colourings": []}
        for b in range(colourings):
            t0 = time.time()
            r = oracle.count(g.row_ptr, g.col_idx, t.parent, t.root, cols[b])
            entry["colourings"].append({"index": b, "total": str(r.total), "max_table_bits": r.max_bits,
                                        "sample_counts": [str(r.per_vertex[i]) for i in idx]})
            print(f"batched {t.name} colouring {b}: {r.total} ({time.time() - t0:.0f}s)", flush=True)
        out["templates"].append(entry)
    with open(os.path.join(HERE, "rmat18_d16_k7_batched.json"), "w") as f:
        json.dump(out, f, indent=1)


def frac(x) -> str:
    return f"{x.numerator}/{x.denominator}"


def differentiable_form(edges: int = 64):
    """The differentiable form's workload: chunglu200k with FP32 weights of
    seed 0, tree8, k = 8, colouring 0 of seed 0: the exact weighted total,
    sampled exact per-vertex values and, for 64 sampled undirected edges,
    the exact gradient (F - F(w_e = 0)) / w_e (F is affine in each weight)."""
    from fractions import Fraction

    g = si.workload_graph("chunglu200k")
    w = si.arc_weights(g, si.edge_weights(g, seed=0))
    col = si.colouring(g.n, 8, 0)
    ids = si.arc_edge_ids(g)
    t0 = time.time()
    base = oracle.count(g.row_ptr, g.col_idx, si.TREE8.parent, 0, col, weights=w)
    F = base.total_value()
    pv = base.per_vertex_values()
    deg = g.degrees()
    idx = sorted(set(int(i) for i in si.sample_indices(SAMPLES, g.n, seed=4)) |
                 set(int(i) for i in deg.argsort()[-32:]))
    out = {"workload": "chunglu200k_tree8_k8_weighted", "graph": "chunglu200k", "n": g.n, "m": g.m,
           "graph_sha256": fingerprint(g), "weights_seed": 0, "template": list(si.TREE8.parent), "root": 0,
           "num_colours": 8, "colouring_seed": 0, "total": frac(F), "sample_vertices": idx,
           "sample_values": [frac(pv[i]) for i in idx], "edges": [], "gradients": [],
           "source": "oracle.count (exact dyadic weighted DP), tests/golden/make_golden.py"}
    print(f"differentiable: F = {float(F):.6e} ({time.time() - t0:.0f}s)", flush=True)
    sample = [int(e) for e in si.sample_indices(edges, g.m, seed=5)]
    for e in sample:
        w0 = w.copy()
        w0[ids == e] = 0.0
        t0 = time.time()
        F0 = oracle.count(g.row_ptr, g.col_idx, si.TREE8.parent, 0, col, weights=w0, per_vertex=False).total_value()
        we = Fraction(float(w[ids == e][0]))
        out["edges"].append(e)
        out["gradients"].append(frac((F - F0) / we))
        print(f"differentiable edge {e}: {float((F - F0) / we):.6e} ({time.time() - t0:.0f}s)", flush=True)
        with open(os.path.join(HERE, "chunglu200k_tree8_k8_weighted.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("all", "tree10"):
        one("rmat20_16m_tree10_k10", "rmat20_16m", si.TREE10, 10, colouring_seed=0)
    if what in ("all", "large12"):
        large_form(12)
    if what in ("all", "large16"):
        large_form(16)
    if what in ("all", "bench"):
        bench_step()
    if what in ("all", "batched"):
        batched_form()
    if what in ("all", "differentiable"):
        differentiable_form()
