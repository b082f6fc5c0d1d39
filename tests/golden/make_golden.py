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


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("all", "tree10"):
        one("rmat20_16m_tree10_k10", "rmat20_16m", si.TREE10, 10, colouring_seed=0)
    if what in ("all", "large12"):
        large_form(12)
    if what in ("all", "large16"):
        large_form(16)
