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
    one("rmat20_16m_tree10_k10", "rmat20_16m", si.TREE10, 10, colouring_seed=0)
