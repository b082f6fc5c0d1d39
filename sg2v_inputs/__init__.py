"""Seeded synthetic inputs for colour-coding tree counting.

Shared by the tests, the benchmark, the smoke check and the oracle harness.
It draws graphs, colourings and edge weights and nothing else: no part of the
counting method's arithmetic lives here.

Every random number is a keyed hash: ``u64(seed, stream, i)`` is the SplitMix64
output function applied to ``base(seed, stream) + i * GOLDEN`` (GOLDEN being
SplitMix64's increment), so any element can be regenerated on its own and the
draws do not depend on batch sizes.

Graphs are simple and undirected and come back as symmetric CSR
(``row_ptr`` int64[n+1], ``col_idx`` int32[nnz], columns sorted within rows).
"Average degree d" means ``m = n*d/2`` unique undirected edges.  Candidate
edges are drawn in index order; self-loops are dropped and the first
occurrence of each pair is kept until ``m`` edges are accepted.
"""
from __future__ import annotations

import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor
from typing import Sequence

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# stream identifiers (fixed so that every consumer draws the same numbers)
STREAM_ER = 1
STREAM_RMAT = 2
STREAM_PERM = 3
STREAM_CHUNG_LU = 4
STREAM_WEIGHTS = 5
STREAM_SAMPLE = 6
STREAM_COLOURS = 1000  # + colouring index


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def _mix_int(z: int) -> int:
    z &= MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & MASK64
    z ^= z >> 31
    return z


def _base(seed: int, stream: int) -> int:
    return _mix_int(_mix_int(seed * GOLDEN + 0x632BE59BD9B4E019) ^ (stream * 0xD1B54A32D192ED03 & MASK64))


def u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Keyed 64-bit hashes for an array of (non-negative) indices."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(_base(seed, stream)) + idx * np.uint64(GOLDEN) + np.uint64(GOLDEN)
    return _mix(z)


def uniform53(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ------------------------------------------------------------------ graphs

@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col_idx: np.ndarray  # int32 [nnz]
    edges: np.ndarray    # int64 [m, 2], u < v, acceptance order
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _chunked(fn, start: int, count: int, chunk: int = 1 << 20):
    """fn(start, count) -> tuple of arrays, evaluated on chunks in threads
    (numpy releases the GIL) and concatenated; results do not depend on the
    chunking because every draw is keyed by its index."""
    pieces = [(s, min(chunk, start + count - s)) for s in range(start, start + count, chunk)]
    if len(pieces) <= 1:
        return fn(start, count)
    with ThreadPoolExecutor(max_workers=min(len(pieces), os.cpu_count() or 1)) as ex:
        outs = list(ex.map(lambda sc: fn(*sc), pieces))
    return tuple(np.concatenate([o[i] for o in outs]) for i in range(len(outs[0])))


def edges_to_csr(n: int, edges: np.ndarray):
    """Symmetric CSR (both arcs of every undirected edge, rows sorted)."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    src = np.concatenate([edges[:, 0], edges[:, 1]]).astype(np.uint64)
    dst = np.concatenate([edges[:, 1], edges[:, 0]]).astype(np.uint64)
    key = np.sort((src << np.uint64(32)) | dst)
    src = (key >> np.uint64(32)).astype(np.int64)
    dst = (key & np.uint64(0xFFFFFFFF)).astype(np.int32)
    counts = np.bincount(src, minlength=n) if n > 0 else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, dst


def arc_edge_ids(g: Graph) -> np.ndarray:
    """For every CSR arc, the index (in g.edges) of its undirected edge."""
    e = g.edges
    m = e.shape[0]
    src = np.concatenate([e[:, 0], e[:, 1]]).astype(np.uint64)
    dst = np.concatenate([e[:, 1], e[:, 0]]).astype(np.uint64)
    ids = np.concatenate([np.arange(m), np.arange(m)])
    order = np.argsort((src << np.uint64(32)) | dst)
    return ids[order].astype(np.int64)


def _accept_unique(n: int, m: int, draw, batch0: int) -> np.ndarray:
    """Draws candidate pairs batch by batch (draw(start, count) -> (u, v)),
    keeps first occurrences of unique non-loop pairs until m are accepted."""
    accepted_keys = np.zeros(0, dtype=np.uint64)
    out = []
    have = 0
    start = 0
    batch = max(batch0, 1024)
    while have < m:
        u, v = draw(start, batch)
        start += batch
        u = u.astype(np.int64)
        v = v.astype(np.int64)
        keep = u != v
        lo = np.minimum(u, v)[keep]
        hi = np.maximum(u, v)[keep]
        keys = (lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64)
        _, first = np.unique(keys, return_index=True)
        first.sort()
        keys = keys[first]
        lo = lo[first]
        hi = hi[first]
        if accepted_keys.size:
            pos = np.searchsorted(accepted_keys, keys)
            pos = np.minimum(pos, accepted_keys.size - 1)
            new = accepted_keys[pos] != keys
            keys, lo, hi = keys[new], lo[new], hi[new]
        take = min(m - have, keys.size)
        keys, lo, hi = keys[:take], lo[:take], hi[:take]
        out.append(np.stack([lo, hi], axis=1))
        accepted_keys = np.sort(np.concatenate([accepted_keys, keys]))
        have += take
        if take == 0 and batch > 64 * max(m, 1):
            raise ValueError("cannot draw enough unique edges")
        batch = int(max(1024, (m - have) * 1.3))
    return np.concatenate(out, axis=0) if out else np.zeros((0, 2), np.int64)


def erdos_renyi(n: int, m: int, seed: int = 0) -> Graph:
    """G(n, m): m distinct uniform vertex pairs."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")

    def draw(start, count):
        idx = np.arange(start, start + count, dtype=np.uint64)
        h = u64(seed, STREAM_ER, idx)
        u = ((h >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
        v = ((h & np.uint64(0xFFFFFFFF)) * np.uint64(n)) >> np.uint64(32)
        return u, v

    e = _accept_unique(n, m, lambda s0, c0: _chunked(draw, s0, c0), int(m * 1.1) + 16)
    rp, ci = edges_to_csr(n, e)
    return Graph(n, rp, ci, e, f"er_n{n}_m{m}_s{seed}")


def rmat(scale: int, m: int, a=0.57, b=0.19, c=0.19, d=0.05, seed: int = 0, permute: bool = True) -> Graph:
    """R-MAT (recursive quadrant choice per level, no noise); vertex ids are
    randomly permuted when `permute` (Graph500 practice)."""
    n = 1 << scale
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT probabilities must sum to 1")
    ta = np.uint64(int(a * 2**32))
    tb = np.uint64(int((a + b) * 2**32))
    tc = np.uint64(int((a + b + c) * 2**32))
    halves = (scale + 1) // 2
    perm = None
    if permute:
        perm = np.argsort(u64(seed, STREAM_PERM, np.arange(n, dtype=np.uint64)), kind="stable").astype(np.int64)
        perm = perm.astype(np.uint64)

    def draw(start, count):
        e = np.arange(start, start + count, dtype=np.uint64)
        u = np.zeros(count, dtype=np.uint64)
        v = np.zeros(count, dtype=np.uint64)
        lvl = 0
        for h in range(halves):
            hv = u64(seed, STREAM_RMAT, e * np.uint64(halves) + np.uint64(h))
            for part in (hv >> np.uint64(32), hv & np.uint64(0xFFFFFFFF)):
                if lvl == scale:
                    break
                rowbit = (part >= tb).astype(np.uint64)
                colbit = (((part >= ta) & (part < tb)) | (part >= tc)).astype(np.uint64)
                u = (u << np.uint64(1)) | rowbit
                v = (v << np.uint64(1)) | colbit
                lvl += 1
        if perm is not None:
            return perm[u.astype(np.int64)], perm[v.astype(np.int64)]
        return u, v

    e = _accept_unique(n, m, lambda s0, c0: _chunked(draw, s0, c0), int(m * 1.3) + 16)
    rp, ci = edges_to_csr(n, e)
    return Graph(n, rp, ci, e, f"rmat_s{scale}_m{m}_s{seed}")


def chung_lu(n: int, m: int, gamma: float = 2.3, seed: int = 0) -> Graph:
    """Chung-Lu power law: endpoint i drawn with probability proportional to
    (i+1)^(-1/(gamma-1)) (ball dropping) until m unique edges exist."""
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def draw(start, count):
        idx = np.arange(2 * start, 2 * (start + count), dtype=np.uint64)
        uu = uniform53(seed, STREAM_CHUNG_LU, idx)
        ends = np.minimum(np.searchsorted(cdf, uu, side="right"), n - 1)
        return ends[0::2], ends[1::2]

    e = _accept_unique(n, m, lambda s0, c0: _chunked(draw, s0, c0), int(m * 1.5) + 16)
    rp, ci = edges_to_csr(n, e)
    return Graph(n, rp, ci, e, f"chunglu_n{n}_m{m}_g{gamma}_s{seed}")


def from_edges(n: int, edges: Sequence[Sequence[int]], name: str = "") -> Graph:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if e.size:
        lo = np.minimum(e[:, 0], e[:, 1])
        hi = np.maximum(e[:, 0], e[:, 1])
        e = np.stack([lo, hi], axis=1)
    rp, ci = edges_to_csr(n, e)
    return Graph(n, rp, ci, e, name)


def path_graph(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def complete_graph(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def tree_as_graph(parent: Sequence[int]) -> Graph:
    return from_edges(len(parent), [(i, p) for i, p in enumerate(parent) if p >= 0], "template")


def random_small_graph(n: int, p_num: int, p_den: int, seed: int) -> Graph:
    """Each of the n(n-1)/2 pairs is an edge with probability p_num/p_den."""
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    if not pairs:
        return from_edges(n, [], f"small_n{n}")
    h = u64(seed, STREAM_ER, np.arange(len(pairs), dtype=np.uint64))
    keep = (h % np.uint64(p_den)) < np.uint64(p_num)
    return from_edges(n, [pr for pr, k in zip(pairs, keep) if k], f"small_n{n}_s{seed}")


# --------------------------------------------------- colourings and weights

def colouring(n: int, num_colours: int, seed: int = 0, index: int = 0) -> np.ndarray:
    """col[v] = floor(num_colours * u), u uniform from key (seed, index, v)."""
    u = uniform53(seed, STREAM_COLOURS + index, np.arange(n, dtype=np.uint64))
    return np.minimum((u * num_colours).astype(np.int64), num_colours - 1).astype(np.int8)


def colourings(n: int, num_colours: int, batch: int, seed: int = 0) -> np.ndarray:
    """[batch, n] int8: colouring b is colouring(n, num_colours, seed, b)."""
    out = np.empty((batch, n), dtype=np.int8)
    for b in range(batch):
        out[b] = colouring(n, num_colours, seed, b)
    return out


def edge_weights(g: Graph, seed: int = 0, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """One float32 weight per undirected edge, uniform in [lo, hi)."""
    u = uniform53(seed, STREAM_WEIGHTS, np.arange(g.m, dtype=np.uint64))
    w = (lo + (hi - lo) * u).astype(np.float32)
    return np.minimum(w, np.float32(np.nextafter(np.float32(hi), np.float32(0))))


def arc_weights(g: Graph, w_edge: np.ndarray) -> np.ndarray:
    """Per-CSR-arc weights (both arcs of an edge carry the edge's weight)."""
    return np.asarray(w_edge, dtype=np.float32)[arc_edge_ids(g)]


def sample_indices(count: int, population: int, seed: int = 0) -> np.ndarray:
    """`count` distinct indices of range(population), seeded."""
    keys = u64(seed, STREAM_SAMPLE, np.arange(population, dtype=np.uint64))
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)


# ------------------------------------------------------- named workloads

@dataclasses.dataclass
class Template:
    parent: tuple
    root: int = 0
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.parent)


PATH5 = Template((-1, 0, 1, 2, 3), 0, "path5")
TREE10 = Template((-1, 0, 1, 1, 0, 4, 5, 5, 2, 6), 0, "tree10")
PATH7 = Template((-1, 0, 1, 2, 3, 4, 5), 0, "path7")
STAR7 = Template((-1, 0, 0, 0, 0, 0, 0), 0, "star7")
TREE7 = Template((-1, 0, 0, 1, 1, 2, 2), 0, "tree7")
TREE8 = Template((-1, 0, 1, 2, 0, 4, 4, 6), 0, "tree8")
TREE15 = Template((-1, 0, 1, 2, 3, 0, 5, 6, 5, 8, 0, 10, 11, 12, 12), 0, "tree15")


def workload_graph(name: str, seed: int = 0) -> Graph:
    """Graphs of the five workloads (and the scaled sibling of the large one)."""
    if name == "er2000":        # 2,000 vertices, average degree 8
        return erdos_renyi(2000, 8000, seed)
    if name == "rmat20_16m":    # R-MAT scale 20, 2^24 undirected edges (avg degree 32)
        return rmat(20, 1 << 24, seed=seed)
    if name == "rmat18_d16":    # R-MAT scale 18, average degree 16
        return rmat(18, (1 << 18) * 8, seed=seed)
    if name == "chunglu200k":   # Chung-Lu 200k vertices, average degree 20, gamma 2.3
        return chung_lu(200_000, 2_000_000, 2.3, seed)
    if name == "rmat20_50m":    # R-MAT scale 20, 5e7 undirected edges
        return rmat(20, 50_000_000, seed=seed)
    if name == "rmat16_50m_sibling":  # scale 16 with the same edge/vertex ratio
        return rmat(16, int(round(50_000_000 / 16)), seed=seed)
    raise KeyError(name)
