"""Alg. 1's outer loop (host logic, CPU): averaging, the stopping rule,
checkpoint/resume and replicas over colourings on two gloo ranks.

The counter here is the exact oracle (finalCount of each colouring as an
exact rational, rounded once), standing in for the GPU session so that the
loop logic is tested without a GPU."""
import json
import math
import os
import socket

import numpy as np
import pytest

import oracle
import sg2v_inputs as si
from paper_2009_11665_b300 import estimator as E

K = 4
PATH4 = (-1, 0, 1, 2)


def _graph():
    return si.erdos_renyi(40, 110, seed=3)


def _counter(g, parent, calls=None, fail_after=None):
    alpha = oracle.automorphisms(parent)
    k = len(parent)

    def count_wave(cols):
        if calls is not None:
            calls.append(cols.shape[0])
            if fail_after is not None and len(calls) > fail_after:
                raise RuntimeError("injected failure")
        out = []
        for c in cols:
            tot = oracle.count(g.row_ptr, g.col_idx, parent, 0, c, per_vertex=False).total
            out.append(float(oracle.estimate(tot, k, alpha)))
        return np.array([out])

    return count_wave


def _colouring(n, seed=11):
    return lambda i: si.colouring(n, K, seed, i)


def test_paper_bound_formula():
    assert E.paper_iterations(4, 0.1, 0.05) == math.ceil(math.exp(4) * math.log(20) / 0.01)
    assert E.paper_iterations(7, 0.5, 0.01, constant=0.5) == math.ceil(0.5 * math.exp(7) * math.log(100) / 0.25)
    with pytest.raises(ValueError):
        E.paper_iterations(4, 0.1, 1.0)


def test_indices_partition_the_colourings():
    seen = []
    for wave_no in range(3):
        for r in range(4):
            seen.extend(E.colouring_indices(r, 4, 5, wave_no).tolist())
    assert sorted(seen) == list(range(60))


def test_average_and_stopping_rule():
    g = _graph()
    est = E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n), K, eps=0.05, delta=0.05, wave=8,
                                  min_colourings=16, max_colourings=400)
    res = est.run()
    # the estimate is the plain average of the finalCounts of the colourings counted
    vals = _counter(g, PATH4)(np.stack([_colouring(g.n)(i) for i in range(res.colourings)]))[0]
    assert res.estimate[0] == pytest.approx(vals.mean(), rel=1e-12)
    assert res.stderr[0] == pytest.approx(vals.std(ddof=1) / math.sqrt(len(vals)), rel=1e-9)
    assert res.colourings % 8 == 0 and res.colourings >= 16
    if res.converged:
        assert res.half_width[0] <= 0.05 * res.estimate[0]
        # one wave earlier it had not converged (or was below the minimum)
        prev = vals[:res.colourings - 8]
        hw_prev = E.NormalDist().inv_cdf(0.95) * prev.std(ddof=1) / math.sqrt(len(prev))
        assert len(prev) < 16 or hw_prev > 0.05 * prev.mean()
    else:
        assert res.colourings == 400


def test_estimate_is_unbiased():
    """Colourful counts scaled by 1/(P alpha) estimate emb(T, G): the mean of
    many colourings lies within a few standard errors of the exact count of
    copies of T (brute force over injective maps)."""
    g = _graph()
    emb = oracle.brute(g.row_ptr, g.col_idx, PATH4, 0, injective_only=True).total / oracle.automorphisms(PATH4)
    est = E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n, seed=5), K, eps=1e-9, delta=0.05, wave=50,
                                  max_colourings=1500)
    res = est.run()
    assert not res.converged and res.colourings == 1500
    assert abs(res.estimate[0] - emb) <= 4.5 * res.stderr[0]


def test_checkpoint_resume_matches_uninterrupted(tmp_path):
    g = _graph()
    ck = str(tmp_path / "state.json")
    calls = []
    first = E.ColourCodingEstimator(_counter(g, PATH4, calls, fail_after=3), _colouring(g.n), K, eps=1e-9,
                                    delta=0.1, wave=6, max_colourings=60, checkpoint=ck)
    with pytest.raises(RuntimeError):
        first.run()
    assert json.load(open(ck))["waves"] == 3
    resumed = E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n), K, eps=1e-9, delta=0.1, wave=6,
                                      max_colourings=60, checkpoint=ck).run()
    straight = E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n), K, eps=1e-9, delta=0.1, wave=6,
                                       max_colourings=60).run()
    assert resumed.colourings == straight.colourings == 60
    assert resumed.estimate[0] == pytest.approx(straight.estimate[0], rel=1e-14)
    with pytest.raises(ValueError):
        E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n), K, eps=1e-9, delta=0.1, wave=5,
                                checkpoint=ck).run()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = _graph()
        est = E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n), K, eps=0.04, delta=0.05, wave=5,
                                      min_colourings=20, max_colourings=300, group=dist.group.WORLD)
        res = est.run()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"estimate": res.estimate.tolist(), "colourings": res.colourings,
                       "converged": res.converged}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(tmp_path):
    """Replicas over colourings: two ranks with waves of 5 count the same
    colourings as one process with waves of 10, sum their statistics after
    every wave and stop together with the same estimate."""
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0 == r1
    g = _graph()
    one = E.ColourCodingEstimator(_counter(g, PATH4), _colouring(g.n), K, eps=0.04, delta=0.05, wave=10,
                                  min_colourings=20, max_colourings=300).run()
    assert r0["colourings"] == one.colourings
    assert r0["converged"] == one.converged
    assert r0["estimate"][0] == pytest.approx(one.estimate[0], rel=1e-12)
