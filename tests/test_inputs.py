"""The seeded workloads have the shapes the benchmark configurations state
(tree sizes follow from the branching structure alone)."""
import json
import os

import numpy as np

from paper_2505_12078_b300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _nodes(b, k, N):
    # b-way branching at stages 0..k-1, then one child per scenario down to stage N
    return sum(b ** t for t in range(k + 1)) + (N - k) * b ** k


def test_batch_draw_shapes():
    specs = synth.batch_specs(512, seed=4)
    assert len(specs) == 512
    for s in specs:
        assert 4 <= s["nx"] <= 64 and s["nu"] == max(1, s["nx"] // 2)
        assert 5 <= s["N"] <= 20 and 2 <= s["b"] <= 4 and 1 <= s["k"] <= min(4, s["N"])
        assert 0.2 <= s["avar"] <= 1.0
    assert sum(_nodes(s["b"], s["k"], s["N"]) for s in specs) == 215384
    assert synth.batch_specs(512, seed=4) == specs   # deterministic


def test_batch_problem_matches_its_spec():
    s = synth.batch_specs(8, seed=4)[3]
    p = synth.batch_problem(s, 3)
    assert p.nx == s["nx"] and p.nu == s["nu"] and p.N == s["N"]
    assert len(p.anc) == _nodes(s["b"], s["k"], s["N"])
    # A = I + 0.1 G with G at spectral radius 1.05
    G = (p.A[0] - np.eye(p.nx)) / 0.1
    assert abs(np.max(np.abs(np.linalg.eigvals(G))) - 1.05) < 1e-10
    # children probabilities of every node sum to one
    kids = {}
    for c in range(1, len(p.anc)):
        kids.setdefault(int(p.anc[c]), []).append(float(p.prob[c]))
    assert all(abs(sum(v) - 1.0) < 1e-12 for v in kids.values())


def test_benchmark_workload_sizes():
    sizes = json.load(open(os.path.join(HERE, "golden", "sizes.json")))
    p = synth.large_raocp()
    assert len(p.anc) == _nodes(3, 4, 15) == 1012
    assert (p.nx, p.nu) == (50, 25)
    assert sizes["large_raocp"]["n"] == len(p.anc)
