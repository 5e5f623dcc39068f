"""Parity at the full sizes of the benchmark workloads, in the launch
configuration that bench.py times: the 1012-node nx=50 problem (whole-CTA
sweeps with the bulk-copy ring) and the ~4096-node tree-shape sweep problems
(b = 2, 4, 8). One evaluation of T and a fixed SPOCK iteration count are
compared with the oracle element by element; the converged FP32 solve of the
large problem, which the oracle cannot run to the end in test time, is
checked through properties that hold at any size (FP64 residual of the FP32
iterate, feasibility, agreement with the FP64 solve on the risk value and
u^0). Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle.spock_oracle import Oracle
from paper_2505_12078_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2505_12078_b300 import build, spock
    build.build()
    spock.load()


def _spock():
    from paper_2505_12078_b300 import spock
    return spock


FULL = {
    "large_1012": synth.large_raocp,
    "sweep_b2": lambda: synth.tree_sweep(2),
    "sweep_b4": lambda: synth.tree_sweep(4),
    "sweep_b8": lambda: synth.tree_sweep(8),
}


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_one_T(name):
    p = FULL[name]()
    o = Oracle(p)
    g = _spock().Problem(p)
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    v = np.random.default_rng(4).standard_normal(o.lay.n_z + o.lay.n_eta)
    ref = o.T(v)
    vt = torch.tensor(v, device="cuda")
    out, _ = g.T(vt)
    assert _relerr(out.cpu().numpy(), ref) < 1e-11
    out32, _ = g.T(vt.float())
    assert _relerr(out32.cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("name", ["large_1012", "sweep_b4"])
def test_full_size_spock_fixed_fp64(name):
    p = FULL[name]()
    o = Oracle(p)
    g = _spock().Problem(p)
    g.set_alpha(o.alpha)
    iters = 10
    ref = o.solve(tol=0.0, max_iters=iters, method="spock")
    res = g.solve(p.x0, _spock().opts(precision=64, tol=0.0, max_iters=iters))
    kinds = [e[1] for e in ref["events"]]
    inf = res["info"]
    assert inf["iters"] == iters and inf["n_T"] == ref["n_T"]
    assert (inf["n_K0"], inf["n_K1"], inf["n_K2"]) == (kinds.count("K0"), kinds.count("K1"), kinds.count("K2"))
    assert _relerr(g.get_iterate(64).cpu().numpy(), ref["v"]) < 1e-10


def test_full_size_converged_fp32_large():
    """The benchmark solve itself: FP32 to ||v - T(v)||_inf <= 1e-4."""
    spock = _spock()
    p = synth.large_raocp()
    g = spock.Problem(p)
    r32 = g.solve(p.x0, spock.opts(precision=32, tol=1e-4, max_iters=200000))
    r64 = g.solve(p.x0, spock.opts(precision=64, tol=1e-4, max_iters=200000))
    assert r32["status"] == 0 and r64["status"] == 0
    assert r32["info"]["res_inf_fp64"] <= 2e-4
    # feasibility of the returned trajectory (box 5 on x, box 2 and ball 3 on u)
    assert np.max(np.abs(r32["x"])) <= 5.0 * (1 + 1e-3)
    assert np.max(np.abs(r32["u"])) <= 2.0 * (1 + 1e-3)
    assert np.max(np.linalg.norm(r32["u"], axis=1)) <= 3.0 * (1 + 1e-3)
    # two approximations of the same optimum, each within the 1e-3 target of it
    assert abs(r32["risk"] - r64["risk"]) <= 2e-3 * max(1.0, abs(r64["risk"]))
    assert np.max(np.abs(r32["u"][0] - r64["u"][0])) <= 2e-3 * max(1.0, np.max(np.abs(r64["u"][0])))


def test_full_size_converged_against_oracle_golden():
    """The benchmark solve against the oracle's solves of the same problem
    (tests/golden/large_raocp_converged.npz, written by
    tests/golden/make_converged.py from the oracle alone): its solve to
    ||v - T(v)||_inf <= 1e-4 and, continued from there, to 1e-6 (the reference
    for the optimum). The termination test of Sec. 5.3 bounds the residual, not
    the distance to the optimum, so two solves to 1e-4 can differ by more than
    1e-3 in u even though each is a valid 1e-4 solution (reading C-19). The
    FP32 and FP64 solves' x and u (relative to max(1, max|.|), on the nodes
    whose path weight under the 1e-6 solve's maximising AV@R weights is
    positive: elsewhere the optimal inputs need not be unique) and risk value
    must lie within max(1e-3, 1.25 x the oracle's own 1e-4 distance) of the
    1e-6 reference. (On the 1012-node problem the oracle's 1e-4 solve is about
    5 % from the 1e-6 solve in x and u on that support, and the two supports
    share few nodes: the maximising weights move with the iterate.) A golden file without the 1e-6 solve compares with the 1e-4
    solve instead, bound 2e-3: two 1e-4 solutions, each within the 1e-3
    target of the optimum, lie within 2e-3 of each other. The whole-vector
    errors are printed."""
    import os
    spock = _spock()
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "large_raocp_converged.npz"))
    p = synth.large_raocp()
    g = spock.Problem(p)
    tight = "tight_x" in d.files
    if tight:   # the reference and its support: the 1e-6 solve's
        rx, ru, rr = d["tight_x"], d["tight_u"], float(d["tight_risk"])
        sel = d["tight_path_weight"] > 1e-9
    else:
        rx, ru, rr = d["x"], d["u"], float(d["risk"])
        sel = d["path_weight"] > 1e-9
    seln = sel[:g.n_nl]
    assert sel.sum() > 10
    sx = max(1.0, float(np.max(np.abs(rx[sel]))))
    su = max(1.0, float(np.max(np.abs(ru[seln]))))
    sr = max(1.0, abs(rr))

    def dist(x, u, risk):
        return (float(np.max(np.abs(x[sel] - rx[sel]))) / sx, float(np.max(np.abs(u[seln] - ru[seln]))) / su,
                abs(risk - rr) / sr)

    if tight:
        own = dist(d["x"], d["u"], float(d["risk"]))   # the oracle's own 1e-4 solve
        bound = [max(1e-3, 1.25 * e) for e in own]
        print(f"oracle 1e-4 solve vs its 1e-6 solve: x {own[0]:.2e} u {own[1]:.2e} risk {own[2]:.2e}; "
              f"bounds {bound[0]:.2e} {bound[1]:.2e} {bound[2]:.2e}")
    else:
        bound = [2e-3, 2e-3, 2e-3]
    for prec in (32, 64):
        r = g.solve(p.x0, spock.opts(precision=prec, tol=1e-4, max_iters=200000))
        assert r["status"] == 0
        e = dist(r["x"], r["u"], r["risk"])
        print(f"FP{prec}: x err {e[0]:.2e} u err {e[1]:.2e} on {int(sel.sum())} support nodes, risk err {e[2]:.2e}, "
              f"all-node x err {np.max(np.abs(r['x'] - rx)):.2e} u err {np.max(np.abs(r['u'] - ru)):.2e}")
        assert all(ei <= bi for ei, bi in zip(e, bound)), (prec, e, bound)
