"""The paper's first case study as a workload (Sec. 8.1): random RAOCPs with
per-event dynamics and full per-event weights Q(w) = (Q0 + Q^w)(Q0 + Q^w)',
boxes on x and u, AV@R with a random level. One evaluation of T and a fixed
SPOCK iteration count against the oracle on problems small enough for it
(n_v between 1e3 and 3e3), and the library's device memory on a problem of
n_v close to 1e5 (the paper reports about 1 GB of CPU and GPU memory for
SPOCK there). Tolerances as in test_gpu_parity."""
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


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


@pytest.mark.parametrize("seed", [0, 3, 5])
def test_case_study_one_T_and_fixed_iterations(seed):
    from paper_2505_12078_b300 import spock
    p = synth.case_study_1(seed, nv_range=(1e3, 3e3))
    o = Oracle(p)
    g = spock.Problem(p)
    alpha, normL = g.alpha()
    assert abs(normL - o.normL) <= 1e-9 * o.normL
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    v = np.random.default_rng(seed).standard_normal(o.lay.n_z + o.lay.n_eta)
    ref = o.T(v)
    out, _ = g.T(torch.tensor(v, device="cuda"))
    assert _relerr(out.cpu().numpy(), ref) < 1e-11
    out32, _ = g.T(torch.tensor(v, device="cuda").float())
    assert _relerr(out32.cpu().numpy(), ref) < 2e-5
    iters = 15
    r = o.solve(tol=0.0, max_iters=iters)
    res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=iters))
    kinds = [e[1] for e in r["events"]]
    assert res["info"]["n_T"] == r["n_T"]
    assert (res["info"]["n_K0"], res["info"]["n_K1"], res["info"]["n_K2"]) == \
        (kinds.count("K0"), kinds.count("K1"), kinds.count("K2"))
    assert _relerr(g.get_iterate(64).cpu().numpy(), r["v"]) < 1e-10


def test_case_study_device_memory_at_1e5_variables():
    """Device bytes the library holds for a case-study problem with n_v near
    1e5 after a solve in FP32 (data, FP64 and FP32 factors, solve buffers) and
    its peak during the offline part. The library keeps FP64 and FP32 copies of
    every factor, so the bound asserted is 2 GB; the measured figure is
    reported by bench.py beside the paper's (about 1 GB combined)."""
    from paper_2505_12078_b300 import spock
    p = synth.case_study_1(0, nv_range=(9e4, 1e5))
    free0, _ = torch.cuda.mem_get_info()
    g = spock.Problem(p)
    r = g.solve(p.x0, spock.opts(precision=32, tol=1e-4, max_iters=200, fp64_check=False))
    held, peak = g.memory()
    free1, _ = torch.cuda.mem_get_info()
    assert 0 < held <= peak < 2 << 30, (held, peak)
    assert free0 - free1 >= held          # the driver's view includes the library's allocations
    assert r["info"]["iters"] > 0


# --- the second case study (Sec. 8.2): delay-driven Beta-quantile trees -------------
@pytest.mark.parametrize("shape", ["wide", "deep"])
def test_delay_tree_problem_parity(shape):
    """Networked control with a sensor-to-controller delay on the two tree
    shapes of the tree-shape study ([n^2, 1, ..] and [n, n, 1, ..], n = 2),
    reduced to N = 6, nx = 8, nu = 4 for the oracle: one T and a fixed SPOCK
    iteration count in FP64."""
    from paper_2505_12078_b300 import spock
    p = synth.ncs_delay(2, shape, N=6, nx=8, nu=4)
    o = Oracle(p)
    g = spock.Problem(p)
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    v = np.random.default_rng(11).standard_normal(o.lay.n_z + o.lay.n_eta)
    out, _ = g.T(torch.tensor(v, device="cuda"))
    assert _relerr(out.cpu().numpy(), o.T(v)) < 1e-11
    r = o.solve(tol=0.0, max_iters=15)
    res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=15))
    assert res["info"]["n_T"] == r["n_T"]
    assert _relerr(g.get_iterate(64).cpu().numpy(), r["v"]) < 1e-10


@pytest.mark.parametrize("shape", ["wide", "deep"])
def test_delay_tree_full_size_one_T(shape):
    """The study's full sizes (N = 48, nx = 100 plant states + 50 delayed
    inputs = 150, nu = 50, AV@R 0.95), n = 2: one T in FP64 and FP32 against
    the oracle (team sweeps with nx > 128)."""
    from paper_2505_12078_b300 import spock
    p = synth.ncs_delay(2, shape)
    o = Oracle(p)
    g = spock.Problem(p)
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    v = np.random.default_rng(12).standard_normal(o.lay.n_z + o.lay.n_eta)
    ref = o.T(v)
    vt = torch.tensor(v, device="cuda")
    out, _ = g.T(vt)
    assert _relerr(out.cpu().numpy(), ref) < 1e-11
    out32, _ = g.T(vt.float())
    assert _relerr(out32.cpu().numpy(), ref) < 2e-5
