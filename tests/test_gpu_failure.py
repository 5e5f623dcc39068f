"""Failure path on the GPU without a GPU fault: a device-side wait that runs
out of its time limit. The test hook spock_debug_wait_fault makes the grid
barriers of a single-problem launch wait for one CTA more than the launch has,
with a 5 ms limit; the first barrier wait then gives up, the launch records the
timeout, every CTA leaves (after its bulk copies have landed) and the call
returns SPOCK_ETIMEOUT. Nothing traps and the context stays usable: the next
solve in the same process succeeds and matches a solve made before the fault."""
import numpy as np
import pytest

from paper_2505_12078_b300 import synth
from tests.problems import constrained

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2505_12078_b300 import build, spock
    build.build()
    spock.load()


@pytest.mark.parametrize("maker", [synth.small_raocp,                                   # team sweeps
                                   lambda: constrained([3, 1, 1], 24, 12, seed=5)])     # whole-CTA sweeps
def test_barrier_wait_runs_out_and_context_survives(maker):
    from paper_2505_12078_b300 import spock
    p = maker()
    g = spock.Problem(p)
    o = spock.opts(precision=64, tol=0.0, max_iters=20)
    before = g.solve(p.x0, o)
    try:
        spock.debug_wait_fault(1, 0.005)
        with pytest.raises(spock.SpockError) as e:
            g.solve(p.x0, o)
        assert e.value.code == -5        # SPOCK_ETIMEOUT
        v = torch.zeros(g.n_v, dtype=torch.float64, device="cuda")
        with pytest.raises(spock.SpockError) as e2:
            g.T(v)
        assert e2.value.code == -5
    finally:
        spock.debug_wait_fault(0, 0.0)
    torch.cuda.synchronize()
    after = g.solve(p.x0, o)
    assert after["status"] == 1          # max_iters reached, as before
    assert np.array_equal(after["x"], before["x"]) and after["risk"] == before["risk"]


def test_wait_fault_arguments_checked():
    from paper_2505_12078_b300 import spock
    for bad in ((-1, 0.0), (5, 0.0), (0, -1.0), (0, 11.0)):
        with pytest.raises(spock.SpockError):
            spock.debug_wait_fault(*bad)
    spock.debug_wait_fault(0, 0.0)
