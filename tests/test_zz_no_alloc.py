"""spock_op_T_noalloc: one evaluation of T for callers that cannot allocate
device memory during the call (an allocator they do not own, a real-time
loop that must not block on an allocation, a fully reserved device). Its
scratch comes from the library's static device array. Checked against
spock_op_T on two calls in a row (the shared array keeps the previous call's
contents, so the second call shows that what must start at zero is reset).

Collected last on purpose (file name), and independent of the other tests:
it creates its own problems and passes in a fresh process as well."""
import numpy as np
import pytest

from paper_2505_12078_b300 import synth
from tests.problems import constrained

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems():
    return [synth.small_raocp(), constrained([3, 2, 1, 1], 37, 19, seed=21, avar=0.35, uball=2.5),
            synth.large_raocp()]


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_T_matches_op_T_on_two_calls(k, precision):
    from paper_2505_12078_b300 import build, spock
    build.build()
    spock.load()
    p = _problems()[k]
    g = spock.Problem(p)
    g.set_x0(p.x0)
    dt = torch.float64 if precision == 64 else torch.float32
    tol = 1e-11 if precision == 64 else 2e-5      # tolerances of the T parity tests
    rng = np.random.default_rng(40 + k)
    for call in range(2):
        v = torch.tensor(rng.standard_normal(g.n_v) * 2.0, dtype=dt, device="cuda")
        ref, st_ref = g.T(v)
        out = torch.full_like(v, float("nan"))
        out, st = g.T_noalloc(v, out)
        torch.cuda.synchronize()
        a = out.double().cpu().numpy()
        b = ref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b))), (call, precision)
        assert abs(st[0] - st_ref[0]) <= tol * max(1.0, st_ref[0])
