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


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_alternating_sizes_share_the_array(precision):
    """Calls on problems of different sizes alternate on the one shared array
    (small -> large -> small -> large): a stale barrier epoch, segment flag or
    control word left by a problem with another grid or segment count would
    show up as a wrong or hung result. Each call matches spock_op_T."""
    from paper_2505_12078_b300 import build, spock
    build.build()
    spock.load()
    ps = [synth.small_raocp(), synth.large_raocp()]
    gs = [spock.Problem(p) for p in ps]
    for p, g in zip(ps, gs):
        g.set_x0(p.x0)
    dt = torch.float64 if precision == 64 else torch.float32
    tol = 1e-11 if precision == 64 else 2e-5
    rng = np.random.default_rng(77)
    for k in (0, 1, 0, 1):
        g = gs[k]
        v = torch.tensor(rng.standard_normal(g.n_v) * 2.0, dtype=dt, device="cuda")
        ref, _ = g.T(v)
        out = torch.full_like(v, float("nan"))
        out, _ = g.T_noalloc(v, out)
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b))), (k, precision)


def test_noalloc_rejects_problems_beyond_the_array():
    """A problem whose scratch (about 2 (n nx + n_nl nu) words plus the control
    data) exceeds the static array gets SPOCK_EUNSUPPORTED and leaves the
    output untouched; the entry point still serves a small problem after it."""
    from paper_2505_12078_b300 import build, spock
    build.build()
    spock.load()
    big = constrained([4, 4, 4, 4] + [1] * 36, 64, 32, seed=31)     # 9557 nodes: ~14.5 MB in FP64
    g = spock.Problem(big)
    g.set_x0(big.x0)
    assert 2 * 8 * (g.n * big.nx + g.n_nl * big.nu) > 8 << 20
    v = torch.zeros(g.n_v, dtype=torch.float64, device="cuda")
    out = torch.full_like(v, 7.0)
    with pytest.raises(spock.SpockError) as e:
        g.T_noalloc(v, out)
    assert e.value.code == -6
    assert bool(torch.all(out == 7.0))
    p = synth.small_raocp()
    s = spock.Problem(p)
    s.set_x0(p.x0)
    w = torch.tensor(np.random.default_rng(5).standard_normal(s.n_v), dtype=torch.float64, device="cuda")
    ref, _ = s.T(w)
    out2, _ = s.T_noalloc(w, torch.empty_like(w))
    assert float(torch.max(torch.abs(out2 - ref))) <= 1e-11 * max(1.0, float(torch.max(torch.abs(ref))))
