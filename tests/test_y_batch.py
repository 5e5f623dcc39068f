"""Batched solves (many uneven problems in one persistent launch) against the
FP64 oracle and against solving each problem alone.

Tolerances as in test_gpu_parity: FP64 fixed-iteration parity <= 1e-10
relative; FP32 converged solutions within 1e-3 relative on the risk value and
u^0. A problem's result does not depend on the other problems of the launch:
its CTA runs the same arithmetic alone or in the mix, so that comparison is
exact."""
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


def _small_specs(k=6):
    """Problems of the uneven batch generator small enough for the oracle."""
    out = []
    for i, s in enumerate(synth.batch_specs(400, seed=4)):
        if s["nx"] <= 12 and s["N"] <= 8 and s["b"] ** s["k"] <= 16:
            out.append((i, s))
        if len(out) == k:
            break
    return out


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


@pytest.fixture(scope="module")
def plants():
    spock = _spock()
    items = []
    for i, s in _small_specs():
        p = synth.batch_problem(s, i)
        o = Oracle(p)
        g = spock.Problem(p)
        g.set_alpha(o.alpha)
        items.append((p, o, g))
    return items


def test_batch_mix_is_uneven(plants):
    sizes = {(p.nx, len(p.anc)) for p, _, _ in plants}
    assert len(sizes) == len(plants)


def test_batch_fixed_cp_fp64(plants):
    """Plain CP for a fixed count, every problem of the batch: <= 1e-10."""
    spock = _spock()
    b = spock.Batch([g for _, _, g in plants], precision=64)
    iters = 60
    res = b.solve([p.x0 for p, _, _ in plants], spock.opts(precision=64, tol=0.0, max_iters=iters, method="cp"))
    for k, (p, o, g) in enumerate(plants):
        ref = o.solve(tol=0.0, max_iters=iters, method="cp")
        assert res["info"][k]["iters"] == iters
        assert _relerr(g.get_iterate(64).cpu().numpy(), ref["v"]) < 1e-10, k
        assert abs(res["risk"][k] - ref["risk"]) <= 1e-10 * max(1, abs(ref["risk"]))
    b.close()


def test_batch_fixed_spock_fp64(plants):
    """SPOCK for a fixed count in FP64: the same number of T evaluations as the
    oracle and the iterate within 1e-10, for every problem of the batch."""
    spock = _spock()
    b = spock.Batch([g for _, _, g in plants], precision=64)
    iters = 25
    res = b.solve([p.x0 for p, _, _ in plants], spock.opts(precision=64, tol=0.0, max_iters=iters))
    for k, (p, o, g) in enumerate(plants):
        ref = o.solve(tol=0.0, max_iters=iters, method="spock")
        assert res["info"][k]["n_T"] == ref["n_T"], k
        assert _relerr(g.get_iterate(64).cpu().numpy(), ref["v"]) < 1e-10, k
    b.close()


def test_batch_fp32_converged_vs_oracle(plants):
    spock = _spock()
    b = spock.Batch([g for _, _, g in plants], precision=32)
    res = b.solve([p.x0 for p, _, _ in plants], spock.opts(precision=32, tol=1e-4, max_iters=20000))
    assert res["status"] == 0, [i["status"] for i in res["info"]]
    for k, (p, o, g) in enumerate(plants):
        ref = o.solve(tol=1e-4, max_iters=20000)
        assert res["info"][k]["res_inf"] <= 1e-4
        assert abs(res["risk"][k] - ref["risk"]) <= 1e-3 * max(1.0, abs(ref["risk"])), k
        u0 = res["u"][k][0]
        assert np.max(np.abs(u0 - ref["u"][0])) <= 1e-3 * max(1.0, np.max(np.abs(ref["u"][0]))), k
    b.close()


def test_batch_alone_equals_mix(plants):
    """Each problem solved alone (a batch of one) gives bit-identical outputs to
    the same problem solved in the mix."""
    spock = _spock()
    o32 = spock.opts(precision=32, tol=1e-4, max_iters=3000)
    mix = spock.Batch([g for _, _, g in plants], precision=32)
    rm = mix.solve([p.x0 for p, _, _ in plants], o32)
    tws = [i["tw"] for i in rm["info"]]
    mix.close()
    for k, (p, o, g) in enumerate(plants):
        one = spock.Batch([g], precision=32)
        one.set_tw([tws[k]])
        r1 = one.solve([p.x0], o32)
        assert np.array_equal(r1["x"][0], rm["x"][k]), k
        assert np.array_equal(r1["u"][0], rm["u"][k]), k
        assert r1["risk"][0] == rm["risk"][k]
        assert r1["info"][0]["iters"] == rm["info"][k]["iters"]
        one.close()


def test_batch_team_widths_and_autotune(plants):
    """Every admissible warps-per-team choice gives the same iterate (FP64,
    fixed CP count, to rounding); the autotuner returns admissible choices."""
    spock = _spock()
    b = spock.Batch([g for _, _, g in plants], precision=64)
    x0s = [p.x0 for p, _, _ in plants]
    o = spock.opts(precision=64, tol=0.0, max_iters=30, method="cp")
    ref = None
    for t in (1, 2, 4, 8):
        tw = [max(t, 1 if g.nx + g.nu <= 64 else 2) for _, _, g in plants]
        b.set_tw(tw)
        b.solve(x0s, o)
        v = [g.get_iterate(64).cpu().numpy() for _, _, g in plants]
        if ref is None:
            ref = v
        else:
            for a, c in zip(v, ref):
                assert _relerr(a, c) < 1e-12
    tw = b.autotune(iters=5)
    for t, (_, _, g) in zip(tw, plants):
        assert t in (1, 2, 4, 8) and 64 * t >= g.nx + g.nu
    res = b.solve(x0s, o)
    for k, (_, _, g) in enumerate(plants):
        assert _relerr(g.get_iterate(64).cpu().numpy(), ref[k]) < 1e-12
    assert res["status"] in (0, 1)
    b.close()


# --- the gang path: problems whose T moves more than 4 MB get a gang of CTAs ---
@pytest.fixture(scope="module")
def gang_mix():
    """Two problems above the gang threshold (FP64: about 5.6 MB and 4.5 MB of
    factors per T) mixed with two small ones from the uneven generator."""
    spock = _spock()
    from tests.problems import constrained
    probs = [constrained([3, 3, 1, 1, 1], 64, 32, seed=41, avar=0.4, uball=2.5),     # 40 nodes
             constrained([2, 2, 2, 1, 1, 1, 1, 1], 48, 24, seed=42, avar=0.7)]      # 55 nodes
    probs += [synth.batch_problem(s, i) for i, s in _small_specs(2)]
    items = []
    for p in probs:
        o = Oracle(p)
        g = spock.Problem(p)
        g.set_alpha(o.alpha)
        items.append((p, o, g))
    return items


def test_gang_problems_are_ganged(gang_mix):
    """The byte count that sizes a gang exceeds the 4 MB unit for the two large
    problems (factors of both sweeps, FP64)."""
    for p, _, g in gang_mix[:2]:
        s = g.sizes
        assert s["factor_bytes_fp64"] > 4.0e6, s["factor_bytes_fp64"]


def test_gang_batch_fixed_spock_fp64(gang_mix):
    """SPOCK for a fixed count in FP64 with gangs of CTAs iterating on the two
    large problems (flag barriers and reductions among the gang's CTAs): the
    oracle's T count and K0/K1/K2 branches and the iterate within 1e-10, for
    every problem of the mix."""
    spock = _spock()
    b = spock.Batch([g for _, _, g in gang_mix], precision=64)
    iters = 25
    res = b.solve([p.x0 for p, _, _ in gang_mix], spock.opts(precision=64, tol=0.0, max_iters=iters))
    for k, (p, o, g) in enumerate(gang_mix):
        ref = o.solve(tol=0.0, max_iters=iters, method="spock")
        assert res["info"][k]["n_T"] == ref["n_T"], k
        assert _relerr(g.get_iterate(64).cpu().numpy(), ref["v"]) < 1e-10, k
        assert abs(res["risk"][k] - ref["risk"]) <= 1e-10 * max(1.0, abs(ref["risk"])), k
    b.close()


def test_gang_batch_fixed_cp_fp64(gang_mix):
    spock = _spock()
    b = spock.Batch([g for _, _, g in gang_mix], precision=64)
    iters = 40
    b.solve([p.x0 for p, _, _ in gang_mix], spock.opts(precision=64, tol=0.0, max_iters=iters, method="cp"))
    for k, (p, o, g) in enumerate(gang_mix):
        ref = o.solve(tol=0.0, max_iters=iters, method="cp")
        assert _relerr(g.get_iterate(64).cpu().numpy(), ref["v"]) < 1e-10, k
    b.close()


def test_gang_alone_equals_mix_fp32(gang_mix):
    """A ganged problem gives bit-identical results alone (a batch of one, same
    gang size) and in the mix."""
    spock = _spock()
    o32 = spock.opts(precision=32, tol=1e-4, max_iters=400)
    mix = spock.Batch([g for _, _, g in gang_mix], precision=32)
    rm = mix.solve([p.x0 for p, _, _ in gang_mix], o32)
    tws = [i["tw"] for i in rm["info"]]
    mix.close()
    for k in (0, 1):
        p, _, g = gang_mix[k]
        one = spock.Batch([g], precision=32)
        one.set_tw([tws[k]])
        r1 = one.solve([p.x0], o32)
        assert np.array_equal(r1["x"][0], rm["x"][k]), k
        assert np.array_equal(r1["u"][0], rm["u"][k]), k
        assert r1["risk"][0] == rm["risk"][k] and r1["info"][0]["iters"] == rm["info"][k]["iters"]
        one.close()


def test_batch_fp64_check_per_problem(gang_mix):
    """With fp64_check the batch reports each problem's FP64 exit check (Sec.
    5.3), equal to spock_check of the problem's final iterate."""
    spock = _spock()
    b = spock.Batch([g for _, _, g in gang_mix], precision=32)
    res = b.solve([p.x0 for p, _, _ in gang_mix],
                  spock.opts(precision=32, tol=1e-4, max_iters=300, fp64_check=True))
    for k, (_, _, g) in enumerate(gang_mix):
        c = g.check(g.get_iterate(32))
        for key in ("xi1", "xi2", "infeas", "gap"):
            assert res["info"][k][key] == c[key], (k, key)
    b.close()
