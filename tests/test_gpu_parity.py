"""GPU parity: every step of the CUDA path against the FP64 oracle on the same
seeded inputs, through the C ABI.

Tolerances. FP64: the kernels reassociate sums (split-K mat-vecs, the reduced
backward recursion of Alg. 2, closed-form S2 projection), so one T
evaluation differs from the oracle by a few ulps times the condition of the
sweep; 1e-11 relative is asserted for one T, 1e-10 relative after a fixed
iteration count (the bar of the fixed-iteration parity). FP32: one T within
2e-5 relative (24-bit mantissa, sweeps of length <= 2N); converged solutions
within 1e-3 relative on x/u (the FP32 target)."""
import numpy as np
import pytest

from oracle.spock_oracle import Oracle
from paper_2505_12078_b300 import synth
from tests.problems import constrained, general, unconstrained

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


CASES = {
    "small": lambda: synth.small_raocp(),
    "ragged_37x19_ball": lambda: constrained([3, 2, 1, 1], 37, 19, seed=21, avar=0.35, uball=2.5),
    "wide_70x40": lambda: constrained([4, 1, 1], 70, 40, seed=22, avar=0.6, uball=3.0),
    "unconstrained_c": lambda: unconstrained([2, 3, 1], 5, 3, seed=23, avar=0.5, c_scale=0.3),
    "chain_only": lambda: constrained([1, 1, 1, 1, 1], 6, 3, seed=24, avar=0.2),
    "minimal_n2": lambda: constrained([1], 3, 2, seed=25, avar=1.0),
    "avar0_branch8": lambda: constrained([8, 1], 9, 4, seed=26, avar=0.0, uball=1.0),
    # nx + nu = 150 > 128: team sweeps (8 warps per team), widest mat-vec variants
    "team_100x50": lambda: constrained([2, 1, 1], 100, 50, seed=27, avar=0.5, uball=3.0),
    # full weights, linear cost terms, general constraint rows (Sec. 3.1-3.2, Prop. 1)
    "full_lin_box": lambda: general([2, 2, 1], 5, 3, seed=61, avar=0.5, box=True),
    "rows_ball_diag_lin": lambda: _with_ball(general([3, 1, 1], 6, 3, seed=62, avar=0.4, dense=False, n_g=3,
                                                     n_gN=2, box=True), 1.2),
    "full_rows_cta": lambda: general([2, 1, 1], 24, 12, seed=63, avar=0.6, n_g=4, n_gN=2, box=True),
    "full_rows_100x50": lambda: general([2, 1], 100, 50, seed=64, avar=0.5, n_g=3, n_gN=1),
    # nx = 150 > 128 (nx + nu = 200 <= 256): team sweeps with the widest variants
    "team_150x50": lambda: constrained([2, 1], 150, 50, seed=28, avar=0.5),
    # correlated full weights on a chain: the (x, u) block of L'L sets ||L||
    "full_corr_chain": lambda: _correlated(general([1, 1, 1], 6, 2, seed=65, avar=1.0, n_g=1, box=True)),
    # l1 edge costs (Prop. 2): whole-CTA sweeps with full weights, boxes and a
    # ball; team sweeps with diagonal weights
    "l1_box_ball": lambda: _with_l1(_with_ball(general([2, 2, 1], 5, 3, seed=66, avar=0.5, box=True), 1.5), 0.3),
    "l1_team_100x50": lambda: _with_l1(constrained([2, 1], 100, 50, seed=67, avar=0.5, uball=3.0), 0.2),
    # the total-variation risk (a conic risk with F != 0, Sec. 3.3): whole-CTA and team sweeps
    "tv_box_ball": lambda: _with_tv(constrained([3, 2, 1], 6, 3, seed=68, avar=0.5, uball=2.0), 0.4),
    "tv_team_100x50": lambda: _with_tv(constrained([2, 1], 100, 50, seed=69, avar=0.5), 0.3),
    # soft-constraint costs (the penalty after Prop. 2), diagonal weights: whole-CTA and team sweeps
    "soft_box_ball": lambda: _with_soft(_with_ball(general([2, 2, 1], 5, 3, seed=75, avar=0.5, box=True,
                                                           dense=False), 1.5), 0.3),
    "soft_team_100x50": lambda: _with_soft(constrained([2, 1], 100, 50, seed=76, avar=0.5), 0.5),
}


def _with_soft(p, level):
    p.soft_max = np.full(p.nx + p.nu, float(level))
    return p


def _with_tv(p, r):
    p.tv = np.full(p.n_nonleaf, float(r))
    return p


def _with_l1(p, lam):
    p.l1 = float(lam)
    return p


def _correlated(p):
    """Q^c = 11' + 0.1 I and Q_N = 11' + 0.1 I: the scaled cost factor's Gram has
    an eigenvalue near nx / 1.1, above the (y, s) blocks' (about 3.7)."""
    nx = p.nx
    W = np.ones((nx, nx)) + 0.1 * np.eye(nx)
    p.Q = np.broadcast_to(W, (len(p.anc) - 1, nx, nx)).copy()
    p.QN = np.broadcast_to(W, (p.n_leaf, nx, nx)).copy()
    return p


def _with_ball(p, r):
    p.u_ball = np.full(p.n_nonleaf, float(r))
    return p


def _pair(name):
    p = CASES[name]()
    o = Oracle(p)
    g = _spock().Problem(p)
    return p, o, g


def _converged_ref(name):
    """risk and u^0 of the oracle's solve of case `name` to 1e-7 (the optimum,
    golden file), and the bounds a 1e-4 point is held to: 1e-3 relative, or
    1.25 x the distance of the oracle's own 1e-4 point from the optimum where
    that is larger (the residual tolerance bounds that distance only up to a
    problem-dependent factor)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "converged_cases.json")) as f:
        d = json.load(f)["cases"][name]
    u0 = np.array(d["u0"])
    su, sr = max(1.0, float(np.max(np.abs(u0)))), max(1.0, abs(d["risk"]))
    e_u = float(np.max(np.abs(np.array(d["at_1e-4"]["u0"]) - u0))) / su
    e_r = abs(d["at_1e-4"]["risk"] - d["risk"]) / sr
    return {"risk": d["risk"], "u": u0[None, :], "tol_u": max(1e-3, 1.25 * e_u) * su,
            "tol_risk": max(1e-3, 1.25 * e_r) * sr}


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


@pytest.mark.parametrize("name", list(CASES))
def test_setup_scalings_alpha_and_alg1(name):
    """Sec. 5.4 scalings, ||L|| and alpha, Alg. 1 factors P, K, R~, Abar."""
    p, o, g = _pair(name)
    Sx, Su, SxN = g.scalings()
    assert np.allclose(Sx, o.Sx, rtol=1e-15) and np.allclose(Su, o.Su, rtol=1e-15)
    assert np.allclose(SxN, o.SxN, rtol=1e-15)
    alpha, normL = g.alpha()
    assert abs(normL - o.normL) <= 1e-10 * o.normL
    P, K, Rt, Ab = g.factors()
    assert _relerr(P, o.Pm) < 1e-11
    assert _relerr(K, o.K) < 1e-11
    assert _relerr(Rt, o.Rt) < 1e-11
    assert _relerr(Ab, o.Abar) < 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_L_and_adjoint(name):
    p, o, g = _pair(name)
    rng = np.random.default_rng(1)
    z = rng.standard_normal(o.lay.n_z)
    eta = rng.standard_normal(o.lay.n_eta)
    zt = torch.tensor(z, device="cuda")
    et = torch.tensor(eta, device="cuda")
    Lz = g.L(zt).cpu().numpy()
    Ltz = g.Lt(et).cpu().numpy()
    assert _relerr(Lz, o.apply_L(z)) < 1e-14
    assert _relerr(Ltz, o.apply_Lt(eta)) < 1e-14
    # adjoint identity on the GPU alone
    assert abs(eta @ Lz - z @ Ltz) <= 1e-12 * max(1.0, abs(eta @ Lz))
    # FP32
    Lz32 = g.L(zt.float()).cpu().numpy()
    assert _relerr(Lz32, o.apply_L(z)) < 1e-6


def _rand_v(o, seed, scale=2.0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(o.lay.n_z + o.lay.n_eta) * scale


@pytest.mark.parametrize("name", list(CASES))
def test_one_T_fp64_and_fp32(name):
    """One evaluation of T from a random point, FP64 and FP32, and the fused
    reductions (max|r|, ||r_z||^2, ||r_eta||^2, <r_eta, L r_z>)."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    for seed in (2, 3):
        v = _rand_v(o, seed)
        ref = o.T(v)
        vt = torch.tensor(v, device="cuda")
        out, stats = g.T(vt)
        got = out.cpu().numpy()
        assert _relerr(got, ref) < 1e-11, name
        r = v - ref
        nz = o.lay.n_z
        assert abs(stats[0] - np.max(np.abs(r))) <= 1e-11 * max(1, np.max(np.abs(r)))
        assert abs(stats[1] - r[:nz] @ r[:nz]) <= 1e-10 * (r @ r)
        assert abs(stats[2] - r[nz:] @ r[nz:]) <= 1e-10 * (r @ r)
        elz = r[nz:] @ o.apply_L(r[:nz])
        assert abs(stats[3] - elz) <= 1e-10 * (r @ r)
        out32, _ = g.T(vt.float())
        assert _relerr(out32.cpu().numpy(), ref) < 2e-5, name


@pytest.mark.parametrize("name", list(CASES))
def test_centred_T_fp32(name):
    """The centred form of T that the centred FP32 iteration runs on
    (spock_op_T_centred): out = T(c + delta) - c for an FP64 centre c (the
    oracle's iterate after 30 SPOCK iterations) and an FP32 increment delta,
    against the oracle's T(c + delta) - c. The error is measured against the
    increments (max|delta|, max|T(c + delta) - c|), not against c: that is the
    point of the form. delta = 0 gives the centre's own step T(c) - c."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    c = o.solve(tol=0.0, max_iters=30)["v"]
    ct = torch.tensor(c, device="cuda")
    rng = np.random.default_rng(41)
    for amp in (0.0, 1e-3, 1e-1):
        delta = (amp * max(1.0, float(np.max(np.abs(c)))) * rng.standard_normal(c.size)).astype(np.float32)
        ref = o.T(c + delta.astype(np.float64)) - c
        out, stats = g.T_centred(ct, torch.tensor(delta, device="cuda"))
        got = out.cpu().numpy().astype(np.float64)
        scale = max(float(np.max(np.abs(ref))), float(np.max(np.abs(delta))))
        assert float(np.max(np.abs(got - ref))) <= 2e-5 * scale, (name, amp)
        r = delta.astype(np.float64) - ref
        assert abs(stats[0] - np.max(np.abs(r))) <= 2e-5 * scale


def test_centred_T_large_centre():
    """With a centre of magnitude 1e3 and increments of 1e-2 the centred form
    keeps its error at the increments' scale (2e-5 of it), far below the
    rounding of c itself in FP32 (about 6e-5)."""
    p, o, g = _pair("ragged_37x19_ball")
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    rng = np.random.default_rng(43)
    c = 1e3 * rng.standard_normal(o.lay.n_z + o.lay.n_eta)
    delta = (1e-2 * rng.standard_normal(c.size)).astype(np.float32)
    ref = o.T(c + delta.astype(np.float64)) - c
    out, _ = g.T_centred(torch.tensor(c, device="cuda"), torch.tensor(delta, device="cuda"))
    scale = max(float(np.max(np.abs(ref))), float(np.max(np.abs(delta))))
    err = float(np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref)))
    assert err <= 2e-5 * scale, (err, scale)


@pytest.mark.parametrize("name", ["small", "ragged_37x19_ball", "unconstrained_c", "avar0_branch8"])
def test_fixed_iterations_cp_fp64(name):
    """Plain CP iterates v <- T(v) from zero for a fixed count: <= 1e-10 relative."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    spock = _spock()
    iters = 60
    ref = o.solve(tol=0.0, max_iters=iters, method="cp")
    res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=iters, method="cp"))
    assert res["info"]["iters"] == iters
    v = g.get_iterate(64).cpu().numpy()
    assert _relerr(v, ref["v"]) < 1e-10
    assert abs(res["risk"] - ref["risk"]) <= 1e-10 * max(1, abs(ref["risk"]))


@pytest.mark.parametrize("name", ["small", "ragged_37x19_ball", "unconstrained_c", "wide_70x40", "team_100x50",
                                  "full_lin_box", "rows_ball_diag_lin", "full_rows_cta", "full_rows_100x50",
                                  "l1_box_ball", "l1_team_100x50", "tv_box_ball", "tv_team_100x50",
                                  "soft_box_ball", "soft_team_100x50"])
def test_fixed_iterations_spock_fp64(name):
    """SPOCK (Alg. 4 with Anderson directions) for a fixed iteration count in
    FP64: same branch sequence counts and iterate within 1e-10 relative."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    spock = _spock()
    iters = 25
    ref = o.solve(tol=0.0, max_iters=iters, method="spock")
    res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=iters))
    inf = res["info"]
    kinds = [e[1] for e in ref["events"]]
    assert inf["iters"] == iters
    assert inf["n_K0"] == kinds.count("K0")
    assert inf["n_K1"] == kinds.count("K1")
    assert inf["n_K2"] == kinds.count("K2")
    assert inf["n_T"] == ref["n_T"]
    v = g.get_iterate(64).cpu().numpy()
    assert _relerr(v, ref["v"]) < 1e-10


@pytest.mark.parametrize("name,recentre", [("small", 0.1), ("ragged_37x19_ball", 0.1), ("chain_only", 0.1),
                                           ("full_lin_box", 0.1), ("rows_ball_diag_lin", 0.1),
                                           ("team_100x50", 0.1), ("small", 0.0), ("ragged_37x19_ball", 0.0),
                                           ("l1_box_ball", 0.1), ("l1_box_ball", 0.0), ("tv_box_ball", 0.1),
                                           ("soft_box_ball", 0.1)])
def test_converged_fp32_vs_oracle(name, recentre):
    """FP32 iteration to ||v - T(v)||_inf <= 1e-4 against the optimum: the
    oracle's FP64 solve to 1e-7 (tests/golden/converged_cases.json, written by
    tests/golden/make_converged_cases.py from the oracle alone). Risk value and
    u^0 within 1e-3 relative, or within 1.25 x the oracle's own 1e-4 point's
    distance where that is larger; FP64 residual check of the returned iterate.
    recentre 0.1: the centred FP32 iteration (its stopping test is the FP64
    residual, so that is <= 1e-4); 0: the plain one."""
    p, o, g = _pair(name)
    spock = _spock()
    ref = _converged_ref(name)
    res = g.solve(p.x0, spock.opts(precision=32, tol=1e-4, max_iters=20000, recentre=recentre))
    assert res["status"] == 0, res["info"]
    if recentre > 0:
        assert res["info"]["res_inf_fp64"] <= 1e-4 and res["info"]["n_recentre"] >= 1
    assert abs(res["risk"] - ref["risk"]) <= ref["tol_risk"]
    assert np.max(np.abs(res["u"][0] - ref["u"][0])) <= ref["tol_u"]
    assert res["info"]["res_inf_fp64"] < 5e-4
    assert np.all(np.abs(res["x"]) <= 5 + 1e-2)


@pytest.mark.parametrize("name", ["small", "ragged_37x19_ball", "unconstrained_c", "wide_70x40", "avar0_branch8",
                                  "full_lin_box", "rows_ball_diag_lin", "full_rows_cta", "l1_box_ball",
                                  "tv_box_ball", "soft_box_ball"])
def test_fp64_check_matches_oracle(name):
    """FP64 exit check (Sec. 5.3) through spock_check on the oracle's own
    iterate after 25 SPOCK iterations: xi1, xi2 (Eq. xi1k), the primal
    infeasibility and the two terms of the complementarity gap against the
    oracle's diagnostics of the same point. The GPU evaluates T in FP64 itself,
    so the quantities agree to the one-T parity (1e-11 of max|v|) divided by
    alpha (xi1, xi2 divide v - T(v) by alpha)."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    g.set_x0(p.x0)
    ref = o.solve(tol=0.0, max_iters=25)
    v = ref["v"]
    c = g.check(torch.tensor(v, device="cuda"))
    scale = 1e-10 * max(1.0, float(np.max(np.abs(v)))) / o.alpha
    assert abs(c["res_inf"] - ref["res_inf"]) <= scale * o.alpha
    assert abs(c["xi1"] - ref["xi1"]) <= scale, (c["xi1"], ref["xi1"])
    assert abs(c["xi2"] - ref["xi2"]) <= scale, (c["xi2"], ref["xi2"])
    assert abs(c["infeas"] - ref["infeas"]) <= scale, (c["infeas"], ref["infeas"])
    nz = o.lay.n_z
    tv = ref["Tv"]
    Lz = o.apply_L(tv[:nz])
    dot = float(tv[nz:] @ Lz)
    sup = o.support_S3(tv[nz:])
    mag = 1e-10 * (float(np.sum(np.abs(tv[nz:] * Lz))) + abs(sup) + 1.0)
    assert abs(c["eta_Lz"] - dot) <= mag
    assert abs(c["support"] - sup) <= mag
    assert abs(c["gap"] - ref["gap"]) <= 2 * mag


@pytest.mark.parametrize("name", ["small", "ragged_37x19_ball"])
def test_solve_reports_fp64_check(name):
    """spock_solve returns the FP64 exit check of its final iterate: for an FP64
    solve of a fixed iteration count it equals the oracle's diagnostics of the
    oracle's iterate (the iterates agree to 1e-10); for an FP32 solve it equals
    spock_check of the FP32 iterate."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    spock = _spock()
    ref = o.solve(tol=0.0, max_iters=25)
    res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=25))
    inf = res["info"]
    scale = 1e-9 * max(1.0, float(np.max(np.abs(ref["v"])))) / o.alpha
    for k in ("xi1", "xi2", "infeas"):
        assert abs(inf[k] - ref[k]) <= scale, (k, inf[k], ref[k])
    assert abs(inf["gap"] - ref["gap"]) <= 1e-8 * max(1.0, abs(ref["gap"]))
    # plain FP32 iteration: the check of its FP32 iterate; centred: of its FP64 iterate
    for recentre, prec in ((0.0, 32), (0.1, 64)):
        r32 = g.solve(p.x0, spock.opts(precision=32, tol=1e-4, max_iters=20000, recentre=recentre))
        c = g.check(g.get_iterate(prec))
        for k in ("xi1", "xi2", "infeas", "gap"):
            assert r32["info"][k] == c[k], (recentre, k)
        assert r32["info"]["res_inf_fp64"] == c["res_inf"]
        # near the solution every measure is small (Sec. 5.3)
        assert max(c["xi1"], c["xi2"]) < 5e-3 / o.alpha and c["infeas"] < 5e-3


@pytest.mark.parametrize("name", ["small", "ragged_37x19_ball", "wide_70x40", "full_rows_cta"])
def test_fixed_iterations_spock_qr_update_fp64(name):
    """SPOCK with the Anderson least squares solved by an updated QR
    factorisation (Givens rotations to drop the oldest pair, Gram-Schmidt to
    append; Sec. 6.2) against the oracle's own QR-updating memory: the same
    K0/K1/K2 counts and T evaluations, the iterate within 1e-10 (FP64, 25
    iterations)."""
    p, o, g = _pair(name)
    g.set_alpha(o.alpha)
    spock = _spock()
    iters = 25
    ref = o.solve(tol=0.0, max_iters=iters, aa="qr_update")
    res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=iters, aa="qr_update"))
    inf = res["info"]
    kinds = [e[1] for e in ref["events"]]
    assert (inf["n_K0"], inf["n_K1"], inf["n_K2"]) == (kinds.count("K0"), kinds.count("K1"), kinds.count("K2"))
    assert inf["n_T"] == ref["n_T"]
    assert _relerr(g.get_iterate(64).cpu().numpy(), ref["v"]) < 1e-10


@pytest.mark.parametrize("name", ["small", "ragged_37x19_ball"])
def test_converged_fp32_qr_update(name):
    """FP32 SPOCK with the QR-updated Anderson memory to 1e-4: risk value and u^0
    within the bounds of test_converged_fp32_vs_oracle of the optimum (the
    oracle's solve to 1e-7)."""
    p, o, g = _pair(name)
    spock = _spock()
    ref = _converged_ref(name)
    res = g.solve(p.x0, spock.opts(precision=32, tol=1e-4, max_iters=20000, aa="qr_update"))
    assert res["status"] == 0, res["info"]
    assert abs(res["risk"] - ref["risk"]) <= ref["tol_risk"]
    assert np.max(np.abs(res["u"][0] - ref["u"][0])) <= ref["tol_u"]


@pytest.mark.parametrize("name", ["l1_box_ball", "tv_box_ball", "soft_box_ball"])
def test_extended_problems_are_single_problem_only(name):
    """A problem with l1 edge costs (Prop. 2), total-variation risks or
    soft-constraint costs is solved by the single-problem calls; the batched
    and serving calls refuse it
    with SPOCK_EUNSUPPORTED (-6) instead of running paths that do not carry its
    auxiliaries or its risk data."""
    spock = _spock()
    p = CASES[name]()
    g = spock.Problem(p)
    with pytest.raises(spock.SpockError) as e:
        spock.Batch([g], precision=32)
    assert e.value.code == -6
    with pytest.raises(spock.SpockError) as e:
        spock.Server([g], precision=32)
    assert e.value.code == -6


def test_soft_costs_need_diagonal_weights_and_no_l1():
    """Soft-constraint costs are refused (SPOCK_EUNSUPPORTED, -6) with full
    weights or together with an l1 term, and a non-finite level is invalid
    (SPOCK_EINVAL, -1)."""
    spock = _spock()
    p = _with_soft(general([2, 1], 3, 2, seed=77, avar=0.5), 0.3)          # full weights
    with pytest.raises(spock.SpockError) as e:
        spock.Problem(p)
    assert e.value.code == -6
    q = _with_l1(CASES["soft_box_ball"](), 0.2)
    with pytest.raises(spock.SpockError) as e:
        spock.Problem(q)
    assert e.value.code == -6
    r = CASES["soft_box_ball"]()
    r.soft_max[0] = np.inf
    with pytest.raises(spock.SpockError) as e:
        spock.Problem(r)
    assert e.value.code == -1
