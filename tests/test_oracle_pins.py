"""Pins of the FP64 oracle against what the paper and the mathematics fix,
independently of the oracle's own code paths (closed forms, textbook
recursions, dense linear algebra, LP duals, brute force)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so

from oracle import spock_oracle as so_
from oracle.spock_oracle import Oracle
from paper_2505_12078_b300 import synth
from tests.problems import constrained, general, unconstrained

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- problem layout -----------------------------------------------------------
def test_sizes_match_hand_count():
    """Vector lengths from the definitions of Sec. 4.3-4.4 (counted by hand)."""
    g = json.load(open(os.path.join(GOLDEN, "sizes.json")))
    for key, ref in g.items():
        if key.startswith("_"):
            continue
        if key == "small_raocp":
            p = synth.small_raocp()
        elif key == "large_raocp":
            p = synth.large_raocp()
        else:
            p = synth.tree_sweep(int(key.split("_")[-1]))
        tr = so_.Tree(p.anc, p.prob)
        assert (tr.n, tr.n_nl, tr.n_l) == (ref["n"], ref["n_nonleaf"], ref["n_leaf"])
        if key in ("small_raocp",):
            o = Oracle(p)
            assert (o.lay.n_z, o.lay.n_eta) == (ref["n_z"], ref["n_eta"])
        else:
            # layout only (no factorisation needed)
            o = Oracle.__new__(Oracle)
            o.P, o.tree, o.n, o.nx, o.nu = p, tr, tr.n, p.nx, p.nu
            o.has_xbox, o.has_ubox, o.has_uball = True, True, p.u_ball is not None
            o.n_c = p.nx + p.nu + (p.nu if p.u_ball is not None else 0)
            o.n_cN = p.nx
            o.l1, o.soft = 0.0, None
            o._layout()
            assert (o.lay.n_z, o.lay.n_eta) == (ref["n_z"], ref["n_eta"])


def test_tree_probabilities_sum_to_one_per_stage():
    """Sec. 3.2: sum over nodes(t) of pi^i = 1."""
    tr = so_.Tree(*synth.tree_from_branching([3, 2, 1, 4], np.random.default_rng(0)))
    for t in range(tr.N + 1):
        assert abs(tr.pi[tr.nodes_at[t]].sum() - 1.0) < 1e-13


# --- risk measures ------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_avar_closed_form_vs_ambiguity_lp_and_conic_dual(seed):
    """AV@R by sorting = max over the ambiguity set (LP) = min of the conic dual
    with the printed b, E, K (Sec. 3.3)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 6))
    Z = rng.standard_normal(n)
    p = rng.dirichlet(np.ones(n))
    a = float(rng.uniform(0.05, 1.0))
    val = so_.avar(Z, p, a)
    # primal: max mu'Z, sum mu = 1, 0 <= mu <= p/a
    lp = so.linprog(-Z, A_eq=np.ones((1, n)), b_eq=[1.0],
                    bounds=[(0.0, p[j] / a) for j in range(n)], method="highs")
    assert lp.status == 0
    assert abs(-lp.fun - val) < 1e-10
    # conic dual: min y'b s.t. E'y = Z, y in K* = R^{2n}_+ x R
    b, E = so_.conic_risk_data(p, a)
    bounds = [(0, None)] * (2 * n) + [(None, None)]
    dual = so.linprog(b, A_eq=E.T, b_eq=Z, bounds=bounds, method="highs")
    assert dual.status == 0
    assert abs(dual.fun - val) < 1e-9


def test_avar_extremes():
    """AV@R_1 = expectation, AV@R_0 = max (Sec. 3.3)."""
    rng = np.random.default_rng(1)
    Z = rng.standard_normal(5)
    p = rng.dirichlet(np.ones(5))
    assert abs(so_.avar(Z, p, 1.0) - p @ Z) < 1e-14
    assert so_.avar(Z, p, 0.0) == Z.max()
    assert abs(so_.avar(Z, p, 1e-9) - Z.max()) < 1e-12


# --- projections ----------------------------------------------------------------
def test_proj_soc_moreau_characterisation():
    """Moreau: v = P(v) - P(-v) with both in SOC (self-dual) and orthogonal
    characterises the projection onto SOC uniquely."""
    rng = np.random.default_rng(2)
    V = rng.standard_normal((400, 7)) * 3
    V[:50, -1] = np.abs(V[:50, -1]) + 10           # inside
    V[50:100, -1] = -np.abs(V[50:100, -1]) - 10    # polar
    P = so_.proj_soc(V)
    Qn = so_.proj_soc(-V)
    assert np.allclose(P - Qn, V, atol=1e-12)
    assert np.all(np.linalg.norm(P[:, :-1], axis=1) <= P[:, -1] + 1e-12)
    assert np.all(np.linalg.norm(Qn[:, :-1], axis=1) <= Qn[:, -1] + 1e-12)
    assert np.allclose(np.sum(P * Qn, axis=1), 0.0, atol=1e-10)


def test_proj_S2_vs_nullspace_basis():
    """proj_S2 equals N N' v with N an orthonormal basis of ker[E', -I, -I]
    (Sec. 4.3), computed by SVD."""
    p = constrained([3, 2, 1], 2, 1, seed=3, avar=0.37)
    o = Oracle(p)
    rng = np.random.default_rng(4)
    z = rng.standard_normal(o.lay.n_z)
    s0, x, u, y, tau, s = o.split_z(z)
    y2, tau2, s2 = o.proj_S2(y, tau, s)
    tr = o.tree
    for i in range(tr.n_nl):
        ch = tr.children[i]
        m = len(ch)
        a = o.avar_level[i]
        Et = np.hstack([a * np.eye(m), -np.eye(m), np.ones((m, 1))])
        G = np.hstack([Et, -np.eye(m), -np.eye(m)])
        Nb = sla.null_space(G)
        v = np.concatenate([y[o.yoff[i]:o.yoff[i + 1]], tau[ch - 1], s[ch - 1]])
        ref = Nb @ (Nb.T @ v)
        got = np.concatenate([y2[o.yoff[i]:o.yoff[i + 1]], tau2[ch - 1], s2[ch - 1]])
        assert np.allclose(got, ref, atol=1e-12)


def _dense_kkt_projection(o, xbar, ubar):
    """min 1/2||x - xbar||^2 + 1/2||u - ubar||^2 s.t. x^0 = x0, x^c = A x^a + B u^a + c,
    solved as one dense KKT system."""
    tr = o.tree
    nx, nu, n = o.nx, o.nu, tr.n
    nX = n * nx + tr.n_nl * nu
    rows = []
    rhs = []
    C0 = np.zeros((nx, nX)); C0[:, :nx] = np.eye(nx)
    rows.append(C0); rhs.append(o.x0s)
    for c in range(1, n):
        a = tr.anc[c]
        Cc = np.zeros((nx, nX))
        Cc[:, c * nx:(c + 1) * nx] = np.eye(nx)
        Cc[:, a * nx:(a + 1) * nx] = -o.At[c - 1]
        Cc[:, n * nx + a * nu:n * nx + (a + 1) * nu] = -o.Bt[c - 1]
        rows.append(Cc); rhs.append(o.ct[c - 1])
    C = np.vstack(rows)
    d = np.concatenate(rhs)
    target = np.concatenate([xbar.ravel(), ubar.ravel()])
    K = np.block([[np.eye(nX), C.T], [C, np.zeros((C.shape[0], C.shape[0]))]])
    sol = np.linalg.solve(K, np.concatenate([target, d]))
    X = sol[:nX]
    return X[:n * nx].reshape(n, nx), X[n * nx:].reshape(tr.n_nl, nu)


@pytest.mark.parametrize("branching,nx,nu,seed", [([2, 1, 2], 3, 2, 0), ([3, 2], 2, 2, 1),
                                                  ([1, 1, 1, 1], 4, 1, 2), ([2, 3, 1], 3, 3, 3)])
def test_proj_S1_equals_dense_kkt(branching, nx, nu, seed):
    """Alg. 1-2 compute the Euclidean projection onto S1 (with affine c)."""
    p = unconstrained(branching, nx, nu, seed, c_scale=0.5)
    o = Oracle(p)
    rng = np.random.default_rng(seed + 10)
    xbar = rng.standard_normal((o.tree.n, nx)) * 2
    ubar = rng.standard_normal((o.tree.n_nl, nu)) * 2
    x, u = o.proj_S1(xbar, ubar)
    xr, ur = _dense_kkt_projection(o, xbar, ubar)
    assert np.allclose(x, xr, atol=1e-11, rtol=1e-11)
    assert np.allclose(u, ur, atol=1e-11, rtol=1e-11)
    x2, u2 = o.proj_S1(x, u)               # idempotent
    assert np.allclose(x2, x, atol=1e-11) and np.allclose(u2, u, atol=1e-11)


# --- the linear operator L --------------------------------------------------------
def test_L_cost_blocks_encode_epigraph():
    """Prop. 1 (q = 0): with tau^c equal to the edge cost of the UNSCALED state
    and input, the cost block of L z minus a lies on the SOC boundary; larger
    tau is strictly inside, smaller strictly outside. Same for the leaf's s^j
    and the terminal cost."""
    p = unconstrained([2, 2, 1], 3, 2, seed=7)
    o = Oracle(p)
    tr = o.tree
    rng = np.random.default_rng(8)
    z = rng.standard_normal(o.lay.n_z)
    s0, x, u, y, tau, s = o.split_z(z)
    xu = x / o.Snode
    uu = u / o.Su
    for c in range(1, tr.n):
        a = tr.anc[c]
        tau[c - 1] = np.sum(p.Q[c - 1] * xu[a] ** 2) + np.sum(p.R[c - 1] * uu[a] ** 2)
    for jj in range(tr.n_l):
        j = tr.n_nl + jj
        s[j - 1] = np.sum(p.QN[jj] * xu[j] ** 2)
    z = o.join_z(s0, x, u, y, tau, s)
    w = o.nx + o.nu + 2
    for delta, sign in ((0.0, 0), (1e-3, 1), (-1e-3, -1)):
        zz = z.copy()
        zz[o.lay.o_tau:o.lay.o_s] += delta
        zz[o.lay.o_s + tr.n_nl - 1:] += delta
        eta = o.apply_L(zz)
        Qb = eta[o.lay.e_q:o.lay.e_cN].reshape(tr.n - 1, w)
        aa = np.zeros(w); aa[-2], aa[-1] = 0.5, -0.5
        d = Qb - aa
        gap = d[:, -1] - np.linalg.norm(d[:, :-1], axis=1)
        QN = eta[o.lay.e_qN:].reshape(tr.n_l, o.nx + 2)
        aN = np.zeros(o.nx + 2); aN[-2], aN[-1] = 0.5, -0.5
        dN = QN - aN
        gapN = dN[:, -1] - np.linalg.norm(dN[:, :-1], axis=1)
        if sign == 0:
            assert np.allclose(gap, 0, atol=1e-12) and np.allclose(gapN, 0, atol=1e-12)
        else:
            assert np.all(np.sign(gap) == sign) and np.all(np.sign(gapN) == sign)


def test_L_constraint_rows_encode_unscaled_sets():
    """The scaled constraint rows of L z lie in the scaled sets exactly when the
    unscaled x, u satisfy the original box and ball constraints (Sec. 5.4)."""
    p = constrained([2, 2, 1], 4, 3, seed=9, uball=1.5)
    o = Oracle(p)
    tr = o.tree
    rng = np.random.default_rng(10)
    for trial in range(20):
        xu = rng.uniform(-6, 6, (tr.n, o.nx))
        uu = rng.uniform(-2.5, 2.5, (tr.n_nl, o.nu))
        z = o.join_z(0.0, xu * o.Snode, uu * o.Su, np.zeros(o.lay.n_y),
                     np.zeros(tr.n - 1), np.zeros(tr.n - 1))
        eta = o.apply_L(z)
        pe = o.proj_S3(eta)
        C = (eta - pe)[o.lay.e_c:o.lay.e_q].reshape(tr.n_nl, o.n_c)
        CN = (eta - pe)[o.lay.e_cN:o.lay.e_qN].reshape(tr.n_l, o.n_cN)
        for i in range(tr.n_nl):
            ok = (np.all(np.abs(xu[i]) <= 5) and np.all(np.abs(uu[i]) <= 2)
                  and np.linalg.norm(uu[i]) <= 1.5)
            assert ok == bool(np.all(np.abs(C[i]) < 1e-14))
        for jj in range(tr.n_l):
            ok = np.all(np.abs(xu[tr.n_nl + jj]) <= 5)
            assert ok == bool(np.all(np.abs(CN[jj]) < 1e-14))


def test_norm_L_dense_svd_and_step_size():
    """alpha ||L|| = 0.99 < 1 (Sec. 4.1); the Lanczos branch agrees with dense SVD."""
    p = constrained([2, 2, 1], 3, 2, seed=11)
    o = Oracle(p)
    ref = np.linalg.svd(o.L.toarray(), compute_uv=False)[0]
    assert abs(o.normL - ref) < 1e-12 * ref
    assert abs(o.alpha * ref - 0.99) < 1e-12
    assert abs(o._norm_L(dense_max=0) - ref) < 1e-10 * ref


# --- the CP operator ---------------------------------------------------------------
def test_T_firmly_nonexpansive_in_M():
    """T is firmly nonexpansive in the M metric (Sec. 4.1):
    ||Tv - Tw||_M^2 <= <Tv - Tw, v - w>_M."""
    p = constrained([2, 2, 1, 1], 3, 2, seed=12, uball=2.5)
    o = Oracle(p)
    rng = np.random.default_rng(13)
    nv = o.lay.n_z + o.lay.n_eta
    for _ in range(30):
        v = rng.standard_normal(nv) * 3
        w = rng.standard_normal(nv) * 3
        d = o.T(v) - o.T(w)
        assert o.M_inner(d, d) <= o.M_inner(d, v - w) + 1e-10


def test_fixed_point_is_invariant():
    """A converged iterate is (numerically) a fixed point and T(v) keeps x^0 = x0."""
    p = constrained([2, 1], 3, 2, seed=16)
    o = Oracle(p)
    r = o.solve(tol=1e-6, max_iters=20000, method="spock")
    assert r["res_inf"] <= 1e-6
    assert np.allclose(r["x"][0], p.x0, atol=1e-13)
    tv = o.T(r["v"])
    assert np.max(np.abs(tv - r["Tv"])) == 0.0


# --- Anderson's acceleration ---------------------------------------------------------
def test_aa_direction_solves_linear_residual():
    """For an affine residual R(v) = A v - b in R^m with m secant pairs, v + psi
    is the zero of R (the type-II AA step is exact); kappa agrees with an
    SVD least-squares solve."""
    rng = np.random.default_rng(14)
    m = 3
    Am = rng.standard_normal((m, m)) + 3 * np.eye(m)
    b = rng.standard_normal(m)
    R = lambda v: Am @ v - b
    vs = [rng.standard_normal(m) for _ in range(m + 1)]
    S = [vs[i + 1] - vs[i] for i in range(m)]
    Y = [R(vs[i + 1]) - R(vs[i]) for i in range(m)]
    v = vs[-1]
    psi = Oracle.aa_direction(R(v), S, Y, k=m + 1, m=m)
    assert np.allclose(R(v + psi), 0.0, atol=1e-10)
    kappa = np.linalg.lstsq(np.column_stack(Y), R(v), rcond=None)[0]
    assert np.allclose(-R(v) - (np.column_stack(S) - np.column_stack(Y)) @ kappa, psi, atol=1e-10)


# --- whole-solve pins ------------------------------------------------------------------
def test_one_branch_tree_is_finite_horizon_lqr():
    """Single scenario, AV@R_1, no constraints: the risk value is x0'P_0 x0 of
    the time-varying Riccati recursion and u^t = K_t x^t."""
    p = unconstrained([1, 1, 1, 1], 3, 2, seed=5)
    o = Oracle(p)
    r = o.solve(tol=1e-10, max_iters=20000, method="spock")
    N = 4
    Ps = [None] * (N + 1)
    Ks = [None] * N
    Ps[N] = np.diag(p.QN[0])
    for t in range(N - 1, -1, -1):
        A, B = p.A[t], p.B[t]
        Q, R = np.diag(p.Q[t]), np.diag(p.R[t])
        H = R + B.T @ Ps[t + 1] @ B
        Ks[t] = -np.linalg.solve(H, B.T @ Ps[t + 1] @ A)
        Ps[t] = Q + A.T @ Ps[t + 1] @ A + A.T @ Ps[t + 1] @ B @ Ks[t]
    V = p.x0 @ Ps[0] @ p.x0
    assert abs(r["risk"] - V) < 1e-7 * max(1.0, abs(V))
    for t in range(N):
        assert np.allclose(r["u"][t], Ks[t] @ r["x"][t], atol=1e-7)


def _tree_riccati(p):
    tr = so_.Tree(p.anc, p.prob)
    Pm = [None] * tr.n
    for jj in range(tr.n_l):
        Pm[tr.n_nl + jj] = np.diag(p.QN[jj])
    for t in range(tr.N - 1, -1, -1):
        for i in tr.nodes_at[t]:
            H = np.zeros((p.nu, p.nu)); G = np.zeros((p.nu, p.nx)); F = np.zeros((p.nx, p.nx))
            for c in tr.children[i]:
                pc = tr.prob[c]
                A, B, P = p.A[c - 1], p.B[c - 1], Pm[c]
                F += pc * (np.diag(p.Q[c - 1]) + A.T @ P @ A)
                H += pc * (np.diag(p.R[c - 1]) + B.T @ P @ B)
                G += pc * (B.T @ P @ A)
            Pm[i] = F - G.T @ np.linalg.solve(H, G)
    return p.x0 @ Pm[0] @ p.x0


def _risk_neutral_qp(p):
    """min sum_c pi^c (x^a'Q^c x^a + u^a'R^c u^a) + sum_j pi^j x^j'QN x^j s.t.
    dynamics, as one dense equality-constrained QP."""
    tr = so_.Tree(p.anc, p.prob)
    nx, nu, n = p.nx, p.nu, tr.n
    nX = n * nx + tr.n_nl * nu
    H = np.zeros((nX, nX))
    for c in range(1, n):
        a = tr.anc[c]
        H[a * nx:(a + 1) * nx, a * nx:(a + 1) * nx] += tr.pi[c] * np.diag(p.Q[c - 1])
        o = n * nx + a * nu
        H[o:o + nu, o:o + nu] += tr.pi[c] * np.diag(p.R[c - 1])
    for jj in range(tr.n_l):
        j = tr.n_nl + jj
        H[j * nx:(j + 1) * nx, j * nx:(j + 1) * nx] += tr.pi[j] * np.diag(p.QN[jj])
    rows, rhs = [], []
    C0 = np.zeros((nx, nX)); C0[:, :nx] = np.eye(nx); rows.append(C0); rhs.append(p.x0)
    for c in range(1, n):
        a = tr.anc[c]
        Cc = np.zeros((nx, nX))
        Cc[:, c * nx:(c + 1) * nx] = np.eye(nx)
        Cc[:, a * nx:(a + 1) * nx] = -p.A[c - 1]
        Cc[:, n * nx + a * nu:n * nx + (a + 1) * nu] = -p.B[c - 1]
        rows.append(Cc); rhs.append(p.c[c - 1])
    C = np.vstack(rows)
    K = np.block([[2 * H, C.T], [C, np.zeros((C.shape[0], C.shape[0]))]])
    sol = np.linalg.solve(K, np.concatenate([np.zeros(nX), np.concatenate(rhs)]))
    X = sol[:nX]
    return float(X @ H @ X)


def test_risk_neutral_tree_riccati_and_kkt():
    """AV@R_1 and no constraints: risk-neutral multistage LQ, equal to the tree
    Riccati value with conditional probabilities and to a dense KKT solve."""
    p = unconstrained([2, 3, 1], 3, 2, seed=6)
    o = Oracle(p)
    r = o.solve(tol=1e-10, max_iters=30000, method="spock")
    V1 = _tree_riccati(p)
    V2 = _risk_neutral_qp(p)
    assert abs(V1 - V2) < 1e-10 * max(1.0, abs(V1))
    assert abs(r["risk"] - V1) < 1e-7 * max(1.0, abs(V1))


def test_one_stage_two_children_avar_bruteforce():
    """N = 1, two children, AV@R_a with a < 1, no constraints:
    V* = max over the ambiguity segment of min_u sum mu_j Z_j(u) (minimax of a
    convex-concave function), inner problem in closed form, outer by golden
    section."""
    p = unconstrained([2], 2, 2, seed=15, avar=0.4)
    o = Oracle(p)
    r = o.solve(tol=1e-10, max_iters=50000, method="spock")
    x0 = p.x0
    pr = p.prob[1:]
    a = 0.4

    def phi(m1):
        mu = np.array([m1, 1 - m1])
        H = np.zeros((p.nu, p.nu)); g = np.zeros(p.nu); const = 0.0
        for j in range(2):
            A, B = p.A[j], p.B[j]
            QN = np.diag(p.QN[j])
            H += mu[j] * (np.diag(p.R[j]) + B.T @ QN @ B)
            g += mu[j] * (B.T @ QN @ A @ x0)
            const += mu[j] * (x0 @ np.diag(p.Q[j]) @ x0 + (A @ x0) @ QN @ (A @ x0))
        u = -np.linalg.solve(H, g)
        return u @ H @ u + 2 * g @ u + const

    lo = max(0.0, 1 - pr[1] / a)
    hi = min(1.0, pr[0] / a)
    gr = (math.sqrt(5) - 1) / 2
    x1, x2 = hi - gr * (hi - lo), lo + gr * (hi - lo)
    f1, f2 = phi(x1), phi(x2)
    for _ in range(200):
        if f1 > f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - gr * (hi - lo); f1 = phi(x1)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + gr * (hi - lo); f2 = phi(x2)
    V = max(phi(lo), phi(hi), f1, f2)
    assert abs(r["risk"] - V) < 1e-7 * max(1.0, abs(V))


def test_constrained_solution_diagnostics_vanish():
    """On a constrained AV@R problem: residual, xi1, xi2, primal infeasibility
    and complementarity gap vanish, the risk value equals the nested AV@R of
    the returned trajectory (Eq. original-problem), constraints hold."""
    p = constrained([2, 2, 1], 3, 2, seed=17, avar=0.5)
    o = Oracle(p)
    r = o.solve(tol=1e-7, max_iters=30000, method="spock")
    assert r["res_inf"] <= 1e-7
    assert r["xi1"] < 1e-5 and r["xi2"] < 1e-5
    assert r["infeas"] < 1e-5 and r["gap"] < 1e-4
    assert abs(r["risk"] - r["nested_risk"]) < 1e-5 * abs(r["risk"])
    assert np.all(np.abs(r["x"]) <= 5 + 1e-5) and np.all(np.abs(r["u"]) <= 2 + 1e-5)


# --- constrained AV@R optima by a second method ------------------------------------
def _nested_avar_nlp(p):
    """The risk-averse problem (Sec. 3) with diagonal weights, boxes and a
    ball, solved without the conic reformulation: the dynamics are substituted
    (x^i affine in the stacked inputs U), and every conditional AV@R_a of the
    nested risk is written as min_t t + (1/a) E_p[(Z - t)_+], the LP dual of
    the maximisation over {mu in the simplex : mu <= p/a} (Sec. 3.3-3.4). With
    one t per non-leaf node and one w >= (Z - t)_+ per edge, the problem is the
    smooth convex program

        min t^0 + (1/a^0) sum_{c child of 0} p^c w^c
        s.t. w^c >= l^c(x^i, u^i) + V^c - t^i,  w^c >= 0   (i = anc(c)),
             V^c = t^c + (1/a^c) sum_{d child of c} p^d w^d (non-leaf c),
             V^c = x^c' Q_N x^c (leaf c), boxes on x^1.. and u, ||u^i|| <= r,

    solved by scipy's SLSQP with exact gradients. An l1 term lambda_0 ||z^i||_1
    (z^i = (x^i, u^i)) enters l^c through e^i >= |z^i| (lambda_0 1'e^i); a
    soft-constraint penalty ||max(0, z^i - z_max)||^2 through q^i >= 0,
    q^i >= z^i - z_max (||q^i||^2). With the total-variation risk (worst
    expectation over {mu in the simplex : ||mu - p||_1 <= r}) the LP dual is
    min t + lambda r + p'g over lambda >= 0, |g_c| <= lambda, g_c >= Z_c - t: w
    plays g (free), one lambda per non-leaf node. Returns (value, u, worst
    constraint violation)."""
    n, nx, nu = len(p.anc), p.nx, p.nu
    d = nx + nu
    n_nl = len(p.avar)
    nU = n_nl * nu
    lam = float(p.l1 or 0.0)
    soft = p.soft_max is not None
    tv = p.tv is not None
    wco = np.array([p.prob[c] / (1.0 if tv else p.avar[p.anc[c]]) for c in range(1, n)])   # w's weight in V
    ch = [[] for _ in range(n)]
    for c in range(1, n):
        ch[p.anc[c]].append(c)
    Phi = np.zeros((n, nx, nU))   # x^i = Phi[i] U + phi[i]
    phi = np.zeros((n, nx))
    phi[0] = p.x0
    for c in range(1, n):
        a = p.anc[c]
        Phi[c] = p.A[c - 1] @ Phi[a]
        Phi[c][:, a * nu:(a + 1) * nu] += p.B[c - 1]
        phi[c] = p.A[c - 1] @ phi[a] + p.c[c - 1]
    it, iw = nU, nU + n_nl
    ie = iw + (n - 1)                       # e^i (l1 term), d per non-leaf node
    iq = ie + (n_nl * d if lam > 0 else 0)  # q^i (soft penalty)
    il = iq + (n_nl * d if soft else 0)     # lambda^i (total-variation risk)
    nz = il + (n_nl if tv else 0)

    def zmap(i):   # z^i = Z U + z0
        Z = np.zeros((d, nU))
        Z[:nx] = Phi[i]
        Z[nx:, i * nu:(i + 1) * nu] = np.eye(nu)
        return Z, np.concatenate([phi[i], np.zeros(nu)])

    def quad(W, y):   # y'Wy and its gradient, W full or its diagonal
        Wy = W @ y if W.ndim == 2 else W * y
        return y @ Wy, 2 * Wy

    def edge_cost(z, c):
        a = p.anc[c]
        U = z[:nU]
        x = Phi[a] @ U + phi[a]
        u = U[a * nu:(a + 1) * nu]
        vx, gx = quad(p.Q[c - 1], x)
        vu, gu = quad(p.R[c - 1], u)
        if p.q is not None:   # linear terms q'x + r'u
            vx, gx = vx + p.q[c - 1] @ x, gx + p.q[c - 1]
            vu, gu = vu + p.r[c - 1] @ u, gu + p.r[c - 1]
        g = np.zeros(nz)
        g[:nU] = Phi[a].T @ gx
        g[a * nu:(a + 1) * nu] += gu
        val = vx + vu
        if lam > 0:
            val += lam * np.sum(z[ie + a * d:ie + (a + 1) * d])
            g[ie + a * d:ie + (a + 1) * d] = lam
        if soft:
            q = z[iq + a * d:iq + (a + 1) * d]
            val += q @ q
            g[iq + a * d:iq + (a + 1) * d] = 2 * q
        return val, g

    def obj(z):
        g = np.zeros(nz)
        g[it] = 1.0
        for c in ch[0]:
            g[iw + c - 1] = wco[c - 1]
        if tv:
            g[il] = p.tv[0]
        return float(g @ z), g

    def edges(z):
        U, t, w = z[:nU], z[it:iw], z[iw:ie]
        val = np.zeros(n - 1)
        J = np.zeros((n - 1, nz))
        for c in range(1, n):
            a = p.anc[c]
            lc, gl = edge_cost(z, c)
            J[c - 1] = -gl
            if c < n_nl:
                V = t[c] + sum(wco[k - 1] * w[k - 1] for k in ch[c])
                J[c - 1, it + c] -= 1.0
                for k in ch[c]:
                    J[c - 1, iw + k - 1] -= wco[k - 1]
                if tv:
                    V += p.tv[c] * z[il + c]
                    J[c - 1, il + c] -= p.tv[c]
            else:
                x = Phi[c] @ U + phi[c]
                V, gV = quad(p.QN[c - n_nl], x)
                if p.qN is not None:
                    V, gV = V + p.qN[c - n_nl] @ x, gV + p.qN[c - n_nl]
                J[c - 1, :nU] -= Phi[c].T @ gV
            val[c - 1] = w[c - 1] - lc - V + t[a]
            J[c - 1, iw + c - 1] += 1.0
            J[c - 1, it + a] += 1.0
        return val, J

    cons = [dict(type="ineq", fun=lambda z: edges(z)[0], jac=lambda z: edges(z)[1])]
    rows, rhs = [], []

    def two_sided(a_row, a0, lo, hi):   # lo <= a_row U + a0 <= hi
        r_ = np.zeros(nz); r_[:nU] = -a_row; rows.append(r_); rhs.append(hi - a0)
        r_ = np.zeros(nz); r_[:nU] = a_row; rows.append(r_); rhs.append(a0 - lo)
    if p.x_lo is not None:
        for i in range(1, n):
            for k in range(nx):
                two_sided(Phi[i][k], phi[i][k], p.x_lo[i, k], p.x_hi[i, k])
    if p.Gx is not None:   # general rows at the non-leaf nodes
        for i in range(n_nl):
            Z, z0 = zmap(i)
            Gz = np.hstack([p.Gx, p.Gu])
            for k in range(Gz.shape[0]):
                two_sided(Gz[k] @ Z, Gz[k] @ z0, p.g_lo[i, k], p.g_hi[i, k])
    if p.GN is not None:   # general rows at the leaves
        for j in range(n_nl, n):
            for k in range(p.GN.shape[0]):
                two_sided(p.GN[k] @ Phi[j], p.GN[k] @ phi[j], p.gN_lo[j - n_nl, k], p.gN_hi[j - n_nl, k])
    for i in range(n_nl):
        Z, z0 = zmap(i)
        for k in range(d):
            if lam > 0:   # e - z >= 0, e + z >= 0
                r_ = np.zeros(nz); r_[:nU] = -Z[k]; r_[ie + i * d + k] = 1.0; rows.append(r_); rhs.append(-z0[k])
                r_ = np.zeros(nz); r_[:nU] = Z[k]; r_[ie + i * d + k] = 1.0; rows.append(r_); rhs.append(z0[k])
            if soft:      # q - z + z_max >= 0
                r_ = np.zeros(nz); r_[:nU] = -Z[k]; r_[iq + i * d + k] = 1.0; rows.append(r_)
                rhs.append(p.soft_max[k] - z0[k])
    if tv:   # lambda^a -/+ g_c >= 0
        for c in range(1, n):
            for sg in (-1.0, 1.0):
                r_ = np.zeros(nz); r_[il + p.anc[c]] = 1.0; r_[iw + c - 1] = sg; rows.append(r_); rhs.append(0.0)
    G, h = np.asarray(rows), np.asarray(rhs)
    cons.append(dict(type="ineq", fun=lambda z: G @ z + h, jac=lambda z: G))
    if p.u_ball is not None:
        def ball(z):
            Ui = z[:nU].reshape(n_nl, nu)
            return p.u_ball ** 2 - np.sum(Ui * Ui, axis=1)

        def ball_jac(z):
            J = np.zeros((n_nl, nz))
            for i in range(n_nl):
                J[i, i * nu:(i + 1) * nu] = -2 * z[i * nu:(i + 1) * nu]
            return J
        cons.append(dict(type="ineq", fun=ball, jac=ball_jac))
    bounds = [(None, None)] * nz
    if p.u_lo is not None:
        for i in range(n_nl):
            for k in range(nu):
                bounds[i * nu + k] = (p.u_lo[i, k], p.u_hi[i, k])
    for k in list(range(iw if not tv else ie, ie)) + list(range(iq, nz)):
        bounds[k] = (0.0, None)
    z0 = np.zeros(nz)
    z0[iw:ie] = 100.0
    z0[il:] = 100.0
    r = so.minimize(lambda z: obj(z)[0], z0, jac=lambda z: obj(z)[1], method="SLSQP", bounds=bounds,
                    constraints=cons, options=dict(ftol=1e-15, maxiter=3000))
    viol = max(0.0, -float(np.min(np.concatenate([c_["fun"](r.x) for c_ in cons]))))
    return float(r.fun), r.x[:nU].reshape(n_nl, nu), viol


@pytest.mark.parametrize("case", ["ball", "u_box", "x_box", "l1", "soft", "tv", "general", "deep"])
def test_constrained_avar_optimum_by_nonlinear_program(case):
    """Constrained problems with AV@R levels below 1 (no closed form): the
    oracle's converged risk value s0 and inputs against the same problem solved
    as a smooth nonlinear program (_nested_avar_nlp: the nested AV@R by its
    Rockafellar-Uryasev form, no cones, no preconditioning, no splitting), on
    cases where the Euclidean ball, the input box or the state box is active
    at the optimum."""
    if case == "ball":
        p = constrained([2, 2], 3, 2, seed=17, avar=0.5, uball=0.6)
    elif case == "deep":   # three stages, a non-branching stage between branching ones, AV@R 0.4
        p = constrained([2, 1, 2], 3, 2, seed=19, avar=0.4, uball=0.6)
        p.avar = np.full_like(p.avar, 0.4)
    elif case == "general":   # full weights, linear terms, general rows at non-leaf nodes and leaves, boxes
        p = general([2, 2], 3, 2, seed=23, avar=0.5, dense=True, linear=True, n_g=2, n_gN=1, box=True)
    elif case in ("l1", "soft", "tv"):   # with the ball, AV@R 0.5
        p = constrained([2, 2], 3, 2, seed=17, avar=0.5, uball=0.6)
        if case == "l1":
            p.l1 = 0.4
        elif case == "soft":
            p.soft_max = np.full(p.nx + p.nu, 0.3)
        else:   # total-variation risk of radius 0.4 at every non-leaf node
            p.tv = np.full(len(p.avar), 0.4)
    else:
        a, ubox, xbox = (0.3, 0.9, 1.2) if case == "u_box" else (0.5, 0.9, 1.1)
        p = constrained([2, 2], 3, 2, seed=17, avar=a)
        p.avar = np.full_like(p.avar, a)
        p.u_lo = np.full_like(p.u_lo, -ubox)
        p.u_hi = np.full_like(p.u_hi, ubox)
        p.x_lo, p.x_hi = p.x_lo.copy(), p.x_hi.copy()
        k = np.arange(1, len(p.anc))[:, None]   # a different box at neighbouring nodes
        p.x_lo[1:], p.x_hi[1:] = -xbox - 0.04 * (k % 3), xbox + 0.04 * ((k + 1) % 3)
    val, U, viol = _nested_avar_nlp(p)
    assert viol < 1e-9
    o = Oracle(p)
    r = o.solve(tol=1e-9, max_iters=30000, method="spock")
    assert r["res_inf"] <= 1e-9
    n_nl = len(p.avar)
    if case in ("ball", "tv", "deep"):   # the constraint under test is active at the optimum
        assert np.max(np.linalg.norm(r["u"], axis=1)) >= 0.6 * (1 - 1e-6)
    elif case == "l1":   # some entries sit at the kink of |.|
        assert np.min(np.abs(r["u"])) <= 1e-6
    elif case == "soft":   # the penalty is active
        assert np.max(np.hstack([r["x"][:len(p.avar)], r["u"]])) > 0.3 + 1e-3
    elif case == "general":   # a general row is active at a non-leaf node and at a leaf
        zs = np.hstack([r["x"][:n_nl], r["u"]]) @ np.hstack([p.Gx, p.Gu]).T
        zN = r["x"][n_nl:] @ p.GN.T
        assert np.min(np.minimum(zs - p.g_lo, p.g_hi - zs)) <= 1e-6
        assert np.min(np.minimum(zN - p.gN_lo, p.gN_hi - zN)) <= 1e-6
    elif case == "u_box":
        assert np.max(np.abs(r["u"])) >= 0.9 * (1 - 1e-6)
    else:
        xs = r["x"][1:]
        assert np.any((xs >= p.x_hi[1:] - 1e-6) | (xs <= p.x_lo[1:] + 1e-6))
    assert abs(r["risk"] - val) <= 1e-7 * abs(val)
    # inputs on the nodes the maximising AV@R weights reach (elsewhere the
    # optimal inputs need not be unique)
    sel = o.path_weights(r["x"], r["u"])[:n_nl] > 1e-9
    assert sel[0] and np.max(np.abs(r["u"][sel] - U[sel])) <= 1e-6


# --- preconditioning (Sec. 5.4), values worked out by hand ----------------------
def _golden_precond():
    return json.load(open(os.path.join(GOLDEN, "precondition_tiny.json")))


@pytest.mark.parametrize("case", ["branchy", "chain"])
def test_preconditioning_hand_values(case):
    """c_hat, S^x, S^u, S^x_N, a_con, the scaled dynamics at a non-leaf and a
    leaf node, the scaled cost factors, x0 and the scaled sets against values
    derived by hand from the formulas of Sec. 5.4 (tests/golden)."""
    from tests.problems import from_spec
    spec = _golden_precond()[case]
    o = Oracle(from_spec(spec))
    ex = spec["expect"]
    chk = lambda got, key: np.testing.assert_allclose(np.asarray(got, dtype=float),  # noqa: E731
                                                      np.asarray(ex[key]["value"], dtype=float),
                                                      rtol=1e-14, atol=1e-15, err_msg=key)
    chk(o.c_hat, "c_hat"); chk(o.Sx, "Sx"); chk(o.Su, "Su"); chk(o.SxN, "SxN")
    chk(o.a_con, "a_con"); chk(o.a_conN, "a_conN")
    nx = spec["nx"]
    if case == "branchy":
        chk(o.At[3], "At_node4"); chk(o.At[7], "At_node8")
        chk(o.Bt[3], "Bt_node4"); chk(o.Bt[7], "Bt_node8")
        chk(o.Qh[7], "Qh_node8"); chk(o.Rh[7], "Rh_node8"); chk(o.QNh[0], "QNh_leaf8")
        chk(o.x0s, "x0s")
        chk(o.box_hi[0], "box_hi_node0")
        chk(o.ball_r[0], "ball_r")
    else:
        nb = o.n_box
        row = np.concatenate([o.Gx[nb], o.Gu[nb]])
        chk(row, "Gu_ball_row0")
        chk(o.box_hi[0], "box_hi_node0")
        chk(o.ball_r[0], "ball_r")
        chk(o.boxN_hi[0], "boxN_hi")
        assert o.Gx.shape == (2 * spec["nu"] + nx, nx)


# --- the Euclidean ball of S3 --------------------------------------------------------
def test_proj_ball_outside_points_closed_form():
    """Projection on {||w|| <= r}: points outside go to r w/||w||, points inside
    stay (hand values: (3, 4) with r = 1 -> (0.6, 0.8), with r = 2.5 ->
    (1.5, 2.0); (0.3, 0.4) and 0 unchanged for r = 1)."""
    got = so_.proj_ball(np.array([[3.0, 4.0], [3.0, 4.0], [0.3, 0.4], [0.0, 0.0]]),
                        np.array([1.0, 2.5, 1.0, 1.0]))
    np.testing.assert_allclose(got, [[0.6, 0.8], [1.5, 2.0], [0.3, 0.4], [0.0, 0.0]], rtol=1e-15, atol=0)


def test_S3_ball_block_projection_and_support():
    """The ball rows of S3 (Eq. S3-def): an eta that is zero except for the u
    ball rows of node 0 projects onto the ball of radius 3/sqrt(2) (chain
    golden problem, a_con = sqrt(2)), and the support function of S3 there
    is r ||eta_ball|| (hand values)."""
    from tests.problems import from_spec
    o = Oracle(from_spec(_golden_precond()["chain"]))
    lay = o.lay
    eta = np.zeros(lay.n_eta)
    base = lay.e_c + o.n_box                  # node 0's ball rows
    eta[base:base + 2] = [3.0, 4.0]
    # keep every translated SOC block at its apex a = (0.., 1/2, -1/2) so it is fixed
    w = o.nx + o.nu + 2
    for c in range(1, o.tree.n):
        eta[lay.e_q + (c - 1) * w + w - 2] = 0.5
        eta[lay.e_q + (c - 1) * w + w - 1] = -0.5
    for j in range(o.tree.n_l):
        eta[lay.e_qN + j * (o.nx + 2) + o.nx] = 0.5
        eta[lay.e_qN + j * (o.nx + 2) + o.nx + 1] = -0.5
    p = o.proj_S3(eta)
    r = 3.0 / math.sqrt(2.0)
    np.testing.assert_allclose(p[base:base + 2], [0.6 * r, 0.8 * r], rtol=1e-15)
    assert np.array_equal(np.delete(p, [base, base + 1]), np.delete(eta, [base, base + 1]))
    # support: ball term r * 5; each apex block contributes <eta, a> = 1/4 + 1/4 = 1/2
    n_soc = (o.tree.n - 1) + o.tree.n_l
    assert abs(o.support_S3(eta) - (5.0 * r + 0.5 * n_soc)) < 1e-13


def test_constrained_solution_diagnostics_vanish_with_ball():
    """As test_constrained_solution_diagnostics_vanish with an active Euclidean
    ball on u, so the ball term of the support function of S3 enters the
    complementarity gap."""
    p = constrained([2, 2, 1], 3, 2, seed=17, avar=0.5, uball=0.6)
    o = Oracle(p)
    r = o.solve(tol=1e-7, max_iters=60000, method="spock")
    assert r["res_inf"] <= 1e-7
    assert np.max(np.linalg.norm(r["u"], axis=1)) >= 0.6 * (1 - 1e-4)   # the ball is active
    assert np.all(np.linalg.norm(r["u"], axis=1) <= 0.6 * (1 + 1e-5))
    assert r["xi1"] < 1e-5 and r["xi2"] < 1e-5
    assert r["infeas"] < 1e-5 and r["gap"] < 1e-4
    assert abs(r["risk"] - r["nested_risk"]) < 1e-5 * abs(r["risk"])


# --- Alg. 4 branch logic on hand-worked maps ---------------------------------------
class _Affine2D(Oracle):
    """Alg. 4 run on a 2-D map instead of the CP operator: Oracle.solve only
    needs T, the M-inner product (here the Euclidean one, M = I) and a start."""

    def __init__(self, T, v0):
        self._T = T
        self._v0 = np.asarray(v0, dtype=np.float64)

    def T(self, v):
        return self._T(v)

    def initial_v(self):
        return self._v0.copy()

    def M_inner(self, a, b):
        return float(a @ b)

    def _result(self, v, tv, iters, n_T, events):
        return dict(v=v, Tv=tv, iters=iters, n_T=n_T, events=events)


def test_supermann_branches_on_averaged_rotation():
    """T = (I + R_theta)/2 (firmly nonexpansive, fixed point 0), theta = 10
    degrees, v0 = (1, 0). With s = sin(theta/2), c = cos(theta/2), worked out by
    hand (Alg. 4, psi = -r while k <= m):
      k=0: omega = zeta = s, so no K0; v~ = T(v0) has residual s c, ratio
           c = 0.9962 > c1, so no K1; rho = ||r~||^2 + <r~, r> = 2 s^2 c^2
           >= sigma s^2 c, so K2: v1 = v0 - (rho/||r~||^2) r~ = v0 - 2 r~ =
           cos(theta) R v0;
      k=1: omega = s cos(theta) <= 0.99 zeta (cos 10 deg = 0.985), K0:
           v2 = T(v1), zeta = s cos(theta);
      k=2: omega/zeta = c > 0.99: no K0; K1 fails on the ratio c again; K2:
           v3 = cos(theta) R v2;
      k=3: omega/zeta = c cos(theta) = 0.981 <= 0.99: K0, v4 = T(v3).
    T evaluations: 1 + 2 + 1 + 2 + 1 = 7."""
    th = math.radians(10.0)
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Tm = 0.5 * (np.eye(2) + Rm)
    o = _Affine2D(lambda v: Tm @ v, [1.0, 0.0])
    r = o.solve(tol=0.0, max_iters=4)
    assert [e[1] for e in r["events"]] == ["K2", "K0", "K2", "K0"]
    assert [e[2] for e in r["events"]] == [0, 0, 0, 0]
    assert r["n_T"] == 7
    v1 = math.cos(th) * Rm @ np.array([1.0, 0.0])
    v2 = Tm @ v1
    v3 = math.cos(th) * Rm @ v2
    v4 = Tm @ v3
    np.testing.assert_allclose(r["v"], v4, rtol=1e-13, atol=1e-15)


def test_supermann_k1_then_k0_on_half_map():
    """T(v) = v/2 (firmly nonexpansive). k=0: omega = zeta, no K0; v~ = T(v0)
    halves the residual (0.5 <= c1) and omega <= omega_safe = zeta: K1, and
    omega_safe becomes ||r~|| + c2^0. k=1..3: each residual is half the last,
    below 0.99 zeta: K0. T evaluations 1 + 1 + 3 = 5; v4 = v0/16."""
    o = _Affine2D(lambda v: 0.5 * v, [4.0, -2.0])
    r = o.solve(tol=0.0, max_iters=4)
    assert [e[1] for e in r["events"]] == ["K1", "K0", "K0", "K0"]
    assert r["n_T"] == 5
    np.testing.assert_allclose(r["v"], np.array([4.0, -2.0]) / 16.0, rtol=1e-15)


# --- quadratic-plus-linear costs, full weights, general constraint rows ----------
def _qp_interior_point(Pq, qq, Gq, hq, tol=1e-12, iters=300):
    """min 1/2 u'Pq u + qq'u s.t. Gq u <= hq by a primal-dual interior-point
    method with Mehrotra's predictor-corrector (slacks s, multipliers z):
    Newton steps on Pq u + qq + Gq'z = 0, Gq u + s = hq, s z = sigma mu."""
    n, m = Pq.shape[0], Gq.shape[0]
    u = np.zeros(n)
    s_ = np.maximum(hq - Gq @ u, 1.0)
    z = np.ones(m)
    sd = 1.0 + np.max(np.abs(qq))
    sp = 1.0 + np.max(np.abs(hq))
    for _ in range(iters):
        rd = Pq @ u + qq + Gq.T @ z
        rp = Gq @ u + s_ - hq
        mu = s_ @ z / m
        if np.max(np.abs(rd)) < tol * sd and np.max(np.abs(rp)) < tol * sp and mu < tol * sd * sp:
            return u
        Kmat = Pq + Gq.T @ ((z / s_)[:, None] * Gq)

        def step(rc):
            du = np.linalg.solve(Kmat, -rd - Gq.T @ ((z / s_) * rp) + Gq.T @ (rc / s_))
            dz = (z / s_) * (Gq @ du + rp) - rc / s_
            ds = -(rc + s_ * dz) / z
            return du, ds, dz

        def maxstep(x, dx):
            neg = dx < 0
            return min(1.0, float(np.min(-x[neg] / dx[neg]))) if np.any(neg) else 1.0

        du, ds, dz = step(s_ * z)
        a_aff = min(maxstep(s_, ds), maxstep(z, dz))
        mu_aff = (s_ + a_aff * ds) @ (z + a_aff * dz) / m
        sigma = (mu_aff / mu) ** 3
        du, ds, dz = step(s_ * z + ds * dz - sigma * mu)
        a = 0.99 * min(maxstep(s_, ds), maxstep(z, dz))
        u, s_, z = u + a * du, s_ + a * ds, z + a * dz
    raise AssertionError("interior point did not converge")


def _risk_neutral_qp_general(p):
    """min sum_c pi^c l^c(x^a, u^a) + sum_j pi^j l_N^j(x^j) with the full
    quadratic-plus-linear costs of Sec. 3.2, s.t. the dynamics and x^0 = x0
    (equalities) and the general rows g_lo <= Gx x + Gu u <= g_hi,
    gN_lo <= GN x <= gN_hi (inequalities): solved as one dense QP, by a KKT
    solve without inequalities, else by SLSQP. Returns (value, x, u)."""
    tr = so_.Tree(p.anc, p.prob)
    nx, nu, n = p.nx, p.nu, tr.n
    nX = n * nx + tr.n_nl * nu
    H = np.zeros((nX, nX))
    f = np.zeros(nX)
    full = lambda W, k: W[k] if np.ndim(W) == 3 else np.diag(W[k])   # noqa: E731
    for c in range(1, n):
        a = tr.anc[c]
        H[a * nx:(a + 1) * nx, a * nx:(a + 1) * nx] += tr.pi[c] * full(p.Q, c - 1)
        o = n * nx + a * nu
        H[o:o + nu, o:o + nu] += tr.pi[c] * full(p.R, c - 1)
        if p.q is not None:
            f[a * nx:(a + 1) * nx] += tr.pi[c] * p.q[c - 1]
        if p.r is not None:
            f[o:o + nu] += tr.pi[c] * p.r[c - 1]
    for jj in range(tr.n_l):
        j = tr.n_nl + jj
        H[j * nx:(j + 1) * nx, j * nx:(j + 1) * nx] += tr.pi[j] * full(p.QN, jj)
        if p.qN is not None:
            f[j * nx:(j + 1) * nx] += tr.pi[j] * p.qN[jj]
    rows, rhs = [], []
    C0 = np.zeros((nx, nX)); C0[:, :nx] = np.eye(nx); rows.append(C0); rhs.append(p.x0)
    for c in range(1, n):
        a = tr.anc[c]
        Cc = np.zeros((nx, nX))
        Cc[:, c * nx:(c + 1) * nx] = np.eye(nx)
        Cc[:, a * nx:(a + 1) * nx] = -p.A[c - 1]
        Cc[:, n * nx + a * nu:n * nx + (a + 1) * nu] = -p.B[c - 1]
        rows.append(Cc); rhs.append(p.c[c - 1])
    C = np.vstack(rows)
    d = np.concatenate(rhs)
    G, lo, hi = [], [], []
    if p.Gx is not None:
        for i in range(tr.n_nl):
            Gi = np.zeros((p.Gx.shape[0], nX))
            Gi[:, i * nx:(i + 1) * nx] = p.Gx
            Gi[:, n * nx + i * nu:n * nx + (i + 1) * nu] = p.Gu
            G.append(Gi); lo.append(p.g_lo[i]); hi.append(p.g_hi[i])
    if p.GN is not None:
        for jj in range(tr.n_l):
            j = tr.n_nl + jj
            Gj = np.zeros((p.GN.shape[0], nX))
            Gj[:, j * nx:(j + 1) * nx] = p.GN
            G.append(Gj); lo.append(p.gN_lo[jj]); hi.append(p.gN_hi[jj])
    K = np.block([[2 * H, C.T], [C, np.zeros((C.shape[0], C.shape[0]))]])
    X = np.linalg.solve(K, np.concatenate([-f, d]))[:nX]
    if G:
        G = np.vstack(G); lo = np.concatenate(lo); hi = np.concatenate(hi)
        # eliminate the dynamics: X = Pm u + p0 (forward simulation from x0)
        nU = tr.n_nl * nu
        Pm = np.zeros((nX, nU)); p0 = np.zeros(nX)
        Pm[n * nx:, :] = np.eye(nU)
        p0[:nx] = p.x0
        for c in range(1, n):
            a = tr.anc[c]
            Pm[c * nx:(c + 1) * nx] = p.A[c - 1] @ Pm[a * nx:(a + 1) * nx]
            Pm[c * nx:(c + 1) * nx, a * nu:(a + 1) * nu] += p.B[c - 1]
            p0[c * nx:(c + 1) * nx] = p.A[c - 1] @ p0[a * nx:(a + 1) * nx] + p.c[c - 1]
        Hu = Pm.T @ H @ Pm
        fu = Pm.T @ (2 * H @ p0 + f)
        Gu_, g0 = G @ Pm, G @ p0
        u = _qp_interior_point(2 * Hu, fu, np.vstack([Gu_, -Gu_]), np.concatenate([hi - g0, g0 - lo]))
        X = Pm @ u + p0
    return float(X @ H @ X + f @ X), X[:n * nx].reshape(n, nx), X[n * nx:].reshape(tr.n_nl, nu)


def test_prop1_translation_with_linear_term_is_the_epigraph():
    """Prop. 1 (Q positive definite, S = I): (z, tau) is in the epigraph of
    z'Qz + q'z exactly when (F z, tau/2, tau/2) minus the oracle's translation
    a lies in the second-order cone, for the scaled factor F that L applies to
    the scaled variables (Sec. 5.4 scalings included). Checked on random
    points just above and just below the epigraph's boundary, edge costs and
    terminal costs."""
    p = general([2, 1], 3, 2, seed=51)
    o = Oracle(p)
    rng = np.random.default_rng(52)
    inside = lambda v: np.linalg.norm(v[:-1]) <= v[-1]   # noqa: E731
    for c in range(1, o.tree.n):
        a = o.tree.anc[c]
        S = o.Snode[a]
        for _ in range(20):
            x, u = rng.standard_normal(p.nx), rng.standard_normal(p.nu)
            ell = o.edge_cost(c, x, u)
            for tau, want in ((ell + 1e-6 * (1 + abs(ell)), True), (ell - 1e-6 * (1 + abs(ell)), False)):
                v = np.concatenate([o.Qh[c - 1] @ (S * x), o.Rh[c - 1] @ (o.Su * u), [tau / 2, tau / 2]])
                assert inside(v - o.a_q[c - 1]) == want
    for jj in range(o.tree.n_l):
        for _ in range(20):
            x = rng.standard_normal(p.nx)
            ell = o.terminal_cost(jj, x)
            for s_, want in ((ell + 1e-6 * (1 + abs(ell)), True), (ell - 1e-6 * (1 + abs(ell)), False)):
                v = np.concatenate([o.QNh[jj] @ (o.SxN * x), [s_ / 2, s_ / 2]])
                assert inside(v - o.a_qN[jj]) == want


def _check_on_likely_nodes(o, r, X, U, tol, pmin=0.05):
    """x and u of the nodes whose path probability is at least pmin (a node
    of probability ~0 barely enters the risk-neutral objective, so its
    trajectory converges far more slowly than the value)."""
    pi = o.tree.pi
    sel = pi >= pmin
    assert np.max(np.abs(r["x"][sel] - X[sel])) < tol
    seln = sel[:o.tree.n_nl]
    assert np.max(np.abs(r["u"][seln] - U[seln])) < tol


def test_risk_neutral_full_weights_linear_terms_kkt():
    """AV@R_1, no constraints, full Q, R, Q_N and linear terms q, r, q_N: the
    oracle's SPOCK solution equals the dense KKT solution of the risk-neutral
    QP (value; trajectory on the likely nodes)."""
    p = general([2, 2, 1], 3, 2, seed=53)
    o = Oracle(p)
    r = o.solve(tol=1e-9, max_iters=20000)
    V, X, U = _risk_neutral_qp_general(p)
    assert abs(r["risk"] - V) < 1e-7 * max(1.0, abs(V))
    _check_on_likely_nodes(o, r, X, U, 1e-5)


def test_risk_neutral_general_rows_vs_qp_solver():
    """AV@R_1 with general rows at every node (Eq. constraints with dense
    Gamma_x, Gamma_u, Gamma_N and box sets), full weights and linear terms:
    the oracle's solution equals the convex QP solved by SLSQP; some rows are
    active."""
    p = general([2, 2, 1], 3, 2, seed=54, n_g=2, n_gN=1, g_scale=0.4)
    o = Oracle(p)
    r = o.solve(tol=1e-9, max_iters=30000)
    V, X, U = _risk_neutral_qp_general(p)
    assert abs(r["risk"] - V) < 1e-6 * max(1.0, abs(V))
    _check_on_likely_nodes(o, r, X, U, 1e-4)
    tr = o.tree
    gx = np.array([p.Gx @ r["x"][i] + p.Gu @ r["u"][i] for i in range(tr.n_nl)])
    act = np.isclose(gx, p.g_lo, atol=1e-6) | np.isclose(gx, p.g_hi, atol=1e-6)
    assert act.any()


def test_general_problem_diagnostics_vanish():
    """AV@R 0.5 with full weights, linear terms, boxes and general rows: the
    residual, xi1, xi2, infeasibility and the complementarity gap (with the
    support function of the translated cones and the general rows) vanish, and
    s0 equals the nested risk of the trajectory with the linear costs."""
    p = general([2, 2, 1], 3, 2, seed=55, avar=0.5, n_g=2, n_gN=1, box=True, g_scale=0.5)
    o = Oracle(p)
    r = o.solve(tol=1e-8, max_iters=30000)
    assert r["res_inf"] <= 1e-8
    assert r["xi1"] < 1e-5 and r["xi2"] < 1e-5
    assert r["infeas"] < 1e-6 and r["gap"] < 1e-5
    assert abs(r["risk"] - r["nested_risk"]) < 1e-5 * max(1.0, abs(r["risk"]))


# --- Anderson least squares with an updated QR factorisation (Sec. 6.2) ---------------
def test_aa_qr_update_matches_a_fresh_least_squares_solve():
    """The QR memory (Givens rotations to drop the oldest pair, Gram-Schmidt
    to append) keeps Y = QR with Q orthonormal and R upper triangular through
    many pushes, and its direction equals -r - (S - Y) kappa with kappa from a
    fresh least-squares solve (numpy lstsq) of the last m pairs."""
    rng = np.random.default_rng(81)
    n, m = 40, 3
    mem = Oracle.QRMemory(m)
    S, Y = [], []
    for it in range(12):
        s_, y = rng.standard_normal(n), rng.standard_normal(n)
        mem.push(s_, y)
        S.append(s_); Y.append(y)
        S, Y = S[-m:], Y[-m:]
        Ym = np.column_stack(Y)
        assert np.allclose(mem.Q @ mem.R, Ym, atol=1e-12)
        assert np.allclose(mem.Q.T @ mem.Q, np.eye(len(Y)), atol=1e-12)
        assert np.allclose(np.tril(mem.R, -1), 0.0)
        r = rng.standard_normal(n)
        kappa = np.linalg.lstsq(Ym, r, rcond=None)[0]
        want = -r - (np.column_stack(S) - Ym) @ kappa
        got = mem.direction(r, k=it + m + 1)
        assert np.allclose(got, want, atol=1e-10)


def test_spock_with_qr_update_follows_the_same_branches():
    """SPOCK with the updated QR and with a fresh Householder factorisation
    take the same K0/K1/K2 branches and reach the same iterate (FP64, a fixed
    iteration count; the two factorisations differ only by rounding)."""
    p = constrained([2, 2, 1], 3, 2, seed=82, avar=0.5, uball=2.0)
    o = Oracle(p)
    a = o.solve(tol=0.0, max_iters=60)
    b = o.solve(tol=0.0, max_iters=60, aa="qr_update")
    assert [e[1] for e in a["events"]] == [e[1] for e in b["events"]]
    assert a["n_T"] == b["n_T"]
    assert np.max(np.abs(a["v"] - b["v"])) < 1e-9 * max(1.0, np.max(np.abs(a["v"])))


# --- l1 stage costs (Prop. 2) ------------------------------------------------------------


def _l1_problem(seed, avar=1.0, box=False, lam=0.3, ball=None):
    p = general([2, 2, 1], 3, 2, seed=seed, avar=avar, box=box)
    p.l1 = lam
    if ball is not None:
        p.u_ball = np.full(p.n_nonleaf, ball)
    return p


def test_l1_rows_encode_prop2_epigraph():
    """Prop. 2: (z, tau) lies in the epigraph of z'Qz + q'z + lambda_0 ||z||_1
    exactly when some theta, lambda with sum lambda <= theta and
    -lambda <= z <= lambda put (z, tau - lambda_0 theta) in the epigraph of the
    quadratic part. With theta = ||z||_1 and lambda = |z| (the smallest
    choice), the rows L gives the child's cost cone and the parent's l1 block
    lie in S3 exactly when the full cost is at most tau; with theta below
    ||z||_1 no lambda satisfies the l1 rows."""
    p = _l1_problem(61)
    o = Oracle(p)
    tr, lay = o.tree, o.lay
    nx, nu, d = o.nx, o.nu, o.nx + o.nu
    rng = np.random.default_rng(3)
    i = 1
    c = tr.children[i][0]
    sc = np.concatenate([o.Snode[i], o.Su])
    for trial in range(40):
        x = rng.standard_normal(nx)
        u = rng.standard_normal(nu)
        cost = o.edge_cost(c, x, u)
        tau = cost + rng.uniform(-0.5, 0.5)
        z = np.zeros(lay.n_z)
        z[lay.o_x + i * nx:lay.o_x + (i + 1) * nx] = o.Snode[i] * x
        z[lay.o_u + i * nu:lay.o_u + (i + 1) * nu] = o.Su * u
        z[lay.o_tau + c - 1] = tau
        zu = np.concatenate([x, u])
        z[o.o_th + i] = np.sum(np.abs(zu))
        z[o.o_lam + i * d:o.o_lam + (i + 1) * d] = sc * np.abs(zu)
        Lz = o.apply_L(z)
        P3 = o.proj_S3(Lz)
        w = nx + nu + 2
        cone = slice(lay.e_q + (c - 1) * w, lay.e_q + c * w)
        rows = slice(o.e_l1 + i * (1 + 2 * d), o.e_l1 + (i + 1) * (1 + 2 * d))
        inside = np.allclose(P3[cone], Lz[cone], atol=1e-12) and np.allclose(P3[rows], Lz[rows], atol=1e-12)
        assert inside == (cost <= tau), (trial, cost, tau)
        # theta below ||z||_1: the first l1 row is negative for the smallest lambda
        z[o.o_th + i] = 0.9 * np.sum(np.abs(zu))
        assert o.apply_L(z)[o.e_l1 + i * (1 + 2 * d)] < 0


def _risk_neutral_l1_qp(p):
    """min sum_c pi^c l^c + sum_j pi^j l_N^j with l^c = x'Qx + u'Ru + q'x + r'u
    + lambda_0 ||(x, u)||_1 on the ancestor's (x, u), s.t. the dynamics and
    x^0 = x0: the l1 term of node i's children weighs pi^i; written with
    t^i >= |(x^i, u^i)| as a QP in (u, t) after eliminating the dynamics and
    solved by the interior-point method above. Returns (value, x, u)."""
    tr = so_.Tree(p.anc, p.prob)
    nx, nu, n = p.nx, p.nu, tr.n
    nX = n * nx + tr.n_nl * nu
    H = np.zeros((nX, nX))
    f = np.zeros(nX)
    full = lambda W, k: W[k] if np.ndim(W) == 3 else np.diag(W[k])   # noqa: E731
    for c in range(1, n):
        a = tr.anc[c]
        H[a * nx:(a + 1) * nx, a * nx:(a + 1) * nx] += tr.pi[c] * full(p.Q, c - 1)
        o = n * nx + a * nu
        H[o:o + nu, o:o + nu] += tr.pi[c] * full(p.R, c - 1)
        if p.q is not None:
            f[a * nx:(a + 1) * nx] += tr.pi[c] * p.q[c - 1]
        if p.r is not None:
            f[o:o + nu] += tr.pi[c] * p.r[c - 1]
    for jj in range(tr.n_l):
        j = tr.n_nl + jj
        H[j * nx:(j + 1) * nx, j * nx:(j + 1) * nx] += tr.pi[j] * full(p.QN, jj)
        if p.qN is not None:
            f[j * nx:(j + 1) * nx] += tr.pi[j] * p.qN[jj]
    nU = tr.n_nl * nu
    Pm = np.zeros((nX, nU)); p0 = np.zeros(nX)
    Pm[n * nx:, :] = np.eye(nU)
    p0[:nx] = p.x0
    for c in range(1, n):
        a = tr.anc[c]
        Pm[c * nx:(c + 1) * nx] = p.A[c - 1] @ Pm[a * nx:(a + 1) * nx]
        Pm[c * nx:(c + 1) * nx, a * nu:(a + 1) * nu] += p.B[c - 1]
        p0[c * nx:(c + 1) * nx] = p.A[c - 1] @ p0[a * nx:(a + 1) * nx] + p.c[c - 1]
    d = nx + nu
    nT = tr.n_nl * d
    Sel = np.zeros((nT, nX))                    # z^i = (x^i, u^i) for every non-leaf node
    wt = np.zeros(nT)
    for i in range(tr.n_nl):
        Sel[i * d:i * d + nx, i * nx:(i + 1) * nx] = np.eye(nx)
        Sel[i * d + nx:(i + 1) * d, n * nx + i * nu:n * nx + (i + 1) * nu] = np.eye(nu)
        wt[i * d:(i + 1) * d] = p.l1 * tr.pi[i]
    Hw = np.zeros((nU + nT, nU + nT))
    Hw[:nU, :nU] = 2 * Pm.T @ H @ Pm
    fw = np.concatenate([Pm.T @ (2 * H @ p0 + f), wt])
    Zu = Sel @ Pm
    G = np.vstack([np.hstack([Zu, -np.eye(nT)]), np.hstack([-Zu, -np.eye(nT)])])
    h = np.concatenate([-Sel @ p0, Sel @ p0])
    wsol = _qp_interior_point(Hw, fw, G, h)
    X = Pm @ wsol[:nU] + p0
    val = float(X @ H @ X + f @ X + wt @ np.abs(Sel @ X))
    return val, X[:n * nx].reshape(n, nx), X[n * nx:].reshape(tr.n_nl, nu)


def test_risk_neutral_l1_costs_vs_qp():
    """AV@R_1, no constraints, full weights, linear terms and an l1 term
    lambda_0 ||(x, u)||_1 in every edge cost (Prop. 2): the oracle's SPOCK
    solution equals the QP with t >= |(x, u)| (value; trajectory on the likely
    nodes); the l1 term is strong enough that some inputs sit at zero."""
    p = _l1_problem(62, lam=0.8)
    o = Oracle(p)
    r = o.solve(tol=1e-9, max_iters=40000)
    V, X, U = _risk_neutral_l1_qp(p)
    assert abs(r["risk"] - V) < 1e-6 * max(1.0, abs(V))
    _check_on_likely_nodes(o, r, X, U, 1e-4)
    assert np.any(np.abs(U) < 1e-6)


def test_l1_problem_diagnostics_vanish():
    """AV@R 0.5 with boxes, a ball, full weights, linear terms and l1 costs: the
    residual, xi1, xi2, infeasibility and the complementarity gap vanish, and
    s0 equals the nested risk of the trajectory with the l1 costs."""
    p = _l1_problem(63, avar=0.5, box=True, lam=0.4, ball=1.5)
    o = Oracle(p)
    r = o.solve(tol=1e-8, max_iters=40000)
    assert r["res_inf"] <= 1e-8
    assert r["xi1"] < 1e-5 and r["xi2"] < 1e-5
    assert r["infeas"] < 1e-6 and r["gap"] < 1e-5
    assert abs(r["risk"] - r["nested_risk"]) < 1e-5 * max(1.0, abs(r["risk"]))


# --- a conic risk with F != 0: the total-variation ball (Sec. 3.3) ----------------------


def _with_tv(p, r):
    p.tv = np.full(p.n_nonleaf, float(r))
    return p


@pytest.mark.parametrize("seed", range(6))
def test_tv_risk_vs_lp_and_conic_primal_and_dual(seed):
    """The closed form of the total-variation risk = max mu'Z over the ball
    (LP in (mu, nu)) = the conic primal max{mu'Z : b - E mu - F nu in K} with
    the b, E, F of conic_risk_data_tv = the conic dual min{y'b : E'y = Z,
    F'y = 0, y in K*} (Eq. primal_risk and dual_risk, F != 0)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 6))
    Z = rng.standard_normal(n)
    p = rng.dirichlet(np.ones(n))
    r = float(rng.choice([0.0, rng.uniform(0.05, 1.0), 2.5]))
    val = so_.tv_risk(Z, p, r)
    # LP: max mu'Z, sum mu = 1, mu >= 0, -nu <= mu - p <= nu, sum nu <= r
    c = np.concatenate([-Z, np.zeros(n)])
    A_ub = np.vstack([np.hstack([np.eye(n), -np.eye(n)]), np.hstack([-np.eye(n), -np.eye(n)]),
                      np.concatenate([np.zeros(n), np.ones(n)])[None, :]])
    b_ub = np.concatenate([p, -p, [r]])
    lp = so.linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=np.concatenate([np.ones(n), np.zeros(n)])[None, :],
                    b_eq=[1.0], bounds=[(0, None)] * n + [(None, None)] * n, method="highs")
    assert lp.status == 0 and abs(-lp.fun - val) < 1e-10
    b, E, F, npos = so_.conic_risk_data_tv(p, r)
    # conic primal: b - E mu - F nu >= 0 on the first npos rows, = 0 on the last
    Ak = np.hstack([E, F])
    prim = so.linprog(np.concatenate([-Z, np.zeros(n)]), A_ub=Ak[:npos], b_ub=b[:npos],
                      A_eq=Ak[npos:], b_eq=b[npos:], bounds=[(None, None)] * (2 * n), method="highs")
    assert prim.status == 0 and abs(-prim.fun - val) < 1e-9
    dual = so.linprog(b, A_eq=np.vstack([E.T, F.T]), b_eq=np.concatenate([Z, np.zeros(n)]),
                      bounds=[(0, None)] * npos + [(None, None)] * (len(b) - npos), method="highs")
    assert dual.status == 0 and abs(dual.fun - val) < 1e-9
    assert abs(so_.tv_risk(Z, p, 0.0) - p @ Z) < 1e-14
    assert abs(so_.tv_risk(Z, p, 2.0) - Z.max()) < 1e-14


def test_proj_S2_with_F_vs_nullspace_basis():
    """With the total-variation risk S2^i = ker[E', -I, -I; F', 0, 0]: the
    projection equals N N' v for an orthonormal basis N of that kernel (SVD)."""
    p = _with_tv(constrained([3, 2, 1], 2, 1, seed=5, avar=0.5), 0.6)
    o = Oracle(p)
    rng = np.random.default_rng(6)
    z = rng.standard_normal(o.lay.n_z)
    s0, x, u, y, tau, s = o.split_z(z)
    y2, tau2, s2 = o.proj_S2(y, tau, s)
    tr = o.tree
    for i in range(tr.n_nl):
        ch = tr.children[i]
        m = len(ch)
        I, O = np.eye(m), np.zeros((m, m))
        Et = np.hstack([I, -I, np.zeros((m, 1)), -I, np.ones((m, 1))])     # E'
        Ft = np.hstack([-I, -I, np.ones((m, 1)), O, np.zeros((m, 1))])     # F'
        G = np.vstack([np.hstack([Et, -I, -I]), np.hstack([Ft, O, O])])
        Nb = sla.null_space(G)
        v = np.concatenate([y[o.yoff[i]:o.yoff[i + 1]], tau[ch - 1], s[ch - 1]])
        got = np.concatenate([y2[o.yoff[i]:o.yoff[i + 1]], tau2[ch - 1], s2[ch - 1]])
        assert np.allclose(got, Nb @ (Nb.T @ v), atol=1e-12)


def test_tv_radius_zero_is_risk_neutral_qp():
    """A total-variation ball of radius 0 is the expectation: the oracle's
    solution with the tv risk equals the risk-neutral QP (value; trajectory on
    the likely nodes), through the y-blocks, S2 with F and the zero cone."""
    p = _with_tv(general([2, 2, 1], 3, 2, seed=57), 0.0)
    o = Oracle(p)
    r = o.solve(tol=1e-9, max_iters=40000)
    V, X, U = _risk_neutral_qp_general(p)
    assert abs(r["risk"] - V) < 1e-7 * max(1.0, abs(V))
    _check_on_likely_nodes(o, r, X, U, 1e-5)


def test_one_stage_two_children_tv_bruteforce():
    """N = 1, two children, total-variation radius 0.5, no constraints:
    V* = max over the ball (a segment mu_1 in [p_1 - r/2, p_1 + r/2]) of the
    inner LQ minimum, by golden section."""
    p = _with_tv(unconstrained([2], 2, 2, seed=16, avar=1.0), 0.5)
    o = Oracle(p)
    r = o.solve(tol=1e-10, max_iters=50000, method="spock")
    x0 = p.x0
    pr = p.prob[1:]

    def phi(m1):
        mu = np.array([m1, 1 - m1])
        H = np.zeros((p.nu, p.nu)); g = np.zeros(p.nu); const = 0.0
        for j in range(2):
            A, B = p.A[j], p.B[j]
            QN = np.diag(p.QN[j])
            H += mu[j] * (np.diag(p.R[j]) + B.T @ QN @ B)
            g += mu[j] * (B.T @ QN @ A @ x0)
            const += mu[j] * (x0 @ np.diag(p.Q[j]) @ x0 + (A @ x0) @ QN @ (A @ x0))
        u = -np.linalg.solve(H, g)
        return u @ H @ u + 2 * g @ u + const

    lo, hi = max(0.0, pr[0] - 0.25), min(1.0, pr[0] + 0.25)
    gr = (math.sqrt(5) - 1) / 2
    x1, x2 = hi - gr * (hi - lo), lo + gr * (hi - lo)
    f1, f2 = phi(x1), phi(x2)
    for _ in range(200):
        if f1 > f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - gr * (hi - lo); f1 = phi(x1)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + gr * (hi - lo); f2 = phi(x2)
    V = max(phi(lo), phi(hi), f1, f2)
    assert abs(r["risk"] - V) < 1e-7 * max(1.0, abs(V))


def test_tv_problem_diagnostics_vanish():
    """Total-variation radius 0.4 with boxes and a ball: residual, xi1, xi2,
    infeasibility and the complementarity gap vanish, and s0 equals the nested
    total-variation risk of the trajectory."""
    p = _with_tv(constrained([3, 2, 1], 3, 2, seed=58, avar=0.5, uball=1.5), 0.4)
    o = Oracle(p)
    r = o.solve(tol=1e-8, max_iters=40000)
    assert r["res_inf"] <= 1e-8
    assert r["xi1"] < 1e-5 and r["xi2"] < 1e-5
    assert r["infeas"] < 1e-6 and r["gap"] < 1e-5
    assert abs(r["risk"] - r["nested_risk"]) < 1e-5 * max(1.0, abs(r["risk"]))


# --- soft-constraint costs (the quadratic penalty after Prop. 2) ----------------------


def _soft_problem(seed, avar=1.0, box=False, level=0.3, ball=None):
    p = general([2, 2, 1], 3, 2, seed=seed, avar=avar, box=box, dense=False)
    p.soft_max = np.full(p.nx + p.nu, float(level))
    if ball is not None:
        p.u_ball = np.full(p.n_nonleaf, ball)
    return p


def test_soft_rows_encode_the_penalised_epigraph():
    """l(z) = z'Qz + q'z + ||max(0, z - z_max)||^2 <= tau exactly when some
    sigma, theta with theta >= 0, theta >= z - z_max, ||theta||^2 <= sigma put
    (z, tau - sigma) in the epigraph of the quadratic part. With the smallest
    choice theta = max(0, z - z_max), sigma = ||theta||^2, the rows L gives the
    child's cost cone and the parent's soft block lie in S3 exactly when the
    full cost is at most tau; with sigma below ||theta||^2 the soft cone fails."""
    p = _soft_problem(71)
    o = Oracle(p)
    tr, lay = o.tree, o.lay
    nx, nu, d = o.nx, o.nu, o.nx + o.nu
    rng = np.random.default_rng(8)
    i = 1
    c = tr.children[i][0]
    sc = np.concatenate([o.Snode[i], o.Su])
    w = nx + nu + 2
    cone = slice(lay.e_q + (c - 1) * w, lay.e_q + c * w)
    rows = slice(o.e_sf + i * (3 * d + 2), o.e_sf + (i + 1) * (3 * d + 2))
    for trial in range(40):
        x = rng.standard_normal(nx)
        u = rng.standard_normal(nu)
        cost = o.edge_cost(c, x, u)
        tau = cost + rng.uniform(-0.5, 0.5)
        zu = np.concatenate([x, u])
        th = np.maximum(0.0, zu - p.soft_max)
        z = np.zeros(lay.n_z)
        z[lay.o_x + i * nx:lay.o_x + (i + 1) * nx] = o.Snode[i] * x
        z[lay.o_u + i * nu:lay.o_u + (i + 1) * nu] = o.Su * u
        z[lay.o_tau + c - 1] = tau
        z[o.o_sg + i] = th @ th
        z[o.o_sth + i * d:o.o_sth + (i + 1) * d] = sc * th
        Lz = o.apply_L(z)
        P3 = o.proj_S3(Lz)
        inside = np.allclose(P3[cone], Lz[cone], atol=1e-12) and np.allclose(P3[rows], Lz[rows], atol=1e-12)
        assert inside == (cost <= tau), (trial, cost, tau)
        if th @ th > 1e-3:
            z[o.o_sg + i] = 0.9 * (th @ th)
            L2 = o.apply_L(z)
            assert not np.allclose(o.proj_S3(L2)[rows], L2[rows], atol=1e-12)


def _risk_neutral_soft_qp(p):
    """min sum_c pi^c (x'Qx + u'Ru + q'x + r'u + ||t^a||^2) + sum_j pi^j l_N^j,
    t^i >= 0, t^i >= (x^i, u^i) - z_max, dynamics eliminated: the penalty of
    node i's children weighs pi^i; a QP in (u, t) by the interior-point method
    above (diagonal weights). Returns (value, x, u)."""
    tr = so_.Tree(p.anc, p.prob)
    nx, nu, n = p.nx, p.nu, tr.n
    nX = n * nx + tr.n_nl * nu
    H = np.zeros((nX, nX))
    f = np.zeros(nX)
    for c in range(1, n):
        a = tr.anc[c]
        H[a * nx:(a + 1) * nx, a * nx:(a + 1) * nx] += tr.pi[c] * np.diag(p.Q[c - 1])
        o = n * nx + a * nu
        H[o:o + nu, o:o + nu] += tr.pi[c] * np.diag(p.R[c - 1])
        if p.q is not None:
            f[a * nx:(a + 1) * nx] += tr.pi[c] * p.q[c - 1]
        if p.r is not None:
            f[o:o + nu] += tr.pi[c] * p.r[c - 1]
    for jj in range(tr.n_l):
        j = tr.n_nl + jj
        H[j * nx:(j + 1) * nx, j * nx:(j + 1) * nx] += tr.pi[j] * np.diag(p.QN[jj])
        if p.qN is not None:
            f[j * nx:(j + 1) * nx] += tr.pi[j] * p.qN[jj]
    nU = tr.n_nl * nu
    Pm = np.zeros((nX, nU)); p0 = np.zeros(nX)
    Pm[n * nx:, :] = np.eye(nU)
    p0[:nx] = p.x0
    for c in range(1, n):
        a = tr.anc[c]
        Pm[c * nx:(c + 1) * nx] = p.A[c - 1] @ Pm[a * nx:(a + 1) * nx]
        Pm[c * nx:(c + 1) * nx, a * nu:(a + 1) * nu] += p.B[c - 1]
        p0[c * nx:(c + 1) * nx] = p.A[c - 1] @ p0[a * nx:(a + 1) * nx] + p.c[c - 1]
    d = nx + nu
    nT = tr.n_nl * d
    Sel = np.zeros((nT, nX))
    wt = np.zeros(nT)
    zmax = np.tile(p.soft_max, tr.n_nl)
    for i in range(tr.n_nl):
        Sel[i * d:i * d + nx, i * nx:(i + 1) * nx] = np.eye(nx)
        Sel[i * d + nx:(i + 1) * d, n * nx + i * nu:n * nx + (i + 1) * nu] = np.eye(nu)
        wt[i * d:(i + 1) * d] = tr.pi[i]
    Hw = np.zeros((nU + nT, nU + nT))
    Hw[:nU, :nU] = 2 * Pm.T @ H @ Pm
    Hw[nU:, nU:] = 2 * np.diag(wt)
    fw = np.concatenate([Pm.T @ (2 * H @ p0 + f), np.zeros(nT)])
    Zu = Sel @ Pm
    G = np.vstack([np.hstack([Zu, -np.eye(nT)]), np.hstack([np.zeros((nT, nU)), -np.eye(nT)])])
    h = np.concatenate([zmax - Sel @ p0, np.zeros(nT)])
    wsol = _qp_interior_point(Hw, fw, G, h)
    X = Pm @ wsol[:nU] + p0
    pen = np.maximum(0.0, Sel @ X - zmax)
    val = float(X @ H @ X + f @ X + wt @ (pen * pen))
    return val, X[:n * nx].reshape(n, nx), X[n * nx:].reshape(tr.n_nl, nu)


def test_risk_neutral_soft_costs_vs_qp():
    """AV@R_1, no hard constraints, diagonal weights, linear terms and the soft
    penalty ||max(0, (x, u) - z_max)||^2 in every edge cost: the oracle's SPOCK
    solution equals the QP with t >= 0, t >= z - z_max (value; trajectory on
    the likely nodes); some penalties are active."""
    p = _soft_problem(72, level=0.2)
    o = Oracle(p)
    r = o.solve(tol=1e-9, max_iters=40000)
    V, X, U = _risk_neutral_soft_qp(p)
    assert abs(r["risk"] - V) < 1e-6 * max(1.0, abs(V))
    _check_on_likely_nodes(o, r, X, U, 1e-4)
    tr = o.tree
    zs = np.hstack([X[:tr.n_nl], U])
    assert np.any(zs > p.soft_max + 1e-6)


def test_soft_problem_diagnostics_vanish():
    """AV@R 0.5 with boxes, a ball and soft-constraint costs: the residual, xi1,
    xi2, infeasibility and the complementarity gap vanish, and s0 equals the
    nested risk of the trajectory with the penalties."""
    p = _soft_problem(73, avar=0.5, box=True, level=0.25, ball=1.5)
    o = Oracle(p)
    r = o.solve(tol=1e-8, max_iters=40000)
    assert r["res_inf"] <= 1e-8
    assert r["xi1"] < 1e-5 and r["xi2"] < 1e-5
    assert r["infeas"] < 1e-6 and r["gap"] < 1e-5
    assert abs(r["risk"] - r["nested_risk"]) < 1e-5 * max(1.0, abs(r["risk"]))
