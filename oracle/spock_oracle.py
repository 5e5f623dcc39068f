"""FP64 CPU oracle for the SPOCK hot path (preconditioned Chambolle-Pock with
SuperMann/Anderson acceleration for scenario-tree RAOCPs).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline leg (and its `--impl reference` arm) may import or call this
module. The product path (the CUDA library and its binding) never does, and
this module imports nothing from it: problem data come from the seeded
generators in paper_2505_12078_b300.synth, which hold no solver arithmetic.

Plain, slow, obviously-correct numpy in float64. Every function cites the
paper passage it follows. Where the paper is silent, garbled or inconsistent
the reading taken is stated at the function.

Pins (tests/test_oracle_pins.py): every step is checked against something
other than itself (closed forms, dense KKT solves, LP solves of the risk,
brute force on tiny trees, invariants). The converged solution of a
constrained problem with AV@R level below 1 has no closed form: it is checked
against the same problem solved as a smooth nonlinear program (the nested
AV@R in its Rockafellar-Uryasev form, dynamics substituted, scipy's SLSQP)
with the ball, the input box, the state box or general rows active (also
with full weights and linear terms, with l1 or soft-constraint costs, and
with the total-variation risk through its LP dual), and against the
invariants that every run satisfies (residual, xi1, xi2 and the
complementarity gap vanish; the nested risk of the returned trajectory
equals s0).

Variable layout (scaled variables, Sec. 4.3 "Sets" and Sec. 4.4 "Linear
operator L"). Nodes are in breadth-first order, children contiguous; the
first n_nl nodes are the non-leaf nodes, the last n_l the leaves.

  z   = [ s0 | x (n*nx) | u (n_nl*nu) | y (sum_i 2 n_i + 1) | tau (n-1) | s (n-1) ]
        (with the total-variation risk, y^i has 3 n_i + 2 entries)
        x^i at 1 + i*nx, u^i at 1 + n*nx + i*nu, y^i at its block offset,
        tau^c and s^c (c >= 1) at index c-1 of their arrays.
  eta = [ eta_y (same blocks as y) | eta_s (n_nl) | eta_c (n_nl*n_c)
        | eta_q ((n-1)*(nx+nu+2)) | eta_cN (n_l*n_cN) | eta_qN (n_l*(nx+2)) ]
        eta_y^i  = y^i, eta_s^i = s^i - b^i'y^i, eta_c^i = Gx x^i + Gu u^i,
        eta_q^c  = (Q^c^(1/2) x^anc, R^c^(1/2) u^anc, tau^c/2, tau^c/2),
        eta_cN^j = GN x^j, eta_qN^j = (QN^j^(1/2) x^j, s^j/2, s^j/2).
  With an l1 term lambda_0 ||(x^anc, u^anc)||_1 in the edge costs (Prop. 2)
  z ends with [ theta (n_nl) | lambda (n_nl*(nx+nu)) ] and eta with the rows
  (theta^i - sum lambda^i/s, lambda^i - (x^i, u^i), lambda^i + (x^i, u^i)) per
  non-leaf node, n_nl*(1 + 2(nx+nu)); the cost cone of every child c of i
  carries (tau^c - lambda_0 theta^i)/2 in its last two entries.
  Constraint rows of a non-leaf node: [x box (nx)] [u box (nu)] [u ball (nu)]
  [general rows Gx x + Gu u (n_g)], each kind present or absent for the whole
  problem; leaf rows: [x box (nx)] [general rows GN x (n_gN)]. Q^(1/2) is the
  elementwise root of a diagonal weight or the upper Cholesky factor of a
  full one. Linear cost terms q, r, q_N enter only through the translation a
  of each cost cone (Prop. 1), not through L.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# SuperMann / Anderson parameters printed in Sec. 5.2 (after Alg. 3) and
# Sec. 6.2 (memory m = 3).
C0 = 0.99
C1 = 0.99
C2 = 0.99
BETA = 0.5
SIGMA = 0.1
LAMBDA = 1.0
AA_MEMORY = 3


# ---------------------------------------------------------------------------
# Scenario tree (Sec. 3.2)
# ---------------------------------------------------------------------------
class Tree:
    """Scenario tree: nodes i, stage(i), anc(i), ch(i), probabilities (Sec. 3.2).

    `prob` is the conditional probability of a node given its ancestor; the
    absolute probability pi^i is the product along the path (the stage sums
    of pi are one when the children's conditional probabilities of every
    node sum to one)."""

    def __init__(self, anc, prob):
        anc = np.asarray(anc, dtype=np.int64)
        prob = np.asarray(prob, dtype=np.float64)
        n = anc.shape[0]
        if n < 2 or anc[0] != -1:
            raise ValueError("tree needs a root (anc[0] = -1) and at least one child")
        stage = np.zeros(n, dtype=np.int64)
        for i in range(1, n):
            if not (0 <= anc[i] < i):
                raise ValueError("nodes must be in breadth-first order (anc[i] < i)")
            stage[i] = stage[anc[i]] + 1
        if np.any(np.diff(stage) < 0) or np.any(np.diff(anc[1:]) < 0):
            raise ValueError("nodes must be stage-major with contiguous children")
        N = int(stage.max())
        children = [[] for _ in range(n)]
        for i in range(1, n):
            children[anc[i]].append(i)
        leaves = np.where(stage == N)[0]
        nonleaf = np.where(stage < N)[0]
        if any(len(children[i]) == 0 for i in nonleaf):
            raise ValueError("every node above stage N needs a child")
        if leaves[0] != len(nonleaf):
            raise ValueError("leaves must be the last nodes")
        for i in nonleaf:
            if abs(prob[children[i]].sum() - 1.0) > 1e-12:
                raise ValueError("children probabilities must sum to one")
        self.n = n
        self.anc = anc
        self.prob = prob
        self.stage = stage
        self.N = N
        self.children = [np.asarray(c, dtype=np.int64) for c in children]
        self.n_nl = len(nonleaf)
        self.n_l = len(leaves)
        self.nodes_at = [np.where(stage == t)[0] for t in range(N + 1)]
        pi = np.ones(n)
        for i in range(1, n):
            pi[i] = pi[anc[i]] * prob[i]
        self.pi = pi
        self.n_ch = np.array([len(c) for c in self.children], dtype=np.int64)


# ---------------------------------------------------------------------------
# Risk measures (Sec. 3.3)
# ---------------------------------------------------------------------------
def avar(Z, p, a):
    """AV@R_a[Z] as the maximum of mu'Z over the ambiguity set
    {sum mu = 1, 0 <= mu <= p/a} (Sec. 3.3, "Average-value-at-risk"); a = 0
    gives max Z. The maximiser fills the largest costs first."""
    Z = np.asarray(Z, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    if a <= 0.0:
        return float(Z.max())
    order = np.argsort(-Z, kind="stable")
    left = 1.0
    val = 0.0
    for j in order:
        w = min(p[j] / a, left)
        val += w * Z[j]
        left -= w
        if left <= 0.0:
            break
    return float(val)


def avar_maximiser(Z, p, a):
    """The maximising mu of AV@R_a[Z] over the ambiguity set
    {sum mu = 1, 0 <= mu <= p/a} (Sec. 3.3, "Average-value-at-risk"): mass
    p_j/a goes to the largest costs first until one unit is placed; a = 0 puts
    the unit on the largest cost."""
    Z = np.asarray(Z, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    mu = np.zeros_like(Z)
    order = np.argsort(-Z, kind="stable")
    if a <= 0.0:
        mu[order[0]] = 1.0
        return mu
    left = 1.0
    for j in order:
        w = min(p[j] / a, left)
        mu[j] = w
        left -= w
        if left <= 0.0:
            break
    return mu


def conic_risk_data(p, a):
    """b and E of the conic representation of AV@R_a on the probability space
    ch(i) (Sec. 3.3, "Conic representation"): b = [p; 0_n; 1],
    E = [a I_n, -I_n, 1_n]^T ((2n+1) x n), K = R^{2n}_+ x {0}, F absent.
    Reading: p is the conditional probability vector of the children (the
    conditional risk mapping acts on the probability space ch(i), Sec. 3.4)."""
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    b = np.concatenate([p, np.zeros(n), [1.0]])
    E = np.vstack([a * np.eye(n), -np.eye(n), np.ones((1, n))])
    return b, E


def tv_risk(Z, p, r):
    """Worst expectation of Z over the total-variation ball {mu in the simplex :
    ||mu - p||_1 <= r} around the children's probabilities p: from mu = p, mass
    min(r/2, 1 - p_top) moves onto an outcome with the largest cost, taken from
    the smallest costs first (each outcome gives at most its p)."""
    return float(tv_maximiser(Z, p, r) @ np.asarray(Z, dtype=np.float64))


def tv_maximiser(Z, p, r):
    """The maximising mu of tv_risk (see there)."""
    Z = np.asarray(Z, dtype=np.float64)
    mu = np.asarray(p, dtype=np.float64).copy()
    top = int(np.argmax(Z))
    move = min(0.5 * r, 1.0 - mu[top])
    mu[top] += move
    for j in np.argsort(Z, kind="stable"):
        if move <= 0.0:
            break
        if j == top:
            continue
        w = min(mu[j], move)
        mu[j] -= w
        move -= w
    return mu


def conic_risk_data_tv(p, r):
    """b, E, F of the conic representation (Sec. 3.3, Eq. primal_risk) of the
    total-variation risk: max mu'Z over mu in the simplex with ||mu - p||_1 <=
    r, with an auxiliary nu >= |mu - p| (n_nu = n, so F != 0). Rows of
    b - E mu - F nu in K = R^{3n+1}_+ x {0}:
      nu - mu + p >= 0 (n), nu + mu - p >= 0 (n), r - 1'nu >= 0 (1),
      mu >= 0 (n), 1 - 1'mu = 0 (1):
    b = [p; -p; r; 0; 1], E = [I; -I; 0; -I; 1'], F = [-I; -I; 1'; 0; 0].
    Returns b, E, F and the number of rows in R_+ (3n + 1)."""
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    I = np.eye(n)
    Z0 = np.zeros((n, n))
    b = np.concatenate([p, -p, [r], np.zeros(n), [1.0]])
    E = np.vstack([I, -I, np.zeros((1, n)), -I, np.ones((1, n))])
    F = np.vstack([-I, -I, np.ones((1, n)), Z0, np.zeros((1, n))])
    return b, E, F, 3 * n + 1


# ---------------------------------------------------------------------------
# Projections onto the pieces of S3 (Sec. 4.3, Eq. S3-def)
# ---------------------------------------------------------------------------
def proj_soc(v):
    """Euclidean projection onto SOC_d = {(w, t) : ||w||_2 <= t}, last entry t.
    Rows of a 2-D array are projected independently."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    w = v[:, :-1]
    t = v[:, -1]
    nw = np.linalg.norm(w, axis=1)
    out = np.zeros_like(v)
    inside = nw <= t
    out[inside] = v[inside]
    mid = (~inside) & (nw > -t)
    if np.any(mid):
        f = (nw[mid] + t[mid]) / 2.0
        out[mid, :-1] = w[mid] * (f / nw[mid])[:, None]
        out[mid, -1] = f
    return out


def proj_ball(v, r):
    """Projection onto {w : ||w||_2 <= r} (rows independently, one radius per row)."""
    v = np.atleast_2d(v)
    nv = np.linalg.norm(v, axis=1)
    r = np.broadcast_to(np.asarray(r, dtype=np.float64), nv.shape)
    scale = np.where(nv > r, r / np.where(nv > 0, nv, 1.0), 1.0)
    return v * scale[:, None]


@dataclass
class Layout:
    n_y: int
    n_z: int
    n_eta: int
    o_x: int
    o_u: int
    o_y: int
    o_tau: int
    o_s: int
    e_y: int
    e_s: int
    e_c: int
    e_q: int
    e_cN: int
    e_qN: int


class Oracle:
    """Plain FP64 implementation of the reformulated problem (Sec. 4) and of the
    numerical algorithm (Sec. 5) for one problem from paper_2505_12078_b300.synth."""

    def __init__(self, prob, alpha=None):
        self.P = prob
        tr = Tree(prob.anc, prob.prob)
        self.tree = tr
        n, nx, nu = tr.n, prob.nx, prob.nu
        self.n, self.nx, self.nu = n, nx, nu
        self.has_xbox = prob.x_lo is not None
        self.has_ubox = prob.u_lo is not None
        self.has_uball = prob.u_ball is not None
        self.n_g = 0 if getattr(prob, "Gx", None) is None else int(np.asarray(prob.Gx).shape[0])
        self.n_gN = 0 if getattr(prob, "GN", None) is None else int(np.asarray(prob.GN).shape[0])
        self.n_c = (nx if self.has_xbox else 0) + (nu if self.has_ubox else 0) + \
                   (nu if self.has_uball else 0) + self.n_g
        self.n_cN = (nx if self.has_xbox else 0) + self.n_gN
        self.l1 = float(getattr(prob, "l1", None) or 0.0)
        sm = getattr(prob, "soft_max", None)
        self.soft = None if sm is None else np.asarray(sm, dtype=np.float64)
        self._layout()
        self._precondition()
        self._offline_s1()
        self._build_L()
        self.normL = self._norm_L()
        self.alpha = 0.99 / self.normL if alpha is None else float(alpha)

    # -- layout ------------------------------------------------------------
    def _layout(self):
        tr = self.tree
        n, nx, nu, n_nl, n_l = tr.n, self.nx, self.nu, tr.n_nl, tr.n_l
        self.tv = None if getattr(self.P, "tv", None) is None else np.asarray(self.P.tv, dtype=np.float64)
        m_ = tr.n_ch[:n_nl]
        self.ylen = (3 * m_ + 2) if self.tv is not None else (2 * m_ + 1)
        self.yoff = np.concatenate([[0], np.cumsum(self.ylen)]).astype(np.int64)
        n_y = int(self.yoff[-1])
        o_x = 1
        o_u = o_x + n * nx
        o_y = o_u + n_nl * nu
        o_tau = o_y + n_y
        o_s = o_tau + (n - 1)
        n_z = o_s + (n - 1)
        e_y = 0
        e_s = n_y
        e_c = e_s + n_nl
        e_q = e_c + n_nl * self.n_c
        e_cN = e_q + (n - 1) * (nx + nu + 2)
        e_qN = e_cN + n_l * self.n_cN
        n_eta = e_qN + n_l * (nx + 2)
        # l1 stage costs (Prop. 2): theta^i and lambda^i (nx + nu) per non-leaf
        # node at the end of z; the rows theta - sum lambda, lambda - z,
        # lambda + z (z = (x^i, u^i)) per non-leaf node at the end of eta
        self.o_th = n_z
        self.o_lam = n_z + (n_nl if self.l1 else 0)
        self.e_l1 = n_eta
        if self.l1:
            n_z = self.o_lam + n_nl * (nx + nu)
            n_eta = self.e_l1 + n_nl * (1 + 2 * (nx + nu))
        # soft-constraint costs (after Prop. 2): sigma^i and theta^i (nx + nu)
        # per non-leaf node next in z; per non-leaf node the rows
        # [theta/s, sigma/2, sigma/2] - a in SOC, theta >= 0, theta - z >= -s z_max
        self.o_sg = n_z
        self.o_sth = n_z + (n_nl if self.soft is not None else 0)
        self.e_sf = n_eta
        if self.soft is not None:
            n_z = self.o_sth + n_nl * (nx + nu)
            n_eta = self.e_sf + n_nl * (3 * (nx + nu) + 2)
        self.lay = Layout(n_y, n_z, n_eta, o_x, o_u, o_y, o_tau, o_s,
                          e_y, e_s, e_c, e_q, e_cN, e_qN)
        # entries of eta_y that lie in R_+ (all but the last entry of each block:
        # the zero cone's dual R of AV@R's and the total-variation risk's sums)
        mask = np.ones(n_y, dtype=bool)
        mask[self.yoff[1:] - 1] = False
        self.ypos = mask

    # -- preconditioning (Sec. 5.4) ----------------------------------------
    def _precondition(self):
        """Diagonal scalings of Sec. 5.4.

        c_hat = sqrt(max_i |ch(i)|) over the whole tree; S^x_kk = c_hat
        max{1, max_i sqrt(Q^i_kk)}, S^u likewise with R^i (i over the non-root
        nodes, which carry the edge costs), S^x_N,kk = max{1, max_j
        sqrt(Q_N^j_kk)}. Reading of the index ranges: x at stages 0..N-1 is
        scaled by S^x, x at stage N by S^x_N, every u by S^u. The constraint
        matrices are multiplied by the inverse scalings (the printed
        "Gamma_N S_x" is read as S_x,N^{-1}) and every constraint row block is
        divided by a = max{1, ||[Gx Sx^{-1}  Gu Su^{-1}]||_2}, the set likewise.
        """
        P, tr = self.P, self.tree
        nx, nu = self.nx, self.nu
        c_hat = math.sqrt(float(tr.n_ch.max()))
        Qd = self._diag(P.Q)
        Rd = self._diag(P.R)
        QNd = self._diag(P.QN)
        self.c_hat = c_hat
        self.Sx = c_hat * np.maximum(1.0, np.sqrt(Qd.max(axis=0)))
        self.Su = c_hat * np.maximum(1.0, np.sqrt(Rd.max(axis=0)))
        self.SxN = np.maximum(1.0, np.sqrt(QNd.max(axis=0)))
        n = tr.n
        Snode = np.empty((n, nx))
        Snode[:] = self.Sx
        Snode[tr.stage == tr.N] = self.SxN
        self.Snode = Snode
        A = np.asarray(P.A, dtype=np.float64)
        B = np.asarray(P.B, dtype=np.float64)
        cc = np.asarray(P.c, dtype=np.float64)
        Sc = Snode[1:]                      # scaling of each child c
        Sp = Snode[tr.anc[1:]]              # scaling of its ancestor
        self.At = Sc[:, :, None] * A / Sp[:, None, :]
        self.Bt = Sc[:, :, None] * B / self.Su[None, None, :]
        self.ct = Sc * cc
        # cost square roots: any F with F'F = Q (Sec. 4.4 writes (Q^i)^{1/2});
        # the elementwise root for diagonal weights, the upper Cholesky factor
        # for dense ones. Scaled: F S^{-1}.
        if np.ndim(P.Q) == 3:
            self.Qh = self._sqrt_weight(P.Q) / Sp[:, None, :]
        else:
            self.Qh = np.sqrt(Qd) / Sp
        if np.ndim(P.R) == 3:
            self.Rh = self._sqrt_weight(P.R) / self.Su[None, None, :]
        else:
            self.Rh = np.sqrt(Rd) / self.Su[None, :]
        SxN_leaf = Snode[tr.n_nl:]
        if np.ndim(P.QN) == 3:
            self.QNh = self._sqrt_weight(P.QN) / SxN_leaf[:, None, :]
        else:
            self.QNh = np.sqrt(QNd) / SxN_leaf
        # constraint matrices of a non-leaf node (unscaled, Eq. constraints):
        # selection rows of the boxes and the ball, then the general rows
        Gx, Gu = [], []
        if self.has_xbox:
            Gx.append(np.eye(nx)); Gu.append(np.zeros((nx, nu)))
        if self.has_ubox:
            Gx.append(np.zeros((nu, nx))); Gu.append(np.eye(nu))
        if self.has_uball:
            Gx.append(np.zeros((nu, nx))); Gu.append(np.eye(nu))
        if self.n_g:
            Gx.append(np.asarray(P.Gx, dtype=np.float64)); Gu.append(np.asarray(P.Gu, dtype=np.float64))
        if self.n_c:
            Gx = np.vstack(Gx)
            Gu = np.vstack(Gu)
            M = np.hstack([Gx / self.Sx[None, :], Gu / self.Su[None, :]])
            self.a_con = max(1.0, float(np.linalg.norm(M, 2)))
            self.Gx = Gx / self.Sx[None, :] / self.a_con
            self.Gu = Gu / self.Su[None, :] / self.a_con
        else:
            self.a_con = 1.0
            self.Gx = np.zeros((0, nx))
            self.Gu = np.zeros((0, nu))
        if self.n_cN:
            GN = []
            if self.has_xbox:
                GN.append(np.eye(nx))
            if self.n_gN:
                GN.append(np.asarray(P.GN, dtype=np.float64))
            MN = np.vstack(GN) / self.SxN[None, :]
            self.a_conN = max(1.0, float(np.linalg.norm(MN, 2)))
            self.GN = MN / self.a_conN
        else:
            self.a_conN = 1.0
            self.GN = np.zeros((0, nx))
        n_nl = tr.n_nl
        lo, hi = [], []
        if self.has_xbox:
            lo.append(P.x_lo[:n_nl]); hi.append(P.x_hi[:n_nl])
        if self.has_ubox:
            lo.append(P.u_lo); hi.append(P.u_hi)
        self.box_lo = (np.hstack(lo) / self.a_con) if lo else np.zeros((n_nl, 0))
        self.box_hi = (np.hstack(hi) / self.a_con) if hi else np.zeros((n_nl, 0))
        self.n_box = self.box_lo.shape[1]
        self.ball_r = (np.asarray(P.u_ball, dtype=np.float64) / self.a_con) if self.has_uball else None
        if self.n_g:
            self.gen_lo = np.asarray(P.g_lo, dtype=np.float64) / self.a_con
            self.gen_hi = np.asarray(P.g_hi, dtype=np.float64) / self.a_con
        if self.n_cN:
            lo, hi = [], []
            if self.has_xbox:
                lo.append(P.x_lo[n_nl:]); hi.append(P.x_hi[n_nl:])
            if self.n_gN:
                lo.append(np.asarray(P.gN_lo, dtype=np.float64)); hi.append(np.asarray(P.gN_hi, dtype=np.float64))
            self.boxN_lo = np.hstack(lo) / self.a_conN
            self.boxN_hi = np.hstack(hi) / self.a_conN
        self._cost_translations()
        self.avar_level = np.asarray(P.avar, dtype=np.float64)
        self.x0s = self.Sx * np.asarray(P.x0, dtype=np.float64)

    def _cost_translations(self):
        """Translation vectors of the cost cones (Prop. 1, quadratic-plus-linear
        costs, Q positive definite so S = I): the epigraph of z'Qz + q'z is
        {(z, tau) : (F z, tau/2, tau/2) - a in SOC} with F any factor with
        F'F = Q (the one L uses) and a = (-F^{-T} q / 2, -kappa/8 + 1/2,
        -kappa/8 - 1/2), kappa = q'Q^{-1}q = ||F^{-T} q||^2. For an edge cost
        F = blockdiag(F_Q, F_R) acts on (x, u). The diagonal scalings of Sec. 5.4
        leave a unchanged (F S^{-1} and S^{-1} q give the same F^{-T} q). Without
        linear terms a = (0, 1/2, -1/2)."""
        P, tr = self.P, self.tree
        nx, nu, n = self.nx, self.nu, tr.n
        W = nx + nu + 2
        self.a_q = np.zeros((n - 1, W))
        self.a_q[:, -2] = 0.5
        self.a_q[:, -1] = -0.5
        self.a_qN = np.zeros((tr.n_l, nx + 2))
        self.a_qN[:, -2] = 0.5
        self.a_qN[:, -1] = -0.5
        q = getattr(P, "q", None)
        r = getattr(P, "r", None)
        qN = getattr(P, "qN", None)

        def ftq(Wm, lin):
            # F^{-T} lin with F the factor of Wm used by L (upper Cholesky factor
            # for full matrices, elementwise root for diagonals)
            Wm = np.asarray(Wm, dtype=np.float64)
            if Wm.ndim == 2:
                return lin / np.sqrt(Wm)
            Lc = np.linalg.cholesky(Wm)                    # Wm = Lc Lc', F = Lc', F^{-T} = Lc^{-1}
            return np.linalg.solve(Lc, lin[..., None])[..., 0]

        if q is not None or r is not None:
            kap = np.zeros(n - 1)
            if q is not None:
                w = ftq(P.Q, np.asarray(q, dtype=np.float64))
                self.a_q[:, :nx] = -0.5 * w
                kap += np.sum(w * w, axis=1)
            if r is not None:
                w = ftq(P.R, np.asarray(r, dtype=np.float64))
                self.a_q[:, nx:nx + nu] = -0.5 * w
                kap += np.sum(w * w, axis=1)
            self.a_q[:, -2] -= kap / 8.0
            self.a_q[:, -1] -= kap / 8.0
        if qN is not None:
            w = ftq(P.QN, np.asarray(qN, dtype=np.float64))
            self.a_qN[:, :nx] = -0.5 * w
            kap = np.sum(w * w, axis=1)
            self.a_qN[:, -2] -= kap / 8.0
            self.a_qN[:, -1] -= kap / 8.0

    @staticmethod
    def _diag(W):
        W = np.asarray(W, dtype=np.float64)
        if W.ndim == 3:
            return np.diagonal(W, axis1=1, axis2=2).copy()
        return W

    @staticmethod
    def _sqrt_weight(W):
        """Upper Cholesky factor F (F'F = W) of every dense weight matrix."""
        Lc = np.linalg.cholesky(np.asarray(W, dtype=np.float64))
        return np.transpose(Lc, (0, 2, 1))

    # -- offline projection data, Alg. 1 -----------------------------------
    def _offline_s1(self):
        """Alg. 1 (projection on S1, offline) on the scaled A, B with unit weights.

        Leaves: P = I. Stage by stage from N-1 down to 0, for all nodes of the
        stage: P~ = B'P (per child), R~ = I + sum B'P B with its Cholesky
        factor, K = -R~^{-1} sum P~ A, Abar = A + B K (per child),
        P = I + K'K + sum Abar' P Abar."""
        tr = self.tree
        nx, nu, n = self.nx, self.nu, tr.n
        Pm = np.zeros((n, nx, nx))
        Pm[tr.n_nl:] = np.eye(nx)
        K = np.zeros((tr.n_nl, nu, nx))
        Rt = np.zeros((tr.n_nl, nu, nu))
        Rchol = np.zeros((tr.n_nl, nu, nu))
        Abar = np.zeros((n - 1, nx, nx))
        for t in range(tr.N):
            st = tr.N - (t + 1)
            par = tr.nodes_at[st]
            ch = tr.nodes_at[st + 1]
            loc = tr.anc[ch] - par[0]
            Bc = self.Bt[ch - 1]
            Ac = self.At[ch - 1]
            Ptil = np.einsum("cxu,cxy->cuy", Bc, Pm[ch])             # B'P
            Rs = np.zeros((len(par), nu, nu))
            np.add.at(Rs, loc, Ptil @ Bc)
            Rpar = np.eye(nu)[None] + Rs
            KA = np.zeros((len(par), nu, nx))
            np.add.at(KA, loc, Ptil @ Ac)
            Lc = np.linalg.cholesky(Rpar)                             # R~ = Lc Lc'
            tmp = sla.solve_triangular(Lc, KA, lower=True)
            Kp = -sla.solve_triangular(np.transpose(Lc, (0, 2, 1)), tmp, lower=False)
            Ab = Ac + Bc @ Kp[loc]
            Pp = np.eye(nx)[None] + np.transpose(Kp, (0, 2, 1)) @ Kp
            np.add.at(Pp, loc, np.transpose(Ab, (0, 2, 1)) @ Pm[ch] @ Ab)
            Pm[par] = Pp
            K[par] = Kp
            Rt[par] = Rpar
            Rchol[par] = Lc
            Abar[ch - 1] = Ab
        self.Pm, self.K, self.Rt, self.Rchol, self.Abar = Pm, K, Rt, Rchol, Abar

    # -- proj S1, Alg. 2 ----------------------------------------------------
    def proj_S1(self, xbar, ubar):
        """Alg. 2 (projection on S1, online): minimiser of
        1/2 sum ||x - xbar||^2 + 1/2 sum ||u - ubar||^2 over the dynamics with
        x^0 = the (scaled) initial state. Reading of the printed subscripts:
        q_0^i, d_{t+1}^i and q_{t+1}^i all denote the node's own q^i, d^i."""
        tr = self.tree
        nx, nu, n = self.nx, self.nu, tr.n
        q = np.zeros((n, nx))
        q[tr.n_nl:] = -xbar[tr.n_nl:]
        d = np.zeros((tr.n_nl, nu))
        for t in range(tr.N):
            st = tr.N - (t + 1)
            par = tr.nodes_at[st]
            ch = tr.nodes_at[st + 1]
            loc = tr.anc[ch] - par[0]
            Bc = self.Bt[ch - 1]
            cc = self.ct[ch - 1]
            Pc = self.Pm[ch]
            dbar = np.zeros((len(par), nu))
            np.add.at(dbar, loc, np.einsum("cxu,cx->cu", Bc, q[ch] + np.einsum("cxy,cy->cx", Pc, cc)))
            rhs = ubar[par] - dbar
            Lc = self.Rchol[par]
            tmp = sla.solve_triangular(Lc, rhs[:, :, None], lower=True)
            dp = sla.solve_triangular(np.transpose(Lc, (0, 2, 1)), tmp, lower=False)[:, :, 0]
            inner = np.einsum("cxy,cy->cx", Pc, np.einsum("cxu,cu->cx", Bc, dp[loc]) + cc) + q[ch]
            qbar = np.zeros((len(par), nx))
            np.add.at(qbar, loc, np.einsum("cyx,cy->cx", self.Abar[ch - 1], inner))
            q[par] = np.einsum("iux,iu->ix", self.K[par], dp - ubar[par]) - xbar[par] + qbar
            d[par] = dp
        x = np.zeros((n, nx))
        u = np.zeros((tr.n_nl, nu))
        x[0] = self.x0s
        for st in range(tr.N):
            par = tr.nodes_at[st]
            ch = tr.nodes_at[st + 1]
            u[par] = np.einsum("iux,ix->iu", self.K[par], x[par]) + d[par]
            pa = tr.anc[ch]
            x[ch] = np.einsum("cxy,cy->cx", self.At[ch - 1], x[pa]) + \
                np.einsum("cxu,cu->cx", self.Bt[ch - 1], u[pa]) + self.ct[ch - 1]
        return x, u

    # -- proj S2 -----------------------------------------------------------
    def proj_S2(self, y, tau, s):
        """Projection of (y^i, tau^[i], s^[i]) onto ker[E_i', -I, -I; F_i', 0, 0]
        for every non-leaf node (Sec. 4.3, S_2; F is absent for AV@R), written
        out as v - G'(GG')^{-1} G v with the dense G of each node (nodes with
        equal child counts are stacked into one batched solve)."""
        tr = self.tree
        y2, tau2, s2 = y.copy(), tau.copy(), s.copy()
        for m in np.unique(tr.n_ch[:tr.n_nl]):
            nodes = np.where(tr.n_ch[:tr.n_nl] == m)[0]
            ly = int(self.ylen[nodes[0]])
            rows = []
            V = np.zeros((len(nodes), ly + 2 * m))
            for a, i in enumerate(nodes):
                ch = tr.children[i]
                _, E, F = self._risk_data(i)
                Gi = np.hstack([E.T, -np.eye(m), -np.eye(m)])
                if F.shape[1]:
                    Gi = np.vstack([Gi, np.hstack([F.T, np.zeros((F.shape[1], 2 * m))])])
                rows.append(Gi)
                V[a] = np.concatenate([y[self.yoff[i]:self.yoff[i + 1]], tau[ch - 1], s[ch - 1]])
            G = np.stack(rows)
            Gv = np.einsum("akj,aj->ak", G, V)
            lam = np.linalg.solve(G @ np.transpose(G, (0, 2, 1)), Gv[:, :, None])[:, :, 0]
            PV = V - np.einsum("akj,ak->aj", G, lam)
            for a, i in enumerate(nodes):
                ch = tr.children[i]
                y2[self.yoff[i]:self.yoff[i + 1]] = PV[a, :ly]
                tau2[ch - 1] = PV[a, ly:ly + m]
                s2[ch - 1] = PV[a, ly + m:]
        return y2, tau2, s2

    # -- linear operator L (Sec. 4.4) --------------------------------------
    def _risk_data(self, i):
        """b, E, F of node i's conic risk (Sec. 3.3): AV@R with the node's level
        (F absent: an empty matrix), or the total-variation ball of radius tv[i]."""
        ch = self.tree.children[i]
        if self.tv is not None:
            b, E, F, _ = conic_risk_data_tv(self.tree.prob[ch], self.tv[i])
            return b, E, F
        b, E = conic_risk_data(self.tree.prob[ch], self.avar_level[i])
        return b, E, np.zeros((E.shape[0], 0))

    def _build_L(self):
        """L as an explicit sparse matrix, block by block as defined in Sec. 4.4:
        ((y^i, s^i - b^i'y^i, Gx x^i + Gu u^i)_{non-leaf i},
         (Q^{i 1/2} x^anc, R^{i 1/2} u^anc, tau^i/2, tau^i/2)_{non-root i},
         (GN x^j, QN^{j 1/2} x^j, s^j/2, s^j/2)_{leaf j})."""
        tr, lay = self.tree, self.lay
        nx, nu, n = self.nx, self.nu, tr.n
        rows, cols, vals = [], [], []

        def add_block(r0, c0, M):
            M = np.atleast_2d(M)
            rr, cc = np.nonzero(M)
            rows.append(r0 + rr); cols.append(c0 + cc); vals.append(M[rr, cc])

        def iz_s(i):
            return 0 if i == 0 else lay.o_s + i - 1

        for i in range(tr.n_nl):
            ch = tr.children[i]
            b, _, _ = self._risk_data(i)
            L_ = self.ylen[i]
            add_block(lay.e_y + self.yoff[i], lay.o_y + self.yoff[i], np.eye(L_))
            r = lay.e_s + i
            add_block(r, iz_s(i), np.ones((1, 1)))
            add_block(r, lay.o_y + self.yoff[i], -b[None, :])
            if self.n_c:
                add_block(lay.e_c + i * self.n_c, lay.o_x + i * nx, self.Gx)
                add_block(lay.e_c + i * self.n_c, lay.o_u + i * nu, self.Gu)
        w = nx + nu + 2
        for c in range(1, n):
            a = tr.anc[c]
            base = lay.e_q + (c - 1) * w
            Qh = self.Qh[c - 1]
            Rh = self.Rh[c - 1]
            add_block(base, lay.o_x + a * nx, np.diag(Qh) if Qh.ndim == 1 else Qh)
            add_block(base + nx, lay.o_u + a * nu, np.diag(Rh) if Rh.ndim == 1 else Rh)
            add_block(base + nx + nu, lay.o_tau + c - 1, np.array([[0.5], [0.5]]))
        for jj in range(tr.n_l):
            j = tr.n_nl + jj
            if self.n_cN:
                add_block(lay.e_cN + jj * self.n_cN, lay.o_x + j * nx, self.GN)
            base = lay.e_qN + jj * (nx + 2)
            QNh = self.QNh[jj]
            add_block(base, lay.o_x + j * nx, np.diag(QNh) if QNh.ndim == 1 else QNh)
            add_block(base + nx, lay.o_s + j - 1, np.array([[0.5], [0.5]]))
        if self.l1:
            # Prop. 2 with the auxiliaries shared by the children of a node (the
            # l1 term of the edge costs of node i's children is the same function
            # of (x^i, u^i) for every child): tau^c - lambda_0 theta^i replaces
            # tau^c in the cone of every child c, and theta^i >= sum_k lambda_k,
            # -lambda_k <= z_k <= lambda_k on the unscaled z = (x^i, u^i). Here
            # lambda is kept scaled like z (lambda~_k = s_k lambda_k), so the rows
            # are theta - sum_k lambda~_k / s_k, lambda~ - z~, lambda~ + z~, all in R_+.
            d = nx + nu
            for c in range(1, n):
                base = lay.e_q + (c - 1) * w
                add_block(base + nx + nu, self.o_th + tr.anc[c], np.array([[-0.5 * self.l1], [-0.5 * self.l1]]))
            for i in range(tr.n_nl):
                sc = np.concatenate([self.Snode[i], self.Su])
                r0 = self.e_l1 + i * (1 + 2 * d)
                ol = self.o_lam + i * d
                add_block(r0, self.o_th + i, np.ones((1, 1)))
                add_block(r0, ol, -(1.0 / sc)[None, :])
                add_block(r0 + 1, ol, np.eye(d))
                add_block(r0 + 1, lay.o_x + i * nx, -np.eye(d)[:, :nx])
                add_block(r0 + 1, lay.o_u + i * nu, -np.eye(d)[:, nx:])
                add_block(r0 + 1 + d, ol, np.eye(d))
                add_block(r0 + 1 + d, lay.o_x + i * nx, np.eye(d)[:, :nx])
                add_block(r0 + 1 + d, lay.o_u + i * nu, np.eye(d)[:, nx:])
        if self.soft is not None:
            # the penalty ||max(0, z - z_max)||^2 of every child's edge cost is the
            # same function of node i's z = (x^i, u^i): tau^c - sigma^i replaces
            # tau^c in every child's cone, sigma^i >= ||theta^i||^2 (a cone of its
            # own, Prop. 1 with Q = I), theta^i >= 0, theta^i >= z - z_max; theta is
            # kept scaled like z (theta~_k = s_k theta_k)
            d = nx + nu
            for c in range(1, n):
                base = lay.e_q + (c - 1) * w
                add_block(base + nx + nu, self.o_sg + tr.anc[c], np.array([[-0.5], [-0.5]]))
            for i in range(tr.n_nl):
                sc = np.concatenate([self.Snode[i], self.Su])
                r0 = self.e_sf + i * (3 * d + 2)
                ot = self.o_sth + i * d
                add_block(r0, ot, np.diag(1.0 / sc))
                add_block(r0 + d, self.o_sg + i, np.array([[0.5], [0.5]]))
                add_block(r0 + d + 2, ot, np.eye(d))
                add_block(r0 + 2 * d + 2, ot, np.eye(d))
                add_block(r0 + 2 * d + 2, lay.o_x + i * nx, -np.eye(d)[:, :nx])
                add_block(r0 + 2 * d + 2, lay.o_u + i * nu, -np.eye(d)[:, nx:])
            self.soft_lo = -np.concatenate([self.Snode[0], self.Su]) * self.soft   # scaled -s z_max
        rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
        self.L = sp.csr_matrix((vals, (rows, cols)), shape=(lay.n_eta, lay.n_z))
        self.LT = self.L.T.tocsr()

    def _norm_L(self, dense_max=2500):
        """||L|| (Sec. 4.1 requires 0 < alpha ||L|| < 1; the paper does not say
        how alpha is chosen: alpha = 0.99/||L||). Dense SVD for small L, else the
        largest eigenvalue of L'L by Lanczos at machine tolerance."""
        if self.lay.n_z <= dense_max:
            return float(np.linalg.norm(self.L.toarray(), 2))
        LtL = (self.LT @ self.L).tocsr()
        ev = spla.eigsh(LtL, k=1, which="LA", tol=1e-15, maxiter=100000,
                        v0=np.ones(self.lay.n_z), return_eigenvectors=False)
        return float(math.sqrt(ev[0]))

    def apply_L(self, z):
        return self.L @ z

    def apply_Lt(self, eta):
        return self.LT @ eta

    # -- proximal operators --------------------------------------------------
    def split_z(self, z):
        tr, lay = self.tree, self.lay
        s0 = z[0]
        x = z[lay.o_x:lay.o_u].reshape(tr.n, self.nx)
        u = z[lay.o_u:lay.o_y].reshape(tr.n_nl, self.nu)
        y = z[lay.o_y:lay.o_tau]
        tau = z[lay.o_tau:lay.o_s]
        s = z[lay.o_s:lay.o_s + tr.n - 1]
        return s0, x, u, y, tau, s

    @staticmethod
    def join_z(s0, x, u, y, tau, s, aux=()):
        return np.concatenate([[s0], x.ravel(), u.ravel(), y, tau, s, aux])

    def prox_f(self, w):
        """prox_{alpha f} with f(z) = s0 + delta_S1(z_1) + delta_S2(z_2)
        (Eq. f): s0 - alpha, proj_S1 (Alg. 2), proj_S2. The auxiliaries of the
        l1 costs (Prop. 2) do not enter f: their prox is the identity."""
        s0, x, u, y, tau, s = self.split_z(w)
        x2, u2 = self.proj_S1(x, u)
        y2, tau2, s2 = self.proj_S2(y, tau, s)
        return self.join_z(s0 - self.alpha, x2, u2, y2, tau2, s2, w[self.o_th:])

    def proj_S3(self, v):
        """Projection onto S3 (Eq. S3-def): (K^i)* = R^{2n_i}_+ x R, R_+, C^i per
        non-leaf node; SOC_{nx+nu+2} + a^i per non-root node; C^j x
        (SOC_{nx+2} + a_N^j) per leaf. With q = r = 0 Proposition 1 gives
        a = (0, 1/2, -1/2); the SOC's last coordinate is its scalar part."""
        tr, lay = self.tree, self.lay
        nx, nu = self.nx, self.nu
        out = v.copy()
        ey = v[lay.e_y:lay.e_s]
        out[lay.e_y:lay.e_s] = np.where(self.ypos, np.maximum(ey, 0.0), ey)
        out[lay.e_s:lay.e_c] = np.maximum(v[lay.e_s:lay.e_c], 0.0)
        if self.n_c:
            C = v[lay.e_c:lay.e_q].reshape(tr.n_nl, self.n_c).copy()
            nb = self.n_box
            C[:, :nb] = np.clip(C[:, :nb], self.box_lo, self.box_hi)
            nbl = nb + (nu if self.has_uball else 0)
            if self.has_uball:
                C[:, nb:nbl] = proj_ball(C[:, nb:nbl], self.ball_r)
            if self.n_g:
                C[:, nbl:] = np.clip(C[:, nbl:], self.gen_lo, self.gen_hi)
            out[lay.e_c:lay.e_q] = C.ravel()
        w = nx + nu + 2
        Qb = v[lay.e_q:lay.e_cN].reshape(tr.n - 1, w)
        out[lay.e_q:lay.e_cN] = (self.a_q + proj_soc(Qb - self.a_q)).ravel()
        if self.n_cN:
            CN = v[lay.e_cN:lay.e_qN].reshape(tr.n_l, self.n_cN)
            out[lay.e_cN:lay.e_qN] = np.clip(CN, self.boxN_lo, self.boxN_hi).ravel()
        QN = v[lay.e_qN:self.e_l1].reshape(tr.n_l, nx + 2)
        out[lay.e_qN:self.e_l1] = (self.a_qN + proj_soc(QN - self.a_qN)).ravel()
        out[self.e_l1:self.e_sf] = np.maximum(v[self.e_l1:self.e_sf], 0.0)     # l1 rows (Prop. 2): R_+
        if self.soft is not None:
            d = nx + nu
            B = v[self.e_sf:].reshape(tr.n_nl, 3 * d + 2)
            O = B.copy()
            a = np.zeros(d + 2); a[-2] = 0.5; a[-1] = -0.5
            O[:, :d + 2] = a + proj_soc(B[:, :d + 2] - a)
            O[:, d + 2:2 * d + 2] = np.maximum(B[:, d + 2:2 * d + 2], 0.0)
            O[:, 2 * d + 2:] = np.maximum(B[:, 2 * d + 2:], self.soft_lo)
            out[self.e_sf:] = O.ravel()
        return out

    def prox_gconj(self, v):
        """prox_{alpha g*}(v) = v - alpha proj_S3(v / alpha) (Moreau identity),
        g = delta_S3 (Eq. g)."""
        return v - self.alpha * self.proj_S3(v / self.alpha)

    # -- CP operator T (Eq. chambolle-pock-operator) --------------------------
    def T(self, v):
        """One Chambolle-Pock step: z+ = prox_{alpha f}(z - alpha L* eta),
        eta+ = prox_{alpha g*}(eta + alpha L(2 z+ - z))."""
        nz = self.lay.n_z
        z, eta = v[:nz], v[nz:]
        zp = self.prox_f(z - self.alpha * self.apply_Lt(eta))
        etap = self.prox_gconj(eta + self.alpha * self.apply_L(2.0 * zp - z))
        return np.concatenate([zp, etap])

    def M_inner(self, a, b):
        """<a, b>_M with M = [I, -alpha L*; -alpha L, I] (Sec. 4.1); M is
        never formed."""
        nz = self.lay.n_z
        az, ae = a[:nz], a[nz:]
        bz, be = b[:nz], b[nz:]
        return float(az @ bz + ae @ be - self.alpha * (ae @ self.apply_L(bz))
                     - self.alpha * (be @ self.apply_L(az)))

    def M_norm(self, a):
        return math.sqrt(max(self.M_inner(a, a), 0.0))

    # -- Anderson's acceleration (Alg. 3) ------------------------------------
    @staticmethod
    def aa_direction(r, S, Y, k, m=AA_MEMORY, rank_tol=1e-10):
        """Alg. 3 with memory m. Reading of the printed update
        psi = -r - (M_r - M_d) kappa: the type-II form with S holding iterate
        differences v^(k) - v^(k-1) and Y residual differences r^(k) - r^(k-1):
        kappa = argmin ||Y kappa - r|| by Householder QR (R kappa = Q'r),
        psi = -r - (S - Y) kappa. For k <= m, psi = -r. A QR factor with
        |R_jj| < rank_tol ||Y||_F falls back to psi = -r."""
        if k <= m or len(Y) == 0:
            return -r
        Ym = np.column_stack(Y)
        Sm = np.column_stack(S)
        Qf, Rf = np.linalg.qr(Ym)
        fro = np.linalg.norm(Ym)
        if fro == 0.0 or np.min(np.abs(np.diag(Rf))) < rank_tol * fro:
            return -r
        kappa = sla.solve_triangular(Rf, Qf.T @ r, lower=False)
        return -r - (Sm - Ym) @ kappa

    class QRMemory:
        """Anderson memory whose least-squares factorisation Y = Q R is updated
        as pairs arrive and leave instead of being recomputed (the improvement
        Sec. 6.2 suggests, with Givens rotations): dropping the oldest column
        leaves R upper Hessenberg, which Givens rotations of neighbouring rows
        make triangular again (the same rotations applied to the columns of
        Q); a new column y is appended by Gram-Schmidt against Q with one
        re-orthogonalisation, giving R's new last column (Q'y, ||y - QQ'y||)."""

        def __init__(self, m):
            self.m = m
            self.S = []
            self.Q = None          # n x k, orthonormal columns
            self.R = np.zeros((0, 0))

        def push(self, s, y):
            if len(self.S) == self.m:
                self._drop_oldest()
            if self.Q is None:
                h = np.zeros(0)
                w = y.copy()
            else:
                h = self.Q.T @ y
                w = y - self.Q @ h
                h2 = self.Q.T @ w
                w = w - self.Q @ h2
                h = h + h2
            rho = float(np.linalg.norm(w))
            k = self.R.shape[0]
            R = np.zeros((k + 1, k + 1))
            R[:k, :k] = self.R
            R[:k, k] = h
            R[k, k] = rho
            self.R = R
            col = (w / rho if rho > 0 else w)[:, None]
            self.Q = col if self.Q is None else np.hstack([self.Q, col])
            self.S.append(s)

        def _drop_oldest(self):
            H = self.R[:, 1:].copy()            # k x (k-1), upper Hessenberg
            Q = self.Q.copy()
            k = H.shape[0]
            for j in range(k - 1):
                a, b = H[j, j], H[j + 1, j]
                r = math.hypot(a, b)
                c, sn = (1.0, 0.0) if r == 0.0 else (a / r, b / r)
                Hj, Hj1 = H[j].copy(), H[j + 1].copy()
                H[j], H[j + 1] = c * Hj + sn * Hj1, -sn * Hj + c * Hj1
                Qj, Qj1 = Q[:, j].copy(), Q[:, j + 1].copy()
                Q[:, j], Q[:, j + 1] = c * Qj + sn * Qj1, -sn * Qj + c * Qj1
            self.R = H[:k - 1, :]
            self.Q = Q[:, :k - 1]
            self.S.pop(0)

        def direction(self, r, k, rank_tol=1e-10):
            """psi of Alg. 3 (type-II reading): kappa = R^{-1} Q'r, psi = -r -
            (S - Y) kappa with Y kappa = Q Q'r; psi = -r for k <= m or when a
            diagonal entry of R is below rank_tol ||Y||_F."""
            if k <= self.m or not self.S:
                return -r
            fro = float(np.linalg.norm(self.R))
            if fro == 0.0 or np.min(np.abs(np.diag(self.R))) < rank_tol * fro:
                return -r
            g = self.Q.T @ r
            kappa = sla.solve_triangular(self.R, g, lower=False)
            return -r - np.column_stack(self.S) @ kappa + self.Q @ g

    # -- SPOCK (Alg. 4) -------------------------------------------------------
    def initial_v(self):
        return np.zeros(self.lay.n_z + self.lay.n_eta)

    def solve(self, v0=None, tol=1e-4, max_iters=5000, method="spock", m=AA_MEMORY,
              max_backtracks=30, rank_tol=1e-10, log=None, aa="householder"):
        """Alg. 4 (SPOCK) or, with method="cp", plain CP iterates v <- T(v).

        Readings: the averagedness constant in rho is that of a firmly
        nonexpansive T (1/2), so rho = ||r~||_M^2 - <r~, v~ - v>_M; the
        backtracking of tau is capped at max_backtracks trials, after which the
        step falls back to v <- T(v); c2^k uses the outer counter k;
        termination when ||v - T(v)||_inf <= tol (eps_rel = 0). After a K1 step
        the residual r~ of the accepted point is the next iterate's residual.
        `log` (a list, optional) receives (k, n_T, ||r||_inf) at every outer
        iteration. aa="householder" factorises the Anderson least-squares
        problem afresh at every iteration, aa="qr_update" keeps its QR
        factorisation and updates it (QRMemory).
        """
        v = self.initial_v() if v0 is None else np.array(v0, dtype=np.float64)
        tv = self.T(v)
        n_T = 1
        r = v - tv
        events = []
        if method == "cp":
            k = 0
            while k < max_iters and np.max(np.abs(r)) > tol:
                v = tv
                tv = self.T(v)
                n_T += 1
                r = v - tv
                k += 1
            return self._result(v, tv, k, n_T, events)
        zeta = self.M_norm(r)
        omega_safe = zeta
        S, Y = [], []
        qrm = self.QRMemory(m) if aa == "qr_update" else None
        v_prev = r_prev = None
        k = 0
        while True:
            if log is not None:
                log.append((k, n_T, float(np.max(np.abs(r)))))
            if np.max(np.abs(r)) <= tol or k >= max_iters:
                break
            if v_prev is not None:
                if qrm is not None:
                    qrm.push(v - v_prev, r - r_prev)
                else:
                    S.append(v - v_prev)
                    Y.append(r - r_prev)
                    if len(S) > m:
                        S.pop(0); Y.pop(0)
            if qrm is not None:
                psi = qrm.direction(r, k, rank_tol)
            else:
                psi = self.aa_direction(r, S, Y, k, m, rank_tol)
            omega = self.M_norm(r)
            v_prev, r_prev = v, r
            if omega <= C0 * zeta:
                v = v + psi
                zeta = omega
                tv = self.T(v); n_T += 1
                r = v - tv
                events.append((k, "K0", 0))
            else:
                tau = 1.0
                accepted = False
                for bt in range(max_backtracks):
                    vt = v + tau * psi
                    tvt = self.T(vt); n_T += 1
                    rt = vt - tvt
                    omt = self.M_norm(rt)
                    if (omega <= omega_safe and omt <= C1 * omega) or omt == 0.0:
                        v, tv, r = vt, tvt, rt
                        omega_safe = omt + C2 ** k
                        events.append((k, "K1", bt))
                        accepted = True
                        break
                    rho = omt ** 2 - self.M_inner(rt, vt - v)
                    if rho >= SIGMA * omt * omega:
                        v = v - LAMBDA * rho / omt ** 2 * rt
                        tv = self.T(v); n_T += 1
                        r = v - tv
                        events.append((k, "K2", bt))
                        accepted = True
                        break
                    tau *= BETA
                if not accepted:
                    v = v_prev - r_prev     # = T(v_prev)
                    tv = self.T(v); n_T += 1
                    r = v - tv
                    events.append((k, "FB", max_backtracks))
            k += 1
        return self._result(v, tv, k, n_T, events)

    # -- results and diagnostics (Sec. 5.3) -----------------------------------
    def _result(self, v, tv, iters, n_T, events):
        nz = self.lay.n_z
        r = v - tv
        zp, etap = tv[:nz], tv[nz:]
        dz, de = v[:nz] - zp, v[nz:] - etap
        xi1 = dz / self.alpha - self.apply_Lt(de)
        xi2 = de / self.alpha - self.apply_L(dz)
        Lz = self.apply_L(zp)
        infeas = Lz - self.proj_S3(Lz)
        gap = abs(float(etap @ Lz) - self.support_S3(etap))
        s0, x, u, y, tau, s = self.split_z(zp)
        x_un = x / self.Snode
        u_un = u / self.Su[None, :]
        return dict(v=v, Tv=tv, iters=iters, n_T=n_T, events=events,
                    res_inf=float(np.max(np.abs(r))),
                    xi1=float(np.max(np.abs(xi1))), xi2=float(np.max(np.abs(xi2))),
                    infeas=float(np.max(np.abs(infeas))), gap=gap,
                    risk=float(s0), x=x_un, u=u_un,
                    nested_risk=self.nested_risk(x_un, u_un))

    def support_S3(self, eta):
        """Support function of S3 at eta, for eta in dom g* (Sec. 5.3 uses g*):
        cone pieces contribute 0, translated cones <eta, a>, boxes
        sum max(eta lo, eta hi), balls r ||eta||."""
        tr, lay = self.tree, self.lay
        nx, nu = self.nx, self.nu
        val = 0.0
        if self.n_c:
            C = eta[lay.e_c:lay.e_q].reshape(tr.n_nl, self.n_c)
            nb = self.n_box
            val += float(np.sum(np.maximum(C[:, :nb] * self.box_lo, C[:, :nb] * self.box_hi)))
            nbl = nb + (nu if self.has_uball else 0)
            if self.has_uball:
                val += float(np.sum(self.ball_r * np.linalg.norm(C[:, nb:nbl], axis=1)))
            if self.n_g:
                val += float(np.sum(np.maximum(C[:, nbl:] * self.gen_lo, C[:, nbl:] * self.gen_hi)))
        w = nx + nu + 2
        Qb = eta[lay.e_q:lay.e_cN].reshape(tr.n - 1, w)
        val += float(np.sum(Qb * self.a_q))
        if self.n_cN:
            CN = eta[lay.e_cN:lay.e_qN].reshape(tr.n_l, self.n_cN)
            val += float(np.sum(np.maximum(CN * self.boxN_lo, CN * self.boxN_hi)))
        QN = eta[lay.e_qN:self.e_l1].reshape(tr.n_l, nx + 2)
        val += float(np.sum(QN * self.a_qN))
        if self.soft is not None:  # translated cone <eta, a>; rows z - theta >= .. : h lo for h <= 0
            d = nx + nu
            B = eta[self.e_sf:].reshape(tr.n_nl, 3 * d + 2)
            val += float(np.sum(0.5 * B[:, d] - 0.5 * B[:, d + 1]))
            H = B[:, 2 * d + 2:]
            val += float(np.sum(np.where(H <= 0.0, H * self.soft_lo, np.inf)))
        return val                 # the l1 rows and theta >= 0 are cones: they contribute 0

    def nested_values(self, x, u):
        """Cost-to-go V^i of a trajectory under the nested risk (Eq.
        original-problem) with the original (unscaled) costs, and the
        maximising conditional weights mu^c of every non-root node (the
        maximiser of the node's risk, AV@R or the total-variation ball, over
        the children of its ancestor, Sec. 3.3-3.4)."""
        P, tr = self.P, self.tree
        V = np.zeros(tr.n)
        mu = np.zeros(tr.n)
        mu[0] = 1.0
        for jj in range(tr.n_l):
            j = tr.n_nl + jj
            V[j] = self.terminal_cost(jj, x[j])
        for t in range(tr.N - 1, -1, -1):
            for i in tr.nodes_at[t]:
                ch = tr.children[i]
                Z = []
                for c in ch:
                    Z.append(self.edge_cost(c, x[i], u[i]) + V[c])
                Z = np.asarray(Z)
                if self.tv is not None:
                    V[i] = tv_risk(Z, tr.prob[ch], self.tv[i])
                    mu[ch] = tv_maximiser(Z, tr.prob[ch], self.tv[i])
                else:
                    V[i] = avar(Z, tr.prob[ch], self.avar_level[i])
                    mu[ch] = avar_maximiser(Z, tr.prob[ch], self.avar_level[i])
        return V, mu

    def path_weights(self, x, u):
        """Product of the maximising conditional weights mu along the path from
        the root to every node: the nodes with positive weight are those whose
        costs enter the nested risk value; elsewhere the optimal inputs need
        not be unique (an AV@R level below one can give children weight 0)."""
        _, mu = self.nested_values(x, u)
        w = np.ones(self.tree.n)
        for i in range(1, self.tree.n):
            w[i] = w[self.tree.anc[i]] * mu[i]
        return w

    def edge_cost(self, c, x, u):
        """l^c(x, u) = x'Q^c x + u'R^c u + q^c'x + r^c'u (+ lambda_0 ||(x, u)||_1,
        Prop. 2) on the ancestor's state and input (Sec. 3.2,
        quadratic-plus-linear costs), original data."""
        P = self.P
        Qc = P.Q[c - 1] if np.ndim(P.Q) == 3 else np.diag(P.Q[c - 1])
        Rc = P.R[c - 1] if np.ndim(P.R) == 3 else np.diag(P.R[c - 1])
        val = x @ Qc @ x + u @ Rc @ u
        if getattr(P, "q", None) is not None:
            val += P.q[c - 1] @ x
        if getattr(P, "r", None) is not None:
            val += P.r[c - 1] @ u
        if self.l1:
            val += self.l1 * (np.sum(np.abs(x)) + np.sum(np.abs(u)))
        if self.soft is not None:
            val += float(np.sum(np.maximum(0.0, np.concatenate([x, u]) - self.soft) ** 2))
        return float(val)

    def terminal_cost(self, jj, x):
        """l_N^j(x) = x'Q_N^j x + q_N^j'x for the jj-th leaf."""
        P = self.P
        QN = P.QN[jj] if np.ndim(P.QN) == 3 else np.diag(P.QN[jj])
        val = x @ QN @ x
        if getattr(P, "qN", None) is not None:
            val += P.qN[jj] @ x
        return float(val)

    def nested_risk(self, x, u):
        """Nested risk of a trajectory (Eq. original-problem) with the original
        (unscaled) costs: leaves V = l_N(x); a non-leaf node takes AV@R_{a_i}
        over its children of l^c(x^i, u^i) + V^c (Sec. 3.4)."""
        V, _ = self.nested_values(x, u)
        return float(V[0])
