"""Seeded synthetic scenario-tree RAOCP generators.

This module only draws random problem data (trees, dynamics, costs, bounds,
initial states). It holds none of the solver's arithmetic, so both the CPU
oracle and the CUDA path take their inputs from it.

Problem data follow the problem statement of the paper (Sec. 3.1-3.5):
  * a scenario tree in breadth-first order (stage-major, children of a node
    contiguous), given by the ancestor of every node and the conditional
    probability of each node given its ancestor (Sec. 3.2);
  * per non-root node c the edge dynamics x^c = A^c x^anc + B^c u^anc + c^c
    (Eq. finite-horizon-evolution) and the edge cost weights Q^c, R^c applied
    to the ancestor's state and input (Sec. 3.2, "Quadratic-plus-linear
    costs"); per leaf the terminal weight Q_N;
  * box constraints on x at every node and on u at every non-leaf node, and
    optionally a Euclidean-ball constraint on u (Eq. constraints);
  * an AV@R level per non-leaf node (Sec. 3.3).

Cost weights are diagonal (every workload here uses diagonal Q, R, Q_N); they
are stored as their diagonals.

Workloads (named by their sizes):
  * small_raocp   : nx=4, nu=2, N=5, 2-way at stages 0-2 (31 nodes), AV@R 0.5
  * large_raocp   : nx=50, nu=25, N=15, 3-way at stages 0-3 (1012 nodes), AV@R 0.3
  * tree_sweep(b) : nx=20, nu=10, N=12, b-way at the first k stages (~4096 nodes)
  * batch(count)  : uneven problems, nx~U{4..64}, nu=nx//2, N~U{5..20}
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class RAOCP:
    """One scenario-tree risk-averse optimal control problem (host arrays)."""

    name: str
    anc: np.ndarray          # int32 [n]; anc[0] = -1
    prob: np.ndarray         # float64 [n]; conditional probability given ancestor, prob[0] = 1
    nx: int
    nu: int
    A: np.ndarray            # float64 [n-1, nx, nx]; entry c-1 holds A^c
    B: np.ndarray            # float64 [n-1, nx, nu]
    c: np.ndarray            # float64 [n-1, nx]
    Q: np.ndarray            # float64 [n-1, nx]  diagonal of Q^c (edge cost on x^anc(c))
    R: np.ndarray            # float64 [n-1, nu]  diagonal of R^c (edge cost on u^anc(c))
    QN: np.ndarray           # float64 [n_leaf, nx] diagonal of Q_N^j
    x_lo: Optional[np.ndarray]  # float64 [n, nx] or None
    x_hi: Optional[np.ndarray]
    u_lo: Optional[np.ndarray]  # float64 [n_nonleaf, nu] or None
    u_hi: Optional[np.ndarray]
    u_ball: Optional[np.ndarray]  # float64 [n_nonleaf] radius or None
    avar: np.ndarray         # float64 [n_nonleaf], AV@R level in [0, 1]
    x0: np.ndarray           # float64 [nx]
    meta: dict = field(default_factory=dict)
    # Optional parts of the problem statement (Sec. 3.1-3.2); None = absent.
    # Q, R, QN above may also be full matrices [.., nx, nx] / [.., nu, nu]
    # (symmetric positive definite) instead of diagonals.
    q: Optional[np.ndarray] = None      # float64 [n-1, nx] linear edge cost on x^anc(c)
    r: Optional[np.ndarray] = None      # float64 [n-1, nu] linear edge cost on u^anc(c)
    qN: Optional[np.ndarray] = None     # float64 [n_leaf, nx] linear terminal cost
    Gx: Optional[np.ndarray] = None     # float64 [n_g, nx] general rows at every non-leaf node:
    Gu: Optional[np.ndarray] = None     # float64 [n_g, nu]   g_lo <= Gx x + Gu u <= g_hi
    g_lo: Optional[np.ndarray] = None   # float64 [n_nonleaf, n_g]
    g_hi: Optional[np.ndarray] = None
    GN: Optional[np.ndarray] = None     # float64 [n_gN, nx] general rows at every leaf:
    gN_lo: Optional[np.ndarray] = None  # float64 [n_leaf, n_gN]   gN_lo <= GN x <= gN_hi
    gN_hi: Optional[np.ndarray] = None
    l1: Optional[float] = None          # lambda_0 >= 0 of an l1 term lambda_0 ||(x^anc, u^anc)||_1 added
                                        # to every edge cost (Prop. 2); None or 0 = none
    soft_max: Optional[np.ndarray] = None   # float64 [nx + nu] finite: every edge cost gets the soft-constraint
                                        # penalty ||max(0, (x^anc, u^anc) - soft_max)||^2 (the quadratic
                                        # penalty after Prop. 2); None = none
    tv: Optional[np.ndarray] = None     # float64 [n_nonleaf] radius r >= 0: the risk of every non-leaf node
                                        # is then the worst expectation over {mu in the simplex :
                                        # ||mu - p||_1 <= r} (a conic risk with F != 0, Sec. 3.3)
                                        # instead of AV@R; None = AV@R with the levels in avar

    @property
    def n(self) -> int:
        return int(self.anc.shape[0])

    @property
    def stage(self) -> np.ndarray:
        st = np.zeros(self.n, dtype=np.int64)
        for i in range(1, self.n):
            st[i] = st[self.anc[i]] + 1
        return st

    @property
    def N(self) -> int:
        return int(self.stage.max())

    @property
    def n_leaf(self) -> int:
        st = self.stage
        return int(np.sum(st == st.max()))

    @property
    def n_nonleaf(self) -> int:
        return self.n - self.n_leaf


def tree_from_branching(branching, rng: np.random.Generator):
    """Breadth-first tree in which every node of stage t has branching[t] children.

    Conditional probabilities of the children of a branching node are drawn
    from Dirichlet(1); a single child has probability 1.
    """
    anc = [-1]
    prob = [1.0]
    frontier = [0]
    for b in branching:
        nxt = []
        for parent in frontier:
            p = rng.dirichlet(np.ones(b)) if b > 1 else np.ones(1)
            for k in range(b):
                anc.append(parent)
                prob.append(float(p[k]))
                nxt.append(len(anc) - 1)
        frontier = nxt
    return np.asarray(anc, dtype=np.int32), np.asarray(prob, dtype=np.float64)


def _spectral_rescale(G: np.ndarray, rho: float) -> np.ndarray:
    r = np.max(np.abs(np.linalg.eigvals(G)))
    return G * (rho / r)


def _dyn_identity_plus(rng, n_edges, nx, nu):
    """A = I + 0.1 G, G ~ N(0,1) rescaled to spectral radius 1.05; B ~ N(0,1)/sqrt(nu)."""
    G = rng.standard_normal((n_edges, nx, nx))          # the same draws, edge after edge
    r = np.max(np.abs(np.linalg.eigvals(G)), axis=-1)   # spectral radius of every G at once
    A = np.eye(nx) + 0.1 * G * (1.05 / r)[:, None, None]
    B = rng.standard_normal((n_edges, nx, nu)) / math.sqrt(nu)
    return A, B


def _make(name, anc, prob, nx, nu, A, B, avar, x0, *, xbound=5.0, ubound=2.0,
          uball=None, Qd=1.0, Rd=0.1, QNd=1.0, meta=None) -> RAOCP:
    n = anc.shape[0]
    st = np.zeros(n, dtype=np.int64)
    for i in range(1, n):
        st[i] = st[anc[i]] + 1
    n_leaf = int(np.sum(st == st.max()))
    n_nl = n - n_leaf
    return RAOCP(
        name=name, anc=anc, prob=prob, nx=nx, nu=nu, A=A, B=B,
        c=np.zeros((n - 1, nx)),
        Q=np.full((n - 1, nx), Qd), R=np.full((n - 1, nu), Rd),
        QN=np.full((n_leaf, nx), QNd),
        x_lo=np.full((n, nx), -xbound) if xbound is not None else None,
        x_hi=np.full((n, nx), xbound) if xbound is not None else None,
        u_lo=np.full((n_nl, nu), -ubound) if ubound is not None else None,
        u_hi=np.full((n_nl, nu), ubound) if ubound is not None else None,
        u_ball=np.full(n_nl, float(uball)) if uball is not None else None,
        avar=np.broadcast_to(np.asarray(avar, dtype=np.float64), (n_nl,)).copy(),
        x0=x0, meta=dict(meta or {}),
    )


def small_raocp(seed: int = 1) -> RAOCP:
    """nx=4, nu=2, N=5, 2-way branching at stages 0-2 (8 scenarios, 31 nodes), AV@R 0.5,
    |x|_inf <= 5, |u|_inf <= 2, Q = I, R = 0.1 I, Q_N = I, x0 ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    nx, nu, N = 4, 2, 5
    anc, prob = tree_from_branching([2, 2, 2, 1, 1], rng)
    A, B = _dyn_identity_plus(rng, anc.shape[0] - 1, nx, nu)
    x0 = rng.uniform(-1.0, 1.0, nx)
    return _make("small_raocp_nx4_nu2_N5_31nodes", anc, prob, nx, nu, A, B, 0.5, x0,
                 meta=dict(seed=seed, N=N))


def large_raocp(seed: int = 2) -> RAOCP:
    """nx=50, nu=25, N=15, 3-way at stages 0-3 (81 scenarios, 1012 nodes), AV@R 0.3,
    box constraints on x (5) and u (2) plus ||u||_2 <= 3 at every non-leaf node.

    Dynamics per node: A_nom + 0.05 N(0,1), A_nom ~ N(0,1) rescaled to spectral
    radius 1.02; B ~ N(0,1)/sqrt(nu)."""
    rng = np.random.default_rng(seed)
    nx, nu, N = 50, 25, 15
    anc, prob = tree_from_branching([3, 3, 3, 3] + [1] * (N - 4), rng)
    n = anc.shape[0]
    A_nom = _spectral_rescale(rng.standard_normal((nx, nx)), 1.02)
    A = A_nom[None, :, :] + 0.05 * rng.standard_normal((n - 1, nx, nx))
    B = rng.standard_normal((n - 1, nx, nu)) / math.sqrt(nu)
    x0 = rng.uniform(-1.0, 1.0, nx)
    return _make("large_raocp_nx50_nu25_N15_1012nodes", anc, prob, nx, nu, A, B, 0.3, x0,
                 uball=3.0, meta=dict(seed=seed, N=N))


def tree_sweep_depth(b: int, N: int = 12, target: int = 4096) -> int:
    """Number of branching stages k for which a b-way tree of horizon N has a
    node count closest (in log ratio) to `target`."""
    best, best_k = None, 1
    for k in range(1, N + 1):
        n = sum(b ** min(t, k) for t in range(N + 1))
        d = abs(math.log(n / float(target)))
        if best is None or d < best:
            best, best_k = d, k
    return best_k


def tree_sweep(b: int, seed: int = 3) -> RAOCP:
    """nx=20, nu=10, N=12, b-way branching at the first k stages (k keeps the node
    count near 4096), dynamics/costs/constraints as in small_raocp, AV@R 0.5."""
    rng = np.random.default_rng(seed * 100 + b)
    nx, nu, N = 20, 10, 12
    k = tree_sweep_depth(b)
    anc, prob = tree_from_branching([b] * k + [1] * (N - k), rng)
    A, B = _dyn_identity_plus(rng, anc.shape[0] - 1, nx, nu)
    x0 = rng.uniform(-1.0, 1.0, nx)
    return _make(f"tree_sweep_b{b}_k{k}_nx20_nu10_N12_{anc.shape[0]}nodes", anc, prob, nx, nu,
                 A, B, 0.5, x0, meta=dict(seed=seed, N=N, b=b, k=k))


def random_tree_raocp(rng: np.random.Generator, nx: int, nu: int, N: int, b: int, k: int,
                      avar: float, name: str = "random", uball=None) -> RAOCP:
    """Tree with b-way branching at the first k stages, dynamics/costs/bounds as in
    small_raocp."""
    anc, prob = tree_from_branching([b] * k + [1] * (N - k), rng)
    A, B = _dyn_identity_plus(rng, anc.shape[0] - 1, nx, nu)
    x0 = rng.uniform(-1.0, 1.0, nx)
    return _make(name, anc, prob, nx, nu, A, B, avar, x0, uball=uball,
                 meta=dict(N=N, b=b, k=k))


def batch_specs(count: int = 512, seed: int = 4):
    """Size draws of the uneven batch: nx~U{4..64}, nu=nx//2, N~U{5..20},
    b~U{2,3,4} at the first k~U{1..min(4,N)} stages, AV@R level ~U[0.2,1]."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        nx = int(rng.integers(4, 65))
        N = int(rng.integers(5, 21))
        b = int(rng.integers(2, 5))
        k = int(rng.integers(1, min(4, N) + 1))
        a = float(rng.uniform(0.2, 1.0))
        specs.append(dict(nx=nx, nu=max(1, nx // 2), N=N, b=b, k=k, avar=a,
                          seed=int(rng.integers(0, 2**31 - 1))))
    return specs


def batch_problem(spec: dict, index: int = 0) -> RAOCP:
    rng = np.random.default_rng(spec["seed"])
    return random_tree_raocp(rng, spec["nx"], spec["nu"], spec["N"], spec["b"], spec["k"],
                             spec["avar"], name=f"batch{index}")


def batch(count: int = 512, seed: int = 4):
    return [batch_problem(s, i) for i, s in enumerate(batch_specs(count, seed))]


def case_study_1(seed: int = 0, nu_max: int = 64, nv_range=(1e3, 1e5)) -> RAOCP:
    """Random RAOCP of the paper's first case study (Sec. 8.1, problem
    statement):
      * N ~ U{5..15}; (n_b, n_w, n_u) uniform on {1 <= b <= 3, 2 <= w <= 10,
        10 <= u <= nu_max} subject to n_v = n_x |nodes(0, N)| + n_u |nodes(0, N-1)|
        in nv_range (rejection sampling); n_x = 2 n_u;
      * scenario tree: n_w children at each of the first n_b stages, one child
        after; the children of a branching node are the events w = 1..n_w with
        one base probability vector pi ~ U(simplex), a non-branching child keeps
        its parent's event;
      * dynamics per event: A(w) = I + A^w, B(w) = B + B^w with B_ij ~ N(0, 1),
        A^w_ij, B^w_ij ~ N(0, 0.01) (variance);
      * costs per event: Q(w) = (Q0 + Q^w)(Q0 + Q^w)', R(w) = (R0 + R^w)(R0 + R^w)'
        with Q0 = diag(U[0, 0.1]), R0 = diag(U[0, 100]), Q^w_ij, R^w_ij ~
        N(0, 0.01); Q_N = Q0 (full matrices throughout);
      * boxes -xbar <= x <= xbar, -ubar <= u <= ubar, xbar ~ U[1, 2]^nx,
        ubar ~ U[0, 0.1]^nu; AV@R_gamma with gamma ~ U[0, 1];
      * x0_i ~ U[-xbar_i/2, xbar_i/2].
    The paper allows n_u up to 300; n_u is capped at nu_max so that n_x = 2 n_u
    stays within the library's compiled limit (n_x <= 128)."""
    rng = np.random.default_rng(seed)
    while True:
        N = int(rng.integers(5, 16))
        b = int(rng.integers(1, 4))
        w = int(rng.integers(2, 11))
        nu = int(rng.integers(10, nu_max + 1))
        nx = 2 * nu
        b_eff = min(b, N)
        nodes_all = sum(w ** min(t, b_eff) for t in range(N + 1))
        nodes_nl = sum(w ** min(t, b_eff) for t in range(N))
        nv = nx * nodes_all + nu * nodes_nl
        if nv_range[0] <= nv <= nv_range[1]:
            break
    pi = rng.dirichlet(np.ones(w))
    # tree with events
    anc, prob, event = [-1], [1.0], [0]
    frontier = [0]
    for t in range(N):
        nxt = []
        for parent in frontier:
            if t < b_eff:
                for k in range(w):
                    anc.append(parent); prob.append(float(pi[k])); event.append(k)
                    nxt.append(len(anc) - 1)
            else:
                anc.append(parent); prob.append(1.0); event.append(event[parent])
                nxt.append(len(anc) - 1)
        frontier = nxt
    anc = np.asarray(anc, dtype=np.int32)
    prob = np.asarray(prob, dtype=np.float64)
    n = len(anc)
    n_leaf = len(frontier)
    n_nl = n - n_leaf
    B0 = rng.standard_normal((nx, nu))
    A_w = np.eye(nx)[None] + 0.1 * rng.standard_normal((w, nx, nx))
    B_w = B0[None] + 0.1 * rng.standard_normal((w, nx, nu))
    q0 = rng.uniform(0.0, 0.1, nx)
    r0 = rng.uniform(0.0, 100.0, nu)
    Qf = np.diag(q0)[None] + 0.1 * rng.standard_normal((w, nx, nx))
    Rf = np.diag(r0)[None] + 0.1 * rng.standard_normal((w, nu, nu))
    Q_w = Qf @ np.transpose(Qf, (0, 2, 1))
    R_w = Rf @ np.transpose(Rf, (0, 2, 1))
    ev = np.asarray(event[1:], dtype=np.int64)
    A = A_w[ev].copy()
    B = B_w[ev].copy()
    Q = Q_w[ev].copy()
    R = R_w[ev].copy()
    QN = np.broadcast_to(np.diag(q0), (n_leaf, nx, nx)).copy()
    xbar = rng.uniform(1.0, 2.0, nx)
    ubar = rng.uniform(0.0, 0.1, nu)
    gamma = float(rng.uniform(0.0, 1.0))
    x0 = rng.uniform(-0.5 * xbar, 0.5 * xbar)
    return RAOCP(
        name=f"case_study_1_s{seed}_N{N}_b{b_eff}_w{w}_nu{nu}_nv{nv}", anc=anc, prob=prob, nx=nx, nu=nu,
        A=A, B=B, c=np.zeros((n - 1, nx)), Q=Q, R=R, QN=QN,
        x_lo=np.broadcast_to(-xbar, (n, nx)).copy(), x_hi=np.broadcast_to(xbar, (n, nx)).copy(),
        u_lo=np.broadcast_to(-ubar, (n_nl, nu)).copy(), u_hi=np.broadcast_to(ubar, (n_nl, nu)).copy(),
        u_ball=None, avar=np.full(n_nl, gamma), x0=x0,
        meta=dict(seed=seed, N=N, n_b=b_eff, n_w=w, n_v=nv))


def beta_quantile_tree(branching, theta: float = 1.0, phi0: float = 0.1):
    """Scenario tree of the delay process of the paper's second case study
    (Sec. 8.2, sensor-to-controller delay): phi^0 = phi0; the m children of a
    node with value phi are equiprobable and take the quantiles of
    Beta(theta phi, theta (1 - phi)) at the centres (2k - 1)/(2m) of m equal
    intervals of [0, 1] (a single child takes the median), kept within
    [1e-12, 1 - 1e-12]. Returns anc, prob and phi per node."""
    from scipy.stats import beta as _beta
    anc, prob, phi = [-1], [1.0], [float(phi0)]
    frontier = [0]
    for m in branching:
        nxt = []
        for parent in frontier:
            f = phi[parent]
            q = (2.0 * np.arange(1, m + 1) - 1.0) / (2.0 * m)
            vals = _beta.ppf(q, theta * f, theta * (1.0 - f))
            # repeated medians drive phi towards 0, where it underflows and the
            # next Beta is undefined: phi is kept in [1e-12, 1 - 1e-12]
            vals = np.clip(np.nan_to_num(vals, nan=1e-12), 1e-12, 1.0 - 1e-12)
            for k in range(m):
                anc.append(parent)
                prob.append(1.0 / m)
                phi.append(float(vals[k]))
                nxt.append(len(anc) - 1)
        frontier = nxt
    return np.asarray(anc, dtype=np.int32), np.asarray(prob, dtype=np.float64), np.asarray(phi)


def ncs_delay(n: int, shape: str = "wide", N: int = 48, nx: int = 100, nu: int = 50, T: float = 0.005,
              theta: float = 1.0, phi0: float = 0.1, avar: float = 0.95, seed: int = 6) -> RAOCP:
    """Networked control system with a sensor-to-controller delay (Sec. 8.2):
    continuous plant xdot = A_c x + B_c u, A_c = I + diag(a), a_i ~ N(0, 0.01),
    B_c = 0.1 ones(nx, nu), sampled every T with the delay sigma = phi T of the
    Beta-quantile tree; branching [n^2, 1, .., 1] (shape "wide") or
    [n, n, 1, .., 1] ("deep"), the same number of scenarios.

    Discretisation (derived here; the paper cites it without printing it):
    over one period the previous input u_{k-1} acts during [kT, kT + sigma)
    and u_k during [kT + sigma, (k+1)T), so with the augmented state
    xt = (x, u_prev) in R^{nx + nu}
        xt^+ = [[Phi, G1(sigma)], [0, 0]] xt + [[G0(sigma)], [I]] u,
    Phi = e^{A_c T}, G1 = int_0^sigma e^{A_c (T - s)} ds B_c,
    G0 = int_sigma^T e^{A_c (T - s)} ds B_c; A_c is diagonal, so the integrals
    are elementwise (e^{l (T - a)} - e^{l (T - b)}) / l. The delay of the
    transition into a node is that node's sigma.
    Sampling time: the paper prints T = 5, with which A_c ~ I grows by about
    e^5 per period; the input matrix B_c has rank one, so the plant is not
    stabilisable, the unit-weight Riccati recursion of Alg. 1 overflows FP64
    over 48 stages, and ||x||_inf <= 3 cannot hold from x0 = 2. The default
    here is T = 0.005 (the same delay structure sigma = phi T), for which the
    open-loop growth over the horizon stays below 1.5.
    Costs Q = 1e-6 I on xt, R = 0.1 I, Q_N = diag(1_nx, 1e-6 1_nu);
    ||x||_inf <= 3 on the plant part, ||u||_inf <= 0.9 (the u_prev part of xt
    gets the input bound, which it satisfies anyway); x0 = (2, .., 2, 0, .., 0);
    AV@R_avar at every node."""
    rng = np.random.default_rng(seed)
    if shape == "wide":
        branching = [n * n] + [1] * (N - 1)
    elif shape == "deep":
        branching = [n, n] + [1] * (N - 2)
    else:
        raise ValueError("shape is 'wide' or 'deep'")
    anc, prob, phi = beta_quantile_tree(branching, theta, phi0)
    lam = 1.0 + 0.1 * rng.standard_normal(nx)
    Bc = 0.1 * np.ones((nx, nu))
    Phi = np.diag(np.exp(lam * T))
    n_nodes = len(anc)
    na = nx + nu
    A = np.zeros((n_nodes - 1, na, na))
    B = np.zeros((n_nodes - 1, na, nu))
    for c in range(1, n_nodes):
        sig = phi[c] * T
        g1 = (np.exp(lam * T) - np.exp(lam * (T - sig))) / lam
        g0 = (np.exp(lam * (T - sig)) - 1.0) / lam
        A[c - 1, :nx, :nx] = Phi
        A[c - 1, :nx, nx:] = g1[:, None] * Bc
        B[c - 1, :nx, :] = g0[:, None] * Bc
        B[c - 1, nx:, :] = np.eye(nu)
    st = np.zeros(n_nodes, dtype=np.int64)
    for i in range(1, n_nodes):
        st[i] = st[anc[i]] + 1
    n_leaf = int(np.sum(st == st.max()))
    n_nl = n_nodes - n_leaf
    xb = np.concatenate([np.full(nx, 3.0), np.full(nu, 0.9)])
    x0 = np.concatenate([np.full(nx, 2.0), np.zeros(nu)])
    return RAOCP(
        name=f"ncs_delay_{shape}_n{n}_N{N}_nx{nx}_nu{nu}_{n_nodes}nodes", anc=anc, prob=prob, nx=na, nu=nu,
        A=A, B=B, c=np.zeros((n_nodes - 1, na)),
        Q=np.full((n_nodes - 1, na), 1e-6), R=np.full((n_nodes - 1, nu), 0.1),
        QN=np.broadcast_to(np.concatenate([np.ones(nx), np.full(nu, 1e-6)]), (n_leaf, na)).copy(),
        x_lo=np.broadcast_to(-xb, (n_nodes, na)).copy(), x_hi=np.broadcast_to(xb, (n_nodes, na)).copy(),
        u_lo=np.full((n_nl, nu), -0.9), u_hi=np.full((n_nl, nu), 0.9), u_ball=None,
        avar=np.full(n_nl, float(avar)), x0=x0, meta=dict(N=N, n=n, shape=shape, seed=seed))
