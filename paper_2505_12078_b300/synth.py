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
