"""Small hand-built problems used by the tests (built from the seeded
generators' building blocks; no solver arithmetic here)."""
import math

import numpy as np

from paper_2505_12078_b300 import synth


def unconstrained(branching, nx, nu, seed, avar=1.0, c_scale=0.0, spread=0.3):
    """Tree with the given branching per stage, random dense A, B, random
    positive diagonal weights, no constraints, AV@R level `avar` everywhere."""
    rng = np.random.default_rng(seed)
    anc, prob = synth.tree_from_branching(branching, rng)
    n = len(anc)
    N = len(branching)
    n_leaf = int(np.prod(branching))
    A = np.eye(nx) + spread * rng.standard_normal((n - 1, nx, nx))
    B = rng.standard_normal((n - 1, nx, nu))
    c = c_scale * rng.standard_normal((n - 1, nx))
    Qd = rng.uniform(0.5, 2.0, (n - 1, nx))
    Rd = rng.uniform(0.5, 2.0, (n - 1, nu))
    QNd = rng.uniform(0.5, 2.0, (n_leaf, nx))
    x0 = rng.uniform(-1.0, 1.0, nx)
    return synth.RAOCP(f"unconstrained_{branching}", anc, prob, nx, nu, A, B, c, Qd, Rd, QNd,
                       None, None, None, None, None, np.full(n - n_leaf, float(avar)), x0,
                       meta=dict(N=N))


def constrained(branching, nx, nu, seed, avar=0.5, uball=None):
    """Tree with the small_raocp generators (box on x and u, optional ball on u)."""
    rng = np.random.default_rng(seed)
    N = len(branching)
    k = sum(1 for b in branching if b > 1)
    b = max(branching)
    p = synth.random_tree_raocp(rng, nx, nu, N, b, k, avar, name=f"constrained_{branching}",
                                uball=uball)
    return p


def from_spec(d, name="golden"):
    """Problem of a golden-file spec: tree (anc, prob), the same A and B on
    every edge, per-node diagonal weights, x/u boxes, u ball, one AV@R level."""
    anc = np.asarray(d["anc"], dtype=np.int32)
    prob = np.asarray(d["prob"], dtype=np.float64)
    n = len(anc)
    nx, nu = int(d["nx"]), int(d["nu"])
    st = np.zeros(n, dtype=np.int64)
    for i in range(1, n):
        st[i] = st[anc[i]] + 1
    n_leaf = int(np.sum(st == st.max()))
    n_nl = n - n_leaf
    A = np.broadcast_to(np.asarray(d["A_all"], dtype=np.float64), (n - 1, nx, nx)).copy()
    B = np.broadcast_to(np.asarray(d["B_all"], dtype=np.float64), (n - 1, nx, nu)).copy()
    xb, ub = float(d["x_bound"]), float(d["u_bound"])
    return synth.RAOCP(
        name, anc, prob, nx, nu, A, B, np.zeros((n - 1, nx)),
        np.asarray(d["Q"], dtype=np.float64), np.asarray(d["R"], dtype=np.float64),
        np.asarray(d["QN"], dtype=np.float64),
        np.full((n, nx), -xb), np.full((n, nx), xb), np.full((n_nl, nu), -ub), np.full((n_nl, nu), ub),
        np.full(n_nl, float(d["u_ball"])), np.full(n_nl, float(d["avar"])),
        np.asarray(d["x0"], dtype=np.float64), meta=dict(N=int(st.max())))


def general(branching, nx, nu, seed, avar=1.0, dense=True, linear=True, n_g=0, n_gN=0, box=False,
            spread=0.1, g_scale=0.6, lin_scale=0.3):
    """Tree with dense positive definite Q, R, Q_N (or random diagonals),
    linear cost terms q, r, q_N, and optional general constraint rows
    g_lo <= Gx x + Gu u <= g_hi (non-leaf) and gN_lo <= GN x <= gN_hi (leaves)
    with random Gx, Gu, GN and bounds of random width around zero."""
    rng = np.random.default_rng(seed)
    anc, prob = synth.tree_from_branching(branching, rng)
    n = len(anc)
    n_leaf = int(np.prod(branching))
    n_nl = n - n_leaf

    def spd(k, m):
        M = rng.standard_normal((k, m, m)) / math.sqrt(m)
        return M @ np.transpose(M, (0, 2, 1)) + 0.5 * np.eye(m)[None]

    A = np.eye(nx) + spread * rng.standard_normal((n - 1, nx, nx))
    B = rng.standard_normal((n - 1, nx, nu))
    if dense:
        Q, R, QN = spd(n - 1, nx), spd(n - 1, nu), spd(n_leaf, nx)
    else:
        Q, R, QN = rng.uniform(0.5, 2.0, (n - 1, nx)), rng.uniform(0.5, 2.0, (n - 1, nu)), \
            rng.uniform(0.5, 2.0, (n_leaf, nx))
    x0 = rng.uniform(-1.0, 1.0, nx)
    p = synth.RAOCP(f"general_{branching}", anc, prob, nx, nu, A, B, np.zeros((n - 1, nx)), Q, R, QN,
                    None, None, None, None, None, np.full(n_nl, float(avar)), x0, meta=dict(N=len(branching)))
    if box:
        p.x_lo, p.x_hi = np.full((n, nx), -5.0), np.full((n, nx), 5.0)
        p.u_lo, p.u_hi = np.full((n_nl, nu), -2.0), np.full((n_nl, nu), 2.0)
    if linear:
        p.q = lin_scale * rng.standard_normal((n - 1, nx))
        p.r = lin_scale * rng.standard_normal((n - 1, nu))
        p.qN = lin_scale * rng.standard_normal((n_leaf, nx))
    # general rows: bounds of random width around the rows' values on the
    # trajectory with u = 0 (so every problem is feasible)
    xr = np.zeros((n, nx))
    xr[0] = x0
    for c in range(1, n):
        xr[c] = A[c - 1] @ xr[anc[c]]
    if n_g:
        p.Gx = rng.standard_normal((n_g, nx))
        p.Gu = rng.standard_normal((n_g, nu))
        mid = xr[:n_nl] @ p.Gx.T
        p.g_lo = mid - g_scale * rng.uniform(0.5, 1.5, (n_nl, n_g))
        p.g_hi = mid + g_scale * rng.uniform(0.5, 1.5, (n_nl, n_g))
    if n_gN:
        p.GN = rng.standard_normal((n_gN, nx))
        mid = xr[n_nl:] @ p.GN.T
        p.gN_lo = mid - g_scale * rng.uniform(0.5, 1.5, (n_leaf, n_gN))
        p.gN_hi = mid + g_scale * rng.uniform(0.5, 1.5, (n_leaf, n_gN))
    return p
