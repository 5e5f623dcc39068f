"""Small hand-built problems used by the tests (built from the seeded
generators' building blocks; no solver arithmetic here)."""
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
