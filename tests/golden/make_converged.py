"""Writes the converged-solution golden files of the benchmark workloads.

Calls only the FP64 oracle (oracle/) on the seeded generators
(paper_2505_12078_b300.synth): nothing here touches the CUDA path. The oracle
runs SPOCK (Alg. 4 with Anderson directions, Alg. 3) from z = eta = 0 to
||v - T(v)||_inf <= 1e-4 (Sec. 5.3 with eps_rel = 0) and the file records

  iters, n_T, the K0/K1/K2/fallback counts, the residual after every outer
  iteration, alpha, the risk value s0, the unscaled x and u of T(v) at exit,
  the path weight of every node under the maximising AV@R weights of the
  nested risk (Sec. 3.3-3.4), and the diagnostics of Sec. 5.3 (xi1, xi2,
  primal infeasibility, complementarity gap, nested risk of the trajectory).

With --tight TOL the solve continues (warm, from the 1e-4 iterate) to TOL and
the tighter x, u and risk are stored beside the others: a reference closer to
the exact optimum than either 1e-4 solution.

Usage: python -m tests.golden.make_converged large_raocp [--tight 1e-6]
       python -m tests.golden.make_converged tree_sweep_b4
The large problem took 60 minutes to 1e-4 (16 134 iterations) and 3.5 hours
more to 1e-6 (55 702 iterations) on two cores of a CPU host.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle.spock_oracle import Oracle  # noqa: E402
from paper_2505_12078_b300 import synth  # noqa: E402

WORKLOADS = {
    "large_raocp": synth.large_raocp,
    "tree_sweep_b4": lambda: synth.tree_sweep(4),
    "tree_sweep_b2": lambda: synth.tree_sweep(2),
    "tree_sweep_b8": lambda: synth.tree_sweep(8),
    "small_raocp": synth.small_raocp,
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(WORKLOADS))
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iters", type=int, default=200000)
    ap.add_argument("--tight", type=float, default=0.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    p = WORKLOADS[a.workload]()
    t0 = time.time()
    o = Oracle(p)
    log = []
    res = o.solve(tol=a.tol, max_iters=a.max_iters, log=log)
    t1 = time.time()
    kinds = [e[1] for e in res["events"]]
    w = o.path_weights(res["x"], res["u"])
    out = dict(
        workload=a.workload, tol=a.tol, alpha=o.alpha, normL=o.normL,
        iters=res["iters"], n_T=res["n_T"],
        n_K0=kinds.count("K0"), n_K1=kinds.count("K1"), n_K2=kinds.count("K2"),
        n_FB=kinds.count("FB"),
        log=np.asarray(log, dtype=np.float64),
        risk=res["risk"], res_inf=res["res_inf"], x=res["x"], u=res["u"], path_weight=w,
        xi1=res["xi1"], xi2=res["xi2"], infeas=res["infeas"], gap=res["gap"],
        nested_risk=res["nested_risk"], seconds=t1 - t0,
    )
    print(f"{a.workload}: {res['iters']} iterations, {res['n_T']} T, res {res['res_inf']:.3e}, "
          f"risk {res['risk']:.8f}, {t1 - t0:.0f} s", flush=True)
    if a.tight > 0:
        log2 = []
        r2 = o.solve(v0=res["v"], tol=a.tight, max_iters=a.max_iters, log=log2)
        out.update(tight_tol=a.tight, tight_iters=r2["iters"], tight_risk=r2["risk"],
                   tight_res_inf=r2["res_inf"], tight_x=r2["x"], tight_u=r2["u"],
                   tight_log=np.asarray(log2, dtype=np.float64),
                   tight_path_weight=o.path_weights(r2["x"], r2["u"]))
        print(f"  tight: {r2['iters']} more iterations, res {r2['res_inf']:.3e}, "
              f"risk {r2['risk']:.10f}, {time.time() - t1:.0f} s", flush=True)
    path = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                 f"{a.workload}_converged.npz")
    np.savez_compressed(path, **out)
    print("wrote", path)


if __name__ == "__main__":
    main()
