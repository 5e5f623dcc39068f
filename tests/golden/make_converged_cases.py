"""Writes tests/golden/converged_cases.json: the optimum of the small parity
cases, for the FP32 converged-solution tests.

Calls only the FP64 oracle (oracle/) on the seeded problem generators of
the tests: nothing here touches the CUDA path. The oracle runs SPOCK (Alg. 4
with Anderson directions, Alg. 3) from z = eta = 0 to ||v - T(v)||_inf <=
1e-7 (Sec. 5.3 with eps_rel = 0) and the file records per case the risk
value s0 and the unscaled u^0 of T(v) at exit, with the iteration count,
and the same for the oracle's own solve to 1e-4 (key "at_1e-4").

Two solutions that each stop at a residual of 1e-4 can sit on opposite sides
of the optimum (on chain_only the oracle's own 1e-4 point has risk 7.8208
against the optimum's 7.8254); a reference this tight keeps the 1e-3 bound of
the tests a statement about the FP32 solution alone. How far a 1e-4 point may
lie from the optimum depends on the problem (on `small` the oracle's own 1e-4
point has u^0 1.19e-3 away from it), so the oracle's 1e-4 solve is stored too.

Usage: python -m tests.golden.make_converged_cases [--all]   (a few minutes, one core)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
for d in (ROOT, os.path.join(ROOT, "tests")):
    if d not in sys.path:
        sys.path.insert(0, d)

from oracle.spock_oracle import Oracle  # noqa: E402
from test_gpu_parity import CASES  # noqa: E402

NAMES = ["small", "ragged_37x19_ball", "chain_only", "full_lin_box", "rows_ball_diag_lin", "team_100x50",
         "l1_box_ball", "tv_box_ball", "soft_box_ball"]
TOL = 1e-7


def main():
    """Solves the cases missing from the file (every case with --all)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "converged_cases.json")
    out = {"tol": TOL, "cases": {}}
    if "--all" not in sys.argv and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name in NAMES:
        if name in out["cases"]:
            continue
        t = time.time()
        o = Oracle(CASES[name]())
        r = o.solve(tol=TOL, max_iters=400000)
        r4 = o.solve(tol=1e-4, max_iters=400000)
        out["cases"][name] = {"iters": int(r["iters"]), "res_inf": float(r["res_inf"]), "risk": float(r["risk"]),
                              "u0": [float(x) for x in r["u"][0]],
                              "at_1e-4": {"iters": int(r4["iters"]), "risk": float(r4["risk"]),
                                          "u0": [float(x) for x in r4["u"][0]]}}
        print(name, r["iters"], f"{time.time() - t:.1f} s", flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
