"""Runs parity cases through the bounds-checked library (libspock_checked.so)
in a process of its own (the binding holds one library per process) and
prints one JSON line: per case the one-T and fixed-iteration errors against
the oracle, the branch counts, and the site of the last failed index check
(0: none). Used by tests/test_gpu_checked.py."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for d in (ROOT, os.path.join(ROOT, "tests")):
    if d not in sys.path:
        sys.path.insert(0, d)

import numpy as np  # noqa: E402


def main():
    import torch
    from paper_2505_12078_b300 import build, spock
    from oracle.spock_oracle import Oracle
    from test_gpu_parity import CASES
    build.build()
    lib = spock.load(build.OUT_CHECKED)
    lib.spock_debug_last_check.restype = __import__("ctypes").c_int
    out = {}
    for name in sys.argv[1:]:
        p = CASES[name]()
        o = Oracle(p)
        g = spock.Problem(p)
        g.set_alpha(o.alpha)
        g.set_x0(p.x0)
        rng = np.random.default_rng(11)
        v = rng.standard_normal(o.lay.n_z + o.lay.n_eta)
        ref = o.T(v)
        got, _ = g.T(torch.tensor(v, device="cuda"))
        e1 = float(np.max(np.abs(got.cpu().numpy() - ref)) / max(1.0, float(np.max(np.abs(ref)))))
        r = o.solve(tol=0.0, max_iters=25)
        res = g.solve(p.x0, spock.opts(precision=64, tol=0.0, max_iters=25))
        vi = g.get_iterate(64).cpu().numpy()
        e2 = float(np.max(np.abs(vi - r["v"])) / max(1.0, float(np.max(np.abs(r["v"])))))
        kinds = [e[1] for e in r["events"]]
        r32 = g.solve(p.x0, spock.opts(precision=32, tol=1e-3, max_iters=20000))
        out[name] = {"one_T": e1, "fixed_25": e2, "n_T": [res["info"]["n_T"], r["n_T"]],
                     "K": [[res["info"]["n_K0"], res["info"]["n_K1"], res["info"]["n_K2"]],
                           [kinds.count("K0"), kinds.count("K1"), kinds.count("K2")]],
                     "fp32_status": r32["status"], "check": int(lib.spock_debug_last_check())}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
