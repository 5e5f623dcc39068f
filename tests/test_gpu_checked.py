"""The bounds-checked build (libspock_checked.so, -DSPOCK_CHECKED): the
iteration kernel checks the indices it derives from the tree (children ranges,
segment nodes, mailbox slots, the factor blocks its bulk copies read) before
use; a failed check skips the access and ends the launch with SPOCK_EDEVICE
instead of touching memory outside its buffers. It stands in for a memory
sanitizer, which is not available here: on parity cases of both sweep
paths and of the extended costs and risks, no check fails and the results stay
within the parity tolerances against the oracle. Runs in a process of its own
(tests/checked_worker.py): one process holds one copy of the library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CASES = ["small", "ragged_37x19_ball", "avar0_branch8", "team_100x50", "full_rows_cta", "l1_box_ball",
         "tv_box_ball", "soft_box_ball"]


def test_checked_build_no_index_check_fails_and_parity_holds():
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "checked_worker.py"), *CASES],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    res = json.loads(line)
    for name in CASES:
        d = res[name]
        assert d["check"] == 0, (name, d)
        assert d["one_T"] < 1e-11, (name, d)
        assert d["fixed_25"] < 1e-10, (name, d)
        assert d["n_T"][0] == d["n_T"][1] and d["K"][0] == d["K"][1], (name, d)
        assert d["fp32_status"] == 0, (name, d)
