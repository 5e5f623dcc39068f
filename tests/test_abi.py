"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/spock.h declares, and rejects malformed problems on the host before
any device call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2505_12078_b300 import build, spock, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return spock.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "spock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spock_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_binding_names():
    assert set(declared_functions()) == set(spock.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert lib.spock_status_str(code)
    assert lib.spock_version() >= 1


def _desc_call(p, mutate):
    """spock_problem_create on a mutated copy; validation fails on the host."""
    anc = np.array(p.anc, dtype=np.int32)
    prob = np.array(p.prob, dtype=np.float64)
    fields = dict(A=p.A, B=p.B, c=p.c, Q=p.Q, R=p.R, QN=p.QN, x_lo=p.x_lo, x_hi=p.x_hi,
                  u_lo=p.u_lo, u_hi=p.u_hi, u_ball=p.u_ball, avar=p.avar)
    fields = {k: (None if v is None else np.array(v, dtype=np.float64)) for k, v in fields.items()}
    nx, nu = p.nx, p.nu
    anc, prob, fields, nx, nu = mutate(anc, prob, fields, nx, nu)
    d = spock.ProblemDesc()
    d.n_nodes = anc.shape[0]
    d.anc = anc.ctypes.data_as(C.POINTER(C.c_int))
    d.prob = prob.ctypes.data_as(C.POINTER(C.c_double))
    d.nx, d.nu = nx, nu
    for k, v in fields.items():
        setattr(d, k, None if v is None else v.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    rc = spock.load().spock_problem_create(C.byref(d), C.byref(h))
    return rc, h


@pytest.mark.parametrize("case", ["not_bfs", "bad_root", "prob_sum", "avar_range", "neg_Q",
                                  "lo_gt_hi", "nan_A", "too_big", "half_box", "leaf_stage"])
def test_invalid_problems_rejected_on_host(lib, case):
    p = synth.small_raocp()

    def mutate(anc, prob, f, nx, nu):
        if case == "not_bfs":
            anc[5], anc[6] = anc[6], anc[5] + 0
            anc[3] = 5
        elif case == "bad_root":
            anc[0] = 0
        elif case == "prob_sum":
            prob[1] = 0.9 * prob[1]
        elif case == "avar_range":
            f["avar"][3] = 1.5
        elif case == "neg_Q":
            f["Q"][2, 1] = -1.0
        elif case == "lo_gt_hi":
            f["x_lo"][4, 0] = 10.0
        elif case == "nan_A":
            f["A"][0, 0, 0] = np.nan
        elif case == "too_big":
            nx = 300
        elif case == "half_box":
            f["u_hi"] = None
        elif case == "leaf_stage":
            anc = anc[:-1].copy()       # one leaf fewer: its sibling structure breaks
            prob = prob[:-1].copy()
        return anc, prob, f, nx, nu

    rc, h = _desc_call(p, mutate)
    assert rc in (-1, -6), rc
    assert not h.value
