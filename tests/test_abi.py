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


def test_batch_and_server_reject_bad_arguments_on_host(lib):
    """Batch and server creation validate their arguments before any device call."""
    out = C.c_void_p()
    assert lib.spock_batch_create(None, 1, 32, C.byref(out)) == -1
    arr = (C.c_void_p * 1)(None)
    assert lib.spock_batch_create(arr, 1, 32, C.byref(out)) == -1        # NULL problem
    assert lib.spock_batch_create(arr, 0, 32, C.byref(out)) == -1        # empty batch
    assert lib.spock_batch_create(arr, 1, 16, C.byref(out)) == -1        # precision
    assert lib.spock_batch_create(arr, 1, 32, None) == -1
    adm = C.c_int()
    assert lib.spock_server_create(None, 1, 32, None, 16, 0, C.byref(out), C.byref(adm)) == -1
    assert lib.spock_server_create(arr, 1, 32, None, 16, 0, C.byref(out), C.byref(adm)) == -1
    assert lib.spock_server_create(arr, 1, 32, None, 0, 0, C.byref(out), C.byref(adm)) == -1
    assert lib.spock_server_submit(None, 0, None, 0, None) == -1
    assert lib.spock_server_poll(None, None, 0, None) == -1
    assert lib.spock_server_outstanding(None) == -1
    lib.spock_batch_destroy(None)
    lib.spock_server_destroy(None)
    assert lib.spock_status_str(2)


def test_algorithmic_bytes_counting():
    """The roofline's byte count on the 31-node problem, by hand: per T the
    factors MB (nx(nx+nu)) and MF ((nx+nu)nx) of every non-root node and MP
    (nu(nx+nu)) and KT (nx nu) of every non-leaf node, plus 8 passes over v;
    per iteration 5 passes over v (the Anderson memory)."""
    import bench
    sizes = dict(n=31, n_nonleaf=23, nx=4, nu=2, n_v=878)
    total, per_T = bench.algorithmic_bytes(sizes, n_T=10, iters=7, word=4)
    factors = 30 * (4 * 6 + 6 * 4) + 23 * (2 * 6 + 4 * 2)
    assert per_T == 4 * (factors + 8 * 878)
    assert total == 10 * per_T + 7 * 4 * 5 * 878


def _desc_call_general(p, mutate):
    """As _desc_call for a problem with full weights, linear terms and
    general rows (every optional field of spock_problem_desc set)."""
    anc = np.array(p.anc, dtype=np.int32)
    prob = np.array(p.prob, dtype=np.float64)
    keys = ("A", "B", "c", "Q", "R", "QN", "x_lo", "x_hi", "u_lo", "u_hi", "u_ball", "avar",
            "q", "r", "qN", "Gx", "Gu", "g_lo", "g_hi", "GN", "gN_lo", "gN_hi")
    f = {k: (None if getattr(p, k) is None else np.array(getattr(p, k), dtype=np.float64)) for k in keys}
    ints = dict(weights_full=int(np.ndim(p.Q) == 3), n_g=f["Gx"].shape[0] if f["Gx"] is not None else 0,
                n_gN=f["GN"].shape[0] if f["GN"] is not None else 0)
    mutate(f, ints)
    d = spock.ProblemDesc()
    d.n_nodes = anc.shape[0]
    d.anc = anc.ctypes.data_as(C.POINTER(C.c_int))
    d.prob = prob.ctypes.data_as(C.POINTER(C.c_double))
    d.nx, d.nu = p.nx, p.nu
    for k, v in f.items():
        setattr(d, k, None if v is None else v.ctypes.data_as(C.POINTER(C.c_double)))
    for k, v in ints.items():
        setattr(d, k, v)
    h = C.c_void_p()
    rc = spock.load().spock_problem_create(C.byref(d), C.byref(h))
    return rc, h


@pytest.mark.parametrize("case", ["asym_Q", "nonpos_R_diag", "nan_q", "neg_n_g", "g_lo_gt_hi", "too_many_rows",
                                  "null_Gx", "gN_lo_gt_hi", "lin_on_zero_weight"])
def test_invalid_general_problems_rejected_on_host(lib, case):
    """Full weights must be symmetric with a positive diagonal, linear terms
    finite and zero where a diagonal weight is zero, general rows well formed
    with lower bounds below upper bounds (checked before any device call)."""
    from tests.problems import general
    p = general([2, 1], 3, 2, seed=71, n_g=2, n_gN=1, box=True)

    def mutate(f, ints):
        if case == "asym_Q":
            f["Q"][1, 0, 2] += 0.5
        elif case == "nonpos_R_diag":
            f["R"][0, 1, 1] = 0.0
        elif case == "nan_q":
            f["q"][2, 1] = np.nan
        elif case == "neg_n_g":
            ints["n_g"] = -1
        elif case == "g_lo_gt_hi":
            f["g_lo"][1, 0] = f["g_hi"][1, 0] + 1.0
        elif case == "too_many_rows":
            ints["n_g"] = 300
        elif case == "null_Gx":
            f["Gx"] = None
        elif case == "gN_lo_gt_hi":
            f["gN_lo"][0, 0] = f["gN_hi"][0, 0] + 1.0
        elif case == "lin_on_zero_weight":
            ints["weights_full"] = 0
            f["Q"] = np.ones((len(p.anc) - 1, p.nx))
            f["Q"][3, 1] = 0.0
            f["R"] = np.ones((len(p.anc) - 1, p.nu))
            f["QN"] = np.ones((p.n_leaf, p.nx))

    rc, h = _desc_call_general(p, mutate)
    assert rc == (-6 if case == "too_many_rows" else -1), rc
    assert not h.value
