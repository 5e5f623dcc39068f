"""Thin ctypes binding of libspock (include/spock.h). Argument marshalling
only: every step of the method runs in the library's CUDA kernels. Device
buffers are torch CUDA tensors (torch provides device memory and streams).

Raises if libspock.so is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspock.so")

SPOCK_OK = 0
SPOCK_MAXITER = 1
SPOCK_PARTIAL = 2
STATUS = {0: "ok", 1: "maxiter", 2: "partial", -1: "einval", -2: "enomem", -3: "enotpd", -4: "edevice",
          -5: "etimeout", -6: "eunsupported"}

EXPORTED = [
    "spock_problem_create", "spock_problem_destroy", "spock_problem_sizes", "spock_problem_alpha",
    "spock_problem_set_alpha", "spock_problem_scalings", "spock_problem_factors",
    "spock_problem_set_x0", "spock_op_T", "spock_op_L", "spock_op_Lt", "spock_solve_opts_default",
    "spock_solve", "spock_solve_device", "spock_get_iterate", "spock_set_iterate",
    "spock_status_str", "spock_version", "spock_op_T_noalloc", "spock_op_T_centred",
    "spock_batch_create", "spock_batch_destroy", "spock_batch_sizes", "spock_batch_set_tw",
    "spock_batch_autotune", "spock_batch_solve",
    "spock_server_create", "spock_server_submit", "spock_server_poll", "spock_server_outstanding",
    "spock_server_destroy", "spock_check", "spock_debug_wait_fault", "spock_server_evict",
    "spock_server_admitted", "spock_debug_last_check",
]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class ProblemDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("anc", _ip), ("prob", _dp), ("nx", C.c_int), ("nu", C.c_int),
                ("A", _dp), ("B", _dp), ("c", _dp), ("Q", _dp), ("R", _dp), ("QN", _dp),
                ("x_lo", _dp), ("x_hi", _dp), ("u_lo", _dp), ("u_hi", _dp), ("u_ball", _dp),
                ("avar", _dp), ("weights_full", C.c_int), ("q", _dp), ("r", _dp), ("qN", _dp),
                ("n_g", C.c_int), ("Gx", _dp), ("Gu", _dp), ("g_lo", _dp), ("g_hi", _dp),
                ("n_gN", C.c_int), ("GN", _dp), ("gN_lo", _dp), ("gN_hi", _dp), ("l1", C.c_double), ("tv", _dp),
                ("soft_max", _dp)]


class Sizes(C.Structure):
    _fields_ = [("n", C.c_int), ("n_nonleaf", C.c_int), ("n_leaf", C.c_int), ("N", C.c_int),
                ("nx", C.c_int), ("nu", C.c_int), ("n_c", C.c_int), ("n_cN", C.c_int),
                ("n_z", C.c_longlong), ("n_eta", C.c_longlong), ("n_v", C.c_longlong),
                ("factor_bytes_fp64", C.c_longlong), ("factor_bytes_fp32", C.c_longlong),
                ("solve_bytes_fp64", C.c_longlong), ("solve_bytes_fp32", C.c_longlong),
                ("device_bytes", C.c_longlong), ("device_peak_bytes", C.c_longlong)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_iters", C.c_int),
                ("max_backtracks", C.c_int), ("method", C.c_int), ("warm_start", C.c_int),
                ("fp64_check", C.c_int), ("aa_mode", C.c_int), ("recentre", C.c_double)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("n_T", C.c_int), ("n_K0", C.c_int),
                ("n_K1", C.c_int), ("n_K2", C.c_int), ("n_fallback", C.c_int),
                ("n_backtracks", C.c_int), ("res_inf", C.c_double), ("res_inf_fp64", C.c_double),
                ("risk", C.c_double), ("device_ms", C.c_double), ("phase_ms", C.c_double * 7),
                ("counters", C.c_double * 8), ("xi1", C.c_double), ("xi2", C.c_double),
                ("infeas", C.c_double), ("gap", C.c_double), ("n_recentre", C.c_int),
                ("kernel_ms", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(self.phase_ms)
        d["counters"] = list(self.counters)
        return d


class BatchInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("n_T", C.c_int), ("tw", C.c_int),
                ("res_inf", C.c_double), ("risk", C.c_double), ("device_ms", C.c_double),
                ("xi1", C.c_double), ("xi2", C.c_double), ("infeas", C.c_double), ("gap", C.c_double)]


class CheckInfo(C.Structure):
    _fields_ = [("res_inf", C.c_double), ("xi1", C.c_double), ("xi2", C.c_double),
                ("infeas", C.c_double), ("gap", C.c_double), ("eta_Lz", C.c_double),
                ("support", C.c_double)]


class ServeResult(C.Structure):
    _fields_ = [("id", C.c_longlong), ("plant", C.c_int), ("status", C.c_int), ("iters", C.c_int),
                ("n_T", C.c_int), ("res_inf", C.c_double), ("risk", C.c_double), ("u0", C.c_double * 64),
                ("device_ms", C.c_double), ("latency_ms", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libspock.so (raises OSError if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libspock.so not built at {path}; run python -m paper_2505_12078_b300.build")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.spock_problem_create.argtypes = [C.POINTER(ProblemDesc), C.POINTER(vp)]
    lib.spock_problem_destroy.argtypes = [vp]
    lib.spock_problem_destroy.restype = None
    lib.spock_problem_sizes.argtypes = [vp, C.POINTER(Sizes)]
    lib.spock_problem_alpha.argtypes = [vp, _dp, _dp]
    lib.spock_problem_set_alpha.argtypes = [vp, C.c_double]
    lib.spock_problem_scalings.argtypes = [vp, _dp, _dp, _dp]
    lib.spock_problem_factors.argtypes = [vp, _dp, _dp, _dp, _dp]
    lib.spock_problem_set_x0.argtypes = [vp, _dp]
    lib.spock_op_T.argtypes = [vp, C.c_int, vp, vp, _dp, vp]
    lib.spock_op_T_noalloc.argtypes = [vp, C.c_int, vp, vp, _dp, vp]
    lib.spock_op_T_centred.argtypes = [vp, vp, vp, vp, _dp, vp]
    lib.spock_op_L.argtypes = [vp, C.c_int, vp, vp, vp]
    lib.spock_op_Lt.argtypes = [vp, C.c_int, vp, vp, vp]
    lib.spock_solve_opts_default.argtypes = [C.POINTER(SolveOpts)]
    lib.spock_solve_opts_default.restype = None
    lib.spock_solve.argtypes = [vp, _dp, C.POINTER(SolveOpts), _dp, _dp, _dp, C.POINTER(Info)]
    lib.spock_solve_device.argtypes = [vp, vp, C.POINTER(SolveOpts), vp, vp, vp, C.POINTER(Info)]
    lib.spock_check.argtypes = [vp, C.c_int, vp, vp, C.POINTER(CheckInfo)]
    lib.spock_get_iterate.argtypes = [vp, C.c_int, vp, vp]
    lib.spock_set_iterate.argtypes = [vp, C.c_int, vp, vp]
    lib.spock_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.POINTER(vp)]
    lib.spock_batch_destroy.argtypes = [vp]
    lib.spock_batch_destroy.restype = None
    _llp = C.POINTER(C.c_longlong)
    lib.spock_batch_sizes.argtypes = [vp, _llp, _llp, _llp]
    lib.spock_batch_set_tw.argtypes = [vp, _ip]
    lib.spock_batch_autotune.argtypes = [vp, C.c_int, _ip]
    lib.spock_batch_solve.argtypes = [vp, _dp, C.POINTER(SolveOpts), _dp, _dp, _dp, C.POINTER(BatchInfo), _dp]
    lib.spock_server_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.POINTER(SolveOpts), C.c_int,
                                        C.c_longlong, C.POINTER(vp), _ip]
    lib.spock_server_submit.argtypes = [vp, C.c_int, _dp, C.c_int, C.POINTER(C.c_longlong)]
    lib.spock_server_poll.argtypes = [vp, C.POINTER(ServeResult), C.c_int, _ip]
    lib.spock_server_outstanding.argtypes = [vp]
    lib.spock_server_outstanding.restype = C.c_longlong
    lib.spock_server_destroy.argtypes = [vp]
    lib.spock_server_destroy.restype = None
    lib.spock_server_evict.argtypes = [vp, C.c_int]
    lib.spock_server_admitted.argtypes = [vp, C.c_int]
    lib.spock_status_str.argtypes = [C.c_int]
    lib.spock_status_str.restype = C.c_char_p
    lib.spock_version.restype = C.c_int
    lib.spock_debug_wait_fault.argtypes = [C.c_int, C.c_double]
    if hasattr(lib, "spock_debug_last_check"):   # a debug entry; libraries built before it lack it
        lib.spock_debug_last_check.argtypes = []
        lib.spock_debug_last_check.restype = C.c_int
    _lib = lib
    return lib


def debug_wait_fault(phantom_ctas=0, wait_limit_s=0.0):
    """Test hook (spock_debug_wait_fault): later single-problem launches wait for
    phantom CTAs at their grid barriers and give up after wait_limit_s."""
    _check(load().spock_debug_wait_fault(int(phantom_ctas), float(wait_limit_s)), "spock_debug_wait_fault")


class SpockError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: status {code} ({STATUS.get(code, '?')})")
        self.code = code


def _check(code, where):
    if code < 0:
        raise SpockError(code, where)
    return code


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def opts(precision=64, tol=1e-4, max_iters=5000, max_backtracks=30, method="spock",
         warm_start=False, fp64_check=True, aa="gram", recentre=None) -> SolveOpts:
    o = SolveOpts()
    load().spock_solve_opts_default(C.byref(o))
    o.precision = int(precision)
    o.tol = float(tol)
    o.max_iters = int(max_iters)
    o.max_backtracks = int(max_backtracks)
    o.method = {"spock": 0, "cp": 1}[method]
    o.warm_start = int(bool(warm_start))
    o.fp64_check = int(bool(fp64_check))
    o.aa_mode = {"gram": 0, "qr_update": 1}[aa]
    if recentre is not None:      # FP32: 0 plain iteration, > 0 centred (library default 0.1)
        o.recentre = float(recentre)
    return o


class Problem:
    """A problem resident on the current CUDA device (created from a synth.RAOCP)."""

    def __init__(self, p):
        lib = load()
        self._keep = []
        d = ProblemDesc()
        anc = np.ascontiguousarray(p.anc, dtype=np.int32)
        arrs = dict(prob=p.prob, A=p.A, B=p.B, c=p.c, Q=p.Q, R=p.R, QN=p.QN, x_lo=p.x_lo,
                    x_hi=p.x_hi, u_lo=p.u_lo, u_hi=p.u_hi, u_ball=p.u_ball, avar=p.avar)
        for k in ("q", "r", "qN", "Gx", "Gu", "g_lo", "g_hi", "GN", "gN_lo", "gN_hi", "tv", "soft_max"):
            arrs[k] = getattr(p, k, None)
        conv = {k: _f64(v) for k, v in arrs.items()}
        self._keep += [anc] + list(conv.values())
        d.n_nodes = anc.shape[0]
        d.anc = anc.ctypes.data_as(_ip)
        d.nx, d.nu = int(p.nx), int(p.nu)
        d.weights_full = int(np.ndim(p.Q) == 3)
        d.n_g = 0 if arrs["Gx"] is None else int(np.asarray(arrs["Gx"]).shape[0])
        d.n_gN = 0 if arrs["GN"] is None else int(np.asarray(arrs["GN"]).shape[0])
        for k, v in conv.items():
            setattr(d, k, _ptr(v))
        d.l1 = float(getattr(p, "l1", None) or 0.0)
        h = C.c_void_p()
        _check(lib.spock_problem_create(C.byref(d), C.byref(h)), "spock_problem_create")
        self.h = h
        self._keep = []
        s = Sizes()
        _check(lib.spock_problem_sizes(h, C.byref(s)), "spock_problem_sizes")
        self.sizes = {k: getattr(s, k) for k, _ in s._fields_}
        self.nx, self.nu = p.nx, p.nu
        self.n, self.n_nl = s.n, s.n_nonleaf
        self.n_z, self.n_eta, self.n_v = s.n_z, s.n_eta, s.n_v

    def close(self):
        if getattr(self, "h", None):
            load().spock_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory(self):
        """(device bytes held now, peak device bytes) from spock_problem_sizes."""
        s = Sizes()
        _check(load().spock_problem_sizes(self.h, C.byref(s)), "spock_problem_sizes")
        return s.device_bytes, s.device_peak_bytes

    # --- setup outputs ---------------------------------------------------------
    def alpha(self):
        a, n = C.c_double(), C.c_double()
        _check(load().spock_problem_alpha(self.h, C.byref(a), C.byref(n)), "alpha")
        return a.value, n.value

    def set_alpha(self, alpha):
        _check(load().spock_problem_set_alpha(self.h, float(alpha)), "set_alpha")

    def scalings(self):
        Sx, Su, SxN = np.zeros(self.nx), np.zeros(self.nu), np.zeros(self.nx)
        _check(load().spock_problem_scalings(self.h, _ptr(Sx), _ptr(Su), _ptr(SxN)), "scalings")
        return Sx, Su, SxN

    def factors(self):
        P = np.zeros((self.n, self.nx, self.nx))
        K = np.zeros((self.n_nl, self.nu, self.nx))
        Rt = np.zeros((self.n_nl, self.nu, self.nu))
        Ab = np.zeros((self.n - 1, self.nx, self.nx))
        _check(load().spock_problem_factors(self.h, _ptr(P), _ptr(K), _ptr(Rt), _ptr(Ab)), "factors")
        return P, K, Rt, Ab

    def set_x0(self, x0):
        x0 = _f64(x0)
        _check(load().spock_problem_set_x0(self.h, _ptr(x0)), "set_x0")

    # --- operators (torch CUDA tensors) ----------------------------------------
    @staticmethod
    def _prec(t):
        import torch
        if t.dtype == torch.float64:
            return 64
        if t.dtype == torch.float32:
            return 32
        raise TypeError("float32 or float64 tensors only")

    def _check_pair(self, v_in, v_out):
        """v_in and v_out: contiguous CUDA tensors of n_v elements, same dtype
        and device, distinct storage (the library writes n_v elements of
        v_in's precision into v_out and reads v_in meanwhile)."""
        assert v_in.is_cuda and v_in.is_contiguous() and v_in.numel() == self.n_v
        assert v_out.is_cuda and v_out.is_contiguous() and v_out.numel() == self.n_v
        if v_out.dtype != v_in.dtype or v_out.device != v_in.device:
            raise TypeError("v_out must have v_in's dtype and device")
        a0, a1 = v_in.data_ptr(), v_in.data_ptr() + v_in.numel() * v_in.element_size()
        b0, b1 = v_out.data_ptr(), v_out.data_ptr() + v_out.numel() * v_out.element_size()
        if a0 < b1 and b0 < a1:
            raise ValueError("v_in and v_out must not overlap")

    def T(self, v_in, v_out=None, stream=None):
        """v_out = T(v_in); returns (v_out, stats[8])."""
        import torch
        assert v_in.is_cuda and v_in.is_contiguous() and v_in.numel() == self.n_v
        if v_out is None:
            v_out = torch.empty_like(v_in)
        self._check_pair(v_in, v_out)
        stats = np.zeros(8)
        _check(load().spock_op_T(self.h, self._prec(v_in), C.c_void_p(v_in.data_ptr()),
                                 C.c_void_p(v_out.data_ptr()), _ptr(stats),
                                 C.c_void_p(stream.cuda_stream if stream else 0)), "spock_op_T")
        return v_out, stats

    def T_centred(self, c, delta, out=None, stream=None):
        """out = T(c + delta) - c through spock_op_T_centred: c a float64 CUDA
        tensor, delta a float32 one (n_v each); returns (out, stats[8])."""
        import torch
        assert c.is_cuda and c.dtype == torch.float64 and c.is_contiguous() and c.numel() == self.n_v
        assert delta.is_cuda and delta.dtype == torch.float32 and delta.is_contiguous() and delta.numel() == self.n_v
        if out is None:
            out = torch.empty_like(delta)
        self._check_pair(delta, out)
        stats = np.zeros(8)
        _check(load().spock_op_T_centred(self.h, C.c_void_p(c.data_ptr()), C.c_void_p(delta.data_ptr()),
                                         C.c_void_p(out.data_ptr()), _ptr(stats),
                                         C.c_void_p(stream.cuda_stream if stream else 0)), "spock_op_T_centred")
        return out, stats

    def T_noalloc(self, v_in, v_out, stream=None):
        """v_out = T(v_in) through spock_op_T_noalloc (no device allocation in
        the call; scratch from the library's static device array)."""
        self._check_pair(v_in, v_out)
        stats = np.zeros(8)
        _check(load().spock_op_T_noalloc(self.h, self._prec(v_in), C.c_void_p(v_in.data_ptr()),
                                         C.c_void_p(v_out.data_ptr()), _ptr(stats),
                                         C.c_void_p(stream.cuda_stream if stream else 0)),
               "spock_op_T_noalloc")
        return v_out, stats

    def L(self, z, eta=None):
        import torch
        assert z.is_cuda and z.numel() == self.n_z
        if eta is None:
            eta = torch.empty(self.n_eta, dtype=z.dtype, device=z.device)
        _check(load().spock_op_L(self.h, self._prec(z), C.c_void_p(z.data_ptr()),
                                 C.c_void_p(eta.data_ptr()), None), "spock_op_L")
        return eta

    def Lt(self, eta, z=None):
        import torch
        assert eta.is_cuda and eta.numel() == self.n_eta
        if z is None:
            z = torch.empty(self.n_z, dtype=eta.dtype, device=eta.device)
        _check(load().spock_op_Lt(self.h, self._prec(eta), C.c_void_p(eta.data_ptr()),
                                  C.c_void_p(z.data_ptr()), None), "spock_op_Lt")
        return z

    # --- solve -------------------------------------------------------------------
    def solve(self, x0, o: SolveOpts = None):
        """Host-buffer solve (end to end). Returns dict(x, u, risk, info, status)."""
        o = o or opts()
        x0 = _f64(x0)
        x = np.zeros((self.n, self.nx))
        u = np.zeros((self.n_nl, self.nu))
        risk = C.c_double()
        info = Info()
        st = _check(load().spock_solve(self.h, _ptr(x0), C.byref(o), _ptr(x), _ptr(u),
                                       C.byref(risk), C.byref(info)), "spock_solve")
        return dict(x=x, u=u, risk=risk.value, info=info.as_dict(), status=st)

    def solve_device(self, x0_dev, o: SolveOpts = None, x_out=None, u_out=None, stream=None):
        o = o or opts()
        info = Info()
        st = _check(load().spock_solve_device(
            self.h, C.c_void_p(x0_dev.data_ptr()), C.byref(o),
            C.c_void_p(x_out.data_ptr()) if x_out is not None else None,
            C.c_void_p(u_out.data_ptr()) if u_out is not None else None,
            C.c_void_p(stream.cuda_stream if stream else 0), C.byref(info)), "spock_solve_device")
        return st, info.as_dict()

    def check(self, v, stream=None):
        """FP64 exit check (Sec. 5.3) of the iterate v (CUDA tensor, n_v): dict of
        res_inf, xi1, xi2, infeas, gap, eta_Lz, support."""
        assert v.is_cuda and v.is_contiguous() and v.numel() == self.n_v
        out = CheckInfo()
        _check(load().spock_check(self.h, self._prec(v), C.c_void_p(v.data_ptr()),
                                  C.c_void_p(stream.cuda_stream if stream else 0), C.byref(out)),
               "spock_check")
        return {k: getattr(out, k) for k, _ in out._fields_}

    def get_iterate(self, precision=64):
        import torch
        dt = torch.float64 if precision == 64 else torch.float32
        v = torch.empty(self.n_v, dtype=dt, device="cuda")
        _check(load().spock_get_iterate(self.h, precision, C.c_void_p(v.data_ptr()), None), "get_iterate")
        torch.cuda.synchronize()
        return v

    def set_iterate(self, v):
        _check(load().spock_set_iterate(self.h, self._prec(v), C.c_void_p(v.data_ptr()), None),
               "set_iterate")


class Batch:
    """Many problems solved together in one persistent launch (spock_batch_*).
    The problems must stay alive and must not be solved on their own while the
    batch is in use."""

    def __init__(self, problems, precision=32):
        lib = load()
        self.problems = list(problems)
        self.count = len(self.problems)
        self.precision = int(precision)
        arr = (C.c_void_p * self.count)(*[p.h for p in self.problems])
        h = C.c_void_p()
        _check(lib.spock_batch_create(arr, self.count, self.precision, C.byref(h)), "spock_batch_create")
        self.h = h
        a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(lib.spock_batch_sizes(h, C.byref(a), C.byref(b), C.byref(c)), "spock_batch_sizes")
        self.x0_total, self.x_total, self.u_total = a.value, b.value, c.value

    def close(self):
        if getattr(self, "h", None):
            load().spock_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tw(self, tw=None):
        t = None if tw is None else np.ascontiguousarray(tw, dtype=np.int32)
        _check(load().spock_batch_set_tw(self.h, None if t is None else t.ctypes.data_as(_ip)), "set_tw")

    def autotune(self, iters=20):
        tw = np.zeros(self.count, dtype=np.int32)
        _check(load().spock_batch_autotune(self.h, int(iters), tw.ctypes.data_as(_ip)), "autotune")
        return tw

    def solve(self, x0s, o: SolveOpts = None):
        """x0s: list of per-problem x0. Returns dict(x=[...], u=[...], risk, info=[...],
        status, total_ms)."""
        o = o or opts(precision=self.precision)
        x0 = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in x0s]))
        assert x0.size == self.x0_total
        x = np.zeros(self.x_total)
        u = np.zeros(self.u_total)
        risk = np.zeros(self.count)
        info = (BatchInfo * self.count)()
        ms = C.c_double()
        st = _check(load().spock_batch_solve(self.h, _ptr(x0), C.byref(o), _ptr(x), _ptr(u), _ptr(risk),
                                             info, C.byref(ms)), "spock_batch_solve")
        xs, us, ox, ou = [], [], 0, 0
        for p in self.problems:
            xs.append(x[ox:ox + p.n * p.nx].reshape(p.n, p.nx)); ox += p.n * p.nx
            us.append(u[ou:ou + p.n_nl * p.nu].reshape(p.n_nl, p.nu)); ou += p.n_nl * p.nu
        infos = [{k: getattr(info[i], k) for k, _ in BatchInfo._fields_} for i in range(self.count)]
        return dict(x=xs, u=us, risk=risk, info=infos, status=st, total_ms=ms.value)


class Server:
    """Serving of MPC requests on resident plants (spock_server_*): requests are
    admitted to the device as CTAs free up, each solved alone in its CTA."""

    def __init__(self, plants, precision=32, o: SolveOpts = None, ring_slots=4096, mem_budget=0):
        lib = load()
        self.plants = list(plants)
        self.precision = int(precision)
        o = o or opts(precision=self.precision)
        arr = (C.c_void_p * len(self.plants))(*[p.h for p in self.plants])
        h = C.c_void_p()
        adm = C.c_int()
        self.status = _check(lib.spock_server_create(arr, len(self.plants), self.precision, C.byref(o),
                                                     int(ring_slots), int(mem_budget), C.byref(h), C.byref(adm)),
                             "spock_server_create")
        self.h = h
        self.admitted = adm.value
        self._buf = (ServeResult * 1024)()

    def close(self):
        if getattr(self, "h", None):
            load().spock_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, plant, x0, warm=True):
        x0 = _f64(x0)
        rid = C.c_longlong()
        _check(load().spock_server_submit(self.h, int(plant), _ptr(x0), int(bool(warm)), C.byref(rid)), "submit")
        return rid.value

    def poll(self):
        """Finished requests as dicts (u0 trimmed to the plant's nu)."""
        out = []
        while True:
            n = C.c_int()
            _check(load().spock_server_poll(self.h, self._buf, len(self._buf), C.byref(n)), "poll")
            for i in range(n.value):
                r = self._buf[i]
                d = {k: getattr(r, k) for k, _ in ServeResult._fields_ if k != "u0"}
                d["u0"] = np.array(r.u0[: self.plants[r.plant].nu])
                out.append(d)
            if n.value < len(self._buf):
                return out

    def outstanding(self):
        return load().spock_server_outstanding(self.h)

    def evict(self, plant):
        """Release the plant's solve buffers (spock_server_evict)."""
        _check(load().spock_server_evict(self.h, int(plant)), "evict")

    def is_admitted(self, plant):
        return bool(_check(load().spock_server_admitted(self.h, int(plant)), "admitted"))

    def drain(self, timeout_s=60.0):
        import time
        res, t0 = [], time.time()
        while self.outstanding() > 0:
            res += self.poll()
            if time.time() - t0 > timeout_s:
                raise TimeoutError("requests still outstanding")
            time.sleep(0.0002)
        return res
