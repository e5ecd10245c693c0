"""mpps -- mixed-precision Paterson--Stockmeyer evaluation of matrix polynomials on GB300.

Python binding of the C ABI in ``include/mpps.h`` (library ``libmpps.so`` built in-tree by
``paper_2312_17396_gb300._build``).  Argument marshalling only: every step of the
evaluation runs in the CUDA kernels of the library.  If the library is missing the calls
raise; there is no CPU fallback.

Matrices are float64, shape (n, n) or (batch, n, n), row-major contiguous.  Inputs may be
CUDA torch tensors (the call is asynchronous on the current torch stream, except for one
read-back of the block norms that the precision rule needs) or host arrays (numpy or CPU
tensors; the library copies them in and out and synchronises).

Paper: X. Liu, "Mixed-Precision Paterson--Stockmeyer Method for Evaluating Polynomials of
Matrices", arXiv 2312.17396.  Algorithm 2.1 (fixed PS), eq. (2.8) (precision rule),
Algorithm 3.1 (Taylor exp), Algorithm 4.1 (general coefficients), eq. (3.6) (scaling and
squaring).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libmpps.so")
_lib = None

FIXED_FP64, MIXED_PAPER, MIXED_NS = 0, 1, 2
FMT_NONE, FMT_FP64, FMT_BF16X3, FMT_TF32, FMT_BF16, FMT_FP8 = -1, 0, 1, 2, 3, 4
F64E_MAX_SLICES = 9


def FMT_F64E(k: int) -> int:
    """Format code of an FP64 product emulated with k exact bf16 slices per operand."""
    return 16 + int(k)


FORMAT_NAMES = {FMT_NONE: "none", FMT_FP64: "fp64", FMT_BF16X3: "bf16x3", FMT_TF32: "tf32",
                FMT_BF16: "bf16", FMT_FP8: "fp8"}
FORMAT_NAMES.update({FMT_F64E(k): f"f64e{k}" for k in range(1, F64E_MAX_SLICES + 1)})
_FMT_BY_NAME = {v: k for k, v in FORMAT_NAMES.items()}
MAX_R = 64
MAX_S = 32
NUM_FORMATS = 5

STATUS = {0: "MPPS_OK", 1: "MPPS_EINVAL", 2: "MPPS_ENOMEM", 3: "MPPS_ECUDA", 4: "MPPS_ETIMEOUT",
          5: "MPPS_ENOTSUP", 6: "MPPS_ECHECK"}


class MppsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Policy(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("s", ctypes.c_int), ("formats", ctypes.c_uint), ("fp64_floor_steps", ctypes.c_int),
                ("f64_slices", ctypes.c_int), ("variable_s", ctypes.c_int),
                ("adjoint_recompute", ctypes.c_int), ("device_plan", ctypes.c_int),
                ("max_squarings", ctypes.c_int), ("mixed_powers", ctypes.c_int)]


class _GroupItem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_int),
                ("m", ctypes.c_int)]


class _PolyItem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_int),
                ("m", ctypes.c_int), ("coeffs", ctypes.POINTER(ctypes.c_double))]


class _Report(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("r", ctypes.c_int), ("nu", ctypes.c_int),
                ("sigma", ctypes.c_int), ("fold", ctypes.c_int),
                ("fmt", ctypes.c_int * (MAX_R + 1)), ("u", ctypes.c_double * (MAX_R + 1)),
                ("normB", ctypes.c_double * (MAX_R + 1)), ("normY", ctypes.c_double),
                ("normX", ctypes.c_double), ("gemms", ctypes.c_int * (NUM_FORMATS + 1)),
                ("cost_ratio", ctypes.c_double), ("pow_fmt", ctypes.c_int * (MAX_S + 1))]


EXPORTS = ("mpps_policy_default", "mpps_plan", "ps_eval", "expm_taylor_ss", "ps_eval_adjoint",
           "mpps_matmul", "mpps_last_error", "mpps_version", "mpps_profile_enable",
           "mpps_profile_reset", "mpps_profile_read", "mpps_matmul_noalloc",
           "mpps_selftest_bounded_wait", "expm_taylor_ss_grouped", "mpps_release_workspace",
           "expm_taylor_ss_adjoint", "mpps_choose_s", "mpps_autotune_enable",
           "mpps_autotune_clear", "mpps_autotune_entries", "expm_pade13", "mpps_plan_adjoint",
           "ps_eval_tape_bytes", "ps_eval_forward_tape", "ps_eval_adjoint_tape",
           "ps_eval_adjoint_f32", "ps_eval_grouped", "lu_solve", "mpps_plan_powers",
           "mpps_matmul_ta")
STORAGE_F64, STORAGE_F32 = 0, 1
PROF_GEMM_F64, PROF_GEMM_TC, PROF_ELEMENTWISE, PROF_GEMM_F64E, PROF_SLICE = 0, 1, 2, 3, 4


def lib():
    """Load libmpps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(_LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.mpps_policy_default.argtypes = [ctypes.POINTER(_Policy)]
        L.mpps_policy_default.restype = None
        L.mpps_plan.argtypes = [ip, ip, dp, ctypes.c_double, ctypes.POINTER(_Policy),
                                ctypes.POINTER(_Report)]
        L.ps_eval.argtypes = [dp, ip, vp, ip, ip, ctypes.POINTER(_Policy), vp,
                              ctypes.POINTER(_Report), vp]
        L.expm_taylor_ss.argtypes = [vp, ip, ip, ip, ctypes.POINTER(_Policy), vp,
                                     ctypes.POINTER(_Report), vp]
        L.ps_eval_adjoint.argtypes = [dp, ip, vp, vp, ip, ip, ctypes.POINTER(_Policy), vp, vp]
        L.expm_taylor_ss_adjoint.argtypes = [vp, vp, ip, ip, ip, ctypes.POINTER(_Policy), vp, vp]
        L.mpps_plan_adjoint.argtypes = [ip, ip, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(_Policy), ctypes.POINTER(_Report)]
        L.mpps_plan_adjoint.restype = ctypes.c_int
        L.ps_eval_tape_bytes.argtypes = [ip, ip, ip, ctypes.POINTER(_Policy)]
        L.ps_eval_tape_bytes.restype = ctypes.c_size_t
        L.ps_eval_forward_tape.argtypes = [dp, ip, vp, ip, ip, ip, ctypes.POINTER(_Policy), vp, vp,
                                           ctypes.c_size_t, vp]
        L.ps_eval_forward_tape.restype = ctypes.c_int
        L.ps_eval_adjoint_tape.argtypes = [dp, ip, vp, ctypes.c_size_t, vp, ip, ip, ip,
                                           ctypes.POINTER(_Policy), vp, vp]
        L.ps_eval_adjoint_tape.restype = ctypes.c_int
        L.ps_eval_adjoint_f32.argtypes = [dp, ip, vp, vp, ip, ip, ctypes.POINTER(_Policy), vp, vp]
        L.ps_eval_adjoint_f32.restype = ctypes.c_int
        L.mpps_choose_s.argtypes = [ip, ctypes.c_double, dp, dp, ip]
        L.mpps_choose_s.restype = ctypes.c_int
        L.expm_pade13.argtypes = [vp, ip, ip, ctypes.POINTER(_Policy), vp, vp]
        L.expm_pade13.restype = ctypes.c_int
        L.lu_solve.argtypes = [vp, vp, ip, ip, ctypes.POINTER(_Policy), vp, vp]
        L.lu_solve.restype = ctypes.c_int
        L.mpps_plan_powers.argtypes = [ip, ip, dp, dp, dp, ctypes.POINTER(_Policy),
                                       ctypes.POINTER(ctypes.c_int), dp]
        L.mpps_plan_powers.restype = ctypes.c_int
        L.mpps_autotune_enable.argtypes = [ctypes.c_int]
        L.mpps_autotune_enable.restype = None
        L.mpps_autotune_clear.argtypes = []
        L.mpps_autotune_clear.restype = None
        L.mpps_autotune_entries.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int]
        L.mpps_autotune_entries.restype = ctypes.c_int
        L.mpps_matmul.argtypes = [vp, vp, vp, ip, ip, ip, vp]
        L.mpps_matmul_ta.argtypes = [vp, vp, vp, ip, ip, ip, vp]
        L.mpps_matmul_ta.restype = ctypes.c_int
        L.mpps_matmul_noalloc.argtypes = [vp, vp, vp, ip, ip, ip, vp]
        L.mpps_matmul_noalloc.restype = ctypes.c_int
        L.expm_taylor_ss_grouped.argtypes = [ctypes.POINTER(_GroupItem), ip, ctypes.POINTER(_Policy),
                                             ctypes.POINTER(_Report), vp]
        L.expm_taylor_ss_grouped.restype = ctypes.c_int
        L.ps_eval_grouped.argtypes = [ctypes.POINTER(_PolyItem), ip, ctypes.POINTER(_Policy),
                                      ctypes.POINTER(_Report), vp]
        L.ps_eval_grouped.restype = ctypes.c_int
        L.mpps_selftest_bounded_wait.argtypes = [ctypes.c_int, vp]
        L.mpps_selftest_bounded_wait.restype = ctypes.c_int
        L.mpps_release_workspace.argtypes = []
        L.mpps_release_workspace.restype = ctypes.c_int
        for f in ("mpps_plan", "ps_eval", "expm_taylor_ss", "ps_eval_adjoint",
                  "expm_taylor_ss_adjoint", "mpps_matmul"):
            getattr(L, f).restype = ctypes.c_int
        L.mpps_profile_enable.argtypes = [ctypes.c_int]
        L.mpps_profile_enable.restype = None
        L.mpps_profile_reset.argtypes = []
        L.mpps_profile_reset.restype = None
        L.mpps_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
        L.mpps_profile_read.restype = ctypes.c_int
        L.mpps_last_error.restype = ctypes.c_char_p
        L.mpps_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise MppsError(status, lib().mpps_last_error().decode(errors="replace"))


# ------------------------------------------------------------------------------------
# policy and reports
# ------------------------------------------------------------------------------------
@dataclass
class Policy:
    """Precision policy (see ``mpps_policy`` in include/mpps.h)."""
    mode: int = MIXED_NS
    tol: float = 2.0 ** -53
    delta: float = 10.0
    s: int = 0
    formats: object = 0x1F          # bitmask or iterable of format names
    fp64_floor_steps: int = 2
    f64_slices: int = 0             # 0: FP64 pipe; k: emulate FP64 products with k slices
    variable_s: bool = False        # the variable-s branch of Algorithm 3.1 (mixed modes)
    adjoint_recompute: bool = False  # adjoints: keep ceil(sqrt(r)) iterates, recompute the rest
    device_plan: bool = False       # the precision rule on the GPU: no read-back of the norms
    max_squarings: int = 0          # expm with device_plan: squaring steps launched (0: read sigma)
    mixed_powers: bool = False      # power tree with the leaves in fewer slices (mpps_plan_powers)

    def _c(self):
        fm = self.formats
        if not isinstance(fm, int):
            mask = 0
            for name in fm:
                mask |= 1 << _FMT_BY_NAME[name]
            fm = mask
        return _Policy(int(self.mode), float(self.tol), float(self.delta), int(self.s),
                       int(fm), int(self.fp64_floor_steps), int(self.f64_slices),
                       int(bool(self.variable_s)), int(bool(self.adjoint_recompute)),
                       int(bool(self.device_plan)), int(self.max_squarings),
                       int(bool(self.mixed_powers)))


FIXED = Policy(mode=FIXED_FP64)
PAPER = Policy(mode=MIXED_PAPER)
NS = Policy(mode=MIXED_NS)
# the same rules with the working-precision products emulated on the tensor cores (8 slices)
FIXED_E = Policy(mode=FIXED_FP64, f64_slices=8)
PAPER_E = Policy(mode=MIXED_PAPER, f64_slices=8)
NS_E = Policy(mode=MIXED_NS, f64_slices=8)


def _report_dict(R: _Report) -> dict:
    r = R.r
    return dict(s=R.s, r=r, nu=R.nu, sigma=R.sigma, fold=bool(R.fold),
                fmt=[None] + [FORMAT_NAMES[R.fmt[i]] for i in range(1, r + 1)],
                u=[None] + [R.u[i] for i in range(1, r + 1)],
                normB=[R.normB[i] for i in range(r + 1)], normY=R.normY, normX=R.normX,
                gemms={FORMAT_NAMES[f]: R.gemms[f] for f in range(NUM_FORMATS)} |
                {"squarings": R.gemms[NUM_FORMATS]},
                cost_ratio=R.cost_ratio,
                pow_fmt=[FORMAT_NAMES.get(R.pow_fmt[j]) for j in range(R.s + 1)])


def plan(m: int, n: int, normB, normY: float, policy: Policy | None = None) -> dict:
    """Host-only precision planner of the library (eq. (2.8); no GPU needed)."""
    nb = np.ascontiguousarray(normB, dtype=np.float64)
    R = _Report()
    pol = (policy or Policy())._c()
    _check(lib().mpps_plan(int(m), int(n), nb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           float(normY), ctypes.byref(pol), ctypes.byref(R)))
    return _report_dict(R)


def plan_powers(m: int, s: int, coeffs, normXpow, normBpart, policy: Policy | None = None):
    """Host-only rule for the leaves of the power tree (mpps_plan_powers; no GPU needed):
    returns (format names of X^0..X^s, the block norms handed to the block rule)."""
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    xp = np.ascontiguousarray(normXpow, dtype=np.float64)
    nb = np.ascontiguousarray(normBpart, dtype=np.float64)
    if c.size != m + 1 or xp.size != s or nb.size != m // s + 1:
        raise ValueError("coeffs, normXpow and normBpart need m+1, s and m//s+1 values")
    fmt = (ctypes.c_int * (s + 1))()
    nbo = np.zeros(m // s + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    pol = (policy or Policy())._c()
    _check(lib().mpps_plan_powers(int(m), int(s), c.ctypes.data_as(dp), xp.ctypes.data_as(dp),
                                  nb.ctypes.data_as(dp), ctypes.byref(pol), fmt,
                                  nbo.ctypes.data_as(dp)))
    return [FORMAT_NAMES.get(fmt[j]) for j in range(s + 1)], nbo


def plan_adjoint(m: int, n: int, normB, normY: float, normX: float,
                 policy: Policy | None = None) -> dict:
    """Host-only planner of the reverse pass: the forward rule with every u_i divided by
    m / min(1, ||X||_1) (mpps_plan_adjoint; no GPU needed)."""
    nb = np.ascontiguousarray(normB, dtype=np.float64)
    R = _Report()
    pol = (policy or Policy())._c()
    _check(lib().mpps_plan_adjoint(int(m), int(n), nb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   float(normY), float(normX), ctypes.byref(pol), ctypes.byref(R)))
    return _report_dict(R)


# ------------------------------------------------------------------------------------
# coefficient sequences (double precision; b_i rounded once)
# ------------------------------------------------------------------------------------
def taylor_exp_coeffs(m: int) -> np.ndarray:
    """b_i = 1/i! (Section 3)."""
    return np.array([1 / math.factorial(i) for i in range(m + 1)])   # int/int: correctly rounded


def pade_exp_num_coeffs(q: int) -> np.ndarray:
    """[q/q] Pade numerator of exp: (2q-j)! q! / ((2q)! j! (q-j)!) (Section 4.1)."""
    f = math.factorial
    return np.array([f(2 * q - j) * f(q) / (f(2 * q) * f(j) * f(q - j)) for j in range(q + 1)])


def pade_exp_den_coeffs(q: int) -> np.ndarray:
    """[q/q] Pade denominator of exp: p_qq(-X) (Section 4.1)."""
    c = pade_exp_num_coeffs(q)
    return c * (-1.0) ** np.arange(q + 1)


def cos_taylor_coeffs(m: int) -> np.ndarray:
    """Taylor cosine in B = X^2: (-1)^k / (2k)! (Section 4.2)."""
    return np.array([(-1) ** k / math.factorial(2 * k) for k in range(m + 1)])


# ------------------------------------------------------------------------------------
# marshalling
# ------------------------------------------------------------------------------------
def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _is_torch(x):
    t = _torch()
    return t is not None and isinstance(x, t.Tensor)


def _prep(A, name):
    """Returns (pointer, batch, n, kind, keepalive) for a float64 square matrix stack."""
    if _is_torch(A):
        torch = _torch()
        if A.dtype != torch.float64:
            raise TypeError(f"{name} must be float64 (got {A.dtype})")
        if not A.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        shape = tuple(A.shape)
        ptr = A.data_ptr()
        kind = "cuda" if A.is_cuda else "host"
        keep = A
    else:
        A = np.ascontiguousarray(A, dtype=np.float64)
        shape = A.shape
        ptr = A.ctypes.data
        kind, keep = "host", A
    if len(shape) == 2:
        batch, n = 1, shape[0]
        if shape[1] != n:
            raise ValueError(f"{name} must be square")
    elif len(shape) == 3:
        batch, n = shape[0], shape[1]
        if shape[2] != n:
            raise ValueError(f"{name} must be a stack of square matrices")
    else:
        raise ValueError(f"{name} must have shape (n, n) or (batch, n, n)")
    return ptr, batch, n, kind, keep


def _empty_like(A, keep):
    if _is_torch(keep):
        return _torch().empty_like(keep)
    return np.empty_like(keep)


def _stream_for(kind, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if kind == "cuda":
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _coef_ptr(coeffs):
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    return c, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(c) - 1


# ------------------------------------------------------------------------------------
# entry points
# ------------------------------------------------------------------------------------
def ps_eval(coeffs, A, policy: Policy | None = None, out=None, report: bool = False, stream=None):
    """p(A) = sum_i coeffs[i] A^i by Paterson--Stockmeyer with the per-step precision rule."""
    ptr, batch, n, kind, keep = _prep(A, "A")
    if out is None:
        out = _empty_like(A, keep)
    optr, ob, on, okind, okeep = _prep(out, "out")
    if (ob, on) != (batch, n):
        raise ValueError("out has the wrong shape")
    c, cp, m = _coef_ptr(coeffs)
    reps = (_Report * batch)() if report else None
    pol = (policy or Policy())._c()
    _check(lib().ps_eval(cp, m, ctypes.c_void_p(ptr), n, batch, ctypes.byref(pol),
                         ctypes.c_void_p(optr), reps, _stream_for(kind, stream)))
    if report:
        return out, [_report_dict(r) for r in reps]
    return out


def expm(A, m: int = 30, policy: Policy | None = None, out=None, report: bool = False, stream=None):
    """exp(A) by the degree-m Taylor polynomial with scaling and squaring (eq. (3.6))."""
    ptr, batch, n, kind, keep = _prep(A, "A")
    if out is None:
        out = _empty_like(A, keep)
    optr, ob, on, _, _ = _prep(out, "out")
    if (ob, on) != (batch, n):
        raise ValueError("out has the wrong shape")
    reps = (_Report * batch)() if report else None
    pol = (policy or Policy())._c()
    _check(lib().expm_taylor_ss(ctypes.c_void_p(ptr), n, batch, int(m), ctypes.byref(pol),
                                ctypes.c_void_p(optr), reps, _stream_for(kind, stream)))
    if report:
        return out, [_report_dict(r) for r in reps]
    return out


def expm_grouped(mats, degrees=None, policy: Policy | None = None, outs=None, report: bool = False,
                 stream=None):
    """exp of many CUDA matrices of different orders (and Taylor degrees) in one call.
    mats: list of (n_i, n_i) float64 CUDA tensors; degrees: list of m_i (default 30)."""
    torch = _torch()
    count = len(mats)
    if degrees is None:
        degrees = [30] * count
    if outs is None:
        outs = [torch.empty_like(a) for a in mats]
    arr = (_GroupItem * max(1, count))()
    for i, (a, o, m) in enumerate(zip(mats, outs, degrees)):
        if not (_is_torch(a) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                and a.dim() == 2 and a.shape[0] == a.shape[1]):
            raise ValueError("expm_grouped takes contiguous square float64 CUDA tensors")
        arr[i] = _GroupItem(a.data_ptr(), o.data_ptr(), int(a.shape[0]), int(m))
    reps = (_Report * count)() if report else None
    pol = (policy or Policy())._c()
    st = ctypes.c_void_p(int(stream)) if stream is not None else \
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(lib().expm_taylor_ss_grouped(arr, count, ctypes.byref(pol), reps, st))
    if report:
        return outs, [_report_dict(r) for r in reps]
    return outs


def ps_eval_grouped(coeffs_list, mats, policy: Policy | None = None, outs=None, report: bool = False,
                    stream=None):
    """p_i(A_i) for many CUDA matrices of different orders, each with its own coefficient
    sequence, in one call (ps_eval_grouped).  coeffs_list: one coefficient array per matrix
    (equal sequences share a bucket)."""
    torch = _torch()
    count = len(mats)
    if len(coeffs_list) != count:
        raise ValueError("one coefficient sequence per matrix")
    if outs is None:
        outs = [torch.empty_like(a) for a in mats]
    arr = (_PolyItem * max(1, count))()
    keep = []
    for i, (a, o, c) in enumerate(zip(mats, outs, coeffs_list)):
        if not (_is_torch(a) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                and a.dim() == 2 and a.shape[0] == a.shape[1]):
            raise ValueError("ps_eval_grouped takes contiguous square float64 CUDA tensors")
        cc, cp, m = _coef_ptr(c)
        keep.append(cc)
        arr[i] = _PolyItem(a.data_ptr(), o.data_ptr(), int(a.shape[0]), int(m), cp)
    reps = (_Report * count)() if report else None
    pol = (policy or Policy())._c()
    st = ctypes.c_void_p(int(stream)) if stream is not None else \
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(lib().ps_eval_grouped(arr, count, ctypes.byref(pol), reps, st))
    if report:
        return outs, [_report_dict(r) for r in reps]
    return outs


def ps_eval_adjoint(coeffs, A, G, out=None, policy: Policy | None = None, stream=None):
    """Gradient of <G, p(A)> with respect to A (reverse mode through the PS steps; products
    on the FP64 pipe, or emulated when policy.f64_slices > 0)."""
    ptr, batch, n, kind, keep = _prep(A, "A")
    gptr, gb, gn, _, _ = _prep(G, "G")
    if (gb, gn) != (batch, n):
        raise ValueError("G must have the shape of A")
    if out is None:
        out = _empty_like(A, keep)
    optr, _, _, _, _ = _prep(out, "out")
    c, cp, m = _coef_ptr(coeffs)
    pol = (policy or Policy(f64_slices=0))._c()
    _check(lib().ps_eval_adjoint(cp, m, ctypes.c_void_p(ptr), ctypes.c_void_p(gptr), n, batch,
                                 ctypes.byref(pol), ctypes.c_void_p(optr), _stream_for(kind, stream)))
    return out


def _storage_of(t):
    torch = _torch()
    if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
        raise ValueError("tape calls take contiguous CUDA tensors")
    if t.dtype == torch.float64:
        return STORAGE_F64
    if t.dtype == torch.float32:
        return STORAGE_F32
    raise TypeError(f"tape calls take float64 or float32 tensors (got {t.dtype})")


def _shape(t):
    if t.dim() == 2:
        return 1, t.shape[0]
    if t.dim() == 3 and t.shape[1] == t.shape[2]:
        return t.shape[0], t.shape[1]
    raise ValueError("expected (n, n) or (batch, n, n)")


def tape_bytes(m: int, n: int, batch: int, policy: Policy | None = None) -> int:
    pol = (policy or Policy())._c()
    nbytes = int(lib().ps_eval_tape_bytes(int(m), int(n), int(batch), ctypes.byref(pol)))
    if nbytes == 0:
        raise MppsError(1, lib().mpps_last_error().decode(errors="replace"))
    return nbytes


def ps_eval_forward_tape(coeffs, A, policy: Policy | None = None, out=None, stream=None):
    """p(A) (float64 or float32 CUDA tensor) and the tape its reverse pass reads: returns
    (out, tape), tape a uint8 CUDA tensor of ps_eval_tape_bytes bytes."""
    torch = _torch()
    storage = _storage_of(A)
    batch, n = _shape(A)
    c, cp, m = _coef_ptr(coeffs)
    pol = (policy or Policy())._c()
    nbytes = tape_bytes(m, n, batch, policy)
    tape = torch.empty(nbytes, dtype=torch.uint8, device=A.device)
    if out is None:
        out = torch.empty_like(A)
    _check(lib().ps_eval_forward_tape(cp, m, ctypes.c_void_p(A.data_ptr()), storage, n, batch,
                                      ctypes.byref(pol), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(tape.data_ptr()), nbytes,
                                      _stream_for("cuda", stream)))
    return out, tape


def ps_eval_adjoint_tape(coeffs, tape, G, policy: Policy | None = None, out=None, stream=None):
    """Gradient of <G, p(A)> from the tape of ps_eval_forward_tape (same coeffs, policy,
    shape and dtype)."""
    torch = _torch()
    storage = _storage_of(G)
    batch, n = _shape(G)
    c, cp, m = _coef_ptr(coeffs)
    pol = (policy or Policy())._c()
    if out is None:
        out = torch.empty_like(G)
    _check(lib().ps_eval_adjoint_tape(cp, m, ctypes.c_void_p(tape.data_ptr()), tape.numel(),
                                      ctypes.c_void_p(G.data_ptr()), storage, n, batch,
                                      ctypes.byref(pol), ctypes.c_void_p(out.data_ptr()),
                                      _stream_for("cuda", stream)))
    return out


def ps_eval_adjoint_f32(coeffs, A, G, out=None, policy: Policy | None = None, stream=None):
    """ps_eval_adjoint for float32 CUDA tensors (evaluated in FP64, gradient rounded to FP32)."""
    torch = _torch()
    for t, nm in ((A, "A"), (G, "G")):
        if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous float32 CUDA tensor")
    batch, n = _shape(A)
    if tuple(G.shape) != tuple(A.shape):
        raise ValueError("G must have the shape of A")
    c, cp, m = _coef_ptr(coeffs)
    pol = (policy or Policy())._c()
    if out is None:
        out = torch.empty_like(A)
    _check(lib().ps_eval_adjoint_f32(cp, m, ctypes.c_void_p(A.data_ptr()),
                                     ctypes.c_void_p(G.data_ptr()), n, batch, ctypes.byref(pol),
                                     ctypes.c_void_p(out.data_ptr()), _stream_for("cuda", stream)))
    return out


def expm_pade(A, policy: Policy | None = None, out=None, stream=None):
    """exp(A) by the [13/13] Pade approximant with scaling and squaring (numerator and
    denominator from one power chain, LU solve, squarings)."""
    ptr, batch, n, kind, keep = _prep(A, "A")
    if out is None:
        out = _empty_like(A, keep)
    optr, ob, on, _, _ = _prep(out, "out")
    if (ob, on) != (batch, n):
        raise ValueError("out has the wrong shape")
    pol = (policy or Policy())._c()
    _check(lib().expm_pade13(ctypes.c_void_p(ptr), n, batch, ctypes.byref(pol),
                             ctypes.c_void_p(optr), _stream_for(kind, stream)))
    return out


def lu_solve(Q, P, policy: Policy | None = None, out=None, stream=None):
    """R = Q^-1 P per matrix by LU with partial pivoting (the q^-1 p solve of the Pade
    approximant): panels on the FP64 pipe, block updates and substitutions as tile products
    in the policy's working precision (f64_slices)."""
    qptr, batch, n, kind, keep = _prep(Q, "Q")
    pptr, pb, pn, pkind, pkeep = _prep(P, "P")   # pkeep: P's (possibly converted) array
    if (pb, pn) != (batch, n) or pkind != kind:
        raise ValueError("P must have the shape and placement of Q")
    if out is None:
        out = _empty_like(Q, keep)
    optr, ob, on, _, _ = _prep(out, "out")
    if (ob, on) != (batch, n):
        raise ValueError("out has the wrong shape")
    pol = (policy or Policy())._c()
    _check(lib().lu_solve(ctypes.c_void_p(qptr), ctypes.c_void_p(pptr), n, batch,
                          ctypes.byref(pol), ctypes.c_void_p(optr), _stream_for(kind, stream)))
    del pkeep
    return out


def expm_adjoint(A, G, m: int = 30, out=None, policy: Policy | None = None, stream=None):
    """Gradient of <G, r(A)> with respect to A for the scaling-and-squaring approximant
    r(A) = p_m(2^-sigma A)^(2^sigma) (reverse mode through the squarings and the PS steps;
    products on the FP64 pipe, or emulated when policy.f64_slices > 0)."""
    ptr, batch, n, kind, keep = _prep(A, "A")
    gptr, gb, gn, _, _ = _prep(G, "G")
    if (gb, gn) != (batch, n):
        raise ValueError("G must have the shape of A")
    if out is None:
        out = _empty_like(A, keep)
    optr, _, _, _, _ = _prep(out, "out")
    pol = (policy or Policy(f64_slices=0))._c()
    _check(lib().expm_taylor_ss_adjoint(ctypes.c_void_p(ptr), ctypes.c_void_p(gptr), n, batch,
                                        int(m), ctypes.byref(pol), ctypes.c_void_p(optr),
                                        _stream_for(kind, stream)))
    return out


def choose_s(m: int, normX: float, normB0, normY) -> int:
    """The library's variable-s rule (mpps_choose_s) on given norms: normB0[k], normY[k] are
    ||B_0||_1 and ||X^s||_1 for s = ceil(sqrt(m)) + k."""
    b0 = np.ascontiguousarray(normB0, dtype=np.float64)
    y = np.ascontiguousarray(normY, dtype=np.float64)
    if b0.shape != y.shape or b0.size < 1:
        raise ValueError("normB0 and normY need the same non-zero length")
    dp = ctypes.POINTER(ctypes.c_double)
    return int(lib().mpps_choose_s(int(m), float(normX), b0.ctypes.data_as(dp),
                                   y.ctypes.data_as(dp), int(b0.size)))


def autotune(on: bool = True) -> None:
    """Switch measured schedule choice on or off (see mpps_autotune_enable)."""
    lib().mpps_autotune_enable(1 if on else 0)


def autotune_clear() -> None:
    lib().mpps_autotune_clear()


def autotune_entries() -> list:
    """The measured choices: dicts with kind ('f64e_split' or 'tc_width'), n, batch,
    variant, choice and the candidates' mean times in ms."""
    L = lib()
    cnt = L.mpps_autotune_entries(None, None, None, None, None, None, 0)
    if cnt == 0:
        return []
    cols = [np.zeros(cnt, dtype=np.int32) for _ in range(5)]
    ms = np.zeros(4 * cnt, dtype=np.float32)
    L.mpps_autotune_entries(*[ctypes.c_void_p(c.ctypes.data) for c in cols],
                            ctypes.c_void_p(ms.ctypes.data), cnt)
    kinds = {0: "f64e_split", 1: "tc_width"}
    return [dict(kind=kinds.get(int(cols[0][i]), int(cols[0][i])), n=int(cols[1][i]),
                 batch=int(cols[2][i]), variant=int(cols[3][i]), choice=int(cols[4][i]),
                 ms=[float(x) for x in ms[4 * i:4 * i + 4]]) for i in range(cnt)]


def matmul(A, B, fmt="fp64", out=None, stream=None):
    """C = A B with the product computed in format `fmt` (name or FMT_* code)."""
    f = _FMT_BY_NAME[fmt] if isinstance(fmt, str) else int(fmt)
    ptr, batch, n, kind, keep = _prep(A, "A")
    bptr, bb, bn, _, _ = _prep(B, "B")
    if (bb, bn) != (batch, n):
        raise ValueError("B must have the shape of A")
    if out is None:
        out = _empty_like(A, keep)
    optr, _, _, _, _ = _prep(out, "out")
    _check(lib().mpps_matmul(ctypes.c_void_p(ptr), ctypes.c_void_p(bptr), ctypes.c_void_p(optr),
                             n, batch, f, _stream_for(kind, stream)))
    return out


def matmul_ta(A, B, fmt="fp64", out=None, stream=None):
    """C = A^T B with the product computed in format `fmt` (mpps_matmul_ta)."""
    f = _FMT_BY_NAME[fmt] if isinstance(fmt, str) else int(fmt)
    ptr, batch, n, kind, keep = _prep(A, "A")
    bptr, bb, bn, _, _ = _prep(B, "B")
    if (bb, bn) != (batch, n):
        raise ValueError("B must have the shape of A")
    if out is None:
        out = _empty_like(A, keep)
    optr, _, _, _, _ = _prep(out, "out")
    _check(lib().mpps_matmul_ta(ctypes.c_void_p(ptr), ctypes.c_void_p(bptr), ctypes.c_void_p(optr),
                                n, batch, f, _stream_for(kind, stream)))
    return out


def profile_enable(on: bool = True) -> None:
    """Record CUDA events around every library kernel launch (benchmark instrumentation)."""
    lib().mpps_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().mpps_profile_reset()


def profile_read(kernel_class: int):
    """(launches, total ms, total executed flops) of one kernel class since the last reset."""
    cnt = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    work = ctypes.c_double(0.0)
    _check(lib().mpps_profile_read(int(kernel_class), ctypes.byref(cnt), ctypes.byref(ms),
                                   ctypes.byref(work)))
    return int(cnt.value), float(ms.value), float(work.value)


def matmul_noalloc(A, B, out, fmt="fp64", stream=None):
    """C = A B like ``matmul`` but through the entry point that allocates no device memory
    (fixed library-owned scratch; device tensors only; `out` must be given)."""
    f = _FMT_BY_NAME[fmt] if isinstance(fmt, str) else int(fmt)
    ptr, batch, n, kind, keep = _prep(A, "A")
    bptr, bb, bn, _, _ = _prep(B, "B")
    optr, ob, on, _, _ = _prep(out, "out")
    if (bb, bn) != (batch, n) or (ob, on) != (batch, n):
        raise ValueError("A, B and out must have the same shape")
    _check(lib().mpps_matmul_noalloc(ctypes.c_void_p(ptr), ctypes.c_void_p(bptr),
                                     ctypes.c_void_p(optr), n, batch, f,
                                     _stream_for(kind, stream)))
    return out


def version() -> str:
    return lib().mpps_version().decode()


def release_workspace() -> None:
    """Return the library's cached device workspaces to the driver (waits for the devices
    that hold them)."""
    _check(lib().mpps_release_workspace())


def _make_autograd():
    torch = _torch()
    if torch is None:  # pragma: no cover
        return None, None

    class PolyFn(torch.autograd.Function):
        """p(A) with a hand-written reverse mode that reuses the forward pass: forward
        ps_eval_forward_tape keeps the powers and Horner iterates on a tape (all of them, or
        with policy.adjoint_recompute every ceil(sqrt(r))-th), backward ps_eval_adjoint_tape
        reads it.  float64 and float32 CUDA tensors go through the library as they are (FP32
        storage is widened and narrowed by its kernels); other dtypes are cast to float64."""

        @staticmethod
        def forward(ctx, A, coeffs, policy=None):
            c = np.asarray(coeffs, dtype=np.float64)
            x = A.detach()
            if x.dtype not in (torch.float64, torch.float32):
                x = x.to(torch.float64)
            x = x.contiguous()
            P, tape = ps_eval_forward_tape(c, x, policy=policy)
            ctx.save_for_backward(tape)
            ctx.coeffs = c
            ctx.policy = policy
            ctx.work_dtype = x.dtype
            ctx.in_dtype = A.dtype
            return P.to(A.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            (tape,) = ctx.saved_tensors
            G = grad_out.detach().to(ctx.work_dtype).contiguous()
            gA = ps_eval_adjoint_tape(ctx.coeffs, tape, G, policy=ctx.policy)
            return gA.to(ctx.in_dtype), None, None

    class ExpmFn(torch.autograd.Function):
        """exp(A) by scaling and squaring (expm) with a hand-written reverse mode
        (expm_adjoint).  FP32 inputs are evaluated in FP64 and returned in the input dtype."""

        @staticmethod
        def forward(ctx, A, m=30, policy=None):
            A64 = A.detach().to(torch.float64).contiguous()
            E = expm(A64, m=m, policy=policy)
            ctx.save_for_backward(A64)
            ctx.m = m
            ctx.policy = policy
            ctx.in_dtype = A.dtype
            return E.to(A.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            (A64,) = ctx.saved_tensors
            G = grad_out.detach().to(torch.float64).contiguous()
            gA = expm_adjoint(A64, G, m=ctx.m, policy=ctx.policy)
            return gA.to(ctx.in_dtype), None, None

    return PolyFn, ExpmFn


PolyFn, ExpmFn = _make_autograd()


def poly(A, coeffs, policy: Policy | None = None):
    """Differentiable p(A) (torch): ``PolyFn.apply`` with a default policy."""
    return PolyFn.apply(A, coeffs, policy)


def expm_differentiable(A, m: int = 30, policy: Policy | None = None):
    """Differentiable exp(A) (torch): ``ExpmFn.apply``; the backward pass differentiates the
    scaling-and-squaring approximant with the same products (policy.f64_slices)."""
    return ExpmFn.apply(A, m, policy)
