"""CPU oracle for mixed-precision Paterson--Stockmeyer (arXiv 2312.17396).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with the
CUDA library (``paper_2312_17396_gb300``) and never imports it.

Contents
--------
* ``mpps_oracle.c`` (built here with gcc into ``_liboracle.so``): Algorithm 2.1 literally
  in double-double and plain double, Horner, explicit powers, scaling and squaring
  (eq. (3.6)), column-block application p(X)^k V, the adjoint as the defining double sum
  of the Frechet derivative, the adjoint of the scaling-and-squaring approximant (chain
  rule through the squarings), and the 1-norm.
* Coefficient sequences as exact rationals (``fractions.Fraction``), converted to
  double-double: Taylor exp b_i = 1/i! (Section 3), the [q/q] Pade numerator and
  denominator of exp (Section 4.1; the Ward example of Section 2 prints the first eight
  numerator coefficients for q = 13), and the Taylor cosine as a polynomial in X^2
  (Section 4.2).
* ``plan``: the precision rule, written step by step from eq. (2.8) and the
  ``fix_params`` branch of Algorithm 3.1 / Algorithm 4.1, with the format ladder of
  Section 4.1.1 generalised to the GPU formats.
* ``cost_ratio``: eq. (3.8).
* ``lu_solve``: R = Q^-1 P by Gaussian elimination with partial pivoting (the q^-1 p solve of
  the Pade approximant, Section 4.1), unblocked, in plain double.
* ``e4m3_round``, ``mx_block_exp``, ``mxfp8_quantize_rows``, ``matmul_mxfp8``: the FP8
  Horner product with block scales (the low-precision products of eq. (2.6) in the 8-bit
  format, each row of the left factor and each column of the right one split into blocks
  of 32 along the inner dimension with one power-of-two scale per block), summed in FP64.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpps_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    flags = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # hardware FMA instead of the libm call; same correctly rounded result
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *flags, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        i = ctypes.c_int
        L.orc_ps_dd.argtypes = [dp, dp, i, i, dp, i, dp, dp, lp]
        L.orc_horner_dd.argtypes = [dp, dp, i, dp, i, dp, dp, lp]
        L.orc_powers_dd.argtypes = [dp, dp, i, dp, i, dp, dp]
        L.orc_expm_ss_dd.argtypes = [dp, dp, i, i, dp, i, i, dp, dp]
        L.orc_ps_apply_dd.argtypes = [dp, dp, i, dp, i, dp, i, ctypes.c_long, dp, dp]
        L.orc_adjoint_dd.argtypes = [dp, dp, i, dp, dp, i, dp, dp]
        L.orc_expm_ss_adjoint_dd.argtypes = [dp, dp, i, dp, dp, i, i, dp, dp]
        L.orc_matmul_dd.argtypes = [dp, dp, dp, dp, i, dp, dp]
        L.orc_ps_d.argtypes = [dp, i, i, dp, i, dp, lp]
        L.orc_expm_ss_d.argtypes = [dp, i, i, dp, i, i, dp]
        L.orc_norm1.argtypes = [dp, i, i]
        L.orc_norm1.restype = ctypes.c_double
        L.orc_num_threads.restype = ctypes.c_int
        for name in ("orc_ps_dd", "orc_horner_dd", "orc_powers_dd", "orc_expm_ss_dd",
                     "orc_ps_apply_dd", "orc_adjoint_dd", "orc_expm_ss_adjoint_dd",
                     "orc_matmul_dd", "orc_ps_d", "orc_expm_ss_d"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------
# coefficient sequences as exact rationals, then double-double
# ---------------------------------------------------------------------------------
def taylor_exp_rational(m: int):
    """b_i = 1/i!, i = 0..m (Section 3)."""
    return [Fraction(1, math.factorial(i)) for i in range(m + 1)]


def pade_exp_num_rational(q: int):
    """Numerator of the [q/q] Pade approximant to exp:
    c_j = (2q-j)! q! / ((2q)! j! (q-j)!), j = 0..q (Section 4.1).  For q = 13 the first
    eight values are the ones printed in the Ward example of Section 2."""
    f = math.factorial
    return [Fraction(f(2 * q - j) * f(q), f(2 * q) * f(j) * f(q - j)) for j in range(q + 1)]


def pade_exp_den_rational(q: int):
    """Denominator q_qq(X) = p_qq(-X): coefficients (-1)^j c_j (Section 4.1)."""
    return [c * (-1) ** j for j, c in enumerate(pade_exp_num_rational(q))]


def cos_taylor_rational(m: int):
    """Taylor cosine as a polynomial in B = X^2: sum_{k=0}^m (-1)^k B^k / (2k)!
    (Section 4.2 evaluates c_m(X^2) by PS)."""
    return [Fraction((-1) ** k, math.factorial(2 * k)) for k in range(m + 1)]


def to_dd(coefs):
    """Exact rationals -> (hi, lo) double-double arrays (hi = nearest double, lo = nearest
    double of the remainder)."""
    hi = np.array([float(c) for c in coefs], dtype=np.float64)
    lo = np.array([float(Fraction(c) - Fraction(float(h))) for c, h in zip(coefs, hi)],
                  dtype=np.float64)
    return hi, lo


def _coef_arrays(coefs):
    if isinstance(coefs, tuple) and len(coefs) == 2:
        return _f64(coefs[0]), _f64(coefs[1])
    coefs = list(coefs)
    if coefs and isinstance(coefs[0], Fraction):
        return to_dd(coefs)
    hi = _f64(coefs)
    return hi, np.zeros_like(hi)


def ceil_sqrt(m: int) -> int:
    """s = ceil(sqrt(m)) computed in integers (Algorithm 2.1, first line)."""
    if m <= 1:
        return 1
    s = math.isqrt(m)
    return s if s * s == m else s + 1


# ---------------------------------------------------------------------------------
# wrappers
# ---------------------------------------------------------------------------------
def ps_dd(coefs, X, s: int = 0):
    """Algorithm 2.1 in double-double.  Returns (P_hi, P_lo, products)."""
    ch, cl = _coef_arrays(coefs)
    m = len(ch) - 1
    X = _f64(X)
    n = X.shape[0]
    ph = np.empty((n, n)); pl = np.empty((n, n))
    cnt = ctypes.c_long(0)
    rc = lib().orc_ps_dd(_p(ch), _p(cl), m, int(s), _p(X), n, _p(ph), _p(pl), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError("orc_ps_dd: bad arguments")
    return ph, pl, cnt.value


def horner_dd(coefs, X):
    ch, cl = _coef_arrays(coefs)
    m = len(ch) - 1
    X = _f64(X); n = X.shape[0]
    ph = np.empty((n, n)); pl = np.empty((n, n)); cnt = ctypes.c_long(0)
    if lib().orc_horner_dd(_p(ch), _p(cl), m, _p(X), n, _p(ph), _p(pl), ctypes.byref(cnt)):
        raise ValueError("orc_horner_dd: bad arguments")
    return ph, pl, cnt.value


def powers_dd(coefs, X):
    ch, cl = _coef_arrays(coefs)
    m = len(ch) - 1
    X = _f64(X); n = X.shape[0]
    ph = np.empty((n, n)); pl = np.empty((n, n))
    if lib().orc_powers_dd(_p(ch), _p(cl), m, _p(X), n, _p(ph), _p(pl)):
        raise ValueError("orc_powers_dd: bad arguments")
    return ph, pl


def expm_ss_dd(A, m: int, sigma: int, s: int = 0, coefs=None):
    """p_m(2^-sigma A)^(2^sigma) in double-double, p_m the degree-m Taylor polynomial."""
    ch, cl = _coef_arrays(coefs if coefs is not None else taylor_exp_rational(m))
    m = len(ch) - 1
    A = _f64(A); n = A.shape[0]
    eh = np.empty((n, n)); el = np.empty((n, n))
    if lib().orc_expm_ss_dd(_p(ch), _p(cl), m, int(s), _p(A), n, int(sigma), _p(eh), _p(el)):
        raise ValueError("orc_expm_ss_dd: bad arguments")
    return eh, el


def ps_apply_dd(coefs, X, V, reps: int = 1):
    """p(X)^reps V by Horner on the column block V (n x k)."""
    ch, cl = _coef_arrays(coefs)
    m = len(ch) - 1
    X = _f64(X); n = X.shape[0]
    V = _f64(V).reshape(n, -1); k = V.shape[1]
    wh = np.empty((n, k)); wl = np.empty((n, k))
    if lib().orc_ps_apply_dd(_p(ch), _p(cl), m, _p(X), n, _p(V), k, int(reps), _p(wh), _p(wl)):
        raise ValueError("orc_ps_apply_dd: bad arguments")
    return wh, wl


def adjoint_dd(coefs, A, G):
    """Gradient of <G, p(A)> with respect to A: sum_k c_k sum_{j<k} (A^T)^j G (A^T)^(k-1-j)."""
    ch, cl = _coef_arrays(coefs)
    m = len(ch) - 1
    A = _f64(A); G = _f64(G); n = A.shape[0]
    dh = np.empty((n, n)); dl = np.empty((n, n))
    if lib().orc_adjoint_dd(_p(ch), _p(cl), m, _p(A), _p(G), n, _p(dh), _p(dl)):
        raise ValueError("orc_adjoint_dd: bad arguments")
    return dh, dl


def expm_ss_adjoint_dd(A, G, m: int, sigma: int, coefs=None):
    """Gradient of <G, p_m(2^-sigma A)^(2^sigma)> with respect to A (sigma fixed): the chain
    rule through the squarings of eq. (3.6) and the defining double sum of the polynomial's
    Frechet derivative, in double-double."""
    ch, cl = _coef_arrays(coefs if coefs is not None else taylor_exp_rational(m))
    m = len(ch) - 1
    A = _f64(A); G = _f64(G); n = A.shape[0]
    dh = np.empty((n, n)); dl = np.empty((n, n))
    if lib().orc_expm_ss_adjoint_dd(_p(ch), _p(cl), m, _p(A), _p(G), n, int(sigma), _p(dh), _p(dl)):
        raise ValueError("orc_expm_ss_adjoint_dd: bad arguments")
    return dh, dl


def matmul_dd(Ah, Al, Bh, Bl):
    Ah = _f64(Ah); Bh = _f64(Bh); n = Ah.shape[0]
    Al = _f64(Al) if Al is not None else np.zeros_like(Ah)
    Bl = _f64(Bl) if Bl is not None else np.zeros_like(Bh)
    ch = np.empty((n, n)); cl = np.empty((n, n))
    lib().orc_matmul_dd(_p(Ah), _p(Al), _p(Bh), _p(Bl), n, _p(ch), _p(cl))
    return ch, cl


def ps_d(coefs, X, s: int = 0):
    """Algorithm 2.1 in plain double (the timed CPU baseline)."""
    c = _f64([float(x) for x in coefs]) if not isinstance(coefs, np.ndarray) else _f64(coefs)
    m = len(c) - 1
    X = _f64(X); n = X.shape[0]
    P = np.empty((n, n)); cnt = ctypes.c_long(0)
    if lib().orc_ps_d(_p(c), m, int(s), _p(X), n, _p(P), ctypes.byref(cnt)):
        raise ValueError("orc_ps_d: bad arguments")
    return P, cnt.value


def expm_ss_d(A, m: int, sigma: int, s: int = 0):
    c = np.array([float(x) for x in taylor_exp_rational(m)])
    A = _f64(A); n = A.shape[0]
    E = np.empty((n, n))
    if lib().orc_expm_ss_d(_p(c), m, int(s), _p(A), n, int(sigma), _p(E)):
        raise ValueError("orc_expm_ss_d: bad arguments")
    return E


def norm1(M) -> float:
    M = _f64(M)
    M2 = M.reshape(M.shape[0], -1)
    return float(lib().orc_norm1(_p(M2), M2.shape[0], M2.shape[1]))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def rel_err_1norm(P_hat, ref_hi, ref_lo=None) -> float:
    """eps = ||P_hat - P||_1 / ||P||_1 (Section 3.4), P given as double-double."""
    D = (np.asarray(P_hat, dtype=np.float64) - ref_hi)
    if ref_lo is not None:
        D = D - ref_lo
    return norm1(D) / norm1(ref_hi)


def sigma_for(A) -> int:
    """Number of squarings so that ||2^-sigma A||_1 <= 1: sigma = max(0, ceil(log2 ||A||_1))."""
    nrm = norm1(A)
    if nrm <= 1.0:
        return 0
    m, e = math.frexp(nrm)          # nrm = m * 2^e, 0.5 <= m < 1
    return e - 1 if m == 0.5 else e


# ---------------------------------------------------------------------------------
# the linear solve of the Pade approximant (Section 4.1: r = q^-1 p)
# ---------------------------------------------------------------------------------
def lu_solve(Q, P):
    """R = Q^-1 P by Gaussian elimination with partial pivoting, unblocked, in plain double.

    Column j: the pivot is the first row i >= j of largest |Q_ij|; rows j and i are
    interchanged (in Q and in the right-hand sides), the multipliers l_ij = Q_ij / Q_jj of
    the rows below are stored in place and those rows lose l_ij times row j.  Then forward
    substitution with the unit lower triangle and back substitution with the upper one.
    Returns (R, piv, info): piv[j] = the row interchanged with row j, info = 0 or the first
    1-based column with a zero pivot (elimination skips that column, as the usual LAPACK
    convention does, and R is then not a solution)."""
    A = np.array(Q, dtype=np.float64, copy=True)
    B = np.array(P, dtype=np.float64, copy=True)
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int64)
    info = 0
    for j in range(n):
        col = np.abs(A[j:, j])
        i = j + int(np.argmax(col))          # argmax returns the first maximum
        piv[j] = i
        if not (A[i, j] != 0.0):
            if info == 0:
                info = j + 1
            continue
        if i != j:
            A[[j, i], :] = A[[i, j], :]
            B[[j, i], :] = B[[i, j], :]
        A[j + 1:, j] /= A[j, j]
        A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:])
    Y = B
    for j in range(n):                        # L Y = B (unit diagonal)
        Y[j + 1:, :] -= np.outer(A[j + 1:, j], Y[j, :])
    for j in range(n - 1, -1, -1):            # U R = Y
        Y[j, :] /= A[j, j]
        Y[:j, :] -= np.outer(A[:j, j], Y[j, :])
    return Y, piv, info


# ---------------------------------------------------------------------------------
# block norms of eq. (1.1) in double-double (inputs to the precision rule)
# ---------------------------------------------------------------------------------
def block_norms_dd(coefs, X, s: int = 0):
    """||B_i||_1 for i = 0..r and ||X^s||_1, from double-double powers of X.
    B_i = sum_{j<s} b_{si+j} X^j (i < r), B_r = sum_{j<=m-sr} b_{sr+j} X^j (eq. (1.1))."""
    ch, cl = _coef_arrays(coefs)
    m = len(ch) - 1
    X = _f64(X); n = X.shape[0]
    s = s if s > 0 else ceil_sqrt(m)
    r = m // s
    pw = [np.eye(n)]
    cur_h, cur_l = np.eye(n), np.zeros((n, n))
    for _ in range(s):
        cur_h, cur_l = matmul_dd(cur_h, cur_l, X, None)
        pw.append(cur_h + cur_l)
    norms = []
    for i in range(r + 1):
        top = s - 1 if i < r else m - s * r
        B = np.zeros((n, n))
        for j in range(top + 1):
            B = B + float(ch[s * i + j]) * pw[j]
        norms.append(norm1(B))
    return norms, norm1(pw[s])


def choose_s(m: int, normX: float, normB0, normY):
    """The variable-s branch of Algorithm 3.1 (fix_params false), step by step.

    Start from s = ceil(sqrt(m)).  The branch is taken only when ||X||_1 <= s/e; then, while
    ||Y||_1 > ||B_0||_1 ||X||_1^s and s < m, the algorithm adds Y/s! to B_0 (B_0 becomes the
    first block for s+1), increments s and forms the next power as Y.  normB0[k] and
    normY[k] are ||B_0|| and ||Y|| = ||X^s|| for s = s0 + k, k < len(normB0); the result is
    at most s0 + len(normB0).  ||X||^s is formed by repeated multiplication.  (The library
    also stops at s = 32, its largest block size.)"""
    s0 = ceil_sqrt(m)
    if not (normX <= s0 / math.e):
        return s0
    s = s0
    for k in range(len(normB0)):
        if s >= m or s >= 32:
            break
        xs = 1.0
        for _ in range(s):
            xs *= normX
        if not (normY[k] > normB0[k] * xs):
            break
        s += 1
    return s


# ---------------------------------------------------------------------------------
# precision rule (eq. (2.8); Algorithm 3.1 fix_params branch; Algorithm 4.1)
# ---------------------------------------------------------------------------------
FMT_FP64, FMT_BF16X3, FMT_TF32, FMT_BF16, FMT_FP8 = 0, 1, 2, 3, 4
FMT_NONE = -1
# unit roundoff of each format's inputs (Section 4.1.1 uses bf16 u = 2^-8 ~ 3.9e-3)
U_FMT = {FMT_FP64: 2.0 ** -53, FMT_BF16X3: 2.0 ** -16, FMT_TF32: 2.0 ** -11,
         FMT_BF16: 2.0 ** -8, FMT_FP8: 2.0 ** -4}
FP32_ACC = 2.0 ** -24
MODE_FIXED, MODE_PAPER, MODE_NS = 0, 1, 2


def FMT_F64E(k):
    """Format code of a product emulated with k exact slices (same numbering as the library)."""
    return 16 + k


def adjoint_divisor(m: int, normX: float) -> float:
    """Tightening of eq. (2.8) for the reverse pass (the paper states no adjoint; this is the
    reading used): the gradient of b_k X^k is a sum of k products X^j E X^(k-1-j), so the
    blocks of degree up to m weigh up to m / ||X|| times more in the gradient than in p(X).
    Divisor d = m / min(1, ||X||_1) (||X||_1 = 0 or >= 1 counts as 1)."""
    x = normX if 0.0 < normX < 1.0 else 1.0
    return m / x


def plan(m: int, n: int, norms, normY: float, mode: int = MODE_PAPER, tol: float = 2.0 ** -53,
         delta: float = 10.0, s: int = 0, formats: int = 0x1F, floor_steps: int = 2,
         f64_slices: int = 0, divisor: float = 1.0):
    """Per-step precisions for the Horner products P_i Y, i = r..1.

    1. s = ceil(sqrt(m)) unless given; r = floor(m/s).
    2. u_i = ||B_0|| tol / (||B_i|| ||Y||^i): eq. (2.8) with nu = 1 (the closed form that
       Algorithm 3.1 uses in its variable-s branch); y^i by repeated multiplication.
       The rule never asks for more than the working precision: u_i = max(tol, u_i).
       A zero block or zero Y contributes nothing: u_i = +inf.
    3. nu = min{i : u_i >= delta * tol} (r+1 if none); u_1..u_{nu-1} = tol.
    4. format_i = the cheapest allowed format F with U_FMT[F] <= u_i and, for formats that
       accumulate in FP32, n * 2^-24 <= u_i (Section 4.1.1's rule max{u* <= u_i}, with the
       accumulation error of the tensor cores added).  FP64 is always allowed.
       With f64_slices = K > 0 the working precision is an emulated product with K slices
       (format F64E(K)) and the ladder continues after BF16X3 with F64E(k), k = 4..K-1,
       whose unit roundoff is taken as 2^(2-7k) (k slices of 7 bits; exact accumulation: no
       n 2^-24 term), and 2^-55 for k = 9 (8 slices with the pairs of order 8).
    5. mode NS: steps i <= floor_steps stay in the working precision.  FIXED: every step.
    6. When s divides m, B_r = b_m I and step r is a scalar multiple of Y: no product
       (format NONE).
    divisor != 1 (the reverse pass, see adjoint_divisor): each u_i of step 2 is divided by it
    before the clamp of step 2 and before steps 3-6.
    Returns dict(s, r, nu, u (list, index 1..r), fmt (index 1..r), fold).
    """
    if m <= 0:
        return dict(s=1, r=0, nu=1, u=[None], fmt=[None], fold=False)
    s = s if s > 0 else ceil_sqrt(m)
    r = m // s
    fold = (m % s == 0)
    eta0 = float(norms[0])
    u = [None] * (r + 1)
    for i in range(1, r + 1):
        eta = float(norms[i])
        yi = 1.0
        for _ in range(i):
            yi = yi * float(normY)
        den = eta * yi
        ui = math.inf if den == 0.0 else (eta0 * tol) / den
        if divisor != 1.0:
            ui = ui / divisor
        u[i] = max(tol, ui)
    nu = r + 1
    for i in range(1, r + 1):
        if u[i] >= delta * tol:
            nu = i
            break
    for i in range(1, nu):
        u[i] = tol
    order = [FMT_FP8, FMT_BF16, FMT_TF32, FMT_BF16X3]
    wp = FMT_F64E(f64_slices) if f64_slices > 0 else FMT_FP64
    fmt = [None] * (r + 1)
    for i in range(1, r + 1):
        f = wp
        if mode != MODE_FIXED and not (mode == MODE_NS and i <= floor_steps):
            found = False
            for F in order:
                if not (formats >> F) & 1:
                    continue
                if U_FMT[F] <= u[i] and n * FP32_ACC <= u[i]:
                    f = F
                    found = True
                    break
            if not found:
                for k in range(4, f64_slices):
                    if (2.0 ** (2 - 7 * k) if k <= 8 else 2.0 ** -55) <= u[i]:
                        f = FMT_F64E(k)
                        break
        fmt[i] = f
    if fold:
        fmt[r] = FMT_NONE
    return dict(s=s, r=r, nu=nu, u=u, fmt=fmt, fold=fold)


def plan_powers(m: int, s: int, coefs, normXpow, normBpart, f64_slices: int,
                tol: float = 2.0 ** -53):
    """Slices of the leaves of the power tree (mixed precision inside the powers, the future
    work of Section 5), stated in the manner of eq. (2.8).

    1. h = ceil(s/2); X^2..X^h come from the chain, Y = X^h X^(s-h), and the leaves
       X^j = X^h X^(j-h), j = h+1..s-1 (L = s-h-1 of them), feed only the blocks
       B_i = sum_j b_{si+j} X^j (i = 0..r, r = floor(m/s), si+j <= m).
    2. A leaf's size is bounded by bx_j = ||X^h|| ||X^(j-h)||; its terms add at most
       e_i = sum_j |b_{si+j}| bx_j to ||B_i||: the block rule gets
       ||B_0||_low = max(0, ||B_0||_partial - e_0) and ||B_i||_partial + e_i (i >= 1).
    3. With S_j = sum_{i: si+j <= m} |b_{si+j}| ||Y||^i (y^i by repeated multiplication),
       u_j = ||B_0||_low tol / (L bx_j S_j) (+inf when the denominator is 0).
    4. Leaf j takes F64E(k) for the smallest k in 4..f64_slices-1 with 2^(2-7k) <= u_j (2^-55
       for k = 9), else the working precision F64E(f64_slices).
    Returns (fmt list over j = 0..s: None for j < 2, the format of X^j otherwise; normB list).
    """
    r = m // s
    h = (s + 1) // 2
    L = s - h - 1
    wp = FMT_F64E(f64_slices)
    bx = {j: float(normXpow[h - 1]) * float(normXpow[j - h - 1]) for j in range(h + 1, s)}
    e = [0.0] * (r + 1)
    for j in range(h + 1, s):
        for i in range(r + 1):
            if s * i + j <= m:
                e[i] += abs(float(coefs[s * i + j])) * bx[j]
    nb = [max(0.0, float(normBpart[0]) - e[0])] + [float(normBpart[i]) + e[i]
                                                     for i in range(1, r + 1)]
    y = float(normXpow[s - 1])
    fmt = [None, None] + [wp] * (s - 1)
    for j in range(h + 1, s):
        S, yi = 0.0, 1.0
        for i in range(r + 1):
            if s * i + j > m:
                break
            S += abs(float(coefs[s * i + j])) * yi
            yi = yi * y
        den = L * bx[j] * S
        uj = math.inf if den == 0.0 else nb[0] * tol / den
        for k in range(4, f64_slices):
            if (2.0 ** (2 - 7 * k) if k <= 8 else 2.0 ** -55) <= uj:
                fmt[j] = FMT_F64E(k)
                break
    return fmt, nb


def cost_ratio(s: int, r: int, digits_wp: float, d):
    """Eq. (3.8) read as a ratio of digit-weighted product counts:
    C_r = ((s-1) D + sum_i d_i) / ((s+r-1) D), D = digits of the working precision.
    (The printed formula writes log10 u for D; Table 1's column is 1 - C_r.)"""
    return ((s - 1) * digits_wp + sum(d)) / ((s + r - 1) * digits_wp)


# ------------------------------------------------------------------------------------
# FP8 (E4M3) products with one power-of-two scale per 32 inner-dimension entries
# ------------------------------------------------------------------------------------
E4M3_MAX = 448.0
MX_BLOCK = 32


def e4m3_round(x):
    """Nearest E4M3 number to x, ties to the even fraction.  E4M3 is the 8-bit float with 4
    exponent bits (bias 7) and 3 fraction bits: normal numbers 2^e (1 + f/8) for e in
    [-6, 8], subnormals j 2^-9 (j < 8), largest finite 448.  Requires |x| <= 448.  The
    spacing of the numbers around |x| is 2^(e-3) with e = max(floor(log2 |x|), -6)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    if np.any(a > E4M3_MAX):
        raise ValueError("e4m3_round: |x| > 448")
    _, E = np.frexp(a)                      # a = f 2^E, f in [0.5, 1): floor(log2 a) = E - 1
    e = np.maximum(E - 1, -6)
    quantum = np.ldexp(1.0, e - 3)
    q = np.round(a / quantum) * quantum     # a / quantum is exact; np.round ties to even
    return np.copysign(q, x)


def mx_block_exp(amax: float) -> int:
    """Shared exponent X of one block with largest magnitude amax: the smallest integer with
    amax 2^-X <= 448, so that the block's entries scaled by 2^-X fit E4M3 without clamping
    (0 for an all-zero block), kept in the range [-127, 127] of the 8-bit scale code
    X + 127."""
    if amax == 0.0:
        return 0
    f, E = math.frexp(amax)                 # amax = f 2^E, f in [0.5, 1)
    X = E - 9 if 512.0 * f <= E4M3_MAX else E - 8
    return min(max(X, -127), 127)


def mxfp8_quantize_rows(M):
    """Each row of M: first its own power of two, 2^-e with e the frexp exponent of the row's
    largest magnitude (rows then lie in (-1, 1); e = 0 for a zero row), then blocks of 32
    consecutive entries, block j scaled by 2^-X_j (mx_block_exp of the block's largest
    magnitude) and rounded to E4M3.  Returns (q, X, e): q the E4M3 values (n_rows x n_cols),
    X the block exponents (n_rows x ceil(n_cols/32)), e the row exponents.  The row equals
    2^e sum_j 2^X_j q_block_j up to the rounding."""
    M = np.asarray(M, dtype=np.float64)
    nr, nc = M.shape
    nb = -(-nc // MX_BLOCK)
    e = np.zeros(nr, dtype=np.int64)
    X = np.zeros((nr, nb), dtype=np.int64)
    q = np.zeros_like(M)
    for i in range(nr):
        rmax = float(np.max(np.abs(M[i]))) if nc else 0.0
        e[i] = math.frexp(rmax)[1] if rmax > 0.0 else 0
        v = np.ldexp(M[i], -int(e[i]))
        for j in range(nb):
            blk = v[j * MX_BLOCK:(j + 1) * MX_BLOCK]
            X[i, j] = mx_block_exp(float(np.max(np.abs(blk))))
            q[i, j * MX_BLOCK:(j + 1) * MX_BLOCK] = e4m3_round(np.ldexp(blk, -int(X[i, j])))
    return q, X, e


def _mx_dequantize(q, X, e):
    scale = np.repeat(np.ldexp(1.0, X), MX_BLOCK, axis=1)[:, :q.shape[1]]
    return np.ldexp(q * scale, e[:, None])


def matmul_mxfp8(A, B):
    """A B with the rows of A and the columns of B quantised by ``mxfp8_quantize_rows``: the
    quantised factors are exact in FP64 and the inner products are summed in FP64.  Also
    returns |A~| |B~| of the quantised factors (the scale of an FP32 accumulation error)."""
    qa, xa, ea = mxfp8_quantize_rows(A)
    qb, xb, eb = mxfp8_quantize_rows(np.asarray(B, dtype=np.float64).T)
    Aq = _mx_dequantize(qa, xa, ea)
    Bq = _mx_dequantize(qb, xb, eb).T
    return Aq @ Bq, np.abs(Aq) @ np.abs(Bq)

