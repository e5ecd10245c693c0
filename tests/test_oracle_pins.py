"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: exact rational
arithmetic, closed forms, special cases that reduce to a textbook or library routine,
printed values of the paper, and invariants.  All run on the CPU.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import GOLDEN

RNG = np.random.default_rng(20231217)


# --------------------------------------------------------------------------------
# helpers: exact rational matrix algebra (small n only)
# --------------------------------------------------------------------------------
def fr_matmul(A, B):
    n = len(A)
    return [[sum((A[i][k] * B[k][j] for k in range(n)), Fraction(0)) for j in range(n)]
            for i in range(n)]


def fr_poly(coefs, X):
    """sum_k c_k X^k, the plain definition, in exact rationals."""
    n = len(X)
    I = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    P = [[Fraction(0)] * n for _ in range(n)]
    K = I
    for k, c in enumerate(coefs):
        if k > 0:
            K = fr_matmul(K, X)
        for i in range(n):
            for j in range(n):
                P[i][j] += c * K[i][j]
    return P


def dyadic_matrix(n, denom=8, lo=-6, hi=7, rng=RNG):
    ints = rng.integers(lo, hi, size=(n, n))
    return ints / denom, [[Fraction(int(v), denom) for v in row] for row in ints]


def max_rel_exact(ph, pl, exact):
    """max_ij |(hi + lo) - exact| / max_ij |exact|, in exact arithmetic."""
    n = len(exact)
    scale = max(abs(v) for row in exact for v in row)
    err = max(abs(Fraction(float(ph[i, j])) + Fraction(float(pl[i, j])) - exact[i][j])
              for i in range(n) for j in range(n))
    return float(err / scale) if scale else float(err)


# --------------------------------------------------------------------------------
# 1. the double-double PS core against exact rational arithmetic
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(2, 4), (3, 9), (4, 16), (3, 13)])
def test_ps_dd_matches_exact_rationals(n, m):
    Xf, Xq = dyadic_matrix(n)
    Xf /= 4.0
    Xq = [[v / 4 for v in row] for row in Xq]
    coefs = oracle.taylor_exp_rational(m)
    exact = fr_poly(coefs, Xq)
    ph, pl, _ = oracle.ps_dd(coefs, Xf)
    assert max_rel_exact(ph, pl, exact) < 1e-30


def test_ps_dd_general_coefficients_exact():
    # signed, non-decaying coefficients: catches sign and index slips in B_i assembly
    coefs = [Fraction(k * (-1) ** k + 1, k + 2) for k in range(12)]
    Xf, Xq = dyadic_matrix(4)
    exact = fr_poly(coefs, Xq)
    for s in (1, 2, 3, 4, 5, 11, 12):
        ph, pl, _ = oracle.ps_dd(coefs, Xf, s=s)
        assert max_rel_exact(ph, pl, exact) < 1e-30, s


def test_planted_mistake_is_caught():
    """A plausible oracle mistake (one coefficient dropped) must fail the exact pin."""
    coefs = oracle.taylor_exp_rational(9)
    Xf, Xq = dyadic_matrix(3)
    exact = fr_poly(coefs, Xq)
    wrong = list(coefs)
    wrong[5] = Fraction(0)
    ph, pl, _ = oracle.ps_dd(wrong, Xf)
    assert max_rel_exact(ph, pl, exact) > 1e-6


# --------------------------------------------------------------------------------
# 2. PS = Horner = explicit powers (eq. (1.1) with s = 1, ceil(sqrt(m)), m)
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("m", [1, 2, 7, 16, 30])
def test_schemes_agree(m):
    n = 9
    X = RNG.standard_normal((n, n))
    X /= oracle.norm1(X)
    c = oracle.taylor_exp_rational(m)
    ref_h, ref_l = oracle.powers_dd(c, X)
    scale = oracle.norm1(ref_h)
    for s in sorted({1, oracle.ceil_sqrt(m), m}):
        ph, pl, _ = oracle.ps_dd(c, X, s=s)
        assert oracle.norm1((ph - ref_h) + (pl - ref_l)) / scale < 1e-29
    hh, hl, cnt = oracle.horner_dd(c, X)
    assert cnt == m
    assert oracle.norm1((hh - ref_h) + (hl - ref_l)) / scale < 1e-29


# --------------------------------------------------------------------------------
# 3. multiplication count of Algorithm 2.1: s - 1 + r (Section 3.4)
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("m,s,expected", [(16, 4, 7), (30, 6, 10), (12, 4, 6), (18, 5, 7),
                                          (24, 5, 8), (13, 4, 6), (42, 7, 12), (182, 14, 26)])
def test_multiplication_count(m, s, expected):
    assert oracle.ceil_sqrt(m) == s
    X = np.diag(np.linspace(0.1, 0.2, 3))
    _, _, cnt = oracle.ps_dd(oracle.taylor_exp_rational(m), X)
    assert cnt == expected == s - 1 + m // s


# --------------------------------------------------------------------------------
# 4. nilpotent Jordan block and lambda*I + J (closed forms; X^s = 0 gives p = B_0)
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("m", [5, 16, 30])
def test_nilpotent_jordan_exact(m):
    n = 8
    J = np.diag(np.ones(n - 1), 1)
    c = oracle.taylor_exp_rational(m)
    chi, clo = oracle.to_dd(c)
    ph, pl, _ = oracle.ps_dd(c, J)
    for i in range(n):
        for j in range(n):
            k = j - i
            if 0 <= k <= m:
                assert ph[i, j] == chi[k] and pl[i, j] == clo[k], (i, j)
            else:
                assert ph[i, j] == 0.0 and pl[i, j] == 0.0


def test_shifted_jordan_derivatives():
    n, m, lam = 6, 12, Fraction(1, 2)
    X = 0.5 * np.eye(n) + np.diag(np.ones(n - 1), 1)
    c = [Fraction(k + 1, 3 ** k) * (-1) ** (k // 2) for k in range(m + 1)]
    ph, pl, _ = oracle.ps_dd(c, X)
    for k in range(n):
        # p^{(k)}(lam)/k! = sum_j c_j binom(j, k) lam^(j-k)
        exact = sum((cj * math.comb(j, k) * lam ** (j - k) for j, cj in enumerate(c) if j >= k),
                    Fraction(0))
        got = Fraction(float(ph[0, k])) + Fraction(float(pl[0, k]))
        assert abs(float((got - exact) / exact)) < 1e-29


def test_nilpotent_strictly_upper_triangular():
    """100*triu(randn(n),1) (Section 3.4.3 class B): X^n = 0, p(X) = sum_{k<n} b_k X^k."""
    n = 5
    X = 100 * np.triu(RNG.standard_normal((n, n)), 1)
    X = np.round(X * 4) / 4  # dyadic entries: exact rationals available
    Xq = [[Fraction(float(v)) for v in row] for row in X]
    c = oracle.taylor_exp_rational(20)
    exact = fr_poly(c[:n], Xq)       # higher powers vanish
    ph, pl, _ = oracle.ps_dd(c, X)
    assert max_rel_exact(ph, pl, exact) < 1e-30


# --------------------------------------------------------------------------------
# 5. diagonal matrices: p(D) = diag(p(d_i))
# --------------------------------------------------------------------------------
def test_diagonal():
    d = [Fraction(k, 8) for k in (-7, -3, 0, 1, 5, 9)]
    c = oracle.pade_exp_num_rational(13)
    ph, pl, _ = oracle.ps_dd(c, np.diag([float(x) for x in d]))
    for i, di in enumerate(d):
        exact = sum((cj * di ** j for j, cj in enumerate(c)), Fraction(0))
        got = Fraction(float(ph[i, i])) + Fraction(float(pl[i, i]))
        assert abs(float(got - exact)) <= 1e-30 * max(1.0, abs(float(exact)))
    off = ph - np.diag(np.diag(ph))
    assert np.all(off == 0.0)


# --------------------------------------------------------------------------------
# 6. exp via scaling and squaring: rotations, group property, library routines
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [0.3, 1.0, 2.5, 7.0])
def test_rotation_generator(theta):
    A = np.array([[0.0, -theta], [theta, 0.0]])
    sigma = oracle.sigma_for(A)
    eh, el = oracle.expm_ss_dd(A, 30, sigma)
    E = eh + el
    ref = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    assert np.max(np.abs(E - ref)) < 4e-16


def test_rotation_generator_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    theta = 2.5
    A = np.array([[0.0, -theta], [theta, 0.0]])
    eh, el = oracle.expm_ss_dd(A, 30, oracle.sigma_for(A))
    c, s = mp.cos(theta), mp.sin(theta)
    ref = [[c, -s], [s, c]]
    for i in range(2):
        for j in range(2):
            got = mp.mpf(float(eh[i, j])) + mp.mpf(float(el[i, j]))
            assert abs(got - ref[i][j]) < mp.mpf("1e-29")


def test_group_property_exp_a_exp_minus_a():
    n = 12
    A = RNG.standard_normal((n, n))
    A *= 3.0 / oracle.norm1(A)
    sg = oracle.sigma_for(A)
    ph, pl = oracle.expm_ss_dd(A, 30, sg)
    mh, ml = oracle.expm_ss_dd(-A, 30, sg)
    ch, cl = oracle.matmul_dd(ph, pl, mh, ml)
    assert np.max(np.abs((ch - np.eye(n)) + cl)) < 1e-27
    # p(A) commutes with A
    ah, al = oracle.matmul_dd(ph, pl, A, None)
    bh, bl = oracle.matmul_dd(A, None, ph, pl)
    assert np.max(np.abs((ah - bh) + (al - bl))) < 1e-27 * np.max(np.abs(ah))


def test_against_scipy_expm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    for n, nrm in [(16, 0.5), (16, 4.0), (24, 32.0)]:
        A = RNG.standard_normal((n, n))
        A *= nrm / oracle.norm1(A)
        eh, el = oracle.expm_ss_dd(A, 30, oracle.sigma_for(A))
        ref = scipy_linalg.expm(A)
        assert oracle.norm1(eh - ref) / oracle.norm1(ref) < 5e-14


def test_against_mpmath_expm():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 45
    n = 5
    A = RNG.standard_normal((n, n))
    A *= 2.0 / oracle.norm1(A)
    eh, el = oracle.expm_ss_dd(A, 30, oracle.sigma_for(A))
    ref = mp.expm(mp.matrix(A.tolist()))
    err = max(abs(mp.mpf(float(eh[i, j])) + mp.mpf(float(el[i, j])) - ref[i, j])
              for i in range(n) for j in range(n))
    scale = max(abs(ref[i, j]) for i in range(n) for j in range(n))
    assert err / scale < mp.mpf("1e-29")


def test_sigma_rule():
    assert oracle.sigma_for(np.array([[0.5]])) == 0
    assert oracle.sigma_for(np.array([[1.0]])) == 0
    assert oracle.sigma_for(np.array([[1.0000001]])) == 1
    assert oracle.sigma_for(np.array([[4.0]])) == 2
    assert oracle.sigma_for(np.array([[32.0]])) == 5
    assert oracle.sigma_for(np.array([[33.0]])) == 6


# --------------------------------------------------------------------------------
# 7. columns of p(X)^k by Horner on vectors agree with the full evaluation
# --------------------------------------------------------------------------------
def test_apply_columns_matches_full():
    n = 20
    A = RNG.standard_normal((n, n))
    A *= 4.0 / oracle.norm1(A)
    sg = oracle.sigma_for(A)
    X = np.ldexp(A, -sg)
    c = oracle.taylor_exp_rational(30)
    eh, el = oracle.expm_ss_dd(A, 30, sg)
    cols = [0, 7, 19]
    V = np.zeros((n, len(cols)))
    for t, j in enumerate(cols):
        V[j, t] = 1.0
    wh, wl = oracle.ps_apply_dd(c, X, V, reps=2 ** sg)
    ref = (eh + el)[:, cols]
    assert np.max(np.abs((wh + wl) - ref)) < 1e-28 * np.max(np.abs(ref)) + 1e-300
    assert np.max(np.abs((wh - eh[:, cols]) + (wl - el[:, cols]))) < 1e-28 * np.max(np.abs(ref))


# --------------------------------------------------------------------------------
# 8. adjoint: block-triangular identity, duality, Daleckii-Krein, finite differences
# --------------------------------------------------------------------------------
def frechet_block(c, A, E):
    """L_p(A, E) from p([[A, E], [0, A]]) = [[p(A), L_p(A, E)], [0, p(A)]]."""
    n = A.shape[0]
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = A; M[n:, n:] = A; M[:n, n:] = E
    ph, pl, _ = oracle.ps_dd(c, M)
    return ph[:n, n:], pl[:n, n:]


def test_adjoint_block_identity_duality():
    n, m = 6, 10
    c = oracle.taylor_exp_rational(m)
    A = RNG.standard_normal((n, n)) * 0.4
    G = RNG.standard_normal((n, n))
    E = RNG.standard_normal((n, n))
    gh, gl = oracle.adjoint_dd(c, A, G)
    Lh, Ll = frechet_block(c, A, E)
    lhs = np.sum((gh + gl) * E)
    rhs = np.sum((Lh + Ll) * G)
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)
    # the gradient is L_p(A^T, G): check it entrywise with the block identity
    Lt_h, Lt_l = frechet_block(c, A.T.copy(), G)
    assert np.max(np.abs((gh - Lt_h) + (gl - Lt_l))) < 1e-28 * np.max(np.abs(gh))


def test_adjoint_diagonal_closed_form():
    d = np.array([-0.7, -0.1, 0.3, 0.9])
    n = len(d)
    c = oracle.taylor_exp_rational(14)
    cf = [float(x) for x in c]
    p = lambda x: sum(cj * x ** j for j, cj in enumerate(cf))
    dp = lambda x: sum(j * cj * x ** (j - 1) for j, cj in enumerate(cf) if j > 0)
    G = RNG.standard_normal((n, n))
    gh, gl = oracle.adjoint_dd(c, np.diag(d), G)
    for i in range(n):
        for j in range(n):
            ref = G[i, j] * (dp(d[i]) if i == j else (p(d[i]) - p(d[j])) / (d[i] - d[j]))
            assert abs(gh[i, j] - ref) < 1e-14 * max(1.0, abs(ref))


def test_adjoint_central_differences():
    n, m = 5, 8
    c = oracle.taylor_exp_rational(m)
    A = RNG.standard_normal((n, n)) * 0.3
    G = RNG.standard_normal((n, n))
    gh, gl = oracle.adjoint_dd(c, A, G)
    h = 1e-6
    for (i, j) in [(0, 0), (1, 3), (4, 2)]:
        E = np.zeros((n, n)); E[i, j] = h
        ph, pl, _ = oracle.ps_dd(c, A + E)
        mh, ml, _ = oracle.ps_dd(c, A - E)
        fd = (np.sum(G * (ph - mh)) + np.sum(G * (pl - ml))) / (2 * h)
        assert abs(fd - gh[i, j]) < 1e-9 * max(1.0, abs(gh[i, j]))


@pytest.mark.parametrize("sigma", [0, 1, 3])
def test_expm_ss_adjoint_block_identity(sigma):
    """The scaling-and-squaring approximant r(A) = p(2^-sigma A)^(2^sigma) is a polynomial in
    A for fixed sigma, so <grad, E> = <G, r([[A, E], [0, A]])_12> with r evaluated by the
    independent forward routine (Algorithm 2.1 then sigma squarings on the 2n matrix)."""
    n, m = 6, 12
    A = RNG.standard_normal((n, n)) * 0.5
    G = RNG.standard_normal((n, n))
    E = RNG.standard_normal((n, n))
    gh, gl = oracle.expm_ss_adjoint_dd(A, G, m, sigma)
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = A; M[n:, n:] = A; M[:n, n:] = E
    eh, el = oracle.expm_ss_dd(M, m, sigma)
    lhs = math.fsum((gh * E).ravel()) + math.fsum((gl * E).ravel())
    rhs = math.fsum((G * eh[:n, n:]).ravel()) + math.fsum((G * el[:n, n:]).ravel())
    scale = math.fsum(np.abs(G * eh[:n, n:]).ravel())
    assert abs(lhs - rhs) < 1e-14 * scale
    # entrywise: grad = L_r(A^T, G) = r([[A^T, G], [0, A^T]])_12
    Mt = np.zeros((2 * n, 2 * n))
    Mt[:n, :n] = A.T; Mt[n:, n:] = A.T; Mt[:n, n:] = G
    th, tl = oracle.expm_ss_dd(Mt, m, sigma)
    assert np.max(np.abs((gh - th[:n, n:]) + (gl - tl[:n, n:]))) < 1e-26 * np.max(np.abs(gh))


def test_expm_ss_adjoint_diagonal_closed_form():
    """For A = diag(d) the gradient is G_ij r[d_i, d_j] (divided differences of the scalar
    r(x) = p(2^-sigma x)^(2^sigma), r'(d_i) on the diagonal), here in 40-digit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    d = np.array([-1.75, -0.5, 0.25, 1.5, 3.0])
    n, m, sigma = len(d), 16, 2
    c = [mpmath.mpf(x.numerator) / x.denominator for x in oracle.taylor_exp_rational(m)]
    p = lambda y: sum(cj * y ** j for j, cj in enumerate(c))
    dp = lambda y: sum(j * cj * y ** (j - 1) for j, cj in enumerate(c) if j > 0)
    q = 2 ** sigma
    r = lambda x: p(mpmath.mpf(x) / q) ** q
    dr = lambda x: p(mpmath.mpf(x) / q) ** (q - 1) * dp(mpmath.mpf(x) / q)
    G = RNG.standard_normal((n, n))
    gh, gl = oracle.expm_ss_adjoint_dd(np.diag(d), G, m, sigma)
    for i in range(n):
        for j in range(n):
            dd_ = dr(d[i]) if i == j else (r(d[i]) - r(d[j])) / (mpmath.mpf(d[i]) - mpmath.mpf(d[j]))
            ref = mpmath.mpf(G[i, j]) * dd_
            got = mpmath.mpf(gh[i, j]) + mpmath.mpf(gl[i, j])
            assert abs(got - ref) <= mpmath.mpf(1e-28) * max(1, abs(ref))


def test_expm_ss_adjoint_central_differences():
    n, m, sigma = 5, 10, 2
    A = RNG.standard_normal((n, n)) * 0.8
    G = RNG.standard_normal((n, n))
    gh, gl = oracle.expm_ss_adjoint_dd(A, G, m, sigma)
    h = 1e-6
    for (i, j) in [(0, 0), (2, 4), (3, 1)]:
        E = np.zeros((n, n)); E[i, j] = h
        ph, pl = oracle.expm_ss_dd(A + E, m, sigma)
        mh, ml = oracle.expm_ss_dd(A - E, m, sigma)
        fd = (np.sum(G * (ph - mh)) + np.sum(G * (pl - ml))) / (2 * h)
        assert abs(fd - gh[i, j]) < 1e-8 * max(1.0, abs(gh[i, j]))


def test_expm_ss_adjoint_pin_catches_planted_mistakes():
    """The block-identity pin above separates the chain rule from plausible slips: the same
    chain in plain double passes it, and the chain with the transposes dropped from the
    squarings' reverse step, or without the final 2^-sigma, fails it."""
    n, m, sigma = 6, 12, 2
    A = RNG.standard_normal((n, n)) * 0.5
    G = RNG.standard_normal((n, n))
    c = oracle.taylor_exp_rational(m)
    Mt = np.zeros((2 * n, 2 * n))
    Mt[:n, :n] = A.T; Mt[n:, n:] = A.T; Mt[:n, n:] = G
    th, tl = oracle.expm_ss_dd(Mt, m, sigma)
    ref = th[:n, n:] + tl[:n, n:]

    def chain(transpose=True, scale=True):
        X = np.ldexp(A, -sigma)
        ph, pl, _ = oracle.ps_dd(c, X)
        S = [ph + pl]
        for _ in range(sigma - 1):
            S.append(S[-1] @ S[-1])
        Sb = G.copy()
        for k in range(sigma - 1, -1, -1):
            T = S[k].T if transpose else S[k]
            Sb = Sb @ T + T @ Sb
        dh, dl = oracle.adjoint_dd(c, X, Sb)
        D = dh + dl
        return np.ldexp(D, -sigma) if scale else D

    rel = lambda D: np.max(np.abs(D - ref)) / np.max(np.abs(ref))
    assert rel(chain()) < 1e-13
    assert rel(chain(transpose=False)) > 1e-3
    assert rel(chain(scale=False)) > 1e-1


def test_choose_s_variable_branch_by_hand():
    """Algorithm 3.1's variable-s loop on norms worked out by hand (m = 30, s0 = 6)."""
    # ||X|| = 3 > 6/e: the branch is not taken
    assert oracle.choose_s(30, 3.0, [0.5], [10.0]) == 6
    # ||X|| = 1/2: ||X||^6 = 1/64, ^7 = 1/128, ^8 = 1/256
    #   s = 6: 0.02 > 0.5/64 = 0.0078 -> 7;  s = 7: 0.015 > 0.0039 -> 8;
    #   s = 8: 0.001 > 0.00195 fails -> stop at 8
    assert oracle.choose_s(30, 0.5, [0.5, 0.5, 0.5], [0.02, 0.015, 0.001]) == 8
    # the first test fails: s stays 6
    assert oracle.choose_s(30, 0.5, [0.5], [0.007]) == 6
    # growth stops at s = m (m = 5, s0 = 3)
    assert oracle.choose_s(5, 0.1, [1e-9] * 5, [1.0] * 5) == 5
    # and after the norms supplied (two of them)
    assert oracle.choose_s(30, 0.5, [1e-9, 1e-9], [1.0, 1.0]) == 8
    # ||X|| exactly at s0/e takes the branch
    assert oracle.choose_s(30, 6 / math.e, [1e-9], [1.0]) == 7


# --------------------------------------------------------------------------------
# 9. the paper's printed worked example and tables
# --------------------------------------------------------------------------------
def _read_kv(path):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out.setdefault(key, []).append(vals)
    return out


def test_ward_pade13_coefficients_exact():
    g = _read_kv(os.path.join(GOLDEN, "ward_pade13.txt"))
    c = oracle.pade_exp_num_rational(13)
    assert c[:4] == [Fraction(v) for v in g["B0_coefficients"][0]]
    assert c[4:8] == [Fraction(v) for v in g["B1_coefficients"][0]]
    # denominator is p(-X)
    assert oracle.pade_exp_den_rational(13) == [(-1) ** j * cj for j, cj in enumerate(c)]
    # c_j sum to the [13/13] approximant's value at 1 over its value at -1 -> e to 1e-25
    num = sum(c); den = sum(oracle.pade_exp_den_rational(13))
    assert abs(float(num / den) - math.e) < 1e-15


def test_ward_example_decay():
    """eq. (2.5) holds on the Ward example with nu = 1: tau_1 << 1 and tau_3 < tau_2 < tau_1.
    The printed magnitudes are not reproducible from the printed data (see the readings
    of the paper in the design notes); only the decay they illustrate is pinned."""
    g = _read_kv(os.path.join(GOLDEN, "ward_pade13.txt"))
    A = np.array([[float(v) for v in row] for row in g["matrix_row"]])
    ell = int(g["scaling_exponent"][0][0]); s = int(g["s"][0][0])
    X = np.ldexp(A, -ell)
    norms, y = oracle.block_norms_dd(oracle.pade_exp_num_rational(13), X, s)
    tau = [norms[i] * y / norms[i - 1] for i in range(1, len(norms))]
    assert tau[0] < 1e-2 and tau[1] < tau[0] and tau[2] < tau[1]


def test_table1_parameters_and_cost_ratio():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1_cauchy100.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, ds, pct = line.split("|")
        D, m, s, r = (int(v) for v in head.split())
        rows.append((D, m, s, r, [int(v) for v in ds.split()], float(pct)))
    assert len(rows) == 4
    for D, m, s, r, d, pct in rows:
        assert oracle.ceil_sqrt(m) == s and m // s == r and len(d) == r
        assert all(d[i] >= d[i + 1] for i in range(r - 1))
        saving = 100.0 * (1.0 - oracle.cost_ratio(s, r, D, d))
        assert abs(saving - pct) < 0.05, (D, saving, pct)


# --------------------------------------------------------------------------------
# 10. the precision rule with hand-derived answers
# --------------------------------------------------------------------------------
F = oracle


def test_plan_hand_case_paper_mode():
    # m = 16, s = 4, r = 4, s | m -> step 4 folded.  tol = 2^-53 = 1.11e-16.
    # u_1 = 1 * tol / (1e-3 * 0.5)     = 2.2e-13 -> only FP64 (nu = 1 since >= 10 tol)
    # u_2 = tol / (1e-9 * 0.25)        = 4.4e-7  -> below 2^-16 -> FP64
    # u_3 = tol / (1e-15 * 0.125)      = 0.89    -> FP8 (2^-4 <= 0.89, 64 * 2^-24 <= 0.89)
    p = F.plan(16, 64, [1.0, 1e-3, 1e-9, 1e-15, 1e-21], 0.5, mode=F.MODE_PAPER)
    assert (p["s"], p["r"], p["nu"], p["fold"]) == (4, 4, 1, True)
    assert p["fmt"][1:] == [F.FMT_FP64, F.FMT_FP64, F.FMT_FP8, F.FMT_NONE]
    assert p["u"][1] == pytest.approx(2.0 ** -53 / 5e-4)
    assert p["u"][3] == pytest.approx(2.0 ** -53 / 1.25e-16)


def test_plan_hand_case_ladder():
    # u_i chosen so that each format boundary is crossed once; n = 16
    tol = 2.0 ** -53
    y = 1.0
    # u_i = tol / eta_i: pick eta_i = tol / target
    targets = [None, 2e-5, 6e-4, 5e-3, 0.07]     # -> BF16X3, TF32, BF16, FP8
    norms = [1.0] + [tol / t for t in targets[1:]] + [1e-30]
    p = F.plan(20, 16, norms, y, mode=F.MODE_PAPER, s=4)   # r = 5, 4 does not... 20 % 4 == 0
    assert p["r"] == 5 and p["fold"]
    assert p["fmt"][1:5] == [F.FMT_BF16X3, F.FMT_TF32, F.FMT_BF16, F.FMT_FP8]
    # masks remove formats: without FP8 and BF16, the 0.07 step falls back to TF32
    mask = (1 << F.FMT_FP64) | (1 << F.FMT_BF16X3) | (1 << F.FMT_TF32)
    q = F.plan(20, 16, norms, y, mode=F.MODE_PAPER, s=4, formats=mask)
    assert q["fmt"][1:5] == [F.FMT_BF16X3, F.FMT_TF32, F.FMT_TF32, F.FMT_TF32]
    # NS floors keep steps 1 and 2 in FP64
    ns = F.plan(20, 16, norms, y, mode=F.MODE_NS, s=4)
    assert ns["fmt"][1:5] == [F.FMT_FP64, F.FMT_FP64, F.FMT_BF16, F.FMT_FP8]
    fx = F.plan(20, 16, norms, y, mode=F.MODE_FIXED, s=4)
    assert fx["fmt"][1:5] == [F.FMT_FP64] * 4 and fx["fmt"][5] == F.FMT_NONE


def test_plan_nu_and_accumulation_check():
    tol = 2.0 ** -53
    # u_1 = tol (not >= 10 tol), u_2 huge -> nu = 2, u_1 reset to tol
    p = F.plan(9, 64, [1.0, 1.0, 1e-20, 1e-30], 1.0, mode=F.MODE_PAPER)
    assert p["s"] == 3 and p["r"] == 3 and p["nu"] == 2
    assert p["u"][1] == tol and p["fmt"][1] == F.FMT_FP64
    assert p["fmt"][2] == F.FMT_FP8
    # with n = 2^20 every FP32-accumulated format needs u_i >= 1/16
    big = F.plan(9, 2 ** 20, [1.0, 1.0, tol / 0.05, 1e-30], 1.0, mode=F.MODE_PAPER)
    assert big["fmt"][2] == F.FMT_FP64
    # zero block: no error contribution -> cheapest format
    z = F.plan(9, 64, [1.0, 0.0, 1e-20, 1e-30], 1.0, mode=F.MODE_PAPER)
    assert z["fmt"][1] == F.FMT_FP8 and z["nu"] == 1


def test_plan_degenerate():
    assert F.plan(0, 8, [1.0], 0.0)["r"] == 0
    p1 = F.plan(1, 8, [1.0, 1.0], 1.0)      # s = 1, r = 1, folded (b_1 I)
    assert (p1["s"], p1["r"], p1["fold"]) == (1, 1, True)


# --------------------------------------------------------------------------------
# 12. the plain-double oracle (the timed CPU baseline): exact on dyadic inputs, and within
#     the rounding-error bound of Algorithm 2.1 (Lemma 2.2 / Theorem 2.1 with every u_i = u)
#     of the double-double oracle
# --------------------------------------------------------------------------------
def _ps_d_bound(coefs, X, s):
    """Normwise form of the fixed-precision bound: the computed P differs from p(X) by at
    most (s - 1 + r + 1) n u sum_k |b_k| || |X| ||_1^k (first order in u)."""
    m = len(coefs) - 1
    r = m // s
    nx = oracle.norm1(np.abs(X))
    tail = sum(abs(float(c)) * nx ** k for k, c in enumerate(coefs))
    return (s + r) * X.shape[0] * 2.0 ** -53 * tail


@pytest.mark.parametrize("n,m", [(3, 9), (4, 16), (2, 7)])
def test_ps_d_exact_on_dyadic_inputs(n, m):
    # dyadic X and coefficients 2^-k: every product and sum of Algorithm 2.1 is exact in
    # double, so the plain-double result equals the exact rational value bit for bit
    Xf, Xq = dyadic_matrix(n, denom=2, lo=-1, hi=2)
    coefs = [Fraction(1, 2 ** k) for k in range(m + 1)]
    exact = fr_poly(coefs, Xq)
    for s in (0, 1, 2, m):
        P, _ = oracle.ps_d([float(c) for c in coefs], Xf, s=s)
        assert all(Fraction(float(P[i, j])) == exact[i][j] for i in range(n) for j in range(n)), s


@pytest.mark.parametrize("n,m", [(5, 7), (33, 16), (64, 30)])
def test_ps_d_within_bound_of_dd(n, m):
    # order-one signed coefficients so that every term of p carries weight
    rng = np.random.default_rng(900 + n + m)
    coefs = list(rng.standard_normal(m + 1) / np.arange(1, m + 2))
    X = rng.standard_normal((n, n))
    X /= oracle.norm1(X)
    s = oracle.ceil_sqrt(m)
    ph, pl, _ = oracle.ps_dd(coefs, X)
    P, cnt = oracle.ps_d(coefs, X)
    assert cnt == s - 1 + m // s
    err = oracle.norm1(P - ph - pl)
    assert err <= _ps_d_bound(coefs, X, s)
    assert err > 0.0          # plain double does round (the comparison is not vacuous)


def test_ps_d_bound_catches_planted_mistakes():
    """Oracle-side slips in a plain-double PS (a dropped block coefficient, one Horner
    step too few) leave the bound by more than two orders of magnitude."""
    n, m = 33, 16
    rng = np.random.default_rng(77)
    coefs = list(rng.standard_normal(m + 1) / np.arange(1, m + 2))
    X = rng.standard_normal((n, n))
    X /= oracle.norm1(X)
    ph, pl, _ = oracle.ps_dd(coefs, X)
    bound = _ps_d_bound(coefs, X, 4)
    dropped = list(coefs); dropped[9] = 0.0
    P1, _ = oracle.ps_d(dropped, X)
    assert oracle.norm1(P1 - ph - pl) > 100 * bound
    short = coefs[:-4]                      # the top block B_r missing
    P2, _ = oracle.ps_d(short, X)
    assert oracle.norm1(P2 - ph - pl) > 100 * bound


@pytest.mark.parametrize("n,norm", [(8, 0.5), (24, 4.0), (40, 32.0)])
def test_expm_ss_d_within_bound_of_dd(n, norm):
    A = RNG.standard_normal((n, n))
    A *= norm / oracle.norm1(A)
    sg = oracle.sigma_for(A)
    eh, el = oracle.expm_ss_dd(A, 30, sg)
    E = oracle.expm_ss_d(A, 30, sg)
    err = oracle.rel_err_1norm(E, eh, el)
    # the polynomial's bound, amplified by 2^sigma through the squarings (Section 3.2)
    assert err <= 50 * n * 2.0 ** -53 * 2 ** sg
    # the result of one squaring too many, p(2^-sigma A)^(2^(sigma+1)) = E^2, and of one too
    # few, p(2^-sigma A)^(2^(sigma-1)) (the oracle run on A/2 with sigma-1), are far outside it
    assert oracle.rel_err_1norm(E @ E, eh, el) > 1e-3
    if sg > 0:
        assert oracle.rel_err_1norm(oracle.expm_ss_d(A / 2, 30, sg - 1), eh, el) > 1e-3


# --------------------------------------------------------------------------------
# 13. the cosine and Pade coefficient sequences against the functions they approximate
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("m", [8, 16])
def test_cos_taylor_coefficients_reproduce_cos(m):
    # c_m(B) with B = D^2, D diagonal: diag(sum_k (-1)^k d^(2k) / (2k)!) = diag(cos d) up to
    # the truncation term |d|^(2m+2) / (2m+2)!
    d = np.linspace(-4.0, 4.0, 13)
    B = np.diag(d * d)
    ph, pl, _ = oracle.ps_dd(oracle.cos_taylor_rational(m), B)
    for i, di in enumerate(d):
        trunc = abs(di) ** (2 * m + 2) / math.factorial(2 * m + 2)
        assert abs(ph[i, i] + pl[i, i] - math.cos(di)) <= trunc + 4e-16, (m, di)
    off = ph - np.diag(np.diag(ph))
    assert np.all(off == 0.0)


def test_cos_pin_catches_planted_mistake():
    # odd factorials in the denominators (the sine's sequence) do not reproduce cos
    wrong = [Fraction((-1) ** k, math.factorial(2 * k + 1)) for k in range(17)]
    B = np.diag([1.0, 2.0, 3.0])
    ph, pl, _ = oracle.ps_dd(wrong, B)
    assert max(abs(ph[i, i] - math.cos(math.sqrt(B[i, i]))) for i in range(3)) > 1e-2


def test_pade_coefficients_approximate_exp():
    # the [13/13] Pade approximant p(x)/q(x) agrees with e^x to order x^27: at |x| <= 1/2 the
    # difference is far below an FP64 ulp; p(-x) is q(x) exactly
    num, den = oracle.pade_exp_num_rational(13), oracle.pade_exp_den_rational(13)
    assert all(d == n * (-1) ** j for j, (n, d) in enumerate(zip(num, den)))
    for x in (Fraction(1, 2), Fraction(-1, 3), Fraction(1, 8)):
        p = sum(c * x ** j for j, c in enumerate(num))
        q = sum(c * x ** j for j, c in enumerate(den))
        assert abs(float(p / q) - math.exp(float(x))) <= 2.0 ** -52 * math.exp(float(x))


# --------------------------------------------------------------------------------
# 14. the 1-norm: maximum column sum, on a non-square matrix whose row and column maxima
#     differ (a row/column swap gives 6 instead of 7)
# --------------------------------------------------------------------------------
def test_norm1_hand_worked_3x4():
    M = np.array([[1.0, -2.0, 0.0, 3.0],
                  [4.0, 0.0, -1.0, 0.0],
                  [0.0, 5.0, 0.0, -1.0]])
    # column sums of |M|: 5, 7, 1, 4 ; row sums: 6, 5, 6
    assert oracle.norm1(M) == 7.0
    assert oracle.norm1(M.T) == 6.0
    assert oracle.norm1(np.array([[-3.0, 2.0, 1.0]])) == 3.0      # one row: max |entry|
    assert oracle.norm1(np.array([[-3.0], [2.0], [1.0]])) == 6.0  # one column: its sum
    R = RNG.standard_normal((7, 5))
    assert oracle.norm1(R) == np.abs(R).sum(axis=0).max()


# --------------------------------------------------------------------------------
# 15. the linear solve of the Pade approximant (Section 4.1: r = q^-1 p)
# --------------------------------------------------------------------------------
def _fr_inverse(A):
    """Gauss-Jordan in exact rationals (no pivoting choice matters for exactness)."""
    n = len(A)
    M = [[Fraction(v) for v in row] + [Fraction(int(i == j)) for j in range(n)]
         for i, row in enumerate(A)]
    for j in range(n):
        p = next(i for i in range(j, n) if M[i][j] != 0)
        M[j], M[p] = M[p], M[j]
        pv = M[j][j]
        M[j] = [v / pv for v in M[j]]
        for i in range(n):
            if i != j and M[i][j] != 0:
                f = M[i][j]
                M[i] = [a - f * b for a, b in zip(M[i], M[j])]
    return [row[n:] for row in M]


def test_lu_solve_hand_worked_3x3():
    # column 0: |4| at row 2 is the largest -> rows 0, 2 swap; the remaining rows read
    # [0, .5, .5] and [0, 1, 2]: column 1's pivot 1 is again in row 2 -> rows 1, 2 swap;
    # U = [[4, 7, 9], [0, 1, 2], [0, 0, -1/2]], det = -2: every step and the inverse are dyadic,
    # so the plain-double result is exact
    Q = [[0.0, 1.0, 2.0], [2.0, 4.0, 5.0], [4.0, 7.0, 9.0]]
    R, piv, info = oracle.lu_solve(np.array(Q), np.eye(3))
    assert info == 0 and list(piv) == [2, 2, 2]
    exact = _fr_inverse(Q)
    assert all(R[i, j] == float(exact[i][j]) for i in range(3) for j in range(3))


def test_lu_solve_exact_on_dyadic_factors():
    # Q = L0 U0 with |l_ij| <= 1/2 (so partial pivoting keeps the diagonal) and small dyadic
    # entries: elimination recovers the factors exactly and R = X0 for P = Q X0
    n = 6
    rng = np.random.default_rng(7)
    L0 = np.tril(rng.integers(-2, 3, (n, n)) / 4.0, -1) + np.eye(n)
    U0 = np.triu(rng.integers(-3, 4, (n, n)).astype(float), 1) + np.diag([2.0, -4, 1, 8, -2, 4])
    X0 = rng.integers(-5, 6, (n, n)).astype(float)
    Q, P = L0 @ U0, L0 @ U0 @ X0
    R, piv, info = oracle.lu_solve(Q, P)
    assert info == 0 and list(piv) == list(range(n))
    assert np.array_equal(R, X0)


def test_lu_solve_pivots_and_solution_match_lapack():
    # the pivot sequence is the one of LAPACK's getrf (first largest magnitude), the
    # solution agrees with getrs to rounding, and the residual is at rounding level
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    for n in (1, 2, 5, 33, 80):
        Q, P = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        R, piv, info = oracle.lu_solve(Q, P)
        lu, pv = sl.lu_factor(Q)
        assert info == 0 and np.array_equal(piv, pv)
        ref = sl.lu_solve((lu, pv), P)
        kappa = np.linalg.cond(Q, 1)
        assert np.abs(R - ref).max() <= 8 * n * kappa * 2.0 ** -53 * np.abs(ref).max()
        assert np.abs(Q @ R - P).max() <= 8 * n * 2.0 ** -53 * np.abs(Q).sum(1).max() * np.abs(R).max()


def test_lu_solve_zero_pivot_info():
    # rows 0 and 2 equal: column 2 loses its pivot (info = 3); a 0 leading entry is not a
    # zero pivot (an interchange cures it): the inverse of a swap is the swap
    Q = np.array([[1.0, 2.0, 3.0], [0.0, 1.0, 4.0], [1.0, 2.0, 3.0]])
    assert oracle.lu_solve(Q, np.eye(3))[2] == 3
    Z = np.array([[0.0, 1.0], [1.0, 0.0]])
    R, piv, info = oracle.lu_solve(Z, np.eye(2))
    assert info == 0 and list(piv) == [1, 1] and np.array_equal(R, Z)


# --------------------------------------------------------------------------------
# FP8 products with block scales
# --------------------------------------------------------------------------------
def _e4m3_table():
    """Every non-negative finite E4M3 number, decoded from its bit fields (exponent bits
    e, fraction bits f: e = 0 gives f 2^-9, otherwise 2^(e-7) (1 + f/8); e = 15, f = 7 is
    NaN), with its code's lowest bit."""
    vals, odd = [], []
    for code in range(0x7F):
        e, f = code >> 3, code & 7
        vals.append(f * 2.0 ** -9 if e == 0 else 2.0 ** (e - 7) * (1 + f / 8))
        odd.append(code & 1)
    return np.array(vals), np.array(odd)


def test_e4m3_table_endpoints():
    v, _ = _e4m3_table()
    assert np.all(np.diff(v) > 0)
    assert v[-1] == oracle.E4M3_MAX and v[1] == 2.0 ** -9 and v[8] == 2.0 ** -6


def test_e4m3_round_matches_torch_float8():
    # torch's float8_e4m3fn conversion from float32 (round to nearest even) on a grid that
    # holds every E4M3 number, every midpoint between neighbours and points just beside them
    torch = pytest.importorskip("torch")
    v, _ = _e4m3_table()
    mids = (v[1:] + v[:-1]) / 2
    pts = np.concatenate([v, mids, np.nextafter(mids.astype(np.float32), np.float32(0)),
                          np.nextafter(mids.astype(np.float32), np.float32(np.inf)),
                          RNG.uniform(0, 448, 20000), 2.0 ** RNG.uniform(-14, 8.8, 20000)])
    pts = pts[pts <= 448].astype(np.float32).astype(np.float64)
    pts = np.concatenate([pts, -pts])
    ref = torch.tensor(pts, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(oracle.e4m3_round(pts), ref)


def test_e4m3_round_is_nearest_even_by_search():
    # independent of the spacing formula: nearest entry of the decoded table, a tie going to
    # the even code
    v, odd = _e4m3_table()
    x = np.concatenate([RNG.uniform(0, 448, 3000), 2.0 ** RNG.uniform(-12, 8.8, 3000),
                        (v[1:] + v[:-1]) / 2])
    x = x[x <= 448]
    got = oracle.e4m3_round(x)
    for xi, gi in zip(x, got):
        d = np.abs(v - xi)
        best = np.flatnonzero(d == d.min())
        pick = best[0] if len(best) == 1 else best[odd[best] == 0][0]
        assert gi == v[pick], (xi, gi, v[pick])
    with pytest.raises(ValueError):
        oracle.e4m3_round(np.array([449.0]))


def test_mx_block_exp_brute_force_and_hand_cases():
    for amax in np.concatenate([2.0 ** RNG.uniform(-60, 60, 2000), [448.0, 449.0, 1.0, 0.875, 0.8751]]):
        X = next(x for x in range(-200, 200) if amax * 2.0 ** -x <= 448.0)
        assert oracle.mx_block_exp(float(amax)) == X
    assert oracle.mx_block_exp(448.0) == 0 and oracle.mx_block_exp(449.0) == 1
    assert oracle.mx_block_exp(1.0) == -8          # 1 * 2^8 = 256 <= 448 < 512
    assert oracle.mx_block_exp(0.0) == 0
    assert oracle.mx_block_exp(2.0 ** -300) == -127 and oracle.mx_block_exp(2.0 ** 300) == 127


def test_mxfp8_quantize_rows_per_block_scales():
    # blocks of one row 2^30 apart: each block keeps 3 fraction bits (relative error 2^-4 at
    # most); one scale per row would flush the small blocks to zero
    n = 96
    M = RNG.uniform(0.5, 1.0, (3, n)) * np.where(RNG.random((3, n)) < 0.5, -1, 1)
    M[:, 32:64] *= 2.0 ** -30
    M[1, 64:] *= 2.0 ** 20
    q, X, e = oracle.mxfp8_quantize_rows(M)
    assert X.shape == (3, 3) and np.all(np.abs(q) <= 448)
    Mq = oracle._mx_dequantize(q, X, e)
    assert np.all(np.abs(Mq - M) <= 2.0 ** -4 * np.abs(M))
    assert X[0, 1] == X[0, 0] - 30
    # integers up to 8 are exact; a ragged tail block and a zero row
    Z = RNG.integers(-8, 9, (4, 45)).astype(float)
    Z[2] = 0
    qz, Xz, ez = oracle.mxfp8_quantize_rows(Z)
    assert np.array_equal(oracle._mx_dequantize(qz, Xz, ez), Z) and ez[2] == 0 and np.all(Xz[2] == 0)


def test_matmul_mxfp8_exact_on_integers_and_bound():
    A = RNG.integers(-4, 5, (37, 70)).astype(float)
    B = RNG.integers(-4, 5, (70, 29)).astype(float)
    C, _ = oracle.matmul_mxfp8(A, B)
    assert np.array_equal(C, A @ B)
    # Gaussian factors: each quantised entry within 2^-4 of the original, or within half a
    # subnormal step 2^(e + X - 10) of its row and block; the product error follows from the
    # factor errors (a transposed or mis-scaled factor would not)
    A = RNG.standard_normal((40, 100)); B = RNG.standard_normal((100, 30))
    C, absprod = oracle.matmul_mxfp8(A, B)
    u = 2.0 ** -4
    deq = []
    for M in (A, B.T):
        q, X, e = oracle.mxfp8_quantize_rows(M)
        Mq = oracle._mx_dequantize(q, X, e)
        half_sub = np.ldexp(1.0, e[:, None] + np.repeat(X, 32, axis=1)[:, :M.shape[1]] - 10)
        assert np.all(np.abs(Mq - M) <= np.maximum(u * np.abs(M), half_sub))
        deq.append(Mq)
    dA, dB = np.abs(deq[0] - A), np.abs(deq[1].T - B)
    bound = dA @ np.abs(B) + np.abs(A) @ dB + dA @ dB + 4 * 100 * 2.0 ** -53 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - A @ B) <= bound)
    assert np.allclose(absprod, np.abs(deq[0]) @ np.abs(deq[1].T))
