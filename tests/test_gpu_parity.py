"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances
* FP64 products and fixed-FP64 PS: 1-norm relative error <= 50 n 2^-53 (the fixed path's
  bound used throughout; Section 3.4 reports errors of order r n u).
* Low-precision products: normwise |C - AB| <= k u_F |A||B| with u_F the format's unit
  roundoff, plus exactness on integer inputs that every format represents exactly.
* Mixed PS: the same 50 n 2^-53 bound, and within 2x of the fixed-FP64 error up to a
  floor of 4 ulps of ||P|| (4 u relative), both measured against the double-double oracle.
  The floor only covers inputs on which the fixed path happens to round almost exactly.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2312_17396_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
FLOOR = 4 * U   # "mixed within 2x of fixed" floor: a few ulps of ||P||


@pytest.fixture(scope="module")
def mpps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_17396_gb300 as m
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# ------------------------------------------------------------------------------------
# products
# ------------------------------------------------------------------------------------
SIZES = [1, 2, 3, 17, 64, 127, 130, 257]


@pytest.mark.parametrize("n", SIZES)
def test_matmul_fp64_vs_oracle(mpps, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((2, n, n)); B = rng.standard_normal((2, n, n))
    C = host(mpps.matmul(dev(A), dev(B), "fp64"))
    for b in range(2):
        ch, cl = oracle.matmul_dd(A[b], None, B[b], None)
        bound = n * U * (np.abs(A[b]) @ np.abs(B[b])) + 1e-300
        assert np.all(np.abs(C[b] - ch - cl) <= bound)


LOW = {"bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16, "tf32": 2.0 ** -11, "fp8": 2.0 ** -4}


@pytest.mark.parametrize("fmt", list(LOW))
@pytest.mark.parametrize("n", [8, 64, 127, 130, 257])
def test_matmul_low_exact_on_integers(mpps, fmt, n):
    """Small integers are exact in every format and their products sum exactly in FP32:
    the tensor-core path must reproduce A B bit for bit (checks operand layout, swizzle,
    descriptors, K/M/N tails and the scaling round trip)."""
    rng = np.random.default_rng(100 + n)
    lim = 4 if fmt == "fp8" else 8
    A = rng.integers(-lim, lim + 1, size=(2, n, n)).astype(np.float64)
    B = rng.integers(-lim, lim + 1, size=(2, n, n)).astype(np.float64)
    A[:, 0, 0] = lim; B[:, 0, 0] = lim     # pin the scale exponents
    C = host(mpps.matmul(dev(A), dev(B), fmt))
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("fmt", list(LOW))
@pytest.mark.parametrize("n", [64, 257])
def test_matmul_low_error_bound(mpps, fmt, n):
    rng = np.random.default_rng(200 + n)
    A = rng.standard_normal((1, n, n)); B = rng.standard_normal((1, n, n))
    C = host(mpps.matmul(dev(A), dev(B), fmt))[0]
    exact = A[0] @ B[0]
    absprod = np.abs(A[0]) @ np.abs(B[0])
    uf = LOW[fmt]
    # rounding of both operands (2 u_F), FP32 accumulation (n 2^-24); FP8 also loses
    # entries below its subnormal range relative to the per-matrix scale
    k = 3.0 if fmt != "fp8" else 4.0
    err = np.linalg.norm(C - exact)
    assert err <= k * (uf + n * 2.0 ** -24) * np.linalg.norm(absprod)


# ------------------------------------------------------------------------------------
# PS evaluation
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("m", [1, 2, 5, 16, 30])
def test_ps_eval_fixed_vs_oracle(mpps, n, m):
    A = inputs.gaussian_matrix(n, seed=1000 + n + m, norm1=1.0)
    coef = mpps.taylor_exp_coeffs(m)
    P = host(mpps.ps_eval(coef, dev(A), policy=mpps.FIXED))
    ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(m), A)
    assert oracle.rel_err_1norm(P, ph, pl) <= 50 * n * U


@pytest.mark.parametrize("n", [17, 64, 130, 257])
@pytest.mark.parametrize("norm", [0.05, 0.5, 1.0])
def test_ps_eval_mixed_vs_fixed(mpps, n, norm):
    m = 30
    A = inputs.gaussian_matrix(n, seed=2000 + n, norm1=norm)
    coef = mpps.taylor_exp_coeffs(m)
    ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(m), A)
    Pf = host(mpps.ps_eval(coef, dev(A), policy=mpps.FIXED))
    ef = oracle.rel_err_1norm(Pf, ph, pl)
    for pol in (mpps.PAPER, mpps.NS):
        Pm, rep = mpps.ps_eval(coef, dev(A), policy=pol, report=True)
        em = oracle.rel_err_1norm(host(Pm), ph, pl)
        assert em <= 50 * n * U
        assert em <= 2 * ef + FLOOR, (pol.mode, em, ef, rep[0]["fmt"])


@pytest.mark.parametrize("n", [64, 130, 257])
@pytest.mark.parametrize("graded", [False, True])
def test_ps_eval_fp8_steps_row_column_scaled(mpps, n, graded):
    # A loose target lets the planner put the high-order Horner steps in FP8; those products
    # scale each row of P_i and each column of Y by its own power of two (and every 32 entries
    # along K by a block scale).  A diagonally
    # similar matrix D G D^-1 (D spanning 2^12) gives rows and columns of very different
    # magnitude.  The normwise result must stay within the target's bound.
    m, tol = 30, 2.0 ** -30
    A = inputs.gaussian_matrix(n, seed=7100 + n, norm1=0.5)
    if graded:
        d = 2.0 ** np.round(np.linspace(0.0, 12.0, n))
        A = (d[:, None] * A) / d[None, :]
    coef = mpps.taylor_exp_coeffs(m)
    ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(m), A)
    pol = mpps.Policy(mode=mpps.MIXED_NS, tol=tol, formats=["fp64", "fp8"])
    P, rep = mpps.ps_eval(coef, dev(A), policy=pol, report=True)
    assert "fp8" in rep[0]["fmt"], rep[0]["fmt"]
    err = oracle.rel_err_1norm(host(P), ph, pl)
    assert err <= 50 * n * tol, (err, rep[0]["fmt"])


def _var_s_expected(coefq, X, m, s_cap):
    """The oracle's variable-s choice from double-double norms, and the smallest relative
    margin of the growth tests it made (a decision closer than that to the threshold could
    flip under the library's own norm rounding)."""
    s0 = oracle.ceil_sqrt(m)
    nx = oracle.norm1(X)
    b0, ys = [], []
    for s in range(s0, s_cap + 1):
        nb, ny = oracle.block_norms_dd(coefq, X, s)
        b0.append(nb[0]); ys.append(ny)
    got = min(oracle.choose_s(m, nx, b0, ys), s_cap)
    margin = min(abs(ys[k] - b0[k] * nx ** (s0 + k)) / ys[k] for k in range(got - s0 + 1 if got < s_cap else got - s0))
    return got, margin


@pytest.mark.parametrize("k", [0, 8])
def test_ps_eval_variable_s(mpps, k):
    """The variable-s branch of Algorithm 3.1: for X = -0.9 I + small noise ||B_0|| < 1, so
    ||Y|| > ||B_0|| ||X||^s and s grows; the chosen s matches the oracle's rule on
    double-double norms and the result keeps the fixed-FP64 accuracy.  A matrix with
    ||B_0|| >= 1 keeps s = ceil(sqrt(m)) and gives the same bits as without the branch."""
    n, m = 64, 30
    rng = np.random.default_rng(55)
    X = -0.9 * np.eye(n) + 0.02 * rng.standard_normal((n, n)) / np.sqrt(n)
    coefq = oracle.taylor_exp_rational(m)
    coef = mpps.taylor_exp_coeffs(m)
    pol = mpps.Policy(mode=mpps.MIXED_NS, variable_s=True, f64_slices=k)
    P, rep = mpps.ps_eval(coef, dev(X), policy=pol, report=True)
    s_cap = min(m, 32, 2 * oracle.ceil_sqrt(m))
    want, margin = _var_s_expected(coefq, X, m, s_cap)
    assert margin > 1e-6
    assert want > oracle.ceil_sqrt(m)
    assert rep[0]["s"] == want, (rep[0]["s"], want)
    ph, pl, _ = oracle.ps_dd(coefq, X)
    assert oracle.rel_err_1norm(host(P), ph, pl) <= 50 * n * U
    # expm takes the branch too; with ||X||_1 < 1 (sigma = 0) and this X the rule would grow
    # s past the library's cap of 2 ceil(sqrt(m)) = 12
    X2 = -0.85 * np.eye(n) + 0.01 * rng.standard_normal((n, n)) / np.sqrt(n)
    assert oracle.sigma_for(X2) == 0
    want2, margin2 = _var_s_expected(coefq, X2, m, s_cap)
    assert margin2 > 1e-6 and want2 == s_cap
    E, erep = mpps.expm(dev(X2), m=m, policy=pol, report=True)
    assert erep[0]["s"] == want2
    eh, el = oracle.expm_ss_dd(X2, m, 0)
    assert oracle.rel_err_1norm(host(E), eh, el) <= 50 * n * U
    # no growth for a Gaussian matrix: identical to the fixed-s evaluation
    G = inputs.gaussian_matrix(n, seed=56, norm1=0.5)
    P1, r1 = mpps.ps_eval(coef, dev(G), policy=pol, report=True)
    P0 = mpps.ps_eval(coef, dev(G), policy=mpps.Policy(mode=mpps.MIXED_NS, f64_slices=k))
    assert r1[0]["s"] == oracle.ceil_sqrt(m)
    assert np.array_equal(host(P1), host(P0))


def test_ps_eval_general_coefficients(mpps):
    n = 96
    A = inputs.gaussian_matrix(n, seed=5, norm1=2.0)
    for coefs_q, coefs_d in [(oracle.pade_exp_num_rational(13), mpps.pade_exp_num_coeffs(13)),
                             (oracle.pade_exp_den_rational(13), mpps.pade_exp_den_coeffs(13)),
                             (oracle.cos_taylor_rational(16), mpps.cos_taylor_coeffs(16))]:
        ph, pl, _ = oracle.ps_dd(coefs_q, A)
        for pol in (mpps.FIXED, mpps.PAPER):
            P = host(mpps.ps_eval(coefs_d, dev(A), policy=pol))
            assert oracle.rel_err_1norm(P, ph, pl) <= 50 * n * U


def test_ps_eval_block_sizes_and_nilpotent(mpps):
    n, m = 40, 20
    coefq = oracle.taylor_exp_rational(m)
    coef = mpps.taylor_exp_coeffs(m)
    A = inputs.gaussian_matrix(n, seed=9, norm1=1.5)
    ph, pl, _ = oracle.ps_dd(coefq, A)
    for s in (1, 2, 3, 7, 20):
        P = host(mpps.ps_eval(coef, dev(A), policy=mpps.Policy(mode=mpps.FIXED_FP64, s=s)))
        assert oracle.rel_err_1norm(P, ph, pl) <= 50 * n * U, s
    N = inputs.strictly_upper(n, seed=3, scale=1.0)
    nh, nl, _ = oracle.ps_dd(coefq, N)
    for pol in (mpps.FIXED, mpps.PAPER):
        P = host(mpps.ps_eval(coef, dev(N), policy=pol))
        assert oracle.rel_err_1norm(P, nh, nl) <= 50 * n * U


def test_ps_eval_batch_and_host_pointers(mpps):
    n, m = 33, 16
    A = inputs.gaussian_batch(3, n, seed=11, norm1=[0.2, 1.0, 3.0])
    coef = mpps.taylor_exp_coeffs(m)
    Pd = host(mpps.ps_eval(coef, dev(A), policy=mpps.NS))
    Ph = mpps.ps_eval(coef, A, policy=mpps.NS)          # numpy in, numpy out
    assert np.array_equal(Pd, Ph)
    for b in range(3):
        ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(m), A[b])
        assert oracle.rel_err_1norm(Pd[b], ph, pl) <= 50 * n * U


def test_degenerate_cases(mpps):
    A = inputs.gaussian_matrix(5, seed=1, norm1=1.0)
    P = host(mpps.ps_eval([2.5], dev(A)))
    assert np.array_equal(P, 2.5 * np.eye(5))
    P1 = host(mpps.ps_eval([1.0], dev(np.array([[3.0]]))))
    assert P1[0, 0] == 1.0
    one = host(mpps.ps_eval(mpps.taylor_exp_coeffs(12), dev(np.array([[0.5]])), policy=mpps.FIXED))
    exact = float(sum(oracle.Fraction(1, 2 ** k) * c for k, c in enumerate(oracle.taylor_exp_rational(12))))
    assert abs(one[0, 0] - exact) <= 4 * U * exact
    empty = torch.empty((0, 4, 4), dtype=torch.float64, device="cuda:0")
    assert mpps.ps_eval([1.0, 1.0], empty).shape == (0, 4, 4)
    with pytest.raises(mpps.MppsError):
        mpps.ps_eval([1.0] * 2000, dev(A))      # r beyond the supported range


# ------------------------------------------------------------------------------------
# scaling and squaring
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [16, 130])
@pytest.mark.parametrize("norm", [0.5, 4.0, 32.0])
def test_expm_vs_oracle(mpps, n, norm):
    A = inputs.gaussian_matrix(n, seed=3000 + n, norm1=norm)
    sg = oracle.sigma_for(A)
    eh, el = oracle.expm_ss_dd(A, 30, sg)
    Ef, rf = mpps.expm(dev(A), m=30, policy=mpps.FIXED, report=True)
    ef = oracle.rel_err_1norm(host(Ef), eh, el)
    assert rf[0]["sigma"] == sg
    # squaring amplifies the polynomial's error by about 2^sigma (Section 3.2)
    tol = 50 * n * U * max(1, 2 ** sg)
    assert ef <= tol
    for pol in (mpps.PAPER, mpps.NS):
        Em = host(mpps.expm(dev(A), m=30, policy=pol))
        em = oracle.rel_err_1norm(Em, eh, el)
        assert em <= tol and em <= 2 * ef + FLOOR, (pol.mode, em, ef)


def test_expm_batch_mixed_sigma(mpps):
    n = 24
    A = inputs.gaussian_batch(4, n, seed=12, norm1=[0.3, 2.0, 9.0, 40.0])
    E, reps = mpps.expm(dev(A), m=30, policy=mpps.NS, report=True)
    E = host(E)
    for b in range(4):
        sg = oracle.sigma_for(A[b])
        assert reps[b]["sigma"] == sg
        eh, el = oracle.expm_ss_dd(A[b], 30, sg)
        assert oracle.rel_err_1norm(E[b], eh, el) <= 50 * n * U * max(1, 2 ** sg)


def test_expm_rotation_and_group_property(mpps):
    theta = 2.5
    R = np.array([[0.0, -theta], [theta, 0.0]])
    E = host(mpps.expm(dev(R), policy=mpps.NS))
    ref = np.array([[np.cos(theta), -np.sin(theta)], [np.sin(theta), np.cos(theta)]])
    assert np.max(np.abs(E - ref)) < 1e-15
    A = inputs.gaussian_matrix(50, seed=4, norm1=3.0)
    Ep = host(mpps.expm(dev(A), policy=mpps.NS)); Em = host(mpps.expm(dev(-A), policy=mpps.NS))
    assert np.max(np.abs(Ep @ Em - np.eye(50))) < 1e-12


# ------------------------------------------------------------------------------------
# adjoint
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(1, 3), (6, 4), (16, 8), (33, 18), (40, 13)])
def test_adjoint_vs_oracle(mpps, n, m):
    rng = np.random.default_rng(n * 100 + m)
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    G = rng.standard_normal((n, n))
    c = oracle.taylor_exp_rational(m)
    gh, gl = oracle.adjoint_dd(c, A, G)
    g = host(mpps.ps_eval_adjoint(mpps.taylor_exp_coeffs(m), dev(A), dev(G)))
    assert oracle.norm1(g - gh - gl) / oracle.norm1(gh) <= 100 * n * U


def test_autograd_function(mpps):
    n, m, batch = 12, 18, 3
    rng = np.random.default_rng(5)
    A = torch.tensor(rng.standard_normal((batch, n, n)) / np.sqrt(n), device="cuda:0",
                     dtype=torch.float64, requires_grad=True)
    coef = mpps.taylor_exp_coeffs(m)
    P = mpps.poly(A, coef, mpps.FIXED)
    G = torch.randn(P.shape, generator=torch.Generator(device="cuda:0").manual_seed(6),
                    device="cuda:0", dtype=P.dtype)
    (P * G).sum().backward()
    for b in range(batch):
        gh, gl = oracle.adjoint_dd(oracle.taylor_exp_rational(m), A[b].detach().cpu().numpy(),
                                   G[b].cpu().numpy())
        got = A.grad[b].cpu().numpy()
        assert oracle.norm1(got - gh - gl) / oracle.norm1(gh) <= 100 * n * U


# ------------------------------------------------------------------------------------
# full-size configuration (n = 1024, m = 30, s = 6): sampled columns against the oracle
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("norm", [0.5, 4.0, 32.0])
def test_expm_n1024_sampled_columns(mpps, norm):
    n = 1024
    A = inputs.gaussian_matrix(n, seed=2, norm1=norm)
    sg = oracle.sigma_for(A)
    X = np.ldexp(A, -sg)
    cols = [0, 511, 1023]
    V = np.zeros((n, len(cols)))
    for t, j in enumerate(cols):
        V[j, t] = 1.0
    wh, wl = oracle.ps_apply_dd(oracle.taylor_exp_rational(30), X, V, reps=2 ** sg)
    ref_norm = np.abs(wh).sum(axis=0)
    # the benchmarked mixed policy: emulated working precision, FP64/3xBF16/TF32/BF16 ladder
    c2 = dataclasses.replace(mpps.NS_E, formats=("fp64", "bf16x3", "tf32", "bf16"))
    errs = {}
    for name, pol in (("fixed", mpps.FIXED), ("ns", mpps.NS), ("paper", mpps.PAPER),
                      ("fixed_e", mpps.FIXED_E), ("ns_e", mpps.NS_E), ("c2", c2)):
        E = host(mpps.expm(dev(A), m=30, policy=pol))
        err = np.abs(E[:, cols] - wh - wl).sum(axis=0) / ref_norm
        assert np.all(err <= 50 * n * U * max(1, 2 ** sg)), (name, err)
        errs[name] = err
    for name in ("ns", "paper", "ns_e", "c2"):
        assert np.all(errs[name] <= 2 * errs["fixed"] + FLOOR), (name, errs[name], errs["fixed"])


# ------------------------------------------------------------------------------------
# FP64 products emulated by exact bf16 slices on the tensor cores
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [8, 64, 130, 257, 1024, 1100])
def test_matmul_f64e_exact_on_small_integers(mpps, n):
    """Integers below 64 in magnitude are one exact slice; their products sum exactly.  At
    n = 1024 and 1100 the tiles are fewer than two per SM, and CTAs split the K range of
    tiles (up to three pieces per tile) and add the pieces' integer sums."""
    rng = np.random.default_rng(300 + n)
    A = rng.integers(-63, 64, size=(2, n, n)).astype(np.float64)
    B = rng.integers(-63, 64, size=(2, n, n)).astype(np.float64)
    for k in (1, 8):
        C = host(mpps.matmul(dev(A), dev(B), f"f64e{k}"))
        assert np.array_equal(C, A @ B), k


@pytest.mark.parametrize("n", [1, 3, 17, 64, 130, 257, 1100])
def test_matmul_f64e_vs_oracle(mpps, n):
    """8 slices: FP64-level error (n up to several 128 x 64 tiles with ragged tails)."""
    rng = np.random.default_rng(400 + n)
    A = rng.standard_normal((1, n, n)); B = rng.standard_normal((1, n, n))
    A[0, 0, :] *= 1e-9                      # a row far below the others: row scaling matters
    C = host(mpps.matmul(dev(A), dev(B), "f64e8"))[0]
    ch, cl = oracle.matmul_dd(A[0], None, B[0], None)
    err = np.abs(C - ch - cl)
    absprod = np.abs(A[0]) @ np.abs(B[0])
    # slices keep 54 bits below each row / column maximum; bound by those maxima
    rmax = np.abs(A[0]).max(axis=1)[:, None]; cmax = np.abs(B[0]).max(axis=0)[None, :]
    bound = 8 * U * (rmax * np.abs(B[0]).sum(axis=0)[None, :] + cmax * np.abs(A[0]).sum(axis=1)[:, None])
    assert np.all(err <= bound + 1e-300)
    assert np.linalg.norm(err) <= 4 * n * U * np.linalg.norm(absprod)


@pytest.mark.parametrize("shift", [(-990, -20), (990, 20), (-600, 580)])
def test_matmul_f64e_extreme_magnitudes(mpps, shift):
    """Rows and columns far from 1 (down to 2^-1010 products): the slicing works from the
    exponent fields and the result scale 2^(eA+eB) leaves the fast power-of-two path when it
    would leave the normal range; against the oracle product scaled by the same powers."""
    n = 130
    rng = np.random.default_rng(77)
    A0 = rng.standard_normal((n, n)); B0 = rng.standard_normal((n, n))
    A = np.ldexp(A0, shift[0]); B = np.ldexp(B0, shift[1])
    C = host(mpps.matmul(dev(A[None]), dev(B[None]), "f64e8"))[0]
    ch, cl = oracle.matmul_dd(A0, None, B0, None)
    ref = np.ldexp(ch, shift[0] + shift[1]); refl = np.ldexp(cl, shift[0] + shift[1])
    rmax = np.abs(A0).max(axis=1)[:, None]; cmax = np.abs(B0).max(axis=0)[None, :]
    bound = 8 * U * (rmax * np.abs(B0).sum(axis=0)[None, :] + cmax * np.abs(A0).sum(axis=1)[:, None])
    err = np.abs(np.ldexp(C, -(shift[0] + shift[1])) - np.ldexp(ref, -(shift[0] + shift[1]))
                 - np.ldexp(refl, -(shift[0] + shift[1])))
    assert np.all(np.isfinite(C))
    assert np.all(err <= bound)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("n", [130, 1024, 4200])
def test_matmul_f64e_nonfinite_entries(mpps, bad, n):
    """A non-finite entry of A poisons its row of the product and one of B its column, as in
    the FP64 product (the emulated path writes NaN there, where FP64 may give +-inf); every
    other entry keeps the emulated product's accuracy.  n = 4200 also takes the path that
    flushes the integer accumulator to FP64."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((n, n)); B = rng.standard_normal((n, n))
    ia, ka = 3, n // 2
    kb, jb = n - 2, n // 3
    A[ia, ka] = bad; B[kb, jb] = bad
    C = host(mpps.matmul(dev(A[None]), dev(B[None]), "f64e8"))[0]
    assert np.all(np.isnan(C[ia, :])) and np.all(np.isnan(C[:, jb]))
    rows = [0, n - 1, ia + 1]; cols = [0, n - 1, jb + 1]
    assert np.all(np.isfinite(C[np.ix_(rows, cols)]))
    Ac = np.where(np.isfinite(A), A, 0.0); Bc = np.where(np.isfinite(B), B, 0.0)
    ref = Ac[rows, :] @ Bc[:, cols]
    bound = 1e-12 * (np.abs(Ac[rows, :]) @ np.abs(Bc[:, cols]))
    # rows and columns without a non-finite entry (A's column ka and B's row kb hold finite
    # values elsewhere, so the sampled rows and columns are unaffected)
    assert np.all(np.abs(C[np.ix_(rows, cols)] - ref) <= bound)


def test_expm_nonfinite_input_propagates(mpps):
    """A NaN entry makes every entry of exp(A) NaN on the FP64 pipe (the powers spread it);
    the emulated path must not drop it: its slicing records the row and column and the
    product writes NaN there, so the powers spread it the same way."""
    n = 96
    A = inputs.gaussian_matrix(n, seed=5, norm1=2.0)
    A[7, 40] = np.nan
    for pol in (mpps.FIXED, mpps.FIXED_E, mpps.NS_E):
        E = host(mpps.expm(dev(A), m=18, policy=pol))
        assert np.all(np.isnan(E)), pol


def test_matmul_f64e_multichunk_sampled(mpps):
    """n = 2100 crosses the 2048-long exact-accumulation chunk (the exact diagonals are
    drained into the 64-bit integer accumulator twice); 8 sampled columns against an
    extended-precision (long double) dot product."""
    n = 2100
    rng = np.random.default_rng(2100)
    A = rng.standard_normal((n, n)); B = rng.standard_normal((n, n))
    A[5, :] *= 1e-7
    C = host(mpps.matmul(dev(A[None]), dev(B[None]), "f64e8"))[0]
    cols = rng.choice(n, size=8, replace=False)
    ref = (A.astype(np.longdouble) @ B[:, cols].astype(np.longdouble))
    err = np.abs(C[:, cols].astype(np.longdouble) - ref).astype(np.float64)
    rmax = np.abs(A).max(axis=1)[:, None]; cmax = np.abs(B[:, cols]).max(axis=0)[None, :]
    bound = 8 * U * (rmax * np.abs(B[:, cols]).sum(axis=0)[None, :]
                     + cmax * np.abs(A).sum(axis=1)[:, None])
    assert np.all(err <= bound)


def test_matmul_f64e_error_falls_with_slices(mpps):
    n = 200
    rng = np.random.default_rng(5)
    A = rng.standard_normal((1, n, n)); B = rng.standard_normal((1, n, n))
    exact = A[0] @ B[0]
    ch, cl = oracle.matmul_dd(A[0], None, B[0], None)
    scale = np.linalg.norm(np.abs(A[0]) @ np.abs(B[0]))
    prev = None
    for k in range(1, 10):
        C = host(mpps.matmul(dev(A), dev(B), f"f64e{k}"))[0]
        err = np.linalg.norm(C - ch - cl) / scale
        assert err <= (2.0 ** (2 - 7 * k) if k <= 8 else 2.0 ** -55), (k, err)
        if prev is not None and k < 9:
            assert err < prev
        prev = err


def test_f64e9_at_most_fp64_error_on_prescribed_eigenvalues(mpps):
    """Pade[13/13] numerator of a Q diag(lambda) Q^T matrix, lambda in [-8, 8] (the n = 2048
    workload's input class, smaller): with the pairs of order 8 (F64E(9)) the all-emulated
    evaluation is within 2x of the FP64-pipe evaluation's error against the oracle."""
    import dataclasses
    n = 384
    A = inputs.prescribed_eigen_matrix(n, seed=5)
    rat = oracle.pade_exp_num_rational(13)
    ph, pl, _ = oracle.ps_dd(rat, A)
    coef = mpps.pade_exp_num_coeffs(13)
    ef = oracle.rel_err_1norm(host(mpps.ps_eval(coef, dev(A), policy=mpps.FIXED)), ph, pl)
    e9 = oracle.rel_err_1norm(host(mpps.ps_eval(coef, dev(A), policy=dataclasses.replace(
        mpps.FIXED_E, f64_slices=9))), ph, pl)
    assert e9 <= 2 * ef, (e9, ef)


@pytest.mark.parametrize("n", [17, 130, 257])
def test_ps_eval_emulated_vs_oracle(mpps, n):
    m = 30
    A = inputs.gaussian_matrix(n, seed=5000 + n, norm1=0.8)
    coef = mpps.taylor_exp_coeffs(m)
    ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(m), A)
    Pf = host(mpps.ps_eval(coef, dev(A), policy=mpps.FIXED))
    ef = oracle.rel_err_1norm(Pf, ph, pl)
    for pol in (mpps.FIXED_E, mpps.PAPER_E, mpps.NS_E):
        P, rep = mpps.ps_eval(coef, dev(A), policy=pol, report=True)
        e = oracle.rel_err_1norm(host(P), ph, pl)
        assert e <= 50 * n * U, (pol.mode, e, rep[0]["fmt"])
        assert e <= 2 * ef + FLOOR, (pol.mode, e, ef, rep[0]["fmt"])


@pytest.mark.parametrize("norm", [0.5, 4.0, 32.0])
def test_expm_emulated_vs_oracle(mpps, norm):
    n = 130
    A = inputs.gaussian_matrix(n, seed=6000, norm1=norm)
    sg = oracle.sigma_for(A)
    eh, el = oracle.expm_ss_dd(A, 30, sg)
    ef = oracle.rel_err_1norm(host(mpps.expm(dev(A), policy=mpps.FIXED)), eh, el)
    for pol in (mpps.FIXED_E, mpps.NS_E, mpps.PAPER_E):
        E = host(mpps.expm(dev(A), policy=pol))
        e = oracle.rel_err_1norm(E, eh, el)
        assert e <= 50 * n * U * max(1, 2 ** sg) and e <= 2 * ef + FLOOR, (pol.mode, e, ef)


def test_expm_emulated_batch_mixed_sigma(mpps):
    n = 40
    A = inputs.gaussian_batch(3, n, seed=13, norm1=[0.3, 5.0, 40.0])
    E, reps = mpps.expm(dev(A), policy=mpps.NS_E, report=True)
    E = host(E)
    for b in range(3):
        sg = oracle.sigma_for(A[b])
        eh, el = oracle.expm_ss_dd(A[b], 30, sg)
        assert oracle.rel_err_1norm(E[b], eh, el) <= 50 * n * U * max(1, 2 ** sg)


def test_expm_emulated_batch_split_k_squarings(mpps):
    """Two 1152 x 1152 matrices (162 tiles each, more than one wave on the SMs): the emulated
    powers and Horner products split K between CTAs, and so do the squarings of both
    matrices (sigma 3 and 1), whose last two run on one matrix through the index list.
    Sampled columns against the oracle's Horner applied to unit vectors."""
    n = 1152
    A = inputs.gaussian_batch(2, n, seed=31, norm1=[6.0, 1.5])
    E = host(mpps.expm(dev(A), m=30, policy=mpps.NS_E))
    cols = [0, 577, n - 1]
    V = np.zeros((n, len(cols)))
    for t, j in enumerate(cols):
        V[j, t] = 1.0
    for b in range(2):
        sg = oracle.sigma_for(A[b])
        wh, wl = oracle.ps_apply_dd(oracle.taylor_exp_rational(30), np.ldexp(A[b], -sg), V,
                                    reps=2 ** sg)
        err = np.abs(E[b][:, cols] - wh - wl).sum(axis=0) / np.abs(wh).sum(axis=0)
        assert np.all(err <= 50 * n * U * max(1, 2 ** sg)), (b, sg, err)


def test_autotune_picks_a_schedule_and_keeps_its_output(mpps):
    """With tuning on, the first product of a shape times both schedules and records the
    fastest; the output is that schedule's, and the next call (from the table) gives the
    same bits.  Small-integer inputs make every schedule exact (A B in FP64)."""
    rng = np.random.default_rng(12)
    A = rng.integers(-63, 64, size=(2, 1024, 1024)).astype(np.float64)
    B = rng.integers(-63, 64, size=(2, 1024, 1024)).astype(np.float64)
    A2 = rng.integers(-63, 64, size=(1, 512, 512)).astype(np.float64)
    B2 = rng.integers(-63, 64, size=(1, 512, 512)).astype(np.float64)
    mpps.autotune_clear()
    mpps.autotune(True)
    try:
        C1 = host(mpps.matmul(dev(A), dev(B), "f64e8"))
        C2 = host(mpps.matmul(dev(A), dev(B), "f64e8"))
        L1 = host(mpps.matmul(dev(A2), dev(B2), "bf16"))
        L2 = host(mpps.matmul(dev(A2), dev(B2), "bf16"))
        ent = {(e["kind"], e["n"], e["batch"], e["variant"]): e for e in mpps.autotune_entries()}
    finally:
        mpps.autotune(False)
        mpps.autotune_clear()
    exact = np.einsum("bij,bjk->bik", A, B)
    assert np.array_equal(C1, exact) and np.array_equal(C2, C1)
    assert np.array_equal(L1[0], A2[0] @ B2[0]) and np.array_equal(L2, L1)
    e = ent[("f64e_split", 1024, 2, 8)]
    assert e["choice"] in (0, 1) and e["ms"][0] > 0 and e["ms"][1] > 0
    t = ent[("tc_width", 512, 1, 3)]
    assert t["choice"] in (0, 1) and t["ms"][0] > 0 and t["ms"][1] > 0


# ------------------------------------------------------------------------------------
# failure path of the bounded waits (no fault: a wait that nothing completes gives up)
# ------------------------------------------------------------------------------------
def test_bounded_wait_reports_timeout_and_context_survives(mpps):
    st = torch.cuda.current_stream().cuda_stream
    rc = mpps.lib().mpps_selftest_bounded_wait(20000, st)      # 20 ms limit
    assert rc == 4                                            # MPPS_ETIMEOUT
    assert b"bounded wait" in mpps.lib().mpps_last_error()
    # the context is still usable: a normal evaluation succeeds afterwards
    A = inputs.gaussian_matrix(32, seed=77, norm1=1.0)
    P = host(mpps.ps_eval(mpps.taylor_exp_coeffs(12), dev(A), policy=mpps.NS_E))
    ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(12), A)
    assert oracle.rel_err_1norm(P, ph, pl) <= 50 * 32 * U


def test_workspace_release_between_calls(mpps):
    """The cached workspace pool can be trimmed between calls; results are unchanged."""
    A = inputs.gaussian_matrix(96, seed=96, norm1=3.0)
    E1 = host(mpps.expm(dev(A), policy=mpps.NS_E))
    mpps.release_workspace()
    E2 = host(mpps.expm(dev(A), policy=mpps.NS_E))
    assert np.array_equal(E1, E2)


def test_sigma_matches_oracle_at_power_of_two_norms(mpps):
    """||A||_1 rescaled to exactly 4 or 32 (no margin): the squaring count the GPU picks must
    equal the oracle's sequential-sum rule even when rounding puts the norm a hair above."""
    n = 200
    for seed in range(6):
        A = np.random.default_rng(seed).standard_normal((n, n))
        for target in (4.0, 32.0):
            B = A * (target / np.abs(A).sum(axis=0).max())
            _, rep = mpps.expm(dev(B), policy=mpps.NS_E, report=True)
            assert rep[0]["sigma"] == oracle.sigma_for(B), (seed, target)


@pytest.mark.parametrize("n,m", [(16, 8), (33, 18), (64, 13)])
def test_adjoint_emulated_vs_oracle(mpps, n, m):
    rng = np.random.default_rng(n * 7 + m)
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    G = rng.standard_normal((n, n))
    gh, gl = oracle.adjoint_dd(oracle.taylor_exp_rational(m), A, G)
    g = host(mpps.ps_eval_adjoint(mpps.taylor_exp_coeffs(m), dev(A), dev(G), policy=mpps.FIXED_E))
    assert oracle.norm1(g - gh - gl) / oracle.norm1(gh) <= 100 * n * U


@pytest.mark.parametrize("n,m,norms", [(16, 30, (0.5, 3.0, 7.0)), (33, 18, (5.0, 0.2)),
                                         (64, 12, (2.5,))])
@pytest.mark.parametrize("k", [0, 8])
def test_expm_adjoint_vs_oracle(mpps, n, m, norms, k):
    """Reverse mode through scaling and squaring (one sigma per matrix, a batch of mixed
    sigma) against the oracle's chain rule in double-double; k = 0: FP64 pipe, k = 8:
    emulated products."""
    batch = len(norms)
    A = inputs.gaussian_batch(batch, n, seed=900 + n, norm1=list(norms))
    rng = np.random.default_rng(n + m)
    G = rng.standard_normal((batch, n, n))
    g = host(mpps.expm_adjoint(dev(A), dev(G), m=m,
                               policy=mpps.Policy(mode=mpps.FIXED_FP64, f64_slices=k)))
    for b in range(batch):
        sg = oracle.sigma_for(A[b])
        gh, gl = oracle.expm_ss_adjoint_dd(A[b], G[b], m, sg)
        err = oracle.norm1(g[b] - gh - gl) / oracle.norm1(gh)
        assert err <= 100 * n * U * max(1, 2 ** sg), (b, sg, err)


def test_expm_autograd_central_differences(mpps):
    """torch autograd through ExpmFn: the backward pass equals expm_adjoint and matches FP64
    central differences of the forward expm."""
    n = 24
    A0 = inputs.gaussian_matrix(n, seed=77, norm1=3.0)
    A = torch.tensor(A0, device="cuda:0", requires_grad=True)
    G = torch.randn((n, n), generator=torch.Generator(device="cuda:0").manual_seed(8),
                    device="cuda:0", dtype=torch.float64)
    E = mpps.expm_differentiable(A)
    (E * G).sum().backward()
    grad = A.grad.cpu().numpy()
    direct = host(mpps.expm_adjoint(dev(A0[None]), G[None].contiguous()))[0]
    assert np.array_equal(grad, direct)
    h = 1e-6
    Gn = G.cpu().numpy()
    for (i, j) in [(0, 0), (3, 17), (20, 5)]:
        D = np.zeros((n, n)); D[i, j] = h
        fp = host(mpps.expm(dev(A0 + D)))
        fm = host(mpps.expm(dev(A0 - D)))
        fd = float(np.sum(Gn * (fp - fm))) / (2 * h)
        assert abs(fd - grad[i, j]) <= 1e-7 * max(1.0, abs(grad[i, j])), (i, j, fd, grad[i, j])


@pytest.mark.parametrize("n,norms", [(16, (0.5, 3.0)), (100, (20.0, 60.0)), (257, (4.0,))])
@pytest.mark.parametrize("pol", ["fixed", "ns_e"])
def test_expm_pade13_vs_oracle(mpps, n, norms, pol):
    """exp by the [13/13] Pade approximant (scaling to theta_13, numerator and denominator
    from one power chain, LU solve, squarings) against the oracle's exp (Taylor degree 30
    with its own scaling, exact to double-double level): the same 50 n u 2^sigma bound as
    the Taylor path (an FP64 numpy model of the algorithm stays below 0.25 n u 2^sigma on
    these inputs)."""
    policy = {"fixed": mpps.FIXED, "ns_e": mpps.NS_E}[pol]
    batch = len(norms)
    A = inputs.gaussian_batch(batch, n, seed=1300 + n, norm1=list(norms))
    E = host(mpps.expm_pade(dev(A), policy=policy))
    theta = 5.371920351148152
    for b in range(batch):
        nrm = np.abs(A[b]).sum(axis=0).max()
        sg = 0
        while nrm * 2.0 ** -sg > theta:
            sg += 1
        eh, el = oracle.expm_ss_dd(A[b], 30, oracle.sigma_for(A[b]))
        err = oracle.rel_err_1norm(E[b], eh, el)
        assert err <= 50 * n * U * max(1, 2 ** sg), (b, sg, err)


@pytest.mark.parametrize("m", [50, 64])
@pytest.mark.parametrize("k", [0, 8])
def test_adjoint_recompute_same_bits(mpps, m, k):
    """Recompute mode keeps every ceil(sqrt(r))-th Horner iterate (and the top one) and
    recomputes the others a segment at a time with the same products: the gradient is the
    stored mode's, bit for bit.  m = 50 (s = 8, r = 6) and m = 64 (r = 8, s | m, top
    iterate r - 1), batch 2; also through scaling and squaring."""
    n = 64
    A = inputs.gaussian_batch(2, n, seed=m + k, norm1=[0.7, 3.0])
    G = np.random.default_rng(m).standard_normal((2, n, n))
    coef = mpps.taylor_exp_coeffs(m)
    keep = mpps.Policy(mode=mpps.FIXED_FP64, f64_slices=k)
    rec = mpps.Policy(mode=mpps.FIXED_FP64, f64_slices=k, adjoint_recompute=True)
    g0 = host(mpps.ps_eval_adjoint(coef, dev(A), dev(G), policy=keep))
    g1 = host(mpps.ps_eval_adjoint(coef, dev(A), dev(G), policy=rec))
    assert np.array_equal(g0, g1)
    gh, gl = oracle.adjoint_dd(oracle.taylor_exp_rational(m), A[0], G[0])
    assert oracle.norm1(g1[0] - gh - gl) / oracle.norm1(gh) <= 100 * n * U
    e0 = host(mpps.expm_adjoint(dev(A), dev(G), m=m, policy=keep))
    e1 = host(mpps.expm_adjoint(dev(A), dev(G), m=m, policy=rec))
    assert np.array_equal(e0, e1)


def test_adjoint_fp32_batch_config_shape(mpps):
    """Batch of FP32-stored 128 x 128 matrices, N(0,1)/sqrt(n) entries, Taylor exp m = 18,
    through the autograd Function with emulated products: the gradient agrees with the
    oracle (rel. err <= 1e-5) and with the block-triangular Frechet identity
    <grad, E> = <G, L_p(A, E)>, L_p(A, E) = p([[A, E], [0, A]])_12, evaluated on the GPU."""
    n, m, batch = 128, 18, 4
    rng = np.random.default_rng(4)
    A32 = torch.tensor(rng.standard_normal((batch, n, n)) / np.sqrt(n), dtype=torch.float32,
                       device="cuda:0", requires_grad=True)
    coef = mpps.taylor_exp_coeffs(m)
    P = mpps.poly(A32, coef, mpps.NS_E)
    assert P.dtype == torch.float32
    G = torch.randn(P.shape, generator=torch.Generator(device="cuda:0").manual_seed(5),
                    device="cuda:0", dtype=P.dtype)
    (P * G).sum().backward()
    grad = A32.grad.double().cpu().numpy()
    A64 = A32.detach().double().cpu().numpy()
    G64 = G.double().cpu().numpy()
    for b in range(2):
        gh, gl = oracle.adjoint_dd(oracle.taylor_exp_rational(m), A64[b], G64[b])
        ref = gh + gl
        assert oracle.norm1(grad[b] - ref) / oracle.norm1(ref) <= 1e-5
    E = rng.standard_normal((n, n))
    M = np.zeros((2 * n, 2 * n)); M[:n, :n] = A64[0]; M[n:, n:] = A64[0]; M[:n, n:] = E
    L = host(mpps.ps_eval(coef, dev(M), policy=mpps.FIXED_E))[:n, n:]
    lhs = float(np.sum(grad[0] * E)); rhs = float(np.sum(G64[0] * L))
    # the gradient is stored in FP32: each entry carries a rounding error of at most 2^-24
    # of itself, which the sum over n^2 products need not cancel; the FP64-level error of
    # the evaluation itself is far below that
    assert abs(lhs - rhs) <= 2.0 ** -24 * float(np.sum(np.abs(grad[0] * E))) + 1e-10 * abs(rhs)


# ------------------------------------------------------------------------------------
# uneven batches (bucketed, zero-padded, one batched evaluation per bucket)
# ------------------------------------------------------------------------------------
def test_expm_grouped_uneven_vs_oracle(mpps):
    rng = np.random.default_rng(31)
    ns = [1, 5, 31, 32, 33, 47, 70, 64, 130, 8, 100, 33]
    ms = [12, 18, 24, 12, 18, 24, 12, 18, 24, 30, 18, 12]
    norms = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=len(ns)))
    mats = []
    for k, n in enumerate(ns):
        A = rng.standard_normal((n, n))
        A *= norms[k] / np.abs(A).sum(axis=0).max()
        mats.append(A)
    for pol in (mpps.NS_E, mpps.FIXED):
        outs, reps = mpps.expm_grouped([dev(A) for A in mats], ms, policy=pol, report=True)
        for A, m, E, R in zip(mats, ms, outs, reps):
            n = A.shape[0]
            sg = oracle.sigma_for(A)
            assert R["sigma"] == sg
            eh, el = oracle.expm_ss_dd(A, m, sg)
            err = oracle.rel_err_1norm(host(E), eh, el)
            # Taylor truncation at degree m on ||X||_1 <= 1 is below 1/(m+1)! * e
            trunc = np.e / float(oracle.math.factorial(m + 1)) * 2 ** sg
            assert err <= 50 * n * U * max(1, 2 ** sg) + trunc, (n, m, err)
