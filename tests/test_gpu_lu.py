"""GPU checks of the LU solve R = Q^-1 P (the q^-1 p solve of the Pade approximant,
Section 4.1): against the oracle's unblocked Gaussian elimination with partial pivoting on
sizes that span one to four 64 x 64 tiles with ragged edges, exactly on permuted diagonal
systems, by the residual at full sizes (n = 2048, and n = 6800 whose first panels exceed the
cluster's shared memory and are factored in place), singular systems, host pointers and an
aliased output."""
import numpy as np
import pytest

import oracle
from paper_2312_17396_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def policies(mpps):
    return {"fp64": mpps.FIXED, "f64e8": mpps.FIXED_E,
            "f64e9": mpps.Policy(mode=mpps.FIXED_FP64, f64_slices=9)}


def residual(Q, R, P, cols=None):
    """max over the columns of ||Q r - p||_inf / (||Q||_inf ||r||_inf): the normwise backward
    error of each computed column."""
    if cols is not None:
        R, P = R[:, cols], P[:, cols]
    res = np.abs(Q @ R - P).max(axis=0)
    return float((res / (np.abs(Q).sum(axis=1).max() * np.abs(R).max(axis=0))).max())


# Gaussian elimination with partial pivoting is backward stable with a growth factor that
# stays small on these inputs: a normwise backward error of 8 n u covers it with room, and
# the forward error is at most kappa_1(Q) times that.
@pytest.mark.parametrize("n", [1, 5, 63, 64, 65, 130, 200])
@pytest.mark.parametrize("pol", ["fp64", "f64e8", "f64e9"])
def test_lu_solve_vs_oracle(mpps, n, pol):
    rng = np.random.default_rng(4000 + n)
    Q = rng.standard_normal((2, n, n))
    P = rng.standard_normal((2, n, n))
    R = host(mpps.lu_solve(dev(Q), dev(P), policy=policies(mpps)[pol]))
    for b in range(2):
        Ro, piv, info = oracle.lu_solve(Q[b], P[b])
        assert info == 0
        kappa = np.linalg.cond(Q[b], 1)
        assert oracle.norm1(R[b] - Ro) <= 8 * n * kappa * U * oracle.norm1(Ro), (b, kappa)
        assert residual(Q[b], R[b], P[b]) <= 8 * n * U


@pytest.mark.parametrize("pol", ["fp64", "f64e8"])
def test_lu_solve_permuted_diagonal_exact(mpps, pol):
    # Q = Pi D (Pi a permutation across tiles, D powers of two): every pivot is the column's
    # only nonzero, the factors are exact, and R = D^-1 Pi^T P exactly for integer P
    n = 150
    rng = np.random.default_rng(5)
    perm = rng.permutation(n)
    d = 2.0 ** rng.integers(-3, 4, n)
    Q = np.zeros((n, n))
    Q[perm, np.arange(n)] = d
    P = rng.integers(-2 ** 20, 2 ** 20, (n, n)).astype(np.float64)
    expect = np.linalg.solve(Q, P)
    assert np.array_equal(expect, (P[perm, :].T / d).T)   # the exact solution, by hand
    R = host(mpps.lu_solve(dev(Q), dev(P), policy=policies(mpps)[pol]))
    assert np.array_equal(R, expect)


def test_lu_solve_singular(mpps):
    n = 70
    rng = np.random.default_rng(6)
    Q = rng.standard_normal((n, n))
    Q[:, 40] = 0.0     # a zero column stays exactly zero through every block update (equal
    for pol in (mpps.FIXED_E, mpps.FIXED):   # rows would not: blocked updates round apart)
        with pytest.raises(mpps.MppsError) as e:
            mpps.lu_solve(dev(Q), dev(np.eye(n)), policy=pol)
        assert e.value.status == 6 and "column 40" in str(e.value)
    Z = np.zeros((1, 3, 3))
    with pytest.raises(mpps.MppsError) as e:
        mpps.lu_solve(dev(Z), dev(Z), policy=mpps.FIXED)
    assert e.value.status == 6 and "column 0" in str(e.value)
    # the library stays usable
    R = host(mpps.lu_solve(dev(np.eye(3)), dev(np.eye(3)), policy=mpps.FIXED_E))
    assert np.array_equal(R, np.eye(3))


def test_lu_solve_host_pointers_and_alias(mpps):
    n = 97
    rng = np.random.default_rng(8)
    Q = rng.standard_normal((3, n, n))
    P = rng.standard_normal((3, n, n))
    ref = host(mpps.lu_solve(dev(Q), dev(P), policy=mpps.FIXED_E))
    Rh = mpps.lu_solve(Q, P, policy=mpps.FIXED_E)                    # host in, host out
    assert np.array_equal(Rh, ref)
    dP = dev(P)
    mpps.lu_solve(dev(Q), dP, policy=mpps.FIXED_E, out=dP)           # R over P
    assert np.array_equal(host(dP), ref)
    for b in range(3):
        assert residual(Q[b], ref[b], P[b]) <= 8 * n * U


@pytest.mark.parametrize("n", [2048, 6800])
def test_lu_solve_large_sampled(mpps, n):
    rng = np.random.default_rng(9000 + n)
    Q = rng.standard_normal((n, n))
    P = rng.standard_normal((n, n))
    cols = rng.choice(n, 6, replace=False)
    for pol in ("f64e8", "fp64") if n == 2048 else ("f64e8",):
        R = host(mpps.lu_solve(dev(Q), dev(P), policy=policies(mpps)[pol]))
        assert np.isfinite(R).all()
        assert residual(Q, R, P, cols) <= 8 * n * U, pol


def test_lu_solve_pade_denominator(mpps):
    # the system the Pade exp solves: q_13(X) R = p_13(X) for X scaled to ||X||_1 = theta_13,
    # assembled on the host in plain double; R approximates exp(X) (the oracle's Taylor exp)
    n = 96
    X = inputs.gaussian_matrix(n, seed=31, norm1=5.371920351148152)
    num = [float(c) for c in oracle.pade_exp_num_rational(13)]
    p = np.zeros((n, n)); q = np.zeros((n, n)); K = np.eye(n)
    for j, c in enumerate(num):
        p += c * K
        q += (-1) ** j * c * K
        K = K @ X
    R = host(mpps.lu_solve(dev(q), dev(p), policy=mpps.FIXED_E))
    eh, el = oracle.expm_ss_dd(X, 30, oracle.sigma_for(X))
    assert oracle.rel_err_1norm(R, eh, el) <= 50 * n * U
