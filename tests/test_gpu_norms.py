"""GPU checks of the block norms that feed the precision rule: FP32 sums of the power table
(Section 3.3: the rule needs the norms only to the right order of magnitude), and the FP64
recomputation of a matrix whose FP32 norms are not finite (powers beyond FP32's range)."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_17396_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("scale", [1.0, 2.0 ** 40])
def test_general_block_norms_fp32_and_fp64_redo(mpps, scale):
    # a batch of two general polynomials' arguments: one of moderate norm (FP32 norms, within
    # 2^-16 of the exact ones) and one whose fourth power (about 2^160) overflows FP32 (its
    # norms are recomputed in FP64: exact to rounding); the results stay within the fixed
    # FP64 bound either way
    n, m = 48, 16
    rng = np.random.default_rng(8800)
    c = rng.standard_normal(m + 1) / np.array([math.factorial(k) for k in range(m + 1)])
    X0 = inputs.gaussian_matrix(n, seed=8801, norm1=1.0)
    X1 = inputs.gaussian_matrix(n, seed=8802, norm1=1.0) * scale
    A = np.stack([X0, X1])
    P, rep = mpps.ps_eval(c, dev(A), policy=mpps.FIXED, report=True)
    P = host(P)
    from fractions import Fraction
    cq = [Fraction(float(v)) for v in c]
    for b, X in enumerate((X0, X1)):
        nb, ny = oracle.block_norms_dd(cq, X)
        got = np.array(rep[b]["normB"])
        tol = 2.0 ** -40 if scale > 1.0 and b == 1 else 2.0 ** -16
        assert np.all(np.abs(got - nb) <= tol * np.abs(nb)), (b, got, nb)
        assert abs(rep[b]["normY"] - ny) <= tol * ny
        assert np.all(np.isfinite(got))
        ph, pl, _ = oracle.ps_dd(cq, X)
        # the rounding bound of the evaluation: 50 n u sum_k |c_k| ||X||^k relative to ||p(X)||
        xn = oracle.norm1(X)
        amp = sum(abs(float(v)) * xn ** k for k, v in enumerate(c)) / oracle.norm1(ph)
        assert oracle.rel_err_1norm(P[b], ph, pl) <= 50 * n * 2.0 ** -53 * max(1.0, amp)
