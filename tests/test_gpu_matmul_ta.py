"""GPU checks of C = A^T B (mpps_matmul_ta): the emulated formats slice A's columns directly
as the left operand, which must give the slices of A^T's rows, so the product equals
mpps_matmul of the transposed A bit for bit (ragged K tails, several tiles, batches); the
other formats transpose first and agree the same way."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("fmt", ["f64e8", "f64e4", "f64e9", "f64e1", "fp64", "bf16", "fp8"])
@pytest.mark.parametrize("n", [1, 17, 64, 127, 130, 300])
def test_matmul_ta_equals_matmul_of_transpose(mpps, fmt, n):
    rng = np.random.default_rng(7700 + n)
    A = rng.standard_normal((2, n, n)) * 2.0 ** rng.integers(-20, 20, (2, 1, n))   # column scales
    B = rng.standard_normal((2, n, n))
    A[1, :, n // 2] = 0.0                      # a zero column of A (a zero row of A^T)
    At = np.ascontiguousarray(np.transpose(A, (0, 2, 1)))
    C = host(mpps.matmul_ta(dev(A), dev(B), fmt))
    R = host(mpps.matmul(dev(At), dev(B), fmt))
    assert np.array_equal(C, R), (fmt, n, np.abs(C - R).max())


def test_matmul_ta_host_pointers(mpps):
    A = inputs.gaussian_batch(3, 96, seed=7, norm1=[1.0, 2.0, 0.5])
    B = inputs.gaussian_batch(3, 96, seed=8, norm1=[1.0, 1.0, 1.0])
    C = mpps.matmul_ta(A, B, "f64e8")
    R = host(mpps.matmul(dev(np.ascontiguousarray(np.transpose(A, (0, 2, 1)))), dev(B), "f64e8"))
    assert np.array_equal(C, R)
