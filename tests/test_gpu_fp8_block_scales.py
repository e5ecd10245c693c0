"""GPU parity of the FP8 product with block scales (tcgen05 kind::mxf8f6f4) against the
oracle's quantisation.

The library rounds each row of A and each column of B to E4M3 after its own power of two
and one power of two per 32 entries along K; the tensor core applies the block scales and
sums in FP32.  The oracle (``oracle.matmul_mxfp8``) quantises the same way, from the format's
definition, and sums in FP64.  Both sides make every rounding decision on exact values, so
the only difference is the FP32 accumulation: |C - C_oracle| <= 2 n 2^-23 |A~||B~| (the
quantised factors), far below one E4M3 rounding step of a single product, so that a
different scale or a different rounding of one entry shows.
"""
import numpy as np
import pytest

import oracle

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


def _block_graded(rng, batch, n, spread):
    """Gaussian entries, each 32-entry block of a row (of A) / column (of B) times its own
    power of two 2^U(-spread, spread): one scale per row would flush the small blocks."""
    nb = -(-n // 32)
    A = rng.standard_normal((batch, n, n))
    B = rng.standard_normal((batch, n, n))
    ga = np.repeat(2.0 ** rng.integers(-spread, spread + 1, (batch, n, nb)), 32, axis=2)[:, :, :n]
    gb = np.repeat(2.0 ** rng.integers(-spread, spread + 1, (batch, nb, n)), 32, axis=1)[:, :n, :]
    return A * ga, B * gb


@pytest.mark.parametrize("n", [1, 8, 31, 64, 127, 130, 257, 300])
def test_fp8_block_scaled_matmul_vs_oracle(mpps, n):
    rng = np.random.default_rng(8100 + n)
    A, B = _block_graded(rng, 2, n, 12)
    A[1, n // 2] = 0.0                      # a zero row
    C = host(mpps.matmul(dev(A), dev(B), "fp8"))
    for b in range(2):
        ref, absq = oracle.matmul_mxfp8(A[b], B[b])
        tol = 2 * n * 2.0 ** -23 * absq
        bad = np.abs(C[b] - ref) > tol
        assert not bad.any(), (b, np.argwhere(bad)[:5], C[b][bad][:5], ref[bad][:5])
    assert np.all(C[1, n // 2] == 0.0)


@pytest.mark.parametrize("n", [96, 256])
def test_fp8_block_scales_keep_each_block(mpps, n):
    # blocks 2^30 apart along K, entries of one block within a factor 2: every product keeps
    # E4M3's relative accuracy, componentwise (one scale per row and column would lose the
    # small blocks entirely)
    rng = np.random.default_rng(8200 + n)
    sgn = lambda s: np.where(rng.random(s) < 0.5, -1.0, 1.0)
    A = rng.uniform(0.5, 1.0, (1, n, n)) * sgn((1, n, n))
    B = rng.uniform(0.5, 1.0, (1, n, n)) * sgn((1, n, n))
    A[:, :, 32:64] *= 2.0 ** -30
    B[:, 32:64, :] *= 2.0 ** 30             # the small blocks of A meet large ones of B
    B[:, 64:96, :] *= 2.0 ** -25
    C = host(mpps.matmul(dev(A), dev(B), "fp8"))[0]
    u = 2.0 ** -4
    absprod = np.abs(A[0]) @ np.abs(B[0])
    assert np.all(np.abs(C - A[0] @ B[0]) <= (2 * u + u * u + 2 * n * 2.0 ** -23) * absprod)


@pytest.mark.parametrize("scale", [2.0 ** -900, 2.0 ** 900])
def test_fp8_block_scaled_matmul_far_from_one(mpps, scale):
    # the row and column powers of two carry any FP64 magnitude through E4M3 and FP32
    n = 130
    rng = np.random.default_rng(8300)
    A, B = _block_graded(rng, 1, n, 6)
    C = host(mpps.matmul(dev(A * scale), dev(B), "fp8"))[0]
    ref, absq = oracle.matmul_mxfp8(A[0] * scale, B[0])
    assert np.all(np.abs(C - ref) <= 2 * n * 2.0 ** -23 * absq)
    assert np.all(np.isfinite(C)) and np.abs(C).max() > 0
