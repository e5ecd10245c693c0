"""The allocation-free product entry point (mpps_matmul_noalloc).

It serves callers that may not allocate device memory (a framework's allocator already
owns the memory, allocator calls are banned on a latency-bound path, or a plug-in is only
handed buffers).  Its scratch is a fixed array inside the library.  This file is collected
last on purpose; it must pass alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_17396_gb300 as m
    m.lib()
    return m


def _call(mpps, A, B, C, fmt):
    L = mpps.lib()
    n, batch = A.shape[-1], A.shape[0]
    f = {"fp64": 0, "bf16x3": 1, "tf32": 2, "bf16": 3, "fp8": 4}[fmt]
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.mpps_matmul_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                 ctypes.c_void_p(C.data_ptr()), n, batch, f, st)


@pytest.mark.parametrize("fmt", ["fp64", "bf16", "bf16x3", "tf32", "fp8"])
@pytest.mark.parametrize("n,batch", [(130, 2), (64, 1), (257, 1)])
def test_noalloc_matches_matmul_twice(mpps, fmt, n, batch):
    rng = np.random.default_rng(n + batch)
    A = torch.from_numpy(rng.standard_normal((batch, n, n))).cuda()
    B = torch.from_numpy(rng.standard_normal((batch, n, n))).cuda()
    ref = mpps.matmul(A, B, fmt).cpu().numpy()
    for _ in range(2):                      # two calls in a row share the scratch array
        C = torch.full_like(A, np.nan)
        assert _call(mpps, A, B, C, fmt) == 0, mpps.lib().mpps_last_error()
        got = C.cpu().numpy()
        # same kernels on the same inputs: within the product tolerance, in fact identical
        assert np.array_equal(got, ref)


def test_noalloc_after_different_sizes(mpps):
    """The array keeps the previous call's contents; a smaller call after a larger one must
    not see stale scales or maxima."""
    rng = np.random.default_rng(3)
    big = torch.from_numpy(1e6 * rng.standard_normal((1, 300, 300))).cuda()
    small = torch.from_numpy(1e-6 * rng.standard_normal((1, 40, 40))).cuda()
    Cb = torch.empty_like(big); Cs = torch.empty_like(small)
    assert _call(mpps, big, big, Cb, "bf16") == 0
    assert _call(mpps, small, small, Cs, "bf16") == 0
    assert np.array_equal(Cs.cpu().numpy(), mpps.matmul(small, small, "bf16").cpu().numpy())


def test_noalloc_rejects_oversize_and_host_pointers(mpps):
    n = 4096                                 # bf16x3 at 4096 needs 128 MiB > the fixed array
    A = torch.zeros((1, n, n), dtype=torch.float64, device="cuda")
    C = torch.empty_like(A)
    assert _call(mpps, A, A, C, "bf16x3") == 1
    assert b"scratch" in mpps.lib().mpps_last_error()
    h = torch.zeros((1, 8, 8), dtype=torch.float64)
    assert _call(mpps, h, h, h, "bf16") == 1
