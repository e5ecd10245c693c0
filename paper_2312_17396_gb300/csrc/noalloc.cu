// noalloc.cu -- mpps_matmul_noalloc: the product of mpps_matmul for callers that are not
// allowed to allocate device memory.  The rounded operand copies, per-matrix scales and the
// error word that the tensor-core product needs live in one file-scope device array of
// fixed size instead of a cudaMallocAsync workspace.
//
// The array is a device symbol: its name in host code is only a host-side handle, so host
// code must not pass it to a kernel.  The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached; the first call on a device
// does that look-up, so make the first call outside any stream capture.
#include "common.cuh"

#include <mutex>

namespace mpps {

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[MPPS_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
mpps_status scratch_address(unsigned char** out) {
    int dev = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("mpps_matmul_noalloc: device index %d out of range", dev);
        return MPPS_ENOTSUP;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return MPPS_ECUDA;
        }
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return MPPS_OK;
}

// Device (or managed) memory that the current device's kernels may touch: a device pointer
// of another GPU is refused, since the kernels and the scratch address belong to this one.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == cur;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mpps

using namespace mpps;

extern "C" mpps_status mpps_matmul_noalloc(const double* A, const double* B, double* C, int n,
                                           int batch, int format, void* stream) {
    clear_error();
    if (n <= 0 || batch < 0 || batch > 65535 || format < MPPS_FMT_FP64 || format > MPPS_FMT_FP8) {
        set_error("mpps_matmul_noalloc: invalid argument (n=%d, batch=%d, format=%d)", n, batch,
                  format);
        return MPPS_EINVAL;
    }
    if (batch == 0) return MPPS_OK;
    if (!A || !B || !C || !on_device(A) || !on_device(B) || !on_device(C)) {
        set_error("mpps_matmul_noalloc: A, B and C must be device pointers");
        return MPPS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long nn = (long long)n * n;
    Epilogue ep = epilogue_plain(C, nn);
    if (format == MPPS_FMT_FP64)   // the FP64 product needs no scratch
        return launch_gemm_f64(A, nn, B, nn, n, batch, ep, st);
    if (format == MPPS_FMT_FP8) {   // block scales along K: FP8 copies, scale codes, exponents
        const size_t wb = align256(fp8mx_ws_bytes(n, batch));
        if (wb + 256 > (size_t)MPPS_NOALLOC_SCRATCH_BYTES) {
            set_error("mpps_matmul_noalloc: n=%d batch=%d format=%d needs %zu bytes of scratch, "
                      "more than the fixed %zu",
                      n, batch, format, wb + 256, (size_t)MPPS_NOALLOC_SCRATCH_BYTES);
            return MPPS_EINVAL;
        }
        unsigned char* base = nullptr;
        mpps_status rc = scratch_address(&base);
        if (rc) return rc;
        int* err = (int*)(base + wb);
        MPPS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        if ((rc = launch_product_fp8mx(A, nn, B, nn, n, batch, ep, fp8mx_ws_carve(base, n, batch), err, st)))
            return rc;
        int h_err = 0;
        MPPS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_err) {
            set_error("a bounded wait in the tensor-core product timed out");
            return MPPS_ETIMEOUT;
        }
        return MPPS_OK;
    }

    // scratch layout: A copy (hi, lo), B^T copy (hi, lo), maxabs a/b, scales a/b, unscale, err
    const int lld = low_ld(n);
    const long long low_bs = (long long)n * lld;
    const size_t es = (size_t)low_elem_bytes(format);
    const bool x3 = format == MPPS_FMT_BF16X3;
    const size_t plane = align256((size_t)batch * low_bs * es);
    const size_t vec = align256(sizeof(double) * (size_t)batch);
    const size_t need = plane * (x3 ? 4 : 2) + 5 * vec + 256;
    if (need > (size_t)MPPS_NOALLOC_SCRATCH_BYTES) {
        set_error("mpps_matmul_noalloc: n=%d batch=%d format=%d needs %zu bytes of scratch, more "
                  "than the fixed %zu",
                  n, batch, format, need, (size_t)MPPS_NOALLOC_SCRATCH_BYTES);
        return MPPS_EINVAL;
    }
    unsigned char* base = nullptr;
    mpps_status rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char* p = base;
    void* ahi = p; p += plane;
    void* alo = x3 ? (void*)p : nullptr; if (x3) p += plane;
    void* bhi = p; p += plane;
    void* blo = x3 ? (void*)p : nullptr; if (x3) p += plane;
    double* ma = (double*)p; p += vec;
    double* mb = (double*)p; p += vec;
    double* sa = (double*)p; p += vec;
    double* sb = (double*)p; p += vec;
    double* un = (double*)p; p += vec;
    int* err = (int*)p;

    // the array keeps the previous call's contents: zero what the kernels accumulate into
    MPPS_CUDA_TRY(cudaMemsetAsync(ma, 0, 2 * vec, st));
    MPPS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    if ((rc = launch_maxabs(A, nn, n, batch, ma, st))) return rc;
    if ((rc = launch_maxabs(B, nn, n, batch, mb, st))) return rc;
    if ((rc = launch_pow2_scales(ma, mb, batch, 0, sa, sb, un, st))) return rc;
    if ((rc = launch_convert(format, A, nn, n, batch, ahi, alo, low_bs, lld, sa, false, st))) return rc;
    if ((rc = launch_convert(format, B, nn, n, batch, bhi, blo, low_bs, lld, sb, true, st))) return rc;
    ep.alpha_b = un;
    if ((rc = launch_gemm_tc(format, ahi, alo, bhi, blo, low_bs, low_bs, lld, n, batch, ep, err, st)))
        return rc;
    int h_err = 0;
    MPPS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) {
        set_error("a bounded wait in the tensor-core product timed out");
        return MPPS_ETIMEOUT;
    }
    return MPPS_OK;
}
