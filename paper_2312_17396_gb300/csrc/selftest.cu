// selftest.cu -- exercises the failure path of the bounded waits without faulting the GPU:
// one CTA waits on an mbarrier that nothing ever arrives on, gives up after a short limit,
// sets the device error word and returns normally.  The host then reports MPPS_ETIMEOUT
// exactly as it would for a stalled tensor-core product.
#include "common.cuh"
#include "tcgen05.cuh"

namespace mpps {
namespace {

__global__ void k_wait_selftest(int* err, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tc::mbar_wait(&bar, 0, err, limit_ns);   // nobody arrives: phase 0 never completes
    __syncthreads();
}

}  // namespace
}  // namespace mpps

using namespace mpps;

extern "C" mpps_status mpps_selftest_bounded_wait(int limit_us, void* stream) {
    clear_error();
    if (limit_us <= 0 || limit_us > 2000000) {
        set_error("mpps_selftest_bounded_wait: limit_us must be in 1..2000000");
        return MPPS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int* d = nullptr;
    MPPS_CUDA_TRY(cudaMallocAsync(&d, sizeof(int), st));
    MPPS_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int), st));
    k_wait_selftest<<<1, 64, 0, st>>>(d, (unsigned long long)limit_us * 1000ull);
    cudaError_t le = cudaGetLastError();
    int h = 0;
    cudaError_t ce = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t se = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    if (le != cudaSuccess || ce != cudaSuccess || se != cudaSuccess) {
        set_error("selftest launch failed: %s",
                  cudaGetErrorString(le != cudaSuccess ? le : (ce != cudaSuccess ? ce : se)));
        return MPPS_ECUDA;
    }
    if (h) {
        set_error("bounded wait gave up after %d us (as intended by the self-test)", limit_us);
        return MPPS_ETIMEOUT;
    }
    return MPPS_OK;
}
