// gemm_f64.cu -- FP64 matrix product on the FP64 tensor pipe (DMMA, mma.sync m16n8k4 f64)
// for the steps the paper keeps in the working precision: the powers X^2..X^s
// (Algorithm 2.1, Fragment 3.1), the Horner products of the early steps (eq. (2.10)) and
// the squarings of eq. (3.6).  The block sum B_{i-1} of a Horner step is fused into the
// epilogue (P_{i-1} = B_{i-1} + P_i Y), so P_i Y never makes a round trip through HBM.
//
// tcgen05 has no FP64 kind; on GB300 the FP64 rate (about 1 TFLOP/s per GPU) is the same
// for DMMA and DFMA, so this kernel is bound by that pipe at every size used here.  The
// tile is 64 x 64 x 16 (8 warps) or 32 x 32 x 16 (4 warps) with a two-stage cp.async
// pipeline; operands are loaded with 8-byte cp.async so that any n (odd included) works.
#include "common.cuh"

namespace mpps {

namespace {

constexpr int BK = 16;
constexpr int APAD = 4, BPAD = 4;   // row pads: conflict-free fragment reads

__device__ __forceinline__ void cp_async8(void* smem, const double* gmem, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int bytes = pred ? 8 : 0;      // 0 -> zero-fill, nothing read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void dmma_16x8x4(double (&d)[4], double a0, double a1, double b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};\n"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a0), "d"(a1), "d"(b0));
}

// Tile BM x BN x BK; WM x WN warps, each owning a (BM/WM) x (BN/WN) block of m16n8
// fragments.  Two-stage cp.async pipeline.
template <int BM, int BN, int WM, int WN>
__global__ void __launch_bounds__(32 * WM * WN)
    k_gemm_f64(const double* __restrict__ A, long long a_bs, const double* __restrict__ B,
               long long b_bs, int n, Epilogue ep, const int* __restrict__ bidx) {
    pdl_wait();
    if (ep.dcount && (int)blockIdx.z >= __ldg(ep.dcount)) return;   // device plan: not run
    constexpr int NT = 32 * WM * WN;
    constexpr int WTM = BM / WM, WTN = BN / WN;   // warp tile
    constexpr int MI = WTM / 16, NI = WTN / 8;    // fragments per warp
    constexpr int A_PER = BM * BK / NT, B_PER = BK * BN / NT;
    static_assert(MI >= 1 && NI >= 1 && A_PER >= 1 && B_PER >= 1, "tile shape");
    __shared__ __align__(16) double As[2][BM][BK + APAD];
    __shared__ __align__(16) double Bs[2][BK][BN + BPAD];

    int ba, bb, b;   // A and B operand matrices, output matrix (grid mode: Epilogue::gnj)
    grid_index(ep, (int)blockIdx.z, bidx ? bidx[blockIdx.z] : (int)blockIdx.z, ba, bb, b);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const double* Ab = A + (long long)ba * a_bs;
    const double* Bb = B + (long long)bb * b_bs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wm = warp / WN, wn = warp % WN;

    // loader: A_PER consecutive doubles of one A row, B_PER of one B row per thread
    const int a_row = tid / (BK / A_PER), a_col = (tid % (BK / A_PER)) * A_PER;
    const int b_row = tid / (BN / B_PER), b_col = (tid % (BN / B_PER)) * B_PER;

    auto load_stage = [&](int stage, int k0) {
        const int gr = m0 + a_row;
#pragma unroll
        for (int q = 0; q < A_PER; ++q) {
            const int gc = k0 + a_col + q;
            const bool ok = gr < n && gc < n;
            cp_async8(&As[stage][a_row][a_col + q], ok ? Ab + (long long)gr * n + gc : Ab, ok);
        }
        const int kr = k0 + b_row;
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
            const int gc = n0 + b_col + q;
            const bool ok = kr < n && gc < n;
            cp_async8(&Bs[stage][b_row][b_col + q], ok ? Bb + (long long)kr * n + gc : Bb, ok);
        }
        cp_async_commit();
    };

    double acc[MI][NI][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0;

    const int nk = (n + BK - 1) / BK;
    load_stage(0, 0);
    for (int kb = 0; kb < nk; ++kb) {
        const int cur = kb & 1;
        cp_async_wait_all();
        __syncthreads();
        if (kb + 1 < nk) load_stage(cur ^ 1, (kb + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double a[MI][2], bf[NI];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                a[mi][0] = As[cur][wm * WTM + mi * 16 + g][kk + t];
                a[mi][1] = As[cur][wm * WTM + mi * 16 + g + 8][kk + t];
            }
#pragma unroll
            for (int ni = 0; ni < NI; ++ni) bf[ni] = Bs[cur][kk + t][wn * WTN + ni * 8 + g];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) dmma_16x8x4(acc[mi][ni], a[mi][0], a[mi][1], bf[ni]);
        }
        __syncthreads();
    }

    // epilogue: accumulator element q of fragment (mi, ni) sits at
    // row = g (+8 for q >= 2), col = 2t + (q & 1)
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = m0 + wm * WTM + mi * 16 + g + (q >> 1) * 8;
                const int col = n0 + wn * WTN + ni * 8 + 2 * t + (q & 1);
                if (row < n && col < n)
                    epilogue_store(ep, b, row, col, n, epilogue_value(ep, b, row, col, n, acc[mi][ni][q]));
            }
}

int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            g_num_sms = v;
        else
            g_num_sms = 152;
    }
    return g_num_sms;
}

}  // namespace

// The FP64 pipe is shared by all CTAs resident on an SM, so the time of a launch is set by
// the most loaded SM: pick the tile that minimises ceil(tiles / SMs) * tile area (ties go
// to the larger tile).
mpps_status launch_gemm_f64(const double* A, long long a_bs, const double* B, long long b_bs,
                            int n, int batch, const Epilogue& ep, cudaStream_t st,
                            const int* bidx) {
    if (batch <= 0) return MPPS_OK;
    ProfScope prof(MPPS_PROF_GEMM_F64, st, 2.0 * n * (double)n * n * batch);
    const long long sms = num_sms();
    const long long t64 = (long long)((n + 63) / 64) * ((n + 63) / 64) * batch;
    const long long t32 = (long long)((n + 31) / 32) * ((n + 31) / 32) * batch;
    const long long load64 = (t64 + sms - 1) / sms * 4096, load32 = (t32 + sms - 1) / sms * 1024;
    if (load32 < load64) {
        dim3 grid((n + 31) / 32, (n + 31) / 32, batch);
        MPPS_CUDA_TRY(launch_pdl(k_gemm_f64<32, 32, 2, 2>, dim3(grid), dim3(128), 0, st, A, a_bs, B, b_bs, n, ep, bidx));
    } else {
        dim3 grid((n + 63) / 64, (n + 63) / 64, batch);
        MPPS_CUDA_TRY(launch_pdl(k_gemm_f64<64, 64, 2, 4>, dim3(grid), dim3(256), 0, st, A, a_bs, B, b_bs, n, ep, bidx));
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

}  // namespace mpps
