// gemm_f64e.cu -- FP64-accurate matrix product on the BF16 tensor cores by exact slice
// products (the splitting method of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59 (2012), adapted to tcgen05 with FP32 accumulation).
//
// On GB300 the FP64 pipe delivers about 1 TFLOP/s while BF16 tensor cores deliver about
// 1900, so the working-precision products of the PS evaluation (powers, early Horner steps,
// squarings) are emulated:
//
//   A (rows scaled by 2^-eA_i, |.| < 1) = sum_{t<k} 2^{-6(t+1)} a_t,  a_t integers, |a_t| <= 64
//   B (cols scaled by 2^-eB_j)          = sum_{q<k} 2^{-6(q+1)} b_q
//   A B ~= 2^{eA_i + eB_j} sum_{d<k} 2^{-6(d+2)} D_d,   D_d = sum_{t+q=d} a_t b_q^T.
//
// Every a_t, b_q entry is an integer of at most 7 bits, exact in bf16; every product is exact
// in FP32 and, for K <= 1024, every diagonal sum D_d is an integer below
// 1024 * 2^10 * (d + 3) <= 2^24 (d <= 13), so the tensor cores accumulate it EXACTLY in FP32.
// Longer K is cut into 1024-chunks whose D_d are drained into FP64 between chunks.  The
// result differs from the exact product only by the slices dropped (t + q >= k) and the
// residual of the k-slice representation, about 2^{-6k} relative to the row and column
// maxima: k = 9 gives FP64-level accuracy.
//
// Kernel: one CTA per 128 x 32 output tile, 6 warps (0-3 epilogue = TMEM lanes, 4 TMA
// producer, 5 MMA issuer).  Per K-block of 32 the producer loads the k slices of the A tile
// (128 x 32 bf16 each) and the k slices of the B^T tile (32 x 32 each), stacked so that the
// B operand of slice t is B_0..B_{k-1-t} (N = 32 (k - t) rows): one MMA per t and K=16 step
// writes its k - t partial products into the TMEM columns 32 (t + q), i.e. straight into
// the accumulator of diagonal d = t + q.  Operands are K-major with the 64-byte swizzle; the
// ring holds up to 8 stages (2 for k = 9; a 16-wide K with the 32-byte swizzle and 4 stages
// measured slower).  All mbarrier waits are bounded.
#include "common.cuh"
#include "tcgen05.cuh"

#include <cudaTypedefs.h>

#include <map>
#include <mutex>

namespace mpps {

int f64e_cluster_choice(int dev, int n, int k, int batch);

namespace {

using namespace tc;

constexpr int OM = 128;                 // output rows per CTA
constexpr int ON = 32;                  // output cols per CTA (= columns per diagonal region)
constexpr int KB = 32;                  // K elements per stage (64 bytes of bf16: two MMA steps)
constexpr int KCHUNK = 1024;            // exact FP32 accumulation bound (see above)
constexpr int A_TILE = OM * KB * 2;     // 8 KB
constexpr int B_TILE = ON * KB * 2;     // 2 KB
constexpr int SMEM_BUDGET = 200 * 1024;
constexpr int MAX_STAGES = 8;
// barriers after the ring: full + empty per stage, chunk_done, tmem_free, TMEM slot
static_assert((2 * MAX_STAGES + 2) * 8 + 4 <= 256, "barrier block exceeds its reserved 256 bytes");

__host__ __device__ inline int stage_bytes(int k) { return k * (A_TILE + B_TILE); }
__host__ __device__ inline int num_stages(int k) {
    int s = SMEM_BUDGET / stage_bytes(k);
    return s > MAX_STAGES ? MAX_STAGES : s;
}
__host__ __device__ inline uint32_t tmem_cols(int k) {
    uint32_t need = (uint32_t)(ON * k), c = 32;
    while (c < need) c <<= 1;
    return c;
}

// Signed base-64 digits of x / 2^e (|x| < 2^e), computed in integers:
//   F = round(x 2^(62-e)) (|F| < 2^62);  for t: p = 56 - 6t, v_t = floor((F + 2^(p-1)) / 2^p),
//   F -= v_t 2^p.  |v_0| <= 64, |v_t| <= 32 (t >= 1); after k digits |F| <= 2^(55-6(k-1)), i.e.
//   x = 2^e (sum_t v_t 2^(-6(t+1)) + r) with |r| <= 2^(-6k-1).  Only one FP64 multiply and one
//   conversion per value: the digit loop runs on the integer pipe.
__device__ __forceinline__ void put_digits(double x, double scale, int k, __nv_bfloat16* dst,
                                           long long pstride) {
    long long F = __double2ll_rn(x * scale);
#pragma unroll 1
    for (int t = 0; t < k; ++t) {
        const int p = 56 - 6 * t;
        const long long v = (F + (1LL << (p - 1))) >> p;
        F -= v << p;
        dst[(long long)t * pstride] = __int2bfloat16_rn((int)v);
    }
}

__device__ __forceinline__ int exp_above(double mx) {
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
    return e;
}

// Row slices (A operand): one warp per row; e_i from the row maximum.
__global__ void k_slice_rows(const double* __restrict__ M, long long bs, int n, int k,
                             __nv_bfloat16* __restrict__ planes, long long plane_bs, int lld,
                             int* __restrict__ exps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp, b = blockIdx.y;
    if (row >= n) return;
    const double* src = M + (long long)b * bs + (long long)row * n;
    double mx = 0.0;
    for (int j = lane; j < n; j += 32) mx = fmax(mx, fabs(src[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exp_above(mx);
    if (lane == 0) exps[(long long)b * n + row] = e;
    const double scale = ldexp(1.0, 62 - e);
    __nv_bfloat16* dst = planes + (long long)b * plane_bs + (long long)row * lld;
    const long long pstride = (long long)n * lld;
    int j = lane;
    for (; j + 96 < n; j += 128) {              // 4 loads in flight per lane
        const double x0 = src[j], x1 = src[j + 32], x2 = src[j + 64], x3 = src[j + 96];
        put_digits(x0, scale, k, dst + j, pstride);
        put_digits(x1, scale, k, dst + j + 32, pstride);
        put_digits(x2, scale, k, dst + j + 64, pstride);
        put_digits(x3, scale, k, dst + j + 96, pstride);
    }
    for (; j < n; j += 32) put_digits(src[j], scale, k, dst + j, pstride);
}

// Row maxima of |M| -> exponents e_i (one warp per row).
__global__ void k_rowexp(const double* __restrict__ M, long long bs, int n, int* __restrict__ exps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp, b = blockIdx.y;
    if (row >= n) return;
    const double* src = M + (long long)b * bs + (long long)row * n;
    double mx = 0.0;
    for (int j = lane; j < n; j += 32) mx = fmax(mx, fabs(src[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) exps[(long long)b * n + row] = exp_above(mx);
}

// Row slices, one thread per element (the exponents come from k_rowexp).
__global__ void k_slice_rows_elem(const double* __restrict__ M, long long bs, int n, int k,
                                  const int* __restrict__ exps, __nv_bfloat16* __restrict__ planes,
                                  long long plane_bs, int lld) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y, b = blockIdx.z;
    if (col >= n) return;
    const int e = exps[(long long)b * n + row];
    put_digits(M[(long long)b * bs + (long long)row * n + col], ldexp(1.0, 62 - e), k,
               planes + (long long)b * plane_bs + (long long)row * lld + col, (long long)n * lld);
}

// Column maxima of |M| (as the bit pattern of a non-negative double; out zeroed first).
__global__ void k_colmax(const double* __restrict__ M, long long bs, int n,
                         unsigned long long* __restrict__ out) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.z;
    if (col >= n) return;
    const int r0 = blockIdx.y * 64, r1 = min(n, r0 + 64);
    const double* src = M + (long long)b * bs + col;
    double mx = 0.0;
    for (int row = r0; row < r1; ++row) mx = fmax(mx, fabs(src[(long long)row * n]));
    atomicMax(out + (long long)b * n + col, (unsigned long long)__double_as_longlong(mx));
}

// Column slices (B operand, written transposed: plane row j = column j of M), 32 x 32 tiles
// through shared memory; e_j from the column maxima.
__global__ void k_slice_cols(const double* __restrict__ M, long long bs, int n, int k,
                             const unsigned long long* __restrict__ colmax,
                             __nv_bfloat16* __restrict__ planes, long long plane_bs, int lld,
                             int* __restrict__ exps) {
    __shared__ double tile[32][33];
    const int b = blockIdx.z, r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const double* src = M + (long long)b * bs;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int row = r0 + i, col = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (row < n && col < n) ? src[(long long)row * n + col] : 0.0;
    }
    __syncthreads();
    const long long pstride = (long long)n * lld;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int col = c0 + i, row = r0 + threadIdx.x;     // output row = column of M
        if (col >= n || row >= n) continue;
        const int e = exp_above(__longlong_as_double((long long)colmax[(long long)b * n + col]));
        if (blockIdx.y == 0 && threadIdx.x == 0) exps[(long long)b * n + col] = e;
        put_digits(tile[threadIdx.x][i], ldexp(1.0, 62 - e), k,
                   planes + (long long)b * plane_bs + (long long)col * lld + row, pstride);
    }
}

// CL > 1: the CTA is one of CL neighbours along the output columns (a cluster) sharing the
// same row block; each loads the A slices t = rank (mod CL) and multicasts them to all CL,
// and every CTA's MMA completion is signalled to all CL (a stage is reloaded only when all
// of them have consumed it).
template <int CL>
__global__ void __launch_bounds__(192, 1)
    k_gemm_f64e(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                int n, int k, int ksA, int ksB, const int* __restrict__ eA,
                const int* __restrict__ eB, Epilogue ep, int* err, const int* __restrict__ bidx) {
    const int S = num_stages(k);
    const int SB = stage_bytes(k);
    const uint32_t TCOLS = tmem_cols(k);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // barrier block after the stage ring: full[MAX_STAGES] | empty[MAX_STAGES] | chunk_done |
    // tmem_free | TMEM address slot  (148 bytes of the 256 reserved)
    uint64_t* full = (uint64_t*)(smem + S * SB);
    uint64_t* empty = full + MAX_STAGES;
    uint64_t* chunk_done = empty + MAX_STAGES;
    uint64_t* tmem_free = chunk_done + 1;
    uint32_t* tmem_slot = (uint32_t*)(tmem_free + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = bidx ? bidx[blockIdx.z] : blockIdx.z;
    const int m0 = blockIdx.y * OM, n0 = blockIdx.x * ON;
    const int nkb = (n + KB - 1) / KB;                      // K-blocks
    const int kb_per_chunk = KCHUNK / KB;
    const int nchunks = (nkb + kb_per_chunk - 1) / kb_per_chunk;

    const uint32_t crank = CL > 1 ? cluster_ctarank() : 0;
    constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CL);
        }
        mbar_init(chunk_done, 1);
        mbar_init(tmem_free, 128);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, TCOLS);
    tc_fence_before();
    __syncthreads();
    if constexpr (CL > 1) cluster_sync();   // peers' barriers exist before any multicast
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        if (lane == 0) {   // TMA producer: k A slices + k B slices per K-block
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % S;
                if (kb >= S && !mbar_wait(&empty[s], ((kb / S) - 1) & 1, err)) break;
                mbar_expect_tx(&full[s], (uint32_t)SB);
                uint8_t* st = smem + s * SB;
                const int kc = kb * KB;
                for (int t = 0; t < k; ++t) {
                    if constexpr (CL > 1) {
                        if (t % CL == (int)crank)
                            tma_load_3d_mc(st + t * A_TILE, &tmA, kc, m0, b * ksA + t, &full[s], kMask);
                    } else {
                        tma_load_3d(st + t * A_TILE, &tmA, kc, m0, b * ksA + t, &full[s]);
                    }
                    tma_load_3d(st + k * A_TILE + t * B_TILE, &tmB, kc, n0, b * ksB + t, &full[s]);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int s = kb % S;
                const int c = kb / kb_per_chunk, kin = kb % kb_per_chunk;
                if (kin == 0 && c > 0) {   // the epilogue must have drained the previous chunk
                    ok = mbar_wait(tmem_free, (c - 1) & 1, err);
                    if (!ok) break;
                    tc_fence_after();
                }
                ok = mbar_wait(&full[s], (kb / S) & 1, err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t abase = smem_u32(smem + s * SB);
                const uint32_t bbase = abase + k * A_TILE;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {        // two K=16 steps per 64-byte row
                    for (int t = 0; t < k; ++t) {
                        const int N = ON * (k - t);
                        const uint32_t acc = (kin == 0 && kk == 0 && t == 0) ? 0u : 1u;
                        const uint64_t ad = sw64_desc(abase + t * A_TILE + kk * 32);
                        const int n1 = N > 256 ? 256 : N;
                        mma_bf16(tmem + (uint32_t)(ON * t), ad, sw64_desc(bbase + kk * 32),
                                 make_idesc(1, OM, n1), acc);
                        if (N > 256)   // rows 256.. of the stacked B: 32 atoms of 512 B further
                            mma_bf16(tmem + (uint32_t)(ON * t + 256), ad,
                                     sw64_desc(bbase + 256 / 8 * 512 + kk * 32),
                                     make_idesc(1, OM, N - 256), acc);
                    }
                }
                if constexpr (CL > 1) tc_commit_mc(&empty[s], kMask);
                else tc_commit(&empty[s]);
                if (kin == kb_per_chunk - 1 || kb == nkb - 1) tc_commit(chunk_done);
            }
            if (!ok) tc_commit(chunk_done);
        }
    } else {
        // epilogue warps 0-3: row = m0 + 32 w + lane; 32 output columns each
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        double sum[ON];
#pragma unroll
        for (int j = 0; j < ON; ++j) sum[j] = 0.0;
        for (int c = 0; c < nchunks; ++c) {
            mbar_wait(chunk_done, c & 1, err);
            tc_fence_after();
            for (int d = 0; d < k; ++d) {
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(ON * d), v);
                const double sc = ldexp(1.0, -6 * (d + 2));
#pragma unroll
                for (int j = 0; j < ON; ++j) sum[j] = fma((double)__uint_as_float(v[j]), sc, sum[j]);
            }
            tc_fence_before();
            mbar_arrive_cta(tmem_free);
        }
        // rows -> a 32 x 33 shared tile per warp (the ring is idle now), then one column per
        // lane: coalesced reads of the power table and coalesced stores
        double* stile = (double*)smem + warp * 32 * 33;
        const int er = row < n ? eA[(long long)b * n + row] : 0;
#pragma unroll
        for (int j = 0; j < ON; ++j) stile[lane * 33 + j] = ldexp(sum[j], er);
        __syncwarp();
        const int col = n0 + lane;
        const int ec = col < n ? eB[(long long)b * n + col] : 0;
#pragma unroll 1
        for (int r4 = 0; r4 < 32; r4 += 4) {      // 4 rows per pass: their loads overlap
            double val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = m0 + warp * 32 + r4 + u;
                val[u] = (r < n && col < n)
                             ? epilogue_value(ep, b, r, col, n, ldexp(stile[(r4 + u) * 33 + lane], ec))
                             : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = m0 + warp * 32 + r4 + u;
                if (r < n && col < n) epilogue_store(ep, b, r, col, n, val[u]);
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
    // no CTA leaves while a peer may still signal its barriers or multicast into it
    if constexpr (CL > 1) cluster_sync();
}

// ---- host -----------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// planes: [batch * k][n][lld] bf16 -> 3-D map (K = n, rows = n, planes), box 32 x rows x 1
bool make_plane_map(CUtensorMap* tm, const void* ptr, int n, int nplanes, int lld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)lld * 2, (cuuint64_t)n * lld * 2};
    cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch with a cluster of `cl` CTAs along the output columns (grid x rounded up to it).
mpps_status launch_f64e_cl(int cl, const CUtensorMap& ta, const CUtensorMap& tb, int n, int k,
                           int ksA, int ksB, const int* eA, const int* eB, int batch,
                           const Epilogue& ep, int* d_err, cudaStream_t st, const int* bidx,
                           int smem) {
    const int gx = (n + ON - 1) / ON;
    dim3 grid((gx + cl - 1) / cl * cl, (n + OM - 1) / OM, batch);
    if (cl == 1) {
        k_gemm_f64e<1><<<grid, 192, smem, st>>>(ta, tb, n, k, ksA, ksB, eA, eB, ep, d_err, bidx);
        MPPS_LAUNCH_CHECK();
        return MPPS_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = (cl == 2)
        ? cudaLaunchKernelEx(&cfg, k_gemm_f64e<2>, ta, tb, n, k, ksA, ksB, eA, eB, ep, d_err, bidx)
        : cudaLaunchKernelEx(&cfg, k_gemm_f64e<4>, ta, tb, n, k, ksA, ksB, eA, eB, ep, d_err, bidx);
    if (e != cudaSuccess) {
        set_error("cluster launch of the emulated FP64 product failed: %s", cudaGetErrorString(e));
        return MPPS_ECUDA;
    }
    return MPPS_OK;
}

}  // namespace

// ---- autotuner: cluster size of the emulated product per (device, size class, slices) ----
// On the first product of a size class (n rounded up to a power of two, batch 1 vs many) the
// three cluster sizes are timed on scratch operands of that size and the fastest is kept
// for the process.  The timing synchronises the device once per class: make a first call
// of each size before capturing a CUDA graph.
namespace {
std::mutex g_tune_mu;
std::map<long long, int> g_tuned;
}

int f64e_cluster_choice(int dev, int n, int k, int batch) {
    int cls = 1;
    while (cls < n) cls <<= 1;
    const long long key = ((long long)dev << 40) | ((long long)cls << 8) | ((long long)k << 1) |
                          (batch > 1 ? 1 : 0);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
    }
    int best = 1;
    // time on scratch buffers: the caller's epilogue may accumulate into its output
    const int ntune = cls < 64 ? 64 : (cls > 2048 ? 2048 : cls);
    const int bt = batch > 1 ? 8 : 1;
    const int lld = low_ld(ntune);
    const size_t plane_b = (size_t)bt * k * ntune * lld * 2;
    void *sa = nullptr, *sb = nullptr, *ex = nullptr, *out = nullptr, *er = nullptr;
    cudaStream_t ts = nullptr;
    bool ok = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&sa, plane_b) == cudaSuccess && cudaMalloc(&sb, plane_b) == cudaSuccess &&
              cudaMalloc(&ex, sizeof(int) * bt * ntune) == cudaSuccess &&
              cudaMalloc(&out, sizeof(double) * bt * ntune * ntune) == cudaSuccess &&
              cudaMalloc(&er, sizeof(int)) == cudaSuccess;
    if (ok) {
        cudaMemsetAsync(sa, 0, plane_b, ts);
        cudaMemsetAsync(sb, 0, plane_b, ts);
        cudaMemsetAsync(ex, 0, sizeof(int) * bt * ntune, ts);
        cudaMemsetAsync(er, 0, sizeof(int), ts);
        CUtensorMap ta, tb;
        ok = make_plane_map(&ta, sa, ntune, bt * k, lld, OM) && make_plane_map(&tb, sb, ntune, bt * k, lld, ON);
        const int smem = num_stages(k) * stage_bytes(k) + 1024 + 256;
        Epilogue ep = epilogue_plain((double*)out, (long long)ntune * ntune);
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int cands[3] = {1, 2, 4};
        for (int ci = 0; ok && ci < 3; ++ci) {
            const int cl = cands[ci];
            if (launch_f64e_cl(cl, ta, tb, ntune, k, k, k, (int*)ex, (int*)ex, bt, ep, (int*)er, ts,
                               nullptr, smem))
                continue;   // warm-up (and skip a size that cannot launch)
            cudaEventRecord(e0, ts);
            for (int rep = 0; rep < 3; ++rep)
                launch_f64e_cl(cl, ta, tb, ntune, k, k, k, (int*)ex, (int*)ex, bt, ep, (int*)er, ts,
                               nullptr, smem);
            cudaEventRecord(e1, ts);
            if (cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = cl; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaGetLastError();
    if (ts) cudaStreamSynchronize(ts);
    cudaFree(sa); cudaFree(sb); cudaFree(ex); cudaFree(out); cudaFree(er);
    if (ts) cudaStreamDestroy(ts);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    return best;
}

size_t f64e_plane_elems(int n, int batch, int k) { return (size_t)batch * k * n * low_ld(n); }

mpps_status launch_slice_rows(const double* M, long long bs, int n, int batch, int k, void* planes,
                              int* exps, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    const int lld = low_ld(n);
    if (n >= 256 && batch <= 65535) {
        // many threads per row: a row-maximum pass, then one thread per element
        k_rowexp<<<dim3((n + 7) / 8, batch), 256, 0, st>>>(M, bs, n, exps);
        MPPS_LAUNCH_CHECK();
        k_slice_rows_elem<<<dim3((n + 127) / 128, n, batch), 128, 0, st>>>(
            M, bs, n, k, exps, (__nv_bfloat16*)planes, (long long)k * n * lld, lld);
    } else {
        dim3 g((n + 7) / 8, batch);
        k_slice_rows<<<g, 256, 0, st>>>(M, bs, n, k, (__nv_bfloat16*)planes, (long long)k * n * lld,
                                        lld, exps);
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_slice_cols(const double* M, long long bs, int n, int batch, int k, void* planes,
                              int* exps, unsigned long long* colmax, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    const int lld = low_ld(n);
    MPPS_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)batch * n, st));
    k_colmax<<<dim3((n + 127) / 128, (n + 63) / 64, batch), 128, 0, st>>>(M, bs, n, colmax);
    MPPS_LAUNCH_CHECK();
    k_slice_cols<<<dim3((n + 31) / 32, (n + 31) / 32, batch), dim3(32, 8), 0, st>>>(
        M, bs, n, k, colmax, (__nv_bfloat16*)planes, (long long)k * n * lld, lld, exps);
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_gemm_f64e(int k, const void* slicesA, int ksA, const int* eA,
                             const void* slicesBt, int ksB, const int* eB, int n, int batch,
                             int nmat, const Epilogue& ep, int* d_err, cudaStream_t st,
                             const int* bidx) {
    if (batch <= 0) return MPPS_OK;
    if (k < 1 || k > MPPS_F64E_MAX_SLICES || ksA < k || ksB < k) {
        set_error("emulated FP64 product: slice count %d outside 1..%d", k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const int lld = low_ld(n);
    CUtensorMap ta, tb;
    if (!make_plane_map(&ta, slicesA, n, nmat * ksA, lld, OM) ||
        !make_plane_map(&tb, slicesBt, n, nmat * ksB, lld, ON)) {
        set_error("cuTensorMapEncodeTiled failed for slice planes (n=%d)", n);
        return MPPS_ECUDA;
    }
    const int smem = num_stages(k) * stage_bytes(k) + 1024 + 256;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    static int attr_done[64] = {0};
    if (!attr_done[dev]) {
        MPPS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f64e<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           SMEM_BUDGET + 1024 + 256));
        MPPS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f64e<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           SMEM_BUDGET + 1024 + 256));
        MPPS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f64e<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           SMEM_BUDGET + 1024 + 256));
        attr_done[dev] = 1;
    }
    const int cl = f64e_cluster_choice(dev, n, k, batch);
    ProfScope prof(MPPS_PROF_GEMM_F64E, st, 2.0 * n * (double)n * n * batch * (k * (k + 1) / 2));
    return launch_f64e_cl(cl, ta, tb, n, k, ksA, ksB, eA, eB, batch, ep, d_err, st, bidx, smem);
}

}  // namespace mpps
