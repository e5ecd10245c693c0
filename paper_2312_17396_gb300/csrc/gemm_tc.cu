// gemm_tc.cu -- low-precision Horner products P_i Y on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in TMEM, operands staged in shared memory by TMA).  These are
// the products that eq. (2.8) lets run at u_i > u: the paper's q(X) part (eq. (2.6)),
// evaluated in the format chosen per step (Section 4.1.1's ladder, GPU formats):
//   BF16    kind::f16,     1 product                        (u = 2^-8)
//   BF16X3  kind::f16,     hi*hi + hi*lo + lo*hi, one TMEM accumulator (u ~ 2^-16)
//   TF32    kind::tf32,    1 product                        (u = 2^-11)
//   FP8     kind::mxf8f6f4 with block scales (E4M3 x E4M3), 1 product   (u = 2^-4)
// all accumulated in FP32.  The epilogue reads the 128 x 128 FP32 tile out of TMEM,
// undoes the operand scales and adds B_{i-1} in FP64 (fused Horner add).
//
// FP8 products scale every 32 entries of K of each row of A and each column of B by their
// own power of two (8-bit codes, MxScales): one scale per row or column cannot hold a row
// whose entries span more than E4M3's 2^17 range, a scale per 32-entry block keeps each
// block's 3 fraction bits.  The tensor core applies the scales itself: per stage the TMA
// warp also fetches the 512-byte scale chunks of A and B, the MMA thread copies them into
// TMEM (tcgen05.cp, one TMEM region per stage) and issues the block-scaled MMAs, the
// instruction descriptor naming the block (byte) each of the four K = 32 steps reads.
//
// Structure: one CTA (8 warps) per 128 x TN output tile (TN = 64 when 128 x 128 tiles would
// leave SMs idle, else 128), K walked in 128-byte slabs (64 bf16 / 32 tf32 / 128 fp8 per
// row) through a 3-4 stage TMA ring with full/empty mbarriers.  Warp 0 lane 0 issues TMA,
// warp 1 lane 0 issues tcgen05.mma (descriptors formed once per stage); then the FP32 tile
// is staged from TMEM into the idle ring and all 8 warps run the FP64 epilogue over it in
// row-major order (coalesced power-table reads and stores, four elements in flight per
// thread).  Both operands are K-major with the 128-byte swizzle.  Every mbarrier wait is
// bounded (about 2 s of %globaltimer); on expiry the kernel sets *err, skips further
// waits, lets the copies in flight land and exits normally.
#include "common.cuh"
#include "tcgen05.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace mpps {

namespace {

using namespace tc;

constexpr int TM = 128;                   // output rows per CTA (TN, the columns, is 64 or 128)
constexpr int SLAB = 128;                 // bytes of K per smem row
constexpr int TILE_BYTES = TM * SLAB;     // 16 KB slot per operand slab (B uses TN rows of it)
template <int FMT>
struct Tc;
template <>
struct Tc<MPPS_FMT_BF16> {
    static constexpr int kOps = 2, kStages = 4, kAB = 1;
};
template <>
struct Tc<MPPS_FMT_BF16X3> {
    static constexpr int kOps = 4, kStages = 3, kAB = 1;
};
template <>
struct Tc<MPPS_FMT_TF32> {
    static constexpr int kOps = 2, kStages = 4, kAB = 2;
};
template <>
struct Tc<MPPS_FMT_FP8> {   // block-scaled only (make_idesc_mx)
    static constexpr int kOps = 2, kStages = 4;
};

template <int FMT, int TN>
__host__ __device__ constexpr uint32_t instr_desc() {
    // D format F32 (bit 4), A/B formats (bits 7-9, 10-12), K-major A and B, N>>3 at
    // bit 17, M>>4 at bit 24.
    return (1u << 4) | ((uint32_t)Tc<FMT>::kAB << 7) | ((uint32_t)Tc<FMT>::kAB << 10) |
           ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

template <int FMT, int TN>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    constexpr uint32_t id = instr_desc<FMT, TN>();
    if constexpr (FMT == MPPS_FMT_TF32) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    }
}

constexpr int MX_CHUNK = 512;              // bytes of scale codes per operand and stage

template <int FMT, bool MX>
__host__ __device__ constexpr int smem_bytes() {
    return Tc<FMT>::kStages * (Tc<FMT>::kOps * TILE_BYTES + (MX ? 2 * MX_CHUNK : 0)) + 1024 + 256;
}

constexpr int TC_THREADS = 512;           // 16 warps: all of them run the epilogue
constexpr int TC_COLGROUPS = TC_THREADS / 128;   // warps per TMEM lane quarter

template <int FMT, int TN, bool MX>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
              int n, Epilogue ep, MxScales mx, int* err) {
    static_assert(!MX || (FMT == MPPS_FMT_FP8 && TN == 64), "block scales: FP8, 128 x 64 tiles");
    constexpr int OPS = Tc<FMT>::kOps, STAGES = Tc<FMT>::kStages;
    constexpr int STAGE_BYTES = OPS * TILE_BYTES + (MX ? 2 * MX_CHUNK : 0);
    // TMEM: the accumulator (TN columns), then for block scales 8 columns per stage (4 for
    // A's codes, 4 for B's)
    constexpr uint32_t TMEM_COLS = MX ? 128 : TN;
    static_assert(!MX || TN + 8 * STAGES <= 128, "scale regions exceed the TMEM allocation");
    constexpr int ESIZE = (FMT == MPPS_FMT_TF32) ? 4 : (FMT == MPPS_FMT_FP8 ? 1 : 2);
    constexpr int KSLAB = SLAB / ESIZE;   // K elements per stage

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.z, m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int nk = (n + KSLAB - 1) / KSLAB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();   // barrier init, TMEM allocation and tensor-map prefetch overlap the previous kernel
    pdl_trigger();
    if (ep.dcount && b >= __ldg(ep.dcount)) {   // not this launch's matrix (device plan)
        tc_fence_before();
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
        return;
    }

    if (warp == 0 && lane == 0) {
        // TMA producer
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, err)) break;
            mbar_expect_tx(&full[s], (OPS / 2) * (TM + TN) * SLAB + (MX ? 2 * MX_CHUNK : 0));
            uint8_t* st = smem + s * STAGE_BYTES;
            const int kc = kb * KSLAB;
            tma_load_3d(st, &tmA, kc, m0, b, &full[s]);
            tma_load_3d(st + TILE_BYTES, &tmB, kc, n0, b, &full[s]);
            if constexpr (MX) {   // this stage's scale chunks: rows m0.., columns n0.., K block kb
                bulk_load(st + OPS * TILE_BYTES,
                          mx.a + b * mx.a_bs + ((long long)(m0 / TM) * mx.kc + kb) * MX_CHUNK,
                          MX_CHUNK, &full[s]);
                bulk_load(st + OPS * TILE_BYTES + MX_CHUNK,
                          mx.b + b * mx.b_bs + ((long long)(n0 / TN) * mx.kc + kb) * MX_CHUNK,
                          MX_CHUNK, &full[s]);
            }
            if constexpr (OPS == 4) {
                tma_load_3d(st + 2 * TILE_BYTES, &tmA2, kc, m0, b, &full[s]);
                tma_load_3d(st + 3 * TILE_BYTES, &tmB2, kc, n0, b, &full[s]);
            }
        }
        // the copies of the last stages land before the ring is reused or the CTA exits
        // (returns at once unless a wait above gave up)
        bool landed = true;
        for (int k2 = kb > STAGES ? kb - STAGES : 0; k2 < kb && landed; ++k2)
            landed = mbar_wait_quiet(&full[k2 % STAGES], (k2 / STAGES) & 1);
        if (!landed) atomicExch(err, 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: 4 instructions per 128-byte slab (K advance of 32 bytes each)
        bool ok = true;
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % STAGES;
            ok = mbar_wait(&full[s], (kb / STAGES) & 1, err);
            if (!ok) break;
            tc_fence_after();
            // descriptors of this stage; the K advance of 32 bytes is +2 in the address field
            const uint64_t da = sw128_desc(smem_u32(smem + s * STAGE_BYTES));
            const uint64_t db = da + (uint64_t)(TILE_BYTES >> 4);
            uint32_t sfa = 0, sfb = 0;
            if constexpr (MX) {   // scale codes into this stage's TMEM columns
                sfa = tmem + (uint32_t)(TN + 8 * s);
                sfb = sfa + 4;
                const uint32_t ss = smem_u32(smem + s * STAGE_BYTES + OPS * TILE_BYTES);
                tmem_cp_32x128b_x4(sfa, plain16_desc(ss));
                tmem_cp_32x128b_x4(sfb, plain16_desc(ss + MX_CHUNK));
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = da + (uint64_t)(2 * kk), bd = db + (uint64_t)(2 * kk);
                if constexpr (MX)
                    mma_mxf8(tmem, ad, bd, make_idesc_mx(TM, TN, kk, kk), sfa, sfb,
                             (kb | kk) != 0 ? 1u : 0u);
                else
                    tc_mma<FMT, TN>(tmem, ad, bd, (kb | kk) != 0 ? 1u : 0u);
                if constexpr (OPS == 4) {
                    const uint64_t ad2 = da + (uint64_t)((2 * TILE_BYTES >> 4) + 2 * kk);
                    const uint64_t bd2 = da + (uint64_t)((3 * TILE_BYTES >> 4) + 2 * kk);
                    tc_mma<FMT, TN>(tmem, ad, bd2, 1u);   // hi * lo
                    tc_mma<FMT, TN>(tmem, ad2, bd, 1u);   // lo * hi
                }
            }
            tc_commit(&empty[s]);
        }
        tc_commit(done);
    }
    __syncwarp();

    mbar_wait(done, 0, err);
    tc_fence_after();

    // Epilogue: the FP32 tile goes from TMEM to shared memory (the ring is idle now; warps w,
    // w + 4, w + 8, w + 12 share TMEM lanes 32 (w % 4).. and split the columns), then all 512
    // threads walk it row-major, four consecutive columns each, so that the reads of the power
    // table and the stores are coalesced along rows: the FP64 block sums of the fused Horner
    // add are latency-bound, and 16 warps hide twice as much as 8.
    constexpr int PITCH = TN + 1;
    float* stile = (float*)smem;
    {
        const int q4 = warp & 3, h = warp >> 2;
        const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
        const int row = q4 * 32 + lane;
#pragma unroll
        for (int c0 = 32 * h; c0 < TN; c0 += 32 * TC_COLGROUPS) {
            uint32_t v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) stile[row * PITCH + c0 + j] = __uint_as_float(v[j]);
        }
    }
    __syncthreads();
    // four consecutive columns per thread: the power-table and addend rows are read two
    // doubles at a time where they are 16-byte aligned
    const bool vep = (n & 3) == 0 && ((((uintptr_t)ep.pw | (uintptr_t)ep.add) & 15) == 0) &&
                     ((ep.pw_bstride | ep.add_bstride) & 1) == 0;
#pragma unroll 1
    for (int e0 = 4 * threadIdx.x; e0 < TM * TN; e0 += 4 * TC_THREADS) {
        const int r = e0 / TN, c = e0 % TN, row = m0 + r, col = n0 + c;
        if (row >= n) continue;
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = f32_to_f64(stile[r * PITCH + c + u]);
        if (vep && col + 3 < n) {
            epilogue_value4(ep, b, row, col, n, v);
#pragma unroll
            for (int u = 0; u < 4; ++u) epilogue_store(ep, b, row, col + u, n, v[u]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (col + u < n)
                    epilogue_store(ep, b, row, col + u, n, epilogue_value(ep, b, row, col + u, n, v[u]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- host side ----------------------------------------------------------------------
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

// 3-D map over (K = n columns, n rows, batch) of a row-major low-precision copy with
// leading dimension lld and batch stride bs (elements); box = one 128-byte slab x 128 rows.
bool make_map(CUtensorMap* tm, int fmt, const void* ptr, int n, int batch, int lld, long long bs,
              int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int es = low_elem_bytes(fmt);
    CUtensorMapDataType dt = fmt == MPPS_FMT_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : fmt == MPPS_FMT_FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)lld * es, (cuuint64_t)bs * es};
    cuuint32_t box[3] = {(cuuint32_t)(SLAB / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(tm, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int FMT, int TN, bool MX = false>
mpps_status launch_fmt(const void* A_hi, const void* A_lo, const void* Bt_hi, const void* Bt_lo,
                       long long a_bs, long long b_bs, int lld, int n, int batch, const Epilogue& ep,
                       int* d_err, cudaStream_t st, MxScales mx = MxScales{}) {
    CUtensorMap ta, tb, ta2, tb2;
    bool ok = make_map(&ta, FMT, A_hi, n, batch, lld, a_bs, TM) &&
              make_map(&tb, FMT, Bt_hi, n, batch, lld, b_bs, TN);
    if (FMT == MPPS_FMT_BF16X3)
        ok = ok && make_map(&ta2, FMT, A_lo, n, batch, lld, a_bs, TM) &&
             make_map(&tb2, FMT, Bt_lo, n, batch, lld, b_bs, TN);
    else {
        ta2 = ta;
        tb2 = tb;
    }
    if (!ok) {
        set_error("cuTensorMapEncodeTiled failed (n=%d, lld=%d)", n, lld);
        return MPPS_ECUDA;
    }
    constexpr int smem = smem_bytes<FMT, MX>();
    // the attribute is a property of the kernel on the current device: set once per device
    static std::mutex attr_mu;
    static bool attr_set[64] = {false};
    {
        int dev = 0;
        MPPS_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) {
            set_error("device index %d out of range", dev);
            return MPPS_ENOTSUP;
        }
        std::lock_guard<std::mutex> lk(attr_mu);
        if (!attr_set[dev]) {
            MPPS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<FMT, TN, MX>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            attr_set[dev] = true;
        }
    }
    dim3 grid((n + TN - 1) / TN, (n + TM - 1) / TM, batch);
    ProfScope prof(MPPS_PROF_GEMM_TC, st,
                   2.0 * n * (double)n * n * batch * (FMT == MPPS_FMT_BF16X3 ? 3 : 1));
    MPPS_CUDA_TRY(launch_pdl(k_gemm_tc<FMT, TN, MX>, dim3(grid), dim3(TC_THREADS), smem, st, ta, tb, ta2, tb2, n, ep, mx, d_err));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t fp8mx_ws_bytes(int n, int batch) {
    const size_t nb = (size_t)batch * n;
    return 2 * al256(nb * low_ld(n)) + al256((size_t)batch * mx_scale_bytes_a(n)) +
           al256((size_t)batch * mx_scale_bytes_b(n)) + 2 * al256(sizeof(int) * nb) +
           al256(sizeof(unsigned long long) * nb);
}

Fp8MxWs fp8mx_ws_carve(void* base, int n, int batch) {
    const size_t nb = (size_t)batch * n;
    uint8_t* p = (uint8_t*)base;
    Fp8MxWs w;
    w.qa = p; p += al256(nb * low_ld(n));
    w.qb = p; p += al256(nb * low_ld(n));
    w.sfa = p; p += al256((size_t)batch * mx_scale_bytes_a(n));
    w.sfb = p; p += al256((size_t)batch * mx_scale_bytes_b(n));
    w.ea = (int*)p; p += al256(sizeof(int) * nb);
    w.eb = (int*)p; p += al256(sizeof(int) * nb);
    w.cmax = (unsigned long long*)p;
    return w;
}

mpps_status launch_product_fp8mx(const double* A, long long a_bs, const double* B, long long b_bs,
                                 int n, int batch, Epilogue ep, const Fp8MxWs& w, int* d_err,
                                 cudaStream_t st) {
    const int lld = low_ld(n);
    const long long q_bs = (long long)n * lld;
    mpps_status rc = launch_convert_mx(A, a_bs, n, batch, w.qa, q_bs, lld, w.sfa, mx_scale_bytes_a(n),
                                       false, w.ea, nullptr, st);
    if (!rc)
        rc = launch_convert_mx(B, b_bs, n, batch, w.qb, q_bs, lld, w.sfb, mx_scale_bytes_b(n), true,
                               w.eb, w.cmax, st);
    if (rc) return rc;
    ep.row_exp = w.ea;
    ep.col_exp = w.eb;
    const MxScales mx{w.sfa, w.sfb, mx_scale_bytes_a(n), mx_scale_bytes_b(n), (n + 127) / 128};
    return launch_gemm_tc(MPPS_FMT_FP8, w.qa, nullptr, w.qb, nullptr, q_bs, q_bs, lld, n, batch, ep,
                          d_err, st, &mx);
}

mpps_status launch_gemm_tc(int fmt, const void* A_hi, const void* A_lo, const void* Bt_hi,
                           const void* Bt_lo, long long a_bs, long long b_bs, int lld, int n,
                           int batch, const Epilogue& ep, int* d_err, cudaStream_t st,
                           const MxScales* mx) {
    if (fmt == MPPS_FMT_FP8) {   // block-scaled, 128 x 64 tiles (the scale chunks' width)
        if (!mx || !mx->a || !mx->b || mx->kc != (n + 127) / 128) {
            set_error("launch_gemm_tc: an FP8 product needs its block scales");
            return MPPS_EINVAL;
        }
        return launch_fmt<MPPS_FMT_FP8, 64, true>(A_hi, A_lo, Bt_hi, Bt_lo, a_bs, b_bs, lld, n, batch,
                                                  ep, d_err, st, *mx);
    }
    // 128 x 64 tiles when 128 x 128 ones would not give every SM two CTAs: the epilogue (FP64
    // block sums) then spreads over twice as many SMs
    const long long tiles128 = (long long)((n + 127) / 128) * ((n + 127) / 128) * batch;
    const bool narrow = tiles128 < 2 * 148;
    // candidate 0: 128 x 64 tiles, 1: 128 x 128 (the rule above, or the tuned choice)
    auto run = [&](int c) -> mpps_status {
#define MPPS_TC_CASE(F)                                                                         \
    case F:                                                                                     \
        return c == 0 ? launch_fmt<F, 64>(A_hi, A_lo, Bt_hi, Bt_lo, a_bs, b_bs, lld, n, batch, ep, \
                                          d_err, st)                                            \
                      : launch_fmt<F, 128>(A_hi, A_lo, Bt_hi, Bt_lo, a_bs, b_bs, lld, n, batch, ep, \
                                           d_err, st);
        switch (fmt) {
            MPPS_TC_CASE(MPPS_FMT_BF16)
            MPPS_TC_CASE(MPPS_FMT_BF16X3)
            MPPS_TC_CASE(MPPS_FMT_TF32)
#undef MPPS_TC_CASE
            default:
                set_error("launch_gemm_tc: unsupported format %d", fmt);
                return MPPS_EINVAL;
        }
    };
    const int tuned = tune_lookup(TUNE_TC_WIDTH, n, batch, fmt);
    const bool inplace = ep.add != nullptr && ep.add == ep.out;   // a re-run would add twice
    if (tuned < 0 && !inplace && !ep.dcount && tune_enabled())   // gated launches: no tuning
        return tune_run(TUNE_TC_WIDTH, n, batch, fmt, 2, st, run);
    return run(tuned >= 0 ? tuned : (narrow ? 0 : 1));
}

}  // namespace mpps
