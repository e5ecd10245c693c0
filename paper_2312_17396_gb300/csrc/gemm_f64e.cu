// gemm_f64e.cu -- FP64-accurate matrix product on the BF16 tensor cores by exact slice
// products (the splitting method of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59 (2012), adapted to tcgen05 with FP32 accumulation).
//
// On GB300 the FP64 pipe delivers about 1 TFLOP/s while BF16 tensor cores deliver about
// 1900, so the working-precision products of the PS evaluation (powers, early Horner steps,
// squarings) are emulated:
//
//   A (rows scaled by 2^-eA_i, |.| < 1) = sum_{t<k} 2^{-7(t+1)} a_t,  a_t integers, |a_t| <= 128
//   B (cols scaled by 2^-eB_j)          = sum_{q<k} 2^{-7(q+1)} b_q
//   A B ~= 2^{eA_i + eB_j - 14} sum_{d<k} 2^{-7d} D_d,   D_d = sum_{t+q=d} a_t b_q^T.
//
// The digits are balanced base 128 (|a_0| <= 128, |a_t| <= 64 for t >= 1), exact in bf16.
// The slice planes hold a'_t = 2^-7t a_t and b'_q = 2^-7q b_q, so that the product
// a'_t b'_q^T is already 2^-7d a_t b_q^T and pairs of different d may share an accumulator.
// Every D_d entry of one K chunk of at most 512 is an integer of magnitude <= 512 (d+3) 2^12
// <= 2^24 for d <= 5, so the tensor cores accumulate D_0..D_5 EXACTLY in FP32, each in its
// own TMEM region; d = 6 and d = 7 (weights <= 2^-42 relative to D_0) have a region each and
// accumulate in FP32 with rounding, far below an FP64 product's own error.  With k = 8 the
// only other errors are the pairs dropped (t + q >= 8) and the 8-digit residual: about
// 2^{-54} of the row and column maxima, FP64-level accuracy with 36 bf16 products.
//
// At the end of every K chunk the exact regions are drained on the integer pipe
// (W = sum_{d<=5} 2^{7(5-d)} D_d as a 64-bit integer, the tails as FP32); with more than one
// chunk, each chunk's W is added to an FP64 accumulator, so W never overflows.  The FP64
// pipe only adds and does the fused epilogue: product = 2^{e-49} W + 2^{e-14} T.
//
// Slice layouts.  A (row slices): slices 2p and 2p+1 of a row share row r of "pair" p,
// alternating 32-element K blocks, [pair][row][K block][slice 2p | slice 2p+1][32], so one TMA
// box row carries 128 bytes (the copy engine's rate grows with the row length: about 150 GB/s
// per SM for 128-byte rows against 96 for 64-byte ones) and lands in the 128-byte swizzle,
// where slice 2p+1 is the same tile read 64 bytes further along K.  B^T (column slices):
// plane q is [row][K] on its own ([plane][row][K]), 64-byte swizzle, so that the planes of
// one tile stack along N.
//
// Kernel: persistent, one CTA per SM, 128 x 64 output tiles, 18 warps (0-15 epilogue: TMEM
// lane quarter = warp % 4, 16-column group = warp / 4; 16 TMA producer; 17 MMA issuer).  Per
// K block of 32 the producer loads the pairs of the A tile (one box each) and the k planes of
// the B^T tile (one 3-D box) on one mbarrier.  The MMA of slice t uses the stacked B operand
// b'_0..b'_{7-t} (N = 64 (8 - t)) and writes regions t..7 in one instruction (two when
// N > 256); with k = 8 that covers all 36 pairs in 12 instructions per K step.  The epilogue
// drains TMEM into registers and releases it at once, so the FP64 epilogue of a tile overlaps
// the MMAs of the next.  All mbarrier waits are bounded.
#include "common.cuh"
#include "tcgen05.cuh"

#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

namespace mpps {

namespace {

using namespace tc;

constexpr int OM = 128;                 // output rows per tile (TMEM lanes)
constexpr int ON = 64;                  // output cols per tile (= columns per TMEM region)
constexpr int KB = 32;                  // K elements per stage (64 bytes of bf16: two MMA steps)
constexpr int KCHUNK = 512;             // exact FP32 accumulation bound of D_0..D_5 (see above)
constexpr int DIGIT = 7;                // bits per slice
constexpr int FLUSH = 8;                // chunks the 64-bit W may sum before an FP64 flush
constexpr int NEXACT = 6;               // diagonals accumulated exactly
constexpr int NREG = 8;                 // TMEM regions: D_0..D_5, d = 6, and d = 7
constexpr int A_PAIR = OM * 4 * KB;     // 16 KB: a pair of A slices, 128-byte rows
constexpr int B_TILE = ON * 2 * KB;     // 4 KB: one B plane, 64-byte rows
constexpr int EPI_WARPS = 16;            // 4 per TMEM lane quarter, 16 columns each
constexpr int EPI_COLS = ON / (EPI_WARPS / 4);
constexpr int THREADS = (EPI_WARPS + 2) * 32;
static_assert(EPI_COLS == 16, "the drain loads 16 TMEM columns per thread");
constexpr int MAX_STAGES = 8;
constexpr int NFULL = MAX_STAGES;       // one fill barrier per stage
constexpr int BAR_BYTES = 1024;
constexpr int SMEM_MAX = 232448;        // 227 KB of opt-in dynamic shared memory
constexpr int SMEM_BUDGET = SMEM_MAX - 1024 - BAR_BYTES;
constexpr int RASTER_G = 8;             // row blocks per raster group (L2 reuse of B)
// barrier block after the ring: full[MAX_STAGES] | empty[MAX_STAGES] | chunk_done |
// tmem_free | mma_done | TMEM address slot
static_assert((NFULL + MAX_STAGES + 3) * 8 + 4 <= BAR_BYTES, "barrier block exceeds its bytes");
static_assert(NREG * ON <= 512, "TMEM regions exceed 512 columns");
constexpr int MAX_PLANES = 8;           // slices per operand (F64E(9) adds pairs, not slices)
static_assert(MAX_PLANES <= NREG, "every slice must start a TMEM region");
static_assert(55 - DIGIT * (MAX_PLANES - 1) >= 1, "the last digit needs a rounding bit");

__host__ __device__ constexpr int num_pairs(int k) { return (k + 1) / 2; }
__host__ __device__ constexpr int stage_bytes(int k) { return num_pairs(k) * A_PAIR + k * B_TILE; }
__host__ __device__ constexpr int num_stages(int k) {
    int s = SMEM_BUDGET / stage_bytes(k);
    return s > MAX_STAGES ? MAX_STAGES : s;
}
__host__ __device__ constexpr uint32_t tmem_cols(int nreg) {
    uint32_t need = (uint32_t)(ON * nreg), c = 32;
    while (c < need) c <<= 1;
    return c;
}

// round_half_even(x 2^(62-e)) for |x| < 2^e (so the result is below 2^62 in magnitude),
// computed from the bit fields of x on the integer pipe: equal to rounding the exact
// product x 2^(62-e) to the nearest integer, ties to even.  Non-finite x gives 0.
__device__ __forceinline__ long long scaled_int(double x, int e) {
    const long long bits = __double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7FF);
    if (ef == 0x7FF) return 0;
    long long m = bits & 0xFFFFFFFFFFFFFLL;
    int E = -1074;                                   // x = m 2^E
    if (ef != 0) { m |= 1LL << 52; E = ef - 1075; }
    const int sh = E + 62 - e;
    long long F;
    if (sh >= 0) {
        F = m << sh;                                 // exact: m 2^sh < 2^62
    } else if (sh < -53) {
        F = 0;                                       // m 2^sh < 1/2
    } else {
        const int k = -sh;
        const long long q = m >> k, r = m & ((1LL << k) - 1), half = 1LL << (k - 1);
        F = q + ((r > half || (r == half && (q & 1))) ? 1 : 0);
    }
    return bits < 0 ? -F : F;
}

// The same value through the FP64 pipe, which the slicing kernels otherwise leave idle: x 2^(62-e)
// is formed exactly by moving the exponent field, and the conversion instruction rounds it to
// the nearest integer, ties to even.  Zero, subnormal and non-finite x, and products below
// the normal range, take the integer path above.
__device__ __noinline__ long long scaled_int_slow(double x, int e) { return scaled_int(x, e); }
__device__ __forceinline__ long long scaled_int_fp64(double x, int e) {
    const long long bits = __double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7ff);
    if (ef != 0 && ef != 0x7ff && ef + 62 - e > 0)
        return __double2ll_rn(__longlong_as_double(bits + ((long long)(62 - e) << 52)));
    return scaled_int_slow(x, e);
}

// Signed base-128 digits of x / 2^e (|x| < 2^e), in offset form: with F = round(x 2^(62-e))
// (|F| < 2^62), p_t = 55 - 7t and G = F + 2^(p_{k-1} - 1) + sum_{t=1}^{k-1} 64 2^(p_t),
//   v_0 = floor(G / 2^55),   v_t = ((G >> p_t) mod 128) - 64   (t >= 1),
// so that F = sum_t v_t 2^(p_t) + r with |r| <= 2^(p_{k-1} - 1): x = 2^e (sum_t v_t 2^(-7(t+1))
// + r 2^-62), |r 2^-62| <= 2^(-7k-1); |v_0| <= 128, -64 <= v_t <= 63.  Every digit comes from G
// alone (no chain through a remainder).  Plane t stores v_t 2^-7t, exact in bf16 (at most 8
// significant bits, so the bf16 is the upper half of the FP32 value; (float)v is formed by
// adding v to the bit pattern of 1.5 2^23).  No FP64 arithmetic: the integer and FP32
// pipes do all of it.  k <= 8 keeps p_{k-1} >= 6.
__host__ __device__ inline long long digit_offset(int k) {
    long long o = 1LL << (55 - DIGIT * (k - 1) - 1);
    for (int t = 1; t < k; ++t) o += 64LL << (55 - DIGIT * t);
    return o;
}

// bf16 bits of digit t of G (see above).
// FP32 bit pattern of v_t 2^-7t (its low 16 bits are zero: the value is exact in bf16).
// M_t = 1.5 2^(23-7t) has an ulp of 2^-7t, so the float whose bits are bits(M_t) + v_t is
// M_t + v_t 2^-7t, and subtracting M_t leaves v_t 2^-7t exactly: one integer add and one
// FP32 subtraction per digit (t is a compile-time constant in every caller).
__device__ __forceinline__ unsigned digit_f32(long long G, int t) {
    const int v = t == 0 ? (int)(G >> 55) : (int)((G >> (55 - DIGIT * t)) & 127) - 64;
    const unsigned mb = 0x4B400000u - ((unsigned)(DIGIT * t) << 23);
    return __float_as_uint(__uint_as_float(mb + (unsigned)v) - __uint_as_float(mb));
}
// bf16 bits of digit t of G (see above).
__device__ __forceinline__ unsigned digit_bits(long long G, int t) { return digit_f32(G, t) >> 16; }
// Two digits' bf16 bits packed in one word (a in the low half): the upper halves of the two
// FP32 patterns, one byte permutation.
__device__ __forceinline__ unsigned digit_pair(long long Ga, long long Gb, int t) {
    return __byte_perm(digit_f32(Ga, t), digit_f32(Gb, t), 0x7632);
}

// Pair layout (see the top of the file): K index j of a row sits at kpos(j) in its pair row,
// slice t at slice_off(t) from its pair's origin; pstride = n 2 lld elements per pair.
__device__ __forceinline__ long long kpos(int j) { return (long long)j + (j & ~(KB - 1)); }
__device__ __forceinline__ long long slice_off(int t, long long pstride) {
    return (long long)(t >> 1) * pstride + (t & 1) * KB;
}

// The KS digits of x (dst = the row's origin + kpos(j)); x = 0 gives KS zero digits.  The
// slice count is a template parameter in every slicing kernel: with the digit positions
// known at compile time each digit is a constant shift and mask of G.
template <int KS>
__device__ __forceinline__ void put_digits(double x, int e, long long goff, __nv_bfloat16* dst,
                                           long long pstride) {
    const long long G = scaled_int_fp64(x, e) + goff;
#pragma unroll
    for (int t = 0; t < KS; ++t)
        dst[slice_off(t, pstride)] = __ushort_as_bfloat16((unsigned short)digit_bits(G, t));
}

// |x| as the bit pattern of a non-negative double, infinity for a NaN: the maximum of these
// bit patterns is the bit pattern of the maximum magnitude, infinity when any entry is not
// finite.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    return a > 0x7ff0000000000000ULL ? 0x7ff0000000000000ULL : a;
}

// Exponent recorded for a row or column with a non-finite entry.  Its digits are all zero
// (scaled_int turns every entry into 0 at this exponent) and the epilogue writes NaN for
// every product entry that involves it, as the FP64 product would have (up to inf vs NaN).
constexpr int kNonFinite = 1 << 29;
constexpr int kExpLimit = 1 << 20;   // e_A + e_B at or above it: a non-finite row or column

// The frexp exponent e of a non-negative double given by its bits (value in [2^(e-1), 2^e));
// 0 for zero, kNonFinite for infinity.  Integer pipe only.
__device__ __forceinline__ int exp_above(unsigned long long a) {
    const int ef = (int)(a >> 52);
    if (a == 0) return 0;
    if (ef == 0x7ff) return kNonFinite;
    return ef != 0 ? ef - 1022 : (64 - __clzll((long long)a)) - 1074;
}

__device__ __forceinline__ unsigned long long max_bits(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Exponent code of |x| recorded by the epilogues (Epilogue::rmax / cmax): 0 for zero,
// 2048 + exp_above(|x|) otherwise (always positive: exp_above >= -1073), kNonFinite + 2048
// for a NaN or infinity; and its inverse for the slicers.
constexpr int kExpCodeBias = 2048;
__device__ __forceinline__ int exp_code(double x) {
    const unsigned long long a = abs_bits(x);
    return a == 0 ? 0 : exp_above(a) + kExpCodeBias;
}
__device__ __forceinline__ int exp_from_code(int c) { return c == 0 ? 0 : c - kExpCodeBias; }

// Row slices (A operand) for short rows (n < 256): one warp per row; e_i from the row
// maximum.
template <int KS>
__global__ void k_slice_rows(const double* __restrict__ M, long long bs, int n, long long goff, __nv_bfloat16* __restrict__ planes,
                             long long plane_bs, int lld, int* __restrict__ exps,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.y >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp, b = blockIdx.y;
    if (row >= n) return;
    const double* src = M + (long long)b * bs + (long long)row * n;
    unsigned long long mx = 0;
    for (int j = lane; j < n; j += 32) mx = max_bits(mx, abs_bits(src[j]));
    for (int o = 16; o > 0; o >>= 1) mx = max_bits(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exp_above(mx);
    if (lane == 0) exps[(long long)b * n + row] = e;
    __nv_bfloat16* dst = planes + (long long)b * plane_bs + (long long)row * 2 * lld;
    const long long pstride = (long long)n * 2 * lld;
    const int n32 = (n + KB - 1) / KB * KB;   // the K tail up to n32 is written as zeros
    for (int j = lane; j < n32; j += 32) put_digits<KS>(j < n ? src[j] : 0.0, e, goff, dst + kpos(j), pstride);
}

// Row slices for rows of up to 256 VPT elements: one 256-thread block per row holds the row
// in registers (VPT values per thread), reduces its maximum (as the bit pattern of a
// non-negative double) and writes the k planes: the row is read once.
template <int KS, int VPT>
__global__ void __launch_bounds__(256) k_slice_rows_blk(const double* __restrict__ M, long long bs,
                                                        int n, long long goff,
                                                        __nv_bfloat16* __restrict__ planes,
                                                        long long plane_bs, int lld,
                                                        int* __restrict__ exps,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.y >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    __shared__ unsigned long long red[8];
    const int row = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const double* src = M + (long long)b * bs + (long long)row * n;
    double v[VPT];
    unsigned long long mx = 0;
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
        const int j = tid + 256 * i;
        v[i] = j < n ? src[j] : 0.0;
        mx = max_bits(mx, abs_bits(v[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = red[w] > mx ? red[w] : mx;
    const int e = exp_above(mx);
    if (tid == 0) exps[(long long)b * n + row] = e;
    __nv_bfloat16* dst = planes + (long long)b * plane_bs + (long long)row * 2 * lld;
    const long long pstride = (long long)n * 2 * lld;
    const int n32 = (n + KB - 1) / KB * KB;   // v = 0 on the K tail n..n32-1
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
        const int j = tid + 256 * i;
        if (j < n32) put_digits<KS>(v[i], e, goff, dst + kpos(j), pstride);
    }
}

// The same with four consecutive columns per thread (n a multiple of 4): two 16-byte loads
// and one 8-byte store per plane for each group.  NG groups per thread, n <= 1024 NG.
template <int KS, int NG>
__global__ void __launch_bounds__(256) k_slice_rows_blk4(const double* __restrict__ M, long long bs,
                                                         int n, long long goff,
                                                         __nv_bfloat16* __restrict__ planes,
                                                         long long plane_bs, int lld,
                                                         int* __restrict__ exps,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.y >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    __shared__ unsigned long long red[8];
    const int row = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const double* src = M + (long long)b * bs + (long long)row * n;
    double v[NG][4];
    unsigned long long mx = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int j = 4 * (tid + 256 * g);
        if (j < n) {
            const double2 a = *reinterpret_cast<const double2*>(src + j);
            const double2 c = *reinterpret_cast<const double2*>(src + j + 2);
            v[g][0] = a.x; v[g][1] = a.y; v[g][2] = c.x; v[g][3] = c.y;
        } else {
            v[g][0] = v[g][1] = v[g][2] = v[g][3] = 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            mx = max_bits(mx, abs_bits(v[g][u]));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = red[w] > mx ? red[w] : mx;
    const int e = exp_above(mx);
    if (tid == 0) exps[(long long)b * n + row] = e;
    __nv_bfloat16* dst = planes + (long long)b * plane_bs + (long long)row * 2 * lld;
    const long long pstride = (long long)n * 2 * lld;
    const int n32 = (n + KB - 1) / KB * KB;   // v = 0 on the K tail n..n32-1
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int j = 4 * (tid + 256 * g);
        if (j >= n32) continue;
        long long G[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) G[u] = scaled_int_fp64(v[g][u], e) + goff;
#pragma unroll
        for (int t = 0; t < KS; ++t) {
            uint2 w;
            w.x = digit_pair(G[0], G[1], t);
            w.y = digit_pair(G[2], G[3], t);
            *reinterpret_cast<uint2*>(dst + slice_off(t, pstride) + kpos(j)) = w;
        }
    }
}

// Row slices with the row maxima already known (recorded by the epilogue of the product that
// wrote M): a streaming pass with no reduction.  V consecutive columns per thread (V = 4:
// n a multiple of 4, 16-byte aligned rows); a 256-thread block covers 256 / TPR rows of TPR
// threads each (TPR = the threads a row needs, a power of two up to 256), grid (column
// groups, row groups, matrices); the K tail up to round_up(n, KB) is written as zeros.
// Column group 0 also writes the row's exponent and zeroes the row's entry of rclear (the
// maxima buffer the next product fills).
template <int KS, int V>
__global__ void __launch_bounds__(256) k_slice_rows_pre(const double* __restrict__ M, long long bs, int n,
                                                        long long goff,
                                                        const int* __restrict__ rmax,
                                                        int* __restrict__ rclear,
                                                        __nv_bfloat16* __restrict__ planes,
                                                        long long plane_bs, int lld,
                                                        int* __restrict__ exps,
        const int* __restrict__ gate, const int* __restrict__ bidx) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    const int b = bidx ? __ldg(bidx + blockIdx.z) : (int)blockIdx.z;   // listed matrices only
    const int n32 = (n + KB - 1) / KB * KB;
    const long long pstride = (long long)n * 2 * lld;
    int tpr = 1;   // threads per row: a power of two covering n32 / V columns, at most 256
    while (tpr < 256 && tpr * V < n32) tpr <<= 1;
    const int rpb = 256 / tpr, sub = threadIdx.x / tpr, lt = threadIdx.x % tpr;
    for (int row = blockIdx.y * rpb + sub; row < n; row += gridDim.y * rpb) {
        const long long ri = (long long)b * n + row;
        const int e = exp_from_code(rmax[ri]);
        const int j = V * (blockIdx.x * tpr + lt);
        if (j == 0) {
            exps[ri] = e;
            if (rclear) rclear[ri] = 0;
        }
        if (j >= n32) continue;
        const double* src = M + (long long)b * bs + (long long)row * n + j;
        __nv_bfloat16* dst = planes + (long long)b * plane_bs + (long long)row * 2 * lld + kpos(j);
        if constexpr (V == 4) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            if (j < n) {
                const double2 a = __ldg(reinterpret_cast<const double2*>(src));
                const double2 c = __ldg(reinterpret_cast<const double2*>(src + 2));
                v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
            }
            long long G[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) G[u] = scaled_int_fp64(v[u], e) + goff;
#pragma unroll
            for (int t = 0; t < KS; ++t) {
                uint2 w;
                w.x = digit_pair(G[0], G[1], t);
                w.y = digit_pair(G[2], G[3], t);
                *reinterpret_cast<uint2*>(dst + slice_off(t, pstride)) = w;
            }
        } else {
            put_digits<KS>(j < n ? __ldg(src) : 0.0, e, goff, dst, pstride);
        }
    }
}

// Row maxima of |M| -> exponents e_i (one warp per row), for rows too long for the above.
__global__ void k_rowexp(const double* __restrict__ M, long long bs, int n, int* __restrict__ exps,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.y >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp, b = blockIdx.y;
    if (row >= n) return;
    const double* src = M + (long long)b * bs + (long long)row * n;
    unsigned long long mx = 0;
    for (int j = lane; j < n; j += 32) mx = max_bits(mx, abs_bits(src[j]));
    for (int o = 16; o > 0; o >>= 1) mx = max_bits(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) exps[(long long)b * n + row] = exp_above(mx);
}

// Row slices, one thread per element (the exponents come from k_rowexp).
template <int KS>
__global__ void k_slice_rows_elem(const double* __restrict__ M, long long bs, int n, long long goff, const int* __restrict__ exps,
                                  __nv_bfloat16* __restrict__ planes, long long plane_bs, int lld,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    const int col = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y, b = blockIdx.z;
    if (col >= (n + KB - 1) / KB * KB) return;   // the K tail n..n32-1 is written as zeros
    const int e = exps[(long long)b * n + row];
    put_digits<KS>(col < n ? M[(long long)b * bs + (long long)row * n + col] : 0.0, e, goff,
               planes + (long long)b * plane_bs + (long long)row * 2 * lld + kpos(col),
               (long long)n * 2 * lld);
}

// Column maxima of |M| (as the bit pattern of a non-negative double; out zeroed first): one
// thread per column over a 16-row chunk, all 16 loads in flight.
__global__ void k_colmax(const double* __restrict__ M, long long bs, int n,
                         unsigned long long* __restrict__ out,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    const int col = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.z;
    if (col >= n) return;
    const int r0 = blockIdx.y * 16;
    const double* src = M + (long long)b * bs + (long long)r0 * n + col;
    unsigned long long mx = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (r0 + i < n) {
            mx = max_bits(mx, abs_bits(__ldg(src + (long long)i * n)));
        }
    }
    atomicMax(out + (long long)b * n + col, mx);
}

// Slices of small square tiles (n <= 64, even) for a grid product, in one launch: block
// b < nI takes the rows of A tile b (A operand, pair layout), block nI + j the columns of B
// tile j (B^T planes).  The tile is staged in shared memory; a row's (column's) exponent
// comes from its maximum magnitude, as in the separate slicers, and the digits are the same.
template <int KS>
__global__ void __launch_bounds__(256) k_slice_tiles(const double* __restrict__ A, long long a_bs,
                                                     int nI, const double* __restrict__ B,
                                                     long long b_bs, int n, long long goff,
                                                     __nv_bfloat16* __restrict__ plA,
                                                     __nv_bfloat16* __restrict__ plB, int lld,
                                                     int* __restrict__ eA, int* __restrict__ eB) {
    pdl_wait();
    pdl_trigger();
    __shared__ double t[64][65];
    __shared__ unsigned long long part[4][64];
    const bool rows = (int)blockIdx.x < nI;
    const int b = rows ? (int)blockIdx.x : (int)blockIdx.x - nI;
    const double* src = rows ? A + (long long)b * a_bs : B + (long long)b * b_bs;
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int r = e >> 6, c = e & 63;
        t[r][c] = (r < n && c < n) ? src[(long long)r * n + c] : 0.0;
    }
    __syncthreads();
    const int q = threadIdx.x >> 6, x = threadIdx.x & 63;   // quarter, row (column) index
    __shared__ int es[64];
    unsigned long long mx = 0;
#pragma unroll
    for (int u = 0; u < 16; ++u)
        mx = max_bits(mx, abs_bits(rows ? t[x][q * 16 + u] : t[q * 16 + u][x]));
    part[q][x] = mx;
    __syncthreads();
    if (q == 0) {
        const int e = exp_above(max_bits(max_bits(part[0][x], part[1][x]), max_bits(part[2][x], part[3][x])));
        es[x] = e;
        if (x < n) (rows ? eA : eB)[(long long)b * n + x] = e;
    }
    __syncthreads();
    if (rows) {   // a warp writes 32 consecutive K of one row per slice
        const long long pstride = (long long)n * 2 * lld;
        __nv_bfloat16* dst = plA + (long long)b * num_pairs(KS) * pstride;
        const int n32 = (n + KB - 1) / KB * KB;   // the K tail up to n32 is written as zeros
        for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
            const int r = idx >> 6, j = idx & 63;
            if (r < n && j < n32)
                put_digits<KS>(j < n ? t[r][j] : 0.0, es[r], goff, dst + (long long)r * 2 * lld + kpos(j),
                               pstride);
        }
    } else {      // a warp writes 32 consecutive K pairs of one plane row (tile column)
        const long long pstride = (long long)n * lld;
        __nv_bfloat16* dst = plB + (long long)b * KS * pstride;
        for (int idx = threadIdx.x; idx < 64 * 32; idx += 256) {
            const int xc = idx >> 5, k0 = 2 * (idx & 31);
            if (xc >= n || k0 >= n) continue;
            const int e = es[xc];
            const long long G0 = scaled_int_fp64(t[k0][xc], e) + goff;
            const long long G1 = scaled_int_fp64(t[k0 + 1][xc], e) + goff;   // 0 past n
            unsigned* d = reinterpret_cast<unsigned*>(dst + (long long)xc * lld + k0);
#pragma unroll
            for (int tt = 0; tt < KS; ++tt) d[(long long)tt * (pstride / 2)] = digit_pair(G0, G1, tt);
        }
    }
}

// Column slices (B operand, written transposed: plane row j = column j of M) through a
// shared 64-row x 32-column block of M (stored column-major, pitch 65); e_j from the column
// maxima (or, CODES, from the exponent codes an epilogue recorded).  Each thread turns two
// consecutive rows of one column (two consecutive K of the plane row) into digits and stores
// both per plane in one 4-byte word.
template <int KS, bool CODES>
__global__ void __launch_bounds__(256) k_slice_cols(const double* __restrict__ M, long long bs,
                                                    int n, long long goff,
                                                    const unsigned long long* __restrict__ colmax,
                                                    const int* __restrict__ codes,
                                                    __nv_bfloat16* __restrict__ planes,
                                                    long long plane_bs, int lld,
                                                    int* __restrict__ exps,
        const int* __restrict__ gate, const int* __restrict__ bidx) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    __shared__ double tile[32][65];
    const int b = bidx ? __ldg(bidx + blockIdx.z) : (int)blockIdx.z;   // listed matrices only
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 32;
    const double* src = M + (long long)b * bs;
    for (int i = threadIdx.y; i < 64; i += blockDim.y) {
        const int row = r0 + i, col = c0 + threadIdx.x;
        tile[threadIdx.x][i] = (row < n && col < n) ? src[(long long)row * n + col] : 0.0;
    }
    __syncthreads();
    const long long pstride = (long long)n * lld;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int col = c0 + i, k0 = r0 + 2 * threadIdx.x;   // plane row col, K k0 and k0 + 1
        if (col >= n || k0 >= n) continue;
        const int e = CODES ? exp_from_code(codes[(long long)b * n + col])
                            : exp_above(colmax[(long long)b * n + col]);
        if (blockIdx.y == 0 && threadIdx.x == 0) exps[(long long)b * n + col] = e;
        const long long G0 = scaled_int_fp64(tile[i][2 * threadIdx.x], e) + goff;
        const long long G1 = scaled_int_fp64(tile[i][2 * threadIdx.x + 1], e) + goff;   // 0 past n
        unsigned* dst = reinterpret_cast<unsigned*>(planes + (long long)b * plane_bs +
                                                    (long long)col * lld + k0);
#pragma unroll
        for (int t = 0; t < KS; ++t) dst[(long long)t * (pstride / 2)] = digit_pair(G0, G1, t);
    }
}

// Both operands of a squaring Q Q from one read of Q: the rows of Q in the A operand's pair
// layout (exponents from the recorded row codes) and its columns as the rows of the B^T planes
// (from the column codes).  64 x 32 tiles (32 x 8 threads) staged in shared memory; the B part
// is k_slice_cols's, the A part takes each tile row in pairs of columns (K positions up to n32:
// the tiles cover them, with zeros past n).  bidx: the listed matrices (planes, exponents and
// codes indexed by the matrix).
template <int KS>
__global__ void __launch_bounds__(256) k_slice_both_pre(const double* __restrict__ M, long long bs,
                                                        int n, long long goff,
                                                        const int* __restrict__ rcodes,
                                                        const int* __restrict__ ccodes,
                                                        __nv_bfloat16* __restrict__ planesA,
                                                        long long plane_bsA,
                                                        __nv_bfloat16* __restrict__ planesB,
                                                        long long plane_bsB, int lld,
                                                        int* __restrict__ expsA,
                                                        int* __restrict__ expsB,
                                                        const int* __restrict__ gate,
                                                        const int* __restrict__ bidx) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    pdl_trigger();
    __shared__ double tile[32][65];
    const int b = bidx ? __ldg(bidx + blockIdx.z) : (int)blockIdx.z;   // listed matrices only
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 32;
    const double* src = M + (long long)b * bs;
    for (int i = threadIdx.y; i < 64; i += blockDim.y) {
        const int row = r0 + i, col = c0 + threadIdx.x;
        tile[threadIdx.x][i] = (row < n && col < n) ? src[(long long)row * n + col] : 0.0;
    }
    __syncthreads();
    // B^T planes: plane row col, K positions k0 and k0 + 1 (rows of Q)
    {
        const long long pstride = (long long)n * lld;
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            const int col = c0 + i, k0 = r0 + 2 * threadIdx.x;
            if (col >= n || k0 >= n) continue;
            const int e = exp_from_code(ccodes[(long long)b * n + col]);
            if (blockIdx.y == 0 && threadIdx.x == 0) expsB[(long long)b * n + col] = e;
            const long long G0 = scaled_int_fp64(tile[i][2 * threadIdx.x], e) + goff;
            const long long G1 = scaled_int_fp64(tile[i][2 * threadIdx.x + 1], e) + goff;
            unsigned* dst = reinterpret_cast<unsigned*>(planesB + (long long)b * plane_bsB +
                                                        (long long)col * lld + k0);
#pragma unroll
            for (int t = 0; t < KS; ++t) dst[(long long)t * (pstride / 2)] = digit_pair(G0, G1, t);
        }
    }
    // A pair layout: row r0 + rho, K positions c and c + 1 (columns of Q), c = c0 + 2 pi
    {
        const long long pstride = (long long)n * 2 * lld;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        for (int item = tid; item < 64 * 16; item += blockDim.x * blockDim.y) {
            const int rho = item >> 4, pi = item & 15;
            const int row = r0 + rho, c = c0 + 2 * pi;
            if (row >= n) continue;
            const int e = exp_from_code(rcodes[(long long)b * n + row]);
            if (blockIdx.x == 0 && pi == 0) expsA[(long long)b * n + row] = e;
            const long long G0 = scaled_int_fp64(tile[2 * pi][rho], e) + goff;
            const long long G1 = scaled_int_fp64(tile[2 * pi + 1][rho], e) + goff;   // 0 past n
            __nv_bfloat16* dst = planesA + (long long)b * plane_bsA + (long long)row * 2 * lld + kpos(c);
#pragma unroll
            for (int t = 0; t < KS; ++t)
                *reinterpret_cast<unsigned*>(dst + slice_off(t, pstride)) = digit_pair(G0, G1, t);
        }
    }
}

// Slices of M's columns in the A operand's pair layout (plane row c = column c of M): the A
// operand M^T without forming the transpose.  e_c from colmax; the K positions n .. n32 get
// zero digits, as the row slicers write them.  64 x 32 transposing tiles (32 x 8 threads),
// two digits per 4-byte store.
template <int KS>
__global__ void __launch_bounds__(256) k_slice_cols_a(const double* __restrict__ M, long long bs,
                                                      int n, long long goff,
                                                      const unsigned long long* __restrict__ colmax,
                                                      __nv_bfloat16* __restrict__ planes,
                                                      long long plane_bs, int lld,
                                                      int* __restrict__ exps) {
    pdl_wait();
    pdl_trigger();
    __shared__ double tile[32][65];
    const int b = blockIdx.z, r0 = blockIdx.y * 64, c0 = blockIdx.x * 32;
    const double* src = M + (long long)b * bs;
    for (int i = threadIdx.y; i < 64; i += blockDim.y) {
        const int row = r0 + i, col = c0 + threadIdx.x;
        tile[threadIdx.x][i] = (row < n && col < n) ? src[(long long)row * n + col] : 0.0;
    }
    __syncthreads();
    const int n32 = (n + KB - 1) / KB * KB;
    const long long pstride = (long long)n * 2 * lld;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int col = c0 + i, k0 = r0 + 2 * threadIdx.x;   // plane row col, K k0 and k0 + 1
        if (col >= n || k0 >= n32) continue;
        const int e = exp_above(colmax[(long long)b * n + col]);
        if (blockIdx.y == 0 && threadIdx.x == 0) exps[(long long)b * n + col] = e;
        const long long G0 = scaled_int_fp64(tile[i][2 * threadIdx.x], e) + goff;
        const long long G1 = scaled_int_fp64(tile[i][2 * threadIdx.x + 1], e) + goff;   // 0 past n
        __nv_bfloat16* dst = planes + (long long)b * plane_bs + (long long)col * 2 * lld + kpos(k0);
#pragma unroll
        for (int t = 0; t < KS; ++t)
            *reinterpret_cast<unsigned*>(dst + slice_off(t, pstride)) = digit_pair(G0, G1, t);
    }
}

// w 2^s rounded to the nearest double (ties to even) on the integer pipe, for |w| < 2^62;
// false (and *out untouched) when the result would not be a normal double.  The magnitude is
// normalised so that its top bit sits at bit 62 (bit 0 is then zero: |w| < 2^62 shifts by at
// least one), 0x1FF plus the kept bit's parity rounds the ten dropped bits half to even, and
// adding the 53-bit significand (implicit bit included) to (exponent - 1) << 52 carries into
// the exponent when the rounding reaches the next power of two.
__device__ __forceinline__ bool i64_to_f64_scaled(long long w, int s, double* out) {
    if (w == 0) { *out = 0.0; return true; }
    const unsigned long long sgn = (unsigned long long)w & 0x8000000000000000ULL;
    const unsigned long long a = w < 0 ? 0ULL - (unsigned long long)w : (unsigned long long)w;
    const int lz = __clzll((long long)a);
    const unsigned long long h = (a << lz) >> 1;
    const unsigned long long r = h + 0x1FFULL + ((h >> 10) & 1ULL);
    const int ed = (63 - lz) + 1023 + s;
    if ((unsigned)(ed - 1) >= 2045u) return false;
    *out = __longlong_as_double((long long)(sgn | (((unsigned long long)(ed - 1) << 52) + (r >> 10))));
    return true;
}
__device__ __forceinline__ bool f32_to_f64_scaled(float f, int s, double* out) {
    const unsigned u = __float_as_uint(f);
    if ((u << 1) == 0) { *out = __longlong_as_double((long long)(u >> 31) << 63); return true; }
    const int ef = (int)((u >> 23) & 0xff);
    if (ef == 0 || ef == 0xff) return false;
    const int ed = ef - 127 + 1023 + s;
    if (ed <= 0 || ed >= 2047) return false;
    *out = __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                            ((unsigned long long)ed << 52) |
                                            ((unsigned long long)(u & 0x7fffff) << 29)));
    return true;
}

// 2^(e-49) W + 2^(e-14) T through the FP64 pipe, for the rare values that leave the range
// of the integer-pipe conversions (and, when the chunks were flushed, from the FP64 partial
// sum acc = 2^35 W instead of W).  Kept out of line: its code would otherwise crowd the
// unrolled fast path.
__device__ __noinline__ double f64e_slow_value(bool flushed, double acc, long long W, float T,
                                               int e) {
    if (e >= kExpLimit) return __longlong_as_double(0x7ff8000000000000LL);   // non-finite input
    return flushed ? ldexp(fma(acc, 0x1p-35, (double)T), e - 14)
                   : ldexp(fma((double)W, 0x1p-35, (double)T), e - 14);
}
__device__ __noinline__ double f64e_store(const Epilogue& ep, int b, int row, int col, int n,
                                          double v) {
    const double r = epilogue_value(ep, b, row, col, n, v);
    epilogue_store(ep, b, row, col, n, r);
    return r;
}

// Four stored values handed back by the store helpers (for the epilogue's maxima).
struct F64x4 {
    double x, y, z, w;
};

// The fused Horner add (block sum from the power table) and/or addend, alpha = 1, for four
// products v0..v3 at columns col0..col0+3 of row `row` (inside the matrix, the power-table
// and addend rows 16-byte aligned): the same operations in the same order as
// epilogue_value, with those rows read two doubles at a time.
__device__ __noinline__ F64x4 f64e_sum_store4(const Epilogue& ep, int b, int row, int col0, int n,
                                                double v0, double v1, double v2, double v3) {
    const long long off = (long long)row * n + col0;
    double v[4] = {v0, v1, v2, v3};
    if (ep.nt >= 0) {
        const int dc = row - col0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (dc == u) v[u] += ep.coef[0];
        const long long nn = (long long)n * n;
        const double* pwrow = ep.pw + (long long)b * ep.pw_bstride + off;
        for (int j = 1; j <= ep.nt; ++j) {
            const double* pp = pwrow + (long long)(j - 1) * nn;
            const double2 p01 = __ldg(reinterpret_cast<const double2*>(pp));
            const double2 p23 = __ldg(reinterpret_cast<const double2*>(pp + 2));
            const double c = ep.coef[j];
            v[0] = fma(c, p01.x, v[0]);
            v[1] = fma(c, p01.y, v[1]);
            v[2] = fma(c, p23.x, v[2]);
            v[3] = fma(c, p23.y, v[3]);
        }
    }
    if (ep.add) {
        const double* ap = ep.add + (long long)b * ep.add_bstride + off;
        const double2 a01 = *reinterpret_cast<const double2*>(ap);
        const double2 a23 = *reinterpret_cast<const double2*>(ap + 2);
        v[0] = fma(ep.add_coef, a01.x, v[0]);
        v[1] = fma(ep.add_coef, a01.y, v[1]);
        v[2] = fma(ep.add_coef, a23.x, v[2]);
        v[3] = fma(ep.add_coef, a23.y, v[3]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) epilogue_store(ep, b, row, col0 + u, n, v[u]);
    return F64x4{v[0], v[1], v[2], v[3]};
}

// The block sum B_{i-1} = coef[0] I + sum_j coef[j] X^j of one thread's 16 products (row
// `row`, columns cb..cb+15, all inside the matrix, 16-byte aligned rows), written into their
// own output entries.  Called while the tile's MMAs run (the epilogue warps are idle then and
// the FP64 pipe is not otherwise busy), so the final epilogue only adds the product to it.
__device__ __noinline__ void f64e_block_sum16(const Epilogue& ep, int b, int row, int cb, int n,
                                              double* __restrict__ orow) {
    const long long nn = (long long)n * n;
    const double* pwrow = ep.pw + (long long)b * ep.pw_bstride + (long long)row * n + cb;
#pragma unroll 1
    for (int g = 0; g < EPI_COLS; g += 4) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        const int dc = row - (cb + g);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (dc == u) v[u] = ep.coef[0];
        for (int j = 1; j <= ep.nt; ++j) {
            const double* pp = pwrow + (long long)(j - 1) * nn + g;
            const double2 p01 = __ldg(reinterpret_cast<const double2*>(pp));
            const double2 p23 = __ldg(reinterpret_cast<const double2*>(pp + 2));
            const double c = ep.coef[j];
            v[0] = fma(c, p01.x, v[0]);
            v[1] = fma(c, p01.y, v[1]);
            v[2] = fma(c, p23.x, v[2]);
            v[3] = fma(c, p23.y, v[3]);
        }
        *reinterpret_cast<double2*>(orow + g) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(orow + g + 2) = make_double2(v[2], v[3]);
    }
}

// Product plus the block sum stored by f64e_block_sum16, for four products at columns
// col0..col0+3, then the store (and the rounded copy for the next step).
__device__ __noinline__ F64x4 f64e_add_stored4(const Epilogue& ep, int b, int row, int col0, int n,
                                                 double v0, double v1, double v2, double v3) {
    const double* op = ep.out + (long long)b * ep.out_bstride + (long long)row * n + col0;
    const double2 s01 = *reinterpret_cast<const double2*>(op);
    const double2 s23 = *reinterpret_cast<const double2*>(op + 2);
    const F64x4 r{v0 + s01.x, v1 + s01.y, v2 + s23.x, v3 + s23.y};
    epilogue_store(ep, b, row, col0, n, r.x);
    epilogue_store(ep, b, row, col0 + 1, n, r.y);
    epilogue_store(ep, b, row, col0 + 2, n, r.z);
    epilogue_store(ep, b, row, col0 + 3, n, r.w);
    return r;
}

// Tile `id` -> (matrix slot z, first row, first column); row blocks are walked in groups of
// RASTER_G with the column index outermost inside a group, so that the CTAs working at the
// same time share few B column blocks and few A row blocks.
struct TileMap {
    int tcols, trows, per_mat;
    __device__ void decode(int id, int& z, int& m0, int& n0) const {
        z = id / per_mat;
        const int rem = id - z * per_mat;
        const int span = RASTER_G * tcols;
        const int grp = rem / span, first = grp * RASTER_G;
        const int gsz = min(RASTER_G, trows - first);
        const int in = rem - grp * span;
        m0 = (first + in % gsz) * OM;
        n0 = (in / gsz) * ON;
    }
};

// Split K (stream-K).  The work is the tile-major sequence of U = tiles x nkb units (one
// output tile, one K block of 32); CTA c of G takes the units [c U / G, (c + 1) U / G), so
// that every CTA gets the same number of K blocks whatever the tile count.  A CTA's work
// is then a list of segments (tile, K blocks kb0..kb1-1): possibly the end of a tile that
// an earlier CTA started, whole tiles, possibly the start of a tile that later CTAs finish.
// The CTA that holds a tile's first K block owns it: every other piece of the tile drains
// its sums (the exact integer W and the FP32 tails T) to the piece's slot of `part` and sets
// its flag to the launch's epoch; the owner adds those pieces in CTA order (W exactly, T in
// a fixed order) and runs the epilogue.  A contributor's piece is its first segment and the
// owner's piece its last, so the owner waits only at the end of its own work, for pieces
// that were computed first.  W of a whole tile sums at most FLUSH chunks, so split launches
// are limited to K <= FLUSH x 512.  U = 0: whole tiles, blockIdx.x + i gridDim.x.
// With dpw > 0 only the last, partial wave is split: every CTA first takes the whole tiles
// blockIdx.x + i gridDim.x, i < dpw (all CTAs on neighbouring tiles at the same K offset,
// so the slice planes they read stay in L2), then its share [base + c U / G, ...) of the
// tail's units.  A contributor's piece is then its first split segment, and an owner's piece
// still its last segment.
constexpr int kMinSplitSlices = 7;

struct Split {
    long long U;            // units split between the CTAs; 0: no split
    long long* partW;       // [G][EPI_WARPS][EPI_COLS][32]
    float* partT;           // [G][EPI_WARPS][EPI_COLS][32]
    unsigned* flags;        // [G][EPI_WARPS]
    unsigned epoch;         // this launch's flag value (never 0)
    long long base;         // first split unit (dpw G nkb)
    int dpw;                // waves of whole tiles before the split tail
};

__device__ __forceinline__ long long split_start(int c, const Split& sp) {
    return sp.base + (long long)c * sp.U / gridDim.x;
}

template <bool SPLIT>
struct Segments {
    long long u, ue;        // split: units left
    int id, total, nkb;     // whole tiles: next tile
    int dpi, dpw;           // split: whole tiles taken so far, and their count
    __device__ Segments(const Split& sp, int total_, int nkb_) {
        total = total_;
        nkb = nkb_;
        id = blockIdx.x;
        dpi = 0;
        dpw = SPLIT ? sp.dpw : 0;
        u = SPLIT ? split_start(blockIdx.x, sp) : 0;
        ue = SPLIT ? split_start(blockIdx.x + 1, sp) : 0;
    }
    __device__ bool next(int& tile, int& kb0, int& kb1) {
        if (!SPLIT) {
            if (id >= total) return false;
            tile = id;
            kb0 = 0;
            kb1 = nkb;
            id += gridDim.x;
            return true;
        }
        if (dpi < dpw) {
            tile = (int)blockIdx.x + dpi * (int)gridDim.x;
            kb0 = 0;
            kb1 = nkb;
            ++dpi;
            return true;
        }
        if (u >= ue) return false;
        tile = (int)(u / nkb);
        kb0 = (int)(u - (long long)tile * nkb);
        kb1 = ue - u < (long long)(nkb - kb0) ? kb0 + (int)(ue - u) : nkb;
        u += kb1 - kb0;
        return true;
    }
};

__device__ __forceinline__ void flag_release(unsigned* f, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned flag_acquire(const unsigned* f) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    return v;
}
// Bounded wait until *f == v (false and *err set after the time limit or when another
// thread gave up).
__device__ __forceinline__ bool flag_wait(const unsigned* f, unsigned v, int* err) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (flag_acquire(f) == v) return true;
        if ((it & 15) == 0) {
            if (*(volatile int*)err != 0) return false;
            const unsigned long long now = globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitNs) {
                atomicExch(err, 1);
                return false;
            }
        }
        __nanosleep(128);
    }
}

// One K=16 step of the split product into the TMEM regions: slice t of A (pair t/2, K offset
// 64 (t & 1) bytes) times the stacked planes b'_0..b'_{NR-1-t} lands in regions t..NR-1 (one
// instruction per 256 columns), then the pairs of order NREG..K-1 (K = 9: t + q = 8) in the
// last region.  Every operand offset and shape is a compile-time constant, so the
// instructions issue back to back: the tensor pipe queues little, and any other work between
// them leaves it idle.  ASC walks the slices upwards with slice 0 first, whose instruction
// covers every region and may start the accumulation (acc0 = 0); otherwise the walk runs
// downwards and ends with slice 0's wide instructions, behind which the wait for the next
// stage hides.
template <int K, int KK, bool ASC>
__device__ __forceinline__ void issue_k16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc0) {
    constexpr int NP = K < MAX_PLANES ? K : MAX_PLANES;
    constexpr int NR = NP < NREG ? NP : NREG;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const int t = ASC ? i : NP - 1 - i;
        const uint64_t ad = da + (uint64_t)(((t >> 1) * A_PAIR + (t & 1) * 64 + KK * 32) >> 4);
        if (t < NR) {
            const int N = ON * (NR - t);
            const uint32_t acc = (ASC && t == 0) ? acc0 : 1u;
            mma_bf16(tmem + (uint32_t)(ON * t), ad, db + (uint64_t)((KK * 32) >> 4),
                     make_idesc(1, OM, N > 256 ? 256 : N), acc);
            if (N > 256)   // B rows 256..: 32 atoms of 512 B further
                mma_bf16(tmem + (uint32_t)(ON * t + 256), ad,
                         db + (uint64_t)((256 * 64 + KK * 32) >> 4),
                         make_idesc(1, OM, N > 256 ? N - 256 : ON), acc);
        }
#pragma unroll
        for (int q = (NREG - t > 0 ? NREG - t : 0); q <= K - 1 - t && q < NP; ++q)
            mma_bf16(tmem + (uint32_t)(ON * (NREG - 1)), ad,
                     db + (uint64_t)((q * B_TILE + KK * 32) >> 4), make_idesc(1, OM, ON), 1u);
    }
}

template <int K, bool SPLIT, bool GRID>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_f64e(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                int n, int kpA, int ksB, int batch, const int* __restrict__ eA,
                const int* __restrict__ eB, Epilogue ep, int* err, const int* __restrict__ bidx,
                Split sp) {
    constexpr int NP = K < MAX_PLANES ? K : MAX_PLANES;   // slices per operand
    constexpr int NPA = num_pairs(NP);                    // slice pairs of A
    constexpr int S = num_stages(NP);
    constexpr int SB = stage_bytes(NP);
    constexpr int NR = NP < NREG ? NP : NREG;         // TMEM regions in use
    constexpr int NX = NP < NEXACT ? NP : NEXACT;     // of which exact
    constexpr uint32_t TCOLS = tmem_cols(NR);
    static_assert(S >= 1, "a stage does not fit in shared memory");

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * SB);     // [stage]: all slices of A and B landed
    uint64_t* empty = full + NFULL;
    uint64_t* chunk_done = empty + MAX_STAGES;
    uint64_t* tmem_free = chunk_done + 1;
    uint64_t* mma_done = tmem_free + 1;
    uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TileMap tm;
    tm.tcols = (n + ON - 1) / ON;
    tm.trows = (n + OM - 1) / OM;
    tm.per_mat = tm.tcols * tm.trows;
    const int nkb = (n + KB - 1) / KB;
    constexpr int kb_per_chunk = KCHUNK / KB;
    const int nchunks = (nkb + kb_per_chunk - 1) / kb_per_chunk;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(chunk_done, 1);
        mbar_init(tmem_free, EPI_WARPS * 32);
        mbar_init(mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();   // barrier init, TMEM allocation and tensor-map prefetch overlap the previous kernel
    pdl_trigger();
    // matrices processed: all, or the device plan's count (0: the launch does nothing; the
    // split schedule then covers the tiles of that many matrices)
    const int nbat = ep.dcount ? min(__ldg(ep.dcount), batch) : batch;
    const int total = tm.per_mat * nbat;
    Split spl = sp;
    if (ep.dcount && sp.U) {   // the device plan's count: the whole range split
        spl.U = (long long)total * nkb;
        spl.base = 0;
        spl.dpw = 0;
    }

    if (warp == EPI_WARPS) {
        if (lane == 0) {   // TMA producer
            uint32_t g = 0;                                   // K blocks issued so far
            int s = 0;                                        // stage of K block g
            uint32_t ph = 0;                                  // its fill parity
            bool ok = true;
            Segments<SPLIT> sg(spl, total, nkb);
            int id, kb0, kb1;
            while (ok && sg.next(id, kb0, kb1)) {
                int z, m0, n0;
                tm.decode(id, z, m0, n0);
                int ba, bb, bo;
                if constexpr (GRID) {
                    grid_index(ep, z, z, ba, bb, bo);
                } else {
                    ba = bb = bidx ? bidx[z] : z;
                }
                (void)bo;
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    if (g >= (uint32_t)S && !(ok = mbar_wait(&empty[s], ph ^ 1, err))) break;
                    uint8_t* st = smem + s * SB;
                    mbar_expect_tx(&full[s], (uint32_t)SB);
                    tma_load_3d(st + NPA * A_PAIR, &tmB, kb * KB, n0, bb * ksB, &full[s]);
#pragma unroll
                    for (int p = 0; p < NPA; ++p)   // pair rows hold 2 KB elements per K block
                        tma_load_3d(st + p * A_PAIR, &tmA, kb * 2 * KB, m0, ba * kpA + p, &full[s]);
                    if (++s == S) { s = 0; ph ^= 1; }
                }
            }
            // the copies of the last stages land before the CTA may exit (returns at once
            // unless this loop or the MMA issuer gave up early)
            const uint32_t lo = g > (uint32_t)S ? g - (uint32_t)S : 0u;
            bool landed = true;
            for (uint32_t gg = lo; gg < g && landed; ++gg)
                landed = mbar_wait_quiet(&full[gg % (uint32_t)S], (gg / S) & 1);
            if (!landed) atomicExch(err, 1);
        }
    } else if (warp == EPI_WARPS + 1) {
        if (lane == 0) {   // MMA issuer: every offset below is a compile-time constant
            uint32_t gc = 0;                                  // chunks consumed
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            const uint32_t ring = smem_u32(smem);
            Segments<SPLIT> sg(spl, total, nkb);
            int id, kb0, kb1;
            while (ok && sg.next(id, kb0, kb1)) {
                for (int kb = kb0; kb < kb1 && ok; ++kb) {
                    const int kin = kb % kb_per_chunk;
                    const bool first = kin == 0 || (SPLIT && kb == kb0);   // starts an accumulation
                    if (first && gc > 0) {   // the epilogue must have drained the last one
                        if (!(ok = mbar_wait(tmem_free, (gc - 1) & 1, err))) break;
                        tc_fence_after();
                    }
                    if (!(ok = mbar_wait(&full[s], ph, err))) break;
                    tc_fence_after();
                    const uint32_t abase = ring + (uint32_t)(s * SB);
                    const uint64_t da = sw128_desc(abase), db = sw64_desc(abase + NPA * A_PAIR);
                    if (first) {
                        issue_k16<K, 0, true>(tmem, da, db, 0u);
                        issue_k16<K, 1, false>(tmem, da, db, 1u);
                    } else {
                        issue_k16<K, 0, false>(tmem, da, db, 1u);
                        issue_k16<K, 1, false>(tmem, da, db, 1u);
                    }
                    if (!ok) break;
                    tc_commit(&empty[s]);
                    if (kin == kb_per_chunk - 1 || kb == kb1 - 1) {
                        tc_commit(chunk_done);
                        ++gc;
                    }
                    if (++s == S) { s = 0; ph ^= 1; }
                }
            }
            // every MMA issued by this thread completes before TMEM is released
            tc_commit(mma_done);
            if (!mbar_wait_quiet(mma_done, 0)) atomicExch(err, 1);
        }
    } else {
        // epilogue warps: row = m0 + 32 (warp % 4) + lane, columns n0 + 16 (warp / 4) + j
        // (a plain epilogue stores the product alone, four doubles at a time where aligned)
        const bool alpha1 = ep.alpha_b == nullptr &&
                            __double_as_longlong(ep.alpha) == 0x3FF0000000000000LL;
        // grid products with alpha = -1 (block updates C - A B): the product is negated
        // exactly and then takes the path of alpha = 1, whose sum has the same roundings
        const bool alpham1 = GRID && ep.alpha_b == nullptr &&
                             __double_as_longlong(ep.alpha) == (long long)0xBFF0000000000000ULL;
        const bool ep_plain = ep.nt < 0 && ep.add == nullptr && ep.low_fmt == MPPS_FMT_NONE && alpha1;
        // fused Horner add and/or addend, alpha = +-1, with 16-byte aligned power-table and
        // addend rows (n a multiple of 4, aligned bases and even batch strides)
        const bool ep_sum = (alpha1 || alpham1) && (ep.nt >= 0 || ep.add != nullptr) &&
                            (n & 3) == 0 &&
                            ((((uintptr_t)ep.pw | (uintptr_t)ep.add) & 15) == 0) &&
                            ((ep.pw_bstride | ep.add_bstride) & 1) == 0;
        // a Horner block sum without addend, computed ahead into the output entries while the
        // MMAs run (not when the chunks are flushed: the entries then hold the FP64 partials)
        const bool ep_pre = ep_sum && alpha1 && ep.nt >= 0 && ep.add == nullptr &&
                            nchunks <= FLUSH &&
                            ((((uintptr_t)ep.out) & 15) == 0) && (ep.out_bstride & 1) == 0;
        const int q4 = warp & 3, h = warp >> 2;   // lane quarter, column group
        const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
        uint32_t gc = 0;
        Segments<SPLIT> sg(spl, total, nkb);
        int id, kb0, kb1;
        while (sg.next(id, kb0, kb1)) {
            int z, m0, n0;
            tm.decode(id, z, m0, n0);
            int ba, bb, b;   // A and B operand matrices, output matrix
            if constexpr (GRID) {
                grid_index(ep, z, z, ba, bb, b);
            } else {
                b = bidx ? bidx[z] : z;
                ba = bb = b;
            }
            long long W[EPI_COLS];
            float T[EPI_COLS];
#pragma unroll
            for (int j = 0; j < EPI_COLS; ++j) { W[j] = 0; T[j] = 0.f; }
            bool ok = true;
            const int row = m0 + q4 * 32 + lane;
            const int cb = n0 + EPI_COLS * h;
            double* orow = ep.out + (long long)b * ep.out_bstride + (long long)row * n + cb;
            const bool vec4 = ((uintptr_t)orow & 31) == 0;
            const bool head = !SPLIT || kb0 == 0;   // this CTA owns the tile
            const bool pre = !GRID && ep_pre && head && row < n && cb + EPI_COLS <= n;
            if (ep.add && row < n && cb < n)   // the addend's 16 entries: one line, early
                asm volatile("prefetch.global.L1 [%0];" ::"l"(ep.add + (long long)b * ep.add_bstride +
                                                              (long long)row * n + cb));
            if (pre) f64e_block_sum16(ep, b, row, cb, n, orow);
            const int c_end = (kb1 - 1) / kb_per_chunk;
            for (int c = kb0 / kb_per_chunk; c <= c_end; ++c, ++gc) {
                ok = __all_sync(0xffffffffu, mbar_wait(chunk_done, gc & 1, err));
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int d = 0; d < NX; ++d) {   // exact regions: W += 2^{7(5-d)} D_d
                    uint32_t v[EPI_COLS];
                    tmem_ld16(tmem + lane_base + (uint32_t)(ON * d + EPI_COLS * h), v);
                    const float up = __int_as_float((127 + DIGIT * d) << 23);   // 2^{7d}
#pragma unroll
                    for (int j = 0; j < EPI_COLS; ++j)
                        W[j] += (long long)__float2int_rn(__uint_as_float(v[j]) * up)
                                << (DIGIT * (NEXACT - 1 - d));
                }
#pragma unroll
                for (int d = NX; d < NR; ++d) {  // tail regions (FP32)
                    uint32_t v[EPI_COLS];
                    tmem_ld16(tmem + lane_base + (uint32_t)(ON * d + EPI_COLS * h), v);
#pragma unroll
                    for (int j = 0; j < EPI_COLS; ++j) T[j] += __uint_as_float(v[j]);
                }
                tc_fence_before();
                mbar_arrive_cta(tmem_free);
                // |W| < 2^58.02 per chunk: every FLUSH chunks it is added, in FP64, to this
                // tile's own output entries (used as scratch), so the integer never overflows
                if (!GRID && nchunks > FLUSH && (c % FLUSH == FLUSH - 1 || c == nchunks - 1) && row < n) {
#pragma unroll
                    for (int j = 0; j < EPI_COLS; ++j) {
                        if (cb + j < n) orow[j] = (c < FLUSH ? 0.0 : orow[j]) + (double)W[j];
                        W[j] = 0;
                    }
                }
            }
            if (!ok) break;
            if constexpr (SPLIT) {
            if (!head) {   // a later piece of a split tile: hand the sums to the owner
                const size_t slot = ((size_t)blockIdx.x * EPI_WARPS + warp) * EPI_COLS * 32 + lane;
#pragma unroll
                for (int j = 0; j < EPI_COLS; ++j) {
                    __stcg(sp.partW + slot + 32 * j, W[j]);
                    __stcg(sp.partT + slot + 32 * j, T[j]);
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) flag_release(sp.flags + (size_t)blockIdx.x * EPI_WARPS + warp, sp.epoch);
                continue;
            }
            if (kb1 < nkb) {   // the owner of a split tile adds the later pieces, in CTA order
                const long long tend = (long long)(id + 1) * nkb;
                for (int c2 = blockIdx.x + 1; c2 < (int)gridDim.x && split_start(c2, spl) < tend; ++c2) {
                    if (split_start(c2 + 1, spl) == split_start(c2, spl)) continue;   // no units: no piece
                    const unsigned* f = sp.flags + (size_t)c2 * EPI_WARPS + warp;
                    bool got = true;
                    if (lane == 0) got = flag_wait(f, sp.epoch, err);
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (!got) { ok = false; break; }
                    (void)flag_acquire(f);   // every lane reads the pieces after an acquire
                    const size_t slot = ((size_t)c2 * EPI_WARPS + warp) * EPI_COLS * 32 + lane;
#pragma unroll
                    for (int j = 0; j < EPI_COLS; ++j) {
                        W[j] += __ldcg(sp.partW + slot + 32 * j);
                        T[j] += __ldcg(sp.partT + slot + 32 * j);
                    }
                }
                if (!ok) break;
            }
            }
            // product = 2^{eA+eB-49} W + 2^{eA+eB-14} T, then the fused epilogue; with
            // ep.rmax / ep.cmax the maxima of the stored values are recorded as well (every
            // lane runs the group loop: the column maxima reduce across the warp's rows)
            const bool inside = row < n;
            const int er = inside ? eA[(long long)ba * n + row] : 0;
            const bool plain = ep_plain && cb + EPI_COLS <= n && nchunks <= FLUSH;
            int mrow = 0;
#pragma unroll
            for (int g = 0; g < EPI_COLS; g += 4) {
                double val[4] = {0.0, 0.0, 0.0, 0.0};
                if (inside) {
                    bool fast = nchunks <= FLUSH;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = g + u;
                        const int e = er + __ldg(eB + (long long)bb * n + min(cb + j, n - 1));
                        double wd = 0.0, td = 0.0;
                        // 2^(e-49) W and 2^(e-14) T formed on the integer pipe, one FP64 add
                        fast = fast && e < kExpLimit && i64_to_f64_scaled(W[j], e - 49, &wd) &&
                               f32_to_f64_scaled(T[j], e - 14, &td);
                        val[u] = wd + td;
                    }
                    if (plain && fast && vec4) {   // four consecutive doubles, 32-byte aligned
                        asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(orow + g),
                                     "d"(val[0]), "d"(val[1]), "d"(val[2]), "d"(val[3]) : "memory");
                    } else if (fast && pre) {
                        const F64x4 r = f64e_add_stored4(ep, b, row, cb + g, n, val[0], val[1],
                                                         val[2], val[3]);
                        val[0] = r.x; val[1] = r.y; val[2] = r.z; val[3] = r.w;
                    } else if (fast && ep_sum && cb + EPI_COLS <= n && nchunks <= FLUSH) {
                        if (alpham1) {
#pragma unroll
                            for (int u = 0; u < 4; ++u) val[u] = -val[u];
                        }
                        const F64x4 r = f64e_sum_store4(ep, b, row, cb + g, n, val[0], val[1],
                                                        val[2], val[3]);
                        val[0] = r.x; val[1] = r.y; val[2] = r.z; val[3] = r.w;
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int col = cb + g + u;
                            val[u] = col < n ? f64e_store(ep, b, row, col, n, fast ? val[u] : f64e_slow_value(
                                                   nchunks > FLUSH, orow[g + u], W[g + u], T[g + u],
                                                   er + __ldg(eB + (long long)bb * n + col)))
                                             : 0.0;
                        }
                    }
                }
                if (!GRID && (ep.rmax || ep.cmax)) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = exp_code(val[u]);
                        mrow = c > mrow ? c : mrow;
                        if (ep.cmax) {   // column maximum over the warp's 32 rows
                            const int cm = (int)__reduce_max_sync(0xffffffffu, (unsigned)c);
                            if (lane == g + u && cb + g + u < n && cm)
                                atomicMax(ep.cmax + (long long)b * n + cb + g + u, cm);
                        }
                    }
                }
            }
            if (!GRID && ep.rmax && inside && mrow) atomicMax(ep.rmax + (long long)b * n + row, mrow);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
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

// A pairs: [npairs][n][2 lld] bf16 -> 3-D map (pair row, rows = n, pairs), box 2 KB x 128 x 1,
// 128-byte swizzle.  The row is read only below 2 round_up(n, KB), whose K tail the row
// slicers write as zeros.
bool make_pair_map(CUtensorMap* tm, const void* ptr, int n, int npairs, int lld) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)2 * lld, (cuuint64_t)n, (cuuint64_t)npairs};
    cuuint64_t strides[2] = {(cuuint64_t)lld * 4, (cuuint64_t)n * lld * 4};
    cuuint32_t box[3] = {(cuuint32_t)(2 * KB), (cuuint32_t)OM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// B^T planes: [nplanes][n][lld] bf16 -> 3-D map (K = n, rows = n, planes), box KB x 64 x
// planes, 64-byte swizzle; the K tail past n reads as zeros.
bool make_plane_map(CUtensorMap* tm, const void* ptr, int n, int nplanes, int lld, int box_planes) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)lld * 2, (cuuint64_t)n * lld * 2};
    cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)ON, (cuuint32_t)box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count(int dev) {
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cache[dev] = v;
    }
    return cache[dev];
}

template <int K, bool GRID = false>
mpps_status launch_k(int dev, int grid, const CUtensorMap& ta, const CUtensorMap& tb, int n,
                     int kpA, int ksB, int batch, const int* eA, const int* eB, const Epilogue& ep,
                     int* d_err, cudaStream_t st, const int* bidx, const Split& sp) {
    constexpr int NP = K < MAX_PLANES ? K : MAX_PLANES;
    constexpr int smem = num_stages(NP) * stage_bytes(NP) + 1024 + BAR_BYTES;
    static_assert(smem <= SMEM_MAX, "shared memory budget exceeded");
    // split K only for the slice counts of working-precision products (7..9); the split
    // kernel is a separate instantiation so that the whole-tile kernel keeps its code
    constexpr bool kSplit = K >= kMinSplitSlices && !GRID;
    static std::mutex attr_mu;
    static bool attr_done[64] = {false};
    std::unique_lock<std::mutex> attr_lk(attr_mu);
    if (!attr_done[dev]) {
        MPPS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f64e<K, false, GRID>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        if (kSplit)
            MPPS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f64e<K, kSplit, false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_done[dev] = true;
    }
    attr_lk.unlock();
    if (kSplit && sp.U > 0)
        MPPS_CUDA_TRY(launch_pdl(k_gemm_f64e<K, kSplit, false>, dim3(grid), dim3(THREADS), smem, st, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, bidx, sp));
    else
        MPPS_CUDA_TRY(launch_pdl(k_gemm_f64e<K, false, GRID>, dim3(grid), dim3(THREADS), smem, st, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, bidx, sp));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

}  // namespace

static int current_sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    return sm_count(dev);
}
size_t f64e_split_flag_bytes() {
    return ((size_t)current_sm_count() * EPI_WARPS * sizeof(unsigned) + 255) / 256 * 256;
}
size_t f64e_split_bytes() {
    return f64e_split_flag_bytes() +
           (size_t)current_sm_count() * EPI_WARPS * EPI_COLS * 32 * (sizeof(long long) + sizeof(float));
}

size_t f64e_plane_elems(int n, int batch, int k) {
    return (size_t)batch * num_pairs(f64e_planes(k)) * n * 2 * low_ld(n);
}

namespace {

template <int KS>
mpps_status slice_rows_k(const double* M, long long bs, int n, int batch, __nv_bfloat16* pl,
                         int* exps, cudaStream_t st, const int* gate) {
    const int lld = low_ld(n);
    const long long goff = digit_offset(KS), pbs = (long long)num_pairs(KS) * n * 2 * lld;
    if (n < 256) {
        MPPS_CUDA_TRY(launch_pdl(k_slice_rows<KS>, dim3(dim3((n + 7) / 8, batch)), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
    } else if (n <= 4096 && n % 4 == 0 && ((uintptr_t)M & 15) == 0 && bs % 2 == 0) {
        const dim3 g(n, batch);
        if (n <= 1024)
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk4<KS, 1>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
        else if (n <= 2048)
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk4<KS, 2>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
        else
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk4<KS, 4>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
    } else if (n <= 4096) {
        const dim3 g(n, batch);
        if (n <= 512)
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk<KS, 2>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
        else if (n <= 1024)
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk<KS, 4>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
        else if (n <= 2048)
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk<KS, 8>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
        else
            MPPS_CUDA_TRY(launch_pdl(k_slice_rows_blk<KS, 16>, dim3(g), dim3(256), 0, st, M, bs, n, goff, pl, pbs, lld, exps, gate));
    } else {
        // long rows: a row-maximum pass, then one thread per element
        MPPS_CUDA_TRY(launch_pdl(k_rowexp, dim3(dim3((n + 7) / 8, batch)), dim3(256), 0, st, M, bs, n, exps, gate));
        MPPS_LAUNCH_CHECK();
        MPPS_CUDA_TRY(launch_pdl(k_slice_rows_elem<KS>, dim3(dim3((n + KB + 127) / 128, n, batch)), dim3(128), 0, st, M, bs, n, goff, exps, pl,
                                 pbs, lld, gate));
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

template <int KS>
mpps_status slice_cols_k(const double* M, long long bs, int n, int batch, __nv_bfloat16* pl,
                         int* exps, unsigned long long* colmax, cudaStream_t st,
                         const int* codes, const int* gate, const int* list = nullptr) {
    const int lld = low_ld(n);
    if (codes) {
        MPPS_CUDA_TRY(launch_pdl(k_slice_cols<KS, true>, dim3(dim3((n + 31) / 32, (n + 63) / 64, batch)),
                                 dim3(dim3(32, 8)), 0, st, M, bs, n, digit_offset(KS),
                                 (const unsigned long long*)nullptr, codes, pl,
                                 (long long)KS * n * lld, lld, exps, gate, list));
        MPPS_LAUNCH_CHECK();
        return MPPS_OK;
    }
    MPPS_CUDA_TRY(launch_pdl(k_slice_cols<KS, false>, dim3(dim3((n + 31) / 32, (n + 63) / 64, batch)), dim3(dim3(32, 8)), 0, st, M, bs, n, digit_offset(KS), (const unsigned long long*)colmax, (const int*)nullptr, pl, (long long)KS * n * lld, lld,
        exps, gate, (const int*)nullptr));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

template <int KS>
mpps_status slice_cols_a_k(const double* M, long long bs, int n, int batch, __nv_bfloat16* pl,
                           int* exps, const unsigned long long* colmax, cudaStream_t st) {
    const int lld = low_ld(n);
    const int n32 = (n + KB - 1) / KB * KB;
    MPPS_CUDA_TRY(launch_pdl(k_slice_cols_a<KS>, dim3((n + 31) / 32, (n32 + 63) / 64, batch), dim3(32, 8), 0, st,
                             M, bs, n, digit_offset(KS), colmax, pl,
                             (long long)num_pairs(KS) * n * 2 * lld, lld, exps));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

}  // namespace

mpps_status launch_slice_cols_a(const double* M, long long bs, int n, int batch, int k, void* planes,
                                int* exps, unsigned long long* colmax, cudaStream_t st) {
    k = f64e_planes(k);
    ProfScope prof(MPPS_PROF_SLICE, st);
    if (batch > 65535) {
        set_error("slice_cols_a: batch %d exceeds the grid limit", batch);
        return MPPS_EINVAL;
    }
    MPPS_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)batch * n, st));
    MPPS_CUDA_TRY(launch_pdl(k_colmax, dim3(dim3((n + 127) / 128, (n + 15) / 16, batch)), dim3(128), 0, st, M, bs, n, colmax,
                             (const int*)nullptr));
    MPPS_LAUNCH_CHECK();
    __nv_bfloat16* pl = (__nv_bfloat16*)planes;
    switch (k) {
        case 1: return slice_cols_a_k<1>(M, bs, n, batch, pl, exps, colmax, st);
        case 2: return slice_cols_a_k<2>(M, bs, n, batch, pl, exps, colmax, st);
        case 3: return slice_cols_a_k<3>(M, bs, n, batch, pl, exps, colmax, st);
        case 4: return slice_cols_a_k<4>(M, bs, n, batch, pl, exps, colmax, st);
        case 5: return slice_cols_a_k<5>(M, bs, n, batch, pl, exps, colmax, st);
        case 6: return slice_cols_a_k<6>(M, bs, n, batch, pl, exps, colmax, st);
        case 7: return slice_cols_a_k<7>(M, bs, n, batch, pl, exps, colmax, st);
        default: return slice_cols_a_k<8>(M, bs, n, batch, pl, exps, colmax, st);
    }
}

mpps_status launch_slice_rows(const double* M, long long bs, int n, int batch, int k, void* planes,
                              int* exps, cudaStream_t st, const int* gate) {
    k = f64e_planes(k);
    ProfScope prof(MPPS_PROF_SLICE, st);
    if (batch > 65535) {
        set_error("slice_rows: batch %d exceeds the grid limit", batch);
        return MPPS_EINVAL;
    }
    __nv_bfloat16* pl = (__nv_bfloat16*)planes;
    switch (k) {
        case 1: return slice_rows_k<1>(M, bs, n, batch, pl, exps, st, gate);
        case 2: return slice_rows_k<2>(M, bs, n, batch, pl, exps, st, gate);
        case 3: return slice_rows_k<3>(M, bs, n, batch, pl, exps, st, gate);
        case 4: return slice_rows_k<4>(M, bs, n, batch, pl, exps, st, gate);
        case 5: return slice_rows_k<5>(M, bs, n, batch, pl, exps, st, gate);
        case 6: return slice_rows_k<6>(M, bs, n, batch, pl, exps, st, gate);
        case 7: return slice_rows_k<7>(M, bs, n, batch, pl, exps, st, gate);
        default: return slice_rows_k<8>(M, bs, n, batch, pl, exps, st, gate);
    }
}

namespace {
template <int KS>
mpps_status slice_rows_pre_k(const double* M, long long bs, int n, int batch, __nv_bfloat16* pl,
                             int* exps, const int* rmax, int* rclear, cudaStream_t st,
                             const int* gate, const int* list) {
    const int lld = low_ld(n);
    const long long goff = digit_offset(KS), pbs = (long long)num_pairs(KS) * n * 2 * lld;
    const int n32 = (n + KB - 1) / KB * KB;
    // the kernel's mapping: TPR threads per row, 256 / TPR rows per block
    auto grid_for = [&](int V) {
        int tpr = 1;
        while (tpr < 256 && tpr * V < n32) tpr <<= 1;
        const int gx = (n32 / V + tpr - 1) / tpr;
        const int rows = (n + 256 / tpr - 1) / (256 / tpr);
        return dim3(gx, rows < 65535 ? rows : 65535, batch);
    };
    if (n % 4 == 0 && ((uintptr_t)M & 15) == 0 && bs % 2 == 0) {
        MPPS_CUDA_TRY(launch_pdl(k_slice_rows_pre<KS, 4>, grid_for(4), dim3(256), 0, st, M, bs, n,
                                 goff, rmax, rclear, pl, pbs, lld, exps, gate, list));
    } else {
        MPPS_CUDA_TRY(launch_pdl(k_slice_rows_pre<KS, 1>, grid_for(1), dim3(256), 0, st, M, bs, n,
                                 goff, rmax, rclear, pl, pbs, lld, exps, gate, list));
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}
}  // namespace

mpps_status launch_slice_rows_pre(const double* M, long long bs, int n, int batch, int k,
                                  void* planes, int* exps, const int* rmax, int* rmax_clear,
                                  cudaStream_t st, const int* gate, const int* list) {
    k = f64e_planes(k);
    ProfScope prof(MPPS_PROF_SLICE, st);
    if (batch > 65535) {
        set_error("slice_rows: batch %d exceeds the grid limit", batch);
        return MPPS_EINVAL;
    }
    __nv_bfloat16* pl = (__nv_bfloat16*)planes;
    switch (k) {
        case 1: return slice_rows_pre_k<1>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        case 2: return slice_rows_pre_k<2>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        case 3: return slice_rows_pre_k<3>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        case 4: return slice_rows_pre_k<4>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        case 5: return slice_rows_pre_k<5>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        case 6: return slice_rows_pre_k<6>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        case 7: return slice_rows_pre_k<7>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
        default: return slice_rows_pre_k<8>(M, bs, n, batch, pl, exps, rmax, rmax_clear, st, gate, list);
    }
}

mpps_status launch_slice_both_pre(const double* M, long long bs, int n, int batch, int k,
                                  void* planesA, int* expsA, const int* rcodes, void* planesB,
                                  int* expsB, const int* ccodes, cudaStream_t st, const int* gate,
                                  const int* list) {
    k = f64e_planes(k);
    ProfScope prof(MPPS_PROF_SLICE, st);
    if (batch > 65535 || n > 65535 * 64) {
        set_error("slice_both: batch %d or n %d exceeds the grid limit", batch, n);
        return MPPS_EINVAL;
    }
    if (batch == 0) return MPPS_OK;
    const int lld = low_ld(n);
    __nv_bfloat16* pa = (__nv_bfloat16*)planesA;
    __nv_bfloat16* pb = (__nv_bfloat16*)planesB;
    const dim3 g((n + 31) / 32, (n + 63) / 64, batch);
#define MPPS_SB_CASE(KS)                                                                            \
    case KS:                                                                                        \
        MPPS_CUDA_TRY(launch_pdl(k_slice_both_pre<KS>, g, dim3(32, 8), 0, st, M, bs, n, digit_offset(KS), \
                                 rcodes, ccodes, pa, (long long)num_pairs(KS) * n * 2 * lld, pb,     \
                                 (long long)KS * n * lld, lld, expsA, expsB, gate, list));           \
        break;
    switch (k) {
        MPPS_SB_CASE(1) MPPS_SB_CASE(2) MPPS_SB_CASE(3) MPPS_SB_CASE(4)
        MPPS_SB_CASE(5) MPPS_SB_CASE(6) MPPS_SB_CASE(7)
        default: MPPS_SB_CASE(8)
    }
#undef MPPS_SB_CASE
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_slice_cols_pre(const double* M, long long bs, int n, int batch, int k,
                                  void* planes, int* exps, const int* cmax, cudaStream_t st,
                                  const int* gate, const int* list) {
    k = f64e_planes(k);
    ProfScope prof(MPPS_PROF_SLICE, st);
    __nv_bfloat16* pl = (__nv_bfloat16*)planes;
    switch (k) {
        case 1: return slice_cols_k<1>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        case 2: return slice_cols_k<2>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        case 3: return slice_cols_k<3>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        case 4: return slice_cols_k<4>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        case 5: return slice_cols_k<5>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        case 6: return slice_cols_k<6>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        case 7: return slice_cols_k<7>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
        default: return slice_cols_k<8>(M, bs, n, batch, pl, exps, nullptr, st, cmax, gate, list);
    }
}

mpps_status launch_slice_cols(const double* M, long long bs, int n, int batch, int k, void* planes,
                              int* exps, unsigned long long* colmax, cudaStream_t st,
                              const int* gate) {
    k = f64e_planes(k);
    ProfScope prof(MPPS_PROF_SLICE, st);
    MPPS_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)batch * n, st));
    MPPS_CUDA_TRY(launch_pdl(k_colmax, dim3(dim3((n + 127) / 128, (n + 15) / 16, batch)), dim3(128), 0, st, M, bs, n, colmax, gate));
    MPPS_LAUNCH_CHECK();
    __nv_bfloat16* pl = (__nv_bfloat16*)planes;
    switch (k) {
        case 1: return slice_cols_k<1>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        case 2: return slice_cols_k<2>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        case 3: return slice_cols_k<3>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        case 4: return slice_cols_k<4>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        case 5: return slice_cols_k<5>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        case 6: return slice_cols_k<6>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        case 7: return slice_cols_k<7>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
        default: return slice_cols_k<8>(M, bs, n, batch, pl, exps, colmax, st, nullptr, gate);
    }
}

mpps_status launch_slice_tiles(int k, const double* A, long long a_bs, int nI, const double* B,
                               long long b_bs, int nJ, int n, void* planesA, int* eA,
                               void* planesB, int* eB, cudaStream_t st) {
    k = f64e_planes(k);
    if (n > 64 || n < 2 || (n & 1)) {
        set_error("slice_tiles: tile size %d outside 2..64 (even)", n);
        return MPPS_EINVAL;
    }
    if (nI < 0 || nJ < 0 || nI + nJ <= 0) return MPPS_OK;
    ProfScope prof(MPPS_PROF_SLICE, st);
    const int lld = low_ld(n);
    __nv_bfloat16* pa = (__nv_bfloat16*)planesA;
    __nv_bfloat16* pb = (__nv_bfloat16*)planesB;
    const dim3 g(nI + nJ);
    switch (k) {
#define MPPS_SLICE_TILES(KS)                                                                     \
    case KS:                                                                                     \
        MPPS_CUDA_TRY(launch_pdl(k_slice_tiles<KS>, g, dim3(256), 0, st, A, a_bs, nI, B, b_bs, n, \
                                 digit_offset(KS), pa, pb, lld, eA, eB));                        \
        break;
        MPPS_SLICE_TILES(1) MPPS_SLICE_TILES(2) MPPS_SLICE_TILES(3) MPPS_SLICE_TILES(4)
        MPPS_SLICE_TILES(5) MPPS_SLICE_TILES(6) MPPS_SLICE_TILES(7)
        default:
        MPPS_SLICE_TILES(8)
#undef MPPS_SLICE_TILES
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_gemm_f64e(int k, const void* slicesA, int ksA, const int* eA,
                             const void* slicesBt, int ksB, const int* eB, int n, int batch,
                             int nmat, const Epilogue& ep, int* d_err, cudaStream_t st,
                             const int* bidx, void* split) {
    if (batch <= 0) return MPPS_OK;
    ksA = f64e_planes(ksA);    // planes stored per matrix
    ksB = f64e_planes(ksB);
    if (k < 1 || k > MPPS_F64E_MAX_SLICES || ksA < f64e_planes(k) || ksB < f64e_planes(k)) {
        set_error("emulated FP64 product: slice count %d outside 1..%d", k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const int lld = low_ld(n);
    const int kpA = num_pairs(ksA);   // slice pairs of A stored per matrix
    CUtensorMap ta, tb;
    if (!make_pair_map(&ta, slicesA, n, nmat * kpA, lld) ||
        !make_plane_map(&tb, slicesBt, n, nmat * ksB, lld, f64e_planes(k))) {
        set_error("cuTensorMapEncodeTiled failed for slice planes (n=%d)", n);
        return MPPS_ECUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const long long tiles = (long long)((n + ON - 1) / ON) * ((n + OM - 1) / OM) * batch;
    if (tiles > 0x7fffffffLL) {
        set_error("emulated FP64 product: %lld tiles exceed the index range", tiles);
        return MPPS_EINVAL;
    }
    const int G = sm_count(dev);
    int grid = (int)(tiles < G ? tiles : G);
    // Split K between CTAs when there are several waves of whole tiles and the last would
    // leave at least a tenth of the SMs' time idle, every CTA keeps at least 16 K blocks and
    // W needs no flush.  (With a single partial wave the split costs more than it saves:
    // each piece adds a TMEM drain during which the tensor pipe waits.)
    const int nkb = (n + KB - 1) / KB;
    const long long waves = (tiles + G - 1) / G;
    const bool can_split = split && k >= kMinSplitSlices &&
                           (nkb + KCHUNK / KB - 1) / (KCHUNK / KB) <= FLUSH && tiles * nkb / G >= 16;
    const int tuned = can_split ? tune_lookup(TUNE_F64E_SPLIT, n, batch, k) : -1;
    // (the split tail: the tiles past the last full wave, at least 16 K blocks per CTA)
    const long long dpw_rule = tiles / G - (tiles % G == 0 ? 1 : 0);
    const bool rule = can_split && waves >= 2 && (waves * G - tiles) * 10 >= waves * G &&
                      (tiles - dpw_rule * G) * nkb >= 16LL * G;
    const int grid_tiles = grid;
    auto run = [&](bool use_split) -> mpps_status {
        Split sp{0, nullptr, nullptr, nullptr, 0u, 0, 0};
        int g = grid_tiles;
        if (use_split) {
            static std::atomic<unsigned> epoch{0};
            unsigned e = epoch.fetch_add(1u) + 1u;
            if (e == 0u) e = epoch.fetch_add(1u) + 1u;
            char* base = (char*)split;
            const size_t nslot = (size_t)G * EPI_WARPS * EPI_COLS * 32;
            // whole tiles for the full waves, the partial last wave split
            sp.dpw = (int)(tiles / G);
            if (sp.dpw * (long long)G == tiles) sp.dpw -= 1;   // (a full last wave: split it)
            sp.base = (long long)sp.dpw * G * nkb;
            sp.U = (tiles - (long long)sp.dpw * G) * nkb;
            sp.flags = (unsigned*)base;
            sp.partW = (long long*)(base + f64e_split_flag_bytes());
            sp.partT = (float*)(sp.partW + nslot);
            sp.epoch = e;
            g = G;
        }
        switch (k) {
            case 1: return launch_k<1>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 2: return launch_k<2>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 3: return launch_k<3>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 4: return launch_k<4>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 5: return launch_k<5>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 6: return launch_k<6>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 7: return launch_k<7>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            case 8: return launch_k<8>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
            default: return launch_k<9>(dev, g, ta, tb, n, kpA, ksB, batch, eA, eB, ep, d_err, st, bidx, sp);
        }
    };
    const int pairs = k <= 8 ? k * (k + 1) / 2 : 43;
    ProfScope prof(MPPS_PROF_GEMM_F64E, st, 2.0 * n * (double)n * n * batch * pairs);
    // with tuning on, the first launch of an eligible shape times both schedules (not when
    // the epilogue accumulates into its own output: a re-run would add twice)
    const bool inplace = ep.add != nullptr && ep.add == ep.out;
    if (can_split && tuned < 0 && !inplace && !ep.dcount && tune_enabled())
        return tune_run(TUNE_F64E_SPLIT, n, batch, k, 2, st,
                        [&](int c) { return run(c == 1); });
    return run(tuned >= 0 ? tuned == 1 : rule);
}

mpps_status launch_gemm_f64e_grid(int k, const void* slicesA, const int* eA, int nmatA,
                                  const void* slicesBt, const int* eB, int nmatB, int n,
                                  const Epilogue& ep, int* d_err, cudaStream_t st) {
    if (nmatA <= 0 || nmatB <= 0) return MPPS_OK;
    if (k < 1 || k > MPPS_F64E_MAX_SLICES || ep.gnj != nmatB || n > KCHUNK || ep.rmax ||
        ep.cmax || ep.nt >= 0) {
        set_error("emulated FP64 grid product: slice count %d, grid width %d (need %d), tile %d "
                  "(at most %d, no block sum or exponent codes)", k, ep.gnj, nmatB, n, KCHUNK);
        return MPPS_EINVAL;
    }
    const int kp = f64e_planes(k);
    const int lld = low_ld(n);
    const int kpA = num_pairs(kp);
    CUtensorMap ta, tb;
    if (!make_pair_map(&ta, slicesA, n, nmatA * kpA, lld) ||
        !make_plane_map(&tb, slicesBt, n, nmatB * kp, lld, kp)) {
        set_error("cuTensorMapEncodeTiled failed for slice planes (n=%d)", n);
        return MPPS_ECUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const long long batch = (long long)nmatA * nmatB;
    const long long tiles = (long long)((n + ON - 1) / ON) * ((n + OM - 1) / OM) * batch;
    if (tiles > 0x7fffffffLL) {
        set_error("emulated FP64 grid product: %lld tiles exceed the index range", tiles);
        return MPPS_EINVAL;
    }
    const int G = sm_count(dev);
    const int grid = (int)(tiles < G ? tiles : G);
    const int pairs = k <= 8 ? k * (k + 1) / 2 : 43;
    ProfScope prof(MPPS_PROF_GEMM_F64E, st, 2.0 * n * (double)n * n * (double)batch * pairs);
    const Split sp{0, nullptr, nullptr, nullptr, 0u, 0, 0};
    const int nb = (int)batch;
    switch (k) {
        case 1: return launch_k<1, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 2: return launch_k<2, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 3: return launch_k<3, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 4: return launch_k<4, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 5: return launch_k<5, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 6: return launch_k<6, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 7: return launch_k<7, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        case 8: return launch_k<8, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
        default: return launch_k<9, true>(dev, grid, ta, tb, n, kpA, kp, nb, eA, eB, ep, d_err, st, nullptr, sp);
    }
}

}  // namespace mpps
