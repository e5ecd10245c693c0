// elementwise.cu -- HBM-bound steps of the PS evaluation: block sums B_i (eq. (1.1)),
// their 1-norms (the inputs of eq. (2.8)), exact power-of-two scaling (eq. (3.6)),
// rounded operand copies for the low-precision products, and small reductions.
#include "common.cuh"

#include <string.h>

#include <math.h>

namespace mpps {

namespace {

constexpr int kColsPerBlock = 128;   // one thread per column (coalesced row reads)
constexpr int kRowsPerChunk = 64;    // rows summed by one thread before writing a partial
constexpr int kRowsF32 = 16;         // the same for the FP32 norms: many short chains
constexpr int kNormCols = 32;        // 2-D norm blocks: 32 columns (lanes) x 8 row slots (warps)
constexpr int kNormSlots = 8;
constexpr int kChunkRows = 64;       // rows of one chunk: 8 per row slot

__device__ __forceinline__ double block_max(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;   // valid in thread 0
}

// Partial column sums of |B_i| (i = 0..r), |X_s| and |X_1| over one chunk of rows.
// B_i = sum_{j=0}^{top_i} b_{si+j} X_j, top_i = s-1 (i < r), m - s r (i = r); X_0 = I.
__global__ void k_block_norms_partial(const double* __restrict__ pw, long long pw_bs, int n,
                                      int s, int m, const double* __restrict__ coef,
                                      double* __restrict__ partial, const int* __restrict__ only) {
    pdl_wait();
    const int col = blockIdx.x * kColsPerBlock + threadIdx.x;
    const int chunk = blockIdx.y, chunks = gridDim.y, b = blockIdx.z;
    const int r = m / s, q = r + 3;
    if (col >= n || (only && !__ldg(only + b))) return;
    double acc[MPPS_MAX_R + 3];
    double x[MPPS_MAX_S + 1];
    for (int t = 0; t < q; ++t) acc[t] = 0.0;
    const long long nn = (long long)n * n;
    const double* base = pw + (long long)b * pw_bs;
    const int r0 = chunk * kRowsPerChunk, r1 = min(n, r0 + kRowsPerChunk);
    for (int row = r0; row < r1; ++row) {
        x[0] = (row == col) ? 1.0 : 0.0;
        for (int j = 1; j <= s; ++j) x[j] = __ldg(base + (long long)(j - 1) * nn + (long long)row * n + col);
        for (int i = 0; i <= r; ++i) {
            const int top = (i < r) ? s - 1 : m - s * r;
            double v = 0.0;
            for (int j = 0; j <= top; ++j) v += __ldg(coef + s * i + j) * x[j];
            acc[i] += fabs(v);
        }
        acc[r + 1] += fabs(x[s]);
        acc[r + 2] += fabs(x[1]);
    }
    for (int t = 0; t < q; ++t)
        partial[(((long long)b * chunks + chunk) * q + t) * n + col] = acc[t];
}

// norms[b*q + t] = max_col sum_chunk partial[b][chunk][t][col]  (fixed summation order).
__global__ void k_norms_finalize(const double* __restrict__ partial, int n, int chunks, int q,
                                 double* __restrict__ norms, const int* __restrict__ only) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x, b = blockIdx.y;
    if (only && !__ldg(only + b)) return;
    double best = 0.0;
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
        double sum = 0.0;
        for (int c = 0; c < chunks; ++c)
            sum += partial[(((long long)b * chunks + c) * q + t) * n + col];
        best = fmax(best, sum);
    }
    best = block_max(best);
    if (threadIdx.x == 0) norms[(long long)b * q + t] = best;
}

// Column sums of |M| over 64-row chunks: 256-thread blocks of 32 columns (the lanes) x 8 row
// slots (the warps); slot w sums rows w, w+8, ..., w+56 of the chunk (8 loads in flight),
// then the 8 slot sums are added in slot order.  The chunk partials are summed in chunk
// order by the finalize kernel: a fixed summation order.
__global__ void __launch_bounds__(256) k_colsum_partial(const double* __restrict__ M, long long bs,
                                                        int n, double* __restrict__ partial) {
    pdl_wait();
    pdl_trigger();
    __shared__ double red[kNormSlots][kNormCols];
    const int lane = threadIdx.x & 31, slot = threadIdx.x >> 5;
    const int col = blockIdx.x * kNormCols + lane;
    const int chunk = blockIdx.y, chunks = gridDim.y, b = blockIdx.z;
    const int r0 = chunk * kChunkRows + slot;
    double acc = 0.0;
    if (col < n) {
        const double* base = M + (long long)b * bs + col;
        double v[kChunkRows / kNormSlots];
#pragma unroll
        for (int k = 0; k < kChunkRows / kNormSlots; ++k) {
            const int row = r0 + kNormSlots * k;
            v[k] = row < n ? __ldg(base + (long long)row * n) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kChunkRows / kNormSlots; ++k) acc += fabs(v[k]);
    }
    red[slot][lane] = acc;
    __syncthreads();
    if (slot == 0 && col < n) {
        double sum = red[0][lane];
#pragma unroll
        for (int w = 1; w < kNormSlots; ++w) sum += red[w][lane];
        partial[((long long)b * chunks + chunk) * n + col] = sum;
    }
}

// One block per matrix: if norms[b] is within 2^-44 (relative) of a power of two, replace
// it by the max of the sequential (row 0..n-1) column sums, the order a plain loop uses.
__global__ void k_norm1_exact_near_pow2(const double* __restrict__ M, long long bs, int n,
                                        double* __restrict__ norms) {
    pdl_wait();
    pdl_trigger();
    const int b = blockIdx.x;
    const double a = norms[b];
    if (!(a > 0.0) || !isfinite(a)) return;
    int e;
    const double f = frexp(a, &e);                       // a = f 2^e, f in [0.5, 1)
    const double gap = fmin(f - 0.5, 1.0 - f);           // distance to 2^(e-1) or 2^e, / 2^e
    if (gap > 0x1p-44) return;
    double best = 0.0;
    const double* base = M + (long long)b * bs;
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
        double acc = 0.0;
        for (int row = 0; row < n; ++row) acc += fabs(base[(long long)row * n + col]);
        best = fmax(best, acc);
    }
    best = block_max(best);
    if (threadIdx.x == 0) norms[b] = best;
}

// FP64 -> FP32 by bit manipulation (truncating the significand; underflow to 0, overflow to
// inf): keeps the conversion off the FP64 pipe.  Used where only magnitudes matter.
__device__ __forceinline__ float narrow(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sgn);
    if (e >= 255) return __uint_as_float(sgn | 0x7f800000u);
    return __uint_as_float(sgn | ((unsigned)e << 23) | (unsigned)((u >> 29) & 0x7fffffu));
}

struct NormCoefs {
    float c[(MPPS_MAX_R + 1) * MPPS_MAX_S];   // b_{is+j} / scale_i
};

// Block norms in FP32: coefficients come normalised per block (|c| <= 1); for exp (||X||_1 <=
// 1, every power entry at most 1 in magnitude) nothing overflows, and entries that underflow
// are negligible against the block's norm.  For a general X a power entry or a sum beyond
// FP32's range gives an infinite norm, which launch_block_norms_redo recomputes in FP64.
// Partial sums in 16-row chunks.
__global__ void k_block_norms_partial_f32(const double* __restrict__ pw, long long pw_bs, int n,
                                          int s, int m, NormCoefs cf,
                                          double* __restrict__ partial) {
    pdl_wait();
    const int col = blockIdx.x * kColsPerBlock + threadIdx.x;
    const int chunk = blockIdx.y, chunks = gridDim.y, b = blockIdx.z;
    const int r = m / s, q = r + 3;
    if (col >= n) return;
    float acc[MPPS_MAX_R + 3];
    float x[MPPS_MAX_S + 1];
    for (int t = 0; t < q; ++t) acc[t] = 0.f;
    const long long nn = (long long)n * n;
    const double* base = pw + (long long)b * pw_bs;
    const int r0 = chunk * kRowsF32, r1 = min(n, r0 + kRowsF32);
    for (int row = r0; row < r1; ++row) {
        x[0] = (row == col) ? 1.f : 0.f;
        for (int j = 1; j <= s; ++j)
            x[j] = narrow(__ldg(base + (long long)(j - 1) * nn + (long long)row * n + col));
        for (int i = 0; i <= r; ++i) {
            const int top = (i < r) ? s - 1 : m - s * r;
            float v = 0.f;
            for (int j = 0; j <= top; ++j) v = fmaf(cf.c[s * i + j], x[j], v);
            acc[i] += fabsf(v);
        }
        acc[r + 1] += fabsf(x[s]);
        acc[r + 2] += fabsf(x[1]);
    }
    for (int t = 0; t < q; ++t)
        partial[(((long long)b * chunks + chunk) * q + t) * n + col] = (double)acc[t];
}

// The same sums with compile-time bounds (s <= 8, r <= 8, the exp degrees up to 72):
// the power values and the block accumulators stay in registers.
constexpr int kRegS = 8, kRegR = 8;
template <int S, int EX>
__global__ void __launch_bounds__(256) k_block_norms_partial_f32_reg(const double* __restrict__ pw,
                                                                     long long pw_bs, int n, int m,
                                                                     NormCoefs cf,
                                                                     double* __restrict__ partial) {
    pdl_wait();
    // 2-D blocks as in k_colsum_partial: 32 columns x 8 row slots over a 64-row chunk, the slot
    // sums added in slot order.  S (the block size s) is a compile-time constant: the r full
    // blocks take S FMAs each without predicates, the last block its top + 1.  EX > 0 adds the
    // column sums of |X_2|..|X_{EX+1}| as outputs r + 3 .. r + 2 + EX.
    constexpr int NA = kRegR + 3 + EX;
    __shared__ float red[kNormSlots][NA][kNormCols];
    const int lane = threadIdx.x & 31, slot = threadIdx.x >> 5;
    const int col = blockIdx.x * kNormCols + lane;
    const int chunk = blockIdx.y, chunks = gridDim.y, b = blockIdx.z;
    const int r = m / S, q = r + 3 + EX, top = m - S * r;
    float acc[NA];
    float x[S + 1];
#pragma unroll
    for (int t = 0; t < NA; ++t) acc[t] = 0.f;
    if (col < n) {
        const long long nn = (long long)n * n;
        const double* base = pw + (long long)b * pw_bs + col;
        const int r0 = chunk * kChunkRows + slot;
#pragma unroll 1
        for (int k4 = 0; k4 < kChunkRows / kNormSlots; k4 += 4) {
            double ld[4][S];   // the powers of four rows: 4 S loads in flight
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int row = r0 + kNormSlots * (k4 + u);
#pragma unroll
                for (int j = 0; j < S; ++j)
                    ld[u][j] = row < n ? __ldg(base + (long long)row * n + (long long)j * nn) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int row = r0 + kNormSlots * (k4 + u);
                if (row >= n) break;
                x[0] = (row == col) ? 1.f : 0.f;
#pragma unroll
                for (int j = 1; j <= S; ++j) x[j] = narrow(ld[u][j - 1]);
#pragma unroll
                for (int i = 0; i < kRegR; ++i) {   // full blocks B_0..B_{r-1}
                    if (i >= r) break;
                    float v = 0.f;
#pragma unroll
                    for (int j = 0; j < S; ++j) v = fmaf(cf.c[S * i + j], x[j], v);
                    acc[i] += fabsf(v);
                }
                float v = 0.f;                       // B_r: terms j <= top
#pragma unroll
                for (int j = 0; j < S; ++j)
                    if (j <= top) v = fmaf(cf.c[S * r + j], x[j], v);
                acc[kRegR] += fabsf(v);
                acc[kRegR + 1] += fabsf(x[S]);
                acc[kRegR + 2] += fabsf(x[1]);
#pragma unroll
                for (int e = 0; e < EX; ++e) acc[kRegR + 3 + e] += fabsf(x[2 + e]);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < NA; ++t) red[slot][t][lane] = acc[t];
    __syncthreads();
    for (int idx = threadIdx.x; idx < q * kNormCols; idx += blockDim.x) {
        const int t = idx / kNormCols, l = idx % kNormCols, c = blockIdx.x * kNormCols + l;
        // accumulator of output t: B_0..B_{r-1}, then B_r, |X_s|, |X_1| in the next three, then
        // the EX extra powers
        const int ti = t < r ? t : kRegR + (t - r);
        if (c >= n) continue;
        float sum = red[0][ti][l];
#pragma unroll
        for (int w = 1; w < kNormSlots; ++w) sum += red[w][ti][l];
        partial[(((long long)b * chunks + chunk) * q + t) * n + c] = (double)sum;
    }
}

struct BlockScales {
    double c[MPPS_MAX_R + 3 + 4];
};

// One thread per column (chunks summed in order), block max, then an order-independent
// atomic max over column blocks (norms must be zeroed first).
__global__ void k_norms_finalize_scaled(const double* __restrict__ partial, int n, int chunks,
                                        int q, BlockScales sc, double* __restrict__ norms) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x, b = blockIdx.z;
    const int col = blockIdx.y * blockDim.x + threadIdx.x;
    double sum = 0.0;
    if (col < n) {
#pragma unroll 8
        for (int c = 0; c < chunks; ++c)
            sum += partial[(((long long)b * chunks + c) * q + t) * n + col];
    }
    const double best = block_max(sum) * sc.c[t];
    if (threadIdx.x == 0)
        atomicMax((unsigned long long*)(norms + (long long)b * q + t),
                  (unsigned long long)__double_as_longlong(best));
}

// Out of line, so that the rare case does not get predicated into the fast path.
__device__ __noinline__ double ldexp_slow(double x, int e) { return ldexp(x, e); }

// x 2^e, exact: the exponent field moves on the integer pipe whenever x and the result are
// normal doubles (zero stays zero); subnormal or non-finite values take ldexp.
__device__ __forceinline__ double scale_pow2(double x, int e) {
    const long long bits = __double_as_longlong(x);
    if ((bits << 1) == 0) return x;
    const int ef = (int)((bits >> 52) & 0x7ff);
    if (ef > 0 && ef < 0x7ff && ef + e > 0 && ef + e < 0x7ff)
        return __longlong_as_double(bits + ((long long)e << 52));
    return ldexp_slow(x, e);
}

__global__ void k_scale_copy(const double* __restrict__ A, long long a_bs, double* __restrict__ X,
                             long long x_bs, long long nn, const int* __restrict__ sigma) {
    pdl_wait();
    const int b = blockIdx.y;
    const int e = sigma ? -sigma[b] : 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x)
        X[b * x_bs + t] = scale_pow2(A[b * a_bs + t], e);
}

// Up to 64 values written from the launch's parameters (no host memory is read by the
// stream, so the write is captured by value into a CUDA graph).
struct Fill64 {
    double v[64];
};
__global__ void k_fill(double* __restrict__ dst, Fill64 vals, int count) {
    pdl_wait();
    if ((int)threadIdx.x < count) dst[threadIdx.x] = vals.v[threadIdx.x];
}

// FP32 storage <-> FP64 evaluation (exact widening; narrowing rounds to nearest).
__global__ void k_widen_f32(const float* __restrict__ a, double* __restrict__ x, long long count) {
    pdl_wait();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        x[t] = (double)a[t];
}
__global__ void k_narrow_f64(const double* __restrict__ x, float* __restrict__ a, long long count) {
    pdl_wait();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        a[t] = (float)x[t];
}

// Gather items of different orders into a zero-padded batch (row-major n_pad x n_pad each)
// and scatter the leading n x n blocks back.
// (Row, column) loops over a 2-D grid: x covers columns, y rows, z the matrices.
__global__ void k_gather_pad(const PadItem* __restrict__ list, int n_pad, double* __restrict__ dst) {
    pdl_wait();
    const PadItem it = list[blockIdx.z];
    double* d = dst + (long long)blockIdx.z * n_pad * n_pad;
    for (int r = blockIdx.y; r < n_pad; r += gridDim.y)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_pad; c += gridDim.x * blockDim.x)
            d[(long long)r * n_pad + c] = (r < it.n && c < it.n) ? it.A[(long long)r * it.n + c] : 0.0;
}

__global__ void k_scatter_unpad(const PadItem* __restrict__ list, int n_pad,
                                const double* __restrict__ src) {
    pdl_wait();
    const PadItem it = list[blockIdx.z];
    const double* sp = src + (long long)blockIdx.z * n_pad * n_pad;
    for (int r = blockIdx.y; r < it.n; r += gridDim.y)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < it.n; c += gridDim.x * blockDim.x)
            it.out[(long long)r * it.n + c] = sp[(long long)r * n_pad + c];
}

// sigma[b] = max(0, ceil(log2 norms[b])) (0 for a non-finite norm), exactly as the host rule.
__global__ void k_sigma(const double* __restrict__ norms, int batch, int* __restrict__ sigma) {
    pdl_wait();
    pdl_trigger();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double a = norms[b];
    int e = 0;
    if (a > 1.0 && isfinite(a)) {
        const double f = frexp(a, &e);     // a = f 2^e, f in [0.5, 1)
        if (f == 0.5) e -= 1;              // a power of two: log2 a exactly
    }
    sigma[b] = e;
}

__global__ void k_select_copy(const double* __restrict__ q0, const double* __restrict__ q1,
                              const int* __restrict__ sigma, double* __restrict__ out, int n,
                              double diag, int sigma_cap) {
    pdl_wait();
    const int b = blockIdx.z;
    const long long nn = (long long)n * n;
    const double* src = ((sigma[b] & 1) ? q1 : q0) + b * nn;
    // a matrix that needed more squarings than were run has no result: NaN
    const bool bad = sigma_cap >= 0 && sigma[b] > sigma_cap;
    for (int r = blockIdx.y; r < n; r += gridDim.y)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
            const long long t = (long long)r * n + c;
            double v = bad ? __longlong_as_double(0x7ff8000000000000LL) : src[t];
            if (r == c) v += diag;
            out[b * nn + t] = v;
        }
}

__global__ void k_combine(int n, const double* __restrict__ extra, long long extra_bs,
                          Epilogue ep) {
    pdl_wait();
    const int b = blockIdx.z;
    // four consecutive columns per thread; the operand rows are read two doubles at a time
    // when n is a multiple of 4 and every base and batch stride keeps them 16-byte aligned
    const bool vec = (n & 3) == 0 &&
                     ((((uintptr_t)extra | (uintptr_t)ep.pw | (uintptr_t)ep.add) & 15) == 0) &&
                     ((extra_bs | ep.pw_bstride | ep.add_bstride) & 1) == 0;
    for (int row = blockIdx.y; row < n; row += gridDim.y)
        for (int col = 4 * (blockIdx.x * blockDim.x + threadIdx.x); col < n;
             col += 4 * gridDim.x * blockDim.x) {
            const double* xr = extra ? extra + b * extra_bs + (long long)row * n + col : nullptr;
            if (vec && col + 3 < n) {
                double v[4] = {0.0, 0.0, 0.0, 0.0};
                if (xr) {
                    const double2 x01 = *reinterpret_cast<const double2*>(xr);
                    const double2 x23 = *reinterpret_cast<const double2*>(xr + 2);
                    v[0] = x01.x; v[1] = x01.y; v[2] = x23.x; v[3] = x23.y;
                }
                epilogue_value4(ep, b, row, col, n, v);
#pragma unroll
                for (int u = 0; u < 4; ++u) epilogue_store(ep, b, row, col + u, n, v[u]);
            } else {
                for (int u = 0; u < 4 && col + u < n; ++u)
                    epilogue_store(ep, b, row, col + u, n,
                                   epilogue_value(ep, b, row, col + u, n, xr ? xr[u] : 0.0));
            }
        }
}

__global__ void k_convert(int fmt, const double* __restrict__ M, long long bs, int n, void* hi,
                          void* lo, long long low_bs, int lld, const double* __restrict__ scale,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    const int b = blockIdx.z;
    const double sc = scale ? scale[b] : 1.0;
    for (int row = blockIdx.y; row < n; row += gridDim.y)
        for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < n; col += gridDim.x * blockDim.x)
            store_low(fmt, hi, lo, b * low_bs + (long long)row * lld + col,
                      M[b * bs + (long long)row * n + col] * sc);
}

// Transposed copy through a 32 x 33 shared tile: out[col][row] = round(M[row][col] * scale).
__global__ void k_convert_t(int fmt, const double* __restrict__ M, long long bs, int n, void* hi,
                            void* lo, long long low_bs, int lld,
                            const double* __restrict__ scale,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    __shared__ double tile[32][33];
    const int b = blockIdx.z;
    const double sc = scale ? scale[b] : 1.0;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const double* base = M + (long long)b * bs;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int row = r0 + i, col = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (row < n && col < n) ? base[(long long)row * n + col] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int orow = c0 + i, ocol = r0 + threadIdx.x;   // out row = source column
        if (orow < n && ocol < n)
            store_low(fmt, hi, lo, (long long)b * low_bs + (long long)orow * lld + ocol,
                      tile[threadIdx.x][i] * sc);
    }
}

struct BlockCoefs {
    double c[MPPS_MAX_S + 1];
};

__global__ void k_axpy_blocks(double* __restrict__ xbar, long long xbar_bs, int n, int t,
                              BlockCoefs c, const double* __restrict__ G, long long g_bs) {
    pdl_wait();
    const int b = blockIdx.y;
    const long long nn = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        const double gv = G[b * g_bs + e];
        for (int j = 1; j <= t; ++j) xbar[b * xbar_bs + (long long)(j - 1) * nn + e] += c.c[j] * gv;
    }
}

__global__ void k_transpose(const double* __restrict__ A, long long a_bs, double* __restrict__ At,
                            int n) {
    pdl_wait();
    __shared__ double tile[32][33];
    const int b = blockIdx.z;
    const long long nn = (long long)n * n;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int row = r0 + i, col = c0 + threadIdx.x;
        if (row < n && col < n) tile[i][threadIdx.x] = A[b * a_bs + (long long)row * n + col];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int orow = c0 + i, ocol = r0 + threadIdx.x;
        if (orow < n && ocol < n) At[b * nn + (long long)orow * n + ocol] = tile[threadIdx.x][i];
    }
}

// |x| as the bit pattern of a non-negative double (NaN as 0); the frexp exponent of such a
// pattern (value in [2^(e-1), 2^e)), 0 for zero and infinity.
__device__ __forceinline__ unsigned long long absbits(double x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    return a > 0x7ff0000000000000ULL ? 0ULL : a;
}
__device__ __forceinline__ int frexp_exp_bits(unsigned long long a) {
    const int ef = (int)(a >> 52);
    if (a == 0 || ef == 0x7ff) return 0;
    return ef != 0 ? ef - 1022 : (64 - __clzll((long long)a)) - 1074;
}

// ---- FP8 copies with block scales (operands of the block-scaled tcgen05 product) --------
// Shared exponent of a 32-entry block whose largest magnitude has the bit pattern `a`: the
// smallest X with max 2^-X <= 448 (E4M3's largest finite number), 0 for a zero block,
// clamped to [-127, 127], the range of the 8-bit code X + 127.
__device__ __forceinline__ int mx_block_exp_bits(unsigned long long a) {
    if (a == 0) return 0;
    const int ef = (int)(a >> 52);
    if (ef == 0) return -127;                        // subnormal double: below every scale
    const int E = ef - 1022;                         // max = f 2^E, f in [0.5, 1)
    // 512 f <= 448  <=>  1 + m 2^-52 <= 1.75  <=>  m <= 3 2^50
    const int X = (a & 0xFFFFFFFFFFFFFULL) <= (3ULL << 50) ? E - 9 : E - 8;
    return X < -127 ? -127 : (X > 127 ? 127 : X);
}

// Nearest E4M3 number to w, ties to the even fraction, from the bits of w.  E4M3: 4
// exponent bits (bias 7), 3 fraction bits, subnormals j 2^-9, largest finite 448.  Callers
// keep |w| <= 448; larger magnitudes give 448, NaN and infinity the NaN code.
__device__ __forceinline__ uint8_t e4m3_rne(double w) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(w);
    const unsigned sgn = (unsigned)(u >> 63) << 7;
    const unsigned long long a = u & 0x7fffffffffffffffULL;
    const int ef = (int)(a >> 52);
    if (ef == 0x7ff) return (uint8_t)(sgn | 0x7F);
    if (a > 0x407C000000000000ULL) return (uint8_t)(sgn | 0x7E);   // above 448
    if (ef == 0) return (uint8_t)sgn;                              // zero, subnormal double
    const int E = ef - 1023;                                       // |w| in [2^E, 2^(E+1))
    const unsigned long long sig = (1ULL << 52) | (a & 0xFFFFFFFFFFFFFULL);
    // |w| / quantum as sig >> sh plus the remainder: quantum 2^-9 below 2^-6, else 2^(E-3)
    const int sh = E < -6 ? 43 - E : 49;
    if (sh > 62) return (uint8_t)sgn;                              // |w| < 2^-19
    unsigned long long qv = sig >> sh;
    const unsigned long long rem = sig & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
    if (rem > half || (rem == half && (qv & 1))) ++qv;
    if (E < -6) return (uint8_t)(sgn | (unsigned)qv);              // code 8 is 2^-6
    int e8 = E + 7;
    if (qv == 16) {   // rounded up into the next binade
        qv = 8;
        ++e8;
    }
    return (uint8_t)(sgn | ((unsigned)e8 << 3) | (unsigned)(qv & 7));
}

// Offset of row (column) r's code for K block j inside the scale array of one matrix, in
// 512-byte chunks per (rpc = 128 rows | 64 columns) x (4 K blocks): (r % 32) 16 +
// (r % rpc) / 32 * 4 + j % 4 within the chunk.
__device__ __forceinline__ long long mx_code_off(int r, int j, int rpc, int kc) {
    return ((long long)(r / rpc) * kc + (j >> 2)) * 512 + (r & 31) * 16 + ((r % rpc) >> 5) * 4 +
           (j & 3);
}

// FP8 copy of each row of M (the A operand): the row's power of two 2^-e (e the frexp
// exponent of its largest magnitude, to out_exp), then per 32-entry block the scale code
// and the E4M3 values.  Rows n .. 128 kc - 1 of the last chunk get neutral codes (127).
// One 256-thread block per row; warp w takes blocks w, w + 8, ...
__global__ void __launch_bounds__(256) k_convert_rows_mx(const double* __restrict__ M, long long bs,
                                                         int n, uint8_t* __restrict__ q,
                                                         long long q_bs, int lld,
                                                         uint8_t* __restrict__ sf, long long sf_bs,
                                                         int kc, int* __restrict__ out_exp,
                                                         const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.y >= __ldg(gate)) return;   // device plan: not run
    __shared__ unsigned long long red[8];
    const int row = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31, nblk = 4 * kc;
    uint8_t* sfm = sf + (long long)b * sf_bs;
    if (row >= n) {
        for (int j = tid; j < nblk; j += blockDim.x) sfm[mx_code_off(row, j, 128, kc)] = 127;
        return;
    }
    const double* src = M + (long long)b * bs + (long long)row * n;
    unsigned long long mx = 0;
    for (int j = tid; j < n; j += blockDim.x) {
        const unsigned long long v = absbits(src[j]);
        mx = v > mx ? v : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    const int e = frexp_exp_bits(mx);
    if (tid == 0) out_exp[(long long)b * n + row] = e;
    uint8_t* dst = q + (long long)b * q_bs + (long long)row * lld;
    for (int j = warp; j < nblk; j += (int)(blockDim.x >> 5)) {
        const int k = 32 * j + lane;
        const double v = k < n ? mul_exp2(src[k], -e) : 0.0;
        unsigned long long bm = absbits(v);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, bm, o);
            bm = t > bm ? t : bm;
        }
        const int X = mx_block_exp_bits(bm);
        if (k < n) dst[k] = e4m3_rne(mul_exp2(v, -X));
        if (lane == 0) sfm[mx_code_off(row, j, 128, kc)] = (uint8_t)(X + 127);
    }
}

// Column maxima of |M| as bit patterns (out zeroed first), one thread per column over a
// 16-row chunk.
__global__ void k_colmax_bits(const double* __restrict__ M, long long bs, int n,
                              unsigned long long* __restrict__ out,
        const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    const int col = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.z;
    if (col >= n) return;
    const int r0 = blockIdx.y * 16;
    const double* src = M + (long long)b * bs + (long long)r0 * n + col;
    unsigned long long mx = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if (r0 + i < n) {
            const unsigned long long a = absbits(__ldg(src + (long long)i * n));
            mx = a > mx ? a : mx;
        }
    atomicMax(out + (long long)b * n + col, mx);
}

// FP8 copy of M transposed (row j = column j of M: the B^T operand): column j's power of
// two 2^-e (e from colmax, to out_exp), then per 32-entry block of the column the scale
// code and the E4M3 values.  A 32 x 32 tile per block (32 x 8 threads): tile row block
// blockIdx.y is one K block, each warp takes whole columns, lanes along K.  Columns n ..
// 64 ceil(n / 64) - 1 and the chunks' unused words (columns 64 .. 127 of a 128-column
// arrangement) get neutral codes (127).
__global__ void k_convert_t_mx(const double* __restrict__ M, long long bs, int n,
                               uint8_t* __restrict__ q, long long q_bs, int lld,
                               uint8_t* __restrict__ sf, long long sf_bs, int kc,
                               const unsigned long long* __restrict__ colmax,
                               int* __restrict__ out_exp, const int* __restrict__ gate) {
    pdl_wait();
    if (gate && (int)blockIdx.z >= __ldg(gate)) return;   // device plan: not run
    __shared__ double tile[32][33];
    const int b = blockIdx.z, j = blockIdx.y, r0 = 32 * j, c0 = blockIdx.x * 32;
    const int lane = threadIdx.x;
    const double* base = M + (long long)b * bs;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int row = r0 + i, col = c0 + lane;
        tile[i][lane] = (row < n && col < n) ? base[(long long)row * n + col] : 0.0;
    }
    __syncthreads();
    uint8_t* sfm = sf + (long long)b * sf_bs;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int col = c0 + i;
        const int e = col < n ? frexp_exp_bits(colmax[(long long)b * n + col]) : 0;
        const double v = mul_exp2(tile[lane][i], -e);
        unsigned long long bm = absbits(v);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, bm, o);
            bm = t > bm ? t : bm;
        }
        const int X = mx_block_exp_bits(bm);
        if (col < n && r0 + lane < n)
            q[(long long)b * q_bs + (long long)col * lld + r0 + lane] = e4m3_rne(mul_exp2(v, -X));
        if (lane == 0) {
            const long long off = mx_code_off(col, j, 64, kc);
            sfm[off] = (uint8_t)(X + 127);
            if ((col & 63) < 32) {   // words 2 and 3 of this lane's row: not read at N = 64
                sfm[off + 8] = 127;
                sfm[off + 12] = 127;
            }
            if (j == 0 && col < n) out_exp[(long long)b * n + col] = e;
        }
    }
}

__global__ void k_maxabs(const double* __restrict__ M, long long bs, long long nn,
                         double* __restrict__ out) {
    pdl_wait();
    const int b = blockIdx.y;
    double v = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x)
        v = fmax(v, fabs(M[b * bs + t]));
    v = block_max(v);
    // non-negative doubles order like their bit patterns
    if (threadIdx.x == 0)
        atomicMax((unsigned long long*)(out + b), (unsigned long long)__double_as_longlong(v));
}

// scale = 2^(target - e) with max < 2^e (frexp), so scaled entries are < 2^target.
__device__ __forceinline__ int pow2_exp_above(double mx) {
    if (!(mx > 0.0) || !isfinite(mx)) return 0;
    int e;
    frexp(mx, &e);
    return e;
}

__global__ void k_pow2_scales(const double* __restrict__ ma, const double* __restrict__ mb,
                              int batch, int target, double* sa, double* sb, double* unscale) {
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const int ea = pow2_exp_above(ma[b]), eb = pow2_exp_above(mb[b]);
    sa[b] = ldexp(1.0, target - ea);
    sb[b] = ldexp(1.0, target - eb);
    unscale[b] = ldexp(1.0, ea + eb - 2 * target);
}

// 256-thread blocks over an n x n matrix per z: x spans ncol column units (columns, or groups
// of columns), y up to 4096 rows (each block row strides by gridDim.y), z the matrices.
inline dim3 grid2d(int ncol, int nmat, int nrow = -1) {
    if (nrow < 0) nrow = ncol;
    const int gx = (ncol + 255) / 256;
    const int gy = nrow < 4096 ? (nrow > 0 ? nrow : 1) : 4096;
    return dim3(gx > 0 ? gx : 1, gy, nmat > 0 ? nmat : 1);
}

inline int grid1d(long long work, int threads, int cap = 4096) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

int block_norms_count(int m, int s) { return m / s + 3; }

size_t block_norms_partial_elems(int n, int batch, int m, int s) {
    const int chunks = (n + kRowsPerChunk - 1) / kRowsPerChunk;
    return (size_t)batch * chunks * block_norms_count(m, s) * n;
}

size_t norm1_partial_elems(int n, int batch) {
    return (size_t)batch * ((n + kChunkRows - 1) / kChunkRows) * n;
}

size_t block_norms_f32_partial_elems(int n, int batch, int m, int s) {
    return (size_t)batch * ((n + kRowsF32 - 1) / kRowsF32) * block_norms_count(m, s) * n;
}

int block_norms_f32_power_norms(int m, int s) {
    return (s >= 4 && s <= kRegS && m / s <= kRegR) ? (s + 1) / 2 - 1 : 0;
}

size_t block_norms_f32_powers_partial_elems(int n, int batch, int m, int s) {
    return (size_t)batch * ((n + kChunkRows - 1) / kChunkRows) *
           (block_norms_count(m, s) + block_norms_f32_power_norms(m, s)) * n;
}

mpps_status launch_block_norms_f32(const double* pw, long long pw_bs, int n, int batch, int s,
                                   int m, const double* coeffs, double* partial, double* norms,
                                   cudaStream_t st, bool power_norms) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    const int ex = power_norms ? block_norms_f32_power_norms(m, s) : 0;
    if (power_norms && ex == 0) {
        set_error("block norms: no power norms for m=%d, s=%d", m, s);
        return MPPS_EINVAL;
    }
    const int r = m / s, q = block_norms_count(m, s) + ex;
    NormCoefs cf;
    BlockScales sc;
    for (int i = 0; i <= r; ++i) {
        const int top = (i < r) ? s - 1 : m - s * r;
        double mx = 0.0;
        for (int j = 0; j <= top; ++j) mx = fmax(mx, fabs(coeffs[s * i + j]));
        sc.c[i] = mx > 0.0 ? mx : 1.0;
        for (int j = 0; j < s; ++j)
            cf.c[s * i + j] = (j <= top) ? (float)(coeffs[s * i + j] / sc.c[i]) : 0.f;
    }
    sc.c[r + 1] = 1.0;
    sc.c[r + 2] = 1.0;
    for (int e = 0; e < ex; ++e) sc.c[r + 3 + e] = 1.0;
    const bool reg = s <= kRegS && m / s <= kRegR;
    const int chunks = reg ? (n + kChunkRows - 1) / kChunkRows : (n + kRowsF32 - 1) / kRowsF32;
    MPPS_CUDA_TRY(cudaMemsetAsync(norms, 0, sizeof(double) * (size_t)batch * q, st));
    const dim3 g2((n + kNormCols - 1) / kNormCols, chunks, batch);
    if (reg) {
        switch (s) {
#define MPPS_BN_CASE(S)                                                                            \
            case S:                                                                                \
                if (ex > 0)                                                                        \
                    MPPS_CUDA_TRY(launch_pdl(k_block_norms_partial_f32_reg<S, (S >= 4 ? (S + 1) / 2 - 1 : 0)>, g2, dim3(256), 0, st, pw, pw_bs, n, m, cf, partial)); \
                else                                                                               \
                    MPPS_CUDA_TRY(launch_pdl(k_block_norms_partial_f32_reg<S, 0>, g2, dim3(256), 0, st, pw, pw_bs, n, m, cf, partial)); \
                break;
            MPPS_BN_CASE(1) MPPS_BN_CASE(2) MPPS_BN_CASE(3) MPPS_BN_CASE(4)
            MPPS_BN_CASE(5) MPPS_BN_CASE(6) MPPS_BN_CASE(7) MPPS_BN_CASE(8)
#undef MPPS_BN_CASE
        }
    } else
        MPPS_CUDA_TRY(launch_pdl(k_block_norms_partial_f32, dim3((n + kColsPerBlock - 1) / kColsPerBlock, chunks, batch), dim3(kColsPerBlock), 0, st, pw, pw_bs, n, s, m, cf, partial));
    MPPS_LAUNCH_CHECK();
    MPPS_CUDA_TRY(launch_pdl(k_norms_finalize_scaled, dim3(dim3(q, (n + 127) / 128, batch)), dim3(128), 0, st, partial, n, chunks, q,
                                                                              sc, norms));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

// redo[b] = 1 when a norm of matrix b is not finite (its FP32 block norms met an entry or a
// sum beyond FP32's range, or the input holds a NaN or an infinity).
__global__ void k_norms_redo_flags(const double* __restrict__ norms, int q, int batch,
                                   int* __restrict__ redo) {
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    int f = 0;
    for (int t = 0; t < q; ++t) f |= isfinite(norms[(long long)b * q + t]) ? 0 : 1;
    redo[b] = f;
}

mpps_status launch_block_norms_redo(const double* pw, long long pw_bs, int n, int batch, int s,
                                    int m, const double* d_coeffs, double* partial, double* norms,
                                    int* redo, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    const int chunks = (n + kRowsPerChunk - 1) / kRowsPerChunk;
    const int q = block_norms_count(m, s);
    MPPS_CUDA_TRY(launch_pdl(k_norms_redo_flags, dim3((batch + 127) / 128), dim3(128), 0, st,
                             (const double*)norms, q, batch, redo));
    MPPS_LAUNCH_CHECK();
    dim3 g((n + kColsPerBlock - 1) / kColsPerBlock, chunks, batch);
    MPPS_CUDA_TRY(launch_pdl(k_block_norms_partial, dim3(g), dim3(kColsPerBlock), 0, st, pw, pw_bs, n, s, m, d_coeffs, partial,
                             (const int*)redo));
    MPPS_LAUNCH_CHECK();
    MPPS_CUDA_TRY(launch_pdl(k_norms_finalize, dim3(dim3(q, batch)), dim3(256), 0, st, partial, n, chunks, q, norms,
                             (const int*)redo));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_norm1(const double* M, long long bs, int n, int batch, double* partial,
                         double* norms, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    // fast chunked sums (64-row partials, summed in chunk order) ...
    const int chunks = (n + kChunkRows - 1) / kChunkRows;
    dim3 g((n + kNormCols - 1) / kNormCols, chunks, batch);
    MPPS_CUDA_TRY(launch_pdl(k_colsum_partial, dim3(g), dim3(256), 0, st, M, bs, n, partial));
    MPPS_LAUNCH_CHECK();
    MPPS_CUDA_TRY(cudaMemsetAsync(norms, 0, sizeof(double) * (size_t)batch, st));
    BlockScales one;
    one.c[0] = 1.0;
    MPPS_CUDA_TRY(launch_pdl(k_norms_finalize_scaled, dim3(dim3(1, (n + 127) / 128, batch)), dim3(128), 0, st, partial, n, chunks, 1,
                                                                             one, norms));
    MPPS_LAUNCH_CHECK();
    // ... and, only for a matrix whose norm lies within 2^-44 of a power of two (where the
    // summation order could move ceil(log2 ||A||_1)), the plain sequential column sums
    MPPS_CUDA_TRY(launch_pdl(k_norm1_exact_near_pow2, dim3(batch), dim3(256), 0, st, M, bs, n, norms));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_scale_copy(const double* A, long long a_bs, double* X, long long x_bs, int n,
                              int batch, const int* d_sigma, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    const long long nn = (long long)n * n;
    MPPS_CUDA_TRY(launch_pdl(k_scale_copy, dim3(dim3(grid1d(nn, 256), batch)), dim3(256), 0, st, A, a_bs, X, x_bs, nn, d_sigma));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

// Bytes copied from the launch's parameters, 2 KB per launch (see Fill64).
struct Fill2K {
    uint4 w[128];
};
__global__ void k_fill_bytes(uint4* __restrict__ dst, Fill2K vals, int words) {
    pdl_wait();
    if ((int)threadIdx.x < words) dst[threadIdx.x] = vals.w[threadIdx.x];
}

mpps_status launch_fill_bytes(void* dst, const void* host, size_t bytes, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    if ((uintptr_t)dst & 15) {
        set_error("fill_bytes: destination not 16-byte aligned");
        return MPPS_EINVAL;
    }
    const unsigned char* src = (const unsigned char*)host;
    for (size_t o = 0; o < bytes; o += sizeof(Fill2K)) {
        Fill2K f;
        const size_t c = bytes - o < sizeof(Fill2K) ? bytes - o : sizeof(Fill2K);
        memset(&f, 0, sizeof(f));
        memcpy(&f, src + o, c);
        MPPS_CUDA_TRY(launch_pdl(k_fill_bytes, dim3(1), dim3(128), 0, st, (uint4*)((char*)dst + o), f,
                                 (int)((c + 15) / 16)));
        MPPS_LAUNCH_CHECK();
    }
    return MPPS_OK;
}

mpps_status launch_fill(double* dst, const double* host_vals, int count, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    for (int o = 0; o < count; o += 64) {
        Fill64 f;
        const int c = count - o < 64 ? count - o : 64;
        for (int i = 0; i < 64; ++i) f.v[i] = i < c ? host_vals[o + i] : 0.0;
        MPPS_CUDA_TRY(launch_pdl(k_fill, dim3(1), dim3(64), 0, st, dst + o, f, c));
        MPPS_LAUNCH_CHECK();
    }
    return MPPS_OK;
}

mpps_status launch_widen_f32(const float* a, double* x, long long count, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_widen_f32, dim3(grid1d(count, 256)), dim3(256), 0, st, a, x, count));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_narrow_f64(const double* x, float* a, long long count, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_narrow_f64, dim3(grid1d(count, 256)), dim3(256), 0, st, x, a, count));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_gather_pad(const PadItem* d_list, int count, int n_pad, double* dst,
                              cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_gather_pad, grid2d(n_pad, count), dim3(256), 0, st, d_list, n_pad, dst));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_scatter_unpad(const PadItem* d_list, int count, int n_pad, const double* src,
                                 cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_scatter_unpad, grid2d(n_pad, count), dim3(256), 0, st, d_list, n_pad, src));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_sigma(const double* norms, int batch, int* sigma, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_sigma, dim3((batch + 127) / 128), dim3(128), 0, st, norms, batch, sigma));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_select_copy(const double* q0, const double* q1, const int* d_sigma, double* out,
                               int n, int batch, double diag, cudaStream_t st, int sigma_cap) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_select_copy, grid2d(n, batch), dim3(256), 0, st, q0, q1, d_sigma, out, n, diag,
                             sigma_cap));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_combine(int n, int batch, const double* extra, long long extra_bs,
                           const Epilogue& ep, cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_combine, grid2d((n + 3) / 4, batch, n), dim3(256), 0, st, n, extra, extra_bs, ep));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_convert(int fmt, const double* M, long long bs, int n, int batch, void* hi,
                           void* lo, long long low_bs, int lld, const double* d_scale,
                           bool transpose, cudaStream_t st, const int* gate) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    if (transpose) {
        dim3 g((n + 31) / 32, (n + 31) / 32, batch);
        MPPS_CUDA_TRY(launch_pdl(k_convert_t, dim3(g), dim3(dim3(32, 8)), 0, st, fmt, M, bs, n, hi, lo, low_bs, lld, d_scale, gate));
    } else {
        MPPS_CUDA_TRY(launch_pdl(k_convert, grid2d(n, batch), dim3(256), 0, st, fmt, M, bs, n, hi, lo, low_bs,
                                 lld, d_scale, gate));
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_convert_mx(const double* M, long long bs, int n, int batch, uint8_t* q,
                              long long q_bs, int lld, uint8_t* sf, long long sf_bs, bool transpose,
                              int* out_exp, unsigned long long* colmax, cudaStream_t st,
                              const int* gate) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    if (batch > 65535) {
        set_error("convert_mx: batch %d exceeds the grid limit", batch);
        return MPPS_EINVAL;
    }
    if (batch == 0 || n <= 0) return MPPS_OK;
    const int kc = (n + 127) / 128;
    if (!transpose) {
        MPPS_CUDA_TRY(launch_pdl(k_convert_rows_mx, dim3(128 * kc, batch), dim3(256), 0, st, M, bs, n,
                                 q, q_bs, lld, sf, sf_bs, kc, out_exp, gate));
    } else {
        MPPS_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)batch * n, st));
        MPPS_CUDA_TRY(launch_pdl(k_colmax_bits, dim3((n + 127) / 128, (n + 15) / 16, batch), dim3(128), 0, st, M, bs, n,
                                 colmax, gate));
        MPPS_LAUNCH_CHECK();
        MPPS_CUDA_TRY(launch_pdl(k_convert_t_mx, dim3(2 * ((n + 63) / 64), 4 * kc, batch), dim3(32, 8), 0, st, M, bs,
                                 n, q, q_bs, lld, sf, sf_bs, kc, colmax, out_exp, gate));
    }
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_maxabs(const double* M, long long bs, int n, int batch, double* out,
                          cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    const long long nn = (long long)n * n;
    MPPS_CUDA_TRY(launch_pdl(k_maxabs, dim3(dim3(grid1d(nn, 256, 1024), batch)), dim3(256), 0, st, M, bs, nn, out));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_pow2_scales(const double* maxabs_a, const double* maxabs_b, int batch,
                               int target_exp, double* scale_a, double* scale_b, double* unscale,
                               cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    MPPS_CUDA_TRY(launch_pdl(k_pow2_scales, dim3((batch + 127) / 128), dim3(128), 0, st, maxabs_a, maxabs_b, batch, target_exp,
                                                         scale_a, scale_b, unscale));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_axpy_blocks(double* xbar, long long xbar_bs, int n, int batch, int t,
                               const double* c, const double* G, long long g_bs,
                               cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    if (t <= 0) return MPPS_OK;
    BlockCoefs bc;
    for (int j = 0; j <= MPPS_MAX_S; ++j) bc.c[j] = (j <= t) ? c[j] : 0.0;
    const long long nn = (long long)n * n;
    MPPS_CUDA_TRY(launch_pdl(k_axpy_blocks, dim3(dim3(grid1d(nn, 256), batch)), dim3(256), 0, st, xbar, xbar_bs, n, t, bc, G, g_bs));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

mpps_status launch_transpose(const double* A, long long a_bs, double* At, int n, int batch,
                             cudaStream_t st) {
    ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
    dim3 g((n + 31) / 32, (n + 31) / 32, batch);
    MPPS_CUDA_TRY(launch_pdl(k_transpose, dim3(g), dim3(dim3(32, 8)), 0, st, A, a_bs, At, n));
    MPPS_LAUNCH_CHECK();
    return MPPS_OK;
}

}  // namespace mpps
