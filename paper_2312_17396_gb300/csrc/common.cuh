// common.cuh -- shared declarations of the mpps CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <functional>

#include "../../include/mpps.h"

namespace mpps {

// ---- error reporting ------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define MPPS_CUDA_TRY(call)                                                            \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::mpps::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                              __FILE__, __LINE__);                                     \
            return MPPS_ECUDA;                                                         \
        }                                                                              \
    } while (0)

#define MPPS_LAUNCH_CHECK()                                                            \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            ::mpps::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                              __FILE__, __LINE__);                                     \
            return MPPS_ECUDA;                                                         \
        }                                                                              \
    } while (0)

// ---- optional launch timing (profile.cu) -----------------------------------------
// RAII: when profiling is enabled, records CUDA events on `st` around the launches made
// while the scope is alive, tagged with a kernel class (MPPS_PROF_*).
struct ProfScope {
    ProfScope(int cls, cudaStream_t st, double work = 0.0);
    ~ProfScope();
    int cls;
    cudaStream_t st;
    cudaEvent_t a, b;
    bool on;
    double work;   // algorithmic flops of the launch (products), 0 for the rest
};

// ---- programmatic dependent launch ------------------------------------------------
// Every kernel of the library is launched with programmatic stream serialization: it may be
// scheduled while the previous kernel on the stream drains, and it calls pdl_wait() before
// it touches memory that an earlier kernel writes (griddepcontrol.wait returns when every
// prerequisite grid has completed and its writes are visible).  Kernels whose grid runs in
// one wave (the persistent products, the slicing kernels, the small reductions) then call
// pdl_trigger(), which lets their dependents launch at once (those CTAs wait in pdl_wait()
// on the SMs the grid leaves free).  Multi-wave grids do not: a dependent launched early would
// hold registers and shared memory on SMs that the grid's later waves still need, so their
// dependents launch as their last blocks exit.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---- fused epilogue of every product ---------------------------------------------
// out = alpha * (A B) + sum_{j=0}^{nt} coef[j] X_j  with X_0 = I and X_j the j-th power
// stored at pw + (j-1) n^2 (+ b * pw_bstride for batch element b).  nt = -1: no sum.
// Optionally also writes a rounded copy of out (times low_scale) for the next product:
// row-major with leading dimension lld, in format low_fmt (BF16X3 writes hi and lo).
struct Epilogue {
    int nt;
    double coef[MPPS_MAX_S + 1];
    const double* pw;
    long long pw_bstride;
    double alpha;                 // used when alpha_b is null
    const double* alpha_b;        // per batch element (device), or null
    // per-row / per-column power-of-two unscaling of a product of scaled operands (device,
    // [batch][n] each, or null): the product term is multiplied by 2^(row_exp + col_exp)
    const int* row_exp;
    const int* col_exp;
    const double* add;            // optional addend: v += add_coef * add[b][row][col]
    long long add_bstride;
    double add_coef;
    double* out;
    long long out_bstride;
    int low_fmt;
    void* low_hi;
    void* low_lo;
    long long low_bstride;
    int lld;
    double low_scale;             // used when low_scale_b is null
    const double* low_scale_b;    // per batch element (device), or null
    // exponent codes of the largest |stored value| per row and per column ([batch][n] each,
    // atomically combined with max; zeroed by the caller), or null: the exponents of the next
    // product's slices, recorded here so that the slicing needs no reduction pass (emulated
    // products only).  Code 0: every entry zero; otherwise 2048 + the frexp exponent of the
    // largest magnitude (the exponent is monotone in |x|, so the maximum of the codes is the
    // code of the maximum).
    int* rmax;
    int* cmax;
    // device-side number of matrices to process (device plan), or null: a launch whose count
    // is 0 does no work, a smaller count processes that prefix of the matrices (or of bidx)
    const int* dcount;
    // device plan: the format of the rounded copy (low_fmt = MPPS_FMT_DEVICE) is read from
    // here; a copy is written only for BF16, TF32 and BF16X3 (FP8 copies are row-scaled by
    // their own pass)
    const int* low_fmt_dev;
    // grid mode (gnj > 0): product z multiplies matrix z / gnj of the A operand with matrix
    // z % gnj of the B operand and writes (and reads its addend at) matrix
    // (z / gnj) gci + (z % gnj) gcj of the output; the products of a blocked factorisation
    // or triangular solve, whose tiles are the matrices (gnj = 0: A, B and the output all
    // take matrix z, or bidx[z])
    int gnj;
    int gci, gcj;
};

// The operand and output matrices of product z (see Epilogue::gnj).
__host__ __device__ __forceinline__ void grid_index(const Epilogue& ep, int z, int b, int& ba,
                                                    int& bb, int& bo) {
    if (ep.gnj > 0) {
        ba = z / ep.gnj;
        bb = z - ba * ep.gnj;
        bo = ba * ep.gci + bb * ep.gcj;
    } else {
        ba = bb = bo = b;
    }
}

// low_fmt value meaning "read the format from Epilogue::low_fmt_dev".
constexpr int MPPS_FMT_DEVICE = 100;

inline Epilogue epilogue_plain(double* out, long long out_bstride) {
    Epilogue e;
    e.nt = -1;
    for (int j = 0; j <= MPPS_MAX_S; ++j) e.coef[j] = 0.0;
    e.pw = nullptr; e.pw_bstride = 0; e.alpha = 1.0; e.alpha_b = nullptr;
    e.row_exp = nullptr; e.col_exp = nullptr;
    e.add = nullptr; e.add_bstride = 0; e.add_coef = 0.0;
    e.out = out; e.out_bstride = out_bstride;
    e.low_fmt = MPPS_FMT_NONE; e.low_hi = nullptr; e.low_lo = nullptr;
    e.low_bstride = 0; e.lld = 0; e.low_scale = 1.0; e.low_scale_b = nullptr;
    e.rmax = nullptr; e.cmax = nullptr;
    e.dcount = nullptr;
    e.low_fmt_dev = nullptr;
    e.gnj = 0; e.gci = 0; e.gcj = 0;
    return e;
}

// ---- rounding of one FP64 value to a product format ----------------------------
// (round to nearest; TF32 is produced as an FP32 bit pattern with the low 13 bits
// cleared after round-to-nearest-even on them)
__device__ __forceinline__ float to_tf32(double v) {
    float f = (float)v;
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) != 0x7f800000u) {        // finite: RNE on the 13 dropped bits
        u += 0x0fffu + ((u >> 13) & 1u);
        u &= 0xffffe000u;
    }
    return __uint_as_float(u);
}

// FP64 rounded to nearest even at KEEP significand bits (7: bf16, 10: tf32) on the integer
// pipe, returned as the FP32 bit pattern of the result (bf16 = its upper half); false for
// values outside the normal FP32 range (zero keeps its sign and succeeds).  Adding
// 2^(drop-1) - 1 plus the kept bit's parity rounds the dropped bits half to even; a carry
// moves into the exponent, up to infinity.
template <int KEEP>
__device__ __forceinline__ bool f64_round_bits(double x, unsigned* out) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 63) << 31;
    if ((u << 1) == 0) { *out = sgn; return true; }
    const int e = (int)((u >> 52) & 0x7ff) - 1023 + 127;
    if (e < 1 || e >= 255) return false;
    constexpr int DROP = 52 - KEEP;
    const unsigned long long m = u & 0xFFFFFFFFFFFFFULL;
    const unsigned long long r = m + ((1ULL << (DROP - 1)) - 1ULL) + ((m >> DROP) & 1ULL);
    *out = sgn | ((((unsigned)e << KEEP) + (unsigned)(r >> DROP)) << (23 - KEEP));
    return true;
}

__device__ __forceinline__ void store_low(int fmt, void* hi, void* lo, long long idx, double v) {
    unsigned bits;
    if (fmt == MPPS_FMT_BF16) {
        ((__nv_bfloat16*)hi)[idx] = f64_round_bits<7>(v, &bits)
                                        ? __ushort_as_bfloat16((unsigned short)(bits >> 16))
                                        : __double2bfloat16(v);
    } else if (fmt == MPPS_FMT_TF32 && f64_round_bits<10>(v, &bits)) {
        ((float*)hi)[idx] = __uint_as_float(bits);
    } else if (fmt == MPPS_FMT_BF16X3) {
        __nv_bfloat16 h = __double2bfloat16(v);
        ((__nv_bfloat16*)hi)[idx] = h;
        ((__nv_bfloat16*)lo)[idx] = __double2bfloat16(v - (double)__bfloat162float(h));
    } else if (fmt == MPPS_FMT_TF32) {
        ((float*)hi)[idx] = to_tf32(v);
    } else if (fmt == MPPS_FMT_FP8) {
        ((__nv_fp8_storage_t*)hi)[idx] = __nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

// v p for p = +2^k: the exponent field moves on the integer pipe when v and the result are
// normal; otherwise (or for any other p) one FP64 multiply.
__device__ __forceinline__ double mul_pow2(double v, double p) {
    const long long pb = __double_as_longlong(p), vb = __double_as_longlong(v);
    const int pe = (int)((pb >> 52) & 0x7ff), ve = (int)((vb >> 52) & 0x7ff);
    if ((pb & (long long)0x800FFFFFFFFFFFFFULL) == 0 && pe > 0 && pe < 0x7ff && ve > 0 && ve < 0x7ff) {
        const int r = ve + pe - 1023;
        if (r > 0 && r < 0x7ff) return __longlong_as_double(vb + ((long long)(pe - 1023) << 52));
    }
    return v * p;
}

// v 2^k, exact when v and the result are normal (the exponent field moves on the integer
// pipe); otherwise one FP64 multiply by 2^k (k clamped to the normal range, then ldexp).
static __device__ __noinline__ double ldexp_out_of_line(double v, int k) { return ldexp(v, k); }
__device__ __forceinline__ double mul_exp2(double v, int k) {
    const long long vb = __double_as_longlong(v);
    const int ve = (int)((vb >> 52) & 0x7ff);
    if (ve > 0 && ve < 0x7ff && ve + k > 0 && ve + k < 0x7ff)
        return __longlong_as_double(vb + ((long long)k << 52));
    return ldexp_out_of_line(v, k);
}

// FP32 -> FP64 (exact) by assembling the bits; zero, subnormal and non-finite values take the
// conversion instruction (an FP64-pipe operation).
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xffu;
    if (ef - 1u < 254u)
        return __hiloint2double((int)((u & 0x80000000u) | ((ef + 896u) << 20) | ((u >> 3) & 0xFFFFFu)),
                                (int)(u << 29));
    return (double)f;
}

// Epilogue value for element (row, col) of batch element b, given the product acc.
__device__ __forceinline__ double epilogue_value(const Epilogue& ep, int b, int row, int col,
                                                 int n, double acc) {
    const double al = ep.alpha_b ? ep.alpha_b[b] : ep.alpha;
    double v = acc;
    const long long alb = __double_as_longlong(al);
    if (alb == 0) v = 0.0;                                 // alpha = 0: no product term
    else if (alb != 0x3FF0000000000000LL) v = mul_pow2(acc, al);   // no multiply by 1
    if (ep.row_exp)
        v = mul_exp2(v, ep.row_exp[(long long)b * n + row] + ep.col_exp[(long long)b * n + col]);
    if (ep.nt >= 0) {
        if (row == col) v += ep.coef[0];
        const double* base = ep.pw + (long long)b * ep.pw_bstride + (long long)row * n + col;
        const long long nn = (long long)n * n;
        for (int j = 1; j <= ep.nt; ++j) v += ep.coef[j] * __ldg(base + (long long)(j - 1) * nn);
    }
    if (ep.add) v += ep.add_coef * ep.add[(long long)b * ep.add_bstride + (long long)row * n + col];
    return v;
}

// epilogue_value for the four products v[0..3] at columns col0..col0+3 of one row (all inside
// the matrix; power-table and addend rows 16-byte aligned): the same operations in the same
// order, with each power-table and addend row read two doubles at a time.
__device__ __forceinline__ void epilogue_value4(const Epilogue& ep, int b, int row, int col0, int n,
                                                double (&v)[4]) {
    const double al = ep.alpha_b ? ep.alpha_b[b] : ep.alpha;
    const long long alb = __double_as_longlong(al);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (alb == 0) v[u] = 0.0;
        else if (alb != 0x3FF0000000000000LL) v[u] = mul_pow2(v[u], al);
    }
    if (ep.row_exp) {
        const int re = ep.row_exp[(long long)b * n + row];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = mul_exp2(v[u], re + ep.col_exp[(long long)b * n + col0 + u]);
    }
    const long long off = (long long)row * n + col0;
    if (ep.nt >= 0) {
        const int dc = row - col0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (dc == u) v[u] += ep.coef[0];
        const double* base = ep.pw + (long long)b * ep.pw_bstride + off;
        const long long nn = (long long)n * n;
        for (int j = 1; j <= ep.nt; ++j) {
            const double* pp = base + (long long)(j - 1) * nn;
            const double2 p01 = __ldg(reinterpret_cast<const double2*>(pp));
            const double2 p23 = __ldg(reinterpret_cast<const double2*>(pp + 2));
            v[0] += ep.coef[j] * p01.x;
            v[1] += ep.coef[j] * p01.y;
            v[2] += ep.coef[j] * p23.x;
            v[3] += ep.coef[j] * p23.y;
        }
    }
    if (ep.add) {
        const double* ap = ep.add + (long long)b * ep.add_bstride + off;
        const double2 a01 = *reinterpret_cast<const double2*>(ap);
        const double2 a23 = *reinterpret_cast<const double2*>(ap + 2);
        v[0] += ep.add_coef * a01.x;
        v[1] += ep.add_coef * a01.y;
        v[2] += ep.add_coef * a23.x;
        v[3] += ep.add_coef * a23.y;
    }
}

__device__ __forceinline__ void epilogue_store(const Epilogue& ep, int b, int row, int col, int n,
                                               double v) {
    ep.out[(long long)b * ep.out_bstride + (long long)row * n + col] = v;
    if (ep.low_fmt != MPPS_FMT_NONE) {
        const int lf = ep.low_fmt == MPPS_FMT_DEVICE ? __ldg(ep.low_fmt_dev) : ep.low_fmt;
        if (lf >= MPPS_FMT_BF16X3 && lf <= MPPS_FMT_BF16)
            store_low(lf, ep.low_hi, ep.low_lo,
                      (long long)b * ep.low_bstride + (long long)row * ep.lld + col,
                      mul_pow2(v, ep.low_scale_b ? ep.low_scale_b[b] : ep.low_scale));
    }
}

// ---- launchers (defined in the .cu files) ----------------------------------------
// FP64 product C = A B on the FP64 tensor pipe (DMMA), batch-strided, fused epilogue.
// bidx (device, optional): grid slice z processes matrix bidx[z] (for batches in which only
// some matrices take a step, e.g. squarings with per-matrix counts).
mpps_status launch_gemm_f64(const double* A, long long a_bs, const double* B, long long b_bs,
                            int n, int batch, const Epilogue& ep, cudaStream_t st,
                            const int* bidx = nullptr);

// Block scales of an FP8 product (tcgen05 kind::mxf8f6f4): one 8-bit code c (scale
// 2^(c - 127)) per row of A and per column of B per 32 entries of K.  Each array holds
// 512-byte chunks, one per (128 rows of A | 64 columns of B) x (128 entries of K): chunk
// (t, kc) at byte (t * kc_count + kc) * 512, and inside it row (column) r, K block j (0..3) at
// (r % 32) * 16 + (r / 32) * 4 + j -- the arrangement tcgen05.cp 32x128b.warpx4 carries into
// the TMEM words the MMA reads (lane r % 32, column r / 32, byte j).  a_bs, b_bs: bytes per
// matrix; kc = ceil(n / 128).
struct MxScales {
    const uint8_t* a;
    const uint8_t* b;
    long long a_bs, b_bs;
    int kc;
};
inline long long mx_scale_bytes_a(int n) { return (long long)((n + 127) / 128) * ((n + 127) / 128) * 512; }
inline long long mx_scale_bytes_b(int n) { return (long long)((n + 63) / 64) * ((n + 127) / 128) * 512; }

// Low-precision product on tcgen05: A_low (row-major, K-major, ld = lld) times B_low^T
// where B_low holds B transposed (row j = column j of B), in format fmt.  acc * alpha is
// passed to the epilogue (alpha undoes the operand scales).  FP8 needs the block scales mx.
mpps_status launch_gemm_tc(int fmt, const void* A_hi, const void* A_lo, const void* Bt_hi,
                           const void* Bt_lo, long long a_bs, long long b_bs, int lld, int n,
                           int batch, const Epilogue& ep, int* d_err, cudaStream_t st,
                           const MxScales* mx = nullptr);

// Workspace of a plain FP8 product C = A B with block scales (fp8mx_ws_bytes bytes, carved
// by fp8mx_ws_carve from a 256-byte aligned base) and the product itself: both conversions,
// then the block-scaled tcgen05 product with the row and column exponents undone in the
// epilogue (ep.row_exp / ep.col_exp are set here).
struct Fp8MxWs {
    uint8_t *qa, *qb, *sfa, *sfb;
    int *ea, *eb;
    unsigned long long* cmax;
};
size_t fp8mx_ws_bytes(int n, int batch);
Fp8MxWs fp8mx_ws_carve(void* base, int n, int batch);
mpps_status launch_product_fp8mx(const double* A, long long a_bs, const double* B, long long b_bs,
                                 int n, int batch, Epilogue ep, const Fp8MxWs& w, int* d_err,
                                 cudaStream_t st);

// FP64-accurate product from exact bf16 slices (gemm_f64e.cu).  Slice planes of A (rows)
// and of B^T (rows of B^T = columns of B) come from launch_slice_rows; eA/eB are the
// per-row exponents it returns.  Planes: [batch][k][n][low_ld(n)] bf16.
size_t f64e_plane_elems(int n, int batch, int k);
// gate (device, optional): the device plan's count; 0 = the launch does nothing.
mpps_status launch_slice_rows(const double* M, long long bs, int n, int batch, int k, void* planes,
                              int* exps, cudaStream_t st, const int* gate = nullptr);
// Column slices of M in the A operand's layout (the A operand M^T, no transpose formed),
// with per-column exponents; colmax: batch * n scratch words.
mpps_status launch_slice_cols_a(const double* M, long long bs, int n, int batch, int k, void* planes,
                                int* exps, unsigned long long* colmax, cudaStream_t st);
// Column slices of M written as rows of the B^T planes; colmax: batch * n scratch words.
mpps_status launch_slice_cols(const double* M, long long bs, int n, int batch, int k, void* planes,
                              int* exps, unsigned long long* colmax, cudaStream_t st,
                              const int* gate = nullptr);
// The same two with the row / column maxima of |M| already known (recorded by the epilogue
// of the emulated product that wrote M, Epilogue::rmax / cmax): no reduction pass.  The row
// variant also zeroes rmax_clear ([batch][n], may be null) for the next product to fill.
// list (device, optional): grid slice z slices matrix list[z] (batch = the listed count),
// as the products' bidx: the squarings slice only the matrices they square.
mpps_status launch_slice_rows_pre(const double* M, long long bs, int n, int batch, int k,
                                  void* planes, int* exps, const int* rmax, int* rmax_clear,
                                  cudaStream_t st, const int* gate = nullptr,
                                  const int* list = nullptr);
mpps_status launch_slice_cols_pre(const double* M, long long bs, int n, int batch, int k,
                                  void* planes, int* exps, const int* cmax, cudaStream_t st,
                                  const int* gate = nullptr, const int* list = nullptr);
// Both of the above from one read of M (the operands of M M): rows into planesA with the
// recorded row codes rcodes, columns into planesB with the column codes ccodes.
mpps_status launch_slice_both_pre(const double* M, long long bs, int n, int batch, int k,
                                  void* planesA, int* expsA, const int* rcodes, void* planesB,
                                  int* expsB, const int* ccodes, cudaStream_t st,
                                  const int* gate = nullptr, const int* list = nullptr);
// Scratch that lets the emulated product split the K range of output tiles between CTAs
// (f64e_split_bytes() bytes, 256-byte aligned; its first f64e_split_flag_bytes() bytes
// zeroed by the caller before the first product that uses it, on the same stream).  Without
// it every CTA works on whole tiles.
size_t f64e_split_bytes();
size_t f64e_split_flag_bytes();
// k slices are used; ksA / ksB planes are stored per matrix (>= k); nmat matrices are
// stored, `batch` of them are processed (all, or those listed in bidx).
mpps_status launch_gemm_f64e(int k, const void* slicesA, int ksA, const int* eA,
                             const void* slicesBt, int ksB, const int* eB, int n, int batch,
                             int nmat, const Epilogue& ep, int* d_err, cudaStream_t st,
                             const int* bidx = nullptr, void* split = nullptr);
// Row slices of nI and column slices of nJ small tiles (n <= 64, even) in one launch, for
// a grid product (the planes and exponents of launch_slice_rows / launch_slice_cols).
mpps_status launch_slice_tiles(int k, const double* A, long long a_bs, int nI, const double* B,
                               long long b_bs, int nJ, int n, void* planesA, int* eA,
                               void* planesB, int* eB, cudaStream_t st);
// Grid mode (Epilogue::gnj = nmatB): the nmatA x nmatB products of every stored A matrix
// with every stored B matrix (k slices stored per matrix), whole tiles, no split.
mpps_status launch_gemm_f64e_grid(int k, const void* slicesA, const int* eA, int nmatA,
                                  const void* slicesBt, const int* eB, int nmatB, int n,
                                  const Epilogue& ep, int* d_err, cudaStream_t st);

// ---- LU factorisation with partial pivoting and the solve Q R = P (lu.cu) -----------
// Device workspace bytes of lu_solve_dev for one n x n system with k-slice products (k = 0:
// FP64 pipe).
size_t lu_workspace_bytes(int n, int k);
// R_b = Q_b^-1 P_b for b < batch (row-major, batch stride n^2, device pointers; R may be
// P).  info[b] (device) gets 0, or j + 1 for the first column j whose pivot is zero.
// d_err: the emulated products' error word (k > 0).
mpps_status lu_solve_dev(const double* Q, const double* P, double* R, int n, int batch, int k,
                         void* ws, int* info, int* d_err, cudaStream_t st);

// ---- measured choice of product schedules (autotune.cu) ---------------------------
constexpr int kTuneMaxCandidates = 4;
enum { TUNE_F64E_SPLIT = 0, TUNE_TC_WIDTH = 1 };
// Whether tuning is on (mpps_autotune_enable, or MPPS_AUTOTUNE=1).
bool tune_enabled();
// The tuned candidate for (kind, n, batch, variant) on the current device, or -1.
int tune_lookup(int kind, int n, int batch, int variant);
// Time launch(c) for c < ncand on stream st, record the fastest, leave its output.
mpps_status tune_run(int kind, int n, int batch, int variant, int ncand, cudaStream_t st,
                     const std::function<mpps_status(int)>& launch);

// Slice planes per operand of an emulated product MPPS_FMT_F64E(k): k, at most 8 (k = 9
// adds slice pairs, not slices).
inline int f64e_planes(int k) { return k < 8 ? k : 8; }

// Element size in bytes of a low-precision operand copy.
inline int low_elem_bytes(int fmt) {
    switch (fmt) {
        case MPPS_FMT_BF16: case MPPS_FMT_BF16X3: return 2;
        case MPPS_FMT_TF32: return 4;
        case MPPS_FMT_FP8: return 1;
        default: return 8;
    }
}
// Leading dimension of low-precision copies: n rounded up to 64 elements (keeps every
// row 16-byte aligned for TMA and the K extent a whole number of 128-byte rows).
inline int low_ld(int n) { return (n + 63) / 64 * 64; }

// Elementwise helpers (elementwise.cu).
// out = ep.alpha * extra + sum_j ep.coef[j] X_j  (extra may be null: treated as 0).
mpps_status launch_combine(int n, int batch, const double* extra, long long extra_bs,
                           const Epilogue& ep, cudaStream_t st);
// ||B_i||_1 (i = 0..r), ||X^s||_1, ||X||_1 per matrix: block_norms_count(m, s) values per
// matrix; the FP64 kernels' partial sums need block_norms_partial_elems(...) doubles.
int block_norms_count(int m, int s);
size_t block_norms_partial_elems(int n, int batch, int m, int s);
// After launch_block_norms_f32 on a general X: the matrices with a norm that is not finite
// (a power entry or a sum beyond FP32's range) get their norms recomputed in FP64 (redo:
// batch flags, scratch).
mpps_status launch_block_norms_redo(const double* pw, long long pw_bs, int n, int batch, int s,
                                    int m, const double* d_coeffs, double* partial, double* norms,
                                    int* redo, cudaStream_t st);
// The same norms in FP32 arithmetic, valid when ||X||_1 <= 1 (the scaled argument of exp):
// the block sums only steer the precision rule and the operand scales, where a relative
// error of 2^-20 is immaterial.  coeffs is the host array b_0..b_m.
size_t block_norms_f32_partial_elems(int n, int batch, int m, int s);
mpps_status launch_block_norms_f32(const double* pw, long long pw_bs, int n, int batch, int s,
                                   int m, const double* coeffs, double* partial, double* norms,
                                   cudaStream_t st, bool power_norms = false);
// power_norms: ||X_2||_1..||X_{h}||_1 (h = ceil(s/2)) follow the r + 3 usual outputs of each
// matrix (the chain powers of the power tree), block_norms_f32_power_norms(m, s) of them (0:
// not available for this m, s); partial then needs block_norms_f32_powers_partial_elems.
int block_norms_f32_power_norms(int m, int s);
size_t block_norms_f32_powers_partial_elems(int n, int batch, int m, int s);
// ||M||_1 per matrix (partial: norm1_partial_elems doubles).
size_t norm1_partial_elems(int n, int batch);
mpps_status launch_norm1(const double* M, long long bs, int n, int batch, double* partial,
                         double* norms, cudaStream_t st);
// X = 2^-sigma[b] A (exact power-of-two scaling; d_sigma null -> plain copy).
mpps_status launch_scale_copy(const double* A, long long a_bs, double* X, long long x_bs, int n,
                              int batch, const int* d_sigma, cudaStream_t st);
// bytes of host memory written to dst (16-byte aligned) by kernels that carry them as
// parameters: no host memory is read by the stream (capturable), whatever its kind.
mpps_status launch_fill_bytes(void* dst, const void* host, size_t bytes, cudaStream_t st);
// dst[0..count) = host_vals (device write from kernel parameters; capturable).
mpps_status launch_fill(double* dst, const double* host_vals, int count, cudaStream_t st);
// FP32 storage: x = (double)a (exact) and a = (float)x (round to nearest), count elements.
mpps_status launch_widen_f32(const float* a, double* x, long long count, cudaStream_t st);
mpps_status launch_narrow_f64(const double* x, float* a, long long count, cudaStream_t st);
// One member of an uneven batch (device pointers), for the padded gather / scatter.
struct PadItem {
    const double* A;
    double* out;
    int n;
    int pad_;
};
mpps_status launch_gather_pad(const PadItem* d_list, int count, int n_pad, double* dst,
                              cudaStream_t st);
mpps_status launch_scatter_unpad(const PadItem* d_list, int count, int n_pad, const double* src,
                                 cudaStream_t st);
// sigma[b] = max(0, ceil(log2 norms[b])) on the device.
mpps_status launch_sigma(const double* norms, int batch, int* sigma, cudaStream_t st);
// out[b] = (sigma[b] odd ? q1 : q0)[b] + diag I  (all contiguous, stride n*n).
// sigma_cap >= 0: matrices with sigma above it get NaN (squarings launched blind).
mpps_status launch_select_copy(const double* q0, const double* q1, const int* d_sigma, double* out,
                               int n, int batch, double diag, cudaStream_t st, int sigma_cap = -1);
// Rounded copies (times scale[b], or 1 if scale is null) for the low-precision products:
// convert keeps the layout, convert_t writes the transpose (row j = column j).
mpps_status launch_convert(int fmt, const double* M, long long bs, int n, int batch, void* hi,
                           void* lo, long long low_bs, int lld, const double* d_scale,
                           bool transpose, cudaStream_t st, const int* gate = nullptr);
// max_ij |M_ij| per matrix, written to out[b] (out must be zeroed first).
// FP8 (E4M3) copy with block scales, the operands of a block-scaled product: each row of M
// (transpose = false, the A operand) or each column (transpose = true, written transposed:
// row j = column j of M, the B^T operand) first gets its own power of two (largest magnitude
// below 1; the exponent that undoes it goes to out_exp[batch][n]), then every 32 consecutive
// entries along K a power-of-two scale code (in sf, the MxScales arrangement, sf_bs bytes per
// matrix; mx_scale_bytes_a / _b) and their E4M3 values (q, row pitch lld bytes, q_bs bytes per
// matrix).  colmax: batch * n scratch words (transpose only).
mpps_status launch_convert_mx(const double* M, long long bs, int n, int batch, uint8_t* q,
                              long long q_bs, int lld, uint8_t* sf, long long sf_bs, bool transpose,
                              int* out_exp, unsigned long long* colmax, cudaStream_t st,
                              const int* gate = nullptr);
mpps_status launch_maxabs(const double* M, long long bs, int n, int batch, double* out,
                          cudaStream_t st);
// For each matrix b: scale[b] = 2^(target - e) and unscale... (power-of-two operand scales)
mpps_status launch_pow2_scales(const double* maxabs_a, const double* maxabs_b, int batch,
                               int target_exp, double* scale_a, double* scale_b,
                               double* unscale, cudaStream_t st);
// X_j += c_j * G for j = 1..t (power-table adjoint of a block sum); c is a host array.
mpps_status launch_axpy_blocks(double* xbar, long long xbar_bs, int n, int batch, int t,
                               const double* c, const double* G, long long g_bs,
                               cudaStream_t st);
// At = A^T per matrix (A with batch stride a_bs, At contiguous).
mpps_status launch_transpose(const double* A, long long a_bs, double* At, int n, int batch,
                             cudaStream_t st);

}  // namespace mpps
