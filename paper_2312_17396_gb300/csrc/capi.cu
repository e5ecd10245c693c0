// capi.cu -- the C ABI of include/mpps.h: argument checks, the host precision planner
// (eq. (2.8), Algorithm 3.1 `fix_params` branch, Algorithm 4.1), workspace layout and the
// order of kernel launches for ps_eval, expm_taylor_ss, ps_eval_adjoint and mpps_matmul.
#include "common.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>


#include <algorithm>
#include <initializer_list>
#include <mutex>
#include <vector>

namespace mpps {

// ---- errors -------------------------------------------------------------------------
static thread_local char g_err[1024];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = '\0'; }

// ---- policy -------------------------------------------------------------------------
struct Pol {
    int mode;
    double tol, delta;
    int s;
    unsigned formats;
    int floor_steps;
    int f64k;   // 0: FP64 pipe; k > 0: working-precision products emulated with k slices
    int var_s;  // variable-s branch of Algorithm 3.1
    int recompute;  // adjoints: checkpoint the Horner iterates, recompute the rest
    int dplan;      // precision rule on the device
    int max_sq;     // expm, device plan: squaring steps launched (0: sigma read back)
    int mixp;       // mixed-precision powers (power tree with cheaper leaves)
};

static Pol resolve(const mpps_policy* p) {
    mpps_policy d;
    mpps_policy_default(&d);
    if (!p) p = &d;
    Pol r;
    r.mode = p->mode;
    r.tol = p->tol > 0 ? p->tol : 0x1p-53;
    r.delta = p->delta > 0 ? p->delta : 10.0;
    r.s = p->s;
    r.formats = (p->formats ? p->formats : 0x1Fu) | 1u;
    r.floor_steps = p->fp64_floor_steps < 0 ? 2 : p->fp64_floor_steps;
    r.f64k = p->f64_slices;
    r.var_s = p->variable_s != 0;
    r.recompute = p->adjoint_recompute != 0;
    r.dplan = p->device_plan != 0;
    r.max_sq = p->max_squarings > 0 ? p->max_squarings : 0;
    r.mixp = p->mixed_powers != 0;
    return r;
}

static int ceil_sqrt_int(int m) {
    if (m <= 1) return 1;
    int s = (int)sqrt((double)m);
    while (s * s < m) ++s;
    while (s > 1 && (s - 1) * (s - 1) >= m) --s;
    return s;
}

// Variable-s branch of Algorithm 3.1: entered when ||X||_1 <= s0/e (s0 = ceil(sqrt(m)));
// s then grows while ||Y|| > ||B_0|| ||X||^s and s < m (||X||^s by repeated multiplication).
static bool var_s_grow(int m, int s, double normX, double normB0, double normY) {
    if (s >= m || s >= MPPS_MAX_S) return false;
    double xs = 1.0;
    for (int j = 0; j < s; ++j) xs *= normX;
    return normY > normB0 * xs;
}

extern "C" int mpps_choose_s(int m, double normX, const double* normB0, const double* normY,
                             int len) {
    if (m < 1 || len < 1 || !normB0 || !normY) return -1;
    const int s0 = ceil_sqrt_int(m);
    const double kE = 2.718281828459045;   // e
    if (!(normX <= (double)s0 / kE)) return s0;
    int k = 0;
    while (k < len && var_s_grow(m, s0 + k, normX, normB0[k], normY[k])) ++k;
    return s0 + k;
}

// unit roundoff of the rounded inputs of each format, and the FP32 accumulation unit
__host__ __device__ inline double u_fmt(int f) {
    switch (f) {
        case MPPS_FMT_FP64: return 0x1p-53;
        case MPPS_FMT_BF16X3: return 0x1p-16;
        case MPPS_FMT_TF32: return 0x1p-11;
        case MPPS_FMT_BF16: return 0x1p-8;
        case MPPS_FMT_FP8: return 0x1p-4;
        default: return 1.0;
    }
}

__host__ __device__ inline bool is_low(int f) { return f >= MPPS_FMT_BF16X3 && f <= MPPS_FMT_FP8; }

// Unit roundoff assigned to an emulated product F64E(k): 2^(2-7k) for k <= 8 slices of 7 bits
// (the slices keep 7k bits below the row/column maxima; the constant covers the dropped pairs
// t + q >= k); 2^-55 for k = 9 (8 slices, pairs up to order 8: the 2^-57 residual of each
// operand dominates).
__host__ __device__ inline double u_f64e(int k) { return k <= 8 ? ldexp(1.0, 2 - 7 * k) : 0x1p-55; }

static double unit_roundoff(int f) {
    if (MPPS_FMT_IS_F64E(f)) return u_f64e(MPPS_F64E_SLICES(f));
    return (f >= 0 && f < MPPS_NUM_FORMATS) ? u_fmt(f) : 1.0;
}

// Precision rank: larger = more precise (used to run a batch step at its most precise ask).
__host__ __device__ inline int prec_rank(int f) {
    if (f == MPPS_FMT_FP64) return 1000;
    if (MPPS_FMT_IS_F64E(f)) return 100 + MPPS_F64E_SLICES(f);
    switch (f) {
        case MPPS_FMT_BF16X3: return 4;
        case MPPS_FMT_TF32: return 3;
        case MPPS_FMT_BF16: return 2;
        case MPPS_FMT_FP8: return 1;
        default: return 0;
    }
}

// Smallest emulated slice count that always counts as "cheaper than the working precision".
constexpr int kF64eMinRung = 4;

// Planner for one matrix.  normB: r+1 norms ||B_0||..||B_r||; normY = ||X^s||.
// div > 1 tightens every u_i of eq. (2.8) by that factor before nu and the formats are chosen
// (the rule of the reverse pass, see plan_adjoint_divisor); div = 1 is the forward rule.
// The leaves of the power tree (policy.mixed_powers): with h = ceil(s/2), X^2..X^h come from
// the chain, Y = X^h X^(s-h), and X^j = X^h X^(j-h) for j = h+1..s-1 feed only the block sums.
// A leaf's product error (about u_F64E(k) ||X^h|| ||X^(j-h)||) reaches p through
// sum_i |b_{si+j}| ||Y||^i; with L leaves sharing eq. (2.8)'s budget ||B_0|| tol, leaf j takes
// the fewest slices whose unit roundoff is at most
//   u_j = ||B_0||_low tol / (L ||X^h|| ||X^(j-h)|| sum_{i: si+j <= m} |b_{si+j}| ||Y||^i).
// The norms are those of the chain powers and of the blocks without their leaf terms
// (normBpart); normB_out gets a lower bound of ||B_0|| and upper bounds of ||B_i||, i >= 1,
// for the block rule.
static bool forms_power_tree(const Pol& P, int s) {
    return P.mixp && P.mode != MPPS_FIXED_FP64 && P.f64k > 0 && s >= 4;
}

static void plan_powers_core(int m, int s, const double* c, const double* nxp, const double* nbp,
                             const Pol& P, int* fmt, double* nbo) {
    const int r = m / s, h = (s + 1) / 2, L = s - h - 1;
    const int wp = MPPS_FMT_F64E(P.f64k);
    for (int j = 0; j <= s; ++j) fmt[j] = j < 2 ? MPPS_FMT_NONE : wp;
    double extra[MPPS_MAX_R + 1];
    for (int i = 0; i <= r; ++i) extra[i] = 0.0;
    for (int j = h + 1; j < s; ++j) {
        const double bx = nxp[h - 1] * nxp[j - h - 1];   // ||X^h|| ||X^(j-h)|| >= ||X^j||
        for (int i = 0; i <= r && s * i + j <= m; ++i) extra[i] += fabs(c[s * i + j]) * bx;
    }
    nbo[0] = nbp[0] - extra[0] > 0.0 ? nbp[0] - extra[0] : 0.0;
    for (int i = 1; i <= r; ++i) nbo[i] = nbp[i] + extra[i];
    const double y = nxp[s - 1];
    for (int j = h + 1; j < s; ++j) {
        const double bx = nxp[h - 1] * nxp[j - h - 1];
        double sum = 0.0, yi = 1.0;
        for (int i = 0; i <= r && s * i + j <= m; ++i) {
            sum += fabs(c[s * i + j]) * yi;
            yi = yi * y;
        }
        const double den = (double)L * bx * sum;
        const double uj = den == 0.0 ? (double)INFINITY : nbo[0] * P.tol / den;
        for (int k = kF64eMinRung; k < P.f64k; ++k)
            if (u_f64e(k) <= uj) {
                fmt[j] = MPPS_FMT_F64E(k);
                break;
            }
    }
}

static mpps_status plan_steps(int m, int n, const double* normB, double normY, const Pol& P,
                              double div, mpps_report* out);
static mpps_status plan_one(int m, int n, const double* normB, double normY, const Pol& P,
                            mpps_report* out) {
    return plan_steps(m, n, normB, normY, P, 1.0, out);
}

// Reverse pass (the paper states no adjoint).  The gradient of a degree-k term b_k X^k is a
// sum of k products X^j E X^(k-1-j), each as large as the term itself times ||E||/||X||, so
// relative to the value the high-order blocks weigh up to m/||X|| times more in the gradient
// than in p(X), while the reference (the low-order block) keeps its weight.  The products of
// reverse step i therefore run in the format the forward rule picks for u_i / d with
// d = m / min(1, ||X||_1).
static double plan_adjoint_divisor(int m, double normX) {
    const double x = (normX > 0.0 && normX < 1.0) ? normX : 1.0;
    return (double)m / x;
}

__host__ __device__ void plan_core(int n, int r, int fold, const double* normB, double normY,
                                   const Pol& P, double div, double* u, int* fmt, int* nu_out);

static mpps_status plan_steps(int m, int n, const double* normB, double normY, const Pol& P,
                              double div, mpps_report* out) {
    memset(out, 0, sizeof(*out));
    for (int i = 0; i <= MPPS_MAX_R; ++i) out->fmt[i] = MPPS_FMT_NONE;
    for (int j = 0; j <= MPPS_MAX_S; ++j) out->pow_fmt[j] = MPPS_FMT_NONE;
    if (m == 0) {
        out->s = 1; out->r = 0; out->nu = 1;
        out->normB[0] = normB ? normB[0] : 0.0;
        out->cost_ratio = 1.0;
        return MPPS_OK;
    }
    int s = P.s > 0 ? std::min(P.s, m) : ceil_sqrt_int(m);
    if (s > MPPS_MAX_S) {
        set_error("block size s=%d exceeds %d", s, MPPS_MAX_S);
        return MPPS_EINVAL;
    }
    if (P.f64k < 0 || P.f64k > MPPS_F64E_MAX_SLICES) {
        set_error("f64_slices=%d outside 0..%d", P.f64k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const int r = m / s;
    if (r > MPPS_MAX_R) {
        set_error("r=floor(m/s)=%d exceeds %d", r, MPPS_MAX_R);
        return MPPS_EINVAL;
    }
    out->s = s;
    out->r = r;
    out->fold = (m % s == 0) ? 1 : 0;
    out->normY = normY;
    for (int i = 0; i <= r; ++i) out->normB[i] = normB[i];
    plan_core(n, r, out->fold, normB, normY, P, div, out->u, out->fmt, &out->nu);
    return MPPS_OK;
}

// eq. (2.8), nu and the format ladder for one matrix, shared by the host planner and the
// device planner (the same operations in the same order: the plans agree bit for bit).
// u and fmt: MPPS_MAX_R + 1 entries, steps 1..r written (fmt[r] = NONE when s | m).
__host__ __device__ void plan_core(int n, int r, int fold, const double* normB, double normY,
                                   const Pol& P, double div, double* u, int* fmt, int* nu_out) {
    const double tol = P.tol;
    // eq. (2.8) with nu = 1, clamped at the working precision
    for (int i = 1; i <= r; ++i) {
        double yi = 1.0;
        for (int k = 0; k < i; ++k) yi = yi * normY;
        const double den = normB[i] * yi;
        double ui = (den == 0.0) ? (double)INFINITY : (normB[0] * tol) / den;
        if (div != 1.0) ui = ui / div;
        u[i] = (ui > tol) ? ui : tol;
    }
    // nu: first step allowed below the working precision; earlier steps get u
    int nu = r + 1;
    for (int i = 1; i <= r; ++i)
        if (u[i] >= P.delta * tol) { nu = i; break; }
    for (int i = 1; i < nu; ++i) u[i] = tol;
    *nu_out = nu;
    // formats: cheapest allowed with unit roundoff <= u_i (and FP32 accumulation <= u_i for
    // the hardware formats); with emulation on, the slice counts 4..k-1 sit between BF16X3
    // and the working precision (their accumulation is exact)
    const int order[4] = {MPPS_FMT_FP8, MPPS_FMT_BF16, MPPS_FMT_TF32, MPPS_FMT_BF16X3};
    const int wp = P.f64k > 0 ? MPPS_FMT_F64E(P.f64k) : MPPS_FMT_FP64;
    for (int i = 1; i <= r; ++i) {
        int f = wp;
        const bool floor_fp64 = (P.mode == MPPS_MIXED_NS && i <= P.floor_steps);
        if (P.mode != MPPS_FIXED_FP64 && !floor_fp64) {
            bool found = false;
            for (int k = 0; k < 4 && !found; ++k) {
                const int F = order[k];
                if (!((P.formats >> F) & 1u)) continue;
                if (u_fmt(F) <= u[i] && (double)n * 0x1p-24 <= u[i]) { f = F; found = true; }
            }
            for (int k = kF64eMinRung; k < P.f64k && !found; ++k)
                if (u_f64e(k) <= u[i]) { f = MPPS_FMT_F64E(k); found = true; }
        }
        fmt[i] = f;
    }
    if (fold) fmt[r] = MPPS_FMT_NONE;
}

// ---- the precision rule on the device ------------------------------------------------
// The call's plan in device memory: the batch's format of each Horner step and, for every
// format code, the number of matrices a launch of that format processes (the batch size if
// the step runs in it, else 0: the gated candidate launches read these counts).
constexpr int kSlots = 32;   // format codes: 0..4, MPPS_FMT_F64E(k) = 16 + k
__host__ __device__ inline int fmt_slot(int f) { return f >= 0 && f < kSlots ? f : kSlots - 1; }
constexpr int kYAnyF64e = 5;  // ycnt slot: some step runs an emulated product
struct DevPlan {
    int fmt[MPPS_MAX_R + 1];
    int cnt[MPPS_MAX_R + 1][kSlots];
    int ycnt[8];   // [f], f = 1..4: some step uses low format f (Y's rounded copy); [5]: F64E
};

__device__ __forceinline__ int exp_above_dev(double x) {   // e with x < 2^e (x > 0), else 0
    if (!(x > 0.0) || !isfinite(x)) return 0;
    int e;
    frexp(x, &e);
    return e;
}

// One block.  Per matrix: plan_core on its norms (eta_0..eta_r, ||Y||, ||X|| at stride q),
// the report fields, and the power-of-two operand scales of its low-precision steps (the
// host planner's arithmetic: beta_i = eta_i + ||Y|| beta_{i+1} with the multiply and the add
// rounded separately).
__global__ void k_plan(const double* __restrict__ norms, int q, int batch, int n, int r, int fold,
                       Pol P, DevPlan* __restrict__ dp, int* __restrict__ rep_fmt,
                       double* __restrict__ rep_u, int* __restrict__ rep_nu, double* __restrict__ sY,
                       double* __restrict__ sP, double* __restrict__ al) {
    pdl_wait();
    __shared__ int key[MPPS_MAX_R + 1];
    __shared__ int sfmt[MPPS_MAX_R + 1];
    for (int i = threadIdx.x; i <= MPPS_MAX_R; i += blockDim.x) key[i] = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
        const double* eta = norms + (size_t)b * q;
        double u[MPPS_MAX_R + 1];
        int f[MPPS_MAX_R + 1];
        int nu = 1;
        for (int i = 0; i <= MPPS_MAX_R; ++i) { u[i] = 0.0; f[i] = MPPS_FMT_NONE; }
        plan_core(n, r, fold, eta, eta[r + 1], P, 1.0, u, f, &nu);
        rep_nu[b] = nu;
        for (int i = 0; i <= r; ++i) {
            rep_fmt[(size_t)b * (MPPS_MAX_R + 1) + i] = f[i];
            rep_u[(size_t)b * (MPPS_MAX_R + 1) + i] = u[i];
        }
        for (int i = 1; i <= r; ++i) atomicMax(&key[i], prec_rank(f[i]) * 64 + (f[i] + 1));
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= MPPS_MAX_R; i += blockDim.x) {
        int fi = (i >= 1 && i <= r && key[i] > 0) ? (key[i] & 63) - 1 : MPPS_FMT_NONE;
        if (fold && i == r) fi = MPPS_FMT_NONE;
        sfmt[i] = fi;
        dp->fmt[i] = fi;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (MPPS_MAX_R + 1) * kSlots; t += blockDim.x) {
        const int i = t / kSlots, c = t % kSlots;
        dp->cnt[i][c] = (sfmt[i] != MPPS_FMT_NONE && fmt_slot(sfmt[i]) == c) ? batch : 0;
    }
    if (threadIdx.x < 8) {
        const int f = threadIdx.x;
        bool used = false;
        for (int i = 1; i <= r; ++i)
            used = used || (f >= 1 && f <= 4 && sfmt[i] == f) ||
                   (f == kYAnyF64e && MPPS_FMT_IS_F64E(sfmt[i]));
        dp->ycnt[f] = used ? batch : 0;
    }
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
        const double* eta = norms + (size_t)b * q;
        const double y = eta[r + 1];
        const int eY = exp_above_dev(y);
        for (int f = 0; f < MPPS_NUM_FORMATS; ++f)
            sY[(size_t)f * batch + b] = f == 0 ? 1.0 : ldexp(1.0, (f == MPPS_FMT_FP8 ? 8 : 0) - eY);
        double beta = 0.0;
        sP[b] = 1.0;
        al[b] = 1.0;
        for (int i = r; i >= 1; --i) {
            beta = __dadd_rn(eta[i], __dmul_rn(y, beta));
            double p = 1.0, a = 1.0;
            if (is_low(sfmt[i])) {
                const int T = sfmt[i] == MPPS_FMT_FP8 ? 8 : 0;
                const int eP = exp_above_dev(beta);
                p = ldexp(1.0, T - eP);
                a = ldexp(1.0, eP + eY - 2 * T);
            }
            sP[(size_t)i * batch + b] = p;
            al[(size_t)i * batch + b] = a;
        }
    }
}

// Squaring lists on the device (max_squarings steps): list k holds, in ascending order, the
// matrices with sigma > k, and count k their number.  A matrix with sigma above the number of
// steps sets bit 1 of the error word.  One block.
__global__ void k_sq_lists(const int* __restrict__ sigma, int batch, int steps, int* __restrict__ lists,
                           int* __restrict__ counts, int* __restrict__ err) {
    pdl_wait();
    __shared__ int part[1024];
    for (int k = 0; k < steps; ++k) {
        int base = 0;
        for (int b0 = 0; b0 < batch; b0 += blockDim.x) {
            const int b = b0 + threadIdx.x;
            const int on = (b < batch && sigma[b] > k) ? 1 : 0;
            part[threadIdx.x] = on;
            __syncthreads();
            for (int o = 1; o < (int)blockDim.x; o <<= 1) {   // inclusive scan
                const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
                __syncthreads();
                part[threadIdx.x] += v;
                __syncthreads();
            }
            if (on) lists[(size_t)k * batch + base + part[threadIdx.x] - 1] = b;
            const int tot = part[blockDim.x - 1];
            __syncthreads();
            base += tot;
        }
        if (threadIdx.x == 0) counts[k] = base;
    }
    for (int b = threadIdx.x; b < batch; b += blockDim.x)
        if (sigma[b] > steps) atomicOr(err, 2);
}

// eq. (3.8): ((s-1) D + sum d_i) / ((s+r-1) D), D = digits of u, d_i = digits of the
// format that ran step i (0 for a step without a product).
static double cost_ratio(const mpps_report& rp, double tol) {
    const double D = -log10(tol);
    double sum = 0.0;
    for (int i = 1; i <= rp.r; ++i)
        if (rp.fmt[i] >= 0) sum += std::min(D, -log10(unit_roundoff(rp.fmt[i])));
    const double den = (rp.s + rp.r - 1) * D;
    return den > 0 ? ((rp.s - 1) * D + sum) / den : 1.0;
}

// ---- workspace ----------------------------------------------------------------------
struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Workspaces come from a private stream-ordered pool per device that keeps freed memory
// (release threshold = all of it): with the default threshold of 0 every synchronisation
// would hand the previous call's workspace back to the driver and the next call would map
// it again.  mpps_release_workspace() trims the pools.
static std::mutex g_poolmu;
static cudaMemPool_t g_pool[64];

static mpps_status workspace_pool(cudaMemPool_t* out) {
    int dev = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return MPPS_ENOTSUP;
    }
    std::lock_guard<std::mutex> lk(g_poolmu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        MPPS_CUDA_TRY(cudaMemPoolCreate(&g_pool[dev], &props));
        uint64_t keep = ~(uint64_t)0;
        MPPS_CUDA_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    *out = g_pool[dev];
    return MPPS_OK;
}

static bool is_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, st);
    }
    mpps_status alloc(size_t bytes, cudaStream_t s) {
        st = s;
        if (bytes == 0) bytes = 256;
        // while the stream is captured into a CUDA graph the allocation becomes a graph
        // memory node of the device's default pool (its address is fixed for the graph)
        cudaError_t e;
        if (is_capturing(s)) {
            e = cudaMallocAsync(&p, bytes, s);
        } else {
            cudaMemPool_t pool = nullptr;
            mpps_status rc = workspace_pool(&pool);
            if (rc) return rc;
            e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
        }
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            set_error("cudaMallocFromPoolAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? MPPS_ENOMEM : MPPS_ECUDA;
        }
        return MPPS_OK;
    }
};

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Every kernel of a call runs on the current device, so a device pointer that lives on
// another GPU would make them touch that GPU's memory: rejected before any work.
static mpps_status check_same_device(const char* fn, std::initializer_list<const void*> ptrs) {
    int cur = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&cur));
    for (const void* p : ptrs) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (a.type == cudaMemoryTypeDevice && a.device != cur) {
            set_error("%s: a matrix pointer lives on device %d but device %d is current", fn,
                      a.device, cur);
            return MPPS_EINVAL;
        }
    }
    return MPPS_OK;
}

static int low_target_exp(int f) { return f == MPPS_FMT_FP8 ? 8 : 0; }

static int exp_above(double x) {   // e with x < 2^e (x > 0), 0 otherwise
    if (!(x > 0.0) || !isfinite(x)) return 0;
    int e;
    frexp(x, &e);
    return e;
}

// ---- sticky per-device error word of the bounded waits --------------------------------
// The tensor-core kernels set *err when a bounded wait gives up.  Instead of synchronising
// every call to read it, each call enqueues a copy of the word into pinned host memory
// behind an event; the word is reported (and cleared) by the first later call on the device
// that finds the event complete, or at once by calls that synchronise anyway.
struct DevErr {
    int* d = nullptr;
    int* h = nullptr;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};
static std::mutex g_errmu;
static DevErr g_deverr[64];

static mpps_status dev_err_get(DevErr** out) {
    int dev = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return MPPS_ENOTSUP;
    }
    std::lock_guard<std::mutex> lk(g_errmu);
    DevErr& e = g_deverr[dev];
    if (!e.d) {
        MPPS_CUDA_TRY(cudaMalloc(&e.d, sizeof(int)));
        MPPS_CUDA_TRY(cudaMemset(e.d, 0, sizeof(int)));
        MPPS_CUDA_TRY(cudaHostAlloc(&e.h, sizeof(int), cudaHostAllocDefault));
        *e.h = 0;
        MPPS_CUDA_TRY(cudaEventCreateWithFlags(&e.ev, cudaEventDisableTiming));
    }
    *out = &e;
    return MPPS_OK;
}

// Report a failure recorded by an earlier call (if its copy has landed).  `wait` forces the
// check (used right after a stream synchronisation).
static mpps_status dev_err_check(DevErr* e, bool wait) {
    std::lock_guard<std::mutex> lk(g_errmu);
    if (!e->pending) return MPPS_OK;
    if (!wait) {
        cudaError_t q = cudaEventQuery(e->ev);
        if (q == cudaErrorNotReady) return MPPS_OK;
        if (q != cudaSuccess) {
            set_error("cudaEventQuery failed: %s", cudaGetErrorString(q));
            return MPPS_ECUDA;
        }
    } else {
        MPPS_CUDA_TRY(cudaEventSynchronize(e->ev));
    }
    e->pending = false;
    if (*e->h) {
        const int v = *e->h;
        *e->h = 0;
        MPPS_CUDA_TRY(cudaMemset(e->d, 0, sizeof(int)));
        if (v & 1) {
            set_error("a bounded wait in a tensor-core product timed out (device error word set)");
            return MPPS_ETIMEOUT;
        }
        set_error("a matrix needed more squarings than policy.max_squarings (its result is NaN)");
        return MPPS_ECHECK;
    }
    return MPPS_OK;
}

static mpps_status dev_err_enqueue(DevErr* e, cudaStream_t st) {
    // under stream capture the word stays on the device; the next call outside a capture
    // copies and reports it
    if (is_capturing(st)) return MPPS_OK;
    std::lock_guard<std::mutex> lk(g_errmu);
    MPPS_CUDA_TRY(cudaMemcpyAsync(e->h, e->d, sizeof(int), cudaMemcpyDeviceToHost, st));
    MPPS_CUDA_TRY(cudaEventRecord(e->ev, st));
    e->pending = true;
    return MPPS_OK;
}

// ---- forward state kept for a reverse pass (the adjoint's tape) -----------------------
// Where the forward pass leaves the power table and the Horner iterates P_1..P_top
// (top = r, or r - 1 when s divides m).  All iterates are kept, or (recompute) every c-th
// with c = ceil(sqrt(r)) and the top one; the others go to two rolling slots and are
// recomputed a segment at a time by the reverse pass.
struct TapeLayout {
    int s = 0, r = 0, fold = 0, i_top = 0;
    int recompute = 0, cseg = 1, ck_top = 0, seg0 = 0, nslots = 0;
    size_t pw_off = 0, slot_off = 0, hdr_off = 0, bytes = 0;
    bool is_ckpt(int j) const { return !recompute || j % cseg == 0 || j == i_top; }
    int ck_slot(int j) const { return !recompute ? j : (j == i_top ? ck_top : j / cseg); }
    int fwd_slot(int j) const { return is_ckpt(j) ? ck_slot(j) : seg0 + (j & 1); }
};

// Per-step formats of the forward and of the reverse Horner products, and the checks that
// tie a tape to its call.
struct TapeHeader {
    int magic, m, n, batch, s, r, storage, pad_;
    int fmt[MPPS_MAX_R + 1];
    int fmt_adj[MPPS_MAX_R + 1];
};
static const int kTapeMagic = 0x6d707073;

struct Keep {
    const TapeLayout* L;
    double* pw;                      // power table [batch][s][n][n]
    double* slots;                   // iterate slots [nslots][batch][n][n]
    int fmt[MPPS_MAX_R + 1];         // out: the batch's format of each Horner step
    std::vector<mpps_report> plans;  // out: per-matrix plans (u_i, norms)
};

// Formats the rule may pick for Horner step i, before the norms are known (device plan):
// the working precision first, then, unless the step is fixed to it, every allowed
// low-precision format and the emulated slice counts below the working precision.
static std::vector<int> step_candidates(const Pol& P, int r, bool fold, int i) {
    std::vector<int> c;
    if (fold && i == r) return c;
    c.push_back(P.f64k > 0 ? MPPS_FMT_F64E(P.f64k) : MPPS_FMT_FP64);
    if (P.mode == MPPS_FIXED_FP64 || (P.mode == MPPS_MIXED_NS && i <= P.floor_steps)) return c;
    for (int F : {MPPS_FMT_BF16X3, MPPS_FMT_TF32, MPPS_FMT_BF16, MPPS_FMT_FP8})
        if ((P.formats >> F) & 1u) c.push_back(F);
    for (int k = kF64eMinRung; k < P.f64k; ++k) c.push_back(MPPS_FMT_F64E(k));
    return c;
}

// Page-locked staging for the early read of sigma (device plan), one per host thread and
// device, with the event that marks its copy.
struct SigmaStage {
    int* h = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    ~SigmaStage() {
        if (h) cudaFreeHost(h);
        if (ev) cudaEventDestroy(ev);
    }
};
static thread_local SigmaStage t_sig[64];

// Streams of a grouped call's buckets: created once per device (non-blocking), shared by
// the calls on that device; every use forks from and joins the caller's stream.
constexpr int kAuxStreams = 8;
static std::mutex g_auxmu;
static cudaStream_t g_aux[64][kAuxStreams];

static mpps_status aux_streams(int k, std::vector<cudaStream_t>* out) {
    int dev = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return MPPS_ENOTSUP;
    }
    std::lock_guard<std::mutex> lk(g_auxmu);
    out->clear();
    for (int j = 0; j < k && j < kAuxStreams; ++j) {
        if (!g_aux[dev][j]) MPPS_CUDA_TRY(cudaStreamCreateWithFlags(&g_aux[dev][j], cudaStreamNonBlocking));
        out->push_back(g_aux[dev][j]);
    }
    if (out->empty()) {
        set_error("no stream for the grouped call");
        return MPPS_ECUDA;
    }
    return MPPS_OK;
}

static mpps_status sigma_stage(int batch, SigmaStage** out) {
    int dev = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return MPPS_ENOTSUP;
    }
    SigmaStage& S = t_sig[dev];
    if (S.cap < (size_t)batch) {
        if (S.h) MPPS_CUDA_TRY(cudaFreeHost(S.h));
        S.h = nullptr;
        MPPS_CUDA_TRY(cudaHostAlloc(&S.h, sizeof(int) * (size_t)batch, cudaHostAllocDefault));
        S.cap = (size_t)batch;
    }
    if (!S.ev) MPPS_CUDA_TRY(cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming));
    *out = &S;
    return MPPS_OK;
}

// ---- the PS evaluation --------------------------------------------------------------
// Evaluates p(X) for a device batch; for expm, X = 2^-sigma A and sigma squarings follow.
// keep (not for expm): the power table and the Horner iterates go where *keep says.
static mpps_status eval_device(const double* coeffs, int m, const double* dA, int n, int batch,
                               const Pol& pol, double* dOut, mpps_report* rep, cudaStream_t st,
                               bool expm, bool sync_at_end, Keep* keep = nullptr,
                               const int* sig_dev = nullptr, const int* sig_host = nullptr) {
    const long long nn = (long long)n * n;
    // ---- m == 0: p = b_0 I
    if (m == 0) {
        Epilogue ep = epilogue_plain(dOut, nn);
        ep.nt = 0;
        ep.coef[0] = coeffs[0];
        ep.alpha = 0.0;
        mpps_status rc = launch_combine(n, batch, nullptr, 0, ep, st);
        if (rc) return rc;
        if (rep)
            for (int b = 0; b < batch; ++b) {
                double nb = fabs(coeffs[0]);
                plan_one(0, n, &nb, 0.0, pol, &rep[b]);
            }
        return MPPS_OK;
    }
    int s = pol.s > 0 ? std::min(pol.s, m) : ceil_sqrt_int(m);
    if (s > MPPS_MAX_S || m / s > MPPS_MAX_R) {
        set_error("m=%d with s=%d is outside the supported range (s<=%d, r<=%d)", m, s, MPPS_MAX_S,
                  MPPS_MAX_R);
        return MPPS_EINVAL;
    }
    // Variable s (Algorithm 3.1, fix_params false): s may grow after the powers, so the
    // power table has room for s_cap powers and the norm buffers for every s up to it.
    const bool var_s = pol.var_s && pol.s <= 0 && pol.mode != MPPS_FIXED_FP64 && m >= 2 && !keep;
    // Device plan: the rule runs on the GPU (k_plan); not with variable s or a tape
    const bool dp = pol.dplan && !var_s && !keep;
    const int sq_steps = (dp && expm) ? pol.max_sq : 0;   // squarings launched blind (0: read)
    // Mixed-precision powers (host plan, fixed s): the power tree of plan_powers_core, whose
    // leaves X^(h+1)..X^(s-1) are formed after the norms, in the slices the rule allows
    const bool mixp = forms_power_tree(pol, s) && !dp && !var_s && !keep;
    const int h = (s + 1) / 2;
    const int s0 = s;
    const int s_cap = var_s ? std::min(std::min(m, MPPS_MAX_S), 2 * s0) : s;
    int r = m / s;
    bool fold = (m % s) == 0;
    int q = block_norms_count(m, s);   // largest at the smallest s
    // mixed powers with exp: ||X^2||..||X^h|| come out of the FP32 block-norm pass as well
    const int ex_pn = (mixp && expm) ? block_norms_f32_power_norms(m, s) : 0;
    const int q_alloc = q + ex_pn;
    size_t partial_elems = norm1_partial_elems(n, batch);
    for (int t = s0; t <= s_cap; ++t)
        partial_elems = std::max(partial_elems,
                                 std::max(block_norms_partial_elems(n, batch, m, t),
                                          block_norms_f32_partial_elems(n, batch, m, t)));
    if (ex_pn > 0)
        partial_elems = std::max(partial_elems, block_norms_f32_powers_partial_elems(n, batch, m, s));
    const long long pw_bs = (long long)s_cap * nn;

    // ---- phase-1 workspace (FP64 part, and slice planes when FP64 is emulated)
    const int K = pol.f64k;                      // slices of an emulated working-precision product
    Arena L;
    double *d_coef, *pw, *Pb0, *Pb1, *partial, *norms, *d_anorm, *tmpT = nullptr, *d_pnorm = nullptr;
    int *d_sigma, *d_err, *d_bidx, *eA = nullptr, *eB = nullptr, *eY = nullptr, *eT = nullptr;
    int* d_redo = nullptr;   // general X: matrices whose FP32 block norms are recomputed in FP64
    __nv_bfloat16 *slA = nullptr, *slB = nullptr, *slY = nullptr, *slT = nullptr;
    char* split = nullptr;   // split-K scratch of the emulated products
    DevPlan* d_plan = nullptr;                      // device plan (dp)
    int *d_rfmt = nullptr, *d_rnu = nullptr, *d_sql = nullptr, *d_sqc = nullptr;
    double *d_ru = nullptr, *d_sc = nullptr;
    // Row / column maxima recorded by the emulated products' epilogues for the slicing of
    // the matrices they write (one buffer per matrix written, zeroed once): powers X_2..X_s
    // (rows), Y (columns), Horner iterates P_0..P_r (rows).  Not with variable s.
    const bool pre = K > 0 && !var_s;
    int* mxbuf = nullptr;
    // (mixed powers: also the columns of X^2..X^(s-h), the tree's B operands)
    const size_t mx_count = pre ? (size_t)(s + 1 + r + 1 + 1 + (mixp ? s + 1 : 0)) * batch * n : 0;
    auto layout1 = [&](Arena& a) {
        d_coef = a.take<double>(m + 1);
        pw = keep ? keep->pw : a.take<double>((size_t)batch * pw_bs);
        Pb0 = a.take<double>((size_t)batch * nn);
        Pb1 = a.take<double>((size_t)batch * nn);
        partial = a.take<double>(partial_elems);
        norms = a.take<double>((size_t)batch * q_alloc);
        d_anorm = a.take<double>(batch);
        d_sigma = a.take<int>(batch);
        d_bidx = a.take<int>((size_t)batch * 64);
        d_redo = expm ? nullptr : a.take<int>(batch);
        if (K > 0) {
            slA = a.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            slB = a.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            slY = a.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            eA = a.take<int>((size_t)batch * n);
            eB = a.take<int>((size_t)batch * n);
            eY = a.take<int>((size_t)batch * n);
            tmpT = a.take<double>((size_t)batch * nn);
            split = a.take<char>(f64e_split_bytes());
            if (pre) mxbuf = a.take<int>(mx_count);
            if (mixp) {
                slT = a.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
                eT = a.take<int>((size_t)batch * n);
                d_pnorm = a.take<double>((size_t)batch * s);
            }
        }
        if (dp) {
            d_plan = (DevPlan*)a.take<char>(sizeof(DevPlan));
            d_rfmt = a.take<int>((size_t)batch * (MPPS_MAX_R + 1));
            d_ru = a.take<double>((size_t)batch * (MPPS_MAX_R + 1));
            d_rnu = a.take<int>(batch);
            d_sc = a.take<double>((size_t)(MPPS_NUM_FORMATS + 2 * (r + 1)) * batch);
            if (sq_steps > 0) {
                d_sql = a.take<int>((size_t)sq_steps * batch);
                d_sqc = a.take<int>(sq_steps);
            }
        }
    };
    layout1(L);
    DevBuf ws1;
    mpps_status rc = ws1.alloc(L.off, st);
    if (rc) return rc;
    L.base = (char*)ws1.p;
    L.off = 0;
    layout1(L);
    if (split) MPPS_CUDA_TRY(cudaMemsetAsync(split, 0, f64e_split_flag_bytes(), st));
    if (mxbuf) MPPS_CUDA_TRY(cudaMemsetAsync(mxbuf, 0, sizeof(int) * mx_count, st));
    const size_t bn = (size_t)batch * n;
    auto mx_pow = [&](int j) { return mxbuf + (size_t)j * bn; };                // rows of X_j
    auto mx_iter = [&](int i) { return mxbuf + (size_t)(s + 1 + i) * bn; };     // rows of P_i
    int* mx_ycol = mxbuf ? mxbuf + (size_t)(s + 1 + r + 1) * bn : nullptr;
    auto mx_colpow = [&](int j) { return mxbuf + (size_t)(s + 1 + r + 2 + j) * bn; };   // cols of X_j
    if ((rc = launch_fill(d_coef, coeffs, m + 1, st))) return rc;
    DevErr* derr = nullptr;
    if ((rc = dev_err_get(&derr))) return rc;
    if ((rc = dev_err_check(derr, false))) return rc;
    d_err = derr->d;

    // emulated product helper: B^T rows (= columns of B) sliced straight from B
    auto slice_cols = [&](const double* Bm, long long bs, int k, __nv_bfloat16* planes,
                          int* ex) -> mpps_status {
        return launch_slice_cols(Bm, bs, n, batch, k, planes, ex, (unsigned long long*)tmpT, st);
    };

    // ---- a1: scaling (expm) or plain copy into X_1
    std::vector<int> sigma(batch, 0);
    SigmaStage* sgs = nullptr;
    if (expm && sig_dev) {   // sigma computed by the caller (device copy, and host copy)
        MPPS_CUDA_TRY(cudaMemcpyAsync(d_sigma, sig_dev, sizeof(int) * batch, cudaMemcpyDeviceToDevice, st));
        if (sig_host) sigma.assign(sig_host, sig_host + batch);
        rc = launch_scale_copy(dA, nn, pw, pw_bs, n, batch, d_sigma, st);
    } else if (expm) {
        // sigma = max(0, ceil(log2 ||A||_1)) on the device; read back with the block norms
        // (device plan: copied to page-locked memory now and waited for before the Horner
        // steps, by which time the GPU has long passed it; or not read at all)
        rc = launch_norm1(dA, nn, n, batch, partial, d_anorm, st);
        if (!rc) rc = launch_sigma(d_anorm, batch, d_sigma, st);
        if (!rc && dp && sq_steps == 0) {
            if (!(rc = sigma_stage(batch, &sgs)) && sgs) {
                MPPS_CUDA_TRY(cudaMemcpyAsync(sgs->h, d_sigma, sizeof(int) * batch,
                                              cudaMemcpyDeviceToHost, st));
                MPPS_CUDA_TRY(cudaEventRecord(sgs->ev, st));
            }
        }
        if (!rc) rc = launch_scale_copy(dA, nn, pw, pw_bs, n, batch, d_sigma, st);
    } else {
        rc = launch_scale_copy(dA, nn, pw, pw_bs, n, batch, nullptr, st);
    }
    if (rc) return rc;

    // ---- a2: powers X_j = X_{j-1} X_1 in the working precision (FP64 pipe or emulated)
    if (K > 0 && s >= 2) {
        rc = slice_cols(pw, pw_bs, K, slB, eB);
        if (rc) return rc;
    }
    auto power = [&](int j) -> mpps_status {   // X_j = X_{j-1} X_1
        Epilogue ep = epilogue_plain(pw + (long long)(j - 1) * nn, pw_bs);
        if (K > 0) {
            if (pre) {   // X_j's rows feed the next power, Y's columns the Horner steps
                if (j < s) ep.rmax = mx_pow(j);
                else ep.cmax = mx_ycol;
            }
            const double* Xa = pw + (long long)(j - 2) * nn;
            mpps_status r1 = (pre && j > 2)
                                 ? launch_slice_rows_pre(Xa, pw_bs, n, batch, K, slA, eA,
                                                         mx_pow(j - 1), nullptr, st)
                                 : launch_slice_rows(Xa, pw_bs, n, batch, K, slA, eA, st);
            if (!r1)
                r1 = launch_gemm_f64e(K, slA, K, eA, slB, K, eB, n, batch, batch, ep, d_err, st,
                                      nullptr, split);
            return r1;
        }
        return launch_gemm_f64(pw + (long long)(j - 2) * nn, pw_bs, pw, pw_bs, n, batch, ep, st);
    };
    if (!mixp) {
        for (int j = 2; j <= s; ++j)
            if ((rc = power(j))) return rc;
    } else {
        // the power tree: X^2..X^h by the chain (rows recorded for the next product, columns of
        // X^2..X^(s-h) for the tree's B operands), then Y = X^h X^(s-h); the leaf slots are
        // zeroed, so that the norms below are those of the blocks without their leaf terms
        for (int j = 2; j <= h; ++j) {
            Epilogue ep = epilogue_plain(pw + (long long)(j - 1) * nn, pw_bs);
            ep.rmax = mx_pow(j);
            if (j <= s - h) ep.cmax = mx_colpow(j);
            const double* Xa = pw + (long long)(j - 2) * nn;
            rc = j > 2 ? launch_slice_rows_pre(Xa, pw_bs, n, batch, K, slA, eA, mx_pow(j - 1),
                                               nullptr, st)
                       : launch_slice_rows(Xa, pw_bs, n, batch, K, slA, eA, st);
            if (!rc)
                rc = launch_gemm_f64e(K, slA, K, eA, slB, K, eB, n, batch, batch, ep, d_err, st,
                                      nullptr, split);
            if (rc) return rc;
        }
        rc = launch_slice_rows_pre(pw + (long long)(h - 1) * nn, pw_bs, n, batch, K, slA, eA,
                                   mx_pow(h), nullptr, st);
        if (!rc)
            rc = launch_slice_cols_pre(pw + (long long)(s - h - 1) * nn, pw_bs, n, batch, K, slT,
                                       eT, mx_colpow(s - h), st);
        if (!rc) {
            Epilogue ep = epilogue_plain(pw + (long long)(s - 1) * nn, pw_bs);
            ep.cmax = mx_ycol;
            rc = launch_gemm_f64e(K, slA, K, eA, slT, K, eT, n, batch, batch, ep, d_err, st,
                                  nullptr, split);
        }
        if (rc) return rc;
        MPPS_CUDA_TRY(cudaMemset2DAsync(pw + (long long)h * nn, (size_t)pw_bs * sizeof(double), 0,
                                        (size_t)(s - h - 1) * nn * sizeof(double), batch, st));
    }

    // ---- variable s (Algorithm 3.1): while a matrix's rule asks for it (mpps_choose_s on
    // ||X||, and ||B_0||, ||Y|| for each s so far), s grows by one and X_s = X_{s-1} X_1 is
    // formed; a batch takes the largest s any of its matrices asks for
    if (var_s) {
        std::vector<std::vector<double>> nb0(batch), ny(batch);
        std::vector<double> nx(batch, 0.0);
        for (;;) {
            q = block_norms_count(m, s);
            r = m / s;
            rc = launch_block_norms_f32(pw, pw_bs, n, batch, s, m, coeffs, partial, norms, st);
            if (!rc && !expm)
                rc = launch_block_norms_redo(pw, pw_bs, n, batch, s, m, d_coef, partial, norms,
                                             d_redo, st);
            if (rc) return rc;
            std::vector<double> h((size_t)batch * q);
            MPPS_CUDA_TRY(cudaMemcpyAsync(h.data(), norms, sizeof(double) * h.size(),
                                          cudaMemcpyDeviceToHost, st));
            MPPS_CUDA_TRY(cudaStreamSynchronize(st));
            bool grow = false;
            for (int b = 0; b < batch; ++b) {
                if (s == s0) nx[b] = h[(size_t)b * q + r + 2];
                nb0[b].push_back(h[(size_t)b * q]);
                ny[b].push_back(h[(size_t)b * q + r + 1]);
                if (mpps_choose_s(m, nx[b], nb0[b].data(), ny[b].data(), (int)nb0[b].size()) > s)
                    grow = true;
            }
            if (!grow || s >= s_cap) break;
            ++s;
            if ((rc = power(s))) return rc;
        }
        r = m / s;
        fold = (m % s) == 0;
        q = block_norms_count(m, s);
    }

    // ---- a3: ||B_i||_1, ||Y||_1, ||X||_1 in FP32: the rule needs them only to the right
    // order of magnitude (Section 3.3).  ||X||_1 <= 1 after the scaling of exp; for a general
    // X the matrices whose FP32 norms are not finite get FP64 ones
    rc = launch_block_norms_f32(pw, pw_bs, n, batch, s, m, coeffs, partial, norms, st, ex_pn > 0);
    if (!rc && !expm)
        rc = launch_block_norms_redo(pw, pw_bs, n, batch, s, m, d_coef, partial, norms, d_redo, st);
    if (rc) return rc;
    // mixed powers: ||X^j||_1 of the chain powers X^2..X^h ([j-1][batch]; ||X|| and ||Y||
    // come with the block norms), when the block-norm pass did not give them
    for (int j = 2; mixp && ex_pn == 0 && j <= h; ++j)
        if ((rc = launch_norm1(pw + (long long)(j - 1) * nn, pw_bs, n, batch, partial,
                               d_pnorm + (size_t)(j - 1) * batch, st)))
            return rc;
    int powfmt[MPPS_MAX_S + 1];
    for (int j = 0; j <= MPPS_MAX_S; ++j)
        powfmt[j] = (j < 2 || j > s) ? MPPS_FMT_NONE : (K > 0 ? MPPS_FMT_F64E(K) : MPPS_FMT_FP64);
    std::vector<double> hn;
    std::vector<mpps_report> rp(batch);
    Pol pol_s = pol;
    pol_s.s = s;
    int fmt[MPPS_MAX_R + 1];
    bool any_f64e = false;
    bool used[MPPS_NUM_FORMATS] = {false, false, false, false, false};
    // device plan: the formats each step may take (fmt[i] is MPPS_FMT_DEVICE unless one)
    std::vector<std::vector<int>> cand(r + 1);
    if (!dp) {
        hn.resize((size_t)batch * (q + ex_pn));
        MPPS_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * hn.size(),
                                      cudaMemcpyDeviceToHost, st));
        std::vector<double> hpn(mixp ? (size_t)batch * s : 0);
        if (mixp && ex_pn == 0)
            MPPS_CUDA_TRY(cudaMemcpyAsync(hpn.data(), d_pnorm, sizeof(double) * hpn.size(),
                                          cudaMemcpyDeviceToHost, st));
        if (expm)
            MPPS_CUDA_TRY(cudaMemcpyAsync(sigma.data(), d_sigma, sizeof(int) * batch,
                                          cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (ex_pn > 0) {   // the power norms follow each matrix's q block norms: move them out
            const size_t qx = (size_t)q + ex_pn;
            for (int b = 0; b < batch; ++b)
                for (int e = 0; e < ex_pn; ++e)
                    hpn[(size_t)(e + 1) * batch + b] = hn[(size_t)b * qx + q + e];
            for (int b = 0; b < batch; ++b)   // compact to stride q (destinations never pass sources)
                for (int i = 0; i < q; ++i) hn[(size_t)b * q + i] = hn[(size_t)b * qx + i];
            hn.resize((size_t)batch * q);
        }
        // mixed powers: each leaf in the most precise format any matrix asks for; the block
        // norms become the bounds the leaf rule derives (lower for B_0, upper for the rest)
        if (mixp) {
            for (int j = h + 1; j < s; ++j) powfmt[j] = MPPS_FMT_NONE;
            for (int b = 0; b < batch; ++b) {
                int pf[MPPS_MAX_S + 1];
                double nbo[MPPS_MAX_R + 1], xp[MPPS_MAX_S];
                for (int j = 1; j <= s; ++j)
                    xp[j - 1] = j == 1 ? hn[(size_t)b * q + r + 2]
                                       : j == s ? hn[(size_t)b * q + r + 1]
                                                : j <= h ? hpn[(size_t)(j - 1) * batch + b] : 0.0;
                plan_powers_core(m, s, coeffs, xp, &hn[(size_t)b * q], pol_s, pf, nbo);
                for (int i = 0; i <= r; ++i) hn[(size_t)b * q + i] = nbo[i];
                for (int j = h + 1; j < s; ++j)
                    if (powfmt[j] == MPPS_FMT_NONE || prec_rank(pf[j]) > prec_rank(powfmt[j]))
                        powfmt[j] = pf[j];
            }
        }

        // ---- a4: plan per matrix; a batch runs each step in the most precise format any
        // of its matrices asks for
        for (int b = 0; b < batch; ++b) {
            rc = plan_one(m, n, &hn[(size_t)b * q], hn[(size_t)b * q + r + 1], pol_s, &rp[b]);
            if (rc) return rc;
            rp[b].normX = hn[(size_t)b * q + r + 2];
            rp[b].sigma = sigma[b];
        }
        for (int i = 1; i <= r; ++i) {
            int f = rp[0].fmt[i];
            for (int b = 1; b < batch; ++b)
                if (prec_rank(rp[b].fmt[i]) > prec_rank(f)) f = rp[b].fmt[i];
            fmt[i] = (fold && i == r) ? MPPS_FMT_NONE : f;
            if (MPPS_FMT_IS_F64E(fmt[i])) any_f64e = true;
            if (fmt[i] != MPPS_FMT_NONE) cand[i].assign(1, fmt[i]);
        }
        // mixed powers: the leaves X^(h+t) = X^h X^t, rows of X^h still in the A slices,
        // columns of X (t = 1) in the B slices, of X^t (t >= 2) sliced from its recorded codes
        for (int j = h + 1; mixp && j < s; ++j) {
            const int t = j - h;
            if (t >= 2 && (rc = launch_slice_cols_pre(pw + (long long)(t - 1) * nn, pw_bs, n, batch,
                                                      K, slT, eT, mx_colpow(t), st)))
                return rc;
            Epilogue ep = epilogue_plain(pw + (long long)(j - 1) * nn, pw_bs);
            if ((rc = launch_gemm_f64e(MPPS_F64E_SLICES(powfmt[j]), slA, K, eA, t >= 2 ? slT : slB,
                                       K, t >= 2 ? eT : eB, n, batch, batch, ep, d_err, st,
                                       nullptr, split)))
                return rc;
        }
    } else {
        // ---- a4 on the device: the same rule (plan_core) per matrix, the batch's formats,
        // the gate counts and the operand scales; nothing is read back
        {
            mpps_report probe;   // validates s, r and f64_slices as the host planner does
            std::vector<double> ones(r + 1, 1.0);
            if ((rc = plan_one(m, n, ones.data(), 1.0, pol_s, &probe))) return rc;
        }
        ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
        MPPS_CUDA_TRY(launch_pdl(k_plan, dim3(1), dim3(256), 0, st, (const double*)norms, q, batch, n,
                                 r, (int)fold, pol_s, d_plan, d_rfmt, d_ru, d_rnu, d_sc,
                                 d_sc + (size_t)MPPS_NUM_FORMATS * batch,
                                 d_sc + (size_t)(MPPS_NUM_FORMATS + r + 1) * batch));
        MPPS_LAUNCH_CHECK();
        for (int i = 1; i <= r; ++i) {
            cand[i] = step_candidates(pol_s, r, fold, i);
            fmt[i] = cand[i].empty() ? MPPS_FMT_NONE
                                     : (cand[i].size() == 1 ? cand[i][0] : MPPS_FMT_DEVICE);
            for (int f : cand[i]) if (MPPS_FMT_IS_F64E(f)) any_f64e = true;
        }
    }
    for (int i = 1; i <= r; ++i)
        for (int f : cand[i]) if (is_low(f)) used[f] = true;
    int max_es = 1;
    for (int f = 1; f < MPPS_NUM_FORMATS; ++f)
        if (used[f]) max_es = std::max(max_es, low_elem_bytes(f));
    const bool any_low = used[1] || used[2] || used[3] || used[4];
    // gate of candidate f of step i (null when the step has a single format)
    auto gate = [&](int i, int f) -> const int* {
        if (!dp || cand[i].size() <= 1) return nullptr;
        return &d_plan->cnt[i][fmt_slot(f)];
    };
    auto has_low_copy = [&](int i) {   // P_i may need a rounded copy from its producer
        for (int f : cand[i]) if (is_low(f) && f != MPPS_FMT_FP8) return true;
        return false;
    };

    // ---- phase-2 workspace: rounded copies and their power-of-two scales
    const int lld = low_ld(n);
    const long long low_bs = (long long)n * lld;
    Arena L2;
    void *Ylo_hi[MPPS_NUM_FORMATS] = {}, *Ylo_lo[MPPS_NUM_FORMATS] = {};
    void *Pl_hi[2] = {}, *Pl_lo[2] = {};
    double *d_sY, *d_sP, *d_alpha;
    // FP8 operands: one power of two per row of P_i and per column of Y (the exponents that
    // undo them, and column-maximum scratch), then one per 32 entries along K (block scale
    // codes of P_i and of Y)
    int *xrowP = nullptr, *xcolY = nullptr;
    unsigned long long* cmax8 = nullptr;
    uint8_t *sfP = nullptr, *sfY = nullptr;
    auto layout2 = [&](Arena& a) {
        for (int f = 1; f < MPPS_NUM_FORMATS; ++f)
            if (used[f]) {
                Ylo_hi[f] = a.take<char>((size_t)batch * low_bs * low_elem_bytes(f));
                if (f == MPPS_FMT_BF16X3) Ylo_lo[f] = a.take<char>((size_t)batch * low_bs * 2);
            }
        for (int k = 0; k < 2; ++k) {
            Pl_hi[k] = a.take<char>(any_low ? (size_t)batch * low_bs * max_es : 0);
            Pl_lo[k] = a.take<char>(used[MPPS_FMT_BF16X3] ? (size_t)batch * low_bs * 2 : 0);
        }
        if (used[MPPS_FMT_FP8]) {
            xrowP = a.take<int>((size_t)batch * n);
            xcolY = a.take<int>((size_t)batch * n);
            cmax8 = a.take<unsigned long long>((size_t)batch * n);
            sfP = a.take<uint8_t>((size_t)batch * mx_scale_bytes_a(n));
            sfY = a.take<uint8_t>((size_t)batch * mx_scale_bytes_b(n));
        }
        // one contiguous block (filled by a single copy, or by the device plan): sY | sP |
        // alpha
        d_sY = dp ? d_sc : a.take<double>((size_t)(MPPS_NUM_FORMATS + 2 * (r + 1)) * batch);
        d_sP = d_sY ? d_sY + (size_t)MPPS_NUM_FORMATS * batch : nullptr;
        d_alpha = d_sP ? d_sP + (size_t)(r + 1) * batch : nullptr;
    };
    DevBuf ws2;
    if (any_low) {
        layout2(L2);
        rc = ws2.alloc(L2.off, st);
        if (rc) return rc;
        L2.base = (char*)ws2.p;
        L2.off = 0;
        layout2(L2);
    }
    if (any_low && !dp) {
        std::vector<double> hs((size_t)(MPPS_NUM_FORMATS + 2 * (r + 1)) * batch, 1.0);
        double* h_sY = hs.data();
        double* h_sP = h_sY + (size_t)MPPS_NUM_FORMATS * batch;
        double* h_al = h_sP + (size_t)(r + 1) * batch;
        for (int b = 0; b < batch; ++b) {
            const double* eta = &hn[(size_t)b * q];
            const double y = hn[(size_t)b * q + r + 1];
            const int eY = exp_above(y);
            for (int f = 1; f < MPPS_NUM_FORMATS; ++f)
                h_sY[(size_t)f * batch + b] = ldexp(1.0, low_target_exp(f) - eY);
            // beta_i = sum_{k>=i} ||B_k|| ||Y||^{k-i} >= ||P_i||_1 >= max |P_i|
            double beta = 0.0;
            for (int i = r; i >= 1; --i) {
                beta = eta[i] + y * beta;
                if (is_low(fmt[i])) {
                    const int T = low_target_exp(fmt[i]);
                    const int eP = exp_above(beta);
                    h_sP[(size_t)i * batch + b] = ldexp(1.0, T - eP);
                    h_al[(size_t)i * batch + b] = ldexp(1.0, eP + eY - 2 * T);
                }
            }
        }
        MPPS_CUDA_TRY(cudaMemcpyAsync(d_sY, hs.data(), sizeof(double) * hs.size(),
                                      cudaMemcpyHostToDevice, st));
    }
    if (any_low) {   // Y's rounded copies (device plan: each only if a step uses its format)
        const int* yg[MPPS_NUM_FORMATS] = {};
        if (dp)
            for (int f = 1; f < MPPS_NUM_FORMATS; ++f) yg[f] = &d_plan->ycnt[f];
        for (int f = 1; f < MPPS_NUM_FORMATS; ++f)
            if (used[f]) {
                rc = f == MPPS_FMT_FP8
                         ? launch_convert_mx(pw + (long long)(s - 1) * nn, pw_bs, n, batch,
                                             (uint8_t*)Ylo_hi[f], low_bs, lld, sfY,
                                             mx_scale_bytes_b(n), true, xcolY, cmax8, st, yg[f])
                         : launch_convert(f, pw + (long long)(s - 1) * nn, pw_bs, n, batch, Ylo_hi[f],
                                          Ylo_lo[f], low_bs, lld, d_sY + (size_t)f * batch, true, st,
                                          yg[f]);
                if (rc) return rc;
            }
    }

    if (any_f64e) {   // Y^T slices for every emulated Horner step (first k planes used)
        // (device plan: gated unless some step runs an emulated product whatever the norms)
        bool fixed_f64e = !dp;
        for (int i = 1; i <= r && !fixed_f64e; ++i)
            fixed_f64e = cand[i].size() == 1 && MPPS_FMT_IS_F64E(cand[i][0]);
        const int* yg = fixed_f64e ? nullptr : &d_plan->ycnt[kYAnyF64e];
        rc = (pre && s >= 2) ? launch_slice_cols_pre(pw + (long long)(s - 1) * nn, pw_bs, n, batch, K,
                                                     slY, eY, mx_ycol, st, yg)
                             : launch_slice_cols(pw + (long long)(s - 1) * nn, pw_bs, n, batch, K, slY, eY,
                                                 (unsigned long long*)tmpT, st, yg);
        if (rc) return rc;
    }

    // ---- a5/a6: Horner in Y with the block sums fused into the product epilogues
    int sig_max = 0;
    if (sgs) {   // device plan: the early copy of sigma (the GPU is well past it by now)
        MPPS_CUDA_TRY(cudaEventSynchronize(sgs->ev));
        for (int b = 0; b < batch; ++b) sigma[b] = sgs->h[b];
    }
    const bool blind = sq_steps > 0 && !(sig_dev && sig_host);
    if (blind) sig_max = sq_steps;   // squarings launched blind, per-matrix on the GPU
    else
        for (int b = 0; b < batch; ++b) sig_max = std::max(sig_max, sigma[b]);
    // row and column maxima of Q_0 .. Q_{sigma-1}, recorded for the squarings' slicing
    DevBuf wsq;
    int* sqmx = nullptr;
    if (pre && expm && sig_max > 0) {
        const size_t cnt = (size_t)2 * sig_max * bn;
        if ((rc = wsq.alloc(sizeof(int) * cnt, st))) return rc;
        sqmx = (int*)wsq.p;
        MPPS_CUDA_TRY(cudaMemsetAsync(sqmx, 0, sizeof(int) * cnt, st));
    }
    auto mx_sq_row = [&](int k) { return sqmx + (size_t)(2 * k) * bn; };
    auto mx_sq_col = [&](int k) { return sqmx + (size_t)(2 * k + 1) * bn; };
    double* Pbuf[2] = {Pb0, Pb1};
    double* dst0 = (expm && sig_max > 0) ? Pb0 : dOut;
    // where each Horner iterate P_j is written (and read by step j): ping-pong buffers, or the
    // tape's slots
    double* Pdst[MPPS_MAX_R + 1];
    Pdst[0] = dst0;
    for (int j = 1; j <= r; ++j)
        Pdst[j] = keep ? keep->slots + (size_t)keep->L->fwd_slot(j) * batch * nn : Pbuf[j & 1];
    const double* Y = pw + (long long)(s - 1) * nn;
    // Emulated squarings work on Q = P - I (Q <- Q Q + 2 Q, exact algebra): the slices of a
    // matrix close to I would be aligned to its unit diagonal and lose the small entries'
    // low bits; Q has no dominant identity part.  The last Horner step writes Q_0 directly.
    const bool qform = expm && sig_max > 0 && K > 0;

    auto make_ep = [&](int i) {   // epilogue producing P_{i-1} = B_{i-1} + (...)
        Epilogue ep = epilogue_plain(Pdst[i - 1], nn);
        ep.nt = s - 1;
        for (int j = 0; j < s; ++j) ep.coef[j] = coeffs[(i - 1) * s + j];
        if (i - 1 == 0 && qform) ep.coef[0] -= 1.0;
        ep.pw = pw;
        ep.pw_bstride = pw_bs;
        const bool dev_copy = i - 1 >= 1 && fmt[i - 1] == MPPS_FMT_DEVICE && has_low_copy(i - 1);
        if (dev_copy || (i - 1 >= 1 && is_low(fmt[i - 1]) && fmt[i - 1] != MPPS_FMT_FP8)) {
            ep.low_fmt = fmt[i - 1];
            if (dev_copy) ep.low_fmt_dev = &d_plan->fmt[i - 1];
            ep.low_hi = Pl_hi[(i - 1) & 1];
            ep.low_lo = Pl_lo[(i - 1) & 1];
            ep.low_bstride = low_bs;
            ep.lld = lld;
            ep.low_scale_b = d_sP + (size_t)(i - 1) * batch;
        }
        return ep;
    };

    // which Horner iterates had their row maxima recorded by the product that wrote them
    bool iter_mx[MPPS_MAX_R + 2] = {false};
    int i_start;
    if (fold) {
        // B_r = b_m I: P_{r-1} = B_{r-1} + b_m Y, no product
        Epilogue ep = make_ep(r);
        ep.alpha = coeffs[m];
        rc = launch_combine(n, batch, Y, pw_bs, ep, st);
        i_start = r - 1;
    } else {
        // P_r = B_r = sum_{j<=m-sr} b_{sr+j} X_j
        Epilogue ep = epilogue_plain(Pdst[r], nn);
        ep.nt = m - s * r;
        for (int j = 0; j <= ep.nt; ++j) ep.coef[j] = coeffs[s * r + j];
        ep.pw = pw;
        ep.pw_bstride = pw_bs;
        ep.alpha = 0.0;
        const bool dev_copy = fmt[r] == MPPS_FMT_DEVICE && has_low_copy(r);
        if (dev_copy || (is_low(fmt[r]) && fmt[r] != MPPS_FMT_FP8)) {
            ep.low_fmt = fmt[r];
            if (dev_copy) ep.low_fmt_dev = &d_plan->fmt[r];
            ep.low_hi = Pl_hi[r & 1];
            ep.low_lo = Pl_lo[r & 1];
            ep.low_bstride = low_bs;
            ep.lld = lld;
            ep.low_scale_b = d_sP + (size_t)r * batch;
        }
        rc = launch_combine(n, batch, nullptr, 0, ep, st);
        i_start = r;
    }
    if (rc) return rc;
    for (int i = i_start; i >= 1; --i) {
        // one launch per format the step may take; with the device plan all but the chosen
        // one find a zero count and return at once
        for (int f : cand[i]) {
            Epilogue ep = make_ep(i);
            const int* g = gate(i, f);
            ep.dcount = g;
            if (f == MPPS_FMT_FP64) {
                rc = launch_gemm_f64(Pdst[i], nn, Y, pw_bs, n, batch, ep, st);
            } else if (MPPS_FMT_IS_F64E(f)) {
                const int k = MPPS_F64E_SLICES(f);
                // P_{i-1} feeds an emulated step (or, as Q_0, the squarings): record its maxima
                // (only when this step's format is certain, so that they are always written)
                const bool certain = cand[i].size() == 1;
                if (pre && certain &&
                    ((i - 1 >= 1 && MPPS_FMT_IS_F64E(fmt[i - 1])) || (i == 1 && qform))) {
                    if (i == 1) {        // Q_0 of the squarings: rows and columns
                        ep.rmax = mx_sq_row(0);
                        ep.cmax = mx_sq_col(0);
                    } else {
                        ep.rmax = mx_iter(i - 1);
                    }
                    iter_mx[i - 1] = true;
                }
                rc = iter_mx[i] ? launch_slice_rows_pre(Pdst[i], nn, n, batch, k, slA, eA, mx_iter(i),
                                                        nullptr, st, g)
                                : launch_slice_rows(Pdst[i], nn, n, batch, k, slA, eA, st, g);
                if (!rc)
                    rc = launch_gemm_f64e(k, slA, k, eA, slY, K, eY, n, batch, batch, ep, d_err, st,
                                          nullptr, split);
            } else if (f == MPPS_FMT_FP8) {
                // the paper's scaled low-precision product with the scales as fine as E4M3
                // needs: a power of two per row of P_i and per column of Y (undone in the
                // epilogue), and one per 32 entries along K applied by the tensor core
                rc = launch_convert_mx(Pdst[i], nn, n, batch, (uint8_t*)Pl_hi[i & 1], low_bs, lld,
                                       sfP, mx_scale_bytes_a(n), false, xrowP, nullptr, st, g);
                ep.row_exp = xrowP;
                ep.col_exp = xcolY;
                const MxScales mx{sfP, sfY, mx_scale_bytes_a(n), mx_scale_bytes_b(n), (n + 127) / 128};
                if (!rc)
                    rc = launch_gemm_tc(f, Pl_hi[i & 1], nullptr, Ylo_hi[f], nullptr, low_bs, low_bs,
                                        lld, n, batch, ep, d_err, st, &mx);
            } else {
                ep.alpha_b = d_alpha + (size_t)i * batch;
                rc = launch_gemm_tc(f, Pl_hi[i & 1], Pl_lo[i & 1], Ylo_hi[f], Ylo_lo[f], low_bs,
                                    low_bs, lld, n, batch, ep, d_err, st);
            }
            if (rc) return rc;
        }
    }

    // ---- a7: squarings (eq. (3.6)), FP64, per-matrix counts
    if (expm && sig_max > 0) {
        std::vector<int> counts(sig_max, 0);
        int* d_lists = d_bidx;
        const int* d_counts = nullptr;   // device plan with blind squarings: counts on the GPU
        DevBuf extra;
        if (blind) {
            ProfScope prof(MPPS_PROF_ELEMENTWISE, st);
            MPPS_CUDA_TRY(launch_pdl(k_sq_lists, dim3(1), dim3(1024), 0, st, (const int*)d_sigma, batch,
                                     sq_steps, d_sql, d_sqc, d_err));
            MPPS_LAUNCH_CHECK();
            d_lists = d_sql;
            d_counts = d_sqc;
            for (int k = 0; k < sig_max; ++k) counts[k] = batch;
        } else {
            std::vector<int> lists((size_t)sig_max * batch);
            for (int k = 0; k < sig_max; ++k)
                for (int b = 0; b < batch; ++b)
                    if (sigma[b] > k) lists[(size_t)k * batch + counts[k]++] = b;
            if ((size_t)sig_max * batch > (size_t)batch * 64) {
                rc = extra.alloc(sizeof(int) * lists.size(), st);
                if (rc) return rc;
                d_lists = (int*)extra.p;
            }
            if ((rc = launch_fill_bytes(d_lists, lists.data(), sizeof(int) * lists.size(), st)))
                return rc;
        }
        for (int k = 0; k < sig_max; ++k) {
            Epilogue ep = epilogue_plain(Pbuf[(k + 1) & 1], nn);
            ep.dcount = d_counts ? d_counts + k : nullptr;
            if (qform) {   // Q_{k+1} = Q_k Q_k + 2 Q_k
                ep.add = Pbuf[k & 1];
                ep.add_bstride = nn;
                ep.add_coef = 2.0;
            }
            if (K > 0) {
                const bool have = pre && (k == 0 ? iter_mx[0] : true);
                if (pre && k + 1 < sig_max) {   // Q_{k+1} is sliced for the next squaring
                    ep.rmax = mx_sq_row(k + 1);
                    ep.cmax = mx_sq_col(k + 1);
                }
                // with the recorded maxima only the matrices of this step's list are sliced
                const int* lk = d_lists + (size_t)k * batch;
                const int* gk = d_counts ? d_counts + k : nullptr;
                if (have)   // rows and columns of Q_k from one read
                    rc = launch_slice_both_pre(Pbuf[k & 1], nn, n, counts[k], K, slA, eA,
                                               mx_sq_row(k), slB, eB, mx_sq_col(k), st, gk, lk);
                else {
                    rc = launch_slice_rows(Pbuf[k & 1], nn, n, batch, K, slA, eA, st);
                    if (!rc) rc = slice_cols(Pbuf[k & 1], nn, K, slB, eB);
                }
                if (!rc)
                    rc = launch_gemm_f64e(K, slA, K, eA, slB, K, eB, n, counts[k], batch, ep, d_err,
                                          st, d_lists + (size_t)k * batch, split);
            } else {
                rc = launch_gemm_f64(Pbuf[k & 1], nn, Pbuf[k & 1], nn, n, counts[k], ep, st,
                                     d_lists + (size_t)k * batch);
            }
            if (rc) return rc;
        }
        rc = launch_select_copy(Pb0, Pb1, d_sigma, dOut, n, batch, qform ? 1.0 : 0.0, st,
                                blind ? sq_steps : -1);
        if (rc) return rc;
    }

    // device plan: what the GPU planned, read back only when a report is asked for
    std::vector<int> dfmt;
    if (dp && rep) {
        std::vector<int> rf((size_t)batch * (MPPS_MAX_R + 1)), rnu(batch);
        std::vector<double> ru((size_t)batch * (MPPS_MAX_R + 1));
        hn.resize((size_t)batch * q);
        dfmt.resize(MPPS_MAX_R + 1);
        MPPS_CUDA_TRY(cudaMemcpyAsync(dfmt.data(), d_plan->fmt, sizeof(int) * dfmt.size(),
                                      cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaMemcpyAsync(rf.data(), d_rfmt, sizeof(int) * rf.size(), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaMemcpyAsync(ru.data(), d_ru, sizeof(double) * ru.size(), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaMemcpyAsync(rnu.data(), d_rnu, sizeof(int) * batch, cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * hn.size(),
                                      cudaMemcpyDeviceToHost, st));
        if (expm)
            MPPS_CUDA_TRY(cudaMemcpyAsync(sigma.data(), d_sigma, sizeof(int) * batch,
                                          cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int b = 0; b < batch; ++b) {
            mpps_report& R = rp[b];
            memset(&R, 0, sizeof(R));
            R.s = s; R.r = r; R.fold = fold ? 1 : 0; R.nu = rnu[b];
            for (int i = 0; i <= MPPS_MAX_R; ++i) R.fmt[i] = MPPS_FMT_NONE;
            for (int i = 0; i <= r; ++i) {
                R.normB[i] = hn[(size_t)b * q + i];
                R.u[i] = i >= 1 ? ru[(size_t)b * (MPPS_MAX_R + 1) + i] : 0.0;
            }
            R.normY = hn[(size_t)b * q + r + 1];
            R.normX = hn[(size_t)b * q + r + 2];
            R.sigma = sigma[b];
        }
        for (int i = 1; i <= r; ++i) fmt[i] = dfmt[i];
    }

    if (any_low || K > 0 || sq_steps > 0) {
        if ((rc = dev_err_enqueue(derr, st))) return rc;
        if ((sync_at_end || (dp && rep)) && (rc = dev_err_check(derr, true))) return rc;
    }

    if (keep) {
        for (int i = 0; i <= MPPS_MAX_R; ++i) keep->fmt[i] = (i >= 1 && i <= r) ? fmt[i] : MPPS_FMT_NONE;
        keep->plans = rp;
    }
    if (rep) {
        for (int b = 0; b < batch; ++b) {
            mpps_report& R = rp[b];
            for (int i = 1; i <= r; ++i) R.fmt[i] = fmt[i];
            for (int j = 0; j <= MPPS_MAX_S; ++j) R.pow_fmt[j] = powfmt[j];
            for (int f = 0; f <= MPPS_NUM_FORMATS; ++f) R.gemms[f] = 0;
            R.gemms[MPPS_FMT_FP64] += s - 1;   // emulated working-precision products count as FP64
            for (int i = 1; i <= r; ++i) {
                if (fmt[i] == MPPS_FMT_NONE) continue;
                const int slot = MPPS_FMT_IS_F64E(fmt[i]) ? MPPS_FMT_FP64 : fmt[i];
                R.gemms[slot] += 1;
            }
            R.gemms[MPPS_NUM_FORMATS] = sigma[b];
            R.cost_ratio = cost_ratio(R, pol.tol);
            rep[b] = R;
        }
    }
    return MPPS_OK;
}

// Host/device marshalling around a device implementation.
struct Staged {
    const double* dev = nullptr;
    DevBuf buf;
};

static mpps_status stage_in(const double* p, size_t elems, cudaStream_t st, Staged& out) {
    if (is_device_ptr(p)) {
        out.dev = p;
        return MPPS_OK;
    }
    mpps_status rc = out.buf.alloc(elems * sizeof(double), st);
    if (rc) return rc;
    MPPS_CUDA_TRY(cudaMemcpyAsync(out.buf.p, p, elems * sizeof(double), cudaMemcpyHostToDevice, st));
    out.dev = (const double*)out.buf.p;
    return MPPS_OK;
}

}  // namespace mpps

using namespace mpps;

namespace mpps {
// One member of an uneven batch, for the grouped evaluations.
struct GItem {
    const double* A;
    double* out;
    int n, m;
    const double* c;   // m + 1 coefficients (host)
};

// Grouped evaluation (expm: Taylor exp with scaling and squaring, else p(A)); items checked.
static mpps_status grouped_eval(const GItem* items, int count, const mpps_policy* policy,
                                mpps_report* rep, cudaStream_t stream, bool expm) {
    cudaStream_t st = stream;
    Pol P = resolve(policy);
    P.dplan = 1;   // every bucket planned on the device: no read-back between buckets
    P.var_s = 0;
    // buckets keyed by (padded order, degree, coefficients), in first-appearance order
    struct Bucket { int n_pad, m; const double* c; std::vector<int> idx; };
    std::vector<Bucket> buckets;
    for (int i = 0; i < count; ++i) {
        const int m = items[i].m;
        const int np = (items[i].n + 31) / 32 * 32;
        size_t k = 0;
        while (k < buckets.size() &&
               !(buckets[k].n_pad == np && buckets[k].m == m &&
                 (buckets[k].c == items[i].c ||
                  std::equal(items[i].c, items[i].c + m + 1, buckets[k].c))))
            ++k;
        if (k == buckets.size()) buckets.push_back({np, m, items[i].c, {}});
        buckets[k].idx.push_back(i);
    }
    const int nb = (int)buckets.size();
    struct Work {
        DevBuf buf;
        PadItem* d_list = nullptr;
        double *dA = nullptr, *dO = nullptr, *partial = nullptr, *anorm = nullptr;
        int* d_sig = nullptr;
        std::vector<double> c;
    };
    std::vector<Work> wk(nb);
    mpps_status rc = MPPS_OK;
    // ---- phase A, on the caller's stream: every bucket gathered into its zero-padded batch,
    // ||A||_1 and sigma per matrix (eq. (3.6))
    for (int k = 0; k < nb; ++k) {
        const Bucket& bk = buckets[k];
        Work& w = wk[k];
        const int cnt = (int)bk.idx.size();
        if (cnt > 65535) {
            set_error("expm_taylor_ss_grouped: more than 65535 items of one size and degree");
            return MPPS_EINVAL;
        }
        const long long nn = (long long)bk.n_pad * bk.n_pad;
        w.c.assign(bk.c, bk.c + bk.m + 1);
        std::vector<PadItem> list(cnt);
        for (int j = 0; j < cnt; ++j) {
            const GItem& it = items[bk.idx[j]];
            list[j] = PadItem{it.A, it.out, it.n, 0};
        }
        Arena a;
        auto lay = [&](Arena& z) {
            w.d_list = (PadItem*)z.take<char>(sizeof(PadItem) * cnt);
            w.dA = z.take<double>((size_t)nn * cnt);
            w.dO = z.take<double>((size_t)nn * cnt);
            w.partial = z.take<double>(norm1_partial_elems(bk.n_pad, cnt));
            w.anorm = z.take<double>(cnt);
            w.d_sig = z.take<int>(cnt);
        };
        lay(a);
        if ((rc = w.buf.alloc(a.off, st))) return rc;
        a.base = (char*)w.buf.p;
        a.off = 0;
        lay(a);
        if ((rc = launch_fill_bytes(w.d_list, list.data(), sizeof(PadItem) * cnt, st))) return rc;
        if ((rc = launch_gather_pad(w.d_list, cnt, bk.n_pad, w.dA, st))) return rc;
        if (!expm) continue;
        if ((rc = launch_norm1(w.dA, nn, bk.n_pad, cnt, w.partial, w.anorm, st))) return rc;
        if ((rc = launch_sigma(w.anorm, cnt, w.d_sig, st))) return rc;
    }
    // one read of every sigma (skipped with blind squarings: then nothing is read back)
    std::vector<int> hsig;
    if (expm && P.max_sq == 0) {
        hsig.resize(count);
        SigmaStage* sgs = nullptr;
        if ((rc = sigma_stage(count, &sgs))) return rc;
        size_t off = 0;
        for (int k = 0; k < nb; ++k) {
            const size_t cnt = buckets[k].idx.size();
            MPPS_CUDA_TRY(cudaMemcpyAsync(sgs->h + off, wk[k].d_sig, sizeof(int) * cnt,
                                          cudaMemcpyDeviceToHost, st));
            off += cnt;
        }
        MPPS_CUDA_TRY(cudaEventRecord(sgs->ev, st));
        MPPS_CUDA_TRY(cudaEventSynchronize(sgs->ev));
        std::copy(sgs->h, sgs->h + count, hsig.begin());
    }
    // ---- phase B: the buckets on up to kAuxStreams streams that fork from the caller's
    // stream and join it again, so that small buckets run side by side
    std::vector<cudaStream_t> aux;
    if ((rc = aux_streams(std::min(nb, kAuxStreams), &aux))) return rc;
    cudaEvent_t fork_ev;
    MPPS_CUDA_TRY(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    MPPS_CUDA_TRY(cudaEventRecord(fork_ev, st));
    for (cudaStream_t sx : aux) MPPS_CUDA_TRY(cudaStreamWaitEvent(sx, fork_ev, 0));
    MPPS_CUDA_TRY(cudaEventDestroy(fork_ev));
    size_t off = 0;
    for (int k = 0; k < nb && !rc; ++k) {
        const Bucket& bk = buckets[k];
        Work& w = wk[k];
        const int cnt = (int)bk.idx.size();
        cudaStream_t sb = aux[k % aux.size()];
        std::vector<mpps_report> brep(rep ? cnt : 0);
        rc = eval_device(w.c.data(), bk.m, w.dA, bk.n_pad, cnt, P, w.dO, rep ? brep.data() : nullptr,
                         sb, expm, false, nullptr, expm ? w.d_sig : nullptr,
                         hsig.empty() ? nullptr : hsig.data() + off);
        if (!rc) rc = launch_scatter_unpad(w.d_list, cnt, bk.n_pad, w.dO, sb);
        if (!rc && rep)
            for (int j = 0; j < cnt; ++j) rep[bk.idx[j]] = brep[j];
        off += cnt;
    }
    // join (also after a failure, so that the workspaces are released in stream order)
    for (cudaStream_t sx : aux) {
        cudaEvent_t jev;
        MPPS_CUDA_TRY(cudaEventCreateWithFlags(&jev, cudaEventDisableTiming));
        MPPS_CUDA_TRY(cudaEventRecord(jev, sx));
        MPPS_CUDA_TRY(cudaStreamWaitEvent(st, jev, 0));
        MPPS_CUDA_TRY(cudaEventDestroy(jev));
    }
    return rc;
}


}  // namespace mpps

extern "C" {

void mpps_policy_default(mpps_policy* p) {
    if (!p) return;
    p->mode = MPPS_MIXED_NS;
    p->tol = 0x1p-53;
    p->delta = 10.0;
    p->s = 0;
    p->formats = 0x1Fu;
    p->fp64_floor_steps = 2;
    p->f64_slices = 0;
    p->variable_s = 0;
    p->adjoint_recompute = 0;
    p->device_plan = 0;
    p->max_squarings = 0;
    p->mixed_powers = 0;
}

mpps_status mpps_plan_powers(int m, int s, const double* coeffs, const double* normXpow,
                             const double* normBpart, const mpps_policy* policy, int* fmt_out,
                             double* normB_out) {
    clear_error();
    if (!coeffs || !normXpow || !normBpart || !fmt_out || !normB_out || m < 1 || s < 1 ||
        s > m || s > MPPS_MAX_S || m / s > MPPS_MAX_R) {
        set_error("mpps_plan_powers: invalid argument (m=%d, s=%d)", m, s);
        return MPPS_EINVAL;
    }
    const Pol P = resolve(policy);
    if (P.f64k < 0 || P.f64k > MPPS_F64E_MAX_SLICES) {
        set_error("f64_slices=%d outside 0..%d", P.f64k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    if (!forms_power_tree(P, s)) {
        set_error("mpps_plan_powers: the policy forms no power tree (mixed_powers %d, mode %d, "
                  "f64_slices %d, s %d)", P.mixp, P.mode, P.f64k, s);
        return MPPS_ENOTSUP;
    }
    plan_powers_core(m, s, coeffs, normXpow, normBpart, P, fmt_out, normB_out);
    return MPPS_OK;
}

mpps_status mpps_release_workspace(void) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_poolmu);
    for (int d = 0; d < 64; ++d)
        if (g_pool[d]) {
            int cur = 0;
            MPPS_CUDA_TRY(cudaGetDevice(&cur));
            MPPS_CUDA_TRY(cudaSetDevice(d));
            cudaError_t e = cudaDeviceSynchronize();
            if (e == cudaSuccess) e = cudaMemPoolTrimTo(g_pool[d], 0);
            cudaSetDevice(cur);
            if (e != cudaSuccess) {
                set_error("mpps_release_workspace: %s", cudaGetErrorString(e));
                return MPPS_ECUDA;
            }
        }
    return MPPS_OK;
}

const char* mpps_last_error(void) { return g_err; }

const char* mpps_version(void) { return "mpps 0.1 (sm_103a)"; }

mpps_status mpps_plan(int m, int n, const double* normB, double normY, const mpps_policy* policy,
                      mpps_report* out) {
    clear_error();
    if (m < 0 || n <= 0 || !normB || !out) {
        set_error("mpps_plan: invalid argument");
        return MPPS_EINVAL;
    }
    Pol P = resolve(policy);
    mpps_status rc = plan_one(m, n, normB, normY, P, out);
    if (rc == MPPS_OK) out->cost_ratio = cost_ratio(*out, P.tol);
    return rc;
}

mpps_status mpps_plan_adjoint(int m, int n, const double* normB, double normY, double normX,
                              const mpps_policy* policy, mpps_report* out) {
    clear_error();
    if (m < 0 || n <= 0 || !normB || !out) {
        set_error("mpps_plan_adjoint: invalid argument");
        return MPPS_EINVAL;
    }
    Pol P = resolve(policy);
    mpps_status rc = plan_steps(m, n, normB, normY, P, m > 0 ? plan_adjoint_divisor(m, normX) : 1.0,
                                out);
    if (rc == MPPS_OK) {
        out->normX = normX;
        out->cost_ratio = cost_ratio(*out, P.tol);
    }
    return rc;
}

static mpps_status check_sizes(int n, int batch) {
    if (n <= 0 || batch < 0 || batch > 65535) {
        set_error("invalid size: n=%d batch=%d (need n>0, 0<=batch<=65535)", n, batch);
        return MPPS_EINVAL;
    }
    return MPPS_OK;
}

static mpps_status run_eval(const double* coeffs, int m, const double* A, int n, int batch,
                            const mpps_policy* policy, double* out, mpps_report* rep, void* stream,
                            bool expm) {
    clear_error();
    mpps_status rc = check_sizes(n, batch);
    if (rc) return rc;
    if (m < 0 || !coeffs) {
        set_error("invalid argument (m=%d, coeffs=%p)", m, (const void*)coeffs);
        return MPPS_EINVAL;
    }
    if (batch == 0) return MPPS_OK;   // nothing to do; empty tensors may have null data
    if (!A || !out) {
        set_error("invalid argument: null matrix pointer");
        return MPPS_EINVAL;
    }
    if ((rc = check_same_device(expm ? "expm_taylor_ss" : "ps_eval", {A, out}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elems = (size_t)batch * n * n;
    Staged a;
    rc = stage_in(A, elems, st, a);
    if (rc) return rc;
    const bool out_dev = is_device_ptr(out);
    DevBuf ob;
    double* dOut = out;
    if (!out_dev) {
        rc = ob.alloc(elems * sizeof(double), st);
        if (rc) return rc;
        dOut = (double*)ob.p;
    }
    Pol P = resolve(policy);
    const bool host_io = !out_dev || !is_device_ptr(A);
    rc = eval_device(coeffs, m, a.dev, n, batch, P, dOut, rep, st, expm, host_io);
    if (rc) return rc;
    if (!out_dev) {
        MPPS_CUDA_TRY(cudaMemcpyAsync(out, dOut, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (!is_device_ptr(A)) {
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MPPS_OK;
}

mpps_status ps_eval(const double* coeffs, int m, const double* A, int n, int batch,
                    const mpps_policy* policy, double* out, mpps_report* rep, void* stream) {
    return run_eval(coeffs, m, A, n, batch, policy, out, rep, stream, false);
}

mpps_status expm_taylor_ss(const double* A, int n, int batch, int m, const mpps_policy* policy,
                           double* out, mpps_report* rep, void* stream) {
    if (m <= 0) m = 30;
    if (m > 170) {
        set_error("expm_taylor_ss: degree m=%d too large", m);
        return MPPS_EINVAL;
    }
    // b_i = 1/i!: each quotient in extended precision, then rounded once to double
    std::vector<double> c(m + 1);
    long double f = 1.0L;
    for (int i = 0; i <= m; ++i) {
        if (i > 0) f /= (long double)i;
        c[i] = (double)f;
    }
    return run_eval(c.data(), m, A, n, batch, policy, out, rep, stream, true);
}

mpps_status expm_taylor_ss_grouped(const mpps_group_item* items, int count,
                                   const mpps_policy* policy, mpps_report* rep, void* stream) {
    clear_error();
    if (count < 0 || (count > 0 && !items)) {
        set_error("expm_taylor_ss_grouped: invalid argument (count=%d)", count);
        return MPPS_EINVAL;
    }
    if (count == 0) return MPPS_OK;
    for (int i = 0; i < count; ++i) {
        const int m = items[i].m <= 0 ? 30 : items[i].m;
        if (items[i].n <= 0 || m > 170 || !items[i].A || !items[i].out ||
            !is_device_ptr(items[i].A) || !is_device_ptr(items[i].out)) {
            set_error("expm_taylor_ss_grouped: item %d invalid (n=%d, m=%d, device pointers "
                      "required)", i, items[i].n, items[i].m);
            return MPPS_EINVAL;
        }
        mpps_status rc = check_same_device("expm_taylor_ss_grouped", {items[i].A, items[i].out});
        if (rc) return rc;
    }
    // Taylor coefficients b_i = 1/i! per degree, each quotient in extended precision
    std::vector<std::vector<double>> taylor(171);
    std::vector<GItem> g(count);
    for (int i = 0; i < count; ++i) {
        const int m = items[i].m <= 0 ? 30 : items[i].m;
        if (taylor[m].empty()) {
            taylor[m].resize(m + 1);
            long double f = 1.0L;
            for (int j = 0; j <= m; ++j) {
                if (j > 0) f /= (long double)j;
                taylor[m][j] = (double)f;
            }
        }
        g[i] = GItem{items[i].A, items[i].out, items[i].n, m, taylor[m].data()};
    }
    return grouped_eval(g.data(), count, policy, rep, (cudaStream_t)stream, true);
}

mpps_status ps_eval_grouped(const mpps_poly_item* items, int count, const mpps_policy* policy,
                            mpps_report* rep, void* stream) {
    clear_error();
    if (count < 0 || (count > 0 && !items)) {
        set_error("ps_eval_grouped: invalid argument (count=%d)", count);
        return MPPS_EINVAL;
    }
    if (count == 0) return MPPS_OK;
    std::vector<GItem> g(count);
    for (int i = 0; i < count; ++i) {
        const mpps_poly_item& it = items[i];
        if (it.n <= 0 || it.m < 0 || !it.coeffs || !it.A || !it.out || !is_device_ptr(it.A) ||
            !is_device_ptr(it.out)) {
            set_error("ps_eval_grouped: item %d invalid (n=%d, m=%d, coefficients and device "
                      "pointers required)", i, it.n, it.m);
            return MPPS_EINVAL;
        }
        mpps_status rc = check_same_device("ps_eval_grouped", {it.A, it.out});
        if (rc) return rc;
        g[i] = GItem{it.A, it.out, it.n, it.m, it.coeffs};
    }
    return grouped_eval(g.data(), count, policy, rep, (cudaStream_t)stream, false);
}

// C = op(A) B, op(A) = A or (trans_a) A^T: the emulated formats slice A's columns as the A
// operand; the others form the transpose first.
static mpps_status matmul_impl(const char* fn, const double* A, const double* B, double* C, int n,
                               int batch, int format, bool trans_a, void* stream) {
    clear_error();
    mpps_status rc = check_sizes(n, batch);
    if (rc) return rc;
    if (!(format >= MPPS_FMT_FP64 && format <= MPPS_FMT_FP8) && !MPPS_FMT_IS_F64E(format)) {
        set_error("%s: invalid format %d", fn, format);
        return MPPS_EINVAL;
    }
    if (batch == 0) return MPPS_OK;
    if (!A || !B || !C) {
        set_error("%s: null matrix pointer", fn);
        return MPPS_EINVAL;
    }
    if ((rc = check_same_device(fn, {A, B, C}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long nn = (long long)n * n;
    const size_t elems = (size_t)batch * nn;
    Staged a, b;
    if ((rc = stage_in(A, elems, st, a))) return rc;
    if ((rc = stage_in(B, elems, st, b))) return rc;
    const bool slice_t = trans_a && MPPS_FMT_IS_F64E(format);
    DevBuf tbuf;
    if (trans_a && !slice_t) {   // the other formats take A^T formed explicitly
        if ((rc = tbuf.alloc(elems * sizeof(double), st))) return rc;
        if ((rc = launch_transpose(a.dev, nn, (double*)tbuf.p, n, batch, st))) return rc;
        a.dev = (double*)tbuf.p;
    }
    const bool c_dev = is_device_ptr(C);
    DevBuf cb;
    double* dC = C;
    if (!c_dev) {
        if ((rc = cb.alloc(elems * sizeof(double), st))) return rc;
        dC = (double*)cb.p;
    }
    Epilogue ep = epilogue_plain(dC, nn);
    if (format == MPPS_FMT_FP64) {
        rc = launch_gemm_f64(a.dev, nn, b.dev, nn, n, batch, ep, st);
        if (rc) return rc;
    } else if (MPPS_FMT_IS_F64E(format)) {
        const int k = MPPS_F64E_SLICES(format);
        Arena L;
        __nv_bfloat16 *sa, *sb;
        int *ea, *eb, *err;
        double* bt;
        char* split;
        auto lay = [&](Arena& z) {
            sa = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, k));
            sb = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, k));
            ea = z.take<int>((size_t)batch * n);
            eb = z.take<int>((size_t)batch * n);
            bt = z.take<double>(elems);
            err = z.take<int>(1);
            split = z.take<char>(f64e_split_bytes());
        };
        lay(L);
        DevBuf ws;
        if ((rc = ws.alloc(L.off, st))) return rc;
        L.base = (char*)ws.p;
        L.off = 0;
        lay(L);
        MPPS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        MPPS_CUDA_TRY(cudaMemsetAsync(split, 0, f64e_split_flag_bytes(), st));
        if ((rc = slice_t ? launch_slice_cols_a(a.dev, nn, n, batch, k, sa, ea,
                                                (unsigned long long*)bt, st)
                          : launch_slice_rows(a.dev, nn, n, batch, k, sa, ea, st)))
            return rc;
        if ((rc = launch_slice_cols(b.dev, nn, n, batch, k, sb, eb, (unsigned long long*)bt, st)))
            return rc;
        if ((rc = launch_gemm_f64e(k, sa, k, ea, sb, k, eb, n, batch, batch, ep, err, st, nullptr,
                                   split)))
            return rc;
        int h_err = 0;
        MPPS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_err) {
            set_error("a bounded wait in the emulated FP64 product timed out");
            return MPPS_ETIMEOUT;
        }
    } else if (format == MPPS_FMT_FP8) {   // block scales along K (tcgen05 kind::mxf8f6f4)
        DevBuf ws;
        const size_t wb = fp8mx_ws_bytes(n, batch);
        if ((rc = ws.alloc(wb + 256, st))) return rc;
        int* err = (int*)((char*)ws.p + wb);
        MPPS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        rc = launch_product_fp8mx(a.dev, nn, b.dev, nn, n, batch, ep, fp8mx_ws_carve(ws.p, n, batch),
                                  err, st);
        if (rc) return rc;
        int h_err = 0;
        MPPS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_err) {
            set_error("a bounded wait in the tensor-core product timed out");
            return MPPS_ETIMEOUT;
        }
    } else {
        const int lld = low_ld(n);
        const long long low_bs = (long long)n * lld;
        const int es = low_elem_bytes(format);
        const bool x3 = format == MPPS_FMT_BF16X3;
        Arena L;
        char *ahi, *alo, *bhi, *blo;
        double *ma, *mb, *sa, *sb, *un;
        int* err;
        auto lay = [&](Arena& z) {
            ahi = z.take<char>((size_t)batch * low_bs * es);
            alo = z.take<char>(x3 ? (size_t)batch * low_bs * es : 0);
            bhi = z.take<char>((size_t)batch * low_bs * es);
            blo = z.take<char>(x3 ? (size_t)batch * low_bs * es : 0);
            ma = z.take<double>(batch);
            mb = z.take<double>(batch);
            sa = z.take<double>(batch);
            sb = z.take<double>(batch);
            un = z.take<double>(batch);
            err = z.take<int>(1);
        };
        lay(L);
        DevBuf ws;
        if ((rc = ws.alloc(L.off, st))) return rc;
        L.base = (char*)ws.p;
        L.off = 0;
        lay(L);
        MPPS_CUDA_TRY(cudaMemsetAsync(ma, 0, sizeof(double) * batch, st));
        MPPS_CUDA_TRY(cudaMemsetAsync(mb, 0, sizeof(double) * batch, st));
        MPPS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        if ((rc = launch_maxabs(a.dev, nn, n, batch, ma, st))) return rc;
        if ((rc = launch_maxabs(b.dev, nn, n, batch, mb, st))) return rc;
        if ((rc = launch_pow2_scales(ma, mb, batch, low_target_exp(format), sa, sb, un, st))) return rc;
        if ((rc = launch_convert(format, a.dev, nn, n, batch, ahi, alo, low_bs, lld, sa, false, st)))
            return rc;
        if ((rc = launch_convert(format, b.dev, nn, n, batch, bhi, blo, low_bs, lld, sb, true, st)))
            return rc;
        ep.alpha_b = un;
        rc = launch_gemm_tc(format, ahi, alo, bhi, blo, low_bs, low_bs, lld, n, batch, ep, err, st);
        if (rc) return rc;
        int h_err = 0;
        MPPS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_err) {
            set_error("a bounded wait in the tensor-core product timed out");
            return MPPS_ETIMEOUT;
        }
    }
    if (!c_dev) {
        MPPS_CUDA_TRY(cudaMemcpyAsync(C, dC, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (!is_device_ptr(A) || !is_device_ptr(B)) {
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MPPS_OK;
}

mpps_status mpps_matmul(const double* A, const double* B, double* C, int n, int batch, int format,
                        void* stream) {
    return matmul_impl("mpps_matmul", A, B, C, n, batch, format, false, stream);
}

mpps_status mpps_matmul_ta(const double* A, const double* B, double* C, int n, int batch,
                           int format, void* stream) {
    return matmul_impl("mpps_matmul_ta", A, B, C, n, batch, format, true, stream);
}

}  // extern "C"

namespace mpps {

// ---- tape of the reverse pass ----------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static mpps_status tape_layout(int m, int n, int batch, const Pol& pol, TapeLayout* L) {
    *L = TapeLayout();
    if (m < 1) {
        L->hdr_off = 0;
        L->bytes = sizeof(TapeHeader);
        return MPPS_OK;
    }
    const int s = pol.s > 0 ? std::min(pol.s, m) : ceil_sqrt_int(m);
    const int r = m / s;
    if (s > MPPS_MAX_S || r > MPPS_MAX_R) {
        set_error("m=%d with s=%d is outside the supported range (s<=%d, r<=%d)", m, s, MPPS_MAX_S,
                  MPPS_MAX_R);
        return MPPS_EINVAL;
    }
    L->s = s;
    L->r = r;
    L->fold = (m % s) == 0;
    L->i_top = L->fold ? r - 1 : r;
    L->recompute = pol.recompute && r >= 3;
    L->cseg = L->recompute ? ceil_sqrt_int(r) : 1;
    L->ck_top = r / L->cseg + 1;
    L->seg0 = r / L->cseg + 2;
    L->nslots = L->recompute ? L->seg0 + std::max(2, L->cseg) : r + 1;
    const size_t nn = (size_t)n * n;
    L->pw_off = 0;
    L->slot_off = align256(sizeof(double) * (size_t)batch * s * nn);
    L->hdr_off = align256(L->slot_off + sizeof(double) * (size_t)L->nslots * batch * nn);
    L->bytes = L->hdr_off + sizeof(TapeHeader);
    return MPPS_OK;
}

// Scratch of a product in any format (product_fmt): slice planes for the emulated products,
// rounded copies and power-of-two scales for the low-precision ones.
struct ProductWs {
    __nv_bfloat16 *slA = nullptr, *slB = nullptr;
    int *eA = nullptr, *eB = nullptr;
    unsigned long long* cmx = nullptr;
    char* split = nullptr;
    char *ahi = nullptr, *alo = nullptr, *bhi = nullptr, *blo = nullptr;
    double *ma = nullptr, *mb = nullptr, *sa = nullptr, *sb = nullptr, *un = nullptr;
    char* fp8 = nullptr;   // FP8 products with block scales (fp8mx_ws_bytes)
    void take(Arena& z, int n, int batch, int kmax, bool low) {
        if (kmax > 0) {
            slA = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, kmax));
            slB = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, kmax));
            eA = z.take<int>((size_t)batch * n);
            eB = z.take<int>((size_t)batch * n);
            cmx = z.take<unsigned long long>((size_t)batch * n);
            split = z.take<char>(f64e_split_bytes());
        }
        if (low) {
            const size_t lb = (size_t)batch * n * low_ld(n) * 4;   // widest low element: 4 bytes
            ahi = z.take<char>(lb);
            alo = z.take<char>(lb);
            bhi = z.take<char>(lb);
            blo = z.take<char>(lb);
            ma = z.take<double>(batch);
            mb = z.take<double>(batch);
            sa = z.take<double>(batch);
            sb = z.take<double>(batch);
            un = z.take<double>(batch);
            fp8 = z.take<char>(fp8mx_ws_bytes(n, batch));
        }
    }
};

// C = A B in format fmt with the fused epilogue ep (alpha = 1): FP64 pipe, emulated
// F64E(k) from exact slices of the rows of A and the columns of B, or a low-precision
// tensor-core product of A and B each scaled by a power of two from its largest entry
// (the building block mpps_matmul offers, used here with an epilogue).
// B's column slices made once for several emulated products with the same B (`planes`
// slices: any product of at most that many uses their leading planes).
struct SlicedB {
    const __nv_bfloat16* pl = nullptr;
    const int* e = nullptr;
    int planes = 0;
};

// a_t (emulated formats only): the A operand is A^T, sliced from A's columns.
static mpps_status product_fmt(int fmt, const double* A, long long a_bs, const double* B,
                               long long b_bs, int n, int batch, Epilogue ep, ProductWs& w,
                               int* d_err, cudaStream_t st, const SlicedB* preB = nullptr,
                               bool a_t = false) {
    const long long nn = (long long)n * n;
    if (a_t && !MPPS_FMT_IS_F64E(fmt)) {
        set_error("product_fmt: a transposed A operand needs an emulated format");
        return MPPS_EINVAL;
    }
    if (fmt == MPPS_FMT_FP64) return launch_gemm_f64(A, a_bs, B, b_bs, n, batch, ep, st);
    if (MPPS_FMT_IS_F64E(fmt)) {
        const int k = MPPS_F64E_SLICES(fmt);
        const bool pre = preB && preB->pl && preB->planes >= k;
        mpps_status rc = a_t ? launch_slice_cols_a(A, a_bs, n, batch, k, w.slA, w.eA, w.cmx, st)
                             : launch_slice_rows(A, a_bs, n, batch, k, w.slA, w.eA, st);
        if (!rc && !pre) rc = launch_slice_cols(B, b_bs, n, batch, k, w.slB, w.eB, w.cmx, st);
        if (!rc)
            rc = launch_gemm_f64e(k, w.slA, k, w.eA, pre ? preB->pl : w.slB, pre ? preB->planes : k,
                                  pre ? preB->e : w.eB, n, batch, batch, ep, d_err, st, nullptr,
                                  w.split);
        return rc;
    }
    if (!is_low(fmt) || !w.ahi) {
        set_error("product_fmt: format %d has no workspace", fmt);
        return MPPS_EINVAL;
    }
    if (fmt == MPPS_FMT_FP8)   // block scales along K instead of one scale per matrix
        return launch_product_fp8mx(A, a_bs, B, b_bs, n, batch, ep, fp8mx_ws_carve(w.fp8, n, batch),
                                    d_err, st);
    const int lld = low_ld(n);
    const long long low_bs = (long long)n * lld;
    MPPS_CUDA_TRY(cudaMemsetAsync(w.ma, 0, sizeof(double) * batch, st));
    MPPS_CUDA_TRY(cudaMemsetAsync(w.mb, 0, sizeof(double) * batch, st));
    mpps_status rc = launch_maxabs(A, a_bs, n, batch, w.ma, st);
    if (!rc) rc = launch_maxabs(B, b_bs, n, batch, w.mb, st);
    if (!rc) rc = launch_pow2_scales(w.ma, w.mb, batch, low_target_exp(fmt), w.sa, w.sb, w.un, st);
    if (!rc) rc = launch_convert(fmt, A, a_bs, n, batch, w.ahi, w.alo, low_bs, lld, w.sa, false, st);
    if (!rc) rc = launch_convert(fmt, B, b_bs, n, batch, w.bhi, w.blo, low_bs, lld, w.sb, true, st);
    if (rc) return rc;
    (void)nn;
    ep.alpha_b = w.un;
    return launch_gemm_tc(fmt, w.ahi, w.alo, w.bhi, w.blo, low_bs, low_bs, lld, n, batch, ep, d_err, st);
}

// The reverse pass's per-step formats: the forward rule of each matrix with u_i tightened by
// plan_adjoint_divisor, the batch taking the most precise format any matrix asks for.
static void adjoint_formats(int m, int n, int r, const Keep& k, const Pol& pol, int* fmt_adj) {
    for (int i = 0; i <= MPPS_MAX_R; ++i) fmt_adj[i] = MPPS_FMT_NONE;
    for (size_t b = 0; b < k.plans.size(); ++b) {
        const mpps_report& R = k.plans[b];
        mpps_report A;
        if (plan_steps(m, n, R.normB, R.normY, pol, plan_adjoint_divisor(m, R.normX), &A)) continue;
        for (int i = 1; i <= r; ++i)
            if (fmt_adj[i] == MPPS_FMT_NONE || prec_rank(A.fmt[i]) > prec_rank(fmt_adj[i]))
                fmt_adj[i] = A.fmt[i];
    }
    const int wp = pol.f64k > 0 ? MPPS_FMT_F64E(pol.f64k) : MPPS_FMT_FP64;
    for (int i = 1; i <= r; ++i)
        if (fmt_adj[i] == MPPS_FMT_NONE) fmt_adj[i] = wp;   // folded step: no product to run
}

// Forward pass into a tape: P_0 = p(X) into dOut, the power table and the Horner iterates
// into the tape, the formats of both passes into its header.  All pointers on the device.
static mpps_status forward_tape_dev(const double* coeffs, int m, const double* dA, int n, int batch,
                                    const Pol& pol, double* dOut, char* tape, const TapeLayout& L,
                                    int storage, cudaStream_t st) {
    TapeHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kTapeMagic;
    h.m = m;
    h.n = n;
    h.batch = batch;
    h.storage = storage;
    for (int i = 0; i <= MPPS_MAX_R; ++i) h.fmt[i] = h.fmt_adj[i] = MPPS_FMT_NONE;
    if (m >= 1) {
        Keep k;
        k.L = &L;
        k.pw = (double*)(tape + L.pw_off);
        k.slots = (double*)(tape + L.slot_off);
        Pol p = pol;
        p.var_s = 0;
        mpps_status rc = eval_device(coeffs, m, dA, n, batch, p, dOut, nullptr, st, false, false, &k);
        if (rc) return rc;
        h.s = L.s;
        h.r = L.r;
        for (int i = 0; i <= MPPS_MAX_R; ++i) h.fmt[i] = k.fmt[i];
        adjoint_formats(m, n, L.r, k, p, h.fmt_adj);
    } else {
        mpps_status rc = eval_device(coeffs, m, dA, n, batch, pol, dOut, nullptr, st, false, false);
        if (rc) return rc;
    }
    MPPS_CUDA_TRY(cudaMemcpyAsync(tape + L.hdr_off, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    return MPPS_OK;
}

// Reverse mode through the PS steps.  Forward: powers X_1..X_s and Horner iterates P_r..P_1
// on the tape.  Backward (f = <G, P_0>):
//   Pbar_0 = G;  for i = 1..r: Bbar_{i-1} = Pbar_{i-1};  Ybar += P_i^T Pbar_{i-1};
//                              Pbar_i = Pbar_{i-1} Y^T;   (fold: step r has P_r = b_m I,
//                              so Ybar += b_m Pbar_{r-1} and the loop stops)
//   Bbar_r = Pbar_r;  Xbar_j += sum_i b_{si+j} Bbar_i;  Xbar_s += Ybar;
//   for j = s..2: Xbar_{j-1} += Xbar_j X_1^T;  Xbar_1 += X_{j-1}^T Xbar_j;   grad = Xbar_1.
// The two products of reverse step i run in the header's fmt_adj[i]; the power chain in the
// working precision.  All pointers on the device.
static mpps_status adjoint_tape_dev(const double* coeffs, int m, const char* tape,
                                    const TapeLayout& L, const double* dG, int n, int batch,
                                    const Pol& pol, double* dGrad, int storage, cudaStream_t st) {
    const long long nn = (long long)n * n;
    const size_t elems = (size_t)batch * nn;
    TapeHeader h;
    MPPS_CUDA_TRY(cudaMemcpyAsync(&h, tape + L.hdr_off, sizeof(h), cudaMemcpyDeviceToHost, st));
    MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.magic != kTapeMagic || h.m != m || h.n != n || h.batch != batch || h.storage != storage ||
        (m >= 1 && (h.s != L.s || h.r != L.r))) {
        set_error("adjoint: the tape was not written by a forward call of this size and policy");
        return MPPS_EINVAL;
    }
    if (m == 0) {
        MPPS_CUDA_TRY(cudaMemsetAsync(dGrad, 0, elems * sizeof(double), st));
        return MPPS_OK;
    }
    const int s = L.s, r = L.r;
    const bool fold = L.fold;
    const int i_top = L.i_top;
    const long long pw_bs = (long long)s * nn;
    const double* pw = (const double*)(tape + L.pw_off);
    double* Pst = (double*)(tape + L.slot_off);   // recompute mode writes its rolling slots
    const int K = pol.f64k;
    const int wp = K > 0 ? MPPS_FMT_F64E(K) : MPPS_FMT_FP64;
    bool any_low = false;
    int kmax = K;
    for (int i = 1; i <= r; ++i) {
        for (int f : {h.fmt[i], h.fmt_adj[i]}) {
            if (is_low(f)) any_low = true;
            if (MPPS_FMT_IS_F64E(f)) kmax = std::max(kmax, MPPS_F64E_SLICES(f));
        }
    }
    // Y^T and X_1^T are the B operand of every reverse step and of every power's adjoint:
    // emulated products slice their columns once
    bool rev_f64e = false;
    for (int i = 1; i <= r; ++i) rev_f64e = rev_f64e || MPPS_FMT_IS_F64E(h.fmt_adj[i]);
    const bool pow_f64e = MPPS_FMT_IS_F64E(wp);
    Arena Z;
    double *xbar, *Ybar, *Pbar0, *Pbar1, *Yt, *X1t, *T;
    __nv_bfloat16 *plYt = nullptr, *plX1t = nullptr;
    int *eYt = nullptr, *eX1t = nullptr;
    ProductWs w;
    auto lay = [&](Arena& z) {
        xbar = z.take<double>((size_t)batch * pw_bs);
        Ybar = z.take<double>(elems);
        Pbar0 = z.take<double>(elems);
        Pbar1 = z.take<double>(elems);
        Yt = z.take<double>(elems);
        X1t = z.take<double>(elems);
        T = z.take<double>(elems);
        if (rev_f64e) {
            plYt = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, kmax));
            eYt = z.take<int>((size_t)batch * n);
        }
        if (pow_f64e) {
            plX1t = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, kmax));
            eX1t = z.take<int>((size_t)batch * n);
        }
        w = ProductWs();
        w.take(z, n, batch, kmax, any_low);
    };
    lay(Z);
    DevBuf ws;
    mpps_status rc = ws.alloc(Z.off, st);
    if (rc) return rc;
    Z.base = (char*)ws.p;
    Z.off = 0;
    lay(Z);
    if (w.split) MPPS_CUDA_TRY(cudaMemsetAsync(w.split, 0, f64e_split_flag_bytes(), st));
    DevErr* derr = nullptr;
    if ((rc = dev_err_get(&derr))) return rc;
    if ((rc = dev_err_check(derr, false))) return rc;
    auto product = [&](int fmt, const double* Am, long long a_bs, const double* Bm, long long b_bs,
                       const Epilogue& ep, const SlicedB* preB = nullptr,
                       bool a_t = false) -> mpps_status {
        return product_fmt(fmt, Am, a_bs, Bm, b_bs, n, batch, ep, w, derr->d, st, preB, a_t);
    };
    auto slotp = [&](int k) { return Pst + (size_t)k * batch * nn; };
    std::vector<double*> loc(r + 1, nullptr);   // where P_j is held now
    for (int j = 1; j <= i_top; ++j)
        if (L.is_ckpt(j)) loc[j] = slotp(L.ck_slot(j));
    const double* Y = pw + (long long)(s - 1) * nn;
    // P_{i-1} = B_{i-1} + P_i Y into dst, in the forward step's format
    auto horner_step = [&](int i, double* dst) -> mpps_status {
        Epilogue ep = epilogue_plain(dst, nn);
        ep.nt = s - 1;
        for (int j = 0; j < s; ++j) ep.coef[j] = coeffs[(i - 1) * s + j];
        ep.pw = pw; ep.pw_bstride = pw_bs;
        return product(h.fmt[i] >= 0 ? h.fmt[i] : wp, loc[i], nn, Y, pw_bs, ep);
    };
    // P_i for the reverse pass (ascending i): a missing one is recomputed with the rest of
    // its segment, P_{k-1} .. P_{i0} from the checkpoint k above
    auto P_at = [&](int i, mpps_status* err) -> double* {
        if (loc[i]) return loc[i];
        const int k = std::min((i / L.cseg + 1) * L.cseg, i_top);
        const int i0 = (i / L.cseg) * L.cseg + 1;
        for (int j = 1; j <= r; ++j)
            if (!L.is_ckpt(j)) loc[j] = nullptr;
        for (int j = k; j > i0; --j) {
            loc[j - 1] = slotp(L.seg0 + (j - 1 - i0));
            if ((*err = horner_step(j, loc[j - 1]))) return nullptr;
        }
        return loc[i];
    };
    MPPS_CUDA_TRY(cudaMemsetAsync(Ybar, 0, elems * sizeof(double), st));
    // Y^T and X_1^T, transposed from the strided power table
    if ((rc = launch_transpose(Y, pw_bs, Yt, n, batch, st))) return rc;
    if ((rc = launch_transpose(pw, pw_bs, X1t, n, batch, st))) return rc;
    SlicedB sYt, sX1t;
    if (rev_f64e) {
        if ((rc = launch_slice_cols(Yt, nn, n, batch, kmax, plYt, eYt, w.cmx, st))) return rc;
        sYt.pl = plYt; sYt.e = eYt; sYt.planes = kmax;
    }
    if (pow_f64e) {
        if ((rc = launch_slice_cols(X1t, nn, n, batch, kmax, plX1t, eX1t, w.cmx, st))) return rc;
        sX1t.pl = plX1t; sX1t.e = eX1t; sX1t.planes = kmax;
    }
    // Pbar_0 = G (read only); Pbar_1, Pbar_2, ... alternate between two buffers
    MPPS_CUDA_TRY(cudaMemsetAsync(xbar, 0, sizeof(double) * batch * pw_bs, st));
    const double* pc = dG;
    bool folded = false;
    for (int i = 1; i <= r; ++i) {
        // Bbar_{i-1} = Pbar_{i-1}: Xbar_j += b_{(i-1)s+j} Pbar_{i-1} for j = 1..s-1
        double c[MPPS_MAX_S + 1];
        for (int j = 0; j < s; ++j) c[j] = coeffs[(i - 1) * s + j];
        if ((rc = launch_axpy_blocks(xbar, pw_bs, n, batch, s - 1, c, pc, nn, st))) return rc;
        if (fold && i == r) {
            // P_r = b_m I: Ybar += b_m Pbar_{r-1}
            Epilogue ep = epilogue_plain(Ybar, nn);
            ep.alpha = coeffs[m];
            ep.add = Ybar; ep.add_bstride = nn; ep.add_coef = 1.0;
            if ((rc = launch_combine(n, batch, pc, nn, ep, st))) return rc;
            folded = true;
            break;
        }
        // Ybar += P_i^T Pbar_{i-1}
        double* Pi = P_at(i, &rc);
        if (rc) return rc;
        {
            Epilogue ep = epilogue_plain(Ybar, nn);
            ep.add = Ybar; ep.add_bstride = nn; ep.add_coef = 1.0;
            if (MPPS_FMT_IS_F64E(h.fmt_adj[i])) {   // P_i^T sliced from P_i's columns
                if ((rc = product(h.fmt_adj[i], Pi, nn, pc, nn, ep, nullptr, true))) return rc;
            } else {
                if ((rc = launch_transpose(Pi, nn, T, n, batch, st))) return rc;
                if ((rc = product(h.fmt_adj[i], T, nn, pc, nn, ep))) return rc;
            }
        }
        // Pbar_i = Pbar_{i-1} Y^T
        double* pn = (i & 1) ? Pbar0 : Pbar1;
        {
            Epilogue ep = epilogue_plain(pn, nn);
            if ((rc = product(h.fmt_adj[i], pc, nn, Yt, nn, ep, &sYt))) return rc;
        }
        pc = pn;
    }
    if (!folded) {   // Bbar_r = Pbar_r, B_r = sum_{j<=m-sr} b_{sr+j} X_j
        double c[MPPS_MAX_S + 1];
        const int t = m - s * r;
        for (int j = 0; j <= t; ++j) c[j] = coeffs[s * r + j];
        if ((rc = launch_axpy_blocks(xbar, pw_bs, n, batch, t, c, pc, nn, st))) return rc;
    }
    // Xbar_s += Ybar
    {
        double c[MPPS_MAX_S + 1] = {0};
        double* xs = xbar + (long long)(s - 1) * nn;
        c[1] = 1.0;
        if ((rc = launch_axpy_blocks(xs, pw_bs, n, batch, 1, c, Ybar, nn, st))) return rc;
    }
    // powers: X_j = X_{j-1} X_1, j = s..2 (working precision: they feed the low-order blocks)
    for (int j = s; j >= 2; --j) {
        double* xj = xbar + (long long)(j - 1) * nn;
        double* xjm = xbar + (long long)(j - 2) * nn;
        // Xbar_{j-1} += Xbar_j X_1^T
        Epilogue e1 = epilogue_plain(xjm, pw_bs);
        e1.add = xjm; e1.add_bstride = pw_bs; e1.add_coef = 1.0;
        if ((rc = product(wp, xj, pw_bs, X1t, nn, e1, &sX1t))) return rc;
        // Xbar_1 += X_{j-1}^T Xbar_j
        Epilogue e2 = epilogue_plain(xbar, pw_bs);
        e2.add = xbar; e2.add_bstride = pw_bs; e2.add_coef = 1.0;
        if (pow_f64e) {   // X_{j-1}^T sliced from the power table's columns
            if ((rc = product(wp, pw + (long long)(j - 2) * nn, pw_bs, xj, pw_bs, e2, nullptr, true)))
                return rc;
        } else {
            if ((rc = launch_scale_copy(pw + (long long)(j - 2) * nn, pw_bs, T, nn, n, batch, nullptr, st)))
                return rc;
            if ((rc = launch_transpose(T, nn, Pbar0, n, batch, st))) return rc;
            if ((rc = product(wp, Pbar0, nn, xj, pw_bs, e2))) return rc;
        }
    }
    if ((rc = launch_scale_copy(xbar, pw_bs, dGrad, nn, n, batch, nullptr, st))) return rc;
    return dev_err_enqueue(derr, st);
}

// The entry points' shared checks; resolves the policy and the tape layout.
static mpps_status tape_args(const char* fn, const double* coeffs, int m, int n, int batch,
                             const mpps_policy* policy, Pol* pol, TapeLayout* L) {
    mpps_status rc = check_sizes(n, batch);
    if (rc) return rc;
    if (m < 0 || !coeffs) {
        set_error("%s: invalid argument (m=%d)", fn, m);
        return MPPS_EINVAL;
    }
    *pol = resolve(policy);
    if (pol->f64k < 0 || pol->f64k > MPPS_F64E_MAX_SLICES) {
        set_error("f64_slices=%d outside 0..%d", pol->f64k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    return tape_layout(m, n, batch, *pol, L);
}

}  // namespace mpps

extern "C" {

size_t ps_eval_tape_bytes(int m, int n, int batch, const mpps_policy* policy) {
    clear_error();
    Pol pol;
    TapeLayout L;
    const double one = 1.0;
    if (tape_args("ps_eval_tape_bytes", &one, m, n, batch, policy, &pol, &L)) return 0;
    return L.bytes;
}

// FP32 storage: widen into a workspace copy (exact); results narrowed to nearest.
static mpps_status widen_in(const void* p, int storage, size_t elems, cudaStream_t st, DevBuf& buf,
                            const double** out) {
    if (storage == MPPS_STORAGE_F64) {
        *out = (const double*)p;
        return MPPS_OK;
    }
    mpps_status rc = buf.alloc(elems * sizeof(double), st);
    if (rc) return rc;
    if ((rc = launch_widen_f32((const float*)p, (double*)buf.p, (long long)elems, st))) return rc;
    *out = (const double*)buf.p;
    return MPPS_OK;
}

static mpps_status storage_args(const char* fn, int storage, std::initializer_list<const void*> ptrs) {
    if (storage != MPPS_STORAGE_F64 && storage != MPPS_STORAGE_F32) {
        set_error("%s: storage %d is neither MPPS_STORAGE_F64 nor MPPS_STORAGE_F32", fn, storage);
        return MPPS_EINVAL;
    }
    for (const void* p : ptrs)
        if (!p || !is_device_ptr(p)) {
            set_error("%s: matrix and tape pointers must be device pointers", fn);
            return MPPS_EINVAL;
        }
    return check_same_device(fn, ptrs);
}

mpps_status ps_eval_forward_tape(const double* coeffs, int m, const void* A, int storage, int n,
                                 int batch, const mpps_policy* policy, void* out, void* tape,
                                 size_t tape_bytes, void* stream) {
    clear_error();
    Pol pol;
    TapeLayout L;
    mpps_status rc = tape_args("ps_eval_forward_tape", coeffs, m, n, batch, policy, &pol, &L);
    if (rc) return rc;
    if (batch == 0) return MPPS_OK;
    if ((rc = storage_args("ps_eval_forward_tape", storage, {A, out, tape}))) return rc;
    if (tape_bytes < L.bytes) {
        set_error("ps_eval_forward_tape: the tape holds %zu bytes, %zu needed (ps_eval_tape_bytes)",
                  tape_bytes, L.bytes);
        return MPPS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elems = (size_t)batch * n * n;
    DevBuf ain, obuf;
    const double* dA = nullptr;
    if ((rc = widen_in(A, storage, elems, st, ain, &dA))) return rc;
    double* dOut = (double*)out;
    if (storage == MPPS_STORAGE_F32) {
        if ((rc = obuf.alloc(elems * sizeof(double), st))) return rc;
        dOut = (double*)obuf.p;
    }
    if ((rc = forward_tape_dev(coeffs, m, dA, n, batch, pol, dOut, (char*)tape, L, storage, st)))
        return rc;
    if (storage == MPPS_STORAGE_F32)
        return launch_narrow_f64(dOut, (float*)out, (long long)elems, st);
    return MPPS_OK;
}

mpps_status ps_eval_adjoint_tape(const double* coeffs, int m, const void* tape, size_t tape_bytes,
                                 const void* G, int storage, int n, int batch,
                                 const mpps_policy* policy, void* gradA, void* stream) {
    clear_error();
    Pol pol;
    TapeLayout L;
    mpps_status rc = tape_args("ps_eval_adjoint_tape", coeffs, m, n, batch, policy, &pol, &L);
    if (rc) return rc;
    if (batch == 0) return MPPS_OK;
    if ((rc = storage_args("ps_eval_adjoint_tape", storage, {tape, G, gradA}))) return rc;
    if (tape_bytes < L.bytes) {
        set_error("ps_eval_adjoint_tape: the tape holds %zu bytes, %zu needed", tape_bytes, L.bytes);
        return MPPS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elems = (size_t)batch * n * n;
    DevBuf gin, gbuf;
    const double* dG = nullptr;
    if ((rc = widen_in(G, storage, elems, st, gin, &dG))) return rc;
    double* dGrad = (double*)gradA;
    if (storage == MPPS_STORAGE_F32) {
        if ((rc = gbuf.alloc(elems * sizeof(double), st))) return rc;
        dGrad = (double*)gbuf.p;
    }
    if ((rc = adjoint_tape_dev(coeffs, m, (const char*)tape, L, dG, n, batch, pol, dGrad, storage, st)))
        return rc;
    if (storage == MPPS_STORAGE_F32)
        return launch_narrow_f64(dGrad, (float*)gradA, (long long)elems, st);
    return MPPS_OK;
}

// Forward into a private tape, then the reverse pass.
static mpps_status adjoint_private(const char* fn, const double* coeffs, int m, const void* A,
                                   const void* G, int storage, int n, int batch,
                                   const mpps_policy* policy, void* gradA, void* stream) {
    clear_error();
    Pol pol;
    TapeLayout L;
    mpps_status rc = tape_args(fn, coeffs, m, n, batch, policy, &pol, &L);
    if (rc) return rc;
    if (batch == 0) return MPPS_OK;
    if (!A || !G || !gradA) {
        set_error("%s: null matrix pointer", fn);
        return MPPS_EINVAL;
    }
    if ((rc = check_same_device(fn, {A, G, gradA}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elems = (size_t)batch * n * n;
    const size_t es = storage == MPPS_STORAGE_F32 ? sizeof(float) : sizeof(double);
    // host matrices are staged in and out (FP64 only; the FP32 variant takes device pointers)
    const bool host_io = !is_device_ptr(A) || !is_device_ptr(G) || !is_device_ptr(gradA);
    if (host_io && storage == MPPS_STORAGE_F32) {
        set_error("%s: device pointers required", fn);
        return MPPS_EINVAL;
    }
    Staged a, g;
    const void *dA = A, *dG = G;
    if (host_io) {
        if ((rc = stage_in((const double*)A, elems, st, a))) return rc;
        if ((rc = stage_in((const double*)G, elems, st, g))) return rc;
        dA = a.dev;
        dG = g.dev;
    }
    DevBuf tb, ob, gb;
    if ((rc = tb.alloc(L.bytes, st))) return rc;
    if ((rc = ob.alloc(elems * es, st))) return rc;
    void* dGrad = gradA;
    if (!is_device_ptr(gradA)) {
        if ((rc = gb.alloc(elems * sizeof(double), st))) return rc;
        dGrad = gb.p;
    }
    if ((rc = ps_eval_forward_tape(coeffs, m, dA, storage, n, batch, policy, ob.p, tb.p, L.bytes, stream)))
        return rc;
    if ((rc = ps_eval_adjoint_tape(coeffs, m, tb.p, L.bytes, dG, storage, n, batch, policy, dGrad,
                                   stream)))
        return rc;
    if (dGrad != gradA) {
        MPPS_CUDA_TRY(cudaMemcpyAsync(gradA, dGrad, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (host_io) {
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    DevErr* derr = nullptr;
    if ((rc = dev_err_get(&derr))) return rc;
    return dev_err_check(derr, host_io);
}

mpps_status ps_eval_adjoint(const double* coeffs, int m, const double* A, const double* G, int n,
                            int batch, const mpps_policy* policy, double* gradA, void* stream) {
    return adjoint_private("ps_eval_adjoint", coeffs, m, A, G, MPPS_STORAGE_F64, n, batch, policy,
                           gradA, stream);
}

mpps_status ps_eval_adjoint_f32(const double* coeffs, int m, const float* A, const float* G, int n,
                                int batch, const mpps_policy* policy, float* gradA, void* stream) {
    return adjoint_private("ps_eval_adjoint_f32", coeffs, m, A, G, MPPS_STORAGE_F32, n, batch,
                           policy, gradA, stream);
}

mpps_status expm_taylor_ss_adjoint(const double* A, const double* G, int n, int batch, int m,
                                   const mpps_policy* policy, double* gradA, void* stream) {
    clear_error();
    mpps_status rc = check_sizes(n, batch);
    if (rc) return rc;
    if (m <= 0) m = 30;
    if (m > 170) {
        set_error("expm_taylor_ss_adjoint: degree m=%d too large", m);
        return MPPS_EINVAL;
    }
    if (batch == 0) return MPPS_OK;
    if (!A || !G || !gradA) {
        set_error("expm_taylor_ss_adjoint: null matrix pointer");
        return MPPS_EINVAL;
    }
    if ((rc = check_same_device("expm_taylor_ss_adjoint", {A, G, gradA}))) return rc;
    const Pol pol = resolve(policy);
    if (pol.f64k < 0 || pol.f64k > MPPS_F64E_MAX_SLICES) {
        set_error("f64_slices=%d outside 0..%d", pol.f64k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const int K = pol.f64k;
    // the polynomial and its reverse pass under the caller's precision rule (the Horner
    // steps of both passes by eq. (2.8), the reverse one tightened as in ps_eval_adjoint);
    // the squarings and their reverse pass in the working precision (FP64 pipe or emulated
    // with K slices): their errors are amplified
    mpps_policy fpol;
    if (policy) fpol = *policy; else mpps_policy_default(&fpol);
    fpol.variable_s = 0;
    std::vector<double> c(m + 1);   // b_i = 1/i!, as in expm_taylor_ss
    {
        long double f = 1.0L;
        for (int i = 0; i <= m; ++i) {
            if (i > 0) f /= (long double)i;
            c[i] = (double)f;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long nn = (long long)n * n;
    const size_t elems = (size_t)batch * nn;
    Staged a, g;
    if ((rc = stage_in(A, elems, st, a))) return rc;
    if ((rc = stage_in(G, elems, st, g))) return rc;
    const bool o_dev = is_device_ptr(gradA);

    // ---- sigma per matrix (eq. (3.6)), X = 2^-sigma A
    Arena L1;
    double *X, *partial, *anorm;
    int* d_sigma;
    auto lay1 = [&](Arena& z) {
        X = z.take<double>(elems);
        partial = z.take<double>(norm1_partial_elems(n, batch));
        anorm = z.take<double>(batch);
        d_sigma = z.take<int>(batch);
    };
    lay1(L1);
    DevBuf ws1;
    if ((rc = ws1.alloc(L1.off, st))) return rc;
    L1.base = (char*)ws1.p;
    L1.off = 0;
    lay1(L1);
    if ((rc = launch_norm1(a.dev, nn, n, batch, partial, anorm, st))) return rc;
    if ((rc = launch_sigma(anorm, batch, d_sigma, st))) return rc;
    if ((rc = launch_scale_copy(a.dev, nn, X, nn, n, batch, d_sigma, st))) return rc;
    std::vector<int> sigma(batch);
    MPPS_CUDA_TRY(cudaMemcpyAsync(sigma.data(), d_sigma, sizeof(int) * batch,
                                  cudaMemcpyDeviceToHost, st));
    MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    int sig_max = 0;
    for (int b = 0; b < batch; ++b) sig_max = std::max(sig_max, sigma[b]);

    // ---- workspace: the squarings S_0..S_{sigma-1}, two upstream buffers, scratch
    Arena L2;
    double *S, *Sb0, *Sb1, *T, *tmp, *Xbar, *dGrad = gradA;
    int* d_lists;
    __nv_bfloat16 *slA = nullptr, *slB = nullptr;
    int *eA = nullptr, *eB = nullptr;
    unsigned long long* cmx = nullptr;
    char* split = nullptr;
    auto lay2 = [&](Arena& z) {
        S = z.take<double>((size_t)std::max(sig_max, 1) * elems);
        Sb0 = z.take<double>(elems);
        Sb1 = z.take<double>(elems);
        T = z.take<double>(elems);
        tmp = z.take<double>(elems);
        Xbar = z.take<double>(elems);
        d_lists = z.take<int>((size_t)std::max(sig_max, 1) * batch);
        if (!o_dev) dGrad = z.take<double>(elems);
        if (K > 0) {
            slA = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            slB = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            eA = z.take<int>((size_t)batch * n);
            eB = z.take<int>((size_t)batch * n);
            cmx = z.take<unsigned long long>((size_t)batch * n);
            split = z.take<char>(f64e_split_bytes());
        }
    };
    lay2(L2);
    DevBuf ws2;
    if ((rc = ws2.alloc(L2.off, st))) return rc;
    L2.base = (char*)ws2.p;
    L2.off = 0;
    lay2(L2);
    if (split) MPPS_CUDA_TRY(cudaMemsetAsync(split, 0, f64e_split_flag_bytes(), st));
    DevErr* derr = nullptr;
    if (K > 0) {
        if ((rc = dev_err_get(&derr))) return rc;
        if ((rc = dev_err_check(derr, false))) return rc;
    }
    // C = Am Bm (+ add) for the `cnt` matrices listed in `list` (all when null)
    auto product = [&](const double* Am, const double* Bm, int cnt, const int* list,
                       const Epilogue& ep) -> mpps_status {
        if (K == 0) return launch_gemm_f64(Am, nn, Bm, nn, n, cnt, ep, st, list);
        mpps_status r1 = launch_slice_rows(Am, nn, n, batch, K, slA, eA, st);
        if (!r1) r1 = launch_slice_cols(Bm, nn, n, batch, K, slB, eB, cmx, st);
        if (!r1)
            r1 = launch_gemm_f64e(K, slA, K, eA, slB, K, eB, n, cnt, batch, ep, derr->d, st, list,
                                  split);
        return r1;
    };

    // ---- forward: S_0 = p(X) (its powers and Horner iterates kept on a tape for the reverse
    // pass), S_{k+1} = S_k^2 for the matrices with sigma > k + 1
    const Pol tpol = resolve(&fpol);
    TapeLayout TL;
    if ((rc = tape_layout(m, n, batch, tpol, &TL))) return rc;
    DevBuf tape;
    if ((rc = tape.alloc(TL.bytes, st))) return rc;
    if ((rc = forward_tape_dev(c.data(), m, X, n, batch, tpol, S, (char*)tape.p, TL, MPPS_STORAGE_F64,
                               st)))
        return rc;
    std::vector<int> lists((size_t)std::max(sig_max, 1) * batch);
    std::vector<int> counts(std::max(sig_max, 1), 0);
    for (int k = 0; k < sig_max; ++k)
        for (int b = 0; b < batch; ++b)
            if (sigma[b] > k) lists[(size_t)k * batch + counts[k]++] = b;
    MPPS_CUDA_TRY(cudaMemcpyAsync(d_lists, lists.data(), sizeof(int) * lists.size(),
                                  cudaMemcpyHostToDevice, st));
    for (int k = 0; k + 1 < sig_max; ++k) {
        // S_{k+1} is needed by the matrices with sigma > k + 1: list k + 1
        Epilogue ep = epilogue_plain(S + (size_t)(k + 1) * elems, nn);
        const double* Sk = S + (size_t)k * elems;
        if ((rc = product(Sk, Sk, counts[k + 1], d_lists + (size_t)(k + 1) * batch, ep))) return rc;
    }

    // ---- backward through the squarings: Sbar_k = Sbar_{k+1} S_k^T + S_k^T Sbar_{k+1}.
    // Step k reads buffer k mod 2 and writes buffer (k + 1) mod 2, so matrix b starts with
    // G in buffer (sigma_b + 1) mod 2 and every matrix ends in buffer 1.
    double* Sb[2] = {Sb0, Sb1};
    for (int b = 0; b < batch; ++b)
        MPPS_CUDA_TRY(cudaMemcpyAsync(Sb[(sigma[b] + 1) & 1] + (size_t)b * nn,
                                      g.dev + (size_t)b * nn, sizeof(double) * nn,
                                      cudaMemcpyDeviceToDevice, st));
    for (int k = sig_max - 1; k >= 0; --k) {
        const int* lk = d_lists + (size_t)k * batch;
        if ((rc = launch_transpose(S + (size_t)k * elems, nn, T, n, batch, st))) return rc;
        Epilogue e1 = epilogue_plain(tmp, nn);   // Sbar_{k+1} S_k^T
        if ((rc = product(Sb[k & 1], T, counts[k], lk, e1))) return rc;
        Epilogue e2 = epilogue_plain(Sb[(k + 1) & 1], nn);   // S_k^T Sbar_{k+1} + that
        e2.add = tmp;
        e2.add_bstride = nn;
        e2.add_coef = 1.0;
        if ((rc = product(T, Sb[k & 1], counts[k], lk, e2))) return rc;
    }
    // ---- through p: Xbar = L_p(X^T, Sbar_0); then Abar = 2^-sigma Xbar
    if ((rc = adjoint_tape_dev(c.data(), m, (const char*)tape.p, TL, Sb[1], n, batch, tpol, Xbar,
                               MPPS_STORAGE_F64, st)))
        return rc;
    if ((rc = launch_scale_copy(Xbar, nn, dGrad, nn, n, batch, d_sigma, st))) return rc;
    if (K > 0) {
        if ((rc = dev_err_enqueue(derr, st))) return rc;
        if (!o_dev && (rc = dev_err_check(derr, true))) return rc;
    }
    if (!o_dev) {
        MPPS_CUDA_TRY(cudaMemcpyAsync(gradA, dGrad, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (K > 0 && (rc = dev_err_check(derr, true))) return rc;
    } else {
        // the workspace above is released stream-ordered; the staged inputs too
        if (!is_device_ptr(A) || !is_device_ptr(G)) MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MPPS_OK;
}

}  // extern "C"

extern "C" {

mpps_status expm_pade13(const double* A, int n, int batch, const mpps_policy* policy, double* out,
                        void* stream) {
    clear_error();
    mpps_status rc = check_sizes(n, batch);
    if (rc) return rc;
    if (batch == 0) return MPPS_OK;
    if (!A || !out) {
        set_error("expm_pade13: null matrix pointer");
        return MPPS_EINVAL;
    }
    if ((rc = check_same_device("expm_pade13", {A, out}))) return rc;
    const Pol pol = resolve(policy);
    if (pol.f64k < 0 || pol.f64k > MPPS_F64E_MAX_SLICES) {
        set_error("f64_slices=%d outside 0..%d", pol.f64k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const int K = pol.f64k;
    cudaStream_t st = (cudaStream_t)stream;
    const long long nn = (long long)n * n;
    const size_t elems = (size_t)batch * nn;
    Staged a;
    if ((rc = stage_in(A, elems, st, a))) return rc;
    const bool o_dev = is_device_ptr(out);

    // [13/13] Pade coefficients c_j = (26-j)! 13! / (26! j! (13-j)!), by the ratio
    // c_{j+1} / c_j = (13 - j) / ((26 - j)(j + 1)); even and odd parts as polynomials in X^2
    double c[14];
    {
        long double v = 1.0L;
        for (int j = 0; j <= 13; ++j) {
            c[j] = (double)v;
            v = v * (long double)(13 - j) / ((long double)(26 - j) * (long double)(j + 1));
        }
    }
    double ce[7], co[7];
    for (int k = 0; k <= 6; ++k) {
        ce[k] = c[2 * k];
        co[k] = c[2 * k + 1];
    }

    // ---- sigma = max(0, ceil(log2(||A||_1 / theta_13))), theta_13 = 5.371920351148152
    Arena L;
    double *X, *X2, *V, *W, *U, *P, *Q, *Rb1, *partial, *anorm, *dOut = out;
    int *d_sigma, *d_lists, *info;
    __nv_bfloat16 *slA = nullptr, *slB = nullptr;
    int *eA = nullptr, *eB = nullptr;
    unsigned long long* cmx = nullptr;
    char* split = nullptr;
    void* luws = nullptr;
    auto lay = [&](Arena& z) {
        X = z.take<double>(elems);
        X2 = z.take<double>(elems);
        V = z.take<double>(elems);
        W = z.take<double>(elems);
        U = z.take<double>(elems);
        P = z.take<double>(elems);
        Q = z.take<double>(elems);
        Rb1 = z.take<double>(elems);
        partial = z.take<double>(norm1_partial_elems(n, batch));
        anorm = z.take<double>(batch);
        d_sigma = z.take<int>(batch);
        d_lists = z.take<int>((size_t)batch * 64);
        info = z.take<int>((size_t)batch);   // first zero pivot of the LU, per matrix
        luws = z.take<char>(lu_workspace_bytes(n, K));
        if (!o_dev) dOut = z.take<double>(elems);
        if (K > 0) {
            slA = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            slB = z.take<__nv_bfloat16>(f64e_plane_elems(n, batch, K));
            eA = z.take<int>((size_t)batch * n);
            eB = z.take<int>((size_t)batch * n);
            cmx = z.take<unsigned long long>((size_t)batch * n);
            split = z.take<char>(f64e_split_bytes());
        }
    };
    lay(L);
    DevBuf ws;
    if ((rc = ws.alloc(L.off, st))) return rc;
    L.base = (char*)ws.p;
    L.off = 0;
    lay(L);
    if (split) MPPS_CUDA_TRY(cudaMemsetAsync(split, 0, f64e_split_flag_bytes(), st));
    DevErr* derr = nullptr;
    if (K > 0) {
        if ((rc = dev_err_get(&derr))) return rc;
        if ((rc = dev_err_check(derr, false))) return rc;
    }
    auto product = [&](const double* Am, const double* Bm, int cnt, const int* list,
                       const Epilogue& ep) -> mpps_status {
        if (K == 0) return launch_gemm_f64(Am, nn, Bm, nn, n, cnt, ep, st, list);
        mpps_status r1 = launch_slice_rows(Am, nn, n, batch, K, slA, eA, st);
        if (!r1) r1 = launch_slice_cols(Bm, nn, n, batch, K, slB, eB, cmx, st);
        if (!r1)
            r1 = launch_gemm_f64e(K, slA, K, eA, slB, K, eB, n, cnt, batch, ep, derr->d, st, list,
                                  split);
        return r1;
    };

    if ((rc = launch_norm1(a.dev, nn, n, batch, partial, anorm, st))) return rc;
    std::vector<double> hnorm(batch);
    MPPS_CUDA_TRY(cudaMemcpyAsync(hnorm.data(), anorm, sizeof(double) * batch,
                                  cudaMemcpyDeviceToHost, st));
    MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    const double theta13 = 5.371920351148152;
    std::vector<int> sigma(batch, 0);
    int sig_max = 0;
    for (int b = 0; b < batch; ++b) {
        int sg = 0;
        if (!std::isfinite(hnorm[b])) {   // no sigma brings it into range; the solve would
            set_error("expm_pade13: ||A||_1 of matrix %d is not finite", b);   // be garbage
            return MPPS_EINVAL;
        }
        if (!(hnorm[b] <= theta13))       // smallest sigma with ||A|| 2^-sigma <= theta_13
            while (ldexp(hnorm[b], -sg) > theta13 && sg < 1000) ++sg;
        sigma[b] = sg;
        sig_max = std::max(sig_max, sg);
    }
    if (sig_max > 64) {
        set_error("expm_pade13: ||A||_1 needs %d squarings (at most 64)", sig_max);
        return MPPS_EINVAL;
    }
    MPPS_CUDA_TRY(cudaMemcpyAsync(d_sigma, sigma.data(), sizeof(int) * batch,
                                  cudaMemcpyHostToDevice, st));
    if ((rc = launch_scale_copy(a.dev, nn, X, nn, n, batch, d_sigma, st))) return rc;

    // ---- numerator and denominator from one power chain: with V = even part and
    // U = X (odd part / X), both polynomials in X^2,  p = V + U,  q = p(-X) = V - U
    {
        Epilogue ep = epilogue_plain(X2, nn);
        if ((rc = product(X, X, batch, nullptr, ep))) return rc;
    }
    if ((rc = ps_eval(ce, 6, X2, n, batch, policy, V, nullptr, stream))) return rc;
    if ((rc = ps_eval(co, 6, X2, n, batch, policy, W, nullptr, stream))) return rc;
    {
        Epilogue ep = epilogue_plain(U, nn);
        if ((rc = product(X, W, batch, nullptr, ep))) return rc;
    }
    for (int sgn = 0; sgn < 2; ++sgn) {   // P = V + U, Q = V - U
        Epilogue ep = epilogue_plain(sgn == 0 ? P : Q, nn);
        ep.alpha = sgn == 0 ? 1.0 : -1.0;
        ep.add = V;
        ep.add_bstride = nn;
        ep.add_coef = 1.0;
        if ((rc = launch_combine(n, batch, U, nn, ep, st))) return rc;
    }
    // ---- R = q^-1 p by LU with partial pivoting, in the products of the working precision
    // (q_13 has no zeros in the disc |x| <= theta_13, so the exact q(X) is nonsingular there;
    // the first zero pivot is still read back at the end: q assembled under a mixed policy is
    // not the exact one)
    if ((rc = lu_solve_dev(Q, P, P, n, batch, K, luws, info, K > 0 ? derr->d : nullptr, st))) return rc;
    // ---- sigma squarings per matrix (index lists), then each result from its buffer
    std::vector<int> lists((size_t)std::max(sig_max, 1) * batch);
    std::vector<int> counts(std::max(sig_max, 1), 0);
    for (int k = 0; k < sig_max; ++k)
        for (int b = 0; b < batch; ++b)
            if (sigma[b] > k) lists[(size_t)k * batch + counts[k]++] = b;
    int* dl = d_lists;
    DevBuf extra;
    if ((size_t)sig_max * batch > (size_t)batch * 64) {
        if ((rc = extra.alloc(sizeof(int) * lists.size(), st))) return rc;
        dl = (int*)extra.p;
    }
    MPPS_CUDA_TRY(cudaMemcpyAsync(dl, lists.data(), sizeof(int) * lists.size(),
                                  cudaMemcpyHostToDevice, st));
    double* buf[2] = {P, Rb1};
    for (int k = 0; k < sig_max; ++k) {
        Epilogue ep = epilogue_plain(buf[(k + 1) & 1], nn);
        if ((rc = product(buf[k & 1], buf[k & 1], counts[k], dl + (size_t)k * batch, ep))) return rc;
    }
    if ((rc = launch_select_copy(buf[0], buf[1], d_sigma, dOut, n, batch, 0.0, st))) return rc;
    if (K > 0 && (rc = dev_err_enqueue(derr, st))) return rc;
    std::vector<int> hinfo((size_t)batch);
    MPPS_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * hinfo.size(), cudaMemcpyDeviceToHost, st));
    if (!o_dev) {
        MPPS_CUDA_TRY(cudaMemcpyAsync(out, dOut, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (K > 0 && (rc = dev_err_check(derr, true))) return rc;
    } else {
        MPPS_CUDA_TRY(cudaStreamSynchronize(st));   // the LU info lives in this call's workspace
        if (K > 0 && (rc = dev_err_check(derr, true))) return rc;
    }
    for (int b = 0; b < batch; ++b)
        if (hinfo[b] != 0) {
            set_error("expm_pade13: q(X) of matrix %d is singular (zero pivot in column %d)", b,
                      hinfo[b] - 1);
            return MPPS_ECHECK;
        }
    return MPPS_OK;
}

mpps_status lu_solve(const double* Q, const double* P, int n, int batch, const mpps_policy* policy,
                     double* R, void* stream) {
    clear_error();
    mpps_status rc = check_sizes(n, batch);
    if (rc) return rc;
    if (batch == 0) return MPPS_OK;
    if (!Q || !P || !R) {
        set_error("lu_solve: null matrix pointer");
        return MPPS_EINVAL;
    }
    if ((rc = check_same_device("lu_solve", {Q, P, R}))) return rc;
    const Pol pol = resolve(policy);
    if (pol.f64k < 0 || pol.f64k > MPPS_F64E_MAX_SLICES) {
        set_error("f64_slices=%d outside 0..%d", pol.f64k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const int K = pol.f64k;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elems = (size_t)batch * n * n;
    Staged q, p;
    if ((rc = stage_in(Q, elems, st, q)) || (rc = stage_in(P, elems, st, p))) return rc;
    const bool o_dev = is_device_ptr(R);
    Arena L;
    int* info = nullptr;
    void* luws = nullptr;
    double* dR = R;
    auto lay = [&](Arena& z) {
        info = z.take<int>((size_t)batch);
        luws = z.take<char>(lu_workspace_bytes(n, K));
        if (!o_dev) dR = z.take<double>(elems);
    };
    lay(L);
    DevBuf ws;
    if ((rc = ws.alloc(L.off, st))) return rc;
    L.base = (char*)ws.p;
    L.off = 0;
    lay(L);
    DevErr* derr = nullptr;
    if (K > 0) {
        if ((rc = dev_err_get(&derr))) return rc;
        if ((rc = dev_err_check(derr, false))) return rc;
    }
    if ((rc = lu_solve_dev(q.dev, p.dev, dR, n, batch, K, luws, info, K > 0 ? derr->d : nullptr, st)))
        return rc;
    if (K > 0 && (rc = dev_err_enqueue(derr, st))) return rc;
    std::vector<int> hinfo((size_t)batch);
    MPPS_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * hinfo.size(), cudaMemcpyDeviceToHost, st));
    if (!o_dev)
        MPPS_CUDA_TRY(cudaMemcpyAsync(R, dR, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
    MPPS_CUDA_TRY(cudaStreamSynchronize(st));
    if (K > 0 && (rc = dev_err_check(derr, true))) return rc;
    for (int b = 0; b < batch; ++b)
        if (hinfo[b] != 0) {
            set_error("lu_solve: Q of system %d is singular (zero pivot in column %d)", b, hinfo[b] - 1);
            return MPPS_ECHECK;
        }
    return MPPS_OK;
}

}  // extern "C"
