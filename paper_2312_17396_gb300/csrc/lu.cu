// lu.cu -- R = Q^-1 P by LU factorisation with partial pivoting: the q(X)^-1 p(X) solve of
// the [13/13] Pade approximant (Section 4.1, the diagonal Pade approximant r_m = q_m^-1 p_m).
//
// Blocked right-looking LU (Golub and Van Loan, Algorithm 3.4.2 with row interchanges), laid
// out for a GPU whose FP64 pipe gives about 1 TFLOP/s while the emulated FP64 product on the
// BF16 tensor cores gives tens of TFLOP/s:
//
//   * Q and P are copied into a tile-major layout: T x T tiles of TB x TB doubles, each tile
//     a contiguous row-major TB x TB matrix, n padded to N = T TB with Q = diag(Q, I) and
//     P = diag(P, 0) (the padded unknowns are zero).  Every block operation below is then a
//     batch of TB x TB products, run by the existing products in grid mode (product z takes
//     A tile z / nJ and B tile z % nJ).
//   * Panel k (tile column k, rows k TB .. N): one thread-block cluster.  CTA c holds rows
//     [c R, (c + 1) R) of the panel in its shared memory (in place in the tiles when the
//     panel is too tall); per column: local pivot candidates, a cluster barrier, the pivot
//     row read from its owner's shared memory, a second barrier, the interchange, the
//     multipliers and the rank-1 update of the panel's later columns (FP64 pipe).  The
//     panel's interchanges leave as a list of (destination, source) rows.
//   * The interchanges applied to the rest of Q and to P (one gather per panel); the
//     diagonal tile's unit-lower and upper triangles inverted column by column (FP64).
//   * U_kJ = L_kk^-1 A_kJ and the trailing update A_IJ -= L_Ik U_kJ as tile products.
//   * The solve: block forward substitution Y_J = L_JJ^-1 (P_J - sum_{I<J} L_JI Y_I) and
//     block back substitution X_J = U_JJ^-1 (Y_J - sum_{I>J} U_JI X_I), written
//     right-looking so that every update is again a batch of tile products.
//
// Products use the working precision of the caller's policy: emulated FP64 with k slices
// (k > 0) or the FP64 pipe (k = 0).  The diagonal blocks enter through their inverses (as in
// the blocked triangular solves of GPU libraries): with partial pivoting |l_ij| <= 1, and
// q(X) is well conditioned for ||X||_1 <= theta_13.
#include "common.cuh"

#include <cooperative_groups.h>

#include <mutex>

namespace cg = cooperative_groups;

namespace mpps {

namespace {

constexpr int TB = 64;                  // tile size
constexpr int PT = 256;                 // threads per panel CTA
constexpr int LDS = TB + 1;             // shared row pitch of the panel (doubles)
constexpr int MAXPAIRS = 2 * TB;        // rows one panel's interchanges can move
constexpr int PAIR_INTS = 1 + 2 * MAXPAIRS;
constexpr int SMEM_DYN_MAX = 216 * 1024;
constexpr int ROWS_SMEM_MAX = (SMEM_DYN_MAX - 2 * TB * 8) / (LDS * 8);

__host__ __device__ __forceinline__ size_t tile_off(int T, int I, int J) {
    return ((size_t)I * T + J) * TB * TB;
}
__host__ __device__ __forceinline__ size_t elem_off(int T, int r, int c) {
    return tile_off(T, r / TB, c / TB) + (size_t)(r % TB) * TB + (c % TB);
}

// dst (tile-major, N = T TB) from the row-major n x n src; the padding holds `diag` on the
// diagonal and zeros elsewhere.  Block (64, 4): 64 consecutive columns of 4 rows.
__global__ void k_lu_to_tiles(const double* __restrict__ src, int n, int T, double diag,
                              double* __restrict__ dst) {
    const int N = T * TB;
    const int c = blockIdx.x * 64 + threadIdx.x, r = blockIdx.y * 4 + threadIdx.y;
    if (r >= N || c >= N) return;
    const double v = (r < n && c < n) ? src[(size_t)r * n + c] : (r == c ? diag : 0.0);
    dst[elem_off(T, r, c)] = v;
}

// The leading n x n block of the tile-major src, row-major into dst.
__global__ void k_lu_from_tiles(const double* __restrict__ src, int n, int T,
                                double* __restrict__ dst) {
    const int c = blockIdx.x * 64 + threadIdx.x, r = blockIdx.y * 4 + threadIdx.y;
    if (r >= n || c >= n) return;
    dst[(size_t)r * n + c] = src[elem_off(T, r, c)];
}

// The interchanges of panel k applied to every tile column of Q except column k (which the
// panel kernel has already permuted) and to every tile column of P: new row dst_i = old row
// src_i for the listed pairs (a permutation of the rows they name).  One warp per half tile
// column (32 columns): each thread reads all source entries of its column, then writes.
__global__ void __launch_bounds__(32) k_lu_swap(double* __restrict__ Qt, double* __restrict__ Pt,
                                                int T, int k, const int* __restrict__ pairs) {
    __shared__ double vals[MAXPAIRS][32];
    const int tc = blockIdx.x >> 1;                  // 0 .. 2T-1: Q's tile columns, then P's
    const bool isq = tc < T;
    const int J = isq ? tc : tc - T;
    if (isq && J == k) return;
    double* M = isq ? Qt : Pt;
    const int col = J * TB + (blockIdx.x & 1) * 32 + threadIdx.x;
    const int cnt = min(__ldg(pairs), MAXPAIRS);
    for (int i = 0; i < cnt; ++i) vals[i][threadIdx.x] = M[elem_off(T, __ldg(pairs + 2 + 2 * i), col)];
    for (int i = 0; i < cnt; ++i) M[elem_off(T, __ldg(pairs + 1 + 2 * i), col)] = vals[i][threadIdx.x];
}

// Column `blockIdx.x` of the inverses of the diagonal tile's unit lower triangle
// (blockIdx.y = 0: L x = e_c by forward substitution, column-oriented) and of its upper
// triangle (blockIdx.y = 1: U x = e_c by back substitution), thread i holding x_i.  The
// tiles are written row-major into invL / invU at tile k.
__global__ void __launch_bounds__(TB) k_lu_tri_inv(const double* __restrict__ Qt, int T, int k,
                                                   double* __restrict__ invL,
                                                   double* __restrict__ invU) {
    const int col = blockIdx.x, i = threadIdx.x;
    const double* D = Qt + tile_off(T, k, k);
    __shared__ double x[TB];
    double xi = i == col ? 1.0 : 0.0;
    x[i] = xi;
    if (blockIdx.y == 0) {
        for (int j = col; j < TB - 1; ++j) {
            __syncthreads();
            const double xj = x[j];
            if (i > j) {
                xi = fma(-D[i * TB + j], xj, xi);
                x[i] = xi;
            }
        }
        invL[(size_t)k * TB * TB + (size_t)i * TB + col] = xi;
    } else {
        for (int j = col; j >= 0; --j) {
            __syncthreads();
            if (i == j) {
                xi = xi / D[j * TB + j];
                x[j] = xi;
            }
            __syncthreads();
            const double xj = x[j];
            if (i < j) xi = fma(-D[i * TB + j], xj, xi);
        }
        invU[(size_t)k * TB * TB + (size_t)i * TB + col] = xi;
    }
}

// ---- panel factorisation (one cluster) ---------------------------------------------------
struct PanelArgs {
    double* Qt;
    int T, k;
    int R;          // panel rows per CTA (CTA c: rows c R .. c R + R - 1, clipped)
    int in_smem;    // 1: rows held in shared memory; 0: worked on in place in the tiles
    int* pairs;     // out: count, then (destination, source) global row pairs
    int* info;      // first zero pivot (1-based global column), 0 if none
};

// The better of two pivot candidates: the larger magnitude, the smaller row on ties (the
// first maximum, as the usual partial pivoting search takes).  A NaN never wins; v = -1
// marks "no row".
__device__ __forceinline__ void cand_max(double& v, int& i, double ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}
__device__ __forceinline__ void cand_warp_max(double& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        cand_max(v, i, ov, oi);
    }
}

// Every thread of every CTA of the cluster runs the same sequence of barriers: no thread
// leaves early, whatever its rows.
__global__ void __launch_bounds__(PT) k_lu_panel(PanelArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank(), CL = (int)cl.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Mk = (a.T - a.k) * TB;                 // panel rows
    const int r0 = c * a.R;
    const int nr = max(0, min(a.R, Mk - r0));
    extern __shared__ __align__(16) double sm[];
    double* rows = sm;                                          // [R][LDS] (in_smem)
    double* urow = sm + (a.in_smem ? (size_t)a.R * LDS : 0);    // the pivot row
    double* tmp = urow + TB;                                    // the old row j (owner of p)
    __shared__ double cand_v;                                   // read by the other CTAs
    __shared__ int cand_i;
    __shared__ double red_v[PT / 32];
    __shared__ int red_i[PT / 32];
    __shared__ int s_p, s_sing, s_ns;
    __shared__ int sl_row[MAXPAIRS], sl_src[MAXPAIRS];          // CTA 0: the interchanges

    auto gptr = [&](int pr) -> double* {   // panel row pr in the tile storage
        return a.Qt + tile_off(a.T, a.k + pr / TB, a.k) + (size_t)(pr % TB) * TB;
    };
    auto own = [&](int lr) -> double* {
        return a.in_smem ? rows + (size_t)lr * LDS : gptr(r0 + lr);
    };
    // entry `col` of panel row pr, wherever its owner keeps it
    auto rload = [&](int pr, int col) -> double {
        const int o = pr / a.R;
        if (a.in_smem) return cl.map_shared_rank(rows, o)[(size_t)(pr - o * a.R) * LDS + col];
        return __ldcg(gptr(pr) + col);
    };

    if (a.in_smem)
        for (int e = tid; e < nr * TB; e += PT) rows[(size_t)(e / TB) * LDS + e % TB] = gptr(r0 + e / TB)[e % TB];
    if (c == 0) {
        for (int s = tid; s < MAXPAIRS; s += PT) {
            sl_row[s] = s;
            sl_src[s] = s;
        }
        if (tid == 0) s_ns = TB;
    }
    cl.sync();   // every CTA of the cluster runs and holds its rows

    for (int j = 0; j < TB; ++j) {
        // (1) this CTA's candidate for column j among its rows j, j+1, ...
        double bv = -1.0;
        int bi = 0x7fffffff;
        for (int lr = tid; lr < nr; lr += PT)
            if (r0 + lr >= j) cand_max(bv, bi, fabs(own(lr)[j]), r0 + lr);
        cand_warp_max(bv, bi);
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
            bv = lane < PT / 32 ? red_v[lane] : -1.0;
            bi = lane < PT / 32 ? red_i[lane] : 0x7fffffff;
            cand_warp_max(bv, bi);
            if (lane == 0) {
                cand_v = bv;
                cand_i = bi;
            }
        }
        cl.sync();   // (2) every CTA's candidate is written
        if (warp == 0) {
            double v = -1.0;
            int i = 0x7fffffff;
            if (lane < CL) {
                v = *cl.map_shared_rank(&cand_v, lane);
                i = *cl.map_shared_rank(&cand_i, lane);
            }
            cand_warp_max(v, i);
            if (lane == 0) {
                s_sing = !(v > 0.0);   // an exactly zero (or NaN) column: no interchange
                s_p = s_sing ? j : i;
            }
        }
        __syncthreads();
        const int p = s_p;
        const bool sing = s_sing != 0;
        if (c == 0 && warp == 0) {   // the interchange list, and the first zero pivot
            if (sing && lane == 0) atomicCAS(a.info, 0, a.k * TB + j + 1);
            if (p != j) {
                int sp = p;
                if (p >= TB) {   // row p's slot among the rows below the diagonal tile
                    sp = -1;
                    const int ns = s_ns;
                    for (int base = TB; base < ns && sp < 0; base += 32) {
                        const int s = base + lane;
                        const unsigned m = __ballot_sync(0xffffffffu, s < ns && sl_row[s] == p);
                        if (m) sp = base + __ffs(m) - 1;
                    }
                    if (sp < 0) {
                        sp = ns;
                        if (lane == 0) {
                            sl_row[sp] = p;
                            sl_src[sp] = p;
                            s_ns = ns + 1;
                        }
                    }
                    __syncwarp();
                }
                if (lane == 0) {
                    const int t = sl_src[j];
                    sl_src[j] = sl_src[sp];
                    sl_src[sp] = t;
                }
                __syncwarp();
            }
        }
        // (3) the pivot row, and (at the owner of row p) the old row j
        const int op = p / a.R;
        if (tid < TB) {
            urow[tid] = rload(p, tid);
            if (op == c && p != j) tmp[tid] = rload(j, tid);
        }
        cl.sync();   // (4) every read of the rows j and p is done
        if (tid < TB && p != j) {
            if (j / a.R == c) own(j - r0)[tid] = urow[tid];
            if (op == c) own(p - r0)[tid] = tmp[tid];
        }
        __syncthreads();
        if (!sing) {
            const double piv = urow[j];
            for (int lr = tid; lr < nr; lr += PT)
                if (r0 + lr > j) own(lr)[j] = own(lr)[j] / piv;
            __syncthreads();
            const int col = tid % TB;
            if (col > j)
                for (int lr = tid / TB; lr < nr; lr += PT / TB)
                    if (r0 + lr > j) {
                        double* rw = own(lr);
                        rw[col] = fma(-rw[j], urow[col], rw[col]);
                    }
        }
        __syncthreads();
    }

    if (a.in_smem)
        for (int e = tid; e < nr * TB; e += PT) gptr(r0 + e / TB)[e % TB] = rows[(size_t)(e / TB) * LDS + e % TB];
    if (c == 0 && tid == 0) {
        int cnt = 0;
        for (int s = 0; s < s_ns; ++s)
            if (sl_src[s] != sl_row[s]) {
                a.pairs[1 + 2 * cnt] = a.k * TB + sl_row[s];
                a.pairs[2 + 2 * cnt] = a.k * TB + sl_src[s];
                ++cnt;
            }
        a.pairs[0] = cnt;
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace

// ---- host -----------------------------------------------------------------------------
namespace {

struct LuLayout {
    int T, N;
    size_t off_Qt, off_Pt, off_invL, off_invU, off_pairs, off_slA, off_slB, off_eA, off_eB,
        off_cmx, bytes;
};

LuLayout lu_layout(int n, int k) {
    LuLayout L;
    L.T = (n + TB - 1) / TB;
    L.N = L.T * TB;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t NN = (size_t)L.N * L.N;
    L.off_Qt = take(NN * sizeof(double));
    L.off_Pt = take(NN * sizeof(double));
    L.off_invL = take((size_t)L.T * TB * TB * sizeof(double));
    L.off_invU = take((size_t)L.T * TB * TB * sizeof(double));
    L.off_pairs = take(PAIR_INTS * sizeof(int));
    const size_t planes = k > 0 ? f64e_plane_elems(TB, L.T, k) * sizeof(__nv_bfloat16) : 0;
    L.off_slA = take(planes);
    L.off_slB = take(planes);
    L.off_eA = take(k > 0 ? (size_t)L.T * TB * sizeof(int) : 0);
    L.off_eB = take(k > 0 ? (size_t)L.T * TB * sizeof(int) : 0);
    L.off_cmx = take(k > 0 ? (size_t)L.T * TB * sizeof(unsigned long long) : 0);
    L.bytes = (off + 255) & ~(size_t)255;
    return L;
}

// Largest cluster the panel kernel can be launched with on this device (16 where the
// hardware allows a non-portable size, else 8, 4, 2 or 1), at its largest shared memory.
int panel_cluster_max(int dev) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev]) return cache[dev];
    int best = 1;
    if (cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN_MAX) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
        for (int cl = 16; cl >= 2; cl >>= 1) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cl);
            cfg.blockDim = dim3(PT);
            cfg.dynamicSmemBytes = SMEM_DYN_MAX;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cl;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int ncl = 0;
            if (cudaOccupancyMaxActiveClusters(&ncl, k_lu_panel, &cfg) == cudaSuccess && ncl >= 1) {
                best = cl;
                break;
            }
            cudaGetLastError();
        }
    }
    cudaGetLastError();
    cache[dev] = best;
    return best;
}

struct LuRun {
    int T, k;
    double *Qt, *Pt, *invL, *invU;
    int* pairs;
    void *slA, *slB;
    int *eA, *eB;
    unsigned long long* cmx;
    int* d_err;
    cudaStream_t st;
    int cl_max;

    // out tile (I gci + J gcj) (-)= A_I B_J (or =) for I < nI, J < nJ, with
    // A_I = A + I a_bs and B_J = B + J b_bs (TB x TB row-major tiles)
    mpps_status products(const double* A, long long a_bs, int nI, const double* B, long long b_bs,
                         int nJ, double* out, int gci, int gcj, bool subtract) const {
        if (nI <= 0 || nJ <= 0) return MPPS_OK;
        const long long tt = (long long)TB * TB;
        Epilogue ep = epilogue_plain(out, tt);
        ep.gnj = nJ;
        ep.gci = gci;
        ep.gcj = gcj;
        if (subtract) {
            ep.alpha = -1.0;
            ep.add = out;
            ep.add_bstride = tt;
            ep.add_coef = 1.0;
        }
        if (k == 0) {   // FP64 pipe: at most 65535 products per launch
            const int per = nJ >= 65535 ? 1 : 65535 / nJ;
            for (int i0 = 0; i0 < nI; i0 += per) {
                const int cnt = nI - i0 < per ? nI - i0 : per;
                Epilogue e = ep;
                e.out = out + (size_t)i0 * gci * tt;
                if (subtract) e.add = e.out;
                mpps_status rc = launch_gemm_f64(A + (size_t)i0 * a_bs, a_bs, B, b_bs, TB, cnt * nJ, e, st);
                if (rc) return rc;
            }
            return MPPS_OK;
        }
        mpps_status rc = launch_slice_rows(A, a_bs, TB, nI, k, slA, eA, st);
        if (!rc) rc = launch_slice_cols(B, b_bs, TB, nJ, k, slB, eB, cmx, st);
        if (!rc) rc = launch_gemm_f64e_grid(k, slA, eA, nI, slB, eB, nJ, TB, ep, d_err, st);
        return rc;
    }

    mpps_status panel(int kk, int* info) const {
        const int Mk = (T - kk) * TB;
        int cl = 1;   // a power of two, about 32 rows or more per CTA
        while (cl * 2 <= cl_max && cl * 2 * 32 <= Mk) cl *= 2;
        const int R = (Mk + cl - 1) / cl;
        const bool in_smem = R <= ROWS_SMEM_MAX;
        PanelArgs a{Qt, T, kk, R, in_smem ? 1 : 0, pairs, info};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(PT);
        cfg.dynamicSmemBytes = (in_smem ? (size_t)R * LDS * 8 : 0) + 2 * TB * 8;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        MPPS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_lu_panel, a));
        MPPS_LAUNCH_CHECK();
        return MPPS_OK;
    }

    // Q = P^T L U in place (tile-major), with the interchanges applied to P as well
    mpps_status factor(int* info) const {
        const long long tt = (long long)TB * TB, trow = (long long)T * tt;
        for (int kk = 0; kk < T; ++kk) {
            mpps_status rc = panel(kk, info);
            if (rc) return rc;
            k_lu_swap<<<2 * T * 2, 32, 0, st>>>(Qt, Pt, T, kk, pairs);
            MPPS_LAUNCH_CHECK();
            k_lu_tri_inv<<<dim3(TB, 2), TB, 0, st>>>(Qt, T, kk, invL, invU);
            MPPS_LAUNCH_CHECK();
            const int nr = T - kk - 1;
            if (nr == 0) break;
            double* Ukj = Qt + tile_off(T, kk, kk + 1);
            // U_kJ = L_kk^-1 A_kJ (J > k), written over A_kJ
            if ((rc = products(invL + kk * tt, 0, 1, Ukj, tt, nr, Ukj, 0, 1, false))) return rc;
            // A_IJ -= L_Ik U_kJ (I, J > k)
            if ((rc = products(Qt + tile_off(T, kk + 1, kk), trow, nr, Ukj, tt, nr,
                               Qt + tile_off(T, kk + 1, kk + 1), T, 1, true)))
                return rc;
        }
        return MPPS_OK;
    }

    // P := U^-1 L^-1 P (P already permuted)
    mpps_status substitute() const {
        const long long tt = (long long)TB * TB, trow = (long long)T * tt;
        mpps_status rc;
        for (int J = 0; J < T; ++J) {   // Y_J = L_JJ^-1 P_J, then P_I -= L_IJ Y_J (I > J)
            double* PJ = Pt + tile_off(T, J, 0);
            if ((rc = products(invL + J * tt, 0, 1, PJ, tt, T, PJ, 0, 1, false))) return rc;
            if (J + 1 < T &&
                (rc = products(Qt + tile_off(T, J + 1, J), trow, T - J - 1, PJ, tt, T,
                               Pt + tile_off(T, J + 1, 0), T, 1, true)))
                return rc;
        }
        for (int J = T - 1; J >= 0; --J) {   // X_J = U_JJ^-1 Y_J, then Y_I -= U_IJ X_J (I < J)
            double* PJ = Pt + tile_off(T, J, 0);
            if ((rc = products(invU + J * tt, 0, 1, PJ, tt, T, PJ, 0, 1, false))) return rc;
            if (J > 0 && (rc = products(Qt + tile_off(T, 0, J), trow, J, PJ, tt, T, Pt, T, 1, true)))
                return rc;
        }
        return MPPS_OK;
    }
};

}  // namespace

size_t lu_workspace_bytes(int n, int k) { return lu_layout(n, k).bytes; }

mpps_status lu_solve_dev(const double* Q, const double* P, double* R, int n, int batch, int k,
                         void* ws, int* info, int* d_err, cudaStream_t st) {
    if (n <= 0 || batch <= 0) return MPPS_OK;
    if (k < 0 || k > MPPS_F64E_MAX_SLICES || (k > 0 && !d_err)) {
        set_error("lu_solve: slice count %d outside 0..%d", k, MPPS_F64E_MAX_SLICES);
        return MPPS_EINVAL;
    }
    const LuLayout L = lu_layout(n, k);
    if ((long long)L.N / 4 > 65535) {
        set_error("lu_solve: n = %d exceeds the tile conversion grid", n);
        return MPPS_EINVAL;
    }
    int dev = 0;
    MPPS_CUDA_TRY(cudaGetDevice(&dev));
    char* base = (char*)ws;
    LuRun run;
    run.T = L.T;
    run.k = k;
    run.Qt = (double*)(base + L.off_Qt);
    run.Pt = (double*)(base + L.off_Pt);
    run.invL = (double*)(base + L.off_invL);
    run.invU = (double*)(base + L.off_invU);
    run.pairs = (int*)(base + L.off_pairs);
    run.slA = k > 0 ? base + L.off_slA : nullptr;
    run.slB = k > 0 ? base + L.off_slB : nullptr;
    run.eA = k > 0 ? (int*)(base + L.off_eA) : nullptr;
    run.eB = k > 0 ? (int*)(base + L.off_eB) : nullptr;
    run.cmx = k > 0 ? (unsigned long long*)(base + L.off_cmx) : nullptr;
    run.d_err = d_err;
    run.st = st;
    run.cl_max = panel_cluster_max(dev);
    const dim3 cb(64, 4), cg_((L.N + 63) / 64, (L.N + 3) / 4), og((n + 63) / 64, (n + 3) / 4);
    const size_t nn = (size_t)n * n;
    MPPS_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, st));
    for (int b = 0; b < batch; ++b) {   // one system after the other, in one workspace
        k_lu_to_tiles<<<cg_, cb, 0, st>>>(Q + b * nn, n, L.T, 1.0, run.Qt);
        MPPS_LAUNCH_CHECK();
        k_lu_to_tiles<<<cg_, cb, 0, st>>>(P + b * nn, n, L.T, 0.0, run.Pt);
        MPPS_LAUNCH_CHECK();
        mpps_status rc = run.factor(info + b);
        if (!rc) rc = run.substitute();
        if (rc) return rc;
        k_lu_from_tiles<<<og, cb, 0, st>>>(run.Pt, n, L.T, R + b * nn);
        MPPS_LAUNCH_CHECK();
    }
    return MPPS_OK;
}

}  // namespace mpps
