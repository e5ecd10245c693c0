// lu.cu -- R = Q^-1 P by LU factorisation with partial pivoting: the q(X)^-1 p(X) solve of
// the [13/13] Pade approximant (Section 4.1, the diagonal Pade approximant r_m = q_m^-1 p_m).
//
// Blocked right-looking LU (Golub and Van Loan, Algorithm 3.4.2 with row interchanges) of the
// augmented matrix [Q | P], laid out for a GPU whose FP64 pipe gives about 1 TFLOP/s while
// the emulated FP64 product on the BF16 tensor cores gives tens of TFLOP/s:
//
//   * [Q | P] is copied into a tile-major layout: T x 2T tiles of TB x TB doubles, each tile
//     a contiguous row-major TB x TB matrix, n padded to N = T TB with Q = diag(Q, I) and
//     P = diag(P, 0) (the padded unknowns are zero).  Every block operation below is then a
//     batch of TB x TB products, run by the existing products in grid mode (product z takes
//     A tile z / nJ and B tile z % nJ).
//   * Panel k (tile column k, rows k TB .. N): one thread-block cluster.  CTA c holds rows
//     [c R, (c + 1) R) of the panel in its shared memory (in place in the tiles when the
//     panel is too tall); per column: local pivot candidates published with copies of their
//     rows, one cluster barrier, the pivot row read from the winner's shared memory, the
//     multipliers and the rank-1 update of the panel's later columns with the interchange
//     folded in (FP64 pipe).  The panel's interchanges leave as a list of (destination,
//     source) rows.
//   * The interchanges applied to the rest of [Q | P] (one gather per panel); the diagonal
//     tile's unit-lower and upper triangles inverted column by column (FP64).
//   * U_kJ = L_kk^-1 A_kJ and the trailing update A_IJ -= L_Ik U_kJ as tile products, over
//     the columns of Q and of P: on P's columns they are the block forward substitution
//     L Y = P, so that P's tiles hold Y when the factorisation ends.
//   * The block back substitution X_J = U_JJ^-1 (Y_J - sum_{I>J} U_JI X_I), written
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
// panel rows a CTA keeps in shared memory: LDS doubles each plus one multiplier
constexpr int ROWS_SMEM_MAX = (SMEM_DYN_MAX / 8 - 2 * TB) / (LDS + 1);

// tile (I, J) of a tile-major array W tiles wide
__host__ __device__ __forceinline__ size_t tile_off(int W, int I, int J) {
    return ((size_t)I * W + J) * TB * TB;
}
__host__ __device__ __forceinline__ size_t elem_off(int W, int r, int c) {
    return tile_off(W, r / TB, c / TB) + (size_t)(r % TB) * TB + (c % TB);
}

// Columns c0 .. c0 + N - 1 of the tile-major array (W tiles wide, N = T TB) from the
// row-major n x n src; the padding holds `diag` on the diagonal and zeros elsewhere.  Block
// (64, 4): 64 consecutive columns of 4 rows.
__global__ void k_lu_to_tiles(const double* __restrict__ src, int n, int T, int W, int c0,
                              double diag, double* __restrict__ dst) {
    const int N = T * TB;
    const int c = blockIdx.x * 64 + threadIdx.x, r = blockIdx.y * 4 + threadIdx.y;
    if (r >= N || c >= N) return;
    const double v = (r < n && c < n) ? src[(size_t)r * n + c] : (r == c ? diag : 0.0);
    dst[elem_off(W, r, c0 + c)] = v;
}

// The leading n x n block of columns c0 .. of the tile-major src, row-major into dst.
__global__ void k_lu_from_tiles(const double* __restrict__ src, int n, int W, int c0,
                                double* __restrict__ dst) {
    const int c = blockIdx.x * 64 + threadIdx.x, r = blockIdx.y * 4 + threadIdx.y;
    if (r >= n || c >= n) return;
    dst[(size_t)r * n + c] = src[elem_off(W, r, c0 + c)];
}

// The interchanges of panel k applied to every tile column of [Q | P] except column k
// (which the panel kernel has already permuted): new row dst_i = old row src_i for the
// listed pairs (a permutation of the rows they name).  A block takes 32 columns: its 8 warps
// read every source entry of them into shared memory (four loads in flight per thread),
// then write the destinations.
__global__ void __launch_bounds__(256) k_lu_swap(double* __restrict__ M, int W, int k,
                                                 const int* __restrict__ pairs) {
    __shared__ double vals[MAXPAIRS][33];
    const int J = blockIdx.x >> 1;
    if (J == k) return;                              // the whole block
    const int cx = threadIdx.x & 31, sy = threadIdx.x >> 5;
    const int col = J * TB + (blockIdx.x & 1) * 32 + cx;
    const int cnt = min(__ldg(pairs), MAXPAIRS);
    for (int i0 = sy; i0 < cnt; i0 += 32) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + 8 * u;
            v[u] = i < cnt ? M[elem_off(W, __ldg(pairs + 2 + 2 * i), col)] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + 8 * u < cnt) vals[i0 + 8 * u][cx] = v[u];
    }
    __syncthreads();
    for (int i = sy; i < cnt; i += 8) M[elem_off(W, __ldg(pairs + 1 + 2 * i), col)] = vals[i][cx];
}

// Column `blockIdx.x` of the inverses of the diagonal tile's unit lower triangle
// (blockIdx.y = 0: L x = e_c by forward substitution, column-oriented) and of its upper
// triangle (blockIdx.y = 1: U x = e_c by back substitution), thread i holding x_i; the tile
// is staged in shared memory first.  The tiles are written row-major into invL / invU at
// tile k.
__global__ void __launch_bounds__(TB) k_lu_tri_inv(const double* __restrict__ M, int W, int k,
                                                   double* __restrict__ invL,
                                                   double* __restrict__ invU) {
    const int col = blockIdx.x, i = threadIdx.x;
    __shared__ double D[TB][TB + 1];
    __shared__ double x[TB];
    const double* src = M + tile_off(W, k, k);
    for (int e = i; e < TB * TB; e += TB) D[e / TB][e % TB] = src[e];
    double xi = i == col ? 1.0 : 0.0;
    x[i] = xi;
    if (blockIdx.y == 0) {
        for (int j = col; j < TB - 1; ++j) {
            __syncthreads();
            const double xj = x[j];
            if (i > j) {
                xi = fma(-D[i][j], xj, xi);
                x[i] = xi;
            }
        }
        invL[(size_t)k * TB * TB + (size_t)i * TB + col] = xi;
    } else {
        for (int j = col; j >= 0; --j) {
            __syncthreads();
            if (i == j) {
                xi = xi / D[j][j];
                x[j] = xi;
            }
            __syncthreads();
            const double xj = x[j];
            if (i < j) xi = fma(-D[i][j], xj, xi);
        }
        invU[(size_t)k * TB * TB + (size_t)i * TB + col] = xi;
    }
}

// ---- panel factorisation (one cluster) ---------------------------------------------------
struct PanelArgs {
    double* M;
    int T, W, k;
    int R;          // panel rows per CTA (CTA c: rows c R .. c R + R - 1, clipped)
    int in_smem;    // 1: rows held in shared memory; 0: worked on in place in the tiles
    int* pairs;     // out: count, then (destination, source) global row pairs
    int* info;      // first zero pivot (1-based global column), 0 if none
};

// Pivot candidates compare on the integer pipe: |x| as the bit pattern of a non-negative
// double orders like |x| (a NaN maps to 0 and never wins).  The better of two candidates
// has the larger magnitude, the smaller row on ties (the first maximum, as the usual partial
// pivoting search takes); (0, INT_MAX) is "no row".
__device__ __forceinline__ unsigned long long piv_key(double x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    return a > 0x7ff0000000000000ULL ? 0ULL : a;
}
__device__ __forceinline__ void cand_max(unsigned long long& v, int& i, unsigned long long ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}

// Every thread of every CTA of the cluster runs the same sequence of barriers: no thread
// leaves early, whatever its rows.  Per column j, one cluster barrier: before it, each CTA
// publishes its candidate (magnitude, row) and a copy of that row, and the owner of row j a
// copy of row j, in the slot of the column's parity; after it, every warp finds the winner
// and the CTA reads the copies it needs from the other CTAs' shared memory.  A CTA writes
// only its own rows, and a slot is written again two columns later, after the next barrier,
// when every read of it is done.  The multipliers use the reciprocal of the pivot (as the
// unblocked LAPACK factorisation does), and the interchange is folded into the update: row
// p is rebuilt from the copy of the old row j.
template <bool SMEM>
__global__ void __launch_bounds__(PT) k_lu_panel(PanelArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank(), CL = (int)cl.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Mk = (a.T - a.k) * TB;                 // panel rows
    const int r0 = c * a.R;
    const int nr = max(0, min(a.R, Mk - r0));
    extern __shared__ __align__(16) double sm[];
    double* rows = sm;                                          // [R][LDS] (SMEM)
    double* urow = sm + (SMEM ? (size_t)a.R * LDS : 0);         // the pivot row
    double* tmp = urow + TB;                                    // the old row j (owner of p)
    double* lmul = tmp + TB;                                    // this column's multipliers
    __shared__ double pub_cand[2][TB];                          // published: candidate row
    __shared__ double pub_rowj[2][TB];                          // published: row j (its owner)
    __shared__ unsigned long long cand_v[2];
    __shared__ int cand_i[2];
    __shared__ double s_pinv;
    __shared__ unsigned long long red_v[PT / 32];
    __shared__ int red_i[PT / 32];
    __shared__ int s_ns, s_p, s_w;
    __shared__ int sl_row[MAXPAIRS], sl_src[MAXPAIRS];          // CTA 0: the interchanges

    auto gptr = [&](int pr) -> double* {   // panel row pr in the tile storage
        return a.M + tile_off(a.W, a.k + pr / TB, a.k) + (size_t)(pr % TB) * TB;
    };
    auto own = [&](int lr) -> double* {
        if constexpr (SMEM) return rows + (size_t)lr * LDS;
        else return gptr(r0 + lr);
    };

    if (SMEM)
        for (int e = tid; e < nr * TB; e += PT) rows[(size_t)(e / TB) * LDS + e % TB] = gptr(r0 + e / TB)[e % TB];
    if (c == 0) {
        for (int s = tid; s < MAXPAIRS; s += PT) {
            sl_row[s] = s;
            sl_src[s] = s;
        }
        if (tid == 0) s_ns = TB;
    }
    __syncthreads();

    for (int j = 0; j < TB; ++j) {
        const int slot = j & 1;
        const bool own_j = j >= r0 && j < r0 + nr;
        if (own_j && tid < TB) pub_rowj[slot][tid] = own(j - r0)[tid];
        // (1) this CTA's candidate for column j among its rows j, j+1, ...
        unsigned long long bv = 0;
        int bi = 0x7fffffff;
        for (int lr = tid; lr < nr; lr += PT)
            if (r0 + lr >= j) cand_max(bv, bi, piv_key(own(lr)[j]), r0 + lr);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            cand_max(bv, bi, __shfl_xor_sync(0xffffffffu, bv, o), __shfl_xor_sync(0xffffffffu, bi, o));
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        bv = red_v[0];
        bi = red_i[0];
#pragma unroll
        for (int w = 1; w < PT / 32; ++w) cand_max(bv, bi, red_v[w], red_i[w]);
        if (tid == 0) {
            cand_v[slot] = bv;
            cand_i[slot] = bi;
        }
        if (tid < TB && bi != 0x7fffffff) pub_cand[slot][tid] = own(bi - r0)[tid];
        cl.sync();   // (2) every CTA's candidate and copies are published
        // (3) the winner, found by warp 0 (one remote read per CTA) and broadcast
        if (warp == 0) {
            unsigned long long v = 0;
            int i = 0x7fffffff, w = lane;
            if (lane < CL) {
                v = cl.map_shared_rank(cand_v, lane)[slot];
                i = cl.map_shared_rank(cand_i, lane)[slot];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int oi = __shfl_xor_sync(0xffffffffu, i, o);
                const int ow = __shfl_xor_sync(0xffffffffu, w, o);
                if (ov > v || (ov == v && oi < i)) {
                    v = ov;
                    i = oi;
                    w = ow;
                }
            }
            if (lane == 0) {
                const bool zero = v == 0;   // an exactly zero (or NaN) column
                s_p = zero ? -1 : i;
                s_w = w;
            }
        }
        __syncthreads();
        const bool sing = s_p < 0;
        const int p = sing ? j : s_p, w = s_w;
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
        if (!sing) {
            const bool swap_p = p != j && p >= r0 && p < r0 + nr;   // this CTA rebuilds row p
            if (tid < TB) {
                const double x = cl.map_shared_rank(&pub_cand[0][0], w)[slot * TB + tid];
                urow[tid] = x;
                if (tid == j) s_pinv = 1.0 / x;   // once, on the FP64 pipe
                if (swap_p) tmp[tid] = cl.map_shared_rank(&pub_rowj[0][0], j / a.R)[slot * TB + tid];
            }
            __syncthreads();
            // (4) the multipliers (row p's from the old row j) and the new row j
            const double pinv = s_pinv;
            for (int lr = tid; lr < nr; lr += PT) {
                const int pr = r0 + lr;
                if (pr > j) lmul[lr] = (pr == p && swap_p ? tmp[j] : own(lr)[j]) * pinv;
            }
            if (own_j && p != j && tid < TB) own(j - r0)[tid] = urow[tid];
            __syncthreads();
            // (5) the rank-1 update of the later columns; row p takes the old row j's entries
            const int col = tid % TB;
            const double u = urow[col];
            if (col > j) {
#pragma unroll 4
                for (int lr = tid / TB; lr < nr; lr += PT / TB) {
                    if (r0 + lr <= j) continue;
                    double* rw = own(lr) + col;
                    *rw = fma(-lmul[lr], u, (swap_p && r0 + lr == p) ? tmp[col] : *rw);
                }
            } else if (col == j) {
                for (int lr = tid / TB; lr < nr; lr += PT / TB)
                    if (r0 + lr > j) own(lr)[j] = lmul[lr];
            } else if (swap_p && (p - r0) % (PT / TB) == tid / TB) {
                own(p - r0)[col] = tmp[col];
            }
        }
        __syncthreads();
    }

    if (SMEM)
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
    int T, N, W;
    size_t off_M, off_invL, off_invU, off_pairs, off_slA, off_slB, off_eA, off_eB, bytes;
};

LuLayout lu_layout(int n, int k) {
    LuLayout L;
    L.T = (n + TB - 1) / TB;
    L.N = L.T * TB;
    L.W = 2 * L.T;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        const size_t at = off;
        off += bytes;
        return at;
    };
    L.off_M = take((size_t)L.T * L.W * TB * TB * sizeof(double));
    L.off_invL = take((size_t)L.T * TB * TB * sizeof(double));
    L.off_invU = take((size_t)L.T * TB * TB * sizeof(double));
    L.off_pairs = take(PAIR_INTS * sizeof(int));
    // A operands: at most T tiles; B operands: at most W tiles (a tile row of [Q | P])
    L.off_slA = take(k > 0 ? f64e_plane_elems(TB, L.T, k) * sizeof(__nv_bfloat16) : 0);
    L.off_slB = take(k > 0 ? f64e_plane_elems(TB, L.W, k) * sizeof(__nv_bfloat16) : 0);
    L.off_eA = take(k > 0 ? (size_t)L.T * TB * sizeof(int) : 0);
    L.off_eB = take(k > 0 ? (size_t)L.W * TB * sizeof(int) : 0);
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
    if (cudaFuncSetAttribute(k_lu_panel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN_MAX) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_lu_panel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_lu_panel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN_MAX) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_lu_panel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
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
            if (cudaOccupancyMaxActiveClusters(&ncl, k_lu_panel<true>, &cfg) == cudaSuccess && ncl >= 1) {
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
    int T, W, k;
    double *M, *invL, *invU;
    int* pairs;
    void *slA, *slB;
    int *eA, *eB;
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
        mpps_status rc = launch_slice_tiles(k, A, a_bs, nI, B, b_bs, nJ, TB, slA, eA, slB, eB, st);
        if (!rc) rc = launch_gemm_f64e_grid(k, slA, eA, nI, slB, eB, nJ, TB, ep, d_err, st);
        return rc;
    }

    mpps_status panel(int kk, int* info) const {
        const int Mk = (T - kk) * TB;
        int cl = 1;   // a power of two, about 32 rows or more per CTA
        while (cl * 2 <= cl_max && cl * 2 * 32 <= Mk) cl *= 2;
        const int R = (Mk + cl - 1) / cl;
        const bool in_smem = R <= ROWS_SMEM_MAX;
        PanelArgs a{M, T, W, kk, R, in_smem ? 1 : 0, pairs, info};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(PT);
        cfg.dynamicSmemBytes = ((in_smem ? (size_t)R * LDS : 0) + 2 * TB + (size_t)R) * sizeof(double);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (in_smem) MPPS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_lu_panel<true>, a));
        else MPPS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_lu_panel<false>, a));
        MPPS_LAUNCH_CHECK();
        return MPPS_OK;
    }

    // Q = P^T L U in place, and P's tiles := L^-1 (interchanged P)
    mpps_status factor(int* info) const {
        const long long tt = (long long)TB * TB, trow = (long long)W * tt;
        for (int kk = 0; kk < T; ++kk) {
            mpps_status rc = panel(kk, info);
            if (rc) return rc;
            k_lu_swap<<<2 * W, 256, 0, st>>>(M, W, kk, pairs);
            MPPS_LAUNCH_CHECK();
            k_lu_tri_inv<<<dim3(TB, 2), TB, 0, st>>>(M, W, kk, invL, invU);
            MPPS_LAUNCH_CHECK();
            const int nr = T - kk - 1, nc = W - kk - 1;
            double* Ukj = M + tile_off(W, kk, kk + 1);
            // U_kJ = L_kk^-1 A_kJ (J > k, Q's columns and P's), written over A_kJ
            if ((rc = products(invL + kk * tt, 0, 1, Ukj, tt, nc, Ukj, 0, 1, false))) return rc;
            // A_IJ -= L_Ik U_kJ (I, J > k)
            if ((rc = products(M + tile_off(W, kk + 1, kk), trow, nr, Ukj, tt, nc,
                               M + tile_off(W, kk + 1, kk + 1), W, 1, true)))
                return rc;
        }
        return MPPS_OK;
    }

    // P's tiles := U^-1 P's tiles
    mpps_status back_substitute() const {
        const long long tt = (long long)TB * TB, trow = (long long)W * tt;
        mpps_status rc;
        for (int J = T - 1; J >= 0; --J) {   // X_J = U_JJ^-1 Y_J, then Y_I -= U_IJ X_J (I < J)
            double* YJ = M + tile_off(W, J, T);
            if ((rc = products(invU + J * tt, 0, 1, YJ, tt, T, YJ, 0, 1, false))) return rc;
            if (J > 0 && (rc = products(M + tile_off(W, 0, J), trow, J, YJ, tt, T,
                                        M + tile_off(W, 0, T), W, 1, true)))
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
    run.W = L.W;
    run.k = k;
    run.M = (double*)(base + L.off_M);
    run.invL = (double*)(base + L.off_invL);
    run.invU = (double*)(base + L.off_invU);
    run.pairs = (int*)(base + L.off_pairs);
    run.slA = k > 0 ? base + L.off_slA : nullptr;
    run.slB = k > 0 ? base + L.off_slB : nullptr;
    run.eA = k > 0 ? (int*)(base + L.off_eA) : nullptr;
    run.eB = k > 0 ? (int*)(base + L.off_eB) : nullptr;
    run.d_err = d_err;
    run.st = st;
    run.cl_max = panel_cluster_max(dev);
    const dim3 cb(64, 4), tg((L.N + 63) / 64, (L.N + 3) / 4), og((n + 63) / 64, (n + 3) / 4);
    const size_t nn = (size_t)n * n;
    MPPS_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, st));
    for (int b = 0; b < batch; ++b) {   // one system after the other, in one workspace
        k_lu_to_tiles<<<tg, cb, 0, st>>>(Q + b * nn, n, L.T, L.W, 0, 1.0, run.M);
        MPPS_LAUNCH_CHECK();
        k_lu_to_tiles<<<tg, cb, 0, st>>>(P + b * nn, n, L.T, L.W, L.N, 0.0, run.M);
        MPPS_LAUNCH_CHECK();
        mpps_status rc = run.factor(info + b);
        if (!rc) rc = run.back_substitute();
        if (rc) return rc;
        k_lu_from_tiles<<<og, cb, 0, st>>>(run.M, n, L.W, L.N, R + b * nn);
        MPPS_LAUNCH_CHECK();
    }
    return MPPS_OK;
}

}  // namespace mpps
