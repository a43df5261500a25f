// Block SVD split of the two-site tensor with truncation, FP64 on the GPU (Section IV:
// the tensor is "wrapped" into a matrix with rows (a, s1) and columns (s2, b), one dense
// block per charge Q; Fig. 1e: the factors are split and the singular values absorbed in
// the sweep direction; Section II-C: singular values below a cutoff are removed).
//
// Each charge block M_Q (rows (s1, i, a), columns (s2, j, b)) is decomposed by one-sided
// Jacobi rotations (Hestenes): the columns of J = M_Q (or M_Q^T when M_Q is wide) are made
// mutually orthogonal by plane rotations applied in a round-robin order, so every round
// rotates k/2 disjoint column pairs in parallel (one thread block per pair, all sectors in
// one launch); V accumulates the rotations.  On convergence the column norms are the singular
// values.  The truncation rule runs on the host on the singular values; the kept singular
// triplets are then written into the caller's left (a, s1, c) and right (c, s2, b) tensors.
//
// Precision: the GB300's FP64 rate is low, and a full FP64 Jacobi run needs ~18 sweeps of
// ~12 r k^2 flops.  The sweeps therefore start on an FP32 copy (J32, V32) until the
// columns are orthogonal to FP32 accuracy (block sweeps: pairs of 16-column blocks, each
// rotated by one Jacobi sweep on its 32 x 32 Gram matrix, see svd_block_sweep_kernel); V32 is made orthonormal in FP64 by two
// Newton-Schulz steps (V <- V (3 I - V^T V) / 2, each squaring the orthogonality error),
// J <- J V in FP64, and FP64 Jacobi sweeps, accumulating into V, finish the
// decomposition (quadratic convergence from the preconditioned start: 2-3 sweeps).  The
// result is the FP64 one-sided Jacobi SVD of J; the FP32 phase only supplies the start.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <tuple>
#include <type_traits>

#include "internal.h"

using heff::fail;

namespace {

struct SvdSector {           // device-side description of one charge block
    int64_t j_off, v_off;    // column-major J (r x k) and V (k x k) in the workspace
    int64_t g_off, w_off;    // FP64 scratch: G (k x k), W (r x k)
    int64_t j32_off, v32_off;    // FP32 copies (offsets in floats from the FP32 region)
    int32_t r, k;            // rows, columns of J (k <= r)
    int32_t transposed;      // 1 when J = M_Q^T
    int32_t s_off;           // first singular value of this sector in the s array
};

struct WriteEntry {          // one output block element range: dst block <- kept vectors
    int64_t dst_off;         // output block offset
    int32_t rows, cols;      // output block shape
    int32_t sec;             // sector
    int32_t vec_row0;        // first row inside the left (or right) singular vectors
    int32_t kept_off;        // offset into the kept-index list of this sector
    int32_t left;            // 1: left tensor A[(a), c] ; 0: right tensor B[c, (b)]
};

}  // namespace

struct heff_svd {
    int nq = 1;
    std::vector<std::vector<int32_t>> Q;       // sector charges
    std::vector<SvdSector> sec;
    // per sector: row groups (i, s1) with row offsets, column groups (s2, j)
    std::vector<std::vector<std::tuple<int, int, int32_t>>> rows, cols;    // (sector idx, phys, offset)
    std::vector<std::vector<int64_t>> xoff;    // per sector: x block offsets [row group][col group]
    std::vector<int32_t> mrows, ncols;         // M_Q shape
    int64_t ws_doubles = 0;
    size_t off_slots = 0;                      // byte offset of the per-pair convergence slots
    int64_t nslots = 0, slot_ld = 0;
    size_t ws_bytes = 0;
    int64_t s_total = 0;
    std::vector<double> s;                     // singular values (per sector, unsorted)
    std::vector<std::vector<int32_t>> kept;    // per sector: kept column indices of J, s descending
    double norm = 0, discarded = 0;
    SvdSector* d_sec = nullptr;
    size_t off_f32 = 0;                        // byte offset of the FP32 region
    heff::BList gram, vg, jv;                  // G = V^T V, W = V G, W = J V (all sectors)
    bool lists_uploaded = false;
    int fp32_sweeps = 0, fp64_sweeps = 0;
    std::vector<int> pair_off;                 // prefix sums of the sectors' pair counts
    int max_k = 0;
    bool computed = false;
    int alpha_nsec = 0, beta_nsec = 0;
    std::vector<int32_t> alpha_dims, beta_dims;
};

namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// scatter x blocks into column-major J (or J^T layout for wide sectors)
__global__ void svd_load_kernel(const SvdSector* __restrict__ secs, const int64_t* __restrict__ tab, int ntab,
                                const double* __restrict__ x, double* __restrict__ ws) {
    // tab: per x block: [sector, x_off, m_rows, n_cols, row0 in M, col0 in M]
    for (int b = blockIdx.x; b < ntab; b += gridDim.x) {
        const int64_t* t = tab + 6 * b;
        const SvdSector s = secs[t[0]];
        const int64_t xo = t[1];
        const int mr = (int)t[2], nc = (int)t[3], r0 = (int)t[4], c0 = (int)t[5];
        double* J = ws + s.j_off;
        for (int e = threadIdx.x; e < mr * nc; e += blockDim.x) {
            const int a = e / nc, c = e % nc;
            const int R = r0 + a, Cc = c0 + c;         // position in M_Q
            const double v = x[xo + e];
            if (!s.transposed) J[(int64_t)Cc * s.r + R] = v;     // J = M: column Cc, row R
            else J[(int64_t)R * s.r + Cc] = v;                    // J = M^T: column R, row Cc
        }
    }
}


// J32 = float(J), V32 = I
__global__ void svd_to_f32_kernel(const SvdSector* __restrict__ secs, const double* __restrict__ ws,
                                  float* __restrict__ f32) {
    const SvdSector s = secs[blockIdx.y];
    const int64_t nj = (int64_t)s.r * s.k, nv = (int64_t)s.k * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nj + nv; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nj) f32[s.j32_off + e] = (float)ws[s.j_off + e];
        else {
            const int64_t v = e - nj;
            f32[s.v32_off + v] = (v % (s.k + 1) == 0) ? 1.f : 0.f;
        }
    }
}

// V = double(V32)
__global__ void svd_v_to_f64_kernel(const SvdSector* __restrict__ secs, const float* __restrict__ f32,
                                    double* __restrict__ ws) {
    const SvdSector s = secs[blockIdx.y];
    const int64_t nv = (int64_t)s.k * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (int64_t)gridDim.x * blockDim.x)
        ws[s.v_off + e] = (double)f32[s.v32_off + e];
}

// Newton-Schulz combine: V = 1.5 V + W, with W = -0.5 V G already formed
__global__ void svd_ns_kernel(const SvdSector* __restrict__ secs, double* __restrict__ ws) {
    const SvdSector s = secs[blockIdx.y];
    const int64_t nv = (int64_t)s.k * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (int64_t)gridDim.x * blockDim.x)
        ws[s.v_off + e] = 1.5 * ws[s.v_off + e] + ws[s.w_off + e];
}

// J = W (the product J V)
__global__ void svd_copy_w_kernel(const SvdSector* __restrict__ secs, double* __restrict__ ws) {
    const SvdSector s = secs[blockIdx.y];
    const int64_t nj = (int64_t)s.r * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nj; e += (int64_t)gridDim.x * blockDim.x)
        ws[s.j_off + e] = ws[s.w_off + e];
}

// One sweep (all rounds) as one cooperative launch: the warps of the grid take the
// (sector, pair) items of a round from a flattened list (pair_off: prefix sums of each
// sector's pair count), rotate, and meet at a grid barrier before the next round.  The
// barrier is a counter and a generation word in global memory; its wait is bounded (about a
// second), after which the kernel sets err and returns.  Each block writes the largest
// off-diagonal measure it saw to block_max[blockIdx.x].
//
// Column norms are carried instead of recomputed per pair (as in the standard one-sided
// Jacobi codes): the sweep starts by computing every column's squared norm into nrm
// (indexed like the singular values, s_off + column), and a rotation by tan(theta) = t of
// columns with squared norms a, b and inner product g leaves exactly a - t g and b + t g
// (the rotation zeroes the inner product).  A pair then needs one dot product instead of
// three.  The updates change a norm by t g, tiny once the columns are nearly orthogonal, and
// the norms are recomputed at the start of every sweep, so the rounding drift stays at a
// few ulps of the column's norm.
constexpr int SVD_SWEEP_NT = 256;
#ifndef SVD_UNROLL
#define SVD_UNROLL 8        // column pieces per lane loaded together in a pair's loops
#endif
constexpr long long SVD_BARRIER_CYCLES = 2ll << 30;

__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen, unsigned int nblocks,
                                             int* err) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int* vgen = gen;
        const unsigned int g = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (*(volatile int*)err || clock64() - t0 > SVD_BARRIER_CYCLES) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(SVD_SWEEP_NT) svd_sweep_kernel(const SvdSector* __restrict__ secs, int nsec,
                                                                 const int* __restrict__ pair_off, int kk_all,
                                                                 T* __restrict__ base, T* __restrict__ nrm,
                                                                 int ncols_all, float* __restrict__ block_max,
                                                                 unsigned int* __restrict__ bar, int* __restrict__ err) {
    constexpr bool F32 = sizeof(T) == 4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int warps = SVD_SWEEP_NT / 32;
    const int gw = blockIdx.x * warps + w, nw = gridDim.x * warps;
    const int npairs = pair_off[nsec];
    float mymax = 0.f;
    constexpr int UJ = SVD_UNROLL;
    // squared column norms (one warp per column; the sectors' s_off are prefix sums of k)
    bool go = true;
    if (ncols_all > 0) {
        for (int item = gw; item < ncols_all; item += nw) {
            int lo = 0, hi = nsec;                       // sector: s_off[lo] <= item < s_off[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (secs[mid].s_off <= item) lo = mid; else hi = mid;
            }
            const SvdSector s = secs[lo];
            const T* c = base + (F32 ? s.j32_off : s.j_off) + (int64_t)(item - s.s_off) * s.r;
            T a = 0;
            for (int i0 = lane; i0 < s.r; i0 += 32 * UJ) {
                T u[UJ];
#pragma unroll
                for (int t = 0; t < UJ; ++t) u[t] = i0 + 32 * t < s.r ? c[i0 + 32 * t] : (T)0;
#pragma unroll
                for (int t = 0; t < UJ; ++t) a = fma(u[t], u[t], a);
            }
            a = warp_sum_t(a);
            if (lane == 0) nrm[item] = a;
        }
        go = grid_barrier(bar, bar + 1, gridDim.x, err);
    }
    for (int round = 0; go && round < kk_all - 1; ++round) {
        for (int item = gw; item < npairs; item += nw) {
            int lo = 0, hi = nsec;                       // sector: pair_off[lo] <= item < pair_off[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pair_off[mid] <= item) lo = mid; else hi = mid;
            }
            const SvdSector s = secs[lo];
            const int kk = s.k + (s.k & 1);
            if (round >= kk - 1) continue;
            const int pair = item - pair_off[lo];
            auto pos = [&](int j) { return j == 0 ? 0 : 1 + (j - 1 + round) % (kk - 1); };
            int p = pos(pair), q = pos(kk - 1 - pair);
            if (p >= s.k || q >= s.k) continue;          // pair with the dummy column
            if (p > q) { const int t = p; p = q; q = t; }
            T* J = base + (F32 ? s.j32_off : s.j_off);
            T* cp = J + (int64_t)p * s.r;
            T* cq = J + (int64_t)q * s.r;
            // (the column pieces of UJ iterations are loaded together: the pair's loops are
            // bound by L2 latency; each lane's sums keep their order)
            T* np = nrm + s.s_off + p;
            T* nq = nrm + s.s_off + q;
            const T a = *np, b = *nq;
            T g = 0;
            for (int i0 = lane; i0 < s.r; i0 += 32 * UJ) {
                T u[UJ], v[UJ];
#pragma unroll
                for (int t = 0; t < UJ; ++t) {
                    const int i = i0 + 32 * t;
                    u[t] = i < s.r ? cp[i] : (T)0;
                    v[t] = i < s.r ? cq[i] : (T)0;
                }
#pragma unroll
                for (int t = 0; t < UJ; ++t) g = fma(u[t], v[t], g);
            }
            g = warp_sum_t(g);
            if (g == (T)0 || a == (T)0 || b == (T)0) continue;
            const double da = a, db = b, dg = g;
            const double meas = fabs(dg) / sqrt(da * db);
            mymax = fmaxf(mymax, (float)meas);
            if (meas < (F32 ? 1e-7 : 1e-15)) continue;
            const double zeta = (db - da) / (2.0 * dg);
            const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cd = 1.0 / sqrt(1.0 + t * t);
            const T c = (T)cd, sn = (T)(cd * t);
            if (lane == 0) {                             // the rotated columns' squared norms
                *np = (T)(da - t * dg);
                *nq = (T)(db + t * dg);
            }
            // rotate the two columns of J and of V in one loop (both only need c, sn)
            T* V = base + (F32 ? s.v32_off : s.v_off);
            T* vp = V + (int64_t)p * s.k;
            T* vq = V + (int64_t)q * s.k;
            constexpr int UR = SVD_UNROLL / 2;
            for (int i0 = lane; i0 < s.r; i0 += 32 * UR) {       // s.k <= s.r
                T u[UR], v[UR], x[UR], y[UR];
#pragma unroll
                for (int t = 0; t < UR; ++t) {
                    const int i = i0 + 32 * t;
                    u[t] = i < s.r ? cp[i] : (T)0;
                    v[t] = i < s.r ? cq[i] : (T)0;
                    x[t] = i < s.k ? vp[i] : (T)0;
                    y[t] = i < s.k ? vq[i] : (T)0;
                }
#pragma unroll
                for (int t = 0; t < UR; ++t) {
                    const int i = i0 + 32 * t;
                    if (i < s.r) {
                        cp[i] = c * u[t] - sn * v[t];
                        cq[i] = sn * u[t] + c * v[t];
                    }
                    if (i < s.k) {
                        vp[i] = c * x[t] - sn * y[t];
                        vq[i] = sn * x[t] + c * y[t];
                    }
                }
            }
        }
        if (!grid_barrier(bar, bar + 1, gridDim.x, err)) break;
    }
    __shared__ float wm[SVD_SWEEP_NT / 32];
    for (int o = 16; o > 0; o >>= 1) mymax = fmaxf(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0) wm[w] = mymax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int i = 0; i < warps; ++i) m = fmaxf(m, wm[i]);
        block_max[blockIdx.x] = m;
    }
}

// Block one-sided Jacobi sweep for the FP32 preconditioning phase.  The columns of each
// sector are grouped into blocks of SVD_BW; a round pairs the blocks round-robin (a block
// left without a partner, or the only block, is processed alone), and one thread block
// takes one block pair: it forms the Gram matrix G = P^T P of the pair's <= 2 SVD_BW columns
// (64-row tiles through shared memory), runs one cyclic Jacobi sweep on G (disjoint
// rotations in parallel; each is the rotation the one-sided method would apply to that
// column pair), accumulates the rotations in W, and updates the columns of J and V by
// P <- P W.  One round per block pair instead of one per column pair: ~SVD_BW times fewer
// grid barriers per sweep, and the work is in small dense products.  Each block writes the
// largest off-diagonal ratio |G_ab| / sqrt(G_aa G_bb) it saw to block_max.
constexpr int SVD_BW = 16, SVD_PC = 2 * SVD_BW;
#ifndef SVD_TR_ROWS
#define SVD_TR_ROWS 128
#endif
constexpr int SVD_TR = SVD_TR_ROWS;
#ifndef HEFF_SVD_BLOCK
#define HEFF_SVD_BLOCK 1    // FP32 phase by block sweeps (0: column-pair sweeps)
#endif

__device__ __forceinline__ int rr_pos(int j, int round, int n) { return j == 0 ? 0 : 1 + (j - 1 + round) % (n - 1); }

#ifndef SVD_BT_THREADS
#define SVD_BT_THREADS 512
#endif
constexpr int SVD_BT = SVD_BT_THREADS;    // threads of a block-pair CTA
__global__ void __launch_bounds__(SVD_BT) svd_block_sweep_kernel(const SvdSector* __restrict__ secs, int nsec,
                                                              const int* __restrict__ bpair_off, int nbb_all,
                                                              float* __restrict__ base, float* __restrict__ block_max,
                                                              unsigned int* __restrict__ bar, int* __restrict__ err) {
    __shared__ float tile[SVD_TR][SVD_PC + 1];
    __shared__ float G[SVD_PC][SVD_PC + 1];
    __shared__ float W[SVD_PC][SVD_PC + 1];
    __shared__ float rc[SVD_PC / 2], rs[SVD_PC / 2];
    __shared__ int col[SVD_PC];
    __shared__ float bmax;
    const int tid = threadIdx.x;
    const int npairs = bpair_off[nsec];
    if (tid == 0) bmax = 0.f;
    for (int round = 0; round < nbb_all - 1; ++round) {
        for (int item = blockIdx.x; item < npairs; item += gridDim.x) {
            int lo = 0, hi = nsec;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (bpair_off[mid] <= item) lo = mid; else hi = mid;
            }
            const SvdSector sc = secs[lo];
            const int nb = (sc.k + SVD_BW - 1) / SVD_BW, nbb = nb + (nb & 1);
            if (round >= (nbb > 1 ? nbb - 1 : 1)) continue;                 // block-uniform
            const int pair = item - bpair_off[lo];
            int bp = nbb > 1 ? rr_pos(pair, round, nbb) : 0;
            int bq = nbb > 1 ? rr_pos(nbb - 1 - pair, round, nbb) : nbb;
            if (bp >= nb) { const int t = bp; bp = bq; bq = t; }              // the real block first
            if (bp >= nb) continue;
            const int np = min(SVD_BW, sc.k - bp * SVD_BW);
            const int nq = bq < nb ? min(SVD_BW, sc.k - bq * SVD_BW) : 0;
            const int nc = np + nq;
            if (tid < SVD_PC) col[tid] = tid < np ? bp * SVD_BW + tid : (tid < nc ? bq * SVD_BW + tid - np : -1);
            float* J = base + sc.j32_off;
            float* V = base + sc.v32_off;
            __syncthreads();
            // 1. G = P^T P, register-tiled: thread t takes the 4 x 4 block blk = t / 8 of G
            //    (rows 4 (blk / 8) .., columns 4 (blk % 8) ..) over the tile rows g, g + 8, ...
            //    (g = t % 8), and the 8 partial sums of a block (8 consecutive lanes) are added
            //    by shuffles: 8 shared-memory loads per 16 FMAs
            static_assert(SVD_PC == 32 && SVD_BT == 512 && SVD_TR % 8 == 0, "Gram tiling assumes 32 columns");
            const int gblk = tid >> 3, gg = tid & 7;
            const int ga0 = 4 * (gblk >> 3), gb0 = 4 * (gblk & 7);
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            // tiles of SVD_TR rows; the next tile's loads are issued into registers before the
            // current tile is used, so their latency overlaps the arithmetic
            constexpr int TE = SVD_TR * SVD_PC / SVD_BT;                    // tile elements per thread
            float nxt[TE];
            auto load_tile = [&](const float* M, int rows, int r0) {
#pragma unroll
                for (int u = 0; u < TE; ++u) {
                    const int e = tid + SVD_BT * u, a = e / SVD_TR, rr = e % SVD_TR;
                    const int cidx = col[a];
                    nxt[u] = (cidx >= 0 && r0 + rr < rows) ? M[(int64_t)cidx * rows + r0 + rr] : 0.f;
                }
            };
            auto stage_tile = [&]() {
#pragma unroll
                for (int u = 0; u < TE; ++u) {
                    const int e = tid + SVD_BT * u;
                    tile[e % SVD_TR][e / SVD_TR] = nxt[u];
                }
            };
            load_tile(J, sc.r, 0);
            for (int r0 = 0; r0 < sc.r; r0 += SVD_TR) {
                stage_tile();
                __syncthreads();
                if (r0 + SVD_TR < sc.r) load_tile(J, sc.r, r0 + SVD_TR);
#pragma unroll 4
                for (int rr = gg; rr < SVD_TR; rr += 8) {
                    float xa[4], xb[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) { xa[i] = tile[rr][ga0 + i]; xb[i] = tile[rr][gb0 + i]; }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], xb[j], acc[i][j]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], o);
            if (gg == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int a = ga0 + i, b = gb0 + j;
                        G[a][b] = (a < nc && b < nc) ? acc[i][j] : (a == b ? 1.f : 0.f);
                    }
            }
            for (int e = tid; e < SVD_PC * SVD_PC; e += SVD_BT) W[e / SVD_PC][e % SVD_PC] = (e / SVD_PC == e % SVD_PC);
            __syncthreads();
            // off-diagonal measure before the rotations (thread t: row t / 16, columns 2 (t % 16) + u)
            {
                const int ga = tid / (SVD_PC / 2), gbp = (tid % (SVD_PC / 2)) * 2;
                float m = 0.f;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int b = gbp + u;
                    if (ga < b && b < nc) {
                        const float d = sqrtf(G[ga][ga] * G[b][b]);
                        if (d > 0.f) m = fmaxf(m, fabsf(G[ga][b]) / d);
                    }
                }
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if ((tid & 31) == 0) atomicMax(reinterpret_cast<int*>(&bmax), __float_as_int(m));
            }
            // 2. one cyclic Jacobi sweep on G: SVD_PC - 1 rounds of SVD_PC / 2 disjoint rotations
            for (int jr = 0; jr < SVD_PC - 1; ++jr) {
                if (tid < SVD_PC / 2) {
                    int a = rr_pos(tid, jr, SVD_PC), b = rr_pos(SVD_PC - 1 - tid, jr, SVD_PC);
                    if (a > b) { const int t = a; a = b; b = t; }
                    const float gab = G[a][b], gaa = G[a][a], gbb = G[b][b];
                    float c = 1.f, sn = 0.f;
                    if (gab != 0.f && gaa > 0.f && gbb > 0.f && fabsf(gab) > 1e-7f * sqrtf(gaa * gbb)) {
                        // the rotation in FP32 (this phase only preconditions; FP64 arithmetic
                        // runs at GB300's much lower FP64 rate): a zeta too large to square
                        // gives t = 0, the limit of the formula
                        const float zeta = (gbb - gaa) / (2.f * gab);
                        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                        c = rsqrtf(fmaf(t, t, 1.f));
                        sn = c * t;
                    }
                    rc[tid] = c;
                    rs[tid] = sn;
                }
                __syncthreads();
                // columns: G <- G R, W <- W R (item: pair j = idx / SVD_PC, row x = idx % SVD_PC)
                for (int idx = tid; idx < (SVD_PC / 2) * SVD_PC; idx += SVD_BT) {
                    const int j = idx / SVD_PC, x = idx % SVD_PC;
                    int a = rr_pos(j, jr, SVD_PC), b = rr_pos(SVD_PC - 1 - j, jr, SVD_PC);
                    if (a > b) { const int t = a; a = b; b = t; }
                    const float c = rc[j], sn = rs[j];
                    if (sn != 0.f) {
                        const float ga_ = G[x][a], gb_ = G[x][b];
                        G[x][a] = c * ga_ - sn * gb_;
                        G[x][b] = sn * ga_ + c * gb_;
                        const float wa = W[x][a], wb = W[x][b];
                        W[x][a] = c * wa - sn * wb;
                        W[x][b] = sn * wa + c * wb;
                    }
                }
                __syncthreads();
                // rows: G <- R^T G
                for (int idx = tid; idx < (SVD_PC / 2) * SVD_PC; idx += SVD_BT) {
                    const int j = idx / SVD_PC, x = idx % SVD_PC;
                    int a = rr_pos(j, jr, SVD_PC), b = rr_pos(SVD_PC - 1 - j, jr, SVD_PC);
                    if (a > b) { const int t = a; a = b; b = t; }
                    const float c = rc[j], sn = rs[j];
                    if (sn != 0.f) {
                        const float ga_ = G[a][x], gb_ = G[b][x];
                        G[a][x] = c * ga_ - sn * gb_;
                        G[b][x] = sn * ga_ + c * gb_;
                    }
                }
                __syncthreads();
            }
            // 3. P <- P W for the columns of J (r rows) and of V (k rows), 128-row tiles,
            //    register-tiled: warp w takes the output columns 2w, 2w + 1 (their W columns
            //    held in registers), lane l the tile rows l, l + 32, l + 64, l + 96: 32 shared-
            //    memory loads per 64 FMAs, coalesced column stores
            static_assert(SVD_BT / 32 == SVD_PC / 2 && SVD_TR == 128, "update tiling: one warp per column pair");
            const int ua = 2 * (tid >> 5), ul = tid & 31;
            float w0[SVD_PC], w1[SVD_PC];
#pragma unroll
            for (int bb = 0; bb < SVD_PC; ++bb) { w0[bb] = W[bb][ua]; w1[bb] = W[bb][ua + 1]; }
            for (int pass = 0; pass < 2; ++pass) {
                float* M = pass == 0 ? J : V;
                const int rows = pass == 0 ? sc.r : sc.k;
                load_tile(M, rows, 0);
                for (int r0 = 0; r0 < rows; r0 += SVD_TR) {
                    stage_tile();
                    __syncthreads();
                    if (r0 + SVD_TR < rows) load_tile(M, rows, r0 + SVD_TR);
                    float o0[4], o1[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = ul + 32 * i;
                        float v0 = 0.f, v1 = 0.f;
#pragma unroll
                        for (int bb = 0; bb < SVD_PC; ++bb) {
                            const float t = tile[rr][bb];
                            v0 = fmaf(t, w0[bb], v0);
                            v1 = fmaf(t, w1[bb], v1);
                        }
                        o0[i] = v0;
                        o1[i] = v1;
                    }
                    __syncthreads();
                    const int c0 = col[ua], c1 = col[ua + 1];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = ul + 32 * i;
                        if (r0 + rr < rows) {
                            if (c0 >= 0) M[(int64_t)c0 * rows + r0 + rr] = o0[i];
                            if (c1 >= 0) M[(int64_t)c1 * rows + r0 + rr] = o1[i];
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, bar + 1, gridDim.x, err)) break;
    }
    __syncthreads();
    if (tid == 0) block_max[blockIdx.x] = bmax;
}

// largest slot value -> out[0] (one block; fixed order)
__global__ void __launch_bounds__(256) svd_offmax_kernel(const float* __restrict__ off, int n, float* __restrict__ out) {
    __shared__ float sh[256];
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) m = fmaxf(m, off[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// column norms of J = singular values
__global__ void svd_norms_kernel(const SvdSector* __restrict__ secs, const double* __restrict__ ws,
                                 double* __restrict__ sv) {
    const SvdSector s = secs[blockIdx.y];
    const int col = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (col >= s.k) return;
    const double* c = ws + s.j_off + (int64_t)col * s.r;
    double a = 0;
    for (int i = lane; i < s.r; i += 32) a = fma(c[i], c[i], a);
    a = warp_sum(a);
    if (lane == 0) sv[s.s_off + col] = sqrt(a);
}

// Write kept singular triplets.  Left vectors of M: columns of J / s (not transposed) or of
// V (transposed); right vectors: columns of V (not transposed) or J / s (transposed).
// A block (i, s1, c): element (a, k) = left[row0 + a, kept_k] * (absorb left ? s : 1)
// B block (c, s2, j): element (k, b) = right[col0 + b, kept_k] * (absorb right ? s : 1)
__global__ void svd_write_kernel(const SvdSector* __restrict__ secs, const WriteEntry* __restrict__ ent,
                                 const int32_t* __restrict__ kept, const double* __restrict__ ws,
                                 const double* __restrict__ sv, double* __restrict__ A, double* __restrict__ B,
                                 int absorb_right) {
    const WriteEntry e = ent[blockIdx.x];
    const SvdSector s = secs[e.sec];
    const double* J = ws + s.j_off;
    const double* V = ws + s.v_off;
    for (int idx = threadIdx.x; idx < e.rows * e.cols; idx += blockDim.x) {
        const int r = idx / e.cols, c = idx % e.cols;
        double v;
        if (e.left) {
            const int kc = kept[e.kept_off + c];                // J column index
            const double sk = sv[s.s_off + kc];
            const int row = e.vec_row0 + r;                      // row of M
            const double u = s.transposed ? V[(int64_t)kc * s.k + row] : J[(int64_t)kc * s.r + row] / sk;
            v = absorb_right ? u : u * sk;
            A[e.dst_off + idx] = v;
        } else {
            const int kc = kept[e.kept_off + r];
            const double sk = sv[s.s_off + kc];
            const int col = e.vec_row0 + c;                      // column of M
            const double w = s.transposed ? J[(int64_t)kc * s.r + col] / sk : V[(int64_t)kc * s.k + col];
            v = absorb_right ? w * sk : w;
            B[e.dst_off + idx] = v;
        }
    }
}

// One block meets the sweeps' grid barrier set up for two blocks: its wait must give up,
// set err and return.
__global__ void barrier_selftest_kernel(unsigned int* bar, int* err) { grid_barrier(bar, bar + 1, 2u, err); }

}  // namespace

void heff::svd_barrier_selftest(unsigned int* bar, int* err, void* stream) {
    barrier_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(bar, err);
}

extern "C" int heff_svd_create(const heff_layout* x, heff_svd** out) {
    heff::clear_error();
    if (!x || !out) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_create: null argument");
    *out = nullptr;
    if (x->idx.size() != 4) return fail(HEFF_ERR_CHARGE_MISMATCH, "x must have order 4");
    const heff::IndexDesc &al = x->idx[0], &p1 = x->idx[1], &p2 = x->idx[2], &be = x->idx[3];
    heff_svd* S = new (std::nothrow) heff_svd();
    if (!S) return fail(HEFF_ERR_OOM, "out of host memory");
    S->nq = x->nq;
    S->alpha_dims = al.dims;
    S->beta_dims = be.dims;
    try {
        std::map<std::vector<int32_t>, int> qid;
        std::vector<std::map<std::pair<int, int>, int32_t>> rpos, cpos;
        // sectors from the x blocks: Q = q(a) + q(s1)
        for (size_t b = 0; b < x->offsets.size(); ++b) {
            const int i = x->keys[b * 4], s1 = x->keys[b * 4 + 1], s2 = x->keys[b * 4 + 2], j = x->keys[b * 4 + 3];
            std::vector<int32_t> q = al.q(i);
            for (int c = 0; c < x->nq; ++c) q[c] += p1.charges[s1 * x->nq + c];
            auto it = qid.find(q);
            int id;
            if (it == qid.end()) {
                id = (int)S->Q.size();
                qid[q] = id;
                S->Q.push_back(q);
                S->rows.emplace_back();
                S->cols.emplace_back();
                rpos.emplace_back();
                cpos.emplace_back();
            } else {
                id = it->second;
            }
            if (!rpos[id].count({i, s1})) { rpos[id][{i, s1}] = 0; S->rows[id].push_back({i, s1, 0}); }
            if (!cpos[id].count({s2, j})) { cpos[id][{s2, j}] = 0; S->cols[id].push_back({s2, j, 0}); }
            (void)p2;
        }
        const int nsec = (int)S->Q.size();
        S->mrows.assign(nsec, 0);
        S->ncols.assign(nsec, 0);
        int64_t o = 0, so = 0, o32 = 0;
        for (int q = 0; q < nsec; ++q) {
            std::sort(S->rows[q].begin(), S->rows[q].end());
            std::sort(S->cols[q].begin(), S->cols[q].end());
            int32_t r = 0;
            for (auto& t : S->rows[q]) { std::get<2>(t) = r; rpos[q][{std::get<0>(t), std::get<1>(t)}] = r; r += al.dims[std::get<0>(t)]; }
            int32_t c = 0;
            for (auto& t : S->cols[q]) { std::get<2>(t) = c; cpos[q][{std::get<0>(t), std::get<1>(t)}] = c; c += be.dims[std::get<1>(t)]; }
            S->mrows[q] = r;
            S->ncols[q] = c;
            SvdSector sc{};
            sc.transposed = c > r;
            sc.r = sc.transposed ? c : r;
            sc.k = sc.transposed ? r : c;
            sc.j_off = o; o += (int64_t)sc.r * sc.k;
            sc.v_off = o; o += (int64_t)sc.k * sc.k;
            sc.g_off = o; o += (int64_t)sc.k * sc.k;
            sc.w_off = o; o += (int64_t)sc.r * sc.k;
            sc.j32_off = o32; o32 += (int64_t)sc.r * sc.k;
            sc.v32_off = o32; o32 += (int64_t)sc.k * sc.k;
            sc.s_off = (int32_t)so; so += sc.k;
            S->sec.push_back(sc);
            // FP64 GEMMs on column-major matrices, as row-major products of transposes:
            // G[i][j] = sum_l V[l,i] V[l,j]
            {
                heff::BProd p{};
                p.a_off = sc.v_off; p.a_rs = sc.k; p.a_cs = 1;
                p.b_off = sc.v_off; p.b_rs = 1; p.b_cs = sc.k;
                p.K = sc.k; p.c1 = -1; p.c2 = -1;
                S->gram.add_block(sc.g_off, sc.k, sc.k, sc.k, {p});
            }
            // W = V G (column-major W[i,j] = row j, column i of W^T): W^T[j][i] = sum_l G[l,j] V[i,l]
            {
                heff::BProd p{};
                p.a_off = sc.g_off; p.a_rs = sc.k; p.a_cs = 1;
                p.b_off = sc.v_off; p.b_rs = sc.k; p.b_cs = 1;
                p.K = sc.k; p.c1 = -1; p.c2 = -1;
                S->vg.add_block(sc.w_off, sc.k, sc.k, sc.k, {p});
            }
            // W = J V (r x k): W^T[j][i] = sum_l V[l,j] J[i,l]
            {
                heff::BProd p{};
                p.a_off = sc.v_off; p.a_rs = sc.k; p.a_cs = 1;
                p.b_off = sc.j_off; p.b_rs = sc.r; p.b_cs = 1;
                p.K = sc.k; p.c1 = -1; p.c2 = -1;
                S->jv.add_block(sc.w_off, sc.r, sc.k, sc.r, {p});
            }
            S->max_k = std::max(S->max_k, sc.k);
        }
        S->s_total = so;
        // load table: [sector, x_off, m_rows, n_cols, row0, col0] per x block
        std::vector<int64_t> tab;
        for (size_t b = 0; b < x->offsets.size(); ++b) {
            const int i = x->keys[b * 4], s1 = x->keys[b * 4 + 1], s2 = x->keys[b * 4 + 2], j = x->keys[b * 4 + 3];
            std::vector<int32_t> q = al.q(i);
            for (int c = 0; c < x->nq; ++c) q[c] += p1.charges[s1 * x->nq + c];
            const int id = qid[q];
            tab.insert(tab.end(), {(int64_t)id, x->offsets[b], (int64_t)al.dims[i], (int64_t)be.dims[j],
                                   (int64_t)rpos[id][{i, s1}], (int64_t)cpos[id][{s2, j}]});
        }
        S->xoff.assign(1, tab);   // stash the load table (one entry)
        S->ws_doubles = o + so + 64;
        const int kk = S->max_k + (S->max_k & 1);
        S->slot_ld = std::max(1, kk / 2);
        S->nslots = (int64_t)nsec * S->slot_ld;
        S->off_slots = ((size_t)S->ws_doubles * sizeof(double) + tab.size() * sizeof(int64_t) + 255) / 256 * 256;
        S->off_f32 = (S->off_slots + (size_t)(S->nslots + 64 + 2 * nsec + 16) * sizeof(float) + 255) / 256 * 256;
        S->ws_bytes = S->off_f32 + (size_t)o32 * sizeof(float) + 1024;
    } catch (const std::bad_alloc&) {
        delete S;
        return fail(HEFF_ERR_OOM, "out of host memory in heff_svd_create");
    }
    *out = S;
    return HEFF_OK;
}

extern "C" int heff_svd_workspace_size(const heff_svd* S, size_t* bytes) {
    heff::clear_error();
    if (!S || !bytes) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_workspace_size: null argument");
    *bytes = S->ws_bytes;
    return HEFF_OK;
}

#define SVD_CK(call)                                                                                     \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return fail(HEFF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

extern "C" int heff_svd_compute(heff_svd* S, const double* x, void* workspace, size_t workspace_bytes,
                                void* stream, int32_t* sweeps_out) {
    heff::clear_error();
    if (!S || !x) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_compute: null argument");
    if (!workspace || workspace_bytes < S->ws_bytes || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(HEFF_ERR_WORKSPACE, "SVD workspace of %zu bytes, needs %zu", workspace_bytes, S->ws_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* ws = static_cast<double*>(workspace);
    double* sv = ws + (S->ws_doubles - S->s_total - 64);
    float* slots = reinterpret_cast<float*>(static_cast<char*>(workspace) + S->off_slots);
    float* offmax = slots + S->nslots;
    const std::vector<int64_t>& tab = S->xoff[0];
    int64_t* d_tab = reinterpret_cast<int64_t*>(ws + S->ws_doubles);
    const int nsec = (int)S->sec.size();
    if (!S->d_sec) SVD_CK(cudaMalloc((void**)&S->d_sec, std::max<size_t>(1, S->sec.size()) * sizeof(SvdSector)));
    SVD_CK(cudaMemcpyAsync(S->d_sec, S->sec.data(), S->sec.size() * sizeof(SvdSector), cudaMemcpyHostToDevice, st));
    SVD_CK(cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    const int ntab = (int)(tab.size() / 6);
    float* f32 = reinterpret_cast<float*>(static_cast<char*>(workspace) + S->off_f32);
    if (ntab) svd_load_kernel<<<std::min(ntab, 4096), 256, 0, st>>>(S->d_sec, d_tab, ntab, x, ws);
    svd_to_f32_kernel<<<dim3(128, nsec), 256, 0, st>>>(S->d_sec, ws, f32);
    heff::count_launches(2);
    if (!S->lists_uploaded) {
        int rc = HEFF_OK;
        for (heff::BList* b : {&S->gram, &S->vg, &S->jv})
            if (!rc) rc = heff::blist_upload(*b);
        if (rc) return rc;
        S->lists_uploaded = true;
    }
    // Jacobi sweeps until the largest off-diagonal measure is below tol: one cooperative
    // launch per sweep (all rounds, grid barrier between rounds)
    const int kk_all = S->max_k + (S->max_k & 1);
    if (S->pair_off.empty()) {
        S->pair_off.push_back(0);
        for (const SvdSector& sc : S->sec) S->pair_off.push_back(S->pair_off.back() + (sc.k + (sc.k & 1)) / 2);
    }
    int* d_pair_off = reinterpret_cast<int*>(slots + S->nslots + 16);
    unsigned int* d_bar = reinterpret_cast<unsigned int*>(d_pair_off + S->pair_off.size());
    int* d_err = reinterpret_cast<int*>(d_bar + 2);
    SVD_CK(cudaMemcpyAsync(d_pair_off, S->pair_off.data(), S->pair_off.size() * sizeof(int), cudaMemcpyHostToDevice,
                           st));
    SVD_CK(cudaMemsetAsync(d_bar, 0, 3 * sizeof(unsigned int), st));
    // stop_below: a sweep whose largest off-diagonal measure (taken before its rotations) is
    // below this ends the loop; for the FP64 phase it is sqrt(tol): Jacobi sweeps converge
    // quadratically, so that sweep's rotations leave the measure near tol, and a further
    // sweep would only confirm it
    auto sweeps = [&](auto* base, float stop_below, int max_sweeps, int& out) -> int {
        using T = typename std::remove_pointer<decltype(base)>::type;
        out = 0;
        if (kk_all < 2) return HEFF_OK;
        int dev = 0, nsm = 0, per_sm = 0;
        SVD_CK(cudaGetDevice(&dev));
        SVD_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        SVD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_sweep_kernel<T>, SVD_SWEEP_NT, 0));
        const int npairs = S->pair_off.back();
        int grid = std::max(1, std::min(nsm * std::max(per_sm, 1), (npairs + 7) / 8));
        grid = std::min<int>(grid, (int)S->nslots);
        const SvdSector* secs = S->d_sec;
        int nsec_i = nsec, kk_i = kk_all;
        T* base_t = base;
        T* nrm_t = reinterpret_cast<T*>(sv);             // the singular-value slots, free until the end
        int ncols_i = (int)S->s_total;
        while (out < max_sweeps) {
            void* args[] = {(void*)&secs, (void*)&nsec_i, (void*)&d_pair_off, (void*)&kk_i, (void*)&base_t,
                            (void*)&nrm_t, (void*)&ncols_i, (void*)&slots, (void*)&d_bar, (void*)&d_err};
            SVD_CK(cudaLaunchCooperativeKernel((const void*)svd_sweep_kernel<T>, dim3(grid), dim3(SVD_SWEEP_NT),
                                               args, 0, st));
            svd_offmax_kernel<<<1, 256, 0, st>>>(slots, grid, offmax);
            heff::count_launches(2);
            float m = 0.f;
            int e = 0;
            SVD_CK(cudaMemcpyAsync(&m, offmax, sizeof(float), cudaMemcpyDeviceToHost, st));
            SVD_CK(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            SVD_CK(cudaStreamSynchronize(st));
            if (e) return fail(HEFF_ERR_TIMEOUT, "SVD sweep: grid barrier timed out");
            ++out;
            if (m < stop_below) break;
        }
        return HEFF_OK;
    };
    // FP32 block sweeps: the same convergence test on the block pairs' Gram matrices
    auto block_sweeps = [&](float* base, float tol, int max_sweeps, int& out) -> int {
        out = 0;
        std::vector<int> boff(1, 0);
        int nbb_all = 2;
        for (const SvdSector& sc : S->sec) {
            const int nb = (sc.k + SVD_BW - 1) / SVD_BW, nbb = nb + (nb & 1);
            boff.push_back(boff.back() + nbb / 2);
            nbb_all = std::max(nbb_all, nbb);
        }
        int* d_boff = d_err + 2;
        SVD_CK(cudaMemcpyAsync(d_boff, boff.data(), boff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        int dev = 0, nsm = 0, per_sm = 0;
        SVD_CK(cudaGetDevice(&dev));
        SVD_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        SVD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_block_sweep_kernel, SVD_BT, 0));
        int grid = std::max(1, std::min(nsm * std::max(per_sm, 1), boff.back()));
        grid = std::min<int>(grid, (int)S->nslots);
        const SvdSector* secs = S->d_sec;
        int nsec_i = nsec, nbb_i = nbb_all;
        float* base_t = base;
        while (out < max_sweeps) {
            void* args[] = {(void*)&secs, (void*)&nsec_i, (void*)&d_boff, (void*)&nbb_i, (void*)&base_t,
                            (void*)&slots, (void*)&d_bar, (void*)&d_err};
            SVD_CK(cudaLaunchCooperativeKernel((const void*)svd_block_sweep_kernel, dim3(grid), dim3(SVD_BT), args, 0,
                                               st));
            svd_offmax_kernel<<<1, 256, 0, st>>>(slots, grid, offmax);
            heff::count_launches(2);
            float m = 0.f;
            int e = 0;
            SVD_CK(cudaMemcpyAsync(&m, offmax, sizeof(float), cudaMemcpyDeviceToHost, st));
            SVD_CK(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            SVD_CK(cudaStreamSynchronize(st));
            if (e) return fail(HEFF_ERR_TIMEOUT, "SVD block sweep: grid barrier timed out");
            ++out;
            if (m < tol) break;
        }
        return HEFF_OK;
    };
    int rc;
    // FP32 preconditioning sweeps (to FP32 accuracy of the dot products)
    if (HEFF_SVD_BLOCK) {
        if ((rc = block_sweeps(f32, 1e-5f, 30, S->fp32_sweeps))) return rc;
    } else if ((rc = sweeps(f32, 1e-5f, 30, S->fp32_sweeps))) {
        return rc;
    }
    // V = orthonormalised double(V32), J = J V
    svd_v_to_f64_kernel<<<dim3(128, nsec), 256, 0, st>>>(S->d_sec, f32, ws);
    heff::count_launches(1);
    for (int it = 0; it < 2; ++it) {
        if ((rc = heff::launch_bgemm(S->gram, ws, ws, ws, nullptr, nullptr, 1.0, stream))) return rc;
        if ((rc = heff::launch_bgemm(S->vg, ws, ws, ws, nullptr, nullptr, -0.5, stream))) return rc;
        svd_ns_kernel<<<dim3(128, nsec), 256, 0, st>>>(S->d_sec, ws);
        heff::count_launches(1);
    }
    if ((rc = heff::launch_bgemm(S->jv, ws, ws, ws, nullptr, nullptr, 1.0, stream))) return rc;
    svd_copy_w_kernel<<<dim3(128, nsec), 256, 0, st>>>(S->d_sec, ws);
    heff::count_launches(1);
    // FP64 sweeps to convergence: off-diagonal measure 1e-14, i.e. stop after the sweep that
    // saw at most 1e-7
    if ((rc = sweeps(ws, 1e-7f, 40, S->fp64_sweeps))) return rc;
    const int sweep = S->fp64_sweeps;
    svd_norms_kernel<<<dim3((S->max_k + 3) / 4 + 1, nsec), 128, 0, st>>>(S->d_sec, ws, sv);
    heff::count_launches(1);
    S->s.assign(S->s_total, 0.0);
    SVD_CK(cudaMemcpyAsync(S->s.data(), sv, S->s_total * sizeof(double), cudaMemcpyDeviceToHost, st));
    SVD_CK(cudaStreamSynchronize(st));
    SVD_CK(cudaGetLastError());
    if (sweeps_out) *sweeps_out = sweep;
    S->computed = true;
    S->kept.clear();
    return HEFF_OK;
}

extern "C" int heff_svd_info(const heff_svd* S, int32_t* fp32_sweeps, int32_t* fp64_sweeps) {
    heff::clear_error();
    if (!S) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_info: null argument");
    if (fp32_sweeps) *fp32_sweeps = S->fp32_sweeps;
    if (fp64_sweeps) *fp64_sweeps = S->fp64_sweeps;
    return HEFF_OK;
}

extern "C" int heff_svd_truncate(heff_svd* S, int32_t m_max, double cutoff, int32_t* nsec_out,
                                 int32_t* charges_out, int32_t* dims_out, double* discarded, double* norm) {
    heff::clear_error();
    if (!S || !nsec_out) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_truncate: null argument");
    if (!S->computed) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_truncate before heff_svd_compute");
    if (m_max < 1) return fail(HEFF_ERR_INVALID_ARG, "m_max must be >= 1");
    double tot = 0;
    for (double v : S->s) tot += v * v;
    const double nrm = std::sqrt(tot);
    S->norm = nrm;
    // candidates (normalised s, sector, rank inside the sector by decreasing s)
    struct Cand { double s; int sec; int rank; int col; };
    std::vector<Cand> cand;
    const int nsec = (int)S->sec.size();
    for (int q = 0; q < nsec; ++q) {
        const SvdSector& sc = S->sec[q];
        std::vector<int> idx(sc.k);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return S->s[sc.s_off + a] > S->s[sc.s_off + b]; });
        for (int r = 0; r < sc.k; ++r)
            cand.push_back({nrm > 0 ? S->s[sc.s_off + idx[r]] / nrm : 0.0, q, r, idx[r]});
    }
    double smax = 0;
    for (auto& c : cand) smax = std::max(smax, c.s);
    auto qabs = [&](int q) { long a = 0; for (int v : S->Q[q]) a += std::abs(v); return a; };
    // order: decreasing s (ties within 1e-12 s_max), then |Q|, Q, rank inside the sector
    std::stable_sort(cand.begin(), cand.end(), [&](const Cand& a, const Cand& b) {
        const double ka = std::nearbyint(a.s / std::max(smax, 1e-300) / 1e-12);
        const double kb = std::nearbyint(b.s / std::max(smax, 1e-300) / 1e-12);
        if (ka != kb) return ka > kb;
        if (qabs(a.sec) != qabs(b.sec)) return qabs(a.sec) < qabs(b.sec);
        if (S->Q[a.sec] != S->Q[b.sec]) return S->Q[a.sec] < S->Q[b.sec];
        return a.rank < b.rank;
    });
    S->kept.assign(nsec, {});
    std::vector<std::vector<std::pair<int, int>>> kr(nsec);   // (rank, col)
    double kept2 = 0, all2 = 0;
    int nk = 0;
    for (auto& c : cand) {
        all2 += c.s * c.s;
        if (c.s >= cutoff && nk < m_max) {
            kr[c.sec].push_back({c.rank, c.col});
            kept2 += c.s * c.s;
            ++nk;
        }
    }
    // new bond: sectors with at least one kept value, in increasing charge order
    std::vector<int> order(nsec);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return S->Q[a] < S->Q[b]; });
    int ns = 0;
    for (int q : order) {
        if (kr[q].empty()) continue;
        std::sort(kr[q].begin(), kr[q].end());
        for (auto& rc : kr[q]) S->kept[q].push_back(rc.second);
        if (charges_out) std::memcpy(charges_out + ns * S->nq, S->Q[q].data(), sizeof(int32_t) * S->nq);
        if (dims_out) dims_out[ns] = (int32_t)kr[q].size();
        ++ns;
    }
    *nsec_out = ns;
    S->discarded = all2 - kept2;
    if (discarded) *discarded = S->discarded;
    if (norm) *norm = nrm;
    return HEFF_OK;
}

extern "C" int heff_svd_singular_values(const heff_svd* S, double* out) {
    heff::clear_error();
    if (!S || !out) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_singular_values: null argument");
    std::vector<int> order(S->sec.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return S->Q[a] < S->Q[b]; });
    int64_t n = 0;
    for (int q : order)
        if (q < (int)S->kept.size())
            for (int c : S->kept[q]) out[n++] = S->s[S->sec[q].s_off + c];
    return HEFF_OK;
}

extern "C" int heff_svd_write(heff_svd* S, const heff_layout* A_layout, const heff_layout* B_layout, double* A,
                              double* B, int32_t absorb_right, void* workspace, size_t workspace_bytes,
                              void* stream) {
    heff::clear_error();
    if (!S || !A_layout || !B_layout || !A || !B) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_write: null argument");
    if (S->kept.empty()) return fail(HEFF_ERR_INVALID_ARG, "heff_svd_write before heff_svd_truncate");
    if (!workspace || workspace_bytes < S->ws_bytes) return fail(HEFF_ERR_WORKSPACE, "SVD workspace too small");
    if (A_layout->idx.size() != 3 || B_layout->idx.size() != 3)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "left/right tensors must have order 3");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* ws = static_cast<double*>(workspace);
    double* sv = ws + (S->ws_doubles - S->s_total - 64);
    // new bond sector number for each kept sector (charge order)
    std::map<std::vector<int32_t>, int> bond;
    const heff::IndexDesc& nb = A_layout->idx[2];
    for (int c = 0; c < nb.nsec; ++c) bond[nb.q(c)] = c;
    std::vector<WriteEntry> ents;
    std::vector<int32_t> keptflat;
    std::vector<int32_t> koff(S->sec.size(), 0);
    for (size_t q = 0; q < S->sec.size(); ++q) {
        koff[q] = (int32_t)keptflat.size();
        keptflat.insert(keptflat.end(), S->kept[q].begin(), S->kept[q].end());
    }
    for (size_t q = 0; q < S->sec.size(); ++q) {
        if (S->kept[q].empty()) continue;
        auto bit = bond.find(S->Q[q]);
        if (bit == bond.end() || nb.dims[bit->second] != (int)S->kept[q].size())
            return fail(HEFF_ERR_CHARGE_MISMATCH, "left tensor bond does not match the truncation");
        const int c = bit->second, nkeep = (int)S->kept[q].size();
        for (auto& t : S->rows[q]) {            // A block (i, s1, c)
            const int64_t off = A_layout->offset_of({std::get<0>(t), std::get<1>(t), c});
            if (off < 0) return fail(HEFF_ERR_CHARGE_MISMATCH, "left tensor block missing");
            ents.push_back({off, S->alpha_dims[std::get<0>(t)], nkeep, (int32_t)q, std::get<2>(t), koff[q], 1});
        }
        for (auto& t : S->cols[q]) {            // B block (c, s2, j)
            const int64_t off = B_layout->offset_of({c, std::get<0>(t), std::get<1>(t)});
            if (off < 0) return fail(HEFF_ERR_CHARGE_MISMATCH, "right tensor block missing");
            ents.push_back({off, nkeep, S->beta_dims[std::get<1>(t)], (int32_t)q, std::get<2>(t), koff[q], 0});
        }
    }
    // the write tables (sized by the truncation) go to temporary device buffers
    WriteEntry* d_ent = nullptr;
    int32_t* d_kept = nullptr;
    SVD_CK(cudaMalloc((void**)&d_ent, std::max<size_t>(1, ents.size()) * sizeof(WriteEntry)));
    SVD_CK(cudaMalloc((void**)&d_kept, std::max<size_t>(1, keptflat.size()) * sizeof(int32_t)));
    SVD_CK(cudaMemcpyAsync(d_ent, ents.data(), ents.size() * sizeof(WriteEntry), cudaMemcpyHostToDevice, st));
    SVD_CK(cudaMemcpyAsync(d_kept, keptflat.data(), keptflat.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (!ents.empty())
        svd_write_kernel<<<(unsigned)ents.size(), 256, 0, st>>>(S->d_sec, d_ent, d_kept, ws, sv, A, B, absorb_right);
    heff::count_launches(1);
    SVD_CK(cudaStreamSynchronize(st));
    cudaFree(d_ent);
    cudaFree(d_kept);
    SVD_CK(cudaGetLastError());
    return HEFF_OK;
}

extern "C" void heff_svd_destroy(heff_svd* S) {
    if (!S) return;
    cudaFree(S->d_sec);
    heff::blist_free(S->gram);
    heff::blist_free(S->vg);
    heff::blist_free(S->jv);
    delete S;
}
