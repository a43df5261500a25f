// FP64 Lanczos eigensolver on the GPU around the H_eff matvec (the eigensolver of the
// two-site DMRG step, Section II-C / III; Lanczos is the fixed-iteration alternative to
// the Davidson routine of Algorithm 1).
//
// Every vector operation runs in FP64 on the device and the loop never synchronises with
// the host.  Per iteration k:
//   w = H v_k                       (heff_apply_prepared; any precision, FP64 vectors)
//   a = v_k . (w - beta_{k-1} v_{k-1}),  w -= beta_{k-1} v_{k-1} + a v_k
//                                   (the three-term recurrence, with ||w||^2 after it)
//   h = V^T w, w -= V h             (classical Gram-Schmidt against v_0..v_k: the full
//                                    reorthogonalisation, with ||w||^2 after it)
//   h2 = V^T w, w -= V h2           (a second pass, only when the first removed more than half
//                                    of ||w||^2: the criterion of Daniel, Gragg, Kaufman and
//                                    Stewart (1976); "twice is enough")
//   alpha_k = a + h_k (+ h2_k), beta_k = ||w||, v_{k+1} = w / beta_k
// The recurrence goes first so that the Gram-Schmidt pass acts on a vector already
// orthogonal to V up to the basis' own small loss of orthogonality: a pass applied to
// H v_k itself would carry that loss, times ||H v_k|| / beta_k, into v_{k+1} (large once
// the start vector is nearly an eigenvector, as in the later sweeps of DMRG).
// then the lowest eigenpair of the (n x n) tridiagonal matrix is found on the device
// (bisection + inverse iteration), and the Ritz vector x = sum_j s_j v_j is formed and
// normalised.  If beta_k falls below 1e-13 |alpha_k| the Krylov space is invariant: the
// remaining iterations become no-ops and the eigenproblem uses the k + 1 vectors built.
// Reductions are two-stage with a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

using heff::fail;

namespace heff {
namespace {

constexpr int RT = 256;          // threads per reduction block
constexpr int RB = 456;          // reduction blocks (partial sums per vector): 3 per SM on 152 SMs
constexpr int VT = 8;            // vectors per multi-dot pass

constexpr int GMAX = 4096;       // largest grid of the element-wise kernels (grid_for)
constexpr int NVMAX = 128;       // basis vectors of one Lanczos workspace, at most

// State in the Lanczos workspace (doubles): [0] n_eff (as double), [1] active flag,
// [2] theta, [3] residual estimate, [4] second Gram-Schmidt pass needed (this step),
// [8..8+NMAX) alpha, [8+NMAX..) beta, then h (NMAX), s (NMAX), partials (RB * NVMAX), the
// partial sums of ||w||^2 after the three-term update (RB) and after a Gram-Schmidt pass
// (GMAX), and a (the three-term projection of the current step).
struct LzLayout {
    int nmax;
    int64_t n;
    size_t off_state, off_h, off_s, off_part, off_wn, off_sq, off_a, off_T, off_V, bytes;
};

LzLayout lz_layout(int64_t n, int n_iter) {
    LzLayout l{};
    l.nmax = n_iter + 1;
    l.n = n;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t o = 0;
    l.off_state = o; o = al(o + sizeof(double) * (8 + 2 * (size_t)l.nmax));
    l.off_h = o;     o = al(o + sizeof(double) * (size_t)l.nmax);
    l.off_s = o;     o = al(o + sizeof(double) * (size_t)l.nmax);
    l.off_part = o;  o = al(o + sizeof(double) * (size_t)RB * NVMAX);
    l.off_wn = o;    o = al(o + sizeof(double) * (size_t)RB);
    l.off_sq = o;    o = al(o + sizeof(double) * (size_t)GMAX);
    l.off_a = o;     o = al(o + sizeof(double));
    l.off_T = o;     o = al(o + sizeof(double) * 2 * (size_t)l.nmax * l.nmax);
    l.off_V = o;     o = al(o + sizeof(double) * (size_t)(l.nmax + 1) * (size_t)n);   // V + w
    l.bytes = o;
    return l;
}

struct Lz {
    double* state;   // n_eff, active, theta, resid, second pass, alpha[nmax], beta[nmax]
    double* h;
    double* s;
    double* part;
    double* wn;      // partial sums of ||w||^2 after the three-term update (RB)
    double* sq;      // partial sums of ||w||^2 after a combine (one per block of its grid)
    double* a;       // the three-term projection a of the current step
    double* T;       // nmax x nmax matrix + nmax x nmax eigenvectors
    double* V;       // (nmax) basis vectors, then w
    int64_t n;
    int nmax;
    double* w() const { return V + (int64_t)nmax * n; }
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;
}

// Whether a gated kernel runs: gate 0 while the iteration is active, gate 1 only when the
// active step also needs its second Gram-Schmidt pass (state[4]).
__device__ __forceinline__ bool gated_off(const double* state, int gate) {
    return state[1] == 0.0 || (gate == 1 && state[4] == 0.0);
}

// partial[b * VT + t] = sum over block b's chunk of V[j0 + t] . w, t < nv
__global__ void __launch_bounds__(RT) multidot_kernel(const double* __restrict__ V, const double* __restrict__ w,
                                                      int64_t n, int j0, int nv, double* __restrict__ part,
                                                      const double* __restrict__ state) {
    __shared__ double sh[RT / 32];
    if (state[1] == 0.0) return;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t beg = (int64_t)blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
    double acc[VT];
#pragma unroll
    for (int t = 0; t < VT; ++t) acc[t] = 0.0;
    // two elements per iteration: 2 (nv + 1) loads in flight per thread
    int64_t i = beg + threadIdx.x;
    for (; i + RT < end; i += 2 * RT) {
        const double w0 = w[i], w1 = w[i + RT];
        double v0[VT], v1[VT];
#pragma unroll
        for (int t = 0; t < VT; ++t) {
            v0[t] = t < nv ? V[(int64_t)(j0 + t) * n + i] : 0.0;
            v1[t] = t < nv ? V[(int64_t)(j0 + t) * n + i + RT] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < VT; ++t) acc[t] = fma(v1[t], w1, fma(v0[t], w0, acc[t]));
    }
    for (; i < end; i += RT) {
        const double wi = w[i];
#pragma unroll
        for (int t = 0; t < VT; ++t)
            if (t < nv) acc[t] = fma(V[(int64_t)(j0 + t) * n + i], wi, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < VT; ++t) {
        if (t >= nv) break;                          // block-uniform
        double s = block_sum(acc[t], sh);
        if (threadIdx.x == 0) part[blockIdx.x * VT + t] = s;
    }
}

// The three-term recurrence of step k, in two launches: mode 0 writes partial sums of
// v_k . (w - beta_{k-1} v_{k-1}) to part[b * VT] (a = their sum, by finish_dots into
// *ap); mode 1 updates w -= beta_{k-1} v_{k-1} + a v_k and writes the partial sums of the
// new ||w||^2 to wn[b].  k = 0 has no v_{k-1} term.
__global__ void __launch_bounds__(RT) three_term_kernel(const double* __restrict__ V, double* __restrict__ w,
                                                        int64_t n, int k, int nmax, double* __restrict__ part,
                                                        double* __restrict__ wn, const double* __restrict__ state,
                                                        const double* __restrict__ ap, int mode) {
    __shared__ double sh[RT / 32];
    if (state[1] == 0.0) return;
    const double* vk = V + (int64_t)k * n;
    const double* vp = k > 0 ? V + (int64_t)(k - 1) * n : vk;
    const double b = k > 0 ? state[8 + nmax + k - 1] : 0.0;
    const double a = mode == 1 ? *ap : 0.0;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * RT;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
        const double x = w[i] - b * vp[i];
        if (mode == 0) {
            acc = fma(vk[i], x, acc);
        } else {
            const double y = x - a * vk[i];
            w[i] = y;
            acc = fma(y, y, acc);
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        if (mode == 0) part[blockIdx.x * VT] = acc;
        else wn[blockIdx.x] = acc;
    }
}

// out[j0 + t] = (accumulate ? out : 0) + sum_b partial[b * VT + t]
__global__ void finish_dots_kernel(const double* __restrict__ part, int nb, int j0, int nv, double* out,
                                   int accumulate, const double* __restrict__ state) {
    __shared__ double sh[RT / 32];
    if (state[1] == 0.0) return;
    for (int t = 0; t < nv; ++t) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b * VT + t];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) out[j0 + t] = accumulate ? out[j0 + t] + v : v;
    }
}

// y[i] = (beta_y * y[i]) + sign * sum_{j < nv} c[j] V[j][i]   (c from device memory); with
// sq, also sq[b] = block b's sum of the new y[i]^2.  With clamp, only the first state[0]
// rows (the Krylov dimension reached) enter: rows never written after a breakdown are not
// read.
__global__ void __launch_bounds__(RT) combine_kernel(const double* __restrict__ V, int64_t n, int nv,
                                                     const double* __restrict__ c, double sign, double beta_y,
                                                     double* __restrict__ y, const double* __restrict__ state,
                                                     int ignore_active, int gate = 0,
                                                     double* __restrict__ sq = nullptr, int clamp = 0) {
    __shared__ double cs[128];
    __shared__ double sh[RT / 32];
    if (!ignore_active && gated_off(state, gate)) return;
    if (clamp) nv = min(nv, (int)state[0]);
    for (int j = threadIdx.x; j < nv; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    // two elements per iteration (their loads in flight together), then the remainder
    const int64_t stride = (int64_t)gridDim.x * RT;
    int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x;
    double yy = 0.0;
    for (; i + stride < n; i += 2 * stride) {
        double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
        for (int j = 0; j < nv; ++j) {
            a0 = fma(cs[j], V[(int64_t)j * n + i], a0);
            a1 = fma(cs[j], V[(int64_t)j * n + i + stride], a1);
        }
        const double y0 = (beta_y == 0.0 ? 0.0 : beta_y * y[i]) + sign * a0;
        const double y1 = (beta_y == 0.0 ? 0.0 : beta_y * y[i + stride]) + sign * a1;
        y[i] = y0;
        y[i + stride] = y1;
        yy = fma(y1, y1, fma(y0, y0, yy));
    }
    for (; i < n; i += stride) {
        double a = 0.0;
#pragma unroll 8
        for (int j = 0; j < nv; ++j) a = fma(cs[j], V[(int64_t)j * n + i], a);
        const double y0 = (beta_y == 0.0 ? 0.0 : beta_y * y[i]) + sign * a;
        y[i] = y0;
        yy = fma(y0, y0, yy);
    }
    if (sq) {                                        // block-uniform
        yy = block_sum(yy, sh);
        if (threadIdx.x == 0) sq[blockIdx.x] = yy;
    }
}

// sum of squares of x into part (stage 1)
__global__ void __launch_bounds__(RT) sumsq_kernel(const double* __restrict__ x, int64_t n, double* part) {
    __shared__ double sh[RT / 32];
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
        a = fma(x[i], x[i], a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x * VT] = a;
}

// dst = src / sqrt(sum part); mode 0: initial vector (sets active and n_eff = 0); mode 2:
// plain; mode 3: plain, only while active
__global__ void __launch_bounds__(RT) normalize_kernel(const double* __restrict__ part, int nb,
                                                       const double* __restrict__ src, double* __restrict__ dst,
                                                       int64_t n, double* state, int mode) {
    __shared__ double sh[RT / 32];
    __shared__ double nrm;
    if (mode == 3 && state[1] == 0.0) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b * VT];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) nrm = sqrt(v);
    __syncthreads();
    const double r = nrm;
    if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        state[0] = 0.0;
        state[1] = r > 0.0 ? 1.0 : 0.0;
    }
    if (!(r > 0.0)) return;
    const double inv = 1.0 / r;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) dst[i] = src[i] * inv;
}

// All the projections of one Gram-Schmidt pass in one launch: block (b, g) computes the
// dots of basis vectors g VT .. g VT + VT - 1 (those below nvec) with w over chunk b, into
// part[j * gridDim.x + b]; vec_finish_kernel adds each vector's partials in a fixed order.
__global__ void __launch_bounds__(RT) multidot_all_kernel(const double* __restrict__ V,
                                                          const double* __restrict__ w, int64_t n, int nvec,
                                                          double* __restrict__ part,
                                                          const double* __restrict__ state, int gate) {
    __shared__ double sh[RT / 32];
    if (gated_off(state, gate)) return;
    const int j0 = blockIdx.y * VT;
    const int nv = nvec - j0 < VT ? nvec - j0 : VT;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t beg = (int64_t)blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
    double acc[VT];
#pragma unroll
    for (int t = 0; t < VT; ++t) acc[t] = 0.0;
    int64_t i = beg + threadIdx.x;
    for (; i + RT < end; i += 2 * RT) {
        const double w0 = w[i], w1 = w[i + RT];
        double v0[VT], v1[VT];
#pragma unroll
        for (int t = 0; t < VT; ++t) {
            v0[t] = t < nv ? V[(int64_t)(j0 + t) * n + i] : 0.0;
            v1[t] = t < nv ? V[(int64_t)(j0 + t) * n + i + RT] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < VT; ++t) acc[t] = fma(v1[t], w1, fma(v0[t], w0, acc[t]));
    }
    for (; i < end; i += RT) {
        const double wi = w[i];
#pragma unroll
        for (int t = 0; t < VT; ++t)
            if (t < nv) acc[t] = fma(V[(int64_t)(j0 + t) * n + i], wi, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < VT; ++t) {
        if (t >= nv) break;                          // block-uniform
        const double sum = block_sum(acc[t], sh);
        if (threadIdx.x == 0) part[(int64_t)(j0 + t) * gridDim.x + blockIdx.x] = sum;
    }
}

// out[j] = sum over b < nb of part[j * nb + b], one block per vector j
__global__ void vec_finish_kernel(const double* __restrict__ part, int nb, double* __restrict__ out,
                                  const double* __restrict__ state, int gate) {
    __shared__ double sh[RT / 32];
    if (gated_off(state, gate)) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[(int64_t)blockIdx.x * nb + b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// beta_k = ||w|| from the nb partial sums of squares; records beta_k and n_eff = k + 1 and
// ends the iteration when beta_k <= 1e-13 |alpha_k| (an invariant Krylov space)
__global__ void lz_beta_kernel(const double* __restrict__ sq, int nb, double* state, int k, int nmax) {
    __shared__ double sh[RT / 32];
    if (state[1] == 0.0) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += sq[b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        const double r = sqrt(v), a = state[8 + k];
        state[8 + nmax + k] = r;
        state[0] = (double)(k + 1);
        if (!(r > 1e-13 * fabs(a)) || !(r > 1e-300)) state[1] = 0.0;
    }
}

// v_{k+1} = w / beta_k while the iteration is active
__global__ void __launch_bounds__(RT) lz_scale_kernel(const double* __restrict__ w, double* __restrict__ v,
                                                      int64_t n, const double* __restrict__ state, int k,
                                                      int nmax) {
    if (state[1] == 0.0) return;
    const double inv = 1.0 / state[8 + nmax + k];
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) v[i] = w[i] * inv;
}

// After the first Gram-Schmidt pass of step k: whether the second runs (state[4]), i.e.
// whether the pass left less than half of ||w||^2 (before: wn, nb1 partials; after: sq, nb2
// partials).
__global__ void lz_second_pass_kernel(double* state, const double* __restrict__ wn, int nb1,
                                      const double* __restrict__ sq, int nb2) {
    __shared__ double sh[RT / 32];
    if (state[1] == 0.0) return;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb1; i += blockDim.x) a += wn[i];
    for (int i = threadIdx.x; i < nb2; i += blockDim.x) b += sq[i];
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) state[4] = (b < 0.5 * a) ? 1.0 : 0.0;
}

// alpha_k = a + h1[k] (+ h2[k] when the second pass ran): every projection of H v_k on v_k
__global__ void set_alpha_kernel(double* state, const double* a, const double* h1, const double* h2, int k) {
    if (state[1] == 0.0) return;
    state[8 + k] = *a + h1[k] + (state[4] != 0.0 ? h2[k] : 0.0);
}

// Lowest eigenpair of the n_eff x n_eff tridiagonal matrix T (diagonal alpha, off-diagonal
// beta), in FP64 on one thread: the eigenvalue by bisection on the Sturm count (the number
// of negative pivots of the LDL^T factorisation of T - x I equals the number of
// eigenvalues below x), the eigenvector by inverse iteration with the tridiagonal system
// solved by Gaussian elimination with partial pivoting.  Writes theta to state[2],
// |beta_{n-1} s_{n-1}| (the Lanczos residual norm of the Ritz pair) to state[3], the
// eigenvector to s; T holds 4 * nmax doubles of scratch.
__global__ void tridiag_eig_kernel(double* state, double* T, double* s, int nmax) {
    // one warp: the 32 lanes evaluate Sturm counts at 32 interior points of the bracket
    // (multisection: each step shrinks it 33-fold), then lane 0 runs the inverse iteration
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int n = (int)state[0];
    for (int i = lane; i < nmax; i += 32) s[i] = 0.0;
    __syncwarp();                        // lane 0 writes s below: the zeros land first
    if (n <= 0) {                        // a zero start vector: no Krylov space
        if (lane == 0) { state[2] = 0.0; state[3] = 0.0; }
        return;
    }
    const double* al = state + 8;
    const double* be = state + 8 + nmax;
    double lo = al[0], hi = al[0];
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < n ? fabs(be[i]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
    }
    const double scale = fmax(fabs(lo), fabs(hi)) + 1e-300;
    auto count_below = [&](double x) {
        int c = 0;
        double d = 1.0;
        for (int i = 0; i < n; ++i) {
            const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
            d = (al[i] - x) - (i > 0 ? b2 / d : 0.0);
            if (d == 0.0) d = -1e-300 * scale;
            if (d < 0.0) ++c;
        }
        return c;
    };
    // the lowest eigenvalue stays in (lo, hi]: count_below(lo) = 0, count_below(hi) >= 1
    for (int it = 0; it < 60 && hi - lo > 4e-16 * scale; ++it) {
        const double step = (hi - lo) / 33.0;
        const double x = lane == 31 ? hi - 0.5 * step : lo + (lane + 1) * step;
        const unsigned below = __ballot_sync(0xffffffffu, count_below(x) >= 1);
        const int k = below ? __ffs(below) - 1 : 32;             // first point with an eigenvalue below
        const double xk = __shfl_sync(0xffffffffu, x, k < 32 ? k : 31);
        const double xk1 = __shfl_sync(0xffffffffu, x, k > 0 ? (k < 32 ? k - 1 : 31) : 0);
        if (k < 32) hi = xk;
        if (k > 0) lo = xk1;
    }
    if (lane != 0) return;
    const double theta = 0.5 * (lo + hi);
    // inverse iteration: (T - theta I) z_new = z, banded LU with partial pivoting.  A pivot
    // below tiny (theta is an eigenvalue to rounding, so one pivot is ~0: exactly 0 when
    // n = 1) is replaced by +-tiny, and z is rescaled by its largest entry before it is
    // normalised, so the large solution neither overflows nor turns into NaN.
    const double tiny = 1e-15 * scale;
    auto guard = [&](double v) { return fabs(v) < tiny ? (v < 0.0 ? -tiny : tiny) : v; };
    double* dl = T;              // sub-diagonal / multipliers
    double* dd = T + nmax;       // diagonal
    double* du = T + 2 * nmax;   // first super-diagonal
    double* du2 = T + 3 * nmax;  // second super-diagonal (fill-in from pivoting)
    for (int i = 0; i < n; ++i) s[i] = 1.0 / sqrt((double)n);
    for (int iter = 0; iter < 4; ++iter) {
        for (int i = 0; i < n; ++i) {
            dd[i] = al[i] - theta;
            du[i] = i + 1 < n ? be[i] : 0.0;
            dl[i] = i + 1 < n ? be[i] : 0.0;
            du2[i] = 0.0;
        }
        for (int i = 0; i + 1 < n; ++i) {
            if (fabs(dd[i]) >= fabs(dl[i])) {              // no row swap
                dd[i] = guard(dd[i]);
                const double f = dl[i] / dd[i];
                dl[i] = f;
                dd[i + 1] -= f * du[i];
                s[i + 1] -= f * s[i];
            } else {                                      // swap rows i and i+1
                const double f = dd[i] / dl[i];
                dd[i] = dl[i];
                dl[i] = f;
                const double t = du[i];
                du[i] = dd[i + 1];
                dd[i + 1] = t - f * dd[i + 1];
                if (i + 2 < n) {
                    du2[i] = du[i + 1];
                    du[i + 1] = -f * du[i + 1];
                }
                const double sv = s[i];
                s[i] = s[i + 1];
                s[i + 1] = sv - f * s[i + 1];
            }
        }
        dd[n - 1] = guard(dd[n - 1]);
        // back substitution
        for (int i = n - 1; i >= 0; --i) {
            double v = s[i];
            if (i + 1 < n) v -= du[i] * s[i + 1];
            if (i + 2 < n) v -= du2[i] * s[i + 2];
            s[i] = v / dd[i];
        }
        double mx = 0.0;
        for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(s[i]));
        if (!(mx > 0.0) || !isfinite(mx)) {           // cannot happen with the guards; keep e_0
            for (int i = 0; i < n; ++i) s[i] = i == 0 ? 1.0 : 0.0;
            break;
        }
        double nr = 0.0;
        for (int i = 0; i < n; ++i) { s[i] /= mx; nr += s[i] * s[i]; }
        nr = sqrt(nr);
        for (int i = 0; i < n; ++i) s[i] /= nr;
    }
    // fix the sign (largest component positive) for reproducible Ritz vectors
    int im = 0;
    for (int i = 1; i < n; ++i) if (fabs(s[i]) > fabs(s[im])) im = i;
    if (s[im] < 0) for (int i = 0; i < n; ++i) s[i] = -s[i];
    state[2] = theta;
    state[3] = fabs(be[n - 1] * s[n - 1]);
}

// ---------------------------------------------------------------- Davidson (Algorithm 1)
// State (doubles): [0] vectors in use, [1] active, [2] lambda, [3] ||q||, [4] ||q|| before
// the Gram-Schmidt passes, [5] tol.

// M[i][j] = M[j][i] = h[j], j <= i
__global__ void dav_set_m_kernel(double* M, const double* h, int i, int maxv, const double* state) {
    if (state[1] == 0.0) return;
    for (int j = threadIdx.x; j <= i; j += blockDim.x) {
        M[i * maxv + j] = h[j];
        M[j * maxv + i] = h[j];
    }
}

// Lowest eigenpair of the leading m x m block of the symmetric M (one thread, cyclic
// Jacobi rotations in FP64 until the off-diagonal mass is below 1e-30 of the total):
// lambda -> state[2], eigenvector (largest component positive) -> s.
__global__ void dav_eig_kernel(const double* M, double* E, double* s, double* state, int m, int maxv) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || state[1] == 0.0) return;
    double* A = E;                    // m x m working copy
    double* Q = E + maxv * maxv;      // accumulated rotations
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) {
            A[r * m + c] = M[r * maxv + c];
            Q[r * m + c] = r == c ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) {
                const double v = A[r * m + c] * A[r * m + c];
                tot += v;
                if (r != c) off += v;
            }
        if (!(off > 1e-30 * tot)) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[p * m + q];
                if (apq == 0.0) continue;
                const double zeta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int k = 0; k < m; ++k) {           // columns p, q
                    const double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = c * akp - sn * akq;
                    A[k * m + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {           // rows p, q
                    const double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = c * apk - sn * aqk;
                    A[q * m + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double qkp = Q[k * m + p], qkq = Q[k * m + q];
                    Q[k * m + p] = c * qkp - sn * qkq;
                    Q[k * m + q] = sn * qkp + c * qkq;
                }
            }
    }
    int lo = 0;
    for (int r = 1; r < m; ++r) if (A[r * m + r] < A[lo * m + lo]) lo = r;
    int im = 0;
    for (int r = 1; r < m; ++r) if (fabs(Q[r * m + lo]) > fabs(Q[im * m + lo])) im = r;
    const double sg = Q[im * m + lo] < 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < maxv; ++r) s[r] = r < m ? sg * Q[r * m + lo] : 0.0;
    state[2] = A[lo * m + lo];
    state[0] = (double)m;
}

// q -= lambda x
__global__ void __launch_bounds__(RT) dav_shift_kernel(double* __restrict__ q, const double* __restrict__ x,
                                                       int64_t n, const double* __restrict__ state) {
    if (state[1] == 0.0) return;
    const double lam = state[2];
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) q[i] -= lam * x[i];
}

// ||q|| -> state[3]; stop (active = 0) when ||q|| < tol max(1, |lambda|) or the subspace is
// full, else remember ||q|| in state[4]
__global__ void dav_check_kernel(const double* __restrict__ part, int nb, double* state, int last) {
    __shared__ double sh[RT / 32];
    if (state[1] == 0.0) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b * VT];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        const double r = sqrt(v);
        state[3] = r;
        state[4] = r;
        if (last || !(r >= state[5] * fmax(1.0, fabs(state[2])))) state[1] = 0.0;
    }
}

// Randomisation (Algorithm 1's remedy for a failed reorthogonalisation): if Gram-Schmidt
// left less than 1e-12 of ||q||, replace q by the caller's random vector
__global__ void __launch_bounds__(RT) dav_random_kernel(const double* __restrict__ part, int nb,
                                                        double* __restrict__ q, const double* __restrict__ rnd,
                                                        int64_t n, const double* __restrict__ state) {
    __shared__ double sh[RT / 32];
    __shared__ int swap;
    if (state[1] == 0.0) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b * VT];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) swap = !(sqrt(v) >= 1e-12 * state[4]);
    __syncthreads();
    if (!swap) return;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) q[i] = rnd[i];
}

int grid_for(int64_t n) {
    int64_t g = (n + RT - 1) / RT;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace
}  // namespace heff

using namespace heff;

extern "C" int heff_lanczos_workspace_size(const heff_plan* plan, int32_t n_iter, size_t* bytes) {
    clear_error();
    if (!plan || !bytes || n_iter < 1 || n_iter > 126)
        return fail(HEFF_ERR_INVALID_ARG, "heff_lanczos_workspace_size: bad arguments (n_iter 1..126)");
    *bytes = lz_layout(plan->nelem_x, n_iter).bytes;
    return HEFF_OK;
}

namespace heff {
namespace {

Lz lz_view(const LzLayout& lay, void* lz_ws, int64_t n) {
    char* base = static_cast<char*>(lz_ws);
    return Lz{reinterpret_cast<double*>(base + lay.off_state), reinterpret_cast<double*>(base + lay.off_h),
              reinterpret_cast<double*>(base + lay.off_s), reinterpret_cast<double*>(base + lay.off_part),
              reinterpret_cast<double*>(base + lay.off_wn), reinterpret_cast<double*>(base + lay.off_sq),
              reinterpret_cast<double*>(base + lay.off_a),
              reinterpret_cast<double*>(base + lay.off_T), reinterpret_cast<double*>(base + lay.off_V), n,
              lay.nmax};
}

// n_iter Lanczos steps from x0 on operators already prepared in apply_ws; x0 may alias x_out
// (it is only read into the first basis vector).
int lanczos_core(heff_plan* plan, const double* x0, int32_t n_iter, double* x_out, double* result,
                 void* apply_ws, size_t apply_ws_bytes, const Lz& z, cudaStream_t st) {
    void* stream = st;
    const int64_t n = z.n;
    const int G = grid_for(n);
    const int GN = G < 1024 ? G : 1024;      // normalize: every block re-sums the RB partials
    int rc;
    // v_0 = x0 / ||x0||
    sumsq_kernel<<<RB, RT, 0, st>>>(x0, n, z.part);
    normalize_kernel<<<GN, RT, 0, st>>>(z.part, RB, x0, z.V, n, z.state, 0);
    count_launches(2);
    for (int k = 0; k < n_iter; ++k) {
        double* vk = z.V + (int64_t)k * n;
        // w = H v_k (skipped work is harmless after breakdown: the result is not used)
        if ((rc = heff_apply_prepared(plan, vk, z.w(), apply_ws, apply_ws_bytes, stream))) return rc;
        // three-term recurrence: a -> z.a, w -= beta_{k-1} v_{k-1} + a v_k
        three_term_kernel<<<RB, RT, 0, st>>>(z.V, z.w(), n, k, z.nmax, z.part, z.wn, z.state, z.a, 0);
        finish_dots_kernel<<<1, RT, 0, st>>>(z.part, RB, 0, 1, z.a, 0, z.state);
        three_term_kernel<<<RB, RT, 0, st>>>(z.V, z.w(), n, k, z.nmax, z.part, z.wn, z.state, z.a, 1);
        count_launches(3);
        // classical Gram-Schmidt: h1 -> z.h, then (when needed) h2 -> z.s; each combine also
        // leaves the partial sums of ||w||^2 in z.sq for the test and the normalisation
        for (int pass = 0; pass < 2; ++pass) {
            double* hp = pass == 0 ? z.h : z.s;
            multidot_all_kernel<<<dim3(RB, (k + VT) / VT), RT, 0, st>>>(z.V, z.w(), n, k + 1, z.part, z.state,
                                                                         pass);
            vec_finish_kernel<<<k + 1, RT, 0, st>>>(z.part, RB, hp, z.state, pass);
            combine_kernel<<<G, RT, 0, st>>>(z.V, n, k + 1, hp, -1.0, 1.0, z.w(), z.state, 0, pass, z.sq);
            count_launches(3);
            if (pass == 0) {
                lz_second_pass_kernel<<<1, RT, 0, st>>>(z.state, z.wn, RB, z.sq, G);
                count_launches(1);
            }
        }
        set_alpha_kernel<<<1, 1, 0, st>>>(z.state, z.a, z.h, z.s, k);
        lz_beta_kernel<<<1, RT, 0, st>>>(z.sq, G, z.state, k, z.nmax);
        lz_scale_kernel<<<G, RT, 0, st>>>(z.w(), z.V + (int64_t)(k + 1) * n, n, z.state, k, z.nmax);
        count_launches(3);
    }
    tridiag_eig_kernel<<<1, 32, 0, st>>>(z.state, z.T, z.s, z.nmax);
    // x = V s (rows beyond n_eff have s = 0), then normalise
    combine_kernel<<<G, RT, 0, st>>>(z.V, n, z.nmax, z.s, 1.0, 0.0, x_out, z.state, 1, 0, nullptr, 1);
    sumsq_kernel<<<RB, RT, 0, st>>>(x_out, n, z.part);
    normalize_kernel<<<GN, RT, 0, st>>>(z.part, RB, x_out, x_out, n, z.state, 2);
    count_launches(4);
    // result: [theta, residual estimate, n_eff, alpha..., beta...]
    cudaMemcpyAsync(result, z.state + 2, sizeof(double) * 2, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(result + 2, z.state, sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(result + 3, z.state + 8, sizeof(double) * 2 * z.nmax, cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_lanczos: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

}  // namespace
}  // namespace heff

extern "C" int heff_lanczos(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                            const double* x0, int32_t n_iter, double* x_out, double* result,
                            void* apply_ws, size_t apply_ws_bytes, void* lz_ws, size_t lz_ws_bytes,
                            void* stream) {
    clear_error();
    if (!plan || !L || !W1 || !W2 || !R || !x0 || !x_out || !result || !lz_ws)
        return fail(HEFF_ERR_INVALID_ARG, "heff_lanczos: null argument");
    if (plan->opts.io_dtype != HEFF_DTYPE_F64)
        return fail(HEFF_ERR_UNSUPPORTED, "heff_lanczos needs a plan with HEFF_DTYPE_F64 tensors");
    if (n_iter < 1 || n_iter > 126) return fail(HEFF_ERR_INVALID_ARG, "n_iter must be 1..126");
    if (plan->nelem_x == 0) return fail(HEFF_ERR_INVALID_ARG, "heff_lanczos: the two-site space is empty");
    const LzLayout lay = lz_layout(plan->nelem_x, n_iter);
    if (lz_ws_bytes < lay.bytes || reinterpret_cast<uintptr_t>(lz_ws) % 256)
        return fail(HEFF_ERR_WORKSPACE, "Lanczos workspace of %zu bytes, needs %zu (256-byte aligned)",
                    lz_ws_bytes, lay.bytes);
    int rc = heff_prepare(plan, L, W1, W2, R, apply_ws, apply_ws_bytes, stream);
    if (rc) return rc;
    return lanczos_core(plan, x0, n_iter, x_out, result, apply_ws, apply_ws_bytes,
                        lz_view(lay, lz_ws, plan->nelem_x), static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------- ground state to a tolerance
namespace heff {
namespace {

// part[b] = sum over block b's chunk of x[i] * y[i]  (mode 0), or of (y[i] - E x[i])^2 with
// E = *e_dev (mode 1); two-stage with a fixed order, like the Lanczos reductions
__global__ void __launch_bounds__(RT) rq_part_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                     int64_t n, const double* __restrict__ e_dev, int mode,
                                                     double* __restrict__ part) {
    __shared__ double sh[RT / 32];
    const double E = mode ? *e_dev : 0.0;
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        if (mode == 0) {
            a = fma(x[i], y[i], a);
        } else {
            const double r = y[i] - E * x[i];
            a = fma(r, r, a);
        }
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void rq_finish_kernel(const double* __restrict__ part, int nb, double* out) {
    __shared__ double sh[RT / 32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) *out = v;
}

// ground-state workspace: the Lanczos workspace, then the cycle's result and 4 scalars
size_t gs_result_off(const LzLayout& lay) { return lay.bytes; }
size_t gs_bytes(const LzLayout& lay) {
    return lay.bytes + (sizeof(double) * (3 + 2 * (size_t)lay.nmax + 8) + 255) / 256 * 256;
}

}  // namespace
}  // namespace heff

extern "C" int heff_ground_state_workspace_size(const heff_plan* plan, int32_t n_iter, size_t* bytes) {
    clear_error();
    if (!plan || !bytes || n_iter < 1 || n_iter > 126)
        return fail(HEFF_ERR_INVALID_ARG, "heff_ground_state_workspace_size: bad arguments (n_iter 1..126)");
    *bytes = gs_bytes(lz_layout(plan->nelem_x, n_iter));
    return HEFF_OK;
}

extern "C" int heff_ground_state(heff_plan* plan, heff_plan* plan64, const void* L, const void* W1,
                                 const void* W2, const void* R, const double* x0, int32_t n_iter,
                                 int32_t max_cycles, double tol, double* x_out, double* result,
                                 void* apply_ws, size_t apply_ws_bytes, void* apply_ws64, size_t apply_ws64_bytes,
                                 void* gs_ws, size_t gs_ws_bytes, void* stream) {
    clear_error();
    if (!plan || !L || !W1 || !W2 || !R || !x0 || !x_out || !result || !gs_ws)
        return fail(HEFF_ERR_INVALID_ARG, "heff_ground_state: null argument");
    if (plan->opts.io_dtype != HEFF_DTYPE_F64)
        return fail(HEFF_ERR_UNSUPPORTED, "heff_ground_state needs a plan with HEFF_DTYPE_F64 tensors");
    if (n_iter < 1 || n_iter > 126 || max_cycles < 1 || !(tol >= 0.0))
        return fail(HEFF_ERR_INVALID_ARG, "heff_ground_state: n_iter 1..126, max_cycles >= 1, tol >= 0");
    if (plan->nelem_x == 0) return fail(HEFF_ERR_INVALID_ARG, "heff_ground_state: the two-site space is empty");
    // the FP64 Rayleigh quotient: plan64, or the plan itself when it is the FP64 path
    heff_plan* p64 = plan64 ? plan64 : (plan->opts.precision == HEFF_PREC_FP64 ? plan : nullptr);
    void* ws64 = plan64 ? apply_ws64 : apply_ws;
    const size_t ws64_bytes = plan64 ? apply_ws64_bytes : apply_ws_bytes;
    if (p64) {
        if (p64->opts.precision != HEFF_PREC_FP64 || p64->opts.io_dtype != HEFF_DTYPE_F64 ||
            p64->nelem_x != plan->nelem_x)
            return fail(HEFF_ERR_INVALID_ARG, "heff_ground_state: plan64 must be an FP64 plan of the same layouts");
        if (plan64 && !apply_ws64) return fail(HEFF_ERR_INVALID_ARG, "heff_ground_state: null apply_ws64");
    }
    const LzLayout lay = lz_layout(plan->nelem_x, n_iter);
    if (gs_ws_bytes < gs_bytes(lay) || reinterpret_cast<uintptr_t>(gs_ws) % 256)
        return fail(HEFF_ERR_WORKSPACE, "ground-state workspace of %zu bytes, needs %zu (256-byte aligned)",
                    gs_ws_bytes, gs_bytes(lay));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Lz z = lz_view(lay, gs_ws, plan->nelem_x);
    double* res = reinterpret_cast<double*>(static_cast<char*>(gs_ws) + gs_result_off(lay));
    double* scal = res + 3 + 2 * lay.nmax;          // [0] x.y, [1] |y - E x|^2
    int rc = heff_prepare(plan, L, W1, W2, R, apply_ws, apply_ws_bytes, stream);
    if (rc) return rc;
    double theta = 0.0, est = 0.0;
    int cycles = 0;
    const double* start = x0;
    for (; cycles < max_cycles;) {
        if ((rc = lanczos_core(plan, start, n_iter, x_out, res, apply_ws, apply_ws_bytes, z, st))) return rc;
        ++cycles;
        start = x_out;                                // the next cycle restarts from the Ritz vector
        double h[2];
        cudaError_t e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_ground_state: %s", cudaGetErrorString(e));
        theta = h[0];
        est = h[1] / (fabs(theta) > 0.0 ? fabs(theta) : 1.0);
        if (!(est > tol)) break;
    }
    result[0] = theta;
    result[1] = theta;
    result[2] = est;
    result[3] = cycles;
    result[4] = (double)cycles * n_iter;
    result[5] = -1.0;
    if (p64) {
        // E = <x|K|x> (x is normalised) with an FP64 apply, and ||K x - E x|| / |E|
        if (p64 != plan && (rc = heff_prepare(p64, L, W1, W2, R, ws64, ws64_bytes, stream))) return rc;
        double* y = z.w();
        if ((rc = heff_apply_prepared(p64, x_out, y, ws64, ws64_bytes, stream))) return rc;
        const int64_t n = z.n;
        rq_part_kernel<<<RB, RT, 0, st>>>(x_out, y, n, nullptr, 0, z.part);
        rq_finish_kernel<<<1, RT, 0, st>>>(z.part, RB, scal);
        rq_part_kernel<<<RB, RT, 0, st>>>(x_out, y, n, scal, 1, z.part);
        rq_finish_kernel<<<1, RT, 0, st>>>(z.part, RB, scal + 1);
        count_launches(4);
        double h[2];
        cudaError_t e = cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_ground_state: %s", cudaGetErrorString(e));
        result[0] = h[0];
        result[5] = sqrt(h[1]) / (fabs(h[0]) > 0.0 ? fabs(h[0]) : 1.0);
    }
    return HEFF_OK;
}

// ---------------------------------------------------------------- Davidson host side
namespace heff {
namespace {

struct DavLayout {
    int maxv;
    size_t off_state, off_M, off_E, off_s, off_h, off_part, off_V, off_VA, off_q, bytes;
};

DavLayout dav_layout(int64_t n, int maxv) {
    DavLayout l{};
    l.maxv = maxv;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t o = 0;
    l.off_state = o; o = al(o + sizeof(double) * 16);
    l.off_M = o;     o = al(o + sizeof(double) * (size_t)maxv * maxv);
    l.off_E = o;     o = al(o + sizeof(double) * 2 * (size_t)maxv * maxv);
    l.off_s = o;     o = al(o + sizeof(double) * (size_t)maxv);
    l.off_h = o;     o = al(o + sizeof(double) * (size_t)maxv);
    l.off_part = o;  o = al(o + sizeof(double) * (size_t)RB * VT);
    l.off_V = o;     o = al(o + sizeof(double) * (size_t)maxv * (size_t)n);
    l.off_VA = o;    o = al(o + sizeof(double) * (size_t)maxv * (size_t)n);
    l.off_q = o;     o = al(o + sizeof(double) * (size_t)n);
    l.bytes = o;
    return l;
}

__global__ void dav_init_state_kernel(double* state, double tol) {
    if (threadIdx.x == 0) state[5] = tol;
}

}  // namespace
}  // namespace heff

extern "C" int heff_davidson_workspace_size(const heff_plan* plan, int32_t max_vecs, size_t* bytes) {
    clear_error();
    if (!plan || !bytes || max_vecs < 1 || max_vecs > 64)
        return fail(HEFF_ERR_INVALID_ARG, "heff_davidson_workspace_size: bad arguments (max_vecs 1..64)");
    *bytes = dav_layout(plan->nelem_x, max_vecs).bytes;
    return HEFF_OK;
}

extern "C" int heff_davidson(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                             const double* x0, const double* rnd, int32_t max_vecs, double tol, double* x_out,
                             double* result, void* apply_ws, size_t apply_ws_bytes, void* dav_ws,
                             size_t dav_ws_bytes, void* stream) {
    clear_error();
    if (!plan || !L || !W1 || !W2 || !R || !x0 || !rnd || !x_out || !result || !dav_ws)
        return fail(HEFF_ERR_INVALID_ARG, "heff_davidson: null argument");
    if (plan->opts.io_dtype != HEFF_DTYPE_F64)
        return fail(HEFF_ERR_UNSUPPORTED, "heff_davidson needs a plan with HEFF_DTYPE_F64 tensors");
    if (max_vecs < 1 || max_vecs > 64) return fail(HEFF_ERR_INVALID_ARG, "max_vecs must be 1..64");
    if (plan->nelem_x == 0) return fail(HEFF_ERR_INVALID_ARG, "heff_davidson: the two-site space is empty");
    if (!(tol >= 0.0)) return fail(HEFF_ERR_INVALID_ARG, "tol must be >= 0");
    const DavLayout lay = dav_layout(plan->nelem_x, max_vecs);
    if (dav_ws_bytes < lay.bytes || reinterpret_cast<uintptr_t>(dav_ws) % 256)
        return fail(HEFF_ERR_WORKSPACE, "Davidson workspace of %zu bytes, needs %zu (256-byte aligned)",
                    dav_ws_bytes, lay.bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(dav_ws);
    double* state = reinterpret_cast<double*>(base + lay.off_state);
    double* M = reinterpret_cast<double*>(base + lay.off_M);
    double* E = reinterpret_cast<double*>(base + lay.off_E);
    double* s = reinterpret_cast<double*>(base + lay.off_s);
    double* h = reinterpret_cast<double*>(base + lay.off_h);
    double* part = reinterpret_cast<double*>(base + lay.off_part);
    double* V = reinterpret_cast<double*>(base + lay.off_V);
    double* VA = reinterpret_cast<double*>(base + lay.off_VA);
    double* q = reinterpret_cast<double*>(base + lay.off_q);
    const int64_t n = plan->nelem_x;
    const int G = grid_for(n);
    const int GN = G < 1024 ? G : 1024;      // normalize: every block re-sums the RB partials
    int rc = heff_prepare(plan, L, W1, W2, R, apply_ws, apply_ws_bytes, stream);
    if (rc) return rc;
    dav_init_state_kernel<<<1, 32, 0, st>>>(state, tol);
    // v_0 = x0 / ||x0|| (sets active when x0 != 0), v^A_0 = A v_0
    sumsq_kernel<<<RB, RT, 0, st>>>(x0, n, part);
    normalize_kernel<<<GN, RT, 0, st>>>(part, RB, x0, V, n, state, 0);
    count_launches(3);
    if ((rc = heff_apply_prepared(plan, V, VA, apply_ws, apply_ws_bytes, stream))) return rc;
    auto gram_schmidt = [&](int nv) {          // q -= V (V^T q) over v_0 .. v_{nv-1}
        for (int j0 = 0; j0 < nv; j0 += VT) {
            const int k = nv - j0 < VT ? nv - j0 : VT;
            multidot_kernel<<<RB, RT, 0, st>>>(V, q, n, j0, k, part, state);
            finish_dots_kernel<<<1, RT, 0, st>>>(part, RB, j0, k, h, 0, state);
            count_launches(2);
        }
        combine_kernel<<<G, RT, 0, st>>>(V, n, nv, h, -1.0, 1.0, q, state, 0);
        count_launches(1);
    };
    for (int i = 0; i < max_vecs; ++i) {
        double* vi = V + (int64_t)i * n;
        // m_ij = (v^A_j)^T v_i, j <= i
        for (int j0 = 0; j0 <= i; j0 += VT) {
            const int k = i + 1 - j0 < VT ? i + 1 - j0 : VT;
            multidot_kernel<<<RB, RT, 0, st>>>(VA, vi, n, j0, k, part, state);
            finish_dots_kernel<<<1, RT, 0, st>>>(part, RB, j0, k, h, 0, state);
            count_launches(2);
        }
        dav_set_m_kernel<<<1, 64, 0, st>>>(M, h, i, max_vecs, state);
        dav_eig_kernel<<<1, 32, 0, st>>>(M, E, s, state, i + 1, max_vecs);
        // x = V s, q = V^A s - lambda x, ||q||
        combine_kernel<<<G, RT, 0, st>>>(V, n, i + 1, s, 1.0, 0.0, x_out, state, 0);
        combine_kernel<<<G, RT, 0, st>>>(VA, n, i + 1, s, 1.0, 0.0, q, state, 0);
        dav_shift_kernel<<<G, RT, 0, st>>>(q, x_out, n, state);
        sumsq_kernel<<<RB, RT, 0, st>>>(q, n, part);
        dav_check_kernel<<<1, RT, 0, st>>>(part, RB, state, i + 1 == max_vecs);
        count_launches(7);
        if (i + 1 == max_vecs) break;
        // orthogonalise q against v_0..v_i (two classical Gram-Schmidt passes), randomise if
        // nothing is left, orthogonalise again, normalise into v_{i+1}, v^A_{i+1} = A v_{i+1}
        gram_schmidt(i + 1);
        gram_schmidt(i + 1);
        sumsq_kernel<<<RB, RT, 0, st>>>(q, n, part);
        dav_random_kernel<<<G, RT, 0, st>>>(part, RB, q, rnd, n, state);
        count_launches(2);
        gram_schmidt(i + 1);
        gram_schmidt(i + 1);
        double* vn = V + (int64_t)(i + 1) * n;
        sumsq_kernel<<<RB, RT, 0, st>>>(q, n, part);
        normalize_kernel<<<GN, RT, 0, st>>>(part, RB, q, vn, n, state, 3);
        count_launches(2);
        if ((rc = heff_apply_prepared(plan, vn, VA + (int64_t)(i + 1) * n, apply_ws, apply_ws_bytes, stream)))
            return rc;
    }
    sumsq_kernel<<<RB, RT, 0, st>>>(x_out, n, part);
    normalize_kernel<<<GN, RT, 0, st>>>(part, RB, x_out, x_out, n, state, 2);
    count_launches(2);
    // result: [lambda, ||q||, vectors used]
    cudaMemcpyAsync(result, state + 2, sizeof(double) * 2, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(result + 2, state, sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_davidson: %s", cudaGetErrorString(e));
    return HEFF_OK;
}
