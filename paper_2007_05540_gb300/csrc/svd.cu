// Block SVD split of the two-site tensor with truncation, FP64 on the GPU (Section IV:
// the tensor is "wrapped" into a matrix with rows (a, s1) and columns (s2, b), one dense
// block per charge Q; Fig. 1e: the factors are split and the singular values absorbed in
// the sweep direction; Section II-C: singular values below a cutoff are removed).
//
// Each charge block M_Q (rows (s1, i, a), columns (s2, j, b)) is decomposed by one-sided
// Jacobi rotations (Hestenes): the columns of J = M_Q (or M_Q^T when M_Q is wide) are made
// mutually orthogonal by plane rotations applied in a round-robin order, so every round
// rotates k/2 disjoint column pairs in parallel (one warp per pair, all sectors in one
// launch); V accumulates the rotations.  On convergence the column norms are the singular
// values.  The truncation rule runs on the host on the singular values; the kept singular
// triplets are then written into the caller's left (a, s1, c) and right (c, s2, b) tensors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <tuple>

#include "internal.h"

using heff::fail;

namespace {

struct SvdSector {           // device-side description of one charge block
    int64_t j_off, v_off;    // column-major J (r x k) and V (k x k) in the workspace
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
    size_t ws_bytes = 0;
    int64_t s_total = 0;
    std::vector<double> s;                     // singular values (per sector, unsorted)
    std::vector<std::vector<int32_t>> kept;    // per sector: kept column indices of J, s descending
    double norm = 0, discarded = 0;
    SvdSector* d_sec = nullptr;
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

__global__ void svd_init_v_kernel(const SvdSector* __restrict__ secs, double* __restrict__ ws) {
    const SvdSector s = secs[blockIdx.y];
    double* V = ws + s.v_off;
    const int64_t n = (int64_t)s.k * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        V[e] = (e % (s.k + 1) == 0) ? 1.0 : 0.0;
}

// one round of the round-robin ordering: warp w of the launch rotates pair i of sector y
__global__ void __launch_bounds__(128) svd_round_kernel(const SvdSector* __restrict__ secs, double* __restrict__ ws,
                                                        int round, unsigned int* __restrict__ off_max) {
    const SvdSector s = secs[blockIdx.y];
    const int kk = s.k + (s.k & 1);                   // padded to even (dummy column = k)
    if (kk < 2 || round >= kk - 1) return;
    const int pair = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (pair >= kk / 2) return;
    auto pos = [&](int j) { return j == 0 ? 0 : 1 + (j - 1 + round) % (kk - 1); };
    int p = pos(pair), q = pos(kk - 1 - pair);
    if (p >= s.k || q >= s.k) return;                 // pair with the dummy column
    if (p > q) { const int t = p; p = q; q = t; }
    double* J = ws + s.j_off;
    double* cp = J + (int64_t)p * s.r;
    double* cq = J + (int64_t)q * s.r;
    double a = 0, b = 0, g = 0;
    for (int i = lane; i < s.r; i += 32) {
        const double u = cp[i], v = cq[i];
        a = fma(u, u, a);
        b = fma(v, v, b);
        g = fma(u, v, g);
    }
    a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
    if (g == 0.0 || a == 0.0 || b == 0.0) return;
    const double meas = fabs(g) / sqrt(a * b);
    if (lane == 0) atomicMax(off_max, __float_as_uint((float)meas));
    if (meas < 1e-15) return;
    const double zeta = (b - a) / (2.0 * g);
    const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
    for (int i = lane; i < s.r; i += 32) {
        const double u = cp[i], v = cq[i];
        cp[i] = c * u - sn * v;
        cq[i] = sn * u + c * v;
    }
    double* V = ws + s.v_off;
    double* vp = V + (int64_t)p * s.k;
    double* vq = V + (int64_t)q * s.k;
    for (int i = lane; i < s.k; i += 32) {
        const double u = vp[i], v = vq[i];
        vp[i] = c * u - sn * v;
        vq[i] = sn * u + c * v;
    }
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

}  // namespace

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
        int64_t o = 0, so = 0;
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
            sc.s_off = (int32_t)so; so += sc.k;
            S->sec.push_back(sc);
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
        S->ws_bytes = (size_t)S->ws_doubles * sizeof(double) + tab.size() * sizeof(int64_t) + 1024;
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
    unsigned int* offmax = reinterpret_cast<unsigned int*>(ws + S->ws_doubles - 8);
    const std::vector<int64_t>& tab = S->xoff[0];
    int64_t* d_tab = reinterpret_cast<int64_t*>(ws + S->ws_doubles);
    const int nsec = (int)S->sec.size();
    if (!S->d_sec) SVD_CK(cudaMalloc((void**)&S->d_sec, std::max<size_t>(1, S->sec.size()) * sizeof(SvdSector)));
    SVD_CK(cudaMemcpyAsync(S->d_sec, S->sec.data(), S->sec.size() * sizeof(SvdSector), cudaMemcpyHostToDevice, st));
    SVD_CK(cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    const int ntab = (int)(tab.size() / 6);
    if (ntab) svd_load_kernel<<<std::min(ntab, 4096), 256, 0, st>>>(S->d_sec, d_tab, ntab, x, ws);
    svd_init_v_kernel<<<dim3(64, nsec), 256, 0, st>>>(S->d_sec, ws);
    heff::count_launches(2);
    const int kk = S->max_k + (S->max_k & 1);
    const int gx = (kk / 2 + 3) / 4;
    int sweep = 0;
    for (; sweep < 40 && kk >= 2; ++sweep) {
        SVD_CK(cudaMemsetAsync(offmax, 0, sizeof(unsigned int), st));
        for (int r = 0; r < kk - 1; ++r)
            svd_round_kernel<<<dim3(std::max(gx, 1), nsec), 128, 0, st>>>(S->d_sec, ws, r, offmax);
        heff::count_launches(kk - 1);
        unsigned int h = 0;
        SVD_CK(cudaMemcpyAsync(&h, offmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        SVD_CK(cudaStreamSynchronize(st));
        float m;
        std::memcpy(&m, &h, sizeof(float));
        if (m < 1e-14f) { ++sweep; break; }
    }
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
    // tables after the load table in the workspace tail
    char* tail = reinterpret_cast<char*>(ws + S->ws_doubles) + S->xoff[0].size() * sizeof(int64_t);
    // the write tables need their own room: use a temporary device buffer owned by the plan
    WriteEntry* d_ent = nullptr;
    int32_t* d_kept = nullptr;
    (void)tail;
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
    delete S;
}
