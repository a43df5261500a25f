// Gradients of the Rayleigh quotient rho = <x|K|x> / <x|x> of the two-site effective
// Hamiltonian K (Section II-C), in FP64 on the block-product engine.  With n = <x|x>,
// y = K x (computed by heff_apply on the caller's plan, any precision):
//   d rho / d x = 2 (y - rho x) / n
//   U[a', (t1 t2 wr), b]  = sum_b' x[a',t1,t2,b'] R[b',wr,b]
//   T1[a', (wl s1 s2), b] = sum_a  L[a',wl,a] x[a,s1,s2,b]
//   W12[wl,t1,t2,s1,s2,wr] = sum_wm W1[wl,t1,s1,wm] W2[wm,t2,s2,wr]
//   d rho / d L[a',wl,a]  = sum W12 U[a',(t1 t2 wr),b] x[a,s1,s2,b] / n
//   d rho / d R[b',wr,b]  = sum W12 x[a',t1,t2,b'] T1[a',(wl s1 s2),b] / n
//   G[wl,t1,t2,s1,s2,wr]  = sum <T1[.,(wl s1 s2),.], U[.,(t1 t2 wr),.]> / n
//   d rho / d W1 = sum_{t2,s2,wr} G W2,  d rho / d W2 = sum_{wl,t1,s1} G W1
// rho is linear in L, R, W1 and W2, so these are exact closed forms (no linearisation).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>

#include "internal.h"

using heff::BDot;
using heff::BList;
using heff::BProd;
using heff::fail;

// One chunk of consecutive left sectors a' of x: its U and T1 blocks are formed, consumed
// (dL of those sectors completely, dR and G partially) and discarded before the next
// chunk, so the intermediates are never held whole when a workspace limit is set.
struct GradChunk {
    BList U, T1, dL, dR;
    std::vector<BDot> gdots;
    std::vector<int32_t> goff;        // CSR over dense G indices
    int64_t t_base = 0;               // T1 offset within the shared intermediate region
    BDot* d_gdots = nullptr;
    int32_t* d_goff = nullptr;
};

struct heff_grad_plan {
    std::vector<GradChunk> chunks;
    std::vector<BDot> xdots;          // chunks of x for <x, x> and <x, y>
    std::vector<int32_t> xoff;
    std::vector<int32_t> w12_off;     // CSR over dense W12 indices: pairs (W1 idx, W2 idx)
    std::vector<int32_t> w12_terms;
    std::vector<int32_t> dw1_off, dw1_terms;   // per W1 entry: pairs (G idx, W2 idx)
    std::vector<int32_t> dw2_off, dw2_terms;   // per W2 entry: pairs (G idx, W1 idx)
    int64_t nx = 0, nR = 0, nW1 = 0, nW2 = 0, ng = 0;
    int64_t off_U = 0, off_W12 = 0, off_G = 0, off_sc = 0, off_part = 0, off_flag = 0;
    size_t ws_bytes = 0;              // for the current precision
    size_t ws_bytes_fp64 = 0, ws_bytes_tc = 0;
    // tensor-core precision: FP32 copies of x, L and R after the FP64 part (double offsets)
    int64_t nL = 0, off_x32 = 0, off_L32 = 0, off_R32 = 0;
    int precision = HEFF_PREC_FP64;   // of the block products (U, T1, dL, dR)
    int64_t npart = 0;
    // device copies
    BDot* d_xdots = nullptr; int32_t* d_xoff = nullptr;
    int32_t *d_w12_off = nullptr, *d_w12_terms = nullptr;
    int32_t *d_dw1_off = nullptr, *d_dw1_terms = nullptr, *d_dw2_off = nullptr, *d_dw2_terms = nullptr;
    bool uploaded = false;
};

namespace {

// out[e] = sum over pairs (i, j) in [off[e], off[e+1]) of a[i] * b[j]
__global__ void pair_sum_kernel(const int32_t* __restrict__ off, const int32_t* __restrict__ terms,
                                const double* __restrict__ a, const double* __restrict__ b,
                                double* __restrict__ out, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = off[e]; t < off[e + 1]; ++t) s += a[terms[2 * t]] * b[terms[2 * t + 1]];
        out[e] = s;
    }
}

// sc = [n, <x,y>, rho]
__global__ void rho_kernel(double* sc) { sc[2] = sc[1] / sc[0]; }

__global__ void div_kernel(double* __restrict__ v, int64_t n, const double* __restrict__ sc) {
    const double inv = 1.0 / sc[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] *= inv;
}

__global__ void dx_kernel(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ sc,
                          double* __restrict__ dx, int64_t n) {
    const double nn = sc[0], rho = sc[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dx[i] = 2.0 * (y[i] - rho * x[i]) / nn;
}

template <typename T>
int up(const std::vector<T>& v, T** d) {
    *d = nullptr;
    if (v.empty()) return HEFF_OK;
    if (cudaMalloc((void**)d, v.size() * sizeof(T)) != cudaSuccess ||
        cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(HEFF_ERR_CUDA, "gradient table upload failed");
    return HEFF_OK;
}

void free_all(heff_grad_plan* g) {
    for (GradChunk& c : g->chunks) {
        heff::blist_free(c.U); heff::blist_free(c.T1); heff::blist_free(c.dL); heff::blist_free(c.dR);
        cudaFree(c.d_gdots); cudaFree(c.d_goff);
        c.d_gdots = nullptr; c.d_goff = nullptr;
    }
    cudaFree(g->d_xdots); cudaFree(g->d_xoff);
    cudaFree(g->d_w12_off); cudaFree(g->d_w12_terms);
    cudaFree(g->d_dw1_off); cudaFree(g->d_dw1_terms); cudaFree(g->d_dw2_off); cudaFree(g->d_dw2_terms);
}

}  // namespace

extern "C" int heff_grad_plan_create(const heff_layout* L, const heff_layout* W1, const heff_layout* W2,
                                     const heff_layout* R, const heff_layout* x, const double* W1_host,
                                     const double* W2_host, size_t ws_limit, heff_grad_plan** out) {
    heff::clear_error();
    if (!L || !W1 || !W2 || !R || !x || !W1_host || !W2_host || !out)
        return fail(HEFF_ERR_INVALID_ARG, "heff_grad_plan_create: null argument");
    *out = nullptr;
    if (x->idx.size() != 4 || L->idx.size() != 3 || R->idx.size() != 3 || W1->idx.size() != 4 || W2->idx.size() != 4)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "tensor orders must be x:4 L:3 R:3 W1:4 W2:4");
    const heff::IndexDesc &alpha = x->idx[0], &beta = x->idx[3];
    if (!L->idx[0].same_sectors(alpha) || !L->idx[2].same_sectors(alpha) || !R->idx[0].same_sectors(beta) ||
        !R->idx[2].same_sectors(beta))
        return fail(HEFF_ERR_CHARGE_MISMATCH, "L and R must live on x's left and right bonds");
    heff_grad_plan* g = new (std::nothrow) heff_grad_plan();
    if (!g) return fail(HEFF_ERR_OOM, "out of host memory");
    try {
        const int kl = W1->idx[0].nsec, km = W1->idx[3].nsec, kr = W2->idx[3].nsec;
        const int d1 = x->idx[1].nsec, d2 = x->idx[2].nsec;
        auto gidx = [&](int wl, int t1, int t2, int s1, int s2, int wr) -> int64_t {
            return ((((((int64_t)wl * d1 + t1) * d2 + t2) * d1 + s1) * d2 + s2) * kr + wr);
        };
        g->ng = (int64_t)kl * d1 * d2 * d1 * d2 * kr;
        g->nx = x->nelem; g->nW1 = W1->nelem; g->nW2 = W2->nelem;
        // W12 pairs (structural, from nonzero host entries)
        std::vector<std::vector<std::pair<int32_t, int32_t>>> w12(g->ng);
        for (size_t e1 = 0; e1 < W1->offsets.size(); ++e1) {
            if (W1_host[W1->offsets[e1]] == 0.0) continue;
            const int wl = W1->keys[e1 * 4], t1 = W1->keys[e1 * 4 + 1], s1 = W1->keys[e1 * 4 + 2], wm = W1->keys[e1 * 4 + 3];
            for (size_t e2 = 0; e2 < W2->offsets.size(); ++e2) {
                if (W2->keys[e2 * 4] != wm || W2_host[W2->offsets[e2]] == 0.0) continue;
                const int t2 = W2->keys[e2 * 4 + 1], s2 = W2->keys[e2 * 4 + 2], wr = W2->keys[e2 * 4 + 3];
                w12[gidx(wl, t1, t2, s1, s2, wr)].push_back({(int32_t)W1->offsets[e1], (int32_t)W2->offsets[e2]});
            }
        }
        g->w12_off.push_back(0);
        for (auto& v : w12) {
            for (auto& p : v) { g->w12_terms.push_back(p.first); g->w12_terms.push_back(p.second); }
            g->w12_off.push_back((int32_t)(g->w12_terms.size() / 2));
        }
        // dW1 / dW2 contraction terms over every allowed W entry
        g->dw1_off.push_back(0);
        for (size_t e1 = 0; e1 < W1->offsets.size(); ++e1) {
            const int wl = W1->keys[e1 * 4], t1 = W1->keys[e1 * 4 + 1], s1 = W1->keys[e1 * 4 + 2], wm = W1->keys[e1 * 4 + 3];
            for (size_t e2 = 0; e2 < W2->offsets.size(); ++e2) {
                if (W2->keys[e2 * 4] != wm) continue;
                const int t2 = W2->keys[e2 * 4 + 1], s2 = W2->keys[e2 * 4 + 2], wr = W2->keys[e2 * 4 + 3];
                g->dw1_terms.push_back((int32_t)gidx(wl, t1, t2, s1, s2, wr));
                g->dw1_terms.push_back((int32_t)W2->offsets[e2]);
            }
            g->dw1_off.push_back((int32_t)(g->dw1_terms.size() / 2));
        }
        g->dw2_off.push_back(0);
        for (size_t e2 = 0; e2 < W2->offsets.size(); ++e2) {
            const int wm = W2->keys[e2 * 4], t2 = W2->keys[e2 * 4 + 1], s2 = W2->keys[e2 * 4 + 2], wr = W2->keys[e2 * 4 + 3];
            for (size_t e1 = 0; e1 < W1->offsets.size(); ++e1) {
                if (W1->keys[e1 * 4 + 3] != wm) continue;
                const int wl = W1->keys[e1 * 4], t1 = W1->keys[e1 * 4 + 1], s1 = W1->keys[e1 * 4 + 2];
                g->dw2_terms.push_back((int32_t)gidx(wl, t1, t2, s1, s2, wr));
                g->dw2_terms.push_back((int32_t)W1->offsets[e1]);
            }
            g->dw2_off.push_back((int32_t)(g->dw2_terms.size() / 2));
        }
        // x blocks by (a sector) and (b sector)
        std::map<int, std::vector<size_t>> x_by_a, x_by_b;
        for (size_t b = 0; b < x->offsets.size(); ++b) {
            x_by_a[x->keys[b * 4]].push_back(b);
            x_by_b[x->keys[b * 4 + 3]].push_back(b);
        }
        using Key5 = std::tuple<int, int, int, int, int>;
        struct Pending { Key5 key; int32_t ldc, m, n; BProd p; };
        std::vector<Pending> ublk, tblk;
        const int nsa = alpha.nsec;
        std::vector<int64_t> need(nsa, 0);                        // U + T1 doubles per left sector
        std::map<std::pair<int, int>, std::pair<int64_t, int64_t>> cnt;   // (a', b) -> (#T1, #U) blocks
        // U(i', t1, t2, wr, j) = x(i', t1, t2, j') R(j', wr, j)
        for (size_t rb = 0; rb < R->offsets.size(); ++rb) {
            const int jp = R->keys[rb * 3], wr = R->keys[rb * 3 + 1], j = R->keys[rb * 3 + 2];
            auto it = x_by_b.find(jp);
            if (it == x_by_b.end()) continue;
            for (size_t xb : it->second) {
                const int ip = x->keys[xb * 4], t1 = x->keys[xb * 4 + 1], t2 = x->keys[xb * 4 + 2];
                const int mi = alpha.dims[ip], mjp = beta.dims[jp], mj = beta.dims[j];
                BProd p{};
                p.a_off = x->offsets[xb]; p.a_rs = mjp; p.a_cs = 1;
                p.b_off = R->offsets[rb]; p.b_rs = mj; p.b_cs = 1;
                p.K = mjp; p.c1 = -1; p.c2 = -1;
                ublk.push_back({Key5{ip, t1, t2, wr, j}, mj, mi, mj, p});
                need[ip] += (int64_t)mi * mj;
                cnt[{ip, j}].second++;
            }
        }
        // T1(i', wl, s1, s2, j) = L(i', wl, i) x(i, s1, s2, j)
        for (size_t lb = 0; lb < L->offsets.size(); ++lb) {
            const int ip = L->keys[lb * 3], wl = L->keys[lb * 3 + 1], i = L->keys[lb * 3 + 2];
            auto it = x_by_a.find(i);
            if (it == x_by_a.end()) continue;
            for (size_t xb : it->second) {
                const int s1 = x->keys[xb * 4 + 1], s2 = x->keys[xb * 4 + 2], j = x->keys[xb * 4 + 3];
                const int mip = alpha.dims[ip], mi = alpha.dims[i], mj = beta.dims[j];
                BProd p{};
                p.a_off = L->offsets[lb]; p.a_rs = mi; p.a_cs = 1;
                p.b_off = x->offsets[xb]; p.b_rs = mj; p.b_cs = 1;
                p.K = mi; p.c1 = -1; p.c2 = -1;
                tblk.push_back({Key5{ip, wl, s1, s2, j}, mj, mip, mj, p});
                need[ip] += (int64_t)mip * mj;
                cnt[{ip, j}].first++;
            }
        }
        // Chunks of consecutive left sectors whose U and T1 fit the limit (0: one chunk)
        auto al = [](int64_t v) { return (v + 31) / 32 * 32; };
        const int64_t CH = 1 << 16;
        const int64_t nxd = (x->nelem + CH - 1) / CH;
        int64_t total_g = 0;
        for (auto& kv : cnt) total_g += kv.second.first * kv.second.second;
        const int64_t fixed = 2 * al(g->ng) + 32 + al(std::max<int64_t>(total_g, nxd));
        std::vector<int> chunk_of(nsa, 0);
        int nchunk = 1;
        if (ws_limit > 0) {
            const int64_t avail = (int64_t)(ws_limit / sizeof(double)) - fixed - 64;
            int64_t biggest = 0;
            for (int q = 0; q < nsa; ++q) biggest = std::max(biggest, need[q]);
            if (biggest > avail) {
                delete g;
                return fail(HEFF_ERR_WORKSPACE, "gradient workspace limit %zu bytes is below the minimum %lld bytes",
                            ws_limit, (long long)((biggest + fixed + 64) * (int64_t)sizeof(double)));
            }
            int64_t cur = 0;
            for (int q = 0; q < nsa; ++q) {
                if (cur + need[q] > avail) { ++nchunk; cur = 0; }
                chunk_of[q] = nchunk - 1;
                cur += need[q];
            }
        }
        g->chunks.resize(nchunk);
        const bool streamed = nchunk > 1;
        std::vector<int64_t> uo(nchunk, 0), to(nchunk, 0);
        std::map<Key5, int64_t> Uoff, Toff;   // block key -> offset within its chunk's region
        for (const Pending& pb : ublk) {
            const int c = chunk_of[std::get<0>(pb.key)];
            Uoff[pb.key] = uo[c];
            g->chunks[c].U.add_block(uo[c], pb.ldc, pb.m, pb.n, {pb.p});
            uo[c] += (int64_t)pb.m * pb.n;
        }
        for (int c = 0; c < nchunk; ++c) g->chunks[c].t_base = al(uo[c]);
        for (const Pending& pb : tblk) {
            const int c = chunk_of[std::get<0>(pb.key)];
            Toff[pb.key] = g->chunks[c].t_base + to[c];
            g->chunks[c].T1.add_block(g->chunks[c].t_base + to[c], pb.ldc, pb.m, pb.n, {pb.p});
            to[c] += (int64_t)pb.m * pb.n;
        }
        int64_t region = 0;
        for (int c = 0; c < nchunk; ++c) region = std::max(region, g->chunks[c].t_base + al(to[c]));
        // dL(i', wl, i) = sum W12 U(i', t1, t2, wr, j) x(i, s1, s2, j)^T: complete within the
        // chunk of i'
        for (size_t lb = 0; lb < L->offsets.size(); ++lb) {
            const int ip = L->keys[lb * 3], wl = L->keys[lb * 3 + 1], i = L->keys[lb * 3 + 2];
            std::vector<BProd> ps;
            auto it = x_by_a.find(i);
            if (it != x_by_a.end())
                for (size_t xb : it->second) {
                    const int s1 = x->keys[xb * 4 + 1], s2 = x->keys[xb * 4 + 2], j = x->keys[xb * 4 + 3];
                    const int mj = beta.dims[j];
                    for (int t1 = 0; t1 < d1; ++t1)
                        for (int t2 = 0; t2 < d2; ++t2)
                            for (int wr = 0; wr < kr; ++wr) {
                                const int64_t e = gidx(wl, t1, t2, s1, s2, wr);
                                if (w12[e].empty()) continue;
                                auto uo_it = Uoff.find({ip, t1, t2, wr, j});
                                if (uo_it == Uoff.end()) continue;
                                BProd p{};
                                p.a_off = uo_it->second; p.a_rs = mj; p.a_cs = 1;
                                p.b_off = x->offsets[xb]; p.b_rs = 1; p.b_cs = mj;   // x^T
                                p.K = mj; p.c1 = (int32_t)e; p.c2 = -1;
                                ps.push_back(p);
                            }
                }
            g->chunks[chunk_of[ip]].dL.add_block(L->offsets[lb], alpha.dims[i], alpha.dims[ip], alpha.dims[i], ps);
        }
        // dR(j', wr, j) = sum W12 x(i', t1, t2, j')^T T1(i', wl, s1, s2, j): a sum over the
        // chunks of i' (accumulated into a zeroed dR when there is more than one chunk)
        for (size_t rb = 0; rb < R->offsets.size(); ++rb) {
            const int jp = R->keys[rb * 3], wr = R->keys[rb * 3 + 1], j = R->keys[rb * 3 + 2];
            std::vector<std::vector<BProd>> ps(nchunk);
            auto it = x_by_b.find(jp);
            if (it != x_by_b.end())
                for (size_t xb : it->second) {
                    const int ip = x->keys[xb * 4], t1 = x->keys[xb * 4 + 1], t2 = x->keys[xb * 4 + 2];
                    const int mjp = beta.dims[jp], mj = beta.dims[j];
                    for (int wl = 0; wl < kl; ++wl)
                        for (int s1 = 0; s1 < d1; ++s1)
                            for (int s2 = 0; s2 < d2; ++s2) {
                                const int64_t e = gidx(wl, t1, t2, s1, s2, wr);
                                if (w12[e].empty()) continue;
                                auto to_it = Toff.find({ip, wl, s1, s2, j});
                                if (to_it == Toff.end()) continue;
                                BProd p{};
                                p.a_off = x->offsets[xb]; p.a_rs = 1; p.a_cs = mjp;   // x^T
                                p.b_off = to_it->second; p.b_rs = mj; p.b_cs = 1;
                                p.K = alpha.dims[ip]; p.c1 = (int32_t)e; p.c2 = -1;
                                ps[chunk_of[ip]].push_back(p);
                            }
                }
            for (int c = 0; c < nchunk; ++c)
                if (!streamed || !ps[c].empty())
                    g->chunks[c].dR.add_block(R->offsets[rb], beta.dims[j], beta.dims[jp], beta.dims[j], ps[c]);
        }
        for (GradChunk& c : g->chunks) c.dR.accumulate = streamed;
        // G dots: T1(i', wl, s1, s2, j) with U(i', t1, t2, wr, j), grouped by chunk and G index
        std::map<std::pair<int, int>, std::vector<std::pair<std::tuple<int, int, int>, int64_t>>> Tby, Uby;
        for (auto& kv : Toff)
            Tby[{std::get<0>(kv.first), std::get<4>(kv.first)}].push_back(
                {{std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first)}, kv.second});
        for (auto& kv : Uoff)
            Uby[{std::get<0>(kv.first), std::get<4>(kv.first)}].push_back(
                {{std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first)}, kv.second});
        int64_t max_gd = 0;
        for (int c = 0; c < nchunk; ++c) {
            std::vector<std::vector<BDot>> gd(g->ng);
            for (auto& kv : Tby) {
                if (chunk_of[kv.first.first] != c) continue;
                auto uit = Uby.find(kv.first);
                if (uit == Uby.end()) continue;
                const int64_t len = (int64_t)alpha.dims[kv.first.first] * beta.dims[kv.first.second];
                for (auto& tb : kv.second)
                    for (auto& ub : uit->second) {
                        const int wl = std::get<0>(tb.first), s1 = std::get<1>(tb.first), s2 = std::get<2>(tb.first);
                        const int t1 = std::get<0>(ub.first), t2 = std::get<1>(ub.first), wr = std::get<2>(ub.first);
                        gd[gidx(wl, t1, t2, s1, s2, wr)].push_back({tb.second, ub.second, len});
                    }
            }
            GradChunk& ch = g->chunks[c];
            ch.goff.push_back(0);
            for (auto& v : gd) {
                ch.gdots.insert(ch.gdots.end(), v.begin(), v.end());
                ch.goff.push_back((int32_t)ch.gdots.size());
            }
            max_gd = std::max<int64_t>(max_gd, (int64_t)ch.gdots.size());
        }
        // x chunks for the scalars
        g->xoff.push_back(0);
        for (int64_t o = 0; o < x->nelem; o += CH) g->xdots.push_back({o, o, std::min(CH, x->nelem - o)});
        g->xoff.push_back((int32_t)g->xdots.size());
        g->nR = R->nelem;
        // workspace layout (doubles): shared U/T1 region, W12, G, scalars, dot partials
        int64_t o = 0;
        g->off_U = o; o += region;
        g->off_W12 = o; o += al(g->ng);
        g->off_G = o; o += al(g->ng);
        g->off_sc = o; o += 32;
        g->npart = std::max<int64_t>(max_gd, (int64_t)g->xdots.size());
        g->off_part = o; o += al(g->npart);
        g->off_flag = o; o += 32;          // sticky error flag of the tensor-core products
        g->ws_bytes_fp64 = (size_t)o * sizeof(double);
        g->nL = L->nelem;
        g->off_x32 = o; o += al((x->nelem + 1) / 2);
        g->off_L32 = o; o += al((L->nelem + 1) / 2);
        g->off_R32 = o; o += al((R->nelem + 1) / 2);
        g->ws_bytes_tc = (size_t)o * sizeof(double);
        g->ws_bytes = g->ws_bytes_fp64;
    } catch (const std::bad_alloc&) {
        delete g;
        return fail(HEFF_ERR_OOM, "out of host memory while planning the gradients");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        int rc = HEFF_OK;
        for (GradChunk& c : g->chunks) {
            for (BList* b : {&c.U, &c.T1, &c.dL, &c.dR})
                if (!rc) rc = heff::blist_upload(*b);
            if (!rc) rc = up(c.gdots, &c.d_gdots);
            if (!rc) rc = up(c.goff, &c.d_goff);
        }
        if (!rc) rc = up(g->xdots, &g->d_xdots);
        if (!rc) rc = up(g->xoff, &g->d_xoff);
        if (!rc) rc = up(g->w12_off, &g->d_w12_off);
        if (!rc) rc = up(g->w12_terms, &g->d_w12_terms);
        if (!rc) rc = up(g->dw1_off, &g->d_dw1_off);
        if (!rc) rc = up(g->dw1_terms, &g->d_dw1_terms);
        if (!rc) rc = up(g->dw2_off, &g->d_dw2_off);
        if (!rc) rc = up(g->dw2_terms, &g->d_dw2_terms);
        if (rc) {
            free_all(g);
            delete g;
            return rc;
        }
        g->uploaded = true;
    } else {
        cudaGetLastError();
    }
    *out = g;
    return HEFF_OK;
}

extern "C" int heff_grad_chunks(const heff_grad_plan* g, int32_t* nchunks) {
    heff::clear_error();
    if (!g || !nchunks) return fail(HEFF_ERR_INVALID_ARG, "heff_grad_chunks: null argument");
    *nchunks = (int32_t)g->chunks.size();
    return HEFF_OK;
}

extern "C" int heff_grad_workspace_size(const heff_grad_plan* g, size_t* bytes) {
    heff::clear_error();
    if (!g || !bytes) return fail(HEFF_ERR_INVALID_ARG, "heff_grad_workspace_size: null argument");
    *bytes = g->ws_bytes;
    return HEFF_OK;
}

extern "C" int heff_backward(heff_grad_plan* g, heff_plan* plan, const double* L, const double* W1,
                             const double* W2, const double* R, const double* x, double* rho, double* dx,
                             double* dL, double* dR, double* dW1, double* dW2, void* apply_ws,
                             size_t apply_ws_bytes, void* grad_ws, size_t grad_ws_bytes, void* stream) {
    heff::clear_error();
    if (!g || !plan || !L || !W1 || !W2 || !R || !x || !rho || !dx || !dL || !dR || !dW1 || !dW2)
        return fail(HEFF_ERR_INVALID_ARG, "heff_backward: null argument");
    if (!g->uploaded) return fail(HEFF_ERR_UNSUPPORTED, "gradient plan was created without a CUDA device");
    if (plan->opts.io_dtype != HEFF_DTYPE_F64)
        return fail(HEFF_ERR_UNSUPPORTED, "heff_backward needs an apply plan with HEFF_DTYPE_F64 tensors");
    if (plan->nelem_x != g->nx) return fail(HEFF_ERR_INVALID_ARG, "apply plan and gradient plan disagree on x");
    if (!grad_ws || grad_ws_bytes < g->ws_bytes || reinterpret_cast<uintptr_t>(grad_ws) % 256)
        return fail(HEFF_ERR_WORKSPACE, "gradient workspace of %zu bytes, needs %zu (256-byte aligned)",
                    grad_ws_bytes, g->ws_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* ws = static_cast<double*>(grad_ws);
    double *Ureg = ws + g->off_U, *W12 = ws + g->off_W12, *G = ws + g->off_G;
    double *sc = ws + g->off_sc, *part = ws + g->off_part;
    int* err = reinterpret_cast<int*>(ws + g->off_flag);
    const bool tc = g->precision != HEFF_PREC_FP64;
    float* x32 = reinterpret_cast<float*>(ws + g->off_x32);
    float* L32 = reinterpret_cast<float*>(ws + g->off_L32);
    float* R32 = reinterpret_cast<float*>(ws + g->off_R32);
    if (tc && cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
        return fail(HEFF_ERR_CUDA, "heff_backward: memset failed");
    // y = K x into dx (dx is overwritten by the gradient below)
    int rc = heff_apply(plan, L, W1, W2, R, x, dx, apply_ws, apply_ws_bytes, stream);
    if (rc) return rc;
    const int nxd = (int)g->xdots.size();
    if ((rc = heff::launch_block_dots(g->d_xdots, nxd, g->d_xoff, x, x, sc + 0, 1, part, 1.0, stream))) return rc;
    if ((rc = heff::launch_block_dots(g->d_xdots, nxd, g->d_xoff, x, dx, sc + 1, 1, part, 1.0, stream))) return rc;
    rho_kernel<<<1, 1, 0, st>>>(sc);
    const int G1 = (int)std::min<int64_t>((g->nx + 255) / 256, 4096);
    dx_kernel<<<G1 > 0 ? G1 : 1, 256, 0, st>>>(x, dx, sc, dx, g->nx);
    cudaMemcpyAsync(rho, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, st);
    heff::count_launches(2);
    // W12 on the device from the current MPO values
    pair_sum_kernel<<<(int)((g->ng + 255) / 256), 256, 0, st>>>(g->d_w12_off, g->d_w12_terms, W1, W2, W12, g->ng);
    heff::count_launches(1);
    if (tc) {   // FP32 operand copies for the tensor-core products, converted once
        int rc2;
        if ((rc2 = heff::launch_convert_f64_f32(x, x32, g->nx, stream)) ||
            (rc2 = heff::launch_convert_f64_f32(L, L32, g->nL, stream)) ||
            (rc2 = heff::launch_convert_f64_f32(R, R32, g->nR, stream)))
            return rc2;
    }
    const bool streamed = g->chunks.size() > 1;
    if (streamed) {   // dR and G are sums over the chunks
        if (cudaMemsetAsync(dR, 0, (size_t)g->nR * sizeof(double), st) != cudaSuccess ||
            cudaMemsetAsync(G, 0, (size_t)g->ng * sizeof(double), st) != cudaSuccess)
            return fail(HEFF_ERR_CUDA, "heff_backward: memset failed");
    }
    for (const GradChunk& c : g->chunks) {
        // U at the start of the shared region, T1 at the chunk's t_base: the lists hold
        // offsets within the region
        if (tc) {
            // the tensor-core products on the FP32 copies; U and T1 in FP32 (the region holds
            // the same element offsets in half the bytes)
            float *U = reinterpret_cast<float*>(Ureg), *T1 = U;
            if ((rc = heff::launch_bgemm_tc(c.U, x32, R32, U, false, nullptr, nullptr, 1.0, stream, nullptr, err)) ||
                (rc = heff::launch_bgemm_tc(c.T1, L32, x32, T1, false, nullptr, nullptr, 1.0, stream, nullptr, err)) ||
                (rc = heff::launch_bgemm_tc(c.dL, U, x32, dL, true, W12, nullptr, 1.0, stream, sc, err)) ||
                (rc = heff::launch_bgemm_tc(c.dR, x32, T1, dR, true, W12, nullptr, 1.0, stream, sc, err)) ||
                (rc = heff::launch_block_dots_f32(c.d_gdots, (int)c.gdots.size(), c.d_goff, T1, U, G, (int)g->ng,
                                                  part, 1.0, stream, streamed)))
                return rc;
            continue;
        }
        double *U = Ureg, *T1 = Ureg;
        if ((rc = heff::launch_bgemm(c.U, x, R, U, nullptr, nullptr, 1.0, stream))) return rc;
        if ((rc = heff::launch_bgemm(c.T1, L, x, T1, nullptr, nullptr, 1.0, stream))) return rc;
        if ((rc = heff::launch_bgemm(c.dL, U, x, dL, W12, nullptr, 1.0, stream, sc))) return rc;
        if ((rc = heff::launch_bgemm(c.dR, x, T1, dR, W12, nullptr, 1.0, stream, sc))) return rc;
        if ((rc = heff::launch_block_dots(c.d_gdots, (int)c.gdots.size(), c.d_goff, T1, U, G, (int)g->ng, part, 1.0,
                                          stream, streamed)))
            return rc;
    }
    // dW1 = G . W2, dW2 = G . W1 (then divided by n)
    pair_sum_kernel<<<(int)((g->nW1 + 255) / 256), 256, 0, st>>>(g->d_dw1_off, g->d_dw1_terms, G, W2, dW1, g->nW1);
    pair_sum_kernel<<<(int)((g->nW2 + 255) / 256), 256, 0, st>>>(g->d_dw2_off, g->d_dw2_terms, G, W1, dW2, g->nW2);
    // divide the W gradients by n
    div_kernel<<<(int)((g->nW1 + 255) / 256), 256, 0, st>>>(dW1, g->nW1, sc);
    div_kernel<<<(int)((g->nW2 + 255) / 256), 256, 0, st>>>(dW2, g->nW2, sc);
    heff::count_launches(4);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_backward: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

extern "C" int heff_grad_plan_set_precision(heff_grad_plan* g, int32_t precision) {
    heff::clear_error();
    if (!g) return fail(HEFF_ERR_INVALID_ARG, "heff_grad_plan_set_precision: null plan");
    if (precision != HEFF_PREC_FP64 && precision != HEFF_PREC_BF16X3)
        return fail(HEFF_ERR_UNSUPPORTED, "gradient block products run in HEFF_PREC_FP64 or HEFF_PREC_BF16X3");
    if (precision == g->precision) return HEFF_OK;
    const int tile = precision == HEFF_PREC_FP64 ? 64 : 128;
    int rc = HEFF_OK;
    for (GradChunk& c : g->chunks)
        for (BList* b : {&c.U, &c.T1, &c.dL, &c.dR}) {
            heff::blist_free(*b);
            b->retile(tile, tile);
            if (g->uploaded && !rc) rc = heff::blist_upload(*b);
        }
    g->precision = precision;
    g->ws_bytes = precision == HEFF_PREC_FP64 ? g->ws_bytes_fp64 : g->ws_bytes_tc;
    if (rc) g->uploaded = false;
    return rc;
}

extern "C" int heff_grad_status(const heff_grad_plan* g, void* grad_ws, size_t grad_ws_bytes, void* stream) {
    heff::clear_error();
    if (!g || !grad_ws) return fail(HEFF_ERR_INVALID_ARG, "heff_grad_status: null argument");
    if (g->precision == HEFF_PREC_FP64) return HEFF_OK;
    if (grad_ws_bytes < g->ws_bytes) return fail(HEFF_ERR_WORKSPACE, "heff_grad_status: workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* d = reinterpret_cast<int*>(static_cast<double*>(grad_ws) + g->off_flag);
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && flag) e = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (e == cudaSuccess && flag) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_grad_status: %s", cudaGetErrorString(e));
    if (flag) return fail(HEFF_ERR_TIMEOUT, "a bounded device-side wait of the gradient products expired");
    return HEFF_OK;
}

extern "C" void heff_grad_plan_destroy(heff_grad_plan* g) {
    if (!g) return;
    free_all(g);
    delete g;
}
