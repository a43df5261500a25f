// Environment extension on the GPU (Section II-C: the left environment A and right
// environment B grow by one site as the sweep moves), in FP64 on the block-product engine.
//
// Left (site tensor A[a, s, b], flows (+1, +1, -1); environment L[a', w, a]):
//   X[(a', w), (s, b)]  = L[a', w, a] . A[a, s, b]                      (step 1)
//   Lnew[c, v, d]       = sum W[w, t, s, v] A[a', t, c]^T . X[(a', w), (s, d)]   (step 2)
// Right (site tensor B[a, s, b]; environment R[b', w, b]):
//   Y[(b', v), (a, s)]  = R[b', v, b] . B[a, s, b]^T                    (step 1)
//   Rnew[c, w, d]       = sum W[w, t, s, v] B[c, t, b'] . Y[(b', v), (d, s)]     (step 2)
// Each charge-matched block pair is one small dense product; step 2 sums, per output
// block, the products whose MPO coefficient is nonzero in the host copy of W.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>

#include "internal.h"

using heff::fail;
using heff::BList;
using heff::BProd;

// Workspace: [error flag, 256 B][intermediate X or Y][tensor-core precision only: FP32 copies
// of env_old and of the site tensor].  The FP64 products keep the intermediate in FP64; the
// tensor-core products read FP32 copies and keep it in FP32.
struct heff_env_plan {
    int side = 0;
    int precision = HEFF_PREC_FP64;   // of the block products
    BList step1, step2;
    int64_t ws_elems = 0;      // intermediate (X or Y) elements
    int64_t n_env = 0, n_site = 0;
    size_t off_x = 256, off_env32 = 0, off_site32 = 0;
    size_t ws_bytes = 0;
    bool uploaded = false;
};

namespace {

using Charge = std::vector<int32_t>;

bool same(const heff::IndexDesc& a, const heff::IndexDesc& b) { return a.same_sectors(b); }

Charge add(const Charge& a, const Charge& b, int sb = 1) {
    Charge r(a);
    for (size_t c = 0; c < r.size(); ++c) r[c] += sb * b[c];
    return r;
}

}  // namespace

extern "C" int heff_env_plan_create(const heff_layout* env_old, const heff_layout* site, const heff_layout* W,
                                    const heff_layout* env_new, const double* W_host, int32_t side,
                                    heff_env_plan** out) {
    heff::clear_error();
    if (!env_old || !site || !W || !env_new || !W_host || !out || (side != 0 && side != 1))
        return fail(HEFF_ERR_INVALID_ARG, "heff_env_plan_create: bad arguments");
    *out = nullptr;
    if (env_old->idx.size() != 3 || env_new->idx.size() != 3 || site->idx.size() != 3 || W->idx.size() != 4)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "orders must be env 3, site 3, W 4");
    const heff::IndexDesc &sa = site->idx[0], &sp = site->idx[1], &sb = site->idx[2];
    if (sa.flow != 1 || sp.flow != 1 || sb.flow != -1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "site tensor flows must be (+1, +1, -1)");
    const heff::IndexDesc& bond_in = side == 0 ? sa : sb;    // bond of env_old
    const heff::IndexDesc& bond_out = side == 0 ? sb : sa;   // bond of env_new
    const heff::IndexDesc &wi = side == 0 ? W->idx[0] : W->idx[3];    // channels of env_old
    const heff::IndexDesc &wo = side == 0 ? W->idx[3] : W->idx[0];    // channels of env_new
    if (!same(env_old->idx[0], bond_in) || !same(env_old->idx[2], bond_in) || !same(env_old->idx[1], wi))
        return fail(HEFF_ERR_CHARGE_MISMATCH, "env_old must be (bond, channel, bond) on the site's %s bond",
                    side == 0 ? "left" : "right");
    if (!same(env_new->idx[0], bond_out) || !same(env_new->idx[2], bond_out) || !same(env_new->idx[1], wo))
        return fail(HEFF_ERR_CHARGE_MISMATCH, "env_new must be (bond, channel, bond) on the site's %s bond",
                    side == 0 ? "right" : "left");
    if (!same(W->idx[1], sp) || !same(W->idx[2], sp))
        return fail(HEFF_ERR_CHARGE_MISMATCH, "W physical indices must match the site tensor");
    heff_env_plan* P = new (std::nothrow) heff_env_plan();
    if (!P) return fail(HEFF_ERR_OOM, "out of host memory");
    P->side = side;
    try {
        const int d = sp.nsec, kw = W->idx[0].nsec, kv = W->idx[3].nsec;
        // W entries kept (nonzero in the host copy) as a dense (w, t, s, v) table, -1: dropped
        std::vector<int32_t> wtab((size_t)kw * d * d * kv, -1);
        for (size_t bk = 0; bk < W->offsets.size(); ++bk) {
            const int32_t* k = &W->keys[bk * 4];
            const int64_t o = W->offsets[bk];
            if (W_host[o] != 0.0) wtab[(((size_t)k[0] * d + k[1]) * d + k[2]) * kv + k[3]] = (int32_t)o;
        }
        auto widx = [&](int w, int t, int s, int v) -> int32_t {
            return wtab[(((size_t)w * d + t) * d + s) * kv + v];
        };
        // site blocks by key
        auto site_off = [&](int a, int s, int b) { return site->offset_of({a, s, b}); };
        std::map<std::tuple<int, int, int, int>, int64_t> inter;   // intermediate blocks -> offset
        int64_t ioff = 0;
        if (side == 0) {
            // X(ia, w, s, jd) = L(ia, w, ib) A(ib, s, jd): needed when some W[w, t, s, v] != 0
            for (size_t bk = 0; bk < env_old->offsets.size(); ++bk) {
                const int ia = env_old->keys[bk * 3], w = env_old->keys[bk * 3 + 1], ib = env_old->keys[bk * 3 + 2];
                for (int s = 0; s < d; ++s) {
                    bool used = false;
                    for (int t = 0; t < d && !used; ++t)
                        for (int v = 0; v < kv && !used; ++v) used = widx(w, t, s, v) >= 0;
                    if (!used) continue;
                    int jd = sb.find(add(sa.q(ib), sp.q(s)));
                    if (jd < 0) continue;
                    int64_t so = site_off(ib, s, jd);
                    if (so < 0) continue;
                    const int mia = sa.dims[ia], mib = sa.dims[ib], mjd = sb.dims[jd];
                    inter[{ia, w, s, jd}] = ioff;
                    BProd p{};
                    p.a_off = env_old->offsets[bk]; p.a_rs = mib; p.a_cs = 1;
                    p.b_off = so; p.b_rs = mjd; p.b_cs = 1;
                    p.K = mib; p.c1 = -1; p.c2 = -1;
                    P->step1.add_block(ioff, mjd, mia, mjd, {p});
                    ioff += (int64_t)mia * mjd;
                }
            }
            // Lnew(jc, v, jd) = sum W[w,t,s,v] A(ia, t, jc)^T X(ia, w, s, jd)
            for (size_t bk = 0; bk < env_new->offsets.size(); ++bk) {
                const int jc = env_new->keys[bk * 3], v = env_new->keys[bk * 3 + 1], jd = env_new->keys[bk * 3 + 2];
                const int mjc = sb.dims[jc], mjd = sb.dims[jd];
                std::vector<BProd> ps;
                for (int t = 0; t < d; ++t) {
                    int ia = sa.find(add(sb.q(jc), sp.q(t), -1));
                    if (ia < 0) continue;
                    int64_t so = site_off(ia, t, jc);
                    if (so < 0) continue;
                    for (int w = 0; w < kw; ++w)
                        for (int s = 0; s < d; ++s) {
                            int32_t c = widx(w, t, s, v);
                            if (c < 0) continue;
                            auto it = inter.find({ia, w, s, jd});
                            if (it == inter.end()) continue;
                            BProd p{};
                            p.a_off = so; p.a_rs = 1; p.a_cs = mjc;          // A^T: (c, a) at a*mjc + c
                            p.b_off = it->second; p.b_rs = mjd; p.b_cs = 1;
                            p.K = sa.dims[ia]; p.c1 = c; p.c2 = -1;
                            ps.push_back(p);
                        }
                }
                P->step2.add_block(env_new->offsets[bk], mjd, mjc, mjd, ps);
            }
        } else {
            // Y(ja, v, id, s) = R(ja, v, jb) B(id, s, jb)^T
            for (size_t bk = 0; bk < env_old->offsets.size(); ++bk) {
                const int ja = env_old->keys[bk * 3], v = env_old->keys[bk * 3 + 1], jb = env_old->keys[bk * 3 + 2];
                for (int s = 0; s < d; ++s) {
                    bool used = false;
                    for (int t = 0; t < d && !used; ++t)
                        for (int w = 0; w < kw && !used; ++w) used = widx(w, t, s, v) >= 0;
                    if (!used) continue;
                    int id = sa.find(add(sb.q(jb), sp.q(s), -1));
                    if (id < 0) continue;
                    int64_t so = site_off(id, s, jb);
                    if (so < 0) continue;
                    const int mja = sb.dims[ja], mjb = sb.dims[jb], mid = sa.dims[id];
                    inter[{ja, v, id, s}] = ioff;
                    BProd p{};
                    p.a_off = env_old->offsets[bk]; p.a_rs = mjb; p.a_cs = 1;
                    p.b_off = so; p.b_rs = 1; p.b_cs = mjb;          // B^T: (b, d) at d*mjb + b
                    p.K = mjb; p.c1 = -1; p.c2 = -1;
                    P->step1.add_block(ioff, mid, mja, mid, {p});
                    ioff += (int64_t)mja * mid;
                }
            }
            // Rnew(ic, w, id) = sum W[w,t,s,v] B(ic, t, ja) Y(ja, v, id, s)
            for (size_t bk = 0; bk < env_new->offsets.size(); ++bk) {
                const int ic = env_new->keys[bk * 3], w = env_new->keys[bk * 3 + 1], id = env_new->keys[bk * 3 + 2];
                const int mic = sa.dims[ic], mid = sa.dims[id];
                std::vector<BProd> ps;
                for (int t = 0; t < d; ++t) {
                    int ja = sb.find(add(sa.q(ic), sp.q(t)));
                    if (ja < 0) continue;
                    int64_t so = site_off(ic, t, ja);
                    if (so < 0) continue;
                    const int mja = sb.dims[ja];
                    for (int v = 0; v < kv; ++v)
                        for (int s = 0; s < d; ++s) {
                            int32_t c = widx(w, t, s, v);
                            if (c < 0) continue;
                            auto it = inter.find({ja, v, id, s});
                            if (it == inter.end()) continue;
                            BProd p{};
                            p.a_off = so; p.a_rs = mja; p.a_cs = 1;
                            p.b_off = it->second; p.b_rs = mid; p.b_cs = 1;
                            p.K = mja; p.c1 = c; p.c2 = -1;
                            ps.push_back(p);
                        }
                }
                P->step2.add_block(env_new->offsets[bk], mid, mic, mid, ps);
            }
        }
        P->ws_elems = ioff;
        P->n_env = env_old->nelem;
        P->n_site = site->nelem;
        auto al = [](size_t v) { return (v + 255) / 256 * 256; };
        const size_t fp64_bytes = P->off_x + al((size_t)ioff * sizeof(double));
        P->off_env32 = P->off_x + al((size_t)ioff * sizeof(float));
        P->off_site32 = P->off_env32 + al((size_t)P->n_env * sizeof(float));
        const size_t tc_bytes = P->off_site32 + al((size_t)P->n_site * sizeof(float));
        P->ws_bytes = std::max(fp64_bytes, tc_bytes);
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(HEFF_ERR_OOM, "out of host memory while planning the environment update");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        int rc;
        if ((rc = heff::blist_upload(P->step1)) || (rc = heff::blist_upload(P->step2))) {
            heff::blist_free(P->step1);
            heff::blist_free(P->step2);
            delete P;
            return rc;
        }
        P->uploaded = true;
    } else {
        cudaGetLastError();
    }
    *out = P;
    return HEFF_OK;
}

extern "C" int heff_env_workspace_size(const heff_env_plan* plan, size_t* bytes) {
    heff::clear_error();
    if (!plan || !bytes) return fail(HEFF_ERR_INVALID_ARG, "heff_env_workspace_size: null argument");
    *bytes = plan->ws_bytes;
    return HEFF_OK;
}

extern "C" int heff_env_flops(const heff_env_plan* plan, double* flops) {
    heff::clear_error();
    if (!plan || !flops) return fail(HEFF_ERR_INVALID_ARG, "heff_env_flops: null argument");
    *flops = plan->step1.flops + plan->step2.flops;
    return HEFF_OK;
}

extern "C" int heff_env_update(heff_env_plan* plan, const double* env_old, const double* site, const double* W,
                               double* env_new, void* workspace, size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (!plan || !env_old || !site || !W || !env_new)
        return fail(HEFF_ERR_INVALID_ARG, "heff_env_update: null argument");
    if (!plan->uploaded) return fail(HEFF_ERR_UNSUPPORTED, "env plan was created without a CUDA device");
    if (!workspace || workspace_bytes < plan->ws_bytes || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(HEFF_ERR_WORKSPACE, "environment workspace of %zu bytes, needs %zu (256-byte aligned)",
                    workspace_bytes, plan->ws_bytes);
    char* ws = static_cast<char*>(workspace);
    int* err = reinterpret_cast<int*>(ws);
    int rc;
    if (plan->precision == HEFF_PREC_FP64) {
        double* X = reinterpret_cast<double*>(ws + plan->off_x);
        if ((rc = heff::launch_bgemm(plan->step1, env_old, site, X, nullptr, nullptr, 1.0, stream))) return rc;
        return heff::launch_bgemm(plan->step2, site, X, env_new, W, nullptr, 1.0, stream);
    }
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    float* X = reinterpret_cast<float*>(ws + plan->off_x);
    float* E32 = reinterpret_cast<float*>(ws + plan->off_env32);
    float* S32 = reinterpret_cast<float*>(ws + plan->off_site32);
    if ((rc = heff::launch_convert_f64_f32(env_old, E32, plan->n_env, stream))) return rc;
    if ((rc = heff::launch_convert_f64_f32(site, S32, plan->n_site, stream))) return rc;
    if ((rc = heff::launch_bgemm_tc(plan->step1, E32, S32, X, false, nullptr, nullptr, 1.0, stream, nullptr, err)))
        return rc;
    return heff::launch_bgemm_tc(plan->step2, S32, X, env_new, true, W, nullptr, 1.0, stream, nullptr, err);
}

extern "C" int heff_env_plan_set_precision(heff_env_plan* plan, int32_t precision) {
    heff::clear_error();
    if (!plan) return fail(HEFF_ERR_INVALID_ARG, "heff_env_plan_set_precision: null plan");
    if (precision != HEFF_PREC_FP64 && precision != HEFF_PREC_BF16X3)
        return fail(HEFF_ERR_UNSUPPORTED, "environment updates run in HEFF_PREC_FP64 or HEFF_PREC_BF16X3");
    if (precision == plan->precision) return HEFF_OK;
    const int tile = precision == HEFF_PREC_FP64 ? 64 : 128;
    heff::blist_free(plan->step1);
    heff::blist_free(plan->step2);
    plan->step1.retile(tile, tile);
    plan->step2.retile(tile, tile);
    plan->precision = precision;
    if (plan->uploaded) {
        int rc;
        if ((rc = heff::blist_upload(plan->step1)) || (rc = heff::blist_upload(plan->step2))) {
            plan->uploaded = false;
            return rc;
        }
    }
    return HEFF_OK;
}

extern "C" int heff_env_status(const heff_env_plan* plan, void* workspace, size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (!plan || !workspace) return fail(HEFF_ERR_INVALID_ARG, "heff_env_status: null argument");
    if (plan->precision == HEFF_PREC_FP64) return HEFF_OK;
    if (workspace_bytes < plan->ws_bytes) return fail(HEFF_ERR_WORKSPACE, "heff_env_status: workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* d = static_cast<int*>(workspace);
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && flag) e = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (e == cudaSuccess && flag) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_env_status: %s", cudaGetErrorString(e));
    if (flag) return fail(HEFF_ERR_TIMEOUT, "a bounded device-side wait of the environment update expired");
    return HEFF_OK;
}

extern "C" void heff_env_plan_destroy(heff_env_plan* plan) {
    if (!plan) return;
    heff::blist_free(plan->step1);
    heff::blist_free(plan->step2);
    delete plan;
}

// ---------------------------------------------------------------- two-site tensor
// x[a, s1, s2, b] = sum_c A[a, s1, c] B[c, s2, b] (Fig. 1d: the two MPS sites joined over
// their shared bond, the starting vector of a bond's eigensolve).  One block product per
// charge-matched (A block, B block) pair, summed per x block; x blocks without a matching
// pair are written as zeros.
struct heff_two_site {
    BList prods;
    bool uploaded = false;
};

extern "C" int heff_two_site_create(const heff_layout* A, const heff_layout* B, const heff_layout* x,
                                    heff_two_site** out) {
    heff::clear_error();
    if (!A || !B || !x || !out) return fail(HEFF_ERR_INVALID_ARG, "heff_two_site_create: null argument");
    *out = nullptr;
    if (A->idx.size() != 3 || B->idx.size() != 3 || x->idx.size() != 4)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "orders must be A 3, B 3, x 4");
    const heff::IndexDesc &aa = A->idx[0], &ap = A->idx[1], &ac = A->idx[2];
    const heff::IndexDesc &bc = B->idx[0], &bp = B->idx[1], &bb = B->idx[2];
    if (aa.flow != 1 || ap.flow != 1 || ac.flow != -1 || bc.flow != 1 || bp.flow != 1 || bb.flow != -1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "A and B flows must be (+1, +1, -1)");
    if (!same(ac, bc) || !same(aa, x->idx[0]) || !same(ap, x->idx[1]) || !same(bp, x->idx[2]) ||
        !same(bb, x->idx[3]))
        return fail(HEFF_ERR_CHARGE_MISMATCH, "A (a, s1, c), B (c, s2, b) and x (a, s1, s2, b) indices disagree");
    heff_two_site* P = new (std::nothrow) heff_two_site();
    if (!P) return fail(HEFF_ERR_OOM, "out of host memory");
    try {
        std::map<std::pair<int, int>, std::vector<std::pair<int, int64_t>>> a_by;   // (a, s1) -> (c, offset)
        for (size_t k = 0; k < A->offsets.size(); ++k)
            a_by[{A->keys[k * 3], A->keys[k * 3 + 1]}].push_back({A->keys[k * 3 + 2], A->offsets[k]});
        for (size_t k = 0; k < x->offsets.size(); ++k) {
            const int a = x->keys[k * 4], s1 = x->keys[k * 4 + 1], s2 = x->keys[k * 4 + 2], b = x->keys[k * 4 + 3];
            const int ma = aa.dims[a], mb = bb.dims[b];
            std::vector<BProd> ps;
            auto it = a_by.find({a, s1});
            if (it != a_by.end())
                for (auto& co : it->second) {
                    const int64_t boff = B->offset_of({co.first, s2, b});
                    if (boff < 0) continue;
                    const int mc = ac.dims[co.first];
                    BProd p{};
                    p.a_off = co.second; p.a_rs = mc; p.a_cs = 1;
                    p.b_off = boff; p.b_rs = mb; p.b_cs = 1;
                    p.K = mc; p.c1 = -1; p.c2 = -1;
                    ps.push_back(p);
                }
            P->prods.add_block(x->offsets[k], mb, ma, mb, ps);
        }
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(HEFF_ERR_OOM, "out of host memory while planning the two-site tensor");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        int rc = heff::blist_upload(P->prods);
        if (rc) {
            heff::blist_free(P->prods);
            delete P;
            return rc;
        }
        P->uploaded = true;
    } else {
        cudaGetLastError();
    }
    *out = P;
    return HEFF_OK;
}

extern "C" int heff_two_site_apply(heff_two_site* P, const double* A, const double* B, double* x, void* stream) {
    heff::clear_error();
    if (!P || !A || !B || !x) return fail(HEFF_ERR_INVALID_ARG, "heff_two_site_apply: null argument");
    if (!P->uploaded) return fail(HEFF_ERR_UNSUPPORTED, "two-site plan was created without a CUDA device");
    return heff::launch_bgemm(P->prods, A, B, x, nullptr, nullptr, 1.0, stream);
}

extern "C" void heff_two_site_destroy(heff_two_site* P) {
    if (!P) return;
    heff::blist_free(P->prods);
    delete P;
}
