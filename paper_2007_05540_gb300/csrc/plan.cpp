// Host planner: the charge-matched block schedule of y = K x (Algorithm 2 applied to
// both contractions of the two-site matvec, Section II-C / Fig. 1d) laid out for the
// GPU kernels.
//
// The matvec is evaluated as two grouped GEMMs around operators with the MPO folded in:
//
//   LW[(a',t1,wm), (a,s1)] = sum_wl W1[wl,t1,s1,wm] L[a',wl,a]        (prepare)
//   RW[(t2,b'), (wm,s2,b)] = sum_wr W2[wm,t2,s2,wr] R[b',wr,b]        (prepare)
//   T [(a',t1,wm), (s2,b)] = sum_(a,s1) LW . x                         (GEMM 1)
//   y [(a',t1), (t2,b')]   = sum_(wm,s2,b) T . RW^T                    (GEMM 2)
//
// x is viewed as the block-diagonal matrix (a s1) x (s2 b) of Section IV (one dense
// block per charge Q = q(a) + q(s1) = q(b) - q(s2) + target); K-contiguous copies of its
// blocks (XT) are the B operand of GEMM 1.  Every operand array has one row pitch, and
// every contraction segment (one charge sector) starts at a multiple of KPAD columns
// with zero padding, so tiles never mix sectors.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <queue>
#include <set>
#include <stdexcept>
#include <tuple>

#include <cuda_runtime.h>

#include "internal.h"

using heff::fail;
using heff::IndexDesc;
using heff::KPAD;
using heff::pad_up;
using Charge = std::vector<int32_t>;

// 1: order the task lists as an LPT assignment for the kernels' static round-robin
#ifndef HEFF_LPT_SCHEDULE
#define HEFF_LPT_SCHEDULE 1
#endif

namespace {

// Cost of one K block of a tensor-core tile, for the LPT ordering and schedule:
// 0: its MMA width (n rounded up to 16); 1: the operand rows it streams (the A box, 64 or
// 128 rows, plus the B box of n rows); 2: the larger of the two, each scaled to a 128 x 256
// tile; 3: their mean.  Chosen per GEMM (GEMM 1 lists, GEMM 2 lists).
#ifndef HEFF_TILE_COST_G1
#define HEFF_TILE_COST_G1 0
#endif
#ifndef HEFF_TILE_COST_G2
#define HEFF_TILE_COST_G2 2
#endif
inline int64_t tile_width_cost(int m, int n, int model) {
    const int64_t mma = (n + 15) / 16 * 16;
    const int64_t rows = (m <= 64 ? 64 : 128) + (n <= 64 ? 64 : (n <= 128 ? 128 : 256));
    if (model == 0) return mma;
    if (model == 1) return rows;
    if (model == 2) return std::max(mma * 384 / 256, rows);
    return (mma * 384 / 256 + rows) / 2;
}

Charge add(const Charge& a, const Charge& b, int sb = 1) {
    Charge r(a);
    for (size_t c = 0; c < r.size(); ++c) r[c] += sb * b[c];
    return r;
}

struct CGroup { int s, sec, dim; int32_t col; int32_t row; };   // (s, bond sector)
struct QSec {
    Charge q;
    std::vector<CGroup> cg;    // (s1, i): columns of XT/LW (padded), rows of T/y
    std::vector<CGroup> eg;    // (s2, j): rows of XT/RW, columns of T inside a wm segment
    int32_t kc = 0;            // padded width of the c-space
    int32_t mrows = 0;         // sum of c-group dims
    int32_t nrows = 0;         // sum of e-group dims
    int64_t xt_row0 = 0, t_row0 = 0, rw_row0 = 0;
    // T column layout: segment (wm, eg index) -> column offset
    std::map<std::pair<int, int>, int32_t> toff;
    int32_t kt = 0;
};

struct RowGroup {              // a block row of LW: (Q, t1, wm) with a' in sector ip
    int q, t1, wm, ip;
    int64_t lw_row0;
    struct Seg { int cg; std::vector<heff::MixTerm> terms; };
    std::vector<Seg> segs;
};

struct RWGroup {               // a block row of RW: (Q', e'-group (t2, j'))
    int q, eg;
    struct Seg { int wm, q_src, eg_src; std::vector<heff::MixTerm> terms; };
    std::vector<Seg> segs;
};

bool check_index(const IndexDesc& a, const IndexDesc& b, int flow_a) {
    return a.same_sectors(b) && a.flow == flow_a;
}

}  // namespace

extern "C" int heff_plan_create(const heff_layout* L, const heff_layout* W1, const heff_layout* W2,
                                const heff_layout* R, const heff_layout* x, const double* W1_host,
                                const double* W2_host, const heff_plan_opts* opts, heff_plan** out) {
    heff::clear_error();
    if (!L || !W1 || !W2 || !R || !x || !W1_host || !W2_host || !opts || !out)
        return fail(HEFF_ERR_INVALID_ARG, "heff_plan_create: null argument");
    *out = nullptr;
    if (opts->precision < HEFF_PREC_FP64 || opts->precision > HEFF_PREC_TF32X3)
        return fail(HEFF_ERR_INVALID_ARG, "unknown precision %d", opts->precision);
    if (opts->io_dtype != HEFF_DTYPE_F64 && opts->io_dtype != HEFF_DTYPE_F32)
        return fail(HEFF_ERR_INVALID_ARG, "unknown io dtype %d", opts->io_dtype);
    if (opts->precision == HEFF_PREC_FP64 && opts->io_dtype != HEFF_DTYPE_F64)
        return fail(HEFF_ERR_UNSUPPORTED, "the FP64 path needs HEFF_DTYPE_F64 tensors");
    if (opts->max_batch < 1 || opts->max_batch > 4096)
        return fail(HEFF_ERR_INVALID_ARG, "max_batch must be 1..4096");
    if (opts->shard_count < 0 || opts->shard_count > 4096 || opts->shard_index < 0 ||
        opts->shard_index >= (opts->shard_count > 1 ? opts->shard_count : 1))
        return fail(HEFF_ERR_INVALID_ARG, "shard_index %d outside 0..shard_count-1 (shard_count %d)",
                    opts->shard_index, opts->shard_count);
    if (x->idx.size() != 4 || L->idx.size() != 3 || R->idx.size() != 3 || W1->idx.size() != 4 ||
        W2->idx.size() != 4)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "tensor orders must be x:4 L:3 R:3 W1:4 W2:4");
    const int nq = x->nq;
    if (L->nq != nq || R->nq != nq || W1->nq != nq || W2->nq != nq)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "all layouts must have the same number of charges");
    const IndexDesc &alpha = x->idx[0], &ph1 = x->idx[1], &ph2 = x->idx[2], &beta = x->idx[3];
    if (alpha.flow != 1 || ph1.flow != 1 || ph2.flow != 1 || beta.flow != -1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "x flows must be (+1,+1,+1,-1)");
    for (int s = 0; s < ph1.nsec; ++s) if (ph1.dims[s] != 1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "physical sectors must have dimension 1");
    for (int s = 0; s < ph2.nsec; ++s) if (ph2.dims[s] != 1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "physical sectors must have dimension 1");
    const IndexDesc &chl = L->idx[1], &chr = R->idx[1], &chm = W1->idx[3];
    if (!check_index(L->idx[0], alpha, -1) || !check_index(L->idx[2], alpha, 1) || chl.flow != 1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "L must be (a' flow -1, wl flow +1, a flow +1) on x's left bond");
    if (!check_index(R->idx[0], beta, -1) || !check_index(R->idx[2], beta, 1) || chr.flow != 1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "R must be (b' flow -1, wr flow +1, b flow +1) on x's right bond");
    if (!check_index(W1->idx[0], chl, 1) || !check_index(W1->idx[1], ph1, 1) ||
        !check_index(W1->idx[2], ph1, -1) || chm.flow != -1)
        return fail(HEFF_ERR_CHARGE_MISMATCH, "W1 must be (wl +1, t1 +1, s1 -1, wm -1) matching L and x");
    if (!W2->idx[0].same_sectors(chm) || W2->idx[0].flow != 1 || !check_index(W2->idx[1], ph2, 1) ||
        !check_index(W2->idx[2], ph2, -1) || !check_index(W2->idx[3], chr, -1))
        return fail(HEFF_ERR_CHARGE_MISMATCH, "W2 must be (wm +1, t2 +1, s2 -1, wr -1) matching W1, x, R");
    for (const IndexDesc* c : {&chl, &chm, &chr})
        for (int s = 0; s < c->nsec; ++s) if (c->dims[s] != 1)
            return fail(HEFF_ERR_CHARGE_MISMATCH, "MPO channel sectors must have dimension 1");
    for (const heff_layout* t : {L, R, W1, W2})
        for (int c = 0; c < nq; ++c) if (t->target[c] != 0)
            return fail(HEFF_ERR_CHARGE_MISMATCH, "L, R, W1, W2 must have target charge 0");
    for (const IndexDesc* b : {&alpha, &beta, &ph1, &ph2})
        for (int s = 0; s < b->nsec; ++s)
            if (b->find(b->q(s)) != s)
                return fail(HEFF_ERR_INVALID_ARG, "bond and physical sectors must have distinct charges");

    heff_plan* P = new (std::nothrow) heff_plan();
    if (!P) return fail(HEFF_ERR_OOM, "out of host memory");
    P->opts = *opts;
    switch (opts->precision) {
        case HEFF_PREC_FP64: P->planes = 1; P->esize = 8; break;
        case HEFF_PREC_BF16X3: P->planes = 2; P->esize = 2; break;
        default: P->planes = 2; P->esize = 4; break;
    }
    P->nelem_x = x->nelem; P->nelem_L = L->nelem; P->nelem_R = R->nelem;
    P->nelem_W1 = W1->nelem; P->nelem_W2 = W2->nelem;
    for (int64_t e = 0; e < W1->nelem; ++e) if (W1_host[e] == 0.0) P->w1_zero.push_back((int32_t)e);
    for (int64_t e = 0; e < W2->nelem; ++e) if (W2_host[e] == 0.0) P->w2_zero.push_back((int32_t)e);

    try {
        const int na = alpha.nsec, nb = beta.nsec, d1 = ph1.nsec, d2 = ph2.nsec;
        const int kl = chl.nsec, km = chm.nsec, kr = chr.nsec;
        const Charge target = x->target;
        // ---- charge sectors of the two-site matrix (a s1) x (s2 b)
        std::map<Charge, int> qid;
        std::vector<QSec> Q;
        std::map<Charge, std::vector<CGroup>> cmap, emap;
        for (int s1 = 0; s1 < d1; ++s1)
            for (int i = 0; i < na; ++i)
                cmap[add(alpha.q(i), ph1.q(s1))].push_back({s1, i, alpha.dims[i], 0, 0});
        for (int s2 = 0; s2 < d2; ++s2)
            for (int j = 0; j < nb; ++j)
                emap[add(add(beta.q(j), ph2.q(s2), -1), target)].push_back({s2, j, beta.dims[j], 0, 0});
        for (auto& kv : cmap) {
            auto it = emap.find(kv.first);
            if (it == emap.end()) continue;
            QSec qs;
            qs.q = kv.first;
            qs.cg = kv.second;
            qs.eg = it->second;
            qid[qs.q] = (int)Q.size();
            Q.push_back(std::move(qs));
        }
        int64_t ld_x = KPAD, rows_x = 0;
        for (auto& qs : Q) {
            int32_t col = 0, row = 0;
            for (auto& g : qs.cg) { g.col = col; g.row = row; col += (int32_t)pad_up(g.dim, KPAD); row += g.dim; }
            qs.kc = col;
            qs.mrows = row;
            row = 0;
            for (auto& g : qs.eg) { g.row = row; row += g.dim; }
            qs.nrows = row;
            qs.xt_row0 = rows_x;
            rows_x += qs.nrows;
            ld_x = std::max<int64_t>(ld_x, qs.kc);
        }
        // ---- MPO entries kept by the schedule (nonzero in the host copies)
        auto w_index = [&](const heff_layout* W, const double* host, int a, int b, int c, int d) -> int32_t {
            int64_t off = W->offset_of({a, b, c, d});
            if (off < 0 || host[off] == 0.0) return -1;
            return (int32_t)off;
        };
        std::vector<int32_t> w1i((size_t)kl * d1 * d1 * km), w2i((size_t)km * d2 * d2 * kr);
        for (int a = 0; a < kl; ++a) for (int t = 0; t < d1; ++t) for (int s = 0; s < d1; ++s)
            for (int m = 0; m < km; ++m) w1i[((a * d1 + t) * d1 + s) * km + m] = w_index(W1, W1_host, a, t, s, m);
        for (int m = 0; m < km; ++m) for (int t = 0; t < d2; ++t) for (int s = 0; s < d2; ++s)
            for (int r = 0; r < kr; ++r) w2i[((m * d2 + t) * d2 + s) * kr + r] = w_index(W2, W2_host, m, t, s, r);
        auto W1i = [&](int a, int t, int s, int m) { return w1i[((a * d1 + t) * d1 + s) * km + m]; };
        auto W2i = [&](int m, int t, int s, int r) { return w2i[((m * d2 + t) * d2 + s) * kr + r]; };

        // ---- charge arithmetic and block lookups as tables (sector charges are distinct, so
        // q(a) + q(wl) == q(a') is a_plus_l[a][wl] == a'), for the row-group loops below
        std::vector<int> a_plus_l((size_t)na * kl), b_plus_r((size_t)nb * kr);
        for (int a = 0; a < na; ++a)
            for (int w = 0; w < kl; ++w) a_plus_l[(size_t)a * kl + w] = alpha.find(add(alpha.q(a), chl.q(w)));
        for (int b = 0; b < nb; ++b)
            for (int w = 0; w < kr; ++w) b_plus_r[(size_t)b * kr + w] = beta.find(add(beta.q(b), chr.q(w)));
        std::vector<int64_t> loff((size_t)na * kl * na, -1), roff((size_t)nb * kr * nb, -1);   // -1: no block
        for (size_t blk = 0; blk < L->offsets.size(); ++blk) {
            const int32_t* k = &L->keys[blk * 3];
            loff[((size_t)k[0] * kl + k[1]) * na + k[2]] = L->offsets[blk];
        }
        for (size_t blk = 0; blk < R->offsets.size(); ++blk) {
            const int32_t* k = &R->keys[blk * 3];
            roff[((size_t)k[0] * kr + k[1]) * nb + k[2]] = R->offsets[blk];
        }

        // ---- canonical flop count (the oracle's two-contraction list algorithm), also per
        // output left sector a' (for the row shards)
        std::vector<double> canon1_ip, canon2_ip;
        {
            // structural pattern of W12 = sum_wm W1 W2 : feeds[(wl,s1,s2)] -> set (t1,t2,wr)
            std::map<std::tuple<int, int, int>, std::set<std::tuple<int, int, int>>> feeds;
            for (int a = 0; a < kl; ++a) for (int t1 = 0; t1 < d1; ++t1) for (int s1 = 0; s1 < d1; ++s1)
                for (int m = 0; m < km; ++m) {
                    if (W1i(a, t1, s1, m) < 0) continue;
                    for (int t2 = 0; t2 < d2; ++t2) for (int s2 = 0; s2 < d2; ++s2) for (int r = 0; r < kr; ++r)
                        if (W2i(m, t2, s2, r) >= 0) feeds[{a, s1, s2}].insert({t1, t2, r});
                }
            std::map<int, std::vector<std::pair<int, int>>> L_by_ket;   // i -> (ip, wl)
            for (size_t b = 0; b < L->offsets.size(); ++b)
                L_by_ket[L->keys[b * 3 + 2]].push_back({L->keys[b * 3 + 0], L->keys[b * 3 + 1]});
            std::map<std::pair<int, int>, std::vector<int>> R_by_ket;   // (wr, j) -> jp
            for (size_t b = 0; b < R->offsets.size(); ++b)
                R_by_ket[{R->keys[b * 3 + 1], R->keys[b * 3 + 2]}].push_back(R->keys[b * 3 + 0]);
            double g1 = 0, g2 = 0;
            canon1_ip.assign(na, 0.0);
            canon2_ip.assign(na, 0.0);
            // the distinct Z blocks (a', t1, t2, wr, b): a dense flag array walked in index
            // (= lexicographic) order, or an ordered set when that domain is very large
            const size_t zdom = (size_t)na * d1 * d2 * kr * nb;
            const bool zdense = zdom <= ((size_t)1 << 26);
            std::vector<char> zseen(zdense ? zdom : 0, 0);
            std::set<std::tuple<int, int, int, int, int>> zkeys;
            for (size_t b = 0; b < x->offsets.size(); ++b) {
                int i = x->keys[b * 4], s1 = x->keys[b * 4 + 1], s2 = x->keys[b * 4 + 2], j = x->keys[b * 4 + 3];
                auto lk = L_by_ket.find(i);
                if (lk == L_by_ket.end()) continue;
                for (auto& pw : lk->second) {
                    auto f = feeds.find({pw.second, s1, s2});
                    if (f == feeds.end() || f->second.empty()) continue;
                    g1 += 2.0 * alpha.dims[pw.first] * alpha.dims[i] * beta.dims[j];
                    canon1_ip[pw.first] += 2.0 * alpha.dims[pw.first] * alpha.dims[i] * beta.dims[j];
                    for (auto& t : f->second) {
                        if (zdense)
                            zseen[((((size_t)pw.first * d1 + std::get<0>(t)) * d2 + std::get<1>(t)) * kr +
                                   std::get<2>(t)) * nb + j] = 1;
                        else
                            zkeys.insert({pw.first, std::get<0>(t), std::get<1>(t), std::get<2>(t), j});
                    }
                }
            }
            auto zflops = [&](int ip, int wr, int j) {
                auto rk = R_by_ket.find({wr, j});
                if (rk == R_by_ket.end()) return;
                for (int jp : rk->second) {
                    const double f = 2.0 * alpha.dims[ip] * beta.dims[j] * beta.dims[jp];
                    g2 += f;
                    canon2_ip[ip] += f;
                }
            };
            if (zdense) {
                for (size_t z = 0; z < zdom; ++z) {
                    if (!zseen[z]) continue;
                    const int j = (int)(z % nb), wr = (int)(z / nb % kr);
                    zflops((int)(z / ((size_t)nb * kr * d2 * d1)), wr, j);
                }
            } else {
                for (auto& z : zkeys) zflops(std::get<0>(z), std::get<3>(z), std::get<4>(z));
            }
            P->flops_canonical = g1 + g2;
            P->stats[16] = (int64_t)g1;
            P->stats[17] = (int64_t)g2;
        }

        // ---- LW row groups (GEMM 1 rows)
        std::vector<RowGroup> rgs;
        std::map<std::tuple<int, int, int>, int> rg_of;   // (q, t1, wm) -> row group
        int64_t rows_lw = 0;
        for (int q = 0; q < (int)Q.size(); ++q)
            for (int t1 = 0; t1 < d1; ++t1)
                for (int wm = 0; wm < km; ++wm) {
                    int ip = alpha.find(add(add(Q[q].q, chm.q(wm)), ph1.q(t1), -1));
                    if (ip < 0) continue;
                    RowGroup rg{q, t1, wm, ip, 0, {}};
                    for (int c = 0; c < (int)Q[q].cg.size(); ++c) {
                        const CGroup& g = Q[q].cg[c];
                        RowGroup::Seg seg{c, {}};
                        for (int wl = 0; wl < kl; ++wl) {
                            if (a_plus_l[(size_t)g.sec * kl + wl] != ip) continue;
                            int32_t wi = W1i(wl, t1, g.s, wm);
                            if (wi < 0) continue;
                            int64_t off = loff[((size_t)ip * kl + wl) * na + g.sec];
                            if (off < 0) continue;
                            seg.terms.push_back({off, wi, 0});
                        }
                        if (!seg.terms.empty()) rg.segs.push_back(std::move(seg));
                    }
                    if (rg.segs.empty()) continue;
                    rg.lw_row0 = rows_lw;
                    rows_lw += alpha.dims[ip];
                    rg_of[{q, t1, wm}] = (int)rgs.size();
                    rgs.push_back(std::move(rg));
                }
        // ---- RW row groups (GEMM 2 columns) and the segments they need
        std::vector<int> q_minus_m((size_t)Q.size() * km, -1);         // sector of Q - q(wm)
        for (int q = 0; q < (int)Q.size(); ++q)
            for (int wm = 0; wm < km; ++wm) {
                auto qi = qid.find(add(Q[q].q, chm.q(wm), -1));
                if (qi != qid.end()) q_minus_m[(size_t)q * km + wm] = qi->second;
            }
        std::vector<RWGroup> rws;
        std::vector<std::set<std::pair<int, int>>> used(Q.size());     // per Q': (wm, src flat eg id)
        for (int q = 0; q < (int)Q.size(); ++q)
            for (int e = 0; e < (int)Q[q].eg.size(); ++e) {
                const CGroup& ge = Q[q].eg[e];                           // (t2, j')
                RWGroup rw{q, e, {}};
                for (int wm = 0; wm < km; ++wm) {
                    const int qsrc = q_minus_m[(size_t)q * km + wm];
                    if (qsrc < 0) continue;
                    const QSec& qs = Q[qsrc];
                    for (int f = 0; f < (int)qs.eg.size(); ++f) {
                        const CGroup& gs = qs.eg[f];                     // (s2, j)
                        RWGroup::Seg seg{wm, qsrc, f, {}};
                        for (int wr = 0; wr < kr; ++wr) {
                            if (b_plus_r[(size_t)gs.sec * kr + wr] != ge.sec) continue;
                            int32_t wi = W2i(wm, ge.s, gs.s, wr);
                            if (wi < 0) continue;
                            int64_t off = roff[((size_t)ge.sec * kr + wr) * nb + gs.sec];
                            if (off < 0) continue;
                            seg.terms.push_back({off, wi, 0});
                        }
                        if (!seg.terms.empty()) {
                            used[q].insert({wm, f});
                            rw.segs.push_back(std::move(seg));
                        }
                    }
                }
                rws.push_back(std::move(rw));
            }
        // ---- T column layout per Q': segments (wm, e-group of Q'-q(wm)) produced and consumed
        auto present = [&](int qsrc, int t1, int wm) { return rg_of.count({qsrc, t1, wm}) > 0; };
        int64_t ld_t = KPAD, rows_t = 0, rows_rw = 0;
        for (int q = 0; q < (int)Q.size(); ++q) {
            QSec& qs = Q[q];
            int32_t col = 0;
            for (auto& u : used[q]) {
                int wm = u.first, f = u.second;
                auto qi = qid.find(add(qs.q, chm.q(wm), -1));
                bool any = false;
                for (int t1 = 0; t1 < d1 && !any; ++t1) any = present(qi->second, t1, wm);
                if (!any) continue;
                qs.toff[{wm, f}] = col;
                col += (int32_t)pad_up(Q[qi->second].eg[f].dim, KPAD);
            }
            qs.kt = col;
            ld_t = std::max<int64_t>(ld_t, col);
            qs.t_row0 = rows_t;
            rows_t += qs.mrows;
            qs.rw_row0 = rows_rw;
            rows_rw += qs.nrows;
        }
        // dense forms of the lookups the task-list loops repeat: row groups present,
        // T column offsets (-1: none), Q + q(wm), and x's block offsets
        std::vector<char> present_tab((size_t)Q.size() * d1 * km, 0);
        for (auto& kv : rg_of)
            present_tab[((size_t)std::get<0>(kv.first) * d1 + std::get<1>(kv.first)) * km + std::get<2>(kv.first)] = 1;
        std::vector<size_t> toff_base((size_t)Q.size() * km + 1, 0);
        for (int q = 0; q < (int)Q.size(); ++q)
            for (int wm = 0; wm < km; ++wm) {
                const int qs_ = q_minus_m[(size_t)q * km + wm];
                toff_base[(size_t)q * km + wm + 1] = toff_base[(size_t)q * km + wm] + (qs_ >= 0 ? Q[qs_].eg.size() : 0);
            }
        std::vector<int32_t> toff_flat(toff_base.back(), -1);
        for (int q = 0; q < (int)Q.size(); ++q)
            for (auto& kv : Q[q].toff) toff_flat[toff_base[(size_t)q * km + kv.first.first] + kv.first.second] = kv.second;
        std::vector<int> q_plus_m((size_t)Q.size() * km, -1);
        for (int q = 0; q < (int)Q.size(); ++q)
            for (int wm = 0; wm < km; ++wm) {
                auto qi = qid.find(add(Q[q].q, chm.q(wm)));
                if (qi != qid.end()) q_plus_m[(size_t)q * km + wm] = qi->second;
            }
        std::vector<int64_t> xoff((size_t)na * d1 * d2 * nb, -1);
        for (size_t blk = 0; blk < x->offsets.size(); ++blk) {
            const int32_t* k = &x->keys[blk * 4];
            xoff[(((size_t)k[0] * d1 + k[1]) * d2 + k[2]) * nb + k[3]] = x->offsets[blk];
        }
        P->rows_x = rows_x; P->ld_x = ld_x; P->rows_lw = std::max<int64_t>(rows_lw, 1);
        P->rows_t = std::max<int64_t>(rows_t, 1); P->ld_t = ld_t; P->rows_rw = std::max<int64_t>(rows_rw, 1);

        // ---- pack tiles (x -> XT)
        for (size_t b = 0; b < x->offsets.size(); ++b) {
            int i = x->keys[b * 4], s1 = x->keys[b * 4 + 1], s2 = x->keys[b * 4 + 2], j = x->keys[b * 4 + 3];
            const QSec& qs = Q[qid.at(add(alpha.q(i), ph1.q(s1)))];
            const CGroup* cg = nullptr; const CGroup* eg = nullptr;
            for (auto& g : qs.cg) if (g.s == s1 && g.sec == i) cg = &g;
            for (auto& g : qs.eg) if (g.s == s2 && g.sec == j) eg = &g;
            if (!cg || !eg) { delete P; return fail(HEFF_ERR_CHARGE_MISMATCH, "internal: x block outside the sector map"); }
            int apad = (int)pad_up(cg->dim, KPAD);
            for (int a0 = 0; a0 < apad; a0 += 32)
                for (int b0 = 0; b0 < eg->dim; b0 += 32)
                    P->pack.push_back({x->offsets[b], qs.xt_row0 + eg->row, cg->col, cg->dim, eg->dim, apad, a0, b0});
        }
        // ---- mix tiles (LW and RW)
        const int MIX_ROWS = 32;
        for (auto& rg : rgs)
            for (auto& sg : rg.segs) {
                const CGroup& g = Q[rg.q].cg[sg.cg];
                int32_t tb = (int32_t)P->terms.size();
                P->terms.insert(P->terms.end(), sg.terms.begin(), sg.terms.end());
                int rows = alpha.dims[rg.ip];
                for (int r0 = 0; r0 < rows; r0 += MIX_ROWS)
                    P->mix.push_back({rg.lw_row0, g.col, rows, g.dim, (int32_t)pad_up(g.dim, KPAD), r0,
                                      std::min(MIX_ROWS, rows - r0), tb, (int32_t)sg.terms.size(), 0});
            }
        for (auto& rw : rws) {
            const QSec& qs = Q[rw.q];
            const CGroup& ge = qs.eg[rw.eg];
            for (auto& sg : rw.segs) {
                auto it = qs.toff.find({sg.wm, sg.eg_src});
                if (it == qs.toff.end()) continue;        // nothing in T multiplies it
                const CGroup& gs = Q[sg.q_src].eg[sg.eg_src];
                int32_t tb = (int32_t)P->terms.size();
                P->terms.insert(P->terms.end(), sg.terms.begin(), sg.terms.end());
                int rows = ge.dim;
                for (int r0 = 0; r0 < rows; r0 += MIX_ROWS)
                    P->mix.push_back({qs.rw_row0 + ge.row, it->second, rows, gs.dim, (int32_t)pad_up(gs.dim, KPAD),
                                      r0, std::min(MIX_ROWS, rows - r0), tb, (int32_t)sg.terms.size(), 1});
            }
        }
        // ---- SMs of the current device (the persistent kernels' width; 148 without one)
        int nsm = 148;
        {
            int ndev = 0, dev = 0, v = 0;
            if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0 && cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
                nsm = v;
            cudaGetLastError();
        }
        // ---- GEMM task lists for one tile shape TM x TN
        auto build_lists = [&](int TM, int TN, heff::GemmList& G1, heff::GemmList& G2) -> bool {
        G1.tm = G2.tm = TM;
        G1.tn = G2.tn = TN;
        // GEMM 1: rows of a row group x columns of one e-group, written into T
        for (auto& rg : rgs) {
            const QSec& qs = Q[rg.q];
            const int qpi = q_plus_m[(size_t)rg.q * km + rg.wm];
            if (qpi < 0) continue;
            const QSec& qp = Q[qpi];
            const CGroup* crow = nullptr;
            for (auto& g : qp.cg) if (g.s == rg.t1 && g.sec == rg.ip) crow = &g;
            if (!crow) continue;
            int32_t sb = (int32_t)G1.segs.size();
            int64_t klen = 0, kuse = 0;
            for (auto& sg : rg.segs) {
                const CGroup& g = qs.cg[sg.cg];
                G1.segs.push_back({g.col, (int32_t)pad_up(g.dim, KPAD)});
                klen += pad_up(g.dim, KPAD);
                kuse += g.dim;
            }
            int32_t sc = (int32_t)rg.segs.size();
            const int mi = alpha.dims[rg.ip];
            for (int f = 0; f < (int)qs.eg.size(); ++f) {
                const int32_t tcol = toff_flat[toff_base[(size_t)qpi * km + rg.wm] + f];
                if (tcol < 0) continue;
                const CGroup& ge = qs.eg[f];
                for (int m0 = 0; m0 < mi; m0 += TM)
                    for (int n0 = 0; n0 < ge.dim; n0 += TN) {
                        heff::GemmTask t{};
                        t.a_row = rg.lw_row0 + m0;
                        t.b_row = qs.xt_row0 + ge.row + n0;
                        t.m = std::min(TM, mi - m0);
                        t.n = std::min(TN, ge.dim - n0);
                        t.c_off = (qp.t_row0 + crow->row + m0) * ld_t + tcol + n0;
                        t.ldc = (int32_t)ld_t;
                        t.n_zero = (n0 + TN >= ge.dim) ? (int32_t)(pad_up(ge.dim, KPAD) - ge.dim) : 0;
                        t.seg_begin = sb;
                        t.seg_count = sc;
                        t.ktotal = (int32_t)klen;
                        G1.tasks.push_back(t);
                        G1.owner.push_back(rg.ip);
                        G1.task_flops.push_back(2.0 * t.m * t.n * klen);
                        G1.task_useful.push_back(2.0 * t.m * t.n * kuse);
                    }
            }
        }
        // GEMM 2: rows of a c'-group (t1, i') x rows of an RW group (t2, j'), written into y
        for (auto& rw : rws) {
            const QSec& qs = Q[rw.q];
            const CGroup& ge = qs.eg[rw.eg];
            for (auto& gc : qs.cg) {
                int32_t sb = (int32_t)G2.segs.size();
                int64_t klen = 0, kuse = 0;
                for (auto& sg : rw.segs) {
                    if (!present_tab[((size_t)sg.q_src * d1 + gc.s) * km + sg.wm]) continue;
                    const int32_t tcol = toff_flat[toff_base[(size_t)rw.q * km + sg.wm] + sg.eg_src];
                    if (tcol < 0) continue;
                    int32_t len = (int32_t)pad_up(Q[sg.q_src].eg[sg.eg_src].dim, KPAD);
                    G2.segs.push_back({tcol, len});
                    klen += len;
                    kuse += Q[sg.q_src].eg[sg.eg_src].dim;
                }
                int32_t sc = (int32_t)G2.segs.size() - sb;
                int64_t yoff = xoff[(((size_t)gc.sec * d1 + gc.s) * d2 + ge.s) * nb + ge.sec];
                if (yoff < 0) return false;
                for (int m0 = 0; m0 < gc.dim; m0 += TM)
                    for (int n0 = 0; n0 < ge.dim; n0 += TN) {
                        heff::GemmTask t{};
                        t.a_row = qs.t_row0 + gc.row + m0;
                        t.b_row = qs.rw_row0 + ge.row + n0;
                        t.m = std::min(TM, gc.dim - m0);
                        t.n = std::min(TN, ge.dim - n0);
                        t.c_off = yoff + (int64_t)m0 * ge.dim + n0;
                        t.ldc = ge.dim;
                        t.n_zero = 0;
                        t.seg_begin = sb;
                        t.seg_count = sc;
                        t.ktotal = (int32_t)klen;
                        G2.tasks.push_back(t);
                        G2.owner.push_back(gc.sec);
                        G2.task_flops.push_back(2.0 * t.m * t.n * klen);
                        G2.task_useful.push_back(2.0 * t.m * t.n * kuse);
                    }
            }
        }
        // longest tasks first (LPT order for the persistent kernels); a tile's tensor time
        // scales with its padded K and its MMA width (n rounded up to 16)
        for (heff::GemmList* g : {&G1, &G2}) {
            const int model = g == &G1 ? HEFF_TILE_COST_G1 : HEFF_TILE_COST_G2;
            std::vector<int64_t> work(g->tasks.size());
            std::vector<size_t> ord(g->tasks.size());
            for (size_t t = 0; t < g->tasks.size(); ++t) {
                int64_t k = 0;
                for (int s = 0; s < g->tasks[t].seg_count; ++s) k += g->segs[g->tasks[t].seg_begin + s].klen;
                work[t] = k * tile_width_cost(g->tasks[t].m, g->tasks[t].n, model);
                ord[t] = t;
            }
            std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
            heff::GemmList s;
            for (size_t t : ord) {
                s.tasks.push_back(g->tasks[t]);
                s.owner.push_back(g->owner[t]);
                s.task_flops.push_back(g->task_flops[t]);
                s.task_useful.push_back(g->task_useful[t]);
            }
            g->tasks.swap(s.tasks);
            g->owner.swap(s.owner);
            g->task_flops.swap(s.task_flops);
            g->task_useful.swap(s.task_useful);
        }
        return true;
        };
        // keep the tasks of the owned left sectors and total their flops
        auto keep_owned = [&](heff::GemmList& G, const std::vector<char>& owned) {
            heff::GemmList s;
            for (size_t t = 0; t < G.tasks.size(); ++t) {
                if (!owned[G.owner[t]]) continue;
                s.tasks.push_back(G.tasks[t]);
                s.owner.push_back(G.owner[t]);
                s.task_flops.push_back(G.task_flops[t]);
                s.task_useful.push_back(G.task_useful[t]);
            }
            G.tasks.swap(s.tasks);
            G.owner.swap(s.owner);
            G.task_flops.swap(s.task_flops);
            G.task_useful.swap(s.task_useful);
            G.flops = G.useful = 0;
            for (size_t t = 0; t < G.tasks.size(); ++t) { G.flops += G.task_flops[t]; G.useful += G.task_useful[t]; }
        };
        const bool tc = opts->precision != HEFF_PREC_FP64;
        if (!build_lists(tc ? 128 : 64, tc ? 256 : 64, P->g1, P->g2) ||
            (tc && !build_lists(128, 128, P->g1_alt, P->g2_alt))) {
            delete P;
            return fail(HEFF_ERR_CHARGE_MISMATCH, "internal: y block missing");
        }
        // ---- row shards: left sectors a' of y assigned to shards by longest-processing-time
        // over their executed GEMM flops (ties: lower sector, then lower shard), identical for
        // every shard index; this plan keeps the work of its own sectors
        std::vector<char> owned(na, 1);
        if (opts->shard_count > 1) {
            std::vector<double> work(na, 0.0);
            for (const heff::GemmList* G : {&P->g1, &P->g2})
                for (size_t t = 0; t < G->tasks.size(); ++t) work[G->owner[t]] += G->task_flops[t];
            std::vector<int> ord(na);
            for (int i = 0; i < na; ++i) ord[i] = i;
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return work[a] > work[b]; });
            std::vector<double> load(opts->shard_count, 0.0);
            for (int i : ord) {
                int best = 0;
                for (int r = 1; r < opts->shard_count; ++r) if (load[r] < load[best]) best = r;
                load[best] += work[i];
                owned[i] = best == opts->shard_index;
            }
            std::set<int64_t> lw_rows;   // LW row groups of owned sectors
            for (auto& rg : rgs) if (owned[rg.ip]) lw_rows.insert(rg.lw_row0);
            std::vector<heff::MixTile> mix;
            for (auto& mt : P->mix)
                if (mt.which != 0 || lw_rows.count(mt.dst_row0)) mix.push_back(mt);
            P->mix.swap(mix);
            double c1 = 0, c2 = 0;
            for (int i = 0; i < na; ++i) if (owned[i]) { c1 += canon1_ip[i]; c2 += canon2_ip[i]; }
            P->flops_canonical = c1 + c2;
            P->stats[16] = (int64_t)c1;
            P->stats[17] = (int64_t)c2;
        }
        for (heff::GemmList* G : {&P->g1, &P->g2, &P->g1_alt, &P->g2_alt}) keep_owned(*G, owned);
        // ---- CTA pairs (tensor-core paths): N = 256 tiles with the same B rows, width and K
        // segments go two to an entry, so that one read of each B box serves both CTAs of a
        // cluster.  A tile left without a partner gets a ghost (no rows: it loads its half of
        // B and computes nothing); tiles without segments (zero output blocks) pair among
        // themselves or with an empty task.
        auto make_pairs = [&](const heff::GemmList& G, heff::GemmList& Pr) {
            Pr = heff::GemmList{};
            Pr.tm = G.tm; Pr.tn = G.tn; Pr.cl = 2;
            Pr.segs = G.segs;
            Pr.flops = G.flops; Pr.useful = G.useful;
            auto push = [&](const heff::GemmTask& k, int32_t owner, double f, double u) {
                Pr.tasks.push_back(k); Pr.owner.push_back(owner);
                Pr.task_flops.push_back(f); Pr.task_useful.push_back(u);
            };
            auto push_task = [&](size_t t) { push(G.tasks[t], G.owner[t], G.task_flops[t], G.task_useful[t]); };
            std::map<std::vector<int64_t>, std::vector<size_t>> groups;
            std::vector<size_t> zero;
            for (size_t t = 0; t < G.tasks.size(); ++t) {
                const heff::GemmTask& k = G.tasks[t];
                if (k.seg_count == 0) { zero.push_back(t); continue; }
                std::vector<int64_t> key = {k.b_row, k.n, k.ktotal};
                for (int j = 0; j < k.seg_count; ++j) {
                    key.push_back(G.segs[k.seg_begin + j].k0);
                    key.push_back(G.segs[k.seg_begin + j].klen);
                }
                groups[key].push_back(t);
            }
            for (auto& kv : groups) {
                const std::vector<size_t>& v = kv.second;
                for (size_t i = 0; i < v.size(); i += 2) {
                    push_task(v[i]);
                    if (i + 1 < v.size()) {
                        push_task(v[i + 1]);
                    } else {
                        heff::GemmTask gh = G.tasks[v[i]];
                        gh.m = 0; gh.n_zero = 0; gh.c_off = 0;
                        push(gh, -1, 0.0, 0.0);
                    }
                }
            }
            for (size_t i = 0; i < zero.size(); i += 2) {
                push_task(zero[i]);
                if (i + 1 < zero.size()) {
                    push_task(zero[i + 1]);
                } else {
                    heff::GemmTask e{};
                    e.ldc = 1;
                    push(e, -1, 0.0, 0.0);
                }
            }
        };
        int ncl = nsm / 2;
        if (tc) {
            make_pairs(P->g1, P->g1_pair);
            make_pairs(P->g2, P->g2_pair);
            int ndev = 0;
            if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) ncl = heff::tc_pair_clusters(nsm, opts->precision);
            cudaGetLastError();
        }
        // ---- static schedule of the persistent tensor-core kernels: CTA c of a grid of
        // min(nsm, tasks) runs tasks c, c + grid, c + 2 grid, ...  Assign the tasks by
        // longest-processing-time (each to the least loaded CTA, longest first; a tile's
        // time ~ (K blocks + a fixed overhead) x MMA width) and interleave the per-CTA lists
        // in that pattern, padding short lists with empty tasks (no rows, no segments).
        // CTA pairs are scheduled the same way, an entry (two tasks) per cluster.
        if (tc && HEFF_LPT_SCHEDULE) {
            for (heff::GemmList* G : {&P->g1, &P->g2, &P->g1_alt, &P->g2_alt, &P->g1_pair, &P->g2_pair}) {
                const int model = (G == &P->g1 || G == &P->g1_alt || G == &P->g1_pair) ? HEFF_TILE_COST_G1
                                                                                        : HEFF_TILE_COST_G2;
                const size_t CLn = (size_t)G->cl;
                const size_t nt = G->tasks.size() / CLn;          // entries
                if (nt == 0) continue;
                const int grid = (int)std::min<size_t>((size_t)(CLn == 2 ? ncl : nsm), nt);
                std::vector<double> work(nt, 0.0);
                for (size_t t = 0; t < nt; ++t)
                    for (size_t r = 0; r < CLn; ++r) {
                        const heff::GemmTask& k = G->tasks[t * CLn + r];
                        work[t] = std::max(work[t], (double)(k.ktotal / KPAD + 4) * tile_width_cost(k.m, k.n, model));
                    }
                std::vector<size_t> ord(nt);
                for (size_t t = 0; t < nt; ++t) ord[t] = t;
                std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
                // least loaded CTA first, the lowest index among equal loads (a min-heap on
                // (load, CTA): O(tasks log grid))
                std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>,
                                    std::greater<std::pair<double, int>>> heap;
                for (int c = 0; c < grid; ++c) heap.push({0.0, c});
                std::vector<std::vector<size_t>> per(grid);
                for (size_t t : ord) {
                    const std::pair<double, int> top = heap.top();
                    heap.pop();
                    per[top.second].push_back(t);
                    heap.push({top.first + work[t], top.second});
                }
                size_t depth = 0;
                for (auto& v : per) depth = std::max(depth, v.size());
                heff::GemmList s2;
                for (size_t j = 0; j < depth; ++j)
                    for (int c = 0; c < grid; ++c)
                        for (size_t r = 0; r < CLn; ++r) {
                            if (j < per[c].size()) {
                                const size_t t = per[c][j] * CLn + r;
                                s2.tasks.push_back(G->tasks[t]);
                                s2.owner.push_back(G->owner[t]);
                                s2.task_flops.push_back(G->task_flops[t]);
                                s2.task_useful.push_back(G->task_useful[t]);
                            } else {
                                heff::GemmTask e{};
                                e.ldc = 1;
                                s2.tasks.push_back(e);
                                s2.owner.push_back(-1);
                                s2.task_flops.push_back(0.0);
                                s2.task_useful.push_back(0.0);
                            }
                        }
                G->tasks.swap(s2.tasks);
                G->owner.swap(s2.owner);
                G->task_flops.swap(s2.task_flops);
                G->task_useful.swap(s2.task_useful);
            }
        }
        for (int i = 0; i < na; ++i) if (owned[i]) P->shard_sectors.push_back(i);
        const int TM = P->g1.tm, TN = P->g1.tn;
        // ---- workspace layout
        auto al = [](size_t v) { return (v + 255) / 256 * 256; };
        const size_t e = (size_t)P->esize * P->planes;
        size_t off = 0;
        P->off_xt = off; off = al(off + e * (size_t)opts->max_batch * P->rows_x * P->ld_x);
        P->off_lw = off; off = al(off + e * (size_t)P->rows_lw * P->ld_x);
        P->off_t = off;  off = al(off + e * (size_t)opts->max_batch * P->rows_t * P->ld_t);
        P->off_rw = off; off = al(off + e * (size_t)P->rows_rw * P->ld_t);
        P->off_flags = off; off = al(off + 256);
        P->ws_bytes = off;
        int64_t* st = P->stats;
        st[0] = (int64_t)Q.size(); st[1] = (int64_t)rgs.size(); st[2] = (int64_t)rws.size();
        st[3] = (int64_t)P->g1.tasks.size(); st[4] = (int64_t)P->g2.tasks.size();
        st[5] = (int64_t)P->pack.size(); st[6] = (int64_t)P->mix.size(); st[7] = (int64_t)P->terms.size();
        st[8] = P->rows_x; st[9] = P->ld_x; st[10] = P->rows_lw; st[11] = P->rows_t; st[12] = P->ld_t;
        st[13] = P->rows_rw; st[14] = TM; st[15] = TN; st[22] = TN;
        st[18] = (int64_t)P->g1.useful; st[19] = (int64_t)P->g2.useful;
        st[20] = (int64_t)P->g1.flops; st[21] = (int64_t)P->g2.flops;
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(HEFF_ERR_OOM, "out of host memory while planning");
    } catch (const std::out_of_range&) {
        delete P;
        return fail(HEFF_ERR_CHARGE_MISMATCH, "internal: charge sector lookup failed");
    }
    int rc = heff::plan_upload(P);
    if (rc != HEFF_OK) {
        heff::plan_free_device(P);
        delete P;
        return rc;
    }
    *out = P;
    return HEFF_OK;
}

extern "C" int heff_plan_shard_sectors(const heff_plan* plan, int32_t* sectors, int32_t* count) {
    heff::clear_error();
    if (!plan || !count) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_shard_sectors: null argument");
    if (sectors) std::memcpy(sectors, plan->shard_sectors.data(), plan->shard_sectors.size() * sizeof(int32_t));
    *count = (int32_t)plan->shard_sectors.size();
    return HEFF_OK;
}

extern "C" int heff_plan_workspace_size(const heff_plan* plan, size_t* bytes) {
    heff::clear_error();
    if (!plan || !bytes) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_workspace_size: null argument");
    *bytes = plan->ws_bytes;
    return HEFF_OK;
}

extern "C" int heff_plan_flops(const heff_plan* plan, double* canonical, double* executed) {
    heff::clear_error();
    if (!plan) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_flops: null plan");
    if (canonical) *canonical = plan->flops_canonical;
    if (executed) *executed = plan->g1.flops + plan->g2.flops;
    return HEFF_OK;
}

extern "C" int heff_plan_stats(const heff_plan* plan, int64_t* stats) {
    heff::clear_error();
    if (!plan || !stats) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_stats: null argument");
    std::memcpy(stats, plan->stats, sizeof(plan->stats));
    return HEFF_OK;
}

extern "C" void heff_plan_destroy(heff_plan* plan) {
    if (!plan) return;
    heff::plan_free_device(plan);
    delete plan;
}

// Copy one schedule table to host memory (for inspection and host-side tests).
// table: 0 pack tiles, 1 mix tiles, 2 mix terms, 3 GEMM-1 tasks, 4 GEMM-1 segments,
// 5 GEMM-2 tasks, 6 GEMM-2 segments.  dst may be NULL to query the size.
extern "C" int heff_plan_export(const heff_plan* plan, int32_t table, void* dst, int64_t* bytes) {
    heff::clear_error();
    if (!plan || !bytes) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_export: null argument");
    const void* src = nullptr;
    size_t n = 0;
    switch (table) {
        case 0: src = plan->pack.data(); n = plan->pack.size() * sizeof(heff::PackTile); break;
        case 1: src = plan->mix.data(); n = plan->mix.size() * sizeof(heff::MixTile); break;
        case 2: src = plan->terms.data(); n = plan->terms.size() * sizeof(heff::MixTerm); break;
        case 3: src = plan->g1.tasks.data(); n = plan->g1.tasks.size() * sizeof(heff::GemmTask); break;
        case 4: src = plan->g1.segs.data(); n = plan->g1.segs.size() * sizeof(heff::KSeg); break;
        case 5: src = plan->g2.tasks.data(); n = plan->g2.tasks.size() * sizeof(heff::GemmTask); break;
        case 6: src = plan->g2.segs.data(); n = plan->g2.segs.size() * sizeof(heff::KSeg); break;
        default: return fail(HEFF_ERR_INVALID_ARG, "unknown table %d", table);
    }
    *bytes = (int64_t)n;
    if (dst && n) std::memcpy(dst, src, n);
    return HEFF_OK;
}
