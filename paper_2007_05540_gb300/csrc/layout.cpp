// Error plumbing and quantum-number block layouts (Section II-D).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace heff {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int IndexDesc::find(const std::vector<int32_t>& qv) const {
    for (int s = 0; s < nsec; ++s) {
        bool eq = true;
        for (int c = 0; c < nq; ++c)
            if (charges[s * nq + c] != qv[c]) { eq = false; break; }
        if (eq) return s;
    }
    return -1;
}

}  // namespace heff

using heff::fail;

extern "C" const char* heff_last_error(void) { return heff::g_last_error.c_str(); }

extern "C" int64_t heff_launch_count(void) { return heff::g_launches.load(); }

extern "C" const char* heff_version(void) { return "heff-gb300 0.1 (sm_103a)"; }

// Enumerate allowed blocks depth-first in lexicographic order, pruning nothing but the
// last index, whose sector is found from the remaining charge.
static void enumerate(const heff_layout& lay, int k, std::vector<int32_t>& key,
                      std::vector<int64_t>& acc, std::vector<int32_t>& keys,
                      std::vector<int64_t>& offs, int64_t& nelem) {
    const int nidx = (int)lay.idx.size();
    const int nq = lay.nq;
    const heff::IndexDesc& ix = lay.idx[k];
    for (int s = 0; s < ix.nsec; ++s) {
        std::vector<int64_t> a2(acc);
        for (int c = 0; c < nq; ++c) a2[c] += (int64_t)ix.flow * ix.charges[s * nq + c];
        key[k] = s;
        if (k + 1 < nidx) {
            enumerate(lay, k + 1, key, a2, keys, offs, nelem);
        } else {
            bool ok = true;
            for (int c = 0; c < nq; ++c)
                if (a2[c] != lay.target[c]) { ok = false; break; }
            if (!ok) continue;
            int64_t size = 1;
            for (int j = 0; j < nidx; ++j) size *= lay.idx[j].dims[key[j]];
            keys.insert(keys.end(), key.begin(), key.end());
            offs.push_back(nelem);
            nelem += size;
        }
    }
}

extern "C" int heff_qn_block_layout(const heff_index* idx, int32_t nidx, const int32_t* target,
                                    heff_layout** out) {
    heff::clear_error();
    if (!idx || !out || nidx < 1 || nidx > 16)
        return fail(HEFF_ERR_INVALID_ARG, "heff_qn_block_layout: bad arguments (nidx=%d)", nidx);
    *out = nullptr;
    const int nq = idx[0].nq;
    if (nq < 1 || nq > 4) return fail(HEFF_ERR_INVALID_ARG, "nq must be 1..4 (got %d)", nq);
    heff_layout* lay = new (std::nothrow) heff_layout();
    if (!lay) return fail(HEFF_ERR_OOM, "out of host memory");
    lay->nq = nq;
    for (int k = 0; k < nidx; ++k) {
        const heff_index& in = idx[k];
        if (in.nq != nq || in.nsec < 1 || !in.charges || !in.dims || (in.flow != 1 && in.flow != -1)) {
            delete lay;
            return fail(HEFF_ERR_INVALID_ARG, "index %d: bad descriptor", k);
        }
        heff::IndexDesc d;
        d.nsec = in.nsec;
        d.nq = nq;
        d.flow = in.flow;
        d.charges.assign(in.charges, in.charges + (size_t)in.nsec * nq);
        d.dims.assign(in.dims, in.dims + in.nsec);
        for (int s = 0; s < d.nsec; ++s) {
            if (d.dims[s] < 1) {
                delete lay;
                return fail(HEFF_ERR_INVALID_ARG, "index %d sector %d: dimension %d < 1", k, s, d.dims[s]);
            }
        }
        lay->idx.push_back(std::move(d));
    }
    lay->target.assign(nq, 0);
    if (target) lay->target.assign(target, target + nq);
    std::vector<int32_t> key(nidx, 0);
    std::vector<int64_t> acc(nq, 0);
    try {
        enumerate(*lay, 0, key, acc, lay->keys, lay->offsets, lay->nelem);
        const int64_t nb = (int64_t)lay->offsets.size();
        for (int64_t b = 0; b < nb; ++b)
            lay->block_of.emplace(std::vector<int32_t>(lay->keys.begin() + b * nidx,
                                                       lay->keys.begin() + (b + 1) * nidx), b);
    } catch (const std::bad_alloc&) {
        delete lay;
        return fail(HEFF_ERR_OOM, "out of host memory while enumerating blocks");
    }
    *out = lay;
    return HEFF_OK;
}

extern "C" int heff_layout_info(const heff_layout* lay, int64_t* nblocks, int64_t* nelem, int32_t* nidx) {
    heff::clear_error();
    if (!lay) return fail(HEFF_ERR_INVALID_ARG, "heff_layout_info: null layout");
    if (nblocks) *nblocks = (int64_t)lay->offsets.size();
    if (nelem) *nelem = lay->nelem;
    if (nidx) *nidx = (int32_t)lay->idx.size();
    return HEFF_OK;
}

extern "C" int heff_layout_blocks(const heff_layout* lay, int32_t* keys, int64_t* offsets) {
    heff::clear_error();
    if (!lay) return fail(HEFF_ERR_INVALID_ARG, "heff_layout_blocks: null layout");
    if (keys && !lay->keys.empty()) std::memcpy(keys, lay->keys.data(), lay->keys.size() * sizeof(int32_t));
    if (offsets && !lay->offsets.empty())
        std::memcpy(offsets, lay->offsets.data(), lay->offsets.size() * sizeof(int64_t));
    return HEFF_OK;
}

extern "C" void heff_layout_destroy(heff_layout* lay) { delete lay; }
