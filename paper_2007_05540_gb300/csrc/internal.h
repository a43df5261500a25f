// Internal declarations shared by the host planner (plan.cpp, capi.cpp) and the
// CUDA translation units.  Nothing here is part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/heff.h"

namespace heff {

// Padding unit of every contraction (K) segment in the workspace operand arrays: one K
// block of the tensor-core kernel (64-byte swizzled rows: 32 bf16 or 16 fp32 elements;
// the FP64 kernel steps K by 16).  K tiles never straddle segments.
#ifndef HEFF_KPAD
#define HEFF_KPAD 32
#endif
constexpr int KPAD = HEFF_KPAD;

inline int64_t pad_up(int64_t v, int64_t p) { return (v + p - 1) / p * p; }

// Programmatic dependent launch of the matvec's kernels (pack, GEMM 1, GEMM 2): each may be
// scheduled while its predecessor on the stream finishes, runs its prologue (barriers,
// tensor memory), and waits (griddepcontrol.wait) before it touches global memory that
// the predecessor or earlier work writes or reads.  0 launches them in plain stream order.
#ifndef HEFF_PDL
#define HEFF_PDL 1
#endif

int fail(int code, const char* fmt, ...);
void clear_error();
void count_launches(int64_t n);

struct IndexDesc {
    int nsec = 0, nq = 0, flow = 1;
    std::vector<int32_t> charges;   // nsec * nq
    std::vector<int32_t> dims;      // nsec
    std::vector<int32_t> q(int s) const {
        return std::vector<int32_t>(charges.begin() + s * nq, charges.begin() + (s + 1) * nq);
    }
    int find(const std::vector<int32_t>& qv) const;
    bool same_sectors(const IndexDesc& o) const { return charges == o.charges && dims == o.dims; }
};

// ---------------------------------------------------------------- device tables
// x block -> XT (x transposed per charge sector, contraction index contiguous)
struct PackTile {
    int64_t x_off;     // element offset of the x block (rows a, cols b, row-major)
    int64_t xt_row0;   // XT row of b = 0 of this block
    int32_t xt_col0;   // XT column of a = 0 of this block
    int32_t m_a, m_b;  // block dims
    int32_t a_pad;     // padded extent of a (multiple of KPAD): columns [m_a, a_pad) get 0
    int32_t a0, b0;    // origin of this 32 x 32 tile inside the block
};

// LW / RW preparation: dst[r][c] = sum_t W[w_idx_t] * src[src_off_t + r * cols + c]
struct MixTile {
    int64_t dst_row0;  // first destination row in LW or RW
    int32_t dst_col0;  // first destination column (segment start)
    int32_t rows, cols, cols_pad;
    int32_t r0, nrows; // row range handled by this tile
    int32_t term_begin, term_count;
    int32_t which;     // 0: L with W1 into LW, 1: R with W2 into RW
};
struct MixTerm {
    int64_t src_off;   // element offset of the environment block
    int32_t w_idx;     // element index into the MPO buffer
    int32_t pad_;
};

// One output tile C[m x n] = sum over segments of A[a_row.., k0:k0+klen] . B[b_row.., k0:k0+klen]^T
struct GemmTask {
    int64_t a_row, b_row;   // first row of the tile in the A and B operand arrays
    int64_t c_off;          // element offset of the tile origin in the output
    int32_t m, n;           // valid rows / columns of the tile
    int32_t ldc;            // output row pitch (elements)
    int32_t n_zero;         // columns [n, n + n_zero) of the tile are written as 0 (padding)
    int32_t seg_begin, seg_count;
    int32_t ktotal;         // sum of the segments' klen (padded contraction length)
    int32_t pad_;
};
struct KSeg {
    int32_t k0, klen;       // column range shared by A and B (klen multiple of KPAD)
};

// ---------------------------------------------------------------- block-product engine
// One output tile C[m x n] (m, n <= 64) = scale * sum over its products of
//   coef * A[a_off + r * a_rs + k * a_cs] * B[b_off + k * b_rs + c * b_cs],  k < K,
// coef = (c1 < 0 ? 1 : coef1[c1]) * (c2 < 0 ? 1 : coef2[c2]).  FP64 throughout.
struct BProd {
    int64_t a_off, b_off;
    int32_t a_rs, a_cs, b_rs, b_cs;
    int32_t K;
    int32_t c1, c2;
    int32_t pad_;
};
struct BTile {
    int64_t c_off;
    int32_t ldc, m, n;
    int32_t prod_begin, prod_count;
    int32_t pad_;
};
struct BList {
    std::vector<BTile> tiles;
    std::vector<BProd> prods;
    BTile* d_tiles = nullptr;
    BProd* d_prods = nullptr;
    double flops = 0;
    bool accumulate = false;   // C += result instead of C = result
    int tile_m = 64, tile_n = 64;   // output tile shape the block list is cut into
    // the output blocks as added (products given for the block origin), kept for re-tiling
    struct Block { int64_t c_off; int32_t ldc, m, n, prod_begin, prod_count; };
    std::vector<Block> blocks;
    std::vector<BProd> block_prods;
    // append the tiles of an m x n output block whose products are given for the block origin
    void add_block(int64_t c_off, int32_t ldc, int32_t m, int32_t n, const std::vector<BProd>& ps);
    // cut every block again into tm x tn tiles (the device tables must be re-uploaded)
    void retile(int tm, int tn);
};
int blist_upload(BList& b);
void blist_free(BList& b);
int launch_bgemm(const BList& b, const double* A, const double* B, double* C, const double* coef1,
                 const double* coef2, double scale, void* stream, const double* inv_scale = nullptr);
// the same products on the tensor cores (BF16x3 split, FP32 accumulation; blockops_tc.cu)
// on FP32 copies of the operands (launch_convert_f64_f32), with an FP32 (c_f64 false) or
// FP64 output; needs 128 x 128 tiles (retile); err: device int raised when a bounded wait
// expires
int launch_bgemm_tc(const BList& b, const float* A, const float* B, void* C, bool c_f64, const double* coef1,
                    const double* coef2, double scale, void* stream, const double* inv_scale, int* err);
// dst[i] = src[i] rounded to FP32 (round to nearest even, on the integer pipes)
int launch_convert_f64_f32(const double* src, float* dst, int64_t n, void* stream);
// out[j] = scale * sum over the dots d in [off[j], off[j+1]) of <X[x_off..], Y[y_off..]>
// (dots sorted by output index; scratch holds one double per dot)
struct BDot {
    int64_t x_off, y_off;
    int64_t len;
};
// (accumulate: out[j] += instead of out[j] =)
int launch_block_dots(const BDot* d_dots, int ndots, const int32_t* d_off, const double* X, const double* Y,
                      double* out, int nout, double* scratch, double scale, void* stream, bool accumulate = false);
int launch_block_dots_f32(const BDot* d_dots, int ndots, const int32_t* d_off, const float* X, const float* Y,
                          double* out, int nout, double* scratch, double scale, void* stream, bool accumulate = false);

constexpr int MAXB = 64;   // batch entries per launch (kernel parameter arrays)
struct PtrBatch { const void* p[MAXB]; };

struct GemmList {
    std::vector<GemmTask> tasks;
    std::vector<KSeg> segs;
    GemmTask* d_tasks = nullptr;
    KSeg* d_segs = nullptr;
    int tm = 0, tn = 0;
    int cl = 1;             // CTAs per entry: 2 = tasks 2e, 2e + 1 share their B tile (cluster pair)
    double flops = 0;       // executed (valid m, n; padded K)
    double useful = 0;      // valid m, n and unpadded K
    // host only, one entry per task: output left sector a' and the task's flop counts
    std::vector<int32_t> owner;
    std::vector<double> task_flops, task_useful;
};

}  // namespace heff

struct heff_layout {
    std::vector<heff::IndexDesc> idx;
    std::vector<int32_t> target;
    int nq = 0;
    std::vector<int32_t> keys;      // nblocks * nidx
    std::vector<int64_t> offsets;   // nblocks
    int64_t nelem = 0;
    std::map<std::vector<int32_t>, int64_t> block_of;
    int64_t offset_of(const std::vector<int32_t>& key) const {
        auto it = block_of.find(key);
        return it == block_of.end() ? -1 : offsets[it->second];
    }
};

struct heff_plan {
    heff_plan_opts opts{};
    int planes = 1;           // values per operand element in the workspace (hi and lo: 2)
    int esize = 8;            // bytes per value
    int64_t nelem_x = 0, nelem_L = 0, nelem_R = 0, nelem_W1 = 0, nelem_W2 = 0;
    // operand arrays (rows x pitch columns; a row holds planes x pitch values, the split
    // precisions' hi and lo interleaved by K block)
    int64_t rows_x = 0, ld_x = 0, rows_lw = 0, rows_t = 0, ld_t = 0, rows_rw = 0;
    // workspace byte offsets
    size_t off_xt = 0, off_lw = 0, off_t = 0, off_rw = 0, off_flags = 0, ws_bytes = 0;
    double flops_canonical = 0;
    std::vector<int32_t> shard_sectors;   // left sectors a' of y this plan computes
    // device tables
    std::vector<heff::PackTile> pack;
    std::vector<heff::MixTile> mix;
    std::vector<heff::MixTerm> terms;
    heff::PackTile* d_pack = nullptr;
    heff::MixTile* d_mix = nullptr;
    heff::MixTerm* d_terms = nullptr;
    // MPO entries the schedule dropped (exactly zero in the host copies), for heff_plan_check_mpo
    std::vector<int32_t> w1_zero, w2_zero;
    int32_t* d_w1_zero = nullptr;
    int32_t* d_w2_zero = nullptr;
    unsigned long long* d_wcount = nullptr;
    heff::GemmList g1, g2;            // active task lists
    heff::GemmList g1_alt, g2_alt;    // the other tile width (tensor-core paths), see heff_plan_autotune
    heff::GemmList g1_pair, g2_pair;  // N = 256 tiles in CTA pairs sharing B (tensor-core paths)
    int64_t stats[24] = {0};
    // tensor-map cache for the tensor-core path: two entries keyed by workspace pointer
    // (two streams alternating workspaces reuse their maps), replaced round-robin
    void* tmap_ws[2] = {nullptr, nullptr};
    int tmap_next = 0;
    alignas(64) unsigned char tmaps[2][13][128];
    int device = 0;
    int num_sms = 0;
    bool uploaded = false;    // false: created without a CUDA device (inspection only)
    // phase timers: events recorded around prepare, pack, GEMM 1, GEMM 2 when enabled
    bool timing = false;
    void* ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_prepare = false;  // whether the last call ran the prepare phase
};

namespace heff {
// launchers (apply.cu)
int launch_pack_batch(heff_plan* p, const void* const* x, int nbatch, void* ws, void* stream);
int launch_mix(heff_plan* p, const void* L, const void* W1, const void* W2, const void* R,
               void* ws, void* stream);
int launch_gemm(heff_plan* p, int which, void* ws, void* const* y, int nbatch, void* stream);
// clusters of two tensor-core CTAs resident at once (tc_gemm.cu; num_sms / 2 without a device)
int tc_pair_clusters(int num_sms, int precision);
// one block waiting at the SVD sweeps' grid barrier set up for two (svd.cu; wait self-test)
void svd_barrier_selftest(unsigned int* bar, int* err, void* stream);
int plan_upload(heff_plan* p);
void plan_free_device(heff_plan* p);
void record_phase(heff_plan* p, int k, void* stream);
}  // namespace heff
