// Packing, operator preparation, the FP64 CUDA-core block GEMMs, and the C-ABI compute
// entry points of the two-site H_eff matvec (Section II-C / Fig. 1d).
//
// One apply is four launches on the caller's stream:
//   mix_kernel   LW = L.W1 and RW = W2.R into the workspace (operator preparation)
//   pack_kernel  x -> XT (per charge sector, transposed so the contraction index is
//                contiguous; hi/lo split for the tensor-core precisions)
//   GEMM 1       T = LW . XT^T              (tensor cores: tc_gemm.cu; FP64: below)
//   GEMM 2       y = T . RW^T               (written straight into y's block layout)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "convert.cuh"
#include "internal.h"

using heff::fail;

namespace heff {

// ------------------------------------------------------------------ element planes
// A workspace operand holds `planes` values per element, of one element type:
//   FP64   : one double
//   BF16X3 : hi = bf16(v), lo = bf16(v - hi)
//   TF32X3 : hi = v with the 13 low mantissa bits cleared (exact in TF32), lo = v - hi
// The two halves of the split precisions are interleaved by 64-byte K blocks within each
// row (split_col): a row of ld columns takes 2 ld elements.
template <int PREC> struct Plane;
template <> struct Plane<HEFF_PREC_FP64> {
    using T = double;
    static __device__ __forceinline__ void split(double v, T& hi, T& lo) { hi = v; lo = 0.0; }
    static __device__ __forceinline__ void store2(T* p, T a, T b) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    }
};
template <> struct Plane<HEFF_PREC_BF16X3> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
        hi = __float2bfloat16_rn(f);
        lo = __float2bfloat16_rn(f - __bfloat162float(hi));
    }
    static __device__ __forceinline__ void split(double v, T& hi, T& lo) { split(f64_to_f32_rn(v), hi, lo); }
    static __device__ __forceinline__ void store2(T* p, T a, T b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __halves2bfloat162(a, b);
    }
};
template <> struct Plane<HEFF_PREC_TF32X3> {
    using T = float;
    // round to the nearest TF32 value (10 explicit mantissa bits), ties away from zero
    static __device__ __forceinline__ float rn_tf32(float f) {
        return __uint_as_float((__float_as_uint(f) + 0x1000u) & 0xffffe000u);
    }
    static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
        hi = rn_tf32(f);
        lo = rn_tf32(f - hi);
    }
    static __device__ __forceinline__ void store2(T* p, T a, T b) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
    static __device__ __forceinline__ void split(double v, T& hi, T& lo) { split(f64_to_f32_rn(v), hi, lo); }
};


// Element conversion of the inputs: FP64 inputs of the split paths go to FP32 on the
// integer pipes (the hardware double -> float conversion runs at GB300's FP64 rate).
template <typename Acc, typename In>
__device__ __forceinline__ Acc to_acc(In v) {
    if constexpr (std::is_same<Acc, float>::value && std::is_same<In, double>::value) return f64_to_f32_rn(v);
    else return (Acc)v;
}

// ------------------------------------------------------------------ dependent launch
// wait for the predecessor grid on the stream (no-op without programmatic launch), and let
// the successor be scheduled onto SMs as this grid's blocks retire
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------ pack x -> XT
// One warp per 32 x 32 tile (four tiles per block): the warp loads the tile's 32 rows a
// (columns b contiguous, one element per lane, all loads in flight), transposes through
// its own shared-memory tile, and writes XT rows b, columns a contiguous (a in [m_a, a_pad)
// are the zero padding), two columns per lane and two rows per pass: every store
// instruction writes two full 32-column row pieces of a half (hi or lo).
constexpr int PACK_WARPS = 4;

template <typename In, int PREC>
__global__ void __launch_bounds__(32 * PACK_WARPS) pack_kernel(const PackTile* __restrict__ tiles, int ntiles,
                                                               PtrBatch xs, char* __restrict__ xt, int64_t ld,
                                                               int64_t batch_elems) {
    using E = typename Plane<PREC>::T;
    constexpr bool SPLIT = PREC != HEFF_PREC_FP64;
    constexpr int KB = 64 / (int)sizeof(E);          // elements per K block of one half
    const int64_t pitch = SPLIT ? 2 * ld : ld;
    using Acc = typename std::conditional<PREC == HEFF_PREC_FP64, double, float>::type;
    __shared__ Acc s[PACK_WARPS][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x * PACK_WARPS + warp;
    if (ti >= ntiles) return;                       // warp-uniform; the block never synchronises
    const PackTile t = tiles[ti];
    const int bz = blockIdx.y;
    Acc (*sw)[33] = s[warp];
    pdl_wait();                                     // x may come from the previous kernel
    pdl_trigger();
    {
        const In* x = static_cast<const In*>(xs.p[bz]) + t.x_off;
        const int b = t.b0 + lane;
        const bool bv = b < t.m_b;
        const int na = t.m_a - t.a0;                // rows of x left in this tile (may be <= 0)
#pragma unroll
        for (int r = 0; r < 32; ++r)
            sw[r][lane] = (bv && r < na) ? to_acc<Acc>(x[(int64_t)(t.a0 + r) * t.m_b + b]) : (Acc)0;
    }
    __syncwarp();
    E* base = reinterpret_cast<E*>(xt) + (int64_t)bz * batch_elems;
    const int c = 2 * (lane & 15), h = lane >> 4;
    const int nb = t.m_b - t.b0;                    // XT rows of this tile
    const int64_t col = t.xt_col0 + t.a0 + c;       // even: both columns in one K block
    const int64_t o0 = (t.xt_row0 + t.b0) * pitch + (SPLIT ? split_col<KB>(col) : col);
#pragma unroll 4
    for (int r = h; r < 32; r += 2) {
        if (r >= nb) break;
        E h0, l0, h1, l1;
        Plane<PREC>::split(sw[c][r], h0, l0);
        Plane<PREC>::split(sw[c + 1][r], h1, l1);
        const int64_t o = o0 + (int64_t)r * pitch;
        Plane<PREC>::store2(base + o, h0, h1);
        if (SPLIT) Plane<PREC>::store2(base + o + KB, l0, l1);
    }
}

// ------------------------------------------------------------------ LW / RW preparation
#ifndef HEFF_MIX_UNROLL
#define HEFF_MIX_UNROLL 4      // column pairs per lane and pass
#endif
#ifndef HEFF_MIX_ROWS
#define HEFF_MIX_ROWS 1        // rows per warp and pass
#endif

struct MixArgs {
    const MixTile* tiles;
    const MixTerm* terms;
    const void *L, *W1, *W2, *R;
    char* lw; int64_t ld_lw;
    char* rw; int64_t ld_rw;
};

template <typename In, int PREC>
__device__ __forceinline__ void mix_tile(const MixTile& t, const MixArgs& a) {
    const MixTerm* __restrict__ terms = a.terms;
    const In* __restrict__ L = static_cast<const In*>(a.L);
    const In* __restrict__ W1 = static_cast<const In*>(a.W1);
    const In* __restrict__ W2 = static_cast<const In*>(a.W2);
    const In* __restrict__ R = static_cast<const In*>(a.R);
    char* __restrict__ lw = a.lw;
    char* __restrict__ rw = a.rw;
    const int64_t ld_lw = a.ld_lw, ld_rw = a.ld_rw;
    // FP64 path accumulates in double; the split paths in float (1-4 terms, each product
    // exact to 24 bits, well inside the 16-bit (bf16 hi+lo) / 22-bit (tf32 hi+lo) split).
    using E = typename Plane<PREC>::T;
    using Acc = typename std::conditional<PREC == HEFF_PREC_FP64, double, float>::type;
    __shared__ Acc coef[64];
    __shared__ int64_t srco[64];
    const In* src = t.which ? R : L;
    const In* W = t.which ? W2 : W1;
    const int nt = t.term_count < 64 ? t.term_count : 64;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
        MixTerm m = terms[t.term_begin + k];
        coef[k] = to_acc<Acc>(W[m.w_idx]);
        srco[k] = m.src_off;
    }
    __syncthreads();
    constexpr bool SPLIT = PREC != HEFF_PREC_FP64;
    constexpr int KB = 64 / (int)sizeof(E);          // elements per K block of one half
    E* base = reinterpret_cast<E*>(t.which ? rw : lw);
    const int64_t pitch = SPLIT ? 2 * (t.which ? ld_rw : ld_lw) : (t.which ? ld_rw : ld_lw);
    // warps over rows, lanes over column pairs: each thread writes two adjacent columns
    // (dst_col0 and cols_pad are multiples of 32, so the pair stores are aligned) of RW rows,
    // U pairs 64 columns apart per pass, with all loads of a term issued before its FMAs
    // (2 RW U loads in flight per thread: the kernel is bound by HBM latency x bytes in flight)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int U = HEFF_MIX_UNROLL;
    constexpr int RW = HEFF_MIX_ROWS;
    const int nw = blockDim.x >> 5;
    for (int rr = warp * RW; rr < t.nrows; rr += nw * RW) {
        int64_t rc[RW];
        bool rv[RW];
#pragma unroll
        for (int i = 0; i < RW; ++i) {
            rv[i] = rr + i < t.nrows;
            rc[i] = (int64_t)(t.r0 + rr + i) * t.cols;
        }
        for (int cb = 2 * lane; cb < t.cols_pad; cb += 64 * U) {
            Acc a0[RW][U], a1[RW][U];
#pragma unroll
            for (int i = 0; i < RW; ++i)
#pragma unroll
                for (int u = 0; u < U; ++u) { a0[i][u] = 0; a1[i][u] = 0; }
            for (int k = 0; k < t.term_count; ++k) {
                const In* s;
                Acc cf;
                if (k < nt) {
                    s = src + srco[k];
                    cf = coef[k];
                } else {                                      // rare: more than 64 terms
                    const MixTerm m = terms[t.term_begin + k];
                    s = src + m.src_off;
                    cf = to_acc<Acc>(W[m.w_idx]);
                }
                In v0[RW][U], v1[RW][U];
#pragma unroll
                for (int i = 0; i < RW; ++i)
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int c = cb + 64 * u;
                        v0[i][u] = rv[i] && c < t.cols ? s[rc[i] + c] : (In)0;
                        v1[i][u] = rv[i] && c + 1 < t.cols ? s[rc[i] + c + 1] : (In)0;
                    }
#pragma unroll
                for (int i = 0; i < RW; ++i)
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        a0[i][u] += cf * to_acc<Acc>(v0[i][u]);
                        a1[i][u] += cf * to_acc<Acc>(v1[i][u]);
                    }
            }
#pragma unroll
            for (int i = 0; i < RW; ++i) {
                if (!rv[i]) break;
                const int64_t o = (t.dst_row0 + t.r0 + rr + i) * pitch;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int c = cb + 64 * u;
                    if (c >= t.cols_pad) break;
                    E h0, l0, h1, l1;
                    Plane<PREC>::split(a0[i][u], h0, l0);
                    Plane<PREC>::split(a1[i][u], h1, l1);
                    const int64_t col = t.dst_col0 + c;     // even: both columns in one K block
                    const int64_t p = o + (SPLIT ? split_col<KB>(col) : col);
                    Plane<PREC>::store2(base + p, h0, h1);
                    if (SPLIT) Plane<PREC>::store2(base + p + KB, l0, l1);
                }
            }
        }
    }
}

#ifndef HEFF_MIX_MINB
#define HEFF_MIX_MINB 6        // resident blocks per SM the register allocation must allow
#endif
template <typename In, int PREC>
__global__ void __launch_bounds__(256, HEFF_MIX_MINB) mix_kernel(MixArgs a) {
    pdl_trigger();                                  // the pack kernel may be scheduled behind it
    mix_tile<In, PREC>(a.tiles[blockIdx.x], a);
}

// ------------------------------------------------------------------ FP64 CUDA-core GEMM
// C[m x n] = sum_seg A[a_row + r, k] B[b_row + c, k] over 64 x 64 tiles, 4 x 4 per thread.
struct GemmArgs {
    const GemmTask* tasks;
    const KSeg* segs;
    int ntasks;
    const char* A; int64_t a_batch_rows;    // operand arrays and their per-batch row offsets
    const char* B; int64_t b_batch_rows;
    int64_t ld;                             // shared row pitch of A and B
    char* C; int64_t c_batch_elems;         // GEMM 1 output (T) and per-batch offset
    PtrBatch y;                             // GEMM 2 outputs (one per batch entry)
    int mode;                               // 0: write T (operand type), 1: write y (io type)
};

__global__ void __launch_bounds__(256) gemm_fp64_kernel(GemmArgs g) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const GemmTask t = g.tasks[blockIdx.x];
    const int bz = blockIdx.y;
    const double* A = reinterpret_cast<const double*>(g.A) + (int64_t)bz * g.a_batch_rows * g.ld;
    const double* B = reinterpret_cast<const double*>(g.B) + (int64_t)bz * g.b_batch_rows * g.ld;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int s = 0; s < t.seg_count; ++s) {
        const KSeg sg = g.segs[t.seg_begin + s];
        for (int k0 = sg.k0; k0 < sg.k0 + sg.klen; k0 += 16) {
            for (int l = 0; l < 4; ++l) {
                int idx = tid + 256 * l, row = idx >> 4, kk = idx & 15;
                As[kk][row] = row < t.m ? A[(t.a_row + row) * g.ld + k0 + kk] : 0.0;
                Bs[kk][row] = row < t.n ? B[(t.b_row + row) * g.ld + k0 + kk] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    double* C = g.mode == 0 ? reinterpret_cast<double*>(g.C) + (int64_t)bz * g.c_batch_elems
                            : static_cast<double*>(const_cast<void*>(g.y.p[bz]));
    for (int i = 0; i < 4; ++i) {
        int r = ty * 4 + i;
        if (r >= t.m) continue;
        for (int j = 0; j < 4; ++j) {
            int c = tx * 4 + j;
            if (c < t.n) C[t.c_off + (int64_t)r * t.ldc + c] = acc[i][j];
            else if (c < t.n + t.n_zero) C[t.c_off + (int64_t)r * t.ldc + c] = 0.0;
        }
    }
}

// ------------------------------------------------------------------ host side
#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return fail(HEFF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
static int upload(const std::vector<T>& v, T** d) {
    *d = nullptr;
    if (v.empty()) return HEFF_OK;
    CK(cudaMalloc((void**)d, v.size() * sizeof(T)));
    CK(cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HEFF_OK;
}

int plan_upload(heff_plan* p) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();          // no device: a host-only plan for inspection
        p->uploaded = false;
        return HEFF_OK;
    }
    CK(cudaGetDevice(&p->device));
    CK(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    int rc;
    if ((rc = upload(p->pack, &p->d_pack)) != HEFF_OK) return rc;
    if ((rc = upload(p->mix, &p->d_mix)) != HEFF_OK) return rc;
    if ((rc = upload(p->terms, &p->d_terms)) != HEFF_OK) return rc;
    for (GemmList* g : {&p->g1, &p->g2, &p->g1_alt, &p->g2_alt, &p->g1_pair, &p->g2_pair}) {
        if ((rc = upload(g->tasks, &g->d_tasks)) != HEFF_OK) return rc;
        if ((rc = upload(g->segs, &g->d_segs)) != HEFF_OK) return rc;
    }
    if ((rc = upload(p->w1_zero, &p->d_w1_zero)) != HEFF_OK) return rc;
    if ((rc = upload(p->w2_zero, &p->d_w2_zero)) != HEFF_OK) return rc;
    CK(cudaMalloc((void**)&p->d_wcount, sizeof(unsigned long long)));
    p->uploaded = true;
    return HEFF_OK;
}

void record_phase(heff_plan* p, int k, void* stream) {
    if (p->timing && p->ev[k]) cudaEventRecord(static_cast<cudaEvent_t>(p->ev[k]), static_cast<cudaStream_t>(stream));
}

void plan_free_device(heff_plan* p) {
    for (int k = 0; k < 5; ++k)
        if (p->ev[k]) { cudaEventDestroy(static_cast<cudaEvent_t>(p->ev[k])); p->ev[k] = nullptr; }
    cudaFree(p->d_pack); cudaFree(p->d_mix); cudaFree(p->d_terms);
    cudaFree(p->d_w1_zero); cudaFree(p->d_w2_zero); cudaFree(p->d_wcount);
    p->d_w1_zero = p->d_w2_zero = nullptr;
    p->d_wcount = nullptr;
    cudaFree(p->g1.d_tasks); cudaFree(p->g1.d_segs); cudaFree(p->g2.d_tasks); cudaFree(p->g2.d_segs);
    for (GemmList* g : {&p->g1_alt, &p->g2_alt, &p->g1_pair, &p->g2_pair}) {
        cudaFree(g->d_tasks); cudaFree(g->d_segs);
        g->d_tasks = nullptr; g->d_segs = nullptr;
    }
    p->d_pack = nullptr; p->d_mix = nullptr; p->d_terms = nullptr;
    p->g1.d_tasks = p->g2.d_tasks = nullptr; p->g1.d_segs = p->g2.d_segs = nullptr;
}


template <typename In, int PREC>
static void launch_pack_t(heff_plan* p, const PtrBatch& xs, int nb, char* ws, cudaStream_t st) {
    const int nt = (int)p->pack.size();
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)((nt + PACK_WARPS - 1) / PACK_WARPS), nb);
    cfg.blockDim = dim3(32 * PACK_WARPS);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = HEFF_PDL ? 1 : 0;
    cudaLaunchKernelEx(&cfg, pack_kernel<In, PREC>, static_cast<const PackTile*>(p->d_pack), nt, xs,
                       ws + p->off_xt, p->ld_x, (int64_t)p->planes * p->rows_x * p->ld_x);
}

int launch_pack_batch(heff_plan* p, const void* const* x, int nbatch, void* ws, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->pack.empty()) return HEFF_OK;
    for (int b0 = 0; b0 < nbatch; b0 += MAXB) {
        int nb = nbatch - b0 < MAXB ? nbatch - b0 : MAXB;
        PtrBatch xs{};
        for (int b = 0; b < nb; ++b) xs.p[b] = x[b0 + b];
        char* w = static_cast<char*>(ws) + (size_t)b0 * p->rows_x * p->ld_x * p->esize * p->planes;
        const bool f32 = p->opts.io_dtype == HEFF_DTYPE_F32;
        switch (p->opts.precision) {
            case HEFF_PREC_FP64: launch_pack_t<double, HEFF_PREC_FP64>(p, xs, nb, w, st); break;
            case HEFF_PREC_BF16X3:
                if (f32) launch_pack_t<float, HEFF_PREC_BF16X3>(p, xs, nb, w, st);
                else launch_pack_t<double, HEFF_PREC_BF16X3>(p, xs, nb, w, st);
                break;
            default:
                if (f32) launch_pack_t<float, HEFF_PREC_TF32X3>(p, xs, nb, w, st);
                else launch_pack_t<double, HEFF_PREC_TF32X3>(p, xs, nb, w, st);
        }
        count_launches(1);
    }
    CK(cudaGetLastError());
    return HEFF_OK;
}

static MixArgs mix_args(heff_plan* p, const void* L, const void* W1, const void* W2, const void* R, char* ws) {
    return MixArgs{p->d_mix, p->d_terms, L, W1, W2, R, ws + p->off_lw, p->ld_x, ws + p->off_rw, p->ld_t};
}

template <typename In, int PREC>
static void launch_mix_t(heff_plan* p, const void* L, const void* W1, const void* W2, const void* R,
                         char* ws, cudaStream_t st) {
    mix_kernel<In, PREC><<<(unsigned)p->mix.size(), 256, 0, st>>>(mix_args(p, L, W1, W2, R, ws));
}

int launch_mix(heff_plan* p, const void* L, const void* W1, const void* W2, const void* R, void* ws,
               void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->mix.empty()) return HEFF_OK;
    char* w = static_cast<char*>(ws);
    const bool f32 = p->opts.io_dtype == HEFF_DTYPE_F32;
    switch (p->opts.precision) {
        case HEFF_PREC_FP64: launch_mix_t<double, HEFF_PREC_FP64>(p, L, W1, W2, R, w, st); break;
        case HEFF_PREC_BF16X3:
            if (f32) launch_mix_t<float, HEFF_PREC_BF16X3>(p, L, W1, W2, R, w, st);
            else launch_mix_t<double, HEFF_PREC_BF16X3>(p, L, W1, W2, R, w, st);
            break;
        default:
            if (f32) launch_mix_t<float, HEFF_PREC_TF32X3>(p, L, W1, W2, R, w, st);
            else launch_mix_t<double, HEFF_PREC_TF32X3>(p, L, W1, W2, R, w, st);
    }
    count_launches(1);
    CK(cudaGetLastError());
    return HEFF_OK;
}

int launch_tc_gemm(heff_plan* p, int which, void* ws, void* const* y, int nbatch, void* stream);

int launch_gemm(heff_plan* p, int which, void* ws, void* const* y, int nbatch, void* stream) {
    if (p->opts.precision != HEFF_PREC_FP64) return launch_tc_gemm(p, which, ws, y, nbatch, stream);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GemmList& gl = which == 1 ? p->g1 : p->g2;
    if (gl.tasks.empty()) return HEFF_OK;
    char* w = static_cast<char*>(ws);
    for (int b0 = 0; b0 < nbatch; b0 += MAXB) {
        int nb = nbatch - b0 < MAXB ? nbatch - b0 : MAXB;
        GemmArgs g{};
        g.tasks = gl.d_tasks;
        g.segs = gl.d_segs;
        g.ntasks = (int)gl.tasks.size();
        if (which == 1) {
            g.A = w + p->off_lw; g.a_batch_rows = 0;
            g.B = w + p->off_xt + (size_t)b0 * p->rows_x * p->ld_x * 8; g.b_batch_rows = p->rows_x;
            g.ld = p->ld_x;
            g.C = w + p->off_t + (size_t)b0 * p->rows_t * p->ld_t * 8; g.c_batch_elems = p->rows_t * p->ld_t;
            g.mode = 0;
        } else {
            g.A = w + p->off_t + (size_t)b0 * p->rows_t * p->ld_t * 8; g.a_batch_rows = p->rows_t;
            g.B = w + p->off_rw; g.b_batch_rows = 0;
            g.ld = p->ld_t;
            for (int b = 0; b < nb; ++b) g.y.p[b] = y[b0 + b];
            g.mode = 1;
        }
        dim3 grid((unsigned)gl.tasks.size(), nb);
        gemm_fp64_kernel<<<grid, 256, 0, st>>>(g);
        count_launches(1);
    }
    CK(cudaGetLastError());
    return HEFF_OK;
}

}  // namespace heff

// ------------------------------------------------------------------ MPO check
// *count += the entries W[idx[i]], i < n, that are not zero
template <typename T>
__global__ void __launch_bounds__(256) mpo_nonzero_at_kernel(const T* __restrict__ W, const int32_t* __restrict__ idx,
                                                             int n, unsigned long long* count) {
    unsigned long long c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        c += W[idx[i]] != (T)0 ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// ------------------------------------------------------------------ C ABI
static int check_ws(const heff_plan* p, void* ws, size_t bytes) {
    if (!p->uploaded) return fail(HEFF_ERR_UNSUPPORTED, "plan was created without a CUDA device");
    if (!ws) return fail(HEFF_ERR_WORKSPACE, "null workspace");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(HEFF_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (bytes < p->ws_bytes)
        return fail(HEFF_ERR_WORKSPACE, "workspace of %zu bytes, plan needs %zu", bytes, p->ws_bytes);
    return HEFF_OK;
}

static int do_prepare(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                      void* workspace, void* stream) {
    heff::record_phase(plan, 0, stream);
    int rc = heff::launch_mix(plan, L, W1, W2, R, workspace, stream);
    heff::record_phase(plan, 1, stream);
    return rc;
}

static int do_gemms(heff_plan* plan, void* const* y, int nbatch, void* workspace, void* stream) {
    int rc;
    if ((rc = heff::launch_gemm(plan, 1, workspace, y, nbatch, stream))) return rc;
    heff::record_phase(plan, 3, stream);
    if ((rc = heff::launch_gemm(plan, 2, workspace, y, nbatch, stream))) return rc;
    heff::record_phase(plan, 4, stream);
    return HEFF_OK;
}

static int do_matvec(heff_plan* plan, const void* const* x, void* const* y, int nbatch, void* workspace,
                     void* stream) {
    int rc;
    if ((rc = heff::launch_pack_batch(plan, x, nbatch, workspace, stream))) return rc;
    heff::record_phase(plan, 2, stream);
    return do_gemms(plan, y, nbatch, workspace, stream);
}

static int do_apply(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                    const void* const* x, void* const* y, int nbatch, void* workspace, void* stream) {
    plan->ev_prepare = true;
    int rc = do_prepare(plan, L, W1, W2, R, workspace, stream);
    return rc ? rc : do_matvec(plan, x, y, nbatch, workspace, stream);
}

extern "C" int heff_prepare(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                            void* workspace, size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (!plan || !L || !W1 || !W2 || !R) return fail(HEFF_ERR_INVALID_ARG, "heff_prepare: null argument");
    int rc = check_ws(plan, workspace, workspace_bytes);
    if (rc) return rc;
    plan->ev_prepare = true;
    return do_prepare(plan, L, W1, W2, R, workspace, stream);
}

extern "C" int heff_apply_prepared(heff_plan* plan, const void* x, void* y, void* workspace,
                                   size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (plan && plan->nelem_x == 0) return HEFF_OK;            // an empty two-site space: y has no elements
    if (!plan || !x || !y) return fail(HEFF_ERR_INVALID_ARG, "heff_apply_prepared: null argument");
    if (x == y) return fail(HEFF_ERR_INVALID_ARG, "y must not alias x");
    int rc = check_ws(plan, workspace, workspace_bytes);
    if (rc) return rc;
    const void* xs[1] = {x};
    void* ys[1] = {y};
    plan->ev_prepare = false;
    heff::record_phase(plan, 1, stream);
    return do_matvec(plan, xs, ys, 1, workspace, stream);
}

extern "C" int heff_apply(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                          const void* x, void* y, void* workspace, size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (plan && plan->nelem_x == 0) return HEFF_OK;            // an empty two-site space: y has no elements
    if (!plan || !L || !W1 || !W2 || !R || !x || !y) return fail(HEFF_ERR_INVALID_ARG, "heff_apply: null argument");
    if (x == y) return fail(HEFF_ERR_INVALID_ARG, "y must not alias x");
    int rc = check_ws(plan, workspace, workspace_bytes);
    if (rc) return rc;
    const void* xs[1] = {x};
    void* ys[1] = {y};
    return do_apply(plan, L, W1, W2, R, xs, ys, 1, workspace, stream);
}

namespace {
struct Staging {
    size_t off[6];      // L, W1, W2, R, x, y
    size_t bytes[6];
    size_t total;
};
Staging staging_layout(const heff_plan* p) {
    const size_t es = p->opts.io_dtype == HEFF_DTYPE_F64 ? 8 : 4;
    const int64_t n[6] = {p->nelem_L, p->nelem_W1, p->nelem_W2, p->nelem_R, p->nelem_x, p->nelem_x};
    Staging s{};
    size_t o = 0;
    for (int k = 0; k < 6; ++k) {
        s.off[k] = o;
        s.bytes[k] = (size_t)n[k] * es;
        o = (o + s.bytes[k] + 255) / 256 * 256;
    }
    s.total = o;
    return s;
}
}  // namespace

extern "C" int heff_apply_host_staging_size(const heff_plan* plan, size_t* bytes) {
    heff::clear_error();
    if (!plan || !bytes) return fail(HEFF_ERR_INVALID_ARG, "heff_apply_host_staging_size: null argument");
    *bytes = staging_layout(plan).total;
    return HEFF_OK;
}

extern "C" int heff_apply_host(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                               const void* x, void* y, void* staging, size_t staging_bytes, void* workspace,
                               size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (plan && plan->nelem_x == 0) return HEFF_OK;            // an empty two-site space: y has no elements
    if (!plan || !L || !W1 || !W2 || !R || !x || !y || !staging)
        return fail(HEFF_ERR_INVALID_ARG, "heff_apply_host: null argument");
    const Staging sl = staging_layout(plan);
    if (staging_bytes < sl.total || reinterpret_cast<uintptr_t>(staging) % 256)
        return fail(HEFF_ERR_WORKSPACE, "staging buffer of %zu bytes, needs %zu (256-byte aligned)", staging_bytes,
                    sl.total);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* d = static_cast<char*>(staging);
    const void* src[5] = {L, W1, W2, R, x};
    for (int k = 0; k < 5; ++k)
        CK(cudaMemcpyAsync(d + sl.off[k], src[k], sl.bytes[k], cudaMemcpyHostToDevice, st));
    int rc = heff_apply(plan, d + sl.off[0], d + sl.off[1], d + sl.off[2], d + sl.off[3], d + sl.off[4],
                        d + sl.off[5], workspace, workspace_bytes, stream);
    if (rc) return rc;
    CK(cudaMemcpyAsync(y, d + sl.off[5], sl.bytes[5], cudaMemcpyDeviceToHost, st));
    return HEFF_OK;
}

extern "C" int heff_apply_batched(heff_plan* plan, const void* L, const void* W1, const void* W2,
                                  const void* R, const void* const* x, void* const* y, int32_t nbatch,
                                  void* workspace, size_t workspace_bytes, void* stream) {
    heff::clear_error();
    if (!plan || !L || !W1 || !W2 || !R || !x || !y)
        return fail(HEFF_ERR_INVALID_ARG, "heff_apply_batched: null argument");
    if (nbatch < 1 || nbatch > plan->opts.max_batch)
        return fail(HEFF_ERR_INVALID_ARG, "nbatch %d outside 1..max_batch (%d)", nbatch, plan->opts.max_batch);
    if (plan->nelem_x == 0) return HEFF_OK;                   // an empty two-site space: no y has elements
    for (int b = 0; b < nbatch; ++b) {
        if (!x[b] || !y[b]) return fail(HEFF_ERR_INVALID_ARG, "null x or y at batch entry %d", b);
        if (x[b] == y[b]) return fail(HEFF_ERR_INVALID_ARG, "y must not alias x (batch entry %d)", b);
    }
    int rc = check_ws(plan, workspace, workspace_bytes);
    if (rc) return rc;
    plan->ev_prepare = true;
    return do_apply(plan, L, W1, W2, R, x, y, nbatch, workspace, stream);
}

// Tile-shape autotuner: time each GEMM with every task list the plan built (N = 256, N = 128,
// N = 256 in CTA pairs) on the caller's inputs and keep the fastest one per GEMM (tensor-core
// precisions only).
namespace {
// the plan's task lists of one GEMM, the active one first
void gemm_variants(heff_plan* p, int which, heff::GemmList* v[HEFF_TILE_VARIANTS]) {
    v[0] = which == 1 ? &p->g1 : &p->g2;
    v[1] = which == 1 ? &p->g1_alt : &p->g2_alt;
    v[2] = which == 1 ? &p->g1_pair : &p->g2_pair;
}
int tile_code(const heff::GemmList& g) { return g.tn * g.cl; }
void record_tiles(heff_plan* p) {
    p->stats[3] = (int64_t)p->g1.tasks.size();
    p->stats[4] = (int64_t)p->g2.tasks.size();
    p->stats[15] = tile_code(p->g1);
    p->stats[22] = tile_code(p->g2);
}
// slot of a tile code in the autotuner's report: 256, 128, 512
int code_slot(int code) { return code == 256 ? 0 : (code == 128 ? 1 : 2); }
}  // namespace

extern "C" int heff_plan_autotune(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                                  const void* x, void* y, void* workspace, size_t workspace_bytes, void* stream,
                                  int32_t* tn_out, float* ms_out) {
    heff::clear_error();
    if (!plan || !L || !W1 || !W2 || !R || !x || !y) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_autotune: null argument");
    int rc = check_ws(plan, workspace, workspace_bytes);
    if (rc) return rc;
    if (ms_out)
        for (int i = 0; i < 2 * HEFF_TILE_VARIANTS; ++i) ms_out[i] = 0.f;
    if (plan->opts.precision != HEFF_PREC_FP64 && !plan->g1_alt.tasks.empty()) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const void* xs[1] = {x};
        void* ys[1] = {y};
        if ((rc = heff::launch_mix(plan, L, W1, W2, R, workspace, stream))) return rc;
        if ((rc = heff::launch_pack_batch(plan, xs, 1, workspace, stream))) return rc;
        // each candidate: one warm-up launch, then the median of 5 separately timed launches
        cudaEvent_t e[6];
        for (auto& ev : e) CK(cudaEventCreate(&ev));
        for (int which = 1; which <= 2 && !rc; ++which) {
            heff::GemmList* v[HEFF_TILE_VARIANTS];
            gemm_variants(plan, which, v);
            float ms[HEFF_TILE_VARIANTS];
            int best = 0;
            for (int c = 0; c < HEFF_TILE_VARIANTS && !rc; ++c) {
                ms[c] = 0.f;
                if (v[c]->tasks.empty() && !v[0]->tasks.empty()) continue;
                std::swap(*v[0], *v[c]);
                rc = heff::launch_gemm(plan, which, workspace, ys, 1, stream);
                CK(cudaEventRecord(e[0], st));
                for (int r = 0; r < 5 && !rc; ++r) {
                    rc = heff::launch_gemm(plan, which, workspace, ys, 1, stream);
                    CK(cudaEventRecord(e[r + 1], st));
                }
                if (!rc) {
                    CK(cudaEventSynchronize(e[5]));
                    float t[5];
                    for (int r = 0; r < 5; ++r) CK(cudaEventElapsedTime(&t[r], e[r], e[r + 1]));
                    std::sort(t, t + 5);
                    ms[c] = t[2];
                    if (ms[c] < ms[best]) best = c;
                }
                std::swap(*v[0], *v[c]);
                if (ms_out && !rc) ms_out[HEFF_TILE_VARIANTS * (which - 1) + code_slot(tile_code(*v[c]))] = ms[c];
            }
            if (rc) break;
            if (best) std::swap(*v[0], *v[best]);
        }
        for (auto& ev : e) cudaEventDestroy(ev);
        if (rc) return rc;
        record_tiles(plan);
    }
    if (tn_out) {
        tn_out[0] = tile_code(plan->g1);
        tn_out[1] = tile_code(plan->g2);
    }
    return HEFF_OK;
}

extern "C" int heff_plan_select_tiles(heff_plan* plan, int32_t tn1, int32_t tn2) {
    heff::clear_error();
    if (!plan) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_select_tiles: null plan");
    const int want[2] = {tn1, tn2};
    for (int which = 1; which <= 2; ++which) {
        heff::GemmList* v[HEFF_TILE_VARIANTS];
        gemm_variants(plan, which, v);
        const int code = want[which - 1];
        if (code == 0 || code == tile_code(*v[0])) continue;
        int c = 1;
        while (c < HEFF_TILE_VARIANTS && tile_code(*v[c]) != code) ++c;
        if (c == HEFF_TILE_VARIANTS || plan->opts.precision == HEFF_PREC_FP64)
            return fail(HEFF_ERR_INVALID_ARG, "tile variant %d is not available for GEMM %d", code, which);
        std::swap(*v[0], *v[c]);
    }
    record_tiles(plan);
    return HEFF_OK;
}

extern "C" int heff_plan_set_timing(heff_plan* plan, int32_t enable) {
    heff::clear_error();
    if (!plan) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_set_timing: null plan");
    if (!plan->uploaded) return fail(HEFF_ERR_UNSUPPORTED, "plan was created without a CUDA device");
    if (enable && !plan->ev[0])
        for (int k = 0; k < 5; ++k) CK(cudaEventCreate(reinterpret_cast<cudaEvent_t*>(&plan->ev[k])));
    plan->timing = enable != 0;
    return HEFF_OK;
}

extern "C" int heff_plan_timings(heff_plan* plan, float* ms) {
    heff::clear_error();
    if (!plan || !ms) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_timings: null argument");
    if (!plan->timing) return fail(HEFF_ERR_INVALID_ARG, "timing is not enabled on this plan");
    cudaEvent_t* e = reinterpret_cast<cudaEvent_t*>(plan->ev);
    CK(cudaEventSynchronize(e[4]));
    ms[0] = 0.f;
    if (plan->ev_prepare) CK(cudaEventElapsedTime(&ms[0], e[0], e[1]));
    CK(cudaEventElapsedTime(&ms[1], e[1], e[2]));
    CK(cudaEventElapsedTime(&ms[2], e[2], e[3]));
    CK(cudaEventElapsedTime(&ms[3], e[3], e[4]));
    return HEFF_OK;
}

extern "C" int heff_plan_check_mpo(const heff_plan* plan, const void* W1, const void* W2, void* stream,
                                   int64_t* violations) {
    heff::clear_error();
    if (!plan || !W1 || !W2 || !violations) return fail(HEFF_ERR_INVALID_ARG, "heff_plan_check_mpo: null argument");
    if (!plan->uploaded) return fail(HEFF_ERR_UNSUPPORTED, "plan was created without a CUDA device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(plan->d_wcount, 0, sizeof(unsigned long long), st));
    const bool f64 = plan->opts.io_dtype == HEFF_DTYPE_F64;
    const struct { const void* W; const int32_t* idx; size_t n; } parts[2] = {
        {W1, plan->d_w1_zero, plan->w1_zero.size()}, {W2, plan->d_w2_zero, plan->w2_zero.size()}};
    for (const auto& pt : parts) {
        if (pt.n == 0) continue;
        const int grid = (int)std::min<size_t>((pt.n + 255) / 256, 1024);
        if (f64)
            mpo_nonzero_at_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(pt.W), pt.idx,
                                                                 (int)pt.n, plan->d_wcount);
        else
            mpo_nonzero_at_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(pt.W), pt.idx,
                                                                (int)pt.n, plan->d_wcount);
        heff::count_launches(1);
    }
    unsigned long long c = 0;
    CK(cudaMemcpyAsync(&c, plan->d_wcount, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *violations = (int64_t)c;
    return HEFF_OK;
}
