// Tensor-core form of the block-product engine of blockops.cu (the charge-matched block-pair
// products of Algorithm 2, summed into output tiles, Section IV "list" algorithm): the same
// tile and product lists, cut into 128 x 128 output tiles, with every product contracted on
// the sm_103a tensor cores in the BF16x3 split (hi = bf16(v), lo = bf16(v - hi); per K block
// A_hi.B_hi + A_hi.B_lo + A_lo.B_hi, FP32 accumulation in tensor memory).
//
// The operands are FP32 copies of the FP64 tensors (convert_f64_f32: one conversion per
// element; converting inside the kernel would redo it for every tile that reads the element,
// and on GB300 the hardware double -> float conversion runs at the FP64 rate).  The output is
// FP32 (intermediates) or FP64 (results).
//
// One CTA per output tile, 9 warps:
//   warps 0..7  producers: per K block of 32 elements they load the 128 rows of the A block
//               and the 128 rows of the (transposed) B block with the product's strides
//               (A scaled by the product's MPO coefficient), split them into bf16
//               hi/lo and write them into the 64-byte-swizzled K-major shared-memory layout
//               the MMA reads; a ring of 3 stages.  An operand whose K index is the
//               contiguous one is read with the lanes of a warp along K (one 256-byte row per
//               load instruction); otherwise each thread takes half a row (16 K values) and
//               the lanes run along the rows, which are then contiguous.  After the last
//               MMA they are the epilogue: tensor memory -> registers -> a per-warp shared-
//               memory transpose -> coalesced FP64 row stores (C = scale * acc, or C +=).
//   warp 8      allocates 128 tensor-memory columns; one thread issues the MMAs.
// Operands come in with arbitrary strides (environment blocks, site tensors, transposed
// views), so the loads are plain global loads rather than TMA copies.  Every mbarrier wait
// is bounded; on expiry the CTA raises the error flag, stops issuing work, waits (bounded)
// for the MMAs it has already issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "convert.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace heff {
namespace {

using namespace ptx;

constexpr int BT_M = 128, BT_N = 128;       // output tile
constexpr int BT_KB = 32;                   // K elements per block: one 64-byte bf16 row
constexpr int BT_STAGES = 3;
constexpr int BT_PWARPS = 8;
constexpr int BT_THREADS = 32 * (BT_PWARPS + 1);
constexpr int BT_PLANE = BT_M * 64;         // one 128-row plane of a K block: 8 KB
constexpr int BT_STAGE = 4 * BT_PLANE;      // A hi, A lo, B hi, B lo
constexpr int BT_BAR = BT_STAGES * BT_STAGE;
constexpr int BT_SMEM = BT_BAR + 256 + 1024;   // + barriers, alignment slack
static_assert(BT_PWARPS * 16 == BT_M && BT_M == BT_N, "two producer threads per A row and per B row");
static_assert(BT_PWARPS * 32 * 33 * 4 <= BT_BAR, "the epilogue transpose fits in the ring");

struct BtArgs {
    const BTile* tiles;
    const BProd* prods;
    const float* A;
    const float* B;
    void* C;                  // float or double (the kernel's TC)
    const double* coef1;
    const double* coef2;
    double scale;
    const double* inv_scale;
    int accumulate;
    int* err;
};

// bf16 hi/lo split of a pair of values, packed as two bf16x2 words
__device__ __forceinline__ void split2(float a, float b, uint32_t& h, uint32_t& l) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(a - __low2float(hh), b - __high2float(hh));
    h = *reinterpret_cast<const uint32_t*>(&hh);
    l = *reinterpret_cast<const uint32_t*>(&ll);
}

// Byte offset of bf16 element k (even) of row r in a plane: 64-byte rows, 16-byte chunk j
// stored at chunk j ^ ((r >> 1) & 3).
__device__ __forceinline__ uint32_t swz(int r, int k) {
    return (uint32_t)r * 64 + ((uint32_t)((k >> 3) ^ ((r >> 1) & 3)) << 4) + (uint32_t)(k & 7) * 2;
}

// Load the K block [k0, k0 + nk) (nk <= 32) of the 128 operand rows r < nrows, element
// (r, k) at src[r * rs + k * ks] (scaled by coef), and write it as bf16 hi/lo into the
// planes at hi / lo.  Called by all BT_PWARPS producer warps (thread index tid < 256).
__device__ __forceinline__ void produce(const float* __restrict__ src, int64_t rs, int64_t ks, int nrows, int k0,
                                        int nk, float coef, uint32_t hi, uint32_t lo, int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    if (ks == 1) {
        // K contiguous: the lanes of a warp read one row's 32 K values (256 bytes) per
        // instruction; each warp takes 16 rows, even lanes store the pair (k, k + 1)
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int r = warp * 16 + i;
            v[i] = (r < nrows && lane < nk) ? coef * src[(int64_t)r * rs + k0 + lane] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float nb = __shfl_down_sync(0xffffffffu, v[i], 1);
            if ((lane & 1) == 0) {
                uint32_t h, l;
                split2(v[i], nb, h, l);
                const uint32_t o = swz(warp * 16 + i, lane);
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(hi + o), "r"(h) : "memory");
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(lo + o), "r"(l) : "memory");
            }
        }
    } else {
        // rows contiguous (or neither): thread = row (lanes along the rows), half the K block
        // each: threads 0..127 take k in [0, 16), threads 128..255 k in [16, 32)
        const int r = tid & 127, kh = (tid >> 7) * 16;
        const float* row = src + (int64_t)r * rs;
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
            v[k] = (r < nrows && kh + k < nk) ? coef * row[(int64_t)(k0 + kh + k) * ks] : 0.f;
        uint32_t h2[8], l2[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) split2(v[2 * p], v[2 * p + 1], h2[p], l2[p]);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t o = swz(r, kh + 8 * j);
            st_shared_v4(hi + o, h2[4 * j], h2[4 * j + 1], h2[4 * j + 2], h2[4 * j + 3]);
            st_shared_v4(lo + o, l2[4 * j], l2[4 * j + 1], l2[4 * j + 2], l2[4 * j + 3]);
        }
    }
}

// resident CTAs per SM the register allocation must allow (2 forces spills of the producer)
#ifndef HEFF_BT_MINB
#define HEFF_BT_MINB 1
#endif
template <typename TC>
__global__ void __launch_bounds__(BT_THREADS, HEFF_BT_MINB) bgemm_tc_kernel(BtArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + BT_BAR);
    uint64_t* empty = full + BT_STAGES;
    uint64_t* done = empty + BT_STAGES;
    uint64_t* drain = done + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const BTile t = g.tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < BT_STAGES; ++s) { mbar_init(&full[s], BT_PWARPS); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == BT_PWARPS) tmem_alloc(tmem_slot, BT_N);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t base = su32(smem);
    // the scale in FP32 (one FP64 divide per thread; the tile's values carry ~1e-5 anyway)
    const float scale = (float)(g.inv_scale ? g.scale / g.inv_scale[0] : g.scale);
    bool have_acc = false;                    // the accumulator holds this tile's sum

    if (warp < BT_PWARPS) {
        // ------------------------------------------------ producers
        int step = 0;
        bool ok = true;
        for (int pi = 0; pi < t.prod_count && ok; ++pi) {
            const BProd p = g.prods[t.prod_begin + pi];
            const float coef = f64_to_f32_rn((p.c1 < 0 ? 1.0 : g.coef1[p.c1]) * (p.c2 < 0 ? 1.0 : g.coef2[p.c2]));
            for (int k0 = 0; k0 < p.K; k0 += BT_KB, ++step) {
                const int s = step % BT_STAGES;
                const uint32_t use = (uint32_t)(step / BT_STAGES);
                if (!(ok = mbar_wait(&empty[s], (use & 1) ^ 1, abort_flag, g.err))) break;
                const int nk = p.K - k0 < BT_KB ? p.K - k0 : BT_KB;
                const uint32_t st = base + (uint32_t)(s * BT_STAGE);
                // A rows r: A[a_off + r a_rs + k a_cs]; B "rows" = output columns c:
                // B[b_off + k b_rs + c b_cs]
                produce(g.A + p.a_off, p.a_rs, p.a_cs, t.m, k0, nk, coef, st, st + BT_PLANE, threadIdx.x);
                produce(g.B + p.b_off, p.b_cs, p.b_rs, t.n, k0, nk, 1.f, st + 2 * BT_PLANE, st + 3 * BT_PLANE,
                        threadIdx.x);
                fence_async_smem();          // the writes are visible to the tensor core's reads
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t nmma = t.n <= 16 ? 16u : (uint32_t)((t.n + 15) & ~15);
        const uint32_t id = idesc_bf16(BT_M, nmma);
        int step = 0;
        bool ok = true, first = true;
        for (int pi = 0; pi < t.prod_count && ok; ++pi) {
            const int K = g.prods[t.prod_begin + pi].K;
            for (int k0 = 0; k0 < K; k0 += BT_KB, ++step) {
                const int s = step % BT_STAGES;
                const uint32_t use = (uint32_t)(step / BT_STAGES);
                if (!(ok = mbar_wait(&full[s], use & 1, abort_flag, g.err))) break;
                tc_fence_after();
                const uint32_t st = base + (uint32_t)(s * BT_STAGE);
                const uint64_t ahi = sdesc64(st), alo = sdesc64(st + BT_PLANE);
                const uint64_t bhi = sdesc64(st + 2 * BT_PLANE), blo = sdesc64(st + 3 * BT_PLANE);
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint64_t o = (uint64_t)(kk * 32) >> 4;     // 32-byte K step in the row
                    umma_bf16(tmem, ahi + o, bhi + o, id, first ? 0u : 1u);
                    umma_bf16(tmem, ahi + o, blo + o, id, 1u);
                    umma_bf16(tmem, alo + o, bhi + o, id, 1u);
                    first = false;
                }
                umma_commit(&empty[s]);
            }
        }
        if (ok && !first) umma_commit(done);           // arrives when every MMA has completed
        else if (ok) mbar_arrive(done);                // nothing to contract: zero tile
        else {
            // aborted: wait (bounded) for the MMAs already issued before the memory goes away
            umma_commit(drain);
            mbar_wait_drain(drain, 0);
        }
    }
    if (warp < BT_PWARPS) {
        // ------------------------------------------------ epilogue
        const bool ok = mbar_wait(done, 0, abort_flag, g.err);
        tc_fence_after();
        int nprod_k = 0;
        for (int pi = 0; pi < t.prod_count; ++pi) nprod_k += g.prods[t.prod_begin + pi].K;
        have_acc = nprod_k > 0;
        if (ok) {
            // two warps per tensor-memory lane quarter (rows q*32 ..), alternate 32-column chunks
            const int q = warp & 3, h = warp >> 2;
            float* tr = reinterpret_cast<float*>(smem) + warp * 32 * 33;   // the ring is idle now
            const int rows = t.m - q * 32 < 32 ? t.m - q * 32 : 32;         // valid rows of this warp
            for (int c0 = 32 * h; c0 < t.n; c0 += 64) {
                __syncwarp();
#pragma unroll
                for (int half = 0; half < 2; ++half) {   // 16 columns per tensor-memory load
                    uint32_t raw[16];
                    if (have_acc) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c0 + 16 * half), raw);
                    else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) raw[i] = 0u;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) tr[lane * 33 + 16 * half + i] = __uint_as_float(raw[i]);
                }
                __syncwarp();
                const int c = c0 + lane;
                if (c < t.n)
                    for (int rr = 0; rr < rows; ++rr) {
                        TC* cp = static_cast<TC*>(g.C) + t.c_off + (int64_t)(q * 32 + rr) * t.ldc + c;
                        const float v = scale * tr[rr * 33 + lane];
                        if constexpr (std::is_same<TC, double>::value) *cp = g.accumulate ? *cp + f32_to_f64(v) : f32_to_f64(v);
                        else *cp = g.accumulate ? *cp + v : v;
                    }
                __syncwarp();
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == BT_PWARPS) {
        tc_fence_after();
        tmem_dealloc(tmem, BT_N);
    }
}

__global__ void __launch_bounds__(256) convert_f64_f32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                                                              int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = f64_to_f32_rn(src[i]);
}

template <typename TC>
int launch_t(const BList& b, const float* A, const float* B, void* C, const double* coef1, const double* coef2,
             double scale, cudaStream_t st, const double* inv_scale, int* err) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(bgemm_tc_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM);
        if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        attr = true;
    }
    BtArgs g{b.d_tiles, b.d_prods, A, B, C, coef1, coef2, scale, inv_scale, b.accumulate ? 1 : 0, err};
    bgemm_tc_kernel<TC><<<(unsigned)b.tiles.size(), BT_THREADS, BT_SMEM, st>>>(g);
    return HEFF_OK;
}

}  // namespace

int launch_bgemm_tc(const BList& b, const float* A, const float* B, void* C, bool c_f64, const double* coef1,
                    const double* coef2, double scale, void* stream, const double* inv_scale, int* err) {
    if (b.tiles.empty()) return HEFF_OK;
    if (b.tile_m != BT_M || b.tile_n != BT_N)
        return fail(HEFF_ERR_INVALID_ARG, "tensor-core block products need %d x %d tiles", BT_M, BT_N);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = c_f64 ? launch_t<double>(b, A, B, C, coef1, coef2, scale, st, inv_scale, err)
                   : launch_t<float>(b, A, B, C, coef1, coef2, scale, st, inv_scale, err);
    if (rc) return rc;
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "bgemm_tc launch: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

int launch_convert_f64_f32(const double* src, float* dst, int64_t n, void* stream) {
    if (n <= 0) return HEFF_OK;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    convert_f64_f32_kernel<<<(unsigned)g, 256, 0, static_cast<cudaStream_t>(stream)>>>(src, dst, n);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "convert launch: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

}  // namespace heff
