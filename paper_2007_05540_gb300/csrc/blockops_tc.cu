// Tensor-core form of the block-product engine of blockops.cu (the charge-matched block-pair
// products of Algorithm 2, summed into output tiles, Section IV "list" algorithm): the same
// tile and product lists, cut into 128 x 128 output tiles, with every product contracted on
// the sm_103a tensor cores in the BF16x3 split (hi = bf16(v), lo = bf16(v - hi); per K block
// A_hi.B_hi + A_hi.B_lo + A_lo.B_hi, FP32 accumulation in tensor memory).
//
// One CTA per output tile, 5 warps:
//   warps 0..3  producers: each thread owns one row of the A block and one row of the
//               (transposed) B block per K block of 32 elements; it loads the 32 FP64 values
//               with the product's strides (scaled by the product's MPO coefficient),
//               splits them into bf16 hi/lo and writes them into the 64-byte-swizzled
//               K-major shared-memory layout the MMA reads; a ring of 3 stages.  After the
//               last MMA they are the epilogue: tensor memory -> registers -> a per-warp
//               shared-memory transpose -> coalesced FP64 row stores (C = scale * acc, or
//               C += scale * acc).
//   warp 4      allocates 128 tensor-memory columns; one thread issues the MMAs.
// Operands come in with arbitrary strides (environment blocks, site tensors, transposed
// views), so the loads are plain global loads rather than TMA copies.  Every mbarrier wait
// is bounded; on expiry the CTA raises the error flag, stops issuing work, waits (bounded)
// for the MMAs it has already issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace heff {
namespace {

using namespace ptx;

constexpr int BT_M = 128, BT_N = 128;       // output tile
constexpr int BT_KB = 32;                   // K elements per block: one 64-byte bf16 row
constexpr int BT_STAGES = 3;
constexpr int BT_PWARPS = 4;
constexpr int BT_THREADS = 32 * (BT_PWARPS + 1);
constexpr int BT_PLANE = BT_M * 64;         // one 128-row plane of a K block: 8 KB
constexpr int BT_STAGE = 4 * BT_PLANE;      // A hi, A lo, B hi, B lo
constexpr int BT_BAR = BT_STAGES * BT_STAGE;
constexpr int BT_SMEM = BT_BAR + 256 + 1024;   // + barriers, alignment slack
static_assert(BT_PWARPS * 32 == BT_M && BT_M == BT_N, "one producer thread per A row and per B row");
static_assert(BT_PWARPS * 32 * 33 * 4 <= BT_BAR, "the epilogue transpose fits in the ring");

struct BtArgs {
    const BTile* tiles;
    const BProd* prods;
    const double* A;
    const double* B;
    double* C;
    const double* coef1;
    const double* coef2;
    double scale;
    const double* inv_scale;
    int accumulate;
    int* err;
};

// Split 32 values into bf16 hi/lo and store them as row r of the two planes at `hi`, `lo`
// (64-byte rows, 16-byte chunk j at j ^ ((r >> 1) & 3)).
__device__ __forceinline__ void store_row(uint32_t hi, uint32_t lo, int r, const float (&v)[32]) {
    uint32_t h2[16], l2[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * p], v[2 * p + 1]);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * p] - __low2float(h), v[2 * p + 1] - __high2float(h));
        h2[p] = *reinterpret_cast<const uint32_t*>(&h);
        l2[p] = *reinterpret_cast<const uint32_t*>(&l);
    }
    const uint32_t ro = (uint32_t)r * 64;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t o = ro + ((uint32_t)(j ^ ((r >> 1) & 3)) << 4);
        st_shared_v4(hi + o, h2[4 * j], h2[4 * j + 1], h2[4 * j + 2], h2[4 * j + 3]);
        st_shared_v4(lo + o, l2[4 * j], l2[4 * j + 1], l2[4 * j + 2], l2[4 * j + 3]);
    }
}

__global__ void __launch_bounds__(BT_THREADS, 2) bgemm_tc_kernel(BtArgs g) {
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
    double scale = g.scale;
    if (g.inv_scale) scale /= g.inv_scale[0];
    bool have_acc = false;                    // the accumulator holds this tile's sum

    if (warp < BT_PWARPS) {
        // ------------------------------------------------ producers
        const int r = threadIdx.x;            // A row and B row (output column) of this thread
        int step = 0;
        bool ok = true;
        for (int pi = 0; pi < t.prod_count && ok; ++pi) {
            const BProd p = g.prods[t.prod_begin + pi];
            const float coef = (float)((p.c1 < 0 ? 1.0 : g.coef1[p.c1]) * (p.c2 < 0 ? 1.0 : g.coef2[p.c2]));
            const double* arow = g.A + p.a_off + (int64_t)r * p.a_rs;
            const double* bcol = g.B + p.b_off + (int64_t)r * p.b_cs;
            const bool av = r < t.m, bv = r < t.n;
            for (int k0 = 0; k0 < p.K; k0 += BT_KB, ++step) {
                const int s = step % BT_STAGES;
                const uint32_t use = (uint32_t)(step / BT_STAGES);
                if (!(ok = mbar_wait(&empty[s], (use & 1) ^ 1, abort_flag, g.err))) break;
                const int nk = p.K - k0 < BT_KB ? p.K - k0 : BT_KB;
                float va[32], vb[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    va[k] = (av && k < nk) ? coef * (float)arow[(int64_t)(k0 + k) * p.a_cs] : 0.f;
                    vb[k] = (bv && k < nk) ? (float)bcol[(int64_t)(k0 + k) * p.b_rs] : 0.f;
                }
                const uint32_t st = base + (uint32_t)(s * BT_STAGE);
                store_row(st, st + BT_PLANE, r, va);
                store_row(st + 2 * BT_PLANE, st + 3 * BT_PLANE, r, vb);
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
            float* tr = reinterpret_cast<float*>(smem) + warp * 32 * 33;   // the ring is idle now
            const int rows = t.m - warp * 32 < 32 ? t.m - warp * 32 : 32;   // valid rows of this warp
            for (int c0 = 0; c0 < t.n; c0 += 32) {
                uint32_t raw[32];
                if (have_acc) tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, raw);
                else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) raw[i] = 0u;
                }
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 32; ++i) tr[lane * 33 + i] = __uint_as_float(raw[i]);
                __syncwarp();
                const int c = c0 + lane;
                if (c < t.n)
                    for (int rr = 0; rr < rows; ++rr) {
                        double* cp = g.C + t.c_off + (int64_t)(warp * 32 + rr) * t.ldc + c;
                        const double v = scale * (double)tr[rr * 33 + lane];
                        *cp = g.accumulate ? *cp + v : v;
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

}  // namespace

int launch_bgemm_tc(const BList& b, const double* A, const double* B, double* C, const double* coef1,
                    const double* coef2, double scale, void* stream, const double* inv_scale, int* err) {
    if (b.tiles.empty()) return HEFF_OK;
    if (b.tile_m != BT_M || b.tile_n != BT_N)
        return fail(HEFF_ERR_INVALID_ARG, "tensor-core block products need %d x %d tiles", BT_M, BT_N);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(bgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM);
        if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        attr = true;
    }
    BtArgs g{b.d_tiles, b.d_prods, A, B, C, coef1, coef2, scale, inv_scale, b.accumulate ? 1 : 0, err};
    bgemm_tc_kernel<<<(unsigned)b.tiles.size(), BT_THREADS, BT_SMEM, static_cast<cudaStream_t>(stream)>>>(g);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "bgemm_tc launch: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

}  // namespace heff
