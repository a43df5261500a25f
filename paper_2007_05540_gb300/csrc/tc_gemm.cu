// Tensor-core grouped GEMM (sm_103a: TMA -> shared memory -> tcgen05.mma -> TMEM) for the
// split-precision paths of the two-site H_eff matvec (Section II-C / Fig. 1d).
//
// Each task is one output tile C[m x n] (m <= 128, n <= TN) = sum over its contraction
// segments of A[a_row + r, k] * B[b_row + c, k].  A and B live in the workspace as hi and
// lo halves of one element type, interleaved by 64-byte K blocks within each row, so one
// TMA box with 128-byte rows brings both halves of a K block:
//   BF16X3: bf16 halves, kind::f16 MMAs;  TF32X3: fp32 halves read as TF32, kind::tf32.
// Every K block does three MMAs, A_hi.B_hi + A_hi.B_lo + A_lo.B_hi, accumulated in FP32
// in tensor memory (the "3-product" split: error ~ 2^-16 (bf16) / 2^-22 (tf32) relative).
//
// Persistent kernel, one CTA per SM (10 warps in BF16x3, 6 in TF32x3), static round-robin
// over the task list (which the planner orders as a longest-processing-time schedule):
//   warp 0      one thread issues the TMA loads of a STAGES-deep shared-memory ring
//   warp 1      allocates TMEM (2 x TN columns); one thread issues the MMAs
//   warps 2..   epilogue (8 warps in BF16x3, two per TMEM lane quarter on alternate
//               32-column chunks; 4 in TF32x3): TMEM -> registers -> global
// Accumulators are double buffered so a tile's epilogue overlaps the next tile's MMAs.
// Long contractions (GEMM 2) are accumulated in chunks of kchunk K blocks: each chunk
// starts a fresh accumulator and the epilogue adds the chunks into y in a fixed order with
// round-to-nearest adds.  The tensor cores' FP32 accumulation drops low bits at every step,
// which biases a long sum toward zero (relative bias growing with the number of steps);
// chunking bounds the steps per accumulator.
// T (GEMM 1) leaves through TMA: each warp splits 32 rows x 32 columns into hi/lo in
// registers, writes them to a swizzled shared-memory box (hi and lo K blocks side by side,
// the workspace's interleaved rows) and issues bulk tensor stores;
// quarters with fewer than 32 valid rows go through an XOR-swizzled transpose and leave
// in 16-byte row pieces (several rows per store instruction); y (GEMM 2, per-block pitch)
// leaves through the same transpose in 128-byte row stores.
// Every mbarrier wait is bounded (about a second); on expiry the CTA raises the
// workspace error flag and stops issuing work; the producer then waits (bounded) for the
// loads it has already issued and the MMA issuer for the MMAs it has already issued, and
// only then is the tensor memory freed and the CTA (with its ring) released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "convert.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

// work order of batched launches: 1 = the batch entries of a task consecutively
#ifndef HEFF_BATCH_INNER
#define HEFF_BATCH_INNER 1
#endif

namespace heff {
namespace {

using namespace ptx;

// Warps: 0 TMA producer, 1 MMA issuer, then the epilogue: 8 warps for BF16X3 (two per
// tensor-memory lane quarter, alternating 32-column chunks), 4 for TF32X3 (whose 32 x 32
// fp32 store boxes need twice the shared memory per warp).
#ifndef HEFF_EPI_WARPS_BF16
#define HEFF_EPI_WARPS_BF16 8
#endif
template <int PREC> __host__ __device__ constexpr int tc_epi_warps() {
    return PREC == HEFF_PREC_BF16X3 ? HEFF_EPI_WARPS_BF16 : 4;
}
template <int PREC> __host__ __device__ constexpr int tc_threads() { return 64 + 32 * tc_epi_warps<PREC>(); }
constexpr int TM = 128;

// Shared-memory ring: STAGES x {A (128 rows), B (TN rows)}, each row one K block of the hi
// half (SWZ = 64 bytes: 32 bf16 / 16 fp32) followed by the same K block of the lo half, in
// the 128-byte swizzle; then 32 KB shared by the epilogue warps (per warp: the TMA store
// boxes of a 32-column chunk of T, or the 32 x 32 float transpose), then barriers.
template <int TN, int STAGES, int SWZ>
struct Smem {
    static constexpr int A_BYTES = TM * 2 * SWZ;
    static constexpr int B_BYTES = TN * 2 * SWZ;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int EPI_OFF = STAGES * STAGE_BYTES;  // 1024-byte aligned
    static constexpr int EPI_BYTES = 32768;
    static constexpr int BAR_OFF = EPI_OFF + EPI_BYTES;
    static constexpr int TOTAL = BAR_OFF + 256 + 1024;    // + barriers, alignment slack
};
static_assert(32 * 32 * 4 <= 32768 / 8, "transpose buffer fits an epilogue slot");

// TMA maps of one GEMM: the A operand with 64- and 128-row boxes, the B operand with 64-,
// 128- and 256-row boxes (a tile loads the smallest box that covers its valid rows; each CTA
// of a pair loads the smallest of 32, 64 or 128 rows that covers its half).
struct TcMaps {
    CUtensorMap a[2];
    CUtensorMap b[3];
    CUtensorMap c;      // T store map: 32 x 32 boxes (GEMM 1 only)
    CUtensorMap bq;     // B operand, 32-row box (a CTA pair's half of a narrow B tile)
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand with SWZ-byte rows swizzled in 8-row
// groups (SWZ = 128: SWIZZLE_128B, groups 1024 B apart; SWZ = 64: SWIZZLE_64B, 512 B).
template <int SWZ>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * SWZ) >> 4) << 32;           // stride byte offset: one 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)(SWZ == 128 ? 2 : (SWZ == 64 ? 4 : 6)) << 61;   // SWIZZLE_128B / 64B / 32B
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B format fmt (1 = BF16, 2 = TF32), K-major, M x N.
__device__ __forceinline__ uint32_t idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (PREC == HEFF_PREC_BF16X3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
    }
}


// CTA-pair forms (cta_group::2): the MMA of a pair is issued by the even CTA and reads A
// and its half of B from each CTA's shared memory at the same offsets; its commit arrives
// on the barrier at this offset in both CTAs.
template <int PREC>
__device__ __forceinline__ void umma2(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (PREC == HEFF_PREC_BF16X3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
    }
}
__device__ __forceinline__ void umma2_commit_both(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
        ::"r"(su32(bar)), "h"((uint16_t)3) : "memory");
}

// Arrives on this CTA's barrier once every MMA of the pair issued before it has completed.
__device__ __forceinline__ void umma2_commit_own(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

// TMA load into this CTA's shared memory, completion signalled on a barrier of either CTA of
// the pair (`bar` is a shared::cluster address).
__device__ __forceinline__ void tma_load_pair(void* dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%3, %4}], [%2];"
        ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// shared::cluster address of this CTA's variable `p` in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of every CTA of the cluster (shared-memory writes before it are visible after).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Bulk tensor store of one shared-memory box; completion tracked by bulk async-groups.
__device__ __forceinline__ void tma_store(const CUtensorMap* map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

struct TcArgs {
    const GemmTask* tasks;
    const KSeg* segs;
    int ntasks, nbatch;
    int64_t a_batch_rows, b_batch_rows;   // row offset per batch entry
    char* C;                              // mode 0: T
    int64_t c_batch_elems;                // element offset of T per batch entry
    int c_batch_rows;                     // the same in rows of the T store map
    PtrBatch y;                           // mode 1: outputs per batch entry
    int mode;                             // 0: write T (interleaved hi/lo rows), 1: write y
    int kchunk;                           // K blocks per accumulation chunk (0: whole tile)
    int y_f64;                            // y element type (mode 1)
    int b0;                               // first batch entry of this launch
    int* err;                             // sticky error flag in the workspace
};

// CL = 1: every CTA runs its own 128-row tiles.  CL = 2: the two CTAs of a cluster run the
// two tiles of one entry (tasks 2e, 2e + 1: the same B rows and K segments) as one M = 256
// tile with pair MMAs (tcgen05 cta_group::2): each CTA loads its own 128 A rows and half of
// the B rows into its ring, the even CTA waits for both halves on its barrier and issues the
// MMAs, whose commits release both rings and hand each CTA the accumulator of its own rows
// in its own tensor memory.  Per CTA this halves the B operand in shared memory (ring
// stages of 32 KB instead of 48 KB) and the shared-memory bytes the tensor core reads per
// MMA.  A pair's second task may be a ghost (m = 0: computed, not stored).
template <int PREC, int TN, int STAGES, int SWZ, int CL>
__global__ void __launch_bounds__(tc_threads<PREC>(), 1)
tc_gemm_kernel(const __grid_constant__ TcMaps maps, TcArgs g) {
    static_assert(SWZ == 64, "a K block of one half is 64 bytes; hi + lo fill a 128-byte row");
    using S = Smem<TN / CL, STAGES, SWZ>;      // B rows per CTA: TN, or TN / 2 in a pair
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;      // [2]
    uint64_t* tempty = tfull + 2;          // [2]
    uint64_t* drain = tempty + 2;          // the MMAs issued before an abort have completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&tfull[a], 1); mbar_init(&tempty[a], tc_epi_warps<PREC>() * CL); }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (CL == 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(su32(tmem_slot)), "r"(2 * TN) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        } else {                               // one warp of each CTA of the pair, collectively
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(su32(tmem_slot)), "r"(2 * TN) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (CL > 1) cluster_sync();  // the peer's barriers exist before anything reaches them
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // programmatic dependent launch: the prologue above touched only this CTA's own state;
    // the operands written by the previous kernel on the stream are read from here on.
    // The successor may then be scheduled onto SMs as these CTAs retire.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t rank = CL > 1 ? cluster_rank() : 0u;
    const long cid = (long)(blockIdx.x / CL), ncl = (long)(gridDim.x / CL);
    const long nent = g.ntasks / CL;                                 // entries per batch
    const long total = nent * g.nbatch;
    // work item gi -> (entry, batch entry).  Batch-inner order: the batch entries of one
    // task follow each other, so the CTAs that run them at the same time share its operand
    // tiles (the A tile of GEMM 1, the B tile of GEMM 2) through L2.  With one batch entry
    // both orders are the planner's order.
    const long nbl = g.nbatch;
    auto ent = [&](long gi) { return HEFF_BATCH_INNER ? gi / nbl : gi % nent; };
    auto bat = [&](long gi) { return (int)(HEFF_BATCH_INNER ? gi % nbl : gi / nent); };
    constexpr int KB = SWZ / (PREC == HEFF_PREC_BF16X3 ? 2 : 4);   // elements per K block
    constexpr int KSUB = SWZ / 32;                                   // MMAs (32-byte K) per block

    // the even CTA's full barriers (pair: both CTAs' loads complete there) and its tempty
    // barriers (pair: both CTAs' epilogues release the accumulators there)
    const uint32_t full_pair = CL > 1 ? cluster_addr(full, 0) : 0u;
    const uint32_t tempty_pair = CL > 1 ? cluster_addr(tempty, 0) : 0u;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        uint32_t st = 0, ph = 0;               // ring stage and its phase parity
        uint32_t issued = 0;                   // stages filled so far
        bool ok = true;
        // the next task and the next segment are loaded one step ahead, so their latency
        // overlaps with the current loads instead of draining the ring
        GemmTask tn = cid < total ? g.tasks[CL * ent(cid) + rank] : GemmTask{};
        for (long gi = cid; gi < total && ok; gi += ncl) {
            const GemmTask t = tn;
            if (gi + ncl < total) tn = g.tasks[CL * ent(gi + ncl) + rank];
            const int b = g.b0 + bat(gi);
            const int ar = (int)(t.a_row + b * g.a_batch_rows), br = (int)(t.b_row + b * g.b_batch_rows);
            const int ia = t.m <= 64 ? 0 : 1, ib = t.n <= 64 ? 0 : (t.n <= 128 ? 1 : 2);
            const CUtensorMap* ma = &maps.a[CL == 1 ? ia : 1];   // a pair always loads 128 A rows
            const CUtensorMap* mb = &maps.b[ib];
            // pair: this CTA's half of the MMA's N columns, and the smallest box covering it
            const int half = (t.n <= 16 ? 16 : (t.n + 15) & ~15) / 2;
            const int hb = half <= 32 ? 0 : (half <= 64 ? 1 : 2);
            const CUtensorMap* mh = hb == 0 ? &maps.bq : &maps.b[hb - 1];
            const uint32_t bytes = CL == 1 ? 2u * (uint32_t)((64 << ia) + (64 << ib)) * SWZ
                                           : (uint32_t)CL * 2u * (uint32_t)(128 + (32 << hb)) * SWZ;
            // a K block at column k of the rows starts at element 2 k of the interleaved rows
            KSeg sn = t.seg_count > 0 ? g.segs[t.seg_begin] : KSeg{};
            for (int s = 0; s < t.seg_count && ok; ++s) {
                const KSeg sg = sn;
                if (s + 1 < t.seg_count) sn = g.segs[t.seg_begin + s + 1];
                for (int k = sg.k0; k < sg.k0 + sg.klen; k += KB) {
                    if (!(ok = mbar_wait(&empty[st], ph ^ 1, abort_flag, g.err))) break;
                    uint8_t* base = smem + st * S::STAGE_BYTES;
                    if constexpr (CL == 1) {
                        mbar_expect_tx(&full[st], bytes);
                        tma_load(base, ma, &full[st], 2 * k, ar);
                        tma_load(base + S::A_BYTES, mb, &full[st], 2 * k, br);
                    } else {
                        // both CTAs' loads complete on the even CTA's barrier, which expects them all
                        const uint32_t fb = full_pair + (uint32_t)(st * sizeof(uint64_t));
                        if (rank == 0) mbar_expect_tx(&full[st], bytes);
                        tma_load_pair(base, ma, fb, 2 * k, ar);
                        tma_load_pair(base + S::A_BYTES, mh, fb, 2 * k, br + (int)rank * half);
                    }
                    ++issued;
                    if (++st == STAGES) { st = 0; ph ^= 1; }
                }
            }
        }
        if (!ok && rank == 0) {
            // aborted: the loads already issued still write this CTA's ring (and, for a pair,
            // the odd CTA's) and complete on these barriers; wait (bounded) for the last
            // STAGES fills to land before the shared memory can go away
            const uint32_t nf = issued < (uint32_t)STAGES ? issued : (uint32_t)STAGES;
            for (uint32_t i = 1; i <= nf; ++i) {
                const uint32_t f = issued - i;
                mbar_wait_drain(&full[f % STAGES], (f / STAGES) & 1);
            }
        }
        if constexpr (CL > 1) {
            // every stage released by the pair's last MMAs: no commit from the even CTA is
            // still on its way to this CTA when it leaves
            for (int s = 0; s < STAGES && ok; ++s) {
                ok = mbar_wait(&empty[st], ph ^ 1, abort_flag, g.err);
                if (++st == STAGES) { st = 0; ph ^= 1; }
            }
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ------------------------------------------------ MMA issuer (the even CTA of a pair)
        constexpr uint32_t FMT = PREC == HEFF_PREC_BF16X3 ? 1u : 2u;
        // This thread feeds the tensor pipe: per K block it only waits, adds constant offsets
        // to precomputed descriptors and issues (no divisions, no descriptor packing).
        const int CH = g.kchunk > 0 ? g.kchunk : 0x7fffffff;
        uint32_t ccount = 0;                   // accumulator chunk counter
        uint32_t st = 0, ph = 0;               // ring stage and its phase parity
        const uint64_t dsc0 = sdesc<2 * SWZ>(su32(smem));
        // the lo half of a K block is SWZ bytes into each 128-byte row
        constexpr uint64_t O_LO = (uint64_t)SWZ >> 4, O_B = S::A_BYTES >> 4, O_STAGE = S::STAGE_BYTES >> 4;
        bool ok = true;
        GemmTask tn = cid < total ? g.tasks[CL * ent(cid) + rank] : GemmTask{};
        for (long gi = cid; gi < total && ok; gi += ncl) {
            const GemmTask t = tn;
            if (gi + ncl < total) tn = g.tasks[CL * ent(gi + ncl) + rank];
            if (t.seg_count == 0) {            // nothing to contract: the epilogue writes zeros
                const uint32_t acc = ccount & 1, use = ccount >> 1;
                if (!(ok = mbar_wait(&tempty[acc], (use & 1) ^ 1, abort_flag, g.err))) break;
                if constexpr (CL == 1) mbar_arrive(&tfull[acc]);
                else umma2_commit_both(&tfull[acc]);
                ++ccount;
                continue;
            }
            const int nkb = t.ktotal / KB;
            const uint32_t nmma = t.n <= 16 ? 16u : (uint32_t)((t.n + 15) & ~15);
            const uint32_t id = idesc(FMT, TM * CL, nmma);
            uint32_t first = 1, acc = 0, d = 0;
            int left = 0;                      // K blocks left in the current chunk
            // the ring holds the tile's K blocks in order: only their number matters here
            for (int kb = 0; kb < nkb && ok; ++kb) {
                if (left == 0) {               // a new accumulation chunk
                    acc = ccount & 1;
                    const uint32_t use = ccount >> 1;
                    if (!(ok = mbar_wait(&tempty[acc], (use & 1) ^ 1, abort_flag, g.err))) break;
                    tc_fence_after();
                    d = tmem + acc * TN;
                    first = 1;
                    left = nkb - kb < CH ? nkb - kb : CH;
                }
                if (!(ok = mbar_wait(&full[st], ph, abort_flag, g.err))) break;
                tc_fence_after();
                const uint64_t ahi = dsc0 + st * O_STAGE, alo = ahi + O_LO;
                const uint64_t bhi = ahi + O_B, blo = bhi + O_LO;
#pragma unroll
                for (int kk = 0; kk < KSUB; ++kk) {
                    const uint64_t o = (uint64_t)(kk * 32) >> 4;     // 32-byte step inside the row
                    if constexpr (CL == 1) {
                        umma<PREC>(d, ahi + o, bhi + o, id, first ? 0u : 1u);
                        umma<PREC>(d, ahi + o, blo + o, id, 1u);
                        umma<PREC>(d, alo + o, bhi + o, id, 1u);
                    } else {
                        umma2<PREC>(d, ahi + o, bhi + o, id, first ? 0u : 1u);
                        umma2<PREC>(d, ahi + o, blo + o, id, 1u);
                        umma2<PREC>(d, alo + o, bhi + o, id, 1u);
                    }
                    first = 0;
                }
                if constexpr (CL == 1) umma_commit(&empty[st]);
                else umma2_commit_both(&empty[st]);
                if (++st == STAGES) { st = 0; ph ^= 1; }
                if (--left == 0) {
                    if constexpr (CL == 1) umma_commit(&tfull[acc]);
                    else umma2_commit_both(&tfull[acc]);
                    ++ccount;
                }
            }
        }
        if (!ok) {
            // aborted: wait (bounded) for the MMAs already issued, which read the ring(s) and
            // write tensor memory, before either is released
            if constexpr (CL == 1) umma_commit(drain);
            else umma2_commit_own(drain);
            mbar_wait_drain(drain, 0);
        }
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue
        // Each warp drains its 32 TMEM lanes (tile rows) 32 columns at a time (tcgen05.ld:
        // thread = row); the warps of a lane quarter take alternate 32-column chunks.  T, full
        // quarters: hi/lo split in registers, swizzled box of 128-byte rows (a K block of hi
        // values, then of lo values) in shared memory, bulk tensor stores (one box for bf16,
        // two for fp32).  Otherwise: transpose through a 32 x 32 buffer (XOR
        // swizzled: conflict-free both ways) and store row by row with consecutive lanes on
        // consecutive columns.
        using E = typename std::conditional<PREC == HEFF_PREC_BF16X3, __nv_bfloat16, float>::type;
        constexpr int NEPI = tc_epi_warps<PREC>();
        constexpr int NH = NEPI / 4;                                // warps per lane quarter
        constexpr int SLOT = S::EPI_BYTES / NEPI;
        // a 32-column chunk of T rows: 32 rows of hi + lo K blocks, 128 bytes per K block
        // (one box for bf16, two for fp32), BOX bytes per box
        constexpr int BOX = 32 * 128;
        constexpr int NBOX = 32 * (int)sizeof(E) / 64;
        static_assert(NBOX * BOX <= SLOT, "the store boxes of a chunk fit an epilogue slot");
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;          // its chunk phase within the quarter
        uint8_t* slot = smem + S::EPI_OFF + (warp - 2) * SLOT;
        float* stage = reinterpret_cast<float*>(slot);
        const uint32_t slot_s = su32(slot);
        const int CH = g.kchunk > 0 ? g.kchunk : 0x7fffffff;
        uint32_t ccount = 0;
        bool live = true;
        for (long gi = cid; gi < total && live; gi += ncl) {
            const GemmTask t = g.tasks[CL * ent(gi) + rank];
            const int brel = bat(gi), b = g.b0 + brel;
            const int nch = (t.seg_count > 0 && CH != 0x7fffffff) ? (t.ktotal / KB + CH - 1) / CH : 1;
          for (int ch = 0; ch < nch; ++ch) {
            const uint32_t acc = ccount & 1, use = ccount >> 1;
            if (!mbar_wait(&tfull[acc], use & 1, abort_flag, g.err)) { live = false; break; }
            tc_fence_after();
            const int ncols = t.n + t.n_zero;
            const int rows = t.m - q * 32 < 32 ? t.m - q * 32 : 32;   // valid rows of this warp
            const bool boxed = g.mode == 0 && rows == 32;              // warp-uniform
            int x0 = 0, yh = 0;
            if (boxed) {
                x0 = (int)(t.c_off % t.ldc);
                yh = (int)(t.c_off / t.ldc) + q * 32 + b * g.c_batch_rows;
            }
            for (int c0 = 32 * h; c0 < ncols; c0 += 32 * NH) {
                uint32_t raw[32];
                if (t.seg_count > 0) {
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * TN + c0, raw);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) raw[i] = 0u;
                }
                if (rows <= 0) continue;                       // warp-uniform
                if (boxed) {
                    // the slot's previous bulk stores must have finished reading it
                    if (lane == 0) bulk_wait_read<0>();
                    __syncwarp();
                    const uint32_t hb = slot_s;
                    const int nv = t.n - c0;                   // valid columns in this chunk
                    if constexpr (PREC == HEFF_PREC_BF16X3) {
                        // row = lane: the 32 hi values (16-byte chunks 0-3), then the 32 lo
                        // values (chunks 4-7), chunk j stored at j ^ (row & 7)
                        uint32_t h2[16], l2[16];
#pragma unroll
                        for (int p = 0; p < 16; ++p) {
                            const float f0 = 2 * p < nv ? __uint_as_float(raw[2 * p]) : 0.f;
                            const float f1 = 2 * p + 1 < nv ? __uint_as_float(raw[2 * p + 1]) : 0.f;
                            const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
                            const __nv_bfloat162 l = __floats2bfloat162_rn(f0 - __low2float(h), f1 - __high2float(h));
                            h2[p] = *reinterpret_cast<const uint32_t*>(&h);
                            l2[p] = *reinterpret_cast<const uint32_t*>(&l);
                        }
                        const uint32_t ro = (uint32_t)lane * 128;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t oh = ro + ((uint32_t)(j ^ (lane & 7)) << 4);
                            const uint32_t ol = ro + ((uint32_t)((4 + j) ^ (lane & 7)) << 4);
                            st_shared_v4(hb + oh, h2[4 * j], h2[4 * j + 1], h2[4 * j + 2], h2[4 * j + 3]);
                            st_shared_v4(hb + ol, l2[4 * j], l2[4 * j + 1], l2[4 * j + 2], l2[4 * j + 3]);
                        }
                    } else {
                        // row = lane: box i holds columns 16 i .. 16 i + 15, the 16 hi values
                        // (chunks 0-3) then the 16 lo values (chunks 4-7), chunk j at j ^ (row & 7)
                        uint32_t hv[32], lv[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const float f = i < nv ? __uint_as_float(raw[i]) : 0.f;
                            // round-to-nearest TF32 hi and lo (both exact for the MMA)
                            const uint32_t h = (__float_as_uint(f) + 0x1000u) & 0xffffe000u;
                            hv[i] = h;
                            lv[i] = (__float_as_uint(f - __uint_as_float(h)) + 0x1000u) & 0xffffe000u;
                        }
                        const uint32_t ro = (uint32_t)lane * 128;
#pragma unroll
                        for (int i = 0; i < 2; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const uint32_t bb = hb + (uint32_t)(i * BOX);
                                const uint32_t oh = ro + ((uint32_t)(j ^ (lane & 7)) << 4);
                                const uint32_t ol = ro + ((uint32_t)((4 + j) ^ (lane & 7)) << 4);
                                const int e = 16 * i + 4 * j;
                                st_shared_v4(bb + oh, hv[e], hv[e + 1], hv[e + 2], hv[e + 3]);
                                st_shared_v4(bb + ol, lv[e], lv[e + 1], lv[e + 2], lv[e + 3]);
                            }
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        // logical column x0 + c0 (a multiple of 32) starts at element 2 (x0 + c0)
#pragma unroll
                        for (int i = 0; i < NBOX; ++i)
                            tma_store(&maps.c, hb + (uint32_t)(i * BOX), 2 * (x0 + c0) + i * (128 / (int)sizeof(E)), yh);
                        bulk_commit();
                    }
                    continue;
                }
                // the transpose buffer overlaps the store boxes: no store may still read them
                if (lane == 0) bulk_wait_read<0>();
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 32; ++i) stage[lane * 32 + (i ^ lane)] = __uint_as_float(raw[i]);
                __syncwarp();
                const int c = c0 + lane;                       // this lane's column
                if (g.mode == 0) {
                    // T rows of a partial quarter: 16-byte stores, each lane one group of VEC
                    // columns of one row, RPI rows per store instruction.  T offsets, pitches
                    // and chunk starts are multiples of 32 elements and a tile's columns
                    // (with its zero padding) end on a multiple of 32, so every group is
                    // aligned, lies in one K block, and a chunk that starts inside the tile
                    // lies inside it.
                    constexpr int VEC = 16 / (int)sizeof(E), LPR = 32 / VEC, RPI = 32 / LPR;
                    const int cc = (lane % LPR) * VEC, rsub = lane / LPR;
                    const int64_t trow = t.c_off / t.ldc, tcol = t.c_off % t.ldc;
                    E* hi = reinterpret_cast<E*>(g.C) + (int64_t)b * g.c_batch_elems + trow * 2 * t.ldc +
                            split_col<KB>(tcol + c0 + cc);
                    E* lo = hi + KB;
                    if (c0 < ncols) {
                        for (int r0 = 0; r0 < rows; r0 += RPI) {
                            const int rr = r0 + rsub;
                            if (rr >= rows) break;
                            uint32_t hv[4], lv[4];
                            if constexpr (PREC == HEFF_PREC_BF16X3) {
#pragma unroll
                                for (int p = 0; p < 4; ++p) {
                                    const int col = cc + 2 * p;
                                    const float f0 = c0 + col < t.n ? stage[rr * 32 + (col ^ rr)] : 0.f;
                                    const float f1 = c0 + col + 1 < t.n ? stage[rr * 32 + ((col + 1) ^ rr)] : 0.f;
                                    const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
                                    const __nv_bfloat162 l = __floats2bfloat162_rn(f0 - __low2float(h),
                                                                                   f1 - __high2float(h));
                                    hv[p] = *reinterpret_cast<const uint32_t*>(&h);
                                    lv[p] = *reinterpret_cast<const uint32_t*>(&l);
                                }
                            } else {
#pragma unroll
                                for (int p = 0; p < 4; ++p) {
                                    const int col = cc + p;
                                    const float f = c0 + col < t.n ? stage[rr * 32 + (col ^ rr)] : 0.f;
                                    const uint32_t h = (__float_as_uint(f) + 0x1000u) & 0xffffe000u;
                                    hv[p] = h;
                                    lv[p] = (__float_as_uint(f - __uint_as_float(h)) + 0x1000u) & 0xffffe000u;
                                }
                            }
                            const int64_t o = (int64_t)(q * 32 + rr) * 2 * t.ldc;
                            *reinterpret_cast<uint4*>(hi + o) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                            *reinterpret_cast<uint4*>(lo + o) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                        }
                    }
                } else if (c < t.n) {
                    // chunk 0 stores, later chunks add (same thread, same order: deterministic);
                    // the previous values of 8 rows are loaded before their stores so the
                    // loads overlap (8 at a time keeps the register count of the kernel low)
                    const int64_t o0 = t.c_off + c;
                    if (g.y_f64) {
                        double* y = static_cast<double*>(const_cast<void*>(g.y.p[brel])) + o0;
                        for (int r0 = 0; r0 < rows; r0 += 8) {
                            double old[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                old[u] = (ch && r0 + u < rows) ? y[(int64_t)(q * 32 + r0 + u) * t.ldc] : 0.0;
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (r0 + u < rows)
                                    y[(int64_t)(q * 32 + r0 + u) * t.ldc] =
                                        old[u] + f32_to_f64(stage[(r0 + u) * 32 + (lane ^ (r0 + u))]);
                        }
                    } else {
                        float* y = static_cast<float*>(const_cast<void*>(g.y.p[brel])) + o0;
                        for (int r0 = 0; r0 < rows; r0 += 8) {
                            float old[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                old[u] = (ch && r0 + u < rows) ? y[(int64_t)(q * 32 + r0 + u) * t.ldc] : 0.f;
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (r0 + u < rows)
                                    y[(int64_t)(q * 32 + r0 + u) * t.ldc] =
                                        old[u] + stage[(r0 + u) * 32 + (lane ^ (r0 + u))];
                        }
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if constexpr (CL == 1) mbar_arrive(&tempty[acc]);
                else mbar_arrive_cluster(tempty_pair + (uint32_t)(acc * sizeof(uint64_t)));
            }
            ++ccount;
          }
        }
        if (lane == 0) bulk_wait_all();      // T complete before the CTA (and its boxes) go away
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    // pair: both CTAs are done with the MMAs, their tensor memory and each other's barriers
    if constexpr (CL > 1) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (CL == 1)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN) : "memory");
    }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// A 2-D map over rows of `pitch` elements whose boxes are box_rows x swz bytes (the
// operand arrays: 128-byte boxes, a K block of the hi half and the same of the lo half).
int make_map(CUtensorMap* m, void* base, int prec, uint64_t rows, uint64_t pitch, uint32_t box_rows, int swz) {
    auto fn = encode_fn();
    if (!fn) return fail(HEFF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const bool bf = prec == HEFF_PREC_BF16X3;
    const uint32_t es = bf ? 2 : 4;
    cuuint64_t dims[2] = {pitch, rows};
    cuuint64_t strides[1] = {pitch * es};
    cuuint32_t box[2] = {(cuuint32_t)swz / es, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                               : (swz == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(HEFF_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return HEFF_OK;
}

// Kernel configurations: K blocks of 64 bytes per half (128-byte rows of hi + lo); N tile
// 256 with a 4-stage ring (4 x 48 KB,
// 512 TMEM columns) or N tile 128 with a 6-stage ring (6 x 32 KB, 256 TMEM columns).
#ifndef HEFF_SWZ_TC
#define HEFF_SWZ_TC 64
#endif
constexpr int SWZ_TC = HEFF_SWZ_TC;      // bytes of one K block of one half (hi + lo: a 128-byte row)
static_assert(SWZ_TC / (int)sizeof(__nv_bfloat16) <= KPAD, "a K block must not span two contraction segments");
// 64-byte K spans per accumulation chunk in GEMM 2 (32 bf16 / 16 tf32 elements each): long
// enough that a chunk's MMAs (about 0.5 us per block at N = 256) hide the epilogue's
// read-add-write of the previous chunk, short enough to bound the accumulation bias
// (measured at m = 4096: norm-wise error of y 1.4e-5 -> 5e-6 (bf16x3), 2.6e-5 -> 3e-6 (tf32x3))
#ifndef HEFF_KCHUNK_BF16
#define HEFF_KCHUNK_BF16 128
#endif
#ifndef HEFF_KCHUNK_TF32
#define HEFF_KCHUNK_TF32 32
#endif
constexpr int KCHUNK_BF16 = HEFF_KCHUNK_BF16;
constexpr int KCHUNK_TF32 = HEFF_KCHUNK_TF32;

template <int PREC, int TN_TC, int CL>
struct TcKernel {
    // a 192 KB ring; a CTA of a pair holds half of the B rows (TN_TC / CL)
    static constexpr int STAGES = (192 * 1024) / (2 * (128 + TN_TC / CL) * SWZ_TC);
    using S = Smem<TN_TC / CL, STAGES, SWZ_TC>;
    static constexpr auto kern = tc_gemm_kernel<PREC, TN_TC, STAGES, SWZ_TC, CL>;

    // shared-memory opt-in (once) and, for pairs, the clusters that fit on the device at once
    static int setup(int num_sms, int* clusters) {
        static bool done = false;
        static int ncl = 0;
        if (!done) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::TOTAL);
            if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            ncl = num_sms / CL;
            if (CL > 1) {
                cudaLaunchConfig_t cfg{};
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3((unsigned)(ncl * CL));
                cfg.blockDim = dim3(tc_threads<PREC>());
                cfg.dynamicSmemBytes = S::TOTAL;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0 && n < ncl) ncl = n;
                cudaGetLastError();
            }
            done = true;
        }
        if (clusters) *clusters = ncl;
        return HEFF_OK;
    }
};

template <int PREC, int TN_TC, int CL>
int launch_tc_t(heff_plan* p, int which, void* ws, void* const* y, int nbatch, cudaStream_t st) {
    using K = TcKernel<PREC, TN_TC, CL>;
    using S = typename K::S;
    const int nsm = p->num_sms > 0 ? p->num_sms : 148;
    int max_cl = 0;
    if (int rc = K::setup(nsm, &max_cl)) return rc;
    char* w = static_cast<char*>(ws);
    const int64_t B = p->opts.max_batch;
    int slot = p->tmap_ws[0] == ws ? 0 : (p->tmap_ws[1] == ws ? 1 : -1);
    const bool fresh = slot < 0;
    if (fresh) {
        slot = p->tmap_next;
        p->tmap_next ^= 1;
        p->tmap_ws[slot] = nullptr;        // set once every map of the entry is encoded
    }
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(p->tmaps[slot]);
    if (fresh) {
        // a workspace new to the plan: clear its sticky error flag (caller memory, contents unknown)
        cudaError_t ez = cudaMemsetAsync(w + p->off_flags, 0, sizeof(int), st);
        if (ez != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(ez));
        // Operand rows interleave the hi and lo halves by K block: 2 ld elements per row, boxes
        // of 128-byte rows (a K block of both halves).
        // [0,1] LW (64, 128 rows)  [2,3,4] XT (64, 128, 256)  [5,6] T (64, 128)  [7,8,9] RW (64, 128, 256)
        // [10] T store boxes: 32 rows x 128 bytes
        struct { char* base; int64_t rows, ld; int slot, nbox; } ops[4] = {
            {w + p->off_lw, p->rows_lw, p->ld_x, 0, 2},
            {w + p->off_xt, B * p->rows_x, p->ld_x, 2, 3},
            {w + p->off_t, B * p->rows_t, p->ld_t, 5, 2},
            {w + p->off_rw, p->rows_rw, p->ld_t, 7, 3}};
        for (auto& o : ops)
            for (int k = 0; k < o.nbox; ++k) {
                int rc = make_map(&m[o.slot + k], o.base, PREC, (uint64_t)o.rows, (uint64_t)(2 * o.ld), 64u << k,
                                  2 * SWZ_TC);
                if (rc) return rc;
            }
        int rc = make_map(&m[10], w + p->off_t, PREC, (uint64_t)(B * p->rows_t), (uint64_t)(2 * p->ld_t), 32u,
                          2 * SWZ_TC);
        if (rc) return rc;
        // [11] XT, [12] RW with 32-row boxes (halves of a 64-row B box for CTA pairs)
        if ((rc = make_map(&m[11], w + p->off_xt, PREC, (uint64_t)(B * p->rows_x), (uint64_t)(2 * p->ld_x), 32u,
                           2 * SWZ_TC)))
            return rc;
        if ((rc = make_map(&m[12], w + p->off_rw, PREC, (uint64_t)p->rows_rw, (uint64_t)(2 * p->ld_t), 32u,
                           2 * SWZ_TC)))
            return rc;
        p->tmap_ws[slot] = ws;
    }
    const GemmList& gl = which == 1 ? p->g1 : p->g2;
    if (gl.tasks.empty()) return HEFF_OK;
    TcMaps maps;
    const int sa = which == 1 ? 0 : 5, sb = which == 1 ? 2 : 7;
    maps.a[0] = m[sa]; maps.a[1] = m[sa + 1];
    maps.b[0] = m[sb]; maps.b[1] = m[sb + 1]; maps.b[2] = m[sb + 2];
    maps.c = m[10];
    maps.bq = m[which == 1 ? 11 : 12];
    for (int b0 = 0; b0 < nbatch; b0 += MAXB) {
        const int nb = nbatch - b0 < MAXB ? nbatch - b0 : MAXB;
        TcArgs g{};
        g.tasks = gl.d_tasks;
        g.segs = gl.d_segs;
        g.ntasks = (int)gl.tasks.size();
        g.nbatch = nb;
        g.b0 = b0;
        g.err = reinterpret_cast<int*>(w + p->off_flags);
        if (which == 1) {
            g.a_batch_rows = 0; g.b_batch_rows = p->rows_x;
            g.C = w + p->off_t;
            g.c_batch_elems = p->rows_t * 2 * p->ld_t;
            g.c_batch_rows = (int)p->rows_t;
            g.mode = 0;
        } else {
            g.a_batch_rows = p->rows_t; g.b_batch_rows = 0;
            for (int b = 0; b < nb; ++b) g.y.p[b] = y[b0 + b];
            g.mode = 1;
            g.kchunk = (PREC == HEFF_PREC_TF32X3 ? KCHUNK_TF32 : KCHUNK_BF16) * 64 / SWZ_TC;
            g.y_f64 = p->opts.io_dtype == HEFF_DTYPE_F64;
        }
        const long total = (long)(g.ntasks / CL) * nb;        // entries (tiles, or pairs of tiles)
        long units = max_cl;                                   // CTAs, or clusters of CL CTAs
        if (total < units) units = total;
        {
            cudaLaunchConfig_t cfg{};
            cudaLaunchAttribute at[2];
            int na = 0;
            if (HEFF_PDL) {
                at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                at[na].val.programmaticStreamSerializationAllowed = 1;
                ++na;
            }
            if (CL > 1) {
                at[na].id = cudaLaunchAttributeClusterDimension;
                at[na].val.clusterDim.x = CL; at[na].val.clusterDim.y = 1; at[na].val.clusterDim.z = 1;
                ++na;
            }
            cfg.gridDim = dim3((unsigned)(units * CL));
            cfg.blockDim = dim3(tc_threads<PREC>());
            cfg.dynamicSmemBytes = S::TOTAL;
            cfg.stream = st;
            cfg.attrs = at;
            cfg.numAttrs = na;
            cudaError_t e = cudaLaunchKernelEx(&cfg, K::kern, maps, g);
            if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "tc_gemm launch: %s", cudaGetErrorString(e));
        }
        count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "tc_gemm launch: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

}  // namespace

int launch_tc_gemm(heff_plan* p, int which, void* ws, void* const* y, int nbatch, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GemmList& gl = which == 1 ? p->g1 : p->g2;
    if (gl.tasks.empty()) return HEFF_OK;         // nothing to contract (no tensor maps needed)
    const bool wide = gl.tn == 256, pair = gl.cl == 2;
    if (p->opts.precision == HEFF_PREC_BF16X3)
        return pair ? launch_tc_t<HEFF_PREC_BF16X3, 256, 2>(p, which, ws, y, nbatch, st)
                    : wide ? launch_tc_t<HEFF_PREC_BF16X3, 256, 1>(p, which, ws, y, nbatch, st)
                           : launch_tc_t<HEFF_PREC_BF16X3, 128, 1>(p, which, ws, y, nbatch, st);
    return pair ? launch_tc_t<HEFF_PREC_TF32X3, 256, 2>(p, which, ws, y, nbatch, st)
                : wide ? launch_tc_t<HEFF_PREC_TF32X3, 256, 1>(p, which, ws, y, nbatch, st)
                       : launch_tc_t<HEFF_PREC_TF32X3, 128, 1>(p, which, ws, y, nbatch, st);
}

int tc_pair_clusters(int num_sms, int precision) {
    int n = num_sms / 2;
    if (precision == HEFF_PREC_BF16X3) TcKernel<HEFF_PREC_BF16X3, 256, 2>::setup(num_sms, &n);
    else if (precision == HEFF_PREC_TF32X3) TcKernel<HEFF_PREC_TF32X3, 256, 2>::setup(num_sms, &n);
    return n;
}

}  // namespace heff

// ---------------------------------------------------------------- bounded-wait self-test
namespace heff {
namespace {

// One thread waits, with the GEMM kernels' own bounded wait, for the first phase of an
// mbarrier on which nothing arrives: the wait must give up, raise the abort flag and the
// error flag, and return.
__global__ void mbar_wait_selftest_kernel(int* err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(&bar, 1);
        mbar_wait(&bar, 0, &abort_flag, err);
    }
}

}  // namespace
}  // namespace heff

extern "C" int heff_wait_selftest(const heff_plan* plan, void* workspace, size_t workspace_bytes, int32_t kind,
                                  void* stream, float* ms_out) {
    using namespace heff;
    if (!plan || !workspace || (kind != 0 && kind != 1))
        return fail(HEFF_ERR_INVALID_ARG, "heff_wait_selftest: null plan/workspace or kind not 0/1");
    if (plan->opts.precision == HEFF_PREC_FP64)
        return fail(HEFF_ERR_INVALID_ARG, "heff_wait_selftest: FP64 plans have no device-side waits");
    if (workspace_bytes < plan->off_flags + 256)
        return fail(HEFF_ERR_WORKSPACE, "heff_wait_selftest: workspace smaller than the plan's");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* f = static_cast<char*>(workspace) + plan->off_flags;
    int* err = reinterpret_cast<int*>(f);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    // error flag at byte 0 of the flag area; the barrier's counter and generation at 64, 68
    if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, 128, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) {
        if (kind == 0) mbar_wait_selftest_kernel<<<1, 32, 0, st>>>(err);
        else svd_barrier_selftest(reinterpret_cast<unsigned int*>(f + 64), err, st);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_wait_selftest: %s", cudaGetErrorString(e));
    if (ms_out) *ms_out = ms;
    return HEFF_OK;
}

extern "C" int heff_workspace_status(const heff_plan* plan, void* workspace, size_t workspace_bytes,
                                     void* stream) {
    using namespace heff;
    if (!plan || !workspace) return fail(HEFF_ERR_INVALID_ARG, "heff_workspace_status: null plan/workspace");
    if (plan->opts.precision == HEFF_PREC_FP64) return HEFF_OK;
    if (workspace_bytes < plan->off_flags + 256)
        return fail(HEFF_ERR_WORKSPACE, "heff_workspace_status: workspace smaller than the plan's");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* d = reinterpret_cast<int*>(static_cast<char*>(workspace) + plan->off_flags);
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && flag) e = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (e == cudaSuccess && flag) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "heff_workspace_status: %s", cudaGetErrorString(e));
    if (flag) return fail(HEFF_ERR_TIMEOUT, "a bounded device-side wait expired (flag %d)", flag);
    return HEFF_OK;
}
