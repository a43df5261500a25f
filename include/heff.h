/*
 * heff.h -- C ABI of the GB300 (sm_103a) two-site effective-Hamiltonian library.
 *
 * The operation (Levy, Solomonik, Clark, "Distributed-Memory DMRG via Sparse and
 * Dense Parallel Tensor Contractions", Section II-C equation for K in the two-site
 * form of Section III, tensor diagram Fig. 1d) is the matrix-free product
 *
 *     y[a',t1,t2,b'] = sum L[a',wl,a] W1[wl,t1,s1,wm] W2[wm,t2,s2,wr] R[b',wr,b] x[a,s1,s2,b]
 *
 * with every tensor block-sparse under U(1) (or U(1)^nq) charge conservation
 * (Section II-D).  All buffers are plain pointers: device pointers for tensors and
 * workspaces, host pointers for metadata.  No function throws; every function that
 * can fail returns an int status (HEFF_OK = 0 or a negative HEFF_ERR_* code) and
 * records a message readable with heff_last_error() on the calling thread.
 *
 * Block layout (shared by every tensor argument).  A tensor index is a list of
 * sectors (charge vector, dimension) plus a flow (+1/-1).  A block is a tuple of
 * sector numbers, one per index, and is allowed when sum_k flow_k * charge_k equals
 * the tensor's target charge.  A tensor's buffer holds all allowed blocks in
 * lexicographic order of their sector tuples, each block dense and row-major over
 * its index dimensions, with no padding.  heff_layout_blocks() returns the tuples and
 * element offsets.  Sectors of the bond and physical indices of x must carry distinct
 * charges; MPO channel indices may repeat a charge.
 *
 * Index conventions expected by heff_plan_create (checked, HEFF_ERR_CHARGE_MISMATCH
 * otherwise):
 *   x, y : (a, s1, s2, b)   flows (+1, +1, +1, -1)   target: any
 *   L    : (a', wl, a)      flows (-1, +1, +1)       target 0   (q(a') = q(a) + q(wl))
 *   R    : (b', wr, b)      flows (-1, +1, +1)       target 0   (q(b') = q(b) + q(wr))
 *   W1   : (wl, t1, s1, wm) flows (+1, +1, -1, -1)   target 0
 *   W2   : (wm, t2, s2, wr) flows (+1, +1, -1, -1)   target 0
 * The bra and ket indices of L are the left bond of x, those of R its right bond;
 * MPO and physical indices have sectors of dimension 1 (one sector per channel or
 * per local state).
 *
 * Ownership.  The caller owns every device buffer (tensors, workspaces).  Layout and
 * plan objects are owned by the library (host metadata plus small device tables
 * allocated at plan creation) until the matching *_destroy call.  Compute calls are
 * asynchronous on the given CUDA stream (a cudaStream_t passed as void*; NULL is the
 * legacy default stream) and never synchronise.  A plan may be used by one stream at
 * a time.
 */
#ifndef HEFF_H
#define HEFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define HEFF_OK 0
#define HEFF_ERR_INVALID_ARG -1     /* null pointer, bad size, bad option           */
#define HEFF_ERR_CHARGE_MISMATCH -2 /* layouts inconsistent with the selection rules */
#define HEFF_ERR_UNSUPPORTED -3     /* precision / dtype / device not supported      */
#define HEFF_ERR_OOM -4             /* host or device allocation failed             */
#define HEFF_ERR_CUDA -5            /* a CUDA runtime/driver call failed            */
#define HEFF_ERR_TIMEOUT -6         /* a bounded device-side wait expired            */
#define HEFF_ERR_WORKSPACE -7       /* workspace too small or misaligned (256 B)     */

/* ---- precisions and element types ----------------------------------------- */
#define HEFF_PREC_FP64 0   /* FP64 CUDA-core block GEMMs (reference GPU path)        */
#define HEFF_PREC_BF16X3 1 /* tcgen05 BF16 hi/lo split, 3 products, FP32 accumulate   */
#define HEFF_PREC_TF32X3 2 /* tcgen05 TF32 hi/lo split, 3 products, FP32 accumulate   */

#define HEFF_DTYPE_F64 0   /* tensors in device memory are double                   */
#define HEFF_DTYPE_F32 1   /* tensors in device memory are float (mixed paths only) */

typedef struct heff_index {
    int32_t nsec;           /* number of sectors (>= 1)                          */
    int32_t nq;             /* charge components (1..4), equal for all indices   */
    const int32_t* charges; /* host, [nsec * nq] row-major                        */
    const int32_t* dims;    /* host, [nsec], each >= 1                            */
    int32_t flow;           /* +1 or -1                                          */
} heff_index;

typedef struct heff_layout heff_layout;
typedef struct heff_plan heff_plan;

typedef struct heff_plan_opts {
    int32_t precision;   /* HEFF_PREC_*                                            */
    int32_t io_dtype;    /* HEFF_DTYPE_*; FP64 precision requires HEFF_DTYPE_F64    */
    int32_t max_batch;   /* largest nbatch passed to heff_apply_batched (>= 1)      */
    int32_t shard_count; /* 0 or 1: the whole y; S > 1: one of S row shards        */
    int32_t shard_index; /* 0 .. S-1 (0 when not sharded)                          */
    int32_t reserved[3]; /* zero                                                   */
} heff_plan_opts;

/*
 * heff_qn_block_layout -- enumerate the allowed blocks of a block-sparse tensor
 * (Section II-D: "a list of quantum number label tuples, one dense block per tuple";
 * the label matching of Algorithm 2).  idx: host array of nidx index descriptors
 * (copied); target: host [nq] charge vector (NULL = zero).  *out receives a new
 * layout.  Errors: INVALID_ARG (nidx < 1 or > 16, nsec < 1, dims < 1, nq outside
 * 1..4 or mixed, flow not +-1), OOM.
 */
int heff_qn_block_layout(const heff_index* idx, int32_t nidx, const int32_t* target,
                         heff_layout** out);

/* Number of blocks, total elements and number of indices of a layout. */
int heff_layout_info(const heff_layout* lay, int64_t* nblocks, int64_t* nelem, int32_t* nidx);

/*
 * Copy the block list to host arrays: keys [nblocks * nidx] (sector numbers, int32) and
 * offsets [nblocks] (element offset of each block in the tensor buffer).  Either may be NULL.
 */
int heff_layout_blocks(const heff_layout* lay, int32_t* keys, int64_t* offsets);

void heff_layout_destroy(heff_layout* lay);

/*
 * heff_plan_create -- build the block-triple schedule of y = K x for fixed layouts
 * (the charge-matched block pairs of Algorithm 2 for both contractions, their GEMM
 * task lists, workspace layout and flop counts) and upload the schedule tables to the
 * current CUDA device.  W1_host / W2_host: host copies of the MPO tensors in their
 * layouts (double); an entry equal to 0.0 is dropped from the schedule, so later calls
 * must pass device MPO tensors that are zero there too (heff_plan_check_mpo counts the
 * entries that are not).  Synchronises once (table
 * upload).  Errors: INVALID_ARG, CHARGE_MISMATCH, UNSUPPORTED, OOM, CUDA.
 *
 * Row shards (one apply spread over S GPUs): every y block belongs to the left sector
 * a' of its first index, and its value needs all of x and R but only the L blocks of
 * that a'.  With opts->shard_count = S > 1 the left sectors are assigned to S shards by
 * longest-processing-time over their GEMM flops (deterministic, the same assignment for
 * every shard_index), and the plan computes only the y blocks of the sectors of shard
 * opts->shard_index: the GEMM tasks of those rows and the LW preparation for them (RW,
 * the packed x and the workspace layout stay those of the whole problem).  The other y
 * blocks are not written, so the sum of the S shards' outputs written into zeroed
 * buffers (an all-reduce) is y.  heff_plan_flops reports the shard's share.
 */
int heff_plan_create(const heff_layout* L, const heff_layout* W1, const heff_layout* W2,
                     const heff_layout* R, const heff_layout* x, const double* W1_host,
                     const double* W2_host, const heff_plan_opts* opts, heff_plan** out);

/*
 * heff_plan_check_mpo -- the plan keeps only the MPO entries that were nonzero in the host
 * copies given to heff_plan_create; an apply ignores the others.  This counts the entries
 * of the device tensors W1, W2 (layouts of the plan, element type opts.io_dtype) that are
 * nonzero at those dropped positions into *violations (host): 0 means the tensors fit the
 * plan.  Not called by the apply entries (it would cost a device pass and a host
 * synchronisation per call).  Synchronises `stream`; not for concurrent use on one plan
 * (one device counter).  Errors: INVALID_ARG, UNSUPPORTED (plan without a device), CUDA.
 */
int heff_plan_check_mpo(const heff_plan* plan, const void* W1, const void* W2, void* stream,
                        int64_t* violations);

/* Left sectors a' (indices into x's first index) whose y blocks this plan computes, in
 * increasing order; sectors may be NULL to query the count. */
int heff_plan_shard_sectors(const heff_plan* plan, int32_t* sectors, int32_t* count);

/* Workspace bytes needed by every call on this plan (for nbatch = max_batch). */
int heff_plan_workspace_size(const heff_plan* plan, size_t* bytes);

/*
 * Flop counts of one apply.  canonical: sum of 2*M*N*K over the block products of the
 * two-contraction list algorithm (L-block x x-block, then the MPO-mixed result x
 * R-block^T), the definition the FP64 oracle counts; executed: sum of 2*M*N*K over the
 * GEMM tiles this plan issues (valid rows and columns, padded K), per product pass.
 */
int heff_plan_flops(const heff_plan* plan, double* canonical, double* executed);

/*
 * Plan statistics for diagnostics, stats[24]: [0] charge sectors, [1] LW row groups,
 * [2] RW row groups, [3] GEMM-1 tasks, [4] GEMM-2 tasks, [5] pack tiles, [6] mix tiles,
 * [7] mix terms, [8] XT rows, [9] XT/LW pitch, [10] LW rows, [11] T rows, [12] T/RW
 * pitch, [13] RW rows, [14] tile M, [15] GEMM-1 tile variant (HEFF_TILE_*), [16] canonical flops of the first
 * contraction, [17] of the second, [18] GEMM-1 flops over valid rows, columns and
 * unpadded K, [19] the same for GEMM 2, [20] GEMM-1 issued flops (padded K), [21] GEMM 2,
 * [22] GEMM-2 tile variant.
 */
int heff_plan_stats(const heff_plan* plan, int64_t* stats /* [24] */);

/*
 * Copy one schedule table of the plan into host memory dst (NULL: query only) and its
 * size in bytes into *bytes.  table: 0 pack tiles, 1 mix tiles, 2 mix terms, 3 GEMM-1
 * tasks, 4 GEMM-1 segments, 5 GEMM-2 tasks, 6 GEMM-2 segments (record formats in
 * csrc/internal.h).  For inspection and host-side testing of the schedule.  A plan
 * created on a machine without a CUDA device is host-only: this call and the query
 * calls work, compute calls return HEFF_ERR_UNSUPPORTED.
 */
int heff_plan_export(const heff_plan* plan, int32_t table, void* dst, int64_t* bytes);

void heff_plan_destroy(heff_plan* plan);

/*
 * heff_apply -- y = K x (Section II-C / Fig. 1d, two-site).  L, W1, W2, R, x: device
 * buffers in their layouts, element type opts.io_dtype; y: device buffer in x's layout
 * (overwritten, must not alias x).  workspace: device, >= heff_plan_workspace_size
 * bytes, 256-byte aligned, not shared with another call in flight.  stream: cudaStream_t.
 * Runs heff_prepare then heff_apply_prepared.  When x's layout has no allowed block (an
 * empty two-site space) y has no elements: this and the other apply entries return HEFF_OK
 * at once (x, y may then be NULL); the eigensolvers reject such a plan (INVALID_ARG).
 * Errors: INVALID_ARG, WORKSPACE, CUDA.
 */
int heff_apply(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
               const void* x, void* y, void* workspace, size_t workspace_bytes, void* stream);

/*
 * heff_prepare -- fold the MPO tensors into the environments inside the workspace
 * (LW = L.W1 summed over wl, RW = W2.R summed over wr), so that repeated applies with the
 * same L, W1, W2, R (an eigensolver's Krylov steps) skip that work.  The prepared state
 * lives in the workspace and is valid until the workspace is reused by another plan.
 */
int heff_prepare(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                 void* workspace, size_t workspace_bytes, void* stream);

/* y = K x using operators prepared in the workspace by heff_prepare. */
int heff_apply_prepared(heff_plan* plan, const void* x, void* y, void* workspace,
                        size_t workspace_bytes, void* stream);

/*
 * heff_apply_host -- heff_apply on tensors in host memory: the five inputs are copied into
 * `staging` (device, >= heff_apply_host_staging_size bytes, 256-byte aligned; laid out as
 * L, W1, W2, R, x, y), the apply runs there, and y is copied back, all asynchronously on
 * `stream` (pinned host memory lets the copies overlap work on other streams; pageable
 * memory makes them synchronous).  Host buffers must stay valid until the stream reaches
 * the end of the call.  Errors: as heff_apply, WORKSPACE for a small staging buffer.
 */
int heff_apply_host_staging_size(const heff_plan* plan, size_t* bytes);
int heff_apply_host(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                    const void* x, void* y, void* staging, size_t staging_bytes, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * heff_apply_batched -- y_b = K x_b for b < nbatch (<= max_batch) vectors sharing L, W1,
 * W2, R: one preparation and one launch of each GEMM over all vectors.  x, y: HOST arrays
 * of nbatch device pointers.  Errors as heff_apply.
 */
int heff_apply_batched(heff_plan* plan, const void* L, const void* W1, const void* W2,
                       const void* R, const void* const* x, void* const* y, int32_t nbatch,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * heff_lanczos -- lowest eigenpair of H_eff by n_iter Lanczos steps (the eigensolver of
 * the two-site DMRG step, Section II-C and III; the fixed-iteration alternative to the
 * Davidson routine of Algorithm 1), all in FP64 on the device except the matvecs, which
 * run in the plan's precision.  Each step applies the three-term recurrence, then one
 * classical Gram-Schmidt pass against the whole basis (full reorthogonalisation), and a
 * second pass when the first removed more than half of the vector's squared norm (the
 * Daniel-Gragg-Kaufman-Stewart criterion); the tridiagonal eigenproblem is solved on the
 * device (bisection on the Sturm count + inverse iteration).  The plan must use
 * HEFF_DTYPE_F64 tensors.
 *   x0      device, nelem(x) doubles: start vector (need not be normalised, must be nonzero)
 *   x_out   device, nelem(x) doubles: normalised Ritz vector of the lowest Ritz value
 *   result  device, 3 + 2 * (n_iter + 1) doubles: [0] lowest Ritz value theta,
 *           [1] Lanczos residual estimate |beta_last * s_last|, [2] Krylov dimension used,
 *           then alpha[n_iter + 1], beta[n_iter + 1]
 *   apply_ws  the plan's workspace (heff_plan_workspace_size), overwritten
 *   lz_ws     >= heff_lanczos_workspace_size bytes, 256-byte aligned, overwritten
 * n_iter 1..126.  If the Krylov space becomes invariant (beta < 1e-13 |alpha|) the
 * remaining steps are skipped on the device.  Asynchronous; never synchronises.
 */
int heff_lanczos_workspace_size(const heff_plan* plan, int32_t n_iter, size_t* bytes);
int heff_lanczos(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                 const double* x0, int32_t n_iter, double* x_out, double* result, void* apply_ws,
                 size_t apply_ws_bytes, void* lz_ws, size_t lz_ws_bytes, void* stream);

/*
 * heff_ground_state -- lowest eigenpair of H_eff to a residual tolerance, with the energy
 * evaluated in FP64 (the eigensolver of the two-site DMRG step, Section II-C and III, run
 * to convergence; the FP64 refinement that lets split-precision matvecs give FP64-accurate
 * energies).  Restarted Lanczos: each cycle runs n_iter steps of heff_lanczos from the
 * previous cycle's Ritz vector (the first from x0), with matvecs in `plan`'s precision, until
 * the cycle's residual estimate |beta_last s_last| / |theta| is <= tol or max_cycles cycles
 * have run.  The energy is then the FP64 Rayleigh quotient <x|K|x> of the normalised Ritz
 * vector x, computed with one apply of `plan64` (an HEFF_PREC_FP64 plan of the same layouts;
 * NULL: `plan` itself when it is an FP64 plan, otherwise no FP64 step), together with the
 * FP64 residual ||K x - E x|| / |E|.  L, W1, W2, R: device doubles (HEFF_DTYPE_F64 plans).
 *   x0      device, nelem(x) doubles, nonzero start vector
 *   x_out   device, nelem(x) doubles: the normalised Ritz vector (may alias x0)
 *   result  HOST, 6 doubles: [0] energy (FP64 Rayleigh quotient, or the last Ritz value
 *           without an FP64 plan), [1] last Ritz value (plan's precision), [2] last residual
 *           estimate / |theta|, [3] cycles run, [4] Lanczos steps (matvecs) run, [5] FP64
 *           residual ||K x - E x|| / |E| (-1 without an FP64 plan)
 *   apply_ws / apply_ws64  the workspaces of plan / plan64 (apply_ws64 ignored when plan64
 *           is NULL)
 *   gs_ws   >= heff_ground_state_workspace_size bytes, 256-byte aligned, overwritten
 * n_iter 1..126, max_cycles >= 1, tol >= 0.  Synchronises `stream` once per cycle (the
 * residual test on the host) and once after the FP64 step.  Errors: INVALID_ARG,
 * UNSUPPORTED (plan without HEFF_DTYPE_F64 tensors), WORKSPACE, CUDA.
 */
int heff_ground_state_workspace_size(const heff_plan* plan, int32_t n_iter, size_t* bytes);
int heff_ground_state(heff_plan* plan, heff_plan* plan64, const void* L, const void* W1, const void* W2,
                      const void* R, const double* x0, int32_t n_iter, int32_t max_cycles, double tol,
                      double* x_out, double* result, void* apply_ws, size_t apply_ws_bytes, void* apply_ws64,
                      size_t apply_ws64_bytes, void* gs_ws, size_t gs_ws_bytes, void* stream);

/*
 * heff_davidson -- lowest eigenpair of H_eff by the Davidson routine of Algorithm 1
 * (no preconditioner; randomisation when re-orthogonalisation fails), all in FP64 on the
 * device except the matvecs (the plan's precision; HEFF_DTYPE_F64 tensors).  Per step i:
 * m_ij = (A v_j)^T v_i for j <= i; the lowest eigenpair (lambda, s) of the leading
 * (i+1) x (i+1) block of M (one-thread Jacobi); x = sum s_j v_j, q = sum s_j A v_j -
 * lambda x; stop when ||q|| < tol max(1, |lambda|) or max_vecs vectors are in use; else q
 * is orthogonalised against v_0..v_i (two classical Gram-Schmidt passes), replaced by
 * `rnd` if less than 1e-12 of it survives (then orthogonalised again), normalised into
 * v_{i+1}.  The paper runs it with a subspace of 2 inside the sweeps (max_vecs = 2).
 *   x0      device, nelem(x) doubles, nonzero start vector
 *   rnd     device, nelem(x) doubles, the random vector of the randomisation step
 *   x_out   device, nelem(x) doubles: normalised x
 *   result  device, 3 doubles: lambda, ||q||, vectors used
 *   dav_ws  >= heff_davidson_workspace_size bytes, 256-byte aligned
 * max_vecs 1..64, tol >= 0.  Asynchronous; never synchronises.
 */
int heff_davidson_workspace_size(const heff_plan* plan, int32_t max_vecs, size_t* bytes);
int heff_davidson(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                  const double* x0, const double* rnd, int32_t max_vecs, double tol, double* x_out,
                  double* result, void* apply_ws, size_t apply_ws_bytes, void* dav_ws, size_t dav_ws_bytes,
                  void* stream);

/*
 * Environment extension (Section II-C: the left environment A and right environment B
 * are grown one site at a time as the sweep moves).  FP64 block products on the GPU.
 *   side 0 (left):  Lnew[c,v,d] = sum A[a,t,c] L[a,w,b] W[w,t,s,v] A[b,s,d]
 *   side 1 (right): Rnew[c,w,d] = sum B[c,t,a] R[a,v,b] W[w,t,s,v] B[d,s,b]
 * Layouts: site (a, s, b) flows (+1, +1, -1); W (w, t, s, v) flows (+1, +1, -1, -1);
 * env_old / env_new (bond, channel, bond) flows (-1, +1, +1) on the site's left / right
 * bond (side 0) or right / left bond (side 1), channels of W's first / last index.
 * W_host: host copy of W in its layout; zero entries are dropped from the schedule.
 * heff_env_update: all tensors are device double buffers; env_new is overwritten;
 * workspace >= heff_env_workspace_size bytes, 256-byte aligned.  Asynchronous.
 */
typedef struct heff_env_plan heff_env_plan;
int heff_env_plan_create(const heff_layout* env_old, const heff_layout* site, const heff_layout* W,
                         const heff_layout* env_new, const double* W_host, int32_t side,
                         heff_env_plan** out);
int heff_env_workspace_size(const heff_env_plan* plan, size_t* bytes);
int heff_env_flops(const heff_env_plan* plan, double* flops);
int heff_env_update(heff_env_plan* plan, const double* env_old, const double* site, const double* W,
                    double* env_new, void* workspace, size_t workspace_bytes, void* stream);
void heff_env_plan_destroy(heff_env_plan* plan);

/*
 * Arithmetic of the environment update's block products.  HEFF_PREC_FP64 (the default):
 * FP64 on the CUDA cores.  HEFF_PREC_BF16X3: on the tensor cores, each operand element split
 * into bf16 hi + lo and three products per K block, FP32 accumulation (about 1e-5 relative
 * per product); the tensors stay FP64 buffers (the update converts env_old and the site
 * tensor to FP32 copies in the workspace, whose size covers both precisions) and the call
 * sequence is unchanged.  Errors:
 * INVALID_ARG, UNSUPPORTED (another precision), CUDA.
 */
int heff_env_plan_set_precision(heff_env_plan* plan, int32_t precision);

/*
 * Read and clear the sticky error flag of an environment-update workspace: HEFF_ERR_TIMEOUT
 * when a bounded wait of a tensor-core product expired in the last update (its output is
 * then incomplete; the context stays usable), else HEFF_OK (always for FP64 plans).
 * Synchronises `stream`.  Errors: INVALID_ARG, WORKSPACE, CUDA.
 */
int heff_env_status(const heff_env_plan* plan, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Two-site tensor of the MPS (Fig. 1d; the starting vector of a bond's eigensolve in the
 * two-site sweep of Section II-C): x[a, s1, s2, b] = sum_c A[a, s1, c] B[c, s2, b].
 * A and B have flows (+1, +1, -1) and share the bond c; x is the (a, s1, s2, b) layout of
 * the bond's problem (flows +1, +1, +1, -1).  heff_two_site_apply writes every x block
 * (zeros where no (A, B) block pair matches); device doubles, asynchronous on `stream`.
 * Errors: INVALID_ARG, CHARGE_MISMATCH (indices disagree), UNSUPPORTED (plan made
 * without a device), CUDA.
 */
typedef struct heff_two_site heff_two_site;
int heff_two_site_create(const heff_layout* A, const heff_layout* B, const heff_layout* x,
                         heff_two_site** out);
int heff_two_site_apply(heff_two_site* plan, const double* A, const double* B, double* x, void* stream);
void heff_two_site_destroy(heff_two_site* plan);

/*
 * Gradients of the Rayleigh quotient rho = <x|K|x> / <x|x> of the effective Hamiltonian
 * K (Section II-C): rho is linear in L, R, W1 and W2, so each gradient is the closed-form
 * contraction of the bra x, the ket x and the other three operators; d rho/dx =
 * 2 (K x - rho x) / <x|x>; rho is undefined at x = 0, where every result is NaN (the
 * call does not synchronise to test for it).  heff_grad_plan_create builds the block-product schedule for
 * the five layouts (host MPO copies drop exactly-zero entries from the W1.W2 pattern; the
 * W gradients are computed for every allowed entry).  heff_backward computes y = K x with
 * `plan` (any precision; HEFF_DTYPE_F64 tensors) and the rest in FP64:
 *   rho: device, 1 double; dx, dL, dR, dW1, dW2: device doubles in the layouts of x, L,
 *   R, W1, W2 (overwritten).  apply_ws: plan workspace; grad_ws >= heff_grad_workspace_size
 *   bytes, 256-byte aligned.  The gradient with respect to a coupling J that W1, W2
 *   depend on is sum dW1 * dW1/dJ + sum dW2 * dW2/dJ (L and R held fixed).
 * Intermediates: U = x.R and T1 = L.x (each about k d^2 times the size of x).  ws_limit = 0
 * keeps them whole; ws_limit > 0 bounds the gradient workspace: the left sectors a' of x
 * are split into chunks of consecutive sectors, and each chunk's U and T1 blocks are
 * formed, consumed (dL of those sectors completely; dR and the W gradients as partial sums
 * added in chunk order) and overwritten by the next chunk, so nothing is computed twice.
 * A limit below the largest single sector's need (plus the small fixed part) fails with
 * HEFF_ERR_WORKSPACE naming the minimum.  heff_grad_chunks reports the chunk count.
 */
typedef struct heff_grad_plan heff_grad_plan;
int heff_grad_plan_create(const heff_layout* L, const heff_layout* W1, const heff_layout* W2,
                          const heff_layout* R, const heff_layout* x, const double* W1_host,
                          const double* W2_host, size_t ws_limit, heff_grad_plan** out);
int heff_grad_chunks(const heff_grad_plan* g, int32_t* nchunks);
int heff_grad_workspace_size(const heff_grad_plan* g, size_t* bytes);
int heff_backward(heff_grad_plan* g, heff_plan* plan, const double* L, const double* W1,
                  const double* W2, const double* R, const double* x, double* rho, double* dx,
                  double* dL, double* dR, double* dW1, double* dW2, void* apply_ws,
                  size_t apply_ws_bytes, void* grad_ws, size_t grad_ws_bytes, void* stream);
void heff_grad_plan_destroy(heff_grad_plan* g);

/*
 * Arithmetic of the gradients' block products (U, T1, dL, dR): HEFF_PREC_FP64 (the default,
 * CUDA cores) or HEFF_PREC_BF16X3 (tensor cores, bf16 hi/lo split, FP32-accumulated; about
 * 1e-5 relative).  The scalars, dx and the W gradients' reductions stay FP64; buffers stay
 * FP64.  With HEFF_PREC_BF16X3 the workspace also holds FP32 copies of x, L and R (the
 * products' operands, converted once per call) and the intermediates in FP32, so
 * heff_grad_workspace_size reports a larger size after the switch (a workspace limit given
 * at plan creation bounds the FP64 layout).  heff_grad_status reads and clears the
 * gradient workspace's sticky error flag
 * (HEFF_ERR_TIMEOUT when a bounded wait of a tensor-core product expired; synchronises).
 * Errors: INVALID_ARG, UNSUPPORTED (another precision), WORKSPACE, CUDA.
 */
int heff_grad_plan_set_precision(heff_grad_plan* g, int32_t precision);
int heff_grad_status(const heff_grad_plan* g, void* grad_ws, size_t grad_ws_bytes, void* stream);

/*
 * Block SVD split of the two-site tensor with truncation (Section IV: the tensor is
 * wrapped into the matrix (a s1) x (s2 b), one dense block per charge Q = q(a) + q(s1);
 * Fig. 1e: split into two order-3 tensors, singular values absorbed in the sweep
 * direction; Section II-C: singular values below a cutoff are removed).  FP64 result on
 * the GPU: one-sided Jacobi per block (rounds of disjoint column-pair rotations), started
 * by FP32 sweeps on a copy, whose rotations are made orthonormal in FP64 (Newton-Schulz)
 * and applied in FP64 before FP64 sweeps finish; the output shapes depend on the
 * truncation, so the call sequence is:
 *   heff_svd_create(x_layout)            host: charge blocks, workspace size
 *   heff_svd_compute(x_dev, ws)           decomposes every block; SYNCHRONISES (per-sweep
 *                                         convergence check, singular values to the host)
 *   heff_svd_truncate(m_max, cutoff, ...) host: on x/||x||, drop s < cutoff, keep at most
 *                                         m_max largest (ties within 1e-12 s_max ordered by
 *                                         (|Q|, Q, rank)); returns the new bond (charges
 *                                         Q in increasing order, dims = kept counts), the
 *                                         discarded weight sum s^2/||x||^2 and ||x||
 *   heff_svd_write(A_layout, B_layout)    writes A[a, s1, c] (flows +1, +1, -1) and
 *                                         B[c, s2, b] (flows +1, +1, -1) on the new bond;
 *                                         absorb_right = 1: B carries S (A is an isometry),
 *                                         0: A carries S.  Synchronises.
 * charges_out: host [nsec * nq] (may be NULL); dims_out: host [nsec] (may be NULL; the
 * caller can first query nsec with both NULL... pass arrays of at least the number of
 * charge blocks of x).
 */
typedef struct heff_svd heff_svd;
int heff_svd_create(const heff_layout* x, heff_svd** out);
int heff_svd_workspace_size(const heff_svd* s, size_t* bytes);
int heff_svd_compute(heff_svd* s, const double* x, void* workspace, size_t workspace_bytes, void* stream,
                     int32_t* sweeps_out);
/* Sweeps of the last heff_svd_compute: FP32 preconditioning sweeps and FP64 sweeps (the
 * latter is heff_svd_compute's sweeps_out); either pointer may be NULL. */
int heff_svd_info(const heff_svd* s, int32_t* fp32_sweeps, int32_t* fp64_sweeps);
int heff_svd_truncate(heff_svd* s, int32_t m_max, double cutoff, int32_t* nsec_out, int32_t* charges_out,
                      int32_t* dims_out, double* discarded_weight, double* norm);
int heff_svd_singular_values(const heff_svd* s, double* out);
int heff_svd_write(heff_svd* s, const heff_layout* A_layout, const heff_layout* B_layout, double* A,
                   double* B, int32_t absorb_right, void* workspace, size_t workspace_bytes, void* stream);
void heff_svd_destroy(heff_svd* s);

/*
 * heff_apply_noalloc -- heff_apply without a caller-provided workspace and without any
 * device allocation.  The paper has no counterpart of it: it exists because some callers
 * cannot call cudaMalloc, for example code running under another framework's memory
 * manager that has already reserved the device memory it may use, or code on a
 * latency-critical path where cudaMalloc's implicit device synchronisation is not
 * acceptable.  The workspace is a fixed array of HEFF_NOALLOC_WORKSPACE_BYTES compiled
 * into the library; every GPU that loads the library holds one copy until the process
 * exits.  Plans whose heff_plan_workspace_size exceeds that size are rejected with
 * HEFF_ERR_WORKSPACE (for example the m = 1024 spin problem in BF16x3 fits, m = 4096
 * does not).  The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's contents, so
 * calls that overlap on the GPU (on different streams or from different threads) race
 * on it and must be serialised by the caller.  Arguments and errors otherwise as
 * heff_apply; the plan must belong to the current device.
 */
#define HEFF_NOALLOC_WORKSPACE_BYTES (128u << 20)
int heff_apply_noalloc(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                       const void* x, void* y, void* stream);

/*
 * heff_apply_noalloc_status -- heff_workspace_status for the built-in workspace of the
 * current device: reads and clears its sticky error flag (HEFF_ERR_TIMEOUT when a bounded
 * device-side wait expired in the last heff_apply_noalloc, whose output is then incomplete).
 * heff_apply_noalloc clears the flag when it starts, so read it after a call whose result
 * matters.  Allocates nothing; synchronises `stream`.  Errors: INVALID_ARG, CUDA.
 */
int heff_apply_noalloc_status(const heff_plan* plan, void* stream);

/*
 * Tensor-core tile variants of a GEMM (the plan builds all three task lists):
 *   HEFF_TILE_256       one CTA per 128 x 256 output tile (the default)
 *   HEFF_TILE_128       one CTA per 128 x 128 output tile
 *   HEFF_TILE_PAIR_256  128 x 256 tiles in pairs that share their B rows and K segments, run
 *                       by the two CTAs of a cluster as one M = 256 tile (tcgen05 pair MMAs,
 *                       cta_group::2): each CTA loads its own 128 A rows and its own half of
 *                       the B rows into its own shared memory, and both CTAs' loads complete
 *                       on the even CTA's barrier, so B is read once per pair (no multicast
 *                       load is issued)
 * Results are bitwise identical across variants (a tile's K order does not depend on them).
 */
#define HEFF_TILE_256 256
#define HEFF_TILE_128 128
#define HEFF_TILE_PAIR_256 512
#define HEFF_TILE_VARIANTS 3

/*
 * heff_plan_autotune -- choose the tile variant of each of the two tensor-core GEMMs by
 * timing every variant on the given inputs (which must be valid tensors for the plan; y and
 * the workspace are overwritten) and keep the fastest in the plan (each candidate: one
 * warm-up launch, then the median of five timed launches).  tn_out (host, may be NULL)
 * receives the chosen variants {GEMM 1, GEMM 2}; ms_out (host, may be NULL, 2 x
 * HEFF_TILE_VARIANTS floats) the median times {GEMM 1: 256, 128, pairs; GEMM 2: 256, 128,
 * pairs} in ms (0 where a variant has no task list).  No-op for the FP64 precision.
 * Synchronises (event timing); call it before capturing applies into a CUDA graph.
 */
int heff_plan_autotune(heff_plan* plan, const void* L, const void* W1, const void* W2, const void* R,
                       const void* x, void* y, void* workspace, size_t workspace_bytes, void* stream,
                       int32_t* tn_out, float* ms_out);

/*
 * Select the tile variant (HEFF_TILE_256, HEFF_TILE_128 or HEFF_TILE_PAIR_256) of GEMM 1 and
 * GEMM 2 without measuring (0 keeps the current choice); heff_plan_autotune picks by timing.
 * Results do not depend on the choice.  Errors: INVALID_ARG (variant not built for this
 * plan, or an FP64 plan).
 */
int heff_plan_select_tiles(heff_plan* plan, int32_t tn1, int32_t tn2);

/*
 * Phase timers (the time breakdown of Section VI / Fig. 7, on the GPU): when enabled,
 * every compute call records CUDA events on its stream around its phases.
 * heff_plan_timings waits for the last call's final event and writes the milliseconds
 * of ms[4] = {prepare, pack, GEMM 1, GEMM 2} (prepare is 0 when the call skipped it).
 */
int heff_plan_set_timing(heff_plan* plan, int32_t enable);
int heff_plan_timings(heff_plan* plan, float* ms);

/*
 * heff_workspace_status -- read and clear the sticky device error flag of an apply workspace.
 * The tensor-core GEMM kernels set it when one of their bounded waits expires (about 1.5 s
 * on an mbarrier that does not complete); that launch then stops issuing work, frees its
 * tensor memory and returns, so its outputs are incomplete but the context stays usable.
 * A GEMM launch clears the flag when the workspace is not one of the last two the plan
 * used.  Synchronises `stream`.  Returns HEFF_ERR_TIMEOUT if the flag was set (and clears
 * it), else HEFF_OK; always HEFF_OK for FP64 plans, whose kernels do not wait.
 * workspace: device, at least heff_plan_workspace_size bytes.  Errors: INVALID_ARG,
 * WORKSPACE (too small), CUDA.
 */
int heff_workspace_status(const heff_plan* plan, void* workspace, size_t workspace_bytes, void* stream);

/*
 * heff_wait_selftest -- check that a device-side bounded wait gives up instead of hanging.
 * Launches one single-block kernel whose wait nothing completes: kind 0 waits with the
 * tensor-core GEMM kernels' mbarrier wait (gives up after 3 * 2^30 clock cycles, about
 * 1.5 s), kind 1 at the SVD sweeps' grid barrier set up for two blocks (2^31 cycles, about
 * 1 s).  On expiry the kernel sets the workspace's sticky error flag, as an expired wait in
 * a GEMM launch does, and returns; read it with heff_workspace_status.  workspace: an apply
 * workspace of `plan` (device); ms_out (host, may be NULL) receives the kernel's duration.
 * Synchronises `stream`.  Errors: INVALID_ARG (null pointer, kind not 0 or 1, FP64 plan),
 * WORKSPACE, CUDA.
 */
int heff_wait_selftest(const heff_plan* plan, void* workspace, size_t workspace_bytes, int32_t kind,
                       void* stream, float* ms_out);

/* Message of the last failed call on this thread ("" if none). */
const char* heff_last_error(void);

/* Number of kernels this library has launched in the process (all threads). */
int64_t heff_launch_count(void);

/* Library version string. */
const char* heff_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HEFF_H */
