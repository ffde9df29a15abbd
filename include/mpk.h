/*
 * mpk.h -- C ABI of the GB300 level-blocked matrix power kernel library (libmpk.so).
 *
 * The library computes the matrix power kernel of "Cache Blocking of Distributed-Memory
 * Parallel Matrix Power Kernels" (Lacey, Alappat, Lange, Hager, Fehske, Wellein):
 *     Y[k] = A^k X,   k = 0..p          (Sec. 3, "MPK computes all vectors y_p = A^p x")
 * for a square CSR matrix A, by level blocking: the rows are split into BFS levels of the
 * graph of A (Sec. 3, level definition and Fig. 1), consecutive levels are grouped so that
 * p+1 groups fit a cache budget (Sec. 3 reuse window, Sec. 6 parameter C), and the
 * (group, power) cells of the Lp diagram are executed in its diagonal order (Fig. 2).
 * On one GPU the paper's inter-process halo exchange (Alg. 2) is replaced by per-chunk
 * completion flags in device memory.  A Chebyshev filter built on the same kernel
 * implements the recurrence of Sec. 7.
 *
 * Conventions for every entry point
 *  - All pointers named *_dev / documented as "device" are CUDA device pointers owned by
 *    the caller unless stated otherwise; host pointers are marked "host".
 *  - Dense blocks are row-major n x m ("nrhs" = m): the m values of one row are contiguous.
 *    A power sequence Y is (p+1) x n x m doubles with Y[0] = X.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work
 *    is enqueued asynchronously on it; device-side failures (a bounded wait that expired)
 *    are reported by mpk_sync_status().  Preprocessing calls (mpk_build_levels, mpk_plan)
 *    synchronise the stream before returning.
 *  - Every function returns an mpk_status and never throws; mpk_last_error() gives a
 *    thread-local message for the last failure on the calling thread.
 *  - Indices are int32: n, nnz < 2^31.  Floating point is IEEE binary64; each row sum is
 *    evaluated in the row's stored order with one fused multiply-add per entry (in binary32
 *    for plans built with opts.accum = MPK_F32, over binary64 vectors).
 */
#ifndef MPK_H
#define MPK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPK_OK = 0,
    MPK_ERR_INVALID = 1,     /* bad argument or malformed CSR (details in mpk_last_error) */
    MPK_ERR_TOO_LARGE = 2,   /* a size exceeds int32 indexing or the library's limits */
    MPK_ERR_OOM = 3,         /* a device allocation failed */
    MPK_ERR_TIMEOUT = 4,     /* a bounded device wait expired; results of that call are void */
    MPK_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    MPK_ERR_BUDGET = 6,      /* the plan would exceed mpk_plan_opts.mem_budget */
    MPK_ERR_UNSUPPORTED = 7  /* valid request the library does not implement (e.g. nrhs 3)  */
} mpk_status;

typedef enum { MPK_F64 = 0, MPK_F32 = 1, MPK_BF16 = 2 } mpk_dtype;

typedef enum {
    MPK_ORDER_ORIGINAL = 0,  /* X and Y use A's row numbering */
    MPK_ORDER_PLAN = 1       /* X and Y use the plan's (BFS-permuted) row numbering */
} mpk_order;

typedef void *mpk_stream;

/* A square CSR matrix in device memory, owned by the caller.  row_ptr has n+1 entries
 * (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz); col has nnz entries in [0, n); val
 * has nnz entries of val_type.  Column order inside a row is free and duplicates are
 * allowed: entries are summed in stored order.  is_symmetric = 1 declares that the
 * sparsity pattern is symmetric, which skips the A + A^T step of the level builder.
 * Precision: a plan stores the values in val_type (8, 4 or 2 bytes an entry) and every
 * kernel widens each value to float64 exactly before its FMA; vectors and accumulation are
 * float64.  The results are those of the float64 computation on the widened values, bit for
 * bit (unless the plan asks for binary32 row sums, opts.accum); values exactly
 * representable in the narrow type (e.g. the {6, -1} or {26, -1} stencil coefficients in
 * bfloat16) therefore give the float64 results unchanged.  In the
 * narrow types every value must be zero or a normal number: mpk_plan fails with
 * MPK_ERR_UNSUPPORTED on a subnormal, infinite or NaN value. */
typedef struct {
    int32_t n;
    int32_t nnz;
    const int32_t *row_ptr;
    const int32_t *col;
    const void *val;
    int32_t val_type;    /* mpk_dtype of val: MPK_F64, MPK_F32 or MPK_BF16 (bfloat16 bits)  */
    int32_t is_symmetric;
} mpk_csr;

typedef struct mpk_levels_s mpk_levels;   /* opaque, library-owned */
typedef struct mpk_plan_s mpk_plan_t;     /* opaque, library-owned */

/* ---------------------------------------------------------------------------------------
 * Levels.  Sec. 3: BFS from a root over the graph of A (pattern of A + A^T, self-loops
 * ignored, the endnote on non-symmetric matrices); L(i+1) holds the untouched neighbours
 * of L(i).  Inside a level vertices are ordered by ascending original index (the order of
 * Fig. 1(c)).  When the search runs dry with vertices left (a disconnected graph) the
 * smallest untouched vertex opens the next level.  perm maps new -> old, iperm old -> new.
 * The result is unique for a given (A, root).  Synchronises `stream`.
 * ------------------------------------------------------------------------------------- */
mpk_status mpk_build_levels(const mpk_csr *A, int32_t root, mpk_stream stream, mpk_levels **out);

/* Levels with a set of roots (host array, ascending, distinct) as level 0: level k is the
 * set of vertices at distance k from the set.  Rooted at a partition's halo rows, level k is
 * the set I_k of DLB-MPK (Sec. 5): the rows k steps from the boundary. */
mpk_status mpk_build_levels_from(const mpk_csr *A, const int32_t *roots, int32_t nroots, mpk_stream stream,
                                 mpk_levels **out);

/* Views into a levels object (device pointers valid until mpk_levels_destroy):
 * level_ptr[num_levels+1] (row offsets of levels in the new order), perm[n], iperm[n],
 * level_of[n].  Any output pointer may be NULL. */
mpk_status mpk_levels_get(const mpk_levels *L, int32_t *n, int32_t *num_levels,
                          const int32_t **level_ptr_dev, const int32_t **perm_dev,
                          const int32_t **iperm_dev, const int32_t **level_of_dev);

/* Frees a levels object (NULL: no-op).  Plans built from it keep their own copies of the
 * permutation and stay valid. */
void mpk_levels_destroy(mpk_levels *L);

/* ---------------------------------------------------------------------------------------
 * Plans.  A plan owns a permuted copy of A (P A P^T, entries kept in stored order, in a
 * sliced layout of 32-row slices), the level groups, the work-unit tables of the
 * level-blocked schedule for every p <= p_max, per-chunk completion flags and a vector
 * workspace.
 *
 * Groups follow the greedy rule of the paper's cache blocking (Sec. 3 reuse window, Sec. 6
 * parameter C): walk the levels in order and add a level to the current group while the
 * group's bytes stay <= floor(cache_bytes / window); a level costs
 * (val_bytes + 4) * nnz + 4 * rows + 16 * nrhs * rows bytes; a level over the budget is a
 * group of its own.  The GPU executes the Lp-diagram cells (group g, power k) along lines
 * g + 3k = const (the paper walks the diagonals g + k = const, whose cells depend on one
 * another in turn); a group is then reused 3p lines later, so window = 3 * p_max + 1
 * groups share the budget (the paper's window is p_m + 1).  Passing L = NULL plans A in
 * its own order with a single group (the unblocked reference configuration).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int32_t p_max;          /* largest power mpk_apply may request (1..31)                 */
    int32_t nrhs;           /* m: 1, 2, 4, 8 or 16 right-hand sides per call; 16 runs on the
                               unstaged block shape (shape 0 or 3) of the staged or the sweep
                               engine, else MPK_ERR_UNSUPPORTED                              */
    int64_t cache_bytes;    /* C in bytes; 0 = three quarters of the device L2 (five
                               quarters with two slices a warp, shape 5 below)               */
    int32_t order;          /* mpk_order of X, Y and the Chebyshev input/output             */
    int32_t chunk_rows;     /* rows per work unit (multiple of 32); 0 = 32 per compute warp
                               and slice of the block shape (512 for shape 2, 1024 for 5)     */
    int64_t wait_limit_ns;  /* bound on every device-side wait; 0 = 2 s                     */
    int64_t mem_budget;     /* bytes the plan may allocate on the device; 0 = no limit     */
    int32_t trace;          /* 1: the level-blocked kernel accumulates timing counters      */
    int32_t level_capped;   /* 1: a row of BFS level L takes powers 1..min(L, p) only, the
                               local phase of DLB-MPK (Alg. 2) with the levels built from the
                               halo rows (mpk_build_levels_from); groups are cut at every level
                               up to p_max; powers above a row's cap are left untouched.
                               Needs levels and MPK_ORDER_PLAN (else MPK_ERR_INVALID);
                               mpk_cheb_filter rejects such a plan                           */
    int32_t engine;         /* MPK_ENGINE_STAGED (0, default) or MPK_ENGINE_WARP (1), below  */
    int32_t shape;          /* block shape of the staged engine: 0 = chosen: 5 for binary32
                               sums over 2-byte values, one RHS and rows of at most 10
                               entries, else from the mean row width (2, else 3 for rows too
                               wide to stage); 1 = 13
                               compute warps, 3072-entry slots, 3 blocks per SM; 2 = 16
                               warps, 4608 entries, 2 blocks; 3 = 14 warps, entries read from
                               global memory;
                               4 = 10 compute warps, 2304-entry slots that also hold the
                               input rows the chunk reads (at most 4 row windows, 1664
                               doubles), 3 blocks per SM: the compute warps read only shared
                               memory.  Shape 4 is never chosen automatically; mpk_plan fails
                               with MPK_ERR_UNSUPPORTED when a chunk's windows do not fit;
                               5 = 16 compute warps taking two 32-row slices each of a unit,
                               9216-entry slots, 2 blocks per SM (1 with 4-byte or wider
                               values, whose slots take the shared memory of two)          */
    int64_t shuffle_seed;   /* race-detection aid: non-zero permutes the staged engine's work
                               units inside every line of the schedule (a valid order whose
                               results must be the same bits); 0 = the natural order         */
    int32_t accum;          /* arithmetic of the row sums: MPK_F64 (0, default) or MPK_F32.
                               MPK_F32 needs values stored as MPK_F32 or MPK_BF16 and the staged
                               (shapes 0-2) or sweep engine, without trace, level caps or
                               batching (else MPK_ERR_UNSUPPORTED).  Each row sum then runs in
                               binary32, one fmaf per entry in stored order, over the binary32
                               rounding (nearest even) of its inputs, and is stored widened
                               exactly into the binary64 results; X, Y, the Chebyshev vectors,
                               its three-term recurrence and its accumulator stay binary64.  The
                               plan keeps a ring of two binary32 copies of the current input
                               (8 * n * nrhs bytes).  mpk_spmv_powers refuses such a plan (its
                               comparator is a plan of engine MPK_ENGINE_SWEEP)               */
    int32_t split_levels;   /* 1: bulky levels are split (Sec. 6's recursion stage s_m, read as
                               breaking a level too large for the budget into pieces): levels
                               group as above while they fit; a level whose bytes exceed
                               floor(cache_bytes / window) closes the current group and is cut
                               into pieces of consecutive rows, each taking rows while its bytes
                               stay within that budget (at least one row), each a group; the next
                               level starts a new group.  A row costs (val_bytes + 4) * nnz(row) +
                               4 + 16 * nrhs bytes.  The work units then run in waves computed
                               from the exact chunk dependencies (w = 3 + group for power 1, then
                               2 more than the largest wave the unit reads), not on the lines
                               g + 3k, so every dependency still runs first.  Needs levels and the
                               staged or sweep engine, without level caps or batching
                               (MPK_ERR_INVALID otherwise).  0 = whole levels (default).      */
} mpk_plan_opts;

/* Engines of the level-blocked kernel (same results bit for bit, same Lp-diagram order):
 *  MPK_ENGINE_STAGED  blocks of one control warp and compute warps; the control warp claims
 *                     chunk units, copies their entries to shared memory with bulk copies and
 *                     polls chunk-level dependency flags.
 *  MPK_ENGINE_WARP    every warp claims items of kWarpSlices 32-row slices on its own, reads
 *                     the entries from global memory (L2) and waits for whole cells (group,
 *                     power k-1) of the three neighbouring groups; no shared memory, full
 *                     occupancy.  Not for batch plans (MPK_ERR_INVALID); mpk_apply_noalloc
 *                     runs such a plan with the staged engine.
 *  MPK_ENGINE_SWEEP   no level blocking: one grid-stride launch per power over the plan's
 *                     sliced copy, with the same row body and the same epilogue (powers or
 *                     Chebyshev recurrence), for matrices whose levels are too bulky for the
 *                     cache budget to give any reuse.  Not for batch or level-capped plans
 *                     (MPK_ERR_INVALID). */
enum { MPK_ENGINE_STAGED = 0, MPK_ENGINE_WARP = 1, MPK_ENGINE_SWEEP = 2 };

/* Fills the defaults described above (p_max = 8, nrhs = 1, order = ORIGINAL). */
void mpk_plan_opts_default(mpk_plan_opts *o);

/* Builds a plan for A (the same matrix the levels were built from).  Synchronises. */
mpk_status mpk_plan(const mpk_csr *A, const mpk_levels *L, const mpk_plan_opts *opts,
                    mpk_stream stream, mpk_plan_t **out);

typedef struct {
    int32_t n, nnz, nrhs, p_max, order;
    int32_t num_levels;           /* 0 for a plan without levels                         */
    int32_t num_groups;
    int32_t num_chunks;
    int64_t group_budget_bytes;   /* floor(cache_bytes / window)                         */
    int32_t window;               /* groups sharing the cache budget: 3 * p_max + 1      */
    int64_t cache_bytes;
    int64_t device_bytes;         /* bytes allocated by the plan                         */
    int64_t padded_entries;       /* entries of the sliced copy including padding        */
    const int32_t *group_level_ptr_dev; /* num_groups+1 level indices (NULL without levels) */
    const int32_t *group_row_ptr_dev;   /* num_groups+1 row offsets                        */
    const int32_t *chunk_row_ptr_dev;   /* num_chunks+1 row offsets                        */
    const int32_t *perm_dev;            /* new -> old (NULL: identity)                     */
    int32_t shape;                /* block shape of the staged engine (0..4, opts.shape - 1) */
    int32_t engine;               /* MPK_ENGINE_STAGED, MPK_ENGINE_WARP or MPK_ENGINE_SWEEP */
    int32_t chunk_rows;           /* rows per chunk limit in effect                      */
    int32_t accum;                /* MPK_F64 or MPK_F32 (opts.accum)                     */
    int32_t split_levels;         /* opts.split_levels; group_level_ptr then holds the level
                                     of each group's first row                             */
} mpk_plan_desc;

mpk_status mpk_plan_describe(const mpk_plan_t *P, mpk_plan_desc *out);

/* Writes the plan's permuted matrix P A P^T as CSR into caller buffers (device):
 * row_ptr[n+1], col[nnz], val[nnz] (float64, the stored values widened).  Asynchronous on
 * `stream`. */
mpk_status mpk_plan_export_csr(const mpk_plan_t *P, int32_t *row_ptr, int32_t *col, double *val,
                               mpk_stream stream);

/* Frees a plan and all device memory it holds (NULL: no-op).  Call it once the work queued
 * on the plan has completed (after mpk_sync_status, or a synchronisation of its streams). */
void mpk_plan_destroy(mpk_plan_t *P);

/* ---------------------------------------------------------------------------------------
 * mpk_apply: Y[k] = A^k X for k = 0..p (Sec. 3; Alg. 2's local phase on one device).
 * X: n x m device block; Y: (p+1) x n x m device block (Y[0] receives a copy of X), in the
 * plan's order (opts.order).  1 <= p <= p_max (p = 0 only copies X).  X must not overlap
 * Y[1..p].  One persistent kernel executes the Lp-diagram cells (group g, power k) in
 * diagonal order, split into row chunks; each chunk waits on the completion flags of the
 * chunks its rows read at power k-1.  With MPK_ORDER_ORIGINAL a gather kernel first takes
 * X into plan order in the plan's workspace, the kernel computes every power there, and a
 * last pass writes Y[1..p] through the permutation (one gather per output row).  Results
 * equal back-to-back SpMV bit for bit.  Not safe to run concurrently with another call on the same plan.
 * ------------------------------------------------------------------------------------- */
mpk_status mpk_apply(const mpk_plan_t *P, const double *X, int32_t p, double *Y, mpk_stream stream);

/* mpk_apply_host: mpk_apply with X and Y in host memory (Sec. 3's powers, the same bits as
 * mpk_apply).  X_host: n x m doubles (host, any host memory; pinned memory keeps the copy
 * asynchronous); Y_host: (p+1) x n x m doubles (host, page-locked: cudaHostAlloc or
 * cudaHostRegister, else MPK_ERR_INVALID), in the plan's order; 0 <= p <= p_max.  One copy
 * takes X to the device (the plan's workspace, no allocation).  With MPK_ORDER_PLAN (or no
 * levels), the staged engine and nrhs 1, the kernel stores every power's rows into Y_host as
 * its units finish, so the transfer to the host overlaps the wavefront; other plan-order plans
 * compute on the device and copy the p+1 blocks afterwards (level-capped plans need the first
 * case, else MPK_ERR_UNSUPPORTED).  With MPK_ORDER_ORIGINAL the powers are written through
 * the permutation straight into Y_host after the kernel (a temporary device copy of X is
 * allocated in stream order).  Asynchronous on `stream`: Y_host is complete when the stream
 * is.  Y_host must not overlap X_host.  Not for batch plans (MPK_ERR_INVALID); not safe to run
 * concurrently with another call on the same plan. */
mpk_status mpk_apply_host(const mpk_plan_t *P, const double *X_host, int32_t p, double *Y_host,
                          mpk_stream stream);

/* mpk_apply_noalloc: mpk_apply for callers that must not allocate device memory while the
 * call runs (the paper has no counterpart).  Such callers include code running while a
 * device allocator is locked or must keep a fixed footprint, and latency-critical loops that
 * cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.  The plan is
 * built beforehand and must use MPK_ORDER_PLAN (or no levels); X, p and Y are as for
 * mpk_apply (0 <= p <= p_max; p = 0 copies X to Y[0]).  The kernel's synchronisation state
 * lives in one fixed array of 2^20 32-bit words (4 MiB) of device memory that the library
 * declares statically, held by every GPU that loads the library until the process exits; a
 * call needs 8 + (p+1) * num_chunks words (8 control words, then one completion flag per
 * chunk and power) and fails with MPK_ERR_TOO_LARGE beyond that (larger chunk_rows means
 * fewer chunks).  The call allocates nothing: it clears the part of the array it uses,
 * launches the kernel and, if `status` (device int, caller-owned, may be NULL) is given,
 * writes MPK_OK or MPK_ERR_TIMEOUT there when the work completes on `stream`.  Every call
 * looks up the array's device address in the current context (cudaGetSymbolAddress, which
 * allocates nothing), so the address follows a device reset (plans do not survive one); the
 * first call on a device loads the array's module: make it before any stream capture.  All
 * calls on a device share the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller. */
mpk_status mpk_apply_noalloc(const mpk_plan_t *P, const double *X, int32_t p, double *Y,
                             int32_t *status, mpk_stream stream);

/* Plain comparator (Alg. 1 without halo exchange): p separate SpMV launches over the
 * plan's matrix copy, same row arithmetic as mpk_apply.  Arguments as for mpk_apply. */
mpk_status mpk_spmv_powers(const mpk_plan_t *P, const double *X, int32_t p, double *Y,
                           mpk_stream stream);

/* ---------------------------------------------------------------------------------------
 * mpk_cheb_filter: out = sum_{k=0..degree} c_k T_k(A') X with A' = (A - shift I) / scale
 * (Sec. 7: v_0 = x, v_1 = A' x, v_{k+1} = 2 A' v_k - v_{k-1}), run as ceil(degree/p_max)
 * level-blocked launches of p_max steps (the paper's blocking of a long recurrence into
 * MPK chunks of p_m).  Per row and step: w = A v_k (stored order), then
 * v_1 = fma(1/scale, w, (-shift/scale) v_0) and v_{k+1} = fma(2/scale, w,
 * fma(-2 shift/scale, v_k, -v_{k-1})); out accumulates c_0 v_0 then fma(c_k, v_k, out).
 * coeff_re (host, degree+1 doubles) are real coefficients.  If coeff_im (host) is not
 * NULL the coefficients are complex and act on pairs of right-hand sides (columns 2j,
 * 2j+1 = real, imaginary part), as in the time step exp(-i dt H) of Sec. 7; nrhs must be
 * even.  X and out: n x m device blocks in the plan's order; scale != 0.
 * ------------------------------------------------------------------------------------- */
mpk_status mpk_cheb_filter(const mpk_plan_t *P, const double *X, int32_t degree,
                           const double *coeff_re, const double *coeff_im, double scale,
                           double shift, double *out, mpk_stream stream);

/* The same filter in pieces, with its state in a caller-owned device buffer that can be saved
 * and restored between pieces (checkpoint/resume at any step; the natural point is a block
 * boundary of p_max steps): 4 x n x nrhs float64 in the plan's row order,
 * mpk_cheb_state_bytes(P) bytes.  Blocks 0..2 are a ring holding v_j in block j % 3 (when the
 * state holds step k, v_k and v_{k-1} are live and the third block is scratch), block 3 is the
 * accumulator.  Save and restore all mpk_cheb_state_bytes(P) bytes.  Any split of the steps
 * gives the same bits as one mpk_cheb_filter call.
 *   mpk_cheb_begin:   state <- v_0 = X, acc = c_0 X (c_0 = c0_re + i c0_im on (re, im) column
 *                     pairs when complex_coeff is 1); the state holds step 0.
 *   mpk_cheb_advance: steps k_begin+1 .. k_end with coefficients coeff_re[k] (and coeff_im[k]),
 *                     k absolute; k_begin must be the step the state holds (the caller tracks
 *                     it); launches of at most p_max steps.
 *   mpk_cheb_finish:  out <- acc (in the numbering opts.order selects).
 * Arguments, errors and streams otherwise as for mpk_cheb_filter.  mpk_cheb_state_bytes returns
 * 0 for a NULL plan. */
int64_t mpk_cheb_state_bytes(const mpk_plan_t *P);
mpk_status mpk_cheb_begin(const mpk_plan_t *P, const double *X, double c0_re, double c0_im, int32_t complex_coeff,
                          double *state, mpk_stream stream);
mpk_status mpk_cheb_advance(const mpk_plan_t *P, double *state, int32_t k_begin, int32_t k_end,
                            const double *coeff_re, const double *coeff_im, double scale, double shift,
                            mpk_stream stream);
mpk_status mpk_cheb_finish(const mpk_plan_t *P, const double *state, double *out, mpk_stream stream);

/* Timing counters of a plan built with opts.trace = 1, accumulated over all launches since
 * the plan was created (host array of MPK_TRACE_COUNTERS int64): 0 units, 1 ns the control
 * warps spent polling dependencies, 2 units whose dependencies were not all met at the first
 * check, 3 ns control warps waited for a free slot, 4 ns compute warps waited for a unit,
 * 5 ns compute warps spent on units, 6 ns summed over blocks from start to exit, 7 launches,
 * 8 SM cycles control warps spent staging, 9 cycles in the acquire fence and hand-over,
 * 10 cycles fetching later tickets, records and flags, 11 cycles decoding the current record,
 * 12 cycles compute warps spent until the x entries of their first batch arrived, 13 cycles
 * from then to the end of the unit (FMAs, stores, publication), 14 ns from a hand-over to
 * the first compute warp seeing it (units the warp waited for), 15 such units, 16 SM cycles
 * summed over blocks from start to exit (cycles per ns = counter 16 / counter 6).
 * Synchronises `stream`.  MPK_ERR_UNSUPPORTED if the plan has no trace. */
#define MPK_TRACE_COUNTERS 17
mpk_status mpk_read_trace(const mpk_plan_t *P, int64_t *counters, mpk_stream stream);

/* ---------------------------------------------------------------------------------------
 * Batched MPK: `count` independent matrices with their own sizes and powers in one plan and
 * one persistent launch per apply.  The plan is that of the block-diagonal direct sum of the
 * matrices (Sec. 3's level blocking applies to it unchanged): block i keeps its own BFS
 * levels and row range, groups never span two blocks, and the blocks' Lp-diagram cells are
 * merged line by line into one ticket space, so that small blocks run side by side.
 * mats[i]: device CSR as for mpk_plan, all of one val_type; p_each[i] in [1, opts->p_max];
 * opts->nrhs applies to every block and opts->order to each block's own numbering (in plan
 * order block i uses the numbering of its own levels, mpk_build_levels(mats[i], 0)).
 * Synchronises.  The plan runs through mpk_batch_apply only (mpk_apply and the others fail
 * with MPK_ERR_INVALID on it).
 * ------------------------------------------------------------------------------------- */
mpk_status mpk_batch_plan(const mpk_csr *mats, int32_t count, const int32_t *p_each,
                          const mpk_plan_opts *opts, mpk_stream stream, mpk_plan_t **out);

/* X[i], Y[i]: host arrays of `count` device pointers; X[i] is n_i x nrhs and Y[i] receives
 * (p_each[i] + 1) x n_i x nrhs, powers 0..p_each[i] of block i (row-major, float64).
 * Y[i] = NULL leaves block i's powers in the plan's workspace only (see mpk_batch_workspace),
 * which saves their copy.  Asynchronous on `stream` (capturable in a CUDA graph); errors as
 * for mpk_apply. */
mpk_status mpk_batch_apply(const mpk_plan_t *P, const double *const *X, double *const *Y, mpk_stream stream);

/* The batch plan's workspace: power k of block i, row r, column j is
 * work[k * power_stride + (row_offsets[i] + r) * nrhs + j] (in plan order) after an apply,
 * valid until the next call on the plan. */
mpk_status mpk_batch_workspace(const mpk_plan_t *P, const double **work, int64_t *power_stride);

/* Number of blocks, their row offsets (count + 1 entries) and powers; NULL outputs are skipped. */
mpk_status mpk_batch_describe(const mpk_plan_t *P, int32_t *count, int32_t *row_offsets, int32_t *powers);

/* Synchronises `stream` and reports a device-side failure of the plan's calls since the
 * last mpk_sync_status (MPK_ERR_TIMEOUT), else MPK_OK or a CUDA error.  The plan keeps its
 * launch epoch on the device, so calls captured in a CUDA graph can be replayed: every replay
 * is a new launch.  (After 2^30 launches made through the API the plan clears its flags;
 * graph replays are not counted.) */
mpk_status mpk_sync_status(const mpk_plan_t *P, mpk_stream stream);

/* Fault injection for tests of the failure path (no counterpart in the paper): in the next
 * level-blocked launch on this plan, work unit (chunk, k) computes its rows but does not
 * publish its completion flag.  Units that read those rows wait until the plan's
 * wait_limit_ns expires, record MPK_ERR_TIMEOUT and leave; every wait stays bounded and
 * the device stays usable.  mpk_sync_status then reports MPK_ERR_TIMEOUT. */
mpk_status mpk_debug_drop_release(mpk_plan_t *P, int32_t chunk, int32_t k);

/* ---------------------------------------------------------------------------------------
 * Measurement aids (the analogue of the paper's load-only bandwidth kernel, Sec. 6).
 * mpk_probe_load: `reps` passes of 16-byte loads over buf[0..bytes) (buf 16-byte aligned,
 * bytes a multiple of 16, else MPK_ERR_INVALID) by ctas_per_sm * #SM blocks of 512 threads; sink is a device int that is written
 * only if a checksum matches a constant.  mpk_probe_dfma: blocks * 256 threads each run
 * `iters` x 8 independent FP64 FMAs; sink as above.
 * ------------------------------------------------------------------------------------- */
mpk_status mpk_probe_load(const void *buf, int64_t bytes, int32_t reps, int32_t ctas_per_sm,
                          int32_t *sink, mpk_stream stream);
mpk_status mpk_probe_dfma(int32_t blocks, int32_t iters, double *sink, mpk_stream stream);

/* One SpMV on the plan-order rows [row_begin, row_end): Y[r] = (A X)[r] for those rows only
 * (X, Y: n x nrhs, plan order, device; other rows of Y untouched).  The per-level steps of
 * DLB-MPK's third phase (Alg. 2).  Asynchronous on `stream`. */
mpk_status mpk_spmv_rows(const mpk_plan_t *P, int32_t row_begin, int32_t row_end, const double *X, double *Y,
                         mpk_stream stream);

/* The row-range SpMV of several plans in one launch: for segment i < count, rows
 * [row_begin[i], row_end[i]) of Y[i] = A_i X[i] with A_i the matrix of plans[i] (plan order,
 * n_i x nrhs, device).  The per-level steps of DLB-MPK's third phase (Alg. 2) taken by every
 * partition at once.  count <= MPK_MAX_ROW_SEGMENTS; the plans of non-empty segments share
 * one value type and one nrhs (else MPK_ERR_INVALID).  The host arrays are read during the
 * call only.  Asynchronous on `stream`. */
#define MPK_MAX_ROW_SEGMENTS 32
mpk_status mpk_spmv_rows_multi(int32_t count, const mpk_plan_t *const *plans, const int32_t *row_begin,
                               const int32_t *row_end, const double *const *X, double *const *Y,
                               mpk_stream stream);

/* dst[dst_idx[t]] = src[src_idx[t]] for t < n, m doubles a row; the index arrays are device
 * int64 row numbers (the caller keeps them in range and the destinations distinct).  src and
 * dst may be one buffer when no destination row is also a source row.  The halo exchange of
 * partitions held on one device.  Asynchronous on `stream`. */
mpk_status mpk_copy_rows(const double *src, const int64_t *src_idx, double *dst, const int64_t *dst_idx, int64_t n,
                         int32_t m, mpk_stream stream);

/* dst[r] = src[idx[r]] for r < n, m doubles a row (device arrays; src and dst do not
 * overlap): the halo exchange between partitions held on one device.  Asynchronous on
 * `stream`. */
mpk_status mpk_gather_rows(const double *src, const int32_t *idx, int32_t n, int32_t m, double *dst,
                           mpk_stream stream);

/* dst[i] = src[i] widened to float64 for i < n, with the conversion the kernels use (src of
 * mpk_dtype val_type, device memory; MPK_ERR_UNSUPPORTED for another type).  Asynchronous
 * on `stream`. */
mpk_status mpk_widen_values(int32_t val_type, const void *src, int64_t n, double *dst, mpk_stream stream);

/* Number of SMs and L2 bytes of the current device. */
mpk_status mpk_device_info(int32_t *num_sms, int64_t *l2_bytes);

const char *mpk_status_string(mpk_status s);
const char *mpk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MPK_H */
