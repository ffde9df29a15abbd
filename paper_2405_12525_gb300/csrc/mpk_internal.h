// Internal declarations shared by the CUDA translation units of libmpk.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <new>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/mpk.h"

namespace mpk {

// ----------------------------------------------------------------------------- errors
// Library code throws Fail; every extern "C" entry point catches it and returns .status.
struct Fail {
    mpk_status status;
};

void set_error(const char *fmt, ...);
[[noreturn]] void fail(mpk_status s, const char *fmt, ...);

#define MPK_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            ::mpk::fail(e_ == cudaErrorMemoryAllocation ? MPK_ERR_OOM : MPK_ERR_CUDA,           \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,       \
                        __LINE__);                                                              \
    } while (0)

#define MPK_LAUNCHED() MPK_CUDA(cudaGetLastError())

// extern "C" entry points: internal failures become an mpk_status
#define MPK_GUARD_BEGIN try {
#define MPK_GUARD_END                                                  \
    }                                                                  \
    catch (const ::mpk::Fail &f) {                                     \
        return f.status;                                               \
    }                                                                  \
    catch (const std::bad_alloc &) {                                   \
        ::mpk::set_error("host allocation failed");                    \
        return MPK_ERR_OOM;                                            \
    }                                                                  \
    catch (...) {                                                      \
        ::mpk::set_error("unexpected internal error");                 \
        return MPK_ERR_CUDA;                                           \
    }

inline cudaStream_t as_stream(mpk_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------------------------------- memory
// Device allocation with byte accounting against an optional budget.
struct Arena {
    int64_t bytes = 0;
    int64_t budget = 0;  // 0 = unlimited
    std::vector<void *> ptrs;
    std::vector<int64_t> sizes;
    void *alloc(int64_t nbytes);
    void free(void *p);  // frees one allocation of this arena (no-op for NULL)
    template <class T> T *alloc_n(int64_t n) { return static_cast<T *>(alloc(n * (int64_t)sizeof(T))); }
    void release();
};

// Temporary device buffer, allocated and freed in the order of stream s (stream-ordered pool:
// no device-wide synchronisation as with cudaFree), freed on scope exit (not counted in a plan).
template <class T> struct Tmp {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    Tmp(int64_t n, cudaStream_t stream) : s(stream) {
        if (n > 0) MPK_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&p), (size_t)n * sizeof(T), s));
    }
    ~Tmp() {
        if (p) cudaFreeAsync(p, s);
    }
    Tmp(const Tmp &) = delete;
    Tmp &operator=(const Tmp &) = delete;
};

// ----------------------------------------------------------------------------- primitives
// out[0..n] = exclusive prefix sum of in[0..n) (out[n] = total).  out may alias in.
void exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
void exclusive_scan(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits of key.
// Inputs are consumed (used as ping-pong buffers); the sorted result is returned through
// *keys_out / *vals_out, which point into either the input or the scratch buffers.
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp,
                      int64_t n, int key_bits, cudaStream_t s, uint32_t **keys_out,
                      uint32_t **vals_out);

void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s);
void iota_i32(int32_t *p, int64_t n, cudaStream_t s);

int device_sms();
int64_t device_l2_bytes();

// ----------------------------------------------------------------------------- value widening
// float32 / bfloat16 -> float64 is exact: both are subsets of binary64 (a bfloat16 is the upper
// half of a binary32).  Done with integer operations on the IEEE 754 encodings, so that it
// adds no work to the FP64 pipe: a normal binary32 keeps its sign, its 8-bit exponent is
// rebiased from 127 to 1023 (+896) into the 11-bit field and its 23-bit fraction becomes the
// top of the 52-bit one.  Zeros, subnormals, infinities and NaNs take separate paths (a
// signaling NaN comes out quiet, as from any IEEE 754 conversion).
__device__ __forceinline__ double widen_binary32(uint32_t u) {
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xffu, f = u & 0x7fffffu;
    if (e - 1u < 254u) return __hiloint2double((int)(sign | ((e + 896u) << 20) | (f >> 3)), (int)(f << 29));
    if (e == 255u)  // infinity, or NaN: payload kept, quiet bit set as an IEEE 754 conversion does
        return __hiloint2double((int)(sign | 0x7ff00000u | (f >> 3) | (f ? 0x80000u : 0u)), (int)(f << 29));
    if (f == 0u) return __hiloint2double((int)sign, 0);                                             // +-0
    // subnormal f * 2^-149: with the leading one of f at bit q the value is 2^(q-149) (1 + rest)
    const int q = 31 - __clz((int)f);
    const uint64_t frac = (uint64_t)(f ^ (1u << q)) << (52 - q);
    return __longlong_as_double((long long)(((uint64_t)sign << 32) | ((uint64_t)(q + 874) << 52) | frac));
}
// The kernels' widening, for the values a plan stores (zeros and normal numbers only, checked
// by the planner): the sign stays, the exponent and fraction move right by 3 bits into the
// binary64 fields and the exponent is rebiased by adding 896 << 20; zero keeps only its sign.
// No branch, five integer operations.
__device__ __forceinline__ double widen_normal32(uint32_t u) {
    const uint32_t mag = u & 0x7fffffffu;
    const uint32_t hi = (mag ? (mag >> 3) + 0x38000000u : 0u) | (u & 0x80000000u);
    return __hiloint2double((int)hi, (int)(u << 29));
}
// 1 when the binary32 bits are a subnormal, an infinity or a NaN
__device__ __forceinline__ int binary32_special(uint32_t u) {
    const uint32_t e = (u >> 23) & 0xffu;
    return e == 255u || (e == 0u && (u & 0x7fffffu) != 0u);
}
__device__ __forceinline__ double widen_value(double v) { return v; }
__device__ __forceinline__ double widen_value(float v) { return widen_binary32(__float_as_uint(v)); }
__device__ __forceinline__ double widen_value(uint16_t v) { return widen_binary32((uint32_t)v << 16); }  // bfloat16 bits

// ----------------------------------------------------------------------------- objects
struct Levels {
    int32_t n = 0;
    int32_t num_levels = 0;
    int32_t *level_ptr = nullptr;  // num_levels + 1
    int32_t *perm = nullptr;       // new -> old
    int32_t *iperm = nullptr;      // old -> new
    int32_t *level_of = nullptr;   // per original vertex
    std::vector<int32_t> h_level_ptr;
    Arena arena;
};

// Arguments of the level-blocked kernel, passed by value.
constexpr int kMaxP = 31;
// Block shapes of the level-blocked kernel: compute warps per block (one 32-row slice each
// per unit, so the default chunk is 32 * comp_warps rows), padded entries a shared-memory
// slot holds (a chunk is cut to fit one), blocks per SM for the single-vector power
// kernel, staging slots per block, and the 8-byte words of input rows a slot holds (x_words,
// 0: none) and the control warps (1, or 2: one polls dependencies, one stages).  Shape 0 suits rows of up to about 7 stored entries (13 slices of width 7 fill a
// slot); shape 1 suits wider rows; shape 2 stages nothing (stage_entries 0: the compute
// warps read the entries from global memory, and chunks are not cut by a slot), for rows so
// wide that a slot holds only a few slices.  Shape 3 also stages the unit's input rows:
// after the dependency poll the control warp copies the (at most four) row windows of the
// input vector that the chunk reads into the slot, and the chunk's column indices are
// staged as 16-bit positions in that window area, so that the compute warps read nothing
// but shared memory.  Every block also has a publisher warp (see publisher_loop).  The
// planner picks shape 1 when its slot holds at least 6 slices of the mean width, else
// shape 2, unless the plan options name a shape (0 or 3 included).
struct BlockShape {
    int comp_warps, stage_entries, blocks, slots, x_words, ctrl_warps;
    int slices_per_warp;  // 32-row slices a compute warp takes per unit (0: one)
};
#ifndef MPK_XS_WARPS
#define MPK_XS_WARPS 10
#endif
#ifndef MPK_XS_ENTRIES
#define MPK_XS_ENTRIES 2304
#endif
#ifndef MPK_XS_BLOCKS
#define MPK_XS_BLOCKS 3
#endif
#ifndef MPK_XS_SLOTS
#define MPK_XS_SLOTS 2
#endif
#ifndef MPK_XS_WORDS
#define MPK_XS_WORDS 1664
#endif
#ifndef MPK_XS_CTL
#define MPK_XS_CTL 1
#endif
// shape 4: compute warps, slot entries and slices a warp takes per unit (at most 32 slices a unit)
#ifndef MPK_S4_WARPS
#define MPK_S4_WARPS 16
#endif
#ifndef MPK_S4_ENTRIES
#define MPK_S4_ENTRIES 9216
#endif
#ifndef MPK_S4_SPW
#define MPK_S4_SPW 2
#endif
constexpr BlockShape kShapes[5] = {{13, 3072, 3, 2, 0, 1},
                                   {16, 4608, 2, 2, 0, 1},
                                   {14, 0, 2, 2, 0, 1},
                                   {MPK_XS_WARPS, MPK_XS_ENTRIES, MPK_XS_BLOCKS, MPK_XS_SLOTS, MPK_XS_WORDS, MPK_XS_CTL},
                                   {MPK_S4_WARPS, MPK_S4_ENTRIES, 2, 2, 0, 1, MPK_S4_SPW}};
constexpr int kNumShapes = 5;
constexpr int kShapeX = 3;  // the shape that stages input rows
// input-row windows of a chunk (shape 3): one per dependency range
constexpr int kXWin = 4;
// 1: chunks whose entries fit a buffer are copied to shared memory by the bulk-copy engine;
// 0: every unit reads its entries from global memory (L2) directly
#ifndef MPK_STAGE
#define MPK_STAGE 1
#endif
constexpr bool kStageChunks = MPK_STAGE != 0;
// dependency ranges kept per chunk (exact sets compressed to this many index ranges)
constexpr int kDepRanges = 4;
// trace counters accumulated in shared memory (the last one, SM cycles, is added directly)
constexpr int kTraceShared = MPK_TRACE_COUNTERS - 1;
// The level-blocked kernel walks the Lp diagram along lines g + kSlotSkew * k = const.  With
// skew 1 (the paper's diagonals) the cells of one line form a dependency chain; with skew 3
// every dependency of a cell lies at least two lines back, so the cells in flight on the
// GPU do not wait on each other.  A group is then reused kSlotSkew * p lines later, so the
// cache budget is shared by kSlotSkew * p_max + 1 groups.
constexpr int kSlotSkew = 3;
// chunk record: 8 ints of chunk data, 2 * kDepRanges ints of dependency ranges, the
// widths of up to kRecSlices slices as bytes (only staged chunks use them) and, for shape 3,
// kXWin input-row windows as (first row, rows, position in the slot's window area in rows);
// the other shapes keep the widths of slices 16..31 in the first 4 window words
constexpr int kRecSlices = 16;      // shape 3 (its windows follow the widths)
constexpr int kRecSlicesWide = 32;  // the other shapes: the window words hold 16 more widths
constexpr int kRecWin = 8 + 2 * kDepRanges + kRecSlices / 4;  // first int of the windows
constexpr int kRecInts = kRecWin + 3 * kXWin;
static_assert(kRecInts <= 32, "a chunk record is read by one lane per int");
static_assert(kRecWin + kRecSlicesWide / 4 - kRecSlices / 4 <= kRecInts, "wide widths in the window words");
static_assert(MPK_S4_WARPS * MPK_S4_SPW <= kRecSlicesWide, "a unit of shape 4 has at most 32 slices");
struct KArgs {
    // sliced matrix copy (plan order)
    const void *val;  // values of the matrix's value type (Plan::val_type)
    const int32_t *col;
    const int64_t *slice_ptr;
    const int32_t *rowlen;
    const int32_t *chunk_row;
    const int32_t *chunk_slice;
    const int2 *dep;
    const int4 *dep_ranges;  // 2 x int4 per chunk: kDepRanges (lo, hi) pairs
    const int4 *chunk_rec;   // kRecInts ints per chunk: rows, slices, entries, ranges, widths, windows
    const uint16_t *lcol;    // shape 3: window-area position of every entry's column (0xffff: padding)
    int32_t n;
    int32_t nchunks;
    // schedule for this launch
    const int32_t *units;
    int64_t nunits;
    int32_t *flags;  // (p+1) x nchunks, epoch-valued
    unsigned int *epoch_word;  // the last launch's epoch: this launch uses *epoch_word + 1
    unsigned int *ticket;
    unsigned int *exit_count;
    int32_t *err;    // err[0] = epoch of a failed launch, err[1] = status code
    int64_t wait_ns;
    int32_t drop_unit;  // test hook: this unit (chunk << 5 | k) skips its release, -1 = none
    unsigned long long *trace;  // timing counters (MPK_TRACE_COUNTERS) or null
    // vectors
    const double *x0;  // power-0 block (plan order)
    double *ybase;     // slot(k) = ybase + (k % ring) * ystride
    int64_t ystride;
    int32_t ring;
    double *y0copy;    // if set, units of power 1 copy their rows of x0 here
    double *yhost = nullptr;  // if set, every power's rows are stored here too (pinned host memory,
                              // device-mapped, plan order, ystride apart): output overlaps compute
    float *shadow;     // binary32 accumulation: ring of 2 blocks (ystride floats apart); slot j & 1
                       // holds the binary32 rounding of step j, the input of step j + 1
    int32_t k_offset;  // absolute index of local power 0 (Chebyshev blocks)
    // Chebyshev recurrence
    double alpha, beta, halpha, hbeta;
    double *acc;
    int32_t complex_coeff;
    double cre[kMaxP + 1];
    double cim[kMaxP + 1];
    // warp-ticketed engine (MPK_ENGINE_WARP): the cells (group g, power k) of this launch in
    // ticket order, each split into items of kWarpSlices slices, and per-cell counters of
    // finished items
    const int64_t *w_item;   // first item of each cell (strictly ascending), w_ncells entries
    const int32_t *w_gk;     // g << 5 | k of each cell
    int64_t w_ncells;
    int64_t w_nitems;
    int32_t *w_cnt;          // (p+1) x nchunks finished slices per (power, chunk); zero at launch start
    unsigned int *w_q;       // kWarpQueues claim counters; zero when the launch starts
    const int32_t *g_row;    // G+1 group row offsets
    const int32_t *g_slice;  // G+1 group slice offsets
    const int32_t *w_slice_chunk;  // chunk of every slice
    const int32_t *w_chunk_nsl;    // slices of every chunk
    int32_t ngroups;
    int32_t p_launch;              // powers of this launch (local 1..p_launch)
};
// warp-ticketed engine: slices per item, claim queues (one per warp of a block)
constexpr int kWarpSlices = 1;
constexpr int kWarpQueues = 16;

struct Plan {
    int32_t n = 0, nnz = 0, m = 1, p_max = 8, order = MPK_ORDER_ORIGINAL;
    int32_t val_type = MPK_F64, val_bytes = 8;  // storage of the matrix values (mpk_dtype)
    int32_t accum = MPK_F64;                     // row-sum arithmetic: MPK_F64 or MPK_F32
    float *shadow = nullptr;                     // binary32 accumulation: 2 x n x m binary32 input ring
    int32_t num_levels = 0, num_groups = 0, num_chunks = 0, num_slices = 0;
    int32_t chunk_rows = 512;
    int32_t shape = 0;  // block shape of the level-blocked kernel (kShapes)
    int64_t cache_bytes = 0, group_budget = 0, padded = 0, wait_ns = 0;
    int32_t window = 0;  // groups sharing the cache budget: kSlotSkew * p_max + 1
    bool identity = false;
    // device data (owned by arena)
    void *val = nullptr;  // val_bytes per padded entry
    int32_t *col = nullptr;
    uint16_t *lcol = nullptr;  // shape 3: column positions in the chunk's input-row windows
    int64_t *slice_ptr = nullptr;
    int32_t *rowlen = nullptr;
    int32_t *chunk_row = nullptr;
    int32_t *chunk_slice = nullptr;
    int2 *dep = nullptr;         // hull of each chunk's dependencies
    int4 *dep_ranges = nullptr;  // exact dependencies as kDepRanges index ranges
    int4 *chunk_rec = nullptr;   // per-chunk records read by the kernel's control warp
    int32_t *group_level_ptr = nullptr;
    int32_t *group_row_ptr = nullptr;
    int32_t *perm = nullptr;   // owned copy (NULL for identity)
    int32_t *iperm = nullptr;
    int32_t *units = nullptr;  // concatenated unit tables for p = 1..p_max
    std::vector<int64_t> unit_off;  // unit_off[p] .. unit_off[p] + nunits(p)
    int32_t *flags = nullptr;
    unsigned int *ctl = nullptr;  // [0] ticket, [1] exit count, [2] err epoch, [3] err code
    double *work = nullptr;       // work_slots blocks of n*m: powers in plan order, or Chebyshev ring + accumulator
    int32_t work_slots = 0;
    int64_t launches = 0;  // launches since the flags were last cleared (wrap guard of the epochs)
    // batch plans (direct sum of several matrices, mpk_batch_plan): instance i owns rows
    // [inst_row[i], inst_row[i+1]) in both numberings and takes powers 1..inst_p[i]
    std::vector<int32_t> inst_row, inst_p;
    std::vector<int32_t> h_chunk_row;  // chunk row offsets on the host (num_chunks + 1)
    bool level_capped = false;        // rows of level L take powers up to min(L, p) (DLB local phase)
    bool split_levels = false;        // bulky levels cut into budget-sized groups, units in wave order
    int32_t level0_rows = 0;          // level-capped plans: rows of level 0 (no unit copies their x)
    // warp-ticketed engine (plans built with engine = MPK_ENGINE_WARP)
    int32_t engine = MPK_ENGINE_STAGED;
    int32_t *g_slice = nullptr;         // G+1 group slice offsets (device)
    int64_t *w_item = nullptr;          // cells of every p, concatenated (device)
    int32_t *w_gk = nullptr;
    std::vector<int64_t> w_cell_off;    // p_max + 2: the cells of p start at w_cell_off[p]
    std::vector<int64_t> w_items;       // p_max + 1: items of a launch with p powers
    int32_t *w_cnt = nullptr;           // (p_max+1) x nchunks counters, then kWarpQueues claim counters
    int32_t *w_slice_chunk = nullptr;   // chunk of every slice (device)
    int32_t *w_chunk_nsl = nullptr;     // slices of every chunk (device)
    int32_t drop_unit = -1;  // armed by mpk_debug_drop_release for the next launch
    unsigned long long *trace = nullptr;  // counters when built with opts.trace
    int grid_mpk[4] = {0, 0, 0, 0};  // persistent grid size per mode
    Arena arena;
};

// kernels (mpk_kernel.cu)
void launch_mpk(const Plan &P, KArgs &a, int mode, cudaStream_t s);
void launch_spmv(const Plan &P, const double *x, double *y, cudaStream_t s);
// one SpMV on the plan-order rows [lo, hi) only
// One launch over row ranges of up to kMaxRowSegs plans (same value type and nrhs).
constexpr int kMaxRowSegs = 32;
struct RowSeg {
    const void *val;
    const int32_t *col;
    const int64_t *slice_ptr;
    const int32_t *chunk_row;
    const int32_t *chunk_slice;
    const double *x;
    double *y;
    int32_t c0, lo, hi;
};
struct RowSegs {
    int32_t count;
    int32_t first[kMaxRowSegs + 1];
    RowSeg seg[kMaxRowSegs];
};
void launch_spmv_rows(const Plan *const *plans, const int32_t *lo, const int32_t *hi, const double *const *x,
                      double *const *y, int count, cudaStream_t s);
void launch_copy_rows(const double *src, const int64_t *src_idx, double *dst, const int64_t *dst_idx, int64_t n,
                      int32_t m, cudaStream_t s);
// Y[k][i] = W[k][iperm[i]] (iperm NULL: W[k][base + i]) for k = k0..p, i < n; W's powers are
// w_pstride doubles apart (< 0: n * m), Y's n * m; Y may be device-mapped host memory (the
// writes of a thread block are whole consecutive rows)
void launch_scatter_powers(const double *W, const int32_t *iperm, double *Y, int32_t n, int32_t m, int32_t p,
                           cudaStream_t s, int64_t w_pstride = -1, int32_t base = 0, int32_t k0 = 1);
// dst[r] = src[perm[r] - base] for r < n (m values a row; perm NULL: the identity)
void launch_gather_rows(const double *src, const int32_t *perm, double *dst, int32_t n, int32_t m,
                        cudaStream_t s, int32_t base = 0);
void launch_scatter_rows(const double *src, const int32_t *iperm, double *dst, int32_t n, int32_t m,
                         cudaStream_t s);
void launch_cheb_init(const double *v0, double *acc, int32_t n, int32_t m, double c0re, double c0im,
                      int complex_coeff, cudaStream_t s);
int occupancy_grid(int mode, int m, bool trace, int vtype, int shape, bool a32 = false);
// dst[i] = src[i] rounded to binary32, nearest even (binary32 accumulation: its first input)
void launch_round_f32(const double *src, int64_t n, float *dst, cudaStream_t s);
// dst[i] = src[i] widened to float64 (src of mpk_dtype vtype), exact
void widen_values(int vtype, const void *src, int64_t n, double *dst, cudaStream_t s);

// level builder (mpk_levels.cu)
// BFS levels from `root`, or from every vertex of `roots` (ascending) as level 0
Levels *build_levels(const mpk_csr *A, int32_t root, cudaStream_t s, const std::vector<int32_t> *roots = nullptr);
void validate_csr(const mpk_csr *A, cudaStream_t s);

// planner (mpk_plan.cu)
// inst_row / inst_p: batch plans only (instance row offsets, count + 1 entries; powers per instance)
// the next launch epoch of P (clears the flags before the epochs could wrap)
void next_epoch(Plan &P, cudaStream_t s);
// kernel arguments of P for the unit table of power p
KArgs base_args(Plan &P, int32_t p);
Plan *build_plan(const mpk_csr *A, const Levels *L, const mpk_plan_opts *o, cudaStream_t s,
                 const std::vector<int32_t> *inst_row = nullptr, const std::vector<int32_t> *inst_p = nullptr);
void export_csr(const Plan &P, int32_t *rp, int32_t *ci, double *va, cudaStream_t s);

// probes (mpk_kernel.cu)
void probe_load(const void *buf, int64_t bytes, int reps, int ctas_per_sm, int32_t *sink, cudaStream_t s);
void probe_dfma(int blocks, int iters, double *sink, cudaStream_t s);

}  // namespace mpk

// handles behind the opaque types of the C ABI
struct mpk_levels_s {
    mpk::Levels *impl;
};
struct mpk_plan_s {
    mpk::Plan *impl;
};
