// Planner: the permuted, sliced matrix copy, level groups, row chunks, chunk dependency
// ranges and the unit tables of the level-blocked schedule.
#include "mpk_internal.h"

#include <algorithm>
#include <climits>

namespace mpk {

static int grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// length of new row r = length of old row perm[r]
__global__ void k_rowlen(int32_t n, const int32_t *rp, const int32_t *perm, int32_t *len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t old = perm ? perm[r] : (int32_t)r;
        len[r] = rp[old + 1] - rp[old];
    }
}

__global__ void k_gather_i32(const int32_t *src, const int32_t *idx, int32_t cnt, int32_t *dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += stride) dst[i] = src[idx[i]];
}

__global__ void k_chunk_of_row(const int32_t *chunk_row, int32_t nchunks, int32_t *chunk_of_row) {
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x)
        for (int32_t r = chunk_row[c] + threadIdx.x; r < chunk_row[c + 1]; r += blockDim.x) chunk_of_row[r] = c;
}

// longest row of each 32-row slice; one thread per slice
__global__ void k_slice_width(const int32_t *slice_row, int32_t nslices, const int32_t *rowlen, int32_t *width) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sl < nslices; sl += stride) {
        int32_t w = 0;
        for (int32_t r = slice_row[sl]; r < slice_row[sl + 1]; ++r) w = max(w, rowlen[r]);
        width[sl] = w;
    }
}

// Copies every row of P A P^T into its slice (entry j of lane l at slice_ptr + 32 j + l),
// relabelling columns through iperm, and folds the chunks each row reads into the
// dependency range of its chunk.  When A is not known to be symmetric, a chunk is also
// added to the ranges of the chunks it reads, so that ranges cover both directions.
__device__ __forceinline__ int value_special(double) { return 0; }
__device__ __forceinline__ int value_special(float v) { return binary32_special(__float_as_uint(v)); }
__device__ __forceinline__ int value_special(uint16_t v) { return binary32_special((uint32_t)v << 16); }

template <class T>
__global__ void k_fill(int32_t n, const int32_t *rp, const int32_t *ci, const T *va, const int32_t *perm,
                       const int32_t *iperm, const int32_t *chunk_row, const int32_t *chunk_slice,
                       const int32_t *chunk_of_row, const int64_t *slice_ptr, T *sval, int32_t *scol,
                       int2 *dep, int symmetric, int32_t *special) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = chunk_of_row[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        const int32_t old = perm ? perm[r] : (int32_t)r;
        const int32_t e0 = rp[old], e1 = rp[old + 1];
        int32_t lo = c, hi = c;
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t nc = iperm ? iperm[ci[e]] : ci[e];
            const int64_t dst = base + 32 * (int64_t)(e - e0);
            sval[dst] = va[e];
            if (value_special(va[e])) *special = 1;  // narrow types: subnormal, infinity or NaN
            scol[dst] = nc;
            const int32_t cc = chunk_of_row[nc];
            lo = min(lo, cc);
            hi = max(hi, cc);
            if (!symmetric) {
                if (dep[cc].x > c) atomicMin(&dep[cc].x, c);
                if (dep[cc].y < c) atomicMax(&dep[cc].y, c);
            }
        }
        if (dep[c].x > lo) atomicMin(&dep[c].x, lo);
        if (dep[c].y < hi) atomicMax(&dep[c].y, hi);
    }
}

__global__ void k_dep_init(int2 *dep, int32_t nchunks) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x)
        dep[c] = make_int2(c, c);
}

// Exact dependency sets: bit (cc - hull_lo[c]) of chunk c's bitmap is set when a row of c
// reads a row of chunk cc (and, for patterns not known to be symmetric, when a row of cc
// reads a row of c).  Every chunk depends on itself.
__global__ void k_dep_bits(int32_t n, const int32_t *rowlen, const int32_t *chunk_row, const int32_t *chunk_slice,
                           const int32_t *cor, const int64_t *slice_ptr, const int32_t *scol, const int2 *hull,
                           const int64_t *word_off, uint32_t *bits, int symmetric) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = cor[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        const int32_t lo_c = hull[c].x;
        auto set = [&](int32_t owner, int32_t owner_lo, int32_t target) {
            const int32_t off = target - owner_lo;
            atomicOr(&bits[word_off[owner] + (off >> 5)], 1u << (off & 31));
        };
        set(c, lo_c, c);
        int32_t last = -1;
        for (int32_t j = 0; j < rowlen[r]; ++j) {
            const int32_t cc = cor[scol[base + 32 * (int64_t)j]];
            if (cc == last) continue;
            last = cc;
            set(c, lo_c, cc);
            if (!symmetric) set(cc, hull[cc].x, c);
        }
    }
}

// Compresses each chunk's bitmap into at most kDepRanges ranges of chunk indices: maximal
// runs of set bits, then the runs separated by the smallest gaps are merged.  Chunks with
// more than 64 runs fall back to their hull.  Empty ranges are (0, -1).
__global__ void k_dep_ranges(int32_t nchunks, const int2 *hull, const int64_t *word_off, const uint32_t *bits,
                             int4 *ranges) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
        const int32_t lo = hull[c].x, hi = hull[c].y;
        const int64_t w0 = word_off[c];
        const int32_t nb = hi - lo + 1;
        int32_t rs[64], re[64];
        int nr = 0;
        bool overflow = false;
        int32_t run_start = -1;
        for (int32_t b = 0; b < nb && !overflow; ++b) {
            const bool on = (bits[w0 + (b >> 5)] >> (b & 31)) & 1u;
            if (on && run_start < 0) run_start = b;
            if (!on && run_start >= 0) {
                if (nr == 64) overflow = true;
                else { rs[nr] = lo + run_start; re[nr] = lo + b - 1; ++nr; }
                run_start = -1;
            }
        }
        if (!overflow && run_start >= 0) {
            if (nr == 64) overflow = true;
            else { rs[nr] = lo + run_start; re[nr] = hi; ++nr; }
        }
        if (overflow || nr == 0) {
            nr = 1;
            rs[0] = lo;
            re[0] = hi;
        }
        while (nr > kDepRanges) {  // merge the pair of neighbouring runs with the smallest gap
            int best = 0;
            for (int q = 1; q + 1 < nr; ++q)
                if (rs[q + 1] - re[q] < rs[best + 1] - re[best]) best = q;
            re[best] = re[best + 1];
            for (int q = best + 1; q + 1 < nr; ++q) {
                rs[q] = rs[q + 1];
                re[q] = re[q + 1];
            }
            --nr;
        }
        int32_t out[2 * kDepRanges];
        for (int q = 0; q < kDepRanges; ++q) {
            out[2 * q] = q < nr ? rs[q] : 0;
            out[2 * q + 1] = q < nr ? re[q] : -1;
        }
        ranges[2 * c] = make_int4(out[0], out[1], out[2], out[3]);
        ranges[2 * c + 1] = make_int4(out[4], out[5], out[6], out[7]);
    }
}

// Input-row windows of shape 3: for chunk c and its dependency range q, the smallest and the
// largest column (plan numbering) that a row of c reads from the chunks of range q.  The
// ranges are disjoint and cover every chunk that c reads, so the windows are disjoint and
// hold every column of c.  xw[kXWin * c + q] = (min, max), (INT_MAX, -1) when c reads none.
__global__ void k_xwin(int32_t n, const int32_t *rowlen, const int32_t *chunk_row, const int32_t *chunk_slice,
                       const int32_t *cor, const int64_t *slice_ptr, const int32_t *scol, const int4 *ranges,
                       int2 *xw) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = cor[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        const int4 r0 = ranges[2 * c], r1 = ranges[2 * c + 1];
        const int32_t rlo[kXWin] = {r0.x, r0.z, r1.x, r1.z}, rhi[kXWin] = {r0.y, r0.w, r1.y, r1.w};
        int32_t mn[kXWin], mx[kXWin];
        for (int q = 0; q < kXWin; ++q) {
            mn[q] = INT_MAX;
            mx[q] = -1;
        }
        for (int32_t j = 0; j < rowlen[r]; ++j) {
            const int32_t col = scol[base + 32 * (int64_t)j];
            const int32_t cc = cor[col];
            for (int q = 0; q < kXWin; ++q)
                if (cc >= rlo[q] && cc <= rhi[q]) {
                    mn[q] = min(mn[q], col);
                    mx[q] = max(mx[q], col);
                    break;
                }
        }
        for (int q = 0; q < kXWin; ++q)
            if (mx[q] >= 0) {
                atomicMin(&xw[kXWin * c + q].x, mn[q]);
                atomicMax(&xw[kXWin * c + q].y, mx[q]);
            }
    }
}

// 16-bit position of every entry's column in its chunk's window area: the window q holding
// the column (win[3 kXWin c + 3q ..] = first row, rows, position in rows) gives
// position + column - first row.  Padding keeps 0xffff.
__global__ void k_lcol(int32_t n, const int32_t *rowlen, const int32_t *chunk_row, const int32_t *chunk_slice,
                       const int32_t *cor, const int64_t *slice_ptr, const int32_t *scol, const int32_t *win,
                       uint16_t *lcol) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = cor[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        const int32_t *w = win + 3 * kXWin * (int64_t)c;
        for (int32_t j = 0; j < rowlen[r]; ++j) {
            const int32_t col = scol[base + 32 * (int64_t)j];
            for (int q = 0; q < kXWin; ++q)
                if (w[3 * q + 1] > 0 && col >= w[3 * q] && col < w[3 * q] + w[3 * q + 1]) {
                    lcol[base + 32 * (int64_t)j] = (uint16_t)(w[3 * q + 2] + col - w[3 * q]);
                    break;
                }
        }
    }
}

// One record of kRecInts ints per chunk with everything the kernel's control warp needs:
// [row0, row1, slice0, padded entries, first entry (lo, hi 32 bits), staged, slices,
//  kDepRanges (lo, hi) dependency ranges, slice widths as bytes].  A chunk is staged in
// shared memory when its entries fit a buffer and its widths fit the record.
__global__ void k_chunk_records(int32_t nchunks, const int32_t *chunk_row, const int32_t *chunk_slice,
                                const int64_t *slice_ptr, const int4 *ranges, int32_t stage_entries, const int32_t *win,
                                int32_t max_slices, int32_t *rec) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
        const int32_t sl0 = chunk_slice[c], sl1 = chunk_slice[c + 1], nsl = sl1 - sl0;
        const int64_t e0 = slice_ptr[sl0], e1 = slice_ptr[sl1];
        const int32_t cnt = (int32_t)(e1 - e0);
        const int staged = kStageChunks && cnt > 0 && cnt <= stage_entries && nsl <= max_slices;
        int32_t *o = rec + (int64_t)kRecInts * c;
        o[0] = chunk_row[c];
        o[1] = chunk_row[c + 1];
        o[2] = sl0;
        o[3] = cnt;
        o[4] = (int32_t)(e0 & 0xffffffffLL);
        o[5] = (int32_t)(e0 >> 32);
        o[6] = staged;
        o[7] = nsl;
        const int4 r0 = ranges[2 * c], r1 = ranges[2 * c + 1];
        o[8] = r0.x; o[9] = r0.y; o[10] = r0.z; o[11] = r0.w;
        o[12] = r1.x; o[13] = r1.y; o[14] = r1.z; o[15] = r1.w;
        uint32_t wb[kRecSlicesWide / 4] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (staged)
            for (int32_t q = 0; q < nsl; ++q) {
                const uint32_t w = (uint32_t)((slice_ptr[sl0 + q + 1] - slice_ptr[sl0 + q]) >> 5);
                wb[q >> 2] |= (w & 0xffu) << (8 * (q & 3));
            }
        for (int q = 0; q < 3 * kXWin; ++q) o[kRecWin + q] = win ? win[3 * kXWin * (int64_t)c + q] : 0;
        // widths of slices 0..15, then (shapes without windows) of slices 16..31 over the windows
        for (int q = 0; q < (win ? kRecSlices : kRecSlicesWide) / 4; ++q) o[16 + q] = (int32_t)wb[q];
    }
}

// Unit tables from their Lp-diagram cells: cell i (group g, power k) holds the chunks
// [c0, c0 + nc) of g and starts at slot off[i] of the table; its units are (c << 5) | k in
// chunk order.
__global__ void k_expand_cells(const int64_t *off, const int4 *cell, int32_t ncells, int32_t *units) {
    for (int32_t i = blockIdx.x; i < ncells; i += gridDim.x) {
        const int4 c = cell[i];  // (c0, nc, k, unused)
        const int64_t o = off[i];
        for (int32_t j = threadIdx.x; j < c.y; j += blockDim.x) units[o + j] = ((c.x + j) << 5) | c.z;
    }
}

template <class T> __global__ void k_widen(const T *src, int64_t n, double *dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = widen_value(src[i]);
}

void widen_values(int vtype, const void *src, int64_t n, double *dst, cudaStream_t s) {
    if (n <= 0) return;
    if (vtype == MPK_F64)
        k_widen<double><<<grid_n(n), 256, 0, s>>>(static_cast<const double *>(src), n, dst);
    else if (vtype == MPK_F32)
        k_widen<float><<<grid_n(n), 256, 0, s>>>(static_cast<const float *>(src), n, dst);
    else if (vtype == MPK_BF16)
        k_widen<uint16_t><<<grid_n(n), 256, 0, s>>>(static_cast<const uint16_t *>(src), n, dst);
    else
        fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
    MPK_LAUNCHED();
}

// sliced copy -> CSR (for inspection and tests), values widened to float64
template <class T>
__global__ void k_export(int32_t n, const int32_t *rowlen, const int32_t *chunk_row, const int32_t *chunk_slice,
                         const int32_t *chunk_of_row, const int64_t *slice_ptr, const T *sval,
                         const int32_t *scol, const int32_t *rp, int32_t *ci, double *va) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = chunk_of_row[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        for (int32_t j = 0; j < rowlen[r]; ++j) {
            ci[rp[r] + j] = scol[base + 32 * (int64_t)j];
            va[rp[r] + j] = widen_value(sval[base + 32 * (int64_t)j]);
        }
    }
}

void export_csr(const Plan &P, int32_t *rp, int32_t *ci, double *va, cudaStream_t s) {
    if (!rp || (P.nnz > 0 && (!ci || !va))) fail(MPK_ERR_INVALID, "NULL output array");
    exclusive_scan(P.rowlen, rp, P.n, s);
    if (P.n == 0) return;
    Tmp<int32_t> cor(P.n, s);
    k_chunk_of_row<<<grid_n(P.num_chunks * 256), 256, 0, s>>>(P.chunk_row, P.num_chunks, cor.p);
    MPK_LAUNCHED();
#define EXPORT(T)                                                                                              \
    k_export<T><<<grid_n(P.n), 256, 0, s>>>(P.n, P.rowlen, P.chunk_row, P.chunk_slice, cor.p, P.slice_ptr, \
                                            static_cast<const T *>(P.val), P.col, rp, ci, va)
    if (P.val_type == MPK_F64)
        EXPORT(double);
    else if (P.val_type == MPK_F32)
        EXPORT(float);
    else
        EXPORT(uint16_t);
#undef EXPORT
    MPK_LAUNCHED();
    MPK_CUDA(cudaStreamSynchronize(s));
}

Plan *build_plan(const mpk_csr *A, const Levels *L, const mpk_plan_opts *o, cudaStream_t s,
                 const std::vector<int32_t> *inst_row, const std::vector<int32_t> *inst_p) {
    if (!o) fail(MPK_ERR_INVALID, "options are NULL");
    validate_csr(A, s);
    if (o->p_max < 1 || o->p_max > kMaxP) fail(MPK_ERR_INVALID, "p_max must be in [1, %d]", kMaxP);
    if (!(o->nrhs == 1 || o->nrhs == 2 || o->nrhs == 4 || o->nrhs == 8 || o->nrhs == 16))
        fail(MPK_ERR_UNSUPPORTED, "nrhs must be 1, 2, 4, 8 or 16 (got %d)", o->nrhs);
    // 16 right-hand sides: a row's 16 x values and sums need the registers of the unstaged
    // shape at one block per SM; the staged shapes and the warp engine would spill
    if (o->nrhs == 16 && ((o->shape > 0 && o->shape != 3) || o->engine == MPK_ENGINE_WARP))
        fail(MPK_ERR_UNSUPPORTED, "16 right-hand sides run on the unstaged block shape (plan option shape 0 or 3) "
                                  "of the staged or the sweep engine");
    if (o->order != MPK_ORDER_ORIGINAL && o->order != MPK_ORDER_PLAN) fail(MPK_ERR_INVALID, "bad order");
    int32_t chunk_rows = o->chunk_rows;  // 0: 32 rows per compute warp of the block shape
    if (chunk_rows != 0 && (chunk_rows < 32 || chunk_rows > 8192 || chunk_rows % 32))
        fail(MPK_ERR_INVALID, "chunk_rows must be a multiple of 32 in [32, 8192]");
    if (o->cache_bytes < 0 || o->mem_budget < 0 || o->wait_limit_ns < 0) fail(MPK_ERR_INVALID, "negative option");
    if (L && L->n != A->n) fail(MPK_ERR_INVALID, "levels were built for n = %d, matrix has n = %d", L->n, A->n);

    const int32_t n = A->n, m = o->nrhs, pmax = o->p_max;
    Plan *P = new Plan();
    try {
        P->arena.budget = o->mem_budget;
        P->n = n;
        P->nnz = A->nnz;
        P->m = m;
        P->p_max = pmax;
        P->val_type = A->val_type;
        P->val_bytes = A->val_type == MPK_F64 ? 8 : (A->val_type == MPK_F32 ? 4 : 2);
        // binary32 accumulation: values stored in float32 or bfloat16 (exact in binary32), the
        // staged or sweep engine, single plans
        if (o->accum != MPK_F64 && o->accum != MPK_F32) fail(MPK_ERR_INVALID, "accum must be MPK_F64 or MPK_F32");
        P->accum = o->accum;
        if (P->accum == MPK_F32) {
            if (A->val_type == MPK_F64)
                fail(MPK_ERR_UNSUPPORTED, "binary32 accumulation needs values stored as float32 or bfloat16");
            if (o->engine == MPK_ENGINE_WARP || o->trace || o->level_capped || inst_row != nullptr ||
                o->shape - 1 == kShapeX)
                fail(MPK_ERR_UNSUPPORTED,
                     "binary32 accumulation runs on the staged engine (any shape but the X-staged one) or the "
                     "sweep engine, without trace, level caps or batching");
        }
        P->order = o->order;
        P->identity = (L == nullptr);
        P->chunk_rows = chunk_rows;
        // Units of two slices a warp (block shape 4) are the planner's choice for binary32 sums
        // over 2-byte values, one right-hand side and short rows (decided here from the mean row
        // length, since the budget shapes the groups the slices are cut from); they want larger
        // groups: measured at 256^3, p = 8, 1.575 / 1.486 / 1.459 / 1.468 ms at C = 96 / 128 /
        // 160 / 192 MB.  Every other plan: three quarters of L2.
        const bool two_slices = o->shape == 5 || (o->shape == 0 && o->accum == MPK_F32 && P->val_bytes == 2 &&
                                                  o->nrhs == 1 && A->nnz <= 10 * (int64_t)A->n);
        P->cache_bytes = o->cache_bytes ? o->cache_bytes : device_l2_bytes() / 4 * (two_slices ? 5 : 3);
        P->window = kSlotSkew * pmax + 1;
        P->group_budget = P->cache_bytes / P->window;
        P->wait_ns = o->wait_limit_ns ? o->wait_limit_ns : 2000000000LL;
        P->num_levels = L ? L->num_levels : 0;
        const bool batch = inst_row != nullptr;
        P->level_capped = o->level_capped != 0;
        if (P->level_capped && (!L || batch || o->order != MPK_ORDER_PLAN))
            fail(MPK_ERR_INVALID, "level_capped needs levels, plan order and no batch");
        P->split_levels = o->split_levels != 0;
        if (P->split_levels && (!L || batch || P->level_capped || o->engine == MPK_ENGINE_WARP))
            fail(MPK_ERR_INVALID, "split_levels needs levels and the staged or sweep engine, without level caps or "
                                  "batching");
        if (batch) {
            if (!L || !inst_p || inst_row->size() != inst_p->size() + 1 || inst_row->back() != n)
                fail(MPK_ERR_INVALID, "inconsistent batch description");
            P->inst_row = *inst_row;
            P->inst_p = *inst_p;
        }

        // ---- permutation (plan-owned copies)
        if (!P->identity && n > 0) {
            P->perm = P->arena.alloc_n<int32_t>(n);
            P->iperm = P->arena.alloc_n<int32_t>(n);
            MPK_CUDA(cudaMemcpyAsync(P->perm, L->perm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            MPK_CUDA(cudaMemcpyAsync(P->iperm, L->iperm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        }
        P->rowlen = P->arena.alloc_n<int32_t>(n > 0 ? n : 1);
        if (n > 0) {
            k_rowlen<<<grid_n(n), 256, 0, s>>>(n, A->row_ptr, P->perm, P->rowlen);
            MPK_LAUNCHED();
        }

        // ---- groups: greedy rule over levels (host), identical to the written rule
        std::vector<int32_t> g_level, g_row;
        if (P->identity) {
            g_row = {0, n};
        } else if (n > 0) {
            const int32_t NL = L->num_levels;
            Tmp<int32_t> prp((int64_t)n + 1, s);
            exclusive_scan(P->rowlen, prp.p, n, s);
            Tmp<int32_t> lvl_nnz((int64_t)NL + 1, s);
            k_gather_i32<<<grid_n(NL + 1), 256, 0, s>>>(prp.p, L->level_ptr, NL + 1, lvl_nnz.p);
            MPK_LAUNCHED();
            std::vector<int32_t> h_nz((size_t)NL + 1);
            MPK_CUDA(cudaMemcpyAsync(h_nz.data(), lvl_nnz.p, sizeof(int32_t) * ((size_t)NL + 1),
                                     cudaMemcpyDeviceToHost, s));
            MPK_CUDA(cudaStreamSynchronize(s));
            const std::vector<int32_t> &lp = L->h_level_ptr;
            const int64_t B = P->group_budget;
            const int64_t vb = P->val_bytes;  // value bytes of the stored type
            // batch plans: a group never holds levels of two instances (every instance is a
            // union of components, numbered after the previous one, so it starts a level)
            std::vector<char> inst_start((size_t)NL, 0);
            if (batch) {
                for (size_t i = 0; i + 1 < P->inst_row.size(); ++i) {
                    if (P->inst_row[i + 1] == P->inst_row[i]) continue;  // empty instance
                    const auto it = std::lower_bound(lp.begin(), lp.begin() + NL, P->inst_row[i]);
                    if (it == lp.begin() + NL || *it != P->inst_row[i])
                        fail(MPK_ERR_INVALID, "instance %zu does not start a level", i);
                    inst_start[it - lp.begin()] = 1;
                }
            }
            int64_t cur = 0, Bl = B;
            size_t inst = 0;
            g_level.push_back(0);
            for (int32_t l = 0; l < NL; ++l) {
                if (batch) {  // each block's groups share the cache with its own window only
                    while (inst + 1 < P->inst_p.size() && lp[l] >= P->inst_row[inst + 1]) ++inst;
                    Bl = P->cache_bytes / (kSlotSkew * P->inst_p[inst] + 1);
                }
                const int64_t rows = lp[l + 1] - lp[l];
                const int64_t nz = (int64_t)h_nz[l + 1] - h_nz[l];
                const int64_t b = (vb + 4) * nz + 4 * rows + 16 * (int64_t)m * rows;
                // level-capped plans: every level below p_max is a group of its own
                const bool cut = P->level_capped && l <= pmax;
                if (l > 0 && !inst_start[l] && !cut && cur + b <= Bl) {
                    cur += b;
                } else {
                    if (l > 0) g_level.push_back(l);
                    cur = b;
                }
            }
            g_level.push_back(NL);
            if (P->level_capped && NL > 0) P->level0_rows = lp[1];
            for (int32_t gl : g_level) g_row.push_back(lp[gl]);
            if (P->split_levels) {
                // Bulky levels split (the recursion stage of Sec. 6, read as breaking a level too
                // large for the budget into pieces): levels group as above while they fit; a level
                // over the budget closes the current group and is cut into pieces of consecutive
                // rows, each taking rows while its bytes stay <= budget (at least one row), each a
                // group; the next level starts a new group.  A row costs (val_bytes + 4) nnz + 4 +
                // 16 m bytes.  group_level_ptr then holds the level of each group's first row.
                std::vector<int32_t> rl((size_t)n), prow((size_t)n + 1);
                MPK_CUDA(cudaMemcpyAsync(rl.data(), P->rowlen, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
                MPK_CUDA(cudaStreamSynchronize(s));
                g_row.assign(1, 0);
                g_level.assign(1, 0);
                int64_t cur2 = 0;
                for (int32_t l = 0; l < NL; ++l) {
                    const int64_t rows = lp[l + 1] - lp[l];
                    const int64_t nz = (int64_t)h_nz[l + 1] - h_nz[l];
                    const int64_t b = (vb + 4) * nz + 4 * rows + 16 * (int64_t)m * rows;
                    if (b > B) {
                        if (l > 0 && g_row.back() != lp[l]) {
                            g_row.push_back(lp[l]);
                            g_level.push_back(l);
                        }
                        int64_t piece = 0;
                        for (int32_t r = lp[l]; r < lp[l + 1]; ++r) {
                            const int64_t rb = (vb + 4) * rl[r] + 4 + 16 * (int64_t)m;
                            if (r > lp[l] && piece + rb > B) {
                                g_row.push_back(r);
                                g_level.push_back(l);
                                piece = 0;
                            }
                            piece += rb;
                        }
                        if (l + 1 < NL) {
                            g_row.push_back(lp[l + 1]);
                            g_level.push_back(l + 1);
                        }
                        cur2 = 0;
                        continue;
                    }
                    if (l > 0 && g_row.back() == lp[l]) {
                        cur2 = b;
                    } else if (l > 0 && cur2 + b <= B) {
                        cur2 += b;
                    } else {
                        if (l > 0) {
                            g_row.push_back(lp[l]);
                            g_level.push_back(l);
                        }
                        cur2 = b;
                    }
                }
                g_row.push_back(lp[NL]);
                g_level.push_back(NL);
            }
        } else {
            g_row = {0, 0};
        }
        const int32_t G = (int32_t)g_row.size() - 1;
        P->num_groups = G;

        // ---- slices: 32-row blocks counted from each group's first row (host)
        std::vector<int32_t> s_row;
        s_row.push_back(0);
        std::vector<int32_t> g_slice;
        for (int32_t g = 0; g < G; ++g) {
            g_slice.push_back((int32_t)s_row.size() - 1);
            for (int32_t r = g_row[g]; r < g_row[g + 1]; r += 32) s_row.push_back(std::min(r + 32, g_row[g + 1]));
        }
        g_slice.push_back((int32_t)s_row.size() - 1);
        const int32_t NS = (int32_t)s_row.size() - 1;
        P->num_slices = NS;
        Tmp<int32_t> d_srow((int64_t)NS + 1, s);
        Tmp<int32_t> d_width(NS, s);
        MPK_CUDA(cudaMemcpyAsync(d_srow.p, s_row.data(), sizeof(int32_t) * ((size_t)NS + 1), cudaMemcpyHostToDevice, s));
        if (NS > 0) {
            k_slice_width<<<grid_n(NS), 256, 0, s>>>(d_srow.p, NS, P->rowlen, d_width.p);
            MPK_LAUNCHED();
        }
        std::vector<int32_t> width((size_t)NS);
        if (NS > 0)
            MPK_CUDA(cudaMemcpyAsync(width.data(), d_width.p, sizeof(int32_t) * (size_t)NS, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> sptr((size_t)NS + 1, 0);
        for (int32_t i = 0; i < NS; ++i) sptr[i + 1] = sptr[i] + 32 * (int64_t)width[i];
        P->padded = sptr[NS];

        // ---- block shape: shape 1 when its slot holds at least 6 slices of the mean
        //      width, else unstaged (measured: 27-point stencils run 1.7x
        //      faster unstaged).  Shape 1's fewer, larger units beat shape 0 on the 3-D
        //      Laplacian (2.20 ms against 2.58 ms at 256^3, p = 8), since the per-unit work of
        //      the control warp sets the pace; for the same reason binary32 sums over 2-byte
        //      values take shape 4 (two slices a warp) when its slot holds 24 slices of the
        //      mean width (1.459 against 1.622 ms at their best budgets); shapes 0 and 3 (input
        //      rows staged too) are taken only when the options name them.
        if (o->shape < 0 || o->shape > kNumShapes) fail(MPK_ERR_INVALID, "shape must be in [0, %d]", kNumShapes);
        int fallback_shape = 0;
        bool try_x = false;
        if (o->shape > 0) {
            fallback_shape = o->shape - 1;
            try_x = fallback_shape == kShapeX;
        } else {
            auto fits = [&](int sh, int slices) {
                return (int64_t)slices * P->padded <= (int64_t)kShapes[sh].stage_entries * std::max(NS, 1);
            };
            fallback_shape = (o->nrhs < 16 && fits(1, 6)) ? 1 : 2;  // up to 24 entries a row on average
            if (two_slices && fits(4, 24)) fallback_shape = 4;      // up to 12 entries a row
            try_x = false;
        }
        const bool x_forced = o->shape - 1 == kShapeX;

        // ---- sliced copy and group tables (independent of the chunks)
        P->group_row_ptr = P->arena.alloc_n<int32_t>(G + 1);
        MPK_CUDA(cudaMemcpyAsync(P->group_row_ptr, g_row.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s));
        if (!P->identity) {
            P->group_level_ptr = P->arena.alloc_n<int32_t>(G + 1);
            MPK_CUDA(cudaMemcpyAsync(P->group_level_ptr, g_level.data(), sizeof(int32_t) * (G + 1),
                                     cudaMemcpyHostToDevice, s));
        }
        P->slice_ptr = P->arena.alloc_n<int64_t>((int64_t)NS + 1);
        MPK_CUDA(cudaMemcpyAsync(P->slice_ptr, sptr.data(), sizeof(int64_t) * ((size_t)NS + 1), cudaMemcpyHostToDevice, s));
        Tmp<int32_t> cor(n, s);
        P->val = P->arena.alloc((P->padded + 32) * P->val_bytes);
        P->col = P->arena.alloc_n<int32_t>(P->padded + 32);
        MPK_CUDA(cudaMemsetAsync(P->val, 0, (size_t)P->val_bytes * (size_t)(P->padded + 32), s));  // +0 in every type
        MPK_CUDA(cudaMemsetAsync(P->col, 0xff, sizeof(int32_t) * (size_t)(P->padded + 32), s));  // padding: col = -1

        std::vector<int32_t> c_row, c_slice, g_chunk;
        std::vector<int32_t> h_win;  // shape 3: kXWin (first row, rows, position) per chunk
        int32_t NC = 0, stage_entries = 0;
        for (int attempt = 0;; ++attempt) {
            P->shape = (attempt == 0 && try_x) ? kShapeX : fallback_shape;
            if (attempt > 0 && P->shape == kShapeX) fail(MPK_ERR_UNSUPPORTED, "block shape 3 does not fit this plan");
            stage_entries = kShapes[P->shape].stage_entries;
            const int64_t chunk_entries = stage_entries > 0 ? stage_entries : INT64_MAX;
            chunk_rows = o->chunk_rows ? o->chunk_rows
                                       : 32 * kShapes[P->shape].comp_warps * std::max(1, kShapes[P->shape].slices_per_warp);
            P->chunk_rows = chunk_rows;

            // ---- chunks: consecutive slices of one group, at most chunk_rows rows and at most
            //      stage_entries padded entries (a single wider slice forms its own chunk)
            c_row.assign(1, 0);
            c_slice.assign(1, 0);
            g_chunk.clear();
            for (int32_t g = 0; g < G; ++g) {
                g_chunk.push_back((int32_t)c_row.size() - 1);
                int32_t s0 = g_slice[g];
                while (s0 < g_slice[g + 1]) {
                    int32_t s1 = s0 + 1;
                    while (s1 < g_slice[g + 1] && s_row[s1 + 1] - s_row[s0] <= chunk_rows &&
                           sptr[s1 + 1] - sptr[s0] <= chunk_entries)
                        ++s1;
                    c_row.push_back(s_row[s1]);
                    c_slice.push_back(s1);
                    s0 = s1;
                }
            }
            g_chunk.push_back((int32_t)c_row.size() - 1);
            NC = (int32_t)c_row.size() - 1;
            P->h_chunk_row = c_row;
            if (NC >= (1 << 26)) fail(MPK_ERR_TOO_LARGE, "too many chunks (%d)", NC);
            P->num_chunks = NC;
            P->chunk_row = P->arena.alloc_n<int32_t>(NC + 1);
            P->chunk_slice = P->arena.alloc_n<int32_t>(NC + 1);
            MPK_CUDA(cudaMemcpyAsync(P->chunk_row, c_row.data(), sizeof(int32_t) * (NC + 1), cudaMemcpyHostToDevice, s));
            MPK_CUDA(cudaMemcpyAsync(P->chunk_slice, c_slice.data(), sizeof(int32_t) * (NC + 1), cudaMemcpyHostToDevice,
                                     s));

            // ---- fill the sliced copy; dependency hulls of the chunks
            P->dep = P->arena.alloc_n<int2>(NC > 0 ? NC : 1);
            if (NC > 0) {
                k_dep_init<<<grid_n(NC), 256, 0, s>>>(P->dep, NC);
                MPK_LAUNCHED();
                k_chunk_of_row<<<grid_n((int64_t)NC * 256), 256, 0, s>>>(P->chunk_row, NC, cor.p);
                MPK_LAUNCHED();
#define FILL(T)                                                                                            \
    k_fill<T><<<grid_n(n), 256, 0, s>>>(n, A->row_ptr, A->col, static_cast<const T *>(A->val), P->perm,    \
                                        P->iperm, P->chunk_row, P->chunk_slice, cor.p, P->slice_ptr,         \
                                        static_cast<T *>(P->val), P->col, P->dep, A->is_symmetric ? 1 : 0, special.p)
                Tmp<int32_t> special(1, s);
                MPK_CUDA(cudaMemsetAsync(special.p, 0, sizeof(int32_t), s));
                if (P->val_type == MPK_F64)
                    FILL(double);
                else if (P->val_type == MPK_F32)
                    FILL(float);
                else
                    FILL(uint16_t);
#undef FILL
                MPK_LAUNCHED();
                int32_t has_special = 0;
                MPK_CUDA(cudaMemcpyAsync(&has_special, special.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                MPK_CUDA(cudaStreamSynchronize(s));
                if (has_special)
                    fail(MPK_ERR_UNSUPPORTED,
                         "float32/bfloat16 storage holds zeros and normal numbers only (a value is subnormal, "
                         "infinite or NaN in the narrow type): use MPK_F64 values");
            }
            // ---- dependency ranges: exact chunk sets as bitmaps over each hull, compressed
            P->dep_ranges = P->arena.alloc_n<int4>(2 * (int64_t)(NC > 0 ? NC : 1));
            if (NC > 0) {
                std::vector<int2> hull((size_t)NC);
                MPK_CUDA(cudaMemcpyAsync(hull.data(), P->dep, sizeof(int2) * (size_t)NC, cudaMemcpyDeviceToHost, s));
                MPK_CUDA(cudaStreamSynchronize(s));
                std::vector<int64_t> woff((size_t)NC + 1, 0);
                for (int32_t c = 0; c < NC; ++c) woff[c + 1] = woff[c] + (hull[c].y - hull[c].x + 32) / 32;
                const int64_t words = woff[NC];
                if (words <= ((int64_t)1 << 27)) {
                    Tmp<int64_t> d_woff((int64_t)NC + 1, s);
                    Tmp<uint32_t> d_bits(words, s);
                    MPK_CUDA(cudaMemcpyAsync(d_woff.p, woff.data(), sizeof(int64_t) * ((size_t)NC + 1),
                                             cudaMemcpyHostToDevice, s));
                    MPK_CUDA(cudaMemsetAsync(d_bits.p, 0, sizeof(uint32_t) * (size_t)words, s));
                    k_dep_bits<<<grid_n(n), 256, 0, s>>>(n, P->rowlen, P->chunk_row, P->chunk_slice, cor.p,
                                                         P->slice_ptr, P->col, P->dep, d_woff.p, d_bits.p,
                                                         A->is_symmetric ? 1 : 0);
                    MPK_LAUNCHED();
                    k_dep_ranges<<<grid_n(NC), 256, 0, s>>>(NC, P->dep, d_woff.p, d_bits.p, P->dep_ranges);
                    MPK_LAUNCHED();
                    MPK_CUDA(cudaStreamSynchronize(s));
                } else {  // bitmaps too large: one range per chunk, the hull
                    std::vector<int4> rr((size_t)2 * NC);
                    for (int32_t c = 0; c < NC; ++c) {
                        rr[2 * c] = make_int4(hull[c].x, hull[c].y, 0, -1);
                        rr[2 * c + 1] = make_int4(0, -1, 0, -1);
                    }
                    MPK_CUDA(cudaMemcpyAsync(P->dep_ranges, rr.data(), sizeof(int4) * rr.size(), cudaMemcpyHostToDevice,
                                             s));
                    MPK_CUDA(cudaStreamSynchronize(s));
                }
            }
            // ---- shape 3: input-row windows per chunk, laid out in the slot's window area
            //      (rows from position 1 on, a gap of 2 / nrhs rows between windows, positions
            //      of the parity of the first row when nrhs = 1; see x_copy in the kernel)
            if (P->shape == kShapeX) {
                bool ok = NC > 0;
                h_win.assign((size_t)3 * kXWin * std::max(NC, 1), 0);
                if (ok) {
                    Tmp<int2> d_xw((int64_t)kXWin * NC, s);
                    std::vector<int2> xw((size_t)kXWin * NC, make_int2(INT_MAX, -1));
                    MPK_CUDA(cudaMemcpyAsync(d_xw.p, xw.data(), sizeof(int2) * xw.size(), cudaMemcpyHostToDevice, s));
                    k_xwin<<<grid_n(n), 256, 0, s>>>(n, P->rowlen, P->chunk_row, P->chunk_slice, cor.p, P->slice_ptr,
                                                     P->col, P->dep_ranges, d_xw.p);
                    MPK_LAUNCHED();
                    MPK_CUDA(cudaMemcpyAsync(xw.data(), d_xw.p, sizeof(int2) * xw.size(), cudaMemcpyDeviceToHost, s));
                    MPK_CUDA(cudaStreamSynchronize(s));
                    const int64_t XW = kShapes[kShapeX].x_words;
                    for (int32_t c = 0; c < NC && ok; ++c) {
                        // every chunk must be staged: its entries fit the slot and its widths the record
                        if (c_slice[c + 1] - c_slice[c] > kRecSlices ||
                            sptr[c_slice[c + 1]] - sptr[c_slice[c]] > stage_entries)
                            ok = false;
                        int64_t pos = 1;
                        for (int q = 0; q < kXWin && ok; ++q) {
                            const int2 w = xw[(size_t)kXWin * c + q];
                            if (w.y < w.x) continue;
                            const int64_t len = (int64_t)w.y - w.x + 1;
                            if (m == 1 && ((pos ^ w.x) & 1)) ++pos;
                            if (m * (pos + len) + 2 > XW) {
                                ok = false;
                                break;
                            }
                            int32_t *hw = &h_win[(size_t)3 * kXWin * c + 3 * q];
                            hw[0] = w.x;
                            hw[1] = (int32_t)len;
                            hw[2] = (int32_t)pos;
                            pos += len + (m == 1 ? 2 : 1);
                        }
                    }
                }
                if (!ok) {
                    if (x_forced)
                        fail(MPK_ERR_UNSUPPORTED,
                             "block shape 3: a chunk's input rows do not fit a staging slot (fewer chunk_rows, or "
                             "another shape)");
                    P->arena.free(P->chunk_row);
                    P->arena.free(P->chunk_slice);
                    P->arena.free(P->dep);
                    P->arena.free(P->dep_ranges);
                    P->chunk_row = P->chunk_slice = nullptr;
                    P->dep = nullptr;
                    P->dep_ranges = nullptr;
                    h_win.clear();
                    continue;
                }
                Tmp<int32_t> d_win((int64_t)h_win.size(), s);
                MPK_CUDA(cudaMemcpyAsync(d_win.p, h_win.data(), sizeof(int32_t) * h_win.size(), cudaMemcpyHostToDevice,
                                         s));
                P->lcol = P->arena.alloc_n<uint16_t>(P->padded + 32);
                MPK_CUDA(cudaMemsetAsync(P->lcol, 0xff, sizeof(uint16_t) * (size_t)(P->padded + 32), s));
                k_lcol<<<grid_n(n), 256, 0, s>>>(n, P->rowlen, P->chunk_row, P->chunk_slice, cor.p, P->slice_ptr,
                                                 P->col, d_win.p, P->lcol);
                MPK_LAUNCHED();
                MPK_CUDA(cudaStreamSynchronize(s));  // d_win goes out of scope
            }
            break;
        }

        P->chunk_rec = reinterpret_cast<int4 *>(P->arena.alloc_n<int32_t>((int64_t)kRecInts * (NC > 0 ? NC : 1)));
        if (NC > 0) {
            Tmp<int32_t> d_win(P->shape == kShapeX ? (int64_t)h_win.size() : 0, s);
            if (P->shape == kShapeX)
                MPK_CUDA(cudaMemcpyAsync(d_win.p, h_win.data(), sizeof(int32_t) * h_win.size(), cudaMemcpyHostToDevice,
                                         s));
            k_chunk_records<<<grid_n(NC), 256, 0, s>>>(NC, P->chunk_row, P->chunk_slice, P->slice_ptr, P->dep_ranges,
                                                      stage_entries, d_win.p,
                                                      // slices a staged chunk may have: what the shape's
                                                      // compute warps read widths for
                                                      kShapes[P->shape].slices_per_warp > 1 ? kRecSlicesWide : kRecSlices,
                                                      reinterpret_cast<int32_t *>(P->chunk_rec));
            MPK_LAUNCHED();
            MPK_CUDA(cudaStreamSynchronize(s));
        }

        // ---- unit tables: Lp-diagram cells (group g, power k) along lines g + kSlotSkew*k
        //      ascending, k ascending inside a line, chunks in row order; unit = chunk << 5 | k
        P->unit_off.assign((size_t)pmax + 2, 0);
        std::vector<int32_t> units;
        if (batch) {
            // one table: every instance's cells up to its own power, instance after instance;
            // blocks claim the next instance's first units while the previous one drains, and
            // about one instance at a time holds the cache.  Each instance keeps its own order,
            // so dependencies keep smaller tickets.
            const int32_t NI = (int32_t)P->inst_p.size();
            std::vector<int32_t> gi0((size_t)NI), gi1((size_t)NI);
            int32_t dmax = 0;
            for (int32_t i = 0; i < NI; ++i) {
                gi0[i] = (int32_t)(std::lower_bound(g_row.begin(), g_row.end() - 1, P->inst_row[i]) - g_row.begin());
                gi1[i] = (int32_t)(std::lower_bound(g_row.begin(), g_row.end() - 1, P->inst_row[i + 1]) - g_row.begin());
                if (P->inst_row[i + 1] == n) gi1[i] = G;
                const int32_t pi = P->inst_p[i];
                if (pi < 1 || pi > pmax) fail(MPK_ERR_INVALID, "instance %d: p = %d outside [1, p_max]", i, pi);
                if (gi1[i] > gi0[i]) dmax = std::max(dmax, gi1[i] - gi0[i] - 1 + kSlotSkew * pi);
            }
            for (int32_t i = 0; i < NI; ++i)
                for (int32_t d = kSlotSkew; d <= dmax; ++d)
                    for (int32_t k = 1; k <= P->inst_p[i]; ++k) {
                        const int32_t g = gi0[i] + d - kSlotSkew * k;
                        if (g < gi0[i] || g >= gi1[i]) continue;
                        for (int32_t c = g_chunk[g]; c < g_chunk[g + 1]; ++c) units.push_back((c << 5) | k);
                    }
            P->unit_off[pmax + 1] = (int64_t)units.size();  // the table of p = p_max is the batch table
        }
        // level-capped plans: group g (a single level below p_max, or levels >= p_max) takes
        // powers up to its first level
        std::vector<int32_t> g_cap((size_t)G, pmax);
        if (P->level_capped)
            for (int32_t g = 0; g < G; ++g) g_cap[g] = std::min(pmax, g_level[g]);
        // race-detection aid: shuffle_seed != 0 permutes the units of every line (all their
        // dependencies lie on earlier lines, so any order inside a line is a valid schedule and
        // must give the same bits); splitmix64 drives a Fisher-Yates shuffle
        uint64_t rng = (uint64_t)o->shuffle_seed;
        auto next_rand = [&rng]() {
            uint64_t z = (rng += 0x9e3779b97f4a7c15ULL);
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
            return z ^ (z >> 31);
        };
        // split plans: the groups of a split level need not read only their neighbours, so the
        // units follow waves computed from the exact chunk dependencies: w(c, 1) = kSlotSkew + g(c),
        // w(c, k) = max{ w(c', k-1) : c' in the dependency ranges of c } + 2, units by increasing
        // (w, k, chunk).  Every dependency has a smaller wave, hence a smaller ticket: the
        // schedule stays deadlock free.  (For unsplit levels this reproduces the lines g + 3k.)
        std::vector<int64_t> wave;  // wave of unit (c, k) at (k - 1) * NC + c
        if (P->split_levels && NC > 0) {
            std::vector<int4> rr((size_t)2 * NC);
            MPK_CUDA(cudaMemcpyAsync(rr.data(), P->dep_ranges, sizeof(int4) * rr.size(), cudaMemcpyDeviceToHost, s));
            MPK_CUDA(cudaStreamSynchronize(s));
            wave.assign((size_t)pmax * NC, 0);
            for (int32_t g = 0; g < G; ++g)
                for (int32_t c = g_chunk[g]; c < g_chunk[g + 1]; ++c) wave[c] = kSlotSkew + g;
            int lg = 1;
            while ((1 << lg) < NC) ++lg;
            std::vector<int64_t> st((size_t)(lg + 1) * NC);  // sparse table of range maxima
            for (int32_t k = 2; k <= pmax; ++k) {
                const int64_t *prev = wave.data() + (size_t)(k - 2) * NC;
                for (int32_t c = 0; c < NC; ++c) st[c] = prev[c];
                for (int j = 1; j <= lg; ++j)
                    for (int32_t c = 0; c + (1 << j) <= NC; ++c)
                        st[(size_t)j * NC + c] =
                            std::max(st[(size_t)(j - 1) * NC + c], st[(size_t)(j - 1) * NC + c + (1 << (j - 1))]);
                auto range_max = [&](int32_t a, int32_t b) {  // inclusive, a <= b
                    int j = 0;
                    while ((2 << j) <= b - a + 1) ++j;
                    return std::max(st[(size_t)j * NC + a], st[(size_t)j * NC + b - (1 << j) + 1]);
                };
                int64_t *cur = wave.data() + (size_t)(k - 1) * NC;
                for (int32_t c = 0; c < NC; ++c) {
                    const int32_t lo4[4] = {rr[2 * c].x, rr[2 * c].z, rr[2 * c + 1].x, rr[2 * c + 1].z};
                    const int32_t hi4[4] = {rr[2 * c].y, rr[2 * c].w, rr[2 * c + 1].y, rr[2 * c + 1].w};
                    int64_t mx = 0;
                    for (int q = 0; q < 4; ++q)
                        if (hi4[q] >= lo4[q]) mx = std::max(mx, range_max(lo4[q], hi4[q]));
                    cur[c] = mx + 2;
                }
            }
        }
        for (int32_t p = 1; p <= pmax && !batch && P->split_levels; ++p) {
            P->unit_off[p] = (int64_t)units.size();
            std::vector<std::pair<int64_t, int32_t>> ord;  // (wave, unit)
            ord.reserve((size_t)p * NC);
            for (int32_t k = 1; k <= p; ++k)
                for (int32_t c = 0; c < NC; ++c) ord.push_back({wave[(size_t)(k - 1) * NC + c], (c << 5) | k});
            std::sort(ord.begin(), ord.end(), [](const std::pair<int64_t, int32_t> &x, const std::pair<int64_t, int32_t> &y) {
                if (x.first != y.first) return x.first < y.first;
                if ((x.second & 31) != (y.second & 31)) return (x.second & 31) < (y.second & 31);
                return x.second < y.second;
            });
            for (size_t j = 0; j < ord.size();) {  // one wave at a time (shuffled on request)
                size_t e = j;
                while (e < ord.size() && ord[e].first == ord[j].first) ++e;
                const size_t line0 = units.size();
                for (size_t q = j; q < e; ++q) units.push_back(ord[q].second);
                if (o->shuffle_seed != 0)
                    for (size_t q = units.size() - 1; q > line0; --q)
                        std::swap(units[q], units[line0 + next_rand() % (q - line0 + 1)]);
                j = e;
            }
        }
        // line order without shuffling: the tables are listed as cells (group, power) here and
        // expanded into units on the device (1.2 M units at 256^3, p_max = 8: a host loop and
        // copy took 2.7 ms); the same order as the host loop below
        const bool cells_on_device = !batch && !P->split_levels && o->shuffle_seed == 0;
        std::vector<int64_t> cell_off;
        std::vector<int4> cell;
        int64_t total_units = 0;
        for (int32_t p = 1; p <= pmax && cells_on_device; ++p) {
            P->unit_off[p] = total_units;
            for (int32_t d = kSlotSkew; d <= G - 1 + kSlotSkew * p; ++d)
                for (int32_t k = 1; k <= p; ++k) {
                    const int32_t g = d - kSlotSkew * k;
                    if (g < 0 || g >= G || k > g_cap[g]) continue;
                    const int32_t nc = g_chunk[g + 1] - g_chunk[g];
                    if (nc <= 0) continue;
                    cell_off.push_back(total_units);
                    cell.push_back(make_int4(g_chunk[g], nc, k, 0));
                    total_units += nc;
                }
        }
        for (int32_t p = 1; p <= pmax && !batch && !P->split_levels && !cells_on_device; ++p) {
            P->unit_off[p] = (int64_t)units.size();
            for (int32_t d = kSlotSkew; d <= G - 1 + kSlotSkew * p; ++d) {
                const size_t line0 = units.size();
                for (int32_t k = 1; k <= p; ++k) {
                    const int32_t g = d - kSlotSkew * k;
                    if (g < 0 || g >= G || k > g_cap[g]) continue;
                    for (int32_t c = g_chunk[g]; c < g_chunk[g + 1]; ++c) units.push_back((c << 5) | k);
                }
                if (o->shuffle_seed != 0)
                    for (size_t j = units.size() - 1; j > line0; --j)
                        std::swap(units[j], units[line0 + next_rand() % (j - line0 + 1)]);
            }
        }
        if (!cells_on_device) total_units = (int64_t)units.size();
        if (!batch) P->unit_off[pmax + 1] = total_units;

        // ---- warp-ticketed engine: the same cells in the same order, split into items of
        //      kWarpSlices slices; counters of finished items per cell
        if (o->engine != MPK_ENGINE_STAGED && o->engine != MPK_ENGINE_WARP && o->engine != MPK_ENGINE_SWEEP)
            fail(MPK_ERR_INVALID, "engine must be MPK_ENGINE_STAGED, MPK_ENGINE_WARP or MPK_ENGINE_SWEEP");
        if (o->engine == MPK_ENGINE_SWEEP) {
            if (batch || P->level_capped) fail(MPK_ERR_INVALID, "batch and level-capped plans need level blocking");
            P->engine = MPK_ENGINE_SWEEP;
        }
        if (o->engine == MPK_ENGINE_WARP) {
            if (batch) fail(MPK_ERR_INVALID, "batch plans run on the staged engine");
            P->engine = MPK_ENGINE_WARP;
            std::vector<int64_t> w_item;
            std::vector<int32_t> w_gk;
            P->w_cell_off.assign((size_t)pmax + 2, 0);
            P->w_items.assign((size_t)pmax + 1, 0);
            for (int32_t p = 1; p <= pmax; ++p) {
                P->w_cell_off[p] = (int64_t)w_item.size();
                int64_t items = 0;
                for (int32_t d = kSlotSkew; d <= G - 1 + kSlotSkew * p; ++d)
                    for (int32_t k = 1; k <= p; ++k) {
                        const int32_t g = d - kSlotSkew * k;
                        if (g < 0 || g >= G || k > g_cap[g]) continue;
                        const int32_t ns = g_slice[g + 1] - g_slice[g];
                        if (ns <= 0) continue;
                        w_item.push_back(items);
                        w_gk.push_back((g << 5) | k);
                        items += (ns + kWarpSlices - 1) / kWarpSlices;
                    }
                P->w_items[p] = items;
                if (items >= ((int64_t)1 << 31) * kWarpQueues) fail(MPK_ERR_TOO_LARGE, "too many items");
            }
            P->w_cell_off[pmax + 1] = (int64_t)w_item.size();
            if (G >= (1 << 26)) fail(MPK_ERR_TOO_LARGE, "too many groups for the warp engine");
            P->g_slice = P->arena.alloc_n<int32_t>((int64_t)G + 1);
            MPK_CUDA(cudaMemcpyAsync(P->g_slice, g_slice.data(), sizeof(int32_t) * ((size_t)G + 1),
                                     cudaMemcpyHostToDevice, s));
            P->w_item = P->arena.alloc_n<int64_t>((int64_t)w_item.size() + 1);
            P->w_gk = P->arena.alloc_n<int32_t>((int64_t)w_gk.size() + 1);
            if (!w_item.empty()) {
                MPK_CUDA(cudaMemcpyAsync(P->w_item, w_item.data(), sizeof(int64_t) * w_item.size(),
                                         cudaMemcpyHostToDevice, s));
                MPK_CUDA(cudaMemcpyAsync(P->w_gk, w_gk.data(), sizeof(int32_t) * w_gk.size(), cudaMemcpyHostToDevice,
                                         s));
            }
            // per chunk: its slices, and in bits 24.. the highest power it computes (a power
            // above it never completes, so a dependency on it is void: level-capped plans)
            std::vector<int32_t> s_chunk((size_t)NS + 1, 0), c_nsl((size_t)NC + 1, 0);
            for (int32_t g = 0; g < G; ++g)
                for (int32_t c = g_chunk[g]; c < g_chunk[g + 1]; ++c) {
                    c_nsl[c] = (c_slice[c + 1] - c_slice[c]) | (g_cap[g] << 24);
                    for (int32_t q = c_slice[c]; q < c_slice[c + 1]; ++q) s_chunk[q] = c;
                }
            P->w_slice_chunk = P->arena.alloc_n<int32_t>((int64_t)NS + 1);
            P->w_chunk_nsl = P->arena.alloc_n<int32_t>((int64_t)NC + 1);
            MPK_CUDA(cudaMemcpyAsync(P->w_slice_chunk, s_chunk.data(), sizeof(int32_t) * ((size_t)NS + 1),
                                     cudaMemcpyHostToDevice, s));
            MPK_CUDA(cudaMemcpyAsync(P->w_chunk_nsl, c_nsl.data(), sizeof(int32_t) * ((size_t)NC + 1),
                                     cudaMemcpyHostToDevice, s));
            P->w_cnt = P->arena.alloc_n<int32_t>((int64_t)(pmax + 1) * std::max(NC, 1) + kWarpQueues);
            MPK_CUDA(cudaStreamSynchronize(s));  // host tables go out of scope
        }
        P->units = P->arena.alloc_n<int32_t>(total_units + 1);
        if (cells_on_device && !cell.empty()) {
            const int32_t ncells = (int32_t)cell.size();
            Tmp<int64_t> d_off(ncells, s);
            Tmp<int4> d_cell(ncells, s);
            MPK_CUDA(cudaMemcpyAsync(d_off.p, cell_off.data(), sizeof(int64_t) * cell_off.size(), cudaMemcpyHostToDevice,
                                     s));
            MPK_CUDA(cudaMemcpyAsync(d_cell.p, cell.data(), sizeof(int4) * cell.size(), cudaMemcpyHostToDevice, s));
            k_expand_cells<<<std::min(ncells, 64 * device_sms()), 128, 0, s>>>(d_off.p, d_cell.p, ncells, P->units);
            MPK_LAUNCHED();
        } else if (!units.empty()) {
            MPK_CUDA(cudaMemcpyAsync(P->units, units.data(), sizeof(int32_t) * units.size(), cudaMemcpyHostToDevice, s));
        }

        // ---- synchronisation state and vector workspace
        P->flags = P->arena.alloc_n<int32_t>((int64_t)(pmax + 1) * (NC > 0 ? NC : 1));
        MPK_CUDA(cudaMemsetAsync(P->flags, 0, sizeof(int32_t) * (size_t)(pmax + 1) * (NC > 0 ? NC : 1), s));
        if (o->trace) {
            P->trace = P->arena.alloc_n<unsigned long long>(MPK_TRACE_COUNTERS);
            MPK_CUDA(cudaMemsetAsync(P->trace, 0, sizeof(unsigned long long) * MPK_TRACE_COUNTERS, s));
        }
        // ticket, exit count, epoch and code of a failed launch, epoch of the last launch
        P->ctl = P->arena.alloc_n<unsigned int>(8);
        MPK_CUDA(cudaMemsetAsync(P->ctl, 0, 8 * sizeof(unsigned int), s));
        P->work_slots = std::max(pmax + 1, 4);  // all powers (original order) or ring of 3 + accumulator
        P->work = P->arena.alloc_n<double>((int64_t)P->work_slots * n * m + 1);
        if (P->accum == MPK_F32) P->shadow = P->arena.alloc_n<float>(2 * (int64_t)n * m + 1);
        MPK_CUDA(cudaStreamSynchronize(s));  // host vectors above must outlive their copies
    } catch (...) {
        P->arena.release();
        delete P;
        throw;
    }
    return P;
}

}  // namespace mpk
