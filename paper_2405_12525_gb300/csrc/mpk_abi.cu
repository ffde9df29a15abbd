// extern "C" entry points of libmpk.so (declared in include/mpk.h).  Argument checks
// happen here; every entry point converts internal failures into an mpk_status.
#include "mpk_internal.h"

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>

namespace mpk {
const char *last_error_text();
}

using namespace mpk;


// ---------------------------------------------------------------------------------------- levels
extern "C" mpk_status mpk_build_levels(const mpk_csr *A, int32_t root, mpk_stream stream, mpk_levels **out) {
    MPK_GUARD_BEGIN
    if (!out) fail(MPK_ERR_INVALID, "out is NULL");
    *out = nullptr;
    Levels *L = build_levels(A, root, as_stream(stream));
    *out = new mpk_levels_s{L};
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_build_levels_from(const mpk_csr *A, const int32_t *roots, int32_t nroots, mpk_stream stream,
                                         mpk_levels **out) {
    MPK_GUARD_BEGIN
    if (!out) fail(MPK_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (nroots < 0 || (nroots > 0 && !roots)) fail(MPK_ERR_INVALID, "bad root list");
    std::vector<int32_t> r(roots, roots + nroots);
    Levels *L = build_levels(A, 0, as_stream(stream), &r);
    *out = new mpk_levels_s{L};
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_levels_get(const mpk_levels *L, int32_t *n, int32_t *num_levels, const int32_t **level_ptr,
                                     const int32_t **perm, const int32_t **iperm, const int32_t **level_of) {
    if (!L || !L->impl) {
        set_error("levels handle is NULL");
        return MPK_ERR_INVALID;
    }
    if (n) *n = L->impl->n;
    if (num_levels) *num_levels = L->impl->num_levels;
    if (level_ptr) *level_ptr = L->impl->level_ptr;
    if (perm) *perm = L->impl->perm;
    if (iperm) *iperm = L->impl->iperm;
    if (level_of) *level_of = L->impl->level_of;
    return MPK_OK;
}

extern "C" void mpk_levels_destroy(mpk_levels *L) {
    if (!L) return;
    if (L->impl) {
        L->impl->arena.release();
        delete L->impl;
    }
    delete L;
}

// ---------------------------------------------------------------------------------------- plans
extern "C" void mpk_plan_opts_default(mpk_plan_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->p_max = 8;
    o->nrhs = 1;
    o->order = MPK_ORDER_ORIGINAL;
}

extern "C" mpk_status mpk_plan(const mpk_csr *A, const mpk_levels *L, const mpk_plan_opts *opts, mpk_stream stream,
                               mpk_plan_t **out) {
    MPK_GUARD_BEGIN
    if (!out) fail(MPK_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (L && !L->impl) fail(MPK_ERR_INVALID, "levels handle is empty");
    Plan *P = build_plan(A, L ? L->impl : nullptr, opts, as_stream(stream));
    *out = new mpk_plan_s{P};
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_plan_describe(const mpk_plan_t *P, mpk_plan_desc *d) {
    if (!P || !P->impl || !d) {
        set_error("NULL plan or descriptor");
        return MPK_ERR_INVALID;
    }
    const Plan &p = *P->impl;
    std::memset(d, 0, sizeof(*d));
    d->n = p.n;
    d->nnz = p.nnz;
    d->nrhs = p.m;
    d->p_max = p.p_max;
    d->order = p.order;
    d->num_levels = p.num_levels;
    d->num_groups = p.num_groups;
    d->num_chunks = p.num_chunks;
    d->group_budget_bytes = p.group_budget;
    d->window = p.window;
    d->cache_bytes = p.cache_bytes;
    d->device_bytes = p.arena.bytes;
    d->padded_entries = p.padded;
    d->group_level_ptr_dev = p.group_level_ptr;
    d->group_row_ptr_dev = p.group_row_ptr;
    d->chunk_row_ptr_dev = p.chunk_row;
    d->perm_dev = p.perm;
    d->shape = p.shape;
    d->engine = p.engine;
    d->chunk_rows = p.chunk_rows;
    d->accum = p.accum;
    d->split_levels = p.split_levels ? 1 : 0;
    return MPK_OK;
}

extern "C" mpk_status mpk_plan_export_csr(const mpk_plan_t *P, int32_t *row_ptr, int32_t *col, double *val,
                                          mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (!P || !P->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    export_csr(*P->impl, row_ptr, col, val, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" void mpk_plan_destroy(mpk_plan_t *P) {
    if (!P) return;
    if (P->impl) {
        P->impl->arena.release();
        delete P->impl;
    }
    delete P;
}

// ---------------------------------------------------------------------------------------- apply
// Each launch of the level-blocked kernel takes the next epoch on the device (ctl[4]); before
// the epochs could wrap, the flags and the epoch are cleared (launches replayed from a CUDA
// graph are not counted here).
void mpk::next_epoch(Plan &P, cudaStream_t s) {
    if (++P.launches >= ((int64_t)1 << 30)) {
        MPK_CUDA(cudaMemsetAsync(P.flags, 0, sizeof(int32_t) * (size_t)(P.p_max + 1) * std::max(1, P.num_chunks), s));
        MPK_CUDA(cudaMemsetAsync(P.ctl + 2, 0, 3 * sizeof(unsigned int), s));
        P.launches = 1;
    }
}

KArgs mpk::base_args(Plan &P, int32_t p) {
    KArgs a;
    std::memset(&a, 0, sizeof(a));
    a.val = P.val;
    a.col = P.col;
    a.lcol = P.lcol;
    a.slice_ptr = P.slice_ptr;
    a.rowlen = P.rowlen;
    a.chunk_row = P.chunk_row;
    a.chunk_slice = P.chunk_slice;
    a.dep = P.dep;
    a.dep_ranges = P.dep_ranges;
    a.chunk_rec = P.chunk_rec;
    a.n = P.n;
    a.nchunks = P.num_chunks;
    a.units = P.units + P.unit_off[p];
    a.nunits = P.unit_off[p + 1] - P.unit_off[p];
    a.flags = P.flags;
    a.epoch_word = P.ctl + 4;
    a.ticket = P.ctl;
    a.exit_count = P.ctl + 1;
    a.err = reinterpret_cast<int32_t *>(P.ctl + 2);
    a.wait_ns = P.wait_ns;
    a.drop_unit = P.drop_unit;
    a.trace = P.trace;
    P.drop_unit = -1;
    a.ystride = (int64_t)P.n * P.m;
    a.shadow = P.shadow;
    a.p_launch = p;
    if (P.engine == MPK_ENGINE_WARP) {
        a.w_item = P.w_item + P.w_cell_off[p];
        a.w_gk = P.w_gk + P.w_cell_off[p];
        a.w_ncells = P.w_cell_off[p + 1] - P.w_cell_off[p];
        a.w_nitems = P.w_items[p];
        a.w_cnt = P.w_cnt;
        a.w_q = reinterpret_cast<unsigned int *>(P.w_cnt + (int64_t)(P.p_max + 1) * std::max(P.num_chunks, 1));
        a.g_row = P.group_row_ptr;
        a.g_slice = P.g_slice;
        a.w_slice_chunk = P.w_slice_chunk;
        a.w_chunk_nsl = P.w_chunk_nsl;
        a.ngroups = P.num_groups;
    }
    return a;
}

static void check_apply_args(const mpk_plan_t *Ph, const double *X, int32_t p, const double *Y) {
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    const Plan &P = *Ph->impl;
    if (!P.inst_row.empty()) fail(MPK_ERR_INVALID, "a batch plan runs through mpk_batch_apply");
    if (p < 0 || p > P.p_max) fail(MPK_ERR_INVALID, "p = %d outside [0, p_max = %d]", p, P.p_max);
    if (P.n > 0 && (!X || !Y)) fail(MPK_ERR_INVALID, "NULL X or Y");
}

extern "C" mpk_status mpk_apply(const mpk_plan_t *Ph, const double *X, int32_t p, double *Y, mpk_stream stream) {
    MPK_GUARD_BEGIN
    check_apply_args(Ph, X, p, Y);
    Plan &P = *const_cast<Plan *>(Ph->impl);
    cudaStream_t s = as_stream(stream);
    const int64_t nm = (int64_t)P.n * P.m;
    if (P.n == 0) return MPK_OK;
    if (p == 0) {
        if (Y != X) MPK_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
        return MPK_OK;
    }
    next_epoch(P, s);
    KArgs a = base_args(P, p);
    a.ring = p + 1;
    if (P.identity || P.order == MPK_ORDER_PLAN) {
        a.x0 = X;
        a.ybase = Y;
        a.y0copy = (Y != X) ? Y : nullptr;
        if (a.y0copy && P.level0_rows > 0)  // level 0 of a level-capped plan has no units
            MPK_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * (size_t)P.level0_rows * P.m, cudaMemcpyDeviceToDevice, s));
        if (P.accum == MPK_F32) launch_round_f32(X, nm, P.shadow, s);  // binary32 input of power 1
        launch_mpk(P, a, 0, s);
    } else {
        // gather X into plan order, compute every power in plan order in the workspace,
        // then write the powers through the permutation (gather by output row)
        launch_gather_rows(X, P.perm, P.work, P.n, P.m, s);
        if (Y != X) MPK_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
        a.x0 = P.work;
        a.ybase = P.work;
        if (P.accum == MPK_F32) launch_round_f32(P.work, nm, P.shadow, s);
        launch_mpk(P, a, 0, s);
        launch_scatter_powers(P.work, P.iperm, Y, P.n, P.m, p, s);
    }
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_apply_host(const mpk_plan_t *Ph, const double *X_host, int32_t p, double *Y_host,
                                     mpk_stream stream) {
    MPK_GUARD_BEGIN
    check_apply_args(Ph, X_host, p, Y_host);
    Plan &P = *const_cast<Plan *>(Ph->impl);
    cudaStream_t s = as_stream(stream);
    const int64_t nm = (int64_t)P.n * P.m;
    if (P.n == 0) return MPK_OK;
    // the output is written by kernels: it must be page-locked host memory with a device address
    cudaPointerAttributes at{};
    MPK_CUDA(cudaPointerGetAttributes(&at, Y_host));
    if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr)
        fail(MPK_ERR_INVALID, "Y_host must be page-locked host memory (cudaHostAlloc or cudaHostRegister)");
    double *yh = static_cast<double *>(at.devicePointer);
    const size_t xbytes = sizeof(double) * (size_t)nm;
    if ((const char *)Y_host < (const char *)X_host + xbytes &&
        (const char *)X_host < (const char *)Y_host + xbytes * (size_t)(p + 1))
        fail(MPK_ERR_INVALID, "Y_host overlaps X_host");
    if (p == 0) {
        MPK_CUDA(cudaMemcpyAsync(Y_host, X_host, xbytes, cudaMemcpyHostToHost, s));
        return MPK_OK;
    }
    if (P.identity || P.order == MPK_ORDER_PLAN) {
        // X into power block 0 of the workspace.  The staged engine with one right-hand side
        // runs the host-output kernel: power-1 units copy X's rows to Y_host[0] and every power's
        // rows go to Y_host as their units finish.  Other plans compute into the workspace and
        // copy the p+1 blocks to Y_host afterwards.
        const bool fused = P.engine == MPK_ENGINE_STAGED && P.m == 1 && P.trace == nullptr;
        if (P.level_capped && !fused)
            fail(MPK_ERR_UNSUPPORTED, "host output of a level-capped plan needs nrhs 1 and the staged engine");
        MPK_CUDA(cudaMemcpyAsync(P.work, X_host, xbytes, cudaMemcpyHostToDevice, s));
        next_epoch(P, s);
        KArgs a = base_args(P, p);
        a.ring = p + 1;
        a.x0 = P.work;
        a.ybase = P.work;
        if (P.accum == MPK_F32) launch_round_f32(P.work, nm, P.shadow, s);
        if (fused) {
            a.y0copy = yh;
            a.yhost = yh;
            if (P.level0_rows > 0)  // level 0 of a level-capped plan has no units
                MPK_CUDA(cudaMemcpyAsync(Y_host, X_host, sizeof(double) * (size_t)P.level0_rows * P.m,
                                         cudaMemcpyHostToHost, s));
            launch_mpk(P, a, 2, s);  // MODE_HOST
        } else {
            launch_mpk(P, a, 0, s);
            MPK_CUDA(cudaMemcpyAsync(Y_host, P.work, xbytes * (size_t)(p + 1), cudaMemcpyDeviceToHost, s));
        }
    } else {
        // X to the device, gathered into plan order, every power in the workspace, then all
        // powers (0..p) written through the permutation into Y_host
        Tmp<double> xd(nm, s);
        MPK_CUDA(cudaMemcpyAsync(xd.p, X_host, xbytes, cudaMemcpyHostToDevice, s));
        launch_gather_rows(xd.p, P.perm, P.work, P.n, P.m, s);
        next_epoch(P, s);
        KArgs a = base_args(P, p);
        a.ring = p + 1;
        a.x0 = P.work;
        a.ybase = P.work;
        if (P.accum == MPK_F32) launch_round_f32(P.work, nm, P.shadow, s);
        launch_mpk(P, a, 0, s);
        launch_scatter_powers(P.work, P.iperm, yh, P.n, P.m, p, s, -1, 0, 0);
    }
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_spmv_powers(const mpk_plan_t *Ph, const double *X, int32_t p, double *Y,
                                      mpk_stream stream) {
    MPK_GUARD_BEGIN
    check_apply_args(Ph, X, p, Y);
    Plan &P = *const_cast<Plan *>(Ph->impl);
    if (P.accum != MPK_F64)
        fail(MPK_ERR_UNSUPPORTED, "the row-range SpMV accumulates in binary64: compare binary32 accumulation with a "
                                  "plan of engine MPK_ENGINE_SWEEP");
    cudaStream_t s = as_stream(stream);
    const int64_t nm = (int64_t)P.n * P.m;
    if (P.n == 0) return MPK_OK;
    if (Y != X) MPK_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
    if (P.identity || P.order == MPK_ORDER_PLAN) {
        for (int k = 1; k <= p; ++k) launch_spmv(P, Y + (k - 1) * nm, Y + k * nm, s);
    } else {
        launch_gather_rows(X, P.perm, P.work, P.n, P.m, s);
        for (int k = 1; k <= p; ++k) launch_spmv(P, P.work + (k - 1) * nm, P.work + k * nm, s);
        launch_scatter_powers(P.work, P.iperm, Y, P.n, P.m, p, s);
    }
    return MPK_OK;
    MPK_GUARD_END
}

// Chebyshev recurrence state: ring of three vectors (v_j in ring slot j % 3, plan order) and the
// accumulator.  cheb_start: v_0 = X (gathered into plan order if the plan keeps A's order),
// acc = c_0 v_0.  cheb_steps: steps k_begin+1 .. k_end, in launches of at most p_max steps; the
// ring indices follow the absolute step, so any split of the steps gives the same bits.
static void cheb_start(Plan &P, const double *X, double c0_re, double c0_im, bool cplx, double *ring, double *acc,
                       cudaStream_t s) {
    const int64_t nm = (int64_t)P.n * P.m;
    if (P.identity || P.order == MPK_ORDER_PLAN)
        MPK_CUDA(cudaMemcpyAsync(ring, X, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
    else
        launch_gather_rows(X, P.perm, ring, P.n, P.m, s);
    launch_cheb_init(ring, acc, P.n, P.m, c0_re, cplx ? c0_im : 0.0, cplx ? 1 : 0, s);
}

static void cheb_steps(Plan &P, double *ring, double *acc, int32_t k_begin, int32_t k_end, const double *coeff_re,
                       const double *coeff_im, double scale, double shift, cudaStream_t s) {
    // same expressions as the recurrence's definition: 2A'v = alpha Av + beta v
    const double alpha = 2.0 / scale, beta = -2.0 * shift / scale;
    const double halpha = 1.0 / scale, hbeta = -shift / scale;
    // binary32 accumulation: the input of step k_begin + 1 is the binary32 rounding of the
    // state's v_{k_begin}; every launch then leaves the rounding of its last step behind
    if (P.accum == MPK_F32 && k_end > k_begin) {
        const int64_t nm = (int64_t)P.n * P.m;
        launch_round_f32(ring + (int64_t)(k_begin % 3) * nm, nm, P.shadow + (int64_t)(k_begin & 1) * nm, s);
    }
    for (int32_t j0 = k_begin; j0 < k_end; j0 += P.p_max) {
        const int32_t pb = std::min(P.p_max, k_end - j0);
        next_epoch(P, s);
        KArgs a = base_args(P, pb);
        a.x0 = ring;
        a.ybase = ring;
        a.ring = 3;
        a.k_offset = j0;
        a.alpha = alpha;
        a.beta = beta;
        a.halpha = halpha;
        a.hbeta = hbeta;
        a.acc = acc;
        a.complex_coeff = coeff_im ? 1 : 0;
        for (int k = 1; k <= pb; ++k) {
            a.cre[k] = coeff_re[j0 + k];
            a.cim[k] = coeff_im ? coeff_im[j0 + k] : 0.0;
        }
        launch_mpk(P, a, 1, s);
    }
}

extern "C" mpk_status mpk_cheb_filter(const mpk_plan_t *Ph, const double *X, int32_t degree, const double *coeff_re,
                                      const double *coeff_im, double scale, double shift, double *out,
                                      mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    Plan &P = *const_cast<Plan *>(Ph->impl);
    if (!P.inst_row.empty()) fail(MPK_ERR_INVALID, "a batch plan runs through mpk_batch_apply");
    if (P.level_capped) fail(MPK_ERR_INVALID, "a level-capped plan computes partial powers only");
    if (degree < 0) fail(MPK_ERR_INVALID, "degree must be >= 0");
    if (!coeff_re) fail(MPK_ERR_INVALID, "coeff_re is NULL");
    if (!(scale != 0.0)) fail(MPK_ERR_INVALID, "scale must be non-zero");
    if (coeff_im && (P.m % 2)) fail(MPK_ERR_INVALID, "complex coefficients need an even nrhs");
    if (P.n > 0 && (!X || !out)) fail(MPK_ERR_INVALID, "NULL X or out");
    if (P.n == 0) return MPK_OK;
    cudaStream_t s = as_stream(stream);
    const int64_t nm = (int64_t)P.n * P.m;
    const bool plan_order = P.identity || P.order == MPK_ORDER_PLAN;
    double *acc = plan_order ? out : P.work + 3 * nm;
    cheb_start(P, X, coeff_re[0], coeff_im ? coeff_im[0] : 0.0, coeff_im != nullptr, P.work, acc, s);
    cheb_steps(P, P.work, acc, 0, degree, coeff_re, coeff_im, scale, shift, s);
    if (!plan_order) launch_scatter_rows(acc, P.iperm, out, P.n, P.m, s);
    return MPK_OK;
    MPK_GUARD_END
}

static void check_cheb_plan(const mpk_plan_t *Ph) {
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    const Plan &P = *Ph->impl;
    if (!P.inst_row.empty()) fail(MPK_ERR_INVALID, "a batch plan runs through mpk_batch_apply");
    if (P.level_capped) fail(MPK_ERR_INVALID, "a level-capped plan computes partial powers only");
}

extern "C" int64_t mpk_cheb_state_bytes(const mpk_plan_t *Ph) {
    if (!Ph || !Ph->impl) return 0;
    return 4 * (int64_t)Ph->impl->n * Ph->impl->m * (int64_t)sizeof(double);
}

extern "C" mpk_status mpk_cheb_begin(const mpk_plan_t *Ph, const double *X, double c0_re, double c0_im,
                                     int32_t complex_coeff, double *state, mpk_stream stream) {
    MPK_GUARD_BEGIN
    check_cheb_plan(Ph);
    Plan &P = *const_cast<Plan *>(Ph->impl);
    if (complex_coeff && (P.m % 2)) fail(MPK_ERR_INVALID, "complex coefficients need an even nrhs");
    if (P.n > 0 && (!X || !state)) fail(MPK_ERR_INVALID, "NULL X or state");
    if (P.n == 0) return MPK_OK;
    const int64_t nm = (int64_t)P.n * P.m;
    cheb_start(P, X, c0_re, c0_im, complex_coeff != 0, state, state + 3 * nm, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_cheb_advance(const mpk_plan_t *Ph, double *state, int32_t k_begin, int32_t k_end,
                                       const double *coeff_re, const double *coeff_im, double scale, double shift,
                                       mpk_stream stream) {
    MPK_GUARD_BEGIN
    check_cheb_plan(Ph);
    Plan &P = *const_cast<Plan *>(Ph->impl);
    if (k_begin < 0 || k_end < k_begin) fail(MPK_ERR_INVALID, "need 0 <= k_begin <= k_end");
    if (!coeff_re) fail(MPK_ERR_INVALID, "coeff_re is NULL");
    if (!(scale != 0.0)) fail(MPK_ERR_INVALID, "scale must be non-zero");
    if (coeff_im && (P.m % 2)) fail(MPK_ERR_INVALID, "complex coefficients need an even nrhs");
    if (P.n > 0 && !state) fail(MPK_ERR_INVALID, "NULL state");
    if (P.n == 0) return MPK_OK;
    const int64_t nm = (int64_t)P.n * P.m;
    cheb_steps(P, state, state + 3 * nm, k_begin, k_end, coeff_re, coeff_im, scale, shift, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_cheb_finish(const mpk_plan_t *Ph, const double *state, double *out, mpk_stream stream) {
    MPK_GUARD_BEGIN
    check_cheb_plan(Ph);
    const Plan &P = *Ph->impl;
    if (P.n > 0 && (!state || !out)) fail(MPK_ERR_INVALID, "NULL state or out");
    if (P.n == 0) return MPK_OK;
    const int64_t nm = (int64_t)P.n * P.m;
    cudaStream_t s = as_stream(stream);
    if (P.identity || P.order == MPK_ORDER_PLAN)
        MPK_CUDA(cudaMemcpyAsync(out, state + 3 * nm, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
    else
        launch_scatter_rows(state + 3 * nm, P.iperm, out, P.n, P.m, s);
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_read_trace(const mpk_plan_t *Ph, int64_t *counters, mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl || !counters) fail(MPK_ERR_INVALID, "NULL plan or output");
    const Plan &P = *Ph->impl;
    if (!P.trace) fail(MPK_ERR_UNSUPPORTED, "plan was built without opts.trace");
    MPK_CUDA(cudaStreamSynchronize(as_stream(stream)));
    MPK_CUDA(cudaMemcpy(counters, P.trace, sizeof(int64_t) * MPK_TRACE_COUNTERS, cudaMemcpyDeviceToHost));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_sync_status(const mpk_plan_t *Ph, mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    Plan &P = *const_cast<Plan *>(Ph->impl);
    MPK_CUDA(cudaStreamSynchronize(as_stream(stream)));
    // ctl[2..3]: epoch and code of the last failed launch, kept until read here
    unsigned int h[2] = {0, 0};
    MPK_CUDA(cudaMemcpy(h, P.ctl + 2, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[1] != 0) {
        MPK_CUDA(cudaMemset(P.ctl + 2, 0, 2 * sizeof(unsigned int)));
        set_error("a bounded device wait expired in a launch of this plan (device epoch %u)", h[0]);
        return (mpk_status)h[1];
    }
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_debug_drop_release(mpk_plan_t *Ph, int32_t chunk, int32_t k) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    Plan &P = *Ph->impl;
    if (chunk < 0 || chunk >= P.num_chunks || k < 1 || k > P.p_max) fail(MPK_ERR_INVALID, "no such unit");
    P.drop_unit = (chunk << 5) | k;
    return MPK_OK;
    MPK_GUARD_END
}

// ---------------------------------------------------------------------------------------- probes
extern "C" mpk_status mpk_probe_load(const void *buf, int64_t bytes, int32_t reps, int32_t ctas_per_sm, int32_t *sink,
                                     mpk_stream stream) {
    MPK_GUARD_BEGIN
    probe_load(buf, bytes, reps, ctas_per_sm, sink, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_probe_dfma(int32_t blocks, int32_t iters, double *sink, mpk_stream stream) {
    MPK_GUARD_BEGIN
    probe_dfma(blocks, iters, sink, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_spmv_rows(const mpk_plan_t *Ph, int32_t row_begin, int32_t row_end, const double *X,
                                    double *Y, mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    const Plan &P = *Ph->impl;
    if (row_begin < 0 || row_end > P.n || row_begin > row_end) fail(MPK_ERR_INVALID, "bad row range");
    if (row_end > row_begin && (!X || !Y)) fail(MPK_ERR_INVALID, "NULL X or Y");
    const Plan *pp = &P;
    launch_spmv_rows(&pp, &row_begin, &row_end, &X, &Y, 1, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_spmv_rows_multi(int32_t count, const mpk_plan_t *const *plans, const int32_t *row_begin,
                                          const int32_t *row_end, const double *const *X, double *const *Y,
                                          mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (count < 0 || count > MPK_MAX_ROW_SEGMENTS) fail(MPK_ERR_INVALID, "count must be in [0, %d]", MPK_MAX_ROW_SEGMENTS);
    if (count == 0) return MPK_OK;
    if (!plans || !row_begin || !row_end || !X || !Y) fail(MPK_ERR_INVALID, "NULL argument array");
    const Plan *pp[MPK_MAX_ROW_SEGMENTS];
    int vt = -1, m = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (!plans[i] || !plans[i]->impl) fail(MPK_ERR_INVALID, "plan %d is NULL", i);
        const Plan &P = *plans[i]->impl;
        pp[i] = &P;
        if (row_begin[i] < 0 || row_end[i] > P.n || row_begin[i] > row_end[i])
            fail(MPK_ERR_INVALID, "bad row range in segment %d", i);
        if (row_end[i] == row_begin[i]) continue;
        if (!X[i] || !Y[i]) fail(MPK_ERR_INVALID, "NULL X or Y in segment %d", i);
        if (vt < 0) {
            vt = P.val_type;
            m = P.m;
        } else if (vt != P.val_type || m != P.m) {
            fail(MPK_ERR_INVALID, "segments need one value type and one nrhs");
        }
    }
    launch_spmv_rows(pp, row_begin, row_end, X, Y, count, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_copy_rows(const double *src, const int64_t *src_idx, double *dst, const int64_t *dst_idx,
                                    int64_t n, int32_t m, mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (n < 0 || m < 1) fail(MPK_ERR_INVALID, "bad sizes");
    if (n > 0 && (!src || !src_idx || !dst || !dst_idx)) fail(MPK_ERR_INVALID, "NULL argument");
    launch_copy_rows(src, src_idx, dst, dst_idx, n, m, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_gather_rows(const double *src, const int32_t *idx, int32_t n, int32_t m, double *dst,
                                      mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (n < 0 || m < 1) fail(MPK_ERR_INVALID, "bad sizes");
    if (n > 0 && (!src || !idx || !dst)) fail(MPK_ERR_INVALID, "NULL argument");
    launch_gather_rows(src, idx, dst, n, m, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_widen_values(int32_t val_type, const void *src, int64_t n, double *dst,
                                       mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (n < 0) fail(MPK_ERR_INVALID, "n < 0");
    if (n > 0 && (!src || !dst)) fail(MPK_ERR_INVALID, "NULL src or dst");
    widen_values(val_type, src, n, dst, as_stream(stream));
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_device_info(int32_t *num_sms, int64_t *l2_bytes) {
    MPK_GUARD_BEGIN
    if (num_sms) *num_sms = device_sms();
    if (l2_bytes) *l2_bytes = device_l2_bytes();
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" const char *mpk_status_string(mpk_status s) {
    switch (s) {
        case MPK_OK: return "ok";
        case MPK_ERR_INVALID: return "invalid argument";
        case MPK_ERR_TOO_LARGE: return "too large";
        case MPK_ERR_OOM: return "out of device memory";
        case MPK_ERR_TIMEOUT: return "device wait timed out";
        case MPK_ERR_CUDA: return "CUDA error";
        case MPK_ERR_BUDGET: return "memory budget exceeded";
        case MPK_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

extern "C" const char *mpk_last_error(void) { return last_error_text(); }
