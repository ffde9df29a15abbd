// Batched MPK: several independent matrices (different sizes and powers, one value type and
// one number of right-hand sides) in one plan and one persistent launch per apply.
//
// The plan is that of the direct sum diag(A_0, ..., A_{c-1}), the block-diagonal matrix whose
// powers are the blocks' powers (Sec. 3's method applied to it unchanged).  The blocks share
// no edge, so the BFS of the direct sum restarts at each block's first row and numbers the
// blocks one after the other: block i keeps its rows [off_i, off_i + n_i) in both numberings,
// and its levels and permutation are those of A_i alone, shifted by off_i.  The planner cuts
// groups at block boundaries and merges the blocks' Lp-diagram tables line by line (each up
// to its own power), so one ticket space serves all blocks and small blocks run side by side.
#include "mpk_internal.h"

#include <algorithm>
#include <vector>

namespace mpk {

// dst[i] = src[i] + add
__global__ void k_copy_add(const int32_t *src, int64_t n, int32_t add, int32_t *dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i] + add;
}

static int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sms() * 16;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

static int value_bytes(int32_t t) {
    if (t == MPK_F64) return 8;
    if (t == MPK_F32) return 4;
    if (t == MPK_BF16) return 2;
    fail(MPK_ERR_UNSUPPORTED, "value type %d", t);
}

}  // namespace mpk

using namespace mpk;

extern "C" mpk_status mpk_batch_plan(const mpk_csr *mats, int32_t count, const int32_t *p_each,
                                     const mpk_plan_opts *opts, mpk_stream stream, mpk_plan_t **out) {
    MPK_GUARD_BEGIN
    if (!out) fail(MPK_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!mats || !p_each || !opts || count < 1) fail(MPK_ERR_INVALID, "need count >= 1 matrices, powers and options");
    cudaStream_t s = as_stream(stream);
    const int32_t vtype = mats[0].val_type;
    const int vb = value_bytes(vtype);
    std::vector<int32_t> inst_row(1, 0), inst_p;
    std::vector<int64_t> nnz_off(1, 0);
    int symmetric = 1;
    for (int32_t i = 0; i < count; ++i) {
        const mpk_csr &A = mats[i];
        if (A.val_type != vtype) fail(MPK_ERR_INVALID, "matrix %d: value type differs from matrix 0", i);
        if (p_each[i] < 1 || p_each[i] > opts->p_max)
            fail(MPK_ERR_INVALID, "matrix %d: p = %d outside [1, p_max = %d]", i, p_each[i], opts->p_max);
        validate_csr(&A, s);
        const int64_t rows = (int64_t)inst_row.back() + A.n, nz = nnz_off.back() + A.nnz;
        if (rows >= ((int64_t)1 << 31) - 1 || nz >= ((int64_t)1 << 31) - 1)
            fail(MPK_ERR_TOO_LARGE, "the batch has %lld rows and %lld entries (limit 2^31 - 1)", (long long)rows,
                 (long long)nz);
        inst_row.push_back((int32_t)rows);
        nnz_off.push_back(nz);
        inst_p.push_back(p_each[i]);
        symmetric &= A.is_symmetric ? 1 : 0;
    }
    const int32_t N = inst_row.back();
    const int64_t NNZ = nnz_off.back();
    // the direct sum in CSR: row pointers and columns shifted by each block's offsets
    Tmp<int32_t> rp((int64_t)N + 1, s), ci(std::max<int64_t>(NNZ, 1), s);
    Tmp<unsigned char> va(std::max<int64_t>(NNZ * vb, 1), s);
    for (int32_t i = 0; i < count; ++i) {
        const mpk_csr &A = mats[i];
        if (A.n > 0)
            k_copy_add<<<grid_for(A.n), 256, 0, s>>>(A.row_ptr, A.n, (int32_t)nnz_off[i], rp.p + inst_row[i]);
        if (A.nnz > 0) {
            k_copy_add<<<grid_for(A.nnz), 256, 0, s>>>(A.col, A.nnz, inst_row[i], ci.p + nnz_off[i]);
            MPK_CUDA(cudaMemcpyAsync(va.p + nnz_off[i] * vb, A.val, (size_t)A.nnz * vb, cudaMemcpyDeviceToDevice, s));
        }
        MPK_LAUNCHED();
    }
    const int32_t last = (int32_t)NNZ;
    MPK_CUDA(cudaMemcpyAsync(rp.p + N, &last, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    mpk_csr D;
    D.n = N;
    D.nnz = (int32_t)NNZ;
    D.row_ptr = rp.p;
    D.col = ci.p;
    D.val = va.p;
    D.val_type = vtype;
    D.is_symmetric = symmetric;
    Levels *L = build_levels(&D, 0, s);
    Plan *P = nullptr;
    try {
        P = build_plan(&D, L, opts, s, &inst_row, &inst_p);
    } catch (...) {
        L->arena.release();
        delete L;
        throw;
    }
    L->arena.release();
    delete L;
    MPK_CUDA(cudaStreamSynchronize(s));  // the temporary direct sum is freed on return
    *out = new mpk_plan_s{P};
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_batch_apply(const mpk_plan_t *Ph, const double *const *X, double *const *Y,
                                      mpk_stream stream) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    Plan &P = *const_cast<Plan *>(Ph->impl);
    if (P.inst_row.empty()) fail(MPK_ERR_INVALID, "not a batch plan (use mpk_apply)");
    if (!X) fail(MPK_ERR_INVALID, "NULL input array");
    const int32_t count = (int32_t)P.inst_p.size();
    if (!Y) fail(MPK_ERR_INVALID, "NULL output array");
    for (int32_t i = 0; i < count; ++i)
        if (P.inst_row[i + 1] > P.inst_row[i] && !X[i]) fail(MPK_ERR_INVALID, "NULL X of matrix %d", i);
    if (P.n == 0) return MPK_OK;
    cudaStream_t s = as_stream(stream);
    const int32_t m = P.m;
    const bool plan_order = P.order == MPK_ORDER_PLAN;
    // every block's X into the workspace (power 0, plan order), one launch over all blocks,
    // then every block's powers out of the workspace
    for (int32_t i = 0; i < count; ++i) {
        const int32_t off = P.inst_row[i], ni = P.inst_row[i + 1] - off;
        if (ni == 0) continue;
        launch_gather_rows(X[i], plan_order ? nullptr : P.perm + off, P.work + (int64_t)off * m, ni, m, s,
                           plan_order ? 0 : off);
        if (Y[i] && Y[i] != X[i])
            MPK_CUDA(cudaMemcpyAsync(Y[i], X[i], sizeof(double) * (size_t)ni * m, cudaMemcpyDeviceToDevice, s));
    }
    next_epoch(P, s);
    KArgs a = base_args(P, P.p_max);  // the batch table
    a.ring = P.p_max + 1;
    a.x0 = P.work;
    a.ybase = P.work;
    launch_mpk(P, a, 0, s);
    const int64_t pstride = (int64_t)P.n * m;
    for (int32_t i = 0; i < count; ++i) {
        const int32_t off = P.inst_row[i], ni = P.inst_row[i + 1] - off;
        if (ni == 0 || !Y[i]) continue;  // NULL: the caller reads block i in the workspace
        launch_scatter_powers(P.work, plan_order ? nullptr : P.iperm + off, Y[i], ni, m, P.inst_p[i], s, pstride,
                              plan_order ? off : 0);
    }
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_batch_describe(const mpk_plan_t *Ph, int32_t *count, int32_t *row_offsets, int32_t *powers) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    const Plan &P = *Ph->impl;
    const int32_t c = (int32_t)P.inst_p.size();
    if (count) *count = c;
    if (row_offsets) std::copy(P.inst_row.begin(), P.inst_row.end(), row_offsets);
    if (powers) std::copy(P.inst_p.begin(), P.inst_p.end(), powers);
    return MPK_OK;
    MPK_GUARD_END
}

extern "C" mpk_status mpk_batch_workspace(const mpk_plan_t *Ph, const double **work, int64_t *power_stride) {
    MPK_GUARD_BEGIN
    if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
    const Plan &P = *Ph->impl;
    if (P.inst_row.empty()) fail(MPK_ERR_INVALID, "not a batch plan");
    if (work) *work = P.work;
    if (power_stride) *power_stride = (int64_t)P.n * P.m;
    return MPK_OK;
    MPK_GUARD_END
}
