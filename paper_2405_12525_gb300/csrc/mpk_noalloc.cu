// mpk_apply_noalloc: the level-blocked MPK of mpk_apply for callers that must not allocate
// device memory during a call.  Examples are code that runs while an allocator is
// locked or must not grow its footprint, latency-critical loops that forbid the implicit
// synchronisation cudaMalloc/cudaFree cause, and hosts that hand the library only
// pre-allocated buffers.  The plan is built beforehand; at call time the kernel's
// synchronisation state (per-chunk completion flags, ticket, exit counter, error word)
// lives in one fixed array in device memory instead of in the plan.
#include "mpk_internal.h"

#include <cstring>

namespace mpk {

// Scratch shared by every call on a device: kNoAllocInts 32-bit words (4 MiB).  Every GPU
// that loads the library holds this array until the process exits.  A call uses
// kNoAllocCtl control words (ticket, exit count, error epoch, error code, last epoch, padding)
// and then (p + 1) * num_chunks completion flags.
constexpr int64_t kNoAllocInts = int64_t(1) << 20;
constexpr int64_t kNoAllocCtl = 8;
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocInts];

// Device address of the array in the current context, looked up on every call (no device
// memory is allocated by the lookup): a cached address could outlive its context, e.g. after
// cudaDeviceReset, when the module is loaded again elsewhere.
static int32_t *scratch_address() {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
        fail(MPK_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
    return static_cast<int32_t *>(ptr);
}

// copies the launch's error code (0 or MPK_ERR_TIMEOUT) to the caller's status word
__global__ void k_noalloc_status(const int32_t *err, int32_t *status) {
    *status = (err[0] == 1) ? (err[1] ? err[1] : (int32_t)MPK_ERR_TIMEOUT) : (int32_t)MPK_OK;
}

}  // namespace mpk

using namespace mpk;

extern "C" mpk_status mpk_apply_noalloc(const mpk_plan_t *Ph, const double *X, int32_t p, double *Y,
                                        int32_t *status, mpk_stream stream) {
    try {
        if (!Ph || !Ph->impl) fail(MPK_ERR_INVALID, "plan is NULL");
        const Plan &P = *Ph->impl;
        if (!P.inst_row.empty()) fail(MPK_ERR_INVALID, "a batch plan runs through mpk_batch_apply");
        if (!(P.identity || P.order == MPK_ORDER_PLAN))
            fail(MPK_ERR_UNSUPPORTED, "mpk_apply_noalloc needs a plan in MPK_ORDER_PLAN (or without levels)");
        if (p < 0 || p > P.p_max) fail(MPK_ERR_INVALID, "p = %d outside [0, p_max = %d]", p, P.p_max);
        if (P.n > 0 && (!X || !Y)) fail(MPK_ERR_INVALID, "NULL X or Y");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (p == 0) {  // as mpk_apply: Y[0] = X, nothing computed, nothing allocated
            if (P.n > 0 && Y != X)
                MPK_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * (size_t)P.n * P.m, cudaMemcpyDeviceToDevice, s));
            if (status) MPK_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
            return MPK_OK;
        }
        // scratch layout: [0..4] ticket, exit count, error epoch, error code, epoch of the last
        // launch (zero: this launch is epoch 1); from [kNoAllocCtl] the completion flags of
        // powers 0..p for every chunk
        const int64_t need = kNoAllocCtl + (int64_t)(p + 1) * (P.num_chunks > 0 ? P.num_chunks : 1);
        if (need > kNoAllocInts)
            fail(MPK_ERR_TOO_LARGE,
                 "mpk_apply_noalloc needs %lld scratch words for %d chunks and p = %d; the fixed scratch holds %lld "
                 "(use mpk_apply, or fewer chunks: larger chunk_rows)",
                 (long long)need, P.num_chunks, p, (long long)kNoAllocInts);
        int32_t *scratch = scratch_address();
        // the previous call's flags and counters are still in the array: start from zero
        MPK_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int32_t) * (size_t)need, s));
        if (P.n > 0) {
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
            a.flags = scratch + kNoAllocCtl;
            a.epoch_word = reinterpret_cast<unsigned int *>(scratch + 4);
            a.ticket = reinterpret_cast<unsigned int *>(scratch);
            a.exit_count = reinterpret_cast<unsigned int *>(scratch + 1);
            a.err = scratch + 2;
            a.wait_ns = P.wait_ns;
            a.drop_unit = -1;
            a.trace = nullptr;
            a.x0 = X;
            a.ybase = Y;
            a.ystride = (int64_t)P.n * P.m;
            a.shadow = P.shadow;
            a.ring = p + 1;
            a.p_launch = p;
            a.y0copy = (Y != X) ? Y : nullptr;
            if (a.y0copy && P.level0_rows > 0)  // level 0 of a level-capped plan has no units
                MPK_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * (size_t)P.level0_rows * P.m,
                                         cudaMemcpyDeviceToDevice, s));
            if (P.accum == MPK_F32) launch_round_f32(X, (int64_t)P.n * P.m, P.shadow, s);  // plan-owned ring
            launch_mpk(P, a, 0, s);
        }
        if (status) {
            k_noalloc_status<<<1, 1, 0, s>>>(scratch + 2, status);
            MPK_LAUNCHED();
        }
        return MPK_OK;
    } catch (const Fail &f) {
        return f.status;
    } catch (...) {
        set_error("unexpected internal error");
        return MPK_ERR_CUDA;
    }
}
