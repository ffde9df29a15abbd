// Hot path: the persistent level-blocked MPK kernel (Sec. 3, Fig. 2; Alg. 2's local phase),
// the plain SpMV comparator (Alg. 1), gather/scatter between row orders, and probes.
//
// Row body.  GB300 executes FP64 FMA at 2 lanes per clock per SM (about 0.6 T FMA/s for
// the whole GPU), so FP64 SpMV is bound by the FP64 pipe about as much as by HBM.  The
// row body therefore spends exactly one DFMA per stored entry and right-hand side: one
// thread owns one row and accumulates its entries sequentially in stored order (no
// shuffle-tree reduction, which would add FP64 additions).  The matrix copy is sliced by
// 32 rows (entry j of lane l at slice_ptr + 32 j + l), so a warp's entries j are
// contiguous and a chunk's entries form one contiguous, 128-byte aligned range that the
// kernel stages into shared memory with one bulk (TMA) copy per array.  All x gathers of
// a row are issued before its FMAs.  The result equals the oracle's fma-per-term row sums
// bit for bit.
#include "mpk_internal.h"

#include <algorithm>

namespace mpk {

constexpr int kBS = 32 * (1 + kCompWarps);  // level-blocked kernel: 1 control warp + compute warps
// blocks per SM the register budget is set for (65536 registers per SM): three blocks of
// 14 warps (40 registers a thread), whose 2 x 3072-entry slots (72 KB) fit three times in
// an SM's shared memory
#ifndef MPK_MIN_BLOCKS
#define MPK_MIN_BLOCKS 3
#endif
// (the single-vector power kernel; wider blocks, the Chebyshev recurrence and the traced
// kernel keep 64 registers a thread at two blocks)
template <int M, int MODE, bool TRACE> struct MpkOcc {
    static constexpr int blocks = (M == 1 && MODE == 0 && !TRACE) ? MPK_MIN_BLOCKS : 2;
};
constexpr int kSpmvBS = 256;        // threads per block of the plain SpMV kernel
// Staging slots: the control warp fills one while the compute warps work on the other.
constexpr int kSlots = 2;
// column indices of staged chunks: copied to shared memory beside the values (1), or read
// from global memory (L2) by the compute warps (0), which halves the slot size for FP64
#ifndef MPK_STAGE_COL
#define MPK_STAGE_COL 1
#endif
constexpr bool kStageCol = MPK_STAGE_COL != 0;
// one slot: kStageEntries values of the matrix's value type, then as many column indices
template <class VT> constexpr int smem_bytes() {
    return kSlots * kStageEntries * (int)(sizeof(typename VT::T) + (kStageCol ? 4 : 0));
}

enum Mode { MODE_POWERS = 0, MODE_CHEB = 1 };

__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(int32_t *p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (TMA, untiled); addresses 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Entries whose x loads are issued together before their FMAs.
template <int M> struct Batch {
    static constexpr int B = M == 1 ? 8 : (M == 2 ? 4 : (M == 4 ? 2 : 1));
};

// acc[i] = sum_j val[j] * x[col[j]*M + i] over a row's entries, in stored order.  Entry j
// of the row is at val[off + 32 j] / col[off + 32 j] (global or shared memory), j < width
// of the row's slice; entries past the row's end are padding with col < 0 and are skipped.
template <int M, int B, class VP, class CP>
__device__ __forceinline__ void row_sum(VP val, CP col, int64_t off, int width, const double *x, double (&acc)[M]) {
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = 0.0;
    for (int j0 = 0; j0 < width; j0 += B) {
        double v[B];
        int32_t c[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (j0 + b < width) {
                v[b] = val[off + 32 * (int64_t)(j0 + b)];
                c[b] = col[off + 32 * (int64_t)(j0 + b)];
            } else {
                v[b] = 0.0;
                c[b] = -1;
            }
        }
        double xv[B][M];
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int i = 0; i < M; ++i) xv[b][i] = (c[b] >= 0) ? x[(int64_t)c[b] * M + i] : 0.0;
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (c[b] >= 0) {
#pragma unroll
                for (int i = 0; i < M; ++i) acc[i] = fma(v[b], xv[b][i], acc[i]);
            }
    }
}

// Continues a row sum from entry j0 (acc already holds entries 0..j0-1).
template <int M, int B, class VP, class CP>
__device__ __forceinline__ void row_sum_from(VP val, CP col, int64_t off, int j_start, int width, const double *x,
                                             double (&acc)[M]) {
    for (int j0 = j_start; j0 < width; j0 += B) {
        double v[B];
        int32_t c[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (j0 + b < width) {
                v[b] = val[off + 32 * (int64_t)(j0 + b)];
                c[b] = col[off + 32 * (int64_t)(j0 + b)];
            } else {
                v[b] = 0.0;
                c[b] = -1;
            }
        }
        double xv[B][M];
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int i = 0; i < M; ++i) xv[b][i] = (c[b] >= 0) ? x[(int64_t)c[b] * M + i] : 0.0;
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (c[b] >= 0) {
#pragma unroll
                for (int i = 0; i < M; ++i) acc[i] = fma(v[b], xv[b][i], acc[i]);
            }
    }
}

// ----------------------------------------------------------------------------- value types
// Matrix values are stored as float64, float32 or bfloat16 and widened to float64 before
// their FMA, exactly and with integer operations only (widen_normal32: the planner admits
// zeros and normal numbers in the narrow types).
struct ValF64 {
    using T = double;
    static __device__ __forceinline__ double widen(double v) { return v; }
};
struct ValF32 {
    using T = float;
    static __device__ __forceinline__ double widen(float v) { return widen_normal32(__float_as_uint(v)); }
};
struct ValBF16 {
    using T = uint16_t;  // bfloat16 bits
    static __device__ __forceinline__ double widen(uint16_t v) { return widen_normal32((uint32_t)v << 16); }
};

// read-only views returning widened values: the immutable matrix copy in global memory, or a
// staged slot in shared memory
template <class VT> struct GVal {
    const typename VT::T *p;
    __device__ __forceinline__ double operator[](int64_t i) const { return VT::widen(__ldg(p + i)); }
};
template <class VT> struct SVal {
    const typename VT::T *p;
    __device__ __forceinline__ double operator[](int64_t i) const { return VT::widen(p[i]); }
};
struct GCol {
    const int32_t *p;
    __device__ __forceinline__ int32_t operator[](int64_t i) const { return __ldg(p + i); }
};

// Epilogue of one row at local power k: store into the plan-order slot, or advance the
// Chebyshev recurrence.
template <int M, int MODE>
__device__ __forceinline__ void row_epilogue(const KArgs &a, int k, int64_t r, const double (&w)[M],
                                             const double *xin) {
    const int j = a.k_offset + k;  // absolute power / recurrence step
    double *y = a.ybase + (int64_t)(j % a.ring) * a.ystride + r * M;
    if constexpr (MODE == MODE_CHEB) {
        double vn[M];
        if (j == 1) {
#pragma unroll
            for (int i = 0; i < M; ++i) vn[i] = fma(a.halpha, w[i], a.hbeta * xin[r * M + i]);
        } else {
            const double *vp2 = a.ybase + (int64_t)((j - 2) % a.ring) * a.ystride + r * M;
#pragma unroll
            for (int i = 0; i < M; ++i) vn[i] = fma(a.alpha, w[i], fma(a.beta, xin[r * M + i], -vp2[i]));
        }
#pragma unroll
        for (int i = 0; i < M; ++i) y[i] = vn[i];
        double *acc = a.acc + r * M;
        const double cr = a.cre[k];
        if (!a.complex_coeff) {
#pragma unroll
            for (int i = 0; i < M; ++i) acc[i] = fma(cr, vn[i], acc[i]);
        } else {
            const double ci = a.cim[k];
#pragma unroll
            for (int i = 0; i + 1 < M; i += 2) {
                double re = acc[i], im = acc[i + 1];
                re = fma(cr, vn[i], re);
                re = fma(-ci, vn[i + 1], re);
                im = fma(cr, vn[i + 1], im);
                im = fma(ci, vn[i], im);
                acc[i] = re;
                acc[i + 1] = im;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) y[i] = w[i];
    }
}

// ----------------------------------------------------------------------------- K-MPK
// Work unit = (row chunk c, local power k).  Units are claimed through one atomic ticket
// in the order of the unit table, which lists the Lp-diagram cells (group g, power k) line
// by line (g + kSlotSkew * k ascending) and, inside a line, k ascending.  Every dependency
// of a unit (chunks holding the rows it reads, at power k-1) lies on an earlier line, so it
// has a smaller ticket: the unit holding the
// smallest unfinished ticket can always run, whichever blocks are resident, and the
// schedule cannot deadlock.  A finished unit publishes flags[k][c] = epoch (release); a
// unit waits until the flags of its dependency ranges at power k-1 equal the epoch
// (acquire).
//
// Warp roles.  Warp 0 (control) claims units, stages each unit's matrix entries into one
// of kSlots shared-memory slots with bulk (TMA) copies and polls the unit's dependencies;
// warps 1..kCompWarps (compute) compute rows, and the last of them to finish a unit
// publishes its completion flag.  Slot b has two mbarriers: full[b] completes when the
// entries have landed and the dependencies are met, empty[b] when every compute warp is
// done with the slot.  The control warp prepares unit i+1 while compute warps work on unit
// i; its claims run three units ahead (tickets, unit ids and chunk records are fetched an
// iteration before they are needed), so only the dependency poll is on its critical path.
// A block processes its tickets in claim order and claims are increasing, so the block
// holding the smallest unfinished ticket is working on it: the schedule stays deadlock
// free with tickets claimed ahead.
// When no ticket is left, or a wait fails, the control warp stores the number of units it
// handed over in s_final; compute warps stop at that unit.  Every wait is bounded by
// a.wait_ns (globaltimer); on expiry the control warp records the epoch and
// MPK_ERR_TIMEOUT in a.err and all blocks drain out; no block exits with a bulk copy of
// its own still in flight.  The last block to exit resets the ticket.
struct UnitInfo {
    int unit;         // chunk << 5 | k
    int row0, row1, slice0;
    int ecount;       // padded entries of the chunk
    int staged;       // entries were copied to the slot's shared buffer
    int nsl;          // slices of the chunk
    int widths[4];    // staged chunks: width of slice q in byte q of the 16 bytes
    long long ebase;  // first entry of the chunk in the sliced copy
};

__device__ __forceinline__ bool timed_out(uint64_t t0, int64_t limit) { return globaltimer() - t0 > (uint64_t)limit; }

__device__ __forceinline__ int slice_width(const int (&w)[4], int q) {
    const int word = (q < 8) ? ((q < 4) ? w[0] : w[1]) : ((q < 12) ? w[2] : w[3]);  // no dynamic indexing
    return (word >> (8 * (q & 3))) & 0xff;
}

// A compute warp handles a unit in two phases.  Phase A reads the column indices of the
// warp's first row batch from shared memory and issues the x gathers; phase B runs the
// FMAs on those x values, finishes any further batches or slices, stores the results and
// publishes the unit.  Phase B directly follows phase A of the same unit: a warp holds no
// unit across a wait, so its lanes, which wait on the slot's mbarrier one by one, always
// work on the same unit.
template <int M> struct Prefetch {
    static constexpr int B = Batch<M>::B;
    int unit;             // -1: nothing pending
    int slot;
    int r;                // this lane's row in the warp's first slice, -1 if none
    int off;              // offset of that row's entries in the slot (staged units)
    int width;            // width of the warp's first slice (staged units)
    double x[B][M];       // x values of the first batch (entries j < min(B, width))
};

template <int M>
__device__ __forceinline__ const double *input_block(const KArgs &a, int k) {
    return (k == 1 && a.k_offset == 0) ? a.x0 : a.ybase + (int64_t)((a.k_offset + k - 1) % a.ring) * a.ystride;
}

// phase A: request the x values of the warp's first batch of unit u (slot b)
template <int M>
__device__ __forceinline__ void phase_a(const KArgs &a, const UnitInfo &u, int b, const int32_t *scol, int cwarp,
                                        int lane, Prefetch<M> &pf) {
    constexpr int B = Batch<M>::B;
    pf.unit = u.unit;
    pf.slot = b;
    const double *xin = input_block<M>(a, u.unit & 31);
    pf.r = -1;
    pf.width = 0;
    pf.off = 0;
    if (u.staged && cwarp < u.nsl) {
        int pre = 0;
#pragma unroll
        for (int q = 0; q < kRecSlices; ++q) pre += (q < cwarp) ? slice_width(u.widths, q) : 0;
        pf.width = slice_width(u.widths, cwarp);
        pf.off = 32 * pre + lane;
        const int r = u.row0 + 32 * cwarp + lane;
        if (r < u.row1) pf.r = r;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int c = (pf.r >= 0 && q < pf.width) ? scol[pf.off + 32 * q] : -1;
#pragma unroll
        for (int i = 0; i < M; ++i) pf.x[q][i] = (c >= 0) ? xin[(int64_t)c * M + i] : 0.0;
    }
}

// phase B: finish unit pf (all of the warp's rows), then publish and release its slot
template <int M, int MODE, class VT>
__device__ __forceinline__ void phase_b(const KArgs &a, int32_t epoch, const Prefetch<M> &pf, const UnitInfo *s_u,
                                        const typename VT::T *sval0, const int32_t *scol0, int *s_done, uint64_t *s_empty,
                                        int cwarp, int lane) {
    constexpr int B = Batch<M>::B;
    const UnitInfo &u = s_u[pf.slot];
    const int k = pf.unit & 31;
    const double *xin = input_block<M>(a, k);
    const SVal<VT> sval{sval0 + pf.slot * kStageEntries};
    const int32_t *scol = kStageCol ? scol0 + pf.slot * kStageEntries : a.col + u.ebase;
    if (u.staged) {
        if (pf.r >= 0) {  // first slice: prefetched first batch, then the rest of the row
            double w[M];
#pragma unroll
            for (int i = 0; i < M; ++i) w[i] = 0.0;
#pragma unroll
            for (int q = 0; q < B; ++q) {
                if (q < pf.width && scol[pf.off + 32 * q] >= 0) {
                    const double v = sval[pf.off + 32 * q];
#pragma unroll
                    for (int i = 0; i < M; ++i) w[i] = fma(v, pf.x[q][i], w[i]);
                }
            }
            if (pf.width > B) row_sum_from<M, 2>(sval, scol, pf.off, B, pf.width, xin, w);  // rare: wide rows
            row_epilogue<M, MODE>(a, k, pf.r, w, xin);
            if (k == 1 && a.y0copy) {
#pragma unroll
                for (int i = 0; i < M; ++i) a.y0copy[(int64_t)pf.r * M + i] = a.x0[(int64_t)pf.r * M + i];
            }
        }
        for (int sl = cwarp + kCompWarps; sl < u.nsl; sl += kCompWarps) {  // further slices (wide chunks)
            const int64_t r = (int64_t)u.row0 + 32 * sl + lane;
            int pre = 0;
#pragma unroll
            for (int q = 0; q < kRecSlices; ++q) pre += (q < sl) ? slice_width(u.widths, q) : 0;
            if (r >= u.row1) continue;
            double w[M];
            row_sum<M, 2>(sval, scol, 32 * pre + lane, slice_width(u.widths, sl), xin, w);  // rare: wide chunks
            row_epilogue<M, MODE>(a, k, r, w, xin);
            if (k == 1 && a.y0copy) {
#pragma unroll
                for (int i = 0; i < M; ++i) a.y0copy[r * M + i] = a.x0[r * M + i];
            }
        }
    } else {  // entries in global memory (chunk too large to stage)
        for (int sl = cwarp; sl < u.nsl; sl += kCompWarps) {
            const int64_t r = (int64_t)u.row0 + 32 * sl + lane;
            if (r >= u.row1) continue;
            const int64_t s0 = __ldg(a.slice_ptr + u.slice0 + sl), s1 = __ldg(a.slice_ptr + u.slice0 + sl + 1);
            double w[M];
            constexpr int BU = kUnstagedBatch < Batch<M>::B ? kUnstagedBatch : Batch<M>::B;
            row_sum<M, BU>(GVal<VT>{static_cast<const typename VT::T *>(a.val) + u.ebase}, GCol{a.col + u.ebase},
                           s0 - u.ebase + lane, (int)((s1 - s0) >> 5), xin, w);
            row_epilogue<M, MODE>(a, k, r, w, xin);
            if (k == 1 && a.y0copy) {
#pragma unroll
                for (int i = 0; i < M; ++i) a.y0copy[r * M + i] = a.x0[r * M + i];
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        // the last compute warp to finish the unit publishes it (release at gpu scope after
        // the other warps' stores were ordered at block scope), then the slot is released
        __threadfence_block();
        if (atomicAdd(&s_done[pf.slot], 1) == kCompWarps - 1) {
            s_done[pf.slot] = 0;
            fence_acq_rel_gpu();
            if (pf.unit != a.drop_unit)
                st_relaxed(a.flags + (int64_t)k * a.nchunks + (pf.unit >> 5), epoch);
        }
        mbar_arrive(&s_empty[pf.slot]);
    }
}

// dependency flags v0 .. v0+127 of a unit (4 per lane); flags past `total` read as ready
__device__ __forceinline__ void dep_load(const KArgs &a, int32_t epoch, int k, const int (&lo)[kDepRanges],
                                         const int (&len)[kDepRanges], int total, int v0, int lane, int (&got)[4]) {
    const int32_t *f = a.flags + (int64_t)(k - 1) * a.nchunks;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int v = v0 + 32 * q + lane;
        int idx = -1;
        if (v < total) {
#pragma unroll
            for (int r = 0; r < kDepRanges; ++r) {
                if (idx < 0 && v < len[r]) idx = lo[r] + v;
                if (idx < 0) v -= len[r];
            }
        }
        got[q] = idx >= 0 ? ld_relaxed(f + idx) : epoch;
    }
}

// all lanes of the control warp: true when every flag of the unit's ranges equals epoch
__device__ __forceinline__ bool deps_ready(const KArgs &a, int32_t epoch, int k, const int (&lo)[kDepRanges],
                                           const int (&len)[kDepRanges], int total, int lane) {
    bool ok = true;
    for (int v0 = 0; v0 < total; v0 += 128) {
        int got[4];
        dep_load(a, epoch, k, lo, len, total, v0, lane, got);
#pragma unroll
        for (int q = 0; q < 4; ++q) ok = ok && got[q] == epoch;
    }
    return __all_sync(0xffffffffu, ok);
}

// dependency ranges of a chunk record (ints 8..15, shuffled from the lanes holding them)
__device__ __forceinline__ int dep_ranges_of(int rec, int (&lo)[kDepRanges], int (&len)[kDepRanges]) {
    int total = 0;
#pragma unroll
    for (int r = 0; r < kDepRanges; ++r) {
        lo[r] = __shfl_sync(0xffffffffu, rec, 8 + 2 * r);
        len[r] = max(0, __shfl_sync(0xffffffffu, rec, 9 + 2 * r) - lo[r] + 1);
        total += len[r];
    }
    return total;
}

template <int M, int MODE, bool TRACE, class VT>
__global__ void __launch_bounds__(kBS, (MpkOcc<M, MODE, TRACE>::blocks)) k_mpk(const KArgs a) {
    using T = typename VT::T;
    const bool tr = TRACE && a.trace != nullptr;  // timing counters (instantiated separately)
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_full[kSlots];
    __shared__ __align__(8) uint64_t s_empty[kSlots];
    __shared__ UnitInfo s_u[kSlots];
    __shared__ volatile int s_final;  // units handed over in total; -1 while the control warp runs
    __shared__ int s_done[kSlots];    // compute warps finished with the slot's unit
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T *const sval0 = reinterpret_cast<T *>(smem);
    int32_t *const scol0 = reinterpret_cast<int32_t *>(smem + kSlots * kStageEntries * sizeof(T));

    const uint64_t t_start = tr ? globaltimer() : 0;
    // trace counters (see mpk_read_trace); s_tarr: time of each slot's last hand-over
    __shared__ unsigned long long s_tr[kTraceShared];
    __shared__ unsigned long long s_tarr[kSlots];
    auto tr_add = [&](int q, unsigned long long v) {
        if (tr) atomicAdd(&s_tr[q], v);
    };
    const long long c_start = tr ? clock64() : 0;
    if (tid < kTraceShared) s_tr[tid] = 0;
    // Epochs live on the device, so that launches replayed from a CUDA graph stay distinct:
    // the last block of a launch stores its epoch, the next launch uses that plus one.
    __shared__ int32_t s_epoch;
    if (tid == 0) {
        s_epoch = (int32_t)ld_relaxed(reinterpret_cast<const int32_t *>(a.epoch_word)) + 1;
        s_final = -1;
        for (int q = 0; q < kSlots; ++q) {
            s_done[q] = 0;
            mbar_init(&s_full[q], 1);
            mbar_init(&s_empty[q], kCompWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int32_t epoch = s_epoch;

    if (warp == 0) {
        // ------------------------------------------------------------------ control warp
        const int32_t *rec = reinterpret_cast<const int32_t *>(a.chunk_rec);
        bool slot_busy[kSlots] = {};  // a handed-over unit may still be computed
        int slot_use[kSlots] = {};    // phase index (i / kSlots) of that hand-over
        bool aborted = false;
        auto record_timeout = [&]() {
            if (lane == 0 && atomicExch(a.err, epoch) != epoch) st_relaxed(a.err + 1, (int)MPK_ERR_TIMEOUT);
        };
        auto unit_at = [&](unsigned int t) -> int { return (int64_t)t < a.nunits ? __ldg(a.units + t) : -1; };
        // claim pipeline, three units deep: unit i (id u_cur, record r_cur), unit i+1 (u_nxt,
        // r_nxt), unit i+2 (id u_nn, held by lane 0) and the ticket t of unit i+3.  At the end
        // of iteration i the record of unit i+2, the id of unit i+3 and one more ticket are
        // fetched, each a full iteration before it is needed.
        auto rec_at = [&](int un) -> int {
            return (un >= 0 && lane < kRecInts) ? __ldg(rec + kRecInts * (int64_t)(un >> 5) + lane) : 0;
        };
        int u_cur = -1, u_nxt = -1, u_nn = -1;
        unsigned int t = 0;
        if (lane == 0) {
            const unsigned int t0 = atomicAdd(a.ticket, 1u);
            const unsigned int t1 = atomicAdd(a.ticket, 1u);
            const unsigned int t2 = atomicAdd(a.ticket, 1u);
            t = atomicAdd(a.ticket, 1u);
            u_cur = unit_at(t0);
            u_nxt = unit_at(t1);
            u_nn = unit_at(t2);
        }
        u_cur = __shfl_sync(0xffffffffu, u_cur, 0);
        u_nxt = __shfl_sync(0xffffffffu, u_nxt, 0);
        int r_cur = rec_at(u_cur);
        int r_nxt = rec_at(u_nxt);
        int i = 0;
        for (;; ++i) {
            if (u_cur < 0) break;  // no more work
            const int b = i % kSlots;
            const long long c0 = tr ? clock64() : 0;
            // current unit
            UnitInfo u;
            u.unit = u_cur;
            u.row0 = __shfl_sync(0xffffffffu, r_cur, 0);
            u.row1 = __shfl_sync(0xffffffffu, r_cur, 1);
            u.slice0 = __shfl_sync(0xffffffffu, r_cur, 2);
            u.ecount = __shfl_sync(0xffffffffu, r_cur, 3);
            u.ebase = (long long)(unsigned int)__shfl_sync(0xffffffffu, r_cur, 4) |
                      ((long long)__shfl_sync(0xffffffffu, r_cur, 5) << 32);
            u.staged = __shfl_sync(0xffffffffu, r_cur, 6);
            u.nsl = __shfl_sync(0xffffffffu, r_cur, 7);
#pragma unroll
            for (int q = 0; q < 4; ++q) u.widths[q] = __shfl_sync(0xffffffffu, r_cur, 16 + q);
            int dlo[kDepRanges], dlen[kDepRanges];
            const int total = dep_ranges_of(r_cur, dlo, dlen);
            if (tr && lane == 0) tr_add(11, clock64() - c0);
            // slot b held unit i-kSlots: wait until it is computed before reusing the slot
            if (slot_busy[b]) {
                const uint64_t t0 = globaltimer();
                bool ok;
                while (!(ok = mbar_try_wait(&s_empty[b], slot_use[b] & 1)))
                    if (timed_out(t0, a.wait_ns)) break;
                if (tr && lane == 0) tr_add(3, globaltimer() - t0);
                if (!ok) {
                    record_timeout();
                    aborted = true;
                    break;
                }
                slot_busy[b] = false;
            }
            // stage the entries
            const long long c2 = tr ? clock64() : 0;
            if (lane == 0) {
                s_u[b] = u;
                if (u.staged) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx_only(&s_full[b], (uint32_t)u.ecount * (uint32_t)(sizeof(T) + (kStageCol ? 4 : 0)));
                    bulk_g2s(sval0 + b * kStageEntries, static_cast<const T *>(a.val) + u.ebase,
                             (uint32_t)(u.ecount * sizeof(T)), &s_full[b]);
                    if (kStageCol)
                        bulk_g2s(scol0 + b * kStageEntries, a.col + u.ebase, (uint32_t)u.ecount * 4u, &s_full[b]);
                }
            }
            if (tr && lane == 0) tr_add(8, clock64() - c2);
            // dependencies of unit i
            const int k = u.unit & 31;
            if (k > 1) {
                const uint64_t t0 = globaltimer();
                while (!deps_ready(a, epoch, k, dlo, dlen, total, lane)) {
                    if (lane == 0) tr_add(2, 1);
                    const bool stop = ld_relaxed(a.err) == epoch || timed_out(t0, a.wait_ns);
                    if (__any_sync(0xffffffffu, stop)) {
                        aborted = true;
                        break;
                    }
                    __nanosleep(32);
                }
                if (tr && lane == 0) tr_add(1, globaltimer() - t0);
            }
            if (lane == 0) tr_add(0, 1);
            if (aborted) {
                // unit i is not handed over: the compute warps stop before it.  Complete the
                // slot's phase so that its bulk copy can be waited for, then wait for it.
                record_timeout();
                if (lane == 0) {
                    s_final = i;
                    mbar_arrive(&s_full[b]);
                }
                if (u.staged) {
                    const uint64_t t1 = globaltimer();
                    while (!mbar_try_wait(&s_full[b], (i / kSlots) & 1))
                        if (timed_out(t1, a.wait_ns)) break;
                }
                break;
            }
            const long long c4 = tr ? clock64() : 0;
            fence_acq_rel_gpu();  // acquire: flags before the compute warps' reads (via full[b])
            __syncwarp();
            if (tr && lane == 0) s_tarr[b] = globaltimer();
            if (lane == 0) mbar_arrive(&s_full[b]);
            const long long c5 = tr ? clock64() : 0;
            if (tr && lane == 0) tr_add(9, c5 - c4);
            slot_busy[b] = true;
            slot_use[b] = i / kSlots;
            // prefetch after the hand-over, so that these loads and the atomic complete during
            // the next units' staging and polls instead of delaying this unit's fence
            const int u2 = __shfl_sync(0xffffffffu, u_nn, 0);
            const int r2 = rec_at(u2);
            int u3 = -1;
            unsigned int t_next = t;
            if (lane == 0) {
                u3 = unit_at(t);                   // id of unit i+3
                t_next = atomicAdd(a.ticket, 1u);  // ticket of unit i+4, claimed whether or not it exists
            }
            u_cur = u_nxt;
            r_cur = r_nxt;
            u_nxt = u2;
            r_nxt = r2;
            u_nn = u3;
            t = t_next;
            if (tr && lane == 0) tr_add(10, clock64() - c5);
        }
        if (lane == 0 && s_final < 0) s_final = i;  // units 0..i-1 were handed over
    } else {
        // ------------------------------------------------------------------ compute warps
        const int cw = warp - 1;
        Prefetch<M> pf;
        pf.unit = -1;
        for (int i = 0;; ++i) {
            const int b = i % kSlots;
            // Each lane waits for itself; whichever iteration a lane leaves the loop in, every
            // lane then runs the same phases of the same unit (one __syncwarp each), so the
            // warp's lanes never hold different units.
            const uint64_t t0 = globaltimer();
            bool got = false, stop = false;
            while (true) {
                if (mbar_try_wait(&s_full[b], (i / kSlots) & 1)) {
                    got = true;
                    break;
                }
                const int fin = s_final;
                if (fin >= 0 && i >= fin) {
                    stop = true;
                    break;
                }
                if (timed_out(t0, 2 * a.wait_ns + 100000000LL)) break;
            }
            if (got) {
                const int fin = s_final;  // set before the hand-over of an aborted unit
                if (fin >= 0 && i >= fin) stop = true;
            }
            if (stop) break;
            if (!got) {  // the control warp gave no sign of life: give up
                if (lane == 0 && atomicExch(a.err, epoch) != epoch) st_relaxed(a.err + 1, (int)MPK_ERR_TIMEOUT);
                break;
            }
            uint64_t t_got = 0;
            if (tr) {
                t_got = globaltimer();
                if (lane == 0) tr_add(4, t_got - t0);
                if (lane == 0 && cw == 0 && t_got - t0 > 1000) {  // waited: how long after the hand-over
                    const unsigned long long ta = s_tarr[b];
                    tr_add(14, t_got > ta ? t_got - ta : 0);
                    tr_add(15, 1);
                }
            }
            {
                const long long c0 = tr ? clock64() : 0;
                phase_a<M>(a, s_u[b], b, kStageCol ? scol0 + b * kStageEntries : a.col + s_u[b].ebase, cw, lane, pf);
                if (tr) {  // wait for the gathers (integer ops only) to split the unit time
                    int h = 0;
#pragma unroll
                    for (int q = 0; q < Batch<M>::B; ++q) h ^= __double2hiint(pf.x[q][0]);
                    int d;
                    asm volatile("add.u32 %0, %1, 0;" : "=r"(d) : "r"(h));
                    const long long c1 = clock64();
                    if (lane == 0) tr_add(12, c1 - c0);
                    phase_b<M, MODE, VT>(a, epoch, pf, s_u, sval0, scol0, s_done, s_empty, cw, lane);
                    if (lane == 0) tr_add(13, clock64() - c1);
                } else {
                    phase_b<M, MODE, VT>(a, epoch, pf, s_u, sval0, scol0, s_done, s_empty, cw, lane);
                }
                pf.unit = -1;
            }
            if (tr && lane == 0) tr_add(5, globaltimer() - t_got);
        }
    }
    if (tr) {
        __syncthreads();
        if (tid == 0) {
            s_tr[6] = globaltimer() - t_start;
            s_tr[7] = blockIdx.x == 0;
            for (int q = 0; q < kTraceShared; ++q) atomicAdd(a.trace + q, s_tr[q]);
            atomicAdd(a.trace + kTraceShared, (unsigned long long)(clock64() - c_start));
        }
    }
    // ---- exit: the last block resets the ticket and stores the epoch for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.exit_count, 1u);
        if (done == gridDim.x - 1) {
            *a.ticket = 0u;
            *a.exit_count = 0u;
            *a.epoch_word = (unsigned int)epoch;
            __threadfence();
        }
    }
}

// ----------------------------------------------------------------------------- K-MPK, warp engine
// The same cells (group g, local power k) in the same order as k_mpk (lines g + kSlotSkew*k
// ascending, k ascending inside a line), split into items of kWarpSlices 32-row slices and
// numbered in that order.  Every warp works alone: warp q of each block claims the items
// q, q + Q, q + 2Q, ... (Q = kWarpQueues) through the claim counter of queue q, so that any
// resident block serves every queue; it waits until the cells (g-1, k-1), (g, k-1) and
// (g+1, k-1) have all their items finished (acquire), computes its slices with the entries
// read from global memory (L2, where the line order keeps the working set), and adds one
// to its cell's counter (release).
// No deadlock: take the smallest claimed, unfinished item m.  Each of its dependencies x < m
// is finished: a claimed x would be held by a warp with an unfinished item below m, and an
// unclaimed x of queue q would lie above every item claimed from q, although the queue-q warp
// of m's block holds an unfinished item of q, which is at least m.  Claims run one item
// ahead; the argument holds for the items being computed.  Every wait is bounded by
// a.wait_ns; on expiry the warp records the epoch and MPK_ERR_TIMEOUT in a.err and leaves,
// and the others leave when they see the error.
// blocks of kWarpBS threads per SM the register budget is set for (no spills)
template <int M, int MODE, class VT> struct WarpOcc {
    static constexpr bool f64 = sizeof(typename VT::T) == 8;
    static constexpr int blocks = !f64 || M > 2 ? 2 : (M == 1 && MODE == 0 ? 4 : 3);
};
constexpr int kWarpBS = 32 * kWarpQueues;

template <int M, int MODE, class VT>
__global__ void __launch_bounds__(kWarpBS, (WarpOcc<M, MODE, VT>::blocks)) k_mpkw(const KArgs a) {
    constexpr int B = Batch<M>::B;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    __shared__ int32_t s_epoch;
    if (threadIdx.x == 0) s_epoch = ld_relaxed(reinterpret_cast<const int32_t *>(a.epoch_word)) + 1;
    __syncthreads();
    const int32_t epoch = s_epoch;
    const auto *val = static_cast<const typename VT::T *>(a.val);
    // lane 0 holds the pending claims (queue positions) of the current and the next item
    unsigned int c_now = 0, c_next = 0;
    if (lane == 0) {
        c_now = atomicAdd(a.w_q + q, 1u);
        c_next = atomicAdd(a.w_q + q, 1u);
    }
    int64_t cell = 0;
    bool failed = false;
    for (;;) {
        const int64_t it = (int64_t)__shfl_sync(0xffffffffu, c_now, 0) * kWarpQueues + q;
        if (it >= a.w_nitems) break;
        // the item's cell: the last one whose first item is <= it (the warp's items ascend)
        for (;;) {
            const int64_t cc = cell + 1 + lane;
            const bool le = cc < a.w_ncells && __ldg(a.w_item + cc) <= it;
            const unsigned int bal = __ballot_sync(0xffffffffu, le);
            cell += __popc(bal);
            if (bal != 0xffffffffu) break;
        }
        const int gk = __ldg(a.w_gk + cell);
        const int g = gk >> 5, k = gk & 31;
        const int j = (int)(it - __ldg(a.w_item + cell));
        const int gs0 = __ldg(a.g_slice + g), gs1 = __ldg(a.g_slice + g + 1);
        const int gr0 = __ldg(a.g_row + g), gr1 = __ldg(a.g_row + g + 1);
        const int s_first = gs0 + j * kWarpSlices, s_end = min(s_first + kWarpSlices, gs1);
        const int c = __ldg(a.w_slice_chunk + s_first);  // items never leave a chunk (one slice)
        if (k > 1) {
            // the chunks this chunk's rows read (its dependency ranges) must have all their
            // slices finished at power k-1
            const int rv = lane < kRecInts ? __ldg(reinterpret_cast<const int32_t *>(a.chunk_rec) +
                                                   (int64_t)kRecInts * c + lane)
                                           : 0;
            int dlo[kDepRanges], dlen[kDepRanges];
            const int total = dep_ranges_of(rv, dlo, dlen);
            const int32_t *cnt = a.w_cnt + (int64_t)(k - 1) * a.nchunks;
            const uint64_t t0 = globaltimer();
            for (int v0 = 0; v0 < total && !failed; v0 += 32) {
                int v = v0 + lane, idx = -1;
                if (v < total) {
#pragma unroll
                    for (int r = 0; r < kDepRanges; ++r) {
                        if (idx < 0 && v < dlen[r]) idx = dlo[r] + v;
                        if (idx < 0) v -= dlen[r];
                    }
                }
                const int ns = idx >= 0 ? __ldg(a.w_chunk_nsl + idx) : 0;
                const int need = (ns >> 24) >= k - 1 ? (ns & 0xffffff) : 0;
                for (;;) {
                    const bool ok = idx < 0 || ld_relaxed(cnt + idx) >= need;
                    if (__all_sync(0xffffffffu, ok)) break;
                    const bool stop = ld_relaxed(a.err) == epoch || timed_out(t0, a.wait_ns);
                    if (__any_sync(0xffffffffu, stop)) {
                        failed = true;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (failed) break;
            fence_acq_rel_gpu();  // acquire: the neighbours' rows before this warp's reads
            __syncwarp();
        }
        const double *xin = input_block<M>(a, k);
        for (int sl = s_first; sl < s_end; ++sl) {
            const int64_t r = (int64_t)gr0 + 32 * (sl - gs0) + lane;
            if (r < gr1) {
                const int64_t e0 = __ldg(a.slice_ptr + sl), e1 = __ldg(a.slice_ptr + sl + 1);
                double w[M];
                row_sum<M, B>(GVal<VT>{val}, GCol{a.col}, e0 + lane, (int)((e1 - e0) >> 5), xin, w);
                row_epilogue<M, MODE>(a, k, r, w, xin);
                if (k == 1 && a.y0copy) {
#pragma unroll
                    for (int i = 0; i < M; ++i) a.y0copy[r * M + i] = a.x0[r * M + i];
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            fence_acq_rel_gpu();  // release: this warp's rows before the count
            atomicAdd(a.w_cnt + (int64_t)k * a.nchunks + c, 1);
        }
        c_now = c_next;
        if (lane == 0) c_next = atomicAdd(a.w_q + q, 1u);
    }
    if (failed && lane == 0 && atomicExch(a.err, epoch) != epoch) st_relaxed(a.err + 1, (int)MPK_ERR_TIMEOUT);
    // ---- exit: the last block stores the epoch for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.exit_count, 1u);
        if (done == gridDim.x - 1) {
            *a.exit_count = 0u;
            *a.epoch_word = (unsigned int)epoch;
            __threadfence();
        }
    }
}

// ----------------------------------------------------------------------------- K-SpMV
// SpMV restricted to row ranges of one or several plans (plan order), one launch: segment
// q covers the plan-order rows [lo, hi) of its plan, whose chunks c0 .. c0+nch-1 overlap
// them; virtual block v belongs to the segment q with first[q] <= v < first[q+1].
template <int M, class VT>
__global__ void __launch_bounds__(kSpmvBS) k_spmv_rows(const RowSegs segs) {
    const int lane = threadIdx.x & 31;
    for (int v = blockIdx.x; v < segs.first[segs.count]; v += gridDim.x) {
        int q = 0;
        while (v >= segs.first[q + 1]) ++q;
        const RowSeg &g = segs.seg[q];
        const auto *val = static_cast<const typename VT::T *>(g.val);
        const int c = g.c0 + (v - segs.first[q]);
        const int r0 = g.chunk_row[c], r1 = g.chunk_row[c + 1], sl0 = g.chunk_slice[c];
        const int nsl = (r1 - r0 + 31) >> 5;
        for (int sl = threadIdx.x >> 5; sl < nsl; sl += kSpmvBS / 32) {
            const int64_t r = (int64_t)r0 + 32 * sl + lane;
            if (r < r1 && r >= g.lo && r < g.hi) {
                const int64_t s0 = g.slice_ptr[sl0 + sl], s1 = g.slice_ptr[sl0 + sl + 1];
                double w[M];
                row_sum<M, Batch<M>::B>(GVal<VT>{val}, GCol{g.col}, s0 + lane, (int)((s1 - s0) >> 5), g.x, w);
#pragma unroll
                for (int i = 0; i < M; ++i) g.y[r * M + i] = w[i];
            }
        }
    }
}

template <class VT>
static void launch_spmv_rows_vt(const RowSegs &segs, int m, cudaStream_t s) {
    const int grid = std::min(segs.first[segs.count], 64 * device_sms());
#define L(MM)                                                 \
    case MM:                                                  \
        k_spmv_rows<MM, VT><<<grid, kSpmvBS, 0, s>>>(segs);   \
        break;
    switch (m) {
        L(1) L(2) L(4) L(8) default : fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
    }
#undef L
    MPK_LAUNCHED();
}

void launch_spmv_rows(const Plan *const *plans, const int32_t *lo, const int32_t *hi, const double *const *x,
                      double *const *y, int count, cudaStream_t s) {
    RowSegs segs{};
    segs.first[0] = 0;
    int vt = -1, m = 0;
    for (int i = 0; i < count; ++i) {
        const Plan &P = *plans[i];
        if (hi[i] <= lo[i]) continue;
        if (vt < 0) {
            vt = P.val_type;
            m = P.m;
        }
        // chunks overlapping [lo, hi): h_chunk_row is ascending, from 0 to n
        const auto &cr = P.h_chunk_row;
        const int32_t c0 = (int32_t)(std::upper_bound(cr.begin(), cr.end(), lo[i]) - cr.begin()) - 1;
        const int32_t c1 = (int32_t)(std::lower_bound(cr.begin(), cr.end(), hi[i]) - cr.begin());
        RowSeg &g = segs.seg[segs.count];
        g.val = P.val;
        g.col = P.col;
        g.slice_ptr = P.slice_ptr;
        g.chunk_row = P.chunk_row;
        g.chunk_slice = P.chunk_slice;
        g.x = x[i];
        g.y = y[i];
        g.c0 = c0;
        g.lo = lo[i];
        g.hi = hi[i];
        segs.first[segs.count + 1] = segs.first[segs.count] + (c1 - c0);
        ++segs.count;
    }
    if (segs.count == 0) return;
    if (vt == MPK_F64) return launch_spmv_rows_vt<ValF64>(segs, m, s);
    if (vt == MPK_F32) return launch_spmv_rows_vt<ValF32>(segs, m, s);
    return launch_spmv_rows_vt<ValBF16>(segs, m, s);
}

// dst[dst_idx[t]] = src[src_idx[t]], m doubles a row (the halo exchange between partitions
// held on one device)
__global__ void k_copy_rows(const double *src, const int64_t *src_idx, double *dst, const int64_t *dst_idx, int64_t n,
                            int32_t m) {
    const int64_t total = n * m, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t r = t / m, i = t - r * m;
        dst[dst_idx[r] * m + i] = src[src_idx[r] * m + i];
    }
}

void launch_copy_rows(const double *src, const int64_t *src_idx, double *dst, const int64_t *dst_idx, int64_t n,
                      int32_t m, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t total = n * m;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 16LL * device_sms());
    k_copy_rows<<<grid, 256, 0, s>>>(src, src_idx, dst, dst_idx, n, m);
    MPK_LAUNCHED();
}

// ----------------------------------------------------------------------------- row moves
// dst[r] = src[perm[r] - base] (m values per row; perm NULL: the identity); coalesced writes
__global__ void k_gather_rows(const double *src, const int32_t *perm, int32_t base, double *dst, int32_t n,
                              int32_t m) {
    const int64_t total = (int64_t)n * m, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t r = t / m, i = t - r * m;
        dst[t] = src[(int64_t)((perm ? perm[r] : (int32_t)r) - base) * m + i];
    }
}

// Chebyshev k = 0 term: acc = c0 * v0 (complex: pairs of columns)
__global__ void k_cheb_init(const double *v0, double *acc, int32_t n, int32_t m, double cr, double ci, int cplx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const double *v = v0 + r * m;
        double *o = acc + r * m;
        if (!cplx) {
            for (int i = 0; i < m; ++i) o[i] = cr * v[i];
        } else {
            for (int i = 0; i + 1 < m; i += 2) {
                double re = cr * v[i];
                re = fma(-ci, v[i + 1], re);
                double im = cr * v[i + 1];
                im = fma(ci, v[i], im);
                o[i] = re;
                o[i + 1] = im;
            }
        }
    }
}

static int grid_rows(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

void launch_gather_rows(const double *src, const int32_t *perm, double *dst, int32_t n, int32_t m, cudaStream_t s,
                        int32_t base) {
    if (n <= 0) return;
    k_gather_rows<<<grid_rows((int64_t)n * m), 256, 0, s>>>(src, perm, base, dst, n, m);
    MPK_LAUNCHED();
}

// dst[i] = src[iperm[i]]: scatter expressed as a gather by output row
void launch_scatter_rows(const double *src, const int32_t *iperm, double *dst, int32_t n, int32_t m, cudaStream_t s) {
    launch_gather_rows(src, iperm, dst, n, m, s);
}

// Y[k][i] = W[k][iperm[i]] for k = 1..p: the powers computed in plan order, written in the
// matrix's own order.  Stores are full, coalesced rows of the output; the gathered reads
// come from rows that neighbouring original rows map to (for a BFS order these sit a few
// levels apart and share cache sectors with the reads of nearby original rows).  One block
// per SM walks tiles of kScatterTile consecutive original rows, power by power, so that the
// sectors a tile reads stay in the SM's L1 until its other rows use them.
constexpr int kScatterBS = 1024, kScatterItems = 16, kScatterTile = kScatterBS * kScatterItems;

__global__ void __launch_bounds__(kScatterBS, 1)
    k_scatter_powers(const double *W, int64_t w_pstride, const int32_t *__restrict__ iperm, int32_t w_row0, double *Y,
                     int32_t n, int32_t m, int32_t p) {
    const int64_t nm = (int64_t)n * m;
    for (int64_t base = (int64_t)blockIdx.x * kScatterTile; base < n; base += (int64_t)gridDim.x * kScatterTile) {
        int32_t src[kScatterItems];
#pragma unroll
        for (int q = 0; q < kScatterItems; ++q) {
            const int64_t i = base + (int64_t)q * kScatterBS + threadIdx.x;
            src[q] = i < n ? (iperm ? __ldg(iperm + i) : w_row0 + (int32_t)i) : -1;
        }
        for (int k = 1; k <= p; ++k) {
            const double *w = W + k * w_pstride;
            double *y = Y + k * nm;
#pragma unroll
            for (int q = 0; q < kScatterItems; ++q) {
                const int64_t i = base + (int64_t)q * kScatterBS + threadIdx.x;
                if (src[q] >= 0)
                    for (int c = 0; c < m; ++c) y[i * m + c] = w[(int64_t)src[q] * m + c];
            }
        }
    }
}

void launch_scatter_powers(const double *W, const int32_t *iperm, double *Y, int32_t n, int32_t m, int32_t p,
                           cudaStream_t s, int64_t w_pstride, int32_t base) {
    if (n <= 0 || p <= 0) return;
    if (w_pstride < 0) w_pstride = (int64_t)n * m;
    k_scatter_powers<<<device_sms(), kScatterBS, 0, s>>>(W, w_pstride, iperm, base, Y, n, m, p);
    MPK_LAUNCHED();
}

void launch_cheb_init(const double *v0, double *acc, int32_t n, int32_t m, double c0re, double c0im, int cplx,
                      cudaStream_t s) {
    if (n <= 0) return;
    k_cheb_init<<<grid_rows(n), 256, 0, s>>>(v0, acc, n, m, c0re, c0im, cplx);
    MPK_LAUNCHED();
}

// ----------------------------------------------------------------------------- launches
template <int M, int MODE, class VT> static void *mpk_fn(bool trace) {
    return trace ? (void *)k_mpk<M, MODE, true, VT> : (void *)k_mpk<M, MODE, false, VT>;
}

template <class VT> static void *select_mpk_vt(int mode, int m, bool trace) {
#define SEL(MM)                                                             \
    if (m == MM) {                                                          \
        if (mode == MODE_POWERS) return mpk_fn<MM, MODE_POWERS, VT>(trace); \
        return mpk_fn<MM, MODE_CHEB, VT>(trace);                            \
    }
    SEL(1) SEL(2) SEL(4) SEL(8)
#undef SEL
    fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
}

static void *select_mpk(int mode, int m, bool trace, int vtype) {
    if (vtype == MPK_F64) return select_mpk_vt<ValF64>(mode, m, trace);
    if (vtype == MPK_F32) return select_mpk_vt<ValF32>(mode, m, trace);
    if (vtype == MPK_BF16) return select_mpk_vt<ValBF16>(mode, m, trace);
    fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
}

static int mpk_smem_bytes(int vtype) {
    return vtype == MPK_F64 ? smem_bytes<ValF64>() : (vtype == MPK_F32 ? smem_bytes<ValF32>() : smem_bytes<ValBF16>());
}

int occupancy_grid(int mode, int m, bool trace, int vtype) {
    static int cache[3][2][2][9] = {};
    if (vtype < 0 || vtype > 2) fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
    int &c = cache[vtype][mode][trace ? 1 : 0][m];
    if (c) return c;
    void *fn = select_mpk(mode, m, trace, vtype);
    const int smem = mpk_smem_bytes(vtype);
    MPK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBS, smem));
    if (per_sm < 1) fail(MPK_ERR_CUDA, "level-blocked kernel cannot be resident (occupancy 0)");
    c = per_sm * device_sms();
    return c;
}

template <class VT> static void *select_mpkw_vt(int mode, int m) {
#define SEL(MM)                                                                              \
    if (m == MM) return mode == MODE_POWERS ? (void *)k_mpkw<MM, MODE_POWERS, VT> : (void *)k_mpkw<MM, MODE_CHEB, VT>;
    SEL(1) SEL(2) SEL(4) SEL(8)
#undef SEL
    fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
}

static void *select_mpkw(int mode, int m, int vtype) {
    if (vtype == MPK_F64) return select_mpkw_vt<ValF64>(mode, m);
    if (vtype == MPK_F32) return select_mpkw_vt<ValF32>(mode, m);
    if (vtype == MPK_BF16) return select_mpkw_vt<ValBF16>(mode, m);
    fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
}

static int occupancy_grid_w(int mode, int m, int vtype) {
    static int cache[3][2][9] = {};
    if (vtype < 0 || vtype > 2 || m < 1 || m > 8) fail(MPK_ERR_UNSUPPORTED, "value type %d, nrhs %d", vtype, m);
    int &c = cache[vtype][mode][m];
    if (c) return c;
    int per_sm = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_mpkw(mode, m, vtype), kWarpBS, 0));
    if (per_sm < 1) fail(MPK_ERR_CUDA, "warp-engine kernel cannot be resident (occupancy 0)");
    c = per_sm * device_sms();
    return c;
}

void launch_mpk(const Plan &P, KArgs &a, int mode, cudaStream_t s) {
    if (a.w_item != nullptr && a.trace == nullptr && a.drop_unit < 0) {  // warp engine
        if (a.w_nitems <= 0) return;
        MPK_CUDA(cudaMemsetAsync(a.w_cnt, 0,
                                 sizeof(int32_t) * ((size_t)(P.p_max + 1) * std::max(P.num_chunks, 1) + kWarpQueues),
                                 s));
        int grid = occupancy_grid_w(mode, P.m, P.val_type);
        const int64_t warps_needed = (a.w_nitems + kWarpQueues - 1) / kWarpQueues;
        if ((int64_t)grid > warps_needed) grid = (int)warps_needed;
        void *args[] = {&a};
        MPK_CUDA(cudaLaunchKernel(select_mpkw(mode, P.m, P.val_type), dim3(grid), dim3(kWarpBS), args, 0, s));
        return;
    }
    if (a.nunits <= 0) return;
    const bool trace = a.trace != nullptr;
    int grid = occupancy_grid(mode, P.m, trace, P.val_type);
    if ((int64_t)grid > a.nunits) grid = (int)a.nunits;
    void *fn = select_mpk(mode, P.m, trace, P.val_type);
    void *args[] = {&a};
    MPK_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kBS), args, mpk_smem_bytes(P.val_type), s));
}

// One plain SpMV over the plan's sliced copy, y = A x (plan order): the row-range kernel
// over all rows.
void launch_spmv(const Plan &P, const double *x, double *y, cudaStream_t s) {
    if (P.num_chunks <= 0 || P.n <= 0) return;
    const Plan *pp = &P;
    const int32_t lo = 0, hi = P.n;
    launch_spmv_rows(&pp, &lo, &hi, &x, &y, 1, s);
}

// ----------------------------------------------------------------------------- probes
__global__ void k_probe_load(const int4 *__restrict__ p, int64_t n16, int reps, int32_t *sink) {
    int acc = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = tid; i < n16; i += nt) {
            const int4 v = __ldcg(p + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x5eed1234) *sink = acc;
}

__global__ void k_probe_dfma(int iters, double *sink) {
    double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
           a7 = a0 + 7;
    const double b = 1.0000001, c = 1e-9;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == 123.456) *sink = s;
}

void probe_load(const void *buf, int64_t bytes, int reps, int ctas_per_sm, int32_t *sink, cudaStream_t s) {
    if (!buf || !sink || bytes <= 0 || bytes % 16 || reps < 1 || ctas_per_sm < 1 || ctas_per_sm > 64)
        fail(MPK_ERR_INVALID, "probe_load: bad arguments");
    k_probe_load<<<device_sms() * ctas_per_sm, 512, 0, s>>>(static_cast<const int4 *>(buf), bytes / 16, reps, sink);
    MPK_LAUNCHED();
}

void probe_dfma(int blocks, int iters, double *sink, cudaStream_t s) {
    if (!sink || blocks < 1 || iters < 1) fail(MPK_ERR_INVALID, "probe_dfma: bad arguments");
    k_probe_dfma<<<blocks, 256, 0, s>>>(iters, sink);
    MPK_LAUNCHED();
}

}  // namespace mpk
