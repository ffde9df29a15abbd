// Device code shared by the translation units of the level-blocked kernel: constants,
// synchronisation helpers, value types, the row body and the persistent kernel k_mpk.
// mpk_kernel.cu includes it for the warp engine, the SpMV and the launches; each
// mpk_kshape<N>.cu instantiates k_mpk for block shape N, so that the shapes compile in
// parallel.
#pragma once
#include "mpk_internal.h"

#include <algorithm>
#include <type_traits>

namespace mpk {

// level-blocked kernel of block shape SH: one control warp and the shape's compute warps
template <int SH> struct Shape {
    static constexpr int CW = kShapes[SH].comp_warps;
    static constexpr int SE = kShapes[SH].stage_entries;
    static constexpr int BS = 32 * (kShapes[SH].ctrl_warps + 1 + CW);  // control, publisher, compute
    static constexpr int SL = kShapes[SH].slots;    // staging slots
    static constexpr int CTL = kShapes[SH].ctrl_warps;  // control warps: 1, or 2 (poll + stage)
    static constexpr int XW = kShapes[SH].x_words;  // input-row words per slot (0: not staged)
    static constexpr bool X = XW > 0;
    static constexpr int SPW = kShapes[SH].slices_per_warp > 1 ? kShapes[SH].slices_per_warp : 1;
    static constexpr int NW = SPW > 1 ? 8 : 4;  // width words of the chunk record it reads
};
// blocks per SM the register budget is set for (65536 registers per SM).  The single-vector
// power kernel runs at the shape's own block count (shape 0: three blocks of 15 warps, 40
// registers a thread; shape 1: two of 18, 56 registers).  Wider blocks, the Chebyshev
// recurrence and the traced kernel run two blocks; the unstaged shape with 4 or more
// right-hand sides runs one block of 96 registers, whose rows of 4-8 columns would spill at
// two (measured: 27-point stencil 100^3, bfloat16, 8 columns, p = 8: 3.88 against 4.88 ms;
// the staged shapes lose at one block: 6.74 against 4.94 ms).
template <int M, int MODE, bool TRACE, int SH> struct MpkOcc {
    static constexpr int blocks = Shape<SH>::X ? kShapes[SH].blocks
                                  : (M == 1 && MODE != 1 /* not the recurrence */ && !TRACE) ? kShapes[SH].blocks
                                  : (Shape<SH>::SE == 0 && M >= 4) ? 1
                                                                    : 2;
};
constexpr int kSpmvBS = 256;        // threads per block of the plain SpMV kernel
// Staging slots (Shape::SL): the control warp fills one while the compute warps work on another.
constexpr int kMaxSlots = 4;
// column indices of staged chunks: copied to shared memory beside the values (1), or read
// from global memory (L2) by the compute warps (0), which halves the slot size for FP64
#ifndef MPK_STAGE_COL
#define MPK_STAGE_COL 1
#endif
constexpr bool kStageCol = MPK_STAGE_COL != 0;
// dynamic shared memory: per slot the shape's stage entries of the matrix's value type, then
// as many column indices (int32; shape 3: 16-bit window positions), then shape 3's input-row
// window area (x_words doubles)
template <class VT, int SH> constexpr int smem_bytes() {
    return Shape<SH>::X ? Shape<SH>::SL * (Shape<SH>::SE * (int)(sizeof(typename VT::T) + 2) + 8 * Shape<SH>::XW)
                        : Shape<SH>::SL * Shape<SH>::SE * (int)(sizeof(typename VT::T) + (kStageCol ? 4 : 0));
}

// MODE_HOST: the powers, each row also stored into host memory (a.yhost) as its unit finishes
enum Mode { MODE_POWERS = 0, MODE_CHEB = 1, MODE_HOST = 2 };


__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// 1: the dependency poll loads its flags with acquire semantics (ld.acquire.gpu) and no fence
// follows it; 0: relaxed loads, then one acquire fence per polled unit.  With 1, the lane that
// read a flag synchronises with the release of the block that set it; the warp barrier then
// orders that lane before lane 0's arrival on the slot's mbarrier (a CTA-scope release), which
// the compute warps acquire before they read x, so the producer's rows are visible to them.
// Measured 3.4 % faster at 256^3 (one fence per unit fewer on the control warp's path).
#ifndef MPK_ACQ_POLL
#define MPK_ACQ_POLL 1
#endif
constexpr bool kAcquirePoll = MPK_ACQ_POLL != 0;
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
__device__ __forceinline__ void bulk_g2s_addr(uint32_t dst, uint64_t src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    bulk_g2s_addr(smem_u32(dst), (uint64_t)src, bytes, bar);
}
// The same copy with an L2 priority: evict_first marks the lines the first to leave L2 (the
// last use of data inside a launch); otherwise the default priority
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, bool evict_first) {
    if (!evict_first) {
        bulk_g2s(dst, src, bytes, bar);
        return;
    }
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Entries whose x loads are issued together before their FMAs.
template <int M> struct Batch {
    static constexpr int B = M == 1 ? 8 : (M == 2 ? 4 : (M == 4 ? 2 : 1));
};

// Fused multiply-add of the accumulator type: binary64, or binary32 (one rounding each).
__device__ __forceinline__ double afma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float afma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// acc[i] = sum_j val[j] * x[col[j]*M + i] over a row's entries, in stored order, in the
// accumulator type AT (binary64, or binary32 with x the binary32 shadow of the input).  Entry
// j of the row is at val[off + 32 j] / col[off + 32 j] (global or shared memory), j < width
// of the row's slice; entries past the row's end are padding with col < 0 and are skipped.
template <int M, int B, class AT, class VP, class CP>
__device__ __forceinline__ void row_sum(VP val, CP col, int64_t off, int width, const AT *x, AT (&acc)[M]) {
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = AT(0);
    for (int j0 = 0; j0 < width; j0 += B) {
        AT v[B];
        int32_t c[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (j0 + b < width) {
                v[b] = val[off + 32 * (int64_t)(j0 + b)];
                c[b] = col[off + 32 * (int64_t)(j0 + b)];
            } else {
                v[b] = AT(0);
                c[b] = -1;
            }
        }
        AT xv[B][M];
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int i = 0; i < M; ++i) xv[b][i] = (c[b] >= 0) ? x[(int64_t)c[b] * M + i] : AT(0);
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (c[b] >= 0) {
#pragma unroll
                for (int i = 0; i < M; ++i) acc[i] = afma(v[b], xv[b][i], acc[i]);
            }
    }
}

// Continues a row sum from entry j0 (acc already holds entries 0..j0-1).
template <int M, int B, class AT, class VP, class CP>
__device__ __forceinline__ void row_sum_from(VP val, CP col, int64_t off, int j_start, int width, const AT *x,
                                             AT (&acc)[M]) {
    for (int j0 = j_start; j0 < width; j0 += B) {
        AT v[B];
        int32_t c[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (j0 + b < width) {
                v[b] = val[off + 32 * (int64_t)(j0 + b)];
                c[b] = col[off + 32 * (int64_t)(j0 + b)];
            } else {
                v[b] = AT(0);
                c[b] = -1;
            }
        }
        AT xv[B][M];
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int i = 0; i < M; ++i) xv[b][i] = (c[b] >= 0) ? x[(int64_t)c[b] * M + i] : AT(0);
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (c[b] >= 0) {
#pragma unroll
                for (int i = 0; i < M; ++i) acc[i] = afma(v[b], xv[b][i], acc[i]);
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
    static __device__ __forceinline__ float widen32(double v) { return (float)v; }  // never instantiated
};
struct ValF32 {
    using T = float;
    static __device__ __forceinline__ double widen(float v) { return widen_normal32(__float_as_uint(v)); }
    static __device__ __forceinline__ float widen32(float v) { return v; }
};
struct ValBF16 {
    using T = uint16_t;  // bfloat16 bits
    static __device__ __forceinline__ double widen(uint16_t v) { return widen_normal32((uint32_t)v << 16); }
    // a bfloat16 is the upper half of a binary32
    static __device__ __forceinline__ float widen32(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }
};
// the stored value in the accumulator type (exact: both types hold every stored value)
template <class VT, class AT> struct ToAcc;
template <class VT> struct ToAcc<VT, double> {
    static __device__ __forceinline__ double get(typename VT::T v) { return VT::widen(v); }
};
template <class VT> struct ToAcc<VT, float> {
    static __device__ __forceinline__ float get(typename VT::T v) { return VT::widen32(v); }
};

// read-only views returning values in the accumulator type: the immutable matrix copy in
// global memory, or a staged slot in shared memory
template <class VT, class AT = double> struct GVal {
    const typename VT::T *p;
    __device__ __forceinline__ AT operator[](int64_t i) const { return ToAcc<VT, AT>::get(__ldg(p + i)); }
};
template <class VT, class AT = double> struct SVal {
    const typename VT::T *p;
    __device__ __forceinline__ AT operator[](int64_t i) const { return ToAcc<VT, AT>::get(p[i]); }
};
struct GCol {
    const int32_t *p;
    __device__ __forceinline__ int32_t operator[](int64_t i) const { return __ldg(p + i); }
};

__device__ __forceinline__ int hi_bits(double v) { return __double2hiint(v); }
__device__ __forceinline__ int hi_bits(float v) { return __float_as_int(v); }

// A row sum in binary64: binary64 sums as they are, binary32 sums widened exactly (integer
// operations on the encoding, every binary32 value including subnormals, infinities, NaNs).
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return widen_binary32(__float_as_uint(v)); }

// The input block the row sums of local power k read: binary64 powers, or, with binary32
// accumulation, the binary32 shadow ring (slot j & 1 holds the binary32 rounding of step j).
// block of the ring that holds power / step j; j < ring always for powers, so the division
// runs only for the Chebyshev recurrence (j is the same in the whole warp)
__device__ __forceinline__ int ring_slot(const KArgs &a, int j) { return j < a.ring ? j : j % a.ring; }
template <int M>
__device__ __forceinline__ const double *input_block(const KArgs &a, int k) {
    return (k == 1 && a.k_offset == 0) ? a.x0 : a.ybase + (int64_t)ring_slot(a, a.k_offset + k - 1) * a.ystride;
}
template <int M, class AT> struct InputAcc {
    static __device__ __forceinline__ const double *get(const KArgs &a, int k) { return input_block<M>(a, k); }
};
template <int M> struct InputAcc<M, float> {
    static __device__ __forceinline__ const float *get(const KArgs &a, int k) {
        return a.shadow + (int64_t)((a.k_offset + k - 1) & 1) * a.ystride;
    }
};

// Rows of global memory a row's epilogue reads, loaded before its FMAs so that their latency
// overlaps the row sum: the row's own input (Chebyshev) and the row two steps back (Chebyshev
// from step 2 on), or the row of x0 copied to Y[0] (powers, power 1).
template <int M> struct EpiRows {
    double own[M], back[M];
};
template <int M, int MODE>
__device__ __forceinline__ void epilogue_load(const KArgs &a, int k, int64_t r, const double *xin, EpiRows<M> &e) {
    const int j = a.k_offset + k;
    if constexpr (MODE == MODE_CHEB) {
#pragma unroll
        for (int i = 0; i < M; ++i) e.own[i] = xin[r * M + i];
        if (j != 1) {
            const double *vp2 = a.ybase + (int64_t)ring_slot(a, j - 2) * a.ystride + r * M;
#pragma unroll
            for (int i = 0; i < M; ++i) e.back[i] = vp2[i];
        }
    } else {
        if (k == 1 && a.y0copy) {
#pragma unroll
            for (int i = 0; i < M; ++i) e.own[i] = a.x0[r * M + i];
        }
    }
}
// Epilogue of one row at local power k with its rows loaded: store into the plan-order slot
// (and Y[0] for power 1), or advance the Chebyshev recurrence (binary64 in both accumulator
// types).  With binary32 accumulation the step's binary32 shadow is stored too: the row sum
// itself for powers, the binary32 rounding of the new recurrence value for Chebyshev.
template <int M, int MODE, class AT>
__device__ __forceinline__ void row_epilogue_loaded(const KArgs &a, int k, int64_t r, const AT (&wa)[M],
                                                    const EpiRows<M> &e) {
    constexpr bool A32 = sizeof(AT) == 4;
    const int j = a.k_offset + k;  // absolute power / recurrence step
    double w[M];
#pragma unroll
    for (int i = 0; i < M; ++i) w[i] = to_f64(wa[i]);
    double *y = a.ybase + (int64_t)ring_slot(a, j) * a.ystride + r * M;
    float *sh = A32 ? a.shadow + (int64_t)(j & 1) * a.ystride + r * M : nullptr;
    if constexpr (MODE == MODE_CHEB) {
        double vn[M];
        if (j == 1) {
#pragma unroll
            for (int i = 0; i < M; ++i) vn[i] = fma(a.halpha, w[i], a.hbeta * e.own[i]);
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) vn[i] = fma(a.alpha, w[i], fma(a.beta, e.own[i], -e.back[i]));
        }
#pragma unroll
        for (int i = 0; i < M; ++i) y[i] = vn[i];
        if constexpr (A32) {
#pragma unroll
            for (int i = 0; i < M; ++i) sh[i] = __double2float_rn(vn[i]);
        }
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
        if (!A32 && k == a.p_launch) {
            // the launch's last power is not read again here: streaming stores, so that it does
            // not push out of L2 the groups still in their reuse window (measured at 256^3,
            // p = 8: 0.8 % faster with binary64 sums, 3 % slower with binary32 sums)
#pragma unroll
            for (int i = 0; i < M; ++i) __stcs(y + i, w[i]);
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) y[i] = w[i];
        }
        if constexpr (A32) {
#pragma unroll
            for (int i = 0; i < M; ++i) sh[i] = (float)wa[i];
        }
        if constexpr (MODE == MODE_HOST) {  // the power's rows in host memory too (never read here)
            double *yh = a.yhost + (int64_t)j * a.ystride + r * M;
#pragma unroll
            for (int i = 0; i < M; ++i) __stcs(yh + i, w[i]);
        }
        if (k == 1 && a.y0copy) {
#pragma unroll
            for (int i = 0; i < M; ++i) a.y0copy[r * M + i] = e.own[i];
        }
    }
}

// Epilogue of one row at local power k: loads its rows, then as row_epilogue_loaded (the
// y0copy of power 1 included).
template <int M, int MODE, class AT>
__device__ __forceinline__ void row_epilogue(const KArgs &a, int k, int64_t r, const AT (&w)[M], const double *xin) {
    EpiRows<M> e;
    epilogue_load<M, MODE>(a, k, r, xin, e);
    row_epilogue_loaded<M, MODE, AT>(a, k, r, w, e);
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
    int widths[8];    // staged chunks: width of slice q in byte q of the 32 bytes (16 for shape 3)
    long long ebase;  // first entry of the chunk in the sliced copy
};

__device__ __forceinline__ bool timed_out(uint64_t t0, int64_t limit) { return globaltimer() - t0 > (uint64_t)limit; }

// NW: the width words a shape uses (8 for two slices a warp, else 4: at most 16 slices)
template <int NW = 4>
__device__ __forceinline__ int slice_width(const int (&w)[8], int q) {
    int word = w[0];
#pragma unroll
    for (int t = 1; t < NW; ++t) word = (q >> 2) == t ? w[t] : word;  // no dynamic indexing
    return (word >> (8 * (q & 3))) & 0xff;
}
// padded entries of the chunk's slices 0 .. q-1 (q <= kRecSlicesWide): the byte widths of the
// whole words before slice q, and the low bytes of its own word, each word summed by one
// four-way byte dot product
template <int NW = 4>
__device__ __forceinline__ int slice_prefix(const int (&w)[8], int q) {
    const int wq = q >> 2;
    const unsigned int part = (1u << (8 * (q & 3))) - 1u;  // bytes of slices before q in word wq
    unsigned int pre = 0;
#pragma unroll
    for (int t = 0; t < NW; ++t) {
        const unsigned int m = t < wq ? 0xffffffffu : (t == wq ? part : 0u);
        pre = __dp4a((unsigned int)w[t] & m, 0x01010101u, pre);
    }
    return (int)pre;
}

// A compute warp handles a unit in two phases.  Phase A reads the column indices of the
// warp's first row batch from shared memory and issues the x gathers; phase B runs the
// FMAs on those x values, finishes any further batches or slices, stores the results and
// publishes the unit.  Phase B directly follows phase A of the same unit: a warp holds no
// unit across a wait, so its lanes, which wait on the slot's mbarrier one by one, always
// work on the same unit.
// Padding entries of the first batch (column -1) are skipped.  Binary32 row sums keep the
// "stored" bits that phase A derived from the columns it read; binary64 sums read the column
// again (measured faster there: the bit mask costs the binary64 loop a register it lacks).
template <class AT> constexpr bool kPadMask = std::is_same<AT, float>::value;
template <int M, class AT = double> struct Prefetch {
    static constexpr int B = Batch<M>::B;
    int unit;             // -1: nothing pending
    int slot;
    int r;                // this lane's row in the warp's first slice, -1 if none
    int off;              // offset of that row's entries in the slot (staged units)
    int width;            // width of the warp's first slice (staged units)
    unsigned int valid;   // binary32 sums: bit q set when entry q of the first batch is stored
    AT x[B][M];           // x values of the first batch (entries j < min(B, width))
};

// phase A: request the x values of the warp's first batch of unit u (slot b)
template <int M, bool STAGING, class AT, int NW = 4>
__device__ __forceinline__ void phase_a(const KArgs &a, const UnitInfo &u, int b, const int32_t *scol, int cwarp,
                                        int lane, Prefetch<M, AT> &pf) {
    constexpr int B = Batch<M>::B;
    pf.unit = u.unit;
    pf.slot = b;
    const AT *xin = InputAcc<M, AT>::get(a, u.unit & 31);
    pf.r = -1;
    pf.width = 0;
    pf.off = 0;
    pf.valid = 0;
    if (STAGING && u.staged && cwarp < u.nsl) {  // shapes without slots never stage
        const int pre = slice_prefix<NW>(u.widths, cwarp);
        pf.width = slice_width<NW>(u.widths, cwarp);
        pf.off = 32 * pre + lane;
        const int r = u.row0 + 32 * cwarp + lane;
        if (r < u.row1) pf.r = r;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int c = (pf.r >= 0 && q < pf.width) ? scol[pf.off + 32 * q] : -1;
        if constexpr (kPadMask<AT>) pf.valid |= (c >= 0 ? 1u : 0u) << q;
#pragma unroll
        for (int i = 0; i < M; ++i) pf.x[q][i] = (c >= 0) ? xin[(int64_t)c * M + i] : AT(0);
    }
}

// Completion of a unit by the compute warps.  Each warp releases the unit's slot (empty[b])
// as soon as it has read everything it needs from the slot into registers, so that the
// control warp can refill the slot while the warp still runs its FMA chain and stores.
// Publication is the publisher warp's job: a compute warp that finished the unit orders its
// stores at block scope and adds one to the unit's finish counter; the publisher warp sees
// the counters of up to 32 consecutive units reach the number of compute warps, issues one
// fence at GPU scope for all of them (it acquires the compute warps' stores through the
// counters and releases them to other blocks) and stores their flags.  No compute warp ever
// waits for a fence at GPU scope.  The counters are indexed by the unit's sequence number in
// the block modulo kDoneRing and only grow (use n of a counter completes at n times the
// number of compute warps), so a lagging publisher never sees a counter that was reset.
constexpr int kDoneRing = 64;
// shapes 0-2 release the slot before their FMA chain too (1), or after their unit (0): the
// early path holds a batch of entries in registers, more than shape 0's 40 a thread allow
#ifndef MPK_EARLY_RELEASE_B
#define MPK_EARLY_RELEASE_B 0
#endif
constexpr bool kEarlyReleaseB = MPK_EARLY_RELEASE_B != 0;
template <int CW>
__device__ __forceinline__ void release_slot(uint64_t *s_empty, int b, int lane) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&s_empty[b]);
}
template <int CW>
__device__ __forceinline__ void publish_unit(const KArgs &a, int32_t epoch, int unit, int seq, int *s_done, int lane) {
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();  // this warp's stores before the count (block scope)
        atomicAdd(&s_done[seq % kDoneRing], 1);
    }
}
// The control warp may record sequence number i in the ring only once the publisher is past
// i - kDoneRing (normally at once; bounded: false if the publisher made no progress in time).
__device__ __forceinline__ bool useq_slot_free(volatile int *s_published, int i, int64_t limit) {
    if (i - *s_published < kDoneRing) return true;
    const uint64_t t0 = globaltimer();
    while (i - *s_published >= kDoneRing)
        if (timed_out(t0, limit)) return false;
    __threadfence_block();
    return true;
}
__device__ __forceinline__ int ld_relaxed_cta_shared(const int *p) {
    int v;
    asm volatile("ld.relaxed.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
// The publisher warp: publishes the block's units in sequence order, up to 32 at a time, until
// every unit handed over (s_final, once set) is published.  Bounded like the compute warps.
template <int CW>
__device__ __forceinline__ void publisher_loop(const KArgs &a, int32_t epoch, const int *s_done, const int *s_useq,
                                               volatile int *s_final, volatile int *s_published, int lane) {
    int j = 0;
    uint64_t t_idle = globaltimer();
    for (;;) {
        const int fin = *s_final;
        const int jl = j + lane;
        bool done = false;
        if (fin < 0 || jl < fin) done = ld_relaxed_cta_shared(&s_done[jl % kDoneRing]) >= CW * (jl / kDoneRing + 1);
        const unsigned int m = __ballot_sync(0xffffffffu, done);
        const int cnt = (m == 0xffffffffu) ? 32 : __ffs(~m) - 1;  // finished units from j on, in a row
        if (cnt > 0) {
            fence_acq_rel_gpu();  // acquires the counted stores, releases them before the flags
            if (lane < cnt) {
                const int un = s_useq[jl % kDoneRing];
                if (un != a.drop_unit) st_relaxed(a.flags + (int64_t)(un & 31) * a.nchunks + (un >> 5), epoch);
            }
            j += cnt;
            __threadfence_block();  // the reads of s_useq before the progress that lets it be reused
            if (lane == 0) *s_published = j;
            t_idle = globaltimer();
            continue;
        }
        if (fin >= 0 && j >= fin) break;  // every unit handed over is published
        if (timed_out(t_idle, 2 * a.wait_ns + 100000000LL)) break;  // the compute warps gave up
        __nanosleep(32);
    }
}

// phase B: finish unit pf (all of the warp's rows), release its slot and publish it
template <int M, int MODE, class VT, int SH, class AT>
__device__ __forceinline__ void phase_b(const KArgs &a, int32_t epoch, const Prefetch<M, AT> &pf, const UnitInfo *s_u,
                                        const typename VT::T *sval0, const int32_t *scol0, int *s_done, uint64_t *s_empty,
                                        int cwarp, int lane, int seq) {
    constexpr int B = Batch<M>::B;
    const UnitInfo u = s_u[pf.slot];  // a copy: the slot is refilled once released
    const int k = pf.unit & 31;
    const double *xin = input_block<M>(a, k);
    const AT *xacc = InputAcc<M, AT>::get(a, k);
    constexpr int kCompWarps = Shape<SH>::CW;
    const SVal<VT, AT> sval{sval0 + pf.slot * Shape<SH>::SE};
    const int32_t *scol = kStageCol ? scol0 + pf.slot * Shape<SH>::SE : a.col + u.ebase;
    bool released = false;
    if (kEarlyReleaseB && Shape<SH>::SE > 0 && u.staged && u.nsl <= kCompWarps && pf.width <= B) {
        // the warp's one slice fits one batch: read its entries, release the slot, then compute
        AT v[B];
        bool on[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
            on[q] = kPadMask<AT> ? ((pf.valid >> q) & 1u) != 0 : (pf.r >= 0 && q < pf.width && scol[pf.off + 32 * q] >= 0);
            v[q] = on[q] ? sval[pf.off + 32 * q] : AT(0);
        }
        EpiRows<M> er;
        if (pf.r >= 0) epilogue_load<M, MODE>(a, k, pf.r, xin, er);
        release_slot<kCompWarps>(s_empty, pf.slot, lane);
        released = true;
        if (pf.r >= 0) {
            AT w[M];
#pragma unroll
            for (int i = 0; i < M; ++i) w[i] = AT(0);
#pragma unroll
            for (int q = 0; q < B; ++q)
                if (on[q]) {
#pragma unroll
                    for (int i = 0; i < M; ++i) w[i] = afma(v[q], pf.x[q][i], w[i]);
                }
            row_epilogue_loaded<M, MODE, AT>(a, k, pf.r, w, er);
        }
    } else if (Shape<SH>::SE > 0 && u.staged) {
        if (pf.r >= 0) {  // first slice: prefetched first batch, then the rest of the row
            AT w[M];
#pragma unroll
            for (int i = 0; i < M; ++i) w[i] = AT(0);
#pragma unroll
            for (int q = 0; q < B; ++q) {
                if (kPadMask<AT> ? ((pf.valid >> q) & 1u) != 0 : (q < pf.width && scol[pf.off + 32 * q] >= 0)) {
                    const AT v = sval[pf.off + 32 * q];
#pragma unroll
                    for (int i = 0; i < M; ++i) w[i] = afma(v, pf.x[q][i], w[i]);
                }
            }
            if (pf.width > B) row_sum_from<M, 2, AT>(sval, scol, pf.off, B, pf.width, xacc, w);  // rare: wide rows
            row_epilogue<M, MODE, AT>(a, k, pf.r, w, xin);
        }
        for (int sl = cwarp + kCompWarps; sl < u.nsl; sl += kCompWarps) {  // further slices (wide chunks)
            const int64_t r = (int64_t)u.row0 + 32 * sl + lane;
            const int pre = slice_prefix<Shape<SH>::NW>(u.widths, sl);
            if (r >= u.row1) continue;
            AT w[M];
            // a second slice of the warp (shapes of two slices a warp: all gathers of a batch at
            // once) or, on the other shapes, the rare chunk wider than the block
            constexpr int BS2 = Shape<SH>::SPW > 1 ? B : 2;
            row_sum<M, BS2, AT>(sval, scol, 32 * pre + lane, slice_width<Shape<SH>::NW>(u.widths, sl), xacc, w);
            row_epilogue<M, MODE, AT>(a, k, r, w, xin);
        }
    } else {  // entries in global memory (chunk too large to stage): the slot holds nothing
        release_slot<kCompWarps>(s_empty, pf.slot, lane);
        released = true;
        for (int sl = cwarp; sl < u.nsl; sl += kCompWarps) {
            const int64_t r = (int64_t)u.row0 + 32 * sl + lane;
            if (r >= u.row1) continue;
            const int64_t s0 = __ldg(a.slice_ptr + u.slice0 + sl), s1 = __ldg(a.slice_ptr + u.slice0 + sl + 1);
            AT w[M];
            // entries whose x loads are issued together: the unstaged shape issues a row's
            // loads in batches; the staged shapes keep this rare path small (registers)
            constexpr int BU = Shape<SH>::SE == 0 ? Batch<M>::B : 1;
            row_sum<M, BU, AT>(GVal<VT, AT>{static_cast<const typename VT::T *>(a.val) + u.ebase},
                               GCol{a.col + u.ebase}, s0 - u.ebase + lane, (int)((s1 - s0) >> 5), xacc, w);
            row_epilogue<M, MODE, AT>(a, k, r, w, xin);
        }
    }
    if (!released) release_slot<kCompWarps>(s_empty, pf.slot, lane);
    publish_unit<kCompWarps>(a, epoch, pf.unit, seq, s_done, lane);
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
        got[q] = idx >= 0 ? (kAcquirePoll ? ld_acquire(f + idx) : ld_relaxed(f + idx)) : epoch;
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

// Two units' dependency flags on one round trip: lanes 0..15 poll unit A's, lanes 16..31 unit
// B's (64 flags a half per round; units of power 1 poll nothing).  Returns A's readiness in
// bit 0 and B's in bit 1 (warp-uniform).  Every flag is loaded with acquire semantics by the
// lane that checks it, as in deps_ready.
__device__ __forceinline__ int deps_ready_pair(const KArgs &a, int32_t epoch, int kA, const int (&loA)[kDepRanges],
                                               const int (&lenA)[kDepRanges], int totA, int kB,
                                               const int (&loB)[kDepRanges], const int (&lenB)[kDepRanges],
                                               int totB, int lane) {
    const bool hiB = lane >= 16;
    const int sl = lane & 15;
    const int k = hiB ? kB : kA;
    const int tot = (k > 1) ? (hiB ? totB : totA) : 0;
    const int tmax = max((kA > 1) ? totA : 0, (kB > 1) ? totB : 0);
    const int32_t *f = a.flags + (int64_t)(k - 1) * a.nchunks;
    bool ok = true;
    for (int v0 = 0; v0 < tmax; v0 += 64) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int v = v0 + 16 * q + sl, idx = -1;
            if (v < tot) {
#pragma unroll
                for (int r = 0; r < kDepRanges; ++r) {
                    const int lo = hiB ? loB[r] : loA[r], len = hiB ? lenB[r] : lenA[r];
                    if (idx < 0 && v < len) idx = lo + v;
                    if (idx < 0) v -= len;
                }
            }
            const int got = idx >= 0 ? ld_acquire(f + idx) : epoch;
            ok = ok && got == epoch;
        }
    }
    const unsigned int m = __ballot_sync(0xffffffffu, ok);
    return ((m & 0xffffu) == 0xffffu ? 1 : 0) | ((m >> 16) == 0xffffu ? 2 : 0);
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


// ----------------------------------------------------------------------------- shape 3
// Input-row windows.  A shape-3 chunk reads its columns from at most kXWin windows of input
// rows; window q holds rows [lo, lo + len) and sits in the slot's window area from row
// position pos on: element (row c, column i) is double number shift + M * (pos + c - lo) + i
// of the area, shift = (address of the input vector / 8) mod 2.  The control warp copies
// each window with one bulk copy, whose global start is rounded down and end rounded up to
// 16 bytes; the planner keeps pos = lo (mod 2) for M = 1 and leaves room around each window,
// so that the rounded copy lands 16-byte aligned, inside the area and clear of the other
// windows.  Only at the very end of the input vector is the end not rounded up: the last 8
// bytes are then copied by a plain load (no read past the vector).
struct XCopy {
    uint64_t src;    // global start, 16-byte aligned
    uint32_t dst;    // shared-memory address, 16-byte aligned
    uint32_t bytes;  // bulk bytes (multiple of 16, may be 0)
    uint64_t tail;   // global address of an 8-byte word copied by a plain load (0: none)
    uint32_t tdst;   // its shared-memory address
};
template <int M>
__device__ __forceinline__ XCopy x_copy(const double *xin, int64_t n, int lo, int len, int pos, uint32_t area) {
    XCopy c{0, 0, 0, 0, 0};
    if (len <= 0) return c;
    const uint64_t shift = ((uint64_t)xin >> 3) & 1u;
    const uint64_t g0 = (uint64_t)(xin + (int64_t)lo * M), g1 = (uint64_t)(xin + (int64_t)(lo + len) * M);
    const uint64_t vend = (uint64_t)(xin + n * M);
    const uint64_t a0 = g0 & ~(uint64_t)15;
    uint64_t a1 = (g1 + 15) & ~(uint64_t)15;
    if (a1 > vend) {  // only when the window ends the vector at an 8 (mod 16) address
        a1 = vend & ~(uint64_t)15;
        c.tail = a1;
    }
    c.src = a0;
    c.dst = area + (uint32_t)(8 * (shift + (uint64_t)M * pos)) - (uint32_t)(g0 - a0);
    c.bytes = (uint32_t)(a1 - a0);
    c.tdst = c.dst + c.bytes;
    return c;
}

// Compute warps of shape 3: every row of the warp's slices, with entries, column positions
// and input rows read from the slot; the slot is released once read, then the unit published.
template <int M, int MODE, class VT, int SH>
__device__ __forceinline__ void phase_x(const KArgs &a, int32_t epoch, const UnitInfo *s_u, int b,
                                        const typename VT::T *sval0, const uint16_t *slc0, const double *sx0,
                                        int *s_done, uint64_t *s_empty, int cwarp, int lane, int seq) {
    constexpr int CW = Shape<SH>::CW, SE = Shape<SH>::SE;
    constexpr int B = Batch<M>::B;
    const UnitInfo u = s_u[b];  // a copy: the slot is refilled once released
    const int k = u.unit & 31;
    const double *xin = input_block<M>(a, k);
    const SVal<VT> sval{sval0 + b * SE};
    const uint16_t *slc = slc0 + b * SE;
    const double *sx = sx0 + b * Shape<SH>::XW + (((uint64_t)xin >> 3) & 1u);
    if (u.nsl <= CW && (cwarp >= u.nsl || slice_width(u.widths, cwarp) <= B)) {
        // at most one slice of at most one batch: read it, release the slot, then compute
        const int pre = slice_prefix(u.widths, cwarp);
        const int width = cwarp < u.nsl ? slice_width(u.widths, cwarp) : 0;
        const int64_t r = (int64_t)u.row0 + 32 * cwarp + lane;
        const bool row = cwarp < u.nsl && r < u.row1;
        const int off = 32 * pre + lane;
        bool on[B];
        double v[B], xv[B][M];
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const int lc = (row && q < width) ? (int)slc[off + 32 * q] : 0xffff;
            on[q] = lc != 0xffff;
            v[q] = on[q] ? sval[off + 32 * q] : 0.0;
#pragma unroll
            for (int i = 0; i < M; ++i) xv[q][i] = on[q] ? sx[M * lc + i] : 0.0;
        }
        EpiRows<M> er;
        if (row) epilogue_load<M, MODE>(a, k, r, xin, er);
        release_slot<CW>(s_empty, b, lane);
        if (row) {
            double w[M];
#pragma unroll
            for (int i = 0; i < M; ++i) w[i] = 0.0;
#pragma unroll
            for (int q = 0; q < B; ++q)
                if (on[q]) {
#pragma unroll
                    for (int i = 0; i < M; ++i) w[i] = fma(v[q], xv[q][i], w[i]);
                }
            row_epilogue_loaded<M, MODE, double>(a, k, r, w, er);
        }
        publish_unit<CW>(a, epoch, u.unit, seq, s_done, lane);
        return;
    }
    for (int sl = cwarp; sl < u.nsl; sl += CW) {
        const int pre = slice_prefix(u.widths, sl);
        const int width = slice_width(u.widths, sl);
        const int64_t r = (int64_t)u.row0 + 32 * sl + lane;
        if (r >= u.row1) continue;
        const int off = 32 * pre + lane;
        EpiRows<M> er;
        epilogue_load<M, MODE>(a, k, r, xin, er);
        double w[M];
#pragma unroll
        for (int i = 0; i < M; ++i) w[i] = 0.0;
        for (int j0 = 0; j0 < width; j0 += B) {
            int lc[B];
            double v[B];
#pragma unroll
            for (int q = 0; q < B; ++q) {
                lc[q] = (j0 + q < width) ? (int)slc[off + 32 * (j0 + q)] : 0xffff;
                v[q] = (lc[q] != 0xffff) ? sval[off + 32 * (j0 + q)] : 0.0;
            }
            double xv[B][M];
#pragma unroll
            for (int q = 0; q < B; ++q)
#pragma unroll
                for (int i = 0; i < M; ++i) xv[q][i] = (lc[q] != 0xffff) ? sx[M * lc[q] + i] : 0.0;
#pragma unroll
            for (int q = 0; q < B; ++q)
                if (lc[q] != 0xffff) {
#pragma unroll
                    for (int i = 0; i < M; ++i) w[i] = fma(v[q], xv[q][i], w[i]);
                }
        }
        row_epilogue_loaded<M, MODE, double>(a, k, r, w, er);
    }
    release_slot<CW>(s_empty, b, lane);
    publish_unit<CW>(a, epoch, u.unit, seq, s_done, lane);
}

template <int M, int MODE, bool TRACE, class VT, int SH, bool A32 = false>
__global__ void __launch_bounds__(Shape<SH>::BS, (MpkOcc<M, MODE, TRACE, SH>::blocks)) k_mpk(const KArgs a) {
    using AT = typename std::conditional<A32, float, double>::type;  // accumulator of the row sums
    static_assert(!(A32 && Shape<SH>::X), "shape 3 stages binary64 input rows only");
    constexpr int kCompWarps = Shape<SH>::CW, kStageEntries = Shape<SH>::SE;
    constexpr int kSlots = Shape<SH>::SL;
    constexpr bool XS = Shape<SH>::X;
    constexpr int kCtl = Shape<SH>::CTL;
    constexpr int kPub = kCtl;  // warp index of the publisher warp (after the control warps)
    constexpr int kRing = 4;  // split control: ready units between the poll and the stage warp
    static_assert(kSlots >= 2 && kSlots <= kMaxSlots, "slots");
    using T = typename VT::T;
    const bool tr = TRACE && a.trace != nullptr;  // timing counters (instantiated separately)
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_full[kSlots];
    __shared__ __align__(8) uint64_t s_empty[kSlots];
    __shared__ UnitInfo s_u[kSlots];
    __shared__ volatile int s_final;  // units handed over in total; -1 while the control warp runs
    __shared__ int s_done[kDoneRing];  // compute warps finished with a unit (by its sequence number)
    __shared__ int s_useq[kDoneRing];  // unit id of each sequence number (for the publisher warp)
    __shared__ volatile int s_published;  // units published so far (the publisher's progress)
    // split control (two control warps): ring of ready units, its mbarriers, stop flag
    __shared__ __align__(8) uint64_t s_rfull[kCtl == 2 ? kRing : 1];
    __shared__ __align__(8) uint64_t s_rfree[kCtl == 2 ? kRing : 1];
    __shared__ int s_ring_unit[kCtl == 2 ? kRing : 1];
    __shared__ int s_ring_rec[kCtl == 2 ? kRing : 1][kRecInts];
    __shared__ volatile int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T *const sval0 = reinterpret_cast<T *>(smem);
    int32_t *const scol0 = reinterpret_cast<int32_t *>(smem + kSlots * kStageEntries * sizeof(T));
    // shape 3: 16-bit column positions after the values, then the input-row window areas
    uint16_t *const slc0 = reinterpret_cast<uint16_t *>(smem + kSlots * kStageEntries * sizeof(T));
    double *const sx0 = reinterpret_cast<double *>(smem + kSlots * kStageEntries * (sizeof(T) + 2));

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
        s_published = 0;
        s_stop = 0;
        for (int q = 0; q < kDoneRing; ++q) s_done[q] = 0;
        for (int q = 0; q < kSlots; ++q) {
            mbar_init(&s_full[q], 1);
            mbar_init(&s_empty[q], kCompWarps);
        }
        if constexpr (kCtl == 2)
            for (int q = 0; q < kRing; ++q) {
                mbar_init(&s_rfull[q], 1);
                mbar_init(&s_rfree[q], 1);
            }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int32_t epoch = s_epoch;

    if (warp == kPub) {
        publisher_loop<kCompWarps>(a, epoch, s_done, s_useq, &s_final, &s_published, lane);
    } else if (warp < kCtl) {
      if constexpr (kCtl == 2) {
        // ---------------------------------------------------------- split control (shape 3)
        // Warp 0 claims units in ticket order, polls their dependencies and pushes each ready
        // unit (its id and chunk record) into a ring of kRing entries; warp 1 takes them in
        // the same order, waits for a free slot, copies the entries and input rows and hands
        // the slot over.  Each warp has one round trip per unit on its path, and the two run
        // side by side.  The poll's acquire reaches the stage warp through the ring's
        // mbarrier (release / acquire at CTA scope) and the compute warps through full[b].
        // An end marker (unit -1) closes the ring; a stage warp that gives up sets s_stop.
        const int32_t *rec = reinterpret_cast<const int32_t *>(a.chunk_rec);
        auto record_timeout = [&]() {
            if (lane == 0 && atomicExch(a.err, epoch) != epoch) st_relaxed(a.err + 1, (int)MPK_ERR_TIMEOUT);
        };
        if (warp == 0) {
            // ------------------------------------------------------ poll warp
            auto unit_at = [&](unsigned int t) -> int { return (int64_t)t < a.nunits ? __ldg(a.units + t) : -1; };
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
            // waits for ring entry q to be free again (consumed kRing pushes ago)
            auto ring_free = [&](int i) -> bool {
                if (i < kRing) return true;
                const int q = i % kRing;
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(&s_rfree[q], ((i / kRing) - 1) & 1)) {
                    if (s_stop) return false;
                    if (timed_out(t0, a.wait_ns)) {
                        record_timeout();
                        return false;
                    }
                }
                return true;
            };
            for (int i = 0;; ++i) {
                const int q = i % kRing;
                bool aborted = false;
                if (u_cur >= 0) {
                    const int k = u_cur & 31;
                    int dlo[kDepRanges], dlen[kDepRanges];
                    const int total = dep_ranges_of(r_cur, dlo, dlen);
                    if (k > 1) {
                        const uint64_t t0 = globaltimer();
                        while (!deps_ready(a, epoch, k, dlo, dlen, total, lane)) {
                            if (lane == 0) tr_add(2, 1);
                            const bool stop = ld_relaxed(a.err) == epoch || timed_out(t0, a.wait_ns) || s_stop;
                            if (__any_sync(0xffffffffu, stop)) {
                                aborted = true;
                                break;
                            }
                            __nanosleep(32);
                        }
                        if (tr && lane == 0) tr_add(1, globaltimer() - t0);
                    }
                    if (lane == 0) tr_add(0, 1);
                }
                if (aborted) record_timeout();
                const bool last = u_cur < 0 || aborted;
                if (!ring_free(i)) break;  // the stage warp stopped, or a wait expired
                if (lane < kRecInts) s_ring_rec[q][lane] = last ? 0 : r_cur;
                if (lane == 0) s_ring_unit[q] = last ? -1 : u_cur;
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_rfull[q]);
                if (last) break;
                u_cur = u_nxt;  // move up, then load into the tail (as the single control warp)
                r_cur = r_nxt;
                u_nxt = __shfl_sync(0xffffffffu, u_nn, 0);
                r_nxt = rec_at(u_nxt);
                if (lane == 0) {
                    u_nn = unit_at(t);
                    t = atomicAdd(a.ticket, 1u);
                }
            }
        } else {
            // ------------------------------------------------------ stage warp
            bool slot_busy[kSlots] = {};
            int slot_use[kSlots] = {};
            int i = 0;
            for (;; ++i) {
                const int q = i % kRing, b = i % kSlots;
                {
                    const uint64_t t0 = globaltimer();
                    bool ok;
                    while (!(ok = mbar_try_wait(&s_rfull[q], (i / kRing) & 1)))
                        if (timed_out(t0, 2 * a.wait_ns + 100000000LL)) break;
                    if (tr && lane == 0) tr_add(12, globaltimer() - t0);
                    if (!ok) {  // the poll warp gave no sign of life
                        record_timeout();
                        break;
                    }
                }
                const int un = s_ring_unit[q];
                const int r_cur = lane < kRecInts ? s_ring_rec[q][lane] : 0;
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_rfree[q]);
                if (un < 0) break;  // end of the units
                UnitInfo u;
                u.unit = un;
                u.row0 = __shfl_sync(0xffffffffu, r_cur, 0);
                u.row1 = __shfl_sync(0xffffffffu, r_cur, 1);
                u.slice0 = __shfl_sync(0xffffffffu, r_cur, 2);
                u.ecount = __shfl_sync(0xffffffffu, r_cur, 3);
                u.ebase = (long long)(unsigned int)__shfl_sync(0xffffffffu, r_cur, 4) |
                          ((long long)__shfl_sync(0xffffffffu, r_cur, 5) << 32);
                u.staged = __shfl_sync(0xffffffffu, r_cur, 6);
                u.nsl = __shfl_sync(0xffffffffu, r_cur, 7);
#pragma unroll
                for (int w = 0; w < Shape<SH>::NW; ++w) u.widths[w] = __shfl_sync(0xffffffffu, r_cur, 16 + w);
                const int k = un & 31;
                XCopy xc{0, 0, 0, 0, 0};
                uint32_t xbytes = 0;
                if constexpr (XS) {
                    const int wsrc = kRecWin + 3 * (lane & (kXWin - 1));
                    const int wlo = __shfl_sync(0xffffffffu, r_cur, wsrc);
                    const int wlen = __shfl_sync(0xffffffffu, r_cur, wsrc + 1);
                    const int wpos = __shfl_sync(0xffffffffu, r_cur, wsrc + 2);
                    if (lane < kXWin)
                        xc = x_copy<M>(input_block<M>(a, k), a.n, wlo, wlen, wpos, smem_u32(sx0 + b * Shape<SH>::XW));
                    xbytes = xc.bytes;
#pragma unroll
                    for (int o = 1; o < kXWin; o <<= 1) xbytes += __shfl_xor_sync(0xffffffffu, xbytes, o);
                }
                if (slot_busy[b]) {
                    const uint64_t t0 = globaltimer();
                    bool ok;
                    while (!(ok = mbar_try_wait(&s_empty[b], slot_use[b] & 1)))
                        if (timed_out(t0, a.wait_ns)) break;
                    if (tr && lane == 0) tr_add(3, globaltimer() - t0);
                    if (!ok) {
                        record_timeout();
                        break;
                    }
                    slot_busy[b] = false;
                }
                if (lane == 0) {
                    s_u[b] = u;
                    if (u.staged) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        constexpr uint32_t cb = XS ? 2u : (kStageCol ? 4u : 0u);
                        mbar_expect_tx_only(&s_full[b], (uint32_t)u.ecount * (uint32_t)(sizeof(T) + cb) + xbytes);
                        // the launch's last power is the last use of the unit's entries
                        const bool last_use = (u.unit & 31) == a.p_launch;
                        bulk_g2s(sval0 + b * kStageEntries, static_cast<const T *>(a.val) + u.ebase,
                                 (uint32_t)(u.ecount * sizeof(T)), &s_full[b], last_use);
                        if constexpr (XS)
                            bulk_g2s(slc0 + b * kStageEntries, a.lcol + u.ebase, (uint32_t)u.ecount * 2u, &s_full[b],
                                     last_use);
                        else if (kStageCol)
                            bulk_g2s(scol0 + b * kStageEntries, a.col + u.ebase, (uint32_t)u.ecount * 4u, &s_full[b],
                                     last_use);
                    }
                }
                if constexpr (XS) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    __syncwarp();
                    if (u.staged && xc.bytes) bulk_g2s_addr(xc.dst, xc.src, xc.bytes, &s_full[b]);
                    if (u.staged && xc.tail) {
                        const double v = *reinterpret_cast<const double *>(xc.tail);
                        asm volatile("st.shared.f64 [%0], %1;" ::"r"(xc.tdst), "d"(v) : "memory");
                    }
                }
                if (!useq_slot_free(&s_published, i, a.wait_ns)) {  // (split control: copies may be in flight)
                    record_timeout();
                    if (lane == 0) mbar_arrive(&s_full[b]);
                    const uint64_t t1 = globaltimer();
                    while (!mbar_try_wait(&s_full[b], (i / kSlots) & 1))
                        if (timed_out(t1, a.wait_ns)) break;
                    break;
                }
                if (lane == 0) s_useq[i % kDoneRing] = un;
                __syncwarp();
                if (tr && lane == 0) s_tarr[b] = globaltimer();
                if (lane == 0) mbar_arrive(&s_full[b]);
                slot_busy[b] = true;
                slot_use[b] = i / kSlots;
            }
            if (lane == 0) {
                s_stop = 1;     // the poll warp pushes nothing more
                s_final = i;    // units 0..i-1 were handed over
            }
        }
      } else {
        // ------------------------------------------------------------------ control warp
        const int32_t *rec = reinterpret_cast<const int32_t *>(a.chunk_rec);
        bool slot_busy[kSlots] = {};  // a handed-over unit may still be computed
        int slot_use[kSlots] = {};    // phase index (i / kSlots) of that hand-over
        bool aborted = false;
        auto record_timeout = [&]() {
            if (lane == 0 && atomicExch(a.err, epoch) != epoch) st_relaxed(a.err + 1, (int)MPK_ERR_TIMEOUT);
        };
        auto unit_at = [&](unsigned int t) -> int { return (int64_t)t < a.nunits ? __ldg(a.units + t) : -1; };
        auto rec_at = [&](int un) -> int {
            return (un >= 0 && lane < kRecInts) ? __ldg(rec + kRecInts * (int64_t)(un >> 5) + lane) : 0;
        };
        // claim pipeline, three units deep: unit i (id u_cur, record r_cur), unit i+1 (u_nxt,
        // r_nxt), unit i+2 (id u_nn, held by lane 0) and the ticket t of unit i+3.  At the end
        // of iteration i the record of unit i+2, the id of unit i+3 and one more ticket are
        // fetched, each a full iteration before it is needed.
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
        bool cur_ready = false, nxt_ready = false;  // dependencies already acquired (paired poll)
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
            for (int q = 0; q < Shape<SH>::NW; ++q) u.widths[q] = __shfl_sync(0xffffffffu, r_cur, 16 + q);
            int dlo[kDepRanges], dlen[kDepRanges];
            const int total = dep_ranges_of(r_cur, dlo, dlen);
            const int k = u.unit & 31;
            // shape 3: lane q < kXWin prepares the copy of input-row window q
            XCopy xc{0, 0, 0, 0, 0};
            uint32_t xbytes = 0;
            if constexpr (XS) {
                const int wsrc = kRecWin + 3 * (lane & (kXWin - 1));
                const int wlo = __shfl_sync(0xffffffffu, r_cur, wsrc);
                const int wlen = __shfl_sync(0xffffffffu, r_cur, wsrc + 1);
                const int wpos = __shfl_sync(0xffffffffu, r_cur, wsrc + 2);
                if (lane < kXWin)
                    xc = x_copy<M>(input_block<M>(a, k), a.n, wlo, wlen, wpos,
                                   smem_u32(sx0 + b * Shape<SH>::XW));
                xbytes = xc.bytes;
#pragma unroll
                for (int o = 1; o < kXWin; o <<= 1) xbytes += __shfl_xor_sync(0xffffffffu, xbytes, o);
            }
            if (tr && lane == 0) tr_add(11, clock64() - c0);
            // dependencies of unit i, polled together with those of unit i+1 (one round trip for
            // two units): a unit found ready this way skips its own poll in the next iteration.
            // Its flags were acquired by lanes 16..31, whose order reaches that unit's hand-over
            // through the warp barrier before lane 0's arrival on full[b].
            auto poll_deps = [&]() {
                const bool known = cur_ready;
                cur_ready = false;
                if (k > 1 && !known) {
                    const uint64_t t0 = globaltimer();
                    int nlo[kDepRanges], nlen[kDepRanges];
                    const int ntot = dep_ranges_of(r_nxt, nlo, nlen);
                    const int kn = u_nxt >= 0 ? (u_nxt & 31) : 0;
                    for (;;) {
                        const int rd = deps_ready_pair(a, epoch, k, dlo, dlen, total, kn, nlo, nlen, ntot, lane);
                        nxt_ready = (rd & 2) != 0 && u_nxt >= 0;
                        if (rd & 1) break;
                        if (lane == 0) tr_add(2, 1);
                        const bool stop = ld_relaxed(a.err) == epoch || timed_out(t0, a.wait_ns);
                        if (__any_sync(0xffffffffu, stop)) {
                            aborted = true;
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (tr && lane == 0) tr_add(1, globaltimer() - t0);
                } else {
                    nxt_ready = false;
                }
            };
            // Shape 3 polls first, while slot b may still be in use: its entries and input
            // rows are then copied together as soon as the slot is free.  Nothing has been
            // staged for unit i if the poll gives up: the compute warps stop before it.
            if constexpr (XS) {
                poll_deps();
                if (aborted) {
                    record_timeout();
                    if (lane == 0) s_final = i;
                    break;
                }
            }
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
            // stage the entries (and announce the window bytes, copied after the poll)
            const long long c2 = tr ? clock64() : 0;
            if (lane == 0) {
                s_u[b] = u;
                if (u.staged) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    constexpr uint32_t cb = XS ? 2u : (kStageCol ? 4u : 0u);
                    mbar_expect_tx_only(&s_full[b], (uint32_t)u.ecount * (uint32_t)(sizeof(T) + cb) + xbytes);
                    // the launch's last power is the last use of the unit's entries: they are
                    // copied with the evict_first priority, so that the groups still in their
                    // reuse window keep their L2 lines (measured at 256^3, p = 8: 1.1 % faster
                    // with binary64 sums, 0.6 % with binary32 sums)
                    const bool last_use = (u.unit & 31) == a.p_launch;
                    bulk_g2s(sval0 + b * kStageEntries, static_cast<const T *>(a.val) + u.ebase,
                             (uint32_t)(u.ecount * sizeof(T)), &s_full[b], last_use);
                    if constexpr (XS)
                        bulk_g2s(slc0 + b * kStageEntries, a.lcol + u.ebase, (uint32_t)u.ecount * 2u, &s_full[b],
                                 last_use);
                    else if (kStageCol)
                        bulk_g2s(scol0 + b * kStageEntries, a.col + u.ebase, (uint32_t)u.ecount * 4u, &s_full[b],
                                 last_use);
                }
            }
            if (tr && lane == 0) tr_add(8, clock64() - c2);
            if constexpr (!XS) poll_deps();
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
            // acquire: the flags before the compute warps' reads (via full[b]); units of power
            // 1 read only x0, written before the launch, and poll nothing
            if (k > 1 && !kAcquirePoll) fence_acq_rel_gpu();
            if constexpr (XS) {
                // the input rows were written through the generic proxy and are now read by
                // bulk copies (async proxy): order the acquired writes before those reads
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __syncwarp();
                if (u.staged && xc.bytes) bulk_g2s_addr(xc.dst, xc.src, xc.bytes, &s_full[b]);
                if (u.staged && xc.tail) {
                    const double v = *reinterpret_cast<const double *>(xc.tail);
                    asm volatile("st.shared.f64 [%0], %1;" ::"r"(xc.tdst), "d"(v) : "memory");
                }
            }
            if (!useq_slot_free(&s_published, i, a.wait_ns)) {
                // the unit's entries are staged but it is not handed over: record the failure,
                // complete the slot's phase for its bulk copy and wait for the copy, then stop
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
                aborted = true;
                break;
            }
            if (lane == 0) s_useq[i % kDoneRing] = u.unit;
            __syncwarp();
            if (tr && lane == 0) s_tarr[b] = globaltimer();
            if (lane == 0) mbar_arrive(&s_full[b]);
            const long long c5 = tr ? clock64() : 0;
            if (tr && lane == 0) tr_add(9, c5 - c4);
            slot_busy[b] = true;
            slot_use[b] = i / kSlots;
            // prefetch after the hand-over, so that these loads and the atomic complete during
            // the next units' staging and polls instead of delaying this unit's fence.  The
            // pipeline moves up first and the loads then land directly in its tail (r_nxt,
            // u_nn, t): nothing in this iteration reads a value still in flight.
            u_cur = u_nxt;
            r_cur = r_nxt;
            u_nxt = __shfl_sync(0xffffffffu, u_nn, 0);  // loaded an iteration ago
            r_nxt = rec_at(u_nxt);
            if (lane == 0) {
                u_nn = unit_at(t);            // id of unit i+3
                t = atomicAdd(a.ticket, 1u);  // ticket of unit i+4, claimed whether or not it exists
            }
            cur_ready = nxt_ready;
            nxt_ready = false;
            if (tr && lane == 0) tr_add(10, clock64() - c5);
        }
        if (lane == 0 && s_final < 0) s_final = i;  // units 0..i-1 were handed over
      }
    } else {
        // ------------------------------------------------------------------ compute warps
        const int cw = warp - kCtl - 1;
        Prefetch<M, AT> pf;
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
            if constexpr (XS) {
                const long long c1 = tr ? clock64() : 0;
                phase_x<M, MODE, VT, SH>(a, epoch, s_u, b, sval0, slc0, sx0, s_done, s_empty, cw, lane, i);
                if (tr && lane == 0) tr_add(13, clock64() - c1);
            } else {
                const long long c0 = tr ? clock64() : 0;
                phase_a<M, (kStageEntries > 0), AT, Shape<SH>::NW>(a, s_u[b], b,
                                                     kStageCol ? scol0 + b * kStageEntries : a.col + s_u[b].ebase, cw,
                                                     lane, pf);
                if (tr) {  // wait for the gathers (integer ops only) to split the unit time
                    int h = 0;
#pragma unroll
                    for (int q = 0; q < Batch<M>::B; ++q) h ^= hi_bits(pf.x[q][0]);
                    int d;
                    asm volatile("add.u32 %0, %1, 0;" : "=r"(d) : "r"(h));
                    const long long c1 = clock64();
                    if (lane == 0) tr_add(12, c1 - c0);
                    phase_b<M, MODE, VT, SH, AT>(a, epoch, pf, s_u, sval0, scol0, s_done, s_empty, cw, lane, i);
                    if (lane == 0) tr_add(13, clock64() - c1);
                } else {
                    phase_b<M, MODE, VT, SH, AT>(a, epoch, pf, s_u, sval0, scol0, s_done, s_empty, cw, lane, i);
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


// ----------------------------------------------------------------------------- shape entry points
template <int M, int MODE, class VT, int SH> static void *mpk_fn(bool trace, bool a32) {
    if (a32) {
        if constexpr (Shape<SH>::X || std::is_same<VT, ValF64>::value) {
            fail(MPK_ERR_UNSUPPORTED, "binary32 accumulation needs float32 or bfloat16 values and a shape other than 3");
        } else {
            if (trace) fail(MPK_ERR_UNSUPPORTED, "trace counters need binary64 accumulation");
            return (void *)k_mpk<M, MODE, false, VT, SH, true>;
        }
    }
    return trace ? (void *)k_mpk<M, MODE, true, VT, SH> : (void *)k_mpk<M, MODE, false, VT, SH>;
}

// the host-output kernel: one right-hand side, no trace counters
template <class VT, int SH> static void *mpk_fn_host(bool a32) {
    if (a32) {
        if constexpr (Shape<SH>::X || std::is_same<VT, ValF64>::value) {
            fail(MPK_ERR_UNSUPPORTED, "binary32 accumulation needs float32 or bfloat16 values and a shape other than 3");
        } else {
            return (void *)k_mpk<1, MODE_HOST, false, VT, SH, true>;
        }
    }
    return (void *)k_mpk<1, MODE_HOST, false, VT, SH>;
}

template <class VT, int SH> static void *select_mpk_vs(int mode, int m, bool trace, bool a32) {
    if (mode == MODE_HOST) {
        if (m != 1 || trace) fail(MPK_ERR_UNSUPPORTED, "host output needs nrhs 1 and no trace counters");
        return mpk_fn_host<VT, SH>(a32);
    }
#define SEL(MM)                                                                           \
    if (m == MM) {                                                                        \
        if (mode == MODE_POWERS) return mpk_fn<MM, MODE_POWERS, VT, SH>(trace, a32);      \
        return mpk_fn<MM, MODE_CHEB, VT, SH>(trace, a32);                                 \
    }
    SEL(1) SEL(2) SEL(4) SEL(8)
    if constexpr (Shape<SH>::SE == 0 && !Shape<SH>::X) {  // 16 columns: the unstaged shape only
        SEL(16)
    }
#undef SEL
    fail(MPK_ERR_UNSUPPORTED, "nrhs %d on this block shape", m);
}

// k_mpk of block shape SH for (mode, nrhs, trace, value type, accumulator), and its dynamic shared memory
template <int SH> void *select_mpk_shape(int mode, int m, bool trace, int vtype, bool a32) {
    if (vtype == MPK_F64) return select_mpk_vs<ValF64, SH>(mode, m, trace, a32);
    if (vtype == MPK_F32) return select_mpk_vs<ValF32, SH>(mode, m, trace, a32);
    if (vtype == MPK_BF16) return select_mpk_vs<ValBF16, SH>(mode, m, trace, a32);
    fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
}

template <int SH> int smem_bytes_shape(int vtype) {
    return vtype == MPK_F64 ? smem_bytes<ValF64, SH>()
                            : (vtype == MPK_F32 ? smem_bytes<ValF32, SH>() : smem_bytes<ValBF16, SH>());
}

// defined in mpk_kshape<N>.cu
void *select_mpk_shape0(int mode, int m, bool trace, int vtype, bool a32);
void *select_mpk_shape1(int mode, int m, bool trace, int vtype, bool a32);
void *select_mpk_shape2(int mode, int m, bool trace, int vtype, bool a32);
void *select_mpk_shape3(int mode, int m, bool trace, int vtype, bool a32);
void *select_mpk_shape4(int mode, int m, bool trace, int vtype, bool a32);

}  // namespace mpk
