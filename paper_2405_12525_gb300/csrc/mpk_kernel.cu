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
#include "mpk_kernel_dev.cuh"

#include <type_traits>

namespace mpk {

// ----------------------------------------------------------------------------- K-MPK, warp engine
// The same cells (group g, local power k) in the same order as k_mpk (lines g + kSlotSkew*k
// ascending, k ascending inside a line), split into items of kWarpSlices 32-row slices and
// numbered in that order.  Every warp works alone: warp q of each block claims the items
// q, q + Q, q + 2Q, ... (Q = kWarpQueues) through the claim counter of queue q, so that any
// resident block serves every queue; it waits until every chunk its rows read (the chunk's
// dependency ranges) has all its slices finished at power k-1 (acquire), computes its slice
// with the entries read from global memory (L2, where the line order keeps the working
// set), and adds one to its chunk's counter at power k (release).
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
                row_sum<M, B, double>(GVal<VT>{val}, GCol{a.col}, e0 + lane, (int)((e1 - e0) >> 5), xin, w);
                row_epilogue<M, MODE, double>(a, k, r, w, xin);
            }
        }
        __syncwarp();
        if (lane == 0 && ((c << 5) | k) != a.drop_unit) {  // test hook: a chunk that never completes
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

// ----------------------------------------------------------------------------- sweep engine
// One power k of the whole matrix, unblocked: blocks walk the plan's chunks, warps their
// slices, with the level-blocked kernel's row body and epilogue (plain powers or the
// Chebyshev recurrence), so the results are the same bits.  One launch per power; stream
// order supplies every dependency.
template <int M, int MODE, class VT, bool A32 = false>
__global__ void __launch_bounds__(kSpmvBS) k_sweep(const KArgs a, int k) {
    using AT = typename std::conditional<A32, float, double>::type;
    const int lane = threadIdx.x & 31;
    const auto *val = static_cast<const typename VT::T *>(a.val);
    const double *xin = input_block<M>(a, k);
    const AT *xacc = InputAcc<M, AT>::get(a, k);
    for (int c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        const int r0 = a.chunk_row[c], r1 = a.chunk_row[c + 1], sl0 = a.chunk_slice[c];
        const int nsl = (r1 - r0 + 31) >> 5;
        for (int sl = threadIdx.x >> 5; sl < nsl; sl += kSpmvBS / 32) {
            const int64_t r = (int64_t)r0 + 32 * sl + lane;
            if (r < r1) {
                const int64_t e0 = a.slice_ptr[sl0 + sl], e1 = a.slice_ptr[sl0 + sl + 1];
                AT w[M];
                row_sum<M, Batch<M>::B, AT>(GVal<VT, AT>{val}, GCol{a.col}, e0 + lane, (int)((e1 - e0) >> 5), xacc,
                                            w);
                row_epilogue<M, MODE, AT>(a, k, r, w, xin);
            }
        }
    }
}

template <class VT> static void *select_sweep_vt(int mode, int m, bool a32) {
#define SEL(MM)                                                                                              \
    if (m == MM) {                                                                                           \
        if (a32) {                                                                                           \
            if constexpr (std::is_same<VT, ValF64>::value)                                                   \
                fail(MPK_ERR_UNSUPPORTED, "binary32 accumulation needs float32 or bfloat16 values");          \
            else                                                                                             \
                return mode == MODE_POWERS ? (void *)k_sweep<MM, MODE_POWERS, VT, true>                      \
                                           : (void *)k_sweep<MM, MODE_CHEB, VT, true>;                       \
        }                                                                                                    \
        return mode == MODE_POWERS ? (void *)k_sweep<MM, MODE_POWERS, VT> : (void *)k_sweep<MM, MODE_CHEB, VT>; \
    }
    SEL(1) SEL(2) SEL(4) SEL(8) SEL(16)
#undef SEL
    fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
}

static void *select_sweep(int mode, int m, int vtype, bool a32) {
    if (vtype == MPK_F64) return select_sweep_vt<ValF64>(mode, m, a32);
    if (vtype == MPK_F32) return select_sweep_vt<ValF32>(mode, m, a32);
    if (vtype == MPK_BF16) return select_sweep_vt<ValBF16>(mode, m, a32);
    fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
}

// ----------------------------------------------------------------------------- K-SpMV
// SpMV restricted to row ranges of one or several plans (plan order), one launch: segment
// q covers the plan-order rows [lo, hi) of its plan, whose chunks c0 .. c0+nch-1 overlap
// them; virtual block v belongs to the segment q with first[q] <= v < first[q+1].
// SINGLE: one segment, read with constant offsets (a parameter indexed by a run-time value
// is copied to local memory first).
template <int M, class VT, bool SINGLE>
__global__ void __launch_bounds__(kSpmvBS) k_spmv_rows(const RowSegs segs) {
    const int lane = threadIdx.x & 31;
    for (int v = blockIdx.x; v < segs.first[SINGLE ? 1 : segs.count]; v += gridDim.x) {
        int q = 0;
        if (!SINGLE)
            while (v >= segs.first[q + 1]) ++q;
        const RowSeg &g = segs.seg[SINGLE ? 0 : q];
        const auto *val = static_cast<const typename VT::T *>(g.val);
        const int c = g.c0 + (v - segs.first[q]);
        const int r0 = g.chunk_row[c], r1 = g.chunk_row[c + 1], sl0 = g.chunk_slice[c];
        const int nsl = (r1 - r0 + 31) >> 5;
        for (int sl = threadIdx.x >> 5; sl < nsl; sl += kSpmvBS / 32) {
            const int64_t r = (int64_t)r0 + 32 * sl + lane;
            if (r < r1 && r >= g.lo && r < g.hi) {
                const int64_t s0 = g.slice_ptr[sl0 + sl], s1 = g.slice_ptr[sl0 + sl + 1];
                double w[M];
                row_sum<M, Batch<M>::B, double>(GVal<VT>{val}, GCol{g.col}, s0 + lane, (int)((s1 - s0) >> 5), g.x, w);
#pragma unroll
                for (int i = 0; i < M; ++i) g.y[r * M + i] = w[i];
            }
        }
    }
}

template <class VT>
static void launch_spmv_rows_vt(const RowSegs &segs, int m, cudaStream_t s) {
    const int grid = std::min(segs.first[segs.count], 64 * device_sms());
#define L(MM)                                                                      \
    case MM:                                                                       \
        if (segs.count == 1)                                                       \
            k_spmv_rows<MM, VT, true><<<grid, kSpmvBS, 0, s>>>(segs);              \
        else                                                                       \
            k_spmv_rows<MM, VT, false><<<grid, kSpmvBS, 0, s>>>(segs);             \
        break;
    switch (m) {
        L(1) L(2) L(4) L(8) L(16) default : fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
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

// dst[i] = src[i] rounded to the nearest binary32 (ties to even): the binary32 input of the
// first step of binary32 accumulation
__global__ void k_round_f32(const double *src, int64_t n, float *dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = __double2float_rn(src[i]);
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

// Y[k][i] = W[k][iperm[i]] for k = k0..p: the powers computed in plan order, written in the
// matrix's own order (Y in device memory, or device-mapped pinned host memory).  Stores are full, coalesced rows of the output; the gathered reads
// come from rows that neighbouring original rows map to (for a BFS order these sit a few
// levels apart and share cache sectors with the reads of nearby original rows).  Each block
// walks tiles of consecutive original rows, power by power, so that the sectors a tile reads
// stay in the SM's L1 until its other rows use them.  A thread first loads all of its rows of
// a power (16 values in flight), then stores them, streaming: the output is not read again,
// and L2 keeps the powers still to be read.  Blocks are small (a quarter of an SM's threads
// and registers) so that they also start beside other kernels' blocks, as in serving.
constexpr int kScatterBS = 256, kScatterValues = 16, kScatterBlocksPerSM = 4;

template <int M>
__global__ void __launch_bounds__(kScatterBS, kScatterBlocksPerSM)
    k_scatter_powers(const double *__restrict__ W, int64_t w_pstride, const int32_t *__restrict__ iperm,
                     int32_t w_row0, double *__restrict__ Y, int32_t n, int32_t p, int32_t k0) {
    constexpr int IT = kScatterValues / M;  // rows of a thread in a tile
    constexpr int64_t kTile = (int64_t)kScatterBS * IT;
    const int64_t nm = (int64_t)n * M;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        int32_t src[IT];
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int64_t i = base + (int64_t)q * kScatterBS + threadIdx.x;
            src[q] = i < n ? (iperm ? __ldg(iperm + i) : w_row0 + (int32_t)i) : -1;
        }
        for (int k = k0; k <= p; ++k) {
            const double *w = W + k * w_pstride;
            double *y = Y + k * nm;
            double v[IT][M];
#pragma unroll
            for (int q = 0; q < IT; ++q)
#pragma unroll
                for (int c = 0; c < M; ++c) v[q][c] = src[q] >= 0 ? __ldg(w + (int64_t)src[q] * M + c) : 0.0;
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                const int64_t i = base + (int64_t)q * kScatterBS + threadIdx.x;
                if (src[q] >= 0) {
#pragma unroll
                    for (int c = 0; c < M; ++c) __stcs(y + i * M + c, v[q][c]);
                }
            }
        }
    }
}

void launch_scatter_powers(const double *W, const int32_t *iperm, double *Y, int32_t n, int32_t m, int32_t p,
                           cudaStream_t s, int64_t w_pstride, int32_t base, int32_t k0) {
    if (n <= 0 || p < k0) return;
    if (w_pstride < 0) w_pstride = (int64_t)n * m;
    const int g = device_sms() * kScatterBlocksPerSM;
    switch (m) {
        case 1: k_scatter_powers<1><<<g, kScatterBS, 0, s>>>(W, w_pstride, iperm, base, Y, n, p, k0); break;
        case 2: k_scatter_powers<2><<<g, kScatterBS, 0, s>>>(W, w_pstride, iperm, base, Y, n, p, k0); break;
        case 4: k_scatter_powers<4><<<g, kScatterBS, 0, s>>>(W, w_pstride, iperm, base, Y, n, p, k0); break;
        case 8: k_scatter_powers<8><<<g, kScatterBS, 0, s>>>(W, w_pstride, iperm, base, Y, n, p, k0); break;
        case 16: k_scatter_powers<16><<<g, kScatterBS, 0, s>>>(W, w_pstride, iperm, base, Y, n, p, k0); break;
        default: fail(MPK_ERR_UNSUPPORTED, "scatter of %d right-hand sides", m);
    }
    MPK_LAUNCHED();
}

void launch_round_f32(const double *src, int64_t n, float *dst, cudaStream_t s) {
    if (n <= 0) return;
    k_round_f32<<<grid_rows(n), 256, 0, s>>>(src, n, dst);
    MPK_LAUNCHED();
}

void launch_cheb_init(const double *v0, double *acc, int32_t n, int32_t m, double c0re, double c0im, int cplx,
                      cudaStream_t s) {
    if (n <= 0) return;
    k_cheb_init<<<grid_rows(n), 256, 0, s>>>(v0, acc, n, m, c0re, c0im, cplx);
    MPK_LAUNCHED();
}

// ----------------------------------------------------------------------------- launches
static void *select_mpk(int mode, int m, bool trace, int vtype, int shape, bool a32) {
    if (shape == 0) return select_mpk_shape0(mode, m, trace, vtype, a32);
    if (shape == 1) return select_mpk_shape1(mode, m, trace, vtype, a32);
    if (shape == 2) return select_mpk_shape2(mode, m, trace, vtype, a32);
    if (shape == 3) return select_mpk_shape3(mode, m, trace, vtype, a32);
    return select_mpk_shape4(mode, m, trace, vtype, a32);
}

static int mpk_smem_bytes(int vtype, int shape) {
    switch (shape) {
        case 0: return smem_bytes_shape<0>(vtype);
        case 1: return smem_bytes_shape<1>(vtype);
        case 2: return smem_bytes_shape<2>(vtype);
        case 3: return smem_bytes_shape<3>(vtype);
        default: return smem_bytes_shape<4>(vtype);
    }
}

static int mpk_block_size(int shape) {
    switch (shape) {
        case 0: return Shape<0>::BS;
        case 1: return Shape<1>::BS;
        case 2: return Shape<2>::BS;
        case 3: return Shape<3>::BS;
        default: return Shape<4>::BS;
    }
}

int occupancy_grid(int mode, int m, bool trace, int vtype, int shape, bool a32) {
    static int cache[3][3][2][5][kNumShapes][2] = {};  // width index: log2 of m (1 .. 16)
    if (vtype < 0 || vtype > 2) fail(MPK_ERR_UNSUPPORTED, "value type %d", vtype);
    if (mode < 0 || mode > 2) fail(MPK_ERR_INVALID, "kernel mode %d", mode);
    if (shape < 0 || shape >= kNumShapes) fail(MPK_ERR_UNSUPPORTED, "block shape %d", shape);
    if (m < 1 || m > 16 || (m & (m - 1))) fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
    int &c = cache[vtype][mode][trace ? 1 : 0][__builtin_ctz((unsigned)m)][shape][a32 ? 1 : 0];
    if (c) return c;
    void *fn = select_mpk(mode, m, trace, vtype, shape, a32);
    const int smem = mpk_smem_bytes(vtype, shape);
    MPK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, mpk_block_size(shape), smem));
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
    const bool a32 = P.accum == MPK_F32;
    if (P.engine == MPK_ENGINE_SWEEP && a.trace == nullptr && a.drop_unit < 0 && a.w_item == nullptr) {
        if (P.num_chunks <= 0) return;
        void *fn = select_sweep(mode, P.m, P.val_type, a32);
        const int grid = std::min(P.num_chunks, 64 * device_sms());
        for (int k = 1; k <= a.p_launch; ++k) {
            void *args[] = {&a, &k};
            MPK_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kSpmvBS), args, 0, s));
        }
        return;
    }
    if (a.w_item != nullptr && a.trace == nullptr) {  // warp engine
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
    int grid = occupancy_grid(mode, P.m, trace, P.val_type, P.shape, a32);
    if ((int64_t)grid > a.nunits) grid = (int)a.nunits;
    void *fn = select_mpk(mode, P.m, trace, P.val_type, P.shape, a32);
    void *args[] = {&a};
    MPK_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(mpk_block_size(P.shape)), args, mpk_smem_bytes(P.val_type, P.shape),
                              s));
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
    if (reinterpret_cast<uintptr_t>(buf) % 16) fail(MPK_ERR_INVALID, "probe_load: buf is not 16-byte aligned");
    k_probe_load<<<device_sms() * ctas_per_sm, 512, 0, s>>>(static_cast<const int4 *>(buf), bytes / 16, reps, sink);
    MPK_LAUNCHED();
}

void probe_dfma(int blocks, int iters, double *sink, cudaStream_t s) {
    if (!sink || blocks < 1 || iters < 1) fail(MPK_ERR_INVALID, "probe_dfma: bad arguments");
    k_probe_dfma<<<blocks, 256, 0, s>>>(iters, sink);
    MPK_LAUNCHED();
}

}  // namespace mpk
