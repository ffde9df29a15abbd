// Hot path: the persistent level-blocked MPK kernel (Sec. 3, Fig. 2; Alg. 2's local phase),
// the plain SpMV comparator (Alg. 1), gather/scatter between row orders, and probes.
//
// Row body.  GB300 executes FP64 FMA at 2 lanes per clock per SM (about 0.6 T FMA/s for
// the whole GPU), so FP64 SpMV is bound by the FP64 pipe about as much as by HBM.  The
// row body therefore spends exactly one DFMA per stored entry and right-hand side: one
// thread owns one row and accumulates its entries sequentially in stored order (no
// shuffle-tree reduction, which would add FP64 additions).  The matrix copy is sliced by
// 32 rows (entry j of lane l at slice_ptr + 32 j + l) so that a warp's loads of entry j
// are contiguous.  The result equals the oracle's fma-per-term row sums bit for bit.
#include "mpk_internal.h"

namespace mpk {

constexpr int kBS = 256;            // threads per block (8 warps)
constexpr int kWarps = kBS / 32;

enum Mode { MODE_PLAN = 0, MODE_SCATTER = 1, MODE_CHEB = 2 };

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

// acc[i] = sum_j val[j] * x[col[j]*M + i] over row r's entries, in stored order
template <int M>
__device__ __forceinline__ void row_sum(const double *__restrict__ val, const int32_t *__restrict__ col,
                                        int64_t base, int len, const double *x, double (&acc)[M]) {
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = 0.0;
    int j = 0;
    for (; j + 1 < len; j += 2) {   // two entries per trip: loads of j+1 overlap the FMAs of j
        const double v0 = __ldg(val + base + 32 * (int64_t)j);
        const double v1 = __ldg(val + base + 32 * (int64_t)(j + 1));
        const int32_t c0 = __ldg(col + base + 32 * (int64_t)j);
        const int32_t c1 = __ldg(col + base + 32 * (int64_t)(j + 1));
        double x0[M], x1[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            x0[i] = x[(int64_t)c0 * M + i];
            x1[i] = x[(int64_t)c1 * M + i];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) acc[i] = fma(v0, x0[i], acc[i]);
#pragma unroll
        for (int i = 0; i < M; ++i) acc[i] = fma(v1, x1[i], acc[i]);
    }
    if (j < len) {
        const double v0 = __ldg(val + base + 32 * (int64_t)j);
        const int32_t c0 = __ldg(col + base + 32 * (int64_t)j);
#pragma unroll
        for (int i = 0; i < M; ++i) acc[i] = fma(v0, x[(int64_t)c0 * M + i], acc[i]);
    }
}

// Epilogue of one row at local power k: store into the plan-order slot, optionally into
// the original-order output, or advance the Chebyshev recurrence.
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
        if constexpr (MODE == MODE_SCATTER) {
            double *yo = a.yorig + (int64_t)j * a.ostride + (int64_t)a.perm[r] * M;
#pragma unroll
            for (int i = 0; i < M; ++i) yo[i] = w[i];
        }
    }
}

// ----------------------------------------------------------------------------- K-MPK
// Work unit = (row chunk c, local power k).  Units are claimed through one atomic ticket
// in the order of the unit table, which lists the Lp-diagram cells (group g, power k)
// diagonal by diagonal (g + k ascending) and, inside a diagonal, k ascending.  Every
// dependency of a unit (chunks holding the rows it reads, at power k-1) lies on an earlier
// diagonal or earlier in the same one, so it has a smaller ticket: the unit holding the
// smallest unfinished ticket can always run, whichever blocks are resident, and the
// schedule cannot deadlock.  A finished unit publishes flags[k][c] = epoch (release);
// a unit waits until flags[k-1][lo..hi] all equal the epoch (acquire).  Each block claims
// its next ticket while it waits for the current one.  Waits are bounded by
// a.wait_ns (globaltimer); on expiry the block records the epoch and MPK_ERR_TIMEOUT in
// a.err and all blocks drain out.  The last block to exit resets the ticket.
template <int M, int MODE>
__global__ void __launch_bounds__(kBS) k_mpk(const KArgs a) {
    __shared__ int s_unit[2];
    __shared__ int2 s_dep[2];
    __shared__ int s_row[2][2];
    __shared__ int s_slice[2];
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    auto claim = [&](int slot) {
        const unsigned int t = atomicAdd(a.ticket, 1u);
        if ((int64_t)t >= a.nunits) {
            s_unit[slot] = -1;
            return;
        }
        const int u = __ldg(a.units + t);
        const int c = u >> 5;
        s_unit[slot] = u;
        s_dep[slot] = __ldg(a.dep + c);
        s_row[slot][0] = __ldg(a.chunk_row + c);
        s_row[slot][1] = __ldg(a.chunk_row + c + 1);
        s_slice[slot] = __ldg(a.chunk_slice + c);
    };

    if (tid == 0) {
        s_abort = 0;
        claim(0);
    }
    __syncthreads();
    int cur = 0;
    while (true) {
        const int u = s_unit[cur];
        if (u < 0) break;
        const int k = u & 31, c = u >> 5;
        if (tid == 32) claim(cur ^ 1);
        if (k > 1 && warp == 0) {
            // wait until the chunks [lo, hi] have finished power k-1
            const int32_t *f = a.flags + (int64_t)(k - 1) * a.nchunks;
            int lo = s_dep[cur].x;
            const int hi = s_dep[cur].y;
            const uint64_t t0 = globaltimer();
            bool failed = false;
            while (true) {
                int first_bad = hi + 1;
                for (int i = lo + lane; i <= hi; i += 32)
                    if (ld_relaxed(f + i) != a.epoch) {
                        first_bad = i;
                        break;
                    }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) first_bad = min(first_bad, __shfl_xor_sync(0xffffffffu, first_bad, d));
                if (first_bad > hi) break;
                lo = first_bad;
                const bool stop = ld_relaxed(a.err) == a.epoch || globaltimer() - t0 > (uint64_t)a.wait_ns;
                if (__any_sync(0xffffffffu, stop)) {
                    failed = true;
                    break;
                }
                __nanosleep(128);
            }
            if (failed) {
                if (lane == 0) {
                    // first block to give up in this launch records the timeout
                    if (atomicExch(a.err, a.epoch) != a.epoch) st_relaxed(a.err + 1, (int)MPK_ERR_TIMEOUT);
                    s_abort = 1;
                }
            } else {
                __threadfence();  // acquire: order the flag reads before the block's data reads
            }
        }
        __syncthreads();
        if (s_abort) break;

        // ---- rows of chunk c at power k
        const int r0 = s_row[cur][0], r1 = s_row[cur][1], sl0 = s_slice[cur];
        const int nsl = (r1 - r0 + 31) >> 5;
        // input block: power (k_offset + k - 1); the very first power reads x0
        const double *xin = (k == 1 && a.k_offset == 0)
                                ? a.x0
                                : a.ybase + (int64_t)((a.k_offset + k - 1) % a.ring) * a.ystride;
        for (int sl = warp; sl < nsl; sl += kWarps) {
            const int64_t r = (int64_t)r0 + 32 * sl + lane;
            if (r < r1) {
                const int64_t base = __ldg(a.slice_ptr + sl0 + sl) + lane;
                const int len = __ldg(a.rowlen + r);
                double w[M];
                row_sum<M>(a.val, a.col, base, len, xin, w);
                row_epilogue<M, MODE>(a, k, r, w, xin);
                if (k == 1 && a.y0copy) {
#pragma unroll
                    for (int i = 0; i < M; ++i) a.y0copy[r * M + i] = a.x0[r * M + i];
                }
            }
        }
        __syncthreads();
        if (tid == 0 && u != a.drop_unit) {
            __threadfence();  // release: the block's stores before the flag
            st_relaxed(a.flags + (int64_t)k * a.nchunks + c, a.epoch);
        }
        cur ^= 1;
    }
    // ---- exit: the last block resets the ticket for the next launch on the stream
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.exit_count, 1u);
        if (done == gridDim.x - 1) {
            *a.ticket = 0u;
            *a.exit_count = 0u;
            __threadfence();
        }
    }
}

// ----------------------------------------------------------------------------- K-SpMV
// One plain SpMV over the plan's sliced copy: y = A x (plan order), same row body.
// One warp per slice.  Optionally also writes yorig[perm[r]].
template <int M>
__global__ void __launch_bounds__(kBS) k_spmv(const double *__restrict__ val, const int32_t *__restrict__ col,
                                              const int64_t *__restrict__ slice_ptr,
                                              const int32_t *__restrict__ rowlen, const int32_t *__restrict__ chunk_row,
                                              const int32_t *__restrict__ chunk_slice, int32_t nchunks,
                                              const double *x, double *y, double *yorig,
                                              const int32_t *__restrict__ perm) {
    const int lane = threadIdx.x & 31;
    // blocks walk chunks; warps walk the chunk's slices
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int r0 = chunk_row[c], r1 = chunk_row[c + 1], sl0 = chunk_slice[c];
        const int nsl = (r1 - r0 + 31) >> 5;
        for (int sl = threadIdx.x >> 5; sl < nsl; sl += kWarps) {
            const int64_t r = (int64_t)r0 + 32 * sl + lane;
            if (r < r1) {
                const int64_t base = slice_ptr[sl0 + sl] + lane;
                double w[M];
                row_sum<M>(val, col, base, rowlen[r], x, w);
#pragma unroll
                for (int i = 0; i < M; ++i) y[r * M + i] = w[i];
                if (yorig) {
                    double *yo = yorig + (int64_t)perm[r] * M;
#pragma unroll
                    for (int i = 0; i < M; ++i) yo[i] = w[i];
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------- row moves
// dst[r] = src[perm[r]] (m values per row); coalesced writes
__global__ void k_gather_rows(const double *src, const int32_t *perm, double *dst, int32_t n, int32_t m) {
    const int64_t total = (int64_t)n * m, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t r = t / m, i = t - r * m;
        dst[t] = src[(int64_t)(perm ? perm[r] : r) * m + i];
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

void launch_gather_rows(const double *src, const int32_t *perm, double *dst, int32_t n, int32_t m, cudaStream_t s) {
    if (n <= 0) return;
    k_gather_rows<<<grid_rows((int64_t)n * m), 256, 0, s>>>(src, perm, dst, n, m);
    MPK_LAUNCHED();
}

// dst[i] = src[iperm[i]]: scatter expressed as a gather by output row
void launch_scatter_rows(const double *src, const int32_t *iperm, double *dst, int32_t n, int32_t m, cudaStream_t s) {
    launch_gather_rows(src, iperm, dst, n, m, s);
}

void launch_cheb_init(const double *v0, double *acc, int32_t n, int32_t m, double c0re, double c0im, int cplx,
                      cudaStream_t s) {
    if (n <= 0) return;
    k_cheb_init<<<grid_rows(n), 256, 0, s>>>(v0, acc, n, m, c0re, c0im, cplx);
    MPK_LAUNCHED();
}

// ----------------------------------------------------------------------------- launches
template <int M, int MODE> static void *mpk_fn() { return (void *)k_mpk<M, MODE>; }

static void *select_mpk(int mode, int m) {
#define SEL(MM)                                            \
    if (m == MM) {                                         \
        if (mode == MODE_PLAN) return mpk_fn<MM, MODE_PLAN>();       \
        if (mode == MODE_SCATTER) return mpk_fn<MM, MODE_SCATTER>(); \
        return mpk_fn<MM, MODE_CHEB>();                    \
    }
    SEL(1) SEL(2) SEL(4) SEL(8)
#undef SEL
    fail(MPK_ERR_UNSUPPORTED, "nrhs %d", m);
}

int occupancy_grid(int mode, int m) {
    static int cache[3][9] = {};
    const int mi = m;
    if (cache[mode][mi]) return cache[mode][mi];
    int per_sm = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_mpk(mode, m), kBS, 0));
    if (per_sm < 1) per_sm = 1;
    cache[mode][mi] = per_sm * device_sms();
    return cache[mode][mi];
}

void launch_mpk(const Plan &P, KArgs &a, int mode, cudaStream_t s) {
    if (a.nunits <= 0) return;
    int grid = occupancy_grid(mode, P.m);
    if ((int64_t)grid > a.nunits) grid = (int)a.nunits;
    void *fn = select_mpk(mode, P.m);
    void *args[] = {&a};
    MPK_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kBS), args, 0, s));
}

void launch_spmv(const Plan &P, const double *x, double *y, double *yorig, int64_t orig_off, cudaStream_t s) {
    if (P.num_chunks <= 0) return;
    int grid = P.num_chunks;
    double *yo = yorig ? yorig + orig_off : nullptr;
#define L(MM)                                                                                                 \
    case MM:                                                                                                  \
        k_spmv<MM><<<grid, kBS, 0, s>>>(P.val, P.col, P.slice_ptr, P.rowlen, P.chunk_row, P.chunk_slice,     \
                                        P.num_chunks, x, y, yo, P.perm);                                      \
        break;
    switch (P.m) {
        L(1) L(2) L(4) L(8) default : fail(MPK_ERR_UNSUPPORTED, "nrhs %d", P.m);
    }
#undef L
    MPK_LAUNCHED();
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
