// Device primitives used by the level builder and the planner: prefix sums, a stable
// LSD radix sort, fills; plus error reporting and allocation accounting.
#include "mpk_internal.h"

#include <cstring>
#include <string>

namespace mpk {

// ----------------------------------------------------------------------------- errors
static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void fail(mpk_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    throw Fail{s};
}

const char *last_error_text() { return g_err; }

// ----------------------------------------------------------------------------- memory
void *Arena::alloc(int64_t nbytes) {
    if (nbytes <= 0) nbytes = 16;
    nbytes = (nbytes + 255) & ~int64_t(255);
    if (budget > 0 && bytes + nbytes > budget)
        fail(MPK_ERR_BUDGET, "plan needs more than its memory budget of %lld bytes", (long long)budget);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)nbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(MPK_ERR_OOM, "cudaMalloc(%lld) failed: %s", (long long)nbytes, cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    sizes.push_back(nbytes);
    bytes += nbytes;
    return p;
}

void Arena::free(void *p) {
    if (!p) return;
    for (size_t i = 0; i < ptrs.size(); ++i)
        if (ptrs[i] == p) {
            cudaFree(p);
            bytes -= sizes[i];
            ptrs.erase(ptrs.begin() + i);
            sizes.erase(sizes.begin() + i);
            return;
        }
}

void Arena::release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    sizes.clear();
    bytes = 0;
}

int device_sms() {
    int dev = 0, v = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    MPK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v;
}

int64_t device_l2_bytes() {
    int dev = 0, v = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    MPK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev));
    return v;
}

// ----------------------------------------------------------------------------- fills
__global__ void k_fill_i32(int32_t *p, int32_t v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void k_iota_i32(int32_t *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
static int grid_for(int64_t n, int bs) {
    int64_t g = (n + bs - 1) / bs;
    int64_t cap = (int64_t)device_sms() * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}
void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    MPK_LAUNCHED();
}
void iota_i32(int32_t *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_iota_i32<<<grid_for(n, 256), 256, 0, s>>>(p, n);
    MPK_LAUNCHED();
}

// ----------------------------------------------------------------------------- scan
// Blocked exclusive scan: a tile of SCAN_TILE elements per block, ITEMS consecutive per
// thread.  Three passes: tile totals, scan of totals (recursive), tile scans with offsets.
constexpr int SCAN_BS = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_BS * SCAN_ITEMS;

template <class T> __device__ T block_exclusive(T v, T *total) {
    __shared__ T warp_sums[SCAN_BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_BS / 32 ? warp_sums[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += o;
        }
        if (lane < SCAN_BS / 32) warp_sums[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31) *total = wi;                         // lanes past the last warp add 0
    }
    __syncthreads();
    T r = warp_sums[warp] + inc - v;
    __syncthreads();
    return r;
}

template <class T> __global__ void k_scan_totals(const T *in, int64_t n, T *totals) {
    const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    __shared__ T tot;
    block_exclusive<T>(s, &tot);
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

template <class T> __global__ void k_scan_tiles(const T *in, T *out, int64_t n, const T *offsets) {
    const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    __shared__ T tot;
    T run = block_exclusive<T>(s, &tot) + (offsets ? offsets[blockIdx.x] : T(0));
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        out[n] = (offsets ? offsets[blockIdx.x] : T(0)) + tot;
}

template <class T> static void scan_impl(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        MPK_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
        return;
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_tiles<T><<<1, SCAN_BS, 0, s>>>(in, out, n, nullptr);
        MPK_LAUNCHED();
        return;
    }
    Tmp<T> totals(tiles + 1, s);
    k_scan_totals<T><<<(unsigned)tiles, SCAN_BS, 0, s>>>(in, n, totals.p);
    MPK_LAUNCHED();
    scan_impl<T>(totals.p, totals.p, tiles, s);
    k_scan_tiles<T><<<(unsigned)tiles, SCAN_BS, 0, s>>>(in, out, n, totals.p);
    MPK_LAUNCHED();
    // the temporary is freed after the stream drains
    MPK_CUDA(cudaStreamSynchronize(s));
}

void exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) { scan_impl<int32_t>(in, out, n, s); }
void exclusive_scan(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }

// ----------------------------------------------------------------------------- radix sort
// One pass sorts by an 8-bit digit.  Tiles of RS_TILE elements are striped over the
// threads (element = tile_base + round * RS_BS + thread) so that rounds in order and
// threads in order visit the tile in element order, which keeps every pass stable.
constexpr int RS_BS = 256, RS_ROUNDS = 8, RS_TILE = RS_BS * RS_ROUNDS, RS_WARPS = RS_BS / 32;

__global__ void k_radix_hist(const uint32_t *keys, int64_t n, int shift, int32_t *counts, int64_t ntiles) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = blockIdx.x * (int64_t)RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * RS_BS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];  // digit-major
}

__global__ void k_radix_scatter(const uint32_t *keys, const uint32_t *vals, int64_t n, int shift,
                                const int32_t *offsets, int64_t ntiles, uint32_t *keys_out,
                                uint32_t *vals_out) {
    __shared__ int32_t s_off[256];
    __shared__ int32_t s_run[256];
    __shared__ int32_t s_cnt[RS_WARPS * 256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    s_off[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
    s_run[t] = 0;
    for (int w = 0; w < RS_WARPS; ++w) s_cnt[w * 256 + t] = 0;
    __syncthreads();
    const int64_t base = blockIdx.x * (int64_t)RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * RS_BS + t;
        const bool valid = i < n;
        uint32_t key = 0, val = 0;
        int d = 256 + lane;  // unique non-digit for invalid lanes
        if (valid) {
            key = keys[i];
            val = vals[i];
            d = (int)((key >> shift) & 255u);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) s_cnt[warp * 256 + d] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over warps, continuing the running count
            int run = s_run[t];
            for (int w = 0; w < RS_WARPS; ++w) {
                const int c = s_cnt[w * 256 + t];
                s_cnt[w * 256 + t] = run;
                run += c;
            }
            s_run[t] = run;
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = (int64_t)s_off[d] + s_cnt[warp * 256 + d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        for (int w = 0; w < RS_WARPS; ++w) s_cnt[w * 256 + t] = 0;
        __syncthreads();
    }
}

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp, int64_t n,
                      int key_bits, cudaStream_t s, uint32_t **keys_out, uint32_t **vals_out) {
    uint32_t *ka = keys, *va = vals, *kb = keys_tmp, *vb = vals_tmp;
    if (n > 0 && key_bits > 0) {
        const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
        if (ntiles * 256 >= (int64_t)1 << 31) fail(MPK_ERR_TOO_LARGE, "radix sort: too many tiles");
        Tmp<int32_t> counts(ntiles * 256 + 1, s);
        for (int shift = 0; shift < key_bits; shift += 8) {
            k_radix_hist<<<(unsigned)ntiles, RS_BS, 0, s>>>(ka, n, shift, counts.p, ntiles);
            MPK_LAUNCHED();
            exclusive_scan(counts.p, counts.p, ntiles * 256, s);
            k_radix_scatter<<<(unsigned)ntiles, RS_BS, 0, s>>>(ka, va, n, shift, counts.p, ntiles, kb, vb);
            MPK_LAUNCHED();
            uint32_t *t;
            t = ka; ka = kb; kb = t;
            t = va; va = vb; vb = t;
        }
        MPK_CUDA(cudaStreamSynchronize(s));
    }
    *keys_out = ka;
    *vals_out = va;
}

}  // namespace mpk
