// Level builder: CSR validation, the pattern of A + A^T, level-synchronous BFS and the
// BFS permutation (Sec. 3, level definition, prose and Fig. 1).
#include "mpk_internal.h"

#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

namespace mpk {
namespace cg = cooperative_groups;

// err[0]: bad row pointer, err[1]: column out of range
__global__ void k_validate(int32_t n, int32_t nnz, const int32_t *rp, const int32_t *ci, int32_t *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t a = rp[i], b = rp[i + 1];
        if (a > b || a < 0 || b > nnz || (i == 0 && a != 0) || (i == n - 1 && b != nnz)) {
            atomicExch(&err[0], 1);
            continue;
        }
        for (int32_t e = a; e < b; ++e) {
            const int32_t c = ci[e];
            if (c < 0 || c >= n) {
                atomicExch(&err[1], 1);
                break;
            }
        }
    }
}

void validate_csr(const mpk_csr *A, cudaStream_t s) {
    if (!A) fail(MPK_ERR_INVALID, "matrix is NULL");
    if (A->n < 0 || A->nnz < 0) fail(MPK_ERR_INVALID, "negative n (%d) or nnz (%d)", A->n, A->nnz);
    if (A->val_type != MPK_F64 && A->val_type != MPK_F32 && A->val_type != MPK_BF16)
        fail(MPK_ERR_UNSUPPORTED, "value type %d (MPK_F64, MPK_F32 or MPK_BF16)", A->val_type);
    if (A->n == 0) return;
    if (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
        fail(MPK_ERR_INVALID, "NULL CSR array");
    Tmp<int32_t> err(2, s);
    MPK_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int32_t), s));
    int g = (int)((A->n + 255) / 256);
    if (g > device_sms() * 16) g = device_sms() * 16;
    k_validate<<<g, 256, 0, s>>>(A->n, A->nnz, A->row_ptr, A->col, err.p);
    MPK_LAUNCHED();
    int32_t h[2];
    MPK_CUDA(cudaMemcpyAsync(h, err.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    MPK_CUDA(cudaStreamSynchronize(s));
    if (h[0]) fail(MPK_ERR_INVALID, "row_ptr is not a valid CSR row pointer (0 .. nnz, non-decreasing)");
    if (h[1]) fail(MPK_ERR_INVALID, "column index outside [0, n)");
}

// ----------------------------------------------------------------------------- A^T pattern
__global__ void k_tcount(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] != i) atomicAdd(&cnt[ci[e]], 1);
}
__global__ void k_tfill(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *pos, int32_t *tci) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] != i) tci[atomicAdd(&pos[ci[e]], 1)] = (int32_t)i;
}

// ----------------------------------------------------------------------------- BFS on the device
// The whole level-synchronous BFS in one cooperative launch (every block resident): per level the
// blocks expand the frontier queue[head, tail) into level lev + 1 (appending at queue[tail + ..]),
// meet at a grid barrier and all read the number found, so every block advances head, tail and
// lev identically.  The counters rotate through three slots: phase q adds to slot q % 3 and
// resets slot (q + 1) % 3, whose last readers (after barrier q - 2) have all passed barrier q - 1.
// A graph whose search runs dry before every vertex is reached continues from the smallest
// untouched vertex (a grid-wide minimum, one barrier), which opens the next level (one more
// barrier to publish it).  Every barrier wait is bounded; on expiry the kernel records the
// failure and all blocks leave.
constexpr int64_t kBfsWaitNs = 2000000000LL;  // bound of one grid-barrier wait (2 s)
struct BfsState {
    unsigned int bar_count;  // arrivals at grid barriers, all rounds
    int32_t cnt[3];    // vertices found per phase
    int32_t minv[3];   // smallest untouched vertex per phase (INT_MAX: none)
    int32_t levels;    // number of levels (written at the end)
    int32_t err;       // 1: a barrier wait expired, 2: the search lost track of untouched vertices
};

__device__ __forceinline__ uint64_t bfs_clock() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// all blocks of the grid, barrier number `round` (counted by the caller, the same in every
// block): the arrivals only grow, and barrier r is passed once r * gridDim.x blocks arrived.
// Thread 0 arrives with an acquire-release add (the block's writes, ordered before it by the
// block barrier, are released; the earlier arrivals acquired) and polls with acquire loads.
// False when the wait expired (recorded in st->err).
__device__ __forceinline__ bool bfs_grid_barrier(BfsState *st, unsigned int round, int64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = round * gridDim.x;
        unsigned int v;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(v) : "l"(&st->bar_count) : "memory");
        s_ok = 1;
        if (v + 1 < target) {
            const uint64_t t0 = bfs_clock();
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&st->bar_count) : "memory");
                if (v >= target) break;
                if (bfs_clock() - t0 > (uint64_t)limit_ns) {
                    atomicCAS(&st->err, 0, 1);
                    s_ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();
    return s_ok != 0;
}

// appends u at queue[tail + *cnt++]; the lanes of a warp that append together (a coalesced
// group) share one atomic, each writing at its rank in the group
__device__ __forceinline__ void bfs_append(int32_t *queue, int64_t tail, int32_t *cnt, int32_t u) {
    cg::coalesced_group g = cg::coalesced_threads();
    int32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(cnt, (int32_t)g.size());
    base = g.shfl(base, 0);
    queue[tail + base + (int64_t)g.thread_rank()] = u;
}

// neighbours ci[e0 .. e1) of v join level `next` unless reached (CAS from -1), eight at a time:
// their columns, then their levels, then the claims, so that a vertex's work is a few memory
// round trips instead of two per neighbour
__device__ __forceinline__ void bfs_visit(const int32_t *ci, int32_t e0, int32_t e1, int32_t v, int32_t *level_of,
                                          int32_t next, int32_t *queue, int64_t tail, int32_t *cnt) {
    for (int32_t eb = e0; eb < e1; eb += 8) {
        int32_t u[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = (eb + q < e1) ? ci[eb + q] : v;
#pragma unroll
        for (int q = 0; q < 8; ++q) l[q] = (u[q] != v) ? level_of[u[q]] : 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (l[q] < 0 && atomicCAS(&level_of[u[q]], -1, next) == -1) bfs_append(queue, tail, cnt, u[q]);
    }
}

__global__ void __launch_bounds__(256) k_bfs_all(const int32_t *rp, const int32_t *ci, const int32_t *tp,
                                                 const int32_t *tci, int32_t *level_of, int32_t *queue, int32_t n,
                                                 int32_t head0, int32_t tail0, BfsState *st, int64_t limit_ns) {
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    int64_t head = head0, tail = tail0, cursor = 0;
    int32_t lev = 0;
    int q = 0;               // phase
    unsigned int round = 0;  // grid barriers passed
    for (;;) {
        // expand level lev
        if (gtid == 0) {
            st->cnt[(q + 1) % 3] = 0;
            st->minv[(q + 1) % 3] = INT_MAX;
        }
        int32_t *cnt = &st->cnt[q % 3];
        for (int64_t t = head + gtid; t < tail; t += gstride) {
            const int32_t v = queue[t];
            bfs_visit(ci, rp[v], rp[v + 1], v, level_of, lev + 1, queue, tail, cnt);
            if (tp) bfs_visit(tci, tp[v], tp[v + 1], v, level_of, lev + 1, queue, tail, cnt);
        }
        if (!bfs_grid_barrier(st, ++round, limit_ns)) return;
        const int32_t found = *(volatile int32_t *)cnt;
        ++q;
        head = tail;
        tail += found;
        if (found > 0) {
            ++lev;
            continue;
        }
        if (tail >= n) break;
        // the search ran dry: the smallest untouched vertex (all below cursor are reached)
        int32_t *mn = &st->minv[q % 3];
        for (int64_t i = cursor + gtid; i < n; i += gstride)
            if (level_of[i] < 0) {
                atomicMin(mn, (int32_t)i);
                break;
            }
        if (gtid == 0) {
            st->cnt[(q + 1) % 3] = 0;
            st->minv[(q + 1) % 3] = INT_MAX;
        }
        if (!bfs_grid_barrier(st, ++round, limit_ns)) return;
        const int32_t v = *(volatile int32_t *)mn;
        ++q;
        if (v == INT_MAX) {
            if (gtid == 0) atomicCAS(&st->err, 0, 2);
            return;
        }
        cursor = v;
        ++lev;
        if (gtid == 0) {
            level_of[v] = lev;
            queue[tail] = v;
        }
        tail += 1;
        if (!bfs_grid_barrier(st, ++round, limit_ns)) return;  // the new root before its expansion
    }
    if (gtid == 0) st->levels = lev + 1;
}

__global__ void k_set_root(int32_t *level_of, int32_t *queue_slot, int32_t v, int32_t level) {
    level_of[v] = level;
    *queue_slot = v;
}

// level 0 = every root (roots distinct)
__global__ void k_set_roots(int32_t *level_of, int32_t *queue, const int32_t *roots, int32_t nroots) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nroots; i += gridDim.x * blockDim.x) {
        level_of[roots[i]] = 0;
        queue[i] = roots[i];
    }
}

__global__ void k_inverse(const uint32_t *perm, int32_t *iperm, int32_t *perm_out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t old = (int32_t)perm[r];
        iperm[old] = (int32_t)r;
        perm_out[r] = old;
    }
}

// level_ptr from the sorted level keys (levels are 0..L-1 without gaps)
__global__ void k_level_bounds(const uint32_t *sorted_levels, int64_t n, int32_t *level_ptr, int32_t L) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t l = (int32_t)sorted_levels[r];
        const int32_t prev = r == 0 ? -1 : (int32_t)sorted_levels[r - 1];
        for (int32_t q = prev + 1; q <= l; ++q) level_ptr[q] = (int32_t)r;
        if (r == n - 1) level_ptr[L] = (int32_t)n;
    }
}

static int grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

Levels *build_levels(const mpk_csr *A, int32_t root, cudaStream_t s, const std::vector<int32_t> *roots) {
    validate_csr(A, s);
    const int32_t n = A->n;
    if (roots) {  // level 0 is the whole root set: a BFS distance from the set
        if (n > 0 && roots->empty()) fail(MPK_ERR_INVALID, "empty root set");
        for (size_t i = 0; i < roots->size(); ++i)
            if ((*roots)[i] < 0 || (*roots)[i] >= n || (i > 0 && (*roots)[i] <= (*roots)[i - 1]))
                fail(MPK_ERR_INVALID, "roots must be ascending, distinct and in [0, %d)", n);
    } else if (n > 0 && (root < 0 || root >= n)) {
        fail(MPK_ERR_INVALID, "root %d outside [0, %d)", root, n);
    }
    Levels *L = new Levels();
    try {
        L->n = n;
        L->level_ptr = L->arena.alloc_n<int32_t>((int64_t)n + 1);
        L->perm = L->arena.alloc_n<int32_t>(n);
        L->iperm = L->arena.alloc_n<int32_t>(n);
        L->level_of = L->arena.alloc_n<int32_t>(n);
        if (n == 0) {
            MPK_CUDA(cudaMemsetAsync(L->level_ptr, 0, sizeof(int32_t), s));
            MPK_CUDA(cudaStreamSynchronize(s));
            L->h_level_ptr = {0};
            return L;
        }
        // pattern of A^T without the diagonal, only when A is not declared symmetric
        Tmp<int32_t> tp(A->is_symmetric ? 0 : (int64_t)n + 1, s);
        Tmp<int32_t> tci(A->is_symmetric ? 0 : (int64_t)A->nnz, s);
        if (!A->is_symmetric) {
            Tmp<int32_t> cnt((int64_t)n + 1, s);
            MPK_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * ((size_t)n + 1), s));
            k_tcount<<<grid_n(n), 256, 0, s>>>(n, A->row_ptr, A->col, cnt.p);
            MPK_LAUNCHED();
            exclusive_scan(cnt.p, tp.p, n, s);
            MPK_CUDA(cudaMemcpyAsync(cnt.p, tp.p, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            k_tfill<<<grid_n(n), 256, 0, s>>>(n, A->row_ptr, A->col, cnt.p, tci.p);
            MPK_LAUNCHED();
            MPK_CUDA(cudaStreamSynchronize(s));
        }
        // level-synchronous BFS; queue holds the levels back to back
        Tmp<int32_t> queue(n, s);
        MPK_CUDA(cudaMemsetAsync(L->level_of, 0xff, sizeof(int32_t) * (size_t)n, s));
        int64_t head = 0, tail = 1;
        if (roots) {
            const int32_t nr = (int32_t)roots->size();
            Tmp<int32_t> d_roots(nr, s);
            MPK_CUDA(cudaMemcpyAsync(d_roots.p, roots->data(), sizeof(int32_t) * (size_t)nr, cudaMemcpyHostToDevice, s));
            k_set_roots<<<grid_n(nr), 256, 0, s>>>(L->level_of, queue.p, d_roots.p, nr);
            MPK_LAUNCHED();
            MPK_CUDA(cudaStreamSynchronize(s));  // the host root list and d_roots go out of scope
            tail = nr;
        } else {
            k_set_root<<<1, 1, 0, s>>>(L->level_of, queue.p, root, 0);
            MPK_LAUNCHED();
        }
        // the levels, in one cooperative launch (every block resident)
        Tmp<BfsState> st(1, s);
        MPK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(BfsState), s));
        int per_sm = 0;
        MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_all, 256, 0));
        if (per_sm < 1) fail(MPK_ERR_CUDA, "the BFS kernel does not fit an SM");
        // two blocks per SM: enough threads for the widest frontiers, few arrivals per barrier
        const int grid = std::min(per_sm, 2) * device_sms();
        const int32_t *rpp = A->row_ptr, *cip = A->col;
        const int32_t *tpp = A->is_symmetric ? nullptr : tp.p;
        const int32_t *tcip = tci.p;
        int32_t *lvl = L->level_of, *qp = queue.p;
        int32_t nn = n, h0 = (int32_t)head, t0 = (int32_t)tail;
        BfsState *stp = st.p;
        int64_t limit = kBfsWaitNs;
        void *args[] = {(void *)&rpp, (void *)&cip, (void *)&tpp, (void *)&tcip, (void *)&lvl, (void *)&qp,
                        (void *)&nn, (void *)&h0, (void *)&t0, (void *)&stp, (void *)&limit};
        MPK_CUDA(cudaLaunchCooperativeKernel((const void *)k_bfs_all, dim3(grid), dim3(256), args, 0, s));
        MPK_LAUNCHED();
        BfsState hs;
        MPK_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(BfsState), cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        if (hs.err == 1) fail(MPK_ERR_TIMEOUT, "BFS: a grid barrier wait expired");
        if (hs.err != 0) fail(MPK_ERR_CUDA, "BFS lost track of unvisited vertices");
        const int32_t lev = hs.levels - 1;
        const int32_t nl = lev + 1;
        L->num_levels = nl;
        // permutation: stable sort of (level, id) pairs with ids ascending as input order
        Tmp<uint32_t> k0(n, s), v0(n, s), k1(n, s), v1(n, s);
        MPK_CUDA(cudaMemcpyAsync(k0.p, L->level_of, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        iota_i32(reinterpret_cast<int32_t *>(v0.p), n, s);
        int bits = 0;
        while (bits < 32 && ((int64_t)1 << bits) < nl) ++bits;
        uint32_t *ks = nullptr, *vs = nullptr;
        radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, n, bits, s, &ks, &vs);
        k_inverse<<<grid_n(n), 256, 0, s>>>(vs, L->iperm, L->perm, n);
        MPK_LAUNCHED();
        k_level_bounds<<<grid_n(n), 256, 0, s>>>(ks, n, L->level_ptr, nl);
        MPK_LAUNCHED();
        L->h_level_ptr.resize((size_t)nl + 1);
        MPK_CUDA(cudaMemcpyAsync(L->h_level_ptr.data(), L->level_ptr, sizeof(int32_t) * ((size_t)nl + 1),
                                 cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        L->arena.release();
        delete L;
        throw;
    }
    return L;
}

}  // namespace mpk
