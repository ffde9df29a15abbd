// Level builder: CSR validation, the pattern of A + A^T, level-synchronous BFS and the
// BFS permutation (Sec. 3, level definition, prose and Fig. 1).
#include "mpk_internal.h"

#include <climits>

namespace mpk {

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
    Tmp<int32_t> err(2);
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

// ----------------------------------------------------------------------------- BFS
// One frontier vertex per thread; neighbours from A's row and (if given) A^T's row.
// A vertex joins the next level by winning the CAS from -1 (levels are BFS distances,
// so the outcome does not depend on which thread wins).
__global__ void k_bfs_expand(const int32_t *front, int32_t fsize, const int32_t *rp, const int32_t *ci,
                             const int32_t *tp, const int32_t *tci, int32_t *level_of, int32_t next_level,
                             int32_t *next, int32_t *next_count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < fsize; t += stride) {
        const int32_t v = front[t];
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t u = ci[e];
            if (u != v && level_of[u] < 0 && atomicCAS(&level_of[u], -1, next_level) == -1)
                next[atomicAdd(next_count, 1)] = u;
        }
        if (tp)
            for (int32_t e = tp[v]; e < tp[v + 1]; ++e) {
                const int32_t u = tci[e];
                if (level_of[u] < 0 && atomicCAS(&level_of[u], -1, next_level) == -1)
                    next[atomicAdd(next_count, 1)] = u;
            }
    }
}

// smallest index >= from with level_of < 0, searched in [from, to)
__global__ void k_first_unvisited(const int32_t *level_of, int64_t from, int64_t to, int32_t *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to; i += stride)
        if (level_of[i] < 0) {
            atomicMin(out, (int32_t)i);
            return;
        }
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
        Tmp<int32_t> tp(A->is_symmetric ? 0 : (int64_t)n + 1);
        Tmp<int32_t> tci(A->is_symmetric ? 0 : (int64_t)A->nnz);
        if (!A->is_symmetric) {
            Tmp<int32_t> cnt((int64_t)n + 1);
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
        Tmp<int32_t> queue(n);
        Tmp<int32_t> dcount(2);
        int32_t *h = nullptr;
        MPK_CUDA(cudaMallocHost(&h, 2 * sizeof(int32_t)));
        struct HostFree {
            int32_t *p;
            ~HostFree() { cudaFreeHost(p); }
        } hf{h};
        MPK_CUDA(cudaMemsetAsync(L->level_of, 0xff, sizeof(int32_t) * (size_t)n, s));
        int64_t head = 0, tail = 1, cursor = 0;
        if (roots) {
            const int32_t nr = (int32_t)roots->size();
            Tmp<int32_t> d_roots(nr);
            MPK_CUDA(cudaMemcpyAsync(d_roots.p, roots->data(), sizeof(int32_t) * (size_t)nr, cudaMemcpyHostToDevice, s));
            k_set_roots<<<grid_n(nr), 256, 0, s>>>(L->level_of, queue.p, d_roots.p, nr);
            MPK_LAUNCHED();
            MPK_CUDA(cudaStreamSynchronize(s));  // the host root list and d_roots go out of scope
            tail = nr;
        } else {
            k_set_root<<<1, 1, 0, s>>>(L->level_of, queue.p, root, 0);
            MPK_LAUNCHED();
        }
        int32_t lev = 0;
        while (true) {
            if (tail > head) {
                MPK_CUDA(cudaMemsetAsync(dcount.p, 0, sizeof(int32_t), s));
                k_bfs_expand<<<grid_n(tail - head), 256, 0, s>>>(queue.p + head, (int32_t)(tail - head), A->row_ptr,
                                                                 A->col, A->is_symmetric ? nullptr : tp.p,
                                                                 tci.p, L->level_of, lev + 1, queue.p + tail,
                                                                 dcount.p);
                MPK_LAUNCHED();
                MPK_CUDA(cudaMemcpyAsync(h, dcount.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                MPK_CUDA(cudaStreamSynchronize(s));
                const int32_t found = h[0];
                head = tail;
                tail += found;
                if (found > 0) {
                    ++lev;
                    continue;
                }
            }
            if (tail >= n) break;
            // disconnected: the smallest untouched vertex opens level lev + 1
            int32_t v = INT_MAX;
            while (v == INT_MAX && cursor < n) {
                const int64_t window = (int64_t)1 << 20;
                const int64_t to = (cursor + window < (int64_t)n) ? cursor + window : (int64_t)n;
                fill_i32(dcount.p + 1, INT_MAX, 1, s);
                k_first_unvisited<<<grid_n(to - cursor), 256, 0, s>>>(L->level_of, cursor, to, dcount.p + 1);
                MPK_LAUNCHED();
                MPK_CUDA(cudaMemcpyAsync(h + 1, dcount.p + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                MPK_CUDA(cudaStreamSynchronize(s));
                v = h[1];
                if (v == INT_MAX) cursor = to;
            }
            if (v == INT_MAX) fail(MPK_ERR_CUDA, "BFS lost track of unvisited vertices");
            cursor = v;
            ++lev;
            k_set_root<<<1, 1, 0, s>>>(L->level_of, queue.p + tail, v, lev);
            MPK_LAUNCHED();
            head = tail;
            tail += 1;
        }
        const int32_t nl = lev + 1;
        L->num_levels = nl;
        // permutation: stable sort of (level, id) pairs with ids ascending as input order
        Tmp<uint32_t> k0(n), v0(n), k1(n), v1(n);
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
