// Planner: the permuted, sliced matrix copy, level groups, row chunks, chunk dependency
// ranges and the unit tables of the level-blocked schedule.
#include "mpk_internal.h"

#include <algorithm>

namespace mpk {

static int grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// length of new row r = length of old row perm[r]
__global__ void k_rowlen(int32_t n, const int32_t *rp, const int32_t *perm, int32_t *len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t old = perm ? perm[r] : (int32_t)r;
        len[r] = rp[old + 1] - rp[old];
    }
}

__global__ void k_gather_i32(const int32_t *src, const int32_t *idx, int32_t cnt, int32_t *dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += stride) dst[i] = src[idx[i]];
}

__global__ void k_chunk_of_row(const int32_t *chunk_row, int32_t nchunks, int32_t *chunk_of_row) {
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x)
        for (int32_t r = chunk_row[c] + threadIdx.x; r < chunk_row[c + 1]; r += blockDim.x) chunk_of_row[r] = c;
}

// 32 x (longest row) entries per slice; one thread per slice
__global__ void k_slice_size(const int32_t *chunk_row, const int32_t *chunk_slice, int32_t nchunks,
                             const int32_t *rowlen, int64_t *size) {
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int32_t r0 = chunk_row[c], r1 = chunk_row[c + 1], s0 = chunk_slice[c];
        for (int32_t sl = threadIdx.x; s0 + sl < chunk_slice[c + 1]; sl += blockDim.x) {
            int32_t w = 0;
            for (int32_t r = r0 + 32 * sl; r < r0 + 32 * sl + 32 && r < r1; ++r) w = max(w, rowlen[r]);
            size[s0 + sl] = 32 * (int64_t)w;
        }
    }
}

// Copies every row of P A P^T into its slice (entry j of lane l at slice_ptr + 32 j + l),
// relabelling columns through iperm, and folds the chunks each row reads into the
// dependency range of its chunk.  When A is not known to be symmetric, a chunk is also
// added to the ranges of the chunks it reads, so that ranges cover both directions.
__global__ void k_fill(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, const int32_t *perm,
                       const int32_t *iperm, const int32_t *chunk_row, const int32_t *chunk_slice,
                       const int32_t *chunk_of_row, const int64_t *slice_ptr, double *sval, int32_t *scol,
                       int2 *dep, int symmetric) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = chunk_of_row[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        const int32_t old = perm ? perm[r] : (int32_t)r;
        const int32_t e0 = rp[old], e1 = rp[old + 1];
        int32_t lo = c, hi = c;
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t nc = iperm ? iperm[ci[e]] : ci[e];
            const int64_t dst = base + 32 * (int64_t)(e - e0);
            sval[dst] = va[e];
            scol[dst] = nc;
            const int32_t cc = chunk_of_row[nc];
            lo = min(lo, cc);
            hi = max(hi, cc);
            if (!symmetric) {
                if (dep[cc].x > c) atomicMin(&dep[cc].x, c);
                if (dep[cc].y < c) atomicMax(&dep[cc].y, c);
            }
        }
        if (dep[c].x > lo) atomicMin(&dep[c].x, lo);
        if (dep[c].y < hi) atomicMax(&dep[c].y, hi);
    }
}

__global__ void k_dep_init(int2 *dep, int32_t nchunks) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x)
        dep[c] = make_int2(c, c);
}

// sliced copy -> CSR (for inspection and tests)
__global__ void k_export(int32_t n, const int32_t *rowlen, const int32_t *chunk_row, const int32_t *chunk_slice,
                         const int32_t *chunk_of_row, const int64_t *slice_ptr, const double *sval,
                         const int32_t *scol, const int32_t *rp, int32_t *ci, double *va) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t c = chunk_of_row[r];
        const int32_t local = (int32_t)r - chunk_row[c];
        const int64_t base = slice_ptr[chunk_slice[c] + (local >> 5)] + (local & 31);
        for (int32_t j = 0; j < rowlen[r]; ++j) {
            ci[rp[r] + j] = scol[base + 32 * (int64_t)j];
            va[rp[r] + j] = sval[base + 32 * (int64_t)j];
        }
    }
}

void export_csr(const Plan &P, int32_t *rp, int32_t *ci, double *va, cudaStream_t s) {
    if (!rp || (P.nnz > 0 && (!ci || !va))) fail(MPK_ERR_INVALID, "NULL output array");
    exclusive_scan(P.rowlen, rp, P.n, s);
    if (P.n == 0) return;
    Tmp<int32_t> cor(P.n);
    k_chunk_of_row<<<grid_n(P.num_chunks * 256), 256, 0, s>>>(P.chunk_row, P.num_chunks, cor.p);
    MPK_LAUNCHED();
    k_export<<<grid_n(P.n), 256, 0, s>>>(P.n, P.rowlen, P.chunk_row, P.chunk_slice, cor.p, P.slice_ptr, P.val,
                                         P.col, rp, ci, va);
    MPK_LAUNCHED();
    MPK_CUDA(cudaStreamSynchronize(s));
}

Plan *build_plan(const mpk_csr *A, const Levels *L, const mpk_plan_opts *o, cudaStream_t s) {
    if (!o) fail(MPK_ERR_INVALID, "options are NULL");
    validate_csr(A, s);
    if (o->p_max < 1 || o->p_max > kMaxP) fail(MPK_ERR_INVALID, "p_max must be in [1, %d]", kMaxP);
    if (!(o->nrhs == 1 || o->nrhs == 2 || o->nrhs == 4 || o->nrhs == 8))
        fail(MPK_ERR_UNSUPPORTED, "nrhs must be 1, 2, 4 or 8 (got %d)", o->nrhs);
    if (o->order != MPK_ORDER_ORIGINAL && o->order != MPK_ORDER_PLAN) fail(MPK_ERR_INVALID, "bad order");
    const int32_t chunk_rows = o->chunk_rows ? o->chunk_rows : 512;
    if (chunk_rows < 32 || chunk_rows > 8192 || chunk_rows % 32)
        fail(MPK_ERR_INVALID, "chunk_rows must be a multiple of 32 in [32, 8192]");
    if (o->cache_bytes < 0 || o->mem_budget < 0 || o->wait_limit_ns < 0) fail(MPK_ERR_INVALID, "negative option");
    if (L && L->n != A->n) fail(MPK_ERR_INVALID, "levels were built for n = %d, matrix has n = %d", L->n, A->n);

    const int32_t n = A->n, m = o->nrhs, pmax = o->p_max;
    Plan *P = new Plan();
    try {
        P->arena.budget = o->mem_budget;
        P->n = n;
        P->nnz = A->nnz;
        P->m = m;
        P->p_max = pmax;
        P->order = o->order;
        P->identity = (L == nullptr);
        P->chunk_rows = chunk_rows;
        P->cache_bytes = o->cache_bytes ? o->cache_bytes : device_l2_bytes() / 2;
        P->group_budget = P->cache_bytes / (pmax + 1);
        P->wait_ns = o->wait_limit_ns ? o->wait_limit_ns : 2000000000LL;
        P->num_levels = L ? L->num_levels : 0;

        // ---- permutation (plan-owned copies)
        if (!P->identity && n > 0) {
            P->perm = P->arena.alloc_n<int32_t>(n);
            P->iperm = P->arena.alloc_n<int32_t>(n);
            MPK_CUDA(cudaMemcpyAsync(P->perm, L->perm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            MPK_CUDA(cudaMemcpyAsync(P->iperm, L->iperm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        }
        P->rowlen = P->arena.alloc_n<int32_t>(n > 0 ? n : 1);
        if (n > 0) {
            k_rowlen<<<grid_n(n), 256, 0, s>>>(n, A->row_ptr, P->perm, P->rowlen);
            MPK_LAUNCHED();
        }

        // ---- groups: greedy rule over levels (host), identical to the written rule
        std::vector<int32_t> g_level, g_row;
        if (P->identity) {
            g_row = {0, n};
        } else if (n > 0) {
            const int32_t NL = L->num_levels;
            Tmp<int32_t> prp((int64_t)n + 1);
            exclusive_scan(P->rowlen, prp.p, n, s);
            Tmp<int32_t> lvl_nnz((int64_t)NL + 1);
            k_gather_i32<<<grid_n(NL + 1), 256, 0, s>>>(prp.p, L->level_ptr, NL + 1, lvl_nnz.p);
            MPK_LAUNCHED();
            std::vector<int32_t> h_nz((size_t)NL + 1);
            MPK_CUDA(cudaMemcpyAsync(h_nz.data(), lvl_nnz.p, sizeof(int32_t) * ((size_t)NL + 1),
                                     cudaMemcpyDeviceToHost, s));
            MPK_CUDA(cudaStreamSynchronize(s));
            const std::vector<int32_t> &lp = L->h_level_ptr;
            const int64_t B = P->group_budget;
            const int64_t vb = 8;  // value bytes (float64)
            int64_t cur = 0;
            g_level.push_back(0);
            for (int32_t l = 0; l < NL; ++l) {
                const int64_t rows = lp[l + 1] - lp[l];
                const int64_t nz = (int64_t)h_nz[l + 1] - h_nz[l];
                const int64_t b = (vb + 4) * nz + 4 * rows + 16 * (int64_t)m * rows;
                if (l > 0 && cur + b <= B) {
                    cur += b;
                } else {
                    if (l > 0) g_level.push_back(l);
                    cur = b;
                }
            }
            g_level.push_back(NL);
            for (int32_t gl : g_level) g_row.push_back(lp[gl]);
        } else {
            g_row = {0, 0};
        }
        const int32_t G = (int32_t)g_row.size() - 1;
        P->num_groups = G;

        // ---- chunks and slices (host)
        std::vector<int32_t> c_row, c_slice, g_chunk;
        c_row.push_back(0);
        c_slice.push_back(0);
        for (int32_t g = 0; g < G; ++g) {
            g_chunk.push_back((int32_t)c_row.size() - 1);
            for (int32_t r = g_row[g]; r < g_row[g + 1]; r += chunk_rows) {
                const int32_t e = std::min(r + chunk_rows, g_row[g + 1]);
                c_row.push_back(e);
                c_slice.push_back(c_slice.back() + (e - r + 31) / 32);
            }
        }
        g_chunk.push_back((int32_t)c_row.size() - 1);
        const int32_t NC = (int32_t)c_row.size() - 1;
        if (NC >= (1 << 26)) fail(MPK_ERR_TOO_LARGE, "too many chunks (%d)", NC);
        const int32_t NS = c_slice.back();
        P->num_chunks = NC;
        P->num_slices = NS;
        P->chunk_row = P->arena.alloc_n<int32_t>(NC + 1);
        P->chunk_slice = P->arena.alloc_n<int32_t>(NC + 1);
        P->group_row_ptr = P->arena.alloc_n<int32_t>(G + 1);
        MPK_CUDA(cudaMemcpyAsync(P->chunk_row, c_row.data(), sizeof(int32_t) * (NC + 1), cudaMemcpyHostToDevice, s));
        MPK_CUDA(cudaMemcpyAsync(P->chunk_slice, c_slice.data(), sizeof(int32_t) * (NC + 1), cudaMemcpyHostToDevice, s));
        MPK_CUDA(cudaMemcpyAsync(P->group_row_ptr, g_row.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s));
        if (!P->identity) {
            P->group_level_ptr = P->arena.alloc_n<int32_t>(G + 1);
            MPK_CUDA(cudaMemcpyAsync(P->group_level_ptr, g_level.data(), sizeof(int32_t) * (G + 1),
                                     cudaMemcpyHostToDevice, s));
        }

        // ---- sliced copy
        P->slice_ptr = P->arena.alloc_n<int64_t>((int64_t)NS + 1);
        Tmp<int32_t> cor(n);
        if (NC > 0) {
            k_slice_size<<<grid_n((int64_t)NC * 256), 256, 0, s>>>(P->chunk_row, P->chunk_slice, NC, P->rowlen,
                                                                   P->slice_ptr);
            MPK_LAUNCHED();
        }
        exclusive_scan(P->slice_ptr, P->slice_ptr, NS, s);
        MPK_CUDA(cudaMemcpyAsync(&P->padded, P->slice_ptr + NS, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        P->val = P->arena.alloc_n<double>(P->padded + 32);
        P->col = P->arena.alloc_n<int32_t>(P->padded + 32);
        MPK_CUDA(cudaMemsetAsync(P->val, 0, sizeof(double) * (size_t)(P->padded + 32), s));
        MPK_CUDA(cudaMemsetAsync(P->col, 0, sizeof(int32_t) * (size_t)(P->padded + 32), s));
        P->dep = P->arena.alloc_n<int2>(NC > 0 ? NC : 1);
        if (NC > 0) {
            k_dep_init<<<grid_n(NC), 256, 0, s>>>(P->dep, NC);
            MPK_LAUNCHED();
            k_chunk_of_row<<<grid_n((int64_t)NC * 256), 256, 0, s>>>(P->chunk_row, NC, cor.p);
            MPK_LAUNCHED();
            k_fill<<<grid_n(n), 256, 0, s>>>(n, A->row_ptr, A->col, static_cast<const double *>(A->val), P->perm,
                                             P->iperm, P->chunk_row, P->chunk_slice, cor.p, P->slice_ptr, P->val,
                                             P->col, P->dep, A->is_symmetric ? 1 : 0);
            MPK_LAUNCHED();
        }

        // ---- unit tables: Lp-diagram order (diagonal d = g + k ascending, then k ascending,
        //      then chunks in row order) for every p = 1..p_max; unit = chunk << 5 | k
        P->unit_off.assign((size_t)pmax + 2, 0);
        std::vector<int32_t> units;
        for (int32_t p = 1; p <= pmax; ++p) {
            P->unit_off[p] = (int64_t)units.size();
            for (int32_t d = 1; d <= G - 1 + p; ++d)
                for (int32_t k = std::max(1, d - G + 1); k <= std::min(p, d); ++k) {
                    const int32_t g = d - k;
                    for (int32_t c = g_chunk[g]; c < g_chunk[g + 1]; ++c) units.push_back((c << 5) | k);
                }
        }
        P->unit_off[pmax + 1] = (int64_t)units.size();
        P->units = P->arena.alloc_n<int32_t>((int64_t)units.size() + 1);
        if (!units.empty())
            MPK_CUDA(cudaMemcpyAsync(P->units, units.data(), sizeof(int32_t) * units.size(), cudaMemcpyHostToDevice, s));

        // ---- synchronisation state and vector workspace
        P->flags = P->arena.alloc_n<int32_t>((int64_t)(pmax + 1) * (NC > 0 ? NC : 1));
        MPK_CUDA(cudaMemsetAsync(P->flags, 0, sizeof(int32_t) * (size_t)(pmax + 1) * (NC > 0 ? NC : 1), s));
        P->ctl = P->arena.alloc_n<unsigned int>(4);
        MPK_CUDA(cudaMemsetAsync(P->ctl, 0, 4 * sizeof(unsigned int), s));
        P->work = P->arena.alloc_n<double>(4 * (int64_t)n * m + 1);
        MPK_CUDA(cudaStreamSynchronize(s));  // host vectors above must outlive their copies
    } catch (...) {
        P->arena.release();
        delete P;
        throw;
    }
    return P;
}

}  // namespace mpk
