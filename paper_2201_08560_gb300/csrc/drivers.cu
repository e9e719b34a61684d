// Graph algorithms over B2SR (Sec. V): BFS (Boolean semiring, visited set as a
// complemented output mask), multi-source BFS (64 frontiers per machine word),
// SSSP (min-plus relaxation rounds), PageRank (plus-times with the
// column-stochastic matrix), connected components (FastSV hooking and
// shortcutting around the min step) and triangle counting (masked SpGEMM on
// the lower triangle).  Each driver loops on the host, one SpMV plus one
// element-wise kernel per iteration, with an iteration cap.
#include <algorithm>
#include <climits>
#include <vector>

#include "b2sr_internal.cuh"

namespace b2sr {
b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s);
b2sr_status spmm64_dispatch(b2sr_matrix* h, const uint64_t* X, uint64_t* Y, const uint64_t* M, int comp,
                            cudaStream_t s);
b2sr_status masked_count(const b2sr_matrix* A, const b2sr_matrix* B, const b2sr_matrix* M, int64_t* count,
                         cudaStream_t s);

static int grid_for(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)sm_count() * 8));
}

// Pinned host word for loop-exit flags.
struct HostFlag {
    int32_t* p = nullptr;
    HostFlag() { if (cudaMallocHost(&p, sizeof(int32_t)) != cudaSuccess) { cudaGetLastError(); p = nullptr; } }
    ~HostFlag() { if (p) cudaFreeHost(p); }
};

static b2sr_status read_flag(const int32_t* dev, HostFlag& hf, cudaStream_t s, int32_t* out) {
    if (!hf.p) return fail(B2SR_ERR_OOM, "pinned flag");
    B2SR_CUDA_TRY(cudaMemcpyAsync(hf.p, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    *out = *hf.p;
    return B2SR_OK;
}

// ---------------------------------------------------------------------------
// BFS
// ---------------------------------------------------------------------------
__global__ void bfs_init_kernel(int32_t* levels, int32_t n, int32_t src, uint32_t* frontier, uint32_t* visited,
                                int64_t words) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n || i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) levels[i] = (i == src) ? 0 : -1;
        if (i < words) {
            uint32_t w = (i == (src >> 5)) ? (1u << (src & 31)) : 0u;
            frontier[i] = w;
            visited[i] = w;
        }
    }
}

// visited |= next; levels[v] = level for every new vertex; count new vertices
__global__ void bfs_update_kernel(const uint32_t* __restrict__ next, uint32_t* __restrict__ visited,
                                  int32_t* __restrict__ levels, int64_t words, int32_t level, int32_t* any) {
    int found = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = next[w];
        if (!b) continue;
        found = 1;
        visited[w] |= b;
        while (b) {
            int c = __ffs(b) - 1;
            b &= b - 1;
            levels[w * 32 + c] = level;
        }
    }
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(any, 1);
}

b2sr_status bfs(b2sr_matrix* h, int32_t src, int32_t* levels, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    const int64_t words = ceil_div(n, 32);
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(3 * words * sizeof(uint32_t) + 16));
    uint32_t* f = buf.as<uint32_t>();
    uint32_t* nx = f + words;
    uint32_t* vis = nx + words;
    int32_t* any = reinterpret_cast<int32_t*>(vis + words);
    bfs_init_kernel<<<grid_for(std::max<int64_t>(n, words)), 256, 0, s>>>(levels, n, src, f, vis, words);
    B2SR_LAUNCH_CHECK("bfs_init_kernel");
    HostFlag hf;
    const int cap = max_iters > 0 ? max_iters : n;
    for (int level = 1; level <= cap + 1; ++level) {
        B2SR_TRY(spmv_dispatch(h, B2SR_BOOL_OR_AND, B2SR_VEC_BITS, f, B2SR_VEC_BITS, nx, vis, 1, nullptr, s));
        B2SR_CUDA_TRY(cudaMemsetAsync(any, 0, sizeof(int32_t), s));
        bfs_update_kernel<<<grid_for(words), 256, 0, s>>>(nx, vis, levels, words, level, any);
        B2SR_LAUNCH_CHECK("bfs_update_kernel");
        int32_t got = 0;
        B2SR_TRY(read_flag(any, hf, s, &got));
        if (!got) return B2SR_OK;
        if (level > cap) break;
        std::swap(f, nx);
    }
    return fail(B2SR_ERR_NOT_CONVERGED, "BFS exceeded max_iters levels");
}

// ---------------------------------------------------------------------------
// multi-source BFS, 64 frontiers per vertex
// ---------------------------------------------------------------------------
__global__ void msbfs_init_kernel(int32_t* levels, int32_t n, int nsrc, unsigned long long* X,
                                  unsigned long long* vis) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * nsrc || i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < (int64_t)n * nsrc) levels[i] = -1;
        if (i < n) { X[i] = 0ull; vis[i] = 0ull; }
    }
}

__global__ void msbfs_seed_kernel(const int32_t* srcs, int nsrc, int32_t n, int32_t* levels, unsigned long long* X,
                                  unsigned long long* vis) {
    int s = threadIdx.x;
    if (s < nsrc) {
        int32_t v = srcs[s];
        levels[(int64_t)s * n + v] = 0;
        atomicOr(X + v, 1ull << s);
        atomicOr(vis + v, 1ull << s);
    }
}

__global__ void msbfs_update_kernel(const unsigned long long* __restrict__ Y, unsigned long long* __restrict__ vis,
                                    int32_t* __restrict__ levels, int32_t n, int32_t level, int32_t* any) {
    int found = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long b = Y[v];
        if (!b) continue;
        found = 1;
        vis[v] |= b;
        while (b) {
            int s = __ffsll((long long)b) - 1;
            b &= b - 1;
            levels[(int64_t)s * n + v] = level;
        }
    }
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(any, 1);
}

b2sr_status bfs_multi(b2sr_matrix* h, const int32_t* srcs_host, int nsrc, int32_t* levels, int max_iters,
                      cudaStream_t s) {
    const int32_t n = h->n;
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(3 * (size_t)n * sizeof(uint64_t) + 64 * sizeof(int32_t) + 16));
    unsigned long long* X = buf.as<unsigned long long>();
    unsigned long long* Y = X + n;
    unsigned long long* vis = Y + n;
    int32_t* dsrc = reinterpret_cast<int32_t*>(vis + n);
    int32_t* any = dsrc + 64;
    B2SR_CUDA_TRY(cudaMemcpyAsync(dsrc, srcs_host, nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    msbfs_init_kernel<<<grid_for((int64_t)n * nsrc), 256, 0, s>>>(levels, n, nsrc, X, vis);
    B2SR_LAUNCH_CHECK("msbfs_init_kernel");
    msbfs_seed_kernel<<<1, 64, 0, s>>>(dsrc, nsrc, n, levels, X, vis);
    B2SR_LAUNCH_CHECK("msbfs_seed_kernel");
    HostFlag hf;
    const int cap = max_iters > 0 ? max_iters : n;
    for (int level = 1; level <= cap + 1; ++level) {
        B2SR_TRY(spmm64_dispatch(h, reinterpret_cast<uint64_t*>(X), reinterpret_cast<uint64_t*>(Y),
                                 reinterpret_cast<uint64_t*>(vis), 1, s));
        B2SR_CUDA_TRY(cudaMemsetAsync(any, 0, sizeof(int32_t), s));
        msbfs_update_kernel<<<grid_for(n), 256, 0, s>>>(Y, vis, levels, n, level, any);
        B2SR_LAUNCH_CHECK("msbfs_update_kernel");
        int32_t got = 0;
        B2SR_TRY(read_flag(any, hf, s, &got));
        if (!got) return B2SR_OK;
        if (level > cap) break;
        std::swap(X, Y);
    }
    return fail(B2SR_ERR_NOT_CONVERGED, "multi-source BFS exceeded max_iters levels");
}

// ---------------------------------------------------------------------------
// SSSP: y = min(d, A min.+ d) until no distance changes
// ---------------------------------------------------------------------------
__global__ void sssp_init_kernel(float* d, int32_t n, int32_t src) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (i == src) ? 0.0f : INFINITY;
}

__global__ void changed_kernel(const float* __restrict__ a, const float* __restrict__ b, int32_t n, int32_t* any) {
    int diff = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        diff |= (a[i] != b[i]);
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(any, 1);
}

b2sr_status sssp(b2sr_matrix* h, const float* w, int32_t src, float* dist, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    DevBuf buf(s);
    B2SR_TRY(buf.alloc((size_t)n * sizeof(float) + 16));
    float* tmp = buf.as<float>();
    int32_t* any = reinterpret_cast<int32_t*>(tmp + n);
    sssp_init_kernel<<<grid_for(n), 256, 0, s>>>(dist, n, src);
    B2SR_LAUNCH_CHECK("sssp_init_kernel");
    HostFlag hf;
    float* cur = dist;
    float* nxt = tmp;
    const int cap = max_iters > 0 ? max_iters : n;
    for (int it = 0; it <= cap; ++it) {
        B2SR_TRY(spmv_dispatch(h, B2SR_MIN_PLUS, B2SR_VEC_F32, cur, B2SR_VEC_F32, nxt, nullptr, 0, w, s));
        B2SR_CUDA_TRY(cudaMemsetAsync(any, 0, sizeof(int32_t), s));
        changed_kernel<<<grid_for(n), 256, 0, s>>>(cur, nxt, n, any);
        B2SR_LAUNCH_CHECK("changed_kernel");
        int32_t got = 0;
        B2SR_TRY(read_flag(any, hf, s, &got));
        std::swap(cur, nxt);
        if (!got) {
            if (cur != dist) B2SR_CUDA_TRY(cudaMemcpyAsync(dist, cur, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
            return B2SR_OK;
        }
    }
    if (cur != dist) B2SR_CUDA_TRY(cudaMemcpyAsync(dist, cur, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return fail(B2SR_ERR_NOT_CONVERGED, "SSSP exceeded max_iters rounds");
}

// ---------------------------------------------------------------------------
// PageRank
// ---------------------------------------------------------------------------
// x^0 = 1/n; c_j = x_j / outdeg_j (0 without out-edges)
__global__ void pr_init_kernel(float* x, float* c, const int32_t* __restrict__ outdeg, int32_t n) {
    const float x0 = 1.0f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = x0;
        int32_t d = outdeg[i];
        c[i] = d > 0 ? x0 / (float)d : 0.0f;
    }
}

// x_i = (1-d) t_i + d y_i; c_i = x_i / outdeg_i
__global__ void pr_step_kernel(const float* __restrict__ y, const float* __restrict__ tele,
                               const int32_t* __restrict__ outdeg, float damp, int32_t n, float* __restrict__ x,
                               float* __restrict__ c) {
    const float tu = 1.0f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float ti = tele ? tele[i] : tu;
        float xi = (1.0f - damp) * ti + damp * y[i];
        x[i] = xi;
        int32_t d = outdeg[i];
        c[i] = d > 0 ? xi / (float)d : 0.0f;
    }
}

b2sr_status pagerank(b2sr_matrix* h, float damp, int iters, const float* tele, float* pr, cudaStream_t s) {
    const int32_t n = h->n;
    if (n == 0) return B2SR_OK;
    B2SR_TRY(ensure_outdeg(h, s));
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(2 * (size_t)n * sizeof(float)));
    float* c = buf.as<float>();
    float* y = c + n;
    pr_init_kernel<<<grid_for(n), 256, 0, s>>>(pr, c, h->outdeg, n);
    B2SR_LAUNCH_CHECK("pr_init_kernel");
    for (int it = 0; it < iters; ++it) {
        B2SR_TRY(spmv_dispatch(h, B2SR_PLUS_TIMES, B2SR_VEC_F32, c, B2SR_VEC_F32, y, nullptr, 0, nullptr, s));
        pr_step_kernel<<<grid_for(n), 256, 0, s>>>(y, tele, h->outdeg, damp, n, pr, c);
        B2SR_LAUNCH_CHECK("pr_step_kernel");
    }
    return B2SR_OK;
}

// ---------------------------------------------------------------------------
// connected components: FastSV (Zhang, Azad, Hu; the linear-algebraic CC the
// paper follows in Sec. V), with the min step as a B2SR SpMV
// ---------------------------------------------------------------------------
__global__ void cc_init_kernel(int32_t* f, int32_t* gf, int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        f[i] = (int32_t)i;
        gf[i] = (int32_t)i;
    }
}

// stochastic hooking: f[f[i]] = min(f[f[i]], mngf[i])
__global__ void cc_hook_kernel(int32_t* f, const int32_t* __restrict__ mngf, int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t fi = f[i];
        int32_t m = mngf[i];
        if (m < fi) atomicMin(f + fi, m);
    }
}

// aggressive hooking and shortcutting: f[i] = min(f[i], mngf[i], gf[i])
__global__ void cc_short_kernel(int32_t* f, const int32_t* __restrict__ mngf, const int32_t* __restrict__ gf,
                                int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = min(f[i], min(mngf[i], gf[i]));
}

// gf' = f[f]; flag if any grandparent changed
__global__ void cc_grand_kernel(const int32_t* __restrict__ f, const int32_t* __restrict__ gf, int32_t* __restrict__ gfn,
                                int32_t n, int32_t* any) {
    int diff = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = f[f[i]];
        gfn[i] = g;
        diff |= (g != gf[i]);
    }
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(any, 1);
}

b2sr_status cc(b2sr_matrix* h, int32_t* labels, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    if (n == 0) return B2SR_OK;
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(3 * (size_t)n * sizeof(int32_t) + 16));
    int32_t* gf = buf.as<int32_t>();
    int32_t* gfn = gf + n;
    int32_t* mngf = gfn + n;
    int32_t* any = mngf + n;
    int32_t* f = labels;
    cc_init_kernel<<<grid_for(n), 256, 0, s>>>(f, gf, n);
    B2SR_LAUNCH_CHECK("cc_init_kernel");
    HostFlag hf;
    const int cap = max_iters > 0 ? max_iters : n;
    for (int it = 0; it <= cap; ++it) {
        B2SR_TRY(spmv_dispatch(h, B2SR_MIN_PLUS, B2SR_VEC_I32, gf, B2SR_VEC_I32, mngf, nullptr, 0, nullptr, s));
        cc_hook_kernel<<<grid_for(n), 256, 0, s>>>(f, mngf, n);
        B2SR_LAUNCH_CHECK("cc_hook_kernel");
        cc_short_kernel<<<grid_for(n), 256, 0, s>>>(f, mngf, gf, n);
        B2SR_LAUNCH_CHECK("cc_short_kernel");
        B2SR_CUDA_TRY(cudaMemsetAsync(any, 0, sizeof(int32_t), s));
        cc_grand_kernel<<<grid_for(n), 256, 0, s>>>(f, gf, gfn, n, any);
        B2SR_LAUNCH_CHECK("cc_grand_kernel");
        int32_t got = 0;
        B2SR_TRY(read_flag(any, hf, s, &got));
        std::swap(gf, gfn);
        if (!got) return B2SR_OK;
    }
    return fail(B2SR_ERR_NOT_CONVERGED, "CC exceeded max_iters rounds");
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_bfs(b2sr_handle h, int32_t src, int32_t* levels, int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (src < 0 || src >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (!levels) return fail(B2SR_ERR_INVALID_ARG, "levels is NULL");
    return bfs(h, src, levels, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_bfs_multi(b2sr_handle h, const int32_t* srcs_host, int nsrc, int32_t* levels,
                                      int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (nsrc < 1 || nsrc > 64) return fail(B2SR_ERR_INVALID_ARG, "nsrc must be in [1, 64]");
    if (!srcs_host || !levels) return fail(B2SR_ERR_INVALID_ARG, "null pointer");
    for (int i = 0; i < nsrc; ++i)
        if (srcs_host[i] < 0 || srcs_host[i] >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    return bfs_multi(h, srcs_host, nsrc, levels, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_sssp(b2sr_handle h, const float* weights, int32_t src, float* dist, int max_iters,
                                 void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (src < 0 || src >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (!dist) return fail(B2SR_ERR_INVALID_ARG, "dist is NULL");
    return sssp(h, weights, src, dist, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_pagerank(b2sr_handle h, float d, int iters, const float* teleport, float* pr,
                                     void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (!pr && h->n > 0) return fail(B2SR_ERR_INVALID_ARG, "pr is NULL");
    if (iters < 0 || !(d >= 0.0f && d <= 1.0f)) return fail(B2SR_ERR_INVALID_ARG, "bad iters or damping");
    return pagerank(h, d, iters, teleport, pr, to_stream(stream));
}

extern "C" b2sr_status b2sr_cc(b2sr_handle h, int32_t* labels, int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (!labels && h->n > 0) return fail(B2SR_ERR_INVALID_ARG, "labels is NULL");
    return cc(h, labels, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_tc(b2sr_handle h, int64_t* count, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (!count) return fail(B2SR_ERR_INVALID_ARG, "count is NULL");
    b2sr_handle L = nullptr;
    B2SR_TRY(b2sr_lower(h, stream, &L));
    b2sr_status st = masked_count(L, L, L, count, to_stream(stream));
    b2sr_destroy(L);
    return st;
}
