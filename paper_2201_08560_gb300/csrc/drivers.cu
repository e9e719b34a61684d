// Graph algorithms over B2SR (Sec. V): BFS (Boolean semiring, visited set as a
// complemented output mask), BFS from a set of sources (which also runs many
// graphs packed block-diagonally in one arena), multi-source BFS (64 frontiers
// per machine word), SSSP (min-plus relaxation rounds), PageRank (plus-times
// with the column-stochastic matrix), connected components (FastSV hooking
// and shortcutting around the min step) and triangle counting (masked SpGEMM
// on the lower triangle).
//
// Level-synchronous loops are captured once as a CUDA graph of several rounds;
// each round's kernels are gated on a device flag that the round's update
// kernel clears when nothing changes, and the graph is replayed until the host
// reads the flag as 0.  One host synchronisation covers several rounds.
#include <algorithm>
#include <climits>
#include <vector>

#include "b2sr_internal.cuh"
#include "captured.cuh"

namespace b2sr {
b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s,
                          const int32_t* gate);
b2sr_status spmm64_dispatch(b2sr_matrix* h, const uint64_t* X, uint64_t* Y, const uint64_t* M, int comp,
                            cudaStream_t s, const int32_t* gate);
b2sr_status masked_count(const b2sr_matrix* A, const b2sr_matrix* B, const b2sr_matrix* M, int64_t* count,
                         cudaStream_t s, int64_t* pairs);

// active <- found (only while active); level counter advances with it
__global__ void advance_kernel(int32_t* active, const int32_t* found, int32_t* level) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *active) {
        *active = *found;
        *level += 1;
    }
}

// ---------------------------------------------------------------------------
// BFS from a set of sources (all at level 0)
// ---------------------------------------------------------------------------
__global__ void bfs_init_kernel(int32_t* levels, int32_t n, uint32_t* frontier, uint32_t* visited, int64_t words) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n || i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) levels[i] = -1;
        if (i < words) { frontier[i] = 0u; visited[i] = 0u; }
    }
}

__global__ void bfs_seed_kernel(const int32_t* srcs, int nsrc, int32_t* levels, uint32_t* frontier,
                                uint32_t* visited) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x) {
        const int32_t v = srcs[i];
        levels[v] = 0;
        atomicOr(frontier + (v >> 5), 1u << (v & 31));
        atomicOr(visited + (v >> 5), 1u << (v & 31));
    }
}

// visited |= next; levels[v] = level+1 for every new vertex; found if any
__global__ void bfs_update_kernel(const uint32_t* __restrict__ next, uint32_t* __restrict__ visited,
                                  int32_t* __restrict__ levels, int64_t words, const int32_t* level,
                                  const int32_t* gate, int32_t* found) {
    if (gate_closed(gate)) return;
    const int32_t lv = *level + 1;
    int any = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = next[w];
        if (!b) continue;
        any = 1;
        visited[w] |= b;
        while (b) {
            int c = __ffs(b) - 1;
            b &= b - 1;
            levels[w * 32 + c] = lv;
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(found, 1);
}

b2sr_status bfs_sources(b2sr_matrix* h, const int32_t* srcs_host, int nsrc, int32_t* levels, int max_iters,
                        cudaStream_t s) {
    const int32_t n = h->n;
    const int64_t words = ceil_div(n, 32);
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(3 * words * sizeof(uint32_t) + (size_t)(nsrc + 8) * sizeof(int32_t)));
    uint32_t* fa = buf.as<uint32_t>();
    uint32_t* fb = fa + words;
    uint32_t* vis = fb + words;
    int32_t* flags = reinterpret_cast<int32_t*>(vis + words);  // active, found, level
    int32_t* dsrc = flags + 8;
    B2SR_CUDA_TRY(cudaMemcpyAsync(dsrc, srcs_host, nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    bfs_init_kernel<<<grid_for(std::max<int64_t>(n, words)), 256, 0, s>>>(levels, n, fa, vis, words);
    B2SR_LAUNCH_CHECK("bfs_init_kernel");
    bfs_seed_kernel<<<(unsigned)ceil_div(nsrc, 256), 256, 0, s>>>(dsrc, nsrc, levels, fa, vis);
    B2SR_LAUNCH_CHECK("bfs_seed_kernel");
    const int32_t init[3] = {1, 0, 0};
    B2SR_CUDA_TRY(cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s));
    int32_t* active = flags;
    int32_t* found = flags + 1;
    int32_t* level = flags + 2;
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n + 1;
    int64_t rounds = 0;
    return run_captured(s, 4, cap + 1, active,
                        [&](cudaStream_t cs, int r) -> b2sr_status {
                            uint32_t* f = (r & 1) ? fb : fa;
                            uint32_t* nx = (r & 1) ? fa : fb;
                            B2SR_TRY(spmv_dispatch(h, B2SR_BOOL_OR_AND, B2SR_VEC_BITS, f, B2SR_VEC_BITS, nx, vis, 1,
                                                   nullptr, cs, active));
                            B2SR_CUDA_TRY(cudaMemsetAsync(found, 0, sizeof(int32_t), cs));
                            bfs_update_kernel<<<grid_for(words), 256, 0, cs>>>(nx, vis, levels, words, level, active,
                                                                               found);
                            B2SR_LAUNCH_CHECK("bfs_update_kernel");
                            advance_kernel<<<1, 32, 0, cs>>>(active, found, level);
                            B2SR_LAUNCH_CHECK("advance_kernel");
                            return B2SR_OK;
                        },
                        &rounds);
}

// ---------------------------------------------------------------------------
// multi-source BFS, 64 frontiers per vertex
// ---------------------------------------------------------------------------
// The lane word: 64 frontiers (uint64) or, for at most 32 sources, 32 (uint32:
// half the bytes per gather, and the SpMV takes the tile_dim-4 kernel).
__device__ __forceinline__ int lowest_lane(unsigned long long b) { return __ffsll((long long)b) - 1; }
__device__ __forceinline__ int lowest_lane(uint32_t b) { return __ffs(b) - 1; }

template <class W>
__global__ void msbfs_init_kernel(int32_t* levels, int32_t n, int nsrc, W* X, W* vis) {
    constexpr int BITS = 8 * (int)sizeof(W);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * nsrc || i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < (int64_t)n * nsrc) levels[i] = -1;
        // unused lanes count as visited, so a vertex every source has reached is
        // all ones in the mask and the SpMM can skip its rows
        if (i < n) { X[i] = (W)0; vis[i] = nsrc < BITS ? (W)~(((W)1 << nsrc) - (W)1) : (W)0; }
    }
}

template <class W>
__global__ void msbfs_seed_kernel(const int32_t* srcs, int nsrc, int32_t n, int32_t* levels, W* X, W* vis) {
    int s = threadIdx.x;
    if (s < nsrc) {
        int32_t v = srcs[s];
        levels[(int64_t)s * n + v] = 0;
        atomicOr(X + v, (W)1 << s);
        atomicOr(vis + v, (W)1 << s);
    }
}

template <class W>
__global__ void msbfs_update_kernel(const W* __restrict__ Y, W* __restrict__ vis, int32_t* __restrict__ levels,
                                    int32_t n, const int32_t* level, const int32_t* gate, int32_t* found) {
    if (gate_closed(gate)) return;
    const int32_t lv = *level + 1;
    int any = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        W b = Y[v];
        if (!b) continue;
        any = 1;
        vis[v] |= b;
        while (b) {
            int s = lowest_lane(b);
            b &= b - 1;
            levels[(int64_t)s * n + v] = lv;
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(found, 1);
}

b2sr_status spmm32_dispatch(b2sr_matrix* h, const uint32_t* X, uint32_t* Y, const uint32_t* M, int comp,
                            cudaStream_t s, const int32_t* gate);

static b2sr_status spmm_lanes(b2sr_matrix* h, const unsigned long long* X, unsigned long long* Y,
                              const unsigned long long* M, cudaStream_t s, const int32_t* gate) {
    return spmm64_dispatch(h, reinterpret_cast<const uint64_t*>(X), reinterpret_cast<uint64_t*>(Y),
                           reinterpret_cast<const uint64_t*>(M), 1, s, gate);
}
static b2sr_status spmm_lanes(b2sr_matrix* h, const uint32_t* X, uint32_t* Y, const uint32_t* M, cudaStream_t s,
                              const int32_t* gate) {
    return spmm32_dispatch(h, X, Y, M, 1, s, gate);
}

template <class W>
static b2sr_status bfs_multi_lanes(b2sr_matrix* h, const int32_t* srcs_host, int nsrc, int32_t* levels,
                                   int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(3 * round_up((size_t)n * sizeof(W), 256) + 72 * sizeof(int32_t)));
    W* X = buf.as<W>();
    W* Yb = reinterpret_cast<W*>(buf.as<char>() + round_up((size_t)n * sizeof(W), 256));
    W* vis = reinterpret_cast<W*>(buf.as<char>() + 2 * round_up((size_t)n * sizeof(W), 256));
    int32_t* dsrc = reinterpret_cast<int32_t*>(buf.as<char>() + 3 * round_up((size_t)n * sizeof(W), 256));
    int32_t* flags = dsrc + 64;  // active, found, level
    B2SR_CUDA_TRY(cudaMemcpyAsync(dsrc, srcs_host, nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    msbfs_init_kernel<W><<<grid_for((int64_t)n * nsrc), 256, 0, s>>>(levels, n, nsrc, X, vis);
    B2SR_LAUNCH_CHECK("msbfs_init_kernel");
    msbfs_seed_kernel<W><<<1, 64, 0, s>>>(dsrc, nsrc, n, levels, X, vis);
    B2SR_LAUNCH_CHECK("msbfs_seed_kernel");
    const int32_t init[3] = {1, 0, 0};
    B2SR_CUDA_TRY(cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s));
    int32_t* active = flags;
    int32_t* found = flags + 1;
    int32_t* level = flags + 2;
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n + 1;
    int64_t rounds = 0;
    return run_captured(s, 4, cap + 1, active,
                        [&](cudaStream_t cs, int r) -> b2sr_status {
                            W* cur = (r & 1) ? Yb : X;
                            W* nxt = (r & 1) ? X : Yb;
                            B2SR_TRY(spmm_lanes(h, cur, nxt, vis, cs, active));
                            B2SR_CUDA_TRY(cudaMemsetAsync(found, 0, sizeof(int32_t), cs));
                            msbfs_update_kernel<W><<<grid_for(n), 256, 0, cs>>>(nxt, vis, levels, n, level, active,
                                                                               found);
                            B2SR_LAUNCH_CHECK("msbfs_update_kernel");
                            advance_kernel<<<1, 32, 0, cs>>>(active, found, level);
                            B2SR_LAUNCH_CHECK("advance_kernel");
                            return B2SR_OK;
                        },
                        &rounds);
}

b2sr_status bfs_multi(b2sr_matrix* h, const int32_t* srcs_host, int nsrc, int32_t* levels, int max_iters,
                      cudaStream_t s) {
    if (nsrc <= 32) return bfs_multi_lanes<uint32_t>(h, srcs_host, nsrc, levels, max_iters, s);
    return bfs_multi_lanes<unsigned long long>(h, srcs_host, nsrc, levels, max_iters, s);
}

// ---------------------------------------------------------------------------
// SSSP: d <- min(d, A min.+ d) until no distance changes
// ---------------------------------------------------------------------------
__global__ void sssp_init_kernel(float* d, int32_t n, int32_t src) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (i == src) ? 0.0f : INFINITY;
}

// found if a distance changed; the round's result becomes the current vector
__global__ void sssp_update_kernel(const float* __restrict__ nxt, float* __restrict__ cur, int32_t n,
                                   const int32_t* gate, int32_t* found) {
    if (gate_closed(gate)) return;
    int diff = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = nxt[i];
        if (v != cur[i]) { diff = 1; cur[i] = v; }
    }
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(found, 1);
}

b2sr_status sssp(b2sr_matrix* h, const float* w, int32_t src, float* dist, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    if (w) B2SR_TRY(ensure_voff(h, s));  // built before capture: capture must not allocate for the handle
    DevBuf buf(s);
    B2SR_TRY(buf.alloc((size_t)n * sizeof(float) + 16));
    float* tmp = buf.as<float>();
    int32_t* flags = reinterpret_cast<int32_t*>(tmp + n);
    sssp_init_kernel<<<grid_for(n), 256, 0, s>>>(dist, n, src);
    B2SR_LAUNCH_CHECK("sssp_init_kernel");
    const int32_t init[3] = {1, 0, 0};
    B2SR_CUDA_TRY(cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s));
    int32_t* active = flags;
    int32_t* found = flags + 1;
    int32_t* level = flags + 2;
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n + 1;
    int64_t rounds = 0;
    return run_captured(s, 16, cap + 1, active,
                        [&](cudaStream_t cs, int) -> b2sr_status {
                            B2SR_TRY(spmv_dispatch(h, B2SR_MIN_PLUS, B2SR_VEC_F32, dist, B2SR_VEC_F32, tmp, nullptr, 0, w,
                                                   cs, active));
                            B2SR_CUDA_TRY(cudaMemsetAsync(found, 0, sizeof(int32_t), cs));
                            sssp_update_kernel<<<grid_for(n), 256, 0, cs>>>(tmp, dist, n, active, found);
                            B2SR_LAUNCH_CHECK("sssp_update_kernel");
                            advance_kernel<<<1, 32, 0, cs>>>(active, found, level);
                            B2SR_LAUNCH_CHECK("advance_kernel");
                            return B2SR_OK;
                        },
                        &rounds);
}

// ---------------------------------------------------------------------------
// PageRank
// ---------------------------------------------------------------------------
// x^0 = 1/n; c_j = x_j / outdeg_j (0 without out-edges).  The rounding of
// every operation is spelled out (no contraction left to the compiler), so the
// batched PageRank of the query server reproduces these values bit for bit.
__global__ void pr_init_kernel(float* x, float* c, const int32_t* __restrict__ outdeg, int32_t n) {
    const float x0 = __fdiv_rn(1.0f, (float)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = x0;
        int32_t d = outdeg[i];
        c[i] = d > 0 ? __fdiv_rn(x0, (float)d) : 0.0f;
    }
}

// x_i = (1-d) t_i + d y_i; c_i = x_i / outdeg_i
__global__ void pr_step_kernel(const float* __restrict__ y, const float* __restrict__ tele,
                               const int32_t* __restrict__ outdeg, float damp, int32_t n, float* __restrict__ x,
                               float* __restrict__ c) {
    const float tu = __fdiv_rn(1.0f, (float)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float ti = tele ? tele[i] : tu;
        float xi = __fmaf_rn(damp, y[i], __fmul_rn(1.0f - damp, ti));
        x[i] = xi;
        int32_t d = outdeg[i];
        c[i] = d > 0 ? __fdiv_rn(xi, (float)d) : 0.0f;
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
        B2SR_TRY(spmv_dispatch(h, B2SR_PLUS_TIMES, B2SR_VEC_F32, c, B2SR_VEC_F32, y, nullptr, 0, nullptr, s, nullptr));
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
    const size_t vb = round_up((size_t)n * sizeof(int32_t), 256);  // each vector 256-byte aligned
    B2SR_TRY(buf.alloc(3 * vb + 256));
    int32_t* gf = buf.as<int32_t>();
    int32_t* gfn = reinterpret_cast<int32_t*>(buf.as<char>() + vb);
    int32_t* mngf = reinterpret_cast<int32_t*>(buf.as<char>() + 2 * vb);
    int32_t* any = reinterpret_cast<int32_t*>(buf.as<char>() + 3 * vb);
    int32_t* f = labels;
    cc_init_kernel<<<grid_for(n), 256, 0, s>>>(f, gf, n);
    B2SR_LAUNCH_CHECK("cc_init_kernel");
    HostFlag hf;
    const int cap = max_iters > 0 ? max_iters : n;
    for (int it = 0; it <= cap; ++it) {
        B2SR_TRY(spmv_dispatch(h, B2SR_MIN_PLUS, B2SR_VEC_I32, gf, B2SR_VEC_I32, mngf, nullptr, 0, nullptr, s, nullptr));
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

// ---------------------------------------------------------------------------
// many graphs in one block-diagonal arena
// ---------------------------------------------------------------------------
// rowptr of graph g placed at rows [base, base + ng), padding rows after it
// empty; its column ids shifted by base.
__global__ void arena_rows_kernel(const int32_t* __restrict__ rp, int32_t ng, int32_t base, int32_t npad,
                                  int64_t eoff, int32_t* __restrict__ out_rp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad;
         i += (int64_t)gridDim.x * blockDim.x)
        out_rp[base + i] = (int32_t)(eoff + rp[i < ng ? i : ng]);
}

__global__ void arena_cols_kernel(const int32_t* __restrict__ ci, int64_t nnz, int32_t base,
                                  int32_t* __restrict__ out_ci) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        out_ci[e] = ci[e] + base;
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_bfs(b2sr_handle h, int32_t src, int32_t* levels, int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (src < 0 || src >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (!levels) return fail(B2SR_ERR_INVALID_ARG, "levels is NULL");
    return bfs_sources(h, &src, 1, levels, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_bfs_sources(b2sr_handle h, const int32_t* srcs_host, int nsrc, int32_t* levels,
                                        int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (nsrc < 1 || !srcs_host || !levels) return fail(B2SR_ERR_INVALID_ARG, "need at least one source and levels");
    for (int i = 0; i < nsrc; ++i)
        if (srcs_host[i] < 0 || srcs_host[i] >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    return bfs_sources(h, srcs_host, nsrc, levels, max_iters, to_stream(stream));
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
    b2sr_status st = masked_count(L, L, L, count, to_stream(stream), nullptr);
    b2sr_destroy(L);
    return st;
}

extern "C" b2sr_status b2sr_from_csr_batch(int ngraphs, const int32_t* n_host, const int32_t* const* rowptrs,
                                           const int32_t* const* colinds, const int64_t* nnz_host, int tile_dim,
                                           void* stream, b2sr_handle* out, int64_t* base_host) {
    clear_error();
    if (!out) return fail(B2SR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (ngraphs < 1 || !n_host || !rowptrs || !colinds || !nnz_host || !base_host)
        return fail(B2SR_ERR_INVALID_ARG, "null pointer or no graphs");
    if (!valid_tile(tile_dim)) return fail(B2SR_ERR_UNSUPPORTED_TILE, "tile_dim must be 4, 8, 16 or 32");
    cudaStream_t s = to_stream(stream);
    int64_t N = 0, NNZ = 0;
    for (int g = 0; g < ngraphs; ++g) {
        if (n_host[g] < 0 || nnz_host[g] < 0 || !rowptrs[g] || (nnz_host[g] > 0 && !colinds[g]))
            return fail(B2SR_ERR_INVALID_ARG, "bad graph " + std::to_string(g));
        base_host[g] = N;
        N += round_up(n_host[g], 32);
        NNZ += nnz_host[g];
    }
    base_host[ngraphs] = N;
    if (N >= (int64_t(1) << 31) || NNZ >= (int64_t(1) << 31)) return fail(B2SR_ERR_INVALID_ARG, "arena too large");
    // every graph's own CSR is checked before it is shifted into the arena: a
    // column outside [0, n_g) would otherwise land in a neighbouring graph
    {
        DevBuf bad(s);
        B2SR_TRY(bad.alloc((size_t)ngraphs * sizeof(int)));
        B2SR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, (size_t)ngraphs * sizeof(int), s));
        for (int g = 0; g < ngraphs; ++g)
            B2SR_TRY(validate_csr_async(n_host[g], rowptrs[g], colinds[g], nnz_host[g], bad.as<int>() + g, s));
        std::vector<int> hbad((size_t)ngraphs);
        B2SR_CUDA_TRY(cudaMemcpyAsync(hbad.data(), bad.p, (size_t)ngraphs * sizeof(int), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        for (int g = 0; g < ngraphs; ++g)
            if (hbad[g]) return fail(B2SR_ERR_INVALID_ARG, "malformed CSR in graph " + std::to_string(g));
    }
    DevBuf rp(s), ci(s);
    B2SR_TRY(rp.alloc((N + 1) * sizeof(int32_t)));
    B2SR_TRY(ci.alloc(std::max<int64_t>(NNZ, 1) * sizeof(int32_t)));
    int64_t eoff = 0;
    for (int g = 0; g < ngraphs; ++g) {
        const int32_t npad = (int32_t)round_up(n_host[g], 32);
        if (npad > 0) {
            arena_rows_kernel<<<grid_for(npad), 256, 0, s>>>(rowptrs[g], n_host[g], (int32_t)base_host[g], npad, eoff,
                                                            rp.as<int32_t>());
            B2SR_LAUNCH_CHECK("arena_rows_kernel");
        }
        if (nnz_host[g] > 0) {
            arena_cols_kernel<<<grid_for(nnz_host[g]), 256, 0, s>>>(colinds[g], nnz_host[g], (int32_t)base_host[g],
                                                                   ci.as<int32_t>() + eoff);
            B2SR_LAUNCH_CHECK("arena_cols_kernel");
        }
        eoff += nnz_host[g];
    }
    const int32_t last = (int32_t)NNZ;
    B2SR_CUDA_TRY(cudaMemcpyAsync(rp.as<int32_t>() + N, &last, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));  // `last` lives on this stack frame
    return b2sr_from_csr((int32_t)N, rp.as<int32_t>(), ci.as<int32_t>(), NNZ, tile_dim, stream, out);
}
