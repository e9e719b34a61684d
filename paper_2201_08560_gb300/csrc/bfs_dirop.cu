// Direction-optimising BFS (Sec. V BFS, with the push/pull switching of
// Beamer, Asanovic and Patterson, "Direction-optimizing breadth-first
// search", SC 2012).
//
// A level either pulls -- the Boolean SpMV of Sec. V, next = A (x) frontier
// masked by ~visited, over every tile -- or pushes: the frontier's tile-rows
// of A^T are walked and every unvisited target of a frontier vertex is set in
// the next bitset with an atomic OR, so the level costs what the frontier
// touches.  Following Beamer et al., the search starts pushing, switches to
// pulling when the frontier's out-edges exceed the unexplored edges / alpha,
// and back to pushing when the frontier falls below n / beta.  The decision
// is taken on the device before every level, and both directions are gated
// on it, so the level loop stays a replayed CUDA graph with one host
// synchronisation per four levels.  Levels are the same in either direction
// (bit-exact with b2sr_bfs).
#include <algorithm>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "captured.cuh"
#include "tile_bits.cuh"

namespace b2sr {
b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s,
                          const int32_t* gate);

namespace {

constexpr int64_t kAlpha = 14;  // Beamer et al.'s switching constants
constexpr int64_t kBeta = 24;

// ctl layout (int64 words)
enum : int {
    C_ACTIVE = 0,  // 1 while the search goes on
    C_LEVEL,       // level of the current frontier
    C_DIR,         // 0 push, 1 pull
    C_PUSH,        // gate of the push kernel
    C_PULL,        // gate of the pull SpMV
    C_NCUR,        // frontier tile-rows in the current list
    C_NNEXT,       // tile-rows appended to the next list
    C_NF,          // frontier vertices
    C_MF,          // frontier out-edges
    C_NF_NEXT,
    C_MF_NEXT,
    C_MU,          // out-edges of unvisited vertices
    C_FOUND,
    C_NLONG,       // long tile-rows (>= kLongRow tiles) in the current long list
    C_NLONG_NEXT,
    C_WORDS
};

// Tile-rows of A^T with at least this many tiles are pushed by every warp
// together (a hub's out-edges), the others by one warp each.
constexpr int32_t kLongRow = 2048;

__global__ void dirop_decide_kernel(long long* ctl, int32_t n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!ctl[C_ACTIVE]) {
        ctl[C_PUSH] = 0;
        ctl[C_PULL] = 0;
        return;
    }
    long long dir = ctl[C_DIR];
    if (dir == 0 && ctl[C_MF] * kAlpha > ctl[C_MU]) dir = 1;
    else if (dir == 1 && ctl[C_NF] * kBeta < (long long)n) dir = 0;
    ctl[C_DIR] = dir;
    ctl[C_PUSH] = dir == 0;
    ctl[C_PULL] = dir == 1;
    ctl[C_NF_NEXT] = 0;
    ctl[C_MF_NEXT] = 0;
    ctl[C_FOUND] = 0;
    ctl[C_NNEXT] = 0;
    ctl[C_NLONG_NEXT] = 0;
}

// Push: a warp per frontier tile-row J of A^T; lanes over its tiles; every
// unvisited target of a frontier row is set in the next bitset.
template <int K>
__global__ void __launch_bounds__(256) dirop_push_kernel(const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ colind,
                                                         const uint8_t* __restrict__ tiles,
                                                         const int32_t* __restrict__ list,
                                                         const int32_t* __restrict__ longs, const uint32_t* frontier,
                                                         const uint32_t* visited, uint32_t* next, const long long* ctl) {
    constexpr int TB = K * (K <= 8 ? 1 : (K == 16 ? 2 : 4));
    constexpr int TW = (TB + 3) / 4;
    if (!ctl[C_PUSH]) return;
    const int64_t ncur = ctl[C_NCUR], nlong = ctl[C_NLONG];
    const int lane = (int)lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // every warp takes a slice of each long tile-row, the short ones a warp each
    auto push_tiles = [&](int32_t J, int64_t t_begin, int64_t t_end, int64_t stride) {
        const uint32_t amask = seg_bits<K>(frontier, J);
        for (int64_t t = t_begin + lane; t < t_end; t += stride) {
            uint32_t wd[TW];
            const uint32_t* tp = reinterpret_cast<const uint32_t*>(tiles + t * TB);
#pragma unroll
            for (int q = 0; q < TW; ++q) wd[q] = __ldg(tp + q);
            uint32_t cols = 0u;  // union of the frontier rows' bits: targets I*K + c
#pragma unroll
            for (int r = 0; r < K; ++r)
                if ((amask >> r) & 1u) cols |= tile_row<K>(wd, r);
            if (!cols) continue;
            const int32_t I = __ldg(colind + t);
            const int64_t base = (int64_t)I * K;
            cols &= ~seg_bits<K>(visited, I);
            if (!cols) continue;
            // the K bits of segment I sit in one 32-bit word of the bitset
            atomicOr(next + (base >> 5), cols << (int)(base & 31));
        }
    };
    for (int64_t e = 0; e < nlong; ++e) {
        const int32_t J = longs[e];
        push_tiles(J, rowptr[J] + gw * 32, rowptr[J + 1], warps * 32);
    }
    for (int64_t e = gw; e < ncur; e += warps) {
        const int32_t J = list[e];
        const int32_t t0 = rowptr[J], t1 = rowptr[J + 1];
        if (t1 - t0 < kLongRow) push_tiles(J, t0, t1, 32);
    }
}

// visited |= next; levels of the new vertices; next frontier's size, out-edges
// and tile-row list (every tile-row of A^T with a new vertex, once).
template <int K>
__global__ void dirop_update_kernel(const uint32_t* __restrict__ next, uint32_t* visited, int32_t* levels,
                                    int64_t words, int32_t n, const int32_t* __restrict__ deg, int32_t* nlist,
                                    const int32_t* __restrict__ rowptrT, int32_t* nlong, long long* ctl) {
    if (!ctl[C_ACTIVE]) return;
    const int32_t lv = (int32_t)ctl[C_LEVEL] + 1;
    long long nf = 0, mf = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = next[w] & ~visited[w];
        if (!b) continue;
        visited[w] |= b;
        uint32_t bb = b;
        while (bb) {
            const int c = __ffs(bb) - 1;
            bb &= bb - 1;
            const int64_t v = w * 32 + c;
            if (v < n) {
                levels[v] = lv;
                nf += 1;
                mf += deg[v];
            }
        }
        // tile-rows of K vertices covered by this word
#pragma unroll
        for (int sgm = 0; sgm < 32 / (K < 32 ? K : 32); ++sgm) {
            constexpr uint32_t kSegMask = K == 32 ? 0xFFFFFFFFu : ((1u << (K & 31)) - 1u);
            const uint32_t part = (b >> ((sgm * K) & 31)) & kSegMask;
            if (part) {
                const int32_t J = (int32_t)((w * 32) / K + sgm);
                nlist[atomicAdd(reinterpret_cast<unsigned long long*>(ctl + C_NNEXT), 1ull)] = J;
                if (rowptrT[J + 1] - rowptrT[J] >= kLongRow)
                    nlong[atomicAdd(reinterpret_cast<unsigned long long*>(ctl + C_NLONG_NEXT), 1ull)] = J;
            }
        }
    }
    // block-level sums, then one atomic per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
        mf += __shfl_xor_sync(0xffffffffu, mf, o);
    }
    if ((threadIdx.x & 31) == 0 && nf) {
        atomicAdd(reinterpret_cast<unsigned long long*>(ctl + C_NF_NEXT), (unsigned long long)nf);
        atomicAdd(reinterpret_cast<unsigned long long*>(ctl + C_MF_NEXT), (unsigned long long)mf);
        atomicExch(reinterpret_cast<unsigned long long*>(ctl + C_FOUND), 1ull);
    }
}

__global__ void dirop_advance_kernel(long long* ctl) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || !ctl[C_ACTIVE]) return;
    ctl[C_ACTIVE] = ctl[C_FOUND];
    ctl[C_LEVEL] += 1;
    ctl[C_MU] -= ctl[C_MF_NEXT];
    ctl[C_NF] = ctl[C_NF_NEXT];
    ctl[C_MF] = ctl[C_MF_NEXT];
    ctl[C_NCUR] = ctl[C_NNEXT];
    ctl[C_NLONG] = ctl[C_NLONG_NEXT];
}

// levels = -1, src = 0; frontier = visited = {src}; list = {src / kT}
__global__ void dirop_init_kernel(int32_t* levels, int32_t n, int64_t words, uint32_t* fa, uint32_t* fb,
                                  uint32_t* vis, int32_t src, int32_t kT, int32_t* list, int32_t* longs,
                                  const int32_t* rowptrT, long long* ctl, const int32_t* deg, long long nnz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n || i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) levels[i] = i == src ? 0 : -1;
        if (i < words) {
            const uint32_t b = i == (src >> 5) ? 1u << (src & 31) : 0u;
            fa[i] = b;
            fb[i] = 0u;
            vis[i] = b;
        }
        if (i == 0) {
            list[0] = src / kT;
            for (int c = 0; c < C_WORDS; ++c) ctl[c] = 0;
            ctl[C_ACTIVE] = 1;
            ctl[C_NCUR] = 1;
            ctl[C_NF] = 1;
            ctl[C_MF] = deg[src];
            ctl[C_MU] = nnz - deg[src];
            const int32_t J = src / kT;
            if (rowptrT[J + 1] - rowptrT[J] >= kLongRow) {
                longs[0] = J;
                ctl[C_NLONG] = 1;
            }
        }
    }
}

}  // namespace

b2sr_status bfs_dirop(b2sr_matrix* h, b2sr_matrix* hT, int32_t src, int32_t* levels, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    const int64_t words = ceil_div(n, 32);
    B2SR_TRY(ensure_outdeg(h, s));  // out-degrees (column counts of A); before capture
    const size_t bw = round_up((size_t)words * 4 + 4, 256);
    const size_t lw = round_up((size_t)hT->ntr * 4 + 4, 256);
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(3 * bw + 4 * lw + 256));
    char* base = buf.as<char>();
    uint32_t* fa = reinterpret_cast<uint32_t*>(base);
    uint32_t* fb = reinterpret_cast<uint32_t*>(base + bw);
    uint32_t* vis = reinterpret_cast<uint32_t*>(base + 2 * bw);
    int32_t* la = reinterpret_cast<int32_t*>(base + 3 * bw);
    int32_t* lb = reinterpret_cast<int32_t*>(base + 3 * bw + lw);
    int32_t* ga = reinterpret_cast<int32_t*>(base + 3 * bw + 2 * lw);  // long tile-rows
    int32_t* gb = reinterpret_cast<int32_t*>(base + 3 * bw + 3 * lw);
    long long* ctl = reinterpret_cast<long long*>(base + 3 * bw + 4 * lw);
    dirop_init_kernel<<<grid_for(std::max<int64_t>(n, words)), 256, 0, s>>>(levels, n, words, fa, fb, vis, src,
                                                                             hT->k, la, ga, hT->rowptr, ctl,
                                                                             h->outdeg, h->nnz);
    B2SR_LAUNCH_CHECK("dirop_init_kernel");
    // the loop's exit flag and the pull gate: the low words of C_ACTIVE and C_PULL (little-endian)
    const int32_t* active32 = reinterpret_cast<const int32_t*>(ctl + C_ACTIVE);
    const int32_t* pull_gate = reinterpret_cast<const int32_t*>(ctl + C_PULL);
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n + 1;
    const int push_grid = sm_count() * 8;
    int64_t rounds = 0;
    return with_tile(hT->k, [&](auto kc) -> b2sr_status {
        constexpr int KT = decltype(kc)::value;
        return run_captured(s, 4, cap + 1, active32,
                                [&](cudaStream_t cs, int r) -> b2sr_status {
                                    uint32_t* f = (r & 1) ? fb : fa;
                                    uint32_t* nx = (r & 1) ? fa : fb;
                                    int32_t* cur = (r & 1) ? lb : la;
                                    int32_t* nxt = (r & 1) ? la : lb;
                                    int32_t* curl = (r & 1) ? gb : ga;
                                    int32_t* nxtl = (r & 1) ? ga : gb;
                                    dirop_decide_kernel<<<1, 32, 0, cs>>>(ctl, n);
                                    B2SR_LAUNCH_CHECK("dirop_decide_kernel");
                                    B2SR_CUDA_TRY(cudaMemsetAsync(nx, 0, words * 4, cs));
                                    dirop_push_kernel<KT><<<push_grid, 256, 0, cs>>>(hT->rowptr, hT->colind, hT->tiles,
                                                                                    cur, curl, f, vis, nx, ctl);
                                    B2SR_LAUNCH_CHECK("dirop_push_kernel");
                                    B2SR_TRY(spmv_dispatch(h, B2SR_BOOL_OR_AND, B2SR_VEC_BITS, f, B2SR_VEC_BITS, nx,
                                                           vis, 1, nullptr, cs, pull_gate));
                                    dirop_update_kernel<KT><<<grid_for(words), 256, 0, cs>>>(nx, vis, levels, words, n,
                                                                                            h->outdeg, nxt,
                                                                                            hT->rowptr, nxtl, ctl);
                                    B2SR_LAUNCH_CHECK("dirop_update_kernel");
                                    dirop_advance_kernel<<<1, 32, 0, cs>>>(ctl);
                                    B2SR_LAUNCH_CHECK("dirop_advance_kernel");
                                    return B2SR_OK;
                                },
                                &rounds);
    });
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_bfs_diropt(b2sr_handle h, b2sr_handle hT, int32_t src, int32_t* levels, int max_iters,
                                       void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (!hT) hT = h;
    B2SR_TRY(check_handle(hT));
    if (hT->n != h->n) return fail(B2SR_ERR_INVALID_ARG, "hT must be the transpose of h (same n)");
    if (src < 0 || src >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (!levels) return fail(B2SR_ERR_INVALID_ARG, "levels is NULL");
    return bfs_dirop(h, hT, src, levels, max_iters, to_stream(stream));
}
