// SSSP by frontier-driven push relaxation over the transposed bit tiles.
//
// b2sr_sssp relaxes every edge in every round (a min-plus SpMV over the whole
// matrix, Sec. V SSSP).  On graphs of large hop diameter -- a 4096 x 4096
// grid needs about 8,000 rounds -- nearly all of that work is wasted: only
// the vertices whose distance dropped in the previous round can improve a
// neighbour.  This driver keeps that set as a bitset plus a list of the
// tile-rows holding it, and pushes only from them.  It reads B2SR of the
// transpose, A^T: tile-row J of A^T lists, in its bits, the out-edges of the
// vertices kJ .. kJ+k-1 (for a symmetric matrix A^T = A and the handle serves
// as its own transpose).
//
// One round: a warp per active tile-row J takes its tiles; for every set bit
// (r, c) of tile (J, I) whose source row r is active, the target kI+c is
// relaxed with dist[kJ+r] + w by an integer atomicMin on the float's bits
// (non-negative floats order like their bit patterns).  A target that
// improves is marked in the next bitset, and its tile-row is appended once to
// the next list.  Distances only decrease, and every value written is the
// length of a path, so the result is the shortest-path fixed point whatever
// the order of the atomics: bit-exact and the same as b2sr_sssp's.
#include <algorithm>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "captured.cuh"
#include "tile_bits.cuh"

namespace b2sr {

struct PushSide {
    uint32_t* act;   // vertices improved in the previous round (bitset)
    int32_t* list;   // their tile-rows, each once
    int32_t* count;  // list length
};

template <int K>
__device__ __forceinline__ void relax_round(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                            const uint8_t* __restrict__ tiles, const int32_t* __restrict__ voff,
                                            const float* __restrict__ w, PushSide cur, PushSide nxt, int32_t* flag,
                                            float* dist, const float* theta, int32_t* relaxed, int64_t warp0,
                                            int64_t warps) {
    constexpr int TB = K * (K <= 8 ? 1 : (K == 16 ? 2 : 4));  // bytes per tile
    constexpr int TW = (TB + 3) / 4;
    const int32_t ncur = *reinterpret_cast<volatile int32_t*>(cur.count);
    const float th = theta ? *reinterpret_cast<const volatile float*>(theta) : INFINITY;
    const int lane = (int)lane_id();
    for (int64_t e = warp0; e < ncur; e += warps) {
        const int32_t J = cur.list[e];
        uint32_t amask = seg_bits<K>(cur.act, J);
        if (theta) {
            // active vertices at or past the threshold wait for a later round
            uint32_t defer = 0u;
            if (lane < K && ((amask >> lane) & 1u) && dist[J * K + lane] >= th) defer = 1u << lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) defer |= __shfl_xor_sync(0xffffffffu, defer, o);
            if (defer) {
                if (lane < K && ((defer >> lane) & 1u)) atomicOr(nxt.act + ((J * K + lane) >> 5), 1u << ((J * K + lane) & 31));
                if (lane == 0 && atomicExch(flag + J, 1) == 0) nxt.list[atomicAdd(nxt.count, 1)] = J;
            }
            amask &= ~defer;
            if (amask && lane == 0) *relaxed = 1;
        }
        const int32_t t0 = rowptr[J], t1 = rowptr[J + 1];
        for (int32_t t = t0 + lane; t < t1; t += 32) {
            uint32_t wd[TW];
            const uint32_t* tp = reinterpret_cast<const uint32_t*>(tiles + (int64_t)t * TB);
#pragma unroll
            for (int q = 0; q < TW; ++q) wd[q] = __ldg(tp + q);
            const int32_t I = __ldg(colind + t);
            const int32_t wbase = voff ? __ldg(voff + t) : 0;
            int qb = 0;  // set bits before the current row (set-bit order of the weights)
#pragma unroll
            for (int r = 0; r < K; ++r) {
                uint32_t bits = tile_row<K>(wd, r);
                if ((amask >> r) & 1u) {
                    const int32_t u = J * K + r;
                    const float du = dist[u];
                    int rank = qb;
                    while (bits) {
                        const int c = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const int32_t v = I * K + c;
                        const float cand = du + (w ? __ldg(w + wbase + rank) : 1.0f);
                        ++rank;
                        const int old = atomicMin(reinterpret_cast<int*>(dist) + v, __float_as_int(cand));
                        if (cand < __int_as_float(old)) {
                            const uint32_t b = 1u << (v & 31);
                            if (!(atomicOr(nxt.act + (v >> 5), b) & b)) {
                                const int32_t JJ = v / K;
                                if (atomicExch(flag + JJ, 1) == 0) nxt.list[atomicAdd(nxt.count, 1)] = JJ;
                            }
                        }
                    }
                }
                qb += __popc(tile_row<K>(wd, r));
            }
        }
    }
}

template <int K>
__global__ void __launch_bounds__(256) push_relax_kernel(const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ colind,
                                                         const uint8_t* __restrict__ tiles,
                                                         const int32_t* __restrict__ voff, const float* __restrict__ w,
                                                         PushSide cur, PushSide nxt, int32_t* flag, float* dist,
                                                         const float* theta, int32_t* relaxed, const int32_t* gate) {
    if (gate && *gate == 0) return;
    relax_round<K>(rowptr, colind, tiles, voff, w, cur, nxt, flag, dist, theta, relaxed,
                   ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, (int64_t)gridDim.x * (blockDim.x >> 5));
}

// After a round: the consumed active set is cleared (it becomes the next
// round's empty "next" set) and the new list's membership flags are reset.
template <int K>
__device__ __forceinline__ void epilogue_round(PushSide cur, PushSide nxt, int32_t* flag, int64_t t0, int64_t nt) {
    const int32_t ncur = *reinterpret_cast<volatile int32_t*>(cur.count);
    const int32_t nnext = *reinterpret_cast<volatile int32_t*>(nxt.count);
    for (int64_t i = t0; i < ncur || i < nnext; i += nt) {
        if (i < ncur) clear_seg<K>(cur.act, cur.list[i]);
        if (i < nnext) flag[nxt.list[i]] = 0;
    }
}

template <int K>
__global__ void push_epilogue_kernel(PushSide cur, PushSide nxt, int32_t* flag, const int32_t* gate) {
    if (gate && *gate == 0) return;
    epilogue_round<K>(cur, nxt, flag, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                      (int64_t)gridDim.x * blockDim.x);
}

// After a round: the next round reads `nxt`, and the list it builds starts
// empty; the loop stops when a round improved nothing.  With a threshold, a
// round that relaxed nothing (everything active waits) raises it by delta.
__device__ __forceinline__ void advance_round(int32_t* cur_count, const int32_t* next_count, int32_t* active,
                                              int32_t* rounds, float* theta, int32_t* relaxed, float delta) {
    *reinterpret_cast<volatile int32_t*>(cur_count) = 0;
    const int32_t nn = *reinterpret_cast<const volatile int32_t*>(next_count);
    *reinterpret_cast<volatile int32_t*>(active) = nn > 0 ? 1 : 0;
    if (theta) {
        if (!*reinterpret_cast<volatile int32_t*>(relaxed) && nn > 0)
            *reinterpret_cast<volatile float*>(theta) = *reinterpret_cast<volatile float*>(theta) + delta;
        *reinterpret_cast<volatile int32_t*>(relaxed) = 0;
    }
    *rounds += 1;
}

__global__ void push_advance_kernel(int32_t* cur_count, const int32_t* next_count, int32_t* active, int32_t* rounds,
                                    float* theta, int32_t* relaxed, float delta) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *active)
        advance_round(cur_count, next_count, active, rounds, theta, relaxed, delta);
}

__global__ void push_init_kernel(float* dist, int32_t n, int32_t src) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dist[i] = (i == src) ? 0.0f : INFINITY;
}

b2sr_status sssp_push(b2sr_matrix* hT, const float* w, int32_t src, float* dist, float delta, int max_iters,
                      cudaStream_t s) {
    const int32_t n = hT->n;
    const int32_t ntr = hT->ntr;
    if (w) B2SR_TRY(ensure_voff(hT, s));  // before capture: capture must not allocate for the handle
    const size_t bw = round_up((size_t)ceil_div(n, 32) * 4 + 4, 256);  // bitsets (+1 word: k=4 byte pairs)
    const size_t lw = round_up((size_t)ntr * 4 + 4, 256);
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(2 * bw + 3 * lw + 256));
    char* base = buf.as<char>();
    PushSide A{reinterpret_cast<uint32_t*>(base), reinterpret_cast<int32_t*>(base + 2 * bw), nullptr};
    PushSide Bs{reinterpret_cast<uint32_t*>(base + bw), reinterpret_cast<int32_t*>(base + 2 * bw + lw), nullptr};
    int32_t* flag = reinterpret_cast<int32_t*>(base + 2 * bw + 2 * lw);
    int32_t* ctl = reinterpret_cast<int32_t*>(base + 2 * bw + 3 * lw);  // countA, countB, active, rounds
    A.count = ctl;
    Bs.count = ctl + 1;
    int32_t* active = ctl + 2;
    int32_t* rounds_dev = ctl + 3;
    // ctl[5]: threshold (float), ctl[6]: relaxed-this-round
    float* theta = delta > 0.0f ? reinterpret_cast<float*>(ctl + 5) : nullptr;
    int32_t* relaxed = ctl + 6;
    B2SR_CUDA_TRY(cudaMemsetAsync(base, 0, 2 * bw + 3 * lw + 256, s));
    push_init_kernel<<<grid_for(n), 256, 0, s>>>(dist, n, src);
    B2SR_LAUNCH_CHECK("push_init_kernel");
    // seed: the source in A, its tile-row in A's list
    const int32_t seed_row = src / hT->k;
    const uint32_t seed_bit = 1u << (src & 31);
    const int32_t one = 1;
    B2SR_CUDA_TRY(cudaMemcpyAsync(A.act + (src >> 5), &seed_bit, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(A.list, &seed_row, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(A.count, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(active, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (theta) B2SR_CUDA_TRY(cudaMemcpyAsync(theta, &delta, sizeof(float), cudaMemcpyHostToDevice, s));
    const int relax_grid = sm_count() * 8;  // warps stride over the active list
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n + 1;
    int64_t rounds = 0;
    const float* wts = w;
    const int32_t* voff = w ? hT->voff : nullptr;
    return with_tile(hT->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        return run_captured(s, 32, cap + 1, active,
                            [&](cudaStream_t cs, int r) -> b2sr_status {
                                const PushSide& cur = (r & 1) ? Bs : A;
                                const PushSide& nxt = (r & 1) ? A : Bs;
                                push_relax_kernel<K><<<relax_grid, 256, 0, cs>>>(hT->rowptr, hT->colind, hT->tiles,
                                                                                voff, wts, cur, nxt, flag, dist,
                                                                                theta, relaxed, active);
                                B2SR_LAUNCH_CHECK("push_relax_kernel");
                                push_epilogue_kernel<K><<<grid_for(ntr), 256, 0, cs>>>(cur, nxt, flag, active);
                                B2SR_LAUNCH_CHECK("push_epilogue_kernel");
                                push_advance_kernel<<<1, 32, 0, cs>>>(cur.count, nxt.count, active, rounds_dev,
                                                                      theta, relaxed, delta);
                                B2SR_LAUNCH_CHECK("push_advance_kernel");
                                return B2SR_OK;
                            },
                            &rounds);
    });
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_sssp_push(b2sr_handle hT, const float* weights_t, int32_t src, float* dist, float delta,
                                      int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(hT));
    if (src < 0 || src >= hT->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (!dist) return fail(B2SR_ERR_INVALID_ARG, "dist is NULL");
    if (!(delta == delta)) return fail(B2SR_ERR_INVALID_ARG, "delta is NaN");
    return sssp_push(hT, weights_t, src, dist, delta, max_iters, to_stream(stream));
}
