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
// the next list.  With delta > 0 the rounds keep a threshold: a vertex whose
// distance is at or past it goes to a far set (bitset + list) instead, where
// it costs nothing until the near set runs dry; then the threshold rises by
// delta and the far set becomes the next round's active set (delta-stepping's
// buckets as a near/far pair of worklists).  Distances only decrease, and
// every value written is the length of a path, so the result is the
// shortest-path fixed point whatever the order of the atomics: bit-exact and
// the same as b2sr_sssp's.
#include <algorithm>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "captured.cuh"
#include "tile_bits.cuh"

namespace b2sr {

struct PushSide {
    uint32_t* act;   // vertex bitset
    int32_t* list;   // tile-rows holding its bits, each once
    int32_t* count;  // list length
};

// Sets vertex v in `side`; the first setter of a bit lists v's tile-row
// unless it is listed already (membership in `listed`).
template <int K>
__device__ __forceinline__ void mark_vertex(PushSide side, int32_t* listed, int32_t v) {
    const uint32_t b = 1u << (v & 31);
    if (!(atomicOr(side.act + (v >> 5), b) & b)) {
        const int32_t J = v / K;
        if (atomicExch(listed + J, 1) == 0) side.list[atomicAdd(side.count, 1)] = J;
    }
}

// ORs the K-bit segment `v` into tile-row J's bits (segments of k = 4 share
// a byte, so every width goes through a word atomic).
template <int K>
__device__ __forceinline__ void or_seg(uint32_t* bits, int32_t J, uint32_t v) {
    constexpr int per = 32 / K;
    atomicOr(bits + J / per, v << ((J % per) * K));
}

// One round.  `far` (with its own list-membership array `farflag`) holds the
// vertices at or past the threshold: they wait there, untouched, until the
// near set runs dry and the threshold moves (delta-stepping's later buckets).
template <int K>
__device__ __forceinline__ void relax_round(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                            const uint8_t* __restrict__ tiles, const int32_t* __restrict__ voff,
                                            const float* __restrict__ w, PushSide cur, PushSide nxt, int32_t* flag,
                                            PushSide far, int32_t* farflag, int* farmin, float* dist,
                                            const float* theta, int64_t warp0, int64_t warps) {
    constexpr int TB = K * (K <= 8 ? 1 : (K == 16 ? 2 : 4));  // bytes per tile
    constexpr int TW = (TB + 3) / 4;
    const int32_t ncur = *reinterpret_cast<volatile int32_t*>(cur.count);
    const float th = theta ? *reinterpret_cast<const volatile float*>(theta) : INFINITY;
    const int lane = (int)lane_id();
    for (int64_t e = warp0; e < ncur; e += warps) {
        const int32_t J = cur.list[e];
        uint32_t amask = seg_bits<K>(cur.act, J);
        if (theta) {
            // active vertices at or past the threshold move to the far set
            uint32_t defer = 0u;
            if (lane < K && ((amask >> lane) & 1u)) {
                const float du = dist[J * K + lane];
                if (du >= th) {
                    defer = 1u << lane;
                    atomicMin(farmin, __float_as_int(du));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) defer |= __shfl_xor_sync(0xffffffffu, defer, o);
            if (defer) {
                if (lane == 0) {
                    or_seg<K>(far.act, J, defer);
                    if (atomicExch(farflag + J, 1) == 0) far.list[atomicAdd(far.count, 1)] = J;
                }
            }
            amask &= ~defer;
        }
        if (!amask) continue;
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
                            if (cand >= th) {
                                atomicMin(farmin, __float_as_int(cand));
                                mark_vertex<K>(far, farflag, v);
                            } else {
                                mark_vertex<K>(nxt, flag, v);
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
                                                         PushSide cur, PushSide nxt, int32_t* flag, PushSide far,
                                                         int32_t* farflag, int* farmin, float* dist,
                                                         const float* theta, const int32_t* gate) {
    if (gate && *gate == 0) return;
    relax_round<K>(rowptr, colind, tiles, voff, w, cur, nxt, flag, far, farflag, farmin, dist, theta,
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

// Loop control words (device).
struct PushCtl {
    int32_t* active;  // 1 while a round has work
    int32_t* rounds;  // rounds run
    int32_t* drain;   // far entries the drain kernel moves into the next set
    float* theta;     // threshold (nullptr: no buckets)
    int* farmin;      // least distance (float bits) that entered the far set since it was last moved
    unsigned long long* worked;  // active tile-rows summed over the rounds
};

// After a round: the next round reads `nxt`, and the list it builds starts
// empty.  When the near set is empty but far vertices wait, the threshold
// rises by delta -- or, past a gap in the distances, to the least far
// distance plus delta, so that the nearest waiting vertex always gets in --
// and the whole far set becomes the next round's active set (whatever is
// still past the threshold moves back in that round).  The loop stops when
// both sets are empty.
__global__ void push_advance_kernel(int32_t* cur_count, int32_t* next_count, int32_t* far_count, PushCtl c,
                                    float delta) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || !*c.active) return;
    *c.worked += (unsigned long long)*reinterpret_cast<volatile int32_t*>(cur_count);
    *reinterpret_cast<volatile int32_t*>(cur_count) = 0;
    int32_t nn = *reinterpret_cast<volatile int32_t*>(next_count);
    int32_t dn = 0;
    if (c.theta) {
        const int32_t fc = *reinterpret_cast<volatile int32_t*>(far_count);
        if (nn == 0 && fc > 0) {
            const float th = *reinterpret_cast<volatile float*>(c.theta);
            const float fm = __int_as_float(*reinterpret_cast<volatile int*>(c.farmin));
            float nt = fmaxf(th + delta, fm + delta);
            if (!(nt > fm)) nt = nextafterf(fm, INFINITY);  // delta below the spacing of floats there
            if (!(nt > th)) nt = nextafterf(th, INFINITY);
            *reinterpret_cast<volatile float*>(c.theta) = nt;
            *reinterpret_cast<volatile int*>(c.farmin) = __float_as_int(INFINITY);
            *reinterpret_cast<volatile int32_t*>(next_count) = fc;
            *reinterpret_cast<volatile int32_t*>(far_count) = 0;
            nn = dn = fc;
        }
    }
    *reinterpret_cast<volatile int32_t*>(c.drain) = dn;
    *reinterpret_cast<volatile int32_t*>(c.active) = nn > 0 ? 1 : 0;
    *c.rounds += 1;
}

// Moves the far set into the (empty) next set: list, bits and membership.
template <int K>
__global__ void push_drain_kernel(PushSide nxt, PushSide far, int32_t* farflag, const int32_t* drain) {
    const int32_t nd = *drain;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t J = far.list[i];
        nxt.list[i] = J;
        or_seg<K>(nxt.act, J, seg_bits<K>(far.act, J));
        clear_seg<K>(far.act, J);
        farflag[J] = 0;
    }
}

__global__ void push_init_kernel(float* dist, int32_t n, int32_t src) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dist[i] = (i == src) ? 0.0f : INFINITY;
}

thread_local int64_t g_last_push_rounds = 0;
thread_local int64_t g_last_push_rows = 0;

b2sr_status sssp_push(b2sr_matrix* hT, const float* w, int32_t src, float* dist, float delta, int max_iters,
                      cudaStream_t s) {
    g_last_push_rounds = 0;
    g_last_push_rows = 0;
    const int32_t n = hT->n;
    const int32_t ntr = hT->ntr;
    if (w) B2SR_TRY(ensure_voff(hT, s));  // before capture: capture must not allocate for the handle
    const size_t bw = round_up((size_t)ceil_div(n, 32) * 4 + 4, 256);  // bitsets (+1 word: k=4 byte pairs)
    const size_t lw = round_up((size_t)ntr * 4 + 4, 256);
    const size_t total = 3 * bw + 5 * lw + 256;
    DevBuf buf(s);
    B2SR_TRY(buf.alloc(total));
    char* base = buf.as<char>();
    int32_t* ctl = reinterpret_cast<int32_t*>(base + 3 * bw + 5 * lw);
    // ctl: countA, countB, countFar, active, rounds, drain, theta (float), farmin (float bits), -,
    // worked (8 bytes at ctl + 10: ctl is 256-byte aligned)
    PushSide A{reinterpret_cast<uint32_t*>(base), reinterpret_cast<int32_t*>(base + 3 * bw), ctl};
    PushSide Bs{reinterpret_cast<uint32_t*>(base + bw), reinterpret_cast<int32_t*>(base + 3 * bw + lw), ctl + 1};
    PushSide F{reinterpret_cast<uint32_t*>(base + 2 * bw), reinterpret_cast<int32_t*>(base + 3 * bw + 2 * lw),
               ctl + 2};
    int32_t* flag = reinterpret_cast<int32_t*>(base + 3 * bw + 3 * lw);
    int32_t* farflag = reinterpret_cast<int32_t*>(base + 3 * bw + 4 * lw);
    PushCtl c{ctl + 3, ctl + 4, ctl + 5, delta > 0.0f ? reinterpret_cast<float*>(ctl + 6) : nullptr, ctl + 7,
              reinterpret_cast<unsigned long long*>(ctl + 10)};
    B2SR_CUDA_TRY(cudaMemsetAsync(base, 0, total, s));
    push_init_kernel<<<grid_for(n), 256, 0, s>>>(dist, n, src);
    B2SR_LAUNCH_CHECK("push_init_kernel");
    // seed: the source in A, its tile-row in A's list
    const int32_t seed_row = src / hT->k;
    const uint32_t seed_bit = 1u << (src & 31);
    const int32_t one = 1;
    B2SR_CUDA_TRY(cudaMemcpyAsync(A.act + (src >> 5), &seed_bit, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(A.list, &seed_row, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(A.count, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(c.active, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (c.theta) B2SR_CUDA_TRY(cudaMemcpyAsync(c.theta, &delta, sizeof(float), cudaMemcpyHostToDevice, s));
    const float inf = INFINITY;
    B2SR_CUDA_TRY(cudaMemcpyAsync(c.farmin, &inf, sizeof(float), cudaMemcpyHostToDevice, s));
    const int relax_grid = sm_count() * 8;  // warps stride over the active list
    const int list_grid = sm_count() * 2;   // threads stride over the lists
    // default round limit: without buckets at most n rounds improve anything;
    // with them every raise of the threshold settles at least one vertex and
    // costs a few rounds beyond the improving ones, so 4n covers both
    const int64_t cap = max_iters > 0 ? max_iters : (c.theta ? 4 * (int64_t)n + 4 : (int64_t)n + 1);
    int64_t replayed = 0;
    const float* wts = w;
    const int32_t* voff = w ? hT->voff : nullptr;
    b2sr_status st = with_tile(hT->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        return run_captured(s, 32, cap + 1, c.active,
                            [&](cudaStream_t cs, int r) -> b2sr_status {
                                const PushSide& cur = (r & 1) ? Bs : A;
                                const PushSide& nxt = (r & 1) ? A : Bs;
                                push_relax_kernel<K><<<relax_grid, 256, 0, cs>>>(hT->rowptr, hT->colind, hT->tiles,
                                                                                voff, wts, cur, nxt, flag, F, farflag,
                                                                                c.farmin, dist, c.theta, c.active);
                                B2SR_LAUNCH_CHECK("push_relax_kernel");
                                push_epilogue_kernel<K><<<list_grid, 256, 0, cs>>>(cur, nxt, flag, c.active);
                                B2SR_LAUNCH_CHECK("push_epilogue_kernel");
                                push_advance_kernel<<<1, 32, 0, cs>>>(cur.count, nxt.count, F.count, c, delta);
                                B2SR_LAUNCH_CHECK("push_advance_kernel");
                                if (c.theta) {
                                    push_drain_kernel<K><<<list_grid, 256, 0, cs>>>(nxt, F, farflag, c.drain);
                                    B2SR_LAUNCH_CHECK("push_drain_kernel");
                                }
                                return B2SR_OK;
                            },
                            &replayed);
    });
    if (st != B2SR_OK) return st;
    int32_t r = 0;
    unsigned long long rows = 0;
    B2SR_CUDA_TRY(cudaMemcpyAsync(&r, c.rounds, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(&rows, c.worked, sizeof(rows), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    g_last_push_rounds = r;
    g_last_push_rows = (int64_t)rows;
    return B2SR_OK;
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

extern "C" b2sr_status b2sr_sssp_push_rounds(int64_t* rounds, int64_t* active_tile_rows) {
    clear_error();
    if (!rounds) return fail(B2SR_ERR_INVALID_ARG, "rounds is NULL");
    *rounds = g_last_push_rounds;
    if (active_tile_rows) *active_tile_rows = g_last_push_rows;
    return B2SR_OK;
}
