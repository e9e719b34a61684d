// Maximal independent set and graph colouring (the MIS and GC rows of
// Table 4: the local-maximum test runs on the tropical max-times semiring,
// the removal of the new members' neighbours on the Boolean semiring).  The
// paper lists both operations without an algorithm; both drivers run the
// synchronous rounds of Luby's algorithm with fixed priorities:
//
//   MIS: every undecided vertex whose key is the largest among itself and its
//        undecided neighbours joins the set; the new members and their
//        neighbours are decided.  The result is the set the sequential greedy
//        algorithm builds in decreasing key order.
//   colouring: every uncoloured vertex whose key is the largest among itself
//        and its uncoloured neighbours takes the round's index as its colour
//        (each round's vertices are independent, so no edge joins two equal
//        colours); colour(v) = 1 + the largest colour among v's higher-key
//        neighbours, 0 if there is none.
//
// Keys are 64-bit: the priority's bits mapped to an unsigned order (+0 and -0
// equal) above the vertex id, so equal priorities order by the larger id and
// all keys differ.  A vertex's own key takes part in its maximum, so a
// self-loop changes nothing.  Decided vertices hold key 0, below every key.
// Rounds are captured as a CUDA graph of gated rounds (captured.cuh).
//
// The colouring's rounds number the longest chain of decreasing keys, which
// on a power-law graph with random priorities runs to well over a thousand:
// re-reading every tile each round (the max-times rounds) then costs that
// many SpMVs.  The push form computes the same colours from counters: cnt[v]
// = neighbours with a larger key still uncoloured; the vertices coloured in
// round r push along their rows, and a vertex whose counter reaches 0 gets
// colour r + 1 and joins the next frontier.  Each edge is read twice in all
// (the count and one push), as in a topological sort by levels.
#include <algorithm>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "captured.cuh"
#include "tile_bits.cuh"

namespace b2sr {
b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s,
                          const int32_t* gate);
b2sr_status spmv_maxkey_dispatch(b2sr_matrix* h, const uint64_t* x, uint64_t* y, const uint32_t* mask, int comp,
                                 cudaStream_t s, const int32_t* gate);

namespace {

__device__ __forceinline__ uint64_t priority_key(float p, int32_t v) {
    uint32_t b = __float_as_uint(p);
    if ((b & 0x7FFFFFFFu) == 0u) b = 0u;                        // -0 orders as +0
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // monotone in p
    return ((uint64_t)o << 32) | (uint32_t)v;
}

// keys of every vertex, all undecided; out[v] = init; bad if a NaN priority
__global__ void keys_init_kernel(const float* __restrict__ prio, int32_t n, uint64_t* __restrict__ key,
                                 uint32_t* __restrict__ undecided, int64_t words, int32_t* __restrict__ out,
                                 int32_t init, int32_t* bad) {
    int nan = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = w * 32;
        const int cnt = (int)min((int64_t)32, (int64_t)n - v0);
        for (int c = 0; c < cnt; ++c) {
            const float p = prio[v0 + c];
            nan |= isnan(p);
            key[v0 + c] = priority_key(p, (int32_t)(v0 + c));
            out[v0 + c] = init;
        }
        undecided[w] = cnt >= 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u);
    }
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(bad, 1);
}

// active <- found (only while active); the round counter advances with it
__global__ void rounds_advance_kernel(int32_t* active, const int32_t* found, int32_t* round) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *active) {
        *active = *found;
        *round += 1;
    }
}

// MIS: undecided local maxima join (J), in_set = 1
__global__ void mis_select_kernel(const uint64_t* __restrict__ key, const uint64_t* __restrict__ mx,
                                  const uint32_t* __restrict__ undecided, uint32_t* __restrict__ joined,
                                  int32_t* __restrict__ in_set, int64_t words, const int32_t* gate) {
    if (gate_closed(gate)) return;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t u = undecided[w], sel = 0u;
        while (u) {
            const int c = __ffs(u) - 1;
            u &= u - 1;
            const int64_t v = w * 32 + c;
            if (key[v] >= mx[v]) {
                sel |= 1u << c;
                in_set[v] = 1;
            }
        }
        joined[w] = sel;
    }
}

// MIS: the new members and their undecided neighbours (nb) are decided
__global__ void mis_remove_kernel(uint64_t* __restrict__ key, uint32_t* __restrict__ undecided,
                                  const uint32_t* __restrict__ joined, const uint32_t* __restrict__ nb, int64_t words,
                                  const int32_t* gate, int32_t* found) {
    if (gate_closed(gate)) return;
    int any = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = undecided[w];
        uint32_t rem = (joined[w] | nb[w]) & u;
        const uint32_t left = u & ~rem;
        if (rem) undecided[w] = left;
        while (rem) {
            const int c = __ffs(rem) - 1;
            rem &= rem - 1;
            key[w * 32 + c] = 0ull;
        }
        any |= left != 0u;
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(found, 1);
}

// colouring: uncoloured local maxima take the round's colour and leave
__global__ void color_select_kernel(uint64_t* __restrict__ key, const uint64_t* __restrict__ mx,
                                    uint32_t* __restrict__ uncoloured, int32_t* __restrict__ colors, int64_t words,
                                    const int32_t* round, const int32_t* gate, int32_t* found) {
    if (gate_closed(gate)) return;
    const int32_t col = *round;
    int any = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t u = uncoloured[w], sel = 0u;
        const uint32_t all = u;
        while (u) {
            const int c = __ffs(u) - 1;
            u &= u - 1;
            const int64_t v = w * 32 + c;
            if (key[v] >= mx[v]) sel |= 1u << c;
        }
        // the maxima were taken before this kernel: clearing keys here is safe
        for (uint32_t b = sel; b;) {
            const int c = __ffs(b) - 1;
            b &= b - 1;
            colors[w * 32 + c] = col;
            key[w * 32 + c] = 0ull;
        }
        if (sel) uncoloured[w] = all & ~sel;
        any |= (all & ~sel) != 0u;
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(found, 1);
}

// ---------------------------------------------------------------------------
// colouring by pushes along the rows of the frontier
// ---------------------------------------------------------------------------
// Tile-rows are listed in segments of kSeg tiles (entry = J << 32 | segment),
// so a hub's long row is shared by many warps.
constexpr int32_t kSeg = 256;

struct Frontier {
    uint32_t* act;    // vertices coloured in the round (bitset)
    int64_t* list;    // segments of their tile-rows, each tile-row once
    int32_t* count;   // list length
};

__device__ __forceinline__ void append_row(const int32_t* __restrict__ rowptr, Frontier f, int32_t* flag, int32_t J) {
    const int32_t len = rowptr[J + 1] - rowptr[J];
    if (len == 0 || atomicExch(flag + J, 1) != 0) return;  // no neighbours, or listed already
    const int32_t nseg = (len + kSeg - 1) / kSeg;
    const int32_t base = atomicAdd(f.count, nseg);
    for (int32_t q = 0; q < nseg; ++q) f.list[base + q] = ((int64_t)J << 32) | q;
}

// every non-empty tile-row, each with its segments (the counting pass)
__global__ void list_all_rows_kernel(const int32_t* __restrict__ rowptr, int32_t ntr, Frontier f) {
    for (int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; J < ntr; J += (int64_t)gridDim.x * blockDim.x) {
        const int32_t len = rowptr[J + 1] - rowptr[J];
        if (len == 0) continue;
        const int32_t nseg = (len + kSeg - 1) / kSeg;
        const int32_t base = atomicAdd(f.count, nseg);
        for (int32_t q = 0; q < nseg; ++q) f.list[base + q] = ((int64_t)J << 32) | q;
    }
}

// COUNT: cnt[v] += 1 for every edge (u, v) of a listed u with key[v] < key[u].
// PUSH: cnt[v] -= 1 likewise; the push that takes it to 0 colours v with
// *level + 1 and lists v in nxt.
template <int K, bool COUNT>
__global__ void __launch_bounds__(256) colour_push_kernel(const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ colind,
                                                          const uint8_t* __restrict__ tiles,
                                                          const uint64_t* __restrict__ key, int32_t* cnt,
                                                          int32_t* colors, Frontier cur, Frontier nxt, int32_t* flag,
                                                          const int32_t* level, const int32_t* gate) {
    if (gate_closed(gate)) return;
    constexpr int TB = K * (K <= 8 ? 1 : (K == 16 ? 2 : 4));  // bytes per tile
    constexpr int TW = (TB + 3) / 4;
    const int32_t ncur = *reinterpret_cast<volatile int32_t*>(cur.count);
    const int32_t col = COUNT ? 0 : *level + 1;
    const int lane = (int)lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < ncur; e += warps) {
        const int64_t ent = cur.list[e];
        const int32_t J = (int32_t)(ent >> 32), q = (int32_t)(ent & 0xFFFFFFFF);
        const uint32_t amask = seg_bits<K>(cur.act, J);
        const int32_t t1 = rowptr[J + 1];
        const int32_t ta = rowptr[J] + q * kSeg, tb = min(t1, ta + kSeg);
        for (int32_t t = ta + lane; t < tb; t += 32) {
            uint32_t wd[TW];
            const uint32_t* tp = reinterpret_cast<const uint32_t*>(tiles + (int64_t)t * TB);
#pragma unroll
            for (int w = 0; w < TW; ++w) wd[w] = __ldg(tp + w);
            const int32_t I = __ldg(colind + t);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                uint32_t bits = tile_row<K>(wd, r);
                if (!((amask >> r) & 1u) || !bits) continue;
                const uint64_t ku = key[(int64_t)J * K + r];
                while (bits) {
                    const int c = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int32_t v = I * K + c;
                    if (key[v] >= ku) continue;  // v is not below u (or is u)
                    if (COUNT) {
                        atomicAdd(cnt + v, 1);
                    } else if (atomicSub(cnt + v, 1) == 1) {
                        colors[v] = col;
                        atomicOr(nxt.act + (v >> 5), 1u << (v & 31));
                        append_row(rowptr, nxt, flag, v / K);
                    }
                }
            }
        }
    }
}

// vertices with no larger neighbour: colour 0, the first frontier
__global__ void colour_seed_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cnt, int32_t n,
                                   int32_t k, int32_t* colors, Frontier f, int32_t* flag) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (cnt[v] != 0) continue;
        colors[v] = 0;
        atomicOr(f.act + (v >> 5), 1u << (v & 31));
        append_row(rowptr, f, flag, (int32_t)(v / k));
    }
}

// listed tile-rows' flags back to 0 (entries of segment 0 stand for the row)
__global__ void unflag_kernel(const Frontier f, int32_t* flag) {
    const int32_t cntl = *f.count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cntl; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ent = f.list[i];
        if ((ent & 0xFFFFFFFF) == 0) flag[ent >> 32] = 0;
    }
}

// after a round: the consumed frontier's bits are cleared (it is the next
// round's empty side) and the new list's flags reset
template <int K>
__global__ void colour_epilogue_kernel(Frontier cur, Frontier nxt, int32_t* flag, const int32_t* gate) {
    if (gate_closed(gate)) return;
    const int32_t nc = *reinterpret_cast<volatile int32_t*>(cur.count);
    const int32_t nn = *reinterpret_cast<volatile int32_t*>(nxt.count);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc || i < nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nc) {
            const int64_t ent = cur.list[i];
            if ((ent & 0xFFFFFFFF) == 0) clear_seg<K>(cur.act, (int32_t)(ent >> 32));
        }
        if (i < nn) {
            const int64_t ent = nxt.list[i];
            if ((ent & 0xFFFFFFFF) == 0) flag[ent >> 32] = 0;
        }
    }
}

// the next round reads nxt; its own next list starts empty; stop when empty
__global__ void colour_advance_kernel(int32_t* cur_count, const int32_t* next_count, int32_t* active, int32_t* level) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *active) {
        *cur_count = 0;
        *active = *next_count > 0 ? 1 : 0;
        *level += 1;
    }
}

struct RoundState {
    uint64_t* key = nullptr;
    uint64_t* mx = nullptr;
    uint32_t* undecided = nullptr;
    uint32_t* joined = nullptr;
    uint32_t* nb = nullptr;
    int32_t* flags = nullptr;  // active, found, round, bad
};

// One allocation: keys and maxima (8-byte), three bitsets, four flags.
b2sr_status setup(b2sr_matrix* h, const float* prio, int32_t* out, int32_t init, DevBuf& buf, RoundState* st,
                  cudaStream_t s) {
    const int32_t n = h->n;
    const int64_t words = ceil_div(n, 32);
    const size_t kb = round_up((size_t)n * 8, 256), bb = round_up((size_t)words * 4, 256);
    B2SR_TRY(buf.alloc(2 * kb + 3 * bb + 256));
    char* p = buf.as<char>();
    st->key = reinterpret_cast<uint64_t*>(p);
    st->mx = reinterpret_cast<uint64_t*>(p + kb);
    st->undecided = reinterpret_cast<uint32_t*>(p + 2 * kb);
    st->joined = reinterpret_cast<uint32_t*>(p + 2 * kb + bb);
    st->nb = reinterpret_cast<uint32_t*>(p + 2 * kb + 2 * bb);
    st->flags = reinterpret_cast<int32_t*>(p + 2 * kb + 3 * bb);
    const int32_t f0[4] = {1, 0, 0, 0};
    B2SR_CUDA_TRY(cudaMemcpyAsync(st->flags, f0, sizeof(f0), cudaMemcpyHostToDevice, s));
    keys_init_kernel<<<grid_for(words), 256, 0, s>>>(prio, n, st->key, st->undecided, words, out, init,
                                                     st->flags + 3);
    B2SR_LAUNCH_CHECK("keys_init_kernel");
    HostFlag hf;
    int32_t bad = 0;
    B2SR_TRY(read_flag(st->flags + 3, hf, s, &bad));
    if (bad) return fail(B2SR_ERR_INVALID_ARG, "NaN priority");
    return B2SR_OK;
}

}  // namespace

b2sr_status mis(b2sr_matrix* h, const float* prio, int32_t* in_set, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    if (n == 0) return B2SR_OK;
    const int64_t words = ceil_div(n, 32);
    DevBuf buf(s);
    RoundState st;
    B2SR_TRY(setup(h, prio, in_set, 0, buf, &st, s));
    int32_t* active = st.flags;
    int32_t* found = st.flags + 1;
    int32_t* round = st.flags + 2;
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n;
    int64_t rounds = 0;
    return run_captured(s, 4, cap, active,
                        [&](cudaStream_t cs, int) -> b2sr_status {
                            B2SR_TRY(spmv_maxkey_dispatch(h, st.key, st.mx, st.undecided, 0, cs, active));
                            mis_select_kernel<<<grid_for(words), 256, 0, cs>>>(st.key, st.mx, st.undecided, st.joined,
                                                                               in_set, words, active);
                            B2SR_LAUNCH_CHECK("mis_select_kernel");
                            B2SR_TRY(spmv_dispatch(h, B2SR_BOOL_OR_AND, B2SR_VEC_BITS, st.joined, B2SR_VEC_BITS,
                                                   st.nb, st.undecided, 0, nullptr, cs, active));
                            B2SR_CUDA_TRY(cudaMemsetAsync(found, 0, sizeof(int32_t), cs));
                            mis_remove_kernel<<<grid_for(words), 256, 0, cs>>>(st.key, st.undecided, st.joined, st.nb,
                                                                               words, active, found);
                            B2SR_LAUNCH_CHECK("mis_remove_kernel");
                            rounds_advance_kernel<<<1, 32, 0, cs>>>(active, found, round);
                            B2SR_LAUNCH_CHECK("rounds_advance_kernel");
                            return B2SR_OK;
                        },
                        &rounds);
}

static b2sr_status color_rounds(b2sr_matrix* h, const float* prio, int32_t* colors, int max_iters, cudaStream_t s) {
    const int32_t n = h->n;
    if (n == 0) return B2SR_OK;
    const int64_t words = ceil_div(n, 32);
    DevBuf buf(s);
    RoundState st;
    B2SR_TRY(setup(h, prio, colors, -1, buf, &st, s));
    int32_t* active = st.flags;
    int32_t* found = st.flags + 1;
    int32_t* round = st.flags + 2;
    const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n;
    int64_t rounds = 0;
    return run_captured(s, 8, cap, active,
                        [&](cudaStream_t cs, int) -> b2sr_status {
                            B2SR_TRY(spmv_maxkey_dispatch(h, st.key, st.mx, st.undecided, 0, cs, active));
                            B2SR_CUDA_TRY(cudaMemsetAsync(found, 0, sizeof(int32_t), cs));
                            color_select_kernel<<<grid_for(words), 256, 0, cs>>>(st.key, st.mx, st.undecided, colors,
                                                                                 words, round, active, found);
                            B2SR_LAUNCH_CHECK("color_select_kernel");
                            rounds_advance_kernel<<<1, 32, 0, cs>>>(active, found, round);
                            B2SR_LAUNCH_CHECK("rounds_advance_kernel");
                            return B2SR_OK;
                        },
                        &rounds);
}

static b2sr_status color_push(b2sr_matrix* h, const float* prio, int32_t* colors, int max_iters, cudaStream_t s) {
    const int32_t n = h->n, ntr = h->ntr;
    const int64_t words = ceil_div(n, 32);
    const int64_t segs = (int64_t)ntr + h->T / kSeg + 1;  // bound on the segments of all tile-rows
    const size_t kb = round_up((size_t)n * 8, 256), cb = round_up((size_t)n * 4, 256);
    const size_t bb = round_up((size_t)(words + 1) * 4, 256), lb = round_up((size_t)segs * 8, 256);
    const size_t fb = round_up((size_t)ntr * 4 + 4, 256);
    DevBuf buf(s);
    const size_t total = kb + cb + 3 * bb + 3 * lb + fb + 256;
    B2SR_TRY(buf.alloc(total));
    char* p = buf.as<char>();
    B2SR_CUDA_TRY(cudaMemsetAsync(p, 0, total, s));
    uint64_t* key = reinterpret_cast<uint64_t*>(p);
    int32_t* cnt = reinterpret_cast<int32_t*>(p + kb);
    uint32_t* all = reinterpret_cast<uint32_t*>(p + kb + cb);
    char* q = p + kb + cb + bb;
    int32_t* ctl = reinterpret_cast<int32_t*>(q + 2 * bb + 3 * lb + fb);  // counts A, B, C; active; level; bad
    Frontier A{reinterpret_cast<uint32_t*>(q), reinterpret_cast<int64_t*>(q + 2 * bb), ctl};
    Frontier Bf{reinterpret_cast<uint32_t*>(q + bb), reinterpret_cast<int64_t*>(q + 2 * bb + lb), ctl + 1};
    Frontier All{all, reinterpret_cast<int64_t*>(q + 2 * bb + 2 * lb), ctl + 2};
    int32_t* flag = reinterpret_cast<int32_t*>(q + 2 * bb + 3 * lb);
    int32_t* active = ctl + 3;
    int32_t* level = ctl + 4;
    int32_t* bad = ctl + 5;
    keys_init_kernel<<<grid_for(words), 256, 0, s>>>(prio, n, key, all, words, colors, -1, bad);
    B2SR_LAUNCH_CHECK("keys_init_kernel");
    HostFlag hf;
    int32_t got = 0;
    B2SR_TRY(read_flag(bad, hf, s, &got));
    if (got) return fail(B2SR_ERR_INVALID_ARG, "NaN priority");
    const int push_grid = sm_count() * 4;  // warps stride over the listed segments
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        // counting pass: every vertex pushes once
        list_all_rows_kernel<<<grid_for(ntr), 256, 0, s>>>(h->rowptr, ntr, All);
        B2SR_LAUNCH_CHECK("list_all_rows_kernel");
        colour_push_kernel<K, true><<<push_grid, 256, 0, s>>>(h->rowptr, h->colind, h->tiles, key, cnt, colors, All,
                                                               All, flag, level, nullptr);
        B2SR_LAUNCH_CHECK("colour_push_kernel");
        colour_seed_kernel<<<grid_for(n), 256, 0, s>>>(h->rowptr, cnt, n, h->k, colors, A, flag);
        B2SR_LAUNCH_CHECK("colour_seed_kernel");
        unflag_kernel<<<grid_for(segs), 256, 0, s>>>(A, flag);
        B2SR_LAUNCH_CHECK("unflag_kernel");
        const int32_t one = 1;
        B2SR_CUDA_TRY(cudaMemcpyAsync(active, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        const int64_t cap = max_iters > 0 ? max_iters : (int64_t)n;
        int64_t rounds = 0;
        return run_captured(s, 16, cap, active,
                            [&](cudaStream_t cs, int r) -> b2sr_status {
                                const Frontier& cur = (r & 1) ? Bf : A;
                                const Frontier& nxt = (r & 1) ? A : Bf;
                                colour_push_kernel<K, false><<<push_grid, 256, 0, cs>>>(
                                    h->rowptr, h->colind, h->tiles, key, cnt, colors, cur, nxt, flag, level, active);
                                B2SR_LAUNCH_CHECK("colour_push_kernel");
                                colour_epilogue_kernel<K><<<grid_for(segs), 256, 0, cs>>>(cur, nxt, flag, active);
                                B2SR_LAUNCH_CHECK("colour_epilogue_kernel");
                                colour_advance_kernel<<<1, 32, 0, cs>>>(cur.count, nxt.count, active, level);
                                B2SR_LAUNCH_CHECK("colour_advance_kernel");
                                return B2SR_OK;
                            },
                            &rounds);
    });
}

b2sr_status color(b2sr_matrix* h, const float* prio, int32_t* colors, int method, int max_iters, cudaStream_t s) {
    if (h->n == 0) return B2SR_OK;
    if (method == B2SR_COLOR_MAX_TIMES) return color_rounds(h, prio, colors, max_iters, s);
    return color_push(h, prio, colors, max_iters, s);
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_mis(b2sr_handle h, const float* priority, int32_t* in_set, int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!priority || !in_set)) return fail(B2SR_ERR_INVALID_ARG, "priority or in_set is NULL");
    return mis(h, priority, in_set, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_color(b2sr_handle h, const float* priority, int32_t* colors, b2sr_color_method method,
                                  int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!priority || !colors)) return fail(B2SR_ERR_INVALID_ARG, "priority or colors is NULL");
    if (method < B2SR_COLOR_AUTO || method > B2SR_COLOR_PUSH) return fail(B2SR_ERR_INVALID_ARG, "bad method");
    return color(h, priority, colors, (int)method, max_iters, to_stream(stream));
}
