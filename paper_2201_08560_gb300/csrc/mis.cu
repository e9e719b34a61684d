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
#include <algorithm>

#include "b2sr_internal.cuh"
#include "captured.cuh"

namespace b2sr {
b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s,
                          const int32_t* gate);
b2sr_status spmv_maxkey_dispatch(b2sr_matrix* h, const uint64_t* x, uint64_t* y, const uint32_t* mask, int comp,
                                 cudaStream_t s, const int32_t* gate);

namespace {

int grid_for(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)sm_count() * 8));
}

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

b2sr_status color(b2sr_matrix* h, const float* prio, int32_t* colors, int max_iters, cudaStream_t s) {
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

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_mis(b2sr_handle h, const float* priority, int32_t* in_set, int max_iters, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!priority || !in_set)) return fail(B2SR_ERR_INVALID_ARG, "priority or in_set is NULL");
    return mis(h, priority, in_set, max_iters, to_stream(stream));
}

extern "C" b2sr_status b2sr_color(b2sr_handle h, const float* priority, int32_t* colors, int max_iters,
                                  void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!priority || !colors)) return fail(B2SR_ERR_INVALID_ARG, "priority or colors is NULL");
    return color(h, priority, colors, max_iters, to_stream(stream));
}
