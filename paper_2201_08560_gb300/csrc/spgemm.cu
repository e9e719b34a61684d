// B2SR SpGEMM: bmm_bin_bin_sum_masked (Table 3, Listing 2; the fused-sum
// triangle-counting kernel of Sec. V) and the Boolean product C = A (x) B.
//
// Masked count: each warp takes a run of consecutive mask tiles (so their
// tile-rows come from one search, then a walk of the row pointers); for a mask
// tile (I, J) the tile-column lists of A's tile-row I and B's tile-row J are
// intersected (binary search of the shorter list's entries in the longer one,
// 32 lanes at a time); every common K adds
//   sum over bits (r, c) of M_IJ of popc(A_IK[r] & B_JK[c]),
// i.e. Listing 2's AND-popc of two bit-rows, restricted to the mask.  Lanes
// accumulate in registers, a warp sums with shuffles and one 64-bit atomic
// per warp joins the global count (integer, so the order does not matter).
//
// Boolean product: expand every tile product A_IK (x) B_KJ, whose row r is
// the OR of B_KJ's rows selected by the bits of A_IK[r]; sort the non-zero
// products by (I, J) with the library's radix sort; OR equal keys into the
// output tiles.
#include <algorithm>

#include "b2sr_internal.cuh"

namespace b2sr {

template <int K>
__device__ __forceinline__ uint32_t gword(const uint8_t* __restrict__ tiles, int64_t t, int r) {
    if (K == 32) return __ldg(reinterpret_cast<const uint32_t*>(tiles) + t * 32 + r);
    if (K == 16) return __ldg(reinterpret_cast<const uint16_t*>(tiles) + t * 16 + r);
    return __ldg(tiles + t * K + r);
}

// a k <= 8 tile as one word: byte r is row r
template <int K>
__device__ __forceinline__ uint64_t tile_word64(const uint8_t* __restrict__ tiles, int64_t t) {
    if (K == 8) return __ldg(reinterpret_cast<const unsigned long long*>(tiles) + t);
    return __ldg(reinterpret_cast<const uint32_t*>(tiles) + t);
}

// Tile positions fit int32 (a handle holds fewer than 2^31 tiles), which keeps
// the searches' arithmetic 32-bit.
__device__ __forceinline__ int32_t lower_bound_i32(const int32_t* __restrict__ a, int32_t lo, int32_t hi, int32_t v) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct MatView {
    const int32_t* rowptr;
    const int32_t* colind;
    const uint8_t* tiles;
    int64_t T;
    int32_t ntr;
};

template <int K>
__global__ void masked_count_kernel(MatView A, MatView B, MatView M, unsigned long long* __restrict__ out,
                                    unsigned long long* __restrict__ pairs) {
    const int lane = (int)lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0, npairs = 0;
    // each warp takes a run of consecutive mask tiles: their tile-row is found
    // once by a binary search and then advanced as the run crosses rows
    const int64_t per = (M.T + nw - 1) / nw;
    const int64_t t0 = gw * per, t1 = min(M.T, t0 + per);
    int32_t I = 0;
    if (t0 < t1) {
        int32_t lo = 0, hi = M.ntr - 1;  // largest I with M.rowptr[I] <= t0
        while (lo < hi) {
            int32_t mid = lo + (hi - lo + 1) / 2;
            if ((int64_t)__ldg(M.rowptr + mid) <= t0) lo = mid; else hi = mid - 1;
        }
        I = lo;
    }
    int64_t row_end = t0 < t1 ? __ldg(M.rowptr + I + 1) : 0;
    for (int64_t mt = t0; mt < t1; ++mt) {
        while (mt >= row_end) row_end = __ldg(M.rowptr + (++I) + 1);
        const int32_t J = __ldg(M.colind + mt);
        // k <= 8: a tile is one 32/64-bit word whose bytes are its rows, so a
        // row is picked by a shift; larger tiles keep their rows in registers
        constexpr int MR = K <= 8 ? 1 : K;
        uint32_t mrow[MR];
        uint64_t mw = 0;
        (void)mrow;
        if constexpr (K <= 8) {
            mw = tile_word64<K>(M.tiles, mt);
        } else {
#pragma unroll
            for (int r = 0; r < K; ++r) mrow[r] = gword<K>(M.tiles, mt, r);
        }
        const int32_t a0 = __ldg(A.rowptr + I), a1 = __ldg(A.rowptr + I + 1);
        const int32_t b0 = __ldg(B.rowptr + J), b1 = __ldg(B.rowptr + J + 1);
        const bool a_short = (a1 - a0) <= (b1 - b0);
        const int32_t s0 = a_short ? a0 : b0, s1 = a_short ? a1 : b1;
        const int32_t l0 = a_short ? b0 : a0, l1 = a_short ? b1 : a1;
        const int32_t* scol = a_short ? A.colind : B.colind;
        const int32_t* lcol = a_short ? B.colind : A.colind;
        int32_t from = l0;  // a lane's entries rise, so each search starts where its last one ended
        for (int32_t p = s0 + lane; p < s1; p += 32) {
            const int32_t Kc = __ldg(scol + p);
            const int32_t q = lower_bound_i32(lcol, from, l1, Kc);
            from = q;
            if (q >= l1 || __ldg(lcol + q) != Kc) continue;
            const int32_t ta = a_short ? p : q;  // tile A_IK
            const int32_t tb = a_short ? q : p;  // tile B_JK
            if constexpr (K <= 8) {
                const uint64_t aw = tile_word64<K>(A.tiles, ta), bw = tile_word64<K>(B.tiles, tb);
                uint64_t m = mw;
                while (m) {
                    const int bit = __ffsll((long long)m) - 1;  // row bit >> 3, column bit & 7
                    m &= m - 1;
                    acc += (unsigned long long)__popc((uint32_t)((aw >> (bit & ~7)) & (bw >> (8 * (bit & 7))) & 0xFFu));
                    ++npairs;
                }
            } else {
                uint32_t brow[K];
#pragma unroll
                for (int c = 0; c < K; ++c) brow[c] = gword<K>(B.tiles, tb, c);
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    uint32_t bits = mrow[r];
                    if (!bits) continue;
                    const uint32_t ar = gword<K>(A.tiles, ta, r);
                    while (bits) {
                        const int c = __ffs(bits) - 1;
                        bits &= bits - 1;
                        uint32_t bc = 0;
#pragma unroll
                        for (int q2 = 0; q2 < K; ++q2) bc = (q2 == c) ? brow[q2] : bc;
                        acc += (unsigned long long)__popc(ar & bc);
                        ++npairs;
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    }
    if (lane == 0) {
        if (acc) atomicAdd(out, acc);
        if (pairs && npairs) atomicAdd(pairs, npairs);
    }
}

// ---------------------------------------------------------------------------
// Boolean SpGEMM (expand, sort, merge)
// ---------------------------------------------------------------------------
__global__ void row_of_tiles_kernel(const int32_t* __restrict__ rowptr, int32_t ntr, int64_t T,
                                    int32_t* __restrict__ tilerow) {
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < ntr;
         I += (int64_t)gridDim.x * blockDim.x)
        for (int64_t t = rowptr[I]; t < rowptr[I + 1]; ++t) tilerow[t] = (int32_t)I;
}

__global__ void product_counts_kernel(const int32_t* __restrict__ a_colind, int64_t TA,
                                      const int32_t* __restrict__ b_rowptr, int32_t* __restrict__ cnt) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < TA;
         a += (int64_t)gridDim.x * blockDim.x) {
        int32_t Kc = a_colind[a];
        cnt[a] = b_rowptr[Kc + 1] - b_rowptr[Kc];
    }
}

template <int K>
__global__ void expand_kernel(const int32_t* __restrict__ a_tilerow, const int32_t* __restrict__ a_colind,
                              const uint8_t* __restrict__ a_tiles, int64_t TA, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ b_rowptr, const int32_t* __restrict__ b_colind,
                              const uint8_t* __restrict__ b_tiles, int64_t P, int sbits,
                              uint64_t* __restrict__ keys, uint32_t* __restrict__ idx,
                              uint32_t* __restrict__ prod) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        // A tile a with off[a] <= p < off[a+1]
        int64_t lo = 0, hi = TA - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const int64_t a = lo;
        const int32_t Kc = a_colind[a];
        const int64_t b = b_rowptr[Kc] + (p - off[a]);
        const int32_t I = a_tilerow[a];
        const int32_t J = b_colind[b];
        uint32_t any = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            uint32_t ar = gword<K>(a_tiles, a, r);
            uint32_t row = 0;
            while (ar) {
                int m = __ffs(ar) - 1;
                ar &= ar - 1;
                row |= gword<K>(b_tiles, b, m);
            }
            prod[p * K + r] = row;
            any |= row;
        }
        keys[p] = any ? (((uint64_t)I << sbits) | (uint64_t)J) : ~0ull;
        idx[p] = (uint32_t)p;
    }
}

__global__ void spgemm_heads_kernel(const uint64_t* __restrict__ keys, int64_t N, int32_t* __restrict__ flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = (keys[e] != ~0ull && (e == 0 || keys[e] != keys[e - 1])) ? 1 : 0;
}

template <int K>
__global__ void spgemm_merge_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx,
                                    const int32_t* __restrict__ flag, const int64_t* __restrict__ tidx, int64_t N,
                                    const uint32_t* __restrict__ prod, int sbits, int32_t* __restrict__ c_colind,
                                    int32_t* __restrict__ c_tilerow, uint32_t* __restrict__ c_tiles32) {
    constexpr int WB = K <= 8 ? 1 : (K == 16 ? 2 : 4);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = keys[e];
        if (key == ~0ull) continue;
        int64_t t = tidx[e] + flag[e] - 1;  // tile of this run
        if (flag[e]) {
            c_colind[t] = (int32_t)(key & ((1ull << sbits) - 1ull));
            c_tilerow[t] = (int32_t)(key >> sbits);
        }
        const uint32_t* pr = prod + (int64_t)idx[e] * K;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            uint32_t v = pr[r];
            if (!v) continue;
            int64_t byte = (t * K + r) * WB;
            atomicOr(c_tiles32 + (byte >> 2), v << ((int)(byte & 3) * 8));
        }
    }
}

__global__ void build_rowptr_from_rows(const int32_t* __restrict__ tilerow, int64_t T, int32_t ntr,
                                       int32_t* __restrict__ rowptr) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t prev = t == 0 ? -1 : tilerow[t - 1];
        int32_t cur = t == T ? ntr : tilerow[t];
        for (int32_t R = prev + 1; R <= cur; ++R) rowptr[R] = (int32_t)t;
    }
}

static MatView view(const b2sr_matrix* h) { return MatView{h->rowptr, h->colind, h->tiles, h->T, h->ntr}; }

// The masked count; `pairs` (device int64, optional) receives the number of
// AND-popc word operations done (one per mask bit per common tile-column).
b2sr_status masked_count(const b2sr_matrix* A, const b2sr_matrix* B, const b2sr_matrix* M, int64_t* count,
                         cudaStream_t s, int64_t* pairs) {
    B2SR_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int64_t), s));
    if (pairs) B2SR_CUDA_TRY(cudaMemsetAsync(pairs, 0, sizeof(int64_t), s));
    if (M->T == 0) return B2SR_OK;
    auto* out = reinterpret_cast<unsigned long long*>(count);
    auto* prs = reinterpret_cast<unsigned long long*>(pairs);
    const double bytes = 3.0 * (4.0 * ((double)A->ntr + 1.0)) + ((double)A->T + B->T + M->T) * (4.0 + tile_bytes(A->k));
    return with_tile(A->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        // runs of eight mask tiles a warp; the blocks are scheduled as SMs free
        // up, which balances runs of long (hub) rows against short ones
        const int64_t warps = ceil_div(M->T, 8);
        const int grid = (int)std::max<int64_t>(1, ceil_div(warps, 8));
        void* tok = timing_begin(s);
        masked_count_kernel<K><<<grid, 256, 0, s>>>(view(A), view(B), view(M), out, prs);
        timing_end(tok, "spgemm_masked", bytes, s);
        B2SR_LAUNCH_CHECK("masked_count_kernel");
        return B2SR_OK;
    });
}

b2sr_status spgemm_bool(const b2sr_matrix* A, const b2sr_matrix* B, cudaStream_t s, b2sr_matrix** out) {
    const int k = A->k;
    const int32_t ntr = A->ntr;
    const int sbits = bits_for((int64_t)ntr + 1);  // all-ones key stays invalid
    int64_t P = 0;
    DevBuf a_tilerow(s), cnt(s), off(s);
    if (A->T > 0) {
        B2SR_TRY(a_tilerow.alloc(A->T * sizeof(int32_t)));
        B2SR_TRY(cnt.alloc((A->T + 1) * sizeof(int32_t)));
        B2SR_TRY(off.alloc((A->T + 1) * sizeof(int64_t)));
        row_of_tiles_kernel<<<grid_wide(ntr), 256, 0, s>>>(A->rowptr, ntr, A->T, a_tilerow.as<int32_t>());
        B2SR_LAUNCH_CHECK("row_of_tiles_kernel");
        product_counts_kernel<<<grid_wide(A->T), 256, 0, s>>>(A->colind, A->T, B->rowptr, cnt.as<int32_t>());
        B2SR_LAUNCH_CHECK("product_counts_kernel");
        B2SR_CUDA_TRY(cudaMemsetAsync(cnt.as<int32_t>() + A->T, 0, sizeof(int32_t), s));
        B2SR_TRY(exclusive_scan_i32_to_i64(cnt.as<int32_t>(), off.as<int64_t>(), A->T + 1, s));
        B2SR_CUDA_TRY(cudaMemcpyAsync(&P, off.as<int64_t>() + A->T, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (P >= (int64_t(1) << 32)) return fail(B2SR_ERR_OOM, "Boolean SpGEMM: too many tile products");
    DevBuf keys(s), ktmp(s), idx(s), itmp(s), prod(s), flag(s), tidx(s);
    uint64_t* skeys = nullptr;
    uint32_t* sidx = nullptr;
    int64_t TC = 0;
    if (P > 0) {
        B2SR_TRY(keys.alloc(P * sizeof(uint64_t)));
        B2SR_TRY(ktmp.alloc(P * sizeof(uint64_t)));
        B2SR_TRY(idx.alloc(P * sizeof(uint32_t)));
        B2SR_TRY(itmp.alloc(P * sizeof(uint32_t)));
        B2SR_TRY(prod.alloc(P * k * sizeof(uint32_t)));
        B2SR_TRY(with_tile(k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            expand_kernel<K><<<grid_wide(P), 256, 0, s>>>(a_tilerow.as<int32_t>(), A->colind, A->tiles, A->T,
                                                         off.as<int64_t>(), B->rowptr, B->colind, B->tiles, P,
                                                         sbits, keys.as<uint64_t>(), idx.as<uint32_t>(),
                                                         prod.as<uint32_t>());
            B2SR_LAUNCH_CHECK("expand_kernel");
            return B2SR_OK;
        }));
        B2SR_TRY(radix_sort_u64_pairs(keys.as<uint64_t>(), ktmp.as<uint64_t>(), idx.as<uint32_t>(),
                                      itmp.as<uint32_t>(), P, 0, 2 * sbits, s, &skeys, &sidx));
        B2SR_TRY(flag.alloc(P * sizeof(int32_t)));
        B2SR_TRY(tidx.alloc(P * sizeof(int64_t)));
        spgemm_heads_kernel<<<grid_wide(P), 256, 0, s>>>(skeys, P, flag.as<int32_t>());
        B2SR_LAUNCH_CHECK("spgemm_heads_kernel");
        B2SR_TRY(exclusive_scan_i32_to_i64(flag.as<int32_t>(), tidx.as<int64_t>(), P, s));
        int64_t last = 0;
        int32_t lastf = 0;
        B2SR_CUDA_TRY(cudaMemcpyAsync(&last, tidx.as<int64_t>() + P - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaMemcpyAsync(&lastf, flag.as<int32_t>() + P - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        TC = last + lastf;
    }
    const int64_t cap = std::max<int64_t>(round_up(TC, kTilePad), kTilePad);
    int32_t* crp = nullptr;
    int32_t* cci = nullptr;
    uint8_t* ct = nullptr;
    auto release = [&](b2sr_status st) {
        dfree(crp, s); dfree(cci, s); dfree(ct, s);
        return st;
    };
    b2sr_status st = dalloc(&crp, (size_t)ntr + 1, s);
    if (st == B2SR_OK) st = dalloc(&cci, (size_t)cap, s);
    if (st == B2SR_OK) st = dalloc(&ct, (size_t)cap * tile_bytes(k), s);
    if (st != B2SR_OK) return release(st);
    cudaError_t e = cudaMemsetAsync(cci, 0, (size_t)cap * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ct, 0, (size_t)cap * tile_bytes(k), s);
    if (e != cudaSuccess) return release(cuda_fail(e, "memset spgemm output"));
    DevBuf ctilerow(s);
    st = ctilerow.alloc(std::max<int64_t>(TC, 1) * sizeof(int32_t));
    if (st != B2SR_OK) return release(st);
    if (P > 0) {
        st = with_tile(k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            spgemm_merge_kernel<K><<<grid_wide(P), 256, 0, s>>>(skeys, sidx, flag.as<int32_t>(), tidx.as<int64_t>(), P,
                                                               prod.as<uint32_t>(), sbits, cci, ctilerow.as<int32_t>(),
                                                               reinterpret_cast<uint32_t*>(ct));
            B2SR_LAUNCH_CHECK("spgemm_merge_kernel");
            return B2SR_OK;
        });
        if (st != B2SR_OK) return release(st);
    }
    build_rowptr_from_rows<<<grid_wide(TC + 1), 256, 0, s>>>(ctilerow.as<int32_t>(), TC, ntr, crp);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return release(cuda_fail(e, "build_rowptr_from_rows"));
    return new_handle_from_tiles(A->n, k, TC, crp, cci, ct, cap, s, out);
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_spgemm_masked_count(b2sr_handle A, b2sr_handle B, b2sr_handle M, int64_t* count,
                                                void* stream) {
    clear_error();
    B2SR_TRY(check_handle(A));
    B2SR_TRY(check_handle(B));
    B2SR_TRY(check_handle(M));
    if (!count) return fail(B2SR_ERR_INVALID_ARG, "count is NULL");
    if (A->n != B->n || A->n != M->n || A->k != B->k || A->k != M->k)
        return fail(B2SR_ERR_INVALID_ARG, "A, B and M need the same n and tile_dim");
    return masked_count(A, B, M, count, to_stream(stream), nullptr);
}

extern "C" b2sr_status b2sr_spgemm_masked_count_work(b2sr_handle A, b2sr_handle B, b2sr_handle M, int64_t* count,
                                                     int64_t* pairs, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(A));
    B2SR_TRY(check_handle(B));
    B2SR_TRY(check_handle(M));
    if (!count || !pairs) return fail(B2SR_ERR_INVALID_ARG, "count or pairs is NULL");
    if (A->n != B->n || A->n != M->n || A->k != B->k || A->k != M->k)
        return fail(B2SR_ERR_INVALID_ARG, "A, B and M need the same n and tile_dim");
    return masked_count(A, B, M, count, to_stream(stream), pairs);
}

extern "C" b2sr_status b2sr_spgemm_bool(b2sr_handle A, b2sr_handle B, void* stream, b2sr_handle* C) {
    clear_error();
    if (!C) return fail(B2SR_ERR_INVALID_ARG, "C is NULL");
    *C = nullptr;
    B2SR_TRY(check_handle(A));
    B2SR_TRY(check_handle(B));
    if (A->n != B->n || A->k != B->k) return fail(B2SR_ERR_INVALID_ARG, "A and B need the same n and tile_dim");
    b2sr_matrix* out = nullptr;
    B2SR_TRY(spgemm_bool(A, B, to_stream(stream), &out));
    *C = out;
    return B2SR_OK;
}
