// B2SR of the transpose (Sec. III-A: the tile index is transposed by taking
// it from CSR to CSC order; Sec. III-B: the tiles themselves need the other
// packing, i.e. each k x k bit tile transposed).  The result is an ordinary
// handle of A^T: vxm (y^T = x^T A) is an SpMV on it, and the push drivers
// (b2sr_sssp_push, b2sr_bfs_diropt) take it as their transpose on directed
// graphs.
//
// Steps: the tile-row of every tile (a binary search of TileRowPtr), keys
// (tile-col, tile-row) sorted with the tile's index as payload (the library's
// own radix sort), the new TileRowPtr from the sorted keys' heads, and every
// tile copied to its new slot with its bits transposed.
#include <algorithm>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "tile_bits.cuh"

namespace b2sr {

namespace {

// key = tile-col << rbits | tile-row, payload = the tile's index
__global__ void tr_keys_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind, int32_t ntr,
                               int64_t T, int rbits, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = ntr;  // the last J with rowptr[J] <= t
        while (hi - lo > 1) {
            const int32_t mid = lo + (hi - lo) / 2;
            if (__ldg(rowptr + mid) <= t) lo = mid;
            else hi = mid;
        }
        keys[t] = ((uint64_t)(uint32_t)__ldg(colind + t) << rbits) | (uint32_t)lo;
        vals[t] = (uint32_t)t;
    }
}

// TileRowPtr of A^T: rowptr[I] = the first sorted position whose tile-col is
// >= I (every I in (previous col, this col] starts here), rowptr[ntr] = T
__global__ void tr_rowptr_kernel(const uint64_t* __restrict__ keys, int64_t T, int32_t ntr, int rbits,
                                 int32_t* __restrict__ rowptr) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= T; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = p == 0 ? -1 : (int64_t)(keys[p - 1] >> rbits);
        const int64_t cur = p == T ? (int64_t)ntr : (int64_t)(keys[p] >> rbits);
        for (int64_t I = prev + 1; I <= cur; ++I) rowptr[I] = (int32_t)p;
    }
}

// The k x k bit matrix held as k row words (bit c of row r = column c) is
// transposed in place by swapping off-diagonal blocks of halving size (j =
// k/2, ..., 1): within every 2j x 2j block, the upper-right j x j block
// (rows r with bit j clear, columns with bit j set) trades places with the
// lower-left one.
template <int K>
__device__ __forceinline__ void transpose_bits(uint32_t (&a)[K]) {
#pragma unroll
    for (int j = K / 2; j >= 1; j >>= 1) {
        // columns c with (c & j) == 0
        const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                         : j == 2 ? 0x33333333u : 0x55555555u;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            if (r & j) continue;
            const uint32_t t = ((a[r] >> j) ^ a[r + j]) & m;
            a[r + j] ^= t;
            a[r] ^= t << j;
        }
    }
}

template <int K>
__global__ void tr_fill_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t T,
                               int rbits, const uint8_t* __restrict__ tiles, int32_t* __restrict__ colind_t,
                               uint8_t* __restrict__ tiles_t) {
    constexpr int TB = K * (K <= 8 ? 1 : K / 8);
    constexpr int TW = (TB + 3) / 4;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < T; p += (int64_t)gridDim.x * blockDim.x) {
        colind_t[p] = (int32_t)(keys[p] & (((uint64_t)1 << rbits) - 1));
        const uint32_t* src = reinterpret_cast<const uint32_t*>(tiles + (int64_t)vals[p] * TB);
        uint32_t w[TW];
#pragma unroll
        for (int q = 0; q < TW; ++q) w[q] = __ldg(src + q);
        uint32_t a[K];
#pragma unroll
        for (int r = 0; r < K; ++r) a[r] = tile_row<K>(w, r);
        transpose_bits<K>(a);
        uint32_t o[TW];
#pragma unroll
        for (int q = 0; q < TW; ++q) o[q] = 0u;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            if (K == 32) o[r] = a[r];
            else if (K == 16) o[r >> 1] |= a[r] << (16 * (r & 1));
            else o[r >> 2] |= a[r] << (8 * (r & 3));
        }
        uint32_t* dst = reinterpret_cast<uint32_t*>(tiles_t + p * TB);
#pragma unroll
        for (int q = 0; q < TW; ++q) dst[q] = o[q];
    }
}

}  // namespace

b2sr_status transpose(const b2sr_matrix* h, cudaStream_t s, b2sr_matrix** out) {
    const int k = h->k;
    const int32_t ntr = h->ntr;
    const int64_t T = h->T;
    const int64_t cap = std::max<int64_t>(round_up(T, kTilePad), kTilePad);
    const int rbits = bits_for(std::max<int32_t>(ntr, 2));
    int32_t* trp = nullptr;
    int32_t* tci = nullptr;
    uint8_t* tt = nullptr;
    auto release = [&](b2sr_status st) {
        dfree(trp, s); dfree(tci, s); dfree(tt, s);
        return st;
    };
    b2sr_status st = dalloc(&trp, (size_t)ntr + 1, s);
    if (st == B2SR_OK) st = dalloc(&tci, (size_t)cap, s);
    if (st == B2SR_OK) st = dalloc(&tt, (size_t)cap * tile_bytes(k), s);
    if (st != B2SR_OK) return release(st);
    cudaError_t e = cudaMemsetAsync(tci, 0, (size_t)cap * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tt, 0, (size_t)cap * tile_bytes(k), s);
    if (e != cudaSuccess) return release(cuda_fail(e, "memset transpose"));
    if (T == 0) {
        st = fill_i32(trp, 0, (int64_t)ntr + 1, s);
    } else {
        DevBuf kv(s);
        const size_t kb = round_up((size_t)T * 8, 256), vb = round_up((size_t)T * 4, 256);
        st = kv.alloc(2 * kb + 2 * vb);
        if (st != B2SR_OK) return release(st);
        uint64_t* keys = kv.as<uint64_t>();
        uint64_t* ktmp = reinterpret_cast<uint64_t*>(kv.as<char>() + kb);
        uint32_t* vals = reinterpret_cast<uint32_t*>(kv.as<char>() + 2 * kb);
        uint32_t* vtmp = reinterpret_cast<uint32_t*>(kv.as<char>() + 2 * kb + vb);
        tr_keys_kernel<<<grid_for(T), 256, 0, s>>>(h->rowptr, h->colind, ntr, T, rbits, keys, vals);
        if ((e = cudaGetLastError()) != cudaSuccess) return release(cuda_fail(e, "tr_keys_kernel"));
        note_launches(1);
        uint64_t* ks = nullptr;
        uint32_t* vs = nullptr;
        st = radix_sort_u64_pairs(keys, ktmp, vals, vtmp, T, 0, 2 * rbits, s, &ks, &vs);
        if (st != B2SR_OK) return release(st);
        tr_rowptr_kernel<<<grid_for(T + 1), 256, 0, s>>>(ks, T, ntr, rbits, trp);
        if ((e = cudaGetLastError()) != cudaSuccess) return release(cuda_fail(e, "tr_rowptr_kernel"));
        note_launches(1);
        st = with_tile(k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            tr_fill_kernel<K><<<grid_for(T), 256, 0, s>>>(ks, vs, T, rbits, h->tiles, tci, tt);
            const cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) return cuda_fail(le, "tr_fill_kernel");
            note_launches(1);
            return B2SR_OK;
        });
    }
    if (st != B2SR_OK) return release(st);
    // the sort's buffers are released (stream-ordered) before the handle is built
    return new_handle_from_tiles(h->n, k, T, trp, tci, tt, cap, s, out);
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_transpose(b2sr_handle h, void* stream, b2sr_handle* out) {
    clear_error();
    if (!out) return fail(B2SR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    B2SR_TRY(check_handle(h));
    if (h->T > (int64_t)UINT32_MAX) return fail(B2SR_ERR_OOM, "more than 2^32 tiles");
    return transpose(h, to_stream(stream), out);
}
