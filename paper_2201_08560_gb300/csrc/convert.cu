// CSR <-> B2SR conversion (Sec. III-A "Bit-tile Indexing System", Sec. III-B
// "Bit Packing", Table 1), the strictly-lower-triangle extraction used by
// triangle counting (Sec. V, TC), the weight side array, and the per-handle
// derived arrays (SpMV chunk schedule, set-bit offsets, column counts).
//
// Conversion: every entry (i, j) becomes the 64-bit key
//   (i/k) << (S+10) | (j/k) << 10 | ((j%k)*k + i%k)
// with S the bit width of a tile index.  Once the keys are in order, equal
// tiles are runs in (tile-row, tile-column) order, run heads become the tiles,
// and each entry ORs its bit into its tile.  When every CSR row is already in
// column order (the usual case) the k rows of a tile-row are k sorted runs and
// the keys are put in order by ranking each entry among its tile-row's rows
// (binary searches) and, at k = 16 and 32, merging groups of eight rows
// pairwise; otherwise a radix sort on the tile part orders them.  Both replace
// the paper's cusparseXcsr2bsrNnz / cusparseScsr2bsr + packing kernels
// (Sec. III-B) and give the same three arrays.
#include <algorithm>
#include <mutex>

#include "b2sr_internal.cuh"

namespace b2sr {

// ---------------------------------------------------------------------------
// input validation
// ---------------------------------------------------------------------------
__global__ void validate_csr_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ colind, int64_t nnz,
                                    int* __restrict__ bad) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz)) atomicOr(bad, 1);
    for (int64_t i = tid; i < n; i += stride)
        if (rowptr[i + 1] < rowptr[i]) atomicOr(bad, 2);
    for (int64_t e = tid; e < nnz; e += stride) {
        int32_t c = colind[e];
        if (c < 0 || c >= n) atomicOr(bad, 4);
    }
}

// Sets *bad (device) non-zero if the CSR is malformed; stream-ordered, no sync.
b2sr_status validate_csr_async(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz, int* bad,
                               cudaStream_t s) {
    validate_csr_kernel<<<grid_wide(std::max<int64_t>(n, nnz)), 256, 0, s>>>(n, rowptr, colind, nnz, bad);
    B2SR_LAUNCH_CHECK("validate_csr_kernel");
    return B2SR_OK;
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
constexpr int kKeyThreads = 256;

// largest r in [lo, hi] with rowptr[r] <= e
__device__ __forceinline__ int32_t row_of(const int32_t* __restrict__ rowptr, int32_t lo, int32_t hi,
                                          int64_t e) {
    while (lo < hi) {
        int32_t mid = lo + (hi - lo + 1) / 2;
        if ((int64_t)__ldg(rowptr + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t entry_key(int32_t i, int32_t j, int k, int sbits) {
    return ((uint64_t)(i / k) << (sbits + 10)) | ((uint64_t)(j / k) << 10) | (uint64_t)((j % k) * k + (i % k));
}

__global__ void __launch_bounds__(kKeyThreads) make_keys_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ colind,
                                                                int64_t nnz, int k, int sbits,
                                                                uint64_t* __restrict__ keys) {
    __shared__ int32_t range[2];
    int64_t b0 = (int64_t)blockIdx.x * kKeyThreads;
    if (b0 >= nnz) return;
    int64_t b1 = min(b0 + kKeyThreads, nnz) - 1;
    if (threadIdx.x == 0) range[0] = row_of(rowptr, 0, n - 1, b0);
    if (threadIdx.x == 1) range[1] = row_of(rowptr, 0, n - 1, b1);
    __syncthreads();
    int64_t e = b0 + threadIdx.x;
    if (e > b1) return;
    int32_t i = row_of(rowptr, range[0], range[1], e);
    keys[e] = entry_key(i, colind[e], k, sbits);
}

// Flags (bit 0 of *unsorted) a row whose columns decrease somewhere; repeated
// columns keep a row sorted.
__global__ void __launch_bounds__(kKeyThreads) sorted_rows_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ colind,
                                                                  int64_t nnz, int* __restrict__ unsorted) {
    __shared__ int32_t range[2];
    int64_t b0 = (int64_t)blockIdx.x * kKeyThreads;
    if (b0 >= nnz) return;
    int64_t b1 = min(b0 + kKeyThreads, nnz) - 1;
    if (threadIdx.x == 0) range[0] = row_of(rowptr, 0, n - 1, b0);
    if (threadIdx.x == 1) range[1] = row_of(rowptr, 0, n - 1, b1);
    __syncthreads();
    int64_t e = b0 + threadIdx.x;
    if (e > b1) return;
    int32_t i = row_of(rowptr, range[0], range[1], e);
    if (e > 0 && e > __ldg(rowptr + i) && __ldg(colind + e - 1) > __ldg(colind + e)) atomicOr(unsorted, 1);
}

// Entries of the same tile-row ahead of column j in row q: those with a
// smaller column, and also those with column j when `ties` (q is an earlier
// row).
__device__ __forceinline__ int64_t count_before(const int32_t* __restrict__ colind, int64_t lo, int64_t hi,
                                                int32_t j, bool ties) {
    const int64_t base = lo;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t x = __ldg(colind + mid);
        if (x < j || (ties && x == j)) lo = mid + 1; else hi = mid;
    }
    return lo - base;
}

// Sorted rows: writes every entry's key straight to its place in the order of
// its group of G rows (G divides k, groups start at multiples of G).  The
// place is the group's first CSR position, plus the entry's offset in its own
// row, plus the entries of the group's other rows that come before it in
// (column, row) order.
template <int G>
__global__ void __launch_bounds__(kKeyThreads) rank_keys_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ colind,
                                                                int64_t nnz, int k, int sbits,
                                                                uint64_t* __restrict__ keys) {
    __shared__ int32_t range[2];
    int64_t b0 = (int64_t)blockIdx.x * kKeyThreads;
    if (b0 >= nnz) return;
    int64_t b1 = min(b0 + kKeyThreads, nnz) - 1;
    if (threadIdx.x == 0) range[0] = row_of(rowptr, 0, n - 1, b0);
    if (threadIdx.x == 1) range[1] = row_of(rowptr, 0, n - 1, b1);
    __syncthreads();
    int64_t e = b0 + threadIdx.x;
    if (e > b1) return;
    const int32_t i = row_of(rowptr, range[0], range[1], e);
    const int32_t j = __ldg(colind + e);
    const int rg = i % G;
    const int32_t g0 = i - rg;
    int64_t dest = (int64_t)__ldg(rowptr + g0) + (e - (int64_t)__ldg(rowptr + i));
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const int32_t iq = g0 + q;
        if (q == rg || iq >= n) continue;
        dest += count_before(colind, __ldg(rowptr + iq), __ldg(rowptr + iq + 1), j, q < rg);
    }
    keys[dest] = entry_key(i, j, k, sbits);
}

// One pairwise merge of sorted runs of `run` rows inside every tile-row (the
// runs a sorted-row conversion leaves when k > 8): each key moves to its
// offset in its own run plus the partner run's keys ahead of it (the left
// run wins ties).
__global__ void merge_runs_kernel(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst, int64_t nnz,
                                  const int32_t* __restrict__ rowptr, int32_t n, int k, int run, int sbits) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = src[e];
        const int r = (int)(x & 1023u) % k;
        const int64_t rowL = (int64_t)(x >> (sbits + 10)) * k + (r & ~(2 * run - 1));
        const int64_t a0 = __ldg(rowptr + min(rowL, (int64_t)n));
        const int64_t m = __ldg(rowptr + min(rowL + run, (int64_t)n));
        const int64_t b1 = __ldg(rowptr + min(rowL + 2 * run, (int64_t)n));
        const bool right = (r & run) != 0;
        int64_t lo = right ? a0 : m, hi = right ? m : b1;
        const int64_t base = lo;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            uint64_t y = src[mid];
            if (y < x || (right && y == x)) lo = mid + 1; else hi = mid;
        }
        dst[a0 + (e - (right ? m : a0)) + (lo - base)] = x;
    }
}

__global__ void mark_heads_kernel(const uint64_t* __restrict__ keys, int64_t N, int32_t* __restrict__ flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = (e == 0 || (keys[e] >> 10) != (keys[e - 1] >> 10)) ? 1 : 0;
}

__global__ void fill_tiles_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ flag,
                                  const int64_t* __restrict__ tidx, int64_t N, int k, int sbits,
                                  int32_t* __restrict__ colind, int32_t* __restrict__ tilerow,
                                  uint32_t* __restrict__ tiles32) {
    const int wb = word_bytes(k);
    const uint64_t jmask = (1ull << sbits) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = keys[e];
        int64_t t = tidx[e] + flag[e] - 1;  // tile of this entry's run (tidx counts heads before e)
        int p = (int)(key & 1023u);
        if (flag[e]) {
            colind[t] = (int32_t)((key >> 10) & jmask);
            tilerow[t] = (int32_t)(key >> (sbits + 10));
        }
        int r = p % k, c = p / k;
        int64_t byte = (t * k + r) * wb + (c >> 3);
        atomicOr(tiles32 + (byte >> 2), 1u << ((int)(byte & 3) * 8 + (c & 7)));
    }
}

// rowptr[R] = first tile of tile-row R, for every R in [0, ntr]
__global__ void build_rowptr_kernel(const int32_t* __restrict__ tilerow, int64_t T, int32_t ntr,
                                    int32_t* __restrict__ rowptr) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t prev = t == 0 ? -1 : tilerow[t - 1];
        int32_t cur = t == T ? ntr : tilerow[t];
        for (int32_t R = prev + 1; R <= cur; ++R) rowptr[R] = (int32_t)t;
    }
}

// ---------------------------------------------------------------------------
// schedule: tile-row of the first tile of every SpMV chunk
// ---------------------------------------------------------------------------
__global__ void chunk_rows_kernel(const int32_t* __restrict__ rowptr, int32_t ntr, int64_t T, int64_t CT,
                                  int64_t nchunks, int32_t* __restrict__ chunk_row) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = min(c * CT, T - 1);
        chunk_row[c] = row_of(rowptr, 0, ntr - 1, t);
    }
}

// Tile-rows that span chunks: the row R that chunk c begins inside, when R
// started in an earlier chunk and ends in c.  kind[c] = 1 (at most
// kSplitShort chunks), 2 (more), 0 (none).
__global__ void split_kind_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ chunk_row,
                                  int64_t T, int64_t CT, int64_t nchunks, int32_t* __restrict__ kshort,
                                  int32_t* __restrict__ klong) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        int32_t ks = 0, kl = 0;
        if (c > 0) {
            const int64_t cs = c * CT, ce = min(cs + CT, T);
            const int32_t R = chunk_row[c];
            const int64_t rs = rowptr[R], re = rowptr[R + 1];
            if (rs < cs && re <= ce) {
                const int64_t np = c - rs / CT + 1;
                if (np <= kSplitShort) ks = 1; else kl = 1;
            }
        }
        kshort[c] = ks;
        klong[c] = kl;
    }
}

__global__ void split_fill_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ chunk_row,
                                  int64_t CT, int64_t nchunks, const int32_t* __restrict__ kshort,
                                  const int32_t* __restrict__ klong, const int64_t* __restrict__ pshort,
                                  const int64_t* __restrict__ plong, int64_t nshort, int32_t* __restrict__ split) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!kshort[c] && !klong[c]) continue;
        const int32_t R = chunk_row[c];
        const int64_t at = kshort[c] ? pshort[c] : nshort + plong[c];
        split[3 * at] = R;
        split[3 * at + 1] = (int32_t)(rowptr[R] / CT);
        split[3 * at + 2] = (int32_t)c;
    }
}

static b2sr_status build_split_list(b2sr_matrix* h, cudaStream_t s) {
    const int64_t CT = chunk_tiles(h->k);
    const int64_t nc = h->nchunks;
    DevBuf ks(s), kl(s), ps(s), pl(s);
    B2SR_TRY(ks.alloc((nc + 1) * sizeof(int32_t)));
    B2SR_TRY(kl.alloc((nc + 1) * sizeof(int32_t)));
    B2SR_TRY(ps.alloc((nc + 1) * sizeof(int64_t)));
    B2SR_TRY(pl.alloc((nc + 1) * sizeof(int64_t)));
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nc, 256), (int64_t)sm_count() * 8));
    split_kind_kernel<<<grid, 256, 0, s>>>(h->rowptr, h->chunk_row, h->T, CT, nc, ks.as<int32_t>(), kl.as<int32_t>());
    B2SR_LAUNCH_CHECK("split_kind_kernel");
    B2SR_CUDA_TRY(cudaMemsetAsync(ks.as<int32_t>() + nc, 0, sizeof(int32_t), s));
    B2SR_CUDA_TRY(cudaMemsetAsync(kl.as<int32_t>() + nc, 0, sizeof(int32_t), s));
    B2SR_TRY(exclusive_scan_i32_to_i64(ks.as<int32_t>(), ps.as<int64_t>(), nc + 1, s));
    B2SR_TRY(exclusive_scan_i32_to_i64(kl.as<int32_t>(), pl.as<int64_t>(), nc + 1, s));
    int64_t ns = 0, nl = 0;
    B2SR_CUDA_TRY(cudaMemcpyAsync(&ns, ps.as<int64_t>() + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(&nl, pl.as<int64_t>() + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    B2SR_TRY(dalloc(&h->split, (size_t)std::max<int64_t>(3 * (ns + nl), 3), s));
    split_fill_kernel<<<grid, 256, 0, s>>>(h->rowptr, h->chunk_row, CT, nc, ks.as<int32_t>(), kl.as<int32_t>(),
                                           ps.as<int64_t>(), pl.as<int64_t>(), ns, h->split);
    B2SR_LAUNCH_CHECK("split_fill_kernel");
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    h->nsplit_short = ns;
    h->nsplit_long = nl;
    return B2SR_OK;
}

b2sr_status build_schedule(b2sr_matrix* h, cudaStream_t s) {
    if (h->T == 0) {
        h->nchunks = 0;
        h->first_row = h->ntr;
        h->last_row = -1;
        return B2SR_OK;
    }
    int64_t CT = chunk_tiles(h->k);
    h->nchunks = ceil_div(h->T, CT);
    B2SR_TRY(dalloc(&h->chunk_row, h->nchunks + 1, s));
    int grid = (int)std::min<int64_t>(ceil_div(h->nchunks + 1, 256), (int64_t)sm_count() * 8);
    chunk_rows_kernel<<<grid, 256, 0, s>>>(h->rowptr, h->ntr, h->T, CT, h->nchunks, h->chunk_row);
    B2SR_LAUNCH_CHECK("chunk_rows_kernel");
    int32_t fr = 0, lr = 0;
    B2SR_CUDA_TRY(cudaMemcpyAsync(&fr, h->chunk_row, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(&lr, h->chunk_row + h->nchunks, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    h->first_row = fr;
    h->last_row = lr;
    return build_split_list(h, s);
}

b2sr_status new_handle_from_tiles(int32_t n, int k, int64_t T, int32_t* rowptr, int32_t* colind,
                                  uint8_t* tiles, int64_t cap, cudaStream_t s, b2sr_matrix** out) {
    b2sr_matrix* h = new b2sr_matrix();
    h->n = n;
    h->k = k;
    h->ntr = (int32_t)ceil_div(n, k);
    h->T = T;
    h->cap = cap;
    h->rowptr = rowptr;
    h->colind = colind;
    h->tiles = tiles;
    h->mtx = new std::mutex();
    cudaGetDevice(&h->device);
    auto cleanup = [&](b2sr_status st) {
        b2sr_destroy(h);
        return st;
    };
    // the SpMV and driver kernels index tiles with int32
    if (T >= (int64_t(1) << 31)) return cleanup(fail(B2SR_ERR_OOM, "more than 2^31 - 1 tiles"));
    DevBuf cnt(s);
    b2sr_status st = cnt.alloc(sizeof(int64_t));
    if (st != B2SR_OK) return cleanup(st);
    st = popcount_bytes(tiles, cap * tile_bytes(k), cnt.as<int64_t>(), s);
    if (st != B2SR_OK) return cleanup(st);
    int64_t nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, cnt.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "copy nnz"));
    st = build_schedule(h, s);  // synchronises s
    if (st != B2SR_OK) return cleanup(st);
    h->nnz = nnz;
    *out = h;
    return B2SR_OK;
}

// ---------------------------------------------------------------------------
// set-bit offsets and column counts (cached on the handle)
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ uint32_t tile_word(const uint8_t* __restrict__ tiles, int64_t t, int r) {
    if (K == 32) return __ldg(reinterpret_cast<const uint32_t*>(tiles) + t * 32 + r);
    if (K == 16) return __ldg(reinterpret_cast<const uint16_t*>(tiles) + t * 16 + r);
    return __ldg(tiles + t * K + r);
}

template <int K>
__global__ void tile_popc_kernel(const uint8_t* __restrict__ tiles, int64_t T, int32_t* __restrict__ cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) c += __popc(tile_word<K>(tiles, t, r));
        cnt[t] = c;
    }
}

__global__ void i64_to_i32_kernel(const int64_t* __restrict__ in, int64_t n, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

template <int K>
__global__ void col_count_kernel(const int32_t* __restrict__ colind, const uint8_t* __restrict__ tiles,
                                 int64_t T, int32_t n, int32_t* __restrict__ deg) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t J = colind[t];
        uint32_t cols = 0;
        int per[K];
#pragma unroll
        for (int c = 0; c < K; ++c) per[c] = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            uint32_t w = tile_word<K>(tiles, t, r);
            cols |= w;
#pragma unroll
            for (int c = 0; c < K; ++c) per[c] += (w >> c) & 1u;
        }
        while (cols) {
            int c = __ffs(cols) - 1;
            cols &= cols - 1;
            int v = 0;
#pragma unroll
            for (int q = 0; q < K; ++q) v = (q == c) ? per[q] : v;
            atomicAdd(deg + J * K + c, v);
        }
    }
}

b2sr_status ensure_voff(b2sr_matrix* h, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(h->mtx));
    if (h->voff) return B2SR_OK;
    int32_t* voff = nullptr;
    B2SR_TRY(dalloc(&voff, h->T + 1, s));
    DevBuf cnt(s), scan(s);
    b2sr_status st = cnt.alloc((h->T + 1) * sizeof(int32_t));
    if (st == B2SR_OK) st = scan.alloc((h->T + 1) * sizeof(int64_t));
    if (st == B2SR_OK) {
        st = with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            if (h->T > 0) tile_popc_kernel<K><<<grid_wide(h->T), 256, 0, s>>>(h->tiles, h->T, cnt.as<int32_t>());
            B2SR_LAUNCH_CHECK("tile_popc_kernel");
            return B2SR_OK;
        });
    }
    if (st == B2SR_OK) {
        cudaMemsetAsync(cnt.as<int32_t>() + h->T, 0, sizeof(int32_t), s);
        st = exclusive_scan_i32_to_i64(cnt.as<int32_t>(), scan.as<int64_t>(), h->T + 1, s);
    }
    if (st == B2SR_OK) {
        i64_to_i32_kernel<<<grid_wide(h->T + 1), 256, 0, s>>>(scan.as<int64_t>(), h->T + 1, voff);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "voff");
    }
    if (st != B2SR_OK) {
        dfree(voff, s);
        return st;
    }
    h->voff = voff;
    return B2SR_OK;
}

b2sr_status ensure_outdeg(b2sr_matrix* h, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(h->mtx));
    if (h->outdeg) return B2SR_OK;
    int32_t* deg = nullptr;
    B2SR_TRY(dalloc(&deg, (size_t)h->ntr * h->k, s));
    cudaError_t e = cudaMemsetAsync(deg, 0, (size_t)h->ntr * h->k * sizeof(int32_t), s);
    if (e != cudaSuccess) { dfree(deg, s); return cuda_fail(e, "memset outdeg"); }
    b2sr_status st = with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        if (h->T > 0) col_count_kernel<K><<<grid_wide(h->T), 256, 0, s>>>(h->colind, h->tiles, h->T, h->n, deg);
        B2SR_LAUNCH_CHECK("col_count_kernel");
        return B2SR_OK;
    });
    if (st == B2SR_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "outdeg");
    }
    if (st != B2SR_OK) { dfree(deg, s); return st; }
    h->outdeg = deg;
    return B2SR_OK;
}

// ---------------------------------------------------------------------------
// B2SR -> CSR
// ---------------------------------------------------------------------------
template <int K>
__global__ void row_nnz_kernel(const int32_t* __restrict__ trp, const uint8_t* __restrict__ tiles,
                               int32_t n, int32_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t I = i / K;
        int r = (int)(i % K);
        int c = 0;
        for (int64_t t = trp[I]; t < trp[I + 1]; ++t) c += __popc(tile_word<K>(tiles, t, r));
        cnt[i] = c;
    }
}

template <int K>
__global__ void row_fill_kernel(const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                const uint8_t* __restrict__ tiles, int32_t n,
                                const int64_t* __restrict__ off, int32_t* __restrict__ rowptr,
                                int32_t* __restrict__ colind) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x) {
        rowptr[i] = (int32_t)off[i];
        if (i == n || colind == nullptr) continue;
        int64_t I = i / K;
        int r = (int)(i % K);
        int64_t w = off[i];
        for (int64_t t = trp[I]; t < trp[I + 1]; ++t) {
            uint32_t bits = tile_word<K>(tiles, t, r);
            while (bits) {
                int c = __ffs(bits) - 1;
                bits &= bits - 1;
                colind[w++] = tci[t] * K + c;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// strictly lower triangle
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ uint32_t strict_lower_mask(int r) {  // columns c < r
    return r == 0 ? 0u : ((r >= 32) ? 0xffffffffu : ((1u << r) - 1u));
}

template <int K>
__global__ void lower_count_kernel(const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                   const uint8_t* __restrict__ tiles, int32_t ntr, int32_t* __restrict__ cnt) {
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < ntr;
         I += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        for (int64_t t = trp[I]; t < trp[I + 1]; ++t) {
            int32_t J = tci[t];
            if (J < I) { ++c; continue; }
            if (J > I) break;
            uint32_t any = 0;
#pragma unroll
            for (int r = 0; r < K; ++r) any |= tile_word<K>(tiles, t, r) & strict_lower_mask<K>(r);
            c += any ? 1 : 0;
        }
        cnt[I] = c;
    }
}

template <int K>
__global__ void lower_fill_kernel(const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                  const uint8_t* __restrict__ tiles, int32_t ntr,
                                  const int64_t* __restrict__ off, int32_t* __restrict__ lrp,
                                  int32_t* __restrict__ lci, uint8_t* __restrict__ ltiles) {
    constexpr int WB = K <= 8 ? 1 : (K == 16 ? 2 : 4);
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I <= ntr;
         I += (int64_t)gridDim.x * blockDim.x) {
        lrp[I] = (int32_t)off[I];
        if (I == ntr) continue;
        int64_t w = off[I];
        for (int64_t t = trp[I]; t < trp[I + 1]; ++t) {
            int32_t J = tci[t];
            if (J > I) break;
            uint32_t rows[K];
            uint32_t any = 0;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                uint32_t v = tile_word<K>(tiles, t, r);
                if (J == I) v &= strict_lower_mask<K>(r);
                rows[r] = v;
                any |= v;
            }
            if (!any) continue;
            lci[w] = J;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                if (WB == 1) ltiles[w * K + r] = (uint8_t)rows[r];
                else if (WB == 2) reinterpret_cast<uint16_t*>(ltiles)[w * K + r] = (uint16_t)rows[r];
                else reinterpret_cast<uint32_t*>(ltiles)[w * K + r] = rows[r];
            }
            ++w;
        }
    }
}

// ---------------------------------------------------------------------------
// weights: CSR order -> set-bit order
// ---------------------------------------------------------------------------
template <int K>
__global__ void weights_kernel(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                               const float* __restrict__ w_csr, int64_t nnz, const int32_t* __restrict__ trp,
                               const int32_t* __restrict__ tci, const uint8_t* __restrict__ tiles,
                               const int32_t* __restrict__ voff, float* __restrict__ w_bits,
                               int* __restrict__ bad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = row_of(rowptr, 0, n - 1, e);
        int32_t j = colind[e];
        int32_t I = i / K, J = j / K;
        int r = i % K, c = j % K;
        int32_t lo = trp[I], hi = trp[I + 1] - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi) / 2;
            if (tci[mid] < J) lo = mid + 1; else hi = mid;
        }
        if (lo > hi || tci[lo] != J) { atomicOr(bad, 1); continue; }
        int64_t t = lo;
        int before = 0;
        for (int q = 0; q < r; ++q) before += __popc(tile_word<K>(tiles, t, q));
        uint32_t word = tile_word<K>(tiles, t, r);
        before += __popc(word & ((1u << c) - 1u));
        w_bits[(int64_t)voff[t] + before] = w_csr[e];
    }
}

}  // namespace b2sr

using namespace b2sr;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" b2sr_status b2sr_from_csr(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                                     int tile_dim, void* stream, b2sr_handle* out) {
    clear_error();
    if (!out) return fail(B2SR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_tile(tile_dim)) return fail(B2SR_ERR_UNSUPPORTED_TILE, "tile_dim must be 4, 8, 16 or 32");
    if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return fail(B2SR_ERR_INVALID_ARG, "bad n or nnz");
    if (!rowptr || (nnz > 0 && !colind)) return fail(B2SR_ERR_INVALID_ARG, "null CSR pointer");
    cudaStream_t s = to_stream(stream);
    const int k = tile_dim;
    const int32_t ntr = (int32_t)ceil_div(n, k);
    const int sbits = bits_for(std::max<int64_t>(ntr, 2));
    if (2 * sbits + 10 > 64) return fail(B2SR_ERR_INVALID_ARG, "matrix too large");

    // validate; note whether every row is in column order
    bool sorted_rows = false;
    {
        DevBuf bad(s);
        B2SR_TRY(bad.alloc(2 * sizeof(int)));
        B2SR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, 2 * sizeof(int), s));
        B2SR_TRY(validate_csr_async(n, rowptr, colind, nnz, bad.as<int>(), s));
        if (nnz > 0 && n > 0) {
            sorted_rows_kernel<<<(unsigned)ceil_div(nnz, kKeyThreads), kKeyThreads, 0, s>>>(n, rowptr, colind, nnz,
                                                                                            bad.as<int>() + 1);
            B2SR_LAUNCH_CHECK("sorted_rows_kernel");
        }
        int hbad[2] = {0, 0};
        B2SR_CUDA_TRY(cudaMemcpyAsync(hbad, bad.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad[0]) return fail(B2SR_ERR_INVALID_ARG, "malformed CSR (rowptr/colind/nnz inconsistent)");
        sorted_rows = hbad[1] == 0;
    }

    // keys in (tile-row, tile-column) order -> heads -> tile index
    int64_t T = 0;
    DevBuf keys(s), ktmp(s), flag(s), tidx(s);
    uint64_t* sorted = nullptr;
    if (nnz > 0) {
        B2SR_TRY(keys.alloc(nnz * sizeof(uint64_t)));
        B2SR_TRY(ktmp.alloc(nnz * sizeof(uint64_t)));
        const unsigned blocks = (unsigned)ceil_div(nnz, kKeyThreads);
        if (sorted_rows) {
            const int G = std::min(k, 8);
            if (G == 4) rank_keys_kernel<4><<<blocks, kKeyThreads, 0, s>>>(n, rowptr, colind, nnz, k, sbits, keys.as<uint64_t>());
            else rank_keys_kernel<8><<<blocks, kKeyThreads, 0, s>>>(n, rowptr, colind, nnz, k, sbits, keys.as<uint64_t>());
            B2SR_LAUNCH_CHECK("rank_keys_kernel");
            uint64_t* cur = keys.as<uint64_t>();
            uint64_t* oth = ktmp.as<uint64_t>();
            for (int run = G; run < k; run *= 2) {
                merge_runs_kernel<<<grid_wide(nnz), 256, 0, s>>>(cur, oth, nnz, rowptr, n, k, run, sbits);
                B2SR_LAUNCH_CHECK("merge_runs_kernel");
                std::swap(cur, oth);
            }
            sorted = cur;
        } else {
            make_keys_kernel<<<blocks, kKeyThreads, 0, s>>>(n, rowptr, colind, nnz, k, sbits, keys.as<uint64_t>());
            B2SR_LAUNCH_CHECK("make_keys_kernel");
            B2SR_TRY(radix_sort_u64(keys.as<uint64_t>(), ktmp.as<uint64_t>(), nnz, 10, 10 + 2 * sbits, s, &sorted));
        }
        B2SR_TRY(flag.alloc(nnz * sizeof(int32_t)));
        B2SR_TRY(tidx.alloc(nnz * sizeof(int64_t)));
        mark_heads_kernel<<<grid_wide(nnz), 256, 0, s>>>(sorted, nnz, flag.as<int32_t>());
        B2SR_LAUNCH_CHECK("mark_heads_kernel");
        B2SR_TRY(exclusive_scan_i32_to_i64(flag.as<int32_t>(), tidx.as<int64_t>(), nnz, s));
        int64_t last = 0;
        int32_t lastf = 0;
        B2SR_CUDA_TRY(cudaMemcpyAsync(&last, tidx.as<int64_t>() + nnz - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaMemcpyAsync(&lastf, flag.as<int32_t>() + nnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        T = last + lastf;
    }

    // outputs
    const int64_t cap = std::max<int64_t>(round_up(T, kTilePad), kTilePad);
    int32_t* o_rowptr = nullptr;
    int32_t* o_colind = nullptr;
    uint8_t* o_tiles = nullptr;
    auto release = [&](b2sr_status st) {
        dfree(o_rowptr, s); dfree(o_colind, s); dfree(o_tiles, s);
        return st;
    };
    b2sr_status st = dalloc(&o_rowptr, (size_t)ntr + 1, s);
    if (st == B2SR_OK) st = dalloc(&o_colind, (size_t)cap, s);
    if (st == B2SR_OK) st = dalloc(&o_tiles, (size_t)cap * tile_bytes(k), s);
    if (st != B2SR_OK) return release(st);
    cudaError_t e = cudaMemsetAsync(o_colind, 0, (size_t)cap * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o_tiles, 0, (size_t)cap * tile_bytes(k), s);
    if (e != cudaSuccess) return release(cuda_fail(e, "memset outputs"));
    {
        DevBuf tilerow(s);
        st = tilerow.alloc(std::max<int64_t>(T, 1) * sizeof(int32_t));
        if (st != B2SR_OK) return release(st);
        if (nnz > 0) {
            fill_tiles_kernel<<<grid_wide(nnz), 256, 0, s>>>(sorted, flag.as<int32_t>(), tidx.as<int64_t>(), nnz, k,
                                                            sbits, o_colind, tilerow.as<int32_t>(),
                                                            reinterpret_cast<uint32_t*>(o_tiles));
            note_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return release(cuda_fail(e, "fill_tiles_kernel"));
        }
        build_rowptr_kernel<<<grid_wide(T + 1), 256, 0, s>>>(tilerow.as<int32_t>(), T, ntr, o_rowptr);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return release(cuda_fail(e, "build_rowptr_kernel"));
    }
    b2sr_matrix* h = nullptr;
    st = new_handle_from_tiles(n, k, T, o_rowptr, o_colind, o_tiles, cap, s, &h);
    if (st != B2SR_OK) return st;  // arrays released by the failed handle
    *out = h;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_to_csr(b2sr_handle h, int32_t* rowptr, int32_t* colind, int64_t* nnz_host,
                                   void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (!rowptr) return fail(B2SR_ERR_INVALID_ARG, "rowptr is NULL");
    cudaStream_t s = to_stream(stream);
    const int32_t n = h->n;
    DevBuf cnt(s), off(s);
    B2SR_TRY(cnt.alloc(((size_t)n + 1) * sizeof(int32_t)));
    B2SR_TRY(off.alloc(((size_t)n + 1) * sizeof(int64_t)));
    B2SR_CUDA_TRY(cudaMemsetAsync(cnt.as<int32_t>() + n, 0, sizeof(int32_t), s));
    B2SR_TRY(with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        if (n > 0) row_nnz_kernel<K><<<grid_wide(n), 256, 0, s>>>(h->rowptr, h->tiles, n, cnt.as<int32_t>());
        B2SR_LAUNCH_CHECK("row_nnz_kernel");
        B2SR_TRY(exclusive_scan_i32_to_i64(cnt.as<int32_t>(), off.as<int64_t>(), (int64_t)n + 1, s));
        row_fill_kernel<K><<<grid_wide((int64_t)n + 1), 256, 0, s>>>(h->rowptr, h->colind, h->tiles, n,
                                                                   off.as<int64_t>(), rowptr, colind);
        B2SR_LAUNCH_CHECK("row_fill_kernel");
        return B2SR_OK;
    }));
    int64_t nnz = 0;
    B2SR_CUDA_TRY(cudaMemcpyAsync(&nnz, off.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    if (nnz_host) *nnz_host = nnz;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_lower(b2sr_handle h, void* stream, b2sr_handle* out) {
    clear_error();
    if (!out) return fail(B2SR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    B2SR_TRY(check_handle(h));
    cudaStream_t s = to_stream(stream);
    const int k = h->k;
    const int32_t ntr = h->ntr;
    DevBuf cnt(s), off(s);
    B2SR_TRY(cnt.alloc(((size_t)ntr + 1) * sizeof(int32_t)));
    B2SR_TRY(off.alloc(((size_t)ntr + 1) * sizeof(int64_t)));
    B2SR_CUDA_TRY(cudaMemsetAsync(cnt.as<int32_t>() + ntr, 0, sizeof(int32_t), s));
    int64_t T = 0;
    B2SR_TRY(with_tile(k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        if (ntr > 0) lower_count_kernel<K><<<grid_wide(ntr), 256, 0, s>>>(h->rowptr, h->colind, h->tiles, ntr, cnt.as<int32_t>());
        B2SR_LAUNCH_CHECK("lower_count_kernel");
        return B2SR_OK;
    }));
    B2SR_TRY(exclusive_scan_i32_to_i64(cnt.as<int32_t>(), off.as<int64_t>(), (int64_t)ntr + 1, s));
    B2SR_CUDA_TRY(cudaMemcpyAsync(&T, off.as<int64_t>() + ntr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t cap = std::max<int64_t>(round_up(T, kTilePad), kTilePad);
    int32_t* lrp = nullptr;
    int32_t* lci = nullptr;
    uint8_t* lt = nullptr;
    auto release = [&](b2sr_status st) {
        dfree(lrp, s); dfree(lci, s); dfree(lt, s);
        return st;
    };
    b2sr_status st = dalloc(&lrp, (size_t)ntr + 1, s);
    if (st == B2SR_OK) st = dalloc(&lci, (size_t)cap, s);
    if (st == B2SR_OK) st = dalloc(&lt, (size_t)cap * tile_bytes(k), s);
    if (st != B2SR_OK) return release(st);
    cudaError_t e = cudaMemsetAsync(lci, 0, (size_t)cap * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lt, 0, (size_t)cap * tile_bytes(k), s);
    if (e != cudaSuccess) return release(cuda_fail(e, "memset lower"));
    st = with_tile(k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        lower_fill_kernel<K><<<grid_wide((int64_t)ntr + 1), 256, 0, s>>>(h->rowptr, h->colind, h->tiles, ntr,
                                                                       off.as<int64_t>(), lrp, lci, lt);
        B2SR_LAUNCH_CHECK("lower_fill_kernel");
        return B2SR_OK;
    });
    if (st != B2SR_OK) return release(st);
    b2sr_matrix* L = nullptr;
    B2SR_TRY(new_handle_from_tiles(h->n, k, T, lrp, lci, lt, cap, s, &L));
    *out = L;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_weights_from_csr(b2sr_handle h, const int32_t* rowptr, const int32_t* colind,
                                             const float* w_csr, float* w_bits, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->nnz == 0) return B2SR_OK;
    if (!rowptr || !colind || !w_csr || !w_bits) return fail(B2SR_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = to_stream(stream);
    B2SR_TRY(ensure_voff(h, s));
    DevBuf bad(s);
    B2SR_TRY(bad.alloc(sizeof(int)));
    B2SR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    B2SR_TRY(with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        weights_kernel<K><<<grid_wide(h->nnz), 256, 0, s>>>(h->n, rowptr, colind, w_csr, h->nnz, h->rowptr,
                                                           h->colind, h->tiles, h->voff, w_bits, bad.as<int>());
        B2SR_LAUNCH_CHECK("weights_kernel");
        return B2SR_OK;
    }));
    int hbad = 0;
    B2SR_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return fail(B2SR_ERR_INVALID_ARG, "CSR does not match the handle");
    return B2SR_OK;
}
