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

// The validation b2sr_from_csr runs, which also finds whether every row is
// in column order.  Row pass: the rowptr checks of validate_csr_kernel, and
// in `starts` (one bit per entry) the entries that begin a row.
__global__ void validate_rows_kernel(int32_t n, const int32_t* __restrict__ rowptr, int64_t nnz,
                                     int* __restrict__ bad, uint32_t* __restrict__ starts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz)) atomicOr(bad, 1);
    for (int64_t i = tid; i < n; i += stride) {
        const int32_t a = rowptr[i], b = rowptr[i + 1];
        if (b < a) atomicOr(bad, 2);
        if (a >= 0 && a < nnz) atomicOr(starts + (a >> 5), 1u << (a & 31));
    }
}

// Entry pass, four entries a step: every column in [0, n) (else bit 4 of
// *bad), and *unsorted set if an entry that does not begin a row has a
// smaller column than the entry before it.
__global__ void validate_entries_kernel(int32_t n, const int32_t* __restrict__ colind, int64_t nnz,
                                        const uint32_t* __restrict__ starts, int* __restrict__ bad,
                                        int* __restrict__ unsorted) {
    const int64_t groups = (nnz + 3) / 4;
    const bool vec = (reinterpret_cast<uintptr_t>(colind) & 15u) == 0;
    bool out = false, down = false;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = g * 4;
        int32_t c[4];
        if (vec && e0 + 4 <= nnz) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(colind) + g);
            c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) c[q] = e0 + q < nnz ? __ldg(colind + e0 + q) : 0;
        }
        const uint32_t sw = __ldg(starts + (e0 >> 5)) >> (e0 & 31);  // e0 % 4 == 0: one word holds all four
        int32_t prev = e0 > 0 ? __ldg(colind + e0 - 1) : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (e0 + q >= nnz) break;
            out |= c[q] < 0 || c[q] >= n;
            down |= e0 + q > 0 && !((sw >> q) & 1u) && prev > c[q];
            prev = c[q];
        }
    }
    if (out) atomicOr(bad, 4);
    if (down) atomicOr(unsorted, 1);
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
// largest r in [lo, hi] with rowptr[r] <= e
__device__ __forceinline__ int32_t row_of(const int32_t* __restrict__ rowptr, int32_t lo, int32_t hi,
                                          int64_t e) {
    while (lo < hi) {
        int32_t mid = lo + (hi - lo + 1) / 2;
        if ((int64_t)__ldg(rowptr + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The entry-parallel kernels below give each thread kRankPer consecutive CSR
// entries.  A thread finds the row of its first entry by a binary search
// between the rows of its block's first and last entries (brow), then walks
// forward through rows as its entries cross them.
constexpr int kRankThreads = 256;
constexpr int kRankPer = 8;
constexpr int kRankEntries = kRankThreads * kRankPer;

// brow[b] = row of entry b * kRankEntries for every block b < nblocks, and
// brow[nblocks] = row of the last entry: one independent search per block, so
// that no block starts with a chain of dependent global loads.  The entries of
// block b lie in rows brow[b] .. brow[b+1].
__global__ void block_rows_kernel(int32_t n, const int32_t* __restrict__ rowptr, int64_t nnz, int64_t nblocks,
                                  int32_t* __restrict__ brow) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nblocks;
         b += (int64_t)gridDim.x * blockDim.x)
        brow[b] = row_of(rowptr, 0, n - 1, b < nblocks ? b * kRankEntries : nnz - 1);
}

// The thread's entries [e0, e1) and the row holding e0: rows i with
// rowptr[i] <= e < rowptr[i+1] = re.  Returns false for a thread with none.
struct EntryRun {  // positions fit int32: the conversion takes nnz < 2^31
    int32_t e0, e1;
    int32_t i;
    int32_t rs, re;  // rowptr[i], rowptr[i+1]
};

// largest r in [lo, hi] with rowptr[r] <= e (int32 positions)
__device__ __forceinline__ int32_t row_of32(const int32_t* __restrict__ rowptr, int32_t lo, int32_t hi, int32_t e) {
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo + 1) / 2;
        if (__ldg(rowptr + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool entry_run(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ brow,
                                          int32_t n, int64_t nnz, EntryRun& u) {
    const int64_t e0 = ((int64_t)blockIdx.x * kRankThreads + threadIdx.x) * kRankPer;
    if (e0 >= nnz) return false;
    u.e0 = (int32_t)e0;
    u.e1 = (int32_t)min(e0 + kRankPer, nnz);
    u.i = row_of32(rowptr, __ldg(brow + blockIdx.x), __ldg(brow + blockIdx.x + 1), u.e0);
    u.rs = __ldg(rowptr + u.i);
    u.re = __ldg(rowptr + u.i + 1);
    return true;
}

// Moves u to the row holding entry e (e >= u.rs); true if the row changed.
// Never passes row n-1 (for a valid CSR, e < nnz lies in a row below n).
__device__ __forceinline__ bool advance_row(const int32_t* __restrict__ rowptr, int32_t n, int32_t e, EntryRun& u) {
    bool moved = false;
    while (e >= u.re && u.i + 1 < n) {
        ++u.i;
        u.rs = u.re;
        u.re = __ldg(rowptr + u.i + 1);
        moved = true;
    }
    return moved;
}

// k is a power of two: shifts and masks instead of divisions by a runtime k.
__device__ __forceinline__ uint64_t entry_key(int32_t i, int32_t j, int k, int sbits) {
    const int lk = __ffs(k) - 1;
    return ((uint64_t)(i >> lk) << (sbits + 10)) | ((uint64_t)(j >> lk) << 10) |
           (uint64_t)(((j & (k - 1)) << lk) | (i & (k - 1)));
}

__global__ void __launch_bounds__(kRankThreads) make_keys_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                                                 const int32_t* __restrict__ brow,
                                                                 const int32_t* __restrict__ colind,
                                                                 int64_t nnz, int k, int sbits,
                                                                 uint64_t* __restrict__ keys) {
    EntryRun u;
    if (!entry_run(rowptr, brow, n, nnz, u)) return;
    for (int32_t e = u.e0; e < u.e1; ++e) {
        advance_row(rowptr, n, e, u);
        keys[e] = entry_key(u.i, __ldg(colind + e), k, sbits);
    }
}

// Sorted rows: writes every entry's key straight to its place in the order of
// its group of G rows (G divides k, groups start at multiples of G).  The
// place is the group's first CSR position, plus the entry's offset in its own
// row, plus, for every other row q of the group, the entries of q ahead of it
// in (column, row) order: those with a smaller column, and those with the same
// column when q is an earlier row.  A thread's first entry in a row finds
// those counts by binary searches (advancing side by side, so that their loads
// overlap); its later entries in the row have columns no smaller, so each
// count moves forward from the last one by a galloping search.
template <int G>
__global__ void __launch_bounds__(kRankThreads) rank_keys_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                                                 const int32_t* __restrict__ brow,
                                                                 const int32_t* __restrict__ colind,
                                                                 int64_t nnz, int k, int sbits,
                                                                 uint64_t* __restrict__ keys) {
    EntryRun u;
    if (!entry_run(rowptr, brow, n, nnz, u)) return;
    // pos[q]: entries of row q of the group ahead of the current entry (from
    // base[q]); end[q]: the row's end.  The entry's own row keeps an empty
    // range.  An entry x of row q is ahead of column j when x < j + tie[q]:
    // the same column counts as ahead in an earlier row.
    int32_t pos[G], end[G], base[G];
    int tie[G];
    int32_t gstart = 0;
    bool fresh = true;
    for (int32_t e = u.e0; e < u.e1; ++e) {
        fresh |= advance_row(rowptr, n, e, u);
        const int32_t j = __ldg(colind + e);
        if (fresh) {
            const int rg = u.i % G;
            const int32_t g0 = u.i - rg;
            gstart = __ldg(rowptr + g0);
            int32_t hi[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int32_t iq = g0 + q;
                const bool live = q != rg && iq < n;
                pos[q] = live ? __ldg(rowptr + iq) : 0;
                end[q] = live ? __ldg(rowptr + iq + 1) : 0;
                base[q] = pos[q];
                hi[q] = end[q];
                tie[q] = q < rg ? 1 : 0;
            }
            // binary searches, side by side
            for (;;) {
                bool more = false;
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (pos[q] < hi[q]) {
                        const int32_t mid = pos[q] + ((hi[q] - pos[q]) >> 1);
                        if (__ldg(colind + mid) < j + tie[q]) pos[q] = mid + 1; else hi[q] = mid;
                        more = true;
                    }
                }
                if (!more) break;
            }
            fresh = false;
        } else {
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int32_t jq = j + tie[q];
                int32_t lo = pos[q], hi = end[q];
                if (lo >= hi || __ldg(colind + lo) >= jq) continue;  // nothing more of row q is ahead
                // gallop: entry lo is ahead; double the step until an entry is not
                int32_t step = 1, last = lo;
                while (hi - last > step) {
                    const int32_t probe = last + step;
                    if (__ldg(colind + probe) >= jq) { hi = probe; break; }
                    last = probe;
                    step <<= 1;
                }
                lo = last + 1;
                while (lo < hi) {
                    const int32_t mid = lo + ((hi - lo) >> 1);
                    if (__ldg(colind + mid) < jq) lo = mid + 1; else hi = mid;
                }
                pos[q] = lo;
            }
        }
        int32_t dest = gstart + (e - u.rs);
#pragma unroll
        for (int q = 0; q < G; ++q) dest += pos[q] - base[q];
        keys[dest] = entry_key(u.i, j, k, sbits);
    }
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
        const int r = (int)(x & 1023u) & (k - 1);
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

// Keys in order -> tiles, in two passes over the keys.  A key whose tile
// (its bits above the low 10) differs from the previous key's is a run head:
// the first entry of a new tile.  Pass 1 counts the heads of every block of
// kFillTile keys; after an exclusive scan of those counts, pass 2 gives each
// key its tile index (the block's offset plus the heads before it), writes
// the column index of every new tile, points rowptr at the first tile of
// every tile-row that begins there, and ORs the bits of each run of keys that
// fall in one 32-bit word of the tile array in one atomic.
constexpr int kFillThreads = 256;
constexpr int kFillItems = 8;  // consecutive keys per thread
constexpr int kFillTile = kFillThreads * kFillItems;

// Loads keys base .. base+kFillItems-1 (those below N) and the key before base.
__device__ __forceinline__ void load_run(const uint64_t* __restrict__ keys, int64_t N, int64_t base,
                                         uint64_t (&key)[kFillItems], uint64_t& before) {
    before = base > 0 && base <= N ? __ldg(keys + base - 1) : 0ull;
    if (base + kFillItems <= N) {
        const ulonglong2* v = reinterpret_cast<const ulonglong2*>(keys + base);  // base is a multiple of 8 keys
#pragma unroll
        for (int q = 0; q < kFillItems / 2; ++q) {
            const ulonglong2 x = __ldg(v + q);
            key[2 * q] = x.x;
            key[2 * q + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kFillItems; ++q) key[q] = base + q < N ? __ldg(keys + base + q) : 0ull;
    }
}

// Bit q of the result: key q of the run is a head.
__device__ __forceinline__ uint32_t run_heads(const uint64_t (&key)[kFillItems], uint64_t before, int64_t base,
                                              int64_t N) {
    uint32_t h = 0;
#pragma unroll
    for (int q = 0; q < kFillItems; ++q) {
        const uint64_t prev = q == 0 ? before : key[q - 1];
        if (base + q < N && (base + q == 0 || (key[q] >> 10) != (prev >> 10))) h |= 1u << q;
    }
    return h;
}

// Sum of v over the block; every thread gets it.  Also returns, in *excl,
// the sum over the threads before this one.
__device__ __forceinline__ int block_scan(int v, int* excl) {
    __shared__ int warp_tot[kFillThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kFillThreads / 32; ++w) {
        const int x = warp_tot[w];
        before += w < wid ? x : 0;
        total += x;
    }
    *excl = before + inc - v;
    return total;
}

__global__ void __launch_bounds__(kFillThreads) count_heads_kernel(const uint64_t* __restrict__ keys, int64_t N,
                                                                   int64_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kFillTile + (int64_t)threadIdx.x * kFillItems;
    uint64_t key[kFillItems], before;
    load_run(keys, N, base, key, before);
    int excl;
    const int total = block_scan(__popc(run_heads(key, before, base, N)), &excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Pass 2 for k <= 8, where a tile (one byte per row) is one 64-bit word:
// the block's keys come in coalesced through shared memory, its tiles and
// their column indices are built in shared memory and leave in coalesced
// stores.  Only a tile whose run of keys crosses a block boundary is ORed
// into global memory by atomics (from both sides).
__device__ __forceinline__ int fill_slot(int i) { return i + (i >> 4); }  // padding: no bank conflicts

__global__ void __launch_bounds__(kFillThreads) fill_small_tiles_kernel(const uint64_t* __restrict__ keys, int64_t N,
                                                                        const int64_t* __restrict__ block_off,
                                                                        int k, int sbits, int32_t ntr, int64_t T,
                                                                        int32_t* __restrict__ colind,
                                                                        int32_t* __restrict__ rowptr,
                                                                        uint32_t* __restrict__ tiles32) {
    __shared__ uint64_t s_key[kFillTile + kFillTile / 16];
    __shared__ unsigned long long s_tile[kFillTile];
    __shared__ int32_t s_col[kFillTile];
    const int64_t b0 = (int64_t)blockIdx.x * kFillTile;
    const int cnt = (int)min((int64_t)kFillTile, N - b0);
    {
        uint64_t v[kFillItems];  // all loads in flight before the first store
#pragma unroll
        for (int q = 0; q < kFillItems; ++q) {
            const int i = q * kFillThreads + threadIdx.x;
            v[q] = i < cnt ? __ldg(keys + b0 + i) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < kFillItems; ++q) {
            const int i = q * kFillThreads + threadIdx.x;
            s_key[fill_slot(i)] = v[q];
            s_tile[i] = 0ull;
        }
    }
    __syncthreads();
    const int q0 = threadIdx.x * kFillItems;
    uint64_t key[kFillItems];
#pragma unroll
    for (int q = 0; q < kFillItems; ++q) key[q] = s_key[fill_slot(q0 + q)];
    const uint64_t before = threadIdx.x > 0 ? s_key[fill_slot(q0 - 1)] : (b0 > 0 ? __ldg(keys + b0 - 1) : 0ull);
    const uint32_t h = run_heads(key, before, b0 + q0, N);
    int excl;
    const int heads = block_scan(__popc(h), &excl);
    const int64_t boff = block_off[blockIdx.x];
    const uint64_t jmask = (1ull << sbits) - 1ull;
    const bool wide = k == 8;
    int lt = excl - 1;  // block-local tile of the run in progress (-1: a tile begun in an earlier block)
    uint64_t acc = 0;
    // A run that begins and ends among this thread's keys owns its tile: a
    // plain shared-memory store.  Runs cut by a thread boundary are ORed in.
    bool owned = false;
    uint64_t lastkey = 0;
    auto flush = [&](bool cut) {
        if (!acc) return;
        if (lt >= 0) {
            if (owned && !cut) s_tile[lt] = acc;
            else atomicOr(&s_tile[lt], (unsigned long long)acc);
        } else if (wide) {
            atomicOr(reinterpret_cast<unsigned long long*>(tiles32) + (boff - 1), (unsigned long long)acc);
        } else {
            atomicOr(tiles32 + (boff - 1), (uint32_t)acc);
        }
        acc = 0;
    };
#pragma unroll
    for (int q = 0; q < kFillItems; ++q) {
        if (q0 + q >= cnt) break;
        const uint64_t x = key[q];
        lastkey = x;
        if ((h >> q) & 1u) {
            flush(false);
            ++lt;
            owned = true;
            s_col[lt] = (int32_t)((x >> 10) & jmask);
            const int64_t I = (int64_t)(x >> (sbits + 10));
            const int64_t Ip = b0 + q0 + q == 0 ? -1 : (int64_t)((q == 0 ? before : key[q - 1]) >> (sbits + 10));
            for (int64_t R = Ip + 1; R <= I; ++R) rowptr[R] = (int32_t)(boff + lt);
        }
        const int p = (int)(x & 1023u);
        acc |= 1ull << ((p & (k - 1)) * 8 + (p >> (__ffs(k) - 1)));
        if (b0 + q0 + q == N - 1)  // tile-rows after the last entry's start at T
            for (int64_t R = (int64_t)(x >> (sbits + 10)) + 1; R <= ntr; ++R) rowptr[R] = (int32_t)T;
    }
    {
        // the last run goes on past this thread unless the next key starts a tile
        const int nq = q0 + kFillItems;
        const int last = min(kFillItems, cnt - q0) - 1;
        bool cut = false;
        if (last >= 0 && b0 + q0 + last + 1 < N) {
            const uint64_t nk = nq < cnt ? s_key[fill_slot(nq)] : __ldg(keys + b0 + q0 + last + 1);
            cut = (nk >> 10) == (lastkey >> 10);
        }
        flush(cut);
    }
    __syncthreads();
    // the block's last tile goes on into the next block unless the next key starts a tile
    const bool cut = b0 + cnt < N && (__ldg(keys + b0 + cnt) >> 10) == (s_key[fill_slot(cnt - 1)] >> 10);
    for (int i = threadIdx.x; i < heads; i += kFillThreads) {
        const int64_t t = boff + i;
        colind[t] = s_col[i];
        const unsigned long long v = s_tile[i];
        const bool shared_tile = cut && i == heads - 1;
        if (wide) {
            unsigned long long* t64 = reinterpret_cast<unsigned long long*>(tiles32);
            if (shared_tile) atomicOr(t64 + t, v); else t64[t] = v;
        } else {
            if (shared_tile) atomicOr(tiles32 + t, (uint32_t)v); else tiles32[t] = (uint32_t)v;
        }
    }
}

__global__ void __launch_bounds__(kFillThreads, 4) fill_tiles_kernel(const uint64_t* __restrict__ keys, int64_t N,
                                                                  const int64_t* __restrict__ block_off, int k,
                                                                  int sbits, int32_t ntr, int64_t T,
                                                                  int32_t* __restrict__ colind,
                                                                  int32_t* __restrict__ rowptr,
                                                                  uint32_t* __restrict__ tiles32) {
    const int64_t base = (int64_t)blockIdx.x * kFillTile + (int64_t)threadIdx.x * kFillItems;
    uint64_t key[kFillItems], before;
    load_run(keys, N, base, key, before);
    const uint32_t h = run_heads(key, before, base, N);
    int excl;
    block_scan(__popc(h), &excl);
    const int wb = word_bytes(k);
    const uint64_t jmask = (1ull << sbits) - 1ull;
    int64_t t = block_off[blockIdx.x] + excl - 1;  // the tile of the run in progress
    // k <= 8: a whole tile (one byte per row) fits one 64-bit register.  A tile
    // whose run of keys begins and ends in this thread is stored outright;
    // only the runs cut by a thread boundary need atomics.
    const bool whole = k <= 8;
    bool owned = false;  // the run in progress began in this thread
    uint64_t tacc = 0;
    int64_t accw = -1;
    uint32_t acc = 0;
    auto flush_tile = [&](bool cut) {
        if (k == 4) {
            if (owned && !cut) tiles32[t] = (uint32_t)tacc;
            else atomicOr(tiles32 + t, (uint32_t)tacc);
        } else {
            unsigned long long* t64 = reinterpret_cast<unsigned long long*>(tiles32);
            if (owned && !cut) t64[t] = tacc;
            else atomicOr(t64 + t, (unsigned long long)tacc);
        }
    };
    int last = -1;
    uint64_t lastkey = 0;
#pragma unroll
    for (int q = 0; q < kFillItems; ++q) {
        if (base + q >= N) break;
        last = q;
        const uint64_t x = key[q];
        lastkey = x;
        if ((h >> q) & 1u) {
            if (whole && q > 0) flush_tile(false);
            ++t;
            owned = true;
            tacc = 0;
            colind[t] = (int32_t)((x >> 10) & jmask);
            const int64_t I = (int64_t)(x >> (sbits + 10));
            const int64_t Ip = base + q == 0 ? -1 : (int64_t)((q == 0 ? before : key[q - 1]) >> (sbits + 10));
            for (int64_t R = Ip + 1; R <= I; ++R) rowptr[R] = (int32_t)t;
        }
        const int p = (int)(x & 1023u);
        const int r = p & (k - 1), c = p >> (__ffs(k) - 1);
        if (whole) {
            tacc |= 1ull << (r * 8 + c);
        } else {
            const int64_t byte = (t * k + r) * wb + (c >> 3);
            if ((byte >> 2) != accw) {
                if (accw >= 0) atomicOr(tiles32 + accw, acc);
                accw = byte >> 2;
                acc = 0;
            }
            acc |= 1u << ((int)(byte & 3) * 8 + (c & 7));
        }
        if (base + q == N - 1)  // tile-rows after the last entry's start at T
            for (int64_t R = (int64_t)(x >> (sbits + 10)) + 1; R <= ntr; ++R) rowptr[R] = (int32_t)T;
    }
    if (last < 0) return;
    if (whole) {
        // the last run goes on into the next thread unless the next key starts a tile
        const int64_t nx = base + last + 1;
        const bool cut = nx < N && (__ldg(keys + nx) >> 10) == (lastkey >> 10);
        flush_tile(cut);
    } else if (accw >= 0) {
        atomicOr(tiles32 + accw, acc);
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

// Column counts go to `copies` copies of the count array (warp w adds into
// copy w % copies), summed at the end: the hub columns' atomics spread over
// several addresses, and so over several L2 slices, instead of queueing on one.
constexpr int kDegCopies = 8;

__global__ void deg_sum_kernel(const int32_t* __restrict__ sub, int64_t stride, int copies, int64_t len,
                               int32_t* __restrict__ deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = 0;
        for (int c = 0; c < copies; ++c) v += __ldg(sub + c * stride + i);
        deg[i] = v;
    }
}

// k = 4: four tiles (16 bytes of words, 16 of column indices) per thread and
// step; the padding after T is zero, so whole groups of four can be read.
// Column c of a tile word (row r in byte r) counts popc(w & (0x01010101 << c)).
__global__ void col_count4_kernel(const int32_t* __restrict__ colind, const uint8_t* __restrict__ tiles,
                                  int64_t groups, int32_t* __restrict__ sub, int64_t stride, int copies) {
    int32_t* __restrict__ deg = sub + (int64_t)((threadIdx.x >> 5) % copies) * stride;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(tiles) + g);
        const int4 J = __ldg(reinterpret_cast<const int4*>(colind) + g);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        const int32_t js[4] = {J.x, J.y, J.z, J.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int v = __popc(ws[q] & (0x01010101u << c));
                if (v) atomicAdd(deg + (int64_t)js[q] * 4 + c, v);
            }
        }
    }
}

template <int K>
__global__ void col_count_kernel(const int32_t* __restrict__ colind, const uint8_t* __restrict__ tiles,
                                 int64_t T, int32_t* __restrict__ sub, int64_t stride, int copies) {
    int32_t* __restrict__ deg = sub + (int64_t)((threadIdx.x >> 5) % copies) * stride;
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
    const int64_t len = (int64_t)h->ntr * h->k;
    int32_t* deg = nullptr;
    B2SR_TRY(dalloc(&deg, (size_t)len, s));
    // copies while they stay under 1 GiB in all
    const int copies = (int)std::max<int64_t>(1, std::min<int64_t>(kDegCopies, (int64_t(1) << 30) / (len * 4 + 1)));
    DevBuf sub(s);
    b2sr_status st = sub.alloc((size_t)copies * len * sizeof(int32_t));
    if (st != B2SR_OK) { dfree(deg, s); return st; }
    cudaError_t e = cudaMemsetAsync(sub.p, 0, (size_t)copies * len * sizeof(int32_t), s);
    if (e != cudaSuccess) { dfree(deg, s); return cuda_fail(e, "memset outdeg"); }
    st = with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        if (h->T > 0 && K == 4)  // cap is a multiple of 512 tiles: groups of four stay inside the arrays
            col_count4_kernel<<<grid_wide(ceil_div(h->T, 4)), 256, 0, s>>>(h->colind, h->tiles, ceil_div(h->T, 4),
                                                                          sub.as<int32_t>(), len, copies);
        else if (h->T > 0)
            col_count_kernel<K><<<grid_wide(h->T), 256, 0, s>>>(h->colind, h->tiles, h->T, sub.as<int32_t>(), len,
                                                                copies);
        B2SR_LAUNCH_CHECK("col_count_kernel");
        deg_sum_kernel<<<grid_wide(len), 256, 0, s>>>(sub.as<int32_t>(), len, copies, len, deg);
        B2SR_LAUNCH_CHECK("deg_sum_kernel");
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

// A tile-row's tiles are in column order, so those strictly left of the
// diagonal are a prefix, found by one binary search; the diagonal tile, if
// present, follows it and keeps only its bits below the diagonal.
template <int K>
__device__ __forceinline__ bool diag_has_lower(const uint8_t* __restrict__ tiles, int64_t t) {
    uint32_t any = 0;
#pragma unroll
    for (int r = 0; r < K; ++r) any |= tile_word<K>(tiles, t, r) & strict_lower_mask<K>(r);
    return any != 0;
}

template <int K>
__global__ void lower_count_kernel(const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                   const uint8_t* __restrict__ tiles, int32_t ntr, int32_t* __restrict__ cnt,
                                   int32_t* __restrict__ pre) {
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < ntr;
         I += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t0 = __ldg(trp + I), t1 = __ldg(trp + I + 1);
        int32_t lo = t0, hi = t1;  // first tile with column >= I
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (__ldg(tci + mid) < I) lo = mid + 1; else hi = mid;
        }
        pre[I] = lo - t0;
        cnt[I] = lo - t0 + ((lo < t1 && __ldg(tci + lo) == I && diag_has_lower<K>(tiles, lo)) ? 1 : 0);
    }
}

// A warp per tile-row: the lanes copy the prefix tile by tile (coalesced),
// then lane 0 writes the masked diagonal tile.
template <int K>
__global__ void lower_fill_kernel(const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                  const uint8_t* __restrict__ tiles, int32_t ntr, const int64_t* __restrict__ off,
                                  const int32_t* __restrict__ pre, int32_t* __restrict__ lrp,
                                  int32_t* __restrict__ lci, uint8_t* __restrict__ ltiles) {
    constexpr int TB = K * (K <= 8 ? 1 : (K == 16 ? 2 : 4));  // bytes per tile
    constexpr int TW = (TB + 3) / 4;                            // 32-bit words per tile
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I <= ntr; I += warps) {
        const int64_t o = off[I];
        if (lane == 0) lrp[I] = (int32_t)o;
        if (I == ntr) continue;
        const int32_t t0 = __ldg(trp + I), t1 = __ldg(trp + I + 1), np = pre[I];
        for (int32_t q = lane; q < np; q += 32) {
            lci[o + q] = __ldg(tci + t0 + q);
            if (TB >= 4) {
                const uint32_t* src = reinterpret_cast<const uint32_t*>(tiles) + (int64_t)(t0 + q) * TW;
                uint32_t* dst = reinterpret_cast<uint32_t*>(ltiles) + (o + q) * TW;
#pragma unroll
                for (int w = 0; w < TW; ++w) dst[w] = __ldg(src + w);
            }
        }
        const int32_t d = t0 + np;
        if (lane == 0 && d < t1 && __ldg(tci + d) == I && diag_has_lower<K>(tiles, d)) {
            const int64_t w = o + np;
            lci[w] = (int32_t)I;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const uint32_t v = tile_word<K>(tiles, d, r) & strict_lower_mask<K>(r);
                if (K <= 8) ltiles[w * K + r] = (uint8_t)v;
                else if (K == 16) reinterpret_cast<uint16_t*>(ltiles)[w * K + r] = (uint16_t)v;
                else reinterpret_cast<uint32_t*>(ltiles)[w * K + r] = v;
            }
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
    const int64_t blocks = ceil_div(nnz, kRankEntries);
    DevBuf brow(s);
    {
        DevBuf bad(s), starts(s);
        const size_t start_words = (size_t)ceil_div(std::max<int64_t>(nnz, 1), 32);
        B2SR_TRY(bad.alloc(2 * sizeof(int)));
        B2SR_TRY(starts.alloc(start_words * sizeof(uint32_t)));
        B2SR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, 2 * sizeof(int), s));
        B2SR_CUDA_TRY(cudaMemsetAsync(starts.p, 0, start_words * sizeof(uint32_t), s));
        validate_rows_kernel<<<grid_wide((int64_t)n + 1), 256, 0, s>>>(n, rowptr, nnz, bad.as<int>(),
                                                                      starts.as<uint32_t>());
        B2SR_LAUNCH_CHECK("validate_rows_kernel");
        if (nnz > 0) {
            validate_entries_kernel<<<grid_wide(ceil_div(nnz, 4)), 256, 0, s>>>(
                n, colind, nnz, starts.as<uint32_t>(), bad.as<int>(), bad.as<int>() + 1);
            B2SR_LAUNCH_CHECK("validate_entries_kernel");
        }
        int hbad[2] = {0, 0};
        B2SR_CUDA_TRY(cudaMemcpyAsync(hbad, bad.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad[0]) return fail(B2SR_ERR_INVALID_ARG, "malformed CSR (rowptr/colind/nnz inconsistent)");
        sorted_rows = hbad[1] == 0;
    }
    if (nnz > 0) {
        B2SR_TRY(brow.alloc((size_t)(blocks + 1) * sizeof(int32_t)));
        block_rows_kernel<<<grid_for(blocks + 1), 256, 0, s>>>(n, rowptr, nnz, blocks, brow.as<int32_t>());
        B2SR_LAUNCH_CHECK("block_rows_kernel");
    }

    // keys in (tile-row, tile-column) order -> heads -> tile index
    int64_t T = 0;
    DevBuf keys(s), ktmp(s), hsum(s), hoff(s);
    const int64_t fill_blocks = ceil_div(nnz, kFillTile);
    uint64_t* sorted = nullptr;
    if (nnz > 0) {
        B2SR_TRY(keys.alloc(nnz * sizeof(uint64_t)));
        B2SR_TRY(ktmp.alloc(nnz * sizeof(uint64_t)));
        const int32_t* br = brow.as<int32_t>();
        if (sorted_rows) {
            const int G = std::min(k, 8);
            if (G == 4)
                rank_keys_kernel<4><<<(unsigned)blocks, kRankThreads, 0, s>>>(n, rowptr, br, colind, nnz, k, sbits,
                                                                            keys.as<uint64_t>());
            else
                rank_keys_kernel<8><<<(unsigned)blocks, kRankThreads, 0, s>>>(n, rowptr, br, colind, nnz, k, sbits,
                                                                            keys.as<uint64_t>());
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
            make_keys_kernel<<<(unsigned)blocks, kRankThreads, 0, s>>>(n, rowptr, br, colind, nnz, k, sbits,
                                                                     keys.as<uint64_t>());
            B2SR_LAUNCH_CHECK("make_keys_kernel");
            B2SR_TRY(radix_sort_u64(keys.as<uint64_t>(), ktmp.as<uint64_t>(), nnz, 10, 10 + 2 * sbits, s, &sorted));
        }
        B2SR_TRY(hsum.alloc(fill_blocks * sizeof(int64_t)));
        B2SR_TRY(hoff.alloc(fill_blocks * sizeof(int64_t)));
        count_heads_kernel<<<(unsigned)fill_blocks, kFillThreads, 0, s>>>(sorted, nnz, hsum.as<int64_t>());
        B2SR_LAUNCH_CHECK("count_heads_kernel");
        B2SR_TRY(exclusive_scan_i64(hsum.as<int64_t>(), hoff.as<int64_t>(), fill_blocks, s));
        int64_t last[2] = {0, 0};
        B2SR_CUDA_TRY(cudaMemcpyAsync(&last[0], hoff.as<int64_t>() + fill_blocks - 1, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaMemcpyAsync(&last[1], hsum.as<int64_t>() + fill_blocks - 1, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        T = last[0] + last[1];
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
    if (nnz > 0) {
        if (k <= 8)
            fill_small_tiles_kernel<<<(unsigned)fill_blocks, kFillThreads, 0, s>>>(
                sorted, nnz, hoff.as<int64_t>(), k, sbits, ntr, T, o_colind, o_rowptr,
                reinterpret_cast<uint32_t*>(o_tiles));
        else
            fill_tiles_kernel<<<(unsigned)fill_blocks, kFillThreads, 0, s>>>(sorted, nnz, hoff.as<int64_t>(), k,
                                                                             sbits, ntr, T, o_colind, o_rowptr,
                                                                             reinterpret_cast<uint32_t*>(o_tiles));
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return release(cuda_fail(e, "fill_tiles_kernel"));
    } else {
        e = cudaMemsetAsync(o_rowptr, 0, ((size_t)ntr + 1) * sizeof(int32_t), s);
        if (e != cudaSuccess) return release(cuda_fail(e, "memset rowptr"));
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
    DevBuf cnt(s), off(s), pre(s);
    B2SR_TRY(cnt.alloc(((size_t)ntr + 1) * sizeof(int32_t)));
    B2SR_TRY(off.alloc(((size_t)ntr + 1) * sizeof(int64_t)));
    B2SR_TRY(pre.alloc(((size_t)ntr + 1) * sizeof(int32_t)));
    B2SR_CUDA_TRY(cudaMemsetAsync(cnt.as<int32_t>() + ntr, 0, sizeof(int32_t), s));
    int64_t T = 0;
    B2SR_TRY(with_tile(k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        if (ntr > 0)
            lower_count_kernel<K><<<grid_wide(ntr), 256, 0, s>>>(h->rowptr, h->colind, h->tiles, ntr, cnt.as<int32_t>(),
                                                                 pre.as<int32_t>());
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
        lower_fill_kernel<K><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)ntr + 1, 8),
                                                                                   (int64_t)sm_count() * 16)),
                               256, 0, s>>>(h->rowptr, h->colind, h->tiles, ntr, off.as<int64_t>(), pre.as<int32_t>(),
                                            lrp, lci, lt);
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
