// B2SR SpMV: the BMV schemes of Table 2 over the semirings of Table 4, and the
// 64-lane Boolean SpMM used by multi-source BFS.
//
// Design (GB300): the paper maps one tile-row to one warp (Listing 1) or 32
// tile-rows to a 1024-thread block (Sec. IV, bmv_bin_full_full).  Power-law
// graphs make that row mapping badly imbalanced (a scale-20 R-MAT tile-row
// can hold 10^4 tiles), so here the unit of work is a fixed-size chunk of
// consecutive tiles instead:
//   * a warp owns a chunk of 32*P tiles (P tiles per lane); persistent warps
//     stream chunks, double-buffering them into shared memory with 16-byte
//     cp.async copies, so the tile stream is read once, fully coalesced;
//   * each lane walks its P tiles in order, accumulating the k row results
//     of the current tile-row and storing every row that starts and ends
//     inside the lane;
//   * rows that cross lanes are joined with a warp-level segmented scan
//     (shuffles, fixed order); rows that cross chunks leave per-chunk partials
//     that a second small kernel joins in chunk order.
// Every reduction order is fixed by the data, so floating-point results are
// bitwise reproducible and independent of the grid size or stream.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "b2sr_internal.cuh"

namespace b2sr {

// ---------------------------------------------------------------------------
// tile words.  A lane holds its P tiles as 32-bit words: TW words per tile
// (k=4: 1, k=8: 2, k=16: 8, k=32: 32); row r of a tile is byte r (k<=8),
// half-word r (k=16) or word r (k=32).
// ---------------------------------------------------------------------------
template <int K>
struct ChunkShape {
    static constexpr int P = tiles_per_lane(K);
    static constexpr int CT = 32 * P;
    static constexpr int TB = K * (K <= 8 ? 1 : (K == 16 ? 2 : 4));
    static constexpr int TW = TB / 4;
    static constexpr int TILE_V4 = P * TB / 16;   // uint4 loads per lane for its tiles
};

template <int K>
__device__ __forceinline__ uint32_t row_word(const uint32_t* w, int r) {
    if (K == 32) return w[r];
    if (K == 16) return (w[r >> 1] >> (16 * (r & 1))) & 0xFFFFu;
    return (w[r >> 2] >> (8 * (r & 3))) & 0xFFu;
}

// Bit r of the result is set iff row r of the tile shares a bit with xs (the
// k-bit segment of the input vector under the tile's column).
template <int K>
__device__ __forceinline__ uint32_t rows_hit(const uint32_t* w, uint32_t xs) {
    if (K == 4 || K == 8) {
        // four rows per word, one per byte: flag the non-zero bytes (high bit
        // per byte), then gather the four flags with one multiply
        const uint32_t rep = xs * 0x01010101u;
        uint32_t out = 0;
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            uint32_t m = w[q] & rep;
            uint32_t h = (((m & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | m) & 0x80808080u;
            out |= (((h >> 7) * 0x00204081u) >> 21 & 0xFu) << (4 * q);
        }
        return out;
    } else if (K == 16) {
        const uint32_t rep = xs | (xs << 16);
        uint32_t out = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t m = w[q] & rep;
            out |= ((m & 0xFFFFu) ? 1u : 0u) << (2 * q);
            out |= ((m >> 16) ? 1u : 0u) << (2 * q + 1);
        }
        return out;
    } else {
        uint32_t out = 0;
#pragma unroll
        for (int r = 0; r < 32; ++r) out |= ((w[r] & xs) ? 1u : 0u) << r;
        return out;
    }
}

__device__ __forceinline__ bool mask_allows(const uint32_t* __restrict__ mask, int comp, int64_t v) {
    if (!mask) return true;
    bool b = (__ldg(mask + (v >> 5)) >> (v & 31)) & 1u;
    return comp ? !b : b;
}

// ---------------------------------------------------------------------------
// semirings.  Each provides V (accumulator value), NV (values per tile-row
// accumulator), ident(), comb(a, b) (a earlier in the fixed order) and
// store(R, acc), which applies the self term, the mask and the overwrite
// rule (empty tile-rows are stored with the identity accumulator).
//   bit-vector schemes (kGather = false): xseg(J) and tile(acc, words, xs);
//   value schemes (kGather = true): one gathered input value per set bit,
//     src() (the values), weighted and apply(acc, x_j, w_ij).
// ---------------------------------------------------------------------------

// bmv_bin_bin_bin[_masked]: bitset in, bitset out, acc = k-bit row mask
template <int K>
struct SemBool {
    using V = uint32_t;
    static constexpr int NV = 1;
    static constexpr bool kGather = false;
    const uint32_t* x;
    uint32_t* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ V ident() const { return 0u; }
    __device__ V comb(V a, V b) const { return a | b; }
    __device__ uint32_t xseg(int32_t J) const { return ld_bits(x, (int64_t)J * K, K); }
    __device__ void tile(V (&acc)[NV], const uint32_t* w, uint32_t xs) const { acc[0] |= rows_hit<K>(w, xs); }
    __device__ void store(int32_t R, const V (&acc)[NV]) const {
        uint32_t v = acc[0];
        if (mask) {
            uint32_t mb = ld_bits(mask, (int64_t)R * K, K);
            v &= comp ? ~mb : mb;
        }
        if (K == 32) {
            y[R] = v;
        } else if (K == 16) {
            reinterpret_cast<uint16_t*>(y)[R] = (uint16_t)v;
        } else if (K == 8) {
            reinterpret_cast<uint8_t*>(y)[R] = (uint8_t)v;
        } else {
            // two tile-rows share a byte: update this nibble atomically
            int sh = (R & 7) * 4;
            atomicAnd(y + (R >> 3), ~(0xFu << sh));
            if (v & 0xFu) atomicOr(y + (R >> 3), (v & 0xFu) << sh);
        }
    }
};

// bmv_bin_bin_full[_masked]: bitset in, int32 counts out (popc of Sec. IV)
template <int K>
struct SemCount {
    using V = int32_t;
    static constexpr int NV = K;
    static constexpr bool kGather = false;
    const uint32_t* x;
    int32_t* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ V ident() const { return 0; }
    __device__ V comb(V a, V b) const { return a + b; }
    __device__ uint32_t xseg(int32_t J) const { return ld_bits(x, (int64_t)J * K, K); }
    __device__ void tile(V (&acc)[NV], const uint32_t* w, uint32_t xs) const {
#pragma unroll
        for (int r = 0; r < K; ++r) acc[r] += __popc(row_word<K>(w, r) & xs);
    }
    __device__ void store(int32_t R, const V (&acc)[NV]) const {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int64_t i = (int64_t)R * K + r;
            if (i < n) y[i] = mask_allows(mask, comp, i) ? acc[r] : 0;
        }
    }
};

// bmv_bin_full_full over plus-times: float in, float out
template <int K>
struct SemPlus {
    using V = float;
    using G = float;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    const float* x;
    float* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    static constexpr bool weighted = false;
    __device__ const float* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return 0.0f; }
    __device__ V comb(V a, V b) const { return a + b; }
    __device__ V apply(V acc, G xv, float) const { return acc + xv; }
    __device__ void store(int32_t R, const V (&acc)[NV]) const {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int64_t i = (int64_t)R * K + r;
            if (i < n) y[i] = mask_allows(mask, comp, i) ? acc[r] : 0.0f;
        }
    }
};

// bmv_bin_full_full over min-plus (relaxation, Sec. V SSSP): float in/out;
// weights in set-bit order (voff[t] = set bits before tile t), or w = 1
template <int K>
struct SemMinPlus {
    using V = float;
    using G = float;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    const float* x;
    float* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    const float* w;
    const int32_t* voff;
    bool weighted;
    __device__ const float* src() const { return x; }
    __device__ const float* wts() const { return w; }
    __device__ const int32_t* voffs() const { return voff; }
    __device__ V ident() const { return INFINITY; }
    __device__ V comb(V a, V b) const { return fminf(a, b); }
    __device__ V apply(V acc, G xv, float wv) const { return fminf(acc, xv + wv); }
    __device__ void store(int32_t R, const V (&acc)[NV]) const {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int64_t i = (int64_t)R * K + r;
            if (i < n) y[i] = mask_allows(mask, comp, i) ? fminf(__ldg(x + i), acc[r]) : INFINITY;
        }
    }
};

// min over neighbours of int32 labels (min-plus with weight 0: the CC step)
template <int K>
struct SemMinI32 {
    using V = int32_t;
    using G = int32_t;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    const int32_t* x;
    int32_t* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    static constexpr bool weighted = false;
    __device__ const int32_t* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return INT_MAX; }
    __device__ V comb(V a, V b) const { return min(a, b); }
    __device__ V apply(V acc, G xv, float) const { return min(acc, xv); }
    __device__ void store(int32_t R, const V (&acc)[NV]) const {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int64_t i = (int64_t)R * K + r;
            if (i < n) y[i] = mask_allows(mask, comp, i) ? min(__ldg(x + i), acc[r]) : INT_MAX;
        }
    }
};

// 64 Boolean frontiers per vertex: Y_i = OR_j X_j, masked by M_i or ~M_i
template <int K>
struct SemOr64 {
    using V = unsigned long long;
    using G = unsigned long long;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    const unsigned long long* x;
    unsigned long long* y;
    const unsigned long long* mask;
    int comp;
    int32_t n;
    static constexpr bool weighted = false;
    __device__ const unsigned long long* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return 0ull; }
    __device__ V comb(V a, V b) const { return a | b; }
    __device__ V apply(V acc, G xv, float) const { return acc | xv; }
    __device__ void store(int32_t R, const V (&acc)[NV]) const {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int64_t i = (int64_t)R * K + r;
            if (i < n) {
                V v = acc[r];
                if (mask) v &= comp ? ~__ldg(mask + i) : __ldg(mask + i);
                y[i] = v;
            }
        }
    }
};

// ---------------------------------------------------------------------------
// kernel arguments
// ---------------------------------------------------------------------------
struct SpmvGeom {
    const int32_t* rowptr;
    const int32_t* colind;
    const uint8_t* tiles;
    const int32_t* chunk_row;
    int64_t T;
    int64_t nchunks;
    int32_t ntr;
};

template <class V>
struct Partials {
    V* val_first;  // [nchunks * NV]: the chunk's first row, begun in an earlier chunk
    V* val_last;   // [nchunks * NV]: the chunk's last row, continued in a later chunk
};

template <int BYTES>
__device__ __forceinline__ void cp_async_gather(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kSpmvThreads = 256;
constexpr int kSpmvWarps = kSpmvThreads / 32;
// gathered values staged per warp (set bits of one chunk); the rest are read directly
template <class G>
struct GatherSlots {
    static constexpr int N = sizeof(G) == 8 ? 512 : 1024;
};

template <class SEM, bool GATHER = SEM::kGather>
struct SmemPerWarp {
    static constexpr int bytes = 0;
};
template <class SEM>
struct SmemPerWarp<SEM, true> {
    using G = typename SEM::G;
    static constexpr int bytes = GatherSlots<G>::N * (int)sizeof(G) + GatherSlots<G>::N * 4;
};

// One warp per chunk of 32*P consecutive tiles; lane l owns tiles
// [cs + l*P, cs + l*P + P).
template <int K, class SEM>
__global__ void __launch_bounds__(kSpmvThreads) spmv_chunks_kernel(SpmvGeom g, SEM sem,
                                                                   Partials<typename SEM::V> part) {
    using S = ChunkShape<K>;
    using V = typename SEM::V;
    constexpr int NV = SEM::NV;
    constexpr int P = S::P;
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    const int64_t c = (int64_t)blockIdx.x * kSpmvWarps + warp;
    if (c >= g.nchunks) return;

    const int64_t cs = c * S::CT;
    const int64_t ce = min(cs + (int64_t)S::CT, g.T);
    const int64_t tl = cs + (int64_t)lane * P;
    const int cnt = (int)max((int64_t)0, min((int64_t)P, ce - tl));

    // ---- issue every load of the lane first: tiles, tile columns ----
    uint4 tv[S::TILE_V4];
    {
        const uint4* src = reinterpret_cast<const uint4*>(g.tiles + tl * S::TB);
#pragma unroll
        for (int q = 0; q < S::TILE_V4; ++q) tv[q] = __ldg(src + q);
    }
    const uint32_t* words = reinterpret_cast<const uint32_t*>(tv);
    int32_t col[P];
    if (P % 4 == 0) {
        const int4* src = reinterpret_cast<const int4*>(g.colind + tl);
#pragma unroll
        for (int q = 0; q < P / 4; ++q) {
            int4 v = __ldg(src + q);
            col[4 * q] = v.x; col[4 * q + 1] = v.y; col[4 * q + 2] = v.z; col[4 * q + 3] = v.w;
        }
    } else {
        const int2* src = reinterpret_cast<const int2*>(g.colind + tl);
#pragma unroll
        for (int q = 0; q < P / 2; ++q) {
            int2 v = __ldg(src + q);
            col[2 * q] = v.x; col[2 * q + 1] = v.y;
        }
    }
    const int32_t r0 = __ldg(g.chunk_row + c);
    const int32_t r1 = __ldg(g.chunk_row + c + 1);

    // ---- input values: one k-bit segment per tile, or one value per set bit ----
    uint32_t xs[SEM::kGather ? 1 : P];
    int gbase = 0;
    if constexpr (!SEM::kGather) {
#pragma unroll
        for (int i = 0; i < P; ++i) xs[i] = sem.xseg(col[i]);
    } else {
        using G = typename SEM::G;
        constexpr int NG = GatherSlots<G>::N;
        G* sx = reinterpret_cast<G*>(smem + warp * SmemPerWarp<SEM>::bytes);
        float* sw = reinterpret_cast<float*>(sx + NG);
        int nb = 0;
#pragma unroll
        for (int i = 0; i < P; ++i)
            if (i < cnt) {
#pragma unroll
                for (int q = 0; q < S::TW; ++q) nb += __popc(words[i * S::TW + q]);
            }
        int incl = nb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        gbase = incl - nb;
        int s = gbase;
        const G* xsrc = sem.src();
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (i < cnt && s < NG) {
                const G* xt = xsrc + (int64_t)col[i] * K;
                const float* wt = sem.weighted ? sem.wts() + __ldg(sem.voffs() + tl + i) : nullptr;
                int qb = 0;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    uint32_t b = row_word<K>(words + i * S::TW, r);
                    while (b && s < NG) {
                        const int cc = __ffs(b) - 1;
                        b &= b - 1;
                        cp_async_gather<sizeof(G)>(sx + s, xt + cc);
                        if (sem.weighted) cp_async_gather<4>(sw + s, wt + qb);
                        ++s;
                        ++qb;
                    }
                }
            }
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
    }

    // ---- tile-row of the lane's first tile: rows r0..r1 span the chunk ----
    int32_t row = r0;
    if (r1 > r0) {
        const int32_t span = r1 - r0;
        int32_t add = 0;
        for (int32_t base = 0; base < span; base += 32) {
            const int32_t j = base + lane;
            const int64_t b = j < span ? (int64_t)__ldg(g.rowptr + r0 + 1 + j) : INT64_MAX;
            // count of boundaries b_j <= tl (b is sorted across lanes)
            int pos = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                int64_t v = __shfl_sync(0xffffffffu, b, pos + step - 1);
                if (v <= tl) pos += step;
            }
            pos += (__shfl_sync(0xffffffffu, b, pos) <= tl) ? 1 : 0;
            add += pos;
            if (__shfl_sync(0xffffffffu, b, 31) > cs + 32 * P) break;  // later windows start past the chunk
        }
        row = r0 + add;
    }

    const bool head_cs = (int64_t)__ldg(g.rowptr + r0) == cs;
    V acc[NV], F[NV], idv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { acc[v] = sem.ident(); F[v] = sem.ident(); idv[v] = sem.ident(); }
    const int32_t first_row = row;
    bool has_end = false;
    bool open = false;
    if (cnt > 0) {
        // empty tile-rows just before a row that starts at this lane's first tile
        if (tl > 0 && (int64_t)__ldg(g.rowptr + row) == tl)
            for (int32_t R = row - 1; R >= 0 && (int64_t)__ldg(g.rowptr + R) == tl; --R) sem.store(R, idv);
        int64_t next = __ldg(g.rowptr + row + 1);
        int s = gbase;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (i < cnt) {
                const int64_t t = tl + i;
                if constexpr (!SEM::kGather) {
                    sem.tile(acc, words + i * S::TW, xs[i]);
                } else {
                    using G = typename SEM::G;
                    constexpr int NG = GatherSlots<G>::N;
                    const G* sx = reinterpret_cast<const G*>(smem + warp * SmemPerWarp<SEM>::bytes);
                    const float* sw = reinterpret_cast<const float*>(sx + NG);
                    const G* xt = sem.src() + (int64_t)col[i] * K;
                    const float* wt = sem.weighted ? sem.wts() + __ldg(sem.voffs() + t) : nullptr;
                    int qb = 0;
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        uint32_t b = row_word<K>(words + i * S::TW, r);
                        while (b) {
                            const int cc = __ffs(b) - 1;
                            b &= b - 1;
                            G xv;
                            float wv = 1.0f;
                            if (s < NG) {
                                xv = sx[s];
                                if (sem.weighted) wv = sw[s];
                            } else {
                                xv = __ldg(xt + cc);
                                if (sem.weighted) wv = __ldg(wt + qb);
                            }
                            acc[r] = sem.apply(acc[r], xv, wv);
                            ++s;
                            ++qb;
                        }
                    }
                }
                open = true;
                if (t + 1 == next) {  // tile-row `row` ends with tile t
                    if (!has_end) {
#pragma unroll
                        for (int v = 0; v < NV; ++v) F[v] = acc[v];
                        has_end = true;
                    } else {
                        sem.store(row, acc);
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) acc[v] = sem.ident();
                    open = false;
                    if (i + 1 < cnt) {
                        int32_t R = row + 1;
                        while ((int64_t)__ldg(g.rowptr + R + 1) == next) { sem.store(R, idv); ++R; }
                        row = R;
                        next = __ldg(g.rowptr + row + 1);
                    }
                }
            }
        }
    }

    // Warp segmented scan of (reset = has_end, value = acc): the open value
    // carried into each lane, joined in lane order.
    bool inc_r = has_end;
    V inc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) inc[v] = acc[v];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const bool o_r = __shfl_up_sync(0xffffffffu, inc_r, d);
        const bool take = lane >= d && !inc_r;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            V o = __shfl_up_sync(0xffffffffu, inc[v], d);
            if (take) inc[v] = sem.comb(o, inc[v]);
        }
        if (take) inc_r = o_r;
    }
    bool ex_r = __shfl_up_sync(0xffffffffu, inc_r, 1);
    if (lane == 0) ex_r = false;
    // the value carried into this lane joins its first segment (every lane
    // takes part in the shuffles; only lanes that close a row use them)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const V o = __shfl_up_sync(0xffffffffu, inc[v], 1);
        if (has_end && lane > 0) F[v] = sem.comb(o, F[v]);
    }
    if (has_end) {
        // this lane closes the tile-row of its first tile
        if (ex_r || head_cs) {
            sem.store(first_row, F);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) part.val_first[c * NV + v] = F[v];
        }
    }

    // chunk tail: the segment still open after the last active lane
    const int la = (int)((ce - 1 - cs) / P);
    const bool tail_open = __shfl_sync(0xffffffffu, open, la);
    const bool tail_r = __shfl_sync(0xffffffffu, inc_r, 31);
    if (lane == 31 && tail_open) {
        if (tail_r || head_cs) {
#pragma unroll
            for (int v = 0; v < NV; ++v) part.val_last[c * NV + v] = inc[v];
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) part.val_first[c * NV + v] = inc[v];
        }
    }
}

// Rows that span chunks: the chunk where such a row ends joins the partials
// of every chunk the row touches, in chunk order, and stores the row.
template <int K, class SEM>
__global__ void spmv_fixup_kernel(SpmvGeom g, SEM sem, Partials<typename SEM::V> part) {
    using S = ChunkShape<K>;
    using V = typename SEM::V;
    constexpr int NV = SEM::NV;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; c < g.nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cs = c * S::CT;
        const int64_t ce = min(cs + (int64_t)S::CT, g.T);
        const int32_t R = g.chunk_row[c];
        const int64_t rs = g.rowptr[R], re = g.rowptr[R + 1];
        if (rs >= cs || re > ce) continue;  // R starts here, or does not end here
        const int64_t ca = rs / S::CT;
        V acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = part.val_last[ca * NV + v];
        for (int64_t q = ca + 1; q <= c; ++q) {
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = sem.comb(acc[v], part.val_first[q * NV + v]);
        }
        sem.store(R, acc);
    }
}

// Plus-times specialisation of the join: fp64 accumulation of the partials.
template <int K>
__global__ void spmv_fixup_plus_kernel(SpmvGeom g, SemPlus<K> sem, Partials<float> part) {
    using S = ChunkShape<K>;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; c < g.nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cs = c * S::CT;
        const int64_t ce = min(cs + (int64_t)S::CT, g.T);
        const int32_t R = g.chunk_row[c];
        const int64_t rs = g.rowptr[R], re = g.rowptr[R + 1];
        if (rs >= cs || re > ce) continue;
        const int64_t ca = rs / S::CT;
        double acc[K];
#pragma unroll
        for (int v = 0; v < K; ++v) acc[v] = (double)part.val_last[ca * K + v];
        for (int64_t q = ca + 1; q <= c; ++q) {
#pragma unroll
            for (int v = 0; v < K; ++v) acc[v] += (double)part.val_first[q * K + v];
        }
        float out[K];
#pragma unroll
        for (int v = 0; v < K; ++v) out[v] = (float)acc[v];
        sem.store(R, out);
    }
}

// Tile-rows before the first tile and after the last one (and every row when
// the matrix has no tiles) get the identity; for bitset outputs the words past
// the last tile-row are cleared.
template <int K, class SEM>
__global__ void spmv_edges_kernel(SEM sem, int32_t lead_end, int32_t trail_begin, int32_t ntr) {
    using V = typename SEM::V;
    V idv[SEM::NV];
#pragma unroll
    for (int v = 0; v < SEM::NV; ++v) idv[v] = sem.ident();
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t R = tid; R < lead_end; R += stride) sem.store((int32_t)R, idv);
    for (int64_t R = trail_begin + tid; R < ntr; R += stride) sem.store((int32_t)R, idv);
}

// Bitset outputs: the bits past the last tile-row (>= nTileRow*k) are never
// stored by a row, so the word holding them is cleared before the rows land.
template <int K>
static b2sr_status clear_bitset_tail(const b2sr_matrix* h, uint32_t* bits, cudaStream_t s) {
    int64_t words = ceil_div(h->n, 32);
    int64_t first = ((int64_t)h->ntr * K) / 32;
    if (first < words) B2SR_CUDA_TRY(cudaMemsetAsync(bits + first, 0, (words - first) * sizeof(uint32_t), s));
    return B2SR_OK;
}

template <int K, class SEM>
static b2sr_status launch_edges(const b2sr_matrix* h, const SEM& sem, cudaStream_t s) {
    int32_t lead_end = h->T == 0 ? h->ntr : h->first_row;
    int32_t trail_begin = h->T == 0 ? h->ntr : h->last_row + 1;
    int64_t work = (int64_t)lead_end + (h->ntr - trail_begin);
    if (work <= 0) return B2SR_OK;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)sm_count() * 4));
    spmv_edges_kernel<K, SEM><<<grid, 256, 0, s>>>(sem, lead_end, trail_begin, h->ntr);
    B2SR_LAUNCH_CHECK("spmv_edges_kernel");
    return B2SR_OK;
}

template <int K, class SEM>
static b2sr_status launch_chunks(const b2sr_matrix* h, const SpmvGeom& g, const SEM& sem,
                                 Partials<typename SEM::V> part, cudaStream_t s) {
    const int smem = kSpmvWarps * SmemPerWarp<SEM>::bytes;
    if (smem > 48 * 1024)
        B2SR_CUDA_TRY(cudaFuncSetAttribute(spmv_chunks_kernel<K, SEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int64_t blocks = ceil_div(h->nchunks, kSpmvWarps);
    spmv_chunks_kernel<K, SEM><<<(unsigned)blocks, kSpmvThreads, smem, s>>>(g, sem, part);
    B2SR_LAUNCH_CHECK("spmv_chunks_kernel");
    return B2SR_OK;
}

template <class V, int NV>
static b2sr_status alloc_partials(DevBuf& pbuf, int64_t nchunks, Partials<V>* part) {
    const size_t vbytes = round_up((size_t)nchunks * NV * sizeof(V), 16);
    B2SR_TRY(pbuf.alloc(2 * vbytes));
    uint8_t* base = pbuf.as<uint8_t>();
    part->val_first = reinterpret_cast<V*>(base);
    part->val_last = reinterpret_cast<V*>(base + vbytes);
    return B2SR_OK;
}

template <int K, class SEM>
static b2sr_status run_spmv(const b2sr_matrix* h, const SEM& sem, uint32_t* bits_out, cudaStream_t s) {
    using V = typename SEM::V;
    SpmvGeom g{h->rowptr, h->colind, h->tiles, h->chunk_row, h->T, h->nchunks, h->ntr};
    if (bits_out) B2SR_TRY(clear_bitset_tail<K>(h, bits_out, s));
    B2SR_TRY((launch_edges<K, SEM>(h, sem, s)));
    if (h->nchunks == 0) return B2SR_OK;
    DevBuf pbuf(s);
    Partials<V> part;
    B2SR_TRY((alloc_partials<V, SEM::NV>(pbuf, h->nchunks, &part)));
    B2SR_TRY((launch_chunks<K, SEM>(h, g, sem, part, s)));
    if (h->nchunks > 1) {
        int fgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->nchunks, 128), (int64_t)sm_count() * 8));
        spmv_fixup_kernel<K, SEM><<<fgrid, 128, 0, s>>>(g, sem, part);
        B2SR_LAUNCH_CHECK("spmv_fixup_kernel");
    }
    return B2SR_OK;
}

template <int K>
static b2sr_status run_spmv_plus(const b2sr_matrix* h, const SemPlus<K>& sem, cudaStream_t s) {
    SpmvGeom g{h->rowptr, h->colind, h->tiles, h->chunk_row, h->T, h->nchunks, h->ntr};
    B2SR_TRY((launch_edges<K, SemPlus<K>>(h, sem, s)));
    if (h->nchunks == 0) return B2SR_OK;
    DevBuf pbuf(s);
    Partials<float> part;
    B2SR_TRY((alloc_partials<float, K>(pbuf, h->nchunks, &part)));
    B2SR_TRY((launch_chunks<K, SemPlus<K>>(h, g, sem, part, s)));
    if (h->nchunks > 1) {
        int fgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->nchunks, 128), (int64_t)sm_count() * 8));
        spmv_fixup_plus_kernel<K><<<fgrid, 128, 0, s>>>(g, sem, part);
        B2SR_LAUNCH_CHECK("spmv_fixup_plus_kernel");
    }
    return B2SR_OK;
}

template <class F>
static b2sr_status with_k(int k, F&& f) {
    switch (k) {
        case 4: return f(std::integral_constant<int, 4>());
        case 8: return f(std::integral_constant<int, 8>());
        case 16: return f(std::integral_constant<int, 16>());
        case 32: return f(std::integral_constant<int, 32>());
        default: return fail(B2SR_ERR_UNSUPPORTED_TILE, "bad tile_dim");
    }
}

b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s) {
    comp = comp ? 1 : 0;
    if (sr == B2SR_BOOL_OR_AND && in_kind == B2SR_VEC_BITS && out_kind == B2SR_VEC_BITS) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_k(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemBool<K> sem{static_cast<const uint32_t*>(x), static_cast<uint32_t*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, static_cast<uint32_t*>(y), s);
        });
    }
    if (sr == B2SR_PLUS_TIMES && in_kind == B2SR_VEC_BITS && out_kind == B2SR_VEC_I32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_k(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemCount<K> sem{static_cast<const uint32_t*>(x), static_cast<int32_t*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, nullptr, s);
        });
    }
    if (sr == B2SR_PLUS_TIMES && in_kind == B2SR_VEC_F32 && out_kind == B2SR_VEC_F32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_k(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemPlus<K> sem{static_cast<const float*>(x), static_cast<float*>(y), mask, comp, h->n};
            return run_spmv_plus<K>(h, sem, s);
        });
    }
    if (sr == B2SR_MIN_PLUS && in_kind == B2SR_VEC_F32 && out_kind == B2SR_VEC_F32) {
        if (weights) B2SR_TRY(ensure_voff(h, s));
        return with_k(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemMinPlus<K> sem{static_cast<const float*>(x), static_cast<float*>(y), mask, comp, h->n, weights,
                              h->voff, weights != nullptr};
            return run_spmv<K>(h, sem, nullptr, s);
        });
    }
    if (sr == B2SR_MIN_PLUS && in_kind == B2SR_VEC_I32 && out_kind == B2SR_VEC_I32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "int32 MIN_PLUS takes no weights (all weights are 0)");
        return with_k(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemMinI32<K> sem{static_cast<const int32_t*>(x), static_cast<int32_t*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, nullptr, s);
        });
    }
    return fail(B2SR_ERR_INVALID_ARG, "unsupported semiring / vector kind combination");
}

b2sr_status spmm64_dispatch(b2sr_matrix* h, const uint64_t* X, uint64_t* Y, const uint64_t* M, int comp,
                            cudaStream_t s) {
    return with_k(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        SemOr64<K> sem{reinterpret_cast<const unsigned long long*>(X), reinterpret_cast<unsigned long long*>(Y),
                       reinterpret_cast<const unsigned long long*>(M), comp ? 1 : 0, h->n};
        return run_spmv<K>(h, sem, nullptr, s);
    });
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_spmv(b2sr_handle h, b2sr_semiring semiring, b2sr_vec in_kind, const void* x,
                                 b2sr_vec out_kind, void* y, const uint32_t* mask, int mask_complement,
                                 const float* weights, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!x || !y)) return fail(B2SR_ERR_INVALID_ARG, "x or y is NULL");
    if (x == y) return fail(B2SR_ERR_INVALID_ARG, "y must not alias x");
    return spmv_dispatch(h, semiring, in_kind, x, out_kind, y, mask, mask_complement, weights, to_stream(stream));
}

extern "C" b2sr_status b2sr_spmm_bits64(b2sr_handle h, const uint64_t* X, uint64_t* Y, const uint64_t* M,
                                        int complement, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!X || !Y)) return fail(B2SR_ERR_INVALID_ARG, "X or Y is NULL");
    if (X == Y) return fail(B2SR_ERR_INVALID_ARG, "Y must not alias X");
    return spmm64_dispatch(h, X, Y, M, complement, to_stream(stream));
}
