// B2SR SpMV: the BMV schemes of Table 2 over the semirings of Table 4, and the
// 64-lane Boolean SpMM used by multi-source BFS.
//
// Design (GB300).  The paper maps one tile-row to one warp (Listing 1) or 32
// tile-rows to a 1024-thread block (Sec. IV, bmv_bin_full_full).  Power-law
// graphs make any row mapping badly imbalanced (a scale-20 R-MAT tile-row can
// hold 10^5 tiles), so the unit of work here is a fixed-size chunk of
// consecutive tiles:
//   * one warp per chunk of 32*P tiles; lane l owns P consecutive tiles and
//     issues every load it needs up front (its tiles and tile columns as
//     16-byte vectors, then the input segments or, for full-precision
//     vectors, one 4/8-byte cp.async gather per set bit into shared memory),
//     so each warp keeps several KB in flight;
//   * the lane walks its tiles in order, accumulating the k row results of
//     the current tile-row and storing every row that starts and ends inside
//     the lane (and the identity for empty tile-rows it passes);
//   * rows that cross lanes are joined with a warp segmented scan (shuffles,
//     fixed order); rows that cross chunks leave per-chunk partials that a
//     second kernel joins, one warp per row, in a fixed order.
// Every reduction order is fixed by the data, so floating-point results are
// bitwise reproducible and independent of launch geometry and stream.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>
#include <string>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "tile_bits.cuh"

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
    static constexpr int TILE_V4 = P * TB / 16;  // uint4 loads per lane for its tiles
    static constexpr int ROW_BITS = K <= 8 ? 8 : K;  // bits per row slot in a word
};

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

// Every output row in [r0, r1) is excluded by a bitset mask (bits all 0, or
// all 1 for a complemented mask): the masked store writes the semiring's
// identity there whatever the tiles hold.  Rows past n store nothing; spans
// of more than 2048 rows are not tested (false).
// Warp-collective.  Semirings whose masked calls sit on a level loop (BFS,
// MIS, colouring) use it; in the others the test's registers cost more
// occupancy than the skip saves, and saturated() is constant false.
__device__ __forceinline__ bool rows_masked_out(const uint32_t* __restrict__ mask, int comp, int32_t n, int64_t r0,
                                                int64_t r1) {
    if (!mask || r1 - r0 > 2048) return false;  // at most two mask words a lane
    r1 = min(r1, (int64_t)n);
    bool ok = true;
    for (int64_t w = (r0 >> 5) + lane_id(); w * 32 < r1; w += 32) {
        const int64_t lo = max(r0, w * 32), hi = min(r1, w * 32 + 32);
        const uint32_t need = (hi - lo >= 32) ? 0xFFFFFFFFu : (((1u << (hi - lo)) - 1u) << (lo - w * 32));
        const uint32_t m = comp ? __ldg(mask + w) : ~__ldg(mask + w);
        ok &= (m & need) == need;
    }
    return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------------------
// accumulator storage: registers (static row index) or shared memory (one
// column per lane, any row index)
// ---------------------------------------------------------------------------
template <class V, int NV>
struct RegAcc {
    V a[NV];
    __device__ __forceinline__ V get(int v) const { return a[v]; }
    __device__ __forceinline__ void set(int v, V x) { a[v] = x; }
};

template <class V, int NV>
struct SmemAcc {
    V* p;  // element v at p[v * 32]
    __device__ __forceinline__ V get(int v) const { return p[v * 32]; }
    __device__ __forceinline__ void set(int v, V x) { p[v * 32] = x; }
};

// ---------------------------------------------------------------------------
// warp shuffles of accumulator values (scalars, and the four-column blocks of
// SemPlus4 one component at a time)
// ---------------------------------------------------------------------------
// Join type of the plus-times partials of rows that cross chunks: a
// compensated fp32 sum.  Each addition is Knuth's TwoSum of the leading parts
// (the exact rounding error, whatever the magnitudes), added to the carried
// error terms; the rounding is spelled out so no contraction or reordering
// can change it.  fp32 keeps the join off the fp64 pipe, which is narrow on
// GB300; the compensation keeps it as accurate as an fp64 join for the few
// hundred partials a row can have.
struct CSum {
    float s, c;
    CSum() = default;
    __device__ __forceinline__ CSum(float a) : s(a), c(0.0f) {}
    __device__ __forceinline__ explicit operator float() const { return __fadd_rn(s, c); }
};

__device__ __forceinline__ CSum csum_add(CSum a, CSum b) {
    const float t = __fadd_rn(a.s, b.s);
    const float bp = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(b.s, bp));
    CSum r;
    r.s = t;
    r.c = __fadd_rn(__fadd_rn(a.c, b.c), e);
    return r;
}

struct CSum4 {  // the same for a four-column block, column by column
    CSum v[4];
    CSum4() = default;
    __device__ __forceinline__ CSum4(float4 a) : v{CSum(a.x), CSum(a.y), CSum(a.z), CSum(a.w)} {}
    __device__ __forceinline__ explicit operator float4() const {
        return make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    }
};

template <class T>
__device__ __forceinline__ T shfl_up(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <class T>
__device__ __forceinline__ T shfl_xor(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float4 shfl_up(float4 v, int d) {
    return make_float4(shfl_up(v.x, d), shfl_up(v.y, d), shfl_up(v.z, d), shfl_up(v.w, d));
}
__device__ __forceinline__ float4 shfl_xor(float4 v, int o) {
    return make_float4(shfl_xor(v.x, o), shfl_xor(v.y, o), shfl_xor(v.z, o), shfl_xor(v.w, o));
}
__device__ __forceinline__ CSum shfl_xor(CSum a, int o) {
    CSum r;
    r.s = shfl_xor(a.s, o);
    r.c = shfl_xor(a.c, o);
    return r;
}
__device__ __forceinline__ CSum4 shfl_xor(CSum4 a, int o) {
    CSum4 r;
#pragma unroll
    for (int i = 0; i < 4; ++i) r.v[i] = shfl_xor(a.v[i], o);
    return r;
}

// ---------------------------------------------------------------------------
// semirings.  Each provides V (accumulator value), NV (values per tile-row
// accumulator), ident(), comb(a, b) (a earlier in the fixed order),
// store(R, acc) (self term, mask, overwrite; empty tile-rows are stored with
// the identity) and a join type J for the cross-chunk join.
//   bit-vector schemes (kGather = false): xseg(J) and tile(acc, words, xs);
//   value schemes (kGather = true): one gathered input per set bit, src(),
//     weighted, wts(), voffs() and apply(acc, x_j, w_ij).
// ---------------------------------------------------------------------------

// Row mask of OR-accumulated, input-masked tile words (k <= 8: a row per
// byte): bit r is set iff byte r is non-zero.  The non-zero bytes get their
// high bit, and one multiply gathers the four high bits of a word.
template <int K>
__device__ __forceinline__ uint32_t nonzero_rows(const uint32_t* w) {
    uint32_t out = 0;
#pragma unroll
    for (int q = 0; q < K / 4; ++q) {
        const uint32_t m = w[q];
        const uint32_t h = (((m & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | m) & 0x80808080u;
        out |= (((h >> 7) * 0x00204081u) >> 21 & 0xFu) << (4 * q);
    }
    return out;
}

// bmv_bin_bin_bin[_masked]: bitset in, bitset out.  For k <= 8 the
// accumulator is the OR of the tile words ANDed with the input segment (one
// word per four rows); OR commutes with "row is non-zero", so the row mask is
// formed only when a row is stored.  For k >= 16 it is the k-bit row mask.
template <int K>
struct SemBool {
    using V = uint32_t;
    using J = uint32_t;
    static constexpr int NV = K <= 8 ? K / 4 : 1;
    static constexpr bool kGather = false;
    const uint32_t* x;
    uint32_t* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ V ident() const { return 0u; }
    __device__ V comb(V a, V b) const { return a | b; }
    __device__ J jcomb(J a, J b) const { return a | b; }
    __device__ uint32_t xseg(int32_t Jc) const { return ld_bits(x, (int64_t)Jc * K, K); }
    __device__ bool saturated(int64_t r0, int64_t r1) const { return rows_masked_out(mask, comp, n, r0, r1); }
    template <class A>
    __device__ void tile(A& acc, const uint32_t* w, uint32_t xs) const {
        if constexpr (K <= 8) {
            const uint32_t rep = xs * 0x01010101u;
#pragma unroll
            for (int q = 0; q < NV; ++q) acc.set(q, acc.get(q) | (w[q] & rep));
        } else {
            acc.set(0, acc.get(0) | rows_hit<K>(w, xs));
        }
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
        uint32_t v;
        if constexpr (K <= 8) {
            uint32_t w[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) w[q] = acc.get(q);
            v = nonzero_rows<K>(w);
        } else {
            v = acc.get(0);
        }
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
    using J = int32_t;
    static constexpr int NV = K;
    static constexpr bool kGather = false;
    const uint32_t* x;
    int32_t* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ V ident() const { return 0; }
    __device__ V comb(V a, V b) const { return a + b; }
    __device__ J jcomb(J a, J b) const { return a + b; }
    __device__ uint32_t xseg(int32_t Jc) const { return ld_bits(x, (int64_t)Jc * K, K); }
    __device__ bool saturated(int64_t, int64_t) const { return false; }
    template <class A>
    __device__ void tile(A& acc, const uint32_t* w, uint32_t xs) const {
#pragma unroll
        for (int r = 0; r < K; ++r) acc.set(r, acc.get(r) + __popc(tile_row<K>(w, r) & xs));
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int64_t i = (int64_t)R * K + r;
            if (i < n) y[i] = mask_allows(mask, comp, i) ? acc.get(r) : 0;
        }
    }
};

// bmv_bin_full_full over plus-times: float in, float out; partials of rows
// that cross chunks are joined with a compensated fp32 sum (CSum)
template <int K>
struct SemPlus {
    using V = float;
    using G = float;
    using J = CSum;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kMayWeight = false;
    static constexpr bool weighted = false;
    const float* x;
    float* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ const float* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return 0.0f; }
    __device__ V comb(V a, V b) const { return a + b; }
    __device__ J jcomb(J a, J b) const { return csum_add(a, b); }
    __device__ V apply(V acc, G xv, float) const { return acc + xv; }
    __device__ V contrib(G xv, float) const { return xv; }
    __device__ bool saturated(int64_t, int64_t) const { return false; }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) y[i] = mask_allows(mask, comp, i) ? v : 0.0f;
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// plus-times over a block of four fp32 columns (vertex-major: x[v] holds the
// four columns' values of vertex v).  Every component is added in exactly the
// order SemPlus adds a single column, and joined the same way, so column b
// of the result is bitwise the SemPlus result for column b.
template <int K>
struct SemPlus4 {
    using V = float4;
    using G = float4;
    using J = CSum4;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kMayWeight = false;
    static constexpr bool weighted = false;
    const float4* x;
    float4* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ const float4* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
    __device__ V comb(V a, V b) const { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
    __device__ J jcomb(J a, J b) const {
        J r;
#pragma unroll
        for (int i = 0; i < 4; ++i) r.v[i] = csum_add(a.v[i], b.v[i]);
        return r;
    }
    __device__ V apply(V acc, G xv, float) const { return comb(acc, xv); }
    __device__ V contrib(G xv, float) const { return xv; }
    __device__ bool saturated(int64_t, int64_t) const { return false; }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) y[i] = mask_allows(mask, comp, i) ? v : ident();
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// bmv_bin_full_full over min-plus (relaxation, Sec. V SSSP): float in/out;
// weights in set-bit order (voff[t] = set bits before tile t), or w = 1.  The
// chunk kernels store the minimum over the neighbours; the diagonal's self
// term min(x_i, .) is applied by spmv_self_kernel once the rows are joined
// (kept out of the chunk kernels, where its extra load per row cost registers
// and spills)
template <int K>
struct SemMinPlus {
    using V = float;
    using G = float;
    using J = float;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kSelfTerm = true;  // x_i joins y_i in spmv_self_kernel
    static constexpr bool kMayWeight = true;
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
    __device__ J jcomb(J a, J b) const { return fminf(a, b); }
    __device__ V apply(V acc, G xv, float wv) const { return fminf(acc, xv + wv); }
    __device__ V contrib(G xv, float wv) const { return xv + wv; }
    __device__ bool saturated(int64_t, int64_t) const { return false; }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) y[i] = mask_allows(mask, comp, i) ? v : INFINITY;
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// min over neighbours of int32 labels (min-plus with weight 0: the CC step);
// the self term x_i is applied after the join, as for SemMinPlus
template <int K>
struct SemMinI32 {
    using V = int32_t;
    using G = int32_t;
    using J = int32_t;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kSelfTerm = true;
    static constexpr bool kMayWeight = false;
    static constexpr bool weighted = false;
    const int32_t* x;
    int32_t* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ const int32_t* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return INT_MAX; }
    __device__ V comb(V a, V b) const { return min(a, b); }
    __device__ J jcomb(J a, J b) const { return min(a, b); }
    __device__ V apply(V acc, G xv, float) const { return min(acc, xv); }
    __device__ V contrib(G xv, float) const { return xv; }
    __device__ bool saturated(int64_t, int64_t) const { return false; }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) y[i] = mask_allows(mask, comp, i) ? v : INT_MAX;
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// bmv_bin_full_full over tropical max-times (Table 4: the local-maximum step
// of MIS and colouring): y_i = max over neighbours j of x_j (A_ij = 1 is the
// multiplicative identity, so x_j passes unchanged); -inf where no neighbour
// or masked out.  max is exact, so the result does not depend on the order.
template <int K>
struct SemMaxF32 {
    using V = float;
    using G = float;
    using J = float;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kMayWeight = false;
    static constexpr bool weighted = false;
    const float* x;
    float* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ const float* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return -INFINITY; }
    __device__ V comb(V a, V b) const { return fmaxf(a, b); }
    __device__ J jcomb(J a, J b) const { return fmaxf(a, b); }
    __device__ V apply(V acc, G xv, float) const { return fmaxf(acc, xv); }
    __device__ V contrib(G xv, float) const { return xv; }
    __device__ bool saturated(int64_t, int64_t) const { return false; }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) y[i] = mask_allows(mask, comp, i) ? v : -INFINITY;
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// max over neighbours of 64-bit keys (priority bits above the vertex id: the
// local-maximum test of MIS and colouring with ties broken by id); 0 is
// below every key and stands for "no undecided neighbour"
template <int K>
struct SemMaxKey {
    using V = unsigned long long;
    using G = unsigned long long;
    using J = unsigned long long;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kMayWeight = false;
    static constexpr bool weighted = false;
    const unsigned long long* x;
    unsigned long long* y;
    const uint32_t* mask;
    int comp;
    int32_t n;
    __device__ const unsigned long long* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return 0ull; }
    __device__ V comb(V a, V b) const { return a > b ? a : b; }
    __device__ J jcomb(J a, J b) const { return a > b ? a : b; }
    __device__ V apply(V acc, G xv, float) const { return acc > xv ? acc : xv; }
    __device__ V contrib(G xv, float) const { return xv; }
    __device__ bool saturated(int64_t r0, int64_t r1) const { return rows_masked_out(mask, comp, n, r0, r1); }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) y[i] = mask_allows(mask, comp, i) ? v : 0ull;
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// Boolean frontiers packed in one word per vertex (lane b of X_j: vertex j is
// in frontier b): Y_i = OR_j X_j, masked by M_i or ~M_i
template <int K, class W>
struct SemOrLanes {
    using V = W;
    using G = W;
    using J = W;
    static constexpr int NV = K;
    static constexpr bool kGather = true;
    static constexpr bool kMayWeight = false;
    static constexpr bool weighted = false;
    const W* x;
    W* y;
    const W* mask;
    int comp;
    int32_t n;
    __device__ const W* src() const { return x; }
    __device__ const float* wts() const { return nullptr; }
    __device__ const int32_t* voffs() const { return nullptr; }
    __device__ V ident() const { return (W)0; }
    __device__ V comb(V a, V b) const { return a | b; }
    __device__ J jcomb(J a, J b) const { return a | b; }
    __device__ V apply(V acc, G xv, float) const { return acc | xv; }
    __device__ V contrib(G xv, float) const { return xv; }
    // Every output row in [r0, r1) is fully masked out (complemented mask of
    // all ones): zero whatever the tiles hold.  Warp-collective.
    __device__ bool saturated(int64_t r0, int64_t r1) const {
        if (!mask || !comp || r1 - r0 > 9 * K) return false;  // up to nine tile-rows
        r1 = min(r1, (int64_t)n);
        bool ok = true;
        for (int64_t i = r0 + lane_id(); i < r1; i += 32) ok &= __ldg(mask + i) == (W)~(W)0;
        return __all_sync(0xffffffffu, ok);
    }
    __device__ void store_row(int32_t R, int r, V v) const {
        int64_t i = (int64_t)R * K + r;
        if (i < n) {
            if (mask) v &= comp ? ~__ldg(mask + i) : __ldg(mask + i);
            y[i] = v;
        }
    }
    template <class A>
    __device__ void store(int32_t R, const A& acc) const {
#pragma unroll
        for (int r = 0; r < K; ++r) store_row(R, r, acc.get(r));
    }
};

// 64 and 32 lanes: the batched BFS packs up to 64 (or, for at most 32
// sources, 32) frontiers into one word per vertex.
template <int K>
using SemOr64 = SemOrLanes<K, unsigned long long>;
template <int K>
using SemOr32 = SemOrLanes<K, uint32_t>;

// ---------------------------------------------------------------------------
// kernel arguments and shared-memory layout
// ---------------------------------------------------------------------------
struct SpmvGeom {
    const int32_t* rowptr;
    const int32_t* colind;
    const uint8_t* tiles;
    const int32_t* chunk_row;
    int64_t T;
    int64_t nchunks;
    int32_t ntr;
    // optional device flag: when it reads 0 the launch does nothing (lets a
    // captured loop of SpMVs run past the point where its driver is done)
    const int32_t* gate;
};

__device__ __forceinline__ bool gated_off(const int32_t* gate) { return gate && *gate == 0; }

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

// Shared memory per warp for the gather schemes (k <= 16): the lanes' tile
// words and tile columns (lane-private, so the flat bit walk can index them),
// NG staged input values (+ NG weights for min-plus) and a one-byte
// (tile, row) tag per staged value.  A chunk with more than NG set bits reads
// its values straight from global memory instead.
template <int K, class SEM, bool GATHER = SEM::kGather>
struct GatherLayout {
    static constexpr int NG = 0;
    static constexpr int bytes = 0;
};
template <int K, class SEM>
struct GatherLayout<K, SEM, true> {
    using G = typename SEM::G;
    using S = ChunkShape<K>;
    // the same for every value type: whether a chunk is staged decides its
    // summation order, and the four-column block must sum like one column
    static constexpr int NG = 512;
    static constexpr int words_off = 0;                                    // [P*TW][32] u32
    static constexpr int col_off = words_off + S::CT * S::TW * 4;          // [P][32] i32
    static constexpr int x_off = col_off + S::CT * 4;                      // [NG] G
    static constexpr int w_off = x_off + NG * (int)sizeof(G);              // [NG] f32 (min-plus)
    static constexpr int tag_off = w_off + (SEM::kMayWeight ? NG * 4 : 0);  // [NG] u8
    static constexpr int pre_off = (tag_off + NG + 15) / 16 * 16;           // [P][32] i32: first slot of each tile
    static constexpr int bytes = pre_off + S::CT * 4;
    static_assert(x_off % 16 == 0 && bytes % 16 == 0, "16-byte staging slots");
};

// ---------------------------------------------------------------------------
// pieces shared by the chunk kernels
// ---------------------------------------------------------------------------
// Tile indices fit in int32 (T < 2^31: TileColInd and TileRowPtr are int32),
// which keeps the walk's compares and shuffles single-word.
struct LaneSpan {
    int32_t cs, ce, tl;
    int cnt;
};

// Tile-row of the lane's first tile, and rowptr[row], rowptr[row+1]; the
// chunk's rows r0..r1 come from the schedule, a window of row pointers from
// one coalesced load, and the search is a shuffle binary search.
struct RowCursor {
    int32_t row;
    int32_t row_start, next;
    bool head_cs;
};

// Row pointers of a chunk's tile-rows r0 .. r0+span+1 that fit one warp
// (lane j holds rowptr[r0 + j]); the search loads any further windows itself.
__device__ __forceinline__ int32_t row_window(const SpmvGeom& g, int32_t r0, int32_t span, int lane) {
    return lane <= span + 1 ? __ldg(g.rowptr + r0 + lane) : INT32_MAX;
}

__device__ __forceinline__ RowCursor locate_row_win(const SpmvGeom& g, int32_t r0, int32_t span, int32_t win,
                                                    const LaneSpan& ls, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    RowCursor rc;
    rc.head_cs = __shfl_sync(FULL, win, 0) == ls.cs;
    int32_t row = r0;
    if (span > 0) {
        // first window: the row starts are lanes 1..31 (lane 0 is rowptr[r0])
        const int32_t b = lane == 0 ? INT32_MIN : win;
        int pos = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int32_t v = __shfl_sync(FULL, b, pos + step - 1);
            if (v <= ls.tl) pos += step;
        }
        pos += (__shfl_sync(FULL, b, pos) <= ls.tl) ? 1 : 0;
        int32_t add = pos - 1;  // lane 0 is always counted
        int32_t last = __shfl_sync(FULL, win, 31);
        for (int32_t base = 32; base <= span && last < ls.ce; base += 32) {
            // further windows (rare: many tile-rows in one chunk)
            const int32_t j = base + lane;
            const int32_t bb = j <= span ? __ldg(g.rowptr + r0 + j) : INT32_MAX;
            int p2 = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int32_t v = __shfl_sync(FULL, bb, p2 + step - 1);
                if (v <= ls.tl) p2 += step;
            }
            p2 += (__shfl_sync(FULL, bb, p2) <= ls.tl) ? 1 : 0;
            add += p2;
            last = __shfl_sync(FULL, bb, 31);
        }
        row = r0 + add;
    }
    const int d = row - r0;
    const int32_t a0 = __shfl_sync(FULL, win, d < 32 ? d : 0);
    const int32_t a1 = __shfl_sync(FULL, win, d + 1 < 32 ? d + 1 : 0);
    rc.row = row;
    rc.row_start = d < 32 ? a0 : __ldg(g.rowptr + row);
    rc.next = d + 1 < 32 ? a1 : __ldg(g.rowptr + row + 1);
    return rc;
}

__device__ __forceinline__ RowCursor locate_row(const SpmvGeom& g, int32_t c, const LaneSpan& ls, int lane) {
    const int32_t r0 = __ldg(g.chunk_row + c);
    const int32_t span = __ldg(g.chunk_row + c + 1) - r0;
    return locate_row_win(g, r0, span, row_window(g, r0, span, lane), ls, lane);
}

// Per-lane walk state: the tile-row being accumulated, where it ends, the
// values of the lane's first tile-row (F) once that row has ended.
template <class SEM, class Acc>
struct Walk {
    int32_t row;
    int32_t next;
    bool has_end = false;
    bool open = false;
    // called after tile t (the lane's i-th of cnt) has been accumulated
    __device__ __forceinline__ void end_tile(const SpmvGeom& g, const SEM& sem, Acc& acc, Acc& F, int32_t t, int i,
                                             int cnt, const RegAcc<typename SEM::V, SEM::NV>& idv) {
        open = true;
        if (t + 1 == next) {  // tile-row `row` ends with tile t
            if (!has_end) {
#pragma unroll
                for (int v = 0; v < SEM::NV; ++v) F.set(v, acc.get(v));
                has_end = true;
            } else {
                sem.store(row, acc);
            }
#pragma unroll
            for (int v = 0; v < SEM::NV; ++v) acc.set(v, sem.ident());
            open = false;
            if (i + 1 < cnt) {
                int32_t R = row + 1;
                while (__ldg(g.rowptr + R + 1) == next) { sem.store(R, idv); ++R; }
                row = R;
                next = __ldg(g.rowptr + row + 1);
            }
        }
    }
};

// Warp segmented scan of (reset = has_end, value = acc), then: lanes that end
// their first tile-row store it (or leave it as the chunk's first partial if
// it began in an earlier chunk); lane 31 leaves the still-open tail.
template <class SEM, class Acc>
__device__ __forceinline__ void close_chunk(const SEM& sem, Partials<typename SEM::V> part, int64_t c,
                                            const LaneSpan& ls, int lane, bool head_cs, int32_t first_row,
                                            bool has_end, bool open, Acc& acc, Acc& F, int P) {
    using V = typename SEM::V;
    constexpr int NV = SEM::NV;
    constexpr unsigned FULL = 0xffffffffu;
    // The reset pattern does not depend on the values, so which scan steps
    // take a neighbour's value is worked out once, then applied per value.
    bool take[5];
    bool inc_r = has_end;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int d = 1 << k;
        const bool o = __shfl_up_sync(FULL, inc_r, d);
        take[k] = lane >= d && !inc_r;
        if (take[k]) inc_r = o;
    }
    bool ex_r = __shfl_up_sync(FULL, inc_r, 1);
    if (lane == 0) ex_r = false;
    const int la = (int)((ls.ce - 1 - ls.cs) / P);
    const bool tail_open = __shfl_sync(FULL, open, la);
    const bool tail_r = __shfl_sync(FULL, inc_r, 31);
    const bool close_here = has_end && (ex_r || head_cs);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        V x = acc.get(v);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const V o = shfl_up(x, 1 << k);
            if (take[k]) x = sem.comb(o, x);
        }
        const V ex = shfl_up(x, 1);
        if (has_end && lane > 0) F.set(v, sem.comb(ex, F.get(v)));
        if (has_end && !close_here) part.val_first[c * NV + v] = F.get(v);
        if (lane == 31 && tail_open) {
            if (tail_r || head_cs) part.val_last[c * NV + v] = x;
            else part.val_first[c * NV + v] = x;
        }
    }
    if (close_here) sem.store(first_row, F);
}

// 32 bytes from global memory in one load, not allocated in L1: each tile
// is read once, and L1 is left to the input-vector gathers.  A whole 32-byte
// sector per instruction: narrower no-allocate loads would fetch a sector
// again for every part of it.
__device__ __forceinline__ void ld32_stream(const void* p, uint32_t (&v)[8]) {
    asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "l"(p));
}

// The same load without `volatile`: the compiler may schedule it with the
// other loads of the lane (the data is read-only while a kernel runs).
__device__ __forceinline__ void ld32_stream_free(const void* p, uint32_t (&v)[8]) {
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "l"(p));
}

// 16 bytes, not allocated in L1.
__device__ __forceinline__ uint4 ld16_stream(const void* p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];\n"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

template <int K>
__device__ __forceinline__ void load_lane_tiles(const SpmvGeom& g, int32_t tl, uint4 (&tv)[ChunkShape<K>::TILE_V4],
                                                int32_t (&col)[ChunkShape<K>::P]) {
    using S = ChunkShape<K>;
    constexpr int P = S::P;
    // a lane's P tiles are P * TB = 32, 64, 128 or 256 bytes, 32-byte aligned (tl is a multiple of P)
    static_assert(S::TILE_V4 % 2 == 0, "whole 32-byte sectors of tiles per lane");
    const uint8_t* src = g.tiles + (int64_t)tl * S::TB;
    if constexpr (K == 4) {
        // k = 4 (32 bytes of tiles and of columns a lane): two 16-byte loads
        // each measured faster here than one 32-byte load (161 against 166 us
        // for the plus-times SpMV on R-MAT 20); from k = 8 the 32-byte load wins
#pragma unroll
        for (int q = 0; q < S::TILE_V4; ++q) tv[q] = ld16_stream(src + 16 * q);
        const uint4 c0 = ld16_stream(g.colind + tl), c1 = ld16_stream(g.colind + tl + 4);
        col[0] = (int32_t)c0.x; col[1] = (int32_t)c0.y; col[2] = (int32_t)c0.z; col[3] = (int32_t)c0.w;
        col[4] = (int32_t)c1.x; col[5] = (int32_t)c1.y; col[6] = (int32_t)c1.z; col[7] = (int32_t)c1.w;
        return;
    }
#pragma unroll
    for (int q = 0; q < S::TILE_V4 / 2; ++q) {
        uint32_t v[8];
        ld32_stream_free(src + 32 * q, v);
        tv[2 * q] = make_uint4(v[0], v[1], v[2], v[3]);
        tv[2 * q + 1] = make_uint4(v[4], v[5], v[6], v[7]);
    }
    if constexpr (P == 8) {  // 32 bytes of column indices: one sector
        uint32_t v[8];
        ld32_stream_free(g.colind + tl, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) col[i] = (int32_t)v[i];
    } else if constexpr (P % 4 == 0) {  // lanes share sectors: cached loads
        const int4* cs = reinterpret_cast<const int4*>(g.colind + tl);
#pragma unroll
        for (int q = 0; q < P / 4; ++q) {
            int4 v = __ldg(cs + q);
            col[4 * q] = v.x; col[4 * q + 1] = v.y; col[4 * q + 2] = v.z; col[4 * q + 3] = v.w;
        }
    } else {
        const int2* cs = reinterpret_cast<const int2*>(g.colind + tl);
#pragma unroll
        for (int q = 0; q < P / 2; ++q) {
            int2 v = __ldg(cs + q);
            col[2 * q] = v.x; col[2 * q + 1] = v.y;
        }
    }
}

// ---------------------------------------------------------------------------
// chunk kernel for the bit-vector schemes (all k) and for the value schemes
// at k = 32: registers hold the accumulators (static row indices)
// ---------------------------------------------------------------------------
template <int K, class SEM>
__global__ void __launch_bounds__(kSpmvThreads) spmv_chunks_kernel(SpmvGeom g, SEM sem,
                                                                   Partials<typename SEM::V> part) {
    using S = ChunkShape<K>;
    using V = typename SEM::V;
    constexpr int NV = SEM::NV;
    constexpr int P = S::P;
    const int warp = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    const int32_t c = (int32_t)blockIdx.x * kSpmvWarps + warp;
    if (c >= g.nchunks || gated_off(g.gate)) return;  // whole warps leave together

    LaneSpan ls;
    ls.cs = c * S::CT;
    ls.ce = min(ls.cs + S::CT, (int32_t)g.T);
    ls.tl = ls.cs + lane * P;
    ls.cnt = max(0, min(P, ls.ce - ls.tl));

    uint4 tv[S::TILE_V4];
    int32_t col[P];
    // a chunk whose every output row is masked out reads no tiles (zero words:
    // the walk still stores its rows and partials, all the identity)
    bool sat = false;
    {
        const int32_t ra = __ldg(g.chunk_row + c), rb = __ldg(g.chunk_row + c + 1);
        sat = sem.saturated((int64_t)ra * K, ((int64_t)rb + 1) * K);
    }
    if (!sat) {
        load_lane_tiles<K>(g, ls.tl, tv, col);
    } else {
#pragma unroll
        for (int q = 0; q < S::TILE_V4; ++q) tv[q] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int i = 0; i < P; ++i) col[i] = 0;
    }
    const uint32_t* words = reinterpret_cast<const uint32_t*>(tv);
    uint32_t xs[SEM::kGather ? 1 : P];
    if constexpr (!SEM::kGather) {
#pragma unroll
        for (int i = 0; i < P; ++i) xs[i] = sem.xseg(col[i]);
    }
    const RowCursor rc = locate_row(g, c, ls, lane);

    RegAcc<V, NV> acc, F, idv;
#pragma unroll
    for (int v = 0; v < NV; ++v) { acc.set(v, sem.ident()); F.set(v, sem.ident()); idv.set(v, sem.ident()); }
    Walk<SEM, RegAcc<V, NV>> wk;
    wk.row = rc.row;
    wk.next = rc.next;
    if (ls.cnt > 0) {
        // empty tile-rows just before a row that starts at this lane's first tile
        if (ls.tl > 0 && rc.row_start == ls.tl)
            for (int32_t R = rc.row - 1; R >= 0 && __ldg(g.rowptr + R) == ls.tl; --R) sem.store(R, idv);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (i < ls.cnt) {
                const int32_t t = ls.tl + i;
                if constexpr (!SEM::kGather) {
                    sem.tile(acc, words + i * S::TW, xs[i]);
                } else {
                    using G = typename SEM::G;
                    const G* xt = sem.src() + (int64_t)col[i] * K;
                    const float* wt = sem.weighted ? sem.wts() + __ldg(sem.voffs() + t) : nullptr;
                    int qb = 0;
#pragma unroll
                    for (int q = 0; q < S::TW; ++q) {
                        uint32_t b = words[i * S::TW + q];
                        while (b) {
                            const int bit = __ffs(b) - 1;
                            b &= b - 1;
                            const int r = q * (32 / S::ROW_BITS) + bit / S::ROW_BITS;
                            const float wv = sem.weighted ? __ldg(wt + qb) : 1.0f;
                            const G xv = __ldg(xt + bit % S::ROW_BITS);
                            if constexpr (sizeof(V) == 8 && NV <= 8) {
                                // 8-byte accumulators: a predicated update of
                                // each row keeps the indices constant (a
                                // runtime index puts the array in local memory)
#pragma unroll
                                for (int v = 0; v < NV; ++v)
                                    if (v == r) acc.set(v, sem.apply(acc.get(v), xv, wv));
                            } else {
                                acc.set(r, sem.apply(acc.get(r), xv, wv));
                            }
                            ++qb;
                        }
                    }
                }
                wk.end_tile(g, sem, acc, F, t, i, ls.cnt, idv);
            }
        }
    }
    close_chunk(sem, part, c, ls, lane, rc.head_cs, rc.row, wk.has_end, wk.open, acc, F, P);
}

// ---------------------------------------------------------------------------
// tile_dim-4 chunk kernel for the bit-vector schemes (Boolean and count
// SpMVs) and the unweighted 4-byte value schemes (plus-times, label min, fp32
// max: one gather per set bit).  At k = 4 a tile is 4 bytes, so the tile
// stream is tiny per tile and the kernel is shaped by per-tile latency:
//   * persistent warps: warp gw takes chunks gw, gw + W, ... and loads the
//     next chunk's tile stream (8 tile words and 8 tile columns a lane, one
//     32-byte load each, marked not to be kept in L1, plus the chunk's row
//     pointers) into registers before it works on the current one, so every
//     warp keeps a chunk in flight;
//   * a chunk inside one tile-row (most chunks of a power-law graph) needs no
//     row search, walk or segmented scan: one fixed-order butterfly joins the
//     lanes; other chunks take the chunk kernel's walk and joins.
// ---------------------------------------------------------------------------
// resident 256-thread blocks the registers are budgeted for (every lane holds
// two chunks' tile words and columns)
constexpr int kK4MinBlocks = 4;


// The tile stream of one chunk as a lane holds it: the chunk's first and last
// tile-rows and their row pointers (lane j: rowptr[ra + j]), whether every
// output row of it is masked out (then no tiles are read and the words are
// zero: the walk still stores its rows and partials, all the identity), and
// the lane's 8 tile words and columns.
struct K4Tiles {
    int32_t ra, rb;
    int32_t win;
    bool sat;
    uint32_t w[8], cu[8];
};

template <class SEM>
__device__ __forceinline__ void k4_load(const SpmvGeom& g, const SEM& sem, int32_t c, int lane, K4Tiles& t) {
    t.ra = __ldg(g.chunk_row + c);
    t.rb = __ldg(g.chunk_row + c + 1);
    t.win = row_window(g, t.ra, t.rb - t.ra, lane);
    t.sat = sem.saturated((int64_t)t.ra * 4, ((int64_t)t.rb + 1) * 4);
    if (!t.sat) {
        // the arrays are padded to whole chunks, so every lane's 32 bytes exist
        const int64_t tl = (int64_t)c * chunk_tiles(4) + lane * 8;
        ld32_stream(reinterpret_cast<const uint32_t*>(g.tiles) + tl, t.w);
        ld32_stream(g.colind + tl, t.cu);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) { t.w[i] = 0u; t.cu[i] = 0u; }
    }
}

// The set bits of one k = 4 tile (row r in byte r) gather their inputs and
// add them to the lane's row accumulators (value schemes).
template <class SEM, class Acc>
__device__ __forceinline__ void k4_gather_tile(const SEM& sem, Acc& acc, uint32_t w, int32_t J) {
    using G = typename SEM::G;
    using V = typename SEM::V;
    const G* xt = sem.src() + (int64_t)J * 4;
    while (w) {
        const int bit = __ffs(w) - 1;
        w &= w - 1;
        const int r = bit >> 3;
        const G xv = __ldg(xt + (bit & 7));
        if constexpr (sizeof(V) == 8) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (v == r) acc.set(v, sem.apply(acc.get(v), xv, 1.0f));
        } else {
            acc.set(r, sem.apply(acc.get(r), xv, 1.0f));
        }
    }
}

// One chunk from its loaded tile stream.
template <class SEM>
__device__ __forceinline__ void k4_chunk(const SpmvGeom& g, const SEM& sem, Partials<typename SEM::V> part, int32_t c,
                                         int lane, const K4Tiles& t) {
    using S = ChunkShape<4>;
    using V = typename SEM::V;
    constexpr int NV = SEM::NV;
    constexpr int P = S::P;
    static_assert(P == 8 && S::TW == 1, "eight one-word tiles a lane");
    LaneSpan ls;
    ls.cs = c * S::CT;
    ls.ce = min(ls.cs + S::CT, (int32_t)g.T);
    ls.tl = ls.cs + lane * P;
    ls.cnt = max(0, min(P, ls.ce - ls.tl));
    const int32_t ra = t.ra, rb = t.rb;
    // the 4-bit input segment under each tile (bit-vector schemes)
    uint32_t xs[SEM::kGather ? 1 : P];
    if constexpr (!SEM::kGather) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const bool ok = i < ls.cnt && t.w[i] != 0u;
            xs[i] = ok ? sem.xseg((int32_t)t.cu[i]) : 0u;
        }
    }
    RegAcc<V, NV> acc, F, idv;
#pragma unroll
    for (int v = 0; v < NV; ++v) { acc.set(v, sem.ident()); F.set(v, sem.ident()); idv.set(v, sem.ident()); }

    if (ra == rb) {
        // The whole chunk lies in tile-row ra (warp-uniform): every lane's
        // tiles add to the same k rows, so no row search, walk or segmented
        // scan is needed -- one fixed-order butterfly joins the lanes.
        const int32_t row_start = __shfl_sync(0xffffffffu, t.win, 0);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (i < ls.cnt) {
                if constexpr (SEM::kGather) k4_gather_tile(sem, acc, t.w[i], (int32_t)t.cu[i]);
                else sem.tile(acc, t.w + i, xs[i]);
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const V other = shfl_xor(acc.get(v), o);
                acc.set(v, (lane & o) ? sem.comb(other, acc.get(v)) : sem.comb(acc.get(v), other));
            }
        }
        if (lane == 0) {
            const bool head = row_start == ls.cs;  // the row begins with this chunk
            if (head && ls.cs > 0)                 // empty tile-rows just before it
                for (int32_t R = ra - 1; R >= 0 && __ldg(g.rowptr + R) == ls.cs; --R) sem.store(R, idv);
            if (head && c + 1 == g.nchunks) {
                sem.store(ra, acc);  // begins and ends in this chunk (the matrix's last)
            } else {
                // continued by later chunks (head) or begun in earlier ones
                V* dst = (head ? part.val_last : part.val_first) + (int64_t)c * NV;
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[v] = acc.get(v);
            }
        }
        return;
    }
    const RowCursor rc = locate_row_win(g, ra, rb - ra, t.win, ls, lane);
    Walk<SEM, RegAcc<V, NV>> wk;
    wk.row = rc.row;
    wk.next = rc.next;
    if (ls.cnt > 0) {
        // empty tile-rows just before a row that starts at this lane's first tile
        if (ls.tl > 0 && rc.row_start == ls.tl)
            for (int32_t R = rc.row - 1; R >= 0 && __ldg(g.rowptr + R) == ls.tl; --R) sem.store(R, idv);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (i < ls.cnt) {
                if constexpr (SEM::kGather) k4_gather_tile(sem, acc, t.w[i], (int32_t)t.cu[i]);
                else sem.tile(acc, t.w + i, xs[i]);
                wk.end_tile(g, sem, acc, F, ls.tl + i, i, ls.cnt, idv);
            }
        }
    }
    close_chunk(sem, part, c, ls, lane, rc.head_cs, rc.row, wk.has_end, wk.open, acc, F, P);
}

template <class SEM>
__global__ void __launch_bounds__(kSpmvThreads, kK4MinBlocks)
    spmv_k4_kernel(SpmvGeom g, SEM sem, Partials<typename SEM::V> part) {
    const int lane = (int)lane_id();
    const int32_t W = (int32_t)gridDim.x * kSpmvWarps;
    int32_t c = (int32_t)blockIdx.x * kSpmvWarps + (threadIdx.x >> 5);
    if (c >= g.nchunks || gated_off(g.gate)) return;  // whole warps leave together
    K4Tiles cur, nxt;
    k4_load(g, sem, c, lane, cur);
    for (;;) {
        const int32_t cn = c + W;
        const bool more = cn < g.nchunks;
        if (more) k4_load(g, sem, cn, lane, nxt);
        k4_chunk(g, sem, part, c, lane, cur);
        if (!more) break;
        c = cn;
        cur = nxt;
    }
}

// ---------------------------------------------------------------------------
// chunk kernel for the value schemes at k <= 16.  Pass 1: each lane walks
// the set bits of its tiles in one flat loop (tile words copied to lane-private
// shared memory so a running word index can address them) and issues one
// cp.async gather per bit, so a warp's input values are all in flight at once;
// each staged value is tagged with its (tile, row).  Pass 2: a second flat
// loop over the tags adds each value to its row's register accumulator (a
// predicated select over the k rows keeps every register index static) and
// closes tiles as the walk passes them.  Lanes with fewer set bits finish
// early instead of idling through per-word loops.
// ---------------------------------------------------------------------------
// Resident blocks the gather kernel is compiled for: wide (16-byte) values
// need the registers of two blocks per SM rather than three.
template <int K, class SEM>
constexpr int gather_min_blocks() {
    return (K >= 16 || sizeof(typename SEM::V) > 8) ? 2 : 3;
}

template <int K, class SEM>
__global__ void __launch_bounds__(kSpmvThreads, (gather_min_blocks<K, SEM>())) spmv_gather_kernel(SpmvGeom g, SEM sem,
                                                                   Partials<typename SEM::V> part) {
    using S = ChunkShape<K>;
    using V = typename SEM::V;
    using G = typename SEM::G;
    using L = GatherLayout<K, SEM>;
    constexpr int NV = SEM::NV;
    constexpr int P = S::P;
    constexpr int TW = S::TW;
    constexpr int RB = S::ROW_BITS;
    constexpr int RPW = 32 / RB;  // rows per 32-bit word
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    const int32_t c = (int32_t)blockIdx.x * kSpmvWarps + warp;
    if (c >= g.nchunks || gated_off(g.gate)) return;  // whole warps leave together

    uint8_t* wsm = smem + warp * L::bytes;
    // lane-interleaved (element e of lane l at [e * 32 + l]): conflict-free
    uint32_t* swords = reinterpret_cast<uint32_t*>(wsm + L::words_off) + lane;
    int32_t* scol = reinterpret_cast<int32_t*>(wsm + L::col_off) + lane;
    G* sx = reinterpret_cast<G*>(wsm + L::x_off);
    float* sw = reinterpret_cast<float*>(wsm + L::w_off);
    uint8_t* stag = wsm + L::tag_off;

    LaneSpan ls;
    ls.cs = c * S::CT;
    ls.ce = min(ls.cs + S::CT, (int32_t)g.T);
    ls.tl = ls.cs + lane * P;
    ls.cnt = max(0, min(P, ls.ce - ls.tl));

    uint4 tv[S::TILE_V4];
    int32_t col[P];
    // a chunk whose every output row is masked out reads no tiles (zero words:
    // the walk still stores its rows and partials, all the identity)
    bool sat = false;
    {
        const int32_t ra = __ldg(g.chunk_row + c), rb = __ldg(g.chunk_row + c + 1);
        sat = sem.saturated((int64_t)ra * K, ((int64_t)rb + 1) * K);
    }
    if (!sat) {
        load_lane_tiles<K>(g, ls.tl, tv, col);
    } else {
#pragma unroll
        for (int q = 0; q < S::TILE_V4; ++q) tv[q] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int i = 0; i < P; ++i) col[i] = 0;
    }
    const uint32_t* words = reinterpret_cast<const uint32_t*>(tv);

    // set bits of the lane's tiles and their slots in the warp's staging area
    int nb = 0;
#pragma unroll
    for (int i = 0; i < P; ++i)
        if (i < ls.cnt) {
#pragma unroll
            for (int q = 0; q < TW; ++q) nb += __popc(words[i * TW + q]);
        }
    int incl = nb;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
    }
    const int gbase = incl - nb;
    const int nbits = __shfl_sync(FULL, incl, 31);
    const bool staged = nbits <= L::NG;  // warp-uniform

    if (staged) {
        // first staging slot of each of the lane's tiles
        int32_t* spre = reinterpret_cast<int32_t*>(wsm + L::pre_off) + lane;
        int run = gbase;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            spre[i * 32] = run;
            if (i < ls.cnt) {
#pragma unroll
                for (int q = 0; q < TW; ++q) run += __popc(words[i * TW + q]);
            }
        }
#pragma unroll
        for (int q = 0; q < P * TW; ++q) swords[q * 32] = words[q];
#pragma unroll
        for (int i = 0; i < P; ++i) scol[i * 32] = col[i];
        int wi = 0;
        uint32_t cur = words[0];
        int ti = -1, qb = 0;
        const G* xt = nullptr;
        const float* wt = nullptr;
        for (int j = 0; j < nb; ++j) {
            while (cur == 0u) cur = swords[(++wi) * 32];
            const int bit = __ffs(cur) - 1;
            cur &= cur - 1;
            const int i = wi / TW;
            if (i != ti) {  // first set bit of tile i
                ti = i;
                qb = 0;
                xt = sem.src() + (int64_t)scol[i * 32] * K;
                if (sem.weighted) wt = sem.wts() + __ldg(sem.voffs() + ls.tl + i);
            }
            const int s = gbase + j;
            cp_async_gather<sizeof(G)>(sx + s, xt + bit % RB);
            if (sem.weighted) cp_async_gather<4>(sw + s, wt + qb);
            stag[s] = (uint8_t)(wi * RPW + bit / RB);  // = i * K + (wi % TW) * RPW + row in word
            ++qb;
        }
        cp_async_commit();
    }

    RegAcc<V, NV> idv;
#pragma unroll
    for (int v = 0; v < NV; ++v) idv.set(v, sem.ident());

    // ---- fast path: a staged chunk spanning at most four tile-rows.  Each
    // tile-row's staged values (contiguous slots, tile order) are dealt to
    // the lanes round-robin, summed in registers, and joined by a fixed
    // butterfly, so no lane waits on another's bit count.
    {
        const int32_t r0 = __ldg(g.chunk_row + c);
        const int32_t span = __ldg(g.chunk_row + c + 1) - r0;
        if (staged && span <= 3) {
            const int32_t win = lane <= span + 1 ? __ldg(g.rowptr + r0 + lane) : INT32_MAX;
            cp_async_wait_all();
            __syncwarp();  // values, tags and slot starts of every lane are visible
            const int32_t* pre = reinterpret_cast<const int32_t*>(wsm + L::pre_off);
            auto slot_of = [&](int32_t t) -> int {  // first slot of chunk tile t (nbits at the chunk end)
                if (t >= ls.ce) return nbits;
                const int32_t o = t - ls.cs;
                return pre[(o % P) * 32 + (o / P)];
            };
            const int32_t a0 = __shfl_sync(FULL, win, 0);
            if (lane == 0 && a0 == ls.cs && ls.cs > 0)  // empty rows just before the chunk's first tile-row
                for (int32_t R = r0 - 1; R >= 0 && __ldg(g.rowptr + R) == ls.cs; --R) sem.store(R, idv);
            for (int j = 0; j <= span; ++j) {
                const int32_t R = r0 + j;
                const int32_t a = __shfl_sync(FULL, win, j), b = __shfl_sync(FULL, win, j + 1);
                if (a == b) {  // empty tile-row inside the chunk's range
                    if (lane == 0 && a >= ls.cs && a < ls.ce && a > 0) sem.store(R, idv);
                    continue;
                }
                const int32_t ts = max(a, ls.cs), te = min(b, ls.ce);
                if (ts >= te) continue;  // its tiles lie outside this chunk
                const int s0 = slot_of(ts), s1 = slot_of(te);
                RegAcc<V, NV> acc;
#pragma unroll
                for (int v = 0; v < NV; ++v) acc.set(v, sem.ident());
                for (int sidx = s0 + lane; sidx < s1; sidx += 32) {
                    const int r = stag[sidx] % K;
                    const V cv = sem.contrib(sx[sidx], sem.weighted ? sw[sidx] : 1.0f);
#pragma unroll
                    for (int u = 0; u < K; ++u) acc.set(u, sem.comb(acc.get(u), r == u ? cv : sem.ident()));
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const V other = shfl_xor(acc.get(v), o);
                        acc.set(v, (lane & o) ? sem.comb(other, acc.get(v)) : sem.comb(acc.get(v), other));
                    }
                }
                if (lane < K) {  // every lane holds the totals: lane r writes row r
                    V v = acc.get(0);
#pragma unroll
                    for (int u = 1; u < K; ++u) v = lane == u ? acc.get(u) : v;
                    const bool started = a >= ls.cs, ended = b <= ls.ce;
                    if (started && ended) sem.store_row(R, lane, v);
                    else if (!started) part.val_first[c * NV + lane] = v;
                    else part.val_last[c * NV + lane] = v;
                }
            }
            return;
        }
    }

    const RowCursor rc = locate_row(g, c, ls, lane);
    RegAcc<V, NV> acc, F;
#pragma unroll
    for (int v = 0; v < NV; ++v) { acc.set(v, sem.ident()); F.set(v, sem.ident()); }
    Walk<SEM, RegAcc<V, NV>> wk;
    wk.row = rc.row;
    wk.next = rc.next;
    if (staged) cp_async_wait_all();  // each lane reads back only the slots it filled

    if (ls.cnt > 0) {
        // empty tile-rows just before a row that starts at this lane's first tile
        if (ls.tl > 0 && rc.row_start == ls.tl)
            for (int32_t R = rc.row - 1; R >= 0 && __ldg(g.rowptr + R) == ls.tl; --R) sem.store(R, idv);
        if (staged) {
            int i = 0;
            for (int j = 0; j < nb; ++j) {
                const int s = gbase + j;
                const int tag = stag[s];
                const int ti = tag / K;
                while (i < ti) {  // every tile has a set bit: the walk passes tile i
                    wk.end_tile(g, sem, acc, F, ls.tl + i, i, ls.cnt, idv);
                    ++i;
                }
                const int r = tag % K;
                const V cv = sem.contrib(sx[s], sem.weighted ? sw[s] : 1.0f);
                // branch-free row select: every row combines either the
                // contribution or the identity
#pragma unroll
                for (int u = 0; u < K; ++u) acc.set(u, sem.comb(acc.get(u), r == u ? cv : sem.ident()));
            }
            for (; i < ls.cnt; ++i) wk.end_tile(g, sem, acc, F, ls.tl + i, i, ls.cnt, idv);
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                if (i < ls.cnt) {
                    const int32_t t = ls.tl + i;
                    const G* xt = sem.src() + (int64_t)col[i] * K;
                    const float* wt = sem.weighted ? sem.wts() + __ldg(sem.voffs() + t) : nullptr;
                    int qb = 0;
#pragma unroll
                    for (int q = 0; q < TW; ++q) {
                        uint32_t b = words[i * TW + q];
                        while (b) {
                            const int bit = __ffs(b) - 1;
                            b &= b - 1;
                            const V cv = sem.contrib(__ldg(xt + bit % RB), sem.weighted ? __ldg(wt + qb) : 1.0f);
                            const int u = bit / RB;
#pragma unroll
                            for (int uu = 0; uu < RPW; ++uu)
                                acc.set(q * RPW + uu, sem.comb(acc.get(q * RPW + uu), u == uu ? cv : sem.ident()));
                            ++qb;
                        }
                    }
                    wk.end_tile(g, sem, acc, F, t, i, ls.cnt, idv);
                }
            }
        }
    }
    close_chunk(sem, part, c, ls, lane, rc.head_cs, rc.row, wk.has_end, wk.open, acc, F, P);
}

// Rows that span chunks, from the handle's split list of (row, first chunk,
// last chunk): the row's partials are the first chunk's val_last and every
// later chunk's val_first, joined in chunk order.  Blocks [0, short_blocks)
// give one thread to each row spanning at most kSplitShort chunks; the
// remaining blocks give a warp to each longer row (lane l folds every 32nd
// partial in order, then a fixed butterfly joins the lanes).
template <int K, class SEM>
__global__ void spmv_fixup_kernel(const int32_t* __restrict__ split, int64_t nshort, int64_t nlong,
                                  int64_t short_blocks, SEM sem, Partials<typename SEM::V> part,
                                  const int32_t* gate) {
    using V = typename SEM::V;
    using J = typename SEM::J;
    constexpr int NV = SEM::NV;
    if (gated_off(gate)) return;
    if ((int64_t)blockIdx.x < short_blocks) {
        if constexpr (SEM::kGather) {
            // value schemes: a thread per (row, value); the NV threads of a
            // row read each partial's NV values side by side
            const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
            const int64_t e = tid / NV;
            const int v = (int)(tid % NV);
            if (e >= nshort) return;
            const int32_t R = split[3 * e], ca = split[3 * e + 1], cb = split[3 * e + 2];
            J acc = (J)part.val_last[(int64_t)ca * NV + v];
            for (int64_t q = ca + 1; q <= cb; ++q) acc = sem.jcomb(acc, (J)part.val_first[q * NV + v]);
            sem.store_row(R, v, (V)acc);
            return;
        }
        const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (e >= nshort) return;
        const int32_t R = split[3 * e], ca = split[3 * e + 1], cb = split[3 * e + 2];
        J acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = (J)part.val_last[(int64_t)ca * NV + v];
        for (int64_t q = ca + 1; q <= cb; ++q) {
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = sem.jcomb(acc[v], (J)part.val_first[q * NV + v]);
        }
        RegAcc<V, NV> out;
#pragma unroll
        for (int v = 0; v < NV; ++v) out.set(v, (V)acc[v]);
        sem.store(R, out);
        return;
    }
    const int lane = (int)lane_id();
    const int64_t e = nshort + ((int64_t)(blockIdx.x - short_blocks) * blockDim.x + threadIdx.x) / 32;
    if (e >= nshort + nlong) return;  // whole warps leave together
    const int32_t R = split[3 * e], ca = split[3 * e + 1], cb = split[3 * e + 2];
    const int64_t np = (int64_t)cb - ca + 1;
    J acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = (J)sem.ident();
    for (int64_t p = lane; p < np; p += 32) {
        const V* src = p == 0 ? part.val_last + (int64_t)ca * NV : part.val_first + (ca + p) * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = sem.jcomb(acc[v], (J)src[v]);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const J other = shfl_xor(acc[v], o);
            acc[v] = (lane & o) ? sem.jcomb(other, acc[v]) : sem.jcomb(acc[v], other);
        }
    }
    if (lane == 0) {
        RegAcc<V, NV> out;
#pragma unroll
        for (int v = 0; v < NV; ++v) out.set(v, (V)acc[v]);
        sem.store(R, out);
    }
}

template <int K, class SEM>
static b2sr_status launch_fixup(const b2sr_matrix* h, const SEM& sem, Partials<typename SEM::V> part,
                                cudaStream_t s, const int32_t* gate) {
    if (h->nsplit_short + h->nsplit_long == 0) return B2SR_OK;
    const int64_t short_blocks = ceil_div(h->nsplit_short * (SEM::kGather ? SEM::NV : 1), 256);
    const int64_t long_blocks = ceil_div(h->nsplit_long, 8);
    spmv_fixup_kernel<K, SEM><<<(unsigned)(short_blocks + long_blocks), 256, 0, s>>>(
        h->split, h->nsplit_short, h->nsplit_long, short_blocks, sem, part, gate);
    B2SR_LAUNCH_CHECK("spmv_fixup_kernel");
    return B2SR_OK;
}

// Tile-rows before the first tile and after the last one (every row when the
// matrix has no tiles) get the identity.
template <int K, class SEM>
__global__ void spmv_edges_kernel(SEM sem, int32_t lead_end, int32_t trail_begin, int32_t ntr,
                                  const int32_t* gate) {
    using V = typename SEM::V;
    if (gated_off(gate)) return;
    RegAcc<V, SEM::NV> idv;
#pragma unroll
    for (int v = 0; v < SEM::NV; ++v) idv.set(v, sem.ident());
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t R = tid; R < lead_end; R += stride) sem.store((int32_t)R, idv);
    for (int64_t R = trail_begin + tid; R < ntr; R += stride) sem.store((int32_t)R, idv);
}

// semirings whose result includes the diagonal's self term (min-plus)
template <class S, class = void>
struct HasSelfTerm : std::false_type {};
template <class S>
struct HasSelfTerm<S, std::void_t<decltype(S::kSelfTerm)>> : std::bool_constant<S::kSelfTerm> {};

template <class T>
__device__ __forceinline__ T min_self(T a, T b) {
    if constexpr (std::is_same<T, float>::value) return fminf(a, b);
    else return min(a, b);
}

// y_i = min(x_i, y_i) on the rows the mask keeps (the min-plus self term)
template <class SEM>
__global__ void spmv_self_kernel(SEM sem, const int32_t* gate) {
    if (gated_off(gate)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sem.n; i += (int64_t)gridDim.x * blockDim.x)
        if (mask_allows(sem.mask, sem.comp, i)) sem.y[i] = min_self(sem.y[i], __ldg(sem.x + i));
}

__global__ void clear_words_kernel(uint32_t* w, int64_t count, const int32_t* gate) {
    if (gated_off(gate)) return;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) w[i] = 0u;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Bitset outputs: bits past the last tile-row (>= nTileRow*k) are never
// stored by a row, so the words holding them are cleared first.
template <int K>
static b2sr_status clear_bitset_tail(const b2sr_matrix* h, uint32_t* bits, cudaStream_t s, const int32_t* gate) {
    int64_t words = ceil_div(h->n, 32);
    int64_t first = ((int64_t)h->ntr * K) / 32;
    if (first >= words) return B2SR_OK;
    if (!gate) {
        B2SR_CUDA_TRY(cudaMemsetAsync(bits + first, 0, (words - first) * sizeof(uint32_t), s));
        return B2SR_OK;
    }
    // gated: a closed gate must leave the output alone (the caller may have filled it another way)
    clear_words_kernel<<<1, 32, 0, s>>>(bits + first, words - first, gate);
    B2SR_LAUNCH_CHECK("clear_words_kernel");
    return B2SR_OK;
}

template <int K, class SEM>
static b2sr_status launch_edges(const b2sr_matrix* h, const SEM& sem, cudaStream_t s, const int32_t* gate) {
    int32_t lead_end = h->T == 0 ? h->ntr : h->first_row;
    int32_t trail_begin = h->T == 0 ? h->ntr : h->last_row + 1;
    int64_t work = (int64_t)lead_end + (h->ntr - trail_begin);
    if (work <= 0) return B2SR_OK;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)sm_count() * 4));
    spmv_edges_kernel<K, SEM><<<grid, 256, 0, s>>>(sem, lead_end, trail_begin, h->ntr, gate);
    B2SR_LAUNCH_CHECK("spmv_edges_kernel");
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

// Algorithmic bytes of one SpMV: the three B2SR arrays once, plus the
// vectors each scheme reads and writes once.
static double spmv_bytes(const b2sr_matrix* h, double vec_bytes) {
    return 4.0 * ((double)h->ntr + 1.0) + (double)h->T * (4.0 + tile_bytes(h->k)) + vec_bytes;
}

// The tile_dim-4 kernel serves, at k = 4, the bit-vector schemes and the
// unweighted value schemes with 4-byte values (plus-times, the label min, fp32
// max); 8-byte values would not fit its registers without spilling.
template <int K, class SEM>
constexpr bool use_k4() {
    if constexpr (!SEM::kGather) return K == 4;
    else return K == 4 && !SEM::kMayWeight && sizeof(typename SEM::V) == 4;
}

// The direct chunk kernel: the tile_dim-4 one where it serves, else the
// general one.
template <int K, class SEM>
static b2sr_status launch_direct(const b2sr_matrix* h, const SEM& sem, Partials<typename SEM::V> part,
                                 cudaStream_t s, const SpmvGeom& g) {
    const unsigned blocks = (unsigned)ceil_div(h->nchunks, kSpmvWarps);
    if constexpr (use_k4<K, SEM>()) {
        // persistent: the resident blocks, each warp looping over chunks
        const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)sm_count() * kK4MinBlocks);
        spmv_k4_kernel<SEM><<<grid, kSpmvThreads, 0, s>>>(g, sem, part);
        B2SR_LAUNCH_CHECK("spmv_k4_kernel");
    } else {
        spmv_chunks_kernel<K, SEM><<<blocks, kSpmvThreads, 0, s>>>(g, sem, part);
        B2SR_LAUNCH_CHECK("spmv_chunks_kernel");
    }
    return B2SR_OK;
}

// the chunk kernel (staged or direct) and the cross-chunk join
template <int K, class SEM>
static b2sr_status run_chunks(const b2sr_matrix* h, const SEM& sem, cudaStream_t s, const char* family,
                              double vec_bytes, const int32_t* gate, const SpmvGeom& g) {
    using V = typename SEM::V;
    DevBuf pbuf(s);
    Partials<V> part;
    B2SR_TRY((alloc_partials<V, SEM::NV>(pbuf, h->nchunks, &part)));
    const unsigned blocks = (unsigned)ceil_div(h->nchunks, kSpmvWarps);
    bool staged = false;
    if constexpr (SEM::kGather && K <= 16) staged = h->schedule != B2SR_SCHED_DIRECT;
    if constexpr (SEM::kGather && K <= 16) if (staged) {
        const int smem = kSpmvWarps * GatherLayout<K, SEM>::bytes;
        if (smem > 48 * 1024)
            B2SR_CUDA_TRY(cudaFuncSetAttribute(spmv_gather_kernel<K, SEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        void* tok = timing_begin(s);
        spmv_gather_kernel<K, SEM><<<blocks, kSpmvThreads, smem, s>>>(g, sem, part);
        timing_end(tok, family, spmv_bytes(h, vec_bytes), s);
        B2SR_LAUNCH_CHECK("spmv_gather_kernel");
    }
    if (!staged) {
        void* tok = timing_begin(s);
        const b2sr_status st = launch_direct<K, SEM>(h, sem, part, s, g);
        timing_end(tok, family, spmv_bytes(h, vec_bytes), s);
        B2SR_TRY(st);
    }
    return launch_fixup<K, SEM>(h, sem, part, s, gate);
}

template <int K, class SEM>
static b2sr_status run_spmv(const b2sr_matrix* h, const SEM& sem, uint32_t* bits_out, cudaStream_t s,
                            const char* family, double vec_bytes, const int32_t* gate) {
    SpmvGeom g{h->rowptr, h->colind, h->tiles, h->chunk_row, h->T, h->nchunks, h->ntr, gate};
    if (bits_out) B2SR_TRY(clear_bitset_tail<K>(h, bits_out, s, gate));
    B2SR_TRY((launch_edges<K, SEM>(h, sem, s, gate)));
    if (h->nchunks > 0) B2SR_TRY((run_chunks<K, SEM>(h, sem, s, family, vec_bytes, gate, g)));
    if constexpr (HasSelfTerm<SEM>::value) {
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->n, 256), (int64_t)sm_count() * 8));
        spmv_self_kernel<SEM><<<grid, 256, 0, s>>>(sem, gate);
        B2SR_LAUNCH_CHECK("spmv_self_kernel");
    }
    return B2SR_OK;
}


b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s,
                          const int32_t* gate) {
    comp = comp ? 1 : 0;
    if (sr == B2SR_BOOL_OR_AND && in_kind == B2SR_VEC_BITS && out_kind == B2SR_VEC_BITS) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemBool<K> sem{static_cast<const uint32_t*>(x), static_cast<uint32_t*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, static_cast<uint32_t*>(y), s, "spmv_bool", (mask ? 3.0 : 2.0) * h->n / 8.0, gate);
        });
    }
    if (sr == B2SR_PLUS_TIMES && in_kind == B2SR_VEC_BITS && out_kind == B2SR_VEC_I32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemCount<K> sem{static_cast<const uint32_t*>(x), static_cast<int32_t*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, nullptr, s, "spmv_count", (mask ? 2.0 : 1.0) * h->n / 8.0 + 4.0 * h->n, gate);
        });
    }
    if (sr == B2SR_PLUS_TIMES && in_kind == B2SR_VEC_F32 && out_kind == B2SR_VEC_F32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemPlus<K> sem{static_cast<const float*>(x), static_cast<float*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, nullptr, s, "spmv_plus", 8.0 * h->n + (mask ? h->n / 8.0 : 0.0), gate);
        });
    }
    if (sr == B2SR_MIN_PLUS && in_kind == B2SR_VEC_F32 && out_kind == B2SR_VEC_F32) {
        if (weights) B2SR_TRY(ensure_voff(h, s));
        return with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemMinPlus<K> sem{static_cast<const float*>(x), static_cast<float*>(y), mask, comp, h->n, weights,
                              h->voff, weights != nullptr};
            return run_spmv<K>(h, sem, nullptr, s, "spmv_minplus",
                               8.0 * h->n + (mask ? h->n / 8.0 : 0.0) +
                                   (weights ? 4.0 * (double)h->nnz + 4.0 * (double)h->T : 0.0), gate);
        });
    }
    if (sr == B2SR_MIN_PLUS && in_kind == B2SR_VEC_I32 && out_kind == B2SR_VEC_I32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "int32 MIN_PLUS takes no weights (all weights are 0)");
        return with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemMinI32<K> sem{static_cast<const int32_t*>(x), static_cast<int32_t*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, nullptr, s, "spmv_min_i32", 8.0 * h->n + (mask ? h->n / 8.0 : 0.0), gate);
        });
    }
    if (sr == B2SR_MAX_TIMES && in_kind == B2SR_VEC_F32 && out_kind == B2SR_VEC_F32) {
        if (weights) return fail(B2SR_ERR_INVALID_ARG, "weights apply to MIN_PLUS only");
        return with_tile(h->k, [&](auto kc) -> b2sr_status {
            constexpr int K = decltype(kc)::value;
            SemMaxF32<K> sem{static_cast<const float*>(x), static_cast<float*>(y), mask, comp, h->n};
            return run_spmv<K>(h, sem, nullptr, s, "spmv_max", 8.0 * h->n + (mask ? h->n / 8.0 : 0.0), gate);
        });
    }
    return fail(B2SR_ERR_INVALID_ARG, "unsupported semiring / vector kind combination");
}

b2sr_status spmm64_dispatch(b2sr_matrix* h, const uint64_t* X, uint64_t* Y, const uint64_t* M, int comp,
                            cudaStream_t s, const int32_t* gate) {
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        SemOr64<K> sem{reinterpret_cast<const unsigned long long*>(X), reinterpret_cast<unsigned long long*>(Y),
                       reinterpret_cast<const unsigned long long*>(M), comp ? 1 : 0, h->n};
        return run_spmv<K>(h, sem, nullptr, s, "spmm_or64", (M ? 24.0 : 16.0) * h->n, gate);
    });
}

// The same over 32-lane words (at most 32 frontiers): half the bytes per
// gather and 4-byte accumulators, which the tile_dim-4 kernel takes.
b2sr_status spmm32_dispatch(b2sr_matrix* h, const uint32_t* X, uint32_t* Y, const uint32_t* M, int comp,
                            cudaStream_t s, const int32_t* gate) {
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        SemOr32<K> sem{X, Y, M, comp ? 1 : 0, h->n};
        return run_spmv<K>(h, sem, nullptr, s, "spmm_or32", (M ? 12.0 : 8.0) * h->n, gate);
    });
}

b2sr_status spmv_maxkey_dispatch(b2sr_matrix* h, const uint64_t* x, uint64_t* y, const uint32_t* mask, int comp,
                                 cudaStream_t s, const int32_t* gate) {
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        SemMaxKey<K> sem{reinterpret_cast<const unsigned long long*>(x), reinterpret_cast<unsigned long long*>(y), mask,
                         comp ? 1 : 0, h->n};
        return run_spmv<K>(h, sem, nullptr, s, "spmv_maxkey", 16.0 * h->n + (mask ? h->n / 8.0 : 0.0), gate);
    });
}

b2sr_status spmm4_dispatch(b2sr_matrix* h, const float* X, float* Y, const uint32_t* M, int comp, cudaStream_t s,
                           const int32_t* gate) {
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        SemPlus4<K> sem{reinterpret_cast<const float4*>(X), reinterpret_cast<float4*>(Y), M, comp ? 1 : 0, h->n};
        return run_spmv<K>(h, sem, nullptr, s, "spmm_plus4", 32.0 * h->n + (M ? h->n / 8.0 : 0.0), gate);
    });
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_spmm_f32x4(b2sr_handle h, const float* X, float* Y, const uint32_t* mask,
                                       int mask_complement, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!X || !Y)) return fail(B2SR_ERR_INVALID_ARG, "X or Y is NULL");
    if (X == Y) return fail(B2SR_ERR_INVALID_ARG, "Y must not alias X");
    if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u)
        return fail(B2SR_ERR_INVALID_ARG, "X and Y must be 16-byte aligned");
    return spmm4_dispatch(h, X, Y, mask, mask_complement, to_stream(stream), nullptr);
}

extern "C" b2sr_status b2sr_spmv(b2sr_handle h, b2sr_semiring semiring, b2sr_vec in_kind, const void* x,
                                 b2sr_vec out_kind, void* y, const uint32_t* mask, int mask_complement,
                                 const float* weights, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!x || !y)) return fail(B2SR_ERR_INVALID_ARG, "x or y is NULL");
    if (x == y) return fail(B2SR_ERR_INVALID_ARG, "y must not alias x");
    return spmv_dispatch(h, semiring, in_kind, x, out_kind, y, mask, mask_complement, weights, to_stream(stream),
                         nullptr);
}

extern "C" b2sr_status b2sr_spmm_bits64(b2sr_handle h, const uint64_t* X, uint64_t* Y, const uint64_t* M,
                                        int complement, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!X || !Y)) return fail(B2SR_ERR_INVALID_ARG, "X or Y is NULL");
    if (X == Y) return fail(B2SR_ERR_INVALID_ARG, "Y must not alias X");
    return spmm64_dispatch(h, X, Y, M, complement, to_stream(stream), nullptr);
}

// ---------------------------------------------------------------------------
// Boolean SpMV without device allocation.
//
// Some callers cannot allocate device memory when they call into the library:
// a host whose own allocator has already reserved the device's free memory,
// or a deployment that must not allocate once it is running (fixed-memory or
// real-time services).  For them b2sr_spmv_bool_noalloc keeps the only scratch
// the Boolean SpMV needs -- the per-chunk partial rows joined by the fixup
// kernel -- in a fixed array compiled into this file.  A device holds its copy
// from the moment the runtime loads this file's device code on it (the first
// SpMV launch or symbol lookup there, under lazy module loading) until the
// process exits or the device is reset.
// ---------------------------------------------------------------------------
namespace b2sr {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device (host code
// cannot use the symbol itself as a device pointer).
static void* noalloc_scratch_ptr(int dev, b2sr_status* st) {
    static std::mutex mu;
    static void* ptrs[64] = {nullptr};
    if (dev < 0 || dev >= 64) {
        *st = fail(B2SR_ERR_INVALID_ARG, "device index out of range for the fixed scratch");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaGetSymbolAddress(fixed scratch)");
            return nullptr;
        }
        ptrs[dev] = p;
    }
    *st = B2SR_OK;
    return ptrs[dev];
}

template <int K>
static b2sr_status run_spmv_bool_fixed(const b2sr_matrix* h, const SemBool<K>& sem, uint32_t* y, void* scratch,
                                       cudaStream_t s) {
    using SEM = SemBool<K>;
    constexpr int NV = SEM::NV;
    const size_t half = round_up((size_t)h->nchunks * NV * sizeof(uint32_t), 256);
    if (2 * half > kNoallocScratchBytes)
        return fail(B2SR_ERR_INVALID_ARG, "matrix too large for b2sr_spmv_bool_noalloc: " +
                                              std::to_string(h->nchunks) + " chunks need " +
                                              std::to_string(2 * half) + " scratch bytes, the fixed array holds " +
                                              std::to_string(kNoallocScratchBytes));
    SpmvGeom g{h->rowptr, h->colind, h->tiles, h->chunk_row, h->T, h->nchunks, h->ntr, nullptr};
    B2SR_TRY(clear_bitset_tail<K>(h, y, s, nullptr));
    B2SR_TRY((launch_edges<K, SEM>(h, sem, s, nullptr)));
    if (h->nchunks == 0) return B2SR_OK;
    // every partial the fixup reads is written by the chunk kernel of the
    // same call, so the scratch needs no clearing between calls
    Partials<uint32_t> part;
    part.val_first = static_cast<uint32_t*>(scratch);
    part.val_last = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(scratch) + half);
    B2SR_TRY((launch_direct<K, SEM>(h, sem, part, s, g)));
    return launch_fixup<K, SEM>(h, sem, part, s, nullptr);
}

}  // namespace b2sr

extern "C" b2sr_status b2sr_spmv_bool_noalloc(b2sr_handle h, const uint32_t* x, uint32_t* y, const uint32_t* mask,
                                              int mask_complement, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (h->n > 0 && (!x || !y)) return fail(B2SR_ERR_INVALID_ARG, "x or y is NULL");
    if (x == y) return fail(B2SR_ERR_INVALID_ARG, "y must not alias x");
    int dev = 0;
    B2SR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != h->device)
        return fail(B2SR_ERR_INVALID_ARG, "the handle belongs to device " + std::to_string(h->device) +
                                              ", the current device is " + std::to_string(dev));
    b2sr_status st = B2SR_OK;
    void* scratch = noalloc_scratch_ptr(dev, &st);
    if (!scratch) return st;
    const int comp = mask_complement ? 1 : 0;
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        SemBool<K> sem{x, y, mask, comp, h->n};
        return run_spmv_bool_fixed<K>(h, sem, y, scratch, to_stream(stream));
    });
}
