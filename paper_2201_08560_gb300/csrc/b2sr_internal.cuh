// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "b2sr.h"

#define B2SR_VERSION "0.1.0"

namespace b2sr {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();
b2sr_status fail(b2sr_status st, const std::string& msg);
b2sr_status cuda_fail(cudaError_t e, const char* what);

// telemetry (telemetry.cu): launch counter and optional per-family event timing
void note_launch();
void note_launches(long long n);
bool timing_on();
// Records events around one launch of `family` moving `bytes` algorithmic bytes;
// call timing_begin before and timing_end after the launch (no-ops when off).
void* timing_begin(cudaStream_t s);
void timing_end(void* tok, const char* family, double bytes, cudaStream_t s);

#define B2SR_CUDA_TRY(expr)                                                 \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) return ::b2sr::cuda_fail(_e, #expr);         \
    } while (0)

// Every kernel launch is followed by this check, which also counts the
// launch for b2sr_launch_count().
#define B2SR_LAUNCH_CHECK(name)                                             \
    do {                                                                    \
        ::b2sr::note_launch();                                              \
        cudaError_t _e = cudaGetLastError();                                \
        if (_e != cudaSuccess) return ::b2sr::cuda_fail(_e, name);          \
    } while (0)

#define B2SR_TRY(expr)                                                      \
    do {                                                                    \
        b2sr_status _s = (expr);                                            \
        if (_s != B2SR_OK) return _s;                                       \
    } while (0)

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
__host__ __device__ inline int word_bytes(int k) { return k <= 8 ? 1 : (k == 16 ? 2 : 4); }
__host__ __device__ inline int tile_bytes(int k) { return k * word_bytes(k); }
inline bool valid_tile(int k) { return k == 4 || k == 8 || k == 16 || k == 32; }

// Tiles per warp-chunk of the SpMV kernels: 32 lanes x P tiles, P = 8, 8, 4, 2
// for k = 4, 8, 16, 32 (1-8 KB of tile data per chunk).
__host__ __device__ constexpr int tiles_per_lane(int k) {
    return k <= 8 ? 8 : (k == 16 ? 4 : 2);
}
__host__ __device__ constexpr int chunk_tiles(int k) { return 32 * tiles_per_lane(k); }
// Arrays are padded (zero-filled) to a multiple of this many tiles so a chunk
// can always be copied whole.
constexpr int64_t kTilePad = 512;
// Rows spanning more chunks than this are joined by a whole warp.
constexpr int kSplitShort = 32;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// device memory through the stream-ordered allocator
// ---------------------------------------------------------------------------
b2sr_status dmalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <class T>
b2sr_status dalloc(T** p, size_t count, cudaStream_t s) {
    return dmalloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// RAII owner for temporaries freed on a stream.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    ~DevBuf() { if (p) dfree(p, s); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    b2sr_status alloc(size_t bytes) { return dmalloc(&p, bytes, s); }
    template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

int sm_count();

// Blocks of 256 threads for a grid-stride loop over n items, at most
// blocks_per_sm per SM (and at least one block).
inline int grid_for(int64_t n, int blocks_per_sm = 8) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)sm_count() * blocks_per_sm));
}
inline int grid_wide(int64_t n) { return grid_for(n, 16); }

// Bits needed to hold the values [0, v).
inline int bits_for(int64_t v) {
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) < v) ++b;
    return b;
}

// Calls f(std::integral_constant<int, k>) for a supported tile_dim k.
template <class F>
b2sr_status with_tile(int k, F&& f) {
    switch (k) {
        case 4: return f(std::integral_constant<int, 4>());
        case 8: return f(std::integral_constant<int, 8>());
        case 16: return f(std::integral_constant<int, 16>());
        case 32: return f(std::integral_constant<int, 32>());
        default: return fail(B2SR_ERR_UNSUPPORTED_TILE, "tile_dim must be 4, 8, 16 or 32");
    }
}

}  // namespace b2sr

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
struct b2sr_matrix {
    int32_t n = 0;
    int32_t k = 0;
    int32_t ntr = 0;       // nTileRow
    int64_t T = 0;         // non-empty tiles
    int64_t nnz = 0;       // set bits
    int64_t cap = 0;       // allocated tiles (T rounded up to kTilePad, >= kTilePad)
    int32_t* rowptr = nullptr;   // [ntr+1]
    int32_t* colind = nullptr;   // [cap], zero padding after T
    uint8_t* tiles = nullptr;    // [cap * k * word_bytes], zero padding after T
    // SpMV schedule: chunk_row[c] = tile-row holding tile min(c*CT, T-1), c in [0, nchunks]
    int32_t* chunk_row = nullptr;
    int64_t nchunks = 0;
    int32_t first_row = 0;       // tile-row of tile 0 (ntr if T == 0)
    int32_t last_row = -1;       // tile-row of tile T-1 (-1 if T == 0)
    // tile-rows that span SpMV chunks: (row, first chunk, last chunk) triples,
    // rows spanning at most kSplitShort chunks first, then the longer ones
    int32_t* split = nullptr;
    int64_t nsplit_short = 0;
    int64_t nsplit_long = 0;
    // lazily built, cached derived arrays (built under the handle's mutex)
    int32_t* voff = nullptr;     // [T+1] set bits before each tile (weights offsets)
    int32_t* outdeg = nullptr;   // [n] ones per column
    int32_t schedule = 0;        // b2sr_schedule: SpMV kernel for value semirings at k <= 16
    int device = 0;
    void* mtx = nullptr;         // std::mutex*
};

namespace b2sr {
b2sr_status check_handle(const b2sr_matrix* h);
b2sr_status ensure_voff(b2sr_matrix* h, cudaStream_t s);
b2sr_status ensure_outdeg(b2sr_matrix* h, cudaStream_t s);
b2sr_status build_schedule(b2sr_matrix* h, cudaStream_t s);
// Sets *bad (device memory) non-zero if rowptr[0] != 0, rowptr[n] != nnz, a
// row pointer decreases or a column lies outside [0, n); stream-ordered.
b2sr_status validate_csr_async(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz, int* bad,
                               cudaStream_t s);
b2sr_status new_handle_from_tiles(int32_t n, int k, int64_t T, int32_t* rowptr, int32_t* colind,
                                  uint8_t* tiles, int64_t cap, cudaStream_t s, b2sr_matrix** out);

// primitives (primitives.cu)
b2sr_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
b2sr_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of keys[0..N) by bits [lo_bit, hi_bit); tmp has N entries.
// Returns in *result which buffer (keys or tmp) holds the sorted keys.
b2sr_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t N, int lo_bit, int hi_bit,
                           cudaStream_t s, uint64_t** result);
// Same, carrying a uint32 payload alongside each key.
b2sr_status radix_sort_u64_pairs(uint64_t* keys, uint64_t* ktmp, uint32_t* vals, uint32_t* vtmp,
                                 int64_t N, int lo_bit, int hi_bit, cudaStream_t s,
                                 uint64_t** kres, uint32_t** vres);
b2sr_status popcount_bytes(const uint8_t* p, int64_t bytes, int64_t* out_dev, cudaStream_t s);
b2sr_status fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s);

inline cudaStream_t to_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace b2sr

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t ld_bits(const uint32_t* __restrict__ bits, int64_t bitoff, int k) {
    // k consecutive bits starting at bitoff (bitoff % k == 0)
    const uint8_t* b8 = reinterpret_cast<const uint8_t*>(bits);
    if (k == 32) return __ldg(bits + (bitoff >> 5));
    if (k == 16) return __ldg(reinterpret_cast<const uint16_t*>(bits) + (bitoff >> 4));
    if (k == 8) return __ldg(b8 + (bitoff >> 3));
    return (__ldg(b8 + (bitoff >> 3)) >> (bitoff & 4)) & 0xFu;
}
