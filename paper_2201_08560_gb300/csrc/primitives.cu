// Error plumbing, stream-ordered allocation and the generic device primitives
// (exclusive scan, stable LSD radix sort, popcount reduction) used by the
// B2SR conversion and SpGEMM kernels.
#include <cstdio>
#include <mutex>
#include <string>

#include "b2sr_internal.cuh"

namespace b2sr {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }

b2sr_status fail(b2sr_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

b2sr_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(B2SR_ERR_OOM, m);
    return fail(B2SR_ERR_CUDA, m);
}

// Device memory comes from a stream-ordered pool of the library's own, one per
// device, created on first use.  It keeps freed memory for reuse (up to a
// quarter of the device) instead of returning it to the driver at every
// synchronisation, so the conversion's sort buffers and every driver's
// temporaries are re-used from call to call rather than mapped again.  Being
// private, it leaves the process's default pool, which the host application
// may tune for itself, untouched.
static cudaMemPool_t library_pool(int dev) {
    static std::once_flag once[64];
    static cudaMemPool_t pools[64] = {nullptr};
    if (dev < 0 || dev >= 64) return nullptr;
    std::call_once(once[dev], [dev] {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
                uint64_t keep = (uint64_t)total_b / 4;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            pools[dev] = pool;
        }
        cudaGetLastError();
    });
    return pools[dev];
}

b2sr_status dmalloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    int dev = 0;
    B2SR_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool = library_pool(dev);
    if (!pool) return fail(B2SR_ERR_CUDA, "could not create the library's memory pool on device " + std::to_string(dev));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(B2SR_ERR_OOM, "cudaMallocFromPoolAsync(" + std::to_string(bytes) + " bytes) failed: " +
                                      cudaGetErrorString(e));
    }
    return B2SR_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// exclusive scan (reduce, scan the block sums, then scan-and-add)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class TIn>
__global__ void __launch_bounds__(kScanThreads) scan_block_sums(const TIn* __restrict__ in, int64_t n,
                                                                int64_t* __restrict__ sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc = 0;
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) acc += (int64_t)in[i];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane_id() == 0) warp_tot[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = threadIdx.x < kScanThreads / 32 ? warp_tot[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// Shared-memory slot of tile item i: one pad word per 16 keeps both the
// striped (item j * kScanThreads + t) and the blocked (item t * kScanItems + j)
// accesses of 64-bit words free of bank conflicts.
__device__ __forceinline__ int scan_slot(int i) { return i + (i >> 4); }

// Exclusive scan of one tile of kScanTile items, plus a per-block offset.
template <class TIn>
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const TIn* __restrict__ in, int64_t n,
                                                           int64_t* __restrict__ out,
                                                           const int64_t* __restrict__ block_off) {
    __shared__ int64_t sm[kScanTile + kScanTile / 16];
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j * kScanThreads + threadIdx.x;
        sm[scan_slot(j * kScanThreads + threadIdx.x)] = i < n ? (int64_t)in[i] : 0;
    }
    __syncthreads();
    int64_t v[kScanItems];
    int64_t run = 0;
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = run;
        run += sm[scan_slot(threadIdx.x * kScanItems + j)];
    }
    // warp inclusive scan of per-thread totals
    int64_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane_id() >= o) inc += t;
    }
    if (lane_id() == 31) warp_tot[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t w = threadIdx.x < kScanThreads / 32 ? warp_tot[threadIdx.x] : 0;
        int64_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if ((int)lane_id() >= o) wi += t;
        }
        if (threadIdx.x < kScanThreads / 32) warp_tot[threadIdx.x] = wi - w;  // exclusive
    }
    __syncthreads();
    int64_t off = (block_off ? block_off[blockIdx.x] : 0) + warp_tot[threadIdx.x >> 5] + (inc - run);
    for (int j = 0; j < kScanItems; ++j) sm[scan_slot(threadIdx.x * kScanItems + j)] = v[j] + off;
    __syncthreads();
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) out[i] = sm[scan_slot(j * kScanThreads + threadIdx.x)];
    }
}

template <class TIn>
static b2sr_status exclusive_scan_impl(const TIn* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return B2SR_OK;
    int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        scan_tiles<TIn><<<1, kScanThreads, 0, s>>>(in, n, out, nullptr);
        B2SR_LAUNCH_CHECK("scan_tiles");
        return B2SR_OK;
    }
    DevBuf sums(s), offs(s);
    B2SR_TRY(sums.alloc(nb * sizeof(int64_t)));
    B2SR_TRY(offs.alloc(nb * sizeof(int64_t)));
    scan_block_sums<TIn><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.as<int64_t>());
    B2SR_LAUNCH_CHECK("scan_block_sums");
    B2SR_TRY(exclusive_scan_impl<int64_t>(sums.as<int64_t>(), offs.as<int64_t>(), nb, s));
    scan_tiles<TIn><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, out, offs.as<int64_t>());
    B2SR_LAUNCH_CHECK("scan_tiles");
    return B2SR_OK;
}

b2sr_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return exclusive_scan_impl<int32_t>(in, out, n, s);
}

b2sr_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return exclusive_scan_impl<int64_t>(in, out, n, s);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
//   pass: per-block digit histogram -> scan (digit-major) -> stable scatter.
//   Within a block, warp w owns items [w*32*I, (w+1)*32*I) and ranks them
//   round by round with __match_any_sync, so equal digits keep input order.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) radix_hist(const uint64_t* __restrict__ keys, int64_t N,
                                                           int shift, int64_t nb,
                                                           int64_t* __restrict__ counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = 0; j < kSortItems; ++j) {
        int64_t i = base + j * kSortThreads + threadIdx.x;
        if (i < N) atomicAdd(&h[(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

template <bool PAIRS>
__global__ void __launch_bounds__(kSortThreads) radix_scatter(const uint64_t* __restrict__ keys,
                                                              const uint32_t* __restrict__ vals,
                                                              int64_t N, int shift, int64_t nb,
                                                              const int64_t* __restrict__ offsets,
                                                              uint64_t* __restrict__ keys_out,
                                                              uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t cnt[kSortWarps][257];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    for (int d = lane; d < 257; d += 32) cnt[w][d] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * 32 * kSortItems;
    uint64_t key[kSortItems];
    uint32_t rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        int64_t i = base + j * 32 + lane;
        bool valid = i < N;
        key[j] = valid ? keys[i] : 0;
        unsigned d = valid ? (unsigned)((key[j] >> shift) & 0xFFu) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = cnt[w][d];
        rank[j] = before + __popc(peers & lt);
        __syncwarp();
        if (lane == 31u - __clz(peers)) cnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    {
        int d = threadIdx.x;  // 256 threads, 256 digits
        uint32_t run = 0;
        for (int ww = 0; ww < kSortWarps; ++ww) {
            uint32_t t = cnt[ww][d];
            cnt[ww][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        int64_t i = base + j * 32 + lane;
        if (i < N) {
            unsigned d = (unsigned)((key[j] >> shift) & 0xFFu);
            int64_t pos = offsets[(int64_t)d * nb + blockIdx.x] + cnt[w][d] + rank[j];
            keys_out[pos] = key[j];
            if (PAIRS) vals_out[pos] = vals[i];
        }
    }
}

// Keys only: the same ranking, then the block's keys are placed in shared
// memory in output order (digit by digit) and written out by consecutive
// threads, so each digit's run goes to global memory in whole sectors.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_staged(const uint64_t* __restrict__ keys, int64_t N,
                                                                     int shift, int64_t nb,
                                                                     const int64_t* __restrict__ offsets,
                                                                     uint64_t* __restrict__ keys_out) {
    __shared__ uint32_t cnt[kSortWarps][257];
    __shared__ uint32_t dstart[256];  // block-local start of each digit's run
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint64_t stage[kSortTile];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    for (int d = lane; d < 257; d += 32) cnt[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * 32 * kSortItems;
    uint64_t key[kSortItems];
    uint32_t rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j * 32 + lane;
        const bool valid = i < N;
        key[j] = valid ? keys[i] : 0;
        const unsigned d = valid ? (unsigned)((key[j] >> shift) & 0xFFu) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = cnt[w][d];
        rank[j] = before + __popc(peers & lt);
        __syncwarp();
        if (lane == 31u - __clz(peers)) cnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps; the digit's block total
    const int d = threadIdx.x;  // 256 threads, 256 digits
    uint32_t total = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
        const uint32_t t = cnt[ww][d];
        cnt[ww][d] = total;
        total += t;
    }
    // exclusive scan of the totals over the digits (warp scans, then warp sums)
    uint32_t inc = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t before_w = 0;
    for (int ww = 0; ww < w; ++ww) before_w += wsum[ww];
    dstart[d] = before_w + inc - total;
    __syncthreads();
    uint32_t nvalid = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) nvalid += wsum[ww];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j * 32 + lane;
        if (i < N) {
            const unsigned dd = (unsigned)((key[j] >> shift) & 0xFFu);
            stage[dstart[dd] + cnt[w][dd] + rank[j]] = key[j];
        }
    }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < nvalid; p += kSortThreads) {
        const uint64_t k = stage[p];
        const unsigned dd = (unsigned)((k >> shift) & 0xFFu);
        keys_out[offsets[(int64_t)dd * nb + blockIdx.x] + (p - dstart[dd])] = k;
    }
}

template <bool PAIRS>
static b2sr_status radix_sort_impl(uint64_t* keys, uint64_t* ktmp, uint32_t* vals, uint32_t* vtmp,
                                   int64_t N, int lo_bit, int hi_bit, cudaStream_t s,
                                   uint64_t** kres, uint32_t** vres) {
    *kres = keys;
    if (vres) *vres = vals;
    if (N <= 1 || hi_bit <= lo_bit) return B2SR_OK;
    int64_t nb = ceil_div(N, kSortTile);
    DevBuf counts(s), offs(s);
    B2SR_TRY(counts.alloc(256 * nb * sizeof(int64_t)));
    B2SR_TRY(offs.alloc(256 * nb * sizeof(int64_t)));
    uint64_t* kin = keys;
    uint64_t* kout = ktmp;
    uint32_t* vin = vals;
    uint32_t* vout = vtmp;
    for (int shift = lo_bit; shift < hi_bit; shift += 8) {
        radix_hist<<<(unsigned)nb, kSortThreads, 0, s>>>(kin, N, shift, nb, counts.as<int64_t>());
        B2SR_LAUNCH_CHECK("radix_hist");
        B2SR_TRY(exclusive_scan_i64(counts.as<int64_t>(), offs.as<int64_t>(), 256 * nb, s));
        if (PAIRS) {
            radix_scatter<PAIRS><<<(unsigned)nb, kSortThreads, 0, s>>>(kin, vin, N, shift, nb,
                                                                       offs.as<int64_t>(), kout, vout);
            B2SR_LAUNCH_CHECK("radix_scatter");
        } else {
            radix_scatter_staged<<<(unsigned)nb, kSortThreads, 0, s>>>(kin, N, shift, nb, offs.as<int64_t>(), kout);
            B2SR_LAUNCH_CHECK("radix_scatter_staged");
        }
        uint64_t* t = kin; kin = kout; kout = t;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    *kres = kin;
    if (vres) *vres = vin;
    return B2SR_OK;
}

b2sr_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t N, int lo_bit, int hi_bit,
                           cudaStream_t s, uint64_t** result) {
    return radix_sort_impl<false>(keys, tmp, nullptr, nullptr, N, lo_bit, hi_bit, s, result, nullptr);
}

b2sr_status radix_sort_u64_pairs(uint64_t* keys, uint64_t* ktmp, uint32_t* vals, uint32_t* vtmp,
                                 int64_t N, int lo_bit, int hi_bit, cudaStream_t s,
                                 uint64_t** kres, uint32_t** vres) {
    return radix_sort_impl<true>(keys, ktmp, vals, vtmp, N, lo_bit, hi_bit, s, kres, vres);
}

// ---------------------------------------------------------------------------
// small utilities
// ---------------------------------------------------------------------------
__global__ void popcount_words(const uint32_t* __restrict__ p, int64_t nwords,
                               unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += __popc(p[i]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane_id() == 0 && acc) atomicAdd(out, acc);
}

b2sr_status popcount_bytes(const uint8_t* p, int64_t bytes, int64_t* out_dev, cudaStream_t s) {
    B2SR_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(int64_t), s));
    int64_t nwords = bytes / 4;  // callers pass 4-byte multiples
    if (nwords == 0) return B2SR_OK;
    int grid = (int)std::min<int64_t>(ceil_div(nwords, 256), (int64_t)sm_count() * 8);
    popcount_words<<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(p), nwords,
                                        reinterpret_cast<unsigned long long*>(out_dev));
    B2SR_LAUNCH_CHECK("popcount_words");
    return B2SR_OK;
}

__global__ void fill_i32_kernel(int32_t* p, int32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

b2sr_status fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return B2SR_OK;
    int grid = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)sm_count() * 8);
    fill_i32_kernel<<<grid, 256, 0, s>>>(p, v, n);
    B2SR_LAUNCH_CHECK("fill_i32");
    return B2SR_OK;
}

}  // namespace b2sr

extern "C" const char* b2sr_last_error(void) { return b2sr::t_last_error.c_str(); }
extern "C" const char* b2sr_version(void) { return B2SR_VERSION; }
