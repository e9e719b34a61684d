// Short-bit-width integer weights as bit-planes (Sec. VII proposes this
// extension of B2SR to weighted graphs: W = sum_p 2^p A_p with each A_p
// binary).  The planes share the pattern's tile index (TileRowPtr,
// TileColInd of the handle); plane p of tile t is a k x k bit tile in the
// handle's packing, stored tile by tile and plane by plane: byte offset
// (t * bits + p) * tile_bytes(k).
//
// SpMV over the planes:
//   bits in  -> int64 out:  y_i = sum_J sum_p 2^p popc(P_p,IJ[r] & x_J)   (exact)
//   fp32 in  -> fp32 out:   y_i = sum_j w_ij x_j, w_ij = sum_p 2^p P_p[i][j]
// Work: a warp per tile-row (lanes stride over its tiles), or a whole
// 256-thread block for tile-rows of more than kLongRow (256) tiles.  Sums
// have a fixed order (lane-sequential, then a fixed tree); the fp32 sums are
// compensated (TwoSum), so their error does not grow with the row's length.
#include <algorithm>
#include <type_traits>

#include "b2sr_internal.cuh"
#include "tile_bits.cuh"

namespace b2sr {

namespace {

constexpr int32_t kLongRow = 256;
constexpr int kLongThreads = 256;

template <int K>
constexpr int tile_bytes_k() { return K * (K <= 8 ? 1 : K / 8); }

// ---------------------------------------------------------------------------
// planes from CSR-ordered weights
// ---------------------------------------------------------------------------
template <int K>
__global__ void planes_fill_kernel(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                   const uint32_t* __restrict__ w, int64_t nnz, int bits,
                                   const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                   const uint8_t* __restrict__ tiles, uint32_t* __restrict__ planes,
                                   int* __restrict__ bad) {
    constexpr int TB = tile_bytes_k<K>();
    constexpr int WB = K <= 8 ? 1 : K / 8;  // bytes per row word
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = n - 1;  // the row i with rowptr[i] <= e < rowptr[i+1]
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo + 1) / 2;
            if (rowptr[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const int32_t i = lo, j = colind[e];
        const uint32_t wv = w[e];
        if (j < 0 || j >= n || (bits < 32 && (wv >> bits) != 0u)) { atomicOr(bad, 1); continue; }
        const int32_t I = i / K, J = j / K;
        const int r = i % K, c = j % K;
        int32_t a = trp[I], b = trp[I + 1];
        while (a < b) {
            const int32_t mid = (a + b) / 2;
            if (tci[mid] < J) a = mid + 1;
            else b = mid;
        }
        if (a == trp[I + 1] || tci[a] != J) { atomicOr(bad, 1); continue; }
        const int64_t t = a;
        const int64_t off = (int64_t)r * WB + (c >> 3);  // byte of bit (r, c) within a tile
        if (!((tiles[t * TB + off] >> (c & 7)) & 1u)) { atomicOr(bad, 1); continue; }
        for (int p = 0; p < bits; ++p) {
            if (!((wv >> p) & 1u)) continue;
            const int64_t byte = (t * bits + p) * TB + off;
            atomicOr(planes + (byte >> 2), 1u << ((int)(byte & 3) * 8 + (c & 7)));
        }
    }
}

// ---------------------------------------------------------------------------
// SpMV over the planes
// ---------------------------------------------------------------------------
struct TwoSum {
    float s = 0.0f, c = 0.0f;
};

__device__ __forceinline__ TwoSum two_sum_add(TwoSum a, float b) {
    const float t = __fadd_rn(a.s, b);
    const float bp = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(b, bp));
    return TwoSum{t, __fadd_rn(a.c, e)};
}

__device__ __forceinline__ TwoSum two_sum_join(TwoSum a, TwoSum b) {
    TwoSum r = two_sum_add(a, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}

__device__ __forceinline__ bool row_kept(const uint32_t* mask, int comp, int64_t i) {
    if (!mask) return true;
    const bool b = (__ldg(mask + (i >> 5)) >> (i & 31)) & 1u;
    return comp ? !b : b;
}

constexpr int kMaxBits = 16;

// The words of every plane of tile t (planes past `bits` read as zero), with
// the loads issued together rather than one plane after another.
template <int TW, int TB>
__device__ __forceinline__ void load_planes(const uint8_t* __restrict__ planes, int bits, int64_t t,
                                            uint32_t (&pw)[kMaxBits][TW]) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(planes + t * bits * TB);  // plane p at src + p * TW
#pragma unroll
    for (int p = 0; p < kMaxBits; ++p)
#pragma unroll
        for (int q = 0; q < TW; ++q) pw[p][q] = 0u;
#pragma unroll
    for (int p = 0; p < kMaxBits; ++p) {
        if (p >= bits) break;
#pragma unroll
        for (int q = 0; q < TW; ++q) pw[p][q] = __ldg(src + p * TW + q);
    }
}

// The contributions of tile t to the K rows of its tile-row.
template <int K, bool BITS>
struct PlaneRows {
    using Acc = typename std::conditional<BITS, long long, TwoSum>::type;
    Acc acc[K];

    __device__ void zero() {
#pragma unroll
        for (int r = 0; r < K; ++r) acc[r] = Acc{};
    }

    // k <= 8: a tile's planes held in registers, so that two tiles' loads
    // can be in flight together (fetch both, then accumulate both)
    struct Fetched {
        uint32_t pw[kMaxBits][(tile_bytes_k<K>() + 3) / 4];
        int32_t J;
        uint32_t xs;
    };

    __device__ __forceinline__ void fetch(const uint8_t* __restrict__ planes, int bits, int64_t t, int32_t J,
                                          const uint32_t* xb, Fetched& f) const {
        constexpr int TB = tile_bytes_k<K>();
        constexpr int TW = TB / 4;
        f.J = J;
        f.xs = BITS ? seg_bits<K>(xb, J) : 1u;
        if (f.xs) {
            load_planes<TW, TB>(planes, bits, t, f.pw);
        } else {
#pragma unroll
            for (int p = 0; p < kMaxBits; ++p)
#pragma unroll
                for (int q = 0; q < TW; ++q) f.pw[p][q] = 0u;
        }
    }

    __device__ __forceinline__ void accumulate(const Fetched& f, int bits, const float* xf) {
        if constexpr (BITS) {
            if (!f.xs) return;
#pragma unroll
            for (int p = 0; p < kMaxBits; ++p) {
                if (p >= bits) break;
#pragma unroll
                for (int r = 0; r < K; ++r) acc[r] += (long long)__popc(tile_row<K>(f.pw[p], r) & f.xs) << p;
            }
        } else {
#pragma unroll
            for (int r = 0; r < K; ++r) {
                uint32_t rows[kMaxBits];
                uint32_t any = 0u;
#pragma unroll
                for (int p = 0; p < kMaxBits; ++p) {
                    rows[p] = tile_row<K>(f.pw[p], r);
                    any |= rows[p];
                }
                while (any) {
                    const int c = __ffs(any) - 1;
                    any &= any - 1;
                    uint32_t wv = 0u;
#pragma unroll
                    for (int p = 0; p < kMaxBits; ++p) {
                        if (p >= bits) break;
                        wv |= ((rows[p] >> c) & 1u) << p;
                    }
                    acc[r] = two_sum_add(acc[r], __fmul_rn((float)wv, __ldg(xf + (int64_t)f.J * K + c)));
                }
            }
        }
    }

    // tiles ta and (if has_b) tb, in that order
    __device__ __forceinline__ void add_pair(const uint8_t* __restrict__ planes, int bits, int64_t ta, int32_t Ja,
                                             bool has_b, int64_t tb, int32_t Jb, const uint32_t* xb,
                                             const float* xf) {
        if constexpr (K <= 8) {
            Fetched fa, fb;
            fetch(planes, bits, ta, Ja, xb, fa);
            if (has_b) fetch(planes, bits, tb, Jb, xb, fb);
            accumulate(fa, bits, xf);
            if (has_b) accumulate(fb, bits, xf);
        } else {
            add_tile(planes, bits, ta, Ja, xb, xf);
            if (has_b) add_tile(planes, bits, tb, Jb, xb, xf);
        }
    }

    // k >= 16: plane by plane from global memory (a tile's planes are too
    // many registers to hold at once)
    __device__ void add_tile(const uint8_t* __restrict__ planes, int bits, int64_t t, int32_t J, const uint32_t* xb,
                             const float* xf) {
        constexpr int TB = tile_bytes_k<K>();
        constexpr int TW = TB / 4;
        if constexpr (BITS) {
            const uint32_t xs = seg_bits<K>(xb, J);
            if (!xs) return;
            for (int p = 0; p < bits; ++p) {
                const uint32_t* pw = reinterpret_cast<const uint32_t*>(planes + (t * bits + p) * TB);
                uint32_t wd[TW];
#pragma unroll
                for (int q = 0; q < TW; ++q) wd[q] = __ldg(pw + q);
#pragma unroll
                for (int r = 0; r < K; ++r) acc[r] += (long long)__popc(tile_row<K>(wd, r) & xs) << p;
            }
        } else {
#pragma unroll
            for (int r = 0; r < K; ++r) {
                uint32_t any = 0u;
                for (int p = 0; p < bits; ++p) {
                    const uint32_t* pw = reinterpret_cast<const uint32_t*>(planes + (t * bits + p) * TB);
                    any |= tile_row<K>(pw, r);
                }
                while (any) {
                    const int c = __ffs(any) - 1;
                    any &= any - 1;
                    uint32_t wv = 0u;
                    for (int p = 0; p < bits; ++p) {
                        const uint32_t* pw = reinterpret_cast<const uint32_t*>(planes + (t * bits + p) * TB);
                        wv |= ((tile_row<K>(pw, r) >> c) & 1u) << p;
                    }
                    acc[r] = two_sum_add(acc[r], __fmul_rn((float)wv, __ldg(xf + (int64_t)J * K + c)));
                }
            }
        }
    }
};

template <class A>
__device__ __forceinline__ A shfl_acc(A v, int o) {
    if constexpr (std::is_same<A, long long>::value) {
        return __shfl_xor_sync(0xffffffffu, v, o);
    } else {
        A r;
        r.s = __shfl_xor_sync(0xffffffffu, v.s, o);
        r.c = __shfl_xor_sync(0xffffffffu, v.c, o);
        return r;
    }
}

template <class A>
__device__ __forceinline__ A join(A a, A b) {
    if constexpr (std::is_same<A, long long>::value) return a + b;
    else return two_sum_join(a, b);
}

template <class A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const A u = shfl_acc(v, o);
        // the lower lane's value first, so every lane forms the same sum
        v = (lane_id() & o) ? join(u, v) : join(v, u);
    }
    return v;
}

template <bool BITS>
__device__ __forceinline__ void store_y(void* y, int64_t i, typename PlaneRows<4, BITS>::Acc v, bool kept) {
    if constexpr (BITS) static_cast<long long*>(y)[i] = kept ? v : 0ll;
    else static_cast<float*>(y)[i] = kept ? __fadd_rn(v.s, v.c) : 0.0f;
}

// a warp per tile-row of at most kLongRow tiles
template <int K, bool BITS>
__global__ void __launch_bounds__(256) planes_rows_kernel(const int32_t* __restrict__ trp,
                                                          const int32_t* __restrict__ tci,
                                                          const uint8_t* __restrict__ planes, int bits, int32_t ntr,
                                                          int32_t n, const uint32_t* xb, const float* xf, void* y,
                                                          const uint32_t* mask, int comp) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = (int)lane_id();
    for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < ntr; I += warps) {
        const int32_t t0 = __ldg(trp + I), t1 = __ldg(trp + I + 1);
        if (t1 - t0 > kLongRow) continue;
        PlaneRows<K, BITS> pr;
        pr.zero();
        for (int32_t t = t0 + lane; t < t1; t += 64) {
            const bool has_b = t + 32 < t1;
            pr.add_pair(planes, bits, t, __ldg(tci + t), has_b, t + 32, has_b ? __ldg(tci + t + 32) : 0, xb, xf);
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const auto v = warp_sum(pr.acc[r]);
            const int64_t i = I * K + r;
            if (lane == r && i < n) store_y<BITS>(y, i, v, row_kept(mask, comp, i));
        }
    }
}

// tile-rows of more than kLongRow tiles, listed
__global__ void planes_long_list_kernel(const int32_t* __restrict__ trp, int32_t ntr, int32_t* list, int32_t* count) {
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < ntr; I += (int64_t)gridDim.x * blockDim.x)
        if (trp[I + 1] - trp[I] > kLongRow) list[atomicAdd(count, 1)] = (int32_t)I;
}

// a block per long tile-row: threads stride over its tiles, then warp sums
// joined in warp order through shared memory
template <int K, bool BITS>
__global__ void __launch_bounds__(kLongThreads) planes_long_kernel(const int32_t* __restrict__ trp,
                                                                   const int32_t* __restrict__ tci,
                                                                   const uint8_t* __restrict__ planes, int bits,
                                                                   const int32_t* list, const int32_t* count,
                                                                   int32_t n, const uint32_t* xb, const float* xf,
                                                                   void* y, const uint32_t* mask, int comp) {
    using Acc = typename PlaneRows<K, BITS>::Acc;
    __shared__ Acc part[kLongThreads / 32][K];
    const int nlong = *count;
    const int warp = threadIdx.x >> 5, lane = (int)lane_id();
    for (int e = blockIdx.x; e < nlong; e += gridDim.x) {
        const int32_t I = list[e];
        const int32_t t0 = __ldg(trp + I), t1 = __ldg(trp + I + 1);
        PlaneRows<K, BITS> pr;
        pr.zero();
        for (int32_t t = t0 + threadIdx.x; t < t1; t += 2 * kLongThreads) {
            const bool has_b = t + kLongThreads < t1;
            pr.add_pair(planes, bits, t, __ldg(tci + t), has_b, t + kLongThreads,
                        has_b ? __ldg(tci + t + kLongThreads) : 0, xb, xf);
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const Acc v = warp_sum(pr.acc[r]);
            if (lane == 0) part[warp][r] = v;
        }
        __syncthreads();
        if (threadIdx.x < K) {
            const int r = threadIdx.x;
            Acc v = part[0][r];
            for (int w = 1; w < kLongThreads / 32; ++w) v = join(v, part[w][r]);
            const int64_t i = (int64_t)I * K + r;
            if (i < n) store_y<BITS>(y, i, v, row_kept(mask, comp, i));
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_planes_from_csr(b2sr_handle h, const int32_t* rowptr, const int32_t* colind,
                                            const uint32_t* w_csr, int bits, void* planes, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (bits < 1 || bits > 16) return fail(B2SR_ERR_INVALID_ARG, "bits must be in [1, 16]");
    if (h->T == 0) return B2SR_OK;
    if (!rowptr || !colind || !w_csr || !planes) return fail(B2SR_ERR_INVALID_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(planes) % 4) return fail(B2SR_ERR_INVALID_ARG, "planes must be 4-byte aligned");
    cudaStream_t s = to_stream(stream);
    const size_t bytes = (size_t)h->T * bits * tile_bytes(h->k);
    B2SR_CUDA_TRY(cudaMemsetAsync(planes, 0, bytes, s));
    DevBuf bad(s);
    B2SR_TRY(bad.alloc(sizeof(int)));
    B2SR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    B2SR_TRY(with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        if (h->nnz > 0)
            planes_fill_kernel<K><<<grid_for(h->nnz), 256, 0, s>>>(h->n, rowptr, colind, w_csr, h->nnz, bits,
                                                                   h->rowptr, h->colind, h->tiles,
                                                                   static_cast<uint32_t*>(planes), bad.as<int>());
        B2SR_LAUNCH_CHECK("planes_fill_kernel");
        return B2SR_OK;
    }));
    int hbad = 0;
    B2SR_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return fail(B2SR_ERR_INVALID_ARG, "CSR does not match the handle, or a weight is too wide");
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_spmv_planes(b2sr_handle h, const void* planes, int bits, b2sr_vec in_kind,
                                        const void* x, b2sr_vec out_kind, void* y, const uint32_t* mask,
                                        int mask_complement, void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (bits < 1 || bits > 16) return fail(B2SR_ERR_INVALID_ARG, "bits must be in [1, 16]");
    const bool bits_in = in_kind == B2SR_VEC_BITS && out_kind == B2SR_VEC_I64;
    const bool f32_in = in_kind == B2SR_VEC_F32 && out_kind == B2SR_VEC_F32;
    if (!bits_in && !f32_in) return fail(B2SR_ERR_INVALID_ARG, "BITS -> I64 or F32 -> F32");
    if (h->n == 0) return B2SR_OK;
    if ((h->T > 0 && !planes) || !x || !y) return fail(B2SR_ERR_INVALID_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(planes) % 4) return fail(B2SR_ERR_INVALID_ARG, "planes must be 4-byte aligned");
    cudaStream_t s = to_stream(stream);
    const int comp = mask_complement ? 1 : 0;
    const uint8_t* pl = static_cast<const uint8_t*>(planes);
    DevBuf lbuf(s);
    B2SR_TRY(lbuf.alloc(((size_t)h->ntr + 2) * sizeof(int32_t)));
    int32_t* count = lbuf.as<int32_t>();
    int32_t* list = count + 1;
    B2SR_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), s));
    planes_long_list_kernel<<<grid_for(h->ntr), 256, 0, s>>>(h->rowptr, h->ntr, list, count);
    B2SR_LAUNCH_CHECK("planes_long_list_kernel");
    return with_tile(h->k, [&](auto kc) -> b2sr_status {
        constexpr int K = decltype(kc)::value;
        const int rows_grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->ntr, 8), sm_count() * 8));
        const int long_grid = sm_count() * 8;
        const uint32_t* xb = static_cast<const uint32_t*>(x);
        const float* xf = static_cast<const float*>(x);
        double bytes = 4.0 * ((double)h->ntr + 1.0) + (double)h->T * (4.0 + (double)bits * tile_bytes(h->k)) +
                       (mask ? h->n / 8.0 : 0.0);
        if (bits_in) {
            void* tok = timing_begin(s);
            planes_rows_kernel<K, true><<<rows_grid, 256, 0, s>>>(h->rowptr, h->colind, pl, bits, h->ntr, h->n, xb,
                                                                  nullptr, y, mask, comp);
            B2SR_LAUNCH_CHECK("planes_rows_kernel");
            planes_long_kernel<K, true><<<long_grid, kLongThreads, 0, s>>>(h->rowptr, h->colind, pl, bits, list,
                                                                            count, h->n, xb, nullptr, y, mask, comp);
            B2SR_LAUNCH_CHECK("planes_long_kernel");
            timing_end(tok, "spmv_planes_count", bytes + h->n / 8.0 + 8.0 * h->n, s);
        } else {
            void* tok = timing_begin(s);
            planes_rows_kernel<K, false><<<rows_grid, 256, 0, s>>>(h->rowptr, h->colind, pl, bits, h->ntr, h->n,
                                                                   nullptr, xf, y, mask, comp);
            B2SR_LAUNCH_CHECK("planes_rows_kernel");
            planes_long_kernel<K, false><<<long_grid, kLongThreads, 0, s>>>(h->rowptr, h->colind, pl, bits, list,
                                                                             count, h->n, nullptr, xf, y, mask, comp);
            B2SR_LAUNCH_CHECK("planes_long_kernel");
            timing_end(tok, "spmv_planes_plus", bytes + 8.0 * h->n, s);
        }
        return B2SR_OK;
    });
}
