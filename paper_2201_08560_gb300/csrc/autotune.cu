// Tile size selection (Sec. III-C "Sampling Profile and Tile Size
// Configuration", Algorithm 1): the sampling estimate of the B2SR size for
// every tile_dim, computed on the device, followed by timed SpMV trials of the
// candidate tile_dims and schedules that the estimate keeps.
//
// Estimate.  Each sampled row i stands for its tile-row i / k; the distinct
// tile columns of that tile-row (column / k over its k rows) are counted, and
// their mean times nTileRow estimates the tile count T_k.  The counting sorts
// (segment, tile column) keys of every sampled tile-row for the four k at once
// and counts segment heads, so the result is an exact integer count.
#include <algorithm>
#include <cmath>
#include <vector>

#include "b2sr_internal.cuh"

namespace b2sr {
b2sr_status spmv_dispatch(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in_kind, const void* x, b2sr_vec out_kind,
                          void* y, const uint32_t* mask, int comp, const float* weights, cudaStream_t s,
                          const int32_t* gate);
b2sr_status spmm64_dispatch(b2sr_matrix* h, const uint64_t* X, uint64_t* Y, const uint64_t* M, int comp,
                            cudaStream_t s, const int32_t* gate);

static const int kTileDims[4] = {4, 8, 16, 32};

// segment g = q * ns + s: rows [r0, r1) of the tile-row of sample s at k = 4 << q
__device__ __forceinline__ void seg_rows(int64_t g, int64_t ns, const int32_t* __restrict__ sample, int32_t n,
                                         int32_t* r0, int32_t* r1, int* k) {
    const int q = (int)(g / ns);
    *k = 4 << q;
    const int32_t I = sample[g - q * ns] / *k;
    *r0 = I * *k;
    *r1 = min(*r0 + *k, n);
}

__global__ void profile_len_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ sample,
                                   int64_t ns, int32_t n, int64_t nnz, int32_t* __restrict__ len, int32_t* bad) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < 4 * ns;
         g += (int64_t)gridDim.x * blockDim.x) {
        int32_t r0, r1;
        int k;
        seg_rows(g, ns, sample, n, &r0, &r1, &k);
        const int32_t a = rowptr[r0], b = rowptr[r1];
        if (a < 0 || b < a || b > nnz) {
            atomicOr(bad, 1);
            len[g] = 0;
        } else {
            len[g] = b - a;
        }
    }
}

// warp per segment: key = segment << 31 | tile column
__global__ void profile_keys_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                    const int32_t* __restrict__ sample, int64_t ns, int32_t n,
                                    const int32_t* __restrict__ len, const int64_t* __restrict__ off,
                                    uint64_t* __restrict__ keys) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < 4 * ns; g += warps) {
        int32_t r0, r1;
        int k;
        seg_rows(g, ns, sample, n, &r0, &r1, &k);
        const int32_t a = rowptr[r0];
        const int32_t m = len[g];
        uint64_t* out = keys + off[g];
        for (int32_t e = lane_id(); e < m; e += 32) {
            const uint32_t c = (uint32_t)colind[a + e];
            out[e] = ((uint64_t)g << 31) | (uint64_t)(c / (uint32_t)k);
        }
    }
}

// distinct keys per k: heads of the sorted key runs, counted per q
__global__ void profile_heads_kernel(const uint64_t* __restrict__ keys, int64_t N, int64_t ns,
                                     unsigned long long* __restrict__ cnt) {
    __shared__ unsigned long long c[4];
    if (threadIdx.x < 4) c[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned local[4] = {0u, 0u, 0u, 0u};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        if (i == 0 || keys[i - 1] != key) {
            const int q = (int)((int64_t)(key >> 31) / ns);
            local[q] += 1u;
        }
    }
    for (int q = 0; q < 4; ++q)
        if (local[q]) atomicAdd(&c[q], (unsigned long long)local[q]);
    __syncthreads();
    if (threadIdx.x < 4 && c[threadIdx.x]) atomicAdd(cnt + threadIdx.x, c[threadIdx.x]);
}

b2sr_status sample_profile(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                           const int32_t* sample_host, int64_t ns, double* est, double* tiles_est, cudaStream_t s) {
    int64_t cnt_host[4] = {0, 0, 0, 0};
    if (ns > 0) {
        const int64_t G = 4 * ns;
        DevBuf meta(s);
        // sample[ns] | len[G] | off[G] (int64) | cnt[4] | bad
        const size_t sample_b = round_up(ns * sizeof(int32_t), 256);
        const size_t len_b = round_up(G * sizeof(int32_t), 256);
        const size_t off_b = round_up(G * sizeof(int64_t), 256);
        B2SR_TRY(meta.alloc(sample_b + len_b + off_b + 256));
        char* base = meta.as<char>();
        int32_t* dsample = reinterpret_cast<int32_t*>(base);
        int32_t* len = reinterpret_cast<int32_t*>(base + sample_b);
        int64_t* off = reinterpret_cast<int64_t*>(base + sample_b + len_b);
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + sample_b + len_b + off_b);
        int32_t* bad = reinterpret_cast<int32_t*>(cnt + 4);
        B2SR_CUDA_TRY(cudaMemcpyAsync(dsample, sample_host, ns * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        B2SR_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long) + sizeof(int32_t), s));
        profile_len_kernel<<<grid_for(G), 256, 0, s>>>(rowptr, dsample, ns, n, nnz, len, bad);
        B2SR_LAUNCH_CHECK("profile_len_kernel");
        B2SR_TRY(exclusive_scan_i32_to_i64(len, off, G, s));
        int64_t tail[2] = {0, 0};
        int32_t last_len = 0, bad_host = 0;
        B2SR_CUDA_TRY(cudaMemcpyAsync(&tail[0], off + G - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaMemcpyAsync(&last_len, len + G - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaMemcpyAsync(&bad_host, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
        if (bad_host) return fail(B2SR_ERR_INVALID_ARG, "rowptr is malformed at a sampled tile-row");
        const int64_t N = tail[0] + last_len;
        if (N > 0) {
            DevBuf kb(s);
            B2SR_TRY(kb.alloc(2 * N * sizeof(uint64_t)));
            uint64_t* keys = kb.as<uint64_t>();
            profile_keys_kernel<<<grid_for(G * 32), 256, 0, s>>>(rowptr, colind, dsample, ns, n, len, off, keys);
            B2SR_LAUNCH_CHECK("profile_keys_kernel");
            uint64_t* sorted = nullptr;
            B2SR_TRY(radix_sort_u64(keys, keys + N, N, 0, 31 + bits_for(G), s, &sorted));
            profile_heads_kernel<<<grid_for(N), 256, 0, s>>>(sorted, N, ns, cnt);
            B2SR_LAUNCH_CHECK("profile_heads_kernel");
        }
        B2SR_CUDA_TRY(cudaMemcpyAsync(cnt_host, cnt, sizeof(cnt_host), cudaMemcpyDeviceToHost, s));
        B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    for (int q = 0; q < 4; ++q) {
        const int k = kTileDims[q];
        const int64_t ntr = ((int64_t)n + k - 1) / k;
        const double t_hat = ns > 0 ? (double)cnt_host[q] / (double)ns * (double)ntr : 0.0;
        const double b2sr_bytes = 4.0 * (double)(ntr + 1) + t_hat * (4.0 + (double)(k * word_bytes(k)));
        const double csr_bytes = 4.0 * ((double)n + 1.0) + 8.0 * (double)nnz;
        if (est) est[q] = b2sr_bytes / csr_bytes;
        if (tiles_est) tiles_est[q] = t_hat;
    }
    return B2SR_OK;
}

// Deterministic synthetic trial vector: bits of a 32-bit hash (bitsets),
// values in [0, 1) (floats) or [0, 2^20) (ints).
__global__ void trial_vector_kernel(uint32_t* v, int64_t words, int kind) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u + 0x7F4A7C15u;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        if (kind == B2SR_VEC_F32) {
            const float f = (float)(h >> 8) * (1.0f / 16777216.0f);
            v[i] = __float_as_uint(f);
        } else if (kind == B2SR_VEC_I32) {
            v[i] = h >> 12;
        } else {
            v[i] = h;
        }
    }
}

static bool scheme_ok(b2sr_semiring sr, b2sr_vec in, b2sr_vec* out) {
    if (sr == B2SR_BOOL_OR_AND && in == B2SR_VEC_BITS) { *out = B2SR_VEC_BITS; return true; }
    if (sr == B2SR_BOOL_OR_AND && in == B2SR_VEC_BITS64) { *out = B2SR_VEC_BITS64; return true; }
    if (sr == B2SR_PLUS_TIMES && in == B2SR_VEC_BITS) { *out = B2SR_VEC_I32; return true; }
    if (sr == B2SR_PLUS_TIMES && in == B2SR_VEC_F32) { *out = B2SR_VEC_F32; return true; }
    if (sr == B2SR_MIN_PLUS && (in == B2SR_VEC_F32 || in == B2SR_VEC_I32)) { *out = in; return true; }
    if (sr == B2SR_MAX_TIMES && in == B2SR_VEC_F32) { *out = B2SR_VEC_F32; return true; }
    return false;
}

static bool has_staged(int k, b2sr_semiring sr, b2sr_vec in) {
    return k <= 16 && in != B2SR_VEC_BITS &&
           (sr == B2SR_PLUS_TIMES || sr == B2SR_MIN_PLUS || sr == B2SR_MAX_TIMES || in == B2SR_VEC_BITS64);
}

static int64_t vec_words(int32_t n, b2sr_vec kind) {
    return kind == B2SR_VEC_BITS ? ceil_div(n, 32) : kind == B2SR_VEC_BITS64 ? 2 * (int64_t)n : n;
}

static b2sr_status run_scheme(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in, b2sr_vec out, const void* x, void* y,
                              cudaStream_t s) {
    if (in == B2SR_VEC_BITS64)
        return spmm64_dispatch(h, static_cast<const uint64_t*>(x), static_cast<uint64_t*>(y), nullptr, 0, s, nullptr);
    return spmv_dispatch(h, sr, in, x, out, y, nullptr, 0, nullptr, s, nullptr);
}

// Mean time of `trials` SpMVs of the scheme on h (after one untimed call).
static b2sr_status time_trials(b2sr_matrix* h, b2sr_semiring sr, b2sr_vec in, b2sr_vec out, const void* x, void* y,
                               int trials, cudaStream_t s, double* us) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    B2SR_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    b2sr_status st = e == cudaSuccess ? B2SR_OK : cuda_fail(e, "cudaEventCreate");
    if (st == B2SR_OK) st = run_scheme(h, sr, in, out, x, y, s);
    if (st == B2SR_OK && (e = cudaEventRecord(e0, s)) != cudaSuccess) st = cuda_fail(e, "cudaEventRecord");
    for (int t = 0; t < trials && st == B2SR_OK; ++t)
        st = run_scheme(h, sr, in, out, x, y, s);
    if (st == B2SR_OK && (e = cudaEventRecord(e1, s)) != cudaSuccess) st = cuda_fail(e, "cudaEventRecord");
    if (st == B2SR_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_fail(e, "cudaEventSynchronize");
    float ms = 0.0f;
    if (st == B2SR_OK && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) st = cuda_fail(e, "elapsed");
    if (st == B2SR_OK) *us = 1000.0 * (double)ms / (double)trials;
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_sample_profile(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                                           const int32_t* sample_host, int64_t nsample, double* est_host,
                                           double* tiles_est_host, void* stream) {
    clear_error();
    if (n < 0 || nnz < 0 || nsample < 0 || (n > 0 && !rowptr) || (nnz > 0 && !colind))
        return fail(B2SR_ERR_INVALID_ARG, "bad sizes or NULL arrays");
    if (nsample > 0 && !sample_host) return fail(B2SR_ERR_INVALID_ARG, "sample_host is NULL");
    if (nsample > (int64_t(1) << 28)) return fail(B2SR_ERR_INVALID_ARG, "nsample above 2^28");
    for (int64_t i = 0; i < nsample; ++i)
        if (sample_host[i] < 0 || sample_host[i] >= n) return fail(B2SR_ERR_INVALID_ARG, "sampled row out of range");
    return sample_profile(n, rowptr, colind, nnz, sample_host, nsample, est_host, tiles_est_host, to_stream(stream));
}

extern "C" b2sr_status b2sr_autotune(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                                     const int32_t* sample_host, int64_t nsample, b2sr_semiring sr, b2sr_vec in_kind,
                                     double keep_ratio, int trials, void* stream, b2sr_handle* out,
                                     b2sr_tune_report_t* rep) {
    clear_error();
    if (!out || !rep) return fail(B2SR_ERR_INVALID_ARG, "out or report is NULL");
    *out = nullptr;
    b2sr_vec out_kind;
    if (!scheme_ok(sr, in_kind, &out_kind)) return fail(B2SR_ERR_INVALID_ARG, "unsupported semiring/vector pair");
    if (trials < 1) return fail(B2SR_ERR_INVALID_ARG, "trials must be >= 1");
    if (keep_ratio > 0.0 && keep_ratio < 1.0) return fail(B2SR_ERR_INVALID_ARG, "keep_ratio must be <= 0 or >= 1");
    cudaStream_t s = to_stream(stream);
    for (int q = 0; q < 4; ++q) {
        rep->tiles[q] = -1;
        rep->trial_us[q][0] = rep->trial_us[q][1] = -1.0;
    }
    rep->tile_dim = 0;
    rep->schedule = B2SR_SCHED_AUTO;
    B2SR_TRY(b2sr_sample_profile(n, rowptr, colind, nnz, sample_host, nsample, rep->est_ratio, rep->est_tiles,
                                 stream));
    const double best_est = *std::min_element(rep->est_ratio, rep->est_ratio + 4);
    DevBuf vb(s);
    const int64_t xw = vec_words(n, in_kind), yw = vec_words(n, out_kind);
    B2SR_TRY(vb.alloc((round_up(xw, 64) + yw + 64) * sizeof(uint32_t)));
    uint32_t* x = vb.as<uint32_t>();
    uint32_t* y = x + round_up(xw, 64);
    if (xw > 0) {
        trial_vector_kernel<<<grid_for(xw), 256, 0, s>>>(x, xw, (int)in_kind);
        B2SR_LAUNCH_CHECK("trial_vector_kernel");
    }
    b2sr_handle best = nullptr;
    double best_us = 0.0;
    for (int q = 0; q < 4; ++q) {
        if (keep_ratio > 0.0 && rep->est_ratio[q] > keep_ratio * best_est) continue;
        b2sr_handle h = nullptr;
        b2sr_status st = b2sr_from_csr(n, rowptr, colind, nnz, kTileDims[q], stream, &h);
        if (st != B2SR_OK) {
            if (best) b2sr_destroy(best);
            return st;
        }
        rep->tiles[q] = h->T;
        int best_sched_here = B2SR_SCHED_AUTO;
        double best_here = -1.0;
        const int nsched = has_staged(kTileDims[q], sr, in_kind) ? 2 : 1;
        for (int v = 0; v < nsched && st == B2SR_OK; ++v) {
            h->schedule = nsched == 1 ? B2SR_SCHED_AUTO : (v == 0 ? B2SR_SCHED_STAGED : B2SR_SCHED_DIRECT);
            double us = 0.0;
            st = time_trials(h, sr, in_kind, out_kind, x, y, trials, s, &us);
            if (st != B2SR_OK) break;
            rep->trial_us[q][v] = us;
            if (best_here < 0.0 || us < best_here) { best_here = us; best_sched_here = h->schedule; }
        }
        if (st != B2SR_OK) {
            b2sr_destroy(h);
            if (best) b2sr_destroy(best);
            return st;
        }
        h->schedule = best_sched_here;
        if (!best || best_here < best_us) {
            if (best) b2sr_destroy(best);
            best = h;
            best_us = best_here;
            rep->tile_dim = kTileDims[q];
            rep->schedule = best_sched_here;
        } else {
            b2sr_destroy(h);
        }
    }
    *out = best;
    return B2SR_OK;
}
