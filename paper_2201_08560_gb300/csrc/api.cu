// Handle-level entry points of the C ABI: validation, sizes, array access and
// release of a B2SR handle (Sec. III-A arrays; sizes as in Sec. III-C).
#include <mutex>

#include "b2sr_internal.cuh"

namespace b2sr {

b2sr_status check_handle(const b2sr_matrix* h) {
    if (!h) return fail(B2SR_ERR_INVALID_ARG, "handle is NULL");
    if (!valid_tile(h->k) || h->n < 0) return fail(B2SR_ERR_INVALID_ARG, "handle is corrupt");
    return B2SR_OK;
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_info(b2sr_handle h, b2sr_info_t* info) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (!info) return fail(B2SR_ERR_INVALID_ARG, "info is NULL");
    info->n = h->n;
    info->tile_dim = h->k;
    info->n_tile_rows = h->ntr;
    info->schedule = h->schedule;
    info->n_tiles = h->T;
    info->nnz = h->nnz;
    info->bytes = 4 * ((int64_t)h->ntr + 1) + 4 * h->T + h->T * tile_bytes(h->k);
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_set_schedule(b2sr_handle h, int schedule) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (schedule < B2SR_SCHED_AUTO || schedule > B2SR_SCHED_DIRECT)
        return fail(B2SR_ERR_INVALID_ARG, "schedule must be B2SR_SCHED_AUTO, _STAGED or _DIRECT");
    h->schedule = schedule;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_arrays(b2sr_handle h, const int32_t** tile_rowptr, const int32_t** tile_colind,
                                   const void** bit_tiles) {
    clear_error();
    B2SR_TRY(check_handle(h));
    if (tile_rowptr) *tile_rowptr = h->rowptr;
    if (tile_colind) *tile_colind = h->colind;
    if (bit_tiles) *bit_tiles = h->tiles;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_export(b2sr_handle h, int32_t* tile_rowptr, int32_t* tile_colind, void* bit_tiles,
                                   void* stream) {
    clear_error();
    B2SR_TRY(check_handle(h));
    cudaStream_t s = to_stream(stream);
    if (tile_rowptr)
        B2SR_CUDA_TRY(cudaMemcpyAsync(tile_rowptr, h->rowptr, ((size_t)h->ntr + 1) * sizeof(int32_t),
                                      cudaMemcpyDeviceToDevice, s));
    if (tile_colind && h->T > 0)
        B2SR_CUDA_TRY(cudaMemcpyAsync(tile_colind, h->colind, (size_t)h->T * sizeof(int32_t),
                                      cudaMemcpyDeviceToDevice, s));
    if (bit_tiles && h->T > 0)
        B2SR_CUDA_TRY(cudaMemcpyAsync(bit_tiles, h->tiles, (size_t)h->T * tile_bytes(h->k),
                                      cudaMemcpyDeviceToDevice, s));
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_destroy(b2sr_handle h) {
    clear_error();
    if (!h) return B2SR_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    // all work that may still read the arrays has to finish first
    cudaError_t e = cudaDeviceSynchronize();
    void* ptrs[] = {h->rowptr, h->colind, h->tiles, h->chunk_row, h->voff, h->outdeg, h->split};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, 0);
    cudaStreamSynchronize(0);
    if (prev != h->device) cudaSetDevice(prev);
    delete static_cast<std::mutex*>(h->mtx);
    delete h;
    if (e != cudaSuccess) return cuda_fail(e, "b2sr_destroy");
    return B2SR_OK;
}
