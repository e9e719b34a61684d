/*
 * b2sr.h -- C ABI of the GB300-native B2SR bit-graph library.
 *
 * Implements the hot path of Bit-GraphBLAS (Chen, Sung, Shen, Tallent,
 * Barker, Li; arXiv 2201.08560): the Bit-Block Compressed Sparse Row (B2SR)
 * storage of a binary adjacency matrix (Sec. III), bit-level SpMV and SpGEMM
 * over it (Sec. IV, Tables 2 and 3) and the GraphBLAS algorithms built on
 * them (Sec. V, Table 4: BFS, SSSP, PageRank, connected components, triangle
 * counting), plus batched multi-source BFS.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns a b2sr_status; 0 is success.  On failure the
 *    calling thread's b2sr_last_error() holds a one-line reason.  No C++
 *    exception crosses this boundary.
 *  - Array pointers are DEVICE pointers (cudaMalloc / PyTorch CUDA tensors on
 *    the current device) unless the parameter name ends in _host.  The caller
 *    owns every input and output buffer and sizes it as documented; a
 *    b2sr_handle owns the B2SR arrays it was built with.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    stream-ordered: a function returns once its kernels are enqueued, except
 *    where it must return a host value (named *_host) or size an allocation;
 *    those synchronise the stream and say so.
 *  - Temporary device memory is taken from the stream-ordered allocator
 *    (cudaMallocAsync) and released on the same stream; failures give
 *    B2SR_ERR_OOM.  A handle is read-only during SpMV/SpGEMM/driver calls, so
 *    one handle may serve several streams at once.
 *  - Vertex ids are int32; n < 2^31; nnz < 2^31.
 *  - Bitsets are LSB-first uint32 words: vertex v is bit v%32 of word v/32.
 *    A bitset over n vertices has ceil(n/32) words; output bits >= n are 0.
 *  - Orientation: entry (i, j) of A is an edge from vertex j to vertex i,
 *    the direction in which y = A x moves values (Sec. V multiplies PageRank
 *    by the column-stochastic A, so column j holds the out-edges of j).  BFS
 *    and SSSP follow edges that way.  For symmetric matrices (undirected
 *    graphs) both orientations coincide.
 *
 * B2SR layout (Sec. III-A, III-B and Table 1)
 * -------------------------------------------
 *  k = tile_dim in {4, 8, 16, 32}; nTileRow = ceil(n/k).
 *  TileRowPtr int32[nTileRow+1]: tiles of tile-row I are [TileRowPtr[I],
 *     TileRowPtr[I+1]).
 *  TileColInd int32[T]: tile column of each non-empty tile, ascending per
 *     tile-row.
 *  BitTiles: k row words per tile, a word being uint8 (k=4, low nibble),
 *     uint8 (k=8), uint16 (k=16) or uint32 (k=32).  Row word r of tile (I,J)
 *     holds matrix row k*I+r; its bit c (LSB = 0) is entry (k*I+r, k*J+c).
 *     Bits outside the n x n matrix are 0.
 *  Storage bytes = 4(nTileRow+1) + 4T + T*k*word_bytes.
 */
#ifndef B2SR_H
#define B2SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    B2SR_OK = 0,
    B2SR_ERR_INVALID_ARG = 1,      /* null pointer, bad size, malformed CSR, bad source */
    B2SR_ERR_UNSUPPORTED_TILE = 2, /* tile_dim not in {4, 8, 16, 32} */
    B2SR_ERR_OOM = 3,              /* device allocation failed */
    B2SR_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed */
    B2SR_ERR_NOT_CONVERGED = 5,    /* an iterative driver hit max_iters */
    B2SR_ERR_ADMISSION_REFUSED = 6,/* reserved: serving admission */
    B2SR_ERR_ABORTED = 7           /* reserved: cancelled work */
} b2sr_status;

typedef struct b2sr_matrix* b2sr_handle;

typedef enum {
    B2SR_BOOL_OR_AND = 0, /* Boolean semiring ({0,1}, OR, AND), Table 4 */
    B2SR_PLUS_TIMES = 1,  /* arithmetic semiring (R, +, x), Table 4 */
    B2SR_MIN_PLUS = 2,    /* tropical min-plus (R u {+inf}, min, +), Table 4 */
    B2SR_MAX_TIMES = 3    /* tropical max-times (R u {-inf}, max, x), Table 4 */
} b2sr_semiring;

typedef enum {
    B2SR_VEC_BITS = 0, /* bitset, ceil(n/32) uint32 words */
    B2SR_VEC_I32 = 1,  /* int32[n] */
    B2SR_VEC_F32 = 2,  /* float[n] */
    B2SR_VEC_BITS64 = 3, /* uint64[n]: 64 Boolean vectors, one bit each per vertex
                            (the b2sr_spmm_bits64 scheme; accepted by b2sr_autotune only) */
    B2SR_VEC_I64 = 4     /* int64[n] (the weighted count of b2sr_spmv_planes) */
} b2sr_vec;

/* SpMV kernel schedule for the value schemes (plus-times on floats, min-plus,
 * b2sr_spmm_bits64, b2sr_spmm_f32x4) at tile_dim <= 16; the Boolean and count schemes and
 * tile_dim 32 have one schedule.  Min and OR results are identical under
 * both; plus-times sums are added in a different fixed order (each schedule
 * bitwise reproducible, both within the fp32 tolerance).  Speed depends on
 * the graph (b2sr_autotune measures it).  The paper stages the dense vector
 * segment of a tile in shared memory (Sec. IV); STAGED is that idea for a
 * gather per set bit, DIRECT reads the vector from global memory. */
typedef enum {
    B2SR_SCHED_AUTO = 0,   /* STAGED where it exists */
    B2SR_SCHED_STAGED = 1, /* set-bit gathers staged in shared memory (cp.async), then reduced */
    B2SR_SCHED_DIRECT = 2  /* each lane walks its tiles and loads x directly */
} b2sr_schedule;

typedef struct {
    int32_t n;           /* vertices (rows = columns) */
    int32_t tile_dim;    /* k */
    int32_t n_tile_rows; /* ceil(n/k) */
    int32_t schedule;    /* b2sr_schedule of the handle */
    int64_t n_tiles;     /* T, non-empty tiles */
    int64_t nnz;         /* set bits = distinct stored entries */
    int64_t bytes;       /* 4(nTileRow+1) + 4T + T*k*word_bytes (Sec. III-C sizes) */
} b2sr_info_t;

/* Thread-local text of the last failure on this thread ("" if none). */
const char* b2sr_last_error(void);

/* Library version string. */
const char* b2sr_version(void);

/* ---------------------------------------------------------------------- */
/* Storage (Sec. III)                                                      */
/* ---------------------------------------------------------------------- */

/* CSR -> B2SR conversion (Sec. III-A "Bit-tile Indexing System", Sec. III-B
 * "Bit Packing"): nTileRow = ceil(n/k); the distinct tile columns of each
 * tile-row give TileRowPtr/TileColInd; every entry (i, j) sets bit j%k of row
 * word i%k of tile (i/k, j/k).
 *   n        vertices, 0 <= n < 2^31
 *   rowptr   device int32[n+1], rowptr[0] = 0, non-decreasing, rowptr[n] = nnz
 *   colind   device int32[nnz], each in [0, n); rows need not be sorted;
 *            repeated entries are OR-ed (the matrix is binary)
 *   tile_dim 4, 8, 16 or 32 (else B2SR_ERR_UNSUPPORTED_TILE)
 *   out      receives a new handle (owned by the caller; b2sr_destroy)
 * The input is validated on the device (B2SR_ERR_INVALID_ARG if malformed).
 * Synchronises `stream` once to learn the tile count. */
b2sr_status b2sr_from_csr(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                          int tile_dim, void* stream, b2sr_handle* out);

/* Many graphs in one B2SR arena: graph g's CSR is placed on the diagonal at
 * rows and columns [base[g], base[g] + n_g), with base[g] a multiple of 32, so
 * that its tiles never share a tile-row or a bitset word with another graph.
 * The result is one block-diagonal matrix on which every SpMV and driver runs
 * all graphs in the same launches (the batching the paper has no counterpart
 * for; Sec. III-A storage applied to the union).
 *   ngraphs   >= 1
 *   n_host    host int32[ngraphs] vertex counts (0 allowed)
 *   rowptrs   host array of ngraphs device int32[n_g+1] pointers
 *   colinds   host array of ngraphs device int32[nnz_g] pointers (ids local)
 *   nnz_host  host int64[ngraphs]
 *   base_host host int64[ngraphs+1] (written): offsets, base[ngraphs] = arena n
 * Fails with B2SR_ERR_INVALID_ARG when the arena reaches 2^31 rows or entries;
 * otherwise as b2sr_from_csr.  Synchronises `stream`. */
b2sr_status b2sr_from_csr_batch(int ngraphs, const int32_t* n_host, const int32_t* const* rowptrs,
                                const int32_t* const* colinds, const int64_t* nnz_host, int tile_dim,
                                void* stream, b2sr_handle* out, int64_t* base_host);

/* B2SR -> CSR (sorted, duplicate-free rows): the inverse of b2sr_from_csr.
 *   rowptr   device int32[n+1] (written)
 *   colind   device int32[nnz] (written) or NULL to query only
 *   nnz_host receives nnz (host int64).  Synchronises `stream`. */
b2sr_status b2sr_to_csr(b2sr_handle h, int32_t* rowptr, int32_t* colind, int64_t* nnz_host,
                        void* stream);

/* Sizes of a handle (host struct). */
b2sr_status b2sr_info(b2sr_handle h, b2sr_info_t* info);

/* Selects the handle's SpMV schedule (b2sr_schedule; the vector staging of
 * Sec. IV or direct loads); B2SR_ERR_INVALID_ARG for another value.  Not synchronised with SpMVs in flight on other host
 * threads; the next SpMV enqueued uses it. */
b2sr_status b2sr_set_schedule(b2sr_handle h, int schedule);

/* Device pointers to the handle's three arrays (owned by the handle; valid
 * until b2sr_destroy).  BitTiles is returned as bytes. */
b2sr_status b2sr_arrays(b2sr_handle h, const int32_t** tile_rowptr, const int32_t** tile_colind,
                        const void** bit_tiles);

/* Copies the three arrays, unpadded, into caller buffers (stream-ordered):
 *   tile_rowptr device int32[nTileRow+1], tile_colind device int32[T],
 *   bit_tiles device bytes[T*k*word_bytes]; any may be NULL to skip it. */
b2sr_status b2sr_export(b2sr_handle h, int32_t* tile_rowptr, int32_t* tile_colind, void* bit_tiles,
                        void* stream);

/* Release a handle (waits for the device to finish with it). NULL is a no-op. */
b2sr_status b2sr_destroy(b2sr_handle h);

/* Strictly lower triangle L of the matrix (entries (i, j) with j < i) as a new
 * B2SR handle with the same tile_dim: the L used by triangle counting
 * (Sec. V, TC).  Synchronises `stream` once. */
b2sr_status b2sr_lower(b2sr_handle h, void* stream, b2sr_handle* out);

/* B2SR of the transpose A^T, as a new handle with the same tile_dim (Sec.
 * III-A: the tile index is transposed by taking TileRowPtr/TileColInd from
 * CSR to CSC order; Sec. III-B: the tiles take the other packing, i.e. each
 * k x k bit tile is transposed).  vxm, y^T = x^T A, is b2sr_spmv on the
 * result; b2sr_sssp_push and b2sr_bfs_diropt take it as their transpose on
 * directed graphs.  Enqueued on `stream`, synchronised before returning (the
 * handle's sizes are read back).  The caller destroys *out.
 * B2SR_ERR_OOM past 2^32 tiles or on allocation failure. */
b2sr_status b2sr_transpose(b2sr_handle h, void* stream, b2sr_handle* out);

/* Reorders per-entry fp32 weights given in CSR order (the CSR that built h,
 * any row order, no repeated entries) into set-bit order: tile by tile, row
 * word by row word, bit by bit.  That is the `weights` layout b2sr_spmv and
 * b2sr_sssp take.  Weighted graphs are outside the paper's binary B2SR (it
 * names short-bit-width weights as future work, Sec. VII); the side array is
 * this library's addition.
 *   w_csr  device float[nnz] (CSR order);  w_bits  device float[nnz] (written) */
b2sr_status b2sr_weights_from_csr(b2sr_handle h, const int32_t* rowptr, const int32_t* colind,
                                  const float* w_csr, float* w_bits, void* stream);

/* ---------------------------------------------------------------------- */
/* SpMV: the BMV schemes of Table 2 over the semirings of Table 4          */
/* ---------------------------------------------------------------------- */

/* y = A (+).(x) x, overwriting y, with an optional output mask applied just
 * before the store (Sec. V, BFS: masked schemes).  Supported combinations:
 *   BOOL_OR_AND, BITS -> BITS  bmv_bin_bin_bin:  y_i = OR_j A_ij AND x_j
 *   PLUS_TIMES,  BITS -> I32   bmv_bin_bin_full: y_i = sum_J popc(A_IJ[r] & x_J)
 *                              (the popc formula of Sec. IV), i.e. the number
 *                              of neighbours j of i with x_j = 1
 *   PLUS_TIMES,  F32  -> F32   bmv_bin_full_full: y_i = sum_{j: A_ij=1} x_j
 *   MIN_PLUS,    F32  -> F32   y_i = min(x_i, min_{j: A_ij=1} x_j + w_ij)
 *                              (Sec. V, SSSP: zeros are +inf off the diagonal
 *                              and 0 on it, so x_i always takes part);
 *                              weights NULL means w = 1
 *   MIN_PLUS,    I32  -> I32   y_i = min(x_i, min_{j: A_ij=1} x_j): every
 *                              weight 0, the CC min step (Sec. V, CC);
 *                              weights must be NULL
 *   MAX_TIMES,   F32  -> F32   y_i = max_{j: A_ij=1} x_j (A_ij = 1 is the
 *                              multiplicative identity), -inf for a row with
 *                              no entries: the local-maximum step of MIS and
 *                              colouring (Table 4, bin-full-full); no
 *                              diagonal term; weights must be NULL
 *   x       device; bitset (ceil(n/32) words), int32[n] or float[n]
 *   y       device; same shapes; must not alias x or mask
 *   mask    device bitset or NULL; if given, y_i is kept where the mask bit
 *           is 1 (mask_complement = 0) or 0 (mask_complement = 1); excluded
 *           outputs get the semiring's additive identity (0 / false / +inf /
 *           INT32_MAX / -inf)
 *   weights device float[nnz] in set-bit order (b2sr_weights_from_csr) or NULL
 * Floating-point sums use a fixed order, so results are bitwise reproducible
 * run to run.  B2SR_ERR_INVALID_ARG for other combinations. */
b2sr_status b2sr_spmv(b2sr_handle h, b2sr_semiring semiring, b2sr_vec in_kind, const void* x,
                      b2sr_vec out_kind, void* y, const uint32_t* mask, int mask_complement,
                      const float* weights, void* stream);

/* Short-bit-width integer weights as bit-planes (Sec. VII: a weighted
 * graph whose weights are small integers is the sum W = sum_p 2^p A_p of
 * binary matrices, each of which B2SR holds).  Plane p of tile t is a k x k
 * bit tile in h's packing (bit (r, c) set iff the entry at row kI+r, column
 * kJ+c has bit p set in its weight), over h's tile index; planes are stored
 * tile by tile, plane by plane: byte offset (t * bits + p) * tile_bytes,
 * tile_bytes = k * word_bytes (4, 8, 32, 128 for k = 4, 8, 16, 32).
 *   rowptr, colind  device; the CSR that built h (any row order, no repeated
 *                   entries)
 *   w_csr    device uint32[nnz], CSR order, each < 2^bits
 *   bits     1..16
 *   planes   device, 4-byte aligned, n_tiles * bits * tile_bytes bytes,
 *            written (zeroed first); owned by the caller
 * B2SR_ERR_INVALID_ARG if an entry is not in h or a weight needs more bits.
 * Synchronises the stream. */
b2sr_status b2sr_planes_from_csr(b2sr_handle h, const int32_t* rowptr, const int32_t* colind,
                                 const uint32_t* w_csr, int bits, void* planes, void* stream);

/* SpMV over bit-plane weights (Sec. VII extension; the bin-bin-full and
 * bin-full-full schemes of Table 2 applied per plane):
 *   BITS -> I64   y_i = sum_J sum_p 2^p popc(P_p,IJ[r] & x_J) = sum_{j: x_j=1} w_ij,
 *                 exact in int64
 *   F32  -> F32   y_i = sum_j w_ij x_j with w_ij = sum_p 2^p (P_p)_ij formed
 *                 exactly per entry; compensated fp32 sums in a fixed order
 *                 (bitwise reproducible)
 *   planes   device, as written by b2sr_planes_from_csr with the same bits
 *   x, y     device; y must not alias x or mask
 *   mask     device bitset or NULL (mask_complement as b2sr_spmv); excluded
 *            outputs are 0
 * A warp per tile-row, a 256-thread block per tile-row of more than 256
 * tiles.  B2SR_ERR_INVALID_ARG for other vector kinds or bits outside 1..16. */
b2sr_status b2sr_spmv_planes(b2sr_handle h, const void* planes, int bits, b2sr_vec in_kind, const void* x,
                             b2sr_vec out_kind, void* y, const uint32_t* mask, int mask_complement,
                             void* stream);

/* Boolean SpMM with 64 frontiers packed per vertex (multi-source BFS step; a
 * batched form of bmv_bin_bin_bin_masked, Table 2, with the complemented
 * visited mask of Sec. V BFS):
 *   Y_i = OR_{j: A_ij=1} X_j, then Y_i &= M_i (complement = 0) or ~M_i (1).
 *   X, Y device uint64[n]; M device uint64[n] or NULL. */
b2sr_status b2sr_spmm_bits64(b2sr_handle h, const uint64_t* X, uint64_t* Y, const uint64_t* M,
                             int complement, void* stream);

/* Plus-times SpMM over a block of four fp32 columns (bmv_bin_full_full of
 * Table 2 on the arithmetic semiring of Table 4, four vectors per pass over
 * the tiles; Sec. V PR batched):
 *   Y[4i+b] = sum_{j: A_ij=1} X[4j+b], b = 0..3, then masked like b2sr_spmv
 *   (masked-out rows get 0).
 *   X, Y device float[4n], vertex-major (the four values of vertex v are
 *   contiguous), 16-byte aligned (else B2SR_ERR_INVALID_ARG); Y must not alias X.
 * Column b of Y is bitwise equal to b2sr_spmv(PLUS_TIMES, F32) on column b
 * of X: each column is summed in the same fixed order. */
b2sr_status b2sr_spmm_f32x4(b2sr_handle h, const float* X, float* Y, const uint32_t* mask,
                            int mask_complement, void* stream);

/* Boolean SpMV that allocates no device memory.  The paper has no
 * counterpart; it exists for callers that cannot allocate device memory when
 * they call in, such as a host whose own allocator already holds the device's
 * free memory, or a service that must not allocate once it is running.
 * Computes exactly what b2sr_spmv computes for BOOL_OR_AND, BITS -> BITS
 * (same x, y, mask and mask_complement meaning), but keeps its scratch (the
 * partial rows of tile-rows that cross chunks) in a fixed 4 MiB array compiled
 * into the library.  It calls no cudaMalloc, cudaFree or allocating routine.
 *  - A device gets its copy of the array when the CUDA runtime loads the
 *    library's SpMV code on it: with lazy module loading (the default since
 *    CUDA 12.2) that is the first SpMV launch or the first call of this
 *    function on that device, and the copy stays until the process exits or
 *    the device is reset.  Make the first call on each device (or any earlier
 *    b2sr_spmv on it) before the caller reserves the device's free memory and
 *    before any stream capture.  That call also looks the copy's address up
 *    (cudaGetSymbolAddress) with the device current; the address is kept for
 *    the process, so do not call this function after cudaDeviceReset.
 *  - h must belong to the current device (else B2SR_ERR_INVALID_ARG): each
 *    device's call uses that device's copy.
 *  - Matrices needing more scratch than the array holds (more than 262,144
 *    chunks at k=8, or 524,288 at k=4/16/32; a chunk is 256 tiles at k=4/8,
 *    128 at k=16, 64 at k=32) are rejected
 *    with B2SR_ERR_INVALID_ARG and a message giving both sizes.
 *  - Every call uses the same array and leaves its contents behind.  Nothing
 *    in it needs clearing (each call writes every value it reads), but calls
 *    that run at the same time on the GPU (other streams, other threads)
 *    overwrite each other's scratch: serialise them. */
b2sr_status b2sr_spmv_bool_noalloc(b2sr_handle h, const uint32_t* x, uint32_t* y, const uint32_t* mask,
                                   int mask_complement, void* stream);

/* ---------------------------------------------------------------------- */
/* SpGEMM: the BMM schemes of Table 3 and the Boolean product              */
/* ---------------------------------------------------------------------- */

/* bmm_bin_bin_sum_masked (Table 3, Listing 2): the sum over the entries (i,j)
 * of M of (A B^T)_ij = |row_i(A) AND row_j(B)|, reduced into one int64 with
 * the reduction fused (Sec. V, TC).  Rows of B are used directly, as
 * Listing 2's popc(r0 & shfl(r1)) does, so triangle counting passes
 * A = B = M = L.  All three handles need the same n and tile_dim.
 *   count  device int64[1] (written, not accumulated). */
b2sr_status b2sr_spgemm_masked_count(b2sr_handle A, b2sr_handle B, b2sr_handle M, int64_t* count,
                                     void* stream);

/* The same masked count (Table 3, bmm_bin_bin_sum_masked) that also reports
 * its integer work, for measurement (no counterpart in the paper): *pairs
 * (device int64[1], written) receives the number of AND-popc operations on
 * one row word each, i.e. over every mask tile (I, J), the bits of M_IJ times
 * the tile-columns K with A_IK and B_JK both stored.  count as above.
 * B2SR_ERR_INVALID_ARG if count or pairs is NULL or the handles disagree. */
b2sr_status b2sr_spgemm_masked_count_work(b2sr_handle A, b2sr_handle B, b2sr_handle M, int64_t* count,
                                          int64_t* pairs, void* stream);

/* Boolean SpGEMM C = A (x) B over OR-AND, output in B2SR with the same
 * tile_dim (not in the paper's Table 3; built from the same tile products):
 * C_IJ[r] = OR_K OR_{m: bit m of A_IK[r]} B_KJ[m].  Synchronises `stream`.
 * B2SR_ERR_OOM for more than 2^32 tile products or 2^31 - 1 result tiles
 * (every handle indexes its tiles with int32). */
b2sr_status b2sr_spgemm_bool(b2sr_handle A, b2sr_handle B, void* stream, b2sr_handle* C);

/* ---------------------------------------------------------------------- */
/* Tile size selection (Sec. III-C, Algorithm 1)                           */
/* ---------------------------------------------------------------------- */

/* Sampling profile (Sec. III-C, Algorithm 1).  Every sampled row i stands for
 * its tile-row i/k; the mean number of distinct tile columns over the sampled
 * tile-rows, times nTileRow, estimates the tile count T_k, and
 *   est[q] = (4(nTileRow+1) + T_k (4 + k word_bytes)) / (4(n+1) + 8 nnz)
 * estimates the B2SR size over the fp32 CSR size, for k = 4, 8, 16, 32
 * (q = 0..3).  Exact (T_k = T) when every row is sampled once and k divides n.
 *   rowptr, colind device CSR (as b2sr_from_csr; rows need not be sorted)
 *   sample_host    host int32[nsample] rows in [0, n), repeats allowed; the
 *                  caller draws them (nsample <= 2^28)
 *   est_host, tiles_est_host host double[4] (either may be NULL)
 * B2SR_ERR_INVALID_ARG for a row out of range or a malformed rowptr at a
 * sampled tile-row.  Synchronises `stream`. */
b2sr_status b2sr_sample_profile(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                                const int32_t* sample_host, int64_t nsample, double* est_host,
                                double* tiles_est_host, void* stream);

typedef struct {
    double est_ratio[4];   /* b2sr_sample_profile estimates, k = 4, 8, 16, 32 */
    double est_tiles[4];
    double trial_us[4][2]; /* mean SpMV time per (k, schedule slot), -1 where not tried;
                              slot 0 = STAGED (or the only schedule), slot 1 = DIRECT */
    int64_t tiles[4];      /* tile count of each converted candidate, -1 if not converted */
    int32_t tile_dim;      /* the chosen k */
    int32_t schedule;      /* the chosen b2sr_schedule */
} b2sr_tune_report_t;

/* Autotuner: the Sec. III-C tile size choice, with the Algorithm 1 estimate as
 * a pre-filter and measured SpMV time as the decision.  k is a candidate if
 * est_ratio[k] <= keep_ratio * min est_ratio (keep_ratio <= 0: every k;
 * 0 < keep_ratio < 1 is B2SR_ERR_INVALID_ARG).  Each candidate is converted
 * and timed over `trials` SpMVs of the (sr, in_kind) scheme on a fixed
 * synthetic vector (BOOL_OR_AND with B2SR_VEC_BITS64: b2sr_spmm_bits64, the
 * multi-source BFS step), under each schedule it has (b2sr_schedule); the fastest
 * handle is returned in *out with that schedule set, the others destroyed.
 * The timings are taken on `stream` while other work may share the device,
 * so the choice is a measurement, not a guarantee.  Synchronises `stream`. */
b2sr_status b2sr_autotune(int32_t n, const int32_t* rowptr, const int32_t* colind, int64_t nnz,
                          const int32_t* sample_host, int64_t nsample, b2sr_semiring sr, b2sr_vec in_kind,
                          double keep_ratio, int trials, void* stream, b2sr_handle* out,
                          b2sr_tune_report_t* report);

/* ---------------------------------------------------------------------- */
/* Graph algorithms (Sec. V)                                               */
/* ---------------------------------------------------------------------- */

/* BFS levels from `src` (Sec. V BFS: Boolean semiring, the visited set as a
 * complemented mask).  levels device int32[n]: 0 at src, -1 if unreachable.
 * At most max_iters levels (<= 0: n); B2SR_ERR_NOT_CONVERGED if exceeded.
 * Synchronises `stream` once per four levels (see b2sr_bfs_sources). */
b2sr_status b2sr_bfs(b2sr_handle h, int32_t src, int32_t* levels, int max_iters, void* stream);

/* BFS from a set of sources, all at level 0 (Sec. V BFS with the first
 * frontier holding every source).  levels[v] is the distance from v to the
 * nearest source, -1 if none reaches it.  On a matrix built by
 * b2sr_from_csr_batch with one source per graph, graph g's levels are
 * levels[base[g] .. base[g] + n_g) and equal a BFS of graph g alone, since
 * no edge joins two graphs: one call runs every graph's BFS at once.
 *   srcs_host host int32[nsrc], nsrc >= 1, each in [0, n), repeats allowed
 *   levels    device int32[n]
 * Level rounds run as a CUDA graph of four gated rounds replayed until a
 * round finds no new vertex: one host synchronisation per four levels.
 * B2SR_ERR_NOT_CONVERGED past max_iters levels (<= 0: n). */
b2sr_status b2sr_bfs_sources(b2sr_handle h, const int32_t* srcs_host, int nsrc, int32_t* levels,
                             int max_iters, void* stream);

/* Direction-optimising BFS (Sec. V BFS; the push/pull switching of Beamer et
 * al., SC 2012).  A level either pulls (the Boolean SpMV of b2sr_bfs over
 * every tile) or pushes (walks only the frontier's tile-rows of A^T and sets
 * unvisited targets with atomic ORs); it starts pushing, pulls once the
 * frontier's out-edges exceed the unexplored edges / 14, and pushes again
 * once the frontier is below n / 24.  The choice is made on the device each
 * level; levels equal b2sr_bfs's bit for bit.
 *   hT  B2SR of A^T (tile-row J lists the out-edges of vertices kJ..kJ+k-1),
 *       NULL for a symmetric matrix (h is its own transpose); same n as h
 * Other arguments as b2sr_bfs; one host synchronisation per four levels. */
b2sr_status b2sr_bfs_diropt(b2sr_handle h, b2sr_handle hT, int32_t src, int32_t* levels, int max_iters,
                            void* stream);

/* Multi-source BFS: up to 64 BFS runs of Sec. V advance together, their
 * frontiers packed as one uint64 per vertex (b2sr_spmm_bits64), or, for at
 * most 32 sources, one uint32 (half the bytes per step; same levels).
 *   srcs_host host int32[nsrc], 1 <= nsrc <= 64
 *   levels    device int32[nsrc * n]: row s holds the levels of srcs_host[s] */
b2sr_status b2sr_bfs_multi(b2sr_handle h, const int32_t* srcs_host, int nsrc, int32_t* levels,
                           int max_iters, void* stream);

/* Single-source shortest paths (Sec. V SSSP): rounds of min-plus SpMV
 * relaxation, d <- min(d, A min.+ d), until no distance changes (the fixed
 * point delta-stepping also reaches).  weights in set-bit order
 * (b2sr_weights_from_csr), non-negative, or NULL for unit weights.
 * dist device float[n]: 0 at src, +inf if unreachable.  Rounds run as a CUDA
 * graph of 16 gated rounds: one host synchronisation per 16 rounds. */
b2sr_status b2sr_sssp(b2sr_handle h, const float* weights, int32_t src, float* dist, int max_iters,
                      void* stream);

/* SSSP by frontier-driven push (Sec. V SSSP; the same fixed point as
 * b2sr_sssp, reached by relaxing only the out-edges of the vertices whose
 * distance dropped in the previous round).  It reads the transpose:
 *   hT         B2SR of A^T (tile-row J lists the out-edges of vertices
 *              kJ .. kJ+k-1); for a symmetric matrix, the matrix's own handle
 *   weights_t  fp32 weights in set-bit order of hT (b2sr_weights_from_csr on
 *              the transposed CSR; for symmetric weights, those of the
 *              matrix), non-negative, or NULL for unit weights
 *   dist       device float[n]: 0 at src, +inf if unreachable
 *   delta      > 0: the buckets of delta-stepping (Sec. V names it): a round
 *              relaxes only active vertices closer than a threshold, which
 *              starts at delta; vertices at or past it wait in a far set
 *              that no round touches until the near set is empty, when the
 *              threshold grows by delta (to the least waiting distance plus
 *              delta, if that is further) and the far set becomes active;
 *              <= 0: every active vertex every round (Bellman-Ford frontier)
 * A round touches only the active tile-rows.  Distances are updated with
 * integer atomicMin on the float bits; the order of updates and delta change
 * the number of rounds, never the result (bit-exact).  Rounds run as a CUDA
 * graph of 32 gated rounds: one host synchronisation per 32 rounds, and one
 * more at the end to read the round count.
 * B2SR_ERR_NOT_CONVERGED past max_iters rounds (<= 0: n, or 4n + 4 with
 * delta > 0). */
b2sr_status b2sr_sssp_push(b2sr_handle hT, const float* weights_t, int32_t src, float* dist, float delta,
                           int max_iters, void* stream);

/* The rounds (relaxation rounds, counting those that only moved the far set
 * in) run by the most recent successful b2sr_sssp_push on the calling host
 * thread, and, if active_tile_rows is not NULL, the active tile-rows those
 * rounds took summed over the rounds; 0 before any call and after a failed
 * one.  Host-only; a measurement aid with no counterpart in the paper (Sec. V
 * reports SSSP times only). */
b2sr_status b2sr_sssp_push_rounds(int64_t* rounds, int64_t* active_tile_rows);

/* PageRank (Sec. V PR): x^0 = 1/n, then `iters` steps of
 *   x_i <- (1-d) t_i + d * sum_{j: A_ij=1} x_j / outdeg(j)
 * with outdeg(j) the number of ones in column j (the column-stochastic
 * matrix); vertices without out-edges pass nothing on.
 *   teleport device float[n] or NULL for uniform 1/n;  pr device float[n]. */
b2sr_status b2sr_pagerank(b2sr_handle h, float d, int iters, const float* teleport, float* pr,
                          void* stream);

/* Connected components (Sec. V CC, FastSV hooking and shortcutting with the
 * min step of b2sr_spmv).  labels device int32[n]: the smallest vertex id in
 * each vertex's component.  Undirected (symmetric) matrices. */
b2sr_status b2sr_cc(b2sr_handle h, int32_t* labels, int max_iters, void* stream);

/* Maximal independent set (the MIS row of Table 4: the local-maximum test on
 * the max-times semiring, the removal of neighbours on the Boolean semiring;
 * the paper names the operation without an algorithm, and this is Luby's
 * synchronous rounds with fixed priorities).  Each vertex carries the key
 * (priority, id), compared by priority and then by the larger id.  A round
 * takes every undecided vertex whose key is the largest among itself and its
 * undecided neighbours into the set and decides it and its neighbours.  The
 * result is the greedy set in decreasing key order: v is in it iff no
 * neighbour with a larger key is.
 *   priority device float[n], not NaN (+0 and -0 are equal)
 *   in_set   device int32[n]: 1 for members, 0 otherwise
 * Symmetric matrices (undirected graphs); self-loops are ignored.  Rounds run
 * as a CUDA graph of 4 gated rounds.  B2SR_ERR_INVALID_ARG for a NaN
 * priority; B2SR_ERR_NOT_CONVERGED if vertices are still undecided after
 * max_iters rounds (<= 0: n), checked every 4 rounds. */
b2sr_status b2sr_mis(b2sr_handle h, const float* priority, int32_t* in_set, int max_iters, void* stream);

/* How b2sr_color computes the colours (the result is the same). */
typedef enum {
    B2SR_COLOR_AUTO = 0,      /* the push form */
    B2SR_COLOR_MAX_TIMES = 1, /* rounds of max-times SpMVs (Table 4, GC) */
    B2SR_COLOR_PUSH = 2       /* counters pushed along the frontier's rows */
} b2sr_color_method;

/* Graph colouring by priority levels (the GC row of Table 4; no algorithm in
 * the paper).  With the keys of b2sr_mis, colour(v) = 0 if no neighbour has a
 * larger key, else 1 + the largest colour among the neighbours that do; each
 * colour class is an independent set.  MAX_TIMES: round r gives colour r to
 * every uncoloured vertex whose key is the largest among itself and its
 * uncoloured neighbours (a max-times SpMV per round, 8 rounds per CUDA-graph
 * replay).  PUSH: cnt[v] = neighbours with a larger key, counted in one pass;
 * the vertices coloured r push along their rows and a vertex whose count
 * reaches 0 takes colour r + 1 (the levels of a topological sort; each edge
 * read twice in all, 16 rounds per replay).
 *   priority device float[n], not NaN
 *   colors   device int32[n]
 * Symmetric matrices; self-loops are ignored.  B2SR_ERR_INVALID_ARG for a NaN
 * priority or an unknown method; B2SR_ERR_NOT_CONVERGED if vertices are still
 * uncoloured after max_iters rounds (<= 0: n), checked at each replay. */
b2sr_status b2sr_color(b2sr_handle h, const float* priority, int32_t* colors, b2sr_color_method method,
                       int max_iters, void* stream);

/* Triangle count (Sec. V TC): sum(L .* (L L^T)) for L = b2sr_lower(h), by
 * b2sr_spgemm_masked_count.  Symmetric matrices.  count device int64[1]. */
b2sr_status b2sr_tc(b2sr_handle h, int64_t* count, void* stream);

/* ---------------------------------------------------------------------- */
/* Measurement support (no counterpart in the paper)                       */
/* ---------------------------------------------------------------------- */

/* Number of kernels the library has launched in this process so far (no
 * counterpart in the paper). */
int64_t b2sr_launch_count(void);

/* Turns CUDA-event timing of the SpMV chunk kernels (no counterpart in the
 * paper) on (1) or off (0).  While
 * on, every such launch is bracketed by two events on its own stream and
 * recorded under its family: "spmv_bool", "spmv_count", "spmv_plus",
 * "spmv_minplus", "spmv_min_i32", "spmv_max", "spmv_maxkey", "spmm_or64",
 * "spmm_or32" (the batched BFS with at most 32 sources), "spmm_plus4" or
 * "spgemm_masked" (the masked-count SpGEMM kernel; its bytes are the three
 * matrices' arrays). */
void b2sr_timing_enable(int on);

/* Timing read-out (no counterpart in the paper).
 * Sum over the recorded launches of `family`: device milliseconds, launch
 * count and algorithmic bytes (the three B2SR arrays plus each vector read or
 * written once).  Waits for the recorded events. */
b2sr_status b2sr_timing_read(const char* family, double* total_ms, int64_t* launches, double* bytes);

/* Drops all recorded launches (no counterpart in the paper). */
b2sr_status b2sr_timing_reset(void);

/* ---------------------------------------------------------------------- */
/* Query serving (no counterpart in the paper: a request loop around the   */
/* Sec. V BFS and PR drivers)                                              */
/* ---------------------------------------------------------------------- */

typedef struct b2sr_server* b2sr_server_t;

typedef struct {
    int64_t submitted, completed, failed, refused; /* since the last reset */
    int64_t steps;          /* batched device steps (one BFS level and one PR iteration per busy slot) */
    double p50_us, p99_us;  /* submit-to-done latency, nearest-rank percentiles */
    double mean_us, max_us;
    double wall_s;          /* first submission to last completion */
    double queries_per_s;   /* completed / wall_s */
    int64_t bytes_in_use;   /* resident graphs plus batch state */
    int64_t budget;
} b2sr_server_stats_t;

/* A query server on the current device, not in the paper (the Sec. V
 * drivers run one query per call).  It keeps graphs resident and batches
 * queries continuously: BFS queries on one graph share a 64-lane bit-SpMM
 * (b2sr_spmm_bits64) and join at a level boundary; PageRank queries share
 * four-column blocks (b2sr_spmm_f32x4) and join at an iteration boundary.  A
 * worker thread drives every graph on its own stream, so different graphs'
 * steps overlap on the device.
 *   budget_bytes   device memory for resident graphs and batch state
 *   max_bfs_lanes  1..64 concurrent BFS queries per graph
 *   max_pr_blocks  four-column PageRank blocks per graph (0: no PageRank)
 * A result is the same alone and in any mix: levels bit-exact; PageRank
 * bitwise equal to b2sr_pagerank with the query's teleport vector. */
b2sr_status b2sr_server_create(int64_t budget_bytes, int max_bfs_lanes, int max_pr_blocks,
                               b2sr_server_t* out);

/* Registers a graph (no counterpart in the paper).  The server borrows the
 * handle: it must stay alive until b2sr_server_destroy.  Its bytes (and its
 * out-degree array, built here) count against the budget;
 * B2SR_ERR_ADMISSION_REFUSED if they do not fit.  Synchronises once. */
b2sr_status b2sr_server_add_graph(b2sr_server_t s, b2sr_handle h, int32_t* graph_id);

/* Budget accounting of a registered graph (no counterpart in the paper):
 * its resident bytes (B2SR arrays with padding, out-degrees), the working
 * memory of its 64-lane BFS batch and of one four-column PageRank block.
 * Any pointer may be NULL. */
b2sr_status b2sr_server_graph_bytes(b2sr_server_t s, int32_t graph, int64_t* resident, int64_t* bfs_batch,
                                    int64_t* pr_block);

/* Submits a BFS query (Sec. V BFS, levels as b2sr_bfs; no counterpart in the
 * paper for the queueing).  levels: device int32[n], written by the server;
 * the caller must not touch it until the query is done.  Returns at once
 * with *query_id.  B2SR_ERR_ADMISSION_REFUSED if the graph's BFS batch can
 * never fit the budget beside the resident graphs. */
b2sr_status b2sr_server_submit_bfs(b2sr_server_t s, int32_t graph, int32_t src, int32_t* levels,
                                   int64_t* query_id);

/* Submits a PageRank query (Sec. V PR, as b2sr_pagerank with damping d and
 * `iters` iterations; no counterpart in the paper for the queueing).
 * src < 0: uniform teleport 1/n; else all teleport mass on src (personalised
 * PageRank).  pr: device float[n], written by the server. */
b2sr_status b2sr_server_submit_pagerank(b2sr_server_t s, int32_t graph, int32_t src, float d, int iters,
                                        float* pr, int64_t* query_id);

/* Waits up to timeout_s seconds (<= 0: just polls) for a query (no
 * counterpart in the paper).  *done = 1 once its output is complete on the
 * device; *latency_us then holds submit-to-done time (may be NULL).  Returns
 * the query's failure status if it failed. */
b2sr_status b2sr_server_wait(b2sr_server_t s, int64_t query_id, double timeout_s, int* done,
                             double* latency_us);

/* Waits until every submitted query is done (no counterpart in the paper);
 * B2SR_ERR_NOT_CONVERGED at the timeout (<= 0: none). */
b2sr_status b2sr_server_drain(b2sr_server_t s, double timeout_s);

/* Counters and latency percentiles (no counterpart in the paper). */
b2sr_status b2sr_server_stats(b2sr_server_t s, b2sr_server_stats_t* stats);

/* Clears the counters and latencies of b2sr_server_stats (no counterpart in the paper). */
b2sr_status b2sr_server_reset_stats(b2sr_server_t s);

/* Stops the worker after the steps in flight, fails the queries not done with
 * B2SR_ERR_ABORTED and frees the server (no counterpart in the paper).  The
 * graphs stay with the caller.  NULL is a no-op. */
b2sr_status b2sr_server_destroy(b2sr_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* B2SR_H */
