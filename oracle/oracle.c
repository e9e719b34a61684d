/*
 * CPU oracle for the B2SR bit-graph hot path (Bit-GraphBLAS, arXiv 2201.08560).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * itself never calls it and shares no code, header or table with it.
 *
 * Conventions (the readings of the paper that the oracle fixes):
 *   - A binary n x n matrix is given as CSR (int32 rowptr[n+1], colind[nnz]).
 *     Functions marked "canonical" need every row sorted and duplicate-free;
 *     orc_csr_canonicalize() produces that form (duplicates are OR-ed, i.e.
 *     a repeated entry is the same single 1 of the binary matrix).
 *   - Bitsets are LSB-first uint32 words: element v is bit (v % 32) of word
 *     v / 32; bits >= n are zero on output.
 *   - B2SR (Sec. III-A, Table 1): nTileRow = ceil(n / k); TileRowPtr has
 *     nTileRow + 1 int32 entries; TileColInd one int32 per non-empty tile,
 *     ascending within a tile-row; BitTiles holds k row words per tile, each
 *     word 1, 1, 2 or 4 bytes for k = 4, 8, 16, 32 (k = 4 uses the low nibble
 *     of a byte).  Row word r of tile (I, J) holds matrix row k*I + r, and its
 *     bit c (LSB = 0) is the entry at column k*J + c.  Padding bits are 0.
 *   - Semiring outputs are overwritten; an output that a mask excludes gets
 *     the semiring's additive identity (false, 0, +inf / INT32_MAX).
 *   - Floating point accumulates in double (fp64).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* helpers                                                                    */
/* ------------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static int bit_get(const uint32_t* bits, int64_t v) {
    return (int)((bits[v >> 5] >> (v & 31)) & 1u);
}

static void bit_set(uint32_t* bits, int64_t v) {
    bits[v >> 5] |= (1u << (v & 31));
}

/* Host threads for the row loops below (the CPU baseline is timed on one
 * thread and on all of them).  Each row's value is computed by one thread in
 * the same order either way, so the results do not depend on the count;
 * rows are dealt in blocks of ROW_BLOCK (a multiple of 32, so a bitset word
 * is written by one thread).  Without OpenMP everything runs on one thread. */
#define ROW_BLOCK 1024

int orc_set_threads(int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* mask_mode: 0 = no mask, 1 = keep where mask bit set, 2 = keep where clear */
static int mask_allows(const uint32_t* mask, int mask_mode, int64_t v) {
    if (mask_mode == 0 || mask == NULL) return 1;
    int b = bit_get(mask, v);
    return mask_mode == 1 ? b : !b;
}

static int word_bytes(int k) {
    switch (k) {
        case 4: return 1;
        case 8: return 1;
        case 16: return 2;
        case 32: return 4;
        default: return 0;
    }
}

int orc_csr_validate(int32_t n, const int32_t* rowptr, const int32_t* colind) {
    if (n < 0 || rowptr[0] != 0) return ORC_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return ORC_EINVAL;
    for (int64_t e = 0; e < rowptr[n]; ++e)
        if (colind[e] < 0 || colind[e] >= n) return ORC_EINVAL;
    return ORC_OK;
}

/* Sort every row and drop repeated entries.  Returns the new nnz, or < 0. */
int64_t orc_csr_canonicalize(int32_t n, const int32_t* rowptr, const int32_t* colind,
                             int32_t* out_rowptr, int32_t* out_colind) {
    if (orc_csr_validate(n, rowptr, colind) != ORC_OK) return ORC_EINVAL;
    int64_t w = 0;
    out_rowptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t s = rowptr[i], e = rowptr[i + 1];
        int64_t start = w;
        for (int64_t p = s; p < e; ++p) out_colind[w++] = colind[p];
        qsort(out_colind + start, (size_t)(w - start), sizeof(int32_t), cmp_i32);
        int64_t u = start;
        for (int64_t p = start; p < w; ++p)
            if (p == start || out_colind[p] != out_colind[p - 1]) out_colind[u++] = out_colind[p];
        w = u;
        out_rowptr[i + 1] = (int32_t)w;
    }
    return w;
}

/* ------------------------------------------------------------------------ */
/* B2SR construction and decoding (Sec. III-A, III-B, Table 1)                */
/* ------------------------------------------------------------------------ */

/* Distinct tile columns of tile-row I, sorted, written to buf; returns count. */
static int64_t tile_row_columns(int32_t n, const int32_t* rowptr, const int32_t* colind, int k,
                                int64_t I, int32_t* buf) {
    int64_t r0 = I * k, r1 = r0 + k < n ? r0 + k : n;
    int64_t m = 0;
    for (int64_t e = rowptr[r0]; e < rowptr[r1]; ++e) buf[m++] = colind[e] / k;
    qsort(buf, (size_t)m, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t p = 0; p < m; ++p)
        if (p == 0 || buf[p] != buf[p - 1]) buf[u++] = buf[p];
    return u;
}

/* Phase 1: TileRowPtr (nTileRow + 1 entries).  Returns the number of non-empty
 * tiles T, or < 0 on invalid input. */
int64_t orc_b2sr_rowptr(int32_t n, const int32_t* rowptr, const int32_t* colind, int k,
                        int32_t* tile_rowptr) {
    if (word_bytes(k) == 0) return ORC_EINVAL;
    if (orc_csr_validate(n, rowptr, colind) != ORC_OK) return ORC_EINVAL;
    int64_t ntr = ((int64_t)n + k - 1) / k;
    int64_t maxm = 0;
    for (int64_t I = 0; I < ntr; ++I) {
        int64_t r0 = I * k, r1 = r0 + k < n ? r0 + k : n;
        int64_t m = rowptr[r1] - rowptr[r0];
        if (m > maxm) maxm = m;
    }
    int32_t* buf = (int32_t*)malloc((size_t)(maxm > 0 ? maxm : 1) * sizeof(int32_t));
    if (!buf) return ORC_ENOMEM;
    int64_t T = 0;
    tile_rowptr[0] = 0;
    for (int64_t I = 0; I < ntr; ++I) {
        T += tile_row_columns(n, rowptr, colind, k, I, buf);
        tile_rowptr[I + 1] = (int32_t)T;
    }
    free(buf);
    return T;
}

/* Phase 2: TileColInd and BitTiles (T * k words of word_bytes(k) bytes each). */
int orc_b2sr_fill(int32_t n, const int32_t* rowptr, const int32_t* colind, int k,
                  const int32_t* tile_rowptr, int32_t* tile_colind, uint8_t* tiles) {
    int wb = word_bytes(k);
    if (wb == 0) return ORC_EINVAL;
    int64_t ntr = ((int64_t)n + k - 1) / k;
    int64_t T = tile_rowptr[ntr];
    memset(tiles, 0, (size_t)(T * k * wb));
    int64_t maxm = 0;
    for (int64_t I = 0; I < ntr; ++I) {
        int64_t r0 = I * k, r1 = r0 + k < n ? r0 + k : n;
        if (rowptr[r1] - rowptr[r0] > maxm) maxm = rowptr[r1] - rowptr[r0];
    }
    int32_t* buf = (int32_t*)malloc((size_t)(maxm > 0 ? maxm : 1) * sizeof(int32_t));
    if (!buf) return ORC_ENOMEM;
    for (int64_t I = 0; I < ntr; ++I) {
        int64_t t0 = tile_rowptr[I];
        int64_t cnt = tile_row_columns(n, rowptr, colind, k, I, buf);
        if (cnt != tile_rowptr[I + 1] - t0) { free(buf); return ORC_EINVAL; }
        memcpy(tile_colind + t0, buf, (size_t)cnt * sizeof(int32_t));
        int64_t r0 = I * k, r1 = r0 + k < n ? r0 + k : n;
        for (int64_t row = r0; row < r1; ++row) {
            for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) {
                int32_t J = colind[e] / k;
                /* position of J in this tile-row's sorted column list */
                int64_t lo = t0, hi = t0 + cnt;
                while (lo < hi) {
                    int64_t mid = (lo + hi) / 2;
                    if (tile_colind[mid] < J) lo = mid + 1; else hi = mid;
                }
                int64_t r = row - r0, c = colind[e] % k;
                uint8_t* word = tiles + (lo * k + r) * wb;
                word[c >> 3] |= (uint8_t)(1u << (c & 7)); /* little-endian word, bit c */
            }
        }
    }
    free(buf);
    return ORC_OK;
}

/* Bytes of the three B2SR arrays: 4(nTileRow+1) + 4T + T*k*word_bytes(k). */
int64_t orc_b2sr_bytes(int32_t n, int k, int64_t T) {
    int64_t ntr = ((int64_t)n + k - 1) / k;
    return 4 * (ntr + 1) + 4 * T + T * k * word_bytes(k);
}

/* Decode B2SR back to a canonical CSR.  out_colind may be NULL to count only.
 * Returns nnz. */
int64_t orc_b2sr_to_csr(int32_t n, int k, const int32_t* tile_rowptr, const int32_t* tile_colind,
                        const uint8_t* tiles, int32_t* out_rowptr, int32_t* out_colind) {
    int wb = word_bytes(k);
    if (wb == 0) return ORC_EINVAL;
    int64_t nnz = 0;
    out_rowptr[0] = 0;
    for (int64_t row = 0; row < n; ++row) {
        int64_t I = row / k, r = row % k;
        for (int64_t t = tile_rowptr[I]; t < tile_rowptr[I + 1]; ++t) {
            const uint8_t* word = tiles + (t * k + r) * wb;
            for (int c = 0; c < k; ++c) {
                if ((word[c >> 3] >> (c & 7)) & 1u) {
                    if (out_colind) out_colind[nnz] = (int32_t)(tile_colind[t] * k + c);
                    ++nnz;
                }
            }
        }
        out_rowptr[row + 1] = (int32_t)nnz;
    }
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* SpMV over the semirings of Table 4 (Table 2 schemes), on canonical CSR     */
/* ------------------------------------------------------------------------ */

/* Boolean OR-AND, bit in / bit out (bmv_bin_bin_bin[_masked], Table 2):
 * y_i = OR_{j in row i} x_j, then AND with mask (mode 1) or its complement
 * (mode 2), applied just before the store (Sec. V, BFS). */
void orc_spmv_bool(int32_t n, const int32_t* rowptr, const int32_t* colind, const uint32_t* x,
                   uint32_t* y, const uint32_t* mask, int mask_mode) {
    memset(y, 0, (size_t)((n + 31) / 32) * sizeof(uint32_t));
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        int hit = 0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) hit |= bit_get(x, colind[e]);
        if (hit && mask_allows(mask, mask_mode, i)) bit_set(y, i);
    }
}

/* Arithmetic (plus-times) with a 1-bit vector, full output (bmv_bin_bin_full,
 * Table 2 and the popc formula of Sec. IV): y_i = |{j in row i : x_j = 1}|. */
void orc_spmv_count(int32_t n, const int32_t* rowptr, const int32_t* colind, const uint32_t* x,
                    int32_t* y, const uint32_t* mask, int mask_mode) {
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = 0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) c += bit_get(x, colind[e]);
        y[i] = mask_allows(mask, mask_mode, i) ? c : 0;
    }
}

/* Arithmetic (plus-times) with a full-precision vector (bmv_bin_full_full):
 * y_i = sum_{j in row i} x_j, summed in fp64 in CSR order. */
void orc_spmv_plus(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* x,
                   double* y, const uint32_t* mask, int mask_mode) {
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += x[colind[e]];
        y[i] = mask_allows(mask, mask_mode, i) ? s : 0.0;
    }
}

/* Tropical min-plus (bmv_bin_full_full with relaxation, Sec. V SSSP):
 * y_i = min(x_i, min_{j in row i} (x_j + w_ij)).  The matrix's zeros are +inf
 * except on the diagonal, where they are 0, so x_i always takes part.
 * w == NULL means every edge weight is 1; otherwise w is in CSR order. */
void orc_spmv_minplus(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* x,
                      const float* w, double* y, const uint32_t* mask, int mask_mode) {
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        double m = x[i];
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            double c = x[colind[e]] + (w ? (double)w[e] : 1.0);
            if (c < m) m = c;
        }
        y[i] = mask_allows(mask, mask_mode, i) ? m : INFINITY;
    }
}

/* Min-plus with every weight 0 on int32 labels (the CC min step, Sec. V CC):
 * y_i = min(x_i, min_{j in row i} x_j). */
void orc_spmv_min_i32(int32_t n, const int32_t* rowptr, const int32_t* colind, const int32_t* x,
                      int32_t* y, const uint32_t* mask, int mask_mode) {
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        int32_t m = x[i];
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (x[colind[e]] < m) m = x[colind[e]];
        y[i] = mask_allows(mask, mask_mode, i) ? m : INT32_MAX;
    }
}

/* Max-times over fp64 values (Table 4's tropical max-times; with a binary A
 * every product is x_j):  y_i = max_{j in row i} x_j, -inf for an empty row
 * or a masked-out output. */
void orc_spmv_max(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* x, double* y,
                  const uint32_t* mask, int mask_mode) {
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        double m = -INFINITY;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (x[colind[e]] > m) m = x[colind[e]];
        y[i] = mask_allows(mask, mask_mode, i) ? m : -INFINITY;
    }
}

/* Boolean SpMM with 64 frontiers packed per vertex (multi-source BFS step):
 * Y_i = OR_{j in row i} X_j, then AND with M_i (mode 1) or ~M_i (mode 2). */
void orc_spmm_or64(int32_t n, const int32_t* rowptr, const int32_t* colind, const uint64_t* X,
                   uint64_t* Y, const uint64_t* M, int mask_mode) {
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t acc = 0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) acc |= X[colind[e]];
        if (M && mask_mode == 1) acc &= M[i];
        if (M && mask_mode == 2) acc &= ~M[i];
        Y[i] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Short-bit-width weights as bit-planes (Sec. VII: an integer weight matrix  */
/* W = sum_p 2^p A_p, each A_p binary)                                        */
/* ------------------------------------------------------------------------ */

/* Bit-planes of integer weights w (CSR order, each < 2^bits) over the tile
 * index of the pattern's B2SR (tile_rowptr, tile_colind as built by
 * orc_b2sr_fill): plane p of tile t holds bit (r, c) iff the entry at row
 * kI+r, column kJ+c has bit p set in its weight.  Layout: tile by tile,
 * plane by plane, k words of word_bytes(k) each.  Duplicate entries OR. */
int orc_b2sr_planes(int32_t n, const int32_t* rowptr, const int32_t* colind, const uint32_t* w, int bits, int k,
                    const int32_t* tile_rowptr, const int32_t* tile_colind, uint8_t* planes) {
    int wb = word_bytes(k);
    if (wb == 0 || bits < 1 || bits > 16) return ORC_EINVAL;
    int64_t ntr = ((int64_t)n + k - 1) / k;
    int64_t T = tile_rowptr[ntr];
    int64_t plane_bytes = (int64_t)k * wb;
    memset(planes, 0, (size_t)(T * bits * plane_bytes));
    for (int64_t row = 0; row < n; ++row) {
        int64_t I = row / k, t0 = tile_rowptr[I], t1 = tile_rowptr[I + 1];
        for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) {
            if (w[e] >> bits) return ORC_EINVAL;
            int32_t J = colind[e] / k;
            int64_t lo = t0, hi = t1;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (tile_colind[mid] < J) lo = mid + 1; else hi = mid;
            }
            if (lo == t1 || tile_colind[lo] != J) return ORC_EINVAL;
            int64_t r = row % k, c = colind[e] % k;
            for (int p = 0; p < bits; ++p)
                if ((w[e] >> p) & 1u) {
                    uint8_t* word = planes + ((lo * bits + p) * k + r) * wb;
                    word[c >> 3] |= (uint8_t)(1u << (c & 7));
                }
        }
    }
    return ORC_OK;
}

/* Weighted count (bmv_bin_bin_full over W): y_i = sum_{j in row i, x_j = 1}
 * w_ij in int64; masked-out rows 0. */
void orc_spmv_wcount(int32_t n, const int32_t* rowptr, const int32_t* colind, const uint32_t* w,
                     const uint32_t* x, int64_t* y, const uint32_t* mask, int mask_mode) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t s = 0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (bit_get(x, colind[e])) s += w[e];
        y[i] = mask_allows(mask, mask_mode, i) ? s : 0;
    }
}

/* Weighted plus-times (bmv_bin_full_full over W): y_i = sum_{j in row i}
 * w_ij x_j in fp64, CSR order; masked-out rows 0. */
void orc_spmv_wplus(int32_t n, const int32_t* rowptr, const int32_t* colind, const uint32_t* w,
                    const double* x, double* y, const uint32_t* mask, int mask_mode) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += (double)w[e] * x[colind[e]];
        y[i] = mask_allows(mask, mask_mode, i) ? s : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* SpGEMM (Table 3 and the Boolean product)                                   */
/* ------------------------------------------------------------------------ */

static int64_t sorted_intersection(const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* Masked sum (bmm_bin_bin_sum_masked, Table 3): sum over the entries (i, j)
 * of M of (A B^T)_ij = |row_i(A) intersect row_j(B)|.  All three canonical. */
int64_t orc_masked_count(int32_t n, const int32_t* a_rowptr, const int32_t* a_colind,
                         const int32_t* b_rowptr, const int32_t* b_colind,
                         const int32_t* m_rowptr, const int32_t* m_colind) {
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = m_rowptr[i]; e < m_rowptr[i + 1]; ++e) {
            int64_t j = m_colind[e];
            total += sorted_intersection(a_colind + a_rowptr[i], a_rowptr[i + 1] - a_rowptr[i],
                                         b_colind + b_rowptr[j], b_rowptr[j + 1] - b_rowptr[j]);
        }
    return total;
}

/* Triangle counting (Sec. V TC): with L the strictly lower triangle,
 * TC = sum(L .* (L L^T)) = sum over edges (i, j), j < i, of
 * |{u < j : u in N(i)} intersect {u < j : u in N(j)}|.  Canonical symmetric input. */
int64_t orc_triangle_count(int32_t n, const int32_t* rowptr, const int32_t* colind) {
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* ri = colind + rowptr[i];
        int64_t li = 0;
        while (li < rowptr[i + 1] - rowptr[i] && ri[li] < i) ++li; /* |N_<(i)| */
        for (int64_t p = 0; p < li; ++p) {
            int64_t j = ri[p];
            const int32_t* rj = colind + rowptr[j];
            int64_t lj = 0;
            while (lj < rowptr[j + 1] - rowptr[j] && rj[lj] < j) ++lj;
            total += sorted_intersection(ri, li, rj, lj);
        }
    }
    return total;
}

/* Boolean SpGEMM C = A (x) B over OR-AND, by Gustavson's row merge.
 * Phase 1 (c_colind == NULL): fills c_rowptr, returns nnz(C).
 * Phase 2: also writes the sorted column indices.  Canonical inputs. */
int64_t orc_spgemm_bool(int32_t n, const int32_t* a_rowptr, const int32_t* a_colind,
                        const int32_t* b_rowptr, const int32_t* b_colind,
                        int32_t* c_rowptr, int32_t* c_colind) {
    int32_t* marker = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* row = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!marker || !row) { free(marker); free(row); return ORC_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) marker[v] = -1;
    int64_t nnz = 0;
    c_rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t m = 0;
        for (int64_t e = a_rowptr[i]; e < a_rowptr[i + 1]; ++e) {
            int64_t kk = a_colind[e];
            for (int64_t f = b_rowptr[kk]; f < b_rowptr[kk + 1]; ++f) {
                int32_t j = b_colind[f];
                if (marker[j] != (int32_t)i) { marker[j] = (int32_t)i; row[m++] = j; }
            }
        }
        qsort(row, (size_t)m, sizeof(int32_t), cmp_i32);
        if (c_colind) memcpy(c_colind + nnz, row, (size_t)m * sizeof(int32_t));
        nnz += m;
        c_rowptr[i + 1] = (int32_t)nnz;
    }
    free(marker);
    free(row);
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* Graph algorithms (Sec. V)                                                  */
/* ------------------------------------------------------------------------ */

/* Orientation: entry (i, j) of A is an edge from j to i, the direction in
 * which y = A x moves values (Sec. V PR multiplies by the column-stochastic A,
 * so column j holds the out-edges of j).  BFS and SSSP follow edges that way;
 * for symmetric matrices either orientation gives the same result.  The
 * out-edges of every vertex are the transpose of the CSR, built here. */
static int transpose_csr(int32_t n, const int32_t* rowptr, const int32_t* colind, const float* w,
                         int32_t** out_ptr, int32_t** out_ind, float** out_w) {
    int64_t nnz = rowptr[n];
    int32_t* tp = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t* ti = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    float* tw = w ? (float*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(float)) : NULL;
    int32_t* fill = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!tp || !ti || (w && !tw) || !fill) { free(tp); free(ti); free(tw); free(fill); return ORC_ENOMEM; }
    for (int64_t e = 0; e < nnz; ++e) tp[colind[e] + 1] += 1;
    for (int32_t j = 0; j < n; ++j) tp[j + 1] += tp[j];
    for (int32_t j = 0; j < n; ++j) fill[j] = tp[j];
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int32_t j = colind[e];
            int32_t at = fill[j]++;
            ti[at] = i;
            if (tw) tw[at] = w[e];
        }
    free(fill);
    *out_ptr = tp;
    *out_ind = ti;
    if (out_w) *out_w = tw;
    return ORC_OK;
}

/* BFS levels by a FIFO queue over the edges j -> i of the entries A_ij:
 * level 0 at src, -1 where unreachable. */
int orc_bfs(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t src, int32_t* levels) {
    if (src < 0 || src >= n) return ORC_EINVAL;
    int32_t *op = NULL, *oi = NULL;
    if (transpose_csr(n, rowptr, colind, NULL, &op, &oi, NULL) != ORC_OK) return ORC_ENOMEM;
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!queue) { free(op); free(oi); return ORC_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) levels[v] = -1;
    int64_t head = 0, tail = 0;
    levels[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = op[u]; e < op[u + 1]; ++e) {
            int32_t v = oi[e];
            if (levels[v] < 0) { levels[v] = levels[u] + 1; queue[tail++] = v; }
        }
    }
    free(queue);
    free(op);
    free(oi);
    return ORC_OK;
}

/* Single-source shortest paths by Dijkstra with a binary heap, in fp64 over
 * fp32 weights, following the edges j -> i of the entries A_ij with weight
 * w_ij (w in CSR order; NULL: unit weights).  Unreachable vertices get +inf.
 * Any SSSP method (delta-stepping, Bellman-Ford) reaches these distances. */
typedef struct { double d; int32_t v; } heap_item;

static void heap_push(heap_item* h, int64_t* size, heap_item it) {
    int64_t i = (*size)++;
    h[i] = it;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item* h, int64_t* size) {
    heap_item top = h[0];
    h[0] = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *size && h[l].d < h[s].d) s = l;
        if (r < *size && h[r].d < h[s].d) s = r;
        if (s == i) break;
        heap_item t = h[s]; h[s] = h[i]; h[i] = t;
        i = s;
    }
    return top;
}

int orc_sssp(int32_t n, const int32_t* rowptr, const int32_t* colind, const float* w, int32_t src,
             double* dist) {
    if (src < 0 || src >= n) return ORC_EINVAL;
    int32_t *op = NULL, *oi = NULL;
    float* ow = NULL;
    if (transpose_csr(n, rowptr, colind, w, &op, &oi, w ? &ow : NULL) != ORC_OK) return ORC_ENOMEM;
    int64_t cap = (int64_t)rowptr[n] + 1;
    heap_item* heap = (heap_item*)malloc((size_t)cap * sizeof(heap_item));
    uint8_t* done = (uint8_t*)calloc((size_t)n, 1);
    if (!heap || !done) { free(heap); free(done); free(op); free(oi); free(ow); return ORC_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
    int64_t size = 0;
    dist[src] = 0.0;
    heap_item s0 = {0.0, src};
    heap_push(heap, &size, s0);
    while (size > 0) {
        heap_item it = heap_pop(heap, &size);
        if (done[it.v]) continue;
        done[it.v] = 1;
        for (int64_t e = op[it.v]; e < op[it.v + 1]; ++e) {
            int32_t v = oi[e];
            double nd = it.d + (ow ? (double)ow[e] : 1.0);
            if (nd < dist[v]) {
                dist[v] = nd;
                heap_item ni = {nd, v};
                heap_push(heap, &size, ni);
            }
        }
    }
    free(heap);
    free(done);
    free(op);
    free(oi);
    free(ow);
    return ORC_OK;
}

/* PageRank by power iteration with the column-stochastic adjacency matrix
 * (Sec. V PR): each 1 at (i, j) carries x_j / outdeg(j), where outdeg(j) is
 * the number of ones in column j.  x^0 = 1/n and, for exactly `iters` steps,
 *     x_i <- (1 - d) * t_i + d * sum_{j in row i} x_j / outdeg(j),
 * with t = teleport (NULL: uniform 1/n).  Vertices with no out-edges pass
 * nothing on (no redistribution of dangling mass).  All in fp64. */
int orc_pagerank(int32_t n, const int32_t* rowptr, const int32_t* colind, double d, int iters,
                 const double* teleport, double* x) {
    if (n <= 0) return ORC_OK;
    int64_t* outdeg = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    double* c = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !c) { free(outdeg); free(c); return ORC_ENOMEM; }
    for (int64_t e = 0; e < rowptr[n]; ++e) outdeg[colind[e]] += 1;
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    for (int t = 0; t < iters; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j) c[j] = outdeg[j] > 0 ? x[j] / (double)outdeg[j] : 0.0;
#pragma omp parallel for schedule(dynamic, ROW_BLOCK)
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += c[colind[e]];
            double ti = teleport ? teleport[i] : 1.0 / (double)n;
            x[i] = (1.0 - d) * ti + d * s;
        }
    }
    free(outdeg);
    free(c);
    return ORC_OK;
}

/* Connected components by union-find; each vertex is labelled with the
 * smallest vertex id of its component (the fixed point FastSV reaches). */
static int32_t uf_find(int32_t* p, int32_t v) {
    while (p[v] != v) { p[v] = p[p[v]]; v = p[v]; }
    return v;
}

int orc_cc(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t* labels) {
    int32_t* p = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!p) return ORC_ENOMEM;
    for (int32_t v = 0; v < n; ++v) p[v] = v;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int32_t a = uf_find(p, i), b = uf_find(p, colind[e]);
            if (a < b) p[b] = a; else if (b < a) p[a] = b;
        }
    /* with the smaller root always kept, every root is its component's minimum */
    for (int32_t v = 0; v < n; ++v) labels[v] = uf_find(p, v);
    free(p);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sampling profile (Sec. III-C, Algorithm 1)                                  */
/* ------------------------------------------------------------------------ */

/* For each k in {4, 8, 16, 32}: every sampled row i stands for its tile-row
 * i / k, whose distinct tile columns (column / k over its k rows) are counted;
 * the mean count times nTileRow estimates T_k, and
 *   est[q] = (4(nTileRow+1) + T_k (4 + k word_bytes(k))) / (4(n+1) + 8 nnz),
 * the B2SR size over the size of an fp32-valued CSR (Sec. VI-B).  The sampled
 * rows are an input (random draws are passed in). */
int orc_sample_profile(int32_t n, const int32_t* rowptr, const int32_t* colind,
                       const int32_t* sample, int64_t nsample, double* est /* [4] */,
                       double* tiles_est /* [4] */) {
    static const int ks[4] = {4, 8, 16, 32};
    int64_t maxm = 0;
    for (int q = 0; q < 4; ++q)
        for (int64_t s = 0; s < nsample; ++s) {
            int64_t I = sample[s] / ks[q];
            int64_t r0 = I * ks[q], r1 = r0 + ks[q] < n ? r0 + ks[q] : n;
            if (rowptr[r1] - rowptr[r0] > maxm) maxm = rowptr[r1] - rowptr[r0];
        }
    int32_t* buf = (int32_t*)malloc((size_t)(maxm > 0 ? maxm : 1) * sizeof(int32_t));
    if (!buf) return ORC_ENOMEM;
    for (int q = 0; q < 4; ++q) {
        int k = ks[q];
        int64_t ntr = ((int64_t)n + k - 1) / k;
        double sum = 0.0;
        for (int64_t s = 0; s < nsample; ++s) {
            if (sample[s] < 0 || sample[s] >= n) { free(buf); return ORC_EINVAL; }
            sum += (double)tile_row_columns(n, rowptr, colind, k, sample[s] / k, buf);
        }
        double t_hat = nsample > 0 ? sum / (double)nsample * (double)ntr : 0.0;
        double b2sr = 4.0 * (double)(ntr + 1) + t_hat * (4.0 + (double)(k * word_bytes(k)));
        double csr = 4.0 * ((double)n + 1.0) + 8.0 * (double)rowptr[n];
        est[q] = b2sr / csr;
        tiles_est[q] = t_hat;
    }
    free(buf);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Maximal independent set and colouring by priority (Table 4: MIS, GC)      */
/* ------------------------------------------------------------------------ */

/* Vertices in decreasing priority (ties: larger id first), the order both
 * functions below follow.  qsort with the priorities in a file-scope pointer
 * (the oracle runs on one thread). */
static const double* g_prio;

static int cmp_prio_desc(const void* pa, const void* pb) {
    int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    if (g_prio[a] != g_prio[b]) return g_prio[a] > g_prio[b] ? -1 : 1;
    return a > b ? -1 : (a < b ? 1 : 0);
}

static int64_t* by_priority_desc(int32_t n, const double* prio) {
    int64_t* order = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!order) return NULL;
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_prio = prio;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_prio_desc);
    return order;
}

/* Greedy maximal independent set in decreasing priority: a vertex joins
 * unless a neighbour already joined.  (With distinct priorities this is the
 * set the synchronous local-maximum rounds of Luby's algorithm reach.)
 * in_set[v] = 1 or 0.  The matrix is read as undirected (symmetric). */
int orc_mis_greedy(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* prio,
                   int32_t* in_set) {
    int64_t* order = by_priority_desc(n, prio);
    if (!order) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i) in_set[i] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t v = order[k];
        int blocked = 0;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1] && !blocked; ++e)
            if (colind[e] != v && in_set[colind[e]]) blocked = 1;
        in_set[v] = !blocked;
    }
    free(order);
    return ORC_OK;
}

/* Colouring by priority levels: colour(v) = 0 if no neighbour has a higher
 * priority, else 1 + the largest colour among higher-priority neighbours
 * (the round in which v becomes a local maximum among uncoloured vertices).
 * Neighbours never share a colour. */
int orc_color_levels(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* prio,
                     int32_t* color) {
    int64_t* order = by_priority_desc(n, prio);
    if (!order) return ORC_ENOMEM;
    for (int64_t k = 0; k < n; ++k) {
        int64_t v = order[k];
        int32_t c = 0;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int64_t u = colind[e];
            if (u == v) continue;
            if (prio[u] > prio[v] || (prio[u] == prio[v] && u > v))
                if (color[u] + 1 > c) c = color[u] + 1;
        }
        color[v] = c;
    }
    free(order);
    return ORC_OK;
}
