/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, single-threaded CPU implementation of the transposition of a
 * multigraph / high-cardinality sparse matrix stored in XCSR, used to check
 * the GPU path.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never calls it.
 *
 * What it computes (Sec. 2 of the paper, "Problem Specification"):
 *   M^T_ij = M_ji, i.e. every edge {i, j, e} of the input becomes {j, i, e}.
 *   XCSR (Sec. 2, the format with per-cell value counts) stores row-major
 *   cells; each cell (i, j) holds a list of values of its own length.
 * Readings taken where the paper is silent:
 *   - inside an output row j the cells are in ascending source-cell order
 *     (the "row-column ordering" of the view-swap step, Sec. 3); with
 *     distinct columns per input row this is ascending source row i;
 *   - a cell's values keep their internal order, byte for byte;
 *   - zero-length cells and empty rows/columns are legal and still move;
 *   - output row blocks use the input's row intervals (Sec. 2: vertex
 *     information stays where it is); P x P counts follow the metadata and
 *     value-count matrices of the view swap (Sec. 3, both steps).
 *
 * Algorithm: the textbook counting transpose (Gustavson 1978, cited by the
 * paper in Sec. 1), written from the definition:
 *   1. deg[j]      = number of cells with column j
 *   2. row_ptr'    = exclusive prefix of deg
 *   3. walk rows i ascending, cells k ascending: q = cursor[col[k]]++,
 *      col'[q] = i, src[q] = k
 *   4. cell_ptr'   = prefix of run lengths taken in output order
 *   5. copy each run's bytes from its source to its output offset
 *   6. P x P: cells[p(i)][p(j)] += 1, values[p(i)][p(j)] += len
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define XO_OK 0
#define XO_EINVAL -1
#define XO_ENOMEM -2
#define XO_EBADINPUT -3

#ifndef XO_MUTANT
#define XO_MUTANT 0 /* >0 only in the pin-strength test: plants one known mistake */
#endif

static inline int64_t ld(const void *p, int o, int64_t i) {
    return o == 4 ? (int64_t)((const int32_t *)p)[i] : ((const int64_t *)p)[i];
}
static inline void st(void *p, int o, int64_t i, int64_t v) {
    if (o == 4) ((int32_t *)p)[i] = (int32_t)v; else ((int64_t *)p)[i] = v;
}

/* partition of row r: largest d with off[d] <= r (binary search) */
static int64_t part_of(const int64_t *off, int64_t P, int64_t r) {
    int64_t lo = 0, hi = P - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (off[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Checks the input is a well-formed XCSR matrix and the partition is a cover
 * of disjoint row intervals (Sec. 2: cover and distinct properties). */
int xo_validate(int64_t R, int64_t N, int64_t C, int64_t V, int o, int s,
                const void *row_ptr, const int32_t *col, const void *cell_ptr,
                int64_t P, const int64_t *off) {
    if (R < 0 || N < 0 || C < 0 || V < 0 || (o != 4 && o != 8) || s <= 0) return XO_EINVAL;
    if (ld(row_ptr, o, 0) != 0 || ld(row_ptr, o, R) != C) return XO_EBADINPUT;
    for (int64_t i = 0; i < R; i++)
        if (ld(row_ptr, o, i + 1) < ld(row_ptr, o, i)) return XO_EBADINPUT;
    if (ld(cell_ptr, o, 0) != 0 || ld(cell_ptr, o, C) != V) return XO_EBADINPUT;
    for (int64_t k = 0; k < C; k++) {
        if (ld(cell_ptr, o, k + 1) < ld(cell_ptr, o, k)) return XO_EBADINPUT;
        if (col[k] < 0 || (int64_t)col[k] >= N) return XO_EBADINPUT;
    }
    if (P < 1) return XO_EINVAL;
    if (off) {
        if (off[0] != 0 || off[P] != R) return XO_EINVAL;
        for (int64_t d = 0; d < P; d++) if (off[d + 1] < off[d]) return XO_EINVAL;
        if (P > 1 && R != N) return XO_EINVAL;
    }
    return XO_OK;
}

/* Full transpose.  Outputs (caller-allocated): t_row_ptr[N+1], t_col[C],
 * t_cell_ptr[C+1] (width o), t_values[V*s]; optional src[C] (int64, the
 * source cell of each output cell); optional part_cells/part_values[P*P]
 * (int64, row-major [source partition][destination partition]). */
int xo_transpose(int64_t R, int64_t N, int64_t C, int64_t V, int o, int s,
                 const void *row_ptr, const int32_t *col, const void *cell_ptr,
                 const uint8_t *values, int64_t P, const int64_t *off,
                 void *t_row_ptr, int32_t *t_col, void *t_cell_ptr, uint8_t *t_values,
                 int64_t *src, int64_t *part_cells, int64_t *part_values) {
    int rc = xo_validate(R, N, C, V, o, s, row_ptr, col, cell_ptr, P, off);
    if (rc != XO_OK) return rc;
    int64_t *cur = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    int64_t *own_src = src ? NULL : (int64_t *)malloc((size_t)(C > 0 ? C : 1) * sizeof(int64_t));
    if (!cur || (!src && !own_src)) { free(cur); free(own_src); return XO_ENOMEM; }
    if (!src) src = own_src;

    /* 1. column degrees */
    for (int64_t k = 0; k < C; k++) cur[col[k] + 1]++;
    /* 2. exclusive prefix -> output row pointers */
    for (int64_t j = 0; j < N; j++) cur[j + 1] += cur[j];
    for (int64_t j = 0; j <= N; j++) st(t_row_ptr, o, j, cur[j]);
    /* 3. walk the input in row-major order and deal each cell to its column */
    for (int64_t i = 0; i < R; i++) {
        int64_t k0 = ld(row_ptr, o, i), k1 = ld(row_ptr, o, i + 1);
#if XO_MUTANT == 1
        /* planted: cells of a row dealt in reverse order */
        for (int64_t k = k1 - 1; k >= k0; k--) {
#else
        for (int64_t k = k0; k < k1; k++) {
#endif
            int64_t q = cur[col[k]]++;
#if XO_MUTANT == 2
            t_col[q] = (int32_t)col[k]; /* planted: keeps the column, not the row */
#else
            t_col[q] = (int32_t)i;
#endif
            src[q] = k;
        }
    }
    /* 4. output cell pointers: running sum of run lengths in output order */
    int64_t acc = 0;
    st(t_cell_ptr, o, 0, 0);
    for (int64_t q = 0; q < C; q++) {
        int64_t k = src[q];
#if XO_MUTANT == 3
        int64_t len = ld(cell_ptr, o, k + 1) - ld(cell_ptr, o, k) + (q == C / 2 ? 1 : 0) - (q == C / 2 + 1 ? 1 : 0);
#else
        int64_t len = ld(cell_ptr, o, k + 1) - ld(cell_ptr, o, k);
#endif
        acc += len;
        st(t_cell_ptr, o, q + 1, acc);
    }
    /* 5. move every run, keeping the order of values inside it */
    for (int64_t q = 0; q < C; q++) {
        int64_t k = src[q];
        int64_t from = ld(cell_ptr, o, k), len = ld(cell_ptr, o, k + 1) - from;
        int64_t to = ld(t_cell_ptr, o, q);
#if XO_MUTANT == 4
        if (len > 1) { /* planted: first two values of a run swapped */
            memcpy(t_values + (size_t)to * s, values + (size_t)(from + 1) * s, (size_t)s);
            memcpy(t_values + (size_t)(to + 1) * s, values + (size_t)from * s, (size_t)s);
            if (len > 2) memcpy(t_values + (size_t)(to + 2) * s, values + (size_t)(from + 2) * s, (size_t)(len - 2) * s);
            continue;
        }
#endif
        if (len > 0) memcpy(t_values + (size_t)to * (size_t)s, values + (size_t)from * (size_t)s, (size_t)len * (size_t)s);
    }
    /* 6. P x P metadata and value counts */
    if (part_cells || part_values) {
        if (part_cells) memset(part_cells, 0, (size_t)(P * P) * sizeof(int64_t));
        if (part_values) memset(part_values, 0, (size_t)(P * P) * sizeof(int64_t));
        int64_t eq[2] = {0, R};
        const int64_t *bounds = off ? off : eq;
        int64_t PP = off ? P : 1;
        for (int64_t i = 0; i < R; i++) {
            int64_t ps = part_of(bounds, PP, i);
            for (int64_t k = ld(row_ptr, o, i); k < ld(row_ptr, o, i + 1); k++) {
#if XO_MUTANT == 5
                int64_t pd = part_of(bounds, PP, i); /* planted: destination taken from the row */
#else
                int64_t pd = part_of(bounds, PP, col[k]);
#endif
                if (part_cells) part_cells[ps * P + pd] += 1;
                if (part_values) part_values[ps * P + pd] += ld(cell_ptr, o, k + 1) - ld(cell_ptr, o, k);
            }
        }
    }
    free(cur);
    free(own_src);
    return XO_OK;
}

/* Column degrees only (deg[N], int64): row_ptr' is their exclusive prefix.
 * Used for full-size checks where the whole transpose is too large. */
int xo_degrees(int64_t C, const int32_t *col, int64_t N, int64_t *deg) {
    memset(deg, 0, (size_t)N * sizeof(int64_t));
    for (int64_t k = 0; k < C; k++) {
        if (col[k] < 0 || (int64_t)col[k] >= N) return XO_EBADINPUT;
        deg[col[k]]++;
    }
    return XO_OK;
}

/* Selected output rows, computed one by one from the definition: output row
 * j lists, in row-major input order, every input cell whose column is j.
 * rows[m] must be strictly ascending.  Two calls: with t_col == NULL it fills
 * cnt[m] (cells per selected row) and vcnt[m] (values per selected row);
 * then, with buffers sized from those counts, it fills the selected rows'
 * cells back to back: t_col (source rows), t_len (run lengths, int64) and
 * t_values (run bytes). */
int xo_rows(int64_t R, int64_t C, int o, int s, const void *row_ptr, const int32_t *col,
            const void *cell_ptr, const uint8_t *values, int64_t m, const int64_t *rows,
            int64_t *cnt, int64_t *vcnt, int32_t *t_col, int64_t *t_len, uint8_t *t_values) {
    (void)C;
    int64_t *pos = NULL, *vpos = NULL;
    if (t_col) {
        pos = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
        vpos = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
        if (!pos || !vpos) { free(pos); free(vpos); return XO_ENOMEM; }
        pos[0] = 0; vpos[0] = 0;
        for (int64_t t = 0; t < m; t++) { pos[t + 1] = pos[t] + cnt[t]; vpos[t + 1] = vpos[t] + vcnt[t]; }
    } else {
        for (int64_t t = 0; t < m; t++) { cnt[t] = 0; vcnt[t] = 0; }
    }
    for (int64_t i = 0; i < R; i++) {
        for (int64_t k = ld(row_ptr, o, i); k < ld(row_ptr, o, i + 1); k++) {
            int64_t j = col[k];
            /* binary search j among the selected rows */
            int64_t lo = 0, hi = m;
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (rows[mid] < j) lo = mid + 1; else hi = mid; }
            if (lo >= m || rows[lo] != j) continue;
            int64_t from = ld(cell_ptr, o, k), len = ld(cell_ptr, o, k + 1) - from;
            if (!t_col) { cnt[lo] += 1; vcnt[lo] += len; continue; }
            t_col[pos[lo]] = (int32_t)i;
            t_len[pos[lo]] = len;
            if (len > 0) memcpy(t_values + (size_t)vpos[lo] * s, values + (size_t)from * s, (size_t)len * s);
            pos[lo] += 1;
            vpos[lo] += len;
        }
    }
    free(pos);
    free(vpos);
    return XO_OK;
}

/* Variable-width values: the paper's second variation of the exchange
 * (Sec. 2, heterogeneous datatypes across edges through MPI_Alltoallw, one
 * datatype per edge).  Value v of the input occupies bytes
 * [val_off[v], val_off[v+1]) of `values` (val_off: int64, V + 1 entries,
 * val_off[0] = 0, non-decreasing; a zero-size value is allowed).  The cells
 * move exactly as in xo_transpose (same output row_ptr', col', cell_ptr');
 * every value keeps its own bytes and its place in its cell's list, so the
 * output lists the same values in the output's cell order:
 *   t_val_off[p + 1] = t_val_off[p] + size of the value now at position p,
 *   t_values[t_val_off[p] ..] = that value's bytes.
 * Outputs (caller-allocated): t_row_ptr[N+1], t_col[C], t_cell_ptr[C+1]
 * (width o), t_val_off[V+1] (int64), t_values[val_off[V]]. */
int xo_transpose_var(int64_t R, int64_t N, int64_t C, int64_t V, int o,
                     const void *row_ptr, const int32_t *col, const void *cell_ptr,
                     const int64_t *val_off, const uint8_t *values,
                     void *t_row_ptr, int32_t *t_col, void *t_cell_ptr,
                     int64_t *t_val_off, uint8_t *t_values) {
    int rc = xo_validate(R, N, C, V, o, 1, row_ptr, col, cell_ptr, 1, NULL);
    if (rc != XO_OK) return rc;
    if (!val_off || val_off[0] != 0) return XO_EBADINPUT;
    for (int64_t v = 0; v < V; v++)
        if (val_off[v + 1] < val_off[v]) return XO_EBADINPUT;
    int64_t *cur = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    int64_t *src = (int64_t *)malloc((size_t)(C > 0 ? C : 1) * sizeof(int64_t));
    if (!cur || !src) { free(cur); free(src); return XO_ENOMEM; }
    /* the cells: degrees, prefix, row-major walk, run offsets (as xo_transpose) */
    for (int64_t k = 0; k < C; k++) cur[col[k] + 1]++;
    for (int64_t j = 0; j < N; j++) cur[j + 1] += cur[j];
    for (int64_t j = 0; j <= N; j++) st(t_row_ptr, o, j, cur[j]);
    for (int64_t i = 0; i < R; i++)
        for (int64_t k = ld(row_ptr, o, i); k < ld(row_ptr, o, i + 1); k++) {
            int64_t q = cur[col[k]]++;
            t_col[q] = (int32_t)i;
            src[q] = k;
        }
    int64_t acc = 0;
    st(t_cell_ptr, o, 0, 0);
    for (int64_t q = 0; q < C; q++) {
        acc += ld(cell_ptr, o, src[q] + 1) - ld(cell_ptr, o, src[q]);
        st(t_cell_ptr, o, q + 1, acc);
    }
    /* the values, one at a time in output order: each keeps its size and bytes */
    int64_t p = 0;
    t_val_off[0] = 0;
    for (int64_t q = 0; q < C; q++) {
        int64_t k = src[q];
        for (int64_t v = ld(cell_ptr, o, k); v < ld(cell_ptr, o, k + 1); v++, p++) {
#if XO_MUTANT == 6
            /* planted: the size of the next value instead of this one (kept
             * inside both buffers so that the mistake shows only in the output) */
            int64_t size = (v + 1 < V) ? val_off[v + 2] - val_off[v + 1] : val_off[v + 1] - val_off[v];
            if (t_val_off[p] + size > val_off[V]) size = val_off[V] - t_val_off[p];
            if (val_off[v] + size > val_off[V]) size = val_off[V] - val_off[v];
            if (size < 0) size = 0;
#else
            int64_t size = val_off[v + 1] - val_off[v];
#endif
#if XO_MUTANT == 7
            /* planted: the values keep their input byte offsets (not moved) */
            t_val_off[p + 1] = val_off[v + 1];
            if (size > 0) memcpy(t_values + val_off[v], values + val_off[v], (size_t)size);
#else
            t_val_off[p + 1] = t_val_off[p] + size;
            if (size > 0) memcpy(t_values + t_val_off[p], values + val_off[v], (size_t)size);
#endif
        }
    }
    free(cur);
    free(src);
    return XO_OK;
}
