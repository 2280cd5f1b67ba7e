/*
 * Sequential CPU oracle for the extremum graph of a piecewise-linear scalar
 * field on a d-dimensional grid (Ande, Subhash & Natarajan, "Tachyon:
 * efficient shared memory parallel computation of extremum graphs").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this file: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Everything here is the plain definition, written out one vertex at a time:
 *
 *   order       v < w  iff  f[v] < f[w], or f[v] == f[w] and v < w
 *               (simulated perturbation, Sec. 3.3; ties go to the larger
 *               linear index).  IEEE comparison, so -0 == +0.
 *   adjacency   Algorithm 1 (GridAdjacency, Sec. 3.2): p ~ q iff the
 *               component-wise differences all lie in {0,1} or all in {0,-1}
 *               and p != q.  The neighbours of v are the in-bounds grid
 *               vertices adjacent to v; there is no periodicity.
 *   link        the neighbours of v with the induced edges (Sec. 3.3); two
 *               link vertices share a link edge iff Algorithm 1 says they are
 *               adjacent.
 *   beta0+      number of connected components of the upper link, by a
 *               union-find that starts from singleton sets and unions the two
 *               end points of every link edge whose end points are both upper
 *               (Sec. 3.3).
 *   classes     Table 1: maximum iff beta0+ == 0, (n-1)-saddle iff
 *               beta0+ >= 2 (multi-saddles included).
 *   gradient    the highest vertex of the upper link (Sec. 3.3); a maximum
 *               points to itself.
 *   label       the maximum reached by following the gradient (Algorithm 2's
 *               inner loop), i.e. the descending manifold of that maximum
 *               (Sec. 2).
 *   reps        UpperLinkRep: the highest vertex of each upper-link component
 *               (Sec. 3.4), reported per saddle in ascending id order.
 *   arcs        (s, label(rep)) for every saddle s and every component,
 *               duplicates removed, sorted by (s, m) (Sec. 2: arc (s,m) iff s
 *               bounds the descending manifold of m).
 *   paths       the geometry of every arc (Algorithm 2): for every saddle s in
 *               ascending order and every component in ascending order of its
 *               representative, the vertices s, rep, gradient(rep), ...,
 *               up to the maximum reached.
 *
 * The minimum graph (Sec. 2, Sec. 5) is the same computation with the order
 * reversed: "higher" becomes "lower" under the same perturbation.
 *
 * Element types (Sec. 5: 8- to 64-bit signed and unsigned integers, 32- and
 * 64-bit floats): two values are compared in their own type, with C's
 * comparison operators on that type; nothing is converted.  The value copies
 * of maxima and saddles are the input's bytes.
 *
 * Vertex index: v = x0 + n0*(x1 + n1*(x2 + ...)), axis 0 fastest.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define EO_MAXD 6
#define EO_MAXNB 126 /* 2*(2^6-1) */

enum { EO_OK = 0, EO_ERR_ARG = 1, EO_ERR_NAN = 2, EO_ERR_OOM = 3 };

/* element types of a field */
enum { EO_F32 = 0, EO_F64 = 1, EO_I8 = 2, EO_U8 = 3, EO_I16 = 4, EO_U16 = 5,
       EO_I32 = 6, EO_U32 = 7, EO_I64 = 8, EO_U64 = 9, EO_NTYPES = 10 };

static size_t eo_dtype_size(int t)
{
    switch (t) {
    case EO_I8: case EO_U8: return 1;
    case EO_I16: case EO_U16: return 2;
    case EO_F32: case EO_I32: case EO_U32: return 4;
    case EO_F64: case EO_I64: case EO_U64: return 8;
    default: return 0;
    }
}

typedef struct eo_result {
    int64_t n;
    int64_t n_max, n_sad, n_paths, n_arcs;
    uint32_t *asc;     /* [n] gradient pointer */
    uint32_t *label;   /* [n] maximum reached */
    uint8_t *beta0p;   /* [n] number of upper-link components */
    uint32_t *maxima;  /* [n_max] ascending */
    int dtype;         /* element type of the field and of the value copies */
    void *max_val;     /* [n_max] value copies, in the field's type */
    uint32_t *saddles; /* [n_sad] ascending */
    uint8_t *sad_b0;   /* [n_sad] */
    void *sad_val;     /* [n_sad] value copies, in the field's type */
    uint64_t *row_ptr; /* [n_sad+1] */
    uint32_t *col;     /* [n_arcs] */
    uint32_t *reps;    /* [n_paths] UpperLinkRep of every saddle, saddles in order,
                          each saddle's representatives in ascending id order */
} eo_result;

/* ---- order (simulated perturbation, Sec. 3.3) ----------------------------- */

/* The field: its values and their element type. */
typedef struct eo_field {
    const void *f;
    int t;
} eo_field;

#define EO_CMP(T) { T x = ((const T *)F->f)[a], y = ((const T *)F->f)[b]; return (x > y) - (x < y); }

/* Sign of f[a] - f[b], comparing the two values in their own type. */
static int eo_cmp_values(const eo_field *F, uint32_t a, uint32_t b)
{
    switch (F->t) {
    case EO_F32: EO_CMP(float)
    case EO_F64: EO_CMP(double)
    case EO_I8: EO_CMP(int8_t)
    case EO_U8: EO_CMP(uint8_t)
    case EO_I16: EO_CMP(int16_t)
    case EO_U16: EO_CMP(uint16_t)
    case EO_I32: EO_CMP(int32_t)
    case EO_U32: EO_CMP(uint32_t)
    case EO_I64: EO_CMP(int64_t)
    default: EO_CMP(uint64_t)
    }
}

static int eo_isnan(const eo_field *F, uint64_t v)
{
    if (F->t == EO_F32) return isnan(((const float *)F->f)[v]);
    if (F->t == EO_F64) return isnan(((const double *)F->f)[v]);
    return 0;
}

/* 1 iff w is higher than v.  With reverse set, "higher" means lower: the
 * minimum graph is the maximum graph of the reversed order. */
static int eo_higher(const eo_field *F, uint32_t v, uint32_t w, int reverse)
{
    int c = eo_cmp_values(F, w, v);
    int up = c > 0 ? 1 : (c < 0 ? 0 : (w > v));
    return reverse ? !up : up;
}

/* ---- Algorithm 1 (GridAdjacency) ------------------------------------------ */

static int eo_grid_adjacency(int d, const int64_t *p, const int64_t *q)
{
    int has_pos = 0, has_neg = 0, has_zero_only = 1;
    for (int i = 0; i < d; i++) {
        int64_t diff = p[i] - q[i];
        if (diff == 1) { has_pos = 1; has_zero_only = 0; }
        else if (diff == -1) { has_neg = 1; has_zero_only = 0; }
        else if (diff != 0) return 0;
    }
    /* U subset of {0,1} or U subset of {0,-1}; p == q is not an edge. */
    if (has_zero_only) return 0;
    return !(has_pos && has_neg);
}

static void eo_coords(int d, const int64_t *ext, uint64_t v, int64_t *x)
{
    for (int i = 0; i < d; i++) {
        x[i] = (int64_t)(v % (uint64_t)ext[i]);
        v /= (uint64_t)ext[i];
    }
}

static uint64_t eo_index(int d, const int64_t *ext, const int64_t *x)
{
    uint64_t v = 0;
    for (int i = d - 1; i >= 0; i--) v = v * (uint64_t)ext[i] + (uint64_t)x[i];
    return v;
}

/* Candidate offsets in {-1,0,1}^d kept by Algorithm 1 against the origin. */
static int eo_offsets(int d, int64_t off[][EO_MAXD])
{
    int64_t zero[EO_MAXD] = {0};
    int cnt = 0, total = 1;
    for (int i = 0; i < d; i++) total *= 3;
    for (int t = 0; t < total; t++) {
        int64_t c[EO_MAXD];
        int r = t;
        for (int i = 0; i < d; i++) { c[i] = (r % 3) - 1; r /= 3; }
        if (eo_grid_adjacency(d, c, zero)) {
            memcpy(off[cnt], c, sizeof(int64_t) * d);
            cnt++;
        }
    }
    return cnt;
}

/* ---- union-find over link vertices (Sec. 3.3) ----------------------------- */

static int eo_find(int *parent, int a)
{
    while (parent[a] != a) {
        parent[a] = parent[parent[a]];
        a = parent[a];
    }
    return a;
}

static void eo_union(int *parent, int a, int b)
{
    a = eo_find(parent, a);
    b = eo_find(parent, b);
    if (a != b) parent[b] = a;
}

/* For one vertex v: the link vertices, which of them are upper, the upper-link
 * components and the highest vertex of each.  Returns beta0+; writes the
 * representatives (one per component, in no particular order) to reps and the
 * gradient (highest upper-link vertex, or v) to *grad. */
static int eo_classify_vertex(const eo_field *f, int d, const int64_t *ext,
                              int nnb, int64_t off[][EO_MAXD], uint32_t v,
                              int reverse, uint32_t *reps, uint32_t *grad)
{
    int64_t xv[EO_MAXD];
    int64_t lx[EO_MAXNB][EO_MAXD];
    uint32_t lid[EO_MAXNB];
    int upper[EO_MAXNB];
    int parent[EO_MAXNB];
    int nl = 0;

    eo_coords(d, ext, v, xv);
    for (int k = 0; k < nnb; k++) {
        int inb = 1;
        for (int i = 0; i < d; i++) {
            int64_t c = xv[i] + off[k][i];
            if (c < 0 || c >= ext[i]) { inb = 0; break; }
            lx[nl][i] = c;
        }
        if (!inb) continue;
        lid[nl] = (uint32_t)eo_index(d, ext, lx[nl]);
        upper[nl] = eo_higher(f, v, lid[nl], reverse);
        parent[nl] = nl;
        nl++;
    }

    /* gradient: highest vertex of the upper link */
    *grad = v;
    for (int a = 0; a < nl; a++)
        if (upper[a] && eo_higher(f, *grad, lid[a], reverse)) *grad = lid[a];

    /* union both end points of every upper-upper link edge */
    for (int a = 0; a < nl; a++)
        for (int b = a + 1; b < nl; b++)
            if (upper[a] && upper[b] && eo_grid_adjacency(d, lx[a], lx[b]))
                eo_union(parent, a, b);

    /* one representative (the highest vertex) per upper component */
    int nc = 0;
    for (int a = 0; a < nl; a++) {
        if (!upper[a] || eo_find(parent, a) != a) continue;
        uint32_t best = lid[a];
        for (int b = 0; b < nl; b++)
            if (upper[b] && eo_find(parent, b) == a && eo_higher(f, best, lid[b], reverse))
                best = lid[b];
        reps[nc++] = best;
    }
    return nc;
}

/* ---- helpers --------------------------------------------------------------- */

static int eo_cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

void eo_free(eo_result *r)
{
    if (!r) return;
    free(r->asc); free(r->label); free(r->beta0p);
    free(r->maxima); free(r->max_val);
    free(r->saddles); free(r->sad_b0); free(r->sad_val);
    free(r->row_ptr); free(r->col); free(r->reps);
    free(r);
}

/* ---- the computation ------------------------------------------------------ */

/* naive != 0: follow the gradient from every vertex to its maximum with no
 * reuse (Algorithm 2's loop, started everywhere).  naive == 0: the same walk,
 * back-filling the labels of every vertex on a walk once its end is known. */
int eo_compute_typed(const void *values, int dtype, int d, const int64_t *ext, int naive,
                     int reverse, eo_result **out)
{
    *out = NULL;
    const size_t es = eo_dtype_size(dtype);
    if (!values || !ext || d < 1 || d > EO_MAXD || es == 0) return EO_ERR_ARG;
    const eo_field field = {values, dtype};
    const eo_field *f = &field;
    uint64_t n = 1;
    for (int i = 0; i < d; i++) {
        if (ext[i] < 1) return EO_ERR_ARG;
        n *= (uint64_t)ext[i];
        if (n > 0xFFFFFFFFull) return EO_ERR_ARG;
    }
    for (uint64_t v = 0; v < n; v++)
        if (eo_isnan(f, v)) return EO_ERR_NAN;

    int64_t off[EO_MAXNB][EO_MAXD];
    int nnb = eo_offsets(d, off);

    eo_result *r = (eo_result *)calloc(1, sizeof(eo_result));
    if (!r) return EO_ERR_OOM;
    r->n = (int64_t)n;
    r->dtype = dtype;
    r->asc = (uint32_t *)malloc(n * sizeof(uint32_t));
    r->label = (uint32_t *)malloc(n * sizeof(uint32_t));
    r->beta0p = (uint8_t *)malloc(n);
    uint32_t *stack = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!r->asc || !r->label || !r->beta0p || !stack) { free(stack); eo_free(r); return EO_ERR_OOM; }

    /* Step 1: classify every vertex (Table 1) and record its gradient. */
    uint32_t reps[EO_MAXNB];
    int64_t n_max = 0, n_sad = 0, n_paths = 0;
    for (uint64_t v = 0; v < n; v++) {
        uint32_t g;
        int b = eo_classify_vertex(f, d, ext, nnb, off, (uint32_t)v, reverse, reps, &g);
        r->asc[v] = g;
        r->beta0p[v] = (uint8_t)b;
        if (b == 0) n_max++;
        if (b >= 2) { n_sad++; n_paths += b; }
    }

    /* Step 2: the maximum at the end of every gradient path. */
    const uint32_t UNSET = 0xFFFFFFFFu;
    if (naive) {
        for (uint64_t v = 0; v < n; v++) {
            uint32_t u = (uint32_t)v;
            while (r->asc[u] != u) u = r->asc[u];
            r->label[v] = u;
        }
    } else {
        for (uint64_t v = 0; v < n; v++) r->label[v] = UNSET;
        for (uint64_t v = 0; v < n; v++) {
            if (r->label[v] != UNSET) continue;
            uint64_t top = 0;
            uint32_t u = (uint32_t)v;
            while (r->label[u] == UNSET && r->asc[u] != u) {
                stack[top++] = u;
                u = r->asc[u];
            }
            uint32_t m = (r->label[u] != UNSET) ? r->label[u] : u;
            r->label[u] = m;
            while (top) r->label[stack[--top]] = m;
        }
    }
    free(stack);

    /* Step 3: nodes and arcs of the extremum graph. */
    r->n_max = n_max;
    r->n_sad = n_sad;
    r->n_paths = n_paths;
    r->maxima = (uint32_t *)malloc((n_max ? n_max : 1) * sizeof(uint32_t));
    r->max_val = malloc((n_max ? n_max : 1) * es);
    r->saddles = (uint32_t *)malloc((n_sad ? n_sad : 1) * sizeof(uint32_t));
    r->sad_b0 = (uint8_t *)malloc(n_sad ? n_sad : 1);
    r->sad_val = malloc((n_sad ? n_sad : 1) * es);
    r->row_ptr = (uint64_t *)malloc((n_sad + 1) * sizeof(uint64_t));
    r->col = (uint32_t *)malloc((n_paths ? n_paths : 1) * sizeof(uint32_t));
    r->reps = (uint32_t *)malloc((n_paths ? n_paths : 1) * sizeof(uint32_t));
    if (!r->maxima || !r->max_val || !r->saddles || !r->sad_b0 || !r->sad_val ||
        !r->row_ptr || !r->col || !r->reps) { eo_free(r); return EO_ERR_OOM; }

    int64_t im = 0, is = 0, ia = 0, ip = 0;
    r->row_ptr[0] = 0;
    for (uint64_t v = 0; v < n; v++) {
        if (r->beta0p[v] == 0) {
            r->maxima[im] = (uint32_t)v;
            memcpy((char *)r->max_val + im * es, (const char *)values + v * es, es);
            im++;
        } else if (r->beta0p[v] >= 2) {
            uint32_t g;
            int b = eo_classify_vertex(f, d, ext, nnb, off, (uint32_t)v, reverse, reps, &g);
            qsort(reps, (size_t)b, sizeof(uint32_t), eo_cmp_u32);
            for (int c = 0; c < b; c++) r->reps[ip++] = reps[c];
            uint32_t ends[EO_MAXNB];
            for (int c = 0; c < b; c++) ends[c] = r->label[reps[c]];
            qsort(ends, (size_t)b, sizeof(uint32_t), eo_cmp_u32);
            for (int c = 0; c < b; c++)
                if (c == 0 || ends[c] != ends[c - 1]) r->col[ia++] = ends[c];
            r->saddles[is] = (uint32_t)v;
            r->sad_b0[is] = (uint8_t)b;
            memcpy((char *)r->sad_val + is * es, (const char *)values + v * es, es);
            is++;
            r->row_ptr[is] = (uint64_t)ia;
        }
    }
    r->n_arcs = ia;
    *out = r;
    return EO_OK;
}

/* float32 field (the library's default element type). */
int eo_compute(const float *f, int d, const int64_t *ext, int naive, int reverse,
               eo_result **out)
{
    return eo_compute_typed(f, EO_F32, d, ext, naive, reverse, out);
}

/* Flat accessors for foreign-function callers. */
void eo_counts(const eo_result *r, int64_t *c5)
{
    c5[0] = r->n; c5[1] = r->n_max; c5[2] = r->n_sad; c5[3] = r->n_paths; c5[4] = r->n_arcs;
}

void eo_copy(const eo_result *r, uint32_t *asc, uint32_t *label, uint8_t *beta0p,
             uint32_t *maxima, void *max_val, uint32_t *saddles, uint8_t *sad_b0,
             void *sad_val, uint64_t *row_ptr, uint32_t *col, uint32_t *reps)
{
    size_t n = (size_t)r->n, es = eo_dtype_size(r->dtype);
    if (asc) memcpy(asc, r->asc, n * sizeof(uint32_t));
    if (label) memcpy(label, r->label, n * sizeof(uint32_t));
    if (beta0p) memcpy(beta0p, r->beta0p, n);
    if (maxima) memcpy(maxima, r->maxima, (size_t)r->n_max * sizeof(uint32_t));
    if (max_val) memcpy(max_val, r->max_val, (size_t)r->n_max * es);
    if (saddles) memcpy(saddles, r->saddles, (size_t)r->n_sad * sizeof(uint32_t));
    if (sad_b0) memcpy(sad_b0, r->sad_b0, (size_t)r->n_sad);
    if (sad_val) memcpy(sad_val, r->sad_val, (size_t)r->n_sad * es);
    if (row_ptr) memcpy(row_ptr, r->row_ptr, (size_t)(r->n_sad + 1) * sizeof(uint64_t));
    if (col) memcpy(col, r->col, (size_t)r->n_arcs * sizeof(uint32_t));
    if (reps) memcpy(reps, r->reps, (size_t)r->n_paths * sizeof(uint32_t));
}

/* Gradient paths (Algorithm 2): per saddle (ascending) and per component (in
 * the order of r->reps), s then the gradient path from the representative to
 * its maximum.  eo_path_vertices gives the total length; eo_paths fills
 * path_ptr[n_paths + 1] (offsets) and path_vtx. */
uint64_t eo_path_vertices(const eo_result *r)
{
    uint64_t total = 0;
    for (int64_t p = 0; p < r->n_paths; p++) {
        uint32_t u = r->reps[p];
        total += 2;
        while (r->asc[u] != u) {
            u = r->asc[u];
            total++;
        }
    }
    return total;
}

void eo_paths(const eo_result *r, uint64_t *path_ptr, uint32_t *path_vtx)
{
    uint64_t at = 0;
    int64_t p = 0;
    for (int64_t i = 0; i < r->n_sad; i++) {
        for (int c = 0; c < r->sad_b0[i]; c++, p++) {
            path_ptr[p] = at;
            uint32_t u = r->reps[p];
            path_vtx[at++] = r->saddles[i];
            path_vtx[at++] = u;
            while (r->asc[u] != u) {
                u = r->asc[u];
                path_vtx[at++] = u;
            }
        }
    }
    path_ptr[p] = at;
}

/* Neighbour offsets kept by Algorithm 1 (for tests of the adjacency itself). */
int eo_neighbour_offsets(int d, int64_t *out /* [2*(2^d-1)*d] */)
{
    if (d < 1 || d > EO_MAXD) return -1;
    int64_t off[EO_MAXNB][EO_MAXD];
    int n = eo_offsets(d, off);
    for (int k = 0; k < n; k++)
        for (int i = 0; i < d; i++) out[k * d + i] = off[k][i];
    return n;
}

int eo_grid_adjacent(int d, const int64_t *p, const int64_t *q)
{
    return eo_grid_adjacency(d, p, q);
}
