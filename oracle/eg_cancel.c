/*
 * Sequential CPU oracle for persistence-directed cancellation (Sec. 3.5 of
 * Ande, Subhash & Natarajan, "Tachyon: efficient shared memory parallel
 * computation of extremum graphs") on a finished extremum graph.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this file; it shares no code, header or constant with the CUDA library.
 *
 * The paper's procedure, step by step:
 *   1. every (n-1)-saddle enters a priority queue keyed by its cost, the
 *      difference in value between the saddle and the second highest maximum
 *      adjacent to it (for a simple saddle, the lower of its two maxima);
 *   2. repeatedly take the saddle at the top and recompute its cost against
 *      the graph as it is now (lazy update);
 *        - cost above the persistence threshold: discard the saddle;
 *        - cost above the key of the new top of the queue: reinsert it with
 *          the recomputed cost;
 *        - otherwise cancel it: every maximum adjacent to it except the
 *          highest (the surviving maximum) is merged into the surviving one
 *          (the gradient paths from the saddle towards them are reversed), so
 *          every arc that ended at a merged maximum now ends at the survivor;
 *   3. until the queue is empty.
 *
 * Readings where the paper leaves a case open (each one is listed with the
 * design notes of the library):
 *   R1 "adjacent maxima" are the distinct maxima the saddle's arcs end at
 *      after the merges done so far.  A saddle with fewer than two has no
 *      second maximum and no cost: it is never cancelled (when taken from the
 *      queue it is discarded).
 *   R2 "highest" is the simulated-perturbation order (value, then vertex id);
 *      for the minimum graph every order is reversed (lowest maximum ==
 *      lowest minimum, cost = saddle value minus the second lowest minimum).
 *   R3 the cost is computed in float32, the field's own precision: 0 when the
 *      two values are equal (equal infinities included), else their
 *      difference rounded once to float32.  A saddle is cancelled only if
 *      its cost is at most the threshold (a float32 as well).
 *   R4 the queue orders saddles by (cost, vertex id), and "above the key of
 *      the new top" compares the same pairs, so equal costs are taken in
 *      ascending vertex id and the process is deterministic.
 *   R5 the paper states that later cancellations never lower a cost; that
 *      holds for simple saddles, but a cancellation that merges two maxima of
 *      a multi-saddle can lower its second highest maximum.  Such a saddle is
 *      given its lower cost at once: it is re-queued with it (a stale queue
 *      entry is skipped), including when it had been discarded and the lower
 *      cost is within the threshold.  With this, every cancellation takes the
 *      saddle of lowest current (cost, id) -- what the paper's steps do
 *      whenever its premise holds.
 *
 * Output: per saddle 1 = still in the graph, 0 = cancelled; per maximum the
 * vertex id of the maximum it was finally merged into (itself if it
 * survives); the number of cancellations.  The simplified graph is the kept
 * saddles with the survivors of their arc ends, duplicates removed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { EC_OK = 0, EC_ERR_ARG = 1, EC_ERR_OOM = 3 };

typedef struct ec_graph {
    int64_t nm, ns;
    const uint32_t *maxima;  /* [nm] vertex ids, ascending */
    const float *max_val;    /* [nm] */
    const uint32_t *saddles; /* [ns] vertex ids, ascending */
    const float *sad_val;    /* [ns] */
    const uint64_t *row_ptr; /* [ns+1] */
    int64_t *end;            /* [row_ptr[ns]] maximum index of every arc end */
    int reverse;             /* minimum graph */
} ec_graph;

/* 1 iff maximum a is higher than maximum b (R2). */
static int ec_higher(const ec_graph *G, int64_t a, int64_t b)
{
    float fa = G->max_val[a], fb = G->max_val[b];
    int up;
    if (fa != fb) up = fa > fb;
    else up = G->maxima[a] > G->maxima[b];
    return G->reverse ? !up : up;
}

/* ---- the current survivor of every maximum (merges always go into the
 * survivor of a cancellation, so a set's root is its highest maximum) ------ */
static int64_t ec_find(int64_t *parent, int64_t a)
{
    int64_t r = a;
    while (parent[r] != r) r = parent[r];
    while (parent[a] != r) {
        int64_t n = parent[a];
        parent[a] = r;
        a = n;
    }
    return r;
}

/* Current adjacent maxima of saddle s (R1): the distinct survivors of its
 * arc ends.  Writes the highest to *h1 and returns their number; *cost gets
 * the cost (R3) when there are at least two. */
static int64_t ec_adjacent(const ec_graph *G, int64_t *parent, int64_t s, int64_t *roots, int64_t *h1,
                           float *cost)
{
    int64_t n = 0;
    for (uint64_t a = G->row_ptr[s]; a < G->row_ptr[s + 1]; a++) {
        int64_t r = ec_find(parent, G->end[a]), k;
        for (k = 0; k < n && roots[k] != r; k++) {}
        if (k == n) roots[n++] = r;
    }
    if (n == 0) return 0;
    int64_t top = roots[0], second = -1;
    for (int64_t k = 1; k < n; k++) {
        if (ec_higher(G, roots[k], top)) {
            second = top;
            top = roots[k];
        } else if (second < 0 || ec_higher(G, roots[k], second)) {
            second = roots[k];
        }
    }
    *h1 = top;
    if (n >= 2) {
        float fm = G->max_val[second], fs = G->sad_val[s];
        *cost = fm == fs ? 0.0f : (G->reverse ? fs - fm : fm - fs);
    }
    return n;
}

/* ---- binary min-heap of (cost, saddle id) entries ------------------------- */
typedef struct ec_entry {
    float cost;
    uint32_t sid;   /* the saddle's vertex id (R4 tie-break) */
    int64_t s;      /* saddle index */
    uint64_t ver;   /* valid iff equal to the saddle's current version (R5) */
} ec_entry;

static int ec_less(const ec_entry *a, const ec_entry *b)
{
    return a->cost < b->cost || (a->cost == b->cost && a->sid < b->sid);
}

typedef struct ec_heap {
    ec_entry *e;
    int64_t n, cap;
} ec_heap;

static int ec_push(ec_heap *H, ec_entry x)
{
    if (H->n == H->cap) {
        int64_t c = H->cap ? 2 * H->cap : 64;
        ec_entry *p = (ec_entry *)realloc(H->e, (size_t)c * sizeof(ec_entry));
        if (!p) return EC_ERR_OOM;
        H->e = p;
        H->cap = c;
    }
    int64_t i = H->n++;
    H->e[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!ec_less(&H->e[i], &H->e[p])) break;
        ec_entry t = H->e[i];
        H->e[i] = H->e[p];
        H->e[p] = t;
        i = p;
    }
    return EC_OK;
}

static ec_entry ec_pop(ec_heap *H)
{
    ec_entry top = H->e[0];
    H->e[0] = H->e[--H->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < H->n && ec_less(&H->e[l], &H->e[m])) m = l;
        if (r < H->n && ec_less(&H->e[r], &H->e[m])) m = r;
        if (m == i) break;
        ec_entry t = H->e[i];
        H->e[i] = H->e[m];
        H->e[m] = t;
        i = m;
    }
    return top;
}

/* saddle states */
enum { EC_WAITING = 0, EC_DISCARDED = 1, EC_CANCELLED = 2 };

/* Persistence-directed cancellation with threshold tau.  col holds the arc
 * ends as maximum vertex ids (the extremum graph's CSR); alive[ns] and
 * survivor[nm] are written; *n_cancelled receives the number of cancelled
 * saddles. */
int ec_cancel(int64_t nm, const uint32_t *maxima, const float *max_val, int64_t ns, const uint32_t *saddles,
              const float *sad_val, const uint64_t *row_ptr, const uint32_t *col, int reverse, float tau,
              uint8_t *alive, uint32_t *survivor, int64_t *n_cancelled)
{
    if (nm < 0 || ns < 0 || isnan(tau) || (ns > 0 && (!saddles || !sad_val || !row_ptr || !alive)) ||
        (nm > 0 && (!maxima || !max_val || !survivor)))
        return EC_ERR_ARG;
    ec_graph G = {nm, ns, maxima, max_val, saddles, sad_val, row_ptr, NULL, reverse};
    uint64_t na = ns > 0 ? row_ptr[ns] : 0;
    int64_t *end = (int64_t *)malloc((size_t)(na + 1) * sizeof(int64_t));
    int64_t *parent = (int64_t *)malloc((size_t)(nm + 1) * sizeof(int64_t));
    int64_t *roots = (int64_t *)malloc((size_t)(na + 1) * sizeof(int64_t));
    int64_t *roots2 = (int64_t *)malloc((size_t)((uint64_t)ns + na + 1) * sizeof(int64_t));
    int64_t *roots3 = (int64_t *)malloc((size_t)(na + 1) * sizeof(int64_t));
    uint8_t *state = (uint8_t *)calloc((size_t)ns + 1, 1);
    uint64_t *ver = (uint64_t *)calloc((size_t)ns + 1, sizeof(uint64_t));
    float *key = (float *)malloc(((size_t)ns + 1) * sizeof(float));
    /* saddles adjacent to each maximum (reverse of the arcs), and the members
     * of every survivor's set as linked lists */
    uint64_t *inc_ptr = (uint64_t *)calloc((size_t)nm + 2, sizeof(uint64_t));
    int64_t *inc = (int64_t *)malloc((size_t)(na + 1) * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((size_t)(nm + 1) * sizeof(int64_t));
    int64_t *last = (int64_t *)malloc((size_t)(nm + 1) * sizeof(int64_t));
    int64_t *size = (int64_t *)malloc((size_t)(nm + 1) * sizeof(int64_t));
    uint64_t *seen = (uint64_t *)calloc((size_t)ns + 1, sizeof(uint64_t));
    ec_heap H = {NULL, 0, 0};
    int st = EC_OK;
    if (!end || !parent || !roots || !roots2 || !roots3 || !state || !ver || !key || !inc_ptr || !inc || !next || !last ||
        !size || !seen) {
        st = EC_ERR_OOM;
        goto out;
    }
    /* arc ends as maximum indices (the maxima are sorted by id) */
    for (uint64_t a = 0; a < na; a++) {
        int64_t lo = 0, hi = nm - 1, at = -1;
        while (lo <= hi) {
            int64_t mid = (lo + hi) / 2;
            if (maxima[mid] == col[a]) {
                at = mid;
                break;
            }
            if (maxima[mid] < col[a]) lo = mid + 1;
            else hi = mid - 1;
        }
        if (at < 0) {
            st = EC_ERR_ARG; /* an arc end that is not a maximum */
            goto out;
        }
        end[a] = at;
    }
    G.end = end;
    for (int64_t m = 0; m < nm; m++) {
        parent[m] = m;
        next[m] = -1;
        last[m] = m;
        size[m] = 1;
    }
    for (uint64_t a = 0; a < na; a++) inc_ptr[end[a] + 1]++;
    for (int64_t m = 0; m < nm; m++) inc_ptr[m + 1] += inc_ptr[m];
    {
        uint64_t *fill = (uint64_t *)malloc(((size_t)nm + 1) * sizeof(uint64_t));
        if (!fill) {
            st = EC_ERR_OOM;
            goto out;
        }
        memcpy(fill, inc_ptr, ((size_t)nm + 1) * sizeof(uint64_t));
        for (int64_t s = 0; s < ns; s++)
            for (uint64_t a = row_ptr[s]; a < row_ptr[s + 1]; a++) inc[fill[end[a]]++] = s;
        free(fill);
    }

    /* step 1: every saddle enters the queue with its initial cost (a saddle
     * without two maxima enters last, R1) */
    for (int64_t s = 0; s < ns; s++) {
        int64_t h1;
        float c = INFINITY;
        if (ec_adjacent(&G, parent, s, roots, &h1, &c) < 2) c = INFINITY;
        key[s] = c;
        ec_entry x = {c, saddles[s], s, 0};
        if ((st = ec_push(&H, x)) != EC_OK) goto out;
    }

    /* steps 2-3 */
    int64_t cancelled = 0;
    uint64_t stamp = 0;
    while (H.n > 0) {
        ec_entry t = ec_pop(&H);
        if (t.ver != ver[t.s] || state[t.s] != EC_WAITING) continue; /* stale (R5) */
        int64_t s = t.s, h1;
        float c = 0.0f;
        int64_t nr = ec_adjacent(&G, parent, s, roots, &h1, &c);
        if (nr < 2 || c > tau) { /* no second maximum (R1), or above the threshold */
            state[s] = EC_DISCARDED;
            continue;
        }
        /* the new top of the queue (stale entries dropped first) */
        while (H.n > 0 && (H.e[0].ver != ver[H.e[0].s] || state[H.e[0].s] != EC_WAITING)) ec_pop(&H);
        ec_entry me = {c, saddles[s], s, 0};
        if (H.n > 0 && ec_less(&H.e[0], &me)) { /* above the top (R4): reinsert */
            key[s] = c;
            me.ver = ++ver[s];
            if ((st = ec_push(&H, me)) != EC_OK) goto out;
            continue;
        }
        /* cancel: merge every adjacent maximum but the highest into it */
        state[s] = EC_CANCELLED;
        cancelled++;
        for (int64_t k = 0; k < nr; k++) {
            int64_t r = roots[k];
            if (r == h1) continue;
            /* saddles adjacent to both r and h1 may now have a lower cost
             * (R5): visit the saddles of the smaller of the two sets */
            int64_t small = size[r] <= size[h1] ? r : h1;
            stamp++;
            int64_t nv = 0;
            for (int64_t m = small; m >= 0; m = next[m])
                for (uint64_t q = inc_ptr[m]; q < inc_ptr[m + 1]; q++) {
                    int64_t x = inc[q];
                    if (seen[x] == stamp || state[x] == EC_CANCELLED) continue;
                    seen[x] = stamp;
                    roots2[nv++] = x;
                }
            parent[r] = h1;
            next[last[h1]] = r;
            last[h1] = last[r];
            size[h1] += size[r];
            for (int64_t q = 0; q < nv; q++) {
                int64_t x = roots2[q], hx;
                float cx = 0.0f;
                int64_t nx = ec_adjacent(&G, parent, x, roots3, &hx, &cx);
                if (nx < 2) continue;
                int lower = cx < key[x];
                int revive = state[x] == EC_DISCARDED && cx <= tau;
                if ((state[x] == EC_WAITING && lower) || revive) {
                    state[x] = EC_WAITING;
                    key[x] = cx;
                    ec_entry y = {cx, saddles[x], x, ++ver[x]};
                    if ((st = ec_push(&H, y)) != EC_OK) goto out;
                }
            }
        }
    }
    for (int64_t s = 0; s < ns; s++) alive[s] = state[s] != EC_CANCELLED;
    for (int64_t m = 0; m < nm; m++) survivor[m] = maxima[ec_find(parent, m)];
    if (n_cancelled) *n_cancelled = cancelled;
out:
    free(end);
    free(parent);
    free(roots);
    free(roots2);
    free(roots3);
    free(state);
    free(ver);
    free(key);
    free(inc_ptr);
    free(inc);
    free(next);
    free(last);
    free(size);
    free(seen);
    free(H.e);
    return st;
}
