/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for delta-stepping
 * single-source shortest paths (Sridhar et al., "Delta-stepping SSSP: from
 * Vertices and Edges to GraphBLAS Implementations", IPDPSW 2019).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this file:
 * only the test-suite, the package smoke check and the benchmark's CPU-baseline
 * leg load it. It shares no code, header, table or helper with the CUDA
 * library; it was written from the paper, not from the GPU kernels.
 *
 * What it computes. A directed graph G = (V, E) stored as CSR (row = out-arcs,
 * Section II-A), non-negative weights, one source s. Distances use the weight
 * type's own addition "(+)":
 *   - fp32: IEEE-754 binary32 addition, round-to-nearest-even (a path sum is
 *     rounded after every arc, left to right); an overflow gives +inf;
 *   - int32: exact integer addition saturated at INT32_MAX, which reads as
 *     "unreachable".
 * dist is the least fixed point of dist[s] = 0, dist[v] = min over arcs (u,v)
 * of dist[u] (+) w(u,v). Because (+) is monotone and x (+) w >= x for w >= 0,
 * every label-correcting order (Dijkstra, Bellman-Ford, delta-stepping for any
 * Delta -- the paper calls delta-stepping label-correcting, Section III) reaches
 * the same bits.
 * pred[v] = the smallest u with an arc (u,v), dist[u] finite and
 * dist[u] (+) w(u,v) == dist[v]; pred[s] = s; pred = -1 when unreached.
 *
 * Readings of the paper taken here (each repeated at its point of use):
 *   R1 zero-weight arcs are light (Section III-A: light means weight <= Delta;
 *      Fig. 1's "0 < A" marks a stored entry);
 *   R2 the outer loop of Fig. 1 (left) runs while some FINITE t is >= i*Delta;
 *   R3 "s = 0" inside the loop of Fig. 1 (left) empties the set S;
 *   R4 bucket(x) = floor(x / Delta) evaluated exactly;
 *   R5 a heavy relaxation whose rounded sum lands back in the current bucket
 *      re-opens that bucket (impossible in exact arithmetic; fp32 can do it);
 *   R6 the set form takes the smallest non-empty bucket next (Section III-C).
 *
 * Parity pins: see the test-suite (brute-force walk enumeration, Floyd-Warshall
 * on integer weights, BFS and Manhattan closed forms, prefix sums on paths,
 * SciPy's Dijkstra on integer weights, a hand-traced bucket schedule).
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math (no FMA contraction, no x87).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_I32 = 0, OR_F32 = 1 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

/* ------------------------------------------------------------------------ */
/* values: a distance is held as a double that stores an exact fp32 or int32 */
/* value (or +inf), so every comparison below is exact.                      */

static double weight_at(int dtype, const void *w, int64_t e) {
    if (dtype == OR_F32) return (double)((const float *)w)[e];
    return (double)((const int32_t *)w)[e];
}

/* d (+) w : the weight type's own addition (see file header) */
static double oplus(int dtype, double d, double w) {
    if (isinf(d)) return INFINITY;
    if (dtype == OR_F32) {
        volatile float a = (float)d, b = (float)w;
        volatile float r = a + b;           /* one binary32 rounding */
        return (double)r;
    } else {
        double r = d + w;                   /* exact: |values| < 2^53 */
        if (r >= 2147483647.0) return INFINITY;
        return r;
    }
}

static void write_dist(int dtype, const double *t, int64_t n, void *dist_out) {
    for (int64_t v = 0; v < n; ++v) {
        if (dtype == OR_F32) ((float *)dist_out)[v] = isinf(t[v]) ? INFINITY : (float)t[v];
        else ((int32_t *)dist_out)[v] = isinf(t[v]) ? INT32_MAX : (int32_t)t[v];
    }
}

/* pred from final distances, by the definition in the file header */
static void pred_from_dist(int64_t n, const int64_t *row_ptr, const int32_t *col,
                           const void *w, int dtype, int32_t src, const double *t,
                           int32_t *pred) {
    for (int64_t v = 0; v < n; ++v) pred[v] = -1;
    for (int64_t u = 0; u < n; ++u) {
        if (isinf(t[u])) continue;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            double c = oplus(dtype, t[u], weight_at(dtype, w, e));
            if (!isinf(c) && c == t[v] && (pred[v] < 0 || (int32_t)u < pred[v])) pred[v] = (int32_t)u;
        }
    }
    pred[src] = src;
}

static int check_args(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                      int dtype, int32_t src) {
    if (n <= 0 || src < 0 || src >= n || (dtype != OR_I32 && dtype != OR_F32)) return OR_EINVAL;
    if (row_ptr[0] != 0) return OR_EINVAL;
    for (int64_t u = 0; u < n; ++u) if (row_ptr[u + 1] < row_ptr[u]) return OR_EINVAL;
    for (int64_t e = 0; e < row_ptr[n]; ++e) {
        if (col[e] < 0 || col[e] >= n) return OR_EINVAL;
        double x = weight_at(dtype, w, e);
        if (!(x >= 0.0) || isinf(x)) return OR_EINVAL;     /* negative, NaN or inf */
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Dijkstra with a binary heap (lazy deletion). Computes the least fixed     */
/* point directly; the efficient reference for large inputs.                 */

typedef struct { double key; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *sz, heap_item x) {
    int64_t i = (*sz)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].key <= h[i].key) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, int64_t *sz) {
    heap_item top = h[0];
    h[0] = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *sz && h[l].key < h[s].key) s = l;
        if (r < *sz && h[r].key < h[s].key) s = r;
        if (s == i) break;
        heap_item t = h[s]; h[s] = h[i]; h[i] = t;
        i = s;
    }
    return top;
}

int or_dijkstra(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                int dtype, int32_t src, void *dist_out, int32_t *pred_out) {
    int rc = check_args(n, row_ptr, col, w, dtype, src);
    if (rc) return rc;
    int64_t m = row_ptr[n];
    double *t = (double *)malloc((size_t)n * sizeof(double));
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    heap_item *h = (heap_item *)malloc((size_t)(m + 1) * sizeof(heap_item));
    if (!t || !done || !h) { free(t); free(done); free(h); return OR_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) t[v] = INFINITY;
    t[src] = 0.0;
    int64_t sz = 0;
    heap_push(h, &sz, (heap_item){0.0, src});
    while (sz > 0) {
        heap_item it = heap_pop(h, &sz);
        int32_t u = it.v;
        if (done[u] || it.key != t[u]) continue;
        done[u] = 1;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            double c = oplus(dtype, t[u], weight_at(dtype, w, e));
            if (c < t[v]) { t[v] = c; heap_push(h, &sz, (heap_item){c, v}); }
        }
    }
    write_dist(dtype, t, n, dist_out);
    pred_from_dist(n, row_ptr, col, w, dtype, src, t, pred_out);
    free(t); free(done); free(h);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Bellman-Ford: sweep every arc until nothing changes -- the fixed-point    */
/* definition written out (at most n sweeps).                                */

int or_bellman_ford(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                    int dtype, int32_t src, void *dist_out, int32_t *pred_out) {
    int rc = check_args(n, row_ptr, col, w, dtype, src);
    if (rc) return rc;
    double *t = (double *)malloc((size_t)n * sizeof(double));
    if (!t) return OR_ENOMEM;
    for (int64_t v = 0; v < n; ++v) t[v] = INFINITY;
    t[src] = 0.0;
    for (int64_t sweep = 0; sweep <= n; ++sweep) {
        int changed = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (isinf(t[u])) continue;
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                double c = oplus(dtype, t[u], weight_at(dtype, w, e));
                if (c < t[col[e]]) { t[col[e]] = c; changed = 1; }
            }
        }
        if (!changed) break;
    }
    write_dist(dtype, t, n, dist_out);
    pred_from_dist(n, row_ptr, col, w, dtype, src, t, pred_out);
    free(t);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Floyd-Warshall on int32 weights (exact integer sums only: with rounding   */
/* the segment-wise association of FW differs from left-to-right path sums). */
/* dist_all is n*n row-major, INT32_MAX = no path.                           */

int or_floyd_warshall_i32(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const int32_t *w, int32_t *dist_all) {
    if (n <= 0 || n > 4096) return OR_EINVAL;
    int64_t *d = (int64_t *)malloc((size_t)(n * n) * sizeof(int64_t));
    if (!d) return OR_ENOMEM;
    const int64_t BIG = INT64_MAX / 4;
    for (int64_t i = 0; i < n * n; ++i) d[i] = BIG;
    for (int64_t i = 0; i < n; ++i) d[i * n + i] = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (w[e] < d[u * n + col[e]]) d[u * n + col[e]] = w[e];
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                if (d[i * n + k] + d[k * n + j] < d[i * n + j]) d[i * n + j] = d[i * n + k] + d[k * n + j];
    for (int64_t i = 0; i < n * n; ++i) dist_all[i] = d[i] >= INT32_MAX ? INT32_MAX : (int32_t)d[i];
    free(d);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Buckets. Section III-B: B_i = { v : i*Delta <= tent(v) < (i+1)*Delta }.    */
/* Reading R4: bucket(x) = floor(x/Delta) evaluated exactly. The quotient is  */
/* computed in double, then corrected with exact fma() sign tests, because a  */
/* rounded quotient can land on the integer just above the true one.         */

int64_t or_bucket_index(double x, double delta) {
    if (isinf(delta)) return 0;                 /* Delta = inf: a single bucket */
    double q = floor(x / delta);
    if (q >= 9007199254740992.0)                 /* beyond 2^53: no exact correction needed */
        return q >= 9.2e18 ? INT64_MAX : (int64_t)q;
    /* the correctly rounded quotient is off by at most one */
    if (q > 0.0 && fma(q, delta, -x) > 0.0) q -= 1.0;           /* q*Delta > x      */
    else if (fma(q + 1.0, delta, -x) <= 0.0) q += 1.0;          /* (q+1)*Delta <= x */
    return (int64_t)q;
}

/* i*Delta <= x < (i+1)*Delta, exactly */
static int in_bucket(double x, double delta, int64_t i) {
    if (isinf(x)) return 0;
    return or_bucket_index(x, delta) == i;
}

/* light(v) = arcs with weight <= Delta (Section III-A; reading R1: zero is light) */
static int is_light(double wv, double delta) { return wv <= delta; }

/* ------------------------------------------------------------------------ */
/* Trace records, used by the tests to compare the two delta-stepping forms  */
/* with each other and with a hand-traced example. One record per vertex     */
/* processed: (bucket i, inner round k >= 0 for a light phase, or -1 - r for  */
/* the r-th heavy phase of that bucket, vertex).                             */

typedef struct { int64_t bucket; int64_t round; int64_t vertex; } or_trace_rec;

typedef struct {
    or_trace_rec *rec;
    int64_t cap, len;
    int64_t overflow;
} trace_buf;

static void trace_add(trace_buf *tb, int64_t b, int64_t k, int64_t v) {
    if (!tb || !tb->rec) return;
    if (tb->len < tb->cap) tb->rec[tb->len] = (or_trace_rec){b, k, v};
    else tb->overflow = 1;
    tb->len++;
}

/* ------------------------------------------------------------------------ */
/* Delta-stepping, vertex/edge ("Meyer & Sanders") set form: Fig. 1 right    */
/* column and Section III. Buckets are explicit sets; relax() moves a vertex  */
/* between them; requests of one phase are generated from the bucket first,  */
/* then applied (Section III-C: "simultaneously process all light edges").    */
/* Bucket B_j is stored as the vertices v with bucket_of[v] == j; a min-heap   */
/* of (j, v) entries finds the smallest non-empty bucket (reading R6), stale  */
/* entries (bucket_of[v] != j) are skipped.                                   */

typedef struct { int64_t b; int32_t v; } bentry;

typedef struct {
    bentry *h;
    int64_t sz, cap;
} bheap;

static int bh_push(bheap *q, int64_t b, int32_t v) {
    if (q->sz == q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 1024;
        bentry *nh = (bentry *)realloc(q->h, (size_t)nc * sizeof(bentry));
        if (!nh) return OR_ENOMEM;
        q->h = nh; q->cap = nc;
    }
    int64_t i = q->sz++;
    q->h[i] = (bentry){b, v};
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (q->h[p].b <= q->h[i].b) break;
        bentry t = q->h[p]; q->h[p] = q->h[i]; q->h[i] = t;
        i = p;
    }
    return OR_OK;
}

static bentry bh_pop(bheap *q) {
    bentry top = q->h[0];
    q->h[0] = q->h[--q->sz];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < q->sz && q->h[l].b < q->h[s].b) s = l;
        if (r < q->sz && q->h[r].b < q->h[s].b) s = r;
        if (s == i) break;
        bentry t = q->h[s]; q->h[s] = q->h[i]; q->h[i] = t;
        i = s;
    }
    return top;
}

typedef struct { int32_t v; double x; } request;

typedef struct {
    double *tent;
    int64_t *bucket_of;   /* -1: in no bucket */
    bheap heap;
    double delta;
} ms_state;

/* procedure relax(v, new_dist) -- Section III-C / Fig. 1 right */
static int ms_relax(ms_state *st, int32_t v, double x) {
    if (x < st->tent[v]) {
        int64_t nb = or_bucket_index(x, st->delta);
        /* B_old = B_old - {v}: implicit, bucket_of[v] changes below */
        st->bucket_of[v] = nb;                          /* B_new = B_new + {v} */
        st->tent[v] = x;                                /* tent(v) = new_dist  */
        return bh_push(&st->heap, nb, v);
    }
    return OR_OK;
}

int or_delta_ms(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                int dtype, int32_t src, double delta, void *dist_out, int32_t *pred_out,
                or_trace_rec *trace, int64_t trace_cap, int64_t *trace_len) {
    int rc = check_args(n, row_ptr, col, w, dtype, src);
    if (rc) return rc;
    if (!(delta > 0.0)) return OR_EINVAL;
    int64_t m = row_ptr[n];
    ms_state st;
    memset(&st, 0, sizeof st);
    st.delta = delta;
    st.tent = (double *)malloc((size_t)n * sizeof(double));
    st.bucket_of = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *bi = (int32_t *)malloc((size_t)n * sizeof(int32_t));       /* members of B[i] */
    int32_t *S = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *inS = (uint8_t *)calloc((size_t)n, 1);
    request *req = (request *)malloc((size_t)(m + 1) * sizeof(request));
    trace_buf tb = {trace, trace_cap, 0, 0};
    if (!st.tent || !st.bucket_of || !bi || !S || !inS || !req) { rc = OR_ENOMEM; goto out; }

    for (int64_t v = 0; v < n; ++v) { st.tent[v] = INFINITY; st.bucket_of[v] = -1; }
    if ((rc = ms_relax(&st, src, 0.0))) goto out;                        /* relax(s, 0) */

    while (st.heap.sz > 0) {                                             /* while B not empty */
        /* smallest non-empty bucket (reading R6) */
        bentry top = st.heap.h[0];
        if (st.bucket_of[top.v] != top.b) { bh_pop(&st.heap); continue; }   /* stale entry */
        int64_t i = top.b;
        int64_t nS = 0;                                                  /* S = {} */
        int64_t heavy_rounds = 0;
        for (;;) {
            int64_t round = 0;
            for (;;) {                                                   /* while B[i] not empty */
                int64_t nb = 0;
                while (st.heap.sz > 0 && st.heap.h[0].b <= i) {
                    bentry x = bh_pop(&st.heap);
                    if (st.bucket_of[x.v] == i) { st.bucket_of[x.v] = -1; bi[nb++] = x.v; }
                }
                if (nb == 0) break;
                /* Req = {(w, tent(v) + c(v,w)) : v in B[i], (v,w) light} */
                int64_t nreq = 0;
                for (int64_t k = 0; k < nb; ++k) {
                    int32_t v = bi[k];
                    trace_add(&tb, i, round, v);
                    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                        double wv = weight_at(dtype, w, e);
                        if (is_light(wv, delta)) req[nreq++] = (request){col[e], oplus(dtype, st.tent[v], wv)};
                    }
                }
                /* S = S u B[i]; B[i] = {} (already emptied above) */
                for (int64_t k = 0; k < nb; ++k) if (!inS[bi[k]]) { inS[bi[k]] = 1; S[nS++] = bi[k]; }
                /* foreach (v, x) in Req: relax(v, x) */
                for (int64_t k = 0; k < nreq; ++k) if ((rc = ms_relax(&st, req[k].v, req[k].x))) goto out;
                ++round;
            }
            /* Req = {(w, tent(v) + c(v,w)) : v in S, (v,w) heavy}; relax each */
            int64_t nreq = 0;
            for (int64_t k = 0; k < nS; ++k) {
                int32_t v = S[k];
                trace_add(&tb, i, -1 - heavy_rounds, v);
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                    double wv = weight_at(dtype, w, e);
                    if (!is_light(wv, delta)) req[nreq++] = (request){col[e], oplus(dtype, st.tent[v], wv)};
                }
            }
            for (int64_t k = 0; k < nS; ++k) inS[S[k]] = 0;
            nS = 0;
            for (int64_t k = 0; k < nreq; ++k) if ((rc = ms_relax(&st, req[k].v, req[k].x))) goto out;
            ++heavy_rounds;
            /* reading R5: a rounded heavy sum may land back in B[i]; process it */
            int reopened = 0;
            while (st.heap.sz > 0) {
                bentry x = st.heap.h[0];
                if (st.bucket_of[x.v] != x.b) { bh_pop(&st.heap); continue; }
                reopened = (x.b <= i);
                break;
            }
            if (!reopened) break;
        }
    }
    {
        double *t = st.tent;
        write_dist(dtype, t, n, dist_out);
        pred_from_dist(n, row_ptr, col, w, dtype, src, t, pred_out);
    }
out:
    if (trace_len) *trace_len = tb.overflow ? -tb.len : tb.len;
    free(st.tent); free(st.bucket_of); free(st.heap.h); free(bi); free(S); free(inS); free(req);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Delta-stepping, linear-algebraic form: Fig. 1 left column, Section IV, on */
/* dense vectors. t, t_Req are |V| vectors with +inf for "no entry";          */
/* t_Bi and S are 0/1 vectors. The min-plus product A^T x is evaluated as the */
/* column-wise min of t[v] (+) a_v over rows v with x[v] present              */
/* (Section IV-C: Req_v = t[v] + a_v, then a min-reduction per column).       */

/* t_Req = A_sel^T (t o mask) over the (min,+) semiring; sel: 1 light, 0 heavy */
static void minplus_vxm(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                        int dtype, double delta, int light, const double *t,
                        const uint8_t *mask, double *t_req) {
    for (int64_t j = 0; j < n; ++j) t_req[j] = INFINITY;
    for (int64_t v = 0; v < n; ++v) {
        if (!mask[v] || isinf(t[v])) continue;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            double wv = weight_at(dtype, w, e);
            /* A_L = A o (0 <= A <= Delta) (reading R1), A_H = A o (A > Delta) */
            if (is_light(wv, delta) != light) continue;
            double x = oplus(dtype, t[v], wv);
            if (x < t_req[col[e]]) t_req[col[e]] = x;
        }
    }
}

int or_delta_la(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                int dtype, int32_t src, double delta, void *dist_out, int32_t *pred_out,
                or_trace_rec *trace, int64_t trace_cap, int64_t *trace_len) {
    int rc = check_args(n, row_ptr, col, w, dtype, src);
    if (rc) return rc;
    if (!(delta > 0.0)) return OR_EINVAL;
    double *t = (double *)malloc((size_t)n * sizeof(double));
    double *t_req = (double *)malloc((size_t)n * sizeof(double));
    uint8_t *t_b = (uint8_t *)malloc((size_t)n);
    uint8_t *S = (uint8_t *)malloc((size_t)n);
    trace_buf tb = {trace, trace_cap, 0, 0};
    if (!t || !t_req || !t_b || !S) { rc = OR_ENOMEM; goto out; }

    for (int64_t v = 0; v < n; ++v) t[v] = INFINITY;                     /* t = inf   */
    t[src] = 0.0;                                                        /* t[s] = 0  */
    int64_t i = 0;                                                       /* i = 0     */
    for (;;) {
        /* while (t >= i*Delta) != 0 -- reading R2: finite entries only */
        int64_t cnt = 0;
        for (int64_t v = 0; v < n; ++v)
            if (!isinf(t[v]) && or_bucket_index(t[v], delta) >= i) ++cnt;
        if (cnt == 0) break;
        memset(S, 0, (size_t)n);                                         /* s = 0 (R3) */
        for (int64_t v = 0; v < n; ++v) t_b[v] = (uint8_t)in_bucket(t[v], delta, i);
        int64_t heavy_rounds = 0;
        for (;;) {
            int64_t round = 0;
            for (;;) {                                                   /* while t_Bi != 0 */
                int any = 0;
                for (int64_t v = 0; v < n; ++v) if (t_b[v]) { any = 1; trace_add(&tb, i, round, v); }
                if (!any) break;
                /* t_Req = A_L^T (t o t_Bi) */
                minplus_vxm(n, row_ptr, col, w, dtype, delta, 1, t, t_b, t_req);
                /* S = ((S + t_Bi) > 0) */
                for (int64_t v = 0; v < n; ++v) S[v] = (uint8_t)((S[v] + t_b[v]) > 0);
                /* t_Bi = (i*Delta <= t_Req < (i+1)*Delta) o (t_Req < t) */
                for (int64_t v = 0; v < n; ++v)
                    t_b[v] = (uint8_t)(in_bucket(t_req[v], delta, i) && t_req[v] < t[v]);
                /* t = min(t, t_Req) */
                for (int64_t v = 0; v < n; ++v) if (t_req[v] < t[v]) t[v] = t_req[v];
                ++round;
            }
            /* t_Req = A_H^T (t o S) */
            for (int64_t v = 0; v < n; ++v) if (S[v]) trace_add(&tb, i, -1 - heavy_rounds, v);
            minplus_vxm(n, row_ptr, col, w, dtype, delta, 0, t, S, t_req);
            /* reading R5: heavy sums rounded back into bucket i re-open it */
            int reopen = 0;
            for (int64_t v = 0; v < n; ++v) {
                t_b[v] = (uint8_t)(in_bucket(t_req[v], delta, i) && t_req[v] < t[v]);
                reopen |= t_b[v];
            }
            /* t = min(t, t_Req) */
            for (int64_t v = 0; v < n; ++v) if (t_req[v] < t[v]) t[v] = t_req[v];
            ++heavy_rounds;
            if (!reopen) break;
            memset(S, 0, (size_t)n);
        }
        i = i + 1;                                                       /* i = i + 1 */
    }
    write_dist(dtype, t, n, dist_out);
    pred_from_dist(n, row_ptr, col, w, dtype, src, t, pred_out);
out:
    if (trace_len) *trace_len = tb.overflow ? -tb.len : tb.len;
    free(t); free(t_req); free(t_b); free(S);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Invariant checker. Counts violations of                                    */
/*   (a) dist[v] <= dist[u] (+) w for every arc (u,v) with u reached;        */
/*   (b) dist[pred[v]] (+) w(pred[v], v) == dist[v] for every reached v != s; */
/*   (c) pred[v] is the smallest such u;  (d) dist[s] == 0, pred[s] == s;     */
/*   (e) unreached v (dist = INF) has pred -1.                                */

int64_t or_check_invariants(int64_t n, const int64_t *row_ptr, const int32_t *col,
                            const void *w, int dtype, int32_t src, const void *dist,
                            const int32_t *pred) {
    int64_t bad = 0;
    double *t = (double *)malloc((size_t)n * sizeof(double));
    int32_t *best = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!t || !best) { free(t); free(best); return -1; }
    for (int64_t v = 0; v < n; ++v) {
        if (dtype == OR_F32) { float x = ((const float *)dist)[v]; t[v] = isinf(x) ? INFINITY : (double)x; }
        else { int32_t x = ((const int32_t *)dist)[v]; t[v] = x == INT32_MAX ? INFINITY : (double)x; }
        best[v] = -1;
    }
    if (t[src] != 0.0 || pred[src] != src) ++bad;                                   /* (d) */
    for (int64_t u = 0; u < n; ++u) {
        if (isinf(t[u])) continue;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            double c = oplus(dtype, t[u], weight_at(dtype, w, e));
            if (c < t[v]) ++bad;                                                       /* (a) */
            if (!isinf(c) && c == t[v] && (best[v] < 0 || (int32_t)u < best[v])) best[v] = (int32_t)u;
        }
    }
    for (int64_t v = 0; v < n; ++v) {
        if (v == src) continue;
        if (isinf(t[v])) { if (pred[v] != -1) ++bad; continue; }                     /* (e) */
        if (pred[v] < 0 || pred[v] >= n) { ++bad; continue; }
        if (best[v] != pred[v]) ++bad;                                               /* (b),(c) */
    }
    free(t); free(best);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Gradient of L = sum over reached v of c[v] * dist[v] with respect to the  */
/* weights (float32 graphs; the paper defines no gradient -- this is the     */
/* derivative of its distances). dist[v] is the (+)-sum of the weights on    */
/* v's shortest-path tree path from s, so raising the weight of v's tree arc */
/* by eps raises dist[x] by eps for every x in the subtree below v (as long  */
/* as the tree stays the same): dL/dw(tree arc of v) = sum of c over that     */
/* subtree, and 0 for arcs outside the tree.                                  */
/* The tree arc of v is an arc (pred[v], v) whose sum reaches dist[v]; among  */
/* parallel arcs that do, the first in pred[v]'s light-then-heavy order       */
/* (light: w <= Delta, Section III-A), input order within each group.         */
/* Subtree sums are accumulated in double by an explicit post-order walk.    */
/* grad (m entries) is ADDED to. Returns 3 when the predecessor graph has a   */
/* cycle (zero-weight ties), where the gradient is undefined.                 */

enum { OR_ECYCLE = 3 };

int or_tree_gradient(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w,
                     int32_t src, double delta, const float *dist, const int32_t *pred,
                     const float *c, double *grad) {
    if (n <= 0 || src < 0 || src >= n) return OR_EINVAL;
    int64_t *tree = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *head = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t *kids = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *stack = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *next = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    double *sum = (double *)malloc((size_t)n * sizeof(double));
    if (!tree || !head || !kids || !stack || !next || !sum) {
        free(tree); free(head); free(kids); free(stack); free(next); free(sum);
        return OR_ENOMEM;
    }
    int rc = OR_OK;
    int64_t reached = 0;
    /* tree arc of every reached v != src */
    for (int64_t v = 0; v < n; ++v) {
        tree[v] = -1;
        if (isinf(dist[v])) continue;
        ++reached;
        if (v == src) continue;
        int32_t u = pred[v];
        if (u < 0 || u >= n) { rc = OR_EINVAL; goto out; }
        for (int pass = 0; pass < 2 && tree[v] < 0; ++pass) {        /* light, then heavy */
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                if (col[e] != v) continue;
                int light = (double)w[e] <= delta;
                if ((pass == 0) != light) continue;
                if (oplus(OR_F32, (double)dist[u], (double)w[e]) == (double)dist[v]) { tree[v] = e; break; }
            }
        }
        if (tree[v] < 0) { rc = OR_EINVAL; goto out; }                /* pred does not realise dist */
    }
    /* children lists (counting sort by parent) */
    for (int64_t v = 0; v <= n; ++v) head[v] = 0;
    for (int64_t v = 0; v < n; ++v) if (tree[v] >= 0) head[pred[v] + 1]++;
    for (int64_t v = 0; v < n; ++v) head[v + 1] += head[v];
    for (int64_t v = 0; v < n; ++v) next[v] = head[v];
    for (int64_t v = 0; v < n; ++v) if (tree[v] >= 0) kids[next[pred[v]]++] = (int32_t)v;
    /* post-order from the source: a vertex is finished after all of its children */
    {
        int64_t top = 0, visited = 0;
        for (int64_t v = 0; v < n; ++v) { next[v] = head[v]; sum[v] = 0.0; }
        stack[top++] = src;
        while (top > 0) {
            int32_t v = stack[top - 1];
            if (next[v] < head[v + 1]) {
                stack[top++] = kids[next[v]++];
            } else {
                --top;
                ++visited;
                sum[v] += (double)c[v];
                if (v != src) {
                    sum[pred[v]] += sum[v];
                    grad[tree[v]] += sum[v];
                }
            }
        }
        if (visited != reached) rc = OR_ECYCLE;                         /* part of the tree hangs off a cycle */
    }
out:
    free(tree); free(head); free(kids); free(stack); free(next); free(sum);
    return rc;
}
