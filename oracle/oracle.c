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
 *     rounded after every arc, left to right);
 *   - int32: exact integer addition.
 * A sum the type cannot hold (fp32: rounds to +inf; int32: >= INT32_MAX, the
 * value that marks "unreachable") is an overflow: when one arc out of a reached
 * vertex overflows at the fixed point, every solver returns OR_EOVERFLOW and
 * writes nothing (reading R14).
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
 *   R6 the set form takes the smallest non-empty bucket next (Section III-C);
 *   R14 overflow of a path sum is an error, not "unreachable" (see above).
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
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ECYCLE = 3, OR_EOVERFLOW = 4 };

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
        if (r >= 2147483647.0) return INFINITY;   /* overflow (R14) */
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

/* Overflow (reading R14; the paper assumes exact reals, Section III): a solve
 * is undefined when, at the fixed point, some arc (u,v) out of a reached u has
 * a sum dist[u] (+) w(u,v) that the weight type cannot hold (int32: >= INT32_MAX;
 * fp32: rounds to +inf). The condition uses final distances only, so it does
 * not depend on the relaxation order. Every solver checks it before writing
 * any output and then returns OR_EOVERFLOW with the outputs untouched. */
static int overflows(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                     int dtype, const double *t) {
    for (int64_t u = 0; u < n; ++u) {
        if (isinf(t[u])) continue;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (isinf(oplus(dtype, t[u], weight_at(dtype, w, e)))) return 1;
    }
    (void)col;
    return 0;
}

/* the end of every solver: the overflow check, then dist and pred */
static int finish(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                  int dtype, int32_t src, const double *t, void *dist_out, int32_t *pred_out) {
    if (overflows(n, row_ptr, col, w, dtype, t)) return OR_EOVERFLOW;
    write_dist(dtype, t, n, dist_out);
    pred_from_dist(n, row_ptr, col, w, dtype, src, t, pred_out);
    return OR_OK;
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
    rc = finish(n, row_ptr, col, w, dtype, src, t, dist_out, pred_out);
    free(t); free(done); free(h);
    return rc;
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
    rc = finish(n, row_ptr, col, w, dtype, src, t, dist_out, pred_out);
    free(t);
    return rc;
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
    rc = finish(n, row_ptr, col, w, dtype, src, st.tent, dist_out, pred_out);
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
    rc = finish(n, row_ptr, col, w, dtype, src, t, dist_out, pred_out);
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
/*   (e) unreached v (dist = INF) has pred -1;                                */
/*   (f) every reached v is realised: a walk from s along tight arcs (arcs    */
/*       with dist[u] (+) w == dist[v]) reaches it. With (a) this pins the     */
/*       least fixed point: (f) gives dist[v] = the rounded sum of one walk,   */
/*       (a) and the monotonicity of (+) give dist[v] <= every walk's sum.     */
/*       Without (f) a labelling that is too small on a cycle of zero-effect  */
/*       arcs (w = 0, or an fp32 w absorbed by a large dist) would pass (a)-(e);*/
/*   (g) following pred from a reached v reaches s, or ends in a cycle whose  */
/*       vertices all have the same distance (a tie the smallest-id rule can  */
/*       close through zero-effect arcs; legal only together with (f)); a     */
/*       chain that leaves the reached set or runs longer than n is counted.  */

int64_t or_check_invariants(int64_t n, const int64_t *row_ptr, const int32_t *col,
                            const void *w, int dtype, int32_t src, const void *dist,
                            const int32_t *pred) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    int64_t bad = 0;
    double *t = (double *)malloc((size_t)n * sizeof(double));
    int32_t *best = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *state = (uint8_t *)calloc((size_t)n, 1);
    if (!t || !best || !queue || !state) { free(t); free(best); free(queue); free(state); return -1; }
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
    /* (f) breadth-first search from s over tight arcs (state 1 = visited) */
    if (t[src] == 0.0) {
        int64_t head = 0, tail = 0;
        queue[tail++] = src;
        state[src] = 1;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                int32_t v = col[e];
                if (state[v]) continue;
                double c = oplus(dtype, t[u], weight_at(dtype, w, e));
                if (!isinf(c) && c == t[v]) { state[v] = 1; queue[tail++] = v; }
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) if (!isinf(t[v]) && !state[v]) ++bad;
    /* (g) pred walks. state: 0/1 not yet classified, 2 on the current walk,
       3 reaches s, 4 ends in an equal-distance cycle, 5 broken chain */
    for (int64_t v = 0; v < n; ++v) if (state[v] == 1) state[v] = 0;
    state[src] = 3;
    for (int64_t v0 = 0; v0 < n; ++v0) {
        if (isinf(t[v0]) || state[v0] >= 3) continue;
        int64_t len = 0;
        int32_t x = (int32_t)v0;
        uint8_t verdict = 5;
        for (;;) {
            if (state[x] >= 3) { verdict = state[x]; break; }
            if (state[x] == 2) {                  /* a cycle closes at x: equal distances? */
                verdict = 4;
                int32_t y = x;
                int64_t k = 0;
                do {
                    int32_t py = pred[y];
                    if (t[py] != t[y]) verdict = 5;
                    y = py;
                } while (y != x && ++k <= n);
                break;
            }
            state[x] = 2;
            queue[len++] = x;
            int32_t px = pred[x];
            if (px < 0 || px >= n || isinf(t[px]) || len > n) { verdict = 5; break; }
            x = px;
        }
        for (int64_t k = 0; k < len; ++k) state[queue[k]] = verdict;
        if (verdict == 5) bad += len;
    }
    free(t); free(best); free(queue); free(state);
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
/* The tree arc of v (reading R11) is, among all arcs (u,v) whose sum        */
/* dist[u] (+) w reaches dist[v], the one with the smallest input index.     */
/* Input arcs are stored row by row, so its tail is the smallest such u,     */
/* which is pred[v]; between parallel arcs of that row the earlier one wins. */
/* (At such a tie L has a kink -- the two arcs' one-sided derivatives        */
/* differ -- and this picks one subgradient by a rule of the input alone.)   */
/* Subtree sums are accumulated in double by an explicit post-order walk.    */
/* grad (m entries) is ADDED to. Returns 3 when the predecessor graph has a   */
/* cycle (zero-weight ties), where the gradient is undefined.                 */

int or_tree_gradient(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w,
                     int32_t src, const float *dist, const int32_t *pred,
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
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {        /* first in input order */
            if (col[e] == v && oplus(OR_F32, (double)dist[u], (double)w[e]) == (double)dist[v]) { tree[v] = e; break; }
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

/* ------------------------------------------------------------------------ */
/* Central differences of the loss in float64: a check of the gradient, not  */
/* a step of the method. For one source and float32 weights w (read as exact */
/* doubles, summed in double), L(w) = sum over reached x of c[x] * D[x] with  */
/* D the float64 shortest-path distances. For every listed arc e,            */
/*   fd = (L(w + eps 1_e) - L(w - eps 1_e)) / (2 eps),                        */
/* with D recomputed only where it can change:                               */
/*  - lowering w_e, e = (u,v), can only lower distances reached through e: a  */
/*    Dijkstra seeded at v with D[u] + w_e - eps finds them;                  */
/*  - raising w_e changes nothing unless e is v's tree arc; then exactly the  */
/*    tree below v may rise: its vertices are solved again from their in-arcs */
/*    out of the rest of the graph (whose distances stay), inside the subtree. */
/* The tree arc of v is the smallest input index among arcs whose float64 sum */
/* equals D[v]. L is piecewise linear in w_e; kink[j] = 1 when some vertex's   */
/* distance is not linear on [w_e - eps, w_e + eps] (it moves by a different  */
/* amount on the two sides), where fd is not the derivative; kink[j] = 2 when */
/* w_e < eps (not tested). The reverse CSR (rrow, rtail, rarc: in-arcs of     */
/* every vertex, their tails and input indices) is passed in.                */

typedef struct {
    int64_t n;
    const int64_t *rp; const int32_t *col; const double *w;
    const int64_t *rrp; const int32_t *rtail; const int64_t *rarc;
    double *D;            /* float64 distances at w                          */
    int64_t *tree;        /* tree arc of every reached v != src, else -1     */
    int64_t *kp;          /* children of every vertex in the tree (CSR)       */
    int32_t *kids;
    double *Dn;           /* perturbed distances of the touched vertices      */
    uint8_t *mark;        /* 1 touched, 2 in the re-solved subtree            */
    int32_t *touched; int64_t nt;
    heap_item *h; int64_t hcap;
    int32_t *stack;
    double *dplus;        /* per-vertex rise under +eps (0 when untouched)     */
    int32_t *plist; int64_t np;
} fd_state;

static void fd_touch(fd_state *s, int32_t x, uint8_t how) {
    if (!s->mark[x]) { s->touched[s->nt++] = x; s->Dn[x] = s->D[x]; }
    s->mark[x] = how;
}

static void fd_reset(fd_state *s) {
    for (int64_t k = 0; k < s->nt; ++k) s->mark[s->touched[k]] = 0;
    s->nt = 0;
}

/* lower w_e to wnew: Dn on the touched vertices */
static void fd_lower(fd_state *s, int64_t e, int32_t u, int32_t v, double wnew) {
    if (isinf(s->D[u])) return;
    double cand = s->D[u] + wnew;
    if (!(cand < s->D[v])) return;
    int64_t sz = 0;
    fd_touch(s, v, 1);
    s->Dn[v] = cand;
    heap_push(s->h, &sz, (heap_item){cand, v});
    while (sz > 0) {
        heap_item it = heap_pop(s->h, &sz);
        int32_t x = it.v;
        if (it.key != s->Dn[x]) continue;
        for (int64_t a = s->rp[x]; a < s->rp[x + 1]; ++a) {
            int32_t y = s->col[a];
            double c = s->Dn[x] + (a == e ? wnew : s->w[a]);
            double cur = s->mark[y] ? s->Dn[y] : s->D[y];
            if (c < cur) {
                fd_touch(s, y, 1);
                s->Dn[y] = c;
                if (sz < s->hcap) heap_push(s->h, &sz, (heap_item){c, y});
            }
        }
    }
}

/* raise w_e to wnew: Dn on the subtree below v when e is v's tree arc */
static void fd_raise(fd_state *s, int64_t e, int32_t v, double wnew) {
    if (s->tree[v] != e) return;
    int64_t top = 0, first = s->nt;
    s->stack[top++] = v;
    while (top > 0) {                                  /* the subtree, marked 2 */
        int32_t x = s->stack[--top];
        fd_touch(s, x, 2);
        s->Dn[x] = INFINITY;
        for (int64_t k = s->kp[x]; k < s->kp[x + 1]; ++k) s->stack[top++] = s->kids[k];
    }
    int64_t sz = 0;
    for (int64_t k = first; k < s->nt; ++k) {          /* entries from outside */
        int32_t x = s->touched[k];
        for (int64_t r = s->rrp[x]; r < s->rrp[x + 1]; ++r) {
            int32_t y = s->rtail[r];
            if (s->mark[y] == 2 || isinf(s->D[y])) continue;
            int64_t a = s->rarc[r];
            double c = s->D[y] + (a == e ? wnew : s->w[a]);
            if (c < s->Dn[x]) s->Dn[x] = c;
        }
        if (!isinf(s->Dn[x])) heap_push(s->h, &sz, (heap_item){s->Dn[x], x});
    }
    while (sz > 0) {                                   /* Dijkstra inside the subtree */
        heap_item it = heap_pop(s->h, &sz);
        int32_t x = it.v;
        if (it.key != s->Dn[x]) continue;
        for (int64_t a = s->rp[x]; a < s->rp[x + 1]; ++a) {
            int32_t y = s->col[a];
            if (s->mark[y] != 2) continue;
            double c = s->Dn[x] + (a == e ? wnew : s->w[a]);
            if (c < s->Dn[y]) {
                s->Dn[y] = c;
                if (sz < s->hcap) heap_push(s->h, &sz, (heap_item){c, y});
            }
        }
    }
}

int or_fd_arcs(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *wf,
               const int64_t *rrow, const int32_t *rtail, const int64_t *rarc,
               int32_t src, const float *c, const int64_t *arcs, int64_t k, double eps,
               double *fd, int32_t *kink) {
    if (n <= 0 || src < 0 || src >= n || !(eps > 0.0)) return OR_EINVAL;
    const int64_t m = row_ptr[n];
    fd_state s;
    memset(&s, 0, sizeof s);
    s.n = n; s.rp = row_ptr; s.col = col; s.rrp = rrow; s.rtail = rtail; s.rarc = rarc;
    double *w = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
    int32_t *tail = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    s.D = (double *)malloc((size_t)n * sizeof(double));
    s.tree = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    s.kp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    s.kids = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    s.Dn = (double *)malloc((size_t)n * sizeof(double));
    s.mark = (uint8_t *)calloc((size_t)n, 1);
    s.touched = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    s.hcap = m + n + 1;
    s.h = (heap_item *)malloc((size_t)s.hcap * sizeof(heap_item));
    s.stack = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    s.dplus = (double *)calloc((size_t)n, sizeof(double));
    s.plist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    int64_t *next = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int rc = OR_OK;
    if (!w || !tail || !s.D || !s.tree || !s.kp || !s.kids || !s.Dn || !s.mark || !s.touched || !s.h ||
        !s.stack || !s.dplus || !s.plist || !done || !next) { rc = OR_ENOMEM; goto out; }
    for (int64_t e = 0; e < m; ++e) w[e] = (double)wf[e];
    for (int64_t u = 0; u < n; ++u) for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tail[e] = (int32_t)u;
    s.w = w;
    /* float64 Dijkstra */
    for (int64_t v = 0; v < n; ++v) { s.D[v] = INFINITY; s.tree[v] = -1; }
    s.D[src] = 0.0;
    {
        int64_t sz = 0;
        heap_push(s.h, &sz, (heap_item){0.0, src});
        while (sz > 0) {
            heap_item it = heap_pop(s.h, &sz);
            int32_t u = it.v;
            if (done[u] || it.key != s.D[u]) continue;
            done[u] = 1;
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                double cnd = s.D[u] + w[e];
                if (cnd < s.D[col[e]]) { s.D[col[e]] = cnd; heap_push(s.h, &sz, (heap_item){cnd, col[e]}); }
            }
        }
    }
    /* tree arcs (smallest input index realising D[v]) and the children lists */
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = tail[e], v = col[e];
        if (v == src || isinf(s.D[u]) || s.tree[v] >= 0) continue;
        if (s.D[u] + w[e] == s.D[v]) s.tree[v] = e;
    }
    for (int64_t v = 0; v < n; ++v) if (s.tree[v] >= 0) s.kp[tail[s.tree[v]] + 1]++;
    for (int64_t v = 0; v < n; ++v) s.kp[v + 1] += s.kp[v];
    for (int64_t v = 0; v <= n; ++v) next[v] = s.kp[v];
    for (int64_t v = 0; v < n; ++v) if (s.tree[v] >= 0) s.kids[next[tail[s.tree[v]]]++] = (int32_t)v;
    for (int64_t j = 0; j < k; ++j) {
        int64_t e = arcs[j];
        fd[j] = 0.0;
        kink[j] = 0;
        if (e < 0 || e >= m) { rc = OR_EINVAL; goto out; }
        if (w[e] < eps) { kink[j] = 2; continue; }
        int32_t u = tail[e], v = col[e];
        double dl = 0.0;
        /* +eps */
        fd_raise(&s, e, v, w[e] + eps);
        s.np = 0;
        for (int64_t t = 0; t < s.nt; ++t) {
            int32_t x = s.touched[t];
            double d = s.Dn[x] - s.D[x];
            dl += (double)c[x] * d;
            s.dplus[x] = d;
            s.plist[s.np++] = x;
        }
        fd_reset(&s);
        /* -eps */
        fd_lower(&s, e, u, v, w[e] - eps);
        for (int64_t t = 0; t < s.nt; ++t) {
            int32_t x = s.touched[t];
            double d = s.D[x] - s.Dn[x];
            dl += (double)c[x] * d;
            if (fabs(d - s.dplus[x]) > 1e-9) kink[j] = 1;
            s.dplus[x] = INFINITY;                      /* compared */
        }
        for (int64_t t = 0; t < s.np; ++t) {             /* rose under +eps, unmoved under -eps */
            int32_t x = s.plist[t];
            if (!isinf(s.dplus[x]) && fabs(s.dplus[x]) > 1e-9) kink[j] = 1;
            s.dplus[x] = 0.0;
        }
        for (int64_t t = 0; t < s.nt; ++t) s.dplus[s.touched[t]] = 0.0;
        fd_reset(&s);
        fd[j] = dl / (2.0 * eps);
    }
out:
    free(w); free(tail); free(s.D); free(s.tree); free(s.kp); free(s.kids); free(s.Dn); free(s.mark);
    free(s.touched); free(s.h); free(s.stack); free(s.dplus); free(s.plist); free(done); free(next);
    return rc;
}
