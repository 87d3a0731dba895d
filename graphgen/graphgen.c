/*
 * graphgen.c -- seeded synthetic graph generators (R-MAT, 2-D grid, Erdos-Renyi)
 * and edge-weight generators.
 *
 * This module produces INPUTS only. It contains none of the shortest-path
 * arithmetic: no relaxation, no bucket logic, no distance sums. Both the CPU
 * oracle tests and the CUDA path consume its output.
 *
 * Randomness is counter-based: every random number is a pure function of
 * (seed, stream, index) through the splitmix64 finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so
 * results are identical on any host and independent of thread count.
 *
 * Built as a plain C shared library with gcc (OpenMP loops; the output does not
 * depend on the thread count); loaded through ctypes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---- counter-based random numbers ------------------------------------- */

static inline uint64_t sm64_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* One 64-bit random word for (seed, stream, index). */
uint64_t gg_hash(uint64_t seed, uint64_t stream, uint64_t index) {
    uint64_t k = sm64_finalise(seed + 0x9E3779B97F4A7C15ULL * (stream + 1));
    return sm64_finalise(k + 0x9E3779B97F4A7C15ULL * (index + 1));
}

/* uniform double in [0,1) with 53 random bits */
static inline double u53(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

enum { ST_RMAT = 1, ST_PERM = 2, ST_WEIGHT = 3, ST_GRID_DROP = 4, ST_ER = 5, ST_LOGN = 6 };

/* ---- R-MAT ---------------------------------------------------------------
 * Chakrabarti, Zhan and Faloutsos, "R-MAT: a recursive model for graph
 * mining" (SDM 2004): each edge picks one quadrant of the adjacency matrix per
 * level with probabilities a, b, c, d = 1-a-b-c; level k fixes bit
 * (scale-1-k) of the source (row) and destination (column) ids.
 */
void gg_rmat_edges(int32_t scale, int64_t n_draws, double a, double b, double c,
                   uint64_t seed, int32_t *src, int32_t *dst) {
    const double ab = a + b, abc = a + b + c;
    const uint64_t skey = sm64_finalise(seed + 0x9E3779B97F4A7C15ULL * (ST_RMAT + 1));
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_draws; ++e) {
        /* one 64-bit word per edge and level pair; 32 random bits per level */
        uint64_t ekey = sm64_finalise(skey + 0x9E3779B97F4A7C15ULL * ((uint64_t)e + 1));
        uint32_t r = 0, q = 0;
        uint64_t word = 0;
        for (int32_t lev = 0; lev < scale; ++lev) {
            if ((lev & 1) == 0)
                word = sm64_finalise(ekey + 0x9E3779B97F4A7C15ULL * ((uint64_t)lev + 1));
            uint32_t bits32 = (lev & 1) ? (uint32_t)(word >> 32) : (uint32_t)word;
            double u = (double)bits32 * (1.0 / 4294967296.0);
            uint32_t rb, cb;
            if (u < a)        { rb = 0; cb = 0; }
            else if (u < ab)  { rb = 0; cb = 1; }
            else if (u < abc) { rb = 1; cb = 0; }
            else              { rb = 1; cb = 1; }
            r = (r << 1) | rb;
            q = (q << 1) | cb;
        }
        src[e] = (int32_t)r;
        dst[e] = (int32_t)q;
    }
}

/* Seeded uniform random permutation of 0..n-1 (Fisher-Yates, Knuth Vol. 2 3.4.2). */
void gg_permutation(int64_t n, uint64_t seed, int32_t *perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t h = gg_hash(seed, ST_PERM, (uint64_t)i);
        int64_t j = (int64_t)(h % (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Apply a vertex relabelling in place: x -> perm[x]. */
void gg_relabel(int64_t m, const int32_t *perm, int32_t *ids) {
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) ids[e] = perm[ids[e]];
}

/* ---- 2-D grid --------------------------------------------------------------
 * rows x cols lattice, vertex id r*cols + c, arcs to the 4 neighbours in both
 * directions; each directed arc is dropped independently with probability
 * drop_p. Returns the number of arcs written (src/dst sized 4*rows*cols).
 */
int64_t gg_grid_edges(int32_t rows, int32_t cols, double drop_p, uint64_t seed,
                      int32_t *src, int32_t *dst) {
    int64_t k = 0, arc = 0;
    static const int dr[4] = {-1, 1, 0, 0};
    static const int dc[4] = {0, 0, -1, 1};
    for (int32_t r = 0; r < rows; ++r)
        for (int32_t c = 0; c < cols; ++c)
            for (int d = 0; d < 4; ++d) {
                int32_t r2 = r + dr[d], c2 = c + dc[d];
                if (r2 < 0 || r2 >= rows || c2 < 0 || c2 >= cols) continue;
                uint64_t h = gg_hash(seed, ST_GRID_DROP, (uint64_t)arc++);
                if (u53(h) < drop_p) continue;
                src[k] = r * cols + c;
                dst[k] = r2 * cols + c2;
                ++k;
            }
    return k;
}

/* ---- Erdos-Renyi G(n, m) draws: m ordered pairs, uniform over n x n. ---- */
void gg_er_edges(int64_t n, int64_t m, uint64_t seed, int32_t *src, int32_t *dst) {
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint64_t h1 = gg_hash(seed, ST_ER, 2u * (uint64_t)e);
        uint64_t h2 = gg_hash(seed, ST_ER, 2u * (uint64_t)e + 1u);
        src[e] = (int32_t)(h1 % (uint64_t)n);
        dst[e] = (int32_t)(h2 % (uint64_t)n);
    }
}

/* ---- CSR assembly ----------------------------------------------------------
 * Two stable counting sorts (by destination, then by source) give the arcs in
 * (source, destination) order; self-loops and repeated arcs are dropped.
 * row_ptr has n+1 entries, col has room for m_raw entries. Returns m.
 */
int64_t gg_build_csr(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                     int64_t *row_ptr, int32_t *col) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *tmp_idx = (int64_t *)malloc((size_t)(m_raw > 0 ? m_raw : 1) * sizeof(int64_t));
    int64_t *ord = (int64_t *)malloc((size_t)(m_raw > 0 ? m_raw : 1) * sizeof(int64_t));
    if (!cnt || !tmp_idx || !ord) { free(cnt); free(tmp_idx); free(ord); return -1; }
    /* pass 1: by destination */
    for (int64_t e = 0; e < m_raw; ++e) cnt[dst[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    for (int64_t e = 0; e < m_raw; ++e) tmp_idx[cnt[dst[e]]++] = e;
    /* pass 2: by source, stable */
    memset(cnt, 0, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m_raw; ++e) cnt[src[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    for (int64_t k = 0; k < m_raw; ++k) { int64_t e = tmp_idx[k]; ord[cnt[src[e]]++] = e; }
    /* compact */
    int64_t m = 0, cur = -1;
    int32_t last_dst = -1;
    for (int64_t v = 0; v <= n; ++v) row_ptr[v] = 0;
    for (int64_t k = 0; k < m_raw; ++k) {
        int64_t e = ord[k];
        int32_t s = src[e], d = dst[e];
        if (s == d) continue;
        if (s == cur && d == last_dst) continue;
        if (s != cur) { cur = s; }
        last_dst = d;
        col[m++] = d;
        row_ptr[s + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    free(cnt); free(tmp_idx); free(ord);
    return m;
}

/* ---- weights --------------------------------------------------------------- */

/* integer weights uniform in {lo..hi} */
void gg_weights_int(int64_t m, int32_t lo, int32_t hi, uint64_t seed, int32_t *w) {
    uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e)
        w[e] = lo + (int32_t)(gg_hash(seed, ST_WEIGHT, (uint64_t)e) % span);
}

/* fp32 weights uniform in [0,1): k * 2^-24 with k a 24-bit random integer (exact in fp32) */
void gg_weights_unit(int64_t m, uint64_t seed, float *w) {
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e)
        w[e] = (float)((double)(gg_hash(seed, ST_WEIGHT, (uint64_t)e) >> 40) * (1.0 / 16777216.0));
}

/* fp32 weights lognormal(mu, sigma) via the Box-Muller transform (Box and Muller 1958) */
void gg_weights_lognormal(int64_t m, double mu, double sigma, uint64_t seed, float *w) {
    const double two_pi = 6.283185307179586476925286766559;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        double u1 = 1.0 - u53(gg_hash(seed, ST_LOGN, 2u * (uint64_t)e));   /* (0,1] */
        double u2 = u53(gg_hash(seed, ST_LOGN, 2u * (uint64_t)e + 1u));
        double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
        w[e] = (float)exp(mu + sigma * z);
    }
}
