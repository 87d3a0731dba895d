// batch.cu -- many delta-stepping solves in one persistent launch, and the
// adjoint of their distances with respect to the weights.
//
// Forward (k_batch). Every block is a team that takes instances (source,
// graph) from a device-side queue and runs each one start to end, with its own
// bucket state in its own slice of the working memory. The phases of one
// instance are those of Fig. 1 (Sections III-C, III-D, IV-C):
//   LIGHT   relax the light arcs of the frontier F (the vertices of bucket i
//           whose distance changed in the previous round): t_Req = A_L^T (t o t_Bi),
//           with the re-introduction filter and t = min(t, t_Req) fused into one
//           64-bit atomicMin per arc on packed[v] = key(t[v]) << 32 | low word;
//   HEAVY   relax the heavy arcs of S, the vertices processed in bucket i:
//           t_Req = A_H^T (t o S);
//   SELECT  the next non-empty bucket: the far list (vertices whose distance
//           fell into a later bucket) is scanned once; vertices of the new
//           bucket i go to F and S, those of later buckets stay, those of
//           processed buckets are dropped.
// A team's phases are separated by block barriers only, so a phase costs a few
// dependent memory round trips; the other teams keep the memory system busy.
// The low word of packed[] is the predecessor vertex, or -- with a tape -- the
// input index of the arc that realised the distance. Input arcs are stored row
// by row, so the minimum over (key, input index) selects the same predecessor
// as the minimum over (key, vertex), and among parallel arcs of that row the
// one with the smallest input index (the tree-arc rule of the gradient).
//
// Adjoint (k_backward). With L = sum_v c[v] * d[v] and d[v] the sum of the
// tree-path weights, dL/dw(e) for the tree arc e = (pred[v], v) is the sum of c
// over the subtree below v. The subtree sums are taken leaves first: a vertex
// is ready once all of its tree children have added their sums to it, so each
// round's ready list depends only on earlier rounds (a topological order of
// the predecessor tree, whatever order the forward run found the distances in).
#include <algorithm>
#include <cooperative_groups.h>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "graph.cuh"
#include "warp_util.cuh"

namespace dsssp {
namespace {

namespace cg = cooperative_groups;
using wu::FULL;
using wu::inf_key;
using wu::key_add;
using wu::lane_id;

constexpr int kTeamThreads = 512;
constexpr int kTeamWarps = kTeamThreads / 32;
constexpr int kTIlp = 4;                    // independent 32-arc steps per warp iteration
constexpr uint32_t kTMinSlice = 32u;         // merge-path units of the smallest slice a warp takes
constexpr uint32_t NONE = 0xFFFFFFFFu;

enum TMode : uint32_t { T_LIGHT = 0, T_HEAVY = 1, T_SELECT = 2, T_DONE = 3 };

enum BStat {
    BS_BUCKETS = 0, BS_LIGHT, BS_HEAVY, BS_SELECT, BS_ALIGHT, BS_AHEAVY, BS_IMPROVE, BS_FARSCAN, BS_NS, BS_TEAM,
    BS_VLIGHT, BS_VHEAVY, kBStats = 16
};

struct BGraphDev {
    const uint4 *vinfo;        // n: (light begin, light end = heavy begin, heavy end, 0)
    const uint2 *arcs;         // m: (head, weight bits), light first per row
    const uint32_t *perm;      // m: split position -> input arc index
    const uint32_t *tail;      // m: arc position -> row (tape only; a row covers the same
                               //    positions in the input and in the split order)
    double delta;
    uint32_t n, m;
};

struct BInstDev {
    void *dist;                // n of the graph's dtype
    int32_t *pred;             // n, or null
    uint32_t *tree;            // tape: input index of v's tree arc (NONE: source / unreached)
    uint32_t *parent;          // tape: pred[v] (NONE: unreached)
    uint32_t graph, src, orig, pad;
};

// Per-team working memory: array x of team t starts at x + t * cap (times the
// array's stride for packed and the two stamps). In a batch plan a vertex's
// packed word and its two stamps share one 16-byte record (strides 2 and 4), so
// a relaxation and the bookkeeping of the improvement it makes touch one 32-byte
// sector; the single-solve workspace keeps them in separate arrays (strides 1).
struct TeamWS {
    unsigned long long *packed;
    uint32_t *nstamp;          // phase stamp of the last push into the next frontier
    uint32_t *sstamp;          // S-round stamp of the last push into S
    uint32_t *fflag;           // instance stamp while the vertex has a far-list entry
    uint2 *F0, *F1, *S0, *S1;  // (vertex, exclusive arc offset)
    uint32_t *X0, *X1;         // far lists
    uint32_t pst;              // packed stride in 64-bit words
    uint32_t sts;              // nstamp / sstamp stride in 32-bit words
};

struct BatchArgs {
    const BGraphDev *graphs;
    const BInstDev *inst;      // in queue order
    uint32_t n_inst;
    uint32_t pad0;
    uint32_t *queue;           // next instance (reset before every launch)
    uint32_t *gen;             // per team: stamp generator, kept across launches
    int *err;                  // first device-side status
    long long *stats;          // n_inst x kBStats, indexed by the caller's instance order
    TeamWS ws;
    unsigned long long cap;    // vertices per team slice
    long long max_phases;
};

// One block's view of the current phase, in its own shared memory: the list the
// phase reads, where its pushes go, and the team counters (in the leader block's
// shared memory, reached through distributed shared memory when the team is a
// cluster of several blocks).
struct Ph {
    uint2 *Fo;                      // next frontier
    unsigned long long *cF;
    uint2 *So;                      // S pushes
    unsigned long long *cS;
    uint32_t *Xo;                   // far-list pushes
    uint32_t *cX;
    const uint2 *in;                // LIGHT / HEAVY: the list read
    const uint32_t *xin;            // SELECT: the far list read
    uint32_t count, arcs;           // its entries and arcs
    uint32_t *nstamp, *sstamp, *fflag;
    uint32_t sts;                   // stride of nstamp / sstamp
    uint32_t *far_min, *next_min;   // team reductions
    uint32_t *ovf;                  // team flag: a relaxation met a sum the weight type cannot hold
    unsigned long long *improve, *a_light, *a_heavy;
    uint32_t T, T_lo, pstamp, sst, fst, mode;
};

// Team control in shared memory. Thread 0 decides the next phase between two
// block barriers; every thread then reads the decision.
struct TeamShared {
    BInstDev I;                              // the instance being solved and its graph
    BGraphDev G;
    uint32_t *nstamp, *sstamp, *fflag;
    unsigned long long ctrF[2], ctrS[2];     // (entries << 32) | arcs
    unsigned long long a_light, a_heavy, improve, far_scanned;
    long long phases, n_light, n_heavy, n_select, buckets, v_light, v_heavy;
    unsigned long long t0;
    uint32_t nX[2];
    uint32_t far_min;                        // <= every key of a live far entry
    uint32_t next_min;                       // SELECT: smallest key kept
    uint32_t ovf;                            // a relaxation met a sum the weight type cannot hold
    uint32_t ovf_bad;                        // the final check confirmed an overflow
    uint32_t capped;                         // the instance reached the phase cap (no result)
    uint32_t mode, cur, scur, xcur, pstamp, sst, T, T_lo, fst, gen, inst;
    uint32_t gen_seen;                       // every block: the leader's generator at instance start
};

// Improved vertices wait in a per-warp record buffer and are classified 32 at
// a time (their stamp exchanges in flight together).
constexpr uint32_t kTRec = 32 + 32 * kTIlp;
// A list entry weighs this many arcs in the merge-path split of a phase.
constexpr uint32_t kTEntryCost = 4;

struct TStage {
    uint32_t fv[wu::kStage], fd[wu::kStage];   // next frontier (vertex, light degree)
    uint32_t sv[wu::kStage], sd[wu::kStage];   // S (vertex, heavy degree)
    uint32_t xv[wu::kStage];                   // far list
    uint32_t iv[kTRec], ik[kTRec];             // improvement records (vertex, new key)
};

struct Team {
    const uint4 *vinfo;
    const uint2 *arcs;
    const uint32_t *perm;      // split position -> input arc index (tape)
    unsigned long long *packed;
    uint32_t n, m;
    uint32_t pst;              // packed stride
    __device__ __forceinline__ unsigned long long *pk(uint32_t v) const { return packed + (size_t)v * pst; }
};

struct TPush {
    bool f, s, x;
    uint32_t fdeg, sdeg;
};

__device__ __forceinline__ void stage_push(const Ph &ph, TStage &ws, uint32_t &nf, uint32_t &ns, uint32_t &nx,
                                           const TPush &p, uint32_t v) {
    if (__ballot_sync(FULL, p.f || p.s || p.x) == 0u) return;
    wu::stage_arc_entry(p.f, v, p.fdeg, ws.fv, ws.fd, nf, ph.Fo, ph.cF);
    wu::stage_arc_entry(p.s, v, p.sdeg, ws.sv, ws.sd, ns, ph.So, ph.cS);
    wu::stage_id(p.x, v, ws.xv, nx, ph.Xo, ph.cX);
}

__device__ __forceinline__ void drain_push(const Ph &ph, TStage &ws, uint32_t &nf, uint32_t &ns, uint32_t &nx) {
    if (nf) wu::flush_arc_entries(ws.fv, ws.fd, nf, ph.Fo, ph.cF);
    if (ns) wu::flush_arc_entries(ws.sv, ws.sd, ns, ph.So, ph.cS);
    if (nx) wu::flush_ids(ws.xv, nx, ph.Xo, ph.cX);
    __syncwarp();
    nf = ns = nx = 0u;
}

// relax(v, new distance) of Section III-C after a strict decrease of t[v]:
// back into bucket i (once per phase into F, once per S round into S), or
// into a later bucket (once into the far list while it has a live entry).
template <int DT>
__device__ __forceinline__ void on_improved(const Team &t, const Ph &ph, uint32_t v, uint32_t ck, TPush &p,
                                            uint32_t &far_min) {
    if (ck < ph.T) {
        const uint32_t prev = atomicExch(ph.nstamp + (size_t)v * ph.sts, ph.pstamp);
        const uint4 vi = t.vinfo[v];
        const uint32_t ss = __ldcg(ph.sstamp + (size_t)v * ph.sts);
        if (prev == ph.pstamp) return;
        p.fdeg = vi.y - vi.x;
        p.f = p.fdeg != 0u;
        if (ss != ph.sst) {
            ph.sstamp[(size_t)v * ph.sts] = ph.sst;
            p.sdeg = vi.z - vi.y;
            p.s = p.sdeg != 0u;
        }
    } else {
        far_min = min(far_min, ck);
        p.x = atomicExch(ph.fflag + v, ph.fst) != ph.fst;
    }
}

// Classify the warp's improvement records 32 at a time (all of them when
// `all`); fewer than 32 stay buffered.
template <int DT>
__device__ __forceinline__ void team_classify(const Team &t, const Ph &ph, TStage &ws, uint32_t &nf,
                                              uint32_t &ns, uint32_t &nx, uint32_t &nrec, uint32_t &far_min,
                                              bool all) {
    const uint32_t lane = lane_id();
    uint32_t start = 0;
    // at most kTRec / 32 chunks: nrec < kTRec
    for (uint32_t it = 0; it < kTRec / 32u && (start + 32u <= nrec || (all && start < nrec)); ++it) {
        const uint32_t idx = start + lane;
        TPush p{};
        uint32_t v = 0;
        if (idx < nrec) {
            v = ws.iv[idx];
            on_improved<DT>(t, ph, v, ws.ik[idx], p, far_min);
        }
        stage_push(ph, ws, nf, ns, nx, p, v);
        start += 32u;
    }
    const uint32_t rest = nrec > start ? nrec - start : 0u;
    uint32_t x = 0, y = 0;
    __syncwarp();
    if (lane < rest) { x = ws.iv[start + lane]; y = ws.ik[start + lane]; }
    __syncwarp();
    if (lane < rest) { ws.iv[lane] = x; ws.ik[lane] = y; }
    __syncwarp();
    nrec = rest;
}

// The calling warp's index within its team and the team's warp count (a team
// is the cluster of blocks that solves one instance; read from special registers).
__device__ __forceinline__ uint32_t team_warp() {
    return (cg::this_cluster().block_rank() * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ uint32_t team_warps() { return (cg::this_cluster().num_blocks() * blockDim.x) >> 5; }
__device__ __forceinline__ uint32_t team_thread() { return cg::this_cluster().block_rank() * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint32_t team_threads() { return cg::this_cluster().num_blocks() * blockDim.x; }

// LIGHT / HEAVY: relax the arcs of one list, split evenly over the team's warps
// (merge-path over the entries' arc offsets; 32-entry window per warp).
template <int DT, bool LIGHT, bool TAPE>
__device__ void team_relax(const Team &t, const Ph &ph, TStage &ws, int *sl, uint32_t &far_min,
                           unsigned long long &improved, unsigned long long &relaxed) {
    const uint32_t gw = team_warp(), nw_all = team_warps();
    const uint2 *list = ph.in;
    const uint32_t count = ph.count, E = ph.arcs;
    const uint32_t lane = lane_id();
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(list) + 1;   // offs[2 * j]
    uint32_t nf = 0, ns = 0, nx = 0, nrec = 0;
    bool ovf = false;                       // a sum the weight type cannot hold
    // merge-path over entries and arcs together (an entry weighs kTEntryCost arcs);
    // the first arc of entry i sits at (i + 1) * kTEntryCost + offs[i]
    const unsigned long long W = (unsigned long long)count * kTEntryCost + E;
    const unsigned long long want_w = (W + kTMinSlice - 1u) / kTMinSlice;
    const uint32_t nw = want_w < (unsigned long long)nw_all ? (uint32_t)want_w : nw_all;
    if (gw < nw) {
        const unsigned long long d0 = W * gw / nw, d1 = W * (gw + 1) / nw;
        uint32_t lo0 = 0, hi0 = count, lo1 = 0, hi1 = count;
        while (hi0 - lo0 > 31u || hi1 - lo1 > 31u) {
            const uint32_t st0 = (hi0 - lo0 + 31u) >> 5, st1 = (hi1 - lo1 + 31u) >> 5;
            const uint32_t p0 = lo0 + lane * st0, p1 = lo1 + lane * st1;
            const bool ok0 = hi0 - lo0 > 31u && p0 < hi0 &&
                             (unsigned long long)(p0 + 1u) * kTEntryCost + __ldcg(offs + 2ull * p0) <= d0;
            const bool ok1 = hi1 - lo1 > 31u && p1 < hi1 &&
                             (unsigned long long)(p1 + 1u) * kTEntryCost + __ldcg(offs + 2ull * p1) <= d1;
            const uint32_t k0 = __popc(__ballot_sync(FULL, ok0)), k1 = __popc(__ballot_sync(FULL, ok1));
            if (hi0 - lo0 > 31u) {
                hi0 = min(hi0, lo0 + k0 * st0);
                lo0 = k0 ? lo0 + (k0 - 1u) * st0 + 1u : lo0;
            }
            if (hi1 - lo1 > 31u) {
                hi1 = min(hi1, lo1 + k1 * st1);
                lo1 = k1 ? lo1 + (k1 - 1u) * st1 + 1u : lo1;
            }
        }
        uint32_t i0, i1, o0, o1;
        {
            const uint32_t p0 = lo0 + lane, p1 = lo1 + lane;
            const uint32_t v0 = p0 <= hi0 ? (p0 < count ? __ldcg(offs + 2ull * p0) : E) : E;
            const uint32_t v1 = p1 <= hi1 ? (p1 < count ? __ldcg(offs + 2ull * p1) : E) : E;
            const bool ok0 = p0 < hi0 && (unsigned long long)(p0 + 1u) * kTEntryCost + v0 <= d0;
            const bool ok1 = p1 < hi1 && (unsigned long long)(p1 + 1u) * kTEntryCost + v1 <= d1;
            const uint32_t k0 = __popc(__ballot_sync(FULL, ok0)), k1 = __popc(__ballot_sync(FULL, ok1));
            i0 = lo0 + k0;
            i1 = lo1 + k1;
            o0 = __shfl_sync(FULL, v0, k0);
            o1 = __shfl_sync(FULL, v1, k1);
        }
        const uint32_t e0 = (uint32_t)min(d0 - (unsigned long long)i0 * kTEntryCost, (unsigned long long)o0);
        const uint32_t e1 = (uint32_t)min(d1 - (unsigned long long)i1 * kTEntryCost, (unsigned long long)o1);
        const uint32_t lo = (i0 < count && e0 == o0) ? i0 : i0 - 1u;
        // window: lane k holds entry jw + k; wend = arc offset just past the window
        uint32_t jw = lo, wv = 0, woff = 0xFFFFFFFFu, wbeg = 0, wkey = inf_key<DT>(), wend = 0;
        auto load_window = [&](uint32_t j) {
            const uint32_t idx = j + lane;
            if (idx < count) {
                const uint2 en = __ldcg(list + idx);
                wv = en.x < t.n ? en.x : 0u;
                woff = en.y;
                wkey = (uint32_t)(__ldcg(t.pk(wv)) >> 32);
                const uint4 vi = t.vinfo[wv];
                wbeg = LIGHT ? vi.x : vi.y;
            } else {
                wv = 0; woff = 0xFFFFFFFFu; wbeg = 0; wkey = inf_key<DT>();
            }
            wend = (j + 32u < count) ? __ldcg(offs + 2ull * (j + 32u)) : E;
        };
        load_window(jw);
        int *own_map = sl + (threadIdx.x >> 5) * 32;
        for (uint32_t base0 = e0; base0 < e1; base0 += 32u * kTIlp) {
            uint32_t ai[kTIlp], ov[kTIlp], okey[kTIlp];
            bool ok[kTIlp];
            #pragma unroll
            for (int k = 0; k < kTIlp; ++k) {
                const uint32_t base = base0 + 32u * (uint32_t)k;
                ok[k] = false;
                ai[k] = 0u;
                ov[k] = 0u;
                okey[k] = inf_key<DT>();
                if (base < e1) {
                    const uint32_t last = min(base + 31u, e1 - 1u);
                    if (last >= wend) {
                        const uint32_t shift = base >= wend ? 32u : 31u - __clz(__ballot_sync(FULL, woff <= base));
                        jw += shift;
                        load_window(jw);
                    }
                    // owner of arc base + lane: the last window entry starting at or before it
                    const int carry = 31 - __clz(__ballot_sync(FULL, woff <= base));
                    const uint32_t next_off = __shfl_sync(FULL, woff, (carry + 1) & 31);
                    const bool one_owner = carry == 31 ? wend > base + 31u : next_off > base + 31u;
                    int own = carry;
                    if (!one_owner) {
                        own_map[lane] = -1;
                        __syncwarp();
                        if (woff > base && woff - base < 32u) own_map[woff - base] = (int)lane;
                        __syncwarp();
                        own = own_map[lane];
                        #pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int x = __shfl_up_sync(FULL, own, o);
                            if ((int)lane >= o) own = max(own, x);
                        }
                        own = max(own, carry);
                        __syncwarp();
                    }
                    ov[k] = __shfl_sync(FULL, wv, own);
                    const uint32_t ooff = __shfl_sync(FULL, woff, own);
                    const uint32_t obeg = __shfl_sync(FULL, wbeg, own);
                    okey[k] = __shfl_sync(FULL, wkey, own);
                    const uint32_t e = base + lane;
                    ai[k] = obeg + (e - ooff);
                    ok[k] = e < e1 && ai[k] < t.m && okey[k] < inf_key<DT>();
                }
            }
            uint2 arc[kTIlp];
            uint32_t pin[kTIlp];       // tape: the arc's input index, loaded beside the arc (same positions)
            #pragma unroll
            for (int k = 0; k < kTIlp; ++k) {
                arc[k] = ok[k] ? __ldcs(t.arcs + ai[k]) : make_uint2(0u, 0u);
                if (TAPE) pin[k] = ok[k] ? __ldcs(t.perm + ai[k]) : NONE;
            }
            uint32_t ck[kTIlp];
            unsigned long long cur[kTIlp], cand[kTIlp];
            #pragma unroll
            for (int k = 0; k < kTIlp; ++k) {
                ck[k] = ok[k] ? key_add<DT>(okey[k], arc[k].y) : inf_key<DT>();
                ovf |= ok[k] && ck[k] >= inf_key<DT>();
                cur[k] = ck[k] < inf_key<DT>() ? __ldcg(t.pk(arc[k].x)) : 0ull;
            }
            // with a tape the low word is the arc's input index
            #pragma unroll
            for (int k = 0; k < kTIlp; ++k) cand[k] = ((unsigned long long)ck[k] << 32) | (TAPE ? pin[k] : ov[k]);
            // packed[v] only decreases: a value read earlier bounds it, so the
            // atomic is skipped when the request cannot win (old = 0: no win)
            unsigned long long old[kTIlp];
            #pragma unroll
            for (int k = 0; k < kTIlp; ++k)
                old[k] = (ck[k] < inf_key<DT>() && cand[k] < cur[k]) ? atomicMin(t.pk(arc[k].x), cand[k]) : 0ull;
            #pragma unroll
            for (int k = 0; k < kTIlp; ++k) {
                const bool imp = cand[k] < old[k] && (uint32_t)(old[k] >> 32) > ck[k];   // strict decrease
                const uint32_t mask = __ballot_sync(FULL, imp);
                if (imp) {
                    const uint32_t r = nrec + __popc(mask & wu::lanemask_lt());
                    ws.iv[r] = arc[k].x;
                    ws.ik[r] = ck[k];
                }
                nrec += __popc(mask);
                if (imp) ++improved;
            }
            if (nrec >= 32u) {
                __syncwarp();
                team_classify<DT>(t, ph, ws, nf, ns, nx, nrec, far_min, false);
            }
        }
        if (lane == 0) relaxed += e1 - e0;
        if (__any_sync(FULL, ovf) && lane == 0) *ph.ovf = 1u;
    }
    if (nrec) {
        __syncwarp();
        team_classify<DT>(t, ph, ws, nf, ns, nx, nrec, far_min, true);
    }
    drain_push(ph, ws, nf, ns, nx);
}

// SELECT: one pass over the far list with the new bucket's bounds [T_lo, T).
template <int DT>
__device__ void team_select(const Team &t, const Ph &ph, TStage &ws, uint32_t &next_min) {
    const uint32_t gw = team_warp(), nw = team_warps();
    const uint32_t *xin = ph.xin;
    const uint32_t count = ph.count;
    const uint32_t lane = lane_id();
    uint32_t nf = 0, ns = 0, nx = 0;
    for (uint32_t base = gw * 32u; base < count; base += nw * 32u) {
        const uint32_t idx = base + lane;
        TPush p{};
        uint32_t v = NONE;
        if (idx < count && (v = __ldcg(xin + idx)) < t.n) {          // written by other blocks of the team
            const uint32_t k = (uint32_t)(__ldcg(t.pk(v)) >> 32);
            if (k < ph.T_lo) {
                ph.fflag[v] = 0u;                    // its bucket was processed
            } else if (k < ph.T) {
                ph.fflag[v] = 0u;                    // B_i of the new bucket: F and S
                const uint4 vi = t.vinfo[v];
                p.fdeg = vi.y - vi.x;
                p.f = p.fdeg != 0u;
                ph.sstamp[(size_t)v * ph.sts] = ph.sst;
                p.sdeg = vi.z - vi.y;
                p.s = p.sdeg != 0u;
            } else {
                p.x = true;                          // a later bucket: stays
                next_min = min(next_min, k);
            }
        }
        stage_push(ph, ws, nf, ns, nx, p, v);
    }
    drain_push(ph, ws, nf, ns, nx);
}

__device__ __forceinline__ uint32_t warp_min(uint32_t x) { return __reduce_min_sync(FULL, x); }

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// The control flow of Fig. 1 for one instance (thread 0, between barriers).
template <int DT>
__device__ __noinline__ void team_decide(TeamShared &s, const BGraphDev &g, const BatchArgs &a) {
    switch (s.mode) {
    case T_LIGHT:
        s.n_light += 1;
        s.v_light += (long long)(s.ctrF[s.cur] >> 32);
        s.ctrF[s.cur] = 0ull;
        s.cur ^= 1u;
        break;
    case T_HEAVY:
        s.n_heavy += 1;
        s.v_heavy += (long long)(s.ctrS[s.scur] >> 32);
        s.ctrS[s.scur] = 0ull;
        s.scur ^= 1u;                        // S pushed during the heavy pass (re-opened bucket)
        s.cur ^= 1u;
        break;
    case T_SELECT:
        s.n_select += 1;
        s.nX[s.xcur] = 0u;
        s.xcur ^= 1u;
        s.cur ^= 1u;
        s.far_min = s.next_min;
        if ((s.ctrF[s.cur] >> 32) != 0ull || (s.ctrS[s.scur] >> 32) != 0ull) s.buckets += 1;
        break;
    default:
        break;
    }
    s.phases += 1;
    if (s.phases >= a.max_phases) {
        atomicCAS(a.err, 0, (int)DSSSP_ERR_NOT_CONVERGED);
        s.capped = 1u;
        s.mode = T_DONE;
        return;
    }
    s.pstamp = ++s.gen;
    if ((s.ctrF[s.cur] >> 32) != 0ull) {             // inner loop of Fig. 1: while t_Bi != 0
        s.mode = T_LIGHT;
    } else if ((s.ctrS[s.scur] >> 32) != 0ull) {     // bucket settled: heavy pass over S
        s.mode = T_HEAVY;
        s.sst = ++s.gen;
    } else if (s.nX[s.xcur] != 0u) {                 // next non-empty bucket
        s.mode = T_SELECT;
        s.T_lo = s.T;
        if (s.far_min < inf_key<DT>()) {
            const int64_t i = bucket_of_key(s.far_min, DT, g.delta);
            s.T = i < INT64_MAX ? bucket_floor_key(i + 1, DT, g.delta) : inf_key<DT>();
        } else {
            s.T = inf_key<DT>();
        }
        s.sst = ++s.gen;
        s.next_min = inf_key<DT>();
    } else {
        s.mode = T_DONE;
    }
}

// A block's view of the next phase (its thread 0, after the leader's
// team_decide): lists from the team's slice of working memory, counters and
// control from the leader's shared memory L.
template <int DT>
__device__ __noinline__ void build_view(Ph &ph, TeamShared *L, const BatchArgs &a, size_t off) {
    const uint32_t mode = L->mode, cur = L->cur, scur = L->scur, xcur = L->xcur;
    ph.mode = mode;
    ph.Fo = (cur ? a.ws.F0 : a.ws.F1) + off;                 // F[cur ^ 1]
    ph.cF = &L->ctrF[cur ^ 1u];
    const uint32_t sp = mode == T_HEAVY ? scur ^ 1u : scur;  // a heavy pass feeds the next S
    ph.So = (sp ? a.ws.S1 : a.ws.S0) + off;
    ph.cS = &L->ctrS[sp];
    const uint32_t xp = mode == T_SELECT ? xcur ^ 1u : xcur; // SELECT rebuilds the far list
    ph.Xo = (xp ? a.ws.X1 : a.ws.X0) + off;
    ph.cX = &L->nX[xp];
    unsigned long long c = 0ull;
    if (mode == T_LIGHT) {
        ph.in = (cur ? a.ws.F1 : a.ws.F0) + off;
        c = L->ctrF[cur];
    } else if (mode == T_HEAVY) {
        ph.in = (scur ? a.ws.S1 : a.ws.S0) + off;
        c = L->ctrS[scur];
    } else {
        ph.in = nullptr;
        c = (unsigned long long)L->nX[xcur] << 32;
    }
    ph.xin = (xcur ? a.ws.X1 : a.ws.X0) + off;
    ph.count = (uint32_t)(c >> 32);
    ph.arcs = (uint32_t)c;
    ph.nstamp = a.ws.nstamp + off * a.ws.sts;
    ph.sstamp = a.ws.sstamp + off * a.ws.sts;
    ph.sts = a.ws.sts;
    ph.fflag = a.ws.fflag + off;
    ph.far_min = &L->far_min;
    ph.next_min = &L->next_min;
    ph.ovf = &L->ovf;
    ph.improve = &L->improve;
    ph.a_light = &L->a_light;
    ph.a_heavy = &L->a_heavy;
    ph.T = L->T;
    ph.T_lo = L->T_lo;
    ph.pstamp = L->pstamp;
    ph.sst = L->sst;
    ph.fst = L->fst;
}

template <int DT, bool TAPE>
__global__ void __launch_bounds__(kTeamThreads, 2) k_batch(BatchArgs a) {
    __shared__ TeamShared s;
    __shared__ Ph ph;
    __shared__ TStage stage[kTeamWarps];
    __shared__ int own_map[kTeamWarps * 32];
    // A team is a cluster of blocks (one block when launched without clusters);
    // block 0 of the cluster (the leader) holds the team's control and counters.
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank(), csize = cl.num_blocks();
    const bool leader = rank == 0u;
    const uint32_t tid = threadIdx.x;
    const uint32_t team = blockIdx.x / csize;
    const size_t off = (size_t)team * a.cap;
    Team t;
    t.packed = a.ws.packed + off * a.ws.pst;
    t.pst = a.ws.pst;
    if (leader && tid == 0) {
        s.gen = a.gen[team];
        s.nstamp = a.ws.nstamp + off * a.ws.sts;
        s.sstamp = a.ws.sstamp + off * a.ws.sts;
        s.fflag = a.ws.fflag + off;
    }
    for (;;) {
        if (leader && tid == 0) s.inst = atomicAdd(a.queue, 1u);
        cl.sync();
        if (tid == 0) {
            const TeamShared *L = cl.map_shared_rank(&s, 0);
            s.inst = L->inst;
            s.gen_seen = L->gen;
            if (s.inst < a.n_inst) {
                s.I = a.inst[s.inst];
                s.G = a.graphs[s.I.graph];
            }
        }
        cl.sync();                              // every block has its copy before the leader moves on
        const uint32_t ii = s.inst;
        if (ii >= a.n_inst) break;
        t.vinfo = s.G.vinfo;
        t.arcs = s.G.arcs;
        t.perm = s.G.perm;
        t.n = s.G.n;
        t.m = s.G.m;
        // stamps restart from 1 before the leader's generator could wrap
        if (s.gen_seen > 0xF0000000u) {
            for (size_t v = team_thread(); v < a.cap; v += team_threads()) {
                a.ws.nstamp[(off + v) * a.ws.sts] = 0u;
                a.ws.sstamp[(off + v) * a.ws.sts] = 0u;
                a.ws.fflag[off + v] = 0u;
            }
            cl.sync();
            if (leader && tid == 0) s.gen = 1u;
        }
        const unsigned long long init = ((unsigned long long)inf_key<DT>() << 32) | NONE;
        for (uint32_t v = team_thread(); v < t.n; v += team_threads()) *t.pk(v) = init;
        cl.sync();
        if (leader && tid == 0) {
            s.t0 = wu::globaltimer();
            s.ctrF[0] = s.ctrF[1] = s.ctrS[0] = s.ctrS[1] = 0ull;
            s.a_light = s.a_heavy = s.improve = s.far_scanned = 0ull;
            s.phases = s.n_light = s.n_heavy = s.n_select = s.v_light = s.v_heavy = 0;
            s.buckets = 1;
            s.nX[0] = s.nX[1] = 0u;
            s.far_min = inf_key<DT>();
            s.next_min = inf_key<DT>();
            s.ovf = 0u;
            s.ovf_bad = 0u;
            s.capped = 0u;
            s.cur = s.scur = s.xcur = 0u;
            s.fst = ++s.gen;
            s.sst = ++s.gen;
            s.pstamp = ++s.gen;
            s.T_lo = 0u;
            s.T = bucket_floor_key(1, DT, s.G.delta);    // bucket 0 holds the source
            const uint32_t src = s.I.src;
            *t.pk(src) = TAPE ? (unsigned long long)NONE : (unsigned long long)src;   // key 0
            const uint4 vi = s.G.vinfo[src];
            if (vi.y > vi.x) {
                a.ws.F0[off] = make_uint2(src, 0u);
                s.ctrF[0] = (1ull << 32) | (vi.y - vi.x);
            }
            if (vi.z > vi.y) {
                a.ws.S0[off] = make_uint2(src, 0u);
                s.ctrS[0] = (1ull << 32) | (vi.z - vi.y);
            }
            s.sstamp[(size_t)src * a.ws.sts] = s.sst;
            s.mode = (s.ctrF[0] >> 32) ? T_LIGHT : ((s.ctrS[0] >> 32) ? T_HEAVY : T_DONE);
            if (s.mode == T_HEAVY) s.sst = ++s.gen;
        }
        cl.sync();
        if (tid == 0) build_view<DT>(ph, cl.map_shared_rank(&s, 0), a, off);
        __syncthreads();
        for (;;) {
            const uint32_t mode = ph.mode;
            if (mode == T_DONE) break;
            uint32_t fmin = inf_key<DT>();
            unsigned long long improved = 0, relaxed = 0;
            TStage &ws = stage[tid >> 5];
            if (mode == T_LIGHT) {
                team_relax<DT, true, TAPE>(t, ph, ws, own_map, fmin, improved, relaxed);
            } else if (mode == T_HEAVY) {
                team_relax<DT, false, TAPE>(t, ph, ws, own_map, fmin, improved, relaxed);
            } else {
                team_select<DT>(t, ph, ws, fmin);
            }
            fmin = warp_min(fmin);
            improved = warp_sum(improved);
            if (lane_id() == 0) {
                if (fmin < inf_key<DT>()) atomicMin(mode == T_SELECT ? ph.next_min : ph.far_min, fmin);
                if (improved) atomicAdd(ph.improve, improved);
                if (relaxed) atomicAdd(mode == T_LIGHT ? ph.a_light : ph.a_heavy, relaxed);
            }
            cl.sync();
            if (leader && tid == 0) {
                if (mode == T_SELECT) s.far_scanned += s.nX[s.xcur];
                team_decide<DT>(s, s.G, a);
            }
            cl.sync();
            if (tid == 0) build_view<DT>(ph, cl.map_shared_rank(&s, 0), a, off);
            __syncthreads();
        }
        // Overflow (reading R14): when a relaxation met a sum the weight type
        // cannot hold, every arc of every reached vertex is tested again with its
        // final distance (one warp per vertex); a confirmed overflow fails the
        // batch with DSSSP_ERR_OVERFLOW and leaves this instance's outputs alone.
        // An instance that reached the phase cap has no result either.
        if (tid == 0) {
            const TeamShared *L = cl.map_shared_rank(&s, 0);   // same values in every block of the team
            s.ovf = L->ovf;
            s.capped = L->capped;
        }
        __syncthreads();
        bool write_out = s.capped == 0u;
        if (s.ovf) {
            uint32_t *bad_flag = &cl.map_shared_rank(&s, 0)->ovf_bad;
            const uint32_t lane = lane_id();
            for (uint32_t v = team_warp(); v < t.n; v += team_warps()) {
                const uint32_t k = (uint32_t)(__ldcg(t.pk(v)) >> 32);
                if (k >= inf_key<DT>()) continue;
                const uint4 vi = t.vinfo[v];
                bool bad = false;
                for (uint32_t e = vi.x + lane; e < vi.z && e < t.m; e += 32u)
                    bad |= key_add<DT>(k, __ldcg(t.arcs + e).y) >= inf_key<DT>();
                if (__any_sync(FULL, bad)) {
                    if (lane == 0) *bad_flag = 1u;
                    break;
                }
            }
            cl.sync();
            if (cl.map_shared_rank(&s, 0)->ovf_bad) {
                write_out = false;
                if (leader && tid == 0) atomicCAS(a.err, 0, (int)DSSSP_ERR_OVERFLOW);
            }
        }
        // unpack: dist = key bits; pred from the low word (tape: via the arc's row)
        if (write_out) {
            const BInstDev &I = s.I;
            const BGraphDev &G = s.G;
            const uint32_t src = I.src;
            uint32_t *dist = reinterpret_cast<uint32_t *>(I.dist);
            for (uint32_t v = team_thread(); v < t.n; v += team_threads()) {
                const unsigned long long p = __ldcg(t.pk(v));
                const uint32_t key = (uint32_t)(p >> 32), low = (uint32_t)p;
                const bool reached = key < inf_key<DT>();
                uint32_t pr = NONE, tree = NONE;
                if (reached) {
                    if (v == src) pr = src;
                    else if (TAPE) { pr = low < t.m ? G.tail[low] : NONE; tree = low < t.m ? low : NONE; }
                    else pr = low;
                }
                dist[v] = key;
                if (I.pred) I.pred[v] = (int32_t)pr;
                if (TAPE) {
                    I.tree[v] = tree;
                    I.parent[v] = pr;
                }
            }
        }
        if (leader && tid == 0) {
            long long *st = a.stats + (size_t)s.I.orig * kBStats;
            st[BS_BUCKETS] = s.buckets;
            st[BS_LIGHT] = s.n_light;
            st[BS_HEAVY] = s.n_heavy;
            st[BS_SELECT] = s.n_select;
            st[BS_ALIGHT] = (long long)s.a_light;
            st[BS_AHEAVY] = (long long)s.a_heavy;
            st[BS_IMPROVE] = (long long)s.improve;
            st[BS_FARSCAN] = (long long)s.far_scanned;
            st[BS_NS] = (long long)(wu::globaltimer() - s.t0);
            st[BS_TEAM] = team;
            st[BS_VLIGHT] = s.v_light;
            st[BS_VHEAVY] = s.v_heavy;
        }
        cl.sync();
    }
    if (leader && tid == 0) a.gen[team] = s.gen;
}

// ---------------------------------------------------------------------------
// Adjoint.

struct BwdArgs {
    const BGraphDev *graphs;
    const BInstDev *inst;      // queue order
    uint32_t n_inst;
    uint32_t pad0;
    uint32_t *queue;
    int *err;
    const float *const *c;     // by the caller's instance order
    double *const *grad64;     // per graph, input arc order
    TeamWS ws;
    unsigned long long cap;
};

__global__ void __launch_bounds__(kTeamThreads, 2) k_backward(BwdArgs a) {
    // a team (cluster of blocks, as in the forward launch) per instance; the
    // ready-list counters live in the leader block's shared memory
    struct BwdShared {
        uint32_t inst, n[2], reached, done;
    };
    __shared__ BwdShared bs;
    cg::cluster_group cl = cg::this_cluster();
    const bool leader = cl.block_rank() == 0u;
    BwdShared *Ls = cl.map_shared_rank(&bs, 0);
    const uint32_t tid = threadIdx.x;
    const uint32_t tt = team_thread(), nt = team_threads();
    const size_t off = (size_t)(blockIdx.x / cl.num_blocks()) * a.cap;
    // subtree sums in the S0 list's memory (8 bytes per vertex, contiguous; the
    // records' stamps are kept for the next forward run)
    double *acc = reinterpret_cast<double *>(a.ws.S0 + off);
    uint32_t *L[2] = {reinterpret_cast<uint32_t *>(a.ws.F0 + off), reinterpret_cast<uint32_t *>(a.ws.F0 + off) + a.cap};
    uint32_t *cnt = reinterpret_cast<uint32_t *>(a.ws.F1 + off);     // children not yet summed
    for (;;) {
        if (leader && tid == 0) bs.inst = atomicAdd(a.queue, 1u);
        cl.sync();
        const uint32_t ii = Ls->inst;
        cl.sync();                              // all have read it before the leader moves on
        if (ii >= a.n_inst) break;
        const BInstDev I = a.inst[ii];
        const uint32_t n = a.graphs[I.graph].n, m = a.graphs[I.graph].m;
        const float *c = a.c[I.orig];
        double *g64 = a.grad64[I.graph];
        for (uint32_t v = tt; v < n; v += nt) { acc[v] = 0.0; cnt[v] = 0u; }
        if (leader && tid == 0) { bs.n[0] = bs.n[1] = 0u; bs.reached = 0u; bs.done = 0u; }
        cl.sync();
        uint32_t reached = 0;
        for (uint32_t v = tt; v < n; v += nt) {
            const uint32_t p = I.parent[v];
            if (p == NONE) continue;
            ++reached;
            if (v != I.src && p < n) atomicAdd(cnt + p, 1u);
        }
        reached = __reduce_add_sync(FULL, reached);
        if (lane_id() == 0 && reached) atomicAdd(&Ls->reached, reached);
        cl.sync();
        for (uint32_t v = tt; v < n; v += nt)                // leaves
            if (I.parent[v] != NONE && __ldcg(cnt + v) == 0u) L[0][atomicAdd(&Ls->n[0], 1u)] = v;
        cl.sync();
        uint32_t cur = 0, done = 0;
        for (;;) {
            const uint32_t cnt_cur = Ls->n[cur];
            if (cnt_cur == 0u) break;
            for (uint32_t k = tt; k < cnt_cur; k += nt) {
                const uint32_t v = __ldcg(L[cur] + k);
                const double sum = __ldcg(acc + v) + (double)c[v];
                ++done;
                if (v == I.src) continue;
                const uint32_t e = I.tree[v], p = I.parent[v];
                if (e < m) atomicAdd(g64 + e, sum);
                if (p < n) {
                    atomicAdd(acc + p, sum);
                    if (atomicSub(cnt + p, 1u) == 1u) L[cur ^ 1u][atomicAdd(&Ls->n[cur ^ 1u], 1u)] = p;
                }
            }
            cl.sync();
            if (leader && tid == 0) bs.n[cur] = 0u;
            cur ^= 1u;
            cl.sync();
        }
        done = __reduce_add_sync(FULL, done);
        if (lane_id() == 0 && done) atomicAdd(&Ls->done, done);
        cl.sync();
        if (leader && tid == 0 && bs.done != bs.reached) atomicCAS(a.err, 0, (int)DSSSP_ERR_DEGENERATE);   // a cycle
        cl.sync();
    }
}

__global__ void k_grad_out(double *const *grad64, float *const *grad_w, const uint32_t *m_of, int accumulate) {
    const uint32_t gi = blockIdx.y;
    const uint32_t m = m_of[gi];
    const double *src = grad64[gi];
    float *dst = grad_w[gi];
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const float g = (float)src[e];
        dst[e] = accumulate ? dst[e] + g : g;
    }
}

// row of every split position (tape: the parent of a tree arc)
__global__ void k_tail(const uint4 *vinfo, uint32_t n, uint32_t *tail) {
    const uint32_t lane = lane_id();
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t u = w; u < n; u += nw) {
        const uint4 vi = vinfo[u];
        for (uint32_t p = vi.x + lane; p < vi.z; p += 32u) tail[p] = u;
    }
}

// A single solve run as one instance of the batch kernel (DSSSP_MODE_TEAM): the
// tables, queue, generator, error word and counters in a small region of the
// graph handle, written here from the launch parameters.
__global__ void k_team_setup(BatchArgs a, BGraphDev gd, BInstDev in, BGraphDev *gslot, BInstDev *islot) {
    if (threadIdx.x == 0) {
        *gslot = gd;
        *islot = in;
        *a.queue = 0u;
        *a.gen = 0u;
        *a.err = 0;
    }
    for (uint32_t i = threadIdx.x; i < (uint32_t)kBStats; i += blockDim.x) a.stats[i] = 0;
}

// Region layout: BGraphDev | BInstDev | queue, generator, error word | counters.
constexpr size_t kTeamGraphOff = 0, kTeamInstOff = 128, kTeamWordsOff = 256, kTeamStatsOff = 384;

}  // namespace

size_t team_region_bytes() { return kTeamStatsOff + sizeof(long long) * kBStats; }

cudaError_t team_solve_launch(dsssp_graph *g, const Split *sp, int32_t src, double delta, void *dist,
                              int32_t *pred, int team_blocks, int64_t max_phases, cudaStream_t st) {
    static_assert(sizeof(BGraphDev) <= kTeamInstOff - kTeamGraphOff, "team region layout");
    static_assert(sizeof(BInstDev) <= kTeamWordsOff - kTeamInstOff, "team region layout");
    char *r = static_cast<char *>(g->team_region);
    const SolveArgs &w = g->args;
    const size_t n = (size_t)g->n;
    BatchArgs a{};
    a.graphs = reinterpret_cast<const BGraphDev *>(r + kTeamGraphOff);
    a.inst = reinterpret_cast<const BInstDev *>(r + kTeamInstOff);
    a.n_inst = 1u;
    a.queue = reinterpret_cast<uint32_t *>(r + kTeamWordsOff);
    a.gen = a.queue + 1;
    a.err = reinterpret_cast<int *>(a.queue + 2);
    a.stats = reinterpret_cast<long long *>(r + kTeamStatsOff);
    a.ws.packed = w.packed;              // the single-solve workspace serves as one team's slice
    a.ws.nstamp = w.near_stamp;
    a.ws.sstamp = w.s_stamp;
    a.ws.fflag = w.b_stamp;
    a.ws.pst = 1u;
    a.ws.sts = 1u;
    a.ws.F0 = w.F0;
    a.ws.F1 = w.F1;
    a.ws.S0 = w.S0;
    a.ws.S1 = w.S1;
    a.ws.X0 = w.OV0;
    a.ws.X1 = w.OV1;
    a.cap = n;
    a.max_phases = max_phases;
    BGraphDev gd{};
    gd.vinfo = sp->vinfo;
    gd.arcs = sp->arcs;
    gd.perm = sp->perm;
    gd.tail = nullptr;
    gd.delta = delta;
    gd.n = (uint32_t)g->n;
    gd.m = (uint32_t)g->m;
    BInstDev in{};
    in.dist = dist;
    in.pred = pred;
    in.src = (uint32_t)src;
    // stamps start from the generator's first value: no stamp of an earlier solve may match
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.near_stamp, 0, n * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.s_stamp, 0, n * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.b_stamp, 0, n * sizeof(uint32_t), st)) != cudaSuccess) return e;
    k_team_setup<<<1, 32, 0, st>>>(a, gd, in, reinterpret_cast<BGraphDev *>(r + kTeamGraphOff),
                                   reinterpret_cast<BInstDev *>(r + kTeamInstOff));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const void *kfn = g->dtype == DSSSP_F32 ? (const void *)k_batch<DSSSP_F32, false>
                                            : (const void *)k_batch<DSSSP_I32, false>;
    if (team_blocks > 8 && (e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                               cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)team_blocks;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)team_blocks);
    cfg.blockDim = dim3(kTeamThreads);
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    void *kargs[] = {&a};
    return cudaLaunchKernelExC(&cfg, kfn, kargs);
}

int *team_err(dsssp_graph *g) { return reinterpret_cast<int *>(static_cast<char *>(g->team_region) + kTeamWordsOff + 8); }

long long *team_stats(dsssp_graph *g) {
    return reinterpret_cast<long long *>(static_cast<char *>(g->team_region) + kTeamStatsOff);
}

void team_stats_to_solve(const long long *st, dsssp_stats *out) {
    out->buckets = st[BS_BUCKETS];
    out->light_phases = st[BS_LIGHT];
    out->heavy_phases = st[BS_HEAVY];
    out->rebin_phases = st[BS_SELECT];
    out->vertices_light = st[BS_VLIGHT];
    out->vertices_heavy = st[BS_VHEAVY];
    out->arcs_light = st[BS_ALIGHT];
    out->arcs_heavy = st[BS_AHEAVY];
    out->far_scanned = st[BS_FARSCAN];
    out->improvements = st[BS_IMPROVE];
    out->ns_total = st[BS_NS];
}

}  // namespace dsssp

using namespace dsssp;

// ---------------------------------------------------------------------------
// Host side.

struct dsssp_batch {
    int device = 0;
    int dtype = 0;
    bool tape = false;
    bool ran = false;
    int32_t n_graphs = 0, n_inst = 0;
    std::vector<dsssp_graph *> graphs;
    std::vector<Split *> splits;
    std::vector<uint32_t> m_of;
    uint32_t teams = 0;
    uint32_t csize = 1;                     // blocks per team (cluster size)
    unsigned long long cap = 0;
    void *mem = nullptr;                    // one device allocation for everything below
    BGraphDev *d_graphs = nullptr;
    BInstDev *d_inst = nullptr;
    uint32_t *d_queue = nullptr;            // [0] forward, [1] backward
    uint32_t *d_gen = nullptr;
    int *d_err = nullptr;
    long long *d_stats = nullptr;
    uint32_t *d_tail = nullptr;             // tape: per graph, m entries
    uint32_t *d_tape = nullptr;             // tape: per instance, tree + parent
    double *d_grad64 = nullptr;             // tape: per graph, m entries
    double **d_grad64_ptr = nullptr;
    float **d_gradw_ptr = nullptr;
    const float **d_c_ptr = nullptr;
    uint32_t *d_m_of = nullptr;
    TeamWS ws{};
    BatchArgs args{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *kfn = nullptr;              // the forward kernel of this plan
    void *h_ptrs = nullptr;                 // pinned staging for backward pointer tables
    long long max_phases = 0;
    // team_blocks = -1: the instances one after another, each by the grid-wide persistent solver
    bool seq = false;
    std::vector<int32_t> seq_graph, seq_src;
    std::vector<void *> seq_dist;
    std::vector<int32_t *> seq_pred;
    std::vector<double> seq_delta;          // per graph
    Ctl *h_ctl = nullptr;                   // pinned: every instance's control block after its solve
};

namespace {

void release(dsssp_batch *b) {
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->mem);
    if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
    for (Split *s : b->splits)
        if (s && s->pins > 0) s->pins--;
    delete b;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

dsssp_status dsssp_batch_create(dsssp_graph *const *graphs, int32_t n_graphs, const double *delta, int32_t n_inst,
                                const int32_t *src, const int32_t *src_graph, void *const *dist,
                                int32_t *const *pred, uint32_t flags, const dsssp_options *opt, void *stream,
                                dsssp_batch **out) {
    if (!out) return DSSSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!graphs || n_graphs < 1 || !delta || n_inst < 1 || !src || !dist) return DSSSP_ERR_INVALID_ARG;
    if (flags & ~DSSSP_BATCH_TAPE) return DSSSP_ERR_INVALID_ARG;
    dsssp_options o;
    dsssp_options_default(&o);
    if (opt) {
        if (opt->struct_size != sizeof(dsssp_options)) return DSSSP_ERR_INVALID_ARG;
        if (opt->block_size && opt->block_size != kTeamThreads) return DSSSP_ERR_INVALID_ARG;
        if (opt->grid_size < 0 || opt->max_phases < 0) return DSSSP_ERR_INVALID_ARG;
        if (opt->grid_size) o.grid_size = opt->grid_size;
        if (opt->max_phases) o.max_phases = opt->max_phases;
        o.team_blocks = opt->team_blocks;
    }
    const int dtype = graphs[0] ? graphs[0]->dtype : -1;
    const int device = graphs[0] ? graphs[0]->device : -1;
    for (int32_t i = 0; i < n_graphs; ++i) {
        if (!graphs[i] || graphs[i]->dtype != dtype || graphs[i]->device != device) return DSSSP_ERR_INVALID_ARG;
        if (!(delta[i] > 0.0)) return DSSSP_ERR_INVALID_ARG;
    }
    const bool tape = (flags & DSSSP_BATCH_TAPE) != 0;
    if (tape && dtype != DSSSP_F32) return DSSSP_ERR_UNSUPPORTED;
    for (int32_t k = 0; k < n_inst; ++k) {
        const int32_t gi = src_graph ? src_graph[k] : 0;
        if (gi < 0 || gi >= n_graphs) return DSSSP_ERR_INVALID_ARG;
        if (src[k] < 0 || (int64_t)src[k] >= graphs[gi]->n || !dist[k]) return DSSSP_ERR_INVALID_ARG;
    }
    DeviceGuard dg(device);
    cudaStream_t st = (cudaStream_t)stream;
    dsssp_batch *b = new (std::nothrow) dsssp_batch();
    if (!b) return DSSSP_ERR_OOM;
    b->device = device;
    b->dtype = dtype;
    b->tape = tape;
    b->n_graphs = n_graphs;
    b->n_inst = n_inst;
    b->max_phases = o.max_phases;
    b->graphs.assign(graphs, graphs + n_graphs);
    auto fail = [&](dsssp_status s) {
        release(b);
        return s;
    };
    // splits (pinned while the plan lives)
    b->splits.assign(n_graphs, nullptr);
    for (int32_t i = 0; i < n_graphs; ++i) {
        Split *sp = nullptr;
        dsssp_status rc = ensure_split(graphs[i], delta[i], st, &sp);
        if (rc != DSSSP_OK) return fail(rc);
        sp->pins++;
        b->splits[i] = sp;
    }
    if (o.team_blocks == -1) {
        // one instance after another on the whole GPU (the single-solve kernel): for workloads
        // whose instances each fill the GPU and whose working sets fit L2 only one at a time
        if (tape) return fail(DSSSP_ERR_UNSUPPORTED);
        b->seq = true;
        b->csize = 0;
        b->seq_delta.assign(delta, delta + n_graphs);
        for (int32_t k = 0; k < n_inst; ++k) {
            b->seq_graph.push_back(src_graph ? src_graph[k] : 0);
            b->seq_src.push_back(src[k]);
            b->seq_dist.push_back(dist[k]);
            b->seq_pred.push_back(pred ? pred[k] : nullptr);
        }
        cudaError_t ce = cudaMallocHost(&b->h_ctl, sizeof(Ctl) * (size_t)n_inst);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(cuda_status(ce));
        }
        *out = b;
        return DSSSP_OK;
    }
    // team size (blocks per instance): a cluster when instances are fewer than the blocks
    int bps = 0, sms = 0;
    const void *kfn = dtype == DSSSP_F32 ? (tape ? (const void *)k_batch<DSSSP_F32, true>
                                                 : (const void *)k_batch<DSSSP_F32, false>)
                                          : (const void *)k_batch<DSSSP_I32, false>;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn, kTeamThreads, 0);
    if (e != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return fail(DSSSP_ERR_CUDA);
    if (bps < 1) return fail(DSSSP_ERR_UNSUPPORTED);
    const long long blocks_max = (long long)bps * sms;
    int csize = o.team_blocks;
    if (csize != 0 && csize != 1 && csize != 2 && csize != 4 && csize != 8 && csize != 16)
        return fail(DSSSP_ERR_INVALID_ARG);
    if (csize == 16) {           // clusters above 8 blocks are opt-in per kernel
        if (cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
            cudaFuncSetAttribute((const void *)k_backward, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            cudaGetLastError();
            return fail(DSSSP_ERR_UNSUPPORTED);
        }
    }
    if (csize == 0) {            // largest power of two <= 8 with instances x team blocks <= 2 x resident blocks
        csize = 1;
        while (csize < 8 && (long long)n_inst * csize <= blocks_max) csize *= 2;
    }
    // co-resident teams of that size (an automatic size halves until clusters of it fit)
    const bool auto_size = o.team_blocks == 0;
    long long max_teams = blocks_max / csize;
    while (csize > 1) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = (unsigned)csize;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(csize * (blocks_max / csize)));
        cfg.blockDim = dim3(kTeamThreads);
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&clusters, kfn, &cfg);
        if (e != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
        if (clusters >= 1) {
            max_teams = clusters;
            break;
        }
        if (!auto_size) return fail(e != cudaSuccess ? cuda_status(e) : DSSSP_ERR_UNSUPPORTED);
        csize /= 2;
        max_teams = blocks_max / csize;
    }
    unsigned long long cap = 1;
    size_t sum_m = 0, sum_n_inst = 0;
    b->m_of.resize(n_graphs);
    for (int32_t i = 0; i < n_graphs; ++i) {
        cap = std::max<unsigned long long>(cap, (unsigned long long)graphs[i]->n);
        b->m_of[i] = (uint32_t)graphs[i]->m;
        sum_m += (size_t)graphs[i]->m;
    }
    for (int32_t k = 0; k < n_inst; ++k) sum_n_inst += (size_t)graphs[src_graph ? src_graph[k] : 0]->n;
    const size_t per_team = (size_t)cap * (8 + 4 + 4 + 4 + 8 * 4 + 4 * 2);
    long long teams = max_teams;
    if (o.grid_size) teams = std::min<long long>(teams, std::max(1, o.grid_size / csize));
    teams = std::min<long long>(teams, n_inst);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && per_team > 0)
        teams = std::max<long long>(1, std::min<long long>(teams, (long long)((free_b / 2) / per_team)));
    b->teams = (uint32_t)teams;
    b->csize = (uint32_t)csize;
    b->cap = cap;
    // one allocation: tables, counters, per-team memory, tape
    size_t bytes = 0;
    const size_t o_graphs = bytes; bytes += up256(sizeof(BGraphDev) * n_graphs);
    const size_t o_inst = bytes;   bytes += up256(sizeof(BInstDev) * n_inst);
    const size_t o_queue = bytes;  bytes += up256(2 * sizeof(uint32_t));
    const size_t o_gen = bytes;    bytes += up256(sizeof(uint32_t) * teams);
    const size_t o_err = bytes;    bytes += up256(sizeof(int));
    const size_t o_stats = bytes;  bytes += up256(sizeof(long long) * kBStats * n_inst);
    const size_t o_mof = bytes;    bytes += up256(sizeof(uint32_t) * n_graphs);
    const size_t o_ws = bytes;     bytes += up256(per_team * teams + 10 * 256);
    size_t o_tail = 0, o_tape = 0, o_g64 = 0, o_g64p = 0, o_gwp = 0, o_cp = 0;
    if (tape) {
        o_tail = bytes; bytes += up256(sizeof(uint32_t) * std::max<size_t>(sum_m, 1));
        o_tape = bytes; bytes += up256(sizeof(uint32_t) * 2 * sum_n_inst);
        o_g64 = bytes;  bytes += up256(sizeof(double) * std::max<size_t>(sum_m, 1));
        o_g64p = bytes; bytes += up256(sizeof(double *) * n_graphs);
        o_gwp = bytes;  bytes += up256(sizeof(float *) * n_graphs);
        o_cp = bytes;   bytes += up256(sizeof(float *) * n_inst);
    }
    char *mem = nullptr;
    if ((e = cudaMalloc(&mem, bytes)) != cudaSuccess) return fail(cuda_status(e));
    b->mem = mem;
    b->d_graphs = (BGraphDev *)(mem + o_graphs);
    b->d_inst = (BInstDev *)(mem + o_inst);
    b->d_queue = (uint32_t *)(mem + o_queue);
    b->d_gen = (uint32_t *)(mem + o_gen);
    b->d_err = (int *)(mem + o_err);
    b->d_stats = (long long *)(mem + o_stats);
    b->d_m_of = (uint32_t *)(mem + o_mof);
    {
        char *w = mem + o_ws;
        auto take = [&](size_t each) {
            char *p = w;
            w += up256(each * cap * teams);
            return p;
        };
        char *rec = take(16);          // (packed, nstamp, sstamp) per vertex
        b->ws.packed = (unsigned long long *)rec;
        b->ws.nstamp = (uint32_t *)rec + 2;
        b->ws.sstamp = (uint32_t *)rec + 3;
        b->ws.pst = 2u;
        b->ws.sts = 4u;
        b->ws.fflag = (uint32_t *)take(4);
        b->ws.F0 = (uint2 *)take(8);
        b->ws.F1 = (uint2 *)take(8);
        b->ws.S0 = (uint2 *)take(8);
        b->ws.S1 = (uint2 *)take(8);
        b->ws.X0 = (uint32_t *)take(4);
        b->ws.X1 = (uint32_t *)take(4);
    }
    if (tape) {
        b->d_tail = (uint32_t *)(mem + o_tail);
        b->d_tape = (uint32_t *)(mem + o_tape);
        b->d_grad64 = (double *)(mem + o_g64);
        b->d_grad64_ptr = (double **)(mem + o_g64p);
        b->d_gradw_ptr = (float **)(mem + o_gwp);
        b->d_c_ptr = (const float **)(mem + o_cp);
        if ((e = cudaMallocHost(&b->h_ptrs, sizeof(void *) * (size_t)(n_graphs + n_inst))) != cudaSuccess)
            return fail(cuda_status(e));
    }
    // tables (host), instances in queue order: largest graphs first
    std::vector<BGraphDev> hg(n_graphs);
    std::vector<double *> hg64(n_graphs, nullptr);
    size_t moff = 0;
    for (int32_t i = 0; i < n_graphs; ++i) {
        hg[i].vinfo = b->splits[i]->vinfo;
        hg[i].arcs = b->splits[i]->arcs;
        hg[i].perm = b->splits[i]->perm;
        hg[i].tail = tape ? b->d_tail + moff : nullptr;
        hg[i].delta = delta[i];
        hg[i].n = (uint32_t)graphs[i]->n;
        hg[i].m = (uint32_t)graphs[i]->m;
        if (tape) hg64[i] = b->d_grad64 + moff;
        moff += (size_t)graphs[i]->m;
    }
    std::vector<int32_t> order(n_inst);
    std::iota(order.begin(), order.end(), 0);
    auto gof = [&](int32_t k) { return src_graph ? src_graph[k] : 0; };
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return graphs[gof(x)]->m + graphs[gof(x)]->n > graphs[gof(y)]->m + graphs[gof(y)]->n;
    });
    std::vector<BInstDev> hi(n_inst);
    std::vector<size_t> tape_off(n_inst, 0);
    size_t toff = 0;
    for (int32_t k = 0; k < n_inst; ++k) {
        tape_off[k] = toff;
        toff += 2 * (size_t)graphs[gof(k)]->n;
    }
    for (int32_t q = 0; q < n_inst; ++q) {
        const int32_t k = order[q];
        BInstDev &d = hi[q];
        d.dist = dist[k];
        d.pred = pred ? pred[k] : nullptr;
        d.graph = (uint32_t)gof(k);
        d.src = (uint32_t)src[k];
        d.orig = (uint32_t)k;
        d.tree = tape ? b->d_tape + tape_off[k] : nullptr;
        d.parent = tape ? b->d_tape + tape_off[k] + graphs[gof(k)]->n : nullptr;
    }
    std::vector<uint32_t> gen1(teams, 1u);
    e = cudaMemcpyAsync(b->d_graphs, hg.data(), sizeof(BGraphDev) * n_graphs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_inst, hi.data(), sizeof(BInstDev) * n_inst, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_gen, gen1.data(), sizeof(uint32_t) * teams, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_m_of, b->m_of.data(), sizeof(uint32_t) * n_graphs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_stats, 0, sizeof(long long) * kBStats * n_inst, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws.packed, 0, 16 * cap * teams, st);   // records: stamps 0
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws.fflag, 0, 4 * cap * teams, st);
    if (tape) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_grad64_ptr, hg64.data(), sizeof(double *) * n_graphs, cudaMemcpyHostToDevice, st);
        for (int32_t i = 0; i < n_graphs && e == cudaSuccess; ++i) {
            if (graphs[i]->m == 0) continue;
            k_tail<<<std::max(1, std::min<int>(4096, (int)((graphs[i]->n + 15) / 16))), 512, 0, st>>>(
                hg[i].vinfo, hg[i].n, (uint32_t *)hg[i].tail);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(cuda_status(e));
    }
    // the launch, as a CUDA graph: reset the queue, then the persistent kernel
    BatchArgs &a = b->args;
    a.graphs = b->d_graphs;
    a.inst = b->d_inst;
    a.n_inst = (uint32_t)n_inst;
    a.queue = b->d_queue;
    a.gen = b->d_gen;
    a.err = b->d_err;
    a.stats = b->d_stats;
    a.ws = b->ws;
    a.cap = cap;
    a.max_phases = o.max_phases;
    cudaGraphNode_t n_memset = nullptr, n_kernel = nullptr;
    e = cudaGraphCreate(&b->graph, 0);
    if (e == cudaSuccess) {
        cudaMemsetParams mp{};
        mp.dst = b->d_queue;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 1;
        mp.height = 1;
        mp.pitch = 4;
        e = cudaGraphAddMemsetNode(&n_memset, b->graph, nullptr, 0, &mp);
    }
    b->kfn = kfn;
    if (e == cudaSuccess) {
        void *kargs[] = {&b->args};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void *>(kfn);
        kp.gridDim = dim3(b->teams * b->csize);
        kp.blockDim = dim3(kTeamThreads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = kargs;
        e = cudaGraphAddKernelNode(&n_kernel, b->graph, &n_memset, 1, &kp);
    }
    if (e == cudaSuccess && b->csize > 1) {
        cudaKernelNodeAttrValue v{};
        v.clusterDim.x = b->csize;
        v.clusterDim.y = 1;
        v.clusterDim.z = 1;
        e = cudaGraphKernelNodeSetAttribute(n_kernel, cudaKernelNodeAttributeClusterDimension, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(cuda_status(e));
    }
    *out = b;
    return DSSSP_OK;
}

dsssp_status dsssp_batch_run(dsssp_batch *b, void *stream) {
    if (!b) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DSSSP_TRY(cudaStreamIsCapturing(st, &cap));
    if (b->seq) {
        if (cap != cudaStreamCaptureStatusNone) return DSSSP_ERR_UNSUPPORTED;
        dsssp_options o;
        dsssp_options_default(&o);
        o.flags = DSSSP_FLAG_ASYNC;
        o.max_phases = b->max_phases;
        for (int32_t k = 0; k < b->n_inst; ++k) {
            dsssp_graph *g = b->graphs[b->seq_graph[k]];
            dsssp_status rc = dsssp_solve(g, b->seq_src[k], b->seq_delta[b->seq_graph[k]], b->seq_dist[k],
                                          b->seq_pred[k], &o, nullptr, stream);
            if (rc != DSSSP_OK) return rc;
            // the solve's counters, for dsssp_batch_sync
            DSSSP_TRY(cudaMemcpyAsync(b->h_ctl + k, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        }
        b->ran = true;
        return DSSSP_OK;
    }
    if (cap == cudaStreamCaptureStatusActive) {
        // the caller is recording a graph of its own: the same two operations go in as its nodes
        DSSSP_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(uint32_t), st));
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = b->csize;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3(b->teams * b->csize);
        cfg.blockDim = dim3(kTeamThreads);
        cfg.stream = st;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        void *kargs[] = {&b->args};
        DSSSP_TRY(cudaLaunchKernelExC(&cfg, b->kfn, kargs));
    } else {
        DSSSP_TRY(cudaGraphLaunch(b->exec, st));
    }
    b->ran = true;
    return DSSSP_OK;
}

dsssp_status dsssp_batch_sync(dsssp_batch *b, dsssp_batch_stats *stats, void *stream) {
    if (!b) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (b->seq) {
        dsssp_status first = DSSSP_OK;
        for (dsssp_graph *g : b->graphs) {            // waits for the stream; each graph's first error
            const dsssp_status rc = dsssp_graph_sync(g, stream);
            if (first == DSSSP_OK) first = rc;
        }
        if (stats) {
            for (int32_t k = 0; k < b->n_inst; ++k) {
                const long long *x = b->h_ctl[k].ss.st;
                dsssp_batch_stats &o = stats[k];
                std::memset(&o, 0, sizeof o);
                o.buckets = x[ST_BUCKETS];
                o.light_phases = x[ST_LIGHT];
                o.heavy_phases = x[ST_HEAVY];
                o.select_phases = x[ST_REBIN];
                o.arcs_light = x[ST_ALIGHT];
                o.arcs_heavy = x[ST_AHEAVY];
                o.improvements = x[ST_IMPROVE];
                o.far_scanned = x[ST_FARSCAN];
                o.ns = x[ST_NSTOTAL];
                o.team = -1;
                o.vertices_light = x[ST_VLIGHT];
                o.vertices_heavy = x[ST_VHEAVY];
            }
        }
        return first;
    }
    int err = 0;
    std::vector<long long> hs;
    DSSSP_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSSSP_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), st));
    if (stats) {
        hs.resize((size_t)kBStats * b->n_inst);
        DSSSP_TRY(cudaMemcpyAsync(hs.data(), b->d_stats, sizeof(long long) * hs.size(), cudaMemcpyDeviceToHost, st));
    }
    DSSSP_TRY(cudaStreamSynchronize(st));
    if (stats) {
        for (int32_t k = 0; k < b->n_inst; ++k) {
            const long long *x = hs.data() + (size_t)k * kBStats;
            dsssp_batch_stats &o = stats[k];
            std::memset(&o, 0, sizeof o);
            o.buckets = x[BS_BUCKETS];
            o.light_phases = x[BS_LIGHT];
            o.heavy_phases = x[BS_HEAVY];
            o.select_phases = x[BS_SELECT];
            o.arcs_light = x[BS_ALIGHT];
            o.arcs_heavy = x[BS_AHEAVY];
            o.improvements = x[BS_IMPROVE];
            o.far_scanned = x[BS_FARSCAN];
            o.ns = x[BS_NS];
            o.team = x[BS_TEAM];
            o.vertices_light = x[BS_VLIGHT];
            o.vertices_heavy = x[BS_VHEAVY];
        }
    }
    return (dsssp_status)err;
}

dsssp_status dsssp_batch_destroy(dsssp_batch *b) {
    if (!b) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    release(b);
    return DSSSP_OK;
}

dsssp_status dsssp_solve_batched(dsssp_graph *const *graphs, int32_t n_graphs, const double *delta, int32_t n_inst,
                                 const int32_t *src, const int32_t *src_graph, void *const *dist,
                                 int32_t *const *pred, const dsssp_options *opt, dsssp_batch_stats *stats,
                                 void *stream) {
    dsssp_batch *b = nullptr;
    dsssp_status rc = dsssp_batch_create(graphs, n_graphs, delta, n_inst, src, src_graph, dist, pred, 0u, opt,
                                         stream, &b);
    if (rc != DSSSP_OK) return rc;
    rc = dsssp_batch_run(b, stream);
    if (rc == DSSSP_OK) rc = dsssp_batch_sync(b, stats, stream);
    dsssp_batch_destroy(b);
    return rc;
}

dsssp_status dsssp_backward(dsssp_batch *b, const float *const *c, float *const *grad_w, uint32_t flags,
                            void *stream) {
    if (!b || !c || !grad_w || (flags & ~DSSSP_BACKWARD_ACCUMULATE)) return DSSSP_ERR_INVALID_ARG;
    if (!b->tape || !b->ran) return DSSSP_ERR_NO_TAPE;
    for (int32_t k = 0; k < b->n_inst; ++k)
        if (!c[k]) return DSSSP_ERR_INVALID_ARG;
    for (int32_t i = 0; i < b->n_graphs; ++i)
        if (!grad_w[i] && b->m_of[i] > 0) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    // pointer tables through pinned staging; the stream orders reuse of the staging buffer
    DSSSP_TRY(cudaStreamSynchronize(st));
    void **hp = (void **)b->h_ptrs;
    for (int32_t i = 0; i < b->n_graphs; ++i) hp[i] = grad_w[i];
    for (int32_t k = 0; k < b->n_inst; ++k) hp[b->n_graphs + k] = (void *)c[k];
    DSSSP_TRY(cudaMemcpyAsync(b->d_gradw_ptr, hp, sizeof(void *) * b->n_graphs, cudaMemcpyHostToDevice, st));
    DSSSP_TRY(cudaMemcpyAsync(b->d_c_ptr, hp + b->n_graphs, sizeof(void *) * b->n_inst, cudaMemcpyHostToDevice, st));
    size_t sum_m = 0;
    uint32_t max_m = 0;
    for (uint32_t m : b->m_of) {
        sum_m += m;
        max_m = std::max(max_m, m);
    }
    if (sum_m) DSSSP_TRY(cudaMemsetAsync(b->d_grad64, 0, sizeof(double) * sum_m, st));
    DSSSP_TRY(cudaMemsetAsync(b->d_queue + 1, 0, sizeof(uint32_t), st));
    BwdArgs ba{};
    ba.graphs = b->d_graphs;
    ba.inst = b->d_inst;
    ba.n_inst = (uint32_t)b->n_inst;
    ba.queue = b->d_queue + 1;
    ba.err = b->d_err;
    ba.c = b->d_c_ptr;
    ba.grad64 = b->d_grad64_ptr;
    ba.ws = b->ws;
    ba.cap = b->cap;
    {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = b->csize;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3(b->teams * b->csize);
        cfg.blockDim = dim3(kTeamThreads);
        cfg.stream = st;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        DSSSP_TRY(cudaLaunchKernelEx(&cfg, k_backward, ba));
    }
    if (max_m) {
        const dim3 grid((unsigned)std::min<uint32_t>(1024u, (max_m + 1023u) / 1024u), (unsigned)b->n_graphs);
        k_grad_out<<<grid, 256, 0, st>>>(b->d_grad64_ptr, b->d_gradw_ptr, b->d_m_of,
                                         (flags & DSSSP_BACKWARD_ACCUMULATE) ? 1 : 0);
        DSSSP_TRY(cudaGetLastError());
    }
    return DSSSP_OK;
}

}  // extern "C"
