// solve.cu -- the delta-stepping hot path on the GPU (Fig. 1; Sections III-IV).
//
// One solve is a sequence of grid-wide phases:
//   LIGHT   relax the light arcs of the frontier (the vertices of bucket i whose
//           distances have not been relaxed yet): t_Req = A_L^T (t o t_Bi),
//           fused with the re-introduction filter (t_Req < t) o t_Bi and with
//           t = min(t, t_Req) (Section IV-C; the fusion of Section VI-B) through
//           one 64-bit atomicMin per arc on packed[v] = key(t[v]) << 32 | pred[v].
//           The first round of a bucket reads the bucket's own slot list (B_i of
//           Section III-B, kept explicitly) and also puts its vertices into S.
//   HEAVY   relax the heavy arcs of S, the vertices processed in bucket i:
//           t_Req = A_H^T (t o S) (Section III-D, Fig. 1);
//   REBIN   when the window of bucket slots is used up, the overflow list is
//           distributed into the slots of the next window (Fig. 1's outer loop;
//           empty buckets are skipped).
// A vertex whose distance strictly decreases into bucket <= i is queued once
// per phase into the next frontier and, once per bucket, into S; a decrease
// into a later bucket of the window appends it once to that bucket's slot.
//
// Load balance: arc lists carry each entry's arc offset within the list, so a
// phase splits the list's flattened arcs into equal contiguous slices, one per
// warp (merge-path). Each warp finds its first entry with a 32-ary search and
// walks a 32-entry window of the list; each 32-arc step maps arcs to owners
// (one entry for all lanes, or a scatter and a prefix-max). A hub's arcs are
// spread over the whole grid. A warp keeps kIlp steps in flight.
//
// DSSSP_MODE_PERSISTENT runs all phases in one cooperative launch; every
// barrier wait is bounded by timeout_ns and ends the kernel with
// DSSSP_ERR_TIMEOUT instead of hanging. Phases with little work run on block 0
// alone (solo). DSSSP_MODE_STEPPED launches one kernel per phase and runs the
// serial step as a 1-warp kernel.
#include <mutex>

#include "dsssp_internal.cuh"
#include "warp_util.cuh"

namespace dsssp {

namespace {

using wu::flush_arc_entries;
using wu::flush_ids;
using wu::FULL;
using wu::globaltimer;
using wu::inf_key;
using wu::kFlush;
using wu::key_add;
using wu::kStage;
using wu::lane_id;
using wu::lanemask_lt;
using wu::stage_arc_entry;
using wu::stage_id;

constexpr int kMaxWarps = 16;          // blocks of at most 512 threads
#ifndef DSSSP_ILP
#define DSSSP_ILP 4
#endif
#ifndef DSSSP_MIN_BLOCKS
#define DSSSP_MIN_BLOCKS 2
#endif

constexpr int kIlp = DSSSP_ILP;        // independent 32-arc steps per warp iteration
constexpr uint32_t kMinSlice = 64u;    // merge-path units of the smallest slice a warp takes
#ifndef DSSSP_ENTRY_COST
#define DSSSP_ENTRY_COST 4
#endif
constexpr uint32_t kEntryCost = DSSSP_ENTRY_COST;   // arcs' worth of work per list entry (merge-path weight)
// Merge-path directory: a warp's slice starts and ends on a multiple of kDirChunk
// units, whose positions in the list are recorded when entries are appended.
constexpr uint32_t kDirChunk = kMinSlice;
constexpr uint32_t kNoSlot = kSlots;

template <typename T>
__device__ __forceinline__ T vload(const T *p) { return *(const volatile T *)p; }

// Per-block copy of what a phase needs: the descriptor and the window's key
// thresholds (bucket wbase + t starts at key thr[t]).
struct BlockView {
    PhaseDesc d;
    uint32_t thr[kSlots + 1];
    int32_t err;            // the control block's error word when the view was taken
    uint32_t gen;           // phase number of the view
    uint32_t thr_epoch;     // window epoch of thr[] (re-read when the view's epoch differs)
};

// A bucket-slot stamp: one per (window, slot) of a solve, never 0 (the value
// vertices start with). Windows are counted by the serial step (wepoch).
__device__ __forceinline__ uint32_t slot_stamp(uint32_t wepoch, uint32_t t) { return ((wepoch << 5) | t) + 1u; }

// ---------------------------------------------------------------------------
// Per-warp staging of pushes in shared memory (wu::stage_*): a list counter,
// shared by the whole grid, is touched once per kFlush staged entries.
// Improved vertices wait in a per-warp record buffer and are classified 32 at a
// time, so the stamp exchanges of a whole batch are in flight together instead
// of one dependent round trip per 32-arc step.
constexpr uint32_t kRec = 32 + 32 * kIlp;

struct WarpStage {
    uint32_t fv[kStage], fd[kStage];             // next frontier (vertex, light degree)
    uint32_t sv[kStage], sd[kStage];             // S (vertex, heavy degree)
    uint32_t bt[kStage], bv[kStage], bd[kStage]; // bucket slots (slot, vertex, light degree; 0: heavy-only list)
    uint32_t ov[kStage];                         // overflow
    uint32_t iv[kRec], ik[kRec];                 // improvement records (vertex, new key)
};

// Append n <= 32 staged slot entries: lanes are grouped by (slot, list); the
// leader of every group takes its slot counter with one atomic, all groups at
// once, and each lane finds its place from its rank and the arc counts of the
// lower lanes of its group.
__device__ __forceinline__ void flush_slot_entries32(const SolveArgs &a, const uint32_t *bt, const uint32_t *bv,
                                                     const uint32_t *bd, uint32_t n) {
    const uint32_t lane = lane_id();
    const bool has = lane < n;
    const uint32_t t = has ? bt[lane] : 0u, v = has ? bv[lane] : 0u, d = has ? bd[lane] : 0u;
    const uint32_t key = has ? ((t << 1) | (d == 0u ? 1u : 0u)) : 0xFFFFFFFFu;
    const uint32_t grp = __match_any_sync(FULL, key);
    const uint32_t below = grp & lanemask_lt();
    const bool leader = below == 0u;
    const uint32_t rank = __popc(below);
    // arc count of the group's lower lanes (excl) and of the whole group (tot)
    uint32_t excl = 0, tot = 0;
    #pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t dj = __shfl_sync(FULL, d, j);
        if ((grp >> j) & 1u) {
            tot += dj;
            if ((uint32_t)j < lane) excl += dj;
        }
    }
    const uint32_t slot = t;
    Ctl *c = a.ctl;
    unsigned long long old = 0;
    if (has && leader) {
        if (key & 1u) old = atomicAdd(&c->nSH[slot], (uint32_t)__popc(grp));          // heavy-only list
        else old = atomicAdd(&c->ctrSL[slot], ((unsigned long long)__popc(grp) << 32) | tot);
    }
    old = __shfl_sync(FULL, old, __ffs(grp) - 1);
    const bool light = has && (key & 1u) == 0u;
    const uint32_t idx = (uint32_t)(old >> 32) + rank, off = (uint32_t)old + excl;
    if (has) {
        if (key & 1u) a.SH[(size_t)slot * a.n + (uint32_t)old + rank] = v;
        else a.SL[(size_t)slot * a.n + idx] = make_uint2(v, off);
    }
    wu::dir_record<kEntryCost, kDirChunk>(a.dir + (size_t)(kDirSL + slot) * a.dcap, light, idx, off, d);
}

__device__ __forceinline__ void flush_slot_entries(const SolveArgs &a, const uint32_t *bt, const uint32_t *bv,
                                                   const uint32_t *bd, uint32_t n) {
    flush_slot_entries32(a, bt, bv, bd, min(n, 32u));
    if (n > 32u) flush_slot_entries32(a, bt + 32, bv + 32, bd + 32, n - 32u);
}

// ---------------------------------------------------------------------------
// Block-local accumulators flushed to the control block.
struct BlockAcc {
    uint32_t ov_min;
    unsigned long long arcs_light, arcs_heavy, improvements, far_scanned;
};

// Pending pushes of one lane in one step.
struct Push {
    bool f, s, b, ov;
    uint32_t fdeg, sdeg, slot, bdeg;
};

// The warp's staged counts; destination lists follow from the phase descriptor.
struct PushCnt {
    uint32_t nf, ns, nb, nov;
};

__device__ __forceinline__ uint2 *dst_F(const SolveArgs &a, const PhaseDesc &d) { return d.cur ? a.F0 : a.F1; }
__device__ __forceinline__ unsigned long long *ctr_F(const SolveArgs &a, const PhaseDesc &d) {
    return &a.ctl->ctrF[d.cur ^ 1u];
}
__device__ __forceinline__ uint2 *dst_S(const SolveArgs &a, const PhaseDesc &d) { return d.spush ? a.S1 : a.S0; }
// directories of the lists written (F0, F1, S0, S1, then the slot lists)
__device__ __forceinline__ uint2 *dir_F(const SolveArgs &a, const PhaseDesc &d) {
    return a.dir + (size_t)(d.cur ? 0u : 1u) * a.dcap;
}
__device__ __forceinline__ uint2 *dir_S(const SolveArgs &a, const PhaseDesc &d) {
    return a.dir + (size_t)(d.spush ? 3u : 2u) * a.dcap;
}
__device__ __forceinline__ unsigned long long *ctr_S(const SolveArgs &a, const PhaseDesc &d) {
    return &a.ctl->ctrS[d.spush];
}
// LIGHT/HEAVY append to the current overflow list; REBIN rebuilds it into the other one
__device__ __forceinline__ uint32_t ov_index(const PhaseDesc &d) {
    return d.mode == MODE_REBIN ? d.ov_cur ^ 1u : d.ov_cur;
}

__device__ __forceinline__ void stage_slot_entry(const SolveArgs &a, bool pred, uint32_t slot, uint32_t v,
                                                 uint32_t deg, WarpStage &ws, uint32_t &cnt) {
    const uint32_t mask = __ballot_sync(FULL, pred);
    if (mask == 0u) return;
    const uint32_t lane = lane_id();
    if (pred) {
        const uint32_t k = cnt + __popc(mask & lanemask_lt());
        ws.bt[k] = slot; ws.bv[k] = v; ws.bd[k] = deg;
    }
    cnt += __popc(mask);
    __syncwarp();
    if (cnt >= kFlush) {
        flush_slot_entries(a, ws.bt, ws.bv, ws.bd, kFlush);
        const uint32_t rest = cnt - kFlush;
        uint32_t x = 0, y = 0, z = 0;
        if (lane < rest) { x = ws.bt[kFlush + lane]; y = ws.bv[kFlush + lane]; z = ws.bd[kFlush + lane]; }
        __syncwarp();
        if (lane < rest) { ws.bt[lane] = x; ws.bv[lane] = y; ws.bd[lane] = z; }
        __syncwarp();
        cnt = rest;
    }
}

__device__ __forceinline__ void stage_pushes(const SolveArgs &a, const PhaseDesc &d, PushCnt &q, WarpStage &ws,
                                             const Push &p, uint32_t v) {
    if (__ballot_sync(FULL, p.f || p.s || p.b || p.ov) == 0u) return;
    stage_arc_entry<kEntryCost, kDirChunk>(p.f, v, p.fdeg, ws.fv, ws.fd, q.nf, dst_F(a, d), ctr_F(a, d), dir_F(a, d));
    stage_arc_entry<kEntryCost, kDirChunk>(p.s, v, p.sdeg, ws.sv, ws.sd, q.ns, dst_S(a, d), ctr_S(a, d), dir_S(a, d));
    stage_slot_entry(a, p.b, p.slot, v, p.bdeg, ws, q.nb);
    const uint32_t oi = ov_index(d);
    stage_id(p.ov, v, ws.ov, q.nov, oi ? a.OV1 : a.OV0, &a.ctl->nOV[oi]);
}

// Flush the partially filled staging buffers (end of a phase).
__device__ __forceinline__ void drain_pushes(const SolveArgs &a, const PhaseDesc &d, PushCnt &q, WarpStage &ws) {
    if (q.nf) flush_arc_entries<kEntryCost, kDirChunk>(ws.fv, ws.fd, q.nf, dst_F(a, d), ctr_F(a, d), dir_F(a, d));
    if (q.ns) flush_arc_entries<kEntryCost, kDirChunk>(ws.sv, ws.sd, q.ns, dst_S(a, d), ctr_S(a, d), dir_S(a, d));
    if (q.nb) flush_slot_entries(a, ws.bt, ws.bv, ws.bd, q.nb);
    if (q.nov) {
        const uint32_t oi = ov_index(d);
        flush_ids(ws.ov, q.nov, oi ? a.OV1 : a.OV0, &a.ctl->nOV[oi]);
    }
    __syncwarp();
    q.nf = q.ns = q.nb = q.nov = 0u;
}

// ---------------------------------------------------------------------------
// Queue v for bucket i (its key is now below T): once per phase into the next
// frontier (its light segment), once per bucket into S (its heavy segment).
// The loads are issued together with the stamp exchange. Arc segments (vinfo)
// are read once per list entry or improvement, packed[] once per relaxed arc:
// segment reads are evict-first so that packed[] keeps its place in L2.
__device__ __forceinline__ void queue_near(const SolveArgs &a, const PhaseDesc &d, uint32_t v, Push &p) {
    const uint32_t prev = atomicExch(a.near_stamp + v, d.qstamp);
    const uint4 vi = __ldcs(a.vinfo + v);
    const uint32_t ss = __ldcg(a.s_stamp + v);
    if (prev == d.qstamp) return;
    p.fdeg = vi.y - vi.x;
    p.f = p.fdeg != 0u;
    if (ss != d.sstamp) {
        a.s_stamp[v] = d.sstamp;
        p.sdeg = vi.z - vi.y;
        p.s = p.sdeg != 0u;
    }
}

// Slot of key k in the window: the largest t with thr[t] <= k (thr[0] <= k < thr[kSlots]).
__device__ __forceinline__ uint32_t slot_of(const uint32_t *thr, uint32_t k) {
    uint32_t lo = 0, hi = kSlots;          // thr[lo] <= k < thr[hi]
    #pragma unroll
    for (int it = 0; it < 5; ++it) {
        const uint32_t mid = (lo + hi) >> 1;
        if (thr[mid] <= k) lo = mid; else hi = mid;
    }
    return lo;
}

// A later bucket: append v once to its slot (if the window holds it) or to the
// overflow list.
template <int DT>
__device__ __forceinline__ void queue_later(const SolveArgs &a, const BlockView &bvw, uint32_t v, uint32_t ckey,
                                            Push &p, uint32_t &ov_min) {
    if (ckey < bvw.thr[kSlots]) {
        const uint32_t t = slot_of(bvw.thr, ckey);
        const uint32_t stamp = slot_stamp(bvw.d.wepoch, t);   // one entry per (vertex, bucket)
        const uint32_t prev = atomicExch(a.b_stamp + v, stamp);
        const uint4 vi = __ldcs(a.vinfo + v);
        if (prev != stamp) {
            p.b = true;
            p.slot = t;
            p.bdeg = vi.y - vi.x;
        }
    } else {
        ov_min = min(ov_min, ckey);
        p.ov = atomicExch(a.ov_flag + v, 1u) == 0u;
    }
}

// relax(v, new_dist) of Section III-C, after the packed atomicMin found a strict
// decrease of t[v]: back into bucket i ((t_Req < t) o t_Bi) or into a later bucket.
template <int DT>
__device__ __forceinline__ void on_improved(const SolveArgs &a, const BlockView &bvw, uint32_t v, uint32_t ckey,
                                            Push &p, uint32_t &ov_min, uint32_t &improved) {
    ++improved;
    if (ckey < bvw.d.T) queue_near(a, bvw.d, v, p);
    else queue_later<DT>(a, bvw, v, ckey, p, ov_min);
}

// First round of a bucket: every vertex of the bucket's slot (both lists) that
// is still in the bucket joins S (S = S u B_i).
__device__ void slot_entries_into_S(const SolveArgs &a, const PhaseDesc &d, PushCnt &q, WarpStage &ws, uint32_t gw,
                                    uint32_t nw) {
    const uint32_t lane = lane_id();
    const uint2 *sl = a.SL + (size_t)d.slot * a.n;
    const uint32_t *sh = a.SH + (size_t)d.slot * a.n;
    const uint32_t total = d.count + d.count2;
    for (uint32_t base = gw * 32u; base < total; base += nw * 32u) {
        const uint32_t idx = base + lane;
        Push p{};
        uint32_t v = 0;
        if (idx < total) {
            v = idx < d.count ? __ldcs(sl + idx).x : __ldcs(sh + (idx - d.count));
            if (v < a.n) {
                const uint32_t k = (uint32_t)(__ldcg(a.packed + v) >> 32);
                const uint4 vi = a.vinfo[v];
                if (k >= d.T_lo && __ldcg(a.s_stamp + v) != d.sstamp) {
                    a.s_stamp[v] = d.sstamp;
                    p.sdeg = vi.z - vi.y;
                    p.s = p.sdeg != 0u;
                }
            }
        }
        stage_pushes(a, d, q, ws, p, v);
    }
}

// Classify the warp's improvement records 32 at a time (all of them when
// `all`): each record runs relax(v, new distance) of Section III-C with its
// stamp exchanges in flight together; fewer than 32 records stay buffered.
template <int DT>
__device__ __forceinline__ void classify_records(const SolveArgs &a, const BlockView &bvw, PushCnt &q, WarpStage &ws,
                                                 uint32_t &nrec, uint32_t &ov_min, uint32_t &improved, bool all) {
    const uint32_t lane = lane_id();
    uint32_t start = 0;
    // at most kRec / 32 chunks: nrec < kRec
    for (uint32_t it = 0; it < kRec / 32u && (start + 32u <= nrec || (all && start < nrec)); ++it) {
        const uint32_t idx = start + lane;
        Push p{};
        uint32_t v = 0;
        if (idx < nrec) {
            v = ws.iv[idx];
            on_improved<DT>(a, bvw, v, ws.ik[idx], p, ov_min, improved);
        }
        stage_pushes(a, bvw.d, q, ws, p, v);
        start += 32u;
    }
    const uint32_t rest = nrec > start ? nrec - start : 0u;     // fewer than 32
    uint32_t x = 0, y = 0;
    __syncwarp();
    if (lane < rest) { x = ws.iv[start + lane]; y = ws.ik[start + lane]; }
    __syncwarp();
    if (lane < rest) { ws.iv[lane] = x; ws.ik[lane] = y; }
    __syncwarp();
    nrec = rest;
}

// LIGHT / HEAVY: relax the arcs of a list, split evenly over the warps.
// The list read is F (LIGHT), the slot `sl` of a bucket's first round (LIGHT,
// sl < kNoSlot) or S (HEAVY); `count` entries holding `E` arcs.
template <int DT, bool LIGHT>
__device__ void phase_arcs(const SolveArgs &a, const BlockView &bvw, BlockAcc &acc, int *slot, WarpStage *stage,
                           uint32_t gw, uint32_t nw_all, uint32_t count, uint32_t E, uint32_t sl) {
    const PhaseDesc &d = bvw.d;
    const uint32_t lane = lane_id();
    const bool from_slot = LIGHT && sl < kNoSlot;
    const uint2 *list = LIGHT ? (from_slot ? a.SL + (size_t)sl * a.n : (d.cur ? a.F1 : a.F0))
                              : (d.scur ? a.S1 : a.S0);
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(list) + 1;   // offs[2 * j]
    const uint32_t T_lo = from_slot ? d.T_lo : 0u;          // only slot entries can be stale
    uint32_t ov_min = inf_key<DT>();
    uint32_t improved = 0, nrec = 0;
    bool ovf = false;                                       // a sum the weight type cannot hold
    PushCnt q{};
    WarpStage &ws = stage[threadIdx.x >> 5];
    if (from_slot) slot_entries_into_S(a, d, q, ws, gw, nw_all);
    // Merge-path over the list's entries and arcs together: an entry costs
    // kEntryCost arcs' worth of work (its share of a window load and of the owner
    // mapping), so a slice of many short segments gets fewer arcs. In merged
    // order the first arc of entry i sits at (i + 1) * kEntryCost + offs[i]. A
    // warp's slice is a run of kDirChunk-unit chunks (small phases use few
    // warps); where a chunk boundary falls in the list was recorded in the list's
    // directory when the entries were appended, so no search is needed.
    const uint2 *dir = a.dir + (size_t)(LIGHT ? (from_slot ? kDirSL + sl : (d.cur ? 1u : 0u)) : (d.scur ? 3u : 2u)) * a.dcap;
    const unsigned long long W = (unsigned long long)count * kEntryCost + E;
    const uint32_t nch = (uint32_t)((W + kDirChunk - 1u) / kDirChunk);
    const uint32_t nw = nch < nw_all ? nch : nw_all;
    if (gw < nw) {
        const uint32_t c0 = (uint32_t)((unsigned long long)nch * gw / nw);
        const uint32_t c1 = (uint32_t)((unsigned long long)nch * (gw + 1u) / nw);
        const unsigned long long d0 = (unsigned long long)c0 * kDirChunk;
        const unsigned long long d1 = c1 < nch ? (unsigned long long)c1 * kDirChunk : W;
        // (i, o) = number of entries whose first arc lies at or before the
        // boundary, and the arc offset of the entry after them (E past the last)
        const uint2 p0 = c0 != 0u ? __ldcg(dir + c0) : make_uint2(0u, 0u);
        const uint2 p1 = c1 < nch ? __ldcg(dir + c1) : make_uint2(count, E);
        const uint32_t i0 = p0.x, o0 = p0.y, i1 = p1.x, o1 = p1.y;
        const uint32_t e0 = (uint32_t)min(d0 - (unsigned long long)i0 * kEntryCost, (unsigned long long)o0);
        const uint32_t e1 = (uint32_t)min(d1 - (unsigned long long)i1 * kEntryCost, (unsigned long long)o1);
        // the entry owning arc e0
        const uint32_t lo = (i0 < count && e0 == o0) ? i0 : i0 - 1u;
        // window: lane k holds entry jw + k; wend = arc offset just past the window.
        // A stale slot entry (its vertex moved to a lower bucket) gets key INF and is skipped.
        uint32_t jw = lo, wv = 0, woff = 0xFFFFFFFFu, wbeg = 0, wkey = inf_key<DT>(), wend = 0;
        // The arcs of stale entries in this warp's slice are taken off the count of
        // relaxed arcs when the window is loaded (`from`: entries starting before it
        // were counted with an earlier window).
        auto load_window = [&](uint32_t j, uint32_t from) {
            const uint32_t idx = j + lane;
            bool stale = false;
            if (idx < count) {
                const uint2 en = __ldcs(list + idx);
                wv = en.x < a.n ? en.x : 0u;          // defensive: ids come from device lists
                woff = en.y;
                const uint32_t k = (uint32_t)(__ldcg(a.packed + wv) >> 32);
                const uint4 vi = __ldcs(a.vinfo + wv);
                wbeg = LIGHT ? vi.x : vi.y;
                stale = T_lo != 0u && k < T_lo;
                wkey = stale ? inf_key<DT>() : k;
            } else {
                wv = 0; woff = 0xFFFFFFFFu; wbeg = 0; wkey = inf_key<DT>();
            }
            wend = (j + 32u < count) ? __ldcg(offs + 2ull * (j + 32u)) : E;
            if (T_lo != 0u) {
                uint32_t nxt = __shfl_down_sync(FULL, woff, 1);
                if (idx + 1u >= count) nxt = E;
                else if (lane == 31u) nxt = wend;
                const uint32_t lo_a = max(woff, e0), hi_a = min(nxt, e1);
                uint32_t skip = (stale && woff >= from && hi_a > lo_a) ? hi_a - lo_a : 0u;
                skip = __reduce_add_sync(FULL, skip);
                if (lane == 0u && skip) atomicAdd(&acc.arcs_light, 0ull - (unsigned long long)skip);
            }
        };
        load_window(jw, 0u);
        int *sl = slot + (threadIdx.x >> 5) * 32;
        // Each iteration maps kIlp 32-arc steps to owners first, then issues their
        // arc loads, distance reads and atomics back to back.
        for (uint32_t base0 = e0; base0 < e1; base0 += 32u * kIlp) {
            uint32_t ai[kIlp], ov[kIlp], okey[kIlp];
            bool ok[kIlp];
            #pragma unroll
            for (int k = 0; k < kIlp; ++k) {
                const uint32_t base = base0 + 32u * (uint32_t)k;
                ok[k] = false;
                ai[k] = 0u;
                ov[k] = 0u;
                okey[k] = inf_key<DT>();
                if (base < e1) {
                    const uint32_t last = min(base + 31u, e1 - 1u);
                    if (last >= wend) {
                        // move the window to the owner of `base` (inside it, or the entry just past it)
                        const uint32_t shift = base >= wend ? 32u : 31u - __clz(__ballot_sync(FULL, woff <= base));
                        jw += shift;
                        load_window(jw, base);
                    }
                    // owner of arc base + lane: the last window entry starting at or before it
                    const int carry = 31 - __clz(__ballot_sync(FULL, woff <= base));
                    const uint32_t next_off = __shfl_sync(FULL, woff, (carry + 1) & 31);
                    const bool one_owner = carry == 31 ? wend > base + 31u : next_off > base + 31u;
                    int own = carry;
                    if (!one_owner) {
                        sl[lane] = -1;
                        __syncwarp();
                        if (woff > base && woff - base < 32u) sl[woff - base] = (int)lane;
                        __syncwarp();
                        own = sl[lane];
                        #pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int t = __shfl_up_sync(FULL, own, o);
                            if ((int)lane >= o) own = max(own, t);
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
                    // defensive bound (true when lists are consistent); stale owners are skipped
                    ok[k] = e < e1 && ai[k] < a.m && okey[k] < inf_key<DT>();
                }
            }
            uint2 arc[kIlp];
            #pragma unroll
            for (int k = 0; k < kIlp; ++k) arc[k] = ok[k] ? __ldcs(a.arcs + ai[k]) : make_uint2(0u, 0u);
            uint32_t ck[kIlp];
            unsigned long long cur[kIlp];
            #pragma unroll
            for (int k = 0; k < kIlp; ++k) {
                ck[k] = ok[k] ? key_add<DT>(okey[k], arc[k].y) : inf_key<DT>();
                ovf |= ok[k] && ck[k] >= inf_key<DT>();
                cur[k] = ck[k] < inf_key<DT>() ? __ldcg(a.packed + arc[k].x) : 0ull;
            }
            // packed[v] only decreases, so a value read earlier bounds it from above:
            // the atomic is skipped when the request cannot win (old = 0 means no win)
            unsigned long long old[kIlp];
            #pragma unroll
            for (int k = 0; k < kIlp; ++k) {
                const unsigned long long cand = ((unsigned long long)ck[k] << 32) | ov[k];
                old[k] = (ck[k] < inf_key<DT>() && cand < cur[k]) ? atomicMin(a.packed + arc[k].x, cand) : 0ull;
            }
            // strict distance decreases become records, classified 32 at a time
            #pragma unroll
            for (int k = 0; k < kIlp; ++k) {
                const unsigned long long cand = ((unsigned long long)ck[k] << 32) | ov[k];
                const bool imp = cand < old[k] && (uint32_t)(old[k] >> 32) > ck[k];
                const uint32_t mask = __ballot_sync(FULL, imp);
                if (imp) {
                    const uint32_t r = nrec + __popc(mask & lanemask_lt());
                    ws.iv[r] = arc[k].x;
                    ws.ik[r] = ck[k];
                }
                nrec += __popc(mask);
            }
            if (nrec >= 32u) {
                __syncwarp();
                classify_records<DT>(a, bvw, q, ws, nrec, ov_min, improved, false);
            }
        }
        if (lane == 0) {
            if (LIGHT) atomicAdd(&acc.arcs_light, (unsigned long long)(e1 - e0));
            else atomicAdd(&acc.arcs_heavy, (unsigned long long)(e1 - e0));
        }
        if (__any_sync(FULL, ovf) && lane == 0) a.ctl->ovf = 1u;
    }
    if (nrec) {
        __syncwarp();
        classify_records<DT>(a, bvw, q, ws, nrec, ov_min, improved, true);
    }
    drain_pushes(a, d, q, ws);
    if (ov_min < inf_key<DT>()) atomicMin(&acc.ov_min, ov_min);
    if (improved) atomicAdd(&acc.improvements, (unsigned long long)improved);
}

// REBIN: the window is used up; every live overflow vertex either is stale (its
// bucket was processed), goes to its slot in the new window, or stays.
template <int DT>
__device__ void phase_rebin(const SolveArgs &a, const BlockView &bvw, BlockAcc &acc, WarpStage *stage,
                            uint32_t gw, uint32_t nw) {
    const PhaseDesc &d = bvw.d;
    const uint32_t lane = lane_id();
    const uint32_t *in = d.ov_cur ? a.OV1 : a.OV0;
    const uint32_t count = d.count;
    uint32_t ov_min = inf_key<DT>();
    PushCnt q{};
    WarpStage &ws = stage[threadIdx.x >> 5];
    for (uint32_t base = gw * 32u; base < count; base += nw * 32u) {
        const uint32_t idx = base + lane;
        Push p{};
        uint32_t v = 0xFFFFFFFFu;
        if (idx < count && (v = __ldcs(in + idx)) < a.n && __ldcg(a.ov_flag + v) == 1u) {
            const uint32_t k = (uint32_t)(__ldcg(a.packed + v) >> 32);
            if (k < bvw.thr[0]) {
                a.ov_flag[v] = 0u;                      // its bucket was processed: stale
            } else if (k < bvw.thr[kSlots]) {
                a.ov_flag[v] = 0u;
                queue_later<DT>(a, bvw, v, k, p, ov_min);
            } else {
                p.ov = true;                            // stays for a later window
                ov_min = min(ov_min, k);
            }
        }
        stage_pushes(a, d, q, ws, p, v);
    }
    drain_pushes(a, d, q, ws);
    if (ov_min < inf_key<DT>()) atomicMin(&acc.ov_min, ov_min);
    if (gw == 0 && lane == 0) atomicAdd(&acc.far_scanned, (unsigned long long)count);
}

// ---------------------------------------------------------------------------
// The published view (Ctl::view): word l holds (phase number << 32) | field l.
__device__ __forceinline__ uint32_t view_field(const PhaseDesc &d, int32_t err, uint32_t l) {
    switch (l) {
    case 0: return d.mode | (d.cur << 3) | (d.scur << 4) | (d.spush << 5) | (d.ov_cur << 6) | (d.solo << 7) |
                   (d.slot << 8);
    case 1: return d.sstamp;
    case 2: return d.qstamp;
    case 3: return d.T;
    case 4: return d.T_lo;
    case 5: return d.count;
    case 6: return d.arcs;
    case 7: return d.count2;
    case 8: return d.count_h;
    case 9: return d.arcs_h;
    case 10: return d.wepoch;
    case 11: return (uint32_t)err;
    default: return 0u;
    }
}

// Lane l of a warp stores field l of the published view into v (the lanes together fill it).
__device__ __forceinline__ void view_store_field(BlockView &v, uint32_t l, uint32_t f, uint32_t gen) {
    switch (l) {
    case 0:
        v.d.mode = f & 7u; v.d.cur = (f >> 3) & 1u; v.d.scur = (f >> 4) & 1u; v.d.spush = (f >> 5) & 1u;
        v.d.ov_cur = (f >> 6) & 1u; v.d.solo = (f >> 7) & 1u; v.d.slot = (f >> 8) & 63u; v.gen = gen;
        break;
    case 1: v.d.sstamp = f; break;
    case 2: v.d.qstamp = f; break;
    case 3: v.d.T = f; break;
    case 4: v.d.T_lo = f; break;
    case 5: v.d.count = f; break;
    case 6: v.d.arcs = f; break;
    case 7: v.d.count2 = f; break;
    case 8: v.d.count_h = f; break;
    case 9: v.d.arcs_h = f; break;
    case 10: v.d.wepoch = f; break;
    case 11: v.err = (int32_t)f; break;
    default: break;
    }
}

__device__ __forceinline__ unsigned long long vload64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

// Warp 0 of a block: take the published view into v once every word carries the
// same phase number and that number is newer than `last` (0xFFFFFFFF: any).
// Block 0 takes every view; the other blocks pass over solo views (block 0 runs
// them alone) and wait for the next view with work for the whole grid, the end,
// or an error. The wait gives up after timeout_ns without progress (a newer
// view of any kind restarts the clock) or when the error word is set. The
// window thresholds are re-read when the view's window epoch is not the one
// v holds. Returns false on an error or a timeout.
template <int DT>
__device__ bool wait_view(const SolveArgs &a, uint32_t last, BlockView &v, bool patient) {
    const uint32_t lane = lane_id();
    Ctl *c = a.ctl;
    uint64_t t0 = globaltimer();
    uint32_t seen = last;
    for (;;) {
        const unsigned long long w = lane < (uint32_t)kViewWords ? vload64(&c->view[lane]) : 0ull;
        const uint32_t g = (uint32_t)(w >> 32), f = (uint32_t)w;
        const uint32_t g0 = __shfl_sync(FULL, g, 0);
        const bool same = __all_sync(FULL, lane >= (uint32_t)kViewWords || g == g0);
        const uint32_t f0 = __shfl_sync(FULL, f, 0), ferr = __shfl_sync(FULL, f, 11);
        const bool newer = last == 0xFFFFFFFFu || (int32_t)(g0 - last) > 0;
        if (same && newer) {
            const bool solo = ((f0 >> 7) & 1u) != 0u;
            if (blockIdx.x == 0 || !solo || (f0 & 7u) == MODE_DONE || ferr != 0u) {
                __threadfence();                       // what the view's phase reads is visible
                const uint32_t ep = __shfl_sync(FULL, f, 10);
                const bool reload = __shfl_sync(FULL, lane == 0u && ep != v.thr_epoch, 0);
                if (lane < (uint32_t)kViewWords) view_store_field(v, lane, f, g0);
                if (reload) {
                    v.thr[lane] = __ldcg(&c->thr[lane]);
                    if (lane == 0u) {
                        v.thr[kSlots] = __ldcg(&c->thr[kSlots]);
                        v.thr_epoch = ep;
                    }
                }
                __syncwarp();
                return true;
            }
            patient = true;                            // a solo stretch: poll slowly
        }
        const uint64_t now = globaltimer();
        if (same && g0 != seen) { seen = g0; t0 = now; }
        int e = 0;
        if (lane == 0u) e = vload(&c->err);
        e = __shfl_sync(FULL, e, 0);
        if (e != 0) {
            if (lane == 0u) v.err = e;
            __syncwarp();
            return false;
        }
        if ((int64_t)(now - t0) > a.timeout_ns) {
            if (lane == 0u) {
                atomicCAS(&c->err, 0, (int)DSSSP_ERR_TIMEOUT);
                v.err = (int32_t)DSSSP_ERR_TIMEOUT;
            }
            __syncwarp();
            return false;
        }
        if (patient) __nanosleep(500);
    }
}

// ---------------------------------------------------------------------------
// Serial step: one warp, after every block has finished a phase. Every load is
// in one batch: the serial state, the phase that ended and the list counters
// (the same words on all lanes), and lane t's bucket slot t (its counters and
// key threshold). Every lane then takes the same decision (the control flow of
// Fig. 1) in registers; lane 0 resets consumed counters and publishes the next
// PhaseDesc. With `out`, the warp also writes the next phase's view there.
template <int DT>
__device__ __noinline__ void serial_step(const SolveArgs &a, BlockView *out) {
    Ctl *c = a.ctl;
    const uint32_t lane = lane_id();
    const bool l0 = lane == 0u;
    // the control part of the serial state goes through registers; the
    // counters of st[] are only added to (lane 0, atomics whose result is unused)
    SerialState s;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(&c->ss);
        uint4 *dst = reinterpret_cast<uint4 *>(&s);
        #pragma unroll
        for (int k = 0; k < kSerialHotVec; ++k) dst[k] = __ldcg(src + k);
    }
    long long *st = c->ss.st;
    auto stat = [&](int k, long long v) {
        if (l0) atomicAdd(reinterpret_cast<unsigned long long *>(st + k), (unsigned long long)v);
    };
    PhaseDesc od;                                  // the phase that just ended
    #pragma unroll
    for (int k = 0; k < kDescVec; ++k)
        reinterpret_cast<uint4 *>(&od)[k] = __ldcg(reinterpret_cast<const uint4 *>(&c->desc) + k);
    unsigned long long ctrF[2] = {__ldcg(&c->ctrF[0]), __ldcg(&c->ctrF[1])};
    unsigned long long ctrS[2] = {__ldcg(&c->ctrS[0]), __ldcg(&c->ctrS[1])};
    const uint32_t nov[2] = {__ldcg(&c->nOV[0]), __ldcg(&c->nOV[1])};
    uint32_t ov_min = __ldcg(&c->ov_min);
    const uint64_t t_first = __ldcg(&c->t_first);
    int32_t err = __ldcg(&c->err);
    // bucket slot `lane` of the window (kSlots == 32 lanes) and the window's end
    const unsigned long long my_sl = __ldcg(&c->ctrSL[lane]);
    const uint32_t my_sh = __ldcg(&c->nSH[lane]);
    uint32_t my_th = __ldcg(&c->thr[lane]);
    uint32_t th_end = __ldcg(&c->thr[kSlots]);
    const uint64_t now = globaltimer();
    // the first slot past the current bucket: its own state for the fusion
    // check, the first non-empty one for the search of the next bucket (the
    // consumed slot of the current bucket lies below it)
    const int first = (int)(s.bucket - s.wbase + 1);
    const uint32_t ne = __ballot_sync(FULL, (int)lane >= first && ((my_sl >> 32) != 0ull || my_sh != 0u));
    const int found = ne ? __ffs(ne) - 1 : -1;
    const int fl = found < 0 ? 0 : found;
    const unsigned long long fsl = __shfl_sync(FULL, my_sl, fl);
    const uint32_t fsh = __shfl_sync(FULL, my_sh, fl);
    const uint32_t flo = __shfl_sync(FULL, my_th, fl);
    const uint32_t fhi_n = __shfl_sync(FULL, my_th, (fl + 1) & 31);
    const uint32_t fhi = fl + 1 < (int)kSlots ? fhi_n : th_end;

    const uint64_t dt = now - s.t_last;
    if (t_first > s.t_last && t_first <= now) {      // persistent mode only
        stat(ST_NSFIRST, (long long)(t_first - s.t_last));
        stat(ST_NSSPREAD, (long long)(now - t_first));
    }
    s.t_last = now;
    const uint32_t mode = s.mode;
    if (mode == MODE_LIGHT) stat(ST_NSLIGHT, (long long)dt);
    else if (mode == MODE_HEAVY || mode == MODE_FUSED) stat(ST_NSHEAVY, (long long)dt);
    else if (mode == MODE_REBIN) stat(ST_NSREBIN, (long long)dt);
    s.phases += 1;
    PhaseDesc nd{};
    nd.slot = kNoSlot;
    bool done = false;
    if (s.phases >= a.max_phases || s.wepoch >= (1u << 27) - 1u) {   // slot stamps hold 27 bits of epoch
        if (l0) {
            const int prev = atomicCAS(&c->err, 0, (int)DSSSP_ERR_NOT_CONVERGED);
            err = prev != 0 ? prev : (int)DSSSP_ERR_NOT_CONVERGED;
        }
        err = __shfl_sync(FULL, err, 0);
        done = true;
    } else {
        switch (mode) {
        case MODE_LIGHT:
            stat(ST_LIGHT, 1);
            if (od.slot < kNoSlot) {               // the bucket's slot is consumed
                stat(ST_VLIGHT, (long long)od.count);
                if (l0) {
                    c->ctrSL[od.slot] = 0ull;
                    c->nSH[od.slot] = 0u;
                }
            } else {
                stat(ST_VLIGHT, (long long)(ctrF[s.cur] >> 32));
                if (l0) c->ctrF[s.cur] = 0ull;
                ctrF[s.cur] = 0ull;
            }
            break;
        case MODE_HEAVY:
            stat(ST_HEAVY, 1);
            stat(ST_VHEAVY, (long long)(ctrS[s.scur] >> 32));
            if (l0) c->ctrS[s.scur] = 0ull;
            ctrS[s.scur] = 0ull;
            s.scur ^= 1u;               // S pushed during the heavy pass (a re-opened bucket)
            s.sround += 1u;
            break;
        case MODE_FUSED:                           // bucket i's S and bucket i+1's slot are consumed
            stat(ST_LIGHT, 1);
            stat(ST_HEAVY, 1);
            stat(ST_VLIGHT, (long long)od.count);
            stat(ST_VHEAVY, (long long)(ctrS[s.scur] >> 32));
            if (l0) {
                c->ctrSL[od.slot] = 0ull;
                c->nSH[od.slot] = 0u;
                c->ctrS[s.scur] = 0ull;
            }
            ctrS[s.scur] = 0ull;
            s.scur ^= 1u;
            s.sround += 1u;
            break;
        case MODE_REBIN:
            stat(ST_REBIN, 1);
            if (l0) c->nOV[s.ov_cur] = 0u;
            s.ov_cur ^= 1u;
            break;
        default:
            done = true;
            break;
        }
    }
    uint32_t next_mode = MODE_DONE;
    if (!done) {
        s.qstamp += 1u;                            // every phase queues under a fresh stamp
        const uint32_t nxt = s.cur ^ 1u;
        if ((ctrF[nxt] >> 32) != 0ull) {           // inner loop of Fig. 1: while t_Bi != 0
            s.cur = nxt;
            next_mode = MODE_LIGHT;
            nd.count = (uint32_t)(ctrF[nxt] >> 32);
            nd.arcs = (uint32_t)ctrF[nxt];
        } else if ((ctrS[s.scur] >> 32) != 0ull) { // bucket settled: heavy pass over S
            // When bucket i+1 already holds vertices, its first light round runs in the
            // same phase as bucket i's heavy pass: heavy weights exceed Delta, so the
            // heavy pass only adds to buckets >= i+1, and what it adds to i+1 is relaxed
            // in i+1's later rounds (the fixed point does not depend on the order).
            if (a.fuse && first >= 0 && found == first) {
                next_mode = MODE_FUSED;
                s.bucket += 1;
                stat(ST_BUCKETS, 1);
                s.T_lo = flo;
                s.T = fhi;
                nd.slot = (uint32_t)found;
                nd.count = (uint32_t)(fsl >> 32);
                nd.arcs = (uint32_t)fsl;
                nd.count2 = fsh;
                nd.count_h = (uint32_t)(ctrS[s.scur] >> 32);
                nd.arcs_h = (uint32_t)ctrS[s.scur];
            } else {
                next_mode = MODE_HEAVY;
                nd.count = (uint32_t)(ctrS[s.scur] >> 32);
                nd.arcs = (uint32_t)ctrS[s.scur];
            }
        } else if (found >= 0) {                   // next non-empty bucket of the window
            s.bucket = s.wbase + found;
            stat(ST_BUCKETS, 1);
            s.T_lo = flo;
            s.T = fhi;
            next_mode = MODE_LIGHT;
            nd.slot = (uint32_t)found;
            nd.count = (uint32_t)(fsl >> 32);
            nd.arcs = (uint32_t)fsl;
            nd.count2 = fsh;
        } else if (nov[s.ov_cur] != 0u) {
            // window used up: the next one starts at the smallest overflow key;
            // lane t resets slot t and sets its threshold, lane 0 also the window's end
            c->ctrSL[lane] = 0ull;
            c->nSH[lane] = 0u;
            s.wepoch += 1u;
            if (ov_min < inf_key<DT>()) {
                // bucket indices saturate at INT64_MAX (a tiny Delta against large
                // distances): every such key then belongs to the window's slot 0
                const int64_t w = bucket_of_key(ov_min, DT, a.delta);
                s.wbase = w;
                s.bucket = w - 1;
                my_th = (int64_t)lane <= INT64_MAX - w ? bucket_floor_key(w + lane, DT, a.delta) : inf_key<DT>();
                if (lane == 0u && my_th > ov_min) my_th = ov_min;         // slot 0 starts at or below the smallest key
                if (lane == 1u && my_th <= ov_min) my_th = ov_min + 1u;   // the smallest key lands in slot 0
                th_end = (int64_t)kSlots <= INT64_MAX - w ? bucket_floor_key(w + kSlots, DT, a.delta) : inf_key<DT>();
            } else {                               // only stale entries remain: drop them all
                my_th = inf_key<DT>();
                th_end = inf_key<DT>();
            }
            c->thr[lane] = my_th;
            if (l0) {
                c->thr[kSlots] = th_end;
                c->ov_min = inf_key<DT>();
            }
            next_mode = MODE_REBIN;
            nd.count = nov[s.ov_cur];
        }
    }
    if (next_mode == MODE_DONE && l0) st[ST_NSTOTAL] = (long long)(now - s.t_start);
    s.mode = next_mode;
    nd.mode = next_mode;
    nd.cur = s.cur;
    nd.scur = s.scur;
    // S pushes: into the current S, except during a heavy pass, which feeds the next one
    const bool heavy = next_mode == MODE_HEAVY || next_mode == MODE_FUSED;
    nd.spush = heavy ? s.scur ^ 1u : s.scur;
    nd.sstamp = heavy ? s.sround + 1u : s.sround;
    nd.qstamp = s.qstamp;
    nd.T = s.T;
    nd.T_lo = nd.slot < kNoSlot ? s.T_lo : 0u;
    nd.ov_cur = s.ov_cur;
    nd.wepoch = s.wepoch;
    // little work: one block runs the phase without a grid-wide barrier
    const uint32_t work = next_mode == MODE_REBIN ? nd.count
                                                  : max(nd.arcs + nd.arcs_h, nd.count + nd.count2 + nd.count_h);
    nd.solo = work <= a.solo_work ? 1u : 0u;
    if (l0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(&s);
        uint4 *dst = reinterpret_cast<uint4 *>(&c->ss);
        #pragma unroll
        for (int k = 0; k < kSerialHotVec; ++k) dst[k] = src[k];
        const uint4 *ds = reinterpret_cast<const uint4 *>(&nd);
        uint4 *dd = reinterpret_cast<uint4 *>(&c->desc);
        #pragma unroll
        for (int k = 0; k < kDescVec; ++k) dd[k] = ds[k];
    }
    // publish: everything above (every lane's writes) reaches memory before any view word
    const uint32_t gen = (uint32_t)s.phases;
    __threadfence();
    __syncwarp();
    if (lane < (uint32_t)kViewWords)
        *(volatile unsigned long long *)&c->view[lane] = ((unsigned long long)gen << 32) | view_field(nd, err, lane);
    if (out != nullptr) {
        out->thr[lane] = my_th;
        if (l0) {
            out->thr[kSlots] = th_end;
            out->d = nd;
            out->err = err;
            out->gen = gen;
            out->thr_epoch = s.wepoch;
        }
    }
}

__device__ __forceinline__ void flush_ov_min(Ctl *c, BlockAcc &acc, uint32_t inf) {
    if (acc.ov_min < inf) {
        atomicMin(&c->ov_min, acc.ov_min);
        acc.ov_min = inf;
    }
}

__device__ __forceinline__ void flush_stats(Ctl *c, BlockAcc &acc) {
    long long *st = c->ss.st;
    if (acc.arcs_light) atomicAdd((unsigned long long *)&st[ST_ALIGHT], acc.arcs_light);
    if (acc.arcs_heavy) atomicAdd((unsigned long long *)&st[ST_AHEAVY], acc.arcs_heavy);
    if (acc.improvements) atomicAdd((unsigned long long *)&st[ST_IMPROVE], acc.improvements);
    if (acc.far_scanned) atomicAdd((unsigned long long *)&st[ST_FARSCAN], acc.far_scanned);
    acc.arcs_light = acc.arcs_heavy = acc.improvements = acc.far_scanned = 0;
}

template <int DT>
__device__ __forceinline__ void acc_init(BlockAcc &acc) {
    acc.ov_min = inf_key<DT>();
    acc.arcs_light = acc.arcs_heavy = acc.improvements = acc.far_scanned = 0;
}

// Grid-wide barrier with a serial step. Warp 0 of every block arrives; in the
// last block to arrive it runs the serial step, which publishes the next view
// (and writes it into that block's own view). The others wait for the view in
// wait_view, bounded by timeout_ns. A solo view goes to block 0 alone: a last
// arrival that is not block 0 then waits like the others. Returns false when
// the block saw the error word set or gave up waiting.
template <int DT>
__device__ bool grid_barrier(const SolveArgs &a, BlockAcc &acc, BlockView &view, int *s_ok) {
    __syncthreads();
    if (threadIdx.x < 32u) {
        const uint32_t lane = threadIdx.x;
        Ctl *c = a.ctl;
        const uint32_t my_gen = view.gen;
        unsigned arrived = 0u;
        if (lane == 0u) {
            flush_ov_min(c, acc, inf_key<DT>());
            __threadfence();
            arrived = atomicAdd(&c->bar_count, 1u);
            if (arrived == 0u) c->t_first = globaltimer();   // phase-time diagnostics
        }
        arrived = __shfl_sync(FULL, arrived, 0);
        bool ok = true;
        if (arrived == a.nblocks - 1u) {
            if (lane == 0u) {
                atomicExch(&c->bar_count, 0u);
                __threadfence();
            }
            __syncwarp();
            serial_step<DT>(a, &view);
            __syncwarp();
            if (blockIdx.x != 0 && view.d.solo != 0u && view.d.mode != MODE_DONE && view.err == 0)
                ok = wait_view<DT>(a, view.gen, view, true);
        } else {
            ok = wait_view<DT>(a, my_gen, view, false);
        }
        if (lane == 0u) *s_ok = ok && view.err == 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Overflow (reading R14: a sum out of a reached vertex that the weight type
// cannot hold makes the solve fail with DSSSP_ERR_OVERFLOW). A relaxation that
// met such a sum may have used a distance that decreased later, so when any
// did, every arc of every reached vertex is tested once more with the final
// distance, after the last phase. One warp per vertex; runs only in that case.
template <int DT>
__device__ void verify_overflow(const SolveArgs &a, uint32_t gw, uint32_t nw) {
    const uint32_t lane = lane_id();
    for (uint32_t v = gw; v < a.n; v += nw) {
        const uint32_t k = (uint32_t)(__ldcg(a.packed + v) >> 32);
        if (k >= inf_key<DT>()) continue;
        const uint4 vi = a.vinfo[v];
        bool bad = false;
        for (uint32_t e = vi.x + lane; e < vi.z && e < a.m; e += 32u)
            bad |= key_add<DT>(k, __ldcg(a.arcs + e).y) >= inf_key<DT>();
        if (__any_sync(FULL, bad)) {
            if (lane == 0) atomicCAS(&a.ctl->err, 0, (int)DSSSP_ERR_OVERFLOW);
            return;
        }
    }
}

template <int DT>
__device__ __forceinline__ void run_phase(const SolveArgs &a, const BlockView &v, BlockAcc &acc, int *slot,
                                          WarpStage *stage, uint32_t gw, uint32_t nw) {
    switch (v.d.mode) {
    case MODE_LIGHT: phase_arcs<DT, true>(a, v, acc, slot, stage, gw, nw, v.d.count, v.d.arcs, v.d.slot); break;
    case MODE_HEAVY: phase_arcs<DT, false>(a, v, acc, slot, stage, gw, nw, v.d.count, v.d.arcs, kNoSlot); break;
    case MODE_FUSED:
        // heavy arcs of bucket i's S, then the first light round of bucket i+1 (its slot)
        phase_arcs<DT, false>(a, v, acc, slot, stage, gw, nw, v.d.count_h, v.d.arcs_h, kNoSlot);
        phase_arcs<DT, true>(a, v, acc, slot, stage, gw, nw, v.d.count, v.d.arcs, v.d.slot);
        break;
    case MODE_REBIN: phase_rebin<DT>(a, v, acc, stage, gw, nw); break;
    default: break;
    }
}

// The warps' staging buffers live in dynamic shared memory (blockDim / 32 of them).
extern __shared__ __align__(16) unsigned char dyn_smem[];

template <int DT>
__global__ void __launch_bounds__(512, DSSSP_MIN_BLOCKS) k_solve_persistent(SolveArgs a) {
    __shared__ int slot[kMaxWarps * 32];
    WarpStage *stage = reinterpret_cast<WarpStage *>(dyn_smem);
    __shared__ BlockView view;
    __shared__ BlockAcc acc;
    __shared__ int s_ok;
    if (a.test_hook == DSSSP_HOOK_STALL_BARRIER && blockIdx.x == 1) return;
    if (threadIdx.x == 0) {
        acc_init<DT>(acc);
        view.thr_epoch = 0xFFFFFFFFu;
        view.err = 0;
    }
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    __syncthreads();
    if (threadIdx.x < 32u) {
        const bool ok = wait_view<DT>(a, 0xFFFFFFFFu, view, false);
        if (threadIdx.x == 0u) s_ok = ok;
    }
    __syncthreads();
    while (s_ok) {
        if (view.err != 0 || view.d.mode == MODE_DONE) break;
        // A solo phase (little work) runs on block 0 only: its phases follow each
        // other with block-level synchronisation and the serial step in warp 0;
        // the other blocks wait for the next view with work for the whole grid.
        const bool solo = view.d.solo != 0u;
        run_phase<DT>(a, view, acc, slot, stage, solo ? wib : gw, solo ? nwb : nw);
        if (solo) {
            __threadfence();             // list entries and flags reach L2 before the serial step reads them
            __syncthreads();
            if (threadIdx.x < 32u) {     // warp 0: the serial step, which also writes the block's next view
                if (threadIdx.x == 0u) {
                    flush_ov_min(a.ctl, acc, inf_key<DT>());
                    __threadfence();
                }
                __syncwarp();
                serial_step<DT>(a, &view);
            }
            __syncthreads();
            continue;
        }
        if (!grid_barrier<DT>(a, acc, view, &s_ok)) break;
    }
    __syncthreads();
    if (vload(&a.ctl->ovf) != 0u && vload(&a.ctl->err) == 0) verify_overflow<DT>(a, gw, nw);
    if (threadIdx.x == 0) flush_stats(a.ctl, acc);
}

// ---- stepped mode: one launch per phase --------------------------------------
template <int DT, uint32_t MODE>
__global__ void __launch_bounds__(512, DSSSP_MIN_BLOCKS) k_phase(SolveArgs a) {
    __shared__ int slot[kMaxWarps * 32];
    WarpStage *stage = reinterpret_cast<WarpStage *>(dyn_smem);
    __shared__ BlockView view;
    __shared__ BlockAcc acc;
    if (threadIdx.x < 32u) {                  // the view k_serial (or k_init) published
        const uint32_t lane = threadIdx.x;
        const unsigned long long w = lane < (uint32_t)kViewWords ? vload64(&a.ctl->view[lane]) : 0ull;
        if (lane < (uint32_t)kViewWords) view_store_field(view, lane, (uint32_t)w, (uint32_t)(w >> 32));
        view.thr[lane] = __ldcg(&a.ctl->thr[lane]);
        if (lane == 0u) view.thr[kSlots] = __ldcg(&a.ctl->thr[kSlots]);
    }
    if (threadIdx.x == 0) acc_init<DT>(acc);
    __syncthreads();
    if (view.d.mode != MODE || view.err != 0) return;
    run_phase<DT>(a, view, acc, slot, stage, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                  (gridDim.x * blockDim.x) >> 5);
    __syncthreads();
    if (threadIdx.x == 0) {
        flush_ov_min(a.ctl, acc, inf_key<DT>());
        flush_stats(a.ctl, acc);
    }
}

// The overflow check of a stepped solve (see verify_overflow).
template <int DT>
__global__ void __launch_bounds__(512) k_verify_overflow(SolveArgs a) {
    if (vload(&a.ctl->ovf) == 0u || vload(&a.ctl->err) != 0) return;
    verify_overflow<DT>(a, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5);
}

// One warp.
template <int DT>
__global__ void k_serial(SolveArgs a) {
    if (vload(&a.ctl->desc.mode) != MODE_DONE) serial_step<DT>(a, nullptr);
}

// ---- init / unpack -------------------------------------------------------------
template <int DT>
__global__ void k_init(SolveArgs a) {
    const uint32_t n = a.n;
    const unsigned long long unreached = ((unsigned long long)inf_key<DT>() << 32) | NO_PRED;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        // t = inf, t[s] = 0 (Fig. 1); the predecessor of s is s
        a.packed[v] = v == a.src ? (unsigned long long)a.src : unreached;
        a.near_stamp[v] = v == a.src ? 1u : 0u;
        a.s_stamp[v] = v == a.src ? 1u : 0u;
        a.b_stamp[v] = 0u;
        a.ov_flag[v] = 0u;
    }
    {
        // directories of F0 and S0, which hold the source's entry (0, offset 0):
        // boundary 0 lies in the entry's own units, every later one in its arcs
        const uint4 vs = a.vinfo[a.src];
        const uint32_t dl = vs.y - vs.x, dh = vs.z - vs.y;
        const uint32_t nl = dl ? (uint32_t)(((unsigned long long)kEntryCost + dl + kDirChunk - 1u) / kDirChunk) : 0u;
        const uint32_t nh = dh ? (uint32_t)(((unsigned long long)kEntryCost + dh + kDirChunk - 1u) / kDirChunk) : 0u;
        uint2 *dF = a.dir, *dS = a.dir + 2ull * a.dcap;
        for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nl; c += gridDim.x * blockDim.x)
            dF[c] = c ? make_uint2(1u, dl) : make_uint2(0u, 0u);
        for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nh; c += gridDim.x * blockDim.x)
            dS[c] = c ? make_uint2(1u, dh) : make_uint2(0u, 0u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *c = a.ctl;
        const uint4 vs = a.vinfo[a.src];
        c->bar_count = 0u;
        c->err = 0;
        c->ovf = 0u;
        c->t_first = 0ull;
        SerialState s{};
        s.mode = MODE_LIGHT;      // B_0 = {s}
        s.qstamp = 1u;
        s.sround = 1u;
        s.bucket = 0;
        s.wbase = 0;
        s.st[ST_BUCKETS] = 1;
        s.t_start = s.t_last = globaltimer();
        for (int t = 0; t <= (int)kSlots; ++t) c->thr[t] = bucket_floor_key(t, DT, a.delta);
        s.T = c->thr[1];
        c->ss = s;
        c->ctrF[0] = (vs.y > vs.x) ? ((1ull << 32) | (vs.y - vs.x)) : 0ull;
        c->ctrF[1] = 0ull;
        c->ctrS[0] = (vs.z > vs.y) ? ((1ull << 32) | (vs.z - vs.y)) : 0ull;
        c->ctrS[1] = 0ull;
        for (int t = 0; t < (int)kSlots; ++t) { c->ctrSL[t] = 0ull; c->nSH[t] = 0u; }
        c->nOV[0] = c->nOV[1] = 0u;
        c->ov_min = inf_key<DT>();
        PhaseDesc d{};
        d.mode = MODE_LIGHT;
        d.slot = kNoSlot;
        d.qstamp = 1u;
        d.sstamp = 1u;
        d.T = s.T;
        d.count = (uint32_t)(c->ctrF[0] >> 32);
        d.arcs = (uint32_t)c->ctrF[0];
        d.solo = d.arcs <= a.solo_work ? 1u : 0u;
        c->desc = d;
        for (uint32_t l = 0; l < (uint32_t)kViewWords; ++l) c->view[l] = view_field(d, 0, l);   // phase 0
        a.F0[0] = make_uint2(a.src, 0u);
        a.S0[0] = make_uint2(a.src, 0u);
    }
}

template <int DT>
__global__ void k_unpack(SolveArgs a, void *dist, int32_t *pred) {
    if (vload(&a.ctl->err) != 0) return;          // outputs are written only on success
    const uint32_t n = a.n;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const unsigned long long p = a.packed[v];
        const uint32_t k = (uint32_t)(p >> 32);
        if (DT == DSSSP_F32) ((float *)dist)[v] = __uint_as_float(k);
        else ((int32_t *)dist)[v] = (int32_t)k;
        if (pred) pred[v] = v == a.src ? (int32_t)a.src : (k >= inf_key<DT>() ? -1 : (int32_t)(uint32_t)p);
    }
}

int grid_for(uint32_t n, int block) {
    long long g = ((long long)n + block - 1) / block;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_init(const SolveArgs &a, cudaStream_t st) {
    if (a.dtype == DSSSP_F32) k_init<DSSSP_F32><<<grid_for(a.n, 256), 256, 0, st>>>(a);
    else k_init<DSSSP_I32><<<grid_for(a.n, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

uint32_t solve_dir_entries(uint32_t n, uint32_t m) {
    return (uint32_t)(((unsigned long long)n * kEntryCost + m) / kDirChunk + 2u);
}

size_t stage_bytes(int block) { return (size_t)(block / 32) * sizeof(WarpStage); }

// Allow the largest staging area on every kernel that uses it (once per device).
cudaError_t allow_stage_smem() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    const int bytes = (int)stage_bytes(512);
    const void *fns[] = {
        (const void *)k_solve_persistent<DSSSP_F32>, (const void *)k_solve_persistent<DSSSP_I32>,
        (const void *)k_phase<DSSSP_F32, MODE_LIGHT>, (const void *)k_phase<DSSSP_I32, MODE_LIGHT>,
        (const void *)k_phase<DSSSP_F32, MODE_HEAVY>, (const void *)k_phase<DSSSP_I32, MODE_HEAVY>,
        (const void *)k_phase<DSSSP_F32, MODE_REBIN>, (const void *)k_phase<DSSSP_I32, MODE_REBIN>,
        (const void *)k_phase<DSSSP_F32, MODE_FUSED>, (const void *)k_phase<DSSSP_I32, MODE_FUSED>};
    for (const void *f : fns) {
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
    }
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

cudaError_t solve_occupancy(int block, int *blocks_per_sm) {
    cudaError_t e = allow_stage_smem();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_solve_persistent<DSSSP_F32>, block,
                                                         stage_bytes(block));
}

cudaError_t launch_solve_persistent(const SolveArgs &a, int grid, int block, cudaStream_t st) {
    void *args[] = {(void *)&a};
    const void *fn = a.dtype == DSSSP_F32 ? (const void *)k_solve_persistent<DSSSP_F32>
                                          : (const void *)k_solve_persistent<DSSSP_I32>;
    cudaError_t e = allow_stage_smem();
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, stage_bytes(block), st);
}

cudaError_t launch_phase_stepped(const SolveArgs &a, uint32_t mode, int grid, int block, cudaStream_t st) {
    cudaError_t e = allow_stage_smem();
    if (e != cudaSuccess) return e;
    const size_t sb = stage_bytes(block);
#define DSSSP_PHASE_CASE(M)                                                              \
    case M:                                                                              \
        if (a.dtype == DSSSP_F32) k_phase<DSSSP_F32, M><<<grid, block, sb, st>>>(a);     \
        else k_phase<DSSSP_I32, M><<<grid, block, sb, st>>>(a);                         \
        break;
    switch (mode) {
        DSSSP_PHASE_CASE(MODE_LIGHT)
        DSSSP_PHASE_CASE(MODE_HEAVY)
        DSSSP_PHASE_CASE(MODE_FUSED)
        DSSSP_PHASE_CASE(MODE_REBIN)
    default: break;
    }
#undef DSSSP_PHASE_CASE
    return cudaGetLastError();
}

cudaError_t launch_serial_step(const SolveArgs &a, cudaStream_t st) {
    if (a.dtype == DSSSP_F32) k_serial<DSSSP_F32><<<1, 32, 0, st>>>(a);
    else k_serial<DSSSP_I32><<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_verify_overflow(const SolveArgs &a, int grid, int block, cudaStream_t st) {
    if (a.dtype == DSSSP_F32) k_verify_overflow<DSSSP_F32><<<grid, block, 0, st>>>(a);
    else k_verify_overflow<DSSSP_I32><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const SolveArgs &a, void *dist, int32_t *pred, cudaStream_t st) {
    if (a.dtype == DSSSP_F32) k_unpack<DSSSP_F32><<<grid_for(a.n, 256), 256, 0, st>>>(a, dist, pred);
    else k_unpack<DSSSP_I32><<<grid_for(a.n, 256), 256, 0, st>>>(a, dist, pred);
    return cudaGetLastError();
}

}  // namespace dsssp
