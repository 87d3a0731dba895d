// solve.cu -- the delta-stepping hot path on the GPU (Fig. 1; Sections III-IV).
//
// One solve is a sequence of grid-wide phases:
//   LIGHT   relax the light arcs of the frontier F (the vertices of bucket i
//           whose distances have not been relaxed yet): t_Req = A_L^T (t o t_Bi),
//           fused with the re-introduction filter (t_Req < t) o t_Bi and with
//           t = min(t, t_Req) (Section IV-C; the fusion of Section VI-B) through
//           one 64-bit atomicMin per arc on packed[v] = key(t[v]) << 32 | pred[v];
//   HEAVY   relax the heavy arcs of S, the vertices processed in bucket i:
//           t_Req = A_H^T (t o S) (Section III-D, Fig. 1);
//   SELECT  the next non-empty bucket: i = bucket(min key of the far pile),
//           then the far pile is compacted into F and S (Fig. 1's outer loop;
//           empty buckets are skipped).
// A vertex whose distance strictly decreases into bucket <= i is queued once
// per phase: its light segment goes to the next F and, once per bucket, its
// heavy segment to S (S = S u t_Bi, Fig. 1). A decrease into a later bucket
// puts it on the far pile.
//
// Load balance: F and S entries carry their arc offset within the list, so a
// phase splits the list's flattened arcs into equal contiguous slices, one per
// warp (merge-path). Each warp finds its first entry with a 32-ary search and
// walks a 32-entry window of the list; each 32-arc step maps arcs to owners
// (one entry for all lanes, or a scatter and a prefix-max). A hub's arcs are
// spread over the whole grid. A warp keeps kIlp steps in flight.
//
// DSSSP_MODE_PERSISTENT runs all phases in one cooperative launch; every
// barrier wait is bounded by timeout_ns and ends the kernel with
// DSSSP_ERR_TIMEOUT instead of hanging. DSSSP_MODE_STEPPED launches one kernel
// per phase and runs the serial step as a 1-thread kernel.
#include "dsssp_internal.cuh"

namespace dsssp {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kMaxWarps = 16;          // blocks of at most 512 threads
constexpr int kIlp = 4;                // independent 32-arc steps per warp iteration
constexpr uint32_t kMinSlice = 32u * kIlp;

enum FarFlag : uint32_t { FAR_NONE = 0, FAR_LIVE = 1, FAR_STALE = 2 };

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ T vload(const T *p) { return *(const volatile T *)p; }

// d (+) w on keys: float32 add rounded to nearest (+inf on overflow), or int32
// add saturated at INT32_MAX. Both operands are below 2^31 for int32.
template <int DT>
__device__ __forceinline__ uint32_t key_add(uint32_t dkey, uint32_t wbits) {
    if (DT == DSSSP_F32) {
        return __float_as_uint(__fadd_rn(__uint_as_float(dkey), __uint_as_float(wbits)));
    } else {
        uint32_t s = dkey + wbits;
        return s >= KEY_INF_I32 ? KEY_INF_I32 : s;
    }
}

template <int DT>
__device__ __forceinline__ constexpr uint32_t inf_key() {
    return DT == DSSSP_F32 ? KEY_INF_F32 : KEY_INF_I32;
}

// ---------------------------------------------------------------------------
// Per-warp staging of pushes in shared memory: a list counter is touched once
// per 32 staged entries, not once per 32-arc step, and list stores are 32-wide.
struct WarpStage {
    uint32_t fv[64], fd[64], fb[64];     // next-frontier entries (vertex, light degree, begin)
    uint32_t sv[64], sd[64], sb[64];     // S entries (vertex, heavy degree, begin)
    uint32_t far[64];                    // far-pile entries
};

// Write n <= 32 staged segment entries (lanes < n) to an F or S list.
__device__ __forceinline__ void flush_seg(const uint32_t *bv, const uint32_t *bd, const uint32_t *bb, uint32_t n,
                                          uint4 *list, unsigned long long *ctr) {
    const uint32_t lane = lane_id();
    const bool has = lane < n;
    const uint32_t v = has ? bv[lane] : 0u, d = has ? bd[lane] : 0u, b = has ? bb[lane] : 0u;
    uint32_t incl = d;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, o);
        if ((int)lane >= o) incl += t;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(ctr, ((unsigned long long)n << 32) | tot);
    old = __shfl_sync(FULL, old, 0);
    if (has) list[(uint32_t)(old >> 32) + lane] = make_uint4(v, (uint32_t)old + incl - d, b, 0u);
}

__device__ __forceinline__ void flush_ids(const uint32_t *bv, uint32_t n, uint32_t *list, uint32_t *counter) {
    const uint32_t lane = lane_id();
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(counter, n);
    base = __shfl_sync(FULL, base, 0);
    if (lane < n) list[base + lane] = bv[lane];
}

// ---------------------------------------------------------------------------
// Block-local accumulators flushed to the control block.
struct BlockAcc {
    uint32_t far_min;
    unsigned long long arcs_light, arcs_heavy, improvements, far_scanned;
};

// Pending pushes of one lane in one step.
struct Push {
    bool f, s, far;
    uint32_t fdeg, fbeg, sdeg, sbeg;
};

// The warp's staged counts. The destination lists follow from the phase
// descriptor (in shared memory) and are resolved only when a buffer is flushed,
// so they do not hold registers in the relaxation loop. LIGHT/HEAVY append to
// the current far list; SELECT rebuilds the far pile into the other one.
struct PushCnt {
    uint32_t nf, ns, nfar;
};

__device__ __forceinline__ uint4 *dst_F(const SolveArgs &a, const PhaseDesc &d) { return d.cur ? a.F0 : a.F1; }
__device__ __forceinline__ unsigned long long *ctr_F(const SolveArgs &a, const PhaseDesc &d) {
    return &a.ctl->ctrF[d.cur ^ 1u];
}
__device__ __forceinline__ uint4 *dst_S(const SolveArgs &a, const PhaseDesc &d) { return d.spush ? a.S1 : a.S0; }
__device__ __forceinline__ unsigned long long *ctr_S(const SolveArgs &a, const PhaseDesc &d) {
    return &a.ctl->ctrS[d.spush];
}
__device__ __forceinline__ uint32_t far_list_index(const PhaseDesc &d) {
    return d.mode == MODE_SELECT ? d.far_cur ^ 1u : d.far_cur;
}
__device__ __forceinline__ uint32_t *dst_FAR(const SolveArgs &a, const PhaseDesc &d) {
    return far_list_index(d) ? a.FAR1 : a.FAR0;
}
__device__ __forceinline__ uint32_t *ctr_FAR(const SolveArgs &a, const PhaseDesc &d) {
    return &a.ctl->nFar[far_list_index(d)];
}

// Stage one (vertex, degree, begin) per pushing lane; flush 32 when full.
template <int LIST>
__device__ __forceinline__ void stage_seg(const SolveArgs &a, const PhaseDesc &d, bool pred, uint32_t v,
                                          uint32_t deg, uint32_t beg, uint32_t *bv, uint32_t *bd, uint32_t *bb,
                                          uint32_t &cnt) {
    const uint32_t mask = __ballot_sync(FULL, pred);
    if (mask == 0u) return;
    const uint32_t lane = lane_id();
    if (pred) {
        const uint32_t k = cnt + __popc(mask & lanemask_lt());
        bv[k] = v; bd[k] = deg; bb[k] = beg;
    }
    cnt += __popc(mask);
    __syncwarp();
    if (cnt >= 32u) {
        if (LIST == 0) flush_seg(bv, bd, bb, 32u, dst_F(a, d), ctr_F(a, d));
        else flush_seg(bv, bd, bb, 32u, dst_S(a, d), ctr_S(a, d));
        const uint32_t rest = cnt - 32u;
        uint32_t x = 0, y = 0, z = 0;
        if (lane < rest) { x = bv[32 + lane]; y = bd[32 + lane]; z = bb[32 + lane]; }
        __syncwarp();
        if (lane < rest) { bv[lane] = x; bd[lane] = y; bb[lane] = z; }
        __syncwarp();
        cnt = rest;
    }
}

__device__ __forceinline__ void stage_far(const SolveArgs &a, const PhaseDesc &d, bool pred, uint32_t v,
                                          uint32_t *bv, uint32_t &cnt) {
    const uint32_t mask = __ballot_sync(FULL, pred);
    if (mask == 0u) return;
    const uint32_t lane = lane_id();
    if (pred) bv[cnt + __popc(mask & lanemask_lt())] = v;
    cnt += __popc(mask);
    __syncwarp();
    if (cnt >= 32u) {
        flush_ids(bv, 32u, dst_FAR(a, d), ctr_FAR(a, d));
        const uint32_t rest = cnt - 32u;
        uint32_t x = 0;
        if (lane < rest) x = bv[32 + lane];
        __syncwarp();
        if (lane < rest) bv[lane] = x;
        __syncwarp();
        cnt = rest;
    }
}

__device__ __forceinline__ void stage_pushes(const SolveArgs &a, const PhaseDesc &d, PushCnt &q, WarpStage &ws,
                                             const Push &p, uint32_t v) {
    if (__ballot_sync(FULL, p.f || p.s || p.far) == 0u) return;
    stage_seg<0>(a, d, p.f, v, p.fdeg, p.fbeg, ws.fv, ws.fd, ws.fb, q.nf);
    stage_seg<1>(a, d, p.s, v, p.sdeg, p.sbeg, ws.sv, ws.sd, ws.sb, q.ns);
    stage_far(a, d, p.far, v, ws.far, q.nfar);
}

// Flush the partially filled staging buffers (end of a phase).
__device__ __forceinline__ void drain_pushes(const SolveArgs &a, const PhaseDesc &d, PushCnt &q, WarpStage &ws) {
    if (q.nf) flush_seg(ws.fv, ws.fd, ws.fb, q.nf, dst_F(a, d), ctr_F(a, d));
    if (q.ns) flush_seg(ws.sv, ws.sd, ws.sb, q.ns, dst_S(a, d), ctr_S(a, d));
    if (q.nfar) flush_ids(ws.far, q.nfar, dst_FAR(a, d), ctr_FAR(a, d));
    __syncwarp();
    q.nf = q.ns = q.nfar = 0u;
}

// Queue v for bucket i (its key is now below T): once per phase into the next
// F (its light segment), once per bucket into S (its heavy segment). A live
// far-pile entry of v becomes stale. The loads are issued together with the
// stamp exchange; they are simply unused when v is already queued.
__device__ __forceinline__ void queue_near(const SolveArgs &a, const PhaseDesc &d, uint32_t v, Push &p,
                                           bool mark_far) {
    const uint32_t prev = atomicExch(a.near_stamp + v, d.qstamp);
    const uint4 vi = a.vinfo[v];
    const uint32_t ss = __ldcg(a.s_stamp + v);
    const uint32_t ff = mark_far ? __ldcg(a.far_flag + v) : FAR_NONE;
    if (prev == d.qstamp) return;
    p.fdeg = vi.y - vi.x;
    p.fbeg = vi.x;
    p.f = p.fdeg != 0u;
    if (ss != d.sstamp) {
        a.s_stamp[v] = d.sstamp;
        p.sdeg = vi.z - vi.y;
        p.sbeg = vi.y;
        p.s = p.sdeg != 0u;
    }
    if (ff == FAR_LIVE) a.far_flag[v] = FAR_STALE;
}

// relax(v, new_dist) of Section III-C, after the packed atomicMin found a strict
// decrease of t[v]: v re-enters bucket i ((t_Req < t) o t_Bi) or goes to the far pile.
template <int DT>
__device__ __forceinline__ void on_improved(const SolveArgs &a, const PhaseDesc &d, uint32_t v, uint32_t ckey,
                                            Push &p, uint32_t &far_min, uint32_t &improved) {
    ++improved;
    if (ckey < d.T) {
        queue_near(a, d, v, p, true);
    } else {
        far_min = min(far_min, ckey);
        p.far = atomicExch(a.far_flag + v, FAR_LIVE) == FAR_NONE;
    }
}

// LIGHT / HEAVY: relax the arcs of a list, split evenly over the warps.
template <int DT, bool LIGHT>
__device__ void phase_arcs(const SolveArgs &a, const PhaseDesc &d, BlockAcc &acc, int *slot, WarpStage *stage,
                           uint32_t gw, uint32_t nw_all) {
    const uint32_t lane = lane_id();
    const uint4 *list = LIGHT ? (d.cur ? a.F1 : a.F0) : (d.scur ? a.S1 : a.S0);
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(list) + 1;   // offs[4 * j]
    const uint32_t count = d.count;
    const uint32_t E = d.arcs;
    // at least kMinSlice arcs per warp: small phases use few warps
    const uint32_t want_w = (E + kMinSlice - 1u) / kMinSlice;
    const uint32_t nw = want_w < nw_all ? want_w : nw_all;
    uint32_t far_min = inf_key<DT>();
    uint32_t improved = 0;
    if (gw < nw) {
        const uint32_t e0 = (uint32_t)(((unsigned long long)E * gw) / nw);
        const uint32_t e1 = (uint32_t)(((unsigned long long)E * (gw + 1)) / nw);
        PushCnt q{};
        WarpStage &ws = stage[threadIdx.x >> 5];
        // last entry whose offset is <= e0 (32-ary search; entry lo always qualifies)
        uint32_t lo = 0, hi = count;
        while (hi - lo > 32u) {
            const uint32_t step = (hi - lo + 31u) >> 5;
            const uint32_t p = lo + lane * step;
            const bool ok = p < hi && __ldcg(offs + 4ull * p) <= e0;
            const uint32_t k = 31u - __clz(__ballot_sync(FULL, ok));
            lo += k * step;
            hi = min(hi, lo + step);
        }
        {
            const uint32_t p = lo + lane;
            const bool ok = p < hi && __ldcg(offs + 4ull * p) <= e0;
            lo += 31u - __clz(__ballot_sync(FULL, ok));
        }
        // window: lane k holds entry jw + k; wend = arc offset just past the window
        uint32_t jw = lo, wv = 0, woff = 0xFFFFFFFFu, wbeg = 0, wkey = inf_key<DT>(), wend = 0;
        auto load_window = [&](uint32_t j) {
            const uint32_t idx = j + lane;
            if (idx < count) {
                const uint4 en = __ldcs(list + idx);
                wv = en.x < a.n ? en.x : 0u;          // defensive: ids come from device lists
                woff = en.y;
                wbeg = en.z;
                wkey = (uint32_t)(__ldcg(a.packed + wv) >> 32);
            } else {
                wv = 0; woff = 0xFFFFFFFFu; wbeg = 0; wkey = inf_key<DT>();
            }
            wend = (j + 32u < count) ? __ldcg(offs + 4ull * (j + 32u)) : E;
        };
        load_window(jw);
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
                        load_window(jw);
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
                    ok[k] = e < e1 && ai[k] < a.m;     // defensive bound; true when lists are consistent
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
            #pragma unroll
            for (int k = 0; k < kIlp; ++k) {
                Push p{};
                const unsigned long long cand = ((unsigned long long)ck[k] << 32) | ov[k];
                if (cand < old[k] && (uint32_t)(old[k] >> 32) > ck[k])      // strict distance decrease
                    on_improved<DT>(a, d, arc[k].x, ck[k], p, far_min, improved);
                stage_pushes(a, d, q, ws, p, arc[k].x);
            }
        }
        drain_pushes(a, d, q, ws);
        if (lane == 0) {
            if (LIGHT) atomicAdd(&acc.arcs_light, (unsigned long long)(e1 - e0));
            else atomicAdd(&acc.arcs_heavy, (unsigned long long)(e1 - e0));
        }
    }
    if (far_min < inf_key<DT>()) atomicMin(&acc.far_min, far_min);
    if (improved) atomicAdd(&acc.improvements, (unsigned long long)improved);
}

// SELECT: compact the far pile. Live entries whose key is below T (bucket <= i)
// are queued into F and S; the rest stay, and their minimum key bounds the next
// bucket; stale entries are dropped. Each lane examines kIlp entries at once.
template <int DT>
__device__ void phase_select(const SolveArgs &a, const PhaseDesc &d, BlockAcc &acc, WarpStage *stage,
                             uint32_t gw, uint32_t nw) {
    const uint32_t lane = lane_id();
    const uint32_t *in = d.far_cur ? a.FAR1 : a.FAR0;
    const uint32_t count = d.count;
    uint32_t far_min = inf_key<DT>();
    PushCnt q{};
    WarpStage &ws = stage[threadIdx.x >> 5];
    const unsigned long long stride = (unsigned long long)nw * 32u * kIlp;
    for (unsigned long long base = (unsigned long long)gw * 32u * kIlp; base < count; base += stride) {
        uint32_t v[kIlp], f[kIlp], k[kIlp];
        #pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const unsigned long long idx = base + 32u * j + lane;
            v[j] = idx < count ? __ldcs(in + idx) : 0xFFFFFFFFu;
        }
        #pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            f[j] = v[j] < a.n ? __ldcg(a.far_flag + v[j]) : FAR_NONE;
            k[j] = v[j] < a.n ? (uint32_t)(__ldcg(a.packed + v[j]) >> 32) : inf_key<DT>();
        }
        #pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            Push p{};
            if (f[j] == FAR_LIVE) {
                if (k[j] < d.T) {
                    a.far_flag[v[j]] = FAR_NONE;
                    queue_near(a, d, v[j], p, false);
                } else {
                    p.far = true;                      // stays on the (rebuilt) far pile
                    far_min = min(far_min, k[j]);
                }
            } else if (f[j] == FAR_STALE) {
                a.far_flag[v[j]] = FAR_NONE;          // stale entry dropped
            }
            stage_pushes(a, d, q, ws, p, v[j]);
        }
    }
    drain_pushes(a, d, q, ws);
    if (far_min < inf_key<DT>()) atomicMin(&acc.far_min, far_min);
    if (gw == 0 && lane == 0) atomicAdd(&acc.far_scanned, (unsigned long long)count);
}

// ---------------------------------------------------------------------------
// Serial step: runs on one thread after every block has finished a phase.
// Loads the serial state and the list counters in one batch, decides the next
// phase (the control flow of Fig. 1) in registers, resets consumed counters
// and publishes the next PhaseDesc.
template <int DT>
__device__ void serial_step(const SolveArgs &a) {
    Ctl *c = a.ctl;
    SerialState s;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(&c->ss);
        uint4 *dst = reinterpret_cast<uint4 *>(&s);
        #pragma unroll
        for (int k = 0; k < (int)(sizeof(SerialState) / 16); ++k) dst[k] = __ldcg(src + k);
    }
    const unsigned long long cf0 = __ldcg(&c->ctrF[0]), cf1 = __ldcg(&c->ctrF[1]);
    const unsigned long long cs0 = __ldcg(&c->ctrS[0]), cs1 = __ldcg(&c->ctrS[1]);
    const uint32_t nfar0 = __ldcg(&c->nFar[0]), nfar1 = __ldcg(&c->nFar[1]);
    const uint32_t far_min = __ldcg(&c->far_min);
    const uint64_t t_first = __ldcg(&c->t_first);
    const uint64_t now = globaltimer();
    const uint64_t dt = now - s.t_last;
    if (t_first > s.t_last && t_first <= now) {      // persistent mode only
        s.st[ST_NSFIRST] += (long long)(t_first - s.t_last);
        s.st[ST_NSSPREAD] += (long long)(now - t_first);
    }
    s.t_last = now;
    unsigned long long ctrF[2] = {cf0, cf1}, ctrS[2] = {cs0, cs1};
    uint32_t nFar[2] = {nfar0, nfar1};
    bool resetF = false, resetS = false, resetFar = false;   // consumed list counters
    uint32_t rF = 0, rS = 0, rFar = 0;
    const uint32_t mode = s.mode;
    PhaseDesc nd{};
    if (mode == MODE_LIGHT) s.st[ST_NSLIGHT] += (long long)dt;
    else if (mode == MODE_HEAVY) s.st[ST_NSHEAVY] += (long long)dt;
    else if (mode == MODE_SELECT) s.st[ST_NSSELECT] += (long long)dt;
    s.phases += 1;
    bool done = false;
    if (s.phases >= a.max_phases) {
        atomicCAS(&c->err, 0, (int)DSSSP_ERR_NOT_CONVERGED);
        done = true;
    } else {
        switch (mode) {
        case MODE_LIGHT:
            s.st[ST_LIGHT] += 1;
            s.st[ST_VLIGHT] += (long long)(ctrF[s.cur] >> 32);
            resetF = true; rF = s.cur; ctrF[s.cur] = 0ull;
            break;
        case MODE_HEAVY:
            s.st[ST_HEAVY] += 1;
            s.st[ST_VHEAVY] += (long long)(ctrS[s.scur] >> 32);
            resetS = true; rS = s.scur; ctrS[s.scur] = 0ull;
            s.scur ^= 1u;               // S pushed during the heavy pass (a re-opened bucket)
            s.sround += 1u;
            break;
        case MODE_SELECT:
            s.st[ST_SELECT] += 1;
            resetFar = true; rFar = s.far_cur; nFar[s.far_cur] = 0u;
            s.far_cur ^= 1u;
            break;
        default:
            done = true;
            break;
        }
    }
    uint32_t next_mode = MODE_DONE;
    bool reset_min = false;
    if (!done) {
        s.qstamp += 1u;                            // every phase queues under a fresh stamp
        const uint32_t nxt = s.cur ^ 1u;
        if ((ctrF[nxt] >> 32) != 0ull) {           // inner loop of Fig. 1: while t_Bi != 0
            if (mode == MODE_SELECT) s.st[ST_BUCKETS] += 1;
            s.cur = nxt;
            next_mode = MODE_LIGHT;
        } else if ((ctrS[s.scur] >> 32) != 0ull) { // bucket settled: heavy pass over S
            if (mode == MODE_SELECT) s.st[ST_BUCKETS] += 1;
            next_mode = MODE_HEAVY;
        } else if (far_min >= inf_key<DT>() && nFar[s.far_cur] == 0u) {
            next_mode = MODE_DONE;                 // nothing left in any bucket
        } else {                                   // next non-empty bucket
            if (far_min >= inf_key<DT>()) {
                s.T = 0u;                          // only stale entries remain: drop them
            } else {
                const int64_t i = bucket_of_key(far_min, DT, a.delta);
                s.bucket = i;
                s.T = i < INT64_MAX ? bucket_floor_key(i + 1, DT, a.delta) : 0u;
                if (s.T <= far_min) s.T = far_min + 1u;     // always take the smallest live key
            }
            reset_min = true;
            next_mode = MODE_SELECT;
        }
    }
    if (next_mode == MODE_DONE) s.st[ST_NSTOTAL] = (long long)(now - s.t_start);
    s.mode = next_mode;
    nd.mode = next_mode;
    nd.cur = s.cur;
    nd.scur = s.scur;
    // S pushes: into the current S, except during a heavy pass, which feeds the next one
    nd.spush = next_mode == MODE_HEAVY ? s.scur ^ 1u : s.scur;
    nd.sstamp = next_mode == MODE_HEAVY ? s.sround + 1u : s.sround;
    nd.far_cur = s.far_cur;
    nd.qstamp = s.qstamp;
    nd.T = s.T;
    if (next_mode == MODE_LIGHT) { nd.count = (uint32_t)(ctrF[s.cur] >> 32); nd.arcs = (uint32_t)ctrF[s.cur]; }
    else if (next_mode == MODE_HEAVY) { nd.count = (uint32_t)(ctrS[s.scur] >> 32); nd.arcs = (uint32_t)ctrS[s.scur]; }
    else if (next_mode == MODE_SELECT) nd.count = nFar[s.far_cur];
    // little work: one block runs the phase without a grid-wide barrier
    nd.solo = (next_mode == MODE_SELECT ? nd.count : nd.arcs) <= a.solo_work ? 1u : 0u;
    // write back: consumed counters, serial state, descriptor
    if (resetF) c->ctrF[rF] = 0ull;
    if (resetS) c->ctrS[rS] = 0ull;
    if (resetFar) c->nFar[rFar] = 0u;
    if (reset_min) c->far_min = inf_key<DT>();
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(&s);
        uint4 *dst = reinterpret_cast<uint4 *>(&c->ss);
        #pragma unroll
        for (int k = 0; k < (int)(sizeof(SerialState) / 16); ++k) dst[k] = src[k];
        const uint4 *ds = reinterpret_cast<const uint4 *>(&nd);
        uint4 *dd = reinterpret_cast<uint4 *>(&c->desc);
        #pragma unroll
        for (int k = 0; k < 4; ++k) dd[k] = ds[k];
    }
}

__device__ __forceinline__ void read_desc(const Ctl *c, PhaseDesc &d) {
    const uint4 *src = reinterpret_cast<const uint4 *>(&c->desc);
    uint4 *dst = reinterpret_cast<uint4 *>(&d);
    #pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = __ldcg(src + k);
}

__device__ __forceinline__ void flush_far_min(Ctl *c, BlockAcc &acc, uint32_t inf) {
    if (acc.far_min < inf) {
        atomicMin(&c->far_min, acc.far_min);
        acc.far_min = inf;
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
    acc.far_min = inf_key<DT>();
    acc.arcs_light = acc.arcs_heavy = acc.improvements = acc.far_scanned = 0;
}

// Grid-wide barrier with a serial step, every wait bounded by timeout_ns.
// Returns false when the solve must stop (done, error recorded, or timed out).
// With run_serial false (after a solo stretch, whose serial steps block 0
// already ran) the last arrival only releases; blocks that wait through a solo
// stretch poll slowly so that they do not load the L2 the solo block uses.
template <int DT>
__device__ bool grid_barrier(const SolveArgs &a, BlockAcc &acc, int *s_ok, bool run_serial, bool patient) {
    __syncthreads();
    if (threadIdx.x == 0) {
        Ctl *c = a.ctl;
        flush_far_min(c, acc, inf_key<DT>());
        __threadfence();
        const unsigned gen = vload(&c->bar_gen);
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (run_serial && arrived == 0u) c->t_first = globaltimer();   // phase-time diagnostics
        if (arrived == a.nblocks - 1u) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            if (run_serial) serial_step<DT>(a);
            __threadfence();
            atomicExch(&c->bar_gen, gen + 1u);
        } else {
            // bounded wait: timeout_ns without progress (a solo block's serial
            // steps advance ss.phases, which restarts the clock)
            uint64_t t0 = globaltimer();
            int64_t seen = patient ? vload(&c->ss.phases) : 0;
            while (vload(&c->bar_gen) == gen) {
                if (vload(&c->err) != 0) break;
                const uint64_t now = globaltimer();
                if (patient) {
                    const int64_t ph = vload(&c->ss.phases);
                    if (ph != seen) { seen = ph; t0 = now; }
                }
                if ((int64_t)(now - t0) > a.timeout_ns) {
                    atomicCAS(&c->err, 0, (int)DSSSP_ERR_TIMEOUT);
                    break;
                }
                if (patient) __nanosleep(500);
            }
            __threadfence();
        }
        *s_ok = vload(&c->err) == 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <int DT>
__device__ __forceinline__ void run_phase(const SolveArgs &a, const PhaseDesc &d, BlockAcc &acc, int *slot,
                                          WarpStage *stage, uint32_t gw, uint32_t nw) {
    switch (d.mode) {
    case MODE_LIGHT: phase_arcs<DT, true>(a, d, acc, slot, stage, gw, nw); break;
    case MODE_HEAVY: phase_arcs<DT, false>(a, d, acc, slot, stage, gw, nw); break;
    case MODE_SELECT: phase_select<DT>(a, d, acc, stage, gw, nw); break;
    default: break;
    }
}

template <int DT>
__global__ void __launch_bounds__(512, 2) k_solve_persistent(SolveArgs a) {
    __shared__ int slot[kMaxWarps * 32];
    __shared__ WarpStage stage[kMaxWarps];
    __shared__ PhaseDesc s_desc;
    __shared__ BlockAcc acc;
    __shared__ int s_ok;
    if (a.test_hook == DSSSP_HOOK_STALL_BARRIER && blockIdx.x == 1) return;
    if (threadIdx.x == 0) acc_init<DT>(acc);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    bool have_desc = false;
    for (;;) {
        if (!have_desc) {
            if (threadIdx.x == 0) read_desc(a.ctl, s_desc);
            __syncthreads();
        }
        have_desc = false;
        if (s_desc.mode == MODE_DONE) break;
        // A solo phase (little work) runs on block 0 only: its phases follow each
        // other with block-level synchronisation and the serial step in thread 0,
        // while the other blocks wait in the grid barrier until a phase with work
        // for the whole grid (or the end) comes.
        const bool solo = s_desc.solo != 0u;
        if (!solo || blockIdx.x == 0) run_phase<DT>(a, s_desc, acc, slot, stage, solo ? wib : gw, solo ? nwb : nw);
        if (solo && blockIdx.x == 0) {
            __threadfence();             // list entries and flags reach L2 before the serial step reads them
            __syncthreads();
            if (threadIdx.x == 0) {
                flush_far_min(a.ctl, acc, inf_key<DT>());
                __threadfence();
                serial_step<DT>(a);
                read_desc(a.ctl, s_desc);
                s_ok = vload(&a.ctl->err) == 0;
            }
            __syncthreads();
            if (!s_ok) break;
            if (s_desc.solo && s_desc.mode != MODE_DONE) {
                have_desc = true;        // next solo phase right away
                continue;
            }
            if (!grid_barrier<DT>(a, acc, &s_ok, false, false)) break;   // release the waiting blocks
        } else if (solo) {
            if (!grid_barrier<DT>(a, acc, &s_ok, false, true)) break;
        } else {
            if (!grid_barrier<DT>(a, acc, &s_ok, true, false)) break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) flush_stats(a.ctl, acc);
}

// ---- stepped mode: one launch per phase --------------------------------------
template <int DT, uint32_t MODE>
__global__ void __launch_bounds__(512, 2) k_phase(SolveArgs a) {
    __shared__ int slot[kMaxWarps * 32];
    __shared__ WarpStage stage[kMaxWarps];
    __shared__ PhaseDesc s_desc;
    __shared__ BlockAcc acc;
    if (threadIdx.x == 0) {
        read_desc(a.ctl, s_desc);
        acc_init<DT>(acc);
    }
    __syncthreads();
    const PhaseDesc &d = s_desc;
    if (d.mode != MODE) return;
    run_phase<DT>(a, d, acc, slot, stage, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                  (gridDim.x * blockDim.x) >> 5);
    __syncthreads();
    if (threadIdx.x == 0) {
        flush_far_min(a.ctl, acc, inf_key<DT>());
        flush_stats(a.ctl, acc);
    }
}

template <int DT>
__global__ void k_serial(SolveArgs a) {
    if (vload(&a.ctl->desc.mode) != MODE_DONE) serial_step<DT>(a);
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
        a.far_flag[v] = FAR_NONE;
        a.s_stamp[v] = v == a.src ? 1u : 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *c = a.ctl;
        const uint4 vs = a.vinfo[a.src];
        c->bar_count = 0u;
        c->bar_gen = 0u;
        c->err = 0;
        SerialState s{};
        s.mode = MODE_LIGHT;      // B_0 = {s}
        s.qstamp = 1u;
        s.sround = 1u;
        s.T = bucket_floor_key(1, DT, a.delta);
        s.st[ST_BUCKETS] = 1;
        s.t_start = s.t_last = globaltimer();
        c->ss = s;
        c->ctrF[0] = (vs.y > vs.x) ? ((1ull << 32) | (vs.y - vs.x)) : 0ull;
        c->ctrF[1] = 0ull;
        c->ctrS[0] = (vs.z > vs.y) ? ((1ull << 32) | (vs.z - vs.y)) : 0ull;
        c->ctrS[1] = 0ull;
        c->nFar[0] = c->nFar[1] = 0u;
        c->far_min = inf_key<DT>();
        PhaseDesc d{};
        d.mode = MODE_LIGHT;
        d.qstamp = 1u;
        d.sstamp = 1u;
        d.T = s.T;
        d.count = (uint32_t)(c->ctrF[0] >> 32);
        d.arcs = (uint32_t)c->ctrF[0];
        d.solo = d.arcs <= a.solo_work ? 1u : 0u;
        c->desc = d;
        a.F0[0] = make_uint4(a.src, 0u, vs.x, 0u);
        a.S0[0] = make_uint4(a.src, 0u, vs.y, 0u);
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

cudaError_t solve_occupancy(int block, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_solve_persistent<DSSSP_F32>, block, 0);
}

cudaError_t launch_solve_persistent(const SolveArgs &a, int grid, int block, cudaStream_t st) {
    void *args[] = {(void *)&a};
    const void *fn = a.dtype == DSSSP_F32 ? (const void *)k_solve_persistent<DSSSP_F32>
                                          : (const void *)k_solve_persistent<DSSSP_I32>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

cudaError_t launch_phase_stepped(const SolveArgs &a, uint32_t mode, int grid, int block, cudaStream_t st) {
#define DSSSP_PHASE_CASE(M)                                                              \
    case M:                                                                              \
        if (a.dtype == DSSSP_F32) k_phase<DSSSP_F32, M><<<grid, block, 0, st>>>(a);      \
        else k_phase<DSSSP_I32, M><<<grid, block, 0, st>>>(a);                          \
        break;
    switch (mode) {
        DSSSP_PHASE_CASE(MODE_LIGHT)
        DSSSP_PHASE_CASE(MODE_HEAVY)
        DSSSP_PHASE_CASE(MODE_SELECT)
    default: break;
    }
#undef DSSSP_PHASE_CASE
    return cudaGetLastError();
}

cudaError_t launch_serial_step(const SolveArgs &a, cudaStream_t st) {
    if (a.dtype == DSSSP_F32) k_serial<DSSSP_F32><<<1, 1, 0, st>>>(a);
    else k_serial<DSSSP_I32><<<1, 1, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const SolveArgs &a, void *dist, int32_t *pred, cudaStream_t st) {
    if (a.dtype == DSSSP_F32) k_unpack<DSSSP_F32><<<grid_for(a.n, 256), 256, 0, st>>>(a, dist, pred);
    else k_unpack<DSSSP_I32><<<grid_for(a.n, 256), 256, 0, st>>>(a, dist, pred);
    return cudaGetLastError();
}

}  // namespace dsssp
