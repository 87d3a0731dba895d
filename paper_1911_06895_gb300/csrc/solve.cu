// solve.cu -- the delta-stepping hot path on the GPU (Fig. 1; Sections III-IV).
//
// One solve is a sequence of grid-wide phases:
//   LIGHT   relax the light arcs of the frontier F (the vertices of bucket i
//           with unrelaxed distances): t_Req = A_L^T (t o t_Bi), fused with the
//           re-introduction filter and t = min(t, t_Req) (Section IV-C, and the
//           fusion of Section VI-B) through one 64-bit atomicMin per arc on
//           packed[v] = key(t[v]) << 32 | pred[v];
//   BIG     the same relaxation for arc segments longer than big_degree,
//           spread evenly over every warp of the grid;
//   HEAVY   relax the heavy arcs of S, the vertices processed in bucket i:
//           t_Req = A_H^T (t o S) (Section III-D, Fig. 1);
//   SELECT  the next non-empty bucket: i = bucket(min key of the far pile),
//           then the far pile is compacted into the new frontier (Fig. 1's
//           outer loop; empty buckets are skipped).
// A vertex whose distance strictly decreases is appended, once, to the next
// frontier when its new bucket is <= i, otherwise to the far pile. S is
// deduplicated with a per-bucket stamp. The phase order is decided by one
// thread in the serial step of the grid barrier.
//
// DSSSP_MODE_PERSISTENT runs all phases in one cooperative launch; every
// barrier wait is bounded by timeout_ns and ends the kernel with
// DSSSP_ERR_TIMEOUT instead of hanging. DSSSP_MODE_STEPPED launches one kernel
// per phase and runs the serial step as a 1-thread kernel (for profiling).
#include "dsssp_internal.cuh"

namespace dsssp {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kMaxWarps = 16;          // blocks of at most 512 threads

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

// Warp-aggregated append: one atomicAdd per warp, lanes write at base + rank.
// Every lane of the warp must call it.
__device__ __forceinline__ void warp_append(bool pred, uint32_t val, uint32_t *list, uint32_t *counter) {
    const uint32_t mask = __ballot_sync(FULL, pred);
    if (mask == 0u) return;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(FULL, base, leader);
    if (pred) list[base + __popc(mask & lanemask_lt())] = val;
}

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

// Per-phase constants every block reads from the control block after a barrier.
struct Desc {
    uint32_t mode, big_kind, cur, far_cur, qstamp, sround, T, count, count2;
};

// Block-local accumulators flushed to the control block.
struct BlockAcc {
    uint32_t far_min;
    unsigned long long arcs_light, arcs_heavy, improvements, far_scanned;
};

// relax(v, new_dist) of Section III-C on the packed word. Returns through
// push_near / push_far whether v must be appended to the next frontier or to
// the far pile.
template <int DT>
__device__ __forceinline__ void relax_arc(const SolveArgs &a, const Desc &d, uint32_t v, uint32_t ckey,
                                          uint32_t u, bool &push_near, bool &push_far, uint32_t &far_min,
                                          uint32_t &improved) {
    push_near = false;
    push_far = false;
    if (ckey >= inf_key<DT>()) return;
    const unsigned long long cand = ((unsigned long long)ckey << 32) | u;
    // packed[v] only decreases, so any earlier value is an upper bound: skip the
    // atomic when the request cannot win
    if (cand >= __ldcg(a.packed + v)) return;
    const unsigned long long old = atomicMin(a.packed + v, cand);
    if (cand >= old) return;
    if ((uint32_t)(old >> 32) <= ckey) return;         // equal distance: predecessor tie-break only
    ++improved;
    if (ckey < d.T) {                                  // new bucket <= i: (t_Req < t) o t_Bi
        push_near = atomicExch(a.near_stamp + v, d.qstamp) != d.qstamp;
    } else {                                           // a later bucket: far pile
        far_min = min(far_min, ckey);
        push_far = atomicExch(a.far_flag + v, 1u) == 0u;
    }
}

// LIGHT / HEAVY: every warp takes batches of 32 list entries (static round
// robin), expands their arc segments cooperatively (exclusive scan of the
// segment lengths, then 32 arcs per step), and relaxes each arc. Segments
// longer than big_degree go to the BIG list instead.
template <int DT, bool LIGHT>
__device__ void phase_segments(const SolveArgs &a, const Desc &d, BlockAcc &acc, uint32_t *sw) {
    const uint32_t lane = lane_id();
    const uint32_t wib = threadIdx.x >> 5;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t *sw_scan = sw + wib * 128;
    uint32_t *sw_beg = sw_scan + 32;
    uint32_t *sw_key = sw_scan + 64;
    uint32_t *sw_u = sw_scan + 96;
    Ctl *c = a.ctl;
    const uint32_t *list = LIGHT ? (d.cur ? a.F1 : a.F0) : a.S;
    const uint32_t count = d.count;
    uint32_t *next = d.cur ? a.F0 : a.F1;
    uint32_t *next_cnt = &c->nF[d.cur ^ 1u];
    uint32_t *farl = d.far_cur ? a.FAR1 : a.FAR0;
    uint32_t *far_cnt = &c->nFar[d.far_cur];
    uint32_t far_min = inf_key<DT>();
    uint32_t improved = 0;
    unsigned long long arcs = 0;

    for (uint32_t batch = gw; (unsigned long long)batch * 32u < count; batch += nw) {
        const uint32_t idx = batch * 32u + lane;
        const bool valid = idx < count;
        uint32_t u = 0, beg = 0, deg = 0, dkey = inf_key<DT>();
        bool addS = false;
        if (valid) {
            u = __ldcg(list + idx);
            dkey = (uint32_t)(__ldcg(a.packed + u) >> 32);
            const uint4 vi = a.vinfo[u];
            if (LIGHT) {
                beg = vi.x;
                deg = vi.y - vi.x;
                addS = __ldcg(a.s_stamp + u) != d.sround;      // S = S u B_i
                if (addS) a.s_stamp[u] = d.sround;
                if (__ldcg(a.far_flag + u) == 1u) a.far_flag[u] = 2u;   // its far entry is now stale
            } else {
                beg = vi.y;
                deg = vi.z - vi.y;
            }
            if (deg > a.big_degree) {
                const unsigned long long old =
                    atomicAdd(&c->big_ctr, (1ull << 32) | (unsigned long long)deg);
                a.BIG[(uint32_t)(old >> 32)] = make_uint4(u, (uint32_t)old, beg, 0u);
                deg = 0;
            }
        }
        if (LIGHT) warp_append(addS, u, a.S, &c->nS);

        uint32_t incl = deg;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if ((int)lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        sw_scan[lane] = incl - deg;
        sw_beg[lane] = beg;
        sw_key[lane] = dkey;
        sw_u[lane] = u;
        __syncwarp();
        arcs += total;
        uint32_t j = 0;
        for (uint32_t base = 0; base < total; base += 32u) {
            const uint32_t e = base + lane;
            bool pn = false, pf = false;
            uint32_t v = 0;
            if (e < total) {
                while (j < 31u && sw_scan[j + 1] <= e) ++j;
                const uint2 arc = a.arcs[sw_beg[j] + (e - sw_scan[j])];
                v = arc.x;
                relax_arc<DT>(a, d, v, key_add<DT>(sw_key[j], arc.y), sw_u[j], pn, pf, far_min, improved);
            }
            warp_append(pn, v, next, next_cnt);
            warp_append(pf, v, farl, far_cnt);
        }
        __syncwarp();
    }
    if (lane == 0 && arcs) {
        if (LIGHT) atomicAdd(&acc.arcs_light, arcs); else atomicAdd(&acc.arcs_heavy, arcs);
    }
    if (far_min < inf_key<DT>()) atomicMin(&acc.far_min, far_min);
    if (improved) atomicAdd(&acc.improvements, (unsigned long long)improved);
}

// BIG: the flattened arcs of the long segments, split evenly over all warps.
template <int DT>
__device__ void phase_big(const SolveArgs &a, const Desc &d, BlockAcc &acc) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nb = d.count;        // entries
    const uint32_t E = d.count2;        // arcs
    Ctl *c = a.ctl;
    uint32_t *next = d.cur ? a.F0 : a.F1;
    uint32_t *next_cnt = &c->nF[d.cur ^ 1u];
    uint32_t *farl = d.far_cur ? a.FAR1 : a.FAR0;
    uint32_t *far_cnt = &c->nFar[d.far_cur];
    uint32_t far_min = inf_key<DT>();
    uint32_t improved = 0;
    const uint32_t e0 = (uint32_t)(((unsigned long long)E * gw) / nw);
    const uint32_t e1 = (uint32_t)(((unsigned long long)E * (gw + 1)) / nw);
    if (e0 < e1) {
        // owner of e0: the last entry whose offset is <= e0
        uint32_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (__ldcg(&a.BIG[mid].y) <= e0) lo = mid; else hi = mid - 1;
        }
        uint32_t j0 = lo;
        for (uint32_t base = e0; base < e1; base += 32u) {
            const uint32_t e = base + lane;
            uint32_t j = j0;
            bool pn = false, pf = false;
            uint32_t v = 0;
            if (e < e1) {
                while (j + 1 < nb && __ldcg(&a.BIG[j + 1].y) <= e) ++j;
                const uint4 b = __ldcg(a.BIG + j);
                const uint32_t dkey = (uint32_t)(__ldcg(a.packed + b.x) >> 32);
                const uint2 arc = a.arcs[b.z + (e - b.y)];
                v = arc.x;
                relax_arc<DT>(a, d, v, key_add<DT>(dkey, arc.y), b.x, pn, pf, far_min, improved);
            }
            warp_append(pn, v, next, next_cnt);
            warp_append(pf, v, farl, far_cnt);
            j0 = __shfl_sync(FULL, j, 31);
        }
    }
    if (far_min < inf_key<DT>()) atomicMin(&acc.far_min, far_min);
    if (improved) atomicAdd(&acc.improvements, (unsigned long long)improved);
}

// SELECT: compact the far pile. Live entries whose key is below T (bucket <= i)
// move to the frontier; the rest stay, and their minimum key bounds the next
// bucket; stale entries are dropped.
template <int DT>
__device__ void phase_select(const SolveArgs &a, const Desc &d, BlockAcc &acc) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    Ctl *c = a.ctl;
    const uint32_t *in = d.far_cur ? a.FAR1 : a.FAR0;
    uint32_t *out = d.far_cur ? a.FAR0 : a.FAR1;
    uint32_t *out_cnt = &c->nFar[d.far_cur ^ 1u];
    uint32_t *next = d.cur ? a.F0 : a.F1;
    uint32_t *next_cnt = &c->nF[d.cur ^ 1u];
    uint32_t far_min = inf_key<DT>();
    const uint32_t count = d.count;
    for (unsigned long long base = (unsigned long long)gw * 32u; base < count; base += (unsigned long long)nw * 32u) {
        const uint32_t idx = (uint32_t)base + lane;
        bool take = false, keep = false;
        uint32_t v = 0;
        if (idx < count) {
            v = __ldcg(in + idx);
            if (__ldcg(a.far_flag + v) == 1u) {
                const uint32_t k = (uint32_t)(__ldcg(a.packed + v) >> 32);
                if (k < d.T) {
                    a.far_flag[v] = 0u;
                    take = atomicExch(a.near_stamp + v, d.qstamp) != d.qstamp;
                } else {
                    keep = true;
                    far_min = min(far_min, k);
                }
            } else {
                a.far_flag[v] = 0u;
            }
        }
        warp_append(take, v, next, next_cnt);
        warp_append(keep, v, out, out_cnt);
    }
    if (far_min < inf_key<DT>()) atomicMin(&acc.far_min, far_min);
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&acc.far_scanned, (unsigned long long)count);
}

// ---------------------------------------------------------------------------
// Serial step: runs on one thread after every block has finished a phase.
// Decides the next phase (the control flow of Fig. 1) and resets consumed lists.
template <int DT>
__device__ void serial_step(const SolveArgs &a) {
    Ctl *c = a.ctl;
    const uint64_t now = globaltimer();
    const uint64_t dt = now - c->t_last;
    c->t_last = now;
    const uint32_t mode = c->mode;
    if (mode == MODE_LIGHT || (mode == MODE_BIG && c->big_kind == 0u)) c->st[ST_NSLIGHT] += (long long)dt;
    else if (mode == MODE_HEAVY || mode == MODE_BIG) c->st[ST_NSHEAVY] += (long long)dt;
    else if (mode == MODE_SELECT) c->st[ST_NSSELECT] += (long long)dt;
    c->phases += 1;
    if (c->phases >= a.max_phases) {
        atomicCAS(&c->err, 0, (int)DSSSP_ERR_NOT_CONVERGED);
        c->mode = MODE_DONE;
        return;
    }
    const uint32_t nxt = c->cur ^ 1u;
    int next;   // 0: after light, 1: after heavy, 2: select
    switch (mode) {
    case MODE_LIGHT:
        c->st[ST_LIGHT] += 1;
        c->st[ST_VLIGHT] += c->nF[c->cur];
        c->nF[c->cur] = 0;
        if ((c->big_ctr >> 32) != 0ull) { c->mode = MODE_BIG; c->big_kind = 0u; return; }
        next = 0;
        break;
    case MODE_BIG:
        c->st[ST_BIGP] += 1;
        c->big_ctr = 0ull;
        next = c->big_kind == 0u ? 0 : 1;
        break;
    case MODE_HEAVY:
        c->st[ST_HEAVY] += 1;
        c->st[ST_VHEAVY] += c->nS;
        c->nS = 0;
        c->sround += 1u;
        if ((c->big_ctr >> 32) != 0ull) { c->mode = MODE_BIG; c->big_kind = 1u; return; }
        next = 1;
        break;
    case MODE_SELECT:
        c->st[ST_SELECT] += 1;
        c->nFar[c->far_cur] = 0;
        c->far_cur ^= 1u;
        if (c->nF[nxt] != 0u) {                 // bucket i has vertices: light rounds
            c->st[ST_BUCKETS] += 1;
            c->cur = nxt; c->qstamp += 1u; c->mode = MODE_LIGHT;
            return;
        }
        next = 2;
        break;
    default:
        return;
    }
    if (next == 0) {                            // inner loop of Fig. 1: while t_Bi != 0
        if (c->nF[nxt] != 0u) { c->cur = nxt; c->qstamp += 1u; c->mode = MODE_LIGHT; }
        else c->mode = MODE_HEAVY;
        return;
    }
    if (next == 1 && c->nF[nxt] != 0u) {        // a rounded heavy sum re-opened bucket i
        c->cur = nxt; c->qstamp += 1u; c->mode = MODE_LIGHT;
        return;
    }
    // next non-empty bucket
    const uint32_t fm = c->far_min;
    if (fm >= inf_key<DT>()) {
        if (c->nFar[c->far_cur] == 0u) {
            c->mode = MODE_DONE;
            c->st[ST_NSTOTAL] = (long long)(now - c->t_start);
            return;
        }
        c->T = 0u;                              // only stale entries remain: drop them
    } else {
        const int64_t i = bucket_of_key(fm, DT, a.delta);
        c->bucket = i;
        c->T = i < INT64_MAX ? bucket_floor_key(i + 1, DT, a.delta) : 0u;
        if (c->T <= fm) c->T = fm + 1u;         // always take the smallest live key
    }
    c->far_min = inf_key<DT>();
    c->mode = MODE_SELECT;
}

__device__ __forceinline__ void read_desc(const Ctl *c, Desc &d) {
    d.mode = vload(&c->mode);
    d.big_kind = vload(&c->big_kind);
    d.cur = vload(&c->cur);
    d.far_cur = vload(&c->far_cur);
    d.qstamp = vload(&c->qstamp);
    d.sround = vload(&c->sround);
    d.T = vload(&c->T);
    d.count = 0;
    d.count2 = 0;
    switch (d.mode) {
    case MODE_LIGHT: d.count = vload(&c->nF[d.cur]); break;
    case MODE_HEAVY: d.count = vload(&c->nS); break;
    case MODE_SELECT: d.count = vload(&c->nFar[d.far_cur]); break;
    case MODE_BIG: {
        const unsigned long long b = vload(&c->big_ctr);
        d.count = (uint32_t)(b >> 32);
        d.count2 = (uint32_t)b;
        break;
    }
    default: break;
    }
}

// Flush the block's far-pile minimum before arriving at a barrier.
__device__ __forceinline__ void flush_far_min(Ctl *c, BlockAcc &acc, uint32_t inf) {
    if (acc.far_min < inf) {
        atomicMin(&c->far_min, acc.far_min);
        acc.far_min = inf;
    }
}

__device__ __forceinline__ void flush_stats(Ctl *c, BlockAcc &acc) {
    if (acc.arcs_light) atomicAdd((unsigned long long *)&c->st[ST_ALIGHT], acc.arcs_light);
    if (acc.arcs_heavy) atomicAdd((unsigned long long *)&c->st[ST_AHEAVY], acc.arcs_heavy);
    if (acc.improvements) atomicAdd((unsigned long long *)&c->st[ST_IMPROVE], acc.improvements);
    if (acc.far_scanned) atomicAdd((unsigned long long *)&c->st[ST_FARSCAN], acc.far_scanned);
    acc.arcs_light = acc.arcs_heavy = acc.improvements = acc.far_scanned = 0;
}

// Grid-wide barrier with a serial step, every wait bounded by timeout_ns.
// Returns false when the solve must stop (error recorded, or timed out).
template <int DT>
__device__ bool grid_barrier(const SolveArgs &a, BlockAcc &acc, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        Ctl *c = a.ctl;
        flush_far_min(c, acc, inf_key<DT>());
        __threadfence();
        const unsigned gen = vload(&c->bar_gen);
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == a.nblocks - 1u) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            serial_step<DT>(a);
            __threadfence();
            atomicExch(&c->bar_gen, gen + 1u);
        } else {
            const uint64_t t0 = globaltimer();
            unsigned sleep_ns = 32;
            while (vload(&c->bar_gen) == gen) {
                if (vload(&c->err) != 0) break;
                if ((int64_t)(globaltimer() - t0) > a.timeout_ns) {
                    atomicCAS(&c->err, 0, (int)DSSSP_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(sleep_ns);
                if (sleep_ns < 256) sleep_ns <<= 1;
            }
            __threadfence();
        }
        *s_ok = (vload(&c->err) == 0) && (vload(&c->mode) != MODE_DONE);
    }
    __syncthreads();
    return *s_ok != 0;
}

template <int DT>
__device__ __forceinline__ void run_phase(const SolveArgs &a, const Desc &d, BlockAcc &acc, uint32_t *sw) {
    switch (d.mode) {
    case MODE_LIGHT: phase_segments<DT, true>(a, d, acc, sw); break;
    case MODE_HEAVY: phase_segments<DT, false>(a, d, acc, sw); break;
    case MODE_BIG: phase_big<DT>(a, d, acc); break;
    case MODE_SELECT: phase_select<DT>(a, d, acc); break;
    default: break;
    }
}

template <int DT>
__global__ void __launch_bounds__(512, 2) k_solve_persistent(SolveArgs a) {
    __shared__ uint32_t sw[kMaxWarps * 128];
    __shared__ Desc s_desc;
    __shared__ BlockAcc acc;
    __shared__ int s_ok;
    if (a.test_hook == DSSSP_HOOK_STALL_BARRIER && blockIdx.x == 1) return;
    if (threadIdx.x == 0) {
        acc.far_min = inf_key<DT>();
        acc.arcs_light = acc.arcs_heavy = acc.improvements = acc.far_scanned = 0;
    }
    for (;;) {
        if (threadIdx.x == 0) read_desc(a.ctl, s_desc);
        __syncthreads();
        const Desc d = s_desc;
        if (d.mode == MODE_DONE) break;
        run_phase<DT>(a, d, acc, sw);
        if (!grid_barrier<DT>(a, acc, &s_ok)) break;
    }
    __syncthreads();
    if (threadIdx.x == 0) flush_stats(a.ctl, acc);
}

// ---- stepped mode: one launch per phase --------------------------------------
template <int DT, uint32_t MODE>
__global__ void __launch_bounds__(512, 2) k_phase(SolveArgs a) {
    __shared__ uint32_t sw[kMaxWarps * 128];
    __shared__ Desc s_desc;
    __shared__ BlockAcc acc;
    if (threadIdx.x == 0) {
        read_desc(a.ctl, s_desc);
        acc.far_min = inf_key<DT>();
        acc.arcs_light = acc.arcs_heavy = acc.improvements = acc.far_scanned = 0;
    }
    __syncthreads();
    const Desc d = s_desc;
    if (d.mode != MODE) return;
    run_phase<DT>(a, d, acc, sw);
    __syncthreads();
    if (threadIdx.x == 0) {
        flush_far_min(a.ctl, acc, inf_key<DT>());
        flush_stats(a.ctl, acc);
    }
}

template <int DT>
__global__ void k_serial(SolveArgs a) {
    if (vload(&a.ctl->mode) != MODE_DONE) serial_step<DT>(a);
}

// ---- init / unpack -------------------------------------------------------------
template <int DT>
__global__ void k_init(SolveArgs a) {
    const uint32_t n = a.n;
    const unsigned long long unreached = ((unsigned long long)inf_key<DT>() << 32) | NO_PRED;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        // t = inf, t[s] = 0 (Fig. 1); predecessor of s is s
        a.packed[v] = v == a.src ? (unsigned long long)a.src : unreached;
        a.near_stamp[v] = 0u;
        a.far_flag[v] = 0u;
        a.s_stamp[v] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *c = a.ctl;
        c->bar_count = 0u;
        c->bar_gen = 0u;
        c->mode = MODE_LIGHT;     // B_0 = {s}
        c->big_kind = 0u;
        c->cur = 0u;
        c->far_cur = 0u;
        c->qstamp = 1u;
        c->sround = 1u;
        c->bucket = 0;
        c->T = bucket_floor_key(1, DT, a.delta);
        c->nF[0] = 1u;
        c->nF[1] = 0u;
        c->nS = 0u;
        c->nFar[0] = c->nFar[1] = 0u;
        c->far_min = inf_key<DT>();
        c->big_ctr = 0ull;
        c->err = 0;
        c->phases = 0;
        for (int k = 0; k < 16; ++k) c->st[k] = 0;
        c->st[ST_BUCKETS] = 1;
        c->t_start = c->t_last = globaltimer();
        a.F0[0] = a.src;
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
        DSSSP_PHASE_CASE(MODE_BIG)
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
