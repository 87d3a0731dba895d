// dsssp_internal.cuh -- device-side state and helpers shared by the library's
// kernels (split, solve) and its host API. Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dsssp.h"

namespace dsssp {

// ----------------------------------------------------------------------------
// Keys. A tentative distance is kept as a 32-bit key whose unsigned order is
// the order of the distances: the IEEE bits of a non-negative float32, or the
// value of a non-negative int32. The paper's t vector (Fig. 1) is stored as
// packed[v] = key(t[v]) << 32 | pred[v], so one 64-bit atomicMin updates the
// distance and keeps the smallest predecessor among equal distances.
constexpr uint32_t KEY_INF_F32 = 0x7F800000u;   // +inf
constexpr uint32_t KEY_INF_I32 = 0x7FFFFFFFu;   // INT32_MAX
constexpr uint32_t NO_PRED = 0xFFFFFFFFu;

__host__ __device__ inline uint32_t key_inf(int dtype) {
    return dtype == DSSSP_F32 ? KEY_INF_F32 : KEY_INF_I32;
}

// Exact value of a key as a double.
__host__ __device__ inline double key_value(uint32_t k, int dtype) {
    if (dtype == DSSSP_F32) {
        union { uint32_t u; float f; } c;
        c.u = k;
        return (double)c.f;
    }
    return (double)k;
}

// bucket(x) = floor(x / Delta) (Section III-B), evaluated exactly: the double
// quotient is correctly rounded, hence at most one above the true floor; an
// exact fma() sign test corrects it.
__host__ __device__ inline int64_t bucket_of_key(uint32_t k, int dtype, double delta) {
    if (delta == (double)INFINITY) return 0;
    double x = key_value(k, dtype);
    double q = floor(x / delta);
    if (q >= 9007199254740992.0) return q >= 9.2e18 ? INT64_MAX : (int64_t)q;
    if (q > 0.0 && fma(q, delta, -x) > 0.0) q -= 1.0;
    else if (fma(q + 1.0, delta, -x) <= 0.0) q += 1.0;
    return (int64_t)q;
}

// Smallest key whose value is >= j * Delta exactly (the lower edge of bucket j);
// key_inf when no finite value qualifies. "key < bucket_floor_key(i+1)" is
// then exactly "bucket(key) <= i".
__host__ __device__ inline uint32_t bucket_floor_key(int64_t j, int dtype, double delta) {
    const uint32_t inf = key_inf(dtype);
    if (delta == (double)INFINITY) return j <= 0 ? 0u : inf;
    if (j <= 0) return 0u;
    const double jd = (double)j;
    const double p = jd * delta;                       // rounded; corrected below
    const double maxv = key_value(inf - 1u, dtype);
    if (!(p <= maxv * 1.0000001)) return inf;
    uint32_t k;
    if (dtype == DSSSP_F32) {
        float f = (float)p;                            // nearest; corrected below
        union { float f; uint32_t u; } c;
        c.f = f;
        k = c.u;
        if (k > inf) k = inf;
    } else {
        double cp = ceil(p);
        k = cp >= (double)inf ? inf : (uint32_t)cp;
    }
    // step down while the previous key still reaches j*Delta, up while k falls short
    for (int it = 0; it < 4 && k > 0u && fma(jd, delta, -key_value(k - 1u, dtype)) <= 0.0; ++it) --k;
    for (int it = 0; it < 4 && k < inf && fma(jd, delta, -key_value(k, dtype)) > 0.0; ++it) ++k;
    return k;
}

// Largest weight key that is light (value <= Delta), Section III-A; light arcs
// are exactly those with key <= light_max_key. Zero is light.
__host__ __device__ inline uint32_t light_max_key(int dtype, double delta) {
    const uint32_t inf = key_inf(dtype);
    if (!(delta < key_value(inf - 1u, dtype))) return inf;   // every finite weight is light
    // smallest key above Delta, minus one
    uint32_t k;
    if (dtype == DSSSP_F32) {
        union { float f; uint32_t u; } c;
        c.f = (float)delta;
        k = c.u;
    } else {
        k = (uint32_t)floor(delta);
    }
    while (k > 0u && key_value(k, dtype) > delta) --k;
    while (k + 1u < inf && key_value(k + 1u, dtype) <= delta) ++k;
    if (key_value(k, dtype) > delta) return 0xFFFFFFFFu;      // nothing is light (delta < 0)
    return k;
}

// ----------------------------------------------------------------------------
// Solver phases. Each phase is one grid-wide step separated by a barrier.
enum Mode : uint32_t {
    MODE_LIGHT = 0,    // relax light arcs of the frontier  (t_Req = A_L^T (t o t_Bi))
    MODE_HEAVY = 1,    // relax heavy arcs of S             (t_Req = A_H^T (t o S))
    MODE_REBIN = 2,    // move overflow vertices into the bucket slots of a new window
    MODE_DONE = 3,
    MODE_FUSED = 4     // the heavy pass of bucket i together with the first light round of bucket i+1
};

// Buckets. Section III-B's B_j are kept explicitly for a window of kSlots
// consecutive buckets [wbase, wbase + kSlots): when a vertex's distance drops
// into bucket j of the window (j > i, the current bucket), it is appended once
// to slot j - wbase -- to the slot's arc list when it has light arcs, to its
// heavy-only list otherwise. A later decrease into a lower bucket leaves the
// entry stale; stale entries are recognised by their key (below the slot's
// lower edge) and skipped. Distances beyond the window go to the overflow list,
// which is redistributed into a new window when the current one is used up.
constexpr uint32_t kSlots = 32;
// Merge-path directories of the single-source solver's arc lists: F0, F1, S0,
// S1, then one per bucket slot.
constexpr uint32_t kDirSL = 4;
constexpr uint32_t kDirLists = kDirSL + kSlots;

// Arc lists (frontier F, set S, slot lists) hold uint2 entries (vertex, exclusive
// arc offset of the entry within its list). An entry is appended with one
// 64-bit atomicAdd of (entries << 32 | arcs) per 32 staged entries, so entry
// positions and arc offsets agree and a phase splits the list's flattened arcs
// evenly over all warps. A vertex's arc segment comes from vinfo.
//
// Control block. The serial step of a barrier (one warp) loads SerialState, the
// list counters and the window's slot counters in one batch, decides the next
// phase in registers and publishes a PhaseDesc that every block reads with
// 16-byte loads, together with the window's thresholds and the error word.

// Everything a block needs to run a phase (64 bytes).
struct alignas(64) PhaseDesc {
    uint32_t mode;
    uint32_t cur;           // F list read (0/1) when not reading a slot; F pushes go to cur^1
    uint32_t scur;          // S list read by a heavy pass
    uint32_t spush;         // S list receiving pushes in this phase
    uint32_t sstamp;        // S stamp of those pushes
    uint32_t qstamp;        // stamp of pushes into the next frontier
    uint32_t T;             // key < T  <=>  bucket <= i (the current bucket)
    uint32_t T_lo;          // entries of a slot list with key < T_lo are stale (0: none)
    uint32_t slot;          // LIGHT: slot read by the first round of a bucket, kSlots otherwise
    uint32_t count;         // entries of the arc list this phase reads (REBIN: overflow entries)
    uint32_t arcs;          // arcs of that list
    uint32_t count2;        // first round: heavy-only entries of the slot
    uint32_t ov_cur;        // overflow list read by REBIN / appended to otherwise
    uint32_t solo;          // 1: block 0 alone runs this phase (little work), the others wait
    uint32_t pad;
    uint32_t wepoch;        // window epoch: changes whenever the window's thresholds do
    uint32_t count_h;       // FUSED: entries of the S list whose heavy arcs are relaxed
    uint32_t arcs_h;        // FUSED: their heavy arcs
};
constexpr int kDescVec = (int)(sizeof(PhaseDesc) / 16);   // 16-byte words of a PhaseDesc

// State only the serial step reads and writes.
struct alignas(16) SerialState {
    uint32_t mode, cur, scur, ov_cur, qstamp, sround, T, T_lo;
    int64_t bucket;         // current bucket i
    int64_t wbase;          // first bucket of the slot window
    int64_t phases;
    uint64_t t_last;        // %globaltimer at the previous barrier
    uint64_t t_start;
    uint32_t wepoch;        // window epoch (refills of the slot window)
    uint32_t pad0;
    long long st[16];       // counters (StatIdx), only ever added to during a solve
};
constexpr int kSerialHotVec = (int)(offsetof(SerialState, st) / 16);   // 16-byte words before st[]

// The published view of the next phase: kViewWords 64-bit words, each the
// phase number (high half) and one 32-bit field (low half). A word is written
// and read as one 8-byte access, so a reader that sees the same phase number
// in every word holds a consistent view without a separate flag or fence.
constexpr int kViewWords = 13;

struct Ctl {
    // barrier words, alone on their line
    unsigned int bar_count;
    unsigned int pad_b;
    int32_t err;            // first dsssp_status != OK
    uint32_t ovf;           // 1: a relaxation met a sum the weight type cannot hold (checked at the end)
    uint64_t t_first;       // %globaltimer of the first arrival at the current barrier
    uint32_t pad1[26];
    unsigned long long view[16];   // the published view (kViewWords used), on its own line
    PhaseDesc desc;                // the serial step's own copy of the current phase
    // key thresholds of the window: bucket wbase + t starts at key thr[t]
    uint32_t thr[kSlots + 1];
    uint32_t pad2[15];
    // counters updated with atomics during a phase
    unsigned long long ctrF[2];          // (entries << 32) | arcs
    unsigned long long ctrS[2];
    unsigned long long ctrSL[kSlots];    // slot arc lists
    uint32_t nSH[kSlots];                // slot heavy-only lists
    uint32_t nOV[2];                     // overflow lists
    uint32_t ov_min;                     // lower bound on the keys of live overflow entries
    uint32_t pad3[13];
    SerialState ss;
};

enum StatIdx {
    ST_BUCKETS = 0, ST_LIGHT = 1, ST_HEAVY = 2, ST_REBIN = 3, ST_VLIGHT = 4, ST_VHEAVY = 5,
    ST_ALIGHT = 6, ST_AHEAVY = 7, ST_FARSCAN = 8, ST_IMPROVE = 9, ST_NSLIGHT = 10, ST_NSHEAVY = 11,
    ST_NSREBIN = 12, ST_NSTOTAL = 13, ST_NSFIRST = 14, ST_NSSPREAD = 15
};

// Per-vertex arc segments of the split layout: [x, y) light, [y, z) heavy.
// uint4 so that one 16-byte load fetches a vertex's segments.

struct SolveArgs {
    const uint4 *vinfo;             // n
    const uint2 *arcs;              // m: (head, weight bits), light-first per row
    unsigned long long *packed;     // n
    uint32_t *near_stamp;           // n: phase stamp of the last push into the next frontier
    uint32_t *s_stamp;              // n: bucket stamp of the last push into S
    uint32_t *b_stamp;              // n: (bucket + 1) of the last push into a slot
    uint32_t *ov_flag;              // n: 1 while the vertex has a live overflow entry
    uint2 *F0, *F1;                 // n each
    uint2 *S0, *S1;                 // n each
    uint2 *SL;                      // kSlots x n
    uint32_t *SH;                   // kSlots x n
    uint32_t *OV0, *OV1;            // n each
    uint2 *dir;                     // kDirLists x dcap: merge-path directory of each arc list
    Ctl *ctl;
    double delta;
    int64_t timeout_ns;
    int64_t max_phases;
    uint32_t n;
    uint32_t m;
    uint32_t src;
    uint32_t inf_key;
    uint32_t solo_work;             // phases with at most this much work run solo
    uint32_t fuse;                  // 1: heavy pass of bucket i fused with the first light round of i+1
    int32_t dtype;
    int32_t test_hook;
    uint32_t nblocks;
    uint32_t dcap;                  // directory entries per list
};

// Launch helpers implemented in solve.cu / split.cu (host side).
cudaError_t launch_validate(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                            uint32_t *wbits, int dtype, uint32_t *off, int *flags, cudaStream_t st);
cudaError_t launch_split(int64_t n, int64_t m, const uint32_t *off, const int32_t *col,
                         const uint32_t *wbits, uint32_t light_max, uint32_t *scratch_pl,
                         uint32_t *scratch_tiles, uint2 *arcs, uint4 *vinfo, uint32_t *perm,
                         cudaStream_t st);
size_t split_scratch_tiles(int64_t m);

cudaError_t launch_init(const SolveArgs &a, cudaStream_t st);
uint32_t solve_dir_entries(uint32_t n, uint32_t m);   // directory entries per list
cudaError_t launch_solve_persistent(const SolveArgs &a, int grid, int block, cudaStream_t st);
cudaError_t solve_occupancy(int block, int *blocks_per_sm);
cudaError_t launch_phase_stepped(const SolveArgs &a, uint32_t mode, int grid, int block,
                                 cudaStream_t st);
cudaError_t launch_serial_step(const SolveArgs &a, cudaStream_t st);
cudaError_t launch_verify_overflow(const SolveArgs &a, int grid, int block, cudaStream_t st);
cudaError_t launch_unpack(const SolveArgs &a, void *dist, int32_t *pred, cudaStream_t st);

}  // namespace dsssp
