// warp_util.cuh -- warp-level helpers shared by the solvers (single-source and batched):
// key arithmetic and per-warp staging of list appends. Not part of the ABI.
#pragma once

#include "dsssp_internal.cuh"

namespace dsssp {
namespace wu {

constexpr uint32_t FULL = 0xffffffffu;

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

template <int DT>
__device__ __forceinline__ constexpr uint32_t inf_key() {
    return DT == DSSSP_F32 ? KEY_INF_F32 : KEY_INF_I32;
}

// d (+) w on keys: float32 add rounded to nearest (+inf on overflow), or int32
// add saturated at INT32_MAX. Both int32 operands are below 2^31.
template <int DT>
__device__ __forceinline__ uint32_t key_add(uint32_t dkey, uint32_t wbits) {
    if (DT == DSSSP_F32) {
        return __float_as_uint(__fadd_rn(__uint_as_float(dkey), __uint_as_float(wbits)));
    } else {
        const uint32_t s = dkey + wbits;
        return s >= KEY_INF_I32 ? KEY_INF_I32 : s;
    }
}

// Staging: a list counter is taken once per kFlush staged entries; a staging
// call adds at most 32, so a buffer holds kStage entries.
constexpr uint32_t kFlush = 64;
constexpr uint32_t kStage = kFlush + 32;

// Append n <= 64 staged (vertex, arc count) pairs to an arc list whose entries
// carry their exclusive arc offset: one 64-bit atomicAdd of (entries << 32 |
// arcs) on the list's counter (global or shared memory). Lane l holds entries
// 2l and 2l+1.
__device__ __forceinline__ void flush_arc_entries(const uint32_t *bv, const uint32_t *bd, uint32_t n, uint2 *list,
                                                  unsigned long long *ctr) {
    const uint32_t lane = lane_id();
    const uint32_t j = 2u * lane;
    const bool h0 = j < n, h1 = j + 1u < n;
    const uint32_t v0 = h0 ? bv[j] : 0u, d0 = h0 ? bd[j] : 0u;
    const uint32_t v1 = h1 ? bv[j + 1u] : 0u, d1 = h1 ? bd[j + 1u] : 0u;
    uint32_t incl = d0 + d1;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, o);
        if ((int)lane >= o) incl += t;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(ctr, ((unsigned long long)n << 32) | tot);
    old = __shfl_sync(FULL, old, 0);
    const uint32_t base = (uint32_t)(old >> 32) + j, off = (uint32_t)old + incl - d0 - d1;
    if (h0) list[base] = make_uint2(v0, off);
    if (h1) list[base + 1u] = make_uint2(v1, off + d0);
}

// Append n <= 64 staged ids to an id list.
__device__ __forceinline__ void flush_ids(const uint32_t *bv, uint32_t n, uint32_t *list, uint32_t *counter) {
    const uint32_t lane = lane_id();
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(counter, n);
    base = __shfl_sync(FULL, base, 0);
    if (lane < n) list[base + lane] = bv[lane];
    if (lane + 32u < n) list[base + lane + 32u] = bv[lane + 32u];
}

// Stage one (vertex, arc count) pair per lane with `pred` (kStage-entry buffer
// per warp); flush kFlush to the list when the buffer holds that many.
__device__ __forceinline__ void stage_arc_entry(bool pred, uint32_t v, uint32_t deg, uint32_t *bv, uint32_t *bd,
                                                uint32_t &cnt, uint2 *list, unsigned long long *ctr) {
    const uint32_t mask = __ballot_sync(FULL, pred);
    if (mask == 0u) return;
    const uint32_t lane = lane_id();
    if (pred) {
        const uint32_t k = cnt + __popc(mask & lanemask_lt());
        bv[k] = v;
        bd[k] = deg;
    }
    cnt += __popc(mask);
    __syncwarp();
    if (cnt >= kFlush) {
        flush_arc_entries(bv, bd, kFlush, list, ctr);
        const uint32_t rest = cnt - kFlush;
        uint32_t x = 0, y = 0;
        if (lane < rest) { x = bv[kFlush + lane]; y = bd[kFlush + lane]; }
        __syncwarp();
        if (lane < rest) { bv[lane] = x; bd[lane] = y; }
        __syncwarp();
        cnt = rest;
    }
}

__device__ __forceinline__ void stage_id(bool pred, uint32_t v, uint32_t *bv, uint32_t &cnt, uint32_t *list,
                                         uint32_t *counter) {
    const uint32_t mask = __ballot_sync(FULL, pred);
    if (mask == 0u) return;
    const uint32_t lane = lane_id();
    if (pred) bv[cnt + __popc(mask & lanemask_lt())] = v;
    cnt += __popc(mask);
    __syncwarp();
    if (cnt >= kFlush) {
        flush_ids(bv, kFlush, list, counter);
        const uint32_t rest = cnt - kFlush;
        uint32_t x = 0;
        if (lane < rest) x = bv[kFlush + lane];
        __syncwarp();
        if (lane < rest) bv[lane] = x;
        __syncwarp();
        cnt = rest;
    }
}

}  // namespace wu
}  // namespace dsssp
