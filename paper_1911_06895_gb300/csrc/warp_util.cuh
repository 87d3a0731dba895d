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

// Merge-path directory of an arc list (C units per entry, then one per arc, in
// list order; a list's merged order is its entries' units back to back). For
// every chunk boundary b = c * S that falls in the units of entry i (arc offset
// off, deg arcs), dir[c] = (number of entries whose first arc lies at or before
// b, arc offset of the entry after those): (i, off) while b lies in the entry's
// own units, (i + 1, off + deg) once b reaches its arcs -- the result of a
// merge-path search for b, recorded when the entry is appended. Each lane passes
// one entry (has = false: none; dir may differ per lane); a lane writes up to
// kDirShort of its boundaries itself and the warp writes the rest together.
constexpr uint32_t kDirShort = 4;

template <uint32_t C, uint32_t S>
__device__ __forceinline__ void dir_record(uint2 *dir, bool has, uint32_t i, uint32_t off, uint32_t deg) {
    static_assert(C <= S, "at most one boundary in an entry's own units");
    const unsigned long long us = (unsigned long long)i * C + off, ua = us + C, ue = ua + deg;
    const uint32_t c0 = has ? (uint32_t)((us + S - 1u) / S) : 0u;   // first boundary >= us
    const uint32_t ca = has ? (uint32_t)((ua + S - 1u) / S) : 0u;   // first boundary >= ua
    const uint32_t ce = has ? (uint32_t)((ue + S - 1u) / S) : 0u;   // first boundary >= ue
    if (c0 < ca) dir[c0] = make_uint2(i, off);
    const uint2 val = make_uint2(i + 1u, off + deg);
    const uint32_t cs = min(ce, ca + kDirShort);
    for (uint32_t c = ca; c < cs; ++c) dir[c] = val;
    uint32_t rest = __ballot_sync(FULL, cs < ce);
    while (rest) {
        const int l = __ffs(rest) - 1;
        uint2 *d = reinterpret_cast<uint2 *>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(dir), l));
        const uint32_t b0 = __shfl_sync(FULL, cs, l), b1 = __shfl_sync(FULL, ce, l);
        const uint2 v = make_uint2(__shfl_sync(FULL, val.x, l), __shfl_sync(FULL, val.y, l));
        for (uint32_t c = b0 + lane_id(); c < b1; c += 32u) d[c] = v;
        rest &= rest - 1u;
    }
}

// Append n <= 64 staged (vertex, arc count) pairs to an arc list whose entries
// carry their exclusive arc offset: one 64-bit atomicAdd of (entries << 32 |
// arcs) on the list's counter (global or shared memory). Lane l holds entries
// 2l and 2l+1. With C > 0 the list's merge-path directory is kept too.
template <uint32_t C = 0, uint32_t S = 1>
__device__ __forceinline__ void flush_arc_entries(const uint32_t *bv, const uint32_t *bd, uint32_t n, uint2 *list,
                                                  unsigned long long *ctr, uint2 *dir = nullptr) {
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
    if (C != 0u) {
        dir_record<C, S>(dir, h0, base, off, d0);
        dir_record<C, S>(dir, h1, base + 1u, off + d0, d1);
    }
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
template <uint32_t C = 0, uint32_t S = 1>
__device__ __forceinline__ void stage_arc_entry(bool pred, uint32_t v, uint32_t deg, uint32_t *bv, uint32_t *bd,
                                                uint32_t &cnt, uint2 *list, unsigned long long *ctr,
                                                uint2 *dir = nullptr) {
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
        flush_arc_entries<C, S>(bv, bd, kFlush, list, ctr, dir);
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
