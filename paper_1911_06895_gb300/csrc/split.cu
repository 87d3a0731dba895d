// split.cu -- graph validation and the light/heavy split (Section III-A, IV-A;
// Fig. 1: A_L = A o (A <= Delta), A_H = A o (A > Delta)).
//
// The split is a stable partition of every CSR row: light arcs first, heavy
// arcs after, each group in input order. It is computed with one global
// exclusive prefix count of light arcs, PL[e] = #light arcs before e:
//   light arc e in row u goes to   begin_u + (PL[e] - PL[begin_u])
//   heavy arc e in row u goes to   e + (PL[end_u] - PL[e])
// so every arc's destination is independent of every other arc's, and rows of
// any length are handled by the same tile-parallel pass (R-MAT rows reach
// ~10^5 arcs). Memory traffic: m * (4 + 4) read twice, m * (8 + 4) written,
// plus the 4-byte prefix array written once and read twice.
#include "dsssp_internal.cuh"

namespace dsssp {

namespace {

constexpr int kSplitBlock = 512;
constexpr int kSplitItems = 8;
constexpr int kTile = kSplitBlock * kSplitItems;   // arcs per tile

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *total) {
    __shared__ uint32_t warp_sums[kSplitBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kSplitBlock / 32 ? warp_sums[lane] : 0u;
        uint32_t si = s;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < kSplitBlock / 32) warp_sums[lane] = si - s;
        if (lane == 31) *total = si;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - x;
    __syncthreads();
    return r;
}

// ---- validation -----------------------------------------------------------
// flags bit 0: malformed CSR; bit 1: bad weight. Also converts row_ptr to the
// 32-bit offsets the kernels use and stores float32 -0.0 as +0.0.
__global__ void k_validate(int64_t n, int64_t m, const int64_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, uint32_t *__restrict__ wbits,
                           int dtype, uint32_t *__restrict__ off, int *flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad_graph = 0, bad_w = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
        int64_t r = row_ptr[i];
        if (i == 0 && r != 0) bad_graph = 1;
        if (i == n && r != m) bad_graph = 1;
        if (i < n && row_ptr[i + 1] < r) bad_graph = 1;
        if (r < 0 || r > m) bad_graph = 1;
        off[i] = (uint32_t)(r < 0 ? 0 : (r > m ? m : r));
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t v = col[e];
        if (v < 0 || (int64_t)v >= n) bad_graph = 1;
        uint32_t b = wbits[e];
        if (dtype == DSSSP_F32) {
            if (b == 0x80000000u) { wbits[e] = 0u; b = 0u; }        // -0.0 -> +0.0
            if (b >= 0x7F800000u) bad_w = 1;                      // negative, inf or NaN
        } else {
            if ((int32_t)b < 0) bad_w = 1;
        }
    }
    if (bad_graph) atomicOr(flags, 1);
    if (bad_w) atomicOr(flags, 2);
}

// ---- split ------------------------------------------------------------------
__global__ void __launch_bounds__(kSplitBlock) k_tile_count(int64_t m, const uint32_t *__restrict__ wbits,
                                                            uint32_t light_max, uint32_t *__restrict__ tiles) {
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
    uint32_t c = 0;
    #pragma unroll
    for (int k = 0; k < kSplitItems; ++k) {
        int64_t e = t0 + (int64_t)k * kSplitBlock + threadIdx.x;
        if (e < m && wbits[e] <= light_max) ++c;
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ uint32_t ws[kSplitBlock / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kSplitBlock / 32; ++i) s += ws[i];
        tiles[blockIdx.x] = s;
    }
}

// exclusive scan of the per-tile counts by one block, in place
__global__ void __launch_bounds__(kSplitBlock) k_tile_scan(int64_t ntiles, uint32_t *__restrict__ tiles) {
    const int64_t per = (ntiles + kSplitBlock - 1) / kSplitBlock;
    const int64_t b = (int64_t)threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = b; i < b + per && i < ntiles; ++i) s += tiles[i];
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, &total);
    for (int64_t i = b; i < b + per && i < ntiles; ++i) {
        uint32_t x = tiles[i];
        tiles[i] = run;
        run += x;
    }
}

// PL[e] for every arc, and PL[m] = total light count
__global__ void __launch_bounds__(kSplitBlock) k_tile_prefix(int64_t m, const uint32_t *__restrict__ wbits,
                                                             uint32_t light_max,
                                                             const uint32_t *__restrict__ tiles,
                                                             uint32_t *__restrict__ pl) {
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
    // thread owns kSplitItems consecutive arcs so the scan is over per-thread sums
    const int64_t e0 = t0 + (int64_t)threadIdx.x * kSplitItems;
    uint32_t flags[kSplitItems];
    uint32_t c = 0;
    #pragma unroll
    for (int k = 0; k < kSplitItems; ++k) {
        int64_t e = e0 + k;
        flags[k] = (e < m && wbits[e] <= light_max) ? 1u : 0u;
        c += flags[k];
    }
    uint32_t total;
    uint32_t run = tiles[blockIdx.x] + block_exclusive_scan(c, &total);
    #pragma unroll
    for (int k = 0; k < kSplitItems; ++k) {
        int64_t e = e0 + k;
        if (e < m) pl[e] = run;
        if (e == m) pl[m] = run;
        run += flags[k];
    }
    if (e0 + kSplitItems == m) pl[m] = run;      // m on the boundary of this thread's items
}

__global__ void k_rows(int64_t n, const uint32_t *__restrict__ off, const uint32_t *__restrict__ pl,
                       uint4 *__restrict__ vinfo) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = off[u], e = off[u + 1];
        uint32_t nl = pl[e] - pl[b];
        vinfo[u] = make_uint4(b, b + nl, e, 0u);
    }
}

// scatter: each thread walks kSplitItems consecutive arcs, tracking their row
__global__ void __launch_bounds__(kSplitBlock) k_scatter(int64_t n, int64_t m, const uint32_t *__restrict__ off,
                                                         const int32_t *__restrict__ col,
                                                         const uint32_t *__restrict__ wbits,
                                                         uint32_t light_max, const uint32_t *__restrict__ pl,
                                                         uint2 *__restrict__ arcs, uint32_t *__restrict__ perm) {
    const int64_t e0 = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kSplitItems;
    if (e0 >= m) return;
    // row of e0: largest u with off[u] <= e0 (skips empty rows)
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)off[mid] <= e0) lo = mid; else hi = mid - 1;
    }
    int64_t u = lo;
    uint32_t rb = off[u], re = off[u + 1];
    uint32_t plb = pl[rb], ple = pl[re];
    for (int k = 0; k < kSplitItems; ++k) {
        int64_t e = e0 + k;
        if (e >= m) break;
        while ((int64_t)re <= e) {               // next non-empty row
            ++u;
            rb = re;
            re = off[u + 1];
            plb = ple;
            ple = pl[re];
        }
        uint32_t w = wbits[e];
        uint32_t p = pl[e];
        uint32_t dst = (w <= light_max) ? rb + (p - plb) : (uint32_t)e + (ple - p);
        arcs[dst] = make_uint2((uint32_t)col[e], w);
        perm[dst] = (uint32_t)e;
    }
}

}  // namespace

cudaError_t launch_validate(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                            uint32_t *wbits, int dtype, uint32_t *off, int *flags, cudaStream_t st) {
    int64_t work = n + 1 > m ? n + 1 : m;
    int grid = (int)((work + 255) / 256);
    if (grid > 65535 * 4) grid = 65535 * 4;
    if (grid < 1) grid = 1;
    k_validate<<<grid, 256, 0, st>>>(n, m, row_ptr, col, wbits, dtype, off, flags);
    return cudaGetLastError();
}

size_t split_scratch_tiles(int64_t m) { return (size_t)((m + kTile - 1) / kTile) + 1; }

cudaError_t launch_split(int64_t n, int64_t m, const uint32_t *off, const int32_t *col,
                         const uint32_t *wbits, uint32_t light_max, uint32_t *pl, uint32_t *tiles,
                         uint2 *arcs, uint4 *vinfo, uint32_t *perm, cudaStream_t st) {
    const int64_t ntiles = (m + kTile - 1) / kTile;
    if (ntiles > 0) {
        k_tile_count<<<(unsigned)ntiles, kSplitBlock, 0, st>>>(m, wbits, light_max, tiles);
        k_tile_scan<<<1, kSplitBlock, 0, st>>>(ntiles, tiles);
        k_tile_prefix<<<(unsigned)ntiles, kSplitBlock, 0, st>>>(m, wbits, light_max, tiles, pl);
    } else {
        cudaMemsetAsync(pl, 0, sizeof(uint32_t), st);
    }
    int rg = (int)((n + 255) / 256);
    if (rg > 65535 * 4) rg = 65535 * 4;
    k_rows<<<rg, 256, 0, st>>>(n, off, pl, vinfo);
    if (ntiles > 0)
        k_scatter<<<(unsigned)ntiles, kSplitBlock, 0, st>>>(n, m, off, col, wbits, light_max, pl, arcs, perm);
    return cudaGetLastError();
}

}  // namespace dsssp
