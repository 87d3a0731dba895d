// noalloc.cu -- dsssp_solve_noalloc: a delta-stepping solve that allocates no
// memory at all, for callers that cannot call cudaMalloc (code running under
// an allocator it must not bypass, inside a memory budget fixed up front, or in
// a context where a device allocation would synchronise or fail).
//
// It computes what dsssp_solve computes (same distances and predecessors, bit
// for bit), but works directly on the caller's device CSR: the light/heavy
// split is applied on the fly while a vertex's row is scanned (light arcs in
// light rounds, heavy arcs in heavy passes), and the frontier, the set S and
// the far pile are dense per-vertex stamps -- the t_Bi / S vectors of the
// linear-algebra form -- instead of compacted lists. All of its working memory
// is one file-scope __device__ array of fixed size, so a graph may have at most
// kNoAllocMaxVertices vertices (any number of arcs up to 2^31 - 1).
//
// Every call uses the same array: calls that overlap on the GPU (for example
// on two streams) race and must be serialised by the caller. Each call clears
// the state it needs before using it.
//
// The same kernels, on working memory allocated with a graph handle, are the
// DSSSP_MODE_DENSE scheme of dsssp_solve: the paper's full-vector form (every
// phase scans all n entries of t_Bi, S or the far pile; the A_L / A_H filters
// fused into the row scans, Section VI-B) as an alternative to the compacted
// lists of the persistent solver.
#include <mutex>

#include "dsssp_internal.cuh"
#include "dense.cuh"

namespace {

using namespace dsssp;

constexpr uint32_t kNoAllocMaxVertices = 1u << 17;   // 131,072
constexpr int kNaBlock = 256;

struct NaScratch {
    unsigned long long packed[kNoAllocMaxVertices];   // key << 32 | pred
    uint32_t fstamp[kNoAllocMaxVertices];             // in the light round with this stamp
    uint32_t sstamp[kNoAllocMaxVertices];             // member of S in the bucket with this stamp
    uint32_t far[kNoAllocMaxVertices];                // 1: a later bucket holds an unprocessed key
    NaCtl ctl;
};

// The fixed working memory (~11 MB), held by every GPU that loads the library.
static __device__ __align__(256) NaScratch g_noalloc_scratch;

__device__ __forceinline__ uint64_t na_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ T na_vload(const T *p) { return *(const volatile T *)p; }

template <int DT>
__device__ __forceinline__ uint32_t na_inf() { return DT == DSSSP_F32 ? KEY_INF_F32 : KEY_INF_I32; }

template <int DT>
__device__ __forceinline__ uint32_t na_add(uint32_t dkey, uint32_t wbits) {
    if (DT == DSSSP_F32) return __float_as_uint(__fadd_rn(__uint_as_float(dkey), __uint_as_float(wbits)));
    const uint32_t s = dkey + wbits;
    return s >= KEY_INF_I32 ? KEY_INF_I32 : s;
}

// Grid barrier with a bounded wait; the last arrival runs `serial` (one thread).
// The wait gives up after timeout_ns without progress: the clock restarts
// whenever another block arrives or a warp reports scanned arcs, so one warp
// scanning a very long row keeps the others waiting as long as it advances.
template <typename F>
__device__ bool na_barrier(NaCtl *c, uint32_t nblocks, int64_t timeout_ns, F serial) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned gen = na_vload(&c->bar_gen);
        if (atomicAdd(&c->bar_count, 1u) == nblocks - 1u) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            serial();
            __threadfence();
            atomicExch(&c->bar_gen, gen + 1u);
        } else {
            uint64_t t0 = na_timer();
            unsigned seen_count = na_vload(&c->bar_count);
            unsigned long long seen_prog = na_vload(&c->progress);
            while (na_vload(&c->bar_gen) == gen) {
                if (na_vload(&c->err) != 0) break;
                const uint64_t now = na_timer();
                const unsigned cnt = na_vload(&c->bar_count);
                const unsigned long long prog = na_vload(&c->progress);
                if (cnt != seen_count || prog != seen_prog) {
                    seen_count = cnt;
                    seen_prog = prog;
                    t0 = now;
                }
                if ((int64_t)(now - t0) > timeout_ns) {
                    atomicCAS(&c->err, 0, (int)DSSSP_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(256);
            }
            __threadfence();
        }
        ok = na_vload(&c->err) == 0;
    }
    __syncthreads();
    return ok != 0;
}

template <typename RP>
struct NaArgs {
    NaMem s;                      // working memory (the fixed array, or a graph handle's)
    const RP *row_ptr;            // int64 (caller's CSR) or uint32 (a graph handle's copy)
    const int32_t *col;
    const uint32_t *wbits;
    void *dist;
    int32_t *pred;
    double delta;
    int64_t timeout_ns;
    int64_t max_phases;
    uint32_t n, m, src, light_max;
    uint32_t nblocks;
    uint32_t validate;            // 1: check the CSR and the weights first
};

// Clear the state of the previous call, check the CSR, seed t[s] = 0.
template <int DT, typename RP>
__global__ void k_na_init(NaArgs<RP> a) {
    const NaMem &s = a.s;
    const uint32_t stride = gridDim.x * blockDim.x;
    const unsigned long long unreached = ((unsigned long long)na_inf<DT>() << 32) | NO_PRED;
    int bad = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        s.packed[v] = v == a.src ? (unsigned long long)a.src : unreached;
        s.fstamp[v] = v == a.src ? 1u : 0u;
        s.sstamp[v] = 0u;
        s.far[v] = 0u;
        if (a.validate) {
            const int64_t b = (int64_t)a.row_ptr[v], e = (int64_t)a.row_ptr[v + 1];
            if (b < 0 || e < b || e > (int64_t)a.m) bad |= 1;
        }
    }
    for (int64_t e = blockIdx.x * blockDim.x + threadIdx.x; a.validate && e < (int64_t)a.m; e += stride) {
        const int32_t h = a.col[e];
        if (h < 0 || (uint32_t)h >= a.n) bad |= 1;
        const uint32_t w = a.wbits[e];
        if (DT == DSSSP_F32 ? (w >= 0x7F800000u && w != 0x80000000u) : (int32_t)w < 0) bad |= 2;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.validate && (a.row_ptr[0] != 0 || (int64_t)a.row_ptr[a.n] != (int64_t)a.m)) bad |= 1;
        NaCtl &c = *s.ctl;
        c.bar_count = 0u;
        c.bar_gen = 0u;
        c.err = 0;
        c.mode = 0u;
        c.round = 1u;
        c.epoch = 1u;
        c.T = bucket_floor_key(1, DT, a.delta);
        c.next_count = 0u;
        c.far_min = na_inf<DT>();
        c.far_count = 0u;
        c.phases = 0;
    }
    if (bad) atomicOr(&s.ctl->flags, bad);
}

// Relax arcs [b, e) of row u (light ones or heavy ones) from key du, one warp.
template <int DT, typename RP>
__device__ void na_relax_row(const NaArgs<RP> &a, uint32_t u, uint32_t du, bool light, uint32_t T, uint32_t round,
                             uint32_t &far_min, uint32_t &next, uint32_t &farn) {
    const NaMem &s = a.s;
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t b = (int64_t)a.row_ptr[u], e = (int64_t)a.row_ptr[u + 1];
    bool ovf = false;
    for (int64_t k = b + lane; k < e; k += 32) {
        // a long row tells waiting blocks that it advances (every 64 x 32 arcs)
        if (lane == 0 && ((k - b) & 2047) == 2047 - 31) atomicAdd(&s.ctl->progress, 1ull);
        uint32_t w = a.wbits[k];
        if (DT == DSSSP_F32 && w == 0x80000000u) w = 0u;            // -0.0 is +0.0
        if ((w <= a.light_max) != light) continue;                   // A_L o t_Bi  /  A_H o S
        const uint32_t v = (uint32_t)a.col[k];
        const uint32_t ck = na_add<DT>(du, w);
        if (ck >= na_inf<DT>()) { ovf = true; continue; }           // checked again at the end
        const unsigned long long cand = ((unsigned long long)ck << 32) | u;
        if (cand >= __ldcg(&s.packed[v])) continue;
        const unsigned long long old = atomicMin(&s.packed[v], cand);
        if (cand >= old || (uint32_t)(old >> 32) <= ck) continue;      // no strict decrease
        if (ck < T) {                                               // back into bucket i
            if (atomicExch(&s.fstamp[v], round + 1u) != round + 1u) ++next;
        } else {                                                    // a later bucket
            far_min = min(far_min, ck);
            if (atomicExch(&s.far[v], 1u) == 0u) ++farn;
        }
    }
    if (__any_sync(0xffffffffu, ovf) && lane == 0) s.ctl->ovf = 1u;
}

template <int DT, typename RP>
__global__ void __launch_bounds__(kNaBlock) k_na_solve(NaArgs<RP> a) {
    const NaMem &s = a.s;
    NaCtl *c = s.ctl;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    __shared__ uint32_t b_far_min, b_next, b_farn;
    // invalid input (found by k_na_init, which completed before this launch):
    // every block leaves before touching the graph
    const int flags = na_vload(&c->flags);
    if (flags != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicCAS(&c->err, 0, (flags & 1) ? (int)DSSSP_ERR_BAD_GRAPH : (int)DSSSP_ERR_NEG_WEIGHT);
        return;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) { b_far_min = na_inf<DT>(); b_next = 0u; b_farn = 0u; }
        __syncthreads();
        if (na_vload(&c->err) != 0) break;
        const uint32_t mode = na_vload(&c->mode);
        if (mode == 3u) break;
        const uint32_t round = na_vload(&c->round), epoch = na_vload(&c->epoch), T = na_vload(&c->T);
        uint32_t far_min = na_inf<DT>(), next = 0u, farn = 0u;
        // each lane tests one vertex; the warp then scans the rows of the selected ones
        for (uint32_t base = gw * 32u; base < a.n; base += nw * 32u) {
            const uint32_t v = base + lane;
            bool sel = false;
            if (v < a.n) {
                if (mode == 0u) sel = __ldcg(&s.fstamp[v]) == round;          // t_Bi
                else if (mode == 1u) sel = __ldcg(&s.sstamp[v]) == epoch;     // S
                else sel = __ldcg(&s.far[v]) == 1u;                            // far pile
            }
            if (mode == 2u) {                                                  // next-bucket search
                if (sel) {
                    const uint32_t k = (uint32_t)(__ldcg(&s.packed[v]) >> 32);
                    if (k < T) {
                        s.far[v] = 0u;
                        if (atomicExch(&s.fstamp[v], round + 1u) != round + 1u) ++next;
                    } else {
                        far_min = min(far_min, k);
                        ++farn;
                    }
                }
                continue;
            }
            uint32_t mask = __ballot_sync(0xffffffffu, sel);
            while (mask) {
                const int l = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t u = base + (uint32_t)l;
                const uint32_t du = (uint32_t)(__ldcg(&s.packed[u]) >> 32);
                if (mode == 0u && lane == 0) {       // S = S u t_Bi; a far key of u is now stale
                    s.sstamp[u] = epoch;
                    s.far[u] = 0u;
                }
                na_relax_row<DT, RP>(a, u, du, mode == 0u, T, round, far_min, next, farn);
            }
        }
        if (far_min < na_inf<DT>()) atomicMin(&b_far_min, far_min);
        if (next) atomicAdd(&b_next, next);
        if (farn) atomicAdd(&b_farn, farn);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (b_far_min < na_inf<DT>()) atomicMin(&c->far_min, b_far_min);
            if (b_next) atomicAdd(&c->next_count, b_next);
            if (b_farn) atomicAdd(&c->far_count, b_farn);
        }
        const double delta = a.delta;
        const int64_t max_phases = a.max_phases;
        const bool ok = na_barrier(c, a.nblocks, a.timeout_ns, [c, mode, delta, max_phases]() {
            // the control flow of Fig. 1, on the dense vectors
            c->phases += 1;
            if (c->phases >= max_phases) {
                atomicCAS(&c->err, 0, (int)DSSSP_ERR_NOT_CONVERGED);
                c->mode = 3u;
                return;
            }
            const uint32_t next_count = c->next_count;
            c->next_count = 0u;
            if (mode == 0u) c->n_light += 1;
            else if (mode == 1u) c->n_heavy += 1;
            else c->n_select += 1;
            if (mode == 1u) c->epoch += 1u;
            if (next_count) {                                    // while t_Bi != 0: another light round
                c->round += 1u;
                c->mode = 0u;
                return;
            }
            if (mode == 0u) { c->mode = 1u; return; }            // bucket settled: heavy pass over S
            const uint32_t fm = c->far_min;
            if (fm >= na_inf<DT>()) { c->mode = 3u; return; }    // no later bucket holds a vertex
            const int64_t i = bucket_of_key(fm, DT, delta);
            uint32_t T = i < INT64_MAX ? bucket_floor_key(i + 1, DT, delta) : 0u;
            if (T <= fm) T = fm + 1u;
            c->T = T;
            c->far_min = na_inf<DT>();
            c->far_count = 0u;
            c->buckets += 1;
            c->mode = 2u;
        });
        if (!ok) break;
    }
}

// Overflow (reading R14): when a relaxation met a sum the weight type cannot
// hold, every arc of every reached vertex is tested again with its final
// distance; a confirmed overflow fails the call with DSSSP_ERR_OVERFLOW.
template <int DT, typename RP>
__global__ void __launch_bounds__(kNaBlock) k_na_verify(NaArgs<RP> a) {
    const NaMem &s = a.s;
    if (na_vload(&s.ctl->ovf) == 0u || na_vload(&s.ctl->err) != 0) return;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t u = gw; u < a.n; u += nw) {
        const uint32_t du = (uint32_t)(__ldcg(&s.packed[u]) >> 32);
        if (du >= na_inf<DT>()) continue;
        bool bad = false;
        for (int64_t k = (int64_t)a.row_ptr[u] + lane; k < (int64_t)a.row_ptr[u + 1]; k += 32) {
            uint32_t w = a.wbits[k];
            if (DT == DSSSP_F32 && w == 0x80000000u) w = 0u;
            bad |= na_add<DT>(du, w) >= na_inf<DT>();
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) atomicCAS(&s.ctl->err, 0, (int)DSSSP_ERR_OVERFLOW);
            return;
        }
    }
}

template <int DT, typename RP>
__global__ void k_na_unpack(NaArgs<RP> a) {
    const NaMem &s = a.s;
    if (na_vload(&s.ctl->err) != 0) return;            // outputs are written only on success
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
        const unsigned long long p = s.packed[v];
        const uint32_t k = (uint32_t)(p >> 32);
        if (DT == DSSSP_F32) ((float *)a.dist)[v] = __uint_as_float(k);
        else ((int32_t *)a.dist)[v] = (int32_t)k;
        if (a.pred) a.pred[v] = v == a.src ? (int32_t)a.src : (k >= na_inf<DT>() ? -1 : (int32_t)(uint32_t)p);
    }
}

template <int DT, typename RP>
cudaError_t enqueue_dense(const NaArgs<RP> &a, int grid, cudaStream_t st) {
    int init_grid = (int)((a.n > a.m ? a.n : a.m) / kNaBlock + 1);
    if (init_grid > 4096) init_grid = 4096;
    k_na_init<DT, RP><<<init_grid, kNaBlock, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel((const void *)k_na_solve<DT, RP>, dim3(grid), dim3(kNaBlock), args, 0, st);
    if (e != cudaSuccess) return e;
    k_na_verify<DT, RP><<<grid, kNaBlock, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_na_unpack<DT, RP><<<(int)(a.n / kNaBlock + 1), kNaBlock, 0, st>>>(a);
    return cudaGetLastError();
}

// Co-resident blocks of the dense solver on this device (both dtypes, both row types).
int dense_grid(int dev) {
    static std::mutex mu;
    static int grid[64] = {};
    if (dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (grid[dev] == 0) {
        int sms = 0, lo = 1 << 30;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const void *fns[] = {(const void *)k_na_solve<DSSSP_F32, int64_t>, (const void *)k_na_solve<DSSSP_I32, int64_t>,
                             (const void *)k_na_solve<DSSSP_F32, uint32_t>, (const void *)k_na_solve<DSSSP_I32, uint32_t>};
        for (const void *f : fns) {
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kNaBlock, 0) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            lo = per_sm < lo ? per_sm : lo;
        }
        grid[dev] = sms * lo;
    }
    return grid[dev];
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
NaScratch *g_na_ptr[kMaxDevices] = {};

dsssp_status na_setup(int dev, NaScratch **ptr, int *grid) {
    if (dev < 0 || dev >= kMaxDevices) return DSSSP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        // In host code g_noalloc_scratch names a host-side stand-in; the kernels
        // need the device address of this device's copy.
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DSSSP_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<NaScratch *>(p);
    }
    *ptr = g_na_ptr[dev];
    *grid = dense_grid(dev);
    return *grid > 0 ? DSSSP_OK : DSSSP_ERR_UNSUPPORTED;
}

}  // namespace

namespace dsssp {

cudaError_t dense_solve_launch(const uint32_t *off, const int32_t *col, const uint32_t *wbits, int dtype,
                               uint32_t n, uint32_t m, uint32_t src, double delta, const NaMem &mem, void *dist,
                               int32_t *pred, int64_t timeout_ns, int64_t max_phases, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int grid = dense_grid(dev);
    if (grid < 1) return cudaErrorNotSupported;
    NaArgs<uint32_t> a{};
    a.s = mem;
    a.row_ptr = off;
    a.col = col;
    a.wbits = wbits;
    a.dist = dist;
    a.pred = pred;
    a.delta = delta;
    a.timeout_ns = timeout_ns;
    a.max_phases = max_phases;
    a.n = n;
    a.m = m;
    a.src = src;
    a.light_max = light_max_key(dtype, delta);
    a.nblocks = (uint32_t)grid;
    a.validate = 0u;                  // the handle's CSR was validated at creation
    if ((e = cudaMemsetAsync(mem.ctl, 0, sizeof(NaCtl), st)) != cudaSuccess) return e;
    return dtype == DSSSP_F32 ? enqueue_dense<DSSSP_F32, uint32_t>(a, grid, st)
                              : enqueue_dense<DSSSP_I32, uint32_t>(a, grid, st);
}

}  // namespace dsssp

extern "C" dsssp_status dsssp_solve_noalloc(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                            const void *w, dsssp_dtype dtype, int32_t src, double delta,
                                            void *dist, int32_t *pred, void *stream) {
    if (n < 1 || m < 0 || m > ((int64_t)1 << 31) - 1 || !row_ptr || (m > 0 && (!col || !w)) || !dist)
        return DSSSP_ERR_INVALID_ARG;
    if (n > (int64_t)kNoAllocMaxVertices) return DSSSP_ERR_TOO_LARGE;
    if (src < 0 || (int64_t)src >= n || !(delta > 0.0) || (dtype != DSSSP_I32 && dtype != DSSSP_F32))
        return DSSSP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // the call waits for its result on the host, which a stream being captured
    // into a CUDA graph does not allow: refuse before any other CUDA call
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) { cudaGetLastError(); return DSSSP_ERR_CUDA; }
    if (cap != cudaStreamCaptureStatusNone) return DSSSP_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return DSSSP_ERR_CUDA; }
    NaScratch *scratch = nullptr;
    int grid = 0;
    dsssp_status st = na_setup(dev, &scratch, &grid);
    if (st != DSSSP_OK) return st;
    NaArgs<int64_t> a{};
    a.s.packed = scratch->packed;
    a.s.fstamp = scratch->fstamp;
    a.s.sstamp = scratch->sstamp;
    a.s.far = scratch->far;
    a.s.ctl = &scratch->ctl;
    a.row_ptr = row_ptr;
    a.col = col;
    a.wbits = static_cast<const uint32_t *>(w);
    a.dist = dist;
    a.pred = pred;
    a.delta = delta;
    a.timeout_ns = 2000000000LL;
    a.max_phases = (int64_t)1 << 26;
    a.n = (uint32_t)n;
    a.m = (uint32_t)m;
    a.src = (uint32_t)src;
    a.light_max = light_max_key(dtype, delta);
    a.nblocks = (uint32_t)grid;
    a.validate = 1u;
    // the previous call's control words, validation flags included, start at zero
    cudaError_t e = cudaMemsetAsync(&scratch->ctl, 0, sizeof(NaCtl), s);
    if (e == cudaSuccess)
        e = dtype == DSSSP_F32 ? enqueue_dense<DSSSP_F32, int64_t>(a, grid, s) : enqueue_dense<DSSSP_I32, int64_t>(a, grid, s);
    int32_t err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&err, &scratch->ctl.err, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DSSSP_ERR_CUDA;
    }
    return (dsssp_status)err;
}
