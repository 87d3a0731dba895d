// api.cu -- host side of the C ABI declared in include/dsssp.h: graph handles,
// the per-Delta split cache, the solver workspace and launch orchestration.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "dense.cuh"
#include "graph.cuh"

using namespace dsssp;

namespace dsssp {

dsssp_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DSSSP_OK;
    if (e == cudaErrorMemoryAllocation) return DSSSP_ERR_OOM;
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) return DSSSP_ERR_UNSUPPORTED;
    return DSSSP_ERR_CUDA;
}

void free_split(Split &s) {
    cudaFree(s.arcs);
    cudaFree(s.vinfo);
    cudaFree(s.perm);
    s = Split{};
}

dsssp_status ensure_split(dsssp_graph *g, double delta, cudaStream_t st, Split **out) {
    g->use_clock++;
    for (auto &s : g->splits) {
        if (s.valid && (s.delta == delta || (std::isinf(s.delta) && std::isinf(delta)))) {
            s.last_use = g->use_clock;
            *out = &s;
            return DSSSP_OK;
        }
    }
    // a free slot, else the least recently used split that no batch holds
    Split *slot = nullptr;
    for (auto &s : g->splits) {
        if (!s.valid) { slot = &s; break; }
        if (s.pins == 0 && (!slot || s.last_use < slot->last_use)) slot = &s;
    }
    if (!slot) return DSSSP_ERR_UNSUPPORTED;
    if (slot->valid) {
        DSSSP_TRY(cudaStreamSynchronize(st));
        free_split(*slot);
    }
    const size_t m = (size_t)g->m, n = (size_t)g->n;
    DSSSP_TRY(cudaMalloc(&slot->arcs, (m ? m : 1) * sizeof(uint2)));
    DSSSP_TRY(cudaMalloc(&slot->vinfo, n * sizeof(uint4)));
    DSSSP_TRY(cudaMalloc(&slot->perm, (m ? m : 1) * sizeof(uint32_t)));
    uint32_t *pl = nullptr, *tiles = nullptr;
    DSSSP_TRY(cudaMallocAsync(&pl, (m + 1) * sizeof(uint32_t), st));
    DSSSP_TRY(cudaMallocAsync(&tiles, split_scratch_tiles((int64_t)m) * sizeof(uint32_t), st));
    const uint32_t lmax = light_max_key(g->dtype, delta);
    cudaError_t e = launch_split(g->n, g->m, g->off, g->col, g->wbits, lmax, pl, tiles, slot->arcs,
                                 slot->vinfo, slot->perm, st);
    cudaFreeAsync(pl, st);
    cudaFreeAsync(tiles, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_split(*slot);
        return cuda_status(e);
    }
    slot->delta = delta;
    slot->valid = true;
    slot->last_use = g->use_clock;
    *out = slot;
    return DSSSP_OK;
}

}  // namespace dsssp

namespace {

__global__ void k_sticky(const int32_t *err, int32_t *sticky) {
    int e = *(const volatile int *)err;
    if (e != 0) atomicCAS(sticky, 0, e);
}

dsssp_status ensure_workspace(dsssp_graph *g) {
    if (g->ws) return DSSSP_OK;
    const size_t n = (size_t)g->n;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t bytes = 0;
    const size_t o_packed = bytes; bytes += up(n * 8);
    const size_t o_near = bytes;   bytes += up(n * 4);
    const size_t o_s = bytes;      bytes += up(n * 4);
    const size_t o_b = bytes;      bytes += up(n * 4);
    const size_t o_ovf = bytes;    bytes += up(n * 4);
    const size_t o_f0 = bytes;     bytes += up(n * 8);
    const size_t o_f1 = bytes;     bytes += up(n * 8);
    const size_t o_s0 = bytes;     bytes += up(n * 8);
    const size_t o_s1 = bytes;     bytes += up(n * 8);
    const size_t o_sl = bytes;     bytes += up(n * 8 * kSlots);
    const size_t o_sh = bytes;     bytes += up(n * 4 * kSlots);
    const size_t o_ov0 = bytes;    bytes += up(n * 4);
    const size_t o_ov1 = bytes;    bytes += up(n * 4);
    const uint32_t dcap = solve_dir_entries((uint32_t)g->n, (uint32_t)g->m);
    const size_t o_dir = bytes;    bytes += up((size_t)dcap * kDirLists * 8);
    const size_t o_ctl = bytes;    bytes += up(sizeof(Ctl));
    const size_t o_nactl = bytes;  bytes += up(sizeof(NaCtl));
    const size_t o_team = bytes;   bytes += up(team_region_bytes());
    const size_t o_sticky = bytes; bytes += up(sizeof(int32_t));
    char *base = nullptr;
    DSSSP_TRY(cudaMalloc(&base, bytes));
    DSSSP_TRY(cudaMemset(base + o_ctl, 0, sizeof(Ctl)));
    DSSSP_TRY(cudaMemset(base + o_sticky, 0, sizeof(int32_t)));
    g->ws = base;
    g->ws_bytes = bytes;
    SolveArgs &a = g->args;
    a.packed = (unsigned long long *)(base + o_packed);
    a.near_stamp = (uint32_t *)(base + o_near);
    a.s_stamp = (uint32_t *)(base + o_s);
    a.b_stamp = (uint32_t *)(base + o_b);
    a.ov_flag = (uint32_t *)(base + o_ovf);
    a.F0 = (uint2 *)(base + o_f0);
    a.F1 = (uint2 *)(base + o_f1);
    a.S0 = (uint2 *)(base + o_s0);
    a.S1 = (uint2 *)(base + o_s1);
    a.SL = (uint2 *)(base + o_sl);
    a.SH = (uint32_t *)(base + o_sh);
    a.OV0 = (uint32_t *)(base + o_ov0);
    a.OV1 = (uint32_t *)(base + o_ov1);
    a.dir = (uint2 *)(base + o_dir);
    a.dcap = dcap;
    a.ctl = (Ctl *)(base + o_ctl);
    g->ctl = a.ctl;
    g->nactl = (NaCtl *)(base + o_nactl);
    g->team_region = base + o_team;
    g->sticky = (int32_t *)(base + o_sticky);
    return DSSSP_OK;
}

void fill_stats(const Ctl &ctl, int grid, int block, dsssp_stats *s) {
    const long long *st = ctl.ss.st;
    std::memset(s, 0, sizeof *s);
    s->buckets = st[ST_BUCKETS];
    s->light_phases = st[ST_LIGHT];
    s->heavy_phases = st[ST_HEAVY];
    s->rebin_phases = st[ST_REBIN];
    s->vertices_light = st[ST_VLIGHT];
    s->vertices_heavy = st[ST_VHEAVY];
    s->arcs_light = st[ST_ALIGHT];
    s->arcs_heavy = st[ST_AHEAVY];
    s->far_scanned = st[ST_FARSCAN];
    s->improvements = st[ST_IMPROVE];
    s->ns_light = st[ST_NSLIGHT];
    s->ns_heavy = st[ST_NSHEAVY];
    s->ns_rebin = st[ST_NSREBIN];
    s->ns_total = st[ST_NSTOTAL];
    s->ns_first_arrival = st[ST_NSFIRST];
    s->ns_arrival_spread = st[ST_NSSPREAD];
    s->grid_size = grid;
    s->block_size = block;
}

}  // namespace

extern "C" {

const char *dsssp_status_string(dsssp_status s) {
    switch (s) {
    case DSSSP_OK: return "ok";
    case DSSSP_ERR_INVALID_ARG: return "invalid argument";
    case DSSSP_ERR_BAD_GRAPH: return "malformed CSR graph";
    case DSSSP_ERR_NEG_WEIGHT: return "negative, NaN or infinite weight";
    case DSSSP_ERR_NOT_CONVERGED: return "phase cap reached before convergence";
    case DSSSP_ERR_TIMEOUT: return "bounded device-side wait timed out";
    case DSSSP_ERR_CUDA: return "CUDA runtime error";
    case DSSSP_ERR_NO_TAPE: return "no tape";
    case DSSSP_ERR_OOM: return "out of device memory";
    case DSSSP_ERR_UNSUPPORTED: return "unsupported device or launch shape";
    case DSSSP_ERR_TOO_LARGE: return "graph exceeds the fixed working memory of the no-allocation solve";
    case DSSSP_ERR_DEGENERATE: return "predecessor graph has a cycle (zero-weight ties): gradient undefined";
    case DSSSP_ERR_OVERFLOW: return "a path sum overflows the weight type";
    }
    return "unknown status";
}

dsssp_status dsssp_options_default(dsssp_options *opt) {
    if (!opt) return DSSSP_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof *opt);
    opt->struct_size = sizeof *opt;
    opt->mode = DSSSP_MODE_PERSISTENT;
    opt->block_size = 512;
    opt->grid_size = 0;
    opt->max_phases = (int64_t)1 << 26;
    opt->timeout_ns = 2000000000LL;
    opt->solo_work = 2048;
    return DSSSP_OK;
}

dsssp_status dsssp_graph_create(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                const void *w, dsssp_dtype dtype, int device_ptrs, void *stream,
                                dsssp_graph **out) {
    if (!out) return DSSSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n > ((int64_t)1 << 31) - 2 || m < 0 || m > ((int64_t)1 << 31) - 1) return DSSSP_ERR_INVALID_ARG;
    if (!row_ptr || (m > 0 && (!col || !w))) return DSSSP_ERR_INVALID_ARG;
    if (dtype != DSSSP_I32 && dtype != DSSSP_F32) return DSSSP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    dsssp_graph *g = new (std::nothrow) dsssp_graph();
    if (!g) return DSSSP_ERR_OOM;
    g->n = n;
    g->m = m;
    g->dtype = dtype;
    auto fail = [&](dsssp_status s) {
        dsssp_graph_destroy(g);
        return s;
    };
    if (cudaGetDevice(&g->device) != cudaSuccess) return fail(DSSSP_ERR_CUDA);
    if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
        return fail(DSSSP_ERR_CUDA);
    const size_t mm = m ? (size_t)m : 1;
    int64_t *rp_dev = nullptr;
    int *flags = nullptr;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&g->off, (size_t)(n + 1) * sizeof(uint32_t))) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMalloc(&g->col, mm * sizeof(int32_t))) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMalloc(&g->wbits, mm * sizeof(uint32_t))) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMallocHost(&g->ctl_host, sizeof(Ctl))) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMallocAsync(&flags, sizeof(int), st)) != cudaSuccess) return fail(cuda_status(e));
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (device_ptrs) {
        rp_dev = const_cast<int64_t *>(row_ptr);
    } else {
        if ((e = cudaMallocAsync(&rp_dev, (size_t)(n + 1) * sizeof(int64_t), st)) != cudaSuccess) return fail(cuda_status(e));
        e = cudaMemcpyAsync(rp_dev, row_ptr, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->col, col, (size_t)m * sizeof(int32_t), kind, st);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->wbits, w, (size_t)m * sizeof(uint32_t), kind, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_validate(n, m, rp_dev, g->col, g->wbits, dtype, g->off, flags, st);
    int hflags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!device_ptrs && rp_dev) cudaFreeAsync(rp_dev, st);
    cudaFreeAsync(flags, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(cuda_status(e));
    }
    if (hflags & 1) return fail(DSSSP_ERR_BAD_GRAPH);
    if (hflags & 2) return fail(DSSSP_ERR_NEG_WEIGHT);
    *out = g;
    return DSSSP_OK;
}

dsssp_status dsssp_graph_destroy(dsssp_graph *g) {
    if (!g) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    for (auto &s : g->splits) free_split(s);
    cudaFree(g->off);
    cudaFree(g->col);
    cudaFree(g->wbits);
    cudaFree(g->ws);
    if (g->ctl_host) cudaFreeHost(g->ctl_host);
    delete g;
    return DSSSP_OK;
}

dsssp_status dsssp_graph_info(const dsssp_graph *g, int64_t *n, int64_t *m, int32_t *dtype) {
    if (!g) return DSSSP_ERR_INVALID_ARG;
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (dtype) *dtype = g->dtype;
    return DSSSP_OK;
}

dsssp_status dsssp_prepare(dsssp_graph *g, double delta, void *stream) {
    if (!g || !(delta > 0.0)) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    Split *s = nullptr;
    return ensure_split(g, delta, (cudaStream_t)stream, &s);
}

dsssp_status dsssp_solve(dsssp_graph *g, int32_t src, double delta, void *dist, int32_t *pred,
                         const dsssp_options *opt_in, dsssp_stats *stats, void *stream) {
    if (!g || !dist || src < 0 || (int64_t)src >= g->n || !(delta > 0.0)) return DSSSP_ERR_INVALID_ARG;
    dsssp_options opt;
    dsssp_options_default(&opt);
    if (opt_in) {
        if (opt_in->struct_size != sizeof(dsssp_options)) return DSSSP_ERR_INVALID_ARG;
        opt.flags = opt_in->flags;
        opt.mode = opt_in->mode;
        if (opt_in->block_size) opt.block_size = opt_in->block_size;
        if (opt_in->grid_size) opt.grid_size = opt_in->grid_size;
        if (opt_in->solo_work) opt.solo_work = opt_in->solo_work;
        if (opt_in->max_phases) opt.max_phases = opt_in->max_phases;
        if (opt_in->timeout_ns) opt.timeout_ns = opt_in->timeout_ns;
        opt.test_hook = opt_in->test_hook;
        opt.team_blocks = opt_in->team_blocks;
    }
    if (opt.block_size < 32 || opt.block_size > 512 || opt.block_size % 32 != 0) return DSSSP_ERR_INVALID_ARG;
    if (opt.max_phases < 1 || opt.timeout_ns < 1 || opt.grid_size < 0) return DSSSP_ERR_INVALID_ARG;
    if (opt.mode != DSSSP_MODE_PERSISTENT && opt.mode != DSSSP_MODE_STEPPED && opt.mode != DSSSP_MODE_DENSE &&
        opt.mode != DSSSP_MODE_TEAM)
        return DSSSP_ERR_INVALID_ARG;
    if (opt.team_blocks != 0 && opt.team_blocks != 1 && opt.team_blocks != 2 && opt.team_blocks != 4 &&
        opt.team_blocks != 8 && opt.team_blocks != 16)
        return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (opt.mode == DSSSP_MODE_DENSE) {
        // the full-vector form on the handle's own CSR; working memory from the workspace
        dsssp_status rc = ensure_workspace(g);
        if (rc != DSSSP_OK) return rc;
        NaMem mem;
        mem.packed = g->args.packed;
        mem.fstamp = g->args.near_stamp;
        mem.sstamp = g->args.s_stamp;
        mem.far = g->args.b_stamp;
        mem.ctl = g->nactl;
        DSSSP_TRY(dense_solve_launch(g->off, g->col, g->wbits, g->dtype, (uint32_t)g->n, (uint32_t)g->m,
                                     (uint32_t)src, delta, mem, dist, pred, opt.timeout_ns, opt.max_phases, st));
        k_sticky<<<1, 1, 0, st>>>(&g->nactl->err, g->sticky);
        DSSSP_TRY(cudaGetLastError());
        if ((opt.flags & DSSSP_FLAG_ASYNC) && !stats) return DSSSP_OK;
        NaCtl hc;
        DSSSP_TRY(cudaMemcpyAsync(&hc, g->nactl, sizeof(NaCtl), cudaMemcpyDeviceToHost, st));
        DSSSP_TRY(cudaStreamSynchronize(st));
        if (stats) {
            std::memset(stats, 0, sizeof *stats);
            stats->buckets = hc.buckets + 1;
            stats->light_phases = hc.n_light;
            stats->heavy_phases = hc.n_heavy;
        }
        if (hc.err != 0) {
            cudaMemsetAsync(g->sticky, 0, sizeof(int32_t), st);
            return (dsssp_status)hc.err;
        }
        return DSSSP_OK;
    }
    Split *sp = nullptr;
    dsssp_status rc = ensure_split(g, delta, st, &sp);
    if (rc != DSSSP_OK) return rc;
    if ((rc = ensure_workspace(g)) != DSSSP_OK) return rc;

    if (opt.mode == DSSSP_MODE_TEAM) {
        // one instance of the batch kernel on one thread-block cluster (16 blocks unless
        // asked otherwise; 8 where a 16-block cluster cannot be scheduled)
        int tb = opt.team_blocks ? opt.team_blocks : 16;
        cudaError_t e = team_solve_launch(g, sp, src, delta, dist, pred, tb, opt.max_phases, st);
        if (e != cudaSuccess && opt.team_blocks == 0) {
            cudaGetLastError();
            tb = 8;
            e = team_solve_launch(g, sp, src, delta, dist, pred, tb, opt.max_phases, st);
        }
        DSSSP_TRY(e);
        k_sticky<<<1, 1, 0, st>>>(team_err(g), g->sticky);
        DSSSP_TRY(cudaGetLastError());
        if ((opt.flags & DSSSP_FLAG_ASYNC) && !stats) return DSSSP_OK;
        int herr = 0;
        long long hst[kTeamStatsCount];
        DSSSP_TRY(cudaMemcpyAsync(&herr, team_err(g), sizeof(int), cudaMemcpyDeviceToHost, st));
        DSSSP_TRY(cudaMemcpyAsync(hst, team_stats(g), sizeof(hst), cudaMemcpyDeviceToHost, st));
        DSSSP_TRY(cudaStreamSynchronize(st));
        if (stats) {
            std::memset(stats, 0, sizeof *stats);
            team_stats_to_solve(hst, stats);
            stats->grid_size = tb;
            stats->block_size = 512;
        }
        if (herr != 0) {
            cudaMemsetAsync(g->sticky, 0, sizeof(int32_t), st);
            return (dsssp_status)herr;
        }
        return DSSSP_OK;
    }

    // grid: all co-resident blocks (the persistent kernel waits on every block)
    if (g->occ_block != opt.block_size) {
        int bps = 0;
        DSSSP_TRY(solve_occupancy(opt.block_size, &bps));
        g->occ_block = opt.block_size;
        g->occ_blocks_per_sm = bps;
    }
    const int max_grid = g->occ_blocks_per_sm * g->sm_count;
    if (max_grid < 1) return DSSSP_ERR_UNSUPPORTED;
    int grid = opt.grid_size ? opt.grid_size : max_grid;
    if (opt.mode == DSSSP_MODE_PERSISTENT && grid > max_grid) return DSSSP_ERR_UNSUPPORTED;
    if (opt.test_hook == DSSSP_HOOK_STALL_BARRIER && grid < 2) return DSSSP_ERR_INVALID_ARG;

    SolveArgs a = g->args;
    a.vinfo = sp->vinfo;
    a.arcs = sp->arcs;
    a.delta = delta;
    a.timeout_ns = opt.timeout_ns;
    a.max_phases = opt.max_phases;
    a.n = (uint32_t)g->n;
    a.m = (uint32_t)g->m;
    // persistent mode only: the stepped mode has no grid barrier to save
    a.solo_work = (opt.mode == DSSSP_MODE_PERSISTENT && opt.solo_work > 0) ? (uint32_t)opt.solo_work : 0u;
    a.fuse = (opt.flags & DSSSP_FLAG_NO_FUSE) ? 0u : 1u;
    a.src = (uint32_t)src;
    a.inf_key = key_inf(g->dtype);
    a.dtype = g->dtype;
    a.test_hook = opt.test_hook;
    a.nblocks = (uint32_t)grid;

    DSSSP_TRY(launch_init(a, st));
    if (opt.mode == DSSSP_MODE_PERSISTENT) {
        DSSSP_TRY(launch_solve_persistent(a, grid, opt.block_size, st));
    } else {
        // host-driven loop: one kernel per phase, the serial step as a 1-warp kernel
        for (int64_t ph = 0;; ++ph) {
            DSSSP_TRY(cudaMemcpyAsync(g->ctl_host, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
            DSSSP_TRY(cudaStreamSynchronize(st));
            const uint32_t mode = g->ctl_host->desc.mode;
            if (mode == MODE_DONE || g->ctl_host->err != 0) break;
            DSSSP_TRY(launch_phase_stepped(a, mode, grid, opt.block_size, st));
            DSSSP_TRY(launch_serial_step(a, st));
        }
        DSSSP_TRY(launch_verify_overflow(a, grid, opt.block_size, st));
    }
    DSSSP_TRY(launch_unpack(a, dist, pred, st));
    k_sticky<<<1, 1, 0, st>>>(&g->ctl->err, g->sticky);
    DSSSP_TRY(cudaGetLastError());
    if ((opt.flags & DSSSP_FLAG_ASYNC) && !stats) return DSSSP_OK;
    DSSSP_TRY(cudaMemcpyAsync(g->ctl_host, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    DSSSP_TRY(cudaStreamSynchronize(st));
    if (stats) fill_stats(*g->ctl_host, grid, opt.block_size, stats);
    const int err = g->ctl_host->err;
    if (err != 0) {
        cudaMemsetAsync(g->sticky, 0, sizeof(int32_t), st);
        return (dsssp_status)err;
    }
    return DSSSP_OK;
}

dsssp_status dsssp_graph_sync(dsssp_graph *g, void *stream) {
    if (!g) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!g->sticky) {
        DSSSP_TRY(cudaStreamSynchronize(st));
        return DSSSP_OK;
    }
    int32_t h = 0;
    DSSSP_TRY(cudaMemcpyAsync(&h, g->sticky, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DSSSP_TRY(cudaMemsetAsync(g->sticky, 0, sizeof(int32_t), st));
    DSSSP_TRY(cudaStreamSynchronize(st));
    return (dsssp_status)h;
}

}  // extern "C"
