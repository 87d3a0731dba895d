// tune.cu -- choice of Delta by timing sample solves on this GPU.
//
// Delta sets how much work delta-stepping does per phase and how many phases
// it needs (Section III: a small Delta approaches Dijkstra's order and many
// phases, a large one Bellman-Ford's redundant relaxations in few phases). The
// paper picks Delta by hand; here a ladder of powers of two around a starting
// point, then a few refinement steps around the fastest, are timed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "graph.cuh"

using namespace dsssp;

namespace {

// Sum of the weights (as doubles) of a graph's arcs.
__global__ void k_weight_sum(const uint32_t *wbits, uint32_t m, int dtype, double *out) {
    double s = 0.0;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
        s += dtype == DSSSP_F32 ? (double)__uint_as_float(wbits[e]) : (double)wbits[e];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31u) == 0) atomicAdd(out, s);
}

dsssp_status start_point(dsssp_graph *g, cudaStream_t st, double *d0) {
    if (g->m == 0) {
        *d0 = 1.0;
        return DSSSP_OK;
    }
    double *dsum = nullptr, hsum = 0.0;
    DSSSP_TRY(cudaMallocAsync(&dsum, sizeof(double), st));
    cudaError_t e = cudaMemsetAsync(dsum, 0, sizeof(double), st);
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<int64_t>(1024, (g->m + 255) / 256);
        k_weight_sum<<<blocks, 256, 0, st>>>(g->wbits, (uint32_t)g->m, g->dtype, dsum);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hsum, dsum, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dsum, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    const double mean_w = hsum / (double)g->m;
    const double mean_deg = (double)g->m / (double)g->n;
    *d0 = mean_w > 0.0 ? 4.0 * mean_w / std::max(1.0, mean_deg) : 1.0;
    return DSSSP_OK;
}

struct Tried {
    double delta;
    double ms;
};

// Device time of k dsssp_solve calls at one Delta (split built before timing);
// solo_work as in dsssp_options (0: default).
dsssp_status time_solves_opt(dsssp_graph *g, const int32_t *src, int32_t k, double delta, cudaStream_t st,
                             double *ms, const dsssp_options &base);

dsssp_status time_solves(dsssp_graph *g, const int32_t *src, int32_t k, double delta, cudaStream_t st, double *ms,
                         int32_t solo_work = 0) {
    dsssp_options o;
    dsssp_options_default(&o);
    if (solo_work) o.solo_work = solo_work;
    return time_solves_opt(g, src, k, delta, st, ms, o);
}

// Device time of k solves with the options `base` (asynchronous, one warm-up solve first).
dsssp_status time_solves_opt(dsssp_graph *g, const int32_t *src, int32_t k, double delta, cudaStream_t st,
                             double *ms, const dsssp_options &base) {
    dsssp_status rc = dsssp_prepare(g, delta, st);
    if (rc != DSSSP_OK) return rc;
    const size_t n = (size_t)g->n;
    void *dist = nullptr;
    int32_t *pred = nullptr;
    DSSSP_TRY(cudaMallocAsync(&dist, n * 4, st));
    DSSSP_TRY(cudaMallocAsync((void **)&pred, n * 4, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dsssp_options o = base;
    o.flags |= DSSSP_FLAG_ASYNC;
    rc = dsssp_solve(g, src[0], delta, dist, pred, &o, nullptr, st);      // warm-up
    if (rc == DSSSP_OK) rc = dsssp_graph_sync(g, st);
    if (rc == DSSSP_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = DSSSP_ERR_CUDA;
    for (int32_t i = 0; i < k && rc == DSSSP_OK; ++i) rc = dsssp_solve(g, src[i], delta, dist, pred, &o, nullptr, st);
    if (rc == DSSSP_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = DSSSP_ERR_CUDA;
    if (rc == DSSSP_OK) rc = dsssp_graph_sync(g, st);
    float t = 0.f;
    if (rc == DSSSP_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = DSSSP_ERR_CUDA;
    *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(dist, st);
    cudaFreeAsync(pred, st);
    cudaStreamSynchronize(st);
    return rc;
}

// Device time per (graph, Delta) pair, each pair's k sources solved as instances
// of one batch; the cost of a pair is the sum of its instances' device times.
dsssp_status time_batch(const std::vector<dsssp_graph *> &gs, const std::vector<double> &deltas,
                        const std::vector<std::vector<int32_t>> &srcs, cudaStream_t st, std::vector<double> &ms) {
    const int32_t np = (int32_t)gs.size();
    std::vector<int32_t> src, sg;
    for (int32_t p = 0; p < np; ++p)
        for (int32_t s : srcs[p]) {
            src.push_back(s);
            sg.push_back(p);
        }
    const int32_t ni = (int32_t)src.size();
    std::vector<void *> dist(ni, nullptr);
    size_t total = 0;
    std::vector<size_t> off(ni);
    for (int32_t i = 0; i < ni; ++i) {
        off[i] = total;
        total += ((size_t)gs[sg[i]]->n * 4 + 255) & ~(size_t)255;
    }
    char *buf = nullptr;
    DSSSP_TRY(cudaMalloc(&buf, std::max<size_t>(total, 256)));
    for (int32_t i = 0; i < ni; ++i) dist[i] = buf + off[i];
    std::vector<dsssp_batch_stats> bst(ni);
    dsssp_batch *b = nullptr;
    dsssp_status rc = dsssp_batch_create(gs.data(), np, deltas.data(), ni, src.data(), sg.data(), dist.data(),
                                         nullptr, 0u, nullptr, st, &b);
    if (rc == DSSSP_OK) rc = dsssp_batch_run(b, st);
    if (rc == DSSSP_OK) rc = dsssp_batch_sync(b, bst.data(), st);
    if (b) dsssp_batch_destroy(b);
    cudaFree(buf);
    if (rc != DSSSP_OK) return rc;
    ms.assign(np, 0.0);
    for (int32_t i = 0; i < ni; ++i) ms[sg[i]] += (double)bst[i].ns * 1e-6;
    return DSSSP_OK;
}

}  // namespace

extern "C" dsssp_status dsssp_autotune(dsssp_graph *const *graphs, int32_t n_graphs, const int32_t *sample_src,
                                       int32_t k, const dsssp_tune_options *opt_in, double *delta_out,
                                       double *ms_out, void *stream) {
    if (!graphs || n_graphs < 1 || !sample_src || k < 1 || !delta_out) return DSSSP_ERR_INVALID_ARG;
    dsssp_tune_options opt;
    std::memset(&opt, 0, sizeof opt);
    opt.struct_size = sizeof opt;
    opt.target = DSSSP_TUNE_SOLVE;
    opt.refine = 2;
    if (opt_in) {
        if (opt_in->struct_size != sizeof(dsssp_tune_options)) return DSSSP_ERR_INVALID_ARG;
        opt = *opt_in;
        if (opt.refine == 0) opt.refine = 2;
    }
    if (opt.target != DSSSP_TUNE_SOLVE && opt.target != DSSSP_TUNE_BATCH) return DSSSP_ERR_INVALID_ARG;
    if (opt.n_candidates < 0 || opt.n_candidates > 16) return DSSSP_ERR_INVALID_ARG;
    for (int32_t i = 0; i < opt.n_candidates; ++i)
        if (!(opt.candidates[i] > 0.0)) return DSSSP_ERR_INVALID_ARG;
    for (int32_t gi = 0; gi < n_graphs; ++gi) {
        if (!graphs[gi] || graphs[gi]->dtype != graphs[0]->dtype) return DSSSP_ERR_INVALID_ARG;
        for (int32_t j = 0; j < k; ++j) {
            const int32_t s = sample_src[(size_t)gi * k + j];
            if (s < 0 || (int64_t)s >= graphs[gi]->n) return DSSSP_ERR_INVALID_ARG;
        }
    }
    DeviceGuard dg(graphs[0]->device);
    cudaStream_t st = (cudaStream_t)stream;
    // candidates per graph
    std::vector<std::vector<Tried>> tried(n_graphs);
    std::vector<std::vector<double>> todo(n_graphs);
    for (int32_t gi = 0; gi < n_graphs; ++gi) {
        if (opt.n_candidates > 0) {
            todo[gi].assign(opt.candidates, opt.candidates + opt.n_candidates);
        } else {
            double d0 = 1.0;
            dsssp_status rc = start_point(graphs[gi], st, &d0);
            if (rc != DSSSP_OK) return rc;
            for (int j = -3; j <= 3; ++j) todo[gi].push_back(std::ldexp(d0, j));
        }
    }
    auto best_of = [&](int32_t gi) {
        const Tried *b = nullptr;
        for (const Tried &t : tried[gi])
            if (!b || t.ms < b->ms) b = &t;
        return b;
    };
    auto evaluate = [&]() -> dsssp_status {
        if (opt.target == DSSSP_TUNE_SOLVE) {
            for (int32_t gi = 0; gi < n_graphs; ++gi)
                for (double d : todo[gi]) {
                    double ms = 0.0;
                    dsssp_status rc = time_solves(graphs[gi], sample_src + (size_t)gi * k, k, d, st, &ms);
                    if (rc != DSSSP_OK) return rc;
                    tried[gi].push_back({d, ms});
                }
        } else {
            // at most 3 Deltas of one graph per tuning batch (a handle caches 4 splits)
            for (size_t c0 = 0;; c0 += 3) {
                std::vector<dsssp_graph *> gs;
                std::vector<double> ds;
                std::vector<std::vector<int32_t>> ss;
                std::vector<int32_t> owner;
                for (int32_t gi = 0; gi < n_graphs; ++gi)
                    for (size_t c = c0; c < std::min(todo[gi].size(), c0 + 3); ++c) {
                        gs.push_back(graphs[gi]);
                        ds.push_back(todo[gi][c]);
                        ss.emplace_back(sample_src + (size_t)gi * k, sample_src + (size_t)(gi + 1) * k);
                        owner.push_back(gi);
                    }
                if (gs.empty()) break;
                std::vector<double> ms;
                dsssp_status rc = time_batch(gs, ds, ss, st, ms);
                if (rc != DSSSP_OK) return rc;
                for (size_t p = 0; p < gs.size(); ++p) tried[owner[p]].push_back({ds[p], ms[p]});
            }
        }
        for (auto &t : todo) t.clear();
        return DSSSP_OK;
    };
    dsssp_status rc = evaluate();
    if (rc != DSSSP_OK) return rc;
    for (int r = 1; r <= opt.refine; ++r) {
        const double step = std::exp2(1.0 / (double)(1 << r));
        for (int32_t gi = 0; gi < n_graphs; ++gi) {
            const double b = best_of(gi)->delta;
            for (double d : {b * step, b / step}) {
                bool seen = false;
                for (const Tried &t : tried[gi]) seen = seen || std::fabs(t.delta - d) <= 1e-12 * d;
                if (!seen) todo[gi].push_back(d);
            }
        }
        if ((rc = evaluate()) != DSSSP_OK) return rc;
    }
    for (int32_t gi = 0; gi < n_graphs; ++gi) {
        const Tried *b = best_of(gi);
        delta_out[gi] = b->delta;
        if (ms_out) ms_out[gi] = b->ms;
    }
    return DSSSP_OK;
}

extern "C" dsssp_status dsssp_tune_team_blocks(dsssp_graph *const *graphs, int32_t n_graphs, const double *delta,
                                               int32_t n_inst, const int32_t *src, const int32_t *src_graph,
                                               void *const *dist, int32_t *const *pred, int32_t *team_blocks_out,
                                               double *ms_out, void *stream) {
    if (!team_blocks_out || !graphs || n_graphs < 1) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(graphs[0] ? graphs[0]->device : 0);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DSSSP_TRY(cudaEventCreate(&e0));
    DSSSP_TRY(cudaEventCreate(&e1));
    double best_ms = std::numeric_limits<double>::infinity();
    int32_t best = 0;
    dsssp_status rc = DSSSP_OK;
    for (int32_t tb : {1, 2, 4, 8, 16, -1}) {
        // -1: one instance after another on the whole GPU (tried for a batch on one graph)
        if (tb == -1 && n_graphs != 1) continue;
        dsssp_options o;
        dsssp_options_default(&o);
        o.team_blocks = tb;
        dsssp_batch *b = nullptr;
        rc = dsssp_batch_create(graphs, n_graphs, delta, n_inst, src, src_graph, dist, pred, 0u, &o, stream, &b);
        if (rc == DSSSP_ERR_UNSUPPORTED) {      // this cluster size cannot be co-scheduled here
            rc = DSSSP_OK;
            continue;
        }
        if (rc != DSSSP_OK) break;
        rc = dsssp_batch_run(b, stream);                                  // warm-up
        if (rc == DSSSP_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = DSSSP_ERR_CUDA;
        if (rc == DSSSP_OK) rc = dsssp_batch_run(b, stream);
        if (rc == DSSSP_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = DSSSP_ERR_CUDA;
        if (rc == DSSSP_OK) rc = dsssp_batch_sync(b, nullptr, stream);
        float t = 0.f;
        if (rc == DSSSP_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = DSSSP_ERR_CUDA;
        dsssp_batch_destroy(b);
        if (rc != DSSSP_OK) break;
        if (t < best_ms) {
            best_ms = t;
            best = tb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DSSSP_OK) return rc;
    if (best == 0) return DSSSP_ERR_UNSUPPORTED;
    *team_blocks_out = best;
    if (ms_out) *ms_out = best_ms;
    return DSSSP_OK;
}

extern "C" dsssp_status dsssp_tune_solo_work(dsssp_graph *g, const int32_t *sample_src, int32_t k, double delta,
                                             int32_t *solo_work_out, double *ms_out, void *stream) {
    if (!g || !sample_src || k < 1 || !solo_work_out || !(delta > 0.0)) return DSSSP_ERR_INVALID_ARG;
    for (int32_t j = 0; j < k; ++j)
        if (sample_src[j] < 0 || (int64_t)sample_src[j] >= g->n) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    double best_ms = std::numeric_limits<double>::infinity();
    int32_t best = 0;
    for (int32_t sw : {-1, 512, 2048, 8192, 32768}) {
        double ms = 0.0;
        dsssp_status rc = time_solves(g, sample_src, k, delta, (cudaStream_t)stream, &ms, sw);
        if (rc != DSSSP_OK) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = sw;
        }
    }
    *solo_work_out = best;
    if (ms_out) *ms_out = best_ms;
    return DSSSP_OK;
}

extern "C" dsssp_status dsssp_tune_schedule(dsssp_graph *g, const int32_t *sample_src, int32_t k, double delta,
                                            dsssp_options *opt_out, double *ms_out, void *stream) {
    if (!g || !sample_src || k < 1 || !opt_out || !(delta > 0.0)) return DSSSP_ERR_INVALID_ARG;
    for (int32_t j = 0; j < k; ++j)
        if (sample_src[j] < 0 || (int64_t)sample_src[j] >= g->n) return DSSSP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    double best_ms = std::numeric_limits<double>::infinity();
    dsssp_options best;
    dsssp_options_default(&best);
    // the persistent grid-wide scheme at each solo threshold
    for (int32_t sw : {-1, 512, 2048, 8192, 32768}) {
        dsssp_options o;
        dsssp_options_default(&o);
        o.solo_work = sw;
        double ms = 0.0;
        dsssp_status rc = time_solves_opt(g, sample_src, k, delta, st, &ms, o);
        if (rc != DSSSP_OK) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = o;
        }
    }
    // one thread-block cluster (a batch team) per solve
    for (int32_t tb : {8, 16}) {
        dsssp_options o;
        dsssp_options_default(&o);
        o.mode = DSSSP_MODE_TEAM;
        o.team_blocks = tb;
        double ms = 0.0;
        dsssp_status rc = time_solves_opt(g, sample_src, k, delta, st, &ms, o);
        if (rc == DSSSP_ERR_UNSUPPORTED || rc == DSSSP_ERR_CUDA) {   // this cluster size cannot run here
            cudaGetLastError();
            continue;
        }
        if (rc != DSSSP_OK) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = o;
        }
    }
    *opt_out = best;
    if (ms_out) *ms_out = best_ms;
    return DSSSP_OK;
}
