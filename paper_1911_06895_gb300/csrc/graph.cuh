// graph.cuh -- the graph handle and its per-Delta split cache, shared by the
// host code of the single-solve API (api.cu) and of batches (batch.cu).
// Not part of the public ABI.
#pragma once

#include "dense.cuh"
#include "dsssp_internal.cuh"

namespace dsssp {

constexpr int kSplitCache = 4;

// One light/heavy layout of the graph's arcs for one Delta (Section III-A).
struct Split {
    double delta = 0.0;
    bool valid = false;
    int pins = 0;               // live batches using this split: never evicted while > 0
    uint64_t last_use = 0;
    uint2 *arcs = nullptr;      // m
    uint4 *vinfo = nullptr;     // n
    uint32_t *perm = nullptr;   // m: split position -> input arc index
};

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

dsssp_status cuda_status(cudaError_t e);

// The split for `delta`, built on `st` when not cached (least recently used
// unpinned split evicted; UNSUPPORTED when all are pinned).
dsssp_status ensure_split(dsssp_graph *g, double delta, cudaStream_t st, Split **out);

// A single solve as one instance of the batch kernel on one thread-block cluster
// of team_blocks blocks (DSSSP_MODE_TEAM), on the handle's workspace and region
// (batch.cu). team_err / team_stats point into the region.
size_t team_region_bytes();
cudaError_t team_solve_launch(dsssp_graph *g, const Split *sp, int32_t src, double delta, void *dist,
                              int32_t *pred, int team_blocks, int64_t max_phases, cudaStream_t st);
int *team_err(dsssp_graph *g);
long long *team_stats(dsssp_graph *g);
void team_stats_to_solve(const long long *st, dsssp_stats *out);
constexpr int kTeamStatsCount = 16;

#define DSSSP_TRY(expr)                                      \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            cudaGetLastError();                              \
            return ::dsssp::cuda_status(_e);                 \
        }                                                    \
    } while (0)

}  // namespace dsssp

struct dsssp_graph {
    int64_t n = 0, m = 0;
    int dtype = 0;
    int device = 0;
    int sm_count = 0;
    uint32_t *off = nullptr;      // n+1
    int32_t *col = nullptr;       // m
    uint32_t *wbits = nullptr;    // m
    dsssp::Split splits[dsssp::kSplitCache];
    uint64_t use_clock = 0;
    // solver workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    dsssp::SolveArgs args{};
    dsssp::Ctl *ctl = nullptr;           // device
    dsssp::NaCtl *nactl = nullptr;       // device: control words of DSSSP_MODE_DENSE solves
    void *team_region = nullptr;         // device: tables and counters of DSSSP_MODE_TEAM solves
    dsssp::Ctl *ctl_host = nullptr;      // pinned host mirror
    int32_t *sticky = nullptr;    // device: first error of asynchronous solves
    int occ_block = 0, occ_blocks_per_sm = 0;
};
