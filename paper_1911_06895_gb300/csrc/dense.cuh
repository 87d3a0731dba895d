// dense.cuh -- the full-vector form of delta-stepping (noalloc.cu): working
// memory and the internal entry used by dsssp_solve's DSSSP_MODE_DENSE.
// Not part of the public ABI.
#pragma once

#include "dsssp_internal.cuh"

namespace dsssp {

// Control words of one dense solve.
struct NaCtl {
    unsigned int bar_count;
    unsigned int bar_gen;
    int32_t err;              // first dsssp_status != OK
    int32_t flags;            // input validation: bit 0 malformed CSR, bit 1 bad weight
    uint32_t mode;            // 0 light round, 1 heavy pass, 2 next-bucket search, 3 done
    uint32_t round;           // frontier stamp of the current light round
    uint32_t epoch;           // S stamp of the current bucket
    uint32_t T;               // key < T  <=>  bucket <= i
    uint32_t next_count;      // vertices stamped for the next light round
    uint32_t far_min;         // lower bound on the keys of far (later-bucket) vertices
    uint32_t far_count;       // vertices on the far pile
    uint32_t ovf;             // 1: a relaxation met a sum the weight type cannot hold
    long long phases;
    unsigned long long progress;   // bumped as rows are scanned: a waiting block's clock restarts on it
    long long n_light, n_heavy, n_select, buckets;   // phase counts by kind
};

// Working memory: n entries per vector, one NaCtl.
struct NaMem {
    unsigned long long *packed;   // key << 32 | pred (the vector t)
    uint32_t *fstamp;             // t_Bi: in the light round with this stamp
    uint32_t *sstamp;             // S: member in the bucket with this stamp
    uint32_t *far;                // 1: a later bucket holds an unprocessed key
    NaCtl *ctl;
};

// DSSSP_MODE_DENSE on a graph handle's CSR (off u32[n+1], col, weight bits):
// init, the cooperative solve, the overflow check and the unpack, enqueued on st.
// The status stays in mem.ctl->err (read it with dense_status).
cudaError_t dense_solve_launch(const uint32_t *off, const int32_t *col, const uint32_t *wbits, int dtype,
                               uint32_t n, uint32_t m, uint32_t src, double delta, const NaMem &mem, void *dist,
                               int32_t *pred, int64_t timeout_ns, int64_t max_phases, cudaStream_t st);

}  // namespace dsssp
