// Internal view of a suspension handle, shared by the translation units of
// libdbs (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dbs.h"
#include "dbs_common.cuh"

struct dbs_ensemble;

struct dbs_suspension {
    dbs_ensemble *solo = nullptr;  // private one-member ensemble of the cluster path
    int path = 0;                  // DBS_PATH_GRID / DBS_PATH_CLUSTER / DBS_PATH_COOP
    double noise_sigma = 0.0;      // additive noise per step (dbs_set_noise); 0 = off
    unsigned long long noise_seed = 0;
    int dyn = 0;                   // DBS_DYN_SPRING / DBS_DYN_SHAPE (dbs_set_dynamics)
    int sd_iters = 1;              // shape-driven: constraint iterations per evaluation
    double *sd_buf = nullptr;      // shape-driven work arrays (see dbs_shape.cu)
    // cooperative dataflow path: tagged record buffer, split, next tag
    ulonglong2 *ll_rec = nullptr;
    int flow_T = 0, flow_G = 0;    // dumbbells per CTA, CTAs
    int flow_creq = 0;             // dbs_set_chunks request (dumbbells per CTA), 0 = built-in
    unsigned flow_base = 1;
    int flow_test_dG = 0;          // diagnostic: the kernel is told G + this many CTAs (0 = the true grid)
    dbs_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t S = 0, N = 0;
    int64_t n_host = 0;
    int status = DBS_OK;
    char msg[256] = "";
    // device state
    double *x = nullptr, *v0 = nullptr, *Fd = nullptr, *Fext = nullptr, *lam = nullptr,
           *sinphi = nullptr, *cosphi = nullptr, *vout = nullptr, *Ftmp = nullptr;
    void *packA = nullptr, *packB = nullptr, *packT = nullptr;
    double2 *trig = nullptr;
    float4 *trig_df = nullptr;
    int64_t trig_hi = -1;  // ring holds (sin, cos)(omega t_k) for k <= trig_hi (last TRIG_RING/2 fills)
    float *part = nullptr;
    unsigned *tickets = nullptr, *done = nullptr;
    int64_t *step = nullptr;
    int *flags = nullptr;
    double *Racc = nullptr, *Rbar = nullptr;
    int64_t avg_m = 0, avg_n0 = 0, avg_maxk = 0;
    double cx = 0, cy = 0, cz = 0;
    double lam_max = 0;
    // launch configuration
    int grid = 1, chunks = 1, bt = 128, sms = 148;
    // row sharding (dbs_shard_set): the i-blocks [shard_ib0, shard_ib0 + shard_nib)
    // this handle computes, and their grid; shard_nib = 0: not sharded
    int shard_ib0 = 0, shard_nib = 0, shard_grid = 0;
    // captured block of GRAPH_STEPS Heun steps
    cudaGraphExec_t graph = nullptr;
};


// helpers defined in dbs_suspension.cu
int fail(dbs_suspension *h, int status, const char *fmt, ...);
int refuse(dbs_suspension *h, int status, const char *msg);  // no sticky status
dbs::EvalArgs base_args(const dbs_suspension *h);
int ensure_trig(dbs_suspension *h, int64_t k_hi, cudaStream_t st = nullptr);  // st: h->stream if null
int check_flags(dbs_suspension *h);
void drop_graph(dbs_suspension *h);
// defined in dbs_suspension.cu (cooperative path)
int coop_setup(dbs_suspension *h);
// defined in dbs_suspension.cu: one APPLY evaluation of the pair-sum kernel with A
void launch_apply(const dbs_suspension *h, const dbs::EvalArgs &A);
// defined in dbs_shape.cu (shape-driven dynamics)
int shape_step(dbs_suspension *h, int64_t n);
int shape_finish(dbs_suspension *h);
int shape_reset(dbs_suspension *h);
void shape_free(dbs_suspension *h);
// defined in dbs_suspension.cu: spring records and forces of the current state into packA / Fd
int spring_repack(dbs_suspension *h);
// defined in dbs_ensemble.cu
int solo_step(dbs_suspension *h, int64_t n);
bool ens_member_ok(const dbs_suspension *h);               // can run on the cluster path
int ens_create(int32_t count, dbs_suspension *const *members, void *stream, dbs_ensemble **out);
int ens_step_v(dbs_ensemble *e, const int64_t *steps);     // member i advances steps[i]
void ens_destroy(dbs_ensemble *e);
const char *ens_error(const dbs_ensemble *e);
constexpr int kTrigRing = 4096;  // entries of the per-handle clock ring
void solo_destroy(dbs_suspension *h);
