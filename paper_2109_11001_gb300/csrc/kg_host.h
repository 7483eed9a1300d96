// kg_host.h -- host-side context of the GB300 DBH library (internal).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kg.h"
#include "kg_internal.cuh"

struct kg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    kg_allocator alloc{};
    bool have_alloc = false;

    kg_params p{};
    std::vector<kg_melt> melts;
    int precision = KG_FP64;
    int M = 0, Mp = 0;           // slots, padded slots

    kg::SimDev sim{};            // host copy
    kg::SimDev *d_sim = nullptr;
    kg::StageDev stage{};        // host copy of the stage in force
    kg::StageDev *d_stage = nullptr;

    std::vector<kg_stage> schedule;
    size_t stage_idx = 0;
    long long stage_left = -1;   // < 0: open-ended
    long long step = 0, sweep = 0;
    double t_since_sweep = 0.0;
    std::vector<double> carry;   // fractional DB attempts per melt
    kg_status latched = KG_ERR_STATE;

    // state
    double *x = nullptr;         // [3][Mp]
    void *u = nullptr;           // [3][Mp] float or double
    int *pid = nullptr;
    float4 *recb = nullptr;
    float4 *dlt[2] = {nullptr, nullptr};
    double4_32a *pos64[2] = {nullptr, nullptr};
    double4_32a *xb = nullptr;
    int cur = 0;                 // ping-pong index of the gather buffer in use

    // Verlet list and its cell grid
    int ncell_md = 0;
    int *cellid = nullptr, *rank = nullptr, *ccount = nullptr, *cstart = nullptr, *clist = nullptr;
    int *bsum = nullptr;         // scan block sums (shared by both grids)
    int maxnb = 0;
    int *nl = nullptr, *nn = nullptr;

    // double-bridging
    int ncell_db = 0;
    int *dbcell = nullptr, *dbrank = nullptr, *dbcount = nullptr, *dbstart = nullptr, *dblist = nullptr;
    void *att = nullptr;         // kg::Attempt[att_cap]
    long long att_cap = 0;
    int *koff = nullptr;         // [n_melts+1] attempt offsets
    int *occ = nullptr, *curmap = nullptr, *img = nullptr, *dirty = nullptr;
    long long *db_stats = nullptr;   // [n_melts][4]

    // scratch
    double *scratch = nullptr;   // [3][Mp] doubles + [3][Mp] + [Mp] ints (gather / staging)
    unsigned *flags = nullptr;   // [0] error bits, [1] rebuild request, [3] max list length, [4] blocks done
    double *partials = nullptr;  // block partial sums for observables
    int partials_cap = 0;
    double *r2tmp = nullptr;     // per-chain <R^2(n)> partial sums
    long long r2tmp_cap = 0;
    int *hist = nullptr;         // histogram counts
    int hist_cap = 0;
    double *fout = nullptr;      // forces for kg_forces

    // instrumentation
    long long launches = 0;      // kernels launched since creation
    bool prof_on = false;
    std::vector<cudaEvent_t> ev; // pairs around step-kernel launches
    int ev_used = 0;
    double prof_ms = 0.0;
    long long prof_n = 0;
};

namespace kg {

struct Attempt {
    int flags;                   // 1: non-empty partner set, 2: accepted
    int c, d;                    // chain of the drawn bond, chain of the chosen partner
    int kind, A, B, pA, pB;      // canonical move
    int jp[4];                   // junction particles (-1: unused)
};

// kg_md.cu
void rebuild_md(kg_ctx *c);                  // conditional on flags[1]
void md_step(kg_ctx *c, long long step);     // one fused force + integrate step
void forces_eval(kg_ctx *c, int melt, long long step, double *F_dev, double *part_dev, int nblk);
void prof_collect(kg_ctx *c);                // fold recorded event pairs into the totals
int forces_blocks(const kg_ctx *c, int melt);

// kg_db.cu
void db_sweep(kg_ctx *c, const std::vector<long long> &K, long long *host_stats /*[n_melts][4]*/);

// kg_obs.cu
void r2n_eval(kg_ctx *c, int melt, double *out_dev);
void hist_eval(kg_ctx *c, int melt, int nbins, int *out_dev);

}  // namespace kg
