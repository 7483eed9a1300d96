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
    double *x = nullptr;         // [3][Mp]; mixed: current only outside kg_step (see xb64)
    double *xb64 = nullptr;      // mixed: binary64 positions at the last Verlet build [3][Mp];
                                 // the current position is xb64 + dlt[cur] (folded at every
                                 // build and at the end of every kg_step call)
    void *u = nullptr;           // [3][Mp] float or double
    int *pid = nullptr;          // particle id of the monomer at each compute index
    int *slot_of = nullptr;      // compute index -> chain-major slot
    int *comp_of = nullptr;      // chain-major slot -> compute index
    int4 *bp = nullptr;          // compute indices of slots s-2, s-1, s+1, s+2 (-1 past a chain end)
    bool clist_valid = false;    // the last Verlet build's cell order can seed a re-sort
    bool sort_after_load = false;  // re-sort after the first build that follows a load
    long long since_sort = 0;
    long long *d_step = nullptr;   // device step counter (index of the step being run)
    bool d_step_stale = true;      // host must write it before the next step
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool graph_failed = false;
    cudaGraphExec_t pexec[2] = {nullptr, nullptr};   // persistent launches (KG_FLAG_PERSISTENT)
    bool persist_failed = false;
    unsigned *pbar = nullptr;    // grid-barrier words of the persistent launch
    bool use_graphs = true;
    long long graph_replays = 0;
    long long sort_interval = 200;
    int block = 128;             // threads per block of the fused step kernel
    int tpm = 1;                 // threads per monomer of the mixed step kernel (1 or 2)
    float4 *recb = nullptr;      // build records: offset from the Verlet-cell corner, cell coordinates
    float4 *recs = nullptr;      // the same in cell order (Verlet-list build)
    float4 *dlt[2] = {nullptr, nullptr};   // (mixed) displacement since the build
    float4 *pg[2] = {nullptr, nullptr};    // (mixed) gather records recb + dlt
    float4 *shtab = nullptr;     // image shift of each stencil code, SHIFT_SLOTS per melt
    double4_32a *pos64[2] = {nullptr, nullptr};
    double4_32a *xb = nullptr;
    int cur = 0;                 // ping-pong index of the gather buffer in use

    // Verlet list and its cell grid
    int ncell_md = 0;
    int *cellid = nullptr, *rank = nullptr, *ccount = nullptr, *cstart = nullptr, *clist = nullptr;
    int *ctmp = nullptr;         // cell-ordered list before the in-cell ranking
    int *bsum = nullptr;         // scan block sums (shared by both grids)
    int maxnb = 0;
    unsigned *nl = nullptr;      // entries j | stencil code << IDX_BITS
    int *nn = nullptr;

    // double-bridging
    int ncell_db = 0;
    int *dbcell = nullptr, *dbrank = nullptr, *dbcount = nullptr, *dbstart = nullptr, *dblist = nullptr;
    float4 *dbrec = nullptr;     // binary32 records on the DB grid (swap-bond prefilter)
    int *dbmark = nullptr;       // per DB cell: number of the last commit of the sweep near it (-1: none)
    int *chain_ver = nullptr;    // per chain: number of the last commit of the sweep that touched it
    int n_chain_total = 0;
    int *dbround = nullptr;      // per melt: position, commits, finished, re-evaluations
    int *att_ver = nullptr;      // per attempt: commits seen by its record
    void *att = nullptr;         // kg::Attempt[att_cap]
    long long att_cap = 0;
    int *koff = nullptr;         // [n_melts+1] attempt offsets
    int *img = nullptr;
    long long *db_stats = nullptr;   // [n_melts][4]

    // learned proposal (kg_mlp.cu, kg_learned.cu)
    float *mlp_master = nullptr;         // binary32 master weights [KG_MLP_NPARAM]
    float *mlp_adam = nullptr;           // Adam moments m, v [2][KG_MLP_NPARAM]
    float *mlp_grad = nullptr;           // gradient + loss [KG_MLP_NPARAM + 1]
    void *mlp_blob = nullptr;            // bf16 image (kg::MlpSmem) for the tensor cores
    void *mlp_w2t = nullptr;             // bf16 W2 transposed, [64][72] (backward)
    long long adam_t = 0;                // Adam steps taken
    long long train_iter = 0;            // minibatches drawn
    double *logf = nullptr, *logt = nullptr;   // per-attempt staging of the sweep log
    int *logn = nullptr;
    long long log_att_cap = 0;
    double *trainf = nullptr, *traint = nullptr;  // training ring [train_cap][24], [train_cap]
    long long train_cap = 0;
    long long *d_train_head = nullptr;   // rows ever appended
    void *tr_buf = nullptr;              // minibatch work arrays
    long long tr_rows = 0;
    unsigned long long *bmax2 = nullptr; // longest bond squared (binary64 bits), per learned sweep
    double *d_io = nullptr;              // device staging for host-pointer calls
    long long d_io_cap = 0;

    // scratch
    double *scratch = nullptr;   // [3][Mp] doubles + [3][Mp] + [Mp] ints (gather / staging)
    unsigned *flags = nullptr;   // [0] error bits, [1] rebuild request, [3] max list length, [4] blocks done,
                                 // [5] Verlet builds, [6] rebuild bodies run inside graphs
    double *partials = nullptr;  // block partial sums for observables
    int partials_cap = 0;
    double *r2tmp = nullptr;     // per-chain <R^2(n)> partial sums
    long long r2tmp_cap = 0;
    int *hist = nullptr;         // histogram counts
    int hist_cap = 0;
    double *fout = nullptr;      // forces for kg_forces
    double *msd_ref = nullptr;   // [3][Mp] reference positions of kg_msd (+ [3][Mp] re-sort scratch)

    // instrumentation
    long long launches = 0;      // kernels launched since creation
    bool prof_on = false;
    std::vector<cudaEvent_t> ev; // pairs around step-kernel launches
    int ev_used = 0;
    double prof_ms = 0.0;
    long long prof_n = 0;
};

namespace kg {

// device memory through the context's allocator (zero-filled on the context's stream)
void *dev_alloc(kg_ctx *c, size_t bytes);
void dev_free(kg_ctx *c, void *p);

constexpr int GRAPH_STEPS = 10;          // MD steps per captured graph (even)
constexpr int PERSIST_STEPS = 50;        // MD steps per persistent launch (even)
constexpr unsigned PERSIST_SPIN = 1u << 24;   // grid-barrier polls (~64 ns apart) before ERR_TIMEOUT
constexpr int RS = 8;                    // ints per melt in the DB commit-round array

struct Attempt {
    int flags;                   // 1: non-empty partner set, 2: accepted
    int c, d;                    // chain of the drawn bond, chain of the chosen partner
    int kind, A, B, pA, pB;      // canonical move
    int jp[4];                   // junction particles (-1: unused)
};

// kg_md.cu
void rebuild_md(kg_ctx *c);                  // conditional on flags[1]
void md_step(kg_ctx *c);                     // one fused force + integrate step (direct launches)
bool md_graph_steps(kg_ctx *c, long long nrep);  // nrep replays of a GRAPH_STEPS-step graph
void set_device_step(kg_ctx *c, long long v);
void forces_eval(kg_ctx *c, int melt, long long step, double *F_dev, double *part_dev, int nblk);
void prof_collect(kg_ctx *c);                // fold recorded event pairs into the totals
void bonded_partners(kg_ctx *c);             // bp from slot_of / comp_of
void md_sort(kg_ctx *c);                     // re-sort the state into the last cell order
void md_materialize(kg_ctx *c);              // mixed: x <- xb64 + dlt[cur]
void graphs_reset(kg_ctx *c);                // drop captured step graphs (their arguments changed)
bool md_persist_steps(kg_ctx *c);            // PERSIST_STEPS steps in one persistent launch (KG_MIXED)

// kg_step.cu
void step_mixed_launch(kg_ctx *c, cudaStream_t st, int cur);   // the mixed path's fused step kernel
// K steps of every melt in one cooperative launch; skip_block >= 0 makes that
// block skip the barriers (self-test of the bounded waits)
cudaError_t persist_launch(kg_ctx *c, cudaStream_t st, int cur, int K, int skip_block, unsigned spin);
void to_slots(kg_ctx *c, int melt, const double *in_comp, double *out_dev, int dims);
void u_to_slots(kg_ctx *c, int melt, double *out_dev);
void pid_to_slots(kg_ctx *c, int melt, int *out_dev);
int forces_blocks(const kg_ctx *c, int melt);

// kg_db.cu
void db_sweep(kg_ctx *c, const std::vector<long long> &K, long long *host_stats /*[n_melts][4]*/);
void db_bin(kg_ctx *c, const std::vector<long long> &K);     // attempt offsets + the >= 1.3 sigma grid
void db_finish(kg_ctx *c, long long *host_stats);             // box shifts, chain partners, stats to host
int db_max_chain_len(const kg_ctx *c);
// reset the commit bookkeeping of a sweep (versions, stamps, rounds)
void db_rounds_reset(kg_ctx *c, long long tot);


// kg_learned.cu
void db_sweep_learned(kg_ctx *c, const std::vector<long long> &K, double lambda, long long *host_stats);
bool db_proposal(kg_ctx *c, int melt, int chain, int bond, double lambda, int *h_n, int *h_ints /*[3][48]*/,
                 double *h_f /*[48][24]*/, double *h_s /*[48]*/, double *h_pi /*[48]*/);

// kg_mlp.cu
bool mlp_ensure(kg_ctx *c);                                  // allocate; zero weights on first use
void mlp_set(kg_ctx *c, const double *w_dev);                // FP64 device vector -> master + bf16 image
void mlp_get(kg_ctx *c, double *w_dev);                      // master -> FP64 device vector
void mlp_infer(kg_ctx *c, const double *f_dev, long long n, double *s_dev);
bool mlp_grad(kg_ctx *c, const double *f_dev, const double *t_dev, long long n, double *loss_grad_dev);
bool mlp_train(kg_ctx *c, int iters, int batch, double lr, double *loss_dev);

// kg_obs.cu
constexpr int R2N_SMEM_MAX = 24 * KG_R2N_MAX_CHAIN_LEN;     // bytes of k_r2n_chain's positions
bool r2n_smem_ready(int N);                                   // opt-in shared memory; false if N is too long
bool r2n_eval(kg_ctx *c, int melt, double *out_dev);          // false: launch failed or N too long
void hist_eval(kg_ctx *c, int melt, int nbins, int *out_dev);
bool msd_reset(kg_ctx *c, int melt);                          // allocates the reference on first use
int msd_blocks(const kg_ctx *c, int melt);
void msd_eval(kg_ctx *c, int melt, double *part_dev);         // block partial sums of |x - ref|^2
void msd_permute(kg_ctx *c, const int *order);                // re-sort (no-op before the first reset)
void sq_eval(kg_ctx *c, int melt, const int *hkl_dev, int nq, double *part_dev /*[nq][64][2]*/, double *S_dev);
void gr_eval(kg_ctx *c, int melt, int R, double r_max, double dr, int nbins, unsigned long long *hist_dev);
constexpr int GR_BINS_MAX = 2048;

}  // namespace kg
