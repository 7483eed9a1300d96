/*
 * kg.h -- C ABI of the GB300 (sm_103a) library for the core-softened
 * double-bridging hybrid (DBH) equilibration of semiflexible Kremer-Grest
 * melts, after Dietz & Hoy, arXiv:2109.11001.
 *
 * The calls follow the paper's statement of the problem:
 *   - a melt of N_ch chains of N monomers in a cubic periodic cell at density
 *     rho, temperature T and bending stiffness kappa (Sec. II.B);
 *   - a sequence of stages (n, duration) of the core-softened pair potential
 *     U_MLJ^n (Eq. 6) with the FENE constant k_n tied to n (Eq. 9), stepped
 *     through the exponent set Xi (Eq. 11) by the schemes of Eqs. 19-20;
 *   - molecular dynamics at time step dt with double-bridging (DB) Monte Carlo
 *     swaps attempted at R_MC = 1e-3 N_ch N / tau under criteria (i) and (ii)
 *     (Sec. II.B, Fig. 1);
 *   - outputs <R^2(n)> (input to the l_K fit of Eq. 14), energies, swap counts.
 *
 * Conventions (all calls):
 *   - Every call returns a kg_status; KG_OK is 0.  kg_strerror() names it.
 *   - Storage is chain-major: slot s = c*N + i of a melt holds monomer i of
 *     chain c; bonds join slots s and s+1 of one chain.  Topology is the slot
 *     order, so no bond arrays cross the ABI.
 *   - Position arrays are (3, M) float64 structure-of-arrays, unwrapped:
 *     x[0..M) = x, x[M..2M) = y, x[2M..3M) = z.  Velocities likewise.
 *   - Pointers passed to kg_load_config / kg_get_config / kg_observables /
 *     kg_get_nlist / kg_forces may be host or device memory (CUDA unified
 *     addressing decides); inputs are copied, the caller keeps ownership.
 *   - The context owns its device memory; all GPU work is enqueued on the
 *     context's stream.  kg_step and kg_db_sweep are asynchronous except for
 *     one status read at their end; device-side errors (overstretched bond,
 *     non-finite value, capacity) are latched and reported by that read.
 *   - After an error the context refuses work (KG_ERR_STATE) until the next
 *     kg_load_config.
 *   - One context per host thread at a time.
 */
#ifndef KG_H
#define KG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kg_ctx kg_ctx;

typedef enum {
    KG_OK = 0,
    KG_ERR_INVALID_ARG = 1,      /* a size, pointer or parameter out of range          */
    KG_ERR_CUDA = 2,             /* a CUDA runtime call failed                          */
    KG_ERR_OOM = 3,              /* device allocation failed                            */
    KG_ERR_BOND_OVERSTRETCH = 4, /* a bond reached r >= R0, where FENE is undefined     */
    KG_ERR_NONFINITE = 5,        /* a force, velocity or position became non-finite     */
    KG_ERR_CAPACITY = 6,         /* neighbour or candidate storage overflowed           */
    KG_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up                  */
    KG_ERR_STATE = 8             /* context holds a latched error or no configuration   */
} kg_status;

/* arithmetic of the MD force path */
enum {
    KG_FP64 = 0,   /* every force term in binary64                                     */
    KG_MIXED = 1   /* pair/bond/angle forces in binary32 from binary64 positions;
                      between Verlet builds a step advances a binary32 displacement,
                      folded into the binary64 positions at each build and at the end
                      of each kg_step; DB energy changes and energy sums binary64      */
};

/* kg_params.flags */
enum {
    KG_FLAG_PAPER_METROPOLIS = 1, /* accept DB swaps with exp(-dE/T) alone (Fig. 1),
                                      without the proposal ratio                      */
    KG_FLAG_PERSISTENT = 2        /* KG_MIXED (ignored with KG_FP64): kg_step advances
                                      every melt in persistent cooperative launches of
                                      50 steps, each held in a captured CUDA graph; the
                                      Verlet rebuild runs inside the launch between grid
                                      barriers, and every barrier wait is bounded (a
                                      block that gives up latches KG_ERR_TIMEOUT).  One
                                      thread per monomer; results equal the default
                                      path's up to binary32 summation order            */
};

/* One melt (Sec. II.B): N_ch chains of N monomers in a cube of side L. */
typedef struct {
    int n_chains;    /* N_ch >= 1                                                      */
    int chain_len;   /* N >= 3                                                          */
    double box;      /* L = (N_ch N / rho)^(1/3); must exceed 7 sigma                   */
    double kappa;    /* bending stiffness of U_ang = kappa (1 - cos theta), Eq. 4       */
} kg_melt;

/* Run parameters.  Several melts of uneven size may share one context; they
 * are independent systems advanced by the same launches. */
typedef struct {
    int n_melts;              /* 1 ... 64                                               */
    const kg_melt *melts;     /* n_melts entries, copied                               */
    double T;                 /* temperature (1, Sec. II.B)                             */
    double gamma;             /* Langevin friction (paper silent; 1)                   */
    double R0;                /* FENE extent, 1.5 (Eq. 3)                               */
    double l0;                /* bond length kept by k_n, 0.960897 (Eq. 7)              */
    double db_bond_max;       /* longest new bond of a DB swap, 1.3 (Sec. II.B (ii))    */
    double r_mc;              /* DB attempts per monomer per tau, 1e-3 (Sec. II.B)      */
    double skin;              /* neighbour-list skin (0.3 when <= 0)                    */
    double fene_qmin;         /* 0: FENE exactly as Eq. 3, r >= R0 is an error;
                                 q in (0, 0.25): the FENE log term is continued beyond
                                 r* = R0 sqrt(1 - q) by the quadratic in r^2 that
                                 matches its value and slope there (finite past R0;
                                 r >= 2 R0 is still an error)                          */
    unsigned long long seed;  /* key of every counter-based random draw                */
    int sort_interval;        /* MD steps between re-sorts of the per-monomer arrays into
                                 cell order (<= 0: 200), tested at the start of each
                                 kg_step call and each 10-step graph; KG_FP64 results do
                                 not depend on it; in KG_MIXED a re-sort forces a Verlet
                                 build, whose timing moves positions at the binary32
                                 rounding level (~1e-7 sigma)                           */
    int block_size;           /* threads per block of the fused step kernel: 64, 128
                                 or 256 (<= 0: 128); results do not depend on it        */
    int precision;            /* KG_FP64 or KG_MIXED                                    */
    int flags;                /* KG_FLAG_*                                              */
    int threads_per_monomer;  /* threads sharing one monomer's step in KG_MIXED: 1 or 2
                                 (<= 0: 1; KG_FP64 always uses 1); results do not
                                 depend on it beyond binary32 summation order           */
    double cell_scale;        /* Verlet-list cells of side >= cell_scale (r_c + skin),
                                 1 ... 3 (<= 0: 1): larger cells mean fewer cells to
                                 bin and sort and more candidates per monomer; lists
                                 and results do not depend on it                        */
} kg_params;

/* One stage of the potential schedule (Eqs. 6, 9, 10, 19-20). */
typedef struct {
    double n_exp;       /* exponent n of U_MLJ^n; n != 6; Xi = {2,...,12} (Eq. 11)      */
    double k_fene;      /* FENE constant; < 0 selects k_n of Eq. 9                      */
    long long n_steps;  /* MD steps spent in the stage                                 */
    double dt;          /* time step of the stage (a dt ramp is a run of stages)      */
} kg_stage;

/* Integer-time observables of one melt (FP64 sums). */
typedef struct {
    double e_pair, e_bond, e_angle, e_kin, virial, temperature, pressure;
    long long step;
} kg_obs;

/* Double-bridging sweep statistics (summed over melts). */
typedef struct {
    long long attempted;    /* attempts drawn                                          */
    long long empty;        /* attempts whose drawn bond had no admissible partner     */
    long long accepted;     /* swaps applied                                           */
    long long reevaluated;  /* re-evaluations of attempts made stale by earlier swaps   */
    long long sweep;        /* index of the sweep just run                             */
} kg_db_stats;

/* Optional device allocator (e.g. a framework's caching allocator).  NULL
 * selects cudaMalloc / cudaFree.  alloc returns NULL on failure. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} kg_allocator;

/* Create a context on `device`, enqueueing on `stream` (a cudaStream_t; NULL
 * selects a new non-blocking stream owned by the context).  Validates p,
 * allocates every device buffer.  The default stage is n = 12 (WCA), k_12,
 * dt = 0.01 until kg_set_potential_schedule is called. */
kg_status kg_create(kg_ctx **out, const kg_params *p, int device, void *stream,
                    const kg_allocator *allocator);

/* Load melt `melt`'s state: x (3, M) unwrapped positions, v (3, M) velocities
 * (NULL: zero), pid (M) particle ids carried through DB swaps (NULL: 0..M-1).
 * The velocity is the state velocity u = v_{n-1/2} of the leapfrog form of
 * velocity Verlet.  Clears a latched error; forces a neighbour-list rebuild.
 * The loaded melt is held in chain order until the first kg_step, which runs
 * its first MD step alone and then re-sorts the state into that step's cell
 * order (gathers stay local from the second step on). */
kg_status kg_load_config(kg_ctx *c, int melt, const double *x, const double *v, const int *pid);

/* Copy melt `melt`'s state out (any pointer may be NULL). */
kg_status kg_get_config(kg_ctx *c, int melt, double *x, double *v, int *pid);

/* Self-test of the persistent launch's bounded barrier waits (KG_MIXED
 * contexts): one persistent launch of two MD steps in which block skip_block
 * (>= 0) never arrives at the grid barrier, so the other blocks give up after
 * `spin` polls (about 64 ns apart), latch KG_ERR_TIMEOUT and return; the call
 * returns that status and the context holds it until the next kg_load_config.
 * With skip_block < 0 it is an ordinary two-step persistent launch (KG_OK).
 * No block waits longer than `spin` polls per barrier. */
kg_status kg_persistent_selftest(kg_ctx *c, int skip_block, unsigned spin);

/* Replace the potential schedule by n_stages stages (copied).  Kernels read
 * the stage parameters from device memory, so a stage change costs one small
 * copy.  After the last stage its parameters stay in force. */
kg_status kg_set_potential_schedule(kg_ctx *c, const kg_stage *stages, int n_stages);

/* Advance every melt by n_steps MD steps: Verlet-list maintenance, U_MLJ^n
 * pairs, U_bond^n bonds (Eq. 10), bending (Eq. 4), Langevin velocity Verlet
 * with Philox4x32-10 noise keyed by (seed, step, slot, melt). */
kg_status kg_step(kg_ctx *c, long long n_steps);

/* One DB sweep per melt.  attempts_per_monomer >= 0: floor(a M + carry)
 * attempts per melt; < 0: the paper's rate R_MC times the MD time elapsed since
 * the previous sweep (Sec. II.B).  Attempts are processed with the semantics
 * of a strictly sequential loop (an attempt sees every swap accepted before
 * it).  stats may be NULL. */
kg_status kg_db_sweep(kg_ctx *c, double attempts_per_monomer, kg_db_stats *stats);

/* As kg_db_sweep with an explicit attempt count per melt (n_melts entries). */
kg_status kg_db_sweep_k(kg_ctx *c, const long long *attempts, kg_db_stats *stats);

/* Longest chain whose <R^2(n)> can be computed (kg_observables, kg_r2n_noalloc):
 * one chain's 3N binary64 positions must fit one block's shared memory. */
#define KG_R2N_MAX_CHAIN_LEN 9685

/* Observables of melt `melt` at the current integer time step (synchronises):
 * energies and virial from the conservative forces, kinetic energy from
 * v_n = u + dt/2 F_n, <R^2(n)> for n = 0..N-1 into r2n (N doubles; NULL to
 * skip; KG_ERR_INVALID_ARG when N > KG_R2N_MAX_CHAIN_LEN), and bond-length
 * (on [0, R0)) / cos(theta) (on [-1, 1]) histograms of n_bins bins (NULL to
 * skip). */
kg_status kg_observables(kg_ctx *c, int melt, kg_obs *out, double *r2n,
                         double *bond_hist, double *cos_hist, int n_bins);

/* Wait for the context's stream; returns the latched device status. */
kg_status kg_sync(kg_ctx *c);

/* Counters: MD step index and DB sweep index (they key the random draws). */
kg_status kg_get_counters(kg_ctx *c, long long *step, long long *sweep);
kg_status kg_set_counters(kg_ctx *c, long long step, long long sweep);

/* Verlet list of melt `melt` built now from the current positions with cutoff
 * r_c + skin: CSR offs (M+1) and nbr (melt-local slots, ascending per row,
 * at most cap entries); *total receives the pair count.  1-2 bonded pairs are
 * excluded; the distance test is r^2 < (r_c + skin)^2 in binary64. */
kg_status kg_get_nlist(kg_ctx *c, int melt, int *offs, int *nbr, long long cap, long long *total);

/* Conservative forces (3, M) of melt `melt` at the current positions, in the
 * context's precision, and e4 = [pair, bond, angle, virial] energies (either
 * pointer may be NULL). */
kg_status kg_forces(kg_ctx *c, int melt, double *F, double *e4);

/* Timing of the fused MD step kernel with CUDA events on the context's
 * stream.  kg_profile(c, 1) starts recording an event pair around every
 * step-kernel launch (and resets the totals); kg_profile(c, 0) stops.
 * kg_profile_read synchronises and returns the summed step-kernel time (ms),
 * its launch count, and the number of kernels the library has launched since
 * kg_create (every kernel, whether or not profiling is on). */
kg_status kg_profile(kg_ctx *c, int enable);
kg_status kg_profile_read(kg_ctx *c, double *step_kernel_ms, long long *step_kernel_launches,
                          long long *kernel_launches);

/* Launch settings picked by kg_autotune. */
typedef struct {
    double skin;          /* Verlet skin (also sets the cell size, >= r_c + skin)      */
    int block_size;       /* threads per block of the fused step kernel                */
    double ms_per_step;   /* measured wall time of one MD step with these settings     */
    int trials;           /* configurations timed                                       */
    int threads_per_monomer;  /* 1 or 2 (KG_MIXED; always 1 for KG_FP64)                */
    double cell_scale;    /* Verlet cell side over (r_c + skin)                          */
} kg_tuning;

/* Autotuner: for the melts of *p in the states x[m], v[m] ((3, M_m) arrays,
 * host or device; v may be NULL) under `stage`, time the better of two
 * windows of trial_steps MD steps (graph-captured, re-sorts off, after one
 * Verlet build, a re-sort into its cell order and a warm-up of trial_steps
 * steps: the layout a long run keeps) for every candidate
 * skin in {0.25, 0.3, 0.4, 0.5, 0.6}, block size in {64, 128, 256} and, for
 * KG_MIXED, threads per monomer in {1, 2}, each in a scratch context of its
 * own, then the cell side (cell_scale 1.15 and 1.3 of r_c + skin) with the
 * best of those; return the fastest in *best (a later candidate must be
 * faster by 0.5% to replace an earlier one, so near-ties keep the smaller
 * skin, block and cell).  The settings do
 * not change results beyond floating-point summation order.  Synchronises. */
kg_status kg_autotune(const kg_params *p, const double *const *x, const double *const *v,
                      const kg_stage *stage, int trial_steps, int device, void *stream,
                      const kg_allocator *allocator, kg_tuning *best);

/* ---- Learned double-bridging proposal (an extension; the paper draws the
 * swap partner uniformly, Fig. 1) ----
 * A network of 24 move features -> 64 (ReLU) -> 64 (ReLU) -> 1 logit scores
 * each admissible swap of the drawn bond; the partner is drawn from
 *     pi_j = (1 - lambda) softmax_j(logits) + lambda / |P(b)|
 * over the bond's partner list (in the list order of Fig. 1's proposal), and
 * the swap is accepted with min(1, exp(-dE/T) q(x'->x) / q(x->x')), q summing
 * the two ways a swap can be proposed (either removed bond drawn).  Any
 * lambda in (0, 1] leaves the Boltzmann distribution of Sec. II.B stationary;
 * lambda = 1 is the uniform proposal.  The network runs on bf16 tensor cores
 * with fp32 accumulation; features, probabilities and the acceptance test are
 * binary64.  A context starts with zero weights (the uniform proposal).
 *
 * Weights: KG_MLP_NPARAM binary64 values packed as W1[64][24], b1[64],
 * W2[64][64], b2[64], w3[64], b3 (row = output unit); stored as binary32.
 * Features of one swap (u-w the drawn bond, X-Y the partner bond, new bonds
 * u-X and Y-w): 0-1 removed bond lengths (sorted), 2-3 new bond lengths
 * (sorted), 4 change of the FENE terms, 5 change of the bending energy, 6-9
 * cos at the four junction vertices before (sorted), 10-13 after, 14-17 cos
 * one vertex further out (sorted), 18 cos between u->w and X->Y, 19 kappa/4,
 * 20 n/12, 21 min(p+1, N-1-p)/N for the drawn bond p, 22 dE = [4] + [5], 23 1.
 * Host pointers below are host memory; sizes are counts of rows. */
#define KG_MLP_NPARAM 5825
#define KG_DB_CAND_MAX 48   /* candidates one bond may have; more is KG_ERR_CAPACITY */

kg_status kg_mlp_set_weights(kg_ctx *c, const double *w);   /* host, KG_MLP_NPARAM; resets Adam */
kg_status kg_mlp_get_weights(kg_ctx *c, double *w);         /* host, KG_MLP_NPARAM (synchronises) */

/* Logits of n feature rows (host, n x 24 -> n); synchronises. */
kg_status kg_mlp_forward(kg_ctx *c, const double *features, long long n, double *logits);

/* Mean binary cross-entropy of sigmoid(logit) against targets t in [0, 1]
 * over n rows (host arrays), and its gradient with respect to the packed
 * weights (host, KG_MLP_NPARAM); synchronises. */
kg_status kg_mlp_loss_grad(kg_ctx *c, const double *features, const double *targets, long long n,
                           double *loss, double *grad);

/* Training log: capacity > 0 keeps the last `capacity` rows that learned
 * sweeps log (the features of every candidate of every non-empty attempt,
 * with target min(1, exp(-dE/T))); 0 turns logging off and frees the log. */
kg_status kg_mlp_log(kg_ctx *c, long long capacity);

/* Copy up to cap logged rows, oldest first, to host features (cap x 24) and
 * targets (cap); *n receives the count; synchronises. */
kg_status kg_mlp_log_read(kg_ctx *c, double *features, double *targets, long long cap, long long *n);

/* iters Adam steps (lr; betas 0.9, 0.999) on minibatches of `batch` rows
 * drawn uniformly from the log (with replacement); *loss receives the last
 * minibatch's mean loss (may be NULL).  KG_ERR_STATE when the log is empty. */
kg_status kg_mlp_train(kg_ctx *c, int iters, int batch, double lr, double *loss);

/* As kg_db_sweep / kg_db_sweep_k with the learned proposal mixed at lambda in
 * (0, 1].  The acceptance always includes the proposal ratio (the
 * KG_FLAG_PAPER_METROPOLIS flag is ignored here). */
kg_status kg_db_sweep_learned(kg_ctx *c, double attempts_per_monomer, double lambda, kg_db_stats *stats);
kg_status kg_db_sweep_learned_k(kg_ctx *c, const long long *attempts, double lambda, kg_db_stats *stats);

/* The learned proposal of one bond (chain, bond) of melt `melt` in the
 * current state: *n candidates (0: none; their list order), their kind (0:
 * partner bond at the same index, 1: at N-2-bond), partner chain and bond,
 * features (n x 24), logits and probabilities pi; host arrays of
 * KG_DB_CAND_MAX (x 24) entries; synchronises. */
kg_status kg_db_proposal(kg_ctx *c, int melt, int chain, int bond, double lambda, int *n, int *kind,
                         int *partner_chain, int *partner_bond, double *features, double *logits,
                         double *prob);

/* Host helpers (no context): k_n of Eq. 9, and the twelve stages of the
 * paper's schedule for (kappa, N) at time step dt (Eqs. 12, 16-20; scheme 1
 * for kappa <= 2.5), each stage's length scaled by `scale` (1: the paper's). */
double kg_kn(double n, double R0, double l0);
kg_status kg_schedule_paper(double kappa, int chain_len, double dt, double scale,
                            kg_stage *out12);

void kg_destroy(kg_ctx *c);
const char *kg_strerror(kg_status s);

/* Monomer mean-squared displacement of `melt` (App. B, Fig. 11): kg_msd_reset
 * records every monomer's current unwrapped position (allocates the reference,
 * 48 bytes per monomer, on first use); kg_msd returns
 *     msd = (1/M) sum_i |r_i(t) - r_i(t_reset)|^2
 * in binary64, summed in a fixed order.  The box shifts that double-bridging
 * swaps add to moved segments (to keep new bonds minimum-image) are added to
 * the reference as well, so a swap, which relabels monomers but moves none,
 * leaves the MSD unchanged.  Running without kg_db_sweep is the paper's
 * core-softening-only ablation.  kg_msd synchronises; KG_ERR_INVALID_ARG
 * before the first kg_msd_reset. */
kg_status kg_msd_reset(kg_ctx *c, int melt);
kg_status kg_msd(kg_ctx *c, int melt, double *msd);

/* The paper's initial state (Sec. II.B): freely rotating chains of
 * chain_len monomers with bond length l0 and a fixed
 * angle theta* between consecutive bonds, cos theta* = (r - 1) / (r + 1),
 * r = l_K / l0 from Eq. 12 (Eq. 13 as printed is garbled; this inverts the
 * FR relation l_K / l0 = (1 + c) / (1 - c)); first monomer uniform in the
 * box, first bond uniform on the sphere, uniform azimuths.  A state whose
 * Eq. 14 fit over N/4 <= n <= N/2 (kg_fit_lk) misses Eq. 12 by more than 2%
 * is redrawn, up to max_attempts (KG_ERR_CAPACITY past that).  Random numbers:
 * Philox4x32-10, key = seed, counter (monomer index in the chain, chain,
 * attempt, 5), u = (w + 1/2) 2^-32.  x: host (3, n_chains chain_len)
 * unwrapped, chain-major; *lk_fit and *attempts may be NULL.  Host only. */
kg_status kg_generate_fr(int n_chains, int chain_len, double box, double kappa, double l0, unsigned long long seed,
                         int max_attempts, double *x, double *lk_fit, int *attempts);

/* Static structure factor of `melt` (App. A): S[a] = |sum_j exp(i q_a . r_j)|^2
 * / M for q_a = 2 pi (h, k, l)_a / L, hkl a host array of nq integer triples
 * (nq <= 65535), S host.  Phases reduced to whole turns in binary64 and
 * evaluated in binary32; sums in binary64, fixed order.  Synchronises. */
kg_status kg_structure_factor(kg_ctx *c, int melt, const int *hkl, int nq, double *S);

/* Pair distribution of `melt` (App. A): g[b] for bins of width r_max / nbins
 * over [0, r_max), the number of ordered pairs i != j at minimum-image distance
 * r in the bin (binary64 distance, as the Verlet build defines it) divided by
 * M rho 4 pi / 3 (r_hi^3 - r_lo^3), rho = M / L^3.  r_max <= L / 2,
 * nbins <= 2048; g host.  Synchronises. */
kg_status kg_pair_distribution(kg_ctx *c, int melt, double r_max, int nbins, double *g);

/* Kuhn length from chain statistics (Eq. 14, Sec. II.B): the l_K that
 * minimises sum_{n = n_lo..n_hi} [r2n[n] / (n l0) - l_K (1 - l_K / (2 n l0)
 * (1 - exp(-2 n l0 / l_K)))]^2, unweighted (the paper does not state its
 * weighting).  r2n: host array of N values, r2n[n] = <R^2(n)> as kg_observables
 * returns it (r2n[0] unused); n_lo, n_hi <= 0 select the paper's N/4 .. N/2.
 * Host computation (bracketing scan on a log grid, then golden-section search
 * in log l_K); no context, no device.  KG_ERR_INVALID_ARG on a bad range,
 * l0 <= 0 or a non-finite value in the range. */
kg_status kg_fit_lk(const double *r2n, int N, double l0, int n_lo, int n_hi, double *lk);

/* Primitive-path analysis (PPA), the N_e measurement of Sec. III: the method of
 * Everaers et al. (Science 303, 823 (2004)), which the paper cites without
 * restating, in this form -- both end monomers of every chain fixed; the n = 12
 * member of Eq. 5 (LJ 12-6 truncated and shifted at 2^(1/6)) only between
 * monomers of different chains (any periodic image), none inside a chain, so
 * bonds keep their FENE part alone (Eq. 10 without U_MLJ, k = k_fene, R0 of
 * kg_params); no bending; the energy minimised by n_iter steps of the
 * integrator at T = 0 (velocity Verlet with friction gamma and no noise) from
 * rest:  v += dt/2 F;  x += dt v;  F = F_c(x) - gamma v;  v += dt/2 F.
 * Runs on a copy of `melt`'s current state; the simulation state is not
 * changed.  Neighbours within 2^(1/6) + skin are listed on a cell grid of side
 * >= 2^(1/6) + skin, rebuilt when a monomer has moved more than skin / 2 (the
 * grid must have 3 to 1024 cells a side, else KG_ERR_INVALID_ARG).
 * precision KG_FP64: everything in binary64.  KG_MIXED: pair vectors from
 * binary32 cell offsets plus binary32 displacements (~1e-7 sigma), bond vectors
 * as binary64 differences rounded to binary32, forces, velocities and the kick
 * in binary32, positions in binary64.
 *
 *   lpp       host, n_chains doubles or NULL: every chain's minimised contour
 *             length sum_i |r_{i+1} - r_i|
 *   x_out     host or device, 3 M doubles (3, M) slot order, or NULL: the
 *             minimised positions
 *   res       host or NULL: lpp_mean, the mean over chains (L_pp of Eq. 22);
 *             fmax, the largest net force on a mobile monomer after the last
 *             step (a convergence measure); builds, the neighbour-list builds;
 *             mean_neighbours, the mean length of the last list
 * Device work space per monomer: 192 (KG_FP64) or 120 (KG_MIXED) bytes of
 * double-buffered state and output, 64 (KG_FP64) or 80 (KG_MIXED) bytes of
 * binary32 records and 137 ints (128 of them the list); plus the cell grid.
 * Synchronises.  A bond reaching R0 returns KG_ERR_BOND_OVERSTRETCH, a
 * non-finite position KG_ERR_NONFINITE, more than 128 listed neighbours or
 * 1024 monomers in one cell KG_ERR_CAPACITY; none of them latches the context. */
typedef struct {
    long long n_iter;         /* minimisation steps (>= 0)                                */
    double dt;                /* step (> 0)                                               */
    double gamma;             /* friction (>= 0)                                          */
    double skin;              /* Verlet skin (> 0)                                        */
    double k_fene;            /* FENE spring; <= 0: k_n of Eq. 9 at n = 12                */
    int precision;            /* KG_FP64 or KG_MIXED                                      */
} kg_ppa_params;

typedef struct {
    double lpp_mean;          /* mean primitive-path length over chains                   */
    double fmax;              /* largest net force on a mobile monomer after the last step */
    long long builds;         /* neighbour-list builds, the first included                */
    double mean_neighbours;   /* mean length of the last interchain list                  */
} kg_ppa_result;

kg_status kg_primitive_path(kg_ctx *c, int melt, const kg_ppa_params *p, double *lpp, double *x_out,
                            kg_ppa_result *res);

/* Entanglement length from the primitive paths (Eq. 22, Sec. III): the N_eK
 * solving (2 N_eK + exp(-2 N_eK) - 1) / (2 N_eK^2) = (L_pp / L)^2 with
 * L = (chain_len - 1) l0, found by bisection in log N_eK (the left-hand side
 * falls monotonically from 1 to 0), and N_e = N_eK l_K / l0 (n_e may be NULL;
 * l_k is then ignored).  KG_ERR_INVALID_ARG unless 0 < L_pp / L < 1.  Host
 * only. */
kg_status kg_entanglement_length(double lpp_mean, int chain_len, double l0, double l_k, double *n_ek,
                                 double *n_e);

/* Largest n_chains * chain_len that kg_r2n_noalloc accepts (its chains may be
 * at most KG_R2N_MAX_CHAIN_LEN long). */
#define KG_NOALLOC_MAX_MONOMERS 2097152

/* <R^2(n)> for n = 0..N-1 of chains whose positions already sit in device
 * memory, computed without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory -- code that runs while another framework owns the whole
 * device heap, or between steps of a latency-critical loop where a
 * cudaMalloc/cudaFree (which can synchronise the device) is not acceptable.
 *
 *   x        device pointer, (3, stride) binary64 SoA, chain-major slots
 *            c*N + i in [0, n_chains*chain_len); unwrapped positions
 *   stride   distance in doubles between the x, y and z rows (>= M; any
 *            64-bit value, indices are formed in 64-bit arithmetic)
 *   out      device pointer to chain_len doubles; out[0] = 0
 *   stream   cudaStream_t to enqueue on (NULL: the default stream)
 *
 * Its per-chain partial sums go to one file-scope device array of
 * KG_NOALLOC_MAX_MONOMERS doubles (16 MiB), which every GPU that loads the
 * library holds until the process exits.  Sizes beyond that maximum (or
 * chains longer than KG_R2N_MAX_CHAIN_LEN) return KG_ERR_INVALID_ARG.  Every
 * call looks up the array's device address (cudaGetSymbolAddress) on the
 * current device, so call it with the device that holds x current; the first
 * call on a device loads the library's kernels there, so make that first call
 * before any stream capture.  Calls share the array and overwrite it
 * completely, so calls that overlap on the GPU (different streams, or devices
 * sharing nothing but this host code) race: serialise them.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
kg_status kg_r2n_noalloc(const double *x, long long stride, int n_chains, int chain_len, double *out,
                         void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KG_H */
