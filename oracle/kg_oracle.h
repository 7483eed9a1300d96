/*
 * kg_oracle.h -- plain, slow FP64 CPU oracle for the core-softened
 * double-bridging hybrid (DBH) method of Dietz & Hoy (arXiv:2109.11001).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this code; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source with the CUDA library.
 *
 * One melt of n_chains linear chains of chain_len monomers in a cubic
 * periodic box of side `box`.  Storage is chain-major: slot s = c*N + i holds
 * monomer i of chain c; bonds join slots s and s+1 of the same chain.
 * Positions are unwrapped, SoA: x[0..M) = x, x[M..2M) = y, x[2M..3M) = z.
 *
 * Units: m = sigma = epsilon = k_B = 1 (Sec. II.A, Sec. II.B).
 */
#ifndef KG_ORACLE_H
#define KG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_chains;            /* N_ch                                        */
    int chain_len;           /* N                                           */
    double box;              /* L; V = N_ch N / rho                         */
    double kappa;            /* bending stiffness, Eq. 4                    */
    double n_exp;            /* exponent n of U_MLJ^n, Eqs. 5-6, set Xi Eq. 11 */
    double k_fene;           /* k_n, Eq. 9 (30 for the standard model)     */
    double R0;               /* FENE maximum extent, 1.5 (Eq. 3)            */
    double T;                /* temperature (1)                             */
    double gamma;            /* Langevin friction (reading; paper silent)  */
    double dt;               /* MD time step                                */
    double db_bond_max;      /* 1.3: longest bond a DB swap may create (Sec. II.B) */
    unsigned long long seed; /* Philox key                                  */
    unsigned int stream;     /* melt index: selects an independent stream  */
    int paper_metropolis;    /* 1: acceptance without the proposal ratio   */
    double fene_qmin;        /* 0: Eq. 3 as printed (r >= R0 is an error);
                                > 0: C1 harmonic continuation beyond
                                r* = R0 sqrt(1 - fene_qmin)               */
} orc_params;

/* status codes */
#define ORC_OK 0
#define ORC_OVERSTRETCH 1   /* a bond reached r >= R0 (FENE undefined)   */
#define ORC_NONFINITE 2
#define ORC_CAPACITY 3
#define ORC_BADARG 4

/* ---- potentials (Sec. II.A) ---- */
double orc_rc(void);                                  /* 2^(1/6)             */
double orc_mlj_u(double n, double r);                 /* Eqs. 5-6, trunc+shift */
double orc_mlj_du(double n, double r);                /* dU/dr               */
double orc_kn(double n, double R0, double l0);        /* Eq. 9               */
double orc_fene_u(double k, double R0, double r);     /* log term of Eq. 10  */
double orc_fene_du(double k, double R0, double r);
double orc_fene_reg_u(double k, double R0, double qmin, double r);   /* regularised */
double orc_fene_reg_du(double k, double R0, double qmin, double r);

/* ---- counter-based RNG ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_gauss3(unsigned long long seed, unsigned int stream, long long step,
                unsigned int slot, double g[3]);

/* ---- neighbour list (set definition, two constructions) ----
 * CSR output: offs[M+1], nbr[offs[i]..offs[i+1]) sorted ascending.
 * Returns total pair count, or -1 when `cap` is too small. */
long long orc_nlist(const orc_params *p, const double *x, double rlist,
                    int use_cells, int *offs, int *nbr, long long cap);

/* ---- forces and energies ----
 * F: 3M conservative force.  e (may be NULL): [pair, bond, angle, virial]. */
int orc_forces(const orc_params *p, const double *x, double *F, double *e);

/* ---- Langevin MD (leapfrog form of velocity Verlet + Langevin) ----
 * State (x_n, u_{n-1/2}); *step = n on entry, n + nsteps on exit. */
int orc_run(const orc_params *p, double *x, double *u, long long *step, long long nsteps);

/* integer-time observables at the current state:
 * out[0..6] = e_pair, e_bond, e_angle, e_kin, virial, temperature, pressure */
int orc_observe(const orc_params *p, const double *x, const double *u, long long step,
                double *out);

/* <R^2(n)> for n = 0..N-1 (out[0] = 0), plain unwrapped differences */
void orc_r2n(const orc_params *p, const double *x, double *out);

/* bond-length histogram on [0, R0) and cos(theta) histogram on [-1, 1] */
void orc_hist(const orc_params *p, const double *x, int nbins, double *bond_h, double *cos_h);

/* ---- double-bridging Monte Carlo (Fig. 1, Sec. II.B) ----
 * K attempts of sweep number `sweep`, processed strictly in order.
 * stats[0] = attempted, stats[1] = with an empty partner set,
 * stats[2] = accepted.  x, u, pid are permuted in place. */
int orc_db_sweep(const orc_params *p, double *x, double *u, int *pid,
                 long long sweep, long long K, long long *stats);

/* partner count |P(b)| of bond b = (chain c, index p) in the given state */
int orc_db_partners(const orc_params *p, const double *x, const int *pid, int c, int b);

/* the partner list of bond (c, b) in proposal order (by the ids of the
 * partner monomer that bonds to (c, b) and of its bond neighbour): kind,
 * chain and bond index of each entry, up to cap; returns |P(b)| */
int orc_db_candidates(const orc_params *p, const double *x, const int *pid, int c, int b, int *kind, int *d,
                      int *q, int cap);

/* topology energy of the chains: sum of FENE log terms + bending (Eq. 4) */
double orc_topo_energy(const orc_params *p, const double *x);

/* ---- learned double-bridging proposal (not in the paper) ----
 * MLP 24 -> 64 -> 64 -> 1 with ReLU; parameters packed as
 * W1[64][24], b1[64], W2[64][64], b2[64], w3[64], b3 (ORC_MLP_NPARAM doubles). */
#define ORC_MLP_NPARAM (64 * 24 + 64 + 64 * 64 + 64 + 64 + 1)
double orc_mlp_forward(const double *w, const double f[24]);

/* features of the swap that pairs bond (chain c, index b) with partner entry
 * (kind, d, q) of its partner list, in the current state */
void orc_move_features(const orc_params *p, const double *x, int c, int b, int kind, int d, int q,
                       double f[24]);

/* One sweep with the learned proposal: the drawn bond's partner is chosen with
 * probability (1 - lambda) softmax(MLP logits) + lambda / |P|, and moves are
 * accepted with min(1, exp(-dE/T) q(x'->x) / q(x->x')).  bf16_in = 1 rounds the
 * features to bfloat16 before the network (the input precision of a bf16
 * tensor-core network); the network itself stays FP64.  log_f / log_t (may be
 * NULL) receive the features and min(1, exp(-dE/T)) of every candidate of every
 * non-empty attempt, up to log_cap rows; *log_n the number written. */
int orc_db_sweep_learned(const orc_params *p, double *x, double *u, int *pid, long long sweep, long long K,
                         const double *w, double lambda, int bf16_in, long long *stats, double *log_f,
                         double *log_t, long long log_cap, long long *log_n);

/* v rounded to the nearest bfloat16 (8 significant bits), ties to even */
double orc_bf16_round(double v);

#ifdef __cplusplus
}
#endif
#endif
