/*
 * kg_oracle.c -- plain FP64 CPU oracle for the core-softened DBH method of
 * Dietz & Hoy, "Facile equilibration of well-entangled semiflexible
 * bead-spring polymer melts" (arXiv:2109.11001).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
 * CPU-baseline leg of the benchmark.  It is written for a reader checking it
 * against the paper, not for speed, and shares no code with the CUDA library.
 * Build with -ffp-contract=off so that every distance is evaluated exactly as
 * written (no fused multiply-add).
 *
 * Readings of points the paper leaves open are marked READING; the same
 * readings are listed in the design notes of the repository.
 */
#include "kg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Potentials, Sec. II.A                                                    */
/* ------------------------------------------------------------------------ */

/* Cutoff r_c = 2^(1/6) sigma (Eq. 2, and Sec. II.A: the simulations use it). */
double orc_rc(void) { return pow(2.0, 1.0 / 6.0); }

/* Eq. 5 with m = 6 is the n-6 Mie potential
 *     U(r) = [6 2^(n/6) r^-n - 2n r^-6] / (n - 6).
 * Eq. 6 uses it for r <= 2^(1/6); the runs truncate at r_c = 2^(1/6) and shift
 * so that U(r_c) = 0.  U^{n-6}(2^(1/6)) = -1 for every n (READING: the shift
 * is therefore +epsilon, the paper does not print it). */
double orc_mlj_u(double n, double r)
{
    if (r >= orc_rc()) return 0.0;
    return (6.0 * pow(2.0, n / 6.0) * pow(r, -n) - 2.0 * n * pow(r, -6.0)) / (n - 6.0) + 1.0;
}

/* dU/dr of the same truncated-shifted form (zero beyond r_c). */
double orc_mlj_du(double n, double r)
{
    if (r >= orc_rc()) return 0.0;
    return (-6.0 * n * pow(2.0, n / 6.0) * pow(r, -n - 1.0) + 12.0 * n * pow(r, -7.0)) / (n - 6.0);
}

/* Eq. 9: FENE constant k_n that keeps the mechanical-equilibrium bond length
 * at l0 (0.960897 sigma) when the pair term is U_MLJ^n. */
double orc_kn(double n, double R0, double l0)
{
    return 6.0 * n * (R0 * R0 - l0 * l0) * (pow(2.0, n / 6.0) * pow(l0, -n) - 2.0 * pow(l0, -6.0))
           / ((n - 6.0) * R0 * R0 * l0 * l0);
}

/* FENE log term of Eqs. 3 and 10: -(k R0^2 / 2) ln(1 - (r/R0)^2). */
double orc_fene_u(double k, double R0, double r)
{
    return -0.5 * k * R0 * R0 * log(1.0 - (r / R0) * (r / R0));
}

double orc_fene_du(double k, double R0, double r)
{
    return k * r / (1.0 - (r / R0) * (r / R0));
}

/* READING: Eq. 3 is singular at r = R0 and the paper's engine (LAMMPS) does
 * not stop there, it limits the force near R0.  With qmin > 0 the log term is
 * kept for q = 1 - (r/R0)^2 >= qmin and continued beyond r* = R0 sqrt(1 - qmin)
 * by the quadratic in r^2 that matches its value and slope at r*:
 *     U = -(k R0^2 / 2) ln(qmin) + k (r^2 - r*^2) / (2 qmin).
 * qmin = 0 is Eq. 3 unchanged. */
double orc_fene_reg_u(double k, double R0, double qmin, double r)
{
    double q = 1.0 - (r / R0) * (r / R0);
    if (qmin <= 0.0 || q >= qmin) return orc_fene_u(k, R0, r);
    double rs2 = (1.0 - qmin) * R0 * R0;
    return -0.5 * k * R0 * R0 * log(qmin) + k * (r * r - rs2) / (2.0 * qmin);
}

double orc_fene_reg_du(double k, double R0, double qmin, double r)
{
    double q = 1.0 - (r / R0) * (r / R0);
    if (qmin <= 0.0 || q >= qmin) return orc_fene_du(k, R0, r);
    return k * r / qmin;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its       */
/* published definition: 10 rounds of two 32x32->64 multiplies with the      */
/* round multipliers 0xD2511F53, 0xCD9E8D57 and a Weyl key schedule with     */
/* increments 0x9E3779B9, 0xBB67AE85.                                        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout shared by every draw: (index, time_lo, time_hi, stream<<4 | purpose),
 * key = (seed_lo, seed_hi).  Purposes: 0 MD noise, 1 DB attempt, 2 DB partner pick. */
static void philox_draw(unsigned long long seed, unsigned int stream, unsigned int purpose,
                        unsigned long long time, uint32_t index, uint32_t out[4])
{
    uint32_t ctr[4] = {index, (uint32_t)time, (uint32_t)(time >> 32), (stream << 4) | purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform in (0,1) from the top 23 bits of a word: (2*(w>>9)+1) * 2^-24 is
 * exactly representable in binary32 and binary64 alike. */
static double unit_open(uint32_t w) { return (double)(2u * (w >> 9) + 1u) * (1.0 / 16777216.0); }

/* Three standard normals by the Box-Muller transform of two uniform pairs. */
void orc_gauss3(unsigned long long seed, unsigned int stream, long long step,
                unsigned int slot, double g[3])
{
    uint32_t r[4];
    philox_draw(seed, stream, 0, (unsigned long long)step, slot, r);
    const double two_pi = 6.283185307179586;
    double u0 = unit_open(r[0]), u1 = unit_open(r[1]);
    double u2 = unit_open(r[2]), u3 = unit_open(r[3]);
    double a = sqrt(-2.0 * log(u0)), b = sqrt(-2.0 * log(u2));
    g[0] = a * cos(two_pi * u1);
    g[1] = a * sin(two_pi * u1);
    g[2] = b * cos(two_pi * u3);
}

/* floor(w * n / 2^64) for a 64-bit word w: an exact integer map onto [0, n). */
static long long mul_hi64(uint64_t w, uint64_t n)
{
    return (long long)(((unsigned __int128)w * n) >> 64);
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                 */
/* ------------------------------------------------------------------------ */

/* minimum image of one coordinate difference (round half to even) */
static double min_image(double d, double L) { return d - L * rint(d / L); }

/* squared minimum-image distance between slots s and t, evaluated as
 * ((dx*dx + dy*dy) + dz*dz) with no contraction */
static double dist2(const double *x, int M, double L, int s, int t)
{
    double dx = min_image(x[t] - x[s], L);
    double dy = min_image(x[M + t] - x[M + s], L);
    double dz = min_image(x[2 * M + t] - x[2 * M + s], L);
    return dx * dx + dy * dy + dz * dz;
}

/* 1-2 bonded pair: same chain, neighbouring positions */
static int bonded12(int N, int s, int t)
{
    return (s / N == t / N) && (s - t == 1 || t - s == 1);
}

/* Linked-cell grid with cells no smaller than rcut. */
typedef struct {
    int n;          /* cells per side (0: use all pairs)                  */
    double h;
    int *head, *next, *cell;
} cellgrid;

static void grid_build(cellgrid *g, const double *x, int M, double L, double rcut)
{
    int n = (int)floor(L / (rcut * (1.0 + 1e-9)));
    g->n = n >= 3 ? n : 0;
    g->head = g->next = g->cell = NULL;
    if (!g->n) return;
    g->h = L / n;
    g->head = (int *)malloc(sizeof(int) * (size_t)n * n * n);
    g->next = (int *)malloc(sizeof(int) * (size_t)M);
    g->cell = (int *)malloc(sizeof(int) * (size_t)M);
    for (long c = 0; c < (long)n * n * n; ++c) g->head[c] = -1;
    for (int s = M - 1; s >= 0; --s) {
        int ci[3];
        for (int d = 0; d < 3; ++d) {
            double w = x[d * M + s] - L * floor(x[d * M + s] / L);
            if (w >= L) w -= L;
            int k = (int)(w / g->h);
            ci[d] = k < n ? (k < 0 ? 0 : k) : n - 1;
        }
        int c = (ci[2] * n + ci[1]) * n + ci[0];
        g->cell[s] = c;
        g->next[s] = g->head[c];
        g->head[c] = s;
    }
}

static void grid_free(cellgrid *g)
{
    free(g->head); free(g->next); free(g->cell);
}

/* Collect into `out` every slot in the 27 cells around slot s (all slots if
 * the grid is too small for cells).  Returns the count. */
static int grid_gather(const cellgrid *g, int M, int s, int *out)
{
    int cnt = 0;
    if (!g->n) {
        for (int t = 0; t < M; ++t) out[cnt++] = t;
        return cnt;
    }
    int n = g->n, c = g->cell[s];
    int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int nx = (cx + dx + n) % n, ny = (cy + dy + n) % n, nz = (cz + dz + n) % n;
                for (int t = g->head[(nz * n + ny) * n + nx]; t >= 0; t = g->next[t]) out[cnt++] = t;
            }
    return cnt;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Neighbour list: the set {(i,j): i != j, not 1-2 bonded, r^2 < rlist^2}.
 * use_cells = 0 tests every pair; 1 uses the linked-cell grid. */
long long orc_nlist(const orc_params *p, const double *x, double rlist,
                    int use_cells, int *offs, int *nbr, long long cap)
{
    int N = p->chain_len, M = p->n_chains * N;
    double L = p->box, rl2 = rlist * rlist;
    cellgrid g;
    if (use_cells) grid_build(&g, x, M, L, rlist);
    else g.n = 0, g.head = g.next = g.cell = NULL;
    int *cand = (int *)malloc(sizeof(int) * (size_t)M);
    long long tot = 0;
    for (int s = 0; s < M; ++s) {
        offs[s] = (int)tot;
        int nc = grid_gather(&g, M, s, cand);
        long long start = tot;
        for (int k = 0; k < nc; ++k) {
            int t = cand[k];
            if (t == s || bonded12(N, s, t)) continue;
            if (dist2(x, M, L, s, t) < rl2) {
                if (tot >= cap) { free(cand); grid_free(&g); return -1; }
                nbr[tot++] = t;
            }
        }
        qsort(nbr + start, (size_t)(tot - start), sizeof(int), cmp_int);
    }
    offs[M] = (int)tot;
    free(cand);
    grid_free(&g);
    return tot;
}

/* ------------------------------------------------------------------------ */
/* Forces and energies                                                      */
/* ------------------------------------------------------------------------ */

/* Adds the pair force of a central potential with derivative du at
 * separation vector d = x_t - x_s of length r. */
static void add_central(double *F, int M, int s, int t, const double d[3], double r, double du)
{
    for (int k = 0; k < 3; ++k) {
        double f = -du * d[k] / r;      /* force on t */
        F[k * M + t] += f;
        F[k * M + s] -= f;
    }
}

/* Conservative forces:
 *   pairs: U_MLJ^n (Eq. 6, truncated/shifted) between all pairs except 1-2
 *          bonded ones (READING: 1-3 and further pairs interact, as in the
 *          standard Kremer-Grest model);
 *   bonds: U_bond^n = U_MLJ^n + FENE with k_n (Eq. 10);
 *   angles: kappa (1 - cos theta), theta between consecutive bond vectors (Eq. 4). */
int orc_forces(const orc_params *p, const double *x, double *F, double *e)
{
    int N = p->chain_len, M = p->n_chains * N;
    double L = p->box, n = p->n_exp, rc = orc_rc(), rc2 = rc * rc;
    double epair = 0.0, ebond = 0.0, eang = 0.0, vir = 0.0;
    memset(F, 0, sizeof(double) * 3 * (size_t)M);

    cellgrid g;
    grid_build(&g, x, M, L, rc);
    int *cand = (int *)malloc(sizeof(int) * (size_t)M);
    for (int s = 0; s < M; ++s) {
        int nc = grid_gather(&g, M, s, cand);
        for (int k = 0; k < nc; ++k) {
            int t = cand[k];
            if (t <= s || bonded12(N, s, t)) continue;
            double d[3] = {min_image(x[t] - x[s], L), min_image(x[M + t] - x[M + s], L),
                           min_image(x[2 * M + t] - x[2 * M + s], L)};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rc2) continue;
            double r = sqrt(r2), du = orc_mlj_du(n, r);
            epair += orc_mlj_u(n, r);
            vir += -du * r;
            add_central(F, M, s, t, d, r, du);
        }
    }
    free(cand);
    grid_free(&g);

    for (int c = 0; c < p->n_chains; ++c) {
        for (int i = 0; i + 1 < N; ++i) {
            int s = c * N + i, t = s + 1;
            double d[3] = {min_image(x[t] - x[s], L), min_image(x[M + t] - x[M + s], L),
                           min_image(x[2 * M + t] - x[2 * M + s], L)};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (p->fene_qmin <= 0.0 ? !(r < p->R0) : !(r < 2.0 * p->R0)) return ORC_OVERSTRETCH;
            double du = orc_mlj_du(n, r) + orc_fene_reg_du(p->k_fene, p->R0, p->fene_qmin, r);
            ebond += orc_mlj_u(n, r) + orc_fene_reg_u(p->k_fene, p->R0, p->fene_qmin, r);
            vir += -du * r;
            add_central(F, M, s, t, d, r, du);
        }
        for (int i = 1; i + 1 < N; ++i) {
            int a = c * N + i - 1, b = a + 1, cc = a + 2;
            double b1[3], b2[3];
            for (int k = 0; k < 3; ++k) {
                b1[k] = min_image(x[k * M + b] - x[k * M + a], L);
                b2[k] = min_image(x[k * M + cc] - x[k * M + b], L);
            }
            double l1 = sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
            double l2 = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
            double cs = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / (l1 * l2);
            eang += p->kappa * (1.0 - cs);
            for (int k = 0; k < 3; ++k) {
                double g1 = b2[k] / (l1 * l2) - cs * b1[k] / (l1 * l1);   /* d cos / d b1 */
                double g2 = b1[k] / (l1 * l2) - cs * b2[k] / (l2 * l2);   /* d cos / d b2 */
                F[k * M + a] += -p->kappa * g1;
                F[k * M + b] += p->kappa * (g1 - g2);
                F[k * M + cc] += p->kappa * g2;
            }
        }
    }
    for (long i = 0; i < 3L * M; ++i)
        if (!isfinite(F[i])) return ORC_NONFINITE;
    if (e) { e[0] = epair; e[1] = ebond; e[2] = eang; e[3] = vir; }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Langevin molecular dynamics                                              */
/* ------------------------------------------------------------------------ */

/* READING (the paper names LAMMPS, Sec. II.B, but no thermostat): velocity
 * Verlet with Langevin friction and Gaussian noise, i.e. per step
 *     v_{n+1/2} = v_n + dt/2 F_n,   x_{n+1} = x_n + dt v_{n+1/2},
 *     F_{n+1} = F_c(x_{n+1}) - gamma v_{n+1/2} + sqrt(2 gamma T / dt) g_{n+1},
 *     v_{n+1} = v_{n+1/2} + dt/2 F_{n+1}.
 * Written in its leapfrog form on the state (x_n, u = v_{n-1/2}):
 *     F_n = F_c(x_n) - gamma u + sqrt(2 gamma T / dt) g_n,
 *     u  <- u + dt F_n,   x <- x + dt u.
 * g_n for slot s is orc_gauss3(seed, stream, n, s). */
int orc_run(const orc_params *p, double *x, double *u, long long *step, long long nsteps)
{
    int M = p->n_chains * p->chain_len;
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    double amp = p->gamma > 0.0 ? sqrt(2.0 * p->gamma * p->T / p->dt) : 0.0;
    int st = ORC_OK;
    for (long long it = 0; it < nsteps && st == ORC_OK; ++it) {
        st = orc_forces(p, x, F, NULL);
        if (st != ORC_OK) break;
        for (int s = 0; s < M; ++s) {
            double g[3];
            orc_gauss3(p->seed, p->stream, *step, (unsigned)s, g);
            for (int k = 0; k < 3; ++k) {
                double f = F[k * M + s] - p->gamma * u[k * M + s] + amp * g[k];
                u[k * M + s] += p->dt * f;
                x[k * M + s] += p->dt * u[k * M + s];
            }
        }
        *step += 1;
    }
    free(F);
    return st;
}

/* Observables at integer time n: energies from the conservative forces, and
 * the velocity v_n = u + dt/2 F_n of the velocity-Verlet form above. */
int orc_observe(const orc_params *p, const double *x, const double *u, long long step, double *out)
{
    int M = p->n_chains * p->chain_len;
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    double e[4];
    int st = orc_forces(p, x, F, e);
    if (st != ORC_OK) { free(F); return st; }
    double amp = p->gamma > 0.0 ? sqrt(2.0 * p->gamma * p->T / p->dt) : 0.0;
    double ekin = 0.0;
    for (int s = 0; s < M; ++s) {
        double g[3];
        orc_gauss3(p->seed, p->stream, step, (unsigned)s, g);
        for (int k = 0; k < 3; ++k) {
            double f = F[k * M + s] - p->gamma * u[k * M + s] + amp * g[k];
            double v = u[k * M + s] + 0.5 * p->dt * f;
            ekin += 0.5 * v * v;
        }
    }
    free(F);
    double V = p->box * p->box * p->box;
    out[0] = e[0]; out[1] = e[1]; out[2] = e[2]; out[3] = ekin; out[4] = e[3];
    out[5] = 2.0 * ekin / (3.0 * M);
    out[6] = (2.0 * ekin + e[3]) / (3.0 * V);
    return ORC_OK;
}

/* <R^2(n)>: mean over chains and i of |x_{i+n} - x_i|^2 (Eq. 14's input). */
void orc_r2n(const orc_params *p, const double *x, double *out)
{
    int N = p->chain_len, M = p->n_chains * N;
    out[0] = 0.0;
    for (int n = 1; n < N; ++n) {
        double sum = 0.0;
        for (int c = 0; c < p->n_chains; ++c)
            for (int i = 0; i + n < N; ++i) {
                int s = c * N + i, t = s + n;
                double dx = x[t] - x[s], dy = x[M + t] - x[M + s], dz = x[2 * M + t] - x[2 * M + s];
                sum += dx * dx + dy * dy + dz * dz;
            }
        out[n] = sum / ((double)p->n_chains * (N - n));
    }
}

void orc_hist(const orc_params *p, const double *x, int nbins, double *bond_h, double *cos_h)
{
    int N = p->chain_len, M = p->n_chains * N;
    double L = p->box;
    for (int b = 0; b < nbins; ++b) bond_h[b] = cos_h[b] = 0.0;
    for (int c = 0; c < p->n_chains; ++c) {
        for (int i = 0; i + 1 < N; ++i) {
            int s = c * N + i;
            double r = sqrt(dist2(x, M, L, s, s + 1));
            int b = (int)floor(r / p->R0 * nbins);
            if (b >= 0 && b < nbins) bond_h[b] += 1.0;
        }
        for (int i = 1; i + 1 < N; ++i) {
            int a = c * N + i - 1;
            double b1[3], b2[3];
            for (int k = 0; k < 3; ++k) {
                b1[k] = min_image(x[k * M + a + 1] - x[k * M + a], L);
                b2[k] = min_image(x[k * M + a + 2] - x[k * M + a + 1], L);
            }
            double cs = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
                        / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
                           * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
            int b = (int)floor((cs + 1.0) * 0.5 * nbins);
            if (b >= nbins) b = nbins - 1;
            if (b < 0) b = 0;
            cos_h[b] += 1.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Double-bridging Monte Carlo (Fig. 1; Sec. II.B criteria (i) and (ii))    */
/* ------------------------------------------------------------------------ */
/*
 * READINGS (Fig. 1 is not reproduced in the text; the paper gives the move's
 * effect, its acceptance and two admissibility criteria):
 *  - A move removes bond (A_p, A_{p+1}) of chain A and bond (B_q, B_{q+1}) of a
 *    different chain B and joins the four ends crosswise so that both chains
 *    keep length N (criterion (i)).  This leaves two kinds:
 *      alpha (q = p):      new bonds (A_p, B_{p+1}), (B_p, A_{p+1});
 *                          A' = A_0..A_p B_{p+1}..B_{N-1}, B' = B_0..B_p A_{p+1}..A_{N-1}
 *      beta  (p+q = N-2):  new bonds (A_p, B_q), (A_{p+1}, B_{q+1});
 *                          A' = A_0..A_p B_q..B_0,  B' = A_{N-1}..A_{p+1} B_{q+1}..B_{N-1}
 *    with A the chain of lower index (so the result does not depend on which
 *    bond was drawn first).
 *  - Admissible iff both new bonds are <= 1.3 sigma (criterion (ii)) and both
 *    removed bonds are <= 1.3 sigma (so the reverse move is admissible too).
 *  - Proposal: draw one of the N_ch (N-1) bonds uniformly; P(b) is the list of
 *    admissible moves that remove b, ordered by the particle id of the monomer
 *    that would bond to b's lower-index end; one entry
 *    is drawn uniformly.  Ties (the same monomer offering both kinds) are
 *    broken by the particle id of the partner bond's other monomer; both keys
 *    follow the monomers, not the slots, so earlier swaps in a sweep that only
 *    relabel slots leave the order unchanged.  q(x->x') = [1/|P(b1)| + 1/|P(b2)|] / N_bonds, and the
 *    move is accepted with probability
 *        min(1, exp(-dE/T) q(x'->x)/q(x->x')),
 *    dE = change of FENE log terms and bending energy of the two chains (the
 *    U_MLJ parts cancel, since a pair moves between the bond sum and the pair
 *    sum with the same U_MLJ^n).  With paper_metropolis the proposal ratio is
 *    dropped, as in Fig. 1's acceptance.
 *  - Moved segments are shifted by a box vector so that each new bond is a
 *    minimum image in unwrapped coordinates; shifts are counted per monomer
 *    during the sweep and added to the positions once, at its end.
 */

typedef struct { int key, key2, kind, d, q; } orc_cand;

static int cmp_cand(const void *a, const void *b)
{
    const orc_cand *x = (const orc_cand *)a, *y = (const orc_cand *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->key2 > y->key2) - (x->key2 < y->key2);
}

/* Admissible partners of bond (chain c, index b), by testing every slot. */
static int enum_partners(const orc_params *p, const double *x, const int *pid, int c, int b,
                         orc_cand *out)
{
    int N = p->chain_len, M = p->n_chains * N;
    double L = p->box, lim2 = p->db_bond_max * p->db_bond_max;
    int u = c * N + b, w = u + 1, cnt = 0;
    if (dist2(x, M, L, u, w) > lim2) return 0;
    for (int t = 0; t < M; ++t) {
        int d = t / N, i = t % N;
        if (d == c) continue;
        if (dist2(x, M, L, u, t) > lim2) continue;
        if (i == b + 1) {                       /* alpha: t = D_{b+1} */
            int up = d * N + b;                 /*        D_b         */
            if (dist2(x, M, L, up, w) <= lim2 && dist2(x, M, L, up, t) <= lim2) {
                if (out) { out[cnt].key = pid[t]; out[cnt].key2 = pid[up]; out[cnt].kind = 0; out[cnt].d = d; out[cnt].q = b; }
                ++cnt;
            }
        }
        if (i == N - 2 - b) {                   /* beta: t = D_q, q = N-2-b */
            if (dist2(x, M, L, t + 1, w) <= lim2 && dist2(x, M, L, t, t + 1) <= lim2) {
                if (out) { out[cnt].key = pid[t]; out[cnt].key2 = pid[t + 1]; out[cnt].kind = 1; out[cnt].d = d; out[cnt].q = i; }
                ++cnt;
            }
        }
    }
    return cnt;
}

int orc_db_partners(const orc_params *p, const double *x, const int *pid, int c, int b)
{
    return enum_partners(p, x, pid, c, b, NULL);
}

int orc_db_candidates(const orc_params *p, const double *x, const int *pid, int c, int b, int *kind, int *d,
                      int *q, int cap)
{
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * 2 * (size_t)p->n_chains * p->chain_len);
    int n = enum_partners(p, x, pid, c, b, cand);
    qsort(cand, (size_t)n, sizeof(orc_cand), cmp_cand);
    for (int j = 0; j < n && j < cap; ++j) { kind[j] = cand[j].kind; d[j] = cand[j].d; q[j] = cand[j].q; }
    free(cand);
    return n;
}

/* FENE log terms plus bending energy of chain c */
static double chain_topo_energy(const orc_params *p, const double *x, int c)
{
    int N = p->chain_len, M = p->n_chains * N;
    double L = p->box, E = 0.0;
    for (int i = 0; i + 1 < N; ++i) {
        int s = c * N + i;
        E += orc_fene_reg_u(p->k_fene, p->R0, p->fene_qmin, sqrt(dist2(x, M, L, s, s + 1)));
    }
    for (int i = 1; i + 1 < N; ++i) {
        int a = c * N + i - 1;
        double b1[3], b2[3];
        for (int k = 0; k < 3; ++k) {
            b1[k] = min_image(x[k * M + a + 1] - x[k * M + a], L);
            b2[k] = min_image(x[k * M + a + 2] - x[k * M + a + 1], L);
        }
        double cs = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
                    / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
                       * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
        E += p->kappa * (1.0 - cs);
    }
    return E;
}

double orc_topo_energy(const orc_params *p, const double *x)
{
    double E = 0.0;
    for (int c = 0; c < p->n_chains; ++c) E += chain_topo_energy(p, x, c);
    return E;
}

/* per-slot record moved by a swap */
typedef struct { double x[3], u[3]; int pid; int img[3]; } slotrec;

static void load_rec(slotrec *r, const double *x, const double *u, const int *pid,
                     const int *img, int M, int s)
{
    for (int k = 0; k < 3; ++k) { r->x[k] = x[k * M + s]; r->u[k] = u[k * M + s]; r->img[k] = img[3 * s + k]; }
    r->pid = pid[s];
}

static void store_rec(const slotrec *r, double *x, double *u, int *pid, int *img, int M, int s)
{
    for (int k = 0; k < 3; ++k) { x[k * M + s] = r->x[k]; u[k * M + s] = r->u[k]; img[3 * s + k] = r->img[k]; }
    pid[s] = r->pid;
}

/* Shift slots [lo, hi] by the box vector that makes (anchor, first) a
 * minimum-image bond in the positions as they will be after the sweep. */
static void shift_segment(const orc_params *p, const double *x, int *img, int first, int anchor,
                          int lo, int hi)
{
    int M = p->n_chains * p->chain_len;
    double L = p->box;
    int sh[3];
    for (int k = 0; k < 3; ++k)
        sh[k] = -((int)rint((x[k * M + first] - x[k * M + anchor]) / L)
                  + img[3 * first + k] - img[3 * anchor + k]);
    for (int s = lo; s <= hi; ++s)
        for (int k = 0; k < 3; ++k) img[3 * s + k] += sh[k];
}

/* Apply the canonical move (kind, A < B, bond pA on A, bond pB on B). */
static void apply_move(const orc_params *p, double *x, double *u, int *pid, int *img,
                       int kind, int A, int B, int pA, int pB, slotrec *tmp)
{
    int N = p->chain_len, M = p->n_chains * N;
    if (kind == 0) {
        for (int i = pA + 1; i < N; ++i) {
            slotrec ra, rb;
            load_rec(&ra, x, u, pid, img, M, A * N + i);
            load_rec(&rb, x, u, pid, img, M, B * N + i);
            store_rec(&rb, x, u, pid, img, M, A * N + i);
            store_rec(&ra, x, u, pid, img, M, B * N + i);
        }
        shift_segment(p, x, img, A * N + pA + 1, A * N + pA, A * N + pA + 1, A * N + N - 1);
        shift_segment(p, x, img, B * N + pA + 1, B * N + pA, B * N + pA + 1, B * N + N - 1);
    } else {
        int q = pB, len = q + 1;                       /* = N - 1 - pA */
        slotrec *ta = tmp, *tb = tmp + len;
        for (int j = 0; j < len; ++j) {
            load_rec(&ta[j], x, u, pid, img, M, A * N + pA + 1 + j);   /* A_{pA+1..N-1} */
            load_rec(&tb[j], x, u, pid, img, M, B * N + j);            /* B_{0..q}      */
        }
        for (int j = 0; j < len; ++j) {
            store_rec(&tb[q - j], x, u, pid, img, M, A * N + pA + 1 + j); /* B_q..B_0       */
            store_rec(&ta[len - 1 - j], x, u, pid, img, M, B * N + j);    /* A_{N-1}..A_{pA+1} */
        }
        shift_segment(p, x, img, A * N + pA + 1, A * N + pA, A * N + pA + 1, A * N + N - 1);
        shift_segment(p, x, img, B * N + q, B * N + q + 1, B * N, B * N + q);
    }
}

int orc_db_sweep(const orc_params *p, double *x, double *u, int *pid,
                 long long sweep, long long K, long long *stats)
{
    int N = p->chain_len, M = p->n_chains * N;
    long long nbonds = (long long)p->n_chains * (N - 1);
    int *img = (int *)calloc(3 * (size_t)M, sizeof(int));
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)M * 2);
    slotrec *save = (slotrec *)malloc(sizeof(slotrec) * 2 * (size_t)N);
    slotrec *tmp = (slotrec *)malloc(sizeof(slotrec) * 2 * (size_t)N);
    long long n_att = 0, n_empty = 0, n_acc = 0;
    int st = ORC_OK;

    for (long long k = 0; k < K; ++k) {
        uint32_t r[4], r2[4];
        philox_draw(p->seed, p->stream, 1, (unsigned long long)sweep, (uint32_t)k, r);
        philox_draw(p->seed, p->stream, 2, (unsigned long long)sweep, (uint32_t)k, r2);
        long long bond = mul_hi64(((uint64_t)r[1] << 32) | r[0], (uint64_t)nbonds);
        double u_acc = ((double)(r[2] >> 5) * 67108864.0 + (double)(r[3] >> 6)) * (1.0 / 9007199254740992.0);
        int c = (int)(bond / (N - 1)), b = (int)(bond % (N - 1));
        ++n_att;

        int np1 = enum_partners(p, x, pid, c, b, cand);
        if (np1 == 0) { ++n_empty; continue; }
        qsort(cand, (size_t)np1, sizeof(orc_cand), cmp_cand);
        orc_cand m = cand[mul_hi64(((uint64_t)r2[1] << 32) | r2[0], (uint64_t)np1)];
        int np2 = enum_partners(p, x, pid, m.d, m.q, NULL);

        int A = c < m.d ? c : m.d, B = c < m.d ? m.d : c;
        int pA = (A == c) ? b : m.q, pB = (A == c) ? m.q : b;

        double e_old = chain_topo_energy(p, x, A) + chain_topo_energy(p, x, B);
        for (int i = 0; i < N; ++i) {
            load_rec(&save[i], x, u, pid, img, M, A * N + i);
            load_rec(&save[N + i], x, u, pid, img, M, B * N + i);
        }
        apply_move(p, x, u, pid, img, m.kind, A, B, pA, pB, tmp);
        double e_new = chain_topo_energy(p, x, A) + chain_topo_energy(p, x, B);
        int nr1 = enum_partners(p, x, pid, A, pA, NULL);
        int nr2 = enum_partners(p, x, pid, B, pB, NULL);
        if (nr1 == 0 || nr2 == 0) { st = ORC_BADARG; break; }   /* reverse must be admissible */

        double ratio = (1.0 / nr1 + 1.0 / nr2) / (1.0 / np1 + 1.0 / np2);
        double a = exp(-(e_new - e_old) / p->T);
        if (!p->paper_metropolis) a *= ratio;
        if (u_acc < a) {
            ++n_acc;
        } else {
            for (int i = 0; i < N; ++i) {
                store_rec(&save[i], x, u, pid, img, M, A * N + i);
                store_rec(&save[N + i], x, u, pid, img, M, B * N + i);
            }
        }
    }
    for (int s = 0; s < M; ++s)
        for (int k = 0; k < 3; ++k) x[k * M + s] += p->box * (double)img[3 * s + k];
    free(img); free(cand); free(save); free(tmp);
    if (stats) { stats[0] = n_att; stats[1] = n_empty; stats[2] = n_acc; }
    return st;
}

/* ------------------------------------------------------------------------ */
/* Learned proposal (not in the paper; a reading of the proposal family      */
/* "any q with q(x->x') > 0 iff q(x'->x) > 0", made exact by the ratio).     */
/* ------------------------------------------------------------------------ */

double orc_mlp_forward(const double *w, const double f[24])
{
    const double *W1 = w, *b1 = W1 + 64 * 24, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *w3 = b2 + 64;
    const double b3 = w3[64];
    double h1[64], h2[64];
    for (int o = 0; o < 64; ++o) {
        double a = b1[o];
        for (int i = 0; i < 24; ++i) a += W1[o * 24 + i] * f[i];
        h1[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < 64; ++o) {
        double a = b2[o];
        for (int i = 0; i < 64; ++i) a += W2[o * 64 + i] * h1[i];
        h2[o] = a > 0.0 ? a : 0.0;
    }
    double s = b3;
    for (int i = 0; i < 64; ++i) s += w3[i] * h2[i];
    return s;
}

static void sort4(double *v)
{
    for (int i = 1; i < 4; ++i) {
        double t = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
        v[j + 1] = t;
    }
}

/* cos of the angle at vertex i of chain c (1 when i is a chain end) */
static double vertex_cos(const orc_params *p, const double *x, int c, int i)
{
    int N = p->chain_len, M = p->n_chains * N;
    if (i < 1 || i > N - 2) return 1.0;
    int a = c * N + i - 1;
    double L = p->box, b1[3], b2[3];
    for (int k = 0; k < 3; ++k) {
        b1[k] = min_image(x[k * M + a + 1] - x[k * M + a], L);
        b2[k] = min_image(x[k * M + a + 2] - x[k * M + a + 1], L);
    }
    return (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
           / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
              * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
}

static void canon(int N, int c, int b, int kind, int d, int q, int *A, int *B, int *pA, int *pB)
{
    (void)N; (void)kind;
    *A = c < d ? c : d;
    *B = c < d ? d : c;
    *pA = (*A == c) ? b : q;
    *pB = (*A == c) ? q : b;
}

/* Features (all a function of the move, not of which of its bonds was drawn):
 *  0-1 removed bond lengths (sorted)      2-3 new bond lengths (sorted)
 *  4   change of FENE log terms           5   change of bending energy
 *  6-9 cos at the four junction vertices before (sorted)
 * 10-13 the same after                   14-17 cos one vertex further out, before (sorted)
 * 18 cos between the removed bonds, each pointing from the monomer that bonds to u to the one that
 *    bonds to w (u -> w and X -> Y, new bonds u-X and Y-w)
 * 19 kappa/4  20 n/12  21 min(p+1, N-1-p)/N  22 dE  23 1
 * Every feature is a function of positions and bonds alone, not of the direction in which a chain's
 * slots are numbered: kinds 0 and 1 are the same reconnection seen from the two numberings. */
void orc_move_features(const orc_params *p, const double *x, int c, int b, int kind, int d, int q,
                       double f[24])
{
    int N = p->chain_len, M = p->n_chains * N;
    double L = p->box;
    int u = c * N + b, w = u + 1, X, Y;
    if (kind == 0) { Y = d * N + b; X = Y + 1; } else { X = d * N + q; Y = X + 1; }
    double o1 = sqrt(dist2(x, M, L, u, w)), o2 = sqrt(dist2(x, M, L, X, Y));
    double n1 = sqrt(dist2(x, M, L, u, X)), n2 = sqrt(dist2(x, M, L, Y, w));
    f[0] = o1 < o2 ? o1 : o2; f[1] = o1 < o2 ? o2 : o1;
    f[2] = n1 < n2 ? n1 : n2; f[3] = n1 < n2 ? n2 : n1;
    f[4] = orc_fene_reg_u(p->k_fene, p->R0, p->fene_qmin, n1) + orc_fene_reg_u(p->k_fene, p->R0, p->fene_qmin, n2)
           - orc_fene_reg_u(p->k_fene, p->R0, p->fene_qmin, o1) - orc_fene_reg_u(p->k_fene, p->R0, p->fene_qmin, o2);
    int A, B, pA, pB;
    canon(N, c, b, kind, d, q, &A, &B, &pA, &pB);
    double before[4] = {vertex_cos(p, x, A, pA), vertex_cos(p, x, A, pA + 1), vertex_cos(p, x, B, pB),
                        vertex_cos(p, x, B, pB + 1)};
    double outer[4] = {vertex_cos(p, x, A, pA - 1), vertex_cos(p, x, A, pA + 2), vertex_cos(p, x, B, pB - 1),
                       vertex_cos(p, x, B, pB + 2)};
    /* the state after the move, on copies of the two chains' positions */
    double *xx = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    memcpy(xx, x, sizeof(double) * 3 * (size_t)M);
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i < N; ++i) {
            int sa = A * N + i, sb = B * N + i, ta, tb;
            if (kind == 0) {
                ta = i > pA ? B * N + i : sa;
                tb = i > pA ? A * N + i : sb;
            } else {
                ta = i > pA ? B * N + (N - 1 - i) : sa;
                tb = i <= pB ? A * N + (N - 1 - i) : sb;
            }
            xx[k * M + sa] = x[k * M + ta];
            xx[k * M + sb] = x[k * M + tb];
        }
    }
    double after[4] = {vertex_cos(p, xx, A, pA), vertex_cos(p, xx, A, pA + 1), vertex_cos(p, xx, B, pB),
                       vertex_cos(p, xx, B, pB + 1)};
    double dbend = 0.0;
    for (int i = 0; i < 4; ++i) dbend += p->kappa * ((1.0 - after[i]) - (1.0 - before[i]));
    free(xx);
    f[5] = dbend;
    sort4(before); sort4(after); sort4(outer);
    for (int i = 0; i < 4; ++i) { f[6 + i] = before[i]; f[10 + i] = after[i]; f[14 + i] = outer[i]; }
    {
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = min_image(x[k * M + w] - x[k * M + u], L);
            e2[k] = min_image(x[k * M + Y] - x[k * M + X], L);
        }
        f[18] = (e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2])
                / (sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2])
                   * sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
    }
    f[19] = p->kappa / 4.0;
    f[20] = p->n_exp / 12.0;
    int lo = b + 1 < N - 1 - b ? b + 1 : N - 1 - b;
    f[21] = (double)lo / N;
    f[22] = f[4] + f[5];
    f[23] = 1.0;
}

/* v rounded to the nearest bfloat16 (8 significant bits), ties to even */
double orc_bf16_round(double v)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    double m = frexp(v, &e);                  /* v = m 2^e, 0.5 <= |m| < 1 */
    return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* proposal weights over a sorted partner list; returns the weight of entry j */
static void proposal_weights(const orc_params *p, const double *x, const double *w, double lambda, int bf16_in,
                             int c, int b, const orc_cand *cand, int n, double *pi)
{
    double smax = -1e300, z = 0.0;
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double f[24];
        orc_move_features(p, x, c, b, cand[j].kind, cand[j].d, cand[j].q, f);
        if (bf16_in)
            for (int i = 0; i < 24; ++i) f[i] = orc_bf16_round(f[i]);
        s[j] = orc_mlp_forward(w, f);
        if (s[j] > smax) smax = s[j];
    }
    for (int j = 0; j < n; ++j) z += exp(s[j] - smax);
    for (int j = 0; j < n; ++j) pi[j] = (1.0 - lambda) * exp(s[j] - smax) / z + lambda / n;
    free(s);
}

/* probability that bond (c, b)'s proposal picks the move with canonical form
 * (kind, A, B, pA, pB) */
static double pick_prob(const orc_params *p, const double *x, const int *pid, const double *w, double lambda,
                        int bf16_in, int c, int b, int kind, int A, int B, int pA, int pB, orc_cand *cand, double *pi)
{
    int N = p->chain_len;
    int n = enum_partners(p, x, pid, c, b, cand);
    if (n == 0) return 0.0;
    qsort(cand, (size_t)n, sizeof(orc_cand), cmp_cand);
    proposal_weights(p, x, w, lambda, bf16_in, c, b, cand, n, pi);
    for (int j = 0; j < n; ++j) {
        int a2, b2, pa2, pb2;
        canon(N, c, b, cand[j].kind, cand[j].d, cand[j].q, &a2, &b2, &pa2, &pb2);
        if (cand[j].kind == kind && a2 == A && b2 == B && pa2 == pA && pb2 == pB) return pi[j];
    }
    return 0.0;
}

int orc_db_sweep_learned(const orc_params *p, double *x, double *u, int *pid, long long sweep, long long K,
                         const double *w, double lambda, int bf16_in, long long *stats, double *log_f,
                         double *log_t, long long log_cap, long long *log_n)
{
    int N = p->chain_len, M = p->n_chains * N;
    long long nbonds = (long long)p->n_chains * (N - 1), nlog = 0;
    int *img = (int *)calloc(3 * (size_t)M, sizeof(int));
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)M * 2);
    double *pi = (double *)malloc(sizeof(double) * (size_t)M * 2);
    slotrec *save = (slotrec *)malloc(sizeof(slotrec) * 2 * (size_t)N);
    slotrec *tmp = (slotrec *)malloc(sizeof(slotrec) * 2 * (size_t)N);
    long long n_att = 0, n_empty = 0, n_acc = 0;
    int st = ORC_OK;
    for (long long k = 0; k < K; ++k) {
        uint32_t r[4], r2[4];
        philox_draw(p->seed, p->stream, 1, (unsigned long long)sweep, (uint32_t)k, r);
        philox_draw(p->seed, p->stream, 2, (unsigned long long)sweep, (uint32_t)k, r2);
        long long bond = mul_hi64(((uint64_t)r[1] << 32) | r[0], (uint64_t)nbonds);
        double u_acc = ((double)(r[2] >> 5) * 67108864.0 + (double)(r[3] >> 6)) * (1.0 / 9007199254740992.0);
        double u_pick = (double)((((uint64_t)r2[1] << 32) | r2[0]) >> 11) * (1.0 / 9007199254740992.0);
        int c = (int)(bond / (N - 1)), b = (int)(bond % (N - 1));
        ++n_att;
        int n1 = enum_partners(p, x, pid, c, b, cand);
        if (n1 == 0) { ++n_empty; continue; }
        qsort(cand, (size_t)n1, sizeof(orc_cand), cmp_cand);
        proposal_weights(p, x, w, lambda, bf16_in, c, b, cand, n1, pi);
        if (log_f) {
            for (int j = 0; j < n1 && nlog < log_cap; ++j, ++nlog) {
                orc_move_features(p, x, c, b, cand[j].kind, cand[j].d, cand[j].q, log_f + 24 * nlog);
                double de = log_f[24 * nlog + 22] / p->T;
                log_t[nlog] = de > 0.0 ? exp(-de) : 1.0;
            }
        }
        int j = 0;
        double cum = pi[0];
        while (j + 1 < n1 && u_pick >= cum) cum += pi[++j];
        orc_cand m = cand[j];
        int A, B, pA, pB;
        canon(N, c, b, m.kind, m.d, m.q, &A, &B, &pA, &pB);
        double f[24];
        orc_move_features(p, x, c, b, m.kind, m.d, m.q, f);
        double dE = f[22];
        /* forward: either removed bond may have been drawn */
        double q_fwd = pi[j] + pick_prob(p, x, pid, w, lambda, bf16_in, m.d, m.q, m.kind, A, B, pA, pB,
                                         cand + M, pi + M);
        for (int i = 0; i < N; ++i) {
            load_rec(&save[i], x, u, pid, img, M, A * N + i);
            load_rec(&save[N + i], x, u, pid, img, M, B * N + i);
        }
        apply_move(p, x, u, pid, img, m.kind, A, B, pA, pB, tmp);
        double q_rev = pick_prob(p, x, pid, w, lambda, bf16_in, A, pA, m.kind, A, B, pA, pB, cand + M, pi + M)
                       + pick_prob(p, x, pid, w, lambda, bf16_in, B, pB, m.kind, A, B, pA, pB, cand + M, pi + M);
        if (q_rev <= 0.0 || q_fwd <= 0.0) { st = ORC_BADARG; break; }
        double a = exp(-dE / p->T) * q_rev / q_fwd;
        if (u_acc < a) {
            ++n_acc;
        } else {
            for (int i = 0; i < N; ++i) {
                store_rec(&save[i], x, u, pid, img, M, A * N + i);
                store_rec(&save[N + i], x, u, pid, img, M, B * N + i);
            }
        }
    }
    for (int s = 0; s < M; ++s)
        for (int k = 0; k < 3; ++k) x[k * M + s] += p->box * (double)img[3 * s + k];
    free(img); free(cand); free(pi); free(save); free(tmp);
    if (stats) { stats[0] = n_att; stats[1] = n_empty; stats[2] = n_acc; }
    if (log_n) *log_n = nlog;
    return st;
}
