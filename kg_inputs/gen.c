/*
 * gen.c -- seeded synthetic melt generator (input data only).
 *
 * Holds none of the method's arithmetic: no potential, force, integrator or
 * Monte Carlo step.  Both the CUDA path and the oracle are fed its output.
 *
 * Recipe: chains are random walks with bond length `bond`; each new bond makes
 * angle theta with the previous one with cos(theta) drawn from a density
 * proportional to exp(kappa cos(theta)) on [-1, 1] and a uniform azimuth; the
 * first monomer of each chain is uniform in the periodic cube.  Monomers are
 * placed round-robin over chains (position index i for every chain, then
 * i + 1); a placement closer than d_min to any monomer already placed is
 * redrawn (d_min shrinks by 10% every 100 failed draws).  Velocities are
 * Maxwell-Boltzmann at temperature T with the total momentum removed.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood, OOPSLA 2014), a Weyl
 * sequence with increment 0x9E3779B97F4A7C15 followed by a 64-bit mixing
 * function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct { uint64_t w; } rng64;

static uint64_t next64(rng64 *r)
{
    uint64_t z = (r->w += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in [0, 1) with 53 bits */
static double unif(rng64 *r) { return (double)(next64(r) >> 11) * (1.0 / 9007199254740992.0); }

static double normal(rng64 *r)
{
    double u = 1.0 - unif(r), w = unif(r);
    return sqrt(-2.0 * log(u)) * cos(6.283185307179586 * w);
}

static double wrap(double a, double L) { return a - L * floor(a / L); }

typedef struct {
    int n;
    double h, L;
    int *head, *next;
    double *w;   /* wrapped positions, 3 per placed particle */
} grid_t;

static int cell_of(const grid_t *g, const double *w)
{
    int c[3];
    for (int d = 0; d < 3; ++d) {
        int k = (int)(w[d] / g->h);
        c[d] = k < 0 ? 0 : (k >= g->n ? g->n - 1 : k);
    }
    return (c[2] * g->n + c[1]) * g->n + c[0];
}

static int clear_of(const grid_t *g, const double *w, double dmin2)
{
    int c = cell_of(g, w), n = g->n;
    int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int nb = ((((cz + dz) % n + n) % n) * n + (((cy + dy) % n + n) % n)) * n + (((cx + dx) % n + n) % n);
                for (int t = g->head[nb]; t >= 0; t = g->next[t]) {
                    double r2 = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        double e = g->w[3 * t + d] - w[d];
                        e -= g->L * rint(e / g->L);
                        r2 += e * e;
                    }
                    if (r2 < dmin2) return 0;
                }
            }
    return 1;
}

/* x, v: (3, M) SoA outputs.  Returns 0 on success. */
int kgi_random_walk_melt(int nch, int N, double L, double kappa, unsigned long long seed, double bond,
                         double d_min, double T, double *x, double *v)
{
    const long M = (long)nch * N;
    rng64 r = {seed};
    grid_t g;
    g.L = L;
    g.n = (int)(L / (d_min > 0.5 ? d_min : 0.5));
    if (g.n < 3) g.n = 3;
    g.h = L / g.n;
    long ncell = (long)g.n * g.n * g.n;
    g.head = (int *)malloc(sizeof(int) * ncell);
    g.next = (int *)malloc(sizeof(int) * M);
    g.w = (double *)malloc(sizeof(double) * 3 * M);
    double *dir = (double *)calloc(3 * (size_t)nch, sizeof(double));
    if (!g.head || !g.next || !g.w || !dir) return 1;
    for (long c = 0; c < ncell; ++c) g.head[c] = -1;
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < nch; ++c) {
            const long s = (long)c * N + i;
            double cand[3], nd[3], w[3];
            for (int tries = 0;; ++tries) {
                if (i == 0) {
                    for (int d = 0; d < 3; ++d) cand[d] = unif(&r) * L;
                } else {
                    if (i == 1) {
                        double z = 2.0 * unif(&r) - 1.0, ph = 6.283185307179586 * unif(&r);
                        double s2 = sqrt(1.0 - z * z);
                        nd[0] = s2 * cos(ph); nd[1] = s2 * sin(ph); nd[2] = z;
                    } else {
                        const double *b = dir + 3 * c;
                        double u = unif(&r), ct;
                        ct = kappa < 1e-12 ? 2.0 * u - 1.0 : 1.0 + log(u + (1.0 - u) * exp(-2.0 * kappa)) / kappa;
                        if (ct > 1.0) ct = 1.0;
                        if (ct < -1.0) ct = -1.0;
                        double st = sqrt(1.0 - ct * ct), ph = 6.283185307179586 * unif(&r);
                        double a[3] = {0, 0, 0};
                        if (fabs(b[0]) < 0.9) a[0] = 1.0; else a[1] = 1.0;
                        double e1[3] = {b[1] * a[2] - b[2] * a[1], b[2] * a[0] - b[0] * a[2], b[0] * a[1] - b[1] * a[0]};
                        double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
                        for (int d = 0; d < 3; ++d) e1[d] /= n1;
                        double e2[3] = {b[1] * e1[2] - b[2] * e1[1], b[2] * e1[0] - b[0] * e1[2], b[0] * e1[1] - b[1] * e1[0]};
                        for (int d = 0; d < 3; ++d) nd[d] = ct * b[d] + st * (cos(ph) * e1[d] + sin(ph) * e2[d]);
                    }
                    for (int d = 0; d < 3; ++d) cand[d] = x[d * M + s - 1] + bond * nd[d];
                }
                for (int d = 0; d < 3; ++d) w[d] = wrap(cand[d], L);
                double dm = d_min * pow(0.9, (double)(tries / 100));
                if (d_min <= 0.0 || clear_of(&g, w, dm * dm)) break;
            }
            for (int d = 0; d < 3; ++d) {
                x[d * M + s] = cand[d];
                g.w[3 * s + d] = w[d];
            }
            if (i > 0) {
                double n2 = 0.0;
                for (int d = 0; d < 3; ++d) n2 += (cand[d] - x[d * M + s - 1]) * (cand[d] - x[d * M + s - 1]);
                for (int d = 0; d < 3; ++d) dir[3 * c + d] = (cand[d] - x[d * M + s - 1]) / sqrt(n2);
            }
            int cl = cell_of(&g, w);
            g.next[s] = g.head[cl];
            g.head[cl] = (int)s;
        }
    }
    double mean[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        for (long s = 0; s < M; ++s) {
            v[d * M + s] = sqrt(T) * normal(&r);
            mean[d] += v[d * M + s];
        }
        mean[d] /= (double)M;
        for (long s = 0; s < M; ++s) v[d * M + s] -= mean[d];
    }
    free(g.head); free(g.next); free(g.w); free(dir);
    return 0;
}
