// kg_ppa.cu -- primitive-path analysis (PPA) of one melt and the entanglement
// length of Eq. 22 (Sec. III).  The paper measures N_e by the PPA of Everaers
// et al. (Science 303, 823 (2004)) without restating it; the form taken here:
//   * both end monomers of every chain stay fixed;
//   * the non-bonded interaction, the n = 12 member of Eq. 5 (LJ 12-6
//     truncated and shifted at 2^(1/6)), acts only between monomers of
//     different chains; inside a chain it is off, 1-2 bonded pairs included,
//     so a bond keeps its FENE part alone (Eq. 10 without U_MLJ);
//   * no bending energy (Eq. 4 off);
//   * the energy is minimised by the path's integrator at T = 0, Langevin
//     velocity Verlet with zero noise (damped dynamics), from rest.
// It runs on a binary64 copy of the melt in slot order (chain-major, s = c N +
// i), (3, M) SoA x, v, F, and leaves the simulation state untouched.
//
// Neighbours: a Verlet list of interchain pairs within r_c + skin, entries
// j | q << IDX_BITS (q the stencil cell, which fixes the periodic image), stored
// column-major (entry k of monomer s at k M + s, so the loads of entry k by a
// warp are one coalesced row), rebuilt on the device whenever a monomer has
// moved more than skin / 2 since the last build (flag word 1).  Steps run as
// a captured CUDA graph of 25 steps, each step drift, a one-thread kernel that
// arms a conditional graph node with the build request, the node holding the
// build kernels, and the force kernel, the scheme of the MD graphs; steps
// outside whole graphs launch the build kernels directly, which return at once
// without a request.  The build bins monomers on a grid of
// n_c^3 cells of side h >= r_c + skin (n_c >= 3), keeps each monomer's binary32
// offset from its cell's corner, sorts every cell by slot (deterministic
// lists and sums) and tests candidates in binary32 on those offsets, with a
// margin that keeps every pair within r_c + skin: the list only has to
// contain the pairs, so its edge need not be exact.
//
// Two force kernels.  Binary64 (KG_FP64): minimum-image distances and forces
// in binary64, the same update order as the definition.  Mixed (KG_MIXED), the
// GB300 path, whose binary64 rate is a small fraction of its binary32 rate:
// the pair vector is (o_j + d_j) - (o_s + d_s) + q h in binary32, o the build
// offset and d the binary64 displacement since the build rounded to binary32,
// so every term is small and the vector is good to ~1e-7 sigma; bond vectors
// are binary64 differences rounded to binary32; forces, velocities and the
// kick are binary32 and the positions binary64, which they step by the
// binary32 increment dt v.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "kg_host.h"

namespace kg {

// kg_md.cu: exclusive scan of the cell counts, the scatter into cell order
// (with the records, w = slot) and the per-cell sort by slot
__global__ void k_scan1(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ bsum, int n,
                        const unsigned *__restrict__ flags);
__global__ void k_scan2(int *__restrict__ out, const int *__restrict__ bsum, int n, int nblk,
                        const unsigned *__restrict__ flags);
__global__ void k_scatter(const int *__restrict__ cellid, const int *__restrict__ rank,
                          const int *__restrict__ start, int *__restrict__ list, int M,
                          const unsigned *__restrict__ flags, const float4 *__restrict__ recb,
                          float4 *__restrict__ recs);
__global__ void k_cellsort(const int *__restrict__ start, int *__restrict__ list, float4 *__restrict__ recs,
                           int *__restrict__ count, int ncell, unsigned *__restrict__ flags);

namespace {

constexpr double PPA_RC = 1.122462048309373;   // 2^(1/6)
constexpr int PPA_MAXNB = 128;                  // list entries per monomer (overflow: capacity error)
constexpr int PPA_GRAPH_ITERS = 25;             // steps per captured graph
constexpr int PPA_BLOCK = 128;
constexpr int PPA_LAUNCHES_PER_ITER = 8;     // direct launches of one step
constexpr int PPA_BUILD_LAUNCHES = 6;        // kernels of one list build

struct PpaArgs {
    int M, N, nc, ncell;
    double L, invL, h, invh;     // box, 1/L, cell side and its inverse
    float hf, rl2f, rc2f;        // binary32 cell side, list radius^2 with margin, r_c^2
    double half_skin2;           // (skin / 2)^2
    double dt, gamma, k, R0sq;
    float dtf, gammaf, kf, invR0sqf, half_skin2f;
    double *x, *v, *F, *xb;      // (3, M) each; xb = positions at the last build (binary64 mode)
    float *v32, *F32;            // (3, M) velocities and forces of the mixed mode
    float4 *rec, *recs, *pg;     // build offsets + cell code; the same in cell order (w = slot); offsets + d
    float4 *dl;                  // mixed: displacement d since the build
    int *cellid, *rank, *count, *start, *list, *nn;
    unsigned *nl;                // entries j | q << IDX_BITS, column-major
    unsigned *flags;             // [0] error bits, [1] rebuild request, [2] builds
};

__device__ __forceinline__ bool fixed_end(const PpaArgs &a, int s)
{
    const int i = s % a.N;
    return i == 0 || i == a.N - 1;
}

__device__ __forceinline__ double min_image(double d, const PpaArgs &a)
{
    return __dsub_rn(d, __dmul_rn(a.L, rint(__dmul_rn(d, a.invL))));
}

// image shift q h of stencil code q = (dz + 1) 9 + (dy + 1) 3 + (dx + 1)
__device__ __forceinline__ float3 stencil_shift(unsigned q, float h)
{
    const int dx = (int)(q % 3u) - 1, dy = (int)((q / 3u) % 3u) - 1, dz = (int)(q / 9u) - 1;
    return make_float3((float)dx * h, (float)dy * h, (float)dz * h);
}

// first half kick and drift of the mobile monomers:
// v <- v + (dt/2) F; x <- x + dt v; request a rebuild past skin / 2
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_drift_f64(PpaArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.M || fixed_end(a, s)) return;
    const double hdt = 0.5 * a.dt;
    double dr2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * a.M + s;
        const double vh = __dadd_rn(a.v[o], __dmul_rn(hdt, a.F[o]));
        const double xn = __dadd_rn(a.x[o], __dmul_rn(a.dt, vh));
        a.v[o] = vh;
        a.x[o] = xn;
        const double e = xn - a.xb[o];
        dr2 += e * e;
    }
    if (!(dr2 <= a.half_skin2)) {
        if (!isfinite(dr2)) atomicOr(a.flags, ERR_NONFINITE);
        atomicOr(a.flags + 1, 1u);
    }
}

// mixed: the same step with binary32 v and F; the increment dt v (binary32)
// goes into the binary64 position and into the binary32 displacement d, and
// the gather record becomes o + d
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_drift_mixed(PpaArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.M || fixed_end(a, s)) return;
    const float hdt = 0.5f * a.dtf;
    const float4 d0 = a.dl[s];
    float dd[3] = {d0.x, d0.y, d0.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * a.M + s;
        const float vh = a.v32[o] + hdt * a.F32[o];
        const float inc = a.dtf * vh;
        a.v32[o] = vh;
        a.x[o] += (double)inc;
        dd[d] += inc;
    }
    a.dl[s] = make_float4(dd[0], dd[1], dd[2], 0.f);
    const float4 r = a.rec[s];
    a.pg[s] = make_float4(r.x + dd[0], r.y + dd[1], r.z + dd[2], r.w);
    const float dr2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    if (!(dr2 <= a.half_skin2f)) {
        if (!isfinite(dr2)) atomicOr(a.flags, ERR_NONFINITE);
        atomicOr(a.flags + 1, 1u);
    }
}

// cell of each monomer from its wrapped position; the build record (offset
// from the cell's corner, cell code), the gather record and the build position
__global__ void __launch_bounds__(256) k_ppa_bin(PpaArgs a)
{
    if (!a.flags[1] || a.flags[0]) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.M) return;
    int cc[3];
    float off[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double xd = a.x[(size_t)d * a.M + s];
        const double w = xd - a.L * floor(xd * a.invL);
        int q = (int)(w * a.invh);
        q = q < 0 ? 0 : (q >= a.nc ? a.nc - 1 : q);
        cc[d] = q;
        off[d] = (float)(w - (double)q * a.h);
        if (a.xb) a.xb[(size_t)d * a.M + s] = xd;
    }
    const float4 r = make_float4(off[0], off[1], off[2], __uint_as_float(pack_code(cc[0], cc[1], cc[2])));
    a.rec[s] = r;
    a.pg[s] = r;
    a.dl[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int c = (cc[2] * a.nc + cc[1]) * a.nc + cc[0];
    a.cellid[s] = c;
    a.rank[s] = atomicAdd(a.count + c, 1);
}

// interchain Verlet list of monomer s from the binary32 build offsets: every t
// of another chain in the 27 cells around s whose vector o_t - o_s + q h is
// shorter than r_c + skin (plus a margin above the offsets' rounding)
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_nlist(PpaArgs a)
{
    if (!a.flags[1] || a.flags[0]) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.M) return;
    const float4 rs = a.rec[s];
    const unsigned code = __float_as_uint(rs.w);
    const int cx = (int)(code & CODE_MASK), cy = (int)((code >> CODE_BITS) & CODE_MASK),
              cz = (int)(code >> (2 * CODE_BITS));
    const unsigned c0 = (unsigned)(s - s % a.N);     // first slot of the chain of s
    int n = 0;
    unsigned q = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = (cz + dz + a.nc) % a.nc;
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = (cy + dy + a.nc) % a.nc;
            for (int dx = -1; dx <= 1; ++dx, ++q) {
                const int c = (z * a.nc + y) * a.nc + (cx + dx + a.nc) % a.nc;
                const float sx = (float)dx * a.hf - rs.x, sy = (float)dy * a.hf - rs.y, sz = (float)dz * a.hf - rs.z;
                const int p1 = a.start[c + 1];
                for (int p = a.start[c]; p < p1; ++p) {
                    const float4 rj = a.recs[p];
                    const int j = __float_as_int(rj.w);
                    if ((unsigned)j - c0 < (unsigned)a.N) continue;   // same chain
                    const float ex = rj.x + sx, ey = rj.y + sy, ez = rj.z + sz;
                    if (ex * ex + ey * ey + ez * ez < a.rl2f) {
                        if (n < PPA_MAXNB) a.nl[(size_t)n * a.M + s] = (unsigned)j | (q << IDX_BITS);
                        ++n;
                    }
                }
            }
        }
    }
    if (n > PPA_MAXNB) {
        atomicOr(a.flags, ERR_NL_CAPACITY);
        n = PPA_MAXNB;
    }
    a.nn[s] = n;
}

// FENE force of the two bonds of mobile monomer s (binary64, unwrapped)
__device__ __forceinline__ void bond_forces(const PpaArgs &a, int s, double xs, double ys, double zs, double &fx,
                                            double &fy, double &fz)
{
    const size_t M = a.M;
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
        const int t = s + side;
        const double bx = __dsub_rn(a.x[t], xs), by = __dsub_rn(a.x[M + t], ys), bz = __dsub_rn(a.x[2 * M + t], zs);
        const double q = __dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz)) / a.R0sq;
        if (!(q < 1.0)) {
            atomicOr(a.flags, ERR_OVERSTRETCH);
            continue;
        }
        const double gb = a.k / (1.0 - q);
        fx += gb * bx;
        fy += gb * by;
        fz += gb * bz;
    }
}

// F <- F_c(x) - gamma v; v <- v + half dt F (half = 0 for the first force)
__device__ __forceinline__ void kick(const PpaArgs &a, int s, double fx, double fy, double fz, double half)
{
    const double hdt = half * a.dt;
    const double f[3] = {fx, fy, fz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * a.M + s;
        const double vh = a.v[o];
        const double Ft = __dsub_rn(f[d], __dmul_rn(a.gamma, vh));
        a.F[o] = Ft;
        a.v[o] = __dadd_rn(vh, __dmul_rn(hdt, Ft));
    }
}

// the thread of monomer 0 retires the build request of this step (every build
// kernel has run) and counts the build
__device__ __forceinline__ void retire_build(const PpaArgs &a, int s)
{
    if (s == 0 && a.flags[1]) {
        if (!a.flags[0]) a.flags[2] += 1u;
        a.flags[1] = 0u;
    }
}

// binary64 force: minimum-image pair vectors, LJ 12-6 between chains
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_force_f64(PpaArgs a, double half)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    retire_build(a, s);
    if (s >= a.M || fixed_end(a, s)) return;
    const size_t M = a.M;
    const double xs = a.x[s], ys = a.x[M + s], zs = a.x[2 * M + s];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    const int n = a.nn[s];
    const double rc2 = PPA_RC * PPA_RC;
    for (int k = 0; k < n; ++k) {
        const int j = (int)(a.nl[(size_t)k * M + s] & IDX_MASK);
        const double ex = min_image(__dsub_rn(a.x[j], xs), a);
        const double ey = min_image(__dsub_rn(a.x[M + j], ys), a);
        const double ez = min_image(__dsub_rn(a.x[2 * M + j], zs), a);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
        if (r2 < rc2) {
            const double ir2 = 1.0 / r2;
            const double ir6 = ir2 * ir2 * ir2;
            const double g = (48.0 * ir6 * ir6 - 24.0 * ir6) * ir2;   // -U'(r)/r, U = 4(r^-12 - r^-6) + 1
            fx -= g * ex;
            fy -= g * ey;
            fz -= g * ez;
        }
    }
    bond_forces(a, s, xs, ys, zs, fx, fy, fz);
    kick(a, s, fx, fy, fz, half);
}

// mixed force: binary32 pair vectors from the gather records and binary32
// LJ 12-6; bond vectors are binary64 differences rounded to binary32, the
// FENE force, friction and kick binary32
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_force_mixed(PpaArgs a, float half)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    retire_build(a, s);
    if (s >= a.M || fixed_end(a, s)) return;
    const size_t M = a.M;
    const float4 ps = a.pg[s];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int n = a.nn[s];
    auto pair = [&](unsigned e, float4 pj) {
        const float3 sh = stencil_shift(e >> IDX_BITS, a.hf);
        const float ex = (pj.x - ps.x) + sh.x, ey = (pj.y - ps.y) + sh.y, ez = (pj.z - ps.z) + sh.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < a.rc2f) {
            const float ir2 = __frcp_rn(r2);
            const float ir6 = ir2 * ir2 * ir2;
            const float g = (48.f * ir6 * ir6 - 24.f * ir6) * ir2;   // -U'(r)/r, U = 4(r^-12 - r^-6) + 1
            fx -= g * ex;
            fy -= g * ey;
            fz -= g * ez;
        }
    };
    // four entries in flight: their list words, then their gathers, then the arithmetic
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        unsigned e[4];
        float4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = __ldg(a.nl + (size_t)(k + u) * M + s);
#pragma unroll
        for (int u = 0; u < 4; ++u) pj[u] = __ldg(a.pg + (e[u] & IDX_MASK));
#pragma unroll
        for (int u = 0; u < 4; ++u) pair(e[u], pj[u]);
    }
    for (; k < n; ++k) {
        const unsigned e = __ldg(a.nl + (size_t)k * M + s);
        pair(e, __ldg(a.pg + (e & IDX_MASK)));
    }
    const double xs = a.x[s], ys = a.x[M + s], zs = a.x[2 * M + s];
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
        const int t = s + side;
        const float bx = (float)(a.x[t] - xs), by = (float)(a.x[M + t] - ys), bz = (float)(a.x[2 * M + t] - zs);
        const float q = (bx * bx + by * by + bz * bz) * a.invR0sqf;
        if (!(q < 1.f)) {
            atomicOr(a.flags, ERR_OVERSTRETCH);
            continue;
        }
        const float gb = a.kf * __frcp_rn(1.f - q);
        fx += gb * bx;
        fy += gb * by;
        fz += gb * bz;
    }
    const float hdt = half * a.dtf;
    const float f[3] = {fx, fy, fz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * M + s;
        const float vh = a.v32[o];
        const float Ft = f[d] - a.gammaf * vh;
        a.F32[o] = Ft;
        a.v32[o] = vh + hdt * Ft;
    }
}

// contour length of every chain (bond order) and the largest net force on a mobile monomer
__global__ void __launch_bounds__(256) k_ppa_lengths(PpaArgs a, double *__restrict__ lpp,
                                                    unsigned long long *__restrict__ fmax_bits)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.M / a.N) return;
    const size_t M = a.M;
    double sum = 0.0, f2max = 0.0;
    for (int i = 0; i + 1 < a.N; ++i) {
        const size_t s = (size_t)c * a.N + i;
        const double bx = __dsub_rn(a.x[s + 1], a.x[s]);
        const double by = __dsub_rn(a.x[M + s + 1], a.x[M + s]);
        const double bz = __dsub_rn(a.x[2 * M + s + 1], a.x[2 * M + s]);
        sum += sqrt(__dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz)));
        if (i > 0) {
            double f[3];
            for (int d = 0; d < 3; ++d) f[d] = a.F32 ? (double)a.F32[d * M + s] : a.F[d * M + s];
            const double f2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
            f2max = f2 > f2max ? f2 : f2max;
        }
    }
    lpp[c] = sum;
    atomicMax(fmax_bits, (unsigned long long)__double_as_longlong(sqrt(f2max)));
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// the conditional list build (each kernel returns at once unless flag word 1 is set)
void enqueue_build(const PpaArgs &a, cudaStream_t st, int *bsum)
{
    const int nbs = nblk(a.ncell, 1024);
    k_ppa_bin<<<nblk(a.M, 256), 256, 0, st>>>(a);
    k_scan1<<<nbs, 1024, 0, st>>>(a.count, a.start, bsum, a.ncell, a.flags);
    k_scan2<<<nbs, 1024, 0, st>>>(a.start, bsum, a.ncell, nbs, a.flags);
    k_scatter<<<nblk(a.M, 256), 256, 0, st>>>(a.cellid, a.rank, a.start, a.list, a.M, a.flags, a.rec, a.recs);
    k_cellsort<<<nblk(a.ncell, 256), 256, 0, st>>>(a.start, a.list, a.recs, a.count, a.ncell, a.flags);
    k_ppa_nlist<<<nblk(a.M, PPA_BLOCK), PPA_BLOCK, 0, st>>>(a);
}

void enqueue_force(const PpaArgs &a, cudaStream_t st, bool mixed, double half)
{
    const int nbm = nblk(a.M, PPA_BLOCK);
    if (mixed) k_ppa_force_mixed<<<nbm, PPA_BLOCK, 0, st>>>(a, (float)half);
    else k_ppa_force_f64<<<nbm, PPA_BLOCK, 0, st>>>(a, half);
}

void enqueue_step(const PpaArgs &a, cudaStream_t st, int *bsum, bool mixed)
{
    const int nbm = nblk(a.M, PPA_BLOCK);
    if (mixed) k_ppa_drift_mixed<<<nbm, PPA_BLOCK, 0, st>>>(a);
    else k_ppa_drift_f64<<<nbm, PPA_BLOCK, 0, st>>>(a);
    enqueue_build(a, st, bsum);
    enqueue_force(a, st, mixed, 0.5);
}

// arms the conditional build node of a captured step with the build request
__global__ void k_ppa_arm(const unsigned *__restrict__ flags, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, (flags[1] && !flags[0]) ? 1u : 0u);
}

// A graph of PPA_GRAPH_ITERS steps: drift, the arm kernel, a conditional node
// holding the list build (run only when a monomer has left its skin), force.
bool capture_steps(const PpaArgs &a, cudaStream_t s1, cudaStream_t s2, int *bsum, bool mixed,
                   cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = cudaStreamBeginCaptureToGraph(s1, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
              cudaSuccess;
    const int nbm = nblk(a.M, PPA_BLOCK);
    for (int i = 0; ok && i < PPA_GRAPH_ITERS; ++i) {
        if (mixed) k_ppa_drift_mixed<<<nbm, PPA_BLOCK, 0, s1>>>(a);
        else k_ppa_drift_f64<<<nbm, PPA_BLOCK, 0, s1>>>(a);
        cudaGraphConditionalHandle h;
        ok = cudaGraphConditionalHandleCreate(&h, g, 0, 0) == cudaSuccess;
        if (!ok) break;
        k_ppa_arm<<<1, 1, 0, s1>>>(a.flags, h);
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        ok = cudaStreamGetCaptureInfo(s1, &cs, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess;
        if (!ok) break;
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        ok = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp) == cudaSuccess &&
             cudaStreamUpdateCaptureDependencies(s1, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                 cudaSuccess;
        if (!ok) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (!ok) break;
        enqueue_build(a, s2, bsum);
        ok = cudaStreamEndCapture(s2, &body) == cudaSuccess;
        if (!ok) break;
        enqueue_force(a, s1, mixed, 0.5);
    }
    cudaGraph_t g_out = nullptr;
    const bool ended = cudaStreamEndCapture(s1, &g_out) == cudaSuccess;
    ok = ok && ended && cudaGetLastError() == cudaSuccess && cudaGraphInstantiate(out, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        *out = nullptr;
    }
    return ok;
}

// Eq. 22's left-hand side (2 x + exp(-2 x) - 1) / (2 x^2); a series below
// x = 1e-3, where the closed form cancels
double eq22_lhs(double x)
{
    if (x < 1e-3) return 1.0 - 2.0 * x / 3.0 + x * x / 3.0 - 2.0 * x * x * x / 15.0;
    return (2.0 * x + std::expm1(-2.0 * x)) / (2.0 * x * x);
}

}  // namespace
}  // namespace kg

using namespace kg;

extern "C" {

kg_status kg_primitive_path(kg_ctx *c, int melt, const kg_ppa_params *pp, double *lpp, double *x_out,
                            kg_ppa_result *res)
{
    if (!c || !pp || melt < 0 || melt >= c->sim.n_melts) return KG_ERR_INVALID_ARG;
    if (!(pp->dt > 0.0) || !(pp->gamma >= 0.0) || !(pp->skin > 0.0) || pp->n_iter < 0) return KG_ERR_INVALID_ARG;
    if (pp->precision != KG_FP64 && pp->precision != KG_MIXED) return KG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    const MeltDev &md = c->sim.melt[melt];
    const double rl = PPA_RC + pp->skin;
    const int nc = (int)std::floor(md.L / rl);
    if (nc < 3 || nc > CODE_MASK + 1) return KG_ERR_INVALID_ARG;   // 27 distinct stencil cells; packed codes
    const bool mixed = pp->precision == KG_MIXED;
    const double k = pp->k_fene > 0.0 ? pp->k_fene : kg_kn(12.0, c->p.R0, c->p.l0);
    const int M = md.M, N = md.N, n_ch = md.n_ch;

    PpaArgs a{};
    a.M = M;
    a.N = N;
    a.nc = nc;
    a.ncell = nc * nc * nc;
    a.L = md.L;
    a.invL = 1.0 / md.L;
    a.h = md.L / nc;
    a.invh = nc / md.L;
    a.hf = (float)a.h;
    a.rl2f = (float)(rl * rl) + 1e-4f;          // margin >> the binary32 error of the offsets
    a.rc2f = (float)(PPA_RC * PPA_RC);
    a.half_skin2 = 0.25 * pp->skin * pp->skin;
    a.dt = pp->dt;
    a.gamma = pp->gamma;
    a.k = k;
    a.R0sq = c->p.R0 * c->p.R0;
    a.dtf = (float)pp->dt;
    a.gammaf = (float)pp->gamma;
    a.kf = (float)k;
    a.invR0sqf = (float)(1.0 / a.R0sq);
    a.half_skin2f = (float)a.half_skin2;

    const size_t m3 = 3 * (size_t)M;
    const int nbs = nblk(a.ncell, 1024);
    std::vector<void *> bufs;
    auto get = [&](size_t bytes) {
        void *p = dev_alloc(c, bytes);
        bufs.push_back(p);
        return p;
    };
    a.x = (double *)get(sizeof(double) * m3);
    if (mixed) {
        a.v32 = (float *)get(sizeof(float) * m3);
        a.F32 = (float *)get(sizeof(float) * m3);
    } else {
        a.v = (double *)get(sizeof(double) * m3);
        a.F = (double *)get(sizeof(double) * m3);
        a.xb = (double *)get(sizeof(double) * m3);
    }
    a.dl = (float4 *)get(sizeof(float4) * M);
    a.rec = (float4 *)get(sizeof(float4) * M);
    a.recs = (float4 *)get(sizeof(float4) * M);
    a.pg = (float4 *)get(sizeof(float4) * M);
    a.cellid = (int *)get(sizeof(int) * M);
    a.rank = (int *)get(sizeof(int) * M);
    a.count = (int *)get(sizeof(int) * ((size_t)a.ncell + 1));
    a.start = (int *)get(sizeof(int) * ((size_t)a.ncell + 1));
    a.list = (int *)get(sizeof(int) * M);
    a.nl = (unsigned *)get(sizeof(unsigned) * (size_t)PPA_MAXNB * M);
    a.nn = (int *)get(sizeof(int) * M);
    a.flags = (unsigned *)get(sizeof(unsigned) * 4);
    int *bsum = (int *)get(sizeof(int) * (size_t)nbs);
    double *d_lpp = (double *)get(sizeof(double) * n_ch);
    unsigned long long *d_fmax = (unsigned long long *)get(sizeof(unsigned long long));
    cudaStream_t gs = nullptr, gs2 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    auto done = [&](kg_status r) {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gs) cudaStreamDestroy(gs);
        if (gs2) cudaStreamDestroy(gs2);
        cudaStreamSynchronize(c->stream);
        for (void *p : bufs) dev_free(c, p);
        return r;
    };
    for (void *p : bufs)
        if (!p) return done(KG_ERR_OOM);

    cudaStream_t st = c->stream;
    kg::to_slots(c, melt, c->x, a.x, 3);               // (3, M) slot order, unwrapped
    static const unsigned one = 1u;
    if (cudaMemcpyAsync(a.flags + 1, &one, sizeof(unsigned), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return done(KG_ERR_CUDA);
    // the first list and force, from rest (v = 0, no kick)
    enqueue_build(a, st, bsum);
    enqueue_force(a, st, mixed, 0.0);
    c->launches += 7;
    long long left = pp->n_iter, graph_steps = 0;
    if (left >= 2 * PPA_GRAPH_ITERS && cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamCreateWithFlags(&gs2, cudaStreamNonBlocking) == cudaSuccess &&
        capture_steps(a, gs, gs2, bsum, mixed, &gexec)) {
        for (; left >= PPA_GRAPH_ITERS; left -= PPA_GRAPH_ITERS, graph_steps += PPA_GRAPH_ITERS)
            if (cudaGraphLaunch(gexec, st) != cudaSuccess) return done(KG_ERR_CUDA);
    }
    c->launches += 3 * graph_steps + PPA_LAUNCHES_PER_ITER * left;   // + the graphs' builds, below
    for (; left > 0; --left) enqueue_step(a, st, bsum, mixed);
    k_ppa_lengths<<<nblk(n_ch, 256), 256, 0, st>>>(a, d_lpp, d_fmax);
    ++c->launches;
    if (cudaGetLastError() != cudaSuccess) return done(KG_ERR_CUDA);

    std::vector<double> h_lpp((size_t)n_ch);
    unsigned h_flags[4] = {0, 0, 0, 0};
    unsigned long long h_fmax = 0;
    if (cudaMemcpyAsync(h_lpp.data(), d_lpp, sizeof(double) * n_ch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_flags, a.flags, sizeof(h_flags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_fmax, d_fmax, sizeof(h_fmax), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return done(KG_ERR_CUDA);
    if (x_out && cudaMemcpyAsync(x_out, a.x, sizeof(double) * m3, cudaMemcpyDefault, st) != cudaSuccess)
        return done(KG_ERR_CUDA);
    if (cudaStreamSynchronize(st) != cudaSuccess) return done(KG_ERR_CUDA);
    if (graph_steps) c->launches += PPA_BUILD_LAUNCHES * (long long)h_flags[2];   // upper bound: all builds
    const unsigned e = h_flags[0];
    if (e & ERR_OVERSTRETCH) return done(KG_ERR_BOND_OVERSTRETCH);
    if (e & ERR_NONFINITE) return done(KG_ERR_NONFINITE);
    if (e & ERR_NL_CAPACITY) return done(KG_ERR_CAPACITY);
    if (lpp)
        for (int i = 0; i < n_ch; ++i) lpp[i] = h_lpp[(size_t)i];
    if (res) {
        double sum = 0.0;
        for (double v : h_lpp) sum += v;               // chain order
        res->lpp_mean = sum / (double)n_ch;
        std::memcpy(&res->fmax, &h_fmax, sizeof(double));
        res->builds = (long long)h_flags[2];
    }
    return done(KG_OK);
}

kg_status kg_entanglement_length(double lpp_mean, int chain_len, double l0, double l_k, double *n_ek, double *n_e)
{
    if (!n_ek || chain_len < 2 || !(l0 > 0.0) || !(lpp_mean > 0.0)) return KG_ERR_INVALID_ARG;
    const double r = lpp_mean / ((double)(chain_len - 1) * l0);
    const double y = r * r;
    if (!(y > 0.0 && y < 1.0)) return KG_ERR_INVALID_ARG;
    // the left-hand side falls monotonically from 1 to 0: bisection in log x
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (eq22_lhs(std::exp(mid)) > y) lo = mid;
        else hi = mid;
    }
    *n_ek = std::exp(0.5 * (lo + hi));
    if (n_e) {
        if (!(l_k > 0.0)) return KG_ERR_INVALID_ARG;
        *n_e = *n_ek * l_k / l0;
    }
    return KG_OK;
}

}  // extern "C"
