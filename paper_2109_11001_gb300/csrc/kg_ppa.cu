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
// It runs on a copy of the melt and leaves the simulation state untouched.
//
// Storage.  The copy lives in cell order: every list build bins the monomers
// on a grid of n_c^3 cells of side h >= r_c + skin (n_c >= 3), sorts them by
// cell (a counting sort, each cell's run ordered by the previous storage index,
// so the order is deterministic) and moves every per-monomer array into that
// order, double-buffered with the buffer in use named by flag word 3.  A
// cell's monomers are then one contiguous run of storage indices, the 32
// monomers of a warp sit in a few neighbouring cells, and the candidate
// loads of the build and the neighbour gathers of the force kernel stay in
// L1 and L2.  Bonds reach their partners through a partner-index array
// refreshed at each build; results return to slot order (chain-major, s = c N
// + i) at the end.
//
// Neighbours: a Verlet list of interchain pairs within r_c + skin, entries
// j | q << IDX_BITS (j a storage index, q the stencil cell, which fixes the
// periodic image), column-major (entry k of monomer p at k M + p, so the loads
// of entry k by a warp are one coalesced row), rebuilt whenever a monomer has
// moved more than skin / 2 since the last build (flag word 1).  Candidates are
// tested in binary32 on the monomers' offsets from their cells' corners, with
// a margin that keeps every pair within r_c + skin: the list only has to
// contain the pairs, so its edge need not be exact.  Steps run as a captured
// CUDA graph of 25 steps, each step drift, a one-thread kernel that arms a
// conditional graph node with the build request, the node holding the build
// kernels, and the force kernel, the scheme of the MD graphs; steps outside
// whole graphs launch the build kernels directly, which return at once without
// a request.
//
// Two force kernels.  Binary64 (KG_FP64): minimum-image distances and forces
// in binary64, the same update order as the definition.  Mixed (KG_MIXED), the
// GB300 path, whose binary64 rate is a small fraction of its binary32 rate:
// the pair vector is (o_j + d_j) - (o_p + d_p) + q h in binary32, o the build
// offset and d the displacement since the build, so every term is small and
// the vector is good to ~1e-7 sigma.  The binary64 position is touched only
// at a build: between builds a monomer's position is its binary64 build
// position plus d, and every step runs in binary32 (a bond vector is its
// build value, a binary64 difference rounded to binary32, plus the
// difference of the two displacements); the build folds d into the binary64
// position.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "kg_host.h"

namespace kg {

// kg_md.cu: exclusive scan of the cell counts
__global__ void k_scan1(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ bsum, int n,
                        const unsigned *__restrict__ flags);
__global__ void k_scan2(int *__restrict__ out, const int *__restrict__ bsum, int n, int nblk,
                        const unsigned *__restrict__ flags);

namespace {

constexpr double PPA_RC = 1.122462048309373;   // 2^(1/6)
constexpr int PPA_MAXNB = 128;                  // list entries per monomer (overflow: capacity error)
constexpr int PPA_CELL_CAP = 1024;              // monomers per cell the build accepts
constexpr int PPA_GRAPH_ITERS = 25;             // steps per captured graph
constexpr int PPA_BLOCK = 128;
constexpr unsigned FIXED_BIT = 0x80000000u;     // record word w: chain index | FIXED_BIT at a chain end

struct PpaArgs {
    int M, N, nc, ncell;
    double L, invL, h, invh;     // box, 1/L, cell side and its inverse
    float hf, rl2f, rc2f;        // binary32 cell side, list radius^2 with margin, r_c^2
    double half_skin2;           // (skin / 2)^2
    double dt, gamma, k, R0sq;
    float dtf, gammaf, kf, invR0sqf, half_skin2f;
    // double-buffered per-monomer state (storage order), buffer flags[3] in use
    double *x0, *x1;             // (3, M) positions (mixed: positions at the last build)
    double *v0, *v1, *F0, *F1;   // (3, M) velocities and forces, binary64 mode
    float *u0, *u1, *G0, *G1;    // (3, M) velocities and forces, mixed mode
    int *slot0, *slot1;          // storage index -> slot
    // single-buffered, rewritten at each build (storage order of the new buffer)
    double *xb;                  // positions at the build (binary64 mode)
    float4 *rec, *pg, *dl;       // build offset + (chain | FIXED_BIT); offset + d; d
    float4 *off;                 // bin output in the old order: offset + cell index
    float4 *bvec;                // mixed: bond vector to the next monomer at the build
    int2 *bp;                    // storage indices of the bonded partners (-1 past an end)
    int *pos_of;                 // slot -> storage index
    int *cellof;                 // packed cell coordinates of each storage index
    int *rank, *count, *start, *list, *nn;
    unsigned *nl;                // entries j | q << IDX_BITS, column-major
    unsigned *flags;             // [0] error bits, [1] rebuild request, [2] builds, [3] buffer in use
};

__device__ __forceinline__ int cur_buf(const PpaArgs &a) { return (int)(a.flags[3] & 1u); }
__device__ __forceinline__ bool build_requested(const PpaArgs &a) { return a.flags[1] && !a.flags[0]; }

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

__device__ __forceinline__ bool is_fixed(const float4 &r) { return (__float_as_uint(r.w) & FIXED_BIT) != 0u; }

// ---- one step: drift, (conditional) build, force ----

// first half kick and drift of the mobile monomers:
// v <- v + (dt/2) F; x <- x + dt v; request a rebuild past skin / 2
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_drift_f64(PpaArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.M || is_fixed(a.rec[p])) return;
    const int cb = cur_buf(a);
    double *x = cb ? a.x1 : a.x0, *v = cb ? a.v1 : a.v0;
    const double *F = cb ? a.F1 : a.F0;
    const double hdt = 0.5 * a.dt;
    double dr2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * a.M + p;
        const double vh = __dadd_rn(v[o], __dmul_rn(hdt, F[o]));
        const double xn = __dadd_rn(x[o], __dmul_rn(a.dt, vh));
        v[o] = vh;
        x[o] = xn;
        const double e = xn - a.xb[o];
        dr2 += e * e;
    }
    if (!(dr2 <= a.half_skin2)) {
        if (!isfinite(dr2)) atomicOr(a.flags, ERR_NONFINITE);
        atomicOr(a.flags + 1, 1u);
    }
}

// mixed: the same step with binary32 v and F; the drift goes into the
// binary32 displacement d since the build, and the gather record becomes o + d
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_drift_mixed(PpaArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.M) return;
    const float4 r = a.rec[p];
    if (is_fixed(r)) return;
    const int cb = cur_buf(a);
    float *u = cb ? a.u1 : a.u0;
    const float *G = cb ? a.G1 : a.G0;
    const float hdt = 0.5f * a.dtf;
    const float4 d0 = a.dl[p];
    float dd[3] = {d0.x, d0.y, d0.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * a.M + p;
        const float vh = u[o] + hdt * G[o];
        u[o] = vh;
        dd[d] += a.dtf * vh;
    }
    a.dl[p] = make_float4(dd[0], dd[1], dd[2], 0.f);
    a.pg[p] = make_float4(r.x + dd[0], r.y + dd[1], r.z + dd[2], r.w);
    const float dr2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    if (!(dr2 <= a.half_skin2f)) {
        if (!isfinite(dr2)) atomicOr(a.flags, ERR_NONFINITE);
        atomicOr(a.flags + 1, 1u);
    }
}

// build 1: cell of each monomer (current order) from its wrapped position,
// its offset from the cell's corner and its rank in the cell; mixed: the
// displacement d is folded into the binary64 position here, each thread on
// its own monomer (the permutation then reads positions only)
__global__ void __launch_bounds__(256) k_ppa_bin(PpaArgs a)
{
    if (!build_requested(a)) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.M) return;
    double *x = cur_buf(a) ? a.x1 : a.x0;
    const float4 dp = a.u0 ? a.dl[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float dd[3] = {dp.x, dp.y, dp.z};
    int cc[3];
    float o[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double xd = x[(size_t)d * a.M + p];
        if (a.u0) {                                    // mixed: fold d into the binary64 position
            xd += (double)dd[d];
            x[(size_t)d * a.M + p] = xd;
        }
        cc[d] = cell_of(xd, a.h, a.invh, a.nc, o[d]);
    }
    const int c = (cc[2] * a.nc + cc[1]) * a.nc + cc[0];
    a.off[p] = make_float4(o[0], o[1], o[2], __int_as_float(c));
    a.rank[p] = atomicAdd(a.count + c, 1);
}

// build 2: the current storage indices in cell order
__global__ void __launch_bounds__(256) k_ppa_scatter(PpaArgs a)
{
    if (!build_requested(a)) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.M) return;
    a.list[a.start[__float_as_int(a.off[p].w)] + a.rank[p]] = p;
}

// build 3: each cell's run ordered by current storage index (deterministic);
// clear the counts for the next build
__global__ void __launch_bounds__(256) k_ppa_cellsort(PpaArgs a)
{
    if (!build_requested(a)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    const int b0 = a.start[c], b1 = a.start[c + 1];
    a.count[c] = 0;
    if (b1 - b0 > PPA_CELL_CAP) {
        atomicOr(a.flags, ERR_NL_CAPACITY);
        return;
    }
    for (int k = b0 + 1; k < b1; ++k) {
        const int v = a.list[k];
        int j = k - 1;
        while (j >= b0 && a.list[j] > v) {
            a.list[j + 1] = a.list[j];
            --j;
        }
        a.list[j + 1] = v;
    }
}

// build 4: move every per-monomer array into cell order (the other buffer);
// the records, displacement, build positions and slot -> storage map
__global__ void __launch_bounds__(256) k_ppa_permute(PpaArgs a)
{
    if (!build_requested(a)) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.M) return;
    const int cb = cur_buf(a);
    const int p = a.list[q];
    const size_t M = a.M;
    const double *xs = cb ? a.x1 : a.x0;
    double *xd = cb ? a.x0 : a.x1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double xv = xs[d * M + p];
        xd[d * M + q] = xv;
        if (a.xb) a.xb[d * M + q] = xv;
    }
    if (a.u0) {
        const float *us = cb ? a.u1 : a.u0, *Gs = cb ? a.G1 : a.G0;
        float *ud = cb ? a.u0 : a.u1, *Gd = cb ? a.G0 : a.G1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ud[d * M + q] = us[d * M + p];
            Gd[d * M + q] = Gs[d * M + p];
        }
    } else {
        const double *vs = cb ? a.v1 : a.v0, *Fs = cb ? a.F1 : a.F0;
        double *vd = cb ? a.v0 : a.v1, *Fd = cb ? a.F0 : a.F1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vd[d * M + q] = vs[d * M + p];
            Fd[d * M + q] = Fs[d * M + p];
        }
    }
    const int s = (cb ? a.slot1 : a.slot0)[p];
    (cb ? a.slot0 : a.slot1)[q] = s;
    a.pos_of[s] = q;
    const int i = s % a.N;
    const unsigned w = (unsigned)(s / a.N) | ((i == 0 || i == a.N - 1) ? FIXED_BIT : 0u);
    const float4 o = a.off[p];
    const float4 r = make_float4(o.x, o.y, o.z, __uint_as_float(w));
    a.rec[q] = r;
    a.pg[q] = r;
    a.dl[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int c = __float_as_int(o.w);
    a.cellof[q] = (int)pack_code(c % a.nc, (c / a.nc) % a.nc, c / (a.nc * a.nc));
}

// build 5 (one thread): the new buffer becomes the one in use
__global__ void k_ppa_flip(PpaArgs a)
{
    if (build_requested(a)) a.flags[3] ^= 1u;
}

// build 6: storage indices of each monomer's bonded partners; mixed: the
// bond vector to the next monomer (binary64 difference rounded to binary32)
__global__ void __launch_bounds__(256) k_ppa_partners(PpaArgs a)
{
    if (!build_requested(a)) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.M) return;
    const int cb = cur_buf(a);
    const int s = (cb ? a.slot1 : a.slot0)[p];
    const int i = s % a.N;
    const int2 b = make_int2(i > 0 ? a.pos_of[s - 1] : -1, i < a.N - 1 ? a.pos_of[s + 1] : -1);
    a.bp[p] = b;
    if (a.bvec && b.y >= 0) {
        const double *x = cb ? a.x1 : a.x0;
        const size_t M = a.M;
        a.bvec[p] = make_float4((float)(x[b.y] - x[p]), (float)(x[M + b.y] - x[M + p]),
                                (float)(x[2 * M + b.y] - x[2 * M + p]), 0.f);
    }
}

// build 7: interchain Verlet list of monomer p from the binary32 build
// offsets: every t of another chain in the 27 cells around p whose vector
// o_t - o_p + q h is shorter than r_c + skin (plus a margin above the offsets'
// rounding)
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_nlist(PpaArgs a)
{
    if (!build_requested(a)) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.M) return;
    const float4 rp = a.rec[p];
    const unsigned chain = __float_as_uint(rp.w) & ~FIXED_BIT;
    const unsigned code = (unsigned)a.cellof[p];
    const int cx = (int)(code & CODE_MASK), cy = (int)((code >> CODE_BITS) & CODE_MASK),
              cz = (int)(code >> (2 * CODE_BITS));
    const int nc = a.nc;
    auto wrap = [nc](int v) { return v < 0 ? v + nc : (v >= nc ? v - nc : v); };
    int n = 0;
    unsigned q = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = wrap(cz + dz);
        for (int dy = -1; dy <= 1; ++dy) {
            const int zy = (z * nc + wrap(cy + dy)) * nc;
            for (int dx = -1; dx <= 1; ++dx, ++q) {
                const int cn = zy + wrap(cx + dx);
                const float sx = (float)dx * a.hf - rp.x, sy = (float)dy * a.hf - rp.y, sz = (float)dz * a.hf - rp.z;
                const int j1 = __ldg(a.start + cn + 1);
                for (int j = __ldg(a.start + cn); j < j1; ++j) {
                    const float4 rj = __ldg(a.rec + j);
                    if ((__float_as_uint(rj.w) & ~FIXED_BIT) == chain) continue;
                    const float ex = rj.x + sx, ey = rj.y + sy, ez = rj.z + sz;
                    if (ex * ex + ey * ey + ez * ez < a.rl2f) {
                        if (n < PPA_MAXNB) a.nl[(size_t)n * a.M + p] = (unsigned)j | (q << IDX_BITS);
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
    a.nn[p] = n;
}

// the thread of monomer 0 retires the build request of this step (every build
// kernel has run) and counts the build
__device__ __forceinline__ void retire_build(const PpaArgs &a, int p)
{
    if (p == 0 && a.flags[1]) {
        if (!a.flags[0]) a.flags[2] += 1u;
        a.flags[1] = 0u;
    }
}

// binary64 force: minimum-image pair vectors, LJ 12-6 between chains, FENE
// bonds; F <- F_c(x) - gamma v; v <- v + half dt F (half = 0 for the first force)
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_force_f64(PpaArgs a, double half)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    retire_build(a, p);
    if (p >= a.M || is_fixed(a.rec[p])) return;
    const int cb = cur_buf(a);
    const double *x = cb ? a.x1 : a.x0;
    double *v = cb ? a.v1 : a.v0, *F = cb ? a.F1 : a.F0;
    const size_t M = a.M;
    const double xs = x[p], ys = x[M + p], zs = x[2 * M + p];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    const int n = a.nn[p];
    const double rc2 = PPA_RC * PPA_RC;
    for (int k = 0; k < n; ++k) {
        const int j = (int)(a.nl[(size_t)k * M + p] & IDX_MASK);
        const double ex = min_image(__dsub_rn(x[j], xs), a);
        const double ey = min_image(__dsub_rn(x[M + j], ys), a);
        const double ez = min_image(__dsub_rn(x[2 * M + j], zs), a);
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
    const int2 b = a.bp[p];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int t = side ? b.y : b.x;
        const double bx = __dsub_rn(x[t], xs), by = __dsub_rn(x[M + t], ys), bz = __dsub_rn(x[2 * M + t], zs);
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
    const double hdt = half * a.dt;
    const double f[3] = {fx, fy, fz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const size_t o = (size_t)d * M + p;
        const double vh = v[o];
        const double Ft = __dsub_rn(f[d], __dmul_rn(a.gamma, vh));
        F[o] = Ft;
        v[o] = __dadd_rn(vh, __dmul_rn(hdt, Ft));
    }
}

// mixed force, all binary32: pair vectors from the gather records, LJ 12-6;
// bond vectors from the build's bond vectors and the displacements; FENE,
// friction and kick
__global__ void __launch_bounds__(PPA_BLOCK) k_ppa_force_mixed(PpaArgs a, float half)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    retire_build(a, p);
    if (p >= a.M) return;
    const float4 ps = a.pg[p];
    if (is_fixed(ps)) return;
    const int cb = cur_buf(a);
    float *u = cb ? a.u1 : a.u0, *G = cb ? a.G1 : a.G0;
    const size_t M = a.M;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int n = a.nn[p];
    for (int k = 0; k < n; ++k) {
        const unsigned e = __ldg(a.nl + (size_t)k * M + p);
        const float4 pj = __ldg(a.pg + (e & IDX_MASK));
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
    }
    const int2 b = a.bp[p];
    const float4 dp = a.dl[p];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int t = side ? b.y : b.x;
        const float4 dt_ = __ldg(a.dl + t);
        const float4 bv = __ldg(a.bvec + (side ? p : t));
        const float sg = side ? 1.f : -1.f;             // the previous bond is -(its bond to p)
        const float bx = sg * bv.x + (dt_.x - dp.x), by = sg * bv.y + (dt_.y - dp.y),
                    bz = sg * bv.z + (dt_.z - dp.z);
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
        const size_t o = (size_t)d * M + p;
        const float vh = u[o];
        const float Ft = f[d] - a.gammaf * vh;
        G[o] = Ft;
        u[o] = vh + hdt * Ft;
    }
}

// ---- results in slot order ----

// one monomer back to slot order; the bits of its net force (0 at a chain end)
__device__ __forceinline__ unsigned long long unpermute_one(const PpaArgs &a, int s, double *__restrict__ xs)
{
    const int cb = cur_buf(a);
    const double *x = cb ? a.x1 : a.x0;
    const size_t M = a.M;
    const int p = a.pos_of[s];
    const float4 dp = a.u0 ? a.dl[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float dd[3] = {dp.x, dp.y, dp.z};
    double f2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d * M + s] = x[d * M + p] + (double)dd[d];
        const double f = a.u0 ? (double)(cb ? a.G1 : a.G0)[d * M + p] : (cb ? a.F1 : a.F0)[d * M + p];
        f2 += f * f;
    }
    const int i = s % a.N;
    return (i > 0 && i < a.N - 1) ? (unsigned long long)__double_as_longlong(sqrt(f2)) : 0ull;
}

// positions back to slot order; the largest net force on a mobile monomer
// (a warp maximum, then one atomic per warp) and the sum of the list lengths
__global__ void __launch_bounds__(256) k_ppa_unpermute(PpaArgs a, double *__restrict__ xs,
                                                      unsigned long long *__restrict__ fmax_bits,
                                                      unsigned long long *__restrict__ nn_sum)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long fb = 0ull;                      // bits of a non-negative double order like it
    unsigned long long nb = 0ull;
    if (s < a.M) {
        fb = unpermute_one(a, s, xs);
        nb = (unsigned long long)a.nn[s];              // list lengths, storage order (any order sums)
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, fb, o);
        fb = t > fb ? t : fb;
        nb += __shfl_down_sync(0xffffffffu, nb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (fb) atomicMax(fmax_bits, fb);
        atomicAdd(nn_sum, nb);
    }
}

// contour length of every chain from slot-order positions: one warp per
// chain, lane l sums bonds l, l + 32, ..., then a fixed-order shuffle tree
__global__ void __launch_bounds__(256) k_ppa_lengths(const double *__restrict__ x, int M, int N,
                                                    double *__restrict__ lpp)
{
    const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= M / N) return;
    double sum = 0.0;
    for (int i = lane; i + 1 < N; i += 32) {
        const size_t s = (size_t)c * N + i;
        const double bx = __dsub_rn(x[s + 1], x[s]);
        const double by = __dsub_rn(x[M + s + 1], x[M + s]);
        const double bz = __dsub_rn(x[2 * (size_t)M + s + 1], x[2 * (size_t)M + s]);
        sum += sqrt(__dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) lpp[c] = sum;
}

__global__ void k_ppa_iota(int *__restrict__ a, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

constexpr int PPA_BUILD_LAUNCHES = 9;        // kernels of one list build
constexpr int PPA_LAUNCHES_PER_ITER = 2 + PPA_BUILD_LAUNCHES;   // direct launches of one step

// the list build (each kernel returns at once unless a build is requested)
void enqueue_build(const PpaArgs &a, cudaStream_t st, int *bsum)
{
    const int nbs = nblk(a.ncell, 1024);
    k_ppa_bin<<<nblk(a.M, 256), 256, 0, st>>>(a);
    k_scan1<<<nbs, 1024, 0, st>>>(a.count, a.start, bsum, a.ncell, a.flags);
    k_scan2<<<nbs, 1024, 0, st>>>(a.start, bsum, a.ncell, nbs, a.flags);
    k_ppa_scatter<<<nblk(a.M, 256), 256, 0, st>>>(a);
    k_ppa_cellsort<<<nblk(a.ncell, 256), 256, 0, st>>>(a);
    k_ppa_permute<<<nblk(a.M, 256), 256, 0, st>>>(a);
    k_ppa_flip<<<1, 1, 0, st>>>(a);
    k_ppa_partners<<<nblk(a.M, 256), 256, 0, st>>>(a);
    k_ppa_nlist<<<nblk(a.M, PPA_BLOCK), PPA_BLOCK, 0, st>>>(a);
}

void enqueue_drift(const PpaArgs &a, cudaStream_t st, bool mixed)
{
    const int nbm = nblk(a.M, PPA_BLOCK);
    if (mixed) k_ppa_drift_mixed<<<nbm, PPA_BLOCK, 0, st>>>(a);
    else k_ppa_drift_f64<<<nbm, PPA_BLOCK, 0, st>>>(a);
}

void enqueue_force(const PpaArgs &a, cudaStream_t st, bool mixed, double half)
{
    const int nbm = nblk(a.M, PPA_BLOCK);
    if (mixed) k_ppa_force_mixed<<<nbm, PPA_BLOCK, 0, st>>>(a, (float)half);
    else k_ppa_force_f64<<<nbm, PPA_BLOCK, 0, st>>>(a, half);
}

void enqueue_step(const PpaArgs &a, cudaStream_t st, int *bsum, bool mixed)
{
    enqueue_drift(a, st, mixed);
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
    for (int i = 0; ok && i < PPA_GRAPH_ITERS; ++i) {
        enqueue_drift(a, s1, mixed);
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
    if (nc < 3 || nc > 1024) return KG_ERR_INVALID_ARG;     // 27 distinct stencil cells; bounded grid
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
    a.x0 = (double *)get(sizeof(double) * m3);
    a.x1 = (double *)get(sizeof(double) * m3);
    if (mixed) {
        a.u0 = (float *)get(sizeof(float) * m3);
        a.u1 = (float *)get(sizeof(float) * m3);
        a.G0 = (float *)get(sizeof(float) * m3);
        a.G1 = (float *)get(sizeof(float) * m3);
    } else {
        a.v0 = (double *)get(sizeof(double) * m3);
        a.v1 = (double *)get(sizeof(double) * m3);
        a.F0 = (double *)get(sizeof(double) * m3);
        a.F1 = (double *)get(sizeof(double) * m3);
        a.xb = (double *)get(sizeof(double) * m3);
    }
    a.slot0 = (int *)get(sizeof(int) * M);
    a.slot1 = (int *)get(sizeof(int) * M);
    a.rec = (float4 *)get(sizeof(float4) * M);
    a.pg = (float4 *)get(sizeof(float4) * M);
    a.dl = (float4 *)get(sizeof(float4) * M);
    a.off = (float4 *)get(sizeof(float4) * M);
    if (mixed) a.bvec = (float4 *)get(sizeof(float4) * M);
    a.bp = (int2 *)get(sizeof(int2) * M);
    a.pos_of = (int *)get(sizeof(int) * M);
    a.cellof = (int *)get(sizeof(int) * M);
    a.rank = (int *)get(sizeof(int) * M);
    a.count = (int *)get(sizeof(int) * ((size_t)a.ncell + 1));
    a.start = (int *)get(sizeof(int) * ((size_t)a.ncell + 1));
    a.list = (int *)get(sizeof(int) * M);
    a.nl = (unsigned *)get(sizeof(unsigned) * (size_t)PPA_MAXNB * M);
    a.nn = (int *)get(sizeof(int) * M);
    a.flags = (unsigned *)get(sizeof(unsigned) * 4);
    int *bsum = (int *)get(sizeof(int) * (size_t)nbs);
    double *d_xs = (double *)get(sizeof(double) * m3);
    double *d_lpp = (double *)get(sizeof(double) * n_ch);
    unsigned long long *d_fmax = (unsigned long long *)get(2 * sizeof(unsigned long long));   // max |F|, sum nn
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
    kg::to_slots(c, melt, c->x, a.x0, 3);              // (3, M) slot order, unwrapped; buffer 0
    k_ppa_iota<<<nblk(M, 256), 256, 0, st>>>(a.slot0, M);
    static const unsigned one = 1u;
    if (cudaMemcpyAsync(a.flags + 1, &one, sizeof(unsigned), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return done(KG_ERR_CUDA);
    // the first build (into cell order) and force, from rest (v = 0, no kick)
    enqueue_build(a, st, bsum);
    enqueue_force(a, st, mixed, 0.0);
    c->launches += 2 + PPA_BUILD_LAUNCHES;
    long long left = pp->n_iter, graph_steps = 0;
    if (left >= 2 * PPA_GRAPH_ITERS && cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamCreateWithFlags(&gs2, cudaStreamNonBlocking) == cudaSuccess &&
        capture_steps(a, gs, gs2, bsum, mixed, &gexec)) {
        for (; left >= PPA_GRAPH_ITERS; left -= PPA_GRAPH_ITERS, graph_steps += PPA_GRAPH_ITERS)
            if (cudaGraphLaunch(gexec, st) != cudaSuccess) return done(KG_ERR_CUDA);
    }
    c->launches += 3 * graph_steps + PPA_LAUNCHES_PER_ITER * left;   // + the graphs' builds, below
    for (; left > 0; --left) enqueue_step(a, st, bsum, mixed);
    k_ppa_unpermute<<<nblk(M, 256), 256, 0, st>>>(a, d_xs, d_fmax, d_fmax + 1);
    k_ppa_lengths<<<nblk(32LL * n_ch, 256), 256, 0, st>>>(d_xs, M, N, d_lpp);
    c->launches += 2;
    if (cudaGetLastError() != cudaSuccess) return done(KG_ERR_CUDA);

    std::vector<double> h_lpp((size_t)n_ch);
    unsigned h_flags[4] = {0, 0, 0, 0};
    unsigned long long h_fmax[2] = {0, 0};
    if (cudaMemcpyAsync(h_lpp.data(), d_lpp, sizeof(double) * n_ch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_flags, a.flags, sizeof(h_flags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_fmax, d_fmax, sizeof(h_fmax), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return done(KG_ERR_CUDA);
    if (x_out && cudaMemcpyAsync(x_out, d_xs, sizeof(double) * m3, cudaMemcpyDefault, st) != cudaSuccess)
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
        std::memcpy(&res->fmax, &h_fmax[0], sizeof(double));
        res->builds = (long long)h_flags[2];
        res->mean_neighbours = (double)h_fmax[1] / (double)M;
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
