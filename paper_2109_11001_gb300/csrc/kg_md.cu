// kg_md.cu -- molecular-dynamics kernels of the GB300 DBH library.
//
//  * cell binning + counting sort + Verlet-list build (every rebuild);
//  * one fused kernel per MD step: U_MLJ^n pairs over the Verlet list (Eq. 6),
//    U_bond^n bonds (Eq. 10), kappa (1 - cos theta) bending (Eq. 4), Langevin
//    friction and Philox noise, and the leapfrog update of (x, u);
//  * a force/energy kernel for observables and parity checks.
// Thread per monomer in compute order: the per-monomer arrays are kept sorted
// by Verlet-list cell (re-sorted every few hundred steps), so a warp's
// neighbours sit in a few contiguous runs of memory.  bp[i] holds the compute
// indices of the monomers two and one before and after along the chain
// (-1 past a chain end); slot_of[i] is the chain-major slot c*N + i, which keys
// the random draws so results do not depend on the order.
#include <cuda_runtime.h>

#include "kg_host.h"
#include "kg_rebuild.cuh"

namespace kg {

// ---------------------------------------------------------------------------
// pair and bond terms (binary32 and binary64 forms of the same formulas)
// U_MLJ^n(r) = c1 r^-n - c2 r^-6 + 1 for r < r_c (Eqs. 5-6, shifted by +epsilon);
// fr = (dU/dr)/r, so the force on i from j at d = x_j - x_i is fr * d.
// ---------------------------------------------------------------------------
template <bool ENERGY>
__device__ __forceinline__ float mlj_fr(const StageDev &st, float r2, float &U)
{
    const float ir2 = __fdividef(1.0f, r2);
    const float ir6 = ir2 * ir2 * ir2;
    float rn;
    if (st.nint == 12) {                 // WCA (Eq. 2): the production potential
        rn = ir6 * ir6;
    } else if (st.nkind == 1) {
        float p = 1.0f;
        for (int k = 0; k < (st.nint >> 1); ++k) p *= ir2;
        if (st.nint & 1) p *= rsqrtf(r2);
        rn = p;
    } else if (st.nkind == 2) {          // n = 23/4: r^-6 r^(1/4)
        rn = ir6 * sqrtf(sqrtf(sqrtf(r2)));
    } else if (st.nkind == 3) {          // n = 13/2: r^-6 r^(-1/2)
        rn = ir6 * sqrtf(rsqrtf(r2));
    } else {
        rn = exp2f(-0.5f * st.nf * log2f(r2));
    }
    if (ENERGY) U = st.c1f * rn - st.c2f * ir6 + 1.0f;
    return (st.c2x6f * ir6 - st.c1xnf * rn) * ir2;
}

template <bool ENERGY>
__device__ __forceinline__ double mlj_fr(const StageDev &st, double r2, double &U)
{
    const double ir2 = 1.0 / r2;
    const double ir6 = ir2 * ir2 * ir2;
    double rn;
    if (st.nkind == 1) {
        double p = 1.0;
        for (int k = 0; k < (st.nint >> 1); ++k) p *= ir2;
        if (st.nint & 1) p *= rsqrt(r2);
        rn = p;
    } else if (st.nkind == 2) {
        rn = ir6 * sqrt(sqrt(sqrt(r2)));
    } else if (st.nkind == 3) {
        rn = ir6 * sqrt(rsqrt(r2));
    } else {
        rn = exp2(-0.5 * st.n * log2(r2));
    }
    if (ENERGY) U = st.c1 * rn - st.c2 * ir6 + 1.0;
    return (6.0 * st.c2 * ir6 - st.n * st.c1 * rn) * ir2;
}

template <typename T> struct V3;
template <> struct V3<float> { using t = float3; };
template <> struct V3<double> { using t = double3; };

template <typename T> __device__ __forceinline__ typename V3<T>::t mk(T a, T b, T c);
template <> __device__ __forceinline__ float3 mk<float>(float a, float b, float c) { return make_float3(a, b, c); }
template <> __device__ __forceinline__ double3 mk<double>(double a, double b, double c) { return make_double3(a, b, c); }

template <typename T3> __device__ __forceinline__ auto dot3(T3 a, T3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T3> __device__ __forceinline__ T3 sub3(T3 a, T3 b) { return T3{a.x - b.x, a.y - b.y, a.z - b.z}; }

template <typename T> __device__ __forceinline__ T st_c(const StageDev &st, int which);
template <> __device__ __forceinline__ float st_c<float>(const StageDev &st, int w)
{
    return w == 0 ? st.kfenef : w == 1 ? st.R0sqf : w == 2 ? st.dtf : w == 3 ? st.gammaf : w == 4 ? st.ampf
         : w == 5 ? st.qminf : w == 6 ? st.r2starf : st.ustarf;
}
template <> __device__ __forceinline__ double st_c<double>(const StageDev &st, int w)
{
    return w == 0 ? st.kfene : w == 1 ? st.R0sq : w == 2 ? st.dt : w == 3 ? st.gamma : w == 4 ? st.amp
         : w == 5 ? st.qmin : w == 6 ? st.r2star : st.ustar;
}

__device__ __forceinline__ float flog(float a) { return logf(a); }
__device__ __forceinline__ double flog(double a) { return log(a); }
__device__ __forceinline__ float frsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double frsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ float frcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double frcp(double a) { return 1.0 / a; }

// ---------------------------------------------------------------------------
// position access policies
// ---------------------------------------------------------------------------
// binary32 gather records p = offset from the build-time cell corner +
// displacement since the build (w: packed cell coordinates).  A Verlet-list
// entry carries the image shift of its pair (the stencil code), so a listed
// pair costs one gather and one table lookup; chain partners, which are not
// in the list, take the shift from the cell codes.
struct GeoMixed {
    using T = float;
    using T3 = float3;
    const float4 *__restrict__ pg;
    const float4 *__restrict__ shtab;    // SHIFT_SLOTS shift vectors per melt
    const float4 *__restrict__ sht;
    int nc;
    float h, L, invL;
    float4 pi;
    __device__ __forceinline__ void melt(const MeltDev &md, int m)
    {
        nc = md.nc; h = md.hf; L = md.Lf; invL = md.invLf;
        sht = shtab + SHIFT_SLOTS * m;
    }
    __device__ __forceinline__ void self(int s) { pi = __ldg(pg + s); }
    __device__ __forceinline__ float3 rel_nl(unsigned e) const
    {
        const float4 pj = __ldg(pg + (e & IDX_MASK));
        const float4 sh = __ldg(sht + (e >> IDX_BITS));
        return make_float3((pj.x - pi.x) + sh.x, (pj.y - pi.y) + sh.y, (pj.z - pi.z) + sh.z);
    }
    __device__ __forceinline__ float3 rel(int j) const { return rec_rel(pi, __ldg(pg + j), nc, h, L, invL); }
};

struct GeoF64 {
    using T = double;
    using T3 = double3;
    const double4_32a *__restrict__ pos;
    double L, invL;
    double4_32a pi;
    __device__ __forceinline__ void melt(const MeltDev &md, int) { L = md.L; invL = md.invL; }
    __device__ __forceinline__ void self(int s) { pi = pos[s]; }
    __device__ __forceinline__ double3 rel(int j) const
    {
        const double4_32a pj = pos[j];
        double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        dx -= L * rint(dx * invL);
        dy -= L * rint(dy * invL);
        dz -= L * rint(dz * invL);
        return make_double3(dx, dy, dz);
    }
    __device__ __forceinline__ double3 rel_nl(unsigned e) const { return rel((int)(e & IDX_MASK)); }
};

template <bool ENERGY, typename T, typename T3>
__device__ __forceinline__ void pair_term(const StageDev &st, T rc2, T3 d, T3 &F, double *e)
{
    const T r2 = dot3(d, d);
    if (!ENERGY) {                       // branch-free: a warp evaluates the force for some lane anyway
        T U;
        T fr = mlj_fr<false>(st, r2, U);
        fr = r2 < rc2 ? fr : (T)0;
        F.x += fr * d.x; F.y += fr * d.y; F.z += fr * d.z;
    } else if (r2 < rc2) {
        T U;
        const T fr = mlj_fr<ENERGY>(st, r2, U);
        F.x += fr * d.x; F.y += fr * d.y; F.z += fr * d.z;
        e[0] += 0.5 * (double)U;
        e[3] -= 0.5 * (double)(fr * r2);
    }
}

// Pair forces on s from its Verlet-list entries k = k0, k0 + stride, ...
// (both directions are stored), four entries in flight.
template <bool ENERGY, class G>
__device__ __forceinline__ void pair_forces(const G &g, const SimDev &S, const StageDev &st, int s,
                                            const unsigned *__restrict__ nl, int cnt, int k0, int stride,
                                            typename G::T3 &F, double *e)
{
    using T = typename G::T;
    using T3 = typename G::T3;
    const T rc2 = (T)S.rc2;
    const size_t Mp = (size_t)S.Mp, step = (size_t)stride * Mp;
    const unsigned *__restrict__ col = nl + s + (size_t)k0 * Mp;
    int k = k0;
    for (; k + 3 * stride < cnt; k += 4 * stride, col += 4 * step) {
        const unsigned e0 = __ldg(col), e1 = __ldg(col + step);
        const unsigned e2 = __ldg(col + 2 * step), e3 = __ldg(col + 3 * step);
        const T3 d0 = g.rel_nl(e0), d1 = g.rel_nl(e1), d2 = g.rel_nl(e2), d3 = g.rel_nl(e3);
        pair_term<ENERGY>(st, rc2, d0, F, e);
        pair_term<ENERGY>(st, rc2, d1, F, e);
        pair_term<ENERGY>(st, rc2, d2, F, e);
        pair_term<ENERGY>(st, rc2, d3, F, e);
    }
    for (; k < cnt; k += stride, col += step) pair_term<ENERGY>(st, rc2, g.rel_nl(__ldg(col)), F, e);
}

// Bond (Eq. 10) and bending (Eq. 4) forces on s from its chain partners.
template <bool ENERGY, class G>
__device__ __forceinline__ void bonded_forces(const G &g, const StageDev &st, const MeltDev &md,
                                              typename G::T rc2, int4 bp, typename G::T3 &F, double *e,
                                              unsigned &err)
{
    using T = typename G::T;
    using T3 = typename G::T3;
    // chain neighbours: bp = (s-2, s-1, s+1, s+2) along the chain, -1 past an end
    const bool hm2 = bp.x >= 0, hm1 = bp.y >= 0, hp1 = bp.z >= 0, hp2 = bp.w >= 0;
    T3 rm2 = mk<T>(0, 0, 0), rm1 = mk<T>(0, 0, 0), rp1 = mk<T>(0, 0, 0), rp2 = mk<T>(0, 0, 0);
    if (hm1) rm1 = g.rel(bp.y);
    if (hm2) rm2 = g.rel(bp.x);
    if (hp1) rp1 = g.rel(bp.z);
    if (hp2) rp2 = g.rel(bp.w);
    // bonds: U_MLJ^n + FENE(k_n) (Eq. 10)
    const T kf = st_c<T>(st, 0), R0sq = st_c<T>(st, 1);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if ((side == 0 && hm1) || (side == 1 && hp1)) {
            const T3 d = side == 0 ? rm1 : rp1;
            const T r2 = dot3(d, d);
            const T qmin = st_c<T>(st, 5);
            T q = (T)1 - r2 / R0sq, fr, Uf = 0;
            if (qmin > (T)0 && q < qmin) {           // continuation beyond r* (kg_params.fene_qmin)
                fr = kf * frcp(qmin);
                if (!(r2 < (T)4 * R0sq)) err |= ERR_OVERSTRETCH;
                if (ENERGY) Uf = st_c<T>(st, 7) + kf * (r2 - st_c<T>(st, 6)) / ((T)2 * qmin);
            } else {
                if (!(r2 < R0sq)) err |= ERR_OVERSTRETCH;
                q = fmax(q, (T)1e-6);                    // finite even when flagged
                fr = kf * frcp(q);
                if (ENERGY) Uf = (T)-0.5 * kf * R0sq * flog(q);
            }
            T U = 0;
            if (r2 < rc2) fr += mlj_fr<ENERGY>(st, r2, U);
            F.x += fr * d.x; F.y += fr * d.y; F.z += fr * d.z;
            if (ENERGY) {
                e[1] += 0.5 * ((double)U + (double)Uf);
                e[3] -= 0.5 * (double)(fr * r2);
            }
        }
    }
    // bending kappa (1 - b1.b2 / |b1||b2|) at the vertices s-1, s, s+1
    const T kap = (T)md.kappa;
    if (kap != (T)0) {
        const T3 Bm2 = sub3(rm1, rm2), Bm1 = mk<T>(-rm1.x, -rm1.y, -rm1.z), B0 = rp1, Bp1 = sub3(rp2, rp1);
        if (hm1 && hp1) {                    // vertex s: force kappa (g1 - g2)
            const T l1 = dot3(Bm1, Bm1), l2 = dot3(B0, B0), inv = frsqrt(l1 * l2), cs = dot3(Bm1, B0) * inv;
            const T c1 = cs * frcp(l1), c2 = cs * frcp(l2);
            F.x += kap * ((B0.x * inv - c1 * Bm1.x) - (Bm1.x * inv - c2 * B0.x));
            F.y += kap * ((B0.y * inv - c1 * Bm1.y) - (Bm1.y * inv - c2 * B0.y));
            F.z += kap * ((B0.z * inv - c1 * Bm1.z) - (Bm1.z * inv - c2 * B0.z));
            if (ENERGY) e[2] += (double)kap * (1.0 - (double)cs);
        }
        if (hp2) {                           // vertex s+1, s is its first end: -kappa g1
            const T l1 = dot3(B0, B0), l2 = dot3(Bp1, Bp1), inv = frsqrt(l1 * l2), cs = dot3(B0, Bp1) * inv;
            const T c1 = cs * frcp(l1);
            F.x -= kap * (Bp1.x * inv - c1 * B0.x);
            F.y -= kap * (Bp1.y * inv - c1 * B0.y);
            F.z -= kap * (Bp1.z * inv - c1 * B0.z);
        }
        if (hm2) {                           // vertex s-1, s is its last end: +kappa g2
            const T l1 = dot3(Bm2, Bm2), l2 = dot3(Bm1, Bm1), inv = frsqrt(l1 * l2), cs = dot3(Bm2, Bm1) * inv;
            const T c2 = cs * frcp(l2);
            F.x += kap * (Bm2.x * inv - c2 * Bm1.x);
            F.y += kap * (Bm2.y * inv - c2 * Bm1.y);
            F.z += kap * (Bm2.z * inv - c2 * Bm1.z);
        }
    }
}

// Conservative force on slot s (chain position i of N) and, with ENERGY, its
// shares of the energies: e[0] pair (1/2 per pair), e[1] bond (1/2 per bond),
// e[2] bending (the angle whose vertex is s), e[3] virial (1/2 per pair/bond).
template <bool ENERGY, class G>
__device__ __forceinline__ typename G::T3 force_on(const G &g, const SimDev &S, const StageDev &st,
                                                   const MeltDev &md, int s, int4 bp,
                                                   const unsigned *__restrict__ nl, int cnt,
                                                   double *e, unsigned &err)
{
    using T = typename G::T;
    typename G::T3 F = mk<T>(0, 0, 0);
    pair_forces<ENERGY>(g, S, st, s, nl, cnt, 0, 1, F, e);
    bonded_forces<ENERGY>(g, st, md, (T)S.rc2, bp, F, e, err);
    return F;
}

// ---------------------------------------------------------------------------
// fused MD step, binary64 path: forces at x_n, then u <- u + dt F_n,
// x <- x + dt u with F_n = F_c - gamma u + sqrt(2 gamma T / dt) g_n,
// g_n = Philox normals (the mixed path's step kernel is in kg_step.cu)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_step_f64(const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp,
                                                 double *__restrict__ x, double *__restrict__ u,
                                                 const double4_32a *__restrict__ pcur, double4_32a *__restrict__ pnext,
                                                 const double4_32a *__restrict__ xb, const unsigned *__restrict__ nl,
                                                 const int *__restrict__ nn, const int *__restrict__ slot_of,
                                                 const int4 *__restrict__ bp, unsigned *__restrict__ flags,
                                                 const long long *__restrict__ stepp)
{
    if (flags[0]) return;                  // a latched error stops the run
    const SimDev &S = *Sp;
    const StageDev &st = *stp;
    const long long step = *stepp;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    bool rebuild = false;
    unsigned err = 0;
    if (s < S.M) {
        const int slot = __ldg(slot_of + s);
        const int m = melt_of(S, slot);
        const MeltDev &md = S.melt[m];
        const int rel = slot - md.off;
        GeoF64 g{pcur, md.L, md.invL, {}};
        g.self(s);
        double3 F = force_on<false>(g, S, st, md, s, __ldg(bp + s), nl, __ldg(nn + s), nullptr, err);
        const double3 gn = gauss3_d(draw(S.seed, m, 0, (unsigned long long)step, (uint32_t)rel));
        const int Mp = S.Mp;
        double3 v = make_double3(u[s], u[Mp + s], u[2 * Mp + s]);
        v.x += st.dt * (F.x - st.gamma * v.x + st.amp * gn.x);
        v.y += st.dt * (F.y - st.gamma * v.y + st.amp * gn.y);
        v.z += st.dt * (F.z - st.gamma * v.z + st.amp * gn.z);
        u[s] = v.x; u[Mp + s] = v.y; u[2 * Mp + s] = v.z;
        const double nx = x[s] + st.dt * v.x, ny = x[Mp + s] + st.dt * v.y, nz = x[2 * Mp + s] + st.dt * v.z;
        x[s] = nx; x[Mp + s] = ny; x[2 * Mp + s] = nz;
        pnext[s] = make_double4_32a(nx, ny, nz, 0.0);
        const double4_32a b = xb[s];
        const double dx = nx - b.x, dy = ny - b.y, dz = nz - b.z;
        rebuild = dx * dx + dy * dy + dz * dz > S.half_skin2;
        if (!isfinite(v.x + v.y + v.z)) err |= ERR_NONFINITE;
    }
    if (__syncthreads_or(rebuild) && threadIdx.x == 0) atomicOr(flags + 1, 1u);
    if (err) atomicOr(flags, err);
}

// ---------------------------------------------------------------------------
// rebuild chain: each kernel returns at once unless flags[1] requests a
// rebuild; the last block of k_nlist to finish clears the request
// ---------------------------------------------------------------------------
// build records (offset from the Verlet-cell corner + cell coordinates),
// gather buffers reset, Verlet-grid cell + rank within it
__global__ void __launch_bounds__(256) k_bin_md(const SimDev *__restrict__ Sp, double *__restrict__ x,
                                               double *__restrict__ xb64,
                                               float4 *__restrict__ recb, float4 *__restrict__ dcur,
                                               float4 *__restrict__ pgcur, double4_32a *__restrict__ pcur,
                                               double4_32a *__restrict__ xb, int *__restrict__ cellid,
                                               int *__restrict__ rank, int *__restrict__ count,
                                               const int *__restrict__ slot_of, unsigned *__restrict__ flags)
{
    if (!flags[1] || flags[0]) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Sp->M) return;
    bin_md_one(*Sp, s, x, xb64, recb, dcur, pgcur, pcur, xb, cellid, rank, count, slot_of, flags);
}

// DB grid: cell of each particle from its wrapped position (cells >= 1.3
// sigma), and its binary32 record (offset from the cell corner, cell
// coordinates) for the swap-bond prefilter
__global__ void __launch_bounds__(256) k_bin_db(const SimDev *__restrict__ Sp, const double *__restrict__ x,
                                               int *__restrict__ cellid, int *__restrict__ rank,
                                               int *__restrict__ count, const int *__restrict__ slot_of,
                                               float4 *__restrict__ rec)
{
    const SimDev &S = *Sp;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.M) return;
    const MeltDev &md = S.melt[melt_of(S, slot_of[s])];
    int cell[3];
    float off[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) cell[d] = cell_of(x[d * S.Mp + s], md.hdb, md.invhdb, md.ndb, off[d]);
    rec[s] = make_float4(off[0], off[1], off[2], __uint_as_float(pack_code(cell[0], cell[1], cell[2])));
    const int c = md.dbcell_off + (cell[2] * md.ndb + cell[1]) * md.ndb + cell[0];
    cellid[s] = c;
    rank[s] = atomicAdd(count + c, 1);
}

// exclusive scan, phase 1: per 1024-element block, local scan + block total
__global__ void __launch_bounds__(1024) k_scan1(const int *__restrict__ in, int *__restrict__ out,
                                               int *__restrict__ bsum, int n, const unsigned *__restrict__ flags)
{
    if (flags && (!flags[1] || flags[0])) return;
    __shared__ int wsum[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int ws = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += t;
        }
        wsum[lane] = ws;
    }
    __syncthreads();
    const int base = w ? wsum[w - 1] : 0;
    if (i < n) out[i] = base + incl - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = base + incl;
}

// phase 2: add the totals of all preceding blocks; out[n] = grand total
__global__ void __launch_bounds__(1024) k_scan2(int *__restrict__ out, const int *__restrict__ bsum, int n,
                                               int nblk, const unsigned *__restrict__ flags)
{
    if (flags && (!flags[1] || flags[0])) return;
    __shared__ int off_s;
    if (threadIdx.x < 32) {
        int acc = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 32) acc += bsum[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) off_s = acc;
    }
    __syncthreads();
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += off_s;
    if (blockIdx.x == nblk - 1 && threadIdx.x == 0) {
        int tot = 0;
        for (int b = 0; b < nblk; ++b) tot += bsum[b];
        out[n] = tot;
    }
}

// slot list in cell order; with recb, the build offsets are copied into the
// same order (recs, w = the compute index) so that a cell's candidates are one
// contiguous run of single 16-byte loads
__global__ void __launch_bounds__(256) k_scatter(const int *__restrict__ cellid, const int *__restrict__ rank,
                                                const int *__restrict__ start, int *__restrict__ list, int M,
                                                const unsigned *__restrict__ flags)
{
    if (flags && (!flags[1] || flags[0])) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < M) scatter_one(s, cellid, rank, start, list);
}

// within-cell order by compute index (deterministic lists), the records in
// the same order, the counts cleared (cellrank_one, kg_rebuild.cuh)
__global__ void __launch_bounds__(256) k_cellrank(const int *__restrict__ cellid, const int *__restrict__ start,
                                                 const int *__restrict__ tmp, int *__restrict__ list,
                                                 const float4 *__restrict__ recb, float4 *__restrict__ recs,
                                                 int *__restrict__ count, int M, unsigned *__restrict__ flags)
{
    if (!flags[1] || flags[0]) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < M && cellrank_one(p, cellid, start, tmp, list, recb, recs, count)) atomicOr(flags, ERR_NL_CAPACITY);
}

// Verlet-list build (the per-monomer work is nlist_one, kg_rebuild.cuh).
// The last block to finish clears the rebuild request.
// (256, 5): at most 48 registers and no spills; more resident warps hide the
// candidate loads (tighter caps spill, looser ones leave the SM half idle)
constexpr int NL_BLOCK = 256;

__global__ void __launch_bounds__(NL_BLOCK, 5) k_nlist(const __grid_constant__ NlArgs A)
{
    __shared__ unsigned go;
    if (threadIdx.x == 0) go = (A.flags[1] && !A.flags[0]) ? 1u : 0u;
    __syncthreads();
    if (!go) return;                                         // block-uniform
    const int s = blockIdx.x * NL_BLOCK + threadIdx.x;
    const unsigned err = nlist_one(A, s);
    if (err) atomicOr(A.flags, err);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(A.flags + 4, 1u) == gridDim.x - 1) {
            A.flags[1] = 0u;
            A.flags[4] = 0u;
            A.flags[5] += 1u;                    // Verlet builds completed
        }
    }
}

// ---------------------------------------------------------------------------
// forces + energies (observables, parity): F_c written as binary64; per block
// partial sums [pair, bond, angle, virial, kinetic] in binary64, where the
// kinetic part uses v_n = u + dt/2 (F_c - gamma u + amp g_n).
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(128) k_forces(const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp,
                                               G g, const void *__restrict__ uptr, int lo, int hi,
                                               const unsigned *__restrict__ nl, const int *__restrict__ nn,
                                               const int *__restrict__ slot_of, const int4 *__restrict__ bp,
                                               double *__restrict__ Fout, double *__restrict__ part,
                                               unsigned *__restrict__ flags, long long step)
{
    using T = typename G::T;
    const SimDev &S = *Sp;
    const StageDev &st = *stp;
    const int s = lo + blockIdx.x * blockDim.x + threadIdx.x;
    double e[5] = {0, 0, 0, 0, 0};
    unsigned err = 0;
    if (s < hi) {
        const int slot = slot_of[s];
        const int m = melt_of(S, slot);
        const MeltDev &md = S.melt[m];
        const int rel = slot - md.off;
        G gg = g;
        gg.melt(md, m);
        gg.self(s);
        const auto F = force_on<true>(gg, S, st, md, s, bp[s], nl, __ldg(nn + s), e, err);
        const int Mp = S.Mp;
        if (Fout) {
            Fout[s] = (double)F.x; Fout[Mp + s] = (double)F.y; Fout[2 * Mp + s] = (double)F.z;
        }
        const double3 gn = gauss3_d(draw(S.seed, m, 0, (unsigned long long)step, (uint32_t)rel));
        const T *u = (const T *)uptr;
        const double ux = (double)u[s], uy = (double)u[Mp + s], uz = (double)u[2 * Mp + s];
        const double vx = ux + 0.5 * st.dt * ((double)F.x - st.gamma * ux + st.amp * gn.x);
        const double vy = uy + 0.5 * st.dt * ((double)F.y - st.gamma * uy + st.amp * gn.y);
        const double vz = uz + 0.5 * st.dt * ((double)F.z - st.gamma * uz + st.amp * gn.z);
        e[4] = 0.5 * (vx * vx + vy * vy + vz * vz);
    }
    if (err) atomicOr(flags, err);
    // deterministic block reduction (fixed tree)
    __shared__ double sh[5][128];
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = e[k];
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) part[blockIdx.x * 5 + k] = sh[k][0];
}

// ---------------------------------------------------------------------------
// compute order: chain partners, re-sorting, and gathers back to slot order
// ---------------------------------------------------------------------------
// bp[i] = compute indices of slots s-2, s-1, s+1, s+2 of i's chain (-1 past an end)
__global__ void __launch_bounds__(256) k_bonded(const SimDev *__restrict__ Sp, const int *__restrict__ slot_of,
                                               const int *__restrict__ comp_of, int4 *__restrict__ bp)
{
    const SimDev &S = *Sp;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S.M) return;
    const int s = slot_of[j];
    const MeltDev &md = S.melt[melt_of(S, s)];
    const int i = (s - md.off) % md.N, N = md.N;
    bp[j] = make_int4(i >= 2 ? comp_of[s - 2] : -1, i >= 1 ? comp_of[s - 1] : -1,
                      i <= N - 2 ? comp_of[s + 1] : -1, i <= N - 3 ? comp_of[s + 2] : -1);
}

// New compute order = the cell order of the last Verlet build (clist): gather
// the per-monomer state into scratch ...
template <typename U>
__global__ void __launch_bounds__(256) k_sort_gather(int M, int Mp, const int *__restrict__ order,
                                                    const double *__restrict__ x, const U *__restrict__ u,
                                                    const int *__restrict__ pid, const int *__restrict__ slot_of,
                                                    double *__restrict__ sx, U *__restrict__ su,
                                                    int *__restrict__ spid, int *__restrict__ sslot)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int o = order[j];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        sx[d * Mp + j] = x[d * Mp + o];
        su[d * Mp + j] = u[d * Mp + o];
    }
    spid[j] = pid[o];
    sslot[j] = slot_of[o];
}

// ... and copy it back, with the inverse map.
template <typename U>
__global__ void __launch_bounds__(256) k_sort_finish(int M, int Mp, double *__restrict__ x, U *__restrict__ u,
                                                    int *__restrict__ pid, int *__restrict__ slot_of,
                                                    int *__restrict__ comp_of, const double *__restrict__ sx,
                                                    const U *__restrict__ su, const int *__restrict__ spid,
                                                    const int *__restrict__ sslot)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        x[d * Mp + j] = sx[d * Mp + j];
        u[d * Mp + j] = su[d * Mp + j];
    }
    pid[j] = spid[j];
    const int s = sslot[j];
    slot_of[j] = s;
    comp_of[s] = j;
}

// out[d][r] = in[d][comp_of[off + r]] for r < n: slot order for the caller
__global__ void __launch_bounds__(256) k_to_slots(const double *__restrict__ in, int in_stride,
                                                 const int *__restrict__ comp_of, int off, int n,
                                                 double *__restrict__ out, int out_stride, int dims)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int j = comp_of[off + r];
    for (int d = 0; d < dims; ++d) out[(size_t)d * out_stride + r] = in[(size_t)d * in_stride + j];
}

__global__ void __launch_bounds__(256) k_to_slots_f(const float *__restrict__ in, int in_stride,
                                                   const int *__restrict__ comp_of, int off, int n,
                                                   double *__restrict__ out, int out_stride)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int j = comp_of[off + r];
    for (int d = 0; d < 3; ++d) out[(size_t)d * out_stride + r] = (double)in[(size_t)d * in_stride + j];
}

__global__ void __launch_bounds__(256) k_to_slots_i(const int *__restrict__ in, const int *__restrict__ comp_of,
                                                   int off, int n, int *__restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = in[comp_of[off + r]];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

void bonded_partners(kg_ctx *c)
{
    ++c->launches;
    k_bonded<<<nblk(c->M, 256), 256, 0, c->stream>>>(c->d_sim, c->slot_of, c->comp_of, c->bp);
}

// Re-sort the per-monomer state into the cell order of the last Verlet build.
// The list then refers to the old order, so a rebuild is requested.
void md_sort(kg_ctx *c)
{
    md_materialize(c);
    const int Mp = c->Mp;
    double *sx = c->scratch;
    int *spid = (int *)(c->scratch + 6 * (size_t)Mp);
    int *sslot = spid + Mp;
    c->launches += 2;
    if (c->precision == KG_MIXED) {
        float *su = (float *)(c->scratch + 3 * (size_t)Mp);
        k_sort_gather<float><<<nblk(c->M, 256), 256, 0, c->stream>>>(c->M, Mp, c->clist, c->x, (const float *)c->u,
                                                                    c->pid, c->slot_of, sx, su, spid, sslot);
        k_sort_finish<float><<<nblk(c->M, 256), 256, 0, c->stream>>>(c->M, Mp, c->x, (float *)c->u, c->pid,
                                                                    c->slot_of, c->comp_of, sx, su, spid, sslot);
    } else {
        double *su = c->scratch + 3 * (size_t)Mp;
        k_sort_gather<double><<<nblk(c->M, 256), 256, 0, c->stream>>>(c->M, Mp, c->clist, c->x,
                                                                     (const double *)c->u, c->pid, c->slot_of, sx,
                                                                     su, spid, sslot);
        k_sort_finish<double><<<nblk(c->M, 256), 256, 0, c->stream>>>(c->M, Mp, c->x, (double *)c->u, c->pid,
                                                                     c->slot_of, c->comp_of, sx, su, spid, sslot);
    }
    if (c->precision == KG_MIXED) {    // sorted current positions become the build positions
        cudaMemcpyAsync(c->xb64, c->x, 3 * (size_t)Mp * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
        cudaMemsetAsync(c->dlt[c->cur], 0, (size_t)Mp * sizeof(float4), c->stream);
    }
    msd_permute(c, c->clist);
    bonded_partners(c);
    static const unsigned one = 1u;
    cudaMemcpyAsync(c->flags + 1, &one, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream);
}

// mixed: current binary64 positions x = xb64 + dlt[cur] (the same sum as the
// build's fold, so a later build finds the same values)
__global__ void __launch_bounds__(256) k_materialize(double *__restrict__ x, const double *__restrict__ xb64,
                                                    const float4 *__restrict__ d, int M, int Mp)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const float4 e = d[s];
    x[s] = xb64[s] + (double)e.x;
    x[Mp + s] = xb64[Mp + s] + (double)e.y;
    x[2 * Mp + s] = xb64[2 * Mp + s] + (double)e.z;
}

void md_materialize(kg_ctx *c)
{
    if (c->precision != KG_MIXED) return;
    ++c->launches;
    k_materialize<<<nblk(c->M, 256), 256, 0, c->stream>>>(c->x, c->xb64, c->dlt[c->cur], c->M, c->Mp);
}

void to_slots(kg_ctx *c, int melt, const double *in_comp, double *out_dev, int dims)
{
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    k_to_slots<<<nblk(md.M, 256), 256, 0, c->stream>>>(in_comp, c->Mp, c->comp_of, md.off, md.M, out_dev, md.M,
                                                       dims);
}

void u_to_slots(kg_ctx *c, int melt, double *out_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    if (c->precision == KG_MIXED)
        k_to_slots_f<<<nblk(md.M, 256), 256, 0, c->stream>>>((const float *)c->u, c->Mp, c->comp_of, md.off, md.M,
                                                             out_dev, md.M);
    else
        k_to_slots<<<nblk(md.M, 256), 256, 0, c->stream>>>((const double *)c->u, c->Mp, c->comp_of, md.off, md.M,
                                                           out_dev, md.M, 3);
}

void pid_to_slots(kg_ctx *c, int melt, int *out_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    k_to_slots_i<<<nblk(md.M, 256), 256, 0, c->stream>>>(c->pid, c->comp_of, md.off, md.M, out_dev);
}

// First kernel of every MD step: advance the device step counter (the index
// of the step about to run) and, inside a captured graph, arm the conditional
// rebuild node with the rebuild request.
__global__ void k_begin_step(long long *__restrict__ stepp, unsigned *__restrict__ flags,
                             cudaGraphConditionalHandle h, int armed)
{
    stepp[0] += 1;
    if (armed) {
        const unsigned go = (flags[1] && !flags[0]) ? 1u : 0u;
        cudaGraphSetConditional(h, go);
        flags[6] += go;                        // rebuild bodies run inside graphs
    }
}

__global__ void k_set_step(long long *__restrict__ stepp, long long v) { stepp[0] = v; }

static void launch_rebuild(kg_ctx *c, cudaStream_t st);

void rebuild_md(kg_ctx *c)
{
    c->launches += 6;
    launch_rebuild(c, c->stream);
}

NlArgs nl_args(const kg_ctx *c)
{
    NlArgs a{};
    a.x = c->x;
    a.recb = c->recb;
    a.recs = c->recs;
    a.start = c->cstart;
    a.nl = c->nl;
    a.nn = c->nn;
    a.flags = c->flags;
    a.slot_of = c->slot_of;
    a.bp = c->bp;
    a.M = c->M;
    a.Mp = c->Mp;
    a.maxnb = c->maxnb;
    a.n_melts = c->sim.n_melts;
    a.rl2 = c->sim.rl2;
    for (int m = 0; m < c->sim.n_melts; ++m) {
        const MeltDev &md = c->sim.melt[m];
        a.melt[m] = MeltNl{md.off, md.cell_off, md.nbk, md.nc, md.hf, md.nl_lo, md.nl_hi, md.L};
    }
    return a;
}

static void launch_rebuild(kg_ctx *c, cudaStream_t st)
{
    const bool mixed = c->precision == KG_MIXED;
    k_bin_md<<<nblk(c->M, 256), 256, 0, st>>>(c->d_sim, c->x, mixed ? c->xb64 : nullptr, c->recb,
                                              mixed ? c->dlt[c->cur] : nullptr,
                                              mixed ? c->pg[c->cur] : nullptr, mixed ? nullptr : c->pos64[c->cur],
                                              c->xb, c->cellid, c->rank, c->ccount, c->slot_of, c->flags);
    const int nb = nblk(c->ncell_md, 1024);
    k_scan1<<<nb, 1024, 0, st>>>(c->ccount, c->cstart, c->bsum, c->ncell_md, c->flags);
    k_scan2<<<nb, 1024, 0, st>>>(c->cstart, c->bsum, c->ncell_md, nb, c->flags);
    k_scatter<<<nblk(c->M, 256), 256, 0, st>>>(c->cellid, c->rank, c->cstart, c->ctmp, c->M, c->flags);
    k_cellrank<<<nblk(c->M, 256), 256, 0, st>>>(c->cellid, c->cstart, c->ctmp, c->clist, c->recb, c->recs, c->ccount,
                                                c->M, c->flags);
    k_nlist<<<nblk(c->M, NL_BLOCK), NL_BLOCK, 0, st>>>(nl_args(c));
}

static void launch_step_kernel(kg_ctx *c, cudaStream_t st, int cur)
{
    if (c->precision == KG_MIXED) {
        step_mixed_launch(c, st, cur);
        return;
    }
    const int nb = nblk(c->M, c->block);
    k_step_f64<<<nb, c->block, 0, st>>>(c->d_sim, c->d_stage, c->x, (double *)c->u, c->pos64[cur], c->pos64[cur ^ 1],
                                        c->xb, c->nl, c->nn, c->slot_of, c->bp, c->flags, c->d_step);
}

// Captured graphs hold the step kernel's by-value arguments (stage
// parameters among them): drop them when those change.
void graphs_reset(kg_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->gexec[k]) {
            cudaGraphExecDestroy(c->gexec[k]);
            c->gexec[k] = nullptr;
        }
        if (c->pexec[k]) {
            cudaGraphExecDestroy(c->pexec[k]);
            c->pexec[k] = nullptr;
        }
    }
}

// PERSIST_STEPS MD steps as one captured graph holding the persistent
// cooperative launch (the barrier words reset first); one graph per starting
// buffer parity.  False if capture or launch is not possible.
bool md_persist_steps(kg_ctx *c)
{
    const int parity = c->cur;
    if (!c->pexec[parity]) {
        if (c->persist_failed) return false;
        if (!c->cap_stream) {
            if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking) != cudaSuccess) {
                c->persist_failed = true;
                return false;
            }
        }
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) ok = persist_launch(c, c->cap_stream, parity, PERSIST_STEPS, -1, PERSIST_SPIN) == cudaSuccess;
        const bool ended = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess;
        ok = ok && ended && cudaGraphInstantiate(&c->pexec[parity], g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            c->pexec[parity] = nullptr;
            c->persist_failed = true;
            return false;
        }
    }
    if (cudaGraphLaunch(c->pexec[parity], c->stream) != cudaSuccess) return false;
    c->launches += 2;                          // barrier reset + the persistent kernel
    c->cur ^= PERSIST_STEPS & 1;
    return true;
}

void set_device_step(kg_ctx *c, long long v)
{
    ++c->launches;
    k_set_step<<<1, 1, 0, c->stream>>>(c->d_step, v);
}

// One MD step: the Verlet list is rebuilt first if the previous step (or a
// configuration load or an accepted swap) asked for it.
void prof_collect(kg_ctx *c)
{
    if (!c->ev_used) return;
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < c->ev_used; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]);
        c->prof_ms += ms;
    }
    c->prof_n += c->ev_used;
    c->ev_used = 0;
}

void md_step(kg_ctx *c)
{
    k_begin_step<<<1, 1, 0, c->stream>>>(c->d_step, c->flags, cudaGraphConditionalHandle{}, 0);
    ++c->launches;
    rebuild_md(c);
    cudaEvent_t e1 = nullptr;
    if (c->prof_on) {
        if (c->ev.empty()) {
            c->ev.resize(2 * 1024);
            for (auto &e : c->ev) cudaEventCreate(&e);
        }
        if (2 * c->ev_used >= (int)c->ev.size()) prof_collect(c);
        cudaEventRecord(c->ev[2 * c->ev_used], c->stream);
        e1 = c->ev[2 * c->ev_used + 1];
        ++c->ev_used;
    }
    ++c->launches;
    launch_step_kernel(c, c->stream, c->cur);
    if (e1) cudaEventRecord(e1, c->stream);
    c->cur ^= 1;
}

// A CUDA graph of GRAPH_STEPS MD steps: per step, the begin kernel, a
// conditional node holding the rebuild chain (run only when a rebuild was
// requested), and the fused step kernel.  GRAPH_STEPS is even, so a replay
// leaves the ping-pong buffers as it found them; one graph per starting buffer.
static bool capture_graph(kg_ctx *c, int parity)
{
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = cudaStreamBeginCaptureToGraph(c->cap_stream, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int cur = parity;
    for (int i = 0; ok && i < GRAPH_STEPS; ++i) {
        cudaGraphConditionalHandle h;
        ok = cudaGraphConditionalHandleCreate(&h, g, 0, 0) == cudaSuccess;
        if (!ok) break;
        k_begin_step<<<1, 1, 0, c->cap_stream>>>(c->d_step, c->flags, h, 1);
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        ok = cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess;
        if (!ok) break;
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        ok = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp) == cudaSuccess &&
             cudaStreamUpdateCaptureDependencies(c->cap_stream, &cn, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies) == cudaSuccess;
        if (!ok) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(c->cap_stream2, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (!ok) break;
        const int save = c->cur;
        c->cur = cur;
        launch_rebuild(c, c->cap_stream2);
        c->cur = save;
        ok = cudaStreamEndCapture(c->cap_stream2, &body) == cudaSuccess;
        if (!ok) break;
        launch_step_kernel(c, c->cap_stream, cur);
        cur ^= 1;
    }
    cudaGraph_t out = nullptr;
    const bool ended = cudaStreamEndCapture(c->cap_stream, &out) == cudaSuccess;
    ok = ok && ended && cudaGetLastError() == cudaSuccess &&
         cudaGraphInstantiate(&c->gexec[parity], g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        c->gexec[parity] = nullptr;
    }
    return ok;
}

bool md_graph_steps(kg_ctx *c, long long nrep)
{
    const int parity = c->cur;
    if (!c->gexec[parity]) {
        if (c->graph_failed) return false;
        if (!c->cap_stream) {
            if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking) != cudaSuccess) {
                c->graph_failed = true;
                return false;
            }
        }
        if (!capture_graph(c, parity)) {
            c->graph_failed = true;
            return false;
        }
    }
    for (long long r = 0; r < nrep; ++r) {
        if (cudaGraphLaunch(c->gexec[parity], c->stream) != cudaSuccess) return false;
        c->launches += 2 * GRAPH_STEPS;        // begin + step kernels; executed rebuilds counted on the device
        ++c->graph_replays;
    }
    return true;
}

int forces_blocks(const kg_ctx *c, int melt) { return nblk(c->sim.melt[melt].M, 128); }

void forces_eval(kg_ctx *c, int melt, long long step, double *F_dev, double *part_dev, int nb)
{
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    if (c->precision == KG_MIXED) {
        GeoMixed g{c->pg[c->cur], c->shtab};
        k_forces<GeoMixed><<<nb, 128, 0, c->stream>>>(c->d_sim, c->d_stage, g, c->u, md.off, md.off + md.M,
                                                     c->nl, c->nn, c->slot_of, c->bp, F_dev, part_dev, c->flags, step);
    } else {
        GeoF64 g{c->pos64[c->cur], 0.0, 0.0, {}};
        k_forces<GeoF64><<<nb, 128, 0, c->stream>>>(c->d_sim, c->d_stage, g, c->u, md.off, md.off + md.M,
                                                   c->nl, c->nn, c->slot_of, c->bp, F_dev, part_dev, c->flags, step);
    }
}

}  // namespace kg
