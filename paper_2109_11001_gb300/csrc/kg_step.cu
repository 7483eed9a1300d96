// kg_step.cu -- the fused MD step of the mixed-precision path (binary32 forces,
// binary64 positions folded from a binary32 displacement at list builds).
//
// One step: U_MLJ^n pair forces over the Verlet list (Eqs. 5-6, truncated and
// shifted at r_c = 2^(1/6)), U_bond^n = U_MLJ^n + FENE bonds (Eq. 10),
// kappa (1 - cos theta) bending (Eq. 4), Langevin friction and Philox noise,
// then the leapfrog update u += dt F, x += dt u (velocity Verlet on the state
// (x_n, u = v_{n-1/2})).
//
// Instruction issue and load latency bound this kernel (its arithmetic per
// byte is low, but the per-entry work of the pair loop is issued for every
// lane of a warp up to the warp's longest list):
//  * every parameter is a by-value kernel argument (constant bank operands,
//    no loads, no registers held for them); a captured graph bakes them in,
//    so graphs are re-captured when the stage changes;
//  * the pair potential is a template on 4n, so each stage of Xi (Eq. 11)
//    gets its own straight-line r^-n;
//  * the pair loop runs to the warp's longest list with per-lane predicates
//    (no divergent loop exits), ILP list entries in flight;
//  * the image shift of an entry's stencil code q is read from three
//    shared-memory word tables of the cell offsets (-1, 0, 1), one per axis
//    (entry q in bank q: conflict-free, three wavefronts where a float4
//    table took about five; the L1 data pipe is this kernel's busiest unit)
//    and scaled by the melt's cell side with one FMA per component;
//  * latency is hidden by resident warps: the pair loop runs before the
//    bonded terms and the noise, holding only its own state, so the kernel
//    fits 32 registers at full occupancy.
#include <cuda_runtime.h>

#include <cmath>

#include "kg_host.h"
#include "kg_rebuild.cuh"

namespace kg {

struct MeltStep {
    int off, nc;
    float h, L, invL, kappa;
};

struct StepArgs {
    const float4 *recb;      // build records: offset from the Verlet-cell corner, packed cell coordinates
    const float4 *dcur;      // displacement since the build (this step)
    float4 *dnext;           //   ... after this step
    const float4 *pcur;      // gather records recb + dcur
    float4 *pnext;           //   ... after this step
    float *u;                // [3][Mp] velocities v_{n-1/2}
    const unsigned *nl;      // Verlet list, column-major [maxnb][Mp], entries j | q << IDX_BITS
    const int *nn;           // list lengths
    const int *slot_of;      // compute index -> chain-major slot (keys the noise)
    const int4 *bp;          // compute indices of chain partners s-2, s-1, s+1, s+2 (-1 past an end)
    unsigned *flags;         // [0] error bits, [1] rebuild request
    const long long *stepp;  // index of the step being run
    unsigned long long seed;
    int M, Mp, n_melts;
    float rc2, half_skin2;
    float dt, gamma, amp;    // Langevin: u += dt (F - gamma u + amp g), amp = sqrt(2 gamma T / dt)
    float c1xn, c2x6, nf;    // fr = (6 c2 r^-6 - n c1 r^-n) / r^2  (U = c1 r^-n - c2 r^-6 + 1)
    float kf, R0sq, inv_R0sq, qmin, kf_qmin, four_R0sq;   // FENE k_n, R0^2, continuation beyond r*
    MeltStep melt[MAX_MELTS];
};

// r^-n from r^2, 1/r^2 and 1/r^6; N4 = 4n (0: any other n, from exp2/log2)
template <int N4>
__device__ __forceinline__ float inv_rn(float r2, float ir2, float ir6, float nf)
{
    if constexpr (N4 == 0) {
        return exp2f(-0.5f * nf * log2f(r2));
    } else if constexpr (N4 == 23) {                 // n = 23/4: r^-6 r^(1/4)
        return ir6 * sqrtf(sqrtf(sqrtf(r2)));
    } else if constexpr (N4 == 26) {                 // n = 13/2: r^-6 r^(-1/2)
        return ir6 * sqrtf(rsqrtf(r2));
    } else {
        static_assert(N4 % 4 == 0, "integer n");
        constexpr int n = N4 / 4;
        float p;
        if constexpr (n >= 6) {
            p = ir6;
#pragma unroll
            for (int k = 3; k < n / 2; ++k) p *= ir2;
        } else {
            p = ir2;
#pragma unroll
            for (int k = 1; k < n / 2; ++k) p *= ir2;
        }
        if constexpr (n & 1) p *= rsqrtf(r2);
        return p;
    }
}

// (dU_MLJ^n/dr) / r at r^2 (binary32)
template <int N4>
__device__ __forceinline__ float mlj_fr32(const StepArgs &P, float r2)
{
    const float ir2 = __fdividef(1.0f, r2);
    const float ir6 = ir2 * ir2 * ir2;
    const float rn = inv_rn<N4>(r2, ir2, ir6, P.nf);
    return __fmul_rn(fmaf(P.c2x6, ir6, -__fmul_rn(P.c1xn, rn)), ir2);
}

__device__ __forceinline__ int melt_index(const StepArgs &P, int slot)
{
    int m = 0;
    while (m + 1 < P.n_melts && slot >= P.melt[m + 1].off) ++m;
    return m;
}

// Arithmetic of the step written with explicit roundings: a sum of two
// products leaves the compiler a choice of which one to fuse, and the choice
// can differ between the kernels that inline the step (standalone and
// persistent), which must give the same bits.  fmaf is always fused,
// __fmul_rn / __fadd_rn / __fsub_rn never.
__device__ __forceinline__ float dot3(float3 a, float3 b)
{
    return fmaf(a.z, b.z, fmaf(a.y, b.y, __fmul_rn(a.x, b.x)));
}

__device__ __forceinline__ void axpy3(float a, float3 x, float3 &y)   // y += a x
{
    y.x = fmaf(a, x.x, y.x);
    y.y = fmaf(a, x.y, y.y);
    y.z = fmaf(a, x.z, y.z);
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b)
{
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}

// a inv - c b: one term of the gradient of cos theta
__device__ __forceinline__ float3 bend_g(float3 a, float inv, float c, float3 b)
{
    return make_float3(fmaf(-c, b.x, __fmul_rn(a.x, inv)), fmaf(-c, b.y, __fmul_rn(a.y, inv)),
                       fmaf(-c, b.z, __fmul_rn(a.z, inv)));
}

// Bond (Eq. 10) and bending (Eq. 4) forces on the monomer whose gather
// record is pi, from its chain partners bp = (s-2, s-1, s+1, s+2).
template <int N4>
__device__ __forceinline__ void bonded32(const StepArgs &P, const float4 *__restrict__ pcur, const MeltStep &md,
                                         float4 pi, int4 bp, float3 &F, unsigned &err)
{
    const bool hm2 = bp.x >= 0, hm1 = bp.y >= 0, hp1 = bp.z >= 0, hp2 = bp.w >= 0;
    float3 rm2 = make_float3(0.f, 0.f, 0.f), rm1 = rm2, rp1 = rm2, rp2 = rm2;
    if (hm1) rm1 = rec_rel(pi, __ldg(pcur + bp.y), md.nc, md.h, md.L, md.invL);
    if (hm2) rm2 = rec_rel(pi, __ldg(pcur + bp.x), md.nc, md.h, md.L, md.invL);
    if (hp1) rp1 = rec_rel(pi, __ldg(pcur + bp.z), md.nc, md.h, md.L, md.invL);
    if (hp2) rp2 = rec_rel(pi, __ldg(pcur + bp.w), md.nc, md.h, md.L, md.invL);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if (side == 0 ? hm1 : hp1) {
            const float3 d = side == 0 ? rm1 : rp1;
            const float r2 = dot3(d, d);
            float q = 1.0f - r2 * P.inv_R0sq, fr;
            if (P.qmin > 0.0f && q < P.qmin) {          // continuation beyond r* (kg_params.fene_qmin)
                fr = P.kf_qmin;
                if (!(r2 < P.four_R0sq)) err |= ERR_OVERSTRETCH;
            } else {
                if (!(r2 < P.R0sq)) err |= ERR_OVERSTRETCH;
                q = fmaxf(q, 1e-6f);                    // finite even when flagged
                fr = P.kf * __fdividef(1.0f, q);
            }
            const float fl = mlj_fr32<N4>(P, r2);
            fr += r2 < P.rc2 ? fl : 0.0f;
            axpy3(fr, d, F);
        }
    }
    const float kap = md.kappa;
    if (kap != 0.0f) {
        const float3 Bm2 = sub3(rm1, rm2);
        const float3 Bm1 = make_float3(-rm1.x, -rm1.y, -rm1.z), B0 = rp1;
        const float3 Bp1 = sub3(rp2, rp1);
        if (hm1 && hp1) {                     // vertex s: force kappa (g1 - g2)
            const float l1 = dot3(Bm1, Bm1), l2 = dot3(B0, B0);
            const float inv = rsqrtf(__fmul_rn(l1, l2)), cs = __fmul_rn(dot3(Bm1, B0), inv);
            const float c1 = __fmul_rn(cs, __fdividef(1.0f, l1)), c2 = __fmul_rn(cs, __fdividef(1.0f, l2));
            axpy3(kap, sub3(bend_g(B0, inv, c1, Bm1), bend_g(Bm1, inv, c2, B0)), F);
        }
        if (hp2) {                            // vertex s+1, s its first end: -kappa g1
            const float l1 = dot3(B0, B0), l2 = dot3(Bp1, Bp1);
            const float inv = rsqrtf(__fmul_rn(l1, l2)), cs = __fmul_rn(dot3(B0, Bp1), inv);
            const float c1 = __fmul_rn(cs, __fdividef(1.0f, l1));
            axpy3(-kap, bend_g(Bp1, inv, c1, B0), F);
        }
        if (hm2) {                            // vertex s-1, s its last end: +kappa g2
            const float l1 = dot3(Bm2, Bm2), l2 = dot3(Bm1, Bm1);
            const float inv = rsqrtf(__fmul_rn(l1, l2)), cs = __fmul_rn(dot3(Bm2, Bm1), inv);
            const float c2 = __fmul_rn(cs, __fdividef(1.0f, l2));
            axpy3(kap, bend_g(Bm2, inv, c2, Bm1), F);
        }
    }
}

constexpr int STEP_ILP = 4;      // Verlet-list entries in flight per lane
// One tile of blockDim threads (all threads of the block call it together):
// the step of the monomers of threads t0 + threadIdx.x.  TPM threads per
// monomer (1 or 2, adjacent lanes): the lanes split the list (entries k =
// sub, sub + TPM, ...); with two, lane 0 adds the bonded terms and lane 1
// draws the noise, the forces are combined with a shuffle, and lane 0 writes
// the state.  The pair loop comes first and holds only its own state (the
// own gather record, the force, the entries in flight), so the kernel fits
// 32 registers at full occupancy; the bonded terms, the noise and the build
// record and displacement for the update follow.  The pair loop runs to the
// warp's longest list in groups of STEP_ILP entries with per-lane
// predicates: an entry past the lane's own list becomes the lane's own record
// with the zero shift (code 13), a valid gather whose term is masked.
template <int N4, int TPM>
__device__ __forceinline__ void step_tile(const StepArgs &P, int t0, const float4 *__restrict__ dcur,
                                          float4 *__restrict__ dnext, const float4 *__restrict__ pcur,
                                          float4 *__restrict__ pnext, long long step, const float *dk)
{
    const int lane = threadIdx.x & 31;
    const int t = t0 + threadIdx.x;
    const int s = t / TPM, sub = t % TPM;
    const bool live = s < P.M;
    const int cnt = live ? __ldg(P.nn + s) : 0;
    const int kmax = __reduce_max_sync(0xffffffffu, cnt);
    unsigned err = 0;
    float3 F = make_float3(0.f, 0.f, 0.f), gn = F;
    int slot = 0, m = 0;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        slot = __ldg(P.slot_of + s);
        m = melt_index(P, slot);
        pi = __ldg(pcur + s);
    }
    const MeltStep &md = P.melt[m];
    const float h = md.h, rc2 = P.rc2;
    const unsigned self = (unsigned)(live ? s : 0) | (13u << IDX_BITS);
    const size_t Mp = (size_t)P.Mp;
    const unsigned *__restrict__ col = P.nl + (live ? s : 0);
    for (int k0 = sub; k0 < kmax; k0 += STEP_ILP * TPM) {
        unsigned e[STEP_ILP];
        float4 pj[STEP_ILP];
#pragma unroll
        for (int i = 0; i < STEP_ILP; ++i) {
            const int k = k0 + i * TPM;
            e[i] = k < cnt ? __ldg(col + (size_t)k * Mp) : self;
        }
#pragma unroll
        for (int i = 0; i < STEP_ILP; ++i) pj[i] = __ldg(pcur + (e[i] & IDX_MASK));
#pragma unroll
        for (int i = 0; i < STEP_ILP; ++i) {
            const unsigned q = e[i] >> IDX_BITS;
            const float dx = fmaf(dk[q], h, pj[i].x - pi.x);
            const float dy = fmaf(dk[32 + q], h, pj[i].y - pi.y);
            const float dz = fmaf(dk[64 + q], h, pj[i].z - pi.z);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
            float fr = mlj_fr32<N4>(P, r2);
            fr = (k0 + i * TPM < cnt && r2 < rc2) ? fr : 0.0f;
            F.x = fmaf(fr, dx, F.x); F.y = fmaf(fr, dy, F.y); F.z = fmaf(fr, dz, F.z);
        }
    }
    float4 rb = make_float4(0.f, 0.f, 0.f, 0.f), dc = rb;
    if (live) {
        if (sub == 0) bonded32<N4>(P, pcur, md, pi, __ldg(P.bp + s), F, err);
        if (sub == TPM - 1)
            gn = gauss3_f(draw(P.seed, m, 0, (unsigned long long)step, (uint32_t)(slot - md.off)));
        rb = __ldg(P.recb + s);
        dc = __ldg(dcur + s);
    }
    if (TPM == 2) {                        // every lane takes part: s is shared by lanes 2i, 2i+1
        F.x += __shfl_xor_sync(0xffffffffu, F.x, 1);
        F.y += __shfl_xor_sync(0xffffffffu, F.y, 1);
        F.z += __shfl_xor_sync(0xffffffffu, F.z, 1);
        const int src = lane | 1;
        gn.x = __shfl_sync(0xffffffffu, gn.x, src);
        gn.y = __shfl_sync(0xffffffffu, gn.y, src);
        gn.z = __shfl_sync(0xffffffffu, gn.z, src);
    }
    bool rebuild = false;
    if (live && sub == 0) {
        const int Mpi = P.Mp;
        float *__restrict__ u = P.u;
        float3 v = make_float3(u[s], u[Mpi + s], u[2 * Mpi + s]);
        v.x = fmaf(P.dt, fmaf(P.amp, gn.x, fmaf(-P.gamma, v.x, F.x)), v.x);
        v.y = fmaf(P.dt, fmaf(P.amp, gn.y, fmaf(-P.gamma, v.y, F.y)), v.y);
        v.z = fmaf(P.dt, fmaf(P.amp, gn.z, fmaf(-P.gamma, v.z, F.z)), v.z);
        u[s] = v.x; u[Mpi + s] = v.y; u[2 * Mpi + s] = v.z;
        float4 d = dc;
        d.x = fmaf(P.dt, v.x, d.x); d.y = fmaf(P.dt, v.y, d.y); d.z = fmaf(P.dt, v.z, d.z);
        dnext[s] = d;
        pnext[s] = make_float4(rb.x + d.x, rb.y + d.y, rb.z + d.z, rb.w);
        rebuild = fmaf(d.z, d.z, fmaf(d.y, d.y, __fmul_rn(d.x, d.x))) > P.half_skin2;
        if (!isfinite(v.x + v.y + v.z)) err |= ERR_NONFINITE;
    }
    // the rebuild vote per warp (no block barrier: a warp with short lists
    // leaves without waiting for the block's longest)
    if (__any_sync(0xffffffffu, rebuild) && lane == 0) atomicOr(P.flags + 1, 1u);
    if (err) atomicOr(P.flags, err);
}

// per-block setup of the step body: the stencil offsets of the 27 codes,
// one table per axis
__device__ __forceinline__ void step_block_setup(float *dk)
{
    if (threadIdx.x < 27) {
        const int q = threadIdx.x;
        dk[q] = (float)(q % 3 - 1);
        dk[32 + q] = (float)((q / 3) % 3 - 1);
        dk[64 + q] = (float)(q / 9 - 1);
    }
}

// One MD step of every monomer.  (256, 8): at most 32 registers, full
// occupancy (a few bytes spilled after the pair loop).  Measured at 1.6M
// monomers (skin 0.5, n = 12): 94.5 us per launch, against 101.3 at 40
// registers and 97.1 at 48; with the bonded terms before the pair loop it
// needed 48 registers and took 103.5 us.
template <int N4, int TPM>
__global__ void __launch_bounds__(256, 8) k_step32(const __grid_constant__ StepArgs P)
{
    __shared__ float dk[96];
    __shared__ unsigned stop;
    step_block_setup(dk);
    if (threadIdx.x == 0) stop = *(volatile unsigned *)P.flags;    // a latched error stops the run
    __syncthreads();
    if (stop) return;                                              // block-uniform
    step_tile<N4, TPM>(P, blockIdx.x * blockDim.x, P.dcur, P.dnext, P.pcur, P.pnext, *P.stepp, dk);
}

// ---------------------------------------------------------------------------
// persistent launch: K MD steps of every melt in one cooperative kernel.  The
// blocks stay resident and walk the work in grid-stride loops; a grid barrier
// separates the step of one timestep from the next and, when a step asked
// for it, the phases of the Verlet rebuild (bin, scan of the cell counts in
// two passes, scatter into cell order, in-cell rank, list).  The barrier's
// last arriver snapshots the error and rebuild words, so every block takes
// the same decisions.  Every barrier wait is bounded: a block that polls
// longer than `spin` latches ERR_TIMEOUT and leaves the kernel.
// ---------------------------------------------------------------------------
struct PersistArgs {
    StepArgs st;                 // its dcur/dnext/pcur/pnext are ignored: the buffers alternate below
    NlArgs nl;
    const SimDev *sim;           // device copy of the melt table (binning)
    float4 *dlt[2], *pg[2];      // displacement and gather buffers, ping-pong
    double *x, *xb64;
    float4 *recb, *recs;
    int *cellid, *rank, *ccount, *cstart, *clist, *ctmp, *bsum;
    int ncell, cur0, K, skip_block;   // skip_block >= 0: that block never arrives (barrier self-test)
    unsigned *bar;               // [0] arrivals, [1] generation, [2] error word and [3] rebuild word at release
    unsigned spin;               // barrier polls before giving up
    long long *stepp;            // device step counter: the last step run
};

// Grid barrier; false if this block gave up waiting.  *snap receives the
// error word (bit 0..) and rebuild request as the last arriver saw them.
__device__ __forceinline__ bool grid_sync(const PersistArgs &A, unsigned *ok_s, uint2 *snap_s)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vb = A.bar;
        const unsigned g = vb[1];
        __threadfence();
        bool ok = true;
        if (atomicAdd(A.bar, 1u) == gridDim.x - 1) {
            vb[2] = *(volatile unsigned *)A.st.flags;
            vb[3] = *((volatile unsigned *)A.st.flags + 1);
            atomicExch(A.bar, 0u);
            __threadfence();
            atomicAdd(A.bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (vb[1] == g) {
                if (++it > A.spin) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *ok_s = ok ? 1u : 0u;
        *snap_s = make_uint2(vb[2], vb[3]);
        if (!ok) atomicOr(A.st.flags, ERR_TIMEOUT);
    }
    __syncthreads();
    return *ok_s != 0;
}

// exclusive scan of the cell counts, pass 1: segment g of 1024 counts, 256
// threads x 4; segment total to bsum[g]
__device__ __forceinline__ void scan_seg(const PersistArgs &A, int g, int *wsum)
{
    const int n = A.ncell, i0 = g * 1024 + threadIdx.x * 4;
    int v[4], tsum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = i0 + k < n ? A.ccount[i0 + k] : 0;
        tsum += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int ws = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += u;
        }
        if (lane < (int)(blockDim.x >> 5)) wsum[lane] = ws;
    }
    __syncthreads();
    int run = (w ? wsum[w - 1] : 0) + incl - tsum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < n) A.cstart[i0 + k] = run;
        run += v[k];
    }
    if (threadIdx.x == blockDim.x - 1) A.bsum[g] = run;
    __syncthreads();
}

// pass 2: add the totals of the preceding segments; cstart[n] = grand total
__device__ __forceinline__ void scan_fix(const PersistArgs &A, int g, int nseg, int *wsum)
{
    if (threadIdx.x < 32) {
        int acc = 0;
        for (int b = threadIdx.x; b < g; b += 32) acc += A.bsum[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) wsum[0] = acc;
    }
    __syncthreads();
    const int off = wsum[0], n = A.ncell;
    for (int k = threadIdx.x; k < 1024; k += blockDim.x) {
        const int i = g * 1024 + k;
        if (i < n) A.cstart[i] += off;
    }
    if (g == nseg - 1 && threadIdx.x == 0) {
        int tot = 0;
        for (int b = 0; b < nseg; ++b) tot += A.bsum[b];
        A.cstart[n] = tot;
    }
    __syncthreads();
}

constexpr int PERSIST_BLOCK = 256;

// One thread per monomer (the persistent launch does not split lists).
// (256, 5): at most 48 registers, as the standalone step and list kernels.
template <int N4>
__global__ void __launch_bounds__(PERSIST_BLOCK, 5) k_persist(const __grid_constant__ PersistArgs A)
{
    __shared__ float dk[96];
    __shared__ unsigned ok_s;
    __shared__ uint2 snap_s;
    __shared__ int wsum[32];
    step_block_setup(dk);
    const StepArgs &P = A.st;
    const long long base = *(volatile long long *)P.stepp;   // the last step run
    const int nthreads = gridDim.x * blockDim.x;
    const int nseg = (A.ncell + 1023) / 1024;
    if ((int)blockIdx.x == A.skip_block) return;              // barrier self-test: never arrives
    int it = 0;
    for (; it < A.K; ++it) {
        if (!grid_sync(A, &ok_s, &snap_s)) return;
        if (snap_s.x) break;                                  // a latched error stops the run
        const int cur = A.cur0 ^ (it & 1);
        if (snap_s.y) {                                       // Verlet rebuild
            for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.M; s += nthreads)
                bin_md_one(*A.sim, s, A.x, A.xb64, A.recb, A.dlt[cur], A.pg[cur], nullptr, nullptr, A.cellid, A.rank,
                           A.ccount, P.slot_of, P.flags);
            if (!grid_sync(A, &ok_s, &snap_s)) return;
            for (int g = blockIdx.x; g < nseg; g += gridDim.x) scan_seg(A, g, wsum);
            if (!grid_sync(A, &ok_s, &snap_s)) return;
            for (int g = blockIdx.x; g < nseg; g += gridDim.x) scan_fix(A, g, nseg, wsum);
            if (!grid_sync(A, &ok_s, &snap_s)) return;
            for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.M; s += nthreads)
                scatter_one(s, A.cellid, A.rank, A.cstart, A.ctmp);
            if (!grid_sync(A, &ok_s, &snap_s)) return;
            for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.M; p += nthreads)
                if (cellrank_one(p, A.cellid, A.cstart, A.ctmp, A.clist, A.recb, A.recs, A.ccount))
                    atomicOr(P.flags, ERR_NL_CAPACITY);
            if (!grid_sync(A, &ok_s, &snap_s)) return;
            for (int s0 = blockIdx.x * blockDim.x; s0 < P.Mp; s0 += nthreads) {    // whole warps
                const unsigned err = nlist_one(A.nl, s0 + threadIdx.x);
                if (err) atomicOr(P.flags, err);
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                P.flags[1] = 0u;                               // request served (before the next release)
                P.flags[5] += 1u;                              // Verlet builds completed
            }
            if (!grid_sync(A, &ok_s, &snap_s)) return;
            if (snap_s.x) break;
        }
        for (int t0 = blockIdx.x * blockDim.x; t0 < P.M; t0 += nthreads)     // block-uniform tiles
            step_tile<N4, 1>(P, t0, A.dlt[cur], A.dlt[cur ^ 1], A.pg[cur], A.pg[cur ^ 1], base + 1 + it, dk);
    }
    if (!grid_sync(A, &ok_s, &snap_s)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.stepp = base + it;
}

// 4n of a stage exponent with its own kernel instantiation, 0 otherwise
static int n4_of(double n)
{
    const double q = 4.0 * n;
    const int k = (int)std::lround(q);
    if (std::fabs(q - (double)k) > 1e-9) return 0;
    switch (k) {
        case 8: case 12: case 16: case 20: case 23: case 26: case 28:
        case 32: case 36: case 40: case 44: case 48: return k;
        default: return 0;
    }
}

template <int N4>
static void launch_n4(const StepArgs &a, int tpm, int block, long long M, cudaStream_t st)
{
    const int nb = (int)((tpm * M + block - 1) / block);
    if (tpm == 2) k_step32<N4, 2><<<nb, block, 0, st>>>(a);
    else k_step32<N4, 1><<<nb, block, 0, st>>>(a);
}

static StepArgs step_args(const kg_ctx *c, int cur)
{
    const StageDev &sg = c->stage;
    StepArgs a{};
    a.recb = c->recb;
    a.dcur = c->dlt[cur];
    a.dnext = c->dlt[cur ^ 1];
    a.pcur = c->pg[cur];
    a.pnext = c->pg[cur ^ 1];
    a.u = (float *)c->u;
    a.nl = c->nl;
    a.nn = c->nn;
    a.slot_of = c->slot_of;
    a.bp = c->bp;
    a.flags = c->flags;
    a.stepp = c->d_step;
    a.seed = c->sim.seed;
    a.M = c->M;
    a.Mp = c->Mp;
    a.n_melts = c->sim.n_melts;
    a.rc2 = c->sim.rc2f;
    a.half_skin2 = c->sim.half_skin2f;
    a.dt = sg.dtf;
    a.gamma = sg.gammaf;
    a.amp = sg.ampf;
    a.c1xn = sg.c1xnf;
    a.c2x6 = sg.c2x6f;
    a.nf = sg.nf;
    a.kf = sg.kfenef;
    a.R0sq = sg.R0sqf;
    a.inv_R0sq = (float)(1.0 / sg.R0sq);
    a.qmin = sg.qminf;
    a.kf_qmin = sg.qmin > 0 ? (float)(sg.kfene / sg.qmin) : 0.0f;
    a.four_R0sq = (float)(4.0 * sg.R0sq);
    for (int m = 0; m < c->sim.n_melts; ++m) {
        const MeltDev &md = c->sim.melt[m];
        a.melt[m] = MeltStep{md.off, md.nc, md.hf, md.Lf, md.invLf, md.kappaf};
    }
    return a;
}

void step_mixed_launch(kg_ctx *c, cudaStream_t st, int cur)
{
    const StepArgs a = step_args(c, cur);
    const int tpm = c->tpm, blk = c->block;
    const long long M = c->M;
    switch (n4_of(c->stage.n)) {
        case 8: launch_n4<8>(a, tpm, blk, M, st); break;
        case 12: launch_n4<12>(a, tpm, blk, M, st); break;
        case 16: launch_n4<16>(a, tpm, blk, M, st); break;
        case 20: launch_n4<20>(a, tpm, blk, M, st); break;
        case 23: launch_n4<23>(a, tpm, blk, M, st); break;
        case 26: launch_n4<26>(a, tpm, blk, M, st); break;
        case 28: launch_n4<28>(a, tpm, blk, M, st); break;
        case 32: launch_n4<32>(a, tpm, blk, M, st); break;
        case 36: launch_n4<36>(a, tpm, blk, M, st); break;
        case 40: launch_n4<40>(a, tpm, blk, M, st); break;
        case 44: launch_n4<44>(a, tpm, blk, M, st); break;
        case 48: launch_n4<48>(a, tpm, blk, M, st); break;
        default: launch_n4<0>(a, tpm, blk, M, st); break;
    }
}

NlArgs nl_args(const kg_ctx *c);                 // kg_md.cu

template <int N4>
static cudaError_t launch_persist(const PersistArgs &a, cudaStream_t st)
{
    const size_t smem = 0;
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist<N4>, PERSIST_BLOCK, smem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(per * nsm));
    cfg.blockDim = dim3(PERSIST_BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persist<N4>, a);
}

// K steps in one cooperative launch (barrier words reset first); skip_block
// >= 0 and a short spin are the barrier self-test.
cudaError_t persist_launch(kg_ctx *c, cudaStream_t st, int cur, int K, int skip_block, unsigned spin)
{
    PersistArgs a{};
    a.st = step_args(c, cur);
    a.nl = nl_args(c);
    a.sim = c->d_sim;
    for (int b = 0; b < 2; ++b) {
        a.dlt[b] = c->dlt[b];
        a.pg[b] = c->pg[b];
    }
    a.x = c->x;
    a.xb64 = c->xb64;
    a.recb = c->recb;
    a.recs = c->recs;
    a.cellid = c->cellid;
    a.rank = c->rank;
    a.ccount = c->ccount;
    a.cstart = c->cstart;
    a.clist = c->clist;
    a.ctmp = c->ctmp;
    a.bsum = c->bsum;
    a.ncell = c->ncell_md;
    a.cur0 = cur;
    a.K = K;
    a.skip_block = skip_block;
    a.bar = c->pbar;
    a.spin = spin;
    a.stepp = c->d_step;
    cudaError_t e = cudaMemsetAsync(c->pbar, 0, 4 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    switch (n4_of(c->stage.n)) {
        case 8: return launch_persist<8>(a, st);
        case 12: return launch_persist<12>(a, st);
        case 16: return launch_persist<16>(a, st);
        case 20: return launch_persist<20>(a, st);
        case 23: return launch_persist<23>(a, st);
        case 26: return launch_persist<26>(a, st);
        case 28: return launch_persist<28>(a, st);
        case 32: return launch_persist<32>(a, st);
        case 36: return launch_persist<36>(a, st);
        case 40: return launch_persist<40>(a, st);
        case 44: return launch_persist<44>(a, st);
        case 48: return launch_persist<48>(a, st);
        default: return launch_persist<0>(a, st);
    }
}

}  // namespace kg
