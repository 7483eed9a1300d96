// kg_rebuild.cuh -- per-item work of the Verlet-list rebuild chain (binning,
// scatter into cell order, in-cell rank, list build), shared by the
// standalone rebuild kernels and the persistent step kernel, so both run the
// same arithmetic.
#pragma once
#include <cuda_runtime.h>

#include "kg_internal.cuh"

namespace kg {

// finite binary64 value (exponent field not all ones), tested on the bits
__device__ __forceinline__ bool finite64(double v)
{
    return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}

// Monomer s: its position (mixed: build position + displacement since the
// build, folded into the binary64 arrays), its Verlet-grid cell and offset
// from the cell corner (the build record), the gather records reset to the
// record, and its rank within its cell (atomic count, aggregated per warp).
__device__ __forceinline__ void bin_md_one(const SimDev &S, int s, double *__restrict__ x, double *__restrict__ xb64,
                                           float4 *__restrict__ recb, float4 *__restrict__ dcur,
                                           float4 *__restrict__ pgcur, double4_32a *__restrict__ pcur,
                                           double4_32a *__restrict__ xb, int *__restrict__ cellid,
                                           int *__restrict__ rank, int *__restrict__ count,
                                           const int *__restrict__ slot_of, unsigned *__restrict__ flags)
{
    const MeltDev &md = S.melt[melt_of(S, slot_of[s])];
    const int Mp = S.Mp;
    double xs[3];
    if (xb64) {                        // mixed: the build position plus the displacement since
        const float4 e = dcur[s];
        xs[0] = __dadd_rn(xb64[s], (double)e.x);
        xs[1] = __dadd_rn(xb64[Mp + s], (double)e.y);
        xs[2] = __dadd_rn(xb64[2 * Mp + s], (double)e.z);
    } else {
        xs[0] = x[s];
        xs[1] = x[Mp + s];
        xs[2] = x[2 * Mp + s];
    }
    if (!(finite64(xs[0]) && finite64(xs[1]) && finite64(xs[2]))) {   // never bin a non-finite position
        atomicOr(flags, ERR_NONFINITE);
        return;
    }
    if (xb64) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xb64[d * Mp + s] = xs[d];
            x[d * Mp + s] = xs[d];     // the band check of the list build reads x
        }
    }
    float off[3];
    int cell[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) cell[d] = cell_of(xs[d], md.h, md.invh, md.nc, off[d]);
    const float4 rb = make_float4(off[0], off[1], off[2], __uint_as_float(pack_code(cell[0], cell[1], cell[2])));
    recb[s] = rb;
    if (dcur) {
        dcur[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        pgcur[s] = make_float4(rb.x + 0.f, rb.y + 0.f, rb.z + 0.f, rb.w);
    }
    if (pcur) {
        const double4_32a p = make_double4_32a(xs[0], xs[1], xs[2], 0.0);
        pcur[s] = p;
        xb[s] = p;
    }
    const int c = md_cell(md, cell[0], cell[1], cell[2]);
    cellid[s] = c;
    // one atomic per cell and warp: monomers in cell order share cells with
    // their lane neighbours (the in-cell order is fixed later by the rank pass)
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, c);
    const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count + c, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    rank[s] = base + __popc(grp & ((1u << lane) - 1u));
}

// Monomer s into its cell's segment of the cell-ordered list, at its
// arrival rank (the in-cell order is fixed afterwards).
__device__ __forceinline__ void scatter_one(int s, const int *__restrict__ cellid, const int *__restrict__ rank,
                                            const int *__restrict__ start, int *__restrict__ list)
{
    list[start[cellid[s]] + rank[s]] = s;
}

// Position p of the cell-ordered list: the monomer the scatter put there
// (in atomic-arrival order within its cell, tmp) moves to its rank by
// compute index among its cell's members, with its build record (w = the
// compute index), so a cell's candidates form one contiguous run in a fixed
// order (deterministic lists).  A cell's first position clears its count for
// the next build.  True if the cell holds more than MAX_CELL_OCC monomers
// (left in arrival order: an error).
__device__ __forceinline__ bool cellrank_one(int p, const int *__restrict__ cellid, const int *__restrict__ start,
                                             const int *__restrict__ tmp, int *__restrict__ list,
                                             const float4 *__restrict__ recb, float4 *__restrict__ recs,
                                             int *__restrict__ count)
{
    const int v = tmp[p];
    const int c = cellid[v];
    const int a = start[c], b = start[c + 1];
    if (p == a) count[c] = 0;
    const bool over = b - a > MAX_CELL_OCC;
    int r = p - a;
    if (!over) {
        r = 0;
        for (int q = a; q < b; ++q) r += tmp[q] < v ? 1 : 0;
    }
    list[a + r] = v;
    const float4 rb = recb[v];
    recs[a + r] = make_float4(rb.x, rb.y, rb.z, __int_as_float(v));
    return over;
}

// ---------------------------------------------------------------------------
// Verlet list of monomer s: every t != s, not 1-2 bonded, with r^2 < (r_c +
// skin)^2.  Candidates come from the 27 cells around the cell of s; a
// candidate j of stencil cell (dx, dy, dz) lies at off_j - (off_s - (dx, dy,
// dz) h) from s with no wrap, because that cell's image sits at (c_s + d) h.
// This binary32 value decides every pair outside the band [nl_lo, nl_hi),
// which bounds its rounding error; pairs inside the band are decided by the
// binary64 distance ((dx*dx + dy*dy) + dz*dz), dx = d - L rint(d/L), exactly
// as the definition.  Each entry stores j with its stencil code q, the image
// shift of the pair until the next build.
//
// A warp walks the 27 stencil cells in lockstep (all 32 lanes must call
// nlist_one together): for cell q every lane runs the warp's largest count of
// that cell; lanes past their own count load the records that follow their
// cell (recs is padded by MAX_CELL_OCC records past the last monomer, so
// every such load is in bounds) and mask them.  The candidate loop has no
// branch but its own: the append is a predicated store, and a pair inside the binary64
// band is taken provisionally and counted; a lane with band pairs re-walks
// its row after the stencil, decides each band entry by the binary64
// distance and compacts the row in place (order kept).  The candidate's
// offsets and compute index arrive in one 16-byte load.
// ---------------------------------------------------------------------------
struct MeltNl {
    int off, cell_off, nbk, nc;
    float h, lo, hi;
    double L;
};

struct NlArgs {
    const double *x;         // binary64 positions [3][Mp] (band decisions)
    const float4 *recb;      // build records of the compute order
    const float4 *recs;      // the same in cell order, w = compute index
    const int *start;        // cell starts (cell order)
    unsigned *nl;            // out: entries j | q << IDX_BITS, column-major [maxnb][Mp]
    int *nn;                 // out: list lengths
    unsigned *flags;
    const int *slot_of;
    const int4 *bp;          // chain partners (1-2 bonded: y, z)
    int M, Mp, maxnb, n_melts;
    double rl2;
    MeltNl melt[MAX_MELTS];
};

__device__ __forceinline__ void st_pred(unsigned *addr, unsigned v, bool p)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u32 [%0], %1;\n\t}"
                 ::"l"(addr), "r"(v), "r"((unsigned)p) : "memory");
}

// binary32 squared distance of the build records of s (ri) and t (rj) for a
// pair in stencil cell (dx, dy, dz) of s: the same expression as the build's
__device__ __forceinline__ float nl_r2(float4 ri, float4 rj, int dx, int dy, int dz, float h)
{
    const float ox = ri.x - (float)dx * h, oy = ri.y - (float)dy * h, oz = ri.z - (float)dz * h;
    const float ex = rj.x - ox, ey = rj.y - oy, ez = rj.z - oz;
    return ex * ex + ey * ey + ez * ez;
}

// The list of monomer s (s >= M: an idle lane that takes part in the warp's
// lockstep and writes nothing); returns error bits.
__device__ __forceinline__ unsigned nlist_one(const NlArgs &A, int s)
{
    constexpr unsigned FULL = 0xffffffffu;
    const bool live = s < A.M;
    const int sv = live ? s : A.M - 1;                       // idle lanes read valid memory, write nothing
    const int slot = __ldg(A.slot_of + sv);
    int m = 0;
    while (m + 1 < A.n_melts && slot >= A.melt[m + 1].off) ++m;
    const MeltNl &md = A.melt[m];
    const int4 bp = __ldg(A.bp + sv);                        // 1-2 bonded partners: bp.y, bp.z
    const float4 ri = __ldg(A.recb + sv);
    const unsigned code = __float_as_uint(ri.w);
    const int cx = (int)(code & CODE_MASK), cy = (int)((code >> CODE_BITS) & CODE_MASK);
    const int cz = (int)(code >> (2 * CODE_BITS));
    const int nc = md.nc, nbk = md.nbk;
    const float h = md.h, lo = md.lo, hi = md.hi;
    const int maxnb = A.maxnb;
    const size_t Mp = (size_t)A.Mp;
    unsigned *__restrict__ out = A.nl + (live ? s : 0);
    int cnt = 0, nband = 0;
    unsigned err = 0;
#pragma unroll 1
    for (int dz = -1; dz <= 1; ++dz) {
        int zz = cz + dz;
        zz = zz < 0 ? nc - 1 : (zz >= nc ? 0 : zz);
#pragma unroll 1
        for (int dy = -1; dy <= 1; ++dy) {
            int yy = cy + dy;
            yy = yy < 0 ? nc - 1 : (yy >= nc ? 0 : yy);
            const int rowb = md.cell_off + (((zz >> 2) * nbk + (yy >> 2)) * nbk << 6) + ((zz & 3) << 4) + ((yy & 3) << 2);
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                int xx = cx + dx;
                xx = xx < 0 ? nc - 1 : (xx >= nc ? 0 : xx);
                const int cell = rowb + ((xx >> 2) << 6) + (xx & 3);
                const int k0 = __ldg(A.start + cell);
                int n = live ? __ldg(A.start + cell + 1) - k0 : 0;
                if (n > MAX_CELL_OCC) {
                    err = ERR_NL_CAPACITY;
                    n = 0;
                }
                const int nmax = __reduce_max_sync(FULL, n);
                const float ox = ri.x - (float)dx * h, oy = ri.y - (float)dy * h, oz = ri.z - (float)dz * h;
                const unsigned tag = (unsigned)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)) << IDX_BITS;
#pragma unroll 2
                for (int j = 0; j < nmax; ++j) {
                    const float4 rj = __ldg(A.recs + k0 + j);
                    const int t = __float_as_int(rj.w);
                    const float ex = rj.x - ox, ey = rj.y - oy, ez = rj.z - oz;
                    const float r2 = ex * ex + ey * ey + ez * ez;
                    const bool take = (j < n) & (r2 < hi) & (t != s) & (t != bp.y) & (t != bp.z);
                    nband += (take & (r2 >= lo)) ? 1 : 0;
                    st_pred(out + (size_t)cnt * Mp, (unsigned)t | tag, take & (cnt < maxnb));
                    cnt += take ? 1 : 0;
                }
            }
        }
    }
    if (nband > 0 && cnt <= maxnb) {                         // rare: decide the band entries in binary64
        int w = 0;
        for (int k = 0; k < cnt; ++k) {
            const unsigned e = out[(size_t)k * Mp];
            const int t = (int)(e & IDX_MASK), q = (int)(e >> IDX_BITS);
            const float r2 = nl_r2(ri, __ldg(A.recb + t), q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1, h);
            const bool keep = r2 < lo || dist2_exact(A.x, A.Mp, md.L, s, t) < A.rl2;
            if (keep) out[(size_t)(w++) * Mp] = e;
        }
        cnt = w;
    }
    if (live) {
        A.nn[s] = cnt < maxnb ? cnt : maxnb;
        if (cnt > maxnb) {
            err |= ERR_NL_CAPACITY;
            atomicMax(A.flags + 3, (unsigned)cnt);
        }
    }
    return err;
}

}  // namespace kg
