// kg_internal.cuh -- device-side data layout and helpers of the GB300 DBH library.
//
// Layout in HBM (all melts of a context are concatenated slot ranges):
//   x        double[3][Mp]   canonical unwrapped positions (SoA)
//   u        float[3][Mp] (mixed) / double[3][Mp] (FP64): state velocity v_{n-1/2}
//   pid      int[Mp]         particle ids carried through double-bridging swaps
//   recb     float4[Mp]      build-time position record: offset from the corner
//                            of its Verlet-grid cell + packed cell coordinates
//   dlt[2]   float4[Mp]      (mixed) displacement since the last build, ping-pong
//   pg[2]    float4[Mp]      (mixed) gather record of the step: recb + dlt, code
//   pos64[2] double4_32a[Mp] (FP64) gather copy of the positions, ping-pong
//   xb       double4_32a[Mp] (FP64) positions at the last build
//   nl       uint[maxnb][Mp] Verlet list, column-major (coalesced per k); an
//                            entry is j | q << IDX_BITS, q the stencil cell
//                            (image shift) of j relative to the owner's cell
//   nn       int[Mp]         list lengths
// Mp is the total slot count rounded up to a multiple of 32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kg {

constexpr int MAX_MELTS = 64;
constexpr int CODE_BITS = 10;           // cells per axis on the code grid <= 1024
constexpr int CODE_MASK = (1 << CODE_BITS) - 1;
constexpr int MAX_CELL_OCC = 1024;      // a cell holding more monomers is reported, never scanned
constexpr int IDX_BITS = 27;            // Verlet-list entry: index bits, then the 5-bit stencil code
constexpr unsigned IDX_MASK = (1u << IDX_BITS) - 1u;
constexpr int SHIFT_SLOTS = 32;         // shift-table entries per melt (27 used)

// device error / status word bits
enum : unsigned {
    ERR_OVERSTRETCH = 1u,
    ERR_NONFINITE = 2u,
    ERR_NL_CAPACITY = 4u,
    ERR_DB_CAPACITY = 8u,
    ERR_TIMEOUT = 16u,
    ERR_DB_INTERNAL = 32u,
};

struct MeltDev {
    int off, M, N, n_ch;          // slots [off, off+M): chain c, position i -> off + c*N + i
    int ch_off;                   // chains of earlier melts (global chain index = ch_off + c)
    double L, invL, kappa;
    float Lf, invLf, kappaf;
    // Verlet-list cell grid (cells >= r_c + skin), numbered brick-major
    // (4x4x4-cell bricks) so that a block of consecutive monomers in cell
    // order has a compact neighbourhood; the position records are offsets
    // from the corners of these cells
    int nc, nbk, cell_off;
    double h, invh;
    float hf;
    float nl_lo, nl_hi;      // binary32 prefilter: r^2 < nl_lo in, r^2 >= nl_hi out
    // double-bridging grid (cells >= db_bond_max); binary32 records on it decide
    // the swap-bond criterion outside the band [db_lo, db_hi) around db_bond_max^2
    int ndb, dbcell_off;
    double hdb, invhdb;
    float hdbf, db_lo, db_hi;
};

// Parameters of the current potential stage (Eqs. 6, 9, 10) and thermostat.
struct StageDev {
    double n, c1, c2;        // U_MLJ^n(r) = c1 r^-n - c2 r^-6 + 1  (r < r_c)
    double kfene, R0sq;      // FENE: -k R0^2/2 ln(1 - r^2/R0^2)
    double qmin, r2star, ustar;  // continuation beyond r*^2 = (1 - qmin) R0^2 (qmin > 0)
    double dt, gamma, T, amp;  // amp = sqrt(2 gamma T / dt)
    float nf, c1f, c2f, kfenef, R0sqf, dtf, gammaf, ampf, qminf, r2starf, ustarf;
    float c2x6f, c1xnf;      // 6 c2 and n c1: fr = (6 c2 r^-6 - n c1 r^-n) / r^2
    int nkind;               // 0: general n, 1: integer n, 2: n = 5.75, 3: n = 6.5
    int nint;
};

struct SimDev {
    MeltDev melt[MAX_MELTS];
    int n_melts, M, Mp, maxnb;
    double rc2, rl2, rl, db_lim2;
    float rc2f, rl2f_lo, rl2f_hi, half_skin2f;
    double half_skin2;
    unsigned long long seed;
    int paper_metropolis;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplies with multipliers 0xD2511F53, 0xCD9E8D57 and a Weyl key
// schedule with increments 0x9E3779B9, 0xBB67AE85.
// Counter layout: (index, time_lo, time_hi, melt<<4 | purpose), key = seed.
// Purposes: 0 MD noise (index = melt-local slot, time = step),
//           1 DB attempt draw, 2 DB partner draw (index = attempt, time = sweep).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw(unsigned long long seed, int melt, unsigned purpose,
                                      unsigned long long time, uint32_t index)
{
    return philox4x32_10(make_uint4(index, (uint32_t)time, (uint32_t)(time >> 32),
                                    ((uint32_t)melt << 4) | purpose),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// (2*(w>>9)+1) * 2^-24: a uniform in (0,1), exact in binary32 and binary64.
__device__ __forceinline__ float unit_open_f(uint32_t w)
{
    return __uint2float_rn(2u * (w >> 9) + 1u) * 5.9604644775390625e-8f;
}
__device__ __forceinline__ double unit_open_d(uint32_t w)
{
    return (double)(2u * (w >> 9) + 1u) * 5.9604644775390625e-8;
}

// Three standard normals by Box-Muller.
__device__ __forceinline__ float3 gauss3_f(uint4 r)
{
    const float a = sqrtf(-2.0f * logf(unit_open_f(r.x)));
    const float b = sqrtf(-2.0f * logf(unit_open_f(r.z)));
    float s, c;
    sincospif(2.0f * unit_open_f(r.y), &s, &c);
    return make_float3(a * c, a * s, b * cospif(2.0f * unit_open_f(r.w)));
}
__device__ __forceinline__ double3 gauss3_d(uint4 r)
{
    const double a = sqrt(-2.0 * log(unit_open_d(r.x)));
    const double b = sqrt(-2.0 * log(unit_open_d(r.z)));
    double s, c;
    sincospi(2.0 * unit_open_d(r.y), &s, &c);
    return make_double3(a * c, a * s, b * cospi(2.0 * unit_open_d(r.w)));
}

// floor(w * n / 2^64): exact integer map of a 64-bit word onto [0, n).
__device__ __forceinline__ long long mul_hi64(unsigned long long w, unsigned long long n)
{
    return (long long)__umul64hi(w, n);
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
__device__ __forceinline__ int melt_of(const SimDev &S, int s)
{
    int m = 0;
    while (m + 1 < S.n_melts && s >= S.melt[m + 1].off) ++m;
    return m;
}

// binary64 minimum image evaluated exactly as d - L*rint(d/L), no contraction
__device__ __forceinline__ double min_image_exact(double d, double L)
{
    return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// squared binary64 distance between slots s and t, ((dx*dx + dy*dy) + dz*dz)
__device__ __forceinline__ double dist2_exact(const double *__restrict__ x, int Mp, double L, int s, int t)
{
    const double dx = min_image_exact(__dsub_rn(x[t], x[s]), L);
    const double dy = min_image_exact(__dsub_rn(x[Mp + t], x[Mp + s]), L);
    const double dz = min_image_exact(__dsub_rn(x[2 * Mp + t], x[2 * Mp + s]), L);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ unsigned pack_code(int cx, int cy, int cz)
{
    return (unsigned)cx | ((unsigned)cy << CODE_BITS) | ((unsigned)cz << (2 * CODE_BITS));
}

__device__ __forceinline__ int wrap_dk(int dk, int n)
{
    if (dk > n / 2) dk -= n;
    else if (dk < -(n / 2)) dk += n;
    return dk;
}

// Verlet-grid cell index of cell coordinates (cx, cy, cz), brick-major.
__device__ __forceinline__ int md_cell(const MeltDev &md, int cx, int cy, int cz)
{
    return md.cell_off + ((((cz >> 2) * md.nbk + (cy >> 2)) * md.nbk + (cx >> 2)) << 6) +
           (((cz & 3) << 4) | ((cy & 3) << 2) | (cx & 3));
}

__device__ __forceinline__ void md_cell_xyz(const MeltDev &md, int cell, int &cx, int &cy, int &cz)
{
    const int r = cell - md.cell_off, b = r >> 6, l = r & 63;
    cx = ((b % md.nbk) << 2) | (l & 3);
    cy = (((b / md.nbk) % md.nbk) << 2) | ((l >> 2) & 3);
    cz = ((b / (md.nbk * md.nbk)) << 2) | (l >> 4);
}

// Cell of a binary64 coordinate on a grid of n cells of side h = L / n per
// period: g = floor(x / h) of the unwrapped coordinate, taken modulo n, and
// the offset x - g h from that cell's corner, rounded once to binary32.
// n h differs from L by at most an ulp of L, so the offsets of monomers in
// different periodic images stay consistent to ~1e-14 sigma.  Four binary64
// operations (binary64 issues at a small fraction of the binary32 rate on
// this GPU), each explicitly rounded so that every kernel inlining it
// computes the same bits.
__device__ __forceinline__ int cell_of(double x, double h, double invh, int n, float &off)
{
    const double g = floor(__dmul_rn(x, invh));
    off = __double2float_rn(__fma_rn(-g, h, x));
    const int c = (int)g % n;
    return c < 0 ? c + n : c;
}

// Minimum-image vector from gather record i to gather record j (binary32):
// p = offset from the build-time cell corner + displacement, w = packed cell
// coordinates.  The cell difference, wrapped to the nearest image, carries
// the integer part, so no large-magnitude value enters the sum.  The wrap is
// unambiguous while |true cell difference| < nc/2, which holds when nc >= 11
// for every pair closer than 6 sigma (two bonds at the 2 R0 error limit,
// cells >= 1.37 sigma, up to half a skin of drift each); smaller grids (small
// boxes) finish with an explicit minimum image of the small vector.
__device__ __forceinline__ float3 rec_rel(float4 pi, float4 pj, int nc, float h, float L, float invL)
{
    const unsigned ci = __float_as_uint(pi.w), cj = __float_as_uint(pj.w);
    const int dkx = wrap_dk((int)(cj & CODE_MASK) - (int)(ci & CODE_MASK), nc);
    const int dky = wrap_dk((int)((cj >> CODE_BITS) & CODE_MASK) - (int)((ci >> CODE_BITS) & CODE_MASK), nc);
    const int dkz = wrap_dk((int)(cj >> (2 * CODE_BITS)) - (int)(ci >> (2 * CODE_BITS)), nc);
    float3 d = make_float3((pj.x - pi.x) + (float)dkx * h, (pj.y - pi.y) + (float)dky * h,
                           (pj.z - pi.z) + (float)dkz * h);
    if (nc < 11) {
        d.x -= L * rintf(d.x * invL);
        d.y -= L * rintf(d.y * invL);
        d.z -= L * rintf(d.z * invL);
    }
    return d;
}

}  // namespace kg
