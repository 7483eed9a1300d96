// kg_db.cuh -- device pieces shared by the uniform and the learned
// double-bridging sweeps: candidate enumeration in a topology view, the
// bond / bending terms of a swap, and the ordered commit.
#pragma once
#include <cuda_runtime.h>

#include "kg_host.h"

namespace kg {

constexpr int CAND_CAP = 48;
constexpr int JCAP = 4096;

struct Cand {
    int key, key2, kind, d, q;
};

struct DBC {
    const double *__restrict__ x;
    int Mp;
    const int *__restrict__ pid;
    const int *__restrict__ cell;
    const int *__restrict__ start;
    const int *__restrict__ list;
    MeltDev md;
    int melt;
    double lim2, kfene, R0, T, qmin, nexp;
};

// topology view: slot -> monomer (occ) and monomer -> slot (cur)
struct ViewMap {
    const int *o;
    const int *c;
    __device__ __forceinline__ int occ(int s) const { return o[s]; }
    __device__ __forceinline__ int cur(int p) const { return c[p]; }
};

// Slot relabelling of one swap; the same map takes x -> x' and x' -> x.
__device__ __forceinline__ int swap_slot(int s, int kind, int A, int B, int pA, int pB, int N, int off)
{
    const int r = s - off, ch = r / N, i = r - ch * N;
    if (kind == 0) {
        if (i > pA) {
            if (ch == A) return off + B * N + i;
            if (ch == B) return off + A * N + i;
        }
    } else {
        if (ch == A && i > pA) return off + B * N + (N - 1 - i);
        if (ch == B && i <= pB) return off + A * N + (N - 1 - i);
    }
    return s;
}

template <class V>
struct ViewMove {
    V b;
    int kind, A, B, pA, pB, N, off;
    __device__ __forceinline__ int occ(int s) const { return b.occ(swap_slot(s, kind, A, B, pA, pB, N, off)); }
    __device__ __forceinline__ int cur(int p) const { return swap_slot(b.cur(p), kind, A, B, pA, pB, N, off); }
};

__device__ __forceinline__ double d2(const DBC &C, int a, int b) { return dist2_exact(C.x, C.Mp, C.md.L, a, b); }

// |P(b)| for bond (chain c, index b) in view v; fills `out` (<= CAND_CAP) if given.
template <class V>
__device__ int count_partners(const DBC &C, const V &v, int c, int b, Cand *out)
{
    const MeltDev &md = C.md;
    const int N = md.N;
    const int us = md.off + c * N + b;
    const int pu = v.occ(us), pw = v.occ(us + 1);
    if (d2(C, pu, pw) > C.lim2) return 0;
    const int n = md.ndb, c0 = C.cell[pu] - md.dbcell_off;
    const int cx = c0 % n, cy = (c0 / n) % n, cz = c0 / (n * n);
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int cell = md.dbcell_off + (((cz + dz + n) % n) * n + (cy + dy + n) % n) * n + (cx + dx + n) % n;
                const int b0 = C.start[cell], e = C.start[cell + 1];
                if (e - b0 > MAX_CELL_OCC) return -1;                  // caller reports capacity
                for (int k = b0; k < e; ++k) {
                    const int t = C.list[k];
                    const int ts = v.cur(t), r = ts - md.off, d = r / N, i = r - d * N;
                    if (d == c) continue;
                    if (d2(C, pu, t) > C.lim2) continue;
                    if (i == b + 1) {                          // kind 0: t = D_{b+1}
                        const int up = v.occ(md.off + d * N + b);
                        if (d2(C, up, pw) <= C.lim2 && d2(C, up, t) <= C.lim2) {
                            if (out && cnt < CAND_CAP) out[cnt] = Cand{C.pid[t], C.pid[up], 0, d, b};
                            ++cnt;
                        }
                    }
                    if (i == N - 2 - b) {                      // kind 1: t = D_q, q = N-2-b
                        const int t1 = v.occ(ts + 1);
                        if (d2(C, t1, pw) <= C.lim2 && d2(C, t, t1) <= C.lim2) {
                            if (out && cnt < CAND_CAP) out[cnt] = Cand{C.pid[t], C.pid[t1], 1, d, i};
                            ++cnt;
                        }
                    }
                }
            }
    return cnt;
}

// FENE log term of a bond of length r (kg_params.fene_qmin continuation beyond r*)
__device__ __forceinline__ double fene_of_r(const DBC &C, double r)
{
    const double q = 1.0 - (r / C.R0) * (r / C.R0);
    if (C.qmin > 0.0 && q < C.qmin)           // continuation beyond r* (kg_params.fene_qmin)
        return -0.5 * C.kfene * C.R0 * C.R0 * log(C.qmin) + C.kfene * (r * r - (1.0 - C.qmin) * C.R0 * C.R0) / (2.0 * C.qmin);
    return -0.5 * C.kfene * C.R0 * C.R0 * log(q);
}

template <class V>
__device__ double bond_fene(const DBC &C, const V &v, int chain, int idx)
{
    const int s = C.md.off + chain * C.md.N + idx;
    return fene_of_r(C, sqrt(d2(C, v.occ(s), v.occ(s + 1))));
}

// cos of the angle at vertex i of `chain` in view v (1 at a chain end)
template <class V>
__device__ double vcos(const DBC &C, const V &v, int chain, int i)
{
    const int N = C.md.N;
    if (i < 1 || i > N - 2) return 1.0;
    const int s = C.md.off + chain * N + i;
    const int a = v.occ(s - 1), b = v.occ(s), c = v.occ(s + 1);
    const double L = C.md.L;
    double b1[3], b2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        b1[k] = min_image_exact(C.x[k * C.Mp + b] - C.x[k * C.Mp + a], L);
        b2[k] = min_image_exact(C.x[k * C.Mp + c] - C.x[k * C.Mp + b], L);
    }
    return (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
           / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
              * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
}

template <class V>
__device__ double bend(const DBC &C, const V &v, int chain, int i)
{
    if (i < 1 || i > C.md.N - 2) return 0.0;
    return C.md.kappa * (1.0 - vcos(C, v, chain, i));
}

__device__ __forceinline__ DBC make_dbc(const SimDev &S, const StageDev &st, int m, const double *x,
                                        const int *pid, const int *cell, const int *start, const int *list,
                                        double T)
{
    DBC C;
    C.x = x; C.Mp = S.Mp; C.pid = pid; C.cell = cell; C.start = start; C.list = list;
    C.md = S.melt[m]; C.melt = m; C.lim2 = S.db_lim2; C.kfene = st.kfene; C.R0 = sqrt(st.R0sq); C.T = T; C.qmin = st.qmin;
    C.nexp = st.n;
    return C;
}

// cells a and b at most R cells apart along every axis (periodic)
__device__ __forceinline__ bool cells_near(int a, int b, int off, int n, int R)
{
    a -= off; b -= off;
    const int ax = a % n, ay = (a / n) % n, az = a / (n * n);
    const int bx = b % n, by = (b / n) % n, bz = b / (n * n);
    int dx = abs(ax - bx), dy = abs(ay - by), dz = abs(az - bz);
    dx = min(dx, n - dx); dy = min(dy, n - dy); dz = min(dz, n - dz);
    return dx <= R && dy <= R && dz <= R;
}

// Ordered validation and commit, one block per melt (P: re-evaluation policy).
// An attempt is re-evaluated against the current topology when an earlier
// accepted swap of the sweep touched one of its two chains, or put a junction
// monomer within P::radius cells of one of the attempt's junction monomers.
// P provides: init (block-wide, before the walk), radius, and reeval (called
// by every thread; it leaves the new record in `out`).
template <class P>
__device__ void db_commit_body(P &pol, const SimDev &S, const StageDev &stg, const double *__restrict__ x,
                               const int *__restrict__ pid, const int *__restrict__ cell,
                               const int *__restrict__ start, const int *__restrict__ list,
                               const int *__restrict__ koff, const Attempt *__restrict__ att,
                               int *__restrict__ occ, int *__restrict__ curmap, int *__restrict__ img,
                               int *__restrict__ dirty, long long *__restrict__ stats, long long sweep,
                               unsigned *flags, int *old_occ)
{
    __shared__ int jcell[JCAP];
    __shared__ int njc;
    __shared__ Attempt a_s;
    __shared__ int need_s, sh[6];
    __shared__ long long n_acc, n_empty, n_re;
    __shared__ int stop_s;
    const int m = blockIdx.x;
    if (threadIdx.x == 0) stop_s = flags[0] != 0;  // one reading for the whole block
    __syncthreads();
    if (stop_s) {                                  // a latched error stops the sweep
        if (threadIdx.x == 0) for (int k = 0; k < 4; ++k) stats[4 * m + k] = 0;
        return;
    }
    const MeltDev &md = S.melt[m];
    const int N = md.N, off = md.off, Mp = S.Mp, tid = threadIdx.x;
    const DBC C = make_dbc(S, stg, m, x, pid, cell, start, list, stg.T);
    const ViewMap V{occ, curmap};
    pol.init();
    const int R = pol.radius(md);
    if (tid == 0) { njc = 0; n_acc = n_empty = n_re = 0; }
    __syncthreads();
    const int k0 = koff[m], K = koff[m + 1] - k0;
    for (int kk = 0; kk < K; ++kk) {
        if (tid == 0) {
            a_s = att[k0 + kk];
            need_s = dirty[off + a_s.c * N] || ((a_s.flags & 1) && dirty[off + a_s.d * N]) || njc > JCAP - 4;
        }
        __syncthreads();
        bool near = false;
        if (!need_s) {
            const int nj = njc;
            for (int j = tid; j < nj; j += blockDim.x) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int p = a_s.jp[q];
                    if (p >= 0 && cells_near(jcell[j], cell[p], md.dbcell_off, md.ndb, R)) near = true;
                }
            }
        }
        const bool need = __syncthreads_or(near || need_s);
        if (need) {
            pol.reeval(C, V, S, sweep, kk, k0 + kk, a_s, flags);
            if (tid == 0) ++n_re;
        }
        __syncthreads();
        if (!(a_s.flags & 1)) {
            if (tid == 0) ++n_empty;
        } else if (a_s.flags & 2) {
            const int kind = a_s.kind, A = a_s.A, B = a_s.B, pA = a_s.pA, pB = a_s.pB;
            const int baseA = off + A * N, baseB = off + B * N;
            for (int i = tid; i < N; i += blockDim.x) {
                old_occ[i] = occ[baseA + i];
                old_occ[N + i] = occ[baseB + i];
            }
            __syncthreads();
            for (int i = tid; i < 2 * N; i += blockDim.x) {
                const int s = i < N ? baseA + i : baseB + (i - N);
                const int src = swap_slot(s, kind, A, B, pA, pB, N, off);
                const int val = src - baseA < N && src >= baseA ? old_occ[src - baseA] : old_occ[N + src - baseB];
                occ[s] = val;
                curmap[val] = s;
            }
            __syncthreads();
            if (tid < 2) {
                // segment 0: A' slots pA+1..N-1 anchored at A' slot pA;
                // segment 1: kind 0 -> B' slots pA+1..N-1 at pA; kind 1 -> B' slots 0..pB at pB+1
                int f, an;
                if (tid == 0) { f = occ[baseA + pA + 1]; an = occ[baseA + pA]; }
                else if (kind == 0) { f = occ[baseB + pA + 1]; an = occ[baseB + pA]; }
                else { f = occ[baseB + pB]; an = occ[baseB + pB + 1]; }
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    sh[3 * tid + d] = -((int)rint(__ddiv_rn(__dsub_rn(x[d * Mp + f], x[d * Mp + an]), md.L))
                                        + img[d * Mp + f] - img[d * Mp + an]);
            }
            __syncthreads();
            for (int i = tid; i < 2 * N; i += blockDim.x) {
                int seg = -1, s;
                if (i < N) {
                    s = baseA + i;
                    if (i > pA) seg = 0;
                } else {
                    const int j = i - N;
                    s = baseB + j;
                    if ((kind == 0 && j > pA) || (kind == 1 && j <= pB)) seg = 1;
                }
                if (seg >= 0) {
                    const int p = occ[s];
#pragma unroll
                    for (int d = 0; d < 3; ++d) img[d * Mp + p] += sh[3 * seg + d];
                }
            }
            if (tid == 0) {
                dirty[baseA] = 1;
                dirty[baseB] = 1;
                for (int q = 0; q < 4; ++q)
                    if (a_s.jp[q] >= 0 && njc < JCAP) jcell[njc++] = cell[a_s.jp[q]];
                ++n_acc;
            }
        }
        pol.after(a_s, k0 + kk);
        __syncthreads();
    }
    if (tid == 0) {
        stats[4 * m + 0] = K;
        stats[4 * m + 1] = n_empty;
        stats[4 * m + 2] = n_acc;
        stats[4 * m + 3] = n_re;
        if (n_acc) atomicOr(flags + 1, 1u);
    }
}

}  // namespace kg
