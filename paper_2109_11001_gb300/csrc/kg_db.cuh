// kg_db.cuh -- device pieces shared by the uniform and the learned
// double-bridging sweeps: candidate enumeration in a topology view, the
// bond / bending terms of a swap, and the ordered commit.
#pragma once
#include <cuda_runtime.h>

#include "kg_host.h"

namespace kg {

constexpr int CAND_CAP = 48;

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
    const float4 *__restrict__ rec;    // binary32 records on the 1.3 sigma grid (k_bin_db)
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

// Swap-bond criterion d2(a, b) <= 1.3^2, decided exactly: the binary32 record
// distance settles every pair outside the band [db_lo, db_hi), which bounds
// its rounding error; pairs inside it take the binary64 distance.
__device__ __forceinline__ bool within(const DBC &C, int a, int b)
{
    const float3 d = rec_rel(__ldg(C.rec + a), __ldg(C.rec + b), C.md.ndb, C.md.hdbf, C.md.Lf, C.md.invLf);
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    if (r2 < C.md.db_lo) return true;
    if (r2 >= C.md.db_hi) return false;
    return d2(C, a, b) <= C.lim2;
}

// per-warp candidate scratch of one partner enumeration
struct __align__(16) WarpCand {
    Cand tmp[CAND_CAP];
    Cand cand[CAND_CAP];
    int n;
};

constexpr unsigned FULL_MASK = 0xffffffffu;

// Admissible partners P(b) of bond (c, b) in view v, one warp: lane q < 27
// scans stencil cell q around the bond's lower monomer.  With ORDER the list
// is left in wc.cand ordered by (key, key2) (the monomer ids of the monomer
// that would bond to the drawn bond's lower end and of the partner bond's
// other monomer).  Returns |P|, or -1 (error bit set) on a capacity overflow.
template <bool ORDER, class V>
__device__ int warp_partners(const DBC &C, const V &v, int c, int b, WarpCand &wc, unsigned &err)
{
    const int lane = threadIdx.x & 31;
    const MeltDev &md = C.md;
    const int N = md.N;
    const int us = md.off + c * N + b;
    const int pu = v.occ(us), pw = v.occ(us + 1);
    if (!within(C, pu, pw)) return 0;
    if (lane == 0) wc.n = 0;
    __syncwarp();
    bool bad = false;
    if (lane < 27) {
        const int n = md.ndb, c0 = C.cell[pu] - md.dbcell_off;
        const int cx = c0 % n, cy = (c0 / n) % n, cz = c0 / (n * n);
        const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
        const int cell = md.dbcell_off + (((cz + dz + n) % n) * n + (cy + dy + n) % n) * n + (cx + dx + n) % n;
        const int b0 = C.start[cell], e = C.start[cell + 1];
        if (e - b0 > MAX_CELL_OCC) {
            bad = true;
        } else {
            for (int k = b0; k < e; ++k) {
                const int t = C.list[k];
                const int ts = v.cur(t), r = ts - md.off, d = r / N, i = r - d * N;
                if (d == c) continue;
                if (i != b + 1 && i != N - 2 - b) continue;   // neither kind can use t
                if (!within(C, pu, t)) continue;
                if (i == b + 1) {                          // kind 0: t = D_{b+1}
                    const int up = v.occ(md.off + d * N + b);
                    if (within(C, up, pw) && within(C, up, t)) {
                        const int pos = atomicAdd(&wc.n, 1);
                        if (ORDER && pos < CAND_CAP) wc.tmp[pos] = Cand{C.pid[t], C.pid[up], 0, d, b};
                    }
                }
                if (i == N - 2 - b) {                      // kind 1: t = D_q, q = N-2-b
                    const int t1 = v.occ(ts + 1);
                    if (within(C, t1, pw) && within(C, t, t1)) {
                        const int pos = atomicAdd(&wc.n, 1);
                        if (ORDER && pos < CAND_CAP) wc.tmp[pos] = Cand{C.pid[t], C.pid[t1], 1, d, i};
                    }
                }
            }
        }
    }
    __syncwarp();
    const int n = wc.n;
    if (__any_sync(FULL_MASK, bad) || n > CAND_CAP) {
        err |= ERR_DB_CAPACITY;
        return -1;
    }
    if (ORDER) {
        for (int j = lane; j < n; j += 32) {       // rank by the (unique) key pair
            const Cand cj = wc.tmp[j];
            int r = 0;
            for (int i = 0; i < n; ++i) {
                const Cand ci = wc.tmp[i];
                r += (ci.key < cj.key) || (ci.key == cj.key && ci.key2 < cj.key2);
            }
            wc.cand[r] = cj;
        }
        __syncwarp();
    }
    return n;
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
                                        const float4 *rec, double T)
{
    DBC C;
    C.x = x; C.Mp = S.Mp; C.pid = pid; C.cell = cell; C.start = start; C.list = list; C.rec = rec;
    C.md = S.melt[m]; C.melt = m; C.lim2 = S.db_lim2; C.kfene = st.kfene; C.R0 = sqrt(st.R0sq); C.T = T; C.qmin = st.qmin;
    C.nexp = st.n;
    return C;
}

// Ordered validation and commit, one block per melt (P: re-evaluation policy).
// An attempt's speculative record is stale when an earlier accepted swap of
// the sweep touched one of its two chains or put a junction monomer within
// P::radius cells of one of the attempt's junction monomers (cells carry the
// sweep's stamp in `mark`).  The walk finds the next attempts that are stale
// or accepted with a block-wide scan, re-evaluates up to one stale attempt
// per warp against the current topology, then takes them in order: the
// re-evaluations before the first acceptance are final, the first accepted
// swap is committed, and the scan resumes after it.  The result is that of
// the strictly sequential loop over attempts.  P provides init (block-wide),
// radius, batch (the most warps that may re-evaluate at once) and reeval (one
// whole warp; lane 0 leaves the new record in `out`).
template <class P>
__device__ void db_commit_body(P &pol, const SimDev &S, const StageDev &stg, const double *__restrict__ x,
                               const int *__restrict__ pid, const int *__restrict__ cell,
                               const int *__restrict__ start, const int *__restrict__ list,
                               const float4 *__restrict__ rec, const int *__restrict__ koff,
                               const Attempt *__restrict__ att, int *__restrict__ occ, int *__restrict__ curmap,
                               int *__restrict__ img, int *__restrict__ dirty, int *__restrict__ mark, int stamp,
                               long long *__restrict__ stats, long long sweep, unsigned *flags, int *old_occ)
{
    constexpr int MAXB = 32;
    __shared__ Attempt bres[MAXB];
    __shared__ int bidx[MAXB], bstale[MAXB], wcnt[32];
    __shared__ int nb_s, sh[6];
    __shared__ unsigned long long n_acc, n_empty, n_re;
    __shared__ long long empty_adj;
    __shared__ int stop_s;
    const int m = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    if (tid == 0) stop_s = flags[0] != 0;          // one reading for the whole block
    __syncthreads();
    if (stop_s) {                                  // a latched error stops the sweep
        if (tid == 0) for (int k = 0; k < 4; ++k) stats[4 * m + k] = 0;
        return;
    }
    const MeltDev &md = S.melt[m];
    const int N = md.N, off = md.off, Mp = S.Mp;
    const DBC C = make_dbc(S, stg, m, x, pid, cell, start, list, rec, stg.T);
    const ViewMap V{occ, curmap};
    pol.init();
    const int R = pol.radius(md);
    const int B = min(min(nw, pol.batch()), MAXB);
    if (tid == 0) { n_acc = n_empty = n_re = 0; empty_adj = 0; }
    __syncthreads();
    const int k0 = koff[m], K = koff[m + 1] - k0;
    {   // empty proposals among the speculative records (corrected as re-evaluations are adopted)
        unsigned long long e = 0;
        for (int k = tid; k < K; k += blockDim.x) e += !(att[k0 + k].flags & 1);
        atomicAdd(&n_empty, e);
    }
    int pos = 0;
    while (pos < K) {
        // 1. the next (up to B) stale or accepted attempts at or after pos, in order
        if (tid == 0) nb_s = 0;
        __syncthreads();
        for (int base = pos;; base += blockDim.x) {
            const int k = base + tid;
            bool inter = false, stale = false;
            if (k < K) {
                const Attempt &a = att[k0 + k];
                stale = dirty[off + a.c * N] || ((a.flags & 1) && dirty[off + a.d * N]);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (a.jp[q] >= 0 && mark[cell[a.jp[q]]] == stamp) stale = true;
                inter = stale || (a.flags & 2);
            }
            const unsigned bal = __ballot_sync(FULL_MASK, inter);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = nb_s;
            for (int w = 0; w < warp; ++w) before += wcnt[w];
            const int o = before + __popc(bal & ((1u << lane) - 1u));
            if (inter && o < B) {
                bidx[o] = k;
                bstale[o] = stale;
            }
            __syncthreads();
            if (tid == 0) {
                int tot = nb_s;
                for (int w = 0; w < nw; ++w) tot += wcnt[w];
                nb_s = min(tot, B);
            }
            __syncthreads();
            if (nb_s >= B || base + (int)blockDim.x >= K) break;
        }
        const int nb = nb_s;
        if (nb == 0) break;                        // everything after pos is final as evaluated
        // 2. stale ones re-evaluated against the current topology, one warp each
        if (warp < nb) {
            const int k = bidx[warp];
            if (bstale[warp]) pol.reeval(C, V, S, sweep, k, k0 + k, warp, bres[warp], flags);
            else if (lane == 0) bres[warp] = att[k0 + k];
        }
        __syncthreads();
        // 3. in order: adopt the re-evaluations up to the first acceptance and commit it
        int next = bidx[nb - 1] + 1;
        for (int i = 0; i < nb; ++i) {
            const Attempt a = bres[i];
            if (bstale[i] && tid == 0) {
                ++n_re;
                empty_adj += (long long)!(a.flags & 1) - (long long)!(att[k0 + bidx[i]].flags & 1);
            }
            if (!(a.flags & 2)) continue;
            const int kind = a.kind, A = a.A, Bc = a.B, pA = a.pA, pB = a.pB;
            const int baseA = off + A * N, baseB = off + Bc * N;
            for (int j = tid; j < N; j += blockDim.x) {
                old_occ[j] = occ[baseA + j];
                old_occ[N + j] = occ[baseB + j];
            }
            __syncthreads();
            for (int j = tid; j < 2 * N; j += blockDim.x) {
                const int s = j < N ? baseA + j : baseB + (j - N);
                const int src = swap_slot(s, kind, A, Bc, pA, pB, N, off);
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
            for (int j = tid; j < 2 * N; j += blockDim.x) {
                int seg = -1, s;
                if (j < N) {
                    s = baseA + j;
                    if (j > pA) seg = 0;
                } else {
                    const int jj = j - N;
                    s = baseB + jj;
                    if ((kind == 0 && jj > pA) || (kind == 1 && jj <= pB)) seg = 1;
                }
                if (seg >= 0) {
                    const int p = occ[s];
#pragma unroll
                    for (int d = 0; d < 3; ++d) img[d * Mp + p] += sh[3 * seg + d];
                }
            }
            // stamp the cells within R of the four junction monomers
            const int n = md.ndb, W = 2 * R + 1;
            for (int q = 0; q < 4; ++q) {
                const int p = a.jp[q];
                if (p < 0) continue;
                const int c0 = cell[p] - md.dbcell_off;
                const int cx = c0 % n, cy = (c0 / n) % n, cz = c0 / (n * n);
                for (int t = tid; t < W * W * W; t += blockDim.x) {
                    const int dx = t % W - R, dy = (t / W) % W - R, dz = t / (W * W) - R;
                    const int xx = ((cx + dx) % n + n) % n, yy = ((cy + dy) % n + n) % n;
                    const int zz = ((cz + dz) % n + n) % n;
                    mark[md.dbcell_off + (zz * n + yy) * n + xx] = stamp;
                }
            }
            if (tid == 0) {
                dirty[baseA] = 1;
                dirty[baseB] = 1;
                ++n_acc;
            }
            next = bidx[i] + 1;
            break;
        }
        pos = next;
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
        stats[4 * m + 0] = K;
        stats[4 * m + 1] = (long long)n_empty + empty_adj;
        stats[4 * m + 2] = (long long)n_acc;
        stats[4 * m + 3] = (long long)n_re;
        if (n_acc) atomicOr(flags + 1, 1u);
    }
}

}  // namespace kg
