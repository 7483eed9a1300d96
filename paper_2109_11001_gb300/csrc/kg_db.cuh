// kg_db.cuh -- device pieces shared by the uniform and the learned
// double-bridging sweeps: candidate enumeration in a topology view, the
// bond / bending terms of a swap, and the ordered commit.
#pragma once
#include <cuda_runtime.h>

#include <climits>

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

// ---------------------------------------------------------------------------
// Ordered commit in rounds.  Every attempt record carries the number of swaps
// committed (in its melt) when it was evaluated, ver[k]; chains and cells of
// the 1.3 sigma grid carry the number of the last commit that touched them
// (chain_ver, cell_ver; -1 for none).  A record is stale when a commit at or
// after its version touched one of its two chains, or stamped a cell within
// P::radius cells of one of its junction monomers: only then can its
// evaluation differ, since swaps preserve positions, the bonds inside moved
// segments and the lengths of the pieces on either side of every bond.
// One round: (A) every stale record at or after the melt's position is
// re-evaluated against the current topology, across the whole GPU, one warp
// per attempt; (B) one block per melt finds the first accepted attempt from
// its position (every record there is now current), commits it (slot maps,
// box shifts, chain and cell stamps) and moves the position past it, or, if
// there is none, finishes the melt (statistics).  Rounds repeat until every
// melt is finished: as many rounds as accepted swaps plus one, and the result
// is that of the strictly sequential loop over attempts.
// round[RS m + 0..4] = position, commits, finished, re-evaluations, and the
// first accepted attempt at or after the position (INT_MAX: none), which pass
// (A) records while it reads every current record, so (B) needs no search.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool stale_rec(const Attempt &a, int v, const int *__restrict__ chain_ver, int choff,
                                          const int *__restrict__ cell, const int *__restrict__ cell_ver)
{
    if (chain_ver[choff + a.c] >= v) return true;
    if ((a.flags & 1) && chain_ver[choff + a.d] >= v) return true;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (a.jp[q] >= 0 && cell_ver[cell[a.jp[q]]] >= v) return true;
    return false;
}

// (A) E provides eval(m, k_in_melt, k_global, Attempt &out) for one whole warp
// (lane 0 leaves the record in out).
template <class E>
__device__ void restale_body(E &ev, const SimDev &S, const int *__restrict__ koff, Attempt *__restrict__ att,
                             int *__restrict__ ver, const int *__restrict__ chain_ver, const int *__restrict__ cell,
                             const int *__restrict__ cell_ver, int *__restrict__ round)
{
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarp = (int)((gridDim.x * blockDim.x) >> 5);
    const int Ktot = koff[S.n_melts];
    for (int base = gw * 32; base < Ktot; base += nwarp * 32) {
        const int k = base + lane;
        bool st = false, live = false;
        int m = 0;
        if (k < Ktot) {
            while (k >= koff[m + 1]) ++m;
            const int *R = round + RS * m;
            if (!R[2] && k - koff[m] >= R[0]) {
                st = stale_rec(att[k], ver[k], chain_ver, S.melt[m].ch_off, cell, cell_ver);
                live = true;
            }
        }
        // fresh records are current: note the first accepted one of each melt
        const int m0 = __shfl_sync(FULL_MASK, m, 0);
        const bool acc = live && !st && (att[k].flags & 2);
        if (__all_sync(FULL_MASK, !live || m == m0)) {  // one melt in the warp: one atomic
            const int first = __reduce_min_sync(FULL_MASK, acc ? k - koff[m] : INT_MAX);
            if (lane == 0 && first != INT_MAX) atomicMin(round + RS * m0 + 4, first);
        } else if (acc) {
            atomicMin(round + RS * m + 4, k - koff[m]);
        }
        unsigned bal = __ballot_sync(FULL_MASK, st);
        while (bal) {
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const int kk = __shfl_sync(FULL_MASK, k, src), mm = __shfl_sync(FULL_MASK, m, src);
            Attempt a;
            ev.eval(mm, kk - koff[mm], kk, a);
            if (lane == 0) {
                att[kk] = a;
                ver[kk] = round[RS * mm + 1];
                atomicAdd(round + RS * mm + 3, 1);
                if (a.flags & 2) atomicMin(round + RS * mm + 4, kk - koff[mm]);
            }
            __syncwarp();
        }
    }
}

// (B) one block per melt; P provides init (block-wide) and radius.
template <class P>
__device__ void commit_next_body(P &pol, const SimDev &S, const double *__restrict__ x, const int *__restrict__ cell,
                                 const int *__restrict__ koff, const Attempt *__restrict__ att,
                                 int *__restrict__ occ, int *__restrict__ curmap, int *__restrict__ img,
                                 int *__restrict__ chain_ver, int *__restrict__ cell_ver, int *__restrict__ round,
                                 long long *__restrict__ stats, unsigned *flags, int *old_occ)
{
    __shared__ int found_s, sh[6], done_s;
    __shared__ unsigned long long n_empty;
    const int m = blockIdx.x, tid = threadIdx.x;
    int *R = round + RS * m;
    if (tid == 0) done_s = R[2] || flags[0] != 0;
    __syncthreads();
    if (done_s) return;
    const MeltDev &md = S.melt[m];
    const int N = md.N, off = md.off, Mp = S.Mp;
    const int k0 = koff[m], K = koff[m + 1] - k0;
    // the first accepted attempt at or after the position, as pass (A) found it
    if (tid == 0) found_s = R[4] < K ? R[4] : K;
    __syncthreads();
    const int found = found_s;
    if (found == K) {                              // the melt is finished
        if (tid == 0) n_empty = 0;
        __syncthreads();
        unsigned long long e = 0;
        for (int k = tid; k < K; k += blockDim.x) e += !(att[k0 + k].flags & 1);
        atomicAdd(&n_empty, e);
        __syncthreads();
        if (tid == 0) {
            stats[4 * m + 0] = K;
            stats[4 * m + 1] = (long long)n_empty;
            stats[4 * m + 2] = R[1];
            stats[4 * m + 3] = R[3];
            if (R[1]) atomicOr(flags + 1, 1u);
            R[2] = 1;
        }
        return;
    }
    pol.init();
    const int Rr = pol.radius(md);
    const Attempt a = att[k0 + found];
    const int kind = a.kind, A = a.A, Bc = a.B, pA = a.pA, pB = a.pB, nc = R[1];
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
    // stamp the two chains and the cells within Rr of the four junction monomers
    const int n = md.ndb, W = 2 * Rr + 1;
    for (int q = 0; q < 4; ++q) {
        const int p = a.jp[q];
        if (p < 0) continue;
        const int c0 = cell[p] - md.dbcell_off;
        const int cx = c0 % n, cy = (c0 / n) % n, cz = c0 / (n * n);
        for (int t = tid; t < W * W * W; t += blockDim.x) {
            const int dx = t % W - Rr, dy = (t / W) % W - Rr, dz = t / (W * W) - Rr;
            const int xx = ((cx + dx) % n + n) % n, yy = ((cy + dy) % n + n) % n;
            const int zz = ((cz + dz) % n + n) % n;
            cell_ver[md.dbcell_off + (zz * n + yy) * n + xx] = nc;
        }
    }
    __syncthreads();
    if (tid == 0) {
        chain_ver[md.ch_off + A] = nc;
        chain_ver[md.ch_off + Bc] = nc;
        R[1] = nc + 1;
        R[0] = found + 1;
        R[4] = INT_MAX;                            // to be found again by the next pass (A)
    }
}

// Commit rounds until every melt is finished (host).  restale() and
// commit_next() enqueue one pass each; the host reads the per-melt finished
// flags after rounds 1, 2, 4, 8 and then every 8 (the passes of a finished melt
// return at once), and stops on a latched device error.
template <class FA, class FB>
void db_rounds(kg_ctx *c, long long tot, FA restale, FB commit_next)
{
    static thread_local int *hround = nullptr;
    if (!hround && cudaMallocHost(&hround, sizeof(int) * (RS * MAX_MELTS + 1)) != cudaSuccess) return;
    const int nm = c->sim.n_melts;
    long long r = 0, next_check = 1;
    while (r <= tot) {                              // at most one round per accepted swap, plus one
        restale();
        commit_next();
        c->launches += 2;
        if (++r < next_check) continue;
        cudaMemcpyAsync(hround, c->dbround, sizeof(int) * RS * nm, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(hround + RS * MAX_MELTS, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return;
        bool all = true;
        for (int m = 0; m < nm; ++m) all = all && hround[RS * m + 2] != 0;
        if (all || hround[RS * MAX_MELTS] != 0) return;
        next_check = r < 8 ? 2 * r : r + 8;
    }
}

}  // namespace kg
