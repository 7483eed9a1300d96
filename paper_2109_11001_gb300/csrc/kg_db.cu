// kg_db.cu -- double-bridging Monte Carlo sweep (Fig. 1; Sec. II.B criteria
// (i) and (ii)) with the semantics of a strictly sequential loop over attempts.
//
// A swap removes bond (A_p, A_{p+1}) and bond (B_q, B_{q+1}) of two chains and
// joins the ends crosswise so both chains keep N monomers:
//   kind 0 (q = p):      A' = A_0..A_p B_{p+1}..B_{N-1},  B' = B_0..B_p A_{p+1}..A_{N-1}
//   kind 1 (p+q = N-2):  A' = A_0..A_p B_q..B_0,          B' = A_{N-1}..A_{p+1} B_{q+1}..B_{N-1}
// (A the lower chain index).  Admissible iff both new and both removed bonds
// are <= 1.3 sigma.  Proposal: a bond drawn uniformly, then one entry of its
// partner list (ordered by monomer ids); acceptance
// min(1, exp(-dE/T) q(x'->x)/q(x->x')) with q ~ 1/|P(b1)| + 1/|P(b2)|.
//
// GPU organisation of one sweep:
//   1. bin every monomer on a grid of >= 1.3 sigma cells (positions do not move
//      during a sweep: swaps only relabel slots);
//   2. k_db_eval: every attempt evaluated in parallel against the pre-sweep
//      topology (one thread each).  A "monomer" here is its compute index; the
//      topology is the pair of maps slot -> monomer (comp_of) and monomer ->
//      slot (slot_of);
//   3. k_db_commit: one block per melt walks the attempts in order.  An attempt
//      is re-evaluated against the current topology when an earlier accepted
//      swap in the sweep touched one of its two chains, or put a junction
//      monomer (whose bonds changed) within one cell of a monomer whose
//      neighbourhood it scanned.  Nothing else an evaluation reads can change:
//      swaps preserve positions, the bonds inside moved segments, and the
//      lengths of the two pieces on either side of every bond.  Accepted swaps
//      rewrite the two maps for the slots of their two chains and add box
//      shifts to a per-monomer counter;
//   4. k_db_finish: the box shifts are added to the positions in place; no
//      monomer data moves (the maps are the topology).
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
    double lim2, kfene, R0, T, qmin;
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

template <class V>
__device__ double bond_fene(const DBC &C, const V &v, int chain, int idx)
{
    const int s = C.md.off + chain * C.md.N + idx;
    const double r = sqrt(d2(C, v.occ(s), v.occ(s + 1)));
    const double q = 1.0 - (r / C.R0) * (r / C.R0);
    if (C.qmin > 0.0 && q < C.qmin)           // continuation beyond r* (kg_params.fene_qmin)
        return -0.5 * C.kfene * C.R0 * C.R0 * log(C.qmin) + C.kfene * (r * r - (1.0 - C.qmin) * C.R0 * C.R0) / (2.0 * C.qmin);
    return -0.5 * C.kfene * C.R0 * C.R0 * log(q);
}

template <class V>
__device__ double bend(const DBC &C, const V &v, int chain, int i)
{
    const int N = C.md.N;
    if (i < 1 || i > N - 2) return 0.0;
    const int s = C.md.off + chain * N + i;
    const int a = v.occ(s - 1), b = v.occ(s), c = v.occ(s + 1);
    const double L = C.md.L;
    double b1[3], b2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        b1[k] = min_image_exact(C.x[k * C.Mp + b] - C.x[k * C.Mp + a], L);
        b2[k] = min_image_exact(C.x[k * C.Mp + c] - C.x[k * C.Mp + b], L);
    }
    const double cs = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
                      / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
                         * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
    return C.md.kappa * (1.0 - cs);
}

template <class V>
__device__ Attempt evaluate(const DBC &C, const V &v, unsigned long long seed, long long sweep, int k,
                            int paper, unsigned &err)
{
    const MeltDev &md = C.md;
    const int N = md.N, off = md.off;
    Attempt a;
    a.flags = 0;
    a.d = -1;
    a.kind = a.A = a.B = a.pA = a.pB = 0;
    a.jp[2] = a.jp[3] = -1;
    const uint4 r = draw(seed, C.melt, 1, (unsigned long long)sweep, (uint32_t)k);
    const uint4 r2 = draw(seed, C.melt, 2, (unsigned long long)sweep, (uint32_t)k);
    const long long nbonds = (long long)md.n_ch * (N - 1);
    const long long bond = mul_hi64(((unsigned long long)r.y << 32) | r.x, (unsigned long long)nbonds);
    const double uacc = ((double)(r.z >> 5) * 67108864.0 + (double)(r.w >> 6)) * (1.0 / 9007199254740992.0);
    const int c = (int)(bond / (N - 1)), b = (int)(bond % (N - 1));
    a.c = c;
    a.jp[0] = v.occ(off + c * N + b);
    a.jp[1] = v.occ(off + c * N + b + 1);
    Cand list[CAND_CAP];
    const int n1 = count_partners(C, v, c, b, list);
    if (n1 == 0) return a;
    if (n1 < 0 || n1 > CAND_CAP) { err |= ERR_DB_CAPACITY; return a; }
    for (int i = 1; i < n1; ++i) {                      // order by (key, key2)
        const Cand t = list[i];
        int j = i - 1;
        while (j >= 0 && (list[j].key > t.key || (list[j].key == t.key && list[j].key2 > t.key2))) {
            list[j + 1] = list[j];
            --j;
        }
        list[j + 1] = t;
    }
    const Cand m = list[mul_hi64(((unsigned long long)r2.y << 32) | r2.x, (unsigned long long)n1)];
    a.flags = 1;
    a.d = m.d;
    a.jp[2] = v.occ(off + m.d * N + m.q);
    a.jp[3] = v.occ(off + m.d * N + m.q + 1);
    const int n2 = count_partners(C, v, m.d, m.q, (Cand *)nullptr);
    if (n2 <= 0) { err |= n2 < 0 ? ERR_DB_CAPACITY : ERR_DB_INTERNAL; a.flags = 1; return a; }
    const int A = c < m.d ? c : m.d, B = c < m.d ? m.d : c;
    const int pA = A == c ? b : m.q, pB = A == c ? m.q : b;
    a.kind = m.kind; a.A = A; a.B = B; a.pA = pA; a.pB = pB;
    const ViewMove<V> w{v, m.kind, A, B, pA, pB, N, off};
    double dE = bond_fene(C, w, A, pA) + bond_fene(C, w, B, pB) - bond_fene(C, v, A, pA) - bond_fene(C, v, B, pB);
    dE += bend(C, w, A, pA) + bend(C, w, A, pA + 1) + bend(C, w, B, pB) + bend(C, w, B, pB + 1);
    dE -= bend(C, v, A, pA) + bend(C, v, A, pA + 1) + bend(C, v, B, pB) + bend(C, v, B, pB + 1);
    const int r1 = count_partners(C, w, A, pA, (Cand *)nullptr);
    const int rr2 = count_partners(C, w, B, pB, (Cand *)nullptr);
    if (r1 <= 0 || rr2 <= 0) { err |= (r1 < 0 || rr2 < 0) ? ERR_DB_CAPACITY : ERR_DB_INTERNAL; a.flags = 1; return a; }
    const double ratio = (1.0 / r1 + 1.0 / rr2) / (1.0 / n1 + 1.0 / n2);
    double acc = exp(-dE / C.T);
    if (!paper) acc *= ratio;
    if (uacc < acc) a.flags |= 2;
    return a;
}

__device__ __forceinline__ DBC make_dbc(const SimDev &S, const StageDev &st, int m, const double *x,
                                        const int *pid, const int *cell, const int *start, const int *list,
                                        double T)
{
    DBC C;
    C.x = x; C.Mp = S.Mp; C.pid = pid; C.cell = cell; C.start = start; C.list = list;
    C.md = S.melt[m]; C.melt = m; C.lim2 = S.db_lim2; C.kfene = st.kfene; C.R0 = sqrt(st.R0sq); C.T = T; C.qmin = st.qmin;
    return C;
}

__global__ void __launch_bounds__(128) k_db_eval(const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp,
                                                const double *__restrict__ x, const int *__restrict__ pid,
                                                const int *__restrict__ cell, const int *__restrict__ start,
                                                const int *__restrict__ list, const int *__restrict__ koff,
                                                const int *__restrict__ comp_of, const int *__restrict__ slot_of,
                                                Attempt *__restrict__ att, long long sweep, unsigned *flags)
{
    if (flags[0]) return;                          // a latched error stops the sweep
    const SimDev &S = *Sp;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= koff[S.n_melts]) return;
    int m = 0;
    while (g >= koff[m + 1]) ++m;
    const DBC C = make_dbc(S, *stp, m, x, pid, cell, start, list, stp->T);
    unsigned err = 0;
    att[g] = evaluate(C, ViewMap{comp_of, slot_of}, S.seed, sweep, g - koff[m], S.paper_metropolis, err);
    if (err) atomicOr(flags, err);
}

__device__ __forceinline__ bool cells_near(int a, int b, int off, int n)
{
    a -= off; b -= off;
    const int ax = a % n, ay = (a / n) % n, az = a / (n * n);
    const int bx = b % n, by = (b / n) % n, bz = b / (n * n);
    int dx = abs(ax - bx), dy = abs(ay - by), dz = abs(az - bz);
    dx = min(dx, n - dx); dy = min(dy, n - dy); dz = min(dz, n - dz);
    return dx <= 1 && dy <= 1 && dz <= 1;
}

// One block per melt: ordered validation and commit.
__global__ void __launch_bounds__(256) k_db_commit(const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp,
                                                  const double *__restrict__ x, const int *__restrict__ pid,
                                                  const int *__restrict__ cell, const int *__restrict__ start,
                                                  const int *__restrict__ list, const int *__restrict__ koff,
                                                  const Attempt *__restrict__ att, int *__restrict__ occ,
                                                  int *__restrict__ curmap, int *__restrict__ img,
                                                  int *__restrict__ dirty, long long *__restrict__ stats,
                                                  long long sweep, unsigned *flags)
{
    extern __shared__ int old_occ[];              // 2N ints
    __shared__ int jcell[JCAP];
    __shared__ int njc;
    __shared__ Attempt a_s;
    __shared__ int need_s, sh[6];
    __shared__ long long n_acc, n_empty, n_re;
    const SimDev &S = *Sp;
    const int m = blockIdx.x;
    if (flags[0]) {                                // a latched error stops the sweep
        if (threadIdx.x == 0) for (int k = 0; k < 4; ++k) stats[4 * m + k] = 0;
        return;
    }
    const MeltDev &md = S.melt[m];
    const int N = md.N, off = md.off, Mp = S.Mp, tid = threadIdx.x;
    const DBC C = make_dbc(S, *stp, m, x, pid, cell, start, list, stp->T);
    const ViewMap V{occ, curmap};
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
                    if (p >= 0 && cells_near(jcell[j], cell[p], md.dbcell_off, md.ndb)) near = true;
                }
            }
        }
        const bool need = __syncthreads_or(near || need_s);
        if (need && tid == 0) {
            unsigned err = 0;
            a_s = evaluate(C, V, S.seed, sweep, kk, S.paper_metropolis, err);
            if (err) atomicOr(flags, err);
            ++n_re;
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

// end of a sweep: box shifts into the positions (x + L*img, as one rounding of
// a product and one of a sum), counters cleared
__global__ void __launch_bounds__(256) k_db_finish(const SimDev *__restrict__ Sp, double *__restrict__ x,
                                                  const int *__restrict__ slot_of, int *__restrict__ img,
                                                  int *__restrict__ dirty)
{
    const SimDev &S = *Sp;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S.M) return;
    const int Mp = S.Mp;
    const double L = S.melt[melt_of(S, slot_of[j])].L;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int k = img[d * Mp + j];
        if (k) x[d * Mp + j] = __dadd_rn(x[d * Mp + j], __dmul_rn(L, (double)k));
        img[d * Mp + j] = 0;
    }
    dirty[j] = 0;
}

// kg_md.cu
__global__ void k_bin_db(const SimDev *__restrict__ Sp, const double *__restrict__ x, int *__restrict__ cellid,
                         int *__restrict__ rank, int *__restrict__ count, const int *__restrict__ slot_of);
__global__ void k_scan1(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ bsum, int n,
                        const unsigned *__restrict__ flags);
__global__ void k_scan2(int *__restrict__ out, const int *__restrict__ bsum, int n, int nblk,
                        const unsigned *__restrict__ flags);
__global__ void k_scatter(const int *__restrict__ cellid, const int *__restrict__ rank,
                          const int *__restrict__ start, int *__restrict__ list, int M,
                          const unsigned *__restrict__ flags, const float4 *__restrict__ recb,
                          float4 *__restrict__ recs);

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

void db_sweep(kg_ctx *c, const std::vector<long long> &K, long long *host_stats)
{
    cudaStream_t st = c->stream;
    const int nm = c->sim.n_melts;
    c->launches += 7;
    std::vector<int> koff(nm + 1, 0);
    for (int m = 0; m < nm; ++m) koff[m + 1] = koff[m] + (int)K[m];
    cudaMemcpyAsync(c->koff, koff.data(), sizeof(int) * (nm + 1), cudaMemcpyHostToDevice, st);
    // 1. grid of >= 1.3 sigma cells
    cudaMemsetAsync(c->dbcount, 0, sizeof(int) * c->ncell_db, st);
    k_bin_db<<<nblk(c->M, 256), 256, 0, st>>>(c->d_sim, c->x, c->dbcell, c->dbrank, c->dbcount, c->slot_of);
    const int nb = nblk(c->ncell_db, 1024);
    k_scan1<<<nb, 1024, 0, st>>>(c->dbcount, c->dbstart, c->bsum, c->ncell_db, nullptr);
    k_scan2<<<nb, 1024, 0, st>>>(c->dbstart, c->bsum, c->ncell_db, nb, nullptr);
    k_scatter<<<nblk(c->M, 256), 256, 0, st>>>(c->dbcell, c->dbrank, c->dbstart, c->dblist, c->M, nullptr,
                                               nullptr, nullptr);
    // 2. speculative evaluation
    Attempt *att = (Attempt *)c->att;
    if (koff[nm] > 0)
        k_db_eval<<<nblk(koff[nm], 128), 128, 0, st>>>(c->d_sim, c->d_stage, c->x, c->pid, c->dbcell, c->dbstart,
                                                       c->dblist, c->koff, c->comp_of, c->slot_of, att, c->sweep,
                                                       c->flags);
    // 3. ordered commit, one block per melt
    int maxN = 0;
    for (int m = 0; m < nm; ++m) maxN = maxN > c->sim.melt[m].N ? maxN : c->sim.melt[m].N;
    k_db_commit<<<nm, 256, sizeof(int) * 2 * maxN, st>>>(c->d_sim, c->d_stage, c->x, c->pid, c->dbcell,
                                                          c->dbstart, c->dblist, c->koff, att, c->comp_of,
                                                          c->slot_of, c->img, c->dirty, c->db_stats, c->sweep,
                                                          c->flags);
    // 4. box shifts into the positions; chain partners follow the new maps
    k_db_finish<<<nblk(c->M, 256), 256, 0, st>>>(c->d_sim, c->x, c->slot_of, c->img, c->dirty);
    bonded_partners(c);
    cudaMemcpyAsync(host_stats, c->db_stats, sizeof(long long) * 4 * nm, cudaMemcpyDeviceToHost, st);
}

}  // namespace kg
