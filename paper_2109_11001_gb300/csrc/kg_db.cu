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
//      during a sweep: swaps only relabel slots) and write its binary32 record
//      there; the 1.3 sigma criterion is decided on the records outside a
//      rounding band and in binary64 inside it, so decisions are exact;
//   2. k_db_eval: every attempt evaluated in parallel against the pre-sweep
//      topology, one warp each (the 27 cells of a partner scan on its lanes).
//      A "monomer" here is its compute index; the topology is the pair of
//      maps slot -> monomer (comp_of) and monomer -> slot (slot_of);
//   3. commit rounds (kg_db.cuh): an attempt's record is stale when an
//      earlier accepted swap in the sweep touched one of its two chains, or
//      put a junction monomer (whose bonds changed) within one cell of a
//      monomer whose neighbourhood it scanned.  Nothing else an evaluation
//      reads can change: swaps preserve positions, the bonds inside moved
//      segments, and the lengths of the two pieces on either side of every
//      bond.  Each round, k_db_restale re-evaluates the stale records across
//      the GPU, then k_db_commit_next (one block per melt) commits the first
//      accepted attempt: the two maps are rewritten for the slots of its two
//      chains and box shifts are added to a per-monomer counter;
//   4. k_db_finish: the box shifts are added to the positions in place; no
//      monomer data moves (the maps are the topology).
#include <cuda_runtime.h>

#include <algorithm>

#include "kg_db.cuh"

namespace kg {

// One attempt, one warp (the partner scans are warp-wide; lane 0 forms dE
// and the decision in binary64 and broadcasts the record).
template <class V>
__device__ Attempt evaluate(const DBC &C, const V &v, WarpCand &wc, unsigned long long seed, long long sweep, int k,
                            int paper, unsigned &err)
{
    const int lane = threadIdx.x & 31;
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
    const int n1 = warp_partners<true>(C, v, c, b, wc, err);
    if (n1 <= 0) return a;                              // empty, or a capacity error (flagged)
    const Cand m = wc.cand[mul_hi64(((unsigned long long)r2.y << 32) | r2.x, (unsigned long long)n1)];
    a.flags = 1;
    a.d = m.d;
    a.jp[2] = v.occ(off + m.d * N + m.q);
    a.jp[3] = v.occ(off + m.d * N + m.q + 1);
    const int n2 = warp_partners<false>(C, v, m.d, m.q, wc, err);
    if (n2 <= 0) { err |= n2 < 0 ? ERR_DB_CAPACITY : ERR_DB_INTERNAL; return a; }
    const int A = c < m.d ? c : m.d, B = c < m.d ? m.d : c;
    const int pA = A == c ? b : m.q, pB = A == c ? m.q : b;
    a.kind = m.kind; a.A = A; a.B = B; a.pA = pA; a.pB = pB;
    const ViewMove<V> w{v, m.kind, A, B, pA, pB, N, off};
    const int r1 = warp_partners<false>(C, w, A, pA, wc, err);
    const int rr2 = warp_partners<false>(C, w, B, pB, wc, err);
    if (r1 <= 0 || rr2 <= 0) { err |= (r1 < 0 || rr2 < 0) ? ERR_DB_CAPACITY : ERR_DB_INTERNAL; return a; }
    int acc_bit = 0;
    if (lane == 0) {
        double dE = bond_fene(C, w, A, pA) + bond_fene(C, w, B, pB) - bond_fene(C, v, A, pA) - bond_fene(C, v, B, pB);
        dE += bend(C, w, A, pA) + bend(C, w, A, pA + 1) + bend(C, w, B, pB) + bend(C, w, B, pB + 1);
        dE -= bend(C, v, A, pA) + bend(C, v, A, pA + 1) + bend(C, v, B, pB) + bend(C, v, B, pB + 1);
        const double ratio = (1.0 / r1 + 1.0 / rr2) / (1.0 / n1 + 1.0 / n2);
        double acc = exp(-dE / C.T);
        if (!paper) acc *= ratio;
        acc_bit = uacc < acc;
    }
    if (__shfl_sync(FULL_MASK, acc_bit, 0)) a.flags |= 2;
    return a;
}

constexpr int EVAL_WARPS_U = 4;                 // attempts (warps) per block of k_db_eval

// (128, 12): at most 40 registers; the partner scans are latency-bound, and
// more resident warps beat the spills (244 against 499 us for 160,000 attempts)
__global__ void __launch_bounds__(32 * EVAL_WARPS_U, 12) k_db_eval(const SimDev *__restrict__ Sp,
                                                              const StageDev *__restrict__ stp,
                                                              const double *__restrict__ x,
                                                              const int *__restrict__ pid,
                                                              const int *__restrict__ cell,
                                                              const int *__restrict__ start,
                                                              const int *__restrict__ list,
                                                              const float4 *__restrict__ rec,
                                                              const int *__restrict__ koff,
                                                              const int *__restrict__ comp_of,
                                                              const int *__restrict__ slot_of,
                                                              Attempt *__restrict__ att, long long sweep,
                                                              unsigned *flags)
{
    __shared__ WarpCand wcs[EVAL_WARPS_U];
    if (flags[0]) return;                          // a latched error stops the sweep (no block barrier follows)
    const SimDev &S = *Sp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * EVAL_WARPS_U + warp;
    if (g >= koff[S.n_melts]) return;
    int m = 0;
    while (g >= koff[m + 1]) ++m;
    const DBC C = make_dbc(S, *stp, m, x, pid, cell, start, list, rec, stp->T);
    unsigned err = 0;
    const Attempt a = evaluate(C, ViewMap{comp_of, slot_of}, wcs[warp], S.seed, sweep, g - koff[m],
                               S.paper_metropolis, err);
    if (lane == 0) {
        att[g] = a;
        if (err) atomicOr(flags, err);
    }
}

// uniform proposal: a stale record is re-evaluated by one warp; the
// staleness radius is one cell
struct UniformEval {
    const SimDev *S;
    const StageDev *st;
    const double *x;
    const int *pid, *cell, *start, *list;
    const float4 *rec;
    const int *comp_of, *slot_of;
    long long sweep;
    unsigned *flags;
    WarpCand *wc;
    __device__ void eval(int m, int k, int, Attempt &out)
    {
        const DBC C = make_dbc(*S, *st, m, x, pid, cell, start, list, rec, st->T);
        unsigned err = 0;
        const Attempt a = evaluate(C, ViewMap{comp_of, slot_of}, *wc, S->seed, sweep, k, S->paper_metropolis, err);
        if ((threadIdx.x & 31) == 0) {
            out = a;
            if (err) atomicOr(flags, err);
        }
    }
};

struct UniformRadius {
    __device__ void init() {}
    __device__ int radius(const MeltDev &) const { return 1; }
};

constexpr int RESTALE_WARPS = 8;

__global__ void __launch_bounds__(32 * RESTALE_WARPS) k_db_restale(
    const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp, const double *__restrict__ x,
    const int *__restrict__ pid, const int *__restrict__ cell, const int *__restrict__ start,
    const int *__restrict__ list, const float4 *__restrict__ rec, const int *__restrict__ koff,
    const int *__restrict__ comp_of, const int *__restrict__ slot_of, Attempt *__restrict__ att, int *__restrict__ ver,
    const int *__restrict__ chain_ver, const int *__restrict__ cell_ver, int *__restrict__ round, long long sweep,
    unsigned *flags)
{
    __shared__ WarpCand wcs[RESTALE_WARPS];
    if (flags[0]) return;                          // a latched error stops the sweep
    UniformEval ev{Sp, stp, x, pid, cell, start, list, rec, comp_of, slot_of, sweep, flags,
                   wcs + (threadIdx.x >> 5)};
    restale_body(ev, *Sp, koff, att, ver, chain_ver, cell, cell_ver, round);
}

constexpr int COMMIT_THREADS = 512;

__global__ void __launch_bounds__(COMMIT_THREADS) k_db_commit_next(
    const SimDev *__restrict__ Sp, const double *__restrict__ x, const int *__restrict__ cell,
    const int *__restrict__ koff, const Attempt *__restrict__ att, int *__restrict__ occ, int *__restrict__ curmap,
    int *__restrict__ img, int *__restrict__ chain_ver, int *__restrict__ cell_ver, int *__restrict__ round,
    long long *__restrict__ stats, unsigned *flags)
{
    extern __shared__ int old_occ[];              // 2N ints
    UniformRadius pol;
    commit_next_body(pol, *Sp, x, cell, koff, att, occ, curmap, img, chain_ver, cell_ver, round, stats, flags,
                     old_occ);
}

// end of a sweep: box shifts into the positions (x + L*img, as one rounding of
// a product and one of a sum), counters cleared
__global__ void __launch_bounds__(256) k_db_finish(const SimDev *__restrict__ Sp, double *__restrict__ x,
                                                  const int *__restrict__ slot_of, int *__restrict__ img,
                                                  double *__restrict__ msd_ref, double *__restrict__ xb64)
{
    const SimDev &S = *Sp;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S.M) return;
    const int Mp = S.Mp;
    const double L = S.melt[melt_of(S, slot_of[j])].L;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int k = img[d * Mp + j];
        if (k) {
            x[d * Mp + j] = __dadd_rn(x[d * Mp + j], __dmul_rn(L, (double)k));
            if (msd_ref) msd_ref[d * Mp + j] = __dadd_rn(msd_ref[d * Mp + j], __dmul_rn(L, (double)k));
            if (xb64) xb64[d * Mp + j] = __dadd_rn(xb64[d * Mp + j], __dmul_rn(L, (double)k));
        }
        img[d * Mp + j] = 0;
    }
}

// kg_md.cu
__global__ void k_bin_db(const SimDev *__restrict__ Sp, const double *__restrict__ x, int *__restrict__ cellid,
                         int *__restrict__ rank, int *__restrict__ count, const int *__restrict__ slot_of,
                         float4 *__restrict__ rec);
__global__ void k_scan1(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ bsum, int n,
                        const unsigned *__restrict__ flags);
__global__ void k_scan2(int *__restrict__ out, const int *__restrict__ bsum, int n, int nblk,
                        const unsigned *__restrict__ flags);
__global__ void k_scatter(const int *__restrict__ cellid, const int *__restrict__ rank,
                          const int *__restrict__ start, int *__restrict__ list, int M,
                          const unsigned *__restrict__ flags);

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

void db_bin(kg_ctx *c, const std::vector<long long> &K)
{
    cudaStream_t st = c->stream;
    const int nm = c->sim.n_melts;
    c->launches += 5;
    std::vector<int> koff(nm + 1, 0);
    for (int m = 0; m < nm; ++m) koff[m + 1] = koff[m] + (int)K[m];
    cudaMemcpyAsync(c->koff, koff.data(), sizeof(int) * (nm + 1), cudaMemcpyHostToDevice, st);
    // grid of >= 1.3 sigma cells
    cudaMemsetAsync(c->dbcount, 0, sizeof(int) * c->ncell_db, st);
    k_bin_db<<<nblk(c->M, 256), 256, 0, st>>>(c->d_sim, c->x, c->dbcell, c->dbrank, c->dbcount, c->slot_of,
                                              c->dbrec);
    const int nb = nblk(c->ncell_db, 1024);
    k_scan1<<<nb, 1024, 0, st>>>(c->dbcount, c->dbstart, c->bsum, c->ncell_db, nullptr);
    k_scan2<<<nb, 1024, 0, st>>>(c->dbstart, c->bsum, c->ncell_db, nb, nullptr);
    k_scatter<<<nblk(c->M, 256), 256, 0, st>>>(c->dbcell, c->dbrank, c->dbstart, c->dblist, c->M, nullptr);
}

void db_finish(kg_ctx *c, long long *host_stats)
{
    cudaStream_t st = c->stream;
    c->launches += 1;
    // box shifts into the positions; chain partners follow the new maps
    k_db_finish<<<nblk(c->M, 256), 256, 0, st>>>(c->d_sim, c->x, c->slot_of, c->img, c->msd_ref, c->xb64);
    bonded_partners(c);
    cudaMemcpyAsync(host_stats, c->db_stats, sizeof(long long) * 4 * c->sim.n_melts, cudaMemcpyDeviceToHost, st);
}

void db_rounds_reset(kg_ctx *c, long long tot)
{
    cudaStream_t st = c->stream;
    cudaMemsetAsync(c->chain_ver, 0xFF, sizeof(int) * (size_t)c->n_chain_total, st);    // -1: untouched
    cudaMemsetAsync(c->dbmark, 0xFF, sizeof(int) * (size_t)c->ncell_db, st);
    std::vector<int> r0((size_t)RS * MAX_MELTS, 0);
    for (int m = 0; m < MAX_MELTS; ++m) r0[(size_t)RS * m + 4] = INT_MAX;   // no accepted attempt known
    cudaMemcpyAsync(c->dbround, r0.data(), sizeof(int) * r0.size(), cudaMemcpyHostToDevice, st);
    if (tot > 0) cudaMemsetAsync(c->att_ver, 0, sizeof(int) * (size_t)tot, st);
}

int db_max_chain_len(const kg_ctx *c)
{
    int maxN = 0;
    for (int m = 0; m < c->sim.n_melts; ++m) maxN = maxN > c->sim.melt[m].N ? maxN : c->sim.melt[m].N;
    return maxN;
}

void db_sweep(kg_ctx *c, const std::vector<long long> &K, long long *host_stats)
{
    cudaStream_t st = c->stream;
    const int nm = c->sim.n_melts;
    long long tot = 0;
    for (long long k : K) tot += k;
    db_bin(c, K);
    // speculative evaluation
    Attempt *att = (Attempt *)c->att;
    if (tot > 0)
        k_db_eval<<<nblk(tot, EVAL_WARPS_U), 32 * EVAL_WARPS_U, 0, st>>>(
            c->d_sim, c->d_stage, c->x, c->pid, c->dbcell, c->dbstart, c->dblist, c->dbrec, c->koff, c->comp_of,
            c->slot_of, att, c->sweep, c->flags);
    // ordered commit in rounds (kg_db.cuh)
    db_rounds_reset(c, tot);
    const int maxN = db_max_chain_len(c);
    const size_t sm = sizeof(int) * 2 * (size_t)maxN;
    cudaFuncSetAttribute(k_db_commit_next, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int rgrid = std::max(1, std::min(nblk(tot, 32 * RESTALE_WARPS), 152 * 8));
    db_rounds(c, tot,
              [&] {
                  k_db_restale<<<rgrid, 32 * RESTALE_WARPS, 0, st>>>(
                      c->d_sim, c->d_stage, c->x, c->pid, c->dbcell, c->dbstart, c->dblist, c->dbrec, c->koff,
                      c->comp_of, c->slot_of, att, c->att_ver, c->chain_ver, c->dbmark, c->dbround, c->sweep,
                      c->flags);
              },
              [&] {
                  k_db_commit_next<<<nm, COMMIT_THREADS, sm, st>>>(c->d_sim, c->x, c->dbcell, c->koff, att,
                                                                   c->comp_of, c->slot_of, c->img, c->chain_ver,
                                                                   c->dbmark, c->dbround, c->db_stats, c->flags);
              });
    c->launches += 1;
    db_finish(c, host_stats);
}

}  // namespace kg
