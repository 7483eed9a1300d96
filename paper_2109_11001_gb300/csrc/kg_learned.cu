// kg_learned.cu -- double-bridging sweep with a learned partner proposal.
//
// The paper draws a swap partner uniformly from the admissible list P(b) of
// the drawn bond (Fig. 1).  Here the list, in the same order, is weighted by
//     pi_j = (1 - lambda) softmax_j(s) + lambda / |P(b)|,
// s_j the logit the network (kg_mlp.cuh) assigns to the features of swap j,
// and the swap is accepted with min(1, exp(-dE/T) q(x'->x) / q(x->x')), where
// q(x->x') = pi_b(move) + pi_b'(move) sums the two ways of proposing it (either
// removed bond drawn) and q(x'->x) the same in the swapped state.  lambda > 0
// keeps every admissible swap proposable, so the chain stays irreducible;
// lambda = 1 is the uniform proposal, with the Hastings ratio of Fig. 1.
//
// Features (24 per swap; u-w the drawn bond, X-Y the partner bond, new bonds
// u-X and Y-w; every value depends on positions and bonds only, not on the
// direction in which a chain's slots are numbered):
//   0-1 removed bond lengths (sorted)       2-3 new bond lengths (sorted)
//   4   change of the FENE terms             5   change of the bending energy
//   6-9 cos at the four junction vertices, before (sorted)
//   10-13 the same after                    14-17 cos one vertex further out (sorted)
//   18  cos between u->w and X->Y            19 kappa/4   20 n/12
//   21  min(p+1, N-1-p)/N (p the drawn bond) 22 dE = 4 + 5   23 1
//
// GPU organisation (one warp per attempt): the warp scans the 27 cells around
// the drawn bond's lower monomer, ranks the candidates by monomer ids, computes
// their features (FP64, one lane each), runs the network on the tensor cores
// in 16-row tiles, and lane 0 forms pi in FP64 in list order.  The forward
// probability of the partner bond and the two reverse probabilities repeat
// this for three more bonds (the reverse ones in the swapped topology view).
// Attempts are evaluated speculatively in parallel and committed in order by
// the shared commit walk (kg_db.cuh); a learned evaluation reads monomers up
// to 2 b_lim + 3 b_max from its junction monomers (b_lim = 1.3 the swap bond
// limit, b_max the longest bond at sweep start), so an accepted swap with a
// junction monomer within that many cells forces a re-evaluation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "kg_db.cuh"
#include "kg_mlp.cuh"

namespace kg {

struct LearnedArgs {
    double lambda;
    const MlpSmem *w;                   // bf16 image of the network
    double *logf, *logt;                // per-attempt log staging (null: no log)
    int *logn;
    const unsigned long long *bmax2;    // longest bond squared, binary64 bits
    const float4 *rec;                  // binary32 records on the DB grid (swap-bond prefilter)
};

// per-warp shared scratch of one proposal evaluation
struct __align__(16) WarpProp : WarpCand {
    double pi[CAND_CAP];
    double dE[CAND_CAP];
    float s[CAND_CAP];
    __nv_bfloat16 F[CAND_CAP * S1];     // features of the candidates, bf16 rows
};

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void sort4(double *v)
{
    for (int i = 1; i < 4; ++i) {
        const double t = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > t) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = t;
    }
}

// Features of swap m of bond (c, b) in view v (one lane).
template <class V>
__device__ void move_features(const DBC &C, const V &v, int c, int b, const Cand &m, double *f)
{
    const MeltDev &md = C.md;
    const int N = md.N, off = md.off;
    const int u = v.occ(off + c * N + b), w = v.occ(off + c * N + b + 1);
    int X, Y;
    if (m.kind == 0) {
        Y = v.occ(off + m.d * N + b);
        X = v.occ(off + m.d * N + b + 1);
    } else {
        X = v.occ(off + m.d * N + m.q);
        Y = v.occ(off + m.d * N + m.q + 1);
    }
    const double o1 = sqrt(d2(C, u, w)), o2 = sqrt(d2(C, X, Y));
    const double n1 = sqrt(d2(C, u, X)), n2 = sqrt(d2(C, Y, w));
    f[0] = o1 < o2 ? o1 : o2;
    f[1] = o1 < o2 ? o2 : o1;
    f[2] = n1 < n2 ? n1 : n2;
    f[3] = n1 < n2 ? n2 : n1;
    f[4] = fene_of_r(C, n1) + fene_of_r(C, n2) - fene_of_r(C, o1) - fene_of_r(C, o2);
    const int A = c < m.d ? c : m.d, B = c < m.d ? m.d : c;
    const int pA = A == c ? b : m.q, pB = A == c ? m.q : b;
    double before[4] = {vcos(C, v, A, pA), vcos(C, v, A, pA + 1), vcos(C, v, B, pB), vcos(C, v, B, pB + 1)};
    double outer[4] = {vcos(C, v, A, pA - 1), vcos(C, v, A, pA + 2), vcos(C, v, B, pB - 1),
                       vcos(C, v, B, pB + 2)};
    const ViewMove<V> mv{v, m.kind, A, B, pA, pB, N, off};
    double after[4] = {vcos(C, mv, A, pA), vcos(C, mv, A, pA + 1), vcos(C, mv, B, pB), vcos(C, mv, B, pB + 1)};
    double db = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) db += md.kappa * ((1.0 - after[i]) - (1.0 - before[i]));
    f[5] = db;
    sort4(before);
    sort4(after);
    sort4(outer);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[6 + i] = before[i];
        f[10 + i] = after[i];
        f[14 + i] = outer[i];
    }
    double e1[3], e2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e1[k] = min_image_exact(C.x[k * C.Mp + w] - C.x[k * C.Mp + u], md.L);
        e2[k] = min_image_exact(C.x[k * C.Mp + Y] - C.x[k * C.Mp + X], md.L);
    }
    f[18] = (e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2])
            / (sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) * sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
    f[19] = md.kappa / 4.0;
    f[20] = C.nexp / 12.0;
    const int lo = b + 1 < N - 1 - b ? b + 1 : N - 1 - b;
    f[21] = (double)lo / N;
    f[22] = f[4] + f[5];
    f[23] = 1.0;
}

// Proposal weights of bond (c, b) in view v: wp.cand[0..n), wp.pi, and (when
// `features` or the network is in use) wp.dE and wp.F; wp.s (the logits) when
// the network ran (lambda < 1 and n > 1, or `logits`).  log_att >= 0 writes the
// FP64 features and targets min(1, exp(-dE/T)) of every candidate to that
// attempt's log rows.  Returns n (0: empty, -1: capacity error).
template <class V>
__device__ int proposal(const DBC &C, const V &v, const MlpSmem &W, WarpProp &wp, const LearnedArgs &la, int c,
                        int b, bool features, long long log_att, unsigned &err, bool logits = false)
{
    const int lane = threadIdx.x & 31;
    const int n = warp_partners<true>(C, v, c, b, wp, err);
    if (n <= 0) return n;
    // A one-entry list proposes its only swap with pi = (1 - lambda) + lambda
    // whatever the logit (the softmax of one value is exactly 1, so pi has the
    // same bits either way): unless the caller wants the logits, the network
    // and, unless dE or the log needs them, the features are skipped
    const bool net = la.lambda < 1.0 && (n > 1 || logits);
    if (net || features) {
        const int nr = (n + 15) & ~15;
        for (int j = lane; j < nr; j += 32) {
            __nv_bfloat16 *row = wp.F + j * S1;
            if (j < n) {
                double f[24];
                move_features(C, v, c, b, wp.cand[j], f);
                wp.dE[j] = f[22];
#pragma unroll
                for (int i = 0; i < 24; ++i) row[i] = __double2bfloat16(f[i]);
                if (log_att >= 0) {
                    double *o = la.logf + (log_att * CAND_CAP + j) * 24;
#pragma unroll
                    for (int i = 0; i < 24; ++i) o[i] = f[i];
                    const double de = f[22] / C.T;
                    la.logt[log_att * CAND_CAP + j] = de > 0.0 ? exp(-de) : 1.0;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) row[i] = __float2bfloat16(0.f);
            }
#pragma unroll
            for (int i = 24; i < 32; ++i) row[i] = __float2bfloat16(0.f);
        }
        if (log_att >= 0 && lane == 0) la.logn[log_att] = n;
        __syncwarp();
    }
    if (net) {
        const int g = lane >> 2;
        for (int r0 = 0; r0 < n; r0 += 16) {
            float s0, s1;
            mlp_forward16(W, wp.F + r0 * S1, s0, s1);
            if ((lane & 3) == 0) {
                if (r0 + g < n) wp.s[r0 + g] = s0;
                if (r0 + g + 8 < n) wp.s[r0 + g + 8] = s1;
            }
        }
        __syncwarp();
    }
    if (lane == 0) {                                // FP64, in list order
        double smax = -1e300, z = 0.0;
        for (int j = 0; j < n; ++j) {
            const double s = net ? (double)wp.s[j] : 0.0;
            if (s > smax) smax = s;
        }
        for (int j = 0; j < n; ++j) z += exp((net ? (double)wp.s[j] : 0.0) - smax);
        for (int j = 0; j < n; ++j)
            wp.pi[j] = (1.0 - la.lambda) * exp((net ? (double)wp.s[j] : 0.0) - smax) / z + la.lambda / n;
    }
    __syncwarp();
    return n;
}

// Probability that bond (c, b)'s proposal picks the swap (kind, A, B, pA, pB).
template <class V>
__device__ double match_prob(const DBC &C, const V &v, const MlpSmem &W, WarpProp &wp, const LearnedArgs &la,
                             int c, int b, int kind, int A, int B, int pA, int pB, unsigned &err)
{
    const int lane = threadIdx.x & 31;
    const int n = proposal(C, v, W, wp, la, c, b, false, -1, err);
    double p = 0.0;
    if (n > 0 && lane == 0) {
        for (int j = 0; j < n; ++j) {
            const Cand &m = wp.cand[j];
            const int a2 = c < m.d ? c : m.d, b2 = c < m.d ? m.d : c;
            const int pa2 = a2 == c ? b : m.q, pb2 = a2 == c ? m.q : b;
            if (m.kind == kind && a2 == A && b2 == B && pa2 == pA && pb2 == pB) {
                p = wp.pi[j];
                break;
            }
        }
    }
    p = __shfl_sync(FULL, p, 0);
    __syncwarp();
    return p;
}

// One attempt (k of this melt's sweep; g its global index), whole warp.
template <class V>
__device__ Attempt learned_eval(const DBC &C, const V &v, const MlpSmem &W, WarpProp &wp, const LearnedArgs &la,
                                unsigned long long seed, long long sweep, int k, int g, unsigned &err)
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
    const double upick = (double)((((unsigned long long)r2.y << 32) | r2.x) >> 11) * (1.0 / 9007199254740992.0);
    const int c = (int)(bond / (N - 1)), b = (int)(bond % (N - 1));
    a.c = c;
    a.jp[0] = v.occ(off + c * N + b);
    a.jp[1] = v.occ(off + c * N + b + 1);
    if (la.logn && lane == 0) la.logn[g] = 0;
    const int n1 = proposal(C, v, W, wp, la, c, b, true, la.logf ? (long long)g : -1LL, err);
    if (n1 <= 0) return a;                         // empty, or a capacity error (bit set)
    int j = 0;
    if (lane == 0) {
        double cum = wp.pi[0];
        while (j + 1 < n1 && upick >= cum) cum += wp.pi[++j];
    }
    j = __shfl_sync(FULL, j, 0);
    const Cand m = wp.cand[j];
    const double pij = wp.pi[j], dE = wp.dE[j];
    __syncwarp();
    a.flags = 1;
    a.d = m.d;
    a.jp[2] = v.occ(off + m.d * N + m.q);
    a.jp[3] = v.occ(off + m.d * N + m.q + 1);
    const int A = c < m.d ? c : m.d, B = c < m.d ? m.d : c;
    const int pA = A == c ? b : m.q, pB = A == c ? m.q : b;
    a.kind = m.kind; a.A = A; a.B = B; a.pA = pA; a.pB = pB;
    const double q_fwd = pij + match_prob(C, v, W, wp, la, m.d, m.q, m.kind, A, B, pA, pB, err);
    const ViewMove<V> w{v, m.kind, A, B, pA, pB, N, off};
    const double q_rev = match_prob(C, w, W, wp, la, A, pA, m.kind, A, B, pA, pB, err)
                         + match_prob(C, w, W, wp, la, B, pB, m.kind, A, B, pA, pB, err);
    if (!(q_rev > 0.0) || !(q_fwd > 0.0)) {
        err |= ERR_DB_INTERNAL;
        return a;
    }
    const double acc = exp(-dE / C.T) * q_rev / q_fwd;
    if (uacc < acc) a.flags |= 2;
    return a;
}

constexpr int EVAL_WARPS = 4;

__host__ __device__ constexpr size_t eval_smem() { return sizeof(MlpSmem) + EVAL_WARPS * sizeof(WarpProp); }

__global__ void __launch_bounds__(32 * EVAL_WARPS) k_dbl_eval(const SimDev *__restrict__ Sp,
                                                             const StageDev *__restrict__ stp,
                                                             const double *__restrict__ x,
                                                             const int *__restrict__ pid,
                                                             const int *__restrict__ cell,
                                                             const int *__restrict__ start,
                                                             const int *__restrict__ list,
                                                             const int *__restrict__ koff,
                                                             const int *__restrict__ comp_of,
                                                             const int *__restrict__ slot_of,
                                                             Attempt *__restrict__ att, long long sweep,
                                                             unsigned *flags, LearnedArgs la)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpSmem &W = *reinterpret_cast<MlpSmem *>(smem);
    WarpProp *wps = reinterpret_cast<WarpProp *>(smem + sizeof(MlpSmem));
    mlp_load(W, la.w);
    __syncthreads();
    if (flags[0]) return;                          // a latched error stops the sweep (no block barrier follows)
    const SimDev &S = *Sp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * EVAL_WARPS + warp;
    if (g >= koff[S.n_melts]) return;
    int m = 0;
    while (g >= koff[m + 1]) ++m;
    const DBC C = make_dbc(S, *stp, m, x, pid, cell, start, list, la.rec, stp->T);
    unsigned err = 0;
    const Attempt a = learned_eval(C, ViewMap{comp_of, slot_of}, W, wps[warp], la, S.seed, sweep, g - koff[m], g, err);
    if (lane == 0) {
        att[g] = a;
        if (err) atomicOr(flags, err);
    }
}

// learned proposal: a stale record is re-evaluated by one warp with the
// network in shared memory; the reach of an evaluation sets the radius
struct LearnedEval {
    const SimDev *S;
    const StageDev *st;
    const double *x;
    const int *pid, *cell, *start, *list;
    const int *comp_of, *slot_of;
    long long sweep;
    unsigned *flags;
    LearnedArgs la;
    const MlpSmem *W;
    WarpProp *wp;
    __device__ void eval(int m, int k, int g, Attempt &out)
    {
        const DBC C = make_dbc(*S, *st, m, x, pid, cell, start, list, la.rec, st->T);
        unsigned err = 0;
        const Attempt a = learned_eval(C, ViewMap{comp_of, slot_of}, *W, *wp, la, S->seed, sweep, k, g, err);
        if ((threadIdx.x & 31) == 0) {
            out = a;
            if (err) atomicOr(flags, err);
        }
    }
};

struct LearnedRadius {
    const unsigned long long *bmax2;
    double lim;                                    // swap bond limit (1.3)
    __device__ void init() {}
    // cells within 2 lim + 3 max(b_max, lim) of a junction monomer, one extra
    // cell against rounding at cell faces
    __device__ int radius(const MeltDev &md) const
    {
        const double bmax = sqrt(__longlong_as_double((long long)*bmax2));
        const double reach = 2.0 * lim + 3.0 * fmax(bmax, lim);
        return (int)ceil(reach * md.invhdb) + 1;
    }
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ constexpr size_t restale_smem() { return sizeof(MlpSmem) + EVAL_WARPS * sizeof(WarpProp); }

__global__ void __launch_bounds__(32 * EVAL_WARPS) k_dbl_restale(
    const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp, const double *__restrict__ x,
    const int *__restrict__ pid, const int *__restrict__ cell, const int *__restrict__ start,
    const int *__restrict__ list, const int *__restrict__ koff, const int *__restrict__ comp_of,
    const int *__restrict__ slot_of, Attempt *__restrict__ att, int *__restrict__ ver,
    const int *__restrict__ chain_ver, const int *__restrict__ cell_ver, int *__restrict__ round, long long sweep,
    unsigned *flags, LearnedArgs la)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpSmem &W = *reinterpret_cast<MlpSmem *>(smem);
    WarpProp *wps = reinterpret_cast<WarpProp *>(smem + sizeof(MlpSmem));
    mlp_load(W, la.w);
    __syncthreads();
    if (flags[0]) return;                          // a latched error stops the sweep (no block barrier follows)
    LearnedEval ev{Sp, stp, x, pid, cell, start, list, comp_of, slot_of, sweep, flags, la, &W,
                   wps + (threadIdx.x >> 5)};
    restale_body(ev, *Sp, koff, att, ver, chain_ver, cell, cell_ver, round);
}

__global__ void __launch_bounds__(256) k_dbl_commit_next(
    const SimDev *__restrict__ Sp, const double *__restrict__ x, const int *__restrict__ cell,
    const int *__restrict__ koff, const Attempt *__restrict__ att, int *__restrict__ occ, int *__restrict__ curmap,
    int *__restrict__ img, int *__restrict__ chain_ver, int *__restrict__ cell_ver, int *__restrict__ round,
    long long *__restrict__ stats, unsigned *flags, const unsigned long long *bmax2)
{
    extern __shared__ int old_occ[];              // 2N ints
    LearnedRadius pol{bmax2, sqrt(Sp->db_lim2)};
    commit_next_body(pol, *Sp, x, cell, koff, att, occ, curmap, img, chain_ver, cell_ver, round, stats, flags,
                     old_occ);
}

// longest bond of all melts, squared, as ordered binary64 bits
__global__ void __launch_bounds__(256) k_bond_max(const SimDev *__restrict__ Sp, const double *__restrict__ x,
                                                 const int *__restrict__ comp_of, unsigned long long *bmax2)
{
    const SimDev &S = *Sp;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0;
    if (s < S.M) {
        const MeltDev &md = S.melt[melt_of(S, s)];
        const int i = (s - md.off) % md.N;
        if (i < md.N - 1) r2 = dist2_exact(x, S.Mp, md.L, comp_of[s], comp_of[s + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmax(r2, __shfl_xor_sync(FULL, r2, o));
    if ((threadIdx.x & 31) == 0 && r2 > 0.0) atomicMax(bmax2, (unsigned long long)__double_as_longlong(r2));
}

// Append the sweep's log rows (attempt order, list order within an attempt)
// to the training ring; one block.
__global__ void __launch_bounds__(1024) k_log_append(const int *__restrict__ logn, int Ktot,
                                                    const double *__restrict__ sf, const double *__restrict__ st,
                                                    double *__restrict__ rf, double *__restrict__ rt, long long cap,
                                                    long long *head, const unsigned *flags)
{
    __shared__ int scan[1024];
    __shared__ long long base, total;
    if (flags[0]) return;
    const int tid = threadIdx.x;
    if (tid == 0) {
        base = *head;
        total = 0;
    }
    __syncthreads();
    // rows that an append of more than `cap` rows overwrites within itself are
    // skipped, so no two writes of one pass land on the same ring slot
    long long mine = 0;
    for (int k = tid; k < Ktot; k += 1024) mine += logn[k];
    atomicAdd(reinterpret_cast<unsigned long long *>(&total), (unsigned long long)mine);
    __syncthreads();
    const long long keep_from = base + total - cap;
    for (int k0 = 0; k0 < Ktot; k0 += 1024) {
        const int k = k0 + tid;
        const int n = k < Ktot ? logn[k] : 0;
        scan[tid] = n;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int add = tid >= o ? scan[tid - o] : 0;
            __syncthreads();
            scan[tid] += add;
            __syncthreads();
        }
        const long long dst0 = base + scan[tid] - n;
        for (int j = 0; j < n; ++j) {
            if (dst0 + j < keep_from) continue;
            const long long dst = (dst0 + j) % cap;
            const double *src = sf + ((long long)k * CAND_CAP + j) * 24;
            for (int i = 0; i < 24; ++i) rf[dst * 24 + i] = src[i];
            rt[dst] = st[(long long)k * CAND_CAP + j];
        }
        __syncthreads();
        if (tid == 0) base += scan[1023];
        __syncthreads();
    }
    if (tid == 0) *head = base;
}

// One bond's learned proposal in the current topology (introspection).
__global__ void __launch_bounds__(32) k_dbl_proposal(const SimDev *__restrict__ Sp, const StageDev *__restrict__ stp,
                                                    const double *__restrict__ x, const int *__restrict__ pid,
                                                    const int *__restrict__ cell, const int *__restrict__ start,
                                                    const int *__restrict__ list, const int *__restrict__ comp_of,
                                                    const int *__restrict__ slot_of, int melt, int c, int b,
                                                    LearnedArgs la, int *out_i, double *out_d, unsigned *flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpSmem &W = *reinterpret_cast<MlpSmem *>(smem);
    WarpProp &wp = *reinterpret_cast<WarpProp *>(smem + sizeof(MlpSmem));
    mlp_load(W, la.w);
    __syncthreads();
    const SimDev &S = *Sp;
    const DBC C = make_dbc(S, *stp, melt, x, pid, cell, start, list, la.rec, stp->T);
    unsigned err = 0;
    // log rows of "attempt" 0 go to out_d[0 .. 48*24) (features) and out_d[48*24 ..) (targets)
    la.logf = out_d;
    la.logt = out_d + CAND_CAP * 24;
    la.logn = out_i;
    const int n = proposal(C, ViewMap{comp_of, slot_of}, W, wp, la, c, b, true, 0, err, true);
    const int lane = threadIdx.x;
    out_i[0] = n;                                  // every lane writes the same value
    for (int j = lane; j < (n > 0 ? n : 0); j += 32) {
        out_i[1 + j] = wp.cand[j].kind;
        out_i[1 + CAND_CAP + j] = wp.cand[j].d;
        out_i[1 + 2 * CAND_CAP + j] = wp.cand[j].q;
        out_d[CAND_CAP * 25 + j] = la.lambda < 1.0 ? (double)wp.s[j] : 0.0;
        out_d[CAND_CAP * 26 + j] = wp.pi[j];
    }
    if (lane == 0 && err) atomicOr(flags, err);
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

static bool ensure_log_staging(kg_ctx *c, long long tot)
{
    if (tot <= c->log_att_cap) return true;
    dev_free(c, c->logf);
    dev_free(c, c->logt);
    dev_free(c, c->logn);
    const long long cap = tot > 2 * c->log_att_cap ? tot : 2 * c->log_att_cap;
    c->logf = (double *)dev_alloc(c, sizeof(double) * 24 * CAND_CAP * (size_t)cap);
    c->logt = (double *)dev_alloc(c, sizeof(double) * CAND_CAP * (size_t)cap);
    c->logn = (int *)dev_alloc(c, sizeof(int) * (size_t)cap);
    c->log_att_cap = (c->logf && c->logt && c->logn) ? cap : 0;
    return c->log_att_cap > 0;
}

static LearnedArgs make_args(kg_ctx *c, double lambda, bool log)
{
    LearnedArgs la;
    la.lambda = lambda;
    la.w = (const MlpSmem *)c->mlp_blob;
    la.logf = log ? c->logf : nullptr;
    la.logt = log ? c->logt : nullptr;
    la.logn = log ? c->logn : nullptr;
    la.bmax2 = c->bmax2;
    la.rec = c->dbrec;
    return la;
}

void db_sweep_learned(kg_ctx *c, const std::vector<long long> &K, double lambda, long long *host_stats)
{
    cudaStream_t st = c->stream;
    const int nm = c->sim.n_melts;
    long long tot = 0;
    for (long long k : K) tot += k;
    const bool log = c->train_cap > 0 && ensure_log_staging(c, tot > 0 ? tot : 1);
    const LearnedArgs la = make_args(c, lambda, log);
    db_bin(c, K);
    cudaMemsetAsync(c->bmax2, 0, sizeof(unsigned long long), st);
    k_bond_max<<<nblk(c->M, 256), 256, 0, st>>>(c->d_sim, c->x, c->comp_of, c->bmax2);
    Attempt *att = (Attempt *)c->att;
    if (tot > 0) {
        cudaFuncSetAttribute(k_dbl_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eval_smem());
        k_dbl_eval<<<nblk(tot, EVAL_WARPS), 32 * EVAL_WARPS, eval_smem(), st>>>(
            c->d_sim, c->d_stage, c->x, c->pid, c->dbcell, c->dbstart, c->dblist, c->koff, c->comp_of, c->slot_of,
            att, c->sweep, c->flags, la);
    }
    // ordered commit in rounds (kg_db.cuh)
    db_rounds_reset(c, tot);
    const int maxN = db_max_chain_len(c);
    const size_t sm = sizeof(int) * 2 * (size_t)maxN;
    cudaFuncSetAttribute(k_dbl_commit_next, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_dbl_restale, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)restale_smem());
    const int rgrid = std::max(1, std::min(nblk(tot, 32 * EVAL_WARPS), 152 * 4));
    db_rounds(c, tot,
              [&] {
                  k_dbl_restale<<<rgrid, 32 * EVAL_WARPS, restale_smem(), st>>>(
                      c->d_sim, c->d_stage, c->x, c->pid, c->dbcell, c->dbstart, c->dblist, c->koff, c->comp_of,
                      c->slot_of, att, c->att_ver, c->chain_ver, c->dbmark, c->dbround, c->sweep, c->flags, la);
              },
              [&] {
                  k_dbl_commit_next<<<nm, 256, sm, st>>>(c->d_sim, c->x, c->dbcell, c->koff, att, c->comp_of,
                                                         c->slot_of, c->img, c->chain_ver, c->dbmark, c->dbround,
                                                         c->db_stats, c->flags, c->bmax2);
              });
    c->launches += 2;
    if (log && tot > 0) {
        k_log_append<<<1, 1024, 0, st>>>(c->logn, (int)tot, c->logf, c->logt, c->trainf, c->traint, c->train_cap,
                                         c->d_train_head, c->flags);
        ++c->launches;
    }
    db_finish(c, host_stats);
}

bool db_proposal(kg_ctx *c, int melt, int chain, int bond, double lambda, int *h_n, int *h_ints, double *h_f,
                 double *h_s, double *h_pi)
{
    cudaStream_t st = c->stream;
    std::vector<long long> K(c->sim.n_melts, 0);
    db_bin(c, K);
    const size_t nd = CAND_CAP * 27, ni = 1 + 3 * CAND_CAP;
    double *dd = (double *)dev_alloc(c, sizeof(double) * nd);
    int *di = (int *)dev_alloc(c, sizeof(int) * ni);
    if (!dd || !di) {
        dev_free(c, dd);
        dev_free(c, di);
        return false;
    }
    const LearnedArgs la = make_args(c, lambda, false);
    const size_t sm = sizeof(MlpSmem) + sizeof(WarpProp);
    cudaFuncSetAttribute(k_dbl_proposal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_dbl_proposal<<<1, 32, sm, st>>>(c->d_sim, c->d_stage, c->x, c->pid, c->dbcell, c->dbstart, c->dblist,
                                      c->comp_of, c->slot_of, melt, chain, bond, la, di, dd, c->flags);
    ++c->launches;
    std::vector<double> hd(nd);
    std::vector<int> hi(ni);
    cudaMemcpyAsync(hd.data(), dd, sizeof(double) * nd, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hi.data(), di, sizeof(int) * ni, cudaMemcpyDeviceToHost, st);
    const bool ok = cudaStreamSynchronize(st) == cudaSuccess;
    dev_free(c, dd);
    dev_free(c, di);
    if (!ok) return false;
    const int n = hi[0];
    *h_n = n;
    for (int j = 0; j < (n > 0 ? n : 0); ++j) {
        h_ints[j] = hi[1 + j];
        h_ints[CAND_CAP + j] = hi[1 + CAND_CAP + j];
        h_ints[2 * CAND_CAP + j] = hi[1 + 2 * CAND_CAP + j];
        for (int i = 0; i < 24; ++i) h_f[j * 24 + i] = hd[j * 24 + i];
        h_s[j] = hd[CAND_CAP * 25 + j];
        h_pi[j] = hd[CAND_CAP * 26 + j];
    }
    return true;
}

}  // namespace kg
