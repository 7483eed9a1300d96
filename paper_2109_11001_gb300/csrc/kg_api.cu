// kg_api.cu -- C ABI of the GB300 DBH library: context lifecycle, potential
// schedule (Eqs. 9, 11, 12, 16-20), and dispatch of the MD / DB / observable
// kernels.  See include/kg.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "kg_host.h"

using kg::MeltDev;
using kg::SimDev;
using kg::StageDev;
using kg::dev_alloc;
using kg::dev_free;

namespace kg {

void *dev_alloc(kg_ctx *c, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (c->have_alloc) p = c->alloc.alloc(bytes, c->alloc.user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) cudaMemsetAsync(p, 0, bytes, c->stream);
    return p;
}

void dev_free(kg_ctx *c, void *p)
{
    if (!p) return;
    if (c->have_alloc) c->alloc.free(p, c->alloc.user);
    else cudaFree(p);
}

}  // namespace kg

namespace {

constexpr double RC = 1.122462048309373;   // 2^(1/6): cutoff and LJ minimum (Eq. 2)

// ---- schedule arithmetic (Sec. II.B) ----
const double XI[12] = {2, 3, 4, 5, 5.75, 6.5, 7, 8, 9, 10, 11, 12};   // Eq. 11

double lk_over_l0(double k)   // Eq. 12
{
    const double flory = k < 1e-4 ? 1.0 + 2.0 * k / 3.0
                                   : (2 * k + std::exp(-2 * k) - 1) / (1 - std::exp(-2 * k) * (2 * k + 1));
    return flory + 0.77 * (std::tanh(-0.03 * k * k - 0.41 * k + 0.16) + 1.0);
}

double kn_of(double n, double R0, double l0)   // Eq. 9
{
    return 6.0 * n * (R0 * R0 - l0 * l0) * (std::pow(2.0, n / 6.0) * std::pow(l0, -n) - 2.0 * std::pow(l0, -6.0))
           / ((n - 6.0) * R0 * R0 * l0 * l0);
}

kg_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return KG_OK;
    if (e == cudaErrorMemoryAllocation) return KG_ERR_OOM;
    return KG_ERR_CUDA;
}

#define KG_TRY(call)                                       \
    do {                                                   \
        kg_status _s = cuda_status(call);                  \
        if (_s != KG_OK) return _s;                        \
    } while (0)

// Stage parameters: U_MLJ^n = c1 r^-n - c2 r^-6 + 1 with c1 = 6 2^(n/6)/(n-6),
// c2 = 2n/(n-6) (Eq. 5 with m = 6, shifted at r_c); FENE k_n from Eq. 9 when
// the stage gives k < 0.
StageDev make_stage(const kg_params &p, const kg_stage &s)
{
    StageDev d{};
    const double n = s.n_exp;
    d.n = n;
    d.c1 = 6.0 * std::pow(2.0, n / 6.0) / (n - 6.0);
    d.c2 = 2.0 * n / (n - 6.0);
    d.kfene = s.k_fene < 0 ? kn_of(n, p.R0, p.l0) : s.k_fene;
    d.R0sq = p.R0 * p.R0;
    d.qmin = p.fene_qmin > 0 ? p.fene_qmin : 0.0;
    d.r2star = (1.0 - d.qmin) * d.R0sq;
    d.ustar = d.qmin > 0 ? -0.5 * d.kfene * d.R0sq * std::log(d.qmin) : 0.0;
    d.qminf = (float)d.qmin; d.r2starf = (float)d.r2star; d.ustarf = (float)d.ustar;
    d.dt = s.dt;
    d.gamma = p.gamma;
    d.T = p.T;
    d.amp = p.gamma > 0 ? std::sqrt(2.0 * p.gamma * p.T / s.dt) : 0.0;
    d.nf = (float)n; d.c1f = (float)d.c1; d.c2f = (float)d.c2; d.kfenef = (float)d.kfene;
    d.c2x6f = (float)(6.0 * d.c2); d.c1xnf = (float)(n * d.c1);
    d.R0sqf = (float)d.R0sq; d.dtf = (float)d.dt; d.gammaf = (float)d.gamma; d.ampf = (float)d.amp;
    const double rn = std::nearbyint(n);
    if (std::fabs(n - rn) < 1e-12 && rn >= 1 && rn <= 64) { d.nkind = 1; d.nint = (int)rn; }
    else if (n == 5.75) d.nkind = 2;
    else if (n == 6.5) d.nkind = 3;
    else d.nkind = 0;
    return d;
}

kg_status upload_stage(kg_ctx *c, const kg_stage &s)
{
    c->stage = make_stage(c->p, s);
    KG_TRY(cudaMemcpyAsync(c->d_stage, &c->stage, sizeof(StageDev), cudaMemcpyHostToDevice, c->stream));
    kg::graphs_reset(c);                     // the step kernel takes the stage by value
    return KG_OK;
}

__global__ void k_d2f(const double *__restrict__ a, float *__restrict__ b, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void k_f2d(const float *__restrict__ a, double *__restrict__ b, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}
__global__ void k_iota(int *__restrict__ a, int n, int base)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = base + i;
}

// Read the device status word; translate latched error bits.
kg_status read_flags(kg_ctx *c, unsigned *host4)
{
    KG_TRY(cudaMemcpyAsync(host4, c->flags, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, c->stream));
    KG_TRY(cudaStreamSynchronize(c->stream));
    const unsigned e = host4[0];
    kg_status s = KG_OK;
    if (e & kg::ERR_OVERSTRETCH) s = KG_ERR_BOND_OVERSTRETCH;
    else if (e & kg::ERR_NONFINITE) s = KG_ERR_NONFINITE;
    else if (e & (kg::ERR_NL_CAPACITY | kg::ERR_DB_CAPACITY | kg::ERR_DB_INTERNAL)) s = KG_ERR_CAPACITY;
    else if (e & kg::ERR_TIMEOUT) s = KG_ERR_TIMEOUT;
    if (s != KG_OK) c->latched = s;
    return s;
}

unsigned *pinned_flags()
{
    static thread_local unsigned *p = nullptr;
    if (!p && cudaMallocHost(&p, 64) != cudaSuccess) p = nullptr;
    return p;
}

kg_status set_rebuild(kg_ctx *c)
{
    static const unsigned one = 1u;
    KG_TRY(cudaMemcpyAsync(c->flags + 1, &one, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
    return KG_OK;
}

}  // namespace

extern "C" {

const char *kg_strerror(kg_status s)
{
    switch (s) {
        case KG_OK: return "ok";
        case KG_ERR_INVALID_ARG: return "invalid argument";
        case KG_ERR_CUDA: return "CUDA runtime error";
        case KG_ERR_OOM: return "device allocation failed";
        case KG_ERR_BOND_OVERSTRETCH: return "bond overstretched (r >= R0)";
        case KG_ERR_NONFINITE: return "non-finite force, velocity or position";
        case KG_ERR_CAPACITY: return "neighbour or candidate capacity exceeded";
        case KG_ERR_TIMEOUT: return "bounded device wait timed out";
        case KG_ERR_STATE: return "context has a latched error or no configuration";
    }
    return "unknown status";
}

double kg_kn(double n, double R0, double l0) { return kn_of(n, R0, l0); }

kg_status kg_schedule_paper(double kappa, int chain_len, double dt, double scale, kg_stage *out)
{
    if (!out || chain_len < 3 || !(dt > 0) || !(scale > 0) || kappa < 0) return KG_ERR_INVALID_ARG;
    const double N = chain_len;
    const double a = 1.6, b = 0.77, f0 = 46.3354;                          // Eq. 15 fit; Sec. II.B f_0
    const double ne = 77.0 * std::exp(-kappa / 1.1) + 9.4;                  // initial N_e estimate
    const double tau_e = ne * ne * lk_over_l0(kappa);                       // Eq. 17 (prefactor dropped)
    const double tau_fix = f0 * N / a * std::exp(b * kappa);               // Eq. 16
    double w[12], s11 = 0, s12 = 0;
    for (int i = 0; i < 12; ++i) {
        w[i] = 1.0 / std::sqrt(XI[i]);
        s12 += w[i];
        if (i < 11) s11 += w[i];
    }
    for (int i = 0; i < 12; ++i) {
        double tau;
        if (kappa <= 2.5)                                                   // Eq. 19
            tau = i < 11 ? w[i] / s11 * (200.0 * N - 2.0 * tau_e) : 2.0 * tau_e;
        else                                                                // Eq. 20
            tau = w[i] / s12 * tau_fix;
        out[i].n_exp = XI[i];
        out[i].k_fene = -1.0;
        out[i].n_steps = (long long)std::nearbyint(scale * tau / dt);
        out[i].dt = dt;
    }
    return KG_OK;
}

kg_status kg_create(kg_ctx **out, const kg_params *p, int device, void *stream, const kg_allocator *allocator)
{
    if (!out || !p || p->n_melts < 1 || p->n_melts > kg::MAX_MELTS || !p->melts) return KG_ERR_INVALID_ARG;
    if (p->precision != KG_FP64 && p->precision != KG_MIXED) return KG_ERR_INVALID_ARG;
    if (!(p->T > 0) || p->gamma < 0 || !(p->R0 > RC) || !(p->l0 > 0) || !(p->db_bond_max > 0) ||
        p->db_bond_max >= p->R0 || p->fene_qmin < 0 || p->fene_qmin >= 0.25 ||
        p->db_bond_max * p->db_bond_max > (1.0 - p->fene_qmin) * p->R0 * p->R0)
        return KG_ERR_INVALID_ARG;
    *out = nullptr;
    {   // every melt: chains of >= 3 monomers in a box that holds the cell grids
        const double skin = p->skin > 0 ? p->skin : 0.3;
        for (int m = 0; m < p->n_melts; ++m) {
            const kg_melt &ml = p->melts[m];
            if (ml.n_chains < 1 || ml.chain_len < 3 || !(ml.box > 7.0) || !(ml.kappa >= 0)) return KG_ERR_INVALID_ARG;
            if (ml.box / (RC + skin) > (1 << kg::CODE_BITS) || ml.box / p->db_bond_max < 3.0) return KG_ERR_INVALID_ARG;
        }
    }
    kg_ctx *c = new (std::nothrow) kg_ctx();
    if (!c) return KG_ERR_OOM;
    c->device = device;
    c->p = *p;
    c->melts.assign(p->melts, p->melts + p->n_melts);
    c->p.melts = c->melts.data();
    if (!(c->p.skin > 0)) c->p.skin = 0.3;
    c->sort_interval = p->sort_interval > 0 ? p->sort_interval : 200;
    c->block = p->block_size > 0 ? p->block_size : 128;
    if (c->block != 64 && c->block != 128 && c->block != 256) { delete c; return KG_ERR_INVALID_ARG; }
    c->tpm = p->threads_per_monomer > 0 ? p->threads_per_monomer : 1;
    if (c->tpm != 1 && c->tpm != 2) { delete c; return KG_ERR_INVALID_ARG; }
    if (p->precision != KG_MIXED) c->tpm = 1;
    c->precision = p->precision;
    if (allocator && allocator->alloc && allocator->free) { c->alloc = *allocator; c->have_alloc = true; }
    auto fail = [&](kg_status s) { kg_destroy(c); return s; };
    if (cudaSetDevice(device) != cudaSuccess) return fail(KG_ERR_CUDA);
    if (stream) c->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(KG_ERR_CUDA);
        c->own_stream = true;
    }

    // geometry of every melt
    SimDev &S = c->sim;
    S.n_melts = p->n_melts;
    const double rl = RC + c->p.skin;
    const double cscale = p->cell_scale > 0 ? p->cell_scale : 1.0;
    if (!(cscale >= 1.0 && cscale <= 3.0)) return fail(KG_ERR_INVALID_ARG);
    long long M = 0, ncell = 0, ndbcell = 0, nchain = 0;
    for (int m = 0; m < p->n_melts; ++m) {
        const kg_melt &ml = c->melts[m];
        if (ml.n_chains < 1 || ml.chain_len < 3 || !(ml.box > 7.0) || ml.kappa < 0) return fail(KG_ERR_INVALID_ARG);
        MeltDev &md = S.melt[m];
        md.off = (int)M;
        md.N = ml.chain_len;
        md.n_ch = ml.n_chains;
        md.M = ml.n_chains * ml.chain_len;
        md.L = ml.box; md.invL = 1.0 / ml.box; md.Lf = (float)ml.box;
        md.kappa = ml.kappa; md.kappaf = (float)ml.kappa;
        md.nc = (int)std::floor(ml.box / (cscale * rl * (1.0 + 1e-9)));
        md.ndb = (int)std::floor(ml.box / (p->db_bond_max * (1.0 + 1e-9)));
        if (md.nc < 3 || md.ndb < 3) return fail(KG_ERR_INVALID_ARG);
        md.h = ml.box / md.nc; md.invh = 1.0 / md.h;
        md.nbk = (md.nc + 3) / 4;
        md.hf = (float)md.h;
        md.invLf = (float)(1.0 / ml.box);
        {   // binary32 prefilter of the Verlet build on cell offsets (k_nlist):
            // the offsets (<= h), the shifted own offset (<= 2h) and the
            // difference (<= 3h) are rounded once each, and h itself once, so a
            // component is off by at most 9 h 2^-24; the band is twice the
            // resulting bound on r^2 near the cutoff.
            const double ec = 9.0 * md.h * std::ldexp(1.0, -24);
            const double er2 = 2.0 * rl * std::sqrt(3.0) * ec + 3.0 * ec * ec + 4.0 * rl * rl * std::ldexp(1.0, -24);
            md.nl_lo = (float)(rl * rl - 2.0 * er2);
            md.nl_hi = (float)(rl * rl + 2.0 * er2);
        }
        if (md.nc > (1 << kg::CODE_BITS)) return fail(KG_ERR_INVALID_ARG);
        md.hdb = ml.box / md.ndb; md.invhdb = 1.0 / md.hdb;
        md.hdbf = (float)md.hdb;
        if (md.ndb > (1 << kg::CODE_BITS)) return fail(KG_ERR_INVALID_ARG);
        if (md.ndb >= 11) {   // same error model as the Verlet prefilter, around db_bond_max^2
            const double lim = p->db_bond_max;
            const double ec = 9.0 * md.hdb * std::ldexp(1.0, -24);
            const double er2 = 2.0 * lim * std::sqrt(3.0) * ec + 3.0 * ec * ec + 4.0 * lim * lim * std::ldexp(1.0, -24);
            md.db_lo = (float)(lim * lim - 2.0 * er2);
            md.db_hi = (float)(lim * lim + 2.0 * er2);
        } else {              // small grids: every pair takes the binary64 distance
            md.db_lo = 0.0f;
            md.db_hi = 3.0e38f;
        }
        md.cell_off = (int)ncell;
        md.dbcell_off = (int)ndbcell;
        md.ch_off = (int)nchain;
        nchain += ml.n_chains;
        ncell += 64LL * md.nbk * md.nbk * md.nbk;
        ndbcell += (long long)md.ndb * md.ndb * md.ndb;
        M += md.M;
    }
    if (M >= (1LL << kg::IDX_BITS) || ncell >= (1LL << 30) || ndbcell >= (1LL << 30)) return fail(KG_ERR_INVALID_ARG);
    c->M = (int)M;
    c->Mp = (int)((M + 31) / 32 * 32);
    c->ncell_md = (int)ncell;
    c->ncell_db = (int)ndbcell;
    c->maxnb = 80;
    S.M = c->M; S.Mp = c->Mp; S.maxnb = c->maxnb;
    S.rc2 = RC * RC; S.rc2f = (float)S.rc2;
    S.rl = rl; S.rl2 = rl * rl;
    S.rl2f_lo = (float)(S.rl2 * (1.0 - 1e-5));
    S.rl2f_hi = (float)(S.rl2 * (1.0 + 1e-5));
    S.half_skin2 = 0.25 * c->p.skin * c->p.skin;
    S.half_skin2f = (float)S.half_skin2;
    S.db_lim2 = p->db_bond_max * p->db_bond_max;
    S.seed = p->seed;
    S.paper_metropolis = (p->flags & KG_FLAG_PAPER_METROPOLIS) ? 1 : 0;
    c->carry.assign(p->n_melts, 0.0);

    // device buffers
    const size_t Mp = c->Mp;
    const size_t ureal = c->precision == KG_MIXED ? sizeof(float) : sizeof(double);
    bool ok = true;
    auto A = [&](size_t bytes) { void *q = dev_alloc(c, bytes); ok = ok && q; return q; };
    c->d_sim = (SimDev *)A(sizeof(SimDev));
    c->d_stage = (StageDev *)A(sizeof(StageDev));
    c->x = (double *)A(3 * Mp * sizeof(double));
    if (c->precision == KG_MIXED) c->xb64 = (double *)A(3 * Mp * sizeof(double));
    c->u = A(3 * Mp * ureal);
    c->pid = (int *)A(Mp * sizeof(int));
    c->recb = (float4 *)A(Mp * sizeof(float4));
    // padded by a cell's worth of records: the list build reads a warp's
    // lockstep candidates past a cell's end without clamping the index
    c->recs = (float4 *)A((Mp + kg::MAX_CELL_OCC) * sizeof(float4));
    c->shtab = (float4 *)A((size_t)kg::SHIFT_SLOTS * kg::MAX_MELTS * sizeof(float4));
    if (c->precision == KG_MIXED) {
        for (int b = 0; b < 2; ++b) {
            c->dlt[b] = (float4 *)A(Mp * sizeof(float4));
            c->pg[b] = (float4 *)A(Mp * sizeof(float4));
        }
    } else {
        c->pos64[0] = (double4_32a *)A(Mp * sizeof(double4_32a));
        c->pos64[1] = (double4_32a *)A(Mp * sizeof(double4_32a));
        c->xb = (double4_32a *)A(Mp * sizeof(double4_32a));
    }
    c->cellid = (int *)A(Mp * sizeof(int));
    c->rank = (int *)A(Mp * sizeof(int));
    c->ccount = (int *)A((size_t)c->ncell_md * sizeof(int));
    c->cstart = (int *)A(((size_t)c->ncell_md + 1) * sizeof(int));
    c->clist = (int *)A(Mp * sizeof(int));
    c->ctmp = (int *)A(Mp * sizeof(int));
    const size_t nbs = (size_t)std::max(c->ncell_md, c->ncell_db) / 1024 + 2;
    c->bsum = (int *)A(nbs * sizeof(int));
    c->nl = (unsigned *)A((size_t)c->maxnb * Mp * sizeof(unsigned));
    c->nn = (int *)A(Mp * sizeof(int));
    c->dbcell = (int *)A(Mp * sizeof(int));
    c->dbrank = (int *)A(Mp * sizeof(int));
    c->dbcount = (int *)A((size_t)c->ncell_db * sizeof(int));
    c->dbstart = (int *)A(((size_t)c->ncell_db + 1) * sizeof(int));
    c->dblist = (int *)A(Mp * sizeof(int));
    c->dbrec = (float4 *)A(Mp * sizeof(float4));
    c->dbmark = (int *)A((size_t)c->ncell_db * sizeof(int));
    c->n_chain_total = (int)nchain;
    c->chain_ver = (int *)A((size_t)nchain * sizeof(int));
    c->dbround = (int *)A(kg::RS * kg::MAX_MELTS * sizeof(int));
    c->koff = (int *)A((kg::MAX_MELTS + 1) * sizeof(int));
    c->slot_of = (int *)A(Mp * sizeof(int));
    c->comp_of = (int *)A(Mp * sizeof(int));
    c->bp = (int4 *)A(Mp * sizeof(int4));
    c->img = (int *)A(3 * Mp * sizeof(int));
    c->db_stats = (long long *)A(4 * kg::MAX_MELTS * sizeof(long long));
    c->scratch = (double *)A(7 * Mp * sizeof(double));
    c->flags = (unsigned *)A(16 * sizeof(unsigned));
    c->pbar = (unsigned *)A(4 * sizeof(unsigned));
    c->d_step = (long long *)A(sizeof(long long));
    c->fout = (double *)A(3 * Mp * sizeof(double));
    c->partials_cap = (int)(Mp / 128 + 2) * 5;
    c->partials = (double *)A((size_t)c->partials_cap * sizeof(double));
    long long r2cap = 0;
    for (int m = 0; m < p->n_melts; ++m) r2cap = std::max(r2cap, (long long)S.melt[m].M);
    c->r2tmp_cap = r2cap;
    c->r2tmp = (double *)A((size_t)r2cap * sizeof(double));
    if (!ok) return fail(KG_ERR_OOM);
    if (cudaMemcpyAsync(c->d_sim, &c->sim, sizeof(SimDev), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return fail(KG_ERR_CUDA);
    {   // image shift of each stencil code q: (q % 3 - 1, q / 3 % 3 - 1, q / 9 - 1) * h, as the build uses it
        std::vector<float4> sh((size_t)kg::SHIFT_SLOTS * kg::MAX_MELTS, make_float4(0.f, 0.f, 0.f, 0.f));
        for (int m = 0; m < p->n_melts; ++m)
            for (int q = 0; q < 27; ++q) {
                const float h = S.melt[m].hf;
                sh[(size_t)kg::SHIFT_SLOTS * m + q] =
                    make_float4((float)(q % 3 - 1) * h, (float)((q / 3) % 3 - 1) * h, (float)(q / 9 - 1) * h, 0.f);
            }
        if (cudaMemcpyAsync(c->shtab, sh.data(), sh.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
            return fail(KG_ERR_CUDA);
    }
    const int nb = (int)((Mp + 255) / 256);
    k_iota<<<nb, 256, 0, c->stream>>>(c->slot_of, (int)Mp, 0);
    k_iota<<<nb, 256, 0, c->stream>>>(c->comp_of, (int)Mp, 0);
    kg::bonded_partners(c);
    kg_stage def{12.0, -1.0, -1, 0.01};
    if (upload_stage(c, def) != KG_OK) return fail(KG_ERR_CUDA);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(KG_ERR_CUDA);
    if (!pinned_flags()) return fail(KG_ERR_OOM);
    c->latched = KG_ERR_STATE;
    *out = c;
    return KG_OK;
}

void kg_destroy(kg_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *bufs[] = {c->d_sim, c->d_stage, c->x, c->xb64, c->u, c->pid, c->recb, c->recs, c->shtab, c->dlt[0], c->dlt[1],
                    c->pg[0], c->pg[1], c->pos64[0],
                    c->pos64[1], c->xb, c->cellid, c->rank, c->ccount, c->cstart, c->clist, c->ctmp, c->bsum, c->nl,
                    c->nn, c->dbcell, c->dbrank, c->dbcount, c->dbstart, c->dblist, c->dbrec, c->dbmark, c->chain_ver, c->dbround, c->att_ver, c->att,
                    c->koff, c->slot_of,
                    c->comp_of, c->bp, c->img, c->db_stats, c->scratch, c->flags, c->fout, c->partials,
                    c->r2tmp, c->hist, c->mlp_master, c->mlp_adam, c->mlp_grad, c->mlp_blob, c->mlp_w2t,
                    c->logf, c->logt, c->logn, c->trainf, c->traint, c->d_train_head, c->tr_buf, c->bmax2,
                    c->d_io, c->msd_ref};
    for (void *b : bufs) dev_free(c, b);
    dev_free(c, c->d_step);
    dev_free(c, c->pbar);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    kg::graphs_reset(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static kg_status check_melt(kg_ctx *c, int melt)
{
    if (!c || melt < 0 || melt >= c->sim.n_melts) return KG_ERR_INVALID_ARG;
    return cudaSetDevice(c->device) == cudaSuccess ? KG_OK : KG_ERR_CUDA;
}

kg_status kg_load_config(kg_ctx *c, int melt, const double *x, const double *v, const int *pid)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (!x) return KG_ERR_INVALID_ARG;
    const MeltDev &md = c->sim.melt[melt];
    const size_t Mm = md.M, Mp = c->Mp;
    for (int d = 0; d < 3; ++d)
        KG_TRY(cudaMemcpyAsync(c->x + d * Mp + md.off, x + d * Mm, Mm * sizeof(double), cudaMemcpyDefault, c->stream));
    if (c->precision == KG_MIXED) {   // build position = the loaded one, no displacement since
        for (int d = 0; d < 3; ++d)
            KG_TRY(cudaMemcpyAsync(c->xb64 + d * Mp + md.off, c->x + d * Mp + md.off, Mm * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->stream));
        KG_TRY(cudaMemsetAsync(c->dlt[c->cur] + md.off, 0, Mm * sizeof(float4), c->stream));
    }
    for (int d = 0; d < 3; ++d) {
        if (c->precision == KG_MIXED) {
            float *u = (float *)c->u + d * Mp + md.off;
            if (v) {
                KG_TRY(cudaMemcpyAsync(c->scratch, v + d * Mm, Mm * sizeof(double), cudaMemcpyDefault, c->stream));
                k_d2f<<<(int)((Mm + 255) / 256), 256, 0, c->stream>>>(c->scratch, u, (int)Mm);
            } else {
                KG_TRY(cudaMemsetAsync(u, 0, Mm * sizeof(float), c->stream));
            }
        } else {
            double *u = (double *)c->u + d * Mp + md.off;
            if (v) KG_TRY(cudaMemcpyAsync(u, v + d * Mm, Mm * sizeof(double), cudaMemcpyDefault, c->stream));
            else KG_TRY(cudaMemsetAsync(u, 0, Mm * sizeof(double), c->stream));
        }
    }
    if (pid) KG_TRY(cudaMemcpyAsync(c->pid + md.off, pid, Mm * sizeof(int), cudaMemcpyDefault, c->stream));
    else k_iota<<<(int)((Mm + 255) / 256), 256, 0, c->stream>>>(c->pid + md.off, (int)Mm, 0);
    // the melt's monomers start in slot order: compute index = slot
    k_iota<<<(int)((Mm + 255) / 256), 256, 0, c->stream>>>(c->slot_of + md.off, (int)Mm, md.off);
    k_iota<<<(int)((Mm + 255) / 256), 256, 0, c->stream>>>(c->comp_of + md.off, (int)Mm, md.off);
    kg::bonded_partners(c);
    c->clist_valid = false;
    c->sort_after_load = true;           // a loaded melt starts in chain order
    {   // keep the count of graph-side rebuild kernels across the reset of the status words
        unsigned f[8];
        KG_TRY(cudaMemcpyAsync(f, c->flags, sizeof(f), cudaMemcpyDeviceToHost, c->stream));
        KG_TRY(cudaStreamSynchronize(c->stream));
        c->launches += 6LL * (long long)f[6];
    }
    KG_TRY(cudaMemsetAsync(c->flags, 0, 16 * sizeof(unsigned), c->stream));
    // a rebuild cut short by an earlier error may have left cell counts behind
    KG_TRY(cudaMemsetAsync(c->ccount, 0, sizeof(int) * (size_t)c->ncell_md, c->stream));
    if ((s = set_rebuild(c)) != KG_OK) return s;
    KG_TRY(cudaStreamSynchronize(c->stream));
    c->latched = KG_OK;
    return KG_OK;
}

kg_status kg_get_config(kg_ctx *c, int melt, double *x, double *v, int *pid)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    const MeltDev &md = c->sim.melt[melt];
    const size_t Mm = md.M;
    if (x) {
        kg::to_slots(c, melt, c->x, c->scratch, 3);
        KG_TRY(cudaMemcpyAsync(x, c->scratch, 3 * Mm * sizeof(double), cudaMemcpyDefault, c->stream));
    }
    if (v) {
        kg::u_to_slots(c, melt, c->scratch + 3 * Mm);
        KG_TRY(cudaMemcpyAsync(v, c->scratch + 3 * Mm, 3 * Mm * sizeof(double), cudaMemcpyDefault, c->stream));
    }
    if (pid) {
        int *tmp = (int *)(c->scratch + 6 * Mm);
        kg::pid_to_slots(c, melt, tmp);
        KG_TRY(cudaMemcpyAsync(pid, tmp, Mm * sizeof(int), cudaMemcpyDefault, c->stream));
    }
    KG_TRY(cudaStreamSynchronize(c->stream));
    return KG_OK;
}

kg_status kg_set_potential_schedule(kg_ctx *c, const kg_stage *stages, int n_stages)
{
    if (!c || !stages || n_stages < 1) return KG_ERR_INVALID_ARG;
    for (int i = 0; i < n_stages; ++i)
        if (!(stages[i].dt > 0) || stages[i].n_exp == 6.0 || !(stages[i].n_exp > 0))
            return KG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    c->schedule.assign(stages, stages + n_stages);
    c->stage_idx = 0;
    c->stage_left = c->schedule[0].n_steps;
    return upload_stage(c, c->schedule[0]);
}

kg_status kg_step(kg_ctx *c, long long n_steps)
{
    if (!c || n_steps < 0) return KG_ERR_INVALID_ARG;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    while (n_steps > 0) {
        // advance past exhausted stages
        while (c->stage_left == 0 && c->stage_idx + 1 < c->schedule.size()) {
            ++c->stage_idx;
            c->stage_left = c->schedule[c->stage_idx].n_steps;
            kg_status s = upload_stage(c, c->schedule[c->stage_idx]);
            if (s != KG_OK) return s;
        }
        long long chunk = n_steps;
        if (c->stage_left > 0) chunk = std::min(chunk, c->stage_left);
        if (c->d_step_stale) {                  // the device counter holds the last step run
            kg::set_device_step(c, c->step - 1);
            c->d_step_stale = false;
        }
        long long done = 0;
        while (done < chunk) {
            if ((c->since_sort >= c->sort_interval || c->sort_after_load) && c->clist_valid) {
                kg::md_sort(c);                 // restore cell order for locality
                c->since_sort = 0;
                c->clist_valid = false;
                c->sort_after_load = false;
            }
            long long n = 1;
            if (c->sort_after_load)             // after a load: one step builds the cell order to sort into
                kg::md_step(c);
            else if (!c->prof_on && (c->p.flags & KG_FLAG_PERSISTENT) && c->precision == KG_MIXED &&
                chunk - done >= kg::PERSIST_STEPS && kg::md_persist_steps(c))
                n = kg::PERSIST_STEPS;
            else if (!c->prof_on && c->use_graphs && chunk - done >= kg::GRAPH_STEPS && kg::md_graph_steps(c, 1))
                n = kg::GRAPH_STEPS;
            else
                kg::md_step(c);
            c->clist_valid = true;              // a Verlet build has run since the last load / sort
            c->step += n;
            c->since_sort += n;
            done += n;
        }
        c->t_since_sweep += chunk * c->stage.dt;
        if (c->stage_left > 0) c->stage_left -= chunk;
        n_steps -= chunk;
    }
    kg::md_materialize(c);                      // current binary64 positions for every other call
    KG_TRY(cudaGetLastError());
    unsigned *h = pinned_flags();
    return read_flags(c, h);
}

kg_status kg_persistent_selftest(kg_ctx *c, int skip_block, unsigned spin)
{
    if (!c || c->precision != KG_MIXED || spin < 1) return KG_ERR_INVALID_ARG;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    if (c->d_step_stale) {
        kg::set_device_step(c, c->step - 1);
        c->d_step_stale = false;
    }
    KG_TRY(kg::persist_launch(c, c->stream, c->cur, 2, skip_block, spin));
    c->step += 2;
    kg::md_materialize(c);
    return read_flags(c, pinned_flags());
}

static kg_status sweep_impl(kg_ctx *c, const long long *attempts, kg_db_stats *stats, bool learned, double lambda)
{
    if (!c || !attempts) return KG_ERR_INVALID_ARG;
    if (learned && !(lambda > 0.0 && lambda <= 1.0)) return KG_ERR_INVALID_ARG;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    const int nm = c->sim.n_melts;
    std::vector<long long> K(attempts, attempts + nm);
    long long tot = 0;
    for (long long k : K) {
        if (k < 0 || k >= (1LL << 31)) return KG_ERR_INVALID_ARG;
        tot += k;
    }
    if (tot >= (1LL << 31)) return KG_ERR_INVALID_ARG;
    if (tot > c->att_cap) {
        dev_free(c, c->att);
        dev_free(c, c->att_ver);
        c->att_cap = std::max(tot, 2 * c->att_cap);
        c->att = dev_alloc(c, (size_t)c->att_cap * sizeof(kg::Attempt));
        c->att_ver = (int *)dev_alloc(c, (size_t)c->att_cap * sizeof(int));
        if (!c->att || !c->att_ver) {
            dev_free(c, c->att);
            dev_free(c, c->att_ver);
            c->att = nullptr;
            c->att_ver = nullptr;
            c->att_cap = 0;
            return KG_ERR_OOM;
        }
    }
    if (learned && !kg::mlp_ensure(c)) return KG_ERR_OOM;
    static thread_local long long *hstats = nullptr;
    if (!hstats && cudaMallocHost(&hstats, sizeof(long long) * 4 * kg::MAX_MELTS) != cudaSuccess) return KG_ERR_OOM;
    // the grid and the record buffers must describe the current positions
    if (learned) kg::db_sweep_learned(c, K, lambda, hstats);
    else kg::db_sweep(c, K, hstats);
    KG_TRY(cudaGetLastError());
    kg_status s = read_flags(c, pinned_flags());
    kg_db_stats out{0, 0, 0, 0, c->sweep};
    for (int m = 0; m < nm; ++m) {
        out.attempted += hstats[4 * m];
        out.empty += hstats[4 * m + 1];
        out.accepted += hstats[4 * m + 2];
        out.reevaluated += hstats[4 * m + 3];
    }
    ++c->sweep;
    c->t_since_sweep = 0.0;
    if (stats) *stats = out;
    return s;
}

static std::vector<long long> paper_attempts(kg_ctx *c, double a)
{
    const int nm = c->sim.n_melts;
    std::vector<long long> K(nm);
    for (int m = 0; m < nm; ++m) {
        const double want = (a >= 0 ? a : c->p.r_mc * c->t_since_sweep) * c->sim.melt[m].M + c->carry[m];
        K[m] = (long long)std::floor(want);
        c->carry[m] = want - (double)K[m];
    }
    return K;
}

kg_status kg_db_sweep_k(kg_ctx *c, const long long *attempts, kg_db_stats *stats)
{
    return sweep_impl(c, attempts, stats, false, 1.0);
}

kg_status kg_db_sweep(kg_ctx *c, double a, kg_db_stats *stats)
{
    if (!c) return KG_ERR_INVALID_ARG;
    const std::vector<long long> K = paper_attempts(c, a);
    return kg_db_sweep_k(c, K.data(), stats);
}

kg_status kg_db_sweep_learned_k(kg_ctx *c, const long long *attempts, double lambda, kg_db_stats *stats)
{
    return sweep_impl(c, attempts, stats, true, lambda);
}

kg_status kg_db_sweep_learned(kg_ctx *c, double a, double lambda, kg_db_stats *stats)
{
    if (!c) return KG_ERR_INVALID_ARG;
    if (!(lambda > 0.0 && lambda <= 1.0)) return KG_ERR_INVALID_ARG;
    const std::vector<long long> K = paper_attempts(c, a);
    return kg_db_sweep_learned_k(c, K.data(), lambda, stats);
}

// ---- learned proposal: weights, log, training ----

static double *io_buffer(kg_ctx *c, long long n)
{
    if (n <= c->d_io_cap) return c->d_io;
    dev_free(c, c->d_io);
    c->d_io_cap = std::max(n, 2 * c->d_io_cap);
    c->d_io = (double *)dev_alloc(c, sizeof(double) * (size_t)c->d_io_cap);
    if (!c->d_io) c->d_io_cap = 0;
    return c->d_io;
}

static kg_status mlp_begin(kg_ctx *c)
{
    if (!c) return KG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    return kg::mlp_ensure(c) ? KG_OK : KG_ERR_OOM;
}

kg_status kg_mlp_set_weights(kg_ctx *c, const double *w)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (!w) return KG_ERR_INVALID_ARG;
    for (int i = 0; i < KG_MLP_NPARAM; ++i)
        if (!std::isfinite(w[i])) return KG_ERR_INVALID_ARG;
    double *d = io_buffer(c, KG_MLP_NPARAM);
    if (!d) return KG_ERR_OOM;
    KG_TRY(cudaMemcpyAsync(d, w, sizeof(double) * KG_MLP_NPARAM, cudaMemcpyHostToDevice, c->stream));
    kg::mlp_set(c, d);
    KG_TRY(cudaGetLastError());
    return cuda_status(cudaStreamSynchronize(c->stream));
}

kg_status kg_mlp_get_weights(kg_ctx *c, double *w)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (!w) return KG_ERR_INVALID_ARG;
    double *d = io_buffer(c, KG_MLP_NPARAM);
    if (!d) return KG_ERR_OOM;
    kg::mlp_get(c, d);
    KG_TRY(cudaMemcpyAsync(w, d, sizeof(double) * KG_MLP_NPARAM, cudaMemcpyDeviceToHost, c->stream));
    return cuda_status(cudaStreamSynchronize(c->stream));
}

kg_status kg_mlp_forward(kg_ctx *c, const double *features, long long n, double *logits)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (n < 0 || (n > 0 && (!features || !logits)) || n > (1LL << 30)) return KG_ERR_INVALID_ARG;
    if (n == 0) return KG_OK;
    double *d = io_buffer(c, 25 * n);
    if (!d) return KG_ERR_OOM;
    KG_TRY(cudaMemcpyAsync(d, features, sizeof(double) * 24 * n, cudaMemcpyHostToDevice, c->stream));
    kg::mlp_infer(c, d, n, d + 24 * n);
    KG_TRY(cudaGetLastError());
    KG_TRY(cudaMemcpyAsync(logits, d + 24 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    return cuda_status(cudaStreamSynchronize(c->stream));
}

kg_status kg_mlp_loss_grad(kg_ctx *c, const double *features, const double *targets, long long n, double *loss,
                           double *grad)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (n <= 0 || n > (1LL << 24) || !features || !targets) return KG_ERR_INVALID_ARG;
    double *d = io_buffer(c, 25 * n + KG_MLP_NPARAM + 1);
    if (!d) return KG_ERR_OOM;
    KG_TRY(cudaMemcpyAsync(d, features, sizeof(double) * 24 * n, cudaMemcpyHostToDevice, c->stream));
    KG_TRY(cudaMemcpyAsync(d + 24 * n, targets, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    double *out = d + 25 * n;
    if (!kg::mlp_grad(c, d, d + 24 * n, n, out)) return KG_ERR_OOM;
    KG_TRY(cudaGetLastError());
    std::vector<double> h(KG_MLP_NPARAM + 1);
    KG_TRY(cudaMemcpyAsync(h.data(), out, sizeof(double) * (KG_MLP_NPARAM + 1), cudaMemcpyDeviceToHost, c->stream));
    KG_TRY(cudaStreamSynchronize(c->stream));
    if (loss) *loss = h[0];
    if (grad) std::copy(h.begin() + 1, h.end(), grad);
    return KG_OK;
}

kg_status kg_mlp_log(kg_ctx *c, long long capacity)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (capacity < 0 || capacity > (1LL << 32)) return KG_ERR_INVALID_ARG;
    KG_TRY(cudaStreamSynchronize(c->stream));
    dev_free(c, c->trainf);
    dev_free(c, c->traint);
    dev_free(c, c->d_train_head);
    c->trainf = c->traint = nullptr;
    c->d_train_head = nullptr;
    c->train_cap = 0;
    if (capacity == 0) return KG_OK;
    c->trainf = (double *)dev_alloc(c, sizeof(double) * 24 * (size_t)capacity);
    c->traint = (double *)dev_alloc(c, sizeof(double) * (size_t)capacity);
    c->d_train_head = (long long *)dev_alloc(c, sizeof(long long));
    if (!c->trainf || !c->traint || !c->d_train_head) {
        dev_free(c, c->trainf);
        dev_free(c, c->traint);
        dev_free(c, c->d_train_head);
        c->trainf = c->traint = nullptr;
        c->d_train_head = nullptr;
        return KG_ERR_OOM;
    }
    c->train_cap = capacity;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

static kg_status train_rows(kg_ctx *c, long long *head)
{
    *head = 0;
    if (c->train_cap <= 0) return KG_OK;
    KG_TRY(cudaMemcpyAsync(head, c->d_train_head, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    return cuda_status(cudaStreamSynchronize(c->stream));
}

kg_status kg_mlp_log_read(kg_ctx *c, double *features, double *targets, long long cap, long long *n)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (cap < 0 || !n || (cap > 0 && (!features || !targets))) return KG_ERR_INVALID_ARG;
    long long head = 0;
    if ((s = train_rows(c, &head)) != KG_OK) return s;
    const long long avail = std::min(head, c->train_cap), take = std::min(avail, cap);
    const long long first = head - avail;
    for (long long done = 0; done < take;) {            // at most two contiguous pieces of the ring
        const long long r = (first + done) % c->train_cap;
        const long long len = std::min(take - done, c->train_cap - r);
        KG_TRY(cudaMemcpyAsync(features + 24 * done, c->trainf + 24 * r, sizeof(double) * 24 * len,
                               cudaMemcpyDeviceToHost, c->stream));
        KG_TRY(cudaMemcpyAsync(targets + done, c->traint + r, sizeof(double) * len, cudaMemcpyDeviceToHost,
                               c->stream));
        done += len;
    }
    KG_TRY(cudaStreamSynchronize(c->stream));
    *n = take;
    return KG_OK;
}

kg_status kg_mlp_train(kg_ctx *c, int iters, int batch, double lr, double *loss)
{
    kg_status s = mlp_begin(c);
    if (s != KG_OK) return s;
    if (iters < 0 || batch < 1 || batch > (1 << 20) || !(lr >= 0.0) || !std::isfinite(lr)) return KG_ERR_INVALID_ARG;
    long long head = 0;
    if ((s = train_rows(c, &head)) != KG_OK) return s;
    if (head <= 0) return KG_ERR_STATE;
    double *d = io_buffer(c, 1);
    if (!d) return KG_ERR_OOM;
    if (!kg::mlp_train(c, iters, batch, lr, d)) return KG_ERR_OOM;
    KG_TRY(cudaGetLastError());
    double h = 0.0;
    KG_TRY(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    KG_TRY(cudaStreamSynchronize(c->stream));
    if (loss) *loss = h;
    return KG_OK;
}

kg_status kg_db_proposal(kg_ctx *c, int melt, int chain, int bond, double lambda, int *n, int *kind,
                         int *partner_chain, int *partner_bond, double *features, double *logits, double *prob)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    const MeltDev &md = c->sim.melt[melt];
    if (chain < 0 || chain >= md.n_ch || bond < 0 || bond > md.N - 2 || !(lambda > 0.0 && lambda <= 1.0) || !n ||
        !kind || !partner_chain || !partner_bond || !features || !logits || !prob)
        return KG_ERR_INVALID_ARG;
    if (!kg::mlp_ensure(c)) return KG_ERR_OOM;
    std::vector<int> ints(3 * KG_DB_CAND_MAX);
    if (!kg::db_proposal(c, melt, chain, bond, lambda, n, ints.data(), features, logits, prob)) return KG_ERR_CUDA;
    if ((s = read_flags(c, pinned_flags())) != KG_OK) return s;
    for (int j = 0; j < *n; ++j) {
        kind[j] = ints[j];
        partner_chain[j] = ints[KG_DB_CAND_MAX + j];
        partner_bond[j] = ints[2 * KG_DB_CAND_MAX + j];
    }
    return KG_OK;
}

kg_status kg_sync(kg_ctx *c)
{
    if (!c) return KG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    kg_status s = read_flags(c, pinned_flags());
    if (s == KG_OK && c->latched != KG_OK) return KG_ERR_STATE;
    return s;
}

kg_status kg_get_counters(kg_ctx *c, long long *step, long long *sweep)
{
    if (!c) return KG_ERR_INVALID_ARG;
    if (step) *step = c->step;
    if (sweep) *sweep = c->sweep;
    return KG_OK;
}

kg_status kg_set_counters(kg_ctx *c, long long step, long long sweep)
{
    if (!c || step < 0 || sweep < 0) return KG_ERR_INVALID_ARG;
    c->step = step;
    c->sweep = sweep;
    c->d_step_stale = true;
    return KG_OK;
}

kg_status kg_forces(kg_ctx *c, int melt, double *F, double *e4)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    kg::rebuild_md(c);
    const int nb = kg::forces_blocks(c, melt);
    kg::forces_eval(c, melt, c->step, c->fout, c->partials, nb);
    const MeltDev &md = c->sim.melt[melt];
    const size_t Mm = md.M, Mp = c->Mp;
    if (F) {
        kg::to_slots(c, melt, c->fout, c->scratch, 3);
        KG_TRY(cudaMemcpyAsync(F, c->scratch, 3 * Mm * sizeof(double), cudaMemcpyDefault, c->stream));
    }
    std::vector<double> part((size_t)nb * 5);
    KG_TRY(cudaMemcpyAsync(part.data(), c->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((s = read_flags(c, pinned_flags())) != KG_OK) return s;
    if (e4) {
        for (int k = 0; k < 4; ++k) e4[k] = 0;
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 4; ++k) e4[k] += part[(size_t)b * 5 + k];
    }
    return KG_OK;
}

// Eq. 14: sum over n of [<R^2(n)>/(n l0) - l_K (1 - l_K/(2 n l0) (1 - exp(-2 n l0/l_K)))]^2
static double lk_objective(const double *r2n, double l0, int lo, int hi, double lk)
{
    double s = 0.0;
    for (int n = lo; n <= hi; ++n) {
        const double a = 2.0 * n * l0 / lk;
        const double w = lk * (1.0 - (1.0 - std::exp(-a)) / a);
        const double y = r2n[n] / (n * l0);
        s += (y - w) * (y - w);
    }
    return s;
}

kg_status kg_fit_lk(const double *r2n, int N, double l0, int n_lo, int n_hi, double *lk)
{
    if (!r2n || !lk || N < 3 || !(l0 > 0.0)) return KG_ERR_INVALID_ARG;
    int lo = n_lo > 0 ? n_lo : N / 4, hi = n_hi > 0 ? n_hi : N / 2;
    lo = std::max(lo, 1);
    if (hi >= N || lo > hi) return KG_ERR_INVALID_ARG;
    for (int n = lo; n <= hi; ++n)
        if (!std::isfinite(r2n[n])) return KG_ERR_INVALID_ARG;
    // bracket the minimum on a logarithmic grid, then golden-section search in log l_K
    const double a0 = std::log(1e-3 * l0), a1 = std::log(1e3 * l0 * hi);
    const int G = 400;
    int best = 0;
    double fbest = 1e300;
    for (int g = 0; g <= G; ++g) {
        const double f = lk_objective(r2n, l0, lo, hi, std::exp(a0 + (a1 - a0) * g / G));
        if (f < fbest) { fbest = f; best = g; }
    }
    double a = a0 + (a1 - a0) * std::max(best - 1, 0) / G, b = a0 + (a1 - a0) * std::min(best + 1, G) / G;
    const double r = 0.5 * (std::sqrt(5.0) - 1.0);
    double c = b - r * (b - a), d = a + r * (b - a);
    double fc = lk_objective(r2n, l0, lo, hi, std::exp(c)), fd = lk_objective(r2n, l0, lo, hi, std::exp(d));
    for (int it = 0; it < 200 && b - a > 1e-14; ++it) {
        if (fc < fd) { b = d; d = c; fd = fc; c = b - r * (b - a); fc = lk_objective(r2n, l0, lo, hi, std::exp(c)); }
        else { a = c; c = d; fc = fd; d = a + r * (b - a); fd = lk_objective(r2n, l0, lo, hi, std::exp(d)); }
    }
    *lk = std::exp(0.5 * (a + b));
    return KG_OK;
}

// Philox4x32-10 (Salmon et al., SC'11) on the host, for the initial-state generator
static void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0; c[1] = (uint32_t)p1; c[2] = n2; c[3] = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

kg_status kg_generate_fr(int n_chains, int chain_len, double box, double kappa, double l0, unsigned long long seed,
                         int max_attempts, double *x, double *lk_fit, int *attempts)
{
    if (n_chains < 1 || chain_len < 8 || !(box > 0.0) || !(kappa >= 0.0) || !(l0 > 0.0) || max_attempts < 1 || !x)
        return KG_ERR_INVALID_ARG;
    const int N = chain_len;
    const size_t M = (size_t)n_chains * N;
    const double r = lk_over_l0(kappa), cos_t = (r - 1.0) / (r + 1.0), sin_t = std::sqrt(1.0 - cos_t * cos_t);
    const double U32 = 2.3283064365386963e-10, TWO_PI = 6.283185307179586;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int lo = std::max(N / 4, 1), hi = N / 2;
    std::vector<double> r2n(N, 0.0);
    for (int a = 0; a < max_attempts; ++a) {
        for (int ch = 0; ch < n_chains; ++ch) {
            double p[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 1.0};
            for (int i = 0; i < N; ++i) {
                uint32_t w[4] = {(uint32_t)i, (uint32_t)ch, (uint32_t)a, 5u};
                philox_host(w, k0, k1);
                auto u = [&](int q) { return ((double)w[q] + 0.5) * U32; };
                if (i == 0) {
                    p[0] = box * u(0); p[1] = box * u(1); p[2] = box * u(2);
                } else {
                    double nb[3];
                    if (i == 1) {                     // first bond uniform on the sphere
                        const double ct = 2.0 * u(0) - 1.0, st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
                        const double ph = TWO_PI * u(1);
                        nb[0] = st * std::cos(ph); nb[1] = st * std::sin(ph); nb[2] = ct;
                    } else {                          // angle theta* to the previous bond, uniform azimuth
                        const double ph = TWO_PI * u(0);
                        const double ax = std::fabs(b[2]) < 0.9 ? 0.0 : 1.0, az = std::fabs(b[2]) < 0.9 ? 1.0 : 0.0;
                        const double cx = b[1] * az - b[2] * 0.0, cy = b[2] * ax - b[0] * az, cz = b[0] * 0.0 - b[1] * ax;
                        const double cn = std::sqrt((cx * cx + cy * cy) + cz * cz);
                        const double e1[3] = {cx / cn, cy / cn, cz / cn};
                        const double e2[3] = {b[1] * e1[2] - b[2] * e1[1], b[2] * e1[0] - b[0] * e1[2],
                                              b[0] * e1[1] - b[1] * e1[0]};
                        const double cp = std::cos(ph), sp = std::sin(ph);
                        for (int k = 0; k < 3; ++k) nb[k] = cos_t * b[k] + sin_t * (cp * e1[k] + sp * e2[k]);
                    }
                    const double n = std::sqrt((nb[0] * nb[0] + nb[1] * nb[1]) + nb[2] * nb[2]);
                    for (int k = 0; k < 3; ++k) {
                        b[k] = nb[k] / n;
                        p[k] = p[k] + l0 * b[k];
                    }
                }
                for (int k = 0; k < 3; ++k) x[k * M + (size_t)ch * N + i] = p[k];
            }
        }
        for (int n = lo; n <= hi; ++n) {              // <R^2(n)> over the fit range
            double s = 0.0;
            for (int ch = 0; ch < n_chains; ++ch)
                for (int i = 0; i + n < N; ++i) {
                    const size_t j = (size_t)ch * N + i;
                    const double dx = x[j + n] - x[j], dy = x[M + j + n] - x[M + j], dz = x[2 * M + j + n] - x[2 * M + j];
                    s += (dx * dx + dy * dy) + dz * dz;
                }
            r2n[n] = s / ((double)n_chains * (N - n));
        }
        double lk = 0.0;
        const kg_status st = kg_fit_lk(r2n.data(), N, l0, lo, hi, &lk);
        if (st != KG_OK) return st;
        if (std::fabs(lk / (r * l0) - 1.0) <= 0.02) {
            if (lk_fit) *lk_fit = lk;
            if (attempts) *attempts = a + 1;
            return KG_OK;
        }
    }
    return KG_ERR_CAPACITY;
}

kg_status kg_structure_factor(kg_ctx *c, int melt, const int *hkl, int nq, double *S)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if (!hkl || !S || nq < 1 || nq > 65535) return KG_ERR_INVALID_ARG;
    int *d_hkl = (int *)dev_alloc(c, sizeof(int) * 3 * (size_t)nq);
    double *d_part = (double *)dev_alloc(c, sizeof(double) * 2 * 64 * (size_t)nq);
    double *d_S = (double *)dev_alloc(c, sizeof(double) * (size_t)nq);
    auto done = [&](kg_status r) { dev_free(c, d_hkl); dev_free(c, d_part); dev_free(c, d_S); return r; };
    if (!d_hkl || !d_part || !d_S) return done(KG_ERR_OOM);
    if (cudaMemcpyAsync(d_hkl, hkl, sizeof(int) * 3 * (size_t)nq, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return done(KG_ERR_CUDA);
    kg::sq_eval(c, melt, d_hkl, nq, d_part, d_S);
    if (cudaMemcpyAsync(S, d_S, sizeof(double) * (size_t)nq, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return done(KG_ERR_CUDA);
    return done(read_flags(c, pinned_flags()));
}

kg_status kg_pair_distribution(kg_ctx *c, int melt, double r_max, int nbins, double *g)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    const MeltDev &md = c->sim.melt[melt];
    if (!g || nbins < 1 || nbins > kg::GR_BINS_MAX || !(r_max > 0.0) || r_max > 0.5 * md.L)
        return KG_ERR_INVALID_ARG;
    unsigned long long *d_h = (unsigned long long *)dev_alloc(c, sizeof(unsigned long long) * nbins);
    if (!d_h) return KG_ERR_OOM;
    std::vector<long long> K(c->sim.n_melts, 0);
    kg::db_bin(c, K);                                   // the >= 1.3 sigma grid of the current positions
    const double dr = r_max / nbins;
    const int R = (int)std::ceil(r_max * md.invhdb);
    kg::gr_eval(c, melt, R, r_max, dr, nbins, d_h);
    std::vector<unsigned long long> h(nbins);
    kg_status out = KG_OK;
    if (cudaMemcpyAsync(h.data(), d_h, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        out = KG_ERR_CUDA;
    if (out == KG_OK) out = read_flags(c, pinned_flags());
    dev_free(c, d_h);
    if (out != KG_OK) return out;
    const double M = md.M, rho = M / (md.L * md.L * md.L), pi = 3.14159265358979323846;
    for (int b = 0; b < nbins; ++b) {
        const double lo = (double)b * dr, hi = (double)(b + 1) * dr;
        g[b] = (double)h[b] / (M * rho * (4.0 / 3.0 * pi * (hi * hi * hi - lo * lo * lo)));
    }
    return KG_OK;
}

kg_status kg_msd_reset(kg_ctx *c, int melt)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    return kg::msd_reset(c, melt) ? KG_OK : KG_ERR_OOM;
}

kg_status kg_msd(kg_ctx *c, int melt, double *msd)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if (!msd || !c->msd_ref) return KG_ERR_INVALID_ARG;
    const int nb = kg::msd_blocks(c, melt);
    if (nb > c->partials_cap) return KG_ERR_CAPACITY;
    kg::msd_eval(c, melt, c->partials);
    std::vector<double> part((size_t)nb);
    KG_TRY(cudaMemcpyAsync(part.data(), c->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((s = read_flags(c, pinned_flags())) != KG_OK) return s;
    double sum = 0.0;
    for (double v : part) sum += v;                  // block order: deterministic
    *msd = sum / (double)c->sim.melt[melt].M;
    return KG_OK;
}

kg_status kg_observables(kg_ctx *c, int melt, kg_obs *out, double *r2n, double *bond_hist, double *cos_hist,
                         int n_bins)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if ((bond_hist || cos_hist) && n_bins < 1) return KG_ERR_INVALID_ARG;
    const MeltDev &md = c->sim.melt[melt];
    if (out) {
        kg::rebuild_md(c);
        const int nb = kg::forces_blocks(c, melt);
        kg::forces_eval(c, melt, c->step, nullptr, c->partials, nb);
        std::vector<double> part((size_t)nb * 5);
        KG_TRY(cudaMemcpyAsync(part.data(), c->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if ((s = read_flags(c, pinned_flags())) != KG_OK) return s;
        double e[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 5; ++k) e[k] += part[(size_t)b * 5 + k];
        const double V = md.L * md.L * md.L;
        out->e_pair = e[0]; out->e_bond = e[1]; out->e_angle = e[2]; out->virial = e[3]; out->e_kin = e[4];
        out->temperature = 2.0 * e[4] / (3.0 * md.M);
        out->pressure = (2.0 * e[4] + e[3]) / (3.0 * V);
        out->step = c->step;
    }
    if (r2n) {
        if (md.N > KG_R2N_MAX_CHAIN_LEN) return KG_ERR_INVALID_ARG;
        if (!kg::r2n_eval(c, melt, c->scratch)) return KG_ERR_CUDA;
        KG_TRY(cudaMemcpyAsync(r2n, c->scratch, sizeof(double) * md.N, cudaMemcpyDefault, c->stream));
    }
    if (bond_hist || cos_hist) {
        if (c->hist_cap < 2 * n_bins) {
            dev_free(c, c->hist);
            c->hist = (int *)dev_alloc(c, sizeof(int) * 2 * n_bins);
            if (!c->hist) { c->hist_cap = 0; return KG_ERR_OOM; }
            c->hist_cap = 2 * n_bins;
        }
        kg::hist_eval(c, melt, n_bins, c->hist);
        std::vector<int> h(2 * (size_t)n_bins);
        KG_TRY(cudaMemcpyAsync(h.data(), c->hist, sizeof(int) * 2 * n_bins, cudaMemcpyDeviceToHost, c->stream));
        KG_TRY(cudaStreamSynchronize(c->stream));
        for (int b = 0; b < n_bins; ++b) {
            if (bond_hist) bond_hist[b] = h[b];
            if (cos_hist) cos_hist[b] = h[n_bins + b];
        }
    }
    KG_TRY(cudaStreamSynchronize(c->stream));
    return KG_OK;
}

kg_status kg_profile(kg_ctx *c, int enable)
{
    if (!c) return KG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    if (enable) {
        kg::prof_collect(c);
        c->prof_ms = 0.0;
        c->prof_n = 0;
    }
    c->prof_on = enable != 0;
    return KG_OK;
}

kg_status kg_profile_read(kg_ctx *c, double *ms, long long *n, long long *launches)
{
    if (!c) return KG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return KG_ERR_CUDA;
    kg::prof_collect(c);
    if (ms) *ms = c->prof_ms;
    if (n) *n = c->prof_n;
    if (launches) {
        // inside graphs the six rebuild kernels run only when requested; the
        // device counts those runs in flags[6]
        unsigned f[8];
        if (cudaMemcpy(f, c->flags, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return KG_ERR_CUDA;
        *launches = c->launches + 6LL * (long long)f[6];
    }
    return KG_OK;
}

// A candidate replaces the best so far only if it is faster by this
// fraction: trials of nearly equal settings then keep the earlier one (the
// smaller skin, block and cell) instead of following timing noise.
constexpr double TUNE_MARGIN = 0.005;

// One autotuner trial: a context with parameters q on the given states
// (re-sorted into cell order after its first step, as after every load),
// warmed up, then timed over two windows of trial_steps MD steps with
// periodic re-sorts off.  *ms: the better window, per MD step.
static kg_status autotune_trial(const kg_params &q0, const double *const *x, const double *const *v,
                                const kg_stage *stage, int trial_steps, int device, void *stream,
                                const kg_allocator *allocator, cudaEvent_t e0, cudaEvent_t e1, double *ms)
{
    kg_params q = q0;
    q.sort_interval = 1 << 30;
    kg_ctx *c = nullptr;
    kg_status s = kg_create(&c, &q, device, stream, allocator);
    if (s != KG_OK) return s;
    kg_stage st = *stage;
    st.n_steps = -1;                                       // open-ended stage for the trial
    for (int m = 0; s == KG_OK && m < q.n_melts; ++m) s = kg_load_config(c, m, x[m], v ? v[m] : nullptr, nullptr);
    if (s == KG_OK) s = kg_set_potential_schedule(c, &st, 1);
    if (s == KG_OK) s = kg_step(c, trial_steps);          // warm-up: re-sort after the first build, graphs
    float best = 1e30f;
    for (int rep = 0; s == KG_OK && rep < 2; ++rep) {
        float t = 0.f;
        cudaEventRecord(e0, c->stream);
        s = kg_step(c, trial_steps);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
        best = t < best ? t : best;
    }
    kg_destroy(c);
    *ms = (double)best / trial_steps;
    return s;
}

kg_status kg_autotune(const kg_params *p, const double *const *x, const double *const *v, const kg_stage *stage,
                      int trial_steps, int device, void *stream, const kg_allocator *allocator, kg_tuning *best)
{
    if (!p || !x || !stage || !best || trial_steps < kg::GRAPH_STEPS) return KG_ERR_INVALID_ARG;
    const double skins[] = {0.25, 0.3, 0.4, 0.5, 0.6};
    const int blocks[] = {64, 128, 256};
    const int tpms[] = {1, 2};
    const int ntpm = p->precision == KG_MIXED ? 2 : 1;
    best->ms_per_step = 1e300;
    best->trials = 0;
    best->cell_scale = 1.0;
    cudaEvent_t e0, e1;
    if (cudaSetDevice(device) != cudaSuccess) return KG_ERR_CUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KG_ERR_CUDA;
    kg_status out = KG_OK;
    for (double skin : skins) {
        for (int bt = 0; out == KG_OK && bt < 3 * ntpm; ++bt) {
            kg_params q = *p;
            q.skin = skin;
            q.block_size = blocks[bt % 3];
            q.threads_per_monomer = tpms[bt / 3];
            q.cell_scale = 1.0;
            double per = 0.0;
            const kg_status s = autotune_trial(q, x, v, stage, trial_steps, device, stream, allocator, e0, e1, &per);
            if (s == KG_ERR_INVALID_ARG) continue;                 // this skin does not fit the box
            if (s != KG_OK) { out = s; break; }
            ++best->trials;
            if (per < best->ms_per_step * (1.0 - TUNE_MARGIN)) {   // earlier (smaller skin) wins ties
                best->ms_per_step = per;
                best->skin = skin;
                best->block_size = q.block_size;
                best->threads_per_monomer = q.threads_per_monomer;
            }
        }
        if (out != KG_OK) break;
    }
    const double scales[] = {1.15, 1.3};
    for (int k = 0; out == KG_OK && best->trials > 0 && k < 2; ++k) {   // the cell side with the best of the rest
        kg_params q = *p;
        q.skin = best->skin;
        q.block_size = best->block_size;
        q.threads_per_monomer = best->threads_per_monomer;
        q.cell_scale = scales[k];
        double per = 0.0;
        const kg_status s = autotune_trial(q, x, v, stage, trial_steps, device, stream, allocator, e0, e1, &per);
        if (s == KG_ERR_INVALID_ARG) continue;                     // fewer than three cells per side
        if (s != KG_OK) { out = s; break; }
        ++best->trials;
        if (per < best->ms_per_step * (1.0 - TUNE_MARGIN)) {
            best->ms_per_step = per;
            best->cell_scale = scales[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out == KG_OK && best->trials == 0) out = KG_ERR_INVALID_ARG;
    return out;
}

kg_status kg_get_nlist(kg_ctx *c, int melt, int *offs, int *nbr, long long cap, long long *total)
{
    kg_status s = check_melt(c, melt);
    if (s != KG_OK) return s;
    if (c->latched != KG_OK) return KG_ERR_STATE;
    if (!offs || !nbr || cap < 0) return KG_ERR_INVALID_ARG;
    if ((s = set_rebuild(c)) != KG_OK) return s;
    kg::rebuild_md(c);
    const MeltDev &md = c->sim.melt[melt];
    const size_t Mm = md.M, Mp = c->Mp;
    std::vector<int> nn(Mm), comp(Mm), slot(Mm);
    std::vector<unsigned> nl((size_t)c->maxnb * Mm);
    KG_TRY(cudaMemcpyAsync(nn.data(), c->nn + md.off, Mm * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    KG_TRY(cudaMemcpyAsync(comp.data(), c->comp_of + md.off, Mm * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    KG_TRY(cudaMemcpyAsync(slot.data(), c->slot_of + md.off, Mm * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    for (int k = 0; k < c->maxnb; ++k)
        KG_TRY(cudaMemcpyAsync(nl.data() + (size_t)k * Mm, c->nl + (size_t)k * Mp + md.off, Mm * sizeof(unsigned),
                               cudaMemcpyDeviceToHost, c->stream));
    if ((s = read_flags(c, pinned_flags())) != KG_OK) return s;
    long long tot = 0;
    std::vector<int> row;
    for (size_t i = 0; i < Mm; ++i) {          // slot i of the melt
        offs[i] = (int)tot;
        row.clear();
        const size_t j = (size_t)(comp[i] - md.off);
        for (int k = 0; k < nn[j]; ++k) row.push_back(slot[(int)(nl[k * Mm + j] & kg::IDX_MASK) - md.off] - md.off);
        std::sort(row.begin(), row.end());
        if (tot + (long long)row.size() > cap) return KG_ERR_CAPACITY;
        std::copy(row.begin(), row.end(), nbr + tot);
        tot += (long long)row.size();
    }
    offs[Mm] = (int)tot;
    if (total) *total = tot;
    return KG_OK;
}

}  // extern "C"
