// kg_obs.cu -- observables: <R^2(n)> (the input of the l_K fit, Eq. 14) and
// bond-length / cos(theta) histograms.  Binary64 sums in a fixed order, so
// repeated calls give identical results.
#include <cuda_runtime.h>

#include "kg_host.h"

namespace kg {

// One block per chain: the chain's unwrapped positions in shared memory;
// thread t accumulates sum_i |x_{i+n} - x_i|^2 for n = t+1, t+1+blockDim, ...
// The row stride Mp is 64-bit: a caller's rows may sit 2^30 or more doubles
// apart, and every index into x is formed in 64-bit arithmetic.
__global__ void __launch_bounds__(256) k_r2n_chain(const double *__restrict__ x, long long Mp, int off, int N,
                                                  double *__restrict__ out /* [n_ch][N] */,
                                                  const int *__restrict__ comp_of /* NULL: slot order */)
{
    extern __shared__ double pos[];          // 3N
    const int c = blockIdx.x;
    const long long base = (long long)off + (long long)c * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const long long j = comp_of ? (long long)comp_of[base + i] : base + i;
        pos[i] = x[j];
        pos[N + i] = x[Mp + j];
        pos[2 * N + i] = x[2 * Mp + j];
    }
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double s = 0.0;
        if (n > 0)
            for (int i = 0; i + n < N; ++i) {
                const double dx = pos[i + n] - pos[i], dy = pos[N + i + n] - pos[N + i],
                             dz = pos[2 * N + i + n] - pos[2 * N + i];
                s += dx * dx + dy * dy + dz * dz;
            }
        out[(size_t)c * N + n] = s;
    }
}

// column sums over chains, in chain order, divided by the number of pairs
__global__ void __launch_bounds__(256) k_r2n_reduce(const double *__restrict__ in, int n_ch, int N,
                                                   double *__restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double s = 0.0;
    for (int c = 0; c < n_ch; ++c) s += in[(size_t)c * N + n];
    out[n] = n == 0 ? 0.0 : s / ((double)n_ch * (double)(N - n));
}

__global__ void __launch_bounds__(256) k_hist(const double *__restrict__ x, int Mp, int off, int M, int N,
                                             double L, double R0, int nbins, int *__restrict__ bond_h,
                                             int *__restrict__ cos_h, const int *__restrict__ comp_of)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const int s = off + r, i = r % N;
    const int j0 = comp_of[s], jm = i >= 1 ? comp_of[s - 1] : j0, jp = i + 1 < N ? comp_of[s + 1] : j0;
    double b1[3], b2[3];
    if (i + 1 < N) {
#pragma unroll
        for (int k = 0; k < 3; ++k) b2[k] = min_image_exact(x[k * Mp + jp] - x[k * Mp + j0], L);
        const double len = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
        const int b = (int)floor(len / R0 * nbins);
        if (b >= 0 && b < nbins) atomicAdd(bond_h + b, 1);
    }
    if (i >= 1 && i + 1 < N) {
#pragma unroll
        for (int k = 0; k < 3; ++k) b1[k] = min_image_exact(x[k * Mp + j0] - x[k * Mp + jm], L);
        const double cs = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
                          / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
                             * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
        int b = (int)floor((cs + 1.0) * 0.5 * nbins);
        b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        atomicAdd(cos_h + b, 1);
    }
}

// Dynamic shared memory of k_r2n_chain for chains of N monomers (3N doubles);
// above 48 KiB the kernel's opt-in limit is raised first.
bool r2n_smem_ready(int N)
{
    const size_t smem = sizeof(double) * 3 * (size_t)N;
    if (N < 1 || smem > (size_t)R2N_SMEM_MAX) return false;
    if (smem <= 48 * 1024) return true;
    return cudaFuncSetAttribute(k_r2n_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

bool r2n_eval(kg_ctx *c, int melt, double *out_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    if (!r2n_smem_ready(md.N)) return false;
    c->launches += 2;
    k_r2n_chain<<<md.n_ch, 256, sizeof(double) * 3 * md.N, c->stream>>>(c->x, (long long)c->Mp, md.off, md.N,
                                                                          c->r2tmp, c->comp_of);
    if (cudaGetLastError() != cudaSuccess) return false;
    k_r2n_reduce<<<(md.N + 255) / 256, 256, 0, c->stream>>>(c->r2tmp, md.n_ch, md.N, out_dev);
    return cudaGetLastError() == cudaSuccess;
}

void hist_eval(kg_ctx *c, int melt, int nbins, int *out_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    cudaMemsetAsync(out_dev, 0, sizeof(int) * 2 * nbins, c->stream);
    ++c->launches;
    k_hist<<<(md.M + 255) / 256, 256, 0, c->stream>>>(c->x, c->Mp, md.off, md.M, md.N, md.L, sqrt(c->stage.R0sq),
                                                      nbins, out_dev, out_dev + nbins, c->comp_of);
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// monomer mean-squared displacement (App. B): ref holds, per compute index,
// the position at the last kg_msd_reset plus every box shift a
// double-bridging swap has since added to the unwrapped position, so
// x - ref is the physical displacement
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_msd_reset(const double *__restrict__ x, double *__restrict__ ref, int Mp,
                                                  int off, int M)
{
    const int j = off + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= off + M) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) ref[(size_t)d * Mp + j] = x[(size_t)d * Mp + j];
}

// block partial sums of |x - ref|^2 in a fixed tree (deterministic)
__global__ void __launch_bounds__(256) k_msd(const double *__restrict__ x, const double *__restrict__ ref, int Mp,
                                            int off, int M, double *__restrict__ part)
{
    __shared__ double sh[256];
    const int j = off + blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (j < off + M) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = x[(size_t)d * Mp + j] - ref[(size_t)d * Mp + j];
            s += v * v;
        }
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// re-sort of the per-monomer state: ref follows its monomers (out[j] = in[order[j]])
__global__ void __launch_bounds__(256) k_msd_permute(const double *__restrict__ in, double *__restrict__ out,
                                                    const int *__restrict__ order, int Mp, int M)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int o = order[j];
#pragma unroll
    for (int d = 0; d < 3; ++d) out[(size_t)d * Mp + j] = in[(size_t)d * Mp + o];
}

static inline int nb256(long long n) { return (int)((n + 255) / 256); }

bool msd_reset(kg_ctx *c, int melt)
{
    if (!c->msd_ref) {
        c->msd_ref = (double *)dev_alloc(c, 6 * (size_t)c->Mp * sizeof(double));
        if (!c->msd_ref) return false;
    }
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    k_msd_reset<<<nb256(md.M), 256, 0, c->stream>>>(c->x, c->msd_ref, c->Mp, md.off, md.M);
    return true;
}

int msd_blocks(const kg_ctx *c, int melt) { return nb256(c->sim.melt[melt].M); }

void msd_eval(kg_ctx *c, int melt, double *part_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    k_msd<<<nb256(md.M), 256, 0, c->stream>>>(c->x, c->msd_ref, c->Mp, md.off, md.M, part_dev);
}

void msd_permute(kg_ctx *c, const int *order)
{
    if (!c->msd_ref) return;
    double *tmp = c->msd_ref + 3 * (size_t)c->Mp;
    c->launches += 1;
    k_msd_permute<<<nb256(c->M), 256, 0, c->stream>>>(c->msd_ref, tmp, order, c->Mp, c->M);
    cudaMemcpyAsync(c->msd_ref, tmp, 3 * (size_t)c->Mp * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

// ---------------------------------------------------------------------------
// static structure factor (App. A): S(q) = |sum_j exp(i q . r_j)|^2 / M for
// q = 2 pi (h, k, l) / L.  The phase is reduced to [0, 1) turns in binary64
// (so unwrapped positions of any size keep their precision) and evaluated by
// sincospif in binary32; sums are binary64, block trees then block order.
// ---------------------------------------------------------------------------
constexpr int SQ_CHUNKS = 64;

__global__ void __launch_bounds__(256) k_sq(const double *__restrict__ x, int Mp, int off, int M, double invL,
                                           const int *__restrict__ hkl, double *__restrict__ part)
{
    __shared__ double sre[256], sim[256];
    const int q = blockIdx.x;
    const double h = hkl[3 * q], k = hkl[3 * q + 1], l = hkl[3 * q + 2];
    double re = 0.0, im = 0.0;
    for (int r = blockIdx.y * blockDim.x + threadIdx.x; r < M; r += gridDim.y * blockDim.x) {
        const int j = off + r;
        const double t = (h * x[j] + k * x[(size_t)Mp + j] + l * x[2 * (size_t)Mp + j]) * invL;
        float sn, cs;
        sincospif(2.0f * (float)(t - floor(t)), &sn, &cs);
        re += cs;
        im += sn;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sre[threadIdx.x] += sre[threadIdx.x + w];
            sim[threadIdx.x] += sim[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * ((size_t)q * gridDim.y + blockIdx.y)] = sre[0];
        part[2 * ((size_t)q * gridDim.y + blockIdx.y) + 1] = sim[0];
    }
}

__global__ void __launch_bounds__(256) k_sq_sum(const double *__restrict__ part, int nq, int G, int M,
                                               double *__restrict__ S)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double re = 0.0, im = 0.0;
    for (int g = 0; g < G; ++g) {
        re += part[2 * ((size_t)q * G + g)];
        im += part[2 * ((size_t)q * G + g) + 1];
    }
    S[q] = (re * re + im * im) / (double)M;
}

void sq_eval(kg_ctx *c, int melt, const int *hkl_dev, int nq, double *part_dev, double *S_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    c->launches += 2;
    k_sq<<<dim3(nq, SQ_CHUNKS), 256, 0, c->stream>>>(c->x, c->Mp, md.off, md.M, md.invL, hkl_dev, part_dev);
    k_sq_sum<<<(nq + 255) / 256, 256, 0, c->stream>>>(part_dev, nq, SQ_CHUNKS, md.M, S_dev);
}

// ---------------------------------------------------------------------------
// pair distribution (App. A): ordered pairs i != j with minimum-image
// distance r < r_max, counted in bins of width dr, on the double-bridging cell
// grid (cells >= 1.3 sigma, stencil of +-R cells, each cell once).  The
// distance is the binary64 expression ((dx*dx + dy*dy) + dz*dz), dx = d - L
// rint(d/L), its IEEE square root and bin floor(r / dr): integer counts, so
// the histogram does not depend on the order of the additions.
// ---------------------------------------------------------------------------
constexpr int GR_MAX_BINS = 2048;

__global__ void __launch_bounds__(256) k_gr(const SimDev *__restrict__ Sp, int melt, const double *__restrict__ x,
                                           const int *__restrict__ cell, const int *__restrict__ start,
                                           const int *__restrict__ list, int R, double r_max, double dr,
                                           int nbins, unsigned long long *__restrict__ hist)
{
    __shared__ unsigned int sh[GR_MAX_BINS];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const SimDev &S = *Sp;
    const MeltDev &md = S.melt[melt];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < md.M) {
        const int i = md.off + r, n = md.ndb;
        const int c0 = cell[i] - md.dbcell_off;
        const int cx = c0 % n, cy = (c0 / n) % n, cz = c0 / (n * n);
        const int w = 2 * R + 1 < n ? 2 * R + 1 : n;         // each cell of the stencil once
        const int o = 2 * R + 1 < n ? -R : 0;
        for (int a = 0; a < w; ++a)
            for (int b = 0; b < w; ++b)
                for (int e = 0; e < w; ++e) {
                    const int zz = 2 * R + 1 < n ? ((cz + o + a) % n + n) % n : a;
                    const int yy = 2 * R + 1 < n ? ((cy + o + b) % n + n) % n : b;
                    const int xx = 2 * R + 1 < n ? ((cx + o + e) % n + n) % n : e;
                    const int cc = md.dbcell_off + (zz * n + yy) * n + xx;
                    for (int k = start[cc]; k < start[cc + 1]; ++k) {
                        const int j = list[k];
                        if (j == i) continue;
                        const double rr = sqrt(dist2_exact(x, S.Mp, md.L, i, j));
                        if (!(rr < r_max)) continue;
                        const int bin = (int)__ddiv_rn(rr, dr);
                        if (bin < nbins) atomicAdd(&sh[bin], 1u);
                    }
                }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
}

void gr_eval(kg_ctx *c, int melt, int R, double r_max, double dr, int nbins, unsigned long long *hist_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    ++c->launches;
    cudaMemsetAsync(hist_dev, 0, sizeof(unsigned long long) * nbins, c->stream);
    k_gr<<<nb256(md.M), 256, 0, c->stream>>>(c->d_sim, melt, c->x, c->dbcell, c->dbstart, c->dblist, R, r_max,
                                             dr, nbins, hist_dev);
}

// <R^2(n)> without any allocation (kg_r2n_noalloc)
// ---------------------------------------------------------------------------
// The per-chain partial sums of k_r2n_chain live in this file-scope array
// instead of a buffer the caller or the library allocates.  Every GPU that
// loads the library holds it (KG_NOALLOC_MAX_MONOMERS doubles, 16 MiB) until
// the process exits.
static __device__ __align__(256) double g_r2n_scratch[KG_NOALLOC_MAX_MONOMERS];

}  // namespace kg

namespace {

// Device address of g_r2n_scratch on the current device.  In host code the
// symbol names a host-side stand-in, not device memory, so it must never be
// handed to a kernel directly.  The address is looked up on every call (the
// lookup allocates nothing), so it stays right after the device's primary
// context has been reset and the module reloaded.
double *scratch_address(kg_status *st)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, kg::g_r2n_scratch) != cudaSuccess) {
        *st = KG_ERR_CUDA;
        return nullptr;
    }
    *st = KG_OK;
    return (double *)p;
}

}  // namespace

extern "C" kg_status kg_r2n_noalloc(const double *x, long long stride, int n_chains, int chain_len, double *out,
                                    void *stream)
{
    if (!x || !out || n_chains < 1 || chain_len < 2 || stride < (long long)n_chains * chain_len)
        return KG_ERR_INVALID_ARG;
    if ((long long)n_chains * chain_len > KG_NOALLOC_MAX_MONOMERS) return KG_ERR_INVALID_ARG;
    if (chain_len > KG_R2N_MAX_CHAIN_LEN) return KG_ERR_INVALID_ARG;
    kg_status st;
    double *scratch = scratch_address(&st);
    if (!scratch) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(double) * 3 * chain_len;
    if (!kg::r2n_smem_ready(chain_len)) return KG_ERR_CUDA;
    kg::k_r2n_chain<<<n_chains, 256, smem, s>>>(x, stride, 0, chain_len, scratch, nullptr);
    kg::k_r2n_reduce<<<(chain_len + 255) / 256, 256, 0, s>>>(scratch, n_chains, chain_len, out);
    return cudaGetLastError() == cudaSuccess ? KG_OK : KG_ERR_CUDA;
}

