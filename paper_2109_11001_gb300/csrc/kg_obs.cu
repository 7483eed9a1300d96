// kg_obs.cu -- observables: <R^2(n)> (the input of the l_K fit, Eq. 14) and
// bond-length / cos(theta) histograms.  Binary64 sums in a fixed order, so
// repeated calls give identical results.
#include <cuda_runtime.h>

#include "kg_host.h"

namespace kg {

// One block per chain: the chain's unwrapped positions in shared memory;
// thread t accumulates sum_i |x_{i+n} - x_i|^2 for n = t+1, t+1+blockDim, ...
__global__ void __launch_bounds__(256) k_r2n_chain(const double *__restrict__ x, int Mp, int off, int N,
                                                  double *__restrict__ out /* [n_ch][N] */)
{
    extern __shared__ double pos[];          // 3N
    const int c = blockIdx.x;
    const int base = off + c * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        pos[i] = x[base + i];
        pos[N + i] = x[Mp + base + i];
        pos[2 * N + i] = x[2 * Mp + base + i];
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
                                             int *__restrict__ cos_h)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const int s = off + r, i = r % N;
    double b1[3], b2[3];
    if (i + 1 < N) {
#pragma unroll
        for (int k = 0; k < 3; ++k) b2[k] = min_image_exact(x[k * Mp + s + 1] - x[k * Mp + s], L);
        const double len = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
        const int b = (int)floor(len / R0 * nbins);
        if (b >= 0 && b < nbins) atomicAdd(bond_h + b, 1);
    }
    if (i >= 1 && i + 1 < N) {
#pragma unroll
        for (int k = 0; k < 3; ++k) b1[k] = min_image_exact(x[k * Mp + s] - x[k * Mp + s - 1], L);
        const double cs = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2])
                          / (sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2])
                             * sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]));
        int b = (int)floor((cs + 1.0) * 0.5 * nbins);
        b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        atomicAdd(cos_h + b, 1);
    }
}

void r2n_eval(kg_ctx *c, int melt, double *out_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    c->launches += 2;
    k_r2n_chain<<<md.n_ch, 256, sizeof(double) * 3 * md.N, c->stream>>>(c->x, c->Mp, md.off, md.N, c->r2tmp);
    k_r2n_reduce<<<(md.N + 255) / 256, 256, 0, c->stream>>>(c->r2tmp, md.n_ch, md.N, out_dev);
}

void hist_eval(kg_ctx *c, int melt, int nbins, int *out_dev)
{
    const MeltDev &md = c->sim.melt[melt];
    cudaMemsetAsync(out_dev, 0, sizeof(int) * 2 * nbins, c->stream);
    ++c->launches;
    k_hist<<<(md.M + 255) / 256, 256, 0, c->stream>>>(c->x, c->Mp, md.off, md.M, md.N, md.L, sqrt(c->stage.R0sq),
                                                      nbins, out_dev, out_dev + nbins);
}

}  // namespace kg
