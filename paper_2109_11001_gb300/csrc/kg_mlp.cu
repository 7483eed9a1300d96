// kg_mlp.cu -- weights, inference and training of the learned proposal's
// network (kg_mlp.cuh) on bf16 tensor cores.
//
// Training minimises the mean binary cross-entropy between sigmoid(s) and the
// logged target min(1, exp(-dE/T)) of each candidate swap, with Adam on the
// binary32 master weights.  One iteration is three launches:
//   k_mlp_fwdbwd  one warp per 16 rows: forward (as in inference), the output
//                 signal ds = (sigmoid(s) - t)/B, d2 = ds w3 [a2 > 0] and
//                 d1 = (d2 W2) [a1 > 0] on the tensor cores; writes the bf16
//                 operands of the weight gradients transposed (row = unit,
//                 column = batch row) and per-tile sums for b1, b2, w3, b3, loss;
//   k_mlp_wgrad_part  dW2 = d2^T h1 and dW1 = d1^T F split along K (the
//                 batch) in chunks of 256 rows: one warp per 16x8 output tile
//                 and chunk (a K = batch loop per warp left the tensor cores
//                 waiting on one dependent chain: 0.65 ms per iteration at
//                 32768 rows, 0.056 ms split); per-chunk sums of the per-tile
//                 sums;
//   k_mlp_wgrad_reduce  the chunks summed in order into the gradient; in
//                 training also each parameter's Adam step (betas 0.9,
//                 0.999) and its entries of the bf16 image.
// Every reduction runs in a fixed order: results do not depend on scheduling.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "kg_host.h"
#include "kg_mlp.cuh"

namespace kg {

constexpr int PART = 3 * MLP_H + 2;                 // b1, b2, w3, b3, loss sums of one tile

__global__ void __launch_bounds__(256) k_mlp_from_f64(const double *__restrict__ w, float *__restrict__ master)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) master[i] = (float)w[i];
}

// bf16 image entries of parameter i
__device__ __forceinline__ void pack_param(int i, float v, MlpSmem *__restrict__ blob, __nv_bfloat16 *__restrict__ w2t)
{
    if (i < P_B1) {
        blob->W1[(i / MLP_IN) * S1 + i % MLP_IN] = __float2bfloat16(v);
    } else if (i < P_W2) {
        blob->b1[i - P_B1] = v;
    } else if (i < P_B2) {
        const int o = (i - P_W2) / MLP_H, k = (i - P_W2) % MLP_H;
        blob->W2[o * S2 + k] = __float2bfloat16(v);
        w2t[k * S2 + o] = __float2bfloat16(v);
    } else if (i < P_W3) {
        blob->b2[i - P_B2] = v;
    } else if (i < P_B3) {
        blob->w3[i - P_W3] = v;
    } else {
        blob->b3 = v;
    }
}

__global__ void __launch_bounds__(256) k_mlp_pack(const float *__restrict__ master, MlpSmem *__restrict__ blob,
                                                 __nv_bfloat16 *__restrict__ w2t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) pack_param(i, master[i], blob, w2t);
}

// 16 feature rows (FP64, 24 per row) -> bf16 tile [16][S1], zero padded
__device__ __forceinline__ void stage_rows(__nv_bfloat16 *T, const double *__restrict__ F, const long long *idx,
                                           int nvalid)
{
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < 16 * 32; e += 32) {
        const int r = e >> 5, k = e & 31;
        T[r * S1 + k] = (r < nvalid && k < MLP_IN) ? __double2bfloat16(F[idx[r] * MLP_IN + k]) : __float2bfloat16(0.f);
    }
}

constexpr int INF_WARPS = 4;

__global__ void __launch_bounds__(32 * INF_WARPS) k_mlp_infer(const MlpSmem *__restrict__ blob,
                                                             const double *__restrict__ F, long long n,
                                                             double *__restrict__ s)
{
    __shared__ MlpSmem W;
    __shared__ __align__(16) __nv_bfloat16 T[INF_WARPS][16 * S1];
    __shared__ long long idx[INF_WARPS][16];
    mlp_load(W, blob);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r0 = ((long long)blockIdx.x * INF_WARPS + warp) * 16;
    if (r0 >= n) return;
    const int nv = n - r0 < 16 ? (int)(n - r0) : 16;
    if (lane < 16) idx[warp][lane] = r0 + (lane < nv ? lane : 0);
    __syncwarp();
    stage_rows(T[warp], F, idx[warp], nv);
    __syncwarp();
    float s0, s1;
    mlp_forward16(W, T[warp], s0, s1);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
        if (g < nv) s[r0 + g] = s0;
        if (g + 8 < nv) s[r0 + g + 8] = s1;
    }
}

// sum over the eight lane groups (lanes with equal lane & 3), fixed order
__device__ __forceinline__ float group_sum(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

struct TrainBufs {
    __nv_bfloat16 *FT, *h1T, *d2T, *d1T;   // [32 | 64][ldT] transposed operands
    float *part;                           // [ntiles][PART]
    float *wpart;                          // [chunks][WG_PART] split-K partials of the weight gradients
    int ldT;
};

// Forward + backward signals of 16-row tiles.  Row r of the batch is
// src row r (head == null, rows < nvalid valid) or a uniform draw from the
// last min(head, cap) rows of the training ring.
__global__ void __launch_bounds__(128) k_mlp_fwdbwd(const MlpSmem *__restrict__ blob,
                                                   const __nv_bfloat16 *__restrict__ w2t,
                                                   const double *__restrict__ F, const double *__restrict__ Tg,
                                                   long long cap, const long long *__restrict__ head,
                                                   unsigned long long seed, long long iter, int nvalid, int ntiles,
                                                   float invB, TrainBufs tb)
{
    __shared__ MlpSmem W;
    __shared__ __align__(16) __nv_bfloat16 W2T[MLP_H * S2];
    __shared__ __align__(16) __nv_bfloat16 T[4][16 * S1];
    __shared__ long long idx[4][16];
    mlp_load(W, blob);
    {
        const int4 *s = reinterpret_cast<const int4 *>(w2t);
        int4 *d = reinterpret_cast<int4 *>(W2T);
        for (int i = threadIdx.x; i < (int)(sizeof(W2T) / 16); i += blockDim.x) d[i] = s[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tile = blockIdx.x * 4 + warp;
    if (tile >= ntiles) return;
    const int r0 = tile * 16;
    const int nv = nvalid - r0 < 16 ? (nvalid - r0 > 0 ? nvalid - r0 : 0) : 16;
    if (lane < 16) {
        long long k = r0 + lane;
        if (head) {
            const long long h = *head, avail = h < cap ? h : cap;
            const uint4 r = draw(seed, 0, 3, (unsigned long long)iter, (uint32_t)(r0 + lane));
            const long long pick = mul_hi64(((unsigned long long)r.y << 32) | r.x, (unsigned long long)avail);
            k = (h - avail + pick) % cap;
        }
        idx[warp][lane] = lane < nv ? k : 0;
    }
    __syncwarp();
    __nv_bfloat16 *Ft = T[warp];
    stage_rows(Ft, F, idx[warp], nv);
    __syncwarp();
    for (int e = lane; e < 16 * 32; e += 32) {          // F^T for dW1
        const int r = e & 15, k = e >> 4;
        tb.FT[(long long)k * tb.ldT + r0 + r] = Ft[r * S1 + k];
    }
    const float t0 = g < nv ? (float)Tg[idx[warp][g]] : 0.f;
    const float t1 = g + 8 < nv ? (float)Tg[idx[warp][g + 8]] : 0.f;

    float a1[8][4], a2[8][4];
    uint32_t h[8][2];
    mlp_layer1(W, Ft, a1);
    mlp_hidden1(W, a1, h);
    mlp_layer2(W, h, a2);
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
#pragma unroll
        for (int q = 0; q < 4; ++q) a2[nt][q] += W.b2[col + (q & 1)];
        p0 += fmaxf(a2[nt][0], 0.f) * W.w3[col] + fmaxf(a2[nt][1], 0.f) * W.w3[col + 1];
        p1 += fmaxf(a2[nt][2], 0.f) * W.w3[col] + fmaxf(a2[nt][3], 0.f) * W.w3[col + 1];
#pragma unroll
        for (int q = 0; q < 4; ++q) a1[nt][q] += W.b1[col + (q & 1)];
        // h1^T for dW2
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&h[nt][0]);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&h[nt][1]);
        tb.h1T[(long long)col * tb.ldT + r0 + g] = lo.x;
        tb.h1T[(long long)(col + 1) * tb.ldT + r0 + g] = lo.y;
        tb.h1T[(long long)col * tb.ldT + r0 + g + 8] = hi.x;
        tb.h1T[(long long)(col + 1) * tb.ldT + r0 + g + 8] = hi.y;
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    const float s0 = p0 + W.b3, s1 = p1 + W.b3;
    // dL/ds and the loss: softplus(s) - t s, softplus(s) = max(s, 0) + log1p(exp(-|s|))
    const float ds0 = g < nv ? (1.f / (1.f + expf(-s0)) - t0) * invB : 0.f;
    const float ds1 = g + 8 < nv ? (1.f / (1.f + expf(-s1)) - t1) * invB : 0.f;
    float lsum = (g < nv ? fmaxf(s0, 0.f) + log1pf(expf(-fabsf(s0))) - t0 * s0 : 0.f)
                 + (g + 8 < nv ? fmaxf(s1, 0.f) + log1pf(expf(-fabsf(s1))) - t1 * s1 : 0.f);
    float dssum = ds0 + ds1;
    // d2 = ds w3 [a2 > 0]; sums for b2 and w3; bf16 d2 in A-fragment order
    uint32_t d2[8][2];
    float *part = tb.part + (long long)tile * PART;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float e0 = a2[nt][0] > 0.f ? ds0 * W.w3[col] : 0.f;
        const float e1 = a2[nt][1] > 0.f ? ds0 * W.w3[col + 1] : 0.f;
        const float e2 = a2[nt][2] > 0.f ? ds1 * W.w3[col] : 0.f;
        const float e3 = a2[nt][3] > 0.f ? ds1 * W.w3[col + 1] : 0.f;
        const float gb0 = group_sum(e0 + e2), gb1 = group_sum(e1 + e3);
        const float gw0 = group_sum(ds0 * fmaxf(a2[nt][0], 0.f) + ds1 * fmaxf(a2[nt][2], 0.f));
        const float gw1 = group_sum(ds0 * fmaxf(a2[nt][1], 0.f) + ds1 * fmaxf(a2[nt][3], 0.f));
        if (g == 0) {
            part[MLP_H + col] = gb0;
            part[MLP_H + col + 1] = gb1;
            part[2 * MLP_H + col] = gw0;
            part[2 * MLP_H + col + 1] = gw1;
        }
        d2[nt][0] = pack_bf16x2(e0, e1);
        d2[nt][1] = pack_bf16x2(e2, e3);
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&d2[nt][0]);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&d2[nt][1]);
        tb.d2T[(long long)col * tb.ldT + r0 + g] = lo.x;
        tb.d2T[(long long)(col + 1) * tb.ldT + r0 + g] = lo.y;
        tb.d2T[(long long)col * tb.ldT + r0 + g + 8] = hi.x;
        tb.d2T[(long long)(col + 1) * tb.ldT + r0 + g + 8] = hi.y;
    }
    // d1 = (d2 W2) [a1 > 0]: B[k = j][n = i] = W2[j][i] = W2T[i][j]
    float d1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) d1[nt][0] = d1[nt][1] = d1[nt][2] = d1[nt][3] = 0.f;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        const uint32_t x0 = d2[2 * kb][0], x1 = d2[2 * kb][1], x2 = d2[2 * kb + 1][0], x3 = d2[2 * kb + 1][1];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16 *w = W2T + (nt * 8 + g) * S2 + kb * 16 + 2 * t;
            mma_bf16(d1[nt], x0, x1, x2, x3, ld_b32(w), ld_b32(w + 8));
        }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float e0 = a1[nt][0] > 0.f ? d1[nt][0] : 0.f, e1 = a1[nt][1] > 0.f ? d1[nt][1] : 0.f;
        const float e2 = a1[nt][2] > 0.f ? d1[nt][2] : 0.f, e3 = a1[nt][3] > 0.f ? d1[nt][3] : 0.f;
        const float gb0 = group_sum(e0 + e2), gb1 = group_sum(e1 + e3);
        if (g == 0) {
            part[col] = gb0;
            part[col + 1] = gb1;
        }
        tb.d1T[(long long)col * tb.ldT + r0 + g] = __float2bfloat16(e0);
        tb.d1T[(long long)(col + 1) * tb.ldT + r0 + g] = __float2bfloat16(e1);
        tb.d1T[(long long)col * tb.ldT + r0 + g + 8] = __float2bfloat16(e2);
        tb.d1T[(long long)(col + 1) * tb.ldT + r0 + g + 8] = __float2bfloat16(e3);
    }
    dssum = group_sum(dssum);
    lsum = group_sum(lsum);
    // rows g and g+8 were summed by lane groups; the four lanes t of group 0 hold
    // the same totals (every t carries the same row values)
    if (lane == 0) {
        part[3 * MLP_H] = dssum;
        part[3 * MLP_H + 1] = lsum;
    }
}

// Weight gradients split along K (the batch): chunk c of WG_ROWS batch rows,
// grid (chunks, 12).  Blocks y < 11: four warps each, one 16x8 output tile per
// warp (y*4 + warp < 32: dW2 = d2^T h1, else dW1 = d1^T F), the chunk's
// partial product on the tensor cores, written lane-major; block y = 11 sums
// the chunk's per-tile sums (b1, b2, w3, b3, loss) in tile order.  Every
// partial is a fixed-order sum, so results do not depend on scheduling.
constexpr int WG_TILES = 44;                       // 32 tiles of dW2, 12 of dW1
constexpr int WG_ROWS = 256;                       // batch rows per chunk (16 row tiles)
constexpr int WG_PART = WG_TILES * 128 + PART;     // partial values of one chunk

__global__ void __launch_bounds__(128) k_mlp_wgrad_part(TrainBufs tb, int ntiles, float *__restrict__ partial)
{
    const int chunk = blockIdx.x, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tile0 = chunk * (WG_ROWS / 16), tile1 = min(ntiles, tile0 + WG_ROWS / 16);
    float *out = partial + (long long)chunk * WG_PART;
    if (blockIdx.y == 11) {                              // per-tile sums, in tile order
        for (int e = threadIdx.x; e < PART; e += blockDim.x) {
            float acc = 0.f;
            for (int k = tile0; k < tile1; ++k) acc += tb.part[(long long)k * PART + e];
            out[WG_TILES * 128 + e] = acc;
        }
        return;
    }
    const int tile = blockIdx.y * 4 + (threadIdx.x >> 5);
    const __nv_bfloat16 *A, *Bm;
    int mt, nt;
    if (tile < 32) {
        A = tb.d2T; Bm = tb.h1T; mt = tile >> 3; nt = tile & 7;
    } else {
        A = tb.d1T; Bm = tb.FT; mt = (tile - 32) / 3; nt = (tile - 32) % 3;
    }
    const long long ld = tb.ldT;
    const __nv_bfloat16 *a_lo = A + (long long)(mt * 16 + g) * ld + 2 * t, *a_hi = a_lo + 8 * ld;
    const __nv_bfloat16 *bp = Bm + (long long)(nt * 8 + g) * ld + 2 * t;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kb = tile0 * 16; kb < tile1 * 16; kb += 16)
        mma_bf16(acc, ld_b32(a_lo + kb), ld_b32(a_hi + kb), ld_b32(a_lo + kb + 8), ld_b32(a_hi + kb + 8),
                 ld_b32(bp + kb), ld_b32(bp + kb + 8));
    float *o = out + tile * 128 + lane * 4;
#pragma unroll
    for (int r = 0; r < 4; ++r) o[r] = acc[r];
}

// Adam step (betas 0.9, 0.999) of parameter i with gradient gi, and its
// entries of the bf16 image.
struct AdamArgs {
    float *master, *m, *v;
    float lr, c1, c2;
    MlpSmem *blob;
    __nv_bfloat16 *w2t;
};

__device__ __forceinline__ void adam_update(const AdamArgs &a, int i, float gi)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mi = b1 * a.m[i] + (1.f - b1) * gi, vi = b2 * a.v[i] + (1.f - b2) * gi * gi;
    a.m[i] = mi;
    a.v[i] = vi;
    const float w = a.master[i] - a.lr * (mi / a.c1) / (sqrtf(vi / a.c2) + eps);
    a.master[i] = w;
    pack_param(i, w, a.blob, a.w2t);
}

// The chunks' partials summed in chunk order into the packed gradient (and,
// with ADAM, the Adam step of each parameter from its gradient).
template <bool ADAM>
__global__ void __launch_bounds__(256) k_mlp_wgrad_reduce(const float *__restrict__ partial, int nchunks, float invB,
                                                         float *__restrict__ grad, AdamArgs adam)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= WG_PART) return;
    float acc = 0.f;
    for (int c = 0; c < nchunks; ++c) acc += partial[(long long)c * WG_PART + i];
    int pi;
    if (i < WG_TILES * 128) {
        const int tile = i >> 7, lane = (i & 127) >> 2, r = i & 3, g = lane >> 2, t = lane & 3;
        if (tile < 32) {
            const int row = (tile >> 3) * 16 + g + (r >> 1) * 8, col = (tile & 7) * 8 + 2 * t + (r & 1);
            pi = P_W2 + row * MLP_H + col;
        } else {
            const int mt = (tile - 32) / 3, nt = (tile - 32) % 3;
            const int row = mt * 16 + g + (r >> 1) * 8, col = nt * 8 + 2 * t + (r & 1);
            pi = P_W1 + row * MLP_IN + col;
        }
    } else {
        const int e = i - WG_TILES * 128;
        if (e < MLP_H) pi = P_B1 + e;
        else if (e < 2 * MLP_H) pi = P_B2 + e - MLP_H;
        else if (e < 3 * MLP_H) pi = P_W3 + e - 2 * MLP_H;
        else if (e == 3 * MLP_H) pi = P_B3;
        else {
            grad[MLP_NPARAM] = acc * invB;               // mean loss
            return;
        }
    }
    grad[pi] = acc;
    if (ADAM) adam_update(adam, pi, acc);
}

__global__ void k_grad_to_f64(const float *__restrict__ g, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= MLP_NPARAM) out[i == MLP_NPARAM ? 0 : i + 1] = (double)g[i];
}

__global__ void k_f32_to_f64(const float *__restrict__ a, double *__restrict__ out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i];
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

bool mlp_ensure(kg_ctx *c)
{
    if (c->mlp_master) return true;
    c->mlp_master = (float *)dev_alloc(c, sizeof(float) * MLP_NPARAM);
    c->mlp_adam = (float *)dev_alloc(c, sizeof(float) * 2 * MLP_NPARAM);
    c->mlp_grad = (float *)dev_alloc(c, sizeof(float) * (MLP_NPARAM + 1));
    c->mlp_blob = dev_alloc(c, sizeof(MlpSmem));
    c->mlp_w2t = dev_alloc(c, sizeof(__nv_bfloat16) * MLP_H * S2);
    c->bmax2 = (unsigned long long *)dev_alloc(c, sizeof(unsigned long long));
    if (c->mlp_master && c->mlp_adam && c->mlp_grad && c->mlp_blob && c->mlp_w2t && c->bmax2) return true;
    void *bufs[] = {c->mlp_master, c->mlp_adam, c->mlp_grad, c->mlp_blob, c->mlp_w2t, c->bmax2};
    for (void *b : bufs) dev_free(c, b);
    c->mlp_master = nullptr;
    c->mlp_adam = c->mlp_grad = nullptr;
    c->mlp_blob = c->mlp_w2t = nullptr;
    c->bmax2 = nullptr;
    return false;
}

void mlp_set(kg_ctx *c, const double *w_dev)
{
    cudaStream_t st = c->stream;
    k_mlp_from_f64<<<nblk(MLP_NPARAM, 256), 256, 0, st>>>(w_dev, c->mlp_master);
    k_mlp_pack<<<nblk(MLP_NPARAM, 256), 256, 0, st>>>(c->mlp_master, (MlpSmem *)c->mlp_blob,
                                                      (__nv_bfloat16 *)c->mlp_w2t);
    cudaMemsetAsync(c->mlp_adam, 0, sizeof(float) * 2 * MLP_NPARAM, st);
    c->adam_t = 0;
    c->launches += 2;
}

void mlp_get(kg_ctx *c, double *w_dev)
{
    k_f32_to_f64<<<nblk(MLP_NPARAM, 256), 256, 0, c->stream>>>(c->mlp_master, w_dev, MLP_NPARAM);
    ++c->launches;
}

void mlp_infer(kg_ctx *c, const double *f_dev, long long n, double *s_dev)
{
    if (n <= 0) return;
    k_mlp_infer<<<nblk(n, 16 * INF_WARPS), 32 * INF_WARPS, 0, c->stream>>>((const MlpSmem *)c->mlp_blob, f_dev, n,
                                                                          s_dev);
    ++c->launches;
}

static bool ensure_train_bufs(kg_ctx *c, int ntiles)
{
    const long long rows = (long long)ntiles * 16;
    if (rows <= c->tr_rows) return true;
    dev_free(c, c->tr_buf);
    const size_t chunks = (size_t)(rows + WG_ROWS - 1) / WG_ROWS;
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)rows * (32 + 3 * MLP_H) + sizeof(float) * (size_t)ntiles * PART +
                         sizeof(float) * chunks * WG_PART;
    c->tr_buf = dev_alloc(c, bytes);
    c->tr_rows = c->tr_buf ? rows : 0;
    return c->tr_buf != nullptr;
}

static TrainBufs train_bufs(kg_ctx *c, int ntiles)
{
    TrainBufs tb;
    tb.ldT = ntiles * 16;
    __nv_bfloat16 *p = (__nv_bfloat16 *)c->tr_buf;
    const size_t ld = (size_t)c->tr_rows;   // stride of the allocation; operands use ldT <= ld
    tb.FT = p;
    tb.h1T = p + 32 * ld;
    tb.d2T = p + (32 + MLP_H) * ld;
    tb.d1T = p + (32 + 2 * MLP_H) * ld;
    tb.part = reinterpret_cast<float *>(p + (32 + 3 * MLP_H) * ld);
    tb.wpart = tb.part + (size_t)(ld / 16) * PART;      // after the allocation's per-tile sums
    return tb;
}

// forward + backward of one batch and the weight gradients; with adam, the
// Adam step fused into the gradient reduction
static void fwd_bwd(kg_ctx *c, const double *F, const double *T, long long cap, const long long *head, long long iter,
                    int nvalid, int ntiles, const AdamArgs *adam)
{
    cudaStream_t st = c->stream;
    TrainBufs tb = train_bufs(c, ntiles);
    const float invB = 1.f / (float)nvalid;
    k_mlp_fwdbwd<<<nblk(ntiles, 4), 128, 0, st>>>((const MlpSmem *)c->mlp_blob, (const __nv_bfloat16 *)c->mlp_w2t, F,
                                                  T, cap, head, c->p.seed, iter, nvalid, ntiles, invB, tb);
    const int nchunks = (ntiles * 16 + WG_ROWS - 1) / WG_ROWS;
    k_mlp_wgrad_part<<<dim3(nchunks, 12), 128, 0, st>>>(tb, ntiles, tb.wpart);
    if (adam)
        k_mlp_wgrad_reduce<true><<<nblk(WG_PART, 256), 256, 0, st>>>(tb.wpart, nchunks, invB, c->mlp_grad, *adam);
    else
        k_mlp_wgrad_reduce<false><<<nblk(WG_PART, 256), 256, 0, st>>>(tb.wpart, nchunks, invB, c->mlp_grad,
                                                                       AdamArgs{});
    c->launches += 3;
}

bool mlp_grad(kg_ctx *c, const double *f_dev, const double *t_dev, long long n, double *loss_grad_dev)
{
    const int ntiles = (int)((n + 15) / 16);
    if (!ensure_train_bufs(c, ntiles)) return false;
    fwd_bwd(c, f_dev, t_dev, 0, nullptr, 0, (int)n, ntiles, nullptr);
    k_grad_to_f64<<<nblk(MLP_NPARAM + 1, 256), 256, 0, c->stream>>>(c->mlp_grad, loss_grad_dev);
    ++c->launches;
    return true;
}

bool mlp_train(kg_ctx *c, int iters, int batch, double lr, double *loss_dev)
{
    const int ntiles = (batch + 15) / 16;
    if (!ensure_train_bufs(c, ntiles)) return false;
    for (int it = 0; it < iters; ++it) {
        ++c->adam_t;
        AdamArgs ad;
        ad.master = c->mlp_master;
        ad.m = c->mlp_adam;
        ad.v = c->mlp_adam + MLP_NPARAM;
        ad.lr = (float)lr;
        ad.c1 = (float)(1.0 - std::pow(0.9, (double)c->adam_t));
        ad.c2 = (float)(1.0 - std::pow(0.999, (double)c->adam_t));
        ad.blob = (MlpSmem *)c->mlp_blob;
        ad.w2t = (__nv_bfloat16 *)c->mlp_w2t;
        fwd_bwd(c, c->trainf, c->traint, c->train_cap, c->d_train_head, c->train_iter++, ntiles * 16, ntiles, &ad);
    }
    k_f32_to_f64<<<1, 32, 0, c->stream>>>(c->mlp_grad + MLP_NPARAM, loss_dev, 1);
    ++c->launches;
    return true;
}

}  // namespace kg
