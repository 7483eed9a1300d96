// kg_mlp.cuh -- the learned double-bridging proposal's network on bf16 tensor
// cores (mma.sync m16n8k16, fp32 accumulate), one warp per 16 rows.
//
// Network: 24 features -> 64 (ReLU) -> 64 (ReLU) -> 1 logit.  Parameters are
// packed as W1[64][24], b1[64], W2[64][64], b2[64], w3[64], b3 (row = output
// unit), KG_MLP_NPARAM values.  The device keeps binary32 master weights and,
// for the tensor cores, a bf16 image (MlpSmem) that every block copies into
// shared memory:
//   layer 1: features and W1 in bf16 (inputs padded 24 -> 32 with zeros),
//            + b1 in fp32, ReLU, rounded to bf16 for layer 2;
//   layer 2: bf16 x bf16 with fp32 accumulate, + b2, ReLU (fp32);
//   output:  fp32 dot with w3, + b3.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kg {

constexpr int MLP_IN = 24, MLP_H = 64;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
constexpr int P_W1 = 0, P_B1 = MLP_H * MLP_IN, P_W2 = P_B1 + MLP_H, P_B2 = P_W2 + MLP_H * MLP_H,
              P_W3 = P_B2 + MLP_H, P_B3 = P_W3 + MLP_H;
// bf16 row strides: 40 (80 B) and 72 (144 B) halves make the eight rows a
// fragment load touches fall in distinct shared-memory banks
constexpr int S1 = 40, S2 = 72;

struct __align__(16) MlpSmem {
    __nv_bfloat16 W1[MLP_H * S1];     // [out][in], in 24..39 zero
    __nv_bfloat16 W2[MLP_H * S2];     // [out][in]
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3, pad[3];
};
static_assert(sizeof(MlpSmem) % 16 == 0, "MlpSmem is copied in 16-byte words");

// block-wide copy of the bf16 image into shared memory (caller synchronises)
__device__ __forceinline__ void mlp_load(MlpSmem &dst, const MlpSmem *__restrict__ src)
{
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// D = A(16x16, row) * B(16x8, col) + D, bf16 inputs, fp32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Fragment ownership (lane = 4 g + t): A rows g and g+8, columns 2t, 2t+1 and
// 2t+8, 2t+9 of each 16-wide k block; B column g, rows 2t, 2t+1, 2t+8, 2t+9;
// C rows g and g+8, columns 2t, 2t+1 of each 8-wide n tile.  The C tiles 2j,
// 2j+1 of one layer are exactly the A fragment of k block j of the next.

// Layer 1 of 16 rows: acc <- F[16][S1] * W1^T (no bias).
__device__ __forceinline__ void mlp_layer1(const MlpSmem &W, const __nv_bfloat16 *F, float (&acc)[8][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kb = 0; kb < 32; kb += 16) {
        const uint32_t a0 = ld_b32(F + g * S1 + kb + 2 * t), a1 = ld_b32(F + (g + 8) * S1 + kb + 2 * t);
        const uint32_t a2 = ld_b32(F + g * S1 + kb + 8 + 2 * t), a3 = ld_b32(F + (g + 8) * S1 + kb + 8 + 2 * t);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16 *w = W.W1 + (nt * 8 + g) * S1 + kb + 2 * t;
            mma_bf16(acc[nt], a0, a1, a2, a3, ld_b32(w), ld_b32(w + 8));
        }
    }
}

// h1 = bf16(relu(acc + b1)) in A-fragment order: h[nt][0] row g, h[nt][1] row g+8
__device__ __forceinline__ void mlp_hidden1(const MlpSmem &W, const float (&acc)[8][4], uint32_t (&h)[8][2])
{
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        h[nt][0] = pack_bf16x2(fmaxf(acc[nt][0] + W.b1[col], 0.f), fmaxf(acc[nt][1] + W.b1[col + 1], 0.f));
        h[nt][1] = pack_bf16x2(fmaxf(acc[nt][2] + W.b1[col], 0.f), fmaxf(acc[nt][3] + W.b1[col + 1], 0.f));
    }
}

// Layer 2: acc <- h1 * W2^T (no bias).
__device__ __forceinline__ void mlp_layer2(const MlpSmem &W, const uint32_t (&h)[8][2], float (&acc)[8][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        const uint32_t a0 = h[2 * kb][0], a1 = h[2 * kb][1], a2 = h[2 * kb + 1][0], a3 = h[2 * kb + 1][1];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16 *w = W.W2 + (nt * 8 + g) * S2 + kb * 16 + 2 * t;
            mma_bf16(acc[nt], a0, a1, a2, a3, ld_b32(w), ld_b32(w + 8));
        }
    }
}

// Logits of 16 rows of bf16 features F[16][S1] (columns 24.. zero): s0 for
// row g, s1 for row g+8, identical in the four lanes of group g.  Sums across
// the group run in a fixed butterfly order, so the result is reproducible.
__device__ __forceinline__ void mlp_forward16(const MlpSmem &W, const __nv_bfloat16 *F, float &s0, float &s1)
{
    const int t = threadIdx.x & 3;
    float acc[8][4];
    uint32_t h[8][2];
    mlp_layer1(W, F, acc);
    mlp_hidden1(W, acc, h);
    mlp_layer2(W, h, acc);
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        p0 += fmaxf(acc[nt][0] + W.b2[col], 0.f) * W.w3[col] + fmaxf(acc[nt][1] + W.b2[col + 1], 0.f) * W.w3[col + 1];
        p1 += fmaxf(acc[nt][2] + W.b2[col], 0.f) * W.w3[col] + fmaxf(acc[nt][3] + W.b2[col + 1], 0.f) * W.w3[col + 1];
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    s0 = p0 + W.b3;
    s1 = p1 + W.b3;
}

}  // namespace kg
