// mlp.cuh -- device code of the learned ray-interval proposal (sm_103a).
//
// A 224 -> 64 -> 64 -> 64 -> 3 MLP with ReLU, FP16 operands and FP32
// accumulation.  Inference runs on the tcgen05 tensor cores (mlp_tc.cuh).
// Training's fused forward and backward pass, whose per-warp fragments feed
// the gradient products, uses the warp-level mma.sync m16n8k16 below: one warp
// owns 16 rays:
// layer 1 reads its A operand (16 rays x 224 inputs) from shared memory; every
// later layer takes the previous layer's accumulator fragments, repacked to
// FP16, directly as its A operand (the m16n8 accumulator layout of two
// adjacent n-tiles is the m16k16 A layout).  Weights live in shared memory,
// transposed for the forward pass (B operand = W^T rows) and in their
// original layout for the backward pass.
#pragma once

#include <cuda_fp16.h>

#include "raycast.cuh"

namespace isaac {

constexpr int MLP_IN = 224, MLP_W = 64, MLP_OUT = 3;
constexpr int MLP_NFREQ = 16, MLP_NGRID = 32;

// FP32 parameter layout (public): W1[224][64] in-major, b1[64], W2[64][64],
// b2[64], W3[64][64], b3[64], W4[64][3], b4[3].
constexpr int P_W1 = 0, P_B1 = P_W1 + MLP_IN * MLP_W, P_W2 = P_B1 + MLP_W;
constexpr int P_B2 = P_W2 + MLP_W * MLP_W, P_W3 = P_B2 + MLP_W, P_B3 = P_W3 + MLP_W * MLP_W;
constexpr int P_W4 = P_B3 + MLP_W, P_B4 = P_W4 + MLP_W * MLP_OUT, N_PARAMS = P_B4 + MLP_OUT;
static_assert(N_PARAMS == 22915, "parameter count");

// FP16 kernel copy: forward T1[64][224], T2[64][64], T3[64][64], T4[8][64]
// (out-major, rows 3..7 zero); backward B2[64][64], B3[64][64] (in-major)
// and B4[64][16] (W4 in-major, outputs padded to 16).
constexpr int H_T1 = 0, H_T2 = H_T1 + MLP_W * MLP_IN, H_T3 = H_T2 + MLP_W * MLP_W;
constexpr int H_T4 = H_T3 + MLP_W * MLP_W, H_B2 = H_T4 + 8 * MLP_W, H_B3 = H_B2 + MLP_W * MLP_W;
constexpr int H_B4 = H_B3 + MLP_W * MLP_W, N_HALF = H_B4 + MLP_W * 16;

// shared-memory leading dimensions (halves), padded so that the 8 rows a
// fragment load touches fall in distinct banks
constexpr int LD_IN = 232, LD_W = 72, LD_B4 = 24, LD_R = 72;

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack_h2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&h);
}

__device__ __forceinline__ unsigned ld32(const __half *p) { return *reinterpret_cast<const unsigned *>(p); }

// A fragment (16 x 16) of a row-major tile: rows = rays, columns = k.
__device__ __forceinline__ void frag_a(const __half *tile, int ld, int row0, int k0, unsigned (&a)[4])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const __half *p = tile + (row0 + g) * ld + k0 + 2 * t;
    a[0] = ld32(p);
    a[1] = ld32(p + 8 * ld);
    a[2] = ld32(p + 8);
    a[3] = ld32(p + 8 * ld + 8);
}

// B fragment (16 x 8): element (k, n) stored at bt[n * ld + k].
__device__ __forceinline__ void frag_b(const __half *bt, int ld, int n0, int k0, unsigned (&b)[2])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const __half *p = bt + (n0 + g) * ld + k0 + 2 * t;
    b[0] = ld32(p);
    b[1] = ld32(p + 8);
}

// Two adjacent n8 accumulator tiles -> one k16 A fragment (optionally ReLU).
__device__ __forceinline__ void acc_to_a(const float (&c0)[4], const float (&c1)[4], unsigned (&a)[4])
{
    a[0] = pack_h2(c0[0], c0[1]);
    a[1] = pack_h2(c0[2], c0[3]);
    a[2] = pack_h2(c1[0], c1[1]);
    a[3] = pack_h2(c1[2], c1[3]);
}

__device__ __forceinline__ void add_bias_relu(float (&c)[4], const float *bias, int n0, bool relu)
{
    const int t = threadIdx.x & 3;
    const float b0 = bias[n0 + 2 * t], b1 = bias[n0 + 2 * t + 1];
    c[0] += b0;
    c[1] += b1;
    c[2] += b0;
    c[3] += b1;
    if (relu)
        for (int i = 0; i < 4; ++i) c[i] = fmaxf(c[i], 0.0f);
}

// Copy the FP16 kernel weights into shared memory (forward; backward optional).
__device__ __forceinline__ void load_weights_smem(const __half *hw, __half *sT1, __half *sT2,
                                                  __half *sT3, __half *sT4, __half *sB2,
                                                  __half *sB3, __half *sB4)
{
    for (int i = threadIdx.x; i < MLP_W * MLP_IN; i += blockDim.x)
        sT1[(i / MLP_IN) * LD_IN + i % MLP_IN] = hw[H_T1 + i];
    for (int i = threadIdx.x; i < MLP_W * MLP_W; i += blockDim.x) {
        sT2[(i / MLP_W) * LD_W + i % MLP_W] = hw[H_T2 + i];
        sT3[(i / MLP_W) * LD_W + i % MLP_W] = hw[H_T3 + i];
        if (sB2) {
            sB2[(i / MLP_W) * LD_W + i % MLP_W] = hw[H_B2 + i];
            sB3[(i / MLP_W) * LD_W + i % MLP_W] = hw[H_B3 + i];
        }
    }
    for (int i = threadIdx.x; i < 8 * MLP_W; i += blockDim.x) sT4[(i / MLP_W) * LD_W + i % MLP_W] = hw[H_T4 + i];
    if (sB4)
        for (int i = threadIdx.x; i < MLP_W * 16; i += blockDim.x) sB4[(i / 16) * LD_B4 + i % 16] = hw[H_B4 + i];
}

// Hidden activations of one warp's 16 rays, kept for the backward pass.
struct Hidden {
    unsigned a2[4][4], a3[4][4], a4[4][4];   // FP16 A fragments of h1, h2, h3
    unsigned m1, m2, m3;                     // ReLU masks (bit i*4+j of n-tile i, element j)
};

// Forward pass of one warp: X rows [row0, row0+16) of the tile -> u (n-tile
// of 8 outputs, 3 used).  Optionally stores h1..h3 transposed into shared
// tiles (feature-major, ray column = col0 + ray).
__device__ __forceinline__ void mlp_forward_warp(const __half *xs, int row0, const __half *sT1,
                                                 const __half *sT2, const __half *sT3,
                                                 const __half *sT4, const float *params,
                                                 float (&u)[4], Hidden *hid, __half *h1t,
                                                 __half *h2t, __half *h3t, int col0)
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    float c[8][4];
    // layer 1
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll 2
    for (int ks = 0; ks < MLP_IN / 16; ++ks) {
        unsigned a[4];
        frag_a(xs, LD_IN, row0, ks * 16, a);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            unsigned b[2];
            frag_b(sT1, LD_IN, nt * 8, ks * 16, b);
            mma16816(c[nt], a, b);
        }
    }
    unsigned A[4][4];
    unsigned mask = 0;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        add_bias_relu(c[nt], params + P_B1, nt * 8, true);
        for (int j = 0; j < 4; ++j) mask |= (c[nt][j] > 0.0f ? 1u : 0u) << (nt * 4 + j);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) acc_to_a(c[2 * j], c[2 * j + 1], A[j]);
    if (hid) {
        hid->m1 = mask;
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) hid->a2[j][q] = A[j][q];
    }
    if (h1t)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int f = nt * 8 + 2 * t;
            h1t[f * LD_R + col0 + g] = __float2half_rn(c[nt][0]);
            h1t[(f + 1) * LD_R + col0 + g] = __float2half_rn(c[nt][1]);
            h1t[f * LD_R + col0 + g + 8] = __float2half_rn(c[nt][2]);
            h1t[(f + 1) * LD_R + col0 + g + 8] = __float2half_rn(c[nt][3]);
        }
    // layers 2 and 3
#pragma unroll
    for (int layer = 2; layer <= 3; ++layer) {
        const __half *sT = layer == 2 ? sT2 : sT3;
        const float *bias = params + (layer == 2 ? P_B2 : P_B3);
        __half *ht = layer == 2 ? h2t : h3t;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                unsigned b[2];
                frag_b(sT, LD_W, nt * 8, ks * 16, b);
                mma16816(c[nt], A[ks], b);
            }
        }
        mask = 0;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            add_bias_relu(c[nt], bias, nt * 8, true);
            for (int j = 0; j < 4; ++j) mask |= (c[nt][j] > 0.0f ? 1u : 0u) << (nt * 4 + j);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc_to_a(c[2 * j], c[2 * j + 1], A[j]);
        if (hid) {
            if (layer == 2) hid->m2 = mask; else hid->m3 = mask;
            for (int j = 0; j < 4; ++j)
                for (int q = 0; q < 4; ++q) (layer == 2 ? hid->a3 : hid->a4)[j][q] = A[j][q];
        }
        if (ht)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int f = nt * 8 + 2 * t;
                ht[f * LD_R + col0 + g] = __float2half_rn(c[nt][0]);
                ht[(f + 1) * LD_R + col0 + g] = __float2half_rn(c[nt][1]);
                ht[f * LD_R + col0 + g + 8] = __float2half_rn(c[nt][2]);
                ht[(f + 1) * LD_R + col0 + g + 8] = __float2half_rn(c[nt][3]);
            }
    }
    // layer 4 (8 output columns, 3 used)
    u[0] = u[1] = u[2] = u[3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        unsigned b[2];
        frag_b(sT4, LD_W, 0, ks * 16, b);
        mma16816(u, A[ks], b);
    }
    const int col = 2 * t;
    const float b0 = col < MLP_OUT ? params[P_B4 + col] : 0.0f;
    const float b1 = col + 1 < MLP_OUT ? params[P_B4 + col + 1] : 0.0f;
    u[0] += b0;
    u[1] += b1;
    u[2] += b0;
    u[3] += b1;
}

__constant__ float c_freq2[MLP_NFREQ] = {
    1.0f, 1.41421356f, 2.0f, 2.82842712f, 4.0f, 5.65685425f, 8.0f, 11.3137085f,
    16.0f, 22.6274170f, 32.0f, 45.2548340f, 64.0f, 90.5096680f, 128.0f, 181.019336f};

// The 224 inputs of one ray: sin/cos(pi * 2^(k/2) * s) of the 6 scalars
// (e/n, d), then 32 samples of the max-opacity grid along the ray's segment.
// half_id selects which half of the inputs this thread writes (0: scalars
// 0-2 and grid samples 0-15; 1: scalars 3-5 and samples 16-31).
__device__ __forceinline__ void ray_features_half(const RayRec &r, float step, const float *grid,
                                                  int cell, int gx, int gy, int gz, float nx,
                                                  float ny, float nz, int half_id, __half *out)
{
    const float s6[6] = {r.ex / nx, r.ey / ny, r.ez / nz, r.dx, r.dy, r.dz};
    // The frequencies 2^(k/2) form two doubling chains (k even from 1, k odd
    // from sqrt(2)): sincospi at the head of each, then the double-angle
    // formulas sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a).
    // A doubling doubles the absolute error, so after the seven of a chain it
    // is ~2^7 * 1e-7, far below the FP16 rounding of the stored value.
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        const int j = half_id * 3 + jj;
#pragma unroll
        for (int chain = 0; chain < 2; ++chain) {
            float sv, cv;
            sincospif(s6[j] * c_freq2[chain], &sv, &cv);
#pragma unroll
            for (int k = chain; k < MLP_NFREQ; k += 2) {
                out[(j * MLP_NFREQ + k) * 2] = __float2half_rn(sv);
                out[(j * MLP_NFREQ + k) * 2 + 1] = __float2half_rn(cv);
                const float s2 = 2.0f * sv * cv;
                cv = (cv - sv) * (cv + sv);
                sv = s2;
            }
        }
    }
    const float L = (float)r.nsteps * step;
    const float inv_cell = 1.0f / (float)cell;
#pragma unroll 4
    for (int ii = 0; ii < MLP_NGRID / 2; ++ii) {
        const int i = half_id * (MLP_NGRID / 2) + ii;
        const float tt = ((float)i + 0.5f) * (1.0f / MLP_NGRID) * L;
        const int cx = min(max((int)floorf(fmaf(tt, r.dx, r.ex) * inv_cell), 0), gx - 1);
        const int cy = min(max((int)floorf(fmaf(tt, r.dy, r.ey) * inv_cell), 0), gy - 1);
        const int cz = min(max((int)floorf(fmaf(tt, r.dz, r.ez) * inv_cell), 0), gz - 1);
        out[6 * 2 * MLP_NFREQ + i] = __float2half_rn(__ldg(grid + ((long long)cz * gy + cy) * gx + cx));
    }
}

}  // namespace isaac
