// mlp_tc.cuh -- inference of the proposal MLP on the 5th-generation tensor
// cores (tcgen05, sm_103a): 128 rays per CTA tile.
//
// The activations of a tile (128 rays x K, FP16) and the weights (N x K,
// FP16, out-major = K-major operand B) sit in shared memory in the canonical
// K-major layout without swizzling: 8 x 16-byte "core matrices" (8 rows of 8
// consecutive k), the core matrices of one 8-row group adjacent along rows
// (stride 128 B), the k-chunks of 8 one "leading dimension" stride apart.  One
// elected thread issues tcgen05.mma (M = 128, N = 64 or 16, K = 16 per
// instruction, FP32 accumulators in 64 TMEM columns), commits them to an
// mbarrier, and the CTA's eight warps read the accumulators back with
// tcgen05.ld (warp w: TMEM lanes 32*(w%4).., columns 32*(w/4)..), add the bias,
// apply ReLU and write the next layer's FP16 operand into the same tile.
// Every wait on the mbarrier is bounded: past the limit the tile is marked
// failed (its rays keep their whole range; forward outputs are NaN) and the
// CTA stops after freeing its TMEM.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

#include "mlp.cuh"

namespace isaac {

constexpr int kTcRows = 128;                         // rays per tile (MMA M)
constexpr int kTcThreads = 256;                      // 2 threads per ray for the features
constexpr int kTcCols = 64;                          // TMEM columns per CTA
constexpr int kTcLboX = kTcRows / 8 * 128;           // k-chunk stride of an activation tile (2048 B)
constexpr int kTcLboW = MLP_W / 8 * 128;             // k-chunk stride of a 64-row weight tile
constexpr int kTcLboW4 = 16 / 8 * 128;               // of the 16-row output weight tile
constexpr int kTcBytesW1 = MLP_W * MLP_IN * 2, kTcBytesW = MLP_W * MLP_W * 2, kTcBytesW4 = 16 * MLP_W * 2;
constexpr int kTcBytesX = kTcRows * MLP_IN * 2;
// shared memory: W1, W2, W3, W4 tiles, the activation tile, biases, mbarrier, TMEM address
constexpr int kTcOffW2 = kTcBytesW1, kTcOffW3 = kTcOffW2 + kTcBytesW, kTcOffW4 = kTcOffW3 + kTcBytesW;
constexpr int kTcOffX = kTcOffW4 + kTcBytesW4, kTcOffBias = kTcOffX + kTcBytesX;
constexpr int kTcOffBar = kTcOffBias + (3 * MLP_W + 4) * 4, kTcSmemBytes = kTcOffBar + 16;
// iterations of the bounded mbarrier wait (each try_wait may itself suspend)
constexpr unsigned kTcWaitLimit = 1u << 22;

// Byte offset of element (row, k) in a K-major tile with k-chunk stride lbo.
__device__ __forceinline__ int tc_off(int row, int k, int lbo)
{
    return (k >> 3) * lbo + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (k-chunk) and
// stride (8-row group) byte offsets, the fixed 0b001 at bits 46-48, no
// swizzling.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, int lbo, int sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulators, FP16 A and B, both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Make generic-proxy writes to shared memory visible to the tensor cores.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Bounded wait for phase `parity` of the mbarrier: true when it completed.
__device__ __forceinline__ bool tc_wait(uint32_t bar, unsigned parity)
{
    for (unsigned it = 0; it < kTcWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, float (&v)[4])
{
    unsigned r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// Copy the FP16 forward weights into their K-major tiles (W4 padded to 16
// rows) and the biases, 16-byte chunks; every thread of the CTA takes part.
__device__ __forceinline__ void tc_load_weights(const __half *hw, const float *params, unsigned char *sm)
{
    for (int i = threadIdx.x; i < MLP_W * (MLP_IN / 8); i += blockDim.x) {
        const int n = i / (MLP_IN / 8), c = i % (MLP_IN / 8);
        *reinterpret_cast<uint4 *>(sm + tc_off(n, 8 * c, kTcLboW)) =
            __ldg(reinterpret_cast<const uint4 *>(hw + H_T1 + n * MLP_IN + 8 * c));
    }
    for (int i = threadIdx.x; i < MLP_W * (MLP_W / 8); i += blockDim.x) {
        const int n = i / (MLP_W / 8), c = i % (MLP_W / 8);
        *reinterpret_cast<uint4 *>(sm + kTcOffW2 + tc_off(n, 8 * c, kTcLboW)) =
            __ldg(reinterpret_cast<const uint4 *>(hw + H_T2 + n * MLP_W + 8 * c));
        *reinterpret_cast<uint4 *>(sm + kTcOffW3 + tc_off(n, 8 * c, kTcLboW)) =
            __ldg(reinterpret_cast<const uint4 *>(hw + H_T3 + n * MLP_W + 8 * c));
    }
    for (int i = threadIdx.x; i < 16 * (MLP_W / 8); i += blockDim.x) {
        const int n = i / (MLP_W / 8), c = i % (MLP_W / 8);
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(sm + kTcOffW4 + tc_off(n, 8 * c, kTcLboW4)) =
            n < 8 ? __ldg(reinterpret_cast<const uint4 *>(hw + H_T4 + n * MLP_W + 8 * c)) : z;
    }
    float *bias = reinterpret_cast<float *>(sm + kTcOffBias);
    for (int i = threadIdx.x; i < 3 * MLP_W + 4; i += blockDim.x) {
        float b = 0.0f;
        if (i < MLP_W) b = params[P_B1 + i];
        else if (i < 2 * MLP_W) b = params[P_B2 + i - MLP_W];
        else if (i < 3 * MLP_W) b = params[P_B3 + i - 2 * MLP_W];
        else if (i - 3 * MLP_W < MLP_OUT) b = params[P_B4 + i - 3 * MLP_W];
        bias[i] = b;
    }
}

// The 224 inputs of one ray into row `row` of the activation tile (K-major):
// half_id 0 writes scalars 0-2 (k 0..95) and grid samples 0-15 (k 192..207),
// half_id 1 scalars 3-5 and samples 16-31 -- the values ray_features_half
// computes, in the same order, eight per 16-byte store.
__device__ __forceinline__ void ray_features_tc(const RayRec &r, float step, const float *grid, int cell,
                                                int gx, int gy, int gz, float nx, float ny, float nz,
                                                int half_id, unsigned char *tile, int row)
{
    const float s6[6] = {r.ex / nx, r.ey / ny, r.ez / nz, r.dx, r.dy, r.dz};
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        const int j = half_id * 3 + jj;
        __half2 v[MLP_NFREQ];   // (sin, cos) of frequency k
#pragma unroll
        for (int chain = 0; chain < 2; ++chain) {
            float sv, cv;
            sincospif(s6[j] * c_freq2[chain], &sv, &cv);
#pragma unroll
            for (int k = chain; k < MLP_NFREQ; k += 2) {
                v[k] = __halves2half2(__float2half_rn(sv), __float2half_rn(cv));
                const float s2 = 2.0f * sv * cv;
                cv = (cv - sv) * (cv + sv);
                sv = s2;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // k-chunk j*4 + q: frequencies 4q .. 4q+3
            uint4 w;
            w.x = *reinterpret_cast<const unsigned *>(&v[4 * q]);
            w.y = *reinterpret_cast<const unsigned *>(&v[4 * q + 1]);
            w.z = *reinterpret_cast<const unsigned *>(&v[4 * q + 2]);
            w.w = *reinterpret_cast<const unsigned *>(&v[4 * q + 3]);
            *reinterpret_cast<uint4 *>(tile + tc_off(row, (j * 4 + q) * 8, kTcLboX)) = w;
        }
    }
    const float L = (float)r.nsteps * step;
    const float inv_cell = 1.0f / (float)cell;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        __half h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = half_id * (MLP_NGRID / 2) + q * 8 + e;
            const float tt = ((float)i + 0.5f) * (1.0f / MLP_NGRID) * L;
            const int cx = min(max((int)floorf(fmaf(tt, r.dx, r.ex) * inv_cell), 0), gx - 1);
            const int cy = min(max((int)floorf(fmaf(tt, r.dy, r.ey) * inv_cell), 0), gy - 1);
            const int cz = min(max((int)floorf(fmaf(tt, r.dz, r.ez) * inv_cell), 0), gz - 1);
            h[e] = __float2half_rn(__ldg(grid + ((long long)cz * gy + cy) * gx + cx));
        }
        *reinterpret_cast<uint4 *>(tile + tc_off(row, 6 * 2 * MLP_NFREQ + (half_id * 2 + q) * 8, kTcLboX)) =
            *reinterpret_cast<const uint4 *>(h);
    }
}

struct TcState {
    uint32_t tmem;       // TMEM base address of the CTA's accumulator columns
    uint32_t bar;        // shared address of the mbarrier
    unsigned phase;      // completed phases of the mbarrier
};

// CTA start: mbarrier, TMEM allocation (warp 0), weights.  Ends with a CTA barrier.
__device__ __forceinline__ TcState tc_begin(const __half *hw, const float *params, unsigned char *sm)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kTcOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kTcOffBar + 8);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_load_weights(hw, params, sm);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    TcState s;
    s.tmem = *reinterpret_cast<volatile uint32_t *>(tslot);
    s.bar = smem_u32(bar);
    s.phase = 0;
    return s;
}

// CTA end: free the TMEM columns (warp 0) once no thread reads them.
__device__ __forceinline__ void tc_end(const TcState &s)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s.tmem), "r"(kTcCols)
                     : "memory");
}

// Issue one layer (thread 0) and wait for it (every thread).  A: the
// activation tile with k_in columns; B: a weight tile of n rows.
__device__ __forceinline__ bool tc_layer(TcState &s, const unsigned char *a_tile, const unsigned char *b_tile,
                                         int k_in, int n, int lbo_b)
{
    if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(a_tile), b0 = smem_u32(b_tile);
        const uint32_t idesc = tc_idesc(kTcRows, n);
        for (int ks = 0; ks < k_in / 16; ++ks)
            tc_mma(s.tmem, tc_desc(a0 + 2 * ks * kTcLboX, kTcLboX, 128), tc_desc(b0 + 2 * ks * lbo_b, lbo_b, 128),
                   idesc, ks > 0);
        tc_commit(s.bar);
    }
    const bool ok = tc_wait(s.bar, s.phase & 1u);
    s.phase += 1;
    tc_fence_after();
    return ok;
}

// Hidden-layer epilogue: bias + ReLU of the accumulators, FP16, into the
// activation tile as the next layer's operand (64 columns); then the CTA
// barrier that hands the tile to the tensor cores.
__device__ __forceinline__ void tc_hidden_epilogue(const TcState &s, unsigned char *tile, const float *bias)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);
    float v[32];
    tc_ld32(s.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __half2 h[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            h[e] = __floats2half2_rn(fmaxf(v[8 * q + 2 * e] + bias[c0 + 8 * q + 2 * e], 0.0f),
                                     fmaxf(v[8 * q + 2 * e + 1] + bias[c0 + 8 * q + 2 * e + 1], 0.0f));
        *reinterpret_cast<uint4 *>(tile + tc_off(row, c0 + 8 * q, kTcLboX)) = *reinterpret_cast<const uint4 *>(h);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
}

// The whole network on the tile whose inputs are in place (after a CTA
// barrier that follows fence_async_smem): returns false if a wait ran out.
// Threads 0..127 then hold u of row threadIdx.x in u[0..2].
__device__ __forceinline__ bool tc_forward_tile(TcState &s, unsigned char *sm, float (&u)[4])
{
    unsigned char *tile = sm + kTcOffX;
    const float *bias = reinterpret_cast<const float *>(sm + kTcOffBias);
    bool ok = tc_layer(s, tile, sm, MLP_IN, MLP_W, kTcLboW);
    if (__syncthreads_and(ok)) tc_hidden_epilogue(s, tile, bias);
    else return false;
    ok = tc_layer(s, tile, sm + kTcOffW2, MLP_W, MLP_W, kTcLboW);
    if (__syncthreads_and(ok)) tc_hidden_epilogue(s, tile, bias + MLP_W);
    else return false;
    ok = tc_layer(s, tile, sm + kTcOffW3, MLP_W, MLP_W, kTcLboW);
    if (__syncthreads_and(ok)) tc_hidden_epilogue(s, tile, bias + 2 * MLP_W);
    else return false;
    ok = tc_layer(s, tile, sm + kTcOffW4, MLP_W, 16, kTcLboW4);
    if (!__syncthreads_and(ok)) return false;
    if (threadIdx.x < kTcRows) {
        const int warp = threadIdx.x >> 5;
        tc_ld4(s.tmem + ((uint32_t)(32 * warp) << 16), u);
        u[0] += bias[3 * MLP_W];
        u[1] += bias[3 * MLP_W + 1];
        u[2] += bias[3 * MLP_W + 2];
    }
    return true;
}

}  // namespace isaac
