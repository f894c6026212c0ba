// mlp.cu -- kernels and entry points of the learned ray-interval proposal:
// FP16 weight copy, input features, forward pass, one fused forward+backward
// training pass with gradient accumulation, Adam.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.h"
#include "mlp.cuh"
#include "mlp_tc.cuh"

namespace isaac {

constexpr float kHuberDelta = 0.02f, kConfWeight = 0.1f;

// ----------------------------------------------------------- FP16 copy

static __global__ void k_mlp_half(const float *__restrict__ p, __half *__restrict__ h)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_HALF; i += gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (i < H_T2) {                       // T1[n][k] = W1[k][n]
            const int n = i / MLP_IN, k = i % MLP_IN;
            v = p[P_W1 + k * MLP_W + n];
        } else if (i < H_T3) {
            const int j = i - H_T2, n = j / MLP_W, k = j % MLP_W;
            v = p[P_W2 + k * MLP_W + n];
        } else if (i < H_T4) {
            const int j = i - H_T3, n = j / MLP_W, k = j % MLP_W;
            v = p[P_W3 + k * MLP_W + n];
        } else if (i < H_B2) {                // T4[n][k] = W4[k][n], n < 3
            const int j = i - H_T4, n = j / MLP_W, k = j % MLP_W;
            v = n < MLP_OUT ? p[P_W4 + k * MLP_OUT + n] : 0.0f;
        } else if (i < H_B3) {
            v = p[P_W2 + (i - H_B2)];
        } else if (i < H_B4) {
            v = p[P_W3 + (i - H_B3)];
        } else {                              // B4[in][o] = W4[in][o], o < 3
            const int j = i - H_B4, in = j / 16, o = j % 16;
            v = o < MLP_OUT ? p[P_W4 + in * MLP_OUT + o] : 0.0f;
        }
        h[i] = __float2half_rn(v);
    }
}

// ------------------------------------------------------------ features

struct KFeat {
    const RayRec *rays;
    long long n;
    float step;
    const float *grid;
    int cell, gx, gy, gz;
    float nx, ny, nz;
    __half *X;
};

static __global__ void k_mlp_features(const __grid_constant__ KFeat p)
{
    const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 1;
    if (i >= p.n) return;
    const RayRec r = p.rays[i];
    ray_features_half(r, p.step, p.grid, p.cell, p.gx, p.gy, p.gz, p.nx, p.ny, p.nz, threadIdx.x & 1,
                      p.X + i * MLP_IN);
}

// ---------------------------------------------------------------- forward

struct KFwd {
    const __half *hw;
    const float *params;
    const __half *X;
    long long n;
    float *U;
};

// Inference on the tensor cores (tcgen05): persistent CTAs take tiles of 128
// rays; the inputs of a tile are copied into its K-major activation tile, the
// network runs as in tc_forward_tile, and threads 0..127 write the outputs of
// their row.  A tile whose tensor-core wait ran out (and every later tile of
// the CTA) gets NaN outputs.
static __global__ void __launch_bounds__(kTcThreads) k_mlp_forward(const __grid_constant__ KFwd p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcState s = tc_begin(p.hw, p.params, smem_raw);
    unsigned char *tile = smem_raw + kTcOffX;
    long long base = blockIdx.x * (long long)kTcRows;
    bool alive = true;
    for (; base < p.n; base += gridDim.x * (long long)kTcRows) {
        for (int i = threadIdx.x; i < kTcRows * (MLP_IN / 8); i += blockDim.x) {
            const int row = i / (MLP_IN / 8), c = i % (MLP_IN / 8);
            const long long r = base + row;
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            if (r < p.n) {   // X is 4-byte aligned: four 4-byte loads per 8 inputs
                const unsigned *src = reinterpret_cast<const unsigned *>(p.X + r * MLP_IN + 8 * c);
                w = make_uint4(__ldg(src), __ldg(src + 1), __ldg(src + 2), __ldg(src + 3));
            }
            *reinterpret_cast<uint4 *>(tile + tc_off(row, 8 * c, kTcLboX)) = w;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        float u[4];
        if (!tc_forward_tile(s, smem_raw, u)) {
            alive = false;
            break;
        }
        const long long r = base + threadIdx.x;
        if (threadIdx.x < kTcRows && r < p.n)
            for (int j = 0; j < MLP_OUT; ++j) p.U[r * MLP_OUT + j] = u[j];
    }
    if (!alive) {
        tc_wait(s.bar, (s.phase - 1u) & 1u);   // let an MMA still in flight finish (bounded)
        const float nan = __int_as_float(0x7fc00000);
        for (; base < p.n; base += gridDim.x * (long long)kTcRows) {
            const long long r = base + threadIdx.x;
            if (threadIdx.x < kTcRows && r < p.n)
                for (int j = 0; j < MLP_OUT; ++j) p.U[r * MLP_OUT + j] = nan;
        }
    }
    tc_end(s);
}

// ---------------------------------------------------------------- training

struct KTrain {
    const __half *hw;
    const float *params;
    float *part;              // per block: kPartStride floats (gradient partial sums, then the loss)
    const __half *X;
    const RayRec *rays;       // jf, jl, nsteps of every training ray
    long long n;
    float inv_n;
    int margin;
};

// The batch gradient is reduced in a fixed order, so a training run is
// bitwise reproducible (and a resumed run equals an uninterrupted one): block
// b of at most kTrainBlocks takes the 64-ray tiles b, b + G, ... and sums
// their gradients, in that order, into its own slot of kPartStride floats
// (no atomics); k_mlp_reduce then adds the G slots in block order.  The grid
// size depends on the batch size only, not on the device.
constexpr int kTrainBlocks = 148;
constexpr int kPartStride = ((N_PARAMS + 1 + 3) / 4) * 4;   // + the loss, 16-byte rows

constexpr int kTrainSmemHalves = MLP_W * LD_IN + 2 * MLP_W * LD_W + 8 * LD_W   // forward weights
                                 + 2 * MLP_W * LD_W + MLP_W * LD_B4             // backward weights
                                 + 64 * LD_IN + MLP_IN * LD_R                   // X, X^T
                                 + 6 * MLP_W * LD_R + 8 * LD_R;                 // h^T, dA^T tiles
constexpr int kTrainSmemBytes = kTrainSmemHalves * 2 + 4 * 64 * 4;

__device__ __forceinline__ float sigmoidf(float x) { return 1.0f / (1.0f + __expf(-x)); }

__device__ __forceinline__ float dhuber(float r)
{
    return fabsf(r) < kHuberDelta ? r / kHuberDelta : (r > 0.0f ? 1.0f : (r < 0.0f ? -1.0f : 0.0f));
}

__device__ __forceinline__ float huberf(float r)
{
    const float a = fabsf(r);
    return a < kHuberDelta ? 0.5f * r * r / kHuberDelta : a - 0.5f * kHuberDelta;
}

// Per-ray output gradient (without the 1/N of the batch mean) and loss.
__device__ __forceinline__ void ray_grad(float u0, float u1, float u2, int jf, int jl, int ns,
                                         int margin, bool valid, float &d0, float &d1, float &d2,
                                         float &loss)
{
    d0 = d1 = d2 = loss = 0.0f;
    if (!valid) return;
    const float te = sigmoidf(u0), tx = sigmoidf(u1), conf = sigmoidf(u2);
    const bool empty = jf < 0;
    const float ye = empty ? 1.0f : (float)jf / (float)ns;
    const float yx = empty ? 0.0f : (float)(jl + 1) / (float)ns;
    float c = 1.0f;
    if (!empty) {
        const float kb = floorf(te * (float)ns) - (float)margin;
        const float ke = ceilf(tx * (float)ns) + (float)margin;
        c = (kb <= (float)jf && ke >= (float)(jl + 1)) ? 1.0f : 0.0f;
    }
    d0 = dhuber(te - ye) * te * (1.0f - te);
    d1 = dhuber(tx - yx) * tx * (1.0f - tx);
    d2 = kConfWeight * (conf - c);
    const float bce = -(c * __logf(fmaxf(conf, 1e-30f)) + (1.0f - c) * __logf(fmaxf(1.0f - conf, 1e-30f)));
    loss = huberf(te - ye) + huberf(tx - yx) + kConfWeight * bce;
}

// dA of one layer: (dA_next . W^T) masked by the layer's ReLU; returns the
// accumulators and stores them transposed (output-major) for the weight grads.
__device__ __forceinline__ void backward_layer(const unsigned (&A)[4][4], int ksteps, const __half *bt,
                                               int ldb, unsigned mask, float (&c)[8][4],
                                               __half *dt, int col0)
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
        for (int ks = 0; ks < ksteps; ++ks) {
            unsigned b[2];
            frag_b(bt, ldb, nt * 8, ks * 16, b);
            mma16816(c[nt], A[ks], b);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (!((mask >> (nt * 4 + j)) & 1u)) c[nt][j] = 0.0f;
        const int f = nt * 8 + 2 * t;
        dt[f * LD_R + col0 + g] = __float2half_rn(c[nt][0]);
        dt[(f + 1) * LD_R + col0 + g] = __float2half_rn(c[nt][1]);
        dt[f * LD_R + col0 + g + 8] = __float2half_rn(c[nt][2]);
        dt[(f + 1) * LD_R + col0 + g + 8] = __float2half_rn(c[nt][3]);
    }
}

static __global__ void __launch_bounds__(128) k_mlp_train(const __grid_constant__ KTrain p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __half *sT1 = reinterpret_cast<__half *>(smem_raw);
    __half *sT2 = sT1 + MLP_W * LD_IN, *sT3 = sT2 + MLP_W * LD_W, *sT4 = sT3 + MLP_W * LD_W;
    __half *sB2 = sT4 + 8 * LD_W, *sB3 = sB2 + MLP_W * LD_W, *sB4 = sB3 + MLP_W * LD_W;
    __half *xs = sB4 + MLP_W * LD_B4, *xt = xs + 64 * LD_IN;
    __half *h1t = xt + MLP_IN * LD_R, *h2t = h1t + MLP_W * LD_R, *h3t = h2t + MLP_W * LD_R;
    __half *d1t = h3t + MLP_W * LD_R, *d2t = d1t + MLP_W * LD_R, *d3t = d2t + MLP_W * LD_R;
    __half *d4t = d3t + MLP_W * LD_R;
    int *s_jf = reinterpret_cast<int *>(d4t + 8 * LD_R), *s_jl = s_jf + 64, *s_ns = s_jl + 64;
    float *s_loss = reinterpret_cast<float *>(s_ns + 64);

    load_weights_smem(p.hw, sT1, sT2, sT3, sT4, sB2, sB3, sB4);
    float *part = p.part + (size_t)blockIdx.x * kPartStride;
    const long long tiles = (p.n + 63) / 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int col0 = warp * 16;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const bool first = tile == blockIdx.x;   // the block's first tile stores, later ones add
        const long long base = tile * 64;
        for (int i = threadIdx.x; i < 64 * MLP_IN; i += blockDim.x) {
            const int rr = i / MLP_IN, k = i % MLP_IN;
            const long long r = base + rr;
            const __half v = r < p.n ? p.X[r * MLP_IN + k] : __float2half_rn(0.0f);
            xs[rr * LD_IN + k] = v;
            xt[k * LD_R + rr] = v;
        }
        for (int i = threadIdx.x; i < 8 * LD_R; i += blockDim.x) d4t[i] = __float2half_rn(0.0f);
        if (threadIdx.x < 64) {
            const long long r = base + threadIdx.x;
            const bool ok = r < p.n;
            s_jf[threadIdx.x] = ok ? p.rays[r].jf : -1;
            s_jl[threadIdx.x] = ok ? p.rays[r].jl : -1;
            s_ns[threadIdx.x] = ok ? p.rays[r].nsteps : 0;
        }
        __syncthreads();

        Hidden hid;
        float u[4];
        mlp_forward_warp(xs, col0, sT1, sT2, sT3, sT4, p.params, u, &hid, h1t, h2t, h3t, col0);

        // output gradient of rays col0+g and col0+g+8 (computed on lanes t == 0)
        const float u2a = __shfl_down_sync(0xffffffffu, u[0], 1), u2b = __shfl_down_sync(0xffffffffu, u[2], 1);
        float da[3] = {0, 0, 0}, db[3] = {0, 0, 0}, la = 0.0f, lb = 0.0f;
        if (t == 0) {
            const int ra = col0 + g, rb = ra + 8;
            ray_grad(u[0], u[1], u2a, s_jf[ra], s_jl[ra], s_ns[ra], p.margin, base + ra < p.n, da[0],
                     da[1], da[2], la);
            ray_grad(u[2], u[3], u2b, s_jf[rb], s_jl[rb], s_ns[rb], p.margin, base + rb < p.n, db[0],
                     db[1], db[2], lb);
            for (int o = 0; o < 3; ++o) {
                d4t[o * LD_R + ra] = __float2half_rn(da[o]);
                d4t[o * LD_R + rb] = __float2half_rn(db[o]);
            }
            s_loss[ra] = la;
            s_loss[rb] = lb;
        }
        const float da2 = __shfl_up_sync(0xffffffffu, da[2], 1), db2 = __shfl_up_sync(0xffffffffu, db[2], 1);
        unsigned A4[4][4];
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) A4[j][q] = 0u;
        if (t == 0) {
            A4[0][0] = pack_h2(da[0], da[1]);
            A4[0][1] = pack_h2(db[0], db[1]);
        } else if (t == 1) {
            A4[0][0] = pack_h2(da2, 0.0f);
            A4[0][1] = pack_h2(db2, 0.0f);
        }
        float c[8][4];
        unsigned A[4][4];
        backward_layer(A4, 1, sB4, LD_B4, hid.m3, c, d3t, col0);        // dA3
        for (int j = 0; j < 4; ++j) acc_to_a(c[2 * j], c[2 * j + 1], A[j]);
        backward_layer(A, 4, sB3, LD_W, hid.m2, c, d2t, col0);          // dA2
        for (int j = 0; j < 4; ++j) acc_to_a(c[2 * j], c[2 * j + 1], A[j]);
        backward_layer(A, 4, sB2, LD_W, hid.m1, c, d1t, col0);          // dA1
        __syncthreads();

        // weight gradients over the tile's 64 rays: dW = H^T . dA (jobs = m-tiles)
        // layer 4: 4 m-tiles x 1 n-tile, layers 3, 2: 4 x 8, layer 1: 14 x 8;
        // every element of the block's slot has one owner thread, the same for
        // every tile, so the slot is updated without atomics
        for (int job = warp; job < 26; job += 4) {
            const __half *at, *bt;
            int mt, nts, wo, out_dim;
            if (job < 4) {
                at = h3t; bt = d4t; mt = job; nts = 1; wo = P_W4; out_dim = MLP_OUT;
            } else if (job < 8) {
                at = h2t; bt = d3t; mt = job - 4; nts = 8; wo = P_W3; out_dim = MLP_W;
            } else if (job < 12) {
                at = h1t; bt = d2t; mt = job - 8; nts = 8; wo = P_W2; out_dim = MLP_W;
            } else {
                at = xt; bt = d1t; mt = job - 12; nts = 8; wo = P_W1; out_dim = MLP_W;
            }
            float acc[8][4];
            for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
            for (int ks = 0; ks < 4; ++ks) {
                unsigned a[4];
                frag_a(at, LD_R, mt * 16, ks * 16, a);
                for (int nt = 0; nt < nts; ++nt) {
                    unsigned b[2];
                    frag_b(bt, LD_R, nt * 8, ks * 16, b);
                    mma16816(acc[nt], a, b);
                }
            }
            for (int nt = 0; nt < nts; ++nt)
                for (int j = 0; j < 4; ++j) {
                    const int in = mt * 16 + g + (j >= 2 ? 8 : 0);
                    const int out = nt * 8 + 2 * t + (j & 1);
                    if (out < out_dim) {
                        float *dst = part + wo + in * out_dim + out;
                        const float v = acc[nt][j] * p.inv_n;
                        *dst = first ? v : *dst + v;
                    }
                }
        }
        // bias gradients: sum of dA over the tile's rays, in ray order
        for (int o = threadIdx.x; o < 3 * MLP_W + MLP_OUT; o += blockDim.x) {
            const __half *row;
            int bo;
            if (o < MLP_W) { row = d1t + o * LD_R; bo = P_B1 + o; }
            else if (o < 2 * MLP_W) { row = d2t + (o - MLP_W) * LD_R; bo = P_B2 + o - MLP_W; }
            else if (o < 3 * MLP_W) { row = d3t + (o - 2 * MLP_W) * LD_R; bo = P_B3 + o - 2 * MLP_W; }
            else { row = d4t + (o - 3 * MLP_W) * LD_R; bo = P_B4 + o - 3 * MLP_W; }
            float sum = 0.0f;
            for (int r = 0; r < 64; ++r) sum += __half2float(row[r]);
            const float v = sum * p.inv_n;
            part[bo] = first ? v : part[bo] + v;
        }
        // the tile's loss, in ray order
        if (threadIdx.x == blockDim.x - 1) {
            float sum = 0.0f;
            for (int r = 0; r < 64; ++r) sum += s_loss[r];
            const float v = sum * p.inv_n;
            part[N_PARAMS] = first ? v : part[N_PARAMS] + v;
        }
        __syncthreads();   // the next tile overwrites the shared tiles
    }
}

// Batch gradient (and loss) = the blocks' slots added in block order.
static __global__ void k_mlp_reduce(const float *__restrict__ part, int blocks, float *grads,
                                    float *loss_sum)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= N_PARAMS; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < blocks; ++b) s += part[(size_t)b * kPartStride + i];
        if (i < N_PARAMS) grads[i] = s;
        else if (loss_sum) *loss_sum += s;
    }
}

// ------------------------------------------------------------------- Adam

static __global__ void k_adam(float *p, const float *g, float *m, float *v, float lr, float b1,
                              float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_PARAMS; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace isaac

using namespace isaac;

static int check_model(const isaac_mlp *m, bool train)
{
    if (!m || !m->params || !m->half_w) return fail(ISAAC_EINVAL, "model params and half_w are required");
    if (train && (!m->grads || !m->adam_m || !m->adam_v))
        return fail(ISAAC_EINVAL, "training needs grads, adam_m and adam_v");
    if (((uintptr_t)m->half_w) % 16 || ((uintptr_t)m->params) % 16)
        return fail(ISAAC_EINVAL, "model buffers must be 16-byte aligned");
    return ISAAC_OK;
}

// ------------------------------------------------- create, checkpoint, destroy

namespace {

// Base pointers of the blocks isaac_mlp_create allocated (isaac_mlp_destroy
// frees only those).
std::mutex g_created_mu;
std::vector<void *> g_created;

constexpr size_t kParamFloats = ((N_PARAMS + 3) / 4) * 4;   // 16-byte aligned arrays

// CRC-32 (reflected, polynomial 0xEDB88320, initial and final XOR ~0: the
// checksum of zlib and PNG), table-driven.
uint32_t crc32_bytes(const unsigned char *b, size_t n)
{
    static uint32_t table[256];
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
    });
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; ++i) c = table[(c ^ b[i]) & 0xFFu] ^ (c >> 8);
    return c ^ 0xFFFFFFFFu;
}

// SplitMix64 (Steele, Lea and Flood 2014): the seeded stream of the initial weights.
uint64_t splitmix64(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct CkptHeader {
    char magic[8];        // "ISAACMLP"
    uint32_t version;     // 1
    uint32_t count;       // ISAAC_MLP_PARAMS
    int32_t step;
    uint32_t flags;       // bit 0: Adam moments follow the parameters
    uint64_t tag;
    uint32_t crc;         // CRC-32 of everything after the header
    unsigned char pad[ISAAC_MLP_CKPT_HEADER - 36];
};
static_assert(sizeof(CkptHeader) == ISAAC_MLP_CKPT_HEADER, "checkpoint header layout");

}  // namespace

extern "C" int64_t isaac_mlp_checkpoint_bytes(int32_t with_adam)
{
    return (int64_t)ISAAC_MLP_CKPT_HEADER + (int64_t)(with_adam ? 3 : 1) * N_PARAMS * 4;
}

extern "C" int isaac_mlp_create(isaac_mlp *m, int32_t train, uint64_t seed, void *stream)
{
    clear_error();
    if (!m) return fail(ISAAC_EINVAL, "model is required");
    const size_t floats = kParamFloats * (train ? 4 : 1);
    const size_t bytes = floats * sizeof(float) + (size_t)N_HALF * sizeof(__half);
    void *base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ISAAC_ENOMEM, "cannot allocate %zu bytes for the model", bytes);
    }
    // He-uniform weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)), zero biases
    std::vector<float> init(N_PARAMS, 0.0f);
    uint64_t state = seed;
    const int layers[4][3] = {{P_W1, MLP_IN, MLP_W}, {P_W2, MLP_W, MLP_W}, {P_W3, MLP_W, MLP_W},
                              {P_W4, MLP_W, MLP_OUT}};
    for (const auto &L : layers) {
        const double lim = std::sqrt(6.0 / (double)L[1]);
        for (int i = 0; i < L[1] * L[2]; ++i) {
            const double u = (double)(splitmix64(state) >> 11) * 0x1.0p-53;
            init[L[0] + i] = (float)((2.0 * u - 1.0) * lim);
        }
    }
    const cudaStream_t st = (cudaStream_t)stream;
    float *f = static_cast<float *>(base);
    isaac_mlp out;
    out.params = f;
    out.grads = train ? f + kParamFloats : nullptr;
    out.adam_m = train ? f + 2 * kParamFloats : nullptr;
    out.adam_v = train ? f + 3 * kParamFloats : nullptr;
    out.half_w = reinterpret_cast<uint16_t *>(f + floats);
    out.step = 0;
    if (cudaMemsetAsync(base, 0, floats * sizeof(float), st) != cudaSuccess ||
        cudaMemcpyAsync(out.params, init.data(), N_PARAMS * sizeof(float), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {   // `init` is a pageable host vector
        const int rc = check_cuda("isaac_mlp_create (initial weights)");
        cudaFree(base);
        return rc;
    }
    k_mlp_half<<<64, 256, 0, st>>>(out.params, reinterpret_cast<__half *>(out.half_w));
    const int rc = check_cuda("isaac_mlp_create");
    if (rc) {
        cudaFree(base);
        return rc;
    }
    {
        std::lock_guard<std::mutex> lock(g_created_mu);
        g_created.push_back(base);
    }
    *m = out;
    return ISAAC_OK;
}

extern "C" int isaac_mlp_destroy(isaac_mlp *m)
{
    clear_error();
    if (!m) return fail(ISAAC_EINVAL, "model is required");
    {
        std::lock_guard<std::mutex> lock(g_created_mu);
        auto it = std::find(g_created.begin(), g_created.end(), static_cast<void *>(m->params));
        if (it == g_created.end())
            return fail(ISAAC_EINVAL, "the model's buffers were not allocated by isaac_mlp_create");
        g_created.erase(it);
    }
    cudaFree(m->params);
    memset(m, 0, sizeof *m);
    return check_cuda("isaac_mlp_destroy");
}

extern "C" int isaac_mlp_save(const isaac_mlp *m, uint64_t tag, void *image, int64_t bytes,
                              void *stream)
{
    clear_error();
    if (!m || !m->params || !image) return fail(ISAAC_EINVAL, "model params and image are required");
    const bool adam = m->adam_m && m->adam_v;
    const int64_t need = isaac_mlp_checkpoint_bytes(adam ? 1 : 0);
    if (bytes < need)
        return fail(ISAAC_ENOMEM, "the image holds %lld bytes, the checkpoint needs %lld",
                    (long long)bytes, (long long)need);
    unsigned char *out = static_cast<unsigned char *>(image);
    float *payload = reinterpret_cast<float *>(out + ISAAC_MLP_CKPT_HEADER);
    const cudaStream_t st = (cudaStream_t)stream;
    // stream-ordered after the caller's training steps; the image is complete
    // when the call returns
    const float *src[3] = {m->params, m->adam_m, m->adam_v};
    for (int k = 0; k < (adam ? 3 : 1); ++k)
        if (cudaMemcpyAsync(payload + (size_t)k * N_PARAMS, src[k], N_PARAMS * sizeof(float),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return check_cuda("isaac_mlp_save (copy)");
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda("isaac_mlp_save (sync)");
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "ISAACMLP", 8);
    h.version = 1;
    h.count = N_PARAMS;
    h.step = m->step;
    h.flags = adam ? 1u : 0u;
    h.tag = tag;
    h.crc = crc32_bytes(out + ISAAC_MLP_CKPT_HEADER, (size_t)(need - ISAAC_MLP_CKPT_HEADER));
    memcpy(out, &h, sizeof h);
    return ISAAC_OK;
}

extern "C" int isaac_mlp_load(isaac_mlp *m, const void *image, int64_t bytes, uint64_t *tag,
                              void *stream)
{
    clear_error();
    if (!m || !image) return fail(ISAAC_EINVAL, "model and image are required");
    if (bytes < ISAAC_MLP_CKPT_HEADER) return fail(ISAAC_EINVAL, "image shorter than the header");
    CkptHeader h;
    memcpy(&h, image, sizeof h);
    if (memcmp(h.magic, "ISAACMLP", 8) != 0) return fail(ISAAC_EINVAL, "not a proposal-network checkpoint");
    if (h.version != 1) return fail(ISAAC_EINVAL, "checkpoint version %u (1 expected)", h.version);
    if (h.count != (uint32_t)N_PARAMS)
        return fail(ISAAC_EINVAL, "checkpoint holds %u parameters (%d expected)", h.count, N_PARAMS);
    const bool adam = (h.flags & 1u) != 0;
    if (h.flags & ~1u) return fail(ISAAC_EINVAL, "unknown checkpoint flags 0x%x", h.flags);
    const int64_t need = isaac_mlp_checkpoint_bytes(adam ? 1 : 0);
    if (bytes < need)
        return fail(ISAAC_EINVAL, "checkpoint truncated: %lld of %lld bytes", (long long)bytes,
                    (long long)need);
    const unsigned char *in = static_cast<const unsigned char *>(image);
    if (crc32_bytes(in + ISAAC_MLP_CKPT_HEADER, (size_t)(need - ISAAC_MLP_CKPT_HEADER)) != h.crc)
        return fail(ISAAC_EINVAL, "checkpoint checksum mismatch (corrupt image)");
    int rc = check_model(m, false);
    if (rc) return rc;
    const float *payload = reinterpret_cast<const float *>(in + ISAAC_MLP_CKPT_HEADER);
    const cudaStream_t st = (cudaStream_t)stream;
    const bool model_adam = m->adam_m && m->adam_v;
    if (cudaMemcpyAsync(m->params, payload, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return check_cuda("isaac_mlp_load (parameters)");
    if (model_adam) {
        // Adam state from the image, or a fresh optimiser (zero moments, step 0)
        for (int k = 0; k < 2; ++k) {
            float *dst = k ? m->adam_v : m->adam_m;
            const cudaError_t e = adam
                ? cudaMemcpyAsync(dst, payload + (size_t)(k + 1) * N_PARAMS, N_PARAMS * sizeof(float),
                                  cudaMemcpyHostToDevice, st)
                : cudaMemsetAsync(dst, 0, N_PARAMS * sizeof(float), st);
            if (e != cudaSuccess) return check_cuda("isaac_mlp_load (Adam state)");
        }
    }
    k_mlp_half<<<64, 256, 0, st>>>(m->params, reinterpret_cast<__half *>(m->half_w));
    // the image may be pageable memory the caller frees after the call
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda("isaac_mlp_load (sync)");
    m->step = model_adam && adam ? h.step : 0;
    if (tag) *tag = h.tag;
    return check_cuda("isaac_mlp_load");
}

extern "C" int isaac_mlp_sync(const isaac_mlp *m, void *stream)
{
    clear_error();
    int rc = check_model(m, false);
    if (rc) return rc;
    k_mlp_half<<<64, 256, 0, (cudaStream_t)stream>>>(m->params, reinterpret_cast<__half *>(m->half_w));
    return check_cuda("isaac_mlp_sync");
}

extern "C" int isaac_mlp_features(const isaac_ray *rays, int64_t n_rays, const int64_t vol_n[3],
                                  float step, const float *grid, int32_t cell, uint16_t *X,
                                  void *stream)
{
    clear_error();
    if (n_rays < 0 || (n_rays > 0 && (!rays || !grid || !X || !vol_n)))
        return fail(ISAAC_EINVAL, "rays, grid, X and vol_n are required");
    if (cell < 1 || !(step > 0.0f)) return fail(ISAAC_EINVAL, "cell and step must be positive");
    if (n_rays == 0) return ISAAC_OK;
    if (((uintptr_t)X) % 4) return fail(ISAAC_EINVAL, "X must be 4-byte aligned");
    KFeat p;
    p.rays = reinterpret_cast<const RayRec *>(rays);
    p.n = n_rays;
    p.step = step;
    p.grid = grid;
    p.cell = cell;
    p.gx = (int)((vol_n[0] + cell - 1) / cell);
    p.gy = (int)((vol_n[1] + cell - 1) / cell);
    p.gz = (int)((vol_n[2] + cell - 1) / cell);
    p.nx = (float)vol_n[0];
    p.ny = (float)vol_n[1];
    p.nz = (float)vol_n[2];
    p.X = reinterpret_cast<__half *>(X);
    const long long threads = 2 * n_rays;
    k_mlp_features<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(p);
    return check_cuda("isaac_mlp_features");
}

extern "C" int isaac_mlp_forward(const isaac_mlp *m, const uint16_t *X, int64_t n_rays, float *U,
                                 void *stream)
{
    clear_error();
    int rc = check_model(m, false);
    if (rc) return rc;
    if (n_rays <= 0) return n_rays == 0 ? ISAAC_OK : fail(ISAAC_EINVAL, "negative ray count");
    if (!X || !U || ((uintptr_t)X) % 4) return fail(ISAAC_EINVAL, "X (4-byte aligned) and U are required");
    KFwd p;
    p.hw = reinterpret_cast<const __half *>(m->half_w);
    p.params = m->params;
    p.X = reinterpret_cast<const __half *>(X);
    p.n = n_rays;
    p.U = U;
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
    const long long blocks = std::min<long long>((n_rays + kTcRows - 1) / kTcRows, (long long)sm_count() * 2);
    k_mlp_forward<<<(unsigned)blocks, kTcThreads, kTcSmemBytes, (cudaStream_t)stream>>>(p);
    return check_cuda("isaac_mlp_forward");
}

extern "C" int isaac_mlp_train_step(isaac_mlp *m, const uint16_t *X, const isaac_ray *rays,
                                    int64_t n_rays, float lr, int32_t margin, float *loss_sum,
                                    void *stream)
{
    clear_error();
    int rc = check_model(m, true);
    if (rc) return rc;
    if (n_rays <= 0 || !X || !rays) return fail(ISAAC_EINVAL, "X, rays and a positive count are required");
    if (((uintptr_t)X) % 4) return fail(ISAAC_EINVAL, "X must be 4-byte aligned");
    if (!std::isfinite(lr) || lr < 0.0f) return fail(ISAAC_EINVAL, "lr must be finite and >= 0");
    const cudaStream_t st = (cudaStream_t)stream;
    const long long tiles = (n_rays + 63) / 64;
    const int blocks = (int)std::min<long long>(tiles, kTrainBlocks);
    // the blocks' partial sums live in the stream's workspace
    KParams wp;
    memset(&wp, 0, sizeof wp);
    void *part = nullptr;
    rc = bind_workspace(wp, st, (size_t)blocks * kPartStride * sizeof(float) + 16, &part);
    if (rc) return rc;
    KTrain p;
    p.hw = reinterpret_cast<const __half *>(m->half_w);
    p.params = m->params;
    p.part = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(part) + 15) & ~uintptr_t(15));
    p.X = reinterpret_cast<const __half *>(X);
    p.rays = reinterpret_cast<const RayRec *>(rays);
    p.n = n_rays;
    p.inv_n = 1.0f / (float)n_rays;
    p.margin = margin;
    cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmemBytes);
    k_mlp_train<<<(unsigned)blocks, 128, kTrainSmemBytes, st>>>(p);
    k_mlp_reduce<<<(N_PARAMS + 256) / 256, 256, 0, st>>>(p.part, blocks, m->grads, loss_sum);
    rc = check_cuda("isaac_mlp_train_step (gradients)");
    if (rc) return rc;
    m->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    k_adam<<<64, 256, 0, st>>>(m->params, m->grads, m->adam_m, m->adam_v, lr, (float)b1, (float)b2,
                               1e-8f, (float)(1.0 - std::pow(b1, m->step)),
                               (float)(1.0 - std::pow(b2, m->step)));
    k_mlp_half<<<64, 256, 0, st>>>(m->params, reinterpret_cast<__half *>(m->half_w));
    return check_cuda("isaac_mlp_train_step (update)");
}

// ------------------------------------------------- proposal inside a frame

namespace isaac {

// One end of a ray's widening: the first sample met walking the samples from
// k_from towards k_to (exclusive; either direction) that lies in a macro cell
// with a nonzero grid value, or -1.  A 3D-DDA over the macro cells
// (Amanatides & Woo 1987) along the walking direction: for each cell the
// samples inside it are those with j * step in [entry, exit) of the cell
// (distances from sample k_from), so a nonzero cell is tested once and
// yields its first sample, if it holds any.  Cells are indexed as the grid
// features index them (floor(p / cell), clamped); an edge cell reaches to
// infinity beyond the grid.  A sample within FP32 rounding of a face may
// count on either side.
__device__ __forceinline__ int walk_to_nonzero(const RayRec &r, float step, const float *grid, int cell,
                                               int gx, int gy, int gz, int k_from, int k_to)
{
    const int dir = k_to >= k_from ? 1 : -1;
    const int J = (k_to - k_from) * dir;          // samples j = 0 .. J-1
    if (J <= 0) return -1;
    const float inf = __int_as_float(0x7f800000);
    const float c = (float)cell, inv_cell = 1.0f / c, inv_step = 1.0f / step;
    const float s0 = (float)k_from * step;
    const float px = fmaf(s0, r.dx, r.ex), py = fmaf(s0, r.dy, r.ey), pz = fmaf(s0, r.dz, r.ez);
    const float vx = dir > 0 ? r.dx : -r.dx, vy = dir > 0 ? r.dy : -r.dy, vz = dir > 0 ? r.dz : -r.dz;
    int cx = min(max((int)floorf(px * inv_cell), 0), gx - 1);
    int cy = min(max((int)floorf(py * inv_cell), 0), gy - 1);
    int cz = min(max((int)floorf(pz * inv_cell), 0), gz - 1);
    const int sx = vx > 0.0f ? 1 : -1, sy = vy > 0.0f ? 1 : -1, sz = vz > 0.0f ? 1 : -1;
    // distance to the next face per axis and between faces (inf: never, or
    // the cell is the grid's last one that way)
    const auto first_face = [&](float pa, float va, int ca, int sa, int ga) {
        if (va == 0.0f || (sa > 0 && ca == ga - 1) || (sa < 0 && ca == 0)) return inf;
        return ((float)(sa > 0 ? ca + 1 : ca) * c - pa) / va;
    };
    float tx = first_face(px, vx, cx, sx, gx), ty = first_face(py, vy, cy, sy, gy);
    float tz = first_face(pz, vz, cz, sz, gz);
    const float dtx = vx != 0.0f ? c / fabsf(vx) : inf, dty = vy != 0.0f ? c / fabsf(vy) : inf;
    const float dtz = vz != 0.0f ? c / fabsf(vz) : inf;
    float s_in = 0.0f;
    // every pass crosses one face; the bound only guards against rounding
    for (int it = 0; it < 3 * (gx + gy + gz) + 8; ++it) {
        const float s_out = fminf(tx, fminf(ty, tz));
        const int j_out = (int)ceilf(fminf(s_out * inv_step, 1.0e9f));   // first sample past the cell
        if (__ldg(grid + ((cz * gy + cy) * gx + cx)) > 0.0f) {
            const int j_in = s_in > 0.0f ? (int)ceilf(s_in * inv_step) : 0;
            if (j_in < min(j_out, J)) return k_from + dir * j_in;
        }
        if (j_out >= J) return -1;
        if (tx <= ty && tx <= tz) {
            cx += sx;
            tx = (sx > 0 ? cx == gx - 1 : cx == 0) ? inf : tx + dtx;
        } else if (ty <= tz) {
            cy += sy;
            ty = (sy > 0 ? cy == gy - 1 : cy == 0) ? inf : ty + dty;
        } else {
            cz += sz;
            tz = (sz > 0 ? cz == gz - 1 : cz == 0) ? inf : tz + dtz;
        }
        s_in = s_out;
    }
    return k_from;   // not reached; widening to the walk's start is always safe
}

struct KPropose {
    WsCounters *ctr;
    RayRec *rays;
    unsigned *longs;          // long-ray list to fill (nullptr: none)
    const __half *hw;
    const float *params;
    const float *grid;
    int cell, gx, gy, gz;
    float step, nx, ny, nz;
    float threshold;
    int margin;
    int widen;
    int hull_only;            // no network: every ray's range is its grid hull
    int *stats;
};

// RayRec::reserved of a confident ray whose range k_mlp_widen has yet to widen
// (its network range is in jf, jl meanwhile).
constexpr int kWidenPending = 1;

// The decision for ray r from its network outputs u (Sec. 3.2's marcher is the
// fallback: an unsure ray keeps its whole range).
__device__ __forceinline__ void propose_decide(const KPropose &p, unsigned r, const float (&u)[4], int &seen,
                                               int &restricted)
{
    ++seen;
    const int ns = p.rays[r].nsteps;
    int kb = 0, ke = ns;
    if (sigmoidf(u[2]) >= p.threshold) {
        const float te = sigmoidf(u[0]), tx = sigmoidf(u[1]);
        kb = (int)floorf(te * (float)ns) - p.margin;
        ke = (int)ceilf(tx * (float)ns) + p.margin;
        ++restricted;
        if (p.widen) {   // k_mlp_widen finishes the ray
            p.rays[r].jf = kb;
            p.rays[r].jl = ke;
            p.rays[r].reserved = kWidenPending;
            return;
        }
        kb = min(max(kb, 0), ns);
        ke = min(max(ke, kb), ns);
        p.rays[r].kbeg = kb;
        p.rays[r].nsteps = ke;
    }
    if (p.longs && ke - kb > kLongRaySamples) {
        p.rays[r].jf = kLongRay;
        p.longs[atomicAdd(&p.ctr->n_long, 1u)] = r;
    }
}

// Persistent CTAs take tiles of 128 rays of the frame's ray list: the inputs
// (two threads per ray) into the K-major activation tile, the network on the
// tensor cores (tc_forward_tile), then one thread per ray decides.  If a
// tensor-core wait runs out, the rays of that tile and the CTA's later tiles
// keep their whole range (the plain march).
static __global__ void __launch_bounds__(kTcThreads) k_mlp_propose(const __grid_constant__ KPropose p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcState s = tc_begin(p.hw, p.params, smem_raw);
    unsigned char *tile = smem_raw + kTcOffX;
    const unsigned n = *(volatile unsigned *)&p.ctr->n_rays;
    const int row = threadIdx.x >> 1, half = threadIdx.x & 1;
    int seen = 0, restricted = 0;
    bool alive = true;
    for (unsigned base = blockIdx.x * kTcRows; base < n; base += gridDim.x * kTcRows) {
        const unsigned r = base + row;
        if (r < n) {
            const RayRec rec = p.rays[r];
            ray_features_tc(rec, p.step, p.grid, p.cell, p.gx, p.gy, p.gz, p.nx, p.ny, p.nz, half, tile, row);
        } else {   // an empty row: zero inputs
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            for (int c = 0; c < 12; ++c)
                *reinterpret_cast<uint4 *>(tile + tc_off(row, (half * 12 + c) * 8, kTcLboX)) = z;
            for (int c = 0; c < 2; ++c)
                *reinterpret_cast<uint4 *>(tile + tc_off(row, (24 + half * 2 + c) * 8, kTcLboX)) = z;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        float u[4];
        if (!tc_forward_tile(s, smem_raw, u)) {
            alive = false;
            break;
        }
        if (threadIdx.x < kTcRows && base + threadIdx.x < n) propose_decide(p, base + threadIdx.x, u, seen, restricted);
    }
    if (!alive) tc_wait(s.bar, (s.phase - 1u) & 1u);   // let an MMA still in flight finish (bounded)
    if (p.stats && (seen | restricted)) {
        atomicAdd(p.stats, seen);
        atomicAdd(p.stats + 1, restricted);
    }
    tc_end(s);
}

// The widening of the confident rays k_mlp_propose marked (network range in
// jf/jl, unclipped): one thread per ray walks from the ray's start forward to
// the range for the first sample in a macro cell with a nonzero grid value,
// and from its end backward for the last one (the whole ray when the range is
// empty); the range becomes the hull of both, clipped to the ray.  A separate
// kernel, so that these dependent walks run at full occupancy rather than in
// the shared-memory-heavy proposal kernel.
static __global__ void __launch_bounds__(128) k_mlp_widen(const __grid_constant__ KPropose p)
{
    const unsigned n = *(volatile unsigned *)&p.ctr->n_rays;
    for (unsigned r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        RayRec rec = p.rays[r];
        if (!p.hull_only && rec.reserved != kWidenPending) continue;
        int kb = p.hull_only ? 0 : rec.jf, ke = p.hull_only ? 0 : rec.jl;   // hull only: empty
        const int ns = rec.nsteps;
        const bool open = ke > kb;
        const int first = walk_to_nonzero(rec, p.step, p.grid, p.cell, p.gx, p.gy, p.gz, 0,
                                          open ? min(max(kb, 0), ns) : ns);
        const int last = walk_to_nonzero(rec, p.step, p.grid, p.cell, p.gx, p.gy, p.gz,
                                         ns - 1, (open ? min(max(ke, 0), ns) : 0) - 1);
        if (open) {              // the hull of the range and the nonzero samples
            if (first >= 0) kb = min(kb, first);
            if (last >= 0) ke = max(ke, last + 1);
        } else if (first >= 0) {
            kb = first;
            ke = max(last, first) + 1;
        }
        kb = min(max(kb, 0), ns);
        ke = min(max(ke, kb), ns);
        p.rays[r].kbeg = kb;
        p.rays[r].nsteps = ke;
        p.rays[r].reserved = 0;
        p.rays[r].jl = -1;
        if (p.longs && ke - kb > kLongRaySamples) {
            p.rays[r].jf = kLongRay;
            p.longs[atomicAdd(&p.ctr->n_long, 1u)] = r;
        } else {
            p.rays[r].jf = -1;
        }
    }
}

static int launch_propose(const KParams &fp, const void *arg, cudaStream_t st)
{
    const isaac_proposal *pr = static_cast<const isaac_proposal *>(arg);
    KPropose p;
    p.ctr = fp.ctr;
    p.rays = fp.rays;
    p.longs = fp.longs;
    p.hw = pr->model ? reinterpret_cast<const __half *>(pr->model->half_w) : nullptr;
    p.params = pr->model ? pr->model->params : nullptr;
    p.hull_only = pr->model == nullptr;
    p.grid = pr->grid;
    p.cell = pr->cell;
    p.gx = (fp.nx + pr->cell - 1) / pr->cell;
    p.gy = (fp.ny + pr->cell - 1) / pr->cell;
    p.gz = (fp.nz + pr->cell - 1) / pr->cell;
    if ((long long)p.gx * p.gy * p.gz > 0x7fffffffLL)
        return fail(ISAAC_ENOTSUP, "the proposal's grid has more than 2^31 - 1 macro cells");
    p.step = fp.step;
    p.nx = (float)fp.nx;
    p.ny = (float)fp.ny;
    p.nz = (float)fp.nz;
    p.threshold = pr->threshold;
    p.margin = pr->margin;
    p.widen = pr->widen != 0;
    p.stats = pr->stats;
    cudaFuncSetAttribute(k_mlp_propose, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
    const int sms = sm_count();
    const long long rect = (long long)(fp.rx1 - fp.rx0) * (fp.ry1 - fp.ry0);
    const long long blocks = std::max(1LL, std::min<long long>((rect + kTcRows - 1) / kTcRows, (long long)sms * 2));
    if (!p.hull_only) k_mlp_propose<<<(unsigned)blocks, kTcThreads, kTcSmemBytes, st>>>(p);
    if (p.widen) {
        const long long wb = std::max(1LL, std::min<long long>((rect + 127) / 128, (long long)sms * 16));
        k_mlp_widen<<<(unsigned)wb, 128, 0, st>>>(p);
    }
    return check_cuda("interval proposal launch");
}

int proposal_hook(const isaac_proposal *pr, const isaac_render_opts *opts, FrameHook *hook)
{
    hook->fn = nullptr;
    hook->arg = nullptr;
    if (!pr) return ISAAC_OK;
    if (pr->model || !pr->widen) {   // no model: the grid's hull alone (needs widen)
        const int rc = check_model(pr->model, false);
        if (rc) return rc;
    }
    if (!pr->grid || pr->cell < 1) return fail(ISAAC_EINVAL, "proposal needs a grid and a cell size >= 1");
    if (!(pr->threshold >= 0.0f) || pr->margin < 0)
        return fail(ISAAC_EINVAL, "proposal threshold must be >= 0 and margin >= 0");
    if (((uintptr_t)pr->stats) % 4) return fail(ISAAC_EINVAL, "proposal stats misaligned");
    (void)opts;
    hook->fn = launch_propose;
    hook->arg = pr;
    return ISAAC_OK;
}

}  // namespace isaac
