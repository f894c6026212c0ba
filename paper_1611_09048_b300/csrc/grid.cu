// grid.cu -- isaac_opacity_grid: the max-opacity grid over macro cells.
//
// Macro cell (i, j, k) of `cell`^3 cells covers the cells [i*cell - 1,
// (i+1)*cell] per axis (the one-cell apron that trilinear samples inside the
// macro cell read), clipped to [-1, n]; its value is the largest blended
// opacity clamp(sum_s w_s * LUT_s(chain_s(v_s)).alpha, 0, 1) over those cells,
// each source read at the cell itself (clamped to the border without guards).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.h"
#include "packed.cuh"

namespace isaac {

struct KGrid {
    KSource src[ISAAC_MAX_ACTIVE];
    KChain ch[ISAAC_MAX_ACTIVE];
    const float4 *lut[ISAAC_MAX_ACTIVE];
    int nact;
    int nx, ny, nz;
    int cell;
    int gx, gy, gz;
    int W, H;             // columns per axis of the apron-extended volume: nx + 2, ny + 2
    int kchunk, nchunks;  // macro cells per z chunk, chunks
    float *cols;          // column maxima: (gz, H, W), workspace
    float *grid;
    // over a packed copy instead of the sources: records of [-1, n]^3, the
    // active packed sources' first component in the record and f_dim
    const unsigned char *rec;
    const float *scales;  // E4M3 brick scales
    int comp_off[ISAAC_MAX_ACTIVE], fdim[ISAAC_MAX_ACTIVE];
    int pbx, pby;         // bricks per axis x, y (E4M3)
};

// Blocks of 256 per SM for the value-range walk of one scalar and the walk
// over 16-bit scalar records (at most 40 registers): 48 warps per SM keep
// more loads in flight than 32.  The float32 opacity walk measured slower so
// (0.1335 -> 0.1366 ms at bubble512) and keeps 4.
constexpr int kScalarWalkBlocksPerSM = 6;

// z-cells whose loads a thread issues together: 16 on the scalar fast paths
// (a walk is bound by the loads in flight), 8 where a cell has several values
template <int FD> constexpr int grid_z() { return FD == 1 ? 16 : 8; }

// Blended opacity of the kGridZ cells zb .. zb+kGridZ-1 of the column whose
// per-source element pointers are cp (z clamped to each source's readable range).
template <int NS, int FD, int kGridZ>
__device__ __forceinline__ void column_alpha(const KGrid &p, const float *const *cp, const float *s_alpha,
                                             int nact, int zb, float (&a)[kGridZ])
{
#pragma unroll
    for (int j = 0; j < kGridZ; ++j) a[j] = 0.0f;
#pragma unroll
    for (int s = 0; s < ISAAC_MAX_ACTIVE; ++s) {
        if (s >= nact) break;
        const KSource &q = p.src[s];
        const int fd = (NS == 1 && FD) ? FD : q.fdim;
        float v[kGridZ][4];
#pragma unroll
        for (int j = 0; j < kGridZ; ++j) {
            const int zi = min(max(min(zb + j, p.nz), q.lo), p.nz - 1 + q.hi_pad);
            const float *b = cp[s] + (long long)zi * q.sz;
            v[j][0] = __ldg(b);
#pragma unroll
            for (int c = 1; c < 4; ++c) v[j][c] = c < fd ? __ldg(b + (long long)c * q.sc) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < kGridZ; ++j) {
            float w[4] = {v[j][0], v[j][1], v[j][2], v[j][3]};
            const float xv = run_chain(p.ch[s], w);
            const float pos = clamp01(xv) * 255.0f;
            const int k = min((int)pos, 254);
            const float f = pos - (float)k;
            a[j] = fmaf(q.w, lerp1(s_alpha[s * 256 + k], s_alpha[s * 256 + k + 1], f), a[j]);
        }
    }
}

// Pass 1: one thread per item = (x, y) column of the apron-extended volume
// [-1, n]^2 and chunk of kchunk macro cells in z; consecutive threads take
// consecutive x, so every load is coalesced, and each column is read once
// (plus the two shared z-cells at chunk borders).  The thread walks z through
// the chunk's cells [k0*cell - 1, k1*cell], kGridZ cells' loads at a time.
// Cell z belongs to macro cells k with k*cell - 1 <= z <= (k+1)*cell (at most
// two for cell >= 2), so the thread keeps two running maxima, for the lowest
// open macro cell and the next, and stores the column maximum of each macro
// cell when z leaves it: cols[k][y+1][x+1], every entry written once.
// NS > 0: NS active sources known at compile time, and with NS == 1 and
// FD > 0 the source's f_dim too (the scalar fast path); 0: read at run time.
template <int NS, int FD>
static __global__ void __launch_bounds__(256, (NS == 1 && FD == 1) ? 4 : 2) k_grid_columns(const __grid_constant__ KGrid p)
{
    constexpr int kGridZ = grid_z<(NS == 1 && FD == 1) ? 1 : 4>();
    __shared__ float s_alpha[ISAAC_MAX_ACTIVE * 256];
    const int nact = NS ? NS : p.nact;
    for (int i = threadIdx.x; i < nact * 256; i += blockDim.x) s_alpha[i] = __ldg(&p.lut[i >> 8][i & 255].w);
    __syncthreads();
    const long long plane = (long long)p.W * p.H;
    const long long items = plane * p.nchunks;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int chunk = (int)(it / plane);
        const long long col = it - (long long)chunk * plane;
        const int yy = (int)(col / p.W), xx = (int)(col - (long long)yy * p.W);
        const int x = xx - 1, y = yy - 1;
        const float *cp[ISAAC_MAX_ACTIVE];
#pragma unroll
        for (int s = 0; s < ISAAC_MAX_ACTIVE; ++s) {
            cp[s] = p.src[0].base;
            if (s < nact) {
                const KSource &q = p.src[s];
                const int xi = min(max(x, q.lo), p.nx - 1 + q.hi_pad);
                const int yi = min(max(y, q.lo), p.ny - 1 + q.hi_pad);
                cp[s] = q.base + ((long long)xi * q.sx + (long long)yi * q.sy);
            }
        }
        const int k0 = chunk * p.kchunk, k1 = min(k0 + p.kchunk, p.gz);
        const int zs = max(k0 * p.cell - 1, -1), ze = min(k1 * p.cell, p.nz);
        int ka = k0;                                            // lowest open macro cell
        int end_a = min((ka + 1) * p.cell, p.nz);               // its last z
        int start_b = ka + 1 < k1 ? (ka + 1) * p.cell - 1 : 0x7fffffff;   // first z of cell ka + 1
        float ma = 0.0f, mb = 0.0f;                             // running maxima of cells ka, ka + 1
        float *out = p.cols + col;
        for (int zb = zs; zb <= ze; zb += kGridZ) {
            float a[kGridZ];
            column_alpha<NS, FD, kGridZ>(p, cp, s_alpha, nact, zb, a);
#pragma unroll
            for (int j = 0; j < kGridZ; ++j) {
                const int z = zb + j;
                if (z > ze) break;
                if (z > end_a) {                  // z left cell ka: store it, open the next
                    out[(long long)ka * plane] = ma;
                    ++ka;
                    ma = mb;
                    mb = 0.0f;
                    end_a = min((ka + 1) * p.cell, p.nz);
                    start_b = ka + 1 < k1 ? (ka + 1) * p.cell - 1 : 0x7fffffff;
                }
                const float al = clamp01(a[j]);
                ma = fmaxf(ma, al);
                mb = z >= start_b ? fmaxf(mb, al) : mb;
            }
        }
        out[(long long)ka * plane] = ma;          // ka == k1 - 1: the walk ends in it
    }
}

// Pass 1 over a packed copy (isaac_opacity_grid_packed): the walk of
// k_grid_columns, reading record (x+1, y+1, z+1) of the [-1, n]^3 box -- which
// already holds the apron trilinear samples read (guards, or the repeated
// border) -- and decoding it as the packed renderer does (E4M3 times its brick
// scale).  The grid is then the one of the dequantised copy.
template <int DT, int PAD>
static __global__ void __launch_bounds__(256, PAD == 1 ? 3 : 4) k_grid_columns_packed(const __grid_constant__ KGrid p)
{
    using IO = RecIO<DT, PAD>;
    constexpr int kZ = PAD <= 1 ? 16 : 16 / PAD;   // records per batch: all loaded before any use
    __shared__ float s_alpha[ISAAC_MAX_ACTIVE * 256];
    for (int i = threadIdx.x; i < p.nact * 256; i += blockDim.x) s_alpha[i] = __ldg(&p.lut[i >> 8][i & 255].w);
    __syncthreads();
    const long long plane = (long long)p.W * p.H;
    const long long items = plane * p.nchunks;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int chunk = (int)(it / plane);
        const long long col = it - (long long)chunk * plane;   // record column (x+1, y+1)
        const int yy = (int)(col / p.W), xx = (int)(col - (long long)yy * p.W);
        const int k0 = chunk * p.kchunk, k1 = min(k0 + p.kchunk, p.gz);
        const int zs = max(k0 * p.cell - 1, -1), ze = min(k1 * p.cell, p.nz);
        int ka = k0;
        int end_a = min((ka + 1) * p.cell, p.nz);
        int start_b = ka + 1 < k1 ? (ka + 1) * p.cell - 1 : 0x7fffffff;
        float ma = 0.0f, mb = 0.0f;
        float *out = p.cols + col;
        for (int zb = zs; zb <= ze; zb += kZ) {
            float r[kZ][PAD];
#pragma unroll
            for (int j = 0; j < kZ; ++j) {
                const int zr = min(zb + j, p.nz) + 1;           // record z (past ze: a repeat, dropped)
                IO::load(p.rec, (long long)zr * plane + col, r[j]);
                if constexpr (DT == ISAAC_E4M3) {
                    float sc[PAD];
                    load_scales<PAD>(p.scales, ((zr >> 3) * p.pby + (yy >> 3)) * p.pbx + (xx >> 3), sc);
#pragma unroll
                    for (int c = 0; c < PAD; ++c) r[j][c] *= sc[c];
                }
            }
            float a[kZ];
#pragma unroll
            for (int j = 0; j < kZ; ++j) {
                float acc = 0.0f;
                for (int s = 0; s < p.nact; ++s) {
                    float w[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float x = 0.0f;
#pragma unroll
                        for (int q = 0; q < PAD; ++q)
                            if (q == p.comp_off[s] + c && c < p.fdim[s]) x = r[j][q];
                        w[c] = x;
                    }
                    const float xv = run_chain(p.ch[s], w);
                    const float pos = clamp01(xv) * 255.0f;
                    const int k = min((int)pos, 254);
                    const float f = pos - (float)k;
                    acc = fmaf(p.src[s].w, lerp1(s_alpha[s * 256 + k], s_alpha[s * 256 + k + 1], f), acc);
                }
                a[j] = acc;
            }
#pragma unroll
            for (int j = 0; j < kZ; ++j) {
                const int z = zb + j;
                if (z > ze) break;
                if (z > end_a) {
                    out[(long long)ka * plane] = ma;
                    ++ka;
                    ma = mb;
                    mb = 0.0f;
                    end_a = min((ka + 1) * p.cell, p.nz);
                    start_b = ka + 1 < k1 ? (ka + 1) * p.cell - 1 : 0x7fffffff;
                }
                const float al = clamp01(a[j]);
                ma = fmaxf(ma, al);
                mb = z >= start_b ? fmaxf(mb, al) : mb;
            }
        }
        out[(long long)ka * plane] = ma;
    }
}

// Pass 1 over a packed copy with one scalar record (pad 1) of one active
// source with the identity chain and CELL-cell macro cells: the branch-free
// walk of k_grid_columns_scalar over records (x+1, y+1, z+1), z clamped to the
// box [-1, n] (reads past it repeat the last record, already in the cell).
template <int DT, int CELL>
static __global__ void __launch_bounds__(256, 4) k_grid_columns_packed_scalar(const __grid_constant__ KGrid p)
{
    using IO = RecIO<DT, 1>;
    __shared__ float2 s_pair[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float a0 = __ldg(&p.lut[0][i].w);
        const float a1 = i < 255 ? __ldg(&p.lut[0][i + 1].w) : a0;
        s_pair[i] = make_float2(a0, a1 - a0);
    }
    __syncthreads();
    const float w = p.src[0].w;
    auto alpha = [&](float v) {
        const float pos = clamp01(v) * 255.0f;
        const int k = min((int)pos, 254);
        const float2 e = s_pair[k];
        return clamp01(fmaf(w, fmaf(pos - (float)k, e.y, e.x), 0.0f));
    };
    const long long plane = (long long)p.W * p.H;
    const long long items = plane * p.nchunks;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int chunk = (int)(it / plane);
        const long long col = it - (long long)chunk * plane;
        const int k0 = chunk * p.kchunk, k1 = min(k0 + p.kchunk, p.gz);
        auto rec = [&](int z) {                  // value of cell z (clamped to [-1, n]) in this column
            float r[1];
            IO::load(p.rec, (long long)(min(max(z, -1), p.nz) + 1) * plane + col, r);
            return r[0];
        };
        float *out = p.cols + col;
        float prev = fmaxf(alpha(rec(k0 * CELL - 1)), alpha(rec(k0 * CELL)));
        for (int k = k0; k < k1; ++k) {
            const int z0 = k * CELL + 1;
            float v[CELL];
            if (z0 + CELL - 1 <= p.nz) {          // inside the box: records at a fixed stride
                const unsigned char *b = p.rec + ((long long)(z0 + 1) * plane + col) * IO::BYTES;
                const long long step = plane * IO::BYTES;
#pragma unroll
                for (int j = 0; j < CELL; ++j) {
                    float r[1];
                    IO::load(b + j * step, 0, r);
                    v[j] = r[0];
                }
            } else {
#pragma unroll
                for (int j = 0; j < CELL; ++j) v[j] = rec(z0 + j);
            }
            float core = 0.0f;
#pragma unroll
            for (int j = 0; j < CELL - 2; ++j) core = fmaxf(core, alpha(v[j]));
            const float next = fmaxf(alpha(v[CELL - 2]), alpha(v[CELL - 1]));
            out[(long long)k * plane] = fmaxf(fmaxf(prev, core), next);
            prev = next;
        }
    }
}

// The same walk over two adjacent columns (2j, 2j+1) of a 16-bit scalar copy
// whose padded row length is even: one 4-byte load per cell pair, so each
// thread keeps twice the bytes in flight of the one-column walk, whose 2-byte
// loads left it bound by memory latency at half the bandwidth of the float32
// walk.  Both columns' maxima are written with one 8-byte store.
template <int DT, int CELL>
static __global__ void __launch_bounds__(256, kScalarWalkBlocksPerSM) k_grid_columns_packed_scalar2(const __grid_constant__ KGrid p)
{
    __shared__ float2 s_pair[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float a0 = __ldg(&p.lut[0][i].w);
        const float a1 = i < 255 ? __ldg(&p.lut[0][i + 1].w) : a0;
        s_pair[i] = make_float2(a0, a1 - a0);
    }
    __syncthreads();
    const float w = p.src[0].w;
    auto alpha = [&](float v) {
        const float pos = clamp01(v) * 255.0f;
        const int k = min((int)pos, 254);
        const float2 e = s_pair[k];
        return clamp01(fmaf(w, fmaf(pos - (float)k, e.y, e.x), 0.0f));
    };
    const long long plane = (long long)p.W * p.H, half = plane >> 1;
    const long long items = half * p.nchunks;
    const unsigned *rec = reinterpret_cast<const unsigned *>(p.rec);
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int chunk = (int)(it / half);
        const long long q = it - (long long)chunk * half;          // word q of a plane: columns 2q, 2q+1
        const int k0 = chunk * p.kchunk, k1 = min(k0 + p.kchunk, p.gz);
        auto pair = [&](int z, float &a, float &b) {                // cells z (clamped to [-1, n])
            unpack2<DT>(__ldg(rec + (long long)(min(max(z, -1), p.nz) + 1) * half + q), a, b);
        };
        float2 *out = reinterpret_cast<float2 *>(p.cols) + q;
        float prev0, prev1;
        {
            float a0, a1, b0, b1;
            pair(k0 * CELL - 1, a0, a1);
            pair(k0 * CELL, b0, b1);
            prev0 = fmaxf(alpha(a0), alpha(b0));
            prev1 = fmaxf(alpha(a1), alpha(b1));
        }
        for (int k = k0; k < k1; ++k) {
            const int z0 = k * CELL + 1;
            unsigned u[CELL];
            if (z0 + CELL - 1 <= p.nz) {
                const unsigned *b = rec + (long long)(z0 + 1) * half + q;
#pragma unroll
                for (int j = 0; j < CELL; ++j) u[j] = __ldg(b + j * half);
            } else {
#pragma unroll
                for (int j = 0; j < CELL; ++j) u[j] = __ldg(rec + (long long)(min(z0 + j, p.nz) + 1) * half + q);
            }
            float core0 = 0.0f, core1 = 0.0f, next0, next1;
#pragma unroll
            for (int j = 0; j < CELL; ++j) {
                float a, b;
                unpack2<DT>(u[j], a, b);
                a = alpha(a);
                b = alpha(b);
                if (j < CELL - 2) {
                    core0 = fmaxf(core0, a);
                    core1 = fmaxf(core1, b);
                } else if (j == CELL - 2) {
                    next0 = a;
                    next1 = b;
                } else {
                    next0 = fmaxf(next0, a);
                    next1 = fmaxf(next1, b);
                }
            }
            out[(long long)k * half] = make_float2(fmaxf(fmaxf(prev0, core0), next0),
                                                   fmaxf(fmaxf(prev1, core1), next1));
            prev0 = next0;
            prev1 = next1;
        }
    }
}

// Pass 1, one scalar source with the identity chain and macro cells of CELL
// cells (the learned proposal's configuration).  Macro cell k covers z in
// [k*CELL - 1, (k+1)*CELL]: the pair {k*CELL - 1, k*CELL} it shares with k-1,
// CELL-2 core cells, and the pair {(k+1)*CELL - 1, (k+1)*CELL} it shares with
// k+1.  The walk loads one pair (entering the chunk) and then CELL cells per
// macro cell: max(previous pair, core, next pair), branch-free.  Reads past the
// volume's clipped range are clamped to the last readable cell, which that
// macro cell already contains, so they do not change its maximum.  The alpha
// table holds (a_k, a_{k+1} - a_k), so a lookup is one 8-byte load and the
// interpolation fmaf(f, a_{k+1} - a_k, a_k) is the one lerp1 computes.
template <int CELL>
static __global__ void __launch_bounds__(256, 4) k_grid_columns_scalar(const __grid_constant__ KGrid p)
{
    __shared__ float2 s_pair[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float a0 = __ldg(&p.lut[0][i].w);
        const float a1 = i < 255 ? __ldg(&p.lut[0][i + 1].w) : a0;
        s_pair[i] = make_float2(a0, a1 - a0);
    }
    __syncthreads();
    const KSource &q = p.src[0];
    const int lo = q.lo, hi = p.nz - 1 + q.hi_pad;
    const long long sz = q.sz;
    const float w = q.w;
    auto alpha = [&](float v) {
        const float pos = clamp01(v) * 255.0f;
        const int k = min((int)pos, 254);
        const float2 e = s_pair[k];
        return clamp01(fmaf(w, fmaf(pos - (float)k, e.y, e.x), 0.0f));
    };
    const long long plane = (long long)p.W * p.H;
    const long long items = plane * p.nchunks;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int chunk = (int)(it / plane);
        const long long col = it - (long long)chunk * plane;
        const int yy = (int)(col / p.W), xx = (int)(col - (long long)yy * p.W);
        const int xi = min(max(xx - 1, lo), p.nx - 1 + q.hi_pad);
        const int yi = min(max(yy - 1, lo), p.ny - 1 + q.hi_pad);
        const float *cp = q.base + ((long long)xi * q.sx + (long long)yi * q.sy);
        const int k0 = chunk * p.kchunk, k1 = min(k0 + p.kchunk, p.gz);
        float *out = p.cols + col;
        float prev;
        {
            const int za = min(max(k0 * CELL - 1, lo), hi), zb = min(max(k0 * CELL, lo), hi);
            prev = fmaxf(alpha(__ldg(cp + za * sz)), alpha(__ldg(cp + zb * sz)));
        }
        for (int k = k0; k < k1; ++k) {
            const int z0 = k * CELL + 1;                 // cells z0 .. z0 + CELL - 1
            float v[CELL];
            if (z0 >= lo && z0 + CELL - 1 <= hi) {
                const float *b = cp + (long long)z0 * sz;
#pragma unroll
                for (int j = 0; j < CELL; ++j) v[j] = __ldg(b + j * sz);
            } else {
#pragma unroll
                for (int j = 0; j < CELL; ++j) v[j] = __ldg(cp + (long long)min(max(z0 + j, lo), hi) * sz);
            }
            float core = 0.0f;
#pragma unroll
            for (int j = 0; j < CELL - 2; ++j) core = fmaxf(core, alpha(v[j]));
            const float next = fmaxf(alpha(v[CELL - 2]), alpha(v[CELL - 1]));
            out[(long long)k * plane] = fmaxf(fmaxf(prev, core), next);
            prev = next;
        }
    }
}

// Pass 2: one warp per macro cell (i, j, k): the largest column maximum over
// its columns x in [i*cell - 1, (i+1)*cell], y likewise (clipped to [-1, n]).
static __global__ void __launch_bounds__(256) k_grid_reduce(const __grid_constant__ KGrid p)
{
    const int lane = threadIdx.x & 31;
    const long long cells = (long long)p.gx * p.gy * p.gz;
    const long long plane = (long long)p.W * p.H;
    for (long long m = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; m < cells;
         m += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int gi = (int)(m % p.gx), gj = (int)((m / p.gx) % p.gy), k = (int)(m / ((long long)p.gx * p.gy));
        const int xs = max(gi * p.cell - 1, -1) + 1, xe = min((gi + 1) * p.cell, p.nx) + 1;
        const int ys = max(gj * p.cell - 1, -1) + 1, ye = min((gj + 1) * p.cell, p.ny) + 1;
        const float *base = p.cols + (long long)k * plane;
        float mx = 0.0f;
        // lanes along x, 8 rows' loads issued together (the data sits in L2,
        // so the reduction is bound by load latency, not bytes)
        for (int x0 = xs; x0 <= xe; x0 += 32) {
            const int xx = x0 + lane;
            for (int y0 = ys; y0 <= ye; y0 += 8) {
                float v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    v[r] = (xx <= xe && y0 + r <= ye) ? __ldg(base + (long long)(y0 + r) * p.W + xx) : 0.0f;
#pragma unroll
                for (int r = 0; r < 8; ++r) mx = fmaxf(mx, v[r]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) p.grid[m] = mx;
    }
}

// Pass 2 for macro cells of CELL = 8 or 16 cells: one block per tile of
// TM x TM macro cells (TM * CELL = 64) of one z layer k.  The block stages the
// tile's 66 x 66 column maxima (its 64 x 64 columns and the one-column apron
// around them, zero outside [-1, n]) in shared memory with row-contiguous
// loads, takes per row the maximum over each macro cell's CELL + 2 columns,
// then per macro cell the maximum over its CELL + 2 rows.  Every column
// maximum is read once (1.06x with the apron), where the warp-per-macro-cell
// reduction read 18-float row pieces at a time.  Maxima are of values in
// [0, 1], so the zero fill changes none.
template <int CELL>
static __global__ void __launch_bounds__(256) k_grid_reduce_tiled(const __grid_constant__ KGrid p)
{
    constexpr int TM = 64 / CELL, R = TM * CELL + 2;
    __shared__ float s_col[R][R + 1];
    __shared__ float s_row[R][TM];
    const int tiles_x = (p.gx + TM - 1) / TM, tiles_y = (p.gy + TM - 1) / TM;
    const int tx = blockIdx.x % tiles_x, ty = (blockIdx.x / tiles_x) % tiles_y;
    const int k = blockIdx.x / (tiles_x * tiles_y);
    const long long plane = (long long)p.W * p.H;
    const float *base = p.cols + (long long)k * plane;
    // padded column xx = x + 1: the tile's columns x in [64 tx - 1, 64 tx + 64]
    const int x0 = tx * TM * CELL, y0 = ty * TM * CELL;
    // every thread's NL loads issued before any is stored (the column maxima
    // sit in L2: the stage is bound by load latency)
    constexpr int NL = (R * R + 255) / 256;
    float v[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {
        const int i = threadIdx.x + 256 * u, r = i / R, c = i - r * R;
        const int xx = x0 + c, yy = y0 + r;
        v[u] = (i < R * R && xx < p.W && yy < p.H) ? __ldg(base + (long long)yy * p.W + xx) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
        const int i = threadIdx.x + 256 * u, r = i / R, c = i - r * R;
        if (i < R * R) s_col[r][c] = v[u];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R * TM; i += blockDim.x) {
        const int r = i / TM, mi = i - r * TM;
        float m = 0.0f;
#pragma unroll
        for (int c = 0; c < CELL + 2; ++c) m = fmaxf(m, s_col[r][mi * CELL + c]);
        s_row[r][mi] = m;
    }
    __syncthreads();
    if (threadIdx.x < TM * TM) {
        const int mj = threadIdx.x / TM, mi = threadIdx.x - mj * TM;
        const int gi = tx * TM + mi, gj = ty * TM + mj;
        if (gi < p.gx && gj < p.gy) {
            float m = 0.0f;
#pragma unroll
            for (int r = 0; r < CELL + 2; ++r) m = fmaxf(m, s_row[mj * CELL + r][mi]);
            p.grid[((long long)k * p.gy + gj) * p.gx + gi] = m;
        }
    }
}

// Pass 2 launch: the tiled form for 8- and 16-cell macro cells, else one
// warp per macro cell.
static int launch_grid_reduce(const KGrid &p, long long cells, int sms, cudaStream_t st)
{
    if (p.cell == 8 || p.cell == 16) {
        const long long tm = 64 / p.cell;
        const long long blocks = ((p.gx + tm - 1) / tm) * ((p.gy + tm - 1) / tm) * (long long)p.gz;
        if (blocks <= 0x7fffffffLL) {
            if (p.cell == 16) k_grid_reduce_tiled<16><<<(unsigned)blocks, 256, 0, st>>>(p);
            else k_grid_reduce_tiled<8><<<(unsigned)blocks, 256, 0, st>>>(p);
            return ISAAC_OK;
        }
    }
    const unsigned b2 = (unsigned)std::max(1LL, std::min((cells * 32 + 255) / 256, (long long)sms * 8));
    k_grid_reduce<<<b2, 256, 0, st>>>(p);
    return ISAAC_OK;
}

// ------------------------------------------------------ value-range grid

struct KRange {
    KSource src;          // the source of this pass
    int nx, ny, nz, cell, gx, gy, gz;
    int slots, slot0;     // components per macro cell in all, first of this source
    int W, H;             // columns per axis of the apron-extended volume
    int kchunk, nchunks;  // macro cells per z chunk, chunks
    float2 *cols;         // per column, macro cell and component: (min, max), workspace
    float *ranges;        // (min, max) per macro cell and slot
};

// The (min, max) a value contributes: a NaN widens to [-inf, +inf].
__device__ __forceinline__ float2 range_of(float v)
{
    const float inf = __int_as_float(0x7f800000);
    return v == v ? make_float2(v, v) : make_float2(-inf, inf);
}
__device__ __forceinline__ float2 range_join(float2 a, float2 b)
{
    return make_float2(fminf(a.x, b.x), fmaxf(a.y, b.y));
}

// Pass 1 of the value-range grid, one source: the same items and walk as
// k_grid_columns (one thread per (x, y) column and z chunk, coalesced loads,
// each column read once), keeping per component the (min, max) of the values
// read for the open macro cell and the next; stored per column when z leaves
// a macro cell: cols[((k * H + y+1) * W + x+1) * FD + c].  CELL > 0: macro
// cells of CELL cells walked as shared pair / core / shared pair (the
// branch-free form of k_grid_columns_scalar); 0: any cell size.
template <int FD, int CELL>
static __global__ void __launch_bounds__(256, CELL > 0 ? (FD == 1 ? kScalarWalkBlocksPerSM : 4) : 2) k_range_columns(const __grid_constant__ KRange p)
{
    constexpr int kZ = CELL > 0 ? CELL : grid_z<FD>();
    const float inf = __int_as_float(0x7f800000);
    const KSource &q = p.src;
    const int lo = q.lo, hi = p.nz - 1 + q.hi_pad;
    const long long plane = (long long)p.W * p.H;
    const long long items = plane * p.nchunks;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int chunk = (int)(it / plane);
        const long long col = it - (long long)chunk * plane;
        const int yy = (int)(col / p.W), xx = (int)(col - (long long)yy * p.W);
        const int xi = min(max(xx - 1, lo), p.nx - 1 + q.hi_pad);
        const int yi = min(max(yy - 1, lo), p.ny - 1 + q.hi_pad);
        const float *cp = q.base + ((long long)xi * q.sx + (long long)yi * q.sy);
        const int k0 = chunk * p.kchunk, k1 = min(k0 + p.kchunk, p.gz);
        float2 *out = p.cols + col * FD;
        auto load = [&](int z, float (&v)[FD]) {
            const float *b = cp + (long long)min(max(z, lo), hi) * q.sz;
#pragma unroll
            for (int c = 0; c < FD; ++c) v[c] = __ldg(b + (long long)c * q.sc);
        };
        if constexpr (CELL > 0) {
            float2 prev[FD];
            {
                float va[FD], vb[FD];
                load(k0 * CELL - 1, va);
                load(k0 * CELL, vb);
#pragma unroll
                for (int c = 0; c < FD; ++c) prev[c] = range_join(range_of(va[c]), range_of(vb[c]));
            }
            for (int k = k0; k < k1; ++k) {
                const int z0 = k * CELL + 1;
                float v[CELL][FD];
#pragma unroll
                for (int j = 0; j < CELL; ++j) load(z0 + j, v[j]);
#pragma unroll
                for (int c = 0; c < FD; ++c) {
                    float2 core = make_float2(inf, -inf);
#pragma unroll
                    for (int j = 0; j < CELL - 2; ++j) core = range_join(core, range_of(v[j][c]));
                    const float2 next = range_join(range_of(v[CELL - 2][c]), range_of(v[CELL - 1][c]));
                    out[(long long)k * plane * FD + c] = range_join(range_join(prev[c], core), next);
                    prev[c] = next;
                }
            }
        } else {
            const int zs = max(k0 * p.cell - 1, -1), ze = min(k1 * p.cell, p.nz);
            int ka = k0;
            int end_a = min((ka + 1) * p.cell, p.nz);
            int start_b = ka + 1 < k1 ? (ka + 1) * p.cell - 1 : 0x7fffffff;
            float2 ra[FD], rb[FD];
#pragma unroll
            for (int c = 0; c < FD; ++c) ra[c] = rb[c] = make_float2(inf, -inf);
            for (int zb = zs; zb <= ze; zb += kZ) {
                float v[kZ][FD];
#pragma unroll
                for (int j = 0; j < kZ; ++j) load(zb + j, v[j]);
#pragma unroll
                for (int j = 0; j < kZ; ++j) {
                    const int z = zb + j;
                    if (z > ze) break;
                    if (z > end_a) {
#pragma unroll
                        for (int c = 0; c < FD; ++c) {
                            out[(long long)ka * plane * FD + c] = ra[c];
                            ra[c] = rb[c];
                            rb[c] = make_float2(inf, -inf);
                        }
                        ++ka;
                        end_a = min((ka + 1) * p.cell, p.nz);
                        start_b = ka + 1 < k1 ? (ka + 1) * p.cell - 1 : 0x7fffffff;
                    }
#pragma unroll
                    for (int c = 0; c < FD; ++c) {
                        const float2 r = range_of(v[j][c]);
                        ra[c] = range_join(ra[c], r);
                        if (z >= start_b) rb[c] = range_join(rb[c], r);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < FD; ++c) out[(long long)ka * plane * FD + c] = ra[c];
        }
    }
}

// Pass 2: one warp per macro cell: per component, the min of the column
// minima and the max of the column maxima over the cell's apron-extended
// columns, written as the slot's (min, max).
template <int FD>
static __global__ void __launch_bounds__(256) k_range_reduce(const __grid_constant__ KRange p)
{
    const float inf = __int_as_float(0x7f800000);
    const int lane = threadIdx.x & 31;
    const long long cells = (long long)p.gx * p.gy * p.gz;
    const long long plane = (long long)p.W * p.H;
    for (long long m = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; m < cells;
         m += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int gi = (int)(m % p.gx), gj = (int)((m / p.gx) % p.gy), k = (int)(m / ((long long)p.gx * p.gy));
        const int xs = max(gi * p.cell - 1, -1) + 1, xe = min((gi + 1) * p.cell, p.nx) + 1;
        const int ys = max(gj * p.cell - 1, -1) + 1, ye = min((gj + 1) * p.cell, p.ny) + 1;
        const float2 *base = p.cols + (long long)k * plane * FD;
        float2 r[FD];
#pragma unroll
        for (int c = 0; c < FD; ++c) r[c] = make_float2(inf, -inf);
        // lanes along x, 6 rows' loads issued together (L2 latency bound; a
        // 16-cell macro cell spans 18 rows)
        constexpr int Q = 6;
        for (int x0 = xs; x0 <= xe; x0 += 32) {
            const int xx = x0 + lane;
            for (int y0 = ys; y0 <= ye; y0 += Q) {
                float2 v[Q][FD];
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int c = 0; c < FD; ++c)
                        v[q][c] = (xx <= xe && y0 + q <= ye)
                                      ? __ldg(base + ((long long)(y0 + q) * p.W + xx) * FD + c)
                                      : make_float2(inf, -inf);
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int c = 0; c < FD; ++c) r[c] = range_join(r[c], v[q][c]);
            }
        }
#pragma unroll
        for (int c = 0; c < FD; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r[c].x = fminf(r[c].x, __shfl_xor_sync(0xffffffffu, r[c].x, o));
                r[c].y = fmaxf(r[c].y, __shfl_xor_sync(0xffffffffu, r[c].y, o));
            }
            if (lane == 0) {
                float *dst = p.ranges + 2 * (m * p.slots + p.slot0 + c);
                dst[0] = r[c].x;
                dst[1] = r[c].y;
            }
        }
    }
}

// ---------------------------------------------------- empty-space flags

struct KEmpty {
    const float *ranges;
    int slots;
    long long cells;
    int nact;
    int fdim[ISAAC_MAX_ACTIVE];
    float w[ISAAC_MAX_ACTIVE];
    KChain ch[ISAAC_MAX_ACTIVE];
    const float4 *lut[ISAAC_MAX_ACTIVE];
    unsigned *flags;      // one bit per macro cell, 32 per word
};

// A macro cell is empty when, for the components' value ranges over its box,
// every source with weight > 0 has LUT opacity exactly 0 on every entry that
// the interval of its chain result can reach, and every reachable LUT entry
// of every source is finite.  A trilinear sample whose position lies in the
// cell interpolates between values of the box, so its opacity is then 0 and
// compositing it is a no-op.  The interpolation itself may round a few ulps
// outside the corners' range: the ranges are widened by 10^-6 relative first.
// One thread per macro cell, a warp per word of 32 bits.
static __global__ void k_empty_flags(const __grid_constant__ KEmpty p)
{
    const int lane = threadIdx.x & 31;
    for (long long gb = blockIdx.x * (long long)blockDim.x + threadIdx.x - lane; gb < p.cells;
         gb += (long long)gridDim.x * blockDim.x) {
        const long long g = gb + lane;
        bool empty = g < p.cells;
        int slot = 0;
        for (int s = 0; s < p.nact && empty; ++s) {
            float lo[4] = {0.0f, 0.0f, 0.0f, 0.0f}, hi[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int c = 0; c < p.fdim[s]; ++c) {
                const float l = p.ranges[2 * (g * p.slots + slot + c)];
                const float h = p.ranges[2 * (g * p.slots + slot + c) + 1];
                lo[c] = l - (fabsf(l) * 1e-6f + 1e-30f);
                hi[c] = h + (fabsf(h) * 1e-6f + 1e-30f);
            }
            slot += p.fdim[s];
            chain_interval(p.ch[s], lo, hi);
            const float pl = clamp01(lo[0]) * 255.0f, ph = clamp01(hi[0]) * 255.0f;
            const int j0 = min((int)pl, 254), j1 = min((int)ph, 254) + 1;
            for (int j = j0; j <= j1; ++j) {
                const float4 e = __ldg(p.lut[s] + j);
                if (!(isfinite(e.x) && isfinite(e.y) && isfinite(e.z) && isfinite(e.w)) ||
                    (p.w[s] > 0.0f && e.w != 0.0f)) {
                    empty = false;
                    break;
                }
            }
        }
        const unsigned bits = __ballot_sync(0xffffffffu, empty);
        if (lane == 0) p.flags[gb >> 5] = bits;
    }
}

int launch_empty_flags(const KParams &kp, int nact, const float *ranges, int slots, long long cells,
                       unsigned *flags, cudaStream_t st)
{
    KEmpty e;
    memset(&e, 0, sizeof e);
    e.ranges = ranges;
    e.slots = slots;
    e.cells = cells;
    e.nact = nact;
    for (int a = 0; a < nact; ++a) {
        e.fdim[a] = kp.src[a].fdim;
        e.w[a] = kp.src[a].w;
        e.ch[a] = kp.ch[a];
        e.lut[a] = kp.lut[a];
    }
    e.flags = flags;
    const long long blocks = std::max(1LL, std::min((cells + 255) / 256, 148LL * 8));
    k_empty_flags<<<(unsigned)blocks, 256, 0, st>>>(e);
    return check_cuda("empty-space flags launch");
}

}  // namespace isaac

using namespace isaac;

extern "C" int isaac_opacity_grid(const isaac_source *sources, const isaac_chain *chains,
                                  int32_t n_sources, const float *luts, const float *weights,
                                  const isaac_render_opts *opts, int32_t cell, float *grid,
                                  int64_t grid_len, void *stream)
{
    clear_error();
    if (!sources || !chains || !weights || !opts || !grid || !luts)
        return fail(ISAAC_EINVAL, "sources, chains, luts, weights, opts and grid are required");
    if (n_sources < 1 || n_sources > ISAAC_MAX_SOURCES)
        return fail(ISAAC_EINVAL, "n_sources %d outside 1..%d", n_sources, ISAAC_MAX_SOURCES);
    if (cell < 2 || cell > 1024) return fail(ISAAC_EINVAL, "cell %d outside 2..1024", cell);
    if (opts->active_mask >> n_sources) return fail(ISAAC_EINVAL, "active_mask beyond n_sources");
    if (opts->flags & ~(ISAAC_LUTS_HOST | ISAAC_MARCH_STAGED)) return fail(ISAAC_EINVAL, "unknown opts.flags bits");
    if (!(opts->flags & ISAAC_LUTS_HOST) && ((uintptr_t)luts) % 16)
        return fail(ISAAC_EINVAL, "luts must be 16-byte aligned");
    KGrid p;
    memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a)
        if (opts->n[a] < 1 || opts->n[a] > (1 << 20)) return fail(ISAAC_EINVAL, "bad volume size");
    p.nx = (int)opts->n[0];
    p.ny = (int)opts->n[1];
    p.nz = (int)opts->n[2];
    p.cell = cell;
    p.gx = (p.nx + cell - 1) / cell;
    p.gy = (p.ny + cell - 1) / cell;
    p.gz = (p.nz + cell - 1) / cell;
    const long long cells = (long long)p.gx * p.gy * p.gz;
    if (grid_len < cells)
        return fail(ISAAC_ENOMEM, "grid holds %lld values, %lld needed", (long long)grid_len, cells);
    if (cells > 0x7fffffffLL) return fail(ISAAC_ENOTSUP, "too many macro cells");
    update_sources(n_sources, opts->active_mask);
    for (int s = 0; s < n_sources; ++s) {
        if (!((opts->active_mask >> s) & 1u)) continue;
        if (p.nact == ISAAC_MAX_ACTIVE)
            return fail(ISAAC_ENOTSUP, "more than %d active sources", ISAAC_MAX_ACTIVE);
        if (!std::isfinite(weights[s])) return fail(ISAAC_EINVAL, "weight %d is not finite", s);
        unsigned nib;
        bool wide;
        // interp = 1: the apron reads [-1, n] on guarded sources
        int rc = prepare_source(sources[s], s, opts->n, 1, weights[s], 4, p.src[p.nact], &nib, &wide);
        if (rc) return rc;
        rc = compile_chain(chains[s], sources[s].f_dim, s, p.ch[p.nact]);
        if (rc) return rc;
        p.lut[p.nact] = reinterpret_cast<const float4 *>(luts) + (size_t)s * 256;
        ++p.nact;
    }
    p.grid = grid;
    const cudaStream_t st = (cudaStream_t)stream;
    if (p.nact == 0) {
        if (cudaMemsetAsync(grid, 0, (size_t)cells * sizeof(float), st) != cudaSuccess)
            return check_cuda("isaac_opacity_grid memset");
        return ISAAC_OK;
    }
    // column maxima in the stream's workspace (ordered before any later frame
    // on the stream that reuses those bytes)
    p.W = p.nx + 2;
    p.H = p.ny + 2;
    p.kchunk = std::max(1, (64 + cell - 1) / cell);
    p.nchunks = (p.gz + p.kchunk - 1) / p.kchunk;
    const size_t col_bytes = (size_t)p.gz * (size_t)p.W * (size_t)p.H * sizeof(float);
    KParams wp;
    memset(&wp, 0, sizeof wp);
    if (opts->flags & ISAAC_LUTS_HOST) {   // staged into the workspace by bind_workspace
        for (int a = 0; a < p.nact; ++a) wp.lut[a] = p.lut[a];
        wp.luts_host = 1;
    }
    void *cols = nullptr;
    int rc = bind_workspace(wp, st, col_bytes + 16, &cols);
    if (rc) return rc;
    if (opts->flags & ISAAC_LUTS_HOST)   // the staged device copies
        for (int a = 0; a < p.nact; ++a) p.lut[a] = wp.lut[a];
    p.cols = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(cols) + 15) & ~uintptr_t(15));
    const int sms = sm_count();
    const long long items = (long long)p.W * p.H * p.nchunks;
    const unsigned b1 = (unsigned)std::max(1LL, std::min((items + 255) / 256, (long long)sms * 4));
    const bool scalar = p.nact == 1 && p.src[0].fdim == 1 && p.ch[0].n == 0;
    if (scalar && cell == 16)
        k_grid_columns_scalar<16><<<b1, 256, 0, st>>>(p);
    else if (scalar && cell == 8)
        k_grid_columns_scalar<8><<<b1, 256, 0, st>>>(p);
    else if (scalar)
        k_grid_columns<1, 1><<<b1, 256, 0, st>>>(p);
    else if (p.nact == 3)
        k_grid_columns<3, 0><<<b1, 256, 0, st>>>(p);
    else
        k_grid_columns<0, 0><<<b1, 256, 0, st>>>(p);
    rc = check_cuda("isaac_opacity_grid columns launch");
    if (rc) return rc;
    launch_grid_reduce(p, cells, sms, st);
    return check_cuda("isaac_opacity_grid reduce launch");
}

extern "C" int isaac_opacity_grid_packed(const isaac_packed *vol, const isaac_chain *chains,
                                         const float *luts, const float *weights,
                                         const isaac_render_opts *opts, int32_t cell, float *grid,
                                         int64_t grid_len, void *stream)
{
    clear_error();
    if (!vol || !chains || !weights || !opts || !grid || !luts)
        return fail(ISAAC_EINVAL, "vol, chains, luts, weights, opts and grid are required");
    if (vol->n_src < 1 || vol->n_src > ISAAC_MAX_ACTIVE)
        return fail(ISAAC_EINVAL, "packed volume has %d sources", vol->n_src);
    if (vol->dtype < ISAAC_F32 || vol->dtype > ISAAC_E4M3) return fail(ISAAC_EINVAL, "unknown dtype %d", vol->dtype);
    if (vol->pad != 1 && vol->pad != 2 && vol->pad != 4 && vol->pad != 8)
        return fail(ISAAC_EINVAL, "pad %d is not 1, 2, 4 or 8", vol->pad);
    int nc = 0;
    for (int i = 0; i < vol->n_src; ++i) {
        if (vol->f_dim[i] < 1 || vol->f_dim[i] > 4)
            return fail(ISAAC_EINVAL, "packed source %d: f_dim %d", i, vol->f_dim[i]);
        nc += vol->f_dim[i];
    }
    if (nc != vol->n_comp || nc > vol->pad) return fail(ISAAC_EINVAL, "inconsistent packed layout");
    if (!vol->data || ((uintptr_t)vol->data) % 16) return fail(ISAAC_EINVAL, "vol->data misaligned");
    if (vol->dtype == ISAAC_E4M3 && (!vol->scales || ((uintptr_t)vol->scales) % 16))
        return fail(ISAAC_EINVAL, "E4M3 volume needs 16-byte aligned scales");
    for (int a = 0; a < 3; ++a)
        if (opts->n[a] != vol->n[a]) return fail(ISAAC_EINVAL, "opts->n differs from the packed volume");
    if (opts->active_mask >> vol->n_src)
        return fail(ISAAC_EINVAL, "active_mask 0x%x has bits beyond the %d packed sources",
                    opts->active_mask, vol->n_src);
    if (cell < 2 || cell > 1024) return fail(ISAAC_EINVAL, "cell %d outside 2..1024", cell);
    if (((uintptr_t)luts) % 16) return fail(ISAAC_EINVAL, "luts must be 16-byte aligned");
    KGrid p;
    memset(&p, 0, sizeof p);
    p.nx = (int)vol->n[0];
    p.ny = (int)vol->n[1];
    p.nz = (int)vol->n[2];
    p.cell = cell;
    p.gx = (p.nx + cell - 1) / cell;
    p.gy = (p.ny + cell - 1) / cell;
    p.gz = (p.nz + cell - 1) / cell;
    const long long cells = (long long)p.gx * p.gy * p.gz;
    if (grid_len < cells)
        return fail(ISAAC_ENOMEM, "grid holds %lld values, %lld needed", (long long)grid_len, cells);
    int off = 0;
    for (int s = 0; s < vol->n_src; ++s) {
        if ((opts->active_mask >> s) & 1u) {
            if (!std::isfinite(weights[s])) return fail(ISAAC_EINVAL, "weight %d is not finite", s);
            int rc = compile_chain(chains[s], vol->f_dim[s], s, p.ch[p.nact]);
            if (rc) return rc;
            p.comp_off[p.nact] = off;
            p.fdim[p.nact] = vol->f_dim[s];
            p.src[p.nact].w = weights[s];
            p.lut[p.nact] = reinterpret_cast<const float4 *>(luts) + (size_t)s * 256;
            ++p.nact;
        }
        off += vol->f_dim[s];
    }
    p.grid = grid;
    const cudaStream_t st = (cudaStream_t)stream;
    if (p.nact == 0) {
        if (cudaMemsetAsync(grid, 0, (size_t)cells * sizeof(float), st) != cudaSuccess)
            return check_cuda("isaac_opacity_grid_packed memset");
        return ISAAC_OK;
    }
    p.rec = static_cast<const unsigned char *>(vol->data);
    p.scales = vol->scales;
    p.pbx = (p.nx + 9) / 8;
    p.pby = (p.ny + 9) / 8;
    p.W = p.nx + 2;
    p.H = p.ny + 2;
    p.kchunk = std::max(1, (64 + cell - 1) / cell);
    p.nchunks = (p.gz + p.kchunk - 1) / p.kchunk;
    const size_t col_bytes = (size_t)p.gz * (size_t)p.W * (size_t)p.H * sizeof(float);
    KParams wp;
    memset(&wp, 0, sizeof wp);
    if (opts->flags & ISAAC_LUTS_HOST) {   // staged into the workspace by bind_workspace
        for (int a = 0; a < p.nact; ++a) wp.lut[a] = p.lut[a];
        wp.luts_host = 1;
    }
    void *cols = nullptr;
    int rc = bind_workspace(wp, st, col_bytes + 16, &cols);
    if (rc) return rc;
    if (opts->flags & ISAAC_LUTS_HOST)   // the staged device copies
        for (int a = 0; a < p.nact; ++a) p.lut[a] = wp.lut[a];
    p.cols = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(cols) + 15) & ~uintptr_t(15));
    const int sms = sm_count();
    const long long items = (long long)p.W * p.H * p.nchunks;
    const unsigned b1 = (unsigned)std::max(1LL, std::min((items + 255) / 256, (long long)sms * 4));
#define ISAAC_GP(DT)                                                                              \
    switch (vol->pad) {                                                                           \
    case 1: k_grid_columns_packed<DT, 1><<<b1, 256, 0, st>>>(p); break;                           \
    case 2: k_grid_columns_packed<DT, 2><<<b1, 256, 0, st>>>(p); break;                           \
    case 4: k_grid_columns_packed<DT, 4><<<b1, 256, 0, st>>>(p); break;                           \
    default: k_grid_columns_packed<DT, 8><<<b1, 256, 0, st>>>(p); break;                          \
    }
    const bool scalar = p.nact == 1 && vol->pad == 1 && p.ch[0].n == 0 && vol->dtype != ISAAC_E4M3 &&
                        (cell == 8 || cell == 16);
    if (scalar && vol->dtype != ISAAC_F32 && p.W % 2 == 0) {
        const long long items2 = (long long)p.W / 2 * p.H * p.nchunks;
        const unsigned b2c = (unsigned)std::max(1LL, std::min((items2 + 255) / 256, (long long)sms * kScalarWalkBlocksPerSM));
#define ISAAC_GPS2(DT)                                                                            \
        if (cell == 16) k_grid_columns_packed_scalar2<DT, 16><<<b2c, 256, 0, st>>>(p);            \
        else k_grid_columns_packed_scalar2<DT, 8><<<b2c, 256, 0, st>>>(p);
        if (vol->dtype == ISAAC_BF16) {
            ISAAC_GPS2(ISAAC_BF16)
        } else {
            ISAAC_GPS2(ISAAC_F16)
        }
#undef ISAAC_GPS2
    } else if (scalar) {
#define ISAAC_GPS(DT)                                                                             \
        if (cell == 16) k_grid_columns_packed_scalar<DT, 16><<<b1, 256, 0, st>>>(p);              \
        else k_grid_columns_packed_scalar<DT, 8><<<b1, 256, 0, st>>>(p);
        switch (vol->dtype) {
        case ISAAC_F32: ISAAC_GPS(ISAAC_F32) break;
        case ISAAC_BF16: ISAAC_GPS(ISAAC_BF16) break;
        default: ISAAC_GPS(ISAAC_F16) break;
        }
#undef ISAAC_GPS
    } else {
        switch (vol->dtype) {
        case ISAAC_F32: ISAAC_GP(ISAAC_F32) break;
        case ISAAC_BF16: ISAAC_GP(ISAAC_BF16) break;
        case ISAAC_F16: ISAAC_GP(ISAAC_F16) break;
        default: ISAAC_GP(ISAAC_E4M3) break;
        }
    }
#undef ISAAC_GP
    rc = check_cuda("isaac_opacity_grid_packed columns launch");
    if (rc) return rc;
    launch_grid_reduce(p, cells, sms, st);
    return check_cuda("isaac_opacity_grid_packed reduce launch");
}

extern "C" int isaac_range_grid(const isaac_source *sources, int32_t n_sources,
                                const isaac_render_opts *opts, int32_t cell, float *ranges,
                                int64_t ranges_len, void *stream)
{
    clear_error();
    if (!sources || !opts || !ranges) return fail(ISAAC_EINVAL, "sources, opts and ranges are required");
    if (n_sources < 1 || n_sources > ISAAC_MAX_SOURCES)
        return fail(ISAAC_EINVAL, "n_sources %d outside 1..%d", n_sources, ISAAC_MAX_SOURCES);
    if (cell < 2 || cell > 1024) return fail(ISAAC_EINVAL, "cell %d outside 2..1024", cell);
    if (opts->active_mask >> n_sources) return fail(ISAAC_EINVAL, "active_mask beyond n_sources");
    if (((uintptr_t)ranges) % 8) return fail(ISAAC_EINVAL, "ranges must be 8-byte aligned");
    for (int a = 0; a < 3; ++a)
        if (opts->n[a] < 1 || opts->n[a] > (1 << 20)) return fail(ISAAC_EINVAL, "bad volume size");
    KRange r;
    memset(&r, 0, sizeof r);
    r.nx = (int)opts->n[0];
    r.ny = (int)opts->n[1];
    r.nz = (int)opts->n[2];
    r.cell = cell;
    r.gx = (r.nx + cell - 1) / cell;
    r.gy = (r.ny + cell - 1) / cell;
    r.gz = (r.nz + cell - 1) / cell;
    const long long cells = (long long)r.gx * r.gy * r.gz;
    KSource ks[ISAAC_MAX_SOURCES];
    int nact = 0, slots = 0;
    update_sources(n_sources, opts->active_mask);
    for (int s = 0; s < n_sources; ++s) {
        if (!((opts->active_mask >> s) & 1u)) continue;
        if (nact == ISAAC_MAX_ACTIVE) return fail(ISAAC_ENOTSUP, "more than %d active sources", ISAAC_MAX_ACTIVE);
        unsigned nib;
        bool wide;
        int rc = prepare_source(sources[s], s, opts->n, 1, 1.0f, 4, ks[nact], &nib, &wide);
        if (rc) return rc;
        slots += sources[s].f_dim;
        ++nact;
    }
    if (nact == 0) return fail(ISAAC_EINVAL, "active_mask selects no source");
    if (ranges_len < cells * slots * 2)
        return fail(ISAAC_ENOMEM, "ranges holds %lld floats, %lld needed", (long long)ranges_len,
                    cells * slots * 2);
    const cudaStream_t st = (cudaStream_t)stream;
    r.slots = slots;
    r.ranges = ranges;
    r.W = r.nx + 2;
    r.H = r.ny + 2;
    r.kchunk = std::max(1, (64 + cell - 1) / cell);
    r.nchunks = (r.gz + r.kchunk - 1) / r.kchunk;
    int fmax_src = 1;
    for (int a = 0; a < nact; ++a) fmax_src = std::max(fmax_src, ks[a].fdim);
    // per-column (min, max) pairs of one source at a time, in the stream's workspace
    const size_t col_bytes = (size_t)r.gz * (size_t)r.W * (size_t)r.H * (size_t)fmax_src * sizeof(float2);
    KParams wp;
    memset(&wp, 0, sizeof wp);
    void *cols = nullptr;
    int rc = bind_workspace(wp, st, col_bytes + 16, &cols);
    if (rc) return rc;
    r.cols = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(cols) + 15) & ~uintptr_t(15));
    const int sms = sm_count();
    const long long items = (long long)r.W * r.H * r.nchunks;
    const unsigned b1 = (unsigned)std::max(1LL, std::min((items + 255) / 256, (long long)sms * 4));
    const unsigned b1s = (unsigned)std::max(1LL, std::min((items + 255) / 256, (long long)sms * kScalarWalkBlocksPerSM));
    const unsigned b2 = (unsigned)std::max(1LL, std::min((cells * 32 + 255) / 256, (long long)sms * 8));
    int slot = 0;
    for (int a = 0; a < nact; ++a) {
        r.src = ks[a];
        r.slot0 = slot;
        switch (ks[a].fdim) {
        case 1:
            if (cell == 16) k_range_columns<1, 16><<<b1s, 256, 0, st>>>(r);
            else if (cell == 8) k_range_columns<1, 8><<<b1s, 256, 0, st>>>(r);
            else k_range_columns<1, 0><<<b1, 256, 0, st>>>(r);
            k_range_reduce<1><<<b2, 256, 0, st>>>(r);
            break;
        case 2:
            k_range_columns<2, 0><<<b1, 256, 0, st>>>(r);
            k_range_reduce<2><<<b2, 256, 0, st>>>(r);
            break;
        case 3:
            k_range_columns<3, 0><<<b1, 256, 0, st>>>(r);
            k_range_reduce<3><<<b2, 256, 0, st>>>(r);
            break;
        default:
            k_range_columns<4, 0><<<b1, 256, 0, st>>>(r);
            k_range_reduce<4><<<b2, 256, 0, st>>>(r);
            break;
        }
        slot += ks[a].fdim;
    }
    return check_cuda("isaac_range_grid launch");
}
