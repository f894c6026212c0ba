// packed.cuh -- reduced-precision storage of the sources and the ray caster
// that samples it (sm_103a).
//
// The pack kernel copies every active source into one record per cell over
// the cells [-1, n]^3: guard cells where the source has them, otherwise the
// border cell repeated (which is exactly what clamping reads), so the render
// kernel needs no border logic.  A record holds `PAD` components (all
// sources' components of the cell, source after source) as float32,
// bfloat16, float16 or FP8 E4M3; E4M3 additionally stores one float32 scale
// per 8^3 brick (bricks counted from cell -1) and component:
// scale = absmax / 448, code = E4M3(value / scale), saturating.  Sampling
// loads one record per trilinear corner (one 16-byte load for up to 8
// 16-bit components) and accumulates everything in float32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "raycast.cuh"

namespace isaac {

// --------------------------------------------------------------- records

template <int DT, int PAD>
struct RecIO;

// float32
template <int PAD>
struct RecIO<ISAAC_F32, PAD> {
    static constexpr int BYTES = 4 * PAD;
    __device__ static void load(const unsigned char *base, long long i, float (&v)[PAD])
    {
        const float *p = reinterpret_cast<const float *>(base) + i * PAD;
        if constexpr (PAD == 1) {
            v[0] = __ldg(p);
        } else if constexpr (PAD == 2) {
            const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
            v[0] = a.x; v[1] = a.y;
        } else {
#pragma unroll
            for (int q = 0; q < PAD / 4; ++q) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(p) + q);
                v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
            }
        }
    }
};

__device__ __forceinline__ float bf16_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float f16_lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
__device__ __forceinline__ float f16_hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

template <int DT>
__device__ __forceinline__ void unpack2(unsigned w, float &a, float &b)
{
    if constexpr (DT == ISAAC_BF16) {
        a = bf16_lo(w);
        b = bf16_hi(w);
    } else {
        a = f16_lo(w);
        b = f16_hi(w);
    }
}

// 16-bit formats
template <int DT, int PAD>
struct Rec16 {
    static constexpr int BYTES = 2 * PAD;
    __device__ static void load(const unsigned char *base, long long i, float (&v)[PAD])
    {
        const unsigned short *p = reinterpret_cast<const unsigned short *>(base) + i * PAD;
        if constexpr (PAD == 1) {
            const unsigned w = __ldg(p);
            float dummy;
            unpack2<DT>(w, v[0], dummy);
        } else if constexpr (PAD == 2) {
            const unsigned w = __ldg(reinterpret_cast<const unsigned *>(p));
            unpack2<DT>(w, v[0], v[1]);
        } else if constexpr (PAD == 4) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
            unpack2<DT>(w.x, v[0], v[1]);
            unpack2<DT>(w.y, v[2], v[3]);
        } else {
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
            unpack2<DT>(w.x, v[0], v[1]);
            unpack2<DT>(w.y, v[2], v[3]);
            unpack2<DT>(w.z, v[4], v[5]);
            unpack2<DT>(w.w, v[6], v[7]);
        }
    }
};
template <int PAD>
struct RecIO<ISAAC_BF16, PAD> : Rec16<ISAAC_BF16, PAD> {};
template <int PAD>
struct RecIO<ISAAC_F16, PAD> : Rec16<ISAAC_F16, PAD> {};

// FP8 E4M3 codes (scaled separately)
__device__ __forceinline__ void e4m3x2(unsigned short w, float &a, float &b)
{
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)w, __NV_E4M3);
    const __half2 hh = *reinterpret_cast<const __half2 *>(&h);
    const float2 f = __half22float2(hh);
    a = f.x;
    b = f.y;
}

template <int PAD>
struct RecIO<ISAAC_E4M3, PAD> {
    static constexpr int BYTES = PAD;
    __device__ static void load(const unsigned char *base, long long i, float (&v)[PAD])
    {
        const unsigned char *p = base + i * PAD;
        if constexpr (PAD == 1) {
            float dummy;
            e4m3x2((unsigned short)__ldg(p), v[0], dummy);
        } else if constexpr (PAD == 2) {
            e4m3x2(__ldg(reinterpret_cast<const unsigned short *>(p)), v[0], v[1]);
        } else if constexpr (PAD == 4) {
            const unsigned w = __ldg(reinterpret_cast<const unsigned *>(p));
            e4m3x2((unsigned short)(w & 0xffffu), v[0], v[1]);
            e4m3x2((unsigned short)(w >> 16), v[2], v[3]);
        } else {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
            e4m3x2((unsigned short)(w.x & 0xffffu), v[0], v[1]);
            e4m3x2((unsigned short)(w.x >> 16), v[2], v[3]);
            e4m3x2((unsigned short)(w.y & 0xffffu), v[4], v[5]);
            e4m3x2((unsigned short)(w.y >> 16), v[6], v[7]);
        }
    }
};

template <int PAD>
__device__ __forceinline__ void load_scales(const float *s, int brick, float (&v)[PAD])
{
    const float *p = s + brick * PAD;
    if constexpr (PAD == 1) {
        v[0] = __ldg(p);
    } else if constexpr (PAD == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = a.x; v[1] = a.y;
    } else {
#pragma unroll
        for (int q = 0; q < PAD / 4; ++q) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(p) + q);
            v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
        }
    }
}

// ------------------------------------------------------------ pack kernels

struct KPackSrc {
    const float *base;   // interior cell (0,0,0), component 0
    long long sx, sy, sz, sc;
    int fdim;
    int guard;
};

struct KPack {
    KPackSrc src[ISAAC_MAX_ACTIVE];
    int nsrc;
    int nx, ny, nz;      // interior cells
    int px, py, pz;      // packed box = n + 2
    int bx, by, bz;      // bricks per axis
    unsigned char *rec;
    float *scales;
};

// All components of packed cell (x, y, z) in [-1, n]^3 (float32).
template <int PAD>
__device__ __forceinline__ void gather_cell(const KPack &p, int x, int y, int z, float (&v)[PAD])
{
#pragma unroll
    for (int c = 0; c < PAD; ++c) v[c] = 0.0f;
    int c0 = 0;
#pragma unroll
    for (int s = 0; s < ISAAC_MAX_ACTIVE; ++s) {
        if (s >= p.nsrc) break;
        const KPackSrc &q = p.src[s];
        int xi = x, yi = y, zi = z;
        if (q.guard == 0) {    // no neighbour data: repeat the border cell
            xi = min(max(xi, 0), p.nx - 1);
            yi = min(max(yi, 0), p.ny - 1);
            zi = min(max(zi, 0), p.nz - 1);
        }
        const float *b = q.base + ((long long)xi * q.sx + (long long)yi * q.sy + (long long)zi * q.sz);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < q.fdim) {
                const int slot = c0 + c;
#pragma unroll
                for (int k = 0; k < PAD; ++k)
                    if (k == slot) v[k] = __ldg(b + (long long)c * q.sc);
            }
        c0 += q.fdim;
    }
}

template <int DT, int PAD>
__device__ __forceinline__ void store_record(unsigned char *rec, long long i, const float (&v)[PAD])
{
    if constexpr (DT == ISAAC_F32) {
        float *o = reinterpret_cast<float *>(rec) + i * PAD;
#pragma unroll
        for (int c = 0; c < PAD; ++c) o[c] = v[c];
    } else {
        unsigned short h[PAD];
#pragma unroll
        for (int c = 0; c < PAD; ++c) {
            if constexpr (DT == ISAAC_BF16)
                h[c] = __bfloat16_as_ushort(__float2bfloat16_rn(v[c]));
            else
                h[c] = __half_as_ushort(__float2half_rn(v[c]));
        }
        unsigned short *o = reinterpret_cast<unsigned short *>(rec) + i * PAD;
#pragma unroll
        for (int c = 0; c < PAD; ++c) o[c] = h[c];
    }
}

// float32 / bfloat16 / float16: one thread per packed cell.
template <int DT, int PAD>
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ KPack p)
{
    const long long total = (long long)p.px * p.py * p.pz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.px);
        const long long r = i / p.px;
        const int y = (int)(r % p.py);
        const int z = (int)(r / p.py);
        float v[PAD];
        gather_cell<PAD>(p, x - 1, y - 1, z - 1, v);
        store_record<DT, PAD>(const_cast<unsigned char *>(p.rec), i, v);
    }
}

// E4M3: one 512-thread block per 8^3 brick; block-wide absmax per component,
// scale = absmax / 448 (1 for an all-zero brick), code = E4M3_sat(v / scale).
template <int PAD>
__global__ void __launch_bounds__(512) k_pack_e4m3(const __grid_constant__ KPack p)
{
    __shared__ float s_max[16][PAD];
    const int b = blockIdx.x;
    const int bxi = b % p.bx, byi = (b / p.bx) % p.by, bzi = b / (p.bx * p.by);
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    const int x = bxi * 8 + lx, y = byi * 8 + ly, z = bzi * 8 + lz;   // packed coordinates
    const bool inside = x < p.px && y < p.py && z < p.pz;
    float v[PAD];
    if (inside) {
        gather_cell<PAD>(p, x - 1, y - 1, z - 1, v);
    } else {
#pragma unroll
        for (int c = 0; c < PAD; ++c) v[c] = 0.0f;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < PAD; ++c) {
        float m = fabsf(v[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_max[warp][c] = m;
    }
    __syncthreads();
    float scale[PAD];
#pragma unroll
    for (int c = 0; c < PAD; ++c) {
        float m = 0.0f;
#pragma unroll
        for (int w = 0; w < 16; ++w) m = fmaxf(m, s_max[w][c]);
        scale[c] = m > 0.0f ? __fdiv_rn(m, 448.0f) : 1.0f;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < PAD; ++c) p.scales[(long long)b * PAD + c] = scale[c];
    }
    if (!inside) return;
    const long long i = ((long long)z * p.py + y) * p.px + x;
    unsigned char code[PAD];
#pragma unroll
    for (int c = 0; c < PAD; ++c)
        code[c] = (unsigned char)__nv_cvt_float_to_fp8(__fdiv_rn(v[c], scale[c]), __NV_SATFINITE, __NV_E4M3);
    unsigned char *o = const_cast<unsigned char *>(p.rec) + i * PAD;
#pragma unroll
    for (int c = 0; c < PAD; ++c) o[c] = code[c];
}

// ---------------------------------------------------------- render kernel

// Per-source component slice of the interpolated record.  With a known
// signature the offsets are compile-time; otherwise they are selected.
template <int PAD>
__device__ __forceinline__ float pick(const float (&v)[PAD], int k)
{
    float r = 0.0f;
#pragma unroll
    for (int j = 0; j < PAD; ++j)
        if (j == k) r = v[j];
    return r;
}

template <unsigned SIG, int I>
struct SigOff {
    static constexpr int value = sig_fdim(SIG, I - 1) + SigOff<SIG, I - 1>::value;
};
template <unsigned SIG>
struct SigOff<SIG, 0> {
    static constexpr int value = 0;
};

template <int I, unsigned SIG, int PAD>
__device__ __forceinline__ void shade_packed(const KParams &p, const float (&v)[PAD],
                                             const float4 *s_lut, float4 &acc)
{
    float in[4];
    if constexpr (SIG != 0) {
        constexpr int FD = sig_fdim(SIG, I);
        constexpr int OFF = SigOff<SIG, I>::value;
#pragma unroll
        for (int c = 0; c < 4; ++c) in[c] = (c < FD && OFF + c < PAD) ? v[(OFF + c) % PAD] : 0.0f;
    } else {
        const int off = p.comp_off[I], fd = p.src[I].fdim;
#pragma unroll
        for (int c = 0; c < 4; ++c) in[c] = c < fd ? pick<PAD>(v, off + c) : 0.0f;
    }
    const float x = run_chain(p.ch[I], in);
    const float4 c = classify(lut_of<I>(p, s_lut), x);
    const float w = p.src[I].w;
    acc.x = fmaf(w, c.x, acc.x);
    acc.y = fmaf(w, c.y, acc.y);
    acc.z = fmaf(w, c.z, acc.z);
    acc.w = fmaf(w, c.w, acc.w);
}

template <unsigned SIG, int PAD, int... Is>
__device__ __forceinline__ void shade_packed_all(const KParams &p, const float (&v)[PAD],
                                                 const float4 *s_lut, float4 &acc,
                                                 std::integer_sequence<int, Is...>)
{
    (shade_packed<Is, SIG, PAD>(p, v, s_lut, acc), ...);
}

template <int DT, int PAD, int INTERP>
__device__ __forceinline__ void sample_packed(const KParams &p, const Geo &g, float (&v)[PAD])
{
    using IO = RecIO<DT, PAD>;
    const long long PX = p.nx + 2, PY = p.ny + 2;
    if (!INTERP) {
        const int x = min(max(g.ix, 0), p.nx - 1) + 1;
        const int y = min(max(g.iy, 0), p.ny - 1) + 1;
        const int z = min(max(g.iz, 0), p.nz - 1) + 1;
        IO::load(p.rec, ((long long)z * PY + y) * PX + x, v);
        if constexpr (DT == ISAAC_E4M3) {
            float s[PAD];
            load_scales<PAD>(p.scales, ((z >> 3) * p.by + (y >> 3)) * p.bx + (x >> 3), s);
#pragma unroll
            for (int c = 0; c < PAD; ++c) v[c] *= s[c];
        }
        return;
    }
    // corners in packed coordinates (cell -1 -> 0), clamped into the box; the
    // record of corner 000 in 64 bits, the other corners at 32-bit offsets
    // from it (a plane of the copy holds at most 4098^2 records)
    const int x0 = min(max(g.ix, -1), p.nx) + 1, x1 = min(max(g.ix + 1, -1), p.nx) + 1;
    const int y0 = min(max(g.iy, -1), p.ny) + 1, y1 = min(max(g.iy + 1, -1), p.ny) + 1;
    const int z0 = min(max(g.iz, -1), p.nz) + 1, z1 = min(max(g.iz + 1, -1), p.nz) + 1;
    const unsigned char *r000 = p.rec + (((long long)z0 * PY + y0) * PX + x0) * IO::BYTES;
    const int ox = x1 - x0, oy = (y1 - y0) * (int)PX, oz = (z1 - z0) * (int)(PX * PY);
    if constexpr (DT == ISAAC_E4M3) {
        // each corner may lie in another brick: accumulate weight * scale * code
        // corner by corner (keeps one corner's record live at a time)
#pragma unroll
        for (int q = 0; q < PAD; ++q) v[q] = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = (k & 1) ? x1 : x0, y = (k & 2) ? y1 : y0, z = (k & 4) ? z1 : z0;
            const float w = g.w[k];
            float cv[PAD], s[PAD];
            IO::load(r000, ((k & 1) ? ox : 0) + ((k & 2) ? oy : 0) + ((k & 4) ? oz : 0), cv);
            load_scales<PAD>(p.scales, ((z >> 3) * p.by + (y >> 3)) * p.bx + (x >> 3), s);
#pragma unroll
            for (int q = 0; q < PAD; ++q) v[q] = fmaf(w * s[q], cv[q], v[q]);
        }
        return;
    }
    float c[8][PAD];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        IO::load(r000, ((k & 1) ? ox : 0) + ((k & 2) ? oy : 0) + ((k & 4) ? oz : 0), c[k]);
    }
#pragma unroll
    for (int q = 0; q < PAD; ++q) {
        v[q] = tri(g, c[0][q], c[1][q], c[2][q], c[3][q], c[4][q], c[5][q], c[6][q], c[7][q]);
    }
}

// Blended RGBA of one sample of the packed copy.  SIG != 0: the NACT packed
// sources with compile-time f_dim (inactive ones carry weight 0).  SIG == 0:
// run-time f_dim and record offsets.
template <int NACT, unsigned SIG, int DT, int PAD, int INTERP>
struct PackedShader {
    __device__ __forceinline__ static float4 shade(const KParams &p, const float4 *s_lut, float x,
                                                   float y, float z)
    {
        const Geo g = sample_geo<INTERP>(x, y, z);
        float v[PAD];
        sample_packed<DT, PAD, INTERP>(p, g, v);
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        shade_packed_all<SIG, PAD>(p, v, s_lut, acc, std::make_integer_sequence<int, NACT>{});
        return acc;
    }
};

// LONG: the long-ray march (MODE_LONG of k_raycast) instead of the march.
template <int NACT, unsigned SIG, int DT, int PAD, int INTERP, int RL, bool LONG = false>
__global__ void __launch_bounds__(kMarchThreads, kMarchBlocksPerSM) k_raycast_packed(const __grid_constant__ KParams p)
{
    __shared__ float4 s_lut[NACT * 256];
    load_luts<NACT>(p, s_lut);
    using Shader = PackedShader<NACT, SIG, DT, PAD, INTERP>;
    if constexpr (LONG)
        march_long<Shader>(p, s_lut);
    else
        march<NACT, Shader, RL>(p, s_lut);
}

// ------------------------------------------------------------- dispatch

using PackedLaunch = void (*)(const KParams &, dim3, cudaStream_t);
using PackLaunch = void (*)(const KPack &, cudaStream_t);

// Specialised signatures of the packed path (f_dim per packed source).
constexpr unsigned k_packed_sigs[] = {0x1u, 0x3u, 0x11u, 0x31u, 0x33u, 0x133u};
constexpr int k_n_packed_sigs = 6;

struct PackedEntry {
    int nact;
    unsigned sig;        // 0 = generic (pad 8)
    int pad;
    int interp;
    int rl;
    bool longpass;       // the long-ray march
    PackedLaunch fn;
};

struct PackedTable {
    const PackedEntry *entries;
    int n_entries;
    PackLaunch pack[4];  // [log2 pad]
};

}  // namespace isaac
