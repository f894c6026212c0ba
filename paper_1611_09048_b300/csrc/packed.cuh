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
    int ncomp;           // record slots in use: 0 .. ncomp-1
    int slot_src[8];     // source of record slot k (slots follow the sources in order)
    int slot_comp[8];    // its component
    int nx, ny, nz;      // interior cells
    int px, py, pz;      // packed box = n + 2
    int bx, by, bz;      // bricks per axis
    unsigned char *rec;
    float *scales;
};

// Source index along one axis for packed coordinate q (cell q - 1 of [-1, n]):
// the guard cell itself where the source has guards, else the border cell
// repeated (exactly what clamping reads).
__device__ __forceinline__ int pack_axis(int q, int n, int guard)
{
    return guard ? q - 1 : min(max(q - 1, 0), n - 1);
}

// One (y, z) row of the packed box: per record slot, the address of its
// component in source cell x = 0 of that row, the source's x stride and
// guard flag.  Rows are warp-uniform, so this is set up once per row.
template <int PAD>
struct PackRow {
    const float *p[PAD];
    long long sx[PAD];
    int guard[PAD];
};

template <int PAD>
__device__ __forceinline__ void pack_row(const KPack &p, int y, int z, PackRow<PAD> &r)
{
#pragma unroll
    for (int k = 0; k < PAD; ++k) {
        if (k < p.ncomp) {
            const KPackSrc &q = p.src[p.slot_src[k]];
            const int yi = pack_axis(y, p.ny, q.guard), zi = pack_axis(z, p.nz, q.guard);
            r.p[k] = q.base + ((long long)yi * q.sy + (long long)zi * q.sz + (long long)p.slot_comp[k] * q.sc);
            r.sx[k] = q.sx;
            r.guard[k] = q.guard;
        } else {
            r.p[k] = nullptr;
            r.sx[k] = 0;
            r.guard[k] = 0;
        }
    }
}

// All record slots of packed cell x of the row (float32; unused slots 0).
template <int PAD>
__device__ __forceinline__ void pack_cell(const KPack &p, const PackRow<PAD> &r, int x, float (&v)[PAD])
{
#pragma unroll
    for (int k = 0; k < PAD; ++k)
        v[k] = k < p.ncomp ? __ldg(r.p[k] + (long long)pack_axis(x, p.nx, r.guard[k]) * r.sx[k]) : 0.0f;
}

__device__ __forceinline__ unsigned short to16(float v, int dt)
{
    return dt == ISAAC_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v))
                            : __half_as_ushort(__float2half_rn(v));
}

// Two values rounded to 16 bits (nearest even) in one 4-byte word, lo in the
// low half: one paired conversion instead of two and a shift.
template <int DT>
__device__ __forceinline__ unsigned pack16x2(float lo, float hi)
{
    if constexpr (DT == ISAAC_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&h);
    } else {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&h);
    }
}

// Record i of the copy in one store as wide as the record (2 to 32 bytes;
// records are aligned to their size: the copy starts 16-byte aligned).
template <int DT, int PAD>
__device__ __forceinline__ void store_record(unsigned char *rec, long long i, const float (&v)[PAD])
{
    if constexpr (DT == ISAAC_F32) {
        float *o = reinterpret_cast<float *>(rec) + i * PAD;
        if constexpr (PAD == 1) {
            o[0] = v[0];
        } else if constexpr (PAD == 2) {
            *reinterpret_cast<float2 *>(o) = make_float2(v[0], v[1]);
        } else {
#pragma unroll
            for (int q = 0; q < PAD / 4; ++q)
                reinterpret_cast<float4 *>(o)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    } else {
        unsigned short *o = reinterpret_cast<unsigned short *>(rec) + i * PAD;
        if constexpr (PAD == 1) {
            o[0] = to16(v[0], DT);
        } else {
            unsigned w[PAD / 2];
#pragma unroll
            for (int c = 0; c < PAD / 2; ++c) w[c] = pack16x2<DT>(v[2 * c], v[2 * c + 1]);
            if constexpr (PAD == 2)
                *reinterpret_cast<unsigned *>(o) = w[0];
            else if constexpr (PAD == 4)
                *reinterpret_cast<uint2 *>(o) = make_uint2(w[0], w[1]);
            else
                *reinterpret_cast<uint4 *>(o) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// float32 / bfloat16 / float16: a warp per (y, z) row of the packed box, its
// lanes along x (coalesced source reads, contiguous record stores); rows are
// spread over the warps of the grid.
template <int DT, int PAD>
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ KPack p)
{
    const int lane = threadIdx.x & 31;
    const int rows = p.py * p.pz;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += nwarps) {
        const int z = r / p.py, y = r - z * p.py;
        PackRow<PAD> row;
        pack_row<PAD>(p, y, z, row);
        const long long i0 = (long long)r * p.px;
        if constexpr (PAD == 1 && DT != ISAAC_F32) {
            if ((p.px & 1) == 0) {
                // 2-byte records, rows of an even length: each lane converts
                // the cell pairs (x, x + 1), x even, and stores a pair as one
                // 4-byte word (rows start 4-byte aligned), 9 pairs' loads in
                // flight per lane
                constexpr int U2 = 9;
                unsigned *rec32 = reinterpret_cast<unsigned *>(p.rec);
                for (int xb = 2 * lane; xb < p.px; xb += 64 * U2) {
                    float v[U2][2];
#pragma unroll
                    for (int u = 0; u < U2; ++u) {
                        const int x = xb + 64 * u;
                        if (x < p.px) {
                            float a[1], b[1];
                            pack_cell<1>(p, row, x, a);
                            pack_cell<1>(p, row, x + 1, b);
                            v[u][0] = a[0];
                            v[u][1] = b[0];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U2; ++u) {
                        const int x = xb + 64 * u;
                        if (x < p.px)
                            rec32[(i0 + x) >> 1] = pack16x2<DT>(v[u][0], v[u][1]);
                    }
                }
                continue;
            }
        }
        // U cells per lane are loaded before any is stored, so that a lane
        // keeps U * ncomp loads in flight (the stores may alias the sources
        // as far as the compiler knows)
        constexpr int U = PAD <= 2 ? 8 : (PAD == 4 ? 4 : 2);
        for (int xb = lane; xb < p.px; xb += 32 * U) {
            float v[U][PAD];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (xb + 32 * u < p.px) pack_cell<PAD>(p, row, xb + 32 * u, v[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (xb + 32 * u < p.px) store_record<DT, PAD>(p.rec, i0 + xb + 32 * u, v[u]);
        }
    }
}

constexpr int kPackBricksX = 4;   // bricks along x per E4M3 pack block (32 lanes)

// The (x, y) column of one thread through the packed box: per record slot,
// the address of its component in source cell (x, y, z = 0), the source's z
// stride and guard flag.
template <int PAD>
struct PackColumn {
    const float *p[PAD];
    long long sz[PAD];
    int guard[PAD];
};

template <int PAD>
__device__ __forceinline__ void pack_column(const KPack &p, int x, int y, PackColumn<PAD> &c)
{
#pragma unroll
    for (int k = 0; k < PAD; ++k) {
        if (k < p.ncomp) {
            const KPackSrc &q = p.src[p.slot_src[k]];
            const int xi = pack_axis(x, p.nx, q.guard), yi = pack_axis(y, p.ny, q.guard);
            c.p[k] = q.base + ((long long)xi * q.sx + (long long)yi * q.sy + (long long)p.slot_comp[k] * q.sc);
            c.sz[k] = q.sz;
            c.guard[k] = q.guard;
        } else {
            c.p[k] = nullptr;
            c.sz[k] = 0;
            c.guard[k] = 0;
        }
    }
}

template <int PAD>
__device__ __forceinline__ void column_cell(const KPack &p, const PackColumn<PAD> &c, int z, float (&v)[PAD])
{
#pragma unroll
    for (int k = 0; k < PAD; ++k)
        v[k] = k < p.ncomp ? __ldg(c.p[k] + (long long)pack_axis(z, p.nz, c.guard[k]) * c.sz[k]) : 0.0f;
}

// v / s rounded once to float32 (round to nearest even), given y = RN(1/s)
// and s in [2^-60, 2^60], by Markstein's method (P. Markstein, IBM J. Res.
// Dev. 34(1), 1990): q0 = RN(v y) lies within 1.5 ulp of v / s; one step
// with the fused multiply-add residual v - s q0 makes q1 faithful (within an
// ulp); the residual of a faithful quotient is exact, and Markstein's theorem
// makes RN(q1 + (v - s q1) y) the correctly rounded quotient.  The range of s
// keeps that residual in the normal range for every v with |v / s| >= 2^-11;
// smaller quotients stay below 2^-10, half of E4M3's smallest subnormal, so
// they quantise to a zero of v's sign either way, as the correctly rounded
// quotient does.  The residual is formed negated, s q - v, and subtracted:
// for v = -0 that keeps the quotient -0 (q + (+0) y would round to +0).
__device__ __forceinline__ float quot_rn(float v, float s, float y)
{
    const float q0 = v * y;
    const float q1 = fmaf(-fmaf(s, q0, -v), y, q0);
    return fmaf(-fmaf(s, q1, -v), y, q1);
}

template <int PAD, bool FAST>
__device__ __forceinline__ void store_e4m3(const KPack &p, const float (&v)[PAD], const float (&sc)[PAD],
                                           const float (&rc)[PAD], unsigned char *o)
{
    // quotients of unused slots are 0, which converts to the code 0
    float q[PAD];
#pragma unroll
    for (int k = 0; k < PAD; ++k)
        q[k] = k < p.ncomp ? (FAST ? quot_rn(v[k], sc[k], rc[k]) : __fdiv_rn(v[k], sc[k])) : 0.0f;
    if constexpr (PAD == 1) {
        *o = (unsigned char)__nv_cvt_float_to_fp8(q[0], __NV_SATFINITE, __NV_E4M3);
    } else {
        // slots 2c and 2c + 1 in one paired conversion (2c in the low byte)
        unsigned h[PAD / 2];
#pragma unroll
        for (int c = 0; c < PAD / 2; ++c)
            h[c] = (unsigned)__nv_cvt_float2_to_fp8x2(make_float2(q[2 * c], q[2 * c + 1]), __NV_SATFINITE,
                                                      __NV_E4M3);
        if constexpr (PAD == 2)
            *reinterpret_cast<unsigned short *>(o) = (unsigned short)h[0];
        else if constexpr (PAD == 4)
            *reinterpret_cast<unsigned *>(o) = h[0] | (h[1] << 16);
        else
            *reinterpret_cast<uint2 *>(o) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    }
}

// E4M3: a 256-thread block per 4 x 1 x 1 bricks: lane = x (8 lanes per brick),
// warp = y, each thread down its column through the brick's 8 z layers.  The
// column's cells are read once, all their loads in flight together, and stay
// in registers: per thread the absmax of each slot over its cells, reduced
// over the brick's 8 lanes by shuffles and over the 8 warps in shared memory;
// scale = absmax / 448 (1 for an all-zero brick); then, from the registers,
// code = E4M3_sat(v / scale) with v / scale rounded once to float32 (by
// quot_rn when every scale of the block lies in [2^-60, 2^60], else by the
// division), one store of the cell's PAD codes.
template <int PAD>
__global__ void __launch_bounds__(256) k_pack_e4m3(const __grid_constant__ KPack p)
{
    __shared__ float s_max[8][kPackBricksX][PAD];
    __shared__ float s_scale[kPackBricksX][PAD];
    __shared__ float s_rcp[kPackBricksX][PAD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = (p.bx + kPackBricksX - 1) / kPackBricksX;
    const int b = blockIdx.x;
    const int bxi = (b % gx) * kPackBricksX, byi = (b / gx) % p.by, bzi = b / (gx * p.by);
    const int x = bxi * 8 + lane, y = byi * 8 + warp;   // packed coordinates
    const bool in_xy = x < p.px && y < p.py;
    const int z0 = bzi * 8, nzb = min(8, p.pz - z0);
    PackColumn<PAD> col;
    pack_column<PAD>(p, in_xy ? x : 0, in_xy ? y : 0, col);
    float v[8][PAD];
    float m[PAD];
#pragma unroll
    for (int k = 0; k < PAD; ++k) m[k] = 0.0f;
    if (in_xy) {
        if (z0 >= 1 && z0 + 8 <= p.nz) {
            // a brick inside the source along z: source layer z - 1 for every
            // slot, guards or not, so each slot's address advances by its z
            // stride from one cell to the next
#pragma unroll
            for (int k = 0; k < PAD; ++k) {
                const float *a = col.p[k] + (long long)(z0 - 1) * col.sz[k];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u][k] = k < p.ncomp ? __ldg(a + u * col.sz[k]) : 0.0f;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u < nzb) column_cell<PAD>(p, col, z0 + u, v[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < nzb) {
#pragma unroll
                for (int k = 0; k < PAD; ++k) m[k] = fmaxf(m[k], fabsf(v[u][k]));
            }
    }
#pragma unroll
    for (int k = 0; k < PAD; ++k) {
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) m[k] = fmaxf(m[k], __shfl_xor_sync(0xffffffffu, m[k], o));
        if ((lane & 7) == 0) s_max[warp][lane >> 3][k] = m[k];
    }
    __syncthreads();
    bool in_range = true;
    if (threadIdx.x < kPackBricksX * PAD) {
        const int j = threadIdx.x / PAD, k = threadIdx.x - j * PAD;
        float a = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) a = fmaxf(a, s_max[w][j][k]);
        const float sc = a > 0.0f ? __fdiv_rn(a, 448.0f) : 1.0f;
        in_range = sc >= 0x1p-60f && sc <= 0x1p60f;
        s_scale[j][k] = sc;
        s_rcp[j][k] = in_range ? __frcp_rn(sc) : 0.0f;
        if (bxi + j < p.bx)
            p.scales[(((long long)bzi * p.by + byi) * p.bx + bxi + j) * PAD + k] = sc;
    }
    const bool fast = __syncthreads_and(in_range) != 0;
    if (!in_xy) return;
    float sc[PAD], rc[PAD];
#pragma unroll
    for (int k = 0; k < PAD; ++k) {
        sc[k] = s_scale[lane >> 3][k];
        rc[k] = s_rcp[lane >> 3][k];
    }
    unsigned char *o = p.rec + (((long long)z0 * p.py + y) * p.px + x) * PAD;
    const long long zstep = (long long)p.py * p.px * PAD;
    if (fast) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < nzb) store_e4m3<PAD, true>(p, v[u], sc, rc, o + u * zstep);
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < nzb) store_e4m3<PAD, false>(p, v[u], sc, rc, o + u * zstep);
    }
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
    // the empty-group vote in single-source kernels only (as in k_raycast)
    const bool zskip = load_luts<NACT>(p, s_lut);
    using Shader = PackedShader<NACT, SIG, DT, PAD, INTERP>;
    if constexpr (LONG) {
        if (NACT == 1 && zskip)
            march_long<Shader, NACT == 1>(p, s_lut);
        else
            march_long<Shader, false>(p, s_lut);
    } else if (NACT == 1 && zskip) {
        march<NACT, Shader, RL, false, false, NACT == 1>(p, s_lut);
    } else {
        march<NACT, Shader, RL, false, false, false>(p, s_lut);
    }
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
