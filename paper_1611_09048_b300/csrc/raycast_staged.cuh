// raycast_staged.cuh -- the staged zero-copy march (sm_103a), an alternative
// to the gather march of raycast.cuh selected by ISAAC_MARCH_STAGED.
//
// One thread per ray: a warp marches the 32 rays of one list chunk (one 8x4
// pixel patch of ray setup) slab by slab, up to kStageSlab samples of each ray
// per slab (halved until the box fits).  Per slab the warp reduces its live
// rays' trilinear corner boxes to
// one box of cells (the corners of a ray's samples lie between those of its
// first and last sample of the slab: positions are monotone in the sample
// index), copies that box of every source into its shared buffer with
// coalesced loads (one float, or one float4 of up to 4 components, per cell),
// and every lane then gathers its samples' corners from shared memory.  A box
// larger than the buffer is read from global memory for that slab instead.
// The corner values, the arithmetic and the compositing order are those of
// march_ray, so the image is the gather march's bit for bit.  The warp stops
// when a vote finds no live ray.
#pragma once

#include "raycast.cuh"

namespace isaac {

constexpr int kStageSlab = 16;       // most samples per ray and slab (halved, down to 2, until the box fits)
constexpr int kStageWarps = 4;       // warps per block
constexpr int kStageBlocksPerSM = 4; // 16 warps per SM, at most 128 registers per thread
constexpr int kStageBytes = 10240;   // shared buffer per warp

// A staged cell takes one float in a scalar source's region, one float4 (up
// to 4 components) otherwise.  Offset of source I's region per 4 cells of the
// box (regions hold a multiple of 4 cells, so every region starts 16-byte
// aligned).
template <unsigned SIG, int I>
__host__ __device__ constexpr int stage_region_quads()
{
    int q = 0;
    for (int j = 0; j < I; ++j) q += sig_fdim(SIG, j) == 1 ? 16 : 64;
    return q;
}

template <unsigned SIG, int NACT>
__host__ __device__ constexpr int stage_bytes_per_cell()
{
    int b = 0;
    for (int j = 0; j < NACT; ++j) b += sig_fdim(SIG, j) == 1 ? 4 : 16;
    return b;
}

// The staged box of one slab: origin and extents in (clamped) cell indices.
struct StageBox {
    int bx, by, bz;      // lowest cell per axis
    int ex, exy;         // cells per row, per plane
    int quads;           // cells of a region / 4
};

// Copy cell i of the box of source I into its region.
template <int I, unsigned SIG, typename Idx>
__device__ __forceinline__ void stage_cell(const KParams &p, unsigned char *buf, const StageBox &b, int i,
                                           int x, int y, int z)
{
    constexpr int FD = sig_fdim(SIG, I);
    const KSource &s = p.src[I];
    const float *c = s.base + (Idx(x) * Idx(s.sx) + Idx(y) * Idx(s.sy) + Idx(z) * Idx(s.sz));
    unsigned char *reg = buf + stage_region_quads<SIG, I>() * b.quads;
    if constexpr (FD == 1) {
        reinterpret_cast<float *>(reg)[i] = __ldg(c);
    } else {
        const Idx cs = sig_aos(SIG, I) ? Idx(1) : Idx(s.sc);
        float4 v;
        v.x = __ldg(c);
        v.y = FD > 1 ? __ldg(c + cs) : 0.0f;
        v.z = FD > 2 ? __ldg(c + 2 * cs) : 0.0f;
        v.w = FD > 3 ? __ldg(c + 3 * cs) : 0.0f;
        reinterpret_cast<float4 *>(reg)[i] = v;
    }
}

template <unsigned SIG, typename Idx, int... Is>
__device__ __forceinline__ void stage_box(const KParams &p, unsigned char *buf, const StageBox &b, int cells,
                                          int lane, std::integer_sequence<int, Is...>)
{
    // cells < 2^12: the float quotients below are exact after truncation
    const float inv_exy = 1.0f / (float)b.exy, inv_ex = 1.0f / (float)b.ex;
#pragma unroll 2
    for (int i = lane; i < cells; i += 32) {
        const int z = (int)(((float)i + 0.5f) * inv_exy);
        const int rem = i - z * b.exy;
        const int y = (int)(((float)rem + 0.5f) * inv_ex);
        const int x = rem - y * b.ex;
        (stage_cell<Is, SIG, Idx>(p, buf, b, i, b.bx + x, b.by + y, b.bz + z), ...);
    }
}

// Value of source I at the sample from the staged box (o[k]: box index of
// trilinear corner k, as in Geo::w).
template <int I, unsigned SIG>
__device__ __forceinline__ void fetch_staged(const Geo &g, const unsigned char *buf, const StageBox &b,
                                             const int (&o)[8], float v[4])
{
    constexpr int FD = sig_fdim(SIG, I);
    const unsigned char *reg = buf + stage_region_quads<SIG, I>() * b.quads;
    if constexpr (FD == 1) {
        const float *f = reinterpret_cast<const float *>(reg);
        v[0] = tri(g, f[o[0]], f[o[1]], f[o[2]], f[o[3]], f[o[4]], f[o[5]], f[o[6]], f[o[7]]);
        v[1] = v[2] = v[3] = 0.0f;
    } else {
        const float4 *f = reinterpret_cast<const float4 *>(reg);
        const float4 c0 = f[o[0]], c1 = f[o[1]], c2 = f[o[2]], c3 = f[o[3]];
        const float4 c4 = f[o[4]], c5 = f[o[5]], c6 = f[o[6]], c7 = f[o[7]];
        v[0] = tri(g, c0.x, c1.x, c2.x, c3.x, c4.x, c5.x, c6.x, c7.x);
        v[1] = FD > 1 ? tri(g, c0.y, c1.y, c2.y, c3.y, c4.y, c5.y, c6.y, c7.y) : 0.0f;
        v[2] = FD > 2 ? tri(g, c0.z, c1.z, c2.z, c3.z, c4.z, c5.z, c6.z, c7.z) : 0.0f;
        v[3] = FD > 3 ? tri(g, c0.w, c1.w, c2.w, c3.w, c4.w, c5.w, c6.w, c7.w) : 0.0f;
    }
}

template <unsigned SIG, int... Is>
__device__ __forceinline__ float4 shade_staged(const KParams &p, const float4 *s_lut, const unsigned char *buf,
                                               const StageBox &b, float x, float y, float z,
                                               std::integer_sequence<int, Is...>)
{
    const Geo g = sample_geo<1>(x, y, z);
    // every source has the same readable range (the host's condition for staging)
    const KSource &s = p.src[0];
    const int x0 = min(max(g.ix, s.lo), p.nx - 1 + s.hi_pad) - b.bx;
    const int x1 = min(max(g.ix + 1, s.lo), p.nx - 1 + s.hi_pad) - b.bx;
    const int y0 = (min(max(g.iy, s.lo), p.ny - 1 + s.hi_pad) - b.by) * b.ex;
    const int y1 = (min(max(g.iy + 1, s.lo), p.ny - 1 + s.hi_pad) - b.by) * b.ex;
    const int z0 = (min(max(g.iz, s.lo), p.nz - 1 + s.hi_pad) - b.bz) * b.exy;
    const int z1 = (min(max(g.iz + 1, s.lo), p.nz - 1 + s.hi_pad) - b.bz) * b.exy;
    const int o[8] = {z0 + y0 + x0, z0 + y0 + x1, z0 + y1 + x0, z0 + y1 + x1,
                      z1 + y0 + x0, z1 + y0 + x1, z1 + y1 + x0, z1 + y1 + x1};
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    ([&] {
        float v[4];
        fetch_staged<Is, SIG>(g, buf, b, o, v);
        const float xv = run_chain(p.ch[Is], v);
        blend(acc, p.src[Is].w, classify(lut_of<Is>(p, s_lut), xv));
    }(), ...);
    return acc;
}

// Lowest trilinear corner cell of a sample along one axis (sample_geo's).
__device__ __forceinline__ int corner_lo(float s, float d, float e) { return (int)floorf(fmaf(s, d, e) - 0.5f); }

template <int NACT, unsigned SIG, typename Idx>
__device__ __forceinline__ void march_staged(const KParams &p, const float4 *s_lut, unsigned char *buf)
{
    using Shader = ZeroCopyShader<NACT, SIG, 1, Idx, false>;
    using Seq = std::make_integer_sequence<int, NACT>;
    constexpr int kCellBytes = stage_bytes_per_cell<SIG, NACT>();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned n_rays = *(volatile unsigned *)&p.ctr->n_rays;
    const unsigned cap = (unsigned)max(p.grab, 1);
    const unsigned per_take = 32u * 2u * gridDim.x * (blockDim.x >> 5);
    const KSource &s0 = p.src[0];
    const int lo = s0.lo, hx = p.nx - 1 + s0.hi_pad, hy = p.ny - 1 + s0.hi_pad, hz = p.nz - 1 + s0.hi_pad;
    unsigned last = 0;
    for (;;) {
        const unsigned grab = min(max((n_rays - min(last, n_rays)) / per_take, 1u), cap);
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&p.ctr->next, 32u * grab);
        first = __shfl_sync(full, first, 0);
        if (first >= n_rays) break;
        last = first;
        for (unsigned c = 0; c < grab; ++c) {
            if (first + c * 32u >= n_rays) break;
            const unsigned idx = first + c * 32u + (unsigned)lane;
            RayRec r;
            bool live = idx < n_rays;
            if (live) {
                r = p.rays[idx];
                live = !(p.longs && r.jf == kLongRay);
            } else {
                r.nsteps = 0;
                r.kbeg = 0;
                r.ex = r.ey = r.ez = r.dx = r.dy = r.dz = 0.0f;
                r.pix = 0;
            }
            const bool owner = live;
            float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f;
            int ns = 0, k = r.kbeg;
            bool done = !live || k >= r.nsteps;
            while (__any_sync(full, !done)) {
                // the longest slab (16, 8, 4 or 2 samples) whose box fits the buffer
                StageBox b;
                long long cells = 0;
                int kend = k;
                bool staged = false;
                for (int slab = kStageSlab;; slab >>= 1) {
                    kend = min(k + slab, r.nsteps);
                    int lx = 0x7fffffff, ly = 0x7fffffff, lz = 0x7fffffff, ux = -0x7fffffff,
                        uy = -0x7fffffff, uz = -0x7fffffff;
                    if (!done) {
                        const float sa = (float)k * p.step, sb = (float)(kend - 1) * p.step;
                        const int ax = corner_lo(sa, r.dx, r.ex), bx = corner_lo(sb, r.dx, r.ex);
                        const int ay = corner_lo(sa, r.dy, r.ey), by = corner_lo(sb, r.dy, r.ey);
                        const int az = corner_lo(sa, r.dz, r.ez), bz = corner_lo(sb, r.dz, r.ez);
                        lx = min(ax, bx);
                        ux = max(ax, bx) + 1;
                        ly = min(ay, by);
                        uy = max(ay, by) + 1;
                        lz = min(az, bz);
                        uz = max(az, bz) + 1;
                    }
                    lx = min(max(__reduce_min_sync(full, lx), lo), hx);
                    ly = min(max(__reduce_min_sync(full, ly), lo), hy);
                    lz = min(max(__reduce_min_sync(full, lz), lo), hz);
                    ux = min(max(__reduce_max_sync(full, ux), lo), hx);
                    uy = min(max(__reduce_max_sync(full, uy), lo), hy);
                    uz = min(max(__reduce_max_sync(full, uz), lo), hz);
                    b.bx = lx;
                    b.by = ly;
                    b.bz = lz;
                    b.ex = ux - lx + 1;
                    b.exy = b.ex * (uy - ly + 1);
                    cells = (long long)b.exy * (uz - lz + 1);
                    b.quads = (int)((cells + 3) >> 2);
                    staged = (long long)b.quads * 4 * kCellBytes <= kStageBytes;
                    if (staged) break;
                    if (slab <= 2) {   // no box fits: gather a whole slab from global memory
                        kend = min(k + kStageSlab, r.nsteps);
                        break;
                    }
                }
                if (staged) {
                    __syncwarp();   // the previous slab's reads of the buffer are done
                    stage_box<SIG, Idx>(p, buf, b, (int)cells, lane, Seq{});
                    __syncwarp();
                }
                for (int kk = k; kk < kend && !done; ++kk) {
                    const float s = (float)kk * p.step;
                    const float x = fmaf(s, r.dx, r.ex), y = fmaf(s, r.dy, r.ey), z = fmaf(s, r.dz, r.ez);
                    const float4 cs = staged ? shade_staged<SIG>(p, s_lut, buf, b, x, y, z, Seq{})
                                             : Shader::shade(p, s_lut, x, y, z);
                    const float a = clamp01(cs.w);
                    const float t = (1.0f - A) * a;
                    C0 = fmaf(t, cs.x, C0);
                    C1 = fmaf(t, cs.y, C1);
                    C2 = fmaf(t, cs.z, C2);
                    A += t;
                    ++ns;
                    done = A >= p.term;
                }
                k = kend;
                if (k >= r.nsteps) done = true;
            }
            if (owner) write_pixel(p, r.pix, C0, C1, C2, A, ns);
        }
    }
}

// The staged zero-copy frame kernel (trilinear, precompiled signatures): the
// LUTs, then one staging buffer per warp, in dynamic shared memory.
template <int NACT, unsigned SIG, typename Idx>
__global__ void __launch_bounds__(kStageWarps * 32, kStageBlocksPerSM) k_raycast_staged(const __grid_constant__ KParams p)
{
    extern __shared__ __align__(16) unsigned char s_stage[];
    float4 *s_lut = reinterpret_cast<float4 *>(s_stage);
    load_luts<NACT>(p, s_lut);
    march_staged<NACT, SIG, Idx>(p, s_lut, s_stage + NACT * 256 * sizeof(float4) + (threadIdx.x >> 5) * kStageBytes);
}

}  // namespace isaac
