// raycast.cuh -- device code of the FP32 volume ray caster (sm_103a).
//
// A frame runs in three kernels on the caller's stream:
//   k_fill_background  background for every pixel outside the screen
//                      rectangle the box can cover; resets the workspace
//                      counters;
//   k_setup_rays       one thread per rectangle pixel: the ray in float-float (camera
//                      unprojection, global/local box and clip-plane interval,
//                      first and last sample on the global grid); misses write
//                      the background, hits are appended to a compact ray list
//                      in the workspace (warp-aggregated, so a chunk of the list
//                      is one 8x4 pixel patch);
//   k_raycast          persistent warps pull chunks of the ray list (dynamic
//                      load balance); RL lanes share one ray and evaluate RL
//                      consecutive samples at once, which are then composited
//                      in order (Sec. 3.2: read -> functor chain -> classify ->
//                      blend -> classical front to back), so the image does not
//                      depend on RL.
// LUTs of the active sources sit in shared memory; chains and source
// descriptors are read from the kernel's constant parameter block (Sec. 3.3
// keeps chains and their parameters in constant memory).  The per-source loop
// is unrolled at compile time over the compacted active sources (Sec. 3.2), so
// inactive sources are never touched.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "isaac_b300.h"
#include "ff.cuh"

namespace isaac {

// Internal functor codes: the public ones, SQRT (POW with every exponent 1/2)
// and AFFINE (a run of ADD/MUL folded into one a*x+b per component).
enum : int {
    K_ADD = 1, K_MUL = 2, K_LENGTH = 3, K_SUM = 4, K_POW = 5, K_LOG = 6, K_SQRT = 7, K_AFFINE = 8
};

struct KOp {
    int code;
    int dim;          // dimension of the value the op consumes
    float a[4];       // arguments (scalar already broadcast); AFFINE: scale
    float b[4];       // AFFINE: offset
};

// Folded chain shapes the kernels run as straight-line code on the first
// component (the only one a chain's result depends on); others are interpreted.
enum : int {
    CH_GENERIC = 0, CH_IDENTITY = 1, CH_AFFINE = 2, CH_LENGTH = 3, CH_LENGTH_AFFINE = 4,
    CH_LENGTH_AFFINE_SQRT = 5, CH_LOG = 6, CH_LOG_AFFINE = 7
};

struct KChain {
    int n;
    int shape;        // CH_*: set by compile_chain from the folded op list
    KOp op[ISAAC_MAX_FUNCTORS];
};

struct KSource {
    const float *base;   // element of interior cell (0,0,0), component 0
    long long sx, sy, sz, sc;
    int fdim;
    int lo;              // lowest readable cell index per axis (-1 with guards, else 0)
    int hi_pad;          // highest readable cell index = n - 1 + hi_pad
    float w;             // blend weight
};

// One entry of the compact ray list (same layout as the public isaac_ray).
struct RayRec {
    float ex, ey, ez;    // local voxel position of the first sample
    int nsteps;          // samples on the global grid inside [t_in, t_out); march stops here
    float dx, dy, dz;    // unit direction
    int pix;             // y * W + x
    int kbeg;            // first sample index to march (0, or a proposal's start)
    int jf, jl;          // label mode: first / last composited sample with opacity > 0 (-1: none)
    int reserved;
};
static_assert(sizeof(RayRec) == 48, "RayRec layout");

// Workspace: counters, then the ray list (one record per rectangle pixel at
// most), then (render workspaces only) the long-ray list: indices of the rays
// an interval proposal left long, which the march takes first with a whole
// warp per ray.
constexpr int kWsHeader = 256;
struct WsCounters {
    unsigned n_rays;     // appended by k_setup_rays
    unsigned next;       // next list entry to march (k_raycast)
    unsigned n_long;     // entries of the long-ray list (appended by the proposal)
    unsigned next_long;  // next long-ray list entry to march
};
// RayRec::jf of a ray that is in the long-ray list (the short-ray pass skips it).
constexpr int kLongRay = -2;
// A proposal puts a ray in the long-ray list when it keeps more samples than this.
constexpr int kLongRaySamples = 96;
// Threads per block and blocks per SM of the frame kernels (k_raycast,
// k_raycast_packed): 32 warps per SM, at most 64 registers per thread.  Each
// block holds its own shared copy of the LUTs (4 KB per source), and shared
// memory comes out of the SRAM that also serves the gathers as L1.  Measured
// at pic512: 256-thread blocks (half the LUT copies) ran at the same speed;
// LUT copies twice as large (a table of entry differences) halved the frame
// rate, the L1 being too small for the gathers' working set.
constexpr int kMarchThreads = 128, kMarchBlocksPerSM = 8;
// Words of empty bits a skipping block stages in shared memory (32768 macro cells).
constexpr int kSkipSharedWords = 1024;

// Key under which the long-ray kernels are registered (the lanes that shade
// one ray's samples per instruction); march_long holds kStreamRays rays per warp.
constexpr int kLongRayLanes = 32;

// March modes: plain (skipping rays on the long-ray list), footprint bitmap,
// visible-span labels, the long-ray list alone, plain with empty-space
// skipping over the macro cells that KParams::empty marks, iso surfaces.
enum : int { MODE_PLAIN = 0, MODE_TOUCH = 1, MODE_LABEL = 2, MODE_LONG = 3, MODE_SKIP = 4, MODE_ISO = 5 };

struct KParams {
    // Host-side geometry in double (the screen rectangle is cut from it).
    double minv[16];                 // inverse of projection * modelview, column-major
    double half_g[3];                // global_n / 2 (world -> global voxel)
    double gn[3];                    // global box [0, gn)
    double llo[3], lhi[3];           // local box in global voxel coordinates
    double clip[ISAAC_MAX_CLIP][4];
    double ndc_sx, ndc_sy;           // 2 / W, 2 / H
    double step_d, inv_step_d;
    // The same geometry as float-float pairs for the device ray setup.  The
    // homogeneous point of pixel (px, py) at NDC depth -1 (ray[0]) and +1
    // (ray[1]), in global voxel coordinates, is c[0] + X c[1] + Y c[2] with
    // X = px - pix_cx, Y = py - pix_cy (both exact in FP32).
    ff ray[2][3][4];
    float pix_cx, pix_cy;            // (W - 1) / 2, (H - 1) / 2
    ff gn_f[3], llo_f[3], lhi_f[3];
    ff clip_f[ISAAC_MAX_CLIP][4];
    ff inv_step_f;
    float step;
    float term;
    float bg[4];
    int n_clip;
    int local_is_global;             // the local box is the global box (no domain split)
    int nx, ny, nz;
    int W, H;
    int rx0, ry0, rx1, ry1;          // rectangle of pixels that can hit the box
    int max_steps;                   // samples on the longest chord of the local box
    int grab;                        // march: most chunks of 32/RL rays a warp takes per atomic
    int luts_host;                   // host only: 1 = lut[] are host addresses still to be
                                     // staged into the workspace, 2 = staged
    // empty-space skipping: one bit per macro cell of skip_cell^3 cells, 32
    // per word (1 = every sample whose position lies in it has opacity 0)
    const unsigned *empty;
    int skip_cell, sgx, sgy, sgz;
    float iso[ISAAC_MAX_ACTIVE];     // iso-surface mode: threshold of each active source
    KSource src[ISAAC_MAX_ACTIVE];
    KChain ch[ISAAC_MAX_ACTIVE];
    const float4 *lut[ISAAC_MAX_ACTIVE];
    uchar4 *fb8;
    float4 *fb32;
    int *nsamp;
    float *depth;                    // optional: distance to the ray's first sample (+inf: none)
    unsigned *touched;               // optional footprint bitmap over [-1, n]^3
    WsCounters *ctr;                 // workspace counters
    RayRec *rays;                    // workspace ray list
    unsigned *longs;                 // workspace long-ray list (nullptr: none)
    // packed (reduced-precision) volume: records over cells [-1, n]^3
    const unsigned char *rec;        // record of cell (x,y,z) at ((z+1)*PY + y+1)*PX + x+1
    const float *scales;             // E4M3: per 8^3 brick (from cell -1), `pad` floats
    int pad;                         // components per record (1, 2, 4 or 8)
    int bx, by;                      // bricks per axis x, y
    int comp_off[ISAAC_MAX_ACTIVE];  // first record component of each active source
};

// Source signature: 4 bits per active source, bits 0-2 = f_dim (0 = read at
// run time), bit 3 = components adjacent in memory (comp_stride == 1).
__host__ __device__ constexpr int sig_fdim(unsigned sig, int i) { return int((sig >> (4 * i)) & 7u); }
__host__ __device__ constexpr bool sig_aos(unsigned sig, int i) { return ((sig >> (4 * i + 3)) & 1u) != 0; }

__device__ __forceinline__ float lerp1(float a, float b, float t) { return fmaf(t, b - a, a); }

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }  // NaN -> 0

__device__ __forceinline__ unsigned char quant8(float x)
{
    float q = floorf(fmaf(255.0f, clamp01(x), 0.5f));
    return (unsigned char)fminf(q, 255.0f);
}

__device__ __forceinline__ float chain_length(int d, const float v[4])
{
    float s = v[0] * v[0];
    if (d > 1) s = fmaf(v[1], v[1], s);
    if (d > 2) s = fmaf(v[2], v[2], s);
    if (d > 3) s = fmaf(v[3], v[3], s);
    return sqrtf(s);
}

// Functor chain of one source (Sec. 3.3, Table 1).  The op list is uniform
// across the launch, so every branch below is uniform across the warp.  The
// common folded shapes run as straight-line code on component 0 with the
// same operations, in the same order, as the op-by-op loop.
__device__ __forceinline__ float run_chain(const KChain &ch, float v[4])
{
    switch (ch.shape) {
    case CH_IDENTITY:
        return v[0];
    case CH_AFFINE:
        return fmaf(ch.op[0].a[0], v[0], ch.op[0].b[0]);
    case CH_LENGTH:
        return chain_length(ch.op[0].dim, v);
    case CH_LENGTH_AFFINE:
        return fmaf(ch.op[1].a[0], chain_length(ch.op[0].dim, v), ch.op[1].b[0]);
    case CH_LENGTH_AFFINE_SQRT: {
        const float x = fmaf(ch.op[1].a[0], chain_length(ch.op[0].dim, v), ch.op[1].b[0]);
        return x > 0.0f ? sqrtf(x) : 0.0f;
    }
    case CH_LOG:
        return logf(fmaxf(v[0], 1e-30f));
    case CH_LOG_AFFINE:
        return fmaf(ch.op[1].a[0], logf(fmaxf(v[0], 1e-30f)), ch.op[1].b[0]);
    default:
        break;
    }
#pragma unroll 1
    for (int i = 0; i < ch.n; ++i) {
        const KOp &o = ch.op[i];
        const int d = o.dim;
        switch (o.code) {
        case K_AFFINE:
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = fmaf(o.a[c], v[c], o.b[c]);
            break;
        case K_ADD:
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] += o.a[c];
            break;
        case K_MUL:
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] *= o.a[c];
            break;
        case K_LENGTH:
            v[0] = chain_length(d, v);
            break;
        case K_SUM: {
            float s = v[0];
            if (d > 1) s += v[1];
            if (d > 2) s += v[2];
            if (d > 3) s += v[3];
            v[0] = s;
        } break;
        case K_SQRT:
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < d) v[c] = v[c] > 0.0f ? sqrtf(v[c]) : 0.0f;
            break;
        case K_POW:
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < d) v[c] = v[c] > 0.0f ? powf(v[c], o.a[c]) : 0.0f;
            break;
        case K_LOG:
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < d) v[c] = logf(fmaxf(v[c], 1e-30f));
            break;
        default:
            break;
        }
    }
    return v[0];
}

// Interval form of run_chain: given, per component, an interval [lo, hi]
// that holds the value, an interval that holds the chain's result as run_chain
// computes it in FP32.  Sums, products, FMAs and square roots round outward
// (directed rounding); pow and log, which have no directed forms, are widened
// by 10^-6 relative (many ulps of their error).  A NaN anywhere widens the
// result to everything.
__device__ __forceinline__ void chain_interval(const KChain &ch, float lo[4], float hi[4])
{
    const float inf = __int_as_float(0x7f800000);
    for (int i = 0; i < ch.n; ++i) {
        const KOp &o = ch.op[i];
        const int d = o.dim;
        switch (o.code) {
        case K_AFFINE:
            for (int c = 0; c < 4; ++c) {
                const float a = o.a[c], b = o.b[c];
                const float l = a >= 0.0f ? __fmaf_rd(a, lo[c], b) : __fmaf_rd(a, hi[c], b);
                const float h = a >= 0.0f ? __fmaf_ru(a, hi[c], b) : __fmaf_ru(a, lo[c], b);
                lo[c] = l;
                hi[c] = h;
            }
            break;
        case K_ADD:
            for (int c = 0; c < 4; ++c) {
                lo[c] = __fadd_rd(lo[c], o.a[c]);
                hi[c] = __fadd_ru(hi[c], o.a[c]);
            }
            break;
        case K_MUL:
            for (int c = 0; c < 4; ++c) {
                const float a = o.a[c];
                const float l = a >= 0.0f ? __fmul_rd(lo[c], a) : __fmul_rd(hi[c], a);
                const float h = a >= 0.0f ? __fmul_ru(hi[c], a) : __fmul_ru(lo[c], a);
                lo[c] = l;
                hi[c] = h;
            }
            break;
        case K_LENGTH:
        case K_SUM: {
            float sl = 0.0f, sh = 0.0f;
            for (int c = 0; c < 4; ++c) {
                if (c >= d) break;
                float ql = lo[c], qh = hi[c];
                if (o.code == K_LENGTH) {   // the square's interval
                    const float m = fmaxf(fabsf(lo[c]), fabsf(hi[c]));
                    const float n = (lo[c] > 0.0f) ? lo[c] : (hi[c] < 0.0f ? -hi[c] : 0.0f);
                    ql = __fmul_rd(n, n);
                    qh = __fmul_ru(m, m);
                }
                sl = __fadd_rd(sl, ql);
                sh = __fadd_ru(sh, qh);
            }
            if (o.code == K_LENGTH) {
                sl = __fsqrt_rd(fmaxf(sl, 0.0f));
                sh = __fsqrt_ru(sh);
            }
            lo[0] = sl;
            hi[0] = sh;
        } break;
        case K_SQRT:
            for (int c = 0; c < 4; ++c)
                if (c < d) {
                    lo[c] = lo[c] > 0.0f ? __fsqrt_rd(lo[c]) : 0.0f;
                    hi[c] = hi[c] > 0.0f ? __fsqrt_ru(hi[c]) : 0.0f;
                }
            break;
        case K_POW:
            for (int c = 0; c < 4; ++c)
                if (c < d) {
                    const float a = o.a[c];
                    float l, h;
                    if (hi[c] <= 0.0f) {
                        l = h = 0.0f;
                    } else {
                        const float pl = lo[c] > 0.0f ? powf(lo[c], a) : (a > 0.0f ? 0.0f : (a < 0.0f ? inf : 1.0f));
                        const float ph = powf(hi[c], a);
                        l = fminf(pl, ph);
                        h = fmaxf(pl, ph);
                        if (lo[c] <= 0.0f) l = 0.0f;            // v <= 0 gives 0
                        l = l - fabsf(l) * 1e-6f;
                        h = h + fabsf(h) * 1e-6f;
                    }
                    lo[c] = l;
                    hi[c] = h;
                }
            break;
        case K_LOG:
            for (int c = 0; c < 4; ++c)
                if (c < d) {
                    const float l = logf(fmaxf(lo[c], 1e-30f)), h = logf(fmaxf(hi[c], 1e-30f));
                    lo[c] = l - (fabsf(l) + 1.0f) * 1e-6f;
                    hi[c] = h + (fabsf(h) + 1.0f) * 1e-6f;
                }
            break;
        default:
            break;
        }
    }
    if (!(lo[0] == lo[0]) || !(hi[0] == hi[0])) {
        lo[0] = -inf;
        hi[0] = inf;
    }
}

// Transfer function: clamp to [0,1], entries at j/255, linear in between.
__device__ __forceinline__ float4 classify(const float4 *lut, float x)
{
    const float pos = clamp01(x) * 255.0f;
    const int j = min((int)pos, 254);
    const float f = pos - (float)j;
    const float4 a = lut[j], b = lut[j + 1];
    return make_float4(lerp1(a.x, b.x, f), lerp1(a.y, b.y, f), lerp1(a.z, b.z, f),
                       lerp1(a.w, b.w, f));
}

__device__ __forceinline__ void blend(float4 &acc, float w, float4 c)
{
    acc.x = fmaf(w, c.x, acc.x);
    acc.y = fmaf(w, c.y, acc.y);
    acc.z = fmaf(w, c.z, acc.z);
    acc.w = fmaf(w, c.w, acc.w);
}

// Geometry of one sample shared by all sources.
struct Geo {
    int ix, iy, iz;      // lower corner (trilinear) or the cell (nearest), unclamped
    float fx, fy, fz;    // fractional position in the corner cell
    float w[8];          // trilinear weight of corner k (bit 0: x+1, bit 1: y+1, bit 2: z+1)
};

template <int INTERP>
__device__ __forceinline__ Geo sample_geo(float x, float y, float z)
{
    Geo g;
    if (INTERP) {
        const float qx = x - 0.5f, qy = y - 0.5f, qz = z - 0.5f;
        const float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
        g.ix = (int)flx;
        g.iy = (int)fly;
        g.iz = (int)flz;
        g.fx = qx - flx;
        g.fy = qy - fly;
        g.fz = qz - flz;
        // the 8 corner weights, once per sample for every source and component
        const float gx = 1.0f - g.fx, gy = 1.0f - g.fy, gz = 1.0f - g.fz;
        const float a00 = gy * gz, a10 = g.fy * gz, a01 = gy * g.fz, a11 = g.fy * g.fz;
        g.w[0] = gx * a00;
        g.w[1] = g.fx * a00;
        g.w[2] = gx * a10;
        g.w[3] = g.fx * a10;
        g.w[4] = gx * a01;
        g.w[5] = g.fx * a01;
        g.w[6] = gx * a11;
        g.w[7] = g.fx * a11;
    } else {
        g.ix = (int)floorf(x);
        g.iy = (int)floorf(y);
        g.iz = (int)floorf(z);
        g.fx = g.fy = g.fz = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) g.w[k] = 0.0f;
    }
    return g;
}

// Trilinear value from the 8 corner values (corner k as in Geo::w): the
// weighted sum, one multiply and seven fused multiply-adds per component.
__device__ __forceinline__ float tri(const Geo &g, float c0, float c1, float c2, float c3, float c4,
                                     float c5, float c6, float c7)
{
    float v = c0 * g.w[0];
    v = fmaf(g.w[1], c1, v);
    v = fmaf(g.w[2], c2, v);
    v = fmaf(g.w[3], c3, v);
    v = fmaf(g.w[4], c4, v);
    v = fmaf(g.w[5], c5, v);
    v = fmaf(g.w[6], c6, v);
    return fmaf(g.w[7], c7, v);
}

template <typename Idx>
__device__ __forceinline__ float ld(const float *b, Idx o) { return __ldg(b + o); }

// The 6 floats e[0..5] (two x-adjacent cells of a 3-component AoS source) in
// four loads: two 8-byte loads at the even-aligned address and two scalars,
// all inside e[0..5].  q = 1 when e is not 8-byte aligned.
__device__ __forceinline__ void ld_pair3(const float *e, float (&v)[6])
{
    const bool q = ((uintptr_t)e & 4u) != 0;
    const float2 a = __ldg(reinterpret_cast<const float2 *>(e + (q ? 1 : 0)));
    const float2 b = __ldg(reinterpret_cast<const float2 *>(e + (q ? 3 : 2)));
    const float c = __ldg(e + (q ? 0 : 4));
    v[0] = q ? c : a.x;
    v[1] = q ? a.x : a.y;
    v[2] = q ? a.y : b.x;
    v[3] = q ? b.x : b.y;
    v[4] = q ? b.y : c;
    v[5] = __ldg(e + 5);
}

// Value of source I at the sample: 8-corner gather + trilinear blend per
// component, or the nearest cell.  Indices are clamped to the readable range
// the host validated against the source's extent, so no access can leave it.
template <int I, unsigned SIG, int INTERP, typename Idx>
__device__ __forceinline__ void fetch_source(const KParams &p, const Geo &g, float v[4])
{
    constexpr int FD = sig_fdim(SIG, I);
    constexpr bool AOS = sig_aos(SIG, I);
    const KSource &s = p.src[I];
    const int fd = FD ? FD : s.fdim;
    const Idx cs = AOS ? Idx(1) : Idx(s.sc);
    const float *base = s.base;
    if (INTERP) {
        const int x0 = min(max(g.ix, s.lo), p.nx - 1 + s.hi_pad);
        const int x1 = min(max(g.ix + 1, s.lo), p.nx - 1 + s.hi_pad);
        const int y0 = min(max(g.iy, s.lo), p.ny - 1 + s.hi_pad);
        const int y1 = min(max(g.iy + 1, s.lo), p.ny - 1 + s.hi_pad);
        const int z0 = min(max(g.iz, s.lo), p.nz - 1 + s.hi_pad);
        const int z1 = min(max(g.iz + 1, s.lo), p.nz - 1 + s.hi_pad);
        const Idx sx = Idx(s.sx), sy = Idx(s.sy), sz = Idx(s.sz);
        const Idx ox0 = Idx(x0) * sx, ox1 = Idx(x1) * sx;
        const Idx o00 = Idx(y0) * sy + Idx(z0) * sz, o10 = Idx(y1) * sy + Idx(z0) * sz;
        const Idx o01 = Idx(y0) * sy + Idx(z1) * sz, o11 = Idx(y1) * sy + Idx(z1) * sz;
        if constexpr (FD == 3 && AOS) {
            // cells contiguous in x and both x-corners distinct: each (y, z) row
            // of the gather is 6 adjacent floats (fewer L1 requests per sample)
            if (s.sx == 3 && x1 == x0 + 1) {
                float r00[6], r10[6], r01[6], r11[6];
                ld_pair3(base + (ox0 + o00), r00);
                ld_pair3(base + (ox0 + o10), r10);
                ld_pair3(base + (ox0 + o01), r01);
                ld_pair3(base + (ox0 + o11), r11);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    v[c] = tri(g, r00[c], r00[3 + c], r10[c], r10[3 + c], r01[c], r01[3 + c], r11[c],
                               r11[3 + c]);
                v[3] = 0.0f;
                return;
            }
        }
        const float *p000 = base + (ox0 + o00), *p100 = base + (ox1 + o00);
        const float *p010 = base + (ox0 + o10), *p110 = base + (ox1 + o10);
        const float *p001 = base + (ox0 + o01), *p101 = base + (ox1 + o01);
        const float *p011 = base + (ox0 + o11), *p111 = base + (ox1 + o11);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c < fd) {
                const Idx co = Idx(c) * cs;
                v[c] = tri(g, ld(p000, co), ld(p100, co), ld(p010, co), ld(p110, co), ld(p001, co),
                           ld(p101, co), ld(p011, co), ld(p111, co));
            } else {
                v[c] = 0.0f;
            }
        }
    } else {
        const int x = min(max(g.ix, 0), p.nx - 1);
        const int y = min(max(g.iy, 0), p.ny - 1);
        const int z = min(max(g.iz, 0), p.nz - 1);
        const float *pc = base + (Idx(x) * Idx(s.sx) + Idx(y) * Idx(s.sy) + Idx(z) * Idx(s.sz));
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (c < fd) ? ld(pc, Idx(c) * cs) : 0.0f;
    }
}

// LUT of active source I: the block's shared copy, or (s_lut == nullptr, the
// batched kernels whose blocks mix requests) the request's global array.
template <int I>
__device__ __forceinline__ const float4 *lut_of(const KParams &p, const float4 *s_lut)
{
    return s_lut ? s_lut + I * 256 : p.lut[I];
}

template <int I, unsigned SIG, int INTERP, typename Idx>
__device__ __forceinline__ void shade_source(const KParams &p, const Geo &g, const float4 *s_lut,
                                             float4 &acc)
{
    float v[4];
    fetch_source<I, SIG, INTERP, Idx>(p, g, v);
    const float x = run_chain(p.ch[I], v);
    blend(acc, p.src[I].w, classify(lut_of<I>(p, s_lut), x));
}

template <unsigned SIG, int INTERP, typename Idx, int... Is>
__device__ __forceinline__ void shade_all(const KParams &p, const Geo &g, const float4 *s_lut,
                                          float4 &acc, std::integer_sequence<int, Is...>)
{
    (shade_source<Is, SIG, INTERP, Idx>(p, g, s_lut, acc), ...);
}

// Footprint: mark the cells a sample reads in the [-1, n]^3 bitmap.
template <int INTERP>
__device__ __forceinline__ void mark_footprint(const KParams &p, const Geo &g)
{
    const int W = p.nx + 2, H = p.ny + 2;
#pragma unroll
    for (int c = 0; c < (INTERP ? 8 : 1); ++c) {
        const int x = min(max(g.ix + (c & 1), -1), p.nx) + 1;
        const int y = min(max(g.iy + ((c >> 1) & 1), -1), p.ny) + 1;
        const int z = min(max(g.iz + ((c >> 2) & 1), -1), p.nz) + 1;
        const long long bit = ((long long)z * H + y) * W + x;
        atomicOr(p.touched + (bit >> 5), 1u << (bit & 31));
    }
}

// Blended RGBA of one sample of the zero-copy sources.
template <int NACT, unsigned SIG, int INTERP, typename Idx, bool TOUCH>
struct ZeroCopyShader {
    __device__ __forceinline__ static float4 shade(const KParams &p, const float4 *s_lut, float x,
                                                   float y, float z)
    {
        const Geo g = sample_geo<INTERP>(x, y, z);
        if (TOUCH) mark_footprint<INTERP>(p, g);
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        shade_all<SIG, INTERP, Idx>(p, g, s_lut, acc, std::make_integer_sequence<int, NACT>{});
        return acc;
    }
};

// ------------------------------------------------------------- ray setup

// Ray setup (camera unprojection, box and clip-plane intervals, the sample
// index range) in float-float arithmetic, ~48 significant bits: the discrete
// decisions (first and last sample) agree with a double-precision computation
// except within ~1e-12 of a tie, at a fraction of the cost of FP64 on B300.
// The first sample's position and the direction are rounded to FP32 for the
// march.
__device__ __forceinline__ RayRec setup_ray(const KParams &p, int px, int py, float *t_first = nullptr)
{
    RayRec r;
    r.nsteps = 0;
    r.ex = r.ey = r.ez = 0.0f;
    r.dx = r.dy = r.dz = 0.0f;
    r.pix = py * p.W + px;
    r.kbeg = 0;
    r.jf = r.jl = -1;
    r.reserved = 0;
    const float X = (float)px - p.pix_cx, Y = (float)py - p.pix_cy;
    ff h[2][4];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            h[e][i] = ff_add(ff_add(p.ray[e][0][i], ff_mulf(p.ray[e][1][i], X)), ff_mulf(p.ray[e][2][i], Y));
    // near point o and unit direction d towards the far point
    const ff inw = ff_rcp(h[0][3]), ifw = ff_rcp(h[1][3]);
    ff o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = ff_mul(h[0][a], inw);
        d[a] = ff_sub(ff_mul(h[1][a], ifw), o[a]);
    }
    const ff il = ff_rsqrt(ff_add(ff_add(ff_mul(d[0], d[0]), ff_mul(d[1], d[1])), ff_mul(d[2], d[2])));
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = ff_mul(d[a], il);
    // a degenerate pixel (point at infinity, zero direction) cannot be cast
    if (!(isfinite(o[0].hi) && isfinite(o[1].hi) && isfinite(o[2].hi) && isfinite(d[0].hi) &&
          isfinite(d[1].hi) && isfinite(d[2].hi)))
        return r;

    // Slab intervals of the global box (t0 = its entry: the origin of the
    // sample grid) and of the local box.  A direction component below 1e-30
    // counts as zero (its slab crossings lie beyond any reachable t).  Without
    // a domain split the two boxes coincide and one pass serves both.
    const float inf = __int_as_float(0x7f800000);
    ff t0 = ff_from(0.0f), tg1 = ff_from(inf), tl0 = ff_from(0.0f), tout = ff_from(inf);
    bool miss = false;
    const bool one_box = p.local_is_global != 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (fabsf(d[a].hi) > 1e-30f) {
            const ff inv = ff_rcp(d[a]);
            ff ta = ff_mul(ff_neg(o[a]), inv), tb = ff_mul(ff_sub(p.gn_f[a], o[a]), inv);
            t0 = ff_max(t0, ff_min(ta, tb));
            tg1 = ff_min(tg1, ff_max(ta, tb));
            if (!one_box) {
                ta = ff_mul(ff_sub(p.llo_f[a], o[a]), inv);
                tb = ff_mul(ff_sub(p.lhi_f[a], o[a]), inv);
                tl0 = ff_max(tl0, ff_min(ta, tb));
                tout = ff_min(tout, ff_max(ta, tb));
            }
        } else if (ff_lt(o[a], p.llo_f[a]) || !ff_lt(o[a], p.lhi_f[a])) {
            miss = true;
        }
    }
    if (one_box) {
        tl0 = t0;
        tout = tg1;
    }
    if (!ff_lt(t0, tg1)) miss = true;
    ff tin = ff_max(t0, tl0);
    for (int i = 0; i < p.n_clip; ++i) {
        const ff *pl = p.clip_f[i];
        const ff s = ff_add(ff_add(ff_add(ff_mul(pl[0], o[0]), ff_mul(pl[1], o[1])), ff_mul(pl[2], o[2])), pl[3]);
        const ff rr = ff_add(ff_add(ff_mul(pl[0], d[0]), ff_mul(pl[1], d[1])), ff_mul(pl[2], d[2]));
        if (rr.hi > 0.0f) {
            tin = ff_max(tin, ff_neg(ff_div(s, rr)));
        } else if (rr.hi < 0.0f) {
            tout = ff_min(tout, ff_neg(ff_div(s, rr)));
        } else if (s.hi < 0.0f) {
            miss = true;
        }
    }
    // the local box is bounded, so a ray inside it has a finite exit
    if (miss || !ff_lt(tin, tout) || !(tout.hi < 1e30f)) return r;
    const long long kf = ff_lt(t0, tin) ? ff_ceil(ff_mul(ff_sub(tin, t0), p.inv_step_f)) : 0LL;
    const long long ke = ff_ceil(ff_mul(ff_sub(tout, t0), p.inv_step_f));
    if (ke <= kf) return r;
    const float kf_hi = (float)kf;
    const ff kff = {kf_hi, (float)(kf - (long long)kf_hi)};
    const ff tf = ff_add(t0, ff_mulf(kff, p.step));
    if (t_first) *t_first = tf.hi;
    r.ex = ff_sub(ff_add(o[0], ff_mul(tf, d[0])), p.llo_f[0]).hi;
    r.ey = ff_sub(ff_add(o[1], ff_mul(tf, d[1])), p.llo_f[1]).hi;
    r.ez = ff_sub(ff_add(o[2], ff_mul(tf, d[2])), p.llo_f[2]).hi;
    r.dx = d[0].hi;
    r.dy = d[1].hi;
    r.dz = d[2].hi;
    r.nsteps = (int)min(ke - kf, (long long)p.max_steps);
    return r;
}

__device__ __forceinline__ void write_pixel(const KParams &p, int pix, float C0, float C1, float C2,
                                            float A, int ns)
{
    const float T = 1.0f - A;
    const float o0 = fmaf(T, p.bg[0], C0), o1 = fmaf(T, p.bg[1], C1);
    const float o2 = fmaf(T, p.bg[2], C2), o3 = fmaf(T, p.bg[3], A);
    p.fb8[pix] = make_uchar4(quant8(o0), quant8(o1), quant8(o2), quant8(o3));
    if (p.fb32) p.fb32[pix] = make_float4(o0, o1, o2, o3);
    if (p.nsamp) p.nsamp[pix] = ns;
}

// Background for every pixel outside the rectangle; resets the counters.
// Rows are spread over the blocks and a row's pixels over the threads (W*H is
// at most 2^30, so pixel indices fit an int).
static __global__ void k_fill_background(const __grid_constant__ KParams p)
{
    // the ray setup that follows may start now: it computes its rays while
    // this fill runs and waits for the fill's writes before its own
    asm volatile("griddepcontrol.launch_dependents;");
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.ctr) {
        p.ctr->n_rays = 0u;
        p.ctr->next = 0u;
        p.ctr->n_long = 0u;
        p.ctr->next_long = 0u;
    }
    for (int y = blockIdx.x; y < p.H; y += gridDim.x) {
        const bool row_in = y >= p.ry0 && y < p.ry1;
        for (int x = threadIdx.x; x < p.W; x += blockDim.x) {
            if (row_in && x >= p.rx0 && x < p.rx1) continue;
            const int i = y * p.W + x;
            write_pixel(p, i, 0.0f, 0.0f, 0.0f, 0.0f, 0);
            if (p.depth) p.depth[i] = __int_as_float(0x7f800000);
        }
    }
}

// One thread per rectangle pixel, 128-thread blocks over 16x8 tiles whose warps
// are 8x4 patches; hits are appended warp by warp.
static __global__ void __launch_bounds__(128) k_setup_rays(const __grid_constant__ KParams p)
{
    const int tiles_x = (p.rx1 - p.rx0 + 15) >> 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int px = p.rx0 + tx * 16 + (warp & 1) * 8 + (lane & 7);
    const int py = p.ry0 + ty * 8 + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = px < p.rx1 && py < p.ry1;
    RayRec r;
    r.nsteps = 0;
    float tf = 0.0f;
    if (inside) r = setup_ray(p, px, py, &tf);
    // launched as a programmatic dependent of the background fill: the ray
    // arithmetic above overlaps the fill; the counters the fill resets and
    // every write below wait for its completion
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const bool hit = inside && r.nsteps > 0;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    unsigned base = 0;
    if (lane == 0 && m) base = atomicAdd(&p.ctr->n_rays, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) {
        p.rays[base + __popc(m & ((1u << lane) - 1u))] = r;
    } else if (inside) {
        write_pixel(p, py * p.W + px, 0.0f, 0.0f, 0.0f, 0.0f, 0);
    }
    if (inside && p.depth) p.depth[py * p.W + px] = hit ? tf : __int_as_float(0x7f800000);
}

// ------------------------------------------------------------------ march

// One ray of the list, marched by the RL lanes of its group.  Lanes of a
// group evaluate samples k+0 .. k+RL-1 together; every lane then composites
// the group's RL samples in order, stopping at the termination sample, so all
// lanes hold the same C and A.
// s_empty: the block's shared copy of the empty bits (SKIP_EMPTY), or null to
// read them from p.empty.
// Whether a shaded sample can change the composite: a positive opacity, or a
// colour that is not finite (0 * inf is NaN, so such a sample is composited
// like any other).
__device__ __forceinline__ bool live_sample(const float4 &c)
{
    return c.w > 0.0f || !(fabsf(c.x) <= 3.402823466e38f && fabsf(c.y) <= 3.402823466e38f &&
                           fabsf(c.z) <= 3.402823466e38f);
}

// ZSKIP: the frame can have samples of opacity 0 (load_luts), so steps whose
// group has nothing to composite are voted on and skipped; the kernels pick
// the instantiation once per block, so dense frames run the loop without it.
template <class Shader, int RL, bool LABEL, bool SKIP_LONG = false, bool SKIP_EMPTY = false,
          bool ZSKIP = false>
__device__ __forceinline__ void march_ray(const KParams &p, const float4 *s_lut, unsigned idx,
                                          int lane, const unsigned *s_empty = nullptr)
{
    const int sub = lane & (RL - 1);
    const RayRec r = p.rays[idx];
    if (SKIP_LONG && p.longs && r.jf == kLongRay) return;   // marched from the long-ray list
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f;
    int ns = 0, jf = -1, jl = -1;
    const unsigned gmask = (RL == 32) ? 0xffffffffu : (((1u << RL) - 1u) << (lane & ~(RL - 1)));
    for (int k = r.kbeg; k < r.nsteps; k += RL) {
        if (SKIP_EMPTY) {
            // The macro cell that owns sample k's position: if it is marked
            // empty, jump to the first sample at or past the ray's exit from its
            // box [m*c, (m+1)*c) per axis.  Every skipped sample lies in that box
            // (up to FP32 rounding, far inside the one-cell apron the marking
            // covers), so it has opacity 0 and compositing it changes nothing.
            const float s0 = (float)k * p.step;
            const float x = fmaf(s0, r.dx, r.ex), y = fmaf(s0, r.dy, r.ey), z = fmaf(s0, r.dz, r.ez);
            const float cz = (float)p.skip_cell;
            const int mx = min(max((int)floorf(x / cz), 0), p.sgx - 1);
            const int my = min(max((int)floorf(y / cz), 0), p.sgy - 1);
            const int mz = min(max((int)floorf(z / cz), 0), p.sgz - 1);
            const long long m = ((long long)mz * p.sgy + my) * p.sgx + mx;
            const unsigned *bits = s_empty ? s_empty : p.empty;
            if ((bits[m >> 5] >> (m & 31)) & 1u) {
                const float inf = __int_as_float(0x7f800000);
                const float ex = r.dx > 0.0f ? ((float)(mx + 1) * cz - x) / r.dx
                               : (r.dx < 0.0f ? ((float)mx * cz - x) / r.dx : inf);
                const float ey = r.dy > 0.0f ? ((float)(my + 1) * cz - y) / r.dy
                               : (r.dy < 0.0f ? ((float)my * cz - y) / r.dy : inf);
                const float ez = r.dz > 0.0f ? ((float)(mz + 1) * cz - z) / r.dz
                               : (r.dz < 0.0f ? ((float)mz * cz - z) / r.dz : inf);
                const float se = fminf(ex, fminf(ey, ez));
                const int jump = se > 0.0f ? (int)fminf(ceilf(se / p.step), 1.0e9f) : 1;
                k += max(jump, 1) - RL;   // the loop adds RL
                continue;
            }
        }
        float4 cs = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (k + sub < r.nsteps) {
            const float s = (float)(k + sub) * p.step;
            cs = Shader::shade(p, s_lut, fmaf(s, r.dx, r.ex), fmaf(s, r.dy, r.ey), fmaf(s, r.dz, r.ez));
        }
        // A group of samples that all have opacity 0 and finite colours
        // composites nothing: t = (1 - A) * 0 = +0 adds +0 to C and A, which
        // leaves them bit for bit as they are, and A stays below the
        // threshold (A < term on entry; with term <= 0 the first sample ends
        // the ray, so that case takes the loop).  Only the sample count moves,
        // so the RL-step in-order loop (RL shuffles of 4 floats) is skipped:
        // empty space of sparse fields is marched at the gather rate.
        if constexpr (ZSKIP) {
            if (A < p.term && !__any_sync(gmask, live_sample(cs))) {
                ns += min(RL, r.nsteps - k);
                continue;
            }
        }
        bool done = false;
        auto composite = [&](const float4 &c, int kq, int j) {
            float4 cj = c;
            if (RL > 1) {
                cj.x = __shfl_sync(gmask, c.x, j, RL);
                cj.y = __shfl_sync(gmask, c.y, j, RL);
                cj.z = __shfl_sync(gmask, c.z, j, RL);
                cj.w = __shfl_sync(gmask, c.w, j, RL);
            }
            if (!done && kq + j < r.nsteps) {
                const float a = clamp01(cj.w);
                if (LABEL && a > 0.0f) {
                    if (jf < 0) jf = kq + j;
                    jl = kq + j;
                }
                const float t = (1.0f - A) * a;
                C0 = fmaf(t, cj.x, C0);
                C1 = fmaf(t, cj.y, C1);
                C2 = fmaf(t, cj.z, C2);
                A += t;
                ++ns;
                done = A >= p.term;
            }
        };
        if constexpr (RL <= 8) {
#pragma unroll
            for (int j = 0; j < RL; ++j) composite(cs, k, j);
        } else {   // wide groups: a partly rolled loop keeps the register count down
#pragma unroll 4
            for (int j = 0; j < RL; ++j) composite(cs, k, j);
        }
        if (done) break;
    }
    if (sub == 0) {
        write_pixel(p, r.pix, C0, C1, C2, A, ns);
        if (LABEL) {
            p.rays[idx].jf = jf;
            p.rays[idx].jl = jl;
        }
    }
}

// Persistent warps with guided self-scheduling: a warp takes chunks of 32/RL
// rays from the list, as many per atomic as 1/(2W) of what was left at its
// previous take (W warps in the grid; at most p.grab, at least one), so that
// long lists need few atomics on the one shared counter while the last
// chunks stay small enough to balance the warps.  Rays on the long-ray list
// are skipped: the long-ray march has taken them.
template <int NACT, class Shader, int RL, bool LABEL = false, bool SKIP_EMPTY = false,
          bool ZSKIP = false>
__device__ __forceinline__ void march(const KParams &p, const float4 *s_lut,
                                      const unsigned *s_empty = nullptr)
{
    constexpr unsigned RAYS = 32 / RL;
    const int lane = threadIdx.x & 31;
    const unsigned n_rays = *(volatile unsigned *)&p.ctr->n_rays;
    const unsigned cap = (unsigned)max(p.grab, 1);
    const unsigned per_take = RAYS * 2u * gridDim.x * (blockDim.x >> 5);
    unsigned last = 0;
    for (;;) {
        const unsigned grab = min(max((n_rays - min(last, n_rays)) / per_take, 1u), cap);
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&p.ctr->next, RAYS * grab);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (first >= n_rays) break;
        last = first;
        for (unsigned c = 0; c < grab; ++c) {
            const unsigned idx = first + c * RAYS + (unsigned)(lane / RL);
            if (first + c * RAYS >= n_rays) break;
            if (idx < n_rays)
                march_ray<Shader, RL, LABEL, !LABEL, SKIP_EMPTY, ZSKIP>(p, s_lut, idx, lane, s_empty);
        }
    }
}

// The long-ray march: the rays an interval proposal left long (a few among
// many short ones), launched before the march of the rest.  A warp holds
// kStreamRays rays (lanes 0 .. kStreamRays-1 own one each).  Per step every
// lane shades kStreamU samples -- sample k + j of a held ray, consecutive j on
// consecutive lanes -- without branches, so the gathers of all of them are in
// flight together (samples of a dead slot or past a window end read clamped
// cells and are dropped), into the warp's shared tile; then each owner lane
// composites its ray's kStreamT samples in order: the same operations in the
// same order as march_ray, so the pixel is bit-identical to the plain march.
// A ray that terminates or ends is written and its slot refilled from the
// list at the next step.  In-order compositing thus costs one lane per ray,
// not every lane of a group, and a window with nothing to composite (ZSKIP)
// costs none.  Since such windows are skipped, one ray per warp with 64-sample
// windows (twice the warps in flight for the few long rays) is the fastest
// shape: 2 rays x 64 samples and 1 ray x 128 samples measured slower.
constexpr int kStreamRays = 1, kStreamU = 2, kStreamT = 32 * kStreamU / kStreamRays;

template <class Shader, bool ZSKIP = false>
__device__ __forceinline__ void march_long(const KParams &p, const float4 *s_lut)
{
    constexpr int kRow = kStreamT + 1;        // padded row: owners' reads hit distinct banks
    __shared__ float4 s_tile[kMarchThreads / 32][kStreamRays * kRow];
    float4 *tile = s_tile[threadIdx.x >> 5];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool owner = lane < kStreamRays;
    const unsigned n_long = *(volatile unsigned *)&p.ctr->n_long;
    RayRec r;
    r.ex = r.ey = r.ez = r.dx = r.dy = r.dz = 0.0f;
    r.nsteps = 0;
    r.pix = 0;
    int k = 0, ns = 0;
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f;
    bool live = false, exhausted = false;
    // every list entry is taken once, so the loop ends after n_long takes
    for (;;) {
        const unsigned need = exhausted ? 0u : __ballot_sync(full, owner && !live);
        if (need) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&p.ctr->next_long, (unsigned)__popc(need));
            base = __shfl_sync(full, base, 0);
            if (base + (unsigned)__popc(need) >= n_long) exhausted = true;
            if (owner && !live) {
                const unsigned i = base + (unsigned)__popc(need & ((1u << lane) - 1u));
                if (i < n_long) {
                    r = p.rays[p.longs[i]];
                    k = r.kbeg;
                    ns = 0;
                    C0 = C1 = C2 = A = 0.0f;
                    live = k < r.nsteps;
                    if (!live) write_pixel(p, r.pix, 0.0f, 0.0f, 0.0f, 0.0f, 0);
                }
            }
        }
        if (!__any_sync(full, live)) {
            if (exhausted) break;
            continue;
        }
        float4 c[kStreamU];
        bool valid[kStreamU];
#pragma unroll
        for (int u = 0; u < kStreamU; ++u) {
            const int slot = u * 32 / kStreamT;            // ray of this sample, uniform per u
            const float ex = __shfl_sync(full, r.ex, slot), ey = __shfl_sync(full, r.ey, slot);
            const float ez = __shfl_sync(full, r.ez, slot), dx = __shfl_sync(full, r.dx, slot);
            const float dy = __shfl_sync(full, r.dy, slot), dz = __shfl_sync(full, r.dz, slot);
            const int ku = __shfl_sync(full, k, slot), nu = __shfl_sync(full, r.nsteps, slot);
            const bool lu = __shfl_sync(full, (int)live, slot) != 0;
            const int kk = ku + (u * 32) % kStreamT + lane;
            valid[u] = lu && kk < nu;
            const float s = (float)kk * p.step;
            c[u] = Shader::shade(p, s_lut, fmaf(s, dx, ex), fmaf(s, dy, ey), fmaf(s, dz, ez));
        }
        // per held ray, whether any of its kStreamT samples can change its
        // composite (live_sample); a ray whose samples cannot only counts them
        unsigned busy = ZSKIP ? 0u : ~0u;
        if constexpr (ZSKIP) {
#pragma unroll
            for (int u = 0; u < kStreamU; ++u)
                if (__any_sync(full, valid[u] && live_sample(c[u]))) busy |= 1u << (u * 32 / kStreamT);
        }
        // alpha is clamped here, on all lanes, rather than in the owner's loop
#pragma unroll
        for (int u = 0; u < kStreamU; ++u) {
            const int slot = u * 32 / kStreamT;
            if ((busy >> slot) & 1u)
                tile[slot * kRow + (u * 32) % kStreamT + lane] =
                    valid[u] ? make_float4(c[u].x, c[u].y, c[u].z, clamp01(c[u].w))
                             : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        __syncwarp();
        if (owner && live) {
            const int nv = min(kStreamT, r.nsteps - k);
            const float4 *row = tile + lane * kRow;
            bool done = false;
            if (((busy >> lane) & 1u) || !(A < p.term)) {
                for (int j = 0; j < nv; ++j) {
                    const float4 cj = row[j];
                    const float t = (1.0f - A) * cj.w;
                    C0 = fmaf(t, cj.x, C0);
                    C1 = fmaf(t, cj.y, C1);
                    C2 = fmaf(t, cj.z, C2);
                    A += t;
                    ++ns;
                    if (A >= p.term) {
                        done = true;
                        break;
                    }
                }
            } else {
                ns += nv;   // nothing in this window can change the composite
            }
            k += kStreamT;
            if (done || k >= r.nsteps) {
                write_pixel(p, r.pix, C0, C1, C2, A, ns);
                live = false;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------- iso surfaces

// Chain value of active source I at a sample.
template <int I, unsigned SIG, int INTERP, typename Idx>
__device__ __forceinline__ float source_value(const KParams &p, const Geo &g)
{
    float v[4];
    fetch_source<I, SIG, INTERP, Idx>(p, g, v);
    return run_chain(p.ch[I], v);
}

template <unsigned SIG, int INTERP, typename Idx, int... Is>
__device__ __forceinline__ void source_values(const KParams &p, const Geo &g, float *v,
                                              std::integer_sequence<int, Is...>)
{
    ((v[Is] = source_value<Is, SIG, INTERP, Idx>(p, g)), ...);
}

// Chain value of active source `which` (a run-time index) at a position.
template <int NACT, unsigned SIG, int INTERP, typename Idx, int I = 0>
__device__ __forceinline__ float value_of(const KParams &p, int which, float x, float y, float z)
{
    if constexpr (I + 1 < NACT) {
        if (which != I) return value_of<NACT, SIG, INTERP, Idx, I + 1>(p, which, x, y, z);
    }
    return source_value<I, SIG, INTERP, Idx>(p, sample_geo<INTERP>(x, y, z));
}

// One ray in iso-surface mode (the reading: samples on the same grid as the
// volume mode; the surface is met at the first sample where some active
// source's chain value reaches its threshold; each crossing source refines
// the crossing by one secant step towards the previous sample, the nearest
// wins (ties: lower source); the normal is the winning source's central-
// difference gradient (one voxel, positions clamped to what the source's
// cells can interpolate: [1/2 - g, n + g - 1/2] with g >= 1 guard layers
// read, [0, n] without), turned towards the viewer; headlight
// Blinn-Phong: rgb = LUT(iso).rgb * (1/4 + 3/4 n.v) + 1/4 (n.v)^32, alpha 1).
// The RL lanes of a group evaluate consecutive samples; a ballot finds the
// first one that crosses.
template <int NACT, unsigned SIG, int INTERP, typename Idx, int RL>
__device__ __forceinline__ void iso_ray(const KParams &p, unsigned idx, int lane)
{
    const int sub = lane & (RL - 1);
    const int base = lane & ~(RL - 1);
    const unsigned gmask = (RL == 32) ? 0xffffffffu : (((1u << RL) - 1u) << base);
    const RayRec r = p.rays[idx];
    float prev[NACT];
#pragma unroll
    for (int i = 0; i < NACT; ++i) prev[i] = 0.0f;
    int win = -1, ns = 0;
    float s_hit = 0.0f;
    for (int k = r.kbeg; k < r.nsteps; k += RL) {
        const int kk = k + sub;
        float v[NACT];
        bool cross = false;
#pragma unroll
        for (int i = 0; i < NACT; ++i) v[i] = -__int_as_float(0x7f800000);
        if (kk < r.nsteps) {
            const float s = (float)kk * p.step;
            const Geo g = sample_geo<INTERP>(fmaf(s, r.dx, r.ex), fmaf(s, r.dy, r.ey), fmaf(s, r.dz, r.ez));
            source_values<SIG, INTERP, Idx>(p, g, v, std::make_integer_sequence<int, NACT>{});
#pragma unroll
            for (int i = 0; i < NACT; ++i) cross |= v[i] >= p.iso[i];
        }
        const unsigned m = (__ballot_sync(gmask, cross) >> base) & (RL == 32 ? 0xffffffffu : ((1u << RL) - 1u));
        if (m) {
            const int j = __ffs(m) - 1;
            const int kj = k + j;
            const float sj = (float)kj * p.step;
            float best = __int_as_float(0x7f800000);
#pragma unroll
            for (int i = 0; i < NACT; ++i) {
                const float vj = __shfl_sync(gmask, v[i], j, RL);
                const float vq = __shfl_sync(gmask, v[i], j > 0 ? j - 1 : 0, RL);
                const float vp = j > 0 ? vq : prev[i];
                if (vj >= p.iso[i]) {
                    const float th = kj == r.kbeg ? sj
                                   : (sj - p.step) + p.step * (p.iso[i] - vp) / (vj - vp);
                    if (th < best) {
                        best = th;
                        win = i;
                    }
                }
            }
            s_hit = best;
            ns += j + 1;
            break;
        }
#pragma unroll
        for (int i = 0; i < NACT; ++i) prev[i] = __shfl_sync(gmask, v[i], RL - 1, RL);
        ns += min(RL, r.nsteps - k);
    }
    if (sub != 0) return;
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f;
    if (win >= 0) {
        const float qx = fmaf(s_hit, r.dx, r.ex), qy = fmaf(s_hit, r.dy, r.ey), qz = fmaf(s_hit, r.dz, r.ez);
        // central differences over one voxel, positions clamped to the range
        // the winning source's readable cells interpolate (guard layers read:
        // -lo, two at most in this mode; none with interpolation off)
        const int gw = INTERP ? -p.src[win].lo : 0;
        const float plo = gw > 0 ? 0.5f - (float)gw : 0.0f, pad = gw > 0 ? (float)gw - 0.5f : 0.0f;
        const float xp = fminf(qx + 1.0f, (float)p.nx + pad), xm = fmaxf(qx - 1.0f, plo);
        const float yp = fminf(qy + 1.0f, (float)p.ny + pad), ym = fmaxf(qy - 1.0f, plo);
        const float zp = fminf(qz + 1.0f, (float)p.nz + pad), zm = fmaxf(qz - 1.0f, plo);
        const float gx = xp > xm ? (value_of<NACT, SIG, INTERP, Idx>(p, win, xp, qy, qz) -
                                    value_of<NACT, SIG, INTERP, Idx>(p, win, xm, qy, qz)) / (xp - xm) : 0.0f;
        const float gy = yp > ym ? (value_of<NACT, SIG, INTERP, Idx>(p, win, qx, yp, qz) -
                                    value_of<NACT, SIG, INTERP, Idx>(p, win, qx, ym, qz)) / (yp - ym) : 0.0f;
        const float gz = zp > zm ? (value_of<NACT, SIG, INTERP, Idx>(p, win, qx, qy, zp) -
                                    value_of<NACT, SIG, INTERP, Idx>(p, win, qx, qy, zm)) / (zp - zm) : 0.0f;
        const float gl = sqrtf(fmaf(gx, gx, fmaf(gy, gy, gz * gz)));
        const float ndl = gl > 0.0f ? fabsf(fmaf(gx, r.dx, fmaf(gy, r.dy, gz * r.dz))) / gl : 1.0f;
        float spec = ndl;
#pragma unroll
        for (int i = 0; i < 5; ++i) spec *= spec;          // ndl^32
        const float4 col = classify(p.lut[win], p.iso[win]);
        const float diff = fmaf(0.75f, ndl, 0.25f);
        C0 = clamp01(fmaf(col.x, diff, 0.25f * spec));
        C1 = clamp01(fmaf(col.y, diff, 0.25f * spec));
        C2 = clamp01(fmaf(col.z, diff, 0.25f * spec));
        A = 1.0f;
    }
    write_pixel(p, r.pix, C0, C1, C2, A, ns);
}

// Persistent warps over the ray list, iso-surface mode.
template <int NACT, unsigned SIG, int INTERP, typename Idx, int RL>
__device__ __forceinline__ void march_iso(const KParams &p)
{
    constexpr unsigned RAYS = 32 / RL;
    const int lane = threadIdx.x & 31;
    const unsigned n_rays = *(volatile unsigned *)&p.ctr->n_rays;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&p.ctr->next, RAYS);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_rays) break;
        const unsigned idx = base + (unsigned)(lane / RL);
        if (idx < n_rays) iso_ray<NACT, SIG, INTERP, Idx, RL>(p, idx, lane);
    }
}

// The active sources' LUTs into shared memory.  For a single source it
// returns (block-uniform) whether a sample can have opacity 0: a LUT entry
// with opacity <= 0 or a weight <= 0; otherwise the march has no use for its
// vote on groups with nothing to composite.  With several sources the march
// has no such vote, and this returns false.
template <int NACT>
__device__ __forceinline__ bool load_luts(const KParams &p, float4 *s_lut)
{
    if constexpr (NACT == 1) {
        int zero = 0;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) {
            const float4 e = __ldg(p.lut[0] + i);
            s_lut[i] = e;
            zero |= !(e.w > 0.0f);
        }
        if (threadIdx.x == 0) zero |= !(p.src[0].w > 0.0f);
        return __syncthreads_or(zero) != 0;
    } else {
        for (int i = threadIdx.x; i < NACT * 256; i += blockDim.x) s_lut[i] = __ldg(p.lut[i >> 8] + (i & 255));
        __syncthreads();
        return false;
    }
}

// The zero-copy frame kernel (128 threads, at most 64 registers per thread).
template <int NACT, unsigned SIG, int INTERP, typename Idx, int RL, int MODE = MODE_PLAIN>
__global__ void __launch_bounds__(kMarchThreads, kMarchBlocksPerSM) k_raycast(const __grid_constant__ KParams p)
{
    __shared__ float4 s_lut[NACT * 256];
    // the vote for groups with nothing to composite is compiled into the
    // single-source kernels only: with several sources a sample composites
    // nothing only where every source is transparent at once, and the larger
    // kernel measured 1.2 % slower on the dense three-source frame
    const bool zskip = load_luts<NACT>(p, s_lut);
    using Shader = ZeroCopyShader<NACT, SIG, INTERP, Idx, MODE == MODE_TOUCH>;
    if constexpr (MODE == MODE_LONG) {
        if (NACT == 1 && zskip)
            march_long<Shader, NACT == 1>(p, s_lut);
        else
            march_long<Shader, false>(p, s_lut);
    }
    else if constexpr (MODE == MODE_ISO)
        march_iso<NACT, SIG, INTERP, Idx, RL>(p);
    else if constexpr (MODE == MODE_SKIP) {
        // the empty bits in shared memory (a ray tests one per macro cell it
        // enters), when they fit: 1024 words, 32768 macro cells
        __shared__ unsigned s_empty[kSkipSharedWords];
        const long long words = ((long long)p.sgx * p.sgy * p.sgz + 31) / 32;
        const bool staged = words <= kSkipSharedWords;
        if (staged)
            for (int i = threadIdx.x; i < (int)words; i += blockDim.x) s_empty[i] = __ldg(p.empty + i);
        __syncthreads();
        if (NACT == 1 && zskip)
            march<NACT, Shader, RL, false, true, NACT == 1>(p, s_lut, staged ? s_empty : nullptr);
        else
            march<NACT, Shader, RL, false, true, false>(p, s_lut, staged ? s_empty : nullptr);
    } else if (NACT == 1 && zskip) {
        march<NACT, Shader, RL, MODE == MODE_LABEL, false, NACT == 1>(p, s_lut);
    } else {
        march<NACT, Shader, RL, MODE == MODE_LABEL, false, false>(p, s_lut);
    }
}

// Copy the ray list (at most `cap` records) and its length out of the workspace.
static __global__ void k_copy_rays(const __grid_constant__ KParams p, RayRec *out, long long cap,
                                   int *count)
{
    const unsigned n = p.ctr->n_rays;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (int)n;
    const long long m = min((long long)n, cap);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = p.rays[i];
}

}  // namespace isaac
