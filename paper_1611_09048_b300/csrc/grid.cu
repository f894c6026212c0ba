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
#include "raycast.cuh"

namespace isaac {

struct KGrid {
    KSource src[ISAAC_MAX_ACTIVE];
    KChain ch[ISAAC_MAX_ACTIVE];
    const float4 *lut[ISAAC_MAX_ACTIVE];
    int nact;
    int nx, ny, nz;
    int cell;
    int gx, gy, gz;
    float *grid;
};

constexpr int kGridThreads = 352;   // 11 warps: one pass over the 18 x 18 columns of a 16^3 cell
// z-cells whose loads a thread issues together: 16 on the scalar fast paths
// (a walk is bound by the loads in flight), 8 where a cell has several values
template <int FD> constexpr int grid_z() { return FD == 1 ? 16 : 8; }

// One block per column (i, j) of macro cells.  Each thread owns (x, y)
// columns of the column's apron-extended footprint -- consecutive threads
// take consecutive x, so a warp's loads are coalesced -- and walks its column
// once in z, grid_z() cells at a time with their loads issued together.  Cell z
// belongs to macro cells k with k*cell - 1 <= z <= (k+1)*cell (at most two
// for cell >= 2), so a thread keeps two running maxima, for the lowest open
// macro cell and the next; when z leaves the lower one, the warp's maximum
// is folded into the grid with one atomic max (opacities are >= 0, so their
// bit patterns order like the values; the grid is zeroed first).
// NS > 0: NS active sources known at compile time, and with NS == 1 and
// FD > 0 the source's f_dim too (the scalar fast path); 0: read at run time.
template <int NS, int FD>
static __global__ void __launch_bounds__(kGridThreads, 2) k_opacity_grid(const __grid_constant__ KGrid p)
{
    constexpr int kGridZ = grid_z<(NS == 1 && FD == 1) ? 1 : 4>();
    __shared__ float s_alpha[ISAAC_MAX_ACTIVE * 256];
    const int nact = NS ? NS : p.nact;
    for (int i = threadIdx.x; i < nact * 256; i += blockDim.x) s_alpha[i] = __ldg(&p.lut[i >> 8][i & 255].w);
    __syncthreads();
    const int gi = blockIdx.x % p.gx, gj = blockIdx.x / p.gx;
    const int x0 = max(gi * p.cell - 1, -1), x1 = min((gi + 1) * p.cell, p.nx);
    const int y0 = max(gj * p.cell - 1, -1), y1 = min((gj + 1) * p.cell, p.ny);
    const int wx = x1 - x0 + 1, wy = y1 - y0 + 1;
    const int lane = threadIdx.x & 31;
    unsigned *grid_bits = reinterpret_cast<unsigned *>(p.grid);
    auto flush = [&](int k, float m) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.0f)
            atomicMax(grid_bits + ((long long)k * p.gy + gj) * p.gx + gi, __float_as_uint(m));
    };
    // every thread of the block runs the same number of column passes, so the
    // warp-wide reductions in flush() see all 32 lanes
    const int passes = (wx * wy + (int)blockDim.x - 1) / (int)blockDim.x;
    for (int pass = 0; pass < passes; ++pass) {
        const int col = pass * blockDim.x + threadIdx.x;
        const bool live = col < wx * wy;
        const int x = x0 + (live ? col % wx : 0), y = y0 + (live ? col / wx : 0);
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
        int ka = 0;                                         // lowest open macro cell
        int end_a = min(p.cell, p.nz);                      // its last z
        int start_b = p.gz > 1 ? p.cell - 1 : 0x7fffffff;   // first z of cell ka + 1
        float ma = 0.0f, mb = 0.0f;                         // running maxima of cells ka, ka + 1
        for (int zb = -1; zb <= p.nz; zb += kGridZ) {
            float a[kGridZ];
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
#pragma unroll
            for (int j = 0; j < kGridZ; ++j) {
                const int z = zb + j;
                if (z > p.nz) break;
                if (z > end_a) {                  // z left cell ka: fold it, open the next
                    flush(ka, ma);
                    ++ka;
                    ma = mb;
                    mb = 0.0f;
                    end_a = min((ka + 1) * p.cell, p.nz);
                    start_b = ka + 1 < p.gz ? (ka + 1) * p.cell - 1 : 0x7fffffff;
                }
                const float al = live ? clamp01(a[j]) : 0.0f;
                ma = fmaxf(ma, al);
                mb = z >= start_b ? fmaxf(mb, al) : mb;
            }
        }
        flush(ka, ma);
        if (ka + 1 < p.gz) flush(ka + 1, mb);
    }
}

// ------------------------------------------------------ value-range grid

// Order-preserving map of non-NaN floats to unsigned (atomic min/max on floats).
__device__ __forceinline__ unsigned ord_enc(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

struct KRange {
    KSource src;          // the source of this pass
    int nx, ny, nz, cell, gx, gy, gz;
    int slots, slot0;     // components per macro cell in all, first of this source
    unsigned *r;          // (min, max) pairs, order-encoded until k_range_decode
};

static __global__ void k_range_init(unsigned *r, long long pairs)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pairs;
         i += (long long)gridDim.x * blockDim.x) {
        r[2 * i] = 0xff800000u;        // ord_enc(+inf)
        r[2 * i + 1] = 0x007fffffu;    // ord_enc(-inf)
    }
}

static __global__ void k_range_decode(unsigned *r, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        r[i] = __float_as_uint(ord_dec(r[i]));
}

// Per macro cell (same boxes as the opacity grid) and component of one
// source, the smallest and largest value read; a NaN widens the component to
// [-inf, +inf].  Same walk as k_opacity_grid: one block per macro-cell
// column, one z-walk per (x, y) column with a two-cell window; a warp's
// minima and maxima are folded into the grid with atomic min / max.
template <int FD>
static __global__ void __launch_bounds__(kGridThreads, 2) k_range_grid(const __grid_constant__ KRange p)
{
    constexpr int kGridZ = grid_z<FD>();
    const float inf = __int_as_float(0x7f800000);
    const KSource &q = p.src;
    const int gi = blockIdx.x % p.gx, gj = blockIdx.x / p.gx;
    const int x0 = max(gi * p.cell - 1, -1), x1 = min((gi + 1) * p.cell, p.nx);
    const int y0 = max(gj * p.cell - 1, -1), y1 = min((gj + 1) * p.cell, p.ny);
    const int wx = x1 - x0 + 1, wy = y1 - y0 + 1;
    const int lane = threadIdx.x & 31;
    auto flush = [&](int k, const float (&mn)[FD], const float (&mx)[FD]) {
        const long long base = (((long long)k * p.gy + gj) * p.gx + gi) * p.slots + p.slot0;
#pragma unroll
        for (int c = 0; c < FD; ++c) {
            const unsigned lo = __reduce_min_sync(0xffffffffu, ord_enc(mn[c]));
            const unsigned hi = __reduce_max_sync(0xffffffffu, ord_enc(mx[c]));
            if (lane == 0) {
                atomicMin(p.r + 2 * (base + c), lo);
                atomicMax(p.r + 2 * (base + c) + 1, hi);
            }
        }
    };
    const int passes = (wx * wy + (int)blockDim.x - 1) / (int)blockDim.x;
    for (int pass = 0; pass < passes; ++pass) {
        const int col = pass * blockDim.x + threadIdx.x;
        const bool live = col < wx * wy;
        const int x = x0 + (live ? col % wx : 0), y = y0 + (live ? col / wx : 0);
        const int xi = min(max(x, q.lo), p.nx - 1 + q.hi_pad);
        const int yi = min(max(y, q.lo), p.ny - 1 + q.hi_pad);
        const float *cp = q.base + ((long long)xi * q.sx + (long long)yi * q.sy);
        int ka = 0;
        int end_a = min(p.cell, p.nz);
        int start_b = p.gz > 1 ? p.cell - 1 : 0x7fffffff;
        float amn[FD], amx[FD], bmn[FD], bmx[FD];
#pragma unroll
        for (int c = 0; c < FD; ++c) {
            amn[c] = bmn[c] = inf;
            amx[c] = bmx[c] = -inf;
        }
        for (int zb = -1; zb <= p.nz; zb += kGridZ) {
            float v[kGridZ][FD];
#pragma unroll
            for (int j = 0; j < kGridZ; ++j) {
                const int zi = min(max(min(zb + j, p.nz), q.lo), p.nz - 1 + q.hi_pad);
                const float *b = cp + (long long)zi * q.sz;
#pragma unroll
                for (int c = 0; c < FD; ++c) v[j][c] = __ldg(b + (long long)c * q.sc);
            }
#pragma unroll
            for (int j = 0; j < kGridZ; ++j) {
                const int z = zb + j;
                if (z > p.nz) break;
                if (z > end_a) {
                    flush(ka, amn, amx);
                    ++ka;
#pragma unroll
                    for (int c = 0; c < FD; ++c) {
                        amn[c] = bmn[c];
                        amx[c] = bmx[c];
                        bmn[c] = inf;
                        bmx[c] = -inf;
                    }
                    end_a = min((ka + 1) * p.cell, p.nz);
                    start_b = ka + 1 < p.gz ? (ka + 1) * p.cell - 1 : 0x7fffffff;
                }
#pragma unroll
                for (int c = 0; c < FD; ++c) {
                    const float val = v[j][c];
                    const bool nan = !(val == val);
                    const float lo = !live ? inf : (nan ? -inf : val);
                    const float hi = !live ? -inf : (nan ? inf : val);
                    amn[c] = fminf(amn[c], lo);
                    amx[c] = fmaxf(amx[c], hi);
                    if (z >= start_b) {
                        bmn[c] = fminf(bmn[c], lo);
                        bmx[c] = fmaxf(bmx[c], hi);
                    }
                }
            }
        }
        flush(ka, amn, amx);
        if (ka + 1 < p.gz) flush(ka + 1, bmn, bmx);
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
    unsigned char *flags;
};

// A macro cell is empty when, for the components' value ranges over its box,
// every source with weight > 0 has LUT opacity exactly 0 on every entry that
// the interval of its chain result can reach, and every reachable LUT entry
// of every source is finite.  A trilinear sample whose position lies in the
// cell interpolates between values of the box, so its opacity is then 0 and
// compositing it is a no-op.  The interpolation itself may round a few ulps
// outside the corners' range: the ranges are widened by 10^-6 relative first.
static __global__ void k_empty_flags(const __grid_constant__ KEmpty p)
{
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < p.cells;
         g += (long long)gridDim.x * blockDim.x) {
        bool empty = true;
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
        p.flags[g] = empty ? 1 : 0;
    }
}

int launch_empty_flags(const KParams &kp, int nact, const float *ranges, int slots, long long cells,
                       unsigned char *flags, cudaStream_t st)
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
    if (((uintptr_t)luts) % 16) return fail(ISAAC_EINVAL, "luts must be 16-byte aligned");
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
    if (p.nact == 0) {
        if (cudaMemsetAsync(grid, 0, (size_t)cells * sizeof(float), (cudaStream_t)stream) != cudaSuccess)
            return check_cuda("isaac_opacity_grid memset");
        return ISAAC_OK;
    }
    if (cudaMemsetAsync(grid, 0, (size_t)cells * sizeof(float), (cudaStream_t)stream) != cudaSuccess)
        return check_cuda("isaac_opacity_grid memset");
    const dim3 blocks((unsigned)(p.gx * p.gy));
    const cudaStream_t st = (cudaStream_t)stream;
    if (p.nact == 1 && p.src[0].fdim == 1 && p.ch[0].n == 0)
        k_opacity_grid<1, 1><<<blocks, kGridThreads, 0, st>>>(p);
    else if (p.nact == 3)
        k_opacity_grid<3, 0><<<blocks, kGridThreads, 0, st>>>(p);
    else
        k_opacity_grid<0, 0><<<blocks, kGridThreads, 0, st>>>(p);
    return check_cuda("isaac_opacity_grid launch");
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
    unsigned *ru = reinterpret_cast<unsigned *>(ranges);
    const long long pairs = cells * slots;
    const unsigned eb = (unsigned)std::max(1LL, std::min((pairs + 255) / 256, 148LL * 8));
    k_range_init<<<eb, 256, 0, st>>>(ru, pairs);
    r.slots = slots;
    r.r = ru;
    int slot = 0;
    for (int a = 0; a < nact; ++a) {
        r.src = ks[a];
        r.slot0 = slot;
        const dim3 blocks((unsigned)(r.gx * r.gy));
        switch (ks[a].fdim) {
        case 1: k_range_grid<1><<<blocks, kGridThreads, 0, st>>>(r); break;
        case 2: k_range_grid<2><<<blocks, kGridThreads, 0, st>>>(r); break;
        case 3: k_range_grid<3><<<blocks, kGridThreads, 0, st>>>(r); break;
        default: k_range_grid<4><<<blocks, kGridThreads, 0, st>>>(r); break;
        }
        slot += ks[a].fdim;
    }
    k_range_decode<<<eb, 256, 0, st>>>(ru, 2 * pairs);
    return check_cuda("isaac_range_grid launch");
}
