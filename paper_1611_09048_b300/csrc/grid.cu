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
constexpr int kGridZ = 8;           // z-cells whose loads are in flight together

// One block per column (i, j) of macro cells.  Each thread owns (x, y)
// columns of the column's apron-extended footprint -- consecutive threads
// take consecutive x, so a warp's loads are coalesced -- and walks its column
// once in z, kGridZ cells at a time with their loads issued together.  Cell z
// belongs to macro cells k with k*cell - 1 <= z <= (k+1)*cell (at most two
// for cell >= 2), so a thread keeps two running maxima, for the lowest open
// macro cell and the next; when z leaves the lower one, the warp's maximum
// is folded into the grid with one atomic max (opacities are >= 0, so their
// bit patterns order like the values; the grid is zeroed first).
static __global__ void __launch_bounds__(kGridThreads, 2) k_opacity_grid(const __grid_constant__ KGrid p)
{
    __shared__ float s_alpha[ISAAC_MAX_ACTIVE * 256];
    for (int i = threadIdx.x; i < p.nact * 256; i += blockDim.x) s_alpha[i] = __ldg(&p.lut[i >> 8][i & 255].w);
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
            if (s < p.nact) {
                const KSource &q = p.src[s];
                const int xi = min(max(x, q.lo), p.nx - 1 + q.hi_pad);
                const int yi = min(max(y, q.lo), p.ny - 1 + q.hi_pad);
                cp[s] = q.base + ((long long)xi * q.sx + (long long)yi * q.sy);
            }
        }
        int ka = 0;                               // lowest open macro cell
        int end_a = min(p.cell, p.nz);            // its last z
        float ma = 0.0f, mb = 0.0f;               // running maxima of cells ka, ka + 1
        for (int zb = -1; zb <= p.nz; zb += kGridZ) {
            float a[kGridZ];
#pragma unroll
            for (int j = 0; j < kGridZ; ++j) a[j] = 0.0f;
#pragma unroll
            for (int s = 0; s < ISAAC_MAX_ACTIVE; ++s) {
                if (s >= p.nact) break;
                const KSource &q = p.src[s];
                float v[kGridZ][4];
#pragma unroll
                for (int j = 0; j < kGridZ; ++j) {
                    const int zi = min(max(min(zb + j, p.nz), q.lo), p.nz - 1 + q.hi_pad);
                    const float *b = cp[s] + (long long)zi * q.sz;
                    v[j][0] = __ldg(b);
#pragma unroll
                    for (int c = 1; c < 4; ++c) v[j][c] = c < q.fdim ? __ldg(b + (long long)c * q.sc) : 0.0f;
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
                }
                const float al = live ? clamp01(a[j]) : 0.0f;
                ma = fmaxf(ma, al);
                if (z >= (ka + 1) * p.cell - 1 && ka + 1 < p.gz) mb = fmaxf(mb, al);
            }
        }
        flush(ka, ma);
        if (ka + 1 < p.gz) flush(ka + 1, mb);
    }
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
    k_opacity_grid<<<(unsigned)(p.gx * p.gy), kGridThreads, 0, (cudaStream_t)stream>>>(p);
    return check_cuda("isaac_opacity_grid launch");
}
