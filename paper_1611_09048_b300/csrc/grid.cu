// grid.cu -- isaac_opacity_grid: the max-opacity grid over macro cells.
//
// Macro cell (i, j, k) of `cell`^3 cells covers the cells [i*cell - 1,
// (i+1)*cell] per axis (the one-cell apron that trilinear samples inside the
// macro cell read), clipped to [-1, n]; its value is the largest blended
// opacity clamp(sum_s w_s * LUT_s(chain_s(v_s)).alpha, 0, 1) over those cells,
// each source read at the cell itself (clamped to the border without guards).
// One 256-thread block per macro cell.
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

__device__ __forceinline__ float alpha_at(const KGrid &p, const float *s_alpha, int x, int y, int z)
{
    float a = 0.0f;
#pragma unroll
    for (int s = 0; s < ISAAC_MAX_ACTIVE; ++s) {
        if (s >= p.nact) break;
        const KSource &q = p.src[s];
        const int xi = min(max(x, q.lo), p.nx - 1 + q.hi_pad);
        const int yi = min(max(y, q.lo), p.ny - 1 + q.hi_pad);
        const int zi = min(max(z, q.lo), p.nz - 1 + q.hi_pad);
        const float *b = q.base + ((long long)xi * q.sx + (long long)yi * q.sy + (long long)zi * q.sz);
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = c < q.fdim ? __ldg(b + (long long)c * q.sc) : 0.0f;
        const float xv = run_chain(p.ch[s], v);
        const float pos = clamp01(xv) * 255.0f;
        const int j = min((int)pos, 254);
        const float f = pos - (float)j;
        a = fmaf(q.w, lerp1(s_alpha[s * 256 + j], s_alpha[s * 256 + j + 1], f), a);
    }
    return clamp01(a);
}

static __global__ void __launch_bounds__(256) k_opacity_grid(const __grid_constant__ KGrid p)
{
    __shared__ float s_alpha[ISAAC_MAX_ACTIVE * 256];
    __shared__ float s_red[8];
    for (int i = threadIdx.x; i < p.nact * 256; i += blockDim.x) s_alpha[i] = __ldg(&p.lut[i >> 8][i & 255].w);
    __syncthreads();
    const int g = blockIdx.x;
    const int gi = g % p.gx, gj = (g / p.gx) % p.gy, gk = g / (p.gx * p.gy);
    const int x0 = max(gi * p.cell - 1, -1), x1 = min((gi + 1) * p.cell, p.nx);
    const int y0 = max(gj * p.cell - 1, -1), y1 = min((gj + 1) * p.cell, p.ny);
    const int z0 = max(gk * p.cell - 1, -1), z1 = min((gk + 1) * p.cell, p.nz);
    const int wx = x1 - x0 + 1, wy = y1 - y0 + 1, wz = z1 - z0 + 1;
    const int total = wx * wy * wz;
    float best = 0.0f;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int x = x0 + i % wx, y = y0 + (i / wx) % wy, z = z0 + i / (wx * wy);
        best = fmaxf(best, alpha_at(p, s_alpha, x, y, z));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_red[w]);
        p.grid[g] = m;
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
    if (cell < 1 || cell > 1024) return fail(ISAAC_EINVAL, "cell %d outside 1..1024", cell);
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
    k_opacity_grid<<<(unsigned)cells, 256, 0, (cudaStream_t)stream>>>(p);
    return check_cuda("isaac_opacity_grid launch");
}
