// source_copy.cu -- the source contract of Sec. 3.2 beyond zero copy:
// isaac_copy_source (a source whose memory is not persistent, copied through
// its accessor into a buffer the caller keeps) and the per-source update
// callback, called for every source before an entry point reads them.
#include <algorithm>
#include <cstring>

#include "common.h"
#include "raycast.cuh"

namespace isaac {

struct KCopy {
    const float *src;         // element of interior cell (0,0,0), component 0
    long long sx, sy, sz, sc;
    int fdim, g;              // components; apron cells copied per side (0 or 1)
    int nx, ny, nz;           // interior cells
    float *dst;               // (nz+2g)(ny+2g)(nx+2g) cells x fdim, x fastest, AoS
};

constexpr int kCopyThreads = 256, kCopyUnroll = 8;

// One warp per (y, z) row of the copied region at a time (rows strided over
// every warp of the grid), its lanes along the row: a row is (nx+2g)*fdim
// contiguous destination elements, and each lane issues up to kCopyUnroll
// strided reads (32 elements apart) before its writes, so even the short
// rows of a scalar source keep 8 loads per lane in flight.  FD = fdim (1..4),
// so the element -> (cell, component) split is a division by a constant.
template <int FD>
static __global__ void __launch_bounds__(kCopyThreads) k_copy_source(const __grid_constant__ KCopy p)
{
    const int X = p.nx + 2 * p.g, Y = p.ny + 2 * p.g, Z = p.nz + 2 * p.g;
    const int row_len = X * FD;
    const long long rows = (long long)Y * Z;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (kCopyThreads / 32);
    for (long long row = blockIdx.x * (long long)(kCopyThreads / 32) + (threadIdx.x >> 5); row < rows;
         row += nwarps) {
        const int y = (int)(row % Y) - p.g, z = (int)(row / Y) - p.g;
        const float *srow = p.src + (long long)y * p.sy + (long long)z * p.sz;
        float *drow = p.dst + row * row_len;
        for (int i0 = lane; i0 < row_len; i0 += 32 * kCopyUnroll) {
            float v[kCopyUnroll];
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u) {
                const int i = i0 + 32 * u;
                if (i < row_len) {
                    const int x = i / FD - p.g, c = i - (i / FD) * FD;
                    v[u] = __ldg(srow + (long long)x * p.sx + (long long)c * p.sc);
                }
            }
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u) {
                const int i = i0 + 32 * u;
                if (i < row_len) drow[i] = v[u];
            }
        }
    }
}

// The update hook (per calling thread).
static thread_local isaac_update_fn t_update = nullptr;
static thread_local void *t_update_user = nullptr;

void update_sources(int32_t n_sources, uint32_t active_mask)
{
    if (!t_update || n_sources < 1 || n_sources > ISAAC_MAX_SOURCES) return;
    for (int s = 0; s < n_sources; ++s) t_update(s, (int32_t)((active_mask >> s) & 1u), t_update_user);
}

}  // namespace isaac

using namespace isaac;

extern "C" int isaac_copy_source(const isaac_source *src, const int64_t n[3], void *dst,
                                 int64_t dst_bytes, isaac_source *out, void *stream)
{
    clear_error();
    if (!src || !n || !dst || !out) return fail(ISAAC_EINVAL, "src, n, dst and out are required");
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || n[a] > (1 << 20)) return fail(ISAAC_EINVAL, "n[%d] = %lld", a, (long long)n[a]);
    if (((uintptr_t)dst) % 16) return fail(ISAAC_EINVAL, "dst must be 16-byte aligned");
    KSource ks;
    unsigned nib;
    bool wide;
    // validated as the renderer would read it with interpolation on
    int rc = prepare_source(*src, 0, n, 1, 1.0f, 4, ks, &nib, &wide);
    if (rc) return rc;
    KCopy p;
    p.g = src->guard >= 1 ? 1 : 0;
    p.fdim = src->f_dim;
    p.nx = (int)n[0];
    p.ny = (int)n[1];
    p.nz = (int)n[2];
    const long long X = p.nx + 2 * p.g, Y = p.ny + 2 * p.g, Z = p.nz + 2 * p.g;
    if ((long double)X * Y * Z * p.fdim * 4 > 4.0e18L) return fail(ISAAC_ENOMEM, "the copy is too large");
    const long long elems = X * Y * Z * p.fdim;
    if (dst_bytes < elems * 4)
        return fail(ISAAC_ENOMEM, "dst holds %lld bytes, the copy needs %lld", (long long)dst_bytes, elems * 4);
    p.src = ks.base;
    p.sx = ks.sx;
    p.sy = ks.sy;
    p.sz = ks.sz;
    p.sc = ks.sc;
    p.dst = static_cast<float *>(dst);
    if ((long long)X * p.fdim > 0x7fffffffLL) return fail(ISAAC_ENOTSUP, "a row of the copy is too long");
    const long long rows = Y * Z;
    const long long wpb = kCopyThreads / 32;   // a warp per row
    const unsigned blocks = (unsigned)std::max(1LL, std::min((rows + wpb - 1) / wpb, (long long)sm_count() * 8));
    const cudaStream_t st = (cudaStream_t)stream;
    switch (p.fdim) {
    case 1: k_copy_source<1><<<blocks, kCopyThreads, 0, st>>>(p); break;
    case 2: k_copy_source<2><<<blocks, kCopyThreads, 0, st>>>(p); break;
    case 3: k_copy_source<3><<<blocks, kCopyThreads, 0, st>>>(p); break;
    default: k_copy_source<4><<<blocks, kCopyThreads, 0, st>>>(p); break;
    }
    rc = check_cuda("isaac_copy_source launch");
    if (rc) return rc;
    isaac_source o;
    memset(&o, 0, sizeof o);
    o.ptr = dst;
    o.extent = elems;
    o.stride[0] = p.fdim;
    o.stride[1] = p.fdim * X;
    o.stride[2] = p.fdim * X * Y;
    o.offset = p.g * (o.stride[0] + o.stride[1] + o.stride[2]);
    o.comp_stride = 1;
    o.f_dim = p.fdim;
    o.guard = p.g;
    *out = o;
    return ISAAC_OK;
}

extern "C" int isaac_set_update_hook(isaac_update_fn fn, void *user)
{
    clear_error();
    t_update = fn;
    t_update_user = user;
    return ISAAC_OK;
}
