// composite.cu -- isaac_composite: sort-last compositing of the partial images
// of disjoint sub-volumes (Sec. 3.4), per pixel in visibility order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "common.h"
#include "raycast.cuh"

namespace isaac {

constexpr int kMaxLayers = 16;

struct KComposite {
    const float4 *rgba[kMaxLayers];
    const float *depth[kMaxLayers];
    int n;
    long long npix;
    float bg[4];
    uchar4 *out8;
    float4 *out32;
};

// One thread per pixel, N = the number of layers (compile time, so every
// array lives in registers).  All 5N loads are issued first.  The rank of
// layer l is the number of layers m whose key (depth, m) is smaller (a NaN
// depth counts as +inf), a permutation, so equal depths keep layer order.
// The over operator then runs front to back in rank order, each step picking
// its layer by register selects.  Reads N * 20 bytes and writes 4 (+16) per
// pixel.
template <int N>
static __global__ void __launch_bounds__(256) k_composite(const __grid_constant__ KComposite p)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.npix;
         i += (long long)gridDim.x * blockDim.x) {
        float d[N];
        float4 c[N];
#pragma unroll
        for (int l = 0; l < N; ++l) {
            d[l] = __ldg(p.depth[l] + i);
            c[l] = __ldg(p.rgba[l] + i);
        }
#pragma unroll
        for (int l = 0; l < N; ++l)
            if (d[l] != d[l]) d[l] = __int_as_float(0x7f800000);
        int rank[N];
#pragma unroll
        for (int l = 0; l < N; ++l) {
            int r = 0;
#pragma unroll
            for (int m = 0; m < N; ++m)
                if (m != l) r += (d[m] < d[l] || (m < l && d[m] == d[l])) ? 1 : 0;
            rank[l] = r;
        }
        float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            float4 q = c[0];
#pragma unroll
            for (int l = 1; l < N; ++l)
                if (rank[l] == r) q = c[l];
            const float T = 1.0f - A;
            C0 = fmaf(T, q.x, C0);
            C1 = fmaf(T, q.y, C1);
            C2 = fmaf(T, q.z, C2);
            A = fmaf(T, q.w, A);
        }
        const float T = 1.0f - A;
        const float o0 = fmaf(T, p.bg[0], C0), o1 = fmaf(T, p.bg[1], C1);
        const float o2 = fmaf(T, p.bg[2], C2), o3 = fmaf(T, p.bg[3], A);
        p.out8[i] = make_uchar4(quant8(o0), quant8(o1), quant8(o2), quant8(o3));
        if (p.out32) p.out32[i] = make_float4(o0, o1, o2, o3);
    }
}

using CompositeFn = void (*)(KComposite);

template <int... Ns>
static CompositeFn composite_fn(int n, std::integer_sequence<int, Ns...>)
{
    static const CompositeFn table[] = {k_composite<Ns + 1>...};
    return table[n - 1];
}

}  // namespace isaac

using namespace isaac;

extern "C" int isaac_composite(const float *const *layers_rgba32, const float *const *layers_depth,
                               int32_t n_layers, int32_t width, int32_t height, const float *bg,
                               uint8_t *rgba8, float *rgba32, void *stream)
{
    clear_error();
    if (!layers_rgba32 || !layers_depth || !bg || !rgba8)
        return fail(ISAAC_EINVAL, "layers, depths, bg and rgba8 are required");
    if (n_layers < 1 || n_layers > kMaxLayers)
        return fail(ISAAC_EINVAL, "n_layers %d outside 1..%d", n_layers, kMaxLayers);
    if (width < 1 || height < 1 || (long long)width * height > (1LL << 31))
        return fail(ISAAC_EINVAL, "image %dx%d", width, height);
    if (((uintptr_t)rgba8) % 4 || ((uintptr_t)rgba32) % 16)
        return fail(ISAAC_EINVAL, "output pointers are misaligned");
    KComposite p;
    memset(&p, 0, sizeof p);
    for (int l = 0; l < n_layers; ++l) {
        if (!layers_rgba32[l] || !layers_depth[l] || ((uintptr_t)layers_rgba32[l]) % 16 ||
            ((uintptr_t)layers_depth[l]) % 4)
            return fail(ISAAC_EINVAL, "layer %d: missing or misaligned buffers", l);
        p.rgba[l] = reinterpret_cast<const float4 *>(layers_rgba32[l]);
        p.depth[l] = layers_depth[l];
    }
    for (int c = 0; c < 4; ++c) {
        if (!std::isfinite(bg[c])) return fail(ISAAC_EINVAL, "bg is not finite");
        p.bg[c] = bg[c];
    }
    p.n = n_layers;
    p.npix = (long long)width * height;
    p.out8 = reinterpret_cast<uchar4 *>(rgba8);
    p.out32 = reinterpret_cast<float4 *>(rgba32);
    const int sms = sm_count();
    const long long blocks = std::max(1LL, std::min((p.npix + 255) / 256, (long long)sms * 8));
    composite_fn(n_layers, std::make_integer_sequence<int, kMaxLayers>{})
        <<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p);
    return check_cuda("isaac_composite launch");
}
