// kernel_table.h -- host-side view of the precompiled frame kernels.
#pragma once

#include <algorithm>
#include <type_traits>
#include <cuda_runtime.h>

namespace isaac {

struct KParams;
struct RayRec;
using FrameLaunch = void (*)(const KParams &, dim3, cudaStream_t);

struct ZcEntry {
    int nact;
    unsigned sig;        // 0 = generic (run-time f_dim)
    int interp;
    int rl;              // lanes per ray
    bool wide;           // 64-bit element offsets
    int mode;            // MODE_PLAIN, MODE_TOUCH (footprint) or MODE_LABEL (visible span)
    FrameLaunch fn;
};

extern const ZcEntry *const k_zc_entries;
extern const int k_n_zc_entries;

// Mode of the staged march (raycast_staged.cu), after the march modes of
// raycast.cuh; its kernels have their own table.
constexpr int kModeStaged = 6;
extern const ZcEntry *const k_staged_entries;
extern const int k_n_staged_entries;

void launch_fill(const KParams &p, cudaStream_t st);
void launch_setup(const KParams &p, cudaStream_t st);
void launch_copy_rays(const KParams &p, RayRec *out, long long cap, int *count, cudaStream_t st);

}  // namespace isaac
