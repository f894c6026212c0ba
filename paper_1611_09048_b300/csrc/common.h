// common.h -- host helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "isaac_b300.h"

namespace isaac {

struct KParams;
struct KSource;
struct KChain;

using FrameLaunch = void (*)(const KParams &, dim3, cudaStream_t);
// Fill the background outside the screen rectangle, then launch `fn` over
// the rectangle's 16x8 tiles (skipped when fn is null or the rectangle empty).
int launch_with(const KParams &p, FrameLaunch fn, cudaStream_t st);

// Record an error message for isaac_last_error() and return `code`.
int fail(int code, const char *fmt, ...);
void clear_error();
// Turn the last CUDA error (if any) into ISAAC_ECUDA.
int check_cuda(const char *what);

int prepare_frame(const isaac_camera *cam, const isaac_plane *clip, int32_t n_clip,
                  const isaac_render_opts *opt, KParams &p);
int prepare_source(const isaac_source &src, int s, const int64_t n[3], int interp, float weight,
                   int elem, KSource &ks, unsigned *nib, bool *wide);
int compile_chain(const isaac_chain &in, int fdim, int s, KChain &out);
int prepare_fb(const isaac_framebuffer *fb, KParams &p);

}  // namespace isaac
