// common.h -- host helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "isaac_b300.h"
#include "kernel_table.h"

namespace isaac {

struct KParams;
struct KSource;
struct KChain;

// Record an error message for isaac_last_error() and return `code`.
int fail(int code, const char *fmt, ...);
void clear_error();
const char *last_error();
// Turn the last CUDA error (if any) into ISAAC_ECUDA.
int check_cuda(const char *what);

int prepare_frame(const isaac_camera *cam, const isaac_plane *clip, int32_t n_clip,
                  const isaac_render_opts *opt, KParams &p);
// reach: guard layers the kernel may read (1; 2 for iso-surface gradients),
// capped by the source's own guard width.
int prepare_source(const isaac_source &src, int s, const int64_t n[3], int interp, float weight,
                   int elem, KSource &ks, unsigned *nib, bool *wide, int reach = 1);
int compile_chain(const isaac_chain &in, int fdim, int s, KChain &out);
int prepare_fb(const isaac_framebuffer *fb, KParams &p);
// Multiprocessor count of the current device (cached per device; 148 if the
// query fails).
int sm_count();

// Calls the calling thread's update hook (isaac_set_update_hook), if any, for
// every source in order (with its active bit), before an entry point reads the
// descriptors.
void update_sources(int32_t n_sources, uint32_t active_mask);

// Validate the sources of isaac_render and fill their part of KParams.
int prepare_sources(const isaac_source *sources, const isaac_chain *chains, int32_t n_sources,
                    const float *luts, const float *weights, const isaac_render_opts *opts,
                    KParams &p, int *nact_out, unsigned *sig_out, bool *wide_out, int reach = 1);
// Zero-copy frame kernel for a source signature and march mode (nullptr if none).
FrameLaunch find_zc(int nact, unsigned sig, int interp, bool wide, int mode, int rl,
                    int *rl_used);

// Work inserted between ray setup and march (the interval proposal).
struct FrameHook {
    int (*fn)(const KParams &p, const void *arg, cudaStream_t st);
    const void *arg;
};
// Validate a proposal and describe it as a hook (proposal may be null: no hook).
int proposal_hook(const isaac_proposal *proposal, const isaac_render_opts *opts, FrameHook *hook);
// Lanes per ray for a rectangle of `rect_pixels` (hint 0 = automatic) when a
// sample gathers `corner_bytes` per trilinear corner (0: unknown).
int choose_lanes(long long rect_pixels, int hint, int corner_bytes = 0);
// Bytes a trilinear corner gathers over the first `nact` sources of p (4 per
// component), the corner_bytes of choose_lanes for a zero-copy frame.
int zc_corner_bytes(const KParams &p, int nact);
// Whether a zero-copy plain frame may use the staged march (opts asks for it,
// trilinear, 32-bit offsets, no footprint, every source with the same readable
// range); the caller still needs a compiled staged kernel for the signature.
bool staging_allowed(const KParams &p, int nact, const isaac_render_opts *opts, bool wide);
// Most march chunks a warp takes per atomic (KParams::grab, guided
// self-scheduling): 16; the environment variable ISAAC_MARCH_GRAB (1..64)
// overrides it, 1 = one chunk per atomic.  Scheduling only: the image does not
// depend on it.
int march_grab();
// Bind the calling stream's workspace (grown as needed) to p.ctr / p.rays /
// p.longs; `extra` more bytes after them, returned in *extra_ptr.
int bind_workspace(KParams &p, cudaStream_t st, size_t extra = 0, void **extra_ptr = nullptr);
// Empty-space bits of the macro cells (32 per word) from a value-range grid.
int launch_empty_flags(const KParams &p, int nact, const float *ranges, int slots, long long cells,
                       unsigned *flags, cudaStream_t st);
// Background + ray setup + optional hook + march kernel `fn` (null: background
// only).  fn_long: the long-ray march of the same sources; with a hook and
// fn_long the hook may fill the long-ray list, which fn_long marches before fn.
int launch_frame_with(KParams &p, FrameLaunch fn, int rl, cudaStream_t st, const FrameHook *hook,
                      FrameLaunch fn_long = nullptr);

}  // namespace isaac
