// vi_context.h -- the context behind vi_ctx and the pieces of it the server
// shares; internal to the library.
#pragma once

#include <cstddef>
#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "../../include/vi.h"
#include "vi_internal.h"

// A loaded volume: the voxels as given ([nz][ny][nx]), their pair bricks and
// the per-brick value ranges.  A context owns one (vi_load_volume); a
// server owns several and lends them to its render slots.
struct VolumeRes {
    void* raw = nullptr;
    size_t raw_cap = 0;
    void* pairs = nullptr;  // pair bricks (vi_internal.h, VolumeView)
    size_t pairs_cap = 0;
    uint32_t* brange = nullptr;
    size_t brange_cap = 0;
    int vtype = -1, nx = 0, ny = 0, nz = 0;
    int nbx = 0, nby = 0, nbz = 0;
    cudaMemPool_t pool = nullptr;  // stream-ordered pool its buffers come from (null: cudaMalloc)
};

struct vi_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sticky = VI_OK;
    uint64_t launches = 0;

    size_t budget = 0;  // 0 = unlimited
    size_t used = 0;
    cudaMemPool_t pool = nullptr;  // stream-ordered pool for its buffers (null: cudaMalloc)

    VolumeRes own;          // the volume vi_load_volume loads
    VolumeRes* vr = &own;   // the volume in use: own, or one a server shares

    float4* tf = nullptr;
    size_t tf_cap = 0;
    int M = 0;
    float vmin = 0.0f, vmax = 1.0f;

    // Brick occupancy (empty-space skipping): prefix count of TF entries with
    // alpha > 0 and per-brick flags (the value ranges belong to the volume).
    int* tfcnt = nullptr;
    size_t tfcnt_cap = 0;
    uint8_t* bflags = nullptr;  // brick flags, skip distances, scratch (nbricks bytes each)
    size_t bflags_cap = 0;
    bool flags_ok = false;  // bflags match the current volume and TF

    bool has_light = false;
    bool light_point = false;             // point light at pos, else directional dir
    float pos[3] = {0.5f, 0.5f, 2.0f};
    float dir[3] = {0.0f, 0.0f, 1.0f};
    float color[3] = {1.0f, 1.0f, 1.0f};

    void* stack_mem = nullptr;   // allocation; the stack starts at the next 512-byte boundary
    size_t stack_cap = 0;
    void* stack = nullptr;
    size_t stack_bytes = 0;      // dense size n R^2 element bytes, as vi_get_attenuation returns
    size_t row_pitch = 0;        // bytes per stack row (the cell layout of vi::StackView)
    vi::StackView sview{};       // texture view of the stack
    int ntex = 0;                // 1 while sview.tex exists
    int stack_valid_shape_n = 0; // slice count, resolution and format the texture views
    int stack_valid_shape_R = 0; // were made for
    int stack_valid_shape_fmt = -1;
    int mode = -1;          // mode of the last build; -1 = none yet
    bool stack_valid = false;
    vi_build_opts bopts{};
    vi::LightFrame lt{};
    bool lt_valid = false;

    float4* out = nullptr;  // staging for host-memory output
    size_t out_cap = 0;
    int32_t* trace = nullptr;
    size_t trace_cap = 0;
    unsigned* counter = nullptr;  // tile counter of the persistent march kernel
    size_t counter_cap = 0;
    int march_block = 0;          // march block size cap (0: one 1024-thread block per SM)
    unsigned* ready = nullptr;    // ready word batched frames wait on (vi_post_ready)
    cudaEvent_t ready_event = nullptr;  // recorded after the ready word was zeroed
    cudaEvent_t posted_event = nullptr; // recorded after the last vi_post_ready
    unsigned post_epoch = 0;      // the last epoch vi_post_ready enqueued
    // Set while the context's stream is being captured into a graph: no buffer
    // may grow then (an allocation would become part of the graph), so a call
    // that needs more memory fails instead (ctx_reserve sizes them first).
    bool capturing = false;
};

namespace vi_detail {
// An NVTX range over one API call (header-only NVTX: without a profiler
// attached, a push or pop is a check of a function pointer).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device allocation under a byte budget (0 = none) with a usage counter; keeps
// the old buffer on failure.  Without a pool: cudaMalloc, and the old buffer is
// freed after `s` drains.  With a pool: allocation and free are ordered on `s`
// (no device-wide synchronisation; freed blocks are reused by the pool).
int ensure_mem(size_t* used, size_t budget, void** p, size_t* cap, size_t bytes, cudaStream_t s,
               cudaMemPool_t pool);
// Frees a buffer: cudaFree, or a free ordered on `s` when it came from `pool`.
void release_mem(size_t* used, void** p, size_t* cap, cudaStream_t s, cudaMemPool_t pool);

// Loads nx*ny*nz voxels into v (pair bricks and brick ranges built on stream s).
int volume_load(VolumeRes* v, size_t* used, size_t budget, const void* data, int dtype, int nx,
                int ny, int nz, int data_on_device, cudaStream_t s, uint64_t* launches);
// Frees the volume's buffers (ordered on `s` when they came from a pool).
void volume_release(VolumeRes* v, size_t* used, cudaStream_t s);
size_t volume_bytes(int dtype, int nx, int ny, int nz);

// Layout of an n-slice R x R stack with esize-byte texels (vi::StackView):
// 2^cells_log2 cells to a row of cells (the smallest power of two at least
// sqrt(n), widened until the rows fit the texture height, within its width),
// `rows` texel rows of `pitch` bytes, and the allocation (`bytes`, with room
// to align the start to 512 bytes).  VI_EINVAL when the stack does not fit
// one 2D texture of `device`; VI_ECUDA when its limits cannot be read.
struct StackLayout {
    int cells_log2;
    size_t rows, pitch, bytes;
};
int stack_layout(int device, int n, int R, size_t esize, StackLayout* out);

// Points the context at a volume it does not own and refreshes the brick
// flags.  The stack goes stale unless keep_stack is set and the context was
// already on v (the caller vouches that v holds the same voxels).
int ctx_bind_volume(vi_ctx* c, VolumeRes* v, bool keep_stack);

// Frees the stack and the output staging of an idle context (its next build
// allocates them again).
void ctx_trim(vi_ctx* c);

// vi_render without waiting: host output is copied asynchronously (a pinned
// buffer overlaps; a pageable one makes the copy synchronous).
int ctx_render_async(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox, float* out,
                     int out_on_device, const vi_render_opts* opts);
// The batched frame of context c (vi_render's checks and parameters; a host
// output is staged in the context's buffer), or a vi_status.  b->index is
// left to the caller.
int ctx_batch_frame(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox, float* out,
                    int out_on_device, const vi_render_opts* opts, vi::BatchFrame* b);
// Enqueues a batch on stream s (after every frame's ready word was zeroed):
// its persistent launches, then a copy of frame f's status word to
// status_dst[f] (host memory); returns without waiting.
cudaError_t enqueue_batch(vi_ctx* const* ctxs, const vi::BatchFrame* frames, int count,
                          unsigned long long wait_ns, int* const* status_dst, cudaStream_t s);

// Grows, ahead of a capture, every buffer a build of an n x R x R stack of
// format fmt (build_stack != 0) and a W x H render (host output staging when
// out_on_device is 0) will use, so that the calls inside the capture allocate
// nothing.  Also makes the stack's texture views.
int ctx_reserve(vi_ctx* c, int build_stack, int n, int R, int fmt, int W, int H,
                int out_on_device);

}  // namespace vi_detail
