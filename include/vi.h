/*
 * vi.h -- C ABI of the GB300 (sm_103a) slice-based illuminated ray casting
 * library: D. Luo, "Interactive volume illumination of slice-based ray
 * casting", arXiv 2008.06134.
 *
 * The method has two passes (Section 3, Fig. 1):
 *   1. vi_build_attenuation: a sweep from the light's viewpoint that builds one
 *      illumination attenuation buffer per slice plane perpendicular to the
 *      light, each formed from the previous one by the transfer-function
 *      opacity (Section 3.2.1, Algorithm 1, Eq. 4, Eq. 8).
 *   2. vi_render: an eye-space ray march that, per sample, reconstructs the
 *      volume trilinearly, classifies it through an RGBA transfer function,
 *      reads the attenuation buffers for a shadow (Section 3.2.2, Eq. 9, Eq. 10),
 *      shell or cone scattering coefficient (Section 3.2.3, Eq. 11), weights the
 *      emission by it (Eq. 7) and composites front to back (Eq. 2, Eq. 3) with
 *      early ray termination.
 *
 * Conventions for every call:
 *   - Every call returns VI_OK (0) or a negative vi_status.  No C++ exception
 *     crosses this boundary.
 *   - A context is bound to one CUDA device and one CUDA stream.  All device
 *     work of a call is enqueued on that stream, in call order.  Calls on one
 *     context must not run concurrently from several host threads.
 *   - Geometry: the volume occupies the unit cube [0,1]^3; voxel (x, y, z) has
 *     its centre at ((x + 1/2)/nx, (y + 1/2)/ny, (z + 1/2)/nz).
 *   - An asynchronous device error is sticky: the next call, or vi_sync,
 *     returns VI_ECUDA and clears it.
 *   - Host input buffers are read by a copy enqueued on the stream.  A
 *     pageable host buffer may be reused when the call returns; a page-locked
 *     (pinned) one only after vi_sync.
 *   - The library owns the device copies of the volume, the transfer function
 *     and the attenuation stack.  The caller owns every buffer it passes.
 */
#ifndef VI_H
#define VI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vi_ctx vi_ctx; /* opaque, library-owned */

typedef enum {
    VI_OK = 0,
    VI_EINVAL = -1,   /* an argument is out of range, NULL where not allowed, or not finite */
    VI_ENOMEM = -2,   /* the memory budget or the device refused an allocation */
    VI_ESTATE = -3,   /* a required input is missing or the stack is stale */
    VI_ECUDA = -4,    /* a CUDA runtime error (launch or asynchronous fault) */
    VI_ETIMEOUT = -5  /* a bounded device-side wait gave up */
} vi_status;

enum { VI_U8 = 0, VI_U16 = 1 };                                  /* voxel types */
enum { VI_NONE = 0, VI_SHADOW = 1, VI_SHELL = 2, VI_CONE = 3 };  /* coefficient modes */
enum { VI_F32 = 0, VI_F16 = 1, VI_BF16 = 2, VI_UNORM16 = 3 };    /* stack storage */
enum { VI_TRANSMITTANCE = 0, VI_OPTICAL_DEPTH = 1 };             /* what the stack holds */
enum { VI_SLICE_NEAREST = 0, VI_SLICE_LINEAR = 1 };              /* slice filtering */
#define VI_DEPTH_MAX 64.0f  /* cap of a stored optical depth: exp(-64) < 2e-28 */
#define VI_MAX_SHELLS 4

/* Options of the attenuation sweep.  NULL means the defaults shown. */
typedef struct {
    int format;                /* VI_F32 (default), VI_F16, VI_BF16 or VI_UNORM16 storage;
                                  the transmittance product is always carried in FP32 */
    float cone_half_angle_deg; /* cone scattering half angle phi (Section 3.2.3), default 15 */
    float shell_radius_vox;    /* shell scattering radius r in voxels (Section 3.2.3), default 1 */
    int opacity_correction;    /* 0 (default): the TF opacity is applied per slice as is;
                                  1: alpha' = 1 - (1 - alpha)^(slice spacing in voxels) */
    float comp_n;              /* darkening compensation (Section 4): each stored slice is
                                  multiplied by (1 + alpha)^comp_n, clamped to 1; 0 = off */
    int quantity;              /* VI_TRANSMITTANCE (default): B_k = prod_{j<k} (1 - alpha_j),
                                  Eq. 4 in product form.  VI_OPTICAL_DEPTH: the extinction form
                                  of Eq. 5-6, B_k = sum_{j<k} -ln(1 - alpha_j) carried in FP32
                                  and capped at VI_DEPTH_MAX; a lookup's light factor is then
                                  exp(-B) of the interpolated depth, and comp_n subtracts
                                  comp_n ln(1 + alpha) (floored at 0).  Not with VI_UNORM16. */
    int shell_count;           /* VI_SHELL: shells at radii r, 2r, ... (Section 3.2.3: the
                                  number and size of the shells can vary), six points each,
                                  equal weights; 0 or 1 (default) = one shell, at most
                                  VI_MAX_SHELLS */
} vi_build_opts;

/* A pinhole (perspective) or orthographic camera in unit-cube coordinates.
   Row 0 of the image is its top; the camera's right vector is
   normalize(forward x up). */
typedef struct {
    int perspective;         /* 1 perspective, 0 orthographic */
    float eye[3];            /* eye (perspective) or centre of the image plane (orthographic) */
    float target[3];         /* a point the view direction passes through */
    float up[3];             /* must not be parallel to target - eye */
    float fovy_deg;          /* perspective: vertical field of view, (0, 180) */
    float ortho_half_height; /* orthographic: half height of the image plane, > 0 */
} vi_camera;

/* Options of the eye pass.  NULL means the defaults shown. */
typedef struct {
    float ert;              /* stop a ray once accumulated opacity > ert; default 2 (off) */
    float bg[4];            /* background RGBA behind the remaining transparency, default 0 */
    float ambient;          /* light factor = ambient + (1 - ambient) * coefficient, default 0 */
    int opacity_correction; /* 1: alpha' = 1 - (1 - alpha)^step_vox; default 0 */
    int32_t* sample_counts; /* optional device buffer of W*H int32: samples composited per
                               pixel (row-major); NULL = not written */
    int32_t* lit_counts;    /* optional device buffer of W*H int32: samples with opacity > 0,
                               the ones that read the stack; NULL = not written */
    int slice_filter;       /* VI_SLICE_NEAREST (default): the slice of Eq. 9 rounded to the
                               nearest plane; VI_SLICE_LINEAR: linear in lambda between slices
                               k0 = clamp(floor(lambda), 0, n - 1) and min(k0 + 1, n - 1) */
} vi_render_opts;

/* Create a context on CUDA device `device` using `cuda_stream` (a cudaStream_t;
   NULL = the legacy default stream).  *out receives the context. */
int vi_create(vi_ctx** out, int device, void* cuda_stream);

/* Free every device buffer of the context (after waiting for its stream). */
int vi_destroy(vi_ctx* ctx);

/* Cap on the device bytes this context may hold (volume + TF + stack + scratch);
   0 = no cap (default).  An allocation above the cap fails with VI_ENOMEM and
   leaves the previous state intact. */
int vi_set_memory_budget(vi_ctx* ctx, size_t bytes);

/* The volume (Section 3: a 3D array of voxels): nx*ny*nz voxels of `dtype`
   (VI_U8 / VI_U16), layout data[z][y][x] with x fastest, each dimension in
   [1, 65536].  data_on_device: 1 if `data` is a device pointer of this context's
   device, 0 for host memory.  Marks the stack stale. */
int vi_load_volume(vi_ctx* ctx, const void* data, int dtype, int nx, int ny, int nz,
                   int data_on_device);

/* RGBA transfer function (Section 2: the classification of data values): M
   entries of straight (not premultiplied) RGBA float32 in host memory, M in
   [2, 8192], evenly spaced over [vmin, vmax] (vmax > vmin), interpolated
   linearly and clamped at both ends.  Marks the stack stale. */
int vi_set_transfer_function(vi_ctx* ctx, const float* rgba, int M, float vmin, float vmax);

/* Directional light (Section 3.2.1): dir is the direction the light travels
   (any finite non-zero length); color multiplies the emission (Eq. 7; NULL =
   white).  Marks the stack stale. */
int vi_set_light(vi_ctx* ctx, const float dir[3], const float color[3]);

/* Point light (not in the paper's experiments, which use a directional light;
   Fig. 7 speaks of a light position): light travels along rays from
   `position` (cube coordinates; at least 1 from the cube centre (1/2, 1/2,
   1/2), outside the cube's circumscribed sphere, else VI_EINVAL).  The
   slices are planes perpendicular to the axis from the light to the centre;
   each stack column is one ray from the light through a perspective texel grid
   that holds the cube; a lookup divides by the depth along the axis.  Shell
   points are S +- q r e_a; cone rings are centred n dL from S towards the
   light, turned about the light direction at S.  color as in vi_set_light.
   Replaces any directional light.  Marks the stack stale. */
int vi_set_point_light(vi_ctx* ctx, const float position[3], const float color[3]);

/* Algorithm 1: build n_slices attenuation buffers of slice_res x slice_res
   texels, slice 0 nearest the light at min of Eq. 8, spacing (max - min)/n.
   Buffer k holds the light arriving at plane k: B_0 = 1,
   B_k = prod_{j<k} (1 - alpha_j).  mode (VI_NONE, VI_SHADOW, VI_SHELL,
   VI_CONE) selects the coefficient vi_render reads; VI_NONE builds nothing.
   Needs a volume, a TF and a light (VI_ESTATE otherwise).  Asynchronous.
   n_slices and slice_res must be >= 1 and n_slices * slice_res^2 <= 2^34, and
   the stack must fit one 2D texture of the device: n_slices cells of
   slice_res^2 texels, C = 2^c cells to a row (slice_res C within the texture
   width, 131072 texels on sm_103a), ceil(n_slices / C) slice_res rows within
   its height (65000); VI_EINVAL otherwise.  Every configuration up to 1024
   slices of 2048^2 fits.  Stacks of 2^29 texel-slices and more are swept with
   a warp's columns in lockstep, smaller ones column by column; both give the
   same values bit for bit.  The environment variable VI_SWEEP_LOCKSTEP_MIN, if
   it holds a number, replaces that threshold (for tests). */
int vi_build_attenuation(vi_ctx* ctx, int n_slices, int slice_res, int mode,
                         const vi_build_opts* opts);

/* Eye pass (Section 3.2.2, 3.2.3, 4): one ray per pixel centre, samples every
   step_vox voxels from where the ray enters the unit cube (a voxel is
   1/max(nx,ny,nz); step_vox in [1e-3, 1e3] and sqrt(3) max(nx,ny,nz) / step_vox
   <= 2^24), front-to-back compositing with the mode's coefficient.
   out_rgba: W*H*4 float32, row-major RGBA, caller-owned, where out_on_device
   says: VI_OUT_DEVICE (1): a device pointer, written asynchronously on the
   context's stream; VI_OUT_HOST (0): host memory, filled when the call
   returns; VI_OUT_HOST_ASYNC (2): host memory, the frame's copy enqueued on
   the context's stream and complete at the next vi_sync (page-locked memory
   lets the copy overlap other work; the buffer must stay valid until then).
   W or H == 0 renders nothing.  VI_ESTATE if the volume or TF is missing or
   the stack (modes other than VI_NONE) is stale. */
enum { VI_OUT_HOST = 0, VI_OUT_DEVICE = 1, VI_OUT_HOST_ASYNC = 2 };
int vi_render(vi_ctx* ctx, const vi_camera* camera, int W, int H, float step_vox,
              float* out_rgba, int out_on_device, const vi_render_opts* opts);

/* Wait for the context's stream; returns (and clears) a sticky error. */
int vi_sync(vi_ctx* ctx);

/* Static text for a vi_status code. */
const char* vi_error_string(int status);

/* ---- Inspection (tests and tools) ---------------------------------------- */

/* Shape and storage of the current stack; any pointer may be NULL. */
int vi_attenuation_info(vi_ctx* ctx, int* n_slices, int* slice_res, int* format,
                        size_t* bytes);

/* Copy the stack as stored ([n][R][R] of the storage format) into `out`
   (out_bytes >= the stack's size); out_on_device as for vi_render (a host
   buffer is filled before the call returns in either host mode).  Waits for
   the copy. */
int vi_get_attenuation(vi_ctx* ctx, void* out, size_t out_bytes, int out_on_device);

/* The empty-space skipping grid of the current volume and TF.  Skipping is
   exact: a sample whose trilinear footprint (Section 3, the 3D texture
   lookup) starts in a brick or cell whose voxels, with the one-voxel apron on
   its high sides, cannot reach a TF entry with alpha > 0 (Section 3.1.1,
   classification) has alpha 0 and contributes nothing to Eq. 3 or Eq. 4.
   dims (may be NULL) receives { nbx, nby, nbz, cnx, cny, cnz }: bricks of
   16^3 voxels and cells of 8^3 voxels per axis (bricks cover the volume,
   rounded up; cells are 2 x 2 x 2 to a brick).  brick_flags (host, nbx nby
   nbz bytes, x fastest) receives 1 for a brick that may yield alpha > 0, else
   0.  cell_skip (host, cnx cny cnz bytes, x fastest) receives 0 for a cell
   that may yield alpha > 0, else the L-infinity distance in cells to the
   nearest such cell within the grid, capped at 32.  A flag is set whenever
   the FP64 TF coordinates of the brick's or cell's value range reach an
   entry with alpha > 0, and only when they come within one entry of one.
   Either buffer may be NULL; a buffer shorter than its grid (brick_bytes,
   cell_bytes) is VI_EINVAL.  VI_ESTATE without a volume and a TF.  Waits for
   the copies. */
int vi_get_skip_grid(vi_ctx* ctx, int* dims, uint8_t* brick_flags, size_t brick_bytes,
                     uint8_t* cell_skip, size_t cell_bytes);

/* Words per record written by vi_trace_pixel. */
#define VI_TRACE_WORDS 40

/* The integer decisions of one pixel's ray, sample by sample, for exact
   comparison with an independent implementation: per sample VI_TRACE_WORDS
   int32 = { i, bits(t_i), bits(lambda), bits(tu), bits(tv), voxel cell x,y,z,
   own lookup cell (k, iu, iv), 8 neighbour cells (k, iu, iv), neighbour count,
   unused }, unused words 0x7fffffff.  rec is host memory of max_rec records;
   recording stops after max_rec samples; *n_rec receives the count.
   Synchronous. */
int vi_trace_pixel(vi_ctx* ctx, const vi_camera* camera, int W, int H, float step_vox,
                   const vi_render_opts* opts, int x, int y, int32_t* rec, int max_rec,
                   int* n_rec);

/* Number of kernels this context has launched so far. */
int vi_launch_count(vi_ctx* ctx, uint64_t* count);

/* Roofline denominators measured on `device` by probe kernels (not part of
   the method): *fp32_tflops, the FP32 FMA rate of eight independent FMA
   chains per thread on every SM; *l2_read_gbs, the read bandwidth of a buffer
   of a quarter of L2 read repeatedly through L2 by every SM.  Each is the
   best of three timed launches (CUDA events) after one warm-up.  Allocates
   and frees its buffers; synchronous. */
int vi_measure_peaks(int device, double* fp32_tflops, double* l2_read_gbs);

/* ---- Batched frames: one persistent launch over several contexts ---------- */

/* Most frames one vi_render_batch call takes. */
#define VI_BATCH_MAX_FRAMES 64

/* One frame of a batch.  The paper renders one frame at a time (Section 4);
   batching is a serving feature.  ctx supplies the volume, TF, light and
   stack (built with VI_F32 or VI_F16 storage, transmittance, one shell, a
   directional light; the options' slice_filter must be VI_SLICE_NEAREST).
   camera, width, height, step_vox and opts as for vi_render; out_rgba is a
   device pointer of width*height*4 float32 (caller-owned).  status is
   written by the call: VI_OK, or VI_ETIMEOUT if the frame's stack was not
   published in time (its output is then incomplete). */
typedef struct {
    vi_ctx* ctx;
    vi_camera camera;
    int width, height;
    float step_vox;
    float* out_rgba;
    vi_render_opts opts;
    int status;
} vi_batch_frame;

/* Publishes the context's stack to batched frames: enqueues on the context's
   stream, after its work so far (normally its vi_build_attenuation), a device
   write of a new epoch to the context's ready word, released to the whole
   device, and records an event after it.  A batch frame of this context
   renders the state published last before the vi_render_batch call. */
int vi_post_ready(vi_ctx* ctx);

/* Renders `count` frames (1..VI_BATCH_MAX_FRAMES) in persistent launches on
   `cuda_stream` (a cudaStream_t of the frames' device; NULL = the legacy
   default stream), for callers that serve many small frames at once.  The
   frames are grouped by kind (voxel type, storage format, mode); each group
   is one launch whose frames are consecutive ranges of a queue of 4 x 8 pixel
   tiles in device memory, and whose warps take (frame, tile) items from it in
   order, so the warps that finish one frame go on with the next.
   The batch is ordered on the stream after each frame's last publication
   (vi_post_ready's event): a kernel that spun on work of another stream could
   hold that work up, since streams share the GPU's hardware work queues.
   Before a frame's tiles a warp still checks, on the device, that the
   frame's context has published (a context that never published waits for
   its first epoch): it waits at most wait_ms, measured on the GPU's
   nanosecond timer and bounded by the SM clock as well.  A wait that runs out
   sets the frame's status to VI_ETIMEOUT and the frame's remaining tiles are
   skipped; the kernel always returns.  Each published frame equals the one vi_render gives from the
   same context.  Synchronous: returns when the launch has finished, with every
   status filled in; VI_OK if all frames rendered, VI_ETIMEOUT if any wait ran
   out, VI_EINVAL for a frame outside the restrictions above, contexts of
   different devices or wait_ms outside [0, 1e7], VI_ESTATE as vi_render for a
   context without its inputs.  The stream must not be captured. */
int vi_render_batch(vi_batch_frame* frames, int count, void* cuda_stream, double wait_ms);

/* ---- Rendering without allocation ----------------------------------------- */

/* Largest frame vi_render_host_noalloc takes: 512 x 512 pixels. */
#define VI_NOALLOC_MAX_PIXELS 262144

/* vi_render for callers that cannot allocate device memory -- a plug-in whose
   host application owns the GPU's memory, a process under a hard device-memory
   cap, a real-time loop where an allocation's latency is not acceptable.  The
   paper has no counterpart; it is a deployment variant of the eye pass.

   It renders with the context's resident volume, TF and stack exactly as
   vi_render does (same kernel, same result) into the caller's host buffer
   out_rgba (W*H*4 float32, row-major RGBA), and allocates nothing: no
   cudaMalloc, no cudaFree, no library-owned growth.  The march's work counter
   and the frame's staging live in one fixed device array inside the library
   (256 B + VI_NOALLOC_MAX_PIXELS * 16 B, about 4 MiB), which every GPU that
   loads the library holds until the process exits.
     - W * H above VI_NOALLOC_MAX_PIXELS returns VI_EINVAL (nothing runs).
     - The first call on a device (and the first after a cudaDeviceReset of
       it) looks up that array's device address in the current CUDA context;
       make it before any stream capture.
     - Every call on every context of a device shares the array: the counter
       is cleared on the stream at each call, the staged frame is overwritten
       (the array keeps the last call's contents), and calls whose GPU work
       overlaps -- two streams, two contexts, two threads -- race on it and
       must be ordered by the caller.
   Synchronous: returns when the frame is in out_rgba.  Other arguments,
   states and errors as vi_render. */
int vi_render_host_noalloc(vi_ctx* ctx, const vi_camera* camera, int W, int H, float step_vox,
                           float* out_rgba, const vi_render_opts* opts);

/* Bounds-check record of a checked build of this library (libvi_checked.so,
   compiled with VI_DEBUG_BOUNDS=1).  In that build every kernel tests each
   voxel, brick, TF, stack, output and grid index before the access; a bad
   index is counted and the access skipped, so a kernel neither traps nor
   faults.  The call waits for the device, stores the number of violations
   since the last call for that device, the site of a first one (1 volume
   footprint, 2 brick flag, 3 TF alpha, 4 TF colour, 5 stack slice or row of a
   lookup, 6 stack store, 7 output pixel, 8 raw voxel, 9 grid build; 0 if
   none) and its index, and clears the record.  The record covers every
   context of the process on the device.  VI_ESTATE from a library built
   without the checks (the outputs are set to 0); VI_EINVAL for a bad device
   or a null pointer. */
int vi_debug_bounds(int device, uint64_t* violations, int* first_site, int64_t* first_index);

/* ---- Serving: continuous batching of render requests ---------------------- */

/* A render server on one device.  It is not in the paper (which renders one
   frame at a time): requests arrive at any time and are admitted in arrival
   order into `slots` concurrent render slots (each a context on its own CUDA
   stream) whenever a slot is free and the device memory they need fits the
   budget, so frames of different requests run on the GPU together.  Volumes
   are registered once and kept resident (pair bricks and brick ranges) up to
   max_resident_volumes (0 = no count limit) and memory_budget bytes in total
   with the slots' buffers (0 = no byte limit); when room is needed an idle
   volume is evicted (vi_server_set_eviction chooses which) and reloaded from
   the caller's host copy when next requested.  A request that can never fit fails with
   VI_ENOMEM; others wait.  All host-side waits are bounded.
   Each slot keeps the attenuation stack of its last request.  A request with
   the same volume, TF (entries and range), light, stack shape, mode and build
   options as a free slot's last one is placed on that slot and renders from
   its stack without a new sweep (a new view of an unchanged scene); other
   requests go to a free slot without a stack, else to the free slot whose
   stack was used longest ago. */
typedef struct vi_server vi_server;

enum { VI_REQ_QUEUED = 0, VI_REQ_RUNNING = 1, VI_REQ_DONE = 2, VI_REQ_FAILED = 3,
       VI_REQ_CANCELLED = 4 };

/* One frame: the same inputs as vi_set_transfer_function, vi_set_light,
   vi_build_attenuation and vi_render on a registered volume.  The TF is
   copied at submission; out_rgba (W*H*4 float32) must stay valid until the
   request finishes (device memory, or host memory -- page-locked to overlap). */
typedef struct {
    int volume_id;
    const float* tf_rgba;
    int tf_entries;
    float tf_vmin, tf_vmax;
    float light_dir[3];
    float light_color[3];
    int n_slices, slice_res, mode;
    vi_build_opts build;
    vi_camera camera;
    int width, height;
    float step_vox;
    vi_render_opts render;
    float* out_rgba;
    int out_on_device;  /* VI_OUT_DEVICE or VI_OUT_HOST (VI_EINVAL otherwise) */
} vi_request;

typedef struct {
    uint64_t submitted, completed, failed, cancelled;
    uint64_t volume_loads, volume_evictions;
    int queued, running, resident_volumes;
    size_t bytes_in_use, peak_bytes;
    uint64_t stack_reuses;  /* requests that rendered from a slot's kept stack */
    uint64_t graph_launches;        /* requests whose device work ran as one CUDA graph */
    uint64_t graph_instantiations;  /* executable graphs created (the rest were updated) */
    uint64_t batches;               /* batches of marches enqueued (vi_server_set_batching) */
    uint64_t batched_frames;        /* frames marched in those batches */
    uint64_t volume_load_bytes;     /* raw voxel bytes copied in by volume_loads */
} vi_server_stats;

/* Create / destroy a server (destroy cancels queued requests, lets running
   ones finish, and frees everything). */
int vi_server_create(vi_server** out, int device, int slots, size_t memory_budget,
                     int max_resident_volumes);
int vi_server_destroy(vi_server* server);

/* Register a volume (as vi_load_volume: data[z][y][x], VI_U8 / VI_U16).  The
   host data must stay valid and unchanged while the server lives: it is
   (re)loaded from it on demand, and kept stacks built from it are reused.
   *volume_id receives its id. */
int vi_server_add_volume(vi_server* server, const void* host_data, int dtype, int nx, int ny,
                         int nz, int* volume_id);

/* Queue a request; *ticket names it.  Malformed requests return VI_EINVAL
   and are not queued. */
int vi_server_submit(vi_server* server, const vi_request* request, uint64_t* ticket);

/* Wait up to timeout_ms for the request to finish (VI_ETIMEOUT otherwise);
   *status receives a VI_REQ_* state and *result its vi_status. */
int vi_server_wait(vi_server* server, uint64_t ticket, double timeout_ms, int* status,
                   int* result);

/* Cancel a request that is still queued (VI_ESTATE once it has started). */
int vi_server_cancel(vi_server* server, uint64_t ticket);

/* Milliseconds since server creation at which the request was submitted,
   started on a slot, and finished (0 until then). */
int vi_server_timing(vi_server* server, uint64_t ticket, double* submit_ms, double* start_ms,
                     double* end_ms);

/* Forget a finished request (VI_ESTATE if it has not finished). */
int vi_server_release(vi_server* server, uint64_t ticket);

int vi_server_get_stats(vi_server* server, vi_server_stats* stats);

/* Launch each request's device work as one CUDA graph (enabled != 0) or as
   separate launches (0, the default); applies to requests started after the
   call.  With graphs, the work a request queues after its uploads (the TF
   copy and the brick flags stay ordinary stream operations) -- the sweep,
   the march, the copy of a host output and the completion callback -- is
   captured from the slot's stream and launched as one graph.  Each slot
   keeps one executable graph per shape of that work (with or without a
   sweep, device or host output) and updates its parameters in place for the
   next request of the same shape, so a graph is instantiated only the first
   time a shape appears on a slot.  The frames are bit-identical to those of
   separate launches (the same kernels with the same parameters).  A request
   whose host output is pageable memory (not capturable) runs with separate
   launches.  Returns VI_EINVAL for a null server. */
int vi_server_set_graphs(vi_server* server, int enabled);

/* Batched marches (1) or one march per request on its slot's stream (0, the
   default); applies to requests admitted after the call.  With batching, the
   requests admitted in one pass of the scheduler run their uploads and
   sweeps on their slots' streams as before and publish their stacks
   (vi_post_ready); their marches are then enqueued together as one batch of
   persistent launches on the server's batch stream (vi_render_batch's
   kernels), each frame's tiles waiting on the device for its slot's stack for
   at most wait_ms (VI_ETIMEOUT fails the request).  Requests outside
   vi_render_batch's restrictions (BF16 / UNORM16 stacks, optical depth,
   several shells, linear slices) keep their own march.  Batching takes
   precedence over graphs for the requests it batches.  Returns VI_EINVAL for
   a null server or wait_ms outside [0, 1e7], VI_ECUDA if the batch stream
   or the status words cannot be made. */
int vi_server_set_batching(vi_server* server, int enabled, double wait_ms);

/* Which idle volume the server evicts when a request needs room (a volume
   count or byte limit).  Serving is not in the paper; this is a residency
   policy of the server.
   VI_EVICT_COST (the default): GreedyDual with the reload cost as the cost.
   The server keeps an aging clock; each use of a volume sets its credit to
   the clock plus its reload cost (its raw voxel bytes in MiB: the
   host-to-device copy and the pair-brick build grow with them); the idle
   volume with the lowest credit is evicted (the least recently used among
   equal credits) and the clock rises to its credit.  A volume that is costly
   to reload therefore stays resident over cheap ones until it has gone
   unused for about its reload cost's worth of the other volumes' evictions.
   VI_EVICT_LRU: the least recently used idle volume.
   Frames do not depend on the policy; only which requests pay a reload does.
   Applies to evictions after the call.  Returns VI_EINVAL for a null server
   or another policy. */
enum { VI_EVICT_LRU = 0, VI_EVICT_COST = 1 };
int vi_server_set_eviction(vi_server* server, int policy);

#ifdef __cplusplus
}
#endif

#endif /* VI_H */
