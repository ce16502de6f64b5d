// vi_internal.h -- parameter blocks shared by the host runtime and the kernels.
//
// Every float here that feeds an integer decision (slice index, texel cell,
// voxel cell, sample count, inside test) is computed on the host in binary32
// with a fixed operation order and no contraction (the "index path"); the
// kernels continue that path with __fmaf_rn / __fadd_rn / __fmul_rn /
// __fdiv_rn / __fsqrt_rn so no compiler contraction or reassociation changes
// a bit.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace vi {

// Light set-up: Eq. 8 (min/max over the cube's vertices), the slice spacing and
// the Eq. 9 ratio, and the light-space frame of Eq. 10 (orthographic light
// view: basis U, V with V = L x U, a square of half extent h about the centre).
// Directional light: L the direction light travels, slices at L.X = min +
// k dL, an orthographic texel grid of half extent h about the centre.
// Point light (point = 1): light travels along rays from P; L is the axis from
// P to the centre, slices are planes at depths (X - P).L = min + k dL, Lc = 0,
// and the texel grid is perspective: texel (i, j) is the ray from P along
// L + u U + v V, with u, v in [-h, h] (h the tangent of the half angle of the
// cone from P holding the cube's circumscribed sphere).
struct LightFrame {
    float L[3];
    float min, max;
    float dL;     // (max - min) / n
    float kappa;  // n / (max - min)
    float Lc;     // L . (1/2, 1/2, 1/2); 0 for a point light
    float U[3], V[3];
    float h;      // sqrt(3)/2 as binary32; point light: tangent half extent
    float sigma;  // R / (2 h): texels per world unit (per unit tangent)
    float rho0;   // (R - 1) / 2
    int n, R;
    int point;    // 1: point light at P
    float P[3];
};

// The volume as pair bricks.  The volume is cut into bricks of B^3 voxels, B =
// 2^kBrickShift (16), stored one after the other in brick order ([bz][by][bx]).
// Brick b holds the voxels its trilinear footprints can touch -- the brick and
// a one-voxel apron on its high sides, (B + 1)^3 voxels with indices clamped
// to the volume -- as x-pairs: for x in [0, B), y and z in [0, B], the pair
// v(x, y, z) | v(x + 1, y, z) << (8 * voxel bytes), [z][y][x], B (B + 1)^2
// pairs from element b B (B + 1)^2.  A footprint is four aligned pair loads
// (rows y and y + 1 of planes z and z + 1), which together are the eight
// voxels in the order c000 c001 c010 c011 c100 c101 c110 c111 (c{z}{y}{x}).
// The layout takes 2 (B + 1)^2 / B^2 = 2.26 times the raw voxels' bytes for
// whole bricks (the footprint octets this replaced took 8 times).
// Checked builds (-DVI_DEBUG_BOUNDS=1, the library libvi_checked.so): every
// voxel-pair, brick-flag, TF, stack-texture, stack-store, output, raw-voxel
// and grid index is tested against its array before the access.  A bad one is
// counted in a device-wide record of the kernel's translation unit (count,
// first site, first index) and the access is skipped: no trap, no fault, the
// kernel runs to its end.  The release build compiles the tests out.
#ifndef VI_DEBUG_BOUNDS
#define VI_DEBUG_BOUNDS 0
#endif
enum DebugSite {
    kSiteOctet = 1,       // volume footprint load (sweep, march)
    kSiteBrick = 2,       // brick flag load (sweep, march)
    kSiteTfAlpha = 3,     // TF alpha entry (sweep, march)
    kSiteTfColour = 4,    // TF RGBA entry (march)
    kSiteStackTex = 5,    // stack texture / slice of a lookup (march)
    kSiteStackStore = 6,  // stack element a sweep store writes
    kSitePixel = 7,       // output pixel (march)
    kSiteRaw = 8,         // raw voxel read (pair-brick and brick-range builds)
    kSiteGrid = 9,        // voxel pair, brick range or brick flag written by a grid build
};

// Bricks of 2^kBrickShift voxels per axis; flags[bz][by][bx] = 1 if a sample
// whose trilinear footprint starts in the brick may have alpha > 0.  16^3
// measured fastest: coarser bricks skip a little less, but each transparent
// run is crossed in fewer steps (256^3 CT cone march 0.985 -> 0.908 ms
// against 8^3;
// 4^3 and 32^3 were slower; 8^3 again 0.841 against 0.784 ms later on).
#ifndef VI_BRICK_SHIFT
#define VI_BRICK_SHIFT 4
#endif
constexpr int kBrickShift = VI_BRICK_SHIFT;
constexpr int kBrick = 1 << kBrickShift;
// Pair bricks: pairs per row, per plane and per brick, and the offsets of the
// footprint's rows y + 1, z + 1 and y + 1, z + 1 from its first pair.
constexpr int kPairRow = kBrick;
constexpr int kPairPlane = kBrick * (kBrick + 1);
constexpr int kPairsPerBrick = kBrick * (kBrick + 1) * (kBrick + 1);

struct VolumeView {
    const void* data;  // pair bricks
    int nx, ny, nz;
    int nbx, nby, nbz;    // bricks per axis
    float fnx, fny, fnz;  // (float)nx ...
};

// Occupancy.  flags[b] != 0: brick b may yield alpha > 0 (the sweep's test;
// one byte per 16^3 brick, index (bz nby + by) nbx + bx).  The skip
// distances live on a finer grid of cells, 2^kCellShift voxels a side (each
// brick holds kCellsPerBrick^3 of them; index (cz cny + cy) cnx + cx):
// skip[c] is 0 for a cell that may yield alpha > 0, else the L-infinity
// distance, in cells and capped at kSkipCap + 1, from c to the nearest such
// cell -- so every cell within skip[c] - 1 of c along each axis cannot.  The
// march tests its samples and takes its transparent runs on the cells; the
// lockstep sweep takes its runs on them.
#ifndef VI_CELL_SHIFT
#define VI_CELL_SHIFT 3
#endif
constexpr int kCellShift = VI_CELL_SHIFT;
static_assert(kCellShift <= kBrickShift && kCellShift >= 1, "cells subdivide the bricks");
constexpr int kCellsPerBrick = 1 << (kBrickShift - kCellShift);  // per axis
constexpr int kSkipCap = 31;

struct GridView {
    const uint8_t* flags;
    const uint8_t* skip;
    int nbx, nby;  // bricks per axis (flags)
    int cnx, cny;  // cells per axis (skip)
#if VI_DEBUG_BOUNDS
    int nbz, cnz;
#endif
};

// The attenuation stack in device memory: one pitched 2D texture of R x R
// cells, 2^cells_log2 cells to a row of cells.  Slice k is the cell in column
// c = k & (2^cells_log2 - 1) and row r = k >> cells_log2: its texel (i, j) is
// element (r R + j) pitch + c R + i.  One texture for every slice keeps the
// lookup's texture handle the same for every lane (a per-lane handle costs a
// loop over the handles a warp holds).  Lookups clamp their coordinates to the
// slice, so a footprint never leaves its cell except with weight 0, and what
// it reads there (the next cell, or a cell no slice uses) is finite: the
// texture memory is zeroed whenever its layout changes.
struct StackView {
    cudaTextureObject_t tex;
    int cells_log2;  // cells to a row of cells = 2^cells_log2
};

// Element offset of slice k's texel (0, 0), for a row pitch of `pitch`
// elements.
__host__ __device__ __forceinline__ size_t slice_origin(int k, int R, int cells_log2,
                                                        size_t pitch) {
    const size_t col = (size_t)(k & ((1 << cells_log2) - 1));
    const size_t row = (size_t)(k >> cells_log2);
    return row * (size_t)R * pitch + col * (size_t)R;
}

struct SweepParams {
    VolumeView vol;
    GridView grid;
    const float4* tf;  // M entries (alpha in .w)
    int M;
    float tf_vmin, tf_scale;  // x = (v - vmin) * scale, scale = (M - 1) / (vmax - vmin)
    LightFrame lt;
    void* stack;              // pitched: see StackView
    size_t row_pitch;         // bytes
    int cells_log2;           // see StackView
    int opacity_correction;
    float spacing_vox;        // slice spacing in voxels (opacity correction exponent)
    float comp_n;             // darkening compensation exponent, 0 = off
    int depth;                // 1: store optical depth (Eq. 5-6), else transmittance
    unsigned* tile_counter;   // work counter of the persistent sweep (zeroed per launch)
    int lockstep;             // 1: a warp's lanes step through the slices together
};

// Stacks of at least this many texel-slices are swept in lockstep: each
// slice's stores of a warp are then coalesced, which pays once the stores
// dominate (1024 x 2048^2: 4.43 vs 7.1 ms; 512 x 1024^2 FP32: 0.664 vs 0.695
// ms), while smaller stacks sweep faster with each lane walking its own column
// (256 x 512^2 and every smaller scalability stack: 0.111 vs 0.140 ms).
#ifndef VI_SWEEP_LOCKSTEP_MIN
#define VI_SWEEP_LOCKSTEP_MIN (1ull << 29)
#endif

// Cap of a stored optical depth (exp(-64) < 2e-28) and the most shells.
constexpr float kDepthMax = 64.0f;
constexpr int kMaxShells = 4;

// Camera frame (binary32 index path): forward f, right r, up u, image-plane
// half extents (sx, sy) at unit distance (perspective) or absolute (ortho).
struct CameraFrame {
    float eye[3], f[3], r[3], u[3];
    float sx, sy;
    int perspective;
    int W, H;
    float dt;      // step_vox / max(nx, ny, nz)
    float inv_dt;  // 1 / dt, for estimates only (the index path uses dt)
};

struct MarchParams {
    VolumeView vol;
    GridView grid;
    const float4* tf;
    int M;
    float tf_vmin, tf_scale;
    LightFrame lt;
    StackView stack;
    CameraFrame cam;
    float shell_off[kMaxShells][6][3];  // light-space offsets of the shell points, per shell
    int shells;             // shells in use (1 .. kMaxShells)
    float shell_reach;      // max |u|, |v| texel offset of the first shell's points
    float shell_r[kMaxShells];  // point light: world radius of shell q + 1
    float tanphi;           // point light: tan of the cone half angle
    int depth;              // 1: the stack holds optical depth; light factor exp(-value)
    int slice_linear;       // 1: linear filtering between slices
    float cone_rad[2];      // ring radii in texels, rings 1 and 2
    float cone_thr;         // 1e-6 * sigma: B_proj fallback threshold
    float ert;
    float bg[4];
    float color[3];
    float ambient;
    int opacity_correction;
    float step_vox;
    float4* out;            // [H][W]
    int32_t* counts;        // optional [H][W]: samples composited
    int32_t* lit;           // optional [H][W]: samples with alpha > 0
    unsigned* tile_counter; // work counter of the persistent march (zeroed per launch)
    int block_threads;      // threads per block at most (0: the kernel's maximum)
};

enum { kTraceWords = 40, kTraceNone = 0x7fffffff };

// Launchers (defined in vi_sweep.cu / vi_march.cu).  Return a cudaError_t.
cudaError_t launch_sweep(const SweepParams& p, int voxel_type, int format, cudaStream_t s);
cudaError_t launch_march(const MarchParams& p, int voxel_type, int format, int mode,
                         cudaStream_t s);
cudaError_t launch_trace(const MarchParams& p, int voxel_type, int format, int mode, int x,
                         int y, int32_t* rec, int max_rec, int* n_rec, cudaStream_t s);
// The pair bricks of the volume and the value range of every brick and of
// every cell (each with its one-voxel apron), in one pass over the raw voxels.
// range: nbricks brick ranges followed by ncells cell ranges (grid_counts).
cudaError_t launch_volume_grid(const void* raw, int nx, int ny, int nz, int voxel_type,
                               void* pairs, uint32_t* range, cudaStream_t s);
// Bricks and cells of an nx x ny x nz volume.
inline void grid_counts(int nx, int ny, int nz, size_t* nbricks, size_t* ncells) {
    const size_t nbx = (size_t)((nx + kBrick - 1) >> kBrickShift);
    const size_t nby = (size_t)((ny + kBrick - 1) >> kBrickShift);
    const size_t nbz = (size_t)((nz + kBrick - 1) >> kBrickShift);
    *nbricks = nbx * nby * nbz;
    *ncells = *nbricks * kCellsPerBrick * kCellsPerBrick * kCellsPerBrick;
}
// Bytes of the pair bricks of an nx x ny x nz volume of voxel_bytes-byte voxels.
inline size_t pair_brick_bytes(int nx, int ny, int nz, size_t voxel_bytes) {
    const size_t bricks = (size_t)((nx + kBrick - 1) >> kBrickShift) *
                          (size_t)((ny + kBrick - 1) >> kBrickShift) *
                          (size_t)((nz + kBrick - 1) >> kBrickShift);
    return bricks * (size_t)kPairsPerBrick * 2 * voxel_bytes;
}
// Device addresses of the fixed scratch behind vi_render_host_noalloc on the
// current device (looked up once per device; no allocation).
constexpr size_t kNoallocMaxPixels = 512 * 512;
cudaError_t noalloc_scratch(unsigned** counter, float4** image);
// One frame of a batched launch (vi_render_batch): its march parameters, the
// ready word its context publishes (vi_post_ready) and the epoch it must
// reach, and its place in the batch's queue of tiles.
struct BatchFrame {
    MarchParams p;
    const unsigned* ready;
    unsigned epoch;
    unsigned first_tile;  // the frame's first item in its launch's queue
    unsigned tiles_x;     // tiles per row
    int kind;             // voxel type * 8 + format * 4 + mode (formats F32 = 0, F16 = 1)
    int index;            // the frame's place in the caller's list (its status word)
};
constexpr int kBatchMaxFrames = 64;
// Enqueues a batch (see vi_render_batch) on stream s: one persistent launch
// per kind of frame present, then a copy of frame f's status word (VI_OK /
// VI_ETIMEOUT) to the host address status_dst[f] (page-locked for the copy to
// be asynchronous).  Returns without waiting.
cudaError_t enqueue_march_batch(const BatchFrame* frames, int count, unsigned long long wait_ns,
                                int* const* status_dst, cudaStream_t s);
// Writes `epoch` to *ready on stream s, ordered after the stream's earlier work
// and released to the whole device.
cudaError_t launch_post_ready(unsigned* ready, unsigned epoch, cudaStream_t s);
// Brick flags from the brick ranges and the TF's prefix count of entries with
// alpha > 0; cell flags from the cell ranges (into tmp), then the cells' skip
// distances from them (three passes, one per axis, through tmp: ncells bytes).
// range as launch_volume_grid writes it.
cudaError_t launch_brick_flags(const uint32_t* range, int nbx, int nby, int nbz,
                               const int* lit_prefix, int M, float vmin, float vmax,
                               uint8_t* flags, uint8_t* skip, uint8_t* tmp, cudaStream_t s);
#if VI_DEBUG_BOUNDS
// Copies the violation record of the sweep, march or grid kernels on the
// current device to out[4] and clears it (waits for the device first).
cudaError_t debug_record_sweep(unsigned out[4]);
cudaError_t debug_record_march(unsigned out[4]);
cudaError_t debug_record_grid(unsigned out[4]);
#endif

}  // namespace vi
