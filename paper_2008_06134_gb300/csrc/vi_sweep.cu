// vi_sweep.cu -- the light-space sweep (Section 3.2.1, Algorithm 1).
//
// One thread per light texel column (i, j).  The column walks the n slice
// planes from the one nearest the light, carrying the transmittance T in an
// FP32 register: it stores T into buffer k (the light arriving at plane k),
// then applies the back-to-front blend of Eq. 4 to a scalar transmittance,
// T <- T (1 - alpha_k).  All n slices come out of one launch (the paper's
// multi-slice-per-pass future work), with no framebuffer read-back.  In the
// extinction form of Eq. 5-6 (DEPTH) the column carries the optical depth
// D <- D + tau_k, tau_k = -ln(1 - alpha_k), capped at kDepthMax, and stores D.
//
// Memory: the volume's pair bricks are read through the read-only path (four
// aligned loads per footprint; for the sizes this targets they fit in L2).  A warp covers a 16 x 2 tile of texels, so its 32
// sample points form a compact patch of the slice plane and its trilinear
// footprints share sectors; each store of slice k writes two 64-byte (FP32)
// or 32-byte (16-bit) row segments.  Slices outside the cube only store (the inside slices of a
// column form one interval, found exactly); inside, a point in a brick that
// cannot yield alpha > 0 skips the gather.  The transfer function's alpha
// column is staged in shared memory.
#include "vi_device.cuh"

namespace vi {

namespace {

constexpr int kSweepThreads = 256;

// 1: the per-lane sweep takes rows of tiles from the middle outwards (config
// 2: 0.104 -> 0.097 ms); 0: raster order.  The lockstep sweep keeps raster
// order (middle-out: 3.23 -> 3.38 ms on the 1024 x 2048^2 stack, whose many
// tiles per warp leave little drain to fill and whose rows lose locality).
#ifndef VI_SWEEP_TILE_ORDER
#define VI_SWEEP_TILE_ORDER 1
#endif

// 1: persistent warps take tiles from a counter; 0: one tile per warp.
#ifndef VI_SWEEP_PERSISTENT
#define VI_SWEEP_PERSISTENT 1
#endif

// Width in texels of a warp's tile for FP32 stacks (16-bit stacks take 16).
// 16 x 2 measured faster than 8 x 4 (0.110 vs 0.116 ms on 256 x 512^2); 4 x 8,
// whose rows cover half a sector, took 0.30 ms.
#ifndef VI_SWEEP_TILE_W32
#define VI_SWEEP_TILE_W32 16
#endif

// Resident blocks per SM the register allocation is fitted to.  Two (up to
// 128 registers a thread) measured fastest: 0.119 ms on the 256 x 512^2
// sweep of a 256^3 CT phantom, against 0.143 / 0.169 ms for three / four blocks; eight- or
// sixteen-slice batches were slower than four.
#ifndef VI_SWEEP_MIN_BLOCKS
#define VI_SWEEP_MIN_BLOCKS 2
#endif
// Slices whose loads are issued together.
#ifndef VI_SWEEP_BATCH
#define VI_SWEEP_BATCH 4
#endif
constexpr int kBatch = VI_SWEEP_BATCH;
// 1: a batch's footprint loads are issued for every slice inside the column's
// interval, beside its brick-flag loads, instead of after them for the
// flagged slices only (the loads then overlap the flags' latency; a slice in
// an unflagged brick drops its footprint unused).  Slower: the 256 x 512^2
// sweep of a 256^3 CT phantom 0.096 -> 0.141 ms, the 1024 x 2048^2 sweep of
// the 1024^3 volume 3.19 -> 3.22 ms.  The flags are a few KB and hit in L1,
// so the wait they cost is short, while the footprints of the empty space
// inside the cube come through L2 and DRAM.
#ifndef VI_SWEEP_SPECULATE
#define VI_SWEEP_SPECULATE 0
#endif
constexpr bool kSpeculate = VI_SWEEP_SPECULATE;
// The lockstep sweep (stacks of 2^29 texel-slices and more) keeps fewer loads
// per lane in flight and more warps per SM: two-slice batches at three blocks
// per SM (80 registers) measured 4.42 ms on the 1024 x 2048^2 FP16 sweep of the
// 1024^3 workload, against 5.06 ms at four-slice batches and two blocks (4.60
// and 4.68 ms at 2 x 4 and 3 x 3; 4.91 ms at 1 x 5).  The per-lane sweep is
// fastest at 4 x 2 (0.111 ms on the 256 x 512^2 sweep; 0.121-0.179 ms for
// the others).
#ifndef VI_SWEEP_LOCKSTEP_MIN_BLOCKS
#define VI_SWEEP_LOCKSTEP_MIN_BLOCKS 3
#endif
#ifndef VI_SWEEP_LOCKSTEP_BATCH
#define VI_SWEEP_LOCKSTEP_BATCH 2
#endif
constexpr int kLockBatch = VI_SWEEP_LOCKSTEP_BATCH;

// A texel column is the line o + s w: for a directional light o is the
// texel's point on the plane through the centre and w = L; for a point light
// o = P and w the texel's ray direction.  Slice k is at s_k = min + k dL - Lc.

// Whether the point of slice k on the column lies in [0,1]^3, evaluated
// exactly as the sweep evaluates it.
__device__ __forceinline__ bool texel_inside(const LightFrame& lt, int k, const float o[3],
                                             const float w[3]) {
    const float sk = __fsub_rn(__fmaf_rn((float)k, lt.dL, lt.min), lt.Lc);
    const float P0 = __fmaf_rn(sk, w[0], o[0]);
    const float P1 = __fmaf_rn(sk, w[1], o[1]);
    const float P2 = __fmaf_rn(sk, w[2], o[2]);
    return P0 >= 0.0f && P0 <= 1.0f && P1 >= 0.0f && P1 <= 1.0f && P2 >= 0.0f && P2 <= 1.0f;
}

// Element offsets of the slices (the cell layout of StackView): slice k's
// texels start slice_origin(k) elements past slice 0's.
struct SliceAddr {
    size_t cell_row;  // elements from a row of cells to the next: R pitch
    int R, cells_log2;
    __device__ __forceinline__ size_t at(int k) const {
        return (size_t)(k >> cells_log2) * cell_row +
               (size_t)((k & ((1 << cells_log2) - 1)) * R);
    }
};

__device__ __forceinline__ SliceAddr slice_addr(const SweepParams& p, size_t esize) {
    return SliceAddr{(size_t)p.lt.R * (p.row_pitch / esize), p.lt.R, p.cells_log2};
}

// One stack store; a checked build first tests the element against the stack
// (its rows of cells).
template <typename T>
__device__ __forceinline__ void put(const SweepParams& p, T* out, size_t at, T v) {
    if (!VI_BOUNDS_OK(kSiteStackStore, (out + at) - static_cast<T*>(p.stack),
                      (long long)(((p.lt.n - 1) >> p.cells_log2) + 1) * p.lt.R *
                          (long long)(p.row_pitch / sizeof(T))))
        return;
    out[at] = v;
}

// Stores v into slices [k0, k1) of a column (out: the column's texel in slice
// 0).  Slices run along a row of cells R elements apart, so each row of cells
// takes one address computation and then one pointer step per store.
// VI_SWEEP_FILL_ROWS 0: the address of every slice from its index instead.
#ifndef VI_SWEEP_FILL_ROWS
#define VI_SWEEP_FILL_ROWS 1
#endif
template <typename T>
__device__ __forceinline__ void fill_slices(const SweepParams& p, T* out, const SliceAddr& slice,
                                            int k0, int k1, T v) {
    if (!VI_SWEEP_FILL_ROWS) {
        for (int k = k0; k < k1; ++k) put(p, out, slice.at(k), v);
        return;
    }
    const int per_row = 1 << slice.cells_log2;
    for (int k = k0; k < k1;) {
        const int row_end = min(k1, (k | (per_row - 1)) + 1);  // first slice of the next row
        size_t at = slice.at(k);
#pragma unroll 4
        for (; k < row_end; ++k, at += (size_t)slice.R) put(p, out, at, v);
    }
}

// Transparent runs of a column (the lockstep sweep, VI_SWEEP_SKIP 1): slice
// k's footprint lies in a skip-grid cell whose skip distance d says that
// every cell within d - 1 of it (along each axis) cannot yield alpha > 0, so
// the slices whose points stay in that box of cells leave T unchanged and
// only store it.  Returns the last slice of the run that starts at k (at most
// kout), or k - 1 if slice k's cell may yield alpha > 0.  The run's end is
// estimated from where the column leaves the box and confirmed on the index
// path: each cell coordinate of P_k is monotone in k, so the slices between
// two confirmed ones lie in the box too.  The per-lane sweep does not take runs:
// its lanes sit at different slices, and one lane's run serialises against
// its neighbours' batches (256 x 512^2 sweep of a 256^3 CT phantom 0.104 ->
// 0.118 ms with them).
#ifndef VI_SWEEP_SKIP
#define VI_SWEEP_SKIP 1
#endif
__device__ __forceinline__ VoxelCoord slice_cell(const LightFrame& lt, const VolumeView& v, int k,
                                                 const float o[3], const float w[3]) {
    const float sk = __fsub_rn(__fmaf_rn((float)k, lt.dL, lt.min), lt.Lc);
    return voxel_coord_inside(v, __fmaf_rn(sk, w[0], o[0]), __fmaf_rn(sk, w[1], o[1]),
                              __fmaf_rn(sk, w[2], o[2]));
}

__device__ __forceinline__ int transparent_run(const SweepParams& p, const float o[3],
                                               const float w[3], int k, int kout) {
    const LightFrame& lt = p.lt;
    const VoxelCoord c0 = slice_cell(lt, p.vol, k, o, w);
    const int d = cell_skip(p.grid, c0);
    if (d == 0) return k - 1;
    const int rad = d - 1;
    // Column parameter s where the footprint's lower corner leaves the box;
    // slice k' sits at s = min + k' dL - Lc.
    const VoxelRay q = voxel_ray(p.vol, o, w);
    const float s_exit = cell_exit(q, c0, rad);
    const float kf = __fdividef(s_exit + lt.Lc - lt.min, lt.dL);
    if (!(kf < 2.0e9f)) return k;  // no exit estimate: the one slice
    const int j = min((int)kf - 1, kout);
    if (j <= k) return k;
    const VoxelCoord cj = slice_cell(lt, p.vol, j, o, w);
    return within_cells(c0, cj, rad) ? j : k;
}

// The slices of a warp's 32 columns, in lockstep: every lane stores slice k at
// the same step, so each slice's stores of the warp are coalesced.  A lane
// applies alpha only inside its own interval [kin, kout]; elsewhere it stores
// its current value, which is the full light before the interval and the light
// that left the cube after it.  Loads of four slices are issued together.
template <typename VoxT, typename Fmt, bool DEPTH>
__device__ __forceinline__ void sweep_lockstep(const SweepParams& p, const float* s_alpha,
                                               const float o[3], const float w[3], float spacing,
                                               int kin, int kout, bool valid,
                                               typename Fmt::T* out, SliceAddr slice) {
    const LightFrame& lt = p.lt;
    const bool has = kin <= kout;
    const int klo = __reduce_min_sync(0xffffffffu, has ? kin : lt.n);
    const int khi = __reduce_max_sync(0xffffffffu, has ? kout : -1);
    float T = DEPTH ? 0.0f : 1.0f;  // transmittance, or optical depth
    const typename Fmt::T one = Fmt::pack(T);
    if (valid) fill_slices(p, out, slice, 0, klo, one);
    int k = klo;
    bool try_skip = true;  // this lane's last batch had no slice that may be lit
    for (; k <= khi; k += kLockBatch) {
        if (VI_SWEEP_SKIP && __all_sync(0xffffffffu, try_skip)) {
            // A warp-wide transparent run: to the first slice any lane may
            // light (before its interval and after it every slice is alpha = 0).
            int run_end;
            if (k > kout) run_end = khi;
            else if (k < kin) run_end = kin - 1;
            else run_end = transparent_run(p, o, w, k, kout);
            const int to = __reduce_min_sync(0xffffffffu, run_end);
            if (to >= k) {
                if (valid) fill_slices(p, out, slice, k, to + 1, Fmt::pack(T));
                k = to + 1 - kLockBatch;  // the loop's step resumes at to + 1
                continue;
            }
        }
        OctetRef ref[kLockBatch];
        bool lit[kLockBatch];
#pragma unroll
        for (int u = 0; u < kLockBatch; ++u) {
            lit[u] = false;
            if (k + u >= kin && k + u <= kout) {
                const float sk = __fsub_rn(__fmaf_rn((float)(k + u), lt.dL, lt.min), lt.Lc);
                const VoxelCoord vc = voxel_coord_inside(p.vol, __fmaf_rn(sk, w[0], o[0]),
                                                         __fmaf_rn(sk, w[1], o[1]),
                                                         __fmaf_rn(sk, w[2], o[2]));
                ref[u] = octet_ref(p.vol, vc);
                lit[u] = brick_may_be_lit(p.grid, vc, ref[u].brick);
            }
        }
        typename Octet<VoxT>::V oct[kLockBatch];
#pragma unroll
        for (int u = 0; u < kLockBatch; ++u)
            if (kSpeculate ? k + u >= kin && k + u <= kout : lit[u])
                oct[u] = octet_load<VoxT>(p.vol, ref[u].idx);
#pragma unroll
        for (int u = 0; u < kLockBatch; ++u) {
            if (k + u > khi) break;
            float alpha = 0.0f;
            if (lit[u]) {
                int e;
                float f;
                tf_coord(trilinear_octet<VoxT>(oct[u], ref[u]), p.tf_vmin, p.tf_scale, p.M, &e,
                         &f);
                if (!VI_BOUNDS_OK(kSiteTfAlpha, e, p.M - 1)) e = 0;
                const float a0 = s_alpha[e];
                alpha = fmaf(f, s_alpha[e + 1] - a0, a0);
                if (p.opacity_correction)
                    alpha = 1.0f - exp2f(spacing * log2f(fmaxf(1.0f - alpha, 0.0f)));
            }
            float stored = T;
            if (p.comp_n != 0.0f)
                stored = DEPTH ? fmaxf(0.0f, T - p.comp_n * log1pf(alpha))
                               : fminf(1.0f, T * powf(1.0f + alpha, p.comp_n));
            if (valid) {
                const typename Fmt::T q = Fmt::pack(stored);
                put(p, out, slice.at(k + u), q);
            }
            if (DEPTH)
                T = fminf(T - log1pf(-alpha), kDepthMax);  // alpha = 1: tau = inf, capped
            else
                T *= (1.0f - alpha);
        }
        try_skip = true;
#pragma unroll
        for (int u = 0; u < kLockBatch; ++u) try_skip = try_skip && !lit[u];
    }
    if (klo <= khi) k = khi + 1;  // the last batch may have run past khi
    const typename Fmt::T last = Fmt::pack(T);
    if (valid) fill_slices(p, out, slice, k, lt.n, last);
}

// Column set-up of texel (i, j): the column's origin o and direction w, its
// slice spacing in voxels (opacity correction), and the interval [kin, kout]
// of slices whose point lies in the cube (kin > kout: none).
__device__ __forceinline__ void column_setup(const SweepParams& p, int i, int j, float o[3],
                                             float w[3], float& spacing, int& kin, int& kout) {
    const LightFrame& lt = p.lt;
    // World position of texel (i, j) on the plane through the centre.
    float qi = __fdiv_rn((float)(2 * i + 1), (float)lt.R);
    float qj = __fdiv_rn((float)(2 * j + 1), (float)lt.R);
    float u = __fmul_rn(__fsub_rn(qi, 1.0f), lt.h);
    float v = __fmul_rn(__fsub_rn(qj, 1.0f), lt.h);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (lt.point) {
            o[a] = lt.P[a];
            w[a] = __fmaf_rn(v, lt.V[a], __fmaf_rn(u, lt.U[a], lt.L[a]));
        } else {
            o[a] = __fmaf_rn(v, lt.V[a], __fmaf_rn(u, lt.U[a], 0.5f));
            w[a] = lt.L[a];
        }
    }
    // Opacity correction: the slice spacing along this column, in voxels.
    spacing = lt.point ? p.spacing_vox * sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2])
                       : p.spacing_vox;

    // Slices whose point lies in the cube form one interval [kin, kout]: every
    // coordinate of P_k is monotone in k even after rounding (each step of the
    // index path is a monotone rounding).  Estimate it in FP32 (FP64 is slow on
    // this part), then settle it with the exact binary32 test.
    float slo = -3.0e38f, shi = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float wa = w[a];
        if (wa != 0.0f) {
            const float inv = 1.0f / wa;
            const float s0 = -o[a] * inv, s1 = (1.0f - o[a]) * inv;
            slo = fmaxf(slo, fminf(s0, s1));
            shi = fminf(shi, fmaxf(s0, s1));
        } else if (o[a] < 0.0f || o[a] > 1.0f) {
            slo = 3.0e38f;
        }
    }
    const float inv_dL = 1.0f / lt.dL;
    const float k0 = (lt.Lc - lt.min) * inv_dL;
    const float klo = fmaf(slo, inv_dL, k0), khi = fmaf(shi, inv_dL, k0);
    kin = (int)fminf(fmaxf(ceilf(klo), 0.0f), (float)lt.n);
    kout = (int)fminf(fmaxf(floorf(khi), -1.0f), (float)(lt.n - 1));
    if (kin > kout) {
        // The estimate says the column misses the cube; a grazing column
        // may still touch it within a slice or two of its closest approach.
        const int kc = (int)fminf(fmaxf(floorf(0.5f * (klo + khi)), 0.0f), (float)(lt.n - 1));
        kin = lt.n;
        kout = -1;
        for (int k = max(kc - 2, 0); k <= min(kc + 2, lt.n - 1); ++k)
            if (texel_inside(lt, k, o, w)) {
                kin = min(kin, k);
                kout = max(kout, k);
            }
    }
    if (kin <= kout) {
        while (kin > 0 && texel_inside(lt, kin - 1, o, w)) --kin;
        while (kin <= kout && !texel_inside(lt, kin, o, w)) ++kin;
        while (kout < lt.n - 1 && texel_inside(lt, kout + 1, o, w)) ++kout;
        while (kout >= kin && !texel_inside(lt, kout, o, w)) --kout;
    }
}

// One texel column (i, j): every slice's value, nearest the light first.
template <typename VoxT, typename Fmt, bool DEPTH, bool LOCKSTEP>
__device__ __forceinline__ void sweep_column(const SweepParams& p, const float* s_alpha, int i,
                                             int j, bool valid) {
    const LightFrame& lt = p.lt;
    if (!LOCKSTEP && !valid) return;
    if (!valid) {  // a lane past the stack's edge: it joins the warp's steps, stores nothing
        i = min(i, lt.R - 1);
        j = min(j, lt.R - 1);
    }
    float o[3], w[3], spacing;
    int kin, kout;
    column_setup(p, i, j, o, w, spacing, kin, kout);

    // Texel (i, j) of slice k: element slice.at(k) past texel (i, j) of slice 0.
    const SliceAddr slice = slice_addr(p, sizeof(typename Fmt::T));
    typename Fmt::T* out = reinterpret_cast<typename Fmt::T*>(static_cast<char*>(p.stack) +
                                                              (size_t)j * p.row_pitch) + i;

    if (LOCKSTEP) {
        if (!valid) {
            kin = lt.n;
            kout = -1;
        }
        sweep_lockstep<VoxT, Fmt, DEPTH>(p, s_alpha, o, w, spacing, kin, kout, valid, out, slice);
        return;
    }
    // Before the cube: full light (transmittance 1, optical depth 0).
    const typename Fmt::T one = Fmt::pack(DEPTH ? 0.0f : 1.0f);
    int k = min(kin, lt.n);
    fill_slices(p, out, slice, 0, k, one);
    // Inside the cube, four slices at a time: their positions, brick flags and
    // footprints do not depend on T, so the loads of a batch are issued together
    // and their latencies overlap; T then runs through the batch in order.
    float T = DEPTH ? 0.0f : 1.0f;  // transmittance, or optical depth
    for (; k <= kout; k += kBatch) {
        OctetRef ref[kBatch];
        bool lit[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const float sk = __fsub_rn(__fmaf_rn((float)(k + u), lt.dL, lt.min), lt.Lc);
            // Slices past kout (the batch's tail) compute an address but never load.
            const VoxelCoord vc = voxel_coord_inside(p.vol, __fmaf_rn(sk, w[0], o[0]),
                                                     __fmaf_rn(sk, w[1], o[1]),
                                                     __fmaf_rn(sk, w[2], o[2]));
            ref[u] = octet_ref(p.vol, vc);
            lit[u] = k + u <= kout && brick_may_be_lit(p.grid, vc, ref[u].brick);
        }
        typename Octet<VoxT>::V oct[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (kSpeculate ? k + u <= kout : lit[u]) oct[u] = octet_load<VoxT>(p.vol, ref[u].idx);
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (k + u > kout) break;
            float alpha = 0.0f;
            if (lit[u]) {
                int e;
                float f;
                tf_coord(trilinear_octet<VoxT>(oct[u], ref[u]), p.tf_vmin, p.tf_scale, p.M, &e,
                         &f);
                if (!VI_BOUNDS_OK(kSiteTfAlpha, e, p.M - 1)) e = 0;
                const float a0 = s_alpha[e];
                alpha = fmaf(f, s_alpha[e + 1] - a0, a0);
                if (p.opacity_correction)
                    alpha = 1.0f - exp2f(spacing * log2f(fmaxf(1.0f - alpha, 0.0f)));
            }
            float stored = T;
            if (p.comp_n != 0.0f)
                stored = DEPTH ? fmaxf(0.0f, T - p.comp_n * log1pf(alpha))
                               : fminf(1.0f, T * powf(1.0f + alpha, p.comp_n));
            const typename Fmt::T q = Fmt::pack(stored);
            put(p, out, slice.at(k + u), q);
            if (DEPTH)
                T = fminf(T - log1pf(-alpha), kDepthMax);  // alpha = 1: tau = inf, capped
            else
                T *= (1.0f - alpha);
        }
    }
    if (kin <= kout) k = kout + 1;  // the last batch may have run past kout
    // Past the cube: the light that left it.
    const typename Fmt::T last = Fmt::pack(T);
    fill_slices(p, out, slice, k, lt.n, last);
}


// Persistent warps: each warp takes TW x TH texel tiles, in raster order, from
// a global counter until none are left.  Columns through the middle of the
// cube are long and those near the corners short; taking tiles as warps free
// up keeps the SMs busy to the end instead of waiting for the last long
// blocks of a fixed grid.  A warp covers TW x TH texels (16 x 2), so each row
// of its store fills whole 32-byte sectors.
template <typename VoxT, typename Fmt, bool DEPTH, bool LOCKSTEP>
__global__ void __launch_bounds__(kSweepThreads, LOCKSTEP ? VI_SWEEP_LOCKSTEP_MIN_BLOCKS
                                                       : VI_SWEEP_MIN_BLOCKS)
    sweep_kernel(const SweepParams p) {
    extern __shared__ float s_alpha[];
    for (int e = threadIdx.x; e < p.M; e += kSweepThreads) s_alpha[e] = p.tf[e].w;
    __syncthreads();
    constexpr int TW = sizeof(typename Fmt::T) == 2 ? 16 : VI_SWEEP_TILE_W32;
    constexpr int TH = 32 / TW;
    const int lane = threadIdx.x & 31;
    const int R = p.lt.R;
    const unsigned tiles_x = (unsigned)(R + TW - 1) / TW;
    const unsigned ntiles = tiles_x * ((unsigned)(R + TH - 1) / TH);
    for (int once = 0;; ++once) {
        unsigned tile = 0;
        if (VI_SWEEP_PERSISTENT) {
            if (lane == 0) tile = atomicAdd(p.tile_counter, 1u);
            tile = __shfl_sync(0xffffffffu, tile, 0);
        } else {  // one tile per warp, in launch order
            if (once) break;
            tile = blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5);
        }
        if (tile >= ntiles) break;
        int trow = (int)(tile / tiles_x);
        if (VI_SWEEP_TILE_ORDER && !LOCKSTEP) {
            // Rows of tiles from the middle outwards: 0, -1, +1, -2, ... from
            // the middle row, so the long columns through the cube come first
            // and the short ones fill the end.
            const int ty = (int)(ntiles / tiles_x), r = trow;
            trow = ty / 2 + ((r & 1) ? -((r + 1) >> 1) : (r >> 1));
        }
        const int i = (int)(tile % tiles_x) * TW + (lane % TW);
        const int j = trow * TH + (lane / TW);
        sweep_column<VoxT, Fmt, DEPTH, LOCKSTEP>(p, s_alpha, i, j, i < R && j < R);
    }
}

// ---------------------------------------------------------------------------
// Chunked sweep.  The product of Algorithm 1 along a column is associative, so
// a block of kChunkWarps warps shares one 16 x 2 texel tile and splits its
// slices into chunks of kChunkLen: warp c takes slices [base + c L, base +
// (c + 1) L) of a round of kChunkWarps L slices.  Each lane computes its
// column's alpha for the chunk and the chunk-local exclusive products in
// registers; the chunk totals meet in shared memory, where each warp forms
// the product of the carry into the round and the totals of the chunks before
// its own (an exclusive scan across warps, in warp order), then stores
// carry-scaled values.  Every slice k of a warp's 32 columns is stored at the
// same step (coalesced), and a tile has kChunkWarps independent chains where
// the per-column walk has one.  Optical depth (DEPTH) carries sums instead of
// products, capped at kDepthMax when stored; the values agree with the serial
// walk up to the FP32 rounding order of the product.
// It is built (VI_SWEEP_CHUNKED=1) but not the default: every shape measured
// slower than the per-column walk, whose 16 warps per SM each carry a tile's
// chain with four slices' loads in flight.  256 x 512^2 FP32: 0.161-0.270 ms
// against 0.110 ms (16 warps x 8 slices: 0.192; 8 x 8 at three or four blocks
// per SM: 0.176 / 0.161; 32 x 8: 0.270; 16 x 16: 0.211); 512 x 1024^2 FP16:
// 0.92-1.45 ms against 0.59 ms.  The block's barriers (three per round) and
// the set-up of each tile's 32 columns, done once while the other warps wait,
// cost more than the extra chains win.
#ifndef VI_SWEEP_CHUNKED
#define VI_SWEEP_CHUNKED 0
#endif
#ifndef VI_SWEEP_CHUNK_WARPS
#define VI_SWEEP_CHUNK_WARPS 16
#endif
#ifndef VI_SWEEP_CHUNK_LEN
#define VI_SWEEP_CHUNK_LEN 8
#endif
#ifndef VI_SWEEP_CHUNK_MIN_BLOCKS
#define VI_SWEEP_CHUNK_MIN_BLOCKS 2
#endif
#ifndef VI_SWEEP_CHUNK_BATCH
#define VI_SWEEP_CHUNK_BATCH 4
#endif
constexpr int kChunkWarps = VI_SWEEP_CHUNK_WARPS;
constexpr int kChunkLen = VI_SWEEP_CHUNK_LEN;
constexpr int kChunkThreads = kChunkWarps * 32;
constexpr int kChunkBatch = VI_SWEEP_CHUNK_BATCH;
static_assert(kChunkLen % kChunkBatch == 0, "a chunk is a whole number of load batches");

// Opacity of slice k on a column whose point lies in the cube (exact index path
// for the point and its cell; FP32 reconstruction and TF).
template <typename VoxT>
__device__ __forceinline__ float column_alpha(const SweepParams& p, const float* s_alpha,
                                              const typename Octet<VoxT>::V& oct,
                                              const OctetRef& ref, float spacing) {
    int e;
    float f;
    tf_coord(trilinear_octet<VoxT>(oct, ref), p.tf_vmin, p.tf_scale, p.M, &e, &f);
    if (!VI_BOUNDS_OK(kSiteTfAlpha, e, p.M - 1)) e = 0;
    const float a0 = s_alpha[e];
    float alpha = fmaf(f, s_alpha[e + 1] - a0, a0);
    if (p.opacity_correction) alpha = 1.0f - exp2f(spacing * log2f(fmaxf(1.0f - alpha, 0.0f)));
    return alpha;
}

template <typename VoxT, typename Fmt, bool DEPTH, bool COMP>
__global__ void __launch_bounds__(kChunkThreads, VI_SWEEP_CHUNK_MIN_BLOCKS)
    sweep_chunked_kernel(const SweepParams p) {
    using T_ = typename Fmt::T;
    extern __shared__ float s_alpha[];  // the TF's alpha column, M entries
    __shared__ float s_o[3][32], s_w[3][32], s_spacing[32], s_carry[32];
    __shared__ float s_total[kChunkWarps][32];
    __shared__ int s_kin[32], s_kout[32], s_range[2];
    __shared__ unsigned s_tile;
    for (int e = threadIdx.x; e < p.M; e += kChunkThreads) s_alpha[e] = p.tf[e].w;
    constexpr int TW = 16, TH = 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LightFrame& lt = p.lt;
    const int R = lt.R, n = lt.n;
    const unsigned tiles_x = (unsigned)(R + TW - 1) / TW;
    const unsigned ntiles = tiles_x * ((unsigned)(R + TH - 1) / TH);
    const SliceAddr slice = slice_addr(p, sizeof(T_));
    const T_ one = Fmt::pack(DEPTH ? 0.0f : 1.0f);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(p.tile_counter, 1u);
        __syncthreads();  // the tile (and, at first, the alpha column) is in place
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        const int i = (int)(tile % tiles_x) * TW + (lane % TW);
        const int j = (int)(tile / tiles_x) * TH + (lane / TW);
        const bool valid = i < R && j < R;
        if (warp == 0) {  // one set-up per column, shared by the block's warps
            float o[3], w[3], spacing;
            int kin, kout;
            column_setup(p, min(i, R - 1), min(j, R - 1), o, w, spacing, kin, kout);
            if (!valid) {
                kin = n;
                kout = -1;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                s_o[a][lane] = o[a];
                s_w[a][lane] = w[a];
            }
            s_spacing[lane] = spacing;
            s_kin[lane] = kin;
            s_kout[lane] = kout;
            s_carry[lane] = DEPTH ? 0.0f : 1.0f;
            const int lo = __reduce_min_sync(0xffffffffu, kin <= kout ? kin : n);
            const int hi = __reduce_max_sync(0xffffffffu, kin <= kout ? kout : -1);
            if (lane == 0) {
                s_range[0] = lo;
                s_range[1] = hi;
            }
        }
        __syncthreads();
        const float o[3] = {s_o[0][lane], s_o[1][lane], s_o[2][lane]};
        const float w[3] = {s_w[0][lane], s_w[1][lane], s_w[2][lane]};
        const float spacing = s_spacing[lane];
        const int kin = s_kin[lane], kout = s_kout[lane];
        const int klo = s_range[0], khi = s_range[1];  // klo > khi: the tile misses the cube
        T_* out = reinterpret_cast<T_*>(static_cast<char*>(p.stack) +
                                        (size_t)min(j, R - 1) * p.row_pitch) + min(i, R - 1);

        // Before the tile's first slice in the cube: full light.
        for (int k = warp; k < min(klo, n); k += kChunkWarps)
            if (valid) {
                put(p, out, slice.at(k), one);
            }
        // Rounds of kChunkWarps chunks over [klo, khi].
        for (int base = klo; base <= khi; base += kChunkWarps * kChunkLen) {
            const int kb = base + warp * kChunkLen;
            float tl[kChunkLen];                  // chunk-local exclusive product (or sum)
            float ex[COMP ? kChunkLen : 1];       // the slice's own alpha, for comp_n
            float T = DEPTH ? 0.0f : 1.0f;
#pragma unroll
            for (int h = 0; h < kChunkLen; h += kChunkBatch) {
                OctetRef ref[kChunkBatch];
                bool lit[kChunkBatch];
#pragma unroll
                for (int u = 0; u < kChunkBatch; ++u) {
                    const int k = kb + h + u;
                    lit[u] = false;
                    if (k >= kin && k <= kout) {
                        const float sk = __fsub_rn(__fmaf_rn((float)k, lt.dL, lt.min), lt.Lc);
                        const VoxelCoord vc =
                            voxel_coord_inside(p.vol, __fmaf_rn(sk, w[0], o[0]),
                                               __fmaf_rn(sk, w[1], o[1]), __fmaf_rn(sk, w[2], o[2]));
                        ref[u] = octet_ref(p.vol, vc);
                        lit[u] = brick_may_be_lit(p.grid, vc, ref[u].brick);
                    }
                }
                typename Octet<VoxT>::V oct[kChunkBatch];
#pragma unroll
                for (int u = 0; u < kChunkBatch; ++u)
                    if (lit[u]) oct[u] = octet_load<VoxT>(p.vol, ref[u].idx);
#pragma unroll
                for (int u = 0; u < kChunkBatch; ++u) {
                    const float alpha =
                        lit[u] ? column_alpha<VoxT>(p, s_alpha, oct[u], ref[u], spacing) : 0.0f;
                    tl[h + u] = T;
                    if (COMP) ex[h + u] = alpha;
                    if (DEPTH)
                        T = T - log1pf(-alpha);  // alpha = 1: tau = inf; capped when stored
                    else
                        T *= (1.0f - alpha);
                }
            }
            s_total[warp][lane] = T;
            __syncthreads();
            float pre = s_carry[lane];
            for (int c = 0; c < warp; ++c)
                pre = DEPTH ? pre + s_total[c][lane] : pre * s_total[c][lane];
#pragma unroll
            for (int u = 0; u < kChunkLen; ++u) {
                const int k = kb + u;
                if (k > khi || !valid) continue;
                float v;
                if (DEPTH) {
                    v = fminf(pre + tl[u], kDepthMax);
                    if (COMP) v = fmaxf(0.0f, v - p.comp_n * log1pf(ex[u]));
                } else {
                    v = pre * tl[u];
                    if (COMP) v = fminf(1.0f, v * powf(1.0f + ex[u], p.comp_n));
                }
                const T_ q = Fmt::pack(v);
                put(p, out, slice.at(k), q);
            }
            __syncthreads();  // every warp has read the carry and the totals
            if (warp == kChunkWarps - 1) s_carry[lane] = DEPTH ? pre + T : pre * T;
        }
        __syncthreads();  // the last carry is in place
        // Past the tile's last slice in the cube: the light that left it.
        float last = s_carry[lane];
        if (DEPTH) last = fminf(last, kDepthMax);
        const T_ q = Fmt::pack(last);
        for (int k = max(khi + 1, 0) + warp; k < n; k += kChunkWarps)
            if (valid) {
                put(p, out, slice.at(k), q);
            }
    }
}

template <typename VoxT, typename Fmt, bool DEPTH>
cudaError_t launch_chunked(const SweepParams& p, cudaStream_t s) {
    const size_t smem = (size_t)p.M * sizeof(float);
    auto kern = p.comp_n != 0.0f ? sweep_chunked_kernel<VoxT, Fmt, DEPTH, true>
                                 : sweep_chunked_kernel<VoxT, Fmt, DEPTH, false>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kChunkThreads, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((p.lt.R + 15) / 16) * ((p.lt.R + 1) / 2);
    long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > tiles) blocks = tiles;
    e = cudaMemsetAsync(p.tile_counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, kChunkThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename VoxT, typename Fmt, bool DEPTH>
cudaError_t launch_typed(const SweepParams& p, cudaStream_t s) {
    if (VI_SWEEP_CHUNKED) return launch_chunked<VoxT, Fmt, DEPTH>(p, s);
    const size_t smem = (size_t)p.M * sizeof(float);
    auto kern = p.lockstep ? sweep_kernel<VoxT, Fmt, DEPTH, true>
                           : sweep_kernel<VoxT, Fmt, DEPTH, false>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepThreads, smem);
    if (e != cudaSuccess) return e;
    // Every SM filled once, never more warps than tiles.
    constexpr int TW = sizeof(typename Fmt::T) == 2 ? 16 : VI_SWEEP_TILE_W32;
    const long long tiles = (long long)((p.lt.R + TW - 1) / TW) * ((p.lt.R + 32 / TW - 1) / (32 / TW));
    long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
    const long long need = (tiles + kSweepThreads / 32 - 1) / (kSweepThreads / 32);
    blocks = (blocks < need && VI_SWEEP_PERSISTENT) ? blocks : need;
    e = cudaMemsetAsync(p.tile_counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, kSweepThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename VoxT>
cudaError_t launch_fmt(const SweepParams& p, int format, cudaStream_t s) {
    if (p.depth) {  // optical depth: not in UNORM16 (its range is [0, 1])
        switch (format) {
            case 0: return launch_typed<VoxT, F32, true>(p, s);
            case 1: return launch_typed<VoxT, F16, true>(p, s);
            case 2: return launch_typed<VoxT, BF16, true>(p, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (format) {
        case 0: return launch_typed<VoxT, F32, false>(p, s);
        case 1: return launch_typed<VoxT, F16, false>(p, s);
        case 2: return launch_typed<VoxT, BF16, false>(p, s);
        case 3: return launch_typed<VoxT, UNORM16, false>(p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_sweep(const SweepParams& p, int voxel_type, int format, cudaStream_t s) {
    if (voxel_type == 0) return launch_fmt<uint8_t>(p, format, s);
    return launch_fmt<uint16_t>(p, format, s);
}

#if VI_DEBUG_BOUNDS
VI_DEBUG_RECORD_ACCESSOR(debug_record_sweep)
#endif

}  // namespace vi
