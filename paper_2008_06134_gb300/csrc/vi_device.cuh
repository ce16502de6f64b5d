// vi_device.cuh -- device helpers shared by the sweep, march and trace kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vi_internal.h"

namespace vi {

// ---------------------------------------------------------------------------
// Bounds checks of checked builds (VI_DEBUG_BOUNDS, see vi_internal.h).
// VI_BOUNDS_OK(site, i, n) is true when 0 <= i < n; otherwise it counts the
// violation in this translation unit's record (the first one's site and index
// kept) and is false, and the caller skips the access.  In release builds it
// is the constant true and its arguments are not evaluated.
#if VI_DEBUG_BOUNDS
static __device__ unsigned g_debug_record[4];  // count, first site, first index (low, high)

__device__ __forceinline__ bool bounds_ok(int site, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&g_debug_record[0], 1u) == 0u) {
        g_debug_record[1] = (unsigned)site;
        g_debug_record[2] = (unsigned)((unsigned long long)i & 0xffffffffull);
        g_debug_record[3] = (unsigned)((unsigned long long)i >> 32);
    }
    return false;
}
#define VI_BOUNDS_OK(site, i, n) ::vi::bounds_ok((site), (long long)(i), (long long)(n))
// Defines the host accessor of this translation unit's record.
#define VI_DEBUG_RECORD_ACCESSOR(name)                                                 \
    cudaError_t name(unsigned out[4]) {                                                \
        cudaError_t e = cudaDeviceSynchronize();                                       \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, g_debug_record, 16);       \
        const unsigned zero[4] = {0u, 0u, 0u, 0u};                                     \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_debug_record, zero, 16);        \
        return e;                                                                      \
    }
#else
#define VI_BOUNDS_OK(site, i, n) true
#endif

// ---------------------------------------------------------------------------
// Stack storage formats.  Accumulation is FP32; these only round at store.

// gather() fetches the 2 x 2 footprint whose lower-left texel is (i0, j0) from
// a pitched 2D texture, given x = i0 + 1, y = j0 + 1 (exact integers, so the
// footprint choice is exact); texture gather returns (i0, j0+1), (i0+1, j0+1),
// (i0+1, j0), (i0, j0) in x, y, z, w.  Raw texels, no filtering: the weights
// are applied in FP32 by the caller.  The texture unit converts each texel
// to FP32 where it can do so exactly or to within an FP32 rounding: binary16
// texels (a half-float texture; binary16 -> binary32 is exact) and UNORM16
// texels (normalised read mode, q / 65535).  BF16 has no texture format: its
// raw 16 bits are gathered and widened with a shift (also exact).
struct F32 {
    using T = float;
    static __device__ __forceinline__ T pack(float x) { return x; }
    static __device__ __forceinline__ void gather(cudaTextureObject_t t, float x, float y,
                                                  float& b00, float& b01, float& b10,
                                                  float& b11) {
        const float4 g = tex2Dgather<float4>(t, x, y, 0);
        b00 = g.w; b01 = g.z; b10 = g.x; b11 = g.y;
    }
};
struct F16 {
    using T = __half;
    static __device__ __forceinline__ T pack(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ void gather(cudaTextureObject_t t, float x, float y,
                                                  float& b00, float& b01, float& b10,
                                                  float& b11) {
        const float4 g = tex2Dgather<float4>(t, x, y, 0);  // binary16 texels, widened
        b00 = g.w; b01 = g.z; b10 = g.x; b11 = g.y;
    }
};
struct BF16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T pack(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ void gather(cudaTextureObject_t t, float x, float y,
                                                  float& b00, float& b01, float& b10,
                                                  float& b11) {
        const uint4 g = tex2Dgather<uint4>(t, x, y, 0);  // raw bfloat16 bits
        b00 = __uint_as_float(g.w << 16); b01 = __uint_as_float(g.z << 16);
        b10 = __uint_as_float(g.x << 16); b11 = __uint_as_float(g.y << 16);
    }
};
// Fixed point on [0, 1] with 16 bits: x = q / 65535.
struct UNORM16 {
    using T = uint16_t;
    static __device__ __forceinline__ T pack(float x) {
        x = fminf(fmaxf(x, 0.0f), 1.0f);
        return (T)__float2uint_rn(x * 65535.0f);
    }
    static __device__ __forceinline__ void gather(cudaTextureObject_t t, float x, float y,
                                                  float& b00, float& b01, float& b10,
                                                  float& b11) {
        const float4 g = tex2Dgather<float4>(t, x, y, 0);  // normalised: q / 65535
        b00 = g.w; b01 = g.z; b10 = g.x; b11 = g.y;
    }
};

// ---------------------------------------------------------------------------
// Index path (binary32, one rounding per operation, never contracted).

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1,
                                         float b2) {
    float p0 = __fmul_rn(a0, b0);
    float p1 = __fmul_rn(a1, b1);
    float p2 = __fmul_rn(a2, b2);
    return __fadd_rn(__fadd_rn(p0, p1), p2);
}

// floor(x) clamped to [lo, hi] as int.
__device__ __forceinline__ int floor_clamp(float x, int lo, int hi) {
    float f = floorf(x);
    f = fminf(fmaxf(f, (float)lo), (float)hi);
    return (int)f;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ---------------------------------------------------------------------------
// Volume reconstruction: trilinear, voxel centres at (idx + 1/2) / N, clamp to
// edge.  Cell indices come from the index path; weights are plain FP32.

struct VoxelCoord {
    int cx, cy, cz;          // floor of the voxel coordinate, clamped to [-1, N]
    int x0, x1, y0, y1, z0, z1;  // footprint corners, clamped to [0, N - 1]
    float wx, wy, wz;        // weights of the upper corners
};

__device__ __forceinline__ VoxelCoord voxel_coord(const VolumeView& v, float P0, float P1,
                                                  float P2) {
    VoxelCoord c;
    float x = __fmaf_rn(P0, v.fnx, -0.5f);
    float y = __fmaf_rn(P1, v.fny, -0.5f);
    float z = __fmaf_rn(P2, v.fnz, -0.5f);
    float flx = floorf(x), fly = floorf(y), flz = floorf(z);
    c.cx = (int)fminf(fmaxf(flx, -1.0f), (float)v.nx);
    c.cy = (int)fminf(fmaxf(fly, -1.0f), (float)v.ny);
    c.cz = (int)fminf(fmaxf(flz, -1.0f), (float)v.nz);
    c.wx = x - flx;
    c.wy = y - fly;
    c.wz = z - flz;
    c.x0 = clampi(c.cx, 0, v.nx - 1);
    c.x1 = clampi(c.cx + 1, 0, v.nx - 1);
    c.y0 = clampi(c.cy, 0, v.ny - 1);
    c.y1 = clampi(c.cy + 1, 0, v.ny - 1);
    c.z0 = clampi(c.cz, 0, v.nz - 1);
    c.z1 = clampi(c.cz + 1, 0, v.nz - 1);
    return c;
}

// voxel_coord for a point known to lie in [0,1]^3 (the sweep's exact inside
// test): x = P N - 1/2 lies in [-1/2, N - 1/2], so floor(x) is already in
// [-1, N - 1] and each corner needs one bound of its clamp.  Same cells and
// weights as voxel_coord for such points.  Points outside give indices out of
// range: the caller must not load through them.
__device__ __forceinline__ VoxelCoord voxel_coord_inside(const VolumeView& v, float P0, float P1,
                                                         float P2) {
    VoxelCoord c;
    float x = __fmaf_rn(P0, v.fnx, -0.5f);
    float y = __fmaf_rn(P1, v.fny, -0.5f);
    float z = __fmaf_rn(P2, v.fnz, -0.5f);
    float flx = floorf(x), fly = floorf(y), flz = floorf(z);
    c.cx = (int)flx;
    c.cy = (int)fly;
    c.cz = (int)flz;
    c.wx = x - flx;
    c.wy = y - fly;
    c.wz = z - flz;
    c.x0 = max(c.cx, 0);
    c.x1 = min(c.cx + 1, v.nx - 1);
    c.y0 = max(c.cy, 0);
    c.y1 = min(c.cy + 1, v.ny - 1);
    c.z0 = max(c.cz, 0);
    c.z1 = min(c.cz + 1, v.nz - 1);
    return c;
}

// Whether b's cell lies within rad cells of a's along every axis.  A cell
// here is the skip grid's cell (2^kCellShift voxels a side) of the
// footprint's lower corner; each of its coordinates is monotone in the
// position along a ray or a light column, so two samples whose cells lie in
// one box of cells have every sample between them in that box too.
__device__ __forceinline__ bool within_cells(const VoxelCoord& a, const VoxelCoord& b, int rad) {
    return abs((a.x0 >> kCellShift) - (b.x0 >> kCellShift)) <= rad &&
           abs((a.y0 >> kCellShift) - (b.y0 >> kCellShift)) <= rad &&
           abs((a.z0 >> kCellShift) - (b.z0 >> kCellShift)) <= rad;
}

// A ray in voxel units for cell-box exits: X_a(t) = o_a N_a + t d_a N_a
// (origin ox, reciprocal rate ix; ix is 0 on an axis the ray does not move
// along).  The footprint's lower corner floor(X_a - 1/2) enters cell b at
// X_a = C b + 1/2, C = 2^kCellShift.
struct VoxelRay {
    float ox[3], ix[3];
};

__device__ __forceinline__ VoxelRay voxel_ray(const VolumeView& v, const float o[3],
                                              const float d[3]) {
    VoxelRay q;
    const float N[3] = {v.fnx, v.fny, v.fnz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q.ox[a] = o[a] * N[a];
        q.ix[a] = d[a] != 0.0f ? __fdividef(1.0f, d[a] * N[a]) : 0.0f;
    }
    return q;
}

// Parameter t at which the footprint's lower corner leaves the box of cells
// within rad of c's cell along every axis (an estimate; callers verify with
// the exact path).  rad = 0: c's cell.
__device__ __forceinline__ float cell_exit(const VoxelRay& q, const VoxelCoord& c, int rad) {
    const int b[3] = {c.x0 >> kCellShift, c.y0 >> kCellShift, c.z0 >> kCellShift};
    float s_exit = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // Moving up, the box ends at cell b + rad + 1; moving down, at b - rad.
        const int edge = q.ix[a] > 0.0f ? b[a] + rad + 1 : b[a] - rad;
        const float plane = (float)(edge * (1 << kCellShift)) + 0.5f;
        if (q.ix[a] != 0.0f) s_exit = fminf(s_exit, (plane - q.ox[a]) * q.ix[a]);
    }
    return s_exit;
}

__device__ __forceinline__ int brick_index(const GridView& g, int x0, int y0, int z0) {
    return ((z0 >> kBrickShift) * g.nby + (y0 >> kBrickShift)) * g.nbx + (x0 >> kBrickShift);
}

__device__ __forceinline__ bool brick_in_grid(const GridView& g, int x0, int y0, int z0) {
    return VI_BOUNDS_OK(kSiteBrick, x0 >> kBrickShift, g.nbx) &&
           VI_BOUNDS_OK(kSiteBrick, y0 >> kBrickShift, g.nby) &&
           VI_BOUNDS_OK(kSiteBrick, z0 >> kBrickShift, g.nbz);
}

// Whether the brick holding the footprint's lower corner may yield alpha > 0.
__device__ __forceinline__ bool brick_may_be_lit(const GridView& g, const VoxelCoord& c) {
    if (!brick_in_grid(g, c.x0, c.y0, c.z0)) return false;
    return __ldg(g.flags + brick_index(g, c.x0, c.y0, c.z0)) != 0;
}

// The same test given the brick's index b (vol_brick of the lower corner).
__device__ __forceinline__ bool brick_may_be_lit(const GridView& g, const VoxelCoord& c, int b) {
    if (!brick_in_grid(g, c.x0, c.y0, c.z0)) return false;
    return __ldg(g.flags + b) != 0;
}

__device__ __forceinline__ int cell_index(const GridView& g, int x0, int y0, int z0) {
    return ((z0 >> kCellShift) * g.cny + (y0 >> kCellShift)) * g.cnx + (x0 >> kCellShift);
}

__device__ __forceinline__ bool cell_in_grid(const GridView& g, int x0, int y0, int z0) {
    return VI_BOUNDS_OK(kSiteBrick, x0 >> kCellShift, g.cnx) &&
           VI_BOUNDS_OK(kSiteBrick, y0 >> kCellShift, g.cny) &&
           VI_BOUNDS_OK(kSiteBrick, z0 >> kCellShift, g.cnz);
}

// Skip distance of the cell holding the footprint's lower corner: 0 if it may
// yield alpha > 0, else 1 + the radius of the box of cells around it that
// cannot (see GridView).
__device__ __forceinline__ int cell_skip(const GridView& g, const VoxelCoord& c) {
    if (!cell_in_grid(g, c.x0, c.y0, c.z0)) return 1;
    return __ldg(g.skip + cell_index(g, c.x0, c.y0, c.z0));
}

// Integer to float without the conversion pipe: v < 2^23 placed in the mantissa
// of 2^23, then 2^23 subtracted (exact).
__device__ __forceinline__ float u2f(unsigned v) {
    return __uint_as_float(0x4b000000u | v) - 8388608.0f;
}

template <typename VoxT>
struct Octet;
template <>
struct Octet<uint16_t> {
    using V = uint4;
    static __device__ __forceinline__ void unpack(const V q, float c[8]) {
        c[0] = u2f(q.x & 0xffffu); c[1] = u2f(q.x >> 16);
        c[2] = u2f(q.y & 0xffffu); c[3] = u2f(q.y >> 16);
        c[4] = u2f(q.z & 0xffffu); c[5] = u2f(q.z >> 16);
        c[6] = u2f(q.w & 0xffffu); c[7] = u2f(q.w >> 16);
    }
};
template <>
struct Octet<uint8_t> {
    using V = uint2;
    static __device__ __forceinline__ void unpack(const V q, float c[8]) {
        c[0] = u2f(q.x & 0xffu); c[1] = u2f((q.x >> 8) & 0xffu);
        c[2] = u2f((q.x >> 16) & 0xffu); c[3] = u2f(q.x >> 24);
        c[4] = u2f(q.y & 0xffu); c[5] = u2f((q.y >> 8) & 0xffu);
        c[6] = u2f((q.y >> 16) & 0xffu); c[7] = u2f(q.y >> 24);
    }
};

// Index of the brick holding voxel (x0, y0, z0): the same index in the pair
// bricks and in the grid's flags and skip distances (one brick grid).
__device__ __forceinline__ int vol_brick(const VolumeView& v, int x0, int y0, int z0) {
    return ((z0 >> kBrickShift) * v.nby + (y0 >> kBrickShift)) * v.nbx + (x0 >> kBrickShift);
}

// The first pair of the footprint whose lower corner is voxel (x0, y0, z0),
// in the pair bricks (see VolumeView), given that voxel's brick b.
__device__ __forceinline__ size_t pair_index_in(int b, int x0, int y0, int z0) {
    constexpr int m = kBrick - 1;
    return (size_t)b * kPairsPerBrick +
           (size_t)(((z0 & m) * (kBrick + 1) + (y0 & m)) * kPairRow + (x0 & m));
}

__device__ __forceinline__ size_t pair_index(const VolumeView& v, int x0, int y0, int z0) {
    return pair_index_in(vol_brick(v, x0, y0, z0), x0, y0, z0);
}

// What a trilinear fetch needs: the first pair of the footprint and the
// weights of its upper corners.  The footprint's upper voxels are clamped
// copies at the high edges; at the low edges (cell -1) the footprint collapses
// onto voxel 0, so the upper corner's weight is 0 there.
struct OctetRef {
    size_t idx;
    int brick;  // the footprint's brick (vol_brick)
    float wx, wy, wz;
};

__device__ __forceinline__ OctetRef octet_ref(const VolumeView& v, const VoxelCoord& c) {
    OctetRef o;
    o.brick = vol_brick(v, c.x0, c.y0, c.z0);
    o.idx = pair_index_in(o.brick, c.x0, c.y0, c.z0);
    o.wx = c.cx < 0 ? 0.0f : c.wx;
    o.wy = c.cy < 0 ? 0.0f : c.wy;
    o.wz = c.cz < 0 ? 0.0f : c.wz;
    return o;
}

// The eight voxels of the footprint whose first pair is idx: four aligned pair
// loads (rows y, y + 1 of planes z, z + 1), packed as one octet (the eight
// voxels in the order c000 c001 c010 c011 c100 c101 c110 c111).
template <typename VoxT>
__device__ __forceinline__ typename Octet<VoxT>::V octet_load(const VolumeView& v, size_t idx) {
    if (!VI_BOUNDS_OK(kSiteOctet, idx + kPairPlane + kPairRow,
                      (long long)v.nbx * v.nby * v.nbz * kPairsPerBrick))
        return typename Octet<VoxT>::V{};
    if constexpr (sizeof(VoxT) == 2) {
        const unsigned* q = static_cast<const unsigned*>(v.data) + idx;
        return make_uint4(__ldg(q), __ldg(q + kPairRow), __ldg(q + kPairPlane),
                          __ldg(q + kPairPlane + kPairRow));
    } else {
        const unsigned short* q = static_cast<const unsigned short*>(v.data) + idx;
        return make_uint2((unsigned)__ldg(q) | ((unsigned)__ldg(q + kPairRow) << 16),
                          (unsigned)__ldg(q + kPairPlane) |
                              ((unsigned)__ldg(q + kPairPlane + kPairRow) << 16));
    }
}

template <typename VoxT>
__device__ __forceinline__ float trilinear_octet(const typename Octet<VoxT>::V oct,
                                                 const OctetRef& o) {
    float q[8];
    Octet<VoxT>::unpack(oct, q);
    float c00 = fmaf(o.wx, q[1] - q[0], q[0]);
    float c01 = fmaf(o.wx, q[3] - q[2], q[2]);
    float c10 = fmaf(o.wx, q[5] - q[4], q[4]);
    float c11 = fmaf(o.wx, q[7] - q[6], q[6]);
    float c0 = fmaf(o.wy, c01 - c00, c00);
    float c1 = fmaf(o.wy, c11 - c10, c10);
    return fmaf(o.wz, c1 - c0, c0);
}

template <typename VoxT>
__device__ __forceinline__ float trilinear_fetch(const VolumeView& v, const VoxelCoord& c) {
    const OctetRef o = octet_ref(v, c);
    return trilinear_octet<VoxT>(octet_load<VoxT>(v, o.idx), o);
}

// The footprint of a sample known to lie in the cube, as the march needs it:
// the footprint's lower corner (clamped to the volume) and the weights
// of the upper corners.  For such a sample x = P N - 1/2 lies in [-1/2, N - 1/2],
// so floor(x) is -1 .. N - 1: at -1 the lower corner clamps to 0 and the
// weight max(x - 0, 0) is 0 (the footprint collapses onto voxel 0), elsewhere
// the weight is x - floor(x).  Same cells and weights as voxel_coord /
// octet_ref, with fewer integer steps.
struct FootprintCell {
    int x0, y0, z0;
    float wx, wy, wz;
};

__device__ __forceinline__ void footprint_axis(float P, float fn, int& i0, float& w) {
    const float x = __fmaf_rn(P, fn, -0.5f);
    const float f0 = fminf(fmaxf(floorf(x), 0.0f), fn - 1.0f);
    i0 = (int)f0;
    w = fmaxf(x - f0, 0.0f);
}

__device__ __forceinline__ FootprintCell footprint_cell(const VolumeView& v, float P0, float P1,
                                                        float P2) {
    FootprintCell c;
    footprint_axis(P0, v.fnx, c.x0, c.wx);
    footprint_axis(P1, v.fny, c.y0, c.wy);
    footprint_axis(P2, v.fnz, c.z0, c.wz);
    return c;
}

__device__ __forceinline__ size_t footprint_index(const VolumeView& v, const FootprintCell& c) {
    return pair_index(v, c.x0, c.y0, c.z0);
}

// The march's test: whether the cell holding the footprint's lower corner may
// yield alpha > 0 (its skip distance is 0 exactly then).
__device__ __forceinline__ bool footprint_may_be_lit(const GridView& g, const FootprintCell& c) {
    if (!cell_in_grid(g, c.x0, c.y0, c.z0)) return false;
    return __ldg(g.skip + cell_index(g, c.x0, c.y0, c.z0)) == 0;
}

// Trilinear value of a footprint's eight voxels (an octet) at its weights.  uint16 voxels are
// unpacked as 2^23 + v (one OR each) and the 2^23 taken off only the four
// lower corners: differences of two such floats are exact, so the result is
// the one trilinear_octet gives, bit for bit.
template <typename VoxT>
__device__ __forceinline__ float trilinear_cell(const typename Octet<VoxT>::V q,
                                                const FootprintCell& c) {
    float m[8];
    if constexpr (sizeof(VoxT) == 2) {
        m[0] = __uint_as_float(0x4b000000u | (q.x & 0xffffu));
        m[1] = __uint_as_float(0x4b000000u | (q.x >> 16));
        m[2] = __uint_as_float(0x4b000000u | (q.y & 0xffffu));
        m[3] = __uint_as_float(0x4b000000u | (q.y >> 16));
        m[4] = __uint_as_float(0x4b000000u | (q.z & 0xffffu));
        m[5] = __uint_as_float(0x4b000000u | (q.z >> 16));
        m[6] = __uint_as_float(0x4b000000u | (q.w & 0xffffu));
        m[7] = __uint_as_float(0x4b000000u | (q.w >> 16));
        constexpr float B = 8388608.0f;
        const float c00 = fmaf(c.wx, m[1] - m[0], m[0] - B);
        const float c01 = fmaf(c.wx, m[3] - m[2], m[2] - B);
        const float c10 = fmaf(c.wx, m[5] - m[4], m[4] - B);
        const float c11 = fmaf(c.wx, m[7] - m[6], m[6] - B);
        const float c0 = fmaf(c.wy, c01 - c00, c00);
        const float c1 = fmaf(c.wy, c11 - c10, c10);
        return fmaf(c.wz, c1 - c0, c0);
    } else {
        Octet<VoxT>::unpack(q, m);
        const float c00 = fmaf(c.wx, m[1] - m[0], m[0]);
        const float c01 = fmaf(c.wx, m[3] - m[2], m[2]);
        const float c10 = fmaf(c.wx, m[5] - m[4], m[4]);
        const float c11 = fmaf(c.wx, m[7] - m[6], m[6]);
        const float c0 = fmaf(c.wy, c01 - c00, c00);
        const float c1 = fmaf(c.wy, c11 - c10, c10);
        return fmaf(c.wz, c1 - c0, c0);
    }
}

// Transfer function position of a value: x in [0, M - 1], entry i = floor(x)
// (at most M - 2) and weight f = x - i.
__device__ __forceinline__ void tf_coord(float v, float vmin, float scale, int M, int* i,
                                         float* f) {
    float x = (v - vmin) * scale;
    x = fminf(fmaxf(x, 0.0f), (float)(M - 1));
    int e = min((int)x, M - 2);
    *i = e;
    *f = x - (float)e;
}

// ---------------------------------------------------------------------------
// Stack lookup (Eq. 9 slice, Eq. 10 UV): nearest slice k = clamp(floor(lambda
// + 1/2), 0, n - 1), bilinear over texel centres at integer (tu, tv) with
// clamp to edge.

__device__ __forceinline__ int slice_index(float lam, int n) {
    return clampi(__float2int_rd(__fadd_rn(lam, 0.5f)), 0, n - 1);
}

// Bilinear lookup in slice k of the stack through its texture view (the
// cell layout of StackView).  Both coordinates are clamped to [0, R - 1]
// first: past an edge the clamp-to-edge footprint holds copies of the edge
// texel, and the clamped point reads the edge texel with weight 1 and its
// neighbour (in the next cell, or zero) with weight 0 -- the same value.
// CLAMP = false skips the clamp: only for a point whose coordinates are known
// to lie in [0, R - 1] already (the clamp would change nothing).
template <typename Fmt, bool CLAMP = true>
__device__ __forceinline__ float bilinear(const StackView& sv, int k, int n, int R, float tu,
                                          float tv, int* rec = nullptr) {
    if (rec) {
        rec[1] = clampi(__float2int_rd(tu), -1, R);
        rec[2] = clampi(__float2int_rd(tv), -1, R);
    }
    const float cu = CLAMP ? fminf(fmaxf(tu, 0.0f), (float)(R - 1)) : tu;
    const float fu = floorf(cu);
    const float wu = cu - fu;
    const float cv = CLAMP ? fminf(fmaxf(tv, 0.0f), (float)(R - 1)) : tv;
    const float fv = floorf(cv);
    const float wv = cv - fv;
    if (!(VI_BOUNDS_OK(kSiteStackTex, k, n) && VI_BOUNDS_OK(kSiteStackTex, (int)fv, R)))
        return 1.0f;
    // Gather takes the footprint's lower-left texel plus one (exact integers):
    // the cell's first column and row, plus one, are below 2^23.
    const float x1 = u2f((unsigned)((k & ((1 << sv.cells_log2) - 1)) * R + 1));
    const float y1 = u2f((unsigned)((k >> sv.cells_log2) * R + 1));
    float b00, b01, b10, b11;
    Fmt::gather(sv.tex, fu + x1, fv + y1, b00, b01, b10, b11);
    const float top = fmaf(wu, b01 - b00, b00);
    const float bot = fmaf(wu, b11 - b10, b10);
    return fmaf(wv, bot - top, top);
}

template <typename Fmt, bool CLAMP = true>
__device__ __forceinline__ float stack_lookup(const StackView& sv, int n, int R, float lam, float tu,
                                              float tv, int* rec = nullptr) {
    const int k = slice_index(lam, n);
    if (rec) rec[0] = k;
    return bilinear<Fmt, CLAMP>(sv, k, n, R, tu, tv, rec);
}

// Whether every point (tu + du, tv + dv) with |du|, |dv| <= reach, each
// coordinate added in binary32, lies in [0, R - 1]: then a lookup's clamp
// changes nothing.  Rounding is monotone, so the rounded sums lie between
// fl(t - reach) and fl(t + reach); t >= reach gives fl(t - reach) >= 0.  NaN
// coordinates fail the test (every comparison with NaN is false).
__device__ __forceinline__ bool lookups_inside(float tu, float tv, float reach, int R) {
    const float hi = (float)(R - 1);
    return tu >= reach && tv >= reach && __fadd_rn(tu, reach) <= hi &&
           __fadd_rn(tv, reach) <= hi;
}

}  // namespace vi
