// vi_grid.cu -- brick occupancy for exact empty-space skipping.
//
// The volume is cut into bricks of 2^kBrickShift voxels per axis (16^3).  For each brick the value range
// over its voxels plus a one-voxel apron on the high side (the voxels a
// trilinear footprint whose lower corner lies in the brick can touch) is kept;
// it changes only with the volume.  From it and the transfer function, a flag
// says whether any value in that range can map to alpha > 0: the TF entries a
// lookup of such a value can touch are a contiguous range, and a prefix count
// of entries with alpha > 0 answers that in O(1).  A sample whose footprint
// starts in an unflagged brick has alpha exactly 0 -- a trilinear value lies
// within its corners' range, and a lerp of two zero entries is zero -- so the
// sweep and the march skip its gather without changing any result.
#include <cmath>

#include "vi_device.cuh"

namespace vi {

namespace {

template <typename VoxT>
__global__ void brick_range_kernel(const VoxT* __restrict__ vol, int nx, int ny, int nz, int nbx,
                                   int nby, int nbz, uint32_t* __restrict__ range) {
    // One warp per brick: the lanes stride over the brick's voxels (x fastest,
    // so a row's loads are coalesced) and combine their extremes at the end.
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nbx * nby * nbz) return;  // the whole warp leaves together
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx << kBrickShift, y0 = by << kBrickShift, z0 = bz << kBrickShift;
    // The brick plus a one-voxel apron on the high side, clamped to the volume.
    const int wx = min(x0 + (1 << kBrickShift), nx - 1) - x0 + 1;
    const int wy = min(y0 + (1 << kBrickShift), ny - 1) - y0 + 1;
    const int wz = min(z0 + (1 << kBrickShift), nz - 1) - z0 + 1;
    uint32_t lo = 0xffffu, hi = 0u;
    for (int t = lane; t < wx * wy * wz; t += 32) {
        const int x = t % wx, yz = t / wx, y = yz % wy, z = yz / wy;
        const size_t at = ((size_t)(z0 + z) * ny + (y0 + y)) * nx + (x0 + x);
        if (!VI_BOUNDS_OK(kSiteRaw, at, (long long)nx * ny * nz)) continue;
        const uint32_t v = vol[at];
        lo = min(lo, v);
        hi = max(hi, v);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) range[b] = (lo << 16) | hi;
}

__global__ void brick_flag_kernel(const uint32_t* __restrict__ range, int nbricks,
                                  const int* __restrict__ lit_prefix, int M, double vmin,
                                  double scale, uint8_t* __restrict__ flags) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbricks) return;
    const double lo = (double)(range[b] >> 16), hi = (double)(range[b] & 0xffffu);
    // Entries a lookup of a value in [lo, hi] can read, widened by one on each
    // side to cover the binary32 rounding of the TF coordinate.
    long e_lo = (long)floor((lo - vmin) * scale) - 1;
    long e_hi = (long)floor((hi - vmin) * scale) + 2;
    e_lo = e_lo < 0 ? 0 : (e_lo > M - 2 ? M - 2 : e_lo);
    e_hi = e_hi < 1 ? 1 : (e_hi > M - 1 ? M - 1 : e_hi);
    if (!(VI_BOUNDS_OK(kSiteGrid, e_lo, M + 1) && VI_BOUNDS_OK(kSiteGrid, e_hi + 1, M + 1)))
        return;
    flags[b] = (lit_prefix[e_hi + 1] - lit_prefix[e_lo]) > 0 ? 1 : 0;
}

}  // namespace

cudaError_t launch_brick_range(const void* raw, int nx, int ny, int nz, int voxel_type,
                               uint32_t* range, cudaStream_t s) {
    const int nbx = (nx + (1 << kBrickShift) - 1) >> kBrickShift;
    const int nby = (ny + (1 << kBrickShift) - 1) >> kBrickShift;
    const int nbz = (nz + (1 << kBrickShift) - 1) >> kBrickShift;
    const int n = nbx * nby * nbz;
    const int threads = 256, blocks = (n + threads / 32 - 1) / (threads / 32);  // a warp per brick
    if (voxel_type == 0)
        brick_range_kernel<uint8_t><<<blocks, threads, 0, s>>>(
            static_cast<const uint8_t*>(raw), nx, ny, nz, nbx, nby, nbz, range);
    else
        brick_range_kernel<uint16_t><<<blocks, threads, 0, s>>>(
            static_cast<const uint16_t*>(raw), nx, ny, nz, nbx, nby, nbz, range);
    return cudaGetLastError();
}

namespace {

// One thread per voxel: gather its 2 x 2 x 2 footprint (clamped) into an octet.
template <typename VoxT>
__global__ void build_octets_kernel(const VoxT* __restrict__ raw, int nx, int ny, int nz,
                                    typename Octet<VoxT>::V* __restrict__ oct) {
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)nx * ny * nz;
    if (id >= total) return;
    const int x = (int)(id % nx), y = (int)((id / nx) % ny), z = (int)(id / ((size_t)nx * ny));
    const int x1 = min(x + 1, nx - 1), y1 = min(y + 1, ny - 1), z1 = min(z + 1, nz - 1);
    auto at = [&](int xx, int yy, int zz) -> unsigned {
        const size_t i = ((size_t)zz * ny + yy) * nx + xx;
        if (!VI_BOUNDS_OK(kSiteRaw, i, (long long)total)) return 0u;
        return raw[i];
    };
    const unsigned c000 = at(x, y, z), c001 = at(x1, y, z), c010 = at(x, y1, z), c011 = at(x1, y1, z);
    const unsigned c100 = at(x, y, z1), c101 = at(x1, y, z1), c110 = at(x, y1, z1), c111 = at(x1, y1, z1);
    if constexpr (sizeof(VoxT) == 2) {
        oct[id] = make_uint4(c000 | (c001 << 16), c010 | (c011 << 16), c100 | (c101 << 16),
                             c110 | (c111 << 16));
    } else {
        oct[id] = make_uint2(c000 | (c001 << 8) | (c010 << 16) | (c011 << 24),
                             c100 | (c101 << 8) | (c110 << 16) | (c111 << 24));
    }
}

}  // namespace

cudaError_t launch_build_octets(const void* raw, int nx, int ny, int nz, int voxel_type,
                                void* octets, cudaStream_t s) {
    const size_t total = (size_t)nx * ny * nz;
    const unsigned threads = 256;
    const size_t blocks = (total + threads - 1) / threads;
    if (voxel_type == 0)
        build_octets_kernel<uint8_t><<<(unsigned)blocks, threads, 0, s>>>(
            static_cast<const uint8_t*>(raw), nx, ny, nz, static_cast<uint2*>(octets));
    else
        build_octets_kernel<uint16_t><<<(unsigned)blocks, threads, 0, s>>>(
            static_cast<const uint16_t*>(raw), nx, ny, nz, static_cast<uint4*>(octets));
    return cudaGetLastError();
}

cudaError_t launch_brick_flags(const uint32_t* range, int nbricks, const int* lit_prefix, int M,
                               float vmin, float vmax, uint8_t* flags, cudaStream_t s) {
    const double scale = (double)(M - 1) / ((double)vmax - (double)vmin);
    const int threads = 256, blocks = (nbricks + threads - 1) / threads;
    brick_flag_kernel<<<blocks, threads, 0, s>>>(range, nbricks, lit_prefix, M, (double)vmin,
                                                 scale, flags);
    return cudaGetLastError();
}

#if VI_DEBUG_BOUNDS
VI_DEBUG_RECORD_ACCESSOR(debug_record_grid)
#endif

}  // namespace vi
