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

// One block per brick builds the brick's footprint octets and its value range
// in one pass over the raw voxels.  The brick and its one-voxel apron on the
// high side (17^3 voxels, each coordinate clamped to the volume) are staged in
// shared memory; a thread then writes the octets of a column of 16 voxels
// along z (a warp's stores cover two contiguous rows) from the tile.  The
// octet of voxel (x, y, z) holds its footprint with the upper corners clamped,
// min(x + 1, nx - 1) and so on -- the staged tile's clamp -- and the union of
// the brick's octets is exactly the brick plus its clamped apron, so the
// brick's range is the min / max over the values of its octets.
// Staging loads a thread keeps in flight (the loop over the tile is unrolled by
// it).  8 measured fastest: 256^3 u16 in 57.6 us (71.5 us not unrolled, 58.3
// us at 4), 512^3 in 427 us (519, 434).
#ifndef VI_GRID_STAGE_UNROLL
#define VI_GRID_STAGE_UNROLL 8
#endif
constexpr int kStageUnroll = VI_GRID_STAGE_UNROLL;
constexpr int kBrick = 1 << kBrickShift;
constexpr int kApron = kBrick + 1;
constexpr int kGridThreads = kBrick * kBrick;  // one thread per (x, y) of the brick
static_assert(kApron * kApron * kApron * sizeof(uint16_t) <= 48 * 1024 && kGridThreads <= 1024,
              "volume_grid_kernel stages a brick and its apron in static shared memory and "
              "runs a thread per (x, y): bricks of at most 16^3 voxels");

template <typename VoxT>
__device__ __forceinline__ typename Octet<VoxT>::V pack_octet(const unsigned c[8]) {
    if constexpr (sizeof(VoxT) == 2) {
        return make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16), c[4] | (c[5] << 16),
                          c[6] | (c[7] << 16));
    } else {
        return make_uint2(c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24),
                          c[4] | (c[5] << 8) | (c[6] << 16) | (c[7] << 24));
    }
}

template <typename VoxT>
__global__ void __launch_bounds__(kGridThreads)
    volume_grid_kernel(const VoxT* __restrict__ raw, int nx, int ny, int nz, int nbx, int nby,
                       typename Octet<VoxT>::V* __restrict__ oct, uint32_t* __restrict__ range) {
    __shared__ VoxT tile[kApron][kApron][kApron];  // [z][y][x]
    __shared__ uint32_t part_lo[kGridThreads / 32], part_hi[kGridThreads / 32];
    const int b = blockIdx.x;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    [[maybe_unused]] const size_t total = (size_t)nx * ny * nz;  // the checked build's bound
#pragma unroll kStageUnroll
    for (int t = threadIdx.x; t < kApron * kApron * kApron; t += kGridThreads) {
        const int x = t % kApron, y = (t / kApron) % kApron, z = t / (kApron * kApron);
        const size_t at = ((size_t)min(z0 + z, nz - 1) * ny + min(y0 + y, ny - 1)) * nx +
                          min(x0 + x, nx - 1);
        tile[z][y][x] = VI_BOUNDS_OK(kSiteRaw, at, (long long)total) ? raw[at] : VoxT(0);
    }
    __syncthreads();
    const int tx = threadIdx.x % kBrick, ty = threadIdx.x / kBrick;
    const int gx = x0 + tx, gy = y0 + ty;
    uint32_t lo = 0xffffu, hi = 0u;
    if (gx < nx && gy < ny) {
        const int zn = min(kBrick, nz - z0);
        for (int z = 0; z < zn; ++z) {
            const unsigned c[8] = {tile[z][ty][tx],         tile[z][ty][tx + 1],
                                   tile[z][ty + 1][tx],     tile[z][ty + 1][tx + 1],
                                   tile[z + 1][ty][tx],     tile[z + 1][ty][tx + 1],
                                   tile[z + 1][ty + 1][tx], tile[z + 1][ty + 1][tx + 1]};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                lo = min(lo, (uint32_t)c[k]);
                hi = max(hi, (uint32_t)c[k]);
            }
            const size_t id = ((size_t)(z0 + z) * ny + gy) * nx + gx;
            if (VI_BOUNDS_OK(kSiteGrid, id, (long long)total)) oct[id] = pack_octet<VoxT>(c);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        part_lo[threadIdx.x >> 5] = lo;
        part_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        lo = threadIdx.x < kGridThreads / 32 ? part_lo[threadIdx.x] : 0xffffu;
        hi = threadIdx.x < kGridThreads / 32 ? part_hi[threadIdx.x] : 0u;
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (threadIdx.x == 0) range[b] = (lo << 16) | hi;
    }
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

cudaError_t launch_volume_grid(const void* raw, int nx, int ny, int nz, int voxel_type,
                               void* octets, uint32_t* range, cudaStream_t s) {
    const int nbx = (nx + kBrick - 1) >> kBrickShift;
    const int nby = (ny + kBrick - 1) >> kBrickShift;
    const int nbz = (nz + kBrick - 1) >> kBrickShift;
    const unsigned blocks = (unsigned)nbx * nby * nbz;
    if (voxel_type == 0)
        volume_grid_kernel<uint8_t><<<blocks, kGridThreads, 0, s>>>(
            static_cast<const uint8_t*>(raw), nx, ny, nz, nbx, nby, static_cast<uint2*>(octets),
            range);
    else
        volume_grid_kernel<uint16_t><<<blocks, kGridThreads, 0, s>>>(
            static_cast<const uint16_t*>(raw), nx, ny, nz, nbx, nby,
            static_cast<uint4*>(octets), range);
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
