// vi_sweep.cu -- the light-space sweep (Section 3.2.1, Algorithm 1).
//
// One thread per light texel column (i, j).  The column walks the n slice
// planes from the one nearest the light, carrying the transmittance T in an
// FP32 register: it stores T into buffer k (the light arriving at plane k),
// then applies the back-to-front blend of Eq. 4 to a scalar transmittance,
// T <- T (1 - alpha_k).  All n slices come out of one launch (the paper's
// multi-slice-per-pass future work), with no framebuffer read-back.
//
// Memory: the volume is read through the read-only path (it fits in L2 for the
// sizes this targets).  A warp covers an 8 x 4 tile of texels, so its 32
// sample points form a compact patch of the slice plane and its trilinear
// footprints share sectors; each store of slice k writes four 32-byte row
// segments (FP32).  A point in a brick that cannot yield alpha > 0 skips the
// gather.  The transfer function's alpha column is staged in shared memory.
#include "vi_device.cuh"

namespace vi {

namespace {

constexpr int kSweepBX = 32, kSweepBY = 8;

template <typename VoxT, typename Fmt>
__global__ void __launch_bounds__(kSweepBX* kSweepBY)
    sweep_kernel(const SweepParams p) {
    extern __shared__ float s_alpha[];
    const int tid = threadIdx.x;
    for (int e = tid; e < p.M; e += kSweepBX * kSweepBY) s_alpha[e] = p.tf[e].w;
    __syncthreads();

    // Block tile 32 x 8 texels; warp w covers columns 8 (w % 4) .. +7, rows
    // 4 (w / 4) .. +3.
    const LightFrame& lt = p.lt;
    const int lane = tid & 31, warp = tid >> 5;
    const int i = blockIdx.x * kSweepBX + (warp & 3) * 8 + (lane & 7);
    const int j = blockIdx.y * kSweepBY + (warp >> 2) * 4 + (lane >> 3);
    if (i >= lt.R || j >= lt.R) return;

    // World position of texel (i, j) on the plane through the centre.
    float qi = __fdiv_rn((float)(2 * i + 1), (float)lt.R);
    float qj = __fdiv_rn((float)(2 * j + 1), (float)lt.R);
    float u = __fmul_rn(__fsub_rn(qi, 1.0f), lt.h);
    float v = __fmul_rn(__fsub_rn(qj, 1.0f), lt.h);
    float base0 = __fmaf_rn(v, lt.V[0], __fmaf_rn(u, lt.U[0], 0.5f));
    float base1 = __fmaf_rn(v, lt.V[1], __fmaf_rn(u, lt.U[1], 0.5f));
    float base2 = __fmaf_rn(v, lt.V[2], __fmaf_rn(u, lt.U[2], 0.5f));

    typename Fmt::T* out = static_cast<typename Fmt::T*>(p.stack) + (size_t)j * lt.R + i;
    const size_t slice = (size_t)lt.R * (size_t)lt.R;
    float T = 1.0f;
    for (int k = 0; k < lt.n; ++k) {
        float dk = __fmaf_rn((float)k, lt.dL, lt.min);
        float sk = __fsub_rn(dk, lt.Lc);
        float P0 = __fmaf_rn(sk, lt.L[0], base0);
        float P1 = __fmaf_rn(sk, lt.L[1], base1);
        float P2 = __fmaf_rn(sk, lt.L[2], base2);
        float alpha = 0.0f;
        VoxelCoord vc;
        if (P0 >= 0.0f && P0 <= 1.0f && P1 >= 0.0f && P1 <= 1.0f && P2 >= 0.0f && P2 <= 1.0f &&
            brick_may_be_lit(p.grid, vc = voxel_coord(p.vol, P0, P1, P2))) {
            float val = trilinear_fetch<VoxT>(p.vol, vc);
            int e;
            float f;
            tf_coord(val, p.tf_vmin, p.tf_scale, p.M, &e, &f);
            float a0 = s_alpha[e];
            alpha = fmaf(f, s_alpha[e + 1] - a0, a0);
            if (p.opacity_correction)
                alpha = 1.0f - exp2f(p.spacing_vox * log2f(fmaxf(1.0f - alpha, 0.0f)));
        }
        float stored = T;
        if (p.comp_n != 0.0f) stored = fminf(1.0f, T * powf(1.0f + alpha, p.comp_n));
        out[(size_t)k * slice] = Fmt::pack(stored);
        T *= (1.0f - alpha);
    }
}

template <typename VoxT, typename Fmt>
cudaError_t launch_typed(const SweepParams& p, cudaStream_t s) {
    dim3 block(kSweepBX * kSweepBY);
    dim3 grid((p.lt.R + kSweepBX - 1) / kSweepBX, (p.lt.R + kSweepBY - 1) / kSweepBY);
    size_t smem = (size_t)p.M * sizeof(float);
    sweep_kernel<VoxT, Fmt><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename VoxT>
cudaError_t launch_fmt(const SweepParams& p, int format, cudaStream_t s) {
    switch (format) {
        case 0: return launch_typed<VoxT, F32>(p, s);
        case 1: return launch_typed<VoxT, F16>(p, s);
        case 2: return launch_typed<VoxT, BF16>(p, s);
        case 3: return launch_typed<VoxT, UNORM16>(p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_sweep(const SweepParams& p, int voxel_type, int format, cudaStream_t s) {
    if (voxel_type == 0) return launch_fmt<uint8_t>(p, format, s);
    return launch_fmt<uint16_t>(p, format, s);
}

}  // namespace vi
