// vi_api.cu -- context, validation, device memory and the C ABI of vi.h.
//
// Host-side set-up of the light (Eq. 8, the Eq. 9 ratio, the Eq. 10 frame)
// and of the camera runs in binary32 with the operation order documented in
// vi_internal.h.  This file must be compiled with -ffp-contract=off for the
// host compiler so that no a*b+c is fused behind our back.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "vi_context.h"

using vi::CameraFrame;
using vi::LightFrame;
using vi::MarchParams;
using vi::SweepParams;
using vi::BatchFrame;

namespace {

// ---------------------------------------------------------------------------
// binary32 index-path helpers (host).

float dot3(const float a[3], const float b[3]) {
    float p0 = a[0] * b[0];
    float p1 = a[1] * b[1];
    float p2 = a[2] * b[2];
    float s = p0 + p1;
    return s + p2;
}

void cross3(const float a[3], const float b[3], float o[3]) {
    float p, q;
    p = a[1] * b[2];
    q = a[2] * b[1];
    o[0] = p - q;
    p = a[2] * b[0];
    q = a[0] * b[2];
    o[1] = p - q;
    p = a[0] * b[1];
    q = a[1] * b[0];
    o[2] = p - q;
}

bool finite3(const float v[3]) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

// Light frame for n slices of R x R texels (Eq. 8, Section 3.2.1, Eq. 9, Eq. 10).
int light_frame(const float dir[3], int n, int R, LightFrame* o) {
    float len = std::sqrt(dot3(dir, dir));
    if (!(len > 0.0f) || !std::isfinite(len)) return VI_EINVAL;
    std::memset(o, 0, sizeof(*o));
    for (int a = 0; a < 3; ++a) o->L[a] = dir[a] / len;
    // Eq. 8: the extreme vertices of [0,1]^3 take the negative (positive)
    // components of L; the sum is formed in axis order.
    float m[3], M[3];
    for (int a = 0; a < 3; ++a) {
        m[a] = o->L[a] < 0.0f ? o->L[a] : 0.0f;
        M[a] = o->L[a] > 0.0f ? o->L[a] : 0.0f;
    }
    float mn = m[0] + m[1];
    mn = mn + m[2];
    float mx = M[0] + M[1];
    mx = mx + M[2];
    o->min = mn;
    o->max = mx;
    float span = mx - mn;
    o->dL = span / (float)n;
    o->kappa = (float)n / span;
    const float c3[3] = {0.5f, 0.5f, 0.5f};
    o->Lc = dot3(o->L, c3);
    // Light view: U from the world axis least aligned with L, V = L x U.
    int ax = 0;
    if (std::fabs(o->L[1]) < std::fabs(o->L[ax])) ax = 1;
    if (std::fabs(o->L[2]) < std::fabs(o->L[ax])) ax = 2;
    float w[3];
    for (int b = 0; b < 3; ++b) {
        float e = (b == ax) ? 1.0f : 0.0f;
        float p = o->L[ax] * o->L[b];
        w[b] = e - p;
    }
    float wn = std::sqrt(dot3(w, w));
    for (int b = 0; b < 3; ++b) o->U[b] = w[b] / wn;
    cross3(o->L, o->U, o->V);
    // Light projection: a square of half extent sqrt(3)/2 about the centre.
    o->h = 0x1.bb67aep-1f;
    float two_h = 2.0f * o->h;
    o->sigma = (float)R / two_h;
    o->rho0 = 0.5f * (float)(R - 1);
    o->n = n;
    o->R = R;
    return VI_OK;
}

// Point light at pos (f4): the frame of a directional light along the axis
// a = (c - pos) / |c - pos|, then depths from pos (min / max over the cube's
// vertices of V.a - pos.a), Lc = 0, and a perspective texel grid of tangent
// half extent h = sqrt(3)/2 / sqrt(|c - pos|^2 - 3/4).  |c - pos| >= 1.
int point_light_frame(const float pos[3], int n, int R, LightFrame* o) {
    if (!finite3(pos)) return VI_EINVAL;
    float q[3] = {0.5f - pos[0], 0.5f - pos[1], 0.5f - pos[2]};
    float dc2 = dot3(q, q);
    float dc = std::sqrt(dc2);
    if (!(dc >= 1.0f) || !std::isfinite(dc)) return VI_EINVAL;
    int rc = light_frame(q, n, R, o);
    if (rc) return rc;
    o->point = 1;
    for (int a = 0; a < 3; ++a) o->P[a] = pos[a];
    float pa = dot3(o->L, pos);
    // min / max over the vertices of V.a - pos.a: the extreme vertices take the
    // negative (positive) components of a, summed in axis order.
    float m[3], M[3];
    for (int a = 0; a < 3; ++a) {
        m[a] = o->L[a] < 0.0f ? o->L[a] : 0.0f;
        M[a] = o->L[a] > 0.0f ? o->L[a] : 0.0f;
    }
    float mn = m[0] + m[1];
    mn = mn + m[2];
    float mx = M[0] + M[1];
    mx = mx + M[2];
    o->min = mn - pa;
    o->max = mx - pa;
    float span = o->max - o->min;
    o->dL = span / (float)n;
    o->kappa = (float)n / span;
    o->Lc = 0.0f;
    const float hs = 0x1.bb67aep-1f;
    float hs2 = hs * hs;
    o->h = hs / std::sqrt(dc2 - hs2);
    float two_h = 2.0f * o->h;
    o->sigma = (float)R / two_h;
    return VI_OK;
}

int camera_frame(const vi_camera* cam, int W, int H, float step_vox, int nmax, CameraFrame* c) {
    if (!finite3(cam->eye) || !finite3(cam->target) || !finite3(cam->up)) return VI_EINVAL;
    std::memset(c, 0, sizeof(*c));
    float fw[3], r0[3];
    for (int a = 0; a < 3; ++a) fw[a] = cam->target[a] - cam->eye[a];
    float nf = std::sqrt(dot3(fw, fw));
    if (!(nf > 0.0f) || !std::isfinite(nf)) return VI_EINVAL;
    for (int a = 0; a < 3; ++a) c->f[a] = fw[a] / nf;
    cross3(c->f, cam->up, r0);
    float nr = std::sqrt(dot3(r0, r0));
    if (!(nr > 0.0f) || !std::isfinite(nr)) return VI_EINVAL;
    for (int a = 0; a < 3; ++a) c->r[a] = r0[a] / nr;
    cross3(c->r, c->f, c->u);
    for (int a = 0; a < 3; ++a) c->eye[a] = cam->eye[a];
    float aspect = (float)W / (float)H;
    if (cam->perspective) {
        if (!(cam->fovy_deg > 0.0f && cam->fovy_deg < 180.0f)) return VI_EINVAL;
        float th = (float)std::tan((double)cam->fovy_deg * (M_PI / 360.0));
        c->sx = th * aspect;
        c->sy = th;
    } else {
        if (!(cam->ortho_half_height > 0.0f) || !std::isfinite(cam->ortho_half_height))
            return VI_EINVAL;
        c->sx = cam->ortho_half_height * aspect;
        c->sy = cam->ortho_half_height;
    }
    c->perspective = cam->perspective ? 1 : 0;
    c->W = W;
    c->H = H;
    c->dt = step_vox / (float)nmax;
    c->inv_dt = 1.0f / c->dt;
    return VI_OK;
}

// Texel-slices from which the sweep runs in lockstep: VI_SWEEP_LOCKSTEP_MIN,
// or the environment variable of that name when it holds a number (a test
// sets it to run the lockstep kernel on stacks small enough to compare with
// an FP64 stack element by element).
double lockstep_threshold() {
    const char* env = std::getenv("VI_SWEEP_LOCKSTEP_MIN");
    if (env && *env) {
        char* end = nullptr;
        const double v = std::strtod(env, &end);
        if (end != env && v >= 0.0) return v;
    }
    return (double)VI_SWEEP_LOCKSTEP_MIN;
}

size_t voxel_bytes(int t) { return t == VI_U8 ? 1 : 2; }
size_t format_bytes(int f) { return f == VI_F32 ? 4 : 2; }

int nmax(const vi_ctx* c) { return std::max(c->vr->nx, std::max(c->vr->ny, c->vr->nz)); }

static_assert(vi::kMaxShells == VI_MAX_SHELLS, "shell limit differs between header and kernels");
static_assert(vi::kDepthMax == VI_DEPTH_MAX, "depth cap differs between header and kernels");

vi_build_opts default_build_opts() {
    vi_build_opts o;
    o.format = VI_F32;
    o.cone_half_angle_deg = 15.0f;
    o.shell_radius_vox = 1.0f;
    o.opacity_correction = 0;
    o.comp_n = 0.0f;
    o.quantity = VI_TRANSMITTANCE;
    o.shell_count = 1;
    return o;
}

vi_render_opts default_render_opts() {
    vi_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.ert = 2.0f;
    return o;
}

int cuda_fail(vi_ctx* c, cudaError_t e) {
    if (e == cudaSuccess) return VI_OK;
    c->sticky = VI_ECUDA;
    return VI_ECUDA;
}

// Grow a device buffer to `bytes` under the context's budget.
int ensure(vi_ctx* c, void** p, size_t* cap, size_t bytes) {
    if (c->capturing && !(bytes <= *cap && *p)) return VI_ESTATE;  // see ctx_reserve
    return vi_detail::ensure_mem(&c->used, c->budget, p, cap, bytes, c->stream, c->pool);
}

void release(vi_ctx* c, void** p, size_t* cap) {
    vi_detail::release_mem(&c->used, p, cap, c->stream, c->pool);
}

// Common prologue of every call on a context.
int enter(vi_ctx* c) {
    if (!c) return VI_EINVAL;
    if (c->sticky != VI_OK) return c->sticky;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    return VI_OK;
}

void mark_stale(vi_ctx* c) { c->stack_valid = false; }

void destroy_stack_textures(vi_ctx* c) {
    if (c->ntex) cudaDestroyTextureObject(c->sview.tex);
    c->ntex = 0;
}

// Pitched stack for n slices of R x R texels of format fmt in the cell layout
// of vi::StackView, and its texture view (rebuilt, and the memory zeroed, only
// when the shape, format or buffer changes).
int setup_stack(vi_ctx* c, int n, int R, int fmt) {
    vi_detail::StackLayout L;
    int rc = vi_detail::stack_layout(c->device, n, R, format_bytes(fmt), &L);
    if (rc) return rc == VI_ECUDA ? cuda_fail(c, cudaGetLastError()) : rc;
    void* before = c->stack_mem;
    rc = ensure(c, &c->stack_mem, &c->stack_cap, L.bytes);
    if (rc) return rc;
    if (before != c->stack_mem) c->stack_valid = false;
    void* base = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(c->stack_mem) + 511) &
                                         ~(uintptr_t)511);
    const bool same = before == c->stack_mem && c->stack == base && c->row_pitch == L.pitch &&
                      c->ntex == 1 && c->sview.cells_log2 == L.cells_log2 &&
                      c->stack_valid_shape_n == n && c->stack_valid_shape_R == R &&
                      c->stack_valid_shape_fmt == fmt;
    c->stack = base;
    c->row_pitch = L.pitch;
    if (same) return VI_OK;
    c->stack_valid = false;
    destroy_stack_textures(c);
    // Lookups read outside a slice only with weight 0, but that must be a
    // finite number: zero what no sweep writes (and everything, for brevity).
    cudaError_t e = cudaMemsetAsync(base, 0, L.rows * L.pitch, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    cudaResourceDesc res;
    std::memset(&res, 0, sizeof(res));
    res.resType = cudaResourceTypePitch2D;
    res.res.pitch2D.devPtr = base;
    // The texture unit widens binary16 texels exactly and reads UNORM16 texels
    // as q / 65535 (normalised read mode); BF16 texels are read as raw bits.
    res.res.pitch2D.desc = fmt == VI_F32   ? cudaCreateChannelDesc<float>()
                           : fmt == VI_F16 ? cudaCreateChannelDescHalf()
                                           : cudaCreateChannelDesc<unsigned short>();
    res.res.pitch2D.width = ((size_t)R) << L.cells_log2;
    res.res.pitch2D.height = L.rows;
    res.res.pitch2D.pitchInBytes = L.pitch;
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof(td));
    td.addressMode[0] = cudaAddressModeClamp;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = fmt == VI_UNORM16 ? cudaReadModeNormalizedFloat : cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&c->sview.tex, &res, &td, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->ntex = 1;
    c->sview.cells_log2 = L.cells_log2;
    c->stack_valid_shape_n = n;
    c->stack_valid_shape_R = R;
    c->stack_valid_shape_fmt = fmt;
    return VI_OK;
}

int nbricks(const vi_ctx* c) { return c->vr->nbx * c->vr->nby * c->vr->nbz; }

vi::VolumeView volume_view(const vi_ctx* c) {
    const VolumeRes* r = c->vr;
    vi::VolumeView v;
    v.data = r->pairs;
    v.nx = r->nx;
    v.ny = r->ny;
    v.nz = r->nz;
    v.nbx = r->nbx;
    v.nby = r->nby;
    v.nbz = r->nbz;
    v.fnx = (float)r->nx;
    v.fny = (float)r->ny;
    v.fnz = (float)r->nz;
    return v;
}

vi::GridView grid_view(const vi_ctx* c) {
    vi::GridView g;
    g.flags = c->bflags;
    g.skip = c->bflags ? c->bflags + nbricks(c) : nullptr;
    g.nbx = c->vr->nbx;
    g.nby = c->vr->nby;
    g.cnx = c->vr->nbx * vi::kCellsPerBrick;
    g.cny = c->vr->nby * vi::kCellsPerBrick;
#if VI_DEBUG_BOUNDS
    g.nbz = c->vr->nbz;
    g.cnz = c->vr->nbz * vi::kCellsPerBrick;
#endif
    return g;
}

// Brick flags from the current brick ranges and TF (both must be present).
int refresh_flags(vi_ctx* c) {
    c->flags_ok = false;
    if (!c->vr->brange || !c->tfcnt || c->vr->vtype < 0 || !c->tf) return VI_OK;
    // Brick flags (a byte per brick), then the cells' skip distances and the
    // passes' scratch (a byte per cell each).
    const size_t nb = (size_t)nbricks(c);
    const size_t nc = nb * vi::kCellsPerBrick * vi::kCellsPerBrick * vi::kCellsPerBrick;
    int rc = ensure(c, reinterpret_cast<void**>(&c->bflags), &c->bflags_cap, nb + 2 * nc);
    if (rc) return rc;
    cudaError_t e = vi::launch_brick_flags(c->vr->brange, c->vr->nbx, c->vr->nby, c->vr->nbz,
                                           c->tfcnt, c->M, c->vmin, c->vmax, c->bflags,
                                           c->bflags + nb, c->bflags + nb + nc, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->launches += 5;
    c->flags_ok = true;
    return VI_OK;
}

int fill_march_params(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox,
                      const vi_render_opts* ro, MarchParams* p) {
    std::memset(p, 0, sizeof(*p));
    int rc = camera_frame(cam, W, H, step_vox, nmax(c), &p->cam);
    if (rc) return rc;
    p->vol = volume_view(c);
    p->grid = grid_view(c);
    p->tf = c->tf;
    p->M = c->M;
    p->tf_vmin = c->vmin;
    p->tf_scale = (float)(c->M - 1) / (c->vmax - c->vmin);
    if (c->lt_valid) p->lt = c->lt;  // else n = R = 0: no lookups
    p->stack = c->sview;
    const LightFrame& lt = p->lt;
    p->shells = c->bopts.shell_count > 1 ? c->bopts.shell_count : 1;
    p->shell_reach = 0.0f;
    if (c->mode == VI_SHELL && c->lt_valid) {
        // Shell q holds the six points S +- q r e_a, as light-space offsets.
        for (int q = 1; q <= p->shells; ++q) {
            float r = ((float)q * c->bopts.shell_radius_vox) / (float)nmax(c);
            for (int a = 0; a < 3; ++a) {
                float rl = r * lt.L[a];
                float ru = r * lt.U[a];
                float rv = r * lt.V[a];
                float off[3] = {rl * lt.kappa, ru * lt.sigma, rv * lt.sigma};
                for (int k = 0; k < 3; ++k) {
                    p->shell_off[q - 1][2 * a][k] = off[k];
                    p->shell_off[q - 1][2 * a + 1][k] = -off[k];
                }
                if (q == 1)
                    p->shell_reach = std::max(p->shell_reach,
                                              std::max(std::fabs(off[1]), std::fabs(off[2])));
            }
        }
    }
    for (int q = 1; q <= p->shells; ++q)
        p->shell_r[q - 1] = ((float)q * c->bopts.shell_radius_vox) / (float)nmax(c);
    p->tanphi = (float)std::tan((double)c->bopts.cone_half_angle_deg * (M_PI / 180.0));
    p->depth = c->bopts.quantity == VI_OPTICAL_DEPTH ? 1 : 0;
    p->slice_linear = ro->slice_filter == VI_SLICE_LINEAR ? 1 : 0;
    if (c->mode == VI_CONE && c->lt_valid) {
        // Ring n sits n slice spacings towards the light; radius n dL tan(phi).
        float tanphi = (float)std::tan((double)c->bopts.cone_half_angle_deg * (M_PI / 180.0));
        for (int q = 0; q < 2; ++q) {
            float dist = (float)(q + 1) * lt.dL;
            float radw = dist * tanphi;
            p->cone_rad[q] = radw * lt.sigma;
        }
        p->cone_thr = 1e-6f * lt.sigma;
    }
    p->ert = ro->ert;
    for (int k = 0; k < 4; ++k) p->bg[k] = ro->bg[k];
    for (int k = 0; k < 3; ++k) p->color[k] = c->color[k];
    p->ambient = ro->ambient;
    p->opacity_correction = ro->opacity_correction ? 1 : 0;
    p->step_vox = step_vox;
    p->counts = ro->sample_counts;
    p->lit = ro->lit_counts;
    p->block_threads = c->march_block;
    return VI_OK;
}

int check_render_inputs(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox,
                        const vi_render_opts* ro) {
    if (!cam || W < 0 || H < 0) return VI_EINVAL;
    if ((long long)W * (long long)H > 0x7fffffffLL) return VI_EINVAL;
    if (!(step_vox >= 1e-3f && step_vox <= 1e3f)) return VI_EINVAL;
    if (!std::isfinite(ro->ert) || !std::isfinite(ro->ambient)) return VI_EINVAL;
    if (ro->slice_filter != VI_SLICE_NEAREST && ro->slice_filter != VI_SLICE_LINEAR)
        return VI_EINVAL;
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(ro->bg[k])) return VI_EINVAL;
    if (c->vr->vtype < 0 || !c->tf || !c->flags_ok || c->mode < 0) return VI_ESTATE;
    if (c->mode != VI_NONE && !c->stack_valid) return VI_ESTATE;
    // A ray crosses at most sqrt(3) of the cube: cap its sample count at 2^24.
    if (1.7320509 * (double)nmax(c) / (double)step_vox > 16777216.0) return VI_EINVAL;
    return VI_OK;
}

}  // namespace

namespace vi_detail {

int stack_layout(int device, int n, int R, size_t esize, StackLayout* out) {
    int max_h = 0, max_w = 0, max_pitch = 0;
    cudaError_t e = cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxTexture2DLinearHeight, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture2DLinearWidth, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxTexture2DLinearPitch, device);
    if (e != cudaSuccess) return VI_ECUDA;
    if (n < 1 || R < 1 || R > max_w || R > max_h) return VI_EINVAL;
    // Cells a row of cells can hold: width and pitch limits.
    auto fits_width = [&](int lg) {
        return lg < 30 && ((size_t)R << lg) <= (size_t)max_w &&
               ((((size_t)R * esize) << lg) + 511) / 512 * 512 <= (size_t)max_pitch;
    };
    auto rows_for = [&](int lg) { return (((size_t)n + ((size_t)1 << lg) - 1) >> lg) * (size_t)R; };
    int lg = 0;
    while ((((size_t)1 << lg) << lg) < (size_t)n && fits_width(lg + 1)) ++lg;
    while (rows_for(lg) > (size_t)max_h && fits_width(lg + 1)) ++lg;
    if (rows_for(lg) > (size_t)max_h) return VI_EINVAL;
    out->cells_log2 = lg;
    out->rows = rows_for(lg);
    out->pitch = ((((size_t)R * esize) << lg) + 511) / 512 * 512;
    out->bytes = out->rows * out->pitch + 512;
    return VI_OK;
}

int ensure_mem(size_t* used, size_t budget, void** p, size_t* cap, size_t bytes, cudaStream_t s,
               cudaMemPool_t pool) {
    if (bytes <= *cap && *p) return VI_OK;
    size_t after = *used - *cap + bytes;
    if (budget && after > budget) return VI_ENOMEM;
    void* q = nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, bytes, pool, s) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VI_ENOMEM;
    }
    if (*p) {
        if (pool) {
            cudaFreeAsync(*p, s);
        } else {
            cudaStreamSynchronize(s);
            cudaFree(*p);
        }
    }
    *p = q;
    *used = after;
    *cap = bytes;
    return VI_OK;
}

void release_mem(size_t* used, void** p, size_t* cap, cudaStream_t s, cudaMemPool_t pool) {
    if (*p) {
        if (pool) cudaFreeAsync(*p, s);
        else cudaFree(*p);
    }
    *used -= *cap;
    *p = nullptr;
    *cap = 0;
}

size_t volume_bytes(int dtype, int nx, int ny, int nz) {
    const size_t raw = (size_t)nx * (size_t)ny * (size_t)nz * voxel_bytes(dtype);
    size_t bricks = 0, cells = 0;
    vi::grid_counts(nx, ny, nz, &bricks, &cells);
    return raw + vi::pair_brick_bytes(nx, ny, nz, voxel_bytes(dtype)) +
           (bricks + cells) * sizeof(uint32_t);
}

int volume_load(VolumeRes* v, size_t* used, size_t budget, const void* data, int dtype, int nx,
                int ny, int nz, int data_on_device, cudaStream_t s, uint64_t* launches) {
    const size_t bytes = (size_t)nx * (size_t)ny * (size_t)nz * voxel_bytes(dtype);
    constexpr int B = 1 << vi::kBrickShift;
    const int nbx = (nx + B - 1) / B, nby = (ny + B - 1) / B, nbz = (nz + B - 1) / B;
    // Check the whole footprint first, so a refusal leaves the old volume intact.
    const size_t pair_bytes = vi::pair_brick_bytes(nx, ny, nz, voxel_bytes(dtype));
    size_t nbricks = 0, ncells = 0;
    vi::grid_counts(nx, ny, nz, &nbricks, &ncells);
    const size_t range_bytes = (nbricks + ncells) * sizeof(uint32_t);  // bricks, then cells
    const size_t have = std::max(v->raw_cap, bytes) - v->raw_cap +
                        std::max(v->pairs_cap, pair_bytes) - v->pairs_cap +
                        std::max(v->brange_cap, range_bytes) - v->brange_cap;
    if (budget && *used + have > budget) return VI_ENOMEM;
    int rc = ensure_mem(used, budget, &v->raw, &v->raw_cap, bytes, s, v->pool);
    if (rc) return rc;
    rc = ensure_mem(used, budget, &v->pairs, &v->pairs_cap, pair_bytes, s, v->pool);
    if (rc) return rc;
    rc = ensure_mem(used, budget, reinterpret_cast<void**>(&v->brange), &v->brange_cap,
                    range_bytes, s, v->pool);
    if (rc) return rc;
    v->vtype = -1;
    cudaError_t e = cudaMemcpyAsync(v->raw, data, bytes,
                                    data_on_device ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyHostToDevice,
                                    s);
    if (e == cudaSuccess)
        e = vi::launch_volume_grid(v->raw, nx, ny, nz, dtype, v->pairs, v->brange, s);
    if (e != cudaSuccess) return VI_ECUDA;
    if (launches) *launches += 1;
    v->vtype = dtype;
    v->nx = nx;
    v->ny = ny;
    v->nz = nz;
    v->nbx = nbx;
    v->nby = nby;
    v->nbz = nbz;
    return VI_OK;
}

void volume_release(VolumeRes* v, size_t* used, cudaStream_t s) {
    release_mem(used, &v->raw, &v->raw_cap, s, v->pool);
    release_mem(used, &v->pairs, &v->pairs_cap, s, v->pool);
    release_mem(used, reinterpret_cast<void**>(&v->brange), &v->brange_cap, s, v->pool);
    v->vtype = -1;
}

int ctx_bind_volume(vi_ctx* c, VolumeRes* v, bool keep_stack) {
    int rc = enter(c);
    if (rc) return rc;
    if (!v || v->vtype < 0) return VI_EINVAL;
    if (!keep_stack || c->vr != v) mark_stale(c);
    c->vr = v;
    c->flags_ok = false;
    return refresh_flags(c);
}

void ctx_trim(vi_ctx* c) {
    cudaStreamSynchronize(c->stream);
    destroy_stack_textures(c);
    release(c, &c->stack_mem, &c->stack_cap);
    release(c, reinterpret_cast<void**>(&c->out), &c->out_cap);
    c->stack = nullptr;
    mark_stale(c);
}

int ctx_render_async(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox, float* out,
                     int out_on_device, const vi_render_opts* opts) {
    int rc = enter(c);
    if (rc) return rc;
    vi_render_opts ro = opts ? *opts : default_render_opts();
    rc = check_render_inputs(c, cam, W, H, step_vox, &ro);
    if (rc) return rc;
    if (W == 0 || H == 0) return VI_OK;
    if (!out) return VI_EINVAL;
    MarchParams p;
    rc = fill_march_params(c, cam, W, H, step_vox, &ro, &p);
    if (rc) return rc;
    rc = ensure(c, reinterpret_cast<void**>(&c->counter), &c->counter_cap, 256);
    if (rc) return rc;
    p.tile_counter = c->counter;
    size_t bytes = (size_t)W * (size_t)H * sizeof(float4);
    if (out_on_device) {
        p.out = reinterpret_cast<float4*>(out);
    } else {
        rc = ensure(c, reinterpret_cast<void**>(&c->out), &c->out_cap, bytes);
        if (rc) return rc;
        p.out = c->out;
    }
    cudaError_t e = vi::launch_march(p, c->vr->vtype, c->bopts.format, c->mode, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    ++c->launches;
    if (!out_on_device) {
        e = cudaMemcpyAsync(out, c->out, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return VI_OK;
}

int ctx_batch_frame(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox, float* out,
                    int out_on_device, const vi_render_opts* opts, BatchFrame* b) {
    int rc = enter(c);
    if (rc) return rc;
    vi_render_opts ro = opts ? *opts : default_render_opts();
    rc = check_render_inputs(c, cam, W, H, step_vox, &ro);
    if (rc) return rc;
    if (W < 1 || H < 1 || !out) return VI_EINVAL;
    const int fmt = c->mode == VI_NONE ? VI_F32 : c->bopts.format;
    if ((fmt != VI_F32 && fmt != VI_F16) || c->bopts.quantity != VI_TRANSMITTANCE ||
        c->bopts.shell_count > 1 || c->light_point || ro.slice_filter != VI_SLICE_NEAREST)
        return VI_EINVAL;
    std::memset(b, 0, sizeof(*b));
    rc = fill_march_params(c, cam, W, H, step_vox, &ro, &b->p);
    if (rc) return rc;
    if (out_on_device) {
        b->p.out = reinterpret_cast<float4*>(out);
    } else {
        rc = ensure(c, reinterpret_cast<void**>(&c->out), &c->out_cap,
                    (size_t)W * (size_t)H * sizeof(float4));
        if (rc) return rc;
        b->p.out = c->out;
    }
    b->ready = c->ready;
    b->epoch = c->post_epoch ? c->post_epoch : 1u;  // never published: its first epoch
    b->tiles_x = (unsigned)(W + 3) / 4;
    b->kind = c->vr->vtype * 8 + fmt * 4 + c->mode;
    return VI_OK;
}

cudaError_t enqueue_batch(vi_ctx* const* ctxs, const BatchFrame* frames, int count,
                          unsigned long long wait_ns, int* const* status_dst, cudaStream_t s) {
    // Every frame's ready word is zero before the batch reads it, and the batch
    // starts after each context's last publication: streams share the GPU's
    // hardware work queues once there are more streams than queues, so a kernel
    // spinning on another stream's later work could hold up that very work.
    // The device-side wait stays as a bounded check (it returns at once here),
    // and runs out only for a context that never published.
    for (int f = 0; f < count; ++f) {
        cudaError_t e = cudaStreamWaitEvent(s, ctxs[f]->ready_event, 0);
        if (e == cudaSuccess && ctxs[f]->post_epoch)
            e = cudaStreamWaitEvent(s, ctxs[f]->posted_event, 0);
        if (e != cudaSuccess) return e;
    }
    return vi::enqueue_march_batch(frames, count, wait_ns, status_dst, s);
}

int ctx_reserve(vi_ctx* c, int build_stack, int n, int R, int fmt, int W, int H,
                int out_on_device) {
    int rc = enter(c);
    if (rc) return rc;
    if (build_stack) {
        if (n < 1 || R < 1 || fmt < VI_F32 || fmt > VI_UNORM16) return VI_EINVAL;
        rc = setup_stack(c, n, R, fmt);
        if (rc) return rc;
    }
    rc = ensure(c, reinterpret_cast<void**>(&c->counter), &c->counter_cap, 256);
    if (rc || out_on_device || W <= 0 || H <= 0) return rc;
    return ensure(c, reinterpret_cast<void**>(&c->out), &c->out_cap,
                  (size_t)W * (size_t)H * sizeof(float4));
}

}  // namespace vi_detail

extern "C" {

const char* vi_error_string(int status) {
    switch (status) {
        case VI_OK: return "ok";
        case VI_EINVAL: return "invalid argument";
        case VI_ENOMEM: return "out of memory (budget or device)";
        case VI_ESTATE: return "missing input or stale attenuation stack";
        case VI_ECUDA: return "CUDA error";
        case VI_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int vi_create(vi_ctx** out, int device, void* cuda_stream) {
    if (!out) return VI_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    if (device < 0 || device >= count) return VI_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    vi_ctx* c = new (std::nothrow) vi_ctx();
    if (!c) return VI_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->bopts = default_build_opts();
    // The ready word of batched frames: zeroed on the context's stream, and an
    // event after the zeroing that every batch waits for, so no batch reads the
    // freshly allocated word before it is zero.
    // It is a plain cudaMalloc of 256 bytes, outside the memory budget (a
    // context made for a server gets the server's pool only after this).
    if (cudaMalloc(reinterpret_cast<void**>(&c->ready), 256) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return VI_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&c->ready_event, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->posted_event, cudaEventDisableTiming) != cudaSuccess ||
        cudaMemsetAsync(c->ready, 0, 256, c->stream) != cudaSuccess ||
        cudaEventRecord(c->ready_event, c->stream) != cudaSuccess) {
        cudaGetLastError();
        if (c->ready_event) cudaEventDestroy(c->ready_event);
        if (c->posted_event) cudaEventDestroy(c->posted_event);
        cudaFree(c->ready);
        delete c;
        return VI_ECUDA;
    }
    *out = c;
    return VI_OK;
}

int vi_destroy(vi_ctx* c) {
    if (!c) return VI_EINVAL;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    vi_detail::volume_release(&c->own, &c->used, c->stream);
    release(c, reinterpret_cast<void**>(&c->tf), &c->tf_cap);
    destroy_stack_textures(c);
    release(c, &c->stack_mem, &c->stack_cap);
    release(c, reinterpret_cast<void**>(&c->out), &c->out_cap);
    release(c, reinterpret_cast<void**>(&c->trace), &c->trace_cap);
    release(c, reinterpret_cast<void**>(&c->tfcnt), &c->tfcnt_cap);
    release(c, reinterpret_cast<void**>(&c->bflags), &c->bflags_cap);
    release(c, reinterpret_cast<void**>(&c->counter), &c->counter_cap);
    cudaFree(c->ready);
    if (c->ready_event) cudaEventDestroy(c->ready_event);
    if (c->posted_event) cudaEventDestroy(c->posted_event);
    delete c;
    return VI_OK;
}

int vi_set_memory_budget(vi_ctx* c, size_t bytes) {
    if (!c) return VI_EINVAL;
    c->budget = bytes;
    return VI_OK;
}

int vi_load_volume(vi_ctx* c, const void* data, int dtype, int nx, int ny, int nz,
                   int data_on_device) {
    vi_detail::NvtxRange nvtx_range("vi_load_volume");
    int rc = enter(c);
    if (rc) return rc;
    if (!data || (dtype != VI_U8 && dtype != VI_U16)) return VI_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 65536 || ny > 65536 || nz > 65536) return VI_EINVAL;
    rc = vi_detail::volume_load(&c->own, &c->used, c->budget, data, dtype, nx, ny, nz,
                                data_on_device, c->stream, &c->launches);
    if (rc == VI_ECUDA) c->sticky = VI_ECUDA;
    if (rc) return rc;  // a budget refusal leaves the previous volume in place
    c->vr = &c->own;
    c->flags_ok = false;
    mark_stale(c);
    return refresh_flags(c);
}

int vi_set_transfer_function(vi_ctx* c, const float* rgba, int M, float vmin, float vmax) {
    vi_detail::NvtxRange nvtx_range("vi_set_transfer_function");
    int rc = enter(c);
    if (rc) return rc;
    if (!rgba || M < 2 || M > 8192) return VI_EINVAL;
    if (!std::isfinite(vmin) || !std::isfinite(vmax) || !(vmax > vmin)) return VI_EINVAL;
    if (!std::isfinite((vmax - vmin))) return VI_EINVAL;
    for (int e = 0; e < M; ++e) {
        for (int ch = 0; ch < 3; ++ch)
            if (!std::isfinite(rgba[4 * e + ch])) return VI_EINVAL;
        float a = rgba[4 * e + 3];
        if (!(a >= 0.0f && a <= 1.0f)) return VI_EINVAL;
    }
    size_t bytes = (size_t)M * sizeof(float4);
    rc = ensure(c, reinterpret_cast<void**>(&c->tf), &c->tf_cap, bytes);
    if (rc) return rc;
    // Prefix count of entries with alpha > 0, for the brick flags.
    std::vector<int> cnt((size_t)M + 1, 0);
    for (int k = 0; k < M; ++k) cnt[k + 1] = cnt[k] + (rgba[4 * k + 3] > 0.0f ? 1 : 0);
    rc = ensure(c, reinterpret_cast<void**>(&c->tfcnt), &c->tfcnt_cap, cnt.size() * sizeof(int));
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(c->tf, rgba, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    // From pageable memory: the copy has left cnt by the time this returns.
    e = cudaMemcpyAsync(c->tfcnt, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice,
                        c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->M = M;
    c->vmin = vmin;
    c->vmax = vmax;
    mark_stale(c);
    return refresh_flags(c);
}

int vi_set_light(vi_ctx* c, const float dir[3], const float color[3]) {
    vi_detail::NvtxRange nvtx_range("vi_set_light");
    int rc = enter(c);
    if (rc) return rc;
    if (!dir || !finite3(dir)) return VI_EINVAL;
    float len2 = dot3(dir, dir);
    if (!(len2 > 0.0f) || !std::isfinite(len2)) return VI_EINVAL;
    if (color && !finite3(color)) return VI_EINVAL;
    for (int a = 0; a < 3; ++a) {
        c->dir[a] = dir[a];
        c->color[a] = color ? color[a] : 1.0f;
    }
    c->has_light = true;
    c->light_point = false;
    mark_stale(c);
    return VI_OK;
}

int vi_set_point_light(vi_ctx* c, const float position[3], const float color[3]) {
    vi_detail::NvtxRange nvtx_range("vi_set_point_light");
    int rc = enter(c);
    if (rc) return rc;
    if (!position || !finite3(position)) return VI_EINVAL;
    LightFrame probe;
    if (point_light_frame(position, 1, 1, &probe)) return VI_EINVAL;  // |c - pos| >= 1
    if (color && !finite3(color)) return VI_EINVAL;
    for (int a = 0; a < 3; ++a) {
        c->pos[a] = position[a];
        c->color[a] = color ? color[a] : 1.0f;
    }
    c->has_light = true;
    c->light_point = true;
    mark_stale(c);
    return VI_OK;
}

int vi_build_attenuation(vi_ctx* c, int n, int R, int mode, const vi_build_opts* opts) {
    vi_detail::NvtxRange nvtx_range("vi_build_attenuation");
    int rc = enter(c);
    if (rc) return rc;
    vi_build_opts o = opts ? *opts : default_build_opts();
    if (n < 1 || R < 1 || R > 65536 || mode < VI_NONE || mode > VI_CONE) return VI_EINVAL;
    if ((double)n * (double)R * (double)R > 17179869184.0) return VI_EINVAL;
    if (o.format < VI_F32 || o.format > VI_UNORM16) return VI_EINVAL;
    if (!(o.cone_half_angle_deg > 0.0f && o.cone_half_angle_deg < 90.0f)) return VI_EINVAL;
    if (!(o.shell_radius_vox > 0.0f) || !std::isfinite(o.shell_radius_vox)) return VI_EINVAL;
    if (!(o.comp_n >= 0.0f) || !std::isfinite(o.comp_n)) return VI_EINVAL;
    if (o.quantity != VI_TRANSMITTANCE && o.quantity != VI_OPTICAL_DEPTH) return VI_EINVAL;
    if (o.quantity == VI_OPTICAL_DEPTH && o.format == VI_UNORM16) return VI_EINVAL;
    if (o.shell_count < 0 || o.shell_count > VI_MAX_SHELLS) return VI_EINVAL;
    if (c->vr->vtype < 0 || !c->tf || !c->flags_ok) return VI_ESTATE;
    if (mode != VI_NONE && !c->has_light) return VI_ESTATE;

    LightFrame lt{};
    bool lt_ok = false;
    if (c->has_light) {
        rc = c->light_point ? point_light_frame(c->pos, n, R, &lt) : light_frame(c->dir, n, R, &lt);
        if (rc) return rc;
        lt_ok = true;
    }
    if (mode == VI_NONE) {
        c->mode = VI_NONE;
        c->bopts = o;
        c->lt = lt;
        c->lt_valid = lt_ok;
        c->stack_valid = false;
        return VI_OK;
    }
    size_t bytes = (size_t)n * (size_t)R * (size_t)R * format_bytes(o.format);
    rc = setup_stack(c, n, R, o.format);  // a refusal leaves the previous stack usable
    if (rc) return rc;
    c->stack_valid = false;

    SweepParams p;
    std::memset(&p, 0, sizeof(p));
    p.vol = volume_view(c);
    p.grid = grid_view(c);
    p.tf = c->tf;
    p.M = c->M;
    p.tf_vmin = c->vmin;
    p.tf_scale = (float)(c->M - 1) / (c->vmax - c->vmin);
    p.lt = lt;
    p.stack = c->stack;
    p.row_pitch = c->row_pitch;
    p.cells_log2 = c->sview.cells_log2;
    p.opacity_correction = o.opacity_correction ? 1 : 0;
    p.spacing_vox = lt.dL * (float)nmax(c);
    p.comp_n = o.comp_n;
    p.depth = o.quantity == VI_OPTICAL_DEPTH ? 1 : 0;
    rc = ensure(c, reinterpret_cast<void**>(&c->counter), &c->counter_cap, 256);
    if (rc) return rc;
    p.tile_counter = c->counter;
    p.lockstep = (double)n * (double)R * (double)R >= lockstep_threshold() ? 1 : 0;
    cudaError_t e = vi::launch_sweep(p, c->vr->vtype, o.format, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    ++c->launches;
    c->mode = mode;
    c->bopts = o;
    c->lt = lt;
    c->lt_valid = true;
    c->stack_bytes = bytes;
    c->stack_valid = true;
    return VI_OK;
}

int vi_render(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox, float* out,
              int out_on_device, const vi_render_opts* opts) {
    vi_detail::NvtxRange nvtx_range("vi_render");
    if (out_on_device != VI_OUT_HOST && out_on_device != VI_OUT_DEVICE &&
        out_on_device != VI_OUT_HOST_ASYNC)
        return VI_EINVAL;
    const bool device = out_on_device == VI_OUT_DEVICE;
    int rc = vi_detail::ctx_render_async(c, cam, W, H, step_vox, out, device ? 1 : 0, opts);
    if (rc || out_on_device != VI_OUT_HOST || W == 0 || H == 0) return rc;
    return cuda_fail(c, cudaStreamSynchronize(c->stream));
}

int vi_sync(vi_ctx* c) {
    vi_detail::NvtxRange nvtx_range("vi_sync");
    if (!c) return VI_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    int s = c->sticky;
    c->sticky = VI_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    return s;
}

int vi_attenuation_info(vi_ctx* c, int* n, int* R, int* format, size_t* bytes) {
    if (!c) return VI_EINVAL;
    bool have = c->stack_valid;
    if (n) *n = have ? c->lt.n : 0;
    if (R) *R = have ? c->lt.R : 0;
    if (format) *format = c->bopts.format;
    if (bytes) *bytes = have ? c->stack_bytes : 0;
    return VI_OK;
}

int vi_get_attenuation(vi_ctx* c, void* out, size_t out_bytes, int out_on_device) {
    vi_detail::NvtxRange nvtx_range("vi_get_attenuation");
    int rc = enter(c);
    if (rc) return rc;
    if (!c->stack_valid) return VI_ESTATE;
    if (!out || out_bytes < c->stack_bytes) return VI_EINVAL;
    if (out_on_device != VI_OUT_HOST && out_on_device != VI_OUT_DEVICE &&
        out_on_device != VI_OUT_HOST_ASYNC)
        return VI_EINVAL;
    out_on_device = out_on_device == VI_OUT_DEVICE;  // the copy is waited for either way
    const int n = c->lt.n, R = c->lt.R;
    const size_t esize = format_bytes(c->bopts.format);
    const size_t row = (size_t)R * esize;
    for (int k = 0; k < n; ++k) {
        cudaError_t e = cudaMemcpy2DAsync(
            static_cast<char*>(out) + (size_t)k * R * row, row,
            static_cast<const char*>(c->stack) +
                vi::slice_origin(k, R, c->sview.cells_log2, c->row_pitch / esize) * esize,
            c->row_pitch,
            row, (size_t)R, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
            c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return cuda_fail(c, e);
}

int vi_trace_pixel(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox,
                   const vi_render_opts* opts, int x, int y, int32_t* rec, int max_rec,
                   int* n_rec) {
    vi_detail::NvtxRange nvtx_range("vi_trace_pixel");
    int rc = enter(c);
    if (rc) return rc;
    vi_render_opts ro = opts ? *opts : default_render_opts();
    rc = check_render_inputs(c, cam, W, H, step_vox, &ro);
    if (rc) return rc;
    if (!rec || !n_rec || max_rec < 0 || max_rec > (1 << 22)) return VI_EINVAL;
    if (x < 0 || y < 0 || x >= W || y >= H) return VI_EINVAL;
    MarchParams p;
    rc = fill_march_params(c, cam, W, H, step_vox, &ro, &p);
    if (rc) return rc;
    p.counts = nullptr;
    p.lit = nullptr;
    size_t bytes = ((size_t)max_rec * vi::kTraceWords + 1) * sizeof(int32_t);
    rc = ensure(c, reinterpret_cast<void**>(&c->trace), &c->trace_cap, bytes);
    if (rc) return rc;
    int32_t* d_rec = c->trace + 1;
    int* d_n = reinterpret_cast<int*>(c->trace);
    cudaError_t e = vi::launch_trace(p, c->vr->vtype, c->bopts.format, c->mode, x, y, d_rec, max_rec,
                                     d_n, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    ++c->launches;
    e = cudaMemcpyAsync(n_rec, d_n, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (*n_rec > 0) {
        e = cudaMemcpyAsync(rec, d_rec, (size_t)(*n_rec) * vi::kTraceWords * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e);
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return VI_OK;
}

int vi_render_host_noalloc(vi_ctx* c, const vi_camera* cam, int W, int H, float step_vox,
                           float* out, const vi_render_opts* opts) {
    vi_detail::NvtxRange nvtx_range("vi_render_host_noalloc");
    int rc = enter(c);
    if (rc) return rc;
    vi_render_opts ro = opts ? *opts : default_render_opts();
    rc = check_render_inputs(c, cam, W, H, step_vox, &ro);
    if (rc) return rc;
    if ((size_t)W * (size_t)H > vi::kNoallocMaxPixels) return VI_EINVAL;
    if (W == 0 || H == 0) return VI_OK;
    if (!out) return VI_EINVAL;
    MarchParams p;
    rc = fill_march_params(c, cam, W, H, step_vox, &ro, &p);
    if (rc) return rc;
    unsigned* counter = nullptr;
    float4* image = nullptr;
    cudaError_t e = vi::noalloc_scratch(&counter, &image);
    if (e != cudaSuccess) return cuda_fail(c, e);
    p.tile_counter = counter;  // zeroed on the stream by the launch
    p.out = image;
    e = vi::launch_march(p, c->vr->vtype, c->bopts.format, c->mode, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    ++c->launches;
    e = cudaMemcpyAsync(out, image, (size_t)W * (size_t)H * sizeof(float4),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = cudaStreamSynchronize(c->stream);
    return cuda_fail(c, e);
}

int vi_post_ready(vi_ctx* c) {
    vi_detail::NvtxRange nvtx_range("vi_post_ready");
    int rc = enter(c);
    if (rc) return rc;
    cudaError_t e = vi::launch_post_ready(c->ready, c->post_epoch + 1u, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->posted_event, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    ++c->post_epoch;
    ++c->launches;
    return VI_OK;
}

int vi_render_batch(vi_batch_frame* frames, int count, void* cuda_stream, double wait_ms) {
    vi_detail::NvtxRange nvtx_range("vi_render_batch");
    if (!frames || count < 1 || count > VI_BATCH_MAX_FRAMES) return VI_EINVAL;
    if (!(wait_ms >= 0.0 && wait_ms <= 1e7)) return VI_EINVAL;
    static_assert(VI_BATCH_MAX_FRAMES == vi::kBatchMaxFrames, "batch limit differs");
    std::vector<BatchFrame> tab((size_t)count);
    int device = -1;
    for (int f = 0; f < count; ++f) {
        vi_batch_frame& fr = frames[f];
        fr.status = VI_OK;
        if (!fr.ctx) return VI_EINVAL;
        if (device < 0) device = fr.ctx->device;
        if (fr.ctx->device != device) return VI_EINVAL;
        if (!fr.out_rgba) return VI_EINVAL;
        const int rc = vi_detail::ctx_batch_frame(fr.ctx, &fr.camera, fr.width, fr.height,
                                                  fr.step_vox, fr.out_rgba, 1, &fr.opts,
                                                  &tab[(size_t)f]);
        if (rc) return rc;
        tab[(size_t)f].index = f;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<int> status((size_t)count, VI_OK);
    std::vector<int*> dst((size_t)count);
    for (int f = 0; f < count; ++f) dst[(size_t)f] = &status[(size_t)f];
    std::vector<vi_ctx*> ctxs((size_t)count);
    for (int f = 0; f < count; ++f) ctxs[(size_t)f] = frames[f].ctx;
    cudaError_t e = vi_detail::enqueue_batch(ctxs.data(), tab.data(), count,
                                             (unsigned long long)(wait_ms * 1e6), dst.data(), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    int rc = VI_OK;
    for (int f = 0; f < count; ++f) {
        frames[f].status = status[(size_t)f];
        if (status[(size_t)f] != VI_OK) rc = VI_ETIMEOUT;
        ++frames[f].ctx->launches;
    }
    return rc;
}

int vi_debug_bounds(int device, uint64_t* violations, int* first_site, int64_t* first_index) {
    if (!violations || !first_site || !first_index) return VI_EINVAL;
    *violations = 0;
    *first_site = 0;
    *first_index = 0;
#if VI_DEBUG_BOUNDS
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    if (device < 0 || device >= count) return VI_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return VI_ECUDA;
    cudaError_t (*const records[3])(unsigned*) = {vi::debug_record_sweep, vi::debug_record_march,
                                                  vi::debug_record_grid};
    for (auto read : records) {
        unsigned r[4] = {0u, 0u, 0u, 0u};
        if (read(r) != cudaSuccess) {
            cudaGetLastError();
            return VI_ECUDA;
        }
        if (r[0] && !*violations) {
            *first_site = (int)r[1];
            *first_index = (int64_t)(((uint64_t)r[3] << 32) | r[2]);
        }
        *violations += r[0];
    }
    return VI_OK;
#else
    (void)device;
    return VI_ESTATE;
#endif
}

int vi_get_skip_grid(vi_ctx* c, int* dims, uint8_t* brick_flags, size_t brick_bytes,
                     uint8_t* cell_skip, size_t cell_bytes) {
    vi_detail::NvtxRange nvtx_range("vi_get_skip_grid");
    int rc = enter(c);
    if (rc) return rc;
    if (!c->flags_ok || !c->bflags) return VI_ESTATE;
    const vi::GridView g = grid_view(c);
    const int nbz = c->vr->nbz, cnz = nbz * vi::kCellsPerBrick;
    const size_t nb = (size_t)nbricks(c), nc = (size_t)g.cnx * g.cny * cnz;
    if ((brick_flags && brick_bytes < nb) || (cell_skip && cell_bytes < nc)) return VI_EINVAL;
    if (dims) {
        const int d[6] = {g.nbx, g.nby, nbz, g.cnx, g.cny, cnz};
        std::memcpy(dims, d, sizeof(d));
    }
    if (brick_flags) {
        cudaError_t e = cudaMemcpyAsync(brick_flags, g.flags, nb, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    if (cell_skip) {
        cudaError_t e = cudaMemcpyAsync(cell_skip, g.skip, nc, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return cuda_fail(c, cudaStreamSynchronize(c->stream));
}

int vi_launch_count(vi_ctx* c, uint64_t* count) {
    if (!c || !count) return VI_EINVAL;
    *count = c->launches;
    return VI_OK;
}

}  // extern "C"
