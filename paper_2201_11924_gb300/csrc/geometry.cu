// Stereo rectification and depth registration (arxiv 2201.11924 Sec. VI-D:
// the stage starts by rectifying the pair onto one image plane and can end by
// registering the depth map to the frame of the RGB camera).
//
// Camera model (the paper gives none): pinhole with Brown-Conrady distortion
// and a rectifying rotation.  For rectified pixel (u, v) the raw position is
//   r = R^T ((u - rcx)/rfx, (v - rcy)/rfy, 1),  x = r.x/r.z,  y = r.y/r.z,
//   x_d = x (1 + k1 r^2 + k2 r^4 + k3 r^6) + 2 p1 x y + p2 (r^2 + 2 x^2),
//   y_d = y (1 + ...) + p1 (r^2 + 2 y^2) + 2 p2 x y,
//   (ur, vr) = (fx x_d + cx, fy y_d + cy),
// computed in fp64 with the correctly rounded __d*_rn operations in a fixed
// order (no contraction into fused multiply-adds), then quantised to 1/256 px
// (fraction rounded half to even, 256 carrying into the next pixel) and
// resampled by 8-bit fixed-point bilinear interpolation.  The map depends
// only on the camera, so a handle computes it once (8 bytes per pixel) and
// every frame resamples with integer arithmetic.
//
// Registration: every valid depth pixel is back-projected, moved by (R, t)
// into the RGB camera, projected and splatted to the nearest RGB pixel with a
// z-buffer (an atomic compare-and-swap loop keeps the smallest depth).
#include "internal.h"

namespace simsense {
namespace {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

constexpr short kNoSource = -32768;

// Map entry of rectified pixel (u, v): source x0, y0 (clamped to [-2, W+1] x
// [-2, H+1], where every tap is outside) and fractions ax, ay in 1/256 px.
__device__ short4 rect_map(const simsense_camera_t& c, int u, int v, int W, int H)
{
    const double xr = ddiv(dsub((double)u, c.rcx), c.rfx);
    const double yr = ddiv(dsub((double)v, c.rcy), c.rfy);
    const double X = dadd(dadd(dmul(c.R[0], xr), dmul(c.R[3], yr)), c.R[6]);
    const double Y = dadd(dadd(dmul(c.R[1], xr), dmul(c.R[4], yr)), c.R[7]);
    const double Z = dadd(dadd(dmul(c.R[2], xr), dmul(c.R[5], yr)), c.R[8]);
    if (!(Z > 0.0)) return make_short4(kNoSource, 0, 0, 0);
    const double x = ddiv(X, Z), y = ddiv(Y, Z);
    const double r2 = dadd(dmul(x, x), dmul(y, y));
    const double radial = dadd(dadd(dadd(1.0, dmul(c.k1, r2)), dmul(dmul(c.k2, r2), r2)),
                               dmul(dmul(dmul(c.k3, r2), r2), r2));
    const double xd = dadd(dadd(dmul(x, radial), dmul(dmul(dmul(2.0, c.p1), x), y)),
                           dmul(c.p2, dadd(r2, dmul(dmul(2.0, x), x))));
    const double yd = dadd(dadd(dmul(y, radial), dmul(c.p1, dadd(r2, dmul(dmul(2.0, y), y)))),
                           dmul(dmul(dmul(2.0, c.p2), x), y));
    const double ur = dadd(dmul(c.fx, xd), c.cx), vr = dadd(dmul(c.fy, yd), c.cy);
    if (!(fabs(ur) < 1e9) || !(fabs(vr) < 1e9)) return make_short4(kNoSource, 0, 0, 0);
    const double fxl = floor(ur), fyl = floor(vr);
    int a = (int)rint(dmul(dsub(ur, fxl), 256.0)), b = (int)rint(dmul(dsub(vr, fyl), 256.0));
    long long xi = (long long)fxl, yi = (long long)fyl;
    if (a == 256) { a = 0; xi++; }
    if (b == 256) { b = 0; yi++; }
    xi = xi < -2 ? -2 : (xi > W + 1 ? W + 1 : xi);
    yi = yi < -2 ? -2 : (yi > H + 1 ? H + 1 : yi);
    return make_short4((short)xi, (short)yi, (short)a, (short)b);
}

__device__ __forceinline__ uint8_t resample(const uint8_t* raw, int W, int H, short4 m)
{
    if (m.x == kNoSource) return 0;
    uint32_t t[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int xx = m.x + (k & 1), yy = m.y + (k >> 1);
        t[k] = (xx >= 0 && xx < W && yy >= 0 && yy < H) ? raw[(size_t)yy * W + xx] : 0u;
    }
    const uint32_t ax = (uint32_t)m.z, ay = (uint32_t)m.w, bx = 256u - ax, by = 256u - ay;
    return (uint8_t)((bx * by * t[0] + ax * by * t[1] + bx * ay * t[2] + ax * ay * t[3] + 32768u) >> 16);
}

__global__ void __launch_bounds__(256)
map_kernel(simsense_camera_t c, int W, int H, short4* __restrict__ map)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    map[i] = rect_map(c, i % W, i / W, W, H);
}

// blockIdx.y = view: (raw0, map0, out0) or (raw1, map1, out1)
__global__ void __launch_bounds__(256)
remap_kernel(const uint8_t* raw0, const short4* __restrict__ map0, uint8_t* out0, const uint8_t* raw1,
             const short4* __restrict__ map1, uint8_t* out1, int W, int H)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    if (blockIdx.y == 0) out0[i] = resample(raw0, W, H, map0[i]);
    else out1[i] = resample(raw1, W, H, map1[i]);
}

// map and resample in one pass (the stand-alone call)
__global__ void __launch_bounds__(256)
rectify_kernel(simsense_camera_t c, const uint8_t* raw, uint8_t* out, int W, int H)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    out[i] = resample(raw, W, H, rect_map(c, i % W, i / W, W, H));
}

__global__ void __launch_bounds__(256)
register_kernel(const float* __restrict__ depth, int W, int H, simsense_registration_t g,
                float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const double Z = depth[i];
    if (!(Z > 0.0)) return;
    const int u = i % W, v = i / W;
    const double X = dmul(ddiv(dsub((double)u, g.cx), g.fx), Z);
    const double Y = dmul(ddiv(dsub((double)v, g.cy), g.fy), Z);
    const double X2 = dadd(dadd(dadd(dmul(g.R[0], X), dmul(g.R[1], Y)), dmul(g.R[2], Z)), g.t[0]);
    const double Y2 = dadd(dadd(dadd(dmul(g.R[3], X), dmul(g.R[4], Y)), dmul(g.R[5], Z)), g.t[1]);
    const double Z2 = dadd(dadd(dadd(dmul(g.R[6], X), dmul(g.R[7], Y)), dmul(g.R[8], Z)), g.t[2]);
    if (!(Z2 > 0.0)) return;
    const double u2 = dadd(dmul(g.fx2, ddiv(X2, Z2)), g.cx2);
    const double v2 = dadd(dmul(g.fy2, ddiv(Y2, Z2)), g.cy2);
    const double pu = floor(dadd(u2, 0.5)), pv = floor(dadd(v2, 0.5));
    if (!(pu >= 0.0 && pu < (double)g.W2 && pv >= 0.0 && pv < (double)g.H2)) return;
    unsigned int* cell = reinterpret_cast<unsigned int*>(out + (size_t)pv * g.W2 + (size_t)pu);
    const float z = __double2float_rn(Z2);
    const unsigned int zb = __float_as_uint(z);
    unsigned int cur = *cell;
    // z-buffer: keep the smallest positive depth (0 = nothing yet); positive
    // floats order like their bit patterns
    while (cur == 0u || zb < cur) {
        const unsigned int prev = atomicCAS(cell, cur, zb);
        if (prev == cur) break;
        cur = prev;
    }
}

inline int blocks_for(long long n) { return (int)((n + 255) / 256); }

}  // namespace

int check_camera(const simsense_camera_t& c)
{
    const double v[] = {c.fx, c.fy, c.cx, c.cy, c.k1, c.k2, c.p1, c.p2, c.k3, c.rfx, c.rfy, c.rcx, c.rcy};
    for (double x : v)
        if (!isfinite(x)) return SIMSENSE_ERR_INVALID_ARG;
    for (double x : c.R)
        if (!isfinite(x)) return SIMSENSE_ERR_INVALID_ARG;
    if (c.fx == 0.0 || c.fy == 0.0 || c.rfx == 0.0 || c.rfy == 0.0) return SIMSENSE_ERR_INVALID_ARG;
    return SIMSENSE_OK;
}

cudaError_t launch_rect_map(const simsense_camera_t& c, int W, int H, short4* map, cudaStream_t s)
{
    map_kernel<<<blocks_for((long long)W * H), 256, 0, s>>>(c, W, H, map);
    return cudaGetLastError();
}

cudaError_t launch_remap(const uint8_t* raw0, const short4* map0, uint8_t* out0, const uint8_t* raw1,
                         const short4* map1, uint8_t* out1, int W, int H, cudaStream_t s)
{
    dim3 grid(blocks_for((long long)W * H), 2);
    remap_kernel<<<grid, 256, 0, s>>>(raw0, map0, out0, raw1, map1, out1, W, H);
    return cudaGetLastError();
}

}  // namespace simsense

using namespace simsense;

extern "C" int simsense_rectify(const uint8_t* raw, uint8_t* out, int W, int H, const simsense_camera_t* cam,
                                struct CUstream_st* stream)
{
    if (!raw || !out || !cam || W < 1 || H < 1 || W > 32000 || H > 32000 || check_camera(*cam) != SIMSENSE_OK)
        return SIMSENSE_ERR_INVALID_ARG;
    rectify_kernel<<<blocks_for((long long)W * H), 256, 0, (cudaStream_t)stream>>>(*cam, raw, out, W, H);
    return cudaGetLastError() == cudaSuccess ? SIMSENSE_OK : SIMSENSE_ERR_CUDA;
}

extern "C" int simsense_register_depth(const float* depth, int W, int H, const simsense_registration_t* reg,
                                       float* out, struct CUstream_st* stream)
{
    if (!depth || !out || !reg || W < 1 || H < 1 || reg->W2 < 1 || reg->H2 < 1 || W > 32000 || H > 32000 ||
        reg->W2 > 32000 || reg->H2 > 32000)
        return SIMSENSE_ERR_INVALID_ARG;
    const double v[] = {reg->fx, reg->fy, reg->cx, reg->cy, reg->fx2, reg->fy2, reg->cx2, reg->cy2};
    for (double x : v)
        if (!isfinite(x)) return SIMSENSE_ERR_INVALID_ARG;
    for (double x : reg->R)
        if (!isfinite(x)) return SIMSENSE_ERR_INVALID_ARG;
    for (double x : reg->t)
        if (!isfinite(x)) return SIMSENSE_ERR_INVALID_ARG;
    if (reg->fx == 0.0 || reg->fy == 0.0) return SIMSENSE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)reg->W2 * reg->H2 * sizeof(float), st);
    if (e == cudaSuccess) {
        register_kernel<<<blocks_for((long long)W * H), 256, 0, st>>>(depth, W, H, *reg, out);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? SIMSENSE_OK : SIMSENSE_ERR_CUDA;
}
