// IR image formation of analytic scenes (arxiv 2201.11924 Sec. VI-A/VI-B):
// the projector of an active-stereo sensor is a textured spot light, surfaces
// reflect with the paper's BSDF mix
//   f = w_d f_d + (1 - w_d) f_s,   w_d = (1 - metallic) (1 - transmission),
// f_d Lambertian, f_s the GGX microfacet term, and a weak ambient light adds
// albedo * ambient.  The paper renders with a Vulkan path tracer and a learned
// denoiser; this kernel is a direct-light ray caster over spheres and
// rectangles (one ray per pixel centre, nearest hit, one shadow ray to the
// projector), so the pair that feeds the depth stage can be generated on the
// device.  Evaluation in fp64 with correctly rounded + - * / and sqrt in a
// fixed order (no contraction into fused multiply-adds); pixel = gain * L
// rounded half to even and clamped to [0, 255].  One thread per pixel and
// view; grid.y = view (0 = left camera at the origin, 1 = right at (b, 0, 0)).
#include "internal.h"

namespace simsense {
namespace {

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dq(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double dot3(const double* a, const double* b)
{
    return da(da(dm(a[0], b[0]), dm(a[1], b[1])), dm(a[2], b[2]));
}
__device__ __forceinline__ void cross3(const double* u, const double* v, double* n)
{
    n[0] = ds(dm(u[1], v[2]), dm(u[2], v[1]));
    n[1] = ds(dm(u[2], v[0]), dm(u[0], v[2]));
    n[2] = ds(dm(u[0], v[1]), dm(u[1], v[0]));
}

// Ray o + t d against one primitive: the smallest t > 1e-9, else -1.
__device__ double hit(const simsense_primitive_t& q, const double* o, const double* d)
{
    const double eps = 1e-9;
    if (q.kind == 0) {
        const double oc[3] = {ds(o[0], q.c[0]), ds(o[1], q.c[1]), ds(o[2], q.c[2])};
        const double a = dot3(d, d), b = dm(2.0, dot3(d, oc)), cc = ds(dot3(oc, oc), dm(q.radius, q.radius));
        const double disc = ds(dm(b, b), dm(dm(4.0, a), cc));
        if (disc < 0.0) return -1.0;
        const double sq = dq(disc);
        double t = dd(ds(-b, sq), dm(2.0, a));
        if (t > eps) return t;
        t = dd(da(-b, sq), dm(2.0, a));
        return t > eps ? t : -1.0;
    }
    double n[3];
    cross3(q.u, q.v, n);
    const double den = dot3(d, n);
    if (den == 0.0) return -1.0;
    const double co[3] = {ds(q.c[0], o[0]), ds(q.c[1], o[1]), ds(q.c[2], o[2])};
    const double t = dd(dot3(co, n), den);
    if (!(t > eps)) return -1.0;
    const double p[3] = {ds(da(o[0], dm(t, d[0])), q.c[0]), ds(da(o[1], dm(t, d[1])), q.c[1]),
                         ds(da(o[2], dm(t, d[2])), q.c[2])};
    const double s = dd(dot3(p, q.u), dot3(q.u, q.u)), w = dd(dot3(p, q.v), dot3(q.v, q.v));
    if (s < -1.0 || s > 1.0 || w < -1.0 || w > 1.0) return -1.0;
    return t;
}

__device__ double radiance(const simsense_primitive_t* prims, int n, const simsense_render_t& rp,
                           const uint8_t* pattern, const double* o, const double* d)
{
    const double PI = 3.14159265358979323846;
    int best = -1;
    double tb = 0.0;
    for (int k = 0; k < n; k++) {
        const double t = hit(prims[k], o, d);
        if (t > 0.0 && (best < 0 || t < tb)) { best = k; tb = t; }
    }
    if (best < 0) return 0.0;
    const simsense_primitive_t& q = prims[best];
    const double p[3] = {da(o[0], dm(tb, d[0])), da(o[1], dm(tb, d[1])), da(o[2], dm(tb, d[2]))};
    double nn[3];
    if (q.kind == 0) {
        nn[0] = dd(ds(p[0], q.c[0]), q.radius);
        nn[1] = dd(ds(p[1], q.c[1]), q.radius);
        nn[2] = dd(ds(p[2], q.c[2]), q.radius);
    } else {
        double m[3];
        cross3(q.u, q.v, m);
        const double len = dq(dot3(m, m));
        nn[0] = dd(m[0], len);
        nn[1] = dd(m[1], len);
        nn[2] = dd(m[2], len);
        if (dot3(nn, d) > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
    }
    double L = dm(rp.ambient, q.albedo);
    const double li[3] = {ds(rp.proj[0], p[0]), ds(rp.proj[1], p[1]), ds(rp.proj[2], p[2])};
    const double dist2 = dot3(li, li), dist = dq(dist2);
    const double iv[3] = {dd(li[0], dist), dd(li[1], dist), dd(li[2], dist)};
    const double ni = dot3(nn, iv);
    const double X[3] = {ds(p[0], rp.proj[0]), ds(p[1], rp.proj[1]), ds(p[2], rp.proj[2])};
    if (ni > 0.0 && X[2] > 0.0) {
        bool lit = true;
        for (int k = 0; k < n && lit; k++) {
            if (k == best) continue;
            const double t = hit(prims[k], p, li);
            if (t > 0.0 && t < 1.0) lit = false;
        }
        const double up = da(dm(rp.pf, dd(X[0], X[2])), rp.pcx), vp = da(dm(rp.pf, dd(X[1], X[2])), rp.pcy);
        const double fu = floor(da(up, 0.5)), fv = floor(da(vp, 0.5));
        double pat = 0.0;
        if (fu >= 0.0 && fu < (double)rp.PW && fv >= 0.0 && fv < (double)rp.PH)
            pat = dd((double)pattern[(size_t)fv * rp.PW + (size_t)fu], 255.0);
        if (lit && pat > 0.0) {
            const double E = dd(dm(dm(rp.power, pat), ni), dist2);
            double ov[3] = {ds(o[0], p[0]), ds(o[1], p[1]), ds(o[2], p[2])};
            const double ol = dq(dot3(ov, ov));
            ov[0] = dd(ov[0], ol);
            ov[1] = dd(ov[1], ol);
            ov[2] = dd(ov[2], ol);
            const double no = dot3(nn, ov);
            const double wd = dm(ds(1.0, q.metallic), ds(1.0, q.transmission));
            const double fd = dd(q.albedo, PI);
            double fs = 0.0;
            if (no > 0.0) {
                double hv[3] = {da(iv[0], ov[0]), da(iv[1], ov[1]), da(iv[2], ov[2])};
                const double hl = dq(dot3(hv, hv));
                hv[0] = dd(hv[0], hl);
                hv[1] = dd(hv[1], hl);
                hv[2] = dd(hv[2], hl);
                const double a = dm(q.roughness, q.roughness), a2 = dm(a, a);
                const double nh = dot3(nn, hv);
                const double den = da(dm(dm(nh, nh), ds(a2, 1.0)), 1.0);
                const double D = dd(a2, dm(dm(PI, den), den));
                const double g1i = dd(dm(2.0, ni), da(ni, dq(da(a2, dm(dm(ds(1.0, a2), ni), ni)))));
                const double g1o = dd(dm(2.0, no), da(no, dq(da(a2, dm(dm(ds(1.0, a2), no), no)))));
                const double F0 = da(dm(0.04, ds(1.0, q.metallic)), dm(q.albedo, q.metallic));
                const double vh = dot3(ov, hv);
                const double m1 = ds(1.0, vh), m2 = dm(m1, m1);
                const double F = da(F0, dm(ds(1.0, F0), dm(dm(m2, m2), m1)));
                fs = dd(dm(dm(D, F), dm(g1i, g1o)), dm(dm(4.0, ni), no));
            }
            L = da(L, dm(da(dm(wd, fd), dm(ds(1.0, wd), fs)), E));
        }
    }
    return dm(rp.gain, L);
}

__global__ void __launch_bounds__(128)
render_kernel(const simsense_primitive_t* __restrict__ prims, int n, simsense_render_t rp,
              const uint8_t* __restrict__ pattern, uint8_t* __restrict__ left, uint8_t* __restrict__ right)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rp.W * rp.H) return;
    const int view = blockIdx.y;
    const int u = i % rp.W, v = i / rp.W;
    const double o[3] = {view ? rp.baseline : 0.0, 0.0, 0.0};
    const double d[3] = {dd(ds((double)u, rp.cx), rp.f), dd(ds((double)v, rp.cy), rp.f), 1.0};
    const double val = rint(radiance(prims, n, rp, pattern, o, d));
    (view ? right : left)[i] = (uint8_t)fmin(fmax(val, 0.0), 255.0);
}

}  // namespace
}  // namespace simsense

using namespace simsense;

extern "C" int simsense_render_ir(const simsense_primitive_t* prims, int n, const simsense_render_t* rp,
                                  const uint8_t* pattern, uint8_t* left, uint8_t* right, struct CUstream_st* stream)
{
    if (!rp || !pattern || !left || !right || n < 0 || n > 4096 || (n > 0 && !prims)) return SIMSENSE_ERR_INVALID_ARG;
    if (rp->W < 1 || rp->H < 1 || rp->W > 16384 || rp->H > 16384 || rp->PW < 1 || rp->PH < 1 || rp->PW > 16384 ||
        rp->PH > 16384)
        return SIMSENSE_ERR_INVALID_ARG;
    const double v[] = {rp->f, rp->cx, rp->cy, rp->baseline, rp->proj[0], rp->proj[1], rp->proj[2], rp->pf,
                        rp->pcx, rp->pcy, rp->power, rp->ambient, rp->gain};
    for (double x : v)
        if (!isfinite(x)) return SIMSENSE_ERR_INVALID_ARG;
    if (rp->f == 0.0 || rp->pf == 0.0) return SIMSENSE_ERR_INVALID_ARG;
    dim3 grid((unsigned)((rp->W * rp->H + 127) / 128), 2);
    render_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(prims, n, *rp, pattern, left, right);
    return cudaGetLastError() == cudaSuccess ? SIMSENSE_OK : SIMSENSE_ERR_CUDA;
}
