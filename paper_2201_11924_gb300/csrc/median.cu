// Median filter of the disparity map (arxiv 2201.11924 Sec. VI-D lists median
// filtering among the disparity post-processing steps), fused with the
// disparity-to-depth conversion.
//
// One thread per pixel: the k x k window (k = 3 or 5, borders replicated) is
// gathered into registers, where invalid pixels carry 0, and its middle value
// is found by a partial selection sort: after pass i the i-th smallest value
// sits at position i, so (k*k)/2 + 1 passes of compare-exchanges leave the
// median at position (k*k)/2.  The output pixel is valid iff the median is
// positive; its depth is f*b / median.
#include "internal.h"

namespace simsense {
namespace {

template <int K>
__global__ void __launch_bounds__(256)
median_kernel(const float* __restrict__ disp, float* __restrict__ depth, float* __restrict__ disp_out,
              int W, int H, float fb)
{
    constexpr int R = K / 2;
    constexpr int NV = K * K;
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    float v[NV];
#pragma unroll
    for (int dy = -R; dy <= R; dy++) {
        const int yy = min(max(y + dy, 0), H - 1);
#pragma unroll
        for (int dx = -R; dx <= R; dx++) {
            const int xx = min(max(x + dx, 0), W - 1);
            v[(dy + R) * K + dx + R] = __ldg(disp + (size_t)yy * W + xx);
        }
    }
#pragma unroll
    for (int i = 0; i <= NV / 2; i++) {
#pragma unroll
        for (int j = i + 1; j < NV; j++) {
            const float a = v[i], b = v[j];
            v[i] = fminf(a, b);
            v[j] = fmaxf(a, b);
        }
    }
    const float med = v[NV / 2];
    const size_t pix = (size_t)y * W + x;
    depth[pix] = med > 0.0f ? __fdiv_rn(fb, med) : 0.0f;
    if (disp_out) disp_out[pix] = med > 0.0f ? med : -1.0f;
}

}  // namespace

cudaError_t launch_median(const Params& p, const float* disp, float* depth, float* disp_out, cudaStream_t s)
{
    dim3 grid((p.W + 31) / 32, (p.H + 7) / 8);
    if (p.median == 3)
        median_kernel<3><<<grid, 256, 0, s>>>(disp, depth, disp_out, p.W, p.H, p.fb);
    else if (p.median == 5)
        median_kernel<5><<<grid, 256, 0, s>>>(disp, depth, disp_out, p.W, p.H, p.fb);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace simsense
