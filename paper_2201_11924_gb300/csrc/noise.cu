// IR sensor noise (arxiv 2201.11924 Sec. VI-C), applied to both views before
// the census when a handle has it switched on, and callable on its own.
//
//   I_noisy = gamma * I_clean + n,   gamma ~ Gamma(k, theta),   n ~ N(mu, sigma^2)
//
// per pixel and view, rounded half to even and clamped to [0, 255].  One
// thread per pixel.  Random numbers come from the counter-based Philox4x64-10
// generator (Salmon, Moraes, Dror and Shaw, SC 2011: ten rounds of two
// 64 x 64 -> 128-bit products, key bumped by two Weyl constants per round)
// with counter (pixel, attempt, frame, view) and key (seed, 0), so every
// pixel's numbers are independent of the launch shape and reproducible.  A
// 64-bit output r gives the uniform ((r >> 41) + 1/2) / 2^23 (exact in single
// precision).  Normals come from the Box-Muller transform of two uniforms
// (z0 for the gamma proposal, z1 for the thermal term) and gamma from
// Marsaglia and Tsang's rejection method for k >= 1 (with d = k - 1/3,
// c = 1/(3 sqrt(d)): v = (1 + c z0)^3 is accepted when ln u2 < z0^2/2 + d -
// d v + d ln v), at most 16 attempts (if all are rejected, gamma = d theta).
#include "internal.h"

namespace simsense {
namespace {

constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kM1 = 0xCA5A826395121157ull;
constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64(uint64_t& x0, uint64_t& x1, uint64_t& x2, uint64_t& x3, uint64_t k0,
                                           uint64_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; round++) {
        const uint64_t hi0 = __umul64hi(kM0, x0), lo0 = kM0 * x0;
        const uint64_t hi1 = __umul64hi(kM1, x2), lo1 = kM1 * x2;
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
        k0 += kW0;
        k1 += kW1;
    }
}

__device__ __forceinline__ float unit23(uint64_t r)
{
    return ((float)(uint32_t)(r >> 41) + 0.5f) * (1.0f / 8388608.0f);
}

// blockIdx.y = view (0 = left, 1 = right) of a two-view launch.
__global__ void __launch_bounds__(256)
noise_kernel(const uint8_t* clean0, uint8_t* noisy0, const uint8_t* clean1, uint8_t* noisy1, int npx, float mu, float sigma, float d, float c, float theta,
             uint64_t seed, uint32_t frame, uint32_t view0)
{
    // (no __restrict__: the noise may be applied in place, each pixel read
    // and then written by the same thread)
    const int view = blockIdx.y;
    const uint8_t* clean = view ? clean1 : clean0;
    uint8_t* noisy = view ? noisy1 : noisy0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += gridDim.x * blockDim.x) {
        float gamma = d * theta, z1 = 0.0f;
        for (int attempt = 0; attempt < 16; attempt++) {
            uint64_t x0 = (uint64_t)i, x1 = (uint64_t)attempt, x2 = frame, x3 = view0 + (uint32_t)view;
            philox4x64(x0, x1, x2, x3, seed, 0);
            const float u0 = unit23(x0), u1 = unit23(x1), u2 = unit23(x2);
            const float rad = sqrtf(-2.0f * logf(u0));
            float s, co;
            sincospif(2.0f * u1, &s, &co);
            const float z0 = rad * co;
            z1 = rad * s;
            const float t = 1.0f + c * z0;
            if (!(t > 0.0f)) continue;
            const float v = t * t * t;
            if (logf(u2) < 0.5f * z0 * z0 + d - d * v + d * logf(v)) {
                gamma = d * v * theta;
                break;
            }
        }
        const float val = gamma * (float)clean[i] + (mu + sigma * z1);
        noisy[i] = (uint8_t)fminf(fmaxf(rintf(val), 0.0f), 255.0f);
    }
}

}  // namespace

int check_noise(const NoiseParams& n)
{
    if (!(n.k >= 1.0f) || !isfinite(n.k) || !(n.theta > 0.0f) || !isfinite(n.theta) || !(n.sigma >= 0.0f) ||
        !isfinite(n.sigma) || !isfinite(n.mu))
        return SIMSENSE_ERR_INVALID_ARG;
    return SIMSENSE_OK;
}

cudaError_t launch_noise(const NoiseParams& n, const uint8_t* clean0, uint8_t* noisy0, const uint8_t* clean1,
                         uint8_t* noisy1, int npx, uint32_t frame, uint32_t view0, cudaStream_t s)
{
    const double d = (double)n.k - 1.0 / 3.0;
    const double c = 1.0 / (3.0 * sqrt(d));
    const int blocks = (npx + 255) / 256 < 4096 ? (npx + 255) / 256 : 4096;
    dim3 grid(blocks > 0 ? blocks : 1, clean1 ? 2 : 1);
    noise_kernel<<<grid, 256, 0, s>>>(clean0, noisy0, clean1, noisy1, npx, n.mu, n.sigma, (float)d, (float)c,
                                      n.theta, n.seed, frame, view0);
    return cudaGetLastError();
}

}  // namespace simsense
