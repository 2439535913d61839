// Per-SM issue rates of the instructions an SGM recurrence can use, measured on
// the GPU: the measured peaks the benchmark line quotes beside the derived
// INT32 peak come from this probe (it is not part of the library).
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/oprates paper_2201_11924_gb300/probes/op_rates.cu && /tmp/oprates
// grid = #SMs blocks x 1024 threads, each thread 8 dependent-rotating chains.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

template <int OP>
__device__ __forceinline__ uint32_t op(uint32_t a, uint32_t b, uint32_t c = 0)
{
    uint32_t d;
    if constexpr (OP == 0) asm volatile("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 1) asm volatile("min.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 2) asm volatile("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 3) asm volatile("xor.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 4) asm volatile("prmt.b32 %0, %1, %2, 0x5432;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 5) asm volatile("popc.b32 %0, %1;" : "=r"(d) : "r"(a ^ 0));
    else if constexpr (OP == 6) asm volatile("shfl.sync.bfly.b32 %0, %1, 1, 0x1f, 0xffffffff;" : "=r"(d) : "r"(a));
    else if constexpr (OP == 7) asm volatile("mad.lo.u32 %0, %1, %2, 7;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 8) asm volatile("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 9) asm volatile("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 10) asm volatile("fma.rn.f16x2 %0, %1, %2, %1;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 11) asm volatile("min.f32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 12) asm volatile("add.rn.f32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 13) d = __vminu4(a, b);
    else if constexpr (OP == 14) asm volatile("min.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 15) asm volatile("min.f32 %0, %1, %2, %1;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 16) asm volatile("add.u32 %0, %1, %2;\n\tadd.u32 %0, %0, %1;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 17) asm volatile("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 18) asm volatile("vadd2.u32.u32.u32 %0, %1, %2, %1;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 19) asm volatile("sub.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 20) asm volatile("min.u16x2 %0, %1, %2;\n\tmin.f16x2 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 21) asm volatile("redux.sync.min.u32 %0, %1, 0xffffffff;" : "=r"(d) : "r"(a));
    else if constexpr (OP == 22) asm volatile("min.u16x2 %0, %1, %2;\n\tadd.u32 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 23) asm volatile("min.u16x2 %0, %1, %2;\n\tadd.rn.f16x2 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 24) asm volatile("min.u32 %0, %1, %2;\n\tmin.f32 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 25) asm volatile("min.u16x2 %0, %1, %2;\n\tprmt.b32 %0, %0, %2, 0x5432;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 26) asm volatile("min.f16x2 %0, %1, %2;\n\tadd.rn.f16x2 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 27) asm volatile("min.u16x2 %0, %1, %2;\n\tmad.lo.u32 %0, %0, %2, 7;" : "=r"(d) : "r"(a), "r"(b));
    // DPX (dynamic-programming) intrinsics: three-input min and fused add-min
    else if constexpr (OP == 28) d = __vimin3_u16x2(a, b, c);
    else if constexpr (OP == 29) d = __viaddmin_u16x2(a, b, c);
    else if constexpr (OP == 30) d = __vimin3_u32(a, b, c);
    else if constexpr (OP == 31) d = __vimin3_s16x2(a, b, c);
    else if constexpr (OP == 32) { d = __vimin3_u16x2(a, b, c); asm volatile("min.u16x2 %0, %0, %1;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 33) { d = __vimin3_u16x2(a, b, c); asm volatile("prmt.b32 %0, %0, %1, 0x5432;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 34) { d = __vimin3_u16x2(a, b, c); asm volatile("add.u32 %0, %0, %1;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 36) asm volatile("and.b32 %0, %1, 0x00ff00ff;\n\txor.b32 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 37) asm volatile("shr.u32 %0, %1, 8;\n\txor.b32 %0, %0, %2;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 38) { d = __vimin3_u16x2(a, b, c); asm volatile("lop3.b32 %0, %0, %1, 0x00ff00ff, 0xc0;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 39) { d = __vimin3_u16x2(a, b, c); asm volatile("mad.lo.u32 %0, %0, 256, %1;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 40) { d = __vimin3_u16x2(a, b, c); asm volatile("shr.u32 %0, %0, 8;" : "+r"(d)); }
    else if constexpr (OP == 41) asm volatile("add.u32 %0, %1, %2;\n\tsub.u32 %0, %0, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    else if constexpr (OP == 42) { d = __vimin3_u16x2(a, b, c); asm volatile("add.u32 %0, %0, %1;\n\tsub.u32 %0, %0, %2;" : "+r"(d) : "r"(b), "r"(c)); }
    else if constexpr (OP == 43) asm volatile("prmt.b32 %0, %1, %2, 0x5432;\n\tlop3.b32 %0, %0, %2, 0x00ff00ff, 0xc0;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 35) { d = __viaddmin_u16x2(a, b, c); asm volatile("min.u16x2 %0, %0, %1;" : "+r"(d) : "r"(b)); }
    // funnel shift (the pair shifted by one cell across two words) and the
    // mixes that tell whether f16 minima, funnel shifts and masks share the
    // pipe of the packed-integer minima
    else if constexpr (OP == 44) asm volatile("shf.r.wrap.b32 %0, %1, %2, 16;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 45) asm volatile("min.u16x2 %0, %1, %2;\n\tshf.r.wrap.b32 %0, %0, %2, 16;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 46) { d = __vimin3_u16x2(a, b, c); asm volatile("min.f16x2 %0, %0, %1;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 47) asm volatile("lop3.b32 %0, %1, %2, 0x00ff00ff, 0xc0;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 48) asm volatile("min.f16x2 %0, %1, %2;\n\tprmt.b32 %0, %0, %2, 0x5432;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 49) asm volatile("min.f16x2 %0, %1, %2;\n\tshf.r.wrap.b32 %0, %0, %2, 16;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 50) { d = __vimin3_u16x2(a, b, c); asm volatile("min.f16x2 %0, %0, %1;\n\tadd.u32 %0, %0, %1;" : "+r"(d) : "r"(b)); }
    else if constexpr (OP == 51) asm volatile("add.rn.f16x2 %0, %1, %2;\n\tlop3.b32 %0, %0, %2, 0x00ff00ff, 0xc0;" : "=r"(d) : "r"(a), "r"(b));
    else if constexpr (OP == 52) asm volatile("add.rn.f16x2 %0, %1, %2;\n\tprmt.b32 %0, %0, %2, 0x4341;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

template <int OP>
__global__ void __launch_bounds__(1024) kern(uint32_t* out, long long* cyc, int iters, uint32_t seed)
{
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = seed * (threadIdx.x + i * 7919u) + i;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = op<OP>(x[i], x[(i + 1) & 7], x[(i + 2) & 7]);
    }
    __syncthreads();
    long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int OP>
void run(const char* name, int nsm, uint32_t* out, long long* cyc, int ops_per_asm = 1)
{
    const int iters = 4096;
    kern<OP><<<nsm, 1024>>>(out, cyc, iters, 12345u);
    kern<OP><<<nsm, 1024>>>(out, cyc, iters, 12345u);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("%s: error %s\n", name, cudaGetErrorString(e)); return; }
    long long h[1024];
    cudaMemcpy(h, cyc, nsm * sizeof(long long), cudaMemcpyDeviceToHost);
    long long mx = 0;
    for (int i = 0; i < nsm; i++) mx = h[i] > mx ? h[i] : mx;
    double ops = 1024.0 * iters * 8 * ops_per_asm;
    printf("%-22s %7.1f results/clk/SM\n", name, ops / (double)mx);
}

// L2 reduction throughput: every thread adds into its own 16-byte slot of an
// L2-resident buffer (n_slots slots, grid-stride), `iters` times.
__global__ void red_v4f16x2(uint4* buf, size_t n_slots, int iters)
{
    size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t one = 0x3c003c00u;   // (1.0, 1.0) in f16x2
    for (int it = 0; it < iters; it++)
        for (size_t i = i0; i < n_slots; i += stride)
            asm volatile("red.global.add.noftz.v4.f16x2 [%0], {%1, %1, %1, %1};" :: "l"(buf + i), "r"(one) : "memory");
}
__global__ void red_u32(uint32_t* buf, size_t n, int iters)
{
    size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; it++)
        for (size_t i = i0; i < n; i += stride)
            asm volatile("red.global.add.u32 [%0], 1;" :: "l"(buf + i) : "memory");
}
__global__ void st_v4(uint4* buf, size_t n_slots, int iters)
{
    size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; it++)
        for (size_t i = i0; i < n_slots; i += stride)
            buf[i] = make_uint4(it, it, it, it);
}

// Latency of one dependent chain (a single warp): cycles per operation.
template <int OP>
__global__ void lat_kernel(uint32_t* out, long long* cyc, int iters, uint32_t seed)
{
    uint32_t x = seed + threadIdx.x, y = seed * 3u + 1u;
    long long t0 = clock64();
    for (int it = 0; it < iters; it++) x = op<OP>(x, y ^ (x & 1u));
    long long t1 = clock64();
    out[threadIdx.x] = x;
    if (threadIdx.x == 0) cyc[0] = t1 - t0;
}

template <int OP>
void lat(const char* name, uint32_t* out, long long* cyc)
{
    const int iters = 4096;
    lat_kernel<OP><<<1, 32>>>(out, cyc, iters, 77u);
    lat_kernel<OP><<<1, 32>>>(out, cyc, iters, 77u);
    cudaDeviceSynchronize();
    long long h = 0;
    cudaMemcpy(&h, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
    printf("latency %-22s %6.1f cycles\n", name, (double)h / iters);
}

void mem_probe(int nsm)
{
    const size_t bytes = 32u << 20;   // 32 MiB: stays in L2
    void* buf;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) { printf("alloc failed\n"); return; }
    cudaMemset(buf, 0, bytes);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 20;
    float ms;
    size_t slots = bytes / 16;
    red_v4f16x2<<<nsm * 4, 512>>>((uint4*)buf, slots, 1);
    cudaEventRecord(e0);
    red_v4f16x2<<<nsm * 4, 512>>>((uint4*)buf, slots, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("red.v4.f16x2 (32 MiB, L2)  %8.1f GB/s payload, %6.1f G red/s\n", bytes * (double)iters / ms / 1e6,
           slots * (double)iters / ms / 1e6);
    red_u32<<<nsm * 4, 512>>>((uint32_t*)buf, bytes / 4, 1);
    cudaEventRecord(e0);
    red_u32<<<nsm * 4, 512>>>((uint32_t*)buf, bytes / 4, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("red.u32     (32 MiB, L2)  %8.1f GB/s payload, %6.1f G red/s\n", bytes * (double)iters / ms / 1e6,
           bytes / 4 * (double)iters / ms / 1e6);
    st_v4<<<nsm * 4, 512>>>((uint4*)buf, slots, 1);
    cudaEventRecord(e0);
    st_v4<<<nsm * 4, 512>>>((uint4*)buf, slots, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("st.v4       (32 MiB, L2)  %8.1f GB/s\n", bytes * (double)iters / ms / 1e6);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) printf("mem probe error %s\n", cudaGetErrorString(e));
    cudaFree(buf);
}

// warp-level (legacy) mma.sync rates: KIND 0 = m16n8k256 b1 and.popc,
// 1 = m16n8k32 e4m3 -> f32, 2 = m16n8k16 f16 -> f32.  VARY: the A operand
// changes every iteration, so a conversion of the operands cannot be hoisted
// out of the loop (with fixed operands it can, and the rate then says
// nothing about a kernel whose operands come from memory).
template <int KIND, bool VARY>
__global__ void __launch_bounds__(512) mma_kern(uint32_t* out, long long* cyc, int iters)
{
    uint32_t a0 = threadIdx.x * 0x9e3779b9u, a1 = a0 ^ 0x5555u, a2 = a0 * 3u, a3 = a1 * 5u, b0 = a0 + 7u, b1 = a1 + 9u;
    const uint32_t m = KIND == 0 ? 0xFFFFFFFFu : 0x3c3c3c3cu;   // finite e4m3 / f16 bit patterns
    a0 &= m; a1 &= m; a2 &= m; a3 &= m; b0 &= m; b1 &= m;
    int c[4][4] = {};
    float f[4][4] = {};
    const long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
        if (VARY) a0 = (a0 ^ ((uint32_t)i & 0x04040404u)) & m;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (KIND == 0)
                asm volatile("mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                             : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                             : "r"(a0), "r"(a1), "r"(a2 + j), "r"(a3), "r"(b0), "r"(b1));
            else if (KIND == 1)
                asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(f[j][0]), "+f"(f[j][1]), "+f"(f[j][2]), "+f"(f[j][3])
                             : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            else
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(f[j][0]), "+f"(f[j][1]), "+f"(f[j][2]), "+f"(f[j][3])
                             : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    const long long t1 = clock64();
    int sum = 0;
    for (int j = 0; j < 4; j++) sum += c[j][0] + c[j][1] + c[j][2] + c[j][3] + (int)(f[j][0] + f[j][1] + f[j][2] + f[j][3]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)sum;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int KIND, bool VARY>
static void run_mma(const char* name, int nsm, uint32_t* out, long long* cyc, double flops_per_mma)
{
    const int iters = 4096;
    mma_kern<KIND, VARY><<<nsm, 512>>>(out, cyc, iters);
    mma_kern<KIND, VARY><<<nsm, 512>>>(out, cyc, iters);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("%s: error %s\n", name, cudaGetErrorString(e)); return; }
    long long h[1024];
    cudaMemcpy(h, cyc, nsm * sizeof(long long), cudaMemcpyDeviceToHost);
    long long mx = 0;
    for (int i = 0; i < nsm; i++) mx = h[i] > mx ? h[i] : mx;
    const double per_clk = 16.0 * iters * 4 / (double)mx;      // 16 warps x iters x 4 per SM
    printf("%-34s %6.3f warp-mma/clk/SM  %8.1f T op/s at 2.07 GHz\n", name, per_clk,
           per_clk * flops_per_mma * nsm * 2.07e9 / 1e12);
}

int main()
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    printf("SMs %d, clock attr %d kHz\n", nsm, clk);
    uint32_t* out;
    long long* cyc;
    cudaMalloc(&out, (size_t)nsm * 1024 * 4);
    cudaMalloc(&cyc, nsm * sizeof(long long));
    run<0>("add.u32", nsm, out, cyc);
    run<19>("sub.u32", nsm, out, cyc);
    run<16>("add.u32 x2 (fusable)", nsm, out, cyc, 2);
    run<1>("min.u32", nsm, out, cyc);
    run<2>("min.u16x2", nsm, out, cyc);
    run<17>("max.u16x2", nsm, out, cyc);
    run<3>("xor.b32", nsm, out, cyc);
    run<4>("prmt.b32", nsm, out, cyc);
    run<5>("popc.b32", nsm, out, cyc);
    run<6>("shfl.bfly", nsm, out, cyc);
    run<7>("mad.lo.u32", nsm, out, cyc);
    run<8>("min.f16x2", nsm, out, cyc);
    run<9>("add.f16x2", nsm, out, cyc);
    run<10>("fma.f16x2", nsm, out, cyc);
    run<14>("min.bf16x2", nsm, out, cyc);
    run<11>("min.f32", nsm, out, cyc);
    run<15>("min.f32 3-input", nsm, out, cyc);
    run<12>("add.f32", nsm, out, cyc);
    run<13>("__vminu4", nsm, out, cyc);
    run<18>("vadd2", nsm, out, cyc);
    run<20>("min.u16x2 + min.f16x2", nsm, out, cyc, 2);
    run<24>("min.u32 + min.f32", nsm, out, cyc, 2);
    run<22>("min.u16x2 + add.u32", nsm, out, cyc, 2);
    run<23>("min.u16x2 + add.f16x2", nsm, out, cyc, 2);
    run<26>("min.f16x2 + add.f16x2", nsm, out, cyc, 2);
    run<25>("min.u16x2 + prmt", nsm, out, cyc, 2);
    run<27>("min.u16x2 + mad.lo.u32", nsm, out, cyc, 2);
    run<21>("redux.sync.min", nsm, out, cyc);
    run<28>("vimin3.u16x2", nsm, out, cyc);
    run<29>("viaddmin.u16x2", nsm, out, cyc);
    run<30>("vimin3.u32", nsm, out, cyc);
    run<31>("vimin3.s16x2", nsm, out, cyc);
    run<32>("vimin3.u16x2 + min.u16x2", nsm, out, cyc, 2);
    run<33>("vimin3.u16x2 + prmt", nsm, out, cyc, 2);
    run<34>("vimin3.u16x2 + add.u32", nsm, out, cyc, 2);
    run<35>("viaddmin.u16x2 + min.u16x2", nsm, out, cyc, 2);
    run<36>("and + xor", nsm, out, cyc, 2);
    run<37>("shr + xor", nsm, out, cyc, 2);
    run<38>("vimin3.u16x2 + lop3", nsm, out, cyc, 2);
    run<39>("vimin3.u16x2 + mad.lo", nsm, out, cyc, 2);
    run<40>("vimin3.u16x2 + shr", nsm, out, cyc, 2);
    run<41>("add + sub (iadd3)", nsm, out, cyc, 2);
    run<42>("vimin3.u16x2 + add + sub", nsm, out, cyc, 3);
    run<43>("prmt + lop3", nsm, out, cyc, 2);
    run<44>("shf.r.wrap (funnel)", nsm, out, cyc);
    run<45>("min.u16x2 + shf.r", nsm, out, cyc, 2);
    run<46>("vimin3.u16x2 + min.f16x2", nsm, out, cyc, 2);
    run<47>("lop3", nsm, out, cyc);
    run<48>("min.f16x2 + prmt", nsm, out, cyc, 2);
    run<49>("min.f16x2 + shf.r", nsm, out, cyc, 2);
    run<50>("vimin3 + min.f16x2 + add", nsm, out, cyc, 3);
    run<51>("add.f16x2 + lop3", nsm, out, cyc, 2);
    run<52>("add.f16x2 + prmt", nsm, out, cyc, 2);
    lat<1>("min.u32", out, cyc);
    lat<2>("min.u16x2", out, cyc);
    lat<4>("prmt", out, cyc);
    lat<0>("add.u32", out, cyc);
    lat<6>("shfl.bfly", out, cyc);
    lat<21>("redux.sync.min", out, cyc);
    lat<5>("popc", out, cyc);
    lat<28>("vimin3.u16x2", out, cyc);
    lat<29>("viaddmin.u16x2", out, cyc);
    mem_probe(nsm);
    if (nsm <= 1024) {
        run_mma<0, false>("mma b1.and.popc m16n8k256", nsm, out, cyc, 16.0 * 8 * 256 * 2);
        run_mma<0, true>("mma b1.and.popc m16n8k256, A varies", nsm, out, cyc, 16.0 * 8 * 256 * 2);
        run_mma<1, false>("mma e4m3 m16n8k32", nsm, out, cyc, 16.0 * 8 * 32 * 2);
        run_mma<1, true>("mma e4m3 m16n8k32, A varies", nsm, out, cyc, 16.0 * 8 * 32 * 2);
        run_mma<2, false>("mma f16 m16n8k16", nsm, out, cyc, 16.0 * 8 * 16 * 2);
        run_mma<2, true>("mma f16 m16n8k16, A varies", nsm, out, cyc, 16.0 * 8 * 16 * 2);
    }
    cudaFree(out);
    cudaFree(cyc);
    return 0;
}
