// peaks.cu -- pipe-throughput microbenchmarks used as roofline denominators by bench.py:
// MUFU ex2 (the transcendental unit that evaluates every proposal weight), FP32 FMA, packed
// FP32x2 FMA, FP64 FMA, the wide-multiply rate of the integer pipe, and whole
// Philox4x32-10 blocks (the method's random numbers), each as sustained operations per second
// over the whole GPU with enough independent chains per thread to hide latency.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

__global__ void ex2_kernel(float *out, int iters)
{
    float v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = -0.001f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[i]));
            v[i] = y - 1.0001f;   // stays in (-1, 0]
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += v[i];
    if (s == 12345.f) out[0] = s;
}

__global__ void fma_kernel(float *out, int iters)
{
    float v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) v[i] = fmaf(v[i], 0.9999f, 0.0001f);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += v[i];
    if (s == 12345.f) out[0] = s;
}

__global__ void fma2_kernel(float *out, int iters)
{
    unsigned long long v[kChains];
    unsigned long long a, b;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(0.9999f), "f"(0.9998f));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(0.0001f), "f"(0.0002f));
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float x = (float)(threadIdx.x + i);
        asm("mov.b64 %0, {%1, %1};" : "=l"(v[i]) : "f"(x));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[i]) : "l"(a), "l"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v[i]));
        s += x + y;
    }
    if (s == 12345.f) out[0] = s;
}

__global__ void dfma_kernel(float *out, int iters)
{
    double v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) v[i] = fma(v[i], 0.9999, 0.0001);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += v[i];
    if (s == 12345.0) out[0] = (float)s;
}

// 32 x 32 -> 64-bit products (low and high words), the arithmetic half of a Philox round.
__global__ void mulwide_kernel(float *out, int iters)
{
    uint32_t v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = threadIdx.x * 2654435761u + (uint32_t)i + 1u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            const uint64_t p = (uint64_t)v[i] * 0xD2511F53u;
            v[i] = (uint32_t)p + (uint32_t)(p >> 32);
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= v[i];
    if (s == 12345u) out[0] = (float)s;
}

// Whole Philox4x32-10 blocks (Salmon et al., SC'11), two independent counters per thread, ten
// rounds each: the generator's own throughput, in blocks of four words per second.
__global__ void philox_kernel(float *out, int iters)
{
    uint32_t c[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        c[j][0] = threadIdx.x;
        c[j][1] = blockIdx.x;
        c[j][2] = (uint32_t)j;
        c[j][3] = 0u;
    }
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            uint32_t x0 = c[j][0], x1 = c[j][1], x2 = c[j][2], x3 = c[j][3] + (uint32_t)it;
            uint32_t k0 = 0x12345678u, k1 = 0x9ABCDEF0u;
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                const uint64_t p0 = (uint64_t)x0 * 0xD2511F53u;
                const uint64_t p1 = (uint64_t)x2 * 0xCD9E8D57u;
                const uint32_t n0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
                const uint32_t n2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
                x1 = (uint32_t)p1;
                x3 = (uint32_t)p0;
                x0 = n0;
                x2 = n2;
                k0 += 0x9E3779B9u;
                k1 += 0xBB67AE85u;
            }
            acc ^= x0 ^ x1 ^ x2 ^ x3;
        }
    }
    if (acc == 12345u) out[0] = (float)acc;
}

template <typename K>
double rate(K kern, int blocks, int threads, int iters, double ops_per_thread_iter)
{
    float *buf = nullptr;
    if (cudaMalloc(&buf, 16) != cudaSuccess) return -1.0;
    kern<<<blocks, threads>>>(buf, 16);   // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    kern<<<blocks, threads>>>(buf, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    return (double)blocks * threads * iters * ops_per_thread_iter / (ms * 1e-3);
}

}  // namespace

// out[0] ex2/s, out[1] FP32 FMA/s (one FMA = 1 op), out[2] FP32x2 FMA lanes/s, out[3] FP64 FMA/s,
// out[4] 32 x 32 -> 64-bit products/s, out[5] Philox4x32-10 blocks/s.
extern "C" int mcmc_pipe_peaks(double *out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    out[0] = rate(ex2_kernel, blocks, threads, 4096, kChains);
    out[1] = rate(fma_kernel, blocks, threads, 16384, kChains);
    out[2] = rate(fma2_kernel, blocks, threads, 8192, 2.0 * kChains);
    out[3] = rate(dfma_kernel, blocks, threads, 256, kChains);
    out[4] = rate(mulwide_kernel, blocks, threads, 4096, kChains);
    out[5] = rate(philox_kernel, blocks, threads, 256, 2.0);
    return 0;
}
