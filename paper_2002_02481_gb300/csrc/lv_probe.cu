// lv_probe.cu -- measured issue rates of the SM pipes the Monte Carlo
// kernels spend their time in: the roofline denominators of a path that is
// bound by arithmetic, not by memory. Each probe kernel runs, per thread,
// eight chains of one instruction kind (inline PTX) on 8 blocks of 256
// threads per SM, and is timed with CUDA events; the rate is operations
// (thread-instructions) per second over the whole GPU at the clock it ran
// at. Floating-point chains cannot be reassociated; in the integer chains
// every step takes an operand from the neighbouring chain (so that no chain
// of bitwise or modular operations on fixed operands collapses into fewer
// instructions) while the eight chains still issue independently within an
// iteration.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lv.h"
#include "lv_internal.h"

namespace lv {

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;      // unrolled by kChains: kChains * kIters operations per thread

template <int OP>
__device__ __forceinline__ void step_f(float& x, float a)
{
    if (OP == LV_PIPE_FFMA) asm volatile("fma.rn.f32 %0, %0, %1, %1;" : "+f"(x) : "f"(a));
    if (OP == LV_PIPE_MUFU_EX2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x));
    if (OP == LV_PIPE_MUFU_LG2) asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(x));
    if (OP == LV_PIPE_MUFU_SIN) asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(x));
    if (OP == LV_PIPE_MUFU_COS) asm volatile("cos.approx.ftz.f32 %0, %0;" : "+f"(x));
    if (OP == LV_PIPE_MUFU_SQRT) asm volatile("sqrt.approx.ftz.f32 %0, %0;" : "+f"(x));
}

template <int OP>
__device__ __forceinline__ void step_i(uint32_t& x, uint32_t y, uint32_t b)
{
    if (OP == LV_PIPE_IMAD) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(y), "r"(b));
    if (OP == LV_PIPE_LOP3) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(y), "r"(b));
}

template <int OP>
__global__ void __launch_bounds__(256) probe_f(float a, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 0.25f + 0.01f * (float)(k + threadIdx.x % 7);
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int k = 0; k < kChains; ++k) step_f<OP>(x[k], a);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;       // keeps the chains live
}

template <int OP>
__global__ void __launch_bounds__(256) probe_i(uint32_t a, uint32_t b, uint32_t* sink)
{
    uint32_t x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (threadIdx.x + a) * 2654435761u + (uint32_t)k;
    for (int it = 0; it < kIters; ++it) {
        uint32_t y[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) y[k] = x[(k + 1) % kChains];       // this iteration's operands
#pragma unroll
        for (int k = 0; k < kChains; ++k) step_i<OP>(x[k], y[k], b);
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= x[k];
    if (s == 0x12345678u) sink[0] = s;
}

// 32 x 32 -> 64-bit multiply-add (the Philox product): acc += x * a in 64 bits.
__global__ void __launch_bounds__(256) probe_imad_wide(uint32_t a, unsigned long long* sink)
{
    unsigned long long acc[kChains];
    uint32_t x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        acc[k] = k;
        x[k] = threadIdx.x * 2246822519u + (uint32_t)k;
    }
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = (uint32_t)acc[(k + 1) % kChains];   // this iteration's operands
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[k]) : "r"(x[k]), "r"(a));
    }
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= acc[k];
    if (s == 0x123456789ull) sink[0] = s;
}

template <typename F>
cudaError_t time_best(F launch, int reps, float* best_ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    launch();                             // warm-up
    *best_ms = 1e30f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, 0);
        launch();
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < *best_ms) *best_ms = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

cudaError_t measure_pipe_peaks(double* out)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void* sink = nullptr;
    e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess) return e;
    const int grid = 8 * sms, block = 256;
    const double ops = (double)grid * block * kChains * kIters;
    float* fs = static_cast<float*>(sink);
    uint32_t* is = static_cast<uint32_t*>(sink);
    auto rate = [&](int slot, auto launch) {
        float ms = 0.0f;
        if (e == cudaSuccess) e = time_best(launch, 3, &ms);
        out[slot] = e == cudaSuccess ? ops / (ms * 1e-3) : 0.0;
    };
    rate(LV_PIPE_FFMA, [&] { probe_f<LV_PIPE_FFMA><<<grid, block>>>(0.999f, fs); });
    rate(LV_PIPE_MUFU_EX2, [&] { probe_f<LV_PIPE_MUFU_EX2><<<grid, block>>>(0.0f, fs); });
    rate(LV_PIPE_MUFU_LG2, [&] { probe_f<LV_PIPE_MUFU_LG2><<<grid, block>>>(0.0f, fs); });
    rate(LV_PIPE_MUFU_SIN, [&] { probe_f<LV_PIPE_MUFU_SIN><<<grid, block>>>(0.0f, fs); });
    rate(LV_PIPE_MUFU_COS, [&] { probe_f<LV_PIPE_MUFU_COS><<<grid, block>>>(0.0f, fs); });
    rate(LV_PIPE_MUFU_SQRT, [&] { probe_f<LV_PIPE_MUFU_SQRT><<<grid, block>>>(0.0f, fs); });
    rate(LV_PIPE_IMAD, [&] { probe_i<LV_PIPE_IMAD><<<grid, block>>>(0x9E3779B9u, 0x7F4A7C15u, is); });
    rate(LV_PIPE_IMAD_WIDE, [&] {
        probe_imad_wide<<<grid, block>>>(0xD2511F53u, static_cast<unsigned long long*>(sink));
    });
    rate(LV_PIPE_LOP3, [&] { probe_i<LV_PIPE_LOP3><<<grid, block>>>(0x9E3779B9u, 0xBB67AE85u, is); });
    cudaFree(sink);
    return e;
}

}  // namespace lv
