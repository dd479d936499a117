// lv_debug.cu -- test-facing kernels: the Philox words and normals the
// Monte Carlo kernels draw, and their per-step time table (Sec. IV-A,
// IV-B, IV-D of arXiv 2002.02481), through the same device functions.
#include "lv_device.cuh"

namespace lv {

namespace {

__global__ void normals_kernel(uint32_t k0, uint32_t k1, uint32_t stream_id, const long long* __restrict__ paths,
                               const uint32_t* __restrict__ blocks, long long n, uint32_t* __restrict__ words,
                               float* __restrict__ z)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const unsigned long long p = (unsigned long long)paths[e];
    const uint32_t c1 = (uint32_t)p;
    const uint32_t c2 = ((uint32_t)(p >> 32) & 0xffffu) | (stream_id << 16);
    uint32_t w0 = blocks[e], w1 = c1, w2 = c2, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, k0, k1);
    words[4 * e + 0] = w0;
    words[4 * e + 1] = w1;
    words[4 * e + 2] = w2;
    words[4 * e + 3] = w3;
    float zz[4];
    normals4(blocks[e], c1, c2, k0, k1, zz);
    for (int q = 0; q < 4; ++q) z[4 * e + q] = zz[q];
}

__global__ void time_table_kernel(const McParams P, int* __restrict__ out_j, float* __restrict__ out_v)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= P.N) return;
    const int4 tb = step_time(P, n);
    out_j[n] = tb.z / P.I;                    // tb.z is the bucket row j I
    out_v[n] = __int_as_float(tb.w);
}

}  // namespace

cudaError_t launch_debug_normals(uint64_t seed, uint32_t stream_id, const long long* paths, const uint32_t* blocks,
                                 long long n, uint32_t* words, float* z, cudaStream_t s)
{
    const int threads = 256;
    normals_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), stream_id, paths, blocks, n, words, z);
    return cudaGetLastError();
}

cudaError_t launch_debug_time_table(const McParams& P, int* out_j, float* out_v, cudaStream_t s)
{
    const int threads = 256;
    time_table_kernel<<<(P.N + threads - 1) / threads, threads, 0, s>>>(P, out_j, out_v);
    return cudaGetLastError();
}

}  // namespace lv
