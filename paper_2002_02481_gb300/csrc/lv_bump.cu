// lv_bump.cu -- batched central bump-and-reprice (arXiv 2002.02481, Sec. III):
// every grid value sigma_ij moved by +eps/2 and -eps/2, and S0 by
// +-eps_S/2, each pair of scenarios priced on the same random numbers, the
// difference divided by the bump. This is the baseline the adjoint is
// compared against.
//
// Scenario s of the 3 + 2 I J scenarios:
//   s = 0, 1             S0 + eps_S/2, S0 - eps_S/2
//   s = 2 + 2e + b       node e = i * J + j (spot-major), b = 0: +eps/2, 1: -eps/2
//   s = 2 + 2 I J        the unbumped model (price)
// so every pair (2q, 2q + 1) lands in the same thread and accumulates into
// slot q = s / 2 of a per-block binary64 row [2 + I J].
//
// A block handles work items (tile of blockDim.x paths, group of M
// scenarios); each thread runs one path for the M scenarios of its group on
// shared Philox normals. Bilinear interpolation is linear in the node
// values, so a bumped sigma is the unbumped one plus +-eps/2 times that
// node's bilinear weight at (S, t); the weight is evaluated only when the
// (warp-uniform) time cell touches the node's time column.
#include <math.h>

#include "lv_device.cuh"

namespace lv {

namespace {

__host__ __device__ inline size_t a16(size_t b) { return (b + 15) & ~size_t(15); }

struct BumpSmem {
    size_t tab, sig, node, ab, acc, tile, total;
};

__host__ __device__ inline BumpSmem bump_layout(int I, int Je, int N, int row_words)
{
    BumpSmem L;
    size_t o = 0;
    L.tab = o;  o += a16(sizeof(int4) * (size_t)N);
    L.sig = o;  o += a16(sizeof(float2) * (size_t)Je * (I - 1));
    L.node = o; o += a16(sizeof(float) * (size_t)I);
    L.ab = o;   o += a16(sizeof(float2) * (size_t)I);
    L.acc = o;  o += a16(sizeof(double) * (size_t)row_words);
    L.tile = o; o += a16(sizeof(int) * 2);
    L.total = o;
    return L;
}

constexpr int kM = 8;   // scenario slots per thread (even: pairs never split)

__global__ void __launch_bounds__(256) bump_kernel(const __grid_constant__ BumpParams Q)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const McParams& P = Q.mc;
    const int B = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    const BumpSmem L = bump_layout(P.I, P.Je, P.N, Q.row_words);
    int4* s_tab = reinterpret_cast<int4*>(smem + L.tab);
    float2* s_sig = reinterpret_cast<float2*>(smem + L.sig);
    float* s_node = reinterpret_cast<float*>(smem + L.node);
    float2* s_ab = reinterpret_cast<float2*>(smem + L.ab);
    double* s_acc = reinterpret_cast<double*>(smem + L.acc);
    int* s_tile = reinterpret_cast<int*>(smem + L.tile);

    for (int e = tid; e < P.Je * (P.I - 1); e += B) s_sig[e] = P.sig2[e];
    for (int e = tid; e < P.I; e += B) s_node[e] = P.node[e];
    for (int e = tid; e < P.I - 1; e += B) s_ab[e] = P.ab[e];
    for (int n = tid; n < P.N; n += B) s_tab[n] = step_time(P, n);
    for (int e = tid; e < Q.row_words; e += B) s_acc[e] = 0.0;
    if (tid == 0) s_tile[0] = (int)atomicAdd(P.tile_counter, 1u);
    __syncthreads();
    SmemGrid g{ s_tab, s_sig, s_node, s_ab };

    const long long n_items = (long long)P.n_tiles * Q.n_groups;
    int it = 0;
    long long item = s_tile[0];
    while (item < n_items) {
        const int grp = (int)(item % Q.n_groups);
        const long long tile = item / Q.n_groups;
        const long long r = tile * B + tid;
        const bool active = r < P.n_paths;
        const int s_first = grp * kM;

        // per slot: start, bumped node (row offset j*I and spot index), signed half bump
        float x[kM];
        int b_i[kM], b_row[kM];
        float b_h[kM];
        bool used[kM];
#pragma unroll
        for (int k = 0; k < kM; ++k) {
            const int s = s_first + k;
            used[k] = s < Q.n_scen;
            x[k] = s == 0 ? Q.x0_up : (s == 1 ? Q.x0_dn : P.x0);
            b_i[k] = -1;
            b_row[k] = -1;
            b_h[k] = 0.0f;
            if (s >= 2 && s < Q.n_scen - 1) {
                const int e = (s - 2) >> 1;
                b_i[k] = e / P.J;
                b_row[k] = (e - b_i[k] * P.J) * P.I;
                b_h[k] = ((s - 2) & 1) ? -Q.eps_half : Q.eps_half;
            }
        }
        float V[kM];
        if (active) {
            const unsigned long long p = (unsigned long long)(P.path_begin + r);
            const uint32_t c1 = (uint32_t)p;
            const uint32_t c2 = ((uint32_t)(p >> 32) & 0xffffu) | (P.stream_id << 16);
            float z[4];
            for (int n0 = 0; n0 < P.N; n0 += 4) {
                normals4((uint32_t)(n0 >> 2), c1, c2, P.k0, P.k1, z);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int n = n0 + q;
                    if (n >= P.N) break;
                    const int4 tb = g.tab[n];
                    const float v = __int_as_float(tb.w);
#pragma unroll
                    for (int k = 0; k < kM; ++k) {
                        if (!used[k]) continue;
                        StepEval e = eval_sigma<false>(P, g, x[k], tb);
                        // time weight of the bumped node: column j (1 - v) or j + 1 (v)
                        if (b_row[k] == tb.z || b_row[k] == tb.z + P.I) {
                            const float wt = b_row[k] == tb.z ? 1.0f - v : v;
                            const float ws = b_i[k] == e.i ? 1.0f - e.u : (b_i[k] == e.i + 1 ? e.u : 0.0f);
                            e.sigma = fmaf(b_h[k], ws * wt, e.sigma);
                        }
                        x[k] = euler_step(P, x[k], e.sigma, z[q]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kM; ++k) {
                const float itm = P.phi * (exp2f(x[k]) - P.K);
                V[k] = itm > 0.0f ? P.disc * itm : 0.0f;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kM; ++k) V[k] = 0.0f;
        }
        // pair differences (and the lone unbumped scenario), warp-reduced in binary64
#pragma unroll
        for (int k = 0; k < kM; k += 2) {
            const int s = s_first + k;
            if (s < Q.n_scen) {     // block-uniform
                double d = (s + 1 < Q.n_scen) ? (double)V[k] - (double)V[k + 1] : (double)V[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
                if (lane == 0) atomicAdd(&s_acc[s >> 1], d);
            }
        }
        if (tid == 0) s_tile[(it + 1) & 1] = (int)atomicAdd(P.tile_counter, 1u);
        __syncthreads();
        ++it;
        item = s_tile[it & 1];
    }
    double* row = Q.partials + (size_t)blockIdx.x * Q.row_words;
    for (int e = tid; e < Q.row_words; e += B) row[e] = s_acc[e];
}

constexpr int kBumpRowsPerChunk = 32;

__global__ void bump_reduce_rows(const double* __restrict__ partials, int G, int row_words,
                                 double* __restrict__ chunks)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= row_words) return;
    const int r0 = blockIdx.y * kBumpRowsPerChunk;
    const int r1 = min(G, r0 + kBumpRowsPerChunk);
    double s = 0.0;
    for (int r = r0; r < r1; ++r) s += partials[(size_t)r * row_words + col];
    chunks[(size_t)blockIdx.y * row_words + col] = s;
}

// out = [price, delta, 0, vega (spot-major)]
__global__ void bump_finalize(const double* __restrict__ chunks, int n_chunks, int row_words, int IJ,
                              long long n_paths, double eps, double eps_S, double* __restrict__ out,
                              unsigned int* tile_counter)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= row_words) return;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += chunks[(size_t)c * row_words + col];
    const double P = (double)n_paths;
    if (col == 0) {
        out[1] = s / (P * eps_S);
        out[2] = 0.0;
        if (tile_counter) *tile_counter = 0u;
    } else if (col <= IJ) {
        out[3 + (col - 1)] = s / (P * eps);
    } else {
        out[0] = s / P;
    }
}

}  // namespace

size_t bump_smem_bytes(int I, int Je, int N, int row_words)
{
    return bump_layout(I, Je, N, row_words).total;
}

int bump_slots_per_thread() { return kM; }

cudaError_t bump_occupancy(int block, size_t smem, int* bps)
{
    cudaError_t e = cudaFuncSetAttribute(bump_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, bump_kernel, block, smem);
}

cudaError_t launch_bump(const BumpParams& b, int grid, int block, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(bump_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    bump_kernel<<<grid, block, smem, s>>>(b);
    return cudaGetLastError();
}

int bump_chunks(int G) { return (G + kBumpRowsPerChunk - 1) / kBumpRowsPerChunk; }

cudaError_t launch_bump_finalize(const double* partials, int G, int row_words, double* chunks, int IJ,
                                 long long n_paths, double eps, double eps_S, double* out,
                                 unsigned int* tile_counter, cudaStream_t s)
{
    const int nch = bump_chunks(G);
    dim3 g1((row_words + 255) / 256, nch);
    bump_reduce_rows<<<g1, 256, 0, s>>>(partials, G, row_words, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bump_finalize<<<(row_words + 255) / 256, 256, 0, s>>>(chunks, nch, row_words, IJ, n_paths, eps, eps_S,
                                                          out, tile_counter);
    return cudaGetLastError();
}

}  // namespace lv
