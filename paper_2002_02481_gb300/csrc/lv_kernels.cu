// lv_kernels.cu -- the main model's Monte Carlo kernels (instantiated from
// lv_mc.cuh), the launchers that route every model to its translation unit,
// and the fixed-order binary64 finalize (level 3 of the bucket sums).
#include "lv_mc.cuh"

namespace lv {

namespace {

// Programmatic dependent launch: the level-3 stages are launched so that
// their blocks may become resident while the kernel before them is still
// running; griddepcontrol.wait returns once that kernel has completed and
// its memory operations are visible, and launch_dependents lets the next
// stage be scheduled early in the same way.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void release_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Level 3, stage 1: rows [chunk * RCH, (chunk + 1) * RCH) of one column
// summed by one thread in a fixed pairwise order, into one binary64 row per
// chunk. All the chunk's loads are issued before the first add, and the tree
// keeps the chain of dependent binary64 adds (64 cycles each on this part)
// five deep. Binary64 arithmetic runs at a small fraction of the binary32
// rate here, so both stages launch one warp per block and 32 columns per
// warp: the adds spread evenly over every SM.
constexpr int kRowsPerChunk = 32;

__device__ __forceinline__ double tree_sum32(double (&v)[32])
{
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; ++i) v[i] += v[i + w];
    return v[0];
}

// A nonzero *flag (the tangent-ratio adjoint met a vanishing 1 + g_n) makes
// every sum, and so every output, NaN.
__global__ void __launch_bounds__(32) reduce_rows_kernel(const double* __restrict__ partials, int G, int row_words,
                                                          const unsigned int* flag, double* __restrict__ chunks)
{
    release_dependents();
    wait_prior_grid();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= row_words) return;
    const int r0 = blockIdx.y * kRowsPerChunk;
    double v[kRowsPerChunk];
#pragma unroll
    for (int q = 0; q < kRowsPerChunk; ++q)
        v[q] = r0 + q < G ? partials[(size_t)(r0 + q) * row_words + col] : 0.0;
    double s = tree_sum32(v);
    if (flag && *flag) s = __longlong_as_double(0x7ff8000000000000ll);
    chunks[(size_t)blockIdx.y * row_words + col] = s;
}

// Level 3, stage 2: the chunks of one column summed in the same way (32 at a
// time, the groups in order); outputs in the ABI layout (vega spot-major),
// price statistics from the scalar sums. With `extra` the last two columns of
// the rows are the sums of d V / d r and d V / d T, written after the vegas
// (out[3 + I J], out[4 + I J]).
__global__ void __launch_bounds__(32) finalize_kernel(const double* __restrict__ chunks, int n_chunks, int row_words,
                                                       int I, int J, long long n_paths, double S0, int want_sums,
                                                       int extra, double* __restrict__ out,
                                                       unsigned int* tile_counter, unsigned int* flag)
{
    wait_prior_grid();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    for (int c0 = 0; c0 < n_chunks; c0 += kRowsPerChunk) {
        double v[kRowsPerChunk];
#pragma unroll
        for (int q = 0; q < kRowsPerChunk; ++q)
            v[q] = (col < row_words && c0 + q < n_chunks) ? chunks[(size_t)(c0 + q) * row_words + col] : 0.0;
        s += tree_sum32(v);
    }
    const double sv2 = __shfl_sync(0xffffffffu, s, 1);      // column 1 (sum of V^2), in block 0
    if (col >= row_words) return;
    const double P = (double)n_paths;
    if (col < 3) {
        if (want_sums) {
            out[col] = s;
        } else if (col == 0) {
            const double mean = s / P;
            const double var = n_paths > 1 ? (sv2 / P - mean * mean) * P / (P - 1.0) : 0.0;
            out[LV_OUT_PRICE_DEV] = mean;
            out[LV_OUT_STDERR_DEV] = (var > 0.0 || var != var) ? sqrt(var / P) : 0.0;   // NaN stays NaN
        } else if (col == 2) {
            out[LV_OUT_DELTA_DEV] = s / (P * S0);
        }
        if (col == 0 && tile_counter) *tile_counter = 0u;
        if (col == 0 && flag) *flag = 0u;
        return;
    }
    if (extra && col >= row_words - 2) {
        out[3 + I * J + (col - (row_words - 2))] = want_sums ? s : s / P;
        return;
    }
    const int e = col - 3;             // time-major bucket j * I + i
    const int j = e / I, i = e - j * I;
    if (j >= J) return;                // padding row of a one-column grid
    out[3 + i * J + j] = want_sums ? s : s / P;
}

}  // namespace

size_t mc_smem_bytes(int I, int Je, int N, int block, bool greeks, bool grid_smem, bool extra, int ppl)
{
    return smem_layout(I, Je, N, block, greeks, grid_smem, extra, ppl).total;
}

int ring_slots_per_warp() { return kRing * kTile; }
int paths_per_tile(bool greeks) { return greeks ? kTile : kPriceTile; }

cudaError_t launch_mc(const McParams& p, int grid, int block, int k, bool greeks, size_t smem,
                      cudaStream_t s)
{
    switch (p.model) {
    case 0: return launch_model_impl<0>(p, grid, block, k, greeks, smem, s);
    case 1: return launch_mc_model1(p, grid, block, k, greeks, smem, s);
    case 2: return launch_mc_model2(p, grid, block, k, greeks, smem, s);
    case 3: return launch_mc_model3(p, grid, block, k, greeks, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t mc_occupancy(int block, int k, bool greeks, int acc, bool dbg, bool grid_smem, int method, int model,
                         bool extra, size_t smem, int* bps, int ppl)
{
    switch (model) {
    case 0: return occupancy_model_impl<0>(block, k, greeks, acc, dbg, grid_smem, method, extra, smem, bps, ppl);
    case 1: return mc_occupancy_model1(block, k, greeks, acc, dbg, grid_smem, method, extra, smem, bps, ppl);
    case 2: return mc_occupancy_model2(block, k, greeks, acc, dbg, grid_smem, method, extra, smem, bps, ppl);
    case 3: return mc_occupancy_model3(block, k, greeks, acc, dbg, grid_smem, method, extra, smem, bps, ppl);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_finalize(const FinalizeParams& f, cudaStream_t s)
{
    const int n_chunks = (f.G + kRowsPerChunk - 1) / kRowsPerChunk;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((f.row_words + 31) / 32, n_chunks);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const unsigned int* flag_c = f.flag;
    cudaError_t e = cudaLaunchKernelEx(&cfg, reduce_rows_kernel, f.partials, f.G, f.row_words, flag_c, f.chunks);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3((f.row_words + 31) / 32);
    return cudaLaunchKernelEx(&cfg, finalize_kernel, (const double*)f.chunks, n_chunks, f.row_words, f.I, f.J,
                              f.n_paths, f.S0, f.want_sums, f.extra, f.out, f.tile_counter, f.flag);
}

int finalize_chunks(int G) { return (G + kRowsPerChunk - 1) / kRowsPerChunk; }

namespace {

// Raw sums (LV_SUM_* layout, vega spot-major) -> price, delta, stderr, vega.
__global__ void finalize_sums_kernel(const double* __restrict__ sums, int IJ, long long n_paths, double S0,
                                     double* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const double P = (double)n_paths;
    if (e == 0) {
        const double mean = sums[0] / P;
        const double var = n_paths > 1 ? (sums[1] / P - mean * mean) * P / (P - 1.0) : 0.0;
        out[LV_OUT_PRICE_DEV] = mean;
        out[LV_OUT_STDERR_DEV] = (var > 0.0 || var != var) ? sqrt(var / P) : 0.0;   // NaN stays NaN
        out[LV_OUT_DELTA_DEV] = sums[2] / (P * S0);
    }
    if (e < IJ) out[3 + e] = sums[3 + e] / P;
}

}  // namespace

cudaError_t launch_finalize_sums(const double* sums, int IJ, long long n_paths, double S0, double* out,
                                 cudaStream_t s)
{
    finalize_sums_kernel<<<(IJ + 255) / 256, 256, 0, s>>>(sums, IJ, n_paths, S0, out);
    return cudaGetLastError();
}

}  // namespace lv
