// lv_internal.h -- interface between the host runtime (lv_api.cu) and the
// device kernels (lv_kernels.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lv {

// Output layout of the finalized result (same values as LV_OUT_* in lv.h).
constexpr int LV_OUT_PRICE_DEV = 0;
constexpr int LV_OUT_DELTA_DEV = 1;
constexpr int LV_OUT_STDERR_DEV = 2;

// Everything a Monte Carlo launch reads, passed by value as a
// __grid_constant__ kernel parameter.
struct McParams {
    // grid (device copies, binary32)
    const float* sig;      // [Je * I] time-major: sigma_ij at j * I + i; Je = max(J, 2)
    const float* node;     // [I] spot nodes s_i
    const float2* ab;      // [I - 1] (1 / (s_{i+1} - s_i), -s_i / (s_{i+1} - s_i))
    const double* tau;     // [J] time nodes
    int I, J, Je;
    int log_uniform;       // spot nodes equally spaced in ln S
    float cell_scale;      // 1 / d(ln s)
    float cell_shift;      // -ln(s_0) / d(ln s)
    float s_lo, s_hi;      // s_0, s_{I-1}

    // option and scheme
    float x0;              // ln S0
    float rdt;             // r dt
    float hdt;             // dt / 2
    float dt;
    float sqdt;            // sqrt(dt)
    float K;
    float disc;            // e^{-rT}
    float phi;             // +1 call, -1 put
    double dt_d;           // dt in binary64 for the time table
    int N;                 // steps

    // random numbers
    uint32_t k0, k1;       // Philox key = seed
    uint32_t stream_id;
    long long path_begin;
    long long n_paths;

    // work decomposition and scratch
    int n_tiles;           // ceil(n_paths / blockDim.x)
    unsigned int* tile_counter;   // zero before the launch, reset by the finalize
    double* partials;      // [gridDim.x][row_words] per-block level-2 accumulators
    int row_words;         // 3 + Je * I
    float* ckpt;           // [n_ck][gridDim.x * blockDim.x] checkpoints of x
    int n_ck;
    int acc_mode;          // 0 FP64, 1 Kahan

    // optional per-path outputs (debug entry point)
    float* dbg_xN;
    float* dbg_V;
    float* dbg_xbar0;
};

struct FinalizeParams {
    const double* partials;
    int G;                 // rows
    int row_words;
    int I, J;
    int acc_mode;
    long long n_paths;
    double S0;
    int want_sums;         // 1: raw sums, 0: price / delta / stderr / vega
    double* chunks;        // [finalize_chunks(G)][row_words] stage-1 sums
    double* out;           // [3 + I * J]
    unsigned int* tile_counter;  // reset to 0
};

int finalize_chunks(int G);

size_t mc_smem_bytes(int I, int Je, int N, int block, bool greeks);

// Launchers; return cudaSuccess or the launch error.
cudaError_t launch_mc(const McParams& p, int grid, int block, int k, bool greeks, size_t smem,
                      cudaStream_t s);
cudaError_t launch_finalize(const FinalizeParams& f, cudaStream_t s);
cudaError_t mc_occupancy(int block, int k, bool greeks, size_t smem, int* blocks_per_sm);

}  // namespace lv
