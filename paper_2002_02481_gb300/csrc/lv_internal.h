// lv_internal.h -- interface between the host runtime (lv_api.cu) and the
// device kernels (lv_kernels.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace lv {

// Output layout of the finalized result (same values as LV_OUT_* in lv.h).
constexpr int LV_OUT_PRICE_DEV = 0;
constexpr int LV_OUT_DELTA_DEV = 1;
constexpr int LV_OUT_STDERR_DEV = 2;

// Everything a Monte Carlo launch reads, passed by value as a
// __grid_constant__ kernel parameter.
struct McParams {
    // grid (device copies, binary32)
    const float2* sig2;    // [Je][I - 1] time-major pairs (sigma_{i,j}, sigma_{i+1,j} - sigma_{i,j});
                           // Je = max(J, 2), row 1 repeats row 0 when J == 1
    const float* node;     // [I] spot nodes s_i
    const float2* ab;      // [I - 1] (1 / (s_{i+1} - s_i), -s_i / (s_{i+1} - s_i))
    const double* tau;     // [J] time nodes
    int I, J, Je;
    int log_uniform;       // spot nodes equally spaced in ln S
    float cell_scale;      // ln 2 / d(ln s): cell index from y = log2 S
    float cell_shift;      // -ln(s_0) / d(ln s)
    float s_lo, s_hi;      // s_0, s_{I-1}

    // option and scheme; the path state is y = log2 S (or S when the model
    // runs the Euler scheme on S)
    int model;             // bit 0: spot weight linear in ln S; bit 1: Euler scheme on S
    int extra;             // adjoint also sums d V / d r and d V / d T (rows end with them)
    float x0;              // log2 S0 (S0 on S)
    float rdt;             // log2(e) r dt (r dt on S)
    float hdt;             // log2(e) dt / 2
    float sqdt2;           // log2(e) sqrt(dt)
    float dt;
    float sqdt;            // sqrt(dt) (natural units, for d x_{n+1} / d sigma_n)
    float K;
    float disc;            // e^{-rT}
    float S0f, inv_S0;     // S0, 1 / S0 (the scaled adjoint of the scheme on S)
    float Tf, r_nat;       // T, r (d price / d r and d price / d T)
    float inv_N, half_inv_sqdt;   // 1 / N, 1 / (2 sqrt(dt))
    float phi;             // +1 call, -1 put
    double dt_d;           // dt in binary64 for the time table
    int N;                 // steps

    // random numbers
    uint32_t k0, k1;       // Philox key = seed
    uint32_t stream_id;
    long long path_begin;
    long long n_paths;

    // work decomposition and scratch
    int n_tiles;           // ceil(n_paths / paths_per_tile()): tiles claimed by warps
    int ppl;               // adjoint: paths per lane of a forward tile (1 or 2; a warp claims ppl tiles)
    unsigned int* tile_counter;   // zero before the launch, reset by the finalize
    double* partials;      // [gridDim.x][row_words] per-block binary64 rows
    int row_words;         // 3 + Je * I (adjoint) or 3 (price only)
    double* warp_rows;     // [gridDim.x * warps][Je * I] per-warp level-2 rows
    float* l1;             // [gridDim.x][Je * I] per-block level-1 binary32 buckets
    float* ckpt;           // [n_ck][gridDim.x * warps * ring_slots_per_warp() * ppl] checkpoints of x
    int n_ck;
    int flush_every;       // reverse batches between level-1 -> level-2 drains
    int grid_smem;         // 1: sigma pairs staged in shared memory, 0: read through L1
    int acc_mode;          // 0 binary64, 1 Kahan binary32
    int method;            // LV_ADJ_REVERSE or LV_ADJ_TANGENT
    unsigned int* flag;    // tangent-ratio adjoint: count of live paths with a vanishing 1 + g_n

    // per-path outputs and near-node decision log (debug entry point only;
    // dbg_xN != null selects the logging instantiation)
    float* dbg_xN;
    float* dbg_V;
    float* dbg_xbar0;
    int* dbg_ev;                        // [dbg_ev_cap][3]: path - path_begin, step, 2 i + inside
    unsigned long long* dbg_ev_count;
    long long dbg_ev_cap;
    float dbg_band;                     // relative distance to a node that is logged
};

// McParams::method of the second-order bucket kernel (besides LV_ADJ_REVERSE
// and LV_ADJ_TANGENT of lv.h).
constexpr int kMethodVanna = 2;

struct FinalizeParams {
    const double* partials;
    int G;                 // rows
    int row_words;
    int I, J;
    long long n_paths;
    double S0;
    int want_sums;         // 1: raw sums, 0: price / delta / stderr / vega
    int extra;             // rows end with the sums of d V / d r and d V / d T
    double* chunks;        // [finalize_chunks(G)][row_words] stage-1 sums
    double* out;           // [3 + I * J]
    unsigned int* tile_counter;  // reset to 0
    unsigned int* flag;          // nonzero: every output NaN; reset to 0 (may be null)
};

int finalize_chunks(int G);
cudaError_t launch_finalize_sums(const double* sums, int IJ, long long n_paths, double S0, double* out,
                                 cudaStream_t s);

// Batched central bump-and-reprice (lv_bump.cu).
struct BumpParams {
    McParams mc;           // grid, option, random numbers, path tiles, tile counter
    int n_scen;            // 3 + 2 I J
    int n_groups;          // ceil(n_scen / slots per thread)
    float eps_half;        // eps / 2 on sigma
    float x0_up, x0_dn;    // ln(S0 + eps_S / 2), ln(S0 - eps_S / 2)
    double* partials;      // [gridDim.x][row_words] per-block binary64 rows
    int row_words;         // 2 + I J
};

size_t bump_smem_bytes(int I, int Je, int N, int row_words);
int bump_slots_per_thread();
int bump_chunks(int G);
cudaError_t bump_occupancy(int block, size_t smem, int* blocks_per_sm);
cudaError_t launch_bump(const BumpParams& b, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_bump_finalize(const double* partials, int G, int row_words, double* chunks, int IJ,
                                 long long n_paths, double eps, double eps_S, double* out,
                                 unsigned int* tile_counter, cudaStream_t s);

size_t mc_smem_bytes(int I, int Je, int N, int block, bool greeks, bool grid_smem, bool extra = false,
                     int ppl = 1);

// Binary64 paths (lv_fp64.cu): the full-FP64 reference adjoint and the
// binary64 bump baseline, main reading only.
struct F64Params {
    const double* spot;    // [I] spot nodes
    const double* sig;     // [I * J] sigma, spot-major (as the ABI takes it)
    const double* tau;     // [J] time nodes
    int I, J, N;
    double x0, x0_up, x0_dn;   // ln S0, ln(S0 +- eps_S / 2)
    double r, dt, sqdt, K, disc, phi, eps_half;
    uint32_t k0, k1, stream_id;
    long long path_begin, n_paths;
    double* partials;      // [gridDim.x][row_words]: adjoint 3 + Je I (time-major), bump 2 + I J
    int row_words;
    unsigned int* flag;    // adjoint: live paths with a vanishing 1 + g_n
    int n_scen, n_groups;  // bump: 3 + 2 I J scenarios in groups of bump64_slots_per_thread()
};

size_t adjoint64_smem_bytes(int N);
size_t bump64_smem_bytes(int N, int row_words);
int bump64_slots_per_thread();
cudaError_t f64_occupancy(bool bump, size_t smem, int* blocks_per_sm);
cudaError_t launch_adjoint64(const F64Params& P, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_bump64(const F64Params& P, int grid, size_t smem, cudaStream_t s);

// Pipe-rate probes (lv_probe.cu): out[LV_PIPE_COUNT] operations per second.
cudaError_t measure_pipe_peaks(double* out);

// Test-facing kernels (lv_debug.cu): Philox words and normals for listed
// (path, block) counters; the per-step time table of a call.
cudaError_t launch_debug_normals(uint64_t seed, uint32_t stream_id, const long long* paths, const uint32_t* blocks,
                                 long long n, uint32_t* words, float* z, cudaStream_t s);
cudaError_t launch_debug_time_table(const McParams& P, int* out_j, float* out_v, cudaStream_t s);

// Launchers; return cudaSuccess or the launch error. An adjoint launch with
// p.dbg_xN != null runs the logging instantiation with k = 4 and binary64
// level 2 whatever k and p.acc_mode say: plan its scratch with k = 4.
cudaError_t launch_mc(const McParams& p, int grid, int block, int k, bool greeks, size_t smem,
                      cudaStream_t s);
cudaError_t launch_finalize(const FinalizeParams& f, cudaStream_t s);
cudaError_t mc_occupancy(int block, int k, bool greeks, int acc, bool dbg, bool grid_smem, int method, int model,
                         bool extra, size_t smem, int* blocks_per_sm, int ppl = 1);

// The kernels of the other models (lv_model1.cu .. lv_model3.cu, one
// translation unit each so that they compile in parallel); they exist for
// checkpoint intervals k = 4 and 8, at one or two paths per lane.
#define LV_DECLARE_MODEL(N)                                                                                \
    cudaError_t launch_mc_model##N(const McParams& p, int grid, int block, int k, bool greeks, size_t smem, \
                                   cudaStream_t s);                                                        \
    cudaError_t mc_occupancy_model##N(int block, int k, bool greeks, int acc, bool dbg, bool grid_smem,    \
                                      int method, bool extra, size_t smem, int* blocks_per_sm, int ppl);
LV_DECLARE_MODEL(1)
LV_DECLARE_MODEL(2)
LV_DECLARE_MODEL(3)
#undef LV_DECLARE_MODEL
constexpr int kModelMaxK = 8;
int ring_slots_per_warp();
int paths_per_tile(bool greeks);   // paths a warp claims at a time (adjoint / price kernel)

}  // namespace lv

// Book of options (lv_book.cu): device tables and launch parameters.
namespace lv {

struct BookSurf {
    int I, J, Je, log_uniform;
    float cell_scale, cell_shift, s_lo, s_hi;
    long long off_sig2, off_node, off_ab, off_tau;   // offsets into the book's grid arrays
    long long risk_off;                              // first double of this surface's aggregated risk
};

struct BookInst {
    int surf, N, phi, stream_id;
    double K, T;
    long long n_paths;
    long long out_off;                               // first double of this option's sums / outputs
    double w;                                        // position weight (aggregated risk)
    double scale;                                    // w / n_paths
};

struct BookItem {
    int inst, first_tile, n_tiles;                    // tiles of 32 paths
};

struct BookRun {
    double log2_S0, r;
    unsigned long long seed;
};

struct BookParams {
    const BookSurf* surfs;
    const BookInst* insts;
    const BookItem* items;
    int n_items;
    const float2* sig2;
    const float* node;
    const float2* ab;
    const double* tau;
    const BookRun* run;
    unsigned int* item_counter;
    double* sums;          // per option [3 + I J] binary64 sums (zeroed before a run)
    double* risk;          // aggregated runs: per surface [3 + I J], the vega part summed with
                           // weights w / n_paths (zeroed before a run); null: per-option vegas
    float* l1;             // [gridDim.x][max_IJe] binary32 buckets per block
    float* ckpt;           // [ceil(max_N / k)][gridDim.x * warps * ring slots]
    int max_I, max_Je, max_N, max_IJe;
};

// ppl: paths per lane of the forward tiles (1 or 2); the FIFO and the
// checkpoint ring (book_ring_slots_per_warp() * ppl per warp) grow with it.
size_t book_smem_bytes(int maxI, int maxJe, int maxN, int block, int ppl);
int book_ring_slots_per_warp();
cudaError_t book_prepare(int k, int ppl);
cudaError_t book_occupancy(int block, int k, int ppl, size_t smem, int* blocks_per_sm);
cudaError_t launch_book(const BookParams& b, int grid, int block, int k, int ppl, size_t smem, cudaStream_t s);
cudaError_t launch_book_finalize(const BookParams& b, int n_inst, int max_IJ, double* out, cudaStream_t s);
cudaError_t launch_book_risk_finalize(const BookParams& b, int n_surf, int n_inst, int max_IJ, double* out,
                                      cudaStream_t s);

}  // namespace lv

#include <string>

#include "lv.h"

namespace lv {
// Records the thread-local message lv_last_error() returns; returns s.
lv_status set_error(lv_status s, const std::string& msg);

// Launch-shape cache shared by the autotuners: lines "key v0 v1 v2 v3 ms" in
// the file named by LV_TUNE_CACHE (the last line of a key wins).
bool tune_cache_lookup(const std::string& key, int vals[4]);
void tune_cache_append(const std::string& key, const int vals[4], double ms);
std::string gpu_name(int device);
}  // namespace lv

// Surface handle (host side; shared by the runtime's source files).
struct lv_surface_s {
    int device = 0;
    int num_sms = 0;
    int adj_method = 0;              // LV_ADJ_REVERSE or LV_ADJ_TANGENT
    int interp = 0;                  // LV_INTERP_S or LV_INTERP_LOGS
    int scheme = 0;                  // LV_SCHEME_LOG or LV_SCHEME_S
    int I = 0, J = 0, Je = 0;
    std::vector<double> spot, time;
    float2* d_sig = nullptr;         // [Je][I-1] pairs (sigma_{i,j}, sigma_{i+1,j} - sigma_{i,j})
    float* d_node = nullptr;
    float2* d_ab = nullptr;
    float2* d_abl = nullptr;         // [I] cell coefficients of the ln-S weight, in y = log2 S
    double* d_tau = nullptr;
    double* d_spot64 = nullptr;      // [I] spot nodes, binary64 (the binary64 kernels)
    double* d_sig64 = nullptr;       // [I * J] sigma, binary64, spot-major
    double* h_sig64_stage = nullptr; // pinned staging for its uploads
    bool sig64_stale = false;        // d_sig64 behind h_sig64_stage: uploaded by the binary64 calls
    float2* h_sig_stage = nullptr;   // pinned staging for sigma uploads
    int log_uniform = 0;
    float cell_scale = 0.0f, cell_shift = 0.0f, s_lo = 0.0f, s_hi = 0.0f;
    int phi = 1;
    cudaStream_t stream = nullptr;
    int acc_mode = LV_ACC_FP64;
    int cfg_block = 0, cfg_k = 0, cfg_bps = 0, cfg_ppl = 0;
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    double* d_res = nullptr;         // [3 + I*J] result of the host-output calls
    double* h_res = nullptr;         // pinned copy of it
    cudaEvent_t ev_start = nullptr;  // optional events around the Monte Carlo kernel
    cudaEvent_t ev_end = nullptr;
};
