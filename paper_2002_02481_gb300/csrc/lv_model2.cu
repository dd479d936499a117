// lv_model2.cu -- the kernels of model 2 (Euler scheme on S), from lv_mc.cuh,
// in a translation unit of their own so that the build compiles the models
// in parallel.
#include "lv_mc.cuh"

namespace lv {

cudaError_t launch_mc_model2(const McParams& p, int grid, int block, int k, bool greeks, size_t smem,
                              cudaStream_t s)
{
    return launch_model_impl<2>(p, grid, block, k, greeks, smem, s);
}

cudaError_t mc_occupancy_model2(int block, int k, bool greeks, int acc, bool dbg, bool grid_smem, int method,
                                 bool extra, size_t smem, int* bps, int ppl)
{
    return occupancy_model_impl<2>(block, k, greeks, acc, dbg, grid_smem, method, extra, smem, bps, ppl);
}

}  // namespace lv
