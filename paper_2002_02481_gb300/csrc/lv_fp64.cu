// lv_fp64.cu -- the same Monte Carlo estimators with every path in binary64
// (arXiv 2002.02481, Sec. III, IV-A..IV-D), main reading only: log-Euler,
// bilinear sigma linear in S and t. Two kernels:
//
//  - adjoint64_kernel: price, delta and every vega bucket, the reference the
//    binary32 kernels' rounding is measured against on the GPU. One path per
//    thread, the pathwise adjoint in its tangent-ratio form (two forward
//    passes, no checkpoints): x_bar_{n+1} = x_bar_N D_N / D_{n+1} with
//    D_{n+1} = D_n (1 + g_n), g_n = h_n S_n d sigma / d S,
//    h_n = sqrt(dt) Z_n - sigma_n dt; sigma_bar_n = x_bar_{n+1} h_n spread
//    over the cell's corners with the bilinear weights, run-length sums in
//    registers, binary64 reductions into the block's row.
//  - bump64_kernel: central bump-and-reprice (Sec. III) with binary64 paths,
//    scenario for scenario as the binary32 bump kernel (lv_bump.cu).
//
// The arithmetic follows the FP64 definition step by step (same expression
// order for sigma, its slope and the Euler step); the transcendental
// functions are CUDA's binary64 ones. Binary64 runs at a small fraction of
// the binary32 rate on this part: these kernels are references, not the
// product path.
#include <math.h>

#include "lv_device.cuh"

namespace lv {

namespace {

// Four binary64 normals of Philox block blk: the same words as normals4,
// u = ((w >> 9) + 1/2) 2^-23 (exact), Z_a = sqrt(-2 ln u_a) cos(2 pi u_b),
// Z_b = sqrt(-2 ln u_a) sin(2 pi u_b).
__device__ __forceinline__ void normals4_f64(uint32_t blk, uint32_t c1, uint32_t c2, uint32_t k0, uint32_t k1,
                                             double z[4])
{
    uint32_t w[4] = { blk, c1, c2, 0u };
    philox4x32_10(w[0], w[1], w[2], w[3], k0, k1);
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const double ua = ((double)(w[2 * pair] >> 9) + 0.5) * 0x1p-23;
        const double ub = ((double)(w[2 * pair + 1] >> 9) + 0.5) * 0x1p-23;
        const double rho = sqrt(-2.0 * log(ua));
        double s, c;
        sincospi(2.0 * ub, &s, &c);
        z[2 * pair] = rho * c;
        z[2 * pair + 1] = rho * s;
    }
}

struct Pt64 {
    int i;
    double u, sigma, dsdS;
};

// Bilinear sigma at (S, time cell j, weight v) and d sigma / d S (0 outside
// [s_0, s_{I-1}]); cell i = the largest i <= I-2 with s_i <= S.
__device__ __forceinline__ Pt64 sigma64(const F64Params& P, double S, int j, double v)
{
    int lo = 0, hi = P.I - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.spot[mid] <= S) lo = mid;
        else hi = mid - 1;
    }
    const int i = lo;
    const double lo_s = P.spot[i], hi_s = P.spot[i + 1];
    double u;
    if (S <= lo_s) u = 0.0;
    else if (S >= hi_s) u = 1.0;
    else u = (S - lo_s) / (hi_s - lo_s);
    const int J = P.J;
    const double s00 = P.sig[i * J + j];
    const double s10 = P.sig[(i + 1) * J + j];
    const double s01 = J > 1 ? P.sig[i * J + j + 1] : 0.0;
    const double s11 = J > 1 ? P.sig[(i + 1) * J + j + 1] : 0.0;
    Pt64 p;
    p.i = i;
    p.u = u;
    const double w0 = (1.0 - u) * (1.0 - v), w1 = u * (1.0 - v), w2 = (1.0 - u) * v, w3 = u * v;
    p.sigma = w0 * s00 + w1 * s10 + w2 * s01 + w3 * s11;
    const bool inside = S >= P.spot[0] && S <= P.spot[P.I - 1];
    p.dsdS = inside ? ((1.0 - v) * (s10 - s00) + v * (s11 - s01)) / (hi_s - lo_s) : 0.0;
    return p;
}

// Time cell and weight of every step (t_n = n dt), in shared memory.
__device__ __forceinline__ void stage_time64(const F64Params& P, int2* s_j, double* s_v)
{
    for (int n = threadIdx.x; n < P.N; n += blockDim.x) {
        const double t = (double)n * P.dt;
        int j = 0;
        double v = 0.0;
        if (P.J > 1) {
            int lo = 0, hi = P.J - 2;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (P.tau[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            j = lo;
            v = (t - P.tau[j]) / (P.tau[j + 1] - P.tau[j]);
            v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        }
        s_j[n] = make_int2(j, j * P.I);
        s_v[n] = v;
    }
}

__device__ __forceinline__ void path_words(const F64Params& P, long long rel, uint32_t& c1, uint32_t& c2)
{
    const unsigned long long p = (unsigned long long)(P.path_begin + rel);
    c1 = (uint32_t)p;
    c2 = ((uint32_t)(p >> 32) & 0xffffu) | (P.stream_id << 16);
}

__device__ __forceinline__ void flush64(double* row, int key, int I, double A, double AU, double Bs, double BU)
{
    atomicAdd(row + key, A - AU);
    atomicAdd(row + key + 1, AU);
    atomicAdd(row + key + I, Bs - BU);
    atomicAdd(row + key + I + 1, BU);
}

constexpr double kTiny64 = 0x1p-40;    // |1 + g_n| below this on a live path: the ratio form is refused

__global__ void __launch_bounds__(128) adjoint64_kernel(const __grid_constant__ F64Params P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int2* s_j = reinterpret_cast<int2*>(smem);
    double* s_v = reinterpret_cast<double*>(smem + ((sizeof(int2) * (size_t)P.N + 15) & ~size_t(15)));
    double* s_red = s_v + ((P.N + 1) & ~1);
    double* row = P.partials + (size_t)blockIdx.x * P.row_words;
    for (int e = threadIdx.x; e < P.row_words; e += blockDim.x) row[e] = 0.0;
    stage_time64(P, s_j, s_v);
    __syncthreads();
    double* vrow = row + 3;              // time-major buckets j I + i
    double sV = 0.0, sV2 = 0.0, sX = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long rel = (long long)blockIdx.x * blockDim.x + threadIdx.x; rel < P.n_paths; rel += stride) {
        uint32_t c1, c2;
        path_words(P, rel, c1, c2);
        double z[4];
        // pass 1: the path, its payoff and D_N
        double x = P.x0, D = 1.0;
        bool tiny = false;
        for (int n = 0; n < P.N; ++n) {
            if ((n & 3) == 0) normals4_f64((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
            const double S = exp(x);
            const Pt64 pt = sigma64(P, S, s_j[n].x, s_v[n]);
            const double h = P.sqdt * z[n & 3] - pt.sigma * P.dt;
            const double f = 1.0 + h * S * pt.dsdS;
            tiny = tiny || fabs(f) < kTiny64;
            D *= f;
            x = x + (P.r - 0.5 * pt.sigma * pt.sigma) * P.dt + pt.sigma * P.sqdt * z[n & 3];
        }
        const double SN = exp(x);
        const double itm = P.phi * (SN - P.K);
        const double V = itm > 0.0 ? P.disc * itm : 0.0;
        const double c = itm > 0.0 ? P.disc * P.phi * SN * D : 0.0;   // x_bar_0 = x_bar_N D_N
        sV += V;
        sV2 += V * V;
        sX += c;
        if (c == 0.0) continue;
        if (tiny) {
            atomicAdd(P.flag, 1u);
            continue;
        }
        // pass 2: the same path again, sigma_bar_n = c h_n / D_{n+1}
        x = P.x0;
        D = 1.0;
        int cur = -1;
        double A = 0.0, AU = 0.0, Bs = 0.0, BU = 0.0;
        for (int n = 0; n < P.N; ++n) {
            if ((n & 3) == 0) normals4_f64((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
            const double S = exp(x);
            const double v = s_v[n];
            const Pt64 pt = sigma64(P, S, s_j[n].x, v);
            const double h = P.sqdt * z[n & 3] - pt.sigma * P.dt;
            D *= 1.0 + h * S * pt.dsdS;
            const double sbar = c * h / D;
            const int key = s_j[n].y + pt.i;
            if (key != cur) {
                if (cur >= 0) flush64(vrow, cur, P.I, A, AU, Bs, BU);
                A = AU = Bs = BU = 0.0;
                cur = key;
            }
            const double b = sbar * v;
            const double a = sbar - b;
            A += a;
            AU += a * pt.u;
            Bs += b;
            BU += b * pt.u;
            x = x + (P.r - 0.5 * pt.sigma * pt.sigma) * P.dt + pt.sigma * P.sqdt * z[n & 3];
        }
        if (cur >= 0) flush64(vrow, cur, P.I, A, AU, Bs, BU);
    }
    // block sums of the scalars (fixed order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sV += __shfl_down_sync(0xffffffffu, sV, o);
        sV2 += __shfl_down_sync(0xffffffffu, sV2, o);
        sX += __shfl_down_sync(0xffffffffu, sX, o);
    }
    if (lane == 0) {
        s_red[3 * warp + 0] = sV;
        s_red[3 * warp + 1] = sV2;
        s_red[3 * warp + 2] = sX;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, cc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_red[3 * w + 0];
            b += s_red[3 * w + 1];
            cc += s_red[3 * w + 2];
        }
        row[0] = a;
        row[1] = b;
        row[2] = cc;
    }
}

constexpr int kM64 = 8;   // scenario slots per thread (even: pairs never split)

// Scenario s of 3 + 2 I J as in lv_bump.cu: s = 0, 1 S0 +- eps_S/2; s = 2 + 2e + b
// node e = i J + j at sigma_e + eps/2 (b = 0) or - eps/2 (b = 1); the last one
// unbumped. Each thread prices one path under kM64 consecutive scenarios on the
// same normals; pair differences go to slot s / 2 of the block's row.
__global__ void __launch_bounds__(128) bump64_kernel(const __grid_constant__ F64Params P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int2* s_j = reinterpret_cast<int2*>(smem);
    double* s_v = reinterpret_cast<double*>(smem + ((sizeof(int2) * (size_t)P.N + 15) & ~size_t(15)));
    double* s_acc = s_v + ((P.N + 1) & ~1);
    for (int e = threadIdx.x; e < P.row_words; e += blockDim.x) s_acc[e] = 0.0;
    stage_time64(P, s_j, s_v);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long n_tiles = (P.n_paths + blockDim.x - 1) / blockDim.x;
    const long long n_items = n_tiles * P.n_groups;
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {     // block-uniform
        const int grp = (int)(item % P.n_groups);
        const long long rel = (item / P.n_groups) * blockDim.x + threadIdx.x;
        const int s_first = grp * kM64;
        double x[kM64], V[kM64], bh[kM64];
        int be[kM64];
#pragma unroll
        for (int k = 0; k < kM64; ++k) {
            const int s = s_first + k;
            x[k] = s == 0 ? P.x0_up : (s == 1 ? P.x0_dn : P.x0);
            be[k] = (s >= 2 && s < P.n_scen - 1) ? (s - 2) >> 1 : -1;
            bh[k] = ((s - 2) & 1) ? -P.eps_half : P.eps_half;
            V[k] = 0.0;
        }
        if (rel < P.n_paths) {
            uint32_t c1, c2;
            path_words(P, rel, c1, c2);
            double z[4];
            for (int n = 0; n < P.N; ++n) {
                if ((n & 3) == 0) normals4_f64((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
                const int j = s_j[n].x;
                const double v = s_v[n];
#pragma unroll
                for (int k = 0; k < kM64; ++k) {
                    if (s_first + k >= P.n_scen) continue;
                    const double S = exp(x[k]);
                    const Pt64 pt = sigma64(P, S, j, v);
                    double sig = pt.sigma;
                    if (be[k] >= 0) {       // + or - eps/2 times the bumped node's bilinear weight
                        const int bi = be[k] / P.J, bj = be[k] - bi * P.J;
                        const double ws = bi == pt.i ? 1.0 - pt.u : (bi == pt.i + 1 ? pt.u : 0.0);
                        const double wt = bj == j ? 1.0 - v : (P.J > 1 && bj == j + 1 ? v : 0.0);
                        sig += bh[k] * (ws * wt);
                    }
                    x[k] = x[k] + (P.r - 0.5 * sig * sig) * P.dt + sig * P.sqdt * z[n & 3];
                }
            }
#pragma unroll
            for (int k = 0; k < kM64; ++k) {
                const double itm = P.phi * (exp(x[k]) - P.K);
                V[k] = itm > 0.0 ? P.disc * itm : 0.0;
            }
        }
#pragma unroll
        for (int k = 0; k < kM64; k += 2) {
            const int s = s_first + k;
            if (s < P.n_scen) {
                double d = (s + 1 < P.n_scen) ? V[k] - V[k + 1] : V[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
                if (lane == 0) atomicAdd(&s_acc[s >> 1], d);
            }
        }
    }
    __syncthreads();
    double* row = P.partials + (size_t)blockIdx.x * P.row_words;
    for (int e = threadIdx.x; e < P.row_words; e += blockDim.x) row[e] = s_acc[e];
}

size_t f64_time_bytes(int N) { return ((sizeof(int2) * (size_t)N + 15) & ~size_t(15)) + sizeof(double) * ((N + 1) & ~1); }

}  // namespace

size_t adjoint64_smem_bytes(int N) { return f64_time_bytes(N) + sizeof(double) * 3 * 4; }
size_t bump64_smem_bytes(int N, int row_words) { return f64_time_bytes(N) + sizeof(double) * (size_t)row_words; }
int bump64_slots_per_thread() { return kM64; }

cudaError_t f64_occupancy(bool bump, size_t smem, int* bps)
{
    const void* k = bump ? (const void*)bump64_kernel : (const void*)adjoint64_kernel;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, 128, smem);
}

cudaError_t launch_adjoint64(const F64Params& P, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(adjoint64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    adjoint64_kernel<<<grid, 128, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_bump64(const F64Params& P, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(bump64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    bump64_kernel<<<grid, 128, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace lv
