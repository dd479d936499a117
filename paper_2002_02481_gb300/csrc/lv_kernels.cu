// lv_kernels.cu -- the Monte Carlo price / pathwise-adjoint kernel and the
// fixed-order finalize (arXiv 2002.02481, Sec. III, IV-A..IV-D).
//
// One persistent kernel per call. Each block claims tiles of blockDim.x
// consecutive paths from a global counter. Per tile:
//   1. forward: every thread simulates one path from x_0 = ln S0 with
//      normals generated in registers, storing x every KCK steps (the
//      checkpoints, in an L2-resident scratch slot owned by the thread);
//   2. payoff and terminal adjoint xbar_N = e^{-rT} 1{phi(S_N-K)>0} phi S_N;
//   3. compaction: paths with xbar_N = 0 have a zero adjoint everywhere, so
//      only the others are queued (block-wide, in path order) and the
//      reverse sweep runs on a dense set of threads;
//   4. reverse sweep: per checkpoint segment, from last to first, recompute
//      KCK steps (same Philox counters) keeping h_n = d x_{n+1} / d sigma_n,
//      g_n = h_n S_n d sigma/d S, the cell and the weight in registers, then
//      walk them backwards: sigma_bar_n = xbar_{n+1} h_n, xbar_n =
//      xbar_{n+1} (1 + g_n), and scatter sigma_bar_n to the four corner
//      buckets;
//   5. bucket accumulation: per-thread run-length sums while the cell is
//      unchanged (level 0), shared-memory binary32 atomics (level 1), and
//      after every tile a per-block binary64 (or Kahan binary32) row in
//      global memory (level 2). A separate fixed-order binary64 reduction
//      over blocks (level 3) produces the outputs.
#include <math.h>

#include "lv_device.cuh"

namespace lv {

namespace {

constexpr int kMaxWarps = 16;   // blockDim.x <= 512

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

struct SmemLayout {
    size_t tab, sig, node, ab, bk, qown, qxb, wcnt, red, tile, total;
};

__host__ __device__ inline SmemLayout smem_layout(int I, int Je, int N, int block, bool greeks)
{
    SmemLayout L;
    size_t o = 0;
    L.tab = o;  o += align16(sizeof(int2) * (size_t)N);
    L.sig = o;  o += align16(sizeof(float) * (size_t)Je * I);
    L.node = o; o += align16(sizeof(float) * (size_t)I);
    L.ab = o;   o += align16(sizeof(float2) * (size_t)I);
    L.bk = o;   if (greeks) o += align16(sizeof(float) * (size_t)Je * I);
    L.qown = o; if (greeks) o += align16(sizeof(int) * (size_t)block);
    L.qxb = o;  if (greeks) o += align16(sizeof(float) * (size_t)block);
    L.wcnt = o; if (greeks) o += align16(sizeof(int) * kMaxWarps);
    L.red = o;  o += align16(sizeof(double) * 3 * kMaxWarps);
    L.tile = o; o += align16(sizeof(int) * 2);
    L.total = o;
    return L;
}

// (j_n * I, v_n) for step n: t_n = n dt, j_n = largest j <= J-2 with
// tau_j <= t_n, v_n = (t_n - tau_j) / (tau_{j+1} - tau_j) clamped to [0, 1];
// decided in binary64.
__device__ int2 time_cell(const McParams& P, int n)
{
    const double t = (double)n * P.dt_d;
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
        v = fmin(fmax(v, 0.0), 1.0);
    }
    return make_int2(j * P.I, __float_as_int((float)v));
}

struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Per-thread accumulation of the payoff, its square and xbar_0 across the
// paths a thread handles (level 2 of the scalars).
struct ScalarAcc {
    double V = 0.0, V2 = 0.0, X = 0.0;
    KahanF kV, kV2, kX;
    __device__ __forceinline__ void add_V(float v, int mode)
    {
        if (mode == LV_ACC_KAHAN_DEV) { kV.add(v); kV2.add(v * v); }
        else { V += (double)v; V2 += (double)v * (double)v; }
    }
    __device__ __forceinline__ void add_X(float x, int mode)
    {
        if (mode == LV_ACC_KAHAN_DEV) kX.add(x);
        else X += (double)x;
    }
    __device__ __forceinline__ void get(int mode, double& a, double& b, double& c) const
    {
        if (mode == LV_ACC_KAHAN_DEV) { a = kV.value(); b = kV2.value(); c = kX.value(); }
        else { a = V; b = V2; c = X; }
    }
    static constexpr int LV_ACC_KAHAN_DEV = 1;
};

template <int KCK, bool GREEKS>
__global__ void __launch_bounds__(512) mc_kernel(const __grid_constant__ McParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const SmemLayout L = smem_layout(P.I, P.Je, P.N, B, GREEKS);
    int2* s_tab = reinterpret_cast<int2*>(smem + L.tab);
    float* s_sig = reinterpret_cast<float*>(smem + L.sig);
    float* s_node = reinterpret_cast<float*>(smem + L.node);
    float2* s_ab = reinterpret_cast<float2*>(smem + L.ab);
    float* s_bk = reinterpret_cast<float*>(smem + L.bk);
    int* s_qown = reinterpret_cast<int*>(smem + L.qown);
    float* s_qxb = reinterpret_cast<float*>(smem + L.qxb);
    int* s_wcnt = reinterpret_cast<int*>(smem + L.wcnt);
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    int* s_tile = reinterpret_cast<int*>(smem + L.tile);

    const int nIJ = P.Je * P.I;
    for (int e = tid; e < nIJ; e += B) s_sig[e] = P.sig[e];
    for (int e = tid; e < P.I; e += B) s_node[e] = P.node[e];
    for (int e = tid; e < P.I - 1; e += B) s_ab[e] = P.ab[e];
    for (int n = tid; n < P.N; n += B) s_tab[n] = time_cell(P, n);
    double* row = P.partials + (size_t)blockIdx.x * P.row_words;
    if (GREEKS) {
        for (int e = tid; e < nIJ; e += B) s_bk[e] = 0.0f;
        for (int e = tid; e < P.row_words; e += B) row[e] = 0.0;
    }
    if (tid == 0) s_tile[0] = (int)atomicAdd(P.tile_counter, 1u);
    __syncthreads();

    SmemGrid g{ s_tab, s_sig, s_node, s_ab };
    const int nseg = (P.N + KCK - 1) / KCK;
    const size_t cks = (size_t)gridDim.x * B;           // checkpoint stride
    float* const ck_base = P.ckpt + (size_t)blockIdx.x * B;
    ScalarAcc acc;

    int it = 0;
    int tile = s_tile[0];
    while (tile < P.n_tiles) {
        const long long first = (long long)tile * B;     // relative to path_begin
        const bool active = first + tid < P.n_paths;
        float xbarN = 0.0f;
        if (active) {
            const unsigned long long p = (unsigned long long)(P.path_begin + first + tid);
            const uint32_t c1 = (uint32_t)p;
            const uint32_t c2 = ((uint32_t)(p >> 32) & 0xffffu) | (P.stream_id << 16);
            float x = P.x0;
            float z[4];
            for (int m = 0; m < nseg; ++m) {
                if (GREEKS) ck_base[(size_t)m * cks + tid] = x;
#pragma unroll
                for (int q = 0; q < KCK; ++q) {
                    const int n = m * KCK + q;
                    if (n < P.N) {
                        if ((q & 3) == 0) normals4((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
                        const int2 tb = g.tab[n];
                        const StepEval e = eval_sigma<false>(P, g, x, tb.x, __int_as_float(tb.y));
                        x = euler_step(P, x, e.sigma, z[q & 3]);
                    }
                }
            }
            const float SN = expf(x);
            const float itm = P.phi * (SN - P.K);
            const float V = itm > 0.0f ? P.disc * itm : 0.0f;
            xbarN = itm > 0.0f ? P.disc * P.phi * SN : 0.0f;
            acc.add_V(V, P.acc_mode);
            if (P.dbg_xN) {
                const long long r = first + tid;
                P.dbg_xN[r] = x;
                P.dbg_V[r] = V;
                P.dbg_xbar0[r] = 0.0f;
            }
        }
        if (GREEKS) {
            // block-wide compaction of the paths with a nonzero adjoint, in path order
            const bool live = xbarN != 0.0f;
            const unsigned bal = __ballot_sync(0xffffffffu, live);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = 0, total = 0;
            const int nw = B >> 5;
            for (int w = 0; w < nw; ++w) {
                const int c = s_wcnt[w];
                off += (w < warp) ? c : 0;
                total += c;
            }
            if (live) {
                const int idx = off + __popc(bal & ((1u << lane) - 1u));
                s_qown[idx] = tid;
                s_qxb[idx] = xbarN;
            }
            __syncthreads();
            if (tid < total) {
                const int owner = s_qown[tid];
                float xbar = s_qxb[tid];
                const unsigned long long p = (unsigned long long)(P.path_begin + first + owner);
                const uint32_t c1 = (uint32_t)p;
                const uint32_t c2 = ((uint32_t)(p >> 32) & 0xffffu) | (P.stream_id << 16);
                const float* ck = ck_base + owner;
                int cur = -1;
                float A = 0.0f, AU = 0.0f, Bs = 0.0f, BU = 0.0f;
                float z[4];
                for (int m = nseg - 1; m >= 0; --m) {
                    float x = ck[(size_t)m * cks];
                    float hq[KCK], gq[KCK], uq[KCK];
                    int iq[KCK];
#pragma unroll
                    for (int q = 0; q < KCK; ++q) {
                        const int n = m * KCK + q;
                        if (n < P.N) {
                            if ((q & 3) == 0) normals4((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
                            const int2 tb = g.tab[n];
                            const StepEval e = eval_sigma<true>(P, g, x, tb.x, __int_as_float(tb.y));
                            const float h = fmaf(P.sqdt, z[q & 3], -e.sigma * P.dt);
                            hq[q] = h;
                            gq[q] = h * (e.S * e.slope);
                            uq[q] = e.u;
                            iq[q] = e.i;
                            x = euler_step(P, x, e.sigma, z[q & 3]);
                        }
                    }
#pragma unroll
                    for (int q = KCK - 1; q >= 0; --q) {
                        const int n = m * KCK + q;
                        if (n < P.N) {
                            const int2 tb = g.tab[n];
                            const int key = tb.x + iq[q];
                            const float v = __int_as_float(tb.y);
                            const float sbar = xbar * hq[q];
                            xbar = fmaf(xbar, gq[q], xbar);
                            if (key != cur) {
                                if (cur >= 0) {
                                    atomicAdd(&s_bk[cur], A - AU);
                                    atomicAdd(&s_bk[cur + 1], AU);
                                    atomicAdd(&s_bk[cur + P.I], Bs - BU);
                                    atomicAdd(&s_bk[cur + P.I + 1], BU);
                                }
                                cur = key;
                                A = AU = Bs = BU = 0.0f;
                            }
                            const float b = sbar * v;
                            const float a = sbar - b;
                            A += a;
                            AU = fmaf(a, uq[q], AU);
                            Bs += b;
                            BU = fmaf(b, uq[q], BU);
                        }
                    }
                }
                if (cur >= 0) {
                    atomicAdd(&s_bk[cur], A - AU);
                    atomicAdd(&s_bk[cur + 1], AU);
                    atomicAdd(&s_bk[cur + P.I], Bs - BU);
                    atomicAdd(&s_bk[cur + P.I + 1], BU);
                }
                acc.add_X(xbar, P.acc_mode);
                if (P.dbg_xN) P.dbg_xbar0[first + owner] = xbar;
            }
        }
        if (tid == 0) s_tile[(it + 1) & 1] = (int)atomicAdd(P.tile_counter, 1u);
        __syncthreads();
        if (GREEKS) {
            // level 2: this tile's buckets into the block's row, then clear them
            if (P.acc_mode == 1) {
                float2* krow = reinterpret_cast<float2*>(row + 3);
                for (int e = tid; e < nIJ; e += B) {
                    float2 k = krow[e];
                    const float y = s_bk[e] - k.y;
                    const float t = k.x + y;
                    k.y = (t - k.x) - y;
                    k.x = t;
                    krow[e] = k;
                    s_bk[e] = 0.0f;
                }
            } else {
                for (int e = tid; e < nIJ; e += B) {
                    row[3 + e] += (double)s_bk[e];
                    s_bk[e] = 0.0f;
                }
            }
        }
        ++it;
        tile = s_tile[it & 1];
    }

    // block reduction of the scalar sums (binary64, fixed order over warps)
    double a, b, c;
    acc.get(P.acc_mode, a, b, c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        s_red[3 * warp + 0] = a;
        s_red[3 * warp + 1] = b;
        s_red[3 * warp + 2] = c;
    }
    __syncthreads();
    if (tid == 0) {
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int w = 0; w < (B >> 5); ++w) {
            sa += s_red[3 * w + 0];
            sb += s_red[3 * w + 1];
            sc += s_red[3 * w + 2];
        }
        row[0] = sa;
        row[1] = sb;
        row[2] = sc;
    }
}

// Level 3, stage 1: rows [chunk * RCH, (chunk + 1) * RCH) summed in order,
// column by column, into one binary64 row per chunk.
constexpr int kRowsPerChunk = 32;

__global__ void reduce_rows_kernel(const double* __restrict__ partials, int G, int row_words,
                                   int acc_mode, double* __restrict__ chunks)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= row_words) return;
    const int r0 = blockIdx.y * kRowsPerChunk;
    const int r1 = min(G, r0 + kRowsPerChunk);
    double s = 0.0;
    if (acc_mode == 1 && col >= 3) {
        for (int r = r0; r < r1; ++r) {
            const float2 k = reinterpret_cast<const float2*>(partials + (size_t)r * row_words)[col];
            s += (double)k.x - (double)k.y;
        }
    } else {
        for (int r = r0; r < r1; ++r) s += partials[(size_t)r * row_words + col];
    }
    chunks[(size_t)blockIdx.y * row_words + col] = s;
}

// Level 3, stage 2: chunks summed in order; outputs in the ABI layout
// (vega spot-major), price statistics from the scalar sums.
__global__ void finalize_kernel(const double* __restrict__ chunks, int n_chunks, int row_words,
                                int I, int J, long long n_paths, double S0, int want_sums,
                                double* __restrict__ out, unsigned int* tile_counter)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= row_words) return;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += chunks[(size_t)c * row_words + col];
    const double P = (double)n_paths;
    if (col < 3) {
        if (want_sums) {
            out[col] = s;
        } else if (col == 0) {
            double sv2 = 0.0;
            for (int c = 0; c < n_chunks; ++c) sv2 += chunks[(size_t)c * row_words + 1];
            const double mean = s / P;
            double var = n_paths > 1 ? (sv2 / P - mean * mean) * P / (P - 1.0) : 0.0;
            out[LV_OUT_PRICE_DEV] = mean;
            out[LV_OUT_STDERR_DEV] = var > 0.0 ? sqrt(var / P) : 0.0;
        } else if (col == 2) {
            out[LV_OUT_DELTA_DEV] = s / (P * S0);
        }
        if (col == 0 && tile_counter) *tile_counter = 0u;
        return;
    }
    const int e = col - 3;             // time-major bucket j * I + i
    const int j = e / I, i = e - j * I;
    if (j >= J) return;                // padding row of a one-column grid
    out[3 + i * J + j] = want_sums ? s : s / P;
}

}  // namespace

size_t mc_smem_bytes(int I, int Je, int N, int block, bool greeks)
{
    return smem_layout(I, Je, N, block, greeks).total;
}

template <int KCK, bool GREEKS>
static cudaError_t launch_one(const McParams& p, int grid, int block, size_t smem, cudaStream_t s)
{
    static bool configured = false;   // per instantiation; the library is single-device per process
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mc_kernel<KCK, GREEKS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mc_kernel<KCK, GREEKS><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <int KCK, bool GREEKS>
static cudaError_t occupancy_one(int block, size_t smem, int* bps)
{
    cudaError_t e = cudaFuncSetAttribute(mc_kernel<KCK, GREEKS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, mc_kernel<KCK, GREEKS>, block, smem);
}

cudaError_t launch_mc(const McParams& p, int grid, int block, int k, bool greeks, size_t smem,
                      cudaStream_t s)
{
    if (!greeks) return launch_one<4, false>(p, grid, block, smem, s);
    switch (k) {
    case 4: return launch_one<4, true>(p, grid, block, smem, s);
    case 8: return launch_one<8, true>(p, grid, block, smem, s);
    case 16: return launch_one<16, true>(p, grid, block, smem, s);
    case 32: return launch_one<32, true>(p, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t mc_occupancy(int block, int k, bool greeks, size_t smem, int* bps)
{
    if (!greeks) return occupancy_one<4, false>(block, smem, bps);
    switch (k) {
    case 4: return occupancy_one<4, true>(block, smem, bps);
    case 8: return occupancy_one<8, true>(block, smem, bps);
    case 16: return occupancy_one<16, true>(block, smem, bps);
    case 32: return occupancy_one<32, true>(block, smem, bps);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_finalize(const FinalizeParams& f, cudaStream_t s)
{
    const int n_chunks = (f.G + kRowsPerChunk - 1) / kRowsPerChunk;
    double* chunks = f.chunks;
    dim3 g1((f.row_words + 255) / 256, n_chunks);
    reduce_rows_kernel<<<g1, 256, 0, s>>>(f.partials, f.G, f.row_words, f.acc_mode, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_kernel<<<(f.row_words + 255) / 256, 256, 0, s>>>(chunks, n_chunks, f.row_words, f.I,
                                                              f.J, f.n_paths, f.S0, f.want_sums,
                                                              f.out, f.tile_counter);
    return cudaGetLastError();
}

int finalize_chunks(int G) { return (G + kRowsPerChunk - 1) / kRowsPerChunk; }

}  // namespace lv
