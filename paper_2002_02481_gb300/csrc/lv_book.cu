// lv_book.cu -- a book of European options on several local-vol grids in
// one persistent launch (prices, deltas and vega buckets of every option).
//
// Work items are (option, range of 32-path tiles), listed longest options
// first, the items of one option consecutive. A block claims items from a
// global counter; when the option changes it restages that option's grid
// and time table in shared memory and rebuilds its launch parameters. Inside
// an item the warps claim tiles from a block-local counter and run the same
// per-path code as the single-option kernel: forward pass with checkpoints
// into the warp's ring of slots, a per-warp queue of paths with a nonzero
// terminal adjoint, checkpointed reverse sweeps on full warps (partial ones
// only to finish an item). At the end of an item the block adds its binary32
// bucket sums and its payoff / adjoint sums to the option's binary64 sums
// with atomics; a finalize kernel divides by the option's path count.
#include <math.h>

#include "lv_device.cuh"

namespace lv {

namespace {

constexpr int kBRing = 4;
constexpr int kBQueue = 64;
constexpr int kBMaxWarps = 8;

__host__ __device__ inline size_t b16(size_t b) { return (b + 15) & ~size_t(15); }

struct BookSmem {
    size_t params, tab, sig, node, ab, qslot, qrel, qxb, acc, red, ctl, total;
};

__host__ __device__ inline BookSmem book_layout(int maxI, int maxJe, int maxN, int block, int ppl = 1)
{
    const int W = block / 32;
    BookSmem L;
    size_t o = 0;
    L.params = o; o += b16(sizeof(McParams));
    L.tab = o;    o += b16(sizeof(int4) * (size_t)maxN);
    L.sig = o;    o += b16(sizeof(float2) * (size_t)maxJe * (maxI - 1));
    L.node = o;   o += b16(sizeof(float) * (size_t)maxI);
    L.ab = o;     o += b16(sizeof(float2) * (size_t)maxI);
    L.qslot = o;  o += b16(sizeof(int) * (size_t)W * kBQueue * ppl);
    L.qrel = o;   o += b16(sizeof(int) * (size_t)W * kBQueue * ppl);
    L.qxb = o;    o += b16(sizeof(float) * (size_t)W * kBQueue * ppl);
    L.acc = o;    o += b16(sizeof(double) * 3 * (size_t)block);
    L.red = o;    o += b16(sizeof(double) * 3 * kBMaxWarps);
    L.ctl = o;    o += b16(sizeof(int) * 4);
    L.total = o;
    return L;
}

// Claims n consecutive tiles of the block's current item for the warp.
__device__ __forceinline__ int warp_claim(int* counter, int n = 1)
{
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(counter, n);
    return __shfl_sync(0xffffffffu, t, 0);
}

// Launch parameters of option `inst` for this run (built by thread 0).
__device__ void build_params(const BookParams& B, int inst, McParams* out)
{
    const BookInst& o = B.insts[inst];
    const BookSurf& s = B.surfs[o.surf];
    const BookRun& run = *B.run;
    McParams P{};
    P.sig2 = B.sig2 + s.off_sig2;
    P.node = B.node + s.off_node;
    P.ab = B.ab + s.off_ab;
    P.tau = B.tau + s.off_tau;
    P.I = s.I;
    P.J = s.J;
    P.Je = s.Je;
    P.log_uniform = s.log_uniform;
    P.cell_scale = s.cell_scale;
    P.cell_shift = s.cell_shift;
    P.s_lo = s.s_lo;
    P.s_hi = s.s_hi;
    const double dt = o.T / (double)o.N;
    const double log2e = 1.4426950408889634;
    P.x0 = (float)run.log2_S0;
    P.rdt = (float)(log2e * run.r * dt);
    P.hdt = (float)(log2e * 0.5 * dt);
    P.sqdt2 = (float)(log2e * sqrt(dt));
    P.dt = (float)dt;
    P.sqdt = (float)sqrt(dt);
    P.K = (float)o.K;
    P.disc = (float)exp(-run.r * o.T);
    P.phi = (float)o.phi;
    P.dt_d = dt;
    P.N = o.N;
    P.k0 = (uint32_t)(run.seed & 0xffffffffu);
    P.k1 = (uint32_t)(run.seed >> 32);
    P.stream_id = (uint32_t)o.stream_id;
    P.path_begin = 0;
    P.n_paths = o.n_paths;
    *out = P;
}

// PPL: paths per lane of a forward tile, as in the single-option kernel: a
// warp claims PPL consecutive 32-path tiles of its item and runs them
// interleaved; the ring groups and the FIFO grow with it.
template <int KCK, int PPL>
__global__ void __launch_bounds__(128, 5) book_kernel(const __grid_constant__ BookParams B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kSlots = 32 * PPL;
    constexpr int kQcap = kBQueue * PPL;
    const int Bk = blockDim.x, W = Bk >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BookSmem L = book_layout(B.max_I, B.max_Je, B.max_N, Bk, PPL);
    McParams* s_par = reinterpret_cast<McParams*>(smem + L.params);
    int4* s_tab = reinterpret_cast<int4*>(smem + L.tab);
    float2* s_sig = reinterpret_cast<float2*>(smem + L.sig);
    float* s_node = reinterpret_cast<float*>(smem + L.node);
    float2* s_ab = reinterpret_cast<float2*>(smem + L.ab);
    int* q_slot = reinterpret_cast<int*>(smem + L.qslot) + warp * kQcap;
    int* q_rel = reinterpret_cast<int*>(smem + L.qrel) + warp * kQcap;
    float* q_xb = reinterpret_cast<float*>(smem + L.qxb) + warp * kQcap;
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);   // [0] item, [1] next tile, [2] staged option
    float* l1 = B.l1 + (size_t)blockIdx.x * B.max_IJe;
    const size_t cks = (size_t)gridDim.x * W * kBRing * kSlots;
    float* const ckw = B.ckpt + (size_t)(blockIdx.x * W + warp) * kBRing * kSlots;
    const SmemGrid g{ s_tab, s_sig, s_node, s_ab };

    for (int e = tid; e < B.max_IJe; e += Bk) l1[e] = 0.0f;
    if (tid == 0) s_ctl[2] = -1;
    __syncthreads();

    while (true) {
        if (tid == 0) s_ctl[0] = (int)atomicAdd(B.item_counter, 1u);
        __syncthreads();
        const int item = s_ctl[0];
        if (item >= B.n_items) break;
        const BookItem it = B.items[item];
        if (it.inst != s_ctl[2]) {
            // restage: this option's grid, time table and parameters
            if (tid == 0) build_params(B, it.inst, s_par);
            __syncthreads();
            const McParams& Q = *s_par;
            for (int e = tid; e < Q.Je * (Q.I - 1); e += Bk) s_sig[e] = Q.sig2[e];
            for (int e = tid; e < Q.I; e += Bk) s_node[e] = Q.node[e];
            for (int e = tid; e < Q.I - 1; e += Bk) s_ab[e] = Q.ab[e];
            for (int n = tid; n < Q.N; n += Bk) s_tab[n] = step_time(Q, n);
            if (tid == 0) s_ctl[2] = it.inst;
        }
        if (tid == 0) s_ctl[1] = it.first_tile;
        __syncthreads();
        const McParams P = *s_par;
        const int tile_end = it.first_tile + it.n_tiles;

        // per-thread binary64 sums in shared memory (keeps them out of the sweep's registers)
        double* acc = reinterpret_cast<double*>(smem + L.acc) + tid;    // [3][block]: V, V^2, xbar_0
        acc[0] = acc[Bk] = acc[2 * Bk] = 0.0;
        int q_head = 0, q_count = 0;
        unsigned fwd_count = 0;
        int tile = warp_claim(&s_ctl[1], PPL);
        while (true) {
            const int g_next = (int)(fwd_count % kBRing);
            const bool more = tile < tile_end;
            const bool reuse = more && q_count > 0 && q_slot[q_head] / kSlots == g_next;
            if (q_count >= 32 || (!more && q_count > 0) || reuse) {
                const int nb = min(32, q_count);
                if (lane < nb) {
                    const int e = (q_head + lane) & (kQcap - 1);
                    const long long rel = q_rel[e];
                    uint32_t c1, c2;
                    path_counter(P, rel, c1, c2);
                    const float xbar = reverse_path<KCK>(P, g, c1, c2, ckw + q_slot[e], cks, q_xb[e], l1);
                    acc[2 * Bk] += (double)xbar;
                }
                q_head = (q_head + nb) & (kQcap - 1);
                q_count -= nb;
                __syncwarp();
                continue;
            }
            if (!more) break;
            if constexpr (PPL == 2) {
                // tiles tile and tile + 1 of this item: two paths per lane (tile + 1 may lie
                // beyond the item, whose paths belong to another block's item)
                const long long rel_a = (long long)tile * 32 + lane, rel_b = rel_a + 32;
                const bool act_b = tile + 1 < tile_end && rel_b < P.n_paths;
                const int slot_a = g_next * kSlots + lane, slot_b = slot_a + 32;
                float xa = 0.0f, xb = 0.0f;
                if (rel_a < P.n_paths) {
                    uint32_t c1a, c2a, c1b, c2b;
                    path_counter(P, rel_a, c1a, c2a);
                    path_counter(P, rel_b, c1b, c2b);
                    float ya, yb;
                    forward_path2<KCK, true, false>(P, g, c1a, c2a, c1b, c2b, ckw + slot_a, ckw + slot_b, cks, rel_a,
                                                    rel_b, false, ya, yb);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 1 && !act_b) break;
                        const float SN = exp2f(h ? yb : ya);
                        const float itm = P.phi * (SN - P.K);
                        const float V = itm > 0.0f ? P.disc * itm : 0.0f;
                        (h ? xb : xa) = itm > 0.0f ? P.disc * P.phi * SN : 0.0f;
                        acc[0] += (double)V;
                        acc[Bk] += (double)V * (double)V;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float xbarN = h ? xb : xa;
                    const bool live = xbarN != 0.0f;
                    const unsigned bal = __ballot_sync(0xffffffffu, live);
                    if (live) {
                        const int e = (q_head + q_count + __popc(bal & ((1u << lane) - 1u))) & (kQcap - 1);
                        q_slot[e] = h ? slot_b : slot_a;
                        q_rel[e] = (int)(h ? rel_b : rel_a);
                        q_xb[e] = xbarN;
                    }
                    q_count += __popc(bal);
                }
                ++fwd_count;
                __syncwarp();
                tile = warp_claim(&s_ctl[1], PPL);
                continue;
            }
            const long long rel = (long long)tile * 32 + lane;
            const bool active = rel < P.n_paths;
            const int slot = g_next * 32 + lane;
            float xbarN = 0.0f;
            if (active) {
                uint32_t c1, c2;
                path_counter(P, rel, c1, c2);
                const float x = forward_path<KCK, true, false>(P, g, c1, c2, ckw + slot, cks, rel);
                const float SN = exp2f(x);
                const float itm = P.phi * (SN - P.K);
                const float V = itm > 0.0f ? P.disc * itm : 0.0f;
                xbarN = itm > 0.0f ? P.disc * P.phi * SN : 0.0f;
                acc[0] += (double)V;
                acc[Bk] += (double)V * (double)V;
            }
            const bool live = xbarN != 0.0f;
            const unsigned bal = __ballot_sync(0xffffffffu, live);
            if (live) {
                const int e = (q_head + q_count + __popc(bal & ((1u << lane) - 1u))) & (kQcap - 1);
                q_slot[e] = slot;
                q_rel[e] = (int)rel;
                q_xb[e] = xbarN;
            }
            q_count += __popc(bal);
            ++fwd_count;
            __syncwarp();
            tile = warp_claim(&s_ctl[1], PPL);
        }

        // end of item: add this block's sums to the option's binary64 sums
        double aV = acc[0], aV2 = acc[Bk], aX = acc[2 * Bk];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            aV += __shfl_down_sync(0xffffffffu, aV, o);
            aV2 += __shfl_down_sync(0xffffffffu, aV2, o);
            aX += __shfl_down_sync(0xffffffffu, aX, o);
        }
        if (lane == 0) {
            s_red[3 * warp + 0] = aV;
            s_red[3 * warp + 1] = aV2;
            s_red[3 * warp + 2] = aX;
        }
        __syncthreads();
        double* sums = B.sums + B.insts[it.inst].out_off;
        if (tid < 3) {
            double t = 0.0;
            for (int w = 0; w < W; ++w) t += s_red[3 * w + tid];
            atomicAdd(&sums[tid], t);
        }
        // vega buckets: the option's own sums, or (aggregated risk) its surface's,
        // scaled by the option's weight over its path count
        const BookInst& inst = B.insts[it.inst];
        double* vsum = B.risk ? B.risk + B.surfs[inst.surf].risk_off + 3 : sums + 3;
        const double vscale = B.risk ? inst.scale : 1.0;
        const int nIJ = P.Je * P.I;
        for (int e = tid; e < nIJ; e += Bk) {
            const float v = l1[e];
            if (v != 0.0f) {
                const int j = e / P.I, i = e - j * P.I;
                if (j < P.J) atomicAdd(&vsum[i * P.J + j], (double)v * vscale);   // spot-major sums
                l1[e] = 0.0f;
            }
        }
        __syncthreads();
    }
}

// Per option: [price, delta, stderr, vega...] from its binary64 sums.
__global__ void book_finalize_kernel(const BookInst* __restrict__ insts, const BookSurf* __restrict__ surfs,
                                     int n_inst, const double* __restrict__ sums, const BookRun* run,
                                     double* __restrict__ out)
{
    const int inst = blockIdx.y;
    if (inst >= n_inst) return;
    const BookInst& o = insts[inst];
    const int IJ = surfs[o.surf].I * surfs[o.surf].J;
    const double* s = sums + o.out_off;
    double* d = out + o.out_off;
    const double P = (double)o.n_paths;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < IJ + 3; e += gridDim.x * blockDim.x) {
        if (e == 0) {
            const double mean = s[0] / P;
            const double var = o.n_paths > 1 ? (s[1] / P - mean * mean) * P / (P - 1.0) : 0.0;
            d[LV_OUT_PRICE_DEV] = mean;
            d[LV_OUT_STDERR_DEV] = var > 0.0 ? sqrt(var / P) : 0.0;
            d[LV_OUT_DELTA_DEV] = s[2] / (P * exp2(run->log2_S0));
        } else if (e >= 3) {
            d[e] = s[e] / P;
        }
    }
}

// Aggregated risk per surface: the weighted option scalars (from each
// option's sums) and the vega part already summed with weights w / n_paths.
__global__ void book_risk_finalize_kernel(const BookInst* __restrict__ insts, const BookSurf* __restrict__ surfs,
                                          int n_inst, const double* __restrict__ sums,
                                          const double* __restrict__ risk, const BookRun* run,
                                          double* __restrict__ out)
{
    const int sf = blockIdx.y;
    const BookSurf& S = surfs[sf];
    const int IJ = S.I * S.J;
    double* d = out + S.risk_off;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < IJ + 3; e += gridDim.x * blockDim.x) {
        if (e >= 3) {
            d[e] = risk[S.risk_off + e];
        } else if (e == 0) {
            const double S0 = exp2(run->log2_S0);
            double price = 0.0, delta = 0.0, var = 0.0;
            for (int o = 0; o < n_inst; ++o) {
                const BookInst& q = insts[o];
                if (q.surf != sf) continue;
                const double* s = sums + q.out_off;
                const double P = (double)q.n_paths;
                const double mean = s[0] / P;
                const double v = q.n_paths > 1 ? (s[1] / P - mean * mean) * P / (P - 1.0) : 0.0;
                price += q.w * mean;
                delta += q.w * s[2] / (P * S0);
                var += q.w * q.w * (v > 0.0 ? v / P : 0.0);
            }
            d[LV_OUT_PRICE_DEV] = price;
            d[LV_OUT_DELTA_DEV] = delta;
            d[LV_OUT_STDERR_DEV] = sqrt(var);
        }
    }
}

template <int KCK, int PPL>
cudaError_t book_launch_k(const BookParams& b, int grid, int block, size_t smem, cudaStream_t s)
{
    book_kernel<KCK, PPL><<<grid, block, smem, s>>>(b);
    return cudaGetLastError();
}

// The book kernel of (k, paths per lane): k in {4, 8}, ppl in {1, 2}.
template <typename F>
cudaError_t with_book_kernel(int k, int ppl, F&& f)
{
    switch (k * 4 + ppl) {
    case 17: return f(book_kernel<4, 1>);
    case 18: return f(book_kernel<4, 2>);
    case 33: return f(book_kernel<8, 1>);
    case 34: return f(book_kernel<8, 2>);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t book_smem_bytes(int maxI, int maxJe, int maxN, int block, int ppl)
{
    return book_layout(maxI, maxJe, maxN, block, ppl).total;
}

int book_ring_slots_per_warp() { return kBRing * 32; }

cudaError_t book_prepare(int k, int ppl)
{
    return with_book_kernel(k, ppl, [](auto kernel) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
}

cudaError_t book_occupancy(int block, int k, int ppl, size_t smem, int* bps)
{
    cudaError_t e = book_prepare(k, ppl);
    if (e != cudaSuccess) return e;
    return with_book_kernel(k, ppl, [&](auto kernel) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kernel, block, smem);
    });
}

cudaError_t launch_book(const BookParams& b, int grid, int block, int k, int ppl, size_t smem, cudaStream_t s)
{
    switch (k * 4 + ppl) {
    case 17: return book_launch_k<4, 1>(b, grid, block, smem, s);
    case 18: return book_launch_k<4, 2>(b, grid, block, smem, s);
    case 33: return book_launch_k<8, 1>(b, grid, block, smem, s);
    case 34: return book_launch_k<8, 2>(b, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_book_risk_finalize(const BookParams& b, int n_surf, int n_inst, int max_IJ, double* out,
                                      cudaStream_t s)
{
    dim3 grid((max_IJ + 3 + 255) / 256, n_surf);
    book_risk_finalize_kernel<<<grid, 256, 0, s>>>(b.insts, b.surfs, n_inst, b.sums, b.risk, b.run, out);
    return cudaGetLastError();
}

cudaError_t launch_book_finalize(const BookParams& b, int n_inst, int max_IJ, double* out, cudaStream_t s)
{
    dim3 grid((max_IJ + 3 + 255) / 256, n_inst);
    book_finalize_kernel<<<grid, 256, 0, s>>>(b.insts, b.surfs, n_inst, b.sums, b.run, out);
    return cudaGetLastError();
}

}  // namespace lv
