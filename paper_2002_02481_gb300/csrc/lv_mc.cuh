// lv_mc.cuh -- the Monte Carlo price / pathwise-adjoint kernels (arXiv
// 2002.02481, Sec. III, IV-A..IV-D), templated on the model (the reading of
// the scheme and of the interpolation, see lv_device.cuh). Every translation
// unit that includes this header instantiates its own kernels with internal
// linkage: lv_kernels.cu the main model, lv_model1..3.cu the others.
//
// Adjoint kernel: persistent, warp-centric, no block-wide barrier in its
// main loop. Every warp repeatedly either
//   (F) claims a tile of 32 consecutive paths from a global counter and runs
//       their forward passes: normals generated in registers, log-Euler
//       steps under the bilinear grid staged in shared memory, x stored every
//       KCK steps (the checkpoints) into one of kRing groups of 32 slots
//       owned by the warp; payoff and terminal adjoint
//       xbar_N = e^{-rT} 1{phi(S_N - K) > 0} phi S_N; the paths with a
//       nonzero xbar_N (all others have a zero adjoint everywhere) are
//       appended to a per-warp FIFO in shared memory; or
//   (R) takes up to 32 queued paths and runs their reverse sweeps: per
//       checkpoint segment, last to first, recompute KCK steps from the
//       checkpoint with the same Philox counters keeping h_n = d x_{n+1} /
//       d sigma_n, g_n = h_n S_n d sigma / d S, the cell and the weight in
//       registers, then walk back: sigma_bar_n = xbar_{n+1} h_n,
//       xbar_n = xbar_{n+1} (1 + g_n), sigma_bar_n spread over the four
//       corner buckets with the bilinear weights.
// A reverse batch runs when 32 paths are queued, when the oldest queued
// path's checkpoint slots are about to be reused by the next forward tile,
// and at the end; so the reverse sweeps run on full warps. With two paths
// per lane (PPL = 2) a warp claims two consecutive tiles and advances each
// lane's two paths together, their binary32 arithmetic in packed .f32x2
// pairs (forward_path2); the slot groups and the FIFO double, the reverse
// batches stay at 32 paths.
//
// Bucket accumulation: run-length sums in registers while the cell is
// unchanged (level 0); binary32 reductions (red.global.add.f32, resolved in
// L2 without a retry loop) into a per-block bucket array in global memory
// (level 1); every few batches a warp drains that array (atomicExch) into
// level 2: the block's binary64 row through binary64 reductions, or in Kahan
// mode a compensated binary32 row the warp owns; at the end each block folds
// what is left into its binary64 row, and a separate fixed-order binary64
// reduction over blocks gives the outputs (level 3).
//
// The DBG instantiation additionally writes per-path results and logs
// every forward step whose spot lies within a relative band of its cell's
// nodes, with the cell and inside-grid decision taken there, so that a
// test can hand the same decisions to the binary64 oracle.
#pragma once

#include <math.h>

#include "lv_device.cuh"

namespace lv {

namespace {

constexpr int kTile = 32;      // paths per warp tile of the adjoint kernel (one per lane)
constexpr int kPriceTile = 64; // paths per warp tile of the price kernel (two per lane)
constexpr int kRing = 4;       // checkpoint slot groups of kTile per warp

constexpr int kQueue = 64;     // per-warp FIFO capacity per path a lane runs in a forward tile
                               // (entries; < 32 + kTile * ppl never overflows kQueue * ppl)
constexpr int kMaxWarps = 8;   // blockDim.x <= 256 (the adjoint kernel runs at most 128)

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Level-2 accumulator of one value: binary64 or Kahan-compensated binary32.
// The slots live in shared memory (one per thread and value), which keeps
// them out of the registers the reverse sweep needs.
struct AccSlot {
    double d;
    float s, c;
};

struct SmemLayout {
    size_t tab, sig, node, ab, tdt, qslot, qrel, qxb, acc, red, total;
};

// extra: the adjoint kernel that also sums d V / d r and d V / d T (the time
// slope table and two more accumulators per thread); ppl: paths per lane of
// the adjoint's forward tiles (the FIFO grows with it).
__host__ __device__ inline SmemLayout smem_layout(int I, int Je, int N, int block, bool greeks, bool grid_smem,
                                                  bool extra = false, int ppl = 1)
{
    const int W = block / 32;
    SmemLayout L;
    size_t o = 0;
    L.tab = o;   o += align16(sizeof(int4) * (size_t)N);
    L.sig = o;   if (grid_smem) o += align16(sizeof(float2) * (size_t)Je * (I - 1));
    L.node = o;  o += align16(sizeof(float) * (size_t)I);
    L.ab = o;    o += align16(sizeof(float2) * (size_t)I);
    L.tdt = o;   if (extra) o += align16(sizeof(float) * (size_t)N);
    // the adjoint kernel slices these three per warp from L.qslot: they stay
    // contiguous because each size is a multiple of 16 bytes (kQueue is)
    static_assert(kQueue % 4 == 0, "FIFO arrays must stay contiguous");
    L.qslot = o; if (greeks) o += align16(sizeof(int) * (size_t)W * kQueue * ppl);
    L.qrel = o;  if (greeks) o += align16(sizeof(int) * (size_t)W * kQueue * ppl);
    L.qxb = o;   if (greeks) o += align16(sizeof(float) * (size_t)W * kQueue * ppl);
    L.acc = o;   o += align16(sizeof(AccSlot) * (extra ? 5 : 3) * (size_t)block);
    L.red = o;   o += align16(sizeof(double) * 3 * kMaxWarps);
    L.total = o;
    return L;
}

// Adds x to a level-2 slot.
template <int ACC>
__device__ __forceinline__ void acc_add(AccSlot& a, float x)
{
    if (ACC == 1) {
        const float y = x - a.c;
        const float t = a.s + y;
        a.c = (t - a.s) - y;
        a.s = t;
    } else {
        a.d += (double)x;
    }
}

template <int ACC>
__device__ __forceinline__ double acc_value(const AccSlot& a)
{
    return ACC == 1 ? (double)a.s - (double)a.c : a.d;
}

// Stages the time table, the spot nodes, the cell coefficients and (when GS)
// the sigma pairs in shared memory; large grids are read from global memory
// through L1 instead, which leaves room for more resident blocks.
template <bool GS, bool EXTRA = false>
__device__ __forceinline__ void stage_grid(const McParams& P, unsigned char* smem, const SmemLayout& L)
{
    const int B = blockDim.x, tid = threadIdx.x;
    int4* s_tab = reinterpret_cast<int4*>(smem + L.tab);
    float2* s_sig = reinterpret_cast<float2*>(smem + L.sig);
    float* s_node = reinterpret_cast<float*>(smem + L.node);
    float2* s_ab = reinterpret_cast<float2*>(smem + L.ab);
    if (GS)
        for (int e = tid; e < P.Je * (P.I - 1); e += B) s_sig[e] = P.sig2[e];
    for (int e = tid; e < P.I; e += B) s_node[e] = P.node[e];
    for (int e = tid; e < P.I - 1; e += B) s_ab[e] = P.ab[e];
    for (int n = tid; n < P.N; n += B) s_tab[n] = step_time(P, n);
    if (EXTRA) {
        float* s_tdt = reinterpret_cast<float*>(smem + L.tdt);
        for (int n = tid; n < P.N; n += B) s_tdt[n] = step_tdt(P, n);
    }
}

// Block sum of three per-thread binary64 values into row[0..2] (fixed order).
__device__ __forceinline__ void block_scalars(double a, double b, double c, double* s_red, double* row, int n = 3)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sa += s_red[3 * w + 0];
            sb += s_red[3 * w + 1];
            sc += s_red[3 * w + 2];
        }
        row[0] = sa;
        row[1] = sb;
        if (n > 2) row[2] = sc;
    }
}

// Claims n consecutive tiles for the warp; returns the first.
__device__ __forceinline__ int claim_tile(unsigned int* counter, unsigned n = 1u)
{
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = (int)atomicAdd(counter, n);
    return __shfl_sync(0xffffffffu, t, 0);
}

template <int ACC>
__device__ __forceinline__ void drain_buckets(float* l1, int nIJ, double* wrow)
{
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < nIJ; e += 32) {
        if (l1[e] == 0.0f) continue;            // a skipped bucket is drained later
        const float v = atomicExch(&l1[e], 0.0f);
        if (ACC == 1) {
            float2* k = reinterpret_cast<float2*>(wrow) + e;
            float2 p = *k;
            const float y = v - p.y;
            const float t = p.x + y;
            p.y = (t - p.x) - y;
            p.x = t;
            *k = p;
        } else {
            atomicAdd(&wrow[e], (double)v);       // the block's row, shared by its warps
        }
    }
}

// PPL: paths per lane of a forward tile. With PPL = 2 a warp claims two
// consecutive 32-path tiles and runs them interleaved (forward_path2: two
// independent dependency chains per lane, the per-step time data loaded once);
// each path's arithmetic is that of PPL = 1, the ring groups and the FIFO
// hold twice as many entries, and the reverse batches are unchanged.
template <int KCK, int ACC, bool DBG, bool GS, int MODEL, bool EXTRA = false, int PPL = 1>
__global__ void __launch_bounds__(128, 5) adjoint_kernel(const __grid_constant__ McParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kSlots = kTile * PPL;      // checkpoint slots per ring group
    constexpr int kQcap = kQueue * PPL;      // FIFO entries per warp
    const int B = blockDim.x, W = B >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SmemLayout L = smem_layout(P.I, P.Je, P.N, B, true, GS, EXTRA, PPL);
    stage_grid<GS, EXTRA>(P, smem, L);
    float* l1 = P.l1 + (size_t)blockIdx.x * (P.Je * P.I);    // this block's level-1 buckets
    // the three FIFO arrays of all warps are contiguous from L.qslot (each
    // W * kQcap words): one base per warp, the others at fixed offsets, which
    // keeps two registers free for the packed forward pass
    int* const q_slot = reinterpret_cast<int*>(smem + L.qslot) + warp * 3 * kQcap;
    int* const q_rel = q_slot + kQcap;
    float* const q_xb = reinterpret_cast<float*>(q_slot + 2 * kQcap);
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    const int nIJ = P.Je * P.I;
    for (int e = tid; e < nIJ; e += B) l1[e] = 0.0f;
    const int wid = blockIdx.x * W + warp;                    // global warp id
    // level 2: binary64 mode drains into the block's own row with binary64
    // reductions; Kahan pairs cannot be updated atomically, so each warp owns one
    double* const row = P.partials + (size_t)blockIdx.x * P.row_words;
    double* wrow;
    if (ACC == 1) {
        wrow = P.warp_rows + (size_t)wid * nIJ;
        for (int e = lane; e < nIJ; e += 32) wrow[e] = 0.0;   // zero as a float2 pair too
    } else {
        wrow = row + 3;
        for (int e = tid; e < nIJ; e += B) wrow[e] = 0.0;
    }
    __syncthreads();

    const SmemGrid g{ reinterpret_cast<const int4*>(smem + L.tab),
                      GS ? reinterpret_cast<const float2*>(smem + L.sig) : P.sig2,
                      reinterpret_cast<const float*>(smem + L.node), reinterpret_cast<const float2*>(smem + L.ab),
                      reinterpret_cast<const float*>(smem + L.tdt) };
    const size_t cks = (size_t)gridDim.x * W * kRing * kSlots;  // checkpoint stride
    float* const ckw = P.ckpt + (size_t)wid * kRing * kSlots;    // this warp's slots

    AccSlot* acc = reinterpret_cast<AccSlot*>(smem + L.acc) + tid;   // [3][block]: V, V^2, xbar_0
    acc[0] = acc[B] = acc[2 * B] = AccSlot{0.0, 0.0f, 0.0f};
    if (EXTRA) acc[3 * B] = acc[4 * B] = AccSlot{0.0, 0.0f, 0.0f};    // d V / d r, d V / d T
    int q_head = 0, q_count = 0, batches = 0;
    unsigned fwd_count = 0;
    int tile = claim_tile(P.tile_counter, PPL);

    while (true) {
        const int g_next = (int)(fwd_count % kRing);
        const bool more = tile < P.n_tiles;
        const bool reuse = more && q_count > 0 && q_slot[q_head] / kSlots == g_next;
        if (q_count >= 32 || (!more && q_count > 0) || reuse) {
            // ---------------- reverse batch over up to 32 queued paths
            const int nb = min(32, q_count);
            if (lane < nb) {
                const int e = (q_head + lane) & (kQcap - 1);
                const int slot = q_slot[e];
                const long long rel = q_rel[e];
                float xbar = q_xb[e];
                uint32_t c1, c2;
                path_counter(P, rel, c1, c2);
                float ra = 0.0f, ta = 0.0f;
                xbar = reverse_path<KCK, MODEL, EXTRA, PPL == 2 && (MODEL & kModelEulerS) == 0>(
                    P, g, c1, c2, ckw + slot, cks, xbar, l1, &ra, &ta);
                acc_add<ACC>(acc[2 * B], xbar);
                if (EXTRA) {
                    acc_add<ACC>(acc[3 * B], ra);
                    acc_add<ACC>(acc[4 * B], ta);
                }
                if (DBG) P.dbg_xbar0[rel] = xbar;
            }
            q_head = (q_head + nb) & (kQcap - 1);
            q_count -= nb;
            __syncwarp();
            if (++batches % P.flush_every == 0)      // the level-2 row, recomputed (one register less)
                drain_buckets<ACC>(l1, nIJ, ACC == 1 ? P.warp_rows + (size_t)wid * nIJ
                                                     : P.partials + (size_t)blockIdx.x * P.row_words + 3);
            continue;
        }
        if (!more) break;

        if constexpr (PPL == 2) {
            // ---------------- forward tiles tile, tile + 1: two paths per lane
            const long long rel_a = (long long)tile * kTile + lane, rel_b = rel_a + kTile;
            const int slot_a = g_next * kSlots + lane, slot_b = slot_a + kTile;
            float xa = 0.0f, xb = 0.0f;
            if (rel_a < P.n_paths) {
                uint32_t c1a, c2a, c1b, c2b;
                path_counter(P, rel_a, c1a, c2a);
                path_counter(P, rel_b, c1b, c2b);
                float ya, yb;
                // packed pairs on the log-Euler readings; Euler on S keeps scalar pairs in
                // this kernel (packed, it needs 82 registers: 5 blocks per SM instead of 6)
                forward_path2<KCK, true, false, MODEL, (MODEL & kModelEulerS) == 0>(
                    P, g, c1a, c2a, c1b, c2b, ckw + slot_a, ckw + slot_b, cks, rel_a, rel_b, false, ya, yb);
                float V;
                payoff<MODEL>(P, ya, V, xa);
                acc_add<ACC>(acc[0], V);
                acc_add<ACC>(acc[B], V * V);
                if (rel_b < P.n_paths) {
                    payoff<MODEL>(P, yb, V, xb);
                    acc_add<ACC>(acc[0], V);
                    acc_add<ACC>(acc[B], V * V);
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
            tile = claim_tile(P.tile_counter, PPL);
            continue;
        }

        // ---------------- forward tile of 32 paths into slot group g_next
        const long long rel = (long long)tile * kTile + lane;
        const bool active = rel < P.n_paths;
        const int slot = g_next * kTile + lane;
        float xbarN = 0.0f;
        if (active) {
            uint32_t c1, c2;
            path_counter(P, rel, c1, c2);
            const float x = forward_path<KCK, true, DBG, MODEL>(P, g, c1, c2, ckw + slot, cks, rel);
            float V;
            payoff<MODEL>(P, x, V, xbarN);
            acc_add<ACC>(acc[0], V);
            acc_add<ACC>(acc[B], V * V);
            if (EXTRA) {                       // the discount's share: -T V and -r V
                acc_add<ACC>(acc[3 * B], -P.Tf * V);
                acc_add<ACC>(acc[4 * B], -P.r_nat * V);
            }
            if (DBG) {
                P.dbg_xN[rel] = ln_spot<MODEL>(x);
                P.dbg_V[rel] = V;
                P.dbg_xbar0[rel] = 0.0f;
            }
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
        tile = claim_tile(P.tile_counter, PPL);
    }

    // fold: remaining level-1 buckets (and, in Kahan mode, every warp row of
    // this block) into the block's binary64 row (after the barrier nothing adds)
    __syncthreads();
    // the kernel that also sums d V / d r and d V / d T recomputes its row here
    // instead of keeping the pointer live through the loop (80 registers, 6
    // blocks per SM, instead of 87 and 5)
    double* const row_f = EXTRA ? P.partials + (size_t)blockIdx.x * P.row_words : row;
    const double* rows0 = P.warp_rows + (size_t)blockIdx.x * W * nIJ;
    for (int e = tid; e < nIJ; e += B) {
        if (ACC == 1) {
            double s = (double)l1[e];
            for (int w = 0; w < W; ++w) {
                const float2 k = reinterpret_cast<const float2*>(rows0 + (size_t)w * nIJ)[e];
                s += (double)k.x - (double)k.y;
            }
            row_f[3 + e] = s;
        } else {
            row_f[3 + e] += (double)l1[e];
        }
    }
    block_scalars(acc_value<ACC>(acc[0]), acc_value<ACC>(acc[B]), acc_value<ACC>(acc[2 * B]), s_red, row_f);
    if (EXTRA) {
        __syncthreads();                       // s_red is reused
        block_scalars(acc_value<ACC>(acc[3 * B]), acc_value<ACC>(acc[4 * B]), 0.0, s_red, row_f + 3 + nIJ, 2);
    }
}

// Tangent-ratio adjoint (LV_ADJ_TANGENT): persistent and warp-centric like
// adjoint_kernel, without checkpoints. A warp claims a tile of 32 paths and
// runs pass 1 (tangent_forward): payoff, xbar_N, and xbar_0 = xbar_N D_N;
// the paths with xbar_N != 0 join the warp's queue with c = xbar_N D_N. At
// 32 queued paths (and at the end) the warp runs pass 2 (tangent_scatter)
// on them as a full-warp batch. Buckets go through the same levels 0-3.
template <int ACC, bool GS, int MODEL, int PPL = 1>
__global__ void __launch_bounds__(128, 6) tangent_kernel(const __grid_constant__ McParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = blockDim.x, W = B >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kQcap = kQueue * PPL;
    const SmemLayout L = smem_layout(P.I, P.Je, P.N, B, true, GS, false, PPL);
    stage_grid<GS>(P, smem, L);
    float* l1 = P.l1 + (size_t)blockIdx.x * (P.Je * P.I);
    int* q_rel = reinterpret_cast<int*>(smem + L.qrel) + warp * kQcap;
    float* q_c = reinterpret_cast<float*>(smem + L.qxb) + warp * kQcap;
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    const int nIJ = P.Je * P.I;
    for (int e = tid; e < nIJ; e += B) l1[e] = 0.0f;
    const int wid = blockIdx.x * W + warp;
    double* const row = P.partials + (size_t)blockIdx.x * P.row_words;
    double* wrow;
    if (ACC == 1) {
        wrow = P.warp_rows + (size_t)wid * nIJ;
        for (int e = lane; e < nIJ; e += 32) wrow[e] = 0.0;
    } else {
        wrow = row + 3;
        for (int e = tid; e < nIJ; e += B) wrow[e] = 0.0;
    }
    __syncthreads();
    const SmemGrid g{ reinterpret_cast<const int4*>(smem + L.tab),
                      GS ? reinterpret_cast<const float2*>(smem + L.sig) : P.sig2,
                      reinterpret_cast<const float*>(smem + L.node), reinterpret_cast<const float2*>(smem + L.ab) };
    AccSlot* acc = reinterpret_cast<AccSlot*>(smem + L.acc) + tid;   // [3][block]: V, V^2, xbar_0
    acc[0] = acc[B] = acc[2 * B] = AccSlot{0.0, 0.0f, 0.0f};
    int q_head = 0, q_count = 0, batches = 0;
    int tile = claim_tile(P.tile_counter, PPL);
    while (true) {
        const bool more = tile < P.n_tiles;
        if (q_count >= 32 || (!more && q_count > 0)) {
            const int nb = min(32, q_count);
            if (lane < nb) {
                const int e = (q_head + lane) & (kQcap - 1);
                uint32_t c1, c2;
                path_counter(P, q_rel[e], c1, c2);
                tangent_scatter<MODEL>(P, g, c1, c2, q_c[e], l1);
            }
            q_head = (q_head + nb) & (kQcap - 1);
            q_count -= nb;
            __syncwarp();
            if (++batches % P.flush_every == 0) drain_buckets<ACC>(l1, nIJ, wrow);
            continue;
        }
        if (!more) break;
        if constexpr (PPL == 2) {
            // pass 1 on tiles tile, tile + 1: two paths per lane in packed pairs
            const long long rel_a = (long long)tile * kTile + lane, rel_b = rel_a + kTile;
            float xa = 0.0f, xb = 0.0f, ca = 0.0f, cb = 0.0f;
            if (rel_a < P.n_paths) {
                uint32_t c1a, c2a, c1b, c2b;
                path_counter(P, rel_a, c1a, c2a);
                path_counter(P, rel_b, c1b, c2b);
                float ya, yb, Da, Db, V;
                bool ta, tb;
                tangent_forward2(P, g, c1a, c2a, c1b, c2b, ya, yb, Da, Db, ta, tb);
                payoff<0>(P, ya, V, xa);
                ca = xa * Da;
                acc_add<ACC>(acc[0], V);
                acc_add<ACC>(acc[B], V * V);
                acc_add<ACC>(acc[2 * B], ca);
                if (ta && xa != 0.0f) atomicAdd(P.flag, 1u);
                if (rel_b < P.n_paths) {
                    payoff<0>(P, yb, V, xb);
                    cb = xb * Db;
                    acc_add<ACC>(acc[0], V);
                    acc_add<ACC>(acc[B], V * V);
                    acc_add<ACC>(acc[2 * B], cb);
                    if (tb && xb != 0.0f) atomicAdd(P.flag, 1u);
                }
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const float x = hh ? xb : xa;
                const bool live = x != 0.0f;
                const unsigned bal = __ballot_sync(0xffffffffu, live);
                if (live) {
                    const int e = (q_head + q_count + __popc(bal & ((1u << lane) - 1u))) & (kQcap - 1);
                    q_rel[e] = (int)(hh ? rel_b : rel_a);
                    q_c[e] = hh ? cb : ca;
                }
                q_count += __popc(bal);
            }
            __syncwarp();
            tile = claim_tile(P.tile_counter, PPL);
            continue;
        }
        const long long rel = (long long)tile * kTile + lane;
        float xbarN = 0.0f, c = 0.0f;
        if (rel < P.n_paths) {
            uint32_t c1, c2;
            path_counter(P, rel, c1, c2);
            float D;
            bool tiny;
            const float y = tangent_forward<MODEL>(P, g, c1, c2, D, tiny);
            float V;
            payoff<MODEL>(P, y, V, xbarN);
            c = xbarN * D;
            acc_add<ACC>(acc[0], V);
            acc_add<ACC>(acc[B], V * V);
            acc_add<ACC>(acc[2 * B], c);
            if (tiny && xbarN != 0.0f) atomicAdd(P.flag, 1u);
        }
        const bool live = xbarN != 0.0f;
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        if (live) {
            const int e = (q_head + q_count + __popc(bal & ((1u << lane) - 1u))) & (kQcap - 1);
            q_rel[e] = (int)rel;
            q_c[e] = c;
        }
        q_count += __popc(bal);
        __syncwarp();
        tile = claim_tile(P.tile_counter, PPL);
    }
    __syncthreads();
    const double* rows0 = P.warp_rows + (size_t)blockIdx.x * W * nIJ;
    for (int e = tid; e < nIJ; e += B) {
        if (ACC == 1) {
            double s = (double)l1[e];
            for (int w = 0; w < W; ++w) {
                const float2 k = reinterpret_cast<const float2*>(rows0 + (size_t)w * nIJ)[e];
                s += (double)k.x - (double)k.y;
            }
            row[3 + e] = s;
        } else {
            row[3 + e] += (double)l1[e];
        }
    }
    block_scalars(acc_value<ACC>(acc[0]), acc_value<ACC>(acc[B]), acc_value<ACC>(acc[2 * B]), s_red, row);
}

// Second-order buckets (lv_price_greeks_vanna): the tangent-ratio kernel's
// structure with pass 2 replaced by vanna_scatter. Pass 1 (tangent_forward)
// gives the payoff and x_bar_0 = x_bar_N D_N, hence Delta_p = x_bar_0 / S0;
// live paths are queued and scattered in full-warp batches. Main reading,
// binary64 level 2. Rows: price sums as usual, buckets d^2 price / (d S0 d
// sigma_ij) summed over paths.
template <bool GS, int PPL = 1>
__global__ void __launch_bounds__(128, 6) vanna_kernel(const __grid_constant__ McParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kQcap = kQueue * PPL;
    const SmemLayout L = smem_layout(P.I, P.Je, P.N, B, true, GS, false, PPL);
    stage_grid<GS>(P, smem, L);
    float* l1 = P.l1 + (size_t)blockIdx.x * (P.Je * P.I);
    int* q_rel = reinterpret_cast<int*>(smem + L.qrel) + warp * kQcap;
    float* q_c = reinterpret_cast<float*>(smem + L.qxb) + warp * kQcap;
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    const int nIJ = P.Je * P.I;
    for (int e = tid; e < nIJ; e += B) l1[e] = 0.0f;
    double* const row = P.partials + (size_t)blockIdx.x * P.row_words;
    double* const wrow = row + 3;
    for (int e = tid; e < nIJ; e += B) wrow[e] = 0.0;
    __syncthreads();
    const SmemGrid g{ reinterpret_cast<const int4*>(smem + L.tab),
                      GS ? reinterpret_cast<const float2*>(smem + L.sig) : P.sig2,
                      reinterpret_cast<const float*>(smem + L.node), reinterpret_cast<const float2*>(smem + L.ab) };
    AccSlot* acc = reinterpret_cast<AccSlot*>(smem + L.acc) + tid;   // [3][block]: V, V^2, xbar_0
    acc[0] = acc[B] = acc[2 * B] = AccSlot{0.0, 0.0f, 0.0f};
    int q_head = 0, q_count = 0, batches = 0;
    int tile = claim_tile(P.tile_counter, PPL);
    while (true) {
        const bool more = tile < P.n_tiles;
        if (q_count >= 32 || (!more && q_count > 0)) {
            const int nb = min(32, q_count);
            if (lane < nb) {
                const int e = (q_head + lane) & (kQcap - 1);
                uint32_t c1, c2;
                path_counter(P, q_rel[e], c1, c2);
                vanna_scatter(P, g, c1, c2, q_c[e] * P.inv_S0, l1);
            }
            q_head = (q_head + nb) & (kQcap - 1);
            q_count -= nb;
            __syncwarp();
            if (++batches % P.flush_every == 0) drain_buckets<0>(l1, nIJ, wrow);
            continue;
        }
        if (!more) break;
        if constexpr (PPL == 2) {
            // pass 1 on tiles tile, tile + 1: two paths per lane in packed pairs
            const long long rel_a = (long long)tile * kTile + lane, rel_b = rel_a + kTile;
            float xa = 0.0f, xb = 0.0f, ca = 0.0f, cb = 0.0f;
            if (rel_a < P.n_paths) {
                uint32_t c1a, c2a, c1b, c2b;
                path_counter(P, rel_a, c1a, c2a);
                path_counter(P, rel_b, c1b, c2b);
                float ya, yb, Da, Db, V;
                bool ta, tb;
                tangent_forward2(P, g, c1a, c2a, c1b, c2b, ya, yb, Da, Db, ta, tb);
                payoff<0>(P, ya, V, xa);
                ca = xa * Da;
                acc_add<0>(acc[0], V);
                acc_add<0>(acc[B], V * V);
                acc_add<0>(acc[2 * B], ca);
                if (ta && xa != 0.0f) atomicAdd(P.flag, 1u);
                if (rel_b < P.n_paths) {
                    payoff<0>(P, yb, V, xb);
                    cb = xb * Db;
                    acc_add<0>(acc[0], V);
                    acc_add<0>(acc[B], V * V);
                    acc_add<0>(acc[2 * B], cb);
                    if (tb && xb != 0.0f) atomicAdd(P.flag, 1u);
                }
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const float x = hh ? xb : xa;
                const bool live = x != 0.0f;
                const unsigned bal = __ballot_sync(0xffffffffu, live);
                if (live) {
                    const int e = (q_head + q_count + __popc(bal & ((1u << lane) - 1u))) & (kQcap - 1);
                    q_rel[e] = (int)(hh ? rel_b : rel_a);
                    q_c[e] = hh ? cb : ca;
                }
                q_count += __popc(bal);
            }
            __syncwarp();
            tile = claim_tile(P.tile_counter, PPL);
            continue;
        }
        const long long rel = (long long)tile * kTile + lane;
        float xbarN = 0.0f, c = 0.0f;
        if (rel < P.n_paths) {
            uint32_t c1, c2;
            path_counter(P, rel, c1, c2);
            float D;
            bool tiny;
            const float y = tangent_forward<0>(P, g, c1, c2, D, tiny);
            float V;
            payoff<0>(P, y, V, xbarN);
            c = xbarN * D;
            acc_add<0>(acc[0], V);
            acc_add<0>(acc[B], V * V);
            acc_add<0>(acc[2 * B], c);
            if (tiny && xbarN != 0.0f) atomicAdd(P.flag, 1u);
        }
        const bool live = xbarN != 0.0f;
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        if (live) {
            const int e = (q_head + q_count + __popc(bal & ((1u << lane) - 1u))) & (kQcap - 1);
            q_rel[e] = (int)rel;
            q_c[e] = c;
        }
        q_count += __popc(bal);
        __syncwarp();
        tile = claim_tile(P.tile_counter, PPL);
    }
    __syncthreads();
    for (int e = tid; e < nIJ; e += B) row[3 + e] += (double)l1[e];
    block_scalars(acc_value<0>(acc[0]), acc_value<0>(acc[B]), acc_value<0>(acc[2 * B]), s_red, row);
}

template <int ACC, bool GS, int MODEL>
__global__ void __launch_bounds__(256, 4) price_kernel(const __grid_constant__ McParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(P.I, P.Je, P.N, blockDim.x, false, GS);
    stage_grid<GS>(P, smem, L);
    __syncthreads();
    const SmemGrid g{ reinterpret_cast<const int4*>(smem + L.tab),
                      GS ? reinterpret_cast<const float2*>(smem + L.sig) : P.sig2,
                      reinterpret_cast<const float*>(smem + L.node), reinterpret_cast<const float2*>(smem + L.ab) };
    const int lane = threadIdx.x & 31;
    AccSlot* acc = reinterpret_cast<AccSlot*>(smem + L.acc) + threadIdx.x;
    acc[0] = acc[blockDim.x] = AccSlot{0.0, 0.0f, 0.0f};
    for (int tile = claim_tile(P.tile_counter); tile < P.n_tiles; tile = claim_tile(P.tile_counter)) {
        const long long rel_a = (long long)tile * kPriceTile + lane, rel_b = rel_a + 32;
        if (rel_a < P.n_paths) {
            uint32_t c1a, c2a, c1b, c2b;
            path_counter(P, rel_a, c1a, c2a);
            path_counter(P, rel_b, c1b, c2b);
            float ya, yb;
            forward_path2<4, false, false, MODEL, true>(P, g, c1a, c2a, c1b, c2b, nullptr, nullptr, 0, rel_a, rel_b,
                                                        false, ya, yb);
            float V, xb;
            payoff<MODEL>(P, ya, V, xb);
            acc_add<ACC>(acc[0], V);
            acc_add<ACC>(acc[blockDim.x], V * V);
            if (rel_b < P.n_paths) {
                payoff<MODEL>(P, yb, V, xb);
                acc_add<ACC>(acc[0], V);
                acc_add<ACC>(acc[blockDim.x], V * V);
            }
        }
    }
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    block_scalars(acc_value<ACC>(acc[0]), acc_value<ACC>(acc[blockDim.x]), 0.0, s_red,
                  P.partials + (size_t)blockIdx.x * P.row_words);
}

template <typename K>
cudaError_t set_smem_attr(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename K>
cudaError_t launch_configured(K kernel, bool& configured, const McParams& p, int grid, int block, size_t smem,
                              cudaStream_t s)
{
    if (!configured) {
        cudaError_t e = set_smem_attr(kernel);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kernel<<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename K>
cudaError_t occupancy(K kernel, int block, size_t smem, int* bps)
{
    cudaError_t e = set_smem_attr(kernel);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kernel, block, smem);
}

// Calls f(kernel, flag) with the instantiation for (greeks, k, acc, dbg, gs)
// of model MODEL: k in {4, 8, 16, 32} for model 0, {4, 8} for the others.
template <int MODEL, bool GS, typename F>
cudaError_t with_kernel_gs(bool greeks, int k, int acc, bool dbg, int method, bool extra, F&& f, int ppl = 1)
{
    if (ppl == 2) {        // two paths per lane: the reverse sweep (k = 4 or 8) of every reading,
                           // the main reading's tangent-ratio adjoint and second-order buckets
        if (!greeks || dbg || extra) return cudaErrorInvalidValue;
        if constexpr (MODEL == 0) {
            static bool cv2 = false, ct2[2] = {};
            if (method == kMethodVanna)
                return acc == 0 ? f(vanna_kernel<GS, 2>, cv2) : cudaErrorInvalidValue;
            if (method == LV_ADJ_TANGENT)
                return acc ? f(tangent_kernel<1, GS, 0, 2>, ct2[1]) : f(tangent_kernel<0, GS, 0, 2>, ct2[0]);
        }
        if (method != LV_ADJ_REVERSE) return cudaErrorInvalidValue;
        static bool cp[4] = {};
        switch (k * 2 + acc) {
        case 8: return f(adjoint_kernel<4, 0, false, GS, MODEL, false, 2>, cp[0]);
        case 9: return f(adjoint_kernel<4, 1, false, GS, MODEL, false, 2>, cp[1]);
        case 16: return f(adjoint_kernel<8, 0, false, GS, MODEL, false, 2>, cp[2]);
        case 17: return f(adjoint_kernel<8, 1, false, GS, MODEL, false, 2>, cp[3]);
        default: break;
        }
        return cudaErrorInvalidValue;
    }
    if (ppl != 1) return cudaErrorInvalidValue;
    if (method == kMethodVanna) {     // second-order buckets: main reading, binary64 level 2
        if constexpr (MODEL == 0) {
            static bool cv = false;
            if (!greeks || dbg || extra || acc != 0) return cudaErrorInvalidValue;
            return f(vanna_kernel<GS>, cv);
        }
        return cudaErrorInvalidValue;
    }
    if (extra) {           // d V / d r and d V / d T: reverse sweep, binary64 level 2, k = 4 or 8
        static bool ce[2] = {};
        if (!greeks || dbg || method != LV_ADJ_REVERSE || acc != 0) return cudaErrorInvalidValue;
        if (k == 4) return f(adjoint_kernel<4, 0, false, GS, MODEL, true>, ce[0]);
        if (k == 8) return f(adjoint_kernel<8, 0, false, GS, MODEL, true>, ce[1]);
        return cudaErrorInvalidValue;
    }
    if (!greeks) {
        static bool c0 = false, c1 = false;
        return acc ? f(price_kernel<1, GS, MODEL>, c1) : f(price_kernel<0, GS, MODEL>, c0);
    }
    if (method == LV_ADJ_TANGENT && !dbg) {
        static bool t0 = false, t1 = false;
        return acc ? f(tangent_kernel<1, GS, MODEL>, t1) : f(tangent_kernel<0, GS, MODEL>, t0);
    }
    if (dbg) {
        static bool cd = false;
        if (k != 4) return cudaErrorInvalidValue;       // scratch must be planned with k = 4
        return f(adjoint_kernel<4, 0, true, GS, MODEL>, cd);
    }
    static bool c[8] = {};
    switch (k * 2 + acc) {
    case 8: return f(adjoint_kernel<4, 0, false, GS, MODEL>, c[0]);
    case 9: return f(adjoint_kernel<4, 1, false, GS, MODEL>, c[1]);
    case 16: return f(adjoint_kernel<8, 0, false, GS, MODEL>, c[2]);
    case 17: return f(adjoint_kernel<8, 1, false, GS, MODEL>, c[3]);
    default: break;
    }
    if constexpr (MODEL == 0) {
        switch (k * 2 + acc) {
        case 32: return f(adjoint_kernel<16, 0, false, GS, 0>, c[4]);
        case 33: return f(adjoint_kernel<16, 1, false, GS, 0>, c[5]);
        case 64: return f(adjoint_kernel<32, 0, false, GS, 0>, c[6]);
        case 65: return f(adjoint_kernel<32, 1, false, GS, 0>, c[7]);
        default: break;
        }
    }
    return cudaErrorInvalidValue;
}

template <int MODEL>
cudaError_t launch_model_impl(const McParams& p, int grid, int block, int k, bool greeks, size_t smem,
                              cudaStream_t s)
{
    auto run = [&](auto kernel, bool& configured) {
        return launch_configured(kernel, configured, p, grid, block, smem, s);
    };
    const bool dbg = p.dbg_xN != nullptr;
    const int ppl = p.ppl > 1 ? p.ppl : 1;
    return p.grid_smem ? with_kernel_gs<MODEL, true>(greeks, k, p.acc_mode, dbg, p.method, p.extra != 0, run, ppl)
                       : with_kernel_gs<MODEL, false>(greeks, k, p.acc_mode, dbg, p.method, p.extra != 0, run, ppl);
}

template <int MODEL>
cudaError_t occupancy_model_impl(int block, int k, bool greeks, int acc, bool dbg, bool gs, int method, bool extra,
                                 size_t smem, int* bps, int ppl = 1)
{
    auto occ = [&](auto kernel, bool&) { return occupancy(kernel, block, smem, bps); };
    return gs ? with_kernel_gs<MODEL, true>(greeks, k, acc, dbg, method, extra, occ, ppl)
              : with_kernel_gs<MODEL, false>(greeks, k, acc, dbg, method, extra, occ, ppl);
}

}  // namespace

}  // namespace lv
