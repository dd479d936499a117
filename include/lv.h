/*
 * lv.h -- C ABI of the GB300 (sm_103a) local-volatility Monte Carlo library.
 *
 * The library prices a European option under Dupire's local-volatility
 * model, dX/X = sigma(X, t) dW (arXiv 2002.02481, Sec. IV-A), with sigma
 * given on a spot x time grid and interpolated bilinearly (Sec. IV-D), by
 * Monte Carlo over explicit Euler paths of the log-spot, and returns the
 * price together with its pathwise adjoint (back-propagation, Sec. III and
 * IV-C): the delta d price / d S0 and one vega bucket d price / d sigma_ij
 * per grid node. Central bump-and-reprice (Sec. III) is provided as the
 * baseline the adjoint is measured against.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an lv_status and never aborts; on failure the
 *    outputs are left untouched and lv_last_error() describes the cause.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership of everything it passes.
 *  - A handle must not be used from two host threads at the same time.
 *    Work runs on the handle's CUDA stream (lv_set_stream; default: the
 *    legacy default stream). Entry points with host outputs synchronise that
 *    stream before returning; the *_device variants only enqueue work.
 *  - Arithmetic: paths in binary32; per-block accumulation of payoffs and
 *    vega buckets in binary64 (or Kahan-compensated binary32, see
 *    lv_set_accumulation); cross-block reduction in binary64, fixed order.
 *  - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *    key (seed & 0xffffffff, seed >> 32) and counter
 *    (step / 4, path & 0xffffffff, ((path >> 32) & 0xffff) | stream_id << 16, 0).
 *    Word w gives the uniform u = ((w >> 9) + 0.5) * 2^-23 in (0, 1); words
 *    (0, 1) and (2, 3) give two normals each by Box-Muller,
 *    Z_a = sqrt(-2 ln u_a) cos(2 pi u_b), Z_b = sqrt(-2 ln u_a) sin(2 pi u_b);
 *    step n uses normal n mod 4 of block n / 4. Results therefore depend only
 *    on (seed, stream_id, path index), not on the launch configuration, up
 *    to the rounding order of the reductions.
 *  - Model: x = ln S, x_{n+1} = x_n + (r - sigma_n^2 / 2) dt + sigma_n sqrt(dt) Z_n
 *    with dt = T / n_steps and sigma_n = sigma(S_n, t_n), t_n = n dt (left
 *    point). Payoff e^{-rT} max(phi (S_N - K), 0), phi = +1 call, -1 put.
 *    Interpolation is bilinear in S and t: cell i is the largest i <= I-2
 *    with s_i <= S (0 below the grid), weight u = (S - s_i) / (s_{i+1} - s_i)
 *    clamped to [0, 1]; the same in time. sigma is flat outside the grid,
 *    and there d sigma / d S = 0. With n_time == 1 sigma does not depend on t.
 *    The payoff indicator is 1{phi (S_N - K) > 0}: a tie contributes 0.
 *  - Vega is d price / d sigma_ij per unit of sigma, stored spot-major at
 *    index i * n_time + j, the same layout as the sigma input.
 */
#ifndef LV_H
#define LV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lv_surface_s* lv_surface_t;
typedef struct lv_book_s* lv_book_t;

typedef enum {
    LV_OK = 0,
    LV_EINVAL = 1,      /* an argument is out of its documented domain */
    LV_ENOMEM = 2,      /* a host or device allocation failed */
    LV_ECUDA = 3,       /* a CUDA runtime call failed (message in lv_last_error) */
    LV_EINTERNAL = 4,   /* a consistency check inside the library failed */
    LV_ENUMERIC = 5     /* the tangent-ratio adjoint met a vanishing factor 1 + g_n (see
                           lv_set_adjoint_method); host outputs are left untouched, device
                           outputs of the call are NaN */
} lv_status;

/* Level-2 (per-block, across path tiles) accumulation of the payoffs and of
 * every vega bucket. */
enum { LV_ACC_FP64 = 0, LV_ACC_KAHAN = 1 };

/* How the pathwise adjoint (Sec. III, IV-C) is evaluated; both give the same
 * derivatives up to rounding.
 *  - LV_ADJ_REVERSE (default): back-propagation through the Euler scheme,
 *    x_bar_n = x_bar_{n+1} (1 + g_n), on checkpoints every k steps.
 *  - LV_ADJ_TANGENT: the recursion is linear, so x_bar_{n+1} =
 *    x_bar_N D_N / D_{n+1} with D_0 = 1, D_{n+1} = D_n (1 + g_n) (the tangent
 *    process d x_n / d x_0). A first forward pass gives D_N per path, hence
 *    x_bar_0 = x_bar_N D_N; a second forward pass over the paths with
 *    x_bar_N != 0 spreads sigma_bar_n = x_bar_N D_N h_n / D_{n+1}. No
 *    checkpoints, no reverse order. When some |1 + g_n| falls below 2^-20 the
 *    ratio loses what the reverse sweep keeps: every device output of the
 *    call is then NaN, and the host-output entry points return LV_ENUMERIC
 *    without writing their outputs.
 * g_n = h_n S_n d sigma / d S and h_n = sqrt(dt) Z_n - sigma_n dt. */
enum { LV_ADJ_REVERSE = 0, LV_ADJ_TANGENT = 1 };

/* The two readings of the scheme besides the main one (Sec. IV-A, IV-D):
 *  - spot weight of the bilinear interpolation linear in S (LV_INTERP_S,
 *    default) or in ln S (LV_INTERP_LOGS: u = (ln S - ln s_i) /
 *    (ln s_{i+1} - ln s_i), clamped);
 *  - Euler scheme on x = ln S (LV_SCHEME_LOG, default: drift r - sigma^2/2)
 *    or on S itself (LV_SCHEME_S: S_{n+1} = S_n (1 + r dt + sigma_n sqrt(dt)
 *    Z_n); a spot at or below 0 is below the grid).
 * The delta is d price / d S0 and the vegas d price / d sigma_ij under every
 * reading. The other readings run checkpoint intervals k = 4 and 8 (larger k
 * are capped at 8); the book and the bump baseline run the main reading. */
enum { LV_INTERP_S = 0, LV_INTERP_LOGS = 1 };
enum { LV_SCHEME_LOG = 0, LV_SCHEME_S = 1 };

/* Layout of the [3 + n_spot * n_time] result of lv_price_greeks_device. */
enum { LV_OUT_PRICE = 0, LV_OUT_DELTA = 1, LV_OUT_STDERR = 2, LV_OUT_VEGA = 3 };

/* Layout of the [3 + n_spot * n_time] raw sums of lv_price_greeks_sums_device:
 * sum of payoffs, sum of squared payoffs, sum of d V / d x_0 (x_0 = ln S0),
 * then the sum over paths of every sigma adjoint (spot-major). Sums from
 * disjoint path ranges add up to the sums of their union. */
enum { LV_SUM_V = 0, LV_SUM_V2 = 1, LV_SUM_XBAR0 = 2, LV_SUM_VEGA = 3 };

/* Largest supported sizes (shared memory holds the grid, the bucket
 * accumulators and the per-step time table). */
#define LV_MAX_STEPS 8192
#define LV_MAX_NODES 16384
#define LV_MAX_PATH_INDEX (((int64_t)1) << 48)

/* lv_surface_create -- stage a local-vol grid on the current CUDA device.
 *   Grid {(s_i, tau_j)} of Sec. IV-A with values sigma_ij.
 *   spot_nodes [n_spot]  strictly increasing, > 0, n_spot >= 2
 *   time_nodes [n_time]  strictly increasing, >= 0, n_time >= 1
 *   sigma [n_spot*n_time] sigma_ij at index i * n_time + j, finite, > 0
 *   n_spot * n_time <= LV_MAX_NODES
 *   out                  receives the handle (owned by the caller; release
 *                        with lv_surface_destroy)
 * The arrays are copied (to binary32 device copies) before return. */
lv_status lv_surface_create(const double* spot_nodes, int32_t n_spot,
                            const double* time_nodes, int32_t n_time,
                            const double* sigma, lv_surface_t* out);

/* Release a handle and its device memory (NULL is ignored). */
void lv_surface_destroy(lv_surface_t h);

/* Replace the grid values (same layout and domain as in lv_surface_create);
 * the host-to-device copy is enqueued on the handle's stream. */
lv_status lv_surface_set_sigma(lv_surface_t h, const double* sigma);

/* +1 call (default), -1 put. */
lv_status lv_set_option_type(lv_surface_t h, int32_t phi);

/* CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * that later calls enqueue on; NULL selects the legacy default stream. A
 * change of stream first waits for the work already enqueued on the old one
 * (the handle's scratch and staging buffers are shared by its calls). */
lv_status lv_set_stream(lv_surface_t h, void* cuda_stream);

/* LV_ACC_FP64 (default) or LV_ACC_KAHAN. */
lv_status lv_set_accumulation(lv_surface_t h, int32_t mode);

/* LV_ADJ_REVERSE (default) or LV_ADJ_TANGENT, for every greeks entry point
 * of the handle except lv_debug_paths (always the reverse sweep). */
lv_status lv_set_adjoint_method(lv_surface_t h, int32_t method);

/* LV_INTERP_S (default) or LV_INTERP_LOGS for later calls on the handle. */
lv_status lv_surface_set_interpolation(lv_surface_t h, int32_t interp);

/* LV_SCHEME_LOG (default) or LV_SCHEME_S for later calls on the handle. */
lv_status lv_set_scheme(lv_surface_t h, int32_t scheme);

/* Launch shape: threads per block (32..128, multiple of 32), checkpoint
 * interval k of the reverse sweep (4, 8, 16 or 32 steps) and resident
 * blocks per SM; 0 keeps the tuned or default value. Results do not depend
 * on it beyond reduction-order rounding. */
lv_status lv_set_launch(lv_surface_t h, int32_t block, int32_t k, int32_t blocks_per_sm);

/* Paths per lane of the adjoint's forward tiles: 1, or 2 (each lane runs two
 * paths interleaved: two independent dependency chains per thread, the
 * per-step grid data loaded once for both, and on the main reading their
 * binary32 arithmetic in packed pairs where that keeps the occupancy); 0 keeps
 * the tuned value, or the default: 2 for calls of at least 6,144 paths per SM
 * (933,888 on 152 SMs), where every warp still gets four pairs of tiles, else 1.
 * Two paths per lane exist for the reverse sweep with checkpoints every 4
 * or 8 steps (every reading of the scheme), the main reading's tangent-ratio
 * adjoint and its second-order buckets; elsewhere the call runs one. The results do not
 * depend on it beyond reduction-order rounding.
 * lv_get_paths_per_lane reads back the value the next call with n_steps steps
 * and n_paths >= 1 paths will use. */
lv_status lv_set_paths_per_lane(lv_surface_t h, int32_t ppl);
lv_status lv_get_paths_per_lane(lv_surface_t h, int32_t n_steps, int64_t n_paths, int32_t* ppl);

/* Record two caller-owned CUDA events (cudaEvent_t, created with timing
 * enabled) on the handle's stream immediately before and after the Monte
 * Carlo kernel of every later call, so that a caller can time that kernel
 * alone; NULL, NULL switches this off. */
lv_status lv_set_kernel_events(lv_surface_t h, void* start_event, void* end_event);

/* Autotuner for one option: times lv_price_greeks_device on this problem
 * over launch shapes (threads per block 64 / 128, checkpoint interval 4 / 8
 * / 16, and for the main reading's reverse sweep at k = 4 and 8 one or two
 * paths per lane), keeps the fastest in the handle (as lv_set_launch and
 * lv_set_paths_per_lane would) and appends it (block, k, paths per lane) to
 * the file named by LV_TUNE_CACHE when that variable is set; later handles
 * with the same grid size and step count then start from it. Runs the
 * problem about 40 times. Outputs may be NULL. */
lv_status lv_tune(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps, int64_t n_paths,
                  uint64_t seed, int32_t* out_block, int32_t* out_k, double* out_ms);

/* Read back the launch shape the next call will use for (n_steps, greeks);
 * blocks_per_sm is that of a call large enough for two paths per lane by
 * default (lv_get_paths_per_lane). */
lv_status lv_get_launch(lv_surface_t h, int32_t n_steps, int32_t greeks,
                        int32_t* block, int32_t* k, int32_t* blocks_per_sm);

/* lv_price -- Monte Carlo price of the option over paths [0, n_paths)
 * (Sec. IV-C: the mean of the discounted payoff).
 *   S0 > 0, r finite, K >= 0, T > 0, 1 <= n_steps <= LV_MAX_STEPS,
 *   1 <= n_paths < 2^31 per call (path indices below LV_MAX_PATH_INDEX).
 *   out_price   host, 1 double
 *   out_stderr  host, 1 double or NULL: standard error of the price */
lv_status lv_price(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                   int64_t n_paths, uint64_t seed, double* out_price, double* out_stderr);

/* lv_price_greeks -- price, delta and every vega bucket by the pathwise
 * adjoint (back-propagation through the Euler scheme, Sec. III / IV-C),
 * from one forward pass and one checkpointed reverse sweep per path.
 *   out_price  host, 1 double
 *   out_delta  host, 1 double
 *   out_vega   host, [n_spot * n_time] doubles, spot-major */
lv_status lv_price_greeks(lv_surface_t h, double S0, double r, double K, double T,
                          int32_t n_steps, int64_t n_paths, uint64_t seed,
                          double* out_price, double* out_delta, double* out_vega);

/* Device-output variant: writes [3 + n_spot * n_time] doubles (layout
 * LV_OUT_*) to d_out (device memory owned by the caller) on the handle's
 * stream, without synchronising. */
lv_status lv_price_greeks_device(lv_surface_t h, double S0, double r, double K, double T,
                                 int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out);

/* Price, delta and vegas (as lv_price_greeks) plus rho = d price / d r and
 * d price / d T, the maturity sensitivity with n_steps fixed (dt = T / N,
 * t_n = n T / N) and the grid fixed in time (Sec. III's pathwise adjoint
 * applied to the two scalar inputs: the derivative of the discount plus
 * sum_n xbar_{n+1} d x_{n+1} / d r (or d T), accumulated in the same reverse
 * sweep). Runs the checkpointed reverse sweep with binary64 level 2 and
 * k = 4 or 8, whatever the handle's adjoint method, accumulation and k say.
 * Host outputs like lv_price_greeks, then out_rho and out_dVdT. */
lv_status lv_price_greeks_ext(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                              int64_t n_paths, uint64_t seed, double* out_price, double* out_delta,
                              double* out_vega, double* out_rho, double* out_dVdT);

/* Same, to d_out (device, caller-owned) laid out [5 + n_spot * n_time]:
 * LV_OUT_PRICE, LV_OUT_DELTA, LV_OUT_STDERR, the vegas from LV_OUT_VEGA,
 * then rho at 3 + n_spot * n_time and d price / d T at 4 + n_spot * n_time;
 * enqueued on the handle's stream without synchronising. */
lv_status lv_price_greeks_ext_device(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                                     int64_t n_paths, uint64_t seed, double* d_out);

/* Raw sums over paths [path_begin, path_end) with a given stream_id
 * (< 65536): [3 + n_spot * n_time] doubles, layout LV_SUM_*, written to
 * device memory d_sums owned by the caller, without synchronising. This is
 * the unit of path-range sharding: sums of disjoint ranges add up. */
lv_status lv_price_greeks_sums_device(lv_surface_t h, double S0, double r, double K, double T,
                                      int32_t n_steps, int64_t path_begin, int64_t path_end,
                                      uint64_t seed, uint32_t stream_id, double* d_sums);

/* Turn raw sums (layout LV_SUM_*, e.g. the element-wise sum of the
 * lv_price_greeks_sums_device results of disjoint path ranges, one per GPU)
 * over n_paths paths into [3 + n_spot * n_time] doubles of layout LV_OUT_*
 * (Sec. IV-C: means over paths; delta = mean d V / d x_0 / S0). d_sums and
 * d_out are device memory owned by the caller; enqueued on the handle's
 * stream without synchronising. */
lv_status lv_finalize_sums_device(lv_surface_t h, const double* d_sums, int64_t n_paths, double S0,
                                  double* d_out);

/* lv_bump_greeks -- central bump-and-reprice (Sec. III), the baseline the
 * adjoint is measured against: every grid value sigma_ij +/- eps/2 and
 * S0 +/- eps_S/2 with eps_S = 1e-4 * S0, each pair of scenarios on the same
 * random numbers (common random numbers), the price difference divided by
 * the bump. One batched launch over the 3 + 2 * n_spot * n_time scenarios.
 * Outputs as in lv_price_greeks (the price is that of the unbumped model).
 *   eps > 0, finite. */
lv_status lv_bump_greeks(lv_surface_t h, double S0, double r, double K, double T,
                         int32_t n_steps, int64_t n_paths, uint64_t seed, double eps,
                         double* out_price, double* out_delta, double* out_vega);

/* lv_price_greeks_vanna -- second-order bucket sensitivities
 * d^2 price / (d S0 d sigma_ij) ("vanna" buckets), an extension of Sec. V's
 * first-order Greeks: out_price and out_delta as in lv_price_greeks, and
 * out_vanna [n_spot * n_time] (spot-major, caller-owned host memory). The
 * pathwise delta Delta_p = e^{-rT} 1{phi (S_N - K) > 0} phi S_N D_N / S0
 * jumps where S_N crosses the strike and where a spot crosses a node, so
 * its own pathwise derivative would be biased; with the path held fixed
 * nothing jumps, and the estimator is the derivative of Delta_p at the
 * fixed path plus Delta_p times the derivative of the path's log density
 * (each Euler step Gaussian): per path and step n it adds
 *   Delta_p [ w_ij(n) a_n + S_n d w_ij / d S (n) b_n ],
 *   a_n = (Z_n^2 - 1) / sigma_n - sqrt(dt) Z_n (1 + k_n / (sigma_n (1 + g_n))),
 *   b_n = h_n / (1 + g_n),
 * k_n = S_n d sigma / d S, g_n = h_n k_n, w_ij the bilinear weights. Two
 * forward passes (no checkpoints), binary32 paths, binary64 level 2. Main
 * reading only (else LV_EINVAL); a live path with |1 + g_n| < 2^-20 gives
 * LV_ENUMERIC (host outputs untouched) or NaN device outputs.
 * lv_price_greeks_vanna_device: the same [3 + I J] (LV_OUT_* layout, the
 * buckets in place of the vegas) into device memory, not synchronised. */
lv_status lv_price_greeks_vanna(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                                int64_t n_paths, uint64_t seed, double* out_price, double* out_delta,
                                double* out_vanna);
lv_status lv_price_greeks_vanna_device(lv_surface_t h, double S0, double r, double K, double T,
                                       int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out);

/* Measured issue rates of the SM pipes the Monte Carlo path is bound by
 * (it reads almost nothing from memory: its roofline is arithmetic, not
 * HBM), the denominators of its roofline fractions. lv_measure_pipe_peaks
 * runs one probe kernel per entry on the current device (eight chains of
 * that instruction per thread, integer chains fed by their neighbours so
 * that none collapses, 8 blocks of 256 threads per SM, best of three runs
 * timed with CUDA events) and writes
 * out_ops_per_s[LV_PIPE_COUNT]: thread-instructions per second over the
 * whole GPU at the clock the probes ran at. Synchronous; about 50 ms. */
enum {
    LV_PIPE_FFMA = 0,       /* fma.rn.f32 */
    LV_PIPE_MUFU_EX2 = 1,   /* ex2.approx.ftz.f32 */
    LV_PIPE_MUFU_LG2 = 2,   /* lg2.approx.ftz.f32 */
    LV_PIPE_MUFU_SIN = 3,   /* sin.approx.ftz.f32 */
    LV_PIPE_MUFU_COS = 4,   /* cos.approx.ftz.f32 */
    LV_PIPE_MUFU_SQRT = 5,  /* sqrt.approx.ftz.f32 */
    LV_PIPE_IMAD = 6,       /* mad.lo.u32 */
    LV_PIPE_IMAD_WIDE = 7,  /* mad.wide.u32 (the Philox product) */
    LV_PIPE_LOP3 = 8,       /* lop3.b32 */
    LV_PIPE_COUNT = 9
};
lv_status lv_measure_pipe_peaks(double* out_ops_per_s);

/* lv_price_greeks_fp64_device -- the same outputs as lv_price_greeks_device
 * (layout LV_OUT_*, device memory owned by the caller, on the handle's
 * stream, not synchronised) with every path in binary64: the full-FP64
 * reference against which the binary32 path's rounding is measured on the
 * GPU (the precision study of Sec. IV-C's mixed-precision reading). Same
 * random numbers (the uniforms are exact in binary64), the same model and
 * decisions as the FP64 definition, the adjoint in its tangent-ratio form
 * (see LV_ADJ_TANGENT) with binary64 sums; CUDA's binary64 exp, log, sqrt
 * and sincospi. Binary64 arithmetic runs at a small fraction of the binary32
 * rate on this part: a reference, not a fast path. Main reading only
 * (LV_INTERP_S, LV_SCHEME_LOG; else LV_EINVAL); ignores lv_set_launch,
 * lv_set_accumulation and lv_set_adjoint_method. A live path with
 * |1 + g_n| < 2^-40 makes every output NaN, as in LV_ADJ_TANGENT.
 * n_paths in [1, 2^48). */
lv_status lv_price_greeks_fp64_device(lv_surface_t h, double S0, double r, double K, double T,
                                      int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out);

/* lv_bump_greeks_fp64 -- lv_bump_greeks (Sec. III: central differences,
 * sigma_ij +- eps/2 and S0 +- eps_S/2, common random numbers) with every
 * bumped path in binary64, so that the differences carry no binary32
 * rounding noise: the bump baseline at the accuracy of the adjoint. The
 * spot bump scales with eps here, eps_S = eps S0 (binary64 differences
 * allow bumps far below the binary32 baseline's fixed 1e-4 S0). Outputs as in lv_bump_greeks (host memory, synchronous).
 * Main reading only (else LV_EINVAL); eps > 0, finite; n_paths in
 * [1, 2^48). */
lv_status lv_bump_greeks_fp64(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                              int64_t n_paths, uint64_t seed, double eps, double* out_price, double* out_delta,
                              double* out_vega);

/* Per-path diagnostics for paths [path_begin, path_begin + m), m <= 2^26,
 * of RNG stream stream_id (< 65536, as in lv_price_greeks_sums_device):
 * terminal log-spot x_N, discounted payoff V and d V / d x_0, each [m]
 * binary32 in host memory owned by the caller (any may be NULL). The values
 * of a path do not depend on the launch shape. Also logs every forward step
 * whose spot S lies within node_band * s of one of its cell's nodes s:
 * out_ev [ev_cap][3] int32 receives (path - path_begin, step, 2 i + inside)
 * with i the spot cell taken and inside = 1 when S lay in [s_0, s_{I-1}]
 * (which switches d sigma / d S on); *out_n_ev the number of such steps
 * (entries beyond ev_cap are counted but not stored; order unspecified).
 * These are the integer decisions a binary64 reimplementation may take
 * differently when S sits within rounding of a node (Sec. IV-D's cell of
 * the bilinear interpolation). */
lv_status lv_debug_paths(lv_surface_t h, double S0, double r, double K, double T,
                         int32_t n_steps, uint64_t seed, uint32_t stream_id, int64_t path_begin, int64_t m,
                         float* out_xN, float* out_V, float* out_xbar0,
                         double node_band, int64_t ev_cap, int32_t* out_ev, int64_t* out_n_ev);

/* The kernels' random numbers (Sec. IV-B, read as Philox4x32-10 with the
 * key, counter and transform given at the top of this file), for tests: for entry e
 * of n (n in [1, 2^24]), the Philox block blocks[e] of path paths[e]
 * (< 2^48) of stream stream_id (< 65536) under key seed. out_words [n][4]
 * receives the four 32-bit words, out_z [n][4] the four binary32 normals
 * the kernels derive from them (Box-Muller on word pairs (0,1), (2,3)).
 * Host arrays owned by the caller; synchronous; no handle needed. */
lv_status lv_debug_normals(uint64_t seed, uint32_t stream_id, const int64_t* paths, const uint32_t* blocks,
                           int64_t n, uint32_t* out_words, float* out_z);

/* The kernels' time table of a call with maturity T and n_steps steps on
 * the handle's grid (Sec. IV-A: sigma at the left point t_n = n T / N;
 * Sec. IV-D: the time cell), for tests: out_j [n_steps] receives the time
 * cell j_n = the largest j <= J-2 with tau_j <= t_n (0 for one time node),
 * out_v [n_steps] the clamped weight (t_n - tau_j) / (tau_{j+1} - tau_j)
 * rounded to binary32 as the kernels use it. Both decided in binary64.
 * Host arrays owned by the caller; synchronous (on the handle's stream). */
lv_status lv_debug_time_table(lv_surface_t h, double T, int32_t n_steps, int32_t* out_j, float* out_v);

/* lv_price_greeks_device_noalloc -- lv_price_greeks_device for callers that
 * cannot allocate device memory during the call: loops with a no-allocation
 * rule, or runtimes that own every device allocation. The paper has no counterpart; it is a
 * deployment variant of the same computation with the same results (up to
 * reduction order) and the same output layout (LV_OUT_*), written to d_out
 * (device memory owned by the caller) on the handle's stream, without
 * synchronising.
 *  - It calls no allocator: its scratch is a static 64 MiB device array that
 *    every GPU loading this library keeps until the process exits. When a
 *    launch at full width does not fit, it runs one path per lane (unless
 *    lv_set_paths_per_lane or the tuner chose two) and then, if still
 *    needed, fewer blocks; a problem whose
 *    single block does not fit (very large n_spot * n_time with many steps)
 *    is rejected with LV_EINVAL and a message giving the bytes needed.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - Every call on a device uses the same array, and the array keeps the
 *    previous call's contents (the call clears what must start at zero):
 *    calls that may overlap on the GPU race and give wrong results. Serialise
 *    them, e.g. on one stream.
 *  - n_paths in [1, 2^31 - 1]; other arguments as in lv_price_greeks. */
lv_status lv_price_greeks_device_noalloc(lv_surface_t h, double S0, double r, double K, double T,
                                         int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out);

/* ---------------------------------------------------------------- book
 * A book of European options on several local-vol grids, priced with all
 * their deltas and vega buckets in one persistent launch (the Monte Carlo
 * of Sec. IV-C over many instruments). Option o uses Philox stream
 * stream_id (< 65536) and paths [0, n_paths): its results equal those of
 * lv_price_greeks_sums_device(surface, S0, r, K, T, n_steps, 0, n_paths,
 * seed, stream_id) finalized, up to reduction order. */
typedef struct {
    int32_t surface;     /* index into the surfaces given to lv_book_create */
    int32_t phi;         /* +1 call, -1 put */
    double K;            /* >= 0 */
    double T;            /* > 0 */
    int32_t n_steps;     /* 1 .. LV_MAX_STEPS */
    int64_t n_paths;     /* 1 .. 2^31 - 1 */
    uint32_t stream_id;  /* < 65536 */
} lv_instrument;

/* Build a book of 1 .. 65535 options: the grids of `surfaces` (all on the current device) are
 * copied, so the surfaces may be destroyed afterwards; `insts` is copied.
 * Outputs of lv_book_run are laid out per option, in the given order, as
 * [3 + n_spot * n_time] doubles (LV_OUT_*); lv_book_output_offsets gives
 * the first index of each. A tuned launch shape is read from the file named
 * by the environment variable LV_TUNE_CACHE when it holds one for this GPU
 * and book shape. */
lv_status lv_book_create(const lv_surface_t* surfaces, int32_t n_surfaces, const lv_instrument* insts,
                         int32_t n_insts, lv_book_t* out);
void lv_book_destroy(lv_book_t b);

/* offsets [n_insts + 1]: option o's results occupy [offsets[o], offsets[o+1]). */
lv_status lv_book_output_offsets(lv_book_t b, int64_t* offsets);

/* Stream for later runs (NULL: a stream the book creates; the legacy
 * default stream cannot be captured into a graph). */
lv_status lv_book_set_stream(lv_book_t b, void* cuda_stream);

/* Run the book for (S0, r, seed): host output [offsets[n_insts]] doubles.
 * The first run captures the whole run (parameter upload, zeroing, the
 * persistent kernel, the finalize and the copy back) into a CUDA graph;
 * later runs replay it. Synchronises the book's stream. */
lv_status lv_book_run(lv_book_t b, double S0, double r, uint64_t seed, double* out);

/* Same without graph or host copy: results to d_out (device, caller-owned),
 * enqueued on the book's stream without synchronising. */
lv_status lv_book_run_device(lv_book_t b, double S0, double r, uint64_t seed, double* d_out);

/* Autotuner: times the book over launch shapes (threads per block 64 / 128,
 * checkpoint interval 4 / 8, paths per work item 2K / 8K / 32K, one or two
 * paths per lane of the forward tiles), keeps the fastest, and appends it
 * to the LV_TUNE_CACHE file when that variable is set (a new book of the
 * same shape starts from it). Outputs the chosen shape and its time in
 * milliseconds (any pointer may be NULL); lv_book_paths_per_lane reads the
 * paths per lane in use. */
lv_status lv_book_tune(lv_book_t b, double S0, double r, uint64_t seed, int32_t* out_block, int32_t* out_k,
                       int32_t* out_item_paths, double* out_ms);
lv_status lv_book_paths_per_lane(lv_book_t b, int32_t* ppl);

/* Sets the book's launch shape explicitly (as the tuner would): threads per
 * block (multiple of 32 in [32, 128]), checkpoint interval k (4 or 8),
 * paths per work item (a multiple of 32), paths per lane (1 or 2). Drops a
 * captured graph; the next lv_book_run captures again. */
lv_status lv_book_set_launch(lv_book_t b, int32_t block, int32_t k, int32_t item_paths, int32_t ppl);

/* Book-level aggregated risk (the portfolio view of the first-order risk of
 * Sec. I and V: one set of vega buckets per surface instead of one per
 * option). With position weights w_o (lv_book_set_weights; 1 by default),
 * per surface s over its options o:
 *   [0] sum_o w_o price_o, [1] sum_o w_o delta_o,
 *   [2] sqrt(sum_o w_o^2 stderr_o^2)  (options on distinct Philox streams are
 *       independent; options sharing a stream and surface are not, and this
 *       figure then understates the error),
 *   [3 + i * n_time + j] sum_o w_o vega_o[i][j].
 * The persistent kernel adds each work item's vega buckets, scaled by
 * w_o / n_paths_o, into its surface's binary64 sums; no per-option vega is
 * written. Weights: [n_insts] finite doubles, copied; later runs use them. */
lv_status lv_book_set_weights(lv_book_t b, const double* weights);

/* offsets [n_surfaces + 1]: surface s's risk occupies [offsets[s], offsets[s+1]). */
lv_status lv_book_risk_offsets(lv_book_t b, int64_t* offsets);

/* Run the book and return the aggregated risk: host output
 * [offsets[n_surfaces]] doubles (graph-captured like lv_book_run). */
lv_status lv_book_run_risk(lv_book_t b, double S0, double r, uint64_t seed, double* out);

/* Same without graph or host copy, to d_out (device, caller-owned),
 * enqueued on the book's stream without synchronising. */
lv_status lv_book_run_risk_device(lv_book_t b, double S0, double r, uint64_t seed, double* d_out);

/* Thread-local description of the last failure on this host thread. */
const char* lv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LV_H */
