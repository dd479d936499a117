// lv_device.cuh -- device building blocks: counter-based normals, the
// bilinear local-vol lookup and one log-Euler step (arXiv 2002.02481,
// Sec. IV-A, IV-B, IV-D).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lv_internal.h"

namespace lv {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products and xors with a Weyl-sequence key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// u = ((w >> 9) + 1/2) 2^-23 = (2m + 1) 2^-24, m < 2^23: the mantissa trick
// gives 1 + m 2^-23 in [1, 2), and subtracting 1 - 2^-24 is exact.
__device__ __forceinline__ float uniform_open01(uint32_t w)
{
    return __uint_as_float((w >> 9) | 0x3f800000u) - __uint_as_float(0x3f7fffffu);
}

__device__ __forceinline__ float sqrt_approx(float a)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ float ex2_approx(float a)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ float lg2_approx(float a)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Four standard normals for Philox block `blk` of a path. Box-Muller on
// word pairs (0,1) and (2,3): Z_a = rho cos(2 pi u_b), Z_b = rho sin(2 pi u_b),
// rho = sqrt(-2 ln u_a). The angle is evaluated as 2 pi (u_b - 1/2) (exact
// shift, keeps the hardware sine/cosine inside [-pi, pi)), which flips the
// sign of both: cos(a + pi) = -cos a, sin(a + pi) = -sin a.
__device__ __forceinline__ void normals4(uint32_t blk, uint32_t c1, uint32_t c2, uint32_t k0,
                                         uint32_t k1, float z[4])
{
    uint32_t w0 = blk, w1 = c1, w2 = c2, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, k0, k1);
    const float m2ln2 = -1.3862943611198906f;   // -2 ln 2
    const float two_pi = 6.2831853071795865f;
    {
        const float rho = sqrt_approx(m2ln2 * lg2_approx(uniform_open01(w0)));
        float s, c;
        __sincosf(two_pi * (uniform_open01(w1) - 0.5f), &s, &c);
        z[0] = -rho * c;
        z[1] = -rho * s;
    }
    {
        const float rho = sqrt_approx(m2ln2 * lg2_approx(uniform_open01(w2)));
        float s, c;
        __sincosf(two_pi * (uniform_open01(w3) - 0.5f), &s, &c);
        z[2] = -rho * c;
        z[3] = -rho * s;
    }
}

// Packed binary32 pairs (add/sub/mul/fma .f32x2, sm_100 and later): one
// instruction rounds each element exactly as the scalar instruction would, so
// two independent paths advanced through them get bit-identical results with
// half the issue slots for that arithmetic. The operands are register pairs;
// constants cannot come from the parameter bank as in scalar code, so each
// constant pair costs two registers.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float lo2(f32x2 r)
{
    float a;
    asm("mov.b64 {%0, _}, %1;" : "=f"(a) : "l"(r));
    return a;
}

__device__ __forceinline__ float hi2(f32x2 r)
{
    float b;
    asm("mov.b64 {_, %0}, %1;" : "=f"(b) : "l"(r));
    return b;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The normals of normals4 for two paths at once, as pairs (path a, path b),
// NEGATED: nz[q] = (-Z_q of a, -Z_q of b), i.e. rho cos / rho sin of the
// shifted angle without normals4's sign flip. Every element is rounded as in
// normals4 (a negation is exact), so -nz[q] is normals4's z[q] bit for bit.
__device__ __forceinline__ void normals4x2_neg(uint32_t blk, uint32_t c1a, uint32_t c2a, uint32_t c1b, uint32_t c2b,
                                               uint32_t k0, uint32_t k1, f32x2 nz[4])
{
    uint32_t a0 = blk, a1 = c1a, a2 = c2a, a3 = 0u;
    uint32_t b0 = blk, b1 = c1b, b2 = c2b, b3 = 0u;
    philox4x32_10(a0, a1, a2, a3, k0, k1);
    philox4x32_10(b0, b1, b2, b3, k0, k1);
    const f32x2 one_m = pk2(__uint_as_float(0x3f7fffffu), __uint_as_float(0x3f7fffffu));
    const f32x2 half = pk2(0.5f, 0.5f);
    const f32x2 m2ln2 = pk2(-1.3862943611198906f, -1.3862943611198906f);
    const f32x2 two_pi = pk2(6.2831853071795865f, 6.2831853071795865f);
#define LV_U2(x, y) sub2(pk2(__uint_as_float(((x) >> 9) | 0x3f800000u), __uint_as_float(((y) >> 9) | 0x3f800000u)), one_m)
    const f32x2 u0 = LV_U2(a0, b0), u1 = LV_U2(a1, b1), u2 = LV_U2(a2, b2), u3 = LV_U2(a3, b3);
#undef LV_U2
    {
        const f32x2 l = mul2(m2ln2, pk2(lg2_approx(lo2(u0)), lg2_approx(hi2(u0))));
        const f32x2 rho = pk2(sqrt_approx(lo2(l)), sqrt_approx(hi2(l)));
        const f32x2 ang = mul2(two_pi, sub2(u1, half));
        float sa, ca, sb, cb;
        __sincosf(lo2(ang), &sa, &ca);
        __sincosf(hi2(ang), &sb, &cb);
        nz[0] = mul2(rho, pk2(ca, cb));
        nz[1] = mul2(rho, pk2(sa, sb));
    }
    {
        const f32x2 l = mul2(m2ln2, pk2(lg2_approx(lo2(u2)), lg2_approx(hi2(u2))));
        const f32x2 rho = pk2(sqrt_approx(lo2(l)), sqrt_approx(hi2(l)));
        const f32x2 ang = mul2(two_pi, sub2(u3, half));
        float sa, ca, sb, cb;
        __sincosf(lo2(ang), &sa, &ca);
        __sincosf(hi2(ang), &sb, &cb);
        nz[2] = mul2(rho, pk2(ca, cb));
        nz[3] = mul2(rho, pk2(sa, sb));
    }
}

// normals4 of one path, NEGATED (nz[q] = -z[q] bit for bit), with the pairs
// (0, 2) and (1, 3) of its binary32 arithmetic in packed pairs: the uniforms'
// shift, the -2 ln 2 scale, the angle's shift and scale, and the rho cos / rho
// sin products, each element rounded as in normals4.
__device__ __forceinline__ void normals4_neg(uint32_t blk, uint32_t c1, uint32_t c2, uint32_t k0, uint32_t k1,
                                             float nz[4])
{
    uint32_t w0 = blk, w1 = c1, w2 = c2, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, k0, k1);
    const f32x2 one_m = pk2(__uint_as_float(0x3f7fffffu), __uint_as_float(0x3f7fffffu));
    const f32x2 u02 = sub2(pk2(__uint_as_float((w0 >> 9) | 0x3f800000u), __uint_as_float((w2 >> 9) | 0x3f800000u)),
                           one_m);
    const f32x2 u13 = sub2(pk2(__uint_as_float((w1 >> 9) | 0x3f800000u), __uint_as_float((w3 >> 9) | 0x3f800000u)),
                           one_m);
    const f32x2 l = mul2(pk2(-1.3862943611198906f, -1.3862943611198906f),
                         pk2(lg2_approx(lo2(u02)), lg2_approx(hi2(u02))));
    const f32x2 rho = pk2(sqrt_approx(lo2(l)), sqrt_approx(hi2(l)));
    const f32x2 ang = mul2(pk2(6.2831853071795865f, 6.2831853071795865f), sub2(u13, pk2(0.5f, 0.5f)));
    float s0, c0, s2, c2v;
    __sincosf(lo2(ang), &s0, &c0);
    __sincosf(hi2(ang), &s2, &c2v);
    const f32x2 zc = mul2(rho, pk2(c0, c2v));
    const f32x2 zs = mul2(rho, pk2(s0, s2));
    nz[0] = lo2(zc);
    nz[1] = lo2(zs);
    nz[2] = hi2(zc);
    nz[3] = hi2(zs);
}

// Time data of step n: t_n = n dt, j_n = the largest j <= J-2 with
// tau_j <= t_n, v_n = (t_n - tau_j) / (tau_{j+1} - tau_j) clamped to
// [0, 1], decided in binary64. Returned as (j (I-1), (j+1) (I-1), j I, bits
// of v): the rows of the sigma pairs for j and j + 1 and the bucket row.
__device__ __forceinline__ int4 step_time(const McParams& P, int n)
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
    return make_int4(j * (P.I - 1), (j + 1) * (P.I - 1), j * P.I, __float_as_int((float)v));
}

// Time slope factor of step n for d price / d T: (n / N) / (tau_{j+1} - tau_j)
// with the cell of step_time while t_n lies in [tau_0, tau_{J-1}) (the grid is
// flat in t outside, and with one time node), else 0; decided in binary64.
__device__ __forceinline__ float step_tdt(const McParams& P, int n)
{
    const double t = (double)n * P.dt_d;
    if (P.J < 2 || t < P.tau[0] || t >= P.tau[P.J - 1]) return 0.0f;
    int lo = 0, hi = P.J - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.tau[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return (float)(((double)n / (double)P.N) / (P.tau[lo + 1] - P.tau[lo]));
}

// Shared-memory view of the grid for one block.
struct SmemGrid {
    const int4* tab;       // [N] per step: (j (I-1), (j+1) (I-1), j I, bits of v)
    const float2* sig2;    // [Je][I-1]: (sigma_{i,j}, sigma_{i+1,j} - sigma_{i,j})
    const float* node;     // [I]
    const float2* ab;      // [I - 1]
    const float* tdt;      // [N] step_tdt (kernels that compute d price / d T)
};

// Spot cell: the largest i <= I-2 with s_i <= S. On log-uniform grids the
// index comes from y = log2 S directly (off by one only when S is within
// binary32 rounding of a node, where the clamped weight gives the same
// value); on other grids a binary search over the nodes.
__device__ __forceinline__ int spot_cell(const McParams& P, const SmemGrid& g, float y, float S)
{
    if (P.log_uniform) {
        const int i = __float2int_rd(fmaf(y, P.cell_scale, P.cell_shift));
        return min(max(i, 0), P.I - 2);
    }
    int lo = 0, hi = P.I - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.node[mid] <= S) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The model a kernel is instantiated for: bit 0 makes the spot weight
// linear in ln S instead of S (the other reading of Sec. IV-D's bilinear
// interpolation on a log-spaced grid); bit 1 runs the Euler scheme on S
// itself instead of ln S (the other reading of Sec. IV-A). The path state x
// is y = log2 S, or S under bit 1. Model 0 is the main reading.
constexpr int kModelLogWeight = 1;
constexpr int kModelEulerS = 2;
constexpr float kLog2e = 1.4426950408889634f;

struct StepEval {
    float S;       // S_n
    float sigma;   // sigma(S_n, t_n)
    float u;       // clamped spot weight
    int i;         // spot cell
    float sslope;  // S d sigma / d S = d sigma / d ln S (0 outside the grid)
    float dsig_t;  // sigma(S, tau_{j+1}) - sigma(S, tau_j) at the step's spot
};

// Bilinear sigma at (S_n, t_n), Sec. IV-D, from the path state x; the
// slope only when WANT_SLOPE. With the ln-S weight the cell coefficients ab
// are (1 / (y_{i+1} - y_i), -y_i / (y_{i+1} - y_i)) in y = log2 s, so that
// d u / d ln S = ab.x log2(e); otherwise they are in S.
template <bool WANT_SLOPE, int MODEL = 0>
__device__ __forceinline__ StepEval eval_sigma(const McParams& P, const SmemGrid& g, float x,
                                               const int4& tb)
{
    StepEval e;
    float y;
    if (MODEL & kModelEulerS) {
        e.S = x;
        y = lg2_approx(fmaxf(x, 1e-30f));       // a spot at or below 0 is below the grid
    } else {
        e.S = ex2_approx(x);
        y = x;
    }
    e.i = spot_cell(P, g, y, e.S);
    const float2 ab = g.ab[e.i];
    e.u = __saturatef(fmaf((MODEL & kModelLogWeight) ? y : e.S, ab.x, ab.y));
    const float2 lo = g.sig2[tb.x + e.i];      // time row j:     sigma_{i,j},   its spot step
    const float2 hi = g.sig2[tb.y + e.i];      // time row j + 1
    const float v = __int_as_float(tb.w);
    const float top = fmaf(e.u, lo.y, lo.x);
    const float bot = fmaf(e.u, hi.y, hi.x);
    e.sigma = fmaf(v, bot - top, top);
    e.dsig_t = bot - top;
    if (WANT_SLOPE) {
        const bool inside = (e.S >= P.s_lo) && (e.S <= P.s_hi);
        const float d = fmaf(v, hi.y - lo.y, lo.y) * ab.x;     // d sigma / d (S or y)
        e.sslope = inside ? ((MODEL & kModelLogWeight) ? d * kLog2e : e.S * d) : 0.0f;
    } else {
        e.sslope = 0.0f;
    }
    return e;
}

// Log-Euler step (Sec. IV-A) on y = x log2(e):
//   y_{n+1} = y_n + log2(e) [(r - sigma^2/2) dt + sigma sqrt(dt) Z]
// with rdt = log2(e) r dt, hdt = log2(e) dt / 2, sqdt2 = log2(e) sqrt(dt).
__device__ __forceinline__ float euler_step(const McParams& P, float y, float sigma, float z)
{
    return y + fmaf(sigma, P.sqdt2 * z, fmaf(-P.hdt * sigma, sigma, P.rdt));
}

// One step of the model's scheme: the log-Euler step, or on S
//   S_{n+1} = S_n (1 + r dt + sigma_n sqrt(dt) Z_n)   (rdt = r dt there).
template <int MODEL>
__device__ __forceinline__ float step_state(const McParams& P, float x, float sigma, float z)
{
    if (MODEL & kModelEulerS) return fmaf(x, fmaf(sigma, P.sqdt * z, P.rdt), x);
    return euler_step(P, x, sigma, z);
}

// Adjoint factors of step n: h = d x_{n+1} / d sigma_n and g with
// d x_{n+1} / d x_n = 1 + g. On ln S: h = sqrt(dt) Z - sigma dt,
// g = h S d sigma / d S. On S the adjoint runs scaled by S0 (xbar_N =
// e^{-rT} phi S0 on paths in the money, so that xbar_0 = d V / d ln S0 as on
// ln S): h = S_n sqrt(dt) Z / S0, g = r dt + sqrt(dt) Z (sigma + S d sigma / d S).
template <int MODEL>
__device__ __forceinline__ void adjoint_factors(const McParams& P, const StepEval& e, float z, float& h, float& g)
{
    if (MODEL & kModelEulerS) {
        const float w = P.sqdt * z;
        h = e.S * P.inv_S0 * w;
        g = fmaf(w, e.sigma + e.sslope, P.rdt);
    } else {
        h = fmaf(P.sqdt, z, -e.sigma * P.dt);
        g = h * e.sslope;
    }
}

// Explicit dependence of x_{n+1} on r and on the maturity T (n_steps fixed:
// dt = T / N, t_n = n T / N, the grid fixed in time), in the adjoint's units:
// on ln S, d x / d r = dt and d x / d T = ((r - sigma^2/2) + sigma Z / (2
// sqrt(dt))) / N + h d sigma / d t (n / N); on S the same with S_n (r dt) and
// S_n (r + sigma Z / (2 sqrt(dt))), over S0 like h.
template <int MODEL>
__device__ __forceinline__ void extra_factors(const McParams& P, const StepEval& e, float z, float h, float tdt,
                                              float& ar, float& at)
{
    const float ttime = h * e.dsig_t * tdt;
    if (MODEL & kModelEulerS) {
        const float s = e.S * P.inv_S0;
        ar = s * P.dt;
        at = fmaf(s * fmaf(e.sigma * z, P.half_inv_sqdt, P.r_nat), P.inv_N, ttime);
    } else {
        ar = P.dt;
        at = fmaf(fmaf(e.sigma * z, P.half_inv_sqdt, fmaf(-0.5f * e.sigma, e.sigma, P.r_nat)), P.inv_N, ttime);
    }
}

// 1 + g_n for the tangent-ratio form (one rounding on ln S).
template <int MODEL>
__device__ __forceinline__ float tangent_factor(const McParams& P, const StepEval& e, float z, float h)
{
    if (MODEL & kModelEulerS) return fmaf(P.sqdt * z, e.sigma + e.sslope, 1.0f + P.rdt);
    return fmaf(h, e.sslope, 1.0f);
}

// Discounted payoff V and terminal adjoint xbar_N from the final state
// (Sec. IV-B): xbar_N = e^{-rT} 1{phi (S_N - K) > 0} phi S_N on ln S, with
// S0 in place of S_N on S (the scaled adjoint of adjoint_factors).
template <int MODEL>
__device__ __forceinline__ void payoff(const McParams& P, float x, float& V, float& xbarN)
{
    const float SN = (MODEL & kModelEulerS) ? x : exp2f(x);
    const float itm = P.phi * (SN - P.K);
    V = itm > 0.0f ? P.disc * itm : 0.0f;
    xbarN = itm > 0.0f ? P.disc * P.phi * ((MODEL & kModelEulerS) ? P.S0f : SN) : 0.0f;
}

// ln S of a path state (per-path diagnostics).
template <int MODEL>
__device__ __forceinline__ float ln_spot(float x)
{
    return (MODEL & kModelEulerS) ? logf(x) : x * 0.6931471805599453f;
}

// Near-node decision log of the DBG instantiation: (path, step, 2 i + inside).
__device__ __forceinline__ void log_cell_decision(const McParams& P, const SmemGrid& g, const StepEval& e,
                                                  long long rel, int n)
{
    const float lo = g.node[e.i], hi = g.node[e.i + 1];
    if (fabsf(e.S - lo) <= P.dbg_band * lo || fabsf(e.S - hi) <= P.dbg_band * hi) {
        const bool inside = (e.S >= P.s_lo) && (e.S <= P.s_hi);
        const unsigned long long k = atomicAdd(P.dbg_ev_count, 1ull);
        if (k < (unsigned long long)P.dbg_ev_cap) {
            P.dbg_ev[3 * k + 0] = (int)rel;
            P.dbg_ev[3 * k + 1] = n;
            P.dbg_ev[3 * k + 2] = 2 * e.i + (inside ? 1 : 0);
        }
    }
}

// Forward pass of one path from x0; checkpoints every KCK steps when STORE.
template <int KCK, bool STORE, bool DBG, int MODEL = 0>
__device__ __forceinline__ float forward_path(const McParams& P, const SmemGrid& g, uint32_t c1, uint32_t c2,
                                              float* ck, size_t cks, long long rel)
{
    float x = P.x0;
    float z[4];
    const int nseg = (P.N + KCK - 1) / KCK;
    for (int m = 0; m < nseg; ++m) {
        if (STORE) ck[(size_t)m * cks] = x;
#pragma unroll
        for (int q = 0; q < KCK; ++q) {
            const int n = m * KCK + q;
            if (n < P.N) {
                if ((q & 3) == 0) normals4((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
                const int4 tb = g.tab[n];
                const StepEval e = eval_sigma<false, MODEL>(P, g, x, tb);
                if (DBG) log_cell_decision(P, g, e, rel, n);
                x = step_state<MODEL>(P, x, e.sigma, z[q & 3]);
            }
        }
    }
    return x;
}

// Forward passes of two paths, interleaved so the scheduler has two
// independent dependency chains; each path's arithmetic is exactly that of
// forward_path (its checkpoints and terminal state are bit-identical), and
// the per-step time data is loaded once for both. Path b is logged only
// when log_b (it may lie past the end of the call's range). With PACK (every
// reading, no logging) the two paths' binary32 arithmetic runs in packed
// pairs: the Box-Muller products and shifts, the spot-cell index, the time
// blend of sigma and the whole Euler step (on y = log2 S or on S); the loads
// and the transcendental unit stay per path. The step uses sqdt2 Z =
// (-sqdt2)(-Z) (sqdt Z on S), exact, so the negated normals need no sign flip.
template <int KCK, bool STORE, bool DBG, int MODEL = 0, bool PACK = false>
__device__ __forceinline__ void forward_path2(const McParams& P, const SmemGrid& g, uint32_t c1a, uint32_t c2a,
                                              uint32_t c1b, uint32_t c2b, float* cka, float* ckb, size_t cks,
                                              long long rel_a, long long rel_b, bool log_b, float& ya_out,
                                              float& yb_out)
{
    const int nseg = (P.N + KCK - 1) / KCK;
    if constexpr (PACK && !DBG) {
        // the path state x is y = log2 S (log-Euler) or S (Euler on S)
        constexpr bool kOnS = (MODEL & kModelEulerS) != 0, kLnW = (MODEL & kModelLogWeight) != 0;
        const f32x2 csc = pk2(P.cell_scale, P.cell_scale), csh = pk2(P.cell_shift, P.cell_shift);
        const f32x2 nsq = pk2(-P.sqdt2, -P.sqdt2), nhdt = pk2(-P.hdt, -P.hdt), rdt = pk2(P.rdt, P.rdt);
        const f32x2 nsqdt = pk2(-P.sqdt, -P.sqdt);
        f32x2 x = pk2(P.x0, P.x0);
        f32x2 nz[4];
        for (int m = 0; m < nseg; ++m) {
            if (STORE) {
                cka[(size_t)m * cks] = lo2(x);
                ckb[(size_t)m * cks] = hi2(x);
            }
#pragma unroll
            for (int q = 0; q < KCK; ++q) {
                const int n = m * KCK + q;
                if (n < P.N) {
                    if ((q & 3) == 0) normals4x2_neg((uint32_t)(n >> 2), c1a, c2a, c1b, c2b, P.k0, P.k1, nz);
                    const int4 tb = g.tab[n];
                    const float v = __int_as_float(tb.w);
                    // eval_sigma<false, MODEL> for both paths
                    float Sa, Sb;
                    f32x2 y;
                    if (kOnS) {
                        Sa = lo2(x);
                        Sb = hi2(x);
                        y = pk2(lg2_approx(fmaxf(Sa, 1e-30f)), lg2_approx(fmaxf(Sb, 1e-30f)));
                    } else {
                        y = x;
                        Sa = ex2_approx(lo2(y));
                        Sb = ex2_approx(hi2(y));
                    }
                    int ia, ib;
                    if (P.log_uniform) {
                        const f32x2 ci = fma2(y, csc, csh);
                        ia = min(max(__float2int_rd(lo2(ci)), 0), P.I - 2);
                        ib = min(max(__float2int_rd(hi2(ci)), 0), P.I - 2);
                    } else {
                        ia = spot_cell(P, g, lo2(y), Sa);
                        ib = spot_cell(P, g, hi2(y), Sb);
                    }
                    const float2 aba = g.ab[ia], abb = g.ab[ib];
                    // the spot weight is linear in S, or in y = log2 S under the ln-S weight
                    const float ua = __saturatef(fmaf(kLnW ? lo2(y) : Sa, aba.x, aba.y));
                    const float ub = __saturatef(fmaf(kLnW ? hi2(y) : Sb, abb.x, abb.y));
                    const float2 loa = g.sig2[tb.x + ia], hia = g.sig2[tb.y + ia];
                    const float2 lob = g.sig2[tb.x + ib], hib = g.sig2[tb.y + ib];
                    const f32x2 top = pk2(fmaf(ua, loa.y, loa.x), fmaf(ub, lob.y, lob.x));
                    const f32x2 bot = pk2(fmaf(ua, hia.y, hia.x), fmaf(ub, hib.y, hib.x));
                    const f32x2 sig = fma2(pk2(v, v), sub2(bot, top), top);
                    if (kOnS) {
                        // step_state: S (1 + r dt + sigma sqrt(dt) Z), sqrt(dt) Z = (-sqrt(dt))(-Z)
                        x = fma2(x, fma2(sig, mul2(nsqdt, nz[q & 3]), rdt), x);
                    } else {
                        // euler_step: y + fma(sigma, sqdt2 Z, fma(-hdt sigma, sigma, rdt))
                        const f32x2 t3 = fma2(mul2(nhdt, sig), sig, rdt);
                        x = add2(x, fma2(sig, mul2(nsq, nz[q & 3]), t3));
                    }
                }
            }
        }
        ya_out = lo2(x);
        yb_out = hi2(x);
        return;
    }
    float ya = P.x0, yb = P.x0;
    float za[4], zb[4];
    for (int m = 0; m < nseg; ++m) {
        if (STORE) {
            cka[(size_t)m * cks] = ya;
            ckb[(size_t)m * cks] = yb;
        }
#pragma unroll
        for (int q = 0; q < KCK; ++q) {
            const int n = m * KCK + q;
            if (n < P.N) {
                if ((q & 3) == 0) {
                    normals4((uint32_t)(n >> 2), c1a, c2a, P.k0, P.k1, za);
                    normals4((uint32_t)(n >> 2), c1b, c2b, P.k0, P.k1, zb);
                }
                const int4 tb = g.tab[n];
                const StepEval ea = eval_sigma<false, MODEL>(P, g, ya, tb);
                const StepEval eb = eval_sigma<false, MODEL>(P, g, yb, tb);
                if (DBG) {
                    log_cell_decision(P, g, ea, rel_a, n);
                    if (log_b) log_cell_decision(P, g, eb, rel_b, n);
                }
                ya = step_state<MODEL>(P, ya, ea.sigma, za[q & 3]);
                yb = step_state<MODEL>(P, yb, eb.sigma, zb[q & 3]);
            }
        }
    }
    ya_out = ya;
    yb_out = yb;
}

// Philox counter words of path `rel` of the call: c1 = path bits 0..31,
// c2 = path bits 32..47 | stream_id << 16 (the path index is path_begin + rel).
__device__ __forceinline__ void path_counter(const McParams& P, long long rel, uint32_t& c1, uint32_t& c2)
{
    const unsigned long long p = (unsigned long long)(P.path_begin + rel);
    c1 = (uint32_t)p;
    c2 = ((uint32_t)(p >> 32) & 0xffffu) | (P.stream_id << 16);
}

// Reverse sweep of one path (Sec. III / IV-C, back-propagation through the
// Euler scheme) from its terminal adjoint xbar = d V / d x_N. Per checkpoint
// segment, last to first: recompute KCK steps from the checkpoint keeping
// h_n = d x_{n+1} / d sigma_n = sqrt(dt) Z_n - sigma_n dt,
// g_n = h_n S_n d sigma / d S, the cell and the spot weight in registers; then
// walk them back: sigma_bar_n = xbar_{n+1} h_n, xbar_n = xbar_{n+1} (1 + g_n),
// and spread sigma_bar_n over the corner buckets (i, j), (i+1, j), (i, j+1),
// (i+1, j+1) with the bilinear weights. Corner sums are kept in registers
// while the cell is unchanged and then added to the block's binary32 buckets
// `l1` (time-major, row j * I) with red.global.add.f32. Returns d V / d x_0.
// With NEG (no extra sums) the recompute takes its normals from
// normals4_neg and uses sqdt Z = (-sqdt)(-Z) and sqdt2 Z = (-sqdt2)(-Z),
// which are exact, so every value is the same bit for bit.
template <int KCK, int MODEL = 0, bool EXTRA = false, bool NEG = false>
__device__ __forceinline__ float reverse_path(const McParams& P, const SmemGrid& g, uint32_t c1, uint32_t c2,
                                              const float* ck, size_t cks, float xbar, float* l1,
                                              float* rho_acc = nullptr, float* t_acc = nullptr)
{
    const int nseg = (P.N + KCK - 1) / KCK;
    int cur = -1;
    float A = 0.0f, AU = 0.0f, Bs = 0.0f, BU = 0.0f;
    float z[4];
    float x_next = ck[(size_t)(nseg - 1) * cks];
    for (int m = nseg - 1; m >= 0; --m) {
        float x = x_next;
        if (m > 0) x_next = ck[(size_t)(m - 1) * cks];    // in flight during this segment
        float hq[KCK], gq[KCK], uq[KCK];
        float aq[EXTRA ? KCK : 1], tq[EXTRA ? KCK : 1];
        int iq[KCK];
#pragma unroll
        for (int q = 0; q < KCK; ++q) {
            const int n = m * KCK + q;
            if (n < P.N) {
                constexpr bool kNeg = NEG && !EXTRA;
                if ((q & 3) == 0) {
                    if (kNeg) normals4_neg((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
                    else normals4((uint32_t)(n >> 2), c1, c2, P.k0, P.k1, z);
                }
                const int4 tb = g.tab[n];
                const StepEval ev = eval_sigma<true, MODEL>(P, g, x, tb);
                if (kNeg) {                    // z holds -Z: adjoint_factors with sqrt(dt) Z = (-sqrt(dt))(-Z)
                    if (MODEL & kModelEulerS) {
                        const float w = -P.sqdt * z[q & 3];
                        hq[q] = ev.S * P.inv_S0 * w;
                        gq[q] = fmaf(w, ev.sigma + ev.sslope, P.rdt);
                    } else {
                        hq[q] = fmaf(-P.sqdt, z[q & 3], -ev.sigma * P.dt);
                        gq[q] = hq[q] * ev.sslope;
                    }
                } else {
                    adjoint_factors<MODEL>(P, ev, z[q & 3], hq[q], gq[q]);
                }
                if (EXTRA) extra_factors<MODEL>(P, ev, z[q & 3], hq[q], g.tdt[n], aq[EXTRA ? q : 0], tq[EXTRA ? q : 0]);
                uq[q] = ev.u;
                iq[q] = ev.i;
                if (kNeg && (MODEL & kModelEulerS)) x = fmaf(x, fmaf(ev.sigma, -P.sqdt * z[q & 3], P.rdt), x);
                else if (kNeg) x = x + fmaf(ev.sigma, -P.sqdt2 * z[q & 3], fmaf(-P.hdt * ev.sigma, ev.sigma, P.rdt));
                else x = step_state<MODEL>(P, x, ev.sigma, z[q & 3]);
            }
        }
#pragma unroll
        for (int q = KCK - 1; q >= 0; --q) {
            const int n = m * KCK + q;
            if (n < P.N) {
                const int4 tb = g.tab[n];
                const int key = tb.z + iq[q];
                const float v = __int_as_float(tb.w);
                const float sbar = xbar * hq[q];
                if (EXTRA) {                             // xbar is still xbar_{n+1}
                    *rho_acc = fmaf(xbar, aq[EXTRA ? q : 0], *rho_acc);
                    *t_acc = fmaf(xbar, tq[EXTRA ? q : 0], *t_acc);
                }
                xbar = fmaf(xbar, gq[q], xbar);
                if (key != cur) {
                    if (cur >= 0) {
                        float* p0 = l1 + cur;
                        float* p1 = p0 + P.I;
                        atomicAdd(p0, A - AU);
                        atomicAdd(p0 + 1, AU);
                        atomicAdd(p1, Bs - BU);
                        atomicAdd(p1 + 1, BU);
                    }
                    A = AU = Bs = BU = 0.0f;
                    cur = key;
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
        float* p0 = l1 + cur;
        float* p1 = p0 + P.I;
        atomicAdd(p0, A - AU);
        atomicAdd(p0 + 1, AU);
        atomicAdd(p1, Bs - BU);
        atomicAdd(p1 + 1, BU);
    }
    return xbar;
}

// Tangent-ratio form of the pathwise adjoint (Sec. III: the adjoint
// recursion xbar_n = xbar_{n+1} (1 + g_n) is linear, so with the tangent
// D_0 = 1, D_{n+1} = D_n (1 + g_n) = d x_{n+1} / d x_0 one has
// xbar_{n+1} = xbar_N D_N / D_{n+1} and xbar_0 = xbar_N D_N).
//
// Pass 1: the forward pass of one path keeping D. Returns y_N = log2 S_N and
// D_N; `tiny` is set when some |1 + g_n| < 2^-20, where dividing by D loses
// what the reverse sweep keeps. The path's arithmetic is that of
// forward_path (same sigma, same Euler step), so y_N is the same.
template <int MODEL = 0>
__device__ __forceinline__ float tangent_forward(const McParams& P, const SmemGrid& g, uint32_t c1, uint32_t c2,
                                                 float& D, bool& tiny)
{
    float y = P.x0;
    float d = 1.0f, fmin = 1.0f;
    float z[4];
    for (int n0 = 0; n0 < P.N; n0 += 4) {
        normals4((uint32_t)(n0 >> 2), c1, c2, P.k0, P.k1, z);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = n0 + q;
            if (n < P.N) {
                const int4 tb = g.tab[n];
                const StepEval e = eval_sigma<true, MODEL>(P, g, y, tb);
                float h, gn;
                adjoint_factors<MODEL>(P, e, z[q], h, gn);
                const float f = tangent_factor<MODEL>(P, e, z[q], h);   // 1 + g_n
                fmin = fminf(fmin, fabsf(f));
                d *= f;
                y = step_state<MODEL>(P, y, e.sigma, z[q]);
            }
        }
    }
    D = d;
    tiny = fmin < 0x1p-20f;
    return y;
}

// Pass 1 for two paths at once (main reading), their binary32 arithmetic in
// packed pairs as in forward_path2: per path every value is rounded as in
// tangent_forward (same y_N, D_N and tiny flag). The slope's time blend and
// spot factor, h = sqdt Z - sigma dt = (-sqdt)(-Z) + (-dt) sigma, 1 + g_n and
// the product D run in pairs; the inside-grid test and the running minimum of
// |1 + g_n| stay per path.
__device__ __forceinline__ void tangent_forward2(const McParams& P, const SmemGrid& g, uint32_t c1a, uint32_t c2a,
                                                 uint32_t c1b, uint32_t c2b, float& ya_out, float& yb_out,
                                                 float& Da, float& Db, bool& tiny_a, bool& tiny_b)
{
    const f32x2 csc = pk2(P.cell_scale, P.cell_scale), csh = pk2(P.cell_shift, P.cell_shift);
    const f32x2 nsq2 = pk2(-P.sqdt2, -P.sqdt2), nhdt = pk2(-P.hdt, -P.hdt), rdt = pk2(P.rdt, P.rdt);
    const f32x2 nsqdt = pk2(-P.sqdt, -P.sqdt), ndt = pk2(-P.dt, -P.dt), one = pk2(1.0f, 1.0f);
    f32x2 y = pk2(P.x0, P.x0), d = one;
    float fmin_a = 1.0f, fmin_b = 1.0f;
    f32x2 nz[4];
    for (int n0 = 0; n0 < P.N; n0 += 4) {
        normals4x2_neg((uint32_t)(n0 >> 2), c1a, c2a, c1b, c2b, P.k0, P.k1, nz);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = n0 + q;
            if (n < P.N) {
                const int4 tb = g.tab[n];
                const float v = __int_as_float(tb.w);
                const f32x2 vv = pk2(v, v);
                // eval_sigma<true, 0> for both paths
                const float Sa = ex2_approx(lo2(y)), Sb = ex2_approx(hi2(y));
                int ia, ib;
                if (P.log_uniform) {
                    const f32x2 ci = fma2(y, csc, csh);
                    ia = min(max(__float2int_rd(lo2(ci)), 0), P.I - 2);
                    ib = min(max(__float2int_rd(hi2(ci)), 0), P.I - 2);
                } else {
                    ia = spot_cell(P, g, lo2(y), Sa);
                    ib = spot_cell(P, g, hi2(y), Sb);
                }
                const float2 aba = g.ab[ia], abb = g.ab[ib];
                const float ua = __saturatef(fmaf(Sa, aba.x, aba.y));
                const float ub = __saturatef(fmaf(Sb, abb.x, abb.y));
                const float2 loa = g.sig2[tb.x + ia], hia = g.sig2[tb.y + ia];
                const float2 lob = g.sig2[tb.x + ib], hib = g.sig2[tb.y + ib];
                const f32x2 top = pk2(fmaf(ua, loa.y, loa.x), fmaf(ub, lob.y, lob.x));
                const f32x2 bot = pk2(fmaf(ua, hia.y, hia.x), fmaf(ub, hib.y, hib.x));
                const f32x2 sig = fma2(vv, sub2(bot, top), top);
                const f32x2 ly = pk2(loa.y, lob.y);
                const f32x2 sl = mul2(pk2(Sa, Sb), mul2(fma2(vv, sub2(pk2(hia.y, hib.y), ly), ly), pk2(aba.x, abb.x)));
                const f32x2 slope = pk2((Sa >= P.s_lo) && (Sa <= P.s_hi) ? lo2(sl) : 0.0f,
                                        (Sb >= P.s_lo) && (Sb <= P.s_hi) ? hi2(sl) : 0.0f);
                // adjoint_factors<0> and tangent_factor<0>
                const f32x2 h = fma2(nsqdt, nz[q], mul2(ndt, sig));
                const f32x2 f = fma2(h, slope, one);
                fmin_a = fminf(fmin_a, fabsf(lo2(f)));
                fmin_b = fminf(fmin_b, fabsf(hi2(f)));
                d = mul2(d, f);
                // euler_step
                const f32x2 t3 = fma2(mul2(nhdt, sig), sig, rdt);
                y = add2(y, fma2(sig, mul2(nsq2, nz[q]), t3));
            }
        }
    }
    ya_out = lo2(y);
    yb_out = hi2(y);
    Da = lo2(d);
    Db = hi2(d);
    tiny_a = fmin_a < 0x1p-20f;
    tiny_b = fmin_b < 0x1p-20f;
}

// Pass 2: regenerates one path (same counters, same arithmetic) and spreads
// sigma_bar_n = c h_n / D_{n+1}, c = xbar_N D_N, over the corner buckets of
// its cell with the bilinear weights, through the same run-length register
// sums and binary32 reductions into `l1` as reverse_path, in time order.
template <int MODEL = 0>
__device__ __forceinline__ void tangent_scatter(const McParams& P, const SmemGrid& g, uint32_t c1, uint32_t c2,
                                                float c, float* l1)
{
    float y = P.x0, d = 1.0f;
    int cur = -1;
    float A = 0.0f, AU = 0.0f, Bs = 0.0f, BU = 0.0f;
    float z[4];
    for (int n0 = 0; n0 < P.N; n0 += 4) {
        normals4((uint32_t)(n0 >> 2), c1, c2, P.k0, P.k1, z);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = n0 + q;
            if (n < P.N) {
                const int4 tb = g.tab[n];
                const StepEval e = eval_sigma<true, MODEL>(P, g, y, tb);
                float h, gn;
                adjoint_factors<MODEL>(P, e, z[q], h, gn);
                d *= tangent_factor<MODEL>(P, e, z[q], h);          // D_{n+1}
                const float sbar = __fdividef(c * h, d);
                const int key = tb.z + e.i;
                if (key != cur) {
                    if (cur >= 0) {
                        float* p0 = l1 + cur;
                        float* p1 = p0 + P.I;
                        atomicAdd(p0, A - AU);
                        atomicAdd(p0 + 1, AU);
                        atomicAdd(p1, Bs - BU);
                        atomicAdd(p1 + 1, BU);
                    }
                    A = AU = Bs = BU = 0.0f;
                    cur = key;
                }
                const float b = sbar * __int_as_float(tb.w);
                const float a = sbar - b;
                A += a;
                AU = fmaf(a, e.u, AU);
                Bs += b;
                BU = fmaf(b, e.u, BU);
                y = step_state<MODEL>(P, y, e.sigma, z[q]);
            }
        }
    }
    if (cur >= 0) {
        float* p0 = l1 + cur;
        float* p1 = p0 + P.I;
        atomicAdd(p0, A - AU);
        atomicAdd(p0 + 1, AU);
        atomicAdd(p1, Bs - BU);
        atomicAdd(p1 + 1, BU);
    }
}

// Second-order buckets d^2 price / (d S0 d sigma_ij), pass 2 of one live
// path (main reading): regenerates the path and adds, per step n,
//   Delta_p [ w_ij(n) a_n + S_n d w_ij / d S (n) b_n ]
//   a_n = (Z_n^2 - 1) / sigma_n - sqrt(dt) Z_n (1 + k_n / (sigma_n (1 + g_n))),
//   b_n = h_n / (1 + g_n),  k_n = S_n d sigma / d S,  g_n = h_n k_n,
// to the corners of its cell: the derivative of the pathwise delta Delta_p at
// the fixed path plus Delta_p times the derivative of the path's log
// density (the Gaussian Euler step), which together are unbiased for the
// second derivative although Delta_p itself jumps at the strike and at the
// nodes. Run-length sums in registers while the cell is unchanged (the
// weight terms as in reverse_path, the slope terms E0 = sum (1 - v) d,
// E1 = sum v d), then binary32 reductions into `l1`.
__device__ __forceinline__ void vanna_scatter(const McParams& P, const SmemGrid& g, uint32_t c1, uint32_t c2,
                                              float delta, float* l1)
{
    float y = P.x0;
    int cur = -1;
    float A = 0.0f, AU = 0.0f, Bs = 0.0f, BU = 0.0f, E0 = 0.0f, E1 = 0.0f;
    float z[4];
    for (int n0 = 0; n0 < P.N; n0 += 4) {
        normals4((uint32_t)(n0 >> 2), c1, c2, P.k0, P.k1, z);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = n0 + q;
            if (n < P.N) {
                const int4 tb = g.tab[n];
                const StepEval e = eval_sigma<true, 0>(P, g, y, tb);
                const float zq = z[q];
                const float h = fmaf(P.sqdt, zq, -e.sigma * P.dt);
                const float f = fmaf(h, e.sslope, 1.0f);                      // 1 + g_n
                const float a = __fdividef(fmaf(zq, zq, -1.0f), e.sigma) -
                                P.sqdt * zq * (1.0f + __fdividef(e.sslope, e.sigma * f));
                const bool inside = (e.S >= P.s_lo) && (e.S <= P.s_hi);
                const float sdu = inside ? e.S * g.ab[e.i].x : 0.0f;          // S d u / d S
                const float c = delta * a;
                const float d = delta * __fdividef(h, f) * sdu;
                const int key = tb.z + e.i;
                if (key != cur) {
                    if (cur >= 0) {
                        float* p0 = l1 + cur;
                        float* p1 = p0 + P.I;
                        atomicAdd(p0, A - AU - E0);
                        atomicAdd(p0 + 1, AU + E0);
                        atomicAdd(p1, Bs - BU - E1);
                        atomicAdd(p1 + 1, BU + E1);
                    }
                    A = AU = Bs = BU = E0 = E1 = 0.0f;
                    cur = key;
                }
                const float v = __int_as_float(tb.w);
                const float cb = c * v, ca = c - cb;
                const float db = d * v;
                A += ca;
                AU = fmaf(ca, e.u, AU);
                Bs += cb;
                BU = fmaf(cb, e.u, BU);
                E0 += d - db;
                E1 += db;
                y = step_state<0>(P, y, e.sigma, zq);
            }
        }
    }
    if (cur >= 0) {
        float* p0 = l1 + cur;
        float* p1 = p0 + P.I;
        atomicAdd(p0, A - AU - E0);
        atomicAdd(p0 + 1, AU + E0);
        atomicAdd(p1, Bs - BU - E1);
        atomicAdd(p1 + 1, BU + E1);
    }
}

}  // namespace lv
