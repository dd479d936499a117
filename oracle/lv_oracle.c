/*
 * lv_oracle.c -- plain FP64 CPU oracle for the Dupire local-volatility Monte
 * Carlo price and its pathwise adjoint (price, delta, one vega bucket per
 * grid node).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's
 * CPU-baseline leg call this file; the CUDA library never does, and it
 * shares no code, header or table with it. It is written for a reader who
 * checks it against the paper by eye: no blocking, no fusion, the whole
 * trajectory of a path is stored and the reverse sweep walks it back.
 *
 * What it follows (sections of arXiv 2002.02481):
 *   Sec. IV-A   dX/X = sigma(X, t) dW, discretised by an explicit Euler
 *               scheme; sigma given on a grid {(x_i, t_j)} of I x J nodes and
 *               interpolated between them.
 *   Sec. IV-B   European call payoff; pseudo-random normals.
 *   Sec. IV-C   price = mean over paths; sensitivities of that mean with
 *               respect to every grid value by back-propagation (AAD).
 *   Sec. IV-D   bilinear interpolation between the grid nodes.
 *   Sec. III    central bump-and-reprice, p0 +/- eps/2, divided by eps.
 *
 * Readings where the paper is silent (each one is listed in the design
 * notes of the repository):
 *   - Euler on x = ln X with drift r - sigma^2/2 and discount e^{-rT}
 *     (r = 0 is the paper's driftless SDE); sigma evaluated at the left
 *     point t_n = n T / N of each step.
 *   - Normals: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *     (seed low 32 bits, seed high 32 bits), counter = (n / 4, path low 32
 *     bits, (path bits 32..47) | stream_id << 16, 0). Each 32-bit word w
 *     becomes u = ((w >> 9) + 1/2) 2^-23, which lies in (0, 1) and is exact
 *     in binary32 and binary64. Box-Muller on word pairs (0,1) and (2,3):
 *     Z_a = sqrt(-2 ln u_a) cos(2 pi u_b), Z_b = sqrt(-2 ln u_a) sin(2 pi u_b);
 *     step n uses Z of word n mod 4.
 *   - Bilinear in S (not ln S) and t. Cell i = the largest i <= I-2 with
 *     s_i <= S (0 below the grid), u = (S - s_i)/(s_{i+1} - s_i) clamped to
 *     [0, 1]; the same in time. Outside the grid sigma is flat and
 *     d sigma/d S = 0. With one time node sigma does not depend on t.
 *   - Two further readings, selected by flags: the spot weight linear in
 *     ln S, u = (ln S - ln s_i)/(ln s_{i+1} - ln s_i) (surface flag
 *     ORC_INTERP_LOGS; Sec. IV-A's grid is uniform in price, the workloads'
 *     nodes are log-spaced), and the Euler scheme on X itself,
 *     X_{n+1} = X_n + r X_n dt + sigma_n X_n sqrt(dt) Z_n (option flag
 *     ORC_SCHEME_X; Sec. IV-A states "tomorrow's price" as today's plus its
 *     increment). Under ORC_SCHEME_X a spot at or below 0 is below the grid.
 *   - Payoff kink: the indicator 1{phi (S_N - K) > 0}, so a tie gives 0.
 *   - Vega is d price / d sigma_ij per unit of sigma.
 *   - Rho is d price / d r; d price / d T is the maturity sensitivity with
 *     the number of steps fixed (dt = T / N, t_n = n T / N) and the grid
 *     fixed in time, so sigma_n moves with t_n through d sigma / d t. Both
 *     come from the same reverse sweep: the derivative of the discount plus
 *     the sum over steps of xbar_{n+1} times d x_{n+1} / d r (or d T).
 *
 * Parity pins (tests/test_oracle_*.py): Philox against cuRAND's host
 * generator; normal moments and a KS test; Black-Scholes price, delta and
 * vega on a flat grid; the per-path vega-sum identity; the martingale
 * property; pathwise put-call parity; adjoint against central differences of
 * the forward estimator; adjoint against torch.autograd on an independent
 * FP64 restatement of the forward.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lv_oracle.h"

/* ------------------------------------------------------------------ Philox */

#define ORC_PI 3.14159265358979323846

/* Philox4x32 round constants: the two multipliers and the two Weyl key
 * increments (golden ratio and sqrt(3) - 1 in 32-bit fixed point) from the
 * SC'11 paper. */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * ldexp(1.0, -23);
}

void orc_counter(uint32_t block, uint64_t path, uint32_t stream_id, uint32_t ctr[4])
{
    ctr[0] = block;
    ctr[1] = (uint32_t)(path & 0xffffffffu);
    ctr[2] = (uint32_t)((path >> 32) & 0xffffu) | (stream_id << 16);
    ctr[3] = 0u;
}

void orc_normals4(uint64_t seed, uint32_t stream_id, uint64_t path, uint32_t block, double z[4])
{
    uint32_t ctr[4], key[2], w[4];
    orc_counter(block, path, stream_id, ctr);
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, w);
    for (int pair = 0; pair < 2; ++pair) {
        double ua = orc_uniform(w[2 * pair]);
        double ub = orc_uniform(w[2 * pair + 1]);
        double radius = sqrt(-2.0 * log(ua));
        double angle = 2.0 * ORC_PI * ub;
        z[2 * pair] = radius * cos(angle);
        z[2 * pair + 1] = radius * sin(angle);
    }
}

void orc_normals(uint64_t seed, uint32_t stream_id, uint64_t path, int32_t n_steps, double* z)
{
    double blk[4];
    for (int32_t n = 0; n < n_steps; ++n) {
        if (n % 4 == 0) orc_normals4(seed, stream_id, path, (uint32_t)(n / 4), blk);
        z[n] = blk[n % 4];
    }
}

/* ------------------------------------------------------ bilinear surface */

/* Largest c in [0, n-2] with nodes[c] <= x (0 when x < nodes[0]). */
static int32_t orc_cell(const double* nodes, int32_t n, double x)
{
    int32_t lo = 0, hi = n - 2;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) / 2;
        if (nodes[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

static double orc_clamp01(double a)
{
    return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
}

/* Bilinear sigma and d sigma / d S at (S, t) in spot cell i; `inside` says
 * whether S lies in [s_0, s_{I-1}] (outside, sigma is flat in S and its
 * S-derivative is 0). */
static void orc_sigma_in_cell(const orc_surface* sf, double S, double t, int32_t i, int inside,
                              orc_point* p)
{
    const int32_t J = sf->n_time;
    const double lo_s = sf->spot[i], hi_s = sf->spot[i + 1];
    const int logs = sf->interp == ORC_INTERP_LOGS;
    /* spot weight, clamped to [0, 1] (decided by comparison first, so that a
     * spot at or below 0 never reaches the logarithm) */
    double u;
    if (S <= lo_s) u = 0.0;
    else if (S >= hi_s) u = 1.0;
    else u = logs ? (log(S) - log(lo_s)) / (log(hi_s) - log(lo_s)) : (S - lo_s) / (hi_s - lo_s);
    /* d u / d S inside the cell */
    double du_dS = logs ? 1.0 / (S * (log(hi_s) - log(lo_s))) : 1.0 / (hi_s - lo_s);

    int32_t j = 0;
    double v = 0.0;
    int t_inside = 0;
    if (J > 1) {
        j = orc_cell(sf->time, J, t);
        v = orc_clamp01((t - sf->time[j]) / (sf->time[j + 1] - sf->time[j]));
        t_inside = t >= sf->time[0] && t < sf->time[J - 1];
    }
    /* sigma_ij lives at sig[i * J + j] */
    double s00 = sf->sigma[i * J + j];
    double s10 = sf->sigma[(i + 1) * J + j];
    double s01 = (J > 1) ? sf->sigma[i * J + j + 1] : 0.0;
    double s11 = (J > 1) ? sf->sigma[(i + 1) * J + j + 1] : 0.0;

    p->i = i;
    p->j = j;
    p->u = u;
    p->v = v;
    p->w[0] = (1.0 - u) * (1.0 - v);   /* node (i,   j)   */
    p->w[1] = u * (1.0 - v);           /* node (i+1, j)   */
    p->w[2] = (1.0 - u) * v;           /* node (i,   j+1) */
    p->w[3] = u * v;                   /* node (i+1, j+1) */
    p->sigma = p->w[0] * s00 + p->w[1] * s10 + p->w[2] * s01 + p->w[3] * s11;
    p->inside = inside;
    p->du_dS = inside ? du_dS : 0.0;
    if (inside)
        p->dsigma_dS = ((1.0 - v) * (s10 - s00) + v * (s11 - s01)) * du_dS;
    else
        p->dsigma_dS = 0.0;
    /* d sigma / d t at fixed S: the time slope of the cell (right derivative at
     * a time node; the grid is flat in t outside [t_0, t_{J-1})) */
    if (t_inside)
        p->dsigma_dt = ((1.0 - u) * (s01 - s00) + u * (s11 - s10)) / (sf->time[j + 1] - sf->time[j]);
    else
        p->dsigma_dt = 0.0;
}

void orc_sigma_eval(const orc_surface* sf, double S, double t, orc_point* p)
{
    const int32_t I = sf->n_spot;
    int32_t i = orc_cell(sf->spot, I, S);
    int inside = (S >= sf->spot[0] && S <= sf->spot[I - 1]);
    orc_sigma_in_cell(sf, S, t, i, inside, p);
}

/* --------------------------------------------------------------- one path */

typedef struct {
    double* x;   /* [N + 1] log-spot trajectory */
    double* z;   /* [N] normals */
} orc_workspace;

typedef struct {
    double V;       /* discounted payoff */
    double xbar0;   /* d V / d x_0 */
    double SN;      /* terminal spot */
    double vtot;    /* sum over buckets of this path's sigma adjoints */
    double rho;     /* d V / d r */
    double dvdt;    /* d V / d T */
    double amp;     /* sum over steps of (|g_n| + k_n^2 dt + 2 sqrt(dt) |Z_n k_n|) / |1 + g_n|,
                       k_n = S_n d sigma / d S, 1 + g_n = d x_{n+1} / d x_n: a bound on how
                       much a relative error e in every S_n moves ln |xbar_0| (at most amp e
                       to first order) */
    int kink;       /* |S_N - K| within the kink band */
} orc_path_result;

/* Decisions imposed from outside. Two integers of the method are decided
 * in floating point: the payoff indicator 1{phi (S_N - K) > 0} and the spot
 * cell of a step (with whether S lies inside the grid, which switches
 * d sigma / d S on). A binary32 implementation may decide them differently
 * for a path whose value lies within rounding of the strike or of a node.
 * Parity tests pass that implementation's decisions for those paths and
 * steps, so both sides take the same decisions. The oracle checks each one
 * against its own path: a decision that differs from its own is applied only
 * when the oracle's own value lies within the stated band of the value that
 * separates the two choices (the strike; the node between two adjacent
 * cells; the edge node for the inside-grid flag); any other is refused.
 * Lists are sorted ascending by path (and step). */
static int orc_forced_itm(const orc_decisions* d, uint64_t path)
{
    if (!d || d->n_itm <= 0) return -1;
    int64_t lo = 0, hi = d->n_itm - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((uint64_t)d->itm_path[mid] == path) return d->itm_val[mid] ? 1 : 0;
        if ((uint64_t)d->itm_path[mid] < path) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* [*first, *last) = the entries of `path` in the cell list. */
static void orc_cell_range(const orc_decisions* d, uint64_t path, int64_t* first, int64_t* last)
{
    *first = *last = 0;
    if (!d || d->n_cell <= 0) return;
    int64_t lo = 0, hi = d->n_cell;
    while (lo < hi) {                      /* first entry with path >= `path` */
        int64_t mid = lo + (hi - lo) / 2;
        if ((uint64_t)d->cell_path[mid] < path) lo = mid + 1;
        else hi = mid;
    }
    *first = lo;
    while (lo < d->n_cell && (uint64_t)d->cell_path[lo] == path) ++lo;
    *last = lo;
}

/* Forced cell code (2 i + inside) of step n, or -1. */
static int32_t orc_forced_cell(const orc_decisions* d, int64_t first, int64_t last, int32_t n)
{
    for (int64_t e = first; e < last; ++e)
        if (d->cell_step[e] == n) return d->cell_code[e];
    return -1;
}

/* Sigma at (S, t) in the cell of `code` (2 i + inside) when code >= 0, else
 * in the oracle's own cell. An imposed code that differs from the oracle's
 * own decision at S must be admissible: an adjacent cell, with S within
 * band * s of the node s between the two cells (the inside flag then agrees:
 * that node is interior), or the same cell with the other inside flag, with
 * S within band * s of the grid's edge node s_0 or s_{I-1} that the flag
 * switches at. Returns ORC_EDECISION otherwise; *overridden says whether the
 * imposed code differed from the oracle's own. */
static int orc_sigma_decided(const orc_surface* sf, double S, double t, int32_t code, double band,
                             orc_point* p, int* overridden)
{
    *overridden = 0;
    if (code < 0) {
        orc_sigma_eval(sf, S, t, p);
        return ORC_OK;
    }
    const int32_t I = sf->n_spot;
    const int32_t i_f = code >> 1;
    const int in_f = code & 1;
    if (i_f > I - 2) return ORC_EDECISION;
    const int32_t i_o = orc_cell(sf->spot, I, S);
    const int in_o = (S >= sf->spot[0] && S <= sf->spot[I - 1]);
    if (i_f != i_o || in_f != in_o) {
        int ok;
        if (i_f != i_o) {
            const double node = sf->spot[i_f > i_o ? i_f : i_o];
            ok = in_f == in_o && (i_f - i_o == 1 || i_o - i_f == 1) && fabs(S - node) <= band * node;
        } else {
            const int near_lo = i_o == 0 && fabs(S - sf->spot[0]) <= band * sf->spot[0];
            const int near_hi = i_o == I - 2 && fabs(S - sf->spot[I - 1]) <= band * sf->spot[I - 1];
            ok = near_lo || near_hi;
        }
        if (!ok) return ORC_EDECISION;
        *overridden = 1;
    }
    orc_sigma_in_cell(sf, S, t, i_f, in_f, p);
    return ORC_OK;
}

/* Simulates one path, and when want_greeks runs its reverse sweep and adds
 * every sigma adjoint to vega[i * J + j] (and |.| to kink_vega for paths
 * flagged near the payoff kink). Imposed decisions are checked as they are
 * applied (ORC_EDECISION for an inadmissible one); ov[0], ov[1] count the
 * applied cell and payoff decisions that differed from the oracle's own. */
static int orc_one_path(const orc_surface* sf, const orc_option* op, uint64_t path,
                        orc_workspace* ws, int want_greeks, double kink_tol,
                        const orc_decisions* dec, double* vega, double* kink_vega,
                        orc_path_result* res, int64_t ov[2])
{
    const int32_t N = op->n_steps, J = sf->n_time;
    const double dt = op->T / (double)N;
    const double sqdt = sqrt(dt);
    double* x = ws->x;
    double* z = ws->z;
    orc_point pt;

    orc_normals(op->seed, op->stream_id, path, N, z);
    int64_t c_first, c_last;
    orc_cell_range(dec, path, &c_first, &c_last);
    const double band = dec ? dec->band : 0.0;
    int overridden, st;

    /* forward: Euler on the log-spot, or on the spot itself (Sec. IV-A);
     * x holds ln S, or S under ORC_SCHEME_X */
    const int on_x = op->scheme == ORC_SCHEME_X;
    x[0] = on_x ? op->S0 : log(op->S0);
    for (int32_t n = 0; n < N; ++n) {
        double t = (double)n * dt;
        double S = on_x ? x[n] : exp(x[n]);
        st = orc_sigma_decided(sf, S, t, orc_forced_cell(dec, c_first, c_last, n), band, &pt, &overridden);
        if (st != ORC_OK) return st;
        ov[0] += overridden;
        if (on_x)
            x[n + 1] = x[n] + op->r * x[n] * dt + pt.sigma * x[n] * sqdt * z[n];
        else
            x[n + 1] = x[n] + (op->r - 0.5 * pt.sigma * pt.sigma) * dt + pt.sigma * sqdt * z[n];
    }

    /* payoff (Sec. IV-B) */
    const double disc = exp(-op->r * op->T);
    const double SN = on_x ? x[N] : exp(x[N]);
    const double itm = (double)op->phi * (SN - op->K);
    res->V = disc * (itm > 0.0 ? itm : 0.0);
    res->SN = SN;
    res->kink = (kink_tol > 0.0) && (fabs(SN - op->K) <= kink_tol * SN);
    res->xbar0 = 0.0;
    res->vtot = 0.0;
    res->rho = 0.0;
    res->dvdt = 0.0;
    res->amp = 0.0;
    /* an imposed payoff decision other than the oracle's own: only at the strike */
    const int forced = orc_forced_itm(dec, path);
    const int own_itm = itm > 0.0;
    if (forced >= 0 && forced != own_itm) {
        if (!(fabs(SN - op->K) <= band * op->K)) return ORC_EDECISION;
        ov[1] += 1;
    }
    if (!want_greeks) return ORC_OK;

    /* reverse sweep over the stored trajectory (back-propagation, Sec. IV-C) */
    const int in_money = forced >= 0 ? forced : own_itm;
    /* xbar = d V / d x_n: x = ln S, or S under ORC_SCHEME_X */
    double xbar = in_money ? disc * (double)op->phi * (on_x ? 1.0 : SN) : 0.0;
    double vtot = 0.0;
    /* the discount's share: d e^{-rT} / d r = -T e^{-rT}, d e^{-rT} / d T = -r e^{-rT} */
    double rho = -op->T * res->V;
    double dvdt = -op->r * res->V;
    double amp = 0.0;
    for (int32_t n = N - 1; n >= 0; --n) {
        double t = (double)n * dt;
        double S = on_x ? x[n] : exp(x[n]);
        st = orc_sigma_decided(sf, S, t, orc_forced_cell(dec, c_first, c_last, n), band, &pt, &overridden);
        if (st != ORC_OK) return st;
        /* d x_{n+1} / d sigma_n */
        double h = on_x ? x[n] * sqdt * z[n] : sqdt * z[n] - pt.sigma * dt;
        double sbar = xbar * h;                     /* adjoint of sigma_n */
        int32_t nodes[4] = { pt.i * J + pt.j, (pt.i + 1) * J + pt.j,
                             pt.i * J + pt.j + 1, (pt.i + 1) * J + pt.j + 1 };
        int n_corners = (J > 1) ? 4 : 2;
        for (int c = 0; c < n_corners; ++c) {
            double contrib = sbar * pt.w[c];
            vega[nodes[c]] += contrib;
            if (res->kink) kink_vega[nodes[c]] += fabs(contrib);
            vtot += contrib;
        }
        /* explicit dependence of x_{n+1} on r and on T (through dt = T / N and
         * t_n = n T / N); xbar is still xbar_{n+1} here */
        double dx_dr, dx_ddt;
        if (on_x) {
            dx_dr = x[n] * dt;
            dx_ddt = op->r * x[n] + pt.sigma * x[n] * z[n] / (2.0 * sqdt);
        } else {
            dx_dr = dt;
            dx_ddt = (op->r - 0.5 * pt.sigma * pt.sigma) + pt.sigma * z[n] / (2.0 * sqdt);
        }
        rho += xbar * dx_dr;
        dvdt += xbar * (dx_ddt / (double)N + h * pt.dsigma_dt * (double)n / (double)N);
        /* d x_{n+1} / d x_n: 1 + h S d sigma/d S on ln S (d sigma/d x = S d sigma/d S);
         * 1 + r dt + sigma sqrt(dt) Z + h d sigma/d S on S */
        double factor;
        if (on_x)
            factor = 1.0 + op->r * dt + pt.sigma * sqdt * z[n] + h * pt.dsigma_dS;
        else
            factor = 1.0 + h * S * pt.dsigma_dS;
        xbar = xbar * factor;
        /* sensitivity of ln |factor| to a relative change e of S_n within the cell
         * (d sigma / d S is constant there): on ln S, d g = (g - k^2 dt) e, with the
         * ln-S weight -k^2 dt e; on S, 2 sqrt(dt) Z k e; the sum bounds all three */
        const double kappa = S * pt.dsigma_dS;
        amp += (fabs(factor - 1.0) + kappa * kappa * dt + 2.0 * sqdt * fabs(z[n] * kappa)) / fabs(factor);
    }
    /* d V / d ln S0 in both cases (= S0 d V / d S0) */
    res->xbar0 = on_x ? xbar * op->S0 : xbar;
    res->vtot = vtot;
    res->rho = rho;
    res->dvdt = dvdt;
    res->amp = amp;
    return ORC_OK;
}

/* ----------------------------------------------------------- path ranges */

typedef struct {
    const orc_surface* sf;
    const orc_option* op;
    int64_t begin, end;
    int want_greeks;
    double kink_tol;
    const orc_decisions* dec;
    double* out;     /* ORC_NSCAL + 2 I J */
    int64_t ov[2];   /* applied decisions that differed from the oracle's own */
    int status;
} orc_job;

static void* orc_job_run(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    const int64_t IJ = (int64_t)jb->sf->n_spot * jb->sf->n_time;
    double* out = jb->out;
    double* vega = out + ORC_NSCAL;
    double* kink_vega = vega + IJ;
    orc_workspace ws;
    ws.x = (double*)malloc(sizeof(double) * (size_t)(jb->op->n_steps + 1));
    ws.z = (double*)malloc(sizeof(double) * (size_t)jb->op->n_steps);
    if (!ws.x || !ws.z) {
        free(ws.x); free(ws.z);
        jb->status = ORC_ENOMEM;
        return NULL;
    }
    jb->status = ORC_OK;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        orc_path_result res;
        const int st = orc_one_path(jb->sf, jb->op, (uint64_t)p, &ws, jb->want_greeks, jb->kink_tol, jb->dec,
                                    vega, kink_vega, &res, jb->ov);
        if (st != ORC_OK) {
            jb->status = st;
            break;
        }
        out[ORC_SUM_V] += res.V;
        out[ORC_SUM_V2] += res.V * res.V;
        out[ORC_SUM_XBAR0] += res.xbar0;
        out[ORC_SUM_XBAR0_2] += res.xbar0 * res.xbar0;
        out[ORC_SUM_VTOT] += res.vtot;
        out[ORC_SUM_VTOT_2] += res.vtot * res.vtot;
        out[ORC_SUM_SN] += res.SN;
        out[ORC_SUM_RHO] += res.rho;
        out[ORC_SUM_RHO_2] += res.rho * res.rho;
        out[ORC_SUM_DVDT] += res.dvdt;
        out[ORC_SUM_DVDT_2] += res.dvdt * res.dvdt;
        if (res.kink) {
            out[ORC_KINK_COUNT] += 1.0;
            out[ORC_KINK_XBAR0] += fabs(res.xbar0);
        }
    }
    free(ws.x);
    free(ws.z);
    return NULL;
}

static int orc_check(const orc_surface* sf, const orc_option* op)
{
    if (!sf || !op || !sf->spot || !sf->time || !sf->sigma) return ORC_EINVAL;
    if (sf->n_spot < 2 || sf->n_time < 1 || op->n_steps < 1 || !(op->T > 0.0) || !(op->S0 > 0.0))
        return ORC_EINVAL;
    if (op->phi != 1 && op->phi != -1) return ORC_EINVAL;
    if (sf->interp != ORC_INTERP_S && sf->interp != ORC_INTERP_LOGS) return ORC_EINVAL;
    if (op->scheme != ORC_SCHEME_LOG && op->scheme != ORC_SCHEME_X) return ORC_EINVAL;
    if (sf->interp == ORC_INTERP_LOGS && !(sf->spot[0] > 0.0)) return ORC_EINVAL;
    return ORC_OK;
}

int orc_run(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t path_end,
            int want_greeks, double kink_tol, int32_t n_threads, double* out)
{
    return orc_run_ex(sf, op, path_begin, path_end, want_greeks, kink_tol, NULL, n_threads, out);
}

static int orc_check_decisions(const orc_decisions* d)
{
    if (!d) return ORC_OK;
    if (!(d->band >= 0.0)) return ORC_EINVAL;
    for (int64_t e = 0; e < d->n_cell; ++e)
        if (d->cell_code[e] < 0 || d->cell_step[e] < 0) return ORC_EINVAL;
    for (int64_t e = 1; e < d->n_itm; ++e)
        if (d->itm_path[e] <= d->itm_path[e - 1]) return ORC_EINVAL;
    for (int64_t e = 1; e < d->n_cell; ++e)
        if (d->cell_path[e] < d->cell_path[e - 1] ||
            (d->cell_path[e] == d->cell_path[e - 1] && d->cell_step[e] <= d->cell_step[e - 1]))
            return ORC_EINVAL;
    return ORC_OK;
}

int orc_run_ex(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t path_end,
               int want_greeks, double kink_tol, const orc_decisions* dec, int32_t n_threads,
               double* out)
{
    if (orc_check_decisions(dec) != ORC_OK) return ORC_EINVAL;
    int st = orc_check(sf, op);
    if (st != ORC_OK) return st;
    if (path_begin < 0 || path_end < path_begin || !out) return ORC_EINVAL;
    const int64_t IJ = (int64_t)sf->n_spot * sf->n_time;
    const int64_t width = ORC_NSCAL + 2 * IJ;
    memset(out, 0, sizeof(double) * (size_t)width);
    int64_t P = path_end - path_begin;
    if (P == 0) return ORC_OK;
    if (n_threads < 1) n_threads = 1;
    if ((int64_t)n_threads > P) n_threads = (int32_t)P;

    orc_job* jobs = (orc_job*)calloc((size_t)n_threads, sizeof(orc_job));
    double* parts = (double*)calloc((size_t)(n_threads * width), sizeof(double));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !parts || !th) {
        free(jobs); free(parts); free(th);
        return ORC_ENOMEM;
    }
    for (int32_t k = 0; k < n_threads; ++k) {
        jobs[k].sf = sf;
        jobs[k].op = op;
        jobs[k].begin = path_begin + P * k / n_threads;
        jobs[k].end = path_begin + P * (k + 1) / n_threads;
        jobs[k].want_greeks = want_greeks;
        jobs[k].kink_tol = kink_tol;
        jobs[k].dec = dec;
        jobs[k].out = parts + (int64_t)k * width;
        jobs[k].status = ORC_EINTERNAL;
    }
    int started = 0;
    for (int32_t k = 1; k < n_threads; ++k) {
        if (pthread_create(&th[k], NULL, orc_job_run, &jobs[k]) != 0) break;
        started = k;
    }
    orc_job_run(&jobs[0]);
    for (int32_t k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    for (int32_t k = started + 1; k < n_threads; ++k) orc_job_run(&jobs[k]);

    st = ORC_OK;
    int64_t ov[2] = { 0, 0 };
    for (int32_t k = 0; k < n_threads; ++k) {     /* fixed order: range 0 first */
        if (jobs[k].status != ORC_OK) st = jobs[k].status;
        for (int64_t e = 0; e < width; ++e) out[e] += jobs[k].out[e];
        ov[0] += jobs[k].ov[0];
        ov[1] += jobs[k].ov[1];
    }
    if (dec && dec->out_overrides) {
        dec->out_overrides[0] = ov[0];
        dec->out_overrides[1] = ov[1];
    }
    free(jobs); free(parts); free(th);
    return st;
}

int orc_finalize(const double* sums, int64_t n_paths, double S0, int64_t IJ, double* res)
{
    if (n_paths < 1 || !sums || !res) return ORC_EINVAL;
    const double P = (double)n_paths;
    const double mean = sums[ORC_SUM_V] / P;
    double var = 0.0;
    if (n_paths > 1) var = (sums[ORC_SUM_V2] / P - mean * mean) * P / (P - 1.0);
    res[0] = mean;                                   /* price */
    res[1] = sums[ORC_SUM_XBAR0] / (P * S0);         /* delta = E[xbar_0] / S0 */
    res[2] = var > 0.0 ? sqrt(var / P) : 0.0;        /* standard error of the price */
    for (int64_t e = 0; e < IJ; ++e) res[3 + e] = sums[ORC_NSCAL + e] / P;
    return ORC_OK;
}

typedef struct {
    const orc_surface* sf;
    const orc_option* op;
    const orc_decisions* dec;
    int64_t first, begin, end;    /* paths [begin, end) written at index p - first */
    double *xN, *V, *xbar0, *amp;
    int64_t ov[2];                /* applied decisions that differed from the oracle's own */
    int status;
} orc_path_job;

static void* orc_path_job_run(void* arg)
{
    orc_path_job* jb = (orc_path_job*)arg;
    const int64_t IJ = (int64_t)jb->sf->n_spot * jb->sf->n_time;
    orc_workspace ws;
    ws.x = (double*)malloc(sizeof(double) * (size_t)(jb->op->n_steps + 1));
    ws.z = (double*)malloc(sizeof(double) * (size_t)jb->op->n_steps);
    double* vega = (double*)calloc((size_t)(2 * IJ), sizeof(double));
    if (!ws.x || !ws.z || !vega) {
        free(ws.x); free(ws.z); free(vega);
        jb->status = ORC_ENOMEM;
        return NULL;
    }
    jb->status = ORC_OK;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        orc_path_result res;
        const int st = orc_one_path(jb->sf, jb->op, (uint64_t)p, &ws, 1, 0.0, jb->dec, vega, vega + IJ, &res, jb->ov);
        if (st != ORC_OK) {
            jb->status = st;
            break;
        }
        const int64_t q = p - jb->first;
        /* ln S_N under either scheme */
        if (jb->xN)
            jb->xN[q] = jb->op->scheme == ORC_SCHEME_X ? log(ws.x[jb->op->n_steps]) : ws.x[jb->op->n_steps];
        if (jb->V) jb->V[q] = res.V;
        if (jb->xbar0) jb->xbar0[q] = res.xbar0;
        if (jb->amp) jb->amp[q] = res.amp;
    }
    free(ws.x); free(ws.z); free(vega);
    return NULL;
}

int orc_paths(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t m,
              int32_t n_threads, double* out_xN, double* out_V, double* out_xbar0)
{
    return orc_paths_ex(sf, op, path_begin, m, NULL, n_threads, out_xN, out_V, out_xbar0, NULL);
}

int orc_paths_ex(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t m,
                 const orc_decisions* dec, int32_t n_threads, double* out_xN, double* out_V,
                 double* out_xbar0, double* out_amp)
{
    int st = orc_check(sf, op);
    if (st != ORC_OK) return st;
    if (orc_check_decisions(dec) != ORC_OK) return ORC_EINVAL;
    if (path_begin < 0 || m < 0) return ORC_EINVAL;
    if (m == 0) return ORC_OK;
    if (n_threads < 1) n_threads = 1;
    if ((int64_t)n_threads > m) n_threads = (int32_t)m;
    orc_path_job* jobs = (orc_path_job*)calloc((size_t)n_threads, sizeof(orc_path_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs); free(th);
        return ORC_ENOMEM;
    }
    for (int32_t k = 0; k < n_threads; ++k) {
        jobs[k].sf = sf;
        jobs[k].op = op;
        jobs[k].dec = dec;
        jobs[k].first = path_begin;
        jobs[k].begin = path_begin + m * k / n_threads;
        jobs[k].end = path_begin + m * (k + 1) / n_threads;
        jobs[k].xN = out_xN;
        jobs[k].V = out_V;
        jobs[k].xbar0 = out_xbar0;
        jobs[k].amp = out_amp;
        jobs[k].status = ORC_EINTERNAL;
    }
    int started = 0;
    for (int32_t k = 1; k < n_threads; ++k) {
        if (pthread_create(&th[k], NULL, orc_path_job_run, &jobs[k]) != 0) break;
        started = k;
    }
    orc_path_job_run(&jobs[0]);
    for (int32_t k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    for (int32_t k = started + 1; k < n_threads; ++k) orc_path_job_run(&jobs[k]);
    st = ORC_OK;
    int64_t ov[2] = { 0, 0 };
    for (int32_t k = 0; k < n_threads; ++k) {
        if (jobs[k].status != ORC_OK) st = jobs[k].status;
        ov[0] += jobs[k].ov[0];
        ov[1] += jobs[k].ov[1];
    }
    if (dec && dec->out_overrides) {
        dec->out_overrides[0] = ov[0];
        dec->out_overrides[1] = ov[1];
    }
    free(jobs); free(th);
    return st;
}

/* --------------------------------------------------------- bump and reprice */

static int orc_price_only(const orc_surface* sf, const orc_option* op, int64_t n_paths,
                          int32_t n_threads, double* sum_V)
{
    const int64_t IJ = (int64_t)sf->n_spot * sf->n_time;
    double* out = (double*)malloc(sizeof(double) * (size_t)(ORC_NSCAL + 2 * IJ));
    if (!out) return ORC_ENOMEM;
    int st = orc_run(sf, op, 0, n_paths, 0, 0.0, n_threads, out);
    *sum_V = out[ORC_SUM_V];
    free(out);
    return st;
}

int orc_bump(const orc_surface* sf, const orc_option* op, int64_t n_paths, double eps_sigma,
             double eps_S0, int32_t n_threads, double* out_vega, double* out_delta)
{
    int st = orc_check(sf, op);
    if (st != ORC_OK) return st;
    if (n_paths < 1 || !(eps_sigma > 0.0) || !(eps_S0 > 0.0)) return ORC_EINVAL;
    const int64_t IJ = (int64_t)sf->n_spot * sf->n_time;
    const double P = (double)n_paths;
    double* bumped = (double*)malloc(sizeof(double) * (size_t)IJ);
    if (!bumped) return ORC_ENOMEM;
    memcpy(bumped, sf->sigma, sizeof(double) * (size_t)IJ);
    orc_surface bs = *sf;
    bs.sigma = bumped;

    /* one central difference per grid value, same seed for both sides (CRN), Sec. III */
    for (int64_t e = 0; e < IJ && st == ORC_OK; ++e) {
        double up = 0.0, dn = 0.0;
        bumped[e] = sf->sigma[e] + 0.5 * eps_sigma;
        st = orc_price_only(&bs, op, n_paths, n_threads, &up);
        bumped[e] = sf->sigma[e] - 0.5 * eps_sigma;
        if (st == ORC_OK) st = orc_price_only(&bs, op, n_paths, n_threads, &dn);
        bumped[e] = sf->sigma[e];
        out_vega[e] = (up - dn) / (P * eps_sigma);
    }
    if (st == ORC_OK) {
        orc_option o2 = *op;
        double up = 0.0, dn = 0.0;
        o2.S0 = op->S0 + 0.5 * eps_S0;
        st = orc_price_only(sf, &o2, n_paths, n_threads, &up);
        o2.S0 = op->S0 - 0.5 * eps_S0;
        if (st == ORC_OK) st = orc_price_only(sf, &o2, n_paths, n_threads, &dn);
        *out_delta = (up - dn) / (P * eps_S0);
    }
    free(bumped);
    return st;
}

/* ------------------------------------------------ second-order buckets */

/* Vanna buckets d^2 price / (d S0 d sigma_ij): the derivative of the delta
 * with respect to every grid value, an extension of the first-order Greeks
 * of Sec. V. The pathwise estimator of the delta,
 *   Delta_p = e^{-rT} 1{phi (S_N - K) > 0} phi S_N D_N / S0,
 *   D_N = prod_n (1 + g_n), g_n = h_n k_n, h_n = sqrt(dt) Z_n - sigma_n dt,
 *   k_n = S_n d sigma / d S (S_n, t_n),
 * is unbiased for the delta, but it jumps where S_N crosses the strike and
 * where a spot crosses a node (d sigma / d S changes cell there), so its own
 * pathwise derivative in sigma_ij would miss those jumps. Written as an
 * integral over the path x = (x_0 .. x_N) against the density p(x) of the
 * Euler chain, E[Delta_p] = int Delta_p(x; sigma) p(x; sigma) dx, and with
 * the path held fixed the indicator and every cell are fixed, so
 *   vanna_ij = E[ d Delta_p / d sigma_ij |_x + Delta_p d ln p(x) / d sigma_ij ].
 * Per step, with w_ij(n) node ij's bilinear weight and at fixed x
 *   d sigma_n / d sigma_ij = w_ij(n),
 *   d k_n / d sigma_ij = S_n d w_ij / d S (n) (inside the grid, else 0),
 *   d h_n / d sigma_n = -sqrt(dt) Z_n / sigma_n
 *     (h_n = (x_{n+1} - x_n - r dt) / sigma_n - sigma_n dt / 2 at fixed x),
 *   d ln p_n / d sigma_n = (Z_n^2 - 1) / sigma_n - sqrt(dt) Z_n
 *     (the Gaussian step, mean x_n + (r - sigma_n^2/2) dt, sd sigma_n sqrt(dt)),
 * so path p adds to bucket ij
 *   Delta_p sum_n [ w_ij(n) a_n + S_n d w_ij / d S (n) b_n ],
 *   a_n = (Z_n^2 - 1) / sigma_n - sqrt(dt) Z_n (1 + k_n / (sigma_n (1 + g_n))),
 *   b_n = h_n / (1 + g_n). */
static int orc_vanna_path(const orc_surface* sf, const orc_option* op, uint64_t path, orc_workspace* ws,
                          const orc_decisions* dec, double* vsum, double* vsq, double* pv, int32_t* touched,
                          double* scal, int64_t ov[2])
{
    const int32_t N = op->n_steps, J = sf->n_time;
    const double dt = op->T / (double)N;
    const double sqdt = sqrt(dt);
    double* x = ws->x;
    double* z = ws->z;
    orc_point pt;
    orc_normals(op->seed, op->stream_id, path, N, z);
    int64_t c_first, c_last;
    orc_cell_range(dec, path, &c_first, &c_last);
    const double band = dec ? dec->band : 0.0;
    int overridden, st;

    /* the path and D_N */
    x[0] = log(op->S0);
    double D = 1.0;
    int tiny = 0;
    for (int32_t n = 0; n < N; ++n) {
        const double t = (double)n * dt, S = exp(x[n]);
        st = orc_sigma_decided(sf, S, t, orc_forced_cell(dec, c_first, c_last, n), band, &pt, &overridden);
        if (st != ORC_OK) return st;
        ov[0] += overridden;
        const double h = sqdt * z[n] - pt.sigma * dt;
        const double f = 1.0 + h * S * pt.dsigma_dS;
        if (fabs(f) < 0x1p-40) tiny = 1;
        D = D * f;
        x[n + 1] = x[n] + (op->r - 0.5 * pt.sigma * pt.sigma) * dt + pt.sigma * sqdt * z[n];
    }
    const double SN = exp(x[N]);
    const double itm = (double)op->phi * (SN - op->K);
    const int forced = orc_forced_itm(dec, path);
    const int own_itm = itm > 0.0;
    if (forced >= 0 && forced != own_itm) {
        if (!(fabs(SN - op->K) <= band * op->K)) return ORC_EDECISION;
        ov[1] += 1;
    }
    const int in_money = forced >= 0 ? forced : own_itm;
    const double delta = in_money ? exp(-op->r * op->T) * (double)op->phi * SN * D / op->S0 : 0.0;
    scal[ORC_VN_DELTA] += delta;
    scal[ORC_VN_DELTA_2] += delta * delta;
    if (delta == 0.0) return ORC_OK;
    if (tiny) {
        scal[ORC_VN_TINY] += 1.0;
        return ORC_OK;
    }
    /* the path's bucket values, then their sums and squares */
    int32_t n_touched = 0;
    double tot = 0.0;
    for (int32_t n = 0; n < N; ++n) {
        const double t = (double)n * dt, S = exp(x[n]);
        st = orc_sigma_decided(sf, S, t, orc_forced_cell(dec, c_first, c_last, n), band, &pt, &overridden);
        if (st != ORC_OK) return st;
        const double kappa = S * pt.dsigma_dS;
        const double h = sqdt * z[n] - pt.sigma * dt;
        const double f = 1.0 + h * kappa;
        const double a = (z[n] * z[n] - 1.0) / pt.sigma - sqdt * z[n] * (1.0 + kappa / (pt.sigma * f));
        const double b = h / f;
        /* d w / d S of the corners (i, j), (i+1, j), (i, j+1), (i+1, j+1) */
        const double v = pt.v;
        const double dw[4] = { -(1.0 - v) * pt.du_dS, (1.0 - v) * pt.du_dS, -v * pt.du_dS, v * pt.du_dS };
        const int32_t nodes[4] = { pt.i * J + pt.j, (pt.i + 1) * J + pt.j, pt.i * J + pt.j + 1,
                                   (pt.i + 1) * J + pt.j + 1 };
        const int n_corners = (J > 1) ? 4 : 2;
        for (int c = 0; c < n_corners; ++c) {
            const double contrib = delta * (pt.w[c] * a + S * dw[c] * b);
            if (pv[nodes[c]] == 0.0 && contrib != 0.0) touched[n_touched++] = nodes[c];
            pv[nodes[c]] += contrib;
            tot += contrib;
        }
    }
    for (int32_t e = 0; e < n_touched; ++e) {
        const int32_t node = touched[e];
        vsum[node] += pv[node];
        vsq[node] += pv[node] * pv[node];
        pv[node] = 0.0;
    }
    scal[ORC_VN_TOT] += tot;
    scal[ORC_VN_TOT_2] += tot * tot;
    return ORC_OK;
}

typedef struct {
    const orc_surface* sf;
    const orc_option* op;
    const orc_decisions* dec;
    int64_t begin, end;
    double* out;       /* ORC_VN_NSCAL + 2 I J */
    int64_t ov[2];
    int status;
} orc_vanna_job;

static void* orc_vanna_job_run(void* arg)
{
    orc_vanna_job* jb = (orc_vanna_job*)arg;
    const int64_t IJ = (int64_t)jb->sf->n_spot * jb->sf->n_time;
    orc_workspace ws;
    ws.x = (double*)malloc(sizeof(double) * (size_t)(jb->op->n_steps + 1));
    ws.z = (double*)malloc(sizeof(double) * (size_t)jb->op->n_steps);
    double* pv = (double*)calloc((size_t)IJ, sizeof(double));
    /* a path touches at most 4 nodes a step; a node may be counted more than once
     * only when its running value returned to exactly 0 */
    int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(4 * jb->op->n_steps + IJ));
    if (!ws.x || !ws.z || !pv || !touched) {
        free(ws.x); free(ws.z); free(pv); free(touched);
        jb->status = ORC_ENOMEM;
        return NULL;
    }
    jb->status = ORC_OK;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        const int st = orc_vanna_path(jb->sf, jb->op, (uint64_t)p, &ws, jb->dec, jb->out + ORC_VN_NSCAL,
                                      jb->out + ORC_VN_NSCAL + IJ, pv, touched, jb->out, jb->ov);
        if (st != ORC_OK) {
            jb->status = st;
            break;
        }
    }
    free(ws.x); free(ws.z); free(pv); free(touched);
    return NULL;
}

int orc_run_vanna(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t path_end,
                  const orc_decisions* dec, int32_t n_threads, double* out)
{
    if (orc_check_decisions(dec) != ORC_OK) return ORC_EINVAL;
    int st = orc_check(sf, op);
    if (st != ORC_OK) return st;
    if (sf->interp != ORC_INTERP_S || op->scheme != ORC_SCHEME_LOG) return ORC_EINVAL;
    if (path_begin < 0 || path_end < path_begin || !out) return ORC_EINVAL;
    const int64_t IJ = (int64_t)sf->n_spot * sf->n_time;
    const int64_t width = ORC_VN_NSCAL + 2 * IJ;
    memset(out, 0, sizeof(double) * (size_t)width);
    const int64_t P = path_end - path_begin;
    if (P == 0) return ORC_OK;
    if (n_threads < 1) n_threads = 1;
    if ((int64_t)n_threads > P) n_threads = (int32_t)P;
    orc_vanna_job* jobs = (orc_vanna_job*)calloc((size_t)n_threads, sizeof(orc_vanna_job));
    double* parts = (double*)calloc((size_t)(n_threads * width), sizeof(double));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !parts || !th) {
        free(jobs); free(parts); free(th);
        return ORC_ENOMEM;
    }
    for (int32_t k = 0; k < n_threads; ++k) {
        jobs[k].sf = sf;
        jobs[k].op = op;
        jobs[k].dec = dec;
        jobs[k].begin = path_begin + P * k / n_threads;
        jobs[k].end = path_begin + P * (k + 1) / n_threads;
        jobs[k].out = parts + (int64_t)k * width;
        jobs[k].status = ORC_EINTERNAL;
    }
    int started = 0;
    for (int32_t k = 1; k < n_threads; ++k) {
        if (pthread_create(&th[k], NULL, orc_vanna_job_run, &jobs[k]) != 0) break;
        started = k;
    }
    orc_vanna_job_run(&jobs[0]);
    for (int32_t k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    for (int32_t k = started + 1; k < n_threads; ++k) orc_vanna_job_run(&jobs[k]);
    st = ORC_OK;
    int64_t ov[2] = { 0, 0 };
    for (int32_t k = 0; k < n_threads; ++k) {     /* fixed order */
        if (jobs[k].status != ORC_OK) st = jobs[k].status;
        for (int64_t e = 0; e < width; ++e) out[e] += jobs[k].out[e];
        ov[0] += jobs[k].ov[0];
        ov[1] += jobs[k].ov[1];
    }
    if (dec && dec->out_overrides) {
        dec->out_overrides[0] = ov[0];
        dec->out_overrides[1] = ov[1];
    }
    free(jobs); free(parts); free(th);
    return st;
}
