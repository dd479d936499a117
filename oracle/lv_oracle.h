/*
 * lv_oracle.h -- interface of the FP64 CPU oracle (test infrastructure
 * only; see lv_oracle.c). Independent of the CUDA library's header.
 */
#ifndef LV_ORACLE_H
#define LV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ORC_EDECISION: an imposed decision (see orc_decisions) that rounding of
 * the path could not have produced. */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EINTERNAL = 4, ORC_EDECISION = 5 };

/* Layout of the sums array filled by orc_run: ORC_NSCAL scalars, then
 * vega[I*J] (sum of sigma adjoints per node, spot-major), then
 * kink_vega[I*J] (sum of |contribution| of paths in the payoff-kink band). */
enum {
    ORC_SUM_V = 0,        /* sum of discounted payoffs */
    ORC_SUM_V2 = 1,       /* sum of squared payoffs */
    ORC_SUM_XBAR0 = 2,    /* sum of d V / d x_0, x_0 = ln S0 (= S0 d V / d S0 under either scheme) */
    ORC_SUM_XBAR0_2 = 3,  /* sum of squares of the above */
    ORC_SUM_VTOT = 4,     /* sum over paths of (sum over nodes of the path's vega) */
    ORC_SUM_VTOT_2 = 5,   /* sum of squares of the above */
    ORC_SUM_SN = 6,       /* sum of terminal spots */
    ORC_KINK_COUNT = 7,   /* paths with |S_N - K| <= kink_tol * S_N */
    ORC_KINK_XBAR0 = 8,   /* sum of |d V / d x_0| over those paths */
    ORC_SUM_RHO = 9,      /* sum of d V / d r (pathwise, discount included) */
    ORC_SUM_RHO_2 = 10,
    ORC_SUM_DVDT = 11,    /* sum of d V / d T (maturity, n_steps fixed, surface fixed in time) */
    ORC_SUM_DVDT_2 = 12,
    ORC_NSCAL = 13
};

/* Interpolation in spot between the nodes of a cell (Sec. IV-D reads as
 * bilinear; the coordinate is open): linear in S or linear in ln S. */
enum { ORC_INTERP_S = 0, ORC_INTERP_LOGS = 1 };
/* Euler scheme (Sec. IV-A): on x = ln X (drift r - sigma^2/2) or on X
 * itself (X_{n+1} = X_n + r X_n dt + sigma_n X_n sqrt(dt) Z_n). */
enum { ORC_SCHEME_LOG = 0, ORC_SCHEME_X = 1 };

typedef struct {
    int32_t n_spot;       /* I >= 2 */
    int32_t n_time;       /* J >= 1 */
    const double* spot;   /* [I], strictly increasing, > 0 */
    const double* time;   /* [J], strictly increasing */
    const double* sigma;  /* [I*J], sigma_ij at i*J + j */
    int32_t interp;       /* ORC_INTERP_* */
} orc_surface;

typedef struct {
    double S0, r, K, T;
    int32_t n_steps;
    int32_t phi;          /* +1 call, -1 put */
    uint64_t seed;
    uint32_t stream_id;
    int32_t scheme;       /* ORC_SCHEME_* */
} orc_option;

typedef struct {
    int32_t i, j;         /* cell */
    double u, v;          /* clamped weights in spot and time */
    double w[4];          /* node weights (i,j), (i+1,j), (i,j+1), (i+1,j+1) */
    double sigma;
    double dsigma_dS;
    double dsigma_dt;     /* 0 outside [t_0, t_{J-1}) and for one time node */
    int32_t inside;       /* S in [s_0, s_{I-1}] (the weights then move with S) */
    double du_dS;         /* d u / d S inside the grid, 0 outside */
} orc_point;

/* Decisions taken from outside for listed paths / steps (see lv_oracle.c):
 * payoff indicator per path; spot-cell code 2 i + inside per (path, step).
 * Both lists sorted ascending (by path, then step). A decision that differs
 * from the oracle's own is accepted only within `band` (relative) of the
 * value that separates the two choices: the strike, the node between two
 * adjacent cells, or the grid's edge node; any other is refused with
 * ORC_EDECISION. out_overrides (nullable, 2 entries) receives how many cell
 * decisions and how many payoff decisions of the call differed from the
 * oracle's own and were applied. */
typedef struct {
    const int64_t* itm_path;
    const int8_t* itm_val;
    int64_t n_itm;
    const int64_t* cell_path;
    const int32_t* cell_step;
    const int32_t* cell_code;
    int64_t n_cell;
    double band;
    int64_t* out_overrides;
} orc_decisions;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t w);
void orc_counter(uint32_t block, uint64_t path, uint32_t stream_id, uint32_t ctr[4]);
void orc_normals4(uint64_t seed, uint32_t stream_id, uint64_t path, uint32_t block, double z[4]);
void orc_normals(uint64_t seed, uint32_t stream_id, uint64_t path, int32_t n_steps, double* z);
void orc_sigma_eval(const orc_surface* sf, double S, double t, orc_point* p);

int orc_run(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t path_end,
            int want_greeks, double kink_tol, int32_t n_threads, double* out);
int orc_run_ex(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t path_end,
               int want_greeks, double kink_tol, const orc_decisions* dec, int32_t n_threads,
               double* out);
int orc_finalize(const double* sums, int64_t n_paths, double S0, int64_t IJ, double* res);
int orc_paths(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t m,
              int32_t n_threads, double* out_xN, double* out_V, double* out_xbar0);
/* out_amp (nullable): per path, the bound on d ln |xbar_0| / d e for a relative
 * error e in every spot of the path (see orc_path_result in lv_oracle.c). */
int orc_paths_ex(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t m,
                 const orc_decisions* dec, int32_t n_threads, double* out_xN, double* out_V,
                 double* out_xbar0, double* out_amp);
int orc_bump(const orc_surface* sf, const orc_option* op, int64_t n_paths, double eps_sigma,
             double eps_S0, int32_t n_threads, double* out_vega, double* out_delta);

/* Second-order bucket sensitivities d^2 price / (d S0 d sigma_ij) (see
 * lv_oracle.c), main reading only (ORC_INTERP_S, ORC_SCHEME_LOG; else
 * ORC_EINVAL). out [ORC_VN_NSCAL + 2 I J]: the scalars below, then the sum
 * over paths of each path's bucket value (spot-major), then the sum of
 * their squares (standard errors). Decisions as in orc_run_ex. */
enum {
    ORC_VN_DELTA = 0,     /* sum of the pathwise delta Delta_p */
    ORC_VN_DELTA_2 = 1,
    ORC_VN_TOT = 2,       /* sum over paths of the path's sum over buckets */
    ORC_VN_TOT_2 = 3,
    ORC_VN_TINY = 4,      /* live paths with |1 + g_n| < 2^-40 (their values are not finite) */
    ORC_VN_NSCAL = 5
};
int orc_run_vanna(const orc_surface* sf, const orc_option* op, int64_t path_begin, int64_t path_end,
                  const orc_decisions* dec, int32_t n_threads, double* out);

#ifdef __cplusplus
}
#endif
#endif
