// lv_api.cu -- host runtime behind the C ABI of include/lv.h: handle
// lifetime, argument validation, launch planning, scratch management and
// the host-output wrappers.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "lv.h"
#include "lv_internal.h"

namespace {

thread_local std::string g_last_error;

lv_status fail(lv_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

}  // namespace

lv_status lv::set_error(lv_status s, const std::string& msg) { return fail(s, msg); }

namespace {
std::mutex g_tune_mu;
}  // namespace

bool lv::tune_cache_lookup(const std::string& key, int vals[4])
{
    const char* path = std::getenv("LV_TUNE_CACHE");
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        char kbuf[512];
        int a = 0, b = 0, c = 0, d = 0;
        double ms = 0.0;
        if (std::sscanf(line, "%511s %d %d %d %d %lf", kbuf, &a, &b, &c, &d, &ms) == 6 && key == kbuf) {
            vals[0] = a;
            vals[1] = b;
            vals[2] = c;
            vals[3] = d;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void lv::tune_cache_append(const std::string& key, const int vals[4], double ms)
{
    const char* path = std::getenv("LV_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %.4f\n", key.c_str(), vals[0], vals[1], vals[2], vals[3], ms);
    std::fclose(f);
}

std::string lv::gpu_name(int device)
{
    // the property query costs tens of microseconds: once per device
    static std::mutex mu;
    static std::map<int, std::string> names;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = names.find(device);
    if (it != names.end()) return it->second;
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    std::string n(prop.name);
    for (char& ch : n)
        if (ch == ' ') ch = '_';
    names[device] = n;
    return n;
}

namespace {

#define LV_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(LV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

// Makes the handle's device current for the duration of a call and
// restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_finite(double a) { return std::isfinite(a); }

}  // namespace


namespace {

lv_status check_sigma(const double* sigma, int64_t n)
{
    if (!sigma) return fail(LV_EINVAL, "sigma is NULL");
    for (int64_t e = 0; e < n; ++e)
        if (!is_finite(sigma[e]) || !(sigma[e] > 0.0))
            return fail(LV_EINVAL, "sigma[" + std::to_string(e) + "] must be finite and > 0");
    return LV_OK;
}

// sigma (spot-major, binary64) -> time-major binary32 pairs per cell of a
// time row: (sigma_{i,j}, sigma_{i+1,j} - sigma_{i,j}), the difference taken
// in binary64; row 0 is repeated when the grid has a single time node.
void pack_sigma(const lv_surface_s* h, const double* sigma, float2* dst)
{
    for (int j = 0; j < h->Je; ++j) {
        const int jj = j < h->J ? j : h->J - 1;
        for (int i = 0; i + 1 < h->I; ++i) {
            const double a = sigma[(size_t)i * h->J + jj];
            const double b = sigma[(size_t)(i + 1) * h->J + jj];
            dst[(size_t)j * (h->I - 1) + i] = make_float2((float)a, (float)(b - a));
        }
    }
}

void free_surface(lv_surface_s* h)
{
    if (!h) return;
    cudaFree(h->d_sig);
    cudaFree(h->d_node);
    cudaFree(h->d_ab);
    cudaFree(h->d_abl);
    cudaFree(h->d_tau);
    cudaFree(h->d_spot64);
    cudaFree(h->d_sig64);
    cudaFreeHost(h->h_sig64_stage);
    cudaFree(h->d_scratch);
    cudaFree(h->d_res);
    cudaFreeHost(h->h_sig_stage);
    cudaFreeHost(h->h_res);
    delete h;
}

lv_status check_option(double S0, double r, double K, double T, int32_t n_steps)
{
    if (!is_finite(S0) || !(S0 > 0.0)) return fail(LV_EINVAL, "S0 must be finite and > 0");
    if (!is_finite(r)) return fail(LV_EINVAL, "r must be finite");
    if (!is_finite(K) || K < 0.0) return fail(LV_EINVAL, "K must be finite and >= 0");
    if (!is_finite(T) || !(T > 0.0)) return fail(LV_EINVAL, "T must be finite and > 0");
    if (n_steps < 1 || n_steps > LV_MAX_STEPS)
        return fail(LV_EINVAL, "n_steps must be in [1, LV_MAX_STEPS]");
    return LV_OK;
}

struct Plan {
    int block = 128, k = 4, bps = 1, grid = 1, ppl = 1;
    bool grid_smem = true;
    size_t smem = 0;
    int n_tiles = 0, n_ck = 0, row_words = 0, n_chunks = 0;
    size_t off_counter = 0, off_part = 0, off_chunks = 0, off_wrows = 0, off_l1 = 0, off_ckpt = 0, total = 0;
};

size_t round_up(size_t b, size_t a) { return (b + a - 1) / a * a; }

// The per-path diagnostics kernel always runs checkpoints every 4 steps with
// binary64 level 2 (per-path values do not depend on either).
std::string adjoint_tune_key(const lv_surface_s* h, int32_t n_steps)
{
    int nb = 0;
    for (int n = n_steps; n > 1; n >>= 1) ++nb;
    return std::string(h->adj_method == LV_ADJ_TANGENT ? "tangent|" : "adjoint|") + lv::gpu_name(h->device) + "|" + std::to_string(h->I) + "x" + std::to_string(h->J) +
           "|N2^" + std::to_string(nb);
}

// Shared memory a block may use and still leave room for the five resident
// blocks the register budget allows; larger grids are read through L1.
constexpr size_t kGridSmemLimit = 44 * 1024;

// extra: the adjoint kernel that also sums d V / d r and d V / d T (reverse
// sweep, binary64 level 2, k = 4 or 8).
// Blocks per SM of one kernel instantiation and launch shape, per device:
// the runtime's occupancy query costs microseconds, so each answer is kept.
using OccKey = std::tuple<int, int, int, bool, int, bool, bool, int, int, bool, size_t, int>;
std::mutex g_occ_mu;
std::map<OccKey, int> g_occ;

bool occ_lookup(const OccKey& key, int* occ)
{
    std::lock_guard<std::mutex> lock(g_occ_mu);
    const auto it = g_occ.find(key);
    if (it == g_occ.end()) return false;
    *occ = it->second;
    return true;
}

void occ_store(const OccKey& key, int occ)
{
    std::lock_guard<std::mutex> lock(g_occ_mu);
    g_occ[key] = occ;
}

// A call of at least this many paths per SM runs two paths per lane unless
// told otherwise: every warp of the adjoint kernel (at most 24 resident per
// SM) then gets at least four pairs of 32-path tiles. Smaller calls run one
// path per lane; measured on a GB300 (k = 4), two paths per lane took 1.03-1.07x
// the time at 2^18 and 2^19 paths and 0.96-0.99x from 2^20 on.
constexpr int64_t kPairMinPathsPerSm = 4 * 64 * 24;

// n_paths < 0: a call large enough for two paths per lane.
lv_status choose_launch(lv_surface_s* h, int32_t n_steps, bool greeks, int* block, int* k, int* bps,
                        bool dbg = false, bool* grid_smem = nullptr, bool extra = false, bool vanna = false,
                        int* ppl_out = nullptr, int64_t n_paths = -1)
{
    *block = h->cfg_block ? h->cfg_block : 128;
    *k = greeks ? (h->cfg_k ? h->cfg_k : 4) : 4;
    int ppl = h->cfg_ppl ? h->cfg_ppl : (n_paths < 0 || n_paths >= kPairMinPathsPerSm * h->num_sms ? 2 : 1);
    const char* cache = std::getenv("LV_TUNE_CACHE");
    if (greeks && !dbg && !h->cfg_block && !h->cfg_k && !h->cfg_ppl && cache && *cache) {
        int v[4];
        if (lv::tune_cache_lookup(adjoint_tune_key(h, n_steps), v) && v[0] >= 32 && v[0] <= 128 &&
            v[0] % 32 == 0 && (v[1] == 4 || v[1] == 8 || v[1] == 16 || v[1] == 32)) {
            *block = v[0];
            *k = v[1];
            ppl = v[2] == 2 ? 2 : 1;
        }
    }
    if (dbg) *k = 4;
    const int model = (h->interp == LV_INTERP_LOGS ? 1 : 0) | (h->scheme == LV_SCHEME_S ? 2 : 0);
    if ((model != 0 || extra) && *k > lv::kModelMaxK) *k = lv::kModelMaxK;
    // two paths per lane: the reverse sweep with checkpoints every 4 or 8 steps (every reading),
    // the main reading's tangent-ratio adjoint and its second-order buckets (no checkpoints)
    const bool pairs = greeks && !dbg && !extra &&
                       ((vanna || h->adj_method == LV_ADJ_TANGENT) ? model == 0 : (*k == 4 || *k == 8));
    if (!pairs) ppl = 1;
    if (ppl_out) *ppl_out = ppl;
    const bool gs = lv::mc_smem_bytes(h->I, h->Je, n_steps, *block, greeks, true, extra, ppl) <= kGridSmemLimit;
    if (grid_smem) *grid_smem = gs;
    const size_t smem = lv::mc_smem_bytes(h->I, h->Je, n_steps, *block, greeks, gs, extra, ppl);
    if (smem > 200 * 1024)
        return fail(LV_EINVAL, "time table does not fit in shared memory (" + std::to_string(smem) + " bytes)");
    int occ = 0;
    const int acc = dbg || extra || vanna ? 0 : h->acc_mode;
    const int method = vanna ? lv::kMethodVanna : (dbg || extra ? LV_ADJ_REVERSE : h->adj_method);
    const OccKey key{h->device, *block, *k, greeks, acc, dbg, gs, method, model, extra, smem, ppl};
    if (!occ_lookup(key, &occ)) {
        LV_CUDA(lv::mc_occupancy(*block, *k, greeks, acc, dbg, gs, method, model, extra, smem, &occ, ppl));
        occ_store(key, occ);
    }
    if (occ < 1) return fail(LV_EINVAL, "launch shape does not fit on an SM");
    *bps = h->cfg_bps ? (h->cfg_bps < occ ? h->cfg_bps : occ) : occ;
    return LV_OK;
}

lv_status make_plan(lv_surface_s* h, int32_t n_steps, int64_t n_paths, bool greeks, bool dbg, Plan* p,
                    bool extra = false, bool vanna = false)
{
    lv_status st = choose_launch(h, n_steps, greeks, &p->block, &p->k, &p->bps, dbg, &p->grid_smem, extra, vanna,
                                 &p->ppl, n_paths);
    if (st != LV_OK) return st;
    p->smem = lv::mc_smem_bytes(h->I, h->Je, n_steps, p->block, greeks, p->grid_smem, extra, p->ppl);
    const int warps = p->block / 32;
    const int64_t tiles = (n_paths + lv::paths_per_tile(greeks) - 1) / lv::paths_per_tile(greeks);   // claimed by warps
    p->n_tiles = (int)tiles;
    const int64_t want_blocks = (tiles + warps - 1) / warps;
    const int64_t slots = (int64_t)p->bps * h->num_sms;
    p->grid = (int)(want_blocks < slots ? want_blocks : slots);
    if (p->grid < 1) p->grid = 1;
    // the tangent-ratio adjoint and the second-order buckets keep no checkpoints
    const bool reverse = !vanna && (dbg || extra || h->adj_method == LV_ADJ_REVERSE);
    p->n_ck = greeks && reverse ? (n_steps + p->k - 1) / p->k : 0;
    const size_t nIJ = (size_t)h->Je * h->I;
    // price-only rows hold the scalars; extra rows end with the sums of d V / d r and d V / d T
    p->row_words = greeks ? 3 + (int)nIJ + (extra ? 2 : 0) : 3;
    p->n_chunks = lv::finalize_chunks(p->grid);
    const size_t total_warps = (size_t)p->grid * warps;
    size_t o = 0;
    p->off_counter = o; o += 256;
    p->off_part = o;    o = round_up(o + sizeof(double) * (size_t)p->grid * p->row_words, 256);
    p->off_chunks = o;  o = round_up(o + sizeof(double) * (size_t)p->n_chunks * p->row_words, 256);
    p->off_wrows = o;                   // per-warp rows: Kahan mode only
    if (greeks && !extra && !vanna && h->acc_mode == LV_ACC_KAHAN)
        o = round_up(o + sizeof(double) * total_warps * nIJ, 256);
    p->off_l1 = o;      if (greeks) o = round_up(o + sizeof(float) * (size_t)p->grid * nIJ, 256);
    p->off_ckpt = o;
    o = round_up(o + sizeof(float) * (size_t)p->n_ck * total_warps * lv::ring_slots_per_warp() * p->ppl, 256);
    p->total = o;
    return LV_OK;
}

lv_status ensure_scratch(lv_surface_s* h, size_t bytes)
{
    if (bytes <= h->scratch_bytes) return LV_OK;
    if (h->d_scratch) {
        LV_CUDA(cudaStreamSynchronize(h->stream));
        LV_CUDA(cudaFree(h->d_scratch));
        h->d_scratch = nullptr;
        h->scratch_bytes = 0;
    }
    const size_t want = round_up(bytes + bytes / 4, 1 << 20);
    if (cudaMalloc(&h->d_scratch, want) != cudaSuccess) {
        cudaGetLastError();
        h->d_scratch = nullptr;
        return fail(LV_ENOMEM, "cannot allocate " + std::to_string(want) + " bytes of scratch");
    }
    h->scratch_bytes = want;
    // the tile counter starts at zero; every finalize resets it
    LV_CUDA(cudaMemsetAsync(h->d_scratch, 0, 256, h->stream));
    return LV_OK;
}

struct McCall {
    double S0, r, K, T;
    int32_t n_steps;
    int64_t path_begin, n_paths;
    uint64_t seed;
    uint32_t stream_id;
    bool greeks;
    bool want_sums;
    double* d_out;           // [3 + I*J] device
    float* dbg_xN = nullptr;
    float* dbg_V = nullptr;
    float* dbg_xbar0 = nullptr;
    int* dbg_ev = nullptr;
    unsigned long long* dbg_ev_count = nullptr;
    int64_t dbg_ev_cap = 0;
    double dbg_band = 0.0;
    // set after brace initialisation, never positionally
    bool extra = false;      // also d V / d r and d V / d T (after the vegas)
    bool vanna = false;      // buckets are d^2 price / (d S0 d sigma_ij) instead of the vegas
};

lv::McParams base_params(const lv_surface_s* h, const McCall& c)
{
    lv::McParams P{};
    P.sig2 = h->d_sig;
    P.node = h->d_node;
    P.ab = h->interp == LV_INTERP_LOGS ? h->d_abl : h->d_ab;
    P.model = (h->interp == LV_INTERP_LOGS ? 1 : 0) | (h->scheme == LV_SCHEME_S ? 2 : 0);
    P.tau = h->d_tau;
    P.I = h->I;
    P.J = h->J;
    P.Je = h->Je;
    P.log_uniform = h->log_uniform;
    P.cell_scale = h->cell_scale;
    P.cell_shift = h->cell_shift;
    P.s_lo = h->s_lo;
    P.s_hi = h->s_hi;
    const double dt = c.T / (double)c.n_steps;
    const double log2e = 1.4426950408889634;
    const bool on_s = h->scheme == LV_SCHEME_S;
    P.x0 = (float)(on_s ? c.S0 : std::log2(c.S0));
    P.rdt = (float)(on_s ? c.r * dt : log2e * c.r * dt);
    P.S0f = (float)c.S0;
    P.inv_S0 = (float)(1.0 / c.S0);
    P.Tf = (float)c.T;
    P.r_nat = (float)c.r;
    P.inv_N = (float)(1.0 / c.n_steps);
    P.half_inv_sqdt = (float)(0.5 / std::sqrt(dt));
    P.hdt = (float)(log2e * 0.5 * dt);
    P.sqdt2 = (float)(log2e * std::sqrt(dt));
    P.dt = (float)dt;
    P.sqdt = (float)std::sqrt(dt);
    P.K = (float)c.K;
    P.disc = (float)std::exp(-c.r * c.T);
    P.phi = (float)h->phi;
    P.dt_d = dt;
    P.N = c.n_steps;
    P.k0 = (uint32_t)(c.seed & 0xffffffffu);
    P.k1 = (uint32_t)(c.seed >> 32);
    P.stream_id = c.stream_id;
    P.path_begin = c.path_begin;
    P.n_paths = c.n_paths;
    P.acc_mode = h->acc_mode;
    P.method = LV_ADJ_REVERSE;
    return P;
}

lv_status run_mc(lv_surface_s* h, const McCall& c)
{
    if (!c.d_out) return fail(LV_EINTERNAL, "no output buffer for the call");
    lv_status st = check_option(c.S0, c.r, c.K, c.T, c.n_steps);
    if (st != LV_OK) return st;
    if (c.n_paths < 1) return fail(LV_EINVAL, "the path range is empty");
    if (c.path_begin < 0 || c.path_begin + c.n_paths > LV_MAX_PATH_INDEX)
        return fail(LV_EINVAL, "path indices must lie in [0, 2^48)");
    if (c.stream_id >= 65536u) return fail(LV_EINVAL, "stream_id must be < 65536");
    if (c.n_paths > 0x7fffffffLL) return fail(LV_EINVAL, "one call handles at most 2^31 - 1 paths");
    if (c.vanna && (h->interp != LV_INTERP_S || h->scheme != LV_SCHEME_LOG))
        return fail(LV_EINVAL, "second-order buckets run the main reading (LV_INTERP_S, LV_SCHEME_LOG) only");
    Plan p;
    st = make_plan(h, c.n_steps, c.n_paths, c.greeks, c.dbg_xN != nullptr, &p, c.extra, c.vanna);
    if (st != LV_OK) return st;
    st = ensure_scratch(h, p.total);
    if (st != LV_OK) return st;
    char* base = static_cast<char*>(h->d_scratch);
    lv::McParams P = base_params(h, c);
    P.n_tiles = p.n_tiles;
    P.ppl = p.ppl;
    P.tile_counter = reinterpret_cast<unsigned int*>(base + p.off_counter);
    P.partials = reinterpret_cast<double*>(base + p.off_part);
    P.row_words = p.row_words;
    P.warp_rows = reinterpret_cast<double*>(base + p.off_wrows);
    P.l1 = reinterpret_cast<float*>(base + p.off_l1);
    P.ckpt = reinterpret_cast<float*>(base + p.off_ckpt);
    P.n_ck = p.n_ck;
    P.flush_every = 8;
    P.grid_smem = p.grid_smem ? 1 : 0;
    P.dbg_xN = c.dbg_xN;
    P.dbg_V = c.dbg_V;
    P.dbg_xbar0 = c.dbg_xbar0;
    P.dbg_ev = c.dbg_ev;
    P.dbg_ev_count = c.dbg_ev_count;
    P.dbg_ev_cap = c.dbg_ev_cap;
    P.dbg_band = (float)c.dbg_band;
    if (c.extra) {                        // reverse sweep, binary64 level 2
        P.extra = 1;
        P.acc_mode = 0;
    }
    if (c.greeks && !c.dbg_xN && !c.extra && h->adj_method == LV_ADJ_TANGENT) {
        P.method = LV_ADJ_TANGENT;
        P.flag = P.tile_counter + 1;      // in the zeroed counter section; the finalize resets it
    }
    if (c.vanna) {                        // two forward passes, binary64 level 2, the same flag
        P.method = lv::kMethodVanna;
        P.acc_mode = 0;
        P.flag = P.tile_counter + 1;
    }
    if (h->ev_start) LV_CUDA(cudaEventRecord(h->ev_start, h->stream));
    LV_CUDA(lv::launch_mc(P, p.grid, p.block, p.k, c.greeks, p.smem, h->stream));
    if (h->ev_end) LV_CUDA(cudaEventRecord(h->ev_end, h->stream));
    lv::FinalizeParams F{};
    F.partials = P.partials;
    F.G = p.grid;
    F.row_words = p.row_words;
    F.I = h->I;
    F.J = h->J;
    F.n_paths = c.n_paths;
    F.S0 = c.S0;
    F.want_sums = c.want_sums ? 1 : 0;
    F.chunks = reinterpret_cast<double*>(base + p.off_chunks);
    F.out = c.d_out;
    F.tile_counter = P.tile_counter;
    F.flag = P.flag;
    F.extra = c.extra ? 1 : 0;
    LV_CUDA(lv::launch_finalize(F, h->stream));
    return LV_OK;
}

// Brings the binary64 sigma on the device up to the last lv_surface_set_sigma
// (stream-ordered before the caller's launches).
lv_status sigma64_current(lv_surface_s* h)
{
    if (h->sig64_stale) {
        LV_CUDA(cudaMemcpyAsync(h->d_sig64, h->h_sig64_stage, sizeof(double) * (size_t)h->I * h->J,
                                cudaMemcpyHostToDevice, h->stream));
        h->sig64_stale = false;
    }
    return LV_OK;
}

lv_status fetch_result(lv_surface_s* h, bool extra = false)
{
    const size_t n = 3 + (size_t)h->I * h->J + (extra ? 2 : 0);
    LV_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    LV_CUDA(cudaStreamSynchronize(h->stream));
    return LV_OK;
}

}  // namespace

extern "C" {

const char* lv_last_error(void) { return g_last_error.c_str(); }

lv_status lv_surface_create(const double* spot_nodes, int32_t n_spot, const double* time_nodes,
                            int32_t n_time, const double* sigma, lv_surface_t* out)
{
    if (!out) return fail(LV_EINVAL, "out is NULL");
    if (!spot_nodes || !time_nodes) return fail(LV_EINVAL, "node arrays must not be NULL");
    if (n_spot < 2) return fail(LV_EINVAL, "n_spot must be >= 2");
    if (n_time < 1) return fail(LV_EINVAL, "n_time must be >= 1");
    if ((int64_t)n_spot * n_time > LV_MAX_NODES)
        return fail(LV_EINVAL, "n_spot * n_time exceeds LV_MAX_NODES");
    for (int i = 0; i < n_spot; ++i) {
        if (!is_finite(spot_nodes[i]) || !(spot_nodes[i] > 0.0))
            return fail(LV_EINVAL, "spot nodes must be finite and > 0");
        if (i > 0 && !(spot_nodes[i] > spot_nodes[i - 1]))
            return fail(LV_EINVAL, "spot nodes must be strictly increasing");
    }
    for (int j = 0; j < n_time; ++j) {
        if (!is_finite(time_nodes[j]) || time_nodes[j] < 0.0)
            return fail(LV_EINVAL, "time nodes must be finite and >= 0");
        if (j > 0 && !(time_nodes[j] > time_nodes[j - 1]))
            return fail(LV_EINVAL, "time nodes must be strictly increasing");
    }
    lv_status st = check_sigma(sigma, (int64_t)n_spot * n_time);
    if (st != LV_OK) return st;

    lv_surface_s* h = new (std::nothrow) lv_surface_s();
    if (!h) return fail(LV_ENOMEM, "out of host memory");
    h->I = n_spot;
    h->J = n_time;
    h->Je = n_time > 1 ? n_time : 2;
    h->spot.assign(spot_nodes, spot_nodes + n_spot);
    h->time.assign(time_nodes, time_nodes + n_time);

    // cell lookup straight from ln S when the nodes are equally spaced in ln S
    const double l0 = std::log(spot_nodes[0]);
    const double dl = (std::log(spot_nodes[n_spot - 1]) - l0) / (n_spot - 1);
    double dev = 0.0;
    for (int i = 0; i < n_spot; ++i)
        dev = std::fmax(dev, std::fabs(std::log(spot_nodes[i]) - (l0 + i * dl)));
    h->log_uniform = dev <= 1e-6 * dl ? 1 : 0;
    h->cell_scale = (float)(std::log(2.0) / dl);   // index from y = log2 S
    h->cell_shift = (float)(-l0 / dl);
    h->s_lo = (float)spot_nodes[0];
    h->s_hi = (float)spot_nodes[n_spot - 1];

    auto bail = [&](lv_status s, const std::string& m) {
        free_surface(h);
        return fail(s, m);
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(LV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return bail(LV_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));

    const size_t nsig = (size_t)h->Je * (h->I - 1);
    const size_t nres = 5 + (size_t)n_spot * n_time;      // room for the extended layout
    if (cudaMalloc(&h->d_sig, sizeof(float2) * nsig) != cudaSuccess ||
        cudaMalloc(&h->d_node, sizeof(float) * n_spot) != cudaSuccess ||
        cudaMalloc(&h->d_ab, sizeof(float2) * n_spot) != cudaSuccess ||
        cudaMalloc(&h->d_abl, sizeof(float2) * n_spot) != cudaSuccess ||
        cudaMalloc(&h->d_tau, sizeof(double) * n_time) != cudaSuccess ||
        cudaMalloc(&h->d_spot64, sizeof(double) * n_spot) != cudaSuccess ||
        cudaMalloc(&h->d_sig64, sizeof(double) * (size_t)n_spot * n_time) != cudaSuccess ||
        cudaMallocHost(&h->h_sig64_stage, sizeof(double) * (size_t)n_spot * n_time) != cudaSuccess ||
        cudaMalloc(&h->d_res, sizeof(double) * nres) != cudaSuccess ||
        cudaMallocHost(&h->h_sig_stage, sizeof(float2) * nsig) != cudaSuccess ||
        cudaMallocHost(&h->h_res, sizeof(double) * nres) != cudaSuccess) {
        cudaGetLastError();
        return bail(LV_ENOMEM, "device or pinned allocation failed");
    }
    std::vector<float> node(n_spot);
    std::vector<float2> ab(n_spot), abl(n_spot);
    for (int i = 0; i < n_spot; ++i) {
        node[i] = (float)spot_nodes[i];
        if (i + 1 < n_spot) {
            const double w = spot_nodes[i + 1] - spot_nodes[i];
            ab[i] = make_float2((float)(1.0 / w), (float)(-spot_nodes[i] / w));
            // the ln-S weight from y = log2 S: u = (y - y_i) / (y_{i+1} - y_i)
            const double y0 = std::log2(spot_nodes[i]), wl = std::log2(spot_nodes[i + 1]) - y0;
            abl[i] = make_float2((float)(1.0 / wl), (float)(-y0 / wl));
        } else {
            ab[i] = abl[i] = make_float2(0.0f, 0.0f);
        }
    }
    pack_sigma(h, sigma, h->h_sig_stage);
    if (cudaMemcpy(h->d_sig, h->h_sig_stage, sizeof(float2) * nsig, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_node, node.data(), sizeof(float) * n_spot, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_ab, ab.data(), sizeof(float2) * n_spot, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_abl, abl.data(), sizeof(float2) * n_spot, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_tau, time_nodes, sizeof(double) * n_time, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_spot64, spot_nodes, sizeof(double) * n_spot, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_sig64, sigma, sizeof(double) * (size_t)n_spot * n_time, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        e = cudaGetLastError();
        return bail(LV_ECUDA, std::string("upload of the grid failed: ") + cudaGetErrorString(e));
    }
    *out = h;
    return LV_OK;
}

void lv_surface_destroy(lv_surface_t h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_surface(h);
}

lv_status lv_surface_set_sigma(lv_surface_t h, const double* sigma)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    lv_status st = check_sigma(sigma, (int64_t)h->I * h->J);
    if (st != LV_OK) return st;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    // the staging buffer may still feed an earlier asynchronous copy
    LV_CUDA(cudaStreamSynchronize(h->stream));
    pack_sigma(h, sigma, h->h_sig_stage);
    // the binary64 copy only feeds the binary64 reference and bump calls, which
    // upload it when they run (sigma64_current); the binary32 pairs go now
    std::memcpy(h->h_sig64_stage, sigma, sizeof(double) * (size_t)h->I * h->J);
    h->sig64_stale = true;
    LV_CUDA(cudaMemcpyAsync(h->d_sig, h->h_sig_stage, sizeof(float2) * (size_t)h->Je * (h->I - 1),
                            cudaMemcpyHostToDevice, h->stream));
    return LV_OK;
}

lv_status lv_set_option_type(lv_surface_t h, int32_t phi)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (phi != 1 && phi != -1) return fail(LV_EINVAL, "phi must be +1 (call) or -1 (put)");
    h->phi = phi;
    return LV_OK;
}

lv_status lv_set_stream(lv_surface_t h, void* cuda_stream)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (s != h->stream) {
        // the scratch and the staging buffers may still be in use on the old stream
        DeviceGuard g(h->device);
        if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
        LV_CUDA(cudaStreamSynchronize(h->stream));
        h->stream = s;
    }
    return LV_OK;
}

lv_status lv_set_accumulation(lv_surface_t h, int32_t mode)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (mode != LV_ACC_FP64 && mode != LV_ACC_KAHAN)
        return fail(LV_EINVAL, "mode must be LV_ACC_FP64 or LV_ACC_KAHAN");
    h->acc_mode = mode;
    return LV_OK;
}

lv_status lv_surface_set_interpolation(lv_surface_t h, int32_t interp)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (interp != LV_INTERP_S && interp != LV_INTERP_LOGS)
        return fail(LV_EINVAL, "interp must be LV_INTERP_S or LV_INTERP_LOGS");
    h->interp = interp;
    return LV_OK;
}

lv_status lv_set_scheme(lv_surface_t h, int32_t scheme)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (scheme != LV_SCHEME_LOG && scheme != LV_SCHEME_S)
        return fail(LV_EINVAL, "scheme must be LV_SCHEME_LOG or LV_SCHEME_S");
    h->scheme = scheme;
    return LV_OK;
}

lv_status lv_set_adjoint_method(lv_surface_t h, int32_t method)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (method != LV_ADJ_REVERSE && method != LV_ADJ_TANGENT)
        return fail(LV_EINVAL, "method must be LV_ADJ_REVERSE or LV_ADJ_TANGENT");
    h->adj_method = method;
    return LV_OK;
}

lv_status lv_set_launch(lv_surface_t h, int32_t block, int32_t k, int32_t blocks_per_sm)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (block != 0 && (block < 32 || block > 128 || block % 32 != 0))
        return fail(LV_EINVAL, "block must be 0 or a multiple of 32 in [32, 128]");
    if (k != 0 && k != 4 && k != 8 && k != 16 && k != 32)
        return fail(LV_EINVAL, "k must be 0, 4, 8, 16 or 32");
    if (blocks_per_sm < 0) return fail(LV_EINVAL, "blocks_per_sm must be >= 0");
    h->cfg_block = block;
    h->cfg_k = k;
    h->cfg_bps = blocks_per_sm;
    return LV_OK;
}

lv_status lv_set_paths_per_lane(lv_surface_t h, int32_t ppl)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (ppl < 0 || ppl > 2) return fail(LV_EINVAL, "paths per lane must be 0, 1 or 2");
    h->cfg_ppl = ppl;
    return LV_OK;
}

lv_status lv_get_paths_per_lane(lv_surface_t h, int32_t n_steps, int64_t n_paths, int32_t* ppl)
{
    if (!h || !ppl) return fail(LV_EINVAL, "NULL argument");
    if (n_steps < 1 || n_steps > LV_MAX_STEPS) return fail(LV_EINVAL, "n_steps out of range");
    if (n_paths < 1) return fail(LV_EINVAL, "n_paths must be >= 1");
    DeviceGuard g(h->device);
    int b = 0, kk = 0, bps = 0, p = 1;
    bool gs = true;
    lv_status st = choose_launch(h, n_steps, true, &b, &kk, &bps, false, &gs, false, false, &p, n_paths);
    if (st != LV_OK) return st;
    *ppl = p;
    return LV_OK;
}

lv_status lv_set_kernel_events(lv_surface_t h, void* start_event, void* end_event)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if ((start_event == nullptr) != (end_event == nullptr))
        return fail(LV_EINVAL, "pass both events or neither");
    h->ev_start = static_cast<cudaEvent_t>(start_event);
    h->ev_end = static_cast<cudaEvent_t>(end_event);
    return LV_OK;
}

lv_status lv_get_launch(lv_surface_t h, int32_t n_steps, int32_t greeks, int32_t* block, int32_t* k,
                        int32_t* blocks_per_sm)
{
    if (!h || !block || !k || !blocks_per_sm) return fail(LV_EINVAL, "NULL argument");
    if (n_steps < 1 || n_steps > LV_MAX_STEPS) return fail(LV_EINVAL, "n_steps out of range");
    DeviceGuard g(h->device);
    int b = 0, kk = 0, bps = 0;
    lv_status st = choose_launch(h, n_steps, greeks != 0, &b, &kk, &bps, false, nullptr);
    if (st != LV_OK) return st;
    *block = b;
    *k = kk;
    *blocks_per_sm = bps;
    return LV_OK;
}

lv_status lv_price(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                   int64_t n_paths, uint64_t seed, double* out_price, double* out_stderr)
{
    if (!h || !out_price) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, false, false, h->d_res};
    lv_status st = run_mc(h, c);
    if (st != LV_OK) return st;
    st = fetch_result(h);
    if (st != LV_OK) return st;
    *out_price = h->h_res[LV_OUT_PRICE];
    if (out_stderr) *out_stderr = h->h_res[LV_OUT_STDERR];
    return LV_OK;
}

lv_status lv_price_greeks_device(lv_surface_t h, double S0, double r, double K, double T,
                                 int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out)
{
    if (!h || !d_out) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, d_out};
    return run_mc(h, c);
}

lv_status lv_price_greeks(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                          int64_t n_paths, uint64_t seed, double* out_price, double* out_delta,
                          double* out_vega)
{
    if (!h || !out_price || !out_delta || !out_vega) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, h->d_res};
    lv_status st = run_mc(h, c);
    if (st != LV_OK) return st;
    st = fetch_result(h);
    if (st != LV_OK) return st;
    if (std::isnan(h->h_res[LV_OUT_PRICE]))    // outputs left untouched, like every failure
        return fail(LV_ENUMERIC, "a factor 1 + g_n vanished on a live path: use LV_ADJ_REVERSE for this grid");
    *out_price = h->h_res[LV_OUT_PRICE];
    *out_delta = h->h_res[LV_OUT_DELTA];
    std::memcpy(out_vega, h->h_res + LV_OUT_VEGA, sizeof(double) * (size_t)h->I * h->J);
    return LV_OK;
}

lv_status lv_price_greeks_ext(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                              int64_t n_paths, uint64_t seed, double* out_price, double* out_delta,
                              double* out_vega, double* out_rho, double* out_dVdT)
{
    if (!h || !out_price || !out_delta || !out_vega || !out_rho || !out_dVdT) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, h->d_res};
    c.extra = true;
    lv_status st = run_mc(h, c);
    if (st != LV_OK) return st;
    st = fetch_result(h, true);
    if (st != LV_OK) return st;
    const size_t IJ = (size_t)h->I * h->J;
    *out_price = h->h_res[LV_OUT_PRICE];
    *out_delta = h->h_res[LV_OUT_DELTA];
    std::memcpy(out_vega, h->h_res + LV_OUT_VEGA, sizeof(double) * IJ);
    *out_rho = h->h_res[3 + IJ];
    *out_dVdT = h->h_res[4 + IJ];
    return LV_OK;
}

lv_status lv_price_greeks_ext_device(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                                     int64_t n_paths, uint64_t seed, double* d_out)
{
    if (!h || !d_out) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, d_out};
    c.extra = true;
    return run_mc(h, c);
}

lv_status lv_price_greeks_vanna_device(lv_surface_t h, double S0, double r, double K, double T,
                                       int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out)
{
    if (!h || !d_out) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, d_out};
    c.vanna = true;
    return run_mc(h, c);
}

lv_status lv_price_greeks_vanna(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                                int64_t n_paths, uint64_t seed, double* out_price, double* out_delta,
                                double* out_vanna)
{
    if (!h || !out_price || !out_delta || !out_vanna) return fail(LV_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, h->d_res};
    c.vanna = true;
    lv_status st = run_mc(h, c);
    if (st != LV_OK) return st;
    st = fetch_result(h);
    if (st != LV_OK) return st;
    if (std::isnan(h->h_res[LV_OUT_PRICE]))    // outputs left untouched, like every failure
        return fail(LV_ENUMERIC, "a factor 1 + g_n vanished on a live path");
    *out_price = h->h_res[LV_OUT_PRICE];
    *out_delta = h->h_res[LV_OUT_DELTA];
    std::memcpy(out_vanna, h->h_res + LV_OUT_VEGA, sizeof(double) * (size_t)h->I * h->J);
    return LV_OK;
}

lv_status lv_price_greeks_sums_device(lv_surface_t h, double S0, double r, double K, double T,
                                      int32_t n_steps, int64_t path_begin, int64_t path_end,
                                      uint64_t seed, uint32_t stream_id, double* d_sums)
{
    if (!h || !d_sums) return fail(LV_EINVAL, "NULL argument");
    if (path_end <= path_begin) return fail(LV_EINVAL, "path_end must exceed path_begin");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{S0, r, K, T, n_steps, path_begin, path_end - path_begin, seed, stream_id, true, true, d_sums};
    return run_mc(h, c);
}

lv_status lv_tune(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps, int64_t n_paths,
                  uint64_t seed, int32_t* out_block, int32_t* out_k, double* out_ms)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    lv_status st = check_option(S0, r, K, T, n_steps);
    if (st != LV_OK) return st;
    if (n_paths < 1 || n_paths > 0x7fffffffLL) return fail(LV_EINVAL, "n_paths must be in [1, 2^31 - 1]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    const int blocks[] = {64, 128};
    const int ks[] = {4, 8, 16};
    const int keep_b = h->cfg_block, keep_k = h->cfg_k, keep_s = h->cfg_bps, keep_p = h->cfg_ppl;
    // two paths per lane exist for the main reading's reverse sweep at k = 4 and 8
    // the reverse sweep under every reading, the tangent-ratio adjoint under the main one
    const bool ppl2 = h->adj_method == LV_ADJ_REVERSE || (h->interp == LV_INTERP_S && h->scheme == LV_SCHEME_LOG);
    cudaEvent_t e0, e1;
    LV_CUDA(cudaEventCreate(&e0));
    LV_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int bb = 128, bk = 4, bp = 1;
    for (int blk : blocks)
        for (int k : ks)
        for (int ppl = 1; ppl <= ((ppl2 && k <= 8) ? 2 : 1); ++ppl) {
            h->cfg_block = blk;
            h->cfg_k = k;
            h->cfg_bps = 0;
            h->cfg_ppl = ppl;
            McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, h->d_res};
            if (run_mc(h, c) != LV_OK) continue;             // warm-up (and scratch growth)
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {          // best of three
                cudaEventRecord(e0, h->stream);
                if (run_mc(h, c) != LV_OK) break;
                cudaEventRecord(e1, h->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t = std::fmin(t, ms);
            }
            if (t < best) {
                best = t;
                bb = blk;
                bk = k;
                bp = ppl;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!(best < 1e299)) {
        h->cfg_block = keep_b;
        h->cfg_k = keep_k;
        h->cfg_bps = keep_s;
        h->cfg_ppl = keep_p;
        return fail(LV_EINTERNAL, "no launch shape ran");
    }
    h->cfg_block = bb;
    h->cfg_k = bk;
    h->cfg_bps = 0;
    h->cfg_ppl = bp;
    const int v[4] = {bb, bk, bp, 0};
    lv::tune_cache_append(adjoint_tune_key(h, n_steps), v, best);
    if (out_block) *out_block = bb;
    if (out_k) *out_k = bk;
    if (out_ms) *out_ms = best;
    return LV_OK;
}

lv_status lv_finalize_sums_device(lv_surface_t h, const double* d_sums, int64_t n_paths, double S0,
                                  double* d_out)
{
    if (!h || !d_sums || !d_out) return fail(LV_EINVAL, "NULL argument");
    if (n_paths < 1) return fail(LV_EINVAL, "n_paths must be >= 1");
    if (!is_finite(S0) || !(S0 > 0.0)) return fail(LV_EINVAL, "S0 must be finite and > 0");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    LV_CUDA(lv::launch_finalize_sums(d_sums, h->I * h->J, n_paths, S0, d_out, h->stream));
    return LV_OK;
}

lv_status lv_bump_greeks(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                         int64_t n_paths, uint64_t seed, double eps, double* out_price,
                         double* out_delta, double* out_vega)
{
    if (!h || !out_price || !out_delta || !out_vega) return fail(LV_EINVAL, "NULL argument");
    lv_status st = check_option(S0, r, K, T, n_steps);
    if (st != LV_OK) return st;
    if (!is_finite(eps) || !(eps > 0.0)) return fail(LV_EINVAL, "eps must be finite and > 0");
    if (h->interp != LV_INTERP_S || h->scheme != LV_SCHEME_LOG)
        return fail(LV_EINVAL, "the bump baseline runs the main reading (LV_INTERP_S, LV_SCHEME_LOG) only");
    if (n_paths < 1 || n_paths > LV_MAX_PATH_INDEX) return fail(LV_EINVAL, "n_paths out of range");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    const int IJ = h->I * h->J;
    const int block = 256;
    const int row_words = 2 + IJ;
    const int n_scen = 3 + 2 * IJ;
    const int M = lv::bump_slots_per_thread();
    const int n_groups = (n_scen + M - 1) / M;
    const size_t smem = lv::bump_smem_bytes(h->I, h->Je, n_steps, row_words);
    if (smem > 200 * 1024) return fail(LV_EINVAL, "grid too large for the bump kernel's shared memory");
    int bps = 0;
    LV_CUDA(lv::bump_occupancy(block, smem, &bps));
    if (bps < 1) return fail(LV_EINVAL, "bump launch shape does not fit on an SM");
    const int64_t tiles = (n_paths + block - 1) / block;
    const int64_t items = tiles * n_groups;
    if (items > (int64_t)0x7fffffff) return fail(LV_EINVAL, "too many paths x scenarios for one call");
    const int64_t slots = (int64_t)bps * h->num_sms;
    const int grid = (int)(items < slots ? items : slots);
    const int nch = lv::bump_chunks(grid);
    size_t o = 256;
    const size_t off_part = o;
    o = round_up(o + sizeof(double) * (size_t)grid * row_words, 256);
    const size_t off_chunks = o;
    o = round_up(o + sizeof(double) * (size_t)nch * row_words, 256);
    st = ensure_scratch(h, o);
    if (st != LV_OK) return st;
    char* base = static_cast<char*>(h->d_scratch);
    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, false, false, h->d_res};
    lv::BumpParams B{};
    B.mc = base_params(h, c);
    B.mc.n_tiles = (int)tiles;
    B.mc.tile_counter = reinterpret_cast<unsigned int*>(base);
    const double eps_S = 1e-4 * S0;
    B.n_scen = n_scen;
    B.n_groups = n_groups;
    B.eps_half = (float)(0.5 * eps);
    B.x0_up = (float)std::log2(S0 + 0.5 * eps_S);
    B.x0_dn = (float)std::log2(S0 - 0.5 * eps_S);
    B.partials = reinterpret_cast<double*>(base + off_part);
    B.row_words = row_words;
    if (h->ev_start) LV_CUDA(cudaEventRecord(h->ev_start, h->stream));
    LV_CUDA(lv::launch_bump(B, grid, block, smem, h->stream));
    if (h->ev_end) LV_CUDA(cudaEventRecord(h->ev_end, h->stream));
    LV_CUDA(lv::launch_bump_finalize(B.partials, grid, row_words, reinterpret_cast<double*>(base + off_chunks),
                                     IJ, n_paths, eps, eps_S, h->d_res, B.mc.tile_counter, h->stream));
    st = fetch_result(h);
    if (st != LV_OK) return st;
    *out_price = h->h_res[LV_OUT_PRICE];
    *out_delta = h->h_res[LV_OUT_DELTA];
    std::memcpy(out_vega, h->h_res + LV_OUT_VEGA, sizeof(double) * (size_t)IJ);
    return LV_OK;
}

lv_status lv_measure_pipe_peaks(double* out_ops_per_s)
{
    if (!out_ops_per_s) return fail(LV_EINVAL, "NULL argument");
    double tmp[LV_PIPE_COUNT] = {};
    LV_CUDA(lv::measure_pipe_peaks(tmp));
    std::memcpy(out_ops_per_s, tmp, sizeof tmp);
    return LV_OK;
}

lv_status lv_price_greeks_fp64_device(lv_surface_t h, double S0, double r, double K, double T,
                                      int32_t n_steps, int64_t n_paths, uint64_t seed, double* d_out)
{
    if (!h || !d_out) return fail(LV_EINVAL, "NULL argument");
    lv_status st = check_option(S0, r, K, T, n_steps);
    if (st != LV_OK) return st;
    if (n_paths < 1 || n_paths > LV_MAX_PATH_INDEX) return fail(LV_EINVAL, "n_paths out of range");
    if (h->interp != LV_INTERP_S || h->scheme != LV_SCHEME_LOG)
        return fail(LV_EINVAL, "the binary64 reference runs the main reading (LV_INTERP_S, LV_SCHEME_LOG) only");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    const size_t smem = lv::adjoint64_smem_bytes(n_steps);
    int bps = 0;
    LV_CUDA(lv::f64_occupancy(false, smem, &bps));
    if (bps < 1) return fail(LV_EINVAL, "binary64 launch does not fit on an SM");
    const int64_t want = (n_paths + 127) / 128;
    const int64_t slots = (int64_t)bps * h->num_sms;
    const int grid = (int)(want < slots ? want : slots);
    const int row_words = 3 + h->Je * h->I;
    size_t o = 256;                                   // [0, 256): tile counter (unused), flag
    const size_t off_part = o;
    o = round_up(o + sizeof(double) * (size_t)grid * row_words, 256);
    const size_t off_chunks = o;
    o = round_up(o + sizeof(double) * (size_t)lv::finalize_chunks(grid) * row_words, 256);
    st = ensure_scratch(h, o);
    if (st != LV_OK) return st;
    char* base = static_cast<char*>(h->d_scratch);
    const double dt = T / (double)n_steps;
    st = sigma64_current(h);
    if (st != LV_OK) return st;
    lv::F64Params P{};
    P.spot = h->d_spot64;
    P.sig = h->d_sig64;
    P.tau = h->d_tau;
    P.I = h->I;
    P.J = h->J;
    P.N = n_steps;
    P.x0 = std::log(S0);
    P.r = r;
    P.dt = dt;
    P.sqdt = std::sqrt(dt);
    P.K = K;
    P.disc = std::exp(-r * T);
    P.phi = (double)h->phi;
    P.k0 = (uint32_t)(seed & 0xffffffffu);
    P.k1 = (uint32_t)(seed >> 32);
    P.n_paths = n_paths;
    P.partials = reinterpret_cast<double*>(base + off_part);
    P.row_words = row_words;
    P.flag = reinterpret_cast<unsigned int*>(base) + 1;    // zero; every finalize resets it
    if (h->ev_start) LV_CUDA(cudaEventRecord(h->ev_start, h->stream));
    LV_CUDA(lv::launch_adjoint64(P, grid, smem, h->stream));
    if (h->ev_end) LV_CUDA(cudaEventRecord(h->ev_end, h->stream));
    lv::FinalizeParams F{};
    F.partials = P.partials;
    F.G = grid;
    F.row_words = row_words;
    F.I = h->I;
    F.J = h->J;
    F.n_paths = n_paths;
    F.S0 = S0;
    F.chunks = reinterpret_cast<double*>(base + off_chunks);
    F.out = d_out;
    F.tile_counter = reinterpret_cast<unsigned int*>(base);
    F.flag = P.flag;
    LV_CUDA(lv::launch_finalize(F, h->stream));
    return LV_OK;
}

lv_status lv_bump_greeks_fp64(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                              int64_t n_paths, uint64_t seed, double eps, double* out_price, double* out_delta,
                              double* out_vega)
{
    if (!h || !out_price || !out_delta || !out_vega) return fail(LV_EINVAL, "NULL argument");
    lv_status st = check_option(S0, r, K, T, n_steps);
    if (st != LV_OK) return st;
    if (!is_finite(eps) || !(eps > 0.0)) return fail(LV_EINVAL, "eps must be finite and > 0");
    if (h->interp != LV_INTERP_S || h->scheme != LV_SCHEME_LOG)
        return fail(LV_EINVAL, "the bump baseline runs the main reading (LV_INTERP_S, LV_SCHEME_LOG) only");
    if (n_paths < 1 || n_paths > LV_MAX_PATH_INDEX) return fail(LV_EINVAL, "n_paths out of range");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    const int IJ = h->I * h->J;
    const int row_words = 2 + IJ;
    const int n_scen = 3 + 2 * IJ;
    const int M = lv::bump64_slots_per_thread();
    const size_t smem = lv::bump64_smem_bytes(n_steps, row_words);
    if (smem > 200 * 1024) return fail(LV_EINVAL, "grid too large for the binary64 bump kernel's shared memory");
    int bps = 0;
    LV_CUDA(lv::f64_occupancy(true, smem, &bps));
    if (bps < 1) return fail(LV_EINVAL, "binary64 bump launch does not fit on an SM");
    const int64_t items = (n_paths + 127) / 128 * ((n_scen + M - 1) / M);
    const int64_t slots = (int64_t)bps * h->num_sms;
    const int grid = (int)(items < slots ? items : slots);
    const int nch = lv::bump_chunks(grid);
    size_t o = 256;
    const size_t off_part = o;
    o = round_up(o + sizeof(double) * (size_t)grid * row_words, 256);
    const size_t off_chunks = o;
    o = round_up(o + sizeof(double) * (size_t)nch * row_words, 256);
    st = ensure_scratch(h, o);
    if (st != LV_OK) return st;
    char* base = static_cast<char*>(h->d_scratch);
    const double dt = T / (double)n_steps;
    const double eps_S = eps * S0;             // the spot bump of the same relative size
    st = sigma64_current(h);
    if (st != LV_OK) return st;
    lv::F64Params P{};
    P.spot = h->d_spot64;
    P.sig = h->d_sig64;
    P.tau = h->d_tau;
    P.I = h->I;
    P.J = h->J;
    P.N = n_steps;
    P.x0 = std::log(S0);
    P.x0_up = std::log(S0 + 0.5 * eps_S);
    P.x0_dn = std::log(S0 - 0.5 * eps_S);
    P.r = r;
    P.dt = dt;
    P.sqdt = std::sqrt(dt);
    P.K = K;
    P.disc = std::exp(-r * T);
    P.phi = (double)h->phi;
    P.eps_half = 0.5 * eps;
    P.k0 = (uint32_t)(seed & 0xffffffffu);
    P.k1 = (uint32_t)(seed >> 32);
    P.n_paths = n_paths;
    P.partials = reinterpret_cast<double*>(base + off_part);
    P.row_words = row_words;
    P.n_scen = n_scen;
    P.n_groups = (n_scen + M - 1) / M;
    if (h->ev_start) LV_CUDA(cudaEventRecord(h->ev_start, h->stream));
    LV_CUDA(lv::launch_bump64(P, grid, smem, h->stream));
    if (h->ev_end) LV_CUDA(cudaEventRecord(h->ev_end, h->stream));
    LV_CUDA(lv::launch_bump_finalize(P.partials, grid, row_words, reinterpret_cast<double*>(base + off_chunks), IJ,
                                     n_paths, eps, eps_S, h->d_res, nullptr, h->stream));
    st = fetch_result(h);
    if (st != LV_OK) return st;
    *out_price = h->h_res[LV_OUT_PRICE];
    *out_delta = h->h_res[LV_OUT_DELTA];
    std::memcpy(out_vega, h->h_res + LV_OUT_VEGA, sizeof(double) * (size_t)IJ);
    return LV_OK;
}

lv_status lv_debug_paths(lv_surface_t h, double S0, double r, double K, double T, int32_t n_steps,
                         uint64_t seed, uint32_t stream_id, int64_t path_begin, int64_t m, float* out_xN,
                         float* out_V, float* out_xbar0, double node_band, int64_t ev_cap, int32_t* out_ev,
                         int64_t* out_n_ev)
{
    if (!h) return fail(LV_EINVAL, "handle is NULL");
    if (m < 1 || m > (int64_t)1 << 26) return fail(LV_EINVAL, "m must be in [1, 2^26]");
    if (ev_cap < 0 || ev_cap > ((int64_t)1 << 28)) return fail(LV_EINVAL, "ev_cap must be in [0, 2^28]");
    if (ev_cap > 0 && !out_ev) return fail(LV_EINVAL, "out_ev is NULL");
    if (!is_finite(node_band) || node_band < 0.0) return fail(LV_EINVAL, "node_band must be >= 0");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    // layout: [0, 256) the 64-bit log counter, then the per-path floats, then the
    // log, each section 256-byte aligned
    const size_t f_bytes = sizeof(float) * 3 * (size_t)m;
    const size_t e_bytes = sizeof(int) * 3 * (size_t)ev_cap;
    const size_t off_f = 256;
    const size_t off_e = round_up(off_f + f_bytes, 256);
    char* d = nullptr;
    if (cudaMalloc(&d, off_e + e_bytes + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(LV_ENOMEM, "cannot allocate the per-path buffers");
    }
    unsigned long long* dcount = reinterpret_cast<unsigned long long*>(d);
    float* df = reinterpret_cast<float*>(d + off_f);
    McCall c{S0, r, K, T, n_steps, path_begin, m, seed, stream_id, true, false, h->d_res};
    c.dbg_xN = df;
    c.dbg_V = df + m;
    c.dbg_xbar0 = df + 2 * m;
    c.dbg_ev = reinterpret_cast<int*>(d + off_e);
    c.dbg_ev_count = dcount;
    c.dbg_ev_cap = ev_cap;
    c.dbg_band = node_band;
    lv_status st = LV_OK;
    cudaError_t e = cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), h->stream);
    if (e != cudaSuccess) st = fail(LV_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if (st == LV_OK) st = run_mc(h, c);
    if (st == LV_OK) {
        std::vector<float> hb(3 * (size_t)m);
        unsigned long long n_ev = 0;
        e = cudaMemcpyAsync(hb.data(), df, f_bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&n_ev, dcount, sizeof(n_ev), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        const int64_t n_copy = (int64_t)n_ev < ev_cap ? (int64_t)n_ev : ev_cap;
        if (e == cudaSuccess && n_copy > 0)
            e = cudaMemcpy(out_ev, d + off_e, sizeof(int) * 3 * (size_t)n_copy, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            st = fail(LV_ECUDA, std::string("per-path copy: ") + cudaGetErrorString(e));
        } else {
            if (out_xN) std::memcpy(out_xN, hb.data(), sizeof(float) * m);
            if (out_V) std::memcpy(out_V, hb.data() + m, sizeof(float) * m);
            if (out_xbar0) std::memcpy(out_xbar0, hb.data() + 2 * m, sizeof(float) * m);
            if (out_n_ev) *out_n_ev = (int64_t)n_ev;
        }
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    return st;
}

lv_status lv_debug_normals(uint64_t seed, uint32_t stream_id, const int64_t* paths, const uint32_t* blocks,
                           int64_t n, uint32_t* out_words, float* out_z)
{
    if (!paths || !blocks || !out_words || !out_z) return fail(LV_EINVAL, "NULL argument");
    if (n < 1 || n > ((int64_t)1 << 24)) return fail(LV_EINVAL, "n must be in [1, 2^24]");
    if (stream_id >= 65536u) return fail(LV_EINVAL, "stream_id must be < 65536");
    for (int64_t e = 0; e < n; ++e)
        if (paths[e] < 0 || paths[e] >= LV_MAX_PATH_INDEX) return fail(LV_EINVAL, "path indices must lie in [0, 2^48)");
    // one allocation: [paths n][blocks n][words 4n][z 4n], each section 256-byte aligned
    const size_t off_b = round_up(sizeof(long long) * (size_t)n, 256);
    const size_t off_w = round_up(off_b + sizeof(uint32_t) * (size_t)n, 256);
    const size_t off_z = round_up(off_w + sizeof(uint32_t) * 4 * (size_t)n, 256);
    const size_t total = off_z + sizeof(float) * 4 * (size_t)n;
    char* d = nullptr;
    if (cudaMalloc(&d, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(LV_ENOMEM, "cannot allocate the normals buffers");
    }
    cudaError_t e = cudaMemcpy(d, paths, sizeof(long long) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + off_b, blocks, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = lv::launch_debug_normals(seed, stream_id, reinterpret_cast<const long long*>(d),
                                     reinterpret_cast<const uint32_t*>(d + off_b), n,
                                     reinterpret_cast<uint32_t*>(d + off_w), reinterpret_cast<float*>(d + off_z), 0);
    if (e == cudaSuccess) e = cudaMemcpy(out_words, d + off_w, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_z, d + off_z, sizeof(float) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LV_ECUDA, std::string("lv_debug_normals: ") + cudaGetErrorString(e));
    return LV_OK;
}

lv_status lv_debug_time_table(lv_surface_t h, double T, int32_t n_steps, int32_t* out_j, float* out_v)
{
    if (!h || !out_j || !out_v) return fail(LV_EINVAL, "NULL argument");
    lv_status st = check_option(1.0, 0.0, 1.0, T, n_steps);
    if (st != LV_OK) return st;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    McCall c{1.0, 0.0, 1.0, T, n_steps, 0, 1, 1, 0u, true, false, h->d_res};
    const lv::McParams P = base_params(h, c);
    const size_t off_v = round_up(sizeof(int) * (size_t)n_steps, 256);
    char* d = nullptr;
    if (cudaMalloc(&d, off_v + sizeof(float) * (size_t)n_steps) != cudaSuccess) {
        cudaGetLastError();
        return fail(LV_ENOMEM, "cannot allocate the time-table buffers");
    }
    cudaError_t e = lv::launch_debug_time_table(P, reinterpret_cast<int*>(d), reinterpret_cast<float*>(d + off_v),
                                                h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_j, d, sizeof(int) * (size_t)n_steps, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_v, d + off_v, sizeof(float) * (size_t)n_steps, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LV_ECUDA, std::string("lv_debug_time_table: ") + cudaGetErrorString(e));
    return LV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of lv_price_greeks_device.
//
// Some callers cannot call cudaMalloc while they run: a real-time loop with a
// no-allocation rule, or an embedding runtime that owns every device
// allocation itself.
// For them the adjoint can run on scratch memory the library reserves once
// when its module is loaded: a file-scope __device__ array, kept by every
// GPU that loads the library until the process exits.

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;     // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device. In host code the array's
// name is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
void* g_static_addr[kMaxDevices] = {};
std::mutex g_static_mu;

lv_status static_scratch(int device, char** out)
{
    if (device < 0 || device >= kMaxDevices) return fail(LV_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(LV_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_static_addr[device] = p;
    }
    *out = static_cast<char*>(g_static_addr[device]);
    return LV_OK;
}

// Scratch layout of one adjoint launch with `grid` blocks (same sections as
// the allocating path); returns the bytes needed.
size_t static_plan_bytes(const lv_surface_s* h, int grid, int block, int k, int ppl, int n_steps, size_t* off_part,
                         size_t* off_chunks, size_t* off_wrows, size_t* off_l1, size_t* off_ckpt)
{
    const size_t nIJ = (size_t)h->Je * h->I;
    const size_t row_words = 3 + nIJ;
    const size_t warps = (size_t)grid * (block / 32);
    const size_t n_ck = h->adj_method == LV_ADJ_TANGENT ? 0 : (size_t)((n_steps + k - 1) / k);
    size_t o = 256;                                               // [0, 256): tile counter, flag
    *off_part = o;   o = round_up(o + sizeof(double) * (size_t)grid * row_words, 256);
    *off_chunks = o; o = round_up(o + sizeof(double) * (size_t)lv::finalize_chunks(grid) * row_words, 256);
    *off_wrows = o;                                               // per-warp rows: Kahan mode only
    if (h->acc_mode == LV_ACC_KAHAN) o = round_up(o + sizeof(double) * warps * nIJ, 256);
    *off_l1 = o;     o = round_up(o + sizeof(float) * (size_t)grid * nIJ, 256);
    *off_ckpt = o;   o = round_up(o + sizeof(float) * n_ck * warps * lv::ring_slots_per_warp() * ppl, 256);
    return o;
}

}  // namespace

extern "C" lv_status lv_price_greeks_device_noalloc(lv_surface_t h, double S0, double r, double K, double T,
                                                    int32_t n_steps, int64_t n_paths, uint64_t seed,
                                                    double* d_out)
{
    if (!h || !d_out) return fail(LV_EINVAL, "NULL argument");
    lv_status st = check_option(S0, r, K, T, n_steps);
    if (st != LV_OK) return st;
    if (n_paths < 1 || n_paths > 0x7fffffffLL) return fail(LV_EINVAL, "n_paths must be in [1, 2^31 - 1]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(LV_ECUDA, "cannot select the handle's device");
    char* base = nullptr;
    st = static_scratch(h->device, &base);
    if (st != LV_OK) return st;

    int block = 0, k = 0, bps = 0, ppl = 1;
    bool grid_smem = true;
    st = choose_launch(h, n_steps, true, &block, &k, &bps, false, &grid_smem, false, false, &ppl, n_paths);
    if (st != LV_OK) return st;
    const int warps = block / 32;
    const int64_t tiles = (n_paths + lv::paths_per_tile(true) - 1) / lv::paths_per_tile(true);
    const int64_t want_blocks = (tiles + warps - 1) / warps;
    size_t off_part = 0, off_chunks = 0, off_wrows = 0, off_l1 = 0, off_ckpt = 0;
    // two paths per lane double each block's checkpoint ring: unless the caller
    // asked for them, run one path per lane when the full-width grid would not
    // fit in the static array at two (one fits about twice as many blocks)
    if (ppl == 2 && h->cfg_ppl == 0) {
        const int64_t full = want_blocks < (int64_t)bps * h->num_sms ? want_blocks : (int64_t)bps * h->num_sms;
        if (static_plan_bytes(h, (int)full, block, k, 2, n_steps, &off_part, &off_chunks, &off_wrows, &off_l1,
                              &off_ckpt) > kStaticScratchBytes) {
            h->cfg_ppl = 1;
            st = choose_launch(h, n_steps, true, &block, &k, &bps, false, &grid_smem, false, false, &ppl, n_paths);
            h->cfg_ppl = 0;
            if (st != LV_OK) return st;
        }
    }
    const int64_t slots = (int64_t)bps * h->num_sms;
    int grid = (int)(want_blocks < slots ? want_blocks : slots);
    // the most blocks (at most the full-width grid) whose scratch fits in the static array;
    // the plan's size grows with the grid, so bisect
    if (static_plan_bytes(h, grid, block, k, ppl, n_steps, &off_part, &off_chunks, &off_wrows, &off_l1, &off_ckpt) >
        kStaticScratchBytes) {
        int lo = 1, hi = grid - 1;
        while (lo < hi) {
            const int mid = lo + (hi - lo + 1) / 2;
            if (static_plan_bytes(h, mid, block, k, ppl, n_steps, &off_part, &off_chunks, &off_wrows, &off_l1,
                                  &off_ckpt) <= kStaticScratchBytes)
                lo = mid;
            else
                hi = mid - 1;
        }
        grid = lo;
    }
    const size_t need = static_plan_bytes(h, grid, block, k, ppl, n_steps, &off_part, &off_chunks, &off_wrows,
                                          &off_l1, &off_ckpt);
    if (need > kStaticScratchBytes)
        return fail(LV_EINVAL, "grid of " + std::to_string(h->I) + " x " + std::to_string(h->J) + " nodes with " +
                               std::to_string(n_steps) + " steps needs " + std::to_string(need) +
                               " bytes of scratch for a single block; the static scratch holds " +
                               std::to_string(kStaticScratchBytes));

    McCall c{S0, r, K, T, n_steps, 0, n_paths, seed, 0u, true, false, d_out};
    lv::McParams P = base_params(h, c);
    P.n_tiles = (int)tiles;
    P.ppl = ppl;
    P.tile_counter = reinterpret_cast<unsigned int*>(base);
    P.partials = reinterpret_cast<double*>(base + off_part);
    P.row_words = 3 + h->Je * h->I;
    P.warp_rows = reinterpret_cast<double*>(base + off_wrows);
    P.l1 = reinterpret_cast<float*>(base + off_l1);
    P.ckpt = reinterpret_cast<float*>(base + off_ckpt);
    P.n_ck = h->adj_method == LV_ADJ_TANGENT ? 0 : (n_steps + k - 1) / k;
    P.flush_every = 8;
    P.grid_smem = grid_smem ? 1 : 0;
    if (h->adj_method == LV_ADJ_TANGENT) {
        P.method = LV_ADJ_TANGENT;
        P.flag = P.tile_counter + 1;
    }
    // the array keeps the previous call's contents: the tile counter and the
    // flag must start at zero (every other section is written before it is read)
    LV_CUDA(cudaMemsetAsync(P.tile_counter, 0, 2 * sizeof(unsigned int), h->stream));
    const size_t smem = lv::mc_smem_bytes(h->I, h->Je, n_steps, block, true, grid_smem, false, ppl);
    LV_CUDA(lv::launch_mc(P, grid, block, k, true, smem, h->stream));
    lv::FinalizeParams F{};
    F.partials = P.partials;
    F.G = grid;
    F.row_words = P.row_words;
    F.I = h->I;
    F.J = h->J;
    F.n_paths = n_paths;
    F.S0 = S0;
    F.want_sums = 0;
    F.chunks = reinterpret_cast<double*>(base + off_chunks);
    F.out = d_out;
    F.tile_counter = P.tile_counter;
    F.flag = P.flag;
    LV_CUDA(lv::launch_finalize(F, h->stream));
    return LV_OK;
}
