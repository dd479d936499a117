// lv_book_api.cu -- host side of the book of options: tables, scratch,
// graph capture of a run, and the launch-shape autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lv.h"
#include "lv_internal.h"

namespace {

using lv::set_error;

#define LV_BCUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return set_error(LV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

struct lv_book_s {
    int device = 0, num_sms = 0;
    std::vector<lv::BookInst> insts;        // in the caller's order
    std::vector<lv::BookSurf> surfs;
    std::vector<int64_t> offsets;           // [n + 1]
    std::vector<int64_t> risk_offsets;      // [n_surfaces + 1]
    int max_I = 0, max_J = 0, max_Je = 0, max_N = 0, max_IJe = 0, max_IJ = 0;
    int64_t total_paths = 0;
    // device tables and grids
    lv::BookSurf* d_surfs = nullptr;
    lv::BookInst* d_insts = nullptr;
    lv::BookItem* d_items = nullptr;
    int n_items = 0;
    float2* d_sig2 = nullptr;
    float* d_node = nullptr;
    float2* d_ab = nullptr;
    double* d_tau = nullptr;
    lv::BookRun* d_run = nullptr;
    lv::BookRun* h_run = nullptr;           // pinned; the graph copies from it
    double* d_sums = nullptr;
    double* d_out = nullptr;
    double* h_out = nullptr;                // pinned
    double* d_risk = nullptr;               // aggregated runs: per-surface sums
    double* d_rout = nullptr;               // aggregated runs: per-surface outputs
    double* h_rout = nullptr;               // pinned
    // scratch for the current launch shape
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned int* d_counter = nullptr;
    float* d_l1 = nullptr;
    float* d_ckpt = nullptr;
    // launch shape
    int block = 128, k = 4, item_tiles = 256, grid = 1, ppl = 1;
    size_t smem = 0;
    // stream and graph
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec_risk = nullptr;
};

namespace {

struct BookDevice {
    int prev = -1;
    explicit BookDevice(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~BookDevice()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void drop_graph(lv_book_s* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->exec_risk) cudaGraphExecDestroy(b->exec_risk);
    b->exec = nullptr;
    b->exec_risk = nullptr;
}

void free_book(lv_book_s* b)
{
    if (!b) return;
    drop_graph(b);
    cudaFree(b->d_surfs);
    cudaFree(b->d_insts);
    cudaFree(b->d_items);
    cudaFree(b->d_sig2);
    cudaFree(b->d_node);
    cudaFree(b->d_ab);
    cudaFree(b->d_tau);
    cudaFree(b->d_run);
    cudaFree(b->d_sums);
    cudaFree(b->d_out);
    cudaFree(b->d_risk);
    cudaFree(b->d_rout);
    cudaFree(b->d_scratch);
    cudaFreeHost(b->h_run);
    cudaFreeHost(b->h_out);
    cudaFreeHost(b->h_rout);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Work items: options longest (steps per path) first, each option's tiles
// split into items of `item_tiles` tiles, the items of one option consecutive.
std::vector<lv::BookItem> make_items(const std::vector<lv::BookInst>& insts, int item_tiles)
{
    std::vector<int> order(insts.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const double ca = (double)insts[a].N * (double)insts[a].n_paths;
        const double cc = (double)insts[c].N * (double)insts[c].n_paths;
        if (insts[a].N != insts[c].N) return insts[a].N > insts[c].N;
        return ca > cc;
    });
    std::vector<lv::BookItem> items;
    for (int o : order) {
        const int tiles = (int)((insts[o].n_paths + 31) / 32);
        for (int t = 0; t < tiles; t += item_tiles)
            items.push_back(lv::BookItem{o, t, std::min(item_tiles, tiles - t)});
    }
    return items;
}

// (Re)builds items and scratch for a launch shape; drops the captured graph.
lv_status configure(lv_book_s* b, int block, int k, int item_tiles, int ppl)
{
    drop_graph(b);
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    const size_t smem = lv::book_smem_bytes(b->max_I, b->max_Je, b->max_N, block, ppl);
    if (smem > 200 * 1024) return set_error(LV_EINVAL, "book grids too large for shared memory");
    int bps = 0;
    LV_BCUDA(lv::book_occupancy(block, k, ppl, smem, &bps));
    if (bps < 1) return set_error(LV_EINVAL, "book launch shape does not fit on an SM");
    std::vector<lv::BookItem> items = make_items(b->insts, item_tiles);
    cudaFree(b->d_items);
    b->d_items = nullptr;
    if (cudaMalloc(&b->d_items, sizeof(lv::BookItem) * items.size()) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LV_ENOMEM, "cannot allocate the work items");
    }
    LV_BCUDA(cudaMemcpy(b->d_items, items.data(), sizeof(lv::BookItem) * items.size(), cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    const int grid = std::max(1, std::min(bps * b->num_sms, b->n_items));
    const size_t warps = (size_t)grid * (block / 32);
    const size_t n_ck = (size_t)((b->max_N + k - 1) / k);
    size_t o = 256;
    const size_t off_l1 = o;
    o = up256(o + sizeof(float) * (size_t)grid * b->max_IJe);
    const size_t off_ck = o;
    o = up256(o + sizeof(float) * n_ck * warps * lv::book_ring_slots_per_warp() * ppl);
    if (o > b->scratch_bytes) {
        cudaFree(b->d_scratch);
        b->d_scratch = nullptr;
        b->scratch_bytes = 0;
        if (cudaMalloc(&b->d_scratch, o) != cudaSuccess) {
            cudaGetLastError();
            return set_error(LV_ENOMEM, "cannot allocate " + std::to_string(o) + " bytes of book scratch");
        }
        b->scratch_bytes = o;
    }
    char* base = static_cast<char*>(b->d_scratch);
    b->d_counter = reinterpret_cast<unsigned int*>(base);
    b->d_l1 = reinterpret_cast<float*>(base + off_l1);
    b->d_ckpt = reinterpret_cast<float*>(base + off_ck);
    b->block = block;
    b->k = k;
    b->item_tiles = item_tiles;
    b->ppl = ppl;
    b->grid = grid;
    b->smem = smem;
    return LV_OK;
}

lv::BookParams params(const lv_book_s* b)
{
    lv::BookParams P{};
    P.surfs = b->d_surfs;
    P.insts = b->d_insts;
    P.items = b->d_items;
    P.n_items = b->n_items;
    P.sig2 = b->d_sig2;
    P.node = b->d_node;
    P.ab = b->d_ab;
    P.tau = b->d_tau;
    P.run = b->d_run;
    P.item_counter = b->d_counter;
    P.sums = b->d_sums;
    P.risk = nullptr;
    P.l1 = b->d_l1;
    P.ckpt = b->d_ckpt;
    P.max_I = b->max_I;
    P.max_Je = b->max_Je;
    P.max_N = b->max_N;
    P.max_IJe = b->max_IJe;
    return P;
}

// Enqueue one run on the book's stream (zeroing, kernel, finalize into d_out).
lv_status enqueue_run(lv_book_s* b, double* d_out)
{
    const size_t n_out = (size_t)b->offsets.back();
    LV_BCUDA(cudaMemsetAsync(b->d_sums, 0, sizeof(double) * n_out, b->stream));
    LV_BCUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->stream));
    const lv::BookParams P = params(b);
    LV_BCUDA(lv::launch_book(P, b->grid, b->block, b->k, b->ppl, b->smem, b->stream));
    LV_BCUDA(lv::launch_book_finalize(P, (int)b->insts.size(), b->max_IJ, d_out, b->stream));
    return LV_OK;
}

// Enqueue one aggregated-risk run: per-option scalar sums, per-surface vega sums.
lv_status enqueue_risk(lv_book_s* b, double* d_out)
{
    const size_t n_out = (size_t)b->offsets.back();
    const size_t n_risk = (size_t)b->risk_offsets.back();
    LV_BCUDA(cudaMemsetAsync(b->d_sums, 0, sizeof(double) * n_out, b->stream));
    LV_BCUDA(cudaMemsetAsync(b->d_risk, 0, sizeof(double) * n_risk, b->stream));
    LV_BCUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->stream));
    lv::BookParams P = params(b);
    P.risk = b->d_risk;
    LV_BCUDA(lv::launch_book(P, b->grid, b->block, b->k, b->ppl, b->smem, b->stream));
    LV_BCUDA(lv::launch_book_risk_finalize(P, (int)b->surfs.size(), (int)b->insts.size(), b->max_IJ, d_out,
                                           b->stream));
    return LV_OK;
}

void set_run(lv_book_s* b, double S0, double r, uint64_t seed)
{
    b->h_run->log2_S0 = std::log2(S0);
    b->h_run->r = r;
    b->h_run->seed = seed;
}

lv_status check_run(double S0, double r)
{
    if (!std::isfinite(S0) || !(S0 > 0.0)) return set_error(LV_EINVAL, "S0 must be finite and > 0");
    if (!std::isfinite(r)) return set_error(LV_EINVAL, "r must be finite");
    return LV_OK;
}

std::string tune_key(const lv_book_s* b)
{
    int nb = 0;
    for (int n = b->max_N; n > 1; n >>= 1) ++nb;
    return "book|" + lv::gpu_name(b->device) + "|IJ" + std::to_string(b->max_IJ) + "|N2^" + std::to_string(nb) +
           "|insts" + std::to_string(b->insts.size());
}

bool read_tuned(const std::string& key, int* block, int* k, int* item_tiles, int* ppl)
{
    int v[4];
    if (!lv::tune_cache_lookup(key, v)) return false;
    if (!(v[1] == 4 || v[1] == 8) || v[0] < 32 || v[0] > 128 || v[0] % 32 != 0 || v[2] < 1) return false;
    if (v[3] != 1 && v[3] != 2) return false;
    *block = v[0];
    *k = v[1];
    *item_tiles = v[2];
    *ppl = v[3];
    return true;
}

void write_tuned(const std::string& key, int block, int k, int item_tiles, int ppl, double ms)
{
    const int v[4] = {block, k, item_tiles, ppl};
    lv::tune_cache_append(key, v, ms);
}

// One run through a CUDA graph captured on first use (per-option outputs, or
// with `risk` the aggregated per-surface risk): parameter upload, zeroing,
// the persistent kernel, the finalize and the copy back; then a host copy.
lv_status run_captured(lv_book_s* b, double S0, double r, uint64_t seed, bool risk, double* out)
{
    if (!b || !out) return set_error(LV_EINVAL, "NULL argument");
    lv_status st = check_run(S0, r);
    if (st != LV_OK) return st;
    BookDevice guard(b->device);
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    set_run(b, S0, r, seed);
    const size_t n_out = risk ? (size_t)b->risk_offsets.back() : (size_t)b->offsets.back();
    cudaGraphExec_t& exec = risk ? b->exec_risk : b->exec;
    double* d_res = risk ? b->d_rout : b->d_out;
    double* h_res = risk ? b->h_rout : b->h_out;
    if (!exec) {
        LV_BCUDA(lv::book_prepare(b->k, b->ppl));
        cudaGraph_t graph = nullptr;
        LV_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        lv_status cst = LV_OK;
        cudaError_t e = cudaMemcpyAsync(b->d_run, b->h_run, sizeof(lv::BookRun), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) cst = set_error(LV_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
        if (cst == LV_OK) cst = risk ? enqueue_risk(b, d_res) : enqueue_run(b, d_res);
        if (cst == LV_OK) {
            e = cudaMemcpyAsync(h_res, d_res, sizeof(double) * n_out, cudaMemcpyDeviceToHost, b->stream);
            if (e != cudaSuccess) cst = set_error(LV_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
        }
        const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
        if (cst != LV_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cst;
        }
        if (ee != cudaSuccess) return set_error(LV_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ee));
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            exec = nullptr;
            return set_error(LV_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        }
    }
    LV_BCUDA(cudaGraphLaunch(exec, b->stream));
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    std::memcpy(out, h_res, sizeof(double) * n_out);
    return LV_OK;
}

}  // namespace

extern "C" {

lv_status lv_book_create(const lv_surface_t* surfaces, int32_t n_surfaces, const lv_instrument* insts,
                         int32_t n_insts, lv_book_t* out)
{
    if (!out || !surfaces || !insts) return set_error(LV_EINVAL, "NULL argument");
    if (n_surfaces < 1 || n_insts < 1) return set_error(LV_EINVAL, "a book needs surfaces and options");
    if (n_insts > 65535) return set_error(LV_EINVAL, "a book holds at most 65535 options");
    int device = -1;
    for (int s = 0; s < n_surfaces; ++s) {
        if (!surfaces[s]) return set_error(LV_EINVAL, "NULL surface");
        if (surfaces[s]->interp != LV_INTERP_S || surfaces[s]->scheme != LV_SCHEME_LOG)
            return set_error(LV_EINVAL, "a book runs the main reading (LV_INTERP_S, LV_SCHEME_LOG) only");
        if (s == 0) device = surfaces[s]->device;
        else if (surfaces[s]->device != device) return set_error(LV_EINVAL, "surfaces on different devices");
    }
    for (int o = 0; o < n_insts; ++o) {
        const lv_instrument& q = insts[o];
        if (q.surface < 0 || q.surface >= n_surfaces) return set_error(LV_EINVAL, "option surface index out of range");
        if (q.phi != 1 && q.phi != -1) return set_error(LV_EINVAL, "phi must be +1 or -1");
        if (!std::isfinite(q.K) || q.K < 0.0) return set_error(LV_EINVAL, "K must be finite and >= 0");
        if (!std::isfinite(q.T) || !(q.T > 0.0)) return set_error(LV_EINVAL, "T must be finite and > 0");
        if (q.n_steps < 1 || q.n_steps > LV_MAX_STEPS) return set_error(LV_EINVAL, "n_steps out of range");
        if (q.n_paths < 1 || q.n_paths > 0x7fffffffLL) return set_error(LV_EINVAL, "n_paths out of range");
        if (q.stream_id >= 65536u) return set_error(LV_EINVAL, "stream_id must be < 65536");
    }
    lv_book_s* b = new (std::nothrow) lv_book_s();
    if (!b) return set_error(LV_ENOMEM, "out of host memory");
    BookDevice guard(device);
    b->device = device;
    auto bail = [&](lv_status st) {
        free_book(b);
        return st;
    };
    if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(set_error(LV_ECUDA, "cannot read the SM count"));

    // grids: concatenate every surface's device arrays
    long long n_sig = 0, n_node = 0, n_ab = 0, n_tau = 0;
    for (int s = 0; s < n_surfaces; ++s) {
        const lv_surface_s* h = surfaces[s];
        lv::BookSurf bs{};
        bs.I = h->I;
        bs.J = h->J;
        bs.Je = h->Je;
        bs.log_uniform = h->log_uniform;
        bs.cell_scale = h->cell_scale;
        bs.cell_shift = h->cell_shift;
        bs.s_lo = h->s_lo;
        bs.s_hi = h->s_hi;
        bs.off_sig2 = n_sig;
        bs.off_node = n_node;
        bs.off_ab = n_ab;
        bs.off_tau = n_tau;
        bs.risk_off = s == 0 ? 0 : b->surfs.back().risk_off + 3 + (long long)b->surfs.back().I * b->surfs.back().J;
        n_sig += (long long)h->Je * (h->I - 1);
        n_node += h->I;
        n_ab += h->I;
        n_tau += h->J;
        b->surfs.push_back(bs);
        b->max_I = std::max(b->max_I, h->I);
        b->max_J = std::max(b->max_J, h->J);
        b->max_Je = std::max(b->max_Je, h->Je);
        b->max_IJe = std::max(b->max_IJe, h->Je * h->I);
        b->max_IJ = std::max(b->max_IJ, h->I * h->J);
    }
    b->offsets.assign(1, 0);
    for (int o = 0; o < n_insts; ++o) {
        const lv_instrument& q = insts[o];
        lv::BookInst bi{};
        bi.surf = q.surface;
        bi.N = q.n_steps;
        bi.phi = q.phi;
        bi.stream_id = (int)q.stream_id;
        bi.K = q.K;
        bi.T = q.T;
        bi.n_paths = q.n_paths;
        bi.out_off = b->offsets.back();
        bi.w = 1.0;
        bi.scale = 1.0 / (double)q.n_paths;
        b->insts.push_back(bi);
        const lv::BookSurf& s = b->surfs[q.surface];
        b->offsets.push_back(b->offsets.back() + 3 + (int64_t)s.I * s.J);
        b->max_N = std::max(b->max_N, q.n_steps);
        b->total_paths += q.n_paths;
    }
    const size_t n_out = (size_t)b->offsets.back();
    b->risk_offsets.assign(1, 0);
    for (const lv::BookSurf& bs : b->surfs) b->risk_offsets.push_back(bs.risk_off + 3 + (int64_t)bs.I * bs.J);
    const size_t n_risk = (size_t)b->risk_offsets.back();
    if (cudaMalloc(&b->d_surfs, sizeof(lv::BookSurf) * b->surfs.size()) != cudaSuccess ||
        cudaMalloc(&b->d_insts, sizeof(lv::BookInst) * b->insts.size()) != cudaSuccess ||
        cudaMalloc(&b->d_sig2, sizeof(float2) * n_sig) != cudaSuccess ||
        cudaMalloc(&b->d_node, sizeof(float) * n_node) != cudaSuccess ||
        cudaMalloc(&b->d_ab, sizeof(float2) * n_ab) != cudaSuccess ||
        cudaMalloc(&b->d_tau, sizeof(double) * n_tau) != cudaSuccess ||
        cudaMalloc(&b->d_run, sizeof(lv::BookRun)) != cudaSuccess ||
        cudaMalloc(&b->d_sums, sizeof(double) * n_out) != cudaSuccess ||
        cudaMalloc(&b->d_out, sizeof(double) * n_out) != cudaSuccess ||
        cudaMalloc(&b->d_risk, sizeof(double) * n_risk) != cudaSuccess ||
        cudaMalloc(&b->d_rout, sizeof(double) * n_risk) != cudaSuccess ||
        cudaMallocHost(&b->h_run, sizeof(lv::BookRun)) != cudaSuccess ||
        cudaMallocHost(&b->h_out, sizeof(double) * n_out) != cudaSuccess ||
        cudaMallocHost(&b->h_rout, sizeof(double) * n_risk) != cudaSuccess) {
        cudaGetLastError();
        return bail(set_error(LV_ENOMEM, "book allocation failed"));
    }
    for (int s = 0; s < n_surfaces; ++s) {
        const lv_surface_s* h = surfaces[s];
        const lv::BookSurf& bs = b->surfs[s];
        if (cudaMemcpy(b->d_sig2 + bs.off_sig2, h->d_sig, sizeof(float2) * h->Je * (h->I - 1),
                       cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemcpy(b->d_node + bs.off_node, h->d_node, sizeof(float) * h->I, cudaMemcpyDeviceToDevice) !=
                cudaSuccess ||
            cudaMemcpy(b->d_ab + bs.off_ab, h->d_ab, sizeof(float2) * h->I, cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemcpy(b->d_tau + bs.off_tau, h->d_tau, sizeof(double) * h->J, cudaMemcpyDeviceToDevice) !=
                cudaSuccess)
            return bail(set_error(LV_ECUDA, "copying a surface into the book failed"));
    }
    if (cudaMemcpy(b->d_surfs, b->surfs.data(), sizeof(lv::BookSurf) * b->surfs.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_insts, b->insts.data(), sizeof(lv::BookInst) * b->insts.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return bail(set_error(LV_ECUDA, "uploading the book tables failed"));
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(set_error(LV_ECUDA, "cannot create the book's stream"));
    b->own_stream = true;
    int block = 128, k = 4, item_tiles = 256, ppl = 1;
    read_tuned(tune_key(b), &block, &k, &item_tiles, &ppl);
    lv_status st = configure(b, block, k, item_tiles, ppl);
    if (st != LV_OK) return bail(st);
    *out = b;
    return LV_OK;
}

void lv_book_destroy(lv_book_t b)
{
    if (!b) return;
    BookDevice guard(b->device);
    cudaStreamSynchronize(b->stream);
    free_book(b);
}

lv_status lv_book_output_offsets(lv_book_t b, int64_t* offsets)
{
    if (!b || !offsets) return set_error(LV_EINVAL, "NULL argument");
    std::memcpy(offsets, b->offsets.data(), sizeof(int64_t) * b->offsets.size());
    return LV_OK;
}

lv_status lv_book_set_stream(lv_book_t b, void* cuda_stream)
{
    if (!b) return set_error(LV_EINVAL, "NULL book");
    BookDevice guard(b->device);
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    drop_graph(b);
    if (cuda_stream) {
        if (b->own_stream) cudaStreamDestroy(b->stream);
        b->own_stream = false;
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else if (!b->own_stream) {
        LV_BCUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    return LV_OK;
}

lv_status lv_book_run_device(lv_book_t b, double S0, double r, uint64_t seed, double* d_out)
{
    if (!b || !d_out) return set_error(LV_EINVAL, "NULL argument");
    lv_status st = check_run(S0, r);
    if (st != LV_OK) return st;
    BookDevice guard(b->device);
    // the pinned parameter block may still feed an earlier asynchronous copy
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    set_run(b, S0, r, seed);
    LV_BCUDA(cudaMemcpyAsync(b->d_run, b->h_run, sizeof(lv::BookRun), cudaMemcpyHostToDevice, b->stream));
    return enqueue_run(b, d_out);
}

lv_status lv_book_run(lv_book_t b, double S0, double r, uint64_t seed, double* out)
{
    return run_captured(b, S0, r, seed, false, out);
}

lv_status lv_book_run_risk(lv_book_t b, double S0, double r, uint64_t seed, double* out)
{
    return run_captured(b, S0, r, seed, true, out);
}

lv_status lv_book_run_risk_device(lv_book_t b, double S0, double r, uint64_t seed, double* d_out)
{
    if (!b || !d_out) return set_error(LV_EINVAL, "NULL argument");
    lv_status st = check_run(S0, r);
    if (st != LV_OK) return st;
    BookDevice guard(b->device);
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    set_run(b, S0, r, seed);
    LV_BCUDA(cudaMemcpyAsync(b->d_run, b->h_run, sizeof(lv::BookRun), cudaMemcpyHostToDevice, b->stream));
    return enqueue_risk(b, d_out);
}

lv_status lv_book_set_weights(lv_book_t b, const double* weights)
{
    if (!b || !weights) return set_error(LV_EINVAL, "NULL argument");
    for (size_t o = 0; o < b->insts.size(); ++o)
        if (!std::isfinite(weights[o])) return set_error(LV_EINVAL, "weights must be finite");
    BookDevice guard(b->device);
    // an enqueued run may still read the table
    LV_BCUDA(cudaStreamSynchronize(b->stream));
    for (size_t o = 0; o < b->insts.size(); ++o) {
        b->insts[o].w = weights[o];
        b->insts[o].scale = weights[o] / (double)b->insts[o].n_paths;
    }
    LV_BCUDA(cudaMemcpy(b->d_insts, b->insts.data(), sizeof(lv::BookInst) * b->insts.size(),
                        cudaMemcpyHostToDevice));
    return LV_OK;
}

lv_status lv_book_risk_offsets(lv_book_t b, int64_t* offsets)
{
    if (!b || !offsets) return set_error(LV_EINVAL, "NULL argument");
    std::memcpy(offsets, b->risk_offsets.data(), sizeof(int64_t) * b->risk_offsets.size());
    return LV_OK;
}

lv_status lv_book_set_launch(lv_book_t b, int32_t block, int32_t k, int32_t item_paths, int32_t ppl)
{
    if (!b) return set_error(LV_EINVAL, "NULL book");
    if (block < 32 || block > 128 || block % 32 != 0)
        return set_error(LV_EINVAL, "block must be a multiple of 32 in [32, 128]");
    if (k != 4 && k != 8) return set_error(LV_EINVAL, "k must be 4 or 8");
    if (item_paths < 32 || item_paths % 32 != 0) return set_error(LV_EINVAL, "item_paths must be a multiple of 32");
    if (ppl != 1 && ppl != 2) return set_error(LV_EINVAL, "paths per lane must be 1 or 2");
    BookDevice guard(b->device);
    return configure(b, block, k, item_paths / 32, ppl);
}

lv_status lv_book_paths_per_lane(lv_book_t b, int32_t* ppl)
{
    if (!b || !ppl) return set_error(LV_EINVAL, "NULL argument");
    *ppl = b->ppl;
    return LV_OK;
}

lv_status lv_book_tune(lv_book_t b, double S0, double r, uint64_t seed, int32_t* out_block, int32_t* out_k,
                       int32_t* out_item_paths, double* out_ms)
{
    if (!b) return set_error(LV_EINVAL, "NULL book");
    lv_status st = check_run(S0, r);
    if (st != LV_OK) return st;
    BookDevice guard(b->device);
    const int blocks[] = {64, 128};
    const int ks[] = {4, 8};
    const int items[] = {64, 256, 1024};
    double best = 1e300;
    int bb = b->block, bk = b->k, bi = b->item_tiles, bp = b->ppl;
    cudaEvent_t e0, e1;
    LV_BCUDA(cudaEventCreate(&e0));
    LV_BCUDA(cudaEventCreate(&e1));
    for (int blk : blocks)
        for (int k : ks)
            for (int it : items)
            for (int ppl = 1; ppl <= 2; ++ppl) {
                st = configure(b, blk, k, it, ppl);
                if (st != LV_OK) continue;
                float ms = 0.0f, t = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    if (lv_book_run_device(b, S0, r, seed, b->d_out) != LV_OK) break;
                    // time the enqueued run: a second identical run between two events
                    cudaEventRecord(e0, b->stream);
                    enqueue_run(b, b->d_out);
                    cudaEventRecord(e1, b->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) break;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t = std::min(t, ms);
                }
                if (t < best) {
                    best = t;
                    bb = blk;
                    bk = k;
                    bi = it;
                    bp = ppl;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st = configure(b, bb, bk, bi, bp);
    if (st != LV_OK) return st;
    if (best < 1e299) write_tuned(tune_key(b), bb, bk, bi, bp, best);
    if (out_block) *out_block = bb;
    if (out_k) *out_k = bk;
    if (out_item_paths) *out_item_paths = bi * 32;
    if (out_ms) *out_ms = best;
    return LV_OK;
}

}  // extern "C"
