// api.cu -- the extern "C" entry points of libditer (declared in include/diter.h).
//
// This file does argument checks, host/device pointer detection, ownership and
// error reporting.  All arithmetic of the method runs in the kernels of
// graph_build.cu, sweep.cu and power.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace diter {

static thread_local std::string g_last_error;

di_status set_error(di_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

di_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky launch error so the next call starts clean
    if (e == cudaErrorMemoryAllocation)
        return set_error(DI_ENOMEM, std::string("out of device memory in ") + what);
    return set_error(DI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// the address a kernel writes p through: p itself for device memory, the mapped address
// for page-locked host memory, NULL for pageable host memory (the caller stages the copy)
void *kernel_ptr(void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    return nullptr;
}

// Graph creation and solves allocate their buffers with cudaMallocAsync from the device's
// default memory pool.  By default the pool hands freed memory back to the driver at every
// synchronization, so the next allocation of the same size goes to the driver again; keeping
// freed memory in the pool (this process only, for its lifetime) makes repeated creates and
// solves allocate from the pool.
static void keep_pool_memory(int dev) {
    static bool done[64] = {};
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

static di_status copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return DI_OK;
    DI_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return DI_OK;
}

// Small page-locked host blocks (each graph's solve and power status, read back after every
// solve) from process-wide slabs: a cudaMallocHost / cudaFreeHost pair took about 0.27 ms on a
// Grace host, most of the fixed cost of creating and freeing a graph.  A slab is never
// returned; its blocks are reused by later graphs.
constexpr size_t kPinBlock = 512;
constexpr int kPinPerSlab = 128;
std::mutex g_pin_mu;
std::vector<void *> g_pin_free;

cudaError_t pinned_block(void **out) {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (g_pin_free.empty()) {
        char *slab = nullptr;
        cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(&slab), kPinBlock * kPinPerSlab);
        if (e != cudaSuccess) return e;
        for (int k = kPinPerSlab - 1; k >= 0; --k) g_pin_free.push_back(slab + kPinBlock * k);
    }
    *out = g_pin_free.back();
    g_pin_free.pop_back();
    return cudaSuccess;
}

void pinned_release(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(p);
}
static_assert(sizeof(SolveState) <= kPinBlock && sizeof(PowerState) <= kPinBlock, "status blocks fit a pinned block");

static void free_graph(di_graph *g) {
    if (!g) return;
    if (g->stream || g->cap) cudaStreamSynchronize(g->stream);
    for (int k = 0; k < kSweepSlots; ++k) {
        if (g->exec[k]) cudaGraphExecDestroy(g->exec[k]);
        if (g->graph[k]) cudaGraphDestroy(g->graph[k]);
    }
    pool_free(g->bp, g->stream);
    void *bufs[] = {g->row_ptr, g->col_idx, g->in_ptr, g->in_src, g->in_dst, g->wpull, g->bin_of, g->V,
                    g->inv_deg, g->inv_deg32, g->hot_ids, g->perm, g->new_of, g->rec64, g->rec32,
                    g->wsel[0], g->wsel[1], g->rowhash, g->region, g->fcount, g->pre, g->sel, g->cls, g->F64, g->F32, g->H, g->part, g->st,
                    g->trace, g->X, g->Z[0], g->Z[1], g->Y, g->ppart, g->pst};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, g->stream);
    cudaStreamSynchronize(g->stream);
    pinned_release(g->h_st);
    pinned_release(g->h_pst);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    for (int k = 0; k < 4; ++k)
        if (g->pev[k]) cudaEventDestroy(g->pev[k]);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete[] g->sweep_ms;
    cudaGetLastError();
    delete g;
}

// The arguments of a batch of k personalized queries, checked and copied to the host:
// hp = seed_ptr[k+1], hs = seeds, hw = weights (empty when w is NULL).
di_status batch_args(di_graph *g, int k, const int32_t *seed_ptr, const int32_t *seeds, const double *w, double tol,
                     std::vector<int32_t> &hp, std::vector<int32_t> &hs, std::vector<double> &hw) {
    if (k < 1 || k > kLanes) return set_error(DI_EINVAL, "a batch holds 1 to 64 queries");
    if (!seed_ptr || !seeds) return set_error(DI_EINVAL, "seed_ptr and seeds are required");
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    cudaStream_t s = g->stream;
    hp.assign((size_t)k + 1, 0);
    DI_CUDA(cudaMemcpyAsync(hp.data(), seed_ptr, sizeof(int32_t) * (k + 1),
                            is_device_ptr(seed_ptr) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if (hp[0] != 0) return set_error(DI_EINVAL, "seed_ptr[0] must be 0");
    for (int q = 0; q < k; ++q)
        if (hp[q + 1] <= hp[q]) return set_error(DI_EINVAL, "every query needs at least one seed");
    const int total = hp[k];
    hs.assign((size_t)total, 0);
    hw.assign(w ? (size_t)total : 0, 0.0);
    DI_CUDA(cudaMemcpyAsync(hs.data(), seeds, sizeof(int32_t) * total,
                            is_device_ptr(seeds) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    if (w)
        DI_CUDA(cudaMemcpyAsync(hw.data(), w, sizeof(double) * total,
                                is_device_ptr(w) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < k; ++q) {
        double sum = 0.0;
        for (int t = hp[q]; t < hp[q + 1]; ++t) {
            if (hs[t] < 0 || hs[t] >= g->n) return set_error(DI_EINVAL, "seed id outside [0, n)");
            const double wt = w ? hw[t] : 1.0;
            if (!std::isfinite(wt) || wt < 0.0) return set_error(DI_EINVAL, "seed weights must be finite and >= 0");
            sum += wt;
        }
        if (!(sum > 0.0)) return set_error(DI_EINVAL, "each query's seed weights need a positive sum");
    }
    return DI_OK;
}

static di_status check_graph(const di_graph *g) {
    if (!g) return set_error(DI_EINVAL, "graph is NULL");
    if (g->untrusted)
        return set_error(DI_ETIMEOUT, "an earlier sweep scan gave up waiting with bulk copies in flight; "
                                      "this graph's device state is not trusted: free it");
    return DI_OK;
}

}  // namespace diter

using namespace diter;

extern "C" {

const char *di_last_error(void) { return g_last_error.c_str(); }

const char *di_version(void) { return "libditer 0.1 (D-iteration, sm_103a)"; }

di_status di_selftest_wait(int32_t polls, int32_t ctas, int32_t *gave_up) {
    g_last_error.clear();
    if (!gave_up) return set_error(DI_EINVAL, "gave_up is NULL");
    if (polls < 1 || polls > (1 << 24)) return set_error(DI_EINVAL, "polls must be in [1, 2^24]");
    if (ctas < 1 || ctas > 1024) return set_error(DI_EINVAL, "ctas must be in [1, 1024]");
    *gave_up = 0;
    return selftest_wait(polls, ctas, gave_up);
}

di_status di_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int64_t nnz, double d,
                          const double *V, void *stream, di_graph **out) {
    g_last_error.clear();
    if (!out) return set_error(DI_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n == INT32_MAX) return set_error(DI_EINVAL, "n must be in [1, 2^31-2]");
    if (nnz < 0 || nnz >= INT32_MAX) return set_error(DI_EINVAL, "nnz must be in [0, 2^31-1)");
    if (!row_ptr) return set_error(DI_EINVAL, "row_ptr is NULL");
    if (nnz > 0 && !col_idx) return set_error(DI_EINVAL, "col_idx is NULL");
    if (!(d > 0.0 && d < 1.0)) return set_error(DI_EINVAL, "d must satisfy 0 < d < 1");
    di_graph *g = new di_graph();
    g->n = n;
    g->nnz = nnz;
    g->d = d;
    g->stream = (cudaStream_t)stream;
    auto fail = [&](di_status s) {
        std::string msg = g_last_error;
        free_graph(g);
        g_last_error = msg;
        return s;
    };
    cudaError_t e = cudaGetDevice(&g->dev);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGetDevice"));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->dev);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
    g->num_sms = sms > 0 ? sms : 152;
    keep_pool_memory(g->dev);
    if ((e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaStreamCreate"));
    if ((e = cudaEventCreate(&g->ev0)) != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaEventCreate(&g->ev1)) != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate"));
    for (int k = 0; k < 4; ++k)
        if ((e = cudaEventCreate(&g->pev[k])) != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate"));
    void *hb = nullptr;
    if ((e = pinned_block(&hb)) != cudaSuccess) return fail(cuda_fail(e, "cudaMallocHost"));
    g->h_st = static_cast<SolveState *>(hb);
    if ((e = pinned_block(&hb)) != cudaSuccess) return fail(cuda_fail(e, "cudaMallocHost"));
    g->h_pst = static_cast<PowerState *>(hb);
    memset(g->h_st, 0, sizeof(SolveState));
    g->sweep_ms = new float[2 * kTraceCap]();
    memset(g->h_pst, 0, sizeof(PowerState));
    cudaStream_t s = g->stream;
    if ((e = cudaMallocAsync(&g->row_ptr, sizeof(int) * (size_t)(n + 1), s)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMallocAsync(row_ptr)"));
    if ((e = cudaMallocAsync(&g->col_idx, sizeof(int) * (size_t)std::max<int64_t>(nnz, 1), s)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMallocAsync(col_idx)"));
    // a host col_idx is copied by build_graph, in pieces overlapped with its in-degree count
    const bool col_on_host = nnz > 0 && !is_device_ptr(col_idx);
    di_status r = copy_in(g->row_ptr, row_ptr, sizeof(int) * (size_t)(n + 1), s);
    if (r == DI_OK && !col_on_host) r = copy_in(g->col_idx, col_idx, sizeof(int) * (size_t)nnz, s);
    if (r != DI_OK) return fail(r);
    if (V) {
        if ((e = cudaMallocAsync(&g->V, sizeof(double) * (size_t)n, s)) != cudaSuccess)
            return fail(cuda_fail(e, "cudaMallocAsync(V)"));
        if ((r = copy_in(g->V, V, sizeof(double) * (size_t)n, s)) != DI_OK) return fail(r);
        if ((r = validate_v(g, g->V)) != DI_OK) return fail(r);
    }
    if ((r = build_graph(g, col_on_host ? col_idx : nullptr)) != DI_OK) return fail(r);
    if ((r = sweep_alloc(g)) != DI_OK) return fail(r);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_fail(e, "graph create"));
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "graph create"));
    *out = g;
    return DI_OK;
}

void di_free(di_graph *g) { free_graph(g); }

di_status di_graph_info(const di_graph *g, int32_t *n, int64_t *nnz, double *d) {
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (d) *d = g->d;
    return DI_OK;
}

}  // extern "C"

namespace diter {
namespace {
__global__ void k_outdeg(int n, const int *__restrict__ row_ptr, int *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = row_ptr[i + 1] - row_ptr[i];
}
}  // namespace

// the Theorem 1 check and load of a saved state (sweep.cu)
di_status set_state(di_graph *g, const double *F_in, bool F_dev, const double *H_in, bool H_dev, double rtol,
                    double *deviation);

static di_status copy_out(void *dst, const void *src_dev, size_t bytes, cudaStream_t s) {
    if (!dst || bytes == 0) return DI_OK;
    DI_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s));
    return DI_OK;
}
}  // namespace diter

extern "C" {

di_status di_graph_export(const di_graph *g, int32_t *perm, int32_t *outdeg, int32_t *in_ptr, int32_t *in_src,
                          int32_t *bin_of, int32_t *in_bin_of, int32_t *cuts) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (in_ptr || in_src || in_bin_of) {
        di_status tr = build_transpose(const_cast<di_graph *>(g));  // built on first use
        if (tr != DI_OK) return tr;
    }
    cudaStream_t s = g->stream;
    const size_t n = (size_t)g->n;
    if (outdeg) {
        int *tmp = nullptr;
        DI_CUDA(cudaMallocAsync(&tmp, sizeof(int) * n, s));
        k_outdeg<<<std::max(1, std::min(1216, (int)((n + 255) / 256))), 256, 0, s>>>(g->n, g->row_ptr, tmp);
        di_status r = copy_out(outdeg, tmp, sizeof(int) * n, s);
        cudaFreeAsync(tmp, s);
        if (r != DI_OK) return r;
    }
    di_status r = copy_out(perm, g->perm, sizeof(int) * n, s);
    if (r == DI_OK) r = copy_out(in_ptr, g->in_ptr, sizeof(int) * (n + 1), s);
    if (r == DI_OK) r = copy_out(in_src, g->in_src, sizeof(int) * (size_t)g->nnz, s);
    if (r == DI_OK) r = copy_out(bin_of, g->bin_of, sizeof(int) * n, s);
    if (r == DI_OK && in_bin_of) {
        int *tmp = nullptr;
        DI_CUDA(cudaMallocAsync(&tmp, sizeof(int) * (size_t)n, s));
        r = in_degree_classes(const_cast<di_graph *>(g), tmp);
        if (r == DI_OK) r = copy_out(in_bin_of, tmp, sizeof(int) * n, s);
        cudaFreeAsync(tmp, s);
    }
    if (r != DI_OK) return r;
    DI_CUDA(cudaStreamSynchronize(s));
    if (cuts) {
        cuts[0] = g->cut1;
        cuts[1] = g->cut2;
        cuts[2] = kInCut1;
        cuts[3] = kInCut2;
    }
    return DI_OK;
}

di_status di_graph_hot_targets(const di_graph *g, int32_t *ids, int32_t *count) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (count) *count = g->n_hot;
    if (ids && g->n_hot > 0) {
        di_status r = copy_out(ids, g->hot_ids, sizeof(int) * (size_t)g->n_hot, g->stream);
        if (r != DI_OK) return r;
        DI_CUDA(cudaStreamSynchronize(g->stream));
    }
    return DI_OK;
}

di_status di_solve_ex(di_graph *g, const di_solve_opts *opts, double *H_out, di_stats *st) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (!opts) return set_error(DI_EINVAL, "opts is NULL");
    di_solve_opts o = *opts;
    if (!(o.tol > 0.0) || !std::isfinite(o.tol)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    if (!(o.beta >= 0.0) || !std::isfinite(o.beta)) return set_error(DI_EINVAL, "beta must be finite and >= 0");
    if (o.prec != DI_FP64 && o.prec != DI_FP32_MIXED) return set_error(DI_EINVAL, "prec must be DI_FP64 or DI_FP32_MIXED");
    if (o.select < DI_SELECT_REF || o.select > DI_SELECT_OP2) return set_error(DI_EINVAL, "select must be 0, 1 or 2");
    if (o.direction < 0 || o.direction > 2) return set_error(DI_EINVAL, "direction must be 0, 1 or 2");
    if (o.scan_wait_polls < 0) return set_error(DI_EINVAL, "scan_wait_polls must be >= 0");
    return run_solve(g, o, nullptr, nullptr, 0, 1.0, H_out, is_device_ptr(H_out), st);
}

di_status di_solve_update(di_graph *g_old, di_graph *g_new, const di_solve_opts *opts, double *H_out, di_stats *st) {
    g_last_error.clear();
    if (!g_old || !g_new) return set_error(DI_EINVAL, "graph is NULL");
    if (di_status cr = check_graph(g_old); cr != DI_OK) return cr;
    if (di_status cr = check_graph(g_new); cr != DI_OK) return cr;
    if (!opts) return set_error(DI_EINVAL, "opts is NULL");
    di_solve_opts o = *opts;
    if (!(o.tol > 0.0) || !std::isfinite(o.tol)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    if (!(o.beta >= 0.0) || !std::isfinite(o.beta)) return set_error(DI_EINVAL, "beta must be finite and >= 0");
    if (o.prec != DI_FP64) return set_error(DI_EINVAL, "a graph update continues an FP64 state: prec must be DI_FP64");
    if (o.select < DI_SELECT_REF || o.select > DI_SELECT_OP2) return set_error(DI_EINVAL, "select must be 0, 1 or 2");
    if (o.direction < 0 || o.direction > 2) return set_error(DI_EINVAL, "direction must be 0, 1 or 2");
    if (o.scan_wait_polls < 0) return set_error(DI_EINVAL, "scan_wait_polls must be >= 0");
    if (g_old->n != g_new->n) return set_error(DI_EINVAL, "the updated graph must have the same nodes");
    if (g_old->d != g_new->d) return set_error(DI_EINVAL, "the updated graph must have the same d");
    if (g_old->last_prec != DI_FP64 || !g_old->F64)
        return set_error(DI_EINVAL, "g_old holds no FP64 D-iteration state: solve it with prec = DI_FP64 first");
    return run_update(g_old, g_new, o, H_out, is_device_ptr(H_out), st);
}

di_status di_solve(di_graph *g, double tol, int64_t max_edge_pushes, di_prec prec, double *H_out, int normalize,
                   di_stats *st) {
    di_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.tol = tol;
    o.beta = 0.5;
    o.max_edge_pushes = max_edge_pushes;
    o.prec = (int32_t)prec;
    o.normalize = normalize;
    return di_solve_ex(g, &o, H_out, st);
}

di_status di_query(di_graph *g, const int32_t *seeds, const double *w, int32_t nseeds, double tol, di_prec prec,
                   double *H_out, di_stats *st) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (nseeds < 1 || !seeds) return set_error(DI_EINVAL, "a query needs at least one seed");
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    if (prec != DI_FP64 && prec != DI_FP32_MIXED) return set_error(DI_EINVAL, "prec must be DI_FP64 or DI_FP32_MIXED");
    cudaStream_t s = g->stream;
    std::vector<int32_t> hs((size_t)nseeds);
    std::vector<double> hw(w ? (size_t)nseeds : 0);
    DI_CUDA(cudaMemcpyAsync(hs.data(), seeds, sizeof(int32_t) * nseeds,
                            is_device_ptr(seeds) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    if (w)
        DI_CUDA(cudaMemcpyAsync(hw.data(), w, sizeof(double) * nseeds,
                                is_device_ptr(w) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    double wsum = 0.0;
    for (int k = 0; k < nseeds; ++k) {
        if (hs[k] < 0 || hs[k] >= g->n) return set_error(DI_EINVAL, "seed id outside [0, n)");
        double wk = w ? hw[k] : 1.0;
        if (!std::isfinite(wk) || wk < 0.0) return set_error(DI_EINVAL, "seed weights must be finite and >= 0");
        wsum += wk;
    }
    if (!(wsum > 0.0)) return set_error(DI_EINVAL, "seed weights must have a positive sum");
    int *dseeds = nullptr;
    double *dw = nullptr;
    DI_CUDA(cudaMallocAsync(&dseeds, sizeof(int) * nseeds, s));
    DI_CUDA(cudaMemcpyAsync(dseeds, hs.data(), sizeof(int) * nseeds, cudaMemcpyHostToDevice, s));
    if (w) {
        DI_CUDA(cudaMallocAsync(&dw, sizeof(double) * nseeds, s));
        DI_CUDA(cudaMemcpyAsync(dw, hw.data(), sizeof(double) * nseeds, cudaMemcpyHostToDevice, s));
    }
    di_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.tol = tol;
    o.beta = 0.5;
    o.prec = (int32_t)prec;
    di_status r = run_solve(g, o, dseeds, dw, nseeds, wsum, H_out, is_device_ptr(H_out), st);
    cudaFreeAsync(dseeds, s);
    if (dw) cudaFreeAsync(dw, s);
    return r;
}

di_status di_query_batch(di_graph *g, int32_t k, const int32_t *seed_ptr, const int32_t *seeds, const double *w,
                         double tol, double *H_out, di_stats *st_q, di_stats *st_all) {
    return di_query_batch_ex(g, k, seed_ptr, seeds, w, tol, 0, H_out, st_q, st_all, nullptr);
}

di_status di_query_batch_ex(di_graph *g, int32_t k, const int32_t *seed_ptr, const int32_t *seeds, const double *w,
                            double tol, int32_t profile, double *H_out, di_stats *st_q, di_stats *st_all,
                            di_profile *prof) {
    g_last_error.clear();
    if (profile != 0 && profile != 1) return set_error(DI_EINVAL, "profile must be 0 or 1");
    if (profile && !prof) return set_error(DI_EINVAL, "prof is NULL");
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    std::vector<int32_t> hp, hs;
    std::vector<double> hw;
    if (di_status r = batch_args(g, k, seed_ptr, seeds, w, tol, hp, hs, hw); r != DI_OK) return r;
    return run_query_batch(g, k, hp.data(), hs.data(), w ? hw.data() : nullptr, tol, -1.0, 1000000, H_out,
                           is_device_ptr(H_out), st_q, st_all, profile ? prof : nullptr);
}

di_status di_power(di_graph *g, double tol, int32_t max_iter, double *X_out, di_stats *st) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    if (max_iter <= 0) max_iter = 100000;
    return run_power(g, tol, max_iter, 0, X_out, is_device_ptr(X_out), st);
}

di_status di_power_ex(di_graph *g, double tol, int32_t max_iter, int32_t profile, double *X_out, di_stats *st,
                      double *pull_ms, double *finalize_ms) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(DI_EINVAL, "tol must be finite and > 0");
    if (max_iter <= 0) max_iter = 100000;
    di_status r = run_power(g, tol, max_iter, profile, X_out, is_device_ptr(X_out), st);
    if (pull_ms) *pull_ms = g->pprof_ms[0];
    if (finalize_ms) *finalize_ms = g->pprof_ms[1];
    return r;
}

di_status di_get_trace(const di_graph *g, di_sweep_record *out, int32_t cap, int32_t *count) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    int avail = g->last_trace_on ? std::min(g->h_st->sweeps, kTraceCap) : 0;
    if (count) *count = avail;
    int k = std::min(avail, std::max(0, (int)cap));
    if (out && k > 0) {
        DI_CUDA(cudaMemcpyAsync(out, g->trace, sizeof(di_sweep_record) * k, cudaMemcpyDeviceToHost, g->stream));
        DI_CUDA(cudaStreamSynchronize(g->stream));
        if (g->sweep_ms && g->prof.sweeps == avail)
            for (int i = 0; i < k; ++i) {
                out[i].scan_ms = g->sweep_ms[2 * i];
                out[i].push_ms = g->sweep_ms[2 * i + 1];
            }
    }
    return DI_OK;
}

di_status di_get_profile(const di_graph *g, di_profile *out) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (!out) return set_error(DI_EINVAL, "out is NULL");
    *out = g->prof;
    return DI_OK;
}

int32_t di_debug_build(void) {
#ifdef DI_DEBUG
    return 1;
#else
    return 0;
#endif
}

di_status di_debug_selftest(uint64_t *word) {
    g_last_error.clear();
#ifdef DI_DEBUG
    unsigned long long w = 0;
    const di_status r = debug_selftest(&w);
    if (word) *word = (uint64_t)w;
    return r;
#else
    if (word) *word = 0;
    return set_error(DI_EINVAL, "di_debug_selftest: this library was built without DI_DEBUG");
#endif
}

di_status di_get_state(const di_graph *g, double *F_out, double *H_out) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (g->last_prec < 0) return set_error(DI_EINVAL, "no D-iteration solve has run on this graph");
    return copy_state(g, F_out, is_device_ptr(F_out), H_out, is_device_ptr(H_out));
}

di_status di_set_state(di_graph *g, const double *F_in, const double *H_in, double rtol, double *deviation) {
    g_last_error.clear();
    if (di_status cr = check_graph(g); cr != DI_OK) return cr;
    if (!F_in || !H_in) return set_error(DI_EINVAL, "F_in and H_in must both be given");
    if (!(rtol >= 0.0) || !std::isfinite(rtol)) return set_error(DI_EINVAL, "rtol must be finite and >= 0");
    if (g->n == 0) {
        if (deviation) *deviation = 0.0;
        return DI_OK;
    }
    return set_state(g, F_in, is_device_ptr(F_in), H_in, is_device_ptr(H_in), rtol, deviation);
}

}  // extern "C"
