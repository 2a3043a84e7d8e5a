// Host side of the batch API (lbm_batch_* in include/lbm.h): many D2Q9 grids
// in one set of population arrays, stepped by one persistent launch per step
// (batch_step_kernel) over a work list of (grid, tile column, plane chunk).
//
// Each grid also has a view context (an lbm_ctx whose geometry carries the
// grid's base offset and the batch-wide population stride, and whose buffers
// and scratch are the batch's), so every per-grid call of the single-grid
// API -- initialisation, populations, macroscopic fields, diagnostics --
// runs unchanged on one grid of the batch.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

struct lbm_batch {
    int n = 0;
    int store = 0;
    size_t elem = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;          // private stream for graph capture
    const KernelTable* K = nullptr;
    std::vector<lbm_ctx*> views;
    std::vector<double> rho_bar_up;      // rho_bar of each grid as uploaded
    std::vector<int> pversion_up;        // parameter version of each grid as uploaded
    long long NP = 0;                    // padded cells of all grids
    void* h[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    void* d_cases = nullptr;             // BatchCase<R>[n]
    BatchItem* d_items = nullptr;
    int n_items = 0, items_cap = 0;
    int* d_counters = nullptr;           // two ints, zero between launches
    int* d_err = nullptr;
    double* fields = nullptr;            // scratch of the views (largest grid)
    double* partial = nullptr;
    int n_partial_blocks = 1024;
    int tile = 1, lz = 16;
    int graph_k = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // by starting buffer
    long long launches = 0;
};

namespace {

int check(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

// Items of the work list in launch order (see lbm_batch_plan).
int make_plan(int n, const int* NX, const int* NZ, int tx, int lz, std::vector<BatchItem>* out) {
    if (n < 1 || tx < 1 || lz < 1) return LBM_EINVAL;
    long long total = 0;
    for (int c = 0; c < n; ++c) {
        if (NX[c] < 1 || NZ[c] < 1) return LBM_EINVAL;
        total += (long long)((NX[c] + tx - 1) / tx) * ((NZ[c] + lz - 1) / lz);
    }
    if (total >= (1LL << 31)) return LBM_EINVAL;
    if (out) {
        out->clear();
        out->reserve((size_t)total);
        for (int c = 0; c < n; ++c)
            for (int z0 = 0; z0 < NZ[c]; z0 += lz)
                for (int x0 = 0; x0 < NX[c]; x0 += tx)
                    out->push_back({c, x0, z0, z0 + lz < NZ[c] ? z0 + lz : NZ[c]});
    }
    return (int)total;
}

void invalidate_graphs(lbm_batch* b) {
    for (int p = 0; p < 2; ++p)
        if (b->gexec[p]) { cudaGraphExecDestroy(b->gexec[p]); b->gexec[p] = nullptr; }
}

int set_items(lbm_batch* b) {
    std::vector<int> NX(b->n), NZ(b->n);
    for (int c = 0; c < b->n; ++c) { NX[c] = b->views[c]->G.NX; NZ[c] = b->views[c]->G.NZ; }
    std::vector<BatchItem> items;
    const int m = make_plan(b->n, NX.data(), NZ.data(), b->K->batch_tile_tx[b->tile], b->lz, &items);
    if (m < 0) return m;
    if (m > b->items_cap) {
        if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
        b->d_items = nullptr;
        b->items_cap = 0;
        if (cudaMallocAsync((void**)&b->d_items, sizeof(BatchItem) * (size_t)m, b->stream) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ENOMEM;
        }
        b->items_cap = m;
    }
    if (check(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * (size_t)m, cudaMemcpyHostToDevice,
                              b->stream)))
        return LBM_ECUDA;
    b->n_items = m;
    invalidate_graphs(b);
    return check(cudaStreamSynchronize(b->stream));
}

// Grid parameters into device memory; again whenever a grid's rho_bar (set by
// its initialisation under force_mode 1) or its wall velocities have changed
// since the last upload.
int upload_cases(lbm_batch* b, bool force) {
    bool dirty = force;
    for (int c = 0; c < b->n && !dirty; ++c)
        dirty = b->views[c]->P.rho_bar != b->rho_bar_up[c] || b->views[c]->pversion != b->pversion_up[c];
    if (!dirty) return LBM_OK;
    std::vector<Geom> G(b->n);
    std::vector<Phys> P(b->n);
    for (int c = 0; c < b->n; ++c) {
        G[c] = b->views[c]->G;
        P[c] = b->views[c]->P;
        b->rho_bar_up[c] = P[c].rho_bar;
        b->pversion_up[c] = b->views[c]->pversion;
    }
    return check(b->K->batch_upload(G.data(), P.data(), b->n, b->d_cases, b->stream));
}

BatchArgs args_for(const lbm_batch* b, int in, cudaStream_t s) {
    BatchArgs a;
    a.hin = b->h[in];
    a.gin = b->g[in];
    a.hout = b->h[1 - in];
    a.gout = b->g[1 - in];
    a.NP = b->NP;
    a.cases = b->d_cases;
    a.items = b->d_items;
    a.n_items = b->n_items;
    a.counters = b->d_counters;
    a.tile = b->tile;
    a.stream = s;
    return a;
}

void sync_views(lbm_batch* b) {
    for (lbm_ctx* v : b->views) v->cur = b->cur;
}

// Graph of graph_k step launches starting from buffer `in`.
int build_graph(lbm_batch* b, int in) {
    // first launch of an instantiation looks up its occupancy: not inside a capture
    BatchArgs prime = args_for(b, in, b->stream);
    prime.n_items = 0;
    if (check(b->K->batch_step(prime))) return LBM_ECUDA;
    if (!b->cap && check(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking))) return LBM_ECUDA;
    if (check(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal))) return LBM_ECUDA;
    int rc = LBM_OK;
    int p = in;
    for (int k = 0; k < b->graph_k && !rc; ++k) {
        rc = check(b->K->batch_step(args_for(b, p, b->cap)));
        p = 1 - p;
    }
    cudaGraph_t graph = nullptr;
    const int re = check(cudaStreamEndCapture(b->cap, &graph));
    if (!rc) rc = re;
    if (!rc) rc = check(cudaGraphInstantiate(&b->gexec[in], graph, 0));
    if (graph) cudaGraphDestroy(graph);
    if (rc) cudaGetLastError();
    return rc;
}

int step_direct(lbm_batch* b, int n) {
    for (int s = 0; s < n; ++s) {
        if (check(b->K->batch_step(args_for(b, b->cur, b->stream)))) return LBM_ECUDA;
        b->launches += 1;
        b->cur = 1 - b->cur;
    }
    return LBM_OK;
}

void free_batch(lbm_batch* b) {
    invalidate_graphs(b);
    for (lbm_ctx* v : b->views) delete v;
    for (int k = 0; k < 2; ++k) {
        if (b->h[k]) cudaFreeAsync(b->h[k], b->stream);
        if (b->g[k]) cudaFreeAsync(b->g[k], b->stream);
    }
    if (b->d_cases) cudaFreeAsync(b->d_cases, b->stream);
    if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
    if (b->d_counters) cudaFreeAsync(b->d_counters, b->stream);
    if (b->d_err) cudaFreeAsync(b->d_err, b->stream);
    if (b->fields) cudaFreeAsync(b->fields, b->stream);
    if (b->partial) cudaFreeAsync(b->partial, b->stream);
    cudaStreamSynchronize(b->stream);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // namespace

extern "C" {

int lbm_batch_plan(int n, const lbm_grid* grids, int tx, int lz, int* items, int max_items) {
    if (n < 1 || !grids || max_items < 0 || (max_items > 0 && !items)) return LBM_EINVAL;
    std::vector<int> NX(n), NZ(n);
    for (int c = 0; c < n; ++c) {
        if (grids[c].nz != 1) return LBM_EINVAL;
        NX[c] = grids[c].nx;   // internal x = user x, internal z = user y
        NZ[c] = grids[c].ny;
    }
    std::vector<BatchItem> v;
    const int m = make_plan(n, NX.data(), NZ.data(), tx, lz, max_items > 0 ? &v : nullptr);
    if (m < 0) return m;
    for (int k = 0; k < max_items && k < m; ++k) {
        items[4 * k + 0] = v[k].c;
        items[4 * k + 1] = v[k].x0;
        items[4 * k + 2] = v[k].z0;
        items[4 * k + 3] = v[k].z1;
    }
    return m;
}

int lbm_batch_create(int n, const lbm_grid* grids, const lbm_params* params, void* cuda_stream, lbm_batch** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (n < 1 || !grids || !params) return LBM_EINVAL;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->store = params[0].store;
    long long base = 0, max_n = 0;
    for (int c = 0; c < n; ++c) {
        lbm_ctx* v = new (std::nothrow) lbm_ctx();
        if (!v) { free_batch(b); return LBM_ENOMEM; }
        b->views.push_back(v);
        int rc = params[c].store == b->store ? ctx_setup(v, &grids[c], LBM_D2Q9, &params[c], cuda_stream, 0)
                                             : LBM_EINVAL;
        if (rc) { free_batch(b); return rc; }
        v->owner = b;
        v->G.base = (int)base;          // blocks are multiples of 32 bytes: aligned
        base += v->G.NP;
        if (base >= (1LL << 31)) { free_batch(b); return LBM_EINVAL; }
        if (v->G.N > max_n) max_n = v->G.N;
    }
    b->K = b->views[0]->K;
    b->elem = b->views[0]->elem;
    if (!b->K->batch_step) { free_batch(b); return LBM_ENOTSUP; }
    b->NP = base;
    b->rho_bar_up.assign(n, 0.0);
    b->pversion_up.assign(n, 0);
    const size_t bytes = b->elem * 9 * (size_t)b->NP;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok = cudaMallocAsync(&b->h[k], bytes, b->stream) == cudaSuccess &&
             cudaMallocAsync(&b->g[k], bytes, b->stream) == cudaSuccess;
        if (ok) {
            cudaMemsetAsync(b->h[k], 0, bytes, b->stream);
            cudaMemsetAsync(b->g[k], 0, bytes, b->stream);
        }
    }
    ok = ok && cudaMallocAsync(&b->d_cases, b->K->batch_case_bytes * (size_t)n, b->stream) == cudaSuccess;
    ok = ok && cudaMallocAsync((void**)&b->d_counters, 2 * sizeof(int), b->stream) == cudaSuccess;
    ok = ok && cudaMallocAsync((void**)&b->d_err, sizeof(int), b->stream) == cudaSuccess;
    ok = ok && cudaMallocAsync((void**)&b->fields, sizeof(double) * 5 * (size_t)max_n, b->stream) == cudaSuccess;
    ok = ok && cudaMallocAsync((void**)&b->partial, sizeof(double) * 8 * b->n_partial_blocks, b->stream) ==
                   cudaSuccess;
    if (!ok) { cudaGetLastError(); free_batch(b); return LBM_ENOMEM; }
    cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(int), b->stream);
    cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
    for (lbm_ctx* v : b->views) {
        v->G.NP = b->NP;                // population stride of the shared arrays
        for (int k = 0; k < 2; ++k) { v->h[k] = b->h[k]; v->g[k] = b->g[k]; }
        v->d_err = b->d_err;
        v->fields = b->fields;
        v->partial = b->partial;
        v->n_partial_blocks = b->n_partial_blocks;
        v->cur = 0;
    }
    int rc = upload_cases(b, true);
    if (!rc) rc = set_items(b);
    if (rc) { free_batch(b); return rc; }
    *out = b;
    return LBM_OK;
}

lbm_ctx* lbm_batch_grid(lbm_batch* b, int i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->views[i];
}

int lbm_batch_step(lbm_batch* b, int n) {
    lbm::NvtxRange range("lbm_batch_step");
    if (!b || n < 0) return LBM_EINVAL;
    int rc = upload_cases(b, false);
    if (rc) return rc;
    if (b->graph_k > 0) {
        while (n >= b->graph_k) {
            if (!b->gexec[b->cur] && (rc = build_graph(b, b->cur))) return rc;
            if (check(cudaGraphLaunch(b->gexec[b->cur], b->stream))) return LBM_ECUDA;
            b->launches += b->graph_k;
            b->cur = (b->cur + b->graph_k) & 1;
            n -= b->graph_k;
        }
    }
    rc = step_direct(b, n);
    sync_views(b);
    return rc;
}

int lbm_batch_step_sequential(lbm_batch* b, int n) {
    if (!b || n < 0) return LBM_EINVAL;
    int rc = LBM_OK;
    for (int s = 0; s < n && !rc; ++s) {
        for (int c = 0; c < b->n && !rc; ++c) {
            const lbm_ctx* v = b->views[c];
            StepArgs a;
            a.hin = b->h[b->cur]; a.gin = b->g[b->cur];
            a.hout = b->h[1 - b->cur]; a.gout = b->g[1 - b->cur];
            a.G = v->G;
            a.p = v->P;
            a.tile = 1;
            a.lz = 16;
            a.stream = b->stream;
            a.maps = nullptr;
            a.error_flag = b->d_err;
            a.wait_polls = 1L << 22;
            rc = check(b->K->step(a));
            b->launches += 1;
        }
        if (!rc) b->cur = 1 - b->cur;
    }
    sync_views(b);
    return rc;
}

int lbm_batch_set_tile(lbm_batch* b, int tile, int lz) {
    if (!b || tile < 0 || tile >= b->K->n_batch_tiles || lz < 1) return LBM_EINVAL;
    b->tile = tile;
    b->lz = lz;
    return set_items(b);
}

int lbm_batch_get_tile(const lbm_batch* b, int* tile, int* lz, int* tx, int* n_items) {
    if (!b) return LBM_EINVAL;
    if (tile) *tile = b->tile;
    if (lz) *lz = b->lz;
    if (tx) *tx = b->K->batch_tile_tx[b->tile];
    if (n_items) *n_items = b->n_items;
    return LBM_OK;
}

int lbm_batch_set_graph(lbm_batch* b, int k) {
    if (!b || k < 0) return LBM_EINVAL;
    if (k != b->graph_k) invalidate_graphs(b);
    b->graph_k = k;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int steps, int* best_tile, int* best_lz, double* best_ms) {
    if (!b || steps < 1) return LBM_EINVAL;
    int rc = upload_cases(b, false);
    if (rc) return rc;
    // the trials advance the state: keep a copy and restore it afterwards
    const size_t bytes = b->elem * 9 * (size_t)b->NP;
    void* save_h = nullptr;
    void* save_g = nullptr;
    if (cudaMallocAsync(&save_h, bytes, b->stream) != cudaSuccess) { cudaGetLastError(); return LBM_ENOMEM; }
    if (cudaMallocAsync(&save_g, bytes, b->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(save_h, b->stream);
        return LBM_ENOMEM;
    }
    const int saved_tile = b->tile, saved_lz = b->lz;
    rc = check(cudaMemcpyAsync(save_h, b->h[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    if (!rc) rc = check(cudaMemcpyAsync(save_g, b->g[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    const bool saved = rc == LBM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc) rc = check(cudaEventCreate(&e0));
    if (!rc) rc = check(cudaEventCreate(&e1));
    const int lzs[4] = {4, 8, 16, 32};
    int bt = b->tile, bl = b->lz;
    float bms = 1e30f;
    for (int t = 0; t < b->K->n_batch_tiles && !rc; ++t) {
        for (int k = 0; k < 4 && !rc; ++k) {
            b->tile = t;
            b->lz = lzs[k];
            rc = set_items(b);
            if (!rc) rc = step_direct(b, 2);
            if (rc) break;
            cudaEventRecord(e0, b->stream);
            rc = step_direct(b, steps);
            cudaEventRecord(e1, b->stream);
            if (!rc) rc = check(cudaEventSynchronize(e1));
            float ms = 0;
            if (!rc) rc = check(cudaEventElapsedTime(&ms, e0, e1));
            if (!rc && ms < bms) { bms = ms; bt = t; bl = lzs[k]; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // the state goes back whether or not a trial failed (a failed trial keeps
    // the tile the batch had)
    if (saved) {
        int rr = check(cudaMemcpyAsync(b->h[0], save_h, bytes, cudaMemcpyDeviceToDevice, b->stream));
        if (!rr) rr = check(cudaMemcpyAsync(b->g[0], save_g, bytes, cudaMemcpyDeviceToDevice, b->stream));
        b->cur = 0;
        if (!rc) rc = rr;
    }
    cudaFreeAsync(save_h, b->stream);
    cudaFreeAsync(save_g, b->stream);
    b->tile = rc ? saved_tile : bt;
    b->lz = rc ? saved_lz : bl;
    const int ri = set_items(b);
    if (!rc) rc = ri;
    sync_views(b);
    if (!rc) rc = check(cudaStreamSynchronize(b->stream));
    if (best_tile) *best_tile = bt;
    if (best_lz) *best_lz = bl;
    if (best_ms) *best_ms = (double)bms / steps;
    return rc;
}

long long lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : 0; }

void lbm_batch_destroy(lbm_batch* b) {
    if (b) free_batch(b);
}

}  // extern "C"
