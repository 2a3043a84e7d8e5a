// Internal interface between the host library (lbm_api.cu) and the
// per-lattice translation units that instantiate the kernels.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbm {

// NVTX range over a host call (steps, initialisation, read-back,
// diagnostics): a profiler's timeline shows the library's calls around its
// kernels.  Costs nothing without a tool attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct TmaMaps;

constexpr int kMaxTiles = 10;   // step kernel variants per (lattice, storage)

// Everything one step launch needs.
struct StepArgs {
    const void* hin;
    const void* gin;
    void* hout;
    void* gout;
    Geom G;
    Phys p;
    int tile, lz;
    cudaStream_t stream;
    const TmaMaps* maps;   // tensor maps of (hin, gin) for a bulk-copy tile
    int* error_flag;       // raised by a bounded wait that gave up
    long wait_polls;       // polls of a bulk-copy pipeline wait before it gives up
};

// Everything one batch step launch needs (see batch_step_kernel).
struct BatchArgs {
    const void* hin;
    const void* gin;
    void* hout;
    void* gout;
    long long NP;          // stride between population arrays of the batch
    const void* cases;     // device array of BatchCase<R>, one per grid
    const void* items;     // device array of BatchItem
    int n_items;
    int* counters;         // two device ints, zero between launches
    int tile;
    cudaStream_t stream;
};

constexpr int kMaxBatchTiles = 4;

struct KernelTable {
    cudaError_t (*step)(const StepArgs& a);
    // tensor maps of one input buffer pair for bulk-copy tile `tile`
    cudaError_t (*make_maps)(int tile, TmaMaps* out, const void* h, const void* g, const Geom& G);
    // true if tile `tile` can run this grid and storage type (shared memory,
    // sizes; bulk-copy and asynchronous-load tiles have limits)
    bool (*tile_ok)(int tile, const Geom& G);
    cudaError_t (*phi)(const void* hin, const Geom& G, const Phys& p, double* phi, cudaStream_t s);
    cudaError_t (*macro)(const void* gin, const Geom& G, const Phys& p, const double* phi, double* P,
                         double* ux, double* uy, double* uz, cudaStream_t s);
    cudaError_t (*init)(void* hout, void* gout, const Geom& G, const Phys& p, const double* phi,
                        const double* ux, const double* uy, const double* uz, const double* P, int neq,
                        cudaStream_t s);
    cudaError_t (*get)(const void* hin, const void* gin, const Geom& G, const Phys& p, double* h,
                       double* g, cudaStream_t s);
    cudaError_t (*set)(void* hout, void* gout, const Geom& G, const Phys& p, const double* h,
                       const double* g, cudaStream_t s);
    // periodic images of the ghost band of a freshly written buffer pair
    cudaError_t (*halo)(void* hout, void* gout, const Geom& G, cudaStream_t s);
    // h_0 += *delta (device double) at every node of buffer h
    cudaError_t (*shift_rest)(void* h, const Geom& G, const Phys& p, const double* delta, cudaStream_t s);
    int n_tiles;            // number of compiled step tile shapes
    int tile_tx[kMaxTiles], tile_ty[kMaxTiles];
    int tile_tma[kMaxTiles];   // 1: bulk tensor copy pipeline, 0: per-thread loads
    // batches of grids (D2Q9; null and 0 for D3Q19)
    cudaError_t (*batch_step)(const BatchArgs& a);
    // BatchCase<R> of n grids from their geometries and parameters into d_cases
    cudaError_t (*batch_upload)(const Geom* G, const Phys* P, int n, void* d_cases, cudaStream_t s);
    size_t batch_case_bytes;
    int n_batch_tiles;
    int batch_tile_tx[kMaxBatchTiles];
    // checked builds: this unit's offset-check flag (0 none, 1 pull, 2 write),
    // cleared by the read; -1 if the read failed; always 0 in other builds
    int (*checked_status)();
};

// One table per (lattice, storage), each defined in its own compilation of
// lbm_tables.cu under the name table_l<lattice>_s<storage>.
#define LBM_TABLE_NAME2(l, s) table_l##l##_s##s
#define LBM_TABLE_NAME(l, s) LBM_TABLE_NAME2(l, s)
const KernelTable* table_l0_s0();
const KernelTable* table_l0_s1();
const KernelTable* table_l0_s2();
const KernelTable* table_l0_s3();
const KernelTable* table_l1_s0();
const KernelTable* table_l1_s1();
const KernelTable* table_l1_s2();
const KernelTable* table_l1_s3();

}  // namespace lbm

// State of one simulation (host side of the C-ABI handle).
struct lbm_ctx {
    int lattice = 0;
    int store = 0;
    int dim = 3;
    lbm_grid grid{};       // user grid
    lbm_params params{};
    lbm::Geom G{};         // internal grid
    lbm::Phys P{};
    const lbm::KernelTable* K = nullptr;
    cudaStream_t stream = nullptr;
    size_t elem = 0;       // bytes per stored population value
    void* h[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;           // buffer holding the current state
    int tile = 0;          // step tile shape index
    int lz = 16;           // planes per CTA chunk
    lbm::TmaMaps maps[2];  // tensor maps of buffer pair 0 and 1 for a bulk-copy tile
    int maps_tile = -1;    // tile the maps were made for
    bool ghosts[2] = {false, false};   // ghost band of buffer b holds the periodic images
    int* d_err = nullptr;  // device flag raised by a bounded wait that gave up
    bool diverged = false; // the last lbm_diagnostics found the state diverged
    long wait_polls = 1L << 22;   // bulk-copy pipeline wait limit (lbm_set_wait_limit)
    double* fields = nullptr;    // scratch: phi, P, ux, uy, uz (5 N doubles)
    double* partial = nullptr;   // scratch: reduction partials
    int n_partial_blocks = 0;
    long long launches = 0;
    int pversion = 0;            // bumped whenever P changes after creation
    int phi_fix_every = 0;       // re-impose the total of phi every k steps (0: never)
    int phi_fix_count = 0;       // steps since the last re-imposition
    double phi_target = 0.0;     // total of phi at the last initialisation
    double* d_fix = nullptr;     // device scratch of the re-imposition: partials, delta
    lbm_batch* owner = nullptr;  // set for the view of one grid of a batch: the
                                 // buffers and scratch belong to the batch,
                                 // which alone steps them
};

namespace lbm {
const KernelTable* table_for(int lattice, int store);
// lbm_create without the buffers (checks, constants, geometry, tables)
int ctx_setup(lbm_ctx* c, const lbm_grid* grid, int lattice, const lbm_params* params, void* cuda_stream,
              int flags);
}  // namespace lbm
