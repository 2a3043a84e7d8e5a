// Internal interface between the host library (lbm_api.cu) and the
// per-lattice translation units that instantiate the kernels.
#pragma once
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbm {

struct TmaMaps;

constexpr int kMaxTiles = 12;   // step kernel variants per (lattice, storage)

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
};

struct KernelTable {
    cudaError_t (*step)(const StepArgs& a);
    // tensor maps of one input buffer pair for bulk-copy tile `tile`
    cudaError_t (*make_maps)(int tile, TmaMaps* out, const void* h, const void* g, const Geom& G);
    // true if bulk-copy tile `tile` can run this grid (shared memory, sizes)
    bool (*tma_ok)(int tile, const Geom& G);
    cudaError_t (*phi)(const void* hin, const Geom& G, const Phys& p, double* phi, cudaStream_t s);
    cudaError_t (*macro)(const void* gin, const Geom& G, const Phys& p, const double* phi, double* P,
                         double* ux, double* uy, double* uz, cudaStream_t s);
    cudaError_t (*init)(void* hout, void* gout, const Geom& G, const Phys& p, const double* phi,
                        const double* ux, const double* uy, const double* uz, const double* P,
                        cudaStream_t s);
    cudaError_t (*get)(const void* hin, const void* gin, const Geom& G, const Phys& p, double* h,
                       double* g, cudaStream_t s);
    cudaError_t (*set)(void* hout, void* gout, const Geom& G, const Phys& p, const double* h,
                       const double* g, cudaStream_t s);
    // periodic images of the ghost band of a freshly written buffer pair
    cudaError_t (*halo)(void* hout, void* gout, const Geom& G, cudaStream_t s);
    int n_tiles;            // number of compiled step tile shapes
    int tile_tx[kMaxTiles], tile_ty[kMaxTiles];
    int tile_tma[kMaxTiles];   // 1: bulk tensor copy pipeline, 0: per-thread loads
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
