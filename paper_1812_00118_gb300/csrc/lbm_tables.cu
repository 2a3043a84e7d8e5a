// Kernel instantiations for ONE (lattice, storage) pair, selected at compile
// time by LBM_LAT (0 = D2Q9, 1 = D3Q19) and LBM_ST (lbm::ST_*).  The build
// compiles this file once per pair so the eight pairs compile in parallel.
#include "lbm_instances.cuh"

#ifndef LBM_LAT
#error "LBM_LAT must be defined"
#endif
#ifndef LBM_ST
#error "LBM_ST must be defined"
#endif

namespace lbm {
namespace {

#if LBM_LAT == 1
// D3Q19: CTA shapes in the x-y plane (nodes).  Tiles 0-3 use per-thread
// loads, 4 the bulk tensor copy pipeline, 5-6 are tiles 0-1 as a one-wave
// launch, 7 loads through cp.async ahead of use (FP32 storage only), 8-9 are
// tile 1 and its one-wave form at 7 CTAs per SM (72 registers instead of 64).
#define LBM_TILES(X)         \
    X(0, hoist, 32, 4, 4)    \
    X(1, split, 32, 4, 8)    \
    X(2, split, 32, 8, 4)    \
    X(3, split, 32, 4, 6)    \
    X(4, tma, 32, 4, 2)      \
    X(5, hoistbal, 32, 4, 4) \
    X(6, splitbal, 32, 4, 8) \
    X(7, async, 32, 4, 4)    \
    X(8, split, 32, 4, 7)    \
    X(9, splitbal, 32, 4, 7)
#else
// D2Q9: the 2-D grid is stored as (nx, 1, ny); CTAs are rows along x
#define LBM_TILES(X)           \
    X(0, hoist, 128, 1, 4)     \
    X(1, split, 128, 1, 8)     \
    X(2, split, 256, 1, 4)     \
    X(3, split, 64, 1, 16)     \
    X(4, tma, 128, 1, 2)       \
    X(5, hoistbal, 128, 1, 4)  \
    X(6, splitbal, 128, 1, 8)  \
    X(7, async, 128, 1, 8)     \
    X(8, split, 128, 1, 7)     \
    X(9, splitbal, 128, 1, 7)
#endif

#define LBM_LAUNCH_hoist(TX, TY, MB) launch_step_tile<LBM_LAT, LBM_ST, TX, TY, MB, true, false>(a)
#define LBM_LAUNCH_split(TX, TY, MB) launch_step_tile<LBM_LAT, LBM_ST, TX, TY, MB, false, false>(a)
#define LBM_LAUNCH_hoistbal(TX, TY, MB) launch_step_tile<LBM_LAT, LBM_ST, TX, TY, MB, true, true>(a)
#define LBM_LAUNCH_splitbal(TX, TY, MB) launch_step_tile<LBM_LAT, LBM_ST, TX, TY, MB, false, true>(a)
#define LBM_LAUNCH_async(TX, TY, MB) launch_async_tile<LBM_LAT, LBM_ST, TX, TY, MB>(a)
#define LBM_LAUNCH_tma(TX, TY, MB) launch_tma_tile<LBM_LAT, LBM_ST, TX, TY, MB>(a)
#define LBM_CASE(ID, KIND, TX, TY, MB) \
    case ID: return LBM_LAUNCH_##KIND(TX, TY, MB);

cudaError_t step_dispatch(const StepArgs& a) {
    switch (a.tile) {
        LBM_TILES(LBM_CASE)
        default: return cudaErrorInvalidValue;
    }
}

#define LBM_MAPS_hoist(TX, TY) cudaErrorInvalidValue
#define LBM_MAPS_split(TX, TY) cudaErrorInvalidValue
#define LBM_MAPS_hoistbal(TX, TY) cudaErrorInvalidValue
#define LBM_MAPS_splitbal(TX, TY) cudaErrorInvalidValue
#define LBM_MAPS_async(TX, TY) cudaErrorInvalidValue
#define LBM_MAPS_tma(TX, TY) make_maps_tile<LBM_LAT, LBM_ST, TX, TY>(out, h, g, G)
#define LBM_MAPS_CASE(ID, KIND, TX, TY, MB) \
    case ID: return LBM_MAPS_##KIND(TX, TY);

cudaError_t maps_dispatch(int tile, TmaMaps* out, const void* h, const void* g, const Geom& G) {
    switch (tile) {
        LBM_TILES(LBM_MAPS_CASE)
        default: return cudaErrorInvalidValue;
    }
}

#define LBM_OK_hoist(TX, TY) true
#define LBM_OK_split(TX, TY) true
#define LBM_OK_hoistbal(TX, TY) true
#define LBM_OK_splitbal(TX, TY) true
#define LBM_OK_async(TX, TY) async_tile_ok<LBM_LAT, LBM_ST, TX, TY>(G)
#define LBM_OK_tma(TX, TY) tma_tile_ok<LBM_LAT, LBM_ST, TX, TY>(G)
#define LBM_OK_CASE(ID, KIND, TX, TY, MB) \
    case ID: return LBM_OK_##KIND(TX, TY);

bool ok_dispatch(int tile, const Geom& G) {
    switch (tile) {
        LBM_TILES(LBM_OK_CASE)
        default: return false;
    }
}

#if LBM_LAT == 0
// Batches of D2Q9 grids: CTA widths along x (the grids of a batch are often
// narrower than the single-grid tiles).
#define LBM_BATCH_TILES(X)  \
    X(0, false, 64, 16)     \
    X(1, false, 128, 8)     \
    X(2, false, 32, 32)     \
    X(3, true, 128, 4)
#define LBM_BATCH_CASE(ID, HOIST, TX, MB) \
    case ID: return launch_batch_tile<LBM_LAT, LBM_ST, TX, MB, HOIST>(a);
cudaError_t batch_dispatch(const BatchArgs& a) {
    switch (a.tile) {
        LBM_BATCH_TILES(LBM_BATCH_CASE)
        default: return cudaErrorInvalidValue;
    }
}
#define LBM_BATCH_TX(ID, HOIST, TX, MB) TX,
#define LBM_BATCH_FIELDS batch_dispatch, batch_upload<LBM_ST>, sizeof(BatchCase<Storage<LBM_ST>::R>), \
                         kMaxBatchTiles, {LBM_BATCH_TILES(LBM_BATCH_TX)}
#else
#define LBM_BATCH_FIELDS nullptr, nullptr, 0, 0, {0, 0, 0, 0}
#endif

#define LBM_TX(ID, KIND, TX, TY, MB) TX,
#define LBM_TY(ID, KIND, TX, TY, MB) TY,
#define LBM_ISTMA_hoist 0
#define LBM_ISTMA_split 0
#define LBM_ISTMA_hoistbal 0
#define LBM_ISTMA_splitbal 0
#define LBM_ISTMA_async 0
#define LBM_ISTMA_tma 1
#define LBM_TMA(ID, KIND, TX, TY, MB) LBM_ISTMA_##KIND,

int checked_status() {
#ifdef LBM_CHECKED
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_checked_err, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_checked_err, &zero, sizeof(int)) != cudaSuccess) return -1;
    }
    return v;
#else
    return 0;
#endif
}

const KernelTable kTable = {step_dispatch, maps_dispatch, ok_dispatch,
                            Launchers<LBM_LAT, LBM_ST>::phi, Launchers<LBM_LAT, LBM_ST>::macro,
                            Launchers<LBM_LAT, LBM_ST>::init, Launchers<LBM_LAT, LBM_ST>::get,
                            Launchers<LBM_LAT, LBM_ST>::set, Launchers<LBM_LAT, LBM_ST>::halo,
                            Launchers<LBM_LAT, LBM_ST>::shift_rest, kMaxTiles,
                            {LBM_TILES(LBM_TX)}, {LBM_TILES(LBM_TY)},
                            {LBM_TILES(LBM_TMA)}, LBM_BATCH_FIELDS, checked_status};

}  // namespace

const KernelTable* LBM_TABLE_NAME(LBM_LAT, LBM_ST)() { return &kTable; }

}  // namespace lbm
