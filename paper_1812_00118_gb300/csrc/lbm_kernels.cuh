// Device code of the phase-field LB step (Otomo, Zhang & Chen, arXiv 1812.00118).
//
// State convention: a population buffer holds, at node x, the values that
// the next step pulls: the pre-collision population of the current state is
// f_i(x, t) = buf_i(x - c_i).  The step kernel therefore reads with a pull
// and writes its post-collision f*_i(x) at x.
//
// Memory layout (ghost-padded SoA): every population array covers a padded
// grid PX x PY x PZ around the NX x NY x NZ nodes, x fastest; node (x, y, z)
// sits at ((z + GZ) PY + (y + GY)) PX + (x + GX), population i at offset
// i * NP.  A pull from x - c_i wraps the coordinate along a periodic axis and
// reads the ghost layer across a wall (halfway bounce-back): the node next to
// the wall writes its outgoing f*_j into array opp(j) at x + c_j, the ghost
// cell its own pull of opp(j) reads, so the pull returns f*_j(x) reflected.
// Ghost widths are 0 along periodic axes (the pulls wrap) unless the context
// was created with a ghost band: the bulk-copy kernels (lbm_tma.cuh) read
// whole boxes, unwrapped, and for them halo_kernel fills the band (kRep = 2
// cells) with the periodic images of the cells the step wrote.
// Rows are padded to 32 bytes, and a nonzero GX (>= 2) is 32 bytes of
// storage, so that every row of nodes starts on a 32-byte sector: a warp's 32
// consecutive stores then fill whole sectors, and bulk tensor copies start
// 16-byte aligned.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_lattice.cuh"

namespace lbm {

// ---------------------------------------------------------------- geometry
constexpr int kRep = 2;   // periodic replication depth in x and y

struct Geom {
    int NX, NY, NZ;   // nodes (internal axes)
    int GX, GY, GZ;   // ghost widths
    int PX, PY, PZ;   // padded extents
    int PXY;          // PX * PY
    long long NP;     // stride between population arrays (< 2^31, checked on
                      // the host): PX * PY * PZ, or for a grid of a batch the
                      // padded size of all its grids
    long long N;      // NX * NY * NZ
    int wall[3];
    int base;         // offset of this grid's padded block in each population
                      // array (0, or the sum of the blocks before it in a batch)
};

// ---------------------------------------------------------------- parameters
// Derived once on the host in double precision (lbm_api.cu).
struct Phys {
    double inv_tau_phi;    // 1 / (M/T + 1/2), Eq. 1
    double theta_coef;     // (M/T) / W, Eq. 4
    double beta, kappa;    // 48 sigma / W and 3 sigma W / 2, Eq. 8
    double rho_L, rho_dif; // rho(phi) = rho_L + phi rho_dif
    double om_L, om_dif;   // 1/tau_mix = om_L + clip(phi) om_dif, Eq. 9
    double g[3];           // body acceleration, internal axes
    int force_mode;        // 0: F = rho g, 1: F = (rho - rho_bar) g
    double rho_bar;
    double eps;            // n = grad phi / (|grad phi| + eps)
    int hocorr;            // Eq. 13 and the corrected velocity definition
    double uw[3][2][3];    // wall velocity of each end (side 0: below 0, 1: above n - 1) of each walled axis
    int moving;            // any wall velocity nonzero
    double h_shift;        // 16-bit storage keeps h_i - w_i h_shift
    double g_shift;        // ... and (g_i - w_i g_shift) * g_scale
    double g_scale, g_inv_scale;
    double dtheta_coef;    // C (M/T) W^2 of the diffusion correction (Eq. 14), 0: off
};

// The same parameters in the arithmetic type of a kernel, converted once on
// the host so that FP32 kernels execute no FP64 conversions.
template <typename R>
struct PhysT {
    R inv_tau_phi, theta_coef, beta, kappa, rho_L, rho_dif, om_L, om_dif;
    R g[3];
    R rho_bar, eps;
    R h_shift, g_shift, g_scale, g_inv_scale;
    R uw[3][2][3];
    R dtheta_coef;
    int moving;
    int force_mode, hocorr;
};

template <typename R>
inline PhysT<R> phys_as(const Phys& p) {
    PhysT<R> q;
    q.inv_tau_phi = (R)p.inv_tau_phi; q.theta_coef = (R)p.theta_coef;
    q.beta = (R)p.beta; q.kappa = (R)p.kappa;
    q.rho_L = (R)p.rho_L; q.rho_dif = (R)p.rho_dif;
    q.om_L = (R)p.om_L; q.om_dif = (R)p.om_dif;
    for (int a = 0; a < 3; ++a) q.g[a] = (R)p.g[a];
    q.rho_bar = (R)p.rho_bar; q.eps = (R)p.eps;
    q.h_shift = (R)p.h_shift; q.g_shift = (R)p.g_shift;
    q.g_scale = (R)p.g_scale; q.g_inv_scale = (R)p.g_inv_scale;
    q.force_mode = p.force_mode; q.hocorr = p.hocorr;
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd)
            for (int k = 0; k < 3; ++k) q.uw[a][sd][k] = (R)p.uw[a][sd][k];
    q.moving = p.moving;
    q.dtheta_coef = (R)p.dtheta_coef;
    return q;
}

// ---------------------------------------------------------------- storage
enum { ST_F64 = 0, ST_F32 = 1, ST_F16S = 2, ST_BF16S = 3 };

template <int ST> struct Storage;
// load / store convert between the stored value and the population itself;
// raw / pack only convert the number format, for step code that works on
// the shifted (and scaled) values directly.
template <> struct Storage<ST_F64> {
    using S = double; using R = double;
    static __device__ __forceinline__ R load(S v, R, R) { return v; }
    static __device__ __forceinline__ S store(R v, R, R) { return v; }
    static __device__ __forceinline__ R raw(S v) { return v; }
    static __device__ __forceinline__ S pack(R v) { return v; }
    static constexpr bool kShifted = false;
};
template <> struct Storage<ST_F32> {
    using S = float; using R = float;
    static __device__ __forceinline__ R load(S v, R, R) { return v; }
    static __device__ __forceinline__ S store(R v, R, R) { return v; }
    static __device__ __forceinline__ R raw(S v) { return v; }
    static __device__ __forceinline__ S pack(R v) { return v; }
    static constexpr bool kShifted = false;
};
template <> struct Storage<ST_F16S> {
    using S = __half; using R = float;
    // v = stored * inv_scale + shift
    static __device__ __forceinline__ R load(S v, R shift, R inv_scale) {
        return fmaf(__half2float(v), inv_scale, shift);
    }
    static __device__ __forceinline__ S store(R v, R shift, R scale) {
        return __float2half_rn((v - shift) * scale);
    }
    static __device__ __forceinline__ R raw(S v) { return __half2float(v); }
    static __device__ __forceinline__ S pack(R v) { return __float2half_rn(v); }
    static constexpr bool kShifted = true;
};
template <> struct Storage<ST_BF16S> {
    using S = __nv_bfloat16; using R = float;
    static __device__ __forceinline__ R load(S v, R shift, R inv_scale) {
        return fmaf(__bfloat162float(v), inv_scale, shift);
    }
    static __device__ __forceinline__ S store(R v, R shift, R scale) {
        return __float2bfloat16_rn((v - shift) * scale);
    }
    static __device__ __forceinline__ R raw(S v) { return __bfloat162float(v); }
    static __device__ __forceinline__ S pack(R v) { return __float2bfloat16_rn(v); }
    static constexpr bool kShifted = true;
};

// Read-only loads: default caching for h (re-read by neighbouring threads of
// the same CTA), L1::no_allocate for g (read once) so g does not evict h.
// Both ask L2 to bring the whole 256-byte block of a missed sector from DRAM
// (L2::256B): the pulls of a warp row cover 128 bytes straddling two lines,
// and the rest of the block is the row the next tile column pulls at the
// same time, so more DRAM requests are in flight per load (at 128^3, D3Q19
// FP32, the step runs 7 % faster with the hint than without).
template <typename S> __device__ __forceinline__ S ld_keep(const S* p);
template <typename S> __device__ __forceinline__ S ld_stream(const S* p);
template <> __device__ __forceinline__ double ld_keep<double>(const double* p) {
    double v; asm("ld.global.nc.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p)); return v;
}
template <> __device__ __forceinline__ float ld_keep<float>(const float* p) {
    float v; asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p)); return v;
}
template <> __device__ __forceinline__ __half ld_keep<__half>(const __half* p) {
    unsigned short v; asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __ushort_as_half(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 ld_keep<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short v; asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __ushort_as_bfloat16(v);
}
template <> __device__ __forceinline__ double ld_stream<double>(const double* p) {
    double v; asm("ld.global.nc.L1::no_allocate.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p)); return v;
}
template <> __device__ __forceinline__ float ld_stream<float>(const float* p) {
    float v; asm("ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p)); return v;
}
template <> __device__ __forceinline__ __half ld_stream<__half>(const __half* p) {
    unsigned short v; asm("ld.global.nc.L1::no_allocate.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __ushort_as_half(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 ld_stream<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short v; asm("ld.global.nc.L1::no_allocate.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __ushort_as_bfloat16(v);
}

// Predicated read-only load (default caching, as ld_keep): 0 where !pred.
// The load sits in the same basic block as its neighbours, so a thread's
// unconditional and predicated loads are issued back to back.
template <typename S> __device__ __forceinline__ S ld_keep_if(const S* p, bool pred);
template <> __device__ __forceinline__ double ld_keep_if<double>(const double* p, bool pred) {
    double v = 0.0;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.L2::256B.f64 %0, [%1];\n\t}"
        : "+d"(v) : "l"(p), "r"((unsigned)pred));
    return v;
}
template <> __device__ __forceinline__ float ld_keep_if<float>(const float* p, bool pred) {
    float v = 0.0f;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.L2::256B.f32 %0, [%1];\n\t}"
        : "+f"(v) : "l"(p), "r"((unsigned)pred));
    return v;
}
template <> __device__ __forceinline__ __half ld_keep_if<__half>(const __half* p, bool pred) {
    unsigned short v = 0;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.L2::256B.b16 %0, [%1];\n\t}"
        : "+h"(v) : "l"(p), "r"((unsigned)pred));
    return __ushort_as_half(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 ld_keep_if<__nv_bfloat16>(const __nv_bfloat16* p, bool pred) {
    unsigned short v = 0;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.L2::256B.b16 %0, [%1];\n\t}"
        : "+h"(v) : "l"(p), "r"((unsigned)pred));
    return __ushort_as_bfloat16(v);
}

// phi = sum_i h_i (after Eq. 4) in the kernels' arithmetic type.  FP32 sums
// are compensated: a running sum seeded with 1 (so every addend is smaller in
// magnitude than the sum, as Fast2Sum requires, while phi stays in [-1/2, 1])
// collects each addition's rounding error exactly, and phi = (s - 1) + e with
// s - 1 exact (Sterbenz).  The moving populations enter in consecutive pairs
// (directions 1 + 2, 3 + 4, ...; each pair sum of two values up to ~phi/9 is
// one rounding of ~4e-9), so the compensated chain has 10 links instead of
// 19.  An uncompensated FP32 sum of 19 values up to phi/3 carries ~1e-7 of
// error into phi, ten times the rounding of the stored h themselves, and the
// stencils of Eq. 12 amplify it; at tau near 1/2 it grows over the steps.
// FP64 sums plainly.  add() is called once per direction in direction order
// inside unrolled loops, so the pairing bookkeeping folds away at compile
// time.
template <typename R>
struct PhiSum {
    R s = 0, e = 0;
    __device__ __forceinline__ void add(R v) { s += v; }
    __device__ __forceinline__ R value() const { return s; }
};
template <>
struct PhiSum<float> {
    float s = 1.0f, e = 0.0f, pend = 0.0f;
    int n = 0;
    __device__ __forceinline__ void link(float v) {
        const float t = __fadd_rn(s, v);
        e = __fadd_rn(e, __fsub_rn(v, __fsub_rn(t, s)));
        s = t;
    }
    __device__ __forceinline__ void add(float v) {
        if (n == 0) link(v);                        // the rest population
        else if (n & 1) pend = v;                   // first of a pair
        else link(__fadd_rn(pend, v));              // the pair
        ++n;
    }
    __device__ __forceinline__ float value() const {
        PhiSum<float> c = *this;
        if (n > 0 && (n & 1) == 0) c.link(pend);    // an unpaired last value
        return __fadd_rn(__fsub_rn(c.s, 1.0f), c.e);
    }
};

// Padded flat offset of (possibly ghost) coordinates.
__device__ __forceinline__ int pidx(const Geom& G, int x, int y, int z) {
    return G.base + ((z + G.GZ) * G.PY + (y + G.GY)) * G.PX + (x + G.GX);
}

// Plane a pull from z - cz reads: wrapped when z is periodic, the ghost plane
// when it is walled.
__device__ __forceinline__ int pull_plane(const Geom& G, int zs) {
    if (G.wall[2]) return zs;
    return zs < 0 ? zs + G.NZ : (zs >= G.NZ ? zs - G.NZ : zs);
}

// Coordinate along an axis for a phi stencil access: periodic wrap, or the
// mirrored adjacent node behind a wall (zero normal gradient of phi).  The
// halo of a CTA tile wider than the grid can lie more than one period out,
// so the wrap is a full modulo; the result is always in [0, n).
__device__ __forceinline__ int stencil_coord(int v, int n, int wall) {
    if (v >= 0 && v < n) return v;
    if (wall) return v < 0 ? 0 : n - 1;
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// Store v at ghost-padded coordinates (x, y, z) of one population array and
// at its periodic images (shifts by +-NX, +-NY along periodic axes) that lie
// in the ghost band (within kRep of the nodes in x, GY in y) and are not a
// node's own cell (a cell in a ghost plane behind a z wall never is).  The z
// axis is never replicated.
template <typename S>
__device__ __forceinline__ void store_rep(S* __restrict__ arr, const Geom& G, int x, int y, int z, S v) {
    arr[pidx(G, x, y, z)] = v;
    // images exist only where the layout has a ghost band on a periodic axis
    const int rx = (G.wall[0] || G.GX < kRep) ? 0 : 1;
    const int ry = (G.wall[1] || G.GY < kRep) ? 0 : 1;
    const int Ry = G.GY < kRep ? G.GY : kRep;
    for (int kx = -rx; kx <= rx; ++kx) {
        for (int ky = -ry; ky <= ry; ++ky) {
            if (kx == 0 && ky == 0) continue;
            const int xs = x + kx * G.NX, ys = y + ky * G.NY;
            if (xs < -kRep || xs >= G.NX + kRep || ys < -Ry || ys >= G.NY + Ry) continue;
            if (xs >= 0 && xs < G.NX && ys >= 0 && ys < G.NY && z >= 0 && z < G.NZ) continue;   // a node's cell
            arr[pidx(G, xs, ys, z)] = v;
        }
    }
}

// Per-direction base pointers of the four population arrays (population i of
// array a starts at a + i*NP).  Passed by value as a kernel parameter.
template <typename S, int Q>
struct DirPtrs {
    const S* hin[Q];
    const S* gin[Q];
    S* hout[Q];
    S* gout[Q];
};

template <typename S, int Q>
inline DirPtrs<S, Q> dir_ptrs(const void* hin, const void* gin, void* hout, void* gout, long long NP) {
    DirPtrs<S, Q> d;
    for (int i = 0; i < Q; ++i) {
        d.hin[i] = (const S*)hin + (long long)i * NP;
        d.gin[i] = (const S*)gin + (long long)i * NP;
        d.hout[i] = (S*)hout + (long long)i * NP;
        d.gout[i] = (S*)gout + (long long)i * NP;
    }
    return d;
}

// Offsets of the cells the pulls of node (x, y, z) read: for c in {-1, 0, 1}
// along each axis, the coordinate x - c wrapped along a periodic axis (so no
// ghost image is needed) or left in the ghost layer across a wall (where the
// bounce-back value is stored); z uses pull_plane.  Index 1 + c.
struct PullOffsets {
    int z[3], r[3], c[3];
};

__device__ __forceinline__ int wrap1(int v, int n, int wall) {
    if (wall) return v;
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// The x-y part (row and column offsets) and the plane part of the offsets,
// separately: along a z-march only the plane part changes.
__device__ __forceinline__ void pull_xy(const Geom& G, int x, int y, PullOffsets& o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = k - 1;
        o.r[k] = (wrap1(y - c, G.NY, G.wall[1]) + G.GY) * G.PX;
        o.c[k] = wrap1(x - c, G.NX, G.wall[0]) + G.GX;
    }
}
__device__ __forceinline__ void pull_z(const Geom& G, int z, PullOffsets& o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) o.z[k] = G.base + (pull_plane(G, z - (k - 1)) + G.GZ) * G.PXY;
}
__device__ __forceinline__ PullOffsets pull_offsets(const Geom& G, int x, int y, int z) {
    PullOffsets o;
    pull_xy(G, x, y, o);
    pull_z(G, z, o);
    return o;
}

// ---------------------------------------------------------------- checked builds
// With LBM_CHECKED (a build option for debugging; the default build has
// none of this) the pull offsets of every plane and every write offset of the
// step kernels are checked against the population arrays before use: an
// offset outside [0, NP) sets this translation unit's flag (read by
// lbm_checked_status: 1 = a pull, 2 = a write) and is replaced by 0, a valid
// element, so a bad index gives a wrong result and a report, never a fault.
// Every pull offset is a sum z[k] + r[j] + c[m], so the extreme sums bound
// all 27.
#ifdef LBM_CHECKED
static __device__ int g_checked_err;
__device__ __forceinline__ void checked_offsets(PullOffsets& o, long long NP) {
    long long lo = 0, hi = 0;
    int mn, mx;
    mn = min(o.z[0], min(o.z[1], o.z[2])); mx = max(o.z[0], max(o.z[1], o.z[2])); lo += mn; hi += mx;
    mn = min(o.r[0], min(o.r[1], o.r[2])); mx = max(o.r[0], max(o.r[1], o.r[2])); lo += mn; hi += mx;
    mn = min(o.c[0], min(o.c[1], o.c[2])); mx = max(o.c[0], max(o.c[1], o.c[2])); lo += mn; hi += mx;
    if (lo < 0 || hi >= NP) {
        atomicExch(&g_checked_err, 1);
        for (int k = 0; k < 3; ++k) o.z[k] = o.r[k] = o.c[k] = 0;
    }
}
__device__ __forceinline__ int checked_write(int off, long long NP) {
    if (off < 0 || off >= NP) {
        atomicExch(&g_checked_err, 2);
        return 0;
    }
    return off;
}
#else
__device__ __forceinline__ void checked_offsets(PullOffsets&, long long) {}
__device__ __forceinline__ int checked_write(int off, long long) { return off; }
#endif

// Address of the value a pull of direction I reads.
template <int LAT, int I, typename S>
__device__ __forceinline__ const S* pull_ptr(const S* const* arr, const PullOffsets& o) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    return arr[I] + (o.z[1 + CZ] + o.r[1 + CY] + o.c[1 + CX]);
}

template <int LAT, int I, bool STREAM, typename S>
__device__ __forceinline__ S pull_pad(const S* const* arr, const PullOffsets& o) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    const S* p = arr[I] + (o.z[1 + CZ] + o.r[1 + CY] + o.c[1 + CX]);
    return STREAM ? ld_stream(p) : ld_keep(p);
}

// Whether a node sits next to a wall (then some of its outgoing values also
// go to bounce-back ghost cells).  The periodic images of the ghost band are
// written after each step by halo_kernel, not by the step kernels.
struct NodeWrites {
    bool wall_adj;
};

template <int LAT>
__device__ __forceinline__ NodeWrites node_writes(const Geom& G, int x, int y, int z) {
    NodeWrites w;
    w.wall_adj = (G.wall[0] && (x == 0 || x == G.NX - 1)) ||
                 (Lattice<LAT>::kHasY && G.wall[1] && (y == 0 || y == G.NY - 1)) ||
                 (G.wall[2] && (z == 0 || z == G.NZ - 1));
    return w;
}

// Write the post-collision value v of direction J at node (x, y, z): its own
// cell `own` and, if the grid has walls (WALLS) and x + c_J crosses one, the
// bounce-back ghost cell of array opp(J).
template <int LAT, int J, bool WALLS, typename S>
__device__ __forceinline__ void write_dir(S* const* arr, const Geom& G, int x, int y, int z, int own,
                                          const NodeWrites& nw, S v) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[J], CY = L::cy[J], CZ = L::cz[J];
    arr[J][checked_write(own, G.NP)] = v;
    if constexpr (WALLS) {
        if (nw.wall_adj) {
            const int tx = x + CX, ty = y + CY, tz = z + CZ;
            const bool wall_cross = (CX != 0 && G.wall[0] && (tx < 0 || tx >= G.NX)) ||
                                    (CY != 0 && G.wall[1] && (ty < 0 || ty >= G.NY)) ||
                                    (CZ != 0 && G.wall[2] && (tz < 0 || tz >= G.NZ));
            // the ghost cell lies across a wall; along the periodic axes the
            // pull wraps, so the cell does too
            if (wall_cross)
                arr[L::opp(J)][checked_write(pidx(G, wrap1(tx, G.NX, G.wall[0]), wrap1(ty, G.NY, G.wall[1]),
                                                  wrap1(tz, G.NZ, G.wall[2])), G.NP)] = v;
        }
    }
}

// Moving walls (halfway bounce-back less the momentum the wall hands over):
// when x + c_J crosses a wall, the value write_dir stored for the bounce-back
// pull of opp(J) becomes v - 2 w_J s (c_J . u_w) / T, with s the density the
// equilibrium carries velocity with (phi for h, rho for g) at x and u_w the
// crossed wall's velocity (the mean of two at a corner).  `store` converts to
// the storage type.
template <int LAT, int J, typename S, typename R, typename Store>
__device__ __forceinline__ void moving_wall_write(S* const* arr, const Geom& G, int x, int y, int z, R v, R s,
                                                  const PhysT<R>& p, Store store) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[J], CY = L::cy[J], CZ = L::cz[J];
    const int t[3] = {x + CX, y + CY, z + CZ};
    const int n[3] = {G.NX, G.NY, G.NZ};
    const int c[3] = {CX, CY, CZ};
    R u0 = (R)0, u1 = (R)0, u2 = (R)0;
    int cnt = 0;
    // selects, not a runtime index into p.uw: an indexed parameter block
    // would be copied to local memory
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] == 0 || !G.wall[a]) continue;
        const bool lo = t[a] < 0, hi = t[a] >= n[a];
        if (!lo && !hi) continue;
        u0 += hi ? p.uw[a][1][0] : p.uw[a][0][0];
        u1 += hi ? p.uw[a][1][1] : p.uw[a][0][1];
        u2 += hi ? p.uw[a][1][2] : p.uw[a][0][2];
        ++cnt;
    }
    if (cnt == 0) return;
    const R cu = ((R)CX * u0 + (R)CY * u1 + (R)CZ * u2) / (R)cnt;
    const R corr = (R)6 * (R)L::w[J] * s * cu;
    arr[L::opp(J)][checked_write(
        pidx(G, wrap1(t[0], G.NX, G.wall[0]), wrap1(t[1], G.NY, G.wall[1]), wrap1(t[2], G.NZ, G.wall[2])), G.NP)] =
        store(v - corr);
}

// Reciprocal on the step path: FP32 takes the approximate hardware
// reciprocal (within 2 ulp) and one Newton-Raphson step r + r (1 - x r),
// which leaves an error of about one rounding without the special-case
// handling of the correctly rounded reciprocal (x is a density here: finite,
// positive, normal); FP64 divides.
__device__ __forceinline__ float recip_fast(float x) {
    const float r = __fdividef(1.0f, x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double recip_fast(double x) { return 1.0 / x; }
// |g| and 1 / (|g| + eps) from g2 = |g|^2 (the interface normal of Eq. 2).
// FP64 as written.  FP32: one approximate reciprocal square root
// r = 1 / sqrt(g2 + eps^2), |g| = g2 r, and r for 1 / (|g| + eps) (relative
// difference below eps / |g|; both give a normal of 0 where grad phi
// vanishes).
__device__ __forceinline__ void norm_inv(double g2, double eps, double* mag, double* inv) {
    *mag = sqrt(g2);
    *inv = 1.0 / (*mag + eps);
}
__device__ __forceinline__ void norm_inv(float g2, float eps, float* mag, float* inv) {
    const float r = rsqrtf(fmaf(eps, eps, g2));
    *mag = g2 * r;
    *inv = r;
}

// compile-time loop helper
template <int I, int N>
struct Unroll {
    template <typename F>
    static __device__ __forceinline__ void run(F&& f) {
        f(std::integral_constant<int, I>{});
        Unroll<I + 1, N>::run(f);
    }
};
template <int N>
struct Unroll<N, N> {
    template <typename F>
    static __device__ __forceinline__ void run(F&&) {}
};

// Dot products with a compile-time integer vector: only the nonzero terms are
// formed (IEEE arithmetic cannot drop 0 * x or x + 0 by itself), +-1
// coefficients become additions and subtractions.
template <int C, typename R>
__device__ __forceinline__ R cmul(R v) {
    if constexpr (C == 1) return v;
    else if constexpr (C == -1) return -v;
    else return (R)C * v;
}
template <int A, int B, typename R>
__device__ __forceinline__ R cdot2(R a, R b) {
    if constexpr (A != 0 && B != 0) return cmul<A>(a) + cmul<B>(b);
    else if constexpr (A != 0) return cmul<A>(a);
    else if constexpr (B != 0) return cmul<B>(b);
    else return (R)0;
}
template <int A, int B, int C, typename R>
__device__ __forceinline__ R cdot3(R a, R b, R c) {
    if constexpr (A != 0 && (B != 0 || C != 0)) return cmul<A>(a) + cdot2<B, C>(b, c);
    else if constexpr (A != 0) return cmul<A>(a);
    else return cdot2<B, C>(b, c);
}

// ---------------------------------------------------------------- local physics
// Everything a node needs after phi, grad phi and lap phi are known and the
// moments of the pulled g are accumulated.  All arithmetic in R.
template <typename R>
struct NodeState {
    R phi, gx, gy, gz, lap;
    R rho, mu, Fx, Fy, Fz;
    R ux, uy, uz, P;
    R usq, ug, uF;
    R pxx, pyy, pzz, pxy, pxz, pyz, tr3;   // Pi (Eq. 12, reading R3) and tr(Pi)/3
    R omega;                               // 1 / tau_mix
    R nx, ny, nz, theta;
};

// m0 = sum g, m1 = sum c g, m2 = sum c c g.  Follows the text after Eq. 12
// for u and P (with the Eq. 13 velocity reading), Eq. 8 for mu, Eq. 9 for
// tau_mix, Eq. 4 for theta.  Pi = m2 - sum c c g^eq with the closed form
//   sum c c g^eq = rho u u + P I - (1/2) sum c c K,
//   sum c c K = s [T(u grad + grad u) - u u (u.grad)] + rho_dif T I (u.grad)
//             + [T(u F + F u) - u u (u.F)] / T,   s = rho_dif + mu / T,
// which holds exactly on D2Q9 and D3Q19 (fourth-order isotropy); the
// oracle sums sum c c (g - g^eq) term by term instead.  Collected for the
// kernel: with V = s grad + F / T and c = s (u.grad) + (u.F) / T,
//   sum c c K = T (u V + V u) - c u u + rho_dif T (u.grad) I,
// and since P - rho_dif T (u.grad) / 2 = T m0,
//   Pi = m2 - T m0 I + u Y + W u,   W = T V / 2,  Y = W - (rho + c / 2) u.
// The flow fields: rho, mu, F, u (with the Eq. 13 velocity reading) and P,
// from phi, its stencils and the zeroth and first moments of g.
template <typename R, bool THREE_D>
__device__ __forceinline__ void node_flow(NodeState<R>& s, const PhysT<R>& p, R m0, R mx, R my, R mz) {
    const R T = (R)(1.0 / 3.0);
    const R rho_dif = (R)p.rho_dif;
    s.rho = (R)p.rho_L + s.phi * rho_dif;
    s.mu = (R)p.beta * s.phi * (s.phi - (R)1) * (s.phi - (R)0.5) - (R)p.kappa * s.lap;
    const R fr = p.force_mode == 0 ? s.rho : s.rho - (R)p.rho_bar;
    s.Fx = fr * (R)p.g[0];
    s.Fy = fr * (R)p.g[1];
    s.Fz = fr * (R)p.g[2];
    const R rho_e = p.hocorr ? s.rho + (R)0.25 * rho_dif * s.lap : s.rho;
    const R inv_rho_e = recip_fast(rho_e);
    s.ux = (mx + (R)0.5 * (s.mu * s.gx + s.Fx)) * inv_rho_e;
    s.uy = THREE_D ? (my + (R)0.5 * (s.mu * s.gy + s.Fy)) * inv_rho_e : (R)0;
    s.uz = (mz + (R)0.5 * (s.mu * s.gz + s.Fz)) * inv_rho_e;
    s.usq = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
    s.ug = s.ux * s.gx + s.uy * s.gy + s.uz * s.gz;
    s.uF = s.ux * s.Fx + s.uy * s.Fy + s.uz * s.Fz;
    s.P = T * m0 + (R)0.5 * T * rho_dif * s.ug;
}

template <typename R, bool THREE_D>
__device__ __forceinline__ void node_state(NodeState<R>& s, const PhysT<R>& p, R m0, R mx, R my, R mz,
                                           R mxx, R myy, R mzz, R mxy, R mxz, R myz) {
    const R T = (R)(1.0 / 3.0);
    const R rho_dif = (R)p.rho_dif;
    node_flow<R, THREE_D>(s, p, m0, mx, my, mz);
    // second moment of g^eq (closed form above, collected), then Pi
    const R sK = rho_dif + (R)3 * s.mu;          // s / T
    const R sK6 = sK * (R)(1.0 / 6.0);           // T s / 2
    const R rhop = s.rho + (R)0.5 * sK * s.ug + (R)1.5 * s.uF;   // rho + c / 2
    const R Tm0 = T * m0;
    const R Wx = sK6 * s.gx + (R)0.5 * s.Fx, Wz = sK6 * s.gz + (R)0.5 * s.Fz;
    const R Yx = Wx - rhop * s.ux, Yz = Wz - rhop * s.uz;
    s.pxx = (mxx - Tm0) + s.ux * (Wx + Yx);
    s.pzz = (mzz - Tm0) + s.uz * (Wz + Yz);
    s.pxz = mxz + s.ux * Yz + s.uz * Wx;
    if (THREE_D) {
        const R Wy = sK6 * s.gy + (R)0.5 * s.Fy;
        const R Yy = Wy - rhop * s.uy;
        s.pyy = (myy - Tm0) + s.uy * (Wy + Yy);
        s.pxy = mxy + s.ux * Yy + s.uy * Wx;
        s.pyz = myz + s.uy * Yz + s.uz * Wy;
    } else {
        s.pyy = s.pxy = s.pyz = (R)0;
    }
    s.tr3 = (s.pxx + s.pyy + s.pzz) * T;
    const R pc = s.phi < (R)0 ? (R)0 : (s.phi > (R)1 ? (R)1 : s.phi);
    s.omega = (R)p.om_L + pc * (R)p.om_dif;
    R gmag, inv;
    norm_inv(s.gx * s.gx + s.gy * s.gy + s.gz * s.gz, (R)p.eps, &gmag, &inv);
    s.nx = s.gx * inv;
    s.ny = s.gy * inv;
    s.nz = s.gz * inv;
    const R d = s.phi - (R)0.5;
    s.theta = (R)p.theta_coef * ((R)1 - (R)4 * d * d);
    // diffusion correction of Eq. 14: delta theta = C (M/T) F |grad phi| with
    // F = -W^2 max(0, (2 phi - 1) lap phi), zero on the tanh profile (dtheta_coef
    // = C (M/T) W^2; 0 leaves theta untouched)
    if (p.dtheta_coef != (R)0) {
        const R t = ((R)2 * s.phi - (R)1) * s.lap;
        s.theta -= (R)p.dtheta_coef * (t > (R)0 ? t : (R)0) * gmag;
    }
}

// Post-collision g*_i (Eq. 10 with G^eq = g^eq + K, Eqs. 6, 7, 11, 13):
//   g*_i = rho Gamma_i + w_i (P/T - rho) + K_i/2 + delta f^eq_i
//        + (1 - 1/tau_mix) w_i/(2T^2) (c_i c_i : Pi - T tr Pi)
// and h*_i (Eq. 1 with Eq. 2).  Gamma_i is shared by both (Eq. 3).
template <int LAT, int I, typename R>
__device__ __forceinline__ void collide_dir(const NodeState<R>& s, const PhysT<R>& p, R h_in,
                                            R* h_out, R* g_out) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    const R w = (R)L::w[I];
    const R cu = cdot3<CX, CY, CZ>(s.ux, s.uy, s.uz);
    // Gamma_i - w_i formed directly: rho Gamma_i - w_i rho would cancel two
    // O(rho w_i) terms and cost FP32 its precision on P
    const R Gm1 = w * ((R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * s.usq);
    const R G = w + Gm1;
    const R cgr = cdot3<CX, CY, CZ>(s.gx, s.gy, s.gz);
    const R cF = cdot3<CX, CY, CZ>(s.Fx, s.Fy, s.Fz);
    const R K = (Gm1 * (R)p.rho_dif + (R)3 * G * s.mu) * (cgr - s.ug) + (R)3 * G * (cF - s.uF);
    // c_i c_i : Pi, diagonal and off-diagonal parts
    const R ccPi = cdot3<CX * CX, CY * CY, CZ * CZ>(s.pxx, s.pyy, s.pzz)
                 + (R)2 * cdot3<CX * CY, CX * CZ, CY * CZ>(s.pxy, s.pxz, s.pyz);
    R gs = s.rho * Gm1 + (R)3 * w * s.P + (R)0.5 * K
         + ((R)1 - s.omega) * w * (R)4.5 * (ccPi - s.tr3);
    if (p.hocorr) gs += w * cu * (R)0.75 * (R)p.rho_dif * s.lap;
    *g_out = gs;
    const R cn = cdot3<CX, CY, CZ>(s.nx, s.ny, s.nz);
    const R heq = s.phi * G + s.theta * w * cn;
    *h_out = h_in + (heq - h_in) * (R)p.inv_tau_phi;
}

// ---------------------------------------------------------------- packed FP32 pairs
// A direction I and its opposite J = opp(I) share every even term of the
// collision (c c : Pi, (c.u)^2, w_i) and see the odd ones (c.u, c.grad phi,
// c.F, c.n) with opposite signs.  FP32 kernels collide the pair in the two
// lanes of float2 registers (lane x: I, lane y: J) with the paired FP32
// instructions of sm_100 and later, one instruction for two directions.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Node quantities the pair collision reads, broadcast to both lanes once per
// node.  w3P, thw, hoc, nwhs depend on w_i: index 0 for the axis weight, 1 for
// the diagonal weight (D3Q19: 1/18, 1/36; D2Q9: 1/9, 1/36).
// SH (16-bit shifted storage): the collision computes the stored values
// themselves, h*_i - w_i h_shift and (g*_i - w_i g_shift) g_scale, so that
// no population is shifted or scaled on its way to memory: every term of g*
// carries g_scale (kF = 1.5 g_scale, and w3P holds w_i (3 P - g_shift)
// g_scale), and h^eq carries the shift -w_i h_shift (nwhs).
struct PairState {
    float2 rho, mu15, hrho_dif, neg_ug, neg_uF15, neg_usq15, phi, inv_tau;
    float2 w3P[2], thw[2], hoc[2], nwhs[2];
    float om45, tr3;   // (1 - 1/tau_mix) * 4.5 (times g_scale with SH) and tr(Pi)/3
    float kF;          // 1.5 g_scale (SH only)
};

template <int LAT, bool SH>
__device__ __forceinline__ PairState pair_state(const NodeState<float>& s, const PhysT<float>& p) {
    using L = Lattice<LAT>;
    constexpr int IA = 1, ID = 4;   // an axis and a diagonal direction
    static_assert(L::cx[IA] * L::cx[IA] + L::cy[IA] * L::cy[IA] + L::cz[IA] * L::cz[IA] == 1, "axis");
    static_assert(L::cx[ID] * L::cx[ID] + L::cy[ID] * L::cy[ID] + L::cz[ID] * L::cz[ID] == 2, "diagonal");
    PairState q;
    const float sc = SH ? p.g_scale : 1.0f;
    q.rho = dup2(SH ? s.rho * sc : s.rho);
    q.mu15 = dup2((SH ? 1.5f * sc : 1.5f) * s.mu);
    q.hrho_dif = dup2((SH ? 0.5f * sc : 0.5f) * p.rho_dif);
    q.neg_ug = dup2(-s.ug);
    q.neg_uF15 = dup2((SH ? -1.5f * sc : -1.5f) * s.uF);
    q.neg_usq15 = dup2(-1.5f * s.usq);
    q.phi = dup2(s.phi);
    q.inv_tau = dup2(p.inv_tau_phi);
    const float wk[2] = {(float)L::w[IA], (float)L::w[ID]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        q.w3P[k] = dup2(SH ? wk[k] * (3.0f * s.P - p.g_shift) * sc : 3.0f * wk[k] * s.P);
        q.thw[k] = dup2(s.theta * wk[k]);
        q.hoc[k] = dup2(p.hocorr ? (SH ? wk[k] * 0.75f * sc : wk[k] * 0.75f) * p.rho_dif * s.lap : 0.0f);
        q.nwhs[k] = dup2(SH ? -wk[k] * p.h_shift : 0.0f);
    }
    q.om45 = (1.0f - s.omega) * (SH ? 4.5f * sc : 4.5f);
    q.tr3 = s.tr3;
    q.kF = SH ? 1.5f * sc : 1.5f;
    return q;
}

// Post-collision g* and h* of the pair (I, opp(I)): the arithmetic of
// collide_dir, two directions per instruction.  hin holds the pulled h of I
// and opp(I) in its lanes.
template <int LAT, int I, bool SH>
__device__ __forceinline__ void collide_pair(const NodeState<float>& s, const PairState& q, float2 hin,
                                             float2* h_out, float2* g_out) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    constexpr int K2 = CX * CX + CY * CY + CZ * CZ;
    constexpr int WK = K2 == 1 ? 0 : 1;
    const float2 w = dup2((float)L::w[I]);
    const float cu = cdot3<CX, CY, CZ>(s.ux, s.uy, s.uz);
    const float cg = cdot3<CX, CY, CZ>(s.gx, s.gy, s.gz);
    const float cF = cdot3<CX, CY, CZ>(s.Fx, s.Fy, s.Fz);
    const float cn = cdot3<CX, CY, CZ>(s.nx, s.ny, s.nz);
    const float2 a = make_float2(cu, -cu);
    // Gamma - w = w (3 c.u + 4.5 (c.u)^2 - 1.5 u.u), formed directly (see collide_dir)
    float2 t = fma2(a, dup2(4.5f), dup2(3.0f));
    t = fma2(t, a, q.neg_usq15);
    const float2 Gm1 = mul2(t, w);
    const float2 G = add2(Gm1, w);
    // K / 2 = (Gm1 rho_dif / 2 + 3 G mu / 2) B + 3 G C / 2 with
    // B = c.grad phi - u.grad phi and C = c.F - u.F; with rho Gm1 it folds into
    // Gm1 (rho + B rho_dif / 2) + G (3 mu B / 2 + 3 C / 2)
    const float2 B = add2(make_float2(cg, -cg), q.neg_ug);
    const float cF15 = (SH ? q.kF : 1.5f) * cF;
    const float2 C15 = add2(make_float2(cF15, -cF15), q.neg_uF15);
    const float2 X = fma2(q.hrho_dif, B, q.rho);
    const float2 Y = fma2(q.mu15, B, C15);
    // c c : Pi, even in c
    const float ccPi = cdot3<CX * CX, CY * CY, CZ * CZ>(s.pxx, s.pyy, s.pzz) +
                       2.0f * cdot3<CX * CY, CX * CZ, CY * CZ>(s.pxy, s.pxz, s.pyz);
    const float filt = (ccPi - q.tr3) * (q.om45 * (float)L::w[I]);
    float2 gs = fma2(a, q.hoc[WK], add2(q.w3P[WK], dup2(filt)));
    gs = fma2(G, Y, gs);
    gs = fma2(Gm1, X, gs);
    *g_out = gs;
    const float2 heq = SH ? fma2(q.phi, G, fma2(q.thw[WK], make_float2(cn, -cn), q.nwhs[WK]))
                          : fma2(q.phi, G, mul2(q.thw[WK], make_float2(cn, -cn)));
    *h_out = fma2(add2(heq, make_float2(-hin.x, -hin.y)), q.inv_tau, hin);
}

// ---------------------------------------------------------------- fused step
// One CTA owns a TX x TY column of nodes in the x-y plane and marches along
// z over a chunk of LZ planes.  Per plane it
//   (1) issues the pulled g loads of its own node on the current plane and,
//       in the same latency window, computes phi = sum of the pulled h on the
//       NEXT plane for the tile plus a one-node halo ring into a four-slot
//       shared-memory ring (phi at a neighbour needs that neighbour's pulled
//       h, so the ring is recomputed; its h reads hit L2),
//   (2) after one barrier, forms the CD stencils from the three resident
//       planes, the moments of g, the local state, and writes h*, g*.
// Four slots make one barrier per plane enough: the slot written in
// iteration j+2 was last read in iteration j, before iteration j+1's barrier.
// HOIST: the g loads of a plane are issued before the phi fill and held in
// registers across it (two latencies overlap, more registers); otherwise the
// fill, the g moments and the collision run as three phases (fewer registers,
// more resident warps to hide the latency).
// The grid is tile columns x chunks along z.  Every column uses the same
// chunk boundaries, so CTAs of neighbouring columns march through the same
// planes at the same time and their halo-ring and chunk-edge re-reads of h
// hit L2.  BAL (one-wave launch): gridDim.z chunks of NZ / gridDim.z planes
// (rounded), the host choosing gridDim.z so that the whole grid is resident
// at once; otherwise chunks of LZ planes.
// ---------------------------------------------------------------- asynchronous loads (FP32)
// 4-byte global -> shared copies that complete in the background (cp.async,
// sm_80 and later): the loads of the next planes stay in flight while the
// CTA collides the current one, with no register held for them.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Moments of the pulled g: m0 = sum g, m1 = sum c g, m2 = sum c c g.
template <typename R>
struct Moments {
    R m0 = 0, mx = 0, my = 0, mz = 0, mxx = 0, myy = 0, mzz = 0, mxy = 0, mxz = 0, myz = 0;
};

// Over opposite pairs (I, J): the odd moments take g_I - g_J, the even ones
// g_I + g_J.  gv(i) returns the pulled g of direction i.  In FP32 the zeroth
// moment, which gives the pressure (P = T m0 + ...), is summed compensated
// like phi (PhiSum: a chain seeded with 1 that collects each addition's
// rounding error): at tau near 1/2 the acoustic modes are barely damped and
// the rounding of a plain 10-term sum accumulates in P over the steps.
template <int LAT, typename GA>
__device__ __forceinline__ auto g_moments(GA gv) {
    using L = Lattice<LAT>;
    using R = decltype(gv(0));
    Moments<R> m;
    PhiSum<float> c0;
    if constexpr (std::is_same<R, float>::value) c0.link(gv(0));
    else m.m0 = gv(0);
    Unroll<1, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = L::op[i];
        if constexpr (i < o) {
            constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
            const R sp = gv(i) + gv(o), dm = gv(i) - gv(o);
            if constexpr (std::is_same<R, float>::value) c0.link(sp);
            else m.m0 += sp;
            if (CX) { m.mx += cmul<CX>(dm); m.mxx += sp; }
            if (CY) { m.my += cmul<CY>(dm); m.myy += sp; }
            if (CZ) { m.mz += cmul<CZ>(dm); m.mzz += sp; }
            if (CX * CY) m.mxy += cmul<CX * CY>(sp);
            if (CX * CZ) m.mxz += cmul<CX * CZ>(sp);
            if (CY * CZ) m.myz += cmul<CY * CZ>(sp);
        }
    });
    if constexpr (std::is_same<R, float>::value) m.m0 = c0.value();
    return m;
}

// Everything of one node after its plane's phi is in the shared ring and the
// moments of its pulled g are known: stencils (three planes of the ring, slots
// sm, s0, sp for z-1, z, z+1; (lx, ly) the node's position in the ring),
// local state, collisions and the writes.  hv(i) returns the node's pulled
// h_i.
template <int LAT, int ST, bool WALLS, int SY, int SX, typename HA>
__device__ __forceinline__ void collide_node(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q>& D,
                                             const Geom& G, const PhysT<typename Storage<ST>::R>& p,
                                             const typename Storage<ST>::R (*phis)[SY][SX], int sm, int s0, int sp,
                                             int lx, int ly, const Moments<typename Storage<ST>::R>& m, HA hv, int x,
                                             int y, int z, int rb) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    constexpr int Q = L::Q;
    NodeState<R> s;
    s.phi = phis[s0][ly][lx];
    // central differences (stencils after Eq. 12):
    // grad phi = sum_i c_i w_i phi(x + c_i) / T  (the -c_i half of the
    // paper's symmetric sum equals the +c_i half), lap = 2 sum w (phi_nb - phi) / T
    // per opposite pair (I, J): phi(x + c_I) - phi(x + c_J) feeds the
    // gradient, phi(x + c_I) + phi(x + c_J) - 2 phi the Laplacian
    R gx = 0, gy = 0, gz = 0, lap = 0;
    Unroll<1, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = L::op[i];
        if constexpr (i < o) {
            constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
            constexpr double W = L::w[i];
            const int slot_p = CZ == 0 ? s0 : (CZ > 0 ? sp : sm);
            const int slot_m = CZ == 0 ? s0 : (CZ > 0 ? sm : sp);
            const R vp = phis[slot_p][ly + CY][lx + CX];
            const R vm = phis[slot_m][ly - CY][lx - CX];
            const R wd = (R)W * (vp - vm);
            if (CX) gx += cmul<CX>(wd);
            if (CY) gy += cmul<CY>(wd);
            if (CZ) gz += cmul<CZ>(wd);
            lap += (R)W * ((vp - s.phi) + (vm - s.phi));
        }
    });
    s.gx = gx * (R)3;
    s.gy = gy * (R)3;
    s.gz = gz * (R)3;
    s.lap = lap * (R)6;
    node_state<R, L::kHasY>(s, p, m.m0, m.mx, m.my, m.mz, m.mxx, m.myy, m.mzz, m.mxy, m.mxz, m.myz);
    const NodeWrites nw = node_writes<LAT>(G, x, y, z);
    const int own = G.base + (z + G.GZ) * G.PXY + rb;
    // moving directions first; the rest population closes sum_i h*_i = phi
    // (Eq. 1 conserves phi at every node; closing it keeps FP32 rounding of
    // sum_i Gamma_i = 1 from biasing the global phi)
    R hsum = 0;
    if constexpr (std::is_same<R, float>::value) {
        // with 16-bit storage hv(i) and the pair collision's outputs are the
        // stored values themselves (pair_state): only the number format is
        // converted on the way to memory
        constexpr bool SH = St::kShifted;
        const PairState q = pair_state<LAT, SH>(s, p);
        float2 hsum2 = make_float2(0.0f, 0.0f);
        auto pk = [&](R v) { return St::pack(v); };
        Unroll<1, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int o = L::op[i];
            if constexpr (i < o) {
                float2 hs, gs;
                collide_pair<LAT, i, SH>(s, q, make_float2(hv(i), hv(o)), &hs, &gs);
                hsum2 = add2(hsum2, hs);
                write_dir<LAT, i, WALLS>(D.hout, G, x, y, z, own, nw, St::pack(hs.x));
                write_dir<LAT, o, WALLS>(D.hout, G, x, y, z, own, nw, St::pack(hs.y));
                write_dir<LAT, i, WALLS>(D.gout, G, x, y, z, own, nw, St::pack(gs.x));
                write_dir<LAT, o, WALLS>(D.gout, G, x, y, z, own, nw, St::pack(gs.y));
                if constexpr (WALLS) {
                    if (p.moving && nw.wall_adj) {
                        // the wall term of g in the units of the stored g
                        const R srho = SH ? s.rho * p.g_scale : s.rho;
                        moving_wall_write<LAT, i>(D.hout, G, x, y, z, hs.x, s.phi, p, pk);
                        moving_wall_write<LAT, o>(D.hout, G, x, y, z, hs.y, s.phi, p, pk);
                        moving_wall_write<LAT, i>(D.gout, G, x, y, z, gs.x, srho, p, pk);
                        moving_wall_write<LAT, o>(D.gout, G, x, y, z, gs.y, srho, p, pk);
                    }
                }
            }
        });
        hsum = hsum2.x + hsum2.y;
    } else {
        Unroll<1, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr double W = L::w[i];
            R hs, gs;
            collide_dir<LAT, i, R>(s, p, hv(i), &hs, &gs);
            hsum += hs;
            write_dir<LAT, i, WALLS>(D.hout, G, x, y, z, own, nw, St::store(hs, (R)W * p.h_shift, (R)1));
            write_dir<LAT, i, WALLS>(D.gout, G, x, y, z, own, nw, St::store(gs, (R)W * p.g_shift, p.g_scale));
            if constexpr (WALLS) {
                if (p.moving && nw.wall_adj) {
                    moving_wall_write<LAT, i>(D.hout, G, x, y, z, hs, s.phi, p,
                                              [&](R v) { return St::store(v, (R)W * p.h_shift, (R)1); });
                    moving_wall_write<LAT, i>(D.gout, G, x, y, z, gs, s.rho, p,
                                              [&](R v) { return St::store(v, (R)W * p.g_shift, p.g_scale); });
                }
            }
        });
    }
    {
        constexpr double W0 = L::w[0];
        R hs, gs;
        collide_dir<LAT, 0, R>(s, p, (R)0, &hs, &gs);
        // stored rest value: phi - sum of the moving h*_i (less w_0 h_shift);
        // with 16-bit storage hsum sums the stored values h*_i - w_i h_shift,
        // so phi - h_shift - hsum is the stored h*_0 - w_0 h_shift (sum w = 1)
        if constexpr (St::kShifted)
            write_dir<LAT, 0, WALLS>(D.hout, G, x, y, z, own, nw, St::pack((s.phi - p.h_shift) - hsum));
        else
            write_dir<LAT, 0, WALLS>(D.hout, G, x, y, z, own, nw, St::store(s.phi - hsum, (R)W0 * p.h_shift, (R)1));
        write_dir<LAT, 0, WALLS>(D.gout, G, x, y, z, own, nw, St::store(gs, (R)W0 * p.g_shift, p.g_scale));
    }
}

template <int LAT, int ST, int TX, int TY>
struct MarchSmem {
    using R = typename Storage<ST>::R;
    static constexpr int HY = Lattice<LAT>::kHasY ? 1 : 0;
    R phis[4][TY + 2 * HY][TX + 2];
    // pulled h of the thread's own node on the last two filled planes: the fill
    // of plane z+1 loads them anyway, the collision of the next iteration
    // reads them back (each thread touches only its own column: no barrier).
    // The moving directions only: the collision closes the rest population
    // with phi.
    R hown[2][Lattice<LAT>::Q - 1][TX * TY];
};

// The march of one CTA over planes [z0, z1) of the tile column at (x0, y0).
// Every thread of the CTA calls it with the same arguments.
template <int LAT, int ST, int TX, int TY, bool HOIST, bool WALLS>
__device__ __forceinline__ void march(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q>& D, const Geom& G,
                                      const PhysT<typename Storage<ST>::R>& p, int x0, int y0, int z0, int z1,
                                      MarchSmem<LAT, ST, TX, TY>& sm) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    constexpr int Q = L::Q;
    constexpr int HY = L::kHasY ? 1 : 0;
    constexpr int SX = TX + 2, SY = TY + 2 * HY;
    auto& phis = sm.phis;
    auto& hown = sm.hown;
    const int tid = threadIdx.x + TX * threadIdx.y;

    // phi of plane zp (unwrapped) into ring slot: every halo position is
    // mapped to the node whose phi it holds (periodic image or wall mirror)
    constexpr int NRING = SX * SY - TX * TY;   // halo positions of the phi tile
    const int tx = threadIdx.x, ty = threadIdx.y;
    auto ring_pos = [&](int k, int* lx, int* ly) {
        if (HY) {
            if (k < SX) { *lx = k; *ly = 0; }
            else if (k < 2 * SX) { *lx = k - SX; *ly = SY - 1; }
            else { const int r = k - 2 * SX; *lx = (r & 1) ? SX - 1 : 0; *ly = 1 + (r >> 1); }
        } else {
            *lx = k == 0 ? 0 : SX - 1;
            *ly = 0;
        }
    };
    // x-y parts of the pull offsets, fixed for the whole march: the thread's
    // own column (the g pulls of an active thread share it) and, when the
    // ring has no more positions than the CTA has threads, its ring position
    PullOffsets own_xy, ring_xy;
    pull_xy(G, stencil_coord(x0 + tx, G.NX, G.wall[0]), HY ? stencil_coord(y0 + ty, G.NY, G.wall[1]) : y0, own_xy);
    ring_xy = own_xy;   // threads without a ring position: valid offsets, loads predicated off
    constexpr bool kOneRing = NRING <= TX * TY;
    int ring_off = 0;
    if (kOneRing && tid < NRING) {
        int lx, ly;
        ring_pos(tid, &lx, &ly);
        ring_off = ly * SX + lx;
        pull_xy(G, stencil_coord(x0 + lx - 1, G.NX, G.wall[0]),
                HY ? stencil_coord(y0 + ly - HY, G.NY, G.wall[1]) : y0, ring_xy);
    }
    // 16-bit storage keeps h_i - w_i h_shift: the fill sums and keeps the
    // stored values as they are (phi = their sum + h_shift, as sum w_i = 1)
    // and the collision works on them, so no population is shifted on load
    // or store
    auto with_shift = [&](R v) {
        if constexpr (St::kShifted) return v + p.h_shift;
        else return v;
    };
    auto ring_phi = [&](PullOffsets po) {
        checked_offsets(po, G.NP);
        PhiSum<R> phi;
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            phi.add(St::raw(pull_pad<LAT, i, false>(D.hin, po)));
        });
        return with_shift(phi.value());
    };
    // the thread's own position (its pulled h kept in hown[hs]) and its share
    // of the halo ring; with one ring position per thread, both sets of loads
    // are issued before either is summed (one latency instead of two).  A
    // warp none of whose threads has a ring
    // position (the ring positions are the lowest thread indices) loads and
    // sums its own column only.
    auto fill = [&](int zp, int slot, int hs) {
        const int zz = stencil_coord(zp, G.NZ, G.wall[2]);
        if constexpr (kOneRing) {
            PullOffsets po = own_xy;
            pull_z(G, zz, po);
            checked_offsets(po, G.NP);
            typename St::S hv[Q];
            if ((tid & ~31) < NRING) {   // uniform over the warp
                PullOffsets pr = ring_xy;
                pull_z(G, zz, pr);
                checked_offsets(pr, G.NP);
                const bool ring = tid < NRING;
                typename St::S rv[Q];
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    hv[i] = ld_keep(pull_ptr<LAT, i>(D.hin, po));
                    rv[i] = ld_keep_if(pull_ptr<LAT, i>(D.hin, pr), ring);
                });
                PhiSum<R> phi, rphi;
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    const R v = St::raw(hv[i]);
                    if constexpr (i > 0) hown[hs][i - 1][tid] = v;
                    phi.add(v);
                    rphi.add(St::raw(rv[i]));
                });
                phis[slot][ty + HY][tx + 1] = with_shift(phi.value());
                if (ring) (&phis[slot][0][0])[ring_off] = with_shift(rphi.value());
            } else {
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    hv[i] = ld_keep(pull_ptr<LAT, i>(D.hin, po));
                });
                PhiSum<R> phi;
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    const R v = St::raw(hv[i]);
                    if constexpr (i > 0) hown[hs][i - 1][tid] = v;
                    phi.add(v);
                });
                phis[slot][ty + HY][tx + 1] = with_shift(phi.value());
            }
        } else {
            {
                PullOffsets po = own_xy;
                pull_z(G, zz, po);
                checked_offsets(po, G.NP);
                PhiSum<R> phi;
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    const R v = St::raw(pull_pad<LAT, i, false>(D.hin, po));
                    if constexpr (i > 0) hown[hs][i - 1][tid] = v;
                    phi.add(v);
                });
                phis[slot][ty + HY][tx + 1] = with_shift(phi.value());
            }
            for (int k = tid; k < NRING; k += TX * TY) {
                int lx, ly;
                ring_pos(k, &lx, &ly);
                const int xx = stencil_coord(x0 + lx - 1, G.NX, G.wall[0]);
                const int yy = HY ? stencil_coord(y0 + ly - HY, G.NY, G.wall[1]) : y0;
                phis[slot][ly][lx] = ring_phi(pull_offsets(G, xx, yy, zz));
            }
        }
    };

    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < G.NX && y < G.NY;
    const int rb = (y + G.GY) * G.PX + x + G.GX;
    fill(z0 - 1, 0, 0);
    fill(z0, 1, 1);

    for (int z = z0; z < z1; ++z) {
        const int j = z - z0;
        PullOffsets po = own_xy;   // x, y are the own column when active
        pull_z(G, z, po);
        checked_offsets(po, G.NP);
        // (1) g of this node (streamed) and the phi fill of the next plane
        Moments<R> m;
        auto g_load = [&](R* gv) {
            Unroll<0, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr double W = L::w[i];
                gv[i] = St::load(pull_pad<LAT, i, true>(D.gin, po), (R)W * p.g_shift, p.g_inv_scale);
            });
        };
        if (HOIST) {
            R gv[Q];
            if (active) g_load(gv);
            fill(z + 1, (j + 2) & 3, j & 1);
            if (active) m = g_moments<LAT>([&](int i) { return gv[i]; });
        } else {
            fill(z + 1, (j + 2) & 3, j & 1);
            if (active) {
                R gv[Q];
                g_load(gv);
                m = g_moments<LAT>([&](int i) { return gv[i]; });
            }
        }
        __syncthreads();
        if (active) {
            auto hv = [&](int i) { return hown[(j + 1) & 1][i - 1][tid]; };   // i >= 1
            // only a node next to a wall writes bounce-back ghost cells: the
            // rest take the wall-free collision (fewer live registers)
            if (WALLS && node_writes<LAT>(G, x, y, z).wall_adj)
                collide_node<LAT, ST, true>(D, G, p, phis, j & 3, (j + 1) & 3, (j + 2) & 3, tx + 1, ty + HY, m, hv, x,
                                            y, z, rb);
            else
                collide_node<LAT, ST, false>(D, G, p, phis, j & 3, (j + 1) & 3, (j + 2) & 3, tx + 1, ty + HY, m, hv,
                                             x, y, z, rb);
        }
    }
}

template <int LAT, int ST, int TX, int TY, int MINB, bool HOIST, bool BAL, bool WALLS>
__global__ void __launch_bounds__(TX * TY, MINB)
step_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G, PhysT<typename Storage<ST>::R> p,
            int LZ) {
    __shared__ MarchSmem<LAT, ST, TX, TY> sm;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = BAL ? (int)((long long)blockIdx.z * G.NZ / gridDim.z) : blockIdx.z * LZ;
    const int z1 = BAL ? (int)((long long)(blockIdx.z + 1) * G.NZ / gridDim.z) : min(z0 + LZ, G.NZ);
    march<LAT, ST, TX, TY, HOIST, WALLS>(D, G, p, x0, y0, z0, z1, sm);
}

// Halo-ring position k of a TX x TY tile (ring of SX x SY, SX = TX + 2,
// SY = TY + 2 HY): the top row, the bottom row, then the side columns.
template <int TX, int TY, int HY>
__device__ __forceinline__ void ring_pos(int k, int* lx, int* ly) {
    constexpr int SX = TX + 2, SY = TY + 2 * HY;
    if (HY) {
        if (k < SX) { *lx = k; *ly = 0; }
        else if (k < 2 * SX) { *lx = k - SX; *ly = SY - 1; }
        else { const int r = k - 2 * SX; *lx = (r & 1) ? SX - 1 : 0; *ly = 1 + (r >> 1); }
    } else {
        *lx = k == 0 ? 0 : SX - 1;
        *ly = 0;
    }
}

template <int LAT, int TX, int TY>
struct AsyncSmem {
    static constexpr int Q = Lattice<LAT>::Q;
    static constexpr int HY = Lattice<LAT>::kHasY ? 1 : 0;
    static constexpr int SX = TX + 2, SY = TY + 2 * HY;
    static constexpr int NT = TX * TY;
    static constexpr int NRING = SX * SY - NT;
    float phis[4][SY][SX];
    float hown[3][Q][NT];    // own pulled h of plane q in slot q % 3 (collided, summed, in flight)
    float gbuf[Q][NT];       // own pulled g of the next plane to reduce
    float ring[Q][NRING];    // pulled h of the halo ring positions of the next plane to sum
};

// The march of march() with every population load issued as cp.async ahead
// of its use: in the iteration of plane z, once the copies of plane z + 1's
// h and plane z's g have landed and been reduced (phi into the shared ring,
// g into its moments), the copies of plane z + 2's h (own position and halo
// ring) and plane z + 1's g are issued, and stay in flight through the
// barrier and the collision of plane z.  Every thread reads back only its own
// copies (cp.async.wait_group suffices); phi goes through the shared ring and
// the one barrier per plane, as in march().  Storage FP32.
template <int LAT, int TX, int TY, bool WALLS>
__device__ __forceinline__ void march_async(const DirPtrs<float, Lattice<LAT>::Q>& D, const Geom& G,
                                            const PhysT<float>& p, int x0, int y0, int z0, int z1,
                                            AsyncSmem<LAT, TX, TY>& sm) {
    using L = Lattice<LAT>;
    using Sm = AsyncSmem<LAT, TX, TY>;
    constexpr int Q = L::Q;
    constexpr int HY = Sm::HY, NT = Sm::NT, NRING = Sm::NRING;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
    const int xo = stencil_coord(x0 + tx, G.NX, G.wall[0]);
    const int yo = HY ? stencil_coord(y0 + ty, G.NY, G.wall[1]) : y0;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < G.NX && y < G.NY;
    const int rb = (y + G.GY) * G.PX + x + G.GX;

    // copies of the pulled h of plane zp: own position into hown[hs], the
    // thread's halo-ring positions into ring
    auto issue_fill = [&](int zp, int hs) {
        const int zz = stencil_coord(zp, G.NZ, G.wall[2]);
        PullOffsets po = pull_offsets(G, xo, yo, zz);
        checked_offsets(po, G.NP);
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            cp_async4(&sm.hown[hs][i][tid], pull_ptr<LAT, i>(D.hin, po));
        });
        for (int r = tid; r < NRING; r += NT) {
            int lx, ly;
            ring_pos<TX, TY, HY>(r, &lx, &ly);
            const int xx = stencil_coord(x0 + lx - 1, G.NX, G.wall[0]);
            const int yy = HY ? stencil_coord(y0 + ly - HY, G.NY, G.wall[1]) : y0;
            PullOffsets pr = pull_offsets(G, xx, yy, zz);
            checked_offsets(pr, G.NP);
            Unroll<0, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                cp_async4(&sm.ring[i][r], pull_ptr<LAT, i>(D.hin, pr));
            });
        }
    };
    // phi of the landed plane (own h in hown[hs]) into ring slot `slot`
    auto sum_fill = [&](int slot, int hs) {
        PhiSum<float> phi;
        Unroll<0, Q>::run([&](auto ic) { phi.add(sm.hown[hs][decltype(ic)::value][tid]); });
        sm.phis[slot][ty + HY][tx + 1] = phi.value();
        for (int r = tid; r < NRING; r += NT) {
            int lx, ly;
            ring_pos<TX, TY, HY>(r, &lx, &ly);
            PhiSum<float> v;
            Unroll<0, Q>::run([&](auto ic) { v.add(sm.ring[decltype(ic)::value][r]); });
            sm.phis[slot][ly][lx] = v.value();
        }
    };
    auto issue_g = [&](int zg) {
        if (!active) return;
        PullOffsets po = pull_offsets(G, x, y, zg);
        checked_offsets(po, G.NP);
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            cp_async4(&sm.gbuf[i][tid], pull_ptr<LAT, i>(D.gin, po));
        });
    };

    // plane index q = z - z0 + 1 (plane z0 - 1 is q = 0); one copy group in flight
    issue_fill(z0 - 1, 0);
    cp_async_commit();
    cp_async_wait<0>();
    sum_fill(0, 0);
    issue_fill(z0, 1);
    cp_async_commit();
    cp_async_wait<0>();
    sum_fill(1, 1);
    issue_fill(z0 + 1, 2);
    issue_g(z0);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        const int q = z - z0 + 1;
        cp_async_wait<0>();   // plane z + 1's h and plane z's g have landed
        sum_fill((q + 1) & 3, (q + 1) % 3);
        Moments<float> m;
        if (active) m = g_moments<LAT>([&](int i) { return sm.gbuf[i][tid]; });
        if (z + 2 <= z1) issue_fill(z + 2, (q + 2) % 3);
        if (z + 1 < z1) issue_g(z + 1);
        cp_async_commit();
        __syncthreads();
        if (active)
            collide_node<LAT, ST_F32, WALLS>(D, G, p, sm.phis, (q - 1) & 3, q & 3, (q + 1) & 3, tx + 1, ty + HY, m,
                                             [&](int i) { return sm.hown[q % 3][i][tid]; }, x, y, z, rb);
    }
    cp_async_wait<0>();
}

template <int LAT, int TX, int TY, int MINB, bool WALLS>
__global__ void __launch_bounds__(TX * TY, MINB)
step_async_kernel(const DirPtrs<float, Lattice<LAT>::Q> D, Geom G, PhysT<float> p, int LZ) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<AsyncSmem<LAT, TX, TY>*>(smem_raw);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * LZ;
    const int z1 = min(z0 + LZ, G.NZ);
    march_async<LAT, TX, TY, WALLS>(D, G, p, x0, y0, z0, z1, sm);
}

// ---------------------------------------------------------------- batch
// One grid of a batch: its geometry (base = its block in the shared
// population arrays) and its parameters in the kernel's arithmetic type.
template <typename R>
struct BatchCase {
    Geom G;
    PhysT<R> p;
};

// Work item: grid c, tile column x0 (y0 = 0), planes [z0, z1).
struct BatchItem {
    int c, x0, z0, z1;
};

// Persistent step over a work list of many grids: CTAs take items in list
// order from an atomic counter (counters[0]) until the list is exhausted; the
// last CTA to finish (counted in counters[1]) sets both back to zero for the
// next launch.  Grids of one batch share the population arrays (population i
// of every grid at D.*[i], grid c from its base), so one parameter block
// serves every item.  Walls are handled per grid (WALLS = true).
template <int LAT, int ST, int TX, int MINB, bool HOIST>
__global__ void __launch_bounds__(TX, MINB)
batch_step_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D,
                  const BatchCase<typename Storage<ST>::R>* __restrict__ cases, const BatchItem* __restrict__ items,
                  int n_items, int* counters) {
    using R = typename Storage<ST>::R;
    __shared__ MarchSmem<LAT, ST, TX, 1> sm;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&counters[0], 1);
        __syncthreads();
        const int k = s_item;
        if (k >= n_items) break;
        const BatchItem it = items[k];
        const Geom G = cases[it.c].G;
        const PhysT<R> p = cases[it.c].p;
        march<LAT, ST, TX, 1, HOIST, true>(D, G, p, it.x0, 0, it.z0, it.z1, sm);
        // the next item's fills overwrite the phi ring, and thread 0 s_item
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // every CTA counted here has made its last claim on counters[0]
        if (atomicAdd(&counters[1], 1) == (int)gridDim.x - 1) {
            counters[0] = 0;
            counters[1] = 0;
        }
    }
}

// ---------------------------------------------------------------- helper kernels
// (node counts are below 2^31, checked on the host: 32-bit division)
__device__ __forceinline__ void node_coords(const Geom& G, long long n, int* x, int* y, int* z) {
    const int k = (int)n;
    const int q = k / G.NX;
    *x = k - q * G.NX;
    *z = q / G.NY;
    *y = q - *z * G.NY;
}

// h_0 += *delta at every node (the rest population pulls from its own cell,
// so phi of every node rises by *delta): the uniform re-imposition of the
// total of phi after 16-bit rounding has moved it.
template <int LAT, int ST>
__global__ void shift_rest_kernel(typename Storage<ST>::S* __restrict__ h0, Geom G, PhysT<typename Storage<ST>::R> p,
                                  const double* __restrict__ delta) {
    using St = Storage<ST>;
    using R = typename St::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    const int x = (int)(n % G.NX), y = (int)((n / G.NX) % G.NY), z = (int)(n / ((long long)G.NX * G.NY));
    const int k = pidx(G, x, y, z);
    const R sh = (R)Lattice<LAT>::w[0] * p.h_shift;
    h0[k] = St::store(St::load(h0[k], sh, (R)1) + (R)*delta, sh, (R)1);
}

// phi = sum_i of the pulled h at every node (double output, node order).
template <int LAT, int ST>
__global__ void phi_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G, Phys p, double* phi) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int x, y, z;
    node_coords(G, n, &x, &y, &z);
    const PullOffsets po = pull_offsets(G, x, y, z);
    double acc = 0;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr double W = L::w[i];
        acc += (double)St::load(pull_pad<LAT, i, false>(D.hin, po), (R)(W * p.h_shift), (R)1);
    });
    phi[n] = acc;
}

// CD stencils of a double field (node order) at node (x, y, z), in the
// arithmetic type R (the values are rounded to R first): FP64 for the
// diagnostics and FP64 storage, FP32 for initialising FP32 and 16-bit
// storage (whose kernels compute in FP32; GB300's FP64 rate is low).
template <int LAT, typename R = double>
__device__ __forceinline__ void stencils(const double* __restrict__ phi, const Geom& G, int x, int y, int z,
                                         R* gx, R* gy, R* gz, R* lap) {
    using L = Lattice<LAT>;
    auto at = [&](int a, int b, int c) { return (R)phi[a + G.NX * (b + G.NY * c)]; };
    const R f = at(x, y, z);
    R ax = 0, ay = 0, az = 0, l = 0;
    Unroll<1, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
        constexpr double W = L::w[i];
        const R v = at(stencil_coord(x + CX, G.NX, G.wall[0]), stencil_coord(y + CY, G.NY, G.wall[1]),
                       stencil_coord(z + CZ, G.NZ, G.wall[2]));
        if (CX) ax += (R)(CX * W) * v;
        if (CY) ay += (R)(CY * W) * v;
        if (CZ) az += (R)(CZ * W) * v;
        l += (R)W * (v - f);
    });
    *gx = (R)3 * ax; *gy = (R)3 * ay; *gz = (R)3 * az; *lap = (R)6 * l;
}

// Macroscopic fields (phi given): P and u (internal axes), written in
// double.  Computed in the kernels' arithmetic type R: FP64 for FP64 storage,
// FP32 for FP32 and 16-bit storage (their values carry FP32 rounding
// already, and GB300's FP64 rate is low).  Only the flow fields of the step
// (node_flow), not the collision's second moments.
template <int LAT, int ST>
__global__ void macro_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G,
                             PhysT<typename Storage<ST>::R> p, const double* __restrict__ phi, double* P, double* ux,
                             double* uy, double* uz) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int x, y, z;
    node_coords(G, n, &x, &y, &z);
    const PullOffsets po = pull_offsets(G, x, y, z);
    NodeState<R> s;
    s.phi = (R)phi[n];
    stencils<LAT, R>(phi, G, x, y, z, &s.gx, &s.gy, &s.gz, &s.lap);
    R m0 = 0, mx = 0, my = 0, mz = 0;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
        constexpr double W = L::w[i];
        const R v = St::load(pull_pad<LAT, i, false>(D.gin, po), (R)W * p.g_shift, p.g_inv_scale);
        m0 += v;
        if (CX) mx += cmul<CX>(v);
        if (CY) my += cmul<CY>(v);
        if (CZ) mz += cmul<CZ>(v);
    });
    node_flow<R, L::kHasY>(s, p, m0, mx, my, mz);
    P[n] = (double)s.P;
    ux[n] = (double)s.ux;
    uy[n] = (double)s.uy;
    uz[n] = (double)s.uz;
}

// Where the value pulled by node (x, y, z) for direction I lives: x - c_I
// wrapped along periodic axes (the real cell; its ghost images are written
// by store_rep), the ghost cell across a wall otherwise.
template <int LAT, int I>
__device__ __forceinline__ void pull_cell(const Geom& G, int x, int y, int z, int* tx, int* ty, int* tz) {
    using L = Lattice<LAT>;
    int a = x - L::cx[I], b = y - L::cy[I], c = z - L::cz[I];
    if (!G.wall[0]) a = a < 0 ? a + G.NX : (a >= G.NX ? a - G.NX : a);
    if (!G.wall[1]) b = b < 0 ? b + G.NY : (b >= G.NY ? b - G.NY : b);
    if (!G.wall[2]) c = c < 0 ? c + G.NZ : (c >= G.NZ ? c - G.NZ : c);
    *tx = a; *ty = b; *tz = c;
}

// Store v at ghost-padded (x, y, z) of one population array and, for a cell
// within kRep of an x or y edge, at its periodic images (store_rep); a cell
// away from the edges has none, and is written once.
template <typename S>
__device__ __forceinline__ void store_cell(S* __restrict__ arr, const Geom& G, int x, int y, int z, S v) {
    const bool near_x = !G.wall[0] && (x < kRep || x >= G.NX - kRep);
    const bool near_y = G.GY > 0 && !G.wall[1] && (y < kRep || y >= G.NY - kRep);
    if (near_x || near_y || x < 0 || x >= G.NX || y < 0 || y >= G.NY) store_rep(arr, G, x, y, z, v);
    else arr[pidx(G, x, y, z)] = v;
}

// Equilibrium initialisation (h = h^eq, g = g^eq of the given fields),
// written where the next pull reads it, in the kernels' arithmetic type R
// (FP32 for FP32 and 16-bit storage, FP64 for FP64 storage): the stored
// values carry the storage rounding either way.
// With neq, g also carries the filtered non-equilibrium part of a state
// that has relaxed onto its flow: Phi_i : Pi(1) (Eq. 11) with the
// Chapman-Enskog estimate Pi(1) = -tau_mix T rho (grad u + grad u^T), grad u
// by the central differences of grad phi.
template <int LAT, int ST>
__global__ void init_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G,
                            PhysT<typename Storage<ST>::R> p, const double* __restrict__ phi,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ uz, const double* __restrict__ P, int neq) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int x, y, z;
    node_coords(G, n, &x, &y, &z);
    NodeState<R> s;
    s.phi = (R)phi[n];
    stencils<LAT, R>(phi, G, x, y, z, &s.gx, &s.gy, &s.gz, &s.lap);
    const R rho_dif = p.rho_dif;
    s.rho = p.rho_L + s.phi * rho_dif;
    s.mu = p.beta * s.phi * (s.phi - (R)1) * (s.phi - (R)0.5) - p.kappa * s.lap;
    const R fr = p.force_mode == 0 ? s.rho : s.rho - p.rho_bar;
    s.Fx = fr * p.g[0]; s.Fy = fr * p.g[1]; s.Fz = fr * p.g[2];
    s.ux = (R)ux[n]; s.uy = L::kHasY ? (R)uy[n] : (R)0; s.uz = (R)uz[n];
    s.P = (R)P[n];
    s.usq = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
    s.ug = s.ux * s.gx + s.uy * s.gy + s.uz * s.gz;
    s.uF = s.ux * s.Fx + s.uy * s.Fy + s.uz * s.Fz;
    const R gmag = sqrt(s.gx * s.gx + s.gy * s.gy + s.gz * s.gz);
    const R inv = (R)1 / (gmag + p.eps);
    s.nx = s.gx * inv; s.ny = s.gy * inv; s.nz = s.gz * inv;
    const R d = s.phi - (R)0.5;
    s.theta = p.theta_coef * ((R)1 - (R)4 * d * d);
    if (p.dtheta_coef != (R)0) {   // Eq. 14, as in node_state
        const R t = ((R)2 * s.phi - (R)1) * s.lap;
        s.theta -= p.dtheta_coef * (t > (R)0 ? t : (R)0) * gmag;
    }
    // Pi(1) components (zero without neq)
    R nxx = 0, nyy = 0, nzz = 0, nxy = 0, nxz = 0, nyz = 0, ntr3 = 0;
    if (neq) {
        R d[3][3], l;   // d[a][b] = d_a u_b
        stencils<LAT, R>(ux, G, x, y, z, &d[0][0], &d[1][0], &d[2][0], &l);
        if (L::kHasY) stencils<LAT, R>(uy, G, x, y, z, &d[0][1], &d[1][1], &d[2][1], &l);
        else d[0][1] = d[1][1] = d[2][1] = (R)0;
        stencils<LAT, R>(uz, G, x, y, z, &d[0][2], &d[1][2], &d[2][2], &l);
        const R pc = s.phi < (R)0 ? (R)0 : (s.phi > (R)1 ? (R)1 : s.phi);
        const R tau = (R)1 / (p.om_L + pc * p.om_dif);
        const R cf = -tau * (R)(1.0 / 3.0) * s.rho;
        nxx = (R)(cf * 2 * d[0][0]); nyy = (R)(cf * 2 * d[1][1]); nzz = (R)(cf * 2 * d[2][2]);
        nxy = (R)(cf * (d[0][1] + d[1][0])); nxz = (R)(cf * (d[0][2] + d[2][0])); nyz = (R)(cf * (d[1][2] + d[2][1]));
        ntr3 = (nxx + nyy + nzz) * (R)(1.0 / 3.0);
    }
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
        constexpr double W = L::w[i];
        const R w = (R)W;
        const R cu = cdot3<CX, CY, CZ>(s.ux, s.uy, s.uz);
        const R Gm1 = w * ((R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * s.usq);   // Gamma_i - w_i
        const R Gm = w + Gm1;
        const R cgr = cdot3<CX, CY, CZ>(s.gx, s.gy, s.gz);
        const R cF = cdot3<CX, CY, CZ>(s.Fx, s.Fy, s.Fz);
        const R K = (Gm1 * rho_dif + (R)3 * Gm * s.mu) * (cgr - s.ug) + (R)3 * Gm * (cF - s.uF);
        R geq = s.rho * Gm1 + (R)3 * w * s.P - (R)0.5 * K;
        if (p.hocorr) geq += w * cu * (R)0.75 * rho_dif * s.lap;
        if (neq) {   // w_i / (2 T^2) (c_i c_i : Pi(1) - T tr Pi(1))
            const R ccp = cdot3<CX * CX, CY * CY, CZ * CZ>(nxx, nyy, nzz) +
                          (R)2 * cdot3<CX * CY, CX * CZ, CY * CZ>(nxy, nxz, nyz);
            geq += (R)4.5 * w * (ccp - ntr3);
        }
        const R heq = s.phi * Gm + s.theta * w * cdot3<CX, CY, CZ>(s.nx, s.ny, s.nz);
        int tx, ty, tz;
        pull_cell<LAT, i>(G, x, y, z, &tx, &ty, &tz);
        store_cell(D.hout[i], G, tx, ty, tz, St::store(heq, w * p.h_shift, (R)1));
        store_cell(D.gout[i], G, tx, ty, tz, St::store(geq, w * p.g_shift, p.g_scale));
    });
}

// Pre-collision populations out (double, population-major, node order).
template <int LAT, int ST>
__global__ void get_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G, Phys p, double* h,
                           double* g) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int x, y, z;
    node_coords(G, n, &x, &y, &z);
    const PullOffsets po = pull_offsets(G, x, y, z);
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr double W = L::w[i];
        h[(long long)i * G.N + n] = (double)St::load(pull_pad<LAT, i, false>(D.hin, po), (R)(W * p.h_shift), (R)1);
        g[(long long)i * G.N + n] = (double)St::load(pull_pad<LAT, i, false>(D.gin, po), (R)(W * p.g_shift),
                                                     (R)p.g_inv_scale);
    });
}

template <int LAT, int ST>
__global__ void set_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G, Phys p,
                           const double* __restrict__ h, const double* __restrict__ g) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using R = typename St::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int x, y, z;
    node_coords(G, n, &x, &y, &z);
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr double W = L::w[i];
        int tx, ty, tz;
        pull_cell<LAT, i>(G, x, y, z, &tx, &ty, &tz);
        store_rep(D.hout[i], G, tx, ty, tz, St::store((R)h[(long long)i * G.N + n], (R)(W * p.h_shift), (R)1));
        store_rep(D.gout[i], G, tx, ty, tz, St::store((R)g[(long long)i * G.N + n], (R)(W * p.g_shift), (R)p.g_scale));
    });
}

// Periodic images of the ghost band after a step.  A ghost cell c of
// population i is pulled by r = c + c_i (a node, or a halo position of a CTA
// tile).  Let R be r wrapped along the periodic axes; if R is not a node the
// cell is never needed.  Otherwise the value R pulls is the one the step
// stored for it, at S = R - c_i wrapped along the periodic axes (the node's
// own cell, or R's bounce-back cell if the pull crosses a wall).
// The halo copies that cell into c when they differ.  Band: x within kRep of
// the nodes, y within GY, every plane (ring cells only), plus the whole band
// area of the ghost planes behind z walls.
template <int LAT, int ST>
__global__ void halo_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G) {
    using L = Lattice<LAT>;
    const int Ry = G.GY < kRep ? G.GY : kRep;
    const int BXW = G.NX + 2 * kRep, BYW = G.NY + 2 * Ry;
    const int ring = BXW * BYW - G.NX * G.NY;
    const long long nA = (long long)ring * G.NZ;
    const long long nB = G.wall[2] ? 2LL * BXW * BYW : 0;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= nA + nB) return;
    int x, y, z;
    if (k < nA) {
        z = (int)(k / ring);
        int r = (int)(k % ring);
        // ring order: Ry rows below, the NY middle rows (2 kRep cells each), Ry rows above
        if (r < Ry * BXW) { y = -Ry + r / BXW; x = -kRep + r % BXW; }
        else if ((r -= Ry * BXW) < G.NY * 2 * kRep) {
            y = r / (2 * kRep);
            const int c = r % (2 * kRep);
            x = c < kRep ? -kRep + c : G.NX + (c - kRep);
        } else {
            r -= G.NY * 2 * kRep;
            y = G.NY + r / BXW; x = -kRep + r % BXW;
        }
    } else {
        k -= nA;
        z = k < BXW * BYW ? -1 : G.NZ;
        const int a = (int)(k % (BXW * BYW));
        x = -kRep + a % BXW;
        y = -Ry + a / BXW;
    }
    auto wrap = [](int v, int n) { return ((v % n) + n) % n; };
    const int dst = pidx(G, x, y, z);
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
        int Rx = x + CX, Ry_ = y + CY, Rz = z + CZ;
        if (!G.wall[0]) Rx = wrap(Rx, G.NX);
        if (!G.wall[1]) Ry_ = wrap(Ry_, G.NY);
        if (!G.wall[2]) Rz = wrap(Rz, G.NZ);
        if (Rx < 0 || Rx >= G.NX || Ry_ < 0 || Ry_ >= G.NY || Rz < 0 || Rz >= G.NZ) return;
        // the cell the step stored it in: a node's own cell or R's bounce-back
        // cell across a wall, wrapped along every periodic axis either way
        int Sx = Rx - CX, Sy = Ry_ - CY, Sz = Rz - CZ;
        if (!G.wall[0]) Sx = wrap(Sx, G.NX);
        if (!G.wall[1]) Sy = wrap(Sy, G.NY);
        if (!G.wall[2]) Sz = wrap(Sz, G.NZ);
        const int src = pidx(G, Sx, Sy, Sz);
        if (src != dst) {
            D.hout[i][dst] = D.hout[i][src];
            D.gout[i][dst] = D.gout[i][src];
        }
    });
}

}  // namespace lbm
