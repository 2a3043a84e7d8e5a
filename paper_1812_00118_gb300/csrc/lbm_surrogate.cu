// Kernels of the learned warm-start surrogate (include/lbm_surrogate.h):
// periodic 3x3 convolutions on BF16 tensor cores with FP32 accumulation, and
// the elementwise, pooling, loss and optimiser kernels around them.
//
// Tensors are channels-last: pixel p = (n H + y) W + x, element (p, c) at
// p * stride + c (a channel stride larger than the channel count lets a
// layer read or write a slice of a wider tensor, which is how the skip
// concatenation is laid out).  Conv weights are [Co][9][Ci] (tap = 3 dy + dx,
// input channels fastest).  Channel counts of convolutions are multiples of
// 16 (zero-padded by the caller), pixel counts multiples of 16.
//
// The forward (and input-gradient) convolution runs on the tcgen05 tensor
// cores with the accumulator in tensor memory (conv_row_kernel for images
// whose width is a multiple of 128, conv_tc_kernel otherwise); so does the
// weight gradient, a GEMM over pixels, for widths that are multiples of 64
// (conv_wgrad_row_kernel), with the warp-level mma.sync m16n8k16 BF16 kernel
// (fragments gathered straight from the channels-last tensors) for the
// rest.  All are implicit GEMMs without an im2col buffer.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include "lbm.h"
#include "lbm_surrogate.h"

namespace {

using bf16 = __nv_bfloat16;

int check(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_pair(const bf16* lo, const bf16* hi) {
    const uint32_t a = *reinterpret_cast<const unsigned short*>(lo);
    const uint32_t b = *reinterpret_cast<const unsigned short*>(hi);
    return a | (b << 16);
}

// pixel p shifted by (dy, dx) with periodic wrap inside its image
__device__ __forceinline__ long long shift_pixel(long long p, int H, int W, int dy, int dx) {
    const long long hw = (long long)H * W;
    const long long n = p / hw;
    const int r = (int)(p - n * hw);
    int y = r / W + dy, x = r % W + dx;
    y = y < 0 ? y + H : (y >= H ? y - H : y);
    x = x < 0 ? x + W : (x >= W ? x - W : x);
    return n * hw + (long long)y * W + x;
}

// ---------------------------------------------------------------- tcgen05 convolution
// The forward convolution (and the input-gradient convolution, the same
// operation on flipped weights) as an implicit GEMM on the fifth-generation
// tensor cores: D[pixel, co] = sum over (tap, ci) of A[pixel, (tap, ci)]
// B[(tap, ci), co], with A the shifted activations and B the weights, both
// bf16 and K-major (channels contiguous), D in FP32 in tensor memory.
//
// A CTA of 128 threads owns 128 consecutive pixels and every output channel
// (MMA shape M = 128, N = Co, K = 16).  The K loop runs over stages (tap,
// block of up to 64 input channels).  Per stage every thread copies its
// pixel's shifted channel row (16-byte cp.async; rows past the last pixel
// are zero-filled) and a share of the tap's weight rows into one of four
// shared-memory buffers, in the no-swizzle canonical layout of the tensor
// core: 8 x 16-byte core matrices, rows 16 bytes apart, 8-row groups 128
// bytes apart (stride byte offset), the 8-channel chunks one after another
// (leading byte offset = rows x 16 bytes).  The copies run two stages ahead
// of the MMAs: once a stage's copies have landed, thread 0 issues its MMAs
// and commits them to the buffer's mbarrier, and a buffer is refilled only
// after its mbarrier shows the MMAs that read it done.  The epilogue reads
// the accumulator back with tcgen05.ld (warp w reads lanes 32w..32w+31, one
// pixel per thread), adds the bias and stores FP32.
//
// Every wait is bounded: a wait that gives up sets *err (read by
// lbm_sg_status) and the CTA skips its epilogue, frees its tensor memory and
// returns.
constexpr int kTcM = 128;        // pixels per CTA (MMA M)
constexpr int kTcK = 64;         // input channels per stage
constexpr int kTcBuf = 4;        // stage buffers in shared memory
constexpr int kTcAhead = 2;      // stages whose copies are in flight ahead of the MMAs
constexpr long kTcPolls = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// true once the phase of the given parity has completed; false after `polls` tries
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long polls) {
    for (long i = 0; i < polls; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// shared-memory matrix descriptor, no swizzle: start address, leading and
// stride byte offsets (all in 16-byte units), descriptor version 1
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N / 8 and M / 16
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// 16 consecutive FP32 columns of the thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128, 1)
conv_tc_kernel(const bf16* __restrict__ x, int csx, const bf16* __restrict__ w, const float* __restrict__ bias,
               float* __restrict__ y, int csy, long long M, int H, int W, int Ci, int Co, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kTcBuf];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long p0 = (long long)blockIdx.x * kTcM;
    const int kcap = Ci < kTcK ? Ci : kTcK;   // channels per stage buffer
    const uint32_t a_bytes = kTcM * kcap * 2, stage_bytes = a_bytes + (uint32_t)Co * kcap * 2;
    const uint32_t sb = smem_u32(smem);
    // buffer b: A at sb + b stage_bytes, B a_bytes after it; its barrier at bar0 + 8 b
    const uint32_t bar0 = smem_u32(&bars[0]);
    const uint32_t ncols = Co <= 32 ? 32u : (Co <= 64 ? 64u : 128u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < kTcBuf; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc_idesc_bf16(kTcM, Co);
    const int nkb = (Ci + kTcK - 1) / kTcK;
    const int nst = 9 * nkb;
    const long long p = p0 + tid;
    const bool in = p < M;
    // the copies of stage st into buffer st % kTcBuf, as one commit group
    auto issue = [&](int st) {
        const uint32_t a_s = sb + (st % kTcBuf) * stage_bytes, b_s = a_s + a_bytes;
        const int tap = st / nkb, kc0 = (st % nkb) * kTcK;
        const int kw = Ci - kc0 < kTcK ? Ci - kc0 : kTcK;
        const bf16* src = x + (in ? shift_pixel(p, H, W, tap / 3 - 1, tap % 3 - 1) : 0) * csx + kc0;
        for (int c = 0; c < kw / 8; ++c) cp_async16(a_s + c * (kTcM * 16) + tid * 16, src + c * 8, in ? 16u : 0u);
        for (int k = tid; k < Co * (kw / 8); k += kTcM) {
            const int co = k % Co, c = k / Co;
            cp_async16(b_s + c * (Co * 16) + co * 16, w + ((long long)co * 9 + tap) * Ci + kc0 + c * 8, 16u);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // stage s commits to barrier s % kTcBuf: its (s / kTcBuf)-th phase
    auto wait_stage = [&](int st) {
        return mbar_wait_bounded(bar0 + 8 * (st % kTcBuf), (uint32_t)(st / kTcBuf) & 1u, kTcPolls);
    };
    bool ok = true;
    int issued = 0;   // stages whose MMAs were issued and committed
    for (int st = 0; st < kTcAhead && st < nst; ++st) issue(st);
    for (int st = 0; st < nst; ++st) {
        // copies run kTcAhead stages ahead; buffer (st + kTcAhead) % kTcBuf was
        // last read by the MMAs of stage st + kTcAhead - kTcBuf
        const int nxt = st + kTcAhead;
        if (nxt < nst) {
            if (nxt >= kTcBuf && !__syncthreads_and(wait_stage(nxt - kTcBuf))) {
                ok = false;
                break;
            }
            issue(nxt);
        }
        // stage st's group is complete once at most the newer ones are pending
        const int newer = (nst - 1 < st + kTcAhead ? nst - 1 : st + kTcAhead) - st;
        if (newer >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
        else if (newer == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        // the copies were written through the generic proxy; the MMAs read through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_s = sb + (st % kTcBuf) * stage_bytes, b_s = a_s + a_bytes;
            const int kc0 = (st % nkb) * kTcK;
            const int kw = Ci - kc0 < kTcK ? Ci - kc0 : kTcK;
            for (int s = 0; s < kw / 16; ++s) {
                const uint64_t ad = tc_smem_desc(a_s + 2 * s * (kTcM * 16), kTcM * 16, 128);
                const uint64_t bd = tc_smem_desc(b_s + 2 * s * (Co * 16), Co * 16, 128);
                tc_mma(tmem, ad, bd, idesc, (st > 0 || s > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8 * (st % kTcBuf))
                         : "memory");
        }
        issued = st + 1;
    }
    // copies still in flight on the failure path land before the CTA leaves
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last committed stage completes after every earlier MMA of the CTA
    // (waited for on the failure path too, before the tensor memory is freed)
    if (issued > 0) {
        const bool done = wait_stage(issued - 1);
        ok = __syncthreads_and(ok && done) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const long long pr = p0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        const bool vec = (csy & 3) == 0 && ((uintptr_t)y & 15) == 0;
        for (int c0 = 0; c0 < Co; c0 += 16) {
            float v[16];
            tc_ld16(trow + (uint32_t)c0, v);
            if (pr < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += bias ? bias[c0 + i] : 0.0f;
                float* out = y + pr * csy + c0;
                if (vec) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4*>(out + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) out[i] = v[i];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (!ok && tid == 0) atomicExch(err, 1);
}

// kTcBuf stage buffers of A (128 pixels) and B (Co weight rows), min(Ci, kTcK) channels each
size_t conv_tc_smem_bytes(int Ci, int Co) {
    const size_t k = Ci < kTcK ? (size_t)Ci : (size_t)kTcK;
    return (size_t)kTcBuf * (kTcM + (size_t)Co) * k * 2;
}

__device__ int g_sg_err;   // a bounded wait of a surrogate kernel gave up

// ---------------------------------------------------------------- tcgen05 convolution, row march
// The same convolution for images whose width is a multiple of 128: a CTA
// owns a 128-pixel segment of one image row and marches down a chunk of
// rows.  The shifted activations of a 3x3 tap are then rows of a halo
// strip: for row r the taps read input rows r - 1, r, r + 1 at pixel
// offsets -1, 0, +1 around the segment.  The strip holds four input rows
// (130 pixels each, the periodic neighbours included) in the tensor core's
// no-swizzle K-major layout, one 16-byte row per (pixel, 8 channels): a tap's
// A operand is the strip row of its dy started (1 + dx) pixels in, 128 rows
// of 16 bytes, 8-row core matrices 128 bytes apart, 8-channel planes 130 x 16
// bytes apart.  Every input row is copied into shared memory once (the tap
// kernel above copies it nine times), the weights of all nine taps stay
// resident for the whole march, and one thread issues the 9 x Ci/16 MMAs of
// a row into one of two tensor-memory accumulators while the CTA writes out
// the previous row from the other and the copy of the next input row is in
// flight.  Every wait is bounded, as in the tap kernel.
constexpr int kRowM = 128;          // pixels of a row segment (MMA M)
constexpr int kRowHalo = kRowM + 2;
constexpr int kRowSlots = 4;        // input rows resident in the strip

__host__ __device__ constexpr uint32_t row_plane_bytes() { return kRowHalo * 16; }
__host__ __device__ inline uint32_t row_slot_bytes(int Ci) { return (uint32_t)(Ci / 8) * row_plane_bytes(); }
__host__ __device__ inline uint32_t row_w_bytes(int Ci, int Co) { return (uint32_t)9 * Co * Ci * 2; }
size_t conv_row_smem_bytes(int Ci, int Co) {
    return (size_t)kRowSlots * row_slot_bytes(Ci) + row_w_bytes(Ci, Co);
}
// tensor-memory columns of the two accumulators (a power of two, at least 32)
__host__ __device__ inline uint32_t row_tmem_cols(int Co) {
    const int need = 2 * Co;
    return need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : 256u));
}

__global__ void __launch_bounds__(128, 1)
conv_row_kernel(const bf16* __restrict__ x, int csx, const bf16* __restrict__ w, const float* __restrict__ bias,
                float* __restrict__ y, int csy, int N, int H, int W, int Ci, int Co, int rows_per_cta, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = W / kRowM;
    const int chunks = (H + rows_per_cta - 1) / rows_per_cta;
    int b = blockIdx.x;
    const int chunk = b % chunks;
    b /= chunks;
    const int seg = b % segs, n = b / segs;
    const int y0 = chunk * rows_per_cta;
    const int y1 = y0 + rows_per_cta < H ? y0 + rows_per_cta : H;
    const int x0 = seg * kRowM;
    const uint32_t sb = smem_u32(smem);
    const uint32_t slot_bytes = row_slot_bytes(Ci);
    const uint32_t wb = sb + kRowSlots * slot_bytes;     // weights: [tap][ci chunk][co][16 bytes]
    const uint32_t bar0 = smem_u32(&bars[0]);
    const uint32_t ncols = row_tmem_cols(Co);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * k) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc_idesc_bf16(kRowM, Co);
    const int nch = Ci / 8;
    const long long img = (long long)n * H * W;
    // input row yy (wrapped) into strip slot yy & 3: pixels x0 - 1 .. x0 + 128 (wrapped)
    auto copy_row = [&](int yy) {
        const int yr = ((yy % H) + H) % H;
        const uint32_t dst = sb + (uint32_t)(yy & 3) * slot_bytes;
        const bf16* row = x + (img + (long long)yr * W) * csx;
        for (int k = tid; k < nch * kRowHalo; k += kRowM) {
            const int c = k / kRowHalo, px = k - c * kRowHalo;
            int xx = x0 - 1 + px;
            xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
            cp_async16(dst + c * row_plane_bytes() + px * 16, row + (long long)xx * csx + c * 8, 16u);
        }
    };
    // prologue: the weights of every tap and input rows y0 - 1 .. y0 + 1, one group
    for (int k = tid; k < 9 * nch * Co; k += kRowM) {
        const int co = k % Co, rest = k / Co, c = rest % nch, tap = rest / nch;
        cp_async16(wb + ((uint32_t)(tap * nch + c) * Co + co) * 16, w + ((long long)co * 9 + tap) * Ci + c * 8, 16u);
    }
    for (int yy = y0 - 1; yy <= y0 + 1; ++yy) copy_row(yy);
    asm volatile("cp.async.commit_group;" ::: "memory");
    bool ok = true;
    // row j of the march (row y0 + j) accumulates in buffer j & 1 and commits
    // to barrier j & 1: the (j >> 1)-th phase of that barrier
    auto wait_row = [&](int j) { return mbar_wait_bounded(bar0 + 8 * (j & 1), (uint32_t)(j >> 1) & 1u, kTcPolls); };
    auto epilogue = [&](int j) {
        const int r = y0 + j;
        const uint32_t acc = tmem + (uint32_t)((j & 1) * Co) + ((uint32_t)(32 * warp) << 16);
        const long long pix = img + (long long)r * W + x0 + 32 * warp + lane;
        float* out = y + pix * csy;
        const bool vec = (csy & 3) == 0 && ((uintptr_t)y & 15) == 0;
        for (int c0 = 0; c0 < Co; c0 += 16) {
            float v[16];
            tc_ld16(acc + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += bias ? bias[c0 + i] : 0.0f;
            if (vec) {
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(out + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) out[c0 + i] = v[i];
            }
        }
    };
    const int nrows = y1 - y0;
    int issued = 0;   // rows whose MMAs were issued and committed
    for (int j = 0; j < nrows && ok; ++j) {
        const int r = y0 + j;
        // (1) row j - 1: its MMAs done (they read strip slot (r - 2) & 3 last),
        // its accumulator out
        if (j > 0) {
            if (!__syncthreads_and(wait_row(j - 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(j - 1);
        }
        // (2) input row r + 2 into the slot row r - 2 held
        const bool more = r + 2 <= y1;
        if (more) {
            copy_row(r + 2);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        // (3) rows r - 1 .. r + 1 landed (only the group just issued may be pending)
        if (more) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // (4) the 9 x Ci/16 MMAs of row r into buffer j & 1
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)((j & 1) * Co);
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                const uint32_t a_s = sb + (uint32_t)((r + dy) & 3) * slot_bytes + (uint32_t)(1 + dx) * 16;
                const uint32_t b_s = wb + (uint32_t)tap * nch * Co * 16;
                for (int s2 = 0; s2 < Ci / 16; ++s2) {
                    const uint64_t ad = tc_smem_desc(a_s + 2 * s2 * row_plane_bytes(), row_plane_bytes(), 128);
                    const uint64_t bd = tc_smem_desc(b_s + 2 * s2 * (Co * 16), Co * 16, 128);
                    tc_mma(acc, ad, bd, idesc, (tap > 0 || s2 > 0) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8 * (j & 1))
                         : "memory");
        }
        issued = j + 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last issued row: its MMAs complete after every earlier one (waited
    // for on the failure path too, before the tensor memory is freed)
    if (issued > 0) {
        const bool done = wait_row(issued - 1);
        const bool all = __syncthreads_and(ok && done) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (all && issued == nrows) epilogue(issued - 1);
        ok = all && ok;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (!ok && tid == 0) atomicExch(err, 1);
}

// partial[chunk, co, tap, ci] = sum over the chunk's pixels p of gy[p, co] x[shift(p, tap), ci];
// one warp per (chunk, tap, 16 output channels, 8 input channels).
constexpr int kChunk = 1024;   // pixels per partial

__global__ void conv_wgrad_kernel(const bf16* __restrict__ x, int csx, const bf16* __restrict__ gy, int csg,
                                  float* __restrict__ partial, long long M, int H, int W, int Ci, int Co) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nco = Co / 16, nci = Ci / 8;
    const long long per_chunk = 9LL * nco * nci;
    const long long nchunks = (M + kChunk - 1) / kChunk;
    if (warp >= nchunks * per_chunk) return;
    const long long chunk = warp / per_chunk;
    int rem = (int)(warp - chunk * per_chunk);
    const int tap = rem / (nco * nci);
    rem -= tap * nco * nci;
    const int co0 = (rem / nci) * 16, ci0 = (rem % nci) * 8;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const long long pb = chunk * kChunk;
    const long long pe = pb + kChunk < M ? pb + kChunk : M;
    for (long long pk = pb; pk < pe; pk += 16) {
        // k index = pixel pk + kk; pixel counts are multiples of 16, so no tail
        const long long q0 = pk + 2 * t, q1 = q0 + 1, q8 = q0 + 8, q9 = q0 + 9;
        const uint32_t a[4] = {pack_pair(gy + q0 * csg + co0 + g, gy + q1 * csg + co0 + g),
                               pack_pair(gy + q0 * csg + co0 + g + 8, gy + q1 * csg + co0 + g + 8),
                               pack_pair(gy + q8 * csg + co0 + g, gy + q9 * csg + co0 + g),
                               pack_pair(gy + q8 * csg + co0 + g + 8, gy + q9 * csg + co0 + g + 8)};
        const uint32_t b[2] = {pack_pair(x + shift_pixel(q0, H, W, dy, dx) * csx + ci0 + g,
                                         x + shift_pixel(q1, H, W, dy, dx) * csx + ci0 + g),
                               pack_pair(x + shift_pixel(q8, H, W, dy, dx) * csx + ci0 + g,
                                         x + shift_pixel(q9, H, W, dy, dx) * csx + ci0 + g)};
        mma_bf16(acc, a, b);
    }
    float* out = partial + chunk * (long long)Co * 9 * Ci;
    const int ci = ci0 + 2 * t;
    out[((long long)(co0 + g) * 9 + tap) * Ci + ci] = acc[0];
    out[((long long)(co0 + g) * 9 + tap) * Ci + ci + 1] = acc[1];
    out[((long long)(co0 + g + 8) * 9 + tap) * Ci + ci] = acc[2];
    out[((long long)(co0 + g + 8) * 9 + tap) * Ci + ci + 1] = acc[3];
}

// ---------------------------------------------------------------- tcgen05 weight gradient, row march
// gw[co, tap, ci] = sum_p gy[p, co] x[p + d(tap), ci] as GEMMs over pixels
// on the tensor cores, for images whose width is a multiple of 32: for each
// tap D_tap (M = co, N = ci) += A (co x pixels) B_tap (ci x pixels)^T with K
// running over pixels.  A CTA owns a segment of P = 64 (or 32) pixels of one
// image row, one tap row dy, a block of at most 128 input channels and a
// chunk of rows; per row (one stage) it copies the gy row segment and the x
// row r + dy (P + 2 pixels, the periodic neighbours included)
// into shared memory in their natural channels-last order (16-byte
// cp.async, one stage ahead), then transposes them with ldmatrix /
// stmatrix.trans into the K-major core-matrix layout the MMAs read: A as
// 128 co rows (rows past Co are never written and their D rows never read),
// B once per dx in {-1, 0, +1}, the window shifted by dx pixels.  The three
// taps of the CTA's dy accumulate in tensor memory over the whole march
// (columns dx Ci + ci, lanes co) and are written out once, as the CTA's
// partial; the partials are summed in a fixed order (deterministic).
constexpr int kWgCn = 128;            // input channels of one CTA at most (3 Cn tensor-memory columns)
constexpr size_t kWgSmemMax = 220 * 1024;   // below the 227 KB per CTA less the kernel's static shared memory

struct WgLayout {
    uint32_t gys, xs;                 // natural row strides (padded by 16 bytes against bank conflicts)
    uint32_t nat_gy, nat;             // bytes of the gy part and of one natural buffer
    uint32_t opA, opB1, op;           // bytes of A, of one B window, of one operand buffer
    uint32_t total;
};
// P pixels of a segment, Cn input channels and Co output channels of a CTA
__host__ __device__ inline WgLayout wg_layout(int P, int Cn, int Co) {
    WgLayout L;
    L.gys = (uint32_t)Co * 2 + 16;
    L.xs = (uint32_t)Cn * 2 + 16;
    L.nat_gy = (uint32_t)P * L.gys;
    L.nat = L.nat_gy + (uint32_t)(P + 2) * L.xs;
    L.opA = (uint32_t)(P / 8) * 128 * 16;
    L.opB1 = (uint32_t)(P / 8) * (uint32_t)Cn * 16;
    L.op = L.opA + 3 * L.opB1;
    L.total = 2 * L.nat + 2 * L.op;
    return L;
}
__host__ __device__ inline uint32_t wg_tmem_cols(int Ci) {
    const int need = 3 * Ci;
    return need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void stsm_x2_trans(uint32_t addr, uint32_t r0, uint32_t r1) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(addr), "r"(r0), "r"(r1)
                 : "memory");
}

__global__ void __launch_bounds__(128, 1)
conv_wgrad_row_kernel(const bf16* __restrict__ x, int csx, const bf16* __restrict__ gy, int csg,
                      float* __restrict__ partial, int N, int H, int W, int Ci, int Co, int P, int Cn,
                      int rows_per_cta, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = W / P;
    const int nsplit = Ci / Cn;
    const int chunks = (H + rows_per_cta - 1) / rows_per_cta;
    int b = blockIdx.x;
    const int dyi = b % 3;
    b /= 3;
    const int ci0 = (b % nsplit) * Cn;
    b /= nsplit;
    const int chunk = b % chunks;
    b /= chunks;
    const int seg = b % segs, n = b / segs;
    const int dy = dyi - 1;
    const int y0 = chunk * rows_per_cta;
    const int y1 = y0 + rows_per_cta < H ? y0 + rows_per_cta : H;
    const int x0 = seg * P;
    const long long pchunk = ((long long)n * segs + seg) * chunks + chunk;
    const WgLayout Lt = wg_layout(P, Cn, Co);
    const uint32_t sb = smem_u32(smem);
    const uint32_t nat0 = sb, op0 = sb + 2 * Lt.nat;
    const uint32_t bar0 = smem_u32(&bars[0]);
    const uint32_t ncols = wg_tmem_cols(Cn);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * k) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc_idesc_bf16(128, Cn);
    const int nco8 = Co / 8, nci8 = Cn / 8;
    const long long img = (long long)n * H * W;
    // natural copies of stage s (row r = y0 + s): the gy row segment and
    // channels ci0 .. ci0 + Cn - 1 of the x row r + dy, pixels x0 - 1 .. x0 + P
    // (wrapped)
    auto copy_stage = [&](int st) {
        const int r = y0 + st;
        const uint32_t nb = nat0 + (uint32_t)(st & 1) * Lt.nat;
        const bf16* grow = gy + (img + (long long)r * W) * csg;
        for (int k = tid; k < P * nco8; k += 128) {
            const int p = k / nco8, c = k - p * nco8;
            cp_async16(nb + p * Lt.gys + c * 16, grow + (long long)(x0 + p) * csg + c * 8, 16u);
        }
        const int yr = (((r + dy) % H) + H) % H;
        const bf16* xrow = x + (img + (long long)yr * W) * csx + ci0;
        for (int k = tid; k < (P + 2) * nci8; k += 128) {
            const int q = k / nci8, c = k - q * nci8;
            int xx = x0 - 1 + q;
            xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
            cp_async16(nb + Lt.nat_gy + q * Lt.xs + c * 16, xrow + (long long)xx * csx + c * 8, 16u);
        }
    };
    // natural buffer st & 1 -> operand buffer st & 1 (K-major: [pixel block][row][8 pixels])
    auto transpose_stage = [&](int st) {
        const uint32_t nb = nat0 + (uint32_t)(st & 1) * Lt.nat;
        const uint32_t ob = op0 + (uint32_t)(st & 1) * Lt.op;
        const int j = (lane >> 3) & 1, i = lane & 7;   // matrix and row a lane addresses (lanes 0-15 count)
        const int npb = P / 8;
        const int na = npb * (nco8 / 2);
        for (int o = warp; o < na; o += 4) {
            const int pb = o % npb, cp = o / npb, c = 2 * cp + j;
            uint32_t r0, r1;
            ldsm_x2(nb + (uint32_t)(8 * pb + i) * Lt.gys + c * 16, r0, r1);
            stsm_x2_trans(ob + (uint32_t)pb * (128 * 16) + (uint32_t)(8 * c + i) * 16, r0, r1);
        }
        const int nbx = 3 * npb * (nci8 / 2);
        for (int o = warp; o < nbx; o += 4) {
            const int w3 = o % 3, rest = o / 3, pb = rest % npb, cp = rest / npb, c = 2 * cp + j;
            const int q = 8 * pb + i + w3;   // staging pixel of window pixel 8 pb + i shifted by dx = w3 - 1
            uint32_t r0, r1;
            ldsm_x2(nb + Lt.nat_gy + (uint32_t)q * Lt.xs + c * 16, r0, r1);
            stsm_x2_trans(ob + Lt.opA + (uint32_t)w3 * Lt.opB1 + (uint32_t)pb * Cn * 16 + (uint32_t)(8 * c + i) * 16, r0,
                          r1);
        }
    };
    auto wait_stage = [&](int st) { return mbar_wait_bounded(bar0 + 8 * (st & 1), (uint32_t)(st >> 1) & 1u, kTcPolls); };
    const int S = y1 - y0;
    bool ok = true;
    int issued = 0;
    copy_stage(0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int st = 0; st < S; ++st) {
        const bool more = st + 1 < S;
        if (more) {   // natural buffer (st + 1) & 1 was last read by the transposes of stage st - 1
            copy_stage(st + 1);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        if (more) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        // operand buffer st & 1 was last read by the MMAs of stage st - 2
        if (st >= 2 && !__syncthreads_and(wait_stage(st - 2))) { ok = false; break; }
        transpose_stage(st);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ob = op0 + (uint32_t)(st & 1) * Lt.op;
            for (int w3 = 0; w3 < 3; ++w3) {
                for (int k = 0; k < P / 16; ++k) {
                    const uint64_t ad = tc_smem_desc(ob + 2 * k * (128 * 16), 128 * 16, 128);
                    const uint64_t bd = tc_smem_desc(ob + Lt.opA + w3 * Lt.opB1 + 2 * k * (Cn * 16), Cn * 16, 128);
                    tc_mma(tmem + (uint32_t)(w3 * Cn), ad, bd, idesc, (st > 0 || k > 0) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8 * (st & 1))
                         : "memory");
        }
        issued = st + 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (issued > 0) {
        const bool done = wait_stage(issued - 1);
        ok = __syncthreads_and(ok && done) != 0 && issued == S;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int co = 32 * warp + lane;
        for (int w3 = 0; w3 < 3; ++w3) {
            const int tap = (dy + 1) * 3 + w3;
            float* out = partial + ((pchunk * Co + co) * 9 + tap) * (long long)Ci + ci0;
            for (int c0 = 0; c0 < Cn; c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(w3 * Cn + c0), v);
                if (co < Co) {
#pragma unroll
                    for (int k = 0; k < 16; k += 4)
                        *reinterpret_cast<float4*>(out + c0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (!ok && tid == 0) atomicExch(err, 1);
}

// gw[k] = sum over chunks of partial[chunk, k], in chunk order
__global__ void sum_chunks_kernel(const float* __restrict__ partial, long long nchunks, long long K,
                                  float* __restrict__ gw) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float s = 0.0f;
    for (long long c = 0; c < nchunks; ++c) s += partial[c * K + k];
    gw[k] = s;
}

// wt[ci, 8 - tap, co] = w[co, tap, ci]: the weights of the input-gradient convolution
__global__ void weight_flip_kernel(const bf16* __restrict__ w, bf16* __restrict__ wt, int Ci, int Co) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)Co * 9 * Ci) return;
    const int ci = (int)(k % Ci);
    const int tap = (int)((k / Ci) % 9);
    const int co = (int)(k / (9LL * Ci));
    wt[((long long)ci * 9 + (8 - tap)) * Co + co] = w[k];
}

}  // namespace

namespace {

constexpr int kThreads = 256;
inline unsigned blocks(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// y (bf16) = max(a, 0), channel slices
__global__ void relu_kernel(const float* __restrict__ a, int csa, bf16* __restrict__ y, int csy, long long npix,
                            int C) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix * C) return;
    const long long p = k / C;
    const int c = (int)(k - p * C);
    y[p * csy + c] = __float2bfloat16_rn(fmaxf(a[p * csa + c], 0.0f));
}

// ga = g where a > 0 else 0 (FP32), and its bf16 copy (optional)
__global__ void relu_bwd_kernel(const float* __restrict__ g, int csg, const float* __restrict__ a, int csa,
                                float* __restrict__ ga, bf16* __restrict__ ga16, long long npix, int C) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix * C) return;
    const long long p = k / C;
    const int c = (int)(k - p * C);
    const float v = a[p * csa + c] > 0.0f ? g[p * csg + c] : 0.0f;
    ga[k] = v;
    if (ga16) ga16[k] = __float2bfloat16_rn(v);
}

__global__ void to_bf16_kernel(const float* __restrict__ a, int csa, bf16* __restrict__ y, int csy, long long npix,
                               int C) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix * C) return;
    const long long p = k / C;
    const int c = (int)(k - p * C);
    y[p * csy + c] = __float2bfloat16_rn(a[p * csa + c]);
}

// out = a + b on channel slices
__global__ void add_kernel(const float* __restrict__ a, int csa, const float* __restrict__ b, int csb,
                           float* __restrict__ out, int cso, long long npix, int C) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix * C) return;
    const long long p = k / C;
    const int c = (int)(k - p * C);
    out[p * cso + c] = a[p * csa + c] + b[p * csb + c];
}

// f x f average pooling, bf16 -> bf16; (N, H, W) the fine grid
__global__ void pool_kernel(const bf16* __restrict__ x, int csx, bf16* __restrict__ y, int csy, int N, int H, int W,
                            int C, int f) {
    const int Hc = H / f, Wc = W / f;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)N * Hc * Wc * C) return;
    const int c = (int)(k % C);
    const long long q = k / C;
    const int xc = (int)(q % Wc), yc = (int)((q / Wc) % Hc);
    const long long n = q / ((long long)Hc * Wc);
    float s = 0.0f;
    for (int i = 0; i < f; ++i)
        for (int j = 0; j < f; ++j) {
            const long long p = (n * H + yc * f + i) * W + xc * f + j;
            s += __bfloat162float(x[p * csx + c]);
        }
    y[q * csy + c] = __float2bfloat16_rn(s / (float)(f * f));
}

// gx[fine] = g[coarse] / f^2
__global__ void pool_bwd_kernel(const float* __restrict__ g, int csg, float* __restrict__ gx, int csx, int N, int H,
                                int W, int C, int f) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)N * H * W * C) return;
    const int c = (int)(k % C);
    const long long p = k / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long long n = p / ((long long)H * W);
    const int Hc = H / f, Wc = W / f;
    const long long q = (n * Hc + y / f) * Wc + x / f;
    gx[p * csx + c] = g[q * csg + c] / (float)(f * f);
}

// nearest upsampling by f, bf16 -> bf16; (N, H, W) the fine grid
__global__ void upsample_kernel(const bf16* __restrict__ x, int csx, bf16* __restrict__ y, int csy, int N, int H,
                                int W, int C, int f) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)N * H * W * C) return;
    const int c = (int)(k % C);
    const long long p = k / C;
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const long long n = p / ((long long)H * W);
    const int Hc = H / f, Wc = W / f;
    const long long q = (n * Hc + yy / f) * Wc + xx / f;
    y[p * csy + c] = x[q * csx + c];
}

// gx[coarse] = sum of g over the f x f block
__global__ void upsample_bwd_kernel(const float* __restrict__ g, int csg, float* __restrict__ gx, int csx, int N,
                                    int H, int W, int C, int f) {
    const int Hc = H / f, Wc = W / f;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)N * Hc * Wc * C) return;
    const int c = (int)(k % C);
    const long long q = k / C;
    const int xc = (int)(q % Wc), yc = (int)((q / Wc) % Hc);
    const long long n = q / ((long long)Hc * Wc);
    float s = 0.0f;
    for (int i = 0; i < f; ++i)
        for (int j = 0; j < f; ++j) {
            const long long p = (n * H + yc * f + i) * W + xc * f + j;
            s += g[p * csg + c];
        }
    gx[q * csx + c] = s;
}

// per-block partial sums of column c of g (rows = pixels), fixed order
__global__ void colsum_partial_kernel(const float* __restrict__ g, int csg, long long npix, int C,
                                      float* __restrict__ part) {
    __shared__ float sh[kThreads];
    const int c = blockIdx.y;
    float s = 0.0f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x)
        s += g[p * csg + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)c * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void colsum_finish_kernel(const float* __restrict__ part, int nb, int C, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) s += part[(long long)c * nb + b];
    out[c] = s;
}

// out = x + delta on the first C channels; g = 2 (out - t) / (npix C) (zero beyond C up to csd);
// block partials of sum (out - t)^2 in FP64
__global__ void mse_kernel(const float* __restrict__ x, int csx, const float* __restrict__ delta, int csd,
                           const float* __restrict__ t, int cst, float* __restrict__ g, long long npix, int C,
                           double* __restrict__ part) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    const double inv = 1.0 / ((double)npix * C);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npix * csd;
         k += (long long)gridDim.x * blockDim.x) {
        const long long p = k / csd;
        const int c = (int)(k - p * csd);
        float gv = 0.0f;
        if (c < C) {
            const double e = (double)x[p * csx + c] + (double)delta[k] - (double)t[p * cst + c];
            s += e * e;
            gv = (float)(2.0 * e * inv);
        }
        g[k] = gv;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void mse_finish_kernel(const double* __restrict__ part, int nb, double inv_count, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    out[0] = s * inv_count;
}

// Adam on FP32 master values, with the bf16 copy used by the convolutions
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2, bf16* __restrict__ w16) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    w[k] = wk;
    if (w16) w16[k] = __float2bfloat16_rn(wk);
}

// LB fields (FP64, x fastest: phi, rho u_x, rho u_y, P) -> normalised channels-last input: channel c = field c / scale c
__global__ void pack_kernel(const double* __restrict__ f0, const double* __restrict__ f1, const double* __restrict__ f2,
                            const double* __restrict__ f3, double s0, double s1, double s2, double s3,
                            float* __restrict__ x32, int cs32, bf16* __restrict__ x16, int cs16, long long npix) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const float v[4] = {(float)(f0[p] / s0), (float)(f1[p] / s1), (float)(f2[p] / s2), (float)(f3[p] / s3)};
    for (int c = 0; c < 4; ++c) x32[p * cs32 + c] = v[c];
    for (int c = 0; c < cs16; ++c) x16[p * cs16 + c] = __float2bfloat16_rn(c < 4 ? v[c] : 0.0f);
}

// (phi, rho u_x, rho u_y, P) = (x + delta) * scale, then u = rho u / rho(phi)
// with phi clipped to [0, 1] inside rho only (a predicted phi a little below
// 0 in the light phase must not make the density vanish or turn negative)
__global__ void unpack_kernel(const float* __restrict__ x32, int cs32, const float* __restrict__ delta, int csd,
                              double* __restrict__ f0, double* __restrict__ f1, double* __restrict__ f2,
                              double* __restrict__ f3, double s0, double s1, double s2, double s3, double rho_L,
                              double rho_dif, const double* __restrict__ phi_rho, long long npix) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double v[4];
    const double s[4] = {s0, s1, s2, s3};
    for (int c = 0; c < 4; ++c) v[c] = ((double)x32[p * cs32 + c] + (double)delta[p * csd + c]) * s[c];
    const double pr = phi_rho ? phi_rho[p] : v[0];
    const double pc = pr < 0.0 ? 0.0 : (pr > 1.0 ? 1.0 : pr);
    const double rho = rho_L + pc * rho_dif;
    f0[p] = v[0];
    f1[p] = v[1] / rho;
    f2[p] = v[2] / rho;
    f3[p] = v[3];
}

__global__ void shift_kernel(double* __restrict__ a, long long n, double s) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) a[k] += s;
}

// block partials of sum (a - b)^2 and sum a^2 (FP64, fixed order)
__global__ void residual_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                        double* __restrict__ part) {
    __shared__ double s0[kThreads], s1[kThreads];
    double d2 = 0.0, a2 = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double d = a[k] - b[k];
        d2 += d * d;
        a2 += a[k] * a[k];
    }
    s0[threadIdx.x] = d2;
    s1[threadIdx.x] = a2;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s0[0]; part[2 * blockIdx.x + 1] = s1[0]; }
}

__global__ void residual_finish_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d2 = 0.0, a2 = 0.0;
    for (int k = 0; k < nb; ++k) { d2 += part[2 * k]; a2 += part[2 * k + 1]; }
    out[0] = d2;
    out[1] = a2;
}

// block partials of (sum P, count) over the bulk heavy phase (phi >= 1 - d)
// and over the bulk light phase (phi <= d), FP64, fixed order
__global__ void phase_pressure_partial_kernel(const double* __restrict__ phi, const double* __restrict__ P,
                                              long long n, double d, double* __restrict__ part) {
    __shared__ double sh[4][kThreads];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double f = phi[k];
        if (f >= 1.0 - d) { a[0] += P[k]; a[1] += 1.0; }
        if (f <= d) { a[2] += P[k]; a[3] += 1.0; }
    }
    for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = a[j];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int j = 0; j < 4; ++j) part[4 * blockIdx.x + j] = sh[j][0];
}

__global__ void phase_pressure_finish_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b)
        for (int j = 0; j < 4; ++j) a[j] += part[4 * b + j];
    out[0] = a[1] > 0.0 ? a[0] / a[1] : 0.0;
    out[1] = a[3] > 0.0 ? a[2] / a[3] : 0.0;
    out[2] = a[1];
    out[3] = a[3];
}

// phi <- clip(phi0 + m (phi - phi0), 0, 1), m = 4 phi0 (1 - phi0): the
// predicted change of phi kept inside the interface band of the start and
// none in the bulk phases; block partials of sum phi0, sum phi, sum 4 phi (1 - phi)
__global__ void phi_project_kernel(double* __restrict__ phi, const double* __restrict__ phi0, long long n,
                                   double* __restrict__ part) {
    __shared__ double s0[kThreads], s1[kThreads], s2[kThreads];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double f0 = phi0[k];
        const double m = 4.0 * f0 * (1.0 - f0);
        double f = f0 + (m > 0.0 ? m : 0.0) * (phi[k] - f0);
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        phi[k] = f;
        a0 += f0;
        a1 += f;
        a2 += 4.0 * f * (1.0 - f);
    }
    s0[threadIdx.x] = a0;
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] += s0[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s0[0];
        part[3 * blockIdx.x + 1] = s1[0];
        part[3 * blockIdx.x + 2] = s2[0];
    }
}

// c = (sum phi0 - sum phi) / sum 4 phi (1 - phi), partials in block order, into part[3 nb]
__global__ void phi_project_finish_kernel(double* __restrict__ part, int nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int b = 0; b < nb; ++b) {
        a0 += part[3 * b];
        a1 += part[3 * b + 1];
        a2 += part[3 * b + 2];
    }
    part[3 * nb] = a2 > 0.0 ? (a0 - a1) / a2 : 0.0;
}

// phi += c 4 phi (1 - phi): the total of phi0 restored by moving the interfaces
__global__ void phi_restore_kernel(double* __restrict__ phi, long long n, const double* __restrict__ c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double f = phi[k];
    phi[k] = f + c[0] * 4.0 * f * (1.0 - f);
}

// b = a + k lap(a), five-point Laplacian, periodic in each H x W image
__global__ void smooth_kernel(const double* __restrict__ a, double* __restrict__ b, int N, int H, int W, double k) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)N * H * W) return;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long long base = p - (long long)y * W - x;
    const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
    const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
    const double c = a[p];
    const double lap = a[base + (long long)y * W + xm] + a[base + (long long)y * W + xp] + a[base + (long long)ym * W + x] +
                       a[base + (long long)yp * W + x] - 4.0 * c;
    b[p] = c + k * lap;
}

constexpr size_t kRowSmemMax = 200 * 1024;

// Shared memory of one SM of the current device (looked up once per device;
// 228 KB, GB300's, if the query fails).
size_t sm_shared_bytes() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 228 * 1024;
    }
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 228 * 1024;
        }
        cached[dev] = v;
    }
    return (size_t)cached[dev];
}

// Dynamic shared memory of a row-march launch: its need, raised if necessary
// so that no more CTAs fit on an SM than its 512 tensor-memory columns serve
// at once (each CTA holds row_tmem_cols(Co) of them for its whole life).
size_t conv_row_launch_smem(size_t need, int Co) {
    const int per_sm = 512 / (int)row_tmem_cols(Co);
    const size_t floor_bytes = sm_shared_bytes() / (size_t)(per_sm + 1) + 1;
    return need > floor_bytes ? need : floor_bytes;
}

// Resident row-march CTAs on the current device (SMs x CTAs per SM), with the
// attribute for large dynamic shared memory set once per device.
cudaError_t conv_row_slots(size_t need, int Co, int* out) {
    static bool attr_set[64] = {};
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(conv_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmemMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_row_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_row_kernel, kRowM, conv_row_launch_smem(need, Co));
    if (e != cudaSuccess) return e;
    *out = sms * (occ > 0 ? occ : 1);
    return cudaSuccess;
}

// Dynamic shared memory of a weight-gradient row-march launch, raised like
// conv_row_launch_smem so that the CTAs an SM holds fit its tensor memory.
size_t wg_launch_smem(size_t need, int Ci) {
    const int per_sm = 512 / (int)wg_tmem_cols(Ci);
    const size_t floor_bytes = sm_shared_bytes() / (size_t)(per_sm + 1) + 1;
    return need > floor_bytes ? need : floor_bytes;
}

// Segment width of the weight-gradient row march (0: the width allows none)
// and the input channels of one CTA.
inline int wg_segment(int W) { return W % 64 == 0 ? 64 : (W % 32 == 0 ? 32 : 0); }
inline int wg_block(int Ci) { return Ci <= kWgCn ? Ci : kWgCn; }

// Row chunks of the weight-gradient row march on the current device: rows
// per CTA and chunks per column (0 rows: the march does not apply to these
// sizes).  One wave: 3 tap rows x channel blocks x N x W / P segments x
// chunks CTAs at most the resident CTAs.
cudaError_t wgrad_row_plan(int N, int H, int W, int Ci, int Co, int* rows, int* chunks) {
    *rows = 0;
    *chunks = 0;
    const int P = wg_segment(W), Cn = wg_block(Ci);
    if (P == 0 || Ci % Cn || Co > 128 || Ci % 16 || Co % 16 || H < 1) return cudaSuccess;
    const WgLayout Lt = wg_layout(P, Cn, Co);
    if (Lt.total > kWgSmemMax) return cudaSuccess;
    static bool attr_set[64] = {};
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(conv_wgrad_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmemMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_wgrad_row_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // CTAs an SM holds: its shared memory (1 KB reserved per CTA) and its 512
    // tensor-memory columns
    const size_t per_cta = wg_launch_smem(Lt.total, Cn) + 1024;
    occ = (int)(sm_shared_bytes() / per_cta);
    const int by_tmem = 512 / (int)wg_tmem_cols(Cn);
    if (occ > by_tmem) occ = by_tmem;
    const long long slots = (long long)sms * (occ > 0 ? occ : 1);
    const long long cols = 3LL * (Ci / Cn) * N * (W / P);
    long long c = slots / cols;
    if (c < 1) c = 1;
    if (c > H) c = H;
    const int r = (int)((H + c - 1) / c);
    *rows = r;
    *chunks = (H + r - 1) / r;
    return cudaSuccess;
}

bool conv_dims_ok(long long M, int Ci, int Co) { return M > 0 && M % 16 == 0 && Ci > 0 && Ci % 16 == 0 && Co > 0 && Co % 16 == 0; }

}  // namespace

extern "C" {

int lbm_sg_conv3x3(const void* x, int csx, const void* w, const float* bias, float* y, int csy, int N, int H, int W,
                   int Ci, int Co, void* stream) {
    const long long M = (long long)N * H * W;
    if (!x || !w || !y || N < 1 || H < 1 || W < 1 || !conv_dims_ok(M, Ci, Co) || csx < Ci || csx % 2 || csy < Co)
        return LBM_EINVAL;
    if (Co > 128) return LBM_EINVAL;
    // 16-byte copies: channel rows and slices start on 16-byte boundaries
    if (csx % 8 || ((uintptr_t)x & 15) || ((uintptr_t)w & 15)) return LBM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = conv_tc_smem_bytes(Ci, Co);
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)conv_tc_smem_bytes(kTcK, 128)) != cudaSuccess)
            return LBM_ECUDA;
        attr_set[dev] = true;
    }
    int* err = nullptr;
    if (cudaGetSymbolAddress((void**)&err, g_sg_err) != cudaSuccess) return LBM_ECUDA;
    // rows of 128-pixel segments: the row-march kernel, when its strip and
    // the weights of all taps fit in shared memory
    const size_t row_smem = conv_row_smem_bytes(Ci, Co);
    if (W % kRowM == 0 && H >= 2 && row_smem <= kRowSmemMax) {
        int slots = 0;
        if (conv_row_slots(row_smem, Co, &slots) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ECUDA;
        }
        int dev = 0, sms = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return LBM_ECUDA;
        const long long cols = (long long)N * (W / kRowM);
        // one CTA per SM: longer marches (the weights and the two halo rows of
        // a chunk are loaded once per CTA) ran faster than two CTAs per SM on
        // half the rows (d1 at 8 x 256^2: 0.127 against 0.135 ms)
        long long chunks = (slots < sms ? slots : sms) / cols;
        if (chunks < 1) chunks = 1;
        if (chunks > H) chunks = H;
        const int rows = (int)((H + chunks - 1) / chunks);
        const long long nb = cols * ((H + rows - 1) / rows);
        conv_row_kernel<<<(unsigned)nb, kRowM, conv_row_launch_smem(row_smem, Co), s>>>(
            (const bf16*)x, csx, (const bf16*)w, bias, y, csy, N, H, W, Ci, Co, rows, err);
        return check(cudaGetLastError());
    }
    const unsigned nb = (unsigned)((M + kTcM - 1) / kTcM);
    conv_tc_kernel<<<nb, kTcM, smem, s>>>((const bf16*)x, csx, (const bf16*)w, bias, y, csy, M, H, W, Ci, Co, err);
    return check(cudaGetLastError());
}

int lbm_sg_status(void* stream) {
    int* err = nullptr;
    if (cudaGetSymbolAddress((void**)&err, g_sg_err) != cudaSuccess) return LBM_ECUDA;
    int h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LBM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ECUDA;
    if (h) {
        const int zero = 0;
        if (cudaMemcpyAsync(err, &zero, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) return LBM_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ECUDA;
        return LBM_ETIMEOUT;
    }
    return LBM_OK;
}

long long lbm_sg_wgrad_scratch_floats(int N, int H, int W, int Ci, int Co) {
    const long long M = (long long)N * H * W;
    long long need = ((M + kChunk - 1) / kChunk) * (long long)Co * 9 * Ci;
    int rows = 0, chunks = 0;
    if (wgrad_row_plan(N, H, W, Ci, Co, &rows, &chunks) == cudaSuccess) {
        if (rows > 0) {
            const long long row_need = (long long)N * (W / wg_segment(W)) * chunks * Co * 9 * Ci;
            if (row_need > need) need = row_need;
        }
    } else {
        cudaGetLastError();   // the plan's failure is reported by lbm_sg_conv3x3_wgrad, not left pending
    }
    return need;
}

int lbm_sg_conv3x3_wgrad(const void* x, int csx, const void* gy, int csg, float* gw, float* scratch,
                         long long scratch_floats, int N, int H, int W, int Ci, int Co, void* stream) {
    const long long M = (long long)N * H * W;
    if (!x || !gy || !gw || !scratch || N < 1 || H < 1 || W < 1 || !conv_dims_ok(M, Ci, Co) || csx < Ci || csg < Co)
        return LBM_EINVAL;
    const long long need = lbm_sg_wgrad_scratch_floats(N, H, W, Ci, Co);
    if (scratch_floats < need) return LBM_EINVAL;
    // rows of 64-pixel segments with 16-byte aligned channel rows: the
    // tcgen05 row march
    int rows = 0, rchunks = 0;
    if (wgrad_row_plan(N, H, W, Ci, Co, &rows, &rchunks) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    if (rows > 0 && csx % 8 == 0 && csg % 8 == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)gy & 15) == 0 &&
        ((uintptr_t)scratch & 15) == 0) {
        int* err = nullptr;
        if (cudaGetSymbolAddress((void**)&err, g_sg_err) != cudaSuccess) return LBM_ECUDA;
        cudaStream_t s = (cudaStream_t)stream;
        const int P = wg_segment(W), Cn = wg_block(Ci);
        const long long pchunks = (long long)N * (W / P) * rchunks;
        const WgLayout Lt = wg_layout(P, Cn, Co);
        conv_wgrad_row_kernel<<<(unsigned)(3 * (Ci / Cn) * pchunks), 128, wg_launch_smem(Lt.total, Cn), s>>>(
            (const bf16*)x, csx, (const bf16*)gy, csg, scratch, N, H, W, Ci, Co, P, Cn, rows, err);
        const long long K = (long long)Co * 9 * Ci;
        sum_chunks_kernel<<<blocks(K), kThreads, 0, s>>>(scratch, pchunks, K, gw);
        return check(cudaGetLastError());
    }
    const long long nchunks = (M + kChunk - 1) / kChunk;
    const long long warps = nchunks * 9LL * (Co / 16) * (Ci / 8);
    cudaStream_t s = (cudaStream_t)stream;
    conv_wgrad_kernel<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, s>>>((const bf16*)x, csx, (const bf16*)gy, csg,
                                                                          scratch, M, H, W, Ci, Co);
    const long long K = (long long)Co * 9 * Ci;
    sum_chunks_kernel<<<blocks(K), kThreads, 0, s>>>(scratch, nchunks, K, gw);
    return check(cudaGetLastError());
}

int lbm_sg_weight_flip(const void* w, void* wt, int Ci, int Co, void* stream) {
    if (!w || !wt || Ci < 1 || Co < 1) return LBM_EINVAL;
    weight_flip_kernel<<<blocks((long long)Co * 9 * Ci), kThreads, 0, (cudaStream_t)stream>>>((const bf16*)w, (bf16*)wt,
                                                                                              Ci, Co);
    return check(cudaGetLastError());
}

int lbm_sg_bias_grad(const float* g, int csg, float* gb, float* scratch, long long npix, int C, void* stream) {
    if (!g || !gb || !scratch || npix < 1 || C < 1 || csg < C) return LBM_EINVAL;
    const int nb = (int)(npix < 64LL * kThreads ? (npix + kThreads - 1) / kThreads : 64);
    cudaStream_t s = (cudaStream_t)stream;
    colsum_partial_kernel<<<dim3(nb, C), kThreads, 0, s>>>(g, csg, npix, C, scratch);
    colsum_finish_kernel<<<blocks(C), kThreads, 0, s>>>(scratch, nb, C, gb);
    return check(cudaGetLastError());
}

int lbm_sg_relu(const float* a, int csa, void* y, int csy, long long npix, int C, void* stream) {
    if (!a || !y || npix < 1 || C < 1 || csa < C || csy < C) return LBM_EINVAL;
    relu_kernel<<<blocks(npix * C), kThreads, 0, (cudaStream_t)stream>>>(a, csa, (bf16*)y, csy, npix, C);
    return check(cudaGetLastError());
}

int lbm_sg_relu_bwd(const float* g, int csg, const float* a, int csa, float* ga, void* ga16, long long npix, int C,
                    void* stream) {
    if (!g || !a || !ga || npix < 1 || C < 1 || csg < C || csa < C) return LBM_EINVAL;
    relu_bwd_kernel<<<blocks(npix * C), kThreads, 0, (cudaStream_t)stream>>>(g, csg, a, csa, ga, (bf16*)ga16, npix, C);
    return check(cudaGetLastError());
}

int lbm_sg_to_bf16(const float* a, int csa, void* y, int csy, long long npix, int C, void* stream) {
    if (!a || !y || npix < 1 || C < 1 || csa < C || csy < C) return LBM_EINVAL;
    to_bf16_kernel<<<blocks(npix * C), kThreads, 0, (cudaStream_t)stream>>>(a, csa, (bf16*)y, csy, npix, C);
    return check(cudaGetLastError());
}

int lbm_sg_add(const float* a, int csa, const float* b, int csb, float* out, int cso, long long npix, int C,
               void* stream) {
    if (!a || !b || !out || npix < 1 || C < 1 || csa < C || csb < C || cso < C) return LBM_EINVAL;
    add_kernel<<<blocks(npix * C), kThreads, 0, (cudaStream_t)stream>>>(a, csa, b, csb, out, cso, npix, C);
    return check(cudaGetLastError());
}

static bool pool_dims_ok(int N, int H, int W, int C, int f) {
    return N >= 1 && f >= 1 && f <= 64 && H >= f && W >= f && H % f == 0 && W % f == 0 && C >= 1;
}

int lbm_sg_pool(const void* x, int csx, void* y, int csy, int N, int H, int W, int C, int f, void* stream) {
    if (!x || !y || !pool_dims_ok(N, H, W, C, f) || csx < C || csy < C) return LBM_EINVAL;
    const long long n = (long long)N * (H / f) * (W / f) * C;
    pool_kernel<<<blocks(n), kThreads, 0, (cudaStream_t)stream>>>((const bf16*)x, csx, (bf16*)y, csy, N, H, W, C, f);
    return check(cudaGetLastError());
}

int lbm_sg_pool_bwd(const float* g, int csg, float* gx, int csx, int N, int H, int W, int C, int f, void* stream) {
    if (!g || !gx || !pool_dims_ok(N, H, W, C, f) || csx < C || csg < C) return LBM_EINVAL;
    pool_bwd_kernel<<<blocks((long long)N * H * W * C), kThreads, 0, (cudaStream_t)stream>>>(g, csg, gx, csx, N, H, W,
                                                                                            C, f);
    return check(cudaGetLastError());
}

int lbm_sg_upsample(const void* x, int csx, void* y, int csy, int N, int H, int W, int C, int f, void* stream) {
    if (!x || !y || !pool_dims_ok(N, H, W, C, f) || csx < C || csy < C) return LBM_EINVAL;
    upsample_kernel<<<blocks((long long)N * H * W * C), kThreads, 0, (cudaStream_t)stream>>>((const bf16*)x, csx,
                                                                                            (bf16*)y, csy, N, H, W, C,
                                                                                            f);
    return check(cudaGetLastError());
}

int lbm_sg_upsample_bwd(const float* g, int csg, float* gx, int csx, int N, int H, int W, int C, int f,
                        void* stream) {
    if (!g || !gx || !pool_dims_ok(N, H, W, C, f) || csx < C || csg < C) return LBM_EINVAL;
    const long long n = (long long)N * (H / f) * (W / f) * C;
    upsample_bwd_kernel<<<blocks(n), kThreads, 0, (cudaStream_t)stream>>>(g, csg, gx, csx, N, H, W, C, f);
    return check(cudaGetLastError());
}

int lbm_sg_mse(const float* x, int csx, const float* delta, int csd, const float* target, int cst, float* g,
               double* scratch, double* loss, long long npix, int C, void* stream) {
    if (!x || !delta || !target || !g || !scratch || !loss || npix < 1 || C < 1 || csd < C || csx < C || cst < C)
        return LBM_EINVAL;
    const int nb = 256;
    cudaStream_t s = (cudaStream_t)stream;
    mse_kernel<<<nb, kThreads, 0, s>>>(x, csx, delta, csd, target, cst, g, npix, C, scratch);
    mse_finish_kernel<<<1, 32, 0, s>>>(scratch, nb, 1.0 / ((double)npix * C), loss);
    return check(cudaGetLastError());
}

int lbm_sg_adam(float* w, float* m, float* v, const float* g, long long n, float lr, float b1, float b2, float eps,
                int step, void* w16, void* stream) {
    if (!w || !m || !v || !g || n < 1 || step < 1 || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1))
        return LBM_EINVAL;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<blocks(n), kThreads, 0, (cudaStream_t)stream>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2, (bf16*)w16);
    return check(cudaGetLastError());
}

int lbm_sg_pack(const double* phi, const double* ux, const double* uy, const double* P, const double scale[4],
                float* x32, int cs32, void* x16, int cs16, long long npix, void* stream) {
    if (!phi || !ux || !uy || !P || !scale || !x32 || !x16 || npix < 1 || cs32 < 4 || cs16 < 4) return LBM_EINVAL;
    for (int c = 0; c < 4; ++c)
        if (!(scale[c] > 0)) return LBM_EINVAL;
    pack_kernel<<<blocks(npix), kThreads, 0, (cudaStream_t)stream>>>(phi, ux, uy, P, scale[0], scale[1], scale[2],
                                                                      scale[3], x32, cs32, (bf16*)x16, cs16, npix);
    return check(cudaGetLastError());
}

int lbm_sg_unpack(const float* x32, int cs32, const float* delta, int csd, double* phi, double* ux, double* uy,
                  double* P, const double scale[4], double rho_L, double rho_dif, const double* phi_rho,
                  long long npix, void* stream) {
    if (!x32 || !delta || !phi || !ux || !uy || !P || !scale || npix < 1 || cs32 < 4 || csd < 4 || !(rho_L > 0))
        return LBM_EINVAL;
    if (phi_rho == phi) return LBM_EINVAL;
    unpack_kernel<<<blocks(npix), kThreads, 0, (cudaStream_t)stream>>>(x32, cs32, delta, csd, phi, ux, uy, P, scale[0],
                                                                        scale[1], scale[2], scale[3], rho_L, rho_dif,
                                                                        phi_rho, npix);
    return check(cudaGetLastError());
}

int lbm_sg_residual(const double* a, const double* b, long long n, double* out, double* scratch, void* stream) {
    if (!a || !b || !out || !scratch || n < 1) return LBM_EINVAL;
    const int nb = 256;
    cudaStream_t s = (cudaStream_t)stream;
    residual_partial_kernel<<<nb, kThreads, 0, s>>>(a, b, n, scratch);
    residual_finish_kernel<<<1, 32, 0, s>>>(scratch, nb, out);
    return check(cudaGetLastError());
}

int lbm_sg_phase_pressure(const double* phi, const double* P, long long n, double d, double* out, double* scratch,
                          void* stream) {
    if (!phi || !P || !out || !scratch || n < 1 || !(d >= 0.0 && d < 0.5)) return LBM_EINVAL;
    const int nb = 256;
    cudaStream_t s = (cudaStream_t)stream;
    phase_pressure_partial_kernel<<<nb, kThreads, 0, s>>>(phi, P, n, d, scratch);
    phase_pressure_finish_kernel<<<1, 32, 0, s>>>(scratch, nb, out);
    return check(cudaGetLastError());
}

int lbm_sg_phi_project(double* phi, const double* phi0, long long n, double* scratch, void* stream) {
    if (!phi || !phi0 || !scratch || n < 1) return LBM_EINVAL;
    const int nb = 256;
    cudaStream_t s = (cudaStream_t)stream;
    phi_project_kernel<<<nb, kThreads, 0, s>>>(phi, phi0, n, scratch);
    phi_project_finish_kernel<<<1, 32, 0, s>>>(scratch, nb);
    phi_restore_kernel<<<blocks(n), kThreads, 0, s>>>(phi, n, scratch + 3 * nb);
    return check(cudaGetLastError());
}

int lbm_sg_smooth(double* a, double* tmp, int N, int H, int W, int iters, double k, void* stream) {
    if (!a || !tmp || N < 1 || H < 1 || W < 1 || iters < 0 || !(k >= 0.0 && k <= 0.25)) return LBM_EINVAL;
    const long long n = (long long)N * H * W;
    cudaStream_t s = (cudaStream_t)stream;
    for (int it = 0; it < iters; ++it) {
        smooth_kernel<<<blocks(n), kThreads, 0, s>>>(a, tmp, N, H, W, k);
        smooth_kernel<<<blocks(n), kThreads, 0, s>>>(tmp, a, N, H, W, k);
    }
    return check(cudaGetLastError());
}

int lbm_sg_shift(double* a, long long n, double s, void* stream) {
    if (!a || n < 1) return LBM_EINVAL;
    shift_kernel<<<blocks(n), kThreads, 0, (cudaStream_t)stream>>>(a, n, s);
    return check(cudaGetLastError());
}

}  // extern "C"
