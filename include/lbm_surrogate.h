/* Kernels of the learned warm-start surrogate (liblbm.so).
 *
 * The paper has no network: these are a service of the library.  A small
 * convolutional network maps the fields (phi, u, P) of a D2Q9 state to the
 * state many steps later; its training and inference run on these kernels,
 * and lbm_init_fields_ex rebuilds the populations from its output
 * (equilibria of Eqs. 2 and 6-7 of the paper plus the filtered Chapman-Enskog
 * non-equilibrium part of g, Eq. 11).
 *
 * Conventions (every function):
 *   - Tensors are channels-last on the device: pixel p = (n H + y) W + x of
 *     N images of H x W, element (p, c) at p * stride + c.  A stride larger
 *     than the channel count reads or writes a slice of a wider tensor (the
 *     caller passes the slice's first element).  "bf16" tensors are arrays of
 *     16-bit bfloat16 values (void*), the rest float or double.
 *   - Convolutions are periodic 3x3, "same" size:
 *       y[p, co] = bias[co] + sum_{dy, dx, ci} w[co, 3 dy + dx, ci] x[p + (dy - 1, dx - 1), ci]
 *     (offsets wrap inside each image); w is bf16 [Co][9][Ci].  Ci and Co
 *     are multiples of 16 (zero-pad), Co <= 128, N H W a multiple of 16.
 *   - Pooling and upsampling are by a factor f (1..64) in both directions;
 *     H and W (always the FINE grid's size) are multiples of f.
 *   - The caller owns every buffer; the functions allocate nothing.  All are
 *     asynchronous on `stream` (NULL: default stream).
 *   - Return LBM_OK, LBM_EINVAL (NULL pointer, bad size or stride),
 *     LBM_ECUDA (launch failed).
 */
#ifndef LBM_SURROGATE_H
#define LBM_SURROGATE_H

#ifdef __cplusplus
extern "C" {
#endif

/* y (float) = periodic 3x3 convolution of x (bf16) with w (bf16), plus bias
 * (float[Co], may be NULL): an implicit GEMM on the tcgen05 tensor cores,
 * bf16 products, FP32 sums in tensor memory, 128 pixels per MMA.  When W is a
 * multiple of 128 and the weights of all nine taps fit in shared memory with
 * four input rows (9 Co Ci + 4 x 130 Ci bf16 values, at most 200 KB), a CTA
 * marches a 128-pixel row segment down a chunk of rows, copying every input
 * row into shared memory once; otherwise a CTA takes 128 consecutive pixels
 * and copies each tap's shifted rows.  Both accumulate the taps in the same
 * order.  x's channel stride csx is a multiple of 8 and x and w start
 * on 16-byte boundaries (the operands are staged in 16-byte copies);
 * LBM_EINVAL otherwise.  A bounded wait inside the kernel that gives up leaves
 * its CTA's part of y unwritten and is reported by lbm_sg_status. */
int lbm_sg_conv3x3(const void* x, int csx, const void* w, const float* bias, float* y, int csy, int N, int H, int W,
                   int Ci, int Co, void* stream);

/* Synchronises `stream` and reports whether a bounded wait of a surrogate
 * kernel gave up since the last call: LBM_ETIMEOUT (the flag is cleared),
 * else LBM_OK; LBM_ECUDA if the copy or the synchronisation failed. */
int lbm_sg_status(void* stream);

/* Floats of scratch lbm_sg_conv3x3_wgrad needs for these sizes on the
 * current device (the row march below sizes its partials by the device's
 * resident CTAs). */
long long lbm_sg_wgrad_scratch_floats(int N, int H, int W, int Ci, int Co);

/* gw (float [Co][9][Ci]) = gradient of sum_p <gy[p], y[p]> with respect to w
 * for y = lbm_sg_conv3x3(x, w): gw[co, tap, ci] = sum_p gy[p, co] x[p + d(tap), ci].
 * x, gy bf16.  When W is a multiple of 32, Co is at most 128, Ci is at
 * most 128 or a multiple of 128, the channel strides are multiples of 8 and
 * x, gy and scratch start on 16-byte boundaries, the sums are GEMMs over
 * pixels on the tcgen05 tensor cores (each CTA marches a 64- or 32-pixel row
 * segment down a chunk of rows for one tap row and a block of at most 128
 * input channels, its operands transposed into shared memory, its three
 * taps accumulated in tensor memory); otherwise warp-level mma.sync over
 * chunks of 1024 pixels.  Deterministic either way: per-CTA (or per-chunk) partials
 * summed in a fixed order.  A bounded wait that gives up is reported by
 * lbm_sg_status. */
int lbm_sg_conv3x3_wgrad(const void* x, int csx, const void* gy, int csg, float* gw, float* scratch,
                         long long scratch_floats, int N, int H, int W, int Ci, int Co, void* stream);

/* wt (bf16 [Ci][9][Co]) = w with input and output channels exchanged and the
 * taps reversed: lbm_sg_conv3x3(gy, wt) is then the gradient with respect to
 * the convolution's input x. */
int lbm_sg_weight_flip(const void* w, void* wt, int Ci, int Co, void* stream);

/* gb[c] = sum_p g[p, c] (float); scratch holds at least 64 C floats. */
int lbm_sg_bias_grad(const float* g, int csg, float* gb, float* scratch, long long npix, int C, void* stream);

/* y (bf16) = max(a, 0). */
int lbm_sg_relu(const float* a, int csa, void* y, int csy, long long npix, int C, void* stream);

/* ga (float, stride C) = g where a > 0, else 0; ga16 (bf16, stride C, may be
 * NULL) its bf16 copy. */
int lbm_sg_relu_bwd(const float* g, int csg, const float* a, int csa, float* ga, void* ga16, long long npix, int C,
                    void* stream);

/* y (bf16) = a rounded to bf16. */
int lbm_sg_to_bf16(const float* a, int csa, void* y, int csy, long long npix, int C, void* stream);

/* out = a + b (float). */
int lbm_sg_add(const float* a, int csa, const float* b, int csb, float* out, int cso, long long npix, int C,
               void* stream);

/* y (bf16, H/f x W/f images) = means of the f x f blocks of x (bf16, H x W). */
int lbm_sg_pool(const void* x, int csx, void* y, int csy, int N, int H, int W, int C, int f, void* stream);
/* gx (float, H x W) = g (float, H/f x W/f) / f^2 spread over each block. */
int lbm_sg_pool_bwd(const float* g, int csg, float* gx, int csx, int N, int H, int W, int C, int f, void* stream);
/* y (bf16, H x W) = x (bf16, H/f x W/f) repeated over each f x f block. */
int lbm_sg_upsample(const void* x, int csx, void* y, int csy, int N, int H, int W, int C, int f, void* stream);
/* gx (float, H/f x W/f) = sums of g (float, H x W) over each block. */
int lbm_sg_upsample_bwd(const float* g, int csg, float* gx, int csx, int N, int H, int W, int C, int f,
                        void* stream);

/* Mean squared error of out = x + delta against target over the first C
 * channels: *loss (device double) = mean (out - target)^2 (FP64 sums), and
 * g (float, stride csd) = d loss / d delta (zero in channels C..csd-1).
 * scratch: 256 doubles. */
int lbm_sg_mse(const float* x, int csx, const float* delta, int csd, const float* target, int cst, float* g,
               double* scratch, double* loss, long long npix, int C, void* stream);

/* One Adam update (bias-corrected, step >= 1) of n FP32 master values w with
 * moments m, v and gradient g; w16 (bf16, may be NULL) receives the rounded
 * weights the convolutions read. */
int lbm_sg_adam(float* w, float* m, float* v, const float* g, long long n, float lr, float b1, float b2, float eps,
                int step, void* w16, void* stream);

/* Network input from one grid's fields (device FP64, x fastest, as
 * lbm_macro writes them: phi, the two components of rho u, P): x32 (float,
 * stride cs32 >= 4) = (phi, rho u_x, rho u_y, P) / scale, x16 (bf16, stride
 * cs16 >= 4) the same rounded, zero in channels 4..cs16-1. */
int lbm_sg_pack(const double* phi, const double* rux, const double* ruy, const double* P, const double scale[4],
                float* x32, int cs32, void* x16, int cs16, long long npix, void* stream);

/* Fields for lbm_init_fields from the network output: (phi, rho u, P) =
 * (x32 + delta) * scale, written as phi, u = rho u / (rho_L + phi_c rho_dif)
 * (the density of the paper's rho(phi), phi_c clipped to [0, 1] so that a
 * slight undershoot of the prediction in the light phase cannot make it
 * vanish) and P.  phi_c is taken from phi_rho (device, npix doubles, not the
 * phi output) when given, e.g. a projected phi, else from the predicted phi. */
int lbm_sg_unpack(const float* x32, int cs32, const float* delta, int csd, double* phi, double* ux, double* uy,
                  double* P, const double scale[4], double rho_L, double rho_dif, const double* phi_rho,
                  long long npix, void* stream);

/* out (device, 2 doubles) = (sum (a - b)^2, sum a^2) over n values, FP64 in
 * a fixed order; scratch: 512 doubles.  The convergence measure of the
 * warm-start comparison: ||P(t) - P(t - k)|| / ||P(t)||. */
int lbm_sg_residual(const double* a, const double* b, long long n, double* out, double* scratch, void* stream);

/* out (device, 4 doubles) = (mean P over the bulk heavy phase phi >= 1 - d,
 * mean P over the bulk light phase phi <= d, and the two node counts), FP64
 * in a fixed order; scratch: 1024 doubles; 0 <= d < 1/2.  out[0] - out[1] is
 * the Laplace pressure jump of the whole state (Section 4.1), the quantity
 * whose relative change between checks is the warm-start comparison's
 * convergence measure. */
int lbm_sg_phase_pressure(const double* phi, const double* P, long long n, double d, double* out, double* scratch,
                          void* stream);

/* iters times two explicit diffusion passes a <- a + k lap(a) (five-point,
 * periodic in each of N images of H x W, 0 <= k <= 1/4, tmp: N H W doubles):
 * removes the block-scale roughness of a prediction before it seeds a run. */
int lbm_sg_smooth(double* a, double* tmp, int N, int H, int W, int iters, double k, void* stream);

/* Projection of a predicted phi (device, n doubles, in place) onto the start
 * phi0: phi <- clip(phi0 + 4 phi0 (1 - phi0) (phi - phi0), 0, 1) keeps the
 * predicted change inside the start's interface band (none in the bulk
 * phases, where 16-bit noise of the prediction would otherwise seed
 * spurious mixed regions and densities below rho_L), then
 * phi <- phi + c 4 phi (1 - phi) with c chosen so that sum phi = sum phi0
 * (Eq. 1 conserves the total; the correction moves the interfaces, not the
 * bulk; c uses the weights before the correction, so the total is restored
 * up to FP64 rounding).  FP64 sums in a fixed order; scratch: 769 doubles. */
int lbm_sg_phi_project(double* phi, const double* phi0, long long n, double* scratch, void* stream);

/* a[k] += s (used to restore the exact total of phi after a prediction). */
int lbm_sg_shift(double* a, long long n, double s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_SURROGATE_H */
