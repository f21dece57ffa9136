/*
 * lc_nn.h -- C ABI of the learned warm start's kernels (sm_103a): a small 3D
 * U-Net proposes the relaxed order parameter Q around a colloid (the defect
 * structure Lintuvuori et al. obtain by relaxation, Sec. 3.2), and the
 * lattice relaxation of lc_lb.h then starts from that proposal.
 *
 * Conventions: every pointer is device memory owned by the caller; all calls
 * are asynchronous on `stream` (a cudaStream_t, NULL = legacy default) and
 * return LC_NN_OK or a negative LC_NN_ERR_*.  Activations are channels-last
 * BF16 ([position][channel], position = x + W*(y + H*z)); weights are
 * [C_out][taps][C_in] BF16 (taps = 27 for a 3x3x3 kernel ordered
 * (dz+1)*9 + (dy+1)*3 + (dx+1), or 1); gradients and masters are FP32.  All
 * boundaries are periodic.  Convolutions accumulate in FP32 on the tensor
 * cores.
 */
#ifndef LC_NN_H
#define LC_NN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { LC_NN_OK = 0, LC_NN_ERR_ARG = -1, LC_NN_ERR_CUDA = -2 };

/* out[p][co] = act(bias[co] + sum_{t,ci} w[co][t][ci] in[p + offset(t)][ci]),
 * act = ReLU if relu else identity.  cin % 16 == 0, cout % 8 == 0,
 * cout <= 80.  out32 (FP32) and/or out16 (BF16) may be NULL. */
int lc_nn_conv3d_fwd(const void* in, const void* w, const float* bias, float* out32, void* out16, int W, int H, int D,
                     int cin, int cout, int taps, int relu, void* stream);
/* Input gradient: din[p][ci] = sum_{t,co} w[co][t][ci] dout[p - offset(t)][co].
 * wt_scratch: cout*cin*taps BF16 of caller memory.  cout % 16 == 0, cin % 8 == 0. */
int lc_nn_conv3d_dgrad(const void* dout, const void* w, void* wt_scratch, float* din32, void* din16, int W, int H,
                       int D, int cin, int cout, int taps, void* stream);
/* Weight gradient, accumulated: dw[co][t][ci] += sum_p dout[p][co] in[p + offset(t)][ci]
 * (dw FP32, cout % 16 == 0, cin % 8 == 0, cin <= 80).  The positions are
 * split into at most 256 chunks whose partial sums go to `partial` (caller
 * memory of lc_nn_wgrad_partial_floats(...) floats) and are then added in
 * chunk order, so the result is the same on every run.  Errors: LC_NN_ERR_ARG. */
int lc_nn_conv3d_wgrad(const void* dout, const void* in, float* dw, float* partial, int W, int H, int D, int cin,
                       int cout, int taps, void* stream);
/* Size in floats of the partial-sum buffer of lc_nn_conv3d_wgrad. */
size_t lc_nn_wgrad_partial_floats(int W, int H, int D, int cin, int cout, int taps);
/* db[c] += sum_p dout[p][c]. */
int lc_nn_bias_grad(const float* dout, float* db, int npos, int c, void* stream);
/* dz = dy * (y > 0) for n elements; dz32 (FP32) and/or dz16 (BF16). */
int lc_nn_relu_bwd(const float* dy, const void* y, float* dz32, void* dz16, size_t n, void* stream);
int lc_nn_cast_bf16(const float* a, void* b, size_t n, void* stream);
/* 2x2x2 mean pooling of an S^3 x c tensor (S even) and its adjoint
 * (din accumulated: din += adjoint(dout)). */
int lc_nn_pool2(const void* in, void* out, int S, int c, void* stream);
int lc_nn_pool2_bwd(const float* dout, float* din, int S, int c, void* stream);
/* out (S^3 x (c1+c2)) = [nearest x2 upsampling of lo ((S/2)^3 x c1), skip (S^3 x c2)]
 * and its adjoint (dlo overwritten, dskip accumulated). */
int lc_nn_up2_concat(const void* lo, const void* skip, void* out, int S, int c1, int c2, void* stream);
int lc_nn_up2_concat_bwd(const float* dout, float* dlo, float* dskip, int S, int c1, int c2, void* stream);
/* Masked mean-square error of pred = base + out[:, 0:5] against target (both
 * npos x 5) over positions with fluid[p] > 0: *loss += inv_count * sum d^2
 * (FP64; caller zeroes it), grad (npos x cout, may be NULL) = dL/dout. */
int lc_nn_mse(const float* out, const float* base, const float* target, const float* fluid, float* grad,
              double* loss, int npos, int cout, double inv_count, void* stream);
/* Long-wavelength term of the loss: the masked error d = (base + out[:, 0:5]
 * - target) * [fluid[p] > 0] averaged over cubes of b^3 positions (box S^3,
 * position p = x + S (y + S z), S divisible by b), E = mean of d over a cube:
 * *loss += inv_count * sum over cubes and components of E^2 (FP64; caller
 * zeroes it or adds to the MSE's), grad[p][c] += inv_count * 2 E / b^3 at
 * fluid positions, c < 5 (accumulated into the MSE's gradient; may be NULL).
 * blk: caller-owned device scratch of (S/b)^3 * 5 floats.  With b = 1 it is
 * the MSE itself.  Errors: LC_NN_ERR_ARG (b < 1, S % b != 0, cout < 5). */
int lc_nn_mse_coarse(const float* out, const float* base, const float* target, const float* fluid, float* grad,
                     double* loss, float* blk, int S, int b, int cout, double inv_count, void* stream);
/* Adam step (step >= 1) on FP32 masters p with moments m, v; p16 (BF16 copy) may be NULL. */
int lc_nn_adam(float* p, const float* g, float* m, float* v, void* p16, size_t n, float lr, float b1, float b2,
               float eps, int step, void* stream);
/* Network input (channels last, cpad >= 9, BF16): [solid indicator, 5 Q
 * components, R/32, pitch/64, 20 w, 0...] from FP64 SoA fields solid ([npos],
 * -1 = fluid) and q ([5][npos]); base (npos x 5, FP32) = Q, fluid = 1 - solid,
 * *nfluid += number of fluid positions.  base, fluid, nfluid may be NULL. */
int lc_nn_pack_input(const double* solid, const double* q, double R, double pitch, double w, void* x16, float* base,
                     float* fluid, double* nfluid, int npos, int cpad, void* stream);
/* a (npos x 5, FP32 channels last) = q ([5][npos] FP64). */
int lc_nn_from_soa(const double* q, float* a, int npos, void* stream);
/* q[c][p] = a[p][c] + base[p][c] for c < 5 (FP64 SoA out; base may be NULL). */
int lc_nn_to_soa(const float* a, const float* base, double* q, int npos, int cout, void* stream);
/* Trilinear x2 upsampling of a periodic cell-centred SoA field [c][S^3] to [c][(2S)^3]. */
int lc_nn_trilinear2(const double* a, double* b, int S, int c, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LC_NN_H */
