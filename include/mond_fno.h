/*
 * mond_fno.h -- C ABI of the learned warm start of the MOND field solve.
 *
 * The paper seeds the iteration with the H of the previous time step
 * (Sect. 5.2 item iv: one iteration then suffices for small steps). This
 * library adds a learned seed: a Fourier neural operator (FNO) on a coarse
 * grid maps the Newtonian field g_N to the converged H; the prediction is
 * upsampled, projected onto its divergence-free part and used as
 * MOND_WARM_GUESS for one iteration (mond_pm_solve_field). The paper has no
 * network; the architecture is fixed by this library:
 *   input  x: 4 channels on n^3 (g_N / s, with s the RMS of g_N, and
 *          log10(|g_N|/a0)/4), output y: 3 channels (H / s);
 *   lift (4 -> C), L Fourier layers v <- gelu(W v + b + K v) (no gelu on
 *   the last), projection (C -> 3); K keeps the modes kx in [0, M),
 *   ky, kz in [-M, M) and mixes channels per mode with complex weights.
 * Parameters are one float32 array (layout in mond_fno_param_count); the
 * forward and backward passes read a bfloat16 copy of it (mond_fno_cast) and
 * accumulate in FP32. All pointers are device pointers owned by the caller;
 * every call enqueues on the given stream and returns 0 or a negative code.
 */
#ifndef MOND_FNO_H
#define MOND_FNO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n;       /* coarse grid side (8..64, a multiple of 4, 2M <= n) */
  int32_t width;   /* channels C (even, 2..32) */
  int32_t modes;   /* modes per axis M */
  int32_t layers;  /* Fourier layers L */
} mond_fno_shape;

/* Number of float32 parameters. Layout: lift P[C][4], p[C]; for each layer
 * W[C][C], b[C], R[K][C][C] complex (re, im interleaved; R[k][j][c] maps
 * input channel j to output c at mode k, K = M (2M)(2M), k = (kz (2M) + ky) M
 * + kx with ky, kz in [0, 2M) standing for frequencies 0..M-1, -M..-1);
 * projection Q[3][C], q[3]. */
int mond_fno_param_count(mond_fno_shape s, int64_t* count);

/* Device workspace bytes for one forward + backward of one sample. */
int mond_fno_workspace_bytes(mond_fno_shape s, size_t* bytes);

/* Seeded initial parameters (float32). */
int mond_fno_init(mond_fno_shape s, uint64_t seed, float* params, void* stream);

/* bfloat16 copy of the parameters used by forward/backward. */
int mond_fno_cast(mond_fno_shape s, const float* params, uint16_t* params_bf16, void* stream);

/* Forward of one sample: x [4][n^3] -> y [3][n^3]; the activations stay in
 * the workspace for mond_fno_backward. */
int mond_fno_forward(mond_fno_shape s, const uint16_t* params_bf16, const float* x, float* y, void* workspace,
                     void* stream);

/* Backward of the sample of the last forward: dy [3][n^3] -> grad (float32,
 * same layout as the parameters) += d loss / d params. */
int mond_fno_backward(mond_fno_shape s, const uint16_t* params_bf16, const float* x, const float* dy, float* grad,
                      void* workspace, void* stream);

/* Relative squared error of one sample, loss = weight sum (y - t)^2 / sum t^2,
 * added to loss_acc[0], and its gradient dy = 2 weight (y - t) / sum t^2.
 * loss_acc points to two device doubles; loss_acc[1] is scratch. count is the
 * number of floats in y, t and dy. */
int mond_fno_loss(int64_t count, const float* y, const float* t, float* dy, float weight, double* loss_acc,
                  void* stream);

/* Adam step on all parameters: params -= lr mhat / (sqrt(vhat) + eps);
 * m, v float32 moments; step = 1, 2, ...; grad is cleared afterwards. When
 * clip_norm > 0 the gradient is first scaled by min(1, clip_norm / |grad|);
 * a gradient with a non-finite norm is dropped (parameters and moments keep
 * their values). scratch: one device double. */
int mond_fno_adam(int64_t count, float* params, float* grad, float* m, float* v, float lr, float beta1, float beta2,
                  float eps, int step, float clip_norm, double* scratch, void* stream);

/* Network input from a fine Newtonian field: g_N [3][N^3] (N = f n) is
 * averaged over f^3 blocks to the coarse grid and normalised: x [4][n^3].
 * scale_out points to 4 device floats, 8-byte aligned: scale_out[0] = s (the
 * RMS of the coarse g_N); scale_out[2..3] are scratch. */
int mond_fno_input(int N, int n, float a0, const float* gN, float* x, float* scale_out, void* stream);

/* Fine field from a coarse network output: H [3][N^3] = s * cubic-convolution
 * upsampling (Keys, a = -1/2; periodic, cell centred; one axis at a time) of
 * y [3][n^3]; s read from scale. N must be a multiple of n, at most 64 n. scratch: device
 * memory of mond_fno_output_scratch_bytes(N, n) bytes. */
int mond_fno_output(int N, int n, const float* y, const float* scale, float* H, void* scratch, void* stream);

/* Scratch bytes mond_fno_output needs (0 if N is not a multiple of n). */
size_t mond_fno_output_scratch_bytes(int N, int n);

/* Means of f^3 blocks of a fine field: fine [ncomp][N^3] -> coarse
 * [ncomp][n^3]. When fine2 is not NULL the blocks of (fine + fine2)/2 are
 * averaged (the centre of the iteration's two-cycle); when scale (a device
 * float) is not NULL the means are divided by scale[0] (training targets in
 * the units of the network output). */
int mond_fno_coarsen(int N, int n, int ncomp, const float* fine, const float* fine2, float* coarse,
                     const float* scale, void* stream);

/* Density of a mixture of Plummer (kind 0) and Hernquist (kind 1) spheres on
 * the N^3 mesh of pixel width s, truncated at radius rmax (pixels): centre
 * [K][3] (pixels from the domain centre), mass [K], radius [K] (pixels). */
int mond_fno_mixture_density(int N, double s, int K, const float* centre, const float* mass, const float* radius,
                             const int* kind, float rmax, float* rho, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MOND_FNO_H */
