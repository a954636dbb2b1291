/*
 * rpm_fno.h -- learned warm start for the cell problem: a 3D spectral neural
 * operator (truncated-Fourier layers) that maps a microstructure to a
 * localisation field, contracted with the macroscopic strain into a
 * strain-field guess; trained on solutions of the solver in rpm.h.
 *
 * The paper has no counterpart: it solves every cell from eps0 = E (Sec. 3,
 * Algorithm 2).  This module only changes the starting field of
 * rpm_solve (its eps0 argument); the solve then runs to the usual stopping
 * criterion, so the converged result does not depend on the network.
 *
 * Network (width W = 16, L layers, m kept modes per axis, periodic N^3 grid):
 *   v0      = P f + p                         per voxel; f = 2 voxel features
 *   v_{l+1} = act_l(A_l v_l + a_l + K_l v_l)  act = GELU (tanh form), none on
 *                                             the last layer
 *   H       = Q v_L + q                       36 channels: H[o][j] = channel 6 o + j
 *   out[o]  = sum_j H[o][j] E_j               strain for macroscopic strain E
 * The output is linear in E, as the solution of the (linear) cell problem
 * is: the network maps the microstructure to a localisation field.
 * K_l: forward DFT of each channel restricted to the kept modes
 * (kx in [0, m); ky, kz in {0..m-1} U {N-m..N-1}: 4 m^3 modes), per-mode complex
 * channel mixing R_l[i][o], and the real inverse of that half spectrum
 * (1 / N^3, doubled for kx >= 1).  Loss: mean squared error over all outputs.
 *
 * Parameter vector (float32, rpm_fno_param_count floats), in this order:
 *   P [16][2]  p [16]  Q [36][16]  q [36]  (then zeros up to float 768)
 *   per layer l, from 768 + l * (272 + 2 * 2m * m * 2m * 256):
 *     A_l [16][16] (out, in)  a_l [16]
 *     R_l [ky_i][kx][kz_i][i][o] complex (re, im), ky_i, kz_i in [0, 2m):
 *         index i < m is frequency i, index i >= m is frequency N - 2m + i.
 * Gradients (rpm_fno_get_grads) use the same layout; for R the pair is
 * (dL/dRe, dL/dIm).
 *
 * Device arrays (caller-owned, float32, contiguous):
 *   feat    [B][2][N][N][N]  voxel features (rpm_fno_features computes
 *                            log10(Young / Young of phase 0) and Poisson ratio)
 *   out     [B][6][N][N][N]  strain components in Voigt order (11,22,33,23,13,12),
 *                            tensor (not engineering) shears
 *   target  as out
 * E_dir: HOST float [B][6], the macroscopic strain of each sample (Voigt
 *        order, tensor shears).
 *
 * All calls are stream-ordered on the stream given at creation (NULL: legacy
 * stream); functions that return host values synchronise it.  Errors:
 * RPM_ERR_INVALID_ARG (bad argument, message in rpm_fno_last_error),
 * RPM_ERR_OOM, RPM_ERR_CUDA.
 */
#ifndef RPM_FNO_H
#define RPM_FNO_H

#include <stddef.h>

#include "rpm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RPM_FNO_WIDTH 16
#define RPM_FNO_MAX_MODES 12
#define RPM_FNO_MAX_LAYERS 8
#define RPM_FNO_MAX_N 128
#define RPM_FNO_MAX_BATCH 64

typedef struct rpm_fno rpm_fno;

/* Arithmetic of the network's transforms (rpm_fno_config.precision). */
#define RPM_FNO_FP32 0  /* float32 throughout (SIMT FMA) */
#define RPM_FNO_BF16 1  /* truncated DFT stages as BF16 tensor-core products with float32
                           accumulation (mma.sync m16n8k16) where N % 16 == 0; everything else
                           float32 */

typedef struct {
  int n;          /* grid side N: 24..128, a multiple of 8, N >= 2 * modes */
  int modes;      /* m: 1..RPM_FNO_MAX_MODES */
  int layers;     /* L: 1..RPM_FNO_MAX_LAYERS */
  int max_batch;  /* largest batch B of any call, 1..RPM_FNO_MAX_BATCH */
  int precision;  /* RPM_FNO_FP32 or RPM_FNO_BF16 */
} rpm_fno_config;

typedef struct {
  float lr, beta1, beta2, eps, weight_decay; /* Adam (decoupled weight decay) */
} rpm_fno_adam;

/* Floats in the parameter vector for m modes and L layers (0 if invalid). */
size_t rpm_fno_param_count(int modes, int layers);

/* Allocate a network and its training buffers (parameters zero). */
rpm_status rpm_fno_create(const rpm_fno_config* cfg, void* cuda_stream, rpm_fno** out);

/* Copy the parameter vector in / out (HOST float [param_count]); set resets Adam. */
rpm_status rpm_fno_set_params(rpm_fno* f, const float* params);
rpm_status rpm_fno_get_params(rpm_fno* f, float* params);
/* Gradients of the last rpm_fno_loss_grad / rpm_fno_train_step (HOST float [param_count]). */
rpm_status rpm_fno_get_grads(rpm_fno* f, float* grads);

/* out = network(feat, E_dir) for a batch of 1..max_batch samples (async). */
rpm_status rpm_fno_forward(rpm_fno* f, int batch, const float* feat, const float* E_dir,
                           float* out);

/* Forward with the activations kept, loss against target, backward: the
 * gradient vector is overwritten.  loss (optional host double) is the mean
 * squared error; it synchronises the stream when given. */
rpm_status rpm_fno_loss_grad(rpm_fno* f, int batch, const float* feat, const float* E_dir,
                             const float* target, double* loss);

/* One Adam step on the current gradients (step count kept in the network). */
rpm_status rpm_fno_adam_step(rpm_fno* f, const rpm_fno_adam* opt);

/* rpm_fno_loss_grad then rpm_fno_adam_step. */
rpm_status rpm_fno_train_step(rpm_fno* f, int batch, const float* feat, const float* E_dir,
                              const float* target, const rpm_fno_adam* opt, double* loss);

/* Voxel features of a phase map: feat[0] = log10(Young(phase) / Young(phase 0)),
 * feat[1] = Poisson ratio, for n voxels (DEVICE phase uint8 [n], DEVICE feat
 * float [2][n]; host moduli of n_phases phases). */
rpm_status rpm_fno_features(const uint8_t* phase, long long n, int n_phases,
                            const rpm_iso* phases, float* feat, void* cuda_stream);

/* Warm start of rpm_solve for the context's cell and macroscopic strain E
 * (nonzero): features of the cell, the network, then the projection onto the
 * compatible fields of mean E (rpm_apply_gamma, RPM_GAMMA_PROJECT).
 * eps0: DEVICE float [6][nz][ny][nx]; the context grid must be N^3.  Returns
 * after eps0 is written (synchronises both streams). */
rpm_status rpm_fno_warm_start(rpm_fno* f, rpm_ctx* ctx, const double E[6], float* eps0);

/* rpm_solve from the learned warm start, with the cold start as the
 * fallback: rpm_fno_warm_start, then rpm_solve from that guess; if that
 * solve diverges or does not converge, rpm_solve again from eps0 = E (the
 * context's own form).  Outputs and info as rpm_solve (info of the last
 * solve, with the F applications, device time and launches of both);
 * used_guess (optional) = 1 when the learned start's solve is the answer. */
rpm_status rpm_fno_solve(rpm_fno* f, rpm_ctx* ctx, const double E[6], float* eps_out,
                         float* sig_out, int out_on_host, rpm_solve_info* info, int* used_guess);

size_t rpm_fno_device_bytes(const rpm_fno* f);
const char* rpm_fno_last_error(const rpm_fno* f);
void rpm_fno_destroy(rpm_fno* f);

#ifdef __cplusplus
}
#endif

#endif /* RPM_FNO_H */
