/*
 * adi_corrector.h -- learned coarse-step corrector for the ADI Maxwell stepper
 * (C-ABI, GB300 / sm_103a).
 *
 * The paper (arXiv 2103.06998) has no learned component; this is an addition
 * on top of its method.  One ADI step of length k*tau (a "coarse" step, k = 8
 * by default) is followed by a 3D convolution net that predicts the difference
 * between k steps of length tau and that one step, both started from the same
 * state.  The plain ADI step stays the fallback and the reference for the error.
 *
 * Net (fixed architecture): four 3x3x3 convolutions with zero padding on the
 * coefficient grid (N_x x N_y x N_z voxels, one voxel per B-spline
 * coefficient), 9 -> 32 -> 32 -> 32 -> 6 channels, ReLU after the first three.
 *   out[z,y,x,co] = b[co] + sum_{dz,dy,dx,ci} in[z+dz-1, y+dy-1, x+dx-1, ci]
 *                   w[tap(dz,dy,dx)][ci][co],   tap = 9 dz + 3 dy + dx.
 * Weights and activations are BF16, products accumulate in FP32 (tensor
 * cores, tcgen05); the master weights, gradients and Adam moments are FP32.
 *
 * Input features of a state (channels 0..8): the six field components E1, E2,
 * E3, H1, H2, H3 divided by s = sqrt(mean of the squared coefficients of all
 * six components), then the row coefficients a, 2b/tau, 4c/tau^2 of the
 * handle's step (dimensionless, in (-1, 1]).  Output channels 0..5: the
 * predicted (fine - coarse) / s.  Correction: fields += s * out, constrained
 * (Dirichlet) coefficients untouched.
 *
 * Device arrays passed to these calls (caller-owned, on the net's device, each
 * 16-byte aligned: the convolutions read them with TMA; ADI_EINVAL / ADI_ECUDA
 * otherwise):
 *   features  X: BF16 [z][y][x][16]  (channels 9..15 are zero)
 *   targets   T: FP32 [z][y][x][8]   (channels 6, 7 are zero)
 *   outputs   Y: FP32 [z][y][x][8]
 * All calls are asynchronous on the net's stream unless they return host data.
 *
 * Errors common to these calls: ADI_EINVAL for a NULL net, handle or array, a
 * misaligned array, handles that do not fit (the net's calls and
 * adi_fields_distance want FP32 handles on the same grid; adi_copy_state wants
 * the same grid, degree and precision), or an argument outside its documented
 * range; ADI_ECUDA when a CUDA call fails (ADI_ENOMEM for an allocation).  Messages: adi_net_last_error(n)
 * (adi_net_last_error(NULL) for a failed create or a NULL net).  Calls that
 * step a handle pass its status through (message in adi_last_error(h)).
 *
 * Parameter vector (FP32, ADI_NET_PARAMS floats): for layer l = 0..3 the
 * weights w_l[27][CI_l][CO_l] then the bias b_l[CO_l], with the padded channel
 * counts CI = (16, 32, 32, 32), CO = (32, 32, 32, 16); the padding entries
 * (layer 0 ci >= 9, layer 3 co >= 6) must be zero and stay zero.
 */
#ifndef ADI_CORRECTOR_H
#define ADI_CORRECTOR_H

#include "adi_maxwell.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adi_net_ctx* adi_net;

#define ADI_NET_PARAMS 83056

/* Create a net for a coefficient grid of N_x x N_y x N_z voxels (each >= 1,
 * N_x <= 1024).  Weights start at zero; the net uses its own stream. */
adi_status adi_net_create(int Nx, int Ny, int Nz, adi_net* out);
/* Issue the net's work on `stream` (a cudaStream_t; NULL: the net's own). */
adi_status adi_net_set_stream(adi_net n, void* stream);
/* Copy the FP32 parameter vector from / to the host (count must be
 * ADI_NET_PARAMS); setting resets the Adam moments and step counter.
 * adi_net_set_params: ADI_ENUMERIC if w holds a NaN or Inf (nothing set). */
adi_status adi_net_set_params(adi_net n, const float* w, size_t count);
adi_status adi_net_get_params(adi_net n, float* w, size_t count);

/* X = features of the fields of FP32 handle h (same grid as the net); the
 * scale s is kept on the device for adi_net_target and adi_net_apply.
 * ADI_ESTATE if h is not factored (its row coefficients are not final). */
adi_status adi_net_features(adi_net n, adi_handle h, void* X);
/* T = (fields(fine) - fields(coarse)) / s, s from the last adi_net_features. */
adi_status adi_net_target(adi_net n, adi_handle fine, adi_handle coarse, float* T);
/* Y = net(X). */
adi_status adi_net_forward(adi_net n, const void* X, float* Y);
/* fields(h) += s * Y on the free coefficients. */
adi_status adi_net_apply(adi_net n, adi_handle h, const float* Y);

/* One training step on one sample: forward, mean squared error against T,
 * backward, Adam (Kingma and Ba) with learning rate lr, betas 0.9 / 0.999,
 * eps 1e-8.  The loss of the sample is accumulated on the device; read (and
 * reset) the running sum with adi_net_loss.  lr must be finite and > 0. */
adi_status adi_net_train_step(adi_net n, const void* X, const float* T, float lr);
/* Gradient of the loss of one sample without updating (for checks):
 * grad receives ADI_NET_PARAMS floats, *loss the loss.  Synchronises. */
adi_status adi_net_gradient(adi_net n, const void* X, const float* T, float* grad, double* loss);
/* Sum of the losses since the last call and their count; synchronises. */
adi_status adi_net_loss(adi_net n, double* sum, int* count);

/* Relative l2 distance ||fields(a) - fields(b)|| / ||fields(b)|| over all six
 * components; synchronises. */
adi_status adi_fields_distance(adi_handle a, adi_handle b, double* rel);
/* Copy the fields and the time of src into dst (same grid, degree and
 * precision; the time steps may differ).  Asynchronous on dst's stream after
 * src's work: the call synchronises src's stream first. */
adi_status adi_copy_state(adi_handle dst, adi_handle src);

/* Guarded time loop with the corrector.  `coarse` steps with dt = k tau and
 * `fine` with tau (same grid, material and source); the state lives in
 * `coarse`.  For each window of guard_every coarse steps: the first step is
 * taken both ways (k fine steps from a copy, one corrected coarse step); if
 * their relative l2 distance exceeds tol, the fine result is kept and the rest
 * of the window runs as plain fine steps (counted in *n_fallback), else the
 * rest of the window runs corrected coarse steps.  m coarse steps in all.
 * *max_err receives the largest guard distance.  Synchronises at each guard.
 * ADI_EINVAL unless m, k, guard_every >= 1, tol > 0, the output pointers are
 * set and coarse's time step is k times fine's. */
adi_status adi_corrector_run(adi_net n, adi_handle coarse, adi_handle fine, int m, int k,
                             int guard_every, double tol, int* n_fallback, double* max_err);

/* Release the net.  NULL is ignored. */
void adi_net_destroy(adi_net n);
/* Last error message of the net (never NULL). */
const char* adi_net_last_error(adi_net n);

#ifdef __cplusplus
}
#endif

#endif /* ADI_CORRECTOR_H */
