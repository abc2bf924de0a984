/* scw_fno.h -- C ABI of the learned surrogate: a Fourier neural operator (FNO)
 * that maps refractive-index slices to the exit-plane field, trained and run on
 * one GPU by hand-written sm_103a kernels.
 *
 * The surrogate is not part of the coupled-wave method of arXiv 2404.07293: it
 * stands in front of it. Where its own error estimate is above a threshold the
 * caller falls back to the plain method (scw_synthesize on a fresh solve), which
 * also produces its training targets (the field on the exit plane z = z_L,
 * Eq. 9 below the sample).
 *
 * Network (Li et al., ICLR 2021, width C = 32, m x m kept frequencies):
 *   features  a[2s] = Re n_s - 1, a[2s+1] = Im n_s of S slices, nearest-upsampled
 *             from in_grid^2 to N^2 pixels
 *   lift      V_0 = P a + p                                  (1x1 convolution)
 *   layer l   Vh = truncated DFT of V_l (kept kx, ky in [-m/2, m/2), unnormalised,
 *             exp(-2 pi i k.x/N)); Wh[k] = R_l[k] Vh[k] (complex C x C per mode);
 *             U = (1/N^2) Re of the inverse sum; Z_l = U + W_l V_l + c_l;
 *             V_{l+1} = GELU(Z_l) (exact erf form), none after the last layer
 *   output    F = Q V_L + q: six channels, Re/Im of E_x, E_y, E_z
 *   head      h = e . mean_pixels(V_L) + e0 predicts log(rel-L2 error)
 *   loss      L = mean_b ||F_b - T_b||^2/||T_b||^2 + mean_b (h_b - log(rel_b))^2,
 *             the head trained on a constant trunk; Adam (b1 0.9, b2 0.999, eps 1e-8)
 *
 * Parameters are one flat FP32 vector (the master copy), in this order:
 *   P [C][2S], p [C]; per layer R [m*m][C][C][2] (re, im), W [C][C] (row = output
 *   channel), c [C]; then Q [6][C], q [6], e [C], e0 [1]. Mode index of (ky, kx) is
 *   (ky + m/2) m + (kx + m/2). Kernels read a BF16 copy (FP32 in FP32 mode) that
 *   every update refreshes.
 *
 * Precision: SCW_FNO_BF16 keeps activations and weights in BF16 and runs the DFT
 * contractions on tcgen05 tensor cores (FP32 accumulation in tensor memory);
 * SCW_FNO_FP32 keeps everything in FP32 on SIMT cores, as a test mode.
 *
 * Layouts (all device, row-major, caller-owned):
 *   n       complex64 [B][S][in_grid][in_grid]   (x fastest)
 *   target  complex64 [B][3][N][N]               (E_x, E_y, E_z; x fastest)
 *   field   complex64 [B][3][N][N]
 * Work is asynchronous on `stream` (a cudaStream_t, NULL = legacy default)
 * except where a host output is requested, which synchronises that stream.
 * Handles own their workspaces and free them on destroy. There is no CPU path.
 */
#ifndef SCW_FNO_H
#define SCW_FNO_H

#include <stddef.h>

#include "scw.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scw_fno_s* scw_fno_t;

typedef enum { SCW_FNO_BF16 = 0, SCW_FNO_FP32 = 1 } scw_fno_precision;

typedef struct {
  int width;     /* channels C; this build supports 32 only                      */
  int grid;      /* N: 16, 32 or 64                                             */
  int modes;     /* m: kept frequencies per axis, a multiple of 4 with m <= N    */
  int layers;    /* Fourier layers, 1..8                                        */
  int slices;    /* S input slices (2S input channels), 1..16                   */
  int in_grid;   /* input grid, divides N                                       */
  int batch_max; /* largest batch passed to any call, 1..4096                   */
  scw_fno_precision precision;
  unsigned long long seed; /* initial parameters: uniform draws from a counter-based
                              generator (splitmix64), scale 1/sqrt(fan-in), R 1/C  */
} scw_fno_desc;

/* Validate `desc`, allocate every workspace for batch_max samples and
 * initialise the parameters. INVALID_ARGUMENT / UNSUPPORTED for shapes outside
 * the ranges above, OUT_OF_MEMORY, CUDA (no sm_103 device). */
scw_status scw_surrogate_create(const scw_fno_desc* desc, scw_fno_t* out);
scw_status scw_surrogate_destroy(scw_fno_t fno);

/* Number of FP32 values in the flat parameter vector. */
scw_status scw_surrogate_param_count(scw_fno_t fno, size_t* count);

/* Copy the flat parameters from / to HOST memory (count must equal
 * scw_surrogate_param_count). Setting them resets the Adam moments and step. */
scw_status scw_surrogate_set_params(scw_fno_t fno, const float* host, size_t count);
scw_status scw_surrogate_get_params(scw_fno_t fno, float* host, size_t count);
/* The gradient of the last forward_backward or train_step, HOST copy. */
scw_status scw_surrogate_get_grads(scw_fno_t fno, float* host, size_t count);

/* Loss and gradient of one batch without updating the parameters.
 * loss: HOST float[3] = {L, L_field, L_head}, or NULL (then nothing synchronises). */
scw_status scw_surrogate_forward_backward(scw_fno_t fno, const void* n, const void* target, int B, float* loss,
                                          void* stream);

/* forward_backward followed by one Adam step with learning rate lr. */
scw_status scw_surrogate_train_step(scw_fno_t fno, const void* n, const void* target, int B, float lr, float* loss,
                                    void* stream);

/* Inference: field [B][3][N][N] complex64 (device); est_err [B] (device float,
 * may be NULL) = exp(h + q), q the calibration offset; need_fallback [B]
 * (device uint8, may be NULL) = est_err > threshold. */
scw_status scw_surrogate_infer(scw_fno_t fno, const void* n, int B, void* field, float* est_err,
                               unsigned char* need_fallback, float threshold, void* stream);

/* Split-conformal calibration: given HOST arrays of the head's estimates
 * est[i] (from infer with q = 0, i.e. exp(h)) and the true rel-L2 errors
 * true_err[i] of `count` calibration samples, set q to the
 * ceil((1 - miss)(count + 1))-th smallest log(true_err/est), so that est*exp(q)
 * bounds the true error with probability >= 1 - miss. q_out (HOST, may be NULL)
 * receives q. scw_surrogate_set_offset sets q directly (0 after create). */
scw_status scw_surrogate_calibrate(scw_fno_t fno, const float* est, const float* true_err, int count, float miss,
                                   float* q_out);
scw_status scw_surrogate_set_offset(scw_fno_t fno, float q);

/* Checkpoint / resume of the whole training state: FP32 master parameters, both
 * Adam moments, the Adam step count and the calibration offset q, as one HOST
 * byte blob (a 32-byte header, then three arrays of param_count floats).
 * Loading refreshes the kernels' parameter copies, so the next train_step after
 * a load gives bit-identical parameters to the one the saved handle would have
 * taken. INVALID_ARGUMENT on a size, magic or parameter-count mismatch. */
scw_status scw_surrogate_state_bytes(scw_fno_t fno, size_t* bytes);
scw_status scw_surrogate_save_state(scw_fno_t fno, void* host, size_t bytes);
scw_status scw_surrogate_load_state(scw_fno_t fno, const void* host, size_t bytes);

/* Per-kernel timing: while on, every call records a CUDA event after each of its
 * launches and synchronises its stream at the end; times (ms, summed since the
 * last enable) and algorithmic FLOPs accumulate per kernel family:
 *   dft    truncated-DFT GEMMs (tensor cores in BF16 mode), forward and backward
 *   layer  inverse-DFT + 1x1-convolution GEMMs with their fused epilogues
 *   dw     weight-gradient GEMMs
 *   mix    per-mode complex mixing, forward and backward
 *   other  lift, projection, loss, head, reductions, Adam */
typedef struct {
  int calls;
  double dft_ms, layer_ms, dw_ms, mix_ms, other_ms, total_ms;
  double dft_flops, layer_flops, dw_flops, mix_flops;
} scw_fno_times;
scw_status scw_surrogate_enable_timing(scw_fno_t fno, int on);
scw_status scw_surrogate_get_timings(scw_fno_t fno, scw_fno_times* out);

/* Kernel launches of one train_step / infer call at batch B (for accounting). */
scw_status scw_surrogate_launches(scw_fno_t fno, int* train_step, int* infer);

#ifdef __cplusplus
}
#endif

#endif /* SCW_FNO_H */
