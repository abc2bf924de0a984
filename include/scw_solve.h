/*
 * scw_solve.h -- C ABI of the coupled-wave solve stage on the GPU (the part of
 * arXiv 2404.07293 that precedes field synthesis: Sec. 2.4-2.5 and Sec. 3.1-3.4).
 *
 * From a layered sample and an incident field it computes exactly the inputs of
 * scw_plan_set_layers (include/scw.h): per layer the E-field rows W of the
 * eigenvectors, the eigenvalues gamma and the mode amplitudes alpha, and the
 * exterior amplitudes p_ref, p_trn. Steps, all on the device:
 *   1. Fourier coefficients of n^2 and 1/n^2 per layer (Eq. 11-12, divided by
 *      Nx Ny), as separable DFTs at the order differences only;
 *   2. the convolution matrices Phi, Psi (Sec. 2.5.2) and the two 2M x 2M
 *      off-diagonal blocks of the property matrix D = [[0, A], [B, 0]] (Eq. 21);
 *   3. the eigenmodes of D from the reduced problem (A B) P = P diag(lambda):
 *      gamma = +-sqrt(lambda), eigenvectors [P; +-B P / gamma] (D^2 is block
 *      diagonal, so its 4M-dimensional eigenproblem splits into one of size 2M),
 *      with the forward branch of Sec. 2.5.3 (Im gamma > 0, or real and > 0);
 *      columns scaled to unit 2-norm;
 *   4. per layer the matrices of the field at its top and bottom (Eq. 24-26) and
 *      the connection product K = B_L T_L^-1 ... B_1 T_1^-1 (Eq. 27) by LU solves;
 *   5. the 6M system of Fig. 2 (Eq. 29 and Gauss' law, Eq. 14) for p_ref, p_trn;
 *   6. alpha_1 = T_1^-1 (G_bar R_bar + C_ref p_ref), alpha_l = T_l^-1 B_{l-1} alpha_{l-1};
 *   7. the E_z rows Psi (s_y Q_Bx - s_x Q_By) of W (Eq. 33).
 * The dense factorisations use cuSOLVER (geev, getrf/getrs) and the dense
 * products cuBLAS, in FP64 (complex128); the assembly, mode, boundary and output
 * steps are the library's own kernels. The eigenvector basis (scale, order and,
 * for repeated eigenvalues, the basis of the eigenspace) is not unique, so W and
 * alpha are not unique either; the field they synthesise, gamma as a set and
 * p_ref, p_trn are.
 *
 * Conventions are those of include/scw.h (orders, s_x = lambda u / X, s_z
 * branch, DEVICE/HOST pointers, status codes, thread-local messages).
 */
#ifndef SCW_SOLVE_H
#define SCW_SOLVE_H

#include "scw.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scw_solver_s* scw_solver_t;

typedef struct {
  int U, V, L;              /* orders along x and y (M = U V), layers                              */
  double lambda, X, Y;      /* vacuum wavelength and lateral period                                */
  const double* z_bounds;   /* HOST [L+1], strictly ascending                                       */
  int Nx, Ny;               /* sample grid of every layer: voxel (p, q) sits at (p X/Nx, q Y/Ny);
                               Nx >= 2U - 1 and Ny >= 2V - 1 (order differences must not alias)   */
  double n_top;             /* real refractive index above the sample                              */
  double n_bot_re, n_bot_im;/* refractive index below the sample                                    */
  double z_inc;             /* plane at which p_inc is given (the paper's z-bar)                   */
} scw_solve_desc;

typedef struct {
  int calls;
  double fourier_ms;        /* step 1                                                               */
  double modes_ms;          /* steps 2-3 (assembly, A B, eigendecompositions, B P, mode scaling)    */
  double connect_ms;        /* step 4 (top/bottom matrices, LU factors, K)                          */
  double system_ms;         /* step 5                                                               */
  double alpha_ms;          /* step 6                                                               */
  double erows_ms;          /* step 7 and the W output                                              */
  double total_ms;
} scw_solve_times;

/* Validates the descriptor and allocates the workspace (about
 * L (2 (4M)^2 + 5 (2M)^2 + 2 M^2) 16 bytes plus 3 (6M)^2 16 bytes). Synchronous. */
scw_status scw_solver_create(const scw_solve_desc* desc, scw_solver_t* out);
scw_status scw_solver_destroy(scw_solver_t solver);

/* Incident amplitudes from a sampled image of one transverse component (Eq. 4 on
 * the pixel grid, divided by Nx Ny; Gauss' law, Eq. 14, gives p_z):
 *   image  DEVICE complex128 [Ny][Nx] (the x component if pol == 0, y if pol == 1)
 *   p_inc  DEVICE complex128 [3][M] (output)
 * SCW_ERR_NUMERIC if light falls in a grazing order (s_z(n_top) = 0). Synchronises. */
scw_status scw_solver_incident(scw_solver_t solver, const void* image, int pol, void* p_inc, void* stream);

/* The solve. Inputs: n DEVICE complex128 [L][Ny][Nx] (refractive index per voxel),
 * p_inc DEVICE complex128 [3][M]. Outputs (DEVICE, caller-owned):
 *   W      complex64  [L][3M][4M]   rows c M + m (c = x, y, z), columns = modes
 *   gamma  complex128 [L][4M]       modes [0, 2M) forward, [2M, 4M) backward (= -forward)
 *   alpha  complex128 [L][4M]
 *   p_ref, p_trn complex128 [3][M]
 * Synchronises the stream. SCW_ERR_NUMERIC when an eigendecomposition does not
 * converge, an LU factor is singular or a mode has gamma = 0 (a grazing wave). */
scw_status scw_solve(scw_solver_t solver, const void* n, const void* p_inc, void* W, void* gamma, void* alpha,
                     void* p_ref, void* p_trn, void* stream);

/* Per-step GPU times of the last scw_solve (CUDA events on its stream). */
scw_status scw_solver_get_times(scw_solver_t solver, scw_solve_times* t);

#ifdef __cplusplus
}
#endif

#endif /* SCW_SOLVE_H */
