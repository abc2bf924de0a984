// Coupled-wave solve stage on the GPU (include/scw_solve.h): from the layered
// sample and the incident amplitudes to W, gamma, alpha and p_ref, p_trn.
//
// Matrices that go through cuBLAS / cuSOLVER are column-major ((i, j) at j ld + i);
// the outputs keep the row-major layouts of include/scw.h. Everything is FP64
// (complex128) until the W output, which is complex64 like scw_plan_set_layers'.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/scw_solve.h"
#include "scw_internal.cuh"

namespace scw {
namespace {

constexpr double kTau = 1e-10;  // forward-mode tolerance of Sec. 2.5.3 (|Im gamma| <= tau |gamma| counts as real)

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zs(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zinv(double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2(b.x / d, -b.y / d);
}
// principal square root (Re >= 0): t = sqrt((|z| + |Re z|) / 2)
__device__ __forceinline__ double2 zsqrt(double2 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}
// exp(i z)
__device__ __forceinline__ double2 zexpi(double2 z) {
  double s, c;
  sincos(z.x, &s, &c);
  const double m = exp(-z.y);
  return make_double2(m * c, m * s);
}

struct OrderGeom {
  int U, V, M;
  double sxs, sys;  // lambda / X, lambda / Y
  __device__ __forceinline__ int u(int m) const { return m % U - U / 2; }
  __device__ __forceinline__ int v(int m) const { return m / U - V / 2; }
  __device__ __forceinline__ double sx(int m) const { return sxs * u(m); }
  __device__ __forceinline__ double sy(int m) const { return sys * v(m); }
};

// Step 1a: row DFT of n^2 (t = 0) and 1/n^2 (t = 1) at the order differences du in [-(U-1), U-1]:
// R[l][t][q][du] = sum_p val[l][q][p] e^{-2 pi i du p / Nx} (twiddles wx[k] = e^{-2 pi i k / Nx}).
__global__ void row_dft_kernel(const double2* __restrict__ n, int L, int Nx, int Ny, int U,
                               const double2* __restrict__ wx, double2* __restrict__ R) {
  const int nu = 2 * U - 1;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)L * 2 * Ny * nu) return;
  const int idu = (int)(i % nu);
  size_t r = i / nu;
  const int q = (int)(r % Ny);
  r /= Ny;
  const int t = (int)(r % 2), l = (int)(r / 2);
  const int dp = ((idu - (U - 1)) % Nx + Nx) % Nx;
  const double2* row = n + ((size_t)l * Ny + q) * Nx;
  double2 acc = make_double2(0.0, 0.0);
  int k = 0;  // (dp p) mod Nx
  for (int p = 0; p < Nx; ++p) {
    const double2 e = zmul(row[p], row[p]);
    const double2 val = t ? zinv(e) : e;
    acc = zadd(acc, zmul(val, wx[k]));
    k += dp;
    if (k >= Nx) k -= Nx;
  }
  R[i] = acc;
}

// Step 1b: tab[l][t][dv][du] = (1 / (Nx Ny)) sum_q R[l][t][q][du] e^{-2 pi i dv q / Ny} (Eq. 11-12).
__global__ void col_dft_kernel(const double2* __restrict__ R, int L, int Nx, int Ny, int U, int V,
                               const double2* __restrict__ wy, double2* __restrict__ tab) {
  const int nu = 2 * U - 1, nv = 2 * V - 1;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)L * 2 * nv * nu) return;
  const int idu = (int)(i % nu);
  size_t r = i / nu;
  const int idv = (int)(r % nv);
  const int lt = (int)(r / nv);
  const int dq = ((idv - (V - 1)) % Ny + Ny) % Ny;
  const double2* col = R + (size_t)lt * Ny * nu + idu;
  double2 acc = make_double2(0.0, 0.0);
  int k = 0;
  for (int q = 0; q < Ny; ++q) {
    acc = zadd(acc, zmul(col[(size_t)q * nu], wy[k]));
    k += dq;
    if (k >= Ny) k -= Ny;
  }
  tab[i] = zs(acc, 1.0 / ((double)Nx * Ny));
}

// Step 2: the off-diagonal blocks of D = [[0, A], [B, 0]] (Eq. 21, reading R3 of the oracle's
// notes: lower block rows re-derived), with Phi[i][j] = phi(u_i - u_j, v_i - v_j), Psi from 1/n^2:
//   A = [[Sx Psi Sy, I - Sx Psi Sx], [Sy Psi Sy - I, -Sy Psi Sx]]
//   B = [[-Sx Sy, Sx^2 - Phi], [Phi - Sy^2, Sy Sx]]
// A, B: [L] column-major 2M x 2M; Psi: [L] column-major M x M.
__global__ void assemble_kernel(const double2* __restrict__ tab, int L, OrderGeom g, double2* __restrict__ A,
                                double2* __restrict__ B, double2* __restrict__ Psi) {
  const int M = g.M, n = 2 * M;
  const int nu = 2 * g.U - 1, nv = 2 * g.V - 1;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)L * n * n) return;
  const int r = (int)(idx % n);
  size_t rest = idx / n;
  const int c = (int)(rest % n), l = (int)(rest / n);
  const int bi = r / M, i = r - bi * M, bj = c / M, j = c - bj * M;
  const int du = g.u(i) - g.u(j) + g.U - 1, dv = g.v(i) - g.v(j) + g.V - 1;
  const double2* te = tab + (size_t)(l * 2) * nv * nu;
  const double2 phi = te[(size_t)dv * nu + du];
  const double2 psi = te[(size_t)nv * nu + (size_t)dv * nu + du];
  const double sxi = g.sx(i), syi = g.sy(i), sxj = g.sx(j), syj = g.sy(j);
  const double dlt = (i == j) ? 1.0 : 0.0;
  double2 a, b;
  if (bi == 0 && bj == 0) {
    a = zs(psi, sxi * syj);
    b = make_double2(-sxi * syi * dlt, 0.0);
  } else if (bi == 0) {
    a = make_double2(dlt - sxi * sxj * psi.x, -sxi * sxj * psi.y);
    b = make_double2(sxi * sxi * dlt - phi.x, -phi.y);
  } else if (bj == 0) {
    a = make_double2(syi * syj * psi.x - dlt, syi * syj * psi.y);
    b = make_double2(phi.x - syi * syi * dlt, phi.y);
  } else {
    a = zs(psi, -syi * sxj);
    b = make_double2(syi * sxi * dlt, 0.0);
  }
  A[idx] = a;
  B[idx] = b;
  if (bi == 0 && bj == 0) Psi[((size_t)l * M + j) * M + i] = psi;
}

// Step 3 (after eig(A B) and B P): per layer l and forward mode j, gamma = sqrt(lambda) on the
// forward branch, the column scale s (unit 2-norm of [P_j; B P_j / gamma]), s / gamma and
// e = exp(i k gamma d). Block per (j, l).
__global__ void modes_kernel(const double2* __restrict__ lam, const double2* __restrict__ P,
                             const double2* __restrict__ BP, int M, double k, const double* __restrict__ thick,
                             double2* __restrict__ gamma_out, double2* __restrict__ gam, double* __restrict__ sc,
                             double2* __restrict__ sg, double2* __restrict__ ex, int* __restrict__ err) {
  const int n = 2 * M, j = blockIdx.x, l = blockIdx.y;
  const size_t cj = ((size_t)l * n + j) * n;  // column j of layer l
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 p = P[cj + i], q = BP[cj + i];
    a += p.x * p.x + p.y * p.y;
    b += q.x * q.x + q.y * q.y;
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double2 w = zsqrt(lam[(size_t)l * n + j]);
  const double aw = hypot(w.x, w.y);
  if (w.y < -kTau * aw) w = make_double2(-w.x, -w.y);  // forward: Im > 0, or (nearly) real and Re >= 0
  if (!(aw > 0.0) || !isfinite(aw)) {
    atomicOr(err, 1);
    w = make_double2(1.0, 0.0);
  }
  const double g2 = w.x * w.x + w.y * w.y;
  const double s = 1.0 / sqrt(red[0][0] + red[1][0] / g2);
  const size_t o = (size_t)l * n + j;
  gam[o] = w;
  sc[o] = s;
  sg[o] = zs(zinv(w), s);
  ex[o] = zexpi(zs(w, k * thick[l]));
  gamma_out[(size_t)l * 2 * n + j] = w;
  gamma_out[(size_t)l * 2 * n + n + j] = make_double2(-w.x, -w.y);
}

// Step 4a: T_l, B_l (Eq. 24-26, reading R6), column-major 4M x 4M. Mode column c: j = c mod 2M,
// backward when c >= 2M; its eigenvector is s_j [P_j; +-B P_j / gamma_j].
//   T = [Q_f, Q_b diag(e)],  B = [Q_f diag(e), Q_b],  e_j = exp(i k gamma_j d)  (exp(-i k gamma_b d) = e_j)
__global__ void top_bottom_kernel(const double2* __restrict__ P, const double2* __restrict__ BP,
                                  const double* __restrict__ sc, const double2* __restrict__ sg,
                                  const double2* __restrict__ ex, int M, int L, double2* __restrict__ T,
                                  double2* __restrict__ Bm) {
  const int n = 2 * M, N = 4 * M;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)L * N * N) return;
  const int r = (int)(idx % N);
  const size_t rest = idx / N;
  const int c = (int)(rest % N), l = (int)(rest / N);
  const bool back = c >= n;
  const int j = back ? c - n : c;
  const size_t o = (size_t)l * n + j;
  const size_t cj = o * n;
  double2 q;
  if (r < n) {
    q = zs(P[cj + r], sc[o]);
  } else {
    q = zmul(BP[cj + r - n], sg[o]);
    if (back) q = make_double2(-q.x, -q.y);
  }
  const double2 qe = zmul(q, ex[o]);
  T[idx] = back ? qe : q;
  Bm[idx] = back ? q : qe;
}

// Step 7a: G_l = diag(s_y) Q_Bx - diag(s_x) Q_By over the forward columns (column-major M x 2M);
// the backward columns' G is -G (their B part is negated).
__global__ void erows_g_kernel(const double2* __restrict__ BP, const double2* __restrict__ sg, OrderGeom g, int L,
                               double2* __restrict__ G) {
  const int M = g.M, n = 2 * M;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)L * M * n) return;
  const int i = (int)(idx % M);
  const size_t rest = idx / M;
  const int j = (int)(rest % n), l = (int)(rest / n);
  const size_t o = (size_t)l * n + j;
  const double2 qbx = zmul(BP[o * n + i], sg[o]);
  const double2 qby = zmul(BP[o * n + M + i], sg[o]);
  G[idx] = zsub(zs(qbx, g.sy(i)), zs(qby, g.sx(i)));
}

// Step 7b: W[l] row-major complex64 [3M][4M]: rows [0, 2M) = s_j P rows (P_x, P_y parts of every
// mode), rows [2M, 3M) = E_z = Psi G (forward) and -Psi G (backward) (Eq. 33).
__global__ void w_out_kernel(const double2* __restrict__ P, const double* __restrict__ sc,
                             const double2* __restrict__ Ez, int M, int L, float2* __restrict__ W) {
  const int n = 2 * M, N = 4 * M;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)L * 3 * M * N) return;
  const int c = (int)(idx % N);
  const size_t rest = idx / N;
  const int r = (int)(rest % (3 * M)), l = (int)(rest / (3 * M));
  const bool back = c >= n;
  const int j = back ? c - n : c;
  const size_t o = (size_t)l * n + j;
  double2 v;
  if (r < n) {
    v = zs(P[o * n + r], sc[o]);
  } else {
    v = Ez[(size_t)l * M * n + (size_t)j * M + (r - n)];
    if (back) v = make_double2(-v.x, -v.y);
  }
  W[idx] = make_float2((float)v.x, (float)v.y);
}

// R = p_to_r(s_x, s_y, s_z) p (Eq. 28, reading R4) for one wave: [p_x; p_y; -s_z p_y + s_y p_z; s_z p_x - s_x p_z]
__device__ __forceinline__ double2 p_to_r_row(int r, int M, OrderGeom g, const double2* sz, double sz_sign,
                                              const double2* p) {
  const int blk = r / M, m = r - blk * M;
  const double2 px = p[m], py = p[M + m], pz = p[2 * M + m];
  const double2 s = zs(sz[m], sz_sign);
  switch (blk) {
    case 0: return px;
    case 1: return py;
    case 2: return zadd(zs(zmul(s, py), -1.0), zs(pz, g.sy(m)));
    default: return zsub(zmul(s, px), zs(pz, g.sx(m)));
  }
}

// Step 5 inputs: R_bar = G_bar o (C(s_z,top) p_inc) (reading R10: G_bar repeats over the four blocks).
__global__ void rbar_kernel(const double2* __restrict__ p_inc, const double2* __restrict__ sz_t, OrderGeom g,
                            double k, double dz0, double2* __restrict__ rbar) {
  const int M = g.M;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 4 * M) return;
  const int m = r % M;
  const double2 gb = zexpi(zs(sz_t[m], k * dz0));
  rbar[r] = zmul(gb, p_to_r_row(r, M, g, sz_t, 1.0, p_inc));
}

// Step 5: the 6M system (column-major), rows [0, 4M): [-K C_ref | C_trn] (Eq. 29), then Gauss'
// law for the reflected and the transmitted wave (Eq. 14). C_ref uses s_z = -s_z(top) (the
// reflected wave travels towards -z), C_trn s_z = s_z(bottom). (K C_ref) needs two columns of K
// per column of C_ref.
__global__ void system_kernel(const double2* __restrict__ K, const double2* __restrict__ sz_t,
                              const double2* __restrict__ sz_b, OrderGeom g, double2* __restrict__ A6) {
  const int M = g.M, N4 = 4 * M, N6 = 6 * M;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)N6 * N6) return;
  const int r = (int)(idx % N6), c = (int)(idx / N6);
  double2 v = make_double2(0.0, 0.0);
  if (r < N4) {
    if (c < 3 * M) {
      const int blk = c / M, m = c - blk * M;
      const double2 sz = make_double2(-sz_t[m].x, -sz_t[m].y);
      const double2* Kc = K + r;  // K[r][col] at col N4 + r
      double2 kc;
      if (blk == 0) kc = zadd(Kc[(size_t)m * N4], zmul(sz, Kc[(size_t)(3 * M + m) * N4]));
      else if (blk == 1) kc = zsub(Kc[(size_t)(M + m) * N4], zmul(sz, Kc[(size_t)(2 * M + m) * N4]));
      else kc = zsub(zs(Kc[(size_t)(2 * M + m) * N4], g.sy(m)), zs(Kc[(size_t)(3 * M + m) * N4], g.sx(m)));
      v = make_double2(-kc.x, -kc.y);
    } else {
      const int cc = c - 3 * M, blk = cc / M, m = cc - blk * M;
      const int rb = r / M, rm = r - rb * M;
      if (rm == m) {
        const double2 sz = sz_b[m];
        if (blk == 0) v = rb == 0 ? make_double2(1.0, 0.0) : (rb == 3 ? sz : v);
        else if (blk == 1) v = rb == 1 ? make_double2(1.0, 0.0) : (rb == 2 ? make_double2(-sz.x, -sz.y) : v);
        else v = rb == 2 ? make_double2(g.sy(m), 0.0) : (rb == 3 ? make_double2(-g.sx(m), 0.0) : v);
      }
    }
  } else if (r < 5 * M) {
    const int i = r - N4;
    if (c == i) v = make_double2(g.sx(i), 0.0);
    else if (c == M + i) v = make_double2(g.sy(i), 0.0);
    else if (c == 2 * M + i) v = make_double2(-sz_t[i].x, -sz_t[i].y);
  } else {
    const int i = r - 5 * M;
    if (c == 3 * M + i) v = make_double2(g.sx(i), 0.0);
    else if (c == 4 * M + i) v = make_double2(g.sy(i), 0.0);
    else if (c == 5 * M + i) v = sz_b[i];
  }
  A6[idx] = v;
}

// Step 6 input: R_bar + C_ref p_ref.
__global__ void alpha1_rhs_kernel(const double2* __restrict__ rbar, const double2* __restrict__ p_ref,
                                  const double2* __restrict__ sz_t, OrderGeom g, double2* __restrict__ y) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 4 * g.M) return;
  y[r] = zadd(rbar[r], p_to_r_row(r, g.M, g, sz_t, -1.0, p_ref));
}

__global__ void identity_kernel(double2* __restrict__ X, int N) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * N) return;
  X[idx] = make_double2((idx % N) == (idx / N) ? 1.0 : 0.0, 0.0);
}

__global__ void copy_z_kernel(const double2* __restrict__ src, double2* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

// Incident amplitudes (Eq. 4 on the pixel grid, reading R11): proj_m = (1/(Nx Ny)) sum image e^{-2 pi i
// (u p/Nx + v q/Ny)}; the image is the x (pol 0) or y (pol 1) component; p_z = -(s_x p_x + s_y p_y) / s_z.
__global__ void incident_kernel(const double2* __restrict__ img, int Nx, int Ny, int pol, OrderGeom g,
                                const double2* __restrict__ wx, const double2* __restrict__ wy,
                                const double2* __restrict__ sz_t, double2* __restrict__ p, int* __restrict__ err) {
  const int m = blockIdx.x;
  const int M = g.M;
  const int du = ((g.u(m) % Nx) + Nx) % Nx, dv = ((g.v(m) % Ny) + Ny) % Ny;
  __shared__ double2 red[256];
  __shared__ double mag[256];
  double2 acc = make_double2(0.0, 0.0);
  double am = 0.0;
  for (int i = threadIdx.x; i < Nx * Ny; i += blockDim.x) {
    const int q = i / Nx, pp = i - q * Nx;
    const int kx = (int)(((long long)du * pp) % Nx), ky = (int)(((long long)dv * q) % Ny);
    acc = zadd(acc, zmul(img[i], zmul(wx[kx], wy[ky])));
    am += hypot(img[i].x, img[i].y);
  }
  red[threadIdx.x] = acc;
  mag[threadIdx.x] = am;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[threadIdx.x] = zadd(red[threadIdx.x], red[threadIdx.x + s]);
      mag[threadIdx.x] += mag[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double inv_n = 1.0 / ((double)Nx * Ny);
  const double2 proj = zs(red[0], inv_n);
  const double noise = 1e-13 * mag[0] * inv_n;  // DFT rounding: an order with |p| below it carries no light
  const double2 px = pol == 0 ? proj : make_double2(0.0, 0.0);
  const double2 py = pol == 0 ? make_double2(0.0, 0.0) : proj;
  const double2 num = zadd(zs(px, g.sx(m)), zs(py, g.sy(m)));
  const double2 sz = sz_t[m];
  double2 pz = make_double2(0.0, 0.0);
  if (sz.x == 0.0 && sz.y == 0.0) {
    if (hypot(num.x, num.y) > noise) atomicOr(err, 2);
  } else {
    pz = zs(zmul(num, zinv(sz)), -1.0);
  }
  p[m] = px;
  p[M + m] = py;
  p[2 * M + m] = pz;
}

unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

std::complex<double> s_z_host(std::complex<double> n, double sx, double sy) {
  std::complex<double> w = std::sqrt(n * n - sx * sx - sy * sy);
  if (w.imag() < 0 || (w.imag() == 0 && w.real() < 0)) w = -w;
  return w;
}

}  // namespace
}  // namespace scw

using namespace scw;

struct scw_solver_s {
  int U = 0, V = 0, L = 0, M = 0, Nx = 0, Ny = 0;
  double lambda = 0, X = 0, Y = 0, n_top = 1, z_inc = 0;
  std::complex<double> n_bot{1.0, 0.0};
  std::vector<double> zb;
  OrderGeom geom{};
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
  cusolverDnParams_t params = nullptr;
  // device workspace
  double2 *wx = nullptr, *wy = nullptr, *R = nullptr, *tab = nullptr;
  double2 *A = nullptr, *B = nullptr, *C = nullptr, *P = nullptr, *BP = nullptr, *lam = nullptr;
  double2 *Psi = nullptr, *G = nullptr, *Ez = nullptr;
  double2 *gam = nullptr, *sg = nullptr, *ex = nullptr;
  double* sc = nullptr;
  double* thick = nullptr;
  double2 *T = nullptr, *Bm = nullptr, *K = nullptr, *Xm = nullptr;
  double2 *A6 = nullptr, *x6 = nullptr, *rbar = nullptr;
  double2 *sz_t = nullptr, *sz_b = nullptr;
  int* ipiv = nullptr;     // [L][4M] then [6M]
  int* info = nullptr;     // [L] geev, [L] getrf, [1] system, [1] getrs
  int* err = nullptr;
  void* dwork = nullptr;
  size_t dwork_bytes = 0;
  std::vector<unsigned char> hwork;
  cudaEvent_t ev[7] = {};
  bool timed = false;
  // the per-layer eigendecompositions are independent (Sec. 4.3, parallelise across L): each
  // worker has its own host thread, cuSOLVER handle, stream and workspace
  struct EigWorker {
    cusolverDnHandle_t h = nullptr;
    cusolverDnParams_t params = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    void* dwork = nullptr;
    std::vector<unsigned char> hwork;
  };
  std::vector<EigWorker> eig;
  size_t geev_dbytes = 0;
  cudaEvent_t ev_ready = nullptr;
};

static void solver_free(scw_solver_t s) {
  if (!s) return;
  void* ptrs[] = {s->wx, s->wy, s->R, s->tab, s->A, s->B, s->C, s->P, s->BP, s->lam, s->Psi, s->G, s->Ez, s->gam,
                  s->sg, s->ex, s->sc, s->thick, s->T, s->Bm, s->K, s->Xm, s->A6, s->x6, s->rbar, s->sz_t, s->sz_b,
                  s->ipiv, s->info, s->err, s->dwork};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  for (auto& w : s->eig) {
    if (w.dwork) cudaFree(w.dwork);
    if (w.done) cudaEventDestroy(w.done);
    if (w.st) cudaStreamDestroy(w.st);
    if (w.params) cusolverDnDestroyParams(w.params);
    if (w.h) cusolverDnDestroy(w.h);
  }
  if (s->ev_ready) cudaEventDestroy(s->ev_ready);
  if (s->params) cusolverDnDestroyParams(s->params);
  if (s->sol) cusolverDnDestroy(s->sol);
  if (s->blas) cublasDestroy(s->blas);
  delete s;
}

template <typename T>
static cudaError_t zalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

static scw_status blas_error(cublasStatus_t st, const char* what) {
  return set_error(SCW_ERR_CUDA, std::string(what) + " failed (cuBLAS status " + std::to_string((int)st) + ")");
}
static scw_status solver_error(cusolverStatus_t st, const char* what) {
  return set_error(SCW_ERR_CUDA, std::string(what) + " failed (cuSOLVER status " + std::to_string((int)st) + ")");
}

#define SCW_CU(x)                                                        \
  do {                                                                   \
    cudaError_t e_ = (x);                                                \
    if (e_ != cudaSuccess) return cuda_error(e_, #x);                    \
  } while (0)
#define SCW_BL(x)                                                        \
  do {                                                                   \
    cublasStatus_t b_ = (x);                                             \
    if (b_ != CUBLAS_STATUS_SUCCESS) return blas_error(b_, #x);          \
  } while (0)
#define SCW_SV(x)                                                        \
  do {                                                                   \
    cusolverStatus_t v_ = (x);                                           \
    if (v_ != CUSOLVER_STATUS_SUCCESS) return solver_error(v_, #x);      \
  } while (0)

extern "C" {

scw_status scw_solver_create(const scw_solve_desc* d, scw_solver_t* out) {
  if (!d || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "desc and out are required");
  *out = nullptr;
  if (d->U < 1 || d->V < 1 || d->L < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "U, V and L must be >= 1");
  if ((long long)d->U * d->V > 2048) return set_error(SCW_ERR_UNSUPPORTED, "U V above 2048");
  if (!(d->lambda > 0) || !(d->X > 0) || !(d->Y > 0))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "lambda, X and Y must be positive");
  if (d->Nx < 2 * d->U - 1 || d->Ny < 2 * d->V - 1 || d->Nx > 8192 || d->Ny > 8192)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "Nx >= 2U - 1 and Ny >= 2V - 1 (at most 8192) are required");
  if (!d->z_bounds) return set_error(SCW_ERR_INVALID_ARGUMENT, "z_bounds is required");
  for (int l = 0; l < d->L; ++l)
    if (!(d->z_bounds[l + 1] > d->z_bounds[l]))
      return set_error(SCW_ERR_INVALID_ARGUMENT, "z_bounds must be strictly ascending");
  if (!(d->n_top > 0)) return set_error(SCW_ERR_INVALID_ARGUMENT, "n_top must be positive");
  scw_status st = check_device();
  if (st != SCW_OK) return st;
  scw_solver_t s = new (std::nothrow) scw_solver_s();
  if (!s) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->U = d->U; s->V = d->V; s->L = d->L; s->M = d->U * d->V; s->Nx = d->Nx; s->Ny = d->Ny;
  s->lambda = d->lambda; s->X = d->X; s->Y = d->Y; s->n_top = d->n_top; s->z_inc = d->z_inc;
  s->n_bot = {d->n_bot_re, d->n_bot_im};
  s->zb.assign(d->z_bounds, d->z_bounds + d->L + 1);
  s->geom = OrderGeom{d->U, d->V, s->M, d->lambda / d->X, d->lambda / d->Y};
  const size_t M = s->M, L = s->L, n = 2 * M, N = 4 * M, nu = 2 * d->U - 1, nv = 2 * d->V - 1;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(zalloc(&s->wx, d->Nx)); A(zalloc(&s->wy, d->Ny));
  A(zalloc(&s->R, L * 2 * d->Ny * nu)); A(zalloc(&s->tab, L * 2 * nv * nu));
  A(zalloc(&s->A, L * n * n)); A(zalloc(&s->B, L * n * n)); A(zalloc(&s->C, L * n * n));
  A(zalloc(&s->P, L * n * n)); A(zalloc(&s->BP, L * n * n)); A(zalloc(&s->lam, L * n));
  A(zalloc(&s->Psi, L * M * M)); A(zalloc(&s->G, L * M * n)); A(zalloc(&s->Ez, L * M * n));
  A(zalloc(&s->gam, L * n)); A(zalloc(&s->sg, L * n)); A(zalloc(&s->ex, L * n)); A(zalloc(&s->sc, L * n));
  A(zalloc(&s->thick, L));
  A(zalloc(&s->T, L * N * N)); A(zalloc(&s->Bm, L * N * N)); A(zalloc(&s->K, N * N)); A(zalloc(&s->Xm, N * N));
  A(zalloc(&s->A6, 36 * M * M)); A(zalloc(&s->x6, 6 * M)); A(zalloc(&s->rbar, 4 * M));
  A(zalloc(&s->sz_t, M)); A(zalloc(&s->sz_b, M));
  A(zalloc(&s->ipiv, L * N + 6 * M)); A(zalloc(&s->info, 2 * L + 2)); A(zalloc(&s->err, 1));
  for (auto& ev : s->ev) A(cudaEventCreate(&ev));
  if (e != cudaSuccess) {
    solver_free(s);
    return e == cudaErrorMemoryAllocation ? set_error(SCW_ERR_OUT_OF_MEMORY, "solver workspace does not fit")
                                          : cuda_error(e, "solver workspace");
  }
  // twiddles e^{-2 pi i k / N} and the exterior s_z (Eq. 2, decaying branch)
  std::vector<double2> wx(d->Nx), wy(d->Ny), szt(M), szb(M);
  for (int k = 0; k < d->Nx; ++k) {
    const double a = -2.0 * M_PI * k / d->Nx;
    wx[k] = make_double2(std::cos(a), std::sin(a));
  }
  for (int k = 0; k < d->Ny; ++k) {
    const double a = -2.0 * M_PI * k / d->Ny;
    wy[k] = make_double2(std::cos(a), std::sin(a));
  }
  for (size_t m = 0; m < M; ++m) {
    const int u = (int)(m % d->U) - d->U / 2, v = (int)(m / d->U) - d->V / 2;
    const double sx = d->lambda * u / d->X, sy = d->lambda * v / d->Y;
    const auto a = s_z_host({d->n_top, 0.0}, sx, sy), b = s_z_host(s->n_bot, sx, sy);
    szt[m] = make_double2(a.real(), a.imag());
    szb[m] = make_double2(b.real(), b.imag());
  }
  std::vector<double> th(L);
  for (size_t l = 0; l < L; ++l) th[l] = s->zb[l + 1] - s->zb[l];
  A(cudaMemcpy(s->wx, wx.data(), wx.size() * sizeof(double2), cudaMemcpyHostToDevice));
  A(cudaMemcpy(s->wy, wy.data(), wy.size() * sizeof(double2), cudaMemcpyHostToDevice));
  A(cudaMemcpy(s->sz_t, szt.data(), M * sizeof(double2), cudaMemcpyHostToDevice));
  A(cudaMemcpy(s->sz_b, szb.data(), M * sizeof(double2), cudaMemcpyHostToDevice));
  A(cudaMemcpy(s->thick, th.data(), L * sizeof(double), cudaMemcpyHostToDevice));
  if (e != cudaSuccess) {
    solver_free(s);
    return cuda_error(e, "solver tables");
  }
  if (cublasCreate(&s->blas) != CUBLAS_STATUS_SUCCESS || cusolverDnCreate(&s->sol) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&s->params) != CUSOLVER_STATUS_SUCCESS) {
    solver_free(s);
    return set_error(SCW_ERR_CUDA, "creating the cuBLAS / cuSOLVER handles failed");
  }
  // workspace: the largest of geev (2M), getrf (4M) and getrf (6M)
  size_t geev_d = 0, geev_h = 0;
  cusolverStatus_t cs = cusolverDnXgeev_bufferSize(s->sol, s->params, CUSOLVER_EIG_MODE_NOVECTOR,
                                                   CUSOLVER_EIG_MODE_VECTOR, (int64_t)n, CUDA_C_64F, s->C,
                                                   (int64_t)n, CUDA_C_64F, s->lam, CUDA_C_64F, nullptr, 1,
                                                   CUDA_C_64F, s->P, (int64_t)n, CUDA_C_64F, &geev_d, &geev_h);
  int lw4 = 0, lw6 = 0;
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverDnZgetrf_bufferSize(s->sol, (int)N, (int)N, reinterpret_cast<cuDoubleComplex*>(s->T), (int)N, &lw4);
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverDnZgetrf_bufferSize(s->sol, (int)(6 * M), (int)(6 * M), reinterpret_cast<cuDoubleComplex*>(s->A6),
                                     (int)(6 * M), &lw6);
  if (cs != CUSOLVER_STATUS_SUCCESS) {
    solver_free(s);
    return solver_error(cs, "workspace query");
  }
  s->dwork_bytes = std::max({(size_t)lw4 * sizeof(double2), (size_t)lw6 * sizeof(double2), (size_t)256});
  if (cudaMalloc(&s->dwork, s->dwork_bytes) != cudaSuccess) {
    solver_free(s);
    return set_error(SCW_ERR_OUT_OF_MEMORY, "solver workspace does not fit");
  }
  s->geev_dbytes = std::max<size_t>(geev_d, 256);
  s->eig.resize((size_t)std::min(d->L, 8));
  bool ok = cudaEventCreateWithFlags(&s->ev_ready, cudaEventDisableTiming) == cudaSuccess;
  for (auto& w : s->eig) {
    ok = ok && cusolverDnCreate(&w.h) == CUSOLVER_STATUS_SUCCESS &&
         cusolverDnCreateParams(&w.params) == CUSOLVER_STATUS_SUCCESS &&
         cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) == cudaSuccess &&
         cusolverDnSetStream(w.h, w.st) == CUSOLVER_STATUS_SUCCESS &&
         cudaMalloc(&w.dwork, s->geev_dbytes) == cudaSuccess;
    if (ok) w.hwork.resize(std::max<size_t>(geev_h, 1));
  }
  if (!ok) {
    solver_free(s);
    return set_error(SCW_ERR_CUDA, "creating the eigensolver workers failed");
  }
  *out = s;
  return SCW_OK;
}

scw_status scw_solver_destroy(scw_solver_t s) {
  solver_free(s);
  return SCW_OK;
}

scw_status scw_solver_incident(scw_solver_t s, const void* image, int pol, void* p_inc, void* stream) {
  if (!s || !image || !p_inc) return set_error(SCW_ERR_INVALID_ARGUMENT, "solver, image and p_inc are required");
  if (pol != 0 && pol != 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "pol must be 0 (x) or 1 (y)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SCW_CU(cudaMemsetAsync(s->err, 0, sizeof(int), st));
  incident_kernel<<<s->M, 256, 0, st>>>(static_cast<const double2*>(image), s->Nx, s->Ny, pol, s->geom, s->wx,
                                        s->wy, s->sz_t, static_cast<double2*>(p_inc), s->err);
  SCW_CU(cudaGetLastError());
  int herr = 0;
  SCW_CU(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SCW_CU(cudaStreamSynchronize(st));
  if (herr) return set_error(SCW_ERR_NUMERIC, "incident light in a grazing order (s_z = 0) has no p_z");
  return SCW_OK;
}

scw_status scw_solve(scw_solver_t s, const void* n_vol, const void* p_inc_v, void* W_v, void* gamma_v,
                     void* alpha_v, void* p_ref_v, void* p_trn_v, void* stream) {
  if (!s || !n_vol || !p_inc_v || !W_v || !gamma_v || !alpha_v || !p_ref_v || !p_trn_v)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "solver and every buffer are required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SCW_BL(cublasSetStream(s->blas, st));
  SCW_SV(cusolverDnSetStream(s->sol, st));
  const int M = s->M, L = s->L, n = 2 * M, N = 4 * M, N6 = 6 * M;
  const int nu = 2 * s->U - 1, nv = 2 * s->V - 1;
  const double k = 2.0 * M_PI / s->lambda;
  const double2* nv_in = static_cast<const double2*>(n_vol);
  const double2* p_inc = static_cast<const double2*>(p_inc_v);
  double2* gamma_out = static_cast<double2*>(gamma_v);
  double2* alpha = static_cast<double2*>(alpha_v);
  auto Z = [](void* q) { return reinterpret_cast<cuDoubleComplex*>(q); };
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  SCW_CU(cudaMemsetAsync(s->err, 0, sizeof(int), st));
  SCW_CU(cudaMemsetAsync(s->info, 0, (2 * L + 2) * sizeof(int), st));
  SCW_CU(cudaEventRecord(s->ev[0], st));

  // 1. Fourier coefficients of n^2 and 1/n^2 at the order differences
  row_dft_kernel<<<nblk((size_t)L * 2 * s->Ny * nu), 256, 0, st>>>(nv_in, L, s->Nx, s->Ny, s->U, s->wx, s->R);
  SCW_CU(cudaGetLastError());
  col_dft_kernel<<<nblk((size_t)L * 2 * nv * nu), 256, 0, st>>>(s->R, L, s->Nx, s->Ny, s->U, s->V, s->wy, s->tab);
  SCW_CU(cudaGetLastError());
  SCW_CU(cudaEventRecord(s->ev[1], st));

  // 2-3. A, B, Psi; C = A B; eig(C) = (lambda, P); B P; forward branch and column scales
  assemble_kernel<<<nblk((size_t)L * n * n), 256, 0, st>>>(s->tab, L, s->geom, s->A, s->B, s->Psi);
  SCW_CU(cudaGetLastError());
  const long long nn = (long long)n * n;
  SCW_BL(cublasZgemmStridedBatched(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, Z(s->A), n, nn, Z(s->B), n, nn,
                                   &zero, Z(s->C), n, nn, L));
  {
    // layers l = w, w + nw, ... on worker w, each on its own host thread and stream
    SCW_CU(cudaEventRecord(s->ev_ready, st));
    int dev = 0;
    SCW_CU(cudaGetDevice(&dev));
    const int nw = (int)s->eig.size();
    std::vector<std::string> errs(nw);
    std::vector<std::thread> th;
    for (int w = 0; w < nw; ++w)
      th.emplace_back([&, w] {
        auto& k = s->eig[w];
        if (cudaSetDevice(dev) != cudaSuccess || cudaStreamWaitEvent(k.st, s->ev_ready, 0) != cudaSuccess) {
          errs[w] = "worker stream setup";
          return;
        }
        for (int l = w; l < L; l += nw) {
          const cusolverStatus_t r = cusolverDnXgeev(
              k.h, k.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, (int64_t)n, CUDA_C_64F,
              s->C + (size_t)l * nn, (int64_t)n, CUDA_C_64F, s->lam + (size_t)l * n, CUDA_C_64F, nullptr, 1,
              CUDA_C_64F, s->P + (size_t)l * nn, (int64_t)n, CUDA_C_64F, k.dwork, s->geev_dbytes, k.hwork.data(),
              k.hwork.size(), s->info + l);
          if (r != CUSOLVER_STATUS_SUCCESS) {
            errs[w] = "cusolverDnXgeev failed (cuSOLVER status " + std::to_string((int)r) + ")";
            return;
          }
        }
        if (cudaEventRecord(k.done, k.st) != cudaSuccess) errs[w] = "worker event";
      });
    for (auto& t : th) t.join();
    for (int w = 0; w < nw; ++w)
      if (!errs[w].empty()) return set_error(SCW_ERR_CUDA, errs[w]);
    for (auto& k : s->eig) SCW_CU(cudaStreamWaitEvent(st, k.done, 0));
  }
  SCW_BL(cublasZgemmStridedBatched(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, Z(s->B), n, nn, Z(s->P), n, nn,
                                   &zero, Z(s->BP), n, nn, L));
  modes_kernel<<<dim3(n, L), 256, 0, st>>>(s->lam, s->P, s->BP, M, k, s->thick, gamma_out, s->gam, s->sc, s->sg,
                                           s->ex, s->err);
  SCW_CU(cudaGetLastError());
  SCW_CU(cudaEventRecord(s->ev[2], st));

  // 4. T_l, B_l; K = B_L T_L^-1 ... B_1 T_1^-1 (T_l keeps its LU factors for step 6)
  top_bottom_kernel<<<nblk((size_t)L * N * N), 256, 0, st>>>(s->P, s->BP, s->sc, s->sg, s->ex, M, L, s->T, s->Bm);
  SCW_CU(cudaGetLastError());
  const size_t NN = (size_t)N * N;
  identity_kernel<<<nblk(NN), 256, 0, st>>>(s->Xm, N);
  SCW_CU(cudaGetLastError());
  for (int l = 0; l < L; ++l) {
    double2* Tl = s->T + (size_t)l * NN;
    int* piv = s->ipiv + (size_t)l * N;
    SCW_SV(cusolverDnZgetrf(s->sol, N, N, Z(Tl), N, Z(s->dwork), piv, s->info + L + l));
    if (l > 0) SCW_CU(cudaMemcpyAsync(s->Xm, s->K, NN * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SCW_SV(cusolverDnZgetrs(s->sol, CUBLAS_OP_N, N, N, Z(Tl), N, piv, Z(s->Xm), N, s->info + 2 * L + 1));
    SCW_BL(cublasZgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, N, N, N, &one, Z(s->Bm + (size_t)l * NN), N, Z(s->Xm), N,
                       &zero, Z(s->K), N));
  }
  SCW_CU(cudaEventRecord(s->ev[3], st));

  // 5. the 6M system for p_ref, p_trn
  const double dz0 = s->zb[0] - s->z_inc;
  rbar_kernel<<<nblk(4 * M), 256, 0, st>>>(p_inc, s->sz_t, s->geom, k, dz0, s->rbar);
  SCW_CU(cudaGetLastError());
  system_kernel<<<nblk((size_t)N6 * N6), 256, 0, st>>>(s->K, s->sz_t, s->sz_b, s->geom, s->A6);
  SCW_CU(cudaGetLastError());
  SCW_CU(cudaMemsetAsync(s->x6, 0, (size_t)N6 * sizeof(double2), st));
  SCW_BL(cublasZgemv(s->blas, CUBLAS_OP_N, N, N, &one, Z(s->K), N, Z(s->rbar), 1, &zero, Z(s->x6), 1));
  int* piv6 = s->ipiv + (size_t)L * N;
  SCW_SV(cusolverDnZgetrf(s->sol, N6, N6, Z(s->A6), N6, Z(s->dwork), piv6, s->info + 2 * L));
  SCW_SV(cusolverDnZgetrs(s->sol, CUBLAS_OP_N, N6, 1, Z(s->A6), N6, piv6, Z(s->x6), N6, s->info + 2 * L + 1));
  copy_z_kernel<<<nblk(3 * M), 256, 0, st>>>(s->x6, static_cast<double2*>(p_ref_v), 3 * M);
  copy_z_kernel<<<nblk(3 * M), 256, 0, st>>>(s->x6 + 3 * M, static_cast<double2*>(p_trn_v), 3 * M);
  SCW_CU(cudaGetLastError());
  SCW_CU(cudaEventRecord(s->ev[4], st));

  // 6. alpha_1 = T_1^-1 (R_bar + C_ref p_ref), alpha_l = T_l^-1 B_{l-1} alpha_{l-1}
  alpha1_rhs_kernel<<<nblk(4 * M), 256, 0, st>>>(s->rbar, s->x6, s->sz_t, s->geom, alpha);
  SCW_CU(cudaGetLastError());
  for (int l = 0; l < L; ++l) {
    double2* al = alpha + (size_t)l * N;
    if (l > 0)
      SCW_BL(cublasZgemv(s->blas, CUBLAS_OP_N, N, N, &one, Z(s->Bm + (size_t)(l - 1) * NN), N, Z(al - N), 1, &zero,
                         Z(al), 1));
    SCW_SV(cusolverDnZgetrs(s->sol, CUBLAS_OP_N, N, 1, Z(s->T + (size_t)l * NN), N, s->ipiv + (size_t)l * N, Z(al),
                            N, s->info + 2 * L + 1));
  }
  SCW_CU(cudaEventRecord(s->ev[5], st));

  // 7. E_z rows and the W output
  erows_g_kernel<<<nblk((size_t)L * M * n), 256, 0, st>>>(s->BP, s->sg, s->geom, L, s->G);
  SCW_CU(cudaGetLastError());
  SCW_BL(cublasZgemmStridedBatched(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, M, n, M, &one, Z(s->Psi), M, (long long)M * M,
                                   Z(s->G), M, (long long)M * n, &zero, Z(s->Ez), M, (long long)M * n, L));
  w_out_kernel<<<nblk((size_t)L * 3 * M * N), 256, 0, st>>>(s->P, s->sc, s->Ez, M, L, static_cast<float2*>(W_v));
  SCW_CU(cudaGetLastError());
  SCW_CU(cudaEventRecord(s->ev[6], st));

  std::vector<int> info(2 * L + 2);
  int herr = 0;
  SCW_CU(cudaMemcpyAsync(info.data(), s->info, info.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  SCW_CU(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SCW_CU(cudaStreamSynchronize(st));
  s->timed = true;
  for (int l = 0; l < L; ++l)
    if (info[l]) return set_error(SCW_ERR_NUMERIC, "eigendecomposition of layer " + std::to_string(l) + " failed (info " +
                                                       std::to_string(info[l]) + ")");
  for (int l = 0; l < L; ++l)
    if (info[L + l]) return set_error(SCW_ERR_NUMERIC, "boundary matrix of layer " + std::to_string(l) + " is singular");
  if (info[2 * L]) return set_error(SCW_ERR_NUMERIC, "the 6M boundary system is singular");
  if (info[2 * L + 1]) return set_error(SCW_ERR_NUMERIC, "an LU solve reported an invalid argument");
  if (herr) return set_error(SCW_ERR_NUMERIC, "a mode has gamma = 0 (grazing wave in a layer)");
  return SCW_OK;
}

scw_status scw_solver_get_times(scw_solver_t s, scw_solve_times* t) {
  if (!s || !t) return set_error(SCW_ERR_INVALID_ARGUMENT, "solver and t are required");
  std::memset(t, 0, sizeof(*t));
  if (!s->timed) return SCW_OK;
  float ms[6], tot = 0.f;
  for (int i = 0; i < 6; ++i) SCW_CU(cudaEventElapsedTime(&ms[i], s->ev[i], s->ev[i + 1]));
  SCW_CU(cudaEventElapsedTime(&tot, s->ev[0], s->ev[6]));
  t->calls = 1;
  t->fourier_ms = ms[0];
  t->modes_ms = ms[1];
  t->connect_ms = ms[2];
  t->system_ms = ms[3];
  t->alpha_ms = ms[4];
  t->erows_ms = ms[5];
  t->total_ms = tot;
  return SCW_OK;
}

}  // extern "C"
