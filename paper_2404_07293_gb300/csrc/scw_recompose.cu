// Step (c): recomposition of the field from its per-plane spectrum (Eq. 10),
//   E_c(x_i, y_j) = sum_{u,v} S_c[u,v] exp(2 pi i (u x_i / X + v y_j / Y)),
// on x_i = x0 + i X/Fx, y_j = y0 + j Y/Fy: an unnormalised inverse 2D DFT of
// the U x V non-zero orders onto the Fx x Fy grid.
//
// Both axes use the same pruned radix-8 decimation. With F = 8 Q and output
// index i = b + Q a (b < Q, a < 8), omega = exp(2 pi i / F):
//   sum_u s_u omega^(u (b + Q a)) = sum_{r<8} e^(2 pi i r a / 8) F_b[r],
//   F_b[r] = sum_{u = r mod 8} s_u omega^(u b).
// So each thread folds the few non-zero inputs into 8 residue bins with one
// table twiddle each (tw[b][u] = omega^(u b) times the origin phase
// exp(2 pi i u x0 / X)), then finishes with an in-register radix-8 inverse
// DFT and writes 8 outputs Q apart. Orders beyond the grid (|u| >= F/2) fold
// exactly, as the sum is only evaluated at grid points.
//
//   x-pass: S[f][c][v][u]      -> T[f][c][v][x]   (V rows per plane)
//   y-pass: T[f][c][v][x-block] -> out[c][f][y][x] (16-byte streaming stores)
#include "scw_internal.cuh"

namespace scw {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ void c_fma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// In-place 8-point inverse DFT, X[a] = sum_r x[r] exp(+2 pi i r a / 8):
// one radix-2 decimation-in-frequency step, then two 4-point DFTs.
__device__ __forceinline__ void idft8(float2 (&x)[8]) {
  const float h = 0.70710678118654752440f;
  const float2 u0 = c_add(x[0], x[4]), u1 = c_add(x[1], x[5]), u2 = c_add(x[2], x[6]), u3 = c_add(x[3], x[7]);
  const float2 d0 = c_sub(x[0], x[4]), d1 = c_sub(x[1], x[5]), d2 = c_sub(x[2], x[6]), d3 = c_sub(x[3], x[7]);
  const float2 v0 = d0;
  const float2 v1 = make_float2(h * (d1.x - d1.y), h * (d1.x + d1.y));    // * exp(i pi/4)
  const float2 v2 = make_float2(-d2.y, d2.x);                             // * i
  const float2 v3 = make_float2(h * (-d3.x - d3.y), h * (d3.x - d3.y));   // * exp(3 i pi/4)
  // 4-point inverse DFTs (twiddle i): even outputs from u, odd outputs from v
  {
    const float2 s0 = c_add(u0, u2), s1 = c_sub(u0, u2), s2 = c_add(u1, u3);
    const float2 t = c_sub(u1, u3);
    const float2 s3 = make_float2(-t.y, t.x);
    x[0] = c_add(s0, s2);
    x[4] = c_sub(s0, s2);
    x[2] = c_add(s1, s3);
    x[6] = c_sub(s1, s3);
  }
  {
    const float2 s0 = c_add(v0, v2), s1 = c_sub(v0, v2), s2 = c_add(v1, v3);
    const float2 t = c_sub(v1, v3);
    const float2 s3 = make_float2(-t.y, t.x);
    x[1] = c_add(s0, s2);
    x[5] = c_sub(s0, s2);
    x[3] = c_add(s1, s3);
    x[7] = c_sub(s1, s3);
  }
}

// One CTA per (plane, component): sum the contraction's partial spectra into
// shared memory, then V * Fx/8 fold+DFT tasks.
__global__ void __launch_bounds__(256) xpass_kernel(const float2* __restrict__ S_part, size_t split_stride,
                                                    const int* __restrict__ nsplit, const float2* __restrict__ twx,
                                                    int U, int V, int Fx, float2* __restrict__ T) {
  extern __shared__ float2 srow[];  // [M]
  const int f = blockIdx.x, c = blockIdx.y;
  const int M = U * V;
  const int ns = nsplit[f];
  const float2* src = S_part + (size_t)f * 3 * M + (size_t)c * M;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < ns; ++s) acc = c_add(acc, src[(size_t)s * split_stride + m]);
    srow[m] = acc;
  }
  __syncthreads();
  const int Q = Fx >> 3;
  const int h = U >> 1;
  float2* dst = T + ((size_t)f * 3 + c) * V * Fx;
  for (int task = threadIdx.x; task < V * Q; task += blockDim.x) {
    const int vi = task / Q, b = task - vi * Q;
    const float2* s = srow + vi * U;
    const float2* tw = twx + (size_t)b * U;
    float2 F[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      F[r] = make_float2(0.f, 0.f);
      for (int ui = (r + h) & 7; ui < U; ui += 8) c_fma(F[r], s[ui], __ldg(tw + ui));
    }
    idft8(F);
    float2* o = dst + (size_t)vi * Fx + b;
#pragma unroll
    for (int a = 0; a < 8; ++a) o[a * Q] = F[a];
  }
}

// One CTA per (64-column block, plane, component); 8 warps, lane l owns the
// column pair (2l, 2l+1) of the block and warp w the residues b = w, w+8, ...
__global__ void __launch_bounds__(256) ypass_kernel(const float2* __restrict__ T, const float2* __restrict__ twy,
                                                    int V, int Fx, int Fy, int Fz, float2* __restrict__ out) {
  extern __shared__ float4 tcol4[];  // [V][32] float4 = [V][64] complex
  float2* tcol = reinterpret_cast<float2*>(tcol4);
  const int xb = blockIdx.x * 64, f = blockIdx.y, c = blockIdx.z;
  const float2* src = T + ((size_t)f * 3 + c) * V * Fx;
  for (int i = threadIdx.x; i < V * 64; i += blockDim.x) {
    const int v = i >> 6, x = i & 63;
    tcol[i] = (xb + x < Fx) ? src[(size_t)v * Fx + xb + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x = xb + 2 * lane;
  const int Q = Fy >> 3;
  const int h = V >> 1;
  float2* dst = out + (((size_t)c * Fz + f) * Fy) * Fx + x;
  for (int b = w; b < Q; b += 8) {
    float2 F0[8], F1[8];
    const float2* tw = twy + (size_t)b * V;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      F0[r] = F1[r] = make_float2(0.f, 0.f);
      for (int vi = (r + h) & 7; vi < V; vi += 8) {
        const float2 t = __ldg(tw + vi);
        const float4 d = tcol4[vi * 32 + lane];
        c_fma(F0[r], make_float2(d.x, d.y), t);
        c_fma(F1[r], make_float2(d.z, d.w), t);
      }
    }
    idft8(F0);
    idft8(F1);
    if (x < Fx) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
        __stcs(reinterpret_cast<float4*>(dst + (size_t)(b + a * Q) * Fx), make_float4(F0[a].x, F0[a].y, F1[a].x, F1[a].y));
    }
  }
}

// S[f][3M] = sum of the contraction's partial spectra (scw_spectrum).
__global__ void gather_kernel(const float2* __restrict__ S_part, size_t split_stride, const int* __restrict__ nsplit,
                              int rows, int Fz, float2* __restrict__ S) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)rows * Fz) return;
  const int f = (int)(i / rows);
  float2 acc = make_float2(0.f, 0.f);
  for (int s = 0; s < nsplit[f]; ++s) acc = c_add(acc, S_part[(size_t)s * split_stride + i]);
  S[i] = acc;
}

cudaError_t launch_xpass(const Plan& p, const float2* S_part, int split_stride_planes, const int* d_nsplit,
                         cudaStream_t st) {
  const size_t split_stride = (size_t)split_stride_planes * 3 * p.M;
  xpass_kernel<<<dim3(p.Fz, 3), 256, (size_t)p.M * sizeof(float2), st>>>(S_part, split_stride, d_nsplit, p.d_twx, p.U,
                                                                        p.V, p.Fx, p.T);
  return cudaGetLastError();
}

cudaError_t launch_ypass(const Plan& p, float2* out, cudaStream_t st) {
  ypass_kernel<<<dim3((p.Fx + 63) / 64, p.Fz, 3), 256, (size_t)p.V * 64 * sizeof(float2), st>>>(p.T, p.d_twy, p.V, p.Fx,
                                                                                               p.Fy, p.Fz, out);
  return cudaGetLastError();
}

cudaError_t launch_recompose(const Plan& p, const float2* S_part, int split_stride_planes, const int* d_nsplit,
                             float2* out, cudaStream_t st) {
  cudaError_t e = launch_xpass(p, S_part, split_stride_planes, d_nsplit, st);
  if (e != cudaSuccess) return e;
  return launch_ypass(p, out, st);
}

cudaError_t launch_gather_spectrum(const Plan& p, float2* S, cudaStream_t st) {
  const size_t n = (size_t)p.Fz * 3 * p.M;
  gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p.S_part, (size_t)p.Fz * 3 * p.M, p.d_nsplit, 3 * p.M,
                                                            p.Fz, S);
  return cudaGetLastError();
}

}  // namespace scw
