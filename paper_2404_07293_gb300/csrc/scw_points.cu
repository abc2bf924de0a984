// Field at arbitrary lateral points (Eq. 10 off the grid): x-z and y-z planes,
// zoomed windows and scattered point sets.
//
//   E_c(x_p, y_p, z_f) = sum_m S_c[m](z_f) phi_m(p),  phi_m(p) = exp(2 pi i (u_m x_p / X + v_m y_p / Y))
//
// With the plan's spectra S [Fz][3][M] this is one dense complex product over
// the M orders, E[p][(f, c)] = sum_m phi_m(p) S_{f,c}[m], written as a real GEMM
// D = A B^T over K = 2M interleaved reals:
//   A[p]        = (Re phi_0, Im phi_0, Re phi_1, Im phi_1, ...)      (points table)
//   B[2j]       = (Re s_0, -Im s_0, ...)  -> D[p][2j]     = Re E_j(p)
//   B[2j + 1]   = (Im s_0,  Re s_0, ...)  -> D[p][2j + 1] = Im E_j(p),   j = f 3 + c.
// Tensor-core plans run it as one BF16 GEMM with split operands: K is tripled,
// A' = [A_hi | A_hi | A_lo] and B' = [B_hi | B_lo | B_hi] (each segment padded to
// Kp = roundup(2M, 64) with zeros), so A'B'^T = A_hi B_hi + A_hi B_lo + A_lo B_hi:
// the split-BF16 product with only lo x lo (~2^-16 relative) dropped. FP32 plans
// run the same product in FP32 on the SIMT GEMM. Both share the epilogue that
// scatters D to the field layout [I][3][Fz][P].
#include <algorithm>

#include "fno_internal.cuh"
#include "scw_internal.cuh"
#include "scw_points.cuh"

namespace scw {

namespace {

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// phi_m(p) with the phase reduced in cycles in FP64: t = u x / X + v y / Y, t - rint(t) in [-1/2, 1/2].
__device__ __forceinline__ float2 point_phase(double2 xy, int m, int U, int V, double invX, double invY) {
  const int u = m % U - U / 2, v = m / U - V / 2;
  double t = (double)u * xy.x * invX + (double)v * xy.y * invY;
  t -= rint(t);
  float s, c;
  sincospif(2.0f * (float)t, &s, &c);
  return make_float2(c, s);
}

// Points table of tensor-core plans: A' [P][3 Kp] bf16 (padding columns are zeroed by the caller).
__global__ void points_table_tc_kernel(const double2* __restrict__ xy, int P, int M, int U, int V, double invX,
                                       double invY, int Kp, __nv_bfloat16* __restrict__ A) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)P * M) return;
  const int p = (int)(i / M), m = (int)(i - (size_t)p * M);
  const float2 ph = point_phase(xy[p], m, U, V, invX, invY);
  __nv_bfloat162 hi, lo;
  split_bf16(ph.x, hi.x, lo.x);
  split_bf16(ph.y, hi.y, lo.y);
  __nv_bfloat162* row = reinterpret_cast<__nv_bfloat162*>(A + (size_t)p * 3 * Kp);
  const int hk = Kp / 2;  // bf16 pairs per segment
  row[m] = hi;
  row[hk + m] = hi;
  row[2 * hk + m] = lo;
}

// Points table of FP32 plans: A [P][2M] float.
__global__ void points_table_fp32_kernel(const double2* __restrict__ xy, int P, int M, int U, int V, double invX,
                                         double invY, float2* __restrict__ A) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)P * M) return;
  const int p = (int)(i / M), m = (int)(i - (size_t)p * M);
  A[i] = point_phase(xy[p], m, U, V, invX, invY);
}

// Spectrum operand of tensor-core plans, B' [2 rows3][3 Kp] bf16, rows3 = 3 Fz
// (split partials of the contraction summed; padding columns stay zero).
__global__ void points_spectrum_tc_kernel(const float2* __restrict__ S_part, size_t split_stride,
                                          const int* __restrict__ nsplit, int rows3, int M, int Kp,
                                          __nv_bfloat16* __restrict__ B) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)rows3 * M) return;
  const int j = (int)(i / M), m = (int)(i - (size_t)j * M);
  const int f = j / 3;
  float2 s = make_float2(0.f, 0.f);
  const int ns = nsplit[f];
  for (int k = 0; k < ns; ++k) {
    const float2 t = S_part[(size_t)k * split_stride + i];  // S_part[k][f][c M + m], i = (f 3 + c) M + m
    s.x += t.x;
    s.y += t.y;
  }
  __nv_bfloat162 h0, l0, h1, l1;
  split_bf16(s.x, h0.x, l0.x);
  split_bf16(-s.y, h0.y, l0.y);
  split_bf16(s.y, h1.x, l1.x);
  split_bf16(s.x, h1.y, l1.y);
  const int hk = Kp / 2;
  __nv_bfloat162* r0 = reinterpret_cast<__nv_bfloat162*>(B + (size_t)(2 * j) * 3 * Kp);
  __nv_bfloat162* r1 = reinterpret_cast<__nv_bfloat162*>(B + (size_t)(2 * j + 1) * 3 * Kp);
  r0[m] = h0;
  r0[hk + m] = l0;
  r0[2 * hk + m] = h0;
  r1[m] = h1;
  r1[hk + m] = l1;
  r1[2 * hk + m] = h1;
}

// Spectrum operand of FP32 plans, B [2 rows3][2M] float.
__global__ void points_spectrum_fp32_kernel(const float2* __restrict__ S_part, size_t split_stride,
                                            const int* __restrict__ nsplit, int rows3, int M,
                                            float2* __restrict__ B) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)rows3 * M) return;
  const int j = (int)(i / M), m = (int)(i - (size_t)j * M);
  const int f = j / 3;
  float2 s = make_float2(0.f, 0.f);
  const int ns = nsplit[f];
  for (int k = 0; k < ns; ++k) {
    const float2 t = S_part[(size_t)k * split_stride + i];
    s.x += t.x;
    s.y += t.y;
  }
  B[(size_t)(2 * j) * M + m] = make_float2(s.x, -s.y);
  B[(size_t)(2 * j + 1) * M + m] = make_float2(s.y, s.x);
}

unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Scattered 3-D points: one warp per (point, illumination). E_c = sum_m S_c[m](z_f) phi_m(p) with
// S of plane slot f = plane[p] I + il (the contraction's partials summed) and phi from the point
// table (split-BF16 tables: hi + lo). out [I][3][P].
template <bool TC>
__global__ void points_scattered_kernel(const float2* __restrict__ S_part, size_t split_stride,
                                        const int* __restrict__ nsplit, const int* __restrict__ plane,
                                        const void* __restrict__ table, int P, int M, int Kp, int I,
                                        float2* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (wid >= (long long)P * I) return;
  const int p = (int)(wid % P), il = (int)(wid / P);
  const int f = plane[p] * I + il;
  const int ns = nsplit[f];
  const float2* S = S_part + (size_t)f * 3 * M;
  float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int m = lane; m < M; m += 32) {
    float2 ph;
    if constexpr (TC) {
      const __nv_bfloat162* row = static_cast<const __nv_bfloat162*>(table) + (size_t)p * 3 * (Kp / 2);
      const __nv_bfloat162 hi = row[m], lo = row[Kp + m];  // segments hi | hi | lo of Kp / 2 pairs each
      ph = make_float2(__bfloat162float(hi.x) + __bfloat162float(lo.x), __bfloat162float(hi.y) + __bfloat162float(lo.y));
    } else {
      ph = static_cast<const float2*>(table)[(size_t)p * M + m];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 s = make_float2(0.f, 0.f);
      for (int k = 0; k < ns; ++k) {
        const float2 t = S[(size_t)k * split_stride + (size_t)c * M + m];
        s.x += t.x;
        s.y += t.y;
      }
      acc[c].x = fmaf(s.x, ph.x, fmaf(-s.y, ph.y, acc[c].x));
      acc[c].y = fmaf(s.x, ph.y, fmaf(s.y, ph.x, acc[c].y));
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, o);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, o);
    }
    if (lane == 0) out[((size_t)il * 3 + c) * P + p] = acc[c];
  }
}

}  // namespace

void points_free(PointTables* t) {
  if (!t) return;
  if (t->d_plane) cudaFree(t->d_plane);
  if (t->d_xy) cudaFree(t->d_xy);
  if (t->A) cudaFree(t->A);
  if (t->B) cudaFree(t->B);
  delete t;
}

scw_status points_build(PointTables** out, const Plan& p, bool tc, const double* xy, int P, cudaStream_t st) {
  PointTables* t = new (std::nothrow) PointTables();
  if (!t) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  const int M = p.M, rows3 = 3 * p.Fz;
  t->P = P;
  t->tc = tc;
  t->rows3 = rows3;
  t->Kp = (2 * M + 63) / 64 * 64;
  const size_t a_bytes = tc ? (size_t)P * 3 * t->Kp * sizeof(__nv_bfloat16) : (size_t)P * M * sizeof(float2);
  const size_t b_bytes = tc ? (size_t)2 * rows3 * 3 * t->Kp * sizeof(__nv_bfloat16) : (size_t)2 * rows3 * M * sizeof(float2);
  cudaError_t e = cudaMalloc(&t->d_xy, (size_t)P * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&t->A, a_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&t->B, b_bytes);
  if (e != cudaSuccess) {
    points_free(t);
    return e == cudaErrorMemoryAllocation ? set_error(SCW_ERR_OUT_OF_MEMORY, "point tables do not fit")
                                          : cuda_error(e, "cudaMalloc (point tables)");
  }
  t->bytes = a_bytes + b_bytes + (size_t)P * sizeof(double2);
  e = cudaMemcpyAsync(t->d_xy, xy, (size_t)P * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && tc) e = cudaMemsetAsync(t->A, 0, a_bytes, st);
  if (e == cudaSuccess && tc) e = cudaMemsetAsync(t->B, 0, b_bytes, st);
  if (e == cudaSuccess) {
    const size_t n = (size_t)P * M;
    if (tc)
      points_table_tc_kernel<<<blocks_for(n, 256), 256, 0, st>>>(t->d_xy, P, M, p.U, p.V, 1.0 / p.X, 1.0 / p.Y,
                                                                 t->Kp, static_cast<__nv_bfloat16*>(t->A));
    else
      points_table_fp32_kernel<<<blocks_for(n, 256), 256, 0, st>>>(t->d_xy, P, M, p.U, p.V, 1.0 / p.X, 1.0 / p.Y,
                                                                   static_cast<float2*>(t->A));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    points_free(t);
    return cuda_error(e, "building the point tables");
  }
  if (tc) {
    // N = 2 rows3 columns of D: the widest tile that does not waste most of itself, narrowed
    // while the grid would leave most SMs idle (few points, e.g. one x-z plane)
    const int N = 2 * rows3;
    t->BN = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long m_tiles = (P + 127) / 128;
    while (t->BN > 64 && m_tiles * ((N + t->BN - 1) / t->BN) < 2LL * sms) t->BN /= 2;
    const long long K = 3LL * t->Kp;
    scw_status s = fno::make_map_bf16(&t->mA, t->A, K, P, K, 128, 64);
    if (s == SCW_OK) s = fno::make_map_bf16(&t->mB, t->B, K, N, K, t->BN, 64);
    if (s != SCW_OK) {
      points_free(t);
      return s;
    }
  }
  *out = t;
  return SCW_OK;
}

scw_status points_set_planes(PointTables& t, const int* plane, int Fz_out, cudaStream_t st) {
  if (!plane) {
    if (t.d_plane) cudaFree(t.d_plane);
    t.d_plane = nullptr;
    return SCW_OK;
  }
  for (int i = 0; i < t.P; ++i)
    if (plane[i] < 0 || plane[i] >= Fz_out) return set_error(SCW_ERR_INVALID_ARGUMENT, "point plane index out of range");
  cudaError_t e = t.d_plane ? cudaSuccess : cudaMalloc(&t.d_plane, (size_t)t.P * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(t.d_plane, plane, (size_t)t.P * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SCW_OK : cuda_error(e, "point planes");
}

cudaError_t points_prepare(const PointTables& t, const Plan& p, cudaStream_t st) {
  if (t.d_plane) return cudaSuccess;  // scattered points read the partials directly
  const size_t n = (size_t)t.rows3 * p.M;
  const size_t stride = (size_t)p.Fz * 3 * p.M;
  if (t.tc)
    points_spectrum_tc_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p.S_part, stride, p.d_nsplit, t.rows3, p.M, t.Kp,
                                                                  static_cast<__nv_bfloat16*>(t.B));
  else
    points_spectrum_fp32_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p.S_part, stride, p.d_nsplit, t.rows3, p.M,
                                                                    static_cast<float2*>(t.B));
  return cudaGetLastError();
}

cudaError_t points_product(const PointTables& t, const Plan& p, float2* out, int* err, uint64_t timeout_ns,
                           cudaStream_t st) {
  if (t.d_plane) {
    const size_t warps = (size_t)t.P * p.I;
    const size_t stride = (size_t)p.Fz * 3 * p.M;
    if (t.tc)
      points_scattered_kernel<true><<<blocks_for(warps * 32, 256), 256, 0, st>>>(
          p.S_part, stride, p.d_nsplit, t.d_plane, t.A, t.P, p.M, t.Kp, p.I, out);
    else
      points_scattered_kernel<false><<<blocks_for(warps * 32, 256), 256, 0, st>>>(
          p.S_part, stride, p.d_nsplit, t.d_plane, t.A, t.P, p.M, t.Kp, p.I, out);
    return cudaGetLastError();
  }
  fno::EpiArgs ea{};
  ea.alpha = 1.f;
  ea.rows = t.P;
  ea.cols = 2 * t.rows3;
  ea.out = reinterpret_cast<float*>(out);
  ea.ld = t.P;
  ea.fz_out = p.Fz_out;
  ea.illum = p.I;
  if (t.tc)
    return fno::launch_gemm_tc(fno::EPI_FIELD, t.BN, t.mA, t.mB, t.mA, t.mA, ea, t.P, 2 * t.rows3, 3 * t.Kp, 1, err,
                               timeout_ns, st);
  return fno::launch_gemm_simt(fno::EPI_FIELD, static_cast<const float*>(t.A), 2LL * p.M,
                               static_cast<const float*>(t.B), 2LL * p.M, ea, t.P, 2 * t.rows3, 2 * p.M, 1, st);
}

}  // namespace scw
