// Complex helpers and the in-register 8-point inverse DFT of the recomposition kernels
// (step (c)).
#pragma once

#include <cuda_runtime.h>

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

}  // namespace scw
