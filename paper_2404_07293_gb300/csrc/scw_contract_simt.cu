// Step (b), plain FP32 path: S_l = W_l C_l as a SIMT complex GEMM
// (Eq. 34 with the per-layer precompute of Sec. 4.1).
//
// W is consumed transposed (Wt[l][j][r], rows r contiguous, made once by
// scw_plan_set_layers) so that a warp's 32 lanes load 32 consecutive rows of
// one mode j in a single coalesced request, while that mode's weights
// C[j][f0..f0+FCH) are a shared-memory broadcast. Each thread accumulates two
// rows x FCH planes in registers; the 4M modes are split across CTAs and the
// partial spectra are summed by the recompose step.
#include "scw_internal.cuh"

namespace scw {

template <int FCH>
__global__ void __launch_bounds__(128) contract_fp32_kernel(const float2* __restrict__ Wt, const float2* __restrict__ C,
                                                            const LayerUnit* __restrict__ units, int n_rblk, int ksplit,
                                                            int M, int F_pad, int Fz, float2* __restrict__ S_part,
                                                            unsigned long long* trace,
                                                            const __grid_constant__ ItemDev chk) {
  extern __shared__ float4 cs4[];
  trace_begin(trace, TRACE_CONTRACT);
  float2* Cs = reinterpret_cast<float2*>(cs4);
  const int split = blockIdx.x % ksplit;
  const int rest = blockIdx.x / ksplit;
  const int rblk = rest % n_rblk;
  const int ui = rest / n_rblk;
  const LayerUnit u = units[ui];
  const int fc0 = blockIdx.y * FCH;
  if (fc0 >= u.nf) return;
  const int K = 4 * M, rows = 3 * M;
  const int per = (K + ksplit - 1) / ksplit;
  const int kb = split * per;
  const int ke = min(K, kb + per);
  const int kc = max(0, ke - kb);

  for (int i = threadIdx.x; i < kc * FCH; i += blockDim.x) {
    const int k = i / FCH, f = i - k * FCH;
    const size_t ci = ((size_t)ui * K + kb + k) * F_pad + fc0 + f;
    Cs[i] = (fc0 + f < F_pad && in_bounds(chk, BND_C, ci)) ? C[ci] : make_float2(0.f, 0.f);
  }
  __syncthreads();

  const int r0 = rblk * 256 + threadIdx.x;
  const int r1 = r0 + 128;
  // W^T rows (layer, mode) and columns r: the loop's largest index, checked once (indices grow with k)
  const bool wt_ok = kc == 0 || in_bounds(chk, BND_WT, ((size_t)u.layer * K + kb + kc - 1) * rows + min(r1, rows - 1));
  const bool v0 = r0 < rows && wt_ok, v1 = r1 < rows && wt_ok;
  float2 a0[FCH], a1[FCH];
#pragma unroll
  for (int f = 0; f < FCH; ++f) a0[f] = a1[f] = make_float2(0.f, 0.f);
  const float2* w = Wt + ((size_t)u.layer * K + kb) * rows;

#pragma unroll 4
  for (int k = 0; k < kc; ++k) {
    const float2 w0 = v0 ? __ldg(w + (size_t)k * rows + r0) : make_float2(0.f, 0.f);
    const float2 w1 = v1 ? __ldg(w + (size_t)k * rows + r1) : make_float2(0.f, 0.f);
    const float4* c = cs4 + (k * FCH) / 2;
#pragma unroll
    for (int q = 0; q < FCH / 2; ++q) {
      const float4 cc = c[q];
      a0[2 * q].x = fmaf(w0.x, cc.x, fmaf(-w0.y, cc.y, a0[2 * q].x));
      a0[2 * q].y = fmaf(w0.x, cc.y, fmaf(w0.y, cc.x, a0[2 * q].y));
      a0[2 * q + 1].x = fmaf(w0.x, cc.z, fmaf(-w0.y, cc.w, a0[2 * q + 1].x));
      a0[2 * q + 1].y = fmaf(w0.x, cc.w, fmaf(w0.y, cc.z, a0[2 * q + 1].y));
      a1[2 * q].x = fmaf(w1.x, cc.x, fmaf(-w1.y, cc.y, a1[2 * q].x));
      a1[2 * q].y = fmaf(w1.x, cc.y, fmaf(w1.y, cc.x, a1[2 * q].y));
      a1[2 * q + 1].x = fmaf(w1.x, cc.z, fmaf(-w1.y, cc.w, a1[2 * q + 1].x));
      a1[2 * q + 1].y = fmaf(w1.x, cc.w, fmaf(w1.y, cc.z, a1[2 * q + 1].y));
    }
  }

  const size_t d0 = ((size_t)split * Fz + u.f0 + fc0) * rows;
  float2* dst = S_part + d0;
#pragma unroll
  for (int f = 0; f < FCH; ++f) {
    if (fc0 + f < u.nf) {
      if (v0 && in_bounds(chk, BND_S_PART, d0 + (size_t)f * rows + r0)) dst[(size_t)f * rows + r0] = a0[f];
      if (v1 && in_bounds(chk, BND_S_PART, d0 + (size_t)f * rows + r1)) dst[(size_t)f * rows + r1] = a1[f];
    }
  }
  trace_end(trace, TRACE_CONTRACT);
}

cudaError_t launch_contract_fp32(const Plan& p, cudaStream_t st) {
  if (p.units.empty()) return cudaSuccess;
  const int n_rblk = (3 * p.M + 255) / 256;
  const int K = 4 * p.M;
  const int per = (K + p.k_split - 1) / p.k_split;
  const bool wide = p.F_pad >= 16;
  const int FCH = wide ? 16 : 8;
  dim3 grid((unsigned)(p.units.size() * n_rblk * p.k_split), (unsigned)((p.F_pad + FCH - 1) / FCH));
  const size_t smem = (size_t)per * FCH * sizeof(float2);
  cudaError_t e;
  if (wide) {
    e = allow_max_smem(reinterpret_cast<const void*>(contract_fp32_kernel<16>));
    if (e != cudaSuccess) return e;
    contract_fp32_kernel<16><<<grid, 128, smem, st>>>(p.Wt, p.Cf, p.d_units, n_rblk, p.k_split, p.M, p.F_pad, p.Fz,
                                                      p.S_part, p.item.trace, p.item);
  } else {
    e = allow_max_smem(reinterpret_cast<const void*>(contract_fp32_kernel<8>));
    if (e != cudaSuccess) return e;
    contract_fp32_kernel<8><<<grid, 128, smem, st>>>(p.Wt, p.Cf, p.d_units, n_rblk, p.k_split, p.M, p.F_pad, p.Fz,
                                                     p.S_part, p.item.trace, p.item);
  }
  return cudaGetLastError();
}

}  // namespace scw
