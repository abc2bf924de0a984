// Internal declarations of the surrogate (Fourier neural operator) kernels.
// The network, its loss and the flat parameter order are defined in
// include/scw_fno.h; this header holds the device-side views of them.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "scw_internal.cuh"

namespace scw {
namespace fno {

constexpr int C = 32;    // channels (width)
constexpr int OUT = 6;   // Re/Im of E_x, E_y, E_z
constexpr int PIX_BLOCK = 256;  // pixels per block of the per-pixel kernels (N*N is a multiple)

// GEMM epilogues. Rows / columns are those of the GEMM's D = A B^T.
enum Epi : int {
  EPI_MODES = 0,      // rows = (sample, channel), columns = (mode, re/im): alpha D -> mode-major complex
                      // out[split][mode][row] (truncated DFTs)
  EPI_LAYER_FWD = 1,  // rows = pixels, columns = (sample, channel): Z = alpha D + c + W V; V' = GELU(Z)
  EPI_LAYER_BWD = 2,  // rows = pixels, columns = (sample, channel): dV = D + W^T dZ; dZ' = dV GELU'(Z)
                      // (GELU'(Z) stored by the forward)
  EPI_DW = 3,         // rows = (sample, o), columns = (sample, i) of 4 samples: keep the diagonal blocks
  EPI_FIELD = 4       // field synthesis at points: rows = points, columns = (plane slot f, component c,
                      // re/im); complex E[(f, c)][p] -> out[il][c][fo][p], f = fo I + il (streaming stores)
};

struct EpiArgs {
  float alpha;
  int rows;            // valid rows of D
  int cols;            // valid columns of D
  int P;               // pixels per sample
  int B;               // valid samples
  float* out;          // EPI_MODES: complex [split][cols/2][ld]; EPI_DW: [group][split][4][C][C]
  long long ld;        // EPI_MODES: row capacity per mode (complex elements)
  long long split_stride;  // EPI_MODES: complex elements per split
  int splits;          // EPI_DW: K splits per group
  const void* w;       // EPI_LAYER_*: W [C][C] (row = output channel), element type T
  const void* bias;    // EPI_LAYER_FWD: c [C] (T), may be null
  const void* x_cl;    // SIMT form: FWD V_l channel-last [B][P][C]; BWD dZ_l channel-last
  const void* g_in;    // BWD: GELU'(Z_{l-1}) channel-last, stored by the forward; null for l = 0
  void* g_out;         // FWD: GELU'(Z_l) channel-last (for the backward), null when not needed
  void* out_cf;        // FWD: V_{l+1} [B][C][P]; BWD: dZ_{l-1} [B][C][P]; null where not read
  void* out_cl;        // FWD: V_{l+1} [B][P][C]; BWD: dZ_{l-1} (or dV_0 for l = 0) [B][P][C]; null
                       // where not read
  int gelu;            // FWD: apply GELU
  int fz_out;          // FIELD: output planes per illumination
  int illum;           // FIELD: illuminations I
};

// ---- element access (T = float or __nv_bfloat16) ----------------------------------------
template <typename T>
__device__ __forceinline__ float to_f(T x);
template <>
__device__ __forceinline__ float to_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// 32 contiguous elements <-> float[32] with 16-byte accesses (p 16-byte aligned)
template <typename T>
__device__ __forceinline__ void ld32(const T* p, float (&v)[32]) {
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 t = q[j];
      v[4 * j] = t.x;
      v[4 * j + 1] = t.y;
      v[4 * j + 2] = t.z;
      v[4 * j + 3] = t.w;
    }
  } else {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 t = q[j];
      const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        v[8 * j + 2 * h] = __uint_as_float(w[h] << 16);
        v[8 * j + 2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
      }
    }
  }
}

// two floats as one bf16x2 word (a in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <typename T>
__device__ __forceinline__ void st32(T* p, const float (&v)[32]) {
  if constexpr (sizeof(T) == 4) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  } else {
    uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[8 * j + 2 * h], v[8 * j + 2 * h + 1]);
        w[h] = *reinterpret_cast<const uint32_t*>(&b);
      }
      q[j] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z), Phi the standard normal CDF and phi its
// density. Phi(z) = (1 + sign(z) erf(|z| / sqrt 2)) / 2 with erf from Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26: erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},
// t = 1 / (1 + p x), x >= 0, |error| <= 1.5e-7. Its factor e^{-x^2} = e^{-z^2/2} is also phi(z) sqrt(2 pi),
// so GELU and GELU' together cost one exponential and one reciprocal.
//
// GELU and GELU' of four values with one reciprocal between them: with d_i = 1 + p x_i and
// r = 1 / (d_0 d_1 d_2 d_3), t_i = r times the other three d_j (a few roundings more than a
// reciprocal each, far below the formula's 1.5e-7). x is clamped at 8, where t poly(t) e^{-x^2}
// is below 1e-28 in either case, so every d_i lies in [1, 3.63] and the product cannot overflow.
// The rest runs on value pairs with the packed FP32x2 instructions (FFMA2 / FMUL2 / FADD2), which
// issue two lanes' worth of arithmetic per instruction: the layer epilogues that apply GELU are
// bound by instruction issue. e^{-z^2/2} = 2^{-z^2 log2(e) / 2} on the special-function unit.
// The poly coefficients carry the factor 1/2 of Phi, so that m = poly E / 2 and
// Phi = 1/2 + sign(z) (1/2 - m).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// GP = false (inference): GELU only.
template <bool GP = true>
__device__ __forceinline__ void gelu4(float (&z)[4], float (&gp)[4]) {
  float d[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = fmaf(0.3275911f, fminf(fabsf(z[i]) * 0.70710678118654752f, 8.f), 1.f);
  const float d01 = d[0] * d[1], d23 = d[2] * d[3];
  const float r = __fdividef(1.f, d01 * d23);
  const float2 T[2] = {__fmul2_rn(make_float2(d[1], d[0]), f2(r * d23)),
                       __fmul2_rn(make_float2(d[3], d[2]), f2(r * d01))};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 Z = make_float2(z[2 * h], z[2 * h + 1]), t = T[h];
    float2 q = __ffma2_rn(t, f2(0.5f * 1.061405429f), f2(0.5f * -1.453152027f));
    q = __ffma2_rn(q, t, f2(0.5f * 1.421413741f));
    q = __ffma2_rn(q, t, f2(0.5f * -0.284496736f));
    q = __ffma2_rn(q, t, f2(0.5f * 0.254829592f));
    q = __fmul2_rn(q, t);  // poly / 2
    const float2 a = __fmul2_rn(__fmul2_rn(Z, Z), f2(-0.72134752044448170f));  // -z^2 log2(e) / 2
    const float2 E = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    const float2 hm = __ffma2_rn(q, make_float2(-E.x, -E.y), f2(0.5f));  // 1/2 - m
    const float2 Phi = __fadd2_rn(make_float2(copysignf(hm.x, Z.x), copysignf(hm.y, Z.y)), f2(0.5f));
    if constexpr (GP) {
      const float2 g = __ffma2_rn(__fmul2_rn(Z, f2(0.39894228040143268f)), E, Phi);
      gp[2 * h] = g.x;
      gp[2 * h + 1] = g.y;
    }
    const float2 o = __fmul2_rn(Z, Phi);
    z[2 * h] = o.x;
    z[2 * h + 1] = o.y;
  }
}

// ---- epilogues, shared by the tensor-core and the SIMT GEMM ------------------------------
// Called once per (row, 32-column chunk starting at col0) with that chunk's accumulators.
// w_s: W as FP32 [C][C] in shared memory; b_s: bias [C] (zeros if none). WACC: the 1x1
// convolution is already in the accumulator (tensor-core path); otherwise it is applied here.
template <int EPI, typename T, bool WACC>
__device__ __forceinline__ void epilogue(const EpiArgs& a, const float* w_s, const float* b_s, int row, int col0,
                                         int split, const float (&acc)[32]) {
  if constexpr (EPI == EPI_MODES) {
    if (row >= a.rows) return;
    float2* o = reinterpret_cast<float2*>(a.out) + (size_t)split * a.split_stride + row;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = col0 / 2 + j;
      if (2 * k < a.cols) o[(size_t)k * a.ld] = make_float2(a.alpha * acc[2 * j], a.alpha * acc[2 * j + 1]);
    }
  } else if constexpr (EPI == EPI_FIELD) {
    if (row >= a.rows) return;
    float2* o = reinterpret_cast<float2*>(a.out) + row;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = col0 / 2 + j;  // k = f 3 + c
      if (2 * k < a.cols) {
        const int f = k / 3, c = k - 3 * f;
        const int fo = f / a.illum, il = f - fo * a.illum;
        __stcs(o + ((size_t)(il * 3 + c) * a.fz_out + fo) * (size_t)a.ld, make_float2(acc[2 * j], acc[2 * j + 1]));
      }
    }
  } else if constexpr (EPI == EPI_LAYER_FWD) {
    const int p = row, b = col0 / C;
    if (p >= a.P || b >= a.B) return;
    const size_t cl = ((size_t)b * a.P + p) * C;
    float z[32];
#pragma unroll
    for (int o = 0; o < C; o += 2) {
      const float2 v = __ffma2_rn(make_float2(acc[o], acc[o + 1]), f2(a.alpha), make_float2(b_s[o], b_s[o + 1]));
      z[o] = v.x;
      z[o + 1] = v.y;
    }
    if constexpr (!WACC) {
      float x[32];
      ld32(static_cast<const T*>(a.x_cl) + cl, x);
#pragma unroll
      for (int o = 0; o < C; ++o) {
        float s = z[o];
#pragma unroll
        for (int i = 0; i < C; ++i) s = fmaf(w_s[o * C + i], x[i], s);
        z[o] = s;
      }
    }
    if (a.gelu && a.g_out) {
      // GELU in place, GELU' for the backward (the same exponentials and reciprocals)
      float gp[32];
#pragma unroll
      for (int q = 0; q < C / 4; ++q) {
        float zz[4] = {z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]}, gg[4];
        gelu4<true>(zz, gg);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          z[4 * q + i] = zz[i];
          gp[4 * q + i] = gg[i];
        }
      }
      st32(static_cast<T*>(a.g_out) + cl, gp);
    } else if (a.gelu) {  // inference: no GELU' to keep
#pragma unroll
      for (int q = 0; q < C / 4; ++q) {
        float zz[4] = {z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]}, gg[4];
        gelu4<false>(zz, gg);
#pragma unroll
        for (int i = 0; i < 4; ++i) z[4 * q + i] = zz[i];
      }
    }
    if (a.out_cl) st32(static_cast<T*>(a.out_cl) + cl, z);
    if (a.out_cf) {
      T* cf = static_cast<T*>(a.out_cf) + (size_t)b * C * a.P + p;
#pragma unroll
      for (int o = 0; o < C; ++o) cf[(size_t)o * a.P] = from_f<T>(z[o]);
    }
  } else if constexpr (EPI == EPI_LAYER_BWD) {
    const int p = row, b = col0 / C;
    if (p >= a.P || b >= a.B) return;
    const size_t cl = ((size_t)b * a.P + p) * C;
    float d[32];
#pragma unroll
    for (int i = 0; i < C; ++i) d[i] = a.alpha * acc[i];
    if constexpr (!WACC) {
      float x[32];
      ld32(static_cast<const T*>(a.x_cl) + cl, x);
#pragma unroll
      for (int i = 0; i < C; ++i) {
        float s = d[i];
#pragma unroll
        for (int o = 0; o < C; ++o) s = fmaf(w_s[o * C + i], x[o], s);
        d[i] = s;
      }
    }
    if (a.g_in) {
      float g[32];
      ld32(static_cast<const T*>(a.g_in) + cl, g);
#pragma unroll
      for (int i = 0; i < C; ++i) d[i] *= g[i];
    }
    if (a.out_cl) st32(static_cast<T*>(a.out_cl) + cl, d);
    if (a.out_cf) {
      T* cf = static_cast<T*>(a.out_cf) + (size_t)b * C * a.P + p;
#pragma unroll
      for (int i = 0; i < C; ++i) cf[(size_t)i * a.P] = from_f<T>(d[i]);
    }
  } else {  // EPI_DW: row = 32 s + o of group g = row / 128; chunk c = (col0 % 128) / 32
    const int g = row / 128, s = (row % 128) / C, o = row % C, c = (col0 % 128) / C;
    if (c != s) return;
    float* dst = a.out + ((((size_t)g * a.splits + split) * 4 + s) * C + o) * C;
    const bool valid = g * 4 + s < a.B;
#pragma unroll
    for (int j = 0; j < 32; j += 4)
      *reinterpret_cast<float4*>(dst + j) = valid ? make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3])
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ---- launchers ---------------------------------------------------------------------------
// Tensor-core GEMM D = A B^T over K (bf16, K-major, TMA maps with 128-byte swizzle and
// a 64-element inner box): A rows in boxes of 128, B rows in boxes of BN (32..256).
// grid = (ceil(M/128), ceil(N/BN), splits); EPI_DW uses grid.x = groups and the same row
// offset for A and B. Each split covers kper 64-wide K blocks.
// EPI_LAYER_*: mA2 / mW are the 1x1-convolution operands (channel-first activations [B][C][P]
// as a 3D map with box {64, 32, kSeg2Samples} and 128-byte swizzle, read MN-major; W or W^T
// [C][C] with box {32, 32} and 64-byte swizzle); they run on the tensor cores as one extra
// K = 32 segment per sample of the tile, into that sample's 32 columns, kSeg2Samples samples
// per operand stage.
cudaError_t launch_gemm_tc(int epi, int BN, const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mA2,
                           const CUtensorMap& mW, const EpiArgs& ea, int M, int N, int K, int splits, int* err,
                           uint64_t timeout_ns, cudaStream_t st);
// Backward truncated DFT of dZ (EPI_MODES into ea, N = 2 m^2 = 512 columns, two tiles of 256)
// fused with the weight gradient (EPI_DW into ew, ew.splits = 2: the two column tiles each take one
// half of K = pixels, a multiple of 128): mA = dZ channel-first, mB = the DFT table D, mV = V
// channel-first (box 128 rows). Tensor-core (BF16) mode only.
cudaError_t launch_gemm_dft_dw(const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mV,
                               const EpiArgs& ea, const EpiArgs& ew, int M, int N, int K, int* err,
                               uint64_t timeout_ns, cudaStream_t st);
// FP32 SIMT GEMM with the same semantics (A [M][lda], B [N][ldb] row-major FP32; for EPI_DW
// rows of B are offset like rows of A).
cudaError_t launch_gemm_simt(int epi, const float* A, long long lda, const float* B, long long ldb,
                             const EpiArgs& ea, int M, int N, int K, int splits, cudaStream_t st);
int gemm_tc_ctas_per_sm(int BN);

// encode a 2D bf16 tensor map: `rows` rows of `cols` elements (row pitch `pitch` elements),
// box {box_cols, box_rows} with box_cols 64 (128-byte swizzle) or 32 (64-byte swizzle),
// out-of-bounds elements read as zero
scw_status make_map_bf16(CUtensorMap* m, const void* base, long long cols, long long rows, long long pitch,
                         int box_rows, int box_cols = 64);
// 1x1-convolution samples per operand stage of the layer products
constexpr int kSeg2Samples = 4;
// encode the 3D bf16 tensor map of channel-first activations [samples][C][P] (P a multiple of
// 128) for the 1x1 convolution: box {64 pixels, C, kSeg2Samples samples}, 128-byte swizzle,
// out-of-bounds samples read as zero
scw_status make_map_act3d(CUtensorMap* m, const void* base, long long P, long long samples);

template <typename T>
cudaError_t launch_tables(T* D, T* E, int N, int m, int Kp, cudaStream_t st);
template <typename T>
cudaError_t launch_lift(const float2* n, const T* params, T* Vcf, T* Vcl, int B, int S, int in_grid, int N,
                        cudaStream_t st);
// mode-major spectra: Vh[split][mode][ld] complex, row b C + i
template <typename T>
cudaError_t launch_mix_fwd(const float2* Vh, int splits, long long split_stride, long long ld, const T* R, T* Wh,
                           float scale, int B, int m, int Kp, cudaStream_t st);
template <typename T>
cudaError_t launch_mix_bwd(const float2* G, const float2* Vh, int splits, long long split_stride, long long ld,
                           const T* R, T* GVh, float* part, int B, int m, int Kp, int N, bool with_gvh,
                           cudaStream_t st);
// Tensor-core mixing (BF16 mode, fno_mix_tc.cu): conj = false is the forward product (out = Wh,
// scale 1/N^2), conj = true the backward-data product (out = GVh, scale 1).
cudaError_t launch_mix_tc(bool conj, const float2* X, int splits, long long split_stride, long long ld,
                          const __nv_bfloat16* R, __nv_bfloat16* out, float scale, int B, int m, int Kp, int* err,
                          uint64_t timeout_ns, cudaStream_t st);
// Tensor-core weight gradient of the mixing (BF16 mode): per block of 128 samples the partial
// dR[k][o][i] = sum_b G conj(Vh) and, in the DC mode's block, the bias partial (layout of mix_bwd's
// partial rows); mix_dr_blocks(B) rows.
cudaError_t launch_mix_dr_tc(const float2* G, const float2* V, int splits, long long split_stride, long long ld,
                             float* part, int B, int m, int N, int* err, uint64_t timeout_ns, cudaStream_t st);
int mix_dr_blocks(int B);
int mix_sample_blocks(int B);
template <typename T>
cudaError_t launch_transpose_w(const T* wcopy, long long off_W0, long long layer_stride, T* WT, int L,
                               cudaStream_t st);
cudaError_t launch_target_norm(const float2* target, float* part, int B, int P, cudaStream_t st);
template <typename T>
cudaError_t launch_project_train(const T* Vcl, const float2* target, const T* params_q, const float* part_tn, T* dZcf,
                                 T* dZcl, float* part_err, float* part_pool, float* part_proj, int B, int P,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_head(const float* part_tn, const float* part_err, const float* part_pool, const T* params_e,
                        float* part_head, float* h_out, float* rel2_out, int B, int P, cudaStream_t st);
template <typename T>
cudaError_t launch_lift_bwd(const T* dV0cl, const float2* n, float* part, int B, int S, int in_grid, int N,
                            cudaStream_t st);
cudaError_t launch_reduce_rows_ex(const float* part, int rows, int width, long long pitch, float scale, float* out,
                                  float* scratch, cudaStream_t st);

// One deterministic partial-sum reduction out[j] += sum_r part[r pitch + j] of a set, all run by
// two launches (reduce_segments). Rows above 256 are summed in ry chunks of `chunk` rows into
// `scratch` ([ry][width]) and the chunks then in a second pass, with the same order of additions
// as launch_reduce_rows_ex.
struct RedSeg {
  const float* part;
  float* out;
  float* scratch;
  long long pitch;
  int rows, width, ry, chunk;
  int item1, item2;  // first item of this segment in pass 1 (gx ry blocks) and pass 2 (gx blocks, ry > 1)
  int wide;          // rows <= 8: each block takes 256 columns and each thread sums its column's rows
};
// Fills ry, chunk, item1, item2 and the scratch slices (from `scratch`, of `scratch_floats`);
// returns false if the scratch is too small.
bool plan_reduce_segments(std::vector<RedSeg>& segs, float* scratch, size_t scratch_floats, int& items1, int& items2);
cudaError_t launch_reduce_segments(const RedSeg* d_segs, int nseg, int items1, int items2, cudaStream_t st);
template <typename T>
cudaError_t launch_adam(float* master, const float* grad, float* m, float* v, T* copy, long long n, float lr,
                        float bc1, float bc2, cudaStream_t st);
template <typename T>
cudaError_t launch_copy_params(const float* master, T* copy, long long n, cudaStream_t st);
template <typename T>
cudaError_t launch_project_infer(const T* Vcl, const T* params_q, float2* field, float* part_pool, int B, int P,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_head_infer(const float* part_pool, const T* params_e, float q, float threshold, float* h_out,
                              float* est, unsigned char* flag, int B, int P, cudaStream_t st);

}  // namespace fno
}  // namespace scw
