// The surrogate's SIMT kernels: DFT tables, lift, per-mode complex mixing
// (forward and backward), projection + loss, error head, lift backward,
// deterministic partial-sum reduction and Adam. Element type T is BF16 in the
// training mode and FP32 in the test mode; accumulations are FP32 throughout.
// Definitions of every quantity are in include/scw_fno.h.
#include "fno_internal.cuh"

namespace scw {
namespace fno {

// ---- DFT tables: D[2k + r][p] = cos(theta) (r = 0) or -sin(theta) (r = 1), E = D^T (pads zero)
// theta = 2 pi ((kx x + ky y) mod N) / N, reduced exactly in integers, evaluated in FP64.
template <typename T>
__global__ void tables_kernel(T* __restrict__ D, T* __restrict__ E, int N, int m, int Kp) {
  const int P = N * N, Kc = 2 * m * m;
  const long long total = (long long)Kc * P;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / P), p = (int)(idx % P);
    const int k = q >> 1;
    const int ky = k / m - m / 2, kx = k % m - m / 2;
    const int y = p / N, x = p % N;
    const int r = (((kx * x + ky * y) % N) + N) % N;
    double s, c;
    sincospi(2.0 * r / N, &s, &c);
    const float v = (q & 1) ? (float)-s : (float)c;
    D[(size_t)q * P + p] = from_f<T>(v);
    E[(size_t)p * Kp + q] = from_f<T>(v);
  }
}

// ---- lift: V_0 = P a + p, a = (Re n - 1, Im n) per slice, nearest upsampling.
// One thread per input pixel: the r x r output pixels it covers share one value.
// The 32 channels are produced eight at a time and stored at once, channel-last
// (one 16-byte chunk per output pixel in BF16) and channel-first (pairs of
// horizontally adjacent pixels in one store when r is even), so that few outputs
// are live at a time. Only the float4 groups of features that can be non-zero
// (the first 2S) enter the products.
template <typename T>
__device__ __forceinline__ void st_same_pair(T* p, float v);
template <>
__device__ __forceinline__ void st_same_pair<float>(float* p, float v) {
  *reinterpret_cast<float2*>(p) = make_float2(v, v);
}
template <>
__device__ __forceinline__ void st_same_pair<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v, v);
}

// 8 contiguous values (p 16-byte aligned)
template <typename T>
__device__ __forceinline__ void st8(T* p, const float (&v)[8]) {
  if constexpr (sizeof(T) == 4) {
    float4* q = reinterpret_cast<float4*>(p);
    q[0] = make_float4(v[0], v[1], v[2], v[3]);
    q[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    *reinterpret_cast<uint4*>(p) = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                              pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 3) lift_kernel(const float2* __restrict__ n, const T* __restrict__ prm,
                                                   T* __restrict__ Vcf, T* __restrict__ Vcl, int B, int S,
                                                   int in_grid, int N) {
  __shared__ __align__(16) float Ps[C * 32];  // [c][32], zero-padded past 2S
  __shared__ float ps[C];
  const int cin = 2 * S;
  for (int i = threadIdx.x; i < C * 32; i += blockDim.x) {
    const int c = i / 32, j = i % 32;
    Ps[i] = j < cin ? to_f(prm[c * cin + j]) : 0.f;
  }
  if (threadIdx.x < C) ps[threadIdx.x] = to_f(prm[C * cin + threadIdx.x]);
  __syncthreads();
  const int P = N * N, Pi = in_grid * in_grid, r = N / in_grid;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)B * Pi) return;
  const int b = (int)(idx / Pi), pi = (int)(idx % Pi);
  const int yi = pi / in_grid, xi = pi % in_grid;
  float a[32];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    float2 v = make_float2(1.f, 0.f);
    if (s < S) v = n[(((size_t)b * S + s) * in_grid + yi) * in_grid + xi];
    a[2 * s] = v.x - 1.0f;
    a[2 * s + 1] = v.y;
  }
  const float4* P4 = reinterpret_cast<const float4*>(Ps);
  const int nf4 = (cin + 3) / 4;  // float4 groups of features that can be non-zero
#pragma unroll 1
  for (int q = 0; q < C / 8; ++q) {
    float o[8];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int c = 8 * q + cc;
      float t = ps[c];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (i < nf4) {
          const float4 w = P4[c * 8 + i];
          t = fmaf(w.x, a[4 * i], fmaf(w.y, a[4 * i + 1], fmaf(w.z, a[4 * i + 2], fmaf(w.w, a[4 * i + 3], t))));
        }
      }
      o[cc] = t;
    }
    for (int dy = 0; dy < r; ++dy) {
      const int row = (yi * r + dy) * N + xi * r;
      if (Vcl != nullptr)  // the channel-last copy only where a consumer reads it (FP32 mode)
        for (int dx = 0; dx < r; ++dx) st8(Vcl + ((size_t)b * P + row + dx) * C + 8 * q, o);
      T* cf = Vcf + ((size_t)b * C + 8 * q) * P + row;
      if ((r & 1) == 0) {
        for (int dx = 0; dx < r; dx += 2) {
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) st_same_pair(cf + (size_t)cc * P + dx, o[cc]);
        }
      } else {
        for (int dx = 0; dx < r; ++dx) {
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) cf[(size_t)cc * P + dx] = from_f<T>(o[cc]);
        }
      }
    }
  }
}

// ---- mixing (per kept mode k, complex C x C), spectra mode-major Vh[split][k][b C + i] ------
// Per kept mode and block of 32 samples the mixing is a 32 x 32 complex product over 32 terms. The
// operands are staged in shared memory as [32][34] complex tiles (16-byte aligned rows) and each
// thread computes a 4 x 4 register tile. The forward takes NM = 4 consecutive modes per CTA (m is
// a multiple of 4, so m^2 is a multiple of NM), so that each (sample, channel) row of the K-major
// output Wh receives its four modes in one 16-byte store; the backward takes one mode per CTA.
constexpr int MIX_SAMPLES = 32;
constexpr int MIX_MODES_FWD = 4;
constexpr int MIX_LD = C + 2;          // row stride of a staged tile (float2): rows stay 16-byte aligned
constexpr int MIX_TILE = C * MIX_LD;   // float2 elements of one staged [32][34] tile

template <typename T>
__device__ __forceinline__ float2 ld_pair(const T* base, size_t pair);
template <>
__device__ __forceinline__ float2 ld_pair<float>(const float* base, size_t pair) {
  return reinterpret_cast<const float2*>(base)[pair];
}
template <>
__device__ __forceinline__ float2 ld_pair<__nv_bfloat16>(const __nv_bfloat16* base, size_t pair) {
  const uint32_t w = reinterpret_cast<const uint32_t*>(base)[pair];
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

template <typename T>
__device__ __forceinline__ void st_pair(T* base, size_t pair, float2 v);
template <>
__device__ __forceinline__ void st_pair<float>(float* base, size_t pair, float2 v) {
  reinterpret_cast<float2*>(base)[pair] = v;
}
template <>
__device__ __forceinline__ void st_pair<__nv_bfloat16>(__nv_bfloat16* base, size_t pair, float2 v) {
  reinterpret_cast<__nv_bfloat162*>(base)[pair] = __floats2bfloat162_rn(v.x, v.y);
}

// NM consecutive complex values (pairs pair .. pair + NM - 1); 16-byte aligned when NM = 4
template <typename T, int NM>
__device__ __forceinline__ void st_pairs(T* base, size_t pair, const float (&re)[NM], const float (&im)[NM]) {
  if constexpr (NM == 4 && sizeof(T) == 2) {
    uint4 u;
    u.x = pack_bf16x2(re[0], im[0]);
    u.y = pack_bf16x2(re[1], im[1]);
    u.z = pack_bf16x2(re[2], im[2]);
    u.w = pack_bf16x2(re[3], im[3]);
    *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat162*>(base) + pair) = u;
  } else if constexpr (NM == 4) {
    float4* q = reinterpret_cast<float4*>(reinterpret_cast<float2*>(base) + pair);
    q[0] = make_float4(re[0], im[0], re[1], im[1]);
    q[1] = make_float4(re[2], im[2], re[3], im[3]);
  } else if constexpr (NM == 2 && sizeof(T) == 2) {
    *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat162*>(base) + pair) =
        make_uint2(pack_bf16x2(re[0], im[0]), pack_bf16x2(re[1], im[1]));
  } else if constexpr (NM == 2) {
    *reinterpret_cast<float4*>(reinterpret_cast<float2*>(base) + pair) = make_float4(re[0], im[0], re[1], im[1]);
  } else {
#pragma unroll
    for (int kk = 0; kk < NM; ++kk) st_pair(base, pair + kk, make_float2(re[kk], im[kk]));
  }
}

// split-summed complex value of a mode-major spectrum
__device__ __forceinline__ float2 ld_spec(const float2* __restrict__ X, size_t off, int splits,
                                          long long split_stride) {
  float2 v = X[off];
  for (int z = 1; z < splits; ++z) {
    const float2 u = X[off + (size_t)z * split_stride];
    v.x += u.x;
    v.y += u.y;
  }
  return v;
}

// Per-mode products as 4 x 4 register tiles: each k-step reads its four values of each operand from one
// staged row in two 16-byte loads (no operand is read as a warp-wide broadcast per product), and a
// thread then does 16 complex multiply-adds.
__device__ __forceinline__ void ld4c(const float2* p, float2 (&v)[4]) {  // p 16-byte aligned
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = make_float2(a.x, a.y);
  v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y);
  v[3] = make_float2(b.z, b.w);
}

// R staged as the parameters' own complex pairs: BF16 pairs (one 32-bit word, rows of 36 words) or
// FP32 pairs (float2, rows of MIX_LD); four consecutive outputs are one 16-byte aligned group.
template <typename T>
struct MixRStage;
template <>
struct MixRStage<__nv_bfloat16> {
  using E = uint32_t;
  static constexpr int LD = C + 4;
  __device__ static E load(const __nv_bfloat16* R, size_t pair) { return reinterpret_cast<const uint32_t*>(R)[pair]; }
  __device__ static void ld4(const E* p, float2 (&v)[4]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = make_float2(__uint_as_float(w[c] << 16), __uint_as_float(w[c] & 0xffff0000u));
  }
};
template <>
struct MixRStage<float> {
  using E = float2;
  static constexpr int LD = MIX_LD;
  __device__ static E load(const float* R, size_t pair) { return reinterpret_cast<const float2*>(R)[pair]; }
  __device__ static void ld4(const E* p, float2 (&v)[4]) { ld4c(p, v); }
};
template <typename T>
constexpr size_t mix_fwd_rs_bytes(int NM) {
  return (size_t)NM * C * MixRStage<T>::LD * sizeof(typename MixRStage<T>::E);
}

// forward: Wh[b][o][k] = scale sum_i R[k][o][i] Vh[b][i][k]
// Thread t owns the tile (mode kk = t / 64, samples 4 sg .. 4 sg + 3, outputs 4 og .. 4 og + 3) with
// sg = (t % 64) / 8 and og = t % 8; R is staged [mode][i][o] and V [mode][i][s]. The results pass
// through shared memory ([mode][s][o]) so that each (sample, output) row of Wh receives its NM modes
// in one store.
template <typename T, int NM>
__global__ void __launch_bounds__(256) mix_fwd_kernel(const float2* __restrict__ Vh, int splits,
                                                      long long split_stride, long long ld, const T* __restrict__ R,
                                                      T* __restrict__ Wh, float scale, int B, int Kp) {
  static_assert(NM * 64 == 256, "one 64-thread group per mode");
  using RS = MixRStage<T>;
  constexpr int RT = C * RS::LD;  // staged R elements per mode
  extern __shared__ __align__(16) float2 mix_smem[];
  typename RS::E* Rs = reinterpret_cast<typename RS::E*>(mix_smem);  // [mode][i][o]
  float2* Vs = reinterpret_cast<float2*>(reinterpret_cast<uint8_t*>(mix_smem) + mix_fwd_rs_bytes<T>(NM));
  // Vs: [mode][i][s], then the results [mode][s][o]
  const int k0 = blockIdx.x * NM, b0 = blockIdx.y * MIX_SAMPLES;
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4 * NM; ++q) {
    const int idx = t + 256 * q, kk = idx / (C * C), row = (idx / C) % C, col = idx % C;
    Rs[kk * RT + col * RS::LD + row] = RS::load(R, ((size_t)(k0 + kk) * C + row) * C + col);
    const int b = b0 + row;
    Vs[kk * MIX_TILE + col * MIX_LD + row] =
        b < B ? ld_spec(Vh, (size_t)(k0 + kk) * ld + (size_t)b * C + col, splits, split_stride)
              : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int kk = t >> 6, sg = (t & 63) >> 3, og = t & 7;
  float re[4][4], im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) re[a][c] = im[a][c] = 0.f;
  const float2* vb = Vs + kk * MIX_TILE + 4 * sg;
  const typename RS::E* rb = Rs + kk * RT + 4 * og;
#pragma unroll 4
  for (int i = 0; i < C; ++i) {
    float2 v[4], r[4];
    ld4c(vb + i * MIX_LD, v);
    RS::ld4(rb + i * RS::LD, r);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        re[a][c] = fmaf(r[c].x, v[a].x, fmaf(-r[c].y, v[a].y, re[a][c]));
        im[a][c] = fmaf(r[c].x, v[a].y, fmaf(r[c].y, v[a].x, im[a][c]));
      }
  }
  __syncthreads();  // every tile is done with Vs
  float2* Os = Vs;  // [mode][s][o], row stride MIX_LD
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      Os[kk * MIX_TILE + (4 * sg + a) * MIX_LD + 4 * og + c] = make_float2(scale * re[a][c], scale * im[a][c]);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < C * MIX_SAMPLES / 256; ++q) {
    const int p = t + 256 * q, sm = p / C, o = p % C, b = b0 + sm;
    if (b >= B) continue;
    float xr[NM], xi[NM];
#pragma unroll
    for (int m2 = 0; m2 < NM; ++m2) {
      const float2 x = Os[m2 * MIX_TILE + sm * MIX_LD + o];
      xr[m2] = x.x;
      xi[m2] = x.y;
    }
    st_pairs<T, NM>(Wh, (((size_t)b * C + o) * Kp) / 2 + k0, xr, xi);
  }
}

// Split row layout of a staged 32-complex row: element j at split_pos(j), so that the two halves
// (j, j + 1) and (j + 2, j + 3) of every aligned group of four sit in two separate 128-byte runs. Eight
// lanes reading eight different groups then touch 128 contiguous bytes per 16-byte load.
// The split layout puts the second half-group at offset 16 and loads 16-byte pairs: it assumes
// 32-element rows and an even row stride.
static_assert(C == 32 && MIX_LD % 2 == 0, "split_pos/ld4s assume C == 32 and an even MIX_LD");
__device__ __forceinline__ int split_pos(int j) { return ((j & 2) << 3) + ((j >> 2) << 1) + (j & 1); }
__device__ __forceinline__ void ld4s(const float2* row, int g, float2 (&v)[4]) {  // group g of a split row
  const float4 a = *reinterpret_cast<const float4*>(row + 2 * g);
  const float4 b = *reinterpret_cast<const float4*>(row + 16 + 2 * g);
  v[0] = make_float2(a.x, a.y);
  v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y);
  v[3] = make_float2(b.z, b.w);
}

// backward (G = dL/dRe + i dL/dIm convention):
//   GVh[b][i][k] = sum_o conj(R[k][o][i]) G[b][o][k]
//   part dR[k][o][i] = sum_b G[b][o][k] conj(Vh[b][i][k])   (this CTA's samples)
//   part dc[o] = N^2 sum_b Re G[b][o][k_dc]                   (the DC mode carries sum_x dZ / N^2)
// part row (one per sample block): [m^2][C][C][2] then [C]
// One CTA per (kept mode, block of 32 samples), 128 threads: threads 0-63 own GVh tiles (samples
// 4 sg .., channels 4 ig ..), threads 64-127 dR tiles (outputs 4 og .., channels 4 ig ..). G is
// staged both as [s][o] and as [o][s], so each product reads its rows contiguously; the rows read
// by eight different groups per warp use the split layout. with_gvh = 0 leaves GVh to the
// tensor-core mixing (BF16 mode): only the dR and dc parts run.
template <typename T>
__global__ void __launch_bounds__(128) mix_bwd_kernel(const float2* __restrict__ G, const float2* __restrict__ Vh,
                                                      int splits, long long split_stride, long long ld,
                                                      const T* __restrict__ R, T* __restrict__ GVh,
                                                      float* __restrict__ part, int B, int m, int Kp, int N,
                                                      int with_gvh) {
  extern __shared__ __align__(16) float2 mix_smem[];
  float2* Rs = mix_smem;                 // [o][i], split rows
  float2* Gs = mix_smem + MIX_TILE;      // [s][o], split rows
  float2* Gt = mix_smem + 2 * MIX_TILE;  // [o][s]
  float2* Vs = mix_smem + 3 * MIX_TILE;  // [s][i], split rows
  const int k = blockIdx.x, b0 = blockIdx.y * MIX_SAMPLES;
  const int t = threadIdx.x;
  const int kdc = (m / 2) * m + m / 2;
  const size_t row0 = (size_t)blockIdx.y * ((size_t)m * m * C * C * 2 + C);
#pragma unroll
  for (int q = 0; q < (C * C) / 128; ++q) {
    const int idx = t + 128 * q, row = idx / C, col = idx % C, sc = split_pos(col);
    Rs[row * MIX_LD + sc] = ld_pair(R, ((size_t)k * C + row) * C + col);
    const int b = b0 + row;
    const size_t off = (size_t)k * ld + (size_t)b * C + col;
    const float2 g = b < B ? ld_spec(G, off, splits, split_stride) : make_float2(0.f, 0.f);
    Gs[row * MIX_LD + sc] = g;
    if (with_gvh) Gt[col * MIX_LD + row] = g;
    Vs[row * MIX_LD + sc] = b < B ? ld_spec(Vh, off, splits, split_stride) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float re[4][4], im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) re[a][c] = im[a][c] = 0.f;
  if (t < 64 && with_gvh) {
    // GVh tile: samples 4 sg + a, channels 4 ig + c; conj(r) g over the outputs o
    const int sg = t >> 3, ig = t & 7;
#pragma unroll 4
    for (int o = 0; o < C; ++o) {
      float2 g[4], r[4];
      ld4c(Gt + o * MIX_LD + 4 * sg, g);
      ld4s(Rs + o * MIX_LD, ig, r);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          re[a][c] = fmaf(r[c].x, g[a].x, fmaf(r[c].y, g[a].y, re[a][c]));
          im[a][c] = fmaf(r[c].x, g[a].y, fmaf(-r[c].y, g[a].x, im[a][c]));
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int b = b0 + 4 * sg + a;
      if (b >= B) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        st_pair(GVh, (((size_t)b * C + 4 * ig + c) * Kp) / 2 + k, make_float2(re[a][c], im[a][c]));
    }
  } else if (t >= 64) {
    // dR tile: outputs 4 og + a, channels 4 ig + c; g conj(v) over the block's samples
    const int og = (t - 64) >> 3, ig = t & 7;
#pragma unroll 4
    for (int sm = 0; sm < MIX_SAMPLES; ++sm) {
      float2 g[4], v[4];
      ld4s(Gs + sm * MIX_LD, og, g);
      ld4s(Vs + sm * MIX_LD, ig, v);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          re[a][c] = fmaf(g[a].x, v[c].x, fmaf(g[a].y, v[c].y, re[a][c]));
          im[a][c] = fmaf(g[a].y, v[c].x, fmaf(-g[a].x, v[c].y, im[a][c]));
        }
    }
    float4* dst = reinterpret_cast<float4*>(part + row0);  // complex pairs (c, c + 1)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const size_t e = ((size_t)k * C + 4 * og + a) * C + 4 * ig;  // complex index, a multiple of 4
      dst[e / 2] = make_float4(re[a][0], im[a][0], re[a][1], im[a][1]);
      dst[e / 2 + 1] = make_float4(re[a][2], im[a][2], re[a][3], im[a][3]);
    }
  }
  if (k == kdc && t < C) {
    float d = 0.f;
    for (int sm = 0; sm < MIX_SAMPLES; ++sm) d += Gs[sm * MIX_LD + split_pos(t)].x;
    part[row0 + (size_t)m * m * C * C * 2 + t] = d * (float)N * (float)N;
  }
}

// W^T of every layer (the backward 1x1 convolution's tensor-core operand): WT[l][i][o] = W_l[o][i]
template <typename T>
__global__ void transpose_w_kernel(const T* __restrict__ wcopy, long long off_W0, long long layer_stride,
                                   T* __restrict__ WT, int L) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L * C * C) return;
  const int l = idx / (C * C), i = (idx / C) % C, o = idx % C;
  WT[idx] = wcopy[off_W0 + (long long)l * layer_stride + o * C + i];
}

// ---- projection, loss and their gradient (training) ----------------------------------------
// part_tn[b][blk] = sum over the block's pixels of |T|^2
__global__ void __launch_bounds__(256) target_norm_kernel(const float2* __restrict__ target, float* __restrict__ part,
                                                          int P) {
  __shared__ float red[8];
  const int b = blockIdx.y, p = blockIdx.x * PIX_BLOCK + threadIdx.x;
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 v = target[((size_t)b * 3 + c) * P + p];
    s += v.x * v.x + v.y * v.y;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[(size_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// F = Q v + q; d = F - T; dF = 2 d / (B ||T_b||^2); dV_L = Q^T dF (= dZ of the last layer).
// Per block of 256 pixels of one sample it also writes the partial sums
//   part_proj row [6 C + 6]: dQ[j][o] = sum_p dF[j][p] V[o][p], dq[j] = sum_p dF[j][p]
//   part_err = sum_p |d|^2, part_pool[C] = sum_p V[o][p]
template <typename T>
__global__ void __launch_bounds__(256, 2) project_train_kernel(const T* __restrict__ Vcl,
                                                               const float2* __restrict__ target,
                                                               const T* __restrict__ prm_q,
                                                               const float* __restrict__ part_tn,
                                                               T* __restrict__ dZcf, T* __restrict__ dZcl,
                                                               float* __restrict__ part_err,
                                                               float* __restrict__ part_pool,
                                                               float* __restrict__ part_proj, int B, int P) {
  __shared__ __align__(16) float Qs[OUT * C + OUT];
  // the block sums below are one product F' V' over the block's pixels: F' = (dF rows, a row of
  // ones, a zero row), V' = (V columns, a column of ones, zero columns)
  __shared__ __align__(16) float Vs[PIX_BLOCK][C + 4];
  __shared__ __align__(16) float Fs[PIX_BLOCK][OUT + 2];  // pixel-major: a tile's two rows in one load
  __shared__ float red[8];
  __shared__ float tn_s;
  const int nblk = gridDim.x, b = blockIdx.y, t = threadIdx.x, p = blockIdx.x * PIX_BLOCK + t;
  for (int i = t; i < OUT * C + OUT; i += blockDim.x) Qs[i] = to_f(prm_q[i]);
  if (t == 0) {
    float s = 0.f;
    for (int j = 0; j < nblk; ++j) s += part_tn[(size_t)b * nblk + j];
    tn_s = s;
  }
  __syncthreads();
  float v[32];
  ld32(Vcl + ((size_t)b * P + p) * C, v);
#pragma unroll
  for (int o = 0; o < C; o += 4) *reinterpret_cast<float4*>(&Vs[t][o]) = make_float4(v[o], v[o + 1], v[o + 2], v[o + 3]);
  *reinterpret_cast<float4*>(&Vs[t][C]) = make_float4(1.f, 0.f, 0.f, 0.f);
  const float4* Q4 = reinterpret_cast<const float4*>(Qs);  // row j: Q4[8 j .. 8 j + 8)
  float d[OUT];
#pragma unroll
  for (int j = 0; j < OUT; ++j) {
    float f = Qs[OUT * C + j];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 q = Q4[8 * j + i];
      f = fmaf(q.x, v[4 * i], fmaf(q.y, v[4 * i + 1], fmaf(q.z, v[4 * i + 2], fmaf(q.w, v[4 * i + 3], f))));
    }
    const float2 tv = target[((size_t)b * 3 + j / 2) * P + p];
    d[j] = f - ((j & 1) ? tv.y : tv.x);
  }
  float e2 = 0.f;
  const float sc = 2.0f / ((float)B * tn_s);
#pragma unroll
  for (int j = 0; j < OUT; ++j) {
    e2 = fmaf(d[j], d[j], e2);
    d[j] *= sc;
  }
  static_assert(OUT == 6, "F' rows: six outputs, a row of ones, a zero row");
  *reinterpret_cast<float4*>(&Fs[t][0]) = make_float4(d[0], d[1], d[2], d[3]);
  *reinterpret_cast<float4*>(&Fs[t][4]) = make_float4(d[4], d[5], 1.f, 0.f);
  __syncwarp();  // Q is re-read from shared memory below rather than held in registers across both products
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < OUT; ++j) {
      const float4 q = Q4[8 * j + i];
      acc.x = fmaf(q.x, d[j], acc.x);
      acc.y = fmaf(q.y, d[j], acc.y);
      acc.z = fmaf(q.z, d[j], acc.z);
      acc.w = fmaf(q.w, d[j], acc.w);
    }
    v[4 * i] = acc.x;  // v now holds dV_L
    v[4 * i + 1] = acc.y;
    v[4 * i + 2] = acc.z;
    v[4 * i + 3] = acc.w;
  }
  if (dZcl != nullptr) st32(dZcl + ((size_t)b * P + p) * C, v);  // read channel-last in FP32 mode only
  T* cf = dZcf + (size_t)b * C * P + p;
#pragma unroll
  for (int o = 0; o < C; ++o) cf[(size_t)o * P] = from_f<T>(v[o]);
#pragma unroll
  for (int o = 16; o; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  if ((t & 31) == 0) red[t >> 5] = e2;
  __syncthreads();
  const size_t blk = (size_t)b * nblk + blockIdx.x;
  if (t == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += red[w];
    part_err[blk] = s;
  }
  // block sums over the 256 pixels: the product F' V' as 2 x 4 register tiles (rows 2 jp, 2 jp + 1;
  // columns 4 og .. 4 og + 3), the pixels split over NSPLIT threads per tile (q = split + NSPLIT i),
  // then the splits summed in a fixed order:
  //   part_proj row: dQ[j][o] = (F' V')[j][o], dq[j] = (F' V')[j][C]; part_pool[o] = (F' V')[OUT][o]
  constexpr int NJP = (OUT + 2) / 2, NOG = (C + 4) / 4, NT = NJP * NOG, NSPLIT = 256 / NT;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  if (t < NT * NSPLIT) {
    const int tile = t % NT, split = t / NT, jp = tile / NOG, og = tile % NOG;
    for (int q = split; q < PIX_BLOCK; q += NSPLIT) {
      const float2 f01 = *reinterpret_cast<const float2*>(&Fs[q][2 * jp]);
      const float f0 = f01.x, f1 = f01.y;
      const float4 w4 = *reinterpret_cast<const float4*>(&Vs[q][4 * og]);
      acc[0][0] = fmaf(f0, w4.x, acc[0][0]);
      acc[0][1] = fmaf(f0, w4.y, acc[0][1]);
      acc[0][2] = fmaf(f0, w4.z, acc[0][2]);
      acc[0][3] = fmaf(f0, w4.w, acc[0][3]);
      acc[1][0] = fmaf(f1, w4.x, acc[1][0]);
      acc[1][1] = fmaf(f1, w4.y, acc[1][1]);
      acc[1][2] = fmaf(f1, w4.z, acc[1][2]);
      acc[1][3] = fmaf(f1, w4.w, acc[1][3]);
    }
  }
  __syncthreads();
  float* red_s = &Vs[0][0];  // the tiles' partial sums [NT NSPLIT][8], over V' (no longer read)
  if (t < NT * NSPLIT) {
#pragma unroll
    for (int e = 0; e < 8; ++e) red_s[t * 8 + e] = acc[e / 4][e % 4];
  }
  __syncthreads();
  for (int q = t; q < OUT * C + OUT + C; q += blockDim.x) {
    int j, o;
    if (q < OUT * C) {
      j = q / C;
      o = q % C;
    } else if (q < OUT * C + OUT) {
      j = q - OUT * C;
      o = C;
    } else {
      j = OUT;
      o = q - OUT * C - OUT;
    }
    const int tile = (j / 2) * NOG + o / 4, e = 4 * (j % 2) + o % 4;
    float sum = 0.f;
    for (int sp = 0; sp < NSPLIT; ++sp) sum += red_s[(sp * NT + tile) * 8 + e];
    if (q < OUT * C + OUT)
      part_proj[blk * (OUT * C + OUT) + q] = sum;
    else
      part_pool[blk * C + o] = sum;
  }
}

// error head and the loss, one warp per sample (lane = channel): h = e . pool + e0,
// rel2 = ||F - T||^2 / ||T||^2, tgt = log(rel2 + 1e-12) / 2, dh = 2 (h - tgt) / B.
// part_head row [C + 3]: dh pool[0..C), dh, rel2 / B, (h - tgt)^2 / B, summed over samples
// into (grad e, grad e0) and (L_field, L_head) by the caller.
template <typename T>
__global__ void __launch_bounds__(256) head_kernel(const float* __restrict__ part_tn, const float* __restrict__ part_err,
                                                   const float* __restrict__ part_pool, const T* __restrict__ prm_e,
                                                   float* __restrict__ part_head, float* __restrict__ h_out,
                                                   float* __restrict__ rel2_out, int B, int nblk, int P) {
  const int lane = threadIdx.x & 31, b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= B) return;
  float pool = 0.f, tn = 0.f, e2 = 0.f;
  for (int j = 0; j < nblk; ++j) pool += part_pool[((size_t)b * nblk + j) * C + lane];
  pool /= (float)P;
  for (int j = lane; j < nblk; j += 32) {
    tn += part_tn[(size_t)b * nblk + j];
    e2 += part_err[(size_t)b * nblk + j];
  }
  float h = to_f(prm_e[lane]) * pool;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    h += __shfl_xor_sync(0xffffffffu, h, o);
    tn += __shfl_xor_sync(0xffffffffu, tn, o);
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  }
  h += to_f(prm_e[C]);
  const float rel2 = e2 / tn;
  const float tgt = 0.5f * logf(rel2 + 1e-12f);
  const float dh = 2.0f * (h - tgt) / (float)B;
  float* row = part_head + (size_t)b * (C + 3);
  row[lane] = dh * pool;
  if (lane == 0) {
    row[C] = dh;
    row[C + 1] = rel2 / (float)B;
    row[C + 2] = (h - tgt) * (h - tgt) / (float)B;
    if (h_out) h_out[b] = h;
    if (rel2_out) rel2_out[b] = rel2;
  }
}

// ---- lift backward: part row [C][2S] then [C]: dP[o][c] = sum dV0[o] a[c], dp[o] = sum dV0[o]
// (dV0, channel-last, is summed over each input pixel's r x r block first: a is constant there)
template <typename T>
__global__ void __launch_bounds__(128) lift_bwd_kernel(const T* __restrict__ dV0cl, const float2* __restrict__ n,
                                                       float* __restrict__ part, int B, int S, int in_grid, int N) {
  __shared__ __align__(16) float dv_s[128][C + 4];  // rows 16-byte aligned
  __shared__ __align__(16) float a_s[128][C + 4];   // features, zero past 2S
  __shared__ __align__(16) float red_s[128][16];
  const int cin = 2 * S, P = N * N, Pi = in_grid * in_grid, r = N / in_grid;
  const int t = threadIdx.x;
  const long long idx = blockIdx.x * 128LL + t;
  const bool valid = idx < (long long)B * Pi;
  float dv[32];
#pragma unroll
  for (int o = 0; o < C; ++o) dv[o] = 0.f;
#pragma unroll
  for (int c = 0; c < C; ++c) a_s[t][c] = 0.f;
  if (valid) {
    const int b = (int)(idx / Pi), pi = (int)(idx % Pi);
    const int yi = pi / in_grid, xi = pi % in_grid;
    for (int dy = 0; dy < r; ++dy)
      for (int dx = 0; dx < r; ++dx) {
        float x[32];
        ld32(dV0cl + ((size_t)b * P + (size_t)(yi * r + dy) * N + xi * r + dx) * C, x);
#pragma unroll
        for (int o = 0; o < C; ++o) dv[o] += x[o];
      }
    for (int s = 0; s < S; ++s) {
      const float2 v = n[(((size_t)b * S + s) * in_grid + yi) * in_grid + xi];
      a_s[t][2 * s] = v.x - 1.0f;
      a_s[t][2 * s + 1] = v.y;
    }
  }
#pragma unroll
  for (int o = 0; o < C; o += 4)
    *reinterpret_cast<float4*>(&dv_s[t][o]) = make_float4(dv[o], dv[o + 1], dv[o + 2], dv[o + 3]);
  __syncthreads();
  // dP over the block's 128 pixels as 4 x 4 register tiles (outputs 4 og .. 4 og + 3, features
  // 4 cg .. 4 cg + 3), the pixels split over nsplit threads per tile (pixels j = split + nsplit i),
  // the splits then summed in a fixed order
  const int ncg = (cin + 3) / 4, ntile = (C / 4) * ncg, nsplit = 128 / ntile;
  if (t < ntile * nsplit) {
    const int tile = t % ntile, split = t / ntile, og = tile / ncg, cg = tile % ncg;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int j = split; j < 128; j += nsplit) {
      const float4 d = *reinterpret_cast<const float4*>(&dv_s[j][4 * og]);
      const float4 a = *reinterpret_cast<const float4*>(&a_s[j][4 * cg]);
      const float dd[4] = {d.x, d.y, d.z, d.w}, aa[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(dd[u], aa[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) red_s[t][4 * u + v] = acc[u][v];
  }
  __syncthreads();
  const int width = C * cin + C;
  float* dst = part + (size_t)blockIdx.x * width;
  for (int q = t; q < width; q += 128) {
    float s = 0.f;
    if (q < C * cin) {
      const int o = q / cin, c = q % cin, tile = (o / 4) * ncg + c / 4, e = 4 * (o % 4) + c % 4;
      for (int sp = 0; sp < nsplit; ++sp) s += red_s[sp * ntile + tile][e];
    } else {
      const int o = q - C * cin;
      float s4[4] = {0.f, 0.f, 0.f, 0.f};  // four independent accumulators (pixels j = 4 i + k), fixed order
      for (int j = 0; j < 128; j += 4)
#pragma unroll
        for (int k = 0; k < 4; ++k) s4[k] += dv_s[j + k][o];
      s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    dst[q] = s;
  }
}

// ---- deterministic column sums: block (32, 8) per 32 columns and a chunk of rows
__global__ void __launch_bounds__(256) reduce_rows_kernel(const float* __restrict__ part, int rows, int width,
                                                          long long pitch, int chunk, float scale,
                                                          float* __restrict__ out, float* __restrict__ scratch) {
  __shared__ float red[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
  float s = 0.f;
  if (col < width)
    for (int r = r0 + threadIdx.y; r < r1; r += 8) s += part[(size_t)r * pitch + col];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && col < width) {
    float t = 0.f;
    for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
    if (scratch)
      scratch[(size_t)blockIdx.y * width + col] = t;
    else
      out[col] += scale * t;
  }
}

// ---- Adam (bias-corrected), refreshes the kernels' copy of the parameters
template <typename T>
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, T* __restrict__ copy, long long n, float lr, float bc1, float bc2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    w[i] = wi;
    copy[i] = from_f<T>(wi);
  }
}

template <typename T>
__global__ void copy_params_kernel(const float* __restrict__ w, T* __restrict__ copy, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    copy[i] = from_f<T>(w[i]);
}

// ---- inference: field and the head's estimate --------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) project_infer_kernel(const T* __restrict__ Vcl, const T* __restrict__ prm_q,
                                                            float2* __restrict__ field, float* __restrict__ part_pool,
                                                            int P) {
  __shared__ float Qs[OUT * C + OUT];
  __shared__ float pool_s[PIX_BLOCK][C + 1];
  const int nblk = gridDim.x, b = blockIdx.y, p = blockIdx.x * PIX_BLOCK + threadIdx.x;
  for (int i = threadIdx.x; i < OUT * C + OUT; i += blockDim.x) Qs[i] = to_f(prm_q[i]);
  __syncthreads();
  float v[32];
  ld32(Vcl + ((size_t)b * P + p) * C, v);
#pragma unroll
  for (int o = 0; o < C; ++o) pool_s[threadIdx.x][o] = v[o];
  float f[OUT];
#pragma unroll
  for (int j = 0; j < OUT; ++j) {
    float s = Qs[OUT * C + j];
#pragma unroll
    for (int o = 0; o < C; ++o) s = fmaf(Qs[j * C + o], v[o], s);
    f[j] = s;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) field[((size_t)b * 3 + c) * P + p] = make_float2(f[2 * c], f[2 * c + 1]);
  __syncthreads();
  if (threadIdx.x < C) {
    float s = 0.f;
    for (int r = 0; r < PIX_BLOCK; ++r) s += pool_s[r][threadIdx.x];
    part_pool[((size_t)b * nblk + blockIdx.x) * C + threadIdx.x] = s;
  }
}

template <typename T>
__global__ void head_infer_kernel(const float* __restrict__ part_pool, const T* __restrict__ prm_e, float q,
                                  float threshold, float* __restrict__ h_out, float* __restrict__ est,
                                  unsigned char* __restrict__ flag, int B, int nblk, int P) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float h = to_f(prm_e[C]);
  for (int o = 0; o < C; ++o) {
    float s = 0.f;
    for (int j = 0; j < nblk; ++j) s += part_pool[((size_t)b * nblk + j) * C + o];
    h = fmaf(to_f(prm_e[o]), s / (float)P, h);
  }
  if (h_out) h_out[b] = h;
  const float e = expf(h + q);
  if (est) est[b] = e;
  if (flag) flag[b] = e > threshold ? 1 : 0;
}

// ---------------------------------------------------------------- launchers ---
static int blocks_for(long long n, int threads, int cap = 152 * 16) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
cudaError_t launch_tables(T* D, T* E, int N, int m, int Kp, cudaStream_t st) {
  const long long n = 2LL * m * m * N * N;
  tables_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(D, E, N, m, Kp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lift(const float2* n, const T* params, T* Vcf, T* Vcl, int B, int S, int in_grid, int N,
                        cudaStream_t st) {
  const long long total = (long long)B * in_grid * in_grid;
  lift_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, params, Vcf, Vcl, B, S, in_grid, N);
  return cudaGetLastError();
}

template <typename T, int NM>
static cudaError_t launch_mix_fwd_t(const float2* Vh, int splits, long long split_stride, long long ld, const T* R,
                                    T* Wh, float scale, int B, int m, int Kp, cudaStream_t st) {
  const size_t smem = mix_fwd_rs_bytes<T>(NM) + (size_t)NM * MIX_TILE * sizeof(float2);
  const void* fn = reinterpret_cast<const void*>(mix_fwd_kernel<T, NM>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(m * m / NM, (B + MIX_SAMPLES - 1) / MIX_SAMPLES);
  mix_fwd_kernel<T, NM><<<grid, 256, smem, st>>>(Vh, splits, split_stride, ld, R, Wh, scale, B, Kp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mix_fwd(const float2* Vh, int splits, long long split_stride, long long ld, const T* R, T* Wh,
                           float scale, int B, int m, int Kp, cudaStream_t st) {
  if ((m * m) % MIX_MODES_FWD) return cudaErrorInvalidValue;
  return launch_mix_fwd_t<T, MIX_MODES_FWD>(Vh, splits, split_stride, ld, R, Wh, scale, B, m, Kp, st);
}

int mix_sample_blocks(int B) { return (B + MIX_SAMPLES - 1) / MIX_SAMPLES; }

template <typename T>
cudaError_t launch_mix_bwd(const float2* G, const float2* Vh, int splits, long long split_stride, long long ld,
                           const T* R, T* GVh, float* part, int B, int m, int Kp, int N, bool with_gvh,
                           cudaStream_t st) {
  const size_t smem = (size_t)4 * MIX_TILE * sizeof(float2);
  const void* fn = reinterpret_cast<const void*>(mix_bwd_kernel<T>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(m * m, mix_sample_blocks(B));
  mix_bwd_kernel<T><<<grid, 128, smem, st>>>(G, Vh, splits, split_stride, ld, R, GVh, part, B, m, Kp, N,
                                              with_gvh ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transpose_w(const T* wcopy, long long off_W0, long long layer_stride, T* WT, int L,
                               cudaStream_t st) {
  transpose_w_kernel<T><<<(L * C * C + 255) / 256, 256, 0, st>>>(wcopy, off_W0, layer_stride, WT, L);
  return cudaGetLastError();
}

cudaError_t launch_target_norm(const float2* target, float* part, int B, int P, cudaStream_t st) {
  target_norm_kernel<<<dim3(P / PIX_BLOCK, B), PIX_BLOCK, 0, st>>>(target, part, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_train(const T* Vcl, const float2* target, const T* params_q, const float* part_tn, T* dZcf,
                                 T* dZcl, float* part_err, float* part_pool, float* part_proj, int B, int P,
                                 cudaStream_t st) {
  project_train_kernel<T><<<dim3(P / PIX_BLOCK, B), PIX_BLOCK, 0, st>>>(Vcl, target, params_q, part_tn, dZcf, dZcl,
                                                                       part_err, part_pool, part_proj, B, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_head(const float* part_tn, const float* part_err, const float* part_pool, const T* params_e,
                        float* part_head, float* h_out, float* rel2_out, int B, int P, cudaStream_t st) {
  head_kernel<T><<<(B + 7) / 8, 256, 0, st>>>(part_tn, part_err, part_pool, params_e, part_head, h_out, rel2_out, B,
                                              P / PIX_BLOCK, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lift_bwd(const T* dV0cl, const float2* n, float* part, int B, int S, int in_grid, int N,
                            cudaStream_t st) {
  const long long total = (long long)B * in_grid * in_grid;
  lift_bwd_kernel<T><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(dV0cl, n, part, B, S, in_grid, N);
  return cudaGetLastError();
}

// Segmented form of reduce_rows_kernel: block b belongs to the last segment whose first item is <= b.
__device__ __forceinline__ int find_segment(const RedSeg* segs, int nseg, int b, bool second) {
  int s = 0;
  for (int i = 1; i < nseg; ++i)
    if ((second ? segs[i].item2 : segs[i].item1) <= b && (!second || segs[i].ry > 1)) s = i;
  return s;
}

__global__ void __launch_bounds__(256) reduce_segments_kernel(const RedSeg* __restrict__ segs, int nseg, int second) {
  __shared__ float red[8][33];
  const int b = blockIdx.x;
  const int si = find_segment(segs, nseg, b, second != 0);
  const RedSeg sg = segs[si];
  if (!second && sg.wide) {
    // few rows: one thread per column, rows added in order (the same additions as the 8-way block form)
    const int col = (b - sg.item1) * 256 + threadIdx.y * 32 + threadIdx.x;
    if (col < sg.width) {
      float t = 0.f;
      for (int r = 0; r < sg.rows; ++r) t += sg.part[(size_t)r * sg.pitch + col];
      sg.out[col] += t;
    }
    return;
  }
  const int gx = (sg.width + 31) / 32;
  const float* src;
  long long pitch;
  int r0, r1, cb, k;
  if (!second) {
    const int local = b - sg.item1;
    k = local / gx;
    cb = local - k * gx;
    src = sg.part;
    pitch = sg.pitch;
    r0 = k * sg.chunk;
    r1 = min(sg.rows, r0 + sg.chunk);
  } else {
    k = 0;
    cb = b - sg.item2;
    src = sg.scratch;
    pitch = sg.width;
    r0 = 0;
    r1 = sg.ry;
  }
  const int col = cb * 32 + threadIdx.x;
  float s = 0.f;
  if (col < sg.width)
    for (int r = r0 + threadIdx.y; r < r1; r += 8) s += src[(size_t)r * pitch + col];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && col < sg.width) {
    float t = 0.f;
    for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
    if (!second && sg.ry > 1)
      sg.scratch[(size_t)k * sg.width + col] = t;
    else
      sg.out[col] += t;
  }
}

bool plan_reduce_segments(std::vector<RedSeg>& segs, float* scratch, size_t scratch_floats, int& items1,
                          int& items2) {
  items1 = items2 = 0;
  size_t used = 0;
  for (auto& sg : segs) {
    sg.wide = sg.rows <= 8 ? 1 : 0;
    const int gx = sg.wide ? (sg.width + 255) / 256 : (sg.width + 31) / 32;
    if (sg.rows <= 256) {
      sg.ry = 1;
      sg.chunk = sg.rows;
      sg.scratch = nullptr;
    } else {
      sg.ry = std::min(64, (sg.rows + 255) / 256);
      sg.chunk = (sg.rows + sg.ry - 1) / sg.ry;
      sg.scratch = scratch + used;
      used += (size_t)sg.ry * sg.width;
    }
    sg.item1 = items1;
    items1 += gx * sg.ry;
    sg.item2 = items2;
    if (sg.ry > 1) items2 += gx;
  }
  return used <= scratch_floats;
}

cudaError_t launch_reduce_segments(const RedSeg* d_segs, int nseg, int items1, int items2, cudaStream_t st) {
  if (nseg == 0 || items1 == 0) return cudaSuccess;
  reduce_segments_kernel<<<items1, dim3(32, 8), 0, st>>>(d_segs, nseg, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || items2 == 0) return e;
  reduce_segments_kernel<<<items2, dim3(32, 8), 0, st>>>(d_segs, nseg, 1);
  return cudaGetLastError();
}

// out[j] += scale * sum_r part[r pitch + j]; rows above 256 go through `scratch`
// (64 rows of `width`) in a second pass so that no thread sums more than ~32 rows.
cudaError_t launch_reduce_rows_ex(const float* part, int rows, int width, long long pitch, float scale, float* out,
                                  float* scratch, cudaStream_t st) {
  if (rows <= 0 || width <= 0) return cudaSuccess;
  const dim3 block(32, 8);
  const unsigned gx = (unsigned)((width + 31) / 32);
  if (rows <= 256 || !scratch) {
    reduce_rows_kernel<<<dim3(gx, 1), block, 0, st>>>(part, rows, width, pitch, rows, scale, out, nullptr);
    return cudaGetLastError();
  }
  const int ry = std::min(64, (rows + 255) / 256);
  const int chunk = (rows + ry - 1) / ry;
  reduce_rows_kernel<<<dim3(gx, ry), block, 0, st>>>(part, rows, width, pitch, chunk, scale, out, scratch);
  reduce_rows_kernel<<<dim3(gx, 1), block, 0, st>>>(scratch, ry, width, width, ry, scale, out, nullptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adam(float* master, const float* grad, float* m, float* v, T* copy, long long n, float lr,
                        float bc1, float bc2, cudaStream_t st) {
  adam_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(master, grad, m, v, copy, n, lr, bc1, bc2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_params(const float* master, T* copy, long long n, cudaStream_t st) {
  copy_params_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(master, copy, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_infer(const T* Vcl, const T* params_q, float2* field, float* part_pool, int B, int P,
                                 cudaStream_t st) {
  project_infer_kernel<T><<<dim3(P / PIX_BLOCK, B), PIX_BLOCK, 0, st>>>(Vcl, params_q, field, part_pool, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_head_infer(const float* part_pool, const T* params_e, float q, float threshold, float* h_out,
                              float* est, unsigned char* flag, int B, int P, cudaStream_t st) {
  head_infer_kernel<T><<<(B + 127) / 128, 128, 0, st>>>(part_pool, params_e, q, threshold, h_out, est, flag, B,
                                                        P / PIX_BLOCK, P);
  return cudaGetLastError();
}

#define SCW_FNO_INSTANTIATE(T)                                                                                       \
  template cudaError_t launch_tables<T>(T*, T*, int, int, int, cudaStream_t);                                      \
  template cudaError_t launch_lift<T>(const float2*, const T*, T*, T*, int, int, int, int, cudaStream_t);          \
  template cudaError_t launch_mix_fwd<T>(const float2*, int, long long, long long, const T*, T*, float, int, int, \
                                         int, cudaStream_t);                                                        \
  template cudaError_t launch_mix_bwd<T>(const float2*, const float2*, int, long long, long long, const T*, T*,   \
                                         float*, int, int, int, int, bool, cudaStream_t);                           \
  template cudaError_t launch_transpose_w<T>(const T*, long long, long long, T*, int, cudaStream_t);              \
  template cudaError_t launch_project_train<T>(const T*, const float2*, const T*, const float*, T*, T*, float*,   \
                                               float*, float*, int, int, cudaStream_t);                            \
  template cudaError_t launch_head<T>(const float*, const float*, const float*, const T*, float*, float*, float*,  \
                                      int, int, cudaStream_t);                                                      \
  template cudaError_t launch_lift_bwd<T>(const T*, const float2*, float*, int, int, int, int, cudaStream_t);      \
  template cudaError_t launch_adam<T>(float*, const float*, float*, float*, T*, long long, float, float, float,   \
                                      cudaStream_t);                                                                \
  template cudaError_t launch_copy_params<T>(const float*, T*, long long, cudaStream_t);                          \
  template cudaError_t launch_project_infer<T>(const T*, const T*, float2*, float*, int, int, cudaStream_t);      \
  template cudaError_t launch_head_infer<T>(const float*, const T*, float, float, float*, float*, unsigned char*,  \
                                            int, int, cudaStream_t);

SCW_FNO_INSTANTIATE(float)
SCW_FNO_INSTANTIATE(__nv_bfloat16)

}  // namespace fno
}  // namespace scw
