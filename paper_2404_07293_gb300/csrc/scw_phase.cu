// Step (a): per-plane mode weights c_j(z) = alpha_j exp(i k gamma_j (z - z_ref,j))
// (paper Eq. 7 and Eq. 30-31, with the per-layer precompute of Sec. 4.1), the
// exterior spectra of Eq. 9, and the one-off conversions of W.
//
// Phase arithmetic: the argument is range-reduced in units of cycles,
//   t = Re(gamma) (z - z_ref) / lambda,  r = t - rint(t)  (|r| <= 1/2),
// and only the reduced r goes to FP32 sincospif(2 r); the decay is
// exp(-2 pi Im(gamma) (z - z_ref) / lambda). The per-mode factors
// Re(gamma)/lambda and the per-plane offsets z - z_ref are formed in FP64 once
// and carried as float pairs (hi + lo); the per-plane product t then uses an
// exact FP32 two-product, because FP64 throughput on this part is a small
// fraction of FP32. Large k Re(gamma) z therefore loses no digits, and
// evanescent Im(gamma) never overflows: with forward modes referenced to the
// layer top and backward modes to its bottom the exponent is never positive
// inside a layer.
#include "scw_internal.cuh"

namespace scw {

__device__ __forceinline__ float2 mode_factor(double2 g, double dz, double inv_lam) {
  const double t = (g.x * inv_lam) * dz;           // cycles
  const double r = t - rint(t);
  const float ex = (float)((g.y * inv_lam) * dz) * -6.2831853071795865f;
  float s, c;
  sincospif(2.0f * (float)r, &s, &c);
  const float mag = expf(ex);
  return make_float2(c * mag, s * mag);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename T> __device__ __forceinline__ T to_lp(float x);
template <> __device__ __forceinline__ __nv_bfloat16 to_lp<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half to_lp<__half>(float x) { return __float2half_rn(x); }
template <typename T> __device__ __forceinline__ float from_lp(T x);
template <> __device__ __forceinline__ float from_lp<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ float from_lp<__half>(__half x) { return __half2float(x); }

template <typename T>
struct Pair { T a, b; };

// Per-plane offsets from both reference planes of a unit's layer, split into
// float pairs (hi + lo == the FP64 difference to ~2^-48 relative).
struct PlaneOffsets {
  float f_hi[kMaxPlanesPerLayer], f_lo[kMaxPlanesPerLayer];  // z - z_{l-1}
  float b_hi[kMaxPlanesPerLayer], b_lo[kMaxPlanesPerLayer];  // z - z_l
};

__device__ __forceinline__ void load_offsets(PlaneOffsets& o, const LayerUnit& u, const double* zplanes,
                                             const double* zb) {
  for (int f = threadIdx.x; f < u.nf; f += blockDim.x) {
    const double z = zplanes[u.f0 + f];
    const double df = z - zb[u.layer], db = z - zb[u.layer + 1];
    o.f_hi[f] = (float)df;
    o.f_lo[f] = (float)(df - (double)o.f_hi[f]);
    o.b_hi[f] = (float)db;
    o.b_lo[f] = (float)(db - (double)o.b_hi[f]);
  }
}

// exp(i k gamma dz) from a = Re(gamma)/lambda split as a_hi + a_lo, c = -2 pi Im(gamma)/lambda
// and dz = d_hi + d_lo. The cycle count t = a dz is formed exactly enough in FP32
// (two-product: p + e == a_hi d_hi exactly), each part range-reduced on its own,
// so no FP64 instruction runs per plane.
__device__ __forceinline__ float2 mode_factor_df(float a_hi, float a_lo, float c, float d_hi, float d_lo) {
  const float p = a_hi * d_hi;
  const float e = fmaf(a_hi, d_hi, -p);
  const float t_lo = fmaf(a_hi, d_lo, fmaf(a_lo, d_hi, e));
  const float r = (p - rintf(p)) + (t_lo - rintf(t_lo));
  float sn, cs;
  sincospif(2.0f * r, &sn, &cs);
  const float mag = expf(c * (d_hi + d_lo));
  return make_float2(cs * mag, sn * mag);
}

struct ModeConst {
  float a_hi, a_lo, c;
  float2 alpha;
};

__device__ __forceinline__ ModeConst mode_const(double2 g, double2 al, double inv_lam) {
  ModeConst m;
  const double a = g.x * inv_lam;
  m.a_hi = (float)a;
  m.a_lo = (float)(a - (double)m.a_hi);
  m.c = (float)(g.y * inv_lam) * -6.2831853071795865f;
  m.alpha = make_float2((float)al.x, (float)al.y);
  return m;
}

// Element offset of (row n, column k) in a tile-major operand with the
// 128-byte swizzle of the tensor cores' K-major shared-memory layout: K is cut
// into chunks of 64 16-bit elements; chunk kc holds `rows` rows of 128 bytes,
// and the 16-byte group g of row n is stored at group g ^ (n mod 8). A chunk is
// then one contiguous block that lands in shared memory as is.
__device__ __forceinline__ size_t swz_offset(int n, int k, int rows) {
  const int kc = k >> 6, e = k & 63;
  const int g = e >> 3;
  return (size_t)kc * rows * 64 + (size_t)n * 64 + (size_t)(((g ^ (n & 7)) << 3) | (e & 7));
}

// B operand of the tensor-core contraction, per work unit nk chunks of NB rows
// (NB = 2 F_pad) in the layout above: row f holds (Re c_j, -Im c_j) at columns
// (2j, 2j+1), row F_pad + f holds (Im c_j, Re c_j); with A = W viewed as
// interleaved reals this gives [Re S | Im S] (the complex product as one real
// GEMM). hi = round(x), lo = round(x - hi). A block is kPhaseModes consecutive modes x
// kPhaseGroups plane groups: thread t takes mode kPhaseModes blockIdx.x + t mod kPhaseModes and
// the planes f = g, g + kPhaseGroups, ... (g = t / kPhaseModes) of its unit; every warp store
// covers whole 128-byte rows. Blocks are (mode block, (item, unit) entry). One group (a thread
// loops over all planes of its mode, whose constants it loads and reduces once) measured faster
// than four (5.2 against 8.3 us per step at 21x21 orders, 32 layers of 8 planes).
constexpr int kPhaseModes = 128;
constexpr int kPhaseGroups = 1;

template <typename T, bool BATCH>
__global__ void __launch_bounds__(kPhaseModes * kPhaseGroups) phases_tc_kernel(const __grid_constant__ ItemDev one,
                                                                      const ItemDev* __restrict__ items,
                                                                      const int2* __restrict__ entries, int F_pad) {
  __shared__ PlaneOffsets off;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the contraction may start streaming W
  trace_begin(one.trace, TRACE_PHASES);
  const int2 e = entries[blockIdx.y];
  const ItemDev& it = BATCH ? items[e.x] : one;
  const LayerUnit u = it.units[e.y];
  const int M = it.M;
  const int j = blockIdx.x * kPhaseModes + (threadIdx.x % kPhaseModes);
  const int fg = threadIdx.x / kPhaseModes;
  const int M4 = 4 * M;
  // the mode's constants are requested before the block waits for the plane offsets
  double2 g = make_double2(0.0, 0.0), al = make_double2(0.0, 0.0);
  const size_t lj = (size_t)u.layer * M4 + j;
  const double2* alpha_lj = it.alpha + lj;  // illumination 0
  if (j < M4) {
    if (in_bounds(it, BND_GAMMA, lj)) g = it.gamma[lj];
    if (in_bounds(it, BND_ALPHA, lj)) al = alpha_lj[0];
  }
  load_offsets(off, u, it.zplanes, it.zbounds);
  __syncthreads();
  if (j < M4) {
    const int NB = 2 * F_pad;
    const ModeConst mc = mode_const(g, al, it.inv_lam);
    const bool fwd = j < 2 * M;
    const size_t base = (size_t)e.y * it.nk * NB * 64;  // B is per work unit
    T* Bhi = static_cast<T*>(it.Bhi) + base;
    T* Blo = static_cast<T*>(it.Blo) + base;
    for (int f = fg; f < F_pad; f += kPhaseGroups) {
      float2 cv = make_float2(0.f, 0.f);
      if (f < u.nf) {
        const float dh = fwd ? off.f_hi[f] : off.b_hi[f];
        const float dl = fwd ? off.f_lo[f] : off.b_lo[f];
        float2 a = mc.alpha;
        if (it.I > 1) {  // plane slot f I + i carries illumination i
          const size_t ia = (size_t)((u.f0 + f) % it.I) * it.alpha_istride;
          const double2 ai = in_bounds(it, BND_ALPHA, lj + ia) ? alpha_lj[ia] : make_double2(0.0, 0.0);
          a = make_float2((float)ai.x, (float)ai.y);
        }
        cv = cmulf(a, mode_factor_df(mc.a_hi, mc.a_lo, mc.c, dh, dl));
      }
      const float v0[2] = {cv.x, -cv.y};
      const float v1[2] = {cv.y, cv.x};
      Pair<T> h0, l0, h1, l1;
      h0.a = to_lp<T>(v0[0]); h0.b = to_lp<T>(v0[1]);
      l0.a = to_lp<T>(v0[0] - from_lp<T>(h0.a)); l0.b = to_lp<T>(v0[1] - from_lp<T>(h0.b));
      h1.a = to_lp<T>(v1[0]); h1.b = to_lp<T>(v1[1]);
      l1.a = to_lp<T>(v1[0] - from_lp<T>(h1.a)); l1.b = to_lp<T>(v1[1] - from_lp<T>(h1.b));
      const size_t i0 = swz_offset(f, 2 * j, NB), i1 = swz_offset(F_pad + f, 2 * j, NB);
      if (in_bounds(it, BND_B, base + i0 + 1)) {  // a pair: its second element is the last one written
        *reinterpret_cast<Pair<T>*>(Bhi + i0) = h0;
        *reinterpret_cast<Pair<T>*>(Blo + i0) = l0;
      }
      if (in_bounds(it, BND_B, base + i1 + 1)) {
        *reinterpret_cast<Pair<T>*>(Bhi + i1) = h1;
        *reinterpret_cast<Pair<T>*>(Blo + i1) = l1;
      }
    }
  }
  trace_end(one.trace, TRACE_PHASES);  // thread 0 (mode kPhaseModes blockIdx.x < 4M) stamps after its planes
}

// FP32 path: C[unit][j][f] complex64, plane index fastest; one thread per mode.
__global__ void __launch_bounds__(128) phases_fp32_kernel(const LayerUnit* __restrict__ units,
                                                          const double* __restrict__ zplanes,
                                                          const double* __restrict__ zb,
                                                          const double2* __restrict__ gamma,
                                                          const double2* __restrict__ alpha, int M, int F_pad,
                                                          double inv_lam, float2* __restrict__ C, int I,
                                                          size_t alpha_istride, unsigned long long* trace,
                                                          const __grid_constant__ ItemDev chk) {
  __shared__ PlaneOffsets off;
  trace_begin(trace, TRACE_PHASES);
  const LayerUnit u = units[blockIdx.y];
  load_offsets(off, u, zplanes, zb);
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int M4 = 4 * M;
  if (j >= M4) return;
  const size_t lj = (size_t)u.layer * M4 + j;
  const ModeConst mc = mode_const(in_bounds(chk, BND_GAMMA, lj) ? gamma[lj] : make_double2(0.0, 0.0),
                                  in_bounds(chk, BND_ALPHA, lj) ? alpha[lj] : make_double2(0.0, 0.0), inv_lam);
  const bool fwd = j < 2 * M;
  float2* dst = C + ((size_t)blockIdx.y * M4 + j) * F_pad;  // C is per work unit
  // plane slot f I + i carries illumination i
  auto alpha_of = [&](int f) {
    if (I == 1) return mc.alpha;
    const size_t ia = (size_t)((u.f0 + f) % I) * alpha_istride + lj;
    const double2 a = in_bounds(chk, BND_ALPHA, ia) ? alpha[ia] : make_double2(0.0, 0.0);
    return make_float2((float)a.x, (float)a.y);
  };
  for (int f = 0; f < F_pad; f += 2) {
    float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
    if (f < u.nf)
      c0 = cmulf(alpha_of(f), mode_factor_df(mc.a_hi, mc.a_lo, mc.c, fwd ? off.f_hi[f] : off.b_hi[f],
                                             fwd ? off.f_lo[f] : off.b_lo[f]));
    if (f + 1 < u.nf)
      c1 = cmulf(alpha_of(f + 1), mode_factor_df(mc.a_hi, mc.a_lo, mc.c, fwd ? off.f_hi[f + 1] : off.b_hi[f + 1],
                                                 fwd ? off.f_lo[f + 1] : off.b_lo[f + 1]));
    if (in_bounds(chk, BND_C, ((size_t)blockIdx.y * M4 + j) * F_pad + f + 1))
      *reinterpret_cast<float4*>(dst + f) = make_float4(c0.x, c0.y, c1.x, c1.y);
  }
  trace_end(trace, TRACE_PHASES);
}

// Exterior planes (Eq. 9 with the reflected wave travelling towards -z):
// S_part[0][f][c M + m]. Plane slot f carries illumination f mod I (p_* are [I][3][M]);
// below the sample an optional pupil mask drops the orders outside the objective's NA.
__global__ void exterior_kernel(const int* __restrict__ ext_planes, const double* __restrict__ zplanes,
                                double z0, double zL, double z_inc, const double2* __restrict__ sz_top,
                                const double2* __restrict__ sz_bot, const double2* __restrict__ p_inc,
                                const double2* __restrict__ p_ref, const double2* __restrict__ p_trn,
                                int M, double inv_lam, float2* __restrict__ S, int I,
                                const float* __restrict__ pupil, unsigned long long* trace,
                                const __grid_constant__ ItemDev chk) {
  trace_begin(trace, TRACE_EXTERIOR);
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int f = ext_planes[blockIdx.y];
  const double z = zplanes[f];
  float2* out = S + (size_t)f * 3 * M;
  const size_t po = (size_t)(f % I) * 3 * M;
  p_inc += po;
  p_ref += po;
  p_trn += po;
  if (z < z0) {
    const double2 st = sz_top[m];
    const float2 gi = mode_factor(st, z - z_inc, inv_lam);
    const float2 gr = mode_factor(st, -(z - z0), inv_lam);
    for (int c = 0; c < 3; ++c) {
      const double2 a = p_inc[c * M + m], b = p_ref[c * M + m];
      const float2 x = cmulf(make_float2((float)a.x, (float)a.y), gi);
      const float2 y = cmulf(make_float2((float)b.x, (float)b.y), gr);
      if (in_bounds(chk, BND_S_PART, (size_t)f * 3 * M + c * M + m)) out[c * M + m] = make_float2(x.x + y.x, x.y + y.y);
    }
  } else {
    const double2 sb = sz_bot[m];
    float2 gt = mode_factor(sb, z - zL, inv_lam);
    if (pupil) gt = make_float2(gt.x * pupil[m], gt.y * pupil[m]);
    for (int c = 0; c < 3; ++c) {
      const double2 a = p_trn[c * M + m];
      if (in_bounds(chk, BND_S_PART, (size_t)f * 3 * M + c * M + m))
        out[c * M + m] = cmulf(make_float2((float)a.x, (float)a.y), gt);
    }
  }
  trace_end(trace, TRACE_EXTERIOR);  // thread 0 always has an order (m = 128 blockIdx.x < M)
}

// ---- one-off conversions of W (plan time) -----------------------------------
// W [L][R = 3M][K8 = 8M] reals (the complex64 layout) -> tile-major, swizzled
// 16-bit copies for the tensor-core contraction: for layer l, row tile t
// (rows RT t .. RT t + rt - 1, rt = min(RT, R - RT t), RT <= 128 the plan's rows per
// tile) and K chunk kc, one contiguous block of rt x 64 elements (swz_offset layout;
// K beyond 8M is zero).
// One thread per (l, row, kc, 16-byte group): 8 reals in, 8 (hi) + 8 (lo) out.
template <typename T, bool SPLIT>
__global__ void convert_tiled_kernel(const float* __restrict__ W, T* __restrict__ hi, T* __restrict__ lo, int L, int R,
                                     int K8, int nk, int RT) {
  const size_t total = (size_t)L * R * nk * 8;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int grp = (int)(g & 7);
    const size_t q = g >> 3;
    const int kc = (int)(q % nk);
    const size_t q2 = q / nk;
    const int row = (int)(q2 % R);
    const int l = (int)(q2 / R);
    const int k0 = kc * 64 + grp * 8;
    float x[8];
    if (k0 < K8) {
      const float4* src = reinterpret_cast<const float4*>(W + ((size_t)l * R + row) * K8 + k0);
      const float4 a = src[0], b = src[1];
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = 0.f;
    }
    const int t = row / RT, n = row - t * RT;
    const int rt = min(RT, R - RT * t);
    const size_t off = (size_t)l * R * nk * 64 + (size_t)t * RT * nk * 64 + (size_t)kc * rt * 64 + (size_t)n * 64 +
                       (size_t)((grp ^ (n & 7)) << 3);
    T h[8], lw[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = to_lp<T>(x[i]);
      if (SPLIT) lw[i] = to_lp<T>(x[i] - from_lp<T>(h[i]));
    }
    *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<uint4*>(h);
    if (SPLIT) *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<uint4*>(lw);
  }
}

// Wt[l][c][r] = W[l][r][c], 32x32 tiles through shared memory.
__global__ void transpose_layers_kernel(const float2* __restrict__ W, float2* __restrict__ Wt, int rows,
                                        int cols) {
  __shared__ float2 tile[32][33];
  const size_t lay = (size_t)blockIdx.z * rows * cols;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = W[lay + (size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) Wt[lay + (size_t)c * rows + r] = tile[threadIdx.x][i];
  }
}

static int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g == 0) g = 1;
  return (int)g;
}

cudaError_t launch_convert_tiled(const float2* W, void* hi, void* lo, int L, int M, int rows_tile, bool bf16_split,
                                 cudaStream_t st) {
  const int R = 3 * M, K8 = 8 * M, nk = (K8 + 63) / 64;
  if (rows_tile < 1 || rows_tile > 128) return cudaErrorInvalidValue;
  const size_t total = (size_t)L * R * nk * 8;
  const float* w = reinterpret_cast<const float*>(W);
  if (bf16_split)
    convert_tiled_kernel<__nv_bfloat16, true><<<grid_for(total, 256), 256, 0, st>>>(
        w, static_cast<__nv_bfloat16*>(hi), static_cast<__nv_bfloat16*>(lo), L, R, K8, nk, rows_tile);
  else
    convert_tiled_kernel<__half, false><<<grid_for(total, 256), 256, 0, st>>>(w, static_cast<__half*>(hi), nullptr,
                                                                              L, R, K8, nk, rows_tile);
  return cudaGetLastError();
}

cudaError_t launch_transpose_layers(const float2* W, float2* Wt, int L, int rows, int cols, cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, L), block(32, 8);
  transpose_layers_kernel<<<grid, block, 0, st>>>(W, Wt, rows, cols);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_phases_tc_t(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries,
                                      int max_M, int F_pad, cudaStream_t st) {
  dim3 grid((4 * max_M + kPhaseModes - 1) / kPhaseModes, n_entries);
  if (items)
    phases_tc_kernel<T, true><<<grid, kPhaseModes * kPhaseGroups, 0, st>>>(one, items, d_entries, F_pad);
  else
    phases_tc_kernel<T, false><<<grid, kPhaseModes * kPhaseGroups, 0, st>>>(one, nullptr, d_entries, F_pad);
  return cudaGetLastError();
}

cudaError_t launch_phases_tc(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries,
                             int max_M, int F_pad, bool bf16, cudaStream_t st) {
  if (n_entries == 0) return cudaSuccess;
  return bf16 ? launch_phases_tc_t<__nv_bfloat16>(one, items, d_entries, n_entries, max_M, F_pad, st)
              : launch_phases_tc_t<__half>(one, items, d_entries, n_entries, max_M, F_pad, st);
}

cudaError_t launch_phases_fp32(const Plan& p, cudaStream_t st) {
  const int n_units = (int)p.units.size();
  if (n_units == 0) return cudaSuccess;
  dim3 grid((4 * p.M + 127) / 128, n_units);
  phases_fp32_kernel<<<grid, 128, 0, st>>>(p.d_units, p.d_zplanes, p.d_zbounds, p.gamma, p.alpha, p.M,
                                           p.F_pad, 1.0 / p.lambda, p.Cf, p.I, (size_t)p.L * 4 * p.M, p.item.trace,
                                           p.item);
  return cudaGetLastError();
}

cudaError_t launch_exterior(const Plan& p, cudaStream_t st) {
  if (p.n_exterior == 0) return cudaSuccess;
  dim3 grid((p.M + 127) / 128, p.n_exterior);
  const double z0 = p.z_bounds.front(), zL = p.z_bounds.back();
  exterior_kernel<<<grid, 128, 0, st>>>(p.d_ext_planes, p.d_zplanes, z0, zL, p.z_inc, p.d_sz_top, p.d_sz_bot,
                                        p.p_inc, p.p_ref, p.p_trn, p.M, 1.0 / p.lambda, p.S_part, p.I, p.d_pupil,
                                        p.item.trace, p.item);
  return cudaGetLastError();
}

}  // namespace scw
