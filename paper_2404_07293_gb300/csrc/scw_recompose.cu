// Step (c): recomposition of the field from its per-plane spectrum (Eq. 10),
//   E_c(x_i, y_j) = sum_{u,v} S_c[u,v] exp(2 pi i (u x_i / X + v y_j / Y)),
// on x_i = x0 + i X/Fx, y_j = y0 + j Y/Fy: an unnormalised inverse 2D DFT of
// the U x V non-zero orders onto the Fx x Fy grid.
//
// Both axes use the same pruned radix-8 decimation. With F = 8 Q and output
// index i = b + Q a (b < Q, a < 8), omega = exp(2 pi i / F):
//   sum_u s_u omega^(u (b + Q a)) = sum_{r<8} e^(2 pi i r a / 8) F_b[r],
//   F_b[r] = sum_{u = r mod 8} s_u omega^(u b).
// The signed orders u are stored at position u mod Up (Up = U rounded up to a
// multiple of 8; fold_pos), so position mod 8 == u mod 8 and consecutive groups
// of 8 stored values land in residues 0..7 in order: every fold is a fully
// unrolled loop over whole groups with independent loads, and at most 7 of the
// Up positions are zero padding. Each table twiddle tw[b][p] = omega^(u b) exp(2 pi i u x0 / X) carries the
// origin phase. An in-register radix-8 inverse DFT finishes the 8 outputs Q
// apart. Orders beyond the grid (|u| >= F/2) fold exactly: the sum is only
// evaluated at grid points.
//
// Plans run the two directions as two kernels (x-pass rows T through L2, then
// the y-pass with contiguous 512-byte warp stores); the allocation-free entry
// point, which has no room for T, runs them fused in one kernel.
#include <algorithm>

#include "scw_fold.cuh"
#include "scw_internal.cuh"
#include "scw_ptx.cuh"

namespace scw {

// Field stores. Row y of plane slice s (its base `dst`, column x included) goes to
// dst + y ld, streaming; TILED: also to every other periodic tile (E repeats with
// the period X, Y). Untiled plans use the plain form, so their y-pass keeps a
// straight sequence of stores.
template <bool TILED>
__device__ __forceinline__ void store_row4(const ItemDev& it, float2* dst, int y, float4 v) {
  float2* r = dst + (long long)y * it.ld;
  if constexpr (!TILED) {
    __stcs(reinterpret_cast<float4*>(r), v);
  } else {
    for (int b = 0; b < it.ty; ++b)
      for (int a = 0; a < it.tx; ++a)
        __stcs(reinterpret_cast<float4*>(r + (long long)b * it.Fy * it.ld + (long long)a * it.Fx), v);
  }
}
template <bool TILED>
__device__ __forceinline__ void store_row2(const ItemDev& it, float2* dst, int y, float2 v) {
  float2* r = dst + (long long)y * it.ld;
  if constexpr (!TILED) {
    __stcs(r, v);
  } else {
    for (int b = 0; b < it.ty; ++b)
      for (int a = 0; a < it.tx; ++a) __stcs(r + (long long)b * it.Fy * it.ld + (long long)a * it.Fx, v);
  }
}

// One CTA per (block of 8 column residues, item-plane, component). The CTA owns
// the 64 output columns x = b + Qx a (b in its 8 residues, a < 8), which are
// exactly the outputs of its residues' x-direction folds, so the x-pass rows
// for its columns are computed once, straight into shared memory:
//   1. the spectrum rows of component c (partial sums of the contraction added)
//      -> srow[V][Up];
//   2. x-direction fold + radix-8 inverse DFT per (row v, residue b)
//      -> tcol[p = fold position of v][local column b_local + 8 a];
//   3. y-direction fold + radix-8 inverse DFT per (column pair, y residue),
//      16-byte streaming stores (each warp store: 8 runs of 8 contiguous columns).
template <bool BATCH>
__global__ void __launch_bounds__(256, 4) recompose_kernel(const __grid_constant__ ItemDev one,
                                                           const ItemDev* __restrict__ items,
                                                           const int2* __restrict__ entries,
                                                           const float2* __restrict__ S_override,
                                                           const int* __restrict__ nsplit_override,
                                                           float2* out_one, float2* const* __restrict__ outs) {
  extern __shared__ float4 sm4[];
  const int2 e = entries[blockIdx.y];
  const ItemDev& it = BATCH ? items[e.x] : one;
  const int Qx = it.Fx >> 3;
  const int b0 = blockIdx.x * 8;
  if (b0 >= Qx) return;
  const int nb = min(8, Qx - b0);
  const int f = e.y, c = blockIdx.z;
  const int U = it.U, V = it.V, M = it.M, Up = it.Up, Vp = it.Vp;
  float4* tcol4 = sm4;                                  // [Vp][32] float4 = [Vp][64] complex
  float2* tcol = reinterpret_cast<float2*>(sm4);
  float2* srow = tcol + (size_t)Vp * 64;                // [V][Up]

  // 1. spectrum rows of component c
  const float2* src = (S_override ? S_override : it.S_part) + (size_t)f * 3 * M + (size_t)c * M;
  const int ns = nsplit_override ? nsplit_override[f] : it.nsplit[f];
  const size_t stride = it.split_stride;
  for (int i = threadIdx.x; i < V * Up; i += blockDim.x) {
    const int vi = i / Up, ui = fold_order(i - vi * Up, U, Up);
    float2 acc = make_float2(0.f, 0.f);
    if (ui >= 0) {
      const float2* s = src + vi * U + ui;
      for (int k = 0; k < ns; ++k) acc = c_add(acc, s[(size_t)k * stride]);
    }
    srow[i] = acc;
  }
  for (int i = threadIdx.x; i < Vp * 64; i += blockDim.x)  // padding rows stay zero
    if (fold_order(i >> 6, V, Vp) < 0) tcol[i] = make_float2(0.f, 0.f);
  __syncthreads();

  // 2. x-direction: fold + DFT for (row vi, residue b0 + bl)
  for (int t = threadIdx.x; t < V * 8; t += blockDim.x) {
    const int vi = t >> 3, bl = t & 7;
    float2 G[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) G[q] = make_float2(0.f, 0.f);
    if (bl < nb) {
      const float2* s = srow + vi * Up;
      const float2* tw = it.twx + b0 + bl;  // [p][b]
      for (int p0 = 0; p0 < Up; p0 += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) c_fma(G[q], s[p0 + q], __ldg(tw + (size_t)(p0 + q) * Qx));
      }
      idft8(G);
    }
    float2* d = tcol + (size_t)fold_pos(vi, V, Vp) * 64 + bl;
#pragma unroll
    for (int a = 0; a < 8; ++a) d[8 * a] = G[a];
  }
  __syncthreads();

  // 3. y-direction: lane l owns local columns (2l, 2l+1) = residues b0 + 2(l & 3) (+1), a = l >> 2
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int bl = 2 * (lane & 3);
  const int x = b0 + bl + Qx * (lane >> 2);
  const bool pair = bl + 1 < nb;
  const bool v16 = pair && ((Qx & 1) == 0);  // x even: 16-byte aligned pair
  const int Fx = it.Fx, Fy = it.Fy;
  const int Qy = Fy >> 3;
  float2* out = BATCH ? outs[e.x] : out_one;
  // plane slot f = (output plane) I + illumination: slice (il 3 + c) Fz_out + fo of the field
  const int fo = f / it.I, il = f - fo * it.I;
  float2* dst = out + ((long long)il * 3 * it.Fz_out + (long long)c * it.Fz_out + fo) * it.pstride + x;
  if (bl >= nb) return;  // no __syncthreads below
  for (int b = w; b < Qy; b += 8) {
    float2 G0[8], G1[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) G0[q] = G1[q] = make_float2(0.f, 0.f);
    const float2* tw = it.twy + (size_t)b * Vp;
    for (int p0 = 0; p0 < Vp; p0 += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 t = __ldg(tw + p0 + q);
        const float4 d = tcol4[(p0 + q) * 32 + lane];
        c_fma(G0[q], make_float2(d.x, d.y), t);
        c_fma(G1[q], make_float2(d.z, d.w), t);
      }
    }
    idft8(G0);
    idft8(G1);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (v16) {
        store_row4<true>(it, dst, b + a * Qy, make_float4(G0[a].x, G0[a].y, G1[a].x, G1[a].y));
      } else {
        store_row2<true>(it, dst, b + a * Qy, G0[a]);
        if (pair) store_row2<true>(it, dst + 1, b + a * Qy, G1[a]);
      }
    }
  }
}

// ---- two-kernel form (plans): x-pass rows through L2, y-pass with 512-byte warp stores ----
constexpr int kSplitUnroll = 8;  // split partials loaded together (more are added one by one)
// Residue loops visit exactly the U (or V) stored orders: for residue r the
// first stored index p >= rot with p = r (mod 8), then every 8th.

// One CTA per (item-plane, component): V * Fx/8 tasks (row vi, residue b).
// The spectrum of component c (split partials summed) is laid out [V][Up] in
// shared memory at the fold positions, padding zero; the fold twiddles [Up][Fx/8]
// follow it when they fit (xpass_twiddles_staged), else they are read through L1.
constexpr size_t kXpassTwBytes = 32 * 1024;

__host__ __device__ __forceinline__ bool xpass_twiddles_staged(int Up, int Fx) {
  return (size_t)Up * (Fx / 8) * sizeof(float2) <= kXpassTwBytes;
}

template <bool BATCH>
__global__ void __launch_bounds__(256) xpass_kernel(const __grid_constant__ ItemDev one,
                                                    const ItemDev* __restrict__ items,
                                                    const int2* __restrict__ entries) {
  extern __shared__ float2 xs_row[];  // [V][Up], then the staged twiddles [Up][Fx/8]
  const int2 e = entries[blockIdx.x];
  const ItemDev& it = BATCH ? items[e.x] : one;
  const int f = e.y, c = blockIdx.y;
  const int U = it.U, V = it.V, M = it.M, Up = it.Up, Fx = it.Fx;
  const int Q = Fx >> 3;
  const bool staged = xpass_twiddles_staged(Up, Fx);
  float2* tw_s = xs_row + V * Up;
  ptx::griddep_launch_dependents();
  if (staged)
    for (int i = threadIdx.x; i < Up * Q; i += blockDim.x)
      tw_s[i] = in_bounds(it, BND_TWX, i) ? __ldg(it.twx + i) : make_float2(0.f, 0.f);
  ptx::griddep_wait();  // the partial spectra come from the preceding contraction
  trace_begin(one.trace, TRACE_XPASS);
  const size_t sbase = (size_t)f * 3 * M + (size_t)c * M;
  const float2* src = it.S_part + sbase;
  const int ns = it.nsplit[f];
  const size_t stride = it.split_stride;
  for (int i0 = 0; i0 < V * Up; i0 += 2 * blockDim.x) {
    // all split partials of two elements are requested before any is used
    float2 v[2][kSplitUnroll];
    int off[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * blockDim.x + threadIdx.x;
      const int vi = i / Up, ui = i < V * Up ? fold_order(i - vi * Up, U, Up) : -1;
      off[h] = ui >= 0 ? vi * U + ui : -1;
      // the element's last partial has the largest index
      if (off[h] >= 0 && !in_bounds(it, BND_S_PART, sbase + (size_t)(ns - 1) * stride + off[h])) off[h] = -1;
#pragma unroll
      for (int k = 0; k < kSplitUnroll; ++k)
        v[h][k] = (off[h] >= 0 && k < ns) ? src[(size_t)k * stride + off[h]] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * blockDim.x + threadIdx.x;
      float2 acc = v[h][0];
#pragma unroll
      for (int k = 1; k < kSplitUnroll; ++k) acc = c_add(acc, v[h][k]);
      if (off[h] >= 0)
        for (int k = kSplitUnroll; k < ns; ++k) acc = c_add(acc, src[(size_t)k * stride + off[h]]);
      if (i < V * Up) xs_row[i] = acc;
    }
  }
  __syncthreads();
  const size_t tbase = ((size_t)f * 3 + c) * V * Fx;
  float2* dst = it.T + tbase;
  const float2* twb = staged ? tw_s : it.twx;  // [p][b]: a warp's lanes read consecutive residues
  for (int t = threadIdx.x; t < V * Q; t += blockDim.x) {
    const int vi = t / Q, b = t - vi * Q;
    // the task's largest indices: its last output (a = 7) and its last twiddle read through L1
    if (!in_bounds(it, BND_T, tbase + (size_t)vi * Fx + b + 7 * Q) ||
        (!staged && !in_bounds(it, BND_TWX, (size_t)(Up - 1) * Q + b)))
      continue;
    const float2* s = xs_row + vi * Up;
    const float2* tw = twb + b;
    float2 G[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) G[r] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int p0 = 0; p0 < Up; p0 += 8) {
#pragma unroll
      for (int r = 0; r < 8; ++r) c_fma(G[r], s[p0 + r], tw[(size_t)(p0 + r) * Q]);
    }
    idft8(G);
    float2* o = dst + (size_t)vi * Fx + b;
#pragma unroll
    for (int a = 0; a < 8; ++a) o[a * Q] = G[a];
  }
  if (one.trace) {
    __syncthreads();
    trace_end(one.trace, TRACE_XPASS);
  }
}

// Fold + radix-8 inverse DFT along y of one tile from its rows in shared memory, and the field stores.
// twy: the item's fold twiddles [Fy/8][Vp] (staged in shared memory, or the global table).
template <bool BATCH, bool PAIR, bool TILED>
__device__ __forceinline__ void ypass_tile(const ItemDev& it, const float4* ys_col4, const float2* twy, int2 e, int c,
                                           int xb, float2* out_one, float2* const* outs) {
  const int f = e.y;
  const int Vp = it.Vp, Fx = it.Fx, Fy = it.Fy;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x = xb + 2 * lane;
  if (x >= Fx) return;  // Fx is a multiple of 8, so x + 1 < Fx as well (no barrier in here)
  const int Q = Fy >> 3;
  float2* out = BATCH ? outs[e.x] : out_one;
  // plane slot f = (output plane) I + illumination: slice (il 3 + c) Fz_out + fo of the field
  const int fo = f / it.I, il = f - fo * it.I;
  const long long obase = ((long long)il * 3 * it.Fz_out + (long long)c * it.Fz_out + fo) * it.pstride + x;
  // the thread's largest field index: element x + 1 of the last row of the last periodic tile
  if (!in_bounds(it, BND_OUT, (size_t)(obase + 1 + (long long)(it.ty * Fy - 1) * it.ld + (long long)(it.tx - 1) * Fx)))
    return;
  float2* dst = out + obase;
  const float4* col = ys_col4 + lane;
  if constexpr (!PAIR) {
    for (int b = w; b < Q; b += 8) {
      const float4* tw = reinterpret_cast<const float4*>(twy + (size_t)b * Vp);  // twiddle pairs (Vp % 8 == 0)
      float2 G0[8], G1[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) G0[r] = G1[r] = make_float2(0.f, 0.f);
      for (int p0 = 0; p0 < Vp; p0 += 8) {
#pragma unroll
        for (int r = 0; r < 8; r += 2) {
          const float4 tt = tw[(p0 + r) >> 1];
          const float2 t0 = make_float2(tt.x, tt.y), t1 = make_float2(tt.z, tt.w);
          const float4 d0 = col[(size_t)(p0 + r) * 32], d1 = col[(size_t)(p0 + r + 1) * 32];
          c_fma(G0[r], make_float2(d0.x, d0.y), t0);
          c_fma(G1[r], make_float2(d0.z, d0.w), t0);
          c_fma(G0[r + 1], make_float2(d1.x, d1.y), t1);
          c_fma(G1[r + 1], make_float2(d1.z, d1.w), t1);
        }
      }
      idft8(G0);
      idft8(G1);
#pragma unroll
      for (int a = 0; a < 8; ++a)
        store_row4<TILED>(it, dst, b + a * Q, make_float4(G0[a].x, G0[a].y, G1[a].x, G1[a].y));
    }
    return;
  }
  for (int b = w; b < Q; b += 16) {
    const bool two = b + 8 < Q;
    const float4* twA = reinterpret_cast<const float4*>(twy + (size_t)b * Vp);  // twiddle pairs
    const float4* twB = two ? twA + (size_t)4 * Vp : twA;
    float2 A0[8], A1[8], B0[8], B1[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) A0[r] = A1[r] = B0[r] = B1[r] = make_float2(0.f, 0.f);
    for (int p0 = 0; p0 < Vp; p0 += 8) {
#pragma unroll
      for (int r = 0; r < 8; r += 2) {
        const float4 ta2 = twA[(p0 + r) >> 1], tb2 = twB[(p0 + r) >> 1];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float4 d = col[(size_t)(p0 + r + h) * 32];
          const float2 ta = h ? make_float2(ta2.z, ta2.w) : make_float2(ta2.x, ta2.y);
          const float2 tb = h ? make_float2(tb2.z, tb2.w) : make_float2(tb2.x, tb2.y);
          const float2 d0 = make_float2(d.x, d.y), d1 = make_float2(d.z, d.w);
          c_fma(A0[r + h], d0, ta);
          c_fma(A1[r + h], d1, ta);
          c_fma(B0[r + h], d0, tb);
          c_fma(B1[r + h], d1, tb);
        }
      }
    }
    idft8(A0);
    idft8(A1);
#pragma unroll
    for (int a = 0; a < 8; ++a)
      store_row4<TILED>(it, dst, b + a * Q, make_float4(A0[a].x, A0[a].y, A1[a].x, A1[a].y));
    if (two) {
      idft8(B0);
      idft8(B1);
#pragma unroll
      for (int a = 0; a < 8; ++a)
        store_row4<TILED>(it, dst, b + 8 + a * Q, make_float4(B0[a].x, B0[a].y, B1[a].x, B1[a].y));
    }
  }
}


// Persistent: CTA k takes the tiles k, k + grid, ...; a tile is (64-column block,
// item-plane, component), t = (entry 3 + c) nxb + column block. The x-pass rows of
// a tile sit at their fold positions in shared memory ([Vp][64], padding rows zero);
// two buffers: the rows of the CTA's next tile are copied in (cp.async) while the
// current tile is folded and stored, so no CTA waits on its loads between tiles.
// Lane l owns the column pair (2l, 2l+1). PAIR: warp w takes the residue pairs
// (b, b + 8), b = w, w + 16, ..., so each shared-memory load feeds four complex FMAs
// (long folds); otherwise one residue b = w, w + 8, ... at a time and twice the
// resident warps (short folds, where latency dominates).
template <bool BATCH, bool STW>
__device__ __forceinline__ void ypass_prefetch(const ItemDev& one, const ItemDev* items, const int2* entries,
                                               int t, int n_tiles, int nxb, int rows_f4, float4* buf) {
  if (t < n_tiles) {
    const int r = t / nxb, xb = (t - r * nxb) * 64;
    const int2 e = entries[r / 3];
    const int c = r - (r / 3) * 3;
    const ItemDev& it = BATCH ? items[e.x] : one;
    if (xb < it.Fx) {
      const size_t tbase = ((size_t)e.y * 3 + c) * it.V * it.Fx;
      const float2* src = it.T + tbase;
      for (int i = threadIdx.x; i < it.Vp * 32; i += blockDim.x) {  // row p = i / 32, column pair i % 32
        const int p = i >> 5, x = xb + 2 * (i & 31);
        const int v = fold_order(p, it.V, it.Vp);
        // Fx is even: a pair is in or out as a whole (its second element has the larger index)
        const bool ok = v >= 0 && x < it.Fx && in_bounds(it, BND_T, tbase + (size_t)v * it.Fx + x + 1);
        ptx::cp_async16(ptx::smem_u32(buf + i), ok ? src + (size_t)v * it.Fx + x : src, ok ? 16u : 0u);
      }
      if constexpr (STW) {  // the fold twiddles [Fy/8][Vp] after the rows
        const float4* tw = reinterpret_cast<const float4*>(it.twy);
        for (int i = threadIdx.x; i < (it.Fy >> 3) * it.Vp / 2; i += blockDim.x)
          ptx::cp_async16(ptx::smem_u32(buf + rows_f4 + i), tw + i, in_bounds(it, BND_TWY, 2 * (size_t)i + 1) ? 16u : 0u);
      }
    }
  }
  ptx::cp_async_commit();
}

// STW: the fold twiddles travel with the rows into shared memory (when the largest table fits).
template <bool BATCH, bool PAIR, bool TILED, bool STW>
__global__ void __launch_bounds__(256, PAIR ? 2 : 4) ypass_kernel(const __grid_constant__ ItemDev one,
                                                       const ItemDev* __restrict__ items,
                                                       const int2* __restrict__ entries, int n_tiles, int nxb,
                                                       int rows_f4, int buf_f4, float2* out_one,
                                                       float2* const* __restrict__ outs) {
  extern __shared__ float4 ys_buf[];  // 2 x ([Vp][32] float4 rows = [Vp][64] complex, then the twiddles)
  int t = blockIdx.x;
  if (t >= n_tiles) return;
  ptx::griddep_wait();  // the x-pass rows come from the preceding kernel
  trace_begin(one.trace, TRACE_YPASS);
  ypass_prefetch<BATCH, STW>(one, items, entries, t, n_tiles, nxb, rows_f4, ys_buf);
  for (int b = 0; t < n_tiles; t += gridDim.x, b ^= 1) {
    ypass_prefetch<BATCH, STW>(one, items, entries, t + gridDim.x, n_tiles, nxb, rows_f4,
                               ys_buf + (size_t)(b ^ 1) * buf_f4);
    ptx::cp_async_wait<1>();  // this thread's copies of tile t have landed
    __syncthreads();          // and everyone's
    const int r = t / nxb, xb = (t - r * nxb) * 64;
    const int2 e = entries[r / 3];
    const int c = r - (r / 3) * 3;
    const ItemDev& it = BATCH ? items[e.x] : one;
    if (xb < it.Fx) {
      const float4* cur = ys_buf + (size_t)b * buf_f4;
      ypass_tile<BATCH, PAIR, TILED>(it, cur, STW ? reinterpret_cast<const float2*>(cur + rows_f4) : it.twy, e, c,
                                     xb, out_one, outs);
    }
    __syncthreads();          // buffer b is free for the prefetch of the next iteration
  }
  ptx::cp_async_wait<0>();
  trace_end(one.trace, TRACE_YPASS);  // the loop's last barrier: every warp has stored its rows
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

size_t xpass_smem_bytes(int V, int Up, int Fx) {
  return ((size_t)V * Up + (xpass_twiddles_staged(Up, Fx) ? (size_t)Up * (Fx / 8) : 0)) * sizeof(float2);
}

cudaError_t launch_xpass(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries,
                         size_t smem_bytes, cudaStream_t st) {
  if (n_entries == 0) return cudaSuccess;
  const size_t xs = smem_bytes;
  cudaError_t e;
  if (items) {
    e = allow_max_smem(reinterpret_cast<const void*>(xpass_kernel<true>));
    if (e != cudaSuccess) return e;
    e = launch_pdl(xpass_kernel<true>, dim3(n_entries, 3), dim3(256), xs, st, one, items, d_entries);
    if (e != cudaSuccess) return e;
  } else {
    e = allow_max_smem(reinterpret_cast<const void*>(xpass_kernel<false>));
    if (e != cudaSuccess) return e;
    e = launch_pdl(xpass_kernel<false>, dim3(n_entries, 3), dim3(256), xs, st, one, (const ItemDev*)nullptr,
                   d_entries);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

constexpr int kYpassTwiddleF4 = 1024;  // fold twiddles staged in shared memory up to 16 KB per table

template <bool PAIR, bool TILED, bool STW>
static cudaError_t launch_ypass_t(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries,
                                  int max_Qx, int max_Vp, int tw_f4, float2* out_one, float2* const* d_outs,
                                  cudaStream_t st) {
  const int nxb = (max_Qx * 8 + 63) / 64;
  const long long tiles = (long long)nxb * n_entries * 3;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int rows_f4 = max_Vp * 32;
  const int buf_f4 = rows_f4 + (STW ? tw_f4 : 0);
  const size_t smem = 2 * (size_t)buf_f4 * sizeof(float4);
  const void* fn = items ? reinterpret_cast<const void*>(ypass_kernel<true, PAIR, TILED, STW>)
                         : reinterpret_cast<const void*>(ypass_kernel<false, PAIR, TILED, STW>);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(tiles, (long long)std::max(1, per_sm) * sms);
  if (items)
    return launch_pdl(ypass_kernel<true, PAIR, TILED, STW>, dim3(grid), dim3(256), smem, st, one, items, d_entries,
                      (int)tiles, nxb, rows_f4, buf_f4, (float2*)nullptr, d_outs);
  return launch_pdl(ypass_kernel<false, PAIR, TILED, STW>, dim3(grid), dim3(256), smem, st, one,
                    (const ItemDev*)nullptr, d_entries, (int)tiles, nxb, rows_f4, buf_f4, out_one,
                    (float2* const*)nullptr);
}

template <bool PAIR>
static cudaError_t launch_ypass_p(bool tiled, const ItemDev& one, const ItemDev* items, const int2* d_entries,
                                  int n_entries, int max_Qx, int max_Vp, int tw_f4, float2* out_one,
                                  float2* const* d_outs, cudaStream_t st) {
  const bool stw = tw_f4 <= kYpassTwiddleF4;
#define SCW_YP(T, S) \
  launch_ypass_t<PAIR, T, S>(one, items, d_entries, n_entries, max_Qx, max_Vp, tw_f4, out_one, d_outs, st)
  if (tiled) return stw ? SCW_YP(true, true) : SCW_YP(true, false);
  return stw ? SCW_YP(false, true) : SCW_YP(false, false);
#undef SCW_YP
}

// Pairs pay where the fold is long enough for the saved shared-memory loads to outweigh the halved
// occupancy: measured on 21 x 21 orders (Vp = 24), one residue per warp is 3 us faster per
// 256^3 step (and 0.08 ms per 128-item sweep), so pairs start at Vp = 32.
bool ypass_pairs(int Vp) { return Vp >= 32; }

cudaError_t launch_ypass(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries, int n_pair,
                         int max_Qx, int max_Vp, int max_twy, bool tiled, float2* out_one, float2* const* d_outs,
                         cudaStream_t st, int* launches) {
  const int tw_f4 = (max_twy + 1) / 2;
  int n = 0;
  cudaError_t e = cudaSuccess;
  if (n_pair > 0) {
    e = launch_ypass_p<true>(tiled, one, items, d_entries, n_pair, max_Qx, max_Vp, tw_f4, out_one, d_outs, st);
    ++n;
  }
  if (e == cudaSuccess && n_entries > n_pair) {
    e = launch_ypass_p<false>(tiled, one, items, d_entries + n_pair, n_entries - n_pair, max_Qx, max_Vp, tw_f4,
                              out_one, d_outs, st);
    ++n;
  }
  if (launches) *launches = n;
  return e;
}

size_t recompose_smem_bytes(int V, int Up, int Vp) { return ((size_t)Vp * 64 + (size_t)V * Up) * sizeof(float2); }

cudaError_t launch_recompose(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries, int max_Qx,
                             size_t smem, const float2* S_override, const int* nsplit_override, float2* out_one,
                             float2* const* d_outs, cudaStream_t st) {
  if (n_entries == 0) return cudaSuccess;
  dim3 grid((max_Qx + 7) / 8, n_entries, 3);
  cudaError_t e;
  if (items) {
    e = allow_max_smem(reinterpret_cast<const void*>(recompose_kernel<true>));
    if (e != cudaSuccess) return e;
    recompose_kernel<true><<<grid, 256, smem, st>>>(one, items, d_entries, S_override, nsplit_override, nullptr,
                                                    d_outs);
  } else {
    e = allow_max_smem(reinterpret_cast<const void*>(recompose_kernel<false>));
    if (e != cudaSuccess) return e;
    recompose_kernel<false><<<grid, 256, smem, st>>>(one, nullptr, d_entries, S_override, nsplit_override, out_one,
                                                     nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_spectrum(const Plan& p, float2* S, cudaStream_t st) {
  const size_t n = (size_t)p.Fz * 3 * p.M;
  gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p.S_part, (size_t)p.Fz * 3 * p.M, p.d_nsplit, 3 * p.M,
                                                            p.Fz, S);
  return cudaGetLastError();
}

}  // namespace scw
