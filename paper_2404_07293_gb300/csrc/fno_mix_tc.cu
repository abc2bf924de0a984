// The surrogate's per-mode complex mixing on the 5th-generation tensor cores (BF16 mode).
//
// For every kept mode k and sample b the spectral convolution mixes the C = 32
// channels with a complex C x C matrix:
//   forward        Wh[b][o][k]  = scale sum_i R[k][o][i] Vh[b][i][k]
//   backward data  GVh[b][i][k] =       sum_o conj(R[k][o][i]) G[b][o][k]
// (Li et al.'s Fourier layer; definitions in include/scw_fno.h). Written with
// interleaved reals, x_j = (Re x_i, Im x_i) at j = 2i, 2i + 1, one mode is the
// real product D[b][n] = sum_j X[b][j] Bk[n][j] with M = 128 samples, N = 64,
// K = 64, where row n = 2o + r of Bk holds the coefficients of output o's real
// (r = 0) or imaginary (r = 1) part:
//   forward   (Re R, -Im R) for r = 0,   (Im R, Re R) for r = 1,  at (2i, 2i + 1)
//   backward  (Re R,  Im R) for r = 0,   (-Im R, Re R) for r = 1  (R[k][o][i], o as K)
// The spectra arrive in FP32 (sum of the DFT's K-split partials) and are split
// into X = X_hi + X_lo (BF16 each), so each mode takes two MMAs into one FP32
// accumulator: the products keep the weights' BF16 and nearly FP32 spectra.
//
// A CTA takes kMixModes = 2 consecutive modes and 128 samples (80 KB of shared memory:
// two CTAs per SM, one wave at 256 samples). All 256 threads stage the operands straight
// from global memory into the 128-byte-swizzled K-major layout the MMA reads (rows of 64
// BF16 = 128 bytes; 16-byte chunk g of row r at g ^ (r mod 8)); one thread issues the 16
// MMAs (2 modes x 4 K-steps x 2 halves) into 2 x 64 TMEM columns; the eight warps then
// read the accumulators (warp w: TMEM lanes of its quadrant w mod 4 = 32 samples, outputs
// 16 (w / 4) .. + 15) and write, per sample and output, the two modes as one 8-byte store
// of the K-major result row.
// The single wait (MMA completion) is bounded by a %globaltimer deadline.
#include "fno_internal.cuh"
#include "scw_ptx.cuh"

namespace scw {
namespace fno {

constexpr int kMixModes = 2;
constexpr int kMixRows = 128;
constexpr int kMaxSplitsUnrolled = 2;  // K-split partials of the spectra loaded in one batch
constexpr uint32_t kMixABytes = kMixRows * 128u;   // one mode's A (hi or lo): 128 rows x 64 BF16
constexpr uint32_t kMixBBytes = 64u * 128u;        // one mode's B: 64 rows x 64 BF16
constexpr uint32_t kMixSmem = 2 * kMixModes * kMixABytes + kMixModes * kMixBBytes + 1024u;

__device__ __forceinline__ uint32_t swz128(int row, int chunk) {
  return (uint32_t)row * 128u + ((uint32_t)(chunk ^ (row & 7)) << 4);
}

// (a, b) as one BF16 pair: a in the low half (the lower address), b in the high half
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) { return pack_bf16x2(a, b); }

template <bool CONJ>
__global__ void __launch_bounds__(256, 2) mix_tc_kernel(const float2* __restrict__ X, int splits,
                                                        long long split_stride, long long ld,
                                                        const __nv_bfloat16* __restrict__ R,
                                                        __nv_bfloat16* __restrict__ out, float scale, int B, int Kp,
                                                        int* err, uint64_t timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base_s;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* A_hi = smem;
  uint8_t* A_lo = smem + kMixModes * kMixABytes;
  uint8_t* Bop = smem + 2 * kMixModes * kMixABytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.x * kMixModes, b0 = blockIdx.y * kMixRows;
  const uint64_t deadline = ptx::globaltimer() + timeout_ns;

  if (threadIdx.x == 0) {
    ptx::mbar_init(ptx::smem_u32(&mma_bar), 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_base_s), kMixModes * 64);
    ptx::tmem_relinquish();
  }

  // Operand loads: a thread stages 8 chunks of A (4 complex values each, one 16-byte chunk of BF16)
  // and 4 chunks of B. Every load it needs (R's words, then the first K-split partial of its A
  // chunks) is issued before any value is used: with so little work per CTA the staging is bound
  // by memory round trips.
  constexpr int kChunks = kMixModes * kMixRows * 8 / 256;  // 8 per thread
  const uint32_t* R32 = reinterpret_cast<const uint32_t*>(R);
  constexpr int kBChunks = kMixModes * 64 * 8 / 256;  // 4 per thread
  // B: per mode 64 rows n = 2 p + r (p the output index), chunk g = K values 8 g .. 8 g + 7
  // (inputs 4 g .. 4 g + 3, re and im). R[k][o][i] is stored as BF16 (re, im) pairs.
  uint32_t rv[kBChunks][4];
#pragma unroll
  for (int jj = 0; jj < kBChunks; ++jj) {
    const int q = threadIdx.x + 256 * jj;
    const int mm = q >> 9, n = (q >> 3) & 63, g = q & 7;
    const int p = n >> 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * g + e;  // the K-side index: input i (forward) or output o (backward)
      rv[jj][e] = CONJ ? R32[((size_t)(k0 + mm) * C + j) * C + p] : R32[((size_t)(k0 + mm) * C + p) * C + j];
    }
  }
  // A: the spectra of 128 samples (K-split partials summed)
  float4 va[kChunks], vb[kChunks];
#pragma unroll
  for (int z = 0; z < kMaxSplitsUnrolled; ++z) {
    if (z >= splits) break;  // uniform
#pragma unroll
    for (int j = 0; j < kChunks; ++j) {
      const int q = threadIdx.x + 256 * j;
      const int mm = q >> 10, r = (q >> 3) & (kMixRows - 1), g = q & 7;
      const int b = b0 + r;
      float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
      if (b < B) {
        const float4* src = reinterpret_cast<const float4*>(X + (size_t)(k0 + mm) * ld + (size_t)b * C + 4 * g +
                                                            (size_t)z * split_stride);
        pa = src[0];
        pb = src[1];
      }
      if (z == 0) {
        va[j] = pa;
        vb[j] = pb;
      } else {
        va[j].x += pa.x; va[j].y += pa.y; va[j].z += pa.z; va[j].w += pa.w;
        vb[j].x += pb.x; vb[j].y += pb.y; vb[j].z += pb.z; vb[j].w += pb.w;
      }
    }
  }
  for (int z = kMaxSplitsUnrolled; z < splits; ++z) {  // more K-split partials than the unrolled ones (rare)
#pragma unroll
    for (int j = 0; j < kChunks; ++j) {
      const int q = threadIdx.x + 256 * j;
      const int mm = q >> 10, r = (q >> 3) & (kMixRows - 1), g = q & 7;
      const int b = b0 + r;
      if (b < B) {
        const float4* src = reinterpret_cast<const float4*>(X + (size_t)(k0 + mm) * ld + (size_t)b * C + 4 * g +
                                                            (size_t)z * split_stride);
        const float4 pa = src[0], pb = src[1];
        va[j].x += pa.x; va[j].y += pa.y; va[j].z += pa.z; va[j].w += pa.w;
        vb[j].x += pb.x; vb[j].y += pb.y; vb[j].z += pb.z; vb[j].w += pb.w;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kChunks; ++j) {
    const int q = threadIdx.x + 256 * j;
    const int mm = q >> 10, r = (q >> 3) & (kMixRows - 1), g = q & 7;
    const float v[8] = {va[j].x, va[j].y, va[j].z, va[j].w, vb[j].x, vb[j].y, vb[j].z, vb[j].w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = bf16x2_bits(v[2 * e], v[2 * e + 1]);
      const float h0 = __uint_as_float(h[e] << 16), h1 = __uint_as_float(h[e] & 0xffff0000u);
      l[e] = bf16x2_bits(v[2 * e] - h0, v[2 * e + 1] - h1);
    }
    const uint32_t off = (uint32_t)mm * kMixABytes + swz128(r, g);
    *reinterpret_cast<uint4*>(A_hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(A_lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
#pragma unroll
  for (int jj = 0; jj < kBChunks; ++jj) {
    const int q = threadIdx.x + 256 * jj;
    const int mm = q >> 9, n = (q >> 3) & 63, g = q & 7;
    const int rr = n & 1;
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float re = __uint_as_float(rv[jj][e] << 16), im = __uint_as_float(rv[jj][e] & 0xffff0000u);
      float c0, c1;  // coefficients of the K-side real and imaginary parts
      if (!CONJ) {
        c0 = rr ? im : re;
        c1 = rr ? re : -im;
      } else {
        c0 = rr ? -im : re;
        c1 = rr ? re : im;
      }
      w[e] = bf16x2_bits(c0, c1);
    }
    *reinterpret_cast<uint4*>(Bop + (uint32_t)mm * kMixBBytes + swz128(n, g)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  // generic-proxy stores become visible to the tensor cores' reads
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = ptx::idesc_f16(true, 128, 64);
#pragma unroll
    for (int mm = 0; mm < kMixModes; ++mm) {
      const uint64_t dh = ptx::sw128_desc(ptx::smem_u32(A_hi + mm * kMixABytes));
      const uint64_t dl = ptx::sw128_desc(ptx::smem_u32(A_lo + mm * kMixABytes));
      const uint64_t db = ptx::sw128_desc(ptx::smem_u32(Bop + mm * kMixBBytes));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // K advance of 16 elements = 32 bytes in the swizzled row
        const uint64_t o = (uint64_t)(2 * kk);
        ptx::mma_f16(tmem + (uint32_t)mm * 64u, dh + o, db + o, idesc, kk > 0 ? 1u : 0u);
        ptx::mma_f16(tmem + (uint32_t)mm * 64u, dl + o, db + o, idesc, 1u);
      }
    }
    ptx::mma_commit(ptx::smem_u32(&mma_bar));
  }
  const bool ok = ptx::mbar_wait(ptx::smem_u32(&mma_bar), 0u, deadline);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
    // let the issued MMAs finish before the tensor memory is released
    if (!ptx::mbar_wait(ptx::smem_u32(&mma_bar), 0u, ptx::drain_deadline(timeout_ns)) && lane == 0)
      atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
  } else {
    ptx::tc_fence_after();
    const int quad = warp & 3, half = warp >> 2;
    const int b = b0 + quad * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
    for (int o0 = 16 * half; o0 < 16 * half + 16; o0 += 4) {
      uint32_t v[kMixModes][8];  // mode mm: outputs o0 .. o0 + 3, (re, im) each
#pragma unroll
      for (int mm = 0; mm < kMixModes; ++mm) ptx::tmem_ld_x8(lane_base + (uint32_t)(mm * 64 + 2 * o0), v[mm]);
      ptx::tmem_wait_ld();
      if (b < B) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t w[kMixModes];
#pragma unroll
          for (int mm = 0; mm < kMixModes; ++mm)
            w[mm] = bf16x2_bits(scale * __uint_as_float(v[mm][2 * e]), scale * __uint_as_float(v[mm][2 * e + 1]));
          // row (b, o) of the K-major result, modes k0, k0 + 1 (k0 even: 8-byte aligned)
          *reinterpret_cast<uint2*>(reinterpret_cast<uint32_t*>(out) + ((size_t)b * C + o0 + e) * (Kp / 2) + k0) =
              make_uint2(w[0], w[1]);
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kMixModes * 64);
  }
}

// ---- weight gradient of the mixing: part[block][k][o][i] = sum over the block's samples of
// G[b][o][k] conj(Vh[b][i][k]) (complex; the reduction over blocks follows), and for the DC mode the
// bias gradient part dc[o] = N^2 sum_b Re G[b][o][k_dc].
// Real form per mode, K = (sample b, re/im) = 2 x 128:
//   A[(i, 0)][(b, *)] = (Re V, Im V),  A[(i, 1)][(b, *)] = (-Im V, Re V)      rows (i, r), 64 per mode
//   B[o][(b, *)]      = (Re G, Im G)                                           rows o, 32 per mode
//   D[(i, 0)][o] = Re sum_b G conj(V),  D[(i, 1)][o] = Im sum_b G conj(V).
// Two modes share one MMA (A rows (mode, i, r) = 128, B rows (mode, o) = 64); only the two diagonal
// 64 x 32 blocks of D are kept. V and G enter as BF16 (a weight gradient summed over the samples,
// FP32 accumulation), which keeps the CTA at 97 KB of shared memory: two per SM, so the 256 CTAs
// of a 256-sample batch run in one wave. The operands are transposed (sample to K) while they are
// staged: a warp reads 32 consecutive channels of one sample (256 contiguous bytes) per load.
constexpr int kDrModes = 2;
constexpr int kDrSamples = 128;
constexpr int kDrKAtoms = 2 * kDrSamples / 64;                   // 64-element K atoms: 4
constexpr uint32_t kDrABytes = 128u * 128u * kDrKAtoms;          // [4 atoms][128 rows][64]
constexpr uint32_t kDrBBytes = 64u * 128u * kDrKAtoms;           // [4 atoms][64 rows][64]
constexpr uint32_t kDrSmem = kDrABytes + kDrBBytes + 1024u;

__global__ void __launch_bounds__(256, 2) mix_dr_tc_kernel(const float2* __restrict__ G, const float2* __restrict__ V,
                                                           int splits, long long split_stride, long long ld,
                                                           float* __restrict__ part, int B, int m, int N, int* err,
                                                           uint64_t timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base_s;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Aop = smem;
  uint8_t* Bop = smem + kDrABytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.x * kDrModes, blk = blockIdx.y, b0 = blk * kDrSamples;
  const uint64_t deadline = ptx::globaltimer() + timeout_ns;
  if (threadIdx.x == 0) {
    ptx::mbar_init(ptx::smem_u32(&mma_bar), 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_base_s), 64);
    ptx::tmem_relinquish();
  }
  // one work item: (mode mm, channel c = lane, quad of samples sq): its 4 samples' values of channel c
  // become one 16-byte K chunk (4 x (re, im)) of the rows for c. A thread has 8 items; the loads of
  // kDrBatch items are issued before any is used (the staging is bound by memory round trips).
  constexpr int kDrItems = kDrModes * (kDrSamples / 4) * C / 256;  // 8 per thread
  constexpr int kDrBatch = 2;
#pragma unroll 1
  for (int j0 = 0; j0 < kDrItems; j0 += kDrBatch) {
    float2 v[kDrBatch][4], g[kDrBatch][4];
#pragma unroll
    for (int j = 0; j < kDrBatch; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) v[j][e] = g[j][e] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int z = 0; z < splits; ++z) {
      float2 va[kDrBatch][4], ga[kDrBatch][4];
#pragma unroll
      for (int j = 0; j < kDrBatch; ++j) {
        const int q = threadIdx.x + 256 * (j0 + j);
        const int c = q & (C - 1), sq = (q >> 5) % (kDrSamples / 4), mm = q / (C * kDrSamples / 4);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int b = b0 + 4 * sq + e;
          va[j][e] = ga[j][e] = make_float2(0.f, 0.f);
          if (b < B) {
            const size_t off = (size_t)(k0 + mm) * ld + (size_t)b * C + c + (size_t)z * split_stride;
            va[j][e] = V[off];
            ga[j][e] = G[off];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kDrBatch; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          v[j][e].x += va[j][e].x; v[j][e].y += va[j][e].y;
          g[j][e].x += ga[j][e].x; g[j][e].y += ga[j][e].y;
        }
    }
#pragma unroll
    for (int j = 0; j < kDrBatch; ++j) {
      const int q = threadIdx.x + 256 * (j0 + j);
      const int c = q & (C - 1), sq = (q >> 5) % (kDrSamples / 4), mm = q / (C * kDrSamples / 4);
      // K index of sample s (0..127) and part r: 2 s + r; atom = (2 s) / 64, chunk = ((2 s) % 64) / 8
      const int s0 = 4 * sq, atom = (2 * s0) >> 6, chunk = ((2 * s0) & 63) >> 3;
      uint32_t a0[4], a1[4], bw[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        a0[e] = pack_bf16x2(v[j][e].x, v[j][e].y);   // row (c, 0): (Re V, Im V)
        a1[e] = pack_bf16x2(-v[j][e].y, v[j][e].x);  // row (c, 1): (-Im V, Re V)
        bw[e] = pack_bf16x2(g[j][e].x, g[j][e].y);   // row o = c:  (Re G, Im G)
      }
      const int ra = mm * 64 + 2 * c, rb = mm * C + c;
      const uint32_t oa0 = (uint32_t)atom * (128u * 128u) + swz128(ra, chunk);
      const uint32_t oa1 = (uint32_t)atom * (128u * 128u) + swz128(ra + 1, chunk);
      const uint32_t ob = (uint32_t)atom * (64u * 128u) + swz128(rb, chunk);
      *reinterpret_cast<uint4*>(Aop + oa0) = make_uint4(a0[0], a0[1], a0[2], a0[3]);
      *reinterpret_cast<uint4*>(Aop + oa1) = make_uint4(a1[0], a1[1], a1[2], a1[3]);
      *reinterpret_cast<uint4*>(Bop + ob) = make_uint4(bw[0], bw[1], bw[2], bw[3]);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = ptx::idesc_f16(true, 128, 64);
    bool first = true;
#pragma unroll 1
    for (int at = 0; at < kDrKAtoms; ++at) {
      const uint64_t ad = ptx::sw128_desc(ptx::smem_u32(Aop + at * 128u * 128u));
      const uint64_t bd = ptx::sw128_desc(ptx::smem_u32(Bop + at * 64u * 128u));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t o = (uint64_t)(2 * kk);
        ptx::mma_f16(tmem, ad + o, bd + o, idesc, first ? 0u : 1u);
        first = false;
      }
    }
    ptx::mma_commit(ptx::smem_u32(&mma_bar));
  }
  // bias gradient of the DC mode, in FP32 from the spectra themselves: thread t sums channel t mod 32
  // over the 16 samples of part t / 32 (independent loads), then the 8 parts are added in order
  const int kdc = (m / 2) * m + m / 2;
  const size_t row0 = (size_t)blk * ((size_t)m * m * C * C * 2 + C);
  __shared__ float dc_part[8][C];
  const bool has_dc = kdc >= k0 && kdc < k0 + kDrModes;  // uniform
  if (has_dc) {
    const int o = threadIdx.x & (C - 1), pt = threadIdx.x >> 5;
    float d = 0.f;
    for (int z = 0; z < splits; ++z) {
      float x[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int b = b0 + 16 * pt + e;
        x[e] = b < B ? G[(size_t)kdc * ld + (size_t)b * C + o + (size_t)z * split_stride].x : 0.f;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) d += x[e];
    }
    dc_part[pt][o] = d;
  }
  __syncthreads();
  if (has_dc && threadIdx.x < C) {
    float d = 0.f;
#pragma unroll
    for (int pt = 0; pt < 8; ++pt) d += dc_part[pt][threadIdx.x];
    part[row0 + (size_t)m * m * C * C * 2 + threadIdx.x] = d * (float)N * (float)N;
  }
  const bool ok = ptx::mbar_wait(ptx::smem_u32(&mma_bar), 0u, deadline);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
    if (!ptx::mbar_wait(ptx::smem_u32(&mma_bar), 0u, ptx::drain_deadline(timeout_ns)) && lane == 0)
      atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
  } else {
    ptx::tc_fence_after();
    // thread = row (mode mm, channel i, part r); its mode's 32 output columns o start at 32 mm
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane, mm = row >> 6, i = (row & 63) >> 1, r = row & 1;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    float* dst = part + row0 + ((size_t)(k0 + mm) * C * C + i) * 2 + r;  // + o C 2
#pragma unroll 1
    for (int o0 = 16 * half; o0 < 16 * half + 16; o0 += 8) {
      uint32_t v[8];
      ptx::tmem_ld_x8(lane_base + (uint32_t)(32 * mm + o0), v);
      ptx::tmem_wait_ld();
#pragma unroll
      for (int e = 0; e < 8; ++e) dst[(size_t)(o0 + e) * C * 2] = __uint_as_float(v[e]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 64);
  }
}

int mix_dr_blocks(int B) { return (B + kDrSamples - 1) / kDrSamples; }

cudaError_t launch_mix_dr_tc(const float2* G, const float2* V, int splits, long long split_stride, long long ld,
                             float* part, int B, int m, int N, int* err, uint64_t timeout_ns, cudaStream_t st) {
  if ((m * m) % kDrModes) return cudaErrorInvalidValue;
  const void* fn = reinterpret_cast<const void*>(mix_dr_tc_kernel);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDrSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid(m * m / kDrModes, (B + kDrSamples - 1) / kDrSamples);
  mix_dr_tc_kernel<<<grid, 256, kDrSmem, st>>>(G, V, splits, split_stride, ld, part, B, m, N, err, timeout_ns);
  return cudaGetLastError();
}

cudaError_t launch_mix_tc(bool conj, const float2* X, int splits, long long split_stride, long long ld,
                          const __nv_bfloat16* R, __nv_bfloat16* out, float scale, int B, int m, int Kp, int* err,
                          uint64_t timeout_ns, cudaStream_t st) {
  if ((m * m) % kMixModes || Kp % 8 || (ld % 2) || (split_stride % 2)) return cudaErrorInvalidValue;
  const void* fn = conj ? reinterpret_cast<const void*>(mix_tc_kernel<true>)
                        : reinterpret_cast<const void*>(mix_tc_kernel<false>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid(m * m / kMixModes, (B + kMixRows - 1) / kMixRows);
  if (conj)
    mix_tc_kernel<true><<<grid, 256, kMixSmem, st>>>(X, splits, split_stride, ld, R, out, scale, B, Kp, err,
                                                     timeout_ns);
  else
    mix_tc_kernel<false><<<grid, 256, kMixSmem, st>>>(X, splits, split_stride, ld, R, out, scale, B, Kp, err,
                                                      timeout_ns);
  return cudaGetLastError();
}

}  // namespace fno
}  // namespace scw
