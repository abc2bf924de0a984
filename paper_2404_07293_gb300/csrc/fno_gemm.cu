// Dense contractions D = A B^T over K with a fused epilogue: the surrogate's
// products and the point-set field product.
//
// Tensor-core form (BF16 mode). A and B are K-major BF16 matrices read by TMA
// (2D tensor maps, 64-element = 128-byte inner box, 128-byte swizzle, zero fill
// out of bounds) into a ring of shared-memory stages; one thread issues
// tcgen05.mma (kind::f16, M = 128, N = BN, K = 16) into an FP32 accumulator in
// tensor memory; eight epilogue warps read it back with tcgen05.ld (one TMEM lane
// per thread = one row of D; two warps per 32-lane quadrant split the columns)
// and apply the epilogue 32 columns at a time.
//   warp 0 lane 0   TMA producer (full/empty mbarriers per stage)
//   warp 1 lane 0   MMA issuer; commits each stage back to the producer
//   warps 2-9       epilogue
// The layer products add the 1x1 convolution as a second K segment: for each
// sample s of the tile, D[:, 32 s .. 32 s + 32) += X_s W^T (X_s = that sample's
// activations at the tile's 128 pixels, K = 32 channels, N = 32 MMAs into the
// sample's own accumulator columns). X_s is read from the channel-first layout
// [B][C][P] as an MN-major operand (pixels contiguous, 128-byte swizzle): two 3D
// TMA boxes of {64 pixels, 32 channels, 4 samples} bring the X_s of four samples
// into one operand stage, beside W, so no channel-last copy of the activations
// is needed.
// Every wait is bounded by a %globaltimer deadline; on timeout the CTA sets the
// error word, lets issued copies and MMAs land, frees its tensor memory and exits.
//
// The products (N = pixels per sample, m = kept modes per axis, C = 32 channels):
//   truncated DFT        Vh [B C][2 m^2]  = V_cf [B C][N^2] . D [2 m^2][N^2]^T, stored
//                        mode-major as complex Vh[mode][B C]                     (EPI_MODES)
//   inverse + 1x1 conv   Z^T [N^2][B C]   = E [N^2][Kp] . Wh [B C][Kp]^T + V_cl W^T,
//                        then + c and GELU in the epilogue                       (EPI_LAYER_FWD)
//   backward of both     dV^T [N^2][B C]  = E . GVh^T + dZ_cl W, * GELU'(Z)      (EPI_LAYER_BWD)
//   weight gradient      dW = sum_b dZ_b V_b^T over pixels, 4 samples per tile  (EPI_DW)
// The field synthesis at arbitrary lateral points uses the same engine for its
// product over the orders, E[point][(plane, component)] (EPI_FIELD, split-BF16
// operands along a tripled K; see scw_points.cu).
// SIMT form (FP32 test mode): the same products and the same epilogue code on
// FP32 operands, 128 rows x 32 columns per CTA.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "fno_internal.cuh"
#include "scw_ptx.cuh"

namespace scw {
namespace fno {

template <int BN>
struct GemmCfg {
  static constexpr uint32_t A_BYTES = 128u * 128u;            // 128 rows x 64 bf16
  static constexpr uint32_t B_BYTES = (uint32_t)BN * 128u;     // BN rows x 64 bf16
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr int ST_RAW = (int)(100u * 1024u / STAGE);   // two CTAs per SM
  static constexpr int STAGES = ST_RAW < 2 ? 2 : (ST_RAW > 6 ? 6 : ST_RAW);
  static constexpr uint32_t SMEM = STAGES * STAGE + 1024u;
  static constexpr uint32_t TMEM_COLS = BN < 32 ? 32u : (uint32_t)BN;
};

constexpr int kGemmThreads = 320;
// one operand stage of the 1x1 convolution: two pixel halves, each kSeg2Samples x [32 channels][64
// pixels] (4 KB per sample, 128-byte rows), then the W tile [32][32] (64-byte rows)
constexpr uint32_t kSeg2SampleBytes = 32u * 128u;
constexpr uint32_t kSeg2HalfBytes = kSeg2Samples * kSeg2SampleBytes;
constexpr uint32_t kSeg2Bytes = 2u * kSeg2HalfBytes + 32u * 64u;

template <int BN, int EPI>
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_tc_kernel(const __grid_constant__ CUtensorMap mA,
                                                                  const __grid_constant__ CUtensorMap mB,
                                                                  const __grid_constant__ CUtensorMap mA2,
                                                                  const __grid_constant__ CUtensorMap mW,
                                                                  const __grid_constant__ EpiArgs ea, int K, int kper,
                                                                  int* err, uint64_t timeout_ns) {
  using Cfg = GemmCfg<BN>;
  constexpr int STAGES = Cfg::STAGES;
  static_assert(EPI == EPI_MODES || EPI == EPI_DW || EPI == EPI_FIELD, "layer products run persistent");
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // EPI_FIELD walks the column tiles fastest, so the CTAs that share a row tile of A run together
  constexpr bool NFAST = (EPI == EPI_FIELD);
  const int m0 = (NFAST ? blockIdx.y : blockIdx.x) * 128;
  const int n0 = (EPI == EPI_DW) ? m0 : (NFAST ? blockIdx.x : blockIdx.y) * BN;
  const int kb0 = blockIdx.z * kper;
  const int nkb = max(0, min(K / 64 - kb0, kper));
  const int total = nkb;
  const uint64_t deadline = ptx::globaltimer() + timeout_ns;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[i]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(&acc_bar), 1);
    ptx::mbar_init(ptx::smem_u32(&drain_bar), 1);
    abort_s = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mA);
    ptx::prefetch_tensormap(&mB);
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_base_s), Cfg::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int st = 0, issued = 0;
    uint32_t ph = 0;
    for (int i = 0; i < total && !abort_s; ++i) {
      if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[st]), ph ^ 1u, deadline)) {
        atomicOr(err, DEV_ERR_TIMEOUT_EMPTY);
        abort_s = 1;
        break;
      }
      const uint32_t fb = ptx::smem_u32(&full_bar[st]);
      const uint32_t sa = ptx::smem_u32(smem + (size_t)st * Cfg::STAGE);
      ptx::mbar_arrive_expect_tx(fb, Cfg::STAGE);
      const int kc = (kb0 + i) * 64;
      ptx::tma_load_2d(sa, &mA, kc, m0, fb);
      ptx::tma_load_2d(sa + Cfg::A_BYTES, &mB, kc, n0, fb);
      ++issued;
      if (++st == STAGES) {
        st = 0;
        ph ^= 1u;
      }
    }
    if (abort_s) {
      const uint64_t d2 = ptx::drain_deadline(timeout_ns);
      for (int back = 1; back <= STAGES && back <= issued; ++back) {
        const int i = issued - back;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[i % STAGES]), (uint32_t)(i / STAGES) & 1u, d2)) {
          atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
          break;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- tcgen05.mma issuer ----------------
    constexpr uint32_t idesc = ptx::idesc_f16(true, 128, BN);
    int st = 0;
    uint32_t ph = 0;
    for (int i = 0; i < total && !abort_s; ++i) {
      if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[st]), ph, deadline)) {
        atomicOr(err, DEV_ERR_TIMEOUT_FULL);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t sa = ptx::smem_u32(smem + (size_t)st * Cfg::STAGE);
      const uint64_t da = ptx::sw128_desc(sa), db = ptx::sw128_desc(sa + Cfg::A_BYTES);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t o = (uint64_t)(2 * kk);  // 16 elements = 32 bytes, in 16-byte units
        ptx::mma_f16(tmem, da + o, db + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      }
      ptx::mma_commit(ptx::smem_u32(&empty_bar[st]));
      if (++st == STAGES) {
        st = 0;
        ph ^= 1u;
      }
    }
    if (!abort_s) {
      ptx::mma_commit(ptx::smem_u32(&acc_bar));
    } else {
      ptx::mma_commit(ptx::smem_u32(&drain_bar));
      if (!ptx::mbar_wait(ptx::smem_u32(&drain_bar), 0u, ptx::drain_deadline(timeout_ns)))
        atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int grp = warp & 3;         // TMEM lanes 32 grp .. 32 grp + 31
    const int half = (warp - 2) >> 2;  // column chunks half, half + 2, ...
    bool ok = true;
    for (;;) {
      if (ptx::mbar_try_wait(ptx::smem_u32(&acc_bar), 0u)) break;
      if (abort_s || ptx::globaltimer() > deadline) {
        ok = false;
        break;
      }
    }
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0 && !abort_s) atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
      abort_s = 1;
    } else {
      ptx::tc_fence_after();
      const int row = m0 + grp * 32 + lane;
      const uint32_t lane_addr = tmem + ((uint32_t)(grp * 32) << 16);
      const int col_end = (EPI == EPI_DW) ? n0 + 128 : ea.cols;
#pragma unroll 1
      for (int c = half; c < BN / 32; c += 2) {
        if (n0 + 32 * c >= col_end) break;  // warp-uniform
        uint32_t r0[8], r1[8], r2[8], r3[8];
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c), r0);
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c + 8), r1);
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c + 16), r2);
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c + 24), r3);
        ptx::tmem_wait_ld();
        float acc[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          acc[j] = total > 0 ? __uint_as_float(r0[j]) : 0.f;
          acc[8 + j] = total > 0 ? __uint_as_float(r1[j]) : 0.f;
          acc[16 + j] = total > 0 ? __uint_as_float(r2[j]) : 0.f;
          acc[24 + j] = total > 0 ? __uint_as_float(r3[j]) : 0.f;
        }
        epilogue<EPI, __nv_bfloat16, true>(ea, nullptr, nullptr, row, n0 + 32 * c, blockIdx.z, acc);
      }
    }
  }

  // ---------------- teardown ----------------
  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// Persistent form of the layer products (EPI_LAYER_FWD / EPI_LAYER_BWD, BN = 256): one
// CTA per SM walks the output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (pixel
// tile fastest, so CTAs in flight share their Wh / GVh tile through L2). Four operand
// stages; two 256-column TMEM accumulators, so the epilogue of one tile runs while the
// MMAs of the next one are issued (acc_full / acc_empty barriers, as in the contraction).
// Twelve epilogue warps (three per TMEM lane quadrant) share the 8 column chunks.
constexpr int kLayerStages = 4;
constexpr uint32_t kLayerStage = GemmCfg<256>::STAGE;
constexpr uint32_t kLayerSmem = kLayerStages * kLayerStage + 1024u;
constexpr int kLayerEpiWarps = 12;  // three per 32-lane TMEM quadrant
constexpr int kLayerThreads = 32 * (2 + kLayerEpiWarps);

// Backward layer epilogue with the GELU'(Z) values (channel-last, BF16, stored by the forward) of
// its row and chunk already in registers: dV = D (the 1x1 convolution is in the accumulator), times
// GELU'(Z) where Z exists. Those rows come from DRAM and do not depend on the accumulator, so the
// persistent kernel loads them one chunk ahead (the first chunk of a tile before the wait for its
// accumulator).
__device__ __forceinline__ void zrow_load(const EpiArgs& a, int row, int col0, uint4 (&q)[4]) {
  const int b = col0 / C;
  if (a.g_in != nullptr && row < a.P && b < a.B) {
    const uint4* s = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(a.g_in) +
                                                    ((size_t)b * a.P + row) * C);
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = __ldg(s + j);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = make_uint4(0u, 0u, 0u, 0u);
  }
}

__device__ __forceinline__ void epilogue_bwd_z(const EpiArgs& a, int row, int col0, const float (&acc)[32],
                                               const uint4 (&q)[4]) {
  const int p = row, b = col0 / C;
  if (p >= a.P || b >= a.B) return;
  const size_t cl = ((size_t)b * a.P + p) * C;
  float d[32];
#pragma unroll
  for (int i = 0; i < C; ++i) d[i] = a.alpha * acc[i];
  if (a.g_in) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t w[4] = {q[j].x, q[j].y, q[j].z, q[j].w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        d[8 * j + 2 * h] *= __uint_as_float(w[h] << 16);
        d[8 * j + 2 * h + 1] *= __uint_as_float(w[h] & 0xffff0000u);
      }
    }
  }
  if (a.out_cl) st32(static_cast<__nv_bfloat16*>(a.out_cl) + cl, d);
  if (a.out_cf) {
    __nv_bfloat16* cf = static_cast<__nv_bfloat16*>(a.out_cf) + (size_t)b * C * a.P + p;
#pragma unroll
    for (int i = 0; i < C; ++i) cf[(size_t)i * a.P] = __float2bfloat16_rn(d[i]);
  }
}

template <int EPI>
__global__ void __launch_bounds__(kLayerThreads, 1) gemm_layer_persistent(const __grid_constant__ CUtensorMap mA,
                                                                         const __grid_constant__ CUtensorMap mB,
                                                                         const __grid_constant__ CUtensorMap mA2,
                                                                         const __grid_constant__ CUtensorMap mW,
                                                                         const __grid_constant__ EpiArgs ea, int K,
                                                                         int m_tiles, int n_tiles, int* err,
                                                                         uint64_t timeout_ns) {
  constexpr int BN = 256;
  constexpr int STAGES = kLayerStages;
  constexpr uint32_t A_BYTES = GemmCfg<256>::A_BYTES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ __align__(16) float w_s[C * C];
  __shared__ __align__(16) float b_s[C];

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = K / 64;
  const uint64_t deadline = ptx::globaltimer() + timeout_ns;
  constexpr bool SEG2 = (EPI == EPI_LAYER_FWD || EPI == EPI_LAYER_BWD);
  const int n_tasks = m_tiles * n_tiles;
  // the layer products walk the row tiles fastest (CTAs in flight share a Wh / GVh tile); the
  // field product and the truncated DFT walk the column tiles fastest (they share a row tile of
  // the points table / the activations)
  constexpr bool NFAST = (EPI == EPI_FIELD || EPI == EPI_MODES);
  auto tile_m0 = [&](int t) { return (NFAST ? t / n_tiles : t % m_tiles) * 128; };
  auto tile_n0 = [&](int t) { return (NFAST ? t % n_tiles : t / m_tiles) * BN; };
  // samples of a tile whose 1x1 convolution runs as an extra K segment, and the operand stages
  // they take (kSeg2Samples samples each)
  auto tile_nseg = [&](int n0) { return SEG2 ? max(0, min(BN / C, ea.B - n0 / C)) : 0; };
  auto tile_ngrp = [&](int n0) { return (tile_nseg(n0) + kSeg2Samples - 1) / kSeg2Samples; };
  static_assert(kSeg2Bytes <= kLayerStage, "a 1x1-convolution stage must fit an operand stage");

  if (threadIdx.x < C) {
    const __nv_bfloat16* bias = static_cast<const __nv_bfloat16*>(ea.bias);
    b_s[threadIdx.x] = bias ? __bfloat162float(bias[threadIdx.x]) : 0.f;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(ptx::smem_u32(&accf_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&acce_bar[i]), kLayerEpiWarps);  // one arrival per epilogue warp
    }
    ptx::mbar_init(ptx::smem_u32(&drain_bar), 1);
    abort_s = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mA);
    ptx::prefetch_tensormap(&mB);
    ptx::prefetch_tensormap(&mA2);
    ptx::prefetch_tensormap(&mW);
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_base_s), 2 * BN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int st = 0, issued = 0;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < n_tasks && !abort_s; t += gridDim.x) {
      const int m0 = tile_m0(t), n0 = tile_n0(t);
      const int total = nkb + tile_ngrp(n0);
      for (int i = 0; i < total && !abort_s; ++i) {
        if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[st]), ph ^ 1u, deadline)) {
          atomicOr(err, DEV_ERR_TIMEOUT_EMPTY);
          abort_s = 1;
          break;
        }
        const uint32_t fb = ptx::smem_u32(&full_bar[st]);
        const uint32_t sa = ptx::smem_u32(smem + (size_t)st * kLayerStage);
        if (i < nkb) {
          ptx::mbar_arrive_expect_tx(fb, kLayerStage);
          ptx::tma_load_2d(sa, &mA, i * 64, m0, fb);
          ptx::tma_load_2d(sa + A_BYTES, &mB, i * 64, n0, fb);
        } else {
          // X_s for samples smp0 .. smp0 + kSeg2Samples - 1 (pixels m0 .. m0 + 63, then
          // m0 + 64 .. m0 + 127; the pixel count is a multiple of 128), then W
          const int smp0 = n0 / C + kSeg2Samples * (i - nkb);
          ptx::mbar_arrive_expect_tx(fb, kSeg2Bytes);
          ptx::tma_load_3d(sa, &mA2, m0, 0, smp0, fb);
          ptx::tma_load_3d(sa + kSeg2HalfBytes, &mA2, m0 + 64, 0, smp0, fb);
          ptx::tma_load_2d(sa + 2u * kSeg2HalfBytes, &mW, 0, 0, fb);
        }
        ++issued;
        if (++st == STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    if (abort_s) {
      const uint64_t d2 = ptx::drain_deadline(timeout_ns);
      for (int back = 1; back <= STAGES && back <= issued; ++back) {
        const int i = issued - back;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[i % STAGES]), (uint32_t)(i / STAGES) & 1u, d2)) {
          atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
          break;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- tcgen05.mma issuer ----------------
    constexpr uint32_t idesc = ptx::idesc_f16(true, 128, BN);
    constexpr uint32_t idesc32 = ptx::idesc_f16(true, 128, 32, true);  // A (activations) MN-major
    int st = 0, lt = 0;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < n_tasks && !abort_s; t += gridDim.x, ++lt) {
      const int n0 = tile_n0(t);
      const int nseg = tile_nseg(n0);
      const int total = nkb + tile_ngrp(n0);
      const int acc = lt & 1;
      if (!ptx::mbar_wait(ptx::smem_u32(&acce_bar[acc]), ((uint32_t)(lt >> 1) & 1u) ^ 1u, deadline)) {
        atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
      for (int i = 0; i < total; ++i) {
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[st]), ph, deadline)) {
          atomicOr(err, DEV_ERR_TIMEOUT_FULL);
          abort_s = 1;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t sa = ptx::smem_u32(smem + (size_t)st * kLayerStage);
        if (i < nkb) {
          const uint64_t da = ptx::sw128_desc(sa), db = ptx::sw128_desc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = (uint64_t)(2 * kk);
            ptx::mma_f16(d_tmem, da + o, db + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          }
        } else {
          const int s0 = kSeg2Samples * (i - nkb);
          const uint64_t db = ptx::sw64_desc(sa + 2u * kSeg2HalfBytes);
          for (int j = 0; j < kSeg2Samples && s0 + j < nseg; ++j) {
            // the two 64-pixel halves of sample j are kSeg2HalfBytes apart; K = 16 channels = 2048 bytes
            const uint64_t da = ptx::sw128_mn_desc(sa + (uint32_t)j * kSeg2SampleBytes, kSeg2HalfBytes);
            const uint32_t d = d_tmem + (uint32_t)(C * (s0 + j));
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
              ptx::mma_f16(d, da + (uint64_t)(kk * (2048 >> 4)), db + (uint64_t)(2 * kk), idesc32, 1u);
          }
        }
        ptx::mma_commit(ptx::smem_u32(&empty_bar[st]));
        if (++st == STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (abort_s) break;
      ptx::mma_commit(ptx::smem_u32(&accf_bar[acc]));
    }
    if (abort_s) {
      ptx::mma_commit(ptx::smem_u32(&drain_bar));
      if (!ptx::mbar_wait(ptx::smem_u32(&drain_bar), 0u, ptx::drain_deadline(timeout_ns)))
        atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int grp = warp & 3;           // TMEM lanes 32 grp .. 32 grp + 31
    const int third = (warp - 2) >> 2;  // column chunks third, third + 3, ...
    int lt = 0;
    for (int t = blockIdx.x; t < n_tasks; t += gridDim.x, ++lt) {
      const int m0 = tile_m0(t), n0 = tile_n0(t);
      const int acc = lt & 1;
      const int row = m0 + grp * 32 + lane;
      uint4 zc[4], zn[4];  // EPI_LAYER_BWD: GELU'(Z) of the current and the next chunk
      if constexpr (EPI == EPI_LAYER_BWD) zrow_load(ea, row, n0 + 32 * third, zc);
      bool ok = true;
      for (;;) {
        if (ptx::mbar_try_wait(ptx::smem_u32(&accf_bar[acc]), (uint32_t)(lt >> 1) & 1u)) break;
        if (abort_s || ptx::globaltimer() > deadline) {
          ok = false;
          break;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0 && !abort_s) atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t lane_addr = tmem + (uint32_t)(acc * BN) + ((uint32_t)(grp * 32) << 16);
#pragma unroll 1
      for (int c = third; c < BN / 32; c += 3) {
        if (n0 + 32 * c >= ea.cols) break;  // warp-uniform
        if constexpr (EPI == EPI_LAYER_BWD) {
          if (c + 3 < BN / 32) zrow_load(ea, row, n0 + 32 * (c + 3), zn);
        }
        uint32_t r0[8], r1[8], r2[8], r3[8];
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c), r0);
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c + 8), r1);
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c + 16), r2);
        ptx::tmem_ld_x8(lane_addr + (uint32_t)(32 * c + 24), r3);
        ptx::tmem_wait_ld();
        float a[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          a[j] = __uint_as_float(r0[j]);
          a[8 + j] = __uint_as_float(r1[j]);
          a[16 + j] = __uint_as_float(r2[j]);
          a[24 + j] = __uint_as_float(r3[j]);
        }
        if constexpr (EPI == EPI_LAYER_BWD) {
          epilogue_bwd_z(ea, row, n0 + 32 * c, a, zc);
#pragma unroll
          for (int j = 0; j < 4; ++j) zc[j] = zn[j];
        } else {
          epilogue<EPI, __nv_bfloat16, true>(ea, w_s, b_s, row, n0 + 32 * c, 0, a);
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&acce_bar[acc]));
    }
  }

  // ---------------- teardown ----------------
  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 2 * BN);
  }
}

template <int EPI>
__global__ void __launch_bounds__(128) gemm_simt_kernel(const float* __restrict__ A, long long lda,
                                                        const float* __restrict__ Bm, long long ldb, EpiArgs ea,
                                                        int a_rows, int NB_rows, int K, int kper) {
  __shared__ float As[32][129];
  __shared__ float Bs[32][33];
  __shared__ __align__(16) float w_s[C * C];
  __shared__ __align__(16) float b_s[C];
  const int t = threadIdx.x;
  if constexpr (EPI == EPI_LAYER_FWD || EPI == EPI_LAYER_BWD) {
    const float* w = static_cast<const float*>(ea.w);
    const float* bias = static_cast<const float*>(ea.bias);
    for (int i = t; i < C * C; i += blockDim.x) w_s[i] = w[i];
    if (t < C) b_s[t] = bias ? bias[t] : 0.f;
  }
  const int m0 = blockIdx.x * 128;
  const int n0 = (EPI == EPI_DW) ? m0 + 32 * blockIdx.y : blockIdx.y * 32;
  const int kbeg = blockIdx.z * kper * 64, kend = min(K, kbeg + kper * 64);
  float acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
  for (int kc = kbeg; kc < kend; kc += 32) {
    const int k = kc + (t & 31);
#pragma unroll 4
    for (int r = t >> 5; r < 128; r += 4) {
      const int row = m0 + r;
      As[t & 31][r] = (row < a_rows && k < kend) ? A[(size_t)row * lda + k] : 0.f;
    }
#pragma unroll
    for (int c = t >> 5; c < 32; c += 4) {
      const int col = n0 + c;
      Bs[t & 31][c] = (col < NB_rows && k < kend) ? Bm[(size_t)col * ldb + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float a = As[kk][t];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = fmaf(a, Bs[kk][j], acc[j]);
    }
    __syncthreads();
  }
  const int col_end = (EPI == EPI_DW) ? m0 + 128 : ea.cols;
  if (n0 < col_end) epilogue<EPI, float, false>(ea, w_s, b_s, m0 + t, n0, blockIdx.z, acc);
}

// ---------------------------------------------------------------- host side ---
template <int BN, int EPI>
static cudaError_t launch_tc_t(const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mA2,
                               const CUtensorMap& mW, const EpiArgs& ea, int M, int N, int K, int splits, int* err,
                               uint64_t timeout_ns, cudaStream_t st) {
  using Cfg = GemmCfg<BN>;
  const void* fn = reinterpret_cast<const void*>(gemm_tc_kernel<BN, EPI>);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  const int nkb = K / 64;
  const int kper = (nkb + splits - 1) / splits;
  const dim3 grid = EPI == EPI_FIELD ? dim3((N + BN - 1) / BN, (M + 127) / 128, splits)
                                     : dim3((M + 127) / 128, EPI == EPI_DW ? 1 : (N + BN - 1) / BN, splits);
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  gemm_tc_kernel<BN, EPI><<<grid, kGemmThreads, Cfg::SMEM, st>>>(mA, mB, mA2, mW, ea, K, kper, err, timeout_ns);
  return cudaGetLastError();
}

// ---- backward truncated DFT of dZ fused with the weight gradient dW = sum_b dZ_b V_b^T ----
// Both products read dZ (channel-first, rows (b, o), K = pixels) as A. Tile (m0, n0) of the DFT
// (2m^2 = 512 output columns, two column tiles of 256) also multiplies, over one half of K (the
// first half for n0 = 0, the second for n0 = 256), its 128 rows of dZ by the same 128 rows of V
// (rows (b, i), a third operand in the stage) into a 128-column accumulator beside the DFT's; the
// diagonal 32 x 32 blocks are the four samples' dW_b partials (K half = split 0 or 1). dZ is then
// read once per layer instead of twice. Stages: A 16 KB + D 32 KB + V 16 KB, three in flight.
// One accumulator pair per CTA (no double buffering: at batch <= 256 every CTA has one tile).
constexpr int kDwStages = 3;
constexpr uint32_t kDwStage = 128u * 128u + 256u * 128u + 128u * 128u;
constexpr uint32_t kDwSmem = kDwStages * kDwStage + 1024u;

__global__ void __launch_bounds__(kLayerThreads, 1) gemm_dft_dw_kernel(const __grid_constant__ CUtensorMap mA,
                                                                      const __grid_constant__ CUtensorMap mB,
                                                                      const __grid_constant__ CUtensorMap mV,
                                                                      const __grid_constant__ EpiArgs ea,
                                                                      const __grid_constant__ EpiArgs ew, int K,
                                                                      int m_tiles, int* err, uint64_t timeout_ns) {
  constexpr int BN = 256, STAGES = kDwStages, n_tiles = 2;
  constexpr uint32_t A_BYTES = 128u * 128u, B_BYTES = 256u * 128u;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar;
  __shared__ __align__(8) uint64_t acce_bar;
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tasks = m_tiles * n_tiles;
  const int nkb = K / 64, half = nkb / 2;  // K blocks; the dW half of tile (m, n): [n half, (n + 1) half)
  const uint64_t deadline = ptx::globaltimer() + timeout_ns;
  // column tiles fastest: the two tiles of a row tile run side by side and share its dZ rows in L2
  auto tile_m0 = [&](int t) { return (t / n_tiles) * 128; };
  auto tile_n = [&](int t) { return t % n_tiles; };

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[i]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(&accf_bar), 1);
    ptx::mbar_init(ptx::smem_u32(&acce_bar), kLayerEpiWarps);
    ptx::mbar_init(ptx::smem_u32(&drain_bar), 1);
    abort_s = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mA);
    ptx::prefetch_tensormap(&mB);
    ptx::prefetch_tensormap(&mV);
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_base_s), 512);  // DFT columns [0, 256), dW columns [256, 384)
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int st = 0, issued = 0;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < n_tasks && !abort_s; t += gridDim.x) {
      const int m0 = tile_m0(t), n = tile_n(t);
      for (int i = 0; i < nkb && !abort_s; ++i) {
        if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[st]), ph ^ 1u, deadline)) {
          atomicOr(err, DEV_ERR_TIMEOUT_EMPTY);
          abort_s = 1;
          break;
        }
        const bool dw = i >= n * half && i < (n + 1) * half;
        const uint32_t fb = ptx::smem_u32(&full_bar[st]);
        const uint32_t sa = ptx::smem_u32(smem + (size_t)st * kDwStage);
        ptx::mbar_arrive_expect_tx(fb, A_BYTES + B_BYTES + (dw ? A_BYTES : 0u));
        ptx::tma_load_2d(sa, &mA, i * 64, m0, fb);
        ptx::tma_load_2d(sa + A_BYTES, &mB, i * 64, n * BN, fb);
        if (dw) ptx::tma_load_2d(sa + A_BYTES + B_BYTES, &mV, i * 64, m0, fb);
        ++issued;
        if (++st == STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    if (abort_s) {
      const uint64_t d2 = ptx::drain_deadline(timeout_ns);
      for (int back = 1; back <= STAGES && back <= issued; ++back) {
        const int i = issued - back;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[i % STAGES]), (uint32_t)(i / STAGES) & 1u, d2)) {
          atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
          break;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- tcgen05.mma issuer ----------------
    constexpr uint32_t idesc = ptx::idesc_f16(true, 128, BN);
    constexpr uint32_t idesc_dw = ptx::idesc_f16(true, 128, 128);
    int st = 0, lt = 0;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < n_tasks && !abort_s; t += gridDim.x, ++lt) {
      const int n = tile_n(t);
      // the epilogue has read the previous tile's accumulators
      if (!ptx::mbar_wait(ptx::smem_u32(&acce_bar), ((uint32_t)lt & 1u) ^ 1u, deadline)) {
        atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      for (int i = 0; i < nkb; ++i) {
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[st]), ph, deadline)) {
          atomicOr(err, DEV_ERR_TIMEOUT_FULL);
          abort_s = 1;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t sa = ptx::smem_u32(smem + (size_t)st * kDwStage);
        const uint64_t da = ptx::sw128_desc(sa), db = ptx::sw128_desc(sa + A_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          ptx::mma_f16(tmem, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, (i > 0 || kk > 0) ? 1u : 0u);
        const int j = i - n * half;  // position in this tile's dW half of K
        if (j >= 0 && j < half) {
          const uint64_t dv = ptx::sw128_desc(sa + A_BYTES + B_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            ptx::mma_f16(tmem + 256u, da + (uint64_t)(2 * kk), dv + (uint64_t)(2 * kk), idesc_dw,
                         (j > 0 || kk > 0) ? 1u : 0u);
        }
        ptx::mma_commit(ptx::smem_u32(&empty_bar[st]));
        if (++st == STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (abort_s) break;
      ptx::mma_commit(ptx::smem_u32(&accf_bar));
    }
    if (abort_s) {
      ptx::mma_commit(ptx::smem_u32(&drain_bar));
      if (!ptx::mbar_wait(ptx::smem_u32(&drain_bar), 0u, ptx::drain_deadline(timeout_ns)))
        atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int grp = warp & 3;           // TMEM lanes 32 grp .. 32 grp + 31
    const int third = (warp - 2) >> 2;  // DFT column chunks third, third + 3, ...; third 0 also takes dW
    int lt = 0;
    for (int t = blockIdx.x; t < n_tasks; t += gridDim.x, ++lt) {
      const int m0 = tile_m0(t), n = tile_n(t);
      bool ok = true;
      for (;;) {
        if (ptx::mbar_try_wait(ptx::smem_u32(&accf_bar), (uint32_t)lt & 1u)) break;
        if (abort_s || ptx::globaltimer() > deadline) {
          ok = false;
          break;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0 && !abort_s) atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      const int row = m0 + grp * 32 + lane;
      const uint32_t lane_addr = tmem + ((uint32_t)(grp * 32) << 16);
      auto load32 = [&](uint32_t col, float (&a)[32]) {
        uint32_t r0[8], r1[8], r2[8], r3[8];
        ptx::tmem_ld_x8(lane_addr + col, r0);
        ptx::tmem_ld_x8(lane_addr + col + 8u, r1);
        ptx::tmem_ld_x8(lane_addr + col + 16u, r2);
        ptx::tmem_ld_x8(lane_addr + col + 24u, r3);
        ptx::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          a[q] = __uint_as_float(r0[q]);
          a[8 + q] = __uint_as_float(r1[q]);
          a[16 + q] = __uint_as_float(r2[q]);
          a[24 + q] = __uint_as_float(r3[q]);
        }
      };
#pragma unroll 1
      for (int c = third; c < BN / 32; c += 3) {
        if (n * BN + 32 * c >= ea.cols) break;  // warp-uniform
        float a[32];
        load32((uint32_t)(32 * c), a);
        epilogue<EPI_MODES, __nv_bfloat16, true>(ea, nullptr, nullptr, row, n * BN + 32 * c, 0, a);
      }
      if (third == 0) {  // the diagonal block of this quadrant's sample: dW_b partial, K half n
        float a[32];
        load32(256u + (uint32_t)(32 * grp), a);
        epilogue<EPI_DW, __nv_bfloat16, true>(ew, nullptr, nullptr, row, 32 * grp, n, a);
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&acce_bar));
    }
  }

  // ---------------- teardown ----------------
  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

cudaError_t launch_gemm_dft_dw(const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mV,
                               const EpiArgs& ea, const EpiArgs& ew, int M, int N, int K, int* err,
                               uint64_t timeout_ns, cudaStream_t st) {
  if (N != 512 || K % 128 != 0 || ew.splits != 2) return cudaErrorInvalidValue;
  const void* fn = reinterpret_cast<const void*>(gemm_dft_dw_kernel);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int m_tiles = (M + 127) / 128;
  const int grid = std::max(1, std::min(2 * m_tiles, sms));
  gemm_dft_dw_kernel<<<grid, kLayerThreads, kDwSmem, st>>>(mA, mB, mV, ea, ew, K, m_tiles, err, timeout_ns);
  return cudaGetLastError();
}

template <int EPI>
static cudaError_t launch_layer_persistent(const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mA2,
                                           const CUtensorMap& mW, const EpiArgs& ea, int M, int N, int K, int* err,
                                           uint64_t timeout_ns, cudaStream_t st) {
  const void* fn = reinterpret_cast<const void*>(gemm_layer_persistent<EPI>);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int m_tiles = (M + 127) / 128, n_tiles = (N + 255) / 256;
  const int grid = std::max(1, std::min(m_tiles * n_tiles, sms));
  gemm_layer_persistent<EPI><<<grid, kLayerThreads, kLayerSmem, st>>>(mA, mB, mA2, mW, ea, K, m_tiles, n_tiles, err,
                                                                      timeout_ns);
  return cudaGetLastError();
}

template <int EPI>
static cudaError_t launch_tc_bn(int BN, const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mA2,
                                const CUtensorMap& mW, const EpiArgs& ea, int M, int N, int K, int splits, int* err,
                                uint64_t timeout_ns, cudaStream_t st) {
  switch (BN) {
    case 32: return launch_tc_t<32, EPI>(mA, mB, mA2, mW, ea, M, N, K, splits, err, timeout_ns, st);
    case 64: return launch_tc_t<64, EPI>(mA, mB, mA2, mW, ea, M, N, K, splits, err, timeout_ns, st);
    case 128: return launch_tc_t<128, EPI>(mA, mB, mA2, mW, ea, M, N, K, splits, err, timeout_ns, st);
    case 256: return launch_tc_t<256, EPI>(mA, mB, mA2, mW, ea, M, N, K, splits, err, timeout_ns, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gemm_tc(int epi, int BN, const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mA2,
                           const CUtensorMap& mW, const EpiArgs& ea, int M, int N, int K, int splits, int* err,
                           uint64_t timeout_ns, cudaStream_t st) {
  if (K % 64 != 0 || splits < 1) return cudaErrorInvalidValue;
  const bool layer = epi == EPI_LAYER_FWD || epi == EPI_LAYER_BWD;
  // the 1x1 segment shares the accumulator: the DFT part must come pre-scaled (alpha 1)
  if (layer && (splits != 1 || BN != 256 || ea.alpha != 1.0f)) return cudaErrorInvalidValue;
  switch (epi) {
    case EPI_MODES:
      // BN 256 without K splits: the persistent form (four stages, overlapped epilogue)
      if (BN == 256 && splits == 1)
        return launch_layer_persistent<EPI_MODES>(mA, mB, mA2, mW, ea, M, N, K, err, timeout_ns, st);
      return launch_tc_bn<EPI_MODES>(BN, mA, mB, mA2, mW, ea, M, N, K, splits, err, timeout_ns, st);
    case EPI_LAYER_FWD:
      return launch_layer_persistent<EPI_LAYER_FWD>(mA, mB, mA2, mW, ea, M, N, K, err, timeout_ns, st);
    case EPI_LAYER_BWD:
      return launch_layer_persistent<EPI_LAYER_BWD>(mA, mB, mA2, mW, ea, M, N, K, err, timeout_ns, st);
    case EPI_DW:
      return BN == 128 ? launch_tc_t<128, EPI_DW>(mA, mB, mA2, mW, ea, M, N, K, splits, err, timeout_ns, st)
                       : cudaErrorInvalidValue;
    case EPI_FIELD:
      if (splits != 1) return cudaErrorInvalidValue;
      // BN 256: the persistent form (epilogue of one tile overlapping the next tile's MMAs)
      return BN == 256 ? launch_layer_persistent<EPI_FIELD>(mA, mB, mA2, mW, ea, M, N, K, err, timeout_ns, st)
                       : launch_tc_bn<EPI_FIELD>(BN, mA, mB, mA2, mW, ea, M, N, K, 1, err, timeout_ns, st);
    default: return cudaErrorInvalidValue;
  }
}

int gemm_tc_ctas_per_sm(int BN) {
  const uint32_t smem = BN == 32    ? GemmCfg<32>::SMEM
                        : BN == 64  ? GemmCfg<64>::SMEM
                        : BN == 128 ? GemmCfg<128>::SMEM
                                    : GemmCfg<256>::SMEM;
  return smem <= 110u * 1024u ? 2 : 1;
}

template <int EPI>
static cudaError_t launch_simt_t(const float* A, long long lda, const float* B, long long ldb, const EpiArgs& ea, int M,
                                 int N, int K, int splits, cudaStream_t st) {
  const int nkb = (K + 63) / 64;
  const int kper = (nkb + splits - 1) / splits;
  const dim3 grid((M + 127) / 128, EPI == EPI_DW ? 4 : (N + 31) / 32, splits);
  // rows of A and B that exist (EPI_DW tiles cover whole 4-sample groups; A and B hold B*C rows)
  const int a_rows = EPI == EPI_DW ? ea.rows : M;
  const int nb_rows = EPI == EPI_DW ? ea.rows : N;
  gemm_simt_kernel<EPI><<<grid, 128, 0, st>>>(A, lda, B, ldb, ea, a_rows, nb_rows, K, kper);
  return cudaGetLastError();
}

cudaError_t launch_gemm_simt(int epi, const float* A, long long lda, const float* B, long long ldb, const EpiArgs& ea,
                             int M, int N, int K, int splits, cudaStream_t st) {
  if (splits < 1) return cudaErrorInvalidValue;
  if ((epi == EPI_LAYER_FWD || epi == EPI_LAYER_BWD) && splits != 1) return cudaErrorInvalidValue;
  switch (epi) {
    case EPI_MODES: return launch_simt_t<EPI_MODES>(A, lda, B, ldb, ea, M, N, K, splits, st);
    case EPI_LAYER_FWD: return launch_simt_t<EPI_LAYER_FWD>(A, lda, B, ldb, ea, M, N, K, splits, st);
    case EPI_LAYER_BWD: return launch_simt_t<EPI_LAYER_BWD>(A, lda, B, ldb, ea, M, N, K, splits, st);
    case EPI_DW: return launch_simt_t<EPI_DW>(A, lda, B, ldb, ea, M, N, K, splits, st);
    case EPI_FIELD: return splits == 1 ? launch_simt_t<EPI_FIELD>(A, lda, B, ldb, ea, M, N, K, 1, st)
                                       : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

scw_status make_map_bf16(CUtensorMap* m, const void* base, long long cols, long long rows, long long pitch,
                         int box_rows, int box_cols) {
  auto fn = encode_fn();
  if (!fn) return set_error(SCW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  if ((reinterpret_cast<uintptr_t>(base) & 15u) || (pitch * 2) % 16 || box_rows < 1 || box_rows > 256 ||
      (box_cols != 64 && box_cols != 32))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "tensor map: base, pitch or box out of range");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SCW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return SCW_OK;
}

scw_status make_map_act3d(CUtensorMap* m, const void* base, long long P, long long samples) {
  auto fn = encode_fn();
  if (!fn) return set_error(SCW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  if ((reinterpret_cast<uintptr_t>(base) & 15u) || P < 128 || P % 128 != 0 || samples < 1)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "tensor map: base or extent out of range");
  cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)C, (cuuint64_t)samples};
  cuuint64_t strides[2] = {(cuuint64_t)(P * 2), (cuuint64_t)(P * C * 2)};
  cuuint32_t box[3] = {64u, (cuuint32_t)C, (cuuint32_t)kSeg2Samples};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SCW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return SCW_OK;
}

}  // namespace fno
}  // namespace scw
