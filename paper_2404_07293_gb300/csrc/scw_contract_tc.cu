// Step (b) on the 5th-generation tensor cores: the per-layer mode contraction
//   S_l = W_l C_l,   W_l in C^{3M x 4M},  C_l[j][f] = c_j(z_f)          (Eq. 34, Sec. 4.1)
// written as one real GEMM. A = W viewed as interleaved reals (3M x 8M: the
// complex64 memory layout itself), B = [[Re C, Im C], [-Im C, Re C]] in the
// same interleaving (8M x NB, NB = 2 F_pad), D = [Re S | Im S] (3M x NB).
//
// Precision modes:
//   split-BF16: A = A_hi + A_lo, B = B_hi + B_lo (BF16 each); the three products
//               A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate in one FP32 TMEM tile.
//   FP16:       A in FP16, B = B_hi + B_lo (FP16); two products.
//
// Persistent, warp-specialised kernel. Work is a list of tasks (item, unit,
// 128-row tile, K split), grouped per CTA on the host longest-first; every role
// walks the same list:
//   warp 0 lane 0   producer: contiguous cp.async.bulk copies (no multicast) of
//                   the pre-swizzled tile-major A tiles (L2 evict-first: W is
//                   streamed once) and B chunks (evict-last: re-read by every row
//                   tile) into a ring of shared-memory stages (full/empty mbarriers)
//   warp 1 lane 0   tcgen05.mma issuer (M = 128, N = NB, K = 16 per instruction)
//                   into one of two TMEM accumulators (acc_full/acc_empty)
//   warps 2-5       epilogue: tcgen05.ld 32 lanes x 8 columns of the other
//                   accumulator, coalesced stores of S_part[split][plane][row]
// so loads, MMAs and the previous task's epilogue overlap. Every wait is bounded
// by a %globaltimer deadline; a timeout sets the error word and all roles stop.
#include "scw_internal.cuh"
#include "scw_ptx.cuh"

namespace scw {

template <int NB, bool SPLIT>
struct TcCfg {
  static constexpr uint32_t A_BYTES = 128u * 64u * 2u;
  static constexpr uint32_t B_BYTES = (uint32_t)NB * 64u * 2u;
  static constexpr int NA = SPLIT ? 2 : 1;
  static constexpr uint32_t STAGE_BYTES = NA * A_BYTES + 2 * B_BYTES;
  // two CTAs per SM while at least three stages fit in ~110 KB, else one CTA with up to ~220 KB
  static constexpr int STAGES_2 = (int)(110u * 1024u / STAGE_BYTES);
  static constexpr int CTAS_PER_SM = STAGES_2 >= 3 ? 2 : 1;
  static constexpr int STAGES_RAW = CTAS_PER_SM == 2 ? STAGES_2 : (int)(220u * 1024u / STAGE_BYTES);
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr uint32_t SMEM = STAGES * STAGE_BYTES + 1024u;
  static constexpr uint32_t ACC_COLS = NB <= 32 ? 32u : (NB <= 64 ? 64u : (NB <= 128 ? 128u : 256u));
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
};

struct TaskGeom {
  int kb, kcount, layer, unit, tile, split, f0, nf, rt;
};

__device__ __forceinline__ TaskGeom task_geom(const int4 tk, const ItemDev& it) {
  TaskGeom g;
  const LayerUnit u = it.units[tk.y];
  const int ks = u.ks > 0 ? u.ks : it.k_split;
  const int per = (it.nk + ks - 1) / ks;
  g.kb = tk.w * per;
  g.kcount = max(0, min(it.nk, g.kb + per) - g.kb);
  g.layer = u.layer;
  g.unit = tk.y;
  g.tile = tk.z;
  g.split = tk.w;
  g.f0 = u.f0;
  g.nf = u.nf;
  g.rt = min(it.rows_tile, 3 * it.M - it.rows_tile * tk.z);  // rows of this tile that exist
  return g;
}

template <int NB, bool SPLIT, bool BATCH>
__global__ void __launch_bounds__(192) contract_tc_kernel(const __grid_constant__ ItemDev one,
                                                          const ItemDev* __restrict__ items,
                                                          const int4* __restrict__ tasks,
                                                          const int* __restrict__ cta_off, int* err,
                                                          uint64_t timeout_ns, int inject_stall) {
  using Cfg = TcCfg<NB, SPLIT>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr int FP = NB / 2;  // plane slots
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t_begin = cta_off[blockIdx.x], t_end = cta_off[blockIdx.x + 1];
  const uint64_t deadline = ptx::globaltimer() + timeout_ns;
  ptx::griddep_launch_dependents();  // the x-pass may be scheduled as CTAs of this grid finish
  trace_begin(one.trace, TRACE_CONTRACT);

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(ptx::smem_u32(&accf_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&acce_bar[i]), 4);  // one arrival per epilogue warp
    }
    ptx::mbar_init(ptx::smem_u32(&drain_bar), 1);
    abort_s = 0;
    ptx::fence_mbar_init();
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
    // ---------------- bulk-copy producer ----------------
    const uint64_t pol_a = ptx::policy_evict_first(), pol_b = ptx::policy_evict_last();
    int st = 0;
    uint32_t ph = 0;
    int issued = 0, skipped = -1;
    // W does not depend on the phase kernel that precedes this grid (programmatic launch): the first
    // ring of stages gets its A copies at once, their B copies follow once that kernel has finished
    bool dep_done = false;
    int npend = 0;
    uint32_t pend_sb[STAGES], pend_fb[STAGES];
    const uint16_t* pend_bh[STAGES];
    const uint16_t* pend_bl[STAGES];
    auto flush_pending = [&]() {
      ptx::griddep_wait();
      for (int q = 0; q < npend; ++q) {
        ptx::bulk_load(pend_sb[q], pend_bh[q], Cfg::B_BYTES, pend_fb[q], pol_b);
        ptx::bulk_load(pend_sb[q] + Cfg::B_BYTES, pend_bl[q], Cfg::B_BYTES, pend_fb[q], pol_b);
      }
      npend = 0;
      dep_done = true;
    };
    for (int t = t_begin; t < t_end && !abort_s; ++t) {
      const int4 tk = tasks[t];
      const ItemDev& it = BATCH ? items[tk.x] : one;
      const TaskGeom g = task_geom(tk, it);
      const int R = 3 * it.M;
      // element offsets of this tile's first chunk in A and of the unit's first chunk in B
      const size_t a0 = (size_t)g.layer * R * it.nk * 64 + (size_t)g.tile * it.rows_tile * it.nk * 64;
      const size_t b0 = (size_t)g.unit * it.nk * NB * 64;
      const uint32_t a_bytes = (uint32_t)g.rt * 128u;
      const uint32_t tx = Cfg::NA * a_bytes + 2u * Cfg::B_BYTES;
      const uint16_t* Ah = static_cast<const uint16_t*>(it.Ahi);
      const uint16_t* Al = static_cast<const uint16_t*>(it.Alo);
      const uint16_t* Bh = static_cast<const uint16_t*>(it.Bhi);
      const uint16_t* Bl = static_cast<const uint16_t*>(it.Blo);
      for (int i = 0; i < g.kcount; ++i) {
        if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[st]), ph ^ 1u, deadline)) {
          atomicOr(err, DEV_ERR_TIMEOUT_EMPTY);
          abort_s = 1;
          break;
        }
        const uint32_t fb = ptx::smem_u32(&full_bar[st]);
        if (inject_stall && blockIdx.x == 0 && issued == 0) {
          skipped = 0;  // failure injection (scw_plan_inject_stall): this stage is never filled
        } else {
          ptx::mbar_arrive_expect_tx(fb, tx);
          const int kc = g.kb + i;
          const uint32_t sa = ptx::smem_u32(smem + (size_t)st * Cfg::STAGE_BYTES);
          const size_t ao = a0 + (size_t)kc * g.rt * 64;
          ptx::bulk_load(sa, Ah + ao, a_bytes, fb, pol_a);
          if (SPLIT) ptx::bulk_load(sa + Cfg::A_BYTES, Al + ao, a_bytes, fb, pol_a);
          const uint32_t sb = sa + Cfg::NA * Cfg::A_BYTES;
          const size_t bo = b0 + (size_t)kc * NB * 64;
          if (dep_done) {
            ptx::bulk_load(sb, Bh + bo, Cfg::B_BYTES, fb, pol_b);
            ptx::bulk_load(sb + Cfg::B_BYTES, Bl + bo, Cfg::B_BYTES, fb, pol_b);
          } else {
            pend_sb[npend] = sb;
            pend_fb[npend] = fb;
            pend_bh[npend] = Bh + bo;
            pend_bl[npend] = Bl + bo;
            if (++npend == STAGES) flush_pending();
          }
        }
        ++issued;
        if (++st == STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    if (!dep_done) flush_pending();  // fewer stages than the ring, or an early stop
    if (abort_s) {
      // let the last issued copies land before the CTA's shared memory goes away
      const uint64_t d2 = ptx::drain_deadline(timeout_ns);
      for (int back = 1; back <= STAGES && back <= issued; ++back) {
        const int i = issued - back;
        if (i == skipped) continue;  // nothing was sent to that stage
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[i % STAGES]), (uint32_t)(i / STAGES) & 1u, d2)) {
          atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
          break;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- tcgen05.mma issuer ----------------
    constexpr uint32_t idesc = ptx::idesc_f16(SPLIT, 128, NB);
    int st = 0;
    uint32_t ph = 0;
    int lt = 0;
    for (int t = t_begin; t < t_end && !abort_s; ++t, ++lt) {
      const int4 tk = tasks[t];
      const ItemDev& it = BATCH ? items[tk.x] : one;
      const TaskGeom g = task_geom(tk, it);
      const int acc = lt & 1;
      if (!ptx::mbar_wait(ptx::smem_u32(&acce_bar[acc]), ((uint32_t)(lt >> 1) & 1u) ^ 1u, deadline)) {
        atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t d_tmem = tmem + (uint32_t)acc * Cfg::ACC_COLS;
      for (int i = 0; i < g.kcount; ++i) {
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[st]), ph, deadline)) {
          atomicOr(err, DEV_ERR_TIMEOUT_FULL);
          abort_s = 1;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t a_hi = ptx::smem_u32(smem + (size_t)st * Cfg::STAGE_BYTES);
        const uint32_t a_lo = a_hi + Cfg::A_BYTES;
        const uint32_t b_hi = a_hi + Cfg::NA * Cfg::A_BYTES;
        const uint32_t b_lo = b_hi + Cfg::B_BYTES;
        const uint64_t dah = ptx::sw128_desc(a_hi), dal = ptx::sw128_desc(a_lo);
        const uint64_t dbh = ptx::sw128_desc(b_hi), dbl = ptx::sw128_desc(b_lo);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          // K advance of 16 elements = 32 bytes inside the 128-byte swizzle row
          const uint64_t o = (uint64_t)(2 * kk);
          ptx::mma_f16(d_tmem, dah + o, dbh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          ptx::mma_f16(d_tmem, dah + o, dbl + o, idesc, 1u);
          if (SPLIT) ptx::mma_f16(d_tmem, dal + o, dbh + o, idesc, 1u);
        }
        ptx::mma_commit(ptx::smem_u32(&empty_bar[st]));
        if (++st == STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
      ptx::mma_commit(ptx::smem_u32(&accf_bar[acc]));
    }
    if (abort_s) {
      // issued MMAs must finish before the tensor memory is released
      ptx::mma_commit(ptx::smem_u32(&drain_bar));
      if (!ptx::mbar_wait(ptx::smem_u32(&drain_bar), 0u, ptx::drain_deadline(timeout_ns)))
        atomicOr(err, DEV_ERR_TIMEOUT_DRAIN);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int grp = warp & 3;  // TMEM lanes 32*grp .. 32*grp+31
    // partial spectra are read back right after this kernel: keep them in L2 while W streams through
    const uint64_t pol_s = ptx::policy_evict_last();
    int lt = 0;
    for (int t = t_begin; t < t_end && !abort_s; ++t, ++lt) {
      const int4 tk = tasks[t];
      const ItemDev& it = BATCH ? items[tk.x] : one;
      const TaskGeom g = task_geom(tk, it);
      const int acc = lt & 1;
      const bool ok = ptx::mbar_wait(ptx::smem_u32(&accf_bar[acc]), (uint32_t)(lt >> 1) & 1u, deadline);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT_ACCUM);
        abort_s = 1;
        break;
      }
      ptx::tc_fence_after();
      const int rows = 3 * it.M;
      const int rl = grp * 32 + lane;  // row within the tile
      const int row = g.tile * it.rows_tile + rl;
      float2* dst = it.S_part + ((size_t)g.split * it.Fz + g.f0) * rows;
      const uint32_t lane_addr = tmem + (uint32_t)acc * Cfg::ACC_COLS + ((uint32_t)(grp * 32) << 16);
#pragma unroll 1
      for (int f0 = 0; f0 < FP; f0 += 8) {
        uint32_t re[8], im[8];
        if (g.kcount > 0) {
          ptx::tmem_ld_x8(lane_addr + (uint32_t)f0, re);
          ptx::tmem_ld_x8(lane_addr + (uint32_t)(FP + f0), im);
          ptx::tmem_wait_ld();
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) re[q] = im[q] = 0u;
        }
        if (rl < g.rt) {
          const size_t d0 = ((size_t)g.split * it.Fz + g.f0) * rows + row;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (f0 + q < g.nf && in_bounds(it, BND_S_PART, d0 + (size_t)(f0 + q) * rows))
              ptx::st_global_hint(dst + (size_t)(f0 + q) * rows + row,
                                  make_float2(__uint_as_float(re[q]), __uint_as_float(im[q])), pol_s);
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
  trace_end(one.trace, TRACE_CONTRACT);
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- host side ---
template <int NB, bool SPLIT>
static cudaError_t launch_tc_t(const ItemDev& one, const ItemDev* items, const TcSchedule& s, int* err,
                               uint64_t timeout_ns, int inject, cudaStream_t st) {
  using Cfg = TcCfg<NB, SPLIT>;
  cudaError_t e;
  if (items) {
    e = allow_max_smem(reinterpret_cast<const void*>(contract_tc_kernel<NB, SPLIT, true>));
    if (e != cudaSuccess) return e;
    e = launch_pdl(contract_tc_kernel<NB, SPLIT, true>, dim3(s.grid), dim3(192), Cfg::SMEM, st, one, items,
                   (const int4*)s.d_tasks, (const int*)s.d_cta_off, err, timeout_ns, inject);
  } else {
    e = allow_max_smem(reinterpret_cast<const void*>(contract_tc_kernel<NB, SPLIT, false>));
    if (e != cudaSuccess) return e;
    e = launch_pdl(contract_tc_kernel<NB, SPLIT, false>, dim3(s.grid), dim3(192), Cfg::SMEM, st, one,
                   (const ItemDev*)nullptr, (const int4*)s.d_tasks, (const int*)s.d_cta_off, err, timeout_ns, inject);
  }
  return e;
}

template <bool SPLIT>
static cudaError_t launch_tc_nb(int NB, const ItemDev& one, const ItemDev* items, const TcSchedule& s, int* err,
                                uint64_t timeout_ns, int inject, cudaStream_t st) {
  switch (NB) {
    case 16: return launch_tc_t<16, SPLIT>(one, items, s, err, timeout_ns, inject, st);
    case 32: return launch_tc_t<32, SPLIT>(one, items, s, err, timeout_ns, inject, st);
    case 48: return launch_tc_t<48, SPLIT>(one, items, s, err, timeout_ns, inject, st);
    case 64: return launch_tc_t<64, SPLIT>(one, items, s, err, timeout_ns, inject, st);
    case 128: return launch_tc_t<128, SPLIT>(one, items, s, err, timeout_ns, inject, st);
    case 256: return launch_tc_t<256, SPLIT>(one, items, s, err, timeout_ns, inject, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_contract_tc(const ItemDev& one, const ItemDev* items, const TcSchedule& s, int NB, bool bf16,
                               int* err, uint64_t timeout_ns, int inject, cudaStream_t st) {
  if (s.n_tasks == 0 || s.grid == 0) return cudaSuccess;
  return bf16 ? launch_tc_nb<true>(NB, one, items, s, err, timeout_ns, inject, st)
              : launch_tc_nb<false>(NB, one, items, s, err, timeout_ns, inject, st);
}

int tc_ctas_per_sm(int NB, bool bf16) {
  switch (NB) {
    case 16: return bf16 ? TcCfg<16, true>::CTAS_PER_SM : TcCfg<16, false>::CTAS_PER_SM;
    case 32: return bf16 ? TcCfg<32, true>::CTAS_PER_SM : TcCfg<32, false>::CTAS_PER_SM;
    case 48: return bf16 ? TcCfg<48, true>::CTAS_PER_SM : TcCfg<48, false>::CTAS_PER_SM;
    case 64: return bf16 ? TcCfg<64, true>::CTAS_PER_SM : TcCfg<64, false>::CTAS_PER_SM;
    case 128: return bf16 ? TcCfg<128, true>::CTAS_PER_SM : TcCfg<128, false>::CTAS_PER_SM;
    default: return 1;
  }
}

}  // namespace scw
