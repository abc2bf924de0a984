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
// One CTA = 4 warps per work unit (active layer, 128-row tile, K split):
//   warp 0 lane 0   TMA producer (3D tensor maps, 128-byte swizzle, no multicast)
//   warp 1 lane 0   tcgen05.mma issuer (M = 128, N = NB, K = 16 per instruction)
//   all 4 warps     epilogue: tcgen05.ld 32 lanes x 8 columns, coalesced stores
//                   of the partial spectrum S_part[split][plane][row].
// Shared-memory stages are recycled through full/empty mbarriers; every wait is
// bounded by a %globaltimer deadline and reports through the error word.
#include <cudaTypedefs.h>

#include "scw_internal.cuh"
#include "scw_ptx.cuh"

namespace scw {

struct TcArgs {
  const LayerUnit* units;
  int n_tiles;   // ceil(3M / 128)
  int ksplit;
  int nk;        // K stages of 64 reals: ceil(8M / 64)
  int rows;      // 3M
  int Fz;
  int F_pad;
  float2* S_part;
  int* err;
  uint64_t timeout_ns;
};

template <int NB, bool SPLIT>
struct TcCfg {
  static constexpr uint32_t A_BYTES = 128u * 64u * 2u;
  static constexpr uint32_t B_BYTES = (uint32_t)NB * 64u * 2u;
  static constexpr int NA = SPLIT ? 2 : 1;
  static constexpr uint32_t STAGE_BYTES = NA * A_BYTES + 2 * B_BYTES;
  // two CTAs per SM while at least two stages fit in ~110 KB, else one CTA with up to ~220 KB
  static constexpr int STAGES_2 = (int)(110u * 1024u / STAGE_BYTES);
  static constexpr int STAGES = STAGES_2 >= 2 ? (STAGES_2 > 8 ? 8 : STAGES_2)
                                              : (int)(220u * 1024u / STAGE_BYTES);
  static constexpr uint32_t SMEM = STAGES * STAGE_BYTES + 1024u;
  static constexpr uint32_t TMEM_COLS = NB <= 32 ? 32u : (NB <= 64 ? 64u : (NB <= 128 ? 128u : 256u));
};

template <int NB, bool SPLIT>
__global__ void __launch_bounds__(128) contract_tc_kernel(const __grid_constant__ CUtensorMap tmAhi,
                                                          const __grid_constant__ CUtensorMap tmAlo,
                                                          const __grid_constant__ CUtensorMap tmBhi,
                                                          const __grid_constant__ CUtensorMap tmBlo, TcArgs args) {
  using Cfg = TcCfg<NB, SPLIT>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ int issued_s, consumed_s;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int split = blockIdx.x % args.ksplit;
  const int rest = blockIdx.x / args.ksplit;
  const int tile = rest % args.n_tiles;
  const int ui = rest / args.n_tiles;
  const LayerUnit u = args.units[ui];
  const int per = (args.nk + args.ksplit - 1) / args.ksplit;
  const int kb = split * per;
  const int kcount = max(0, min(args.nk, kb + per) - kb);
  const uint64_t deadline = ptx::globaltimer() + args.timeout_ns;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[i]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(&acc_bar), 1);
    abort_s = 0;
    issued_s = 0;
    consumed_s = 0;
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

  if (kcount > 0 && warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    ptx::prefetch_tensormap(&tmAhi);
    if (SPLIT) ptx::prefetch_tensormap(&tmAlo);
    ptx::prefetch_tensormap(&tmBhi);
    ptx::prefetch_tensormap(&tmBlo);
    int i = 0;
    for (; i < kcount; ++i) {
      const int st = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[st]), ph ^ 1u, deadline)) {
        atomicOr(args.err, DEV_ERR_TIMEOUT_EMPTY);
        abort_s = 1;
        break;
      }
      if (abort_s) break;
      const uint32_t fb = ptx::smem_u32(&full_bar[st]);
      ptx::mbar_arrive_expect_tx(fb, Cfg::STAGE_BYTES);
      const int k0 = (kb + i) * 64;
      const uint32_t sa = ptx::smem_u32(smem + (size_t)st * Cfg::STAGE_BYTES);
      ptx::tma_load_3d(sa, &tmAhi, k0, tile * 128, u.layer, fb);
      if (SPLIT) ptx::tma_load_3d(sa + Cfg::A_BYTES, &tmAlo, k0, tile * 128, u.layer, fb);
      const uint32_t sb = sa + Cfg::NA * Cfg::A_BYTES;
      ptx::tma_load_3d(sb, &tmBhi, k0, 0, ui, fb);
      ptx::tma_load_3d(sb + Cfg::B_BYTES, &tmBlo, k0, 0, ui, fb);
    }
    issued_s = i;
  } else if (kcount > 0 && warp == 1 && lane == 0) {
    // ---------------- tcgen05.mma issuer ----------------
    constexpr uint32_t idesc = ptx::idesc_f16(SPLIT, 128, NB);
    int i = 0;
    for (; i < kcount; ++i) {
      const int st = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[st]), ph, deadline)) {
        atomicOr(args.err, DEV_ERR_TIMEOUT_FULL);
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
        ptx::mma_f16(tmem, dah + o, dbh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        ptx::mma_f16(tmem, dah + o, dbl + o, idesc, 1u);
        if (SPLIT) ptx::mma_f16(tmem, dal + o, dbh + o, idesc, 1u);
      }
      ptx::mma_commit(ptx::smem_u32(&empty_bar[st]));
    }
    consumed_s = i;
    ptx::mma_commit(ptx::smem_u32(&acc_bar));  // always arrives, even after an abort
  }
  __syncwarp();

  // ---------------- epilogue ----------------
  bool ok = true;
  if (kcount > 0) {
    ok = ptx::mbar_wait(ptx::smem_u32(&acc_bar), 0u, deadline);
    if (!ok) atomicOr(args.err, DEV_ERR_TIMEOUT_ACCUM);
  }
  const int all_ok = __syncthreads_and(ok ? 1 : 0);
  ptx::tc_fence_after();
  const bool have_acc = (kcount > 0) && all_ok && !abort_s;
  const int row = tile * 128 + warp * 32 + lane;
  float2* dst = args.S_part + ((size_t)split * args.Fz + u.f0) * args.rows;
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  for (int f0 = 0; f0 < args.F_pad; f0 += 8) {
    uint32_t re[8], im[8];
    if (have_acc) {
      ptx::tmem_ld_x8(lane_addr + (uint32_t)f0, re);
      ptx::tmem_ld_x8(lane_addr + (uint32_t)(args.F_pad + f0), im);
      ptx::tmem_wait_ld();
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) re[q] = im[q] = 0u;
    }
    if (row < args.rows) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (f0 + q < u.nf)
          dst[(size_t)(f0 + q) * args.rows + row] = make_float2(__uint_as_float(re[q]), __uint_as_float(im[q]));
    }
  }

  // ---------------- teardown ----------------
  ptx::tc_fence_before();
  __syncthreads();
  if (abort_s && threadIdx.x == 0) {
    // let copies that were issued but never consumed land before the CTA exits
    const uint64_t d2 = ptx::globaltimer() + args.timeout_ns;
    for (int i = consumed_s; i < issued_s; ++i)
      if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[i % STAGES]), (uint32_t)(i / STAGES) & 1u, d2)) {
        atomicOr(args.err, DEV_ERR_TIMEOUT_DRAIN);
        break;
      }
  }
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- host side ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static bool encode_3d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t d0, uint64_t d1,
                      uint64_t d2, uint32_t b0, uint32_t b1, std::string& why) {
  auto fn = encode_fn();
  if (!fn) {
    why = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};  // 16-bit elements
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    why = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

bool encode_tensor_maps(Plan& p, std::string& why) {
  const uint64_t K8 = 8ull * p.M, R = 3ull * p.M;
  const bool bf = p.precision == SCW_PREC_SPLIT_BF16;
  const CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const void* a_hi = bf ? static_cast<const void*>(p.Whi) : static_cast<const void*>(p.Wh);
  const void* a_lo = bf ? static_cast<const void*>(p.Wlo) : static_cast<const void*>(p.Wh);
  if (!encode_3d(&p.tmA_hi, dt, a_hi, K8, R, p.L, 64, 128, why)) return false;
  if (!encode_3d(&p.tmA_lo, dt, a_lo, K8, R, p.L, 64, 128, why)) return false;
  const uint64_t nu = p.units.size();
  if (!encode_3d(&p.tmB_hi, dt, p.Bhi, K8, p.NB, nu, 64, p.NB, why)) return false;
  if (!encode_3d(&p.tmB_lo, dt, p.Blo, K8, p.NB, nu, 64, p.NB, why)) return false;
  return true;
}

template <int NB, bool SPLIT>
static cudaError_t launch_tc_t(const Plan& p, cudaStream_t st) {
  using Cfg = TcCfg<NB, SPLIT>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<NB, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcArgs a;
  a.units = p.d_units;
  a.n_tiles = (3 * p.M + 127) / 128;
  a.ksplit = p.k_split;
  a.nk = (8 * p.M + 63) / 64;
  a.rows = 3 * p.M;
  a.Fz = p.Fz;
  a.F_pad = p.F_pad;
  a.S_part = p.S_part;
  a.err = p.d_err;
  a.timeout_ns = p.timeout_ns;
  const unsigned grid = (unsigned)(p.units.size() * a.n_tiles * a.ksplit);
  contract_tc_kernel<NB, SPLIT><<<grid, 128, Cfg::SMEM, st>>>(p.tmA_hi, p.tmA_lo, p.tmB_hi, p.tmB_lo, a);
  return cudaGetLastError();
}

template <bool SPLIT>
static cudaError_t launch_tc_nb(const Plan& p, cudaStream_t st) {
  switch (p.NB) {
    case 16: return launch_tc_t<16, SPLIT>(p, st);
    case 32: return launch_tc_t<32, SPLIT>(p, st);
    case 48: return launch_tc_t<48, SPLIT>(p, st);
    case 64: return launch_tc_t<64, SPLIT>(p, st);
    case 128: return launch_tc_t<128, SPLIT>(p, st);
    case 256: return launch_tc_t<256, SPLIT>(p, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_contract_tc(const Plan& p, cudaStream_t st) {
  if (p.units.empty()) return cudaSuccess;
  return p.precision == SCW_PREC_SPLIT_BF16 ? launch_tc_nb<true>(p, st) : launch_tc_nb<false>(p, st);
}

}  // namespace scw
