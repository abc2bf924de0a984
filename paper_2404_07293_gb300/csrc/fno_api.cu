// Host side of the surrogate: workspace ownership, parameter initialisation,
// the launch sequences of forward / backward / Adam / inference, and the
// split-conformal calibration of the error head. See include/scw_fno.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/scw_fno.h"
#include "fno_internal.cuh"

using namespace scw;
using namespace scw::fno;

struct scw_fno_s {
  scw_fno_desc d{};
  bool bf16 = true;
  int N = 0, P = 0, m = 0, Kc = 0, Kp = 0, L = 0, S = 0, in_grid = 0, Bmax = 0, nblk = 0;
  size_t esz = 2;  // bytes per activation / weight-copy element

  // flat parameter offsets (elements)
  long long n_params = 0, off_P = 0, off_R[8] = {}, off_W[8] = {}, off_c[8] = {}, off_Q = 0, off_e = 0;

  float* master = nullptr;  // FP32 parameters
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  void* wcopy = nullptr;    // T copy read by the kernels
  int step = 0;
  float q_cal = 0.f;

  void* D = nullptr;        // [Kc][P]
  void* E = nullptr;        // [P][Kp]
  void* Vcf[9] = {};        // [Bmax][C][P]
  void* Vcl[9] = {};        // [Bmax][P][C]
  void* Gcl[8] = {};        // GELU'(Z_l) [Bmax][P][C], stored by the training forward
  float* Vh[8] = {};        // complex [kMaxSplit][Kc/2][Bmax C] (mode-major)
  float* GWh = nullptr;     // same shape as one Vh
  void* WT = nullptr;       // [L][C][C]: W_l transposed (tensor-core operand of the backward 1x1)
  void* Wh = nullptr;       // [Bmax C][Kp]
  void* GVh = nullptr;
  void* dZcf[2] = {};
  void* dZcl[2] = {};
  float* part_tn = nullptr, *part_err = nullptr, *part_pool = nullptr, *part_proj = nullptr;
  float* part_lift = nullptr, *part_head = nullptr, *scratch = nullptr;
  float* part_mix[8] = {};  // per layer: the gradient partials are reduced together after the backward pass
  float* part_dw[8] = {};
  size_t scratch_floats = 0;
  // the backward pass's partial-sum reductions, all run by two launches at its end (per batch size)
  RedSeg* d_segs = nullptr;
  int segs_B = -1, nseg = 0, seg_items1 = 0, seg_items2 = 0;
  float* loss_d = nullptr, *h_d = nullptr, *rel2_d = nullptr;
  int* d_err = nullptr;
  uint64_t timeout_ns = 2000000000ull;

  CUtensorMap map_Vcf[9], map_dZcf[2], map_D, map_E, map_Wh, map_GVh;
  // 1x1-convolution operands: channel-first activations read MN-major (3D maps), W and W^T
  CUtensorMap map_Vx[8], map_dZx[2], map_W[8], map_WT[8];

  std::vector<void*> allocs;
  size_t bytes = 0;
  int launches_train = 0, launches_infer = 0;
  int counter = 0;  // launches of the current call

  // per-kernel timing (scw_surrogate_enable_timing): one event after every launch
  bool timing = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> cats;
  std::vector<double> flops;
  cudaStream_t tstream = nullptr;
  double acc_ms[5] = {}, acc_flops[5] = {};
  int timed_calls = 0;
};

enum { CAT_DFT = 0, CAT_LAYER = 1, CAT_DW = 2, CAT_MIX = 3, CAT_OTHER = 4 };

static constexpr int kMaxSplit = 8;

static cudaError_t falloc(scw_fno_s* f, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    f->allocs.push_back(*p);
    f->bytes += bytes;
  }
  return e;
}

static void free_all(scw_fno_s* f) {
  for (void* p : f->allocs) cudaFree(p);
  f->allocs.clear();
  if (f->d_segs) cudaFree(f->d_segs);
  f->d_segs = nullptr;
  f->segs_B = -1;
  for (cudaEvent_t ev : f->events) cudaEventDestroy(ev);
  f->events.clear();
}

// splitmix64 (Steele, Lea and Flood 2014): counter-based uniform draws
static double uniform_pm1(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

static int dft_splits(const scw_fno_s* f, int B, int BN) {
  if (f->bf16 && BN == 256) return 1;  // the persistent GEMM form: deep pipeline, no K splits
  const int tiles = ((B * C + 127) / 128) * ((f->Kc + BN - 1) / BN);
  int ks = std::max(1, (2 * 152) / std::max(1, tiles));
  ks = std::min(ks, kMaxSplit);
  ks = std::min(ks, std::max(1, f->P / 64 / 4));  // at least 4 K blocks per split
  return ks;
}

static int dw_splits(const scw_fno_s* f, int B) {
  const int groups = (B + 3) / 4;
  int ks = std::max(1, (2 * 152) / std::max(1, groups));
  ks = std::min(ks, kMaxSplit);
  ks = std::min(ks, std::max(1, f->P / 64 / 4));
  return ks;
}

static int dft_bn(const scw_fno_s* f) { return f->Kc >= 256 ? 256 : (f->Kc >= 128 ? 128 : (f->Kc >= 64 ? 64 : 32)); }

// record timing event i (created on first use)
static cudaError_t mark(scw_fno_s* f, size_t i) {
  while (i >= f->events.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    f->events.push_back(ev);
  }
  return cudaEventRecord(f->events[i], f->tstream);
}

static scw_status launch_ok(scw_fno_s* f, cudaError_t e, const char* what, int cat = CAT_OTHER, double flops = 0) {
  if (e != cudaSuccess) return cuda_error(e, what);
  ++f->counter;
  if (f->timing) {
    f->cats.push_back(cat);
    f->flops.push_back(flops);
    e = mark(f, f->cats.size());
    if (e != cudaSuccess) return cuda_error(e, "timing event");
  }
  return SCW_OK;
}

static scw_status begin_call(scw_fno_s* f, cudaStream_t st) {
  f->counter = 0;
  if (!f->timing) return SCW_OK;
  f->tstream = st;
  f->cats.clear();
  f->flops.clear();
  // event 0 marks the start; timed launch i ends at event i + 1
  cudaError_t e = mark(f, 0);
  if (e != cudaSuccess) return cuda_error(e, "timing event");
  return SCW_OK;
}

static scw_status end_call(scw_fno_s* f) {
  if (!f->timing) return SCW_OK;
  cudaError_t e = cudaEventSynchronize(f->events[f->cats.size()]);
  if (e != cudaSuccess) return cuda_error(e, "timing sync");
  for (size_t i = 0; i < f->cats.size(); ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, f->events[i], f->events[i + 1]);
    if (e != cudaSuccess) return cuda_error(e, "timing read");
    f->acc_ms[f->cats[i]] += ms;
    f->acc_flops[f->cats[i]] += f->flops[i];
  }
  ++f->timed_calls;
  return SCW_OK;
}

#define FNO_TRY(expr)              \
  do {                             \
    scw_status s_ = (expr);        \
    if (s_ != SCW_OK) return s_;   \
  } while (0)

template <typename T>
static T* at(void* base, long long off) {
  return static_cast<T*>(base) + off;
}

// W^T copies for the backward 1x1 convolution on the tensor cores (BF16 mode)
static cudaError_t refresh_wt(scw_fno_s* f, cudaStream_t st) {
  if (!f->bf16) return cudaSuccess;
  const long long stride = f->L > 1 ? f->off_W[1] - f->off_W[0] : 0;
  return launch_transpose_w<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(f->wcopy), f->off_W[0], stride,
                                           static_cast<__nv_bfloat16*>(f->WT), f->L, st);
}

// ---------------------------------------------------------------- forward ---
template <typename T>
static scw_status forward(scw_fno_s* f, const float2* n, int B, bool keep_z, cudaStream_t st) {
  const int BC = B * C;
  // BF16 mode reads the layer inputs channel-first only; the FP32 (SIMT) mode also reads them
  // channel-last
  FNO_TRY(launch_ok(f, launch_lift<T>(n, at<T>(f->wcopy, f->off_P), static_cast<T*>(f->Vcf[0]),
                                      f->bf16 ? nullptr : static_cast<T*>(f->Vcl[0]), B, f->S, f->in_grid, f->N,
                                      st),
                    "lift"));
  const long long ld = (long long)f->Bmax * C;                // complex elements per mode
  const long long vstride = ld * (f->Kc / 2);                 // complex elements per split
  const float inv_n2 = 1.f / ((float)f->N * (float)f->N);
  for (int l = 0; l < f->L; ++l) {
    const int bn = dft_bn(f);
    const int ks = dft_splits(f, B, bn);
    EpiArgs ea{};
    ea.alpha = 1.f;
    ea.rows = BC;
    ea.cols = f->Kc;
    ea.out = f->Vh[l];
    ea.ld = ld;
    ea.split_stride = vstride;
    cudaError_t e = f->bf16 ? launch_gemm_tc(EPI_MODES, bn, f->map_Vcf[l], f->map_D, f->map_D, f->map_D, ea, BC,
                                             f->Kc, f->P, ks, f->d_err, f->timeout_ns, st)
                            : launch_gemm_simt(EPI_MODES, static_cast<const float*>(f->Vcf[l]), f->P,
                                               static_cast<const float*>(f->D), f->P, ea, BC, f->Kc, f->P, ks, st);
    FNO_TRY(launch_ok(f, e, "truncated DFT", CAT_DFT, 2.0 * BC * f->Kc * f->P));
    // Wh carries the inverse transform's 1/N^2 so that the 1x1 convolution can share its accumulator
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
      e = launch_mix_tc(false, reinterpret_cast<const float2*>(f->Vh[l]), ks, vstride, ld, at<T>(f->wcopy, f->off_R[l]),
                        static_cast<T*>(f->Wh), inv_n2, B, f->m, f->Kp, f->d_err, f->timeout_ns, st);
    else
      e = launch_mix_fwd<T>(reinterpret_cast<const float2*>(f->Vh[l]), ks, vstride, ld, at<T>(f->wcopy, f->off_R[l]),
                            static_cast<T*>(f->Wh), inv_n2, B, f->m, f->Kp, st);
    FNO_TRY(launch_ok(f, e, "mode mixing", CAT_MIX, 8.0 * f->m * f->m * C * C * B));
    EpiArgs eb{};
    eb.alpha = 1.f;
    eb.rows = f->P;
    eb.cols = BC;
    eb.P = f->P;
    eb.B = B;
    eb.w = at<T>(f->wcopy, f->off_W[l]);
    eb.bias = at<T>(f->wcopy, f->off_c[l]);
    eb.x_cl = f->Vcl[l];
    eb.g_out = (keep_z && l < f->L - 1) ? f->Gcl[l] : nullptr;
    // V_L feeds the projection (channel-last) only; the others feed the next layer and the
    // weight gradients (channel-first)
    eb.out_cf = l < f->L - 1 ? f->Vcf[l + 1] : nullptr;
    eb.out_cl = (!f->bf16 || l == f->L - 1) ? f->Vcl[l + 1] : nullptr;
    eb.gelu = l < f->L - 1 ? 1 : 0;
    e = f->bf16 ? launch_gemm_tc(EPI_LAYER_FWD, 256, f->map_E, f->map_Wh, f->map_Vx[l], f->map_W[l], eb, f->P, BC,
                                 f->Kp, 1, f->d_err, f->timeout_ns, st)
                : launch_gemm_simt(EPI_LAYER_FWD, static_cast<const float*>(f->E), f->Kp,
                                   static_cast<const float*>(f->Wh), f->Kp, eb, f->P, BC, f->Kp, 1, st);
    FNO_TRY(launch_ok(f, e, "inverse DFT + 1x1 convolution", CAT_LAYER, 2.0 * f->P * BC * (f->Kc + C)));
  }
  return SCW_OK;
}

// A reduction of the backward pass, queued for reduce_all.
static void reduce_into(std::vector<RedSeg>& segs, const float* part, int rows, int width, long long pitch,
                        float* out) {
  RedSeg sg{};
  sg.part = part;
  sg.out = out;
  sg.pitch = pitch;
  sg.rows = rows;
  sg.width = width;
  segs.push_back(sg);
}

// Every queued reduction in two launches; the table is uploaded when the batch size changes.
static scw_status reduce_all(scw_fno_s* f, std::vector<RedSeg>& segs, int B, cudaStream_t st) {
  if (f->segs_B != B) {
    if (!plan_reduce_segments(segs, f->scratch, f->scratch_floats, f->seg_items1, f->seg_items2))
      return set_error(SCW_ERR_UNSUPPORTED, "reduction scratch too small");
    if (f->d_segs) cudaFree(f->d_segs);
    f->d_segs = nullptr;
    cudaError_t e = cudaMalloc(&f->d_segs, segs.size() * sizeof(RedSeg));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f->d_segs, segs.data(), segs.size() * sizeof(RedSeg), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // segs is a local table
    if (e != cudaSuccess) return cuda_error(e, "reduction table");
    f->nseg = (int)segs.size();
    f->segs_B = B;
  }
  cudaError_t e = launch_reduce_segments(f->d_segs, f->nseg, f->seg_items1, f->seg_items2, st);
  if (f->seg_items2) ++f->counter;
  return launch_ok(f, e, "partial-sum reductions");
}

// ---------------------------------------------------------------- backward ---
template <typename T>
static scw_status forward_backward(scw_fno_s* f, const float2* n, const float2* target, int B, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(f->grad, 0, (size_t)f->n_params * sizeof(float), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
  FNO_TRY(forward<T>(f, n, B, true, st));
  const int BC = B * C, P = f->P, nblk = f->nblk;
  std::vector<RedSeg> segs;
  FNO_TRY(launch_ok(f, launch_target_norm(target, f->part_tn, B, P, st), "target norm"));
  FNO_TRY(launch_ok(f, launch_project_train<T>(static_cast<const T*>(f->Vcl[f->L]), target, at<T>(f->wcopy, f->off_Q),
                                               f->part_tn, static_cast<T*>(f->dZcf[0]),
                                               f->bf16 ? nullptr : static_cast<T*>(f->dZcl[0]), f->part_err,
                                               f->part_pool, f->part_proj, B, P, st),
                    "projection"));
  reduce_into(segs, f->part_proj, B * nblk, OUT * C + OUT, OUT * C + OUT, f->grad + f->off_Q);
  FNO_TRY(launch_ok(f, launch_head<T>(f->part_tn, f->part_err, f->part_pool, at<T>(f->wcopy, f->off_e), f->part_head,
                                      f->h_d, f->rel2_d, B, P, st),
                    "error head"));
  e = cudaMemsetAsync(f->loss_d, 0, 4 * sizeof(float), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
  reduce_into(segs, f->part_head, B, C + 1, C + 3, f->grad + f->off_e);
  reduce_into(segs, f->part_head + C + 1, B, 2, C + 3, f->loss_d + 1);
  const long long ld = (long long)f->Bmax * C;
  const long long vstride = ld * (f->Kc / 2);
  const long long mix_w = (long long)f->m * f->m * C * C * 2;
  int cur = 0;
  for (int l = f->L - 1; l >= 0; --l) {
    const int bn = dft_bn(f);
    const int ks = dft_splits(f, B, bn);
    EpiArgs ea{};
    ea.alpha = 1.f / ((float)f->N * (float)f->N);
    ea.rows = BC;
    ea.cols = f->Kc;
    ea.out = f->GWh;
    ea.ld = ld;
    ea.split_stride = vstride;
    // dW_l = sum_b dZ_b V_b^T
    const int groups = (B + 3) / 4;
    EpiArgs ew{};
    ew.rows = BC;
    ew.B = B;
    ew.out = f->part_dw[l];
    // at 2 m^2 = 512 kept-mode columns both products run in one kernel that reads dZ once (the two
    // column tiles of the DFT each take one half of the pixels of dW: two partials)
    const bool fused = f->bf16 && bn == 256 && ks == 1 && f->Kc == 512 && P % 128 == 0;
    const int kw = fused ? 2 : dw_splits(f, B);
    ew.splits = kw;
    if (fused) {
      e = launch_gemm_dft_dw(f->map_dZcf[cur], f->map_D, f->map_Vcf[l], ea, ew, BC, f->Kc, P, f->d_err,
                             f->timeout_ns, st);
      FNO_TRY(launch_ok(f, e, "truncated DFT of dZ and weight gradient", CAT_DFT,
                        2.0 * BC * f->Kc * P + 2.0 * BC * C * P));
    } else {
      e = f->bf16 ? launch_gemm_tc(EPI_MODES, bn, f->map_dZcf[cur], f->map_D, f->map_D, f->map_D, ea, BC, f->Kc, P,
                                   ks, f->d_err, f->timeout_ns, st)
                  : launch_gemm_simt(EPI_MODES, static_cast<const float*>(f->dZcf[cur]), P,
                                     static_cast<const float*>(f->D), P, ea, BC, f->Kc, P, ks, st);
      FNO_TRY(launch_ok(f, e, "truncated DFT of dZ", CAT_DFT, 2.0 * BC * f->Kc * P));
      e = f->bf16 ? launch_gemm_tc(EPI_DW, 128, f->map_dZcf[cur], f->map_Vcf[l], f->map_D, f->map_D, ew, groups * 128,
                                   groups * 128, P, kw, f->d_err, f->timeout_ns, st)
                  : launch_gemm_simt(EPI_DW, static_cast<const float*>(f->dZcf[cur]), P,
                                     static_cast<const float*>(f->Vcf[l]), P, ew, groups * 128, groups * 128, P, kw,
                                     st);
      FNO_TRY(launch_ok(f, e, "weight gradient", CAT_DW, 2.0 * BC * C * P));
    }
    reduce_into(segs, f->part_dw[l], groups * kw * 4, C * C, C * C, f->grad + f->off_W[l]);
    // mixing backward
    constexpr bool tc_mix = std::is_same<T, __nv_bfloat16>::value;
    const int sb = tc_mix ? mix_dr_blocks(B) : mix_sample_blocks(B);
    if constexpr (tc_mix) {
      // GVh = R^H G and the per-block dR, dc partials on the tensor cores
      FNO_TRY(launch_ok(f, launch_mix_tc(true, reinterpret_cast<const float2*>(f->GWh), ks, vstride, ld,
                                         at<T>(f->wcopy, f->off_R[l]), static_cast<T*>(f->GVh), 1.f, B, f->m,
                                         f->Kp, f->d_err, f->timeout_ns, st),
                        "mode mixing backward (data)", CAT_MIX, 8.0 * f->m * f->m * C * C * B));
      FNO_TRY(launch_ok(f, launch_mix_dr_tc(reinterpret_cast<const float2*>(f->GWh),
                                            reinterpret_cast<const float2*>(f->Vh[l]), ks, vstride, ld,
                                            f->part_mix[l], B, f->m, f->N, f->d_err, f->timeout_ns, st),
                        "mode mixing backward (weights)", CAT_MIX, 8.0 * f->m * f->m * C * C * B));
    } else {
      FNO_TRY(launch_ok(f, launch_mix_bwd<T>(reinterpret_cast<const float2*>(f->GWh),
                                             reinterpret_cast<const float2*>(f->Vh[l]), ks, vstride, ld,
                                             at<T>(f->wcopy, f->off_R[l]), static_cast<T*>(f->GVh), f->part_mix[l],
                                             B, f->m, f->Kp, f->N, true, st),
                        "mode mixing backward", CAT_MIX, 16.0 * f->m * f->m * C * C * B));
    }
    reduce_into(segs, f->part_mix[l], sb, (int)mix_w, mix_w + C, f->grad + f->off_R[l]);
    reduce_into(segs, f->part_mix[l] + mix_w, sb, C, mix_w + C, f->grad + f->off_c[l]);
    // dV_l = Re IDFT(GVh) + W^T dZ, times GELU'(Z_{l-1})
    EpiArgs eb{};
    eb.alpha = 1.f;
    eb.rows = P;
    eb.cols = BC;
    eb.P = P;
    eb.B = B;
    eb.w = at<T>(f->wcopy, f->off_W[l]);
    eb.x_cl = f->dZcl[cur];
    eb.g_in = l > 0 ? f->Gcl[l - 1] : nullptr;
    eb.out_cf = l > 0 ? f->dZcf[1 - cur] : nullptr;  // dV_0 is consumed channel-last only (lift backward)
    eb.out_cl = (!f->bf16 || l == 0) ? f->dZcl[1 - cur] : nullptr;
    e = f->bf16 ? launch_gemm_tc(EPI_LAYER_BWD, 256, f->map_E, f->map_GVh, f->map_dZx[cur], f->map_WT[l], eb, P, BC,
                                 f->Kp, 1, f->d_err, f->timeout_ns, st)
                : launch_gemm_simt(EPI_LAYER_BWD, static_cast<const float*>(f->E), f->Kp,
                                   static_cast<const float*>(f->GVh), f->Kp, eb, P, BC, f->Kp, 1, st);
    FNO_TRY(launch_ok(f, e, "layer backward", CAT_LAYER, 2.0 * P * BC * (f->Kc + C)));
    cur = 1 - cur;
  }
  FNO_TRY(launch_ok(f, launch_lift_bwd<T>(static_cast<const T*>(f->dZcl[cur]), n, f->part_lift, B, f->S, f->in_grid,
                                          f->N, st),
                    "lift backward"));
  const int lift_rows = (B * f->in_grid * f->in_grid + 127) / 128;
  reduce_into(segs, f->part_lift, lift_rows, C * 2 * f->S + C, C * 2 * f->S + C, f->grad + f->off_P);
  return reduce_all(f, segs, B, st);
}

template <typename T>
static scw_status infer_t(scw_fno_s* f, const float2* n, int B, float2* field, float* est, unsigned char* flag,
                          float threshold, cudaStream_t st) {
  FNO_TRY(forward<T>(f, n, B, false, st));
  FNO_TRY(launch_ok(f, launch_project_infer<T>(static_cast<const T*>(f->Vcl[f->L]), at<T>(f->wcopy, f->off_Q), field,
                                               f->part_pool, B, f->P, st),
                    "projection"));
  FNO_TRY(launch_ok(f, launch_head_infer<T>(f->part_pool, at<T>(f->wcopy, f->off_e), f->q_cal, threshold, f->h_d, est,
                                            flag, B, f->P, st),
                    "error head"));
  return SCW_OK;
}

static scw_status read_loss(scw_fno_s* f, float* loss, cudaStream_t st) {
  if (!loss) return SCW_OK;
  cudaError_t e = cudaMemcpyAsync(loss, f->loss_d, 3 * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "loss read-back");
  loss[0] = loss[1] + loss[2];
  int err = 0;
  e = cudaMemcpy(&err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "error word read-back");
  if (err) return set_error(SCW_ERR_TIMEOUT, "a tensor-core GEMM wait ran out (code " + std::to_string(err) + ")");
  if (!std::isfinite(loss[0])) return set_error(SCW_ERR_NUMERIC, "loss is not finite");
  return SCW_OK;
}

static scw_status check_batch(const scw_fno_s* f, const void* n, int B) {
  if (!f) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle is NULL");
  if (!n) return set_error(SCW_ERR_INVALID_ARGUMENT, "n is NULL");
  if (B < 1 || B > f->Bmax) return set_error(SCW_ERR_INVALID_ARGUMENT, "B must be in [1, batch_max]");
  return SCW_OK;
}

extern "C" {

scw_status scw_surrogate_create(const scw_fno_desc* d, scw_fno_t* out) {
  if (!d || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "desc and out are required");
  *out = nullptr;
  if (d->width != C) return set_error(SCW_ERR_UNSUPPORTED, "width must be 32");
  if (d->grid != 16 && d->grid != 32 && d->grid != 64) return set_error(SCW_ERR_UNSUPPORTED, "grid must be 16, 32 or 64");
  if (d->modes < 4 || d->modes % 4 || d->modes > d->grid)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "modes must be a multiple of 4 in [4, grid]");
  if (d->layers < 1 || d->layers > 8) return set_error(SCW_ERR_INVALID_ARGUMENT, "layers must be in [1, 8]");
  if (d->slices < 1 || d->slices > 16) return set_error(SCW_ERR_INVALID_ARGUMENT, "slices must be in [1, 16]");
  if (d->in_grid < 1 || d->grid % d->in_grid) return set_error(SCW_ERR_INVALID_ARGUMENT, "in_grid must divide grid");
  if (d->batch_max < 1 || d->batch_max > 4096) return set_error(SCW_ERR_INVALID_ARGUMENT, "batch_max must be in [1, 4096]");
  if (d->precision != SCW_FNO_BF16 && d->precision != SCW_FNO_FP32)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "unknown precision");
  scw_status s = check_device();
  if (s != SCW_OK) return s;

  scw_fno_s* f = new (std::nothrow) scw_fno_s();
  if (!f) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  f->d = *d;
  f->bf16 = d->precision == SCW_FNO_BF16;
  f->esz = f->bf16 ? 2 : 4;
  f->N = d->grid;
  f->P = d->grid * d->grid;
  f->m = d->modes;
  f->Kc = 2 * d->modes * d->modes;
  f->Kp = (f->Kc + 63) / 64 * 64;
  f->L = d->layers;
  f->S = d->slices;
  f->in_grid = d->in_grid;
  f->Bmax = d->batch_max;
  f->nblk = f->P / PIX_BLOCK;

  // flat parameter layout
  long long o = 0;
  f->off_P = o;
  o += (long long)C * 2 * f->S + C;
  for (int l = 0; l < f->L; ++l) {
    f->off_R[l] = o;
    o += (long long)f->m * f->m * C * C * 2;
    f->off_W[l] = o;
    o += C * C;
    f->off_c[l] = o;
    o += C;
  }
  f->off_Q = o;
  o += OUT * C + OUT;
  f->off_e = o;
  o += C + 1;
  f->n_params = o;

  const size_t Bm = (size_t)f->Bmax, P = (size_t)f->P, esz = f->esz;
  const size_t act = Bm * C * P * esz;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = falloc(f, p, bytes);
  };
  A((void**)&f->master, f->n_params * 4);
  A((void**)&f->grad, f->n_params * 4);
  A((void**)&f->adam_m, f->n_params * 4);
  A((void**)&f->adam_v, f->n_params * 4);
  A(&f->wcopy, f->n_params * esz);
  A(&f->D, (size_t)f->Kc * P * esz);
  A(&f->E, P * f->Kp * esz);
  for (int l = 0; l <= f->L; ++l) {
    A(&f->Vcf[l], act);
    A(&f->Vcl[l], act);
  }
  for (int l = 0; l + 1 < f->L; ++l) A(&f->Gcl[l], act);
  for (int l = 0; l < f->L; ++l) A((void**)&f->Vh[l], (size_t)kMaxSplit * Bm * C * f->Kc * 4);
  A((void**)&f->GWh, (size_t)kMaxSplit * Bm * C * f->Kc * 4);
  A(&f->Wh, Bm * C * f->Kp * esz);
  A(&f->GVh, Bm * C * f->Kp * esz);
  for (int i = 0; i < 2; ++i) {
    A(&f->dZcf[i], act);
    A(&f->dZcl[i], act);
  }
  A((void**)&f->part_head, Bm * (C + 3) * 4);
  A((void**)&f->part_tn, Bm * f->nblk * 4);
  A((void**)&f->part_err, Bm * f->nblk * 4);
  A((void**)&f->part_pool, Bm * f->nblk * C * 4);
  A((void**)&f->part_proj, Bm * f->nblk * (OUT * C + OUT) * 4);
  for (int l = 0; l < f->L; ++l)
    A((void**)&f->part_mix[l], (size_t)mix_sample_blocks(f->Bmax) * ((size_t)f->m * f->m * C * C * 2 + C) * 4);
  A(&f->WT, (size_t)f->L * C * C * esz);
  for (int l = 0; l < f->L; ++l) A((void**)&f->part_dw[l], ((Bm + 3) / 4) * kMaxSplit * 4 * C * C * 4);
  A((void**)&f->part_lift, ((Bm * f->in_grid * f->in_grid + 127) / 128) * (C * 2 * f->S + C) * 4);
  // reduction chunks: at most 64 rows of every reduced width, for the projection, the weight
  // gradients of every layer and the lift
  f->scratch_floats = (size_t)64 * ((OUT * C + OUT) + (size_t)f->L * C * C + (C * 2 * f->S + C) + 4096);
  A((void**)&f->scratch, f->scratch_floats * 4);
  A((void**)&f->loss_d, 4 * 4);
  A((void**)&f->h_d, Bm * 4);
  A((void**)&f->rel2_d, Bm * 4);
  A((void**)&f->d_err, 4);
  if (e != cudaSuccess) {
    free_all(f);
    delete f;
    return cuda_error(e, "surrogate workspace");
  }
  // constant tables, zero pads, parameters
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaMemsetAsync(f->E, 0, P * f->Kp * esz, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->Wh, 0, Bm * C * f->Kp * esz, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->GVh, 0, Bm * C * f->Kp * esz, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->d_err, 0, 4, st);
  if (e == cudaSuccess)
    e = f->bf16 ? launch_tables<__nv_bfloat16>(static_cast<__nv_bfloat16*>(f->D), static_cast<__nv_bfloat16*>(f->E),
                                               f->N, f->m, f->Kp, st)
                : launch_tables<float>(static_cast<float*>(f->D), static_cast<float*>(f->E), f->N, f->m, f->Kp, st);
  std::vector<float> init((size_t)f->n_params, 0.f);
  {
    auto fill = [&](long long off, long long count, double scale) {
      for (long long i = 0; i < count; ++i) init[off + i] = (float)(scale * uniform_pm1(d->seed, off + i));
    };
    fill(f->off_P, (long long)C * 2 * f->S, 1.0 / std::sqrt(2.0 * f->S));
    for (int l = 0; l < f->L; ++l) {
      fill(f->off_R[l], (long long)f->m * f->m * C * C * 2, 1.0 / C);
      fill(f->off_W[l], C * C, 1.0 / std::sqrt((double)C));
    }
    fill(f->off_Q, OUT * C, 1.0 / std::sqrt((double)C));
    fill(f->off_e, C, 1.0 / std::sqrt((double)C));
  }
  if (e == cudaSuccess) e = cudaMemcpy(f->master, init.data(), f->n_params * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(f->adam_m, 0, f->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(f->adam_v, 0, f->n_params * 4);
  if (e == cudaSuccess)
    e = f->bf16 ? launch_copy_params<__nv_bfloat16>(f->master, static_cast<__nv_bfloat16*>(f->wcopy), f->n_params, st)
                : launch_copy_params<float>(f->master, static_cast<float*>(f->wcopy), f->n_params, st);
  if (e == cudaSuccess) e = refresh_wt(f, st);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(f);
    delete f;
    return cuda_error(e, "surrogate initialisation");
  }
  if (f->bf16) {
    const long long BCm = (long long)f->Bmax * C;
    s = make_map_bf16(&f->map_D, f->D, f->P, f->Kc, f->P, dft_bn(f));
    if (s == SCW_OK) s = make_map_bf16(&f->map_E, f->E, f->Kp, f->P, f->Kp, 128);
    if (s == SCW_OK) s = make_map_bf16(&f->map_Wh, f->Wh, f->Kp, BCm, f->Kp, 256);
    if (s == SCW_OK) s = make_map_bf16(&f->map_GVh, f->GVh, f->Kp, BCm, f->Kp, 256);
    for (int l = 0; l <= f->L && s == SCW_OK; ++l) s = make_map_bf16(&f->map_Vcf[l], f->Vcf[l], f->P, BCm, f->P, 128);
    for (int i = 0; i < 2 && s == SCW_OK; ++i) s = make_map_bf16(&f->map_dZcf[i], f->dZcf[i], f->P, BCm, f->P, 128);
    for (int l = 0; l < f->L && s == SCW_OK; ++l) {
      s = make_map_act3d(&f->map_Vx[l], f->Vcf[l], f->P, f->Bmax);
      if (s == SCW_OK)
        s = make_map_bf16(&f->map_W[l], static_cast<__nv_bfloat16*>(f->wcopy) + f->off_W[l], C, C, C, C, 32);
      if (s == SCW_OK)
        s = make_map_bf16(&f->map_WT[l], static_cast<__nv_bfloat16*>(f->WT) + (size_t)l * C * C, C, C, C, C, 32);
    }
    for (int i = 0; i < 2 && s == SCW_OK; ++i) s = make_map_act3d(&f->map_dZx[i], f->dZcf[i], f->P, f->Bmax);
    if (s != SCW_OK) {
      free_all(f);
      delete f;
      return s;
    }
  }
  *out = f;
  return SCW_OK;
}

scw_status scw_surrogate_destroy(scw_fno_t f) {
  if (!f) return SCW_OK;
  free_all(f);
  delete f;
  return SCW_OK;
}

scw_status scw_surrogate_param_count(scw_fno_t f, size_t* count) {
  if (!f || !count) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle and count are required");
  *count = (size_t)f->n_params;
  return SCW_OK;
}

scw_status scw_surrogate_set_params(scw_fno_t f, const float* host, size_t count) {
  if (!f || !host) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle and host are required");
  if (count != (size_t)f->n_params) return set_error(SCW_ERR_INVALID_ARGUMENT, "count differs from the parameter count");
  cudaError_t e = cudaMemcpy(f->master, host, count * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(f->adam_m, 0, count * 4);
  if (e == cudaSuccess) e = cudaMemset(f->adam_v, 0, count * 4);
  if (e == cudaSuccess)
    e = f->bf16 ? launch_copy_params<__nv_bfloat16>(f->master, static_cast<__nv_bfloat16*>(f->wcopy), f->n_params, 0)
                : launch_copy_params<float>(f->master, static_cast<float*>(f->wcopy), f->n_params, 0);
  if (e == cudaSuccess) e = refresh_wt(f, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "set_params");
  f->step = 0;
  return SCW_OK;
}

static scw_status copy_out(const float* dev, float* host, size_t count, size_t expect) {
  if (!host) return set_error(SCW_ERR_INVALID_ARGUMENT, "host is required");
  if (count != expect) return set_error(SCW_ERR_INVALID_ARGUMENT, "count differs from the parameter count");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, dev, count * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SCW_OK : cuda_error(e, "copy to host");
}

scw_status scw_surrogate_get_params(scw_fno_t f, float* host, size_t count) {
  if (!f) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle is NULL");
  return copy_out(f->master, host, count, (size_t)f->n_params);
}

scw_status scw_surrogate_get_grads(scw_fno_t f, float* host, size_t count) {
  if (!f) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle is NULL");
  return copy_out(f->grad, host, count, (size_t)f->n_params);
}

scw_status scw_surrogate_forward_backward(scw_fno_t f, const void* n, const void* target, int B, float* loss,
                                          void* stream) {
  FNO_TRY(check_batch(f, n, B));
  if (!target) return set_error(SCW_ERR_INVALID_ARGUMENT, "target is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FNO_TRY(begin_call(f, st));
  scw_status s = f->bf16 ? forward_backward<__nv_bfloat16>(f, static_cast<const float2*>(n),
                                                          static_cast<const float2*>(target), B, st)
                         : forward_backward<float>(f, static_cast<const float2*>(n), static_cast<const float2*>(target),
                                                   B, st);
  f->launches_train = f->counter;
  if (s != SCW_OK) return s;
  FNO_TRY(end_call(f));
  return read_loss(f, loss, st);
}

scw_status scw_surrogate_train_step(scw_fno_t f, const void* n, const void* target, int B, float lr, float* loss,
                                    void* stream) {
  FNO_TRY(check_batch(f, n, B));
  if (!target) return set_error(SCW_ERR_INVALID_ARGUMENT, "target is NULL");
  if (!(lr >= 0.f)) return set_error(SCW_ERR_INVALID_ARGUMENT, "lr must be >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FNO_TRY(begin_call(f, st));
  scw_status s = f->bf16 ? forward_backward<__nv_bfloat16>(f, static_cast<const float2*>(n),
                                                          static_cast<const float2*>(target), B, st)
                         : forward_backward<float>(f, static_cast<const float2*>(n), static_cast<const float2*>(target),
                                                   B, st);
  if (s != SCW_OK) return s;
  ++f->step;
  const float bc1 = (float)(1.0 - std::pow(0.9, f->step)), bc2 = (float)(1.0 - std::pow(0.999, f->step));
  cudaError_t e = f->bf16 ? launch_adam<__nv_bfloat16>(f->master, f->grad, f->adam_m, f->adam_v,
                                                       static_cast<__nv_bfloat16*>(f->wcopy), f->n_params, lr, bc1, bc2,
                                                       st)
                          : launch_adam<float>(f->master, f->grad, f->adam_m, f->adam_v, static_cast<float*>(f->wcopy),
                                               f->n_params, lr, bc1, bc2, st);
  FNO_TRY(launch_ok(f, e, "Adam"));
  if (f->bf16) FNO_TRY(launch_ok(f, refresh_wt(f, st), "W transpose"));
  f->launches_train = f->counter;
  FNO_TRY(end_call(f));
  return read_loss(f, loss, st);
}

scw_status scw_surrogate_infer(scw_fno_t f, const void* n, int B, void* field, float* est_err,
                               unsigned char* need_fallback, float threshold, void* stream) {
  FNO_TRY(check_batch(f, n, B));
  if (!field) return set_error(SCW_ERR_INVALID_ARGUMENT, "field is NULL");
  if ((reinterpret_cast<uintptr_t>(field) & 7u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "field must be 8-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FNO_TRY(begin_call(f, st));
  scw_status s = f->bf16 ? infer_t<__nv_bfloat16>(f, static_cast<const float2*>(n), B, static_cast<float2*>(field),
                                                 est_err, need_fallback, threshold, st)
                         : infer_t<float>(f, static_cast<const float2*>(n), B, static_cast<float2*>(field), est_err,
                                          need_fallback, threshold, st);
  f->launches_infer = f->counter;
  if (s != SCW_OK) return s;
  return end_call(f);
}

scw_status scw_surrogate_calibrate(scw_fno_t f, const float* est, const float* true_err, int count, float miss,
                                   float* q_out) {
  if (!f || !est || !true_err) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle, est and true_err are required");
  if (count < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "count must be >= 1");
  if (!(miss > 0.f && miss < 1.f)) return set_error(SCW_ERR_INVALID_ARGUMENT, "miss must be in (0, 1)");
  std::vector<double> r((size_t)count);
  for (int i = 0; i < count; ++i) {
    if (!(est[i] > 0.f) || !(true_err[i] > 0.f)) return set_error(SCW_ERR_INVALID_ARGUMENT, "estimates and errors must be > 0");
    r[i] = std::log((double)true_err[i]) - std::log((double)est[i]);
  }
  std::sort(r.begin(), r.end());
  long long k = (long long)std::ceil((1.0 - miss) * (count + 1)) - 1;
  k = std::min<long long>(std::max<long long>(k, 0), count - 1);
  f->q_cal = (float)r[(size_t)k];
  if (q_out) *q_out = f->q_cal;
  return SCW_OK;
}

scw_status scw_surrogate_set_offset(scw_fno_t f, float q) {
  if (!f) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle is NULL");
  f->q_cal = q;
  return SCW_OK;
}

// checkpoint blob: header, then master, m, v (FP32, param_count each)
struct StateHeader {
  uint32_t magic;    // 'SCWF'
  uint32_t version;  // 1
  uint64_t n_params;
  int32_t step;
  float q_cal;
  uint64_t reserved;
};
static_assert(sizeof(StateHeader) == 32, "checkpoint header is 32 bytes");
static constexpr uint32_t kStateMagic = 0x46574353u;

scw_status scw_surrogate_state_bytes(scw_fno_t f, size_t* bytes) {
  if (!f || !bytes) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle and bytes are required");
  *bytes = sizeof(StateHeader) + 3 * (size_t)f->n_params * sizeof(float);
  return SCW_OK;
}

scw_status scw_surrogate_save_state(scw_fno_t f, void* host, size_t bytes) {
  if (!f || !host) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle and host are required");
  const size_t n = (size_t)f->n_params;
  if (bytes != sizeof(StateHeader) + 3 * n * sizeof(float))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "bytes differs from scw_surrogate_state_bytes");
  StateHeader h{kStateMagic, 1u, (uint64_t)n, f->step, f->q_cal, 0};
  std::memcpy(host, &h, sizeof(h));
  float* dst = reinterpret_cast<float*>(static_cast<uint8_t*>(host) + sizeof(h));
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(dst, f->master, n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(dst + n, f->adam_m, n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(dst + 2 * n, f->adam_v, n * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SCW_OK : cuda_error(e, "save_state");
}

scw_status scw_surrogate_load_state(scw_fno_t f, const void* host, size_t bytes) {
  if (!f || !host) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle and host are required");
  const size_t n = (size_t)f->n_params;
  if (bytes != sizeof(StateHeader) + 3 * n * sizeof(float))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "bytes differs from scw_surrogate_state_bytes");
  StateHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (h.magic != kStateMagic || h.version != 1u || h.n_params != (uint64_t)n || h.step < 0)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "not a checkpoint of this surrogate shape");
  const float* src = reinterpret_cast<const float*>(static_cast<const uint8_t*>(host) + sizeof(h));
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(f->master, src, n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->adam_m, src + n, n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->adam_v, src + 2 * n, n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = f->bf16 ? launch_copy_params<__nv_bfloat16>(f->master, static_cast<__nv_bfloat16*>(f->wcopy), f->n_params, 0)
                : launch_copy_params<float>(f->master, static_cast<float*>(f->wcopy), f->n_params, 0);
  if (e == cudaSuccess) e = refresh_wt(f, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "load_state");
  f->step = h.step;
  f->q_cal = h.q_cal;
  return SCW_OK;
}

scw_status scw_surrogate_enable_timing(scw_fno_t f, int on) {
  if (!f) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle is NULL");
  f->timing = on != 0;
  for (int c = 0; c < 5; ++c) f->acc_ms[c] = f->acc_flops[c] = 0;
  f->timed_calls = 0;
  return SCW_OK;
}

scw_status scw_surrogate_get_timings(scw_fno_t f, scw_fno_times* out) {
  if (!f || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle and out are required");
  out->calls = f->timed_calls;
  out->dft_ms = f->acc_ms[CAT_DFT];
  out->layer_ms = f->acc_ms[CAT_LAYER];
  out->dw_ms = f->acc_ms[CAT_DW];
  out->mix_ms = f->acc_ms[CAT_MIX];
  out->other_ms = f->acc_ms[CAT_OTHER];
  out->total_ms = 0;
  for (int c = 0; c < 5; ++c) out->total_ms += f->acc_ms[c];
  out->dft_flops = f->acc_flops[CAT_DFT];
  out->layer_flops = f->acc_flops[CAT_LAYER];
  out->dw_flops = f->acc_flops[CAT_DW];
  out->mix_flops = f->acc_flops[CAT_MIX];
  return SCW_OK;
}

scw_status scw_surrogate_launches(scw_fno_t f, int* train_step, int* infer) {
  if (!f) return set_error(SCW_ERR_INVALID_ARGUMENT, "handle is NULL");
  if (train_step) *train_step = f->launches_train;
  if (infer) *infer = f->launches_infer;
  return SCW_OK;
}

}  // extern "C"
