// Internal declarations shared by the libscw translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/scw.h"

namespace scw {

// Device error word bits (atomicOr'ed by kernels, read by scw_plan_check).
enum : int {
  DEV_ERR_TIMEOUT_FULL = 1,    // consumer wait on a filled stage ran out
  DEV_ERR_TIMEOUT_EMPTY = 2,   // producer wait on a free stage ran out
  DEV_ERR_TIMEOUT_ACCUM = 4,   // epilogue wait on the accumulator ran out
  DEV_ERR_TIMEOUT_DRAIN = 8,   // wait for in-flight copies after an abort ran out
  DEV_ERR_BAD_SHAPE = 16       // a kernel saw a launch shape it cannot handle
};

constexpr int kMaxFx = 4096;
constexpr int kMaxM = 4096;         // U*V
constexpr int kMaxPlanesPerLayer = 128;  // per contraction pass (N <= 256)

// Plane slot of an active layer: which layer, where its planes start in the
// global plane list and how many it has.
struct LayerUnit {
  int layer;
  int f0;
  int nf;
  int pad;
};

struct Plan {
  // description
  int U = 0, V = 0, M = 0, L = 0, Fx = 0, Fy = 0, Fz = 0;
  double lambda = 0, X = 0, Y = 0, x0 = 0, y0 = 0, n_top = 1, z_inc = 0;
  double n_bot_re = 1, n_bot_im = 0;
  int precision = 0;
  unsigned flags = 0;
  std::vector<double> z_bounds, z_planes;
  uint64_t timeout_ns = 2000000000ull;

  // plane assignment (host copies)
  std::vector<int> plane_region;  // -1 above, 0..L-1 layer, L below
  std::vector<LayerUnit> units;
  int F_pad = 8;      // plane slots per layer (multiple of 8)
  int NB = 16;        // 2 * F_pad: real columns of the tensor-core B operand
  int k_split = 1;
  int n_exterior = 0;

  // device tables
  int* d_err = nullptr;
  LayerUnit* d_units = nullptr;
  double* d_zplanes = nullptr;
  double* d_zbounds = nullptr;     // [L+1]
  int* d_nsplit = nullptr;         // [Fz] partial sums to add per plane
  int* d_nsplit1 = nullptr;        // [Fz] all ones (caller-given spectra)
  int* d_ext_planes = nullptr;     // [n_exterior] plane indices outside the sample
  double2* d_sz_top = nullptr;     // [M]
  double2* d_sz_bot = nullptr;     // [M]
  float2* d_twx = nullptr;         // [Fx/8][U]
  float2* d_twy = nullptr;         // [Fy/8][V]

  // attached inputs (not owned)
  const double2* gamma = nullptr;
  const double2* alpha = nullptr;
  const double2* p_inc = nullptr;
  const double2* p_ref = nullptr;
  const double2* p_trn = nullptr;
  bool layers_set = false;

  // converted W (owned)
  __nv_bfloat16* Whi = nullptr;   // [L][3M][8M]
  __nv_bfloat16* Wlo = nullptr;
  __half* Wh = nullptr;           // [L][3M][8M]
  float2* Wt = nullptr;           // [L][4M][3M]

  // per-synthesis workspace (owned)
  void* Bhi = nullptr;            // [unit][NB][8M] bf16 or fp16
  void* Blo = nullptr;
  float2* Cf = nullptr;           // [unit][4M][F_pad] (FP32 path)
  float2* S_part = nullptr;       // [k_split][Fz][3M]
  float2* T = nullptr;            // [Fz][3][V][Fx]

  // host-IO copies (owned, SCW_FLAG_HOST_IO)
  float2* hio_W = nullptr;
  double2* hio_gamma = nullptr;
  double2* hio_alpha = nullptr;
  double2* hio_p = nullptr;       // [3][3][M]: inc, ref, trn
  float2* hio_out = nullptr;

  CUtensorMap tmA_hi, tmA_lo, tmB_hi, tmB_lo;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last W conversion
  bool timing = false;
  std::vector<cudaEvent_t> tev;   // 5 events per timed synthesize call
  size_t tev_used = 0;
  bool convert_pending = false;
  size_t workspace_bytes = 0;
  double convert_ms = 0;
  int kernels_per_synthesis = 0;
};

// error reporting (thread-local message)
scw_status set_error(scw_status s, const std::string& msg);
scw_status cuda_error(cudaError_t e, const char* what);

// launchers (host side), each returns cudaSuccess or the launch error
cudaError_t launch_convert_split_bf16(const float2* W, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                      size_t n_complex, cudaStream_t st);
cudaError_t launch_convert_fp16(const float2* W, __half* h, size_t n_complex, cudaStream_t st);
cudaError_t launch_transpose_layers(const float2* W, float2* Wt, int L, int rows, int cols,
                                    cudaStream_t st);
cudaError_t launch_phases_tc(const Plan& p, cudaStream_t st);
cudaError_t launch_phases_fp32(const Plan& p, cudaStream_t st);
cudaError_t launch_exterior(const Plan& p, cudaStream_t st);
cudaError_t launch_contract_tc(const Plan& p, cudaStream_t st);
cudaError_t launch_contract_fp32(const Plan& p, cudaStream_t st);
cudaError_t launch_recompose(const Plan& p, const float2* S_part, int S_splits_stride_planes,
                             const int* d_nsplit, float2* out, cudaStream_t st);
cudaError_t launch_gather_spectrum(const Plan& p, float2* S, cudaStream_t st);
cudaError_t launch_xpass(const Plan& p, const float2* S_part, int split_stride_planes, const int* d_nsplit,
                         cudaStream_t st);
cudaError_t launch_ypass(const Plan& p, float2* out, cudaStream_t st);

bool encode_tensor_maps(Plan& p, std::string& why);

}  // namespace scw
