// Internal declarations shared by the libscw translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/scw.h"

namespace scw {

// Device error word bits (atomicOr'ed by kernels, read by scw_plan_check).
enum : int {
  DEV_ERR_TIMEOUT_FULL = 1,    // consumer wait on a filled stage ran out
  DEV_ERR_TIMEOUT_EMPTY = 2,   // producer wait on a free stage ran out
  DEV_ERR_TIMEOUT_ACCUM = 4,   // wait on an accumulator buffer ran out
  DEV_ERR_TIMEOUT_DRAIN = 8,   // wait for in-flight work after an abort ran out
  DEV_ERR_TIMEOUT_DEP = 16,    // wait on a cross-CTA dependency counter ran out
  DEV_ERR_BOUNDS = 32          // SCW_FLAG_DEBUG_BOUNDS: an index left its buffer (the access was skipped)
};

// Buffers whose indices the SCW_FLAG_DEBUG_BOUNDS path checks (ItemDev::bnd holds their extents).
enum : int { BND_S_PART = 0, BND_T, BND_TWX, BND_TWY, BND_B, BND_GAMMA, BND_ALPHA, BND_OUT, BND_C, BND_WT,
             BND_COUNT };

// Kernel trace (scw_plan_enable_trace): per slot, the %globaltimer nanoseconds at which the first CTA
// of a kernel began its work (after any wait on the kernel before it) and the last CTA finished:
// trace[2 slot] = min over CTAs, trace[2 slot + 1] = max over CTAs.
enum : int { TRACE_PHASES = 0, TRACE_EXTERIOR = 1, TRACE_CONTRACT = 2, TRACE_XPASS = 3, TRACE_YPASS = 4,
             TRACE_SLOTS = 8 };

__device__ __forceinline__ unsigned long long trace_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// thread 0 of each CTA stamps; a null trace pointer (tracing off) costs one predicated branch
__device__ __forceinline__ void trace_begin(unsigned long long* tr, int slot) {
  if (tr != nullptr && threadIdx.x == 0) atomicMin(tr + 2 * slot, trace_clock());
}
__device__ __forceinline__ void trace_end(unsigned long long* tr, int slot) {
  if (tr != nullptr && threadIdx.x == 0) atomicMax(tr + 2 * slot + 1, trace_clock());
}

constexpr int kMaxFx = 4096;
constexpr int kMaxM = 4096;              // U*V
constexpr int kMaxPlanesPerLayer = 128;  // per contraction pass (N <= 256)

// Plane slot of an active layer: which layer, where its planes start in the
// global plane list and how many it has.
struct LayerUnit {
  int layer;
  int f0;
  int nf;
  int ks;  // K splits of this unit's contraction tasks (tensor-core plans; 0 = the item's k_split)
};

// Everything a kernel needs to know about one synthesis item. Kernels take it
// by value (__grid_constant__) for a single plan, or index a device array of
// them for a batch.
struct ItemDev {
  const void* Ahi;         // tensor-core A = W: tile-major swizzled [L][tiles][nk][rows][64] (hi or FP16)
  const void* Alo;         // low part (split-BF16 only)
  const LayerUnit* units;
  const double* zplanes;
  const double* zbounds;
  const double2* gamma;
  const double2* alpha;
  void* Bhi;               // [unit][nk][NB][64], same swizzled layout
  void* Blo;
  float2* S_part;          // [k_split][Fz][3M]
  const int* nsplit;       // [Fz]
  const float2* twx;       // [Up][Fx/8]   fold twiddles at wrapped positions (fold_pos; residue b
                           //               fastest: the lanes of an x-pass warp take consecutive b)
  const float2* twy;       // [Fy/8][Vp]
  float2* T;               // [Fz][3][V][Fx] x-pass rows (plans only)
  size_t split_stride;     // Fz * 3M
  double inv_lam;
  int M, U, V, Fx, Fy, Fz;
  int F_pad, k_split, n_tiles, nk, n_units;
  int Up, Vp;              // padded fold lengths roundup(U, 8), roundup(V, 8)
  int I, Fz_out;           // illuminations; output planes per illumination (Fz = I Fz_out,
                           // plane index f = (output plane) I + illumination)
  size_t alpha_istride;    // L 4M: alpha elements per illumination
  int tx, ty;              // periodic tiles of the field along x and y
  long long ld, pstride;   // field row pitch and plane-slice stride (complex elements)
  unsigned long long* trace;  // kernel trace stamps [TRACE_SLOTS][2], or null (tracing off)
  int rows_tile;           // rows of W per contraction row tile (<= 128)
  int dbg;                 // SCW_FLAG_DEBUG_BOUNDS: kernels check every global index against bnd
  int* err;                // the plan's device error word (DEV_ERR_BOUNDS)
  unsigned long long bnd[BND_COUNT];  // extents in elements of the checked buffers (dbg only)
};

// Index check of the debug path: true when element i of buffer `buf` exists (always true for
// plans without SCW_FLAG_DEBUG_BOUNDS: one uniform branch); otherwise record DEV_ERR_BOUNDS and
// return false so that the caller skips the access.
__device__ __forceinline__ bool in_bounds(const ItemDev& it, int buf, size_t i) {
  if (!it.dbg || i < it.bnd[buf]) return true;
  atomicOr(it.err, DEV_ERR_BOUNDS);
  return false;
}

struct PointTables;  // scw_points.cuh

struct Plan {
  // description
  int U = 0, V = 0, M = 0, L = 0, Fx = 0, Fy = 0, Fz = 0;  // Fz = I Fz_out plane slots
  int I = 1, Fz_out = 0;                                  // illuminations, output planes each
  int tiles_x = 1, tiles_y = 1;                           // periodic tiling of the field
  long long out_ld = 0, out_pstride = 0;                  // field pitches (complex elements)
  double pupil_na = 0;
  double lambda = 0, X = 0, Y = 0, x0 = 0, y0 = 0, n_top = 1, z_inc = 0;
  double n_bot_re = 1, n_bot_im = 0;
  int precision = 0;
  unsigned flags = 0;
  std::vector<double> z_bounds, z_planes;

  // plane assignment (host copies)
  std::vector<int> plane_region;  // -1 above, 0..L-1 layer, L below
  std::vector<LayerUnit> units;
  int F_pad = 8;      // plane slots per layer (multiple of 8)
  int NB = 16;        // 2 * F_pad: real columns of the tensor-core B operand
  int k_split = 1;                // the largest K split over the units (S_part holds that many partials)
  int rows_tile = 128;            // rows of W per contraction row tile (ItemDev::rows_tile)
  unsigned long long bnd_real[BND_COUNT] = {};  // buffer extents (SCW_FLAG_DEBUG_BOUNDS plans)
  std::vector<int> unit_ks;        // per-unit K split (tensor-core plans; empty = k_split everywhere)
  int n_exterior = 0;

  // device tables
  LayerUnit* d_units = nullptr;
  double* d_zplanes = nullptr;
  double* d_zbounds = nullptr;     // [L+1]
  int* d_nsplit = nullptr;         // [Fz] partial sums to add per plane
  int* d_nsplit1 = nullptr;        // [Fz] all ones (caller-given spectra)
  int* d_ext_planes = nullptr;     // [n_exterior] plane indices outside the sample
  double2* d_sz_top = nullptr;     // [M]
  double2* d_sz_bot = nullptr;     // [M]
  float2* d_twx = nullptr;         // [Up][Fx/8]
  float2* d_twy = nullptr;         // [Fy/8][Vp]
  float* d_pupil = nullptr;        // [M] 1 / 0 transmission of the pupil (pupil_na > 0)
  PointTables* pts = nullptr;      // lateral point set (scw_plan_set_points), owned

  // attached inputs (not owned)
  const double2* gamma = nullptr;
  const double2* alpha = nullptr;
  const double2* p_inc = nullptr;
  const double2* p_ref = nullptr;
  const double2* p_trn = nullptr;
  bool layers_set = false;

  // converted W (owned)
  __nv_bfloat16* Whi = nullptr;   // tile-major swizzled, L * 3M * nk * 64 elements
  __nv_bfloat16* Wlo = nullptr;
  __half* Wh = nullptr;           // same layout
  float2* Wt = nullptr;           // [L][4M][3M]

  // per-synthesis workspace (owned)
  void* Bhi = nullptr;            // [unit][nk][NB][64] bf16 or fp16 (swizzled)
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

  ItemDev item;                   // host copy of the kernels' view of this item

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last W conversion
  bool convert_pending = false;
  size_t workspace_bytes = 0;
  double convert_ms = 0;
};

// Contraction schedule of a set of items: tasks (item, unit, row tile, split)
// grouped per persistent CTA, longest first (LPT).
struct TcSchedule {
  int4* d_tasks = nullptr;
  int* d_cta_off = nullptr;       // [grid + 1]
  int grid = 0;
  int n_tasks = 0;
  double max_load = 0, mean_load = 0;  // in K-stages, for the autotuner's report
};

// Fold layout of the recomposition: the signed order u of an axis with n orders
// (u in [-floor(n/2), n - 1 - floor(n/2)]) sits at position u mod np, np = roundup(n, 8),
// so that position mod 8 = u mod 8 and a fold over residues walks whole groups of 8
// positions; the positions between the largest positive and the smallest wrapped
// negative order hold zeros.
__host__ __device__ __forceinline__ int fold_np(int n) { return (n + 7) / 8 * 8; }
__host__ __device__ __forceinline__ int fold_pos(int ui, int n, int np) {
  const int u = ui - n / 2;
  return u >= 0 ? u : u + np;
}
// order index ui at position pos, or -1 for a zero position
__host__ __device__ __forceinline__ int fold_order(int pos, int n, int np) {
  const int h = n / 2;
  if (pos <= n - 1 - h) return pos + h;
  if (pos >= np - h) return pos - np + h;
  return -1;
}

// Launch with programmatic stream serialisation (the kernel may start before its predecessor on
// the stream ends and waits for it with griddepcontrol.wait before reading its results).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per (kernel, device): the attribute call is not repeated on the launch path.
cudaError_t allow_max_smem(const void* kernel);

// error reporting (thread-local message)
scw_status set_error(scw_status s, const std::string& msg);
scw_status cuda_error(cudaError_t e, const char* what);
scw_status check_device();  // SCW_OK on an sm_103 device

// launchers (host side), each returns cudaSuccess or the launch error
cudaError_t launch_convert_tiled(const float2* W, void* hi, void* lo, int L, int M, int rows_tile, bool bf16_split,
                                 cudaStream_t st);
cudaError_t launch_transpose_layers(const float2* W, float2* Wt, int L, int rows, int cols, cudaStream_t st);

// step (a): unit entries are (item, unit) pairs; items == nullptr means "the single item `one`"
cudaError_t launch_phases_tc(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries,
                             int max_M, int F_pad, bool bf16, cudaStream_t st);
cudaError_t launch_phases_fp32(const Plan& p, cudaStream_t st);
cudaError_t launch_exterior(const Plan& p, cudaStream_t st);

// step (b)
// inject: failure injection for tests; the first CTA leaves its first operand stage
// unfilled, so its bounded waits run out and it reports DEV_ERR_TIMEOUT_* (0 in production)
cudaError_t launch_contract_tc(const ItemDev& one, const ItemDev* items, const TcSchedule& s, int NB, bool bf16,
                               int* err, uint64_t timeout_ns, int inject, cudaStream_t st);
cudaError_t launch_contract_fp32(const Plan& p, cudaStream_t st);
int tc_ctas_per_sm(int NB, bool bf16);

// step (c): plane entries are (item, plane) pairs; S_override / nsplit_override replace the
// contraction's partial spectra with caller-given spectra
size_t recompose_smem_bytes(int V, int Up, int Vp);
// smem_bytes: the largest xpass_smem_bytes of the items
size_t xpass_smem_bytes(int V, int Up, int Fx);
cudaError_t launch_xpass(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries,
                         size_t smem_bytes, cudaStream_t st);
// entries [0, n_pair) run the two-residue y-pass (long folds, ypass_pairs(Vp)), the rest the
// one-residue y-pass; *launches receives the number of kernels launched (0, 1 or 2)
bool ypass_pairs(int Vp);
// max_twy: the largest fold-twiddle table (Fy/8) Vp of the items, in complex elements (staged in
// shared memory when it fits); tiled: some item has periodic tiles (selects the y-pass that stores
// every tile)
cudaError_t launch_ypass(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries, int n_pair,
                         int max_Qx, int max_Vp, int max_twy, bool tiled, float2* out_one, float2* const* d_outs,
                         cudaStream_t st, int* launches);
cudaError_t launch_recompose(const ItemDev& one, const ItemDev* items, const int2* d_entries, int n_entries, int max_Qx,
                             size_t smem, const float2* S_override, const int* nsplit_override, float2* out_one,
                             float2* const* d_outs, cudaStream_t st);
cudaError_t launch_gather_spectrum(const Plan& p, float2* S, cudaStream_t st);


}  // namespace scw
