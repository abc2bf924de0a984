// Host side of libscw: argument validation, plane-to-layer assignment,
// order / twiddle tables, workspace ownership, the contraction schedule and its
// autotuner, CUDA-graph replay, and the launch sequence of scw_synthesize and
// scw_synthesize_batched. See include/scw.h for the contract of each entry point.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <queue>

#include "scw_internal.cuh"
#include "scw_points.cuh"

namespace scw {

static thread_local std::string g_last_error;

scw_status set_error(scw_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

scw_status cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? SCW_ERR_OUT_OF_MEMORY : SCW_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// s_z = sqrt(n^2 - sx^2 - sy^2) on the decaying branch (Eq. 2): principal
// root, negated when its imaginary part is negative (or zero with Re < 0).
static std::complex<double> s_z(std::complex<double> n, double sx, double sy) {
  std::complex<double> w = std::sqrt(n * n - std::complex<double>(sx * sx + sy * sy, 0.0));
  if (w.imag() < 0 || (w.imag() == 0 && w.real() < 0)) w = -w;
  return w;
}

// exp(2 pi i t) with t reduced to [-1/2, 1/2] in FP64 first.
static float2 cis_cycles(double t) {
  const double r = t - std::nearbyint(t);
  return make_float2((float)std::cos(2.0 * M_PI * r), (float)std::sin(2.0 * M_PI * r));
}

// Stream on which plan creation queues its table uploads, clears and autotune launches: the
// caller's stream for scw_plan / scw_plan_batched, nullptr (the legacy default stream) for the
// *_create forms. Creation synchronises it before returning.
static thread_local cudaStream_t t_setup = nullptr;

struct SetupStream {
  cudaStream_t prev;
  explicit SetupStream(cudaStream_t s) : prev(t_setup) { t_setup = s; }
  ~SetupStream() { t_setup = prev; }
};

template <typename T>
static cudaError_t dalloc(T** p, size_t count, size_t& total) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e == cudaSuccess) total += count * sizeof(T);
  return e;
}

template <typename T>
static cudaError_t upload(T** p, const std::vector<T>& v, size_t& total) {
  cudaError_t e = dalloc(p, v.size(), total);
  if (e != cudaSuccess || v.empty()) return e;
  e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, t_setup);
  return e == cudaSuccess ? cudaStreamSynchronize(t_setup) : e;  // v is the caller's temporary
}

static void free_item(Plan* p) {
  if (!p) return;
  points_free(p->pts);
  void* ptrs[] = {p->d_units,   p->d_zplanes, p->d_zbounds, p->d_nsplit,   p->d_nsplit1, p->d_ext_planes, p->d_pupil,
                  p->d_sz_top,  p->d_sz_bot,  p->d_twx,     p->d_twy,      p->Whi,       p->Wlo,
                  p->Wh,        p->Wt,        p->Bhi,       p->Blo,        p->Cf,        p->S_part,
                  p->T,         p->hio_W,     p->hio_gamma, p->hio_alpha,  p->hio_p,     p->hio_out};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

cudaError_t allow_max_smem(const void* kernel) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first == kernel && d.second == dev) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  // the dynamic limit plus the kernel's static shared memory may not exceed the opt-in maximum
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.push_back({kernel, dev});
  return e;
}

static int round_planes(int nf) {
  static const int slots[] = {8, 16, 24, 32, 64, 128};
  for (int s : slots)
    if (nf <= s) return s;
  return -1;
}

static int device_sms() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// ---------------------------------------------------------------- one item ---
static scw_status validate_desc(const scw_desc* d) {
  if (!d) return set_error(SCW_ERR_INVALID_ARGUMENT, "desc is NULL");
  if (d->U < 1 || d->V < 1 || d->L < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "U, V and L must be >= 1");
  if ((long long)d->U * d->V > kMaxM) return set_error(SCW_ERR_UNSUPPORTED, "U*V exceeds 4096");
  if (d->V > 96) return set_error(SCW_ERR_UNSUPPORTED, "V above 96 (y-pass shared tile)");
  if (!(d->lambda > 0) || !(d->X > 0) || !(d->Y > 0))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "lambda, X and Y must be positive");
  if (d->Fx < 8 || d->Fy < 8 || d->Fx % 8 || d->Fy % 8 || d->Fx > kMaxFx || d->Fy > kMaxFx)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "Fx and Fy must be multiples of 8 in [8, 4096]");
  if (d->Fz < 1 || d->Fz > 65535) return set_error(SCW_ERR_INVALID_ARGUMENT, "Fz must be in [1, 65535]");
  if (d->illuminations < 0 || d->illuminations > 256)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "illuminations must be in [0, 256]");
  if ((long long)std::max(1, d->illuminations) * d->Fz > 65535)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "illuminations * Fz must be <= 65535");
  if (!(d->pupil_na >= 0.0) || !std::isfinite(d->pupil_na))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "pupil_na must be finite and >= 0");
  if (d->tiles_x < 0 || d->tiles_y < 0 || d->tiles_x > 64 || d->tiles_y > 64)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "tiles_x and tiles_y must be in [0, 64]");
  {
    const long long W = (long long)std::max(1, d->tiles_x) * d->Fx, H = (long long)std::max(1, d->tiles_y) * d->Fy;
    const long long ld = d->out_ld ? d->out_ld : W;
    if (d->out_ld < 0 || d->out_plane_stride < 0 || ld < W || (ld & 1))
      return set_error(SCW_ERR_INVALID_ARGUMENT, "out_ld must be even and >= tiles_x Fx");
    if (d->out_plane_stride && (d->out_plane_stride < (H - 1) * ld + W || (d->out_plane_stride & 1)))
      return set_error(SCW_ERR_INVALID_ARGUMENT, "out_plane_stride must be even and hold one plane");
    if ((d->flags & SCW_FLAG_HOST_IO) && (d->out_ld || d->out_plane_stride))
      return set_error(SCW_ERR_UNSUPPORTED, "host IO writes the packed field (no custom pitches)");
  }
  if (!d->z_bounds || !d->z_planes) return set_error(SCW_ERR_INVALID_ARGUMENT, "z_bounds and z_planes are required");
  if (d->precision < SCW_PREC_FP32 || d->precision > SCW_PREC_FP16)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "unknown precision");
  if (d->k_split < 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "k_split must be >= 0");
  for (int l = 0; l < d->L; ++l)
    if (!(d->z_bounds[l + 1] > d->z_bounds[l]))
      return set_error(SCW_ERR_INVALID_ARGUMENT, "z_bounds must be strictly ascending");
  for (int f = 0; f < d->Fz; ++f) {
    if (!std::isfinite(d->z_planes[f])) return set_error(SCW_ERR_INVALID_ARGUMENT, "non-finite z plane");
    if (f && d->z_planes[f] < d->z_planes[f - 1])
      return set_error(SCW_ERR_INVALID_ARGUMENT, "z_planes must be non-decreasing");
  }
  if (!(d->n_top > 0)) return set_error(SCW_ERR_INVALID_ARGUMENT, "n_top must be positive");
  return SCW_OK;
}

scw_status check_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3)
    return set_error(SCW_ERR_CUDA, "libscw is built for sm_103a (GB300); device is sm_" + std::to_string(prop.major) +
                                       std::to_string(prop.minor));
  return SCW_OK;
}

// Plane assignment and the natural plane-slot count of a descriptor.
static scw_status assign_planes(Plan* p, std::vector<int>& ext, int& max_nf) {
  const double z0 = p->z_bounds.front(), zL = p->z_bounds.back();
  p->plane_region.resize(p->Fz);
  for (int f = 0; f < p->Fz; ++f) {
    const double z = p->z_planes[f];
    int r;
    if (z < z0) r = -1;
    else if (z > zL) r = p->L;
    else {  // half-open layers [z_{l-1}, z_l), the last one closed (Sec. 2.6.2)
      r = (int)(std::upper_bound(p->z_bounds.begin(), p->z_bounds.end(), z) - p->z_bounds.begin()) - 1;
      r = std::min(r, p->L - 1);
    }
    p->plane_region[f] = r;
    if (r < 0 || r >= p->L) ext.push_back(f);
  }
  p->n_exterior = (int)ext.size();
  if (p->n_exterior && !(p->flags & SCW_FLAG_EXTERIOR))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "planes outside [z0, zL] need SCW_FLAG_EXTERIOR");
  max_nf = 0;
  for (int f = 0; f < p->Fz;) {  // active layers, split into chunks of at most kMaxPlanesPerLayer planes
    const int r = p->plane_region[f];
    int g = f;
    while (g < p->Fz && p->plane_region[g] == r) ++g;
    if (r >= 0 && r < p->L)
      for (int s = f; s < g; s += kMaxPlanesPerLayer) {
        LayerUnit u{r, s, std::min(kMaxPlanesPerLayer, g - s), 0};
        p->units.push_back(u);
        max_nf = std::max(max_nf, u.nf);
      }
    f = g;
  }
  return SCW_OK;
}

#define SCW_TRY(x)                                   \
  do {                                               \
    cudaError_t _e = (x);                            \
    if (_e != cudaSuccess) return cuda_error(_e, #x); \
  } while (0)

// Tables and every buffer except S_part (whose size depends on the split).
static scw_status build_item(Plan* p, const std::vector<int>& ext) {
  std::vector<double2> szt(p->M), szb(p->M);
  std::vector<float> pupil(p->M, 1.f);
  for (int m = 0; m < p->M; ++m) {
    const int u = m % p->U - p->U / 2, v = m / p->U - p->V / 2;
    const double sx = p->lambda * u / p->X, sy = p->lambda * v / p->Y;
    if (p->pupil_na > 0 && sx * sx + sy * sy > p->pupil_na * p->pupil_na * (1.0 + 1e-12)) pupil[m] = 0.f;
    const auto a = s_z(std::complex<double>(p->n_top, 0.0), sx, sy);
    const auto b = s_z(std::complex<double>(p->n_bot_re, p->n_bot_im), sx, sy);
    szt[m] = make_double2(a.real(), a.imag());
    szb[m] = make_double2(b.real(), b.imag());
  }
  // fold tables: order u at position u mod Up (fold_pos), rows padded to a multiple of 8
  ItemDev& it = p->item;
  std::memset(&it, 0, sizeof(it));
  it.Up = fold_np(p->U);
  it.Vp = fold_np(p->V);
  const int Qx = p->Fx / 8, Qy = p->Fy / 8;
  std::vector<float2> twx((size_t)Qx * it.Up, make_float2(0.f, 0.f)), twy((size_t)Qy * it.Vp, make_float2(0.f, 0.f));
  for (int b = 0; b < Qx; ++b)
    for (int ui = 0; ui < p->U; ++ui) {
      const int u = ui - p->U / 2;
      twx[(size_t)fold_pos(ui, p->U, it.Up) * Qx + b] = cis_cycles((double)u * b / p->Fx + u * p->x0 / p->X);
    }
  for (int b = 0; b < Qy; ++b)
    for (int vi = 0; vi < p->V; ++vi) {
      const int v = vi - p->V / 2;
      twy[(size_t)b * it.Vp + fold_pos(vi, p->V, it.Vp)] = cis_cycles((double)v * b / p->Fy + v * p->y0 / p->Y);
    }
  std::vector<int> ones(p->Fz, 1);
  size_t& tot = p->workspace_bytes;
  const size_t L = p->L, M = p->M;
  const size_t n_units = p->units.size();
  SCW_TRY(upload(&p->d_units, p->units, tot));
  SCW_TRY(upload(&p->d_zplanes, p->z_planes, tot));
  SCW_TRY(upload(&p->d_zbounds, p->z_bounds, tot));
  SCW_TRY(upload(&p->d_nsplit1, ones, tot));
  SCW_TRY(upload(&p->d_ext_planes, ext, tot));
  SCW_TRY(upload(&p->d_sz_top, szt, tot));
  SCW_TRY(upload(&p->d_sz_bot, szb, tot));
  if (p->pupil_na > 0) SCW_TRY(upload(&p->d_pupil, pupil, tot));
  SCW_TRY(upload(&p->d_twx, twx, tot));
  SCW_TRY(upload(&p->d_twy, twy, tot));
  SCW_TRY(dalloc(&p->T, (size_t)p->Fz * 3 * p->V * p->Fx, tot));
  if (n_units > 0) {
    if (p->precision == SCW_PREC_FP32) {
      SCW_TRY(dalloc(&p->Wt, L * 3 * M * 4 * M, tot));
      SCW_TRY(dalloc(&p->Cf, n_units * 4 * M * p->F_pad, tot));
    } else {
      const size_t nk = (8 * M + 63) / 64;
      const size_t nA = L * 3 * M * nk * 64, nB = n_units * nk * p->NB * 64;
      if (p->precision == SCW_PREC_SPLIT_BF16) {
        SCW_TRY(dalloc(&p->Whi, nA, tot));
        SCW_TRY(dalloc(&p->Wlo, nA, tot));
      } else {
        SCW_TRY(dalloc(&p->Wh, nA, tot));
      }
      uint16_t *bh = nullptr, *bl = nullptr;
      SCW_TRY(dalloc(&bh, nB, tot));
      p->Bhi = bh;
      SCW_TRY(dalloc(&bl, nB, tot));
      p->Blo = bl;
      SCW_TRY(cudaMemsetAsync(p->Bhi, 0, nB * 2, t_setup));
      SCW_TRY(cudaMemsetAsync(p->Blo, 0, nB * 2, t_setup));
    }
  }
  if (p->flags & SCW_FLAG_HOST_IO) {
    SCW_TRY(dalloc(&p->hio_W, L * 3 * M * 4 * M, tot));
    SCW_TRY(dalloc(&p->hio_gamma, L * 4 * M, tot));
    SCW_TRY(dalloc(&p->hio_alpha, p->I * L * 4 * M, tot));
    SCW_TRY(dalloc(&p->hio_p, p->I * 9 * M, tot));
    SCW_TRY(dalloc(&p->hio_out, (size_t)3 * p->Fz * p->out_pstride, tot));
  }
  SCW_TRY(cudaEventCreate(&p->ev0));
  SCW_TRY(cudaEventCreate(&p->ev1));
  return SCW_OK;
}

// S_part and the split table for the chosen k_split, then the kernels' view of the item.
static scw_status finish_item(Plan* p) {
  size_t& tot = p->workspace_bytes;
  if (p->S_part) {
    cudaFree(p->S_part);
    p->S_part = nullptr;
  }
  if (p->d_nsplit) {
    cudaFree(p->d_nsplit);
    p->d_nsplit = nullptr;
  }
  const size_t M = p->M;
  // per-unit K splits (the contraction's tasks and the partials the x-pass sums per plane)
  if ((int)p->unit_ks.size() != (int)p->units.size()) p->unit_ks.clear();
  std::vector<int> nsplit(p->Fz, 1);
  int ks_max = 1;
  for (size_t u = 0; u < p->units.size(); ++u) {
    const int ks = p->unit_ks.empty() ? p->k_split : p->unit_ks[u];
    p->units[u].ks = ks;
    ks_max = std::max(ks_max, ks);
    for (int f = p->units[u].f0; f < p->units[u].f0 + p->units[u].nf; ++f) nsplit[f] = ks;
  }
  p->k_split = std::max(p->k_split, ks_max);
  if (!p->units.empty()) {
    SCW_TRY(cudaMemcpyAsync(p->d_units, p->units.data(), p->units.size() * sizeof(LayerUnit), cudaMemcpyHostToDevice,
                            t_setup));
    SCW_TRY(cudaStreamSynchronize(t_setup));
  }
  SCW_TRY(upload(&p->d_nsplit, nsplit, tot));
  const int n_tiles = (3 * p->M + p->rows_tile - 1) / p->rows_tile;
  SCW_TRY(dalloc(&p->S_part, (size_t)p->k_split * p->Fz * 3 * M, tot));
  SCW_TRY(cudaMemsetAsync(p->S_part, 0, (size_t)p->k_split * p->Fz * 3 * M * sizeof(float2), t_setup));
  ItemDev& it = p->item;
  it.units = p->d_units;
  it.zplanes = p->d_zplanes;
  it.zbounds = p->d_zbounds;
  it.gamma = p->gamma;
  it.alpha = p->alpha;
  it.Ahi = p->precision == SCW_PREC_SPLIT_BF16 ? static_cast<const void*>(p->Whi) : static_cast<const void*>(p->Wh);
  it.Alo = p->Wlo;
  it.Bhi = p->Bhi;
  it.Blo = p->Blo;
  it.S_part = p->S_part;
  it.nsplit = p->d_nsplit;
  it.twx = p->d_twx;
  it.twy = p->d_twy;
  it.T = p->T;
  it.split_stride = (size_t)p->Fz * 3 * M;
  it.inv_lam = 1.0 / p->lambda;
  it.M = p->M; it.U = p->U; it.V = p->V; it.Fx = p->Fx; it.Fy = p->Fy; it.Fz = p->Fz;
  it.I = p->I; it.Fz_out = p->Fz_out; it.alpha_istride = (size_t)p->L * 4 * p->M;
  it.tx = p->tiles_x; it.ty = p->tiles_y; it.ld = p->out_ld; it.pstride = p->out_pstride;
  it.F_pad = p->F_pad;
  it.k_split = p->k_split;
  it.n_tiles = n_tiles;
  it.rows_tile = p->rows_tile;
  if (p->flags & SCW_FLAG_DEBUG_BOUNDS) {
    const unsigned long long nk = (8 * M + 63) / 64, Fz = p->Fz, L = p->L, nu = p->units.size();
    unsigned long long* b = p->bnd_real;
    b[BND_S_PART] = (unsigned long long)p->k_split * Fz * 3 * M;
    b[BND_T] = Fz * 3 * p->V * p->Fx;
    b[BND_TWX] = (unsigned long long)fold_np(p->U) * (p->Fx / 8);
    b[BND_TWY] = (unsigned long long)(p->Fy / 8) * fold_np(p->V);
    b[BND_B] = p->precision == SCW_PREC_FP32 ? 0 : nu * nk * p->NB * 64;
    b[BND_GAMMA] = L * 4 * M;
    b[BND_ALPHA] = (unsigned long long)p->I * L * 4 * M;
    b[BND_OUT] = (unsigned long long)((long long)(p->I * 3 * p->Fz_out - 1) * p->out_pstride +
                                      (long long)(p->tiles_y * p->Fy - 1) * p->out_ld + (long long)p->tiles_x * p->Fx);
    b[BND_C] = p->precision == SCW_PREC_FP32 ? nu * 4 * M * p->F_pad : 0;
    b[BND_WT] = p->precision == SCW_PREC_FP32 ? L * 4 * M * 3 * M : 0;
    it.dbg = 1;
    for (int k = 0; k < BND_COUNT; ++k) it.bnd[k] = b[k];
  }
  it.nk = (8 * p->M + 63) / 64;
  it.n_units = (int)p->units.size();
  return SCW_OK;
}

static scw_status create_item(const scw_desc* d, int force_F_pad, Plan** out) {
  *out = nullptr;
  Plan* p = new (std::nothrow) Plan();
  if (!p) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  p->U = d->U; p->V = d->V; p->M = d->U * d->V; p->L = d->L;
  // I illuminations share every plane: plane slot f I + i is output plane f of illumination i
  p->I = std::max(1, d->illuminations);
  p->Fz_out = d->Fz;
  p->Fx = d->Fx; p->Fy = d->Fy; p->Fz = p->I * d->Fz;
  p->pupil_na = d->pupil_na;
  p->tiles_x = std::max(1, d->tiles_x);
  p->tiles_y = std::max(1, d->tiles_y);
  p->out_ld = d->out_ld ? d->out_ld : (long long)p->tiles_x * d->Fx;
  p->out_pstride = d->out_plane_stride ? d->out_plane_stride : (long long)p->tiles_y * d->Fy * p->out_ld;
  p->lambda = d->lambda; p->X = d->X; p->Y = d->Y; p->x0 = d->x0; p->y0 = d->y0;
  p->n_top = d->n_top; p->n_bot_re = d->n_bot_re; p->n_bot_im = d->n_bot_im; p->z_inc = d->z_inc;
  p->precision = d->precision; p->flags = d->flags;
  p->z_bounds.assign(d->z_bounds, d->z_bounds + d->L + 1);
  p->z_planes.clear();
  for (int f = 0; f < d->Fz; ++f)
    for (int i = 0; i < p->I; ++i) p->z_planes.push_back(d->z_planes[f]);
  std::vector<int> ext;
  int max_nf = 0;
  scw_status s = assign_planes(p, ext, max_nf);
  if (s != SCW_OK) {
    free_item(p);
    return s;
  }
  p->F_pad = std::max({8, round_planes(std::max(max_nf, 1)), force_F_pad});
  p->NB = 2 * p->F_pad;
  p->k_split = std::max(1, d->k_split);
  s = build_item(p, ext);
  if (s != SCW_OK) {
    free_item(p);
    return s;
  }
  *out = p;
  return SCW_OK;
}

// ------------------------------------------------------- contraction schedule ---
struct TaskCost {
  double cost;
  int4 t;
};

// Tasks of one item; uks (optional) gives each unit its own K split instead of ks.
static void item_tasks(const Plan* p, int item, int ks, std::vector<TaskCost>& out,
                       const std::vector<int>* uks = nullptr) {
  const int nk = (8 * p->M + 63) / 64;
  const int tiles = (3 * p->M + p->rows_tile - 1) / p->rows_tile;
  for (int u = 0; u < (int)p->units.size(); ++u) {
    const int k = uks ? (*uks)[u] : ks;
    const int per = (nk + k - 1) / k;
    for (int t = 0; t < tiles; ++t)
      for (int s = 0; s < k; ++s) {
        const int kc = std::max(0, std::min(nk, s * per + per) - s * per);
        out.push_back({kc + 2.0, make_int4(item, u, t, s)});  // +2 stages: epilogue and hand-off
      }
  }
}

// Longest-processing-time-first assignment of tasks to G persistent CTAs.
static void lpt(std::vector<TaskCost>& tasks, int G, std::vector<int>& cta_off, std::vector<int4>& order,
                double& max_load, double& mean_load) {
  std::stable_sort(tasks.begin(), tasks.end(), [](const TaskCost& a, const TaskCost& b) { return a.cost > b.cost; });
  using E = std::pair<double, int>;
  std::priority_queue<E, std::vector<E>, std::greater<E>> heap;
  for (int g = 0; g < G; ++g) heap.push({0.0, g});
  std::vector<std::vector<int4>> per(G);
  for (const auto& tc : tasks) {
    E e = heap.top();
    heap.pop();
    per[e.second].push_back(tc.t);
    heap.push({e.first + tc.cost, e.second});
  }
  max_load = 0;
  double sum = 0;
  while (!heap.empty()) {
    max_load = std::max(max_load, heap.top().first);
    sum += heap.top().first;
    heap.pop();
  }
  mean_load = G ? sum / G : 0;
  cta_off.assign(G + 1, 0);
  order.clear();
  for (int g = 0; g < G; ++g) {
    cta_off[g] = (int)order.size();
    order.insert(order.end(), per[g].begin(), per[g].end());
  }
  cta_off[G] = (int)order.size();
}

static int schedule_grid(int n_tasks, int NB, bool bf16, int ctas_per_sm = 0) {
  const int cps = ctas_per_sm > 0 ? std::min(ctas_per_sm, tc_ctas_per_sm(NB, bf16)) : tc_ctas_per_sm(NB, bf16);
  return std::max(1, std::min(n_tasks, device_sms() * cps));
}

// Makespan (in K-stages) of a set of per-item splits under LPT.
static double model_makespan(const std::vector<Plan*>& items, const std::vector<int>& ks, int NB, bool bf16) {
  std::vector<TaskCost> t;
  for (size_t i = 0; i < items.size(); ++i) item_tasks(items[i], (int)i, ks[i], t);
  if (t.empty()) return 0;
  std::vector<int> off;
  std::vector<int4> order;
  double mx, mean;
  lpt(t, schedule_grid((int)t.size(), NB, bf16), off, order, mx, mean);
  return mx;
}

// Schedule of the tasks of every item, or (unit_begin < unit_end) only of those
// units of item 0; ctas_per_sm > 0 caps the persistent grid per SM.
// SCW_FLAG_DEBUG_BOUNDS: the ranges a contraction task's bulk copies and epilogue stores cover, as the
// kernel derives them (task_geom), against the buffers' allocations.
static scw_status check_task_ranges(const Plan* p, const int4& tk) {
  const int R = 3 * p->M, nk = (8 * p->M + 63) / 64;
  const LayerUnit& u = p->units[tk.y];
  const int ks = u.ks > 0 ? u.ks : p->k_split;
  const int per = (nk + ks - 1) / ks;
  const int kb = tk.w * per, kcount = std::max(0, std::min(nk, kb + per) - kb);
  const int rt = std::min(p->rows_tile, R - p->rows_tile * tk.z);
  const size_t a_end = (size_t)u.layer * R * nk * 64 + (size_t)tk.z * p->rows_tile * nk * 64 + (size_t)(kb + kcount) * rt * 64;
  const size_t b_end = ((size_t)tk.y * nk + kb + kcount) * p->NB * 64;
  const size_t s_end = ((size_t)tk.w * p->Fz + u.f0 + u.nf - 1) * R + (size_t)p->rows_tile * tk.z + rt;
  std::string why;
  if (rt <= 0 || tk.w >= ks || u.layer < 0 || u.layer >= p->L) why = "its row tile, split or layer";
  else if (a_end > (size_t)p->L * R * nk * 64) why = "W";
  else if (b_end > p->units.size() * (size_t)nk * p->NB * 64) why = "the B operand";
  else if (s_end > (size_t)p->k_split * p->Fz * R) why = "the partial spectra";
  if (why.empty()) return SCW_OK;
  return set_error(SCW_ERR_BOUNDS, "contraction task (unit " + std::to_string(tk.y) + ", tile " + std::to_string(tk.z) +
                                       ", split " + std::to_string(tk.w) + ") would reach outside " + why);
}

static scw_status upload_schedule(const std::vector<Plan*>& items, int NB, bool bf16, TcSchedule& s,
                                  int ctas_per_sm = 0, int unit_begin = 0, int unit_end = 0) {
  std::vector<TaskCost> t;
  for (size_t i = 0; i < items.size(); ++i)
    item_tasks(items[i], (int)i, items[i]->k_split, t, items[i]->unit_ks.empty() ? nullptr : &items[i]->unit_ks);
  if (unit_begin < unit_end) {
    std::vector<TaskCost> keep;
    for (const auto& tc : t)
      if (tc.t.y >= unit_begin && tc.t.y < unit_end) keep.push_back(tc);
    t.swap(keep);
  }
  if (s.d_tasks) cudaFree(s.d_tasks);
  if (s.d_cta_off) cudaFree(s.d_cta_off);
  s.d_tasks = nullptr;
  s.d_cta_off = nullptr;
  s.n_tasks = (int)t.size();
  if (t.empty()) {
    s.grid = 0;
    return SCW_OK;
  }
  for (const auto& tc : t)
    if (items[tc.t.x]->flags & SCW_FLAG_DEBUG_BOUNDS) {
      scw_status st = check_task_ranges(items[tc.t.x], tc.t);
      if (st != SCW_OK) return st;
    }
  s.grid = schedule_grid(s.n_tasks, NB, bf16, ctas_per_sm);
  std::vector<int> off;
  std::vector<int4> order;
  lpt(t, s.grid, off, order, s.max_load, s.mean_load);
  size_t tot = 0;
  SCW_TRY(upload(&s.d_tasks, order, tot));
  SCW_TRY(upload(&s.d_cta_off, off, tot));
  return SCW_OK;
}

// k_split per item from a target number of K-stages per task.
static std::vector<int> splits_for_target(const std::vector<Plan*>& items, int target) {
  std::vector<int> ks;
  for (auto* p : items) {
    const int nk = (8 * p->M + 63) / 64;
    ks.push_back(std::max(1, std::min(16, (nk + target / 2) / target)));
  }
  return ks;
}

// FP32 path: ~4 waves of work units and a shared-memory slice of C <= 96 KB per CTA.
static int fp32_split(const Plan* p) {
  const int K = 4 * p->M;
  const int slots = device_sms() * 2 * 4;
  const int per_split_units = (int)p->units.size() * ((3 * p->M + 255) / 256);
  int ks = per_split_units ? (slots + per_split_units - 1) / per_split_units : 1;
  ks = std::max(1, std::min(ks, std::max(1, K / 128)));
  const int fch = p->F_pad >= 16 ? 16 : 8;
  ks = std::max(ks, (int)(((size_t)K * fch * 8 + 96 * 1024 - 1) / (96 * 1024)));
  return std::min(ks, K);
}

}  // namespace scw

using namespace scw;

// ------------------------------------------------------------------ the plan ---
struct scw_plan_s {
  std::vector<Plan*> items;
  bool batched = false;
  int precision = 0;
  bool tc = false, bf16 = false;
  int NB = 16, F_pad = 8;
  uint64_t timeout_ns = 2000000000ull;
  int* d_err = nullptr;
  // tables over all items
  ItemDev* d_items = nullptr;      // batched plans only
  int2* d_unit_entries = nullptr;
  int n_unit_entries = 0;
  int2* d_plane_entries = nullptr;  // y-pass-pair class first (ypass_pairs), then the rest
  int n_plane_entries = 0;
  int n_pair_entries = 0;
  bool tiled = false;  // some item stores periodic tiles
  int max_twy = 0;     // largest y fold-twiddle table (complex elements)
  int inject_stall = 0;            // scw_plan_inject_stall (tests of the timeout path)
  unsigned long long* d_trace = nullptr;  // kernel trace stamps (scw_plan_enable_trace), or null
  TcSchedule sched;
  float2** d_outs = nullptr;
  float2** h_outs = nullptr;       // pinned
  int max_M = 0, max_Qx = 0, max_V = 0, max_Vp = 0;
  size_t xpass_smem = 0;
  size_t rec_smem = 0;
  // graph replay
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* graph_key = nullptr;
  bool direct_done = false;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> tev;
  size_t tev_used = 0;
  int kernels_per_synthesis = 0;
  std::string tune_report;
  // layer-group pipelining (single tensor-core plans): group g's recompose runs on
  // st2 while group g+1 is contracted on the caller's stream
  int groups = 1;
  std::vector<TcSchedule> gsched;
  std::vector<int> gplane;          // [groups + 1] offsets into the plane entries
  cudaStream_t st2 = nullptr;
  std::vector<cudaEvent_t> gev;     // contraction of group g done
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // host-IO pipeline (scw_synthesize_host on tensor-core plans): per layer group g the copy of
  // its W on st_in, its conversion and synthesis on the caller's stream, and the copy of its
  // planes of the field on st_out, so that both copy directions overlap each other and the kernels
  int hgroups = 0;
  std::vector<TcSchedule> hsched;
  std::vector<int> hplane, hunit, hlayer;  // [hgroups + 1] offsets: plane slots, units, layers
  cudaStream_t st_in = nullptr, st_out = nullptr;
  std::vector<cudaEvent_t> hev_in, hev_comp;
  cudaEvent_t hev_start = nullptr, hev_small = nullptr, hev_out = nullptr;
};

static void free_plan(scw_plan_t P) {
  if (!P) return;
  for (auto* p : P->items) free_item(p);
  void* ptrs[] = {P->d_err, P->d_items, P->d_unit_entries, P->d_plane_entries, P->sched.d_tasks,
                  P->sched.d_cta_off, P->d_outs, P->d_trace};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (P->h_outs) cudaFreeHost(P->h_outs);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  for (cudaEvent_t ev : P->tev) cudaEventDestroy(ev);
  for (auto& g : P->gsched) {
    if (g.d_tasks) cudaFree(g.d_tasks);
    if (g.d_cta_off) cudaFree(g.d_cta_off);
  }
  for (cudaEvent_t ev : P->gev) cudaEventDestroy(ev);
  for (auto& g : P->hsched) {
    if (g.d_tasks) cudaFree(g.d_tasks);
    if (g.d_cta_off) cudaFree(g.d_cta_off);
  }
  for (cudaEvent_t ev : P->hev_in) cudaEventDestroy(ev);
  for (cudaEvent_t ev : P->hev_comp) cudaEventDestroy(ev);
  for (cudaEvent_t ev : {P->hev_start, P->hev_small, P->hev_out})
    if (ev) cudaEventDestroy(ev);
  if (P->st_in) cudaStreamDestroy(P->st_in);
  if (P->st_out) cudaStreamDestroy(P->st_out);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->st2) cudaStreamDestroy(P->st2);
  delete P;
}

static void invalidate_graph(scw_plan_t P) {
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  P->gexec = nullptr;
  P->graph_key = nullptr;
  P->direct_done = false;
}

static scw_status upload_items(scw_plan_t P, cudaStream_t st) {
  if (!P->batched) return SCW_OK;
  std::vector<ItemDev> h(P->items.size());
  for (size_t i = 0; i < P->items.size(); ++i) h[i] = P->items[i]->item;
  cudaError_t e = cudaMemcpyAsync(P->d_items, h.data(), h.size() * sizeof(ItemDev), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "uploading item descriptors");
  e = cudaStreamSynchronize(st);  // h is a local copy
  if (e != cudaSuccess) return cuda_error(e, "uploading item descriptors");
  return SCW_OK;
}

// Event slot k of the current timed call (nullptr when timing is off).
static constexpr int kMarks = 5;  // events per timed call: before (a), (b), x-pass, y-pass; after

static cudaEvent_t timing_event(scw_plan_t P, int k) {
  if (!P->timing) return nullptr;
  const size_t i = P->tev_used + (size_t)k;
  if (i >= kMarks * 4096) return nullptr;
  while (P->tev.size() <= i) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    P->tev.push_back(ev);
  }
  return P->tev[i];
}

static void mark(scw_plan_t P, int k, cudaStream_t st, bool marks) {
  if (!marks) return;
  cudaEvent_t ev = timing_event(P, k);
  if (ev) cudaEventRecord(ev, st);
}

// Steps (a) and (b) for every item.
static scw_status enqueue_spectrum(scw_plan_t P, cudaStream_t st, bool marks, int& n) {
  cudaError_t e;
  const ItemDev& one = P->items[0]->item;
  const ItemDev* items = P->batched ? P->d_items : nullptr;
  mark(P, 0, st, marks);
  if (P->tc) {
    e = launch_phases_tc(one, items, P->d_unit_entries, P->n_unit_entries, P->max_M, P->F_pad, P->bf16, st);
    if (e != cudaSuccess) return cuda_error(e, "phase kernel launch");
    if (P->n_unit_entries) ++n;
  } else {
    for (auto* p : P->items)
      if (!p->units.empty()) {
        e = launch_phases_fp32(*p, st);
        if (e != cudaSuccess) return cuda_error(e, "phase kernel launch");
        ++n;
      }
  }
  for (auto* p : P->items)
    if (p->n_exterior) {
      e = launch_exterior(*p, st);
      if (e != cudaSuccess) return cuda_error(e, "exterior kernel launch");
      ++n;
    }
  mark(P, 1, st, marks);
  if (P->tc) {
    e = launch_contract_tc(one, items, P->sched, P->NB, P->bf16, P->d_err, P->timeout_ns, P->inject_stall, st);
    if (e != cudaSuccess) return cuda_error(e, "contraction kernel launch");
    if (P->sched.n_tasks) ++n;
  } else {
    for (auto* p : P->items)
      if (!p->units.empty()) {
        e = launch_contract_fp32(*p, st);
        if (e != cudaSuccess) return cuda_error(e, "contraction kernel launch");
        ++n;
      }
  }
  return SCW_OK;
}

// Pipelined order: phases, then per group g the contraction of g on `st` and
// the recompose of g on st2 once that contraction is done; st2 joins `st` at
// the end. Groups cover disjoint units and plane ranges, so nothing is shared
// between the overlapping kernels.
static scw_status enqueue_pipelined(scw_plan_t P, float2* out_one, cudaStream_t st, int& n) {
  n = 0;
  cudaError_t e;
  Plan* p = P->items[0];
  const ItemDev& one = p->item;
  e = launch_phases_tc(one, nullptr, P->d_unit_entries, P->n_unit_entries, P->max_M, P->F_pad, P->bf16, st);
  if (e != cudaSuccess) return cuda_error(e, "phase kernel launch");
  ++n;
  if (p->n_exterior) {
    e = launch_exterior(*p, st);
    if (e != cudaSuccess) return cuda_error(e, "exterior kernel launch");
    ++n;
  }
  e = cudaEventRecord(P->ev_fork, st);  // st2 must not start before the previous step ended on st
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  e = cudaStreamWaitEvent(P->st2, P->ev_fork, 0);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
  for (int g = 0; g < P->groups; ++g) {
    e = launch_contract_tc(one, nullptr, P->gsched[g], P->NB, P->bf16, P->d_err, P->timeout_ns, P->inject_stall, st);
    if (e != cudaSuccess) return cuda_error(e, "contraction kernel launch");
    if (P->gsched[g].n_tasks) ++n;
    e = cudaEventRecord(P->gev[g], st);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    e = cudaStreamWaitEvent(P->st2, P->gev[g], 0);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
    const int nb = P->gplane[g + 1] - P->gplane[g];
    if (nb == 0) continue;
    const int2* ent = P->d_plane_entries + P->gplane[g];
    e = launch_xpass(one, nullptr, ent, nb, P->xpass_smem, P->st2);
    if (e != cudaSuccess) return cuda_error(e, "x-pass launch");
    int ny = 0;
    e = launch_ypass(one, nullptr, ent, nb, ypass_pairs(one.Vp) ? nb : 0, P->max_Qx, P->max_Vp, P->max_twy, P->tiled, out_one, nullptr,
                     P->st2, &ny);
    if (e != cudaSuccess) return cuda_error(e, "y-pass launch");
    n += 1 + ny;
  }
  e = cudaEventRecord(P->ev_join, P->st2);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  e = cudaStreamWaitEvent(st, P->ev_join, 0);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
  return SCW_OK;
}

static scw_status enqueue_synthesis(scw_plan_t P, float2* out_one, cudaStream_t st, bool marks, int& n) {
  if (P->groups > 1 && !marks) return enqueue_pipelined(P, out_one, st, n);
  n = 0;
  scw_status s = enqueue_spectrum(P, st, marks, n);
  if (s != SCW_OK) return s;
  const ItemDev& one = P->items[0]->item;
  const ItemDev* items = P->batched ? P->d_items : nullptr;
  mark(P, 2, st, marks);
  cudaError_t e = launch_xpass(one, items, P->d_plane_entries, P->n_plane_entries, P->xpass_smem, st);
  if (e != cudaSuccess) return cuda_error(e, "x-pass launch");
  mark(P, 3, st, marks);
  int ny = 0;
  e = launch_ypass(one, items, P->d_plane_entries, P->n_plane_entries, P->n_pair_entries, P->max_Qx, P->max_Vp, P->max_twy, P->tiled,
                   out_one, P->d_outs, st, &ny);
  if (e != cudaSuccess) return cuda_error(e, "y-pass launch");
  mark(P, 4, st, marks);
  n += 1 + ny;
  if (marks && P->timing && P->tev_used + kMarks <= P->tev.size()) P->tev_used += kMarks;
  return SCW_OK;
}

// Timed launches go out directly (with events between kernels); otherwise the
// first call for a given output launches directly and captures the same
// sequence into a CUDA graph, later calls replay the graph.
static scw_status run_synthesis(scw_plan_t P, float2* out_one, cudaStream_t st) {
  int n = 0;
  if (P->timing) {
    scw_status s = enqueue_synthesis(P, out_one, st, true, n);
    P->kernels_per_synthesis = n;
    return s;
  }
  const void* key = P->batched ? static_cast<const void*>(P->d_outs) : static_cast<const void*>(out_one);
  if (P->gexec && P->graph_key == key) {
    cudaError_t e = cudaGraphLaunch(P->gexec, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
    return SCW_OK;
  }
  scw_status s = enqueue_synthesis(P, out_one, st, false, n);
  if (s != SCW_OK) return s;
  P->kernels_per_synthesis = n;
  invalidate_graph(P);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
  s = enqueue_synthesis(P, out_one, P->cap_stream, false, n);
  e = cudaStreamEndCapture(P->cap_stream, &g);
  if (s != SCW_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&P->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    P->gexec = nullptr;
    return cuda_error(e, "cudaGraphInstantiate");
  }
  P->graph_key = key;
  return SCW_OK;
}

// Choose the contraction splits: a makespan model over targets of K-stages per
// task, then (SCW_FLAG_AUTOTUNE) timing of the best model candidates on the
// device; the choice is cached per device, order counts, plane slots and precision.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

static scw_status choose_splits(scw_plan_t P, bool timed, const std::vector<int>& user_ks) {
  if (!P->tc) {
    for (size_t i = 0; i < P->items.size(); ++i) {
      Plan* p = P->items[i];
      p->k_split = user_ks[i] > 0 ? user_ks[i] : fp32_split(p);
      scw_status s = finish_item(p);
      if (s != SCW_OK) return s;
    }
    return SCW_OK;
  }
  for (auto* p : P->items) p->unit_ks.clear();
  bool all_user = true;
  for (int k : user_ks) all_user = all_user && k > 0;
  std::vector<int> best_ks;
  if (all_user) {
    best_ks = user_ks;
  } else {
    static const int targets[] = {4, 6, 8, 10, 12, 16, 24, 32, 48, 64};
    std::vector<std::pair<double, int>> cand;
    for (int T : targets) {
      auto ks = splits_for_target(P->items, T);
      double ms = model_makespan(P->items, ks, P->NB, P->bf16);
      int ntask = 0;
      for (size_t i = 0; i < ks.size(); ++i) ntask += ks[i];
      cand.push_back({ms * (1.0 + 1e-6 * ntask), T});
    }
    std::sort(cand.begin(), cand.end());
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    std::string key = std::string(prop.name) + "|" + std::to_string(P->NB) + "|" + std::to_string(P->bf16);
    for (auto* p : P->items) key += "|" + std::to_string(p->M) + "x" + std::to_string(p->units.size());
    int chosen = cand.front().second;
    bool cached = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto itc = g_tune_cache.find(key);
      if (itc != g_tune_cache.end()) {
        chosen = itc->second;
        cached = true;
      }
    }
    P->tune_report = "model: T=" + std::to_string(cand.front().second) + " makespan " +
                     std::to_string(cand.front().first);
    if (timed && !cached) {
      // time the three best model candidates with the real kernel on the plan's buffers
      const int n_try = std::min<int>(3, (int)cand.size());
      float best_ms = 1e30f;
      cudaStream_t ts = t_setup ? t_setup : P->cap_stream;
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      for (int c = 0; c < n_try; ++c) {
        const int T = cand[c].second;
        auto ks = splits_for_target(P->items, T);
        for (size_t i = 0; i < P->items.size(); ++i) {
          P->items[i]->k_split = ks[i];
          scw_status s = finish_item(P->items[i]);
          if (s != SCW_OK) return s;
        }
        scw_status s = upload_items(P, ts);
        if (s != SCW_OK) return s;
        s = upload_schedule(P->items, P->NB, P->bf16, P->sched);
        if (s != SCW_OK) return s;
        const ItemDev* items = P->batched ? P->d_items : nullptr;
        launch_contract_tc(P->items[0]->item, items, P->sched, P->NB, P->bf16, P->d_err, P->timeout_ns, 0, ts);
        cudaEventRecord(a, ts);
        for (int r = 0; r < 3; ++r)
          launch_contract_tc(P->items[0]->item, items, P->sched, P->NB, P->bf16, P->d_err, P->timeout_ns, 0, ts);
        cudaEventRecord(b, ts);
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) return cuda_error(e, "autotune timing");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        P->tune_report += "; T=" + std::to_string(T) + " " + std::to_string(ms / 3) + " ms";
        if (ms < best_ms) {
          best_ms = ms;
          chosen = T;
        }
      }
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaMemsetAsync(P->d_err, 0, sizeof(int), ts);
      cudaStreamSynchronize(ts);
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune_cache[key] = chosen;
    }
    best_ks = splits_for_target(P->items, chosen);
    for (size_t i = 0; i < P->items.size(); ++i)
      if (user_ks[i] > 0) best_ks[i] = user_ks[i];
    P->tune_report += "; chosen T=" + std::to_string(chosen) + (cached ? " (cached)" : "");
  }
  // A single plan's tasks rarely divide evenly over the persistent CTAs. Mixing two neighbouring
  // splits over the units (x units with b = a + 1, the rest with a) gives LPT tasks of two sizes
  // to pack; keep the mix whose modelled makespan is lowest (ties: the uniform split).
  if (!P->batched && user_ks[0] <= 0 && !P->items[0]->units.empty()) {
    Plan* p = P->items[0];
    const int k = best_ks[0], nu = (int)p->units.size();
    auto makespan = [&](const std::vector<int>& uks) {
      std::vector<TaskCost> t;
      item_tasks(p, 0, k, t, &uks);
      std::vector<int> off;
      std::vector<int4> order;
      double mx = 0, mean = 0;
      lpt(t, schedule_grid((int)t.size(), P->NB, P->bf16), off, order, mx, mean);
      return mx;
    };
    std::vector<int> best(nu, k);
    double best_ms = makespan(best);
    const int step = std::max(1, nu / 64);
    for (int a = std::max(1, k - 1); a <= k; ++a)
      for (int x = 0; x <= nu; x += step) {
        std::vector<int> uks(nu);
        for (int u = 0; u < nu; ++u) uks[u] = u < x ? a + 1 : a;
        const double ms = makespan(uks);
        if (ms < best_ms - 1e-9) {
          best_ms = ms;
          best = uks;
        }
      }
    if (best != std::vector<int>(nu, k)) {
      p->unit_ks = best;
      P->tune_report += "; unit splits mixed (modelled makespan " + std::to_string(best_ms) + ")";
    }
  }
  for (size_t i = 0; i < P->items.size(); ++i) {
    P->items[i]->k_split = best_ks[i];
    scw_status s = finish_item(P->items[i]);
    if (s != SCW_OK) return s;
  }
  return upload_schedule(P->items, P->NB, P->bf16, P->sched);
}

// Shared tail of single and batched plan creation.
static scw_status finish_plan(scw_plan_t P, const std::vector<int>& user_ks, bool timed) {
  size_t tot = 0;
  SCW_TRY(dalloc(&P->d_err, 1, tot));
  SCW_TRY(cudaMemsetAsync(P->d_err, 0, sizeof(int), t_setup));
  SCW_TRY(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  for (auto* p : P->items) p->item.err = P->d_err;  // debug-path reports (finish_item keeps it)
  std::vector<int2> ue, pe;
  for (size_t i = 0; i < P->items.size(); ++i) {
    Plan* p = P->items[i];
    for (int u = 0; u < (int)p->units.size(); ++u) ue.push_back(make_int2((int)i, u));
    for (int f = 0; f < p->Fz; ++f) pe.push_back(make_int2((int)i, f));
    P->max_M = std::max(P->max_M, p->M);
    P->max_Qx = std::max(P->max_Qx, p->Fx / 8);
    P->max_V = std::max(P->max_V, p->V);
    P->xpass_smem = std::max(P->xpass_smem, xpass_smem_bytes(p->V, p->item.Up, p->Fx));
    P->max_Vp = std::max(P->max_Vp, p->item.Vp);
    P->rec_smem = std::max(P->rec_smem, recompose_smem_bytes(p->V, p->item.Up, p->item.Vp));
    P->tiled = P->tiled || p->tiles_x > 1 || p->tiles_y > 1;
    P->max_twy = std::max(P->max_twy, (p->Fy / 8) * p->item.Vp);
  }
  // plane entries of items with long y folds first: they run the two-residue y-pass
  std::stable_partition(pe.begin(), pe.end(),
                        [&](const int2& en) { return ypass_pairs(P->items[en.x]->item.Vp); });
  P->n_pair_entries = 0;
  for (const int2& en : pe) P->n_pair_entries += ypass_pairs(P->items[en.x]->item.Vp) ? 1 : 0;
  P->n_unit_entries = (int)ue.size();
  P->n_plane_entries = (int)pe.size();
  SCW_TRY(upload(&P->d_unit_entries, ue, tot));
  SCW_TRY(upload(&P->d_plane_entries, pe, tot));
  SCW_TRY(dalloc(&P->d_outs, P->items.size(), tot));
  SCW_TRY(cudaMallocHost(reinterpret_cast<void**>(&P->h_outs), P->items.size() * sizeof(float2*)));
  if (P->batched) SCW_TRY(dalloc(&P->d_items, P->items.size(), tot));
  scw_status s = choose_splits(P, timed, user_ks);
  if (s != SCW_OK) return s;
  s = upload_items(P, t_setup ? t_setup : P->cap_stream);
  if (s != SCW_OK) return s;
  cudaError_t e = cudaStreamSynchronize(t_setup);
  return e == cudaSuccess ? SCW_OK : cuda_error(e, "plan set-up stream");
}

static scw_status check_item_index(scw_plan_t P, int item) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (item < 0 || item >= (int)P->items.size()) return set_error(SCW_ERR_INVALID_ARGUMENT, "item index out of range");
  return SCW_OK;
}

// W into the chosen precision's layout (transposed FP32, or tile-major swizzled 16-bit).
static cudaError_t convert_w(Plan* p, const float2* w, cudaStream_t st) {
  if (p->precision == SCW_PREC_FP32) return launch_transpose_layers(w, p->Wt, p->L, 3 * p->M, 4 * p->M, st);
  if (p->precision == SCW_PREC_SPLIT_BF16)
    return launch_convert_tiled(w, p->Whi, p->Wlo, p->L, p->M, p->rows_tile, true, st);
  return launch_convert_tiled(w, p->Wh, nullptr, p->L, p->M, p->rows_tile, false, st);
}

// Conversion of layers [lb, le) of W (tensor-core plans; the tiled layout is contiguous per layer).
static cudaError_t convert_w_layers(Plan* p, const float2* w, int lb, int le, cudaStream_t st) {
  const size_t M = p->M, R = 3 * M, nk = (8 * M + 63) / 64;
  const size_t in_off = (size_t)lb * R * 4 * M, out_off = (size_t)lb * R * nk * 64;
  if (p->precision == SCW_PREC_SPLIT_BF16)
    return launch_convert_tiled(w + in_off, p->Whi + out_off, p->Wlo + out_off, le - lb, p->M, p->rows_tile, true, st);
  return launch_convert_tiled(w + in_off, p->Wh + out_off, nullptr, le - lb, p->M, p->rows_tile, false, st);
}

// Groups of the host-IO pipeline: contiguous units, the layers they span and their plane slots.
static scw_status host_groups(scw_plan_t P) {
  if (P->hgroups) return SCW_OK;
  Plan* p = P->items[0];
  const int nu = (int)p->units.size();
  const int G = std::max(1, std::min(8, nu));
  P->hsched.resize(G);
  P->hplane.assign(G + 1, 0);
  P->hunit.assign(G + 1, 0);
  P->hlayer.assign(G + 1, 0);
  // boundaries between layers only (a layer with more plane slots than one work unit holds spans
  // several units, which stay in one group: its W is converted once, by that group)
  int ub = 0;
  for (int g = 0; g < G; ++g) {
    int ue = (g + 1 < G) ? std::max(ub, (int)((long long)nu * (g + 1) / G)) : nu;
    while (ue < nu && ue > 0 && p->units[ue].layer == p->units[ue - 1].layer) ++ue;
    if (ue > ub) {  // (an empty range would mean "every unit" to upload_schedule)
      scw_status s = upload_schedule(P->items, P->NB, P->bf16, P->hsched[g], 0, ub, ue);
      if (s != SCW_OK) return s;
    }
    P->hunit[g + 1] = ue;
    P->hplane[g + 1] = (ue < nu) ? p->units[ue].f0 : p->Fz;
    P->hlayer[g + 1] = (ue < nu) ? p->units[ue].layer : p->L;
    ub = ue;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&P->st_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->st_out, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&P->hev_start, &P->hev_small, &P->hev_out})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  P->hev_in.assign(G, nullptr);
  P->hev_comp.assign(G, nullptr);
  for (int g = 0; g < G && e == cudaSuccess; ++g) {
    e = cudaEventCreateWithFlags(&P->hev_in[g], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->hev_comp[g], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return cuda_error(e, "host pipeline streams");
  P->hgroups = G;
  return SCW_OK;
}

static scw_status set_layers_item(scw_plan_t P, int idx, const void* W, const void* gamma, const void* alpha,
                                  const void* p_inc, const void* p_ref, const void* p_trn, cudaStream_t st);

// scw_synthesize_host on tensor-core plans: layer group g's W goes in on st_in while group g-1 is
// converted and synthesised on `st` and group g-2's planes of the field come back on st_out.
static scw_status synthesize_host_pipelined(scw_plan_t P, const void* W, const void* gamma, const void* alpha,
                                            const void* const* pio, void* out, cudaStream_t st) {
  Plan* p = P->items[0];
  scw_status s = host_groups(P);
  if (s != SCW_OK) return s;
  const int G = P->hgroups;
  const size_t L = p->L, M = p->M, wl = 3 * M * 4 * M;  // complex elements of W per layer
  const float2* Wh = static_cast<const float2*>(W);
  cudaError_t e;
#define SCW_TRY_E(x, what)                          \
  do {                                              \
    e = (x);                                        \
    if (e != cudaSuccess) return cuda_error(e, what); \
  } while (0)
  SCW_TRY_E(cudaEventRecord(P->hev_start, st), "cudaEventRecord");
  SCW_TRY_E(cudaStreamWaitEvent(P->st_in, P->hev_start, 0), "cudaStreamWaitEvent");
  SCW_TRY_E(cudaStreamWaitEvent(P->st_out, P->hev_start, 0), "cudaStreamWaitEvent");
  SCW_TRY_E(cudaMemcpyAsync(p->hio_gamma, gamma, L * 4 * M * sizeof(double2), cudaMemcpyHostToDevice, P->st_in),
            "cudaMemcpyAsync");
  SCW_TRY_E(cudaMemcpyAsync(p->hio_alpha, alpha, p->I * L * 4 * M * sizeof(double2), cudaMemcpyHostToDevice, P->st_in),
            "cudaMemcpyAsync");
  const double2 *pi = nullptr, *pr = nullptr, *pt = nullptr;
  if (pio[0] && pio[1] && pio[2]) {
    const size_t np = (size_t)p->I * 3 * M;
    for (int k = 0; k < 3; ++k)
      SCW_TRY_E(cudaMemcpyAsync(p->hio_p + k * np, pio[k], np * sizeof(double2), cudaMemcpyHostToDevice, P->st_in),
                "cudaMemcpyAsync");
    pi = p->hio_p; pr = p->hio_p + np; pt = p->hio_p + 2 * np;
  }
  SCW_TRY_E(cudaEventRecord(P->hev_small, P->st_in), "cudaEventRecord");
  for (int g = 0; g < G; ++g) {
    const size_t lb = P->hlayer[g], le = P->hlayer[g + 1];
    SCW_TRY_E(cudaMemcpyAsync(p->hio_W + lb * wl, Wh + lb * wl, (le - lb) * wl * sizeof(float2),
                              cudaMemcpyHostToDevice, P->st_in), "cudaMemcpyAsync");
    SCW_TRY_E(cudaEventRecord(P->hev_in[g], P->st_in), "cudaEventRecord");
  }
  // the layers point at the plan's own device copies (attached once, without converting here)
  if (!p->layers_set || p->gamma != p->hio_gamma || p->p_inc != pi) {
    p->gamma = p->hio_gamma; p->alpha = p->hio_alpha;
    p->p_inc = pi; p->p_ref = pr; p->p_trn = pt;
    p->item.gamma = p->gamma; p->item.alpha = p->alpha;
    p->layers_set = true;
    invalidate_graph(P);
  }
  const ItemDev& one = p->item;
  SCW_TRY_E(cudaStreamWaitEvent(st, P->hev_small, 0), "cudaStreamWaitEvent");
  if (p->n_exterior) SCW_TRY_E(launch_exterior(*p, st), "exterior kernel launch");
  const size_t slice = (size_t)p->out_pstride;  // complex elements per output plane
  for (int g = 0; g < G; ++g) {
    SCW_TRY_E(cudaStreamWaitEvent(st, P->hev_in[g], 0), "cudaStreamWaitEvent");
    if (P->hlayer[g + 1] > P->hlayer[g])
      SCW_TRY_E(convert_w_layers(p, p->hio_W, P->hlayer[g], P->hlayer[g + 1], st), "W conversion launch");
    const int ub = P->hunit[g], nu = P->hunit[g + 1] - ub;
    if (nu > 0) {
      SCW_TRY_E(launch_phases_tc(one, nullptr, P->d_unit_entries + ub, nu, P->max_M, P->F_pad, P->bf16, st),
                "phase kernel launch");
      SCW_TRY_E(launch_contract_tc(one, nullptr, P->hsched[g], P->NB, P->bf16, P->d_err, P->timeout_ns,
                                   P->inject_stall, st), "contraction kernel launch");
    }
    const int fb = P->hplane[g], nb = P->hplane[g + 1] - fb;
    if (nb > 0) {
      const int2* ent = P->d_plane_entries + fb;
      SCW_TRY_E(launch_xpass(one, nullptr, ent, nb, P->xpass_smem, st), "x-pass launch");
      int ny = 0;
      SCW_TRY_E(launch_ypass(one, nullptr, ent, nb, ypass_pairs(one.Vp) ? nb : 0, P->max_Qx, P->max_Vp, P->max_twy,
                             P->tiled, p->hio_out, nullptr, st, &ny), "y-pass launch");
    }
    SCW_TRY_E(cudaEventRecord(P->hev_comp[g], st), "cudaEventRecord");
    SCW_TRY_E(cudaStreamWaitEvent(P->st_out, P->hev_comp[g], 0), "cudaStreamWaitEvent");
    // plane slots [fb, fb + nb) are output planes [fb / I, (fb + nb) / I) of every illumination
    const int I = p->I, fo_b = fb / I, fo_n = nb / I;
    if (fo_n > 0)
      for (int il = 0; il < I; ++il)
        for (int c = 0; c < 3; ++c) {
          const size_t off = ((size_t)(il * 3 + c) * p->Fz_out + fo_b) * slice;
          SCW_TRY_E(cudaMemcpyAsync(static_cast<float2*>(out) + off, p->hio_out + off, fo_n * slice * sizeof(float2),
                                    cudaMemcpyDeviceToHost, P->st_out), "cudaMemcpyAsync");
        }
  }
  SCW_TRY_E(cudaEventRecord(P->hev_out, P->st_out), "cudaEventRecord");
  SCW_TRY_E(cudaStreamWaitEvent(st, P->hev_out, 0), "cudaStreamWaitEvent");
  SCW_TRY_E(cudaStreamSynchronize(st), "cudaStreamSynchronize");
#undef SCW_TRY_E
  return SCW_OK;
}

static scw_status set_layers_item(scw_plan_t P, int idx, const void* W, const void* gamma, const void* alpha,
                                  const void* p_inc, const void* p_ref, const void* p_trn, cudaStream_t st) {
  Plan* p = P->items[idx];
  if (!W || !gamma || !alpha) return set_error(SCW_ERR_INVALID_ARGUMENT, "W, gamma and alpha are required");
  if ((p->flags & SCW_FLAG_EXTERIOR) && (!p_inc || !p_ref || !p_trn))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "SCW_FLAG_EXTERIOR needs p_inc, p_ref and p_trn");
  if ((reinterpret_cast<uintptr_t>(W) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "W must be 16-byte aligned");
  p->gamma = static_cast<const double2*>(gamma);
  p->alpha = static_cast<const double2*>(alpha);
  p->p_inc = static_cast<const double2*>(p_inc);
  p->p_ref = static_cast<const double2*>(p_ref);
  p->p_trn = static_cast<const double2*>(p_trn);
  p->item.gamma = p->gamma;
  p->item.alpha = p->alpha;
  const float2* w = static_cast<const float2*>(W);
  cudaError_t e = cudaEventRecord(p->ev0, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  if (!p->units.empty()) {
    e = convert_w(p, w, st);
    if (e != cudaSuccess) return cuda_error(e, "W conversion launch");
  }
  e = cudaEventRecord(p->ev1, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  p->convert_pending = true;
  p->layers_set = true;
  if (P->batched) {
    e = cudaMemcpyAsync(P->d_items + idx, &p->item, sizeof(ItemDev), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "item descriptor upload");
  } else {
    invalidate_graph(P);  // the graph holds the item by value
  }
  return SCW_OK;
}

extern "C" {

int scw_version(void) { return 2; }

const char* scw_last_error(void) { return g_last_error.c_str(); }

const char* scw_status_string(scw_status s) {
  switch (s) {
    case SCW_OK: return "ok";
    case SCW_ERR_INVALID_ARGUMENT: return "invalid argument";
    case SCW_ERR_UNSUPPORTED: return "unsupported";
    case SCW_ERR_OUT_OF_MEMORY: return "out of memory";
    case SCW_ERR_CUDA: return "CUDA error";
    case SCW_ERR_TIMEOUT: return "device wait timed out";
    case SCW_ERR_NUMERIC: return "non-finite value";
    case SCW_ERR_STATE: return "call order violated";
    case SCW_ERR_BOUNDS: return "index outside its buffer";
  }
  return "unknown status";
}

scw_status scw_plan(const scw_desc* d, void* stream, scw_plan_t* out) {
  SetupStream guard(static_cast<cudaStream_t>(stream));
  if (!out) return set_error(SCW_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = nullptr;
  scw_status s = validate_desc(d);
  if (s != SCW_OK) return s;
  s = check_device();
  if (s != SCW_OK) return s;
  scw_plan_t P = new (std::nothrow) scw_plan_s();
  if (!P) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  Plan* p = nullptr;
  s = create_item(d, 0, &p);
  if (s != SCW_OK) {
    free_plan(P);
    return s;
  }
  P->items.push_back(p);
  P->precision = d->precision;
  P->tc = d->precision != SCW_PREC_FP32;
  P->bf16 = d->precision == SCW_PREC_SPLIT_BF16;
  P->F_pad = p->F_pad;
  P->NB = p->NB;
  s = finish_plan(P, {d->k_split}, (d->flags & SCW_FLAG_AUTOTUNE) != 0);
  if (s != SCW_OK) {
    free_plan(P);
    return s;
  }
  *out = P;
  return SCW_OK;
}

scw_status scw_plan_create(const scw_desc* d, scw_plan_t* out) { return scw_plan(d, nullptr, out); }

scw_status scw_plan_batched(const scw_desc* descs, int n, void* stream, scw_plan_t* out) {
  SetupStream guard(static_cast<cudaStream_t>(stream));
  if (!out) return set_error(SCW_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = nullptr;
  if (!descs || n < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "need at least one item");
  for (int i = 0; i < n; ++i) {
    scw_status s = validate_desc(&descs[i]);
    if (s != SCW_OK) return set_error(s, "item " + std::to_string(i) + ": " + g_last_error);
    if (descs[i].precision != descs[0].precision)
      return set_error(SCW_ERR_INVALID_ARGUMENT, "all items of a batch share one precision");
    if (descs[i].flags & SCW_FLAG_HOST_IO)
      return set_error(SCW_ERR_UNSUPPORTED, "SCW_FLAG_HOST_IO is for single plans");
  }
  scw_status s = check_device();
  if (s != SCW_OK) return s;
  scw_plan_t P = new (std::nothrow) scw_plan_s();
  if (!P) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  P->batched = true;
  P->precision = descs[0].precision;
  P->tc = P->precision != SCW_PREC_FP32;
  P->bf16 = P->precision == SCW_PREC_SPLIT_BF16;
  // every item of a tensor-core batch shares one plane-slot count (one N for the MMA)
  int fpad = 8;
  for (int i = 0; i < n; ++i) {
    Plan probe;
    probe.L = descs[i].L;
    probe.Fz = descs[i].Fz;
    probe.flags = descs[i].flags | SCW_FLAG_EXTERIOR;
    probe.z_bounds.assign(descs[i].z_bounds, descs[i].z_bounds + descs[i].L + 1);
    probe.z_planes.assign(descs[i].z_planes, descs[i].z_planes + descs[i].Fz);
    std::vector<int> ext;
    int max_nf = 0;
    assign_planes(&probe, ext, max_nf);
    fpad = std::max(fpad, round_planes(std::max(max_nf, 1)));
  }
  std::vector<int> user_ks;
  bool timed = false;
  for (int i = 0; i < n; ++i) {
    Plan* p = nullptr;
    s = create_item(&descs[i], P->tc ? fpad : 0, &p);
    if (s != SCW_OK) {
      free_plan(P);
      return set_error(s, "item " + std::to_string(i) + ": " + g_last_error);
    }
    P->items.push_back(p);
    user_ks.push_back(descs[i].k_split);
    timed = timed || (descs[i].flags & SCW_FLAG_AUTOTUNE);
  }
  P->F_pad = fpad;
  P->NB = 2 * fpad;
  s = finish_plan(P, user_ks, timed);
  if (s != SCW_OK) {
    free_plan(P);
    return s;
  }
  *out = P;
  return SCW_OK;
}

scw_status scw_plan_batched_create(const scw_desc* descs, int n, scw_plan_t* out) {
  return scw_plan_batched(descs, n, nullptr, out);
}

scw_status scw_plan_destroy(scw_plan_t plan) {
  if (plan) {
    cudaDeviceSynchronize();
    free_plan(plan);
  }
  return SCW_OK;
}

scw_status scw_plan_set_layers(scw_plan_t P, const void* W, const void* gamma, const void* alpha, const void* p_inc,
                               const void* p_ref, const void* p_trn, void* stream) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (P->batched) return set_error(SCW_ERR_STATE, "batched plan: use scw_plan_batched_set_layers");
  return set_layers_item(P, 0, W, gamma, alpha, p_inc, p_ref, p_trn, static_cast<cudaStream_t>(stream));
}

scw_status scw_plan_batched_set_layers(scw_plan_t P, int item, const void* W, const void* gamma, const void* alpha,
                                       const void* p_inc, const void* p_ref, const void* p_trn, void* stream) {
  scw_status s = check_item_index(P, item);
  if (s != SCW_OK) return s;
  return set_layers_item(P, item, W, gamma, alpha, p_inc, p_ref, p_trn, static_cast<cudaStream_t>(stream));
}

scw_status scw_synthesize(scw_plan_t P, void* out, void* stream) {
  if (!P || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and out are required");
  if (P->batched) return set_error(SCW_ERR_STATE, "batched plan: use scw_synthesize_batched");
  if (!P->items[0]->layers_set) return set_error(SCW_ERR_STATE, "scw_plan_set_layers has not been called");
  if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "out must be 16-byte aligned");
  return run_synthesis(P, static_cast<float2*>(out), static_cast<cudaStream_t>(stream));
}

scw_status scw_synthesize_batched(scw_plan_t P, const void* item_table, void* const* outs, void* stream) {
  if (!P || (!outs && !item_table) || (outs && item_table))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and exactly one of item_table and outs are required");
  if (!P->batched) return set_error(SCW_ERR_STATE, "single plan: use scw_synthesize");
  for (size_t i = 0; i < P->items.size(); ++i) {
    if (!P->items[i]->layers_set) return set_error(SCW_ERR_STATE, "item " + std::to_string(i) + " has no layers");
    if (outs && (!outs[i] || (reinterpret_cast<uintptr_t>(outs[i]) & 15u) != 0))
      return set_error(SCW_ERR_INVALID_ARGUMENT, "every out must be non-NULL and 16-byte aligned");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (item_table) {
    // the device table is copied in stream order: the previous replay on `st` has read the old one
    if ((reinterpret_cast<uintptr_t>(item_table) & 7u) != 0)
      return set_error(SCW_ERR_INVALID_ARGUMENT, "item_table must be 8-byte aligned");
    cudaError_t e = cudaMemcpyAsync(P->d_outs, item_table, P->items.size() * sizeof(float2*), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "item table copy");
    return run_synthesis(P, nullptr, st);
  }
  // the previous call's copy of the pointer table must have been consumed before it is rewritten
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  for (size_t i = 0; i < P->items.size(); ++i) P->h_outs[i] = static_cast<float2*>(outs[i]);
  e = cudaMemcpyAsync(P->d_outs, P->h_outs, P->items.size() * sizeof(float2*), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "output table upload");
  return run_synthesis(P, nullptr, st);
}

scw_status scw_spectrum(scw_plan_t P, void* S, void* stream) {
  if (!P || !S) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and S are required");
  if (P->batched) return set_error(SCW_ERR_STATE, "not available on a batched plan");
  if (!P->items[0]->layers_set) return set_error(SCW_ERR_STATE, "scw_plan_set_layers has not been called");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int n = 0;
  scw_status s = enqueue_spectrum(P, st, false, n);
  if (s != SCW_OK) return s;
  cudaError_t e = launch_gather_spectrum(*P->items[0], static_cast<float2*>(S), st);
  if (e != cudaSuccess) return cuda_error(e, "gather launch");
  return SCW_OK;
}

scw_status scw_recompose(scw_plan_t P, const void* S, void* out, void* stream) {
  if (!P || !S || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan, S and out are required");
  if (P->batched) return set_error(SCW_ERR_STATE, "not available on a batched plan");
  if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "out must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan* p = P->items[0];
  cudaError_t e = launch_recompose(p->item, nullptr, P->d_plane_entries, P->n_plane_entries, P->max_Qx, P->rec_smem,
                                   static_cast<const float2*>(S), p->d_nsplit1, static_cast<float2*>(out), nullptr, st);
  if (e != cudaSuccess) return cuda_error(e, "recompose launch");
  return SCW_OK;
}

scw_status scw_plan_set_points(scw_plan_t P, const double* xy, int n_points) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (P->batched) return set_error(SCW_ERR_UNSUPPORTED, "point sets are for single plans");
  if (n_points < 0 || n_points > (1 << 22)) return set_error(SCW_ERR_INVALID_ARGUMENT, "n_points must be in [0, 2^22]");
  if (n_points > 0 && !xy) return set_error(SCW_ERR_INVALID_ARGUMENT, "xy is required");
  for (int i = 0; i < 2 * n_points; ++i)
    if (!std::isfinite(xy[i])) return set_error(SCW_ERR_INVALID_ARGUMENT, "non-finite point coordinate");
  Plan* p = P->items[0];
  if (p->pts) {  // earlier calls may still read the old tables
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  }
  points_free(p->pts);
  p->pts = nullptr;
  if (n_points == 0) return SCW_OK;
  return points_build(&p->pts, *p, P->tc, xy, n_points, P->cap_stream);
}

scw_status scw_plan_set_point_planes(scw_plan_t P, const int* plane) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (P->batched) return set_error(SCW_ERR_UNSUPPORTED, "point sets are for single plans");
  Plan* p = P->items[0];
  if (!p->pts) return set_error(SCW_ERR_STATE, "scw_plan_set_points has not been called");
  cudaError_t e = cudaDeviceSynchronize();  // earlier calls may still read the old table
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  return points_set_planes(*p->pts, plane, p->Fz_out, P->cap_stream);
}

scw_status scw_synthesize_points(scw_plan_t P, void* out, void* stream) {
  if (!P || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and out are required");
  if (P->batched) return set_error(SCW_ERR_UNSUPPORTED, "point sets are for single plans");
  Plan* p = P->items[0];
  if (!p->layers_set) return set_error(SCW_ERR_STATE, "scw_plan_set_layers has not been called");
  if (!p->pts) return set_error(SCW_ERR_STATE, "scw_plan_set_points has not been called");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool marks = P->timing;
  int n = 0;
  scw_status s = enqueue_spectrum(P, st, marks, n);
  if (s != SCW_OK) return s;
  mark(P, 2, st, marks);
  cudaError_t e = points_prepare(*p->pts, *p, st);
  if (e != cudaSuccess) return cuda_error(e, "point spectrum launch");
  mark(P, 3, st, marks);
  e = points_product(*p->pts, *p, static_cast<float2*>(out), P->d_err, P->timeout_ns, st);
  if (e != cudaSuccess) return cuda_error(e, "point product launch");
  mark(P, 4, st, marks);
  if (marks && P->tev_used + kMarks <= P->tev.size()) P->tev_used += kMarks;
  P->kernels_per_synthesis = n + 2;
  return SCW_OK;
}

scw_status scw_synthesize_host(scw_plan_t P, const void* W, const void* gamma, const void* alpha, const void* p_inc,
                               const void* p_ref, const void* p_trn, void* out, void* stream) {
  if (!P || !W || !gamma || !alpha || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "missing argument");
  if (P->batched) return set_error(SCW_ERR_STATE, "not available on a batched plan");
  Plan* p = P->items[0];
  if (!(p->flags & SCW_FLAG_HOST_IO)) return set_error(SCW_ERR_STATE, "plan was created without SCW_FLAG_HOST_IO");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((p->flags & SCW_FLAG_EXTERIOR) && (!p_inc || !p_ref || !p_trn))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "SCW_FLAG_EXTERIOR needs p_inc, p_ref and p_trn");
  if (P->tc && !p->units.empty() && P->groups == 1) {
    const void* pio[3] = {p_inc, p_ref, p_trn};
    return synthesize_host_pipelined(P, W, gamma, alpha, pio, out, st);
  }
  const size_t L = p->L, M = p->M;
  cudaError_t e;
#define SCW_CP(dst, src, bytes, kind)                              \
  do {                                                             \
    e = cudaMemcpyAsync((dst), (src), (bytes), (kind), st);        \
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync"); \
  } while (0)
  SCW_CP(p->hio_W, W, L * 3 * M * 4 * M * sizeof(float2), cudaMemcpyHostToDevice);
  SCW_CP(p->hio_gamma, gamma, L * 4 * M * sizeof(double2), cudaMemcpyHostToDevice);
  SCW_CP(p->hio_alpha, alpha, p->I * L * 4 * M * sizeof(double2), cudaMemcpyHostToDevice);
  const double2 *pi = nullptr, *pr = nullptr, *pt = nullptr;
  if (p_inc && p_ref && p_trn) {
    const size_t np = (size_t)p->I * 3 * M;  // each of p_inc, p_ref, p_trn: [I][3][M]
    SCW_CP(p->hio_p, p_inc, np * sizeof(double2), cudaMemcpyHostToDevice);
    SCW_CP(p->hio_p + np, p_ref, np * sizeof(double2), cudaMemcpyHostToDevice);
    SCW_CP(p->hio_p + 2 * np, p_trn, np * sizeof(double2), cudaMemcpyHostToDevice);
    pi = p->hio_p; pr = p->hio_p + np; pt = p->hio_p + 2 * np;
  }
  // same device buffers every call: the layers are re-attached without dropping the graph
  if (!p->layers_set || p->gamma != p->hio_gamma) {
    scw_status s = set_layers_item(P, 0, p->hio_W, p->hio_gamma, p->hio_alpha, pi, pr, pt, st);
    if (s != SCW_OK) return s;
  } else {
    e = convert_w(p, p->hio_W, st);
    if (e != cudaSuccess) return cuda_error(e, "W conversion launch");
  }
  scw_status s = run_synthesis(P, p->hio_out, st);
  if (s != SCW_OK) return s;
  SCW_CP(out, p->hio_out, (size_t)3 * p->Fz * p->out_pstride * sizeof(float2), cudaMemcpyDeviceToHost);
#undef SCW_CP
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  return SCW_OK;
}

scw_status scw_plan_check(scw_plan_t P, void* stream) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  int word = 0;
  e = cudaMemcpy(&word, P->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "reading the device error word");
  if (word) {
    cudaMemset(P->d_err, 0, sizeof(int));
    if (word == DEV_ERR_BOUNDS)
      return set_error(SCW_ERR_BOUNDS, "a kernel formed an index outside its buffer (SCW_FLAG_DEBUG_BOUNDS; the "
                                       "access was skipped, so this call's results are invalid)");
    return set_error(SCW_ERR_TIMEOUT, "device error word " + std::to_string(word) +
                                          " (1: stage fill, 2: stage free, 4: accumulator, 8: drain, 16: dependency)");
  }
  return SCW_OK;
}

scw_status scw_plan_set_timeout_ns(scw_plan_t P, uint64_t ns) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (ns == 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "timeout must be positive");
  P->timeout_ns = ns;
  invalidate_graph(P);
  return SCW_OK;
}

scw_status scw_plan_inject_stall(scw_plan_t P, int on) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (!P->tc) return set_error(SCW_ERR_UNSUPPORTED, "stall injection exists in the tensor-core contraction only");
  P->inject_stall = on ? 1 : 0;
  invalidate_graph(P);
  return SCW_OK;
}

scw_status scw_plan_enable_timing(scw_plan_t P, int on) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  P->timing = on != 0;
  P->tev_used = 0;
  return SCW_OK;
}

scw_status scw_plan_get_timings(scw_plan_t P, scw_kernel_times* t) {
  if (!P || !t) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and t are required");
  std::memset(t, 0, sizeof(*t));
  const size_t calls = P->tev_used / kMarks;
  for (size_t c = 0; c < calls; ++c) {
    cudaEvent_t* ev = &P->tev[kMarks * c];
    cudaError_t e = cudaEventSynchronize(ev[kMarks - 1]);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize");
    float ms[kMarks - 1], tot;
    for (int k = 0; k < kMarks - 1; ++k) {
      e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
      if (e != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime");
    }
    cudaEventElapsedTime(&tot, ev[0], ev[kMarks - 1]);
    t->phases_ms += ms[0];
    t->contract_ms += ms[1];
    t->xpass_ms += ms[2];
    t->ypass_ms += ms[3];
    t->recompose_ms += ms[2] + ms[3];
    t->total_ms += tot;
  }
  t->calls = (int)calls;
  if (calls) {
    t->phases_ms /= calls;
    t->contract_ms /= calls;
    t->xpass_ms /= calls;
    t->ypass_ms /= calls;
    t->recompose_ms /= calls;
    t->total_ms /= calls;
  }
  P->tev_used = 0;
  return SCW_OK;
}

static void trace_init_values(unsigned long long* h) {
  for (int s = 0; s < TRACE_SLOTS; ++s) {
    h[2 * s] = ~0ull;
    h[2 * s + 1] = 0ull;
  }
}

scw_status scw_plan_enable_trace(scw_plan_t P, int on) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  cudaError_t e = cudaDeviceSynchronize();  // no kernel of this plan may still hold the old pointer
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  if (on && !P->d_trace) {
    e = cudaMalloc(reinterpret_cast<void**>(&P->d_trace), 2 * TRACE_SLOTS * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_error(e, "trace buffer");
    unsigned long long h[2 * TRACE_SLOTS];
    trace_init_values(h);
    e = cudaMemcpy(P->d_trace, h, sizeof(h), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "trace buffer");
  } else if (!on && P->d_trace) {
    cudaFree(P->d_trace);
    P->d_trace = nullptr;
  }
  for (auto* p : P->items) p->item.trace = P->d_trace;
  invalidate_graph(P);  // the kernels take the pointer by value: recapture
  return upload_items(P, nullptr);
}

scw_status scw_plan_debug_set_extent(scw_plan_t P, int buffer, unsigned long long elements) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (buffer < 0 || buffer >= BND_COUNT) return set_error(SCW_ERR_INVALID_ARGUMENT, "unknown buffer");
  if (!(P->items[0]->flags & SCW_FLAG_DEBUG_BOUNDS)) return set_error(SCW_ERR_STATE, "plan without SCW_FLAG_DEBUG_BOUNDS");
  cudaError_t e = cudaDeviceSynchronize();  // no kernel of this plan may still read the old extents
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  for (auto* p : P->items) {
    const unsigned long long real = p->bnd_real[buffer];
    p->item.bnd[buffer] = elements == 0 ? real : std::min(real, elements);
  }
  invalidate_graph(P);
  return upload_items(P, nullptr);
}

scw_status scw_plan_get_trace(scw_plan_t P, double* us, int n_slots) {
  if (!P || !us || n_slots < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan, us and n_slots > 0 are required");
  if (!P->d_trace) return set_error(SCW_ERR_STATE, "tracing is off (scw_plan_enable_trace)");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  unsigned long long h[2 * TRACE_SLOTS];
  e = cudaMemcpy(h, P->d_trace, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "trace read-back");
  unsigned long long t0 = ~0ull;
  for (int s = 0; s < TRACE_SLOTS; ++s)
    if (h[2 * s + 1] != 0ull) t0 = std::min(t0, h[2 * s]);
  for (int s = 0; s < n_slots; ++s) {
    const bool used = s < TRACE_SLOTS && h[2 * s + 1] != 0ull && h[2 * s] != ~0ull;
    us[2 * s] = used ? (double)(h[2 * s] - t0) * 1e-3 : -1.0;
    us[2 * s + 1] = used ? (double)(h[2 * s + 1] - t0) * 1e-3 : -1.0;
  }
  trace_init_values(h);
  e = cudaMemcpy(P->d_trace, h, sizeof(h), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "trace reset");
  return SCW_OK;
}

scw_status scw_plan_get_info(scw_plan_t P, scw_plan_info* info) {
  if (!P || !info) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and info are required");
  std::memset(info, 0, sizeof(*info));
  for (auto* p : P->items) {
    if (p->convert_pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(p->ev1) == cudaSuccess && cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess)
        p->convert_ms = ms;
      p->convert_pending = false;
    }
    info->M = std::max(info->M, p->M);
    info->active_layers += (int)p->units.size();
    info->k_split = std::max(info->k_split, p->k_split);
    info->exterior_planes += p->n_exterior;
    info->workspace_bytes += p->workspace_bytes;
    info->convert_ms += p->convert_ms;
  }
  info->planes_per_layer_pad = P->F_pad;
  info->kernels_per_synthesis = P->kernels_per_synthesis;
  info->items = (int)P->items.size();
  info->contract_ctas = P->sched.grid;
  info->contract_tasks = P->sched.n_tasks;
  info->schedule_max_load = P->sched.max_load;
  info->schedule_mean_load = P->sched.mean_load;
  return SCW_OK;
}

const char* scw_plan_tune_report(scw_plan_t P) { return P ? P->tune_report.c_str() : ""; }

scw_status scw_plan_set_pipeline(scw_plan_t P, int groups) {
  if (!P) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (groups < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "groups must be >= 1");
  if (groups > 1 && (P->batched || !P->tc))
    return set_error(SCW_ERR_UNSUPPORTED, "pipelining is for single tensor-core plans");
  Plan* p = P->items[0];
  const int nu = (int)p->units.size();
  groups = std::max(1, std::min(groups, nu));
  for (auto& g : P->gsched) {
    if (g.d_tasks) cudaFree(g.d_tasks);
    if (g.d_cta_off) cudaFree(g.d_cta_off);
  }
  P->gsched.clear();
  P->gplane.clear();
  invalidate_graph(P);
  P->groups = groups;
  if (groups == 1) return SCW_OK;
  cudaError_t e;
  if (!P->st2) {
    e = cudaStreamCreateWithFlags(&P->st2, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamCreateWithFlags");
    e = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventCreate");
  }
  while ((int)P->gev.size() < groups) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventCreate");
    P->gev.push_back(ev);
  }
  // contiguous unit groups; group g's planes run up to the first plane of group g+1
  P->gsched.resize(groups);
  P->gplane.assign(groups + 1, 0);
  for (int g = 0; g < groups; ++g) {
    const int ub = (int)((long long)nu * g / groups), ue = (int)((long long)nu * (g + 1) / groups);
    scw_status s = upload_schedule(P->items, P->NB, P->bf16, P->gsched[g], 1, ub, ue);
    if (s != SCW_OK) return s;
    P->gplane[g + 1] = (g + 1 < groups) ? p->units[ue].f0 : p->Fz;
  }
  return SCW_OK;
}

}  // extern "C"
