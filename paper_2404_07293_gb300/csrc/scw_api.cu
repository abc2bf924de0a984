// Host side of libscw: argument validation, plane-to-layer assignment,
// order / twiddle tables, workspace ownership and the launch sequence of
// scw_synthesize. See include/scw.h for the contract of each entry point.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>

#include "scw_internal.cuh"

struct scw_plan_s : public scw::Plan {};

namespace scw {

static thread_local std::string g_last_error;

scw_status set_error(scw_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

scw_status cuda_error(cudaError_t e, const char* what) {
  return set_error(SCW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
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
  return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_plan(Plan* p) {
  if (!p) return;
  void* ptrs[] = {p->d_err,   p->d_units,  p->d_zplanes, p->d_zbounds, p->d_nsplit, p->d_nsplit1,
                  p->d_ext_planes, p->d_sz_top, p->d_sz_bot, p->d_twx, p->d_twy,   p->Whi,
                  p->Wlo,     p->Wh,       p->Wt,        p->Bhi,       p->Blo,      p->Cf,
                  p->S_part,  p->T,        p->hio_W,     p->hio_gamma, p->hio_alpha, p->hio_p,
                  p->hio_out};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  for (cudaEvent_t ev : p->tev) cudaEventDestroy(ev);
  delete static_cast<scw_plan_s*>(p);
}

static int round_planes(int nf) {
  static const int slots[] = {8, 16, 24, 32, 64, 128};
  for (int s : slots)
    if (nf <= s) return s;
  return -1;
}

}  // namespace scw

using namespace scw;

extern "C" {

int scw_version(void) { return 1; }

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
  }
  return "unknown status";
}

scw_status scw_plan_create(const scw_desc* d, scw_plan_t* out) {
  if (!out) return set_error(SCW_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = nullptr;
  if (!d) return set_error(SCW_ERR_INVALID_ARGUMENT, "desc is NULL");
  if (d->U < 1 || d->V < 1 || d->L < 1) return set_error(SCW_ERR_INVALID_ARGUMENT, "U, V and L must be >= 1");
  if ((long long)d->U * d->V > kMaxM) return set_error(SCW_ERR_UNSUPPORTED, "U*V exceeds 4096");
  if (d->V > 96) return set_error(SCW_ERR_UNSUPPORTED, "V above 96 (y-pass shared tile)");
  if (!(d->lambda > 0) || !(d->X > 0) || !(d->Y > 0))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "lambda, X and Y must be positive");
  if (d->Fx < 8 || d->Fy < 8 || d->Fx % 8 || d->Fy % 8 || d->Fx > kMaxFx || d->Fy > kMaxFx)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "Fx and Fy must be multiples of 8 in [8, 4096]");
  if (d->Fz < 1 || d->Fz > 65535) return set_error(SCW_ERR_INVALID_ARGUMENT, "Fz must be in [1, 65535]");
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

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3)
    return set_error(SCW_ERR_CUDA, "libscw is built for sm_103a (GB300); device is sm_" + std::to_string(prop.major) +
                                       std::to_string(prop.minor));

  Plan* p = new (std::nothrow) scw_plan_s();
  if (!p) return set_error(SCW_ERR_OUT_OF_MEMORY, "host allocation failed");
  p->U = d->U; p->V = d->V; p->M = d->U * d->V; p->L = d->L;
  p->Fx = d->Fx; p->Fy = d->Fy; p->Fz = d->Fz;
  p->lambda = d->lambda; p->X = d->X; p->Y = d->Y; p->x0 = d->x0; p->y0 = d->y0;
  p->n_top = d->n_top; p->n_bot_re = d->n_bot_re; p->n_bot_im = d->n_bot_im; p->z_inc = d->z_inc;
  p->precision = d->precision; p->flags = d->flags;
  p->z_bounds.assign(d->z_bounds, d->z_bounds + d->L + 1);
  p->z_planes.assign(d->z_planes, d->z_planes + d->Fz);

  // plane -> region: half-open layers [z_{l-1}, z_l), the last one closed (Sec. 2.6.2)
  const double z0 = p->z_bounds.front(), zL = p->z_bounds.back();
  p->plane_region.resize(p->Fz);
  std::vector<int> ext;
  for (int f = 0; f < p->Fz; ++f) {
    const double z = p->z_planes[f];
    int r;
    if (z < z0) r = -1;
    else if (z > zL) r = p->L;
    else {
      r = (int)(std::upper_bound(p->z_bounds.begin(), p->z_bounds.end(), z) - p->z_bounds.begin()) - 1;
      r = std::min(r, p->L - 1);
    }
    p->plane_region[f] = r;
    if (r < 0 || r >= p->L) ext.push_back(f);
  }
  p->n_exterior = (int)ext.size();
  if (p->n_exterior && !(p->flags & SCW_FLAG_EXTERIOR)) {
    free_plan(p);
    return set_error(SCW_ERR_INVALID_ARGUMENT, "planes outside [z0, zL] need SCW_FLAG_EXTERIOR");
  }
  // active layers, split into chunks of at most kMaxPlanesPerLayer planes
  int max_nf = 0;
  for (int f = 0; f < p->Fz;) {
    const int r = p->plane_region[f];
    int g = f;
    while (g < p->Fz && p->plane_region[g] == r) ++g;
    if (r >= 0 && r < p->L) {
      for (int s = f; s < g; s += kMaxPlanesPerLayer) {
        LayerUnit u{r, s, std::min(kMaxPlanesPerLayer, g - s), 0};
        p->units.push_back(u);
        max_nf = std::max(max_nf, u.nf);
      }
    }
    f = g;
  }
  p->F_pad = std::max(8, round_planes(std::max(max_nf, 1)));
  p->NB = 2 * p->F_pad;

  // split of the 4M modes: aim for ~4 waves of work units, keep >= 4 K-stages per unit
  const int n_units = (int)p->units.size();
  const int K = 4 * p->M;
  if (d->k_split > 0) {
    p->k_split = d->k_split;
  } else if (n_units > 0) {
    const int slots = prop.multiProcessorCount * 2 * 4;
    const bool fp32 = p->precision == SCW_PREC_FP32;
    const int per_split_units = n_units * (fp32 ? (3 * p->M + 255) / 256 : (3 * p->M + 127) / 128);
    int ks = (slots + per_split_units - 1) / per_split_units;
    const int min_k = fp32 ? 128 : 4 * 32;  // modes per split (4 K-stages of 32 complex)
    ks = std::max(1, std::min(ks, std::max(1, K / min_k)));
    if (fp32) {  // shared-memory slice of C per CTA stays <= 96 KB
      const int fch = p->F_pad >= 16 ? 16 : 8;
      const int need = (int)(((size_t)K * fch * 8 + 96 * 1024 - 1) / (96 * 1024));
      ks = std::max(ks, need);
    }
    p->k_split = ks;
  }
  if (p->k_split > K) p->k_split = K;
  if (p->precision == SCW_PREC_FP32) {
    const int fch = p->F_pad >= 16 ? 16 : 8;
    const size_t per = (K + p->k_split - 1) / p->k_split;
    if (per * fch * 8 > 200 * 1024) {
      free_plan(p);
      return set_error(SCW_ERR_UNSUPPORTED, "k_split too small for the FP32 contraction's shared memory");
    }
  }

  // host tables
  std::vector<double2> szt(p->M), szb(p->M);
  for (int m = 0; m < p->M; ++m) {
    const int u = m % p->U - p->U / 2, v = m / p->U - p->V / 2;
    const double sx = p->lambda * u / p->X, sy = p->lambda * v / p->Y;
    const auto a = s_z(std::complex<double>(p->n_top, 0.0), sx, sy);
    const auto b = s_z(std::complex<double>(p->n_bot_re, p->n_bot_im), sx, sy);
    szt[m] = make_double2(a.real(), a.imag());
    szb[m] = make_double2(b.real(), b.imag());
  }
  const int Qx = p->Fx / 8, Qy = p->Fy / 8;
  std::vector<float2> twx((size_t)Qx * p->U), twy((size_t)Qy * p->V);
  for (int b = 0; b < Qx; ++b)
    for (int ui = 0; ui < p->U; ++ui) {
      const int u = ui - p->U / 2;
      twx[(size_t)b * p->U + ui] = cis_cycles((double)u * b / p->Fx + u * p->x0 / p->X);
    }
  for (int b = 0; b < Qy; ++b)
    for (int vi = 0; vi < p->V; ++vi) {
      const int v = vi - p->V / 2;
      twy[(size_t)b * p->V + vi] = cis_cycles((double)v * b / p->Fy + v * p->y0 / p->Y);
    }
  std::vector<int> nsplit(p->Fz), ones(p->Fz, 1);
  for (int f = 0; f < p->Fz; ++f) nsplit[f] = (p->plane_region[f] >= 0 && p->plane_region[f] < p->L) ? p->k_split : 1;

  size_t& tot = p->workspace_bytes;
  const size_t L = p->L, M = p->M;
#define SCW_TRY(x)                                   \
  do {                                               \
    cudaError_t _e = (x);                            \
    if (_e != cudaSuccess) {                         \
      free_plan(p);                                  \
      if (_e == cudaErrorMemoryAllocation)           \
        return set_error(SCW_ERR_OUT_OF_MEMORY, #x); \
      return cuda_error(_e, #x);                     \
    }                                                \
  } while (0)
  SCW_TRY(dalloc(&p->d_err, 1, tot));
  SCW_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
  SCW_TRY(upload(&p->d_units, p->units, tot));
  SCW_TRY(upload(&p->d_zplanes, p->z_planes, tot));
  SCW_TRY(upload(&p->d_zbounds, p->z_bounds, tot));
  SCW_TRY(upload(&p->d_nsplit, nsplit, tot));
  SCW_TRY(upload(&p->d_nsplit1, ones, tot));
  SCW_TRY(upload(&p->d_ext_planes, ext, tot));
  SCW_TRY(upload(&p->d_sz_top, szt, tot));
  SCW_TRY(upload(&p->d_sz_bot, szb, tot));
  SCW_TRY(upload(&p->d_twx, twx, tot));
  SCW_TRY(upload(&p->d_twy, twy, tot));
  SCW_TRY(dalloc(&p->S_part, (size_t)p->k_split * p->Fz * 3 * M, tot));
  SCW_TRY(cudaMemset(p->S_part, 0, (size_t)p->k_split * p->Fz * 3 * M * sizeof(float2)));
  SCW_TRY(dalloc(&p->T, (size_t)p->Fz * 3 * p->V * p->Fx, tot));
  if (n_units > 0) {
    if (p->precision == SCW_PREC_FP32) {
      SCW_TRY(dalloc(&p->Wt, L * 3 * M * 4 * M, tot));
      SCW_TRY(dalloc(&p->Cf, (size_t)n_units * 4 * M * p->F_pad, tot));
    } else {
      const size_t nA = L * 3 * M * 8 * M, nB = (size_t)n_units * p->NB * 8 * M;
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
      SCW_TRY(cudaMemset(p->Bhi, 0, nB * 2));
      SCW_TRY(cudaMemset(p->Blo, 0, nB * 2));
      std::string why;
      if (!encode_tensor_maps(*p, why)) {
        free_plan(p);
        return set_error(SCW_ERR_CUDA, why);
      }
    }
  }
  if (p->flags & SCW_FLAG_HOST_IO) {
    SCW_TRY(dalloc(&p->hio_W, L * 3 * M * 4 * M, tot));
    SCW_TRY(dalloc(&p->hio_gamma, L * 4 * M, tot));
    SCW_TRY(dalloc(&p->hio_alpha, L * 4 * M, tot));
    SCW_TRY(dalloc(&p->hio_p, 9 * M, tot));
    SCW_TRY(dalloc(&p->hio_out, (size_t)3 * p->Fz * p->Fy * p->Fx, tot));
  }
  SCW_TRY(cudaEventCreate(&p->ev0));
  SCW_TRY(cudaEventCreate(&p->ev1));
#undef SCW_TRY
  *out = static_cast<scw_plan_s*>(p);
  return SCW_OK;
}

scw_status scw_plan_destroy(scw_plan_t plan) {
  if (plan) {
    cudaDeviceSynchronize();
    free_plan(plan);
  }
  return SCW_OK;
}

scw_status scw_plan_set_layers(scw_plan_t p, const void* W, const void* gamma, const void* alpha, const void* p_inc,
                               const void* p_ref, const void* p_trn, void* stream) {
  if (!p) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (!W || !gamma || !alpha) return set_error(SCW_ERR_INVALID_ARGUMENT, "W, gamma and alpha are required");
  if ((p->flags & SCW_FLAG_EXTERIOR) && (!p_inc || !p_ref || !p_trn))
    return set_error(SCW_ERR_INVALID_ARGUMENT, "SCW_FLAG_EXTERIOR needs p_inc, p_ref and p_trn");
  if ((reinterpret_cast<uintptr_t>(W) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "W must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->gamma = static_cast<const double2*>(gamma);
  p->alpha = static_cast<const double2*>(alpha);
  p->p_inc = static_cast<const double2*>(p_inc);
  p->p_ref = static_cast<const double2*>(p_ref);
  p->p_trn = static_cast<const double2*>(p_trn);
  const size_t L = p->L, M = p->M;
  const float2* w = static_cast<const float2*>(W);
  cudaError_t e = cudaEventRecord(p->ev0, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  if (!p->units.empty()) {
    if (p->precision == SCW_PREC_FP32) e = launch_transpose_layers(w, p->Wt, p->L, 3 * p->M, 4 * p->M, st);
    else if (p->precision == SCW_PREC_SPLIT_BF16) e = launch_convert_split_bf16(w, p->Whi, p->Wlo, L * 3 * M * 4 * M, st);
    else e = launch_convert_fp16(w, p->Wh, L * 3 * M * 4 * M, st);
    if (e != cudaSuccess) return cuda_error(e, "W conversion launch");
  }
  e = cudaEventRecord(p->ev1, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  p->convert_pending = true;
  p->layers_set = true;
  return SCW_OK;
}

// Event slot k of the current timed call (nullptr when timing is off).
static cudaEvent_t timing_event(scw_plan_t p, int k) {
  if (!p->timing) return nullptr;
  const size_t i = p->tev_used + (size_t)k;
  if (i >= 5 * 4096) return nullptr;
  while (p->tev.size() <= i) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    p->tev.push_back(ev);
  }
  return p->tev[i];
}

static void mark(scw_plan_t p, int k, cudaStream_t st) {
  cudaEvent_t ev = timing_event(p, k);
  if (ev) cudaEventRecord(ev, st);
}

static scw_status run_spectrum(scw_plan_t p, cudaStream_t st, int& launches) {
  cudaError_t e;
  launches = 0;
  mark(p, 0, st);
  if (!p->units.empty()) {
    e = (p->precision == SCW_PREC_FP32) ? launch_phases_fp32(*p, st) : launch_phases_tc(*p, st);
    if (e != cudaSuccess) return cuda_error(e, "phase kernel launch");
    ++launches;
  }
  if (p->n_exterior) {
    e = launch_exterior(*p, st);
    if (e != cudaSuccess) return cuda_error(e, "exterior kernel launch");
    ++launches;
  }
  mark(p, 1, st);
  if (!p->units.empty()) {
    e = (p->precision == SCW_PREC_FP32) ? launch_contract_fp32(*p, st) : launch_contract_tc(*p, st);
    if (e != cudaSuccess) return cuda_error(e, "contraction kernel launch");
    ++launches;
  }
  return SCW_OK;
}

scw_status scw_synthesize(scw_plan_t p, void* out, void* stream) {
  if (!p || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and out are required");
  if (!p->layers_set) return set_error(SCW_ERR_STATE, "scw_plan_set_layers has not been called");
  if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "out must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int n = 0;
  scw_status s = run_spectrum(p, st, n);
  if (s != SCW_OK) return s;
  mark(p, 2, st);
  cudaError_t e = launch_xpass(*p, p->S_part, p->Fz, p->d_nsplit, st);
  if (e != cudaSuccess) return cuda_error(e, "x-pass launch");
  mark(p, 3, st);
  e = launch_ypass(*p, static_cast<float2*>(out), st);
  if (e != cudaSuccess) return cuda_error(e, "y-pass launch");
  mark(p, 4, st);
  if (p->timing && p->tev_used + 5 <= p->tev.size()) p->tev_used += 5;
  p->kernels_per_synthesis = n + 2;
  return SCW_OK;
}

scw_status scw_spectrum(scw_plan_t p, void* S, void* stream) {
  if (!p || !S) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and S are required");
  if (!p->layers_set) return set_error(SCW_ERR_STATE, "scw_plan_set_layers has not been called");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int n = 0;
  scw_status s = run_spectrum(p, st, n);
  if (s != SCW_OK) return s;
  cudaError_t e = launch_gather_spectrum(*p, static_cast<float2*>(S), st);
  if (e != cudaSuccess) return cuda_error(e, "gather launch");
  return SCW_OK;
}

scw_status scw_recompose(scw_plan_t p, const void* S, void* out, void* stream) {
  if (!p || !S || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan, S and out are required");
  if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "out must be 16-byte aligned");
  cudaError_t e = launch_recompose(*p, static_cast<const float2*>(S), p->Fz, p->d_nsplit1, static_cast<float2*>(out),
                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "recompose launch");
  return SCW_OK;
}

scw_status scw_synthesize_host(scw_plan_t p, const void* W, const void* gamma, const void* alpha, const void* p_inc,
                               const void* p_ref, const void* p_trn, void* out, void* stream) {
  if (!p || !W || !gamma || !alpha || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "missing argument");
  if (!(p->flags & SCW_FLAG_HOST_IO)) return set_error(SCW_ERR_STATE, "plan was created without SCW_FLAG_HOST_IO");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t L = p->L, M = p->M;
  cudaError_t e;
#define SCW_CP(dst, src, bytes, kind)                          \
  do {                                                         \
    e = cudaMemcpyAsync((dst), (src), (bytes), (kind), st);    \
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync"); \
  } while (0)
  SCW_CP(p->hio_W, W, L * 3 * M * 4 * M * sizeof(float2), cudaMemcpyHostToDevice);
  SCW_CP(p->hio_gamma, gamma, L * 4 * M * sizeof(double2), cudaMemcpyHostToDevice);
  SCW_CP(p->hio_alpha, alpha, L * 4 * M * sizeof(double2), cudaMemcpyHostToDevice);
  const double2 *pi = nullptr, *pr = nullptr, *pt = nullptr;
  if (p_inc && p_ref && p_trn) {
    SCW_CP(p->hio_p, p_inc, 3 * M * sizeof(double2), cudaMemcpyHostToDevice);
    SCW_CP(p->hio_p + 3 * M, p_ref, 3 * M * sizeof(double2), cudaMemcpyHostToDevice);
    SCW_CP(p->hio_p + 6 * M, p_trn, 3 * M * sizeof(double2), cudaMemcpyHostToDevice);
    pi = p->hio_p; pr = p->hio_p + 3 * M; pt = p->hio_p + 6 * M;
  }
  scw_status s = scw_plan_set_layers(p, p->hio_W, p->hio_gamma, p->hio_alpha, pi, pr, pt, stream);
  if (s != SCW_OK) return s;
  s = scw_synthesize(p, p->hio_out, stream);
  if (s != SCW_OK) return s;
  SCW_CP(out, p->hio_out, (size_t)3 * p->Fz * p->Fy * p->Fx * sizeof(float2), cudaMemcpyDeviceToHost);
#undef SCW_CP
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  return SCW_OK;
}

scw_status scw_plan_check(scw_plan_t p, void* stream) {
  if (!p) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  int word = 0;
  e = cudaMemcpy(&word, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "reading the device error word");
  if (word) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return set_error(SCW_ERR_TIMEOUT, "device error word " + std::to_string(word) +
                                          " (1: stage fill, 2: stage free, 4: accumulator, 8: drain)");
  }
  return SCW_OK;
}

scw_status scw_plan_set_timeout_ns(scw_plan_t p, uint64_t ns) {
  if (!p) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  if (ns == 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "timeout must be positive");
  p->timeout_ns = ns;
  return SCW_OK;
}

scw_status scw_plan_enable_timing(scw_plan_t p, int on) {
  if (!p) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan is NULL");
  p->timing = on != 0;
  p->tev_used = 0;
  return SCW_OK;
}

scw_status scw_plan_get_timings(scw_plan_t p, scw_kernel_times* t) {
  if (!p || !t) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and t are required");
  std::memset(t, 0, sizeof(*t));
  const size_t calls = p->tev_used / 5;
  for (size_t c = 0; c < calls; ++c) {
    cudaEvent_t* ev = &p->tev[5 * c];
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize");
    float ms[4], tot;
    for (int k = 0; k < 4; ++k) {
      e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
      if (e != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime");
    }
    cudaEventElapsedTime(&tot, ev[0], ev[4]);
    t->phases_ms += ms[0];
    t->contract_ms += ms[1];
    t->xpass_ms += ms[2];
    t->ypass_ms += ms[3];
    t->total_ms += tot;
  }
  t->calls = (int)calls;
  if (calls) {
    t->phases_ms /= calls;
    t->contract_ms /= calls;
    t->xpass_ms /= calls;
    t->ypass_ms /= calls;
    t->total_ms /= calls;
  }
  p->tev_used = 0;
  return SCW_OK;
}

scw_status scw_plan_get_info(scw_plan_t p, scw_plan_info* info) {
  if (!p || !info) return set_error(SCW_ERR_INVALID_ARGUMENT, "plan and info are required");
  if (p->convert_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p->ev1) == cudaSuccess && cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess)
      p->convert_ms = ms;
    p->convert_pending = false;
  }
  info->M = p->M;
  info->active_layers = (int)p->units.size();
  info->planes_per_layer_pad = p->F_pad;
  info->k_split = p->k_split;
  info->exterior_planes = p->n_exterior;
  info->workspace_bytes = p->workspace_bytes;
  info->convert_ms = p->convert_ms;
  info->kernels_per_synthesis = p->kernels_per_synthesis;
  return SCW_OK;
}

}  // extern "C"
