// scw_recompose_noalloc: the recompose step of scw_recompose for callers that
// cannot allocate device memory. Its scratch -- the fold twiddle tables, a
// per-plane split count and the plane table -- lives in one file-scope
// __device__ array instead of a plan's cudaMalloc'ed workspace. The kernel is
// the library's own recompose kernel, unchanged.
#include <cstring>
#include <mutex>

#include "scw_internal.cuh"

namespace scw {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // SCW_NOALLOC_SCRATCH_BYTES in scw.h

// Shared by every call on a device; held by each device that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device addresses of g_noalloc_scratch, looked up once per device.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {nullptr};

// The fold twiddles exp(2 pi i (u b / F + u x0 / X)) in the padded layouts the
// recompose kernels read (order u at position u mod np, fold_pos; zeros elsewhere;
// x table [p][b], y table [b][p]),
// with the argument reduced in FP64 as a plan does on the host; the all-ones
// split count; and the (item 0, plane f) entry table.
__global__ void noalloc_setup_kernel(float2* twx, int U, int Up, int Fx, double x0_over_X, float2* twy, int V,
                                     int Vp, int Fy, double y0_over_Y, int* ones, int2* entries, int Fz) {
  const int nx = (Fx / 8) * Up, ny = (Fy / 8) * Vp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx + ny + Fz; i += gridDim.x * blockDim.x) {
    if (i < nx + ny) {
      const bool isx = i < nx;
      const int k = isx ? i : i - nx;
      const int np = isx ? Up : Vp, n = isx ? U : V;
      // x table [p][b] (residue fastest), y table [b][p]
      const int Qx = Fx / 8;
      const int b = isx ? k % Qx : k / np;
      const int idx = fold_order(isx ? k / Qx : k - b * np, n, np);
      float2 w = make_float2(0.f, 0.f);
      if (idx >= 0) {
        const int u = idx - n / 2;
        const double t = isx ? ((double)u * b / Fx + u * x0_over_X) : ((double)u * b / Fy + u * y0_over_Y);
        const double r = t - rint(t);
        double s, c;
        sincospi(2.0 * r, &s, &c);
        w = make_float2((float)c, (float)s);
      }
      (isx ? twx : twy)[k] = w;
    } else {
      const int f = i - nx - ny;
      ones[f] = 1;
      entries[f] = make_int2(0, f);
    }
  }
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace scw

using namespace scw;

extern "C" scw_status scw_recompose_noalloc(int U, int V, double X, double Y, int Fx, int Fy, int Fz, double x0,
                                            double y0, const void* S, void* out, void* stream) {
  if (!S || !out) return set_error(SCW_ERR_INVALID_ARGUMENT, "S and out are required");
  if (U < 1 || V < 1 || (long long)U * V > kMaxM || V > 96)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "need 1 <= U, 1 <= V <= 96, U*V <= 4096");
  if (!(X > 0) || !(Y > 0)) return set_error(SCW_ERR_INVALID_ARGUMENT, "X and Y must be positive");
  if (Fx < 8 || Fy < 8 || Fx % 8 || Fy % 8 || Fx > kMaxFx || Fy > kMaxFx)
    return set_error(SCW_ERR_INVALID_ARGUMENT, "Fx and Fy must be multiples of 8 in [8, 4096]");
  if (Fz < 1 || Fz > 65535) return set_error(SCW_ERR_INVALID_ARGUMENT, "Fz must be in [1, 65535]");
  if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0) return set_error(SCW_ERR_INVALID_ARGUMENT, "out must be 16-byte aligned");

  // scratch layout: twx | twy | ones | entries, each 256-byte aligned
  const int Up = fold_np(U), Vp = fold_np(V);
  const size_t b_twx = align256(sizeof(float2) * (size_t)(Fx / 8) * Up);
  const size_t b_twy = align256(sizeof(float2) * (size_t)(Fy / 8) * Vp);
  const size_t b_one = align256(sizeof(int) * (size_t)Fz);
  const size_t b_ent = align256(sizeof(int2) * (size_t)Fz);
  const size_t need = b_twx + b_twy + b_one + b_ent;
  if (need > kNoAllocScratchBytes)
    return set_error(SCW_ERR_UNSUPPORTED, "scw_recompose_noalloc needs " + std::to_string(need) +
                                              " bytes of scratch, above its fixed " +
                                              std::to_string(kNoAllocScratchBytes) +
                                              " (twiddle and plane tables); use scw_recompose with a plan");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(SCW_ERR_UNSUPPORTED, "device ordinal above 63");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      // first call on this device (with it current): the host-side name of the
      // array is not a device address, so ask the runtime for the real one
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
      g_noalloc_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  }

  // the kernels' view of the sizes and scratch pointers, passed by value; it owns nothing
  ItemDev it;
  std::memset(&it, 0, sizeof(it));
  it.M = U * V; it.U = U; it.V = V; it.Fx = Fx; it.Fy = Fy; it.Fz = Fz;
  it.Up = Up;
  it.Vp = Vp;
  it.I = 1;
  it.Fz_out = Fz;
  it.tx = it.ty = 1;
  it.ld = Fx;
  it.pstride = (long long)Fy * Fx;
  it.split_stride = (size_t)Fz * 3 * U * V;
  float2* twx = reinterpret_cast<float2*>(base);
  float2* twy = reinterpret_cast<float2*>(base + b_twx);
  int* ones = reinterpret_cast<int*>(base + b_twx + b_twy);
  int2* entries = reinterpret_cast<int2*>(base + b_twx + b_twy + b_one);
  it.twx = twx;
  it.twy = twy;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (Fx / 8) * Up + (Fy / 8) * Vp + Fz;
  noalloc_setup_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(
      twx, U, Up, Fx, x0 / X, twy, V, Vp, Fy, y0 / Y, ones, entries, Fz);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "noalloc setup launch");
  e = launch_recompose(it, nullptr, entries, Fz, Fx / 8, recompose_smem_bytes(V, Up, Vp),
                       static_cast<const float2*>(S), ones, static_cast<float2*>(out), nullptr, st);
  if (e != cudaSuccess) return cuda_error(e, "recompose launch");
  return SCW_OK;
}
