// scw_recompose_noalloc: the recompose step (x-pass + y-pass of scw_recompose)
// for callers that cannot allocate device memory. Its scratch -- the twiddle
// tables, a per-plane split count and the x-pass rows T -- lives in one
// file-scope __device__ array instead of a plan's cudaMalloc'ed workspace.
// The kernels are the library's own x-pass and y-pass, unchanged.
#include <mutex>

#include "scw_internal.cuh"

namespace scw {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // SCW_NOALLOC_SCRATCH_BYTES in scw.h

// Shared by every call on a device; held by each device that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device addresses of g_noalloc_scratch, looked up once per device.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {nullptr};

// Twiddles exp(2 pi i (u b / F + u x0 / X)) with the argument reduced in FP64
// (same tables a plan builds on the host) and the all-ones split count.
__global__ void noalloc_setup_kernel(float2* twx, int U, int Fx, double x0_over_X, float2* twy, int V, int Fy,
                                     double y0_over_Y, int* ones, int Fz) {
  const int Qx = Fx / 8, Qy = Fy / 8;
  const int nx = Qx * U, ny = Qy * V;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx + ny + Fz; i += gridDim.x * blockDim.x) {
    if (i < nx + ny) {
      const bool isx = i < nx;
      const int k = isx ? i : i - nx;
      const int n = isx ? U : V;
      const int b = k / n, idx = k - b * n;
      const int u = idx - n / 2;
      const double t = isx ? ((double)u * b / Fx + u * x0_over_X) : ((double)u * b / Fy + u * y0_over_Y);
      const double r = t - rint(t);
      double s, c;
      sincospi(2.0 * r, &s, &c);
      (isx ? twx : twy)[k] = make_float2((float)c, (float)s);
    } else {
      ones[i - nx - ny] = 1;
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

  // scratch layout: twx | twy | ones | T, each 256-byte aligned
  const size_t b_twx = align256(sizeof(float2) * (size_t)(Fx / 8) * U);
  const size_t b_twy = align256(sizeof(float2) * (size_t)(Fy / 8) * V);
  const size_t b_one = align256(sizeof(int) * (size_t)Fz);
  const size_t b_T = sizeof(float2) * (size_t)Fz * 3 * V * Fx;
  const size_t need = b_twx + b_twy + b_one + b_T;
  if (need > kNoAllocScratchBytes)
    return set_error(SCW_ERR_UNSUPPORTED, "scw_recompose_noalloc needs " + std::to_string(need) +
                                              " bytes of scratch, above its fixed " +
                                              std::to_string(kNoAllocScratchBytes) +
                                              " (3 Fz V Fx complex64 plus tables); use scw_recompose with a plan");

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

  Plan p;  // a stack descriptor of the sizes and scratch pointers; it owns nothing
  p.U = U; p.V = V; p.M = U * V; p.Fx = Fx; p.Fy = Fy; p.Fz = Fz;
  p.X = X; p.Y = Y; p.x0 = x0; p.y0 = y0;
  p.d_twx = reinterpret_cast<float2*>(base);
  p.d_twy = reinterpret_cast<float2*>(base + b_twx);
  int* ones = reinterpret_cast<int*>(base + b_twx + b_twy);
  p.T = reinterpret_cast<float2*>(base + b_twx + b_twy + b_one);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (Fx / 8) * U + (Fy / 8) * V + Fz;
  noalloc_setup_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(
      p.d_twx, U, Fx, x0 / X, p.d_twy, V, Fy, y0 / Y, ones, Fz);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "noalloc setup launch");
  e = launch_xpass(p, static_cast<const float2*>(S), Fz, ones, st);
  if (e != cudaSuccess) return cuda_error(e, "x-pass launch");
  e = launch_ypass(p, static_cast<float2*>(out), st);
  if (e != cudaSuccess) return cuda_error(e, "y-pass launch");
  return SCW_OK;
}
