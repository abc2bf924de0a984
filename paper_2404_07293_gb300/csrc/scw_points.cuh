// Point-set recomposition (scw_plan_set_points / scw_synthesize_points).
#pragma once

#include "scw_internal.cuh"

namespace scw {

// Tables of one plan's point set. Tensor-core plans: A' = points table [P][3 Kp]
// and B' = spectrum operand [6 Fz][3 Kp] (BF16, split segments hi|hi|lo and
// hi|lo|hi) with their TMA maps; FP32 plans: A [P][2M] and B [6 Fz][2M] (float).
struct PointTables {
  int P = 0, Kp = 0, BN = 0, rows3 = 0;
  bool tc = false;
  size_t bytes = 0;
  double2* d_xy = nullptr;
  void* A = nullptr;
  void* B = nullptr;
  int* d_plane = nullptr;  // per-point output plane (scattered 3-D points), or null
  CUtensorMap mA, mB;
};

// Uploads xy [P][2] (host), builds the points table; synchronises `st`.
scw_status points_build(PointTables** out, const Plan& p, bool tc, const double* xy, int P, cudaStream_t st);
void points_free(PointTables* t);
// spectrum operand from the plan's partial spectra (after steps (a) and (b))
cudaError_t points_prepare(const PointTables& t, const Plan& p, cudaStream_t st);
// scattered 3-D points: plane [P] (host) -> d_plane; null clears
scw_status points_set_planes(PointTables& t, const int* plane, int Fz_out, cudaStream_t st);
// the point product into out [I][3][Fz][P] complex64 (or [I][3][P] with per-point planes)
cudaError_t points_product(const PointTables& t, const Plan& p, float2* out, int* err, uint64_t timeout_ns,
                           cudaStream_t st);

}  // namespace scw
