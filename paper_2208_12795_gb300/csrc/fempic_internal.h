// Library-internal declarations shared by the host mesh builder and the CUDA
// translation unit.  Not part of the public ABI (see include/fempic_env.h).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "fempic_env.h"

namespace fempic {

// Local topology of a tet with sorted nodes.
constexpr int kLocalEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
constexpr int kLocalFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
constexpr int kWallOther = -7;  // boundary face not on a bbox plane
constexpr int kMaxSpecies = 8;

struct HostMesh {
  int64_t nn = 0, ne = 0, nf = 0, nt = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  std::vector<double> xyz;       // [nn][3]
  std::vector<int32_t> tn;       // [nt][4] sorted node ids
  std::vector<int32_t> en;       // [ne][2]
  std::vector<int32_t> fn;       // [nf][3]
  std::vector<int32_t> te;       // [nt][6]
  std::vector<int32_t> tf;       // [nt][4]
  std::vector<int32_t> nb;       // [nt][4] neighbour or wall code
  std::vector<double> geom;      // [nt][12]: x0, grad l1, grad l2, grad l3
  // point-location grid: every tet listed in each cell its bbox overlaps
  int gd[3] = {1, 1, 1};
  double ginv[3] = {0, 0, 0};
  std::vector<int64_t> gstart;   // [ncell + 1]
  std::vector<int32_t> gtet;     // ascending tet ids per cell
};

// Builds every table from the raw description.  Returns FEMPIC_OK or an error
// code with a message in *err.
int build_host_mesh(const fempic_mesh_desc& d, HostMesh* m, std::string* err);

// Cell index along axis a (monotone in x, clamped): shared by the host grid
// builder and the device query so that both agree exactly.
inline int grid_cell(double x, double lo, double ginv, int gd) {
  double f = __builtin_floor((x - lo) * ginv);
  if (!(f >= 0.0)) return 0;
  if (f > (double)(gd - 1)) return gd - 1;
  return (int)f;
}

// Precision form of an env (FEMPIC_FP64 or FEMPIC_MIXED).
int env_precision(const fempic_env* env);

// The env's device status counters (fempic_stats order).  In the debug
// build (FEMPIC_BOUNDS_CHECK) slot 3 counts mesh-table indices found out of
// range and skipped; kernels of other translation units that read mesh
// tables count there too, so that fempic_error_count reports them.
unsigned long long* env_stats(fempic_env* env);

// Every host-side argument check of fempic_push_step, without device work:
// FEMPIC_OK or the code and message fempic_push_step would return.
int validate_push_step(const fempic_particles* p, const fempic_envelope* envl, double omega0, double t,
                       double dt);

}  // namespace fempic
