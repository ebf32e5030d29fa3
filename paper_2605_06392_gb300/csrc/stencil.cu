// Spatial base matrices of the synthetic SPDE-like models on a regular grid
// (Section II-A: Q_p is built from sparse spatial and temporal base matrices).
//   Cm = I, G = 5-point graph Laplacian with natural boundary (degree on the
//   diagonal, -1 per grid neighbour), GG = G G (13-point stencil).
// All three are returned on GG's pattern (which contains G's and Cm's), in
// CSR with sorted columns: the layout inla_model_spec expects.
#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"

extern "C" bta_status inla_grid_stencil(int32_t nx, int32_t ny, int32_t* nnz, int32_t* row_ptr,
                                        int32_t* col, double* val_C, double* val_G,
                                        double* val_GG) {
  if (nx < 1 || ny < 1 || !nnz) return BTA_ERR_ARG;
  const int ns = nx * ny;
  std::vector<std::map<int, double>> G(ns);
  for (int iy = 0; iy < ny; ++iy)
    for (int ix = 0; ix < nx; ++ix) {
      int s = iy * nx + ix;
      G[s][s] += 0.0;
      const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
      for (int q = 0; q < 4; ++q) {
        int jx = ix + dx[q], jy = iy + dy[q];
        if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) continue;
        G[s][jy * nx + jx] -= 1.0;
        G[s][s] += 1.0;
      }
    }
  std::vector<std::map<int, double>> GG(ns);
  for (int s = 0; s < ns; ++s)
    for (const auto& [r, gr] : G[s])
      for (const auto& [c, gc] : G[r]) GG[s][c] += gr * gc;
  int64_t total = 0;
  for (int s = 0; s < ns; ++s) total += (int64_t)GG[s].size();
  if (!row_ptr) {
    *nnz = (int32_t)total;
    return BTA_OK;
  }
  if (*nnz < total || !col || !val_C || !val_G || !val_GG) return BTA_ERR_ARG;
  int32_t e = 0;
  row_ptr[0] = 0;
  for (int s = 0; s < ns; ++s) {
    for (const auto& [c, v] : GG[s]) {
      col[e] = c;
      auto it = G[s].find(c);
      val_G[e] = it == G[s].end() ? 0.0 : it->second;
      val_C[e] = c == s ? 1.0 : 0.0;
      val_GG[e] = v;
      ++e;
    }
    row_ptr[s + 1] = e;
  }
  *nnz = e;
  return BTA_OK;
}
