// Host-only set-up helpers (no CUDA calls).
#pragma once

#include <cstdio>
#include <vector>

#include "mg.h"
#include "mg_internal.h"

namespace mgk {

struct LevelGeom {
  int n[3];
  int off[3];  // nests: origin in parent cells; full levels: 0
  double h;
  bool nest;
};

void laplacian_1d(int order, double* w);
void coarsest_kernel(int order, int m0, int m1, int m2, double h, std::vector<double>& K);
bool build_levels(const mg_config* cfg, std::vector<LevelGeom>& out, int* base_index, char* msg,
                  size_t len);

}  // namespace mgk
