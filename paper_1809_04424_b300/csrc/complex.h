// complex.h -- the result object behind the opaque vr_complex handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <vector>

#include "../../include/vr.h"

struct vr_complex {
  int32_t n = 0, d = 0, maxdim = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t count[4] = {0, 0, 0, 0};
  int32_t *verts[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t *grade[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t *colptr[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t *rowidx[4] = {nullptr, nullptr, nullptr, nullptr};
  double *grade_value = nullptr;
  int64_t ngrades = 0;
  vr_build_stats stats{};
  // Device flags word as the build's last kernel left it (flags raised after
  // the build's last size read: a bounded wait that gave up, an internal
  // check); read by vr_complex_status and vr_complex_to_host.  Null for
  // batch results (their flags travel in the per-cloud descriptors).
  int32_t *late_flags = nullptr;
  std::vector<void *> allocs;   // device allocations owned by this result
  std::shared_ptr<void> arena;  // shared batch arenas this result views
  bool owned = true;            // false for views into a batch's arenas
  bool in_batch = false;        // owned by a vr_batch: vr_complex_free ignores it
  // Persistence pairs and bars (vr_complex_barcode), device arrays owned by
  // this object whatever `owned` says.
  std::vector<void *> bar_allocs;
  bool pairs_done = false;
  int32_t *killed_by_edge = nullptr;  // dim 0: vertex killed by each edge (-1: none)
  int32_t *vkill = nullptr;           // per vertex: its killing edge (-1: never)
  uint8_t *msf = nullptr;             // per edge: in the spanning forest (zero column of D1)
  int32_t *pair_tri = nullptr;        // per triangle: the edge it kills (-1: none)
  int32_t *pair_edge = nullptr;       // per edge: the triangle killing it (-1: none)
  int32_t *pair_tet = nullptr;        // per tetrahedron: the triangle it kills (-1: none)
  int32_t *pair_tri2 = nullptr;       // per triangle: the tetrahedron killing it (-1: none)
  int64_t nbars[4] = {-1, -1, -1, -1};
  int32_t *bar_birth[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t *bar_death[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace vr {
// Keep stream-ordered pool memory reserved between calls (once per device).
void keep_pool_warm();
vr_status build_dmat(const void *D, int32_t n, vr_dtype dtype, int32_t maxdim, double maxrad, cudaStream_t s,
                     vr_complex *res);
vr_status complex_barcode(vr_complex *c, int dim, cudaStream_t s, int64_t *nbars);
vr_status build_cloud(const void *dpts, int32_t n, int32_t d, vr_dtype dtype, int32_t maxdim, double maxrad,
                      cudaStream_t s, vr_complex *res);
}
