// Internal declarations shared by the host runtime and the kernel launchers
// of libgscl.so.  Nothing here is part of the C ABI (include/gscl.h).
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (header only; the driver is reached at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gscl.h"

namespace gscl {

// A grid handle's state.  The buffer is borrowed (Section 3: a grid is a
// storage object plus the stencil shape that fixes its halo).
struct Grid {
  int32_t ndim = 0;
  int32_t dtype = 0;
  int32_t elem = 0;  // bytes per element
  int64_t n[3] = {1, 1, 1};
  int32_t halo[3] = {0, 0, 0};
  int64_t pitch = 0;   // elements per row
  int64_t off = 0;     // leading pad (elements)
  int64_t plane = 0;   // elements per z plane
  int64_t bytes = 0;   // storage size
  char *buf = nullptr; // borrowed device buffer
  int64_t buf_bytes = 0;
  int device = -1;
  // address of interior element (i, j, k); i, j, k may be negative (halo)
  char *elem_ptr(int64_t i, int64_t j, int64_t k) const {
    return buf + elem * (off + ((k + halo[2]) * (n[1] + 2 * halo[1]) + (j + halo[1])) * pitch + (i + halo[0]));
  }
};

int32_t dtype_bytes(int32_t dtype);
gscl_status compute_layout(int32_t ndim, const int64_t n[3], const int32_t halo[3], int32_t dtype, Grid *g);

// Handle registry: copies a live grid's state into *out, or GSCL_ERR_STATE.
gscl_status lookup(gscl_grid h, Grid *out);
// Exchanges the storage of two live handles of identical layout.
gscl_status swap_storage(gscl_grid a, gscl_grid b);

// Per-thread error detail for gscl_last_error().
gscl_status fail(gscl_status s, const char *fmt, ...);
gscl_status cuda_fail(cudaError_t e, const char *what);

// Device-side error word of the current device (bounded-wait timeouts).
int *device_error_word();
// After a synchronisation: reads and clears the word; GSCL_ERR_TIMEOUT or
// GSCL_ERR_RANGE if a flag was set, GSCL_OK otherwise.
gscl_status take_device_error();

// Tensor-map encoder reached through the runtime's driver entry point.
gscl_status encode_tensor_map_3d(CUtensorMap *map, const Grid &g, uint32_t box_x, uint32_t box_y);

int sm_count();
int max_smem_per_block();
int smem_per_sm();  // shared memory of one SM (all resident CTAs together)

}  // namespace gscl
