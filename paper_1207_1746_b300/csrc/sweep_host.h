// Host-side pieces shared by the single-grid entry points (sweep.cu) and the
// batched ones (batch.cu): operator validation against grids, launch
// planning and kernel dispatch.
#pragma once

#include <vector>

#include "sweep_kernel.cuh"

namespace gscl {

// Handles resolved and validated for one call.
struct Bound {
  const gscl_stencil *op = nullptr;
  std::vector<Grid> in, out;
  std::vector<gscl_grid> in_h, out_h;
  int64_t lo[3], hi[3];
  bool empty = false;
};

// Tile shape knobs (0 = the default for the dtype).
struct TileCfg {
  int nw = 0;            // warps per CTA
  int pf = 0;            // planes prefetched beyond the stencil's z reach
  bool generic = false;  // interpret the term list even if a compiled structure matches
  bool narrow = false;   // batches, FP32 / BF16: 64-column tiles with 4 rows per warp
  bool compact = false;  // red-black sweeps, IEEE FP64, star family: only the colour's elements
};

bool overlaps(const Grid &a, const Grid &b);

// Validates handles, shapes, dtypes, the range, every term and aliasing
// (Section 3's rules for stencil operators and do_all: an output bound also
// as an input is read only at offset 0).  The other iteration spaces allow
// more reads of such an output, which must then be the same grid:
//  - ordered_axis >= 0 (ordered iteration spaces): one step of ordered_step
//    along ordered_axis (the element visited just before);
//  - colored (red-black colouring): offsets with odd dx + dy + dz;
//  - diamond (do_diamond): dz = 0 and dx, dy of one sign (elements processed
//    before, or after, the core element).
gscl_status bind(const gscl_stencil *op, bool need_value, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                 int32_t n_out, const gscl_range *range, Bound *b, int ordered_axis = -1, int ordered_step = 0,
                 bool colored = false, bool diamond = false);

// Compile-time operator with the descriptor's structure, or OP_GENERIC.
int match_static(const std::vector<gscl_term> &terms, int n_in, int n_out, std::vector<int> *perm);

// Tile geometry, shared-memory ring, term table and the grid's InstDesc.
gscl_status make_plan(const Bound &b, bool reduce, Plan *pl, TileCfg cfg);

// Launches (or, with occupancy_only, sizes) the kernel a plan names.
gscl_status launch(const Plan &pl, int dtype, int red, cudaStream_t stream, int *occupancy_only);
// Current arithmetic of FP64 grids (GSCL_FP64_IEEE or GSCL_FP64_PAIR); make_plan records it in the plan.
int fp64_arith();
bool fp64_int_add();

// Temporal blocking (tb.cu): sweeps fused per pass for a call (K = 1: none)
// and, on 2D grids, the tile shape; one pass from in[0] into out[0]; the
// plan and launch of the 3D kernels; the 2D kernel's launch; the tuner.
struct TbChoice {
  int K = 1;
  int tile = 0;  // 2D grids: index of the tile shape (tb2d_kernel.cuh)
};
bool tb2d_eligible(const Bound &b, int op);
TbChoice tb_choice(const Bound &b, int op, int sweeps);
gscl_status run_tb_pass(const Bound &b, int op, TbChoice c, bool halo_swap, cudaStream_t stream);
gscl_status make_tb_plan(const Bound &b, int K, Plan *pl);
gscl_status launch_tb(const Plan &pl, int dtype, int K, cudaStream_t stream);
// the 3D two-sweep pass (single grids, or a batch's work-list when pl.batch);
// occupancy_only: CTAs per SM instead of a launch
gscl_status launch_tb2_pass(const Plan &pl, int dtype, cudaStream_t stream, int *occupancy_only);
bool tb_eligible(const Bound &b, int op);
struct Tb2dArgs;
gscl_status launch_tb2d(const Plan &pl, int dtype, const Tb2dArgs &a, cudaStream_t stream);
gscl_status tune_sweeps(const Bound &b, int op, int trial_sweeps, cudaStream_t st, int *best_out);

}  // namespace gscl
