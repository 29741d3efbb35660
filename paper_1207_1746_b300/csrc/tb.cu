// Host side of temporal blocking (tb2_kernel.cuh, tb_kernel.cuh for 3D grids,
// tb2d_kernel.cuh for 2D grids): eligibility, planning, launching and tuning
// of K fused sweeps per pass.
#include <stdlib.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sweep_host.h"
#include "tb2_kernel.cuh"
#include "tb2d_kernel.cuh"
#include "tb_kernel.cuh"

namespace gscl {
namespace {

template <typename T, int K, bool RHS>
constexpr bool tb_fits() {
  return TbShape<T, K>::smem_bytes(RHS) <= 227 * 1024;
}

template <typename T, int K, class Def>
gscl_status launch_tb_t(const Plan &pl, cudaStream_t stream) {
  using S = TbShape<T, K>;
  constexpr bool RHS = Def::NIN > 1;
  if constexpr (!tb_fits<T, K, RHS>()) {
    return fail(GSCL_ERR_UNSUPPORTED, "temporal factor %d does not fit in shared memory", K);
  } else {
    auto kern = tb_kernel<T, K, Def>;
    constexpr size_t smem = S::smem_bytes(RHS);
    // the shared-memory attribute is per device: set it, and ask the
    // occupancy, once on each device the kernel runs on
    constexpr int kDevices = 64;
    static std::mutex mu;
    static int per_sm_of[kDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kDevices) return fail(GSCL_ERR_UNSUPPORTED, "device %d beyond the supported count", dev);
    int per_sm = 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      if (!per_sm_of[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
        if (e != cudaSuccess) return cuda_fail(e, "temporal-blocking kernel set-up");
        per_sm_of[dev] = nb > 0 ? nb : 1;
      }
      per_sm = per_sm_of[dev];
    }
    const long long ctas = std::min<long long>(pl.work, (long long)sm_count() * per_sm);
    if (ctas < 1) return GSCL_OK;
    kern<<<(unsigned)ctas, 256, smem, stream>>>(pl.P);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "temporal-blocking kernel launch");
  }
}

template <typename T, int K>
gscl_status launch_tb_op(const Plan &pl, cudaStream_t stream) {
  switch (pl.op) {
    case OP_STAR7: return launch_tb_t<T, K, OpStar7>(pl, stream);
    case OP_HEAT7_RHS: return launch_tb_t<T, K, OpHeat7Rhs>(pl, stream);
    case OP_JACOBI7_RHS: return launch_tb_t<T, K, OpJacobi7Rhs>(pl, stream);
  }
  return fail(GSCL_ERR_INVALID, "no temporal-blocking kernel for operator %d", pl.op);
}

// K = 2: the vector-lane kernel (tb2_kernel.cuh), one wave with programmatic
// dependent launch like the single sweeps; batches (pl.batch) launch its
// work-list form over pl.batch_ctas CTAs.  occupancy_only: report the CTAs
// per SM instead of launching.
template <typename T, class Def, bool BATCH>
gscl_status launch_tb2_t(const Plan &pl, cudaStream_t stream, int *occupancy_only) {
  auto kern = tb2_kernel<T, Def, BATCH>;
  constexpr size_t smem = Tb2Shape<T>::smem_bytes();
  constexpr int kDevices = 64;
  static std::mutex mu;
  static int per_sm_of[kDevices] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kDevices) return fail(GSCL_ERR_UNSUPPORTED, "device %d beyond the supported count", dev);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!per_sm_of[dev]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int nb = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
      if (e != cudaSuccess) return cuda_fail(e, "two-sweep kernel set-up");
      per_sm_of[dev] = nb > 0 ? nb : 1;
    }
    per_sm = per_sm_of[dev];
  }
  if (occupancy_only) {
    *occupancy_only = per_sm;
    return GSCL_OK;
  }
  const long long ctas = BATCH ? (long long)pl.batch_ctas : std::min<long long>(pl.work, (long long)sm_count() * per_sm);
  if (ctas < 1) return GSCL_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, pl.P);
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "two-sweep kernel launch");
}

template <typename T, class Def>
gscl_status launch_tb2_def(const Plan &pl, cudaStream_t stream, int *occupancy_only) {
  return pl.batch ? launch_tb2_t<T, Def, true>(pl, stream, occupancy_only)
                  : launch_tb2_t<T, Def, false>(pl, stream, occupancy_only);
}

template <typename T>
gscl_status launch_tb2(const Plan &pl, cudaStream_t stream, int *occupancy_only = nullptr) {
  switch (pl.op) {
    case OP_STAR7: return launch_tb2_def<T, OpStar7>(pl, stream, occupancy_only);
    case OP_HEAT7_RHS: return launch_tb2_def<T, OpHeat7Rhs>(pl, stream, occupancy_only);
    case OP_JACOBI7_RHS: return launch_tb2_def<T, OpJacobi7Rhs>(pl, stream, occupancy_only);
  }
  return fail(GSCL_ERR_INVALID, "no temporal-blocking kernel for operator %d", pl.op);
}

template <typename T>
gscl_status launch_tb_k(const Plan &pl, int K, cudaStream_t stream) {
  switch (K) {
    case 2: return launch_tb2<T>(pl, stream);
    case 3: return launch_tb_op<T, 3>(pl, stream);
    case 4: return launch_tb_op<T, 4>(pl, stream);
  }
  return fail(GSCL_ERR_UNSUPPORTED, "temporal factor %d", K);
}

// ---- 2D grids: K sweeps per launch over tiles of one of the kTb2dShapes shapes
template <typename T, class Def>
gscl_status launch_tb2d_t(const Plan &pl, const Tb2dArgs &a, cudaStream_t stream) {
  auto kern = tb2d_kernel<T, Def>;
  constexpr size_t kMaxSmem = tb2d_smem_bytes<T>(kTb2dMaxK, 64, 32);
  const size_t smem = tb2d_smem_bytes<T>(a.K, a.TX, a.TY);
  if (a.K < 2 || a.K > kTb2dMaxK || smem > kMaxSmem) return fail(GSCL_ERR_UNSUPPORTED, "temporal factor %d", a.K);
  // the shared-memory attribute is per device; occupancy per (device, bytes)
  constexpr int kDevices = 64;
  static std::mutex mu;
  static bool attr_set[kDevices] = {};
  static std::map<std::pair<int, size_t>, int> per_sm_of;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kDevices) return fail(GSCL_ERR_UNSUPPORTED, "device %d beyond the supported count", dev);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr_set[dev]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
      if (e != cudaSuccess) return cuda_fail(e, "2D temporal-blocking kernel set-up");
      attr_set[dev] = true;
    }
    auto it = per_sm_of.find(std::make_pair(dev, smem));
    if (it == per_sm_of.end()) {
      int nb = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kTb2dThreads, smem);
      if (e != cudaSuccess) return cuda_fail(e, "2D temporal-blocking occupancy");
      it = per_sm_of.emplace(std::make_pair(dev, smem), nb > 0 ? nb : 1).first;
    }
    per_sm = it->second;
  }
  const long long ctas = std::min<long long>(a.n_tiles, (long long)sm_count() * per_sm);
  if (ctas < 1) return GSCL_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(kTb2dThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, pl.P, a);
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "2D temporal-blocking kernel launch");
}

template <typename T>
gscl_status launch_tb2d_op(const Plan &pl, const Tb2dArgs &a, cudaStream_t stream) {
  switch (pl.op) {
    case OP_JACOBI5_2D: return launch_tb2d_t<T, OpJacobi5_2D>(pl, a, stream);
  }
  return fail(GSCL_ERR_INVALID, "no 2D temporal-blocking kernel for operator %d", pl.op);
}

// The tile arguments of a single 2D grid.
Tb2dArgs tb2d_single_args(const Grid &g, int K, int tile, bool halo_swap) {
  Tb2dArgs a{};
  a.halo_swap = halo_swap ? 1 : 0;
  a.K = K;
  a.TX = tb2d_tile_x(tile);
  a.TY = tb2d_tile_y(tile);
  a.tiles_x = (int32_t)((g.n[0] + a.TX - 1) / a.TX);
  a.n_tiles = a.tiles_x * (int32_t)((g.n[1] + a.TY - 1) / a.TY);
  a.tiles = nullptr;
  return a;
}

template <typename T>
int max_factor(int) {
  if (tb_fits<T, 4, true>()) return 4;
  if (tb_fits<T, 3, true>()) return 3;
  return 2;
}

}  // namespace

gscl_status launch_tb2_pass(const Plan &pl, int dtype, cudaStream_t stream, int *occupancy_only) {
  if (dtype == GSCL_F32) return launch_tb2<float>(pl, stream, occupancy_only);
  if (dtype == GSCL_BF16) return launch_tb2<__nv_bfloat16>(pl, stream, occupancy_only);
  return fail(GSCL_ERR_DTYPE, "two-sweep passes are for FP32 / BF16 storage");
}

gscl_status launch_tb2d(const Plan &pl, int dtype, const Tb2dArgs &a, cudaStream_t stream) {
  switch (dtype) {
    case GSCL_F64: return launch_tb2d_op<double>(pl, a, stream);
    case GSCL_F32: return launch_tb2d_op<float>(pl, a, stream);
    case GSCL_BF16: return launch_tb2d_op<__nv_bfloat16>(pl, a, stream);
  }
  return fail(GSCL_ERR_DTYPE, "no 2D temporal blocking for dtype %d", dtype);
}

// Temporal factors (and 2D tile shapes) chosen by gscl_tune_sweeps, per
// (operator, dtype, extent).
std::mutex g_tb_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int64_t>, TbChoice> g_tb_tuned;

std::tuple<int, int, int64_t, int64_t, int64_t> tb_key(int op, const Grid &g) {
  return std::make_tuple(op, g.dtype, g.n[0], g.n[1], g.n[2]);
}

// 2D radius-1 single-input operators over the whole interior of a grid of
// one plane, any storage (IEEE arithmetic for FP64 grids: the pair kernels'
// rounding differs).
bool tb2d_eligible(const Bound &b, int op) {
  if (op != OP_JACOBI5_2D || b.in.size() != 1 || b.out.size() != 1) return false;
  const Grid &g = b.in[0];
  if (g.n[2] != 1) return false;
  if (g.dtype == GSCL_F64 && fp64_arith() != GSCL_FP64_IEEE) return false;
  if (g.dtype != GSCL_F64 && g.dtype != GSCL_F32 && g.dtype != GSCL_BF16) return false;
  for (int a = 0; a < 3; ++a)
    if (b.lo[a] != 0 || b.hi[a] != g.n[a]) return false;
  return true;
}

bool tb_eligible(const Bound &b, int op) {
  if (tb2d_eligible(b, op)) return true;
  if (op != OP_STAR7 && op != OP_HEAT7_RHS && op != OP_JACOBI7_RHS) return false;
  const Grid &g = b.in[0];
  if (g.ndim != 3 || (g.dtype != GSCL_F32 && g.dtype != GSCL_BF16)) return false;
  for (int a = 0; a < 3; ++a)
    if (b.lo[a] != 0 || b.hi[a] != g.n[a]) return false;
  return true;
}

// Sweeps fused per pass for this call (K = 1: none), and for 2D grids the
// tile shape: GSCL_TEMPORAL=K (and GSCL_TEMPORAL_TILE for the 2D shape) if
// set, else what gscl_tune_sweeps measured for this operator, dtype and
// extent, else 1.  On B300 single 7-point sweeps of 3D grids outrun fused
// ones (the tuner keeps K = 1 there), while small 2D grids, whose sweeps
// are bound by launches, gain from fusing.  Only the radius-1 star
// operators in FP32 / BF16 over the whole interior of a 3D grid and the 2D
// 5-point operators qualify: FP64 3D sweeps are bound by the FP64 pipe,
// where the redundant halo work of fused sweeps costs more than the bytes
// it saves.
TbChoice tb_choice(const Bound &b, int op, int sweeps) {
  TbChoice c;
  if (sweeps < 2 || !tb_eligible(b, op)) return c;
  const Grid &g = b.in[0];
  if (const char *e = getenv("GSCL_TEMPORAL")) {
    c.K = atoi(e);
    if (const char *t = getenv("GSCL_TEMPORAL_TILE")) c.tile = std::max(0, std::min(kTb2dShapes - 1, atoi(t)));
  } else {
    std::lock_guard<std::mutex> lk(g_tb_mu);
    auto it = g_tb_tuned.find(tb_key(op, g));
    if (it != g_tb_tuned.end()) c = it->second;
  }
  int kmax;
  if (tb2d_eligible(b, op)) kmax = kTb2dMaxK;
  else kmax = g.dtype == GSCL_F32 ? max_factor<float>(op) : max_factor<__nv_bfloat16>(op);
  c.K = std::max(1, std::min(c.K, std::min(kmax, sweeps)));
  return c;
}

// The single-sweep plan with its tiles and tensor-map boxes replaced by the
// temporal-blocking tile (TX x TY grown by K) for the same operator.
template <typename T>
void tb_geometry(int K, int *TX, int *TY, int *BW0, int *BH0) {
  switch (K) {
    case 2: *TX = TbShape<T, 2>::TX, *TY = TbShape<T, 2>::TY, *BW0 = TbShape<T, 2>::BW0, *BH0 = TbShape<T, 2>::BH0; break;
    case 3: *TX = TbShape<T, 3>::TX, *TY = TbShape<T, 3>::TY, *BW0 = TbShape<T, 3>::BW0, *BH0 = TbShape<T, 3>::BH0; break;
    default: *TX = TbShape<T, 4>::TX, *TY = TbShape<T, 4>::TY, *BW0 = TbShape<T, 4>::BW0, *BH0 = TbShape<T, 4>::BH0;
  }
}

gscl_status make_tb_plan(const Bound &b, int K, Plan *pl) {
  if (gscl_status s = make_plan(b, false, pl, TileCfg{})) return s;
  const Grid &g = b.in[0];
  if (K == 2) {
    // 128 x 14 output tiles; u boxes (128 + 2 AX) x 18, f boxes 128 x 16
    const int AX = 16 / g.elem;
    SweepParams &P = pl->P;
    if (gscl_status s = encode_tensor_map_3d(&P.inst.tmap[0], b.in[0], (uint32_t)(128 + 2 * AX), 18)) return s;
    if (b.in.size() > 1)
      if (gscl_status s = encode_tensor_map_3d(&P.inst.tmap[1], b.in[1], 128, 16)) return s;
    P.inst.x_base = 0;
    P.inst.y_base = 0;
    P.inst.tiles_x = (int32_t)((g.n[0] + 127) / 128);
    P.inst.tiles_y = (int32_t)((g.n[1] + 13) / 14);
    pl->work = (long long)P.inst.tiles_x * P.inst.tiles_y * g.n[2];
    return GSCL_OK;
  }
  int TX, TY, BW0, BH0;
  if (g.dtype == GSCL_F32) tb_geometry<float>(K, &TX, &TY, &BW0, &BH0);
  else tb_geometry<__nv_bfloat16>(K, &TX, &TY, &BW0, &BH0);
  SweepParams &P = pl->P;
  if (gscl_status s = encode_tensor_map_3d(&P.inst.tmap[0], b.in[0], (uint32_t)BW0, (uint32_t)BH0)) return s;
  P.inst.x_base = 0;
  P.inst.y_base = 0;
  P.inst.tiles_x = (int32_t)((g.n[0] + TX - 1) / TX);
  P.inst.tiles_y = (int32_t)((g.n[1] + TY - 1) / TY);
  pl->work = (long long)P.inst.tiles_x * P.inst.tiles_y * g.n[2];
  return GSCL_OK;
}

// One pass of c.K sweeps from in[0] into out[0]; halo_swap (2D grids): the
// pass's input iterate has out[0]'s halo under single sweeps (tb2d_kernel.cuh).
gscl_status run_tb_pass(const Bound &b, int op, TbChoice c, bool halo_swap, cudaStream_t stream) {
  Plan pl;
  if (tb2d_eligible(b, op)) {
    if (gscl_status s = make_plan(b, false, &pl, TileCfg{})) return s;
    return launch_tb2d(pl, b.in[0].dtype, tb2d_single_args(b.in[0], c.K, c.tile, halo_swap), stream);
  }
  if (gscl_status s = make_tb_plan(b, c.K, &pl)) return s;
  return launch_tb(pl, b.in[0].dtype, c.K, stream);
}

gscl_status launch_tb(const Plan &pl, int dtype, int K, cudaStream_t stream) {
  if (dtype == GSCL_F32) return launch_tb_k<float>(pl, K, stream);
  if (dtype == GSCL_BF16) return launch_tb_k<__nv_bfloat16>(pl, K, stream);
  return fail(GSCL_ERR_DTYPE, "temporal blocking is for FP32 / BF16 storage");
}

// Times the candidate factors (3D grids: K = 1 .. 4; 2D grids: K = 1, 2, 3,
// 4, 6, 8, 12, 16 over every tile shape) on the caller's grids, passes from
// in[0] into out[0] (at least 48 sweeps per candidate on 2D grids, whose
// passes take microseconds), and records the fastest per sweep.
gscl_status tune_sweeps(const Bound &b, int op, int trial_sweeps, cudaStream_t st, int *best_out) {
  TbChoice best;
  *best_out = 1;
  if (!tb_eligible(b, op)) return GSCL_OK;
  const Grid &g = b.in[0];
  const bool two_d = tb2d_eligible(b, op);
  std::vector<TbChoice> cands;
  cands.push_back(TbChoice{});
  if (two_d) {
    for (int K : {2, 3, 4, 6, 8, 12, 16})
      for (int t = 0; t < kTb2dShapes; ++t) cands.push_back(TbChoice{K, t});
  } else {
    const int kmax = g.dtype == GSCL_F32 ? max_factor<float>(op) : max_factor<__nv_bfloat16>(op);
    for (int K = 2; K <= kmax; ++K) cands.push_back(TbChoice{K, 0});
  }
  const int trial = two_d ? std::max(trial_sweeps, 48) : trial_sweeps;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  Plan single;
  const bool have_single = make_plan(b, false, &single, TileCfg{}) == GSCL_OK;
  for (const TbChoice &c : cands) {
    if (c.K == 1 && !have_single) continue;
    auto once = [&] {
      return c.K == 1 ? launch(single, g.dtype, RED_NONE, st, nullptr) : run_tb_pass(b, op, c, false, st);
    };
    if (once() != GSCL_OK) continue;  // warm-up (and kernel set-up)
    const int passes = std::max(1, trial / c.K);
    cudaEventRecord(e0, st);
    for (int i = 0; i < passes; ++i) once();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const float per_sweep = ms / (passes * c.K);
    if (per_sweep < best_ms) {
      best_ms = per_sweep;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tb_mu);
    g_tb_tuned[tb_key(op, g)] = best;
  }
  *best_out = best.K;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "temporal tuning launches");
}

}  // namespace gscl
