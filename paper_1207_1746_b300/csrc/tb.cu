// Host side of temporal blocking (tb_kernel.cuh): eligibility, planning and
// launching of K fused sweeps per pass.
#include <stdlib.h>

#include <mutex>

#include "sweep_host.h"
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
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [&] {
      attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int nb = 0;
      if (attr_err == cudaSuccess) attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
      per_sm = nb > 0 ? nb : 1;
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "temporal-blocking kernel set-up");
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

template <typename T>
gscl_status launch_tb_k(const Plan &pl, int K, cudaStream_t stream) {
  switch (K) {
    case 2: return launch_tb_op<T, 2>(pl, stream);
    case 3: return launch_tb_op<T, 3>(pl, stream);
    case 4: return launch_tb_op<T, 4>(pl, stream);
  }
  return fail(GSCL_ERR_UNSUPPORTED, "temporal factor %d", K);
}

template <typename T>
int max_factor(int op) {
  const bool rhs = op != OP_STAR7;
  if (rhs ? tb_fits<T, 4, true>() : tb_fits<T, 4, false>()) return 4;
  if (rhs ? tb_fits<T, 3, true>() : tb_fits<T, 3, false>()) return 3;
  return 2;
}

}  // namespace

// Sweeps fused per pass for this call (1: none).  Only the radius-1 star
// operators in FP32 / BF16 over the whole interior of a 3D grid qualify:
// FP64 sweeps are bound by the FP64 pipe, where the redundant halo work of
// fused sweeps costs more than the bytes it saves.
int tb_factor(const Bound &b, int op, int sweeps) {
  if (sweeps < 2 || (op != OP_STAR7 && op != OP_HEAT7_RHS && op != OP_JACOBI7_RHS)) return 1;
  const Grid &g = b.in[0];
  if (g.ndim != 3 || (g.dtype != GSCL_F32 && g.dtype != GSCL_BF16)) return 1;
  for (int a = 0; a < 3; ++a)
    if (b.lo[a] != 0 || b.hi[a] != g.n[a]) return 1;
  int K = 2;
  if (const char *e = getenv("GSCL_TEMPORAL")) K = atoi(e);
  const int kmax = g.dtype == GSCL_F32 ? max_factor<float>(op) : max_factor<__nv_bfloat16>(op);
  K = std::max(1, std::min(K, std::min(kmax, sweeps)));
  return K;
}

// The single-sweep plan with its tiles and tensor-map boxes replaced by the
// temporal-blocking tile (TX x TY grown by K) for the same operator.
gscl_status make_tb_plan(const Bound &b, int K, Plan *pl) {
  if (gscl_status s = make_plan(b, false, pl, TileCfg{})) return s;
  const Grid &g = b.in[0];
  int TX, TY, BW0, BH0, BWF, BHF;
  if (g.dtype == GSCL_F32) {
    using S2 = TbShape<float, 2>;
    TX = S2::TX;
    TY = S2::TY;
    const int vec = 16 / 4, axk = (K + vec - 1) / vec * vec;
    BW0 = TX + 2 * axk;
    BH0 = TY + 2 * K;
    BWF = BW0;
    BHF = TY + 2 * (K - 1);
  } else {
    using S2 = TbShape<__nv_bfloat16, 2>;
    TX = S2::TX;
    TY = S2::TY;
    const int vec = 16 / 2, axk = (K + vec - 1) / vec * vec;
    BW0 = TX + 2 * axk;
    BH0 = TY + 2 * K;
    BWF = BW0;
    BHF = TY + 2 * (K - 1);
  }
  SweepParams &P = pl->P;
  if (gscl_status s = encode_tensor_map_3d(&P.inst.tmap[0], b.in[0], (uint32_t)BW0, (uint32_t)BH0)) return s;
  if (b.in.size() > 1)
    if (gscl_status s = encode_tensor_map_3d(&P.inst.tmap[1], b.in[1], (uint32_t)BWF, (uint32_t)BHF)) return s;
  P.inst.x_base = 0;
  P.inst.y_base = 0;
  P.inst.tiles_x = (int32_t)((g.n[0] + TX - 1) / TX);
  P.inst.tiles_y = (int32_t)((g.n[1] + TY - 1) / TY);
  pl->work = (long long)P.inst.tiles_x * P.inst.tiles_y * g.n[2];
  return GSCL_OK;
}

gscl_status launch_tb(const Plan &pl, int dtype, int K, cudaStream_t stream) {
  if (dtype == GSCL_F32) return launch_tb_k<float>(pl, K, stream);
  if (dtype == GSCL_BF16) return launch_tb_k<__nv_bfloat16>(pl, K, stream);
  return fail(GSCL_ERR_DTYPE, "temporal blocking is for FP32 / BF16 storage");
}

}  // namespace gscl
