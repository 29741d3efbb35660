// do_diamond (Section 3): the cells (i-1, j) and (i, j-1) are processed before
// the cell (i, j).  The paper has it for 2D grids; a 3D grid is taken plane by
// plane, the planes independent of each other.
//
// The range of every plane is cut into 32 x 32 tiles.  Once the tile
// diagonals 0 .. d-1 are done, the tiles (ti, tj) with ti + tj = d depend on
// nothing still to come, so one launch per tile diagonal processes them, one
// warp per tile and plane.  Inside its tile the warp walks the tile's own
// anti-diagonals: at step t lane j computes element (t - j, j), whose
// predecessors (i-1, j) and (i, j-1) were computed at step t - 1.
//
// Every input's tile, with the apron its reads need, is staged in shared
// memory with coalesced row loads.  An output bound also as an input is
// updated in that tile as the wavefront passes, so later elements read the
// new values, and written back with coalesced rows at the end; other outputs
// are stored directly.  What each read sees is fixed by the order: at offsets
// with dx, dy <= 0 an element already processed (by this warp, or by an
// earlier diagonal's launch), at dx, dy >= 0 one not yet processed (later in
// this warp, or in a later launch).  Reads with mixed signs would depend on
// the schedule, and the binding rejects them for an output (GSCL_ERR_ALIAS).
// Terms reading another plane (dz != 0) read global memory directly; they
// never name an output.
#include <algorithm>

#include "sweep_host.h"
#include "sweep_kernel.cuh"

namespace gscl {
namespace {

constexpr int kDT = 32;  // tile side (one lane per tile row)

struct DiaTerm {
  int16_t in;    // input grid, or -1: the operator's value
  int16_t coef;  // coefficient grid, or -1
  int16_t out;   // output, or -1: a term of the value
  int16_t dx, dy, dz;
  int16_t direct;  // dz != 0: read from global memory
  int16_t pad;
  float wf;
  double wd;
};

struct DiaParams {
  const char *in[kMaxIn];
  int64_t in_pitch[kMaxIn], in_plane[kMaxIn];  // elements
  int64_t in_x0[kMaxIn], in_x1[kMaxIn];        // the grid's storage along x: [-h, n + h)
  int64_t in_y0[kMaxIn], in_y1[kMaxIn];        // ... and along y
  int32_t ax[kMaxIn], ry[kMaxIn];              // apron of input a's tile
  int32_t tw[kMaxIn];                          // its row width, kDT + 2 ax
  int32_t toff[kMaxIn];                        // its element offset in shared memory
  char *out[kMaxOut_];
  int64_t out_pitch[kMaxOut_], out_plane[kMaxOut_];
  uint32_t alias[kMaxOut_];  // bit a: input a names output m's grid
  DiaTerm terms[kMaxTerms];
  int32_t n_in, n_out, n_terms;
  int64_t lo[3], hi[3];
  int32_t d, ti0;  // this launch's tile diagonal and its first tile's column
};

__device__ __forceinline__ double dia_weight(const DiaTerm &t, double) { return t.wd; }
__device__ __forceinline__ float dia_weight(const DiaTerm &t, float) { return t.wf; }

template <typename T>
__global__ void __launch_bounds__(kDT) diamond_kernel(const __grid_constant__ DiaParams P) {
  using A = typename Arith<T>::A;
  extern __shared__ __align__(16) unsigned char dia_smem[];
  T *tiles = reinterpret_cast<T *>(dia_smem);
  const int lane = threadIdx.x;
  const int ti = P.ti0 + (int)blockIdx.x, tj = P.d - ti;
  const int64_t z = P.lo[2] + blockIdx.y;
  const int64_t x0 = P.lo[0] + (int64_t)ti * kDT, y0 = P.lo[1] + (int64_t)tj * kDT;

  // stage each input's tile and apron; cells outside the grid's storage are
  // skipped (no term reads them: the binding checked every read of the range)
  for (int a = 0; a < P.n_in; ++a) {
    const T *g = reinterpret_cast<const T *>(P.in[a]) + z * P.in_plane[a];
    T *t = tiles + P.toff[a];
    const int rows = kDT + 2 * P.ry[a], w = P.tw[a];
    for (int r = 0; r < rows; ++r) {
      const int64_t y = y0 - P.ry[a] + r;
      if (y < P.in_y0[a] || y >= P.in_y1[a]) continue;
      for (int c = lane; c < w; c += 32) {
        const int64_t x = x0 - P.ax[a] + c;
        if (x >= P.in_x0[a] && x < P.in_x1[a]) t[r * w + c] = g[y * P.in_pitch[a] + x];
      }
    }
  }
  __syncwarp();

  const int j = lane;
  const int64_t y = y0 + j;
  const int ni = (int)min((int64_t)kDT, P.hi[0] - x0), nj = (int)min((int64_t)kDT, P.hi[1] - y0);
  for (int t = 0; t < ni + nj - 1; ++t) {
    const int i = t - j;
    if (j < nj && i >= 0 && i < ni) {
      A v = A(0);
      A o[kMaxOut_];
#pragma unroll
      for (int m = 0; m < kMaxOut_; ++m) o[m] = A(0);
      for (int q = 0; q < P.n_terms; ++q) {  // value terms come first
        const DiaTerm &tm = P.terms[q];
        A x;
        if (tm.in < 0) {
          x = v;
        } else if (tm.direct) {
          const T *g = reinterpret_cast<const T *>(P.in[tm.in]);
          x = to_arith(g[(z + tm.dz) * P.in_plane[tm.in] + (y + tm.dy) * P.in_pitch[tm.in] + (x0 + i + tm.dx)]);
        } else {
          const int a = tm.in;
          x = to_arith(tiles[P.toff[a] + (j + P.ry[a] + tm.dy) * P.tw[a] + (i + P.ax[a] + tm.dx)]);
        }
        if (tm.coef >= 0) {
          const int c = tm.coef;
          x = x * to_arith(tiles[P.toff[c] + (j + P.ry[c]) * P.tw[c] + (i + P.ax[c])]);
        }
        const A w = dia_weight(tm, A(0));
        if (tm.out < 0) {
          v = fma(w, x, v);
        } else {
#pragma unroll
          for (int m = 0; m < kMaxOut_; ++m)
            if (tm.out == m) o[m] = fma(w, x, o[m]);
        }
      }
      // every output of this element is computed before any is stored
#pragma unroll
      for (int m = 0; m < kMaxOut_; ++m) {
        if (m >= P.n_out) continue;
        const T val = from_arith<T>(o[m]);
        if (P.alias[m]) {
          for (int a = 0; a < P.n_in; ++a)
            if ((P.alias[m] >> a) & 1u) tiles[P.toff[a] + (j + P.ry[a]) * P.tw[a] + (i + P.ax[a])] = val;
        } else {
          reinterpret_cast<T *>(P.out[m])[z * P.out_plane[m] + y * P.out_pitch[m] + (x0 + i)] = val;
        }
      }
    }
    __syncwarp();
  }

  // outputs updated in shared memory go back with coalesced rows
  for (int m = 0; m < P.n_out; ++m) {
    if (!P.alias[m]) continue;
    const int a = __ffs((int)P.alias[m]) - 1;
    T *g = reinterpret_cast<T *>(P.out[m]) + z * P.out_plane[m];
    const T *t = tiles + P.toff[a];
    for (int r = 0; r < nj; ++r)
      for (int c = lane; c < ni; c += 32) g[(y0 + r) * P.out_pitch[m] + x0 + c] = t[(r + P.ry[a]) * P.tw[a] + c + P.ax[a]];
  }
}

template <typename T>
gscl_status launch_diamond_t(DiaParams &P, size_t smem, int tiles_x, int tiles_y, int planes, cudaStream_t st) {
  auto kern = diamond_kernel<T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "do_diamond set-up");
  }
  for (int d = 0; d < tiles_x + tiles_y - 1; ++d) {
    const int t0 = std::max(0, d - (tiles_y - 1)), t1 = std::min(d, tiles_x - 1);
    P.d = d;
    P.ti0 = t0;
    kern<<<dim3((unsigned)(t1 - t0 + 1), (unsigned)planes), kDT, smem, st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "do_diamond launch");
  }
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" gscl_status gscl_do_diamond(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                                       int32_t n_out, const gscl_range *range, void *stream) {
  if (!op) return fail(GSCL_ERR_INVALID, "do_diamond needs an operator");
  if (n_out < 1) return fail(GSCL_ERR_INVALID, "do_diamond needs an output");
  Bound b;
  if (gscl_status s = bind(op, false, in, n_in, out, n_out, range, &b, -1, 0, false, true)) return s;
  if (b.empty) return GSCL_OK;
  const int64_t planes = b.hi[2] - b.lo[2];
  if (planes > 65535) return fail(GSCL_ERR_UNSUPPORTED, "do_diamond takes at most 65535 planes per call");
  DiaParams P;
  memset(&P, 0, sizeof P);
  P.n_in = n_in;
  P.n_out = n_out;
  const int elem = b.in[0].elem;
  const int align = 16 / elem;
  int base = 0;
  for (int a = 0; a < n_in; ++a) {
    const Grid &g = b.in[a];
    int ax = 0, ry = 0;
    for (int t = 0; t < op->n_terms; ++t) {
      const gscl_term &tm = op->terms[t];
      if (tm.in != a) continue;
      ax = std::max(ax, abs((int)tm.dx));
      ry = std::max(ry, abs((int)tm.dy));
    }
    P.in[a] = g.elem_ptr(0, 0, 0);
    P.in_pitch[a] = g.pitch;
    P.in_plane[a] = g.plane;
    P.in_x0[a] = -g.halo[0];
    P.in_x1[a] = g.n[0] + g.halo[0];
    P.in_y0[a] = -g.halo[1];
    P.in_y1[a] = g.n[1] + g.halo[1];
    P.ax[a] = ax;
    P.ry[a] = ry;
    P.tw[a] = kDT + 2 * ax;
    P.toff[a] = base;
    base += (P.tw[a] * (kDT + 2 * ry) + align - 1) / align * align;
  }
  const size_t smem = (size_t)base * elem;
  if (smem > (size_t)max_smem_per_block())
    return fail(GSCL_ERR_UNSUPPORTED, "do_diamond needs %zu bytes of shared memory for its tiles", smem);
  for (int m = 0; m < n_out; ++m) {
    const Grid &g = b.out[m];
    P.out[m] = g.elem_ptr(0, 0, 0);
    P.out_pitch[m] = g.pitch;
    P.out_plane[m] = g.plane;
    for (int a = 0; a < n_in; ++a)
      if (overlaps(g, b.in[a])) P.alias[m] |= 1u << a;  // bind has checked it is the same grid
  }
  // value terms first, then the outputs' terms, each group in descriptor order
  int nt = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < op->n_terms; ++t) {
      const gscl_term &tm = op->terms[t];
      if ((tm.out == GSCL_VALUE) != (pass == 0)) continue;
      DiaTerm &d = P.terms[nt++];
      d.in = tm.in == GSCL_VALUE ? -1 : (int16_t)tm.in;
      d.coef = tm.coef == GSCL_NONE ? -1 : (int16_t)tm.coef;
      d.out = tm.out == GSCL_VALUE ? -1 : (int16_t)tm.out;
      d.dx = tm.dx;
      d.dy = tm.dy;
      d.dz = tm.dz;
      d.direct = (int16_t)(d.in >= 0 && tm.dz != 0);
      d.wf = (float)tm.w;
      d.wd = tm.w;
    }
  P.n_terms = nt;
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = b.lo[a];
    P.hi[a] = b.hi[a];
  }
  const int tiles_x = (int)((b.hi[0] - b.lo[0] + kDT - 1) / kDT);
  const int tiles_y = (int)((b.hi[1] - b.lo[1] + kDT - 1) / kDT);
  cudaStream_t st = (cudaStream_t)stream;
  switch (b.in[0].dtype) {
    case GSCL_F64: return launch_diamond_t<double>(P, smem, tiles_x, tiles_y, (int)planes, st);
    case GSCL_F32: return launch_diamond_t<float>(P, smem, tiles_x, tiles_y, (int)planes, st);
    case GSCL_BF16: return launch_diamond_t<__nv_bfloat16>(P, smem, tiles_x, tiles_y, (int)planes, st);
  }
  return fail(GSCL_ERR_DTYPE, "unknown dtype");
}
