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

// Every staged tile has the same apron (AX columns, RY rows: the largest
// reach of any term) and row width TW = kDT + 2 AX, so element (i, j) of the
// tile sits at j TW + i plus a per-term constant, and a lane's position
// advances by one element per step.
struct DiaTerm {
  int16_t in;      // input grid, or -1: the operator's value
  int16_t coef;    // coefficient grid, or -1
  int16_t direct;  // dz != 0: read from global memory
  int16_t dx, dy, dz;
  int32_t soff;    // staged read: shared-memory offset of the read minus j TW + i
  int32_t coff;    // the coefficient's, likewise
  float wf;
  double wd;
};

struct DiaParams {
  const char *in[kMaxIn];
  int64_t in_pitch[kMaxIn], in_plane[kMaxIn];  // elements
  int64_t in_x0[kMaxIn], in_x1[kMaxIn];        // the grid's storage along x: [-h, n + h)
  int64_t in_y0[kMaxIn], in_y1[kMaxIn];        // ... and along y
  int32_t toff[kMaxIn];                        // element offset of input a's tile (-1: not staged)
  int32_t AX, RY, TW;                          // the common apron and row width
  char *out[kMaxOut_];
  int64_t out_pitch[kMaxOut_], out_plane[kMaxOut_];
  uint32_t alias[kMaxOut_];  // bit a: input a names output m's grid
  DiaTerm terms[kMaxTerms];  // value terms, then output 0's, output 1's, ...
  int32_t n_in, n_out, n_value_terms;
  int32_t out_begin[kMaxOut_ + 1];
  int64_t lo[3], hi[3];
  int32_t d, ti0;  // this launch's tile diagonal and its first tile's column
};

__device__ __forceinline__ double dia_weight(const DiaTerm &t, double) { return t.wd; }
__device__ __forceinline__ float dia_weight(const DiaTerm &t, float) { return t.wf; }

// Compiled operators: the common 2D recurrences with every term's input and
// offset a constant (weights stay runtime values, in P.terms order).  Input 0
// is the output updated in place, input 1 the right-hand side; the reach is
// one element, so tile rows are kDT + 2 wide.  A term is (dx, dy, input).
struct DiaShapeTerm {
  int dx, dy, in;
};
template <int N>
struct DiaShapeTable {
  DiaShapeTerm t[N];
};
enum DiaShapeId { DIA_INTERPRETED = -1, DIA_SAT = 0, DIA_GS5, DIA_GS5F, DIA_SOR5F, DIA_SHAPES };
struct DiaSat {  // x = f + x(i-1,j) + x(i,j-1) - x(i-1,j-1): summed-area table
  static constexpr int NT = 4, NIN = 2;
  static constexpr DiaShapeTable<NT> table = {{{0, 0, 1}, {-1, 0, 0}, {0, -1, 0}, {-1, -1, 0}}};
};
struct DiaGs5 {  // x = sum of the 4 neighbours (natural-order Gauss-Seidel, Laplace)
  static constexpr int NT = 4, NIN = 1;
  static constexpr DiaShapeTable<NT> table = {{{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}}};
};
struct DiaGs5F {  // ... and a right-hand side
  static constexpr int NT = 5, NIN = 2;
  static constexpr DiaShapeTable<NT> table = {{{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}}};
};
struct DiaSor5F {  // x = a x + sum of the 4 neighbours + f: SOR
  static constexpr int NT = 6, NIN = 2;
  static constexpr DiaShapeTable<NT> table = {{{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}}};
};
struct DiaInterpreted {};

template <typename T>
__device__ __forceinline__ typename Arith<T>::A dia_term(const DiaParams &P, const DiaTerm &tm, const T *tiles,
                                                         int pos, int64_t z, int64_t y, int64_t x,
                                                         typename Arith<T>::A v) {
  using A = typename Arith<T>::A;
  A r;
  if (tm.in < 0) {
    r = v;
  } else if (tm.direct) {
    const T *g = reinterpret_cast<const T *>(P.in[tm.in]);
    r = to_arith(g[(z + tm.dz) * P.in_plane[tm.in] + (y + tm.dy) * P.in_pitch[tm.in] + (x + tm.dx)]);
  } else {
    r = to_arith(tiles[pos + tm.soff]);
  }
  if (tm.coef >= 0) r = r * to_arith(tiles[pos + tm.coff]);
  return r;
}

// A compiled term that reads a value the wavefront has just produced: the
// output (input 0) at (i-1, j), (i, j-1) or (i-1, j-1).
GSCL_HD constexpr int dia_wave(const DiaShapeTerm &st) {
  return st.in != 0 ? 0 : (st.dx == -1 && st.dy == 0) ? 1 : (st.dx == 0 && st.dy == -1) ? 2
                                                       : (st.dx == -1 && st.dy == -1) ? 3 : 0;
}

template <class S>
GSCL_HD constexpr bool dia_has_sw() {
  for (int q = 0; q < S::NT; ++q)
    if (dia_wave(S::table.t[q]) == 3) return true;
  return false;
}

// The compiled walk of one tile: lane j computes element (t - j, j) at step
// t.  The values the wavefront produced reach the element in registers: its
// own result of step t - 1 is (i-1, j), lane j-1's results of steps t - 1
// and t - 2 (a warp shuffle) are (i, j-1) and (i-1, j-1); on the tile's first
// column or row they are the staged apron (finished by an earlier launch).
// Every other read (old values at dx, dy >= 0 and the right-hand side) is of
// an element that no step of this launch has written yet, so the reads for
// step t + 1 are issued during step t.  Results are also written to input
// 0's tile for the write-back.  Each element takes the same terms in the
// same order as the interpreted loop.
template <typename T, class S>
__device__ __forceinline__ void dia_walk_compiled(const DiaParams &P, T *tiles, int j, int ni, int nj) {
  using A = typename Arith<T>::A;
  constexpr int TWc = kDT + 2;
  constexpr bool kSW = dia_has_sw<S>();
  T *u = tiles + P.toff[0];
  const int jrow = (j + 1) * TWc + 1;  // tile offset of element (0, j)
  const bool jok = j < nj;
  A pre[S::NT];
#pragma unroll
  for (int q = 0; q < S::NT; ++q) pre[q] = A(0);
  // the reads of element (i, j) that the wavefront does not produce
  auto prefetch = [&](int i) {
    if (jok && i >= 0 && i < ni) {
      const int pos = jrow + i;
      static_for<S::NT>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr DiaShapeTerm st = S::table.t[q];
        if constexpr (dia_wave(st) == 0) pre[q] = to_arith(tiles[P.toff[st.in] + pos + st.dy * TWc + st.dx]);
      });
    }
  };
  prefetch(-j);
  A prev1 = A(0), prev2 = A(0);  // this lane's results of the last two steps
  for (int t = 0; t < ni + nj - 1; ++t) {
    const int i = t - j;
    const A up1 = __shfl_up_sync(0xffffffffu, prev1, 1);
    A up2 = A(0);
    if constexpr (kSW) up2 = __shfl_up_sync(0xffffffffu, prev2, 1);
    A cur[S::NT];
#pragma unroll
    for (int q = 0; q < S::NT; ++q) cur[q] = pre[q];
    prefetch(i + 1);
    A res = A(0);
    if (jok && i >= 0 && i < ni) {
      const int pos = jrow + i;
      A o = A(0);
      static_for<S::NT>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr DiaShapeTerm st = S::table.t[q];
        constexpr int wv = dia_wave(st);
        A x;
        if constexpr (wv == 1) x = i > 0 ? prev1 : to_arith(u[pos - 1]);
        else if constexpr (wv == 2) x = j > 0 ? up1 : to_arith(u[pos - TWc]);
        else if constexpr (wv == 3) x = (i > 0 && j > 0) ? up2 : to_arith(u[pos - TWc - 1]);
        else x = cur[q];
        o = fma(dia_weight(P.terms[q], A(0)), x, o);
      });
      const T r = from_arith<T>(o);
      u[pos] = r;
      res = to_arith(r);
    }
    prev2 = prev1;
    prev1 = res;
  }
}

template <typename T, class S>
__global__ void __launch_bounds__(kDT) diamond_kernel(const __grid_constant__ DiaParams P) {
  using A = typename Arith<T>::A;
  extern __shared__ __align__(16) unsigned char dia_smem[];
  T *tiles = reinterpret_cast<T *>(dia_smem);
  const int lane = threadIdx.x;
  const int ti = P.ti0 + (int)blockIdx.x, tj = P.d - ti;
  const int64_t z = P.lo[2] + blockIdx.y;
  const int64_t x0 = P.lo[0] + (int64_t)ti * kDT, y0 = P.lo[1] + (int64_t)tj * kDT;
  const int TW = P.TW, rows = kDT + 2 * P.RY;

  // stage each input's tile and apron; cells outside the grid's storage are
  // skipped (no term reads them: the binding checked every read of the range).
  // FP32 / FP64: cp.async, so every row of every tile is in flight at once.
  for (int a = 0; a < P.n_in; ++a) {
    if (P.toff[a] < 0) continue;
    const T *g = reinterpret_cast<const T *>(P.in[a]) + z * P.in_plane[a];
    T *t = tiles + P.toff[a];
    for (int r = 0; r < rows; ++r) {
      const int64_t y = y0 - P.RY + r;
      if (y < P.in_y0[a] || y >= P.in_y1[a]) continue;
      for (int c = lane; c < TW; c += 32) {
        const int64_t x = x0 - P.AX + c;
        if (x < P.in_x0[a] || x >= P.in_x1[a]) continue;
        if constexpr (sizeof(T) >= 4) {
          const uint32_t sa = (uint32_t)__cvta_generic_to_shared(t + r * TW + c);
          const T *src = g + y * P.in_pitch[a] + x;
          if constexpr (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
          else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
        } else {
          t[r * TW + c] = g[y * P.in_pitch[a] + x];
        }
      }
    }
  }
  if constexpr (sizeof(T) >= 4) asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();

  const int j = lane;
  const int64_t y = y0 + j;
  const int ni = (int)min((int64_t)kDT, P.hi[0] - x0), nj = (int)min((int64_t)kDT, P.hi[1] - y0);
  const int centre = P.RY * TW + P.AX;  // offset of the core element of a staged read
  if constexpr (!std::is_same<S, DiaInterpreted>::value) {
    dia_walk_compiled<T, S>(P, tiles, j, ni, nj);
  } else {
    for (int t = 0; t < ni + nj - 1; ++t) {
      const int i = t - j;
      if (j < nj && i >= 0 && i < ni) {
        const int pos = j * TW + i;
        A v = A(0);
        for (int q = 0; q < P.n_value_terms; ++q) {
          const DiaTerm &tm = P.terms[q];
          v = fma(dia_weight(tm, A(0)), dia_term<T>(P, tm, tiles, pos, z, y, x0 + i, v), v);
        }
        A o[kMaxOut_];
#pragma unroll
        for (int m = 0; m < kMaxOut_; ++m) {
          o[m] = A(0);
          if (m < P.n_out)
            for (int q = P.out_begin[m]; q < P.out_begin[m + 1]; ++q) {
              const DiaTerm &tm = P.terms[q];
              o[m] = fma(dia_weight(tm, A(0)), dia_term<T>(P, tm, tiles, pos, z, y, x0 + i, v), o[m]);
            }
        }
        // every output of this element is computed before any is stored
#pragma unroll
        for (int m = 0; m < kMaxOut_; ++m) {
          if (m >= P.n_out) continue;
          const T val = from_arith<T>(o[m]);
          if (P.alias[m]) {
            for (int a = 0; a < P.n_in; ++a)
              if ((P.alias[m] >> a) & 1u) tiles[P.toff[a] + pos + centre] = val;
          } else {
            reinterpret_cast<T *>(P.out[m])[z * P.out_plane[m] + y * P.out_pitch[m] + (x0 + i)] = val;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();

  // outputs updated in shared memory go back with coalesced rows
  for (int m = 0; m < P.n_out; ++m) {
    if (!P.alias[m]) continue;
    const int a = __ffs((int)P.alias[m]) - 1;
    T *g = reinterpret_cast<T *>(P.out[m]) + z * P.out_plane[m];
    const T *t = tiles + P.toff[a] + centre;
    for (int r = 0; r < nj; ++r)
      for (int c = lane; c < ni; c += 32) g[(y0 + r) * P.out_pitch[m] + x0 + c] = t[r * TW + c];
  }
}

template <typename T, class S>
gscl_status launch_diamond_s(DiaParams &P, size_t smem, int tiles_x, int tiles_y, int planes, cudaStream_t st) {
  auto kern = diamond_kernel<T, S>;
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

template <typename T>
gscl_status launch_diamond_t(DiaParams &P, int shape, size_t smem, int tiles_x, int tiles_y, int planes,
                             cudaStream_t st) {
  switch (shape) {
    case DIA_SAT: return launch_diamond_s<T, DiaSat>(P, smem, tiles_x, tiles_y, planes, st);
    case DIA_GS5: return launch_diamond_s<T, DiaGs5>(P, smem, tiles_x, tiles_y, planes, st);
    case DIA_GS5F: return launch_diamond_s<T, DiaGs5F>(P, smem, tiles_x, tiles_y, planes, st);
    case DIA_SOR5F: return launch_diamond_s<T, DiaSor5F>(P, smem, tiles_x, tiles_y, planes, st);
  }
  return launch_diamond_s<T, DiaInterpreted>(P, smem, tiles_x, tiles_y, planes, st);
}

struct DiaShapeDesc {
  int id, nt, nin;
  const DiaShapeTerm *t;
};

template <class S>
DiaShapeDesc dia_desc(int id) {
  return DiaShapeDesc{id, S::NT, S::NIN, S::table.t};
}

// The compiled shape of a call: one output, bound also as input 0 and as no
// other input, no value terms, no coefficients, every term in the table's
// order with the table's offsets (GSCL_GENERIC_ONLY=1: none).
int diamond_shape(const gscl_stencil *op, int n_in, int n_out, const DiaParams &P) {
  const char *env = getenv("GSCL_GENERIC_ONLY");
  if (env && env[0] && env[0] != '0') return DIA_INTERPRETED;
  if (n_out != 1 || P.alias[0] != 1u || P.AX != 1 || P.RY != 1) return DIA_INTERPRETED;
  static const DiaShapeDesc shapes[] = {dia_desc<DiaSat>(DIA_SAT), dia_desc<DiaGs5>(DIA_GS5),
                                        dia_desc<DiaGs5F>(DIA_GS5F), dia_desc<DiaSor5F>(DIA_SOR5F)};
  for (const DiaShapeDesc &d : shapes) {
    if (d.nt != op->n_terms || d.nin != n_in) continue;
    bool ok = true;
    for (int q = 0; q < d.nt && ok; ++q) {
      const gscl_term &tm = op->terms[q];
      ok = tm.out == 0 && tm.coef == GSCL_NONE && tm.dz == 0 && tm.in == d.t[q].in && tm.dx == d.t[q].dx &&
           tm.dy == d.t[q].dy;
    }
    if (ok) return d.id;
  }
  return DIA_INTERPRETED;
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
  // the common apron: the largest x / y reach of any staged read
  int AX = 0, RY = 0;
  bool staged[kMaxIn] = {};
  for (int t = 0; t < op->n_terms; ++t) {
    const gscl_term &tm = op->terms[t];
    if (tm.coef != GSCL_NONE) staged[tm.coef] = true;
    if (tm.in == GSCL_VALUE || tm.dz != 0) continue;
    staged[tm.in] = true;
    AX = std::max(AX, abs((int)tm.dx));
    RY = std::max(RY, abs((int)tm.dy));
  }
  for (int m = 0; m < n_out; ++m)  // an output updated in place is staged even if no term reads it
    for (int a = 0; a < n_in; ++a)
      if (overlaps(b.out[m], b.in[a])) staged[a] = true;
  const int TW = kDT + 2 * AX;
  const int tile = (TW * (kDT + 2 * RY) + align - 1) / align * align;
  P.AX = AX;
  P.RY = RY;
  P.TW = TW;
  int base = 0;
  for (int a = 0; a < n_in; ++a) {
    const Grid &g = b.in[a];
    P.in[a] = g.elem_ptr(0, 0, 0);
    P.in_pitch[a] = g.pitch;
    P.in_plane[a] = g.plane;
    P.in_x0[a] = -g.halo[0];
    P.in_x1[a] = g.n[0] + g.halo[0];
    P.in_y0[a] = -g.halo[1];
    P.in_y1[a] = g.n[1] + g.halo[1];
    P.toff[a] = staged[a] ? base : -1;
    if (staged[a]) base += tile;
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
  // value terms, then each output's terms, each group in descriptor order
  int nt = 0;
  auto push = [&](const gscl_term &tm) {
    DiaTerm &d = P.terms[nt++];
    d.in = tm.in == GSCL_VALUE ? -1 : (int16_t)tm.in;
    d.coef = tm.coef == GSCL_NONE ? -1 : (int16_t)tm.coef;
    d.dx = tm.dx;
    d.dy = tm.dy;
    d.dz = tm.dz;
    d.direct = (int16_t)(d.in >= 0 && tm.dz != 0);
    d.soff = (d.in >= 0 && !d.direct) ? P.toff[d.in] + (RY + tm.dy) * TW + AX + tm.dx : 0;
    d.coff = d.coef >= 0 ? P.toff[d.coef] + RY * TW + AX : 0;
    d.wf = (float)tm.w;
    d.wd = tm.w;
  };
  for (int t = 0; t < op->n_terms; ++t)
    if (op->terms[t].out == GSCL_VALUE) push(op->terms[t]);
  P.n_value_terms = nt;
  for (int m = 0; m < n_out; ++m) {
    P.out_begin[m] = nt;
    for (int t = 0; t < op->n_terms; ++t)
      if (op->terms[t].out == m) push(op->terms[t]);
  }
  P.out_begin[n_out] = nt;
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = b.lo[a];
    P.hi[a] = b.hi[a];
  }
  const int tiles_x = (int)((b.hi[0] - b.lo[0] + kDT - 1) / kDT);
  const int tiles_y = (int)((b.hi[1] - b.lo[1] + kDT - 1) / kDT);
  const int shape = diamond_shape(op, n_in, n_out, P);
  cudaStream_t st = (cudaStream_t)stream;
  switch (b.in[0].dtype) {
    case GSCL_F64: return launch_diamond_t<double>(P, shape, smem, tiles_x, tiles_y, (int)planes, st);
    case GSCL_F32: return launch_diamond_t<float>(P, shape, smem, tiles_x, tiles_y, (int)planes, st);
    case GSCL_BF16: return launch_diamond_t<__nv_bfloat16>(P, shape, smem, tiles_x, tiles_y, (int)planes, st);
  }
  return fail(GSCL_ERR_DTYPE, "unknown dtype");
}
