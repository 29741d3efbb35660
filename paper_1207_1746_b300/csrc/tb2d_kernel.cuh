// Temporal blocking of 2D radius-1 operators (the 5-point Jacobi family):
// K sweeps per launch, the paper's wide ghost areas (Section 2) held in
// shared memory.  A 2D grid of a few MB is swept in a few microseconds, so
// its single sweeps are bound by the launch and the grid-wide dependence
// between sweeps, not by memory or arithmetic; fusing K sweeps pays K - 1
// of those for each launch, at the price of recomputing a frame of K cells
// around each tile.
//
// A CTA owns a TX x TY tile.  It loads the tile grown by K cells on each side
// (the frame) into two shared buffers: buffer 0 gets in[0]'s interior and
// the halo iterate j0 has under single sweeps, buffer 1 the halo iterate
// j0 + 1 has (only points outside the interior).  Stage s = 1..K computes
// sweep j0 + s on the tile grown by K - s cells (the points whose inputs
// stage s - 1 produced), from buffer (s odd ? 0 : 1) into the other; points
// outside the interior are never written, so each buffer keeps its halo.
// Stage K stores the tile to out[0].  Every point evaluates the operator's
// terms in table order with the fused multiply-adds the single sweep uses,
// and each stage is rounded to the storage type as a single sweep stores it,
// so a pass is bit-identical to K single sweeps.
//
// Single sweeps leave iterate j in in[0]'s storage (of the call) for even j
// and in out[0]'s for odd j, each with that grid's halo.  A run of fused
// passes and single sweeps puts iterate j0 (the input of launch L0) in
// in[0]'s storage when L0 is even: when j0 and L0 differ in parity the
// iterate sits in the other grid, and the pass takes its halos swapped
// (`halo_swap`), so grids whose halos differ still see single sweeps' halos.
// The host also keeps the number of launches of a run of the parity of its
// sweeps, so each handle ends naming the storage single sweeps leave it.
#pragma once

#include <vector>

#include "sweep_kernel.cuh"

namespace gscl {

// A launch's tiles: single grids enumerate theirs from the tile count along
// x; batches pass a list of (instance, x0, y0) triples.
struct Tb2dArgs {
  const int4 *tiles;  // batches: one entry per tile; nullptr for a single grid
  int32_t n_tiles, tiles_x;
  int32_t K, TX, TY;
  int32_t halo_swap;  // 1: buffer 0 takes out[0]'s halo and buffer 1 in[0]'s
};

// Tile shapes the planner and the tuners choose from (index into this list).
constexpr int kTb2dShapes = 4;
__host__ __device__ constexpr int tb2d_tile_x(int i) { return i == 0 ? 32 : i == 1 ? 32 : i == 2 ? 16 : 64; }
__host__ __device__ constexpr int tb2d_tile_y(int i) { return i == 0 ? 16 : i == 1 ? 32 : i == 2 ? 16 : 32; }
constexpr int kTb2dMaxK = 16;
constexpr int kTb2dThreads = 512;  // 16 warps

template <typename T>
__host__ __device__ constexpr size_t tb2d_smem_bytes(int K, int TX, int TY) {
  return 2 * sizeof(T) * (size_t)(TX + 2 * K) * (size_t)(TY + 2 * K);
}

// Sizes of the sweeps of each launch of a run of `sweeps` sweeps with up to
// K fused per launch: fused passes while more than K sweeps remain (the last
// launch stays a single sweep, so in[0] ends holding the previous iterate),
// and, when the launch count and the sweep count differ in parity, the last
// pass shortened by one sweep (one launch more), so the handles end naming
// the storage single sweeps leave them.
inline std::vector<int> tb_launch_plan(int sweeps, int K) {
  std::vector<int> sizes;
  for (int done = 0; done < sweeps;) {
    const int k = (K > 1 && sweeps - done > K) ? K : 1;
    sizes.push_back(k);
    done += k;
  }
  if (((long long)sizes.size() - sweeps) % 2 != 0) {
    for (int i = (int)sizes.size() - 1; i >= 0; --i)
      if (sizes[i] > 1) {
        const int k = sizes[i];
        sizes[i] = k - 1;
        sizes.insert(sizes.begin() + i + 1, 1);
        break;
      }
  }
  return sizes;
}

// 2D compile-time operators the kernel takes: one input and one output, every
// term reading input 0 within one cell in x and y, no coefficient grid, no
// returned value.
template <class Def>
__host__ __device__ constexpr bool tb2d_capable() {
  if (Def::NIN != 1 || Def::NOUT != 1) return false;
  for (int i = 0; i < Def::NT; ++i) {
    const OpTerm &t = Def::table.t[i];
    if (t.in != 0 || t.coef >= 0 || t.out != 0 || t.dz != 0) return false;
    if (t.dx < -1 || t.dx > 1 || t.dy < -1 || t.dy > 1) return false;
  }
  return true;
}

// One point of stage s: the terms in table order from `cur` (frame row
// stride FW), as the single sweep evaluates them.
template <typename T, class Def>
__device__ __forceinline__ typename Arith<T>::A tb2d_point(const T *cur, int FW, int fy, int fx,
                                                           const typename Arith<T>::A (&w)[Def::NT]) {
  using A = typename Arith<T>::A;
  A acc = A(0);
  static_for<Def::NT>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr OpTerm tm = Def::table.t[i];
    acc = fma(w[i], to_arith(cur[(fy + tm.dy) * FW + fx + tm.dx]), acc);
  });
  return acc;
}

template <typename T, class Def>
__global__ void __launch_bounds__(kTb2dThreads) tb2d_kernel(const __grid_constant__ SweepParams P, const Tb2dArgs a) {
  static_assert(tb2d_capable<Def>(), "tb2d_kernel takes 2D radius-1 single-input operators");
  using A = typename Arith<T>::A;
  constexpr int NWARP = kTb2dThreads / 32;
  // every extern __shared__ array of a translation unit is one symbol: keep
  // the 128-byte alignment the TMA kernels compiled beside this one declare
  extern __shared__ __align__(128) unsigned char tb2d_smem[];
  const int K = a.K, FW = a.TX + 2 * K, FH = a.TY + 2 * K;
  T *buf0 = reinterpret_cast<T *>(tb2d_smem);
  T *buf1 = buf0 + FW * FH;
  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  A w[Def::NT];
#pragma unroll
  for (int i = 0; i < Def::NT; ++i) w[i] = term_weight(P.terms[i], A(0));
  // the previous sweep (or pass) wrote in[0]
  pdl_wait();

  for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    int inst = 0;
    int64_t x0, y0;
    if (a.tiles) {
      const int4 d = a.tiles[t];
      inst = d.x;
      x0 = d.y;
      y0 = d.z;
    } else {
      x0 = (int64_t)(t % a.tiles_x) * a.TX;
      y0 = (int64_t)(t / a.tiles_x) * a.TY;
    }
    const InstDesc &I = P.insts ? P.insts[inst] : P.inst;
    const int64_t nx = I.hi[0], ny = I.hi[1];  // the range is the whole interior
    const T *src = reinterpret_cast<const T *>(I.in[0].base);
    T *dst = reinterpret_cast<T *>(I.out[0].base);
    const int64_t sp = I.in[0].pitch, dp = I.out[0].pitch;
    // halos of iterates j0 (buffer 0) and j0 + 1 (buffer 1)
    const T *h0 = a.halo_swap ? dst : src;
    const T *h1 = a.halo_swap ? src : dst;
    const int64_t hp0 = a.halo_swap ? dp : sp, hp1 = a.halo_swap ? sp : dp;

    // the frame, within one cell of the interior; zeros farther out, where no
    // stage reads
    for (int fy = wy; fy < FH; fy += NWARP) {
      const int64_t Y = y0 - K + fy;
      for (int fx = lane; fx < FW; fx += 32) {
        const int64_t X = x0 - K + fx;
        const bool near = X >= -1 && X <= nx && Y >= -1 && Y <= ny;
        const bool inside = X >= 0 && X < nx && Y >= 0 && Y < ny;
        buf0[fy * FW + fx] = inside ? src[Y * sp + X] : (near ? h0[Y * hp0 + X] : from_arith<T>(A(0)));
        buf1[fy * FW + fx] = (near && !inside) ? h1[Y * hp1 + X] : from_arith<T>(A(0));
      }
    }
    __syncthreads();

    for (int s = 1; s <= K; ++s) {
      const T *cur = (s & 1) ? buf0 : buf1;
      T *nxt = (s & 1) ? buf1 : buf0;
      // the stage's region (the tile grown by K - s cells), its points dealt
      // to the threads in order, two per thread per round (two independent
      // FMA chains): no lane idles on rows narrower than a warp, which
      // matters since the FP64 pipe binds
      const int rw = FW - 2 * s, rn = rw * (FH - 2 * s);
      for (int i0 = tid; i0 < rn; i0 += 2 * kTb2dThreads) {
        const int i1 = i0 + kTb2dThreads;
        const int fy0 = s + i0 / rw, fx0 = s + i0 % rw;
        const int fy1 = i1 < rn ? s + i1 / rw : fy0, fx1 = i1 < rn ? s + i1 % rw : fx0;
        const int64_t Y0 = y0 - K + fy0, X0 = x0 - K + fx0, Y1 = y0 - K + fy1, X1 = x0 - K + fx1;
        const bool in0 = X0 >= 0 && X0 < nx && Y0 >= 0 && Y0 < ny;
        const bool in1 = i1 < rn && X1 >= 0 && X1 < nx && Y1 >= 0 && Y1 < ny;
        if (!in0 && !in1) continue;
        const A v0 = tb2d_point<T, Def>(cur, FW, fy0, fx0, w);
        const A v1 = tb2d_point<T, Def>(cur, FW, fy1, fx1, w);
        if (s < K) {
          if (in0) nxt[fy0 * FW + fx0] = from_arith<T>(v0);
          if (in1) nxt[fy1 * FW + fx1] = from_arith<T>(v1);
        } else {  // stage K covers exactly the tile
          if (in0) dst[Y0 * dp + X0] = from_arith<T>(v0);
          if (in1) dst[Y1 * dp + X1] = from_arith<T>(v1);
        }
      }
      __syncthreads();
    }
  }
  // this CTA's work is done: the next launch may begin (it waits for this grid)
  pdl_launch_dependents();
}

}  // namespace gscl
