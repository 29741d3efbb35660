// Temporal blocking: K sweeps of a radius-1 ping-pong operator per pass over
// HBM (the paper's "wide ghost areas", Section 2, applied on chip).
//
// A CTA owns an xy tile of TX x TY points and streams its column through z.
// All K stages work in one 128 x 16 frame: the tile grown by K - 1 cells on
// each side (TX = 128 - 2(K-1), TY = 16 - 2(K-1), TX rounded down to 16
// bytes), with the main sweep kernel's thread layout (lane l owns columns
// l + 32e, warp w owns rows w and w + 8).  Step s loads plane s of the run
// (z = zb - K + s) of u (input 0) by TMA; stage t = 1..K computes sweep t at
// plane index s - t over the frame, reading sweep t - 1 (the loaded planes
// for t = 1, a padded 3-plane shared-memory ring of sweep t - 1 otherwise);
// stage t's values are valid on the frame shrunk by t - 1 cells, which is
// all stage t + 1 reads; stage K stores the tile.  The right-hand side
// (input 1, read at the core element only) comes straight from global
// memory: each plane is re-read within K steps, from L2.  Points outside the
// interior keep their halo value at every sweep, as single sweeps do; each
// point evaluates the operator's terms in the same order with the same fused
// multiply-adds as sweep_kernel, so K fused sweeps are bit-identical to K
// single sweeps (intermediate sweeps are rounded to the storage type, as a
// single sweep stores them).
#pragma once

#include "sweep_kernel.cuh"

namespace gscl {

template <typename T, int K>
struct TbShape {
  static constexpr int VX = 4, VY = 2, NW = 8;             // 128 x 16 frame, 256 threads
  static constexpr int FW = 32 * VX, FH = NW * VY;
  static constexpr int vec = 16 / (int)sizeof(T);
  static constexpr int TX = (FW - 2 * (K - 1)) / vec * vec;  // tile (x0 stays 16-byte aligned)
  static constexpr int TY = FH - 2 * (K - 1);
  static constexpr int AXK = (K + vec - 1) / vec * vec;      // x apron of the loaded box
  static constexpr int BW0 = TX + 2 * AXK, BH0 = TY + 2 * K;  // u box: tile grown by K (x: by AXK)
  static constexpr int PF = 1;
  static constexpr int R = 3 + PF;                           // loaded planes in the ring
  static constexpr int SE0 = (BW0 * BH0 * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr int SW = FW + 2, SH = FH + 2;             // stage planes, padded by one cell
  static constexpr int SS = (SW * SH + 31) / 32 * 32;
  __host__ __device__ static constexpr size_t smem_bytes(bool) {
    return kBarBytes + sizeof(T) * ((size_t)R * SE0 + (size_t)(K - 1) * 3 * SS);
  }
};

// One point: the operator's terms in table order; u read through a plane
// triple whose pointers sit at the point (row stride RS), the rhs given.
template <class Def, typename T, int RS, int I>
__device__ __forceinline__ void tb_term(const SweepParams &P, const T *up, const T *uc, const T *un,
                                        typename Arith<T>::A f, typename Arith<T>::A &acc) {
  constexpr OpTerm t = Def::table.t[I];
  using A = typename Arith<T>::A;
  A x;
  if constexpr (t.in == 0) {
    const T *pl = t.dz < 0 ? up : (t.dz > 0 ? un : uc);
    x = to_arith(pl[t.dy * RS + t.dx]);
  } else {
    x = f;
  }
  acc = fma(term_weight(P.terms[I], A(0)), x, acc);
}

template <class Def, typename T, int RS, int... I>
__device__ __forceinline__ typename Arith<T>::A tb_point(const SweepParams &P, const T *up, const T *uc, const T *un,
                                                         typename Arith<T>::A f, std::integer_sequence<int, I...>) {
  typename Arith<T>::A acc = 0;
  (tb_term<Def, T, RS, I>(P, up, uc, un, f, acc), ...);
  return acc;
}

template <typename T, int K, class Def>
__global__ void __launch_bounds__(256) tb_kernel(const __grid_constant__ SweepParams P) {
  using S = TbShape<T, K>;
  using A = typename Arith<T>::A;
  constexpr bool RHS = Def::NIN > 1;
  constexpr int R = S::R;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  T *ring0 = reinterpret_cast<T *>(smem + kBarBytes);
  T *stages = ring0 + R * S::SE0;  // sweep t's ring at (t - 1) * 3 * SS
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  if (tid == 0) {
    for (int r = 0; r < R; ++r) mbar_init(&bars[r], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();

  const InstDesc &I = P.inst;
  const int64_t nx = I.hi[0], ny = I.hi[1], nz = I.hi[2];  // the range is the whole interior
  const long long W = (long long)I.tiles_x * I.tiles_y * nz;
  const long long run_end = W * (blockIdx.x + 1) / gridDim.x;
  uint32_t issued = 0, waited = 0;  // planes issued / waited by this CTA (both in order)
  int wslot = 0, islot = 0;
  uint32_t wpar = 0;
  bool ok = true;
  constexpr uint32_t tx_bytes = (uint32_t)(sizeof(T) * S::BW0 * S::BH0);

  for (long long pos = W * blockIdx.x / gridDim.x; pos < run_end;) {
    const long long col = pos / nz;
    const long long zoff = pos - col * nz;
    const int zlen = (int)min(nz - zoff, run_end - pos);
    pos += zlen;
    const int64_t x0 = (int64_t)(col % I.tiles_x) * S::TX;
    const int64_t y0 = (int64_t)(col / I.tiles_x) * S::TY;
    const int64_t zb = zoff;
    const int total = zlen + 2 * K;
    // ring slot of this run's first plane: every plane issued so far has been
    // waited for, so the wait position (the same in every thread) is the issue
    // position (thread 0's alone)
    const int slot_first = wslot;

    auto issue = [&](int s) {
      const int slot = islot;
      islot = islot + 1 == R ? 0 : islot + 1;
      uint64_t *bar = &bars[slot];
      mbar_arrive_expect_tx(bar, tx_bytes);
      tma_load_3d(ring0 + slot * S::SE0, &I.tmap[0], bar, (int)(x0 - S::AXK) + I.cx_add[0], (int)(y0 - K) + I.cy_add[0],
                  (int)(zb - K + s) + I.cz_add[0]);
      ++issued;
    };
    if (tid == 0)
      for (int s = 0; s < min(R, total); ++s) issue(s);

    // this thread's frame points: lx = lane + 32 e, ly = wy + 8 r; tile coords gx = lx - (K-1), gy = ly - (K-1)
    bool xin[S::VX], yin[S::VY];
#pragma unroll
    for (int e = 0; e < S::VX; ++e) {
      const int64_t X = x0 + lane + 32 * e - (K - 1);
      xin[e] = X >= 0 && X < nx;
    }
#pragma unroll
    for (int r = 0; r < S::VY; ++r) {
      const int64_t Y = y0 + wy + 8 * r - (K - 1);
      yin[r] = Y >= 0 && Y < ny;
    }

    // rhs register queue: fq[t - 1] holds this thread's rhs values of plane
    // index s - t (what stage t reads at step s); plane s is loaded during
    // step s, one step before its first use, and shifts down the queue.
    A fq[RHS ? K : 1][S::VY][S::VX];
#pragma unroll
    for (int t = 0; t < (RHS ? K : 1); ++t)
#pragma unroll
      for (int r = 0; r < S::VY; ++r)
#pragma unroll
        for (int e = 0; e < S::VX; ++e) fq[t][r][e] = A(0);

    for (int s = 0; s < total; ++s) {
      A fnext[S::VY][S::VX];
      if constexpr (RHS) {
        const int64_t qn = zb - K + s;
        const bool zin = qn >= 0 && qn < nz;
        const T *f_row = reinterpret_cast<const T *>(I.in[1].base) + qn * I.in[1].plane;
#pragma unroll
        for (int r = 0; r < S::VY; ++r) {
          const int64_t Y = y0 + wy + 8 * r - (K - 1);
#pragma unroll
          for (int e = 0; e < S::VX; ++e) {
            const int64_t X = x0 + lane + 32 * e - (K - 1);
            fnext[r][e] = (zin && yin[r] && xin[e]) ? to_arith(f_row[Y * I.in[1].pitch + X]) : A(0);
          }
        }
      }
      if (ok) {
        ok = mbar_wait_bounded(&bars[wslot], wpar);
        if (ok) {
          ++waited;
          if (++wslot == R) {
            wslot = 0;
            wpar ^= 1u;
          }
        } else {
          s_abort = 1;
          atomicOr(P.err, 1);
        }
      }
      // every thread reaches every barrier below, whether or not its wait succeeded
#pragma unroll
      for (int t = 1; t <= K; ++t) {
        {
          if (ok && s >= 2 * t) {
            const int qi = s - t;                 // plane index of sweep t computed now
            const int64_t q = zb - K + qi;
            const bool zin = q >= 0 && q < nz;
#pragma unroll
            for (int r = 0; r < S::VY; ++r) {
              const int ly = wy + 8 * r;
              const int64_t Y = y0 + ly - (K - 1);
#pragma unroll
              for (int e = 0; e < S::VX; ++e) {
                const int lx = lane + 32 * e;
                const int64_t X = x0 + lx - (K - 1);
                const bool in = zin && yin[r] && xin[e];
                A f = 0;
                if constexpr (RHS) f = fq[t - 1][r][e];
                T val;
                if (t == 1) {
                  const int off = (ly + 1) * S::BW0 + lx - (K - 1) + S::AXK;
                  const T *uc = ring0 + ((slot_first + qi) % R) * S::SE0 + off;
                  if (in) {
                    const T *up = ring0 + ((slot_first + qi - 1) % R) * S::SE0 + off;
                    const T *un = ring0 + ((slot_first + qi + 1) % R) * S::SE0 + off;
                    val = from_arith<T>(
                        tb_point<Def, T, S::BW0>(P, up, uc, un, f, std::make_integer_sequence<int, Def::NT>{}));
                  } else {
                    val = *uc;
                  }
                } else {
                  const T *src = stages + (t - 2) * 3 * S::SS + (ly + 1) * S::SW + lx + 1;
                  const T *uc = src + (qi % 3) * S::SS;
                  if (in) {
                    const T *up = src + ((qi + 2) % 3) * S::SS;
                    const T *un = src + ((qi + 1) % 3) * S::SS;
                    val = from_arith<T>(
                        tb_point<Def, T, S::SW>(P, up, uc, un, f, std::make_integer_sequence<int, Def::NT>{}));
                  } else {
                    val = *uc;
                  }
                }
                if (t < K) {
                  stages[(t - 1) * 3 * S::SS + (qi % 3) * S::SS + (ly + 1) * S::SW + lx + 1] = val;
                } else if (lx >= K - 1 && lx < K - 1 + S::TX && ly >= K - 1 && ly < K - 1 + S::TY && X < nx &&
                           Y < ny) {
                  reinterpret_cast<T *>(I.out[0].base)[q * I.out[0].plane + Y * I.out[0].pitch + X] = val;
                }
              }
            }
          }
        }
        if (t < K) __syncthreads();
      }
      if constexpr (RHS) {
#pragma unroll
        for (int t = K - 1; t > 0; --t)
#pragma unroll
          for (int r = 0; r < S::VY; ++r)
#pragma unroll
            for (int e = 0; e < S::VX; ++e) fq[t][r][e] = fq[t - 1][r][e];
#pragma unroll
        for (int r = 0; r < S::VY; ++r)
#pragma unroll
          for (int e = 0; e < S::VX; ++e) fq[0][r][e] = fnext[r][e];
      }
      __syncthreads();
      if (s_abort) break;
      // loaded plane s - 2 is no longer read: its slot takes plane s - 2 + R
      if (tid == 0 && s >= 2 && s - 2 + R < total) issue(s - 2 + R);
    }
    if (s_abort) break;
  }
  if (s_abort) {
    if (tid == 0)
      for (uint32_t g = waited; g < issued; ++g) mbar_wait_bounded(&bars[g % (uint32_t)R], (g / (uint32_t)R) & 1u);
    __syncthreads();
  }
}

}  // namespace gscl
