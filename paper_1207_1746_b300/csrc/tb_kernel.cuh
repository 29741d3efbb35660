// Temporal blocking: K sweeps of a radius-1 ping-pong operator per pass over
// HBM (the paper's "wide ghost areas", Section 2, applied on chip).
//
// A CTA owns an xy tile of TX x TY points and streams its column through z.
// Step s loads plane z_s = zb - K + s of u (input 0) and of the right-hand
// side (input 1, if any) by TMA; stage t = 1..K then computes sweep t at
// plane z_s - t over the tile grown by K - t cells on each side, reading
// sweep t - 1 (the loaded planes for t = 1, a 3-plane shared-memory ring of
// sweep t - 1 otherwise); stage K writes the tile to HBM.  Points outside
// the interior keep their halo value at every sweep, as single sweeps do.
// Each point evaluates the operator's terms in the same order with the same
// fused multiply-adds as sweep_kernel, so K fused sweeps are bit-identical
// to K single sweeps.  Intermediate sweeps are rounded to the storage type,
// as a single sweep stores them.
#pragma once

#include "sweep_kernel.cuh"

namespace gscl {

template <typename T, int K>
struct TbShape {
  static constexpr int VX = 4, VY = 2, NW = 8;         // 128 x 16 tile, 256 threads
  static constexpr int TX = 32 * VX, TY = NW * VY;
  static constexpr int vec = 16 / (int)sizeof(T);
  static constexpr int AXK = (K + vec - 1) / vec * vec;  // x apron of the loaded boxes
  static constexpr int BW0 = TX + 2 * AXK, BH0 = TY + 2 * K;      // u box
  static constexpr int BWF = TX + 2 * AXK, BHF = TY + 2 * (K - 1);  // rhs box
  static constexpr int PF = 1;
  static constexpr int R = K + 1 + PF;                  // loaded planes kept per input
  static constexpr int SE0 = (BW0 * BH0 * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr int SEF = (BWF * BHF * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  __host__ __device__ static constexpr int W(int t) { return TX + 2 * (K - t); }  // width of sweep t's region
  __host__ __device__ static constexpr int H(int t) { return TY + 2 * (K - t); }
  __host__ __device__ static constexpr int SS(int t) { return (W(t) * H(t) + 31) / 32 * 32; }  // one plane of sweep t
  __host__ __device__ static constexpr int stage_base(int t) {  // element offset of sweep t's 3-plane ring
    int b = 0;
    for (int i = 1; i < t; ++i) b += 3 * SS(i);
    return b;
  }
  static constexpr int RING0 = 0, RINGF = R * SE0, STAGES = R * SE0 + R * SEF;
  __host__ __device__ static constexpr size_t smem_bytes(bool rhs) {
    return kBarBytes + sizeof(T) * ((size_t)R * SE0 + (rhs ? (size_t)R * SEF : 0) + (size_t)stage_base(K));
  }
};

// One point of the operator: the table's terms in order, u read through a
// source plane triple (rows of width SW, origin already at the point) and the
// rhs at the point.
template <class Def, typename T, int SW, int I>
__device__ __forceinline__ void tb_term(const SweepParams &P, const T *up, const T *uc, const T *un, const T *fp,
                                        typename Arith<T>::A &acc) {
  constexpr OpTerm t = Def::table.t[I];
  using A = typename Arith<T>::A;
  A x;
  if constexpr (t.in == 0) {
    const T *pl = t.dz < 0 ? up : (t.dz > 0 ? un : uc);
    x = to_arith(pl[t.dy * SW + t.dx]);
  } else {
    x = to_arith(fp[0]);
  }
  acc = fma(term_weight(P.terms[I], A(0)), x, acc);
}

template <class Def, typename T, int SW, int... I>
__device__ __forceinline__ typename Arith<T>::A tb_point(const SweepParams &P, const T *up, const T *uc, const T *un,
                                                         const T *fp, std::integer_sequence<int, I...>) {
  typename Arith<T>::A acc = 0;
  (tb_term<Def, T, SW, I>(P, up, uc, un, fp, acc), ...);
  return acc;
}

// What the stages of one step need.
template <typename T>
struct TbCtx {
  const T *ring0, *ringf;
  T *stages;
  int slot_first;  // ring slot of loaded plane 0 of the current run
  int s;           // step: loaded plane index s of the run
  int64_t zb, x0, y0, nx, ny, nz;
};

// Stage t (1 <= t < K): sweep t at plane index s - t over the tile grown by
// K - t, into sweep t's 3-plane ring.
template <typename T, int K, class Def, int t>
__device__ __forceinline__ void tb_stage(const SweepParams &P, const TbCtx<T> &c) {
  using S = TbShape<T, K>;
  constexpr bool RHS = Def::NIN > 1;
  constexpr int Wt = S::W(t), Ht = S::H(t);
  if (c.s >= 2 * t) {
    const int qi = c.s - t;
    const int64_t q = c.zb - K + qi;
    T *dst = c.stages + S::stage_base(t) + (qi % 3) * S::SS(t);
    const bool zin = q >= 0 && q < c.nz;
    for (int p = threadIdx.x; p < Wt * Ht; p += blockDim.x) {
      const int ly = p / Wt, lx = p - ly * Wt;
      const int gx = lx - (K - t), gy = ly - (K - t);  // tile-relative
      const int64_t X = c.x0 + gx, Y = c.y0 + gy;
      const bool in = zin && X >= 0 && X < c.nx && Y >= 0 && Y < c.ny;
      const T *fp = nullptr;
      if constexpr (RHS) fp = c.ringf + ((c.slot_first + qi) % S::R) * S::SEF + (gy + K - 1) * S::BWF + gx + S::AXK;
      T val;
      if constexpr (t == 1) {
        const int off = (gy + K) * S::BW0 + gx + S::AXK;
        const T *uc = c.ring0 + ((c.slot_first + qi) % S::R) * S::SE0 + off;
        if (in) {
          const T *up = c.ring0 + ((c.slot_first + qi - 1) % S::R) * S::SE0 + off;
          const T *un = c.ring0 + ((c.slot_first + qi + 1) % S::R) * S::SE0 + off;
          val = from_arith<T>(tb_point<Def, T, S::BW0>(P, up, uc, un, RHS ? fp : uc,
                                                       std::make_integer_sequence<int, Def::NT>{}));
        } else {
          val = *uc;
        }
      } else {
        constexpr int sw = S::W(t - 1);
        const int off = (gy + (K - t + 1)) * sw + gx + (K - t + 1);
        const T *src = c.stages + S::stage_base(t - 1);
        const T *uc = src + (qi % 3) * S::SS(t - 1) + off;
        if (in) {
          const T *up = src + ((qi + 2) % 3) * S::SS(t - 1) + off;
          const T *un = src + ((qi + 1) % 3) * S::SS(t - 1) + off;
          val = from_arith<T>(
              tb_point<Def, T, sw>(P, up, uc, un, RHS ? fp : uc, std::make_integer_sequence<int, Def::NT>{}));
        } else {
          val = *uc;
        }
      }
      dst[p] = val;
    }
  }
  __syncthreads();
}

template <typename T, int K, class Def, int... ts>
__device__ __forceinline__ void tb_stages(const SweepParams &P, const TbCtx<T> &c, std::integer_sequence<int, ts...>) {
  (tb_stage<T, K, Def, ts + 1>(P, c), ...);
}

template <typename T, int K, class Def>
__global__ void __launch_bounds__(256) tb_kernel(const __grid_constant__ SweepParams P) {
  using S = TbShape<T, K>;
  using A = typename Arith<T>::A;
  constexpr bool RHS = Def::NIN > 1;
  constexpr int TX = S::TX, TY = S::TY, R = S::R;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  T *sm = reinterpret_cast<T *>(smem + kBarBytes);
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  if (tid == 0) {
    for (int r = 0; r < R; ++r) mbar_init(&bars[r], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();

  const InstDesc &I = P.inst;
  TbCtx<T> c;
  c.ring0 = sm + S::RING0;
  c.ringf = sm + S::RINGF;
  c.stages = sm + (RHS ? S::STAGES : S::RINGF);
  c.nx = I.hi[0];  // the range is the whole interior
  c.ny = I.hi[1];
  c.nz = I.hi[2];
  const long long W = (long long)I.tiles_x * I.tiles_y * c.nz;
  const long long run_end = W * (blockIdx.x + 1) / gridDim.x;
  uint32_t issued = 0, waited = 0;  // planes issued / waited by this CTA (both in order)
  int wslot = 0, islot = 0;
  uint32_t wpar = 0;
  bool ok = true;
  const uint32_t tx_bytes = (uint32_t)(sizeof(T) * (S::BW0 * S::BH0 + (RHS ? S::BWF * S::BHF : 0)));

  for (long long pos = W * blockIdx.x / gridDim.x; pos < run_end;) {
    const long long col = pos / c.nz;
    const long long zoff = pos - col * c.nz;
    const int zlen = (int)min(c.nz - zoff, run_end - pos);
    pos += zlen;
    c.x0 = (int64_t)(col % I.tiles_x) * TX;
    c.y0 = (int64_t)(col / I.tiles_x) * TY;
    c.zb = zoff;
    const int total = zlen + 2 * K;
    c.slot_first = islot;

    auto issue = [&](int s) {
      const int slot = islot;
      islot = islot + 1 == R ? 0 : islot + 1;
      uint64_t *bar = &bars[slot];
      mbar_arrive_expect_tx(bar, tx_bytes);
      const int zp = (int)(c.zb - K + s);
      tma_load_3d(const_cast<T *>(c.ring0) + slot * S::SE0, &I.tmap[0], bar, (int)(c.x0 - S::AXK) + I.cx_add[0],
                  (int)(c.y0 - K) + I.cy_add[0], zp + I.cz_add[0]);
      if constexpr (RHS)
        tma_load_3d(const_cast<T *>(c.ringf) + slot * S::SEF, &I.tmap[1], bar, (int)(c.x0 - S::AXK) + I.cx_add[1],
                    (int)(c.y0 - (K - 1)) + I.cy_add[1], zp + I.cz_add[1]);
      ++issued;
    };
    if (tid == 0)
      for (int s = 0; s < min(R, total); ++s) issue(s);

    for (int s = 0; s < total; ++s) {
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
      __syncthreads();
      if (s_abort) break;
      c.s = s;
      tb_stages<T, K, Def>(P, c, std::make_integer_sequence<int, K - 1>{});
      // stage K: the tile, to HBM
      if (s >= 2 * K) {
        const int qi = s - K;
        const int64_t q = c.zb - K + qi;
        constexpr int sw = S::W(K - 1);
        const T *src = c.stages + S::stage_base(K - 1);
#pragma unroll
        for (int r = 0; r < S::VY; ++r) {
          const int gy = wy + r * S::NW;
          const int64_t Y = c.y0 + gy;
#pragma unroll
          for (int e = 0; e < S::VX; ++e) {
            const int gx = lane + 32 * e;
            const int64_t X = c.x0 + gx;
            if (Y < c.ny && X < c.nx) {
              const int off = (gy + 1) * sw + gx + 1;
              const T *uc = src + (qi % 3) * S::SS(K - 1) + off;
              const T *up = src + ((qi + 2) % 3) * S::SS(K - 1) + off;
              const T *un = src + ((qi + 1) % 3) * S::SS(K - 1) + off;
              const T *fp = uc;
              if constexpr (RHS) fp = c.ringf + ((c.slot_first + qi) % R) * S::SEF + (gy + K - 1) * S::BWF + gx + S::AXK;
              const A acc = tb_point<Def, T, sw>(P, up, uc, un, fp, std::make_integer_sequence<int, Def::NT>{});
              T *dst = reinterpret_cast<T *>(I.out[0].base) + q * I.out[0].plane + Y * I.out[0].pitch + X;
              *dst = from_arith<T>(acc);
            }
          }
        }
      }
      __syncthreads();
      // the loaded plane s - K is no longer read: its slot takes plane s - K + R
      if (tid == 0 && s >= K && s - K + R < total) issue(s - K + R);
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
