// Two sweeps per pass over HBM with vector lanes (temporal blocking, K = 2:
// the paper's wide ghost areas, Section 2, applied on chip).
//
// A CTA owns an output tile of 128 x 14 points of one tile column and
// streams it through a run of z planes.  Per step s (plane index q = s of
// the run, z = zb - 2 + q):
//   stage 1 computes sweep 1 at plane q - 1 over the frame: the tile grown
//     by one row on each side (16 rows) and by one column on each side (the
//     128 tile columns as 16-byte lane groups, like the vector-lane sweep,
//     plus the two edge columns as single elements); the values go to a
//     four-plane ring in shared memory, rounded to the storage type exactly
//     as a single sweep stores them;
//   one block barrier;
//   stage 2 computes sweep 2 at plane q - 2 over the tile from that ring and
//     stores it.
// u comes through a four-slot TMA ring of (128 + 2 AX) x 18 boxes, f through
// a four-slot ring of 128 x 16 boxes (the edge columns read f from global
// memory).  Four slots keep stage 2 of step s and stage 1 of step s + 1 on
// disjoint planes, so one barrier per step suffices.  Frame points outside
// the interior keep the grid's halo value, as a single sweep leaves the halo
// of its output, and every point evaluates the operator's terms in table
// order with the FMAs a single sweep uses, so a pass is bit-identical to two
// single sweeps.
#pragma once

#include "sweep_kernel.cuh"

namespace gscl {

template <typename T>
struct Tb2Shape {
  static constexpr int G = 16 / (int)sizeof(T);  // columns per lane group (16 bytes)
  static constexpr int LPR = 128 / G;            // lanes per frame row
  static constexpr int RPS = 32 / LPR;           // row blocks per warp
  static constexpr int NW = 8;
  static constexpr int VY = 16 / (NW * RPS);     // frame rows per thread
  static constexpr int FH = 16;                  // frame rows
  static constexpr int TX = 128, TY = FH - 2;    // output tile
  static constexpr int AX = G;                   // x apron of the u box (16 bytes)
  static constexpr int BW = TX + 2 * AX, BH = FH + 2;
  static constexpr int R = 4;
  static constexpr int SE_U = (BW * BH * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr int SE_F = (TX * FH * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr int SE_1 = (BW * FH * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr size_t smem_bytes() { return kBarBytes + sizeof(T) * (size_t)R * (SE_U + SE_F + SE_1); }
};

// BATCH: the CTA walks its segments of a batch's work-list (instance, tile
// column, z run; P.insts holds the instances' descriptors with this kernel's
// boxes) instead of its share of one grid's (tile, plane) pairs.
template <typename T, class Def, bool BATCH = false>
__global__ void __launch_bounds__(256) tb2_kernel(const __grid_constant__ SweepParams P) {
  using S = Tb2Shape<T>;
  constexpr int G = S::G, VY = S::VY, BW = S::BW, R = S::R;
  constexpr bool RHS = Def::NIN > 1;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *ubar = reinterpret_cast<uint64_t *>(smem);
  uint64_t *fbar = ubar + R;
  T *uring = reinterpret_cast<T *>(smem + kBarBytes);
  T *fring = uring + R * S::SE_U;
  T *u1ring = fring + R * S::SE_F;
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  const int cg = lane % S::LPR, rb = lane / S::LPR;
  const int fr0 = (wy * S::RPS + rb) * VY;  // this thread's first frame row
  if (tid == 0) {
    for (int r = 0; r < R; ++r) {
      mbar_init(&ubar[r], 1);
      mbar_init(&fbar[r], 1);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  pdl_wait();

  const int64_t nz0 = P.inst.hi[2];
  const long long W = BATCH ? 0 : (long long)P.inst.tiles_x * P.inst.tiles_y * nz0;
  const long long run_end = W * (blockIdx.x + 1) / gridDim.x;
  long long pos = W * blockIdx.x / gridDim.x;
  int sg = 0, sg_end = 0;
  if constexpr (BATCH) {
    sg = P.cta_seg[blockIdx.x];
    sg_end = P.cta_seg[blockIdx.x + 1];
  }
  // ring positions of the next run's plane 0, advanced identically in every
  // thread; issued counts are thread 0's (it issues), waited counts each
  // thread's own (both only drain copies after a wait gave up)
  uint32_t u_pos = 0, f_pos = 0;
  uint32_t u_issued = 0, u_waited = 0, f_issued = 0, f_waited = 0;
  bool ok = true;
  constexpr uint32_t u_bytes = (uint32_t)(sizeof(T) * BW * S::BH);
  constexpr uint32_t f_bytes = (uint32_t)(sizeof(T) * S::TX * S::FH);
  float w[Def::NT];
#pragma unroll
  for (int i = 0; i < Def::NT; ++i) w[i] = P.terms[i].wf;

  for (;;) {
    const InstDesc *Ip;
    long long col, zoff;
    int zlen;
    if constexpr (BATCH) {
      if (sg >= sg_end) break;
      const Segment seg = P.segs[sg++];
      Ip = &P.insts[seg.inst];
      col = seg.col;
      zoff = seg.zoff;
      zlen = seg.zlen;
    } else {
      if (pos >= run_end) break;
      Ip = &P.inst;
      col = pos / nz0;
      zoff = pos - col * nz0;
      zlen = (int)min(nz0 - zoff, run_end - pos);
      pos += zlen;
    }
    const InstDesc &I = *Ip;
    const int64_t nx = I.hi[0], ny = I.hi[1], nz = I.hi[2];  // the range is the whole interior
    const int64_t x0 = (int64_t)(col % I.tiles_x) * S::TX;
    const int64_t y0 = (int64_t)(col / I.tiles_x) * S::TY;
    const int64_t zb = zoff;
    const int total = zlen + 4;  // u planes zb - 2 .. zb + zlen + 1
    const uint32_t u0 = u_pos, f0 = f_pos;  // ring positions of this run's plane 0
    u_pos += (uint32_t)total;
    if (RHS) f_pos += (uint32_t)total;
    // stage 2 of the previous run's last step read f after that step's barrier
    __syncthreads();

    auto issue_u = [&](int q) {
      const uint32_t g = u0 + (uint32_t)q;
      uint64_t *bar = &ubar[g % R];
      mbar_arrive_expect_tx(bar, u_bytes);
      tma_load_3d(uring + (g % R) * S::SE_U, &I.tmap[0], bar, (int)(x0 - S::AX) + I.cx_add[0],
                  (int)(y0 - 2) + I.cy_add[0], (int)(zb - 2 + q) + I.cz_add[0]);
      u_issued = g + 1;
    };
    auto issue_f = [&](int q) {
      const uint32_t g = f0 + (uint32_t)q;
      uint64_t *bar = &fbar[g % R];
      mbar_arrive_expect_tx(bar, f_bytes);
      tma_load_3d(fring + (g % R) * S::SE_F, &I.tmap[1], bar, (int)x0 + I.cx_add[1], (int)(y0 - 1) + I.cy_add[1],
                  (int)(zb - 2 + q) + I.cz_add[1]);
      f_issued = g + 1;
    };
    if (tid == 0) {
      for (int q = 0; q < min(R, total); ++q) issue_u(q);
      if constexpr (RHS)
        for (int q = 0; q < min(R, total); ++q) issue_f(q);
    }

    // this thread's frame rows and group columns
    int64_t yr[VY];
    bool yin[VY];
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      yr[r] = y0 - 1 + fr0 + r;
      yin[r] = yr[r] >= 0 && yr[r] < ny;
    }
    const int64_t xg = x0 + G * cg;
    bool xin[G];
#pragma unroll
    for (int e = 0; e < G; ++e) xin[e] = xg + e >= 0 && xg + e < nx;
    float zq[3][VY][G];  // u centre columns of planes q - 1, q, q + 1 (stage 1)

    for (int s = 0; s < total; ++s) {
      if (ok) {
        ok = mbar_wait_bounded(&ubar[(u0 + s) % R], ((u0 + s) / R) & 1u);
        if (ok) ++u_waited;
        if (ok && RHS) {
          ok = mbar_wait_bounded(&fbar[(f0 + s) % R], ((f0 + s) / R) & 1u);
          if (ok) ++f_waited;
        }
        if (!ok) {
          s_abort = 1;
          atomicOr(P.err, 1);
        }
      }
      // ---- stage 1: sweep 1 at plane q = s - 1
      if (ok && s >= 2) {
        const int q = s - 1;
        const int64_t z = zb - 2 + q;
        const bool zin = z >= 0 && z < nz;
        const T *up = uring + ((u0 + q - 1) % R) * S::SE_U;
        const T *uc = uring + ((u0 + q) % R) * S::SE_U;
        const T *un = uring + ((u0 + q + 1) % R) * S::SE_U;
        const T *fp = fring + ((f0 + q) % R) * S::SE_F;
        T *o1 = u1ring + (q % R) * S::SE_1;
        // the z queue: planes q - 1, q, q + 1 at this thread's rows
        if (s == 2) {
#pragma unroll
          for (int r = 0; r < VY; ++r) {
            load_group<G>(up + (fr0 + r + 1) * BW + S::AX + G * cg, zq[0][r]);
            load_group<G>(uc + (fr0 + r + 1) * BW + S::AX + G * cg, zq[1][r]);
          }
        } else {
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int e = 0; e < G; ++e) {
              zq[0][r][e] = zq[1][r][e];
              zq[1][r][e] = zq[2][r][e];
            }
        }
#pragma unroll
        for (int r = 0; r < VY; ++r) load_group<G>(un + (fr0 + r + 1) * BW + S::AX + G * cg, zq[2][r]);
#pragma unroll
        for (int r = 0; r < VY; ++r) {
          const int br = fr0 + r + 1;  // box row of this frame row
          const T *rowc = uc + br * BW + S::AX + G * cg;
          float o[G];
#pragma unroll
          for (int e = 0; e < G; ++e) o[e] = 0.0f;
          static_for<Def::NT>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr OpTerm t = Def::table.t[i];
            float x[G];
            if constexpr (t.in == 1) {
              load_group<G>(fp + (fr0 + r) * S::TX + G * cg, x);
            } else if constexpr (t.dy == 0 && t.dx == 0) {
#pragma unroll
              for (int e = 0; e < G; ++e) x[e] = zq[t.dz + 1][r][e];
            } else if constexpr (t.dx != 0) {  // x neighbour: the group shifted, one element from the ring
#pragma unroll
              for (int e = 0; e < G; ++e) {
                const int k = e + t.dx;
                x[e] = (k >= 0 && k < G) ? zq[1][r][k < 0 ? 0 : (k >= G ? G - 1 : k)] : to_arith(rowc[k]);
              }
            } else {  // y neighbour
              if constexpr (t.dy < 0) {
                if (r + t.dy >= 0) {
#pragma unroll
                  for (int e = 0; e < G; ++e) x[e] = zq[1][(r + t.dy) < 0 ? 0 : r + t.dy][e];
                } else {
                  load_group<G>(rowc + t.dy * BW, x);
                }
              } else {
                if (r + t.dy < VY) {
#pragma unroll
                  for (int e = 0; e < G; ++e) x[e] = zq[1][(r + t.dy) >= VY ? VY - 1 : r + t.dy][e];
                } else {
                  load_group<G>(rowc + t.dy * BW, x);
                }
              }
            }
            fma_group<G>(w[i], x, o);
          });
          // outside the interior the grid keeps its halo value
          float res[G];
#pragma unroll
          for (int e = 0; e < G; ++e) res[e] = (zin && yin[r] && xin[e]) ? to_arith(from_arith<T>(o[e])) : zq[1][r][e];
          store_group<G>(o1 + (fr0 + r) * BW + S::AX + G * cg, res);
        }
        // the frame's edge columns x0 - 1 (lane group 0) and x0 + 128 (the last group), one element each
        if (cg == 0 || cg == S::LPR - 1) {
          const int ex = cg == 0 ? -1 : S::TX;  // column relative to x0
          const int64_t X = x0 + ex;
          const bool xe = X >= 0 && X < nx;
#pragma unroll
          for (int r = 0; r < VY; ++r) {
            const int br = fr0 + r + 1;
            const int bc = S::AX + ex;
            float acc = 0.0f;
            static_for<Def::NT>([&](auto ic) {
              constexpr int i = decltype(ic)::value;
              constexpr OpTerm t = Def::table.t[i];
              float xv;
              if constexpr (t.in == 1) {
                xv = (zin && yin[r] && xe)
                         ? to_arith(reinterpret_cast<const T *>(I.in[1].base)[z * I.in[1].plane + yr[r] * I.in[1].pitch + X])
                         : 0.0f;
              } else {
                const T *pl = t.dz < 0 ? up : (t.dz > 0 ? un : uc);
                xv = to_arith(pl[(br + t.dy) * BW + bc + t.dx]);
              }
              acc = fmaf(w[i], xv, acc);
            });
            const float keep = to_arith(uc[br * BW + bc]);
            o1[(fr0 + r) * BW + bc] = from_arith<T>((zin && yin[r] && xe) ? to_arith(from_arith<T>(acc)) : keep);
          }
        }
      }
      __syncthreads();
      if (s_abort) break;
      if (tid == 0) {
        // u plane s - 2 is read no more (stage 1 of this step was its last use); f plane s - 3 neither
        if (s >= 2 && s + 2 < total) issue_u(s + 2);
        if (RHS && s >= 3 && s + 1 < total) issue_f(s + 1);
      }
      // ---- stage 2: sweep 2 at plane q = s - 2, frame rows 1 .. 14
      if (ok && s >= 4) {
        const int q = s - 2;
        const int64_t z = zb - 2 + q;
        const bool zin = z >= 0 && z < nz;
        const T *pp = u1ring + ((q - 1) % R) * S::SE_1;
        const T *pc = u1ring + (q % R) * S::SE_1;
        const T *pn = u1ring + ((q + 1) % R) * S::SE_1;
        const T *fp = fring + ((f0 + q) % R) * S::SE_F;
#pragma unroll
        for (int r = 0; r < VY; ++r) {
          const int fr = fr0 + r;
          if (fr < 1 || fr > S::TY) continue;
          const T *rowc = pc + fr * BW + S::AX + G * cg;
          float c[G];
          load_group<G>(rowc, c);
          float o[G];
#pragma unroll
          for (int e = 0; e < G; ++e) o[e] = 0.0f;
          static_for<Def::NT>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr OpTerm t = Def::table.t[i];
            float x[G];
            if constexpr (t.in == 1) {
              load_group<G>(fp + fr * S::TX + G * cg, x);
            } else if constexpr (t.dx == 0 && t.dy == 0 && t.dz == 0) {
#pragma unroll
              for (int e = 0; e < G; ++e) x[e] = c[e];
            } else if constexpr (t.dx != 0) {
#pragma unroll
              for (int e = 0; e < G; ++e) {
                const int k = e + t.dx;
                x[e] = (k >= 0 && k < G) ? c[k < 0 ? 0 : (k >= G ? G - 1 : k)] : to_arith(rowc[k]);
              }
            } else {
              const T *pl = t.dz < 0 ? pp : (t.dz > 0 ? pn : pc);
              load_group<G>(pl + (fr + t.dy) * BW + S::AX + G * cg, x);
            }
            fma_group<G>(w[i], x, o);
          });
          if (zin && yin[r]) {
            T *dst = reinterpret_cast<T *>(I.out[0].base) + z * I.out[0].plane + yr[r] * I.out[0].pitch + xg;
            if (xin[0] && xin[G - 1]) {
              store_group<G>(dst, o);
            } else {
#pragma unroll
              for (int e = 0; e < G; ++e)
                if (xin[e]) dst[e] = from_arith<T>(o[e]);
            }
          }
        }
      }
    }
    if (s_abort) break;
  }
  pdl_launch_dependents();
  if (s_abort) {
    if (tid == 0) {
      for (uint32_t g = u_waited; g < u_issued; ++g) mbar_wait_bounded(&ubar[g % R], (g / R) & 1u);
      for (uint32_t g = f_waited; g < f_issued; ++g) mbar_wait_bounded(&fbar[g % R], (g / R) & 1u);
    }
    __syncthreads();
  }
}

}  // namespace gscl
