// Operators whose structure is fixed at compile time.
//
// The paper's library keeps a generic implementation of every construct and
// picks up a better-suited one when it exists (Section 1).  Here the generic
// implementation is the runtime term loop of sweep_kernel; the operators
// below are the structures the benchmark workloads use, compiled with every
// offset, grid and ring position as a constant so that each term costs one
// shared-memory load and one fused multiply-add per point.  A descriptor
// matches one of them when its terms have the same (dx, dy, dz, in, coef,
// out) multiset; the weights stay runtime values.  Host and device share
// these tables (constexpr).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define GSCL_HD __host__ __device__
#else
#define GSCL_HD
#endif

namespace gscl {

// in = -1: the operator's value; out = -1: a term of the value; coef = -1: none
struct OpTerm {
  int dx, dy, dz, in, coef, out;
};

template <int N>
struct TermTable {
  OpTerm t[N];
};

enum StaticOpId {
  OP_GENERIC = -1,
  OP_HEAT7_RHS = 0,     // u' = w0 u + sum6 w_i u(nbr) + w7 f         (u, f) -> u'
  OP_STAR7,             // u' = w0 u + sum6 w_i u(nbr)                 (u) -> u'
  OP_JACOBI7_RHS,       // u' = sum6 w_i u(nbr) + w6 f                 (u, f) -> u'
  OP_JACOBI5_2D,        // u' = sum4 w_i u(nbr)                        2D (u) -> u'
  OP_CLIMATE,           // 13-point biharmonic x kappa + vertical advection x w + tendency, 8 -> 3
  OP_HEAT7_RHS_FUSED,   // value r = sum6 + u + f terms; u' = u + w r  (u, f) -> u', r
  OP_HEAT7_FUSED,       // value r = sum6 + u terms; u' = u + w r      (u) -> u', r
  OP_RESIDUAL7_RHS,     // value r = sum6 + u + f terms, no output     (u, f) -> r
  OP_DIFFERENCE,        // value a - b style: a(0), b(0) terms         (a, b) -> v
  OP_IDENTITY,          // value in0(0)                                (a) -> v
  OP_COUNT
};

#define GSCL_AXIAL6(in, out) {1, 0, 0, in, -1, out}, {-1, 0, 0, in, -1, out}, {0, 1, 0, in, -1, out}, \
                             {0, -1, 0, in, -1, out}, {0, 0, 1, in, -1, out}, {0, 0, -1, in, -1, out}

struct OpHeat7Rhs {
  static constexpr int NIN = 2, NOUT = 1, NT = 8;
  static constexpr TermTable<NT> table = {{{0, 0, 0, 0, -1, 0}, GSCL_AXIAL6(0, 0), {0, 0, 0, 1, -1, 0}}};
};
struct OpStar7 {
  static constexpr int NIN = 1, NOUT = 1, NT = 7;
  static constexpr TermTable<NT> table = {{{0, 0, 0, 0, -1, 0}, GSCL_AXIAL6(0, 0)}};
};
struct OpJacobi7Rhs {
  static constexpr int NIN = 2, NOUT = 1, NT = 7;
  static constexpr TermTable<NT> table = {{GSCL_AXIAL6(0, 0), {0, 0, 0, 1, -1, 0}}};
};
struct OpJacobi5_2D {
  static constexpr int NIN = 1, NOUT = 1, NT = 4;
  static constexpr TermTable<NT> table = {{{1, 0, 0, 0, -1, 0}, {-1, 0, 0, 0, -1, 0}, {0, 1, 0, 0, -1, 0},
                                           {0, -1, 0, 0, -1, 0}}};
};

constexpr TermTable<51> climate_table() {
  TermTable<51> r{};
  const int bih[13][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {1, -1}, {-1, 1}, {-1, -1},
                          {2, 0}, {-2, 0}, {0, 2}, {0, -2}};
  int k = 0;
  for (int m = 0; m < 3; ++m) {
    r.t[k++] = OpTerm{0, 0, 0, m, -1, m};
    for (int b = 0; b < 13; ++b) r.t[k++] = OpTerm{bih[b][0], bih[b][1], 0, m, 3, m};
    r.t[k++] = OpTerm{0, 0, 1, m, 4, m};
    r.t[k++] = OpTerm{0, 0, -1, m, 4, m};
    r.t[k++] = OpTerm{0, 0, 0, 5 + m, -1, m};
  }
  return r;
}
struct OpClimate {
  static constexpr int NIN = 8, NOUT = 3, NT = 51;
  static constexpr TermTable<NT> table = climate_table();
};

// value terms come first: a table is evaluated in order
struct OpHeat7RhsFused {
  static constexpr int NIN = 2, NOUT = 1, NT = 10;
  static constexpr TermTable<NT> table = {{GSCL_AXIAL6(0, -1), {0, 0, 0, 0, -1, -1}, {0, 0, 0, 1, -1, -1},
                                           {0, 0, 0, 0, -1, 0}, {0, 0, 0, -1, -1, 0}}};
};
struct OpHeat7Fused {
  static constexpr int NIN = 1, NOUT = 1, NT = 9;
  static constexpr TermTable<NT> table = {{GSCL_AXIAL6(0, -1), {0, 0, 0, 0, -1, -1}, {0, 0, 0, 0, -1, 0},
                                           {0, 0, 0, -1, -1, 0}}};
};
struct OpResidual7Rhs {
  static constexpr int NIN = 2, NOUT = 0, NT = 8;
  static constexpr TermTable<NT> table = {{GSCL_AXIAL6(0, -1), {0, 0, 0, 0, -1, -1}, {0, 0, 0, 1, -1, -1}}};
};
struct OpDifference {
  static constexpr int NIN = 2, NOUT = 0, NT = 2;
  static constexpr TermTable<NT> table = {{{0, 0, 0, 0, -1, -1}, {0, 0, 0, 1, -1, -1}}};
};
struct OpIdentity {
  static constexpr int NIN = 1, NOUT = 0, NT = 1;
  static constexpr TermTable<NT> table = {{{0, 0, 0, 0, -1, -1}}};
};

#undef GSCL_AXIAL6

// Inputs an operator reads only at the core element (as a term's grid at
// offset (0,0,0), or as a coefficient, which is always read there) need one
// plane box without halo per z step: the sweep kernel stages them in a
// two-slot "centre ring" loaded one step ahead, apart from the ring of plane
// boxes that the neighbourhood reads need.
template <class Def>
GSCL_HD constexpr bool centre_only(int in) {
  bool used = false;
  for (int i = 0; i < Def::NT; ++i) {
    const OpTerm &t = Def::table.t[i];
    if (t.coef == in) used = true;
    if (t.in == in) {
      used = true;
      if (t.dx != 0 || t.dy != 0 || t.dz != 0) return false;
    }
  }
  return used;
}

template <class Def>
constexpr uint32_t centre_mask() {
  uint32_t m = 0;
  for (int a = 0; a < Def::NIN; ++a)
    if (centre_only<Def>(a)) m |= 1u << a;
  return m;
}

// IEEE FP64 sweeps are bound by the FP64 pipe: there the centre ring's extra
// wait per step costs more than the shared memory it frees gains for an
// operator with one centre-only input (the heat family's RHS), but an
// operator with many (the climate operator's coefficients and tendencies)
// frees enough for a second resident CTA.
constexpr int kCentreFp64Min = 4;
template <class Def>
GSCL_HD constexpr int centre_count() {
  int n = 0;
  for (int a = 0; a < Def::NIN; ++a) n += centre_only<Def>(a) ? 1 : 0;
  return n;
}

template <class Op>
constexpr bool op_has_value() {
  for (int i = 0; i < Op::NT; ++i)
    if (Op::table.t[i].out < 0) return true;
  return false;
}

// Centre-ring inputs of a compile-time operator (none for the generic one).
inline uint32_t static_centre_mask(int op) {
  switch (op) {
    case OP_HEAT7_RHS: return centre_mask<OpHeat7Rhs>();
    case OP_STAR7: return centre_mask<OpStar7>();
    case OP_JACOBI7_RHS: return centre_mask<OpJacobi7Rhs>();
    case OP_JACOBI5_2D: return centre_mask<OpJacobi5_2D>();
    case OP_CLIMATE: return centre_mask<OpClimate>();
    case OP_HEAT7_RHS_FUSED: return centre_mask<OpHeat7RhsFused>();
    case OP_HEAT7_FUSED: return centre_mask<OpHeat7Fused>();
    case OP_RESIDUAL7_RHS: return centre_mask<OpResidual7Rhs>();
    case OP_DIFFERENCE: return centre_mask<OpDifference>();
    case OP_IDENTITY: return centre_mask<OpIdentity>();
  }
  return 0;
}

// The axial group: six consecutive table terms reading one input at the six
// unit offsets, without coefficient, into one destination (the star / heat
// family's neighbour sum).  Returns the index of its first term, or -1.
// When the six weights are bit-identical, IEEE FP64 sweeps evaluate
// w (x+ + x-) ... as w times a tree sum of the six values, two of whose
// additions run on the integer pipe (fp64_int.cuh): the same result within
// a few rounding errors of the neighbour sum, and fewer FP64 operations.
template <class Def>
GSCL_HD constexpr int axial_group() {
  for (int i = 0; i + 6 <= Def::NT; ++i) {
    const OpTerm &t0 = Def::table.t[i];
    if (t0.in < 0 || t0.coef >= 0) continue;
    int seen = 0;
    bool ok = true;
    for (int k = 0; k < 6 && ok; ++k) {
      const OpTerm &t = Def::table.t[i + k];
      const int ax = (t.dx != 0) + (t.dy != 0) + (t.dz != 0);
      const int mag = (t.dx < 0 ? -t.dx : t.dx) + (t.dy < 0 ? -t.dy : t.dy) + (t.dz < 0 ? -t.dz : t.dz);
      ok = t.in == t0.in && t.coef < 0 && t.out == t0.out && ax == 1 && mag == 1;
      if (ok) {
        const int bit = t.dx == 1 ? 0 : t.dx == -1 ? 1 : t.dy == 1 ? 2 : t.dy == -1 ? 3 : t.dz == 1 ? 4 : 5;
        ok = ((seen >> bit) & 1) == 0;
        seen |= 1 << bit;
      }
    }
    if (ok && seen == 63) return i;
  }
  return -1;
}

// Coefficient groups: consecutive terms of one coefficient run (one
// coefficient grid, one destination) reading one input at nonzero offsets of
// one class (the same |dx|, |dy|, |dz| up to order), four of them or two: the
// climate operator's biharmonic rings and its vertical pair.  With the four
// weights bit-identical a group of four is summed as (x0 + x1) + (x2 + x3)
// with the first addition on the integer pipe; a pair whose weights are
// opposite is differenced, x0 - x1, on the integer pipe.
template <class Def>
GSCL_HD constexpr int offset_class(int i) {
  const OpTerm &t = Def::table.t[i];
  int a = t.dx < 0 ? -t.dx : t.dx, b = t.dy < 0 ? -t.dy : t.dy, c = t.dz < 0 ? -t.dz : t.dz;
  if (a > b) { const int x = a; a = b; b = x; }
  if (b > c) { const int x = b; b = c; c = x; }
  if (a > b) { const int x = a; a = b; b = x; }
  return (a * 64 + b) * 64 + c;
}
template <class Def>
GSCL_HD constexpr bool coef_link(int i, int j) {
  const OpTerm &a = Def::table.t[i], &b = Def::table.t[j];
  return a.in >= 0 && a.coef >= 0 && a.in == b.in && a.coef == b.coef && a.out == b.out &&
         offset_class<Def>(i) != 0 && offset_class<Def>(i) == offset_class<Def>(j);
}
template <class Def>
GSCL_HD constexpr int coef_group_len(int s) {
  int n = 1;
  while (s + n < Def::NT && coef_link<Def>(s, s + n)) ++n;
  return n;
}
// the first term of the coefficient group holding term i, or -1
template <class Def>
GSCL_HD constexpr int coef_group_start(int i) {
  if (i < 0 || i >= Def::NT) return -1;
  int s = i;
  while (s > 0 && coef_link<Def>(s - 1, s)) --s;
  const int n = coef_group_len<Def>(s);
  return (n == 2 || n == 4) ? s : -1;
}
template <class Def>
GSCL_HD constexpr bool has_groups() {
  bool any = axial_group<Def>() >= 0;
  for (int i = 0; i < Def::NT; ++i) any = any || coef_group_start<Def>(i) >= 0;
  return any;
}
// the length of the coefficient group starting at each term (0 elsewhere)
template <int N>
struct IntTable {
  int v[N];
};
template <class Def>
constexpr IntTable<Def::NT> coef_group_lens() {
  IntTable<Def::NT> r{};
  for (int i = 0; i < Def::NT; ++i) r.v[i] = coef_group_start<Def>(i) == i ? coef_group_len<Def>(i) : 0;
  return r;
}

// Whether the weights (w[i]: table term i's weight) allow the group
// evaluation: the axial group's six equal, every group of four equal, every
// pair opposite; false for an operator without groups.
template <class Def>
bool group_weights_ok(const double *w) {
  auto bits = [](double x) {
    unsigned long long u = 0;
    __builtin_memcpy(&u, &x, sizeof u);
    return u;
  };
  if constexpr (!has_groups<Def>()) return false;
  constexpr int ga = axial_group<Def>();
  if (ga >= 0)
    for (int k = 1; k < 6; ++k)
      if (bits(w[ga + k]) != bits(w[ga])) return false;
  constexpr IntTable<Def::NT> lens = coef_group_lens<Def>();
  for (int i = 0; i < Def::NT; ++i) {
    const int n = lens.v[i];
    if (n == 2 && bits(w[i + 1]) != (bits(w[i]) ^ (1ull << 63))) return false;
    if (n == 4)
      for (int k = 1; k < 4; ++k)
        if (bits(w[i + k]) != bits(w[i])) return false;
  }
  return true;
}

inline bool static_group_weights_ok(int op, const double *w) {
  switch (op) {
    case OP_HEAT7_RHS: return group_weights_ok<OpHeat7Rhs>(w);
    case OP_STAR7: return group_weights_ok<OpStar7>(w);
    case OP_JACOBI7_RHS: return group_weights_ok<OpJacobi7Rhs>(w);
    case OP_CLIMATE: return group_weights_ok<OpClimate>(w);
    case OP_HEAT7_RHS_FUSED: return group_weights_ok<OpHeat7RhsFused>(w);
    case OP_HEAT7_FUSED: return group_weights_ok<OpHeat7Fused>(w);
    case OP_RESIDUAL7_RHS: return group_weights_ok<OpResidual7Rhs>(w);
  }
  return false;
}

inline int static_axial_group(int op) {
  switch (op) {
    case OP_HEAT7_RHS: return axial_group<OpHeat7Rhs>();
    case OP_STAR7: return axial_group<OpStar7>();
    case OP_JACOBI7_RHS: return axial_group<OpJacobi7Rhs>();
    case OP_HEAT7_RHS_FUSED: return axial_group<OpHeat7RhsFused>();
    case OP_HEAT7_FUSED: return axial_group<OpHeat7Fused>();
    case OP_RESIDUAL7_RHS: return axial_group<OpResidual7Rhs>();
  }
  return -1;
}

}  // namespace gscl
