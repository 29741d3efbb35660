/*
 * gscl_oracle.c -- plain FP64 CPU oracle for the two iteration spaces of the
 * generic stencil library: do_all and do_reduce, the ordered iteration
 * spaces, do_diamond and red-black colouring (Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load this code.  The CUDA
 * library never includes, links or calls it, and it shares no code with it.
 *
 * What it computes (Section 3, definitions of "stencil operator",
 * "stencil computation", do_all and do_reduce):
 *
 *   A grid is a dense d-dimensional array G(i0, .., i_{d-1}) (d = 2 or 3;
 *   a 2D grid is a 3D grid with nz = 1 and no z halo).  Around the interior
 *   each grid carries a halo of width h[axis]: the cells a stencil operator
 *   may read at a fixed offset from the core element (Section 3, "stencil
 *   shape ... defines the halo").
 *
 *   A stencil operator is given as a list of terms
 *        t = (dx, dy, dz, in, coef, out, w)
 *   and, at a core element p, computes
 *        value(p)  = sum over terms with out == VALUE of  w * X_t(p) * C_t(p)
 *        out_m(p)  = sum over terms with out == m      of  w * X_t(p) * C_t(p)
 *   where X_t(p) = In_in(p + (dx,dy,dz)), or value(p) when in == VALUE
 *   (offset 0: the operator's own return value, which is how two operators
 *   are fused into one scan, Section 5.2), and C_t(p) = In_coef(p) or 1 when
 *   coef == NONE.  Terms are summed in the order given, each product formed
 *   as (w * X) * C, with no fused multiply-add (the file is compiled with
 *   -ffp-contract=off).  Outputs are written only at the core element.
 *
 *   do_all applies the operator at every core element of an iteration range
 *   [lo, hi) (interior coordinates), in lexicographic (k, j, i) order; the
 *   paper guarantees no order, so the operator must not read an output grid
 *   at a non-zero offset, and the oracle requires output arrays distinct from
 *   input arrays.
 *
 *   do_reduce is do_all whose per-element return values are reduced to one
 *   value by a commutative operator (Section 3).  Here the returned value is
 *   value(p) (or In_0(p) when the operator is empty), reduced in lexicographic
 *   order by one of
 *        SUM    : Neumaier's compensated sum (Neumaier 1974),
 *        MAXABS : max |v| (NaN if any v is NaN),
 *        L2     : sqrt of the Neumaier-compensated sum of v*v.
 *
 * Two builds of this file.  The checker (gcc -O2 -ffp-contract=off) runs
 * every loop in the order written above.  The timing build, used only to
 * time the oracle as the CPU baseline (-O3 -march=native -fopenmp, still
 * without FMA contraction), computes independent elements on several
 * threads, plane by plane, and reduces their values in the same
 * lexicographic order, so both builds return the same numbers.
 *
 * Layout (the oracle's own, unrelated to the library's): each grid is a
 * dense C-order array of (nz+2hz) x (ny+2hy) x (nx+2hx) doubles, x fastest;
 * element (i,j,k) of the interior, with -h <= i < n+h, is at
 *        ((k+hz)*(ny+2hy) + (j+hy))*(nx+2hx) + (i+hx).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ORC_MUTANT (tests only, never set in a normal build) plants one known
 * mistake so the test suite can show that its pins detect it. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

#define ORC_VALUE 254 /* in == ORC_VALUE: the operator's value; out == ORC_VALUE: term of the value */
#define ORC_NONE 255  /* coef == ORC_NONE: no coefficient grid */

enum { ORC_OK = 0, ORC_BAD_ARG = 1, ORC_BAD_RANGE = 2 };
enum { ORC_SUM = 0, ORC_MAXABS = 1, ORC_L2 = 2, ORC_WITHIN = 3 };

typedef struct {
  int32_t dx, dy, dz;
  int32_t in, coef, out;
  double w;
} orc_term;

typedef struct {
  int64_t nx, ny, nz;  /* interior extent, shared by every grid of one call */
} orc_extent;

typedef struct {
  const double *data;  /* dense array with halo, layout above */
  int32_t hx, hy, hz;  /* this grid's halo */
} orc_grid;

typedef struct {
  double *data;
  int32_t hx, hy, hz;
} orc_out_grid;

static int64_t orc_index(const orc_extent *e, int32_t hx, int32_t hy, int32_t hz,
                         int64_t i, int64_t j, int64_t k) {
  int64_t X = e->nx + 2 * (int64_t)hx;
  int64_t Y = e->ny + 2 * (int64_t)hy;
#if ORC_MUTANT == 5
  if (Y == X) return ((k + hz) * Y + (i + hx)) * X + (j + hy); /* x and y exchanged */
#endif
  return ((k + hz) * Y + (j + hy)) * X + (i + hx);
}

/* Reads element (i,j,k) of input grid g; the caller has checked it lies
 * inside the grid's interior plus halo. */
static double orc_read(const orc_extent *e, const orc_grid *g, int64_t i, int64_t j, int64_t k) {
  return g->data[orc_index(e, g->hx, g->hy, g->hz, i, j, k)];
}

/* Every read p + offset of every core element in [lo, hi) must fall inside
 * [-h, n+h) of the grid it reads; coefficient reads are at offset 0. */
static int orc_check(const orc_extent *e, int n_in, const orc_grid *in, int n_out,
                     int n_terms, const orc_term *terms, const int64_t lo[3], const int64_t hi[3]) {
  const int64_t n[3] = {e->nx, e->ny, e->nz};
  for (int a = 0; a < 3; ++a) {
    if (lo[a] < 0 || hi[a] > n[a] || lo[a] > hi[a]) return ORC_BAD_RANGE;
  }
  for (int t = 0; t < n_terms; ++t) {
    const orc_term *tm = &terms[t];
    if (tm->out != ORC_VALUE && (tm->out < 0 || tm->out >= n_out)) return ORC_BAD_ARG;
    if (tm->coef != ORC_NONE && (tm->coef < 0 || tm->coef >= n_in)) return ORC_BAD_ARG;
    if (tm->in == ORC_VALUE) {
      if (tm->dx || tm->dy || tm->dz || tm->out == ORC_VALUE) return ORC_BAD_ARG;
      continue;
    }
    if (tm->in < 0 || tm->in >= n_in) return ORC_BAD_ARG;
    const orc_grid *g = &in[tm->in];
    const int32_t h[3] = {g->hx, g->hy, g->hz};
    const int32_t d[3] = {tm->dx, tm->dy, tm->dz};
    for (int a = 0; a < 3; ++a) {
      if (lo[a] >= hi[a]) continue;
      if (lo[a] + d[a] < -(int64_t)h[a] || hi[a] - 1 + d[a] > n[a] - 1 + h[a]) return ORC_BAD_RANGE;
    }
  }
  return ORC_OK;
}

/* The operator at one core element.  abs_mode evaluates the "absolute
 * stencil" S(p) = sum |w| |X| |C| instead (with the value's own absolute
 * stencil standing in for |value|), which the tests use to scale
 * per-element tolerances. */
static double orc_term_sum(const orc_extent *e, const orc_grid *in, int n_terms, const orc_term *terms,
                           int target, double value, int abs_mode, int64_t i, int64_t j, int64_t k) {
  double acc = 0.0;
  for (int t = 0; t < n_terms; ++t) {
    const orc_term *tm = &terms[t];
    if (tm->out != target) continue;
#if ORC_MUTANT == 3
    if (t == n_terms - 1) continue; /* last term dropped */
#endif
#if ORC_MUTANT == 1
    double x = (tm->in == ORC_VALUE) ? value : orc_read(e, &in[tm->in], i - tm->dx, j + tm->dy, k + tm->dz);
#elif ORC_MUTANT == 7
    double x = (tm->in == ORC_VALUE) ? 0.0 : orc_read(e, &in[tm->in], i + tm->dx, j + tm->dy, k + tm->dz);
#else
    double x = (tm->in == ORC_VALUE) ? value : orc_read(e, &in[tm->in], i + tm->dx, j + tm->dy, k + tm->dz);
#endif
#if ORC_MUTANT == 2
    int64_t cdx = tm->dx > in[tm->coef == ORC_NONE ? 0 : tm->coef].hx ? 0 : tm->dx;
    double c = (tm->coef == ORC_NONE) ? 1.0 : orc_read(e, &in[tm->coef], i + (cdx >= 0 ? cdx : 0), j, k);
#else
    double c = (tm->coef == ORC_NONE) ? 1.0 : orc_read(e, &in[tm->coef], i, j, k);
#endif
    double w = tm->w;
#if ORC_MUTANT == 11
    if (abs_mode) { x = fabs(x); w = fabs(w); } /* the coefficient's absolute value dropped */
#elif ORC_MUTANT == 12
    if (abs_mode) { c = fabs(c); w = fabs(w); } /* the read value's absolute value dropped */
#else
    if (abs_mode) { x = fabs(x); c = fabs(c); w = fabs(w); }
#endif
    acc = acc + (w * x) * c;
  }
  return acc;
}

/* do_all over [lo, hi).  value_out (optional) receives value(p) for every
 * core element, dense in (k, j, i) order over the range. */
int orc_do_all(const orc_extent *e, int n_in, const orc_grid *in, int n_out, const orc_out_grid *out,
               int n_terms, const orc_term *terms, const int64_t lo[3], const int64_t hi[3],
               int abs_mode, double *value_out) {
  int rc = orc_check(e, n_in, in, n_out, n_terms, terms, lo, hi);
  if (rc) return rc;
  const int64_t nx = hi[0] - lo[0], ny = hi[1] - lo[1];
  /* Elements are independent (outputs never alias inputs), so the timing
   * build (-fopenmp) may spread the planes over threads; the values are the
   * same in any order. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t k = lo[2]; k < hi[2]; ++k)
    for (int64_t j = lo[1]; j < hi[1]; ++j)
      for (int64_t i = lo[0]; i < hi[0]; ++i) {
        double v = orc_term_sum(e, in, n_terms, terms, ORC_VALUE, 0.0, abs_mode, i, j, k);
        for (int m = 0; m < n_out; ++m) {
          double r = orc_term_sum(e, in, n_terms, terms, m, v, abs_mode, i, j, k);
          out[m].data[orc_index(e, out[m].hx, out[m].hy, out[m].hz, i, j, k)] = r;
        }
        if (value_out) value_out[((k - lo[2]) * ny + (j - lo[1])) * nx + (i - lo[0])] = v;
      }
  return ORC_OK;
}

/* Threads the timing build (-fopenmp) uses from now on (n >= 1); returns the
 * count in effect, 1 in the correctness build, which has no threads. */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Ordered iteration spaces (Section 3): do_i/j/k_inc visit (i-1,j,k),
 * (i,j-1,k), (i,j,k-1) respectively before (i,j,k); the _dec forms visit the
 * +1 neighbour first.  axis: 0 = i, 1 = j, 2 = k; inc: 1 for _inc, 0 for
 * _dec.  The ordered axis is the outer loop, walked in that direction, so
 * every element comes after its predecessor along it.  Reads see the grids'
 * current contents: an output grid that is also bound as an input is seen
 * already updated at the elements visited before.  At each element every
 * output is computed before any is stored. */
int orc_do_ordered(int axis, int inc, const orc_extent *e, int n_in, const orc_grid *in, int n_out,
                   const orc_out_grid *out, int n_terms, const orc_term *terms, const int64_t lo[3],
                   const int64_t hi[3]) {
  if (axis < 0 || axis > 2 || n_out < 1 || n_out > 8) return ORC_BAD_ARG;
  int rc = orc_check(e, n_in, in, n_out, n_terms, terms, lo, hi);
  if (rc) return rc;
  const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2; /* the two other axes */
  double r[8];
  for (int64_t s = 0; s < hi[axis] - lo[axis]; ++s) {
    const int64_t c = inc ? lo[axis] + s : hi[axis] - 1 - s;
    for (int64_t u = lo[a2]; u < hi[a2]; ++u)
      for (int64_t w = lo[a1]; w < hi[a1]; ++w) {
        int64_t p[3];
        p[axis] = c;
        p[a1] = w;
        p[a2] = u;
        double v = orc_term_sum(e, in, n_terms, terms, ORC_VALUE, 0.0, 0, p[0], p[1], p[2]);
        for (int m = 0; m < n_out; ++m) r[m] = orc_term_sum(e, in, n_terms, terms, m, v, 0, p[0], p[1], p[2]);
        for (int m = 0; m < n_out; ++m)
          out[m].data[orc_index(e, out[m].hx, out[m].hy, out[m].hz, p[0], p[1], p[2])] = r[m];
      }
  }
  return ORC_OK;
}

/* Coloured (red-black) application, the use Section 3 gives for stateful
 * stencils (operators that may query the index of the core element): the
 * operator is applied only at core elements whose index sum i + j + k (a 2D
 * grid has k = 0) has the parity `color` (0 or 1), in lexicographic order,
 * reading the grids' current contents.  An output may also be bound as an
 * input; at each element every output is computed before any is stored.
 * Elements of the other colour are left as they are.  With the 7-point
 * Poisson operator in place, colour 0 then colour 1 is one red-black
 * Gauss-Seidel iteration. */
int orc_do_colored(int color, const orc_extent *e, int n_in, const orc_grid *in, int n_out,
                   const orc_out_grid *out, int n_terms, const orc_term *terms, const int64_t lo[3],
                   const int64_t hi[3]) {
  if ((color != 0 && color != 1) || n_out < 1 || n_out > 8) return ORC_BAD_ARG;
  int rc = orc_check(e, n_in, in, n_out, n_terms, terms, lo, hi);
  if (rc) return rc;
  double r[8];
  for (int64_t k = lo[2]; k < hi[2]; ++k)
    for (int64_t j = lo[1]; j < hi[1]; ++j)
      for (int64_t i = lo[0]; i < hi[0]; ++i) {
#if ORC_MUTANT == 9
        if (((i + j) & 1) != color) continue; /* k left out of the colour */
#else
        if (((i + j + k) & 1) != color) continue;
#endif
        double v = orc_term_sum(e, in, n_terms, terms, ORC_VALUE, 0.0, 0, i, j, k);
        for (int m = 0; m < n_out; ++m) r[m] = orc_term_sum(e, in, n_terms, terms, m, v, 0, i, j, k);
        for (int m = 0; m < n_out; ++m) out[m].data[orc_index(e, out[m].hx, out[m].hy, out[m].hz, i, j, k)] = r[m];
      }
  return ORC_OK;
}

/* do_diamond (Section 3): cells (i-1, j) and (i, j-1) are processed before
 * cell (i, j).  The paper has it for 2D grids; a 3D grid is taken plane by
 * plane, the planes independent.  Lexicographic order (j outer, i inner)
 * is one order that respects it.  Reads see the grids' current contents, so
 * an output bound also as an input is seen updated at elements processed
 * before (offsets with dx, dy <= 0) and not yet updated at elements
 * processed after (dx, dy >= 0); at each element every output is computed
 * before any is stored. */
int orc_do_diamond(const orc_extent *e, int n_in, const orc_grid *in, int n_out, const orc_out_grid *out,
                   int n_terms, const orc_term *terms, const int64_t lo[3], const int64_t hi[3]) {
  if (n_out < 1 || n_out > 8) return ORC_BAD_ARG;
  int rc = orc_check(e, n_in, in, n_out, n_terms, terms, lo, hi);
  if (rc) return rc;
  double r[8];
  for (int64_t k = lo[2]; k < hi[2]; ++k)
    for (int64_t jj = lo[1]; jj < hi[1]; ++jj) {
#if ORC_MUTANT == 10
      const int64_t j = hi[1] - 1 - (jj - lo[1]); /* rows in reverse */
#else
      const int64_t j = jj;
#endif
      for (int64_t i = lo[0]; i < hi[0]; ++i) {
        double v = orc_term_sum(e, in, n_terms, terms, ORC_VALUE, 0.0, 0, i, j, k);
        for (int m = 0; m < n_out; ++m) r[m] = orc_term_sum(e, in, n_terms, terms, m, v, 0, i, j, k);
        for (int m = 0; m < n_out; ++m) out[m].data[orc_index(e, out[m].hx, out[m].hy, out[m].hz, i, j, k)] = r[m];
      }
    }
  return ORC_OK;
}

/* Neumaier's improvement of Kahan summation: the running compensation c
 * collects the rounding error of every addition, taken from whichever
 * operand is larger in magnitude. */
typedef struct { double s, c; } orc_neumaier;

static void orc_neumaier_add(orc_neumaier *a, double x) {
#if ORC_MUTANT == 4
  a->s += x; /* plain recursive sum */
  return;
#endif
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

/* The reduction's running state, fed one value at a time in lexicographic
 * order. */
typedef struct {
  int op;
  double eps;
  orc_neumaier acc;
  double mx;
  int saw_nan;
  int all_within; /* logical_and of |v| <= eps (a NaN compares false) */
} orc_reduction;

static void orc_reduce_add(orc_reduction *r, double v) {
  if (r->op == ORC_WITHIN) {
    r->all_within = r->all_within && (fabs(v) <= r->eps);
  } else if (r->op == ORC_SUM) {
    orc_neumaier_add(&r->acc, v);
  } else if (r->op == ORC_L2) {
#if ORC_MUTANT == 8
    orc_neumaier_add(&r->acc, fabs(v)); /* norm 1 instead of norm 2 */
#else
    orc_neumaier_add(&r->acc, v * v);
#endif
  } else {
#if ORC_MUTANT == 6
    if (0) r->saw_nan = 1;
#else
    if (isnan(v)) r->saw_nan = 1;
#endif
    else if (fabs(v) > r->mx) r->mx = fabs(v);
  }
}

/* The value reduced at element (i, j, k): In_0 itself with no operator,
 * else the operator's value, its outputs written as by orc_do_all. */
static double orc_reduce_element(const orc_extent *e, const orc_grid *in, int n_out, const orc_out_grid *out,
                                 int n_terms, const orc_term *terms, int64_t i, int64_t j, int64_t k) {
  if (n_terms == 0) return orc_read(e, &in[0], i, j, k);
  double v = orc_term_sum(e, in, n_terms, terms, ORC_VALUE, 0.0, 0, i, j, k);
  for (int m = 0; m < n_out; ++m) {
    double r = orc_term_sum(e, in, n_terms, terms, m, v, 0, i, j, k);
    out[m].data[orc_index(e, out[m].hx, out[m].hy, out[m].hz, i, j, k)] = r;
  }
  return v;
}

/* do_reduce over [lo, hi): writes the reduced value to *result.  With
 * n_terms == 0 the per-element value is In_0(p) and no output is written;
 * otherwise the operator runs as in orc_do_all (outputs included) and its
 * value is reduced. */
static int reduce_impl(int op, double eps, const orc_extent *e, int n_in, const orc_grid *in, int n_out,
                       const orc_out_grid *out, int n_terms, const orc_term *terms,
                       const int64_t lo[3], const int64_t hi[3], double *result) {
  if (n_terms == 0) {
    if (n_in < 1 || n_out != 0) return ORC_BAD_ARG;
    orc_term id = {0, 0, 0, 0, ORC_NONE, ORC_VALUE, 1.0};
    int rc = orc_check(e, n_in, in, 0, 1, &id, lo, hi);
    if (rc) return rc;
  } else {
    int rc = orc_check(e, n_in, in, n_out, n_terms, terms, lo, hi);
    if (rc) return rc;
  }
  orc_reduction red = {op, eps, {0.0, 0.0}, 0.0, 0, 1};
#ifdef _OPENMP
  /* timing build: every element's value (and outputs) in parallel over
   * planes into a buffer, then the same lexicographic reduction */
  const int64_t nx = hi[0] - lo[0], ny = hi[1] - lo[1], nz = hi[2] - lo[2];
  const int64_t count = (nx > 0 && ny > 0 && nz > 0) ? nx * ny * nz : 0;
  double *vals = count ? (double *)malloc((size_t)count * sizeof(double)) : NULL;
  if (count && !vals) return ORC_BAD_ARG;
#pragma omp parallel for schedule(static)
  for (int64_t k = lo[2]; k < hi[2]; ++k)
    for (int64_t j = lo[1]; j < hi[1]; ++j)
      for (int64_t i = lo[0]; i < hi[0]; ++i)
        vals[((k - lo[2]) * ny + (j - lo[1])) * nx + (i - lo[0])] =
            orc_reduce_element(e, in, n_out, out, n_terms, terms, i, j, k);
  for (int64_t q = 0; q < count; ++q) orc_reduce_add(&red, vals[q]);
  free(vals);
#else
  for (int64_t k = lo[2]; k < hi[2]; ++k)
    for (int64_t j = lo[1]; j < hi[1]; ++j)
      for (int64_t i = lo[0]; i < hi[0]; ++i)
        orc_reduce_add(&red, orc_reduce_element(e, in, n_out, out, n_terms, terms, i, j, k));
#endif
  if (op == ORC_WITHIN) *result = red.all_within ? 1.0 : 0.0;
  else if (op == ORC_SUM) *result = red.acc.s + red.acc.c;
  else if (op == ORC_L2) *result = sqrt(red.acc.s + red.acc.c);
  else *result = red.saw_nan ? NAN : red.mx;
  return ORC_OK;
}

int orc_do_reduce(int op, const orc_extent *e, int n_in, const orc_grid *in, int n_out,
                  const orc_out_grid *out, int n_terms, const orc_term *terms,
                  const int64_t lo[3], const int64_t hi[3], double *result) {
  if (op != ORC_SUM && op != ORC_MAXABS && op != ORC_L2) return ORC_BAD_ARG;
  return reduce_impl(op, 0.0, e, n_in, in, n_out, out, n_terms, terms, lo, hi, result);
}

/* Section 5.2's convergence test as a reduction: the logical_and over the
 * range of |value| <= eps, as 1.0 or 0.0 (1.0 for an empty range). */
int orc_do_reduce_within(double eps, const orc_extent *e, int n_in, const orc_grid *in, int n_out,
                         const orc_out_grid *out, int n_terms, const orc_term *terms,
                         const int64_t lo[3], const int64_t hi[3], double *result) {
  if (!(eps >= 0.0)) return ORC_BAD_ARG;
  return reduce_impl(ORC_WITHIN, eps, e, n_in, in, n_out, out, n_terms, terms, lo, hi, result);
}
