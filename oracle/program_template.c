/*
 * program_template.c -- oracle side of run-time compiled point operators.
 *
 * TEST INFRASTRUCTURE ONLY (see gscl_oracle.c).  oracle.py pastes a point
 * operator's body (C statements reading in<a>(dx, dy, dz), the index i, j, k,
 * and assigning out<m>) into the marked places, compiles it with gcc
 * (-O2 -ffp-contract=off, FP64) and runs it over a range in lexicographic
 * order, as do_all applies a stencil operator at every core element
 * (Section 3); the body's `value` at each element can be returned for
 * do_reduce.  A read beyond the declared reach returns 0 and is counted.
 */
#include <math.h>
#include <stdint.h>

typedef double real;

typedef struct {
  int64_t nx, ny, nz;
} orc_extent;

typedef struct {
  const double *data;
  int32_t hx, hy, hz;
} orc_grid;

typedef struct {
  double *data;
  int32_t hx, hy, hz;
} orc_out_grid;

static int64_t orc_at(const orc_extent *e, int32_t hx, int32_t hy, int32_t hz, int64_t i, int64_t j, int64_t k) {
  return ((k + hz) * (e->ny + 2 * hy) + (j + hy)) * (e->nx + 2 * hx) + (i + hx);
}

static double orc_in(const orc_extent *e, const orc_grid *g, int64_t i, int64_t j, int64_t k, int dx, int dy,
                     int dz, const int32_t reach[3], int64_t *outside) {
  if (dx < -reach[0] || dx > reach[0] || dy < -reach[1] || dy > reach[1] || dz < -reach[2] || dz > reach[2]) {
    ++*outside;
    return 0.0;
  }
  return g->data[orc_at(e, g->hx, g->hy, g->hz, i + dx, j + dy, k + dz)];
}

/* values (optional): the body's `value` at every core element of the range,
 * dense in (k, j, i) order. */
int orc_program(const orc_extent *e, const orc_grid *in, const orc_out_grid *out, const int64_t lo[3],
                const int64_t hi[3], const int32_t reach[3], int64_t *outside, double *values) {
  int64_t q = 0;
  for (int64_t k = lo[2]; k < hi[2]; ++k)
    for (int64_t j = lo[1]; j < hi[1]; ++j)
      for (int64_t i = lo[0]; i < hi[0]; ++i) {
/*@DEFS@*/
        real value = 0;
/*@DECL@*/
        {
/*@BODY@*/
        }
        if (values) values[q++] = value;
/*@STORES@*/
      }
  return 0;
}
