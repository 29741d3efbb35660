/*
 * gscl.h -- C ABI of the B300 generic stencil library (libgscl.so).
 *
 * The library implements the two iteration spaces on the hot path of the
 * generic stencil library of Bianco and Varetto, "A Generic Library for
 * Stencil Computations" (arXiv 1207.1746):
 *
 *   do_all     apply a stencil operator at every core element of an
 *              iteration range, in no guaranteed order (Section 3);
 *   do_reduce  the same, reducing the operator's per-element return value
 *              with a commutative operator (Section 3, and the fused
 *              diffusion + convergence loop of Section 5.2);
 *
 * plus the grids they run on (Section 3: a regular grid is a d-dimensional
 * array; its stencil shape fixes the halo an operator may read) and the
 * ping-pong swap of Section 5.2.  Every computation runs in hand-written
 * sm_103a CUDA kernels; there is no host fallback.
 *
 * Conventions shared by every entry point:
 *  - Return value: a gscl_status.  GSCL_OK means the arguments were valid and
 *    the work was enqueued on the given stream; device-side failures surface
 *    at the next gscl_sync() (or another synchronising call) on that stream.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  All work is asynchronous unless a function says
 *    otherwise.  The calling thread's current CUDA device must be the device
 *    that owns the grids.
 *  - Memory: the library never allocates grid storage.  Device buffers are
 *    owned by the caller (for example a PyTorch tensor) and borrowed by the
 *    handles that wrap them; the caller keeps them alive until the handle is
 *    destroyed and all work on them has completed.
 *  - Handles are opaque 64-bit ids; a destroyed or never-created id is
 *    rejected with GSCL_ERR_STATE (a call on a stale handle is an error, not
 *    undefined behaviour; compare Fig. 2b, where an iteration space outside a
 *    valid context is an error).
 *  - Thread safety: calls may come from several host threads; the handle
 *    registry is locked internally.  Concurrent kernels that write the same
 *    grid race, as any CUDA work does.
 */
#ifndef GSCL_H
#define GSCL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gscl_status {
  GSCL_OK = 0,
  GSCL_ERR_INVALID = 1,     /* malformed argument: NULL pointer, bad count or code, misaligned buffer */
  GSCL_ERR_RANGE = 2,       /* iteration range outside the interior, or a read outside a grid's halo */
  GSCL_ERR_ALIAS = 3,       /* an output is read at a non-zero offset, or bound twice */
  GSCL_ERR_DTYPE = 4,       /* the grids of one call do not share one storage dtype */
  GSCL_ERR_SHAPE = 5,       /* the grids of one call do not share one interior extent / layout */
  GSCL_ERR_OOM = 6,         /* a caller-supplied buffer or workspace is too small */
  GSCL_ERR_CUDA = 7,        /* a CUDA runtime or driver call failed */
  GSCL_ERR_STATE = 8,       /* destroyed or unknown handle */
  GSCL_ERR_TIMEOUT = 9,     /* a bounded device-side wait gave up (reported by gscl_sync) */
  GSCL_ERR_UNSUPPORTED = 10 /* valid request outside what the library implements (e.g. too many terms) */
} gscl_status;

typedef enum gscl_dtype {
  GSCL_F64 = 0,  /* FP64 storage, FP64 arithmetic */
  GSCL_F32 = 1,  /* FP32 storage, FP32 arithmetic */
  GSCL_BF16 = 2  /* BF16 storage, FP32 arithmetic, round-to-nearest-even stores */
} gscl_dtype;

typedef enum gscl_reduce_op {
  GSCL_SUM = 0,    /* sum of the values, FP64 with compensation */
  GSCL_MAXABS = 1, /* max |value| (NaN if any value is NaN); 0 for an empty range */
  GSCL_L2 = 2      /* sqrt(sum of value^2), FP64 with compensation */
} gscl_reduce_op;

typedef uint64_t gscl_grid; /* 0 is never a valid handle */

/* Term input / output codes beside ordinary grid indices. */
#define GSCL_VALUE 254 /* in: the operator's returned value at the core element; out: a term of that value */
#define GSCL_NONE 255  /* coef: no coefficient grid */
#define GSCL_MAX_TERMS 64
#define GSCL_MAX_IN 8
#define GSCL_MAX_OUT 3
#define GSCL_MAX_HALO 4

/*
 * One term of a stencil operator (Section 3: an operator reads elements of
 * several grids at fixed offsets from the core element and may write the
 * core element of its output grids; it may also return a value):
 *
 *   out == m (0 <= m < n_out):  out_m(p)  += w * X * C
 *   out == GSCL_VALUE:          value(p)  += w * X * C
 *
 * with X = in_grid[in](p + (dx,dy,dz)), or X = value(p) when in == GSCL_VALUE
 * (then the offset must be 0 and out must be an output index), and
 * C = in_grid[coef](p) (coefficient read at the core element) or 1 when
 * coef == GSCL_NONE.  value(p) is formed from its terms before any output,
 * so a term of an output may use it: that is how two operators share one
 * scan (the paper's fuse(), Section 5.2).  Terms may be given in any order;
 * the sum over an output's terms is evaluated in an unspecified order with
 * fused multiply-adds in the grids' arithmetic type.  On IEEE FP64 grids,
 * terms that differ only in the sign pattern of their offset (one input, one
 * coefficient, one destination; the six neighbours of a 7-point star, the
 * rings of a biharmonic) and have equal weights (a pair: opposite weights)
 * may be summed first and weighted once: w * (x1 + x2 + ...).  Every
 * addition is an IEEE binary64 addition rounded to nearest (some of them are
 * computed on the integer pipe, with identical results), so the value differs
 * from the term-by-term sum only by rounding.  The environment variable
 * GSCL_FP64_INT_ADD=0 keeps one fused multiply-add per term.
 */
typedef struct gscl_term {
  int8_t dx, dy, dz;
  uint8_t in, coef, out;
  uint16_t reserved; /* must be 0 */
  double w;
} gscl_term;

typedef struct gscl_stencil {
  int32_t n_terms;          /* 1 .. GSCL_MAX_TERMS */
  int32_t reserved;         /* must be 0 */
  const gscl_term *terms;   /* host memory, read during the call only */
} gscl_stencil;

/* Iteration range in interior coordinates, half-open [lo, hi) per axis
 * (x, y, z).  For a 2D grid the z range must be [0, 1). */
typedef struct gscl_range {
  int64_t lo[3], hi[3];
} gscl_range;

/* Layout facts of a grid handle. */
typedef struct gscl_grid_desc {
  int32_t ndim;
  int32_t dtype;
  int64_t n[3];            /* interior points per axis x, y, z (z = 1 in 2D) */
  int32_t halo[3];         /* halo per axis (z halo 0 in 2D) */
  int32_t elem_bytes;
  int64_t pitch_elems;     /* row pitch */
  int64_t offset_elems;    /* leading pad so interior element (0,0,0) is 128-byte aligned */
  int64_t plane_elems;     /* pitch * (n[1] + 2 halo[1]) */
  int64_t bytes;           /* storage size */
  void *dev_buf;           /* borrowed device buffer */
} gscl_grid_desc;

/*
 * Storage layout of a grid (x fastest; a 2D grid has nz = 1, hz = 0):
 *   element (i, j, k), -h <= index < n + h per axis, is at element
 *   offset_elems + ((k + hz) * (ny + 2hy) + (j + hy)) * pitch_elems + (i + hx)
 * of the buffer.  pitch_elems is a multiple of 128 bytes and offset_elems
 * makes interior element (0,0,0) 128-byte aligned, so tiles of interior
 * rows can be moved with TMA and 16-byte vectors.
 *
 * gscl_grid_layout computes the layout without creating anything.  Every
 * output pointer is required.  Errors: GSCL_ERR_INVALID for ndim not 2 or
 * 3, n < 1, halo < 0 or > GSCL_MAX_HALO, a non-zero z halo or nz != 1 in
 * 2D, an unknown dtype.
 */
gscl_status gscl_grid_layout(int32_t ndim, const int64_t n[3], const int32_t halo[3], int32_t dtype,
                             int64_t *pitch_elems, int64_t *offset_elems, int64_t *bytes);

/*
 * Wraps a caller-owned device buffer of at least the layout's `bytes` as a
 * grid.  The buffer must be 128-byte aligned (GSCL_ERR_INVALID otherwise);
 * buf_bytes smaller than the layout gives GSCL_ERR_OOM.  The handle borrows
 * the buffer: destroying the handle does not free it.  Contents are not
 * touched.
 */
gscl_status gscl_grid_create(int32_t ndim, const int64_t n[3], const int32_t halo[3], int32_t dtype,
                             void *dev_buf, int64_t buf_bytes, gscl_grid *out);

/* Releases a handle (not its buffer).  GSCL_ERR_STATE for an unknown handle. */
gscl_status gscl_grid_destroy(gscl_grid g);

/* Fills *out with the handle's layout and current buffer (which gscl_swap
 * and multi-sweep gscl_do_all may exchange between handles). */
gscl_status gscl_grid_info(gscl_grid g, gscl_grid_desc *out);

/*
 * Copies between a dense host array and the grid, halo included.  The host
 * array has (nz + 2hz) x (ny + 2hy) x (nx + 2hx) elements of the grid's dtype,
 * x fastest.  Asynchronous on `stream` (pinned host memory makes it truly
 * so); the host array must stay valid until the stream reaches the copy.
 */
gscl_status gscl_grid_copy_from_host(gscl_grid g, const void *host, void *stream);
gscl_status gscl_grid_copy_to_host(gscl_grid g, void *host, void *stream);

/*
 * Exchanges the storage of two grids of identical layout (Section 5.2,
 * swap_grids): O(1), no data moves, halos travel with their storage.  The
 * handle values stay where they are; what each names is exchanged.
 * GSCL_ERR_SHAPE if the layouts differ.  Not stream-ordered: the caller
 * swaps between enqueued sweeps, as with any pointer exchange.
 */
gscl_status gscl_swap(gscl_grid *a, gscl_grid *b);

/*
 * do_all (Section 3): applies the operator at every core element of `range`
 * (NULL = the whole interior) reading grids in[0..n_in) and writing
 * out[0..n_out) at the core elements only.  Halos are never written.
 *
 *  - All grids share ndim, interior extent and dtype (GSCL_ERR_SHAPE /
 *    GSCL_ERR_DTYPE); halos may differ per grid, and every read p + offset
 *    must stay inside the read grid's halo for every p in the range
 *    (GSCL_ERR_RANGE).
 *  - do_all promises no order (Section 3), so an output grid that is also an
 *    input may be read only at offset 0 (GSCL_ERR_ALIAS otherwise), and no
 *    grid may be an output twice.
 *  - 1 <= n_in <= GSCL_MAX_IN, 1 <= n_out <= GSCL_MAX_OUT,
 *    n_terms <= GSCL_MAX_TERMS (GSCL_ERR_UNSUPPORTED beyond).
 *  - sweeps >= 1.  sweeps > 1 repeats the operator with in[0] and out[0] as
 *    a ping-pong pair (identical layouts, GSCL_ERR_SHAPE otherwise): sweep s
 *    reads the previous sweep's result in place of in[0], with the halo of
 *    the grid that result went to, as single sweeps alternate.  On return
 *    out[0] names the result of the last sweep and in[0] that of the sweep
 *    before it (the two handles may have exchanged storage, as by
 *    gscl_swap; halos travel with their storage, so ping-pong grids usually
 *    carry identical halos).  Sweeps fused per launch (gscl_tune_sweeps)
 *    give the same results, the storage each handle names included (3D
 *    grids: when in[0] and out[0] carry identical halos; 2D grids: always);
 *    the last launch of a call is always a single sweep.
 *  - An empty range enqueues nothing.
 */
gscl_status gscl_do_all(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                        int32_t n_out, const gscl_range *range, int32_t sweeps, void *stream);

/*
 * Red-black colouring, the use Section 3 gives for stateful stencils
 * (operators that may query the index of their core element): applies the
 * operator only at the core elements of `range` whose interior index sum
 * i + j + k (k = 0 on 2D grids) has the parity `color` (0 or 1); elements of
 * the other colour are not written.  half_sweeps >= 1 applications alternate
 * the colour, starting with `color`, each reading the previous one's result.
 *
 *  - An output may also be an input when both name the same grid (the same
 *    storage and layout; GSCL_ERR_ALIAS otherwise), read at offset 0 or at
 *    offsets with odd dx + dy + dz: elements of the other colour, which the
 *    call does not write, so the update is well defined in place.  Any other
 *    read of it is GSCL_ERR_ALIAS.
 *  - With the 7-point Poisson operator u <- (sum6 u + f) / 6 in place, colour
 *    0 then colour 1 is one red-black Gauss-Seidel iteration; the weights
 *    (1 - w) on u(0) and w / 6 on the others give SOR with factor w.
 *  - Other rules as gscl_do_all (n_out >= 1, GSCL_ERR_INVALID for a colour
 *    outside {0, 1} or half_sweeps < 1).  Asynchronous on `stream`.
 */
gscl_status gscl_do_colored(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                            int32_t n_out, const gscl_range *range, int32_t color, int32_t half_sweeps,
                            void *stream);

/*
 * Which implementation gscl_do_all / gscl_do_reduce pick for this operator
 * with n_in inputs and n_out outputs.  Section 1 of the paper keeps a generic
 * implementation of every construct and uses a better-suited one where it
 * exists; likewise the library runs any operator through a generic kernel
 * that interprets the term list, and a few operator structures (the 7-point
 * heat / Jacobi / Poisson / residual operators, the 2D 5-point Jacobi, the
 * 8-input / 3-output climate operator, differences and identities) through
 * kernels compiled for that structure, with the weights still taken from the
 * descriptor.  Returns a non-negative id for a compiled structure, -1 for the
 * generic kernel.  Host-only; setting the environment variable
 * GSCL_GENERIC_ONLY=1 makes every call use the generic kernel.
 */
int32_t gscl_stencil_specialization(const gscl_stencil *op, int32_t n_in, int32_t n_out);

/*
 * dst(p) = alpha * src(p) (+ dst(p) when accumulate != 0) over `range`
 * (NULL = the interior), for any pair of storage dtypes: the casts and the
 * correction of mixed-precision iterative refinement (an FP64 iterate
 * corrected by an FP32 solve: u64 += d32; an FP64 residual handed to the
 * FP32 solve: r32 = r64).  Arithmetic in FP64, one rounding to dst's type
 * (round to nearest even).  Halos are not touched.  Grids must share the
 * interior extent (GSCL_ERR_SHAPE); src may be dst itself.  No counterpart
 * in the paper: the mixed-precision solves of the serving workload need it.
 */
gscl_status gscl_convert(gscl_grid dst, gscl_grid src, double alpha, int32_t accumulate, const gscl_range *range,
                         void *stream);

/*
 * Autotuner for multi-sweep gscl_do_all: times sweeps fused per pass
 * (temporal blocking; the paper's wide ghost areas, Section 2, kept on chip)
 * on these grids, passes from in[0] into out[0] (in[0] is left unchanged),
 * and records the fastest per sweep for this operator structure, dtype and
 * extent; later multi-sweep calls use it (GSCL_TEMPORAL=K overrides, with
 * GSCL_TEMPORAL_TILE=0..3 choosing a 2D tile shape).  Fused passes are
 * bit-identical to single sweeps.  Candidates: the radius-1 7-point star
 * operators with FP32 / BF16 storage over the whole interior of a 3D grid,
 * K = 1 .. 4 (trial_sweeps sweeps each); the 2D 5-point operators over the
 * whole interior of a one-plane grid (any storage, IEEE arithmetic for
 * FP64), K = 1, 2, 3, 4, 6, 8, 12, 16 over four tile shapes (at least 48
 * sweeps each).  Otherwise *best_factor = 1.  Synchronises.
 */
gscl_status gscl_tune_sweeps(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                             int32_t n_out, int32_t trial_sweeps, void *stream, int32_t *best_factor);

/* Orders of the ordered iteration spaces (Section 3). */
typedef enum {
  GSCL_I_INC = 0, /* (i-1, j, k) is visited before (i, j, k) */
  GSCL_I_DEC = 1, /* (i+1, j, k) before (i, j, k) */
  GSCL_J_INC = 2, /* (i, j-1, k) before (i, j, k) */
  GSCL_J_DEC = 3, /* (i, j+1, k) before (i, j, k) */
  GSCL_K_INC = 4, /* (i, j, k-1) before (i, j, k) */
  GSCL_K_DEC = 5  /* (i, j, k+1) before (i, j, k) */
} gscl_order;

/*
 * Ordered iteration spaces (Section 3: do_j_inc, do_j_dec, do_k_inc,
 * do_k_dec): applies the operator at every core element of the range so that
 * along the ordered axis each element comes after its predecessor (other
 * axes in any order); outputs are written as by gscl_do_all.
 *
 *  - An output grid may also be bound as an input (the same handle, or a
 *    handle of the same storage and layout).  Terms read it at offset 0 (the
 *    value before this element is written) or at the element visited just
 *    before along the ordered axis ((0,0,-1) for GSCL_K_INC, (0,1,0) for
 *    GSCL_J_DEC, ...), which holds the value this call wrote there, or at the
 *    range's first element the grid's current content (halo or untouched
 *    interior).  Any other read of it is GSCL_ERR_ALIAS.  This is how a
 *    recurrence along a column is written: running sums, bidiagonal forward
 *    or backward substitution (x(k) = g(k) - m(k) x(k-1) with m a coefficient
 *    grid), upwind integration.
 *  - At each element every output is computed before any is stored; the
 *    stored (rounded) value is what the next element reads.
 *  - Terms may also write the returned value (out = GSCL_VALUE) and read it
 *    (in = GSCL_VALUE), as in do_all; it is not reduced.
 *  - Along y and z one thread walks one column; along x (GSCL_I_INC /
 *    GSCL_I_DEC) a warp stages 32 steps of 32 rows in shared memory at a time
 *    and takes operators with at most 8 distinct element loads per element
 *    (GSCL_ERR_UNSUPPORTED beyond).
 *  - Errors, range and dtype rules as gscl_do_all (n_out >= 1).  Asynchronous
 *    on `stream`.
 */
gscl_status gscl_do_ordered(int32_t order, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                            const gscl_grid *out, int32_t n_out, const gscl_range *range, void *stream);

/*
 * Which implementation gscl_do_ordered picks for this call (the interior as
 * range), in *shape: a non-negative id for a recurrence compiled for its
 * structure, -1 for the interpreted term loop with look-ahead loads, -2 for
 * the interpreted loop with loads per term (more than 8 distinct loads per
 * element, or BF16 storage), -3 for the interpreted loop on rows along x
 * staged in shared memory (GSCL_I_INC / GSCL_I_DEC; the compiled structures
 * report their ids along x too).  The compiled structures, with the terms in
 * this order and the weights a, b, c any values:
 *   0  x = a x(prev) + b f                   (running sums)
 *   1  x = b f + a x(prev)
 *   2  x = a g + b m x(prev)                 (bidiagonal substitution)
 *   3  x = b m x(prev) + a g
 *   4  x = a f + b g + c x(prev)
 * where x(prev) is the output read at the element just visited and f, g, m
 * are grids read at any offsets.  Every path computes the same operations in
 * the same order, so their results are bit-identical.  Host-only; arguments
 * and errors as gscl_do_ordered; GSCL_GENERIC_ONLY=1 in the environment
 * turns the compiled structures off.
 */
gscl_status gscl_ordered_specialization(int32_t order, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                                        const gscl_grid *out, int32_t n_out, int32_t *shape);

/*
 * do_diamond (Section 3): applies the operator at every core element of the
 * range so that (i-1, j, k) and (i, j-1, k) are processed before (i, j, k).
 * The paper defines it for 2D grids; a 3D grid is taken plane by plane, the
 * planes independent (and in any order).
 *
 *  - An output may also be an input when both name the same grid (the same
 *    storage and layout; GSCL_ERR_ALIAS otherwise).  Terms read it in the
 *    same plane (dz = 0) at offsets whose dx and dy have one sign: dx, dy <= 0
 *    reads an element already processed, holding the value this call wrote
 *    there (or the grid's content outside the range), and dx, dy >= 0 one not
 *    yet processed, holding its value from before the call.  Mixed signs, or
 *    another plane, would depend on the schedule: GSCL_ERR_ALIAS.  This is how
 *    2D recurrences are written: summed-area tables
 *    (x = f + x(i-1,j) + x(i,j-1) - x(i-1,j-1)) and Gauss-Seidel in the
 *    natural order (u = (u(i-1,j) + u(i,j-1) + u(i+1,j) + u(i,j+1)) / 4).
 *  - At each element every output is computed before any is stored; the
 *    stored (rounded) value is what later elements read.
 *  - Value terms (out = GSCL_VALUE, in = GSCL_VALUE) as in gscl_do_all; the
 *    value is not reduced.
 *  - GSCL_ERR_UNSUPPORTED beyond 65535 planes, or when the input tiles with
 *    their aprons exceed shared memory.  Other errors, range and dtype rules
 *    as gscl_do_all (n_out >= 1).  Asynchronous on `stream`.
 */
gscl_status gscl_do_diamond(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                            int32_t n_out, const gscl_range *range, void *stream);

/*
 * Arithmetic of FP64 grids (not an operation of the paper; a B300 precision
 * mode).  GSCL_FP64_IEEE (default): IEEE FP64 fused multiply-adds, bound on
 * B300 by its FP64 pipe (about 1.7 per clock per SM).  GSCL_FP64_PAIR: each
 * double read is split on the integer pipe into two floats (24 + 24
 * significant bits; the split error is below 2^-47 |x|), terms are
 * accumulated with an exact FP32 two-product and a two-sum, and the stored
 * value is the double nearest the pair.  The error of one operator
 * evaluation is then a small multiple of 2^-47 S(p), S(p) = sum |w X C|
 * (the absolute stencil), inside the FP64 tolerance of 1e-13 S(p) but about
 * 2^6 above IEEE FP64.  A pair holds magnitudes from about 2^-100 to below
 * 2^128 (FP32's exponent range): grids whose values or intermediate results
 * leave that range need IEEE FP64 (beyond it values become infinite, below it
 * they lose bits); NaN propagates, and an infinity becomes NaN.  Storage,
 * traffic and reductions (FP64 accumulation)
 * are the same in both modes; ordered iteration spaces and gscl_convert keep
 * IEEE FP64.  Process-wide; the environment variable GSCL_FP64_ARITH=pair sets
 * the initial mode.  Kernels already enqueued keep the mode they were
 * launched with.
 */
typedef enum { GSCL_FP64_IEEE = 0, GSCL_FP64_PAIR = 1 } gscl_fp64_arithmetic;
gscl_status gscl_set_fp64_arithmetic(int32_t mode);
int32_t gscl_get_fp64_arithmetic(void);

/* Bytes of device workspace one gscl_do_reduce call needs (a constant). */
int64_t gscl_reduce_workspace_bytes(void);

/*
 * do_reduce (Section 3): runs the operator like gscl_do_all (outputs, if
 * n_out > 0, are written exactly as do_all writes them: the fused operator
 * of Section 5.2) and reduces its returned value over the range with `op`.
 * op == NULL reduces in[0] itself (n_out must be 0); otherwise the operator
 * needs at least one term with out == GSCL_VALUE.
 *
 *  - result: one double.  result_on_host = 0: a device pointer, written
 *    asynchronously.  result_on_host = 1: a host pointer; the call copies the
 *    value back, synchronises `stream` and then reads the device error word
 *    as gscl_sync does: if a bounded device-side wait gave up (in this call
 *    or in earlier work on the device) the value is not to be trusted and the
 *    call returns GSCL_ERR_TIMEOUT (GSCL_ERR_RANGE for a run-time compiled
 *    operator's out-of-reach read), clearing the flag.
 *  - workspace: device memory of gscl_reduce_workspace_bytes() bytes.  Each
 *    call clears the arrival ticket it needs (its first 256 bytes) on
 *    `stream` before the launch, so the contents left by any earlier call,
 *    including one whose wait gave up, do not matter.  Calls that may
 *    overlap on the GPU (different streams) need separate workspaces.
 *    GSCL_ERR_OOM if workspace_bytes is too small.
 *  - Accumulation is FP64 for every dtype: SUM and L2 are compensated across
 *    z-steps, threads and CTAs, and combined in a fixed order, so a given
 *    launch configuration gives bit-identical results run to run.  An empty
 *    range gives 0.
 */
gscl_status gscl_do_reduce(int32_t reduce_op, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                           const gscl_grid *out, int32_t n_out, const gscl_range *range, double *result,
                           int32_t result_on_host, void *workspace, int64_t workspace_bytes, void *stream);

/*
 * The convergence test of Section 5.2 as a reduction: do_reduce of the
 * operator's returned value with logical_and over the per-element tests
 * |value| <= eps.  *result is 1.0 if every element of the range passes (also
 * for an empty range) and 0.0 otherwise; a NaN value fails.  Equivalent to
 * max |value| <= eps, computed by the MAXABS tree and decided on the device
 * by the last CTA, so the decision can stay on the GPU (result_on_host = 0).
 * Arguments, outputs, workspace and errors as gscl_do_reduce; eps must be
 * >= 0 (GSCL_ERR_INVALID otherwise).
 */
gscl_status gscl_do_reduce_within(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                                  int32_t n_out, const gscl_range *range, double eps, double *result,
                                  int32_t result_on_host, void *workspace, int64_t workspace_bytes, void *stream);

/*
 * Batched sweeps (many independent grid sets of one operator).
 *
 * A batch binds one operator to n_inst instances; instance i uses grids
 * in[i * n_in .. i * n_in + n_in) and out[i * n_out .. i * n_out + n_out),
 * each instance validated as gscl_do_all validates one call (instances may
 * differ in extent, not in dtype).  Every sweep of all instances is one
 * launch: a host-built work-list splits the instances' (tile, z plane) work
 * evenly over one wave of CTAs, so uneven instances share the GPU without
 * one launch per instance.  The batch owns a small device allocation for its
 * tables (freed by gscl_batch_destroy); grid storage stays the caller's.
 * Batches hold their instances' handles: destroy the batch before them.
 * No counterpart in the paper: batching is how the library serves many
 * small solves at once on one GPU.
 */
typedef uint64_t gscl_batch;

gscl_status gscl_batch_create(const gscl_stencil *op, int32_t n_inst, const gscl_grid *in, int32_t n_in,
                              const gscl_grid *out, int32_t n_out, gscl_batch *out_batch);
gscl_status gscl_batch_destroy(gscl_batch b);

/* Number of CTAs and work-list segments of one launch, and the compiled
 * operator structure used (as gscl_stencil_specialization, -1 generic). */
gscl_status gscl_batch_info(gscl_batch b, int32_t *ctas, int32_t *segments, int32_t *specialization);

/* Tile shape (core elements, x by y) the batch's launches use: the dtype's
 * default, or what gscl_batch_tune chose (FP32 / BF16 batches may get
 * 64-column tiles with 4 rows per warp, which waste fewer lanes on narrow
 * grids). */
gscl_status gscl_batch_tile(gscl_batch b, int32_t *tile_x, int32_t *tile_y);

/*
 * `sweeps` sweeps of every instance with in[0] / out[0] as the ping-pong
 * pair, exactly as gscl_do_all(..., sweeps) on each instance alone (same
 * point arithmetic, so bit-identical results); on return out[0] names the
 * last result and in[0] the one before it.  Batches of 2D grids under a
 * 5-point operator may fuse several sweeps per launch (gscl_batch_tune,
 * gscl_batch_set_temporal): the last launch stays a single sweep.
 * use_graph != 0 captures the group's launches once per (sweeps, starting
 * buffer) in a CUDA graph and replays it on `stream`.
 */
gscl_status gscl_batch_run(gscl_batch b, int32_t sweeps, int32_t use_graph, void *stream);

/*
 * Temporal blocking of a batch (the paper's wide ghost areas, Section 2):
 * sweeps fused per launch (1: none) and its tile (x by y core elements; 0 x
 * 0 when nothing fuses).  gscl_batch_set_temporal sets them:
 * sweeps_per_launch in [1, 16], tile_shape in [0, 4) naming 32 x 16,
 * 32 x 32, 16 x 16 or 64 x 32 tiles (GSCL_ERR_INVALID otherwise).  Batches
 * of one-plane (2D) grids under a 5-point operator with one input and one
 * output fuse up to 16 sweeps (IEEE arithmetic for FP64 grids); batches of
 * 3D FP32 / BF16 grids under a radius-1 7-point star operator fuse two
 * (128 x 14 tiles, tile_shape ignored; in[0] and out[0] of each instance
 * must carry identical halos, as for gscl_do_all's fused passes).  Other
 * requests return GSCL_ERR_UNSUPPORTED.  Results are bit-identical to
 * single sweeps.  No counterpart in the
 * paper's API: its ghost width is a grid property, here it is a launch
 * choice.
 */
gscl_status gscl_batch_temporal(gscl_batch b, int32_t *sweeps_per_launch, int32_t *tile_x, int32_t *tile_y);
gscl_status gscl_batch_set_temporal(gscl_batch b, int32_t sweeps_per_launch, int32_t tile_shape);

/*
 * Coloured batches: red-black sweeps (Section 3, stateful stencils: the
 * colour of core element (i, j, k) is the parity of i + j + k) of many
 * independent grid sets, every half-sweep of all of them in one launch.
 *
 * gscl_batch_create_colored takes ops[0 .. n_inst): one operator per
 * instance.  They must share the structure of ops[0] (the same number of
 * terms, each with the same offsets, grids and destination) and may differ
 * in their weights, so each instance can carry its own factor (the SOR
 * factor that is optimal for its own grid size, for instance).  Instance i
 * is validated as gscl_do_colored validates one call with ops[i]: its
 * output may also be an input (the same grid), read at offset 0 or at odd
 * offsets, and is then updated in place.  n_out >= 1.  Other rules,
 * ownership and the batch's device tables as gscl_batch_create.
 *
 * gscl_batch_run_colored applies each instance's operator at the elements
 * of colour `color` (0 or 1), then of the other colour, half_sweeps times in
 * all (GSCL_ERR_INVALID for another colour or half_sweeps < 1), exactly as
 * gscl_do_colored(ops[i], ..., color, half_sweeps) on each instance alone
 * (same point arithmetic: bit-identical results).  use_graph != 0 captures
 * the launches once per (color, half_sweeps) in a CUDA graph and replays
 * it.  Asynchronous on `stream`.  A coloured batch is run only this way:
 * gscl_batch_run, gscl_batch_reduce and gscl_batch_tune reject it.
 */
gscl_status gscl_batch_create_colored(const gscl_stencil *ops, int32_t n_inst, const gscl_grid *in, int32_t n_in,
                                      const gscl_grid *out, int32_t n_out, gscl_batch *out_batch);
gscl_status gscl_batch_run_colored(gscl_batch b, int32_t color, int32_t half_sweeps, int32_t use_graph,
                                   void *stream);

/*
 * One sweep of the batch's operator (outputs written as gscl_do_reduce
 * writes them) reducing its returned value per instance into results[i]
 * (device memory, n_inst doubles).  Per-instance sums are folded in a fixed
 * order for a given batch; they agree with gscl_do_reduce on the instance
 * alone to rounding (the partition into partial sums differs).
 */
gscl_status gscl_batch_reduce(gscl_batch b, int32_t reduce_op, double *results, void *stream);

/*
 * Autotuner: times two groups of trial_sweeps sweeps (in[0] -> out[0], so
 * in[0] is left unchanged and out[0] receives one sweep) for each tile shape
 * (warps per CTA 2/4/8 x prefetched planes 1/2/3, and for FP32 / BF16
 * batches both the default 128-column tiles and 64-column tiles with 4 rows
 * per warp), keeps the shape whose better group was fastest and reports its
 * warps and prefetch (gscl_batch_tile gives the tile).  Batches that can
 * fuse sweeps (gscl_batch_set_temporal) then time the factors (2D: 1, 2, 3,
 * 4, 6, 8, 12 and 16 sweeps per launch over the four fused tile shapes, at
 * least 48 sweeps each; 3D: 1 and 2, trial_sweeps sweeps each) and keep the
 * fastest per sweep (gscl_batch_temporal reports it).
 * Synchronises `stream`.
 */
gscl_status gscl_batch_tune(gscl_batch b, int32_t trial_sweeps, void *stream, int32_t *warps, int32_t *prefetch);

/*
 * gscl_do_reduce_noalloc -- gscl_do_reduce for callers that cannot allocate
 * device memory.  The paper has no counterpart: this entry point exists for
 * the library's users, not for the method.
 *
 * Who needs it: programs that give all device memory to their own allocator
 * at start-up and forbid allocations afterwards (a C or Fortran simulation
 * code with a fixed memory plan, or a host framework whose memory pool must
 * not be bypassed, because cudaMalloc and cudaFree synchronise the device
 * and fragment that pool), and plain C callers that hold their grid buffers
 * but have no device allocator at hand for a workspace.
 *
 * Same arguments and results as gscl_do_reduce without `workspace` /
 * `workspace_bytes`; same launch configuration, hence the same reduction
 * order and bit-identical results.  Its scratch (arrival ticket, result slot
 * and one 16-byte partial per CTA) is a fixed array inside the library of
 * 256 + 16 * GSCL_NOALLOC_MAX_PARTIALS bytes (131,328 bytes), present on
 * every GPU that loads the library until the process exits.  Nothing is
 * allocated by the call (no cudaMalloc, no library allocator).
 *
 *  - Limit: a launch that needs more than GSCL_NOALLOC_MAX_PARTIALS CTAs is
 *    rejected with GSCL_ERR_UNSUPPORTED (gscl_last_error gives the count);
 *    use gscl_do_reduce with a workspace for it.  Launches use one wave of
 *    CTAs (SMs x resident CTAs per SM; at most 4736 on a 148-SM GPU).
 *  - The first call on each device looks up the scratch array's device
 *    address (with that device current) and caches it; make that first call
 *    before any stream capture.
 *  - Every call, on every stream, shares the one array, which keeps the last
 *    call's contents; each call clears the ticket it needs on its stream.
 *    Calls that can overlap on the GPU (different streams, or several host
 *    threads) race on it: keep them on one stream.
 */
#define GSCL_NOALLOC_MAX_PARTIALS 8192
gscl_status gscl_do_reduce_noalloc(int32_t reduce_op, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                                   const gscl_grid *out, int32_t n_out, const gscl_range *range, double *result,
                                   int32_t result_on_host, void *stream);

/*
 * Waits for `stream` and reports device-side failures of the library's
 * kernels enqueued on this device since the last gscl_sync: GSCL_ERR_RANGE if
 * a run-time compiled operator read outside its declared reach (the read
 * returned 0 and touched no memory), GSCL_ERR_TIMEOUT if a bounded wait inside
 * a kernel gave up, GSCL_ERR_CUDA for a CUDA error.  Clears the device-side
 * flag.
 */
gscl_status gscl_sync(void *stream);

/*
 * Self-test of the failure path above (no counterpart in the paper): enqueues
 * one thread that waits, with the library's bounded device-side wait, on a
 * barrier nothing arrives on.  After about 2 s the wait gives up and flags
 * the device error word, so the next gscl_sync returns GSCL_ERR_TIMEOUT; the
 * context stays usable.  Nothing faults, traps or hangs.
 */
gscl_status gscl_selftest_bounded_wait(void *stream);

/*
 * Point operators compiled at run time.  In the paper a stencil operator is a
 * C++ function object compiled with the program (Section 3, Fig. 1b), so any
 * arithmetic can run at a core element; here the operator may also be given
 * as source text, compiled by NVRTC for sm_103a into a do_all kernel.
 *
 * `body` is a block of CUDA C++ statements, run once per core element, that
 *  - reads input a at an offset as in<a>(dx, dy, dz) (in0 .. in<n_in - 1>),
 *    a value of type `real` (double for FP64 grids, float for FP32 and BF16);
 *  - may use the core element's interior index i, j, k (long long), as the
 *    paper's stateful stencils query indices;
 *  - assigns out0 .. out<n_out - 1> (type real, starting at 0), stored at the
 *    core element after the body has run (0 <= n_out <= GSCL_MAX_OUT), and may
 *    assign `value`, which gscl_do_reduce_program reduces;
 *  - may call CUDA's device math functions.  C++ promotion applies: a double
 *    literal makes an FP32 program's expression FP64; write (real) casts or
 *    f-suffixed literals to keep FP32 arithmetic.
 * `reach[3]` bounds |dx|, |dy|, |dz| of every read.  A read beyond it returns
 * 0, touches no memory and makes the next gscl_sync return GSCL_ERR_RANGE.
 *
 * gscl_program_create compiles the body for grids of `dtype` (host-only; no
 * GPU needed): GSCL_ERR_INVALID with the compiler's log in gscl_last_error()
 * if it does not compile, GSCL_ERR_UNSUPPORTED if NVRTC is not installed.
 * gscl_program_destroy releases it (GSCL_ERR_STATE for an unknown handle).
 *
 * gscl_do_all_program runs it as gscl_do_all runs an operator: n_in / n_out
 * and the dtype must be the program's; the range and halo rules apply to the
 * declared reach; an output may also be an input only with reach {0, 0, 0};
 * sweeps > 1 ping-pongs in[0] and out[0] as gscl_do_all does.  The module is
 * loaded on the current device at its first launch there.  Asynchronous on
 * `stream`.
 */
typedef uint64_t gscl_program;
gscl_status gscl_program_create(const char *body, int32_t n_in, int32_t n_out, int32_t dtype, const int32_t reach[3],
                                gscl_program *out);
gscl_status gscl_program_destroy(gscl_program p);
gscl_status gscl_do_all_program(gscl_program p, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                                int32_t n_out, const gscl_range *range, int32_t sweeps, void *stream);

/*
 * do_reduce with a compiled body (Section 3): the body may also assign
 * `value` (type real, starting at 0); its value at every core element of the
 * range is reduced with reduce_op (GSCL_SUM compensated, GSCL_MAXABS, GSCL_L2)
 * in FP64, deterministically, and outputs (n_out may be 0 for a program
 * created with n_out = 0) are written as by gscl_do_all_program: a fused sweep
 * and its residual in one call.  The values go through a stream-ordered FP64
 * array over the range (8 bytes per element, allocated and freed on
 * `stream`).  result, result_on_host, workspace and errors as gscl_do_reduce;
 * an empty range reduces nothing (SUM, MAXABS and L2 give 0).
 */
gscl_status gscl_do_reduce_program(gscl_program p, int32_t reduce_op, const gscl_grid *in, int32_t n_in,
                                   const gscl_grid *out, int32_t n_out, const gscl_range *range, double *result,
                                   int32_t result_on_host, void *workspace, int64_t workspace_bytes, void *stream);

/*
 * FMA throughput of this device in FLOP/s (2 per fused multiply-add) for
 * dtype GSCL_F64 or GSCL_F32: a measurement aid for the ALU roofline of the
 * FP64 sweeps, not an operation of the paper.  Every SM is filled with
 * threads running independent a <- a * b + c chains (8 * iters FMAs per
 * thread); several chain counts and block sizes are timed with CUDA events
 * on `stream` (best of three launches each) and the fastest is reported.
 * Synchronises the stream; GSCL_ERR_DTYPE for other dtypes.
 */
gscl_status gscl_fma_throughput(int32_t dtype, int32_t iters, double *flops_per_s, void *stream);

/* Static English description of a status code. */
const char *gscl_status_str(gscl_status s);

/* Detail of the most recent failing call on this host thread ("" if none). */
const char *gscl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GSCL_H */
