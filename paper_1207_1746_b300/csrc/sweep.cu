// Host side of do_all / do_reduce: validation of the operator against the
// grids (Section 3's rules: reads only at fixed offsets inside the stencil
// shape's halo, writes only at the core element, no order promised),
// launch planning and the C ABI entry points.
#include <atomic>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sweep_host.h"
#include "tb2d_kernel.cuh"

namespace gscl {

bool overlaps(const Grid &a, const Grid &b) { return a.buf < b.buf + b.bytes && b.buf < a.buf + a.bytes; }

// Validates handles, shapes, dtypes, the range, every term and aliasing.
gscl_status bind(const gscl_stencil *op, bool need_value, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                 int32_t n_out, const gscl_range *range, Bound *b, int ordered_axis, int ordered_step,
                 bool colored, bool diamond) {
  if (n_in < 1 || n_in > kMaxIn) return fail(GSCL_ERR_UNSUPPORTED, "n_in = %d outside [1, %d]", n_in, kMaxIn);
  if (n_out < 0 || n_out > kMaxOut_) return fail(GSCL_ERR_UNSUPPORTED, "n_out = %d outside [0, %d]", n_out, kMaxOut_);
  if (!in || (n_out > 0 && !out)) return fail(GSCL_ERR_INVALID, "grid arrays are required");
  b->op = op;
  b->in.resize(n_in);
  b->out.resize(n_out);
  for (int a = 0; a < n_in; ++a) {
    if (gscl_status s = lookup(in[a], &b->in[a])) return s;
    b->in_h.push_back(in[a]);
  }
  for (int m = 0; m < n_out; ++m) {
    if (gscl_status s = lookup(out[m], &b->out[m])) return s;
    b->out_h.push_back(out[m]);
  }
  const Grid &g0 = b->in[0];
  int dev = -1;
  cudaGetDevice(&dev);
  auto check_same = [&](const Grid &g) -> gscl_status {
    if (g.device != dev) return fail(GSCL_ERR_INVALID, "grid lives on device %d, current device is %d", g.device, dev);
    if (g.dtype != g0.dtype) return fail(GSCL_ERR_DTYPE, "grids of one call must share a dtype");
    if (g.ndim != g0.ndim || g.n[0] != g0.n[0] || g.n[1] != g0.n[1] || g.n[2] != g0.n[2])
      return fail(GSCL_ERR_SHAPE, "grids of one call must share ndim and interior extent");
    return GSCL_OK;
  };
  for (auto &g : b->in)
    if (gscl_status s = check_same(g)) return s;
  for (auto &g : b->out)
    if (gscl_status s = check_same(g)) return s;
  for (int a = 0; a < 3; ++a) {
    b->lo[a] = range ? range->lo[a] : 0;
    b->hi[a] = range ? range->hi[a] : g0.n[a];
    if (b->lo[a] < 0 || b->hi[a] > g0.n[a] || b->lo[a] > b->hi[a])
      return fail(GSCL_ERR_RANGE, "range [%lld, %lld) on axis %d outside the interior [0, %lld)", (long long)b->lo[a],
                  (long long)b->hi[a], a, (long long)g0.n[a]);
    if (b->lo[a] == b->hi[a]) b->empty = true;
  }
  for (int m = 0; m < n_out; ++m)
    for (int m2 = 0; m2 < m; ++m2)
      if (overlaps(b->out[m], b->out[m2])) return fail(GSCL_ERR_ALIAS, "outputs %d and %d share storage", m2, m);
  if (!op) {
    if (!need_value) return fail(GSCL_ERR_INVALID, "do_all needs an operator");
    if (n_out != 0) return fail(GSCL_ERR_INVALID, "reducing in[0] itself writes no output");
    return GSCL_OK;
  }
  if (op->reserved != 0) return fail(GSCL_ERR_INVALID, "stencil reserved field must be 0");
  if (op->n_terms < 1 || op->n_terms > kMaxTerms)
    return fail(GSCL_ERR_UNSUPPORTED, "n_terms = %d outside [1, %d]", op->n_terms, kMaxTerms);
  if (!op->terms) return fail(GSCL_ERR_INVALID, "terms is NULL");
  bool has_value = false;
  for (int t = 0; t < op->n_terms; ++t) {
    const gscl_term &tm = op->terms[t];
    if (tm.reserved != 0) return fail(GSCL_ERR_INVALID, "term %d: reserved field must be 0", t);
    if (tm.out != GSCL_VALUE && tm.out >= n_out)
      return fail(GSCL_ERR_INVALID, "term %d writes output %d of %d", t, tm.out, n_out);
    if (tm.out == GSCL_VALUE) has_value = true;
    if (tm.coef != GSCL_NONE && tm.coef >= n_in)
      return fail(GSCL_ERR_INVALID, "term %d: coefficient grid %d of %d", t, tm.coef, n_in);
    if (tm.in == GSCL_VALUE) {
      if (tm.dx || tm.dy || tm.dz) return fail(GSCL_ERR_INVALID, "term %d reads the value at a non-zero offset", t);
      if (tm.out == GSCL_VALUE) return fail(GSCL_ERR_INVALID, "term %d: the value cannot feed itself", t);
      continue;
    }
    if (tm.in >= n_in) return fail(GSCL_ERR_INVALID, "term %d reads input %d of %d", t, tm.in, n_in);
    const Grid &g = b->in[tm.in];
    const int d[3] = {tm.dx, tm.dy, tm.dz};
    for (int a = 0; a < 3; ++a) {
      if (abs(d[a]) > GSCL_MAX_HALO) return fail(GSCL_ERR_RANGE, "term %d: offset %d beyond the maximum halo", t, d[a]);
      if (b->empty) continue;
      if (b->lo[a] + d[a] < -(int64_t)g.halo[a] || b->hi[a] - 1 + d[a] > g.n[a] - 1 + g.halo[a])
        return fail(GSCL_ERR_RANGE, "term %d reads input %d at offset %d on axis %d, outside its halo %d", t, tm.in,
                    d[a], a, g.halo[a]);
    }
  }
  if (need_value && !has_value) return fail(GSCL_ERR_INVALID, "do_reduce needs a term with out == GSCL_VALUE");
  // an output may also be an input only if every read of it is at offset 0
  // (ordered iteration spaces: or at the element visited just before;
  // red-black colouring: or at an offset with odd dx + dy + dz, an element of
  // the other colour, which the call does not write)
  for (int m = 0; m < n_out; ++m)
    for (int a = 0; a < n_in; ++a) {
      if (!overlaps(b->out[m], b->in[a])) continue;
      const Grid &go = b->out[m], &gi = b->in[a];
      if ((ordered_axis >= 0 || colored || diamond) &&
          (go.buf != gi.buf || go.off != gi.off || go.pitch != gi.pitch || go.plane != gi.plane))
        return fail(GSCL_ERR_ALIAS, "output %d overlaps input %d without being the same grid", m, a);
      for (int t = 0; t < op->n_terms; ++t) {
        const gscl_term &tm = op->terms[t];
        if (tm.in != a || !(tm.dx || tm.dy || tm.dz)) continue;
        const int d[3] = {tm.dx, tm.dy, tm.dz};
        const bool previous = ordered_axis >= 0 && d[ordered_axis] == ordered_step &&
                              d[(ordered_axis + 1) % 3] == 0 && d[(ordered_axis + 2) % 3] == 0;
        const bool other_colour = colored && ((d[0] + d[1] + d[2]) & 1);
        const bool one_sign = diamond && d[2] == 0 && ((d[0] <= 0 && d[1] <= 0) || (d[0] >= 0 && d[1] >= 0));
        if (!previous && !other_colour && !one_sign)
          return fail(GSCL_ERR_ALIAS, "output %d is input %d, read at a non-zero offset by term %d", m, a, t);
      }
    }
  return GSCL_OK;
}

// ---------------------------------------------------------------- matching
struct StaticDesc {
  int id;
  int nin, nout, nt;
  const OpTerm *t;
};

template <class Def>
StaticDesc desc_of(int id) {
  return StaticDesc{id, Def::NIN, Def::NOUT, Def::NT, Def::table.t};
}

const std::vector<StaticDesc> &static_ops() {
  static const std::vector<StaticDesc> ops = {
      desc_of<OpHeat7Rhs>(OP_HEAT7_RHS),         desc_of<OpStar7>(OP_STAR7),
      desc_of<OpJacobi7Rhs>(OP_JACOBI7_RHS),     desc_of<OpJacobi5_2D>(OP_JACOBI5_2D),
      desc_of<OpClimate>(OP_CLIMATE),            desc_of<OpHeat7RhsFused>(OP_HEAT7_RHS_FUSED),
      desc_of<OpHeat7Fused>(OP_HEAT7_FUSED),     desc_of<OpResidual7Rhs>(OP_RESIDUAL7_RHS),
      desc_of<OpDifference>(OP_DIFFERENCE),      desc_of<OpIdentity>(OP_IDENTITY)};
  return ops;
}

OpTerm key_of(const gscl_term &t) {
  return OpTerm{t.dx, t.dy, t.dz, t.in == GSCL_VALUE ? -1 : (int)t.in, t.coef == GSCL_NONE ? -1 : (int)t.coef,
                t.out == GSCL_VALUE ? -1 : (int)t.out};
}

bool same_key(const OpTerm &a, const OpTerm &b) {
  return a.dx == b.dx && a.dy == b.dy && a.dz == b.dz && a.in == b.in && a.coef == b.coef && a.out == b.out;
}

// Finds a compile-time operator with the descriptor's structure; on success
// perm[i] is the descriptor term that supplies table term i's weight.
int match_static(const std::vector<gscl_term> &terms, int n_in, int n_out, std::vector<int> *perm) {
  const char *env = getenv("GSCL_GENERIC_ONLY");
  if (env && env[0] && env[0] != '0') return OP_GENERIC;
  for (const StaticDesc &d : static_ops()) {
    if (d.nin != n_in || d.nout != n_out || d.nt != (int)terms.size()) continue;
    std::vector<bool> used(terms.size(), false);
    perm->assign(d.nt, -1);
    bool ok = true;
    for (int i = 0; i < d.nt && ok; ++i) {
      ok = false;
      for (size_t j = 0; j < terms.size(); ++j) {
        if (!used[j] && same_key(d.t[i], key_of(terms[j]))) {
          used[j] = true;
          (*perm)[i] = (int)j;
          ok = true;
          break;
        }
      }
    }
    if (ok) return d.id;
  }
  return OP_GENERIC;
}

// Columns (TX = 32 VX) and rows per thread, as the kernels are instantiated.
int vx_for(int dtype) { return dtype == GSCL_F64 ? VxOf<double>::value : VxOf<float>::value; }
int vy_for(int dtype) { return dtype == GSCL_F64 ? VyOf<double>::value : VyOf<float>::value; }

gscl_status make_plan(const Bound &b, bool reduce, Plan *pl, TileCfg cfg) {
  SweepParams &P = pl->P;
  memset(&P, 0, sizeof P);
  P.within = -1.0;  // MAXABS reports the maximum (gscl_do_reduce_within sets a tolerance)
  P.color = -1;     // every element (gscl_do_colored sets a colour)
  const Grid &g0 = b.in[0];
  const int n_in = (int)b.in.size(), n_out = (int)b.out.size();
  const int elem = g0.elem;
  std::vector<gscl_term> terms;
  if (b.op) {
    terms.assign(b.op->terms, b.op->terms + b.op->n_terms);
  } else {
    gscl_term id = {0, 0, 0, 0, GSCL_NONE, GSCL_VALUE, 0, 1.0};
    terms.push_back(id);
  }
  std::vector<int> perm;
  pl->op = cfg.generic ? OP_GENERIC : match_static(terms, n_in, n_out, &perm);
  // narrow tiles: compiled for batches of compile-time operators, FP32 / BF16
  const bool narrow = cfg.narrow && g0.dtype != GSCL_F64 && batch_capable(pl->op);
  // colour-compacted red-black sweeps: a warp spans 64 VX columns
  const bool compact = cfg.compact && g0.dtype == GSCL_F64 && !cfg.generic && compact_capable(pl->op) && !reduce;
  // reach per input grid (coefficient reads are at the core element)
  int rxa[kMaxIn] = {}, rya[kMaxIn] = {}, rz = 0, rx_max = 0;
  for (auto &t : terms) {
    if (t.in == GSCL_VALUE) continue;
    rxa[t.in] = std::max(rxa[t.in], abs((int)t.dx));
    rya[t.in] = std::max(rya[t.in], abs((int)t.dy));
    rz = std::max(rz, abs((int)t.dz));
    rx_max = std::max(rx_max, abs((int)t.dx));
  }
  // vector lanes (StaticOpV): compile-time operators on FP32 / BF16 grids,
  // G = 16 / element bytes contiguous columns per lane, 128-column tiles
  // whose rows take 128 / G lanes (RPS row blocks per warp)
  const int G = 16 / elem;
  const bool vlanes = !narrow && pl->op != OP_GENERIC && (g0.dtype == GSCL_F32 || g0.dtype == GSCL_BF16) &&
                      rx_max <= G;
  const int VX = narrow ? 2 : (vlanes ? G : vx_for(g0.dtype));
  const int TX = vlanes ? 128 : (compact ? 64 : 32) * VX;
  const int RPS = vlanes ? 32 * G / 128 : 1;
  const int vec = 16 / elem;  // TMA x coordinates stay multiples of 16 bytes
  int AXa[kMaxIn], BWa[kMaxIn];
  for (int a = 0; a < n_in; ++a) {
    AXa[a] = (rxa[a] + vec - 1) / vec * vec;
    BWa[a] = TX + 2 * AXa[a];
  }
  const int nz_range = (int)(b.hi[2] - b.lo[2]);
  const int smem_cap = max_smem_per_block();
  // FP64 grids: the arithmetic is fixed here, with the plan
  pl->pair = g0.dtype == GSCL_F64 && fp64_arith() == GSCL_FP64_PAIR;
  // inputs read only at the core element go to the two-slot centre ring
  // (IEEE FP64: only for operators with kCentreFp64Min or more such inputs;
  // the kernel's operator tables make the same choice; the colour-compacted
  // kernel reads every input from the plane ring)
  const uint32_t smask = static_centre_mask(pl->op);
  const bool ieee64 = g0.dtype == GSCL_F64 && !pl->pair;
  // IEEE FP64 compile-time operators whose term groups have equal (pairs:
  // opposite) weights: the group evaluation with some additions on the
  // integer pipe (static_ops.h; a batch records this per instance)
  pl->eqw = false;
  if (ieee64 && pl->op != OP_GENERIC && fp64_int_add()) {
    double wt[kMaxTerms];
    for (size_t i = 0; i < perm.size() && i < (size_t)kMaxTerms; ++i) wt[i] = terms[perm[i]].w;
    pl->eqw = static_group_weights_ok(pl->op, wt);
  }
  const uint32_t cmask =
      (compact || (ieee64 && __builtin_popcount(smask) < kCentreFp64Min)) ? 0u : smask;
  auto centre = [&](int a) { return ((cmask >> a) & 1u) != 0; };
  // warps per CTA (each warp owns VY rows of the tile) and planes prefetched
  const int VY = narrow ? 4 : vy_for(g0.dtype);
  // defaults from tile sweeps on the 256^3 heat workload (B300): FP64 4 warps,
  // FP32 / BF16 8 warps, one plane prefetched beyond the stencil's reach
  int NW = g0.dtype == GSCL_F64 ? 4 : 8, PF = nz_range > 1 ? 1 : 0;
  if (const char *e = getenv("GSCL_TILE_WARPS")) NW = std::max(1, std::min(8, atoi(e)));
  if (const char *e = getenv("GSCL_PREFETCH")) PF = nz_range > 1 ? std::max(1, std::min(6, atoi(e))) : 0;
  if (cfg.nw > 0) NW = std::min(8, cfg.nw);
  if (cfg.pf > 0 && nz_range > 1) PF = std::min(6, cfg.pf);
  int TY = NW * VY * RPS;
  size_t smem = 0;
  int R = 0, SEa[kMaxIn] = {}, BHa[kMaxIn] = {};
  for (;;) {
    TY = NW * VY * RPS;
    R = 2 * rz + 1 + PF;
    size_t ring = 0;
    for (int a = 0; a < n_in; ++a) {
      BHa[a] = TY + 2 * rya[a];
      SEa[a] = (BWa[a] * BHa[a] * elem + 127) / 128 * 128 / elem;
      ring += (size_t)(centre(a) ? 2 : R) * SEa[a] * elem;
    }
    smem = kBarBytes + ring;
    if (smem <= (size_t)smem_cap && R <= kMaxRing) {
      // IEEE FP64 sweeps (bound by the FP64 pipe's latency at low occupancy):
      // give up the prefetched plane when that lets a second CTA reside
      if (ieee64 && PF > 0 && !getenv("GSCL_PREFETCH") && cfg.pf <= 0) {
        const size_t per_sm = (size_t)smem_per_sm(), reserve = 1024;
        size_t fewer = kBarBytes;
        for (int a = 0; a < n_in; ++a) fewer += (size_t)(centre(a) ? 2 : R - 1) * SEa[a] * elem;
        if (per_sm / (smem + reserve) < 2 && per_sm / (fewer + reserve) >= 2) {
          --PF;
          continue;
        }
      }
      break;
    }
    if (PF > 1) --PF;
    else if (NW > 1) NW /= 2;
    else return fail(GSCL_ERR_UNSUPPORTED, "operator needs %zu bytes of shared memory per CTA", smem);
  }
  for (int a = 0; a < n_in; ++a)
    if (BWa[a] > 256 || BHa[a] > 256) return fail(GSCL_ERR_UNSUPPORTED, "tile box too large for TMA");
  int nt = 0;
  auto push = [&](const gscl_term &t) {
    DevTerm &d = P.terms[nt++];
    d.in = t.in == GSCL_VALUE ? -1 : (int16_t)t.in;
    d.coef = t.coef == GSCL_NONE ? -1 : (int16_t)t.coef;
    d.dz = t.dz;
    d.toff = t.in == GSCL_VALUE ? 0 : (rya[t.in] + t.dy) * BWa[t.in] + AXa[t.in] + t.dx;
    d.wf = (float)t.w;
    d.wd = t.w;
    d.wl = (float)(t.w - (double)d.wf);
  };
  if (pl->op != OP_GENERIC) {
    // table order (value terms first); the kernel reads only the weights
    for (int i : perm) push(terms[i]);
    for (int i = 0; i < (int)perm.size(); ++i)
      if (terms[perm[i]].out == GSCL_VALUE) P.n_value_terms = i + 1;
    for (int m = 0; m <= n_out; ++m) P.out_begin[m] = nt;
  } else {
    for (auto &t : terms)
      if (t.out == GSCL_VALUE) push(t);
    P.n_value_terms = nt;
    for (int m = 0; m < n_out; ++m) {
      P.out_begin[m] = nt;
      for (auto &t : terms)
        if (t.out == m) push(t);
    }
    P.out_begin[n_out] = nt;
  }
  P.n_in = n_in;
  P.n_out = n_out;
  for (int m = 0; m < n_out; ++m) {
    const Grid &g = b.out[m];
    P.inst.out[m].base = g.elem_ptr(0, 0, 0);
    P.inst.out[m].pitch = g.pitch;
    P.inst.out[m].plane = g.plane;
  }
  for (int a = 0; a < n_in; ++a) {
    const Grid &g = b.in[a];
    if (gscl_status s = encode_tensor_map_3d(&P.inst.tmap[a], g, (uint32_t)BWa[a], (uint32_t)BHa[a])) return s;
    P.inst.in[a].base = g.elem_ptr(0, 0, 0);
    P.inst.in[a].pitch = g.pitch;
    P.inst.in[a].plane = g.plane;
    P.inst.cx_add[a] = (int32_t)(g.halo[0] + g.off);
    P.inst.cy_add[a] = g.halo[1];
    P.inst.cz_add[a] = g.halo[2];
  }
  for (int a = 0; a < 3; ++a) {
    P.inst.lo[a] = b.lo[a];
    P.inst.hi[a] = b.hi[a];
  }
  P.inst.x_base = b.lo[0] / TX * TX;
  P.inst.y_base = b.lo[1];
  P.inst.tiles_x = (int32_t)((b.hi[0] - P.inst.x_base + TX - 1) / TX);
  P.inst.tiles_y = (int32_t)((b.hi[1] - b.lo[1] + TY - 1) / TY);
  const int threads = 32 * NW;
  P.R = R;
  P.rz = rz;
  uint32_t tx = 0, ctx = 0;
  int base = 0;
  for (int a = 0; a < n_in; ++a) {
    P.in_bw[a] = BWa[a];
    P.in_bh[a] = BHa[a];
    P.in_ax[a] = AXa[a];
    P.in_ry[a] = rya[a];
    P.in_se[a] = SEa[a];
    P.in_base[a] = base;
    base += (centre(a) ? 2 : R) * SEa[a];
    if (centre(a)) ctx += (uint32_t)(BWa[a] * BHa[a] * elem);
    else tx += (uint32_t)(BWa[a] * BHa[a] * elem);
  }
  P.tx_bytes = tx;
  P.cmask = cmask;
  P.ctx_bytes = ctx;
  // Column-aligned launches (one z range of one tile column per CTA) let L2
  // serve the halo rows that neighbouring tiles share; they pay off where the
  // sweep is bound by HBM (FP32 / BF16 sweeps and reductions, whose squares
  // are summed on the FP32 pipe).  FP64 sweeps and reductions are bound by
  // the FP64 pipe and keep the even split over every resident CTA slot.
  P.zalt = g0.dtype == GSCL_F64 ? 0 : 1;
  if (const char *e = getenv("GSCL_ZALT")) P.zalt = atoi(e) != 0;
  P.err = device_error_word();
  if (!P.err) return fail(GSCL_ERR_CUDA, "device error word unavailable");
  pl->threads = threads;
  pl->smem = smem;
  pl->narrow = narrow;
  pl->compact = compact;
  pl->vec = vlanes;
  pl->tile_x = TX;
  pl->tile_y = TY;
  pl->work = (long long)P.inst.tiles_x * P.inst.tiles_y * nz_range;
  pl->max_ctas = reduce ? kMaxReduceCtas : 0x7fffffff;
  return GSCL_OK;
}

namespace {

template <typename T, int VX, bool BATCH>
gscl_status launch_generic_b(const Plan &pl, int red, cudaStream_t stream, int *occ) {
  switch (red) {
    case RED_NONE: return launch_t<T, VX, RED_NONE, GenericOp, BATCH>(pl, stream, occ);
    case RED_SUM: return launch_t<T, VX, RED_SUM, GenericOp, BATCH>(pl, stream, occ);
    case RED_MAXABS: return launch_t<T, VX, RED_MAXABS, GenericOp, BATCH>(pl, stream, occ);
    case RED_L2: return launch_t<T, VX, RED_L2, GenericOp, BATCH>(pl, stream, occ);
  }
  return fail(GSCL_ERR_INVALID, "unknown reduction");
}

template <typename T>
gscl_status launch_generic(const Plan &pl, int red, cudaStream_t stream, int *occ) {
  constexpr int VX = VxOf<T>::value;
  return pl.batch ? launch_generic_b<T, VX, true>(pl, red, stream, occ)
                  : launch_generic_b<T, VX, false>(pl, red, stream, occ);
}

}  // namespace

// Arithmetic of FP64 grids: IEEE FP64 (default) or pairs of FP32 numbers.
std::atomic<int> g_fp64_arith{-1};

// The axial-sum evaluation of IEEE FP64 sweeps (GSCL_FP64_INT_ADD=0 turns
// it off: every term then takes its own FMA in table order).
bool fp64_int_add() {
  const char *e = getenv("GSCL_FP64_INT_ADD");
  return !(e && e[0] == '0');
}

int fp64_arith() {
  int m = g_fp64_arith.load();
  if (m < 0) {  // first use: GSCL_FP64_ARITH=pair selects the pair arithmetic
    const char *e = getenv("GSCL_FP64_ARITH");
    m = (e && strcmp(e, "pair") == 0) ? GSCL_FP64_PAIR : GSCL_FP64_IEEE;
    int expect = -1;
    g_fp64_arith.compare_exchange_strong(expect, m);
    m = g_fp64_arith.load();
  }
  return m;
}

// Launches (or, with occupancy_only, sizes) the kernel a plan names.
gscl_status launch(const Plan &pl, int dtype, int red, cudaStream_t stream, int *occupancy_only) {
  const bool pair = dtype == GSCL_F64 && pl.pair;
  if (pl.op != OP_GENERIC) {
    switch (dtype) {
      case GSCL_F64:
        return pair ? launch_static_f64pair(pl, red, stream, occupancy_only)
                    : launch_static_f64(pl, red, stream, occupancy_only);
      case GSCL_F32: return launch_static_f32(pl, red, stream, occupancy_only);
      case GSCL_BF16: return launch_static_bf16(pl, red, stream, occupancy_only);
    }
    return fail(GSCL_ERR_DTYPE, "unknown dtype");
  }
  switch (dtype) {
    case GSCL_F64:
      return pair ? launch_generic<f64pair>(pl, red, stream, occupancy_only)
                  : launch_generic<double>(pl, red, stream, occupancy_only);
    case GSCL_F32: return launch_generic<float>(pl, red, stream, occupancy_only);
    case GSCL_BF16: return launch_generic<__nv_bfloat16>(pl, red, stream, occupancy_only);
  }
  return fail(GSCL_ERR_DTYPE, "unknown dtype");
}

}  // namespace gscl

using namespace gscl;

extern "C" {

int64_t gscl_reduce_workspace_bytes(void) { return kWorkspaceBytes; }

gscl_status gscl_set_fp64_arithmetic(int32_t mode) {
  if (mode != GSCL_FP64_IEEE && mode != GSCL_FP64_PAIR) return fail(GSCL_ERR_INVALID, "unknown FP64 arithmetic %d", mode);
  g_fp64_arith.store(mode);
  return GSCL_OK;
}

int32_t gscl_get_fp64_arithmetic(void) { return fp64_arith(); }

int32_t gscl_stencil_specialization(const gscl_stencil *op, int32_t n_in, int32_t n_out) {
  if (!op || !op->terms || op->n_terms < 1 || op->n_terms > kMaxTerms) return OP_GENERIC;
  std::vector<gscl_term> terms(op->terms, op->terms + op->n_terms);
  std::vector<int> perm;
  return match_static(terms, n_in, n_out, &perm);
}

gscl_status gscl_do_all(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                        int32_t n_out, const gscl_range *range, int32_t sweeps, void *stream) {
  if (sweeps < 1) return fail(GSCL_ERR_INVALID, "sweeps must be >= 1");
  if (n_out < 1) return fail(GSCL_ERR_INVALID, "do_all needs at least one output");
  Bound b;
  if (gscl_status s = bind(op, false, in, n_in, out, n_out, range, &b)) return s;
  if (b.empty) return GSCL_OK;
  if (sweeps > 1) {
    const Grid &a = b.in[0], &c = b.out[0];
    if (a.halo[0] != c.halo[0] || a.halo[1] != c.halo[1] || a.halo[2] != c.halo[2])
      return fail(GSCL_ERR_SHAPE, "multi-sweep ping-pong needs in[0] and out[0] of identical layout");
    if (overlaps(a, c)) return fail(GSCL_ERR_ALIAS, "multi-sweep ping-pong needs distinct in[0] and out[0]");
  }
  Grid src = b.in[0], dst = b.out[0];
  TbChoice tc;
  int sop = OP_GENERIC;
  if (sweeps > 1) {
    std::vector<gscl_term> terms(op->terms, op->terms + op->n_terms);
    std::vector<int> perm;
    sop = match_static(terms, n_in, n_out, &perm);
    tc = tb_choice(b, sop, sweeps);
  }
  // fused passes of up to K sweeps (bit-identical to K single sweeps), the
  // last launch a single sweep and the launch count of the parity of the
  // sweep count (tb_launch_plan), so both handles end as after single sweeps
  const std::vector<int> plan = tb_launch_plan(sweeps, tc.K);
  int launches = 0, done = 0;
  for (int k : plan) {
    b.in[0] = src;
    b.out[0] = dst;
    for (size_t a = 1; a < b.in.size(); ++a)  // another input naming the ping-pong grid follows it
      if (b.in_h[a] == b.in_h[0]) b.in[a] = src;
    Plan pl;
    if (k > 1) {
      TbChoice c = tc;
      c.K = k;
      // the input iterate `done` sits in the other grid than single sweeps put it in
      const bool halo_swap = ((done - launches) & 1) != 0;
      if (gscl_status st = run_tb_pass(b, sop, c, halo_swap, (cudaStream_t)stream)) return st;
    } else {
      if (gscl_status st = make_plan(b, false, &pl, TileCfg{})) return st;
      if (gscl_status st = launch(pl, b.in[0].dtype, RED_NONE, (cudaStream_t)stream, nullptr)) return st;
    }
    done += k;
    ++launches;
    std::swap(src, dst);
  }
  // an even number of launches leaves the result in in[0]'s storage: exchange
  // the handles so out[0] names it
  if (launches > 1 && launches % 2 == 0) return swap_storage(in[0], out[0]);
  return GSCL_OK;
}

// Colour-compacted red-black sweeps where they exist (GSCL_COLOR_COMPACT=0
// turns them off: every element evaluated, the colour's stored).
static bool colour_compact() {
  const char *e = getenv("GSCL_COLOR_COMPACT");
  return !(e && e[0] == '0');
}

gscl_status gscl_do_colored(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                            int32_t n_out, const gscl_range *range, int32_t color, int32_t half_sweeps,
                            void *stream) {
  if (color != 0 && color != 1) return fail(GSCL_ERR_INVALID, "color must be 0 or 1, got %d", color);
  if (half_sweeps < 1) return fail(GSCL_ERR_INVALID, "half_sweeps must be >= 1");
  if (n_out < 1) return fail(GSCL_ERR_INVALID, "do_colored needs at least one output");
  Bound b;
  if (gscl_status s = bind(op, false, in, n_in, out, n_out, range, &b, -1, 0, true)) return s;
  if (b.empty) return GSCL_OK;
  Plan pl;
  TileCfg cfg;
  cfg.compact = colour_compact();
  if (gscl_status s = make_plan(b, false, &pl, cfg)) return s;
  for (int h = 0; h < half_sweeps; ++h) {
    pl.P.color = (color + h) & 1;
    if (gscl_status s = launch(pl, b.in[0].dtype, RED_NONE, (cudaStream_t)stream, nullptr)) return s;
  }
  return GSCL_OK;
}

gscl_status gscl_tune_sweeps(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                             int32_t n_out, int32_t trial_sweeps, void *stream, int32_t *best_factor) {
  if (!best_factor) return fail(GSCL_ERR_INVALID, "best_factor is required");
  if (trial_sweeps < 1) return fail(GSCL_ERR_INVALID, "trial_sweeps must be >= 1");
  Bound b;
  if (gscl_status s = bind(op, false, in, n_in, out, n_out, nullptr, &b)) return s;
  if (n_out < 1 || b.empty) return fail(GSCL_ERR_INVALID, "tuning needs an output and a non-empty interior");
  std::vector<gscl_term> terms(op->terms, op->terms + op->n_terms);
  std::vector<int> perm;
  int best = 1;
  gscl_status s = tune_sweeps(b, match_static(terms, n_in, n_out, &perm), trial_sweeps, (cudaStream_t)stream, &best);
  *best_factor = best;
  return s;
}

}  // extern "C"

namespace gscl {
namespace {

// do_reduce with `red`; within >= 0 turns MAXABS into the all-within test.
gscl_status reduce_call(int red, double within, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                        const gscl_grid *out, int32_t n_out, const gscl_range *range, double *result,
                        int32_t result_on_host, void *workspace, int64_t workspace_bytes, void *stream) {
  if (!result) return fail(GSCL_ERR_INVALID, "result is NULL");
  if (!workspace) return fail(GSCL_ERR_INVALID, "workspace is NULL");
  if (((uintptr_t)workspace) % 16) return fail(GSCL_ERR_INVALID, "workspace must be 16-byte aligned");
  if (workspace_bytes < kWorkspaceBytes)
    return fail(GSCL_ERR_OOM, "workspace has %lld bytes, needs %lld", (long long)workspace_bytes,
                (long long)kWorkspaceBytes);
  Bound b;
  if (gscl_status s = bind(op, true, in, n_in, out, n_out, range, &b)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  double *dev_result = result_on_host ? reinterpret_cast<double *>((char *)workspace + 8) : result;
  if (b.empty) {
    // an empty range: 0 for the sums and the maximum, "all within" for the test
    if (within >= 0.0) {
      static const double one = 1.0;
      cudaError_t e = cudaMemcpyAsync(dev_result, &one, sizeof(double), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `one` is pageable host memory
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    } else {
      cudaError_t e = cudaMemsetAsync(dev_result, 0, sizeof(double), st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
  } else {
    Plan pl;
    if (gscl_status s = make_plan(b, true, &pl, TileCfg{})) return s;
    // the arrival ticket starts at zero whatever an earlier call left: a CTA
    // whose bounded wait gave up returns without taking its ticket
    cudaError_t e = cudaMemsetAsync(workspace, 0, 256, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    pl.P.workspace = (unsigned char *)workspace;
    pl.P.result = dev_result;
    pl.P.within = within;
    if (gscl_status s = launch(pl, b.in[0].dtype, red, st, nullptr)) return s;
  }
  if (result_on_host) {
    cudaError_t e = cudaMemcpyAsync(result, dev_result, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    // a wait that gave up leaves a partial result: report it with the value
    return take_device_error();
  }
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

extern "C" {

gscl_status gscl_do_reduce(int32_t reduce_op, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                           const gscl_grid *out, int32_t n_out, const gscl_range *range, double *result,
                           int32_t result_on_host, void *workspace, int64_t workspace_bytes, void *stream) {
  int red;
  switch (reduce_op) {
    case GSCL_SUM: red = RED_SUM; break;
    case GSCL_MAXABS: red = RED_MAXABS; break;
    case GSCL_L2: red = RED_L2; break;
    default: return fail(GSCL_ERR_INVALID, "unknown reduce op %d", reduce_op);
  }
  return reduce_call(red, -1.0, op, in, n_in, out, n_out, range, result, result_on_host, workspace,
                     workspace_bytes, stream);
}

gscl_status gscl_do_reduce_within(const gscl_stencil *op, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                                  int32_t n_out, const gscl_range *range, double eps, double *result,
                                  int32_t result_on_host, void *workspace, int64_t workspace_bytes, void *stream) {
  if (!(eps >= 0.0)) return fail(GSCL_ERR_INVALID, "eps must be >= 0");
  return reduce_call(RED_MAXABS, eps, op, in, n_in, out, n_out, range, result, result_on_host, workspace,
                     workspace_bytes, stream);
}

}  // extern "C"

// ===================================================================== no-alloc reduce
// A do_reduce for callers that cannot hand the library a workspace.  Its
// scratch (the arrival ticket, the result slot and one partial sum per CTA)
// lives in the fixed array below instead of caller memory.
namespace gscl {
namespace {

constexpr int kNoAllocMaxCtas = GSCL_NOALLOC_MAX_PARTIALS;
constexpr int64_t kNoAllocScratchBytes = 256 + 16LL * kNoAllocMaxCtas;
constexpr int kMaxDevices = 64;

// One copy per device that loads the library, zero at load, held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol's
// name in host code is only a handle for the runtime, so the address is
// asked for once per device, with that device current, and cached.
gscl_status noalloc_scratch(unsigned char **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(GSCL_ERR_UNSUPPORTED, "device %d beyond the supported count", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the built-in reduce scratch");
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char *)g_noalloc_ptr[dev];
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

extern "C" gscl_status gscl_do_reduce_noalloc(int32_t reduce_op, const gscl_stencil *op, const gscl_grid *in,
                                              int32_t n_in, const gscl_grid *out, int32_t n_out,
                                              const gscl_range *range, double *result, int32_t result_on_host,
                                              void *stream) {
  int red;
  switch (reduce_op) {
    case GSCL_SUM: red = RED_SUM; break;
    case GSCL_MAXABS: red = RED_MAXABS; break;
    case GSCL_L2: red = RED_L2; break;
    default: return fail(GSCL_ERR_INVALID, "unknown reduce op %d", reduce_op);
  }
  if (!result) return fail(GSCL_ERR_INVALID, "result is NULL");
  Bound b;
  if (gscl_status s = bind(op, true, in, n_in, out, n_out, range, &b)) return s;
  unsigned char *scratch = nullptr;
  if (gscl_status s = noalloc_scratch(&scratch)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  double *dev_result = result_on_host ? reinterpret_cast<double *>(scratch + 8) : result;
  if (b.empty) {
    cudaError_t e = cudaMemsetAsync(dev_result, 0, sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  } else {
    Plan pl;
    if (gscl_status s = make_plan(b, true, &pl, TileCfg{})) return s;
    pl.max_ctas = kNoAllocMaxCtas;  // launch rejects a grid whose partials would not fit
    // the arrival ticket must start at zero whatever an earlier call left
    cudaError_t e = cudaMemsetAsync(scratch, 0, 256, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    pl.P.workspace = scratch;
    pl.P.result = dev_result;
    if (gscl_status s = launch(pl, b.in[0].dtype, red, st, nullptr)) return s;
  }
  if (result_on_host) {
    cudaError_t e = cudaMemcpyAsync(result, dev_result, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return take_device_error();
  }
  return GSCL_OK;
}
