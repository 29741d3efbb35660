// Batched sweeps: many independent grid sets (instances) of one operator,
// each sweep of all of them in one launch of the sweep kernel, whose CTAs
// walk a host-built work-list of (instance, tile column, z run) segments
// that splits the total (tile, plane) work evenly over one wave of CTAs.
// Repeated sweeps alternate two device tables of instance descriptors
// (in[0] -> out[0] and back), so a whole sweep group can be captured once in
// a CUDA graph and replayed.  Per-instance reductions write one partial per
// segment and a second kernel folds each instance's segments in order.
// Coloured batches (red-black sweeps, Section 3's stateful stencils) update
// their instances in place, one colour per launch, and take one operator per
// instance: the same term structure with the instance's own weights, which
// the kernel reads from a per-instance weight table.  Batches of 2D grids
// under a 5-point operator may fuse K sweeps per launch (tb2d_kernel.cuh):
// their launches then walk a list of (instance, tile) pairs.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "sweep_host.h"
#include "tb2_kernel.cuh"
#include "tb2d_kernel.cuh"

namespace gscl {
namespace {

struct Batch {
  int n_inst = 0, n_in = 0, n_out = 0, dtype = 0;
  std::vector<gscl_term> terms;
  gscl_stencil st{};
  bool colored = false;                           // red-black batch: in place, one operator per instance
  std::vector<std::vector<gscl_term>> inst_terms;  // coloured batches: instance i's operator
  std::vector<gscl_stencil> inst_st;
  std::vector<gscl_grid> in_h, out_h;
  bool has_value = false;
  TileCfg cfg;
  // state built for the current buffers
  bool built = false;
  std::vector<char *> buf_a, buf_b;  // in[0] / out[0] storage when built (table 0 reads a, writes b)
  Plan base;
  int G = 0, S = 0;
  char *dev = nullptr;
  size_t dev_bytes = 0;
  InstDesc *tab[2] = {nullptr, nullptr};
  Segment *segs = nullptr;
  int32_t *cta_seg = nullptr, *inst_seg = nullptr;
  double *partials = nullptr;
  InstWeights *wtab = nullptr;  // one weight row per instance
  // temporal blocking of 2D batches: whether every instance qualifies, the
  // sweeps fused per launch (1: none), the tile shape and its tile list
  bool tb_ok = false;
  int tb_k = 1, tb_tile = 0;
  int4 *tb_tiles = nullptr;
  int tb_n = 0, tb_cap = 0;
  std::vector<int64_t> nx, ny;  // instance extents (tile lists)
  // 3D batches of the radius-1 star operators (FP32 / BF16): two-sweep
  // passes (tb2_kernel.cuh) from their own descriptor tables (the pass's
  // boxes) and work-list
  bool tb3_ok = false;
  Plan tb3_base;
  char *tb3_dev = nullptr;
  size_t tb3_bytes = 0;
  InstDesc *tb3_tab[2] = {nullptr, nullptr};
  Segment *tb3_segs = nullptr;
  int32_t *tb3_cta = nullptr;
  int tb3_G = 0;
  // (first table, sweeps) or, for coloured batches, (2 + first colour, half-sweeps)
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  cudaStream_t cap_stream = nullptr;
  std::mutex mu;
};

std::mutex g_batch_mu;
std::map<uint64_t, std::unique_ptr<Batch>> g_batches;
uint64_t g_next_batch = 1;

Batch *find_batch(gscl_batch h) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  auto it = g_batches.find(h);
  return it == g_batches.end() ? nullptr : it->second.get();
}

void drop_graphs(Batch *bt) {
  for (auto &kv : bt->graphs) cudaGraphExecDestroy(kv.second);
  bt->graphs.clear();
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The (instance, x0, y0) list of the 2D tiles of the batch's tile shape,
// uploaded for fused launches (nothing when the batch does not fuse).
gscl_status build_tb_tiles(Batch *bt) {
  bt->tb_n = 0;
  if (!bt->tb_ok || bt->tb_k < 2) return GSCL_OK;
  const int TX = tb2d_tile_x(bt->tb_tile), TY = tb2d_tile_y(bt->tb_tile);
  std::vector<int4> tiles;
  for (int i = 0; i < bt->n_inst; ++i)
    for (int64_t y = 0; y < bt->ny[i]; y += TY)
      for (int64_t x = 0; x < bt->nx[i]; x += TX) tiles.push_back(make_int4(i, (int)x, (int)y, 0));
  if ((int)tiles.size() > bt->tb_cap) {
    if (bt->tb_tiles) cudaFree(bt->tb_tiles);
    bt->tb_tiles = nullptr;
    bt->tb_cap = 0;
    cudaError_t e = cudaMalloc(&bt->tb_tiles, sizeof(int4) * tiles.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc of the batch's tile list");
    bt->tb_cap = (int)tiles.size();
  }
  cudaError_t e = cudaMemcpy(bt->tb_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "uploading the batch's tile list");
  bt->tb_n = (int)tiles.size();
  return GSCL_OK;
}

// Work-list for one wave of G CTAs over instances of work[i] (tile, plane)
// pairs each (nz[i] planes per tile column): run b = [W b / G, W (b+1) / G)
// split at instance and column ends.
void make_worklist(const std::vector<long long> &work, const std::vector<int64_t> &nz, long long G,
                   std::vector<Segment> *segs, std::vector<int32_t> *cta_seg, std::vector<int32_t> *inst_seg) {
  const int n = (int)work.size();
  long long W = 0;
  for (long long w : work) W += w;
  segs->clear();
  cta_seg->assign(G + 1, 0);
  inst_seg->assign(n + 1, -1);
  int inst = 0;
  long long inst_start = 0;
  for (long long b = 0; b < G; ++b) {
    (*cta_seg)[b] = (int32_t)segs->size();
    long long pos = W * b / G;
    const long long end = W * (b + 1) / G;
    while (pos < end) {
      while (pos >= inst_start + work[inst]) inst_start += work[inst++];
      if ((*inst_seg)[inst] < 0) (*inst_seg)[inst] = (int32_t)segs->size();
      const long long local = pos - inst_start;
      const long long col = local / nz[inst];
      const long long zoff = local - col * nz[inst];
      const long long len = std::min(end - pos, nz[inst] - zoff);
      segs->push_back(Segment{inst, (int32_t)col, (int32_t)zoff, (int32_t)len});
      pos += len;
    }
  }
  (*cta_seg)[G] = (int32_t)segs->size();
  (*inst_seg)[n] = (int32_t)segs->size();
  for (int i = n - 1; i >= 0; --i)
    if ((*inst_seg)[i] < 0) (*inst_seg)[i] = (*inst_seg)[i + 1];
}

// Plans every instance in both ping-pong directions, builds the work-list
// for one wave and uploads the tables.
gscl_status build(Batch *bt) {
  drop_graphs(bt);
  bt->built = false;
  const int n = bt->n_inst;
  std::vector<InstDesc> tabs[2];
  tabs[0].resize(n);
  tabs[1].resize(n);
  std::vector<long long> work(n);
  std::vector<int64_t> nz(n);
  std::vector<InstWeights> wrows(n);
  bt->buf_a.assign(n, nullptr);
  bt->buf_b.assign(n, nullptr);
  TileCfg cfg = bt->cfg;
  bool any_eqw = false, all_eqw = true;  // instances allowing the group evaluation (flags in the weight rows)
  bool tb_ok = !bt->colored && bt->n_in == 1 && bt->n_out == 1;
  bool tb3_ok = !bt->colored && bt->n_out == 1;
  std::vector<InstDesc> tabs3[2];
  tabs3[0].resize(n);
  tabs3[1].resize(n);
  std::vector<long long> work3(n);
  bt->nx.assign(n, 0);
  bt->ny.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    Bound b;
    const gscl_stencil *op = bt->colored ? &bt->inst_st[i] : &bt->st;
    if (gscl_status s = bind(op, false, &bt->in_h[(size_t)i * bt->n_in], bt->n_in,
                             bt->n_out ? &bt->out_h[(size_t)i * bt->n_out] : nullptr, bt->n_out, nullptr, &b, -1, 0,
                             bt->colored))
      return s;
    if (b.in[0].dtype != bt->dtype) return fail(GSCL_ERR_DTYPE, "instance %d has another dtype", i);
    if (b.empty) return fail(GSCL_ERR_INVALID, "instance %d has an empty interior", i);
    if (!bt->colored && bt->n_out &&
        (b.in[0].halo[0] != b.out[0].halo[0] || b.in[0].halo[1] != b.out[0].halo[1] ||
         b.in[0].halo[2] != b.out[0].halo[2] || overlaps(b.in[0], b.out[0])))
      return fail(GSCL_ERR_SHAPE, "instance %d: in[0] and out[0] must be distinct grids of one layout", i);
    for (int dir = 0; dir < 2; ++dir) {
      Bound bd = b;
      if (dir == 1) {
        if (bt->n_out < 1 || bt->colored) break;  // coloured batches work in place: one direction
        std::swap(bd.in[0], bd.out[0]);
        for (int a = 1; a < bt->n_in; ++a)
          if (bd.in_h[a] == bd.in_h[0]) bd.in[a] = bd.in[0];
      }
      Plan pl;
      if (gscl_status s = make_plan(bd, bt->has_value, &pl, cfg)) return s;
      if (i == 0 && dir == 0) {
        if (pl.op != OP_GENERIC && !batch_capable(pl.op)) {
          cfg.generic = true;  // no batched kernel for this structure: interpret the term list
          bt->cfg.generic = true;
          if (gscl_status s = make_plan(bd, bt->has_value, &pl, cfg)) return s;
        }
        bt->base = pl;
      } else if (pl.op != bt->base.op || pl.smem != bt->base.smem || pl.threads != bt->base.threads ||
                 pl.P.R != bt->base.P.R || memcmp(pl.P.in_bw, bt->base.P.in_bw, sizeof pl.P.in_bw) != 0 ||
                 memcmp(pl.P.in_bh, bt->base.P.in_bh, sizeof pl.P.in_bh) != 0) {
        return fail(GSCL_ERR_SHAPE, "instance %d plans a different tile shape", i);
      }
      tabs[dir][i] = pl.P.inst;
      // 3D two-sweep passes: the pass's own boxes and tiles
      tb3_ok = tb3_ok && pl.op != OP_GENERIC && tb_eligible(bd, pl.op) && !tb2d_eligible(bd, pl.op);
      if (tb3_ok) {
        Plan tp;
        if (make_tb_plan(bd, 2, &tp) != GSCL_OK) {
          tb3_ok = false;
        } else {
          tabs3[dir][i] = tp.P.inst;
          if (dir == 0) work3[i] = tp.work;
          if (i == 0 && dir == 0) bt->tb3_base = tp;
        }
      }
      if (dir == 0) {
        tb_ok = tb_ok && tb2d_eligible(bd, pl.op);
        bt->nx[i] = bd.in[0].n[0];
        bt->ny[i] = bd.in[0].n[1];
        work[i] = pl.work;
        nz[i] = pl.P.inst.hi[2] - pl.P.inst.lo[2];
        // this instance's weights in the order of the launch's term table
        memset(&wrows[i], 0, sizeof(InstWeights));
        for (int k = 0; k < pl.P.out_begin[pl.P.n_out]; ++k) {
          wrows[i].wd[k] = pl.P.terms[k].wd;
          wrows[i].wf[k] = pl.P.terms[k].wf;
          wrows[i].wl[k] = pl.P.terms[k].wl;
        }
        wrows[i].eq = pl.eqw ? 1 : 0;
        any_eqw = any_eqw || pl.eqw;
        all_eqw = all_eqw && pl.eqw;
      }
    }
    bt->buf_a[i] = b.in[0].buf;
    bt->buf_b[i] = (bt->n_out && !bt->colored) ? b.out[0].buf : nullptr;
  }
  Plan &base = bt->base;
  base.batch = true;
  base.eqw = any_eqw;
  base.eq_mixed = any_eqw && !all_eqw;
  // one wave of CTAs
  int occ = 0;
  const int red_probe = bt->n_out ? RED_NONE : RED_L2;
  if (gscl_status s = launch(base, bt->dtype, red_probe, nullptr, &occ)) return s;
  long long W = 0;
  for (long long w : work) W += w;
  const long long G = std::max(1LL, std::min<long long>(W, (long long)sm_count() * occ));
  std::vector<Segment> segs;
  std::vector<int32_t> cta_seg, inst_seg;
  make_worklist(work, nz, G, &segs, &cta_seg, &inst_seg);
  // device blob: two tables, segments, CTA and instance segment starts, partials
  const size_t t_bytes = align_up(sizeof(InstDesc) * n, 256);
  const size_t s_bytes = align_up(sizeof(Segment) * segs.size(), 256);
  const size_t c_bytes = align_up(sizeof(int32_t) * (G + 1), 256);
  const size_t i_bytes = align_up(sizeof(int32_t) * (n + 1), 256);
  const size_t p_bytes = align_up(16 * segs.size(), 256);
  const size_t w_bytes = align_up(sizeof(InstWeights) * n, 256);
  const size_t need = 2 * t_bytes + s_bytes + c_bytes + i_bytes + p_bytes + w_bytes;
  if (need > bt->dev_bytes) {
    if (bt->dev) cudaFree(bt->dev);
    bt->dev = nullptr;
    bt->dev_bytes = 0;
    cudaError_t e = cudaMalloc(&bt->dev, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc of the batch tables");
    bt->dev_bytes = need;
  }
  char *p = bt->dev;
  bt->tab[0] = (InstDesc *)p;
  bt->tab[1] = (InstDesc *)(p + t_bytes);
  bt->segs = (Segment *)(p + 2 * t_bytes);
  bt->cta_seg = (int32_t *)(p + 2 * t_bytes + s_bytes);
  bt->inst_seg = (int32_t *)(p + 2 * t_bytes + s_bytes + c_bytes);
  bt->partials = (double *)(p + 2 * t_bytes + s_bytes + c_bytes + i_bytes);
  bt->wtab = (InstWeights *)(p + 2 * t_bytes + s_bytes + c_bytes + i_bytes + p_bytes);
  cudaError_t e = cudaMemcpy(bt->tab[0], tabs[0].data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && bt->n_out && !bt->colored)
    e = cudaMemcpy(bt->tab[1], tabs[1].data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->wtab, wrows.data(), sizeof(InstWeights) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->segs, segs.data(), sizeof(Segment) * segs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->cta_seg, cta_seg.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->inst_seg, inst_seg.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "uploading the batch tables");
  bt->G = (int)G;
  bt->S = (int)segs.size();
  bt->tb_ok = tb_ok;
  bt->tb3_ok = false;
  if (tb3_ok) {
    // the two-sweep pass's work-list over one wave of its CTAs
    Plan &tb = bt->tb3_base;
    tb.batch = true;
    int occ3 = 0;
    if (launch_tb2_pass(tb, bt->dtype, nullptr, &occ3) == GSCL_OK) {
      long long W3 = 0;
      for (long long w : work3) W3 += w;
      const long long G3 = std::max(1LL, std::min<long long>(W3, (long long)sm_count() * std::max(1, occ3)));
      std::vector<Segment> segs3;
      std::vector<int32_t> cta3, inst3;
      make_worklist(work3, nz, G3, &segs3, &cta3, &inst3);
      const size_t t3 = align_up(sizeof(InstDesc) * n, 256), s3 = align_up(sizeof(Segment) * segs3.size(), 256);
      const size_t c3 = align_up(sizeof(int32_t) * (G3 + 1), 256);
      const size_t need3 = 2 * t3 + s3 + c3;
      cudaError_t e3 = cudaSuccess;
      if (need3 > bt->tb3_bytes) {
        if (bt->tb3_dev) cudaFree(bt->tb3_dev);
        bt->tb3_dev = nullptr;
        bt->tb3_bytes = 0;
        e3 = cudaMalloc(&bt->tb3_dev, need3);
        if (e3 == cudaSuccess) bt->tb3_bytes = need3;
      }
      if (e3 == cudaSuccess) {
        bt->tb3_tab[0] = (InstDesc *)bt->tb3_dev;
        bt->tb3_tab[1] = (InstDesc *)(bt->tb3_dev + t3);
        bt->tb3_segs = (Segment *)(bt->tb3_dev + 2 * t3);
        bt->tb3_cta = (int32_t *)(bt->tb3_dev + 2 * t3 + s3);
        e3 = cudaMemcpy(bt->tb3_tab[0], tabs3[0].data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice);
        if (e3 == cudaSuccess)
          e3 = cudaMemcpy(bt->tb3_tab[1], tabs3[1].data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice);
        if (e3 == cudaSuccess)
          e3 = cudaMemcpy(bt->tb3_segs, segs3.data(), sizeof(Segment) * segs3.size(), cudaMemcpyHostToDevice);
        if (e3 == cudaSuccess)
          e3 = cudaMemcpy(bt->tb3_cta, cta3.data(), sizeof(int32_t) * (G3 + 1), cudaMemcpyHostToDevice);
      }
      if (e3 != cudaSuccess) return cuda_fail(e3, "uploading the batch's two-sweep tables");
      bt->tb3_G = (int)G3;
      tb.batch_ctas = (int)G3;
      tb.P.segs = bt->tb3_segs;
      tb.P.cta_seg = bt->tb3_cta;
      bt->tb3_ok = true;
    }
  }
  if (!tb_ok && !(bt->tb3_ok && bt->tb_k == 2)) bt->tb_k = 1;
  if (gscl_status s = build_tb_tiles(bt)) return s;
  base.batch_ctas = (int)G;
  base.P.segs = bt->segs;
  base.P.cta_seg = bt->cta_seg;
  base.P.seg_partials = bt->partials;
  base.P.inst_w = bt->wtab;
  bt->built = true;
  return GSCL_OK;
}

// Which table reads the buffers in[0] names now (0 or 1); rebuilds the
// tables when the instances' buffers are not the two the tables know.
gscl_status current_table(Batch *bt, int *which) {
  if (bt->built) {
    int t = -1;
    bool consistent = true;
    for (int i = 0; i < bt->n_inst && consistent; ++i) {
      Grid g;
      if (gscl_status s = lookup(bt->in_h[(size_t)i * bt->n_in], &g)) return s;
      const int ti = g.buf == bt->buf_a[i] ? 0 : (bt->n_out && g.buf == bt->buf_b[i] ? 1 : -1);
      if (ti < 0 || (t >= 0 && ti != t)) consistent = false;
      t = ti;
    }
    if (consistent) {
      *which = t;
      return GSCL_OK;
    }
  }
  if (gscl_status s = build(bt)) return s;
  *which = 0;
  return GSCL_OK;
}

// Launches that `sweeps` sweeps take (tb_launch_plan).
int batch_launches(const Batch *bt, int sweeps) { return (int)tb_launch_plan(sweeps, bt->tb_k).size(); }

// One launch: a fused pass of k sweeps (k > 1) or one sweep, reading table t
// (halo_swap as in tb2d_kernel.cuh).
gscl_status enqueue_launch(Batch *bt, int t, int k, cudaStream_t stream, bool halo_swap = false) {
  if (k > 1 && bt->tb3_ok) {  // a 3D batch: the two-sweep pass over its own tables
    Plan pl = bt->tb3_base;
    pl.P.insts = bt->tb3_tab[t];
    return launch_tb2_pass(pl, bt->dtype, stream, nullptr);
  }
  Plan pl = bt->base;
  pl.P.insts = bt->tab[t];
  if (k > 1) {
    Tb2dArgs a{};
    a.tiles = bt->tb_tiles;
    a.n_tiles = bt->tb_n;
    a.halo_swap = halo_swap ? 1 : 0;
    a.K = k;
    a.TX = tb2d_tile_x(bt->tb_tile);
    a.TY = tb2d_tile_y(bt->tb_tile);
    return launch_tb2d(pl, bt->dtype, a, stream);
  }
  return launch(pl, bt->dtype, RED_NONE, stream, nullptr);
}

gscl_status enqueue_sweeps(Batch *bt, int first, int sweeps, cudaStream_t stream) {
  int L = 0, done = 0;
  for (int k : tb_launch_plan(sweeps, bt->tb_k)) {
    if (gscl_status st = enqueue_launch(bt, (first + L) & 1, k, stream, ((done - L) & 1) != 0)) return st;
    done += k;
    ++L;
  }
  return GSCL_OK;
}

// half_sweeps launches of a coloured batch, the colour alternating from `color`.
gscl_status enqueue_colored(Batch *bt, int color, int half_sweeps, cudaStream_t stream) {
  Plan pl = bt->base;
  pl.P.insts = bt->tab[0];
  for (int h = 0; h < half_sweeps; ++h) {
    pl.P.color = (color + h) & 1;
    if (gscl_status st = launch(pl, bt->dtype, RED_NONE, stream, nullptr)) return st;
  }
  return GSCL_OK;
}

// Replays (capturing it first, once) the graph of `key`'s launches, or
// enqueues them directly.
template <class Enqueue>
gscl_status run_group(Batch *bt, std::pair<int, int> key, bool use_graph, cudaStream_t st, Enqueue enqueue) {
  if (!use_graph) return enqueue(st);
  auto it = bt->graphs.find(key);
  if (it == bt->graphs.end()) {
    if (!bt->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    cudaError_t e = cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    gscl_status s = enqueue(bt->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(bt->cap_stream, &graph);
    if (s != GSCL_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    it = bt->graphs.emplace(key, exec).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second, st);
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "cudaGraphLaunch");
}

template <int RED>
gscl_status finalize(Batch *bt, double *results, cudaStream_t stream) {
  const int threads = 128, per_block = threads / 32;  // one warp per instance
  batch_finalize_kernel<RED><<<(bt->n_inst + per_block - 1) / per_block, threads, 0, stream>>>(
      bt->partials, bt->inst_seg, bt->n_inst, results);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "batch finalize launch");
}

// gscl_batch_create and gscl_batch_create_colored: ops holds one operator
// (plain batches) or one per instance (coloured batches).
gscl_status create_batch(const gscl_stencil *ops, bool colored, int32_t n_inst, const gscl_grid *in, int32_t n_in,
                         const gscl_grid *out, int32_t n_out, gscl_batch *out_batch) {
  if (!out_batch) return fail(GSCL_ERR_INVALID, "out_batch is required");
  *out_batch = 0;
  if (n_inst < 1 || n_inst > (1 << 20)) return fail(GSCL_ERR_INVALID, "n_inst = %d outside [1, 2^20]", n_inst);
  const gscl_stencil *op = ops;
  if (!op || !op->terms || op->n_terms < 1 || op->n_terms > kMaxTerms)
    return fail(GSCL_ERR_INVALID, "a batch needs an operator with 1..%d terms", kMaxTerms);
  if (n_in < 1 || n_in > kMaxIn || n_out < 0 || n_out > kMaxOut_ || !in || (n_out && !out))
    return fail(GSCL_ERR_INVALID, "bad grid counts or arrays");
  if (colored && n_out < 1) return fail(GSCL_ERR_INVALID, "a coloured batch needs an output");
  std::unique_ptr<Batch> bt(new Batch());
  bt->n_inst = n_inst;
  bt->n_in = n_in;
  bt->n_out = n_out;
  bt->colored = colored;
  bt->terms.assign(op->terms, op->terms + op->n_terms);
  bt->st = gscl_stencil{op->n_terms, 0, bt->terms.data()};
  if (colored) {
    // one operator per instance, all of the first one's structure
    bt->inst_terms.resize(n_inst);
    bt->inst_st.resize(n_inst);
    for (int i = 0; i < n_inst; ++i) {
      const gscl_stencil &oi = ops[i];
      if (!oi.terms || oi.n_terms != op->n_terms)
        return fail(GSCL_ERR_INVALID, "instance %d: its operator must have the first one's %d terms", i, op->n_terms);
      for (int t = 0; t < op->n_terms; ++t) {
        const gscl_term &a = oi.terms[t], &b = op->terms[t];
        if (a.dx != b.dx || a.dy != b.dy || a.dz != b.dz || a.in != b.in || a.coef != b.coef || a.out != b.out)
          return fail(GSCL_ERR_INVALID, "instance %d: term %d differs from the first operator's beyond its weight",
                      i, t);
      }
      bt->inst_terms[i].assign(oi.terms, oi.terms + oi.n_terms);
      bt->inst_st[i] = gscl_stencil{oi.n_terms, 0, bt->inst_terms[i].data()};
    }
  }
  bt->in_h.assign(in, in + (size_t)n_inst * n_in);
  if (n_out) bt->out_h.assign(out, out + (size_t)n_inst * n_out);
  for (auto &t : bt->terms)
    if (t.out == GSCL_VALUE) bt->has_value = true;
  // GSCL_BATCH_NARROW=1 starts the batch on the narrow tiles (the tuner
  // chooses between the shapes by timing)
  if (const char *e = getenv("GSCL_BATCH_NARROW")) bt->cfg.narrow = atoi(e) != 0;
  // coloured batches of FP64 grids use the colour-compacted kernel where it
  // exists, as gscl_do_colored does (GSCL_COLOR_COMPACT=0 turns it off)
  if (colored) {
    const char *e = getenv("GSCL_COLOR_COMPACT");
    bt->cfg.compact = !(e && e[0] == '0');
  }
  Grid g0;
  if (gscl_status s = lookup(bt->in_h[0], &g0)) return s;
  bt->dtype = g0.dtype;
  if (gscl_status s = build(bt.get())) return s;  // validates every instance
  std::lock_guard<std::mutex> lk(g_batch_mu);
  const uint64_t id = g_next_batch++;
  g_batches[id].reset(bt.release());
  *out_batch = id;
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" {

gscl_status gscl_batch_create(const gscl_stencil *op, int32_t n_inst, const gscl_grid *in, int32_t n_in,
                              const gscl_grid *out, int32_t n_out, gscl_batch *out_batch) {
  return create_batch(op, false, n_inst, in, n_in, out, n_out, out_batch);
}

gscl_status gscl_batch_create_colored(const gscl_stencil *ops, int32_t n_inst, const gscl_grid *in, int32_t n_in,
                                      const gscl_grid *out, int32_t n_out, gscl_batch *out_batch) {
  return create_batch(ops, true, n_inst, in, n_in, out, n_out, out_batch);
}

gscl_status gscl_batch_run_colored(gscl_batch h, int32_t color, int32_t half_sweeps, int32_t use_graph,
                                   void *stream) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  if (color != 0 && color != 1) return fail(GSCL_ERR_INVALID, "color must be 0 or 1, got %d", color);
  if (half_sweeps < 1) return fail(GSCL_ERR_INVALID, "half_sweeps must be >= 1");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (!bt->colored) return fail(GSCL_ERR_INVALID, "not a coloured batch (gscl_batch_create_colored makes one)");
  int first = 0;
  if (gscl_status s = current_table(bt, &first)) return s;
  return run_group(bt, std::make_pair(2 + color, (int)half_sweeps), use_graph != 0, (cudaStream_t)stream,
                   [&](cudaStream_t st) { return enqueue_colored(bt, color, half_sweeps, st); });
}

gscl_status gscl_batch_destroy(gscl_batch h) {
  std::unique_ptr<Batch> bt;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batches.find(h);
    if (it == g_batches.end()) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
    bt = std::move(it->second);
    g_batches.erase(it);
  }
  drop_graphs(bt.get());
  if (bt->cap_stream) cudaStreamDestroy(bt->cap_stream);
  if (bt->dev) cudaFree(bt->dev);
  if (bt->tb_tiles) cudaFree(bt->tb_tiles);
  if (bt->tb3_dev) cudaFree(bt->tb3_dev);
  return GSCL_OK;
}

gscl_status gscl_batch_info(gscl_batch h, int32_t *ctas, int32_t *segments, int32_t *specialization) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (ctas) *ctas = bt->G;
  if (segments) *segments = bt->S;
  if (specialization) *specialization = bt->base.op;
  return GSCL_OK;
}

gscl_status gscl_batch_tile(gscl_batch h, int32_t *tile_x, int32_t *tile_y) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (tile_x) *tile_x = bt->base.tile_x;
  if (tile_y) *tile_y = bt->base.tile_y;
  return GSCL_OK;
}

gscl_status gscl_batch_temporal(gscl_batch h, int32_t *sweeps_per_launch, int32_t *tile_x, int32_t *tile_y) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (sweeps_per_launch) *sweeps_per_launch = bt->tb_k;
  const bool d3 = bt->tb3_ok && bt->tb_k > 1;
  if (tile_x) *tile_x = bt->tb_k > 1 ? (d3 ? Tb2Shape<float>::TX : tb2d_tile_x(bt->tb_tile)) : 0;
  if (tile_y) *tile_y = bt->tb_k > 1 ? (d3 ? Tb2Shape<float>::TY : tb2d_tile_y(bt->tb_tile)) : 0;
  return GSCL_OK;
}

gscl_status gscl_batch_set_temporal(gscl_batch h, int32_t sweeps_per_launch, int32_t tile_shape) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  if (sweeps_per_launch < 1 || sweeps_per_launch > kTb2dMaxK)
    return fail(GSCL_ERR_INVALID, "sweeps_per_launch = %d outside [1, %d]", sweeps_per_launch, kTb2dMaxK);
  if (tile_shape < 0 || tile_shape >= kTb2dShapes)
    return fail(GSCL_ERR_INVALID, "tile_shape = %d outside [0, %d)", tile_shape, kTb2dShapes);
  std::lock_guard<std::mutex> lk(bt->mu);
  int first = 0;
  if (gscl_status s = current_table(bt, &first)) return s;
  if (sweeps_per_launch > 1 && !bt->tb_ok && !(bt->tb3_ok && sweeps_per_launch == 2))
    return fail(GSCL_ERR_UNSUPPORTED,
                "batches fuse sweeps of 2D grids under a 5-point operator (up to 16) or two sweeps of 3D FP32 / "
                "BF16 grids under a 7-point star operator");
  drop_graphs(bt);
  bt->tb_k = sweeps_per_launch;
  bt->tb_tile = tile_shape;
  return build_tb_tiles(bt);
}

gscl_status gscl_batch_run(gscl_batch h, int32_t sweeps, int32_t use_graph, void *stream) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  if (sweeps < 1) return fail(GSCL_ERR_INVALID, "sweeps must be >= 1");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (bt->n_out < 1) return fail(GSCL_ERR_INVALID, "this batch's operator has no output to sweep");
  if (bt->colored) return fail(GSCL_ERR_INVALID, "a coloured batch sweeps by colour (gscl_batch_run_colored)");
  int first = 0;
  if (gscl_status s = current_table(bt, &first)) return s;
  if (gscl_status s = run_group(bt, std::make_pair(first, (int)sweeps), use_graph != 0, (cudaStream_t)stream,
                                [&](cudaStream_t st) { return enqueue_sweeps(bt, first, sweeps, st); }))
    return s;
  if (batch_launches(bt, sweeps) % 2 == 0)  // out[0] names the last launch's result, as in gscl_do_all
    for (int i = 0; i < bt->n_inst; ++i)
      if (gscl_status s = swap_storage(bt->in_h[(size_t)i * bt->n_in], bt->out_h[(size_t)i * bt->n_out])) return s;
  return GSCL_OK;
}

gscl_status gscl_batch_reduce(gscl_batch h, int32_t reduce_op, double *results, void *stream) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  if (!results) return fail(GSCL_ERR_INVALID, "results is NULL");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (!bt->has_value) return fail(GSCL_ERR_INVALID, "the batch's operator returns no value");
  if (bt->colored) return fail(GSCL_ERR_INVALID, "a coloured batch does not reduce (it updates in place)");
  int red;
  switch (reduce_op) {
    case GSCL_SUM: red = RED_SUM; break;
    case GSCL_MAXABS: red = RED_MAXABS; break;
    case GSCL_L2: red = RED_L2; break;
    default: return fail(GSCL_ERR_INVALID, "unknown reduce op %d", reduce_op);
  }
  int first = 0;
  if (gscl_status s = current_table(bt, &first)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl = bt->base;
  pl.P.insts = bt->tab[first];
  if (gscl_status s = launch(pl, bt->dtype, red, st, nullptr)) return s;
  switch (red) {
    case RED_SUM: return finalize<RED_SUM>(bt, results, st);
    case RED_MAXABS: return finalize<RED_MAXABS>(bt, results, st);
    default: return finalize<RED_L2>(bt, results, st);
  }
}

gscl_status gscl_batch_tune(gscl_batch h, int32_t trial_sweeps, void *stream, int32_t *warps, int32_t *prefetch) {
  Batch *bt = find_batch(h);
  if (!bt) return fail(GSCL_ERR_STATE, "unknown or destroyed batch");
  if (trial_sweeps < 1) return fail(GSCL_ERR_INVALID, "trial_sweeps must be >= 1");
  std::lock_guard<std::mutex> lk(bt->mu);
  if (bt->colored) return fail(GSCL_ERR_INVALID, "coloured batches are not tuned");
  cudaStream_t st = (cudaStream_t)stream;
  const int red = bt->n_out ? RED_NONE : RED_L2;
  const TileCfg keep = bt->cfg;
  float best_ms = 1e30f;
  TileCfg best = keep;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int nws[] = {2, 4, 8};
  const int pfs[] = {1, 2, 3};
  // tile shape: the dtype's default, and for FP32 / BF16 the narrow 64-column
  // tiles (4 rows per warp) that waste fewer lanes on narrow grids
  const int shapes = bt->dtype == GSCL_F64 ? 1 : 2;
  // GSCL_TUNE_LOG=1 prints every trial's time to stderr
  const char *log_env = getenv("GSCL_TUNE_LOG");
  const bool log = log_env && log_env[0] == '1';
  for (int narrow = 0; narrow < shapes; ++narrow)
  for (int nw : nws)
    for (int pf : pfs) {
      bt->cfg = TileCfg{nw, pf, keep.generic, narrow != 0};
      gscl_status bs = build(bt);
      if (bs != GSCL_OK) {  // e.g. does not fit in shared memory
        if (log) fprintf(stderr, "gscl_batch_tune: narrow %d warps %d prefetch %d: %s\n", narrow, nw, pf,
                         gscl_last_error());
        continue;
      }
      int first = 0;
      if (current_table(bt, &first) != GSCL_OK) continue;
      Plan pl = bt->base;
      pl.P.insts = bt->tab[first];  // in[0] -> out[0] every trial: in[0] is left as it was
      if (red != RED_NONE) pl.P.seg_partials = bt->partials;
      if (launch(pl, bt->dtype, red, st, nullptr) != GSCL_OK) {
        if (log) fprintf(stderr, "gscl_batch_tune: narrow %d warps %d prefetch %d: launch failed: %s\n", narrow,
                         nw, pf, gscl_last_error());
        continue;
      }
      // the better of two timed groups: one group can catch a slow moment
      float ms = 1e30f;
      bool timed = true;
      for (int rep = 0; rep < 2 && timed; ++rep) {
        cudaEventRecord(e0, st);
        for (int s = 0; s < trial_sweeps; ++s) launch(pl, bt->dtype, red, st, nullptr);
        cudaEventRecord(e1, st);
        timed = cudaEventSynchronize(e1) == cudaSuccess;
        float t = 0.f;
        if (timed) cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (!timed) break;
      if (log)
        fprintf(stderr, "gscl_batch_tune: narrow %d warps %d prefetch %d: tile %d x %d, %d CTAs, %.4f ms per sweep\n",
                narrow, nw, pf, bt->base.tile_x, bt->base.tile_y, bt->G, ms / trial_sweeps);
      if (ms < best_ms) {
        best_ms = ms;
        best = bt->cfg;
      }
    }
  bt->cfg = best;
  const int keep_k = bt->tb_k, keep_tile = bt->tb_tile;
  bt->tb_k = 1;
  if (gscl_status s = build(bt)) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
  }
  // 2D batches: sweeps fused per launch (K = 1, 2, 3, 4, 6, 8, 12, 16) x the
  // tile shapes, on the tuned single-sweep tiles; at least 48 sweeps per
  // candidate (a fused launch of a small 2D batch takes microseconds)
  if (bt->tb_ok && red == RED_NONE) {
    int first = 0;
    float best_sweep = 1e30f;
    int best_k = 1, best_tile = 0;
    const int trial = std::max((int)trial_sweeps, 48);
    if (current_table(bt, &first) == GSCL_OK) {
      for (int K : {1, 2, 3, 4, 6, 8, 12, 16})
        for (int t = 0; t < (K == 1 ? 1 : kTb2dShapes); ++t) {
          bt->tb_k = K;
          bt->tb_tile = t;
          if (build_tb_tiles(bt) != GSCL_OK) continue;
          if (enqueue_launch(bt, first, K, st) != GSCL_OK) continue;  // warm-up (kernel set-up)
          const int passes = std::max(1, trial / K);
          float ms = 1e30f;
          bool timed = true;
          for (int rep = 0; rep < 2 && timed; ++rep) {
            cudaEventRecord(e0, st);
            for (int p = 0; p < passes; ++p) enqueue_launch(bt, first, K, st);
            cudaEventRecord(e1, st);
            timed = cudaEventSynchronize(e1) == cudaSuccess;
            float tm = 0.f;
            if (timed) cudaEventElapsedTime(&tm, e0, e1);
            ms = std::min(ms, tm);
          }
          if (!timed) break;
          const float per_sweep = ms / (passes * K);
          if (log)
            fprintf(stderr, "gscl_batch_tune: %d sweeps per launch, tile %d x %d: %.5f ms per sweep\n", K,
                    tb2d_tile_x(t), tb2d_tile_y(t), per_sweep);
          if (per_sweep < best_sweep) {
            best_sweep = per_sweep;
            best_k = K;
            best_tile = t;
          }
        }
    }
    bt->tb_k = best_k;
    bt->tb_tile = best_tile;
  } else if (bt->tb3_ok && red == RED_NONE) {
    // 3D batches: single sweeps against two-sweep passes (trial_sweeps each)
    int first = 0;
    float best_sweep = 1e30f;
    int best_k = 1;
    if (current_table(bt, &first) == GSCL_OK) {
      for (int K : {1, 2}) {
        bt->tb_k = K;
        if (enqueue_launch(bt, first, K, st) != GSCL_OK) continue;  // warm-up (kernel set-up)
        const int passes = std::max(1, (int)trial_sweeps / K);
        float ms = 1e30f;
        bool timed = true;
        for (int rep = 0; rep < 2 && timed; ++rep) {
          cudaEventRecord(e0, st);
          for (int p = 0; p < passes; ++p) enqueue_launch(bt, first, K, st);
          cudaEventRecord(e1, st);
          timed = cudaEventSynchronize(e1) == cudaSuccess;
          float tm = 0.f;
          if (timed) cudaEventElapsedTime(&tm, e0, e1);
          ms = std::min(ms, tm);
        }
        if (!timed) break;
        const float per_sweep = ms / (passes * K);
        if (log) fprintf(stderr, "gscl_batch_tune: %d sweeps per launch (3D): %.5f ms per sweep\n", K, per_sweep);
        if (per_sweep < best_sweep) {
          best_sweep = per_sweep;
          best_k = K;
        }
      }
    }
    bt->tb_k = best_k;
  } else {
    bt->tb_k = (bt->tb_ok || bt->tb3_ok) ? keep_k : 1;
    bt->tb_tile = keep_tile;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graphs(bt);
  if (gscl_status s = build_tb_tiles(bt)) return s;
  if (warps) *warps = best.nw;
  if (prefetch) *prefetch = best.pf;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "tuning launches");
}

}  // extern "C"
