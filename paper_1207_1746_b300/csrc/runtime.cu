// Host runtime of libgscl.so: grid layout, the handle registry, host copies,
// swap, status strings, error detail, the device error word and tensor maps.
#include <algorithm>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <memory>
#include <mutex>
#include <vector>

#include "gscl_internal.h"

namespace gscl {

// ------------------------------------------------------------------ errors
static thread_local char t_last_error[512] = "";

gscl_status fail(gscl_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof t_last_error, fmt, ap);
  va_end(ap);
  return s;
}

gscl_status cuda_fail(cudaError_t e, const char *what) {
  return fail(GSCL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ layout
int32_t dtype_bytes(int32_t dtype) {
  switch (dtype) {
    case GSCL_F64: return 8;
    case GSCL_F32: return 4;
    case GSCL_BF16: return 2;
    default: return 0;
  }
}

// Rows padded to 128 bytes, leading pad so interior (0,0,0) sits on a
// 128-byte boundary (the pitch keeps every interior row aligned too).
gscl_status compute_layout(int32_t ndim, const int64_t n[3], const int32_t halo[3], int32_t dtype, Grid *g) {
  if (!n || !halo) return fail(GSCL_ERR_INVALID, "n and halo are required");
  if (ndim != 2 && ndim != 3) return fail(GSCL_ERR_INVALID, "ndim must be 2 or 3, got %d", ndim);
  int32_t elem = dtype_bytes(dtype);
  if (!elem) return fail(GSCL_ERR_INVALID, "unknown dtype %d", dtype);
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1) return fail(GSCL_ERR_INVALID, "n[%d] = %lld must be >= 1", a, (long long)n[a]);
    if (halo[a] < 0 || halo[a] > GSCL_MAX_HALO)
      return fail(GSCL_ERR_INVALID, "halo[%d] = %d outside [0, %d]", a, halo[a], GSCL_MAX_HALO);
  }
  if (ndim == 2 && (n[2] != 1 || halo[2] != 0))
    return fail(GSCL_ERR_INVALID, "a 2D grid has n[2] = 1 and halo[2] = 0");
  const int64_t align = 128 / elem;  // elements per 128 bytes
  g->ndim = ndim;
  g->dtype = dtype;
  g->elem = elem;
  for (int a = 0; a < 3; ++a) {
    g->n[a] = n[a];
    g->halo[a] = halo[a];
  }
  g->off = (align - halo[0] % align) % align;
  const int64_t row = g->off + n[0] + 2 * (int64_t)halo[0];
  g->pitch = (row + align - 1) / align * align;
  g->plane = g->pitch * (n[1] + 2 * (int64_t)halo[1]);
  g->bytes = g->plane * (n[2] + 2 * (int64_t)halo[2]) * elem;
  const int64_t limit = (int64_t)1 << 47;
  if (g->bytes <= 0 || g->bytes > limit) return fail(GSCL_ERR_INVALID, "grid too large");
  // TMA addresses the array with 32-bit coordinates of at most 2^31 - 1 per axis
  if (g->pitch >= ((int64_t)1 << 31) || n[1] + 2 * halo[1] >= ((int64_t)1 << 31) ||
      n[2] + 2 * halo[2] >= ((int64_t)1 << 31))
    return fail(GSCL_ERR_INVALID, "grid axis too long");
  return GSCL_OK;
}

// ------------------------------------------------------------------ registry
// Handle = (slot index + 1) << 20 | generation (20 bits); a destroyed slot
// bumps its generation so stale ids never match a later grid.
namespace {
struct Slot {
  Grid grid;
  uint32_t gen = 1;
  bool live = false;
};
std::mutex g_mu;
std::vector<std::unique_ptr<Slot>> g_slots;
std::vector<uint32_t> g_free;

constexpr uint64_t kGenBits = 20;
constexpr uint64_t kGenMask = (1ull << kGenBits) - 1;

Slot *find_locked(gscl_grid h) {
  if (h == 0) return nullptr;
  uint64_t idx = (h >> kGenBits) - 1;
  uint32_t gen = (uint32_t)(h & kGenMask);
  if (idx >= g_slots.size()) return nullptr;
  Slot *s = g_slots[idx].get();
  if (!s->live || s->gen != gen) return nullptr;
  return s;
}
}  // namespace

gscl_status lookup(gscl_grid h, Grid *out) {
  std::lock_guard<std::mutex> lk(g_mu);
  Slot *s = find_locked(h);
  if (!s) return fail(GSCL_ERR_STATE, "unknown or destroyed grid handle 0x%llx", (unsigned long long)h);
  *out = s->grid;
  return GSCL_OK;
}

static bool same_layout(const Grid &a, const Grid &b) {
  return a.ndim == b.ndim && a.dtype == b.dtype && a.n[0] == b.n[0] && a.n[1] == b.n[1] && a.n[2] == b.n[2] &&
         a.halo[0] == b.halo[0] && a.halo[1] == b.halo[1] && a.halo[2] == b.halo[2] && a.device == b.device;
}

gscl_status swap_storage(gscl_grid a, gscl_grid b) {
  std::lock_guard<std::mutex> lk(g_mu);
  Slot *sa = find_locked(a);
  Slot *sb = find_locked(b);
  if (!sa || !sb) return fail(GSCL_ERR_STATE, "swap of an unknown or destroyed grid handle");
  if (sa == sb) return GSCL_OK;
  if (!same_layout(sa->grid, sb->grid)) return fail(GSCL_ERR_SHAPE, "swap of grids with different layouts");
  std::swap(sa->grid.buf, sb->grid.buf);
  std::swap(sa->grid.buf_bytes, sb->grid.buf_bytes);
  return GSCL_OK;
}

// ------------------------------------------------------------------ devices
int sm_count() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

int max_smem_per_block() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

int smem_per_sm() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  return v;
}

// One int per device: bit 0 = a bounded wait timed out, bit 1 = a run-time
// compiled operator read outside its declared reach.  A __device__
// variable exists once per device and is zero when the module loads.  Host
// code reaches it only through cudaGetSymbolAddress.
__device__ int g_device_error;

int *device_error_word() {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
  return (int *)p;
}

// Reads the current device's error word after the caller has synchronised,
// clears it and turns a set flag into a status (reported once).
gscl_status take_device_error() {
  int *word = device_error_word();
  if (!word) return fail(GSCL_ERR_CUDA, "device error word unavailable");
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, word, sizeof flag, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  if (flag) {
    int zero = 0;
    cudaMemcpy(word, &zero, sizeof zero, cudaMemcpyHostToDevice);
    if (flag & 2) return fail(GSCL_ERR_RANGE, "a run-time compiled operator read outside its declared reach");
    return fail(GSCL_ERR_TIMEOUT, "a bounded device-side wait gave up (flag %d)", flag);
  }
  return GSCL_OK;
}

// ------------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// A 3D map over the whole padded array: dim0 = pitch (x), dim1 = padded rows
// (y), dim2 = padded planes (z); box = box_x x box_y x 1.  Out-of-bounds
// box elements read as zero.
gscl_status encode_tensor_map_3d(CUtensorMap *map, const Grid &g, uint32_t box_x, uint32_t box_y) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) return fail(GSCL_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMapDataType dt = g.dtype == GSCL_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : g.dtype == GSCL_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  // x extent: the elements a row actually holds (leading pad, halo, interior,
  // halo).  Box columns past it are the row's padding: TMA fills them
  // instead of fetching them, and no stencil reads them.
  cuuint64_t dims[3] = {(cuuint64_t)std::min<int64_t>(g.pitch, g.off + g.n[0] + 2 * (int64_t)g.halo[0]),
                        (cuuint64_t)(g.n[1] + 2 * g.halo[1]), (cuuint64_t)(g.n[2] + 2 * g.halo[2])};
  cuuint64_t strides[2] = {(cuuint64_t)(g.pitch * g.elem), (cuuint64_t)(g.plane * g.elem)};
  cuuint32_t box[3] = {box_x, box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  // L2 fetch granularity of the boxes' misses: 64 B measured best on B300
  // (256^3 FP32 sweep 0.0415 -> 0.0393 ms, 96 uneven grids' DRAM reads
  // 1.76 -> 1.39 GB per sweep against 256 B; unchanged for FP64).  Larger
  // promotion over-fetches the short rows of narrow grids and tile edges.
  CUtensorMapL2promotion promo = CU_TENSOR_MAP_L2_PROMOTION_L2_64B;
  if (const char *e = getenv("GSCL_L2_PROMOTION")) {
    const int v = atoi(e);
    promo = v == 0 ? CU_TENSOR_MAP_L2_PROMOTION_NONE
            : v == 64 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
            : v == 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
            : v == 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                       : promo;
  }
  CUresult r = enc(map, dt, 3, g.buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(GSCL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GSCL_OK;
}

// Host copies: rows of a dense array (width elements each) into the grid's pitched rows:
// one CTA per row at a time, threads across the row.
template <typename E>
__global__ void unpack_rows_kernel(E *dst, const E *src, int64_t width, int64_t pitch, int64_t rows) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < width; c += blockDim.x) dst[r * pitch + c] = src[r * width + c];
}

}  // namespace gscl

using namespace gscl;

// ====================================================================== C ABI
extern "C" {

const char *gscl_status_str(gscl_status s) {
  switch (s) {
    case GSCL_OK: return "ok";
    case GSCL_ERR_INVALID: return "invalid argument";
    case GSCL_ERR_RANGE: return "range or stencil offset outside the grid";
    case GSCL_ERR_ALIAS: return "output grid aliased by a shifted read or bound twice";
    case GSCL_ERR_DTYPE: return "grids of one call differ in dtype";
    case GSCL_ERR_SHAPE: return "grids of one call differ in extent or layout";
    case GSCL_ERR_OOM: return "buffer or workspace too small";
    case GSCL_ERR_CUDA: return "CUDA error";
    case GSCL_ERR_STATE: return "unknown or destroyed handle";
    case GSCL_ERR_TIMEOUT: return "device-side wait timed out";
    case GSCL_ERR_UNSUPPORTED: return "unsupported by this library";
  }
  return "unknown status";
}

const char *gscl_last_error(void) { return t_last_error; }

gscl_status gscl_grid_layout(int32_t ndim, const int64_t n[3], const int32_t halo[3], int32_t dtype,
                             int64_t *pitch_elems, int64_t *offset_elems, int64_t *bytes) {
  if (!pitch_elems || !offset_elems || !bytes) return fail(GSCL_ERR_INVALID, "output pointers are required");
  Grid g;
  gscl_status s = compute_layout(ndim, n, halo, dtype, &g);
  if (s != GSCL_OK) return s;
  *pitch_elems = g.pitch;
  *offset_elems = g.off;
  *bytes = g.bytes;
  return GSCL_OK;
}

gscl_status gscl_grid_create(int32_t ndim, const int64_t n[3], const int32_t halo[3], int32_t dtype, void *dev_buf,
                             int64_t buf_bytes, gscl_grid *out) {
  if (!out) return fail(GSCL_ERR_INVALID, "out is required");
  *out = 0;
  Grid g;
  gscl_status s = compute_layout(ndim, n, halo, dtype, &g);
  if (s != GSCL_OK) return s;
  if (!dev_buf) return fail(GSCL_ERR_INVALID, "dev_buf is NULL");
  if (((uintptr_t)dev_buf) % 128) return fail(GSCL_ERR_INVALID, "dev_buf must be 128-byte aligned");
  if (buf_bytes < g.bytes)
    return fail(GSCL_ERR_OOM, "buffer has %lld bytes, layout needs %lld", (long long)buf_bytes, (long long)g.bytes);
  g.buf = (char *)dev_buf;
  g.buf_bytes = buf_bytes;
  if (cudaGetDevice(&g.device) != cudaSuccess) g.device = -1;
  std::lock_guard<std::mutex> lk(g_mu);
  uint32_t idx;
  if (!g_free.empty()) {
    idx = g_free.back();
    g_free.pop_back();
  } else {
    idx = (uint32_t)g_slots.size();
    g_slots.emplace_back(new Slot());
  }
  Slot *slot = g_slots[idx].get();
  slot->grid = g;
  slot->live = true;
  *out = ((uint64_t)(idx + 1) << kGenBits) | slot->gen;
  return GSCL_OK;
}

gscl_status gscl_grid_destroy(gscl_grid h) {
  std::lock_guard<std::mutex> lk(g_mu);
  Slot *s = find_locked(h);
  if (!s) return fail(GSCL_ERR_STATE, "destroy of an unknown or destroyed grid handle");
  s->live = false;
  s->gen = (s->gen + 1) & kGenMask;
  if (s->gen == 0) s->gen = 1;
  g_free.push_back((uint32_t)((h >> kGenBits) - 1));
  return GSCL_OK;
}

gscl_status gscl_grid_info(gscl_grid h, gscl_grid_desc *out) {
  if (!out) return fail(GSCL_ERR_INVALID, "out is required");
  Grid g;
  gscl_status s = lookup(h, &g);
  if (s != GSCL_OK) return s;
  out->ndim = g.ndim;
  out->dtype = g.dtype;
  for (int a = 0; a < 3; ++a) {
    out->n[a] = g.n[a];
    out->halo[a] = g.halo[a];
  }
  out->elem_bytes = g.elem;
  out->pitch_elems = g.pitch;
  out->offset_elems = g.off;
  out->plane_elems = g.plane;
  out->bytes = g.bytes;
  out->dev_buf = g.buf;
  return GSCL_OK;
}

// Host -> device goes through a dense device copy and a row-scatter kernel:
// a strided host-to-device copy of short rows runs at 15.6 GB/s on B300
// against 38.8 GB/s for one contiguous copy (256^3 FP64 grid, pinned memory).
// Device -> host strided copies run at full speed (56 GB/s) and stay 2D.
static gscl_status copy2d(const Grid &g, void *host, bool to_host, void *stream) {
  const size_t width = (size_t)(g.n[0] + 2 * g.halo[0]) * g.elem;
  const size_t rows = (size_t)(g.n[1] + 2 * g.halo[1]) * (size_t)(g.n[2] + 2 * g.halo[2]);
  char *dev = g.buf + g.off * g.elem;
  cudaStream_t st = (cudaStream_t)stream;
  if (!to_host) {
    void *tmp = nullptr;
    if (cudaMallocAsync(&tmp, width * rows, st) == cudaSuccess) {
      cudaError_t e = cudaMemcpyAsync(tmp, host, width * rows, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) {
        cudaFreeAsync(tmp, st);
        return cuda_fail(e, "cudaMemcpyAsync");
      }
      const int64_t w = (int64_t)(width / g.elem);
      const unsigned blocks = (unsigned)std::min<size_t>(rows, (size_t)sm_count() * 16);
      switch (g.elem) {
        case 8: unpack_rows_kernel<<<blocks, 256, 0, st>>>((uint64_t *)dev, (const uint64_t *)tmp, w, g.pitch, (int64_t)rows); break;
        case 4: unpack_rows_kernel<<<blocks, 256, 0, st>>>((uint32_t *)dev, (const uint32_t *)tmp, w, g.pitch, (int64_t)rows); break;
        default: unpack_rows_kernel<<<blocks, 256, 0, st>>>((uint16_t *)dev, (const uint16_t *)tmp, w, g.pitch, (int64_t)rows); break;
      }
      e = cudaGetLastError();
      cudaFreeAsync(tmp, st);
      if (e != cudaSuccess) return cuda_fail(e, "unpacking host rows");
      return GSCL_OK;
    }
    cudaGetLastError();  // no room for the dense copy: the strided copy below
  }
  cudaError_t e = to_host ? cudaMemcpy2DAsync(host, width, dev, g.pitch * g.elem, width, rows,
                                              cudaMemcpyDeviceToHost, st)
                          : cudaMemcpy2DAsync(dev, g.pitch * g.elem, host, width, width, rows,
                                              cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
  return GSCL_OK;
}

gscl_status gscl_grid_copy_from_host(gscl_grid h, const void *host, void *stream) {
  if (!host) return fail(GSCL_ERR_INVALID, "host pointer is NULL");
  Grid g;
  gscl_status s = lookup(h, &g);
  if (s != GSCL_OK) return s;
  return copy2d(g, const_cast<void *>(host), false, stream);
}

gscl_status gscl_grid_copy_to_host(gscl_grid h, void *host, void *stream) {
  if (!host) return fail(GSCL_ERR_INVALID, "host pointer is NULL");
  Grid g;
  gscl_status s = lookup(h, &g);
  if (s != GSCL_OK) return s;
  return copy2d(g, host, true, stream);
}

gscl_status gscl_swap(gscl_grid *a, gscl_grid *b) {
  if (!a || !b) return fail(GSCL_ERR_INVALID, "swap needs two handle pointers");
  return swap_storage(*a, *b);
}

gscl_status gscl_sync(void *stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return take_device_error();
}

}  // extern "C"
