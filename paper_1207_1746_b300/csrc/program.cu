// Point operators compiled at run time.
//
// In the paper a stencil operator is a C++ function object compiled with the
// program (Section 3, Fig. 1b), so any arithmetic can run at each core
// element.  Here an operator can also arrive as source text: a block of CUDA
// C++ statements that reads inputs through in0(dx, dy, dz) .. in7(..), may
// use the core element's index (i, j, k) as the paper's stateful stencils do,
// and assigns out0 .. out2.  NVRTC compiles it into a do_all kernel for
// sm_103a when the program is created; the module is loaded on a device at
// its first launch there.
//
// Two kernels are generated.  The plain one: a 32 x 8 block of threads per
// (x, y) tile of the range, each CTA walking a run of planes two at a time,
// every read a load from global memory (L1 and L2 keep the neighbours of
// adjacent elements); it serves FP64 grids and in-place calls.  The staged
// one (FP32 / BF16): a 64 x 8 tile per CTA whose inputs' planes, with their
// apron, stream through a shared-memory ring filled two planes ahead by
// 16-byte cp.async copies; the body reads the ring.
// Each read checks its offset against the reach declared at creation, so a
// body that reads farther stays inside the grids: the read returns 0 and
// sets bit 1 of the device error word, which gscl_sync reports as
// GSCL_ERR_RANGE.
//
// NVRTC is opened with dlopen and the driver's module calls are taken from
// the runtime (cudaGetDriverEntryPointByVersion), so the library loads on
// machines without either.
#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sweep_host.h"

namespace gscl {
namespace {

// ------------------------------------------------------------------ NVRTC
struct Nvrtc {
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  bool ok = false;
};

const Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so"};
    void *h = nullptr;
    for (const char *nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) return;
    n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
    n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
    n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
  });
  return n;
}

// ------------------------------------------------------------------ driver module calls
struct Driver {
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleGetFunction) get = nullptr;
  decltype(&cuLaunchKernel) launch = nullptr;
  decltype(&cuModuleUnload) unload = nullptr;
  decltype(&cuFuncSetAttribute) set_attr = nullptr;
  bool ok = false;
};

const Driver &driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [](const char *name) -> void * {
      void *p = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess)
        return nullptr;
      return p;
    };
    d.load = (decltype(d.load))get("cuModuleLoadData");
    d.get = (decltype(d.get))get("cuModuleGetFunction");
    d.launch = (decltype(d.launch))get("cuLaunchKernel");
    d.unload = (decltype(d.unload))get("cuModuleUnload");
    d.set_attr = (decltype(d.set_attr))get("cuFuncSetAttribute");
    d.ok = d.load && d.get && d.launch && d.unload && d.set_attr;
  });
  return d;
}

// ------------------------------------------------------------------ kernel source
// Parameters of the generated kernel; the source below declares the same
// layout (every field 8 bytes).
struct JitParams {
  const void *in[kMaxIn];
  long long in_pitch[kMaxIn], in_plane[kMaxIn];
  long long in_x0[kMaxIn], in_x1[kMaxIn], in_y0[kMaxIn], in_y1[kMaxIn];  // staged copies: row bounds
  void *out[kMaxOut_];
  long long out_pitch[kMaxOut_], out_plane[kMaxOut_];
  long long lo[3], hi[3];
  double *vout;  // do_reduce: the value at (i, j, k) goes to vout[(k-lo) v_plane + (j-lo) v_pitch + (i-lo)]
  long long v_pitch, v_plane;
  int *err;
};

const char *kJitTemplate = R"SRC(
typedef %s real;
typedef %s gscl_stor;
#define GSCL_RX %d
#define GSCL_RY %d
#define GSCL_RZ %d
#define GSCL_NIN %d
#define GSCL_NOUT %d
#define GSCL_PF 2
struct GsclJitParams {
  const gscl_stor *in[%d];
  long long in_pitch[%d], in_plane[%d];
  long long in_x0[%d], in_x1[%d], in_y0[%d], in_y1[%d];
  gscl_stor *out[%d];
  long long out_pitch[%d], out_plane[%d];
  long long lo[3], hi[3];
  double *vout;
  long long v_pitch, v_plane;
  int *err;
};
__device__ __forceinline__ real gscl_ld(double x) { return (real)x; }
__device__ __forceinline__ real gscl_ld(float x) { return (real)x; }
__device__ __forceinline__ real gscl_ld(unsigned short x) { return (real)__uint_as_float((unsigned)x << 16); }
__device__ __forceinline__ unsigned short __ldg(const unsigned short *p) {
  unsigned short v;
  asm("ld.global.nc.u16 %%0, [%%1];" : "=h"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void gscl_st(double *p, real v) { *p = (double)v; }
__device__ __forceinline__ void gscl_st(float *p, real v) { *p = (float)v; }
// float -> bfloat16, round to nearest even on the bit pattern (NaN kept quiet)
__device__ __forceinline__ void gscl_st(unsigned short *p, real v) {
  unsigned u = __float_as_uint((float)v);
  if ((u & 0x7fffffffu) > 0x7f800000u) { *p = (unsigned short)((u >> 16) | 0x40u); return; }
  u += 0x7fffu + ((u >> 16) & 1u);
  *p = (unsigned short)(u >> 16);
}
// NC: no output shares storage with an input, so reads take the read-only path
template <bool NC>
__device__ __forceinline__ void gscl_program_body(const GsclJitParams &P) {
  const long long i = P.lo[0] + (long long)blockIdx.x * 32 + threadIdx.x;
  const long long j = P.lo[1] + (long long)blockIdx.y * 8 + threadIdx.y;
  if (i >= P.hi[0] || j >= P.hi[1]) return;
  bool gscl_bad = false;
  auto gscl_rd = [&](int a, long long k, int dx, int dy, int dz) -> real {
    if (dx < -GSCL_RX || dx > GSCL_RX || dy < -GSCL_RY || dy > GSCL_RY || dz < -GSCL_RZ || dz > GSCL_RZ) {
      gscl_bad = true;
      return (real)0;
    }
    const gscl_stor *p = P.in[a] + k * P.in_plane[a] + j * P.in_pitch[a] + i;
    const long long off = dz * P.in_plane[a] + dy * P.in_pitch[a] + dx;
    if (NC) return gscl_ld(__ldg(p + off));
    return gscl_ld(p[off]);
  };
  // the body at element (i, j, k), its outputs returned through o[]
  auto gscl_eval = [&](long long k, real *gscl_o) {
%s
    real value = 0;
%s
    {
%s
    }
%s
    gscl_o[GSCL_NOUT] = value;
  };
  // this CTA's run of planes, two at a time: both elements' reads are issued
  // before either is stored, and neighbouring planes share their reads in L1
  const long long nz = P.hi[2] - P.lo[2];
  const long long chunk = (nz + gridDim.z - 1) / gridDim.z;
  const long long k0 = P.lo[2] + (long long)blockIdx.z * chunk;
  const long long k1 = k0 + chunk < P.hi[2] ? k0 + chunk : P.hi[2];
  for (long long k = k0; k < k1; k += 2) {
    real oa[GSCL_NOUT + 1], ob[GSCL_NOUT + 1];
    gscl_eval(k, oa);
    const bool two = k + 1 < k1;
    if (two) gscl_eval(k + 1, ob);
%s
    if (P.vout) {
      double *v = P.vout + (k - P.lo[2]) * P.v_plane + (j - P.lo[1]) * P.v_pitch + (i - P.lo[0]);
      v[0] = (double)oa[GSCL_NOUT];
      if (two) v[P.v_plane] = (double)ob[GSCL_NOUT];
    }
  }
  if (gscl_bad) atomicOr(P.err, 2);
}
extern "C" __global__ void __launch_bounds__(256) gscl_program_kernel(const __grid_constant__ GsclJitParams P) {
  gscl_program_body<false>(P);
}
extern "C" __global__ void __launch_bounds__(256) gscl_program_kernel_nc(const __grid_constant__ GsclJitParams P) {
  gscl_program_body<true>(P);
}
// Staged variant: a 64 x 8 tile of core elements per CTA, each input's planes
// with their apron in a shared-memory ring of R slots, copied GSCL_PF planes
// ahead with cp.async (BF16: plain copies); the CTA walks its run of planes.
__device__ __forceinline__ void gscl_cp16(void *s, const void *g) {
  asm volatile("cp.async.cg.shared.global [%%0], [%%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g) : "memory");
}
// Rows are staged in 16-byte vectors: the tile's columns start at a multiple
// of 64 from the interior origin (128-byte aligned), the apron AX is the reach
// rounded up to a vector, so every vector is aligned; a vector is copied when
// it lies within [-c, pitch - c) of its row (c = leading pad + halo, see the
// host), inside the grid's storage whatever its row.
extern "C" __global__ void __launch_bounds__(256) gscl_program_staged(const __grid_constant__ GsclJitParams P) {
  extern __shared__ __align__(16) unsigned char gscl_sm[];
  gscl_stor *ring = reinterpret_cast<gscl_stor *>(gscl_sm);
  constexpr int VEC = 16 / (int)sizeof(gscl_stor);
  constexpr int AX = (GSCL_RX + VEC - 1) / VEC * VEC;
  constexpr int W = 64 + 2 * AX, WV = W / VEC, H = 8 + 2 * GSCL_RY, SLOT = W * H, R = 2 * GSCL_RZ + 1 + GSCL_PF;
  const int tid = threadIdx.y * 32 + threadIdx.x, lane = threadIdx.x, wy = threadIdx.y;
  const long long x0 = P.lo[0] / 64 * 64 + (long long)blockIdx.x * 64, y0 = P.lo[1] + (long long)blockIdx.y * 8;
  const long long nz = P.hi[2] - P.lo[2];
  const long long chunk = (nz + gridDim.z - 1) / gridDim.z;
  const long long k0 = P.lo[2] + (long long)blockIdx.z * chunk;
  const long long k1 = k0 + chunk < P.hi[2] ? k0 + chunk : P.hi[2];
  if (k0 >= k1) return;
  const long long kb = k0 - GSCL_RZ;  // the plane slot 0 held first
  bool gscl_bad = false;
  auto issue = [&](long long kp) {  // copies of plane kp into its slot, one commit group
    if (kp < k1 + GSCL_RZ) {
      const int slot = (int)((kp - kb) %% R);
      for (int a = 0; a < GSCL_NIN; ++a) {
        const gscl_stor *g = P.in[a] + kp * P.in_plane[a];
        gscl_stor *sl = ring + (a * R + slot) * SLOT;
        for (int idx = tid; idx < H * WV; idx += 256) {
          const int row = idx / WV, cv = idx - row * WV;
          const long long x = x0 - AX + cv * VEC, y = y0 - GSCL_RY + row;
          if (x < P.in_x0[a] || x + VEC > P.in_x1[a] || y < P.in_y0[a] || y >= P.in_y1[a]) continue;
          gscl_cp16(sl + row * W + cv * VEC, g + y * P.in_pitch[a] + x);
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // pos: the core element's offset in a slot; sk: the slot of plane k
  auto gscl_rs = [&](int a, int pos, int sk, int dx, int dy, int dz) -> real {
    if (dx < -GSCL_RX || dx > GSCL_RX || dy < -GSCL_RY || dy > GSCL_RY || dz < -GSCL_RZ || dz > GSCL_RZ) {
      gscl_bad = true;
      return (real)0;
    }
    int sl = sk + dz;
    sl = sl >= R ? sl - R : (sl < 0 ? sl + R : sl);
    return gscl_ld(ring[(a * R + sl) * SLOT + pos + dy * W + dx]);
  };
  auto gscl_eval = [&](long long i, long long j, long long k, int gscl_pos, int gscl_sk, real *gscl_o) {
%s
    real value = 0;
%s
    {
%s
    }
%s
    gscl_o[GSCL_NOUT] = value;
  };
  for (long long kp = kb; kp < k0 + GSCL_RZ + GSCL_PF; ++kp) issue(kp);
  for (long long k = k0; k < k1; ++k) {
    asm volatile("cp.async.wait_group %%0;" ::"n"(GSCL_PF - 1) : "memory");  // this thread's copies of plane k + RZ
    __syncthreads();                     // everyone's; and every read of plane k - RZ - 1 is done
    issue(k + GSCL_RZ + GSCL_PF);        // into the slot plane k - RZ - 1 held
    const long long j = y0 + wy;
    const int sk = (int)((k - kb) %% R);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const long long i = x0 + lane + 32 * e;
      if (i >= P.lo[0] && i < P.hi[0] && j < P.hi[1]) {
        real o[GSCL_NOUT + 1];
        gscl_eval(i, j, k, (wy + GSCL_RY) * W + lane + 32 * e + AX, sk, o);
%s
        if (P.vout) P.vout[(k - P.lo[2]) * P.v_plane + (j - P.lo[1]) * P.v_pitch + (i - P.lo[0])] = (double)o[GSCL_NOUT];
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (gscl_bad) atomicOr(P.err, 2);
}
)SRC";

std::string make_source(const char *body, int n_in, int n_out, int dtype, const int32_t reach[3]) {
  std::string defs, decl, ret, stores;
  for (int a = 0; a < n_in; ++a)
    defs += "#define in" + std::to_string(a) + "(dx, dy, dz) gscl_rd(" + std::to_string(a) + ", k, (dx), (dy), (dz))\n";
  for (int m = 0; m < n_out; ++m) {
    const std::string M = std::to_string(m);
    decl += "    real out" + M + " = 0;\n";
    ret += "    gscl_o[" + M + "] = out" + M + ";\n";
    stores += "    gscl_st(P.out[" + M + "] + k * P.out_plane[" + M + "] + j * P.out_pitch[" + M + "] + i, oa[" + M +
              "]);\n    if (two) gscl_st(P.out[" + M + "] + (k + 1) * P.out_plane[" + M + "] + j * P.out_pitch[" + M +
              "] + i, ob[" + M + "]);\n";
  }
  std::string defs_s, undefs, stores_s;
  for (int a = 0; a < n_in; ++a) {
    const std::string A = std::to_string(a);
    undefs += "#undef in" + A + "\n";
    defs_s += "#define in" + A + "(dx, dy, dz) gscl_rs(" + A + ", gscl_pos, gscl_sk, (dx), (dy), (dz))\n";
  }
  for (int m = 0; m < n_out; ++m) {
    const std::string M = std::to_string(m);
    stores_s += "        gscl_st(P.out[" + M + "] + k * P.out_plane[" + M + "] + j * P.out_pitch[" + M + "] + i, o[" + M +
                "]);\n";
  }
  const char *real = dtype == GSCL_F64 ? "double" : "float";
  const char *stor = dtype == GSCL_F64 ? "double" : dtype == GSCL_F32 ? "float" : "unsigned short";
  // the generated struct has fixed-size arrays like JitParams
  std::vector<char> buf(strlen(kJitTemplate) + 2 * (defs.size() + decl.size() + strlen(body) + ret.size()) +
                        stores.size() + stores_s.size() + undefs.size() + defs_s.size() + 1024);
  const std::string defs2 = undefs + defs_s;
  snprintf(buf.data(), buf.size(), kJitTemplate, real, stor, reach[0], reach[1], reach[2], n_in, n_out, kMaxIn,
           kMaxIn, kMaxIn, kMaxIn, kMaxIn, kMaxIn, kMaxIn, kMaxOut_, kMaxOut_, kMaxOut_, defs.c_str(), decl.c_str(),
           body, ret.c_str(), stores.c_str(), defs2.c_str(), decl.c_str(), body, ret.c_str(), stores_s.c_str());
  return std::string(buf.data());
}

// ------------------------------------------------------------------ program registry
struct Program {
  int n_in = 0, n_out = 0, dtype = 0;
  int32_t reach[3] = {0, 0, 0};
  std::vector<char> cubin;
  std::map<int, CUfunction> fn, fn_nc, fn_st;  // per device: plain reads / read-only path / staged
  std::map<int, CUmodule> mod;
};

std::mutex g_prog_mu;
std::map<uint64_t, Program> g_progs;
uint64_t g_prog_next = 1;
std::map<std::string, std::vector<char>> g_cubins;  // generated source -> its cubin (compile once per process)

// kind: 0 plain reads, 1 read-only path, 2 staged in shared memory
// GSCL_PROGRAM_STAGED=0 keeps every launch on the plain kernels.
bool staged_enabled() {
  const char *e = getenv("GSCL_PROGRAM_STAGED");
  return !(e && e[0] == '0');
}

CUfunction program_function(Program &p, int kind, gscl_status *st) {
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = p.fn.find(dev);
  if (it != p.fn.end()) return kind == 2 ? p.fn_st[dev] : kind == 1 ? p.fn_nc[dev] : it->second;
  const Driver &d = driver();
  if (!d.ok) {
    *st = fail(GSCL_ERR_CUDA, "the driver's module functions are not available");
    return nullptr;
  }
  cudaFree(nullptr);  // the runtime's context is current on this thread
  CUmodule m = nullptr;
  CUresult r = d.load(&m, p.cubin.data());
  if (r != CUDA_SUCCESS) {
    *st = fail(GSCL_ERR_CUDA, "loading the compiled operator failed (%d)", (int)r);
    return nullptr;
  }
  CUfunction f = nullptr, fnc = nullptr, fst = nullptr;
  r = d.get(&f, m, "gscl_program_kernel");
  if (r == CUDA_SUCCESS) r = d.get(&fnc, m, "gscl_program_kernel_nc");
  if (r == CUDA_SUCCESS) r = d.get(&fst, m, "gscl_program_staged");
  if (r != CUDA_SUCCESS) {
    d.unload(m);
    *st = fail(GSCL_ERR_CUDA, "the compiled operator has no kernel (%d)", (int)r);
    return nullptr;
  }
  p.mod[dev] = m;
  p.fn[dev] = f;
  p.fn_nc[dev] = fnc;
  p.fn_st[dev] = fst;
  return kind == 2 ? fst : kind == 1 ? fnc : f;
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" gscl_status gscl_program_create(const char *body, int32_t n_in, int32_t n_out, int32_t dtype,
                                           const int32_t reach[3], gscl_program *out) {
  if (!body || !out || !reach) return fail(GSCL_ERR_INVALID, "body, reach and out are required");
  if (n_in < 1 || n_in > kMaxIn) return fail(GSCL_ERR_UNSUPPORTED, "n_in = %d outside [1, %d]", n_in, kMaxIn);
  if (n_out < 0 || n_out > kMaxOut_) return fail(GSCL_ERR_UNSUPPORTED, "n_out = %d outside [0, %d]", n_out, kMaxOut_);
  if (dtype != GSCL_F64 && dtype != GSCL_F32 && dtype != GSCL_BF16) return fail(GSCL_ERR_DTYPE, "unknown dtype");
  for (int a = 0; a < 3; ++a)
    if (reach[a] < 0 || reach[a] > 64) return fail(GSCL_ERR_INVALID, "reach[%d] = %d outside [0, 64]", a, reach[a]);
  const Nvrtc &nv = nvrtc();
  if (!nv.ok) return fail(GSCL_ERR_UNSUPPORTED, "NVRTC (libnvrtc.so) is not available");
  const std::string src = make_source(body, n_in, n_out, dtype, reach);
  Program p;
  p.n_in = n_in;
  p.n_out = n_out;
  p.dtype = dtype;
  for (int a = 0; a < 3; ++a) p.reach[a] = reach[a];
  {
    std::lock_guard<std::mutex> lk(g_prog_mu);
    auto c = g_cubins.find(src);
    if (c != g_cubins.end()) {
      p.cubin = c->second;
      const uint64_t h = g_prog_next++;
      g_progs[h] = std::move(p);
      *out = h;
      return GSCL_OK;
    }
  }
  nvrtcProgram prog = nullptr;
  if (nv.create(&prog, src.c_str(), "gscl_program.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return fail(GSCL_ERR_INVALID, "NVRTC could not create the program");
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "--diag-suppress=177,550"};
  const nvrtcResult cr = nv.compile(prog, 4, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t n = 0;
    nv.log_size(prog, &n);
    std::string log(n + 1, '\0');
    if (n) nv.log(prog, &log[0]);
    nv.destroy(&prog);
    return fail(GSCL_ERR_INVALID, "the operator did not compile: %s", log.c_str());
  }
  size_t n = 0;
  nv.cubin_size(prog, &n);
  p.cubin.resize(n);
  nv.cubin(prog, p.cubin.data());
  nv.destroy(&prog);
  std::lock_guard<std::mutex> lk(g_prog_mu);
  g_cubins[src] = p.cubin;
  const uint64_t h = g_prog_next++;
  g_progs[h] = std::move(p);
  *out = h;
  return GSCL_OK;
}

extern "C" gscl_status gscl_program_destroy(gscl_program h) {
  std::lock_guard<std::mutex> lk(g_prog_mu);
  auto it = g_progs.find(h);
  if (it == g_progs.end()) return fail(GSCL_ERR_STATE, "no such program");
  const Driver &d = driver();
  if (d.ok) {
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &m : it->second.mod) {
      cudaSetDevice(m.first);
      d.unload(m.second);
    }
    cudaSetDevice(cur);
  }
  g_progs.erase(it);
  return GSCL_OK;
}

namespace gscl {
namespace {

// The program over the range `sweeps` times (do_all); with vout, one sweep
// that also stores the body's value at every core element of the range into
// the dense FP64 array vout (rows of v_pitch, planes of v_plane elements).
gscl_status run_program(gscl_program h, const gscl_grid *in, int32_t n_in, const gscl_grid *out, int32_t n_out,
                        const gscl_range *range, int32_t sweeps, void *stream, double *vout, long long v_pitch,
                        long long v_plane, Bound *bound_out) {
  if (sweeps < 1) return fail(GSCL_ERR_INVALID, "sweeps must be >= 1");
  std::lock_guard<std::mutex> lk(g_prog_mu);
  auto it = g_progs.find(h);
  if (it == g_progs.end()) return fail(GSCL_ERR_STATE, "no such program");
  Program &p = it->second;
  if (n_in != p.n_in || n_out != p.n_out)
    return fail(GSCL_ERR_INVALID, "the program was compiled for %d inputs and %d outputs", p.n_in, p.n_out);
  // bind with the corners of the declared reach of every input: the range and
  // halo checks, and the alias rule (an output may be an input only with reach 0)
  std::vector<gscl_term> terms;
  for (int a = 0; a < n_in; ++a)
    for (int s = -1; s <= 1; s += 2)
      terms.push_back(gscl_term{(int8_t)(s * p.reach[0]), (int8_t)(s * p.reach[1]), (int8_t)(s * p.reach[2]),
                                (uint8_t)a, GSCL_NONE, GSCL_VALUE, 0, 0.0});
  gscl_stencil st{(int32_t)terms.size(), 0, terms.data()};
  Bound b;
  if (gscl_status s = bind(&st, false, in, n_in, out, n_out, range, &b)) return s;
  if (b.in[0].dtype != p.dtype) return fail(GSCL_ERR_DTYPE, "the program was compiled for another dtype");
  if (bound_out) *bound_out = b;
  if (b.empty || (vout && v_pitch == 0)) return GSCL_OK;
  if (sweeps > 1) {
    if (n_out < 1) return fail(GSCL_ERR_INVALID, "multi-sweep ping-pong needs an output");
    const Grid &a = b.in[0], &c = b.out[0];
    if (a.halo[0] != c.halo[0] || a.halo[1] != c.halo[1] || a.halo[2] != c.halo[2])
      return fail(GSCL_ERR_SHAPE, "multi-sweep ping-pong needs in[0] and out[0] of identical layout");
    if (overlaps(a, c)) return fail(GSCL_ERR_ALIAS, "multi-sweep ping-pong needs distinct in[0] and out[0]");
  }
  bool shared = false;  // an output is also an input (reach 0, point-wise in place)
  for (int m = 0; m < n_out; ++m)
    for (int a = 0; a < n_in; ++a) shared |= overlaps(b.out[m], b.in[a]);
  // the staged kernel for FP32 / BF16 grids when its shared-memory ring fits
  // and no output is an input (the ring would hold a copy older than this
  // element's write).  FP64 sweeps are bound by the FP64 pipe, where the plain
  // kernel's extra warps win (0.291 against 0.333 ms per 256^3 heat sweep).
  const int elem = b.in[0].elem;
  const int vec = 16 / elem, ax = (p.reach[0] + vec - 1) / vec * vec;
  const size_t ring_bytes = (size_t)n_in * (2 * p.reach[2] + 3) * (64 + 2 * ax) * (8 + 2 * p.reach[1]) * elem;
  const bool staged = !shared && elem <= 4 && ring_bytes <= 200 * 1024 && staged_enabled();
  gscl_status fst = GSCL_OK;
  CUfunction f = program_function(p, staged ? 2 : shared ? 0 : 1, &fst);
  if (!f) return fst;
  if (staged) {
    CUresult ra = driver().set_attr(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)ring_bytes);
    if (ra != CUDA_SUCCESS) return fail(GSCL_ERR_CUDA, "shared memory for the compiled operator (%d)", (int)ra);
  }
  int *err = device_error_word();
  if (!err) return fail(GSCL_ERR_CUDA, "device error word unavailable");
  JitParams P;
  memset(&P, 0, sizeof P);
  for (int a = 0; a < n_in; ++a) {
    const Grid &g = b.in[a];
    P.in_pitch[a] = g.pitch;
    P.in_plane[a] = g.plane;
    // the staged kernel's vectors: [-c, pitch - c) of a row, c = leading pad + halo
    P.in_x0[a] = -(g.off + g.halo[0]);
    P.in_x1[a] = g.pitch - (g.off + g.halo[0]);
    P.in_y0[a] = -g.halo[1];
    P.in_y1[a] = g.n[1] + g.halo[1];
  }
  for (int m = 0; m < n_out; ++m) {
    P.out_pitch[m] = b.out[m].pitch;
    P.out_plane[m] = b.out[m].plane;
  }
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = b.lo[a];
    P.hi[a] = b.hi[a];
  }
  P.err = err;
  P.vout = vout;
  P.v_pitch = v_pitch;
  P.v_plane = v_plane;
  const long long nx = b.hi[0] - b.lo[0], ny = b.hi[1] - b.lo[1], nz = b.hi[2] - b.lo[2];
  const long long xspan = staged ? b.hi[0] - b.lo[0] / 64 * 64 : nx;  // staged tiles start at a multiple of 64
  const unsigned gx = (unsigned)((xspan + (staged ? 63 : 31)) / (staged ? 64 : 32)), gy = (unsigned)((ny + 7) / 8);
  // CTAs of 256 threads: 8 per SM, or as many as the staged rings fit; the
  // staged kernel keeps runs of at least 8 planes (each run reloads its z halo)
  const long long per_sm = staged ? std::max<long long>(1, std::min<long long>(8, (227 * 1024) / (long long)ring_bytes)) : 8;
  const long long target = (long long)sm_count() * per_sm;
  const long long zmax = staged ? std::max(1LL, nz / 8) : nz;
  const unsigned gz = (unsigned)std::max(1LL, std::min(zmax, (target + gx * gy - 1) / ((long long)gx * gy)));
  if (gy > 65535 || gz > 65535) return fail(GSCL_ERR_UNSUPPORTED, "range too large for one launch");
  const Driver &d = driver();
  Grid src = b.in[0], dst;  // ping-pong pair in[0] / out[0] (no output: in[0] alone)
  if (n_out > 0) dst = b.out[0];
  for (int s = 0; s < sweeps; ++s) {
    for (int a = 0; a < n_in; ++a) P.in[a] = b.in[a].elem_ptr(0, 0, 0);
    for (int m = 0; m < n_out; ++m) P.out[m] = b.out[m].elem_ptr(0, 0, 0);
    P.in[0] = src.elem_ptr(0, 0, 0);
    for (int a = 1; a < n_in; ++a)  // another input naming the ping-pong grid follows it
      if (b.in_h[a] == b.in_h[0]) P.in[a] = src.elem_ptr(0, 0, 0);
    if (n_out > 0) P.out[0] = dst.elem_ptr(0, 0, 0);
    void *args[] = {&P};
    CUresult r = d.launch(f, gx, gy, gz, 32, 8, 1, staged ? (unsigned)ring_bytes : 0, (CUstream)stream, args, nullptr);
    if (r != CUDA_SUCCESS) return fail(GSCL_ERR_CUDA, "launching the compiled operator failed (%d)", (int)r);
    std::swap(src, dst);
  }
  if (sweeps > 1 && sweeps % 2 == 0) return swap_storage(in[0], out[0]);
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

extern "C" gscl_status gscl_do_all_program(gscl_program h, const gscl_grid *in, int32_t n_in, const gscl_grid *out,
                                           int32_t n_out, const gscl_range *range, int32_t sweeps, void *stream) {
  if (n_out < 1) return fail(GSCL_ERR_INVALID, "do_all needs at least one output");
  return run_program(h, in, n_in, out, n_out, range, sweeps, stream, nullptr, 0, 0, nullptr);
}

extern "C" gscl_status gscl_do_reduce_program(gscl_program h, int32_t reduce_op, const gscl_grid *in, int32_t n_in,
                                              const gscl_grid *out, int32_t n_out, const gscl_range *range,
                                              double *result, int32_t result_on_host, void *workspace,
                                              int64_t workspace_bytes, void *stream) {
  if (!result) return fail(GSCL_ERR_INVALID, "result is NULL");
  if (reduce_op != GSCL_SUM && reduce_op != GSCL_MAXABS && reduce_op != GSCL_L2)
    return fail(GSCL_ERR_INVALID, "unknown reduce op %d", reduce_op);
  // validate first (no launch), then size the value array on the range
  Bound b;
  if (gscl_status s = run_program(h, in, n_in, out, n_out, range, 1, stream, (double *)1, 0, 0, &b)) return s;
  const int64_t ext[3] = {std::max<int64_t>(1, b.hi[0] - b.lo[0]), std::max<int64_t>(1, b.hi[1] - b.lo[1]),
                          std::max<int64_t>(1, b.hi[2] - b.lo[2])};
  const int32_t nohalo[3] = {0, 0, 0};
  int64_t pitch = 0, off = 0, bytes = 0;
  if (gscl_status s = gscl_grid_layout(3, ext, nohalo, GSCL_F64, &pitch, &off, &bytes)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  void *buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, (size_t)bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync of the value array");
  gscl_grid vg = 0;
  gscl_status s = gscl_grid_create(3, ext, nohalo, GSCL_F64, buf, bytes, &vg);
  if (s == GSCL_OK) {
    double *vout = (double *)buf + off;
    if (b.empty) {
      // an empty range: reduce nothing (the value array is not read)
      gscl_range none = {{0, 0, 0}, {0, 0, 0}};
      s = gscl_do_reduce(reduce_op, nullptr, &vg, 1, nullptr, 0, &none, result, result_on_host, workspace,
                         workspace_bytes, stream);
    } else {
      s = run_program(h, in, n_in, out, n_out, range, 1, stream, vout, pitch, pitch * ext[1], nullptr);
      if (s == GSCL_OK)
        s = gscl_do_reduce(reduce_op, nullptr, &vg, 1, nullptr, 0, nullptr, result, result_on_host, workspace,
                           workspace_bytes, stream);
    }
    gscl_grid_destroy(vg);
  }
  cudaFreeAsync(buf, st);
  return s;
}
