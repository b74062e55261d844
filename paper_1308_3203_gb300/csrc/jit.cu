// Compiled intervals: a program's bytecode translated to straight-line code
// (translate.cpp) and compiled at run time into its own interval kernel,
// whose body is the interpreter kernel's (interp_kernel.cuh) with the
// compiled engine (jit_engine.cuh) in place of the bytecode interpreter.
//
// The source is the engine's headers (embedded into the library at build
// time), the translated function and a table of the access sites the
// pre-filter proved private for the launch shape (so a private access
// compiles to no log append at all).  NVRTC turns it into an sm_103a cubin;
// cudaLibraryLoadData loads it.  Kernels are cached by their source text:
// one compile (a fraction of a second) per program, launch shape and mode,
// however many checks follow.  NVRTC is loaded with dlopen on first use;
// without it the library keeps to the interpreter.
#include <dlfcn.h>

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvrtc.h>

#include "device.cuh"
#include "jit.h"

namespace rc {

std::string translate_program(const Program &p, const std::string &fn_name);

namespace {

#include "jit_headers.inc"  // kJitHeaderNames, kJitHeaderTexts, kJitHeaderCount (written by build.py)

struct Nvrtc {
  bool tried = false, ok = false;
  std::string why;
  nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
  nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
  nvrtcResult (*log_size)(nvrtcProgram, size_t *);
  nvrtcResult (*log)(nvrtcProgram, char *);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
  nvrtcResult (*cubin)(nvrtcProgram, char *);
  nvrtcResult (*destroy)(nvrtcProgram *);
  const char *(*err)(nvrtcResult);
};

Nvrtc g_nvrtc;
std::mutex g_jit_mu;
std::map<std::string, JitKernel> g_jit_cache;
double g_jit_seconds = 0;
uint64_t g_jit_compiles = 0;

bool load_nvrtc(Nvrtc &n) {
  if (n.tried) return n.ok;
  n.tried = true;
  std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
  if (const char *h = std::getenv("CUDA_HOME")) names.push_back(std::string(h) + "/lib64/libnvrtc.so.13");
  names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
  void *h = nullptr;
  for (const std::string &nm : names)
    if ((h = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) {
    n.why = "NVRTC (libnvrtc.so.13) not found";
    return false;
  }
  auto sym = [&](const char *s) { return dlsym(h, s); };
  n.create = reinterpret_cast<decltype(n.create)>(sym("nvrtcCreateProgram"));
  n.compile = reinterpret_cast<decltype(n.compile)>(sym("nvrtcCompileProgram"));
  n.log_size = reinterpret_cast<decltype(n.log_size)>(sym("nvrtcGetProgramLogSize"));
  n.log = reinterpret_cast<decltype(n.log)>(sym("nvrtcGetProgramLog"));
  n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(sym("nvrtcGetCUBINSize"));
  n.cubin = reinterpret_cast<decltype(n.cubin)>(sym("nvrtcGetCUBIN"));
  n.destroy = reinterpret_cast<decltype(n.destroy)>(sym("nvrtcDestroyProgram"));
  n.err = reinterpret_cast<decltype(n.err)>(sym("nvrtcGetErrorString"));
  n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy && n.err;
  if (!n.ok) n.why = "NVRTC is missing entry points";
  return n.ok;
}

void emit(std::string &o, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void emit(std::string &o, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  o += buf;
}

}  // namespace

std::string jit_source(const Program &P, const std::vector<Insn> &code, const JitShape &shape) {
  std::string o;
  o += "#ifdef __CUDACC_RTC__\n"
       "typedef signed char int8_t; typedef unsigned char uint8_t; typedef short int16_t;\n"
       "typedef unsigned short uint16_t; typedef int int32_t; typedef unsigned int uint32_t;\n"
       "typedef long long int64_t; typedef unsigned long long uint64_t;\n"
       "#define INT32_MIN (-2147483647 - 1)\n"
       "#endif\n"
       "#include \"jit_engine.cuh\"\n";
  // the pre-filter's private access sites for this launch shape (bytecode order)
  o += "__host__ __device__ constexpr bool rc_jit_private(unsigned site) {\n  switch (site) {\n";
  uint32_t site = 0, n_priv = 0;
  for (const Insn &in : code) {
    if (in.op != OP_LD && in.op != OP_ST) continue;
    if (in.ctl & CTL_PRIV) {
      emit(o, "    case %u:\n", site);
      n_priv++;
    }
    site++;
  }
  o += n_priv ? "      return true;\n" : "";
  o += "    default:\n      return false;\n  }\n}\n";
  o += translate_program(P, "rc_jit_run");
  emit(o,
       "struct RcJitProgram {\n"
       "  static constexpr uint32_t kRegs = %u;\n"
       "  template <bool kRes>\n"
       "  __device__ __forceinline__ static void run(::rc::JitCtx<kRes> &cx, int32_t (&r)[%u], uint32_t &pc,\n"
       "                                             uint32_t &st) {\n"
       "    rc_jit_run<kRes>(cx, r, pc, st);\n"
       "  }\n"
       "};\n",
       P.n_regs, P.n_regs);
  emit(o,
       "extern \"C\" __global__ void __launch_bounds__(%u, %u) rc_jit_kernel(::rc::InterpArgs A) {\n"
       "  ::rc::interp_body<%s>(A, ::rc::JitEngine<%s, RcJitProgram>{});\n"
       "}\n",
       shape.threads, shape.min_blocks, shape.resident ? "true" : "false", shape.resident ? "true" : "false");
  return o;
}

bool jit_available(std::string *why) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  const bool ok = load_nvrtc(g_nvrtc);
  if (!ok && why) *why = g_nvrtc.why;
  return ok;
}

// Compile (or find in the cache) the interval kernel of `code` (P's bytecode
// with the private flags of this launch shape) for one launch shape and mode.
JitKernel jit_kernel(const Program &P, const std::vector<Insn> &code, const JitShape &shape) {
  const std::string src = jit_source(P, code, shape);
  const std::string key = (shape.load ? "L" : "C") + src;  // compile-only entries hold no kernel
  std::lock_guard<std::mutex> lk(g_jit_mu);
  auto it = g_jit_cache.find(key);
  if (it != g_jit_cache.end()) return it->second;
  if (!load_nvrtc(g_nvrtc)) throw JitError{g_nvrtc.why};
  const auto t0 = std::chrono::steady_clock::now();
  nvrtcProgram prog = nullptr;
  nvrtcResult r = g_nvrtc.create(&prog, src.c_str(), "rc_jit.cu", (int)kJitHeaderCount, kJitHeaderTexts,
                                 kJitHeaderNames);
  if (r != NVRTC_SUCCESS) throw JitError{std::string("nvrtcCreateProgram: ") + g_nvrtc.err(r)};
  struct Guard {
    Nvrtc &n;
    nvrtcProgram &p;
    ~Guard() {
      if (p) n.destroy(&p);
    }
  } guard{g_nvrtc, prog};
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-DNDEBUG"};
  r = g_nvrtc.compile(prog, 3, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    g_nvrtc.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) g_nvrtc.log(prog, &log[0]);
    throw JitError{std::string("NVRTC compile of the interval kernel failed: ") + g_nvrtc.err(r) + "\n" +
                   log.substr(0, 4000)};
  }
  size_t nb = 0;
  if (g_nvrtc.cubin_size(prog, &nb) != NVRTC_SUCCESS || nb == 0) throw JitError{"NVRTC returned no cubin"};
  std::vector<char> cubin(nb);
  if (g_nvrtc.cubin(prog, cubin.data()) != NVRTC_SUCCESS) throw JitError{"NVRTC returned no cubin"};
  JitKernel k;
  k.cubin_bytes = nb;
  if (shape.load) {
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) throw JitError{std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e)};
    cudaKernel_t kern = nullptr;
    e = cudaLibraryGetKernel(&kern, lib, "rc_jit_kernel");
    if (e != cudaSuccess) throw JitError{std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e)};
    k.fn = reinterpret_cast<const void *>(kern);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k.fn);
    if (e != cudaSuccess) throw JitError{std::string("cudaFuncGetAttributes: ") + cudaGetErrorString(e)};
    k.static_smem = fa.sharedSizeBytes;
    k.regs = (uint32_t)fa.numRegs;
    k.local_bytes = fa.localSizeBytes;
    e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kMaxSmemPerBlock - k.static_smem));
    if (e != cudaSuccess) throw JitError{std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e)};
  }
  g_jit_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  g_jit_compiles++;
  g_jit_cache.emplace(key, k);
  return k;
}

void jit_stats(uint64_t *compiles, double *seconds) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  *compiles = g_jit_compiles;
  *seconds = g_jit_seconds;
}

void launch_jit(const JitKernel &k, const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s) {
  count_launch();
  InterpArgs arg = a;
  void *params[] = {&arg};
  const uint32_t split = a.split > 1 ? a.split : 1;  // CTAs per work-group
  const cudaError_t e = cudaLaunchKernel(k.fn, dim3(n_groups * split), dim3(a.S / split), params, smem, s);
  if (e != cudaSuccess) throw JitError{std::string("launch of a compiled interval kernel: ") + cudaGetErrorString(e)};
}

cudaError_t launch_jit_resident(const JitKernel &k, const InterpArgs &a, uint32_t n_groups, size_t smem,
                                cudaStream_t s) {
  count_launch();
  InterpArgs arg = a;
  void *params[] = {&arg};
  return cudaLaunchCooperativeKernel(k.fn, dim3(n_groups), dim3(a.S), params, smem, s);
}

int jit_blocks_per_sm(const JitKernel &k, uint32_t S, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, (int)S, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace rc
