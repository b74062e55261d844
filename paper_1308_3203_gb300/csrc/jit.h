// Compiled intervals (jit.cu): per-program interval kernels built at run
// time with NVRTC from the translated bytecode and the compiled engine.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bytecode.h"
#include "kernel_types.cuh"

namespace rc {

struct JitError {
  std::string msg;
};

// What one interval kernel is compiled for.
struct JitShape {
  bool resident = false;    // one cooperative launch runs every interval
  uint32_t threads = 1024;  // __launch_bounds__: the group size
  uint32_t min_blocks = 1;  //   and the CTAs that must fit on one SM
  bool load = true;         // load the cubin (false: compile only, no device needed)
};

struct JitKernel {
  const void *fn = nullptr;  // a cudaKernel_t, usable wherever the runtime takes a kernel
  size_t static_smem = 0;
  uint32_t regs = 0;
  size_t local_bytes = 0;    // spill / stack bytes per thread
  size_t cubin_bytes = 0;
};

// NVRTC can be loaded (why: the reason when not).
bool jit_available(std::string *why);
// The kernel source of `code` (the program's bytecode, CTL_PRIV marking the
// private accesses of the launch shape) for `shape`.
std::string jit_source(const Program &P, const std::vector<Insn> &code, const JitShape &shape);
// Compiled (or cached) kernel; throws JitError.
JitKernel jit_kernel(const Program &P, const std::vector<Insn> &code, const JitShape &shape);
void jit_stats(uint64_t *compiles, double *seconds);
void launch_jit(const JitKernel &k, const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s);
cudaError_t launch_jit_resident(const JitKernel &k, const InterpArgs &a, uint32_t n_groups, size_t smem,
                                cudaStream_t s);
int jit_blocks_per_sm(const JitKernel &k, uint32_t S, size_t smem);

}  // namespace rc
