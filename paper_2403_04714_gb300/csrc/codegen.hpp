// codegen.hpp -- generated-CUDA lowering and its run-time compilation.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "compiler.hpp"

namespace rtl {

struct GenUnit {
    std::string name, source;
};

// CUDA sources for every process (in n_chunks units) plus the dispatcher and
// the kernels rtl_gen_d0 / rtl_gen_d1 (digests off / on) for lane mapping `mode`.
int gen_cuda(const Netlist& nl, const Partition& part, int mode, int n_chunks, std::vector<GenUnit>& out,
             std::string& err);
void gen_process(const Netlist& nl, const Partition& part, const RegLayout& L, size_t p, int mode, std::string& o);

// A loaded generated module.
struct GenModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel[2] = {nullptr, nullptr};   // [digest]
    double compile_seconds = 0;
    bool cached = false;
};

// Compile the units with NVRTC (relocatable cubins, in parallel) and link them
// with nvJitLink (no GPU needed).  Linked cubins are cached on disk under
// `cache_dir` (empty: no cache) by a hash of the sources and options.
int jit_compile(const std::vector<GenUnit>& units, const std::string& cache_dir, std::vector<char>& linked,
                bool* cached, double* seconds, std::string& err);
// Load a linked cubin on the current device and look up its kernels.
int jit_load(const std::vector<char>& linked, GenModule& out, std::string& err);
void jit_unload(GenModule& m);

}  // namespace rtl
