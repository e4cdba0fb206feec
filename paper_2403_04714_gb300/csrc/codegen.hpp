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
// one kernel for lane mapping `mode`: rtl_gen_d1 with the per-cycle digest
// code in every process function, or rtl_gen_d0 without any (its process
// functions are that much shorter, which the instruction caches feel).
int gen_cuda(const Netlist& nl, const Partition& part, int mode, bool digest, int n_chunks, std::vector<GenUnit>& out,
             std::string& err);
void gen_process(const Netlist& nl, const Partition& part, const RegLayout& L, size_t p, int mode, bool digest,
                 std::string& o);

// A loaded generated module.
struct GenModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;                 // rtl_gen_d0 or rtl_gen_d1
    double compile_seconds = 0;
    bool cached = false;
};

// Compile the units with NVRTC (relocatable cubins, in parallel) and link them
// with nvJitLink (no GPU needed).  Linked cubins are cached on disk under
// `cache_dir` (empty: no cache) by a hash of the sources and options.
int jit_compile(const std::vector<GenUnit>& units, const std::string& cache_dir, std::vector<char>& linked,
                bool* cached, double* seconds, std::string& err);
// Load a linked cubin on the current device and look up its kernel.
int jit_load(const std::vector<char>& linked, bool digest, GenModule& out, std::string& err);
void jit_unload(GenModule& m);

}  // namespace rtl
