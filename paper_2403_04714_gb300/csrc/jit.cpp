// jit.cpp -- run-time compilation of generated CUDA (NVRTC + nvJitLink).
//
// Each generated unit is compiled by NVRTC to a relocatable sm_103a cubin on
// its own thread; nvJitLink links them into one module (one kernel can then
// call every process function, which the grid barrier needs), and the module
// is loaded with cudaLibraryLoadData.  Linked modules are cached on disk by a
// hash of every source and option.
#include <nvJitLink.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <thread>

#include "../../include/sim.h"
#include "codegen.hpp"

namespace rtl {

extern const char* const kEmbeddedAbiHeader;   // abi_device.h (embedded at build time)
extern const char* const kEmbeddedRtHeader;    // sim_rt.cuh

namespace {

const char* const kArch = "sm_103a";

uint64_t fnv1a(uint64_t h, const std::string& s) {
    for (unsigned char c : s) {
        h ^= c;
        h *= 0x100000001B3ULL;
    }
    return h;
}

bool read_file(const std::string& path, std::vector<char>& out) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    out.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
    return !out.empty();
}

void write_file(const std::string& path, const std::vector<char>& data) {
    std::string tmp = path + ".tmp" + std::to_string(uint64_t(std::hash<std::thread::id>()(std::this_thread::get_id())));
    {
        std::ofstream f(tmp, std::ios::binary);
        if (!f) return;
        f.write(data.data(), std::streamsize(data.size()));
    }
    std::rename(tmp.c_str(), path.c_str());
}

// Registers per thread for generated code.  Process functions with many live
// values would otherwise claim up to 255 registers and hold one 256-thread
// CTA per SM.  Measured on the 200k-op netlist with 4,096 instances (8-warp
// CTAs): uncapped 3.6M instance-cycles/s; 64 registers (4 CTAs per SM) 6.9M;
// 80 (3 CTAs) 7.5M; 96 and 128 (2 CTAs) 4.8-5.0M.  Spills fall from 1.9 GB
// to 1.3 GB of local traffic per simulated cycle between 64 and 80.
std::string max_registers() {
    const char* m = getenv("RTLSIM_GEN_MAXRREG");
    return m ? m : "80";
}

// The kernel entry's launch bound must leave every process function its
// register cap: the largest CTA, in groups of 4 warps (one per SM
// sub-partition), whose threads x cap fit the 65,536-register file.
int max_threads() {
    const int cap = std::max(16, std::min(255, atoi(max_registers().c_str())));
    return std::max(128, std::min(1024, 65536 / (cap * 128) * 128));
}

int compile_unit(const GenUnit& u, std::vector<char>& cubin, std::string& err) {
    nvrtcProgram prog;
    const char* hdr[2] = {kEmbeddedAbiHeader, kEmbeddedRtHeader};
    const char* hdr_names[2] = {"abi_device.h", "sim_rt.cuh"};
    if (nvrtcCreateProgram(&prog, u.source.c_str(), u.name.c_str(), 2, hdr, hdr_names) != NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed for " + u.name;
        return SIM_ERR_CUDA;
    }
    std::string arch = std::string("--gpu-architecture=") + kArch;
    std::vector<const char*> opts = {arch.c_str(), "-rdc=true", "--std=c++17", "-default-device", "-w"};
    std::string maxr = "--maxrregcount=" + max_registers();
    opts.push_back(maxr.c_str());
    std::string thr = "-DRTLSIM_GEN_MAX_THREADS=" + std::to_string(max_threads());
    opts.push_back(thr.c_str());
    nvrtcResult r = nvrtcCompileProgram(prog, int(opts.size()), opts.data());
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        err = "NVRTC " + u.name + ": " + nvrtcGetErrorString(r) + "\n" + log.substr(0, 4000);
        nvrtcDestroyProgram(&prog);
        return SIM_ERR_CUDA;
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin.resize(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    return SIM_OK;
}

int link_units(const std::vector<std::vector<char>>& cubins, const std::vector<GenUnit>& units, std::vector<char>& out,
               std::string& err) {
    nvJitLinkHandle h;
    std::string arch = std::string("-arch=") + kArch;
    const char* lopts[] = {arch.c_str()};
    if (nvJitLinkCreate(&h, 1, lopts) != NVJITLINK_SUCCESS) {
        err = "nvJitLinkCreate failed";
        return SIM_ERR_CUDA;
    }
    auto fail = [&](const char* what) {
        size_t n = 0;
        nvJitLinkGetErrorLogSize(h, &n);
        std::string log(n, '\0');
        if (n) nvJitLinkGetErrorLog(h, &log[0]);
        err = std::string("nvJitLink ") + what + ": " + log.substr(0, 4000);
        nvJitLinkDestroy(&h);
        return SIM_ERR_CUDA;
    };
    for (size_t i = 0; i < cubins.size(); i++)
        if (nvJitLinkAddData(h, NVJITLINK_INPUT_CUBIN, cubins[i].data(), cubins[i].size(), units[i].name.c_str()) !=
            NVJITLINK_SUCCESS)
            return fail("add");
    if (nvJitLinkComplete(h) != NVJITLINK_SUCCESS) return fail("link");
    size_t n = 0;
    nvJitLinkGetLinkedCubinSize(h, &n);
    out.resize(n);
    nvJitLinkGetLinkedCubin(h, out.data());
    nvJitLinkDestroy(&h);
    return SIM_OK;
}

}  // namespace

int jit_compile(const std::vector<GenUnit>& units, const std::string& cache_dir, std::vector<char>& linked,
                bool* cached, double* seconds, std::string& err) {
    auto t0 = std::chrono::steady_clock::now();
    uint64_t h = 0xcbf29ce484222325ULL;
    h = fnv1a(h, kArch);
    h = fnv1a(h, "maxrreg=" + max_registers() + " threads=" + std::to_string(max_threads()));
    h = fnv1a(h, kEmbeddedAbiHeader);
    h = fnv1a(h, kEmbeddedRtHeader);
    for (auto& u : units) h = fnv1a(fnv1a(h, u.name), u.source);
    char hex[32];
    snprintf(hex, sizeof hex, "%016llx", (unsigned long long)h);
    std::string path = cache_dir.empty() ? std::string() : cache_dir + "/rtl_" + hex + ".cubin";
    *cached = !path.empty() && read_file(path, linked);
    if (!*cached) {
        std::vector<std::vector<char>> cubins(units.size());
        std::vector<std::string> errs(units.size());
        std::vector<int> rcs(units.size(), SIM_OK);
        std::atomic<size_t> next{0};
        unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), unsigned(units.size())));
        std::vector<std::thread> th;
        for (unsigned k = 0; k < nt; k++)
            th.emplace_back([&] {
                for (size_t i; (i = next.fetch_add(1)) < units.size();) rcs[i] = compile_unit(units[i], cubins[i], errs[i]);
            });
        for (auto& t : th) t.join();
        for (size_t i = 0; i < units.size(); i++)
            if (rcs[i]) {
                err = errs[i];
                return rcs[i];
            }
        int rc = link_units(cubins, units, linked, err);
        if (rc) return rc;
        if (!path.empty()) write_file(path, linked);
    }
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SIM_OK;
}

int jit_load(const std::vector<char>& linked, bool digest, GenModule& out, std::string& err) {
    cudaError_t e = cudaLibraryLoadData(&out.lib, linked.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
        return SIM_ERR_CUDA;
    }
    e = cudaLibraryGetKernel(&out.kernel, out.lib, digest ? "rtl_gen_d1" : "rtl_gen_d0");
    if (e != cudaSuccess) {
        err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
        cudaLibraryUnload(out.lib);
        out.lib = nullptr;
        return SIM_ERR_CUDA;
    }
    return SIM_OK;
}

void jit_unload(GenModule& m) {
    if (m.lib) cudaLibraryUnload(m.lib);
    m.lib = nullptr;
    m.kernel = nullptr;
}

}  // namespace rtl
