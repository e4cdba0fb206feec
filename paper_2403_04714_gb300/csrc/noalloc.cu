// noalloc.cu -- state digests without any device allocation.
//
// sim_state_digests() accumulates each instance's digest in a device buffer
// that the library allocates (cudaMalloc) the first time it is needed.  Some
// callers cannot let a library allocate: hosts that hand out all device
// memory from their own pool or arena and forbid allocations behind their
// back, callers that must not incur the implicit device synchronisation of
// cudaMalloc/cudaFree in a latency-critical loop, and code that is only
// allowed to touch memory it was given.  sim_state_digests_noalloc() computes
// the same digests with its accumulator in a fixed, file-scope device array
// instead, so it calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/sim.h"
#include "device.hpp"

struct sim_batch;

namespace rtl {
// Views of a batch's device tables and state (defined in runtime.cpp).
int batch_views(sim_batch* b, DevProg* P, DevState* S, const uint64_t** mem_word_off, uint64_t* mem_words,
                uint32_t* I, uint32_t* n_inst, uint32_t* par, cudaStream_t* stream);
int batch_sync(sim_batch* b);
int set_error(int code, const std::string& msg);
}  // namespace rtl

namespace {

// Accumulator of the allocation-free digest: one 64-bit word per instance.
// Every GPU that loads the library holds this 512 KiB array until the process
// exits.  All calls share it and it keeps the last call's contents.
constexpr uint32_t kMaxInstances = 1u << 16;
static __device__ __align__(256) unsigned long long g_digest_scratch[kMaxInstances];

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 output function (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t reg_value(const rtl::DevState& S, uint32_t par, uint32_t cls, uint32_t idx,
                                              uint32_t inst) {
    if (cls == rtl::RC_W64) return S.w64[par][(uint64_t)idx * S.I + inst];
    if (cls == rtl::RC_W32) return S.w32[par][(uint64_t)idx * S.I + inst];
    uint32_t word = S.bits[par][(uint64_t)idx * S.bit_stride + inst / S.pack];
    return (word >> (inst % S.pack)) & 1u;
}

// Same digest as k_state_digest: each thread sums a chunk of registers and
// memory words of one instance into acc[inst].
__global__ void k_state_digest_noalloc(rtl::DevProg P, rtl::DevState S, uint32_t par, const uint64_t* mem_word_off,
                                       uint64_t mem_words, unsigned long long* acc, uint32_t n_inst, uint32_t chunk) {
    uint32_t inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= n_inst) return;
    uint64_t first = (uint64_t)blockIdx.y * chunk;
    uint64_t items = (uint64_t)P.n_reg + mem_words;
    uint64_t last = first + chunk < items ? first + chunk : items;
    uint64_t sum = 0;
    for (uint64_t j = first; j < last; j++) {
        if (j < P.n_reg) {
            sum += mix64((j * kGamma + 1ULL) ^ reg_value(S, par, P.reg_cls[j], P.reg_idx[j], inst));
        } else {
            uint64_t w = j - P.n_reg;
            uint32_t m = 0;
            while (m + 1 < P.n_mem && mem_word_off[m + 1] <= w) m++;
            uint64_t a = w - mem_word_off[m];
            uint64_t h = ((1ULL << 40) + ((uint64_t)m << 24) + a) * kGamma + 1ULL;
            sum += mix64(h ^ S.mem[P.mem_base[m] + a * S.I + inst]);
        }
    }
    atomicAdd(acc + inst, (unsigned long long)sum);
}

// Device address of g_digest_scratch, looked up once per device.
std::mutex g_lock;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rtl::set_error(SIM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return rtl::set_error(SIM_ERR_STATE, "device index out of range");
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_digest_scratch);
        if (e != cudaSuccess || !p)
            return rtl::set_error(SIM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned long long*>(g_scratch_addr[dev]);
    return SIM_OK;
}

}  // namespace

extern "C" int sim_state_digests_noalloc(sim_batch* b, uint64_t* out) {
    if (!b || !out) return rtl::set_error(SIM_ERR_BADARG, "null argument");
    rtl::DevProg P;
    rtl::DevState S;
    const uint64_t* mem_word_off = nullptr;
    uint64_t mem_words = 0;
    uint32_t I = 0, n_inst = 0, par = 0;
    cudaStream_t st = nullptr;
    int rc = rtl::batch_views(b, &P, &S, &mem_word_off, &mem_words, &I, &n_inst, &par, &st);
    if (rc) return rc;
    if (I > kMaxInstances)
        return rtl::set_error(SIM_ERR_CAPACITY, "sim_state_digests_noalloc handles at most 65536 instances (batch has " +
                                                    std::to_string(I) + ")");
    rc = rtl::batch_sync(b);
    if (rc) return rc;
    unsigned long long* acc = nullptr;
    rc = scratch_address(&acc);
    if (rc) return rc;
    // the array keeps the previous call's sums: clear the part this call uses
    cudaError_t e = cudaMemsetAsync(acc, 0, size_t(I) * 8, st);
    const uint32_t chunk = 256;
    uint64_t items = (uint64_t)P.n_reg + mem_words;
    dim3 grid((I + 127) / 128, uint32_t((items + chunk - 1) / chunk));
    if (e == cudaSuccess && grid.y > 0) {
        k_state_digest_noalloc<<<grid, 128, 0, st>>>(P, S, par, mem_word_off, mem_words, acc, I, chunk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, acc, size_t(n_inst) * 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return rtl::set_error(SIM_ERR_CUDA, std::string("state digest: ") + cudaGetErrorString(e));
    return SIM_OK;
}
