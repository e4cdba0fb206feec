// noalloc.cu -- state digests without any device allocation.
//
// sim_state_digests() accumulates each instance's digest in a device buffer
// that the library allocates (cudaMalloc) the first time it is needed.  Some
// callers cannot let a library allocate: hosts that hand out all device
// memory from their own pool or arena and forbid allocations behind their
// back, callers that must not incur the implicit device synchronisation of
// cudaMalloc/cudaFree in a latency-critical loop, and code that is only
// allowed to touch memory it was given.  sim_state_digests_noalloc() computes
// the same digests, with the same kernel, into a fixed file-scope device
// array instead, so it calls no cudaMalloc, cudaFree or other allocating
// routine.
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
                uint32_t* I, uint32_t* n_inst, uint32_t* par, cudaStream_t* stream, int* device);
int batch_sync(sim_batch* b);
int set_error(int code, const std::string& msg);
// The full-state digest kernel of sim_state_digests (kernels.cu): adds each
// instance's digest into out[inst], which the caller clears first.
cudaError_t launch_state_digest(cudaStream_t st, const DevProg& P, const DevState& S, uint32_t par,
                                const uint64_t* mem_word_off, uint64_t mem_words, uint64_t* out, uint32_t n_inst);
}  // namespace rtl

namespace {

// Accumulator of the allocation-free digest: one 64-bit word per instance.
// Every GPU that loads the library holds this 512 KiB array until the process
// exits.  All calls share it and it keeps the last call's contents.
constexpr uint32_t kMaxInstances = 1u << 16;
static __device__ __align__(256) unsigned long long g_digest_scratch[kMaxInstances];

// Device address of g_digest_scratch, looked up once per device with that
// device current.  (In host code the array's name is only a host-side
// stand-in, never a device address.)
std::mutex g_lock;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(int dev, uint64_t** out) {
    if (dev < 0 || dev >= kMaxDevices) return rtl::set_error(SIM_ERR_STATE, "device index out of range");
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_digest_scratch);
        if (e != cudaSuccess || !p)
            return rtl::set_error(SIM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<uint64_t*>(g_scratch_addr[dev]);
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
    int dev = 0, cur = -1;
    int rc = rtl::batch_views(b, &P, &S, &mem_word_off, &mem_words, &I, &n_inst, &par, &st, &dev);
    if (rc) return rc;
    if (I > kMaxInstances)
        return rtl::set_error(SIM_ERR_CAPACITY, "sim_state_digests_noalloc handles at most 65536 instances (batch has " +
                                                    std::to_string(I) + ")");
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return rtl::set_error(SIM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (cur != dev)
        return rtl::set_error(SIM_ERR_STATE, "make the batch's device (" + std::to_string(dev) + ") current first");
    rc = rtl::batch_sync(b);
    if (rc) return rc;
    uint64_t* acc = nullptr;
    rc = scratch_address(dev, &acc);
    if (rc) return rc;
    // the array keeps the previous call's sums: clear the part this call uses
    e = cudaMemsetAsync(acc, 0, size_t(I) * 8, st);
    if (e == cudaSuccess) e = rtl::launch_state_digest(st, P, S, par, mem_word_off, mem_words, acc, I);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, acc, size_t(n_inst) * 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return rtl::set_error(SIM_ERR_CUDA, std::string("state digest: ") + cudaGetErrorString(e));
    return SIM_OK;
}
