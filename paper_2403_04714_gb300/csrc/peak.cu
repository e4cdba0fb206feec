// peak.cu -- measured integer issue rate of the GPU (the ALU roof).
//
// The interpreter's work is 32/64-bit integer ALU instructions; the chip's
// ceiling for them is the issue rate of the integer pipes.  This kernel keeps
// every SM sub-partition busy with independent chains of the instruction
// kinds the interpreter uses most (three-input add, three-input logic), so
// that the timed rate is issue-limited, not latency-limited.  The paper has
// no counterpart (it reports no device peaks).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/sim.h"

namespace {

constexpr int kChains = 8;          // independent dependence chains per thread
constexpr int kOpsPerChain = 2;     // one add and one logic op per chain and iteration

__global__ void k_int_peak(uint32_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = threadIdx.x * 0x9E3779B9u + c * 0x85EBCA6Bu + seed;
    const uint32_t k1 = blockIdx.x | 1u, k2 = seed ^ 0x27D4EB2Fu;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            a[c] = a[c] + k1 + i;           // IADD3
            a[c] = (a[c] ^ k2) & (a[c] | i);  // LOP3
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) x ^= a[c];
    if (x == 0x5EEDu) sink[0] = x;         // keeps every chain live
}

}  // namespace

extern "C" int sim_measure_int_peak(uint32_t iters, double* lane_ops_per_s) {
    if (!lane_ops_per_s || iters == 0) return SIM_ERR_BADARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SIM_ERR_CUDA;
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    int rc = SIM_OK;
    const int threads = 256, blocks = sms * 8;      // 64 warps per SM: latency fully hidden
    if (cudaMalloc(&sink, 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        rc = SIM_ERR_CUDA;
    } else {
        k_int_peak<<<blocks, threads, 0, st>>>(iters / 8 + 1, 1u, sink);      // warm-up
        cudaEventRecord(e0, st);
        k_int_peak<<<blocks, threads, 0, st>>>(iters, 2u, sink);
        cudaEventRecord(e1, st);
        float ms = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0) {
            rc = SIM_ERR_CUDA;
        } else {
            const double ops = double(blocks) * threads * double(iters) * kChains * kOpsPerChain;
            *lane_ops_per_s = ops / (ms * 1e-3);
        }
    }
    cudaGetLastError();
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return rc;
}
