// sim_rt.cuh -- device runtime shared by the bytecode kernels (kernels.cu) and
// the generated per-process code compiled at run time: stimulus, register
// and memory access, write-record forwarding and commit, digests, and the
// bounded grid barrier.  Compiled by nvcc into the library and passed to
// NVRTC as an in-memory header.
#pragma once
#include "abi_device.h"

#ifndef SIM_ERR_TIMEOUT
#define SIM_ERR_TIMEOUT (-6)
#endif

namespace rtl {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 output function (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t wmask(uint32_t w) { return ~0ULL >> (64 - w); }   // w in 1..64

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) { return *(volatile const int32_t*)p; }


__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier on one monotonic 64-bit arrival counter (zeroed before
// each launch): barrier number g of the launch is complete once the counter
// reaches (g+1) x gridDim.x.  Each CTA adds its arrival with a release
// reduction (no round trip: the CTA's stores of the cycle, ordered before it
// by __syncthreads, become visible to every CTA that acquires the count) and
// then polls the counter with acquire loads; nobody has to reset a counter or
// publish a generation word, so the last arrival releases everyone directly.
// Every wait is bounded: past `timeout_ns`, or once another CTA has recorded
// an error, the CTA records SIM_ERR_TIMEOUT (first error wins) and returns
// false.  With `rec` set, thread 0 stores the time the whole CTA arrived
// (rec[0]) and the time the barrier released it (rec[1]), from %globaltimer.
static __device__ bool grid_barrier(uint32_t* bar, uint32_t& gen, uint64_t timeout_ns, int32_t* err, bool skip,
                                    uint64_t* rec = nullptr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (rec) rec[0] = globaltimer_ns();
        unsigned long long* count = reinterpret_cast<unsigned long long*>(bar);
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x;
        if (!skip) red_release_add(count, 1ull);
        const uint64_t start = globaltimer_ns();
        while (ld_acquire_u64(count) < target) {
            if (ld_volatile(err) != 0) { ok = 0; break; }
            if (globaltimer_ns() - start > timeout_ns) {
                atomicCAS(err, 0, (int32_t)SIM_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        gen++;
        if (rec) rec[1] = globaltimer_ns();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ uint64_t load_reg(const DevState& S, uint32_t par, uint32_t cls, uint32_t idx, uint32_t inst) {
    if (cls == RC_W64) return S.w64[par][(uint64_t)idx * S.I + inst];
    if (cls == RC_W32) return S.w32[par][(uint64_t)idx * S.I + inst];
    uint32_t word = S.bits[par][(uint64_t)idx * S.bit_stride + inst / S.pack];
    return (word >> (inst % S.pack)) & 1u;
}

__device__ __forceinline__ uint64_t stimulus(const DevProg& P, const DevState& S, uint64_t key, uint32_t k, uint32_t inst,
                                             uint64_t t, uint32_t w) {
    if (S.any_hold) {
        uint64_t j = (uint64_t)k * S.I + inst;
        if (S.hold_flag[j]) return S.hold_val[j] & wmask(w);
    }
    if (S.t_off) t -= S.t_off[inst];     // pooled slot: the job's own cycle count
    return mix64(key + (t * P.n_in + k + 1) * kGamma) & wmask(w);
}

__device__ __forceinline__ uint64_t mem_hash(uint32_t m, uint64_t a) {
    return ((1ULL << 40) + ((uint64_t)m << 24) + a) * kGamma + 1ULL;
}

// Read memory m at addr for inst as of the clock edge: the array plus the
// pending write records of the previous cycle (highest port wins).
__device__ __forceinline__ uint64_t mem_read(const DevProg& P, const DevState& S, uint32_t m, uint64_t addr, uint32_t inst,
                                             uint32_t prev, bool pending) {
    uint64_t v = S.mem[P.mem_base[m] + addr * S.I + inst];
    if (pending) {
        for (uint32_t j = P.mport_off[m]; j < P.mport_off[m + 1]; j++) {
            const uint64_t* r = S.rec[prev] + ((uint64_t)P.mport_id[j] * S.I + inst) * 2;
            uint64_t ea = r[0];
            if ((ea >> 63) && (ea & ~(1ULL << 63)) == addr) v = r[1];
        }
    }
    return v;
}

// Apply the previous cycle's write records of memory m for one instance
// (ascending port order) and return the change of the memory digest.
__device__ __forceinline__ uint64_t mem_commit(const DevProg& P, const DevState& S, uint32_t m, uint32_t inst, uint32_t prev,
                                               bool digest) {
    uint64_t delta = 0;
    for (uint32_t j = P.mport_off[m]; j < P.mport_off[m + 1]; j++) {
        const uint64_t* r = S.rec[prev] + ((uint64_t)P.mport_id[j] * S.I + inst) * 2;
        uint64_t ea = r[0];
        if (ea >> 63) {
            uint64_t addr = ea & ~(1ULL << 63);
            uint64_t* cell = S.mem + P.mem_base[m] + addr * S.I + inst;
            uint64_t old = *cell, nv = r[1];
            *cell = nv;
            if (digest) delta += mix64(mem_hash(m, addr) ^ nv) - mix64(mem_hash(m, addr) ^ old);
        }
    }
    return delta;
}

__device__ __forceinline__ void ring_add(const DevState& S, uint64_t t, int32_t col, uint64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(S.ring + (t % S.ring_cap) * S.n_tracked + col),
              (unsigned long long)v);
}

// Memory part of the digest at cycle t (records of t-1 just applied).
__device__ __forceinline__ void mem_digest_update(const DevState& S, uint32_t m, uint32_t inst, uint64_t t, uint64_t delta) {
    int32_t col = S.track[inst];
    if (col < 0) return;
    uint64_t* md = S.mem_dig + (uint64_t)m * S.I + inst;
    uint64_t v = *md + delta;
    *md = v;
    ring_add(S, t, col, v);
}

// Task k -> (process p, instance group g).  Group-major: the processes of one
// group are neighbours.  Process-major in waves: the groups are split into
// waves of `wave_groups` (whose state fits in L2); within a wave the tasks of
// one process are neighbours, so warps that run together share its code.
__device__ __forceinline__ void task_coords(const LaunchArgs& A, uint32_t n_proc, uint32_t task, uint32_t& p,
                                            uint32_t& g) {
    if (!A.proc_major) {
        p = task % n_proc;
        g = task / n_proc;
        return;
    }
    const uint32_t G = A.n_tasks / n_proc;
    const uint32_t W = A.wave_groups ? (A.wave_groups < G ? A.wave_groups : G) : G;
    const uint32_t per_wave = W * n_proc;
    const uint32_t wave = task / per_wave, r = task % per_wave;
    const uint32_t gw = (wave + 1) * W <= G ? W : G - wave * W;    // the last wave may be short
    p = r / gw;
    g = wave * W + r % gw;
}

// Apply the last cycle's write records after the final barrier of a launch
// (or in a launch of its own after per-cycle launches).
static __device__ void final_commit(const DevProg& P, const DevState& S, uint64_t t_end, uint64_t gtid,
                                    uint64_t gthreads) {
    const uint32_t prev = uint32_t((t_end - 1) & 1);
    const uint64_t total = (uint64_t)P.n_mem * S.I;
    for (uint64_t e = gtid; e < total; e += gthreads) {
        uint32_t m = uint32_t(e / S.I), inst = uint32_t(e % S.I);
        if (P.mport_off[m] == P.mport_off[m + 1]) continue;
        bool dig = S.ring_cap && S.track[inst] >= 0;
        uint64_t delta = mem_commit(P, S, m, inst, prev, dig);
        if (dig) mem_digest_update(S, m, inst, t_end, delta);
    }
}

// Input values of cycle t for every (input, instance), k-major so that the
// lanes of a generated process function (consecutive instances) read
// consecutive words: each input is hashed once per instance and cycle instead
// of once in every process that reads it (about 80 processes per input on the
// 200k-op netlist).  Grid-stride over the calling threads.
__device__ __forceinline__ void fill_stim(const DevProg& P, const DevState& S, uint64_t t, uint64_t tid,
                                          uint64_t nth) {
    uint64_t* out = S.stim[t & 1];
    const uint32_t I = S.I;
    const uint64_t n = (uint64_t)P.n_in * I;
    const bool small = n <= 0xffffffffull;     // 32-bit division (the usual case)
    for (uint64_t e = tid; e < n; e += nth) {
        const uint32_t k = small ? uint32_t(e) / I : uint32_t(e / I);
        const uint32_t inst = small ? uint32_t(e) - k * I : uint32_t(e % I);
        out[e] = stimulus(P, S, S.key[inst], k, inst, t, P.in_w[k]);
    }
}

}  // namespace rtl

// ---------------------------------------------------------------------------
// Kernels for generated code (compiled at run time with the generated units).
// The per-process functions rtl_p<k> and the dispatcher come from codegen.cpp.
// ---------------------------------------------------------------------------
#ifdef RTLSIM_GENERATED
extern "C" __device__ void rtl_dispatch(uint32_t p, const rtl::DevProg* __restrict__ P,
                                        const rtl::DevState* __restrict__ S, uint32_t g, uint64_t t, bool pending,
                                        uint32_t lane, uint64_t* __restrict__ dacc, int32_t col);

namespace rtl {

// Same cycle loop as the bytecode kernel.  LANE_INST (mode 2): every lane runs
// its instance through the process function.  LANE_OP (mode 1): lane 0 runs
// the process for one instance.
template <int MODE, bool DIGEST>
__device__ __forceinline__ void gen_cycles(const DevProg* __restrict__ Pg, const DevState* __restrict__ Sg,
                                           const LaunchArgs& A) {
    const DevProg& P = *Pg;
    const DevState& S = *Sg;
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t warp = blockIdx.x * A.warps_per_cta + wib;
    const uint32_t tw = gridDim.x * A.warps_per_cta;
    const uint64_t t_base = A.t0_dev ? *A.t0_dev + A.t0 : A.t0;
    uint32_t gen = 0;
    for (uint32_t c = 0; c < A.n; c++) {
        const uint64_t t = t_base + c;
        const bool pending = c > 0 || A.pending_first;
        uint64_t* rec = (A.phase && c < A.phase_n) ? A.phase + ((uint64_t)c * gridDim.x + blockIdx.x) * 3 : nullptr;
        if (rec && threadIdx.x == 0) rec[0] = globaltimer_ns();
        const uint32_t G = A.n_tasks / P.n_proc;
        const uint32_t n_iter = A.cta_major ? ((P.n_proc + gridDim.x - 1) / gridDim.x) *
                                                  ((G + A.warps_per_cta - 1) / A.warps_per_cta)
                                            : (A.n_tasks + tw - 1) / tw;
        for (uint32_t it = 0; it < n_iter; it++) {
            uint32_t p, g;
            if (A.cta_major) {
                // CTA-major: all groups of one process stay on one CTA (one SM)
                const uint32_t gper = (G + A.warps_per_cta - 1) / A.warps_per_cta;
                p = blockIdx.x + (it / gper) * gridDim.x;
                g = wib + (it % gper) * A.warps_per_cta;
                if (p >= P.n_proc || g >= G) continue;
            } else {
                const uint32_t task = warp + it * tw;
                if (task >= A.n_tasks) break;
                task_coords(A, P.n_proc, task, p, g);
            }
            uint64_t dacc = 0;
            if (MODE == 2) {
                const uint32_t inst = g * 32u + lane;
                const int32_t col = DIGEST ? S.track[inst] : -1;
                rtl_dispatch(p, Pg, Sg, g, t, pending, lane, &dacc, col);
                if (DIGEST && col >= 0) {
                    if (p == 0) dacc += S.rom_dig[inst];
                    ring_add(S, t + 1, col, dacc);
                }
            } else {
                const int32_t col = DIGEST ? S.track[g] : -1;
                if (lane == 0) {
                    rtl_dispatch(p, Pg, Sg, g, t, pending, 0, &dacc, col);
                    if (DIGEST && col >= 0) {
                        if (p == 0) dacc += S.rom_dig[g];
                        ring_add(S, t + 1, col, dacc);
                    }
                }
                __syncwarp();
            }
        }
        // the next cycle's input values (read after the barrier, or by the next
        // launch); the step's first cycle had its own filled before the launch
        if (S.stim[0])
            fill_stim(P, S, t + 1, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        if (A.grid_sync) {
            const bool skip = (int32_t)blockIdx.x == A.skip_cta && c == 0;
            if (!grid_barrier(S.bar, gen, A.timeout_ns, S.err, skip, rec ? rec + 1 : nullptr)) return;
        }
    }
    if (A.grid_sync && A.n > 0)
        final_commit(P, S, t_base + A.n, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                     (uint64_t)gridDim.x * blockDim.x);
}

}  // namespace rtl

// Threads per CTA the generated kernels are compiled for: 1024 at the default
// 64-register cap; a higher cap (RTLSIM_GEN_MAXRREG) compiles for fewer.
#ifndef RTLSIM_GEN_MAX_THREADS
#define RTLSIM_GEN_MAX_THREADS 1024
#endif

// One kernel per generated module: rtl_gen_d1 (digests on) calls process
// functions that carry the digest code, rtl_gen_d0 calls ones without it.
#define RTLSIM_GEN_KERNEL_NAME_false rtl_gen_d0
#define RTLSIM_GEN_KERNEL_NAME_true rtl_gen_d1
#define RTLSIM_GEN_CAT(a, b) a##b
#define RTLSIM_GEN_KERNEL(MODE, DIGEST)                                                                       \
    extern "C" __global__ void __launch_bounds__(RTLSIM_GEN_MAX_THREADS)                                      \
        RTLSIM_GEN_CAT(RTLSIM_GEN_KERNEL_NAME_, DIGEST)(const rtl::DevProg* P, const rtl::DevState* S,        \
                                                        rtl::LaunchArgs A) {                                  \
        rtl::gen_cycles<MODE, DIGEST>(P, S, A);                                                               \
    }
#endif
