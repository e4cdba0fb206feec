// pool.hpp -- instance pools used by the server (continuous batching).
//
// A pool is a batch of `capacity` instance slots of one netlist.  Jobs of that
// netlist occupy contiguous slot ranges; every step advances all slots, each
// slot counting its own cycles from the moment its job was admitted, so jobs
// that arrive while others run share the same launches.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

struct sim_netlist;
struct sim_batch;

namespace rtl {
// persistent: each pool_step is one persistent launch (grid barrier between
// cycles, grid sized to the active instance groups); else per-cycle graphs.
int pool_create(sim_netlist* nl, uint32_t capacity, bool persistent, sim_batch** out);
// Give slots [lo, lo+n) to a job: stimulus keys of instances 0..n-1 of `seed`,
// cycle origin = the pool's current cycle, state reset to the initial state.
int pool_admit(sim_batch* b, uint32_t lo, uint32_t n, uint64_t seed);
// Enqueue `n` cycles for the active slots (asynchronous on the pool's stream);
// *kernels receives the number of kernels it launched.
int pool_step(sim_batch* b, uint64_t n, uint64_t* kernels);
// Simulate only instance groups [0, n_groups) (32 slots each) from the next
// step on: slots are taken first-fit, so the occupied ones sit at the front.
// A persistent step then launches at most max_grid / share CTAs, so that
// `share` pools stepping at once fit on the GPU side by side.
int pool_set_active(sim_batch* b, uint32_t n_groups, uint32_t share);
// State digests of slots [lo, lo+n) (synchronises the pool's stream).
int pool_digests(sim_batch* b, uint32_t lo, uint32_t n, uint64_t* out);
// Device bytes a pool of `capacity` slots of this netlist holds.
size_t pool_footprint(const sim_netlist* nl, uint32_t capacity);
cudaStream_t pool_stream(sim_batch* b);
uint64_t pool_cycle(sim_batch* b);
}  // namespace rtl
