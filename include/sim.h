/*
 * sim.h -- C ABI of the GB300 BSP RTL simulator.
 *
 * The simulator runs the per-clock-cycle bulk-synchronous evaluation of a
 * partitioned word-level netlist (Parendi, Sec. 3.2 "BSP RTL Simulation" and
 * Sec. 5.1 "Partitioning"): every register's combinational cone is a fiber,
 * fibers are merged into processes by submodular load balancing, each
 * process computes its registers' next values from the current values, the
 * next values are committed to double-buffered state, and one grid-wide
 * barrier separates simulated cycles.
 *
 * Conventions for every function below:
 *   - the return value is SIM_OK (0) or a negative SIM_ERR_* code, and
 *     sim_last_error() then holds a message for the calling thread;
 *   - handles are created and owned by the library; the caller releases
 *     them with the matching *_destroy, batches before their netlist;
 *   - buffers passed in are copied before the call returns, buffers passed
 *     out are caller-owned host memory of the stated size;
 *   - no C++ exception ever crosses this boundary.
 *
 * Netlist text format (`rtlnet 1`): see the module docstring of
 * paper_2403_04714_gb300/netgen.py.  Inputs, registers, memories and nodes are
 * numbered from 0 in file order.  Semantics per simulated cycle: inputs are
 * drawn (or held), all nodes are evaluated from current register and memory
 * values, registers take their next-state values, then memory write ports
 * apply in ascending port order (the highest port wins an address).
 *
 * Clocks (paper Sec. 5, limitations: one top-level clock plus gated or
 * divided ones): `gate r e` lets register r take its next value only in
 * cycles where node e is nonzero; `clock r d` puts register r on the rising
 * edge of the 1-bit register d, which comes after d's own update, so r's next
 * value and gate see the registers of earlier clock domains already updated
 * in that cycle.  The loader lowers both to single-clock next-value logic
 * (the reported op count includes it); a memory read in the cone of a
 * register on a divided clock, a loop of clock registers or a clock register
 * wider than one bit is a PARSE or WIDTH error.
 */
#ifndef GB300_RTLSIM_SIM_H
#define GB300_RTLSIM_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    SIM_OK = 0,
    SIM_ERR_PARSE = -1,      /* malformed netlist text */
    SIM_ERR_COMB_LOOP = -2,  /* combinational cycle (paper Sec. 5.3: compile fails) */
    SIM_ERR_WIDTH = -3,      /* width/slice/concat/compare inconsistency */
    SIM_ERR_CAPACITY = -4,   /* a process does not fit the per-warp on-chip budget (Sec. 5.1 stage 4) */
    SIM_ERR_OOM = -5,        /* device or host allocation failed */
    SIM_ERR_TIMEOUT = -6,    /* a grid barrier wait ran past its limit */
    SIM_ERR_CUDA = -7,       /* a CUDA runtime call failed */
    SIM_ERR_BADARG = -8,     /* argument out of range or null */
    SIM_ERR_ADMISSION = -9,  /* job larger than the server's memory cap */
    SIM_ERR_STATE = -10      /* call not valid in the current state */
};

/* signal kinds for sim_poke / sim_peek */
enum { SIM_SIG_INPUT = 0, SIM_SIG_REG = 1 };

/* How a warp maps onto the netlist.
 *   LANE_OP:   one warp runs one process of one instance; its 32 lanes run
 *              independent nodes of the same schedule step (single instance).
 *   LANE_INST: one warp runs one process for 32 instances, lane = instance,
 *              with instance-minor state (batched stimulus instances).
 *   AUTO:      LANE_INST when n_inst >= 32, else LANE_OP. */
enum { SIM_MODE_AUTO = 0, SIM_MODE_LANE_OP = 1, SIM_MODE_LANE_INST = 2 };

/* How cycles are launched.
 *   PERSISTENT:  one cooperative launch per sim_step keeps every process
 *                resident and crosses cycles with a flag-based grid barrier.
 *   PER_CYCLE:   one kernel launch per simulated cycle; the launch boundary
 *                is the barrier (the plain baseline).
 *   PER_CYCLE_GRAPH: the PER_CYCLE launch chain captured once into a CUDA
 *                graph and replayed.
 *   PERSISTENT_GRAPH: the PERSISTENT launch of a step (barrier reset,
 *                cooperative launch, cycle-base advance) captured into a CUDA
 *                graph per step length and replayed. */
enum { SIM_KERNEL_PERSISTENT = 0, SIM_KERNEL_PER_CYCLE = 1, SIM_KERNEL_PER_CYCLE_GRAPH = 2,
       SIM_KERNEL_PERSISTENT_GRAPH = 3 };

/* How processes are lowered.
 *   BYTECODE:  a compact 16-byte instruction stream run by one interpreter
 *              kernel (no compile step).
 *   GENERATED: straight-line CUDA per process (values in registers),
 *              compiled for sm_103a at the first sim_create_instances of
 *              each lane mapping with NVRTC and nvJitLink; linked modules are
 *              cached under $RTLSIM_GENCACHE when that is set. */
enum { SIM_LOWER_BYTECODE = 0, SIM_LOWER_GENERATED = 1 };

/* Task order.  GROUP_MAJOR: neighbouring warps run different processes of
 * the same instances (their state stays in L2).  PROCESS_MAJOR: neighbouring
 * warps run the same process for different instance groups (its code and
 * program stay hot in the SM).  CTA_MAJOR (generated LANE_INST only): each
 * CTA runs every instance group of its processes, so a process's code is
 * fetched by one SM.  AUTO: PROCESS_MAJOR for LANE_INST. */
/* Partitioning strategy (sim_config.partitioner). */
enum { SIM_PART_SLB = 0, SIM_PART_HYPERGRAPH = 1 };

enum { SIM_ORDER_AUTO = 0, SIM_ORDER_GROUP_MAJOR = 1, SIM_ORDER_PROCESS_MAJOR = 2, SIM_ORDER_CTA_MAJOR = 3 };

typedef struct sim_config {
    uint32_t struct_size;       /* sizeof(sim_config) */
    int32_t mode;               /* SIM_MODE_* */
    int32_t kernel;             /* SIM_KERNEL_* */
    uint32_t target_processes;  /* SLB target count; 0 = by mapping: one instance 4 per SM (8 when that leaves a
                                   straggler well above the slowest fiber), cluster exchange one per warp of the
                                   resident clusters, lane = instance 4 per SM (bytecode) or 2 (generated) */
    uint32_t warps_per_cta;     /* 0 = autotuned */
    uint32_t max_slots;         /* per-process value-slot cap; 0 = from the shared-memory budget */
    uint32_t digest_capacity;   /* per-cycle digest ring length in cycles; 0 = digests off */
    uint32_t timeout_ms;        /* grid-barrier wait limit (default 2000) */
    uint64_t big_array_bytes;   /* SLB stage-1 threshold (paper default 128 KiB) */
    uint32_t disable_stage3;    /* testing: skip the conservative merge */
    uint32_t seed_partition;    /* testing: 0 = SLB; else a random partition with this seed */
    uint32_t lowering;          /* SIM_LOWER_BYTECODE or SIM_LOWER_GENERATED */
    uint32_t task_order;        /* SIM_ORDER_*: how (process, instance group) tasks map to warps */
    uint32_t phase_samples;     /* persistent launches time their first N cycles per CTA (0 = off) */
    uint32_t wave_groups;       /* process-major order: instance groups (of 32) per wave; 0 = fit ~64 MB of state */
    uint32_t cluster_size;      /* 0 = off; 2..16: thread-block clusters of this many CTAs exchange register values
                                 * through distributed shared memory (LANE_OP, bytecode, persistent kernel, one
                                 * instance; see sim_create_instances).  A grid of one cluster synchronises with
                                 * the cluster's barrier instead of the grid barrier.  Cluster grids are plain
                                 * (not cooperative) launches: a step that runs while another persistent
                                 * launch holds SMs may not get all its CTAs at once and then ends with
                                 * SIM_ERR_TIMEOUT (never a hang). */
    uint32_t partitioner;       /* SIM_PART_SLB (bottom-up merge, Sec. 5.1) or SIM_PART_HYPERGRAPH (k-way
                                 * hypergraph partition of the fibers minimising duplicated work, the
                                 * alternative strategy of Sec. 7) */
    uint32_t chain;             /* LANE_OP shared-memory programs: 2 = a lane may run a dependent pair of operators
                                 * in one step (the first result passed on in a register), 0/1 = one dependence
                                 * level per step (the default).  Pairs help when each SM sub-partition runs one
                                 * warp and cost issue slots when warps share one. */
    uint32_t reserved[1];
} sim_config;

typedef struct sim_netlist_info {
    uint32_t n_inputs, n_regs, n_mems, n_wports;
    uint64_t n_nodes;           /* all nodes including leaves */
    uint64_t n_ops;             /* combinational operators */
    uint32_t n_fibers;          /* sinks: registers plus memories with write ports */
    uint32_t n_processes;       /* after SLB */
    uint64_t fiber_cost_sum;    /* sum of fiber costs (duplication at one fiber per process) */
    uint64_t process_cost_sum;  /* sum of process costs after merging (duplicated work) */
    uint64_t process_cost_max;  /* straggler process cost (paper Sec. 4.3, t_comp bound) */
    uint64_t fiber_cost_max;    /* slowest fiber: the lower bound max_i t_i */
    uint32_t max_bundles;       /* longest LANE_OP schedule in 32-wide steps */
    uint32_t max_slots;         /* largest value-slot count of a process */
    uint64_t instr_count;       /* lowered instructions over all processes */
    uint64_t cut_words;         /* register words read across processes per cycle */
} sim_netlist_info;

typedef struct sim_netlist sim_netlist;
typedef struct sim_batch sim_batch;

/* Fill cfg with defaults (AUTO mode, persistent kernel, digests off). */
void sim_config_default(sim_config *cfg);

/* Parse, check, partition (fibers -> SLB processes, paper Sec. 5.1) and lower
 * a netlist.  `text` holds `len` bytes of rtlnet text (copied).  `cfg` may be
 * NULL for defaults.  Errors: PARSE, COMB_LOOP, WIDTH, CAPACITY, BADARG, OOM. */
int sim_load_netlist(const void *text, size_t len, const sim_config *cfg, sim_netlist **out);
int sim_netlist_get_info(const sim_netlist *nl, sim_netlist_info *out);
void sim_netlist_destroy(sim_netlist *nl);

/* Generate and compile (NVRTC + nvJitLink, no GPU needed) the generated-CUDA
 * lowering of one lane mapping ahead of sim_create_instances, e.g. to fill
 * the $RTLSIM_GENCACHE cache.  This compiles the module without per-cycle
 * digest code (batches with digest_capacity = 0); a batch that keeps digests
 * compiles its own module, whose process functions add the digest terms, at
 * its sim_create_instances.  *seconds: compile (or cache read) time;
 * *cached: 1 if the linked module came from the cache.  Errors: BADARG, CUDA
 * (compile or link failure, message in sim_last_error). */
int sim_netlist_compile_generated(sim_netlist *nl, int32_t mode, double *seconds, int32_t *cached);

/* Introspection of the compiled program (tests and tools).  With out == NULL
 * *bytes receives the table size; otherwise min(*bytes, size) bytes are
 * copied to out and *bytes receives the size.  Tables (`which`):
 *   0 LANE_OP bundles (16-byte instructions, 32 per bundle)
 *   1 LANE_OP first bundle of each process (u32)   2 LANE_OP bundle counts (u32)
 *   3 LANE_INST instructions (16 bytes)            4 LANE_INST first instruction (u32)
 *   5 LANE_INST instruction counts (u32)           6 process of each fiber (i32)
 *   7 sink of each fiber: register r >= 0, or -1-m for memory m (i32)
 *   8 cost of each fiber (u64)                     9 cost of each process (u64)
 *  10 register storage class (u8: 0 1-bit, 1 <=32-bit, 2 <=64-bit)
 *  11 register index within its class (u32)
 *  12 LANE_OP slot count of each process (u32)    13 LANE_INST slot count (u32)
 *  14 LANE_OP compact programs kept in shared memory (u32 words: per process
 *     the step count n, n step words (first instruction | count << 16 |
 *     flags: bit 31 not operators only, bit 30 leaves only, up to 128 of
 *     them), padded to a multiple of 4 words, then the 16-byte instructions)
 *                                                  15 first word of each (u32)
 *  16 words of each (u32)
 *  Cluster exchange (cluster_size > 0; empty otherwise):
 *  17 process of each warp of the grid (u32, 0xffffffff = idle)
 *  18 first mirror entry of each CTA (u32, grid + 1 offsets)
 *  19 register held by each mirror entry (u32)
 *  20 {CTAs per cluster, warps per CTA, grid CTAs, mirror entries per CTA, cross-process register reads
 *      inside a cluster, reads across clusters} (u64 x 6)
 *  21 log2 of the depth of each memory (u8)
 * Errors: BADARG. */
int sim_netlist_table(const sim_netlist *nl, int32_t which, void *out, size_t *bytes);

/* Allocate device state for n_inst instances (cudaMalloc), initialised to the
 * netlist's register init values and memory images, cycle 0.  The state is
 * the paper's current/next split (Sec. 3.2, Fig. bsp_sim): two register
 * buffers, the current one read and the next one written in each cycle.  Instance i's
 * stimulus key is output i+1 of the SplitMix64 stream seeded with `seed`.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream); every
 * device operation of the batch is ordered on it.  A netlist loaded with
 * cluster_size > 0 takes n_inst == 1 and runs the persistent kernel as a
 * cluster launch; CAPACITY if its clusters cannot all be resident at once.
 * Errors: BADARG, OOM, CAPACITY, CUDA. */
int sim_create_instances(sim_netlist *nl, uint32_t n_inst, uint64_t seed, void *cuda_stream,
                         sim_batch **out);
void sim_batch_destroy(sim_batch *b);

/* Test-driver access between steps (Sec. 5.3, Limitations: the host does
 * not interact with the simulation in every cycle; inputs come from the
 * on-device stimulus unless held here).
 * Input: hold `value` (overrides the stimulus from the next cycle on, until
 * sim_unpoke).  Register: overwrite its current value.  Takes effect before
 * the next sim_step.  Value is reduced to the signal width.  sim_poke_mem
 * overwrites one memory word (address below the depth, else BADARG).
 * All three synchronise the batch's stream.  Errors: BADARG, CUDA, STATE. */
int sim_poke(sim_batch *b, uint32_t inst, int32_t kind, uint32_t index, uint64_t value);
int sim_unpoke(sim_batch *b, uint32_t inst, uint32_t input);
int sim_poke_mem(sim_batch *b, uint32_t inst, uint32_t mem, uint64_t addr, uint64_t value);

/* Enqueue n_cycles simulated cycles on the batch's stream (asynchronous).
 * One simulated cycle is one BSP superstep (Sec. 3.2, Fig. bsp_sim): every
 * process reads current values, computes its registers' next values and its
 * memories' write records (differential exchange, Sec. 5.2), then all
 * processes meet at one barrier (the paper's two barriers become one with
 * double-buffered state; Sec. 4.1 is the cost of that barrier).
 * A barrier time-out is reported by the next sim_sync; after a device error
 * the batch refuses further steps, peeks and digests with STATE until
 * sim_restore loads a checkpoint.  Errors: BADARG, CUDA, STATE, TIMEOUT. */
int sim_step(sim_batch *b, uint64_t n_cycles);
int sim_sync(sim_batch *b);

/* Read state after the last completed cycle (synchronises the stream); the
 * test driver's view of the current values (Sec. 3.2, Sec. 5.3).
 * sim_peek_regs: all n_regs registers of one instance, in register order.
 * sim_peek_mems: all 2^lg words of memory `mem` of one instance, in address
 * order (out holds the memory's depth).  Errors: BADARG, CUDA, STATE. */
int sim_peek(sim_batch *b, uint32_t inst, int32_t kind, uint32_t index, uint64_t *out);
int sim_peek_mem(sim_batch *b, uint32_t inst, uint32_t mem, uint64_t addr, uint64_t *out);
int sim_peek_regs(sim_batch *b, uint32_t inst, uint64_t *out /* n_regs values */);
int sim_peek_mems(sim_batch *b, uint32_t inst, uint32_t mem, uint64_t *out /* depth values */);
int sim_cycle(sim_batch *b, uint64_t *out);

/* Digest of the current state of each instance, computed on the device:
 * sum over registers r of mix(H(r) ^ reg[r]) plus sum over memory words of
 * mix(H(2^40 + m*2^24 + a) ^ mem[m][a]) modulo 2^64, H(x) = x*gamma + 1,
 * mix = SplitMix64 output function.  out holds n_inst values. */
int sim_state_digests(sim_batch *b, uint64_t *out);

/* The same digests as sim_state_digests, for callers that cannot let the
 * library allocate device memory (an embedding host that owns every device
 * byte through its own pool, or a latency-critical loop that must not pay
 * the device-wide synchronisation of cudaMalloc/cudaFree).  The paper has
 * no counterpart: this is an interface choice of this library.
 *   - No cudaMalloc, cudaFree or other allocating call is made.  The
 *     per-instance accumulator is a fixed 512 KiB device array inside the
 *     library (at most 65536 instances, padded count); larger batches get
 *     SIM_ERR_CAPACITY.  Every GPU that loads the library keeps that array
 *     until the process exits.
 *   - `out` receives n_inst digests; it may be device memory or host memory
 *     (it is written with cudaMemcpyDefault).  The call synchronises.
 *   - The batch's device must be current (otherwise STATE).  The first
 *     call on a device looks up the array's device address for that device
 *     and keeps it; make that first call before any stream capture.  A
 *     cudaDeviceReset invalidates that address together with every handle
 *     of this library: do not use the library on that device afterwards in
 *     the same process.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     threads, other streams) race and may return wrong sums. */
int sim_state_digests_noalloc(sim_batch *b, uint64_t *out);

/* Per-cycle digests (ring of sim_config.digest_capacity cycles) are kept for
 * the instances listed here (default: instance 0).  Call before sim_step. */
int sim_track_digests(sim_batch *b, const uint32_t *insts, uint32_t n);
/* Digests of states first..first+n-1 of a tracked instance (state t = after
 * t cycles), still inside the ring.  Synchronises. */
int sim_digests(sim_batch *b, uint32_t inst, uint64_t first_cycle, uint64_t n, uint64_t *out);

/* One end-to-end step through host memory: copies n_inst*n_inputs held input
 * values (NULL = free-running stimulus) host->device, runs n_cycles, and
 * copies the n_inst final state digests device->host.  Synchronises. */
int sim_step_host(sim_batch *b, uint64_t n_cycles, const uint64_t *held_inputs, uint64_t *out_digests);

/* Checkpoint: registers, memories, held inputs and the cycle counter, i.e.
 * the whole current state of Sec. 3.2 (a cycle's result depends on nothing
 * else), so a run resumed from it is the same run.  The blob is malloc'd by
 * the library; release it with sim_free_blob.  sim_restore also clears a
 * batch's failed state.  Errors: BADARG, OOM, CUDA, STATE (blob of another
 * netlist or batch shape). */
int sim_save(sim_batch *b, void **blob, size_t *len);
int sim_restore(sim_batch *b, const void *blob, size_t len);
void sim_free_blob(void *blob);

/* Launch geometry actually used by the last sim_step: ctas, warps/cta,
 * processes, tasks per cycle; and how many kernels it launched. */
int sim_launch_info(sim_batch *b, uint32_t *ctas, uint32_t *warps_per_cta, uint32_t *tasks_per_cycle,
                    uint64_t *kernels_launched);

/* Phase times of the first n cycles of the last persistent launch (needs
 * sim_config.phase_samples >= n), in ns, three per cycle: compute (from the
 * earliest CTA starting the cycle to the last CTA arriving at the barrier:
 * the straggler's t_comp + t_comm, paper Eq. sim_rate), sync (last arrival
 * to last release: t_sync) and the whole cycle.  Synchronises. */
int sim_phase_times(sim_batch *b, uint32_t n, double *out);

/* Testing hook: make one CTA skip its barrier arrival once on the next
 * persistent sim_step, so the other CTAs' bounded waits expire and the step
 * returns SIM_ERR_TIMEOUT.  No fault, trap or unbounded wait is involved. */
int sim_debug_skip_arrival(sim_batch *b, uint32_t timeout_ms);

/* ---- serving: continuous batching of simulation jobs ---------------------
 * The paper motivates simulation throughput by many regression runs of one
 * design (Sec. 1 and the nightly-regression cost model of Sec. 6, Cost
 * Comparison); here independent jobs share the device.
 * A server keeps one instance pool per netlist in device memory.  Jobs of
 * the same netlist share the pool's launches (each job's instances occupy a
 * run of slots and count cycles from their admission); pools of different
 * netlists step concurrently on their own streams.  A job is admitted when
 * its pool has free slots, or when a new pool fits under hbm_cap_bytes
 * (idle pools are released to make room); otherwise it waits in arrival
 * order without blocking jobs of other netlists.  Finished jobs free their
 * slots at the next step boundary.  A job's results (per-instance state
 * digests) are identical to the same instances run alone with
 * sim_create_instances(netlist, n_inst, seed) and sim_step(n_cycles). */
typedef struct sim_server sim_server;
enum { SIM_JOB_QUEUED = 0, SIM_JOB_RUNNING = 1, SIM_JOB_DONE = 2, SIM_JOB_FAILED = 3 };

typedef struct sim_server_config {
    uint32_t struct_size;       /* sizeof(sim_server_config) */
    uint32_t pool_slots;        /* instance slots per pool (default 1024) */
    uint64_t hbm_cap_bytes;     /* device-memory cap for all pools (default 150 GiB) */
    uint32_t chunk_cycles;      /* cycles per pool step (default 1000) */
    uint32_t persistent;        /* 1 (default): a pool step is one persistent launch that runs all its jobs'
                                 * instance groups across the step's cycles (grid barrier between cycles, grid
                                 * sized to the groups in use, so pools of other netlists still share the GPU);
                                 * 0: one launch per cycle, replayed from a CUDA graph */
    uint32_t reserved[6];
} sim_server_config;

typedef struct sim_job {
    sim_netlist *netlist;       /* must stay alive until the job is done */
    uint32_t n_inst;            /* instances 0..n_inst-1 of `seed` */
    uint64_t seed;
    uint64_t n_cycles;
} sim_job;

typedef struct sim_job_status {
    int32_t state;              /* SIM_JOB_* */
    uint32_t n_inst;
    uint64_t cycles_done;
    double t_arrive, t_start, t_done;   /* seconds since the server started */
} sim_job_status;

void sim_server_config_default(sim_server_config *cfg);
int sim_server_create(const sim_server_config *cfg, sim_server **out);
/* Queue a job; returns its id.  Errors: BADARG, ADMISSION (a single job larger
 * than the cap). */
int sim_submit(sim_server *s, const sim_job *job, uint64_t *job_id);
/* Status of a job (never blocks).  A failed job returns SIM_ERR_STATE with
 * the reason in sim_last_error(). */
int sim_poll(sim_server *s, uint64_t job_id, sim_job_status *st);
/* Block until the job is done or failed, at most timeout_ms (SIM_ERR_TIMEOUT). */
int sim_server_wait(sim_server *s, uint64_t job_id, uint32_t timeout_ms);
/* Per-instance final state digests of a done job (n_inst values). */
int sim_job_digests(sim_server *s, uint64_t job_id, uint64_t *out);
/* Totals: instance-cycles simulated, kernels launched, pool bytes in use. */
int sim_server_stats(sim_server *s, uint64_t *instance_cycles, uint64_t *kernels, uint64_t *bytes_in_use);
/* Device bytes a pool of `slots` instance slots of this netlist holds (the
 * quantity admission compares with hbm_cap_bytes). */
size_t sim_server_footprint(const sim_netlist *nl, uint32_t slots);
/* Stops the worker after the steps in flight and frees every pool. */
void sim_server_destroy(sim_server *s);

const char *sim_last_error(void);

/* Measured integer issue rate of the current device (the ALU roof of the
 * interpreter): independent chains of three-input adds and three-input logic
 * ops on every SM, `iters` iterations per thread, timed with CUDA events;
 * *lane_ops_per_s = instructions x 32 lanes per second.  The paper has no
 * counterpart.  Errors: BADARG, CUDA. */
int sim_measure_int_peak(uint32_t iters, double *lane_ops_per_s);

#ifdef __cplusplus
}
#endif
#endif
