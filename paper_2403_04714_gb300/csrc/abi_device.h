// abi_device.h -- plain data shared by the host runtime, the CUDA kernels and
// the generated per-process code compiled at run time (NVRTC): register
// classes, the bytecode instruction, and the device views of a program, a
// batch's state and a launch.  No standard-library types.
#pragma once
#if defined(__CUDACC_RTC__)
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
#else
#include <cstdint>
#endif

namespace rtl {

// Register storage classes (instance-minor planes on the device).
enum RegClass : uint8_t { RC_BIT = 0, RC_W32 = 1, RC_W64 = 2 };

// ------------------------------------------------------------------------
// Device bytecode.  16 bytes per instruction.
// ------------------------------------------------------------------------
enum DOp : uint8_t {
    D_NOP = 0, D_LDR, D_LDI, D_CONST, D_MEMRD,
    D_ADD, D_SUB, D_MUL, D_AND, D_OR, D_XOR, D_SHL, D_SHR, D_EQ, D_LT,
    D_MUX, D_SLICE, D_CONCAT,
    D_STR, D_WREC, D_COMMIT,
    D_LDM,      // register value from this CTA's mirror (cluster exchange)
    D_STX,      // next register value into a cluster peer's mirror
    D_COUNT
};

struct DIns {
    uint8_t op, w;
    uint16_t dst, a, b, c, x;
    uint32_t imm;
};

// LANE_OP step word of a shared-memory program: first instruction (bits
// 0-15), instruction count (bits 16-23), kStepGeneric when the step holds
// anything other than the 13 operators (leaves, memory reads, stores), and
// kStepLeaf when it holds only leaves (register, mirror, input, constant):
// such a step may hold up to kLeafStepMax instructions, four per lane.
constexpr uint32_t kStepGeneric = 1u << 31;
constexpr uint32_t kStepLeaf = 1u << 30;
// A chain step (also kStepGeneric) holds two rows (bits 24-27 of the step
// word hold the row count) of n = count / 2 operators: lane i runs operator
// i, then operator n + i, without a warp barrier between them (D_NOP in the
// second row where a lane has one operator).  A second-row operator's imm
// bits 0/1/2 mark operands a/b/c that are the lane's first result, taken
// from a register (their slot fields name that result's slot, so the two
// rows also read as sequential steps).
constexpr uint32_t kStepChain = 1u << 29;
// A store step (also kStepGeneric) holds only register stores (D_STR) and
// mirror stores (D_STX), up to kLeafStepMax of them, four per lane.  Only
// programs without operator pairs have them (measured: with pairs the store
// step's code slows the pair loop more than the steps it saves).
constexpr uint32_t kStepStore = 1u << 28;
constexpr uint32_t kStepRowsShift = 24;
constexpr uint32_t kStepRowsMask = 0xfu;
constexpr uint32_t kChainMax = 2;
constexpr uint32_t kStepCountMask = 0xffu;
constexpr uint32_t kLeafStepMax = 128;



// Program tables of one lowered netlist (device pointers).
struct DevProg {
    const DIns* s_ins;          // LANE_OP bundles (32 instructions per row)
    const uint32_t* s_off;
    const uint32_t* s_len;
    const uint32_t* c_words;    // LANE_OP compact programs (step table + instructions)
    const uint32_t* c_off;      // per process: first word
    const uint32_t* c_size;     // per process: words (multiple of 4)
    const DIns* b_ins;          // LANE_INST linear streams
    const uint32_t* b_off;
    const uint32_t* b_len;
    const uint32_t* mport_off;  // write ports of each memory (n_mem+1 offsets)
    const uint32_t* mport_id;
    const uint8_t* mem_lg;
    const uint8_t* mem_w;
    const uint64_t* mem_base;   // first word of memory m (instance-minor: word (base + a*I + inst))
    const uint8_t* in_w;
    const uint8_t* reg_cls;
    const uint32_t* reg_idx;
    // cluster exchange (null unless the netlist was lowered for clusters)
    const uint32_t* warp_proc;  // process of each warp of the grid, kNoProc if idle
    const uint32_t* mir_off;    // per CTA: first mirror entry (grid+1 offsets)
    const uint32_t* mir_reg;    // register held by each mirror entry
    const uint32_t* warp_off;   // per warp: start of its slots in its CTA's shared memory (64-bit words)
    const uint32_t* warp_slots; // per warp: its slot words, the last one spare (program follows)
    uint32_t n_proc, n_in, n_reg, n_mem, n_wport;
};

constexpr uint32_t kNoProc = 0xffffffffu;

// State of one batch of instances (device pointers).
struct DevState {
    uint32_t* bits[2];          // 1-bit registers: [n_bit][bit_stride] words, `pack` instances per word
    uint32_t* w32[2];           // 2..32-bit registers: [n_w32][I]
    uint64_t* w64[2];           // 33..64-bit registers: [n_w64][I]
    uint64_t* mem;              // all memories, instance-minor
    uint64_t* rec[2];           // write records [n_wport][I][2]: (en<<63 | addr, data)
    const uint64_t* key;        // stimulus key per instance
    const uint64_t* t_off;      // per instance: cycle at which its job started (pooled serving), or null
    const uint64_t* hold_val;   // [n_in][I]
    const uint8_t* hold_flag;   // [n_in][I]
    uint64_t* ring;             // per-cycle digests [cap][n_tracked]
    const int32_t* track;       // per instance: ring column or -1
    uint64_t* mem_dig;          // running memory digest part [n_mem][I]
    const uint64_t* rom_dig;    // digest of the memories without write ports, per instance
    uint32_t* bar;              // grid barrier words: [0] arrivals, [1] generation
    int32_t* err;               // first error code of the launch (0 = none)
    uint64_t* stim[2];          // generated code: input k of instance i at cycle t in stim[t & 1][k * I + i], or null
    uint32_t I;                 // instances (padded to the lane-group size)
    uint32_t pack;              // instances per bit word (32 LANE_INST, 1 LANE_OP)
    uint32_t bit_stride;        // words per 1-bit register
    uint32_t any_hold;          // some input is held
    uint32_t ring_cap;          // 0 = digests off
    uint32_t n_tracked;
};

struct LaunchArgs {
    const uint64_t* t0_dev;     // if set, the first cycle is *t0_dev + t0 (graph replays)
    uint64_t t0;                // first cycle of this launch
    uint32_t n;                 // cycles in this launch
    uint32_t pending_first;     // records of cycle t0-1 are not yet applied
    uint32_t grid_sync;         // persistent: grid barrier after every cycle, then final commit
    int32_t skip_cta;           // testing: this CTA skips its first barrier arrival (-1 none)
    uint64_t timeout_ns;        // barrier wait limit
    uint32_t warps_per_cta;
    uint32_t slot_words;        // per-warp slot area in 64-bit words (even)
    uint32_t prog_words;        // per-warp resident program area in 32-bit words (0 = read from global)
    uint32_t n_tasks;           // processes x instance groups
    uint32_t group;             // instances per task (1 LANE_OP, 32 LANE_INST)
    uint32_t proc_major;        // process-major task order (in waves), else group-major
    uint32_t wave_groups;       // instance groups per wave of the process-major order (0 = all)
    uint32_t cta_major;         // CTA c runs processes c, c+grid, ...; its warps split the groups
    uint64_t* phase;            // per sampled cycle and CTA: {cycle start, CTA arrived, released} (ns), or null
    uint32_t phase_n;           // cycles recorded from the start of the launch
    uint32_t cluster;           // CTAs per thread-block cluster (0 = no cluster exchange)
    uint32_t mirror_words;      // per-CTA mirror entries per buffer (64-bit words)
    uint32_t one_cluster;       // the grid is one cluster: cluster barrier instead of the grid barrier
    uint32_t mirror_off;        // start of the mirror in a cluster CTA's shared memory (64-bit words)
    uint32_t grid;              // launch shape the batch planned (checked by the cluster kernel on entry)
    uint32_t smem_bytes;        // dynamic shared memory the batch planned
    uint32_t pairs;             // the LANE_OP programs hold operator pair steps
};

}  // namespace rtl
