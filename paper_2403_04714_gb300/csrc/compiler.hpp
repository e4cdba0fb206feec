// compiler.hpp -- host side of the simulator: netlist IR, fiber extraction,
// submodular-load-balancing partitioner and lowering to the device bytecode.
//
// Paper map:
//   * data-dependence graph with current/next register split: Sec. 3.2
//   * fibers (the nodes that produce one register's next value, found by a
//     reverse crawl from each sink): Sec. 3.2 and Sec. 5.1
//   * process cost tau(f_i U f_j) = t_i + t_j - tau(f_i n f_j): Sec. 4.3
//   * four-stage merge (big arrays, multi-device cut, conservative merge,
//     relaxed merge): Sec. 5.1
//   * differential exchange of arrays (only write records travel): Sec. 5.2
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "abi_device.h"

namespace rtl {

enum Op : uint8_t {
    OP_INPUT, OP_REG, OP_CONST, OP_MEMRD,
    OP_ADD, OP_SUB, OP_MUL, OP_AND, OP_OR, OP_XOR, OP_SHL, OP_SHR, OP_EQ, OP_LT,
    OP_MUX, OP_SLICE, OP_CONCAT, OP_COUNT
};

struct Node {
    uint8_t op = 0;
    uint8_t w = 0;
    int32_t a = -1, b = -1, c = -1;  // operands (node ids); index for input/reg/mem; slice: b = lo
    uint64_t k = 0;                  // constant value
};

struct WPort { int32_t mem, en, addr, data; };

struct Netlist {
    std::vector<uint8_t> in_w;
    std::vector<uint8_t> reg_w;
    std::vector<uint64_t> reg_init;
    std::vector<int32_t> reg_next;
    std::vector<uint8_t> mem_lg, mem_w;
    std::vector<std::vector<std::pair<uint32_t, uint64_t>>> mem_init;  // sparse images
    std::vector<Node> nodes;
    std::vector<WPort> wports;
    std::vector<int32_t> level;      // combinational depth of each node (leaves 0)
    std::vector<std::vector<int32_t>> mem_ports;  // write ports of each memory, ascending
    uint64_t n_ops = 0;
};

// Parse and check.  Returns 0 or a negative SIM_ERR_* code with a message.
int parse_netlist(const char* text, size_t len, Netlist& out, std::string& err);

inline RegClass reg_class(int w) { return w == 1 ? RC_BIT : (w <= 32 ? RC_W32 : RC_W64); }
static_assert(sizeof(DIns) == 16, "DIns is 16 bytes");

struct PartitionConfig {
    uint32_t target = 0;              // process count target (0 = no limit)
    uint64_t big_array_bytes = 128 * 1024;   // stage-1 threshold (paper default)
    uint64_t mem_budget_bytes = 0;    // per-process data-memory budget, 0 = none
    bool stage3 = true;
    uint32_t random_seed = 0;         // != 0: random balanced partition (tests)
    bool hypergraph = false;          // RepCut-style k-way hypergraph partition instead of SLB stages 3/4
    uint32_t cand_cap = 48;           // partner candidates examined per merge
};

struct Fiber {
    std::vector<int32_t> nodes;   // sorted node ids of the cone (leaves included)
    int32_t reg = -1;             // sink register, or -1
    int32_t mem = -1;             // sink memory (all its write ports), or -1
    uint64_t cost = 0;
};

struct Partition {
    std::vector<Fiber> fibers;
    std::vector<std::vector<int32_t>> procs;   // fiber ids of each process
    std::vector<uint64_t> proc_cost;
    uint64_t fiber_cost_sum = 0, fiber_cost_max = 0;
    uint64_t proc_cost_sum = 0, proc_cost_max = 0;
    uint64_t cut_words = 0;
};

uint64_t node_cost(const Netlist& nl, int32_t id);
void extract_fibers(const Netlist& nl, std::vector<Fiber>& out);
// SLB (paper Sec. 5.1): stage 1 array merge, stage 3 conservative merge,
// stage 4 relaxed merge to the target count.  Returns 0 or SIM_ERR_CAPACITY.
int partition(const Netlist& nl, const PartitionConfig& cfg, Partition& out, std::string& err);

// Cost of a union of sorted node sets (shared nodes counted once).
uint64_t union_cost(const Netlist& nl, const std::vector<int32_t>& a, const std::vector<int32_t>& b);
uint64_t inter_cost(const Netlist& nl, const std::vector<int32_t>& a, const std::vector<int32_t>& b);

// ------------------------------------------------------------------------
// Lowering
// ------------------------------------------------------------------------
struct Lowered {
    // LANE_OP: 32-wide bundles, one row per schedule step
    std::vector<DIns> s_ins;          // bundles * 32
    std::vector<uint32_t> s_off;      // per process: first bundle
    std::vector<uint32_t> s_len;      // per process: bundle count
    std::vector<uint32_t> s_slots;    // per process: slot count
    // LANE_OP compact program (what a warp keeps in shared memory): per
    // process a bundle table (first instruction | count << 16, one word per
    // step) followed by the step instructions without padding, 16-byte aligned
    std::vector<uint32_t> c_words;    // packed programs, 32-bit words
    std::vector<uint32_t> c_off;      // per process: first word (multiple of 4)
    std::vector<uint32_t> c_size;     // per process: words (multiple of 4)
    // LANE_INST: linear instruction list
    std::vector<DIns> b_ins;
    std::vector<uint32_t> b_off, b_len, b_slots;
    uint32_t max_bundles = 0, max_s_slots = 0, max_b_slots = 0;
    std::vector<int32_t> commit_proc; // per memory: process holding its write ports (-1 none)
};

// chain = 2: the compact programs run dependent operator pairs in one step
// (one lane, the first result kept in a register); otherwise one level per step.
int lower(const Netlist& nl, const Partition& part, Lowered& out, std::string& err, uint32_t chain = 0);

// Cluster exchange.  Processes are placed on a grid of thread-block
// clusters (C CTAs of W warps, one process per warp) so that producers and
// consumers of register values share a cluster where the greedy placement
// can arrange it.  Each CTA keeps a double-buffered mirror of the registers
// its processes read from producers inside the cluster: such reads become
// D_LDM (from the mirror) and each producer appends D_STX instructions that
// write the next value into the mirror of every consuming CTA of its cluster
// (distributed shared memory); reads across clusters stay D_LDR (HBM/L2).
struct ClusterPlan {
    uint32_t C = 0, W = 0, grid = 0;
    std::vector<uint32_t> warp_proc;   // process of each warp (grid * W), kNoProc if idle
    std::vector<uint32_t> mir_off;     // per CTA: first mirror entry (grid + 1 offsets)
    std::vector<uint32_t> mir_reg;     // register held by each mirror entry
    uint32_t mirror_words = 0;         // largest per-CTA mirror (entries per buffer)
    uint64_t reads_local = 0;          // cross-process register reads inside a cluster
    uint64_t reads_remote = 0;         // ... and across clusters
};
// Rewrites the LANE_OP tables of `low` (bundles and compact programs); with
// `wide_stores` (programs without operator pairs) the mirror stores join the
// wide store steps.
int lower_clusters(const Netlist& nl, const Partition& part, uint32_t C, uint32_t W, Lowered& low, ClusterPlan& plan,
                   std::string& err, bool wide_stores);

// register index -> (class, index in class)
struct RegLayout {
    std::vector<uint8_t> cls;
    std::vector<uint32_t> idx;
    uint32_t count[3] = {0, 0, 0};
};
RegLayout reg_layout(const Netlist& nl);

}  // namespace rtl
