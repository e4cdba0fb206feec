// runtime.cpp -- C ABI of the simulator (include/sim.h): netlist handles,
// batches of instances in device memory, stepping, peek/poke, digests.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sim.h"
#include "codegen.hpp"
#include "compiler.hpp"
#include "device.hpp"

namespace rtl {
cudaError_t prepare_cycles_kernel(int mode, size_t smem);
cudaError_t occupancy_cycles(int mode, int threads, size_t smem, int* blocks_per_sm);
cudaError_t launch_cycles(int mode, bool digest, bool cooperative, int grid, int threads, size_t smem, cudaStream_t st,
                          const DevProg& P, const DevState& S, const LaunchArgs& A);
cudaError_t launch_commit(int grid, cudaStream_t st, const DevProg& P, const DevState& S, uint64_t t_end,
                          const uint64_t* t0_dev);
cudaError_t prepare_cluster_kernel(size_t smem, uint32_t C);
cudaError_t occupancy_clusters(int grid, int threads, size_t smem, uint32_t C, int* n_clusters);
cudaError_t launch_cycles_cl(bool digest, int grid, int threads, size_t smem, uint32_t C, cudaStream_t st,
                             const DevProg& P, const DevState& S, const LaunchArgs& A);
cudaError_t launch_advance(cudaStream_t st, uint64_t* t0_dev, uint64_t n);
cudaError_t launch_stim(cudaStream_t st, const DevProg& P, const DevState& S, uint64_t t, const uint64_t* t0_dev);
cudaError_t launch_set_u64(cudaStream_t st, uint64_t* p, uint64_t v);
cudaError_t launch_state_digest(cudaStream_t st, const DevProg& P, const DevState& S, uint32_t par,
                                const uint64_t* mem_word_off, uint64_t mem_words, uint64_t* out, uint32_t n_inst);
}  // namespace rtl

using namespace rtl;

namespace {

thread_local std::string g_err;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

int set_err(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// On failure the runtime's last-error slot is read back (and so cleared), so
// that a later launch check does not report this call's error again.
#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            (void)cudaGetLastError();                                                         \
            return set_err(e_ == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA,      \
                           std::string(#expr) + ": " + cudaGetErrorString(e_));               \
        }                                                                                     \
    } while (0)

uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t mask_w(int w) { return w >= 64 ? ~0ULL : ((1ULL << w) - 1); }
uint64_t reg_hash(uint64_t r) { return r * kGamma + 1ULL; }
uint64_t mem_hash(uint64_t m, uint64_t a) { return reg_hash((1ULL << 40) + (m << 24) + a); }

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    return n;
}

// Dynamic shared memory a CTA of our kernels may use: the device's opt-in
// limit less 1 KB for the kernels' static shared variables.
size_t smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 220 * 1024;
    }
    return size_t(v) - 1024;
}

// Shared memory a cluster CTA requests at least: more than half an SM's,
// so that no SM holds two CTAs of the grid (a doubly loaded SM would be the
// straggler of every cycle).
constexpr size_t kClusterCtaSmemMin = 116 * 1024;

// Clusters of C CTAs (one per SM) that can be resident at once; without a
// GPU (compile-only use) an even share of the SMs.
int resident_clusters(uint32_t C, uint32_t W) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || prepare_cluster_kernel(kClusterCtaSmemMin, C) != cudaSuccess ||
        occupancy_clusters(int(C) * 64, int(W) * 32, kClusterCtaSmemMin, C, &n) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return std::max(1, sm_count() / int(C));
    }
    return n;
}

// A device allocation released with the owner.
struct DBuf {
    void* p = nullptr;
    size_t n = 0;
    ~DBuf() { reset(); }
    void reset() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    int alloc(size_t bytes) {
        reset();
        n = bytes;
        if (!bytes) return SIM_OK;
        CUDA_TRY(cudaMalloc(&p, bytes));
        return SIM_OK;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

template <class T>
int upload(DBuf& b, const std::vector<T>& v, cudaStream_t st) {
    int rc = b.alloc(v.size() * sizeof(T));
    if (rc) return rc;
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return SIM_OK;
}

}  // namespace

struct sim_netlist {
    sim_config cfg;
    // generated-CUDA lowering, per lane mapping (built on first use)
    std::mutex gen_mu;
    // [lane mapping][digest]: the process functions with or without digest code
    std::vector<char> gen_cubin[3][2];
    rtl::GenModule gen[3][2];
    double gen_seconds[3][2] = {};
    bool gen_cached[3][2] = {};
    ~sim_netlist() {
        for (auto& gm : gen)
            for (auto& g : gm) rtl::jit_unload(g);
    }
    Netlist nl;
    Partition part;
    Lowered low;
    ClusterPlan cplan;                    // cluster exchange placement (cfg.cluster_size > 0)
    RegLayout layout;
    sim_netlist_info info{};
    std::vector<uint32_t> mport_off, mport_id;
    std::vector<uint64_t> mem_word_off;   // per-instance word offset of each memory (+ total)
};

namespace rtl { struct PoolExtra; void pool_extra_free(PoolExtra*); }

struct sim_batch {
    sim_netlist* nl = nullptr;
    sim_config cfg{};                      // the configuration this batch was created with
    rtl::PoolExtra* pool = nullptr;        // set for server pools
    bool generated = false;                // processes run as generated CUDA
    const void* gen_kernel[2] = {nullptr, nullptr};
    DevState S_uploaded{};
    cudaStream_t stream = nullptr;
    int mode = SIM_MODE_LANE_OP;
    int kernel = SIM_KERNEL_PERSISTENT;
    uint32_t n_inst = 0, I = 0;
    uint64_t seed = 0, cycle = 0;
    // program tables
    DBuf s_ins, s_off, s_len, c_words, c_off, c_size, b_ins, b_off, b_len, mport_off, mport_id, mem_lg, mem_w, mem_base,
        in_w, reg_cls, reg_idx, mem_word_off, warp_proc, mir_off, mir_reg, warp_off, warp_slots;
    bool cluster = false;                   // cluster exchange kernel (k_cycles_cl)
    uint32_t mirror_off = 0;                // cluster CTA layout: mirror start (64-bit words)
    // state
    DBuf bits[2], w32[2], w64[2], mem, rec[2], key, hold_val, hold_flag, ring, track, mem_dig, rom_dig, bar, err, t0_dev,
        scratch, P_dev, S_dev, phase, stim;
    uint32_t phase_n = 0, phase_grid = 0;   // phase timers of the last persistent launch
    DevProg P{};
    DevState S{};
    std::vector<uint8_t> h_hold_flag;     // host mirror
    std::vector<uint64_t> h_hold_val;
    std::vector<int32_t> h_track;
    std::vector<uint32_t> tracked;
    // launch geometry
    int threads = 256, warps = 8, grid = 0, max_grid = 0;
    size_t smem = 0;
    uint32_t slot_words = 0, prog_words = 0, n_tasks = 0;
    uint32_t proc_major = 0;                // task order (see LaunchArgs)
    uint32_t wave_groups = 0;
    uint32_t cta_major = 0;
    uint64_t kernels_launched = 0;
    int32_t skip_cta = -1;
    uint64_t timeout_ns = 2000000000ULL;   // configured barrier wait limit
    uint64_t skip_timeout_ns = 0;          // wait limit of the one debug step that skips an arrival
    // After a device error (a barrier time-out) a launch has left the state
    // part-way through a cycle: the batch refuses steps, peeks and digests
    // until sim_restore loads a checkpoint.
    bool failed = false;
    std::string fail_reason;
    // graph replay of per-cycle launches
    cudaGraphExec_t graph = nullptr;
    uint32_t graph_chunk = 0;
    uint32_t graph_tasks = 0;              // tasks per cycle the graph was captured for
    cudaGraphExec_t pgraph = nullptr;      // captured persistent step
    uint64_t pgraph_n = 0;
    uint64_t pgraph_timeout = 0;
    DevState pgraph_state{};
    DevState graph_state{};               // state descriptor captured in the graph
    bool own_stream = false;
    int device = 0;                        // device current when the batch was created
    ~sim_batch() {
        if (pool) rtl::pool_extra_free(pool);
        if (graph) cudaGraphExecDestroy(graph);
        if (pgraph) cudaGraphExecDestroy(pgraph);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
    // copies ordered on the batch's stream, complete on return
    int h2d(void* dst, const void* src, size_t n) {
        if (!n) return SIM_OK;
        CUDA_TRY(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        return SIM_OK;
    }
    int d2h(void* dst, const void* src, size_t n) {
        if (!n) return SIM_OK;
        CUDA_TRY(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        return SIM_OK;
    }
};

namespace {
int ensure_compiled(sim_netlist* h, int mode, bool digest);
int create_instances(sim_netlist* nl, const sim_config& cfg, uint32_t n_inst, uint64_t seed, void* cuda_stream,
                     sim_batch** out);
}

extern "C" {

const char* sim_last_error(void) { return g_err.c_str(); }

void sim_config_default(sim_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->struct_size = sizeof(sim_config);
    cfg->mode = SIM_MODE_AUTO;
    cfg->kernel = SIM_KERNEL_PERSISTENT;
    cfg->timeout_ms = 2000;
    cfg->big_array_bytes = 128 * 1024;
}

int sim_load_netlist(const void* text, size_t len, const sim_config* cfg, sim_netlist** out) {
    if (!text || !out) return set_err(SIM_ERR_BADARG, "null argument");
    *out = nullptr;
    try {
        std::unique_ptr<sim_netlist> h(new sim_netlist());
        sim_config_default(&h->cfg);
        if (cfg) {
            if (cfg->struct_size != sizeof(sim_config)) return set_err(SIM_ERR_BADARG, "sim_config.struct_size mismatch");
            h->cfg = *cfg;
        }
        std::string err;
        int rc = parse_netlist(static_cast<const char*>(text), len, h->nl, err);
        if (rc) return set_err(rc, err);
        PartitionConfig pc;
        pc.big_array_bytes = h->cfg.big_array_bytes;
        pc.stage3 = !h->cfg.disable_stage3;
        pc.random_seed = h->cfg.seed_partition;
        if (h->cfg.partitioner > SIM_PART_HYPERGRAPH) return set_err(SIM_ERR_BADARG, "unknown partitioner");
        pc.hypergraph = h->cfg.partitioner == SIM_PART_HYPERGRAPH;
        uint32_t target = h->cfg.target_processes;
        // defaults measured on GB300: one process per warp of 8-warp CTAs for a
        // single instance; with lane = instance four processes per SM for the
        // bytecode and two for generated code (fewer fibers duplicated across
        // processes: mid x 4,096 15.0-15.2M against 14.2-14.4M
        // instance-cycles/s at four); with cluster exchange one process per
        // warp of every resident cluster CTA
        if (!target && h->cfg.cluster_size >= 2 && h->cfg.cluster_size <= 16) {
            const uint32_t W = h->cfg.warps_per_cta ? h->cfg.warps_per_cta : 8;
            target = uint32_t(resident_clusters(h->cfg.cluster_size, W)) * h->cfg.cluster_size * W;
        }
        const bool adaptive = !target && h->cfg.mode != SIM_MODE_LANE_INST;
        if (!target)
            target = uint32_t(sm_count()) *
                     (h->cfg.mode == SIM_MODE_LANE_INST && h->cfg.lowering == SIM_LOWER_GENERATED ? 2 : 4);
        pc.target = target;
        rc = partition(h->nl, pc, h->part, err);
        if (rc) return set_err(rc, err);
        // one instance: four processes per SM unless merging that far leaves a
        // straggler well above the slowest fiber (the t_comp bound of the
        // partition); then eight.  Measured on GB300: the 200k-op netlist
        // reaches its bound at four (fewer warps per SM, shorter steps), the
        // 2M-op mesh keeps gaining up to eight.
        if (adaptive && h->part.proc_cost_max * 4 > h->part.fiber_cost_max * 5) {
            pc.target = uint32_t(sm_count()) * 8;
            rc = partition(h->nl, pc, h->part, err);
            if (rc) return set_err(rc, err);
        }
        if (h->cfg.chain > kChainMax) return set_err(SIM_ERR_BADARG, "chain must be 0, 1 or 2");
        rc = lower(h->nl, h->part, h->low, err, h->cfg.chain);
        if (rc) return set_err(rc, err);
        if (h->cfg.cluster_size) {
            const uint32_t C = h->cfg.cluster_size;
            if (C < 2 || C > 16) return set_err(SIM_ERR_BADARG, "cluster_size must be 0 or 2..16");
            if (h->cfg.mode == SIM_MODE_LANE_INST || h->cfg.lowering == SIM_LOWER_GENERATED)
                return set_err(SIM_ERR_BADARG, "cluster exchange runs the per-operation bytecode (LANE_OP)");
            if (h->cfg.kernel != SIM_KERNEL_PERSISTENT)
                return set_err(SIM_ERR_BADARG, "cluster exchange runs the persistent kernel");
            const uint32_t W = h->cfg.warps_per_cta ? h->cfg.warps_per_cta : 8;
            if (W > 32) return set_err(SIM_ERR_BADARG, "warps_per_cta above 32");
            rc = lower_clusters(h->nl, h->part, C, W, h->low, h->cplan, err, h->cfg.chain < 2);
            if (rc) return set_err(rc, err);
        }
        h->layout = reg_layout(h->nl);
        const Netlist& nl = h->nl;
        h->mport_off.assign(1, 0);
        for (auto& ports : nl.mem_ports) {
            for (int32_t p : ports) h->mport_id.push_back(uint32_t(p));
            h->mport_off.push_back(uint32_t(h->mport_id.size()));
        }
        h->mem_word_off.assign(1, 0);
        for (uint8_t lg : nl.mem_lg) h->mem_word_off.push_back(h->mem_word_off.back() + (1ULL << lg));
        sim_netlist_info& I = h->info;
        I.n_inputs = uint32_t(nl.in_w.size());
        I.n_regs = uint32_t(nl.reg_w.size());
        I.n_mems = uint32_t(nl.mem_lg.size());
        I.n_wports = uint32_t(nl.wports.size());
        I.n_nodes = nl.nodes.size();
        I.n_ops = nl.n_ops;
        I.n_fibers = uint32_t(h->part.fibers.size());
        I.n_processes = uint32_t(h->part.procs.size());
        I.fiber_cost_sum = h->part.fiber_cost_sum;
        I.fiber_cost_max = h->part.fiber_cost_max;
        I.process_cost_sum = h->part.proc_cost_sum;
        I.process_cost_max = h->part.proc_cost_max;
        I.max_bundles = h->low.max_bundles;
        I.max_slots = std::max(h->low.max_s_slots, h->low.max_b_slots);
        I.instr_count = h->low.b_ins.size();
        I.cut_words = h->part.cut_words;
        *out = h.release();
        return SIM_OK;
    } catch (const std::bad_alloc&) {
        return set_err(SIM_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return set_err(SIM_ERR_PARSE, e.what());
    }
}

int sim_netlist_get_info(const sim_netlist* nl, sim_netlist_info* out) {
    if (!nl || !out) return set_err(SIM_ERR_BADARG, "null argument");
    *out = nl->info;
    return SIM_OK;
}

void sim_netlist_destroy(sim_netlist* nl) { delete nl; }

int sim_netlist_compile_generated(sim_netlist* nl, int32_t mode, double* seconds, int32_t* cached) {
    if (!nl || (mode != SIM_MODE_LANE_OP && mode != SIM_MODE_LANE_INST)) return set_err(SIM_ERR_BADARG, "bad argument");
    int rc = ensure_compiled(nl, mode, false);
    if (rc) return rc;
    if (seconds) *seconds = nl->gen_seconds[mode][0];
    if (cached) *cached = nl->gen_cached[mode][0] ? 1 : 0;
    return SIM_OK;
}

int sim_netlist_table(const sim_netlist* nl, int32_t which, void* out, size_t* bytes) {
    if (!nl || !bytes) return set_err(SIM_ERR_BADARG, "null argument");
    const Lowered& L = nl->low;
    const Partition& P = nl->part;
    std::vector<int32_t> i32;
    std::vector<uint64_t> u64;
    const void* src = nullptr;
    size_t n = 0;
    auto pick = [&](const auto& v) {
        src = v.data();
        n = v.size() * sizeof(v[0]);
    };
    switch (which) {
    case 0: pick(L.s_ins); break;
    case 1: pick(L.s_off); break;
    case 2: pick(L.s_len); break;
    case 3: pick(L.b_ins); break;
    case 4: pick(L.b_off); break;
    case 5: pick(L.b_len); break;
    case 6:
        i32.assign(P.fibers.size(), -1);
        for (size_t p = 0; p < P.procs.size(); p++)
            for (int32_t f : P.procs[p]) i32[f] = int32_t(p);
        pick(i32);
        break;
    case 7:
        for (auto& f : P.fibers) i32.push_back(f.reg >= 0 ? f.reg : -1 - f.mem);
        pick(i32);
        break;
    case 8:
        for (auto& f : P.fibers) u64.push_back(f.cost);
        pick(u64);
        break;
    case 9: pick(P.proc_cost); break;
    case 10: pick(nl->layout.cls); break;
    case 11: pick(nl->layout.idx); break;
    case 12: pick(L.s_slots); break;
    case 13: pick(L.b_slots); break;
    case 14: pick(L.c_words); break;
    case 15: pick(L.c_off); break;
    case 16: pick(L.c_size); break;
    case 17: pick(nl->cplan.warp_proc); break;
    case 18: pick(nl->cplan.mir_off); break;
    case 19: pick(nl->cplan.mir_reg); break;
    case 20: {
        const ClusterPlan& cp = nl->cplan;
        if (cp.C) u64 = {cp.C, cp.W, cp.grid, cp.mirror_words, cp.reads_local, cp.reads_remote};
        pick(u64);
        break;
    }
    case 21: pick(nl->nl.mem_lg); break;
    default: return set_err(SIM_ERR_BADARG, "unknown table");
    }
    if (out) memcpy(out, src, std::min(n, *bytes));
    *bytes = n;
    return SIM_OK;
}

}  // extern "C"

namespace {

// Generate and compile (once per lane mapping) the netlist's CUDA lowering.
int ensure_compiled(sim_netlist* h, int mode, bool digest) {
    std::lock_guard<std::mutex> g(h->gen_mu);
    if (!h->gen_cubin[mode][digest].empty()) return SIM_OK;
    std::vector<rtl::GenUnit> units;
    std::string err;
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int chunks = int(std::min<size_t>(std::max<size_t>(1, h->part.procs.size() / 16), size_t(hw) * 2));
    int rc = rtl::gen_cuda(h->nl, h->part, mode, digest, chunks, units, err);
    if (rc) return set_err(rc, err);
    if (const char* dump = getenv("RTLSIM_GEN_DUMP")) {     // developer aid: keep the generated sources
        for (auto& u : units) {
            FILE* f = fopen((std::string(dump) + "/" + u.name).c_str(), "w");
            if (f) {
                fwrite(u.source.data(), 1, u.source.size(), f);
                fclose(f);
            }
        }
    }
    const char* dir = getenv("RTLSIM_GENCACHE");
    std::string cache = dir ? dir : "";
    if (!cache.empty()) {
        std::string mk = "mkdir -p '" + cache + "'";
        if (system(mk.c_str()) != 0) cache.clear();
    }
    bool cached = false;
    double sec = 0;
    rc = rtl::jit_compile(units, cache, h->gen_cubin[mode][digest], &cached, &sec, err);
    if (rc) return set_err(rc, err);
    h->gen_seconds[mode][digest] = sec;
    h->gen_cached[mode][digest] = cached;
    return SIM_OK;
}

int ensure_loaded(sim_netlist* h, int mode, bool digest) {
    int rc = ensure_compiled(h, mode, digest);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(h->gen_mu);
    if (h->gen[mode][digest].lib) return SIM_OK;
    std::string err;
    rc = rtl::jit_load(h->gen_cubin[mode][digest], digest, h->gen[mode][digest], err);
    if (rc) return set_err(rc, err);
    return SIM_OK;
}

// Launch plan for generated code: no shared memory, occupancy from registers.
int plan_launch_gen(sim_batch* b) {
    const int sms = sm_count();
    const uint32_t n_proc = uint32_t(b->nl->part.procs.size());
    b->n_tasks = b->mode == SIM_MODE_LANE_INST ? n_proc * (b->I / 32) : n_proc * b->I;
    b->slot_words = 0;
    b->prog_words = 0;
    b->smem = 0;
    // generated kernels: up to 1024 threads per CTA at 64 registers per thread
    int warps = std::min(32, b->cfg.warps_per_cta ? int(b->cfg.warps_per_cta) : 8);
    b->warps = warps;
    b->threads = warps * 32;
    int occ = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, b->gen_kernel[b->cfg.digest_capacity > 0],
                                                           b->threads, 0));
    if (occ < 1) return set_err(SIM_ERR_CAPACITY, "generated kernel does not fit on an SM");
    b->max_grid = occ * sms;
    int need = int((b->n_tasks + warps - 1) / warps);
    b->grid = std::max(1, std::min(need, b->max_grid));
    return SIM_OK;
}

// Keep the device copy of the state view (read by generated code) current.
int sync_state_view(sim_batch* b) {
    if (!b->generated || memcmp(&b->S_uploaded, &b->S, sizeof(DevState)) == 0) return SIM_OK;
    int rc = b->h2d(b->S_dev.p, &b->S, sizeof(DevState));
    if (rc) return rc;
    b->S_uploaded = b->S;
    return SIM_OK;
}

cudaError_t launch_any(sim_batch* b, bool cooperative, int grid, const LaunchArgs& A) {
    if (b->cluster)
        return launch_cycles_cl(b->S.ring_cap > 0, grid, b->threads, b->smem, b->nl->cplan.C, b->stream, b->P, b->S, A);
    if (!b->generated)
        return launch_cycles(b->mode, b->S.ring_cap > 0, cooperative, grid, b->threads, b->smem, b->stream, b->P, b->S, A);
    const void* f = b->gen_kernel[b->S.ring_cap > 0 ? 1 : 0];
    const DevProg* Pd = b->P_dev.as<DevProg>();
    const DevState* Sd = b->S_dev.as<DevState>();
    LaunchArgs a = A;
    void* args[] = {&Pd, &Sd, &a};
    if (cooperative) return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(b->threads), args, 0, b->stream);
    return cudaLaunchKernel(f, dim3(grid), dim3(b->threads), args, 0, b->stream);
}

// Largest sum of compact-program sizes over the processes one warp owns
// (process p belongs to warp p mod total_warps), in 32-bit words.
uint32_t resident_words(const Lowered& L, uint32_t total_warps) {
    std::vector<uint64_t> per(std::min<size_t>(total_warps, L.c_size.size()), 0);
    for (size_t p = 0; p < L.c_size.size(); p++) per[p % per.size()] += L.c_size[p];
    uint64_t mx = 0;
    for (uint64_t v : per) mx = std::max(mx, v);
    return uint32_t(std::min<uint64_t>(mx, 0xffffffffu));
}

// Cluster exchange: one process per warp on the planned grid of clusters;
// slots, resident program and the two mirror buffers in shared memory.
int plan_launch_cluster(sim_batch* b) {
    const Lowered& L = b->nl->low;
    const ClusterPlan& cp = b->nl->cplan;
    const size_t smem_cap = smem_limit();
    b->warps = int(cp.W);
    b->threads = int(cp.W) * 32;
    b->grid = int(cp.grid);
    b->max_grid = b->grid;
    b->n_tasks = uint32_t(b->nl->part.procs.size());
    b->slot_words = (L.max_s_slots + 2) & ~1u;
    b->prog_words = 0;
    // pack each CTA's warps by their own process's slots (plus one spare) and
    // program; every area starts on 16 bytes (even slot words, programs in
    // multiples of 4 words)
    std::vector<uint32_t> warp_off(cp.warp_proc.size(), 0), warp_slots(cp.warp_proc.size(), 0);
    uint64_t max_cta = 0;
    for (uint32_t c = 0; c < cp.grid; c++) {
        uint64_t off = 0;
        for (uint32_t w = 0; w < cp.W; w++) {
            const size_t i = size_t(c) * cp.W + w;
            const uint32_t p = cp.warp_proc[i];
            warp_off[i] = uint32_t(off);
            if (p == kNoProc) continue;
            warp_slots[i] = (L.s_slots[p] + 2) & ~1u;
            off += warp_slots[i] + L.c_size[p] / 2;
        }
        max_cta = std::max(max_cta, off);
    }
    b->mirror_off = uint32_t(max_cta);
    b->smem = size_t(max_cta) * 8 + size_t(cp.mirror_words) * 16;
    b->smem = std::max(b->smem, kClusterCtaSmemMin);
    if (b->smem > smem_cap)
        return set_err(SIM_ERR_CAPACITY, "cluster CTA needs " + std::to_string(b->smem) +
                                             " bytes of shared memory (limit " + std::to_string(smem_cap) + ")");
    CUDA_TRY(prepare_cluster_kernel(b->smem, cp.C));
    int n_clusters = 0;
    CUDA_TRY(occupancy_clusters(b->grid, b->threads, b->smem, cp.C, &n_clusters));
    if (uint64_t(n_clusters) * cp.C < uint64_t(b->grid))
        return set_err(SIM_ERR_CAPACITY, std::to_string(cp.grid / cp.C) + " clusters of " + std::to_string(cp.C) +
                                             " CTAs requested, " + std::to_string(n_clusters) + " can be resident");
    int rc;
    if ((rc = upload(b->warp_off, warp_off, b->stream)) || (rc = upload(b->warp_slots, warp_slots, b->stream))) return rc;
    b->P.warp_off = b->warp_off.as<uint32_t>();
    b->P.warp_slots = b->warp_slots.as<uint32_t>();
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->cluster = true;
    return SIM_OK;
}

// Choose warps per CTA and grid for a batch (both lane mappings).  LANE_OP
// keeps each warp's programs resident in shared memory when they fit.
int plan_launch(sim_batch* b) {
    const Lowered& L = b->nl->low;
    const int sms = sm_count();
    const size_t smem_cap = smem_limit();
    const uint32_t n_proc = uint32_t(b->nl->part.procs.size());
    if (b->mode == SIM_MODE_LANE_INST) {
        b->slot_words = L.max_b_slots * 32;
        b->n_tasks = n_proc * (b->I / 32);
    } else {
        b->slot_words = (L.max_s_slots + 2) & ~1u;   // at least one spare slot (the operator steps' dummy)
        b->n_tasks = n_proc * b->I;
    }
    size_t slot_bytes = size_t(b->slot_words) * 8;
    if (slot_bytes > smem_cap)
        return set_err(SIM_ERR_CAPACITY, "a process needs " + std::to_string(slot_bytes) +
                                             " bytes of value slots per warp (limit " + std::to_string(smem_cap) + ")");
    int warps = b->cfg.warps_per_cta ? int(b->cfg.warps_per_cta) : 8;
    if (!b->cfg.warps_per_cta && b->mode == SIM_MODE_LANE_OP)   // one process per warp, one CTA per SM
        warps = int(std::min<uint64_t>(16, std::max<uint64_t>(1, (uint64_t(n_proc) * b->I + sms - 1) / sms)));
    while (warps > 1 && size_t(warps) * slot_bytes > smem_cap) warps /= 2;
    b->warps = warps;
    b->threads = warps * 32;
    b->prog_words = 0;
    int occ = 0;
    if (b->mode == SIM_MODE_LANE_OP) {
        // one process per warp when the grid allows it; re-plan with the
        // smaller grid if the resident programs lower occupancy
        uint32_t grid = (n_proc + warps - 1) / warps;
        for (int iter = 0; iter < 3; iter++) {
            uint32_t pw = (resident_words(L, grid * warps) + 3) & ~3u;
            size_t smem = size_t(warps) * (slot_bytes + size_t(pw) * 4);
            if (smem > smem_cap) break;
            CUDA_TRY(prepare_cycles_kernel(b->mode, smem));
            CUDA_TRY(occupancy_cycles(b->mode, b->threads, smem, &occ));
            if (occ < 1) break;
            uint32_t max_grid = uint32_t(occ * sms);
            if (grid <= max_grid) {
                b->prog_words = pw;
                b->smem = smem;
                b->max_grid = int(max_grid);
                b->grid = int(grid);
                return SIM_OK;
            }
            grid = max_grid;
        }
    }
    b->smem = size_t(warps) * slot_bytes;
    CUDA_TRY(prepare_cycles_kernel(b->mode, b->smem));
    CUDA_TRY(occupancy_cycles(b->mode, b->threads, b->smem, &occ));
    if (occ < 1) return set_err(SIM_ERR_CAPACITY, "kernel does not fit on an SM");
    b->max_grid = occ * sms;
    int need = int((b->n_tasks + warps - 1) / warps);
    b->grid = std::max(1, std::min(need, b->max_grid));
    return SIM_OK;
}

int upload_program(sim_batch* b) {
    sim_netlist* h = b->nl;
    const Netlist& nl = h->nl;
    const Lowered& L = h->low;
    cudaStream_t st = b->stream;
    int rc;
    std::vector<uint64_t> mem_base(nl.mem_lg.size());
    for (size_t m = 0; m < nl.mem_lg.size(); m++) mem_base[m] = h->mem_word_off[m] * b->I;
    if ((rc = upload(b->s_ins, L.s_ins, st)) || (rc = upload(b->s_off, L.s_off, st)) || (rc = upload(b->s_len, L.s_len, st)) ||
        (rc = upload(b->c_words, L.c_words, st)) || (rc = upload(b->c_off, L.c_off, st)) ||
        (rc = upload(b->c_size, L.c_size, st)) ||
        (rc = upload(b->b_ins, L.b_ins, st)) || (rc = upload(b->b_off, L.b_off, st)) || (rc = upload(b->b_len, L.b_len, st)) ||
        (rc = upload(b->mport_off, h->mport_off, st)) || (rc = upload(b->mport_id, h->mport_id, st)) ||
        (rc = upload(b->mem_lg, nl.mem_lg, st)) || (rc = upload(b->mem_w, nl.mem_w, st)) ||
        (rc = upload(b->mem_base, mem_base, st)) || (rc = upload(b->in_w, nl.in_w, st)) ||
        (rc = upload(b->reg_cls, h->layout.cls, st)) || (rc = upload(b->reg_idx, h->layout.idx, st)) ||
        (rc = upload(b->mem_word_off, h->mem_word_off, st)) || (rc = upload(b->warp_proc, h->cplan.warp_proc, st)) ||
        (rc = upload(b->mir_off, h->cplan.mir_off, st)) || (rc = upload(b->mir_reg, h->cplan.mir_reg, st)))
        return rc;
    DevProg& P = b->P;
    P.s_ins = b->s_ins.as<DIns>();
    P.s_off = b->s_off.as<uint32_t>();
    P.s_len = b->s_len.as<uint32_t>();
    P.c_words = b->c_words.as<uint32_t>();
    P.c_off = b->c_off.as<uint32_t>();
    P.c_size = b->c_size.as<uint32_t>();
    P.b_ins = b->b_ins.as<DIns>();
    P.b_off = b->b_off.as<uint32_t>();
    P.b_len = b->b_len.as<uint32_t>();
    P.mport_off = b->mport_off.as<uint32_t>();
    P.mport_id = b->mport_id.as<uint32_t>();
    P.mem_lg = b->mem_lg.as<uint8_t>();
    P.mem_w = b->mem_w.as<uint8_t>();
    P.mem_base = b->mem_base.as<uint64_t>();
    P.in_w = b->in_w.as<uint8_t>();
    P.reg_cls = b->reg_cls.as<uint8_t>();
    P.reg_idx = b->reg_idx.as<uint32_t>();
    P.warp_proc = b->warp_proc.as<uint32_t>();
    P.mir_off = b->mir_off.as<uint32_t>();
    P.mir_reg = b->mir_reg.as<uint32_t>();
    P.n_proc = uint32_t(h->part.procs.size());
    P.n_in = uint32_t(nl.in_w.size());
    P.n_reg = uint32_t(nl.reg_w.size());
    P.n_mem = uint32_t(nl.mem_lg.size());
    P.n_wport = uint32_t(nl.wports.size());
    return SIM_OK;
}

// Initial state: register init values, memory images, keys, digests.
int init_state(sim_batch* b) {
    sim_netlist* h = b->nl;
    const Netlist& nl = h->nl;
    const RegLayout& L = h->layout;
    cudaStream_t st = b->stream;
    const uint64_t I = b->I;
    DevState& S = b->S;
    S.I = b->I;
    S.pack = b->mode == SIM_MODE_LANE_INST ? 32 : 1;
    S.bit_stride = uint32_t((I + S.pack - 1) / S.pack);
    int rc;
    for (int k = 0; k < 2; k++) {
        if ((rc = b->bits[k].alloc(size_t(L.count[RC_BIT]) * S.bit_stride * 4)) ||
            (rc = b->w32[k].alloc(size_t(L.count[RC_W32]) * I * 4)) || (rc = b->w64[k].alloc(size_t(L.count[RC_W64]) * I * 8)) ||
            (rc = b->rec[k].alloc(nl.wports.size() * I * 16)))
            return rc;
        S.bits[k] = b->bits[k].as<uint32_t>();
        S.w32[k] = b->w32[k].as<uint32_t>();
        S.w64[k] = b->w64[k].as<uint64_t>();
        S.rec[k] = b->rec[k].as<uint64_t>();
        if (b->rec[k].n) CUDA_TRY(cudaMemsetAsync(b->rec[k].p, 0, b->rec[k].n, st));
    }
    // register planes of buffer 0 from init values (host-built, one plane at a time)
    {
        std::vector<uint32_t> bitw(size_t(L.count[RC_BIT]) * S.bit_stride);
        std::vector<uint32_t> w32(size_t(L.count[RC_W32]) * I);
        std::vector<uint64_t> w64(size_t(L.count[RC_W64]) * I);
        for (size_t r = 0; r < nl.reg_w.size(); r++) {
            uint64_t v = nl.reg_init[r];
            uint32_t ix = L.idx[r];
            if (L.cls[r] == RC_W64) std::fill(w64.begin() + size_t(ix) * I, w64.begin() + size_t(ix + 1) * I, v);
            else if (L.cls[r] == RC_W32) std::fill(w32.begin() + size_t(ix) * I, w32.begin() + size_t(ix + 1) * I, uint32_t(v));
            else {
                uint32_t word = (v & 1) ? (S.pack == 32 ? 0xffffffffu : 1u) : 0u;
                std::fill(bitw.begin() + size_t(ix) * S.bit_stride, bitw.begin() + size_t(ix + 1) * S.bit_stride, word);
            }
        }
        if (!bitw.empty()) CUDA_TRY(cudaMemcpyAsync(S.bits[0], bitw.data(), bitw.size() * 4, cudaMemcpyHostToDevice, st));
        if (!w32.empty()) CUDA_TRY(cudaMemcpyAsync(S.w32[0], w32.data(), w32.size() * 4, cudaMemcpyHostToDevice, st));
        if (!w64.empty()) CUDA_TRY(cudaMemcpyAsync(S.w64[0], w64.data(), w64.size() * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    // memories
    const uint64_t words = h->mem_word_off.back();
    if ((rc = b->mem.alloc(size_t(words) * I * 8))) return rc;
    S.mem = b->mem.as<uint64_t>();
    if (b->mem.n) {
        CUDA_TRY(cudaMemsetAsync(S.mem, 0, b->mem.n, st));
        std::vector<uint64_t> row(I);
        for (size_t m = 0; m < nl.mem_lg.size(); m++)
            for (auto& [a, v] : nl.mem_init[m]) {
                std::fill(row.begin(), row.end(), v);
                CUDA_TRY(cudaMemcpyAsync(S.mem + (h->mem_word_off[m] + a) * I, row.data(), I * 8, cudaMemcpyHostToDevice, st));
                CUDA_TRY(cudaStreamSynchronize(st));
            }
    }
    // stimulus keys: output inst+1 of the SplitMix64 stream seeded with `seed`
    {
        std::vector<uint64_t> keys(I);
        for (uint64_t i = 0; i < I; i++) keys[i] = host_mix64(b->seed + (i + 1) * kGamma);
        if ((rc = upload(b->key, keys, st))) return rc;
        S.key = b->key.as<uint64_t>();
    }
    b->h_hold_flag.assign(nl.in_w.size() * I, 0);
    b->h_hold_val.assign(nl.in_w.size() * I, 0);
    if ((rc = upload(b->hold_flag, b->h_hold_flag, st)) || (rc = upload(b->hold_val, b->h_hold_val, st))) return rc;
    S.hold_flag = b->hold_flag.as<uint8_t>();
    S.hold_val = b->hold_val.as<uint64_t>();
    S.any_hold = 0;
    // memory digest part (same initial image in every instance)
    {
        std::vector<uint64_t> md(nl.mem_lg.size() * I);
        for (size_t m = 0; m < nl.mem_lg.size(); m++) {
            std::vector<uint64_t> img(1ULL << nl.mem_lg[m], 0);
            for (auto& [a, v] : nl.mem_init[m]) img[a] = v;
            uint64_t d = 0;
            for (uint64_t a = 0; a < img.size(); a++) d += host_mix64(mem_hash(m, a) ^ img[a]);
            std::fill(md.begin() + m * I, md.begin() + (m + 1) * I, d);
        }
        if ((rc = upload(b->mem_dig, md, st))) return rc;
        S.mem_dig = b->mem_dig.as<uint64_t>();
        // memories without write ports: their digest term is added each cycle by process 0
        std::vector<uint64_t> rd(I, 0);
        for (size_t m = 0; m < nl.mem_lg.size(); m++)
            if (nl.mem_ports[m].empty())
                for (uint64_t i = 0; i < I; i++) rd[i] += md[m * I + i];
        if ((rc = upload(b->rom_dig, rd, st))) return rc;
        S.rom_dig = b->rom_dig.as<uint64_t>();
    }
    if ((rc = b->bar.alloc(16)) || (rc = b->err.alloc(16)) || (rc = b->t0_dev.alloc(8))) return rc;
    S.bar = b->bar.as<uint32_t>();
    S.err = b->err.as<int32_t>();
    CUDA_TRY(cudaMemsetAsync(b->bar.p, 0, 16, st));
    CUDA_TRY(cudaMemsetAsync(b->err.p, 0, 16, st));
    CUDA_TRY(cudaMemsetAsync(b->t0_dev.p, 0, 8, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SIM_OK;
}

// Digest of the initial state (identical for every instance).
uint64_t initial_digest(const sim_netlist* h) {
    const Netlist& nl = h->nl;
    uint64_t d = 0;
    for (size_t r = 0; r < nl.reg_w.size(); r++) d += host_mix64(reg_hash(r) ^ nl.reg_init[r]);
    for (size_t m = 0; m < nl.mem_lg.size(); m++) {
        std::vector<uint64_t> img(1ULL << nl.mem_lg[m], 0);
        for (auto& [a, v] : nl.mem_init[m]) img[a] = v;
        for (uint64_t a = 0; a < img.size(); a++) d += host_mix64(mem_hash(m, a) ^ img[a]);
    }
    return d;
}

int setup_tracking(sim_batch* b, const std::vector<uint32_t>& insts) {
    const uint32_t cap = b->cfg.digest_capacity;
    DevState& S = b->S;
    b->tracked = insts;
    b->h_track.assign(b->I, -1);
    for (size_t k = 0; k < insts.size(); k++) b->h_track[insts[k]] = int32_t(k);
    int rc = upload(b->track, b->h_track, b->stream);
    if (rc) return rc;
    S.track = b->track.as<int32_t>();
    S.ring_cap = cap;
    S.n_tracked = uint32_t(insts.size());
    if (cap && !insts.empty()) {
        std::vector<uint64_t> ring(size_t(cap) * insts.size(), 0);
        uint64_t d0 = initial_digest(b->nl);
        for (size_t k = 0; k < insts.size(); k++) ring[k] = d0;   // state 0 in slot 0
        if ((rc = upload(b->ring, ring, b->stream))) return rc;
        S.ring = b->ring.as<uint64_t>();
    } else {
        S.ring_cap = 0;
        S.ring = nullptr;
    }
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return SIM_OK;
}

int check_err(sim_batch* b) {
    int32_t e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, b->err.p, 4, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (e) {
        CUDA_TRY(cudaMemsetAsync(b->err.p, 0, 4, b->stream));
        const std::string what = e == SIM_ERR_TIMEOUT ? "grid barrier wait timed out" : "device error";
        b->failed = true;
        b->fail_reason = what + " in the step ending at cycle " + std::to_string(b->cycle);
        return set_err(e, what);
    }
    return SIM_OK;
}

// A batch whose last launch failed holds a state part-way through a cycle.
int refuse_failed(const sim_batch* b) {
    if (!b->failed) return SIM_OK;
    return set_err(SIM_ERR_STATE, "batch failed (" + b->fail_reason + "): restore a checkpoint or recreate it");
}

LaunchArgs base_args(sim_batch* b) {
    LaunchArgs A{};
    A.t0_dev = nullptr;
    A.skip_cta = -1;
    A.timeout_ns = b->timeout_ns;
    A.warps_per_cta = uint32_t(b->warps);
    A.slot_words = b->slot_words;
    A.prog_words = b->prog_words;
    A.n_tasks = b->n_tasks;
    A.group = b->mode == SIM_MODE_LANE_INST ? 32 : 1;
    A.proc_major = b->proc_major;
    A.wave_groups = b->wave_groups;
    A.cta_major = b->cta_major;
    A.pairs = b->nl->cfg.chain >= 2 ? 1u : 0u;
    if (b->cluster) {
        A.cluster = b->nl->cplan.C;
        A.mirror_words = b->nl->cplan.mirror_words;
        A.one_cluster = uint32_t(b->grid) == b->nl->cplan.C;
        A.mirror_off = b->mirror_off;
        A.grid = uint32_t(b->grid);
        A.smem_bytes = uint32_t(b->smem);
    }
    return A;
}

// Zero the ring slots of cycles t0+1 .. t0+n before they are accumulated.
int clear_ring(sim_batch* b, uint64_t t0, uint64_t n) {
    DevState& S = b->S;
    if (!S.ring_cap) return SIM_OK;
    const size_t row = size_t(S.n_tracked) * 8;
    for (uint64_t t = t0 + 1; t <= t0 + n; t++) {
        uint64_t s = t % S.ring_cap;
        uint64_t run = std::min<uint64_t>(t0 + n - t + 1, S.ring_cap - s);
        CUDA_TRY(cudaMemsetAsync(S.ring + s * S.n_tracked, 0, row * run, b->stream));
        t += run - 1;
    }
    return SIM_OK;
}

int step_persistent(sim_batch* b, uint64_t n) {
    LaunchArgs A = base_args(b);
    if (b->cfg.phase_samples) {
        const uint32_t want = std::min<uint64_t>(b->cfg.phase_samples, n);
        const size_t bytes = size_t(b->cfg.phase_samples) * b->grid * 24;
        if (b->phase.n < bytes) {
            int rc = b->phase.alloc(bytes);
            if (rc) return rc;
        }
        A.phase = b->phase.as<uint64_t>();
        A.phase_n = want;
        b->phase_n = want;
        b->phase_grid = uint32_t(b->grid);
    }
    A.t0 = b->cycle;
    A.n = uint32_t(n);
    A.pending_first = 0;
    A.grid_sync = 1;
    A.skip_cta = b->skip_cta;
    if (b->skip_cta >= 0) A.timeout_ns = b->skip_timeout_ns;   // only the debug step waits less
    b->skip_cta = -1;
    CUDA_TRY(cudaMemsetAsync(b->bar.p, 0, 8, b->stream));
    int rc = sync_state_view(b);
    if (rc) return rc;
    if (b->S.stim[0]) {
        CUDA_TRY(launch_stim(b->stream, b->P, b->S, b->cycle, nullptr));
        b->kernels_launched++;
    }
    CUDA_TRY(launch_any(b, true, b->grid, A));
    b->kernels_launched++;
    return SIM_OK;
}

// Launch-per-cycle grid: one warp per task, except that resident LANE_OP
// programs were laid out for the planned grid.
int per_cycle_grid(sim_batch* b) {
    if (b->prog_words) return b->grid;
    return std::max(1, int((b->n_tasks + b->warps - 1) / b->warps));
}

// The persistent step captured into a CUDA graph (one graph per step length),
// replayed with the cycle base read from device memory.
int step_persistent_graph(sim_batch* b, uint64_t n) {
    int rc = sync_state_view(b);
    if (rc) return rc;
    if (b->skip_cta >= 0) return step_persistent(b, n);
    if (!b->pgraph || b->pgraph_n != n || b->pgraph_timeout != b->timeout_ns ||
        memcmp(&b->pgraph_state, &b->S, sizeof(DevState)) != 0) {
        if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
        b->pgraph = nullptr;
        b->pgraph_state = b->S;
        cudaGraph_t g;
        CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        LaunchArgs A = base_args(b);
        A.t0_dev = b->t0_dev.as<uint64_t>();
        A.t0 = 0;
        A.n = uint32_t(n);
        A.pending_first = 0;
        A.grid_sync = 1;
        cudaError_t e = cudaMemsetAsync(b->bar.p, 0, 8, b->stream);
        if (e == cudaSuccess) e = launch_stim(b->stream, b->P, b->S, 0, A.t0_dev);
        if (e == cudaSuccess) e = launch_any(b, true, b->grid, A);
        if (e == cudaSuccess) e = launch_advance(b->stream, b->t0_dev.as<uint64_t>(), n);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return set_err(SIM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        e = cudaGraphInstantiate(&b->pgraph, g, 0);
        cudaGraphDestroy(g);
        CUDA_TRY(e);
        b->pgraph_n = n;
        b->pgraph_timeout = b->timeout_ns;
    }
    CUDA_TRY(launch_set_u64(b->stream, b->t0_dev.as<uint64_t>(), b->cycle));
    CUDA_TRY(cudaGraphLaunch(b->pgraph, b->stream));
    b->kernels_launched += b->S.stim[0] ? 4 : 3;
    return SIM_OK;
}

int step_per_cycle(sim_batch* b, uint64_t n) {
    int rc = sync_state_view(b);
    if (rc) return rc;
    LaunchArgs A = base_args(b);
    A.n = 1;
    A.grid_sync = 0;
    int grid = per_cycle_grid(b);
    if (b->S.stim[0]) {
        CUDA_TRY(launch_stim(b->stream, b->P, b->S, b->cycle, nullptr));
        b->kernels_launched++;
    }
    for (uint64_t k = 0; k < n; k++) {
        A.t0 = b->cycle + k;
        A.pending_first = k > 0;
        CUDA_TRY(launch_any(b, false, grid, A));
    }
    CUDA_TRY(launch_commit(std::max(1, b->grid), b->stream, b->P, b->S, b->cycle + n, nullptr));
    b->kernels_launched += n + 1;
    return SIM_OK;
}

// Per-cycle launches replayed from a captured CUDA graph: one graph holds
// `chunk` cycle launches, the final commit and the advance of the device
// cycle base, so it can be replayed for any starting cycle.
int step_graph(sim_batch* b, uint64_t n) {
    const uint32_t chunk = 64;
    int src = sync_state_view(b);
    if (src) return src;
    if (!b->graph || b->graph_chunk != chunk || b->graph_tasks != b->n_tasks ||
        memcmp(&b->graph_state, &b->S, sizeof(DevState)) != 0) {
        b->graph_state = b->S;
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        cudaGraph_t g;
        CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        LaunchArgs A = base_args(b);
        A.t0_dev = b->t0_dev.as<uint64_t>();
        A.n = 1;
        A.grid_sync = 0;
        int grid = per_cycle_grid(b);
        cudaError_t e = launch_stim(b->stream, b->P, b->S, 0, A.t0_dev);
        for (uint32_t k = 0; k < chunk && e == cudaSuccess; k++) {
            A.t0 = k;
            A.pending_first = k > 0;
            e = launch_any(b, false, grid, A);
        }
        if (e == cudaSuccess) e = launch_commit(std::max(1, b->grid), b->stream, b->P, b->S, chunk, A.t0_dev);
        if (e == cudaSuccess) e = launch_advance(b->stream, b->t0_dev.as<uint64_t>(), chunk);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return set_err(SIM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        CUDA_TRY(e);
        b->graph_chunk = chunk;
        b->graph_tasks = b->n_tasks;
    }
    uint64_t done = 0;
    CUDA_TRY(launch_set_u64(b->stream, b->t0_dev.as<uint64_t>(), b->cycle));
    b->kernels_launched++;
    while (n - done >= chunk) {
        CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
        b->kernels_launched += chunk + (b->S.stim[0] ? 3 : 2);
        done += chunk;
    }
    if (done < n) {
        uint64_t save = b->cycle;
        b->cycle += done;
        int rc = step_per_cycle(b, n - done);
        b->cycle = save;
        if (rc) return rc;
    }
    return SIM_OK;
}

sim_batch* B(void* p) { return static_cast<sim_batch*>(p); }

int check_inst(sim_batch* b, uint32_t inst) {
    if (!b) return set_err(SIM_ERR_BADARG, "null batch");
    if (inst >= b->n_inst) return set_err(SIM_ERR_BADARG, "instance out of range");
    return SIM_OK;
}

// Address of register r of `inst` in buffer par (device pointer, element size, bit).
void reg_addr(sim_batch* b, uint32_t par, uint32_t r, uint32_t inst, void** p, int* bytes, int* bit) {
    const RegLayout& L = b->nl->layout;
    uint64_t ix = L.idx[r];
    const DevState& S = b->S;
    *bit = -1;
    if (L.cls[r] == RC_W64) { *p = S.w64[par] + ix * S.I + inst; *bytes = 8; }
    else if (L.cls[r] == RC_W32) { *p = S.w32[par] + ix * S.I + inst; *bytes = 4; }
    else { *p = S.bits[par] + ix * S.bit_stride + inst / S.pack; *bytes = 4; *bit = int(inst % S.pack); }
}

}  // namespace

extern "C" {

int sim_create_instances(sim_netlist* nl, uint32_t n_inst, uint64_t seed, void* cuda_stream, sim_batch** out) {
    if (!nl) return set_err(SIM_ERR_BADARG, "bad argument");
    return create_instances(nl, nl->cfg, n_inst, seed, cuda_stream, out);
}

}  // extern "C"

namespace {

// sim_create_instances with an explicit configuration (server pools override
// the lane mapping, kernel and digests without touching the netlist's).
int create_instances(sim_netlist* nl, const sim_config& cfg, uint32_t n_inst, uint64_t seed, void* cuda_stream,
                     sim_batch** out) {
    if (!nl || !out || n_inst == 0) return set_err(SIM_ERR_BADARG, "bad argument");
    *out = nullptr;
    try {
        std::unique_ptr<sim_batch> b(new sim_batch());
        b->nl = nl;
        b->cfg = cfg;
        CUDA_TRY(cudaGetDevice(&b->device));
        b->stream = static_cast<cudaStream_t>(cuda_stream);
        if (!b->stream) {     // a private stream (graph capture needs a non-legacy stream)
            CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
            b->own_stream = true;
        }
        b->n_inst = n_inst;
        b->seed = seed;
        b->mode = cfg.mode == SIM_MODE_AUTO ? (n_inst >= 32 ? SIM_MODE_LANE_INST : SIM_MODE_LANE_OP) : cfg.mode;
        b->kernel = cfg.kernel;
        b->I = b->mode == SIM_MODE_LANE_INST ? (n_inst + 31) / 32 * 32 : n_inst;
        b->timeout_ns = uint64_t(cfg.timeout_ms ? cfg.timeout_ms : 2000) * 1000000ULL;
        // lane = instance: process-major task order unless the config asks otherwise
        b->proc_major = cfg.task_order == SIM_ORDER_PROCESS_MAJOR || cfg.task_order == SIM_ORDER_CTA_MAJOR ||
                        (cfg.task_order == SIM_ORDER_AUTO && b->mode == SIM_MODE_LANE_INST);
        // waves trade code reuse for L2 reuse of the state; measured on the
        // 4096-instance mid batch, code reuse wins (one wave of all groups)
        b->wave_groups = cfg.wave_groups;
        b->cta_major = cfg.task_order == SIM_ORDER_CTA_MAJOR;
        int rc;
        if (cfg.cluster_size && (n_inst != 1 || b->mode != SIM_MODE_LANE_OP))
            return set_err(SIM_ERR_BADARG, "a netlist lowered for cluster exchange runs one instance (LANE_OP)");
        if ((rc = upload_program(b.get())) || (rc = init_state(b.get()))) return rc;
        if (cfg.cluster_size) {
            if ((rc = plan_launch_cluster(b.get()))) return rc;
        } else if (cfg.lowering == SIM_LOWER_GENERATED) {
            // the module whose process functions carry digest code only when
            // this batch keeps per-cycle digests
            const bool dig = cfg.digest_capacity > 0;
            if ((rc = ensure_loaded(nl, b->mode, dig))) return rc;
            b->generated = true;
            b->gen_kernel[dig] = reinterpret_cast<const void*>(nl->gen[b->mode][dig].kernel);
            // the input values of the current and the next cycle (generated
            // process functions read them instead of hashing every input)
            const size_t n_in = nl->nl.in_w.size();
            if (n_in) {
                if ((rc = b->stim.alloc(2 * n_in * size_t(b->I) * 8))) return rc;
                b->S.stim[0] = b->stim.as<uint64_t>();
                b->S.stim[1] = b->S.stim[0] + n_in * size_t(b->I);
            }
            if ((rc = b->P_dev.alloc(sizeof(DevProg))) || (rc = b->S_dev.alloc(sizeof(DevState))) ||
                (rc = b->h2d(b->P_dev.p, &b->P, sizeof(DevProg))) || (rc = plan_launch_gen(b.get())))
                return rc;
        } else if ((rc = plan_launch(b.get()))) {
            return rc;
        }
        if ((rc = setup_tracking(b.get(), {0}))) return rc;
        *out = b.release();
        return SIM_OK;
    } catch (const std::bad_alloc&) {
        return set_err(SIM_ERR_OOM, "host allocation failed");
    }
}

}  // namespace

extern "C" {

void sim_batch_destroy(sim_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    delete b;
}

int sim_track_digests(sim_batch* b, const uint32_t* insts, uint32_t n) {
    if (!b || (n && !insts)) return set_err(SIM_ERR_BADARG, "bad argument");
    if (b->cycle != 0) return set_err(SIM_ERR_STATE, "digest tracking must be set before the first step");
    std::vector<uint32_t> v(insts, insts + n);
    for (uint32_t i : v)
        if (i >= b->n_inst) return set_err(SIM_ERR_BADARG, "tracked instance out of range");
    return setup_tracking(b, v);
}

int sim_step(sim_batch* b, uint64_t n_cycles) {
    if (!b) return set_err(SIM_ERR_BADARG, "null batch");
    if (int rc = refuse_failed(b)) return rc;
    if (n_cycles == 0) return SIM_OK;
    const uint32_t cap = b->S.ring_cap;
    uint64_t left = n_cycles;
    while (left) {
        // with digests on, a launch may not wrap the ring
        uint64_t n = cap ? std::min<uint64_t>(left, cap - 1) : std::min<uint64_t>(left, 1u << 30);
        int rc = clear_ring(b, b->cycle, n);
        if (rc) return rc;
        if (b->kernel == SIM_KERNEL_PER_CYCLE) rc = step_per_cycle(b, n);
        else if (b->kernel == SIM_KERNEL_PER_CYCLE_GRAPH) rc = step_graph(b, n);
        else if (b->kernel == SIM_KERNEL_PERSISTENT_GRAPH) rc = step_persistent_graph(b, n);
        else rc = step_persistent(b, n);
        if (rc) return rc;
        b->cycle += n;
        left -= n;
    }
    return SIM_OK;
}

int sim_sync(sim_batch* b) {
    if (!b) return set_err(SIM_ERR_BADARG, "null batch");
    if (int rc = refuse_failed(b)) return rc;
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return check_err(b);
}

int sim_cycle(sim_batch* b, uint64_t* out) {
    if (!b || !out) return set_err(SIM_ERR_BADARG, "null argument");
    *out = b->cycle;
    return SIM_OK;
}

int sim_poke(sim_batch* b, uint32_t inst, int32_t kind, uint32_t index, uint64_t value) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    const Netlist& nl = b->nl->nl;
    rc = sim_sync(b);
    if (rc) return rc;
    if (kind == SIM_SIG_INPUT) {
        if (index >= nl.in_w.size()) return set_err(SIM_ERR_BADARG, "input out of range");
        size_t j = size_t(index) * b->I + inst;
        b->h_hold_flag[j] = 1;
        b->h_hold_val[j] = value & mask_w(nl.in_w[index]);
        CUDA_TRY(cudaMemcpyAsync(b->hold_flag.as<uint8_t>() + j, &b->h_hold_flag[j], 1, cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaMemcpyAsync(b->hold_val.as<uint64_t>() + j, &b->h_hold_val[j], 8, cudaMemcpyHostToDevice, b->stream));
        b->S.any_hold = 1;
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        return SIM_OK;
    }
    if (kind != SIM_SIG_REG) return set_err(SIM_ERR_BADARG, "bad signal kind");
    if (index >= nl.reg_w.size()) return set_err(SIM_ERR_BADARG, "register out of range");
    value &= mask_w(nl.reg_w[index]);
    void* p;
    int bytes, bit;
    reg_addr(b, uint32_t(b->cycle & 1), index, inst, &p, &bytes, &bit);
    if (bit < 0) {
        if ((rc = b->h2d(p, &value, bytes))) return rc;
    } else {
        uint32_t word;
        if ((rc = b->d2h(&word, p, 4))) return rc;
        word = (word & ~(1u << bit)) | (uint32_t(value & 1) << bit);
        if ((rc = b->h2d(p, &word, 4))) return rc;
    }
    return SIM_OK;
}

int sim_unpoke(sim_batch* b, uint32_t inst, uint32_t input) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    if (input >= b->nl->nl.in_w.size()) return set_err(SIM_ERR_BADARG, "input out of range");
    rc = sim_sync(b);
    if (rc) return rc;
    size_t j = size_t(input) * b->I + inst;
    b->h_hold_flag[j] = 0;
    if ((rc = b->h2d(b->hold_flag.as<uint8_t>() + j, &b->h_hold_flag[j], 1))) return rc;
    b->S.any_hold = std::any_of(b->h_hold_flag.begin(), b->h_hold_flag.end(), [](uint8_t f) { return f != 0; });
    return SIM_OK;
}

int sim_poke_mem(sim_batch* b, uint32_t inst, uint32_t mem, uint64_t addr, uint64_t value) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    const Netlist& nl = b->nl->nl;
    if (mem >= nl.mem_lg.size() || addr >= (1ULL << nl.mem_lg[mem])) return set_err(SIM_ERR_BADARG, "memory address out of range");
    rc = sim_sync(b);
    if (rc) return rc;
    value &= mask_w(nl.mem_w[mem]);
    uint64_t* cell = b->S.mem + (b->nl->mem_word_off[mem] + addr) * b->I + inst;
    uint64_t old, md;
    if ((rc = b->d2h(&old, cell, 8))) return rc;
    if ((rc = b->h2d(cell, &value, 8))) return rc;
    uint64_t* mdp = b->S.mem_dig + size_t(mem) * b->I + inst;
    if ((rc = b->d2h(&md, mdp, 8))) return rc;
    uint64_t delta = host_mix64(mem_hash(mem, addr) ^ value) - host_mix64(mem_hash(mem, addr) ^ old);
    md += delta;
    if ((rc = b->h2d(mdp, &md, 8))) return rc;
    if (nl.mem_ports[mem].empty()) {
        uint64_t rd;
        uint64_t* rdp = b->rom_dig.as<uint64_t>() + inst;
        if ((rc = b->d2h(&rd, rdp, 8))) return rc;
        rd += delta;
        if ((rc = b->h2d(rdp, &rd, 8))) return rc;
    }
    return SIM_OK;
}

int sim_peek(sim_batch* b, uint32_t inst, int32_t kind, uint32_t index, uint64_t* out) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    if (!out) return set_err(SIM_ERR_BADARG, "null output");
    const Netlist& nl = b->nl->nl;
    rc = sim_sync(b);
    if (rc) return rc;
    if (kind == SIM_SIG_INPUT) {
        if (index >= nl.in_w.size()) return set_err(SIM_ERR_BADARG, "input out of range");
        size_t j = size_t(index) * b->I + inst;
        if (b->h_hold_flag[j]) *out = b->h_hold_val[j];
        else {
            uint64_t key = host_mix64(b->seed + (uint64_t(inst) + 1) * kGamma);
            *out = host_mix64(key + (b->cycle * nl.in_w.size() + index + 1) * kGamma) & mask_w(nl.in_w[index]);
        }
        return SIM_OK;
    }
    if (kind != SIM_SIG_REG) return set_err(SIM_ERR_BADARG, "bad signal kind");
    if (index >= nl.reg_w.size()) return set_err(SIM_ERR_BADARG, "register out of range");
    void* p;
    int bytes, bit;
    reg_addr(b, uint32_t(b->cycle & 1), index, inst, &p, &bytes, &bit);
    uint64_t v = 0;
    if ((rc = b->d2h(&v, p, bytes))) return rc;
    if (bit >= 0) v = (v >> bit) & 1;
    *out = v;
    return SIM_OK;
}

int sim_peek_mem(sim_batch* b, uint32_t inst, uint32_t mem, uint64_t addr, uint64_t* out) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    const Netlist& nl = b->nl->nl;
    if (!out || mem >= nl.mem_lg.size() || addr >= (1ULL << nl.mem_lg[mem])) return set_err(SIM_ERR_BADARG, "bad argument");
    rc = sim_sync(b);
    if (rc) return rc;
    if ((rc = b->d2h(out, b->S.mem + (b->nl->mem_word_off[mem] + addr) * b->I + inst, 8))) return rc;
    return SIM_OK;
}

int sim_peek_mems(sim_batch* b, uint32_t inst, uint32_t mem, uint64_t* out) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    const Netlist& nl = b->nl->nl;
    if (!out || mem >= nl.mem_lg.size()) return set_err(SIM_ERR_BADARG, "bad argument");
    rc = sim_sync(b);
    if (rc) return rc;
    const size_t depth = size_t(1) << nl.mem_lg[mem];
    // instance-minor layout: word a of instance inst is at (base + a) * I + inst
    CUDA_TRY(cudaMemcpy2DAsync(out, 8, b->S.mem + b->nl->mem_word_off[mem] * b->I + inst, size_t(b->I) * 8, 8, depth,
                               cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return SIM_OK;
}

int sim_peek_regs(sim_batch* b, uint32_t inst, uint64_t* out) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    if (!out) return set_err(SIM_ERR_BADARG, "null output");
    rc = sim_sync(b);
    if (rc) return rc;
    const RegLayout& L = b->nl->layout;
    const DevState& S = b->S;
    const uint32_t par = uint32_t(b->cycle & 1);
    std::vector<uint64_t> v64(L.count[RC_W64]);
    std::vector<uint32_t> v32(L.count[RC_W32]), v1(L.count[RC_BIT]);
    if (!v64.empty())
        CUDA_TRY(cudaMemcpy2DAsync(v64.data(), 8, S.w64[par] + inst, size_t(S.I) * 8, 8, v64.size(),
                                   cudaMemcpyDeviceToHost, b->stream));
    if (!v32.empty())
        CUDA_TRY(cudaMemcpy2DAsync(v32.data(), 4, S.w32[par] + inst, size_t(S.I) * 4, 4, v32.size(),
                                   cudaMemcpyDeviceToHost, b->stream));
    if (!v1.empty())
        CUDA_TRY(cudaMemcpy2DAsync(v1.data(), 4, S.bits[par] + inst / S.pack, size_t(S.bit_stride) * 4, 4, v1.size(),
                                   cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (size_t r = 0; r < L.cls.size(); r++) {
        uint32_t ix = L.idx[r];
        if (L.cls[r] == RC_W64) out[r] = v64[ix];
        else if (L.cls[r] == RC_W32) out[r] = v32[ix];
        else out[r] = (v1[ix] >> (inst % S.pack)) & 1;
    }
    return SIM_OK;
}

int sim_state_digests(sim_batch* b, uint64_t* out) {
    if (!b || !out) return set_err(SIM_ERR_BADARG, "null argument");
    int rc = sim_sync(b);
    if (rc) return rc;
    if (b->scratch.n < size_t(b->I) * 8)
        if ((rc = b->scratch.alloc(size_t(b->I) * 8))) return rc;
    uint64_t* d = b->scratch.as<uint64_t>();
    CUDA_TRY(cudaMemsetAsync(d, 0, size_t(b->I) * 8, b->stream));
    CUDA_TRY(launch_state_digest(b->stream, b->P, b->S, uint32_t(b->cycle & 1), b->mem_word_off.as<uint64_t>(),
                                 b->nl->mem_word_off.back(), d, b->I));
    b->kernels_launched++;
    CUDA_TRY(cudaMemcpyAsync(out, d, size_t(b->n_inst) * 8, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return SIM_OK;
}

int sim_digests(sim_batch* b, uint32_t inst, uint64_t first_cycle, uint64_t n, uint64_t* out) {
    int rc = check_inst(b, inst);
    if (rc) return rc;
    if (!out && n) return set_err(SIM_ERR_BADARG, "null output");
    const DevState& S = b->S;
    if (!S.ring_cap) return set_err(SIM_ERR_STATE, "digests are off (sim_config.digest_capacity = 0)");
    int col = b->h_track[inst];
    if (col < 0) return set_err(SIM_ERR_STATE, "instance is not tracked");
    if (n == 0) return SIM_OK;
    if (first_cycle + n - 1 > b->cycle || first_cycle + S.ring_cap <= b->cycle)
        return set_err(SIM_ERR_BADARG, "requested cycles are not in the digest ring");
    rc = sim_sync(b);
    if (rc) return rc;
    std::vector<uint64_t> ring(size_t(S.ring_cap) * S.n_tracked);
    if ((rc = b->d2h(ring.data(), S.ring, ring.size() * 8))) return rc;
    for (uint64_t k = 0; k < n; k++) out[k] = ring[((first_cycle + k) % S.ring_cap) * S.n_tracked + col];
    return SIM_OK;
}

int sim_step_host(sim_batch* b, uint64_t n_cycles, const uint64_t* held_inputs, uint64_t* out_digests) {
    if (!b || !out_digests) return set_err(SIM_ERR_BADARG, "null argument");
    const size_t n_in = b->nl->nl.in_w.size();
    if (held_inputs && n_in) {
        // host layout [inst][input] -> device [input][inst]
        for (size_t k = 0; k < n_in; k++)
            for (uint32_t i = 0; i < b->n_inst; i++) {
                b->h_hold_val[k * b->I + i] = held_inputs[size_t(i) * n_in + k] & mask_w(b->nl->nl.in_w[k]);
                b->h_hold_flag[k * b->I + i] = 1;
            }
        CUDA_TRY(cudaMemcpyAsync(b->hold_val.p, b->h_hold_val.data(), b->h_hold_val.size() * 8, cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaMemcpyAsync(b->hold_flag.p, b->h_hold_flag.data(), b->h_hold_flag.size(), cudaMemcpyHostToDevice, b->stream));
        b->S.any_hold = 1;
    }
    int rc = sim_step(b, n_cycles);
    if (rc) return rc;
    return sim_state_digests(b, out_digests);
}

// ---- checkpoints -----------------------------------------------------------
namespace {
struct BlobHeader {
    uint64_t magic, version, n_reg, n_mem_words, I, mode, cycle, n_in;
};
constexpr uint64_t kMagic = 0x314B505453525447ULL;
}  // namespace

int sim_save(sim_batch* b, void** blob, size_t* len) {
    if (!b || !blob || !len) return set_err(SIM_ERR_BADARG, "null argument");
    int rc = sim_sync(b);
    if (rc) return rc;
    const RegLayout& L = b->nl->layout;
    const DevState& S = b->S;
    const uint32_t par = uint32_t(b->cycle & 1);
    size_t nb = size_t(L.count[RC_BIT]) * S.bit_stride * 4, n32 = size_t(L.count[RC_W32]) * S.I * 4,
           n64 = size_t(L.count[RC_W64]) * S.I * 8, nm = b->mem.n, nmd = b->mem_dig.n, nh = b->h_hold_val.size();
    size_t total = sizeof(BlobHeader) + nb + n32 + n64 + nm + nmd + nh * 9;
    char* p = static_cast<char*>(malloc(total));
    if (!p) return set_err(SIM_ERR_OOM, "host allocation failed");
    BlobHeader h{kMagic, 1, b->nl->nl.reg_w.size(), b->nl->mem_word_off.back(), S.I, uint64_t(b->mode), b->cycle, b->nl->nl.in_w.size()};
    memcpy(p, &h, sizeof h);
    char* q = p + sizeof h;
    auto d2h = [&](const void* src, size_t n) {
        if (n && b->d2h(q, src, n) != SIM_OK) return false;
        q += n;
        return true;
    };
    if (!d2h(S.bits[par], nb) || !d2h(S.w32[par], n32) || !d2h(S.w64[par], n64) || !d2h(S.mem, nm) || !d2h(S.mem_dig, nmd)) {
        free(p);
        return set_err(SIM_ERR_CUDA, "checkpoint copy failed");
    }
    if (nh) {
        memcpy(q, b->h_hold_val.data(), nh * 8);
        q += nh * 8;
        memcpy(q, b->h_hold_flag.data(), nh);
    }
    *blob = p;
    *len = total;
    return SIM_OK;
}

int sim_restore(sim_batch* b, const void* blob, size_t len) {
    if (!b || !blob) return set_err(SIM_ERR_BADARG, "null argument");
    // a failed batch may be restored: wait for its stream and drop the error
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    int rc = check_err(b);
    if (rc && !b->failed) return rc;     // a runtime failure, not the launch's error word
    BlobHeader h;
    if (len < sizeof h) return set_err(SIM_ERR_BADARG, "checkpoint too short");
    memcpy(&h, blob, sizeof h);
    const RegLayout& L = b->nl->layout;
    DevState& S = b->S;
    if (h.magic != kMagic || h.version != 1 || h.n_reg != b->nl->nl.reg_w.size() || h.I != S.I ||
        h.mode != uint64_t(b->mode) || h.n_mem_words != b->nl->mem_word_off.back())
        return set_err(SIM_ERR_BADARG, "checkpoint does not match this batch");
    size_t nb = size_t(L.count[RC_BIT]) * S.bit_stride * 4, n32 = size_t(L.count[RC_W32]) * S.I * 4,
           n64 = size_t(L.count[RC_W64]) * S.I * 8, nm = b->mem.n, nmd = b->mem_dig.n, nh = b->h_hold_val.size();
    if (len != sizeof h + nb + n32 + n64 + nm + nmd + nh * 9) return set_err(SIM_ERR_BADARG, "checkpoint size mismatch");
    const uint32_t par = uint32_t(h.cycle & 1);
    const char* q = static_cast<const char*>(blob) + sizeof h;
    auto h2d = [&](void* dst, size_t n) {
        if (n && b->h2d(dst, q, n) != SIM_OK) return false;
        q += n;
        return true;
    };
    if (!h2d(S.bits[par], nb) || !h2d(S.w32[par], n32) || !h2d(S.w64[par], n64) || !h2d(S.mem, nm) || !h2d(S.mem_dig, nmd))
        return set_err(SIM_ERR_CUDA, "restore copy failed");
    if (nh) {
        memcpy(b->h_hold_val.data(), q, nh * 8);
        q += nh * 8;
        memcpy(b->h_hold_flag.data(), q, nh);
        if ((rc = b->h2d(b->hold_val.p, b->h_hold_val.data(), nh * 8))) return rc;
        if ((rc = b->h2d(b->hold_flag.p, b->h_hold_flag.data(), nh))) return rc;
        S.any_hold = std::any_of(b->h_hold_flag.begin(), b->h_hold_flag.end(), [](uint8_t f) { return f != 0; });
    }
    for (int k = 0; k < 2; k++)
        if (b->rec[k].n) CUDA_TRY(cudaMemsetAsync(b->rec[k].p, 0, b->rec[k].n, b->stream));
    b->cycle = h.cycle;
    b->failed = false;
    b->fail_reason.clear();
    return SIM_OK;
}

void sim_free_blob(void* blob) { free(blob); }

int sim_phase_times(sim_batch* b, uint32_t n, double* out) {
    if (!b || (n && !out)) return set_err(SIM_ERR_BADARG, "bad argument");
    if (n > b->phase_n) return set_err(SIM_ERR_STATE, "fewer cycles were recorded (set sim_config.phase_samples)");
    int rc = sim_sync(b);
    if (rc) return rc;
    std::vector<uint64_t> raw(size_t(n) * b->phase_grid * 3);
    if ((rc = b->d2h(raw.data(), b->phase.p, raw.size() * 8))) return rc;
    for (uint32_t c = 0; c < n; c++) {
        uint64_t start = ~0ULL, arrive = 0, release = 0;
        for (uint32_t k = 0; k < b->phase_grid; k++) {
            const uint64_t* r = &raw[(size_t(c) * b->phase_grid + k) * 3];
            start = std::min(start, r[0]);
            arrive = std::max(arrive, r[1]);
            release = std::max(release, r[2]);
        }
        out[c * 3 + 0] = double(arrive - start);
        out[c * 3 + 1] = double(release - arrive);
        out[c * 3 + 2] = double(release - start);
    }
    return SIM_OK;
}

int sim_launch_info(sim_batch* b, uint32_t* ctas, uint32_t* warps_per_cta, uint32_t* tasks_per_cycle,
                    uint64_t* kernels_launched) {
    if (!b) return set_err(SIM_ERR_BADARG, "null batch");
    if (ctas) *ctas = uint32_t(b->grid);
    if (warps_per_cta) *warps_per_cta = uint32_t(b->warps);
    if (tasks_per_cycle) *tasks_per_cycle = b->n_tasks;
    if (kernels_launched) *kernels_launched = b->kernels_launched;
    return SIM_OK;
}

int sim_debug_skip_arrival(sim_batch* b, uint32_t timeout_ms) {
    if (!b) return set_err(SIM_ERR_BADARG, "null batch");
    if (b->grid < 2) return set_err(SIM_ERR_STATE, "needs at least two CTAs");
    b->skip_cta = 0;
    b->skip_timeout_ns = uint64_t(timeout_ms) * 1000000ULL;
    return SIM_OK;
}

}  // extern "C"

// ---- internal views for noalloc.cu -------------------------------------------
namespace rtl {

int set_error(int code, const std::string& msg) { return set_err(code, msg); }

int batch_views(sim_batch* b, DevProg* P, DevState* S, const uint64_t** mem_word_off, uint64_t* mem_words, uint32_t* I,
                uint32_t* n_inst, uint32_t* par, cudaStream_t* stream, int* device) {
    if (!b) return set_err(SIM_ERR_BADARG, "null batch");
    *device = b->device;
    *P = b->P;
    *S = b->S;
    *mem_word_off = b->mem_word_off.as<uint64_t>();
    *mem_words = b->nl->mem_word_off.back();
    *I = b->I;
    *n_inst = b->n_inst;
    *par = uint32_t(b->cycle & 1);
    *stream = b->stream;
    return SIM_OK;
}

int batch_sync(sim_batch* b) { return sim_sync(b); }

}  // namespace rtl

// ---- instance pools for the server (pool.hpp) ---------------------------------
#include "pool.hpp"

namespace rtl {
cudaError_t launch_reset_slots(cudaStream_t st, const DevProg& P, const DevState& S, uint32_t par, uint32_t lo, uint32_t n,
                               const uint64_t* reg_init, const uint64_t* mem_image, const uint64_t* mem_word_off,
                               uint64_t mem_words, const uint64_t* mem_init_dig, uint64_t rom_init_dig);

struct PoolExtra {
    DBuf t_off, reg_init, mem_image, mem_init_dig;
    uint64_t rom_init_dig = 0;
};

size_t pool_footprint(const sim_netlist* h, uint32_t capacity) {
    const Netlist& nl = h->nl;
    const RegLayout& L = h->layout;
    uint64_t I = (uint64_t(capacity) + 31) / 32 * 32;
    uint64_t per = 2 * (uint64_t(L.count[RC_W64]) * 8 + uint64_t(L.count[RC_W32]) * 4 + (L.count[RC_BIT] + 7) / 8);
    // memories, write records, held inputs (value + flag) and, with generated
    // code, the input values of two cycles
    per += h->mem_word_off.back() * 8 + nl.wports.size() * 32 + nl.in_w.size() * (9 + 16) + nl.mem_lg.size() * 8 + 40;
    uint64_t prog = (h->low.s_ins.size() + h->low.b_ins.size()) * 16 + h->low.c_words.size() * 4;
    return size_t(per * I + prog + 2 * h->mem_word_off.back() * 8);
}

int pool_create(sim_netlist* nl, uint32_t capacity, bool persistent, sim_batch** out) {
    if (!nl || !out || capacity == 0) return set_err(SIM_ERR_BADARG, "bad argument");
    // a pool runs lane = instance with no digest ring, whatever the netlist
    // was loaded for (its LANE_INST program is always there, also when the
    // LANE_OP program was lowered for clusters): one persistent launch per
    // step, or per-cycle launches replayed from a graph
    sim_config cfg = nl->cfg;
    cfg.mode = SIM_MODE_LANE_INST;
    cfg.kernel = persistent ? SIM_KERNEL_PERSISTENT : SIM_KERNEL_PER_CYCLE_GRAPH;
    cfg.digest_capacity = 0;
    cfg.cluster_size = 0;
    int rc = create_instances(nl, cfg, capacity, 0, nullptr, out);
    if (rc) return rc;
    sim_batch* b = *out;
    std::unique_ptr<PoolExtra> x(new PoolExtra());
    const Netlist& N = nl->nl;
    std::vector<uint64_t> zeros(b->I, 0), image(nl->mem_word_off.back(), 0), mdig(N.mem_lg.size(), 0);
    for (size_t m = 0; m < N.mem_lg.size(); m++) {
        for (auto& [a, v] : N.mem_init[m]) image[nl->mem_word_off[m] + a] = v;
        uint64_t d = 0;
        for (uint64_t a = 0; a < (1ULL << N.mem_lg[m]); a++)
            d += host_mix64(mem_hash(m, a) ^ image[nl->mem_word_off[m] + a]);
        mdig[m] = d;
        if (N.mem_ports[m].empty()) x->rom_init_dig += d;
    }
    if ((rc = upload(x->t_off, zeros, b->stream)) || (rc = upload(x->reg_init, N.reg_init, b->stream)) ||
        (rc = upload(x->mem_image, image, b->stream)) || (rc = upload(x->mem_init_dig, mdig, b->stream))) {
        sim_batch_destroy(b);
        *out = nullptr;
        return rc;
    }
    b->S.t_off = x->t_off.as<uint64_t>();
    b->pool = x.release();
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return SIM_OK;
}

int pool_admit(sim_batch* b, uint32_t lo, uint32_t n, uint64_t seed) {
    if (!b || !b->pool || n == 0 || uint64_t(lo) + n > b->n_inst) return set_err(SIM_ERR_BADARG, "bad slot range");
    PoolExtra* x = b->pool;
    std::vector<uint64_t> keys(n), offs(n, b->cycle);
    for (uint32_t j = 0; j < n; j++) keys[j] = host_mix64(seed + (uint64_t(j) + 1) * kGamma);
    CUDA_TRY(cudaMemcpyAsync(b->key.as<uint64_t>() + lo, keys.data(), n * 8, cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaMemcpyAsync(x->t_off.as<uint64_t>() + lo, offs.data(), n * 8, cudaMemcpyHostToDevice, b->stream));
    for (size_t k = 0; k < b->nl->nl.in_w.size(); k++)
        std::fill(b->h_hold_flag.begin() + k * b->I + lo, b->h_hold_flag.begin() + k * b->I + lo + n, 0);
    CUDA_TRY(launch_reset_slots(b->stream, b->P, b->S, uint32_t(b->cycle & 1), lo, n, x->reg_init.as<uint64_t>(),
                                x->mem_image.as<uint64_t>(), b->mem_word_off.as<uint64_t>(), b->nl->mem_word_off.back(),
                                x->mem_init_dig.as<uint64_t>(), x->rom_init_dig));
    b->kernels_launched++;
    CUDA_TRY(cudaStreamSynchronize(b->stream));    // the host vectors above go out of scope
    return SIM_OK;
}

int pool_step(sim_batch* b, uint64_t n, uint64_t* kernels) {
    const uint64_t k0 = b->kernels_launched;
    int rc = sim_step(b, n);
    *kernels = b->kernels_launched - k0;
    return rc;
}

int pool_set_active(sim_batch* b, uint32_t n_groups, uint32_t share) {
    if (!b || !b->pool || b->mode != SIM_MODE_LANE_INST || n_groups == 0 || uint64_t(n_groups) * 32 > b->I)
        return set_err(SIM_ERR_BADARG, "bad active group count");
    b->n_tasks = uint32_t(b->nl->part.procs.size()) * n_groups;
    // a persistent step holds only the CTAs its tasks need, and at most its
    // share of the GPU, leaving the other SMs to the pools of other netlists
    const int cap = std::max(1, b->max_grid / int(std::max(1u, share)));
    b->grid = std::max(1, std::min(int((b->n_tasks + b->warps - 1) / b->warps), cap));
    return SIM_OK;
}

void pool_extra_free(PoolExtra* x) { delete x; }

int pool_digests(sim_batch* b, uint32_t lo, uint32_t n, uint64_t* out) {
    if (!b || uint64_t(lo) + n > b->n_inst) return set_err(SIM_ERR_BADARG, "bad slot range");
    std::vector<uint64_t> all(b->n_inst);
    int rc = sim_state_digests(b, all.data());
    if (rc) return rc;
    std::copy(all.begin() + lo, all.begin() + lo + n, out);
    return SIM_OK;
}

cudaStream_t pool_stream(sim_batch* b) { return b->stream; }
uint64_t pool_cycle(sim_batch* b) { return b->cycle; }

}  // namespace rtl
