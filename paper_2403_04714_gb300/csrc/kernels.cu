// kernels.cu -- sm_103a kernels of the BSP simulator.
//
// One simulated clock cycle (paper Sec. 3.2): every process reads *current*
// register values (buffer t&1), evaluates its fibers' nodes in dependence
// order, and writes *next* values (buffer (t+1)&1) and memory write records;
// then a barrier.  Double-buffered state makes the paper's two barriers per
// cycle (compute, exchange) one: next values are written straight into the
// buffer the consumers read after the barrier, so the exchange is the store
// itself (HBM/L2 between processes).  Memory writes travel as (en, addr,
// data) records, never whole arrays (differential exchange, Sec. 5.2): the
// records of cycle t are applied to the array by its owning process during
// cycle t+1, while readers in cycle t+1 forward from them, so every read sees
// the array as of the clock edge.
//
// Two lane mappings share one bytecode:
//   LANE_OP   warp = (process, instance); lanes run up to 32 independent
//             nodes of one schedule step, __syncwarp between steps.
//   LANE_INST warp = (process, 32 instances); lane = instance, uniform
//             control flow, instance-minor state (coalesced 128/256 B rows),
//             1-bit registers packed 32 instances per word with __ballot_sync.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/sim.h"
#include "device.hpp"
#include "sim_rt.cuh"

namespace rtl {

__device__ __forceinline__ uint4 ld_ins(const DIns* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

// ---------------------------------------------------------------------------
// Instruction semantics (shared by both lane mappings)
// ---------------------------------------------------------------------------
struct Dec {
    uint32_t op, w, dst, a, b, c, x, imm;
};

__device__ __forceinline__ Dec decode(uint4 r) {
    Dec d;
    d.op = r.x & 0xff;
    d.w = (r.x >> 8) & 0xff;
    d.dst = r.x >> 16;
    d.a = r.y & 0xffff;
    d.b = r.y >> 16;
    d.c = r.z & 0xffff;
    d.x = r.z >> 16;
    d.imm = r.w;
    return d;
}

__device__ __forceinline__ uint64_t alu(uint32_t op, uint64_t a, uint64_t b, uint64_t c, uint32_t x) {
    switch (op) {
    case D_ADD: return a + b;
    case D_SUB: return a - b;
    case D_MUL: return a * b;
    case D_AND: return a & b;
    case D_OR: return a | b;
    case D_XOR: return a ^ b;
    case D_SHL: return b >= 64 ? 0 : a << b;
    case D_SHR: return b >= 64 ? 0 : a >> b;
    case D_EQ: return a == b ? 1 : 0;
    case D_LT: return a < b ? 1 : 0;
    case D_MUX: return a != 0 ? b : c;
    case D_SLICE: return a >> x;           // lo < 64 (checked at load)
    case D_CONCAT: return (a << x) | b;    // width(b) < 64 (checked at load)
    default: return 0;
    }
}

// ---------------------------------------------------------------------------
// LANE_INST: one warp, one process, 32 instances (lane = instance).
// ---------------------------------------------------------------------------
template <bool DIGEST>
__device__ void task_lane_inst(const DevProg& P, const DevState& S, uint32_t p, uint32_t g, uint64_t t, bool pending,
                               uint64_t* __restrict__ sl, uint32_t lane) {
    const uint32_t inst = g * 32 + lane;
    const uint32_t par = uint32_t(t & 1), nxt = par ^ 1;
    const uint64_t key = S.key[inst];
    const int32_t col = DIGEST ? S.track[inst] : -1;
    uint64_t dacc = 0;
    const DIns* ip = P.b_ins + P.b_off[p];
    const uint32_t n = P.b_len[p];
#define SL(s) sl[(s) * 32 + lane]
    for (uint32_t i = 0; i < n; i++) {
        Dec d = decode(ld_ins(ip + i));
        switch (d.op) {
        case D_NOP:
            break;
        case D_LDR:
            SL(d.dst) = load_reg(S, par, d.c, d.b | (d.x << 16), inst);
            break;
        case D_LDI:
            SL(d.dst) = stimulus(P, S, key, d.imm, inst, t, d.w);
            break;
        case D_CONST:
            SL(d.dst) = (uint64_t)d.imm | ((uint64_t)d.a << 32) | ((uint64_t)d.b << 48);
            break;
        case D_MEMRD: {
            uint64_t addr = SL(d.a) & ((1ULL << P.mem_lg[d.imm]) - 1);
            SL(d.dst) = mem_read(P, S, d.imm, addr, inst, nxt, pending);
            break;
        }
        case D_STR: {
            uint64_t v = SL(d.a) & wmask(d.w);
            uint32_t idx = d.b | (d.x << 16);
            if (d.c == RC_W64) {
                S.w64[nxt][(uint64_t)idx * S.I + inst] = v;
            } else if (d.c == RC_W32) {
                S.w32[nxt][(uint64_t)idx * S.I + inst] = uint32_t(v);
            } else {
                uint32_t word = __ballot_sync(0xffffffffu, v & 1);
                if (lane == 0) S.bits[nxt][(uint64_t)idx * S.bit_stride + g] = word;
            }
            if (DIGEST && col >= 0) dacc += mix64(((uint64_t)d.imm * kGamma + 1ULL) ^ v);
            break;
        }
        case D_WREC: {
            uint64_t en = SL(d.a) != 0;
            uint64_t addr = SL(d.b) & ((1ULL << d.x) - 1);
            uint64_t data = SL(d.c) & wmask(d.w);
            uint64_t* r = S.rec[par] + ((uint64_t)d.imm * S.I + inst) * 2;
            r[0] = en ? ((1ULL << 63) | addr) : 0;
            r[1] = data;
            break;
        }
        case D_COMMIT:
            if (pending) {
                uint64_t delta = mem_commit(P, S, d.imm, inst, nxt, DIGEST && col >= 0);
                if (DIGEST) mem_digest_update(S, d.imm, inst, t, delta);
            }
            break;
        case D_MUX:
            SL(d.dst) = alu(D_MUX, SL(d.a), SL(d.b), SL(d.c), 0) & wmask(d.w);
            break;
        default:
            SL(d.dst) = alu(d.op, SL(d.a), SL(d.b), 0, d.x) & wmask(d.w);
        }
    }
#undef SL
    if (DIGEST && col >= 0) {
        if (p == 0) dacc += S.rom_dig[inst];    // memories without write ports never change in a step
        ring_add(S, t + 1, col, dacc);
    }
}

// ---------------------------------------------------------------------------
// Thread-block-cluster primitives (distributed shared memory, sm_90+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Store into the same shared-memory offset of CTA `rank` of this cluster.
__device__ __forceinline__ void st_peer_u64(uint32_t local_addr, uint32_t rank, uint64_t v) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local_addr), "r"(rank));
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(ra), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}

__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t n;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
    return n;
}

// Hardware cluster barrier (all threads of every CTA of the cluster); used
// only where every thread is known to arrive: kernel entry and exit.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_peer(uint64_t* bar, uint32_t rank) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(ra) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Per-cycle barrier of a grid that is one cluster (bounded like the grid
// barrier).  Each CTA arrives once on the barrier of every CTA of the cluster
// (release at cluster scope: its stores of the cycle, into peers' mirrors and
// global memory, become visible to whoever completes the phase) and then
// waits on its own.  Cycles alternate between two barriers so that an early
// arrival for cycle c+1 can never complete the phase of cycle c.
static __device__ bool cluster_barrier(uint64_t* bars, uint32_t c, uint32_t C, uint64_t timeout_ns, int32_t* err,
                                       bool skip, uint64_t* rec = nullptr) {
    __shared__ int s_ok;
    uint64_t* bar = bars + (c & 1);
    __syncthreads();
    if (threadIdx.x == 0 && rec) rec[0] = globaltimer_ns();
    if (threadIdx.x < C && !skip) mbar_arrive_peer(bar, threadIdx.x);
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t start = globaltimer_ns();
        while (!mbar_try_wait(bar, (c >> 1) & 1)) {
            if (ld_volatile(err) != 0) { ok = 0; break; }
            if (globaltimer_ns() - start > timeout_ns) {
                atomicCAS(err, 0, (int32_t)SIM_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        if (rec) rec[1] = globaltimer_ns();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// LANE_OP: one warp, one process, one instance; lanes run a 32-wide step.
// ---------------------------------------------------------------------------
// All 13 operators without branches: every candidate result is formed and the
// opcode selects one, so lanes running different operators in one schedule
// step follow a single instruction path (no serialised divergent paths).  One
// left and one right shift serve the four shift-like operators (the amount is
// b for shl/shr and the static x for slice/concat), and add/sub share one
// adder (b complemented with a carry in for sub); a select tree on the bits of
// op - D_ADD (operators in enum order) picks the result in four levels.
__device__ __forceinline__ uint64_t alu_select(uint32_t op, uint64_t a, uint64_t b, uint64_t c, uint32_t x) {
    const uint32_t k = op - D_ADD;
    const bool k0 = k & 1u, k1 = k & 2u, k2 = k & 4u, k3 = k & 8u;
    const bool dyn = (k >> 1) == 3u;                                         // SHL, SHR
    const uint32_t s = (dyn ? uint32_t(b) : x) & 63u;
    const uint64_t L = a << s, R = a >> s;
    const uint64_t neg = 0ull - uint64_t(k0);
    const uint64_t p0 = a + (b ^ neg) + uint64_t(k0);                         // ADD, SUB
    const uint64_t p1 = k0 ? (a & b) : a * b;                                // MUL, AND
    const uint64_t p2 = k0 ? (a ^ b) : (a | b);                              // OR, XOR
    const uint64_t p3 = b >= 64 ? 0ull : (k0 ? R : L);                       // SHL, SHR
    const uint64_t p4 = k0 ? (uint64_t)(a < b) : (uint64_t)(a == b);         // EQ, LT
    const uint64_t p5 = k0 ? R : (a != 0 ? b : c);                           // MUX, SLICE
    const uint64_t p6 = L | b;                                               // CONCAT
    const uint64_t q0 = k1 ? p1 : p0, q1 = k1 ? p3 : p2, q2 = k1 ? p5 : p4;
    const uint64_t r0 = k2 ? q1 : q0, r1 = k2 ? p6 : q2;
    return k3 ? r1 : r0;
}

// Next value of a register into its plane (one instance per warp: pack == 1).
template <bool DIGEST>
__device__ __forceinline__ void store_reg(const Dec& d, uint64_t v, const DevState& S, uint32_t inst, uint32_t nxt,
                                          int32_t col, uint64_t& dacc) {
    const uint32_t idx = d.b | (d.x << 16);
    if (d.c == RC_W64) S.w64[nxt][(uint64_t)idx * S.I + inst] = v;
    else if (d.c == RC_W32) S.w32[nxt][(uint64_t)idx * S.I + inst] = uint32_t(v);
    else S.bits[nxt][(uint64_t)idx * S.bit_stride + inst] = uint32_t(v);
    if (DIGEST && col >= 0) dacc += mix64(((uint64_t)d.imm * kGamma + 1ULL) ^ v);
}

template <bool DIGEST>
__device__ __forceinline__ void exec_lane_op(const Dec& d, const DevProg& P, const DevState& S, uint32_t inst, uint64_t t,
                                             uint64_t key, int32_t col, bool pending, uint64_t* __restrict__ sl,
                                             uint64_t& dacc, const uint64_t* mir_cur = nullptr,
                                             uint32_t mir_nxt = 0) {
    const uint32_t par = uint32_t(t & 1), nxt = par ^ 1;
    if (d.op >= D_ADD && d.op <= D_CONCAT) {
        sl[d.dst] = alu_select(d.op, sl[d.a], sl[d.b], sl[d.c], d.x) & wmask(d.w);
        return;
    }
    switch (d.op) {
    case D_NOP:
        break;
    case D_LDR:
        sl[d.dst] = load_reg(S, par, d.c, d.b | (d.x << 16), inst);
        break;
    case D_LDI:
        sl[d.dst] = stimulus(P, S, key, d.imm, inst, t, d.w);
        break;
    case D_CONST:
        sl[d.dst] = (uint64_t)d.imm | ((uint64_t)d.a << 32) | ((uint64_t)d.b << 48);
        break;
    case D_MEMRD: {
        uint64_t addr = sl[d.a] & ((1ULL << P.mem_lg[d.imm]) - 1);
        sl[d.dst] = mem_read(P, S, d.imm, addr, inst, nxt, pending);
        break;
    }
    case D_STR:
        store_reg<DIGEST>(d, sl[d.a] & wmask(d.w), S, inst, nxt, col, dacc);
        break;
    case D_WREC: {
        uint64_t en = sl[d.a] != 0;
        uint64_t addr = sl[d.b] & ((1ULL << d.x) - 1);
        uint64_t data = sl[d.c] & wmask(d.w);
        uint64_t* r = S.rec[par] + ((uint64_t)d.imm * S.I + inst) * 2;
        r[0] = en ? ((1ULL << 63) | addr) : 0;
        r[1] = data;
        break;
    }
    case D_COMMIT:
        if (pending) {
            uint64_t delta = mem_commit(P, S, d.imm, inst, nxt, DIGEST && col >= 0);
            if (DIGEST) mem_digest_update(S, d.imm, inst, t, delta);
        }
        break;
    case D_LDM:   // mirror entry (cluster exchange): this cycle's value of a register
        sl[d.dst] = mir_cur[d.b | (d.x << 16)];
        break;
    case D_STX:   // next value into the mirror of cluster CTA d.c
        st_peer_u64(mir_nxt + 8u * (d.b | (d.x << 16)), d.c, sl[d.a] & wmask(d.w));
        break;
    default:
        break;
    }
}

// Value of a leaf instruction (register, mirror entry, input, constant).
__device__ __forceinline__ uint64_t leaf_value(const Dec& d, const DevProg& P, const DevState& S, uint32_t inst,
                                               uint64_t t, uint64_t key, const uint64_t* mir_cur) {
    if (d.op == D_LDR) return load_reg(S, uint32_t(t & 1), d.c, d.b | (d.x << 16), inst);
    if (d.op == D_LDM) return mir_cur[d.b | (d.x << 16)];
    if (d.op == D_LDI) return stimulus(P, S, key, d.imm, inst, t, d.w);
    return (uint64_t)d.imm | ((uint64_t)d.a << 32) | ((uint64_t)d.b << 48);   // D_CONST
}

template <bool DIGEST>
__device__ __forceinline__ void finish_lane_op(const DevState& S, uint32_t p, uint32_t inst, uint64_t t, int32_t col,
                                               uint32_t lane, uint64_t dacc) {
    if (DIGEST && col >= 0) {
        if (p == 0 && lane == 0) dacc += S.rom_dig[inst];    // memories without write ports
        for (int o = 16; o; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
        if (lane == 0) ring_add(S, t + 1, col, dacc);
    }
}

// Program rows read from global memory (32-wide padded rows).
template <bool DIGEST>
__device__ void task_lane_op(const DevProg& P, const DevState& S, uint32_t p, uint32_t inst, uint64_t t, bool pending,
                             uint64_t* __restrict__ sl, uint32_t lane) {
    const uint64_t key = S.key[inst];
    const int32_t col = DIGEST ? S.track[inst] : -1;
    uint64_t dacc = 0;
    const DIns* bp = P.s_ins + (uint64_t)P.s_off[p] * 32 + lane;
    const uint32_t nb = P.s_len[p];
    uint4 raw = nb ? ld_ins(bp) : make_uint4(0, 0, 0, 0);
    for (uint32_t b = 0; b < nb; b++) {
        uint4 next_raw = (b + 1 < nb) ? ld_ins(bp + (uint64_t)(b + 1) * 32) : make_uint4(0, 0, 0, 0);
        exec_lane_op<DIGEST>(decode(raw), P, S, inst, t, key, col, pending, sl, dacc);
        __syncwarp();
        raw = next_raw;
    }
    finish_lane_op<DIGEST>(S, p, inst, t, col, lane, dacc);
}

// Result of one operator instruction, reduced to its width.
__device__ __forceinline__ uint64_t eval_op(const Dec& d, uint64_t a, uint64_t b, uint64_t c) {
    return alu_select(d.op, a, b, c, d.x) & wmask(d.w);
}

// Program resident in shared memory: `prog` holds the step count, the step
// table (first instruction | count << 16 | flags) and, 16-byte aligned, the
// instructions.  Operator-only steps run on all 32 lanes without a branch:
// lanes past the step's count repeat its first instruction and write the
// spare slot `dummy` (the last word of the warp's slot region), which no
// instruction reads.
// PAIRS: the program was lowered with operator pairs, whose steps are tested
// first (a program without them never pays that test).
template <bool DIGEST, bool PAIRS>
__device__ void task_lane_op_res(const DevProg& P, const DevState& S, uint32_t p, uint32_t inst, uint64_t t,
                                 bool pending, uint64_t* __restrict__ sl, const uint32_t* __restrict__ prog,
                                 uint32_t lane, uint32_t dummy, const uint64_t* mir_cur = nullptr,
                                 uint32_t mir_nxt = 0) {
    const uint64_t key = S.key[inst];
    const int32_t col = DIGEST ? S.track[inst] : -1;
    uint64_t dacc = 0;
    const uint32_t nb = prog[0];
    const uint32_t* table = prog + 1;
    const uint4* ins = reinterpret_cast<const uint4*>(prog + ((nb + 4) & ~3u));
    uint32_t e = nb ? table[0] : 0;
    for (uint32_t b = 0; b < nb;) {
        if (PAIRS) {
            // a run of pair steps (most of a pair program) in a loop of its own:
            // no step-kind dispatch on this path
            while (e & kStepChain) {
                // two rows: each lane's first operator, then its second one (no
                // warp barrier between them); imm bits 0/1/2 take operands
                // a/b/c of the second from the first result.  The second row's
                // slot operands hold values of earlier steps (a slot written in
                // this step is never read here except through the flags), so
                // they are loaded together with the first row's, before its
                // store.
                const uint32_t e_next = b + 1 < nb ? table[b + 1] : 0;
                const uint32_t first = e & 0xffff, n = ((e >> 16) & kStepCountMask) >> 1;
                const bool on = lane < n;
                const uint32_t i1 = on ? first + lane : first;
                const Dec d1 = decode(ins[i1]);
                const Dec d2 = decode(ins[i1 + n]);
                const uint64_t a1 = sl[d1.a], b1 = sl[d1.b], c1 = sl[d1.c];
                const uint64_t a2s = sl[d2.a], b2s = sl[d2.b], c2s = sl[d2.c];
                const uint64_t r1 = eval_op(d1, a1, b1, c1);
                const uint64_t r2 = eval_op(d2, (d2.imm & 1u) ? r1 : a2s, (d2.imm & 2u) ? r1 : b2s,
                                            (d2.imm & 4u) ? r1 : c2s);
                sl[on ? d1.dst : dummy] = r1;
                sl[on && d2.op != D_NOP ? d2.dst : dummy] = r2;
                __syncwarp();
                e = e_next;
                b++;
            }
            if (b >= nb) break;
        } else {
            // a run of operator steps in a loop of its own likewise
            while (!(e & kStepGeneric) && b < nb) {
                const uint32_t e_next = b + 1 < nb ? table[b + 1] : 0;
                const uint32_t first = e & 0xffff, cnt = (e >> 16) & kStepCountMask;
                const bool on = lane < cnt;
                const Dec d = decode(ins[on ? first + lane : first]);
                sl[on ? d.dst : dummy] = eval_op(d, sl[d.a], sl[d.b], sl[d.c]);
                __syncwarp();
                e = e_next;
                b++;
            }
            if (b >= nb) break;
        }
        const uint32_t e_next = b + 1 < nb ? table[b + 1] : 0;
        const uint32_t first = e & 0xffff, cnt = (e >> 16) & kStepCountMask;
        if (!(e & kStepGeneric)) {
            // operator step: all 32 lanes, no branch (idle lanes write the spare slot)
            const bool on = lane < cnt;
            const Dec d = decode(ins[on ? first + lane : first]);
            sl[on ? d.dst : dummy] = eval_op(d, sl[d.a], sl[d.b], sl[d.c]);
        } else if (!PAIRS && (e & kStepStore)) {
            // programs without pairs: up to four register or mirror stores per
            // lane, every slot value loaded before the first store
            uint4 raw[4];
            uint64_t v[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) {
                const uint32_t i = k * 32 + lane;
                raw[k] = ins[first + (i < cnt ? i : 0)];
                const Dec d = decode(raw[k]);
                v[k] = sl[d.a] & wmask(d.w);
            }
            const uint32_t nxt = uint32_t(t & 1) ^ 1u;
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) {
                if (k * 32 + lane >= cnt) break;
                const Dec d = decode(raw[k]);
                if (d.op == D_STX) st_peer_u64(mir_nxt + 8u * (d.b | (d.x << 16)), d.c, v[k]);
                else store_reg<DIGEST>(d, v[k], S, inst, nxt, col, dacc);
            }
        } else if (e & kStepLeaf) {
            // up to four leaves per lane, every load in flight before the
            // first value is stored; idle lanes write the spare slot
            uint64_t v[4];
            uint32_t dst[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) {
                const uint32_t i = k * 32 + lane;
                v[k] = 0;
                dst[k] = dummy;
                if (i < cnt) {
                    const Dec d = decode(ins[first + i]);
                    dst[k] = d.dst;
                    v[k] = leaf_value(d, P, S, inst, t, key, mir_cur);
                }
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) sl[dst[k]] = v[k];
        } else if (lane < cnt) {
            exec_lane_op<DIGEST>(decode(ins[first + lane]), P, S, inst, t, key, col, pending, sl, dacc, mir_cur,
                                 mir_nxt);
        }
        __syncwarp();
        e = e_next;
        b++;
    }
    finish_lane_op<DIGEST>(S, p, inst, t, col, lane, dacc);
}

template <int MODE, bool DIGEST, bool PAIRS>
__global__ void __launch_bounds__(1024) k_cycles(DevProg P, DevState S, LaunchArgs A) {
    extern __shared__ __align__(16) uint64_t smem[];
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t warp = blockIdx.x * A.warps_per_cta + wib;
    const uint32_t tw = gridDim.x * A.warps_per_cta;
    uint64_t* sl = smem + (uint64_t)wib * (A.slot_words + A.prog_words / 2);
    uint32_t* prog = reinterpret_cast<uint32_t*>(sl + A.slot_words);
    const bool resident = MODE == SIM_MODE_LANE_OP && A.prog_words > 0;
    if (resident) {
        // copy the compact programs of the processes this warp owns (p = warp + k*tw)
        uint32_t off = 0;
        for (uint32_t p = warp; p < P.n_proc; p += tw) {
            const uint4* src = reinterpret_cast<const uint4*>(P.c_words + P.c_off[p]);
            uint4* dst = reinterpret_cast<uint4*>(prog + off);
            for (uint32_t k = lane; k < P.c_size[p] / 4; k += 32) dst[k] = __ldg(src + k);
            off += P.c_size[p];
        }
        __syncwarp();
    }
    const uint64_t t_base = A.t0_dev ? *A.t0_dev + A.t0 : A.t0;
    uint32_t gen = 0;
    for (uint32_t c = 0; c < A.n; c++) {
        const uint64_t t = t_base + c;
        const bool pending = c > 0 || A.pending_first;
        uint64_t* rec = (A.phase && c < A.phase_n) ? A.phase + ((uint64_t)c * gridDim.x + blockIdx.x) * 3 : nullptr;
        if (rec && threadIdx.x == 0) rec[0] = globaltimer_ns();
        if (resident) {
            uint32_t off = 0;
            for (uint32_t p = warp; p < P.n_proc; p += tw) {
                for (uint32_t g = 0; g < S.I; g++)
                    task_lane_op_res<DIGEST, PAIRS>(P, S, p, g, t, pending, sl, prog + off, lane, A.slot_words - 1);
                off += P.c_size[p];
            }
        } else {
            for (uint32_t task = warp; task < A.n_tasks; task += tw) {
                // process-major order: neighbouring warps run the same process
                // for different instance groups (its code and constants stay hot)
            uint32_t p, g;
            task_coords(A, P.n_proc, task, p, g);
                if (MODE == SIM_MODE_LANE_INST) task_lane_inst<DIGEST>(P, S, p, g, t, pending, sl, lane);
                else task_lane_op<DIGEST>(P, S, p, g, t, pending, sl, lane);
            }
        }
        if (A.grid_sync) {
            bool skip = (int32_t)blockIdx.x == A.skip_cta && c == 0;
            if (!grid_barrier(S.bar, gen, A.timeout_ns, S.err, skip, rec ? rec + 1 : nullptr)) return;
        }
    }
    if (A.grid_sync && A.n > 0)
        final_commit(P, S, t_base + A.n, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Cluster exchange (LANE_OP, resident programs, one instance): warp w runs
// process warp_proc[w]; each CTA keeps a double-buffered mirror of the
// registers its processes read from producers in its cluster, which the
// producers write with D_STX straight into the consumer's shared memory.
// Mirror buffer t&1 holds cycle t's values; at launch it is filled from the
// global state, which producers keep writing for readers in other clusters,
// for the host and for the next launch.
template <bool DIGEST, bool PAIRS>
__global__ void __launch_bounds__(1024) k_cycles_cl(DevProg P, DevState S, LaunchArgs A) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ __align__(8) uint64_t cbar[2];
    // the lowering addresses peers by rank within clusters of A.cluster CTAs
    // and the warps' areas by the planned layout: a launch of any other shape
    // (grid, block, cluster or shared memory; the same for every CTA) does
    // nothing but report it
    if (cluster_nctarank() != A.cluster || gridDim.x != A.grid || gridDim.x % A.cluster != 0 ||
        blockDim.x != A.warps_per_cta * 32 || dynamic_smem_bytes() < A.smem_bytes) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(S.err, 0, (int32_t)SIM_ERR_STATE);
        return;
    }
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t warp = blockIdx.x * A.warps_per_cta + wib;
    // warps' areas packed by their own process's needs (slots, then program)
    const uint32_t slot_words = P.warp_slots[warp];
    uint64_t* sl = smem + P.warp_off[warp];
    uint32_t* prog = reinterpret_cast<uint32_t*>(sl + slot_words);
    uint64_t* mirror = smem + A.mirror_off;
    const uint32_t p = P.warp_proc[warp];
    if (p != kNoProc) {
        const uint4* src = reinterpret_cast<const uint4*>(P.c_words + P.c_off[p]);
        uint4* dst = reinterpret_cast<uint4*>(prog);
        for (uint32_t k = lane; k < P.c_size[p] / 4; k += 32) dst[k] = __ldg(src + k);
        __syncwarp();
    }
    const uint64_t t_base = A.t0_dev ? *A.t0_dev + A.t0 : A.t0;
    {
        const uint32_t par = uint32_t(t_base & 1);
        const uint32_t lo = P.mir_off[blockIdx.x], hi = P.mir_off[blockIdx.x + 1];
        for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const uint32_t r = P.mir_reg[i];
            mirror[(uint64_t)par * A.mirror_words + (i - lo)] = load_reg(S, par, P.reg_cls[r], P.reg_idx[r], 0);
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(&cbar[0], A.cluster);
        mbar_init(&cbar[1], A.cluster);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync_all();   // every CTA of the cluster runs; mirrors and barriers are ready
    uint32_t gen = 0;
    bool ok = true;
    for (uint32_t c = 0; c < A.n && ok; c++) {
        const uint64_t t = t_base + c;
        const bool pending = c > 0 || A.pending_first;
        uint64_t* rec = (A.phase && c < A.phase_n) ? A.phase + ((uint64_t)c * gridDim.x + blockIdx.x) * 3 : nullptr;
        if (rec && threadIdx.x == 0) rec[0] = globaltimer_ns();
        if (p != kNoProc) {
            const uint32_t par = uint32_t(t & 1);
            const uint64_t* mc = mirror + (uint64_t)par * A.mirror_words;
            const uint32_t mn = smem_addr(mirror + (uint64_t)(par ^ 1) * A.mirror_words);
            task_lane_op_res<DIGEST, PAIRS>(P, S, p, 0, t, pending, sl, prog, lane, slot_words - 1, mc, mn);
        }
        const bool skip = (int32_t)blockIdx.x == A.skip_cta && c == 0;
        if (A.one_cluster && A.skip_cta < 0) {
            // every thread of the cluster reaches this point every cycle (no
            // early exit exists on this path), so the hardware cluster
            // barrier cannot wait forever; release/acquire at cluster scope
            // orders the cycle's shared, distributed and global stores
            if (rec && threadIdx.x == 0) rec[1] = globaltimer_ns();
            cluster_sync_all();
            if (rec && threadIdx.x == 0) rec[2] = globaltimer_ns();
        } else if (A.one_cluster)
            ok = cluster_barrier(cbar, c, A.cluster, A.timeout_ns, S.err, skip, rec ? rec + 1 : nullptr);
        else
            ok = grid_barrier(S.bar, gen, A.timeout_ns, S.err, skip, rec ? rec + 1 : nullptr);
    }
    cluster_sync_all();   // no CTA exits while a peer may still write into its shared memory
    if (ok && A.n > 0)
        final_commit(P, S, t_base + A.n, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

__global__ void k_commit(DevProg P, DevState S, uint64_t t_end, const uint64_t* t0_dev) {
    if (t0_dev) t_end += *t0_dev;
    final_commit(P, S, t_end, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Input values of a step's first cycle (generated code), before its first
// cycle launch; the cycle base is read from device memory in graph replays.
__global__ void k_stim(DevProg P, DevState S, uint64_t t, const uint64_t* t0_dev) {
    if (t0_dev) t += *t0_dev;
    fill_stim(P, S, t, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Advance the device-resident cycle base of a replayed graph chunk.
__global__ void k_advance(uint64_t* t0_dev, uint64_t n) { *t0_dev += n; }

// Set it (stream-ordered, so the host need not wait for a copy).
__global__ void k_set_u64(uint64_t* p, uint64_t v) { *p = v; }

// Reset instances [lo, lo+n) of buffer `par` to the initial state: register
// init values, memory images, memory digest terms and held inputs.  Used by
// the server when a job takes over instance slots of a pool.
__global__ void k_reset_slots(DevProg P, DevState S, uint32_t par, uint32_t lo, uint32_t n, const uint64_t* reg_init,
                              const uint64_t* mem_image, const uint64_t* mem_word_off, uint64_t mem_words,
                              const uint64_t* mem_init_dig, uint64_t rom_init_dig) {
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, gth = (uint64_t)gridDim.x * blockDim.x;
    // registers: one thread per (register, instance), or per (register, word) for packed 1-bit planes
    const uint32_t w_lo = lo / S.pack, w_hi = (lo + n - 1) / S.pack;
    for (uint64_t e = gtid; e < (uint64_t)P.n_reg * n; e += gth) {
        uint32_t r = uint32_t(e / n), inst = lo + uint32_t(e % n);
        uint32_t cls = P.reg_cls[r], idx = P.reg_idx[r];
        if (cls == RC_W64) S.w64[par][(uint64_t)idx * S.I + inst] = reg_init[r];
        else if (cls == RC_W32) S.w32[par][(uint64_t)idx * S.I + inst] = uint32_t(reg_init[r]);
    }
    for (uint64_t e = gtid; e < (uint64_t)P.n_reg * (w_hi - w_lo + 1); e += gth) {
        uint32_t r = uint32_t(e / (w_hi - w_lo + 1)), wi = w_lo + uint32_t(e % (w_hi - w_lo + 1));
        if (P.reg_cls[r] != RC_BIT) continue;
        uint32_t b0 = wi * S.pack, mask = 0;
        for (uint32_t b = 0; b < S.pack; b++)
            if (b0 + b >= lo && b0 + b < lo + n) mask |= 1u << b;
        uint32_t* word = S.bits[par] + (uint64_t)P.reg_idx[r] * S.bit_stride + wi;
        *word = (*word & ~mask) | ((reg_init[r] & 1) ? mask : 0u);
    }
    for (uint64_t e = gtid; e < mem_words * n; e += gth) {
        uint64_t wdx = e / n;
        uint32_t inst = lo + uint32_t(e % n), m = 0;
        while (m + 1 < P.n_mem && mem_word_off[m + 1] <= wdx) m++;
        uint64_t a = wdx - mem_word_off[m];
        S.mem[P.mem_base[m] + a * S.I + inst] = mem_image[wdx];
    }
    for (uint64_t e = gtid; e < (uint64_t)P.n_mem * n; e += gth) {
        uint32_t m = uint32_t(e / n), inst = lo + uint32_t(e % n);
        S.mem_dig[(uint64_t)m * S.I + inst] = mem_init_dig[m];
    }
    for (uint64_t e = gtid; e < n; e += gth) const_cast<uint64_t*>(S.rom_dig)[lo + e] = rom_init_dig;
    for (uint64_t e = gtid; e < (uint64_t)P.n_in * n; e += gth)
        const_cast<uint8_t*>(S.hold_flag)[(e / n) * S.I + lo + e % n] = 0;
}

// Full digest of buffer `par`: registers (part 0) and memory words (part 1),
// each thread summing a chunk of items for one instance.
__global__ void k_state_digest(DevProg P, DevState S, uint32_t par, const uint64_t* mem_word_off, uint64_t mem_words,
                               uint64_t* out, uint32_t n_inst, uint32_t chunk) {
    uint32_t inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= n_inst) return;
    uint64_t first = (uint64_t)blockIdx.y * chunk;
    uint64_t items = (uint64_t)P.n_reg + mem_words;
    uint64_t last = first + chunk < items ? first + chunk : items;
    uint64_t acc = 0;
    for (uint64_t j = first; j < last; j++) {
        if (j < P.n_reg) {
            uint64_t v = load_reg(S, par, P.reg_cls[j], P.reg_idx[j], inst);
            acc += mix64((j * kGamma + 1ULL) ^ v);
        } else {
            uint64_t w = j - P.n_reg;
            uint32_t m = 0;
            while (m + 1 < P.n_mem && mem_word_off[m + 1] <= w) m++;
            uint64_t a = w - mem_word_off[m];
            acc += mix64(mem_hash(m, a) ^ S.mem[P.mem_base[m] + a * S.I + inst]);
        }
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(out + inst), (unsigned long long)acc);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
template <int MODE, bool DIGEST, bool PAIRS>
static void* kfun() { return reinterpret_cast<void*>(&k_cycles<MODE, DIGEST, PAIRS>); }

// The kernel for a lane mapping, digests on or off, and (LANE_OP) programs
// with or without operator pairs.
static void* cycles_fn(int mode, bool digest, bool pairs) {
    if (mode == SIM_MODE_LANE_INST)
        return digest ? kfun<SIM_MODE_LANE_INST, true, false>() : kfun<SIM_MODE_LANE_INST, false, false>();
    if (pairs) return digest ? kfun<SIM_MODE_LANE_OP, true, true>() : kfun<SIM_MODE_LANE_OP, false, true>();
    return digest ? kfun<SIM_MODE_LANE_OP, true, false>() : kfun<SIM_MODE_LANE_OP, false, false>();
}

// The dynamic shared-memory limit is a per-function attribute shared by every
// batch in the process (and every thread): it is only ever raised, so a
// smaller batch never lowers it under a larger one.
cudaError_t prepare_cycles_kernel(int mode, size_t smem) {
    static std::mutex mu;
    static size_t set_to[3][2][2] = {};
    std::lock_guard<std::mutex> g(mu);
    for (int d = 0; d < 2; d++)
        for (int q = 0; q < 2; q++) {
            if (smem <= set_to[mode][d][q]) continue;
            cudaError_t e =
                cudaFuncSetAttribute(cycles_fn(mode, d, q), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
            set_to[mode][d][q] = smem;
        }
    return cudaSuccess;
}

// (the variants with and without pairs fit alike: the lower of the two)
cudaError_t occupancy_cycles(int mode, int threads, size_t smem, int* blocks_per_sm) {
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cycles_fn(mode, false, false), threads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cycles_fn(mode, false, true), threads, smem);
    *blocks_per_sm = a < b ? a : b;
    return e;
}

cudaError_t launch_cycles(int mode, bool digest, bool cooperative, int grid, int threads, size_t smem, cudaStream_t st,
                          const DevProg& P, const DevState& S, const LaunchArgs& A) {
    void* f = cycles_fn(mode, digest, A.pairs != 0);
    DevProg p = P;
    DevState s = S;
    LaunchArgs a = A;
    void* args[] = {&p, &s, &a};
    if (cooperative) return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(threads), args, smem, st);
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, st);
}

static void* cycles_cl_fn(bool digest, bool pairs) {
    if (pairs) return digest ? reinterpret_cast<void*>(&k_cycles_cl<true, true>) : reinterpret_cast<void*>(&k_cycles_cl<false, true>);
    return digest ? reinterpret_cast<void*>(&k_cycles_cl<true, false>) : reinterpret_cast<void*>(&k_cycles_cl<false, false>);
}

// Shared-memory limit (monotonic, as for k_cycles) and, above the portable
// cluster size of 8, the non-portable cluster size opt-in.
cudaError_t prepare_cluster_kernel(size_t smem, uint32_t C) {
    static std::mutex mu;
    static size_t set_to[4] = {0, 0, 0, 0};
    static bool nonportable[4] = {false, false, false, false};
    std::lock_guard<std::mutex> g(mu);
    for (int v = 0; v < 4; v++) {
        void* f = cycles_cl_fn(v & 1, v >> 1);
        if (smem > set_to[v]) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
            set_to[v] = smem;
        }
        if (C > 8 && !nonportable[v]) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
            nonportable[v] = true;
        }
    }
    return cudaSuccess;
}

static cudaLaunchConfig_t cluster_config(int grid, int threads, size_t smem, uint32_t C, cudaStream_t st,
                                         cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Clusters of C CTAs that can be resident at once.
cudaError_t occupancy_clusters(int grid, int threads, size_t smem, uint32_t C, int* n_clusters) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config(grid, threads, smem, C, nullptr, at);
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&a, cycles_cl_fn(false, false), &cfg);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&b, cycles_cl_fn(false, true), &cfg);
    *n_clusters = a < b ? a : b;
    return e;
}

// A grid of several clusters synchronises with the grid barrier, so all of
// them must be resident at once: the planner checked that with the cluster
// occupancy query (one CTA per SM), and the barrier's wait is bounded, so a
// grid that is not resident ends with SIM_ERR_TIMEOUT rather than a hang.
// Plain cluster launch: the cooperative attribute together with a cluster
// dimension made the launch fail under the profiler with a device fault.
cudaError_t launch_cycles_cl(bool digest, int grid, int threads, size_t smem, uint32_t C, cudaStream_t st,
                             const DevProg& P, const DevState& S, const LaunchArgs& A) {
    DevProg p = P;
    DevState s = S;
    LaunchArgs a = A;
    void* args[] = {&p, &s, &a};
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config(grid, threads, smem, C, st, at);
    return cudaLaunchKernelExC(&cfg, cycles_cl_fn(digest, A.pairs != 0), args);
}

cudaError_t launch_commit(int grid, cudaStream_t st, const DevProg& P, const DevState& S, uint64_t t_end,
                          const uint64_t* t0_dev) {
    k_commit<<<grid, 256, 0, st>>>(P, S, t_end, t0_dev);
    return cudaGetLastError();
}

cudaError_t launch_reset_slots(cudaStream_t st, const DevProg& P, const DevState& S, uint32_t par, uint32_t lo, uint32_t n,
                               const uint64_t* reg_init, const uint64_t* mem_image, const uint64_t* mem_word_off,
                               uint64_t mem_words, const uint64_t* mem_init_dig, uint64_t rom_init_dig) {
    k_reset_slots<<<256, 256, 0, st>>>(P, S, par, lo, n, reg_init, mem_image, mem_word_off, mem_words, mem_init_dig,
                                       rom_init_dig);
    return cudaGetLastError();
}

cudaError_t launch_stim(cudaStream_t st, const DevProg& P, const DevState& S, uint64_t t, const uint64_t* t0_dev) {
    const uint64_t n = (uint64_t)P.n_in * S.I;
    if (!S.stim[0] || n == 0) return cudaSuccess;
    k_stim<<<uint32_t(std::min<uint64_t>((n + 255) / 256, 4096)), 256, 0, st>>>(P, S, t, t0_dev);
    return cudaGetLastError();
}

cudaError_t launch_set_u64(cudaStream_t st, uint64_t* p, uint64_t v) {
    k_set_u64<<<1, 1, 0, st>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_advance(cudaStream_t st, uint64_t* t0_dev, uint64_t n) {
    k_advance<<<1, 1, 0, st>>>(t0_dev, n);
    return cudaGetLastError();
}

cudaError_t launch_state_digest(cudaStream_t st, const DevProg& P, const DevState& S, uint32_t par,
                                const uint64_t* mem_word_off, uint64_t mem_words, uint64_t* out, uint32_t n_inst) {
    const uint32_t chunk = 256;
    uint64_t items = (uint64_t)P.n_reg + mem_words;
    dim3 grid((n_inst + 127) / 128, uint32_t((items + chunk - 1) / chunk));
    if (grid.y == 0) return cudaSuccess;
    k_state_digest<<<grid, 128, 0, st>>>(P, S, par, mem_word_off, mem_words, out, n_inst, chunk);
    return cudaGetLastError();
}

}  // namespace rtl
