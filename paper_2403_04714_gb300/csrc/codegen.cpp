// codegen.cpp -- lower processes to generated CUDA (the second lowering).
//
// Each process (a union of fibers, paper Sec. 3.2 / Sec. 5.1) becomes one
// straight-line __device__ function: every node value is a local variable
// (32-bit when the node is at most 32 bits wide), constants are folded into
// the expressions, and a mask is applied only where the operand widths do not
// already bound the result.  Memory ports, stimulus, digests and the grid
// barrier come from sim_rt.cuh, shared with the bytecode kernels.  Nodes are
// emitted sink by sink in depth-first post-order, so values die soon after
// they are produced.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/sim.h"
#include "codegen.hpp"

namespace rtl {

namespace {

std::string hex64(uint64_t v) {
    char b[32];
    snprintf(b, sizeof b, "0x%llxull", (unsigned long long)v);
    return b;
}

uint64_t mask_of(int w) { return w >= 64 ? ~0ULL : ((1ULL << w) - 1); }

// The operator's result is below 2^w without masking (operands are always
// below 2^width(operand)).
bool fits(const Netlist& nl, const Node& d) {
    auto W = [&](int32_t i) { return int(nl.nodes[i].w); };
    switch (d.op) {
    case OP_ADD: case OP_SUB: case OP_MUL: case OP_SHL: return d.w == 64 || d.w == 32;
    case OP_AND: return std::min(W(d.a), W(d.b)) <= d.w;
    case OP_OR: case OP_XOR: return std::max(W(d.a), W(d.b)) <= d.w;
    case OP_EQ: case OP_LT: case OP_CONCAT: return true;
    case OP_MUX: return std::max(W(d.b), W(d.c)) <= d.w;
    case OP_SLICE: return d.b + int(d.w) >= W(d.a);
    case OP_SHR: return W(d.a) <= d.w;
    default: return true;
    }
}

struct Emitter {
    const Netlist& nl;
    const RegLayout& L;
    int mode;
    bool digest;                  // emit the per-cycle digest terms
    std::string& o;
    std::vector<int32_t> local;   // node -> local index (-1 = not in this process)
    std::vector<uint8_t> done;

    const char* ty(int w) const { return w <= 32 ? "uint32_t" : "uint64_t"; }

    // Operand expression: a folded literal for constants, else the variable.
    std::string ref(int32_t n) const {
        const Node& d = nl.nodes[n];
        if (d.op == OP_CONST) return d.w <= 32 ? std::to_string(uint32_t(d.k)) + "u" : hex64(d.k);
        return "v" + std::to_string(local[n]);
    }
    std::string ref64(int32_t n) const { return "((uint64_t)" + ref(n) + ")"; }
    bool wide(int32_t n) const { return nl.nodes[n].w > 32; }

    void node(int32_t n) {
        const Node& d = nl.nodes[n];
        if (d.op == OP_CONST) return;     // folded into its users
        const std::string v = "v" + std::to_string(local[n]);
        const std::string T = ty(d.w);
        const std::string msk = d.w <= 32 ? std::to_string(uint32_t(mask_of(d.w))) + "u" : hex64(mask_of(d.w));
        std::string e;
        switch (d.op) {
        case OP_REG: {
            const uint32_t ix = L.idx[d.a];
            if (L.cls[d.a] == RC_W64) e = "c64[" + std::to_string(ix) + "ull * I + inst]";
            else if (L.cls[d.a] == RC_W32) e = "c32[" + std::to_string(ix) + "ull * I + inst]";
            else if (mode == SIM_MODE_LANE_INST) e = "(c1[" + std::to_string(ix) + "ull * BS + g] >> lane) & 1u";
            else e = "c1[" + std::to_string(ix) + "ull * BS + inst]";
            break;
        }
        case OP_INPUT:      // the value filled for this cycle (already reduced to the input's width)
            e = "(" + T + ")stv[" + std::to_string(d.a) + "ull * I + inst]";
            break;
        case OP_MEMRD:
            e = "(" + T + ")mem_read(P, S, " + std::to_string(d.a) + "u, " + ref64(d.b) + " & " +
                hex64(mask_of(nl.mem_lg[d.a])) + ", inst, nxt, pending)";
            break;
        case OP_ADD: case OP_SUB: case OP_MUL: case OP_AND: case OP_OR: case OP_XOR: {
            const char* sym = d.op == OP_ADD ? "+" : d.op == OP_SUB ? "-" : d.op == OP_MUL ? "*"
                            : d.op == OP_AND ? "&" : d.op == OP_OR ? "|" : "^";
            bool w64 = d.w > 32 || wide(d.a) || wide(d.b);
            std::string a = w64 ? ref64(d.a) : "((uint32_t)" + ref(d.a) + ")";
            std::string b = w64 ? ref64(d.b) : "((uint32_t)" + ref(d.b) + ")";
            e = "(" + a + " " + sym + " " + b + ")";
            if (!fits(nl, d)) e = "(" + e + " & " + (w64 ? hex64(mask_of(d.w)) : msk) + ")";
            e = "(" + T + ")" + e;
            break;
        }
        case OP_SHL: case OP_SHR: {
            const bool left = d.op == OP_SHL;
            const Node& bn = nl.nodes[d.b];
            std::string a64 = ref64(d.a);
            std::string core;
            if (bn.op == OP_CONST) {
                if (bn.k >= 64) core = "0ull";
                else core = "(" + a64 + (left ? " << " : " >> ") + std::to_string(bn.k) + ")";
            } else {
                std::string s = ref64(d.b);
                core = "(" + s + " >= 64 ? 0ull : " + a64 + (left ? " << " : " >> ") + s + ")";
            }
            if (!fits(nl, d)) core = "(" + core + " & " + hex64(mask_of(d.w)) + ")";
            e = "(" + T + ")" + core;
            break;
        }
        case OP_EQ: case OP_LT:
            e = "(uint32_t)(" + ref64(d.a) + (d.op == OP_EQ ? " == " : " < ") + ref64(d.b) + ")";
            break;
        case OP_MUX: {
            bool w64 = d.w > 32 || wide(d.b) || wide(d.c);
            std::string b = w64 ? ref64(d.b) : "((uint32_t)" + ref(d.b) + ")";
            std::string c = w64 ? ref64(d.c) : "((uint32_t)" + ref(d.c) + ")";
            e = "(" + ref(d.a) + " != 0 ? " + b + " : " + c + ")";
            if (!fits(nl, d)) e = "(" + e + " & " + (w64 ? hex64(mask_of(d.w)) : msk) + ")";
            e = "(" + T + ")" + e;
            break;
        }
        case OP_SLICE: {
            std::string core = "(" + ref64(d.a) + " >> " + std::to_string(d.b) + ")";
            if (!fits(nl, d)) core = "(" + core + " & " + hex64(mask_of(d.w)) + ")";
            e = "(" + T + ")" + core;
            break;
        }
        case OP_CONCAT: {
            int wb = nl.nodes[d.b].w;
            e = "(" + T + ")((" + ref64(d.a) + " << " + std::to_string(wb) + ") | " + ref64(d.b) + ")";
            break;
        }
        default:
            e = "0u";
        }
        o += "    const " + T + " " + v + " = " + e + ";\n";
    }

    void store(int32_t r) {
        const int32_t src = nl.reg_next[r];
        const int wr = nl.reg_w[r];
        std::string val = ref64(src);
        if (nl.nodes[src].w > wr) val = "(" + val + " & " + hex64(mask_of(wr)) + ")";
        const uint32_t ix = L.idx[r];
        o += "    { const uint64_t sv = " + val + ";\n";
        if (L.cls[r] == RC_W64) {
            o += "      n64[" + std::to_string(ix) + "ull * I + inst] = sv;\n";
        } else if (L.cls[r] == RC_W32) {
            o += "      n32[" + std::to_string(ix) + "ull * I + inst] = (uint32_t)sv;\n";
        } else if (mode == SIM_MODE_LANE_INST) {
            o += "      const uint32_t wb = __ballot_sync(0xffffffffu, (sv & 1u) != 0);\n"
                 "      if (lane == 0) n1[" + std::to_string(ix) + "ull * BS + g] = wb;\n";
        } else {
            o += "      n1[" + std::to_string(ix) + "ull * BS + inst] = (uint32_t)sv;\n";
        }
        if (digest)
            o += "      if (col >= 0) *dacc += mix64((" + hex64(uint64_t(r) * 0x9E3779B97F4A7C15ULL + 1ULL) + ") ^ sv);\n";
        o += "    }\n";
    }

    void wrec(int32_t port) {
        const WPort& w = nl.wports[port];
        o += "    { uint64_t* rr = S.rec[par] + (" + std::to_string(port) + "ull * I + inst) * 2;\n"
             "      rr[0] = " + ref(w.en) + " != 0 ? ((1ull << 63) | (" + ref64(w.addr) + " & " +
             hex64(mask_of(nl.mem_lg[w.mem])) + ")) : 0ull;\n"
             "      rr[1] = " + ref64(w.data) + " & " + hex64(mask_of(nl.mem_w[w.mem])) + "; }\n";
    }

    void commit(int32_t m) {
        if (!digest) {
            o += "    if (pending) mem_commit(P, S, " + std::to_string(m) + "u, inst, nxt, false);\n";
            return;
        }
        o += "    if (pending) { const uint64_t dl = mem_commit(P, S, " + std::to_string(m) +
             "u, inst, nxt, S.ring_cap != 0 && col >= 0);\n"
             "      if (S.ring_cap) mem_digest_update(S, " + std::to_string(m) + "u, inst, t, dl); }\n";
    }

    // depth-first post-order over a node's cone
    void emit_cone(int32_t root) {
        std::vector<std::pair<int32_t, int>> st{{root, 0}};
        while (!st.empty()) {
            auto& [n, k] = st.back();
            const Node& d = nl.nodes[n];
            int32_t ops[3];
            int nops = 0;
            switch (d.op) {
            case OP_INPUT: case OP_REG: case OP_CONST: break;
            case OP_MEMRD: ops[nops++] = d.b; break;
            case OP_SLICE: ops[nops++] = d.a; break;
            case OP_MUX: ops[nops++] = d.a; ops[nops++] = d.b; ops[nops++] = d.c; break;
            default: ops[nops++] = d.a; ops[nops++] = d.b;
            }
            if (k < nops) {
                int32_t c = ops[k++];
                if (!done[local[c]]) st.push_back({c, 0});
                continue;
            }
            int32_t fin = n;
            st.pop_back();
            if (!done[local[fin]]) {
                done[local[fin]] = 1;
                node(fin);
            }
        }
    }
};

}  // namespace

namespace {

// Order in which a process's fibers are emitted: greedily the fiber that
// uses most of the values already computed for earlier fibers (shared logic),
// so that those values are consumed, and can die, soon after they are made;
// ties go to the fiber with the least new work, then to the lower index.  The
// live intermediate values of a process function set its register pressure.
std::vector<int32_t> fiber_order(const Partition& part, size_t p, const std::vector<int32_t>& local, size_t n_local) {
    const auto& fibs = part.procs[p];
    std::vector<int32_t> order;
    order.reserve(fibs.size());
    std::vector<uint8_t> made(n_local, 0), taken(fibs.size(), 0);
    for (size_t k = 0; k < fibs.size(); k++) {
        size_t best = fibs.size();
        int64_t best_shared = -1, best_new = 0;
        for (size_t i = 0; i < fibs.size(); i++) {
            if (taken[i]) continue;
            int64_t shared = 0, fresh = 0;
            for (int32_t n : part.fibers[fibs[i]].nodes) (made[local[n]] ? shared : fresh)++;
            if (shared > best_shared || (shared == best_shared && fresh < best_new)) {
                best = i;
                best_shared = shared;
                best_new = fresh;
            }
        }
        taken[best] = 1;
        order.push_back(fibs[best]);
        for (int32_t n : part.fibers[fibs[best]].nodes) made[local[n]] = 1;
    }
    return order;
}

}  // namespace

void gen_process(const Netlist& nl, const Partition& part, const RegLayout& L, size_t p, int mode, bool digest,
                 std::string& o) {
    std::vector<int32_t> nodes;
    for (int32_t f : part.procs[p]) nodes.insert(nodes.end(), part.fibers[f].nodes.begin(), part.fibers[f].nodes.end());
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    Emitter E{nl, L, mode, digest, o, std::vector<int32_t>(nl.nodes.size(), -1), std::vector<uint8_t>(nodes.size(), 0)};
    bool has_input = false;
    for (size_t i = 0; i < nodes.size(); i++) {
        E.local[nodes[i]] = int32_t(i);
        has_input |= nl.nodes[nodes[i]].op == OP_INPUT;
    }
    o += "extern \"C\" __device__ __noinline__ void rtl_p" + std::to_string(p) +
         "(const rtl::DevProg* __restrict__ Pp, const rtl::DevState* __restrict__ Sp, uint32_t g, uint64_t t, "
         "bool pending, uint32_t lane, uint64_t* __restrict__ dacc, int32_t col) {\n"
         "    using namespace rtl;\n"
         "    const DevProg& P = *Pp;\n    const DevState& S = *Sp;\n"
         "    const uint32_t par = (uint32_t)(t & 1), nxt = par ^ 1u;\n"
         "    const uint64_t I = S.I, BS = S.bit_stride;\n";
    o += mode == SIM_MODE_LANE_INST ? "    const uint32_t inst = g * 32u + lane;\n" : "    const uint32_t inst = g;\n";
    o += "    const uint64_t* __restrict__ c64 = S.w64[par];\n    uint64_t* __restrict__ n64 = S.w64[nxt];\n"
         "    const uint32_t* __restrict__ c32 = S.w32[par];\n    uint32_t* __restrict__ n32 = S.w32[nxt];\n"
         "    const uint32_t* __restrict__ c1 = S.bits[par];\n    uint32_t* __restrict__ n1 = S.bits[nxt];\n"
         "    (void)c64; (void)n64; (void)c32; (void)n32; (void)c1; (void)n1; (void)BS; (void)lane; (void)pending;\n";
    if (has_input) o += "    const uint64_t* __restrict__ stv = S.stim[par];\n";
    for (int32_t f : part.procs[p])
        if (part.fibers[f].mem >= 0) E.commit(part.fibers[f].mem);
    for (int32_t f : fiber_order(part, p, E.local, nodes.size())) {
        const Fiber& fb = part.fibers[f];
        if (fb.reg >= 0) {
            E.emit_cone(nl.reg_next[fb.reg]);
            E.store(fb.reg);
        } else {
            for (int32_t port : nl.mem_ports[fb.mem]) {
                const WPort& w = nl.wports[port];
                E.emit_cone(w.en);
                E.emit_cone(w.addr);
                E.emit_cone(w.data);
                E.wrec(port);
            }
        }
    }
    o += "}\n\n";
}

int gen_cuda(const Netlist& nl, const Partition& part, int mode, bool digest, int n_chunks, std::vector<GenUnit>& out,
             std::string& err) {
    (void)err;
    const RegLayout L = reg_layout(nl);
    const size_t NP = part.procs.size();
    out.clear();
    const std::string proto = "(const rtl::DevProg* __restrict__, const rtl::DevState* __restrict__, uint32_t, uint64_t, "
                              "bool, uint32_t, uint64_t* __restrict__, int32_t)";
    // chunks of process functions, balanced by node count
    std::vector<uint64_t> weight(NP, 0);
    uint64_t total = 0;
    for (size_t p = 0; p < NP; p++) {
        for (int32_t f : part.procs[p]) weight[p] += part.fibers[f].nodes.size();
        total += weight[p];
    }
    n_chunks = std::max(1, std::min<int>(n_chunks, int(NP)));
    size_t p = 0;
    for (int c = 0; c < n_chunks && p < NP; c++) {
        GenUnit u;
        u.name = "rtl_chunk" + std::to_string(c) + ".cu";
        u.source = "#include \"sim_rt.cuh\"\n\n";
        uint64_t goal = total * uint64_t(c + 1) / uint64_t(n_chunks), acc = 0;
        for (size_t q = 0; q < p; q++) acc += weight[q];
        do {
            gen_process(nl, part, L, p, mode, digest, u.source);
            acc += weight[p];
            p++;
        } while (p < NP && (acc < goal || c == n_chunks - 1));
        out.push_back(std::move(u));
    }
    // dispatcher and kernels
    GenUnit k;
    k.name = "rtl_kernels.cu";
    k.source = "#define RTLSIM_GENERATED 1\n#include \"sim_rt.cuh\"\n\n";
    for (size_t q = 0; q < NP; q++) k.source += "extern \"C\" __device__ void rtl_p" + std::to_string(q) + proto + ";\n";
    k.source += "\nextern \"C\" __device__ void rtl_dispatch(uint32_t p, const rtl::DevProg* __restrict__ P, "
                "const rtl::DevState* __restrict__ S, uint32_t g, uint64_t t, bool pending, uint32_t lane, "
                "uint64_t* __restrict__ dacc, int32_t col) {\n    switch (p) {\n";
    for (size_t q = 0; q < NP; q++)
        k.source += "    case " + std::to_string(q) + ": rtl_p" + std::to_string(q) + "(P, S, g, t, pending, lane, dacc, col); return;\n";
    k.source += "    default: return;\n    }\n}\n\nRTLSIM_GEN_KERNEL(" + std::to_string(mode) + ", " +
                (digest ? "true" : "false") + ")\n";
    out.push_back(std::move(k));
    return SIM_OK;
}

}  // namespace rtl
