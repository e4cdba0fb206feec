// compiler.cpp -- parse/check, fibers, SLB partitioning and lowering.
#include "compiler.hpp"

#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <numeric>
#include <queue>
#include <random>
#include <unordered_map>
#include <unordered_set>

#include "../../include/sim.h"

namespace rtl {

// ------------------------------------------------------------------------
// Parser
// ------------------------------------------------------------------------
namespace {

struct Cursor {
    const char* p;
    const char* end;
    long line = 1;
};

static const char* kOpNames[OP_COUNT] = {
    "input", "reg", "const", "memrd", "add", "sub", "mul", "and", "or", "xor",
    "shl", "shr", "eq", "lt", "mux", "slice", "concat"};

inline bool is_space(char c) { return c == ' ' || c == '\t' || c == '\r'; }

// Split one line into tokens (pointer, length); stops at '#'.
int split_line(Cursor& cur, const char** tok, int* tlen, int maxtok) {
    int nt = 0;
    while (cur.p < cur.end && *cur.p != '\n') {
        while (cur.p < cur.end && is_space(*cur.p)) cur.p++;
        if (cur.p >= cur.end || *cur.p == '\n') break;
        if (*cur.p == '#') {
            while (cur.p < cur.end && *cur.p != '\n') cur.p++;
            break;
        }
        const char* s = cur.p;
        while (cur.p < cur.end && !is_space(*cur.p) && *cur.p != '\n') cur.p++;
        if (nt < maxtok) {
            tok[nt] = s;
            tlen[nt] = int(cur.p - s);
        }
        nt++;
    }
    if (cur.p < cur.end && *cur.p == '\n') cur.p++;
    return nt;
}

bool tok_u64(const char* s, int n, uint64_t& out) {
    if (n <= 0 || n > 40) return false;
    char buf[48];
    memcpy(buf, s, n);
    buf[n] = 0;
    if (buf[0] == '-') return false;
    char* e = nullptr;
    out = strtoull(buf, &e, 0);
    return *e == 0;
}

bool tok_i32(const char* s, int n, int32_t& out) {
    uint64_t v;
    if (!tok_u64(s, n, v) || v > 0x7fffffffULL) return false;
    out = int32_t(v);
    return true;
}

bool tok_eq(const char* s, int n, const char* lit) { return int(strlen(lit)) == n && !memcmp(s, lit, n); }

inline uint64_t mask_w(int w) { return w >= 64 ? ~0ULL : ((1ULL << w) - 1); }

}  // namespace

// Node checks, op count, and the levels of a Kahn order (longest path from
// a leaf); a node left out of the order lies on a combinational loop.
static int check_graph(Netlist& nl, std::string& err) {
    const int32_t N = int32_t(nl.nodes.size());
    std::vector<int32_t> indeg(N, 0);
    nl.n_ops = 0;
    for (int32_t i = 0; i < N; i++) {
        Node& d = nl.nodes[i];
        auto bad = [&](const char* what) { err = "node " + std::to_string(i) + ": " + what; };
        switch (d.op) {
        case OP_INPUT:
            if (d.a >= int32_t(nl.in_w.size())) { bad("input out of range"); return SIM_ERR_PARSE; }
            if (d.w != nl.in_w[d.a]) { bad("input width mismatch"); return SIM_ERR_WIDTH; }
            continue;
        case OP_REG:
            if (d.a >= int32_t(nl.reg_w.size())) { bad("register out of range"); return SIM_ERR_PARSE; }
            if (d.w != nl.reg_w[d.a]) { bad("register width mismatch"); return SIM_ERR_WIDTH; }
            continue;
        case OP_CONST:
            continue;
        case OP_MEMRD:
            if (d.a >= int32_t(nl.mem_lg.size()) || d.b >= N) { bad("memrd out of range"); return SIM_ERR_PARSE; }
            if (d.w != nl.mem_w[d.a]) { bad("memrd width mismatch"); return SIM_ERR_WIDTH; }
            indeg[i] = 1;
            break;
        case OP_SLICE:
            if (d.a >= N) { bad("operand out of range"); return SIM_ERR_PARSE; }
            if (d.b + int(d.w) > int(nl.nodes[d.a].w)) { bad("slice out of range"); return SIM_ERR_WIDTH; }
            indeg[i] = 1;
            break;
        case OP_CONCAT:
            if (d.a >= N || d.b >= N) { bad("operand out of range"); return SIM_ERR_PARSE; }
            if (int(d.w) != int(nl.nodes[d.a].w) + int(nl.nodes[d.b].w)) { bad("concat width mismatch"); return SIM_ERR_WIDTH; }
            indeg[i] = 2;
            break;
        case OP_EQ:
        case OP_LT:
            if (d.w != 1) { bad("compare must be 1 bit"); return SIM_ERR_WIDTH; }
            [[fallthrough]];
        default:
            if (d.a >= N || d.b >= N || (d.op == OP_MUX && d.c >= N)) { bad("operand out of range"); return SIM_ERR_PARSE; }
            indeg[i] = d.op == OP_MUX ? 3 : 2;
        }
        nl.n_ops++;
    }
    // consumers (CSR) and Kahn order; level = longest path from a leaf
    auto for_operands = [&](const Node& d, auto&& f) {
        switch (d.op) {
        case OP_INPUT: case OP_REG: case OP_CONST: return;
        case OP_MEMRD: f(d.b); return;
        case OP_SLICE: f(d.a); return;
        case OP_MUX: f(d.a); f(d.b); f(d.c); return;
        default: f(d.a); f(d.b); return;
        }
    };
    std::vector<int64_t> off(N + 1, 0);
    for (int32_t i = 0; i < N; i++) for_operands(nl.nodes[i], [&](int32_t o) { off[o + 1]++; });
    for (int32_t i = 0; i < N; i++) off[i + 1] += off[i];
    std::vector<int32_t> users(off[N]);
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int32_t i = 0; i < N; i++) for_operands(nl.nodes[i], [&](int32_t o) { users[fill[o]++] = i; });
    }
    nl.level.assign(N, 0);
    std::vector<int32_t> q;
    q.reserve(N);
    for (int32_t i = 0; i < N; i++)
        if (indeg[i] == 0) q.push_back(i);
    for (size_t h = 0; h < q.size(); h++) {
        int32_t i = q[h];
        for (int64_t u = off[i]; u < off[i + 1]; u++) {
            int32_t j = users[u];
            nl.level[j] = std::max(nl.level[j], nl.level[i] + 1);
            if (--indeg[j] == 0) q.push_back(j);
        }
    }
    if (int32_t(q.size()) != N) { err = "combinational loop"; return SIM_ERR_COMB_LOOP; }
    return SIM_OK;
}

// Gated and divided clocks (Sec. 5, limitations: one top-level clock plus any
// number of gated or divided ones), lowered to a single clock so that the
// partitioner, the lowerings and the kernels see a plain netlist.
//
// Reading, in Verilog's event order: a register with `gate r e` takes its
// next value at an edge of its clock only when e is nonzero; a register with
// `clock r d` is clocked by the rising edge of the 1-bit register d, which
// comes after d's own domain has updated, so its next value and gate see the
// state after that update.  With depth(r) = length of r's chain of clock
// registers, the value a register q holds when domain k evaluates is
//     q's value after its own edge, if depth(q) < k;   q's current value otherwise,
// and q's value after its own edge is
//     U(q) = fire(q) ? (gate(q) != 0 ? next(q) : q) : q,
//     fire(q) = 1 on the top clock,  (d == 0) & U(d) for clock register d,
// with next(q) and gate(q) evaluated in q's own domain.  Everything is then a
// function of the state at the start of the cycle: each register's next node
// becomes U(q), built from copies of the cones it reads in its domain (a copy
// replaces each read of an earlier domain's register by that register's U).
// A memory read in a divided domain is rejected (write ports are on the top
// clock, and their data would have to be forwarded).
static int lower_clocks(Netlist& nl, const std::vector<std::pair<int32_t, int32_t>>& gate_items,
                        const std::vector<std::pair<int32_t, int32_t>>& clock_items, std::string& err) {
    const int32_t R = int32_t(nl.reg_w.size());
    const int32_t N0 = int32_t(nl.nodes.size());
    std::vector<int32_t> gate(R, -1), clk(R, -1), depth(R, 0);
    for (auto& [r, x] : gate_items) {
        if (r < 0 || r >= R) { err = "gate of unknown register"; return SIM_ERR_PARSE; }
        if (gate[r] >= 0) { err = "register " + std::to_string(r) + " has two gate items"; return SIM_ERR_PARSE; }
        if (x < 0 || x >= N0) { err = "gate node out of range"; return SIM_ERR_PARSE; }
        gate[r] = x;
    }
    for (auto& [r, d] : clock_items) {
        if (r < 0 || r >= R) { err = "clock of unknown register"; return SIM_ERR_PARSE; }
        if (clk[r] >= 0) { err = "register " + std::to_string(r) + " has two clock items"; return SIM_ERR_PARSE; }
        if (d < 0 || d >= R || d == r) { err = "bad clock register"; return SIM_ERR_PARSE; }
        if (nl.reg_w[d] != 1) { err = "clock register must be 1 bit"; return SIM_ERR_WIDTH; }
        clk[r] = d;
    }
    int32_t max_depth = 0;
    for (int32_t r = 0; r < R; r++) {
        int32_t dp = 0;
        for (int32_t q = clk[r]; q >= 0; q = clk[q])
            if (++dp > R) { err = "loop of clock registers"; return SIM_ERR_PARSE; }
        depth[r] = dp;
        max_depth = std::max(max_depth, dp);
    }
    auto add = [&](uint8_t op, int w, int32_t a, int32_t b = -1, int32_t c = -1, uint64_t k = 0) {
        Node nd;
        nd.op = op;
        nd.w = uint8_t(w);
        nd.a = a;
        nd.b = b;
        nd.c = c;
        nd.k = k;
        nl.nodes.push_back(nd);
        return int32_t(nl.nodes.size() - 1);
    };
    std::vector<int32_t> reg_read(R, -1), after(R, -1), rose(R, -1);
    auto read_of = [&](int32_t r) {
        if (reg_read[r] < 0) reg_read[r] = add(OP_REG, nl.reg_w[r], r);
        return reg_read[r];
    };
    int32_t zero1 = -1;
    // copy of the cone of `root` as domain k sees it (k = 0: the graph
    // itself); the copies are memoised per (domain, node), in a hash map so
    // that a long chain of divided clocks costs only the cones it visits
    std::unordered_map<uint64_t, int32_t> memo;
    std::vector<int32_t> stack;
    auto in_domain = [&](int32_t k, int32_t root, int32_t& out) -> int {
        if (k == 0) { out = root; return SIM_OK; }
        auto key = [&](int32_t i) { return (uint64_t(uint32_t(k)) << 32) | uint32_t(i); };
        auto get = [&](int32_t i) {
            auto it = memo.find(key(i));
            return it == memo.end() ? -1 : it->second;
        };
        stack.assign(1, root);
        while (!stack.empty()) {
            const int32_t i = stack.back();
            if (get(i) >= 0) { stack.pop_back(); continue; }
            const Node nd = nl.nodes[i];
            if (nd.op == OP_MEMRD) {
                err = "memory read under a divided clock (node " + std::to_string(i) + ")";
                return SIM_ERR_PARSE;
            }
            if (nd.op == OP_REG) {
                memo[key(i)] = depth[nd.a] < k ? after[nd.a] : i;
                stack.pop_back();
                continue;
            }
            if (nd.op == OP_INPUT || nd.op == OP_CONST) { memo[key(i)] = i; stack.pop_back(); continue; }
            const int32_t ops[3] = {nd.a, nd.op == OP_SLICE ? -1 : nd.b, nd.op == OP_MUX ? nd.c : -1};
            int32_t mapped[3] = {-1, -1, -1};
            bool ready = true;
            for (int j = 0; j < 3; j++) {
                if (ops[j] < 0) continue;
                mapped[j] = get(ops[j]);
                if (mapped[j] < 0) { stack.push_back(ops[j]); ready = false; }
            }
            if (!ready) continue;
            stack.pop_back();
            bool same = true;
            for (int j = 0; j < 3; j++) same = same && (ops[j] < 0 || mapped[j] == ops[j]);
            if (same) { memo[key(i)] = i; continue; }
            Node cp = nd;
            cp.a = mapped[0];
            if (nd.op != OP_SLICE) cp.b = mapped[1];
            if (nd.op == OP_MUX) cp.c = mapped[2];
            nl.nodes.push_back(cp);
            memo[key(i)] = int32_t(nl.nodes.size() - 1);
        }
        out = get(root);
        return SIM_OK;
    };
    for (int32_t k = 0; k <= max_depth; k++) {
        for (int32_t r = 0; r < R; r++) {
            if (depth[r] != k) continue;
            const int w = nl.reg_w[r];
            if (k == 0 && gate[r] < 0) {
                // unchanged register; its value after the edge, at its own width
                const int32_t nx = nl.reg_next[r];
                const int wn = nl.nodes[nx].w;
                after[r] = wn == w ? nx : wn > w ? add(OP_SLICE, w, nx, 0)
                                                 : add(OP_OR, w, nx, add(OP_CONST, w, -1, -1, -1, 0));
                continue;
            }
            int32_t nx, sel = -1;
            int rc = in_domain(k, nl.reg_next[r], nx);
            if (rc) return rc;
            if (k > 0) {
                const int32_t d = clk[r];
                if (rose[d] < 0) {
                    if (zero1 < 0) zero1 = add(OP_CONST, 1, -1, -1, -1, 0);
                    rose[d] = add(OP_AND, 1, add(OP_EQ, 1, read_of(d), zero1), after[d]);
                }
                sel = rose[d];
            }
            if (gate[r] >= 0) {
                int32_t g;
                rc = in_domain(k, gate[r], g);
                if (rc) return rc;
                if (sel < 0) {
                    sel = g;
                } else {
                    if (zero1 < 0) zero1 = add(OP_CONST, 1, -1, -1, -1, 0);
                    sel = add(OP_MUX, 1, g, sel, zero1);
                }
            }
            after[r] = add(OP_MUX, w, sel, nx, read_of(r));
        }
    }
    for (int32_t r = 0; r < R; r++)
        if (depth[r] > 0 || gate[r] >= 0) nl.reg_next[r] = after[r];
    return SIM_OK;
}

int parse_netlist(const char* text, size_t len, Netlist& nl, std::string& err) {
    Cursor cur{text, text + len};
    const char* tok[8];
    int tl[8];
    bool header = false, ended = false;
    std::vector<std::pair<int32_t, int32_t>> nexts, gate_items, clock_items;
    char msg[256];
    auto fail = [&](int code, const char* what) {
        snprintf(msg, sizeof msg, "line %ld: %s", cur.line, what);
        err = msg;
        return code;
    };
    while (cur.p < cur.end) {
        int nt = split_line(cur, tok, tl, 8);
        long line = cur.line++;
        (void)line;
        if (nt == 0) continue;
        if (ended) return fail(SIM_ERR_PARSE, "content after end");
        if (nt > 8) return fail(SIM_ERR_PARSE, "too many fields");
        if (!header) {
            if (nt != 2 || !tok_eq(tok[0], tl[0], "rtlnet") || !tok_eq(tok[1], tl[1], "1"))
                return fail(SIM_ERR_PARSE, "expected 'rtlnet 1'");
            header = true;
            continue;
        }
        const char* k = tok[0];
        int kl = tl[0];
        if (tok_eq(k, kl, "n")) {
            Node nd;
            int32_t w;
            if (nt < 3 || !tok_i32(tok[2], tl[2], w)) return fail(SIM_ERR_PARSE, "bad node");
            int op = -1;
            for (int i = 0; i < OP_COUNT; i++)
                if (tok_eq(tok[1], tl[1], kOpNames[i])) op = i;
            if (op < 0) return fail(SIM_ERR_PARSE, "unknown op");
            if (w < 1 || w > 64) return fail(SIM_ERR_WIDTH, "node width out of range");
            nd.op = uint8_t(op);
            nd.w = uint8_t(w);
            int want = op == OP_MUX ? 3 : (op == OP_INPUT || op == OP_REG || op == OP_CONST) ? 1 : 2;
            if (nt != 3 + want) return fail(SIM_ERR_PARSE, "wrong operand count");
            if (op == OP_CONST) {
                if (!tok_u64(tok[3], tl[3], nd.k)) return fail(SIM_ERR_PARSE, "bad constant");
                nd.k &= mask_w(w);
            } else {
                int32_t v[3] = {-1, -1, -1};
                for (int i = 0; i < want; i++)
                    if (!tok_i32(tok[3 + i], tl[3 + i], v[i])) return fail(SIM_ERR_PARSE, "bad operand");
                nd.a = v[0];
                nd.b = v[1];
                nd.c = v[2];
            }
            nl.nodes.push_back(nd);
        } else if (tok_eq(k, kl, "in")) {
            int32_t w;
            if (nt < 2 || !tok_i32(tok[1], tl[1], w)) return fail(SIM_ERR_PARSE, "bad in");
            if (w < 1 || w > 64) return fail(SIM_ERR_WIDTH, "input width out of range");
            nl.in_w.push_back(uint8_t(w));
        } else if (tok_eq(k, kl, "reg")) {
            int32_t w;
            uint64_t init;
            if (nt < 3 || !tok_i32(tok[1], tl[1], w) || !tok_u64(tok[2], tl[2], init))
                return fail(SIM_ERR_PARSE, "bad reg");
            if (w < 1 || w > 64) return fail(SIM_ERR_WIDTH, "register width out of range");
            nl.reg_w.push_back(uint8_t(w));
            nl.reg_init.push_back(init & mask_w(w));
            nl.reg_next.push_back(-1);
        } else if (tok_eq(k, kl, "mem")) {
            int32_t lg, w;
            if (nt < 3 || !tok_i32(tok[1], tl[1], lg) || !tok_i32(tok[2], tl[2], w))
                return fail(SIM_ERR_PARSE, "bad mem");
            if (lg > 24) return fail(SIM_ERR_WIDTH, "memory depth out of range");
            if (w < 1 || w > 64) return fail(SIM_ERR_WIDTH, "memory width out of range");
            nl.mem_lg.push_back(uint8_t(lg));
            nl.mem_w.push_back(uint8_t(w));
            nl.mem_init.emplace_back();
        } else if (tok_eq(k, kl, "next")) {
            int32_t r, x;
            if (nt != 3 || !tok_i32(tok[1], tl[1], r) || !tok_i32(tok[2], tl[2], x))
                return fail(SIM_ERR_PARSE, "bad next");
            nexts.emplace_back(r, x);
        } else if (tok_eq(k, kl, "gate") || tok_eq(k, kl, "clock")) {
            int32_t r, x;
            if (nt != 3 || !tok_i32(tok[1], tl[1], r) || !tok_i32(tok[2], tl[2], x))
                return fail(SIM_ERR_PARSE, "bad gate or clock item");
            (tok_eq(k, kl, "gate") ? gate_items : clock_items).emplace_back(r, x);
        } else if (tok_eq(k, kl, "wport")) {
            int32_t v[4];
            if (nt != 5) return fail(SIM_ERR_PARSE, "bad wport");
            for (int i = 0; i < 4; i++)
                if (!tok_i32(tok[1 + i], tl[1 + i], v[i])) return fail(SIM_ERR_PARSE, "bad wport");
            nl.wports.push_back({v[0], v[1], v[2], v[3]});
        } else if (tok_eq(k, kl, "minit")) {
            int32_t m;
            uint64_t a, v;
            if (nt != 4 || !tok_i32(tok[1], tl[1], m) || !tok_u64(tok[2], tl[2], a) || !tok_u64(tok[3], tl[3], v))
                return fail(SIM_ERR_PARSE, "bad minit");
            if (m >= int32_t(nl.mem_lg.size()) || a >= (1ULL << nl.mem_lg[m]))
                return fail(SIM_ERR_PARSE, "minit out of range");
            nl.mem_init[m].push_back({uint32_t(a), v & mask_w(nl.mem_w[m])});
        } else if (tok_eq(k, kl, "end")) {
            ended = true;
        } else {
            return fail(SIM_ERR_PARSE, "unknown item");
        }
    }
    if (!header) { err = "missing 'rtlnet 1' header"; return SIM_ERR_PARSE; }
    if (!ended) { err = "missing 'end'"; return SIM_ERR_PARSE; }

    // ---- structural checks ------------------------------------------------
    const int32_t N = int32_t(nl.nodes.size());
    for (auto& [r, x] : nexts) {
        if (r < 0 || r >= int32_t(nl.reg_w.size())) { err = "next of unknown register"; return SIM_ERR_PARSE; }
        if (nl.reg_next[r] >= 0) { err = "register has two next nodes"; return SIM_ERR_PARSE; }
        if (x < 0 || x >= N) { err = "next node out of range"; return SIM_ERR_PARSE; }
        nl.reg_next[r] = x;
    }
    for (size_t r = 0; r < nl.reg_next.size(); r++)
        if (nl.reg_next[r] < 0) { err = "register " + std::to_string(r) + " has no next node"; return SIM_ERR_PARSE; }
    for (auto& wp : nl.wports)
        if (wp.mem < 0 || wp.mem >= int32_t(nl.mem_lg.size()) || wp.en >= N || wp.addr >= N || wp.data >= N) {
            err = "write port out of range";
            return SIM_ERR_PARSE;
        }
    nl.mem_ports.assign(nl.mem_lg.size(), {});
    for (size_t p = 0; p < nl.wports.size(); p++) nl.mem_ports[nl.wports[p].mem].push_back(int32_t(p));

    int rc = check_graph(nl, err);
    if (rc) return rc;
    if (gate_items.empty() && clock_items.empty()) return SIM_OK;
    rc = lower_clocks(nl, gate_items, clock_items, err);
    if (rc) return rc;
    return check_graph(nl, err);      // levels and op count of the lowered graph
}

// ------------------------------------------------------------------------
// Fibers and costs
// ------------------------------------------------------------------------
// Estimated issue cost of one node in the device interpreter (the paper
// leaves its cost estimate unstated, Sec. 5.1): one unit per simple op,
// more for 64-bit multiply, the stimulus hash and memory reads.
uint64_t node_cost(const Netlist& nl, int32_t id) {
    const Node& d = nl.nodes[id];
    switch (d.op) {
    case OP_CONST: return 1;
    case OP_INPUT: return 3;
    case OP_MEMRD: return 3;
    case OP_MUL: return d.w > 32 ? 3 : 2;
    default: return 1;
    }
}

static uint64_t sink_cost(const Netlist& nl, const Fiber& f) {
    if (f.reg >= 0) return 1;                                 // the register store
    return uint64_t(nl.mem_ports[f.mem].size()) * 2 + 2;       // write records + commit
}

void extract_fibers(const Netlist& nl, std::vector<Fiber>& out) {
    const int32_t N = int32_t(nl.nodes.size());
    std::vector<uint32_t> stamp(N, 0);
    uint32_t epoch = 0;
    std::vector<int32_t> stack;
    auto crawl = [&](Fiber& f, int32_t root) {
        stack.push_back(root);
        while (!stack.empty()) {
            int32_t i = stack.back();
            stack.pop_back();
            if (stamp[i] == epoch) continue;
            stamp[i] = epoch;
            f.nodes.push_back(i);
            const Node& d = nl.nodes[i];
            switch (d.op) {
            case OP_INPUT: case OP_REG: case OP_CONST: break;
            case OP_MEMRD: stack.push_back(d.b); break;
            case OP_SLICE: stack.push_back(d.a); break;
            case OP_MUX: stack.push_back(d.a); stack.push_back(d.b); stack.push_back(d.c); break;
            default: stack.push_back(d.a); stack.push_back(d.b);
            }
        }
    };
    out.clear();
    out.reserve(nl.reg_w.size() + nl.mem_lg.size());
    // one fiber per register: the reverse crawl from its next-value node (Sec. 5.1)
    for (size_t r = 0; r < nl.reg_w.size(); r++) {
        Fiber f;
        f.reg = int32_t(r);
        ++epoch;
        crawl(f, nl.reg_next[r]);
        out.push_back(std::move(f));
    }
    // one fiber per memory with write ports: all its ports' cones together,
    // so one process applies the memory's write records in port order
    for (size_t m = 0; m < nl.mem_lg.size(); m++) {
        if (nl.mem_ports[m].empty()) continue;
        Fiber f;
        f.mem = int32_t(m);
        ++epoch;
        for (int32_t p : nl.mem_ports[m]) {
            crawl(f, nl.wports[p].en);
            crawl(f, nl.wports[p].addr);
            crawl(f, nl.wports[p].data);
        }
        out.push_back(std::move(f));
    }
    for (auto& f : out) {
        std::sort(f.nodes.begin(), f.nodes.end());
        uint64_t c = sink_cost(nl, f);
        for (int32_t i : f.nodes) c += node_cost(nl, i);
        f.cost = c;
    }
}

uint64_t union_cost(const Netlist& nl, const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    uint64_t c = 0;
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
        int32_t x;
        if (j >= b.size() || (i < a.size() && a[i] < b[j])) x = a[i++];
        else if (i >= a.size() || b[j] < a[i]) x = b[j++];
        else { x = a[i]; i++; j++; }
        c += node_cost(nl, x);
    }
    return c;
}

uint64_t inter_cost(const Netlist& nl, const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    uint64_t c = 0;
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] < b[j]) i++;
        else if (b[j] < a[i]) j++;
        else { c += node_cost(nl, a[i]); i++; j++; }
    }
    return c;
}

// ------------------------------------------------------------------------
// Submodular load balancing (paper Sec. 5.1)
// ------------------------------------------------------------------------
namespace {

// A hypergraph over local vertex ids 0..n-1: the vertex set of one bisection,
// or a coarsening of it (used by the hypergraph partitioning strategy).
struct LocalHg {
    int32_t n = 0;
    std::vector<int64_t> vw;                  // vertex weights
    std::vector<std::vector<int32_t>> pins;   // edge -> vertices (at least 2, ascending)
    std::vector<int64_t> ew;                  // edge weights
    std::vector<int64_t> inc_off;             // vertex -> edges (CSR)
    std::vector<int32_t> inc;

    void build_incidence() {
        inc_off.assign(size_t(n) + 1, 0);
        for (auto& pl : pins)
            for (int32_t v : pl) inc_off[v + 1]++;
        for (int32_t v = 0; v < n; v++) inc_off[v + 1] += inc_off[v];
        inc.resize(inc_off[n]);
        std::vector<int64_t> fill(inc_off.begin(), inc_off.end() - 1);
        for (size_t e = 0; e < pins.size(); e++)
            for (int32_t v : pins[e]) inc[fill[v]++] = int32_t(e);
    }
};

int64_t cut_weight(const LocalHg& h, const std::vector<int8_t>& side) {
    int64_t c = 0;
    for (size_t e = 0; e < h.pins.size(); e++) {
        bool on[2] = {false, false};
        for (int32_t v : h.pins[e]) on[side[v]] = true;
        if (on[0] && on[1]) c += h.ew[e];
    }
    return c;
}

// One coarsening level: every vertex pairs with the unmatched neighbour it
// shares the most weight with (an edge of s pins adds w / (s - 1); edges of
// more than 64 pins are ignored for the rating), if the pair stays under
// `max_vw`.  False if the level would shrink the vertex count by under 10 %.
bool coarsen(const LocalHg& h, int64_t max_vw, LocalHg& c, std::vector<int32_t>& map) {
    map.assign(h.n, -1);
    std::vector<double> score(h.n, 0.0);
    std::vector<int32_t> touched;
    int32_t nc = 0;
    for (int32_t v = 0; v < h.n; v++) {
        if (map[v] >= 0) continue;
        touched.clear();
        for (int64_t t = h.inc_off[v]; t < h.inc_off[v + 1]; t++) {
            const auto& pl = h.pins[h.inc[t]];
            if (pl.size() > 64) continue;
            const double r = double(h.ew[h.inc[t]]) / double(pl.size() - 1);
            for (int32_t u : pl) {
                if (u == v || map[u] >= 0) continue;
                if (score[u] == 0.0) touched.push_back(u);
                score[u] += r;
            }
        }
        int32_t best = -1;
        double bs = 0.0;
        for (int32_t u : touched) {
            if (h.vw[v] + h.vw[u] <= max_vw && score[u] > bs) { best = u; bs = score[u]; }
            score[u] = 0.0;
        }
        map[v] = nc;
        if (best >= 0) map[best] = nc;
        nc++;
    }
    if (double(nc) > 0.9 * double(h.n)) return false;
    c.n = nc;
    c.vw.assign(nc, 0);
    for (int32_t v = 0; v < h.n; v++) c.vw[map[v]] += h.vw[v];
    c.pins.clear();
    c.ew.clear();
    std::vector<int32_t> pl;
    for (size_t e = 0; e < h.pins.size(); e++) {
        pl.clear();
        for (int32_t v : h.pins[e]) pl.push_back(map[v]);
        std::sort(pl.begin(), pl.end());
        pl.erase(std::unique(pl.begin(), pl.end()), pl.end());
        if (pl.size() < 2) continue;
        c.pins.push_back(pl);
        c.ew.push_back(h.ew[e]);
    }
    c.build_incidence();
    return true;
}

// Greedy growth of side 0 from `seed` along the heaviest connections until
// it weighs at least target0 (disconnected parts: the next vertex in order).
void grow_side(const LocalHg& h, int32_t seed, int64_t target0, std::vector<int8_t>& side) {
    side.assign(h.n, 1);
    std::vector<int64_t> conn(h.n, 0);
    std::vector<char> on0(h.pins.size(), 0);
    std::priority_queue<std::pair<int64_t, int32_t>> q;
    int64_t w0 = 0;
    int32_t next = 0, v = seed;
    while (w0 < target0) {
        while (v < 0 && !q.empty()) {
            auto [cv, u] = q.top();
            q.pop();
            if (side[u] == 1 && conn[u] == cv) v = u;
        }
        if (v < 0) {
            while (next < h.n && side[next] == 0) next++;
            if (next == h.n) break;
            v = next;
        }
        side[v] = 0;
        w0 += h.vw[v];
        for (int64_t t = h.inc_off[v]; t < h.inc_off[v + 1]; t++) {
            const int32_t e = h.inc[t];
            if (on0[e]) continue;
            on0[e] = 1;
            for (int32_t u : h.pins[e])
                if (side[u] == 1) {
                    conn[u] += h.ew[e];
                    q.push({conn[u], u});
                }
        }
        v = -1;
    }
}

// Fiduccia-Mattheyses passes on a bisection: moves of the highest cut gain
// that keep each side under its cap, each vertex once per pass, then the
// best prefix of the pass is kept.
void fm_refine(const LocalHg& h, std::vector<int8_t>& side, const int64_t cap[2], int passes) {
    const size_t E = h.pins.size();
    std::vector<int32_t> cnt[2] = {std::vector<int32_t>(E), std::vector<int32_t>(E)};
    std::vector<int64_t> gain(h.n);
    std::vector<int32_t> lock(h.n, 0);
    for (int pass = 1; pass <= passes; pass++) {
        for (size_t e = 0; e < E; e++) {
            cnt[0][e] = cnt[1][e] = 0;
            for (int32_t u : h.pins[e]) cnt[side[u]][e]++;
        }
        using GE = std::pair<int64_t, int32_t>;
        std::priority_queue<GE> heap[2];
        int64_t ws[2] = {0, 0};
        for (int32_t v = 0; v < h.n; v++) {
            const int s0 = side[v];
            int64_t g = 0;
            for (int64_t t = h.inc_off[v]; t < h.inc_off[v + 1]; t++) {
                const int32_t e = h.inc[t];
                if (cnt[s0][e] == 1) g += h.ew[e];
                if (cnt[1 - s0][e] == 0) g -= h.ew[e];
            }
            gain[v] = g;
            heap[s0].push({g, v});
            ws[s0] += h.vw[v];
        }
        std::vector<int32_t> moves;
        int64_t cum = 0, best = 0;
        size_t best_len = 0;
        const size_t limit = std::max<size_t>(64, size_t(h.n) / 2);
        while (moves.size() < limit) {
            int32_t pick = -1;
            int64_t pick_g = 0;
            for (int s0 = 0; s0 < 2; s0++) {
                while (!heap[s0].empty()) {
                    auto [g, u] = heap[s0].top();
                    if (lock[u] == pass || side[u] != s0 || gain[u] != g) { heap[s0].pop(); continue; }
                    if (ws[1 - s0] + h.vw[u] > cap[1 - s0]) break;     // the best move does not fit
                    if (pick < 0 || g > pick_g) { pick = u; pick_g = g; }
                    break;
                }
            }
            if (pick < 0) break;
            const int from = side[pick], to = 1 - from;
            lock[pick] = pass;
            auto bump = [&](int32_t u, int64_t d) {
                if (lock[u] == pass) return;
                gain[u] += d;
                heap[side[u]].push({gain[u], u});
            };
            for (int64_t t = h.inc_off[pick]; t < h.inc_off[pick + 1]; t++) {
                const int32_t e = h.inc[t];
                const int64_t w = h.ew[e];
                if (cnt[to][e] == 0) { for (int32_t u : h.pins[e]) bump(u, w); }
                else if (cnt[to][e] == 1) {
                    for (int32_t u : h.pins[e])
                        if (side[u] == to) bump(u, -w);
                }
                cnt[from][e]--;
                cnt[to][e]++;
                if (cnt[from][e] == 0) { for (int32_t u : h.pins[e]) bump(u, -w); }
                else if (cnt[from][e] == 1) {
                    for (int32_t u : h.pins[e])
                        if (side[u] == from && u != pick) bump(u, w);
                }
            }
            side[pick] = int8_t(to);
            ws[from] -= h.vw[pick];
            ws[to] += h.vw[pick];
            moves.push_back(pick);
            cum += pick_g;
            if (cum > best) { best = cum; best_len = moves.size(); }
        }
        for (size_t m = moves.size(); m > best_len; m--) side[moves[m - 1]] ^= 1;   // roll back
        if (best <= 0) break;
    }
}

// Multilevel bisection (coarsen by heavy-connection matching, bisect the
// coarsest level from a few seeds, then project back refining every level),
// side 0 aiming at target0 of the weight.
void multilevel_bisect(const LocalHg& h0, int64_t target0, std::vector<int8_t>& side) {
    int64_t W = 0;
    for (int64_t x : h0.vw) W += x;
    const int64_t cap[2] = {int64_t(double(target0) * 1.03) + 1, int64_t(double(W - target0) * 1.03) + 1};
    std::deque<LocalHg> coarse;
    std::vector<std::vector<int32_t>> maps;
    const LocalHg* cur = &h0;
    const int64_t max_vw = std::max<int64_t>(1, W / 60);
    while (cur->n > 120) {
        LocalHg c;
        std::vector<int32_t> m;
        if (!coarsen(*cur, max_vw, c, m)) break;
        coarse.push_back(std::move(c));
        maps.push_back(std::move(m));
        cur = &coarse.back();
    }
    // the coarsest level: the best of a few growth seeds, each refined
    std::vector<int8_t> best_side, s;
    int64_t best_cut = -1;
    const int32_t n = cur->n;
    for (int32_t seed : {int32_t(0), n / 3, (2 * n) / 3, n - 1}) {
        if (seed < 0 || seed >= n) continue;
        grow_side(*cur, seed, target0, s);
        fm_refine(*cur, s, cap, 6);
        const int64_t c = cut_weight(*cur, s);
        if (best_cut < 0 || c < best_cut) { best_cut = c; best_side = s; }
    }
    side.swap(best_side);
    for (size_t lv = maps.size(); lv-- > 0;) {
        const LocalHg& fine = lv == 0 ? h0 : coarse[lv - 1];
        std::vector<int8_t> fs(fine.n);
        for (int32_t v = 0; v < fine.n; v++) fs[v] = side[maps[lv][v]];
        fm_refine(fine, fs, cap, 4);
        side.swap(fs);
    }
}

}  // namespace

namespace {

struct Proc {
    std::vector<int32_t> nodes;    // sorted union of the fibers' nodes
    std::vector<int32_t> fibers;
    uint64_t sink = 0;             // stores/records/commits of its fibers
    uint64_t cost = 0;             // tau = sum of node costs (deduplicated) + sinks
    uint64_t mem = 0;              // data memory: registers touched and arrays read (bytes)
    bool alive = true;
};

struct Slb {
    const Netlist& nl;
    const PartitionConfig& cfg;
    std::vector<Fiber>& fib;
    std::vector<Proc> P;
    std::vector<int32_t> proc_of_fiber;
    std::vector<int32_t> writer_fiber;              // register -> fiber writing it
    std::vector<std::vector<int32_t>> reader_fibers;  // register -> fibers reading it
    std::vector<std::vector<int32_t>> reads_of_fiber; // fiber -> registers read
    std::vector<char> pinned;                         // fiber grouped by stage 1 (stays with its array)

    Slb(const Netlist& n, const PartitionConfig& c, std::vector<Fiber>& f) : nl(n), cfg(c), fib(f) {}

    uint64_t node_set_cost(const std::vector<int32_t>& nodes) const {
        uint64_t c = 0;
        for (int32_t i : nodes) c += node_cost(nl, i);
        return c;
    }

    uint64_t data_mem(const std::vector<int32_t>& nodes, const std::vector<int32_t>& fibers) const {
        uint64_t m = 8 * fibers.size();
        std::unordered_set<int32_t> arrays;
        for (int32_t i : nodes) {
            const Node& d = nl.nodes[i];
            if (d.op == OP_REG) m += 8;
            if (d.op == OP_MEMRD) arrays.insert(d.a);
        }
        for (int32_t f : fibers)
            if (fib[f].mem >= 0) arrays.insert(fib[f].mem);
        for (int32_t a : arrays) m += 8ULL << nl.mem_lg[a];
        return m;
    }

    void init() {
        const size_t F = fib.size();
        writer_fiber.assign(nl.reg_w.size(), -1);
        reader_fibers.assign(nl.reg_w.size(), {});
        reads_of_fiber.assign(F, {});
        for (size_t f = 0; f < F; f++) {
            if (fib[f].reg >= 0) writer_fiber[fib[f].reg] = int32_t(f);
            for (int32_t i : fib[f].nodes)
                if (nl.nodes[i].op == OP_REG) {
                    reader_fibers[nl.nodes[i].a].push_back(int32_t(f));
                    reads_of_fiber[f].push_back(nl.nodes[i].a);
                }
        }
        P.resize(F);
        proc_of_fiber.resize(F);
        pinned.assign(F, 0);
        for (size_t f = 0; f < F; f++) {
            P[f].nodes = fib[f].nodes;
            P[f].fibers = {int32_t(f)};
            P[f].sink = sink_cost(nl, fib[f]);
            P[f].cost = fib[f].cost;
            P[f].mem = data_mem(P[f].nodes, P[f].fibers);
            proc_of_fiber[f] = int32_t(f);
        }
    }

    void merge_into(int32_t p, int32_t q) {   // q is absorbed by p
        std::vector<int32_t> u;
        u.reserve(P[p].nodes.size() + P[q].nodes.size());
        std::set_union(P[p].nodes.begin(), P[p].nodes.end(), P[q].nodes.begin(), P[q].nodes.end(),
                       std::back_inserter(u));
        P[p].nodes.swap(u);
        for (int32_t f : P[q].fibers) {
            P[p].fibers.push_back(f);
            proc_of_fiber[f] = p;
        }
        P[p].sink += P[q].sink;
        P[p].cost = node_set_cost(P[p].nodes) + P[p].sink;
        P[p].mem = data_mem(P[p].nodes, P[p].fibers);
        P[q].alive = false;
        P[q].nodes.clear();
        P[q].nodes.shrink_to_fit();
        P[q].fibers.clear();
    }

    // processes that read a register p writes or write a register p reads
    void partners(int32_t p, std::vector<int32_t>& out) {
        out.clear();
        std::unordered_set<int32_t> seen;
        auto add = [&](int32_t q) {
            if (q != p && P[q].alive && seen.insert(q).second) out.push_back(q);
        };
        for (int32_t f : P[p].fibers) {
            for (int32_t r : reads_of_fiber[f]) {
                if (writer_fiber[r] >= 0) add(proc_of_fiber[writer_fiber[r]]);
                if (out.size() >= cfg.cand_cap) return;
            }
        }
        for (int32_t f : P[p].fibers) {
            if (fib[f].reg < 0) continue;
            for (int32_t g : reader_fibers[fib[f].reg]) {
                add(proc_of_fiber[g]);
                if (out.size() >= cfg.cand_cap) return;
            }
        }
    }

    bool mem_ok(int32_t p, int32_t q) const {
        if (!cfg.mem_budget_bytes) return true;
        std::vector<int32_t> u;
        std::set_union(P[p].nodes.begin(), P[p].nodes.end(), P[q].nodes.begin(), P[q].nodes.end(),
                       std::back_inserter(u));
        std::vector<int32_t> fs(P[p].fibers);
        fs.insert(fs.end(), P[q].fibers.begin(), P[q].fibers.end());
        return data_mem(u, fs) <= cfg.mem_budget_bytes;
    }

    // Stage 1: fibers that touch the same very large array are merged up front
    // so no process later needs several large arrays (Sec. 5.1, footnote).
    void stage1() {
        std::vector<std::vector<int32_t>> users(nl.mem_lg.size());
        for (size_t f = 0; f < fib.size(); f++) {
            std::unordered_set<int32_t> arrays;
            for (int32_t i : fib[f].nodes)
                if (nl.nodes[i].op == OP_MEMRD) arrays.insert(nl.nodes[i].a);
            if (fib[f].mem >= 0) arrays.insert(fib[f].mem);
            for (int32_t a : arrays) users[a].push_back(int32_t(f));
        }
        for (size_t m = 0; m < users.size(); m++) {
            uint64_t bytes = (uint64_t(nl.mem_w[m] + 7) / 8) << nl.mem_lg[m];
            if (bytes < cfg.big_array_bytes || users[m].size() < 2) continue;
            for (int32_t f : users[m]) pinned[f] = 1;
            int32_t p = proc_of_fiber[users[m][0]];
            for (size_t k = 1; k < users[m].size(); k++) {
                int32_t q = proc_of_fiber[users[m][k]];
                if (q != p) merge_into(p, q);
            }
        }
    }

    size_t alive_count() const {
        size_t n = 0;
        for (auto& p : P) n += p.alive;
        return n;
    }

    // Stage 3: conservative merge.  Repeatedly take the cheapest process and
    // merge it with a process it communicates with, if the merged cost does
    // not exceed the current worst cost and memory fits; otherwise try the
    // two cheapest; otherwise skip it (Sec. 5.1).  Among partners, take the
    // one sharing the most work, then the cheapest, then the lowest id.
    void stage3(size_t target) {
        using E = std::pair<uint64_t, int32_t>;
        std::priority_queue<E, std::vector<E>, std::greater<E>> heap;
        uint64_t worst = 0;
        for (size_t p = 0; p < P.size(); p++)
            if (P[p].alive) {
                heap.push({P[p].cost, int32_t(p)});
                worst = std::max(worst, P[p].cost);
            }
        size_t count = alive_count();
        std::vector<uint8_t> done(P.size(), 0);
        std::vector<int32_t> cand;
        auto valid = [&](const E& e) { return P[e.second].alive && !done[e.second] && P[e.second].cost == e.first; };
        while (count > target && !heap.empty()) {
            E top = heap.top();
            heap.pop();
            if (!valid(top)) continue;
            int32_t p = top.second;
            partners(p, cand);
            int32_t best = -1;
            uint64_t best_shared = 0, best_cost = 0;
            for (int32_t q : cand) {
                uint64_t shared = inter_cost(nl, P[p].nodes, P[q].nodes);
                uint64_t merged = P[p].cost + P[q].cost - shared;
                if (merged > worst || !mem_ok(p, q)) continue;
                if (best < 0 || shared > best_shared || (shared == best_shared && (P[q].cost < best_cost ||
                                                        (P[q].cost == best_cost && q < best)))) {
                    best = q;
                    best_shared = shared;
                    best_cost = P[q].cost;
                }
            }
            if (best < 0) {
                // the two cheapest: p and the next valid heap entry
                while (!heap.empty() && !valid(heap.top())) heap.pop();
                if (!heap.empty()) {
                    int32_t q = heap.top().second;
                    uint64_t merged = P[p].cost + P[q].cost - inter_cost(nl, P[p].nodes, P[q].nodes);
                    if (merged <= worst && mem_ok(p, q)) best = q;
                }
            }
            if (best < 0) {
                done[p] = 1;
                continue;
            }
            merge_into(p, best);
            heap.push({P[p].cost, p});
            count--;
        }
    }

    // Stage 4: relaxed merge when stage 3 misses the target: the remaining
    // processes, most expensive first, each go to the bin whose merged cost
    // is lowest among the cheapest bins and the bins it communicates with
    // (the worst cost may grow).  Fails if memory cannot fit.
    int stage4(size_t target, std::string& err) {
        std::vector<int32_t> order;
        for (size_t p = 0; p < P.size(); p++)
            if (P[p].alive) order.push_back(int32_t(p));
        if (order.size() <= target) return SIM_OK;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return P[a].cost > P[b].cost; });
        // the first `target` processes seed the bins
        std::vector<int32_t> bins(order.begin(), order.begin() + target);
        std::vector<int32_t> bin_of_proc(P.size(), -1);
        for (size_t i = 0; i < bins.size(); i++) bin_of_proc[bins[i]] = int32_t(i);
        using E = std::pair<uint64_t, int32_t>;
        std::priority_queue<E, std::vector<E>, std::greater<E>> heap;
        for (size_t i = 0; i < bins.size(); i++) heap.push({P[bins[i]].cost, int32_t(i)});
        std::vector<int32_t> cand, part;
        for (size_t k = target; k < order.size(); k++) {
            int32_t p = order[k];
            cand.clear();
            std::vector<E> popped;
            while (!heap.empty() && popped.size() < 8) {
                E e = heap.top();
                heap.pop();
                if (P[bins[e.second]].cost != e.first) continue;
                popped.push_back(e);
                cand.push_back(e.second);
            }
            for (auto& e : popped) heap.push(e);
            partners(p, part);
            for (int32_t q : part)
                if (bin_of_proc[q] >= 0) cand.push_back(bin_of_proc[q]);
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            int32_t best = -1;
            uint64_t best_merged = 0;
            for (int32_t b : cand) {
                int32_t q = bins[b];
                if (!mem_ok(q, p)) continue;
                uint64_t merged = P[p].cost + P[q].cost - inter_cost(nl, P[p].nodes, P[q].nodes);
                if (best < 0 || merged < best_merged || (merged == best_merged && P[q].cost < P[bins[best]].cost)) {
                    best = b;
                    best_merged = merged;
                }
            }
            if (best < 0) {
                err = "a process does not fit the per-process memory budget";
                return SIM_ERR_CAPACITY;
            }
            merge_into(bins[best], p);
            heap.push({P[bins[best]].cost, best});
        }
        return SIM_OK;
    }

    // Hypergraph partitioning, the alternative strategy the paper compares
    // with its bottom-up merge (Sec. 7, "Partitioning Strategies", after
    // RepCut): the vertices are the fibers (after stage 1's array groups), each
    // combinational node shared by several fibers is a hyperedge over them
    // weighted by the node's cost (nodes with the same fibers form one
    // hyperedge), and the processes are the parts of a k-way partition.  A
    // hyperedge that spans lambda parts is computed lambda times, so the
    // connectivity cut sum (lambda - 1) w(e) is exactly the duplicated work.
    // The partition is by recursive multilevel bisection (heavy-connection
    // coarsening, greedy growth from a few seeds on the coarsest level,
    // Fiduccia-Mattheyses refinement on every level) under a balance bound on
    // the vertex weights (a vertex weighs its own nodes plus an equal share of
    // each shared node).
    struct Hg {
        std::vector<std::vector<int32_t>> pins;     // edge -> vertices
        std::vector<uint64_t> ew;                   // edge weight
        std::vector<int64_t> vw;                    // vertex weight (balance)
        std::vector<int64_t> inc_off;               // vertex -> edges (CSR)
        std::vector<int32_t> inc;
    };

    void build_hypergraph(const std::vector<int32_t>& verts, Hg& h) const {
        const int32_t V = int32_t(verts.size());
        const size_t N = nl.nodes.size();
        std::vector<int32_t> users_n(N + 1, 0);
        for (int32_t v = 0; v < V; v++)
            for (int32_t i : P[verts[v]].nodes) users_n[i + 1]++;
        for (size_t i = 0; i < N; i++) users_n[i + 1] += users_n[i];
        std::vector<int32_t> users(users_n[N]);
        {
            std::vector<int32_t> fill(users_n.begin(), users_n.end() - 1);
            for (int32_t v = 0; v < V; v++)
                for (int32_t i : P[verts[v]].nodes) users[fill[i]++] = v;   // ascending v
        }
        std::vector<double> share(V, 0.0);
        h.vw.assign(V, 0);
        std::unordered_map<uint64_t, std::vector<int32_t>> by_hash;   // pin-list hash -> edges
        for (size_t i = 0; i < N; i++) {
            const int32_t b = users_n[i], e = users_n[i + 1];
            if (e == b) continue;
            const uint64_t c = node_cost(nl, int32_t(i));
            if (e - b == 1) { h.vw[users[b]] += int64_t(c); continue; }
            uint64_t hs = 1469598103934665603ULL;
            for (int32_t k = b; k < e; k++) hs = (hs ^ uint64_t(users[k])) * 1099511628211ULL;
            int32_t found = -1;
            for (int32_t ed : by_hash[hs])
                if (h.pins[ed].size() == size_t(e - b) && std::equal(users.begin() + b, users.begin() + e, h.pins[ed].begin())) {
                    found = ed;
                    break;
                }
            if (found < 0) {
                found = int32_t(h.pins.size());
                h.pins.emplace_back(users.begin() + b, users.begin() + e);
                h.ew.push_back(0);
                by_hash[hs].push_back(found);
            }
            h.ew[found] += c;
            for (int32_t k = b; k < e; k++) share[users[k]] += double(c) / double(e - b);
        }
        for (int32_t v = 0; v < V; v++) h.vw[v] += int64_t(P[verts[v]].sink) + int64_t(share[v] + 0.5) + 1;
        h.inc_off.assign(V + 1, 0);
        for (auto& pl : h.pins) for (int32_t v : pl) h.inc_off[v + 1]++;
        for (int32_t v = 0; v < V; v++) h.inc_off[v + 1] += h.inc_off[v];
        h.inc.resize(h.inc_off[V]);
        std::vector<int64_t> fill(h.inc_off.begin(), h.inc_off.end() - 1);
        for (size_t ed = 0; ed < h.pins.size(); ed++)
            for (int32_t v : h.pins[ed]) h.inc[fill[v]++] = int32_t(ed);
    }

    // Scratch arrays of the recursive bisection, indexed by global vertex or edge.
    struct HgWork {
        std::vector<int32_t> part, stamp, loc, estamp;
        int32_t epoch = 0;
    };

    // Split `set` (ascending, size >= k) into parts first_part .. first_part + k - 1.
    void bisect(const Hg& h, std::vector<int32_t> set, size_t k, int32_t first_part, HgWork& w) const {
        if (k <= 1) {                               // callers keep set.size() >= k
            for (int32_t v : set) w.part[v] = first_part;
            return;
        }
        const size_t k0 = k / 2;
        // the set's own hypergraph: its vertices, and the edges with two or more pins in it
        const int32_t my = ++w.epoch;
        LocalHg L;
        L.n = int32_t(set.size());
        L.vw.resize(set.size());
        for (size_t i = 0; i < set.size(); i++) {
            w.stamp[set[i]] = my;
            w.loc[set[i]] = int32_t(i);
            L.vw[i] = h.vw[set[i]];
        }
        std::vector<int32_t> pl;
        for (int32_t v : set)
            for (int64_t t = h.inc_off[v]; t < h.inc_off[v + 1]; t++) {
                const int32_t ed = h.inc[t];
                if (w.estamp[ed] == my) continue;
                w.estamp[ed] = my;
                pl.clear();
                for (int32_t u : h.pins[ed])
                    if (w.stamp[u] == my) pl.push_back(w.loc[u]);
                if (pl.size() < 2) continue;
                L.pins.push_back(pl);
                L.ew.push_back(int64_t(h.ew[ed]));
            }
        L.build_incidence();
        int64_t W = 0;
        for (int64_t x : L.vw) W += x;
        std::vector<int8_t> side;
        multilevel_bisect(L, int64_t(double(W) * double(k0) / double(k)), side);
        std::vector<int32_t> s0, s1;
        for (size_t i = 0; i < set.size(); i++) (side[i] == 0 ? s0 : s1).push_back(set[i]);
        // every part gets a vertex: a side with fewer vertices than parts
        // takes the lightest vertices of the other side
        auto top_up = [&](std::vector<int32_t>& to, std::vector<int32_t>& from, size_t need) {
            if (to.size() >= need) return;
            std::sort(from.begin(), from.end(), [&](int32_t a, int32_t b) { return h.vw[a] > h.vw[b]; });
            while (to.size() < need) { to.push_back(from.back()); from.pop_back(); }
            std::sort(from.begin(), from.end());
            std::sort(to.begin(), to.end());
        };
        top_up(s0, s1, k0);
        top_up(s1, s0, k - k0);
        set.clear();
        set.shrink_to_fit();
        L = LocalHg();
        bisect(h, std::move(s0), k0, first_part, w);
        bisect(h, std::move(s1), k - k0, first_part + int32_t(k0), w);
    }

    // Straggler relief after the hypergraph partition, whose balance bound is
    // on estimated vertex weights: move one fiber at a time (never one that
    // stage 1 grouped with a big array) off the most expensive process to the
    // process, among the cheapest and its communication partners, that keeps
    // the larger of the two new costs lowest, while that lowers the worst cost.
    void relieve_stragglers(size_t max_moves) {
        using E = std::pair<uint64_t, int32_t>;
        std::priority_queue<E> worst;
        std::priority_queue<E, std::vector<E>, std::greater<E>> cheap;
        for (size_t p = 0; p < P.size(); p++)
            if (P[p].alive) { worst.push({P[p].cost, int32_t(p)}); cheap.push({P[p].cost, int32_t(p)}); }
        std::vector<int32_t> cand, part;
        std::vector<int32_t> mult(nl.nodes.size(), 0), mult_stamp(nl.nodes.size(), 0);
        for (size_t it = 0; it < max_moves; it++) {
            while (!worst.empty() && (!P[worst.top().second].alive || P[worst.top().second].cost != worst.top().first))
                worst.pop();
            if (worst.empty()) return;
            const int32_t p = worst.top().second;
            if (P[p].fibers.size() < 2) return;
            cand.clear();
            std::vector<E> popped;
            while (!cheap.empty() && popped.size() < 8) {
                E e = cheap.top();
                cheap.pop();
                if (!P[e.second].alive || P[e.second].cost != e.first) continue;
                popped.push_back(e);
                if (e.second != p) cand.push_back(e.second);
            }
            for (auto& e : popped) cheap.push(e);
            partners(p, part);
            cand.insert(cand.end(), part.begin(), part.end());
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) { return P[a].cost < P[b].cost; });
            // cost of p without fiber f: minus the nodes no other fiber of p uses
            for (int32_t f : P[p].fibers)
                for (int32_t i : fib[f].nodes) {
                    if (mult_stamp[i] != int32_t(it + 1)) { mult_stamp[i] = int32_t(it + 1); mult[i] = 0; }
                    mult[i]++;
                }
            int32_t bf = -1, bq = -1;
            uint64_t bmax = P[p].cost, bp = 0;   // a move must lower the worst cost
            for (int32_t f : P[p].fibers) {
                if (pinned[f]) continue;                 // stage 1 keeps it with its array
                uint64_t own = sink_cost(nl, fib[f]);
                for (int32_t i : fib[f].nodes)
                    if (mult[i] == 1) own += node_cost(nl, i);
                const uint64_t np_f = P[p].cost - own;
                if (np_f >= bmax) continue;
                for (int32_t q : cand) {
                    // lower bound: the fiber shares all its nodes with q
                    if (P[q].cost + sink_cost(nl, fib[f]) >= bmax) break;
                    const uint64_t nq = P[q].cost + fib[f].cost - inter_cost(nl, fib[f].nodes, P[q].nodes);
                    if (std::max(np_f, nq) < bmax) { bf = f; bq = q; bmax = std::max(np_f, nq); bp = np_f; }
                }
            }
            if (bf < 0) return;
            // the process without the fiber
            std::vector<int32_t> rest, u, tmp;
            for (int32_t f : P[p].fibers)
                if (f != bf) {
                    rest.push_back(f);
                    tmp.clear();
                    std::set_union(u.begin(), u.end(), fib[f].nodes.begin(), fib[f].nodes.end(), std::back_inserter(tmp));
                    u.swap(tmp);
                }
            const uint64_t sink_p = P[p].sink - sink_cost(nl, fib[bf]);
            const uint64_t np = node_set_cost(u) + sink_p;
            if (np != bp) return;                        // equal by construction; stop if not
            std::vector<int32_t> uq;
            std::set_union(P[bq].nodes.begin(), P[bq].nodes.end(), fib[bf].nodes.begin(), fib[bf].nodes.end(),
                           std::back_inserter(uq));
            std::vector<int32_t> fq(P[bq].fibers);
            fq.push_back(bf);
            if (cfg.mem_budget_bytes && data_mem(uq, fq) > cfg.mem_budget_bytes) return;
            P[p].nodes.swap(u);
            P[p].fibers.swap(rest);
            P[p].sink = sink_p;
            P[p].cost = np;
            P[p].mem = data_mem(P[p].nodes, P[p].fibers);
            P[bq].nodes.swap(uq);
            P[bq].fibers.swap(fq);
            P[bq].sink += sink_cost(nl, fib[bf]);
            P[bq].cost = node_set_cost(P[bq].nodes) + P[bq].sink;
            P[bq].mem = data_mem(P[bq].nodes, P[bq].fibers);
            proc_of_fiber[bf] = bq;
            worst.push({P[p].cost, p});
            worst.push({P[bq].cost, bq});
            cheap.push({P[p].cost, p});
            cheap.push({P[bq].cost, bq});
        }
    }

    void hypergraph_partition(size_t target) {
        std::vector<int32_t> verts;
        for (size_t p = 0; p < P.size(); p++)
            if (P[p].alive) verts.push_back(int32_t(p));
        if (verts.size() <= target) return;
        Hg h;
        build_hypergraph(verts, h);
        const int32_t V = int32_t(verts.size());
        const size_t E = h.pins.size();
        std::vector<int32_t> all(V);
        std::iota(all.begin(), all.end(), 0);
        HgWork w;
        w.part.assign(V, -1);
        w.stamp.assign(V, 0);
        w.loc.assign(V, 0);
        w.estamp.assign(E, 0);
        bisect(h, all, target, 0, w);
        const std::vector<int32_t>& part = w.part;
        std::vector<int32_t> head(target, -1);
        for (int32_t v = 0; v < V; v++) {
            int32_t& hd = head[part[v]];
            if (hd < 0) hd = verts[v];
            else merge_into(hd, verts[v]);
        }
        relieve_stragglers(4 * target);
    }

    void random_partition(size_t target, uint32_t seed) {
        std::mt19937 rng(seed);
        target = std::max<size_t>(1, std::min(target ? target : 64, P.size()));
        std::vector<int32_t> bins(target, -1);
        std::vector<int32_t> order(P.size());
        std::iota(order.begin(), order.end(), 0);
        std::shuffle(order.begin(), order.end(), rng);
        for (size_t k = 0; k < order.size(); k++) {
            size_t b = k < target ? k : rng() % target;
            if (bins[b] < 0) bins[b] = order[k];
            else merge_into(bins[b], order[k]);
        }
    }
};

}  // namespace

int partition(const Netlist& nl, const PartitionConfig& cfg, Partition& out, std::string& err) {
    extract_fibers(nl, out.fibers);
    out.fiber_cost_sum = out.fiber_cost_max = 0;
    for (auto& f : out.fibers) {
        out.fiber_cost_sum += f.cost;
        out.fiber_cost_max = std::max(out.fiber_cost_max, f.cost);
    }
    Slb s(nl, cfg, out.fibers);
    s.init();
    if (cfg.random_seed) {
        s.random_partition(cfg.target, cfg.random_seed);
    } else if (cfg.hypergraph) {
        s.stage1();
        s.hypergraph_partition(cfg.target ? cfg.target : s.P.size());
    } else {
        s.stage1();
        size_t target = cfg.target ? cfg.target : s.P.size();
        if (cfg.stage3) s.stage3(target);
        int rc = s.stage4(target, err);
        if (rc) return rc;
    }
    out.procs.clear();
    out.proc_cost.clear();
    out.proc_cost_sum = out.proc_cost_max = 0;
    for (auto& p : s.P) {
        if (!p.alive) continue;
        std::vector<int32_t> fs = p.fibers;
        std::sort(fs.begin(), fs.end());
        out.procs.push_back(std::move(fs));
        out.proc_cost.push_back(p.cost);
        out.proc_cost_sum += p.cost;
        out.proc_cost_max = std::max(out.proc_cost_max, p.cost);
    }
    // cut: register words a process reads but another process writes
    std::vector<int32_t> proc_of_reg(nl.reg_w.size(), -1);
    for (size_t p = 0; p < out.procs.size(); p++)
        for (int32_t f : out.procs[p])
            if (out.fibers[f].reg >= 0) proc_of_reg[out.fibers[f].reg] = int32_t(p);
    out.cut_words = 0;
    for (size_t p = 0; p < out.procs.size(); p++) {
        std::unordered_set<int32_t> regs;
        for (int32_t f : out.procs[p])
            for (int32_t i : out.fibers[f].nodes)
                if (nl.nodes[i].op == OP_REG && proc_of_reg[nl.nodes[i].a] != int32_t(p)) regs.insert(nl.nodes[i].a);
        out.cut_words += regs.size();
    }
    return SIM_OK;
}

// ------------------------------------------------------------------------
// Lowering
// ------------------------------------------------------------------------
RegLayout reg_layout(const Netlist& nl) {
    RegLayout L;
    L.cls.resize(nl.reg_w.size());
    L.idx.resize(nl.reg_w.size());
    for (size_t r = 0; r < nl.reg_w.size(); r++) {
        RegClass c = reg_class(nl.reg_w[r]);
        L.cls[r] = c;
        L.idx[r] = L.count[c]++;
    }
    return L;
}

namespace {

// One schedule item: a node's value, or a sink action.
struct Item {
    int kind;          // 0 = node, 1 = register store, 2 = write record, 3 = memory commit
    int32_t id;        // node id / register / port / memory
    int level;
    uint8_t op;        // for sorting within a level
    int phase = 0;     // LANE_OP order: 0 memory commits, 1 leaves, 2 operators, 3 stores and write records
};

constexpr uint16_t kNoSlot = 0xffff;

// Slot allocation over a sequence of steps.  Each step defines some values
// and uses some; a value's slot is released after its last use.  With
// `free_before_def` a step's operands whose last use is this step are
// released before its own definitions (sequential execution); otherwise only
// after the step completes (32 lanes run the step at once).
struct SlotAlloc {
    std::vector<uint16_t> free_list;
    uint32_t next = 0;
    uint16_t get() {
        if (!free_list.empty()) {
            uint16_t s = free_list.back();
            free_list.pop_back();
            return s;
        }
        return uint16_t(next++);
    }
    void put(uint16_t s) { free_list.push_back(s); }
};

}  // namespace

namespace {

// One step of a shared-memory program.
struct CStep {
    uint32_t flags = 0;
    std::vector<DIns> ins;
};

// Program layout: word 0 = step count n, words 1..n = step words (first
// instruction | count << 16 | flags), padded to a multiple of 4 words, then
// the 16-byte instructions.
int append_program(const std::vector<CStep>& steps, std::vector<uint32_t>& words, std::string& err) {
    const uint32_t nb = uint32_t(steps.size()), tw = (nb + 4) & ~3u;
    const size_t base = words.size();
    words.resize(base + tw, 0);
    words[base] = nb;
    uint32_t first = 0;
    for (uint32_t b = 0; b < nb; b++) {
        words[base + 1 + b] = first | (uint32_t(steps[b].ins.size()) << 16) | steps[b].flags;
        for (const DIns& d : steps[b].ins) {
            uint32_t w4[4];
            memcpy(w4, &d, 16);
            words.insert(words.end(), w4, w4 + 4);
        }
        first += uint32_t(steps[b].ins.size());
    }
    if (first > 0xffff) {
        err = "process has too many instructions for one program";
        return SIM_ERR_CAPACITY;
    }
    return SIM_OK;
}


// Compact program with operator chains (sim_config.chain = K = 2; the
// scheduler takes any K, the interpreter runs pairs).  Operators are
// scheduled in dependence order; an operator whose operands are all ready
// before the step of one of them, d, or come from d's lane in that step, runs
// in d's step right after d on the same lane (up to K operators per lane),
// taking d's result from a register instead of from the slot after a warp
// barrier.  A step with chains (kStepChain) holds R rows of its n lanes'
// operators (D_NOP where a lane's chain is shorter); imm bits 0/1/2 mark
// operands a/b/c that are the previous result of the lane.  Memory reads never
// chain.  Slots are allocated over the compact steps (a value lives from its
// step to the end of the step of its last use).
// Measured on the mid netlist (one GB300, 4-CTA clusters): pairs take the
// slowest process from 66 to 40 steps and the rate from 77-78k to 83-84k
// cycles/s; chains of three or four (31 and 28 steps) gain nothing more,
// because every lane of a step pays for its longest chain: a chained
// operator saves one step entry but adds a row (a decode, operand loads, a
// store and an evaluation) to the whole step.  A variant
// that kept only the pairs' second operators (no D_NOP, lanes with a pair
// first) made smaller programs but measured 4 % slower on the same GPU
// (79.3k against 82.6k cycles/s), so the rows stay full.
template <class MakeIns, class Operands>
int chained_program(const Netlist& nl, const std::vector<Item>& items, const std::vector<int32_t>& local, size_t n_local,
                    MakeIns& make_ins, Operands& operands, Lowered& out, size_t p, uint32_t K, std::string& err) {
    std::vector<size_t> commits, leaves, opers, sinks;
    for (size_t i = 0; i < items.size(); i++)
        (items[i].phase == 0 ? commits : items[i].phase == 1 ? leaves : items[i].phase == 2 ? opers : sinks).push_back(i);
    const size_t no = opers.size();
    std::vector<int32_t> op_of_local(n_local, -1);
    for (size_t k = 0; k < no; k++) op_of_local[local[items[opers[k]].id]] = int32_t(k);
    std::vector<int32_t> ostep(no, 0), olane(no, 0);
    std::vector<std::vector<std::vector<int32_t>>> lanes;   // step -> lane -> operators in order
    std::vector<uint8_t> has_memrd, has_chain;
    std::vector<int32_t> deps;
    for (size_t k = 0; k < no; k++) {
        const bool memrd = nl.nodes[items[opers[k]].id].op == OP_MEMRD;
        deps.clear();
        operands(items[opers[k]], [&](int32_t n) {
            const int32_t q = op_of_local[local[n]];
            if (q >= 0) deps.push_back(q);
        });
        int32_t s = 0;
        for (int32_t q : deps) s = std::max(s, ostep[q] + 1);
        bool placed = false;
        if (!memrd && s > 0 && !has_memrd[s - 1])
            for (int32_t d : deps) {
                if (ostep[d] != s - 1 || nl.nodes[items[opers[d]].id].op == OP_MEMRD) continue;
                auto& L = lanes[s - 1][olane[d]];
                if (L.back() != d || L.size() >= K) continue;
                bool ok = true;
                for (int32_t q : deps) ok &= ostep[q] < s - 1 || olane[q] == olane[d];
                if (!ok) continue;
                L.push_back(int32_t(k));
                ostep[k] = s - 1;
                olane[k] = olane[d];
                has_chain[s - 1] = 1;
                placed = true;
                break;
            }
        if (placed) continue;
        while (size_t(s) < lanes.size() && (lanes[s].size() >= 32 || (memrd && has_chain[s]))) s++;
        if (size_t(s) == lanes.size()) {
            lanes.emplace_back();
            has_memrd.push_back(0);
            has_chain.push_back(0);
        }
        ostep[k] = s;
        olane[k] = int32_t(lanes[s].size());
        lanes[s].push_back({int32_t(k)});
        if (memrd) has_memrd[s] = 1;
    }
    // steps as lists of item indices (-1 = D_NOP of a shorter chain)
    struct PStep { uint32_t flags; std::vector<int64_t> its; uint32_t lanes; };
    std::vector<PStep> ps;
    for (size_t k = 0; k < commits.size(); k += 32) {
        PStep st{kStepGeneric, {}, 0};
        for (size_t j = k; j < std::min(commits.size(), k + 32); j++) st.its.push_back(int64_t(commits[j]));
        ps.push_back(std::move(st));
    }
    for (size_t k = 0; k < leaves.size(); k += kLeafStepMax) {
        PStep st{kStepGeneric | kStepLeaf, {}, 0};
        for (size_t j = k; j < std::min(leaves.size(), k + kLeafStepMax); j++) st.its.push_back(int64_t(leaves[j]));
        ps.push_back(std::move(st));
    }
    for (size_t s = 0; s < lanes.size(); s++) {
        uint32_t rows = 1;
        for (auto& L : lanes[s]) rows = std::max<uint32_t>(rows, uint32_t(L.size()));
        PStep st{has_memrd[s] ? kStepGeneric : rows > 1 ? (kStepGeneric | kStepChain | (rows << kStepRowsShift)) : 0u,
                 {}, uint32_t(lanes[s].size())};
        for (uint32_t r = 0; r < rows; r++)
            for (auto& L : lanes[s]) st.its.push_back(r < L.size() ? int64_t(opers[L[r]]) : -1);
        ps.push_back(std::move(st));
    }
    for (size_t k = 0; k < sinks.size(); k += 32) {
        PStep st{kStepGeneric, {}, 0};
        for (size_t j = k; j < std::min(sinks.size(), k + 32); j++) st.its.push_back(int64_t(sinks[j]));
        ps.push_back(std::move(st));
    }
    // value lifetimes over the compact steps
    std::vector<int32_t> last(n_local, -1);
    for (size_t b = 0; b < ps.size(); b++)
        for (int64_t i : ps[b].its)
            if (i >= 0) operands(items[size_t(i)], [&](int32_t n) { last[local[n]] = std::max(last[local[n]], int32_t(b)); });
    std::vector<uint16_t> slot(n_local, kNoSlot);
    SlotAlloc A;
    std::vector<std::vector<uint16_t>> release(ps.size() + 1);
    std::vector<CStep> steps;
    for (size_t b = 0; b < ps.size(); b++) {
        for (uint16_t sl : release[b]) A.put(sl);
        for (int64_t i : ps[b].its) {
            if (i < 0 || items[size_t(i)].kind != 0) continue;
            const int32_t l = local[items[size_t(i)].id];
            slot[l] = A.get();
            release[std::max(last[l], int32_t(b)) + 1].push_back(slot[l]);
        }
        CStep st;
        st.flags = ps[b].flags;
        const uint32_t n = ps[b].lanes;
        for (size_t j = 0; j < ps[b].its.size(); j++) {
            const int64_t i = ps[b].its[j];
            if (i < 0) {
                DIns nop{};                   // D_NOP (its result goes to the spare slot)
                nop.w = 64;
                st.ins.push_back(nop);
                continue;
            }
            DIns d = make_ins(items[size_t(i)], slot);
            if ((ps[b].flags & kStepChain) && j >= n) {
                // operands that are the lane's previous result come from its register
                const int32_t prev = local[items[size_t(ps[b].its[j - n])].id];
                const Node& nd = nl.nodes[items[size_t(i)].id];
                auto is_prev = [&](int32_t node) { return local[node] == prev; };
                if (is_prev(nd.a)) d.imm |= 1u;
                if (nd.op != OP_SLICE && is_prev(nd.b)) d.imm |= 2u;
                if (nd.op == OP_MUX && is_prev(nd.c)) d.imm |= 4u;
            }
            st.ins.push_back(d);
        }
        steps.push_back(std::move(st));
    }
    if (A.next > 0xfff0) { err = "process needs too many value slots"; return SIM_ERR_CAPACITY; }
    out.s_slots[p] = std::max<uint32_t>(out.s_slots[p], std::max<uint32_t>(1, A.next));
    out.c_off[p] = uint32_t(out.c_words.size());
    int rc = append_program(steps, out.c_words, err);
    if (rc) return rc;
    out.c_size[p] = uint32_t(out.c_words.size()) - out.c_off[p];
    return SIM_OK;
}

}  // namespace

int lower(const Netlist& nl, const Partition& part, Lowered& out, std::string& err, uint32_t chain) {
    RegLayout L = reg_layout(nl);
    const size_t NP = part.procs.size();
    out = Lowered();
    out.s_off.resize(NP);
    out.s_len.resize(NP);
    out.s_slots.resize(NP);
    out.c_off.resize(NP);
    out.c_size.resize(NP);
    out.b_off.resize(NP);
    out.b_len.resize(NP);
    out.b_slots.resize(NP);
    out.commit_proc.assign(nl.mem_lg.size(), -1);
    std::vector<int32_t> local(nl.nodes.size(), -1);

    for (size_t p = 0; p < NP; p++) {
        // node set: union of the process's fibers
        std::vector<int32_t> nodes;
        for (int32_t f : part.procs[p]) nodes.insert(nodes.end(), part.fibers[f].nodes.begin(), part.fibers[f].nodes.end());
        std::sort(nodes.begin(), nodes.end());
        nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
        for (size_t i = 0; i < nodes.size(); i++) local[nodes[i]] = int32_t(i);

        std::vector<Item> items;
        items.reserve(nodes.size() + part.procs[p].size() * 2);
        for (int32_t id : nodes) items.push_back({0, id, nl.level[id], nl.nodes[id].op});
        for (int32_t f : part.procs[p]) {
            const Fiber& fb = part.fibers[f];
            if (fb.reg >= 0) {
                items.push_back({1, fb.reg, nl.level[nl.reg_next[fb.reg]] + 1, 255});
            } else {
                out.commit_proc[fb.mem] = int32_t(p);
                items.push_back({3, fb.mem, 0, 254});
                for (int32_t port : nl.mem_ports[fb.mem]) {
                    const WPort& w = nl.wports[port];
                    int lv = std::max({nl.level[w.en], nl.level[w.addr], nl.level[w.data]}) + 1;
                    items.push_back({2, port, lv, 253});
                }
            }
        }
        // steps: memory commits, then leaves, then the operators by level,
        // then register stores and write records (their values stay in slots
        // until the end); within a level by operator kind (less divergence in a
        // step), then id.  Operator steps hold operators only, apart from the
        // rare memory reads, so the interpreter runs them without branches;
        // leaf steps hold leaves only, so their loads can all be in flight.
        auto phase = [&](const Item& it) {
            if (it.kind == 1 || it.kind == 2) return 3;
            if (it.kind == 3) return 0;
            const uint8_t op = nl.nodes[it.id].op;
            return (op == OP_INPUT || op == OP_REG || op == OP_CONST) ? 1 : 2;
        };
        for (auto& it : items) it.phase = phase(it);
        std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
            if (a.phase != b.phase) return a.phase < b.phase;
            if (a.level != b.level) return a.level < b.level;
            if (a.op != b.op) return a.op < b.op;
            if (a.kind != b.kind) return a.kind < b.kind;
            return a.id < b.id;
        });
        // bundle index of each item (32 per step, never mixing levels)
        std::vector<uint32_t> bundle(items.size());
        uint32_t nb = 0;
        {
            int cur_level = -1, cur_phase = -1;
            uint32_t fill = 0;
            for (size_t i = 0; i < items.size(); i++) {
                // operators never share a step with their own operands; the
                // leaves and the stores have no dependences among themselves
                const int lv = items[i].phase == 2 ? items[i].level : 0;
                if (lv != cur_level || items[i].phase != cur_phase || fill == 32) {
                    nb++;
                    fill = 0;
                    cur_level = lv;
                    cur_phase = items[i].phase;
                }
                bundle[i] = nb - 1;
                fill++;
            }
        }
        // last use (bundle and sequential position) of each local value
        std::vector<int32_t> last_b(nodes.size(), -1);
        auto use = [&](int32_t node, size_t i) {
            int32_t l = local[node];
            last_b[l] = std::max<int32_t>(last_b[l], int32_t(bundle[i]));
        };
        auto operands = [&](const Item& it, auto&& f) {
            if (it.kind == 0) {
                const Node& d = nl.nodes[it.id];
                switch (d.op) {
                case OP_INPUT: case OP_REG: case OP_CONST: break;
                case OP_MEMRD: f(d.b); break;
                case OP_SLICE: f(d.a); break;
                case OP_MUX: f(d.a); f(d.b); f(d.c); break;
                default: f(d.a); f(d.b);
                }
            } else if (it.kind == 1) {
                f(nl.reg_next[it.id]);
            } else if (it.kind == 2) {
                const WPort& w = nl.wports[it.id];
                f(w.en); f(w.addr); f(w.data);
            }
        };
        for (size_t i = 0; i < items.size(); i++) operands(items[i], [&](int32_t o) { use(o, i); });

        auto make_ins = [&](const Item& it, const std::vector<uint16_t>& slot) {
            DIns d{};
            d.op = D_NOP;
            auto S = [&](int32_t node) { return slot[local[node]]; };
            if (it.kind == 0) {
                const Node& n = nl.nodes[it.id];
                d.w = n.w;
                d.dst = slot[local[it.id]];
                switch (n.op) {
                case OP_INPUT: d.op = D_LDI; d.imm = uint32_t(n.a); break;
                case OP_REG:
                    d.op = D_LDR;
                    d.c = L.cls[n.a];
                    d.b = uint16_t(L.idx[n.a] & 0xffff);
                    d.x = uint16_t(L.idx[n.a] >> 16);
                    d.imm = uint32_t(n.a);
                    break;
                case OP_CONST:
                    d.op = D_CONST;
                    d.imm = uint32_t(n.k);
                    d.a = uint16_t(n.k >> 32);
                    d.b = uint16_t(n.k >> 48);
                    break;
                case OP_MEMRD: d.op = D_MEMRD; d.a = S(n.b); d.imm = uint32_t(n.a); break;
                case OP_SLICE: d.op = D_SLICE; d.a = S(n.a); d.x = uint16_t(n.b); break;
                case OP_CONCAT: d.op = D_CONCAT; d.a = S(n.a); d.b = S(n.b); d.x = nl.nodes[n.b].w; break;
                case OP_MUX: d.op = D_MUX; d.a = S(n.a); d.b = S(n.b); d.c = S(n.c); break;
                default:
                    d.op = uint8_t(D_ADD + (n.op - OP_ADD));
                    d.a = S(n.a);
                    d.b = S(n.b);
                }
            } else if (it.kind == 1) {
                int32_t r = it.id;
                d.op = D_STR;
                d.w = nl.reg_w[r];
                d.a = S(nl.reg_next[r]);
                d.c = L.cls[r];
                d.b = uint16_t(L.idx[r] & 0xffff);
                d.x = uint16_t(L.idx[r] >> 16);
                d.imm = uint32_t(r);
            } else if (it.kind == 2) {
                const WPort& w = nl.wports[it.id];
                d.op = D_WREC;
                d.a = S(w.en);
                d.b = S(w.addr);
                d.c = S(w.data);
                d.w = nl.mem_w[w.mem];
                d.x = nl.mem_lg[w.mem];
                d.imm = uint32_t(it.id);
            } else {
                d.op = D_COMMIT;
                d.imm = uint32_t(it.id);
            }
            return d;
        };

        // ---- LANE_OP: 32-wide bundles, slots freed after a bundle completes
        {
            std::vector<uint16_t> slot(nodes.size(), kNoSlot);
            SlotAlloc A;
            std::vector<std::vector<uint16_t>> release(nb + 1);
            size_t i = 0;
            out.s_off[p] = uint32_t(out.s_ins.size() / 32);
            for (uint32_t b = 0; b < nb; b++) {
                for (uint16_t s : release[b]) A.put(s);
                size_t base = out.s_ins.size();
                out.s_ins.resize(base + 32, DIns{});
                int lane = 0;
                for (; i < items.size() && bundle[i] == b; i++, lane++) {
                    const Item& it = items[i];
                    if (it.kind == 0) {
                        int32_t l = local[it.id];
                        slot[l] = A.get();
                        if (last_b[l] >= 0) release[last_b[l] + 1].push_back(slot[l]);
                        else release[b + 1].push_back(slot[l]);
                    }
                    out.s_ins[base + lane] = make_ins(it, slot);
                }
            }
            out.s_len[p] = nb;
            out.s_slots[p] = std::max<uint32_t>(1, A.next);
            if (A.next > 0xfff0) { err = "process needs too many value slots"; return SIM_ERR_CAPACITY; }
        }
        if (chain >= 2) {
            int rc = chained_program(nl, items, local, nodes.size(), make_ins, operands, out, p, chain, err);
            if (rc) return rc;
        } else {
            // compact copy: the occupied lanes of each row; up to four rows of
            // leaves (which never share a slot: all their consumers come later)
            // form one wide step of up to 128 instructions, and so do up to
            // four rows of register stores
            std::vector<uint32_t> count(nb, 0);
            for (size_t k = 0; k < items.size(); k++) count[bundle[k]]++;
            std::vector<CStep> steps;
            for (uint32_t b = 0; b < nb; b++) {
                const DIns* row = &out.s_ins[(size_t(out.s_off[p]) + b) * 32];
                bool operators_only = true, leaves_only = count[b] > 0, stores_only = count[b] > 0;
                for (uint32_t l = 0; l < count[b]; l++) {
                    operators_only &= row[l].op >= D_ADD && row[l].op <= D_CONCAT;
                    leaves_only &= row[l].op == D_LDR || row[l].op == D_LDI || row[l].op == D_CONST;
                    stores_only &= row[l].op == D_STR;
                }
                const uint32_t wide = leaves_only ? kStepLeaf : stores_only ? kStepStore : 0u;
                const uint32_t flags = (operators_only ? 0u : kStepGeneric) | wide;
                if (wide && !steps.empty() && (steps.back().flags & wide) &&
                    steps.back().ins.size() + count[b] <= kLeafStepMax) {
                    steps.back().ins.insert(steps.back().ins.end(), row, row + count[b]);
                    continue;
                }
                steps.push_back(CStep{flags, std::vector<DIns>(row, row + count[b])});
            }
            out.c_off[p] = uint32_t(out.c_words.size());
            int rc = append_program(steps, out.c_words, err);
            if (rc) return rc;
            out.c_size[p] = uint32_t(out.c_words.size()) - out.c_off[p];
        }
        // ---- LANE_INST: sequential list in depth-first post-order from each
        // sink (a value is computed right before its first consumer, which
        // keeps few values live), operand slots reusable by the result
        {
            std::vector<int32_t> item_of_node(nodes.size(), -1);
            for (size_t i = 0; i < items.size(); i++)
                if (items[i].kind == 0) item_of_node[local[items[i].id]] = int32_t(i);
            std::vector<int32_t> seq;
            seq.reserve(items.size());
            std::vector<uint8_t> emitted(items.size(), 0);
            std::vector<std::pair<int32_t, int>> stack;   // (item, next operand to visit)
            auto ops_of = [&](int32_t it, std::vector<int32_t>& v) {
                v.clear();
                operands(items[it], [&](int32_t o) { v.push_back(item_of_node[local[o]]); });
            };
            std::vector<int32_t> tmp;
            auto visit = [&](int32_t root) {
                if (emitted[root]) return;
                stack.push_back({root, 0});
                while (!stack.empty()) {
                    auto& [it, k] = stack.back();
                    ops_of(it, tmp);
                    if (k < int(tmp.size())) {
                        int32_t o = tmp[k++];
                        if (!emitted[o]) stack.push_back({o, 0});
                        continue;
                    }
                    int32_t done_it = it;
                    stack.pop_back();
                    if (!emitted[done_it]) {
                        emitted[done_it] = 1;
                        seq.push_back(done_it);
                    }
                }
            };
            for (size_t i = 0; i < items.size(); i++)      // commits first
                if (items[i].kind == 3) visit(int32_t(i));
            for (size_t i = 0; i < items.size(); i++)      // then every sink's cone
                if (items[i].kind == 1 || items[i].kind == 2) visit(int32_t(i));
            // last sequential use of each value in this order
            std::vector<int32_t> last_seq(nodes.size(), -1);
            for (size_t k = 0; k < seq.size(); k++)
                operands(items[seq[k]], [&](int32_t o) { last_seq[local[o]] = int32_t(k); });
            std::vector<uint16_t> slot(nodes.size(), kNoSlot);
            SlotAlloc A;
            out.b_off[p] = uint32_t(out.b_ins.size());
            std::vector<uint16_t> freed;
            for (size_t k = 0; k < seq.size(); k++) {
                const Item& it = items[seq[k]];
                freed.clear();
                operands(it, [&](int32_t o) {
                    int32_t l = local[o];
                    if (last_seq[l] == int32_t(k)) freed.push_back(slot[l]);
                });
                std::sort(freed.begin(), freed.end());
                freed.erase(std::unique(freed.begin(), freed.end()), freed.end());
                DIns d;
                if (it.kind == 0) {
                    // operands are read before the result is written, so the
                    // result may take a slot freed by this very instruction
                    int32_t l = local[it.id];
                    for (uint16_t s : freed) A.put(s);
                    slot[l] = A.get();
                    d = make_ins(it, slot);
                    if (last_seq[l] < 0) A.put(slot[l]);
                } else {
                    d = make_ins(it, slot);
                    for (uint16_t s : freed) A.put(s);
                }
                out.b_ins.push_back(d);
            }
            out.b_len[p] = uint32_t(seq.size());
            out.b_slots[p] = std::max<uint32_t>(1, A.next);
            if (A.next > 0xfff0) { err = "process needs too many value slots"; return SIM_ERR_CAPACITY; }
        }
        out.max_bundles = std::max(out.max_bundles, out.c_words[out.c_off[p]]);   // steps of the compact program
        out.max_s_slots = std::max(out.max_s_slots, out.s_slots[p]);
        out.max_b_slots = std::max(out.max_b_slots, out.b_slots[p]);
        for (int32_t id : nodes) local[id] = -1;
    }
    return SIM_OK;
}


// ---------------------------------------------------------------------------
// Cluster placement and exchange lowering
// ---------------------------------------------------------------------------
namespace {

// Steps of process p from its compact program.
std::vector<CStep> read_steps(const Lowered& low, size_t p) {
    const uint32_t* w = low.c_words.data() + low.c_off[p];
    const uint32_t nb = w[0], tw = (nb + 4) & ~3u;
    const DIns* ins = reinterpret_cast<const DIns*>(w + tw);
    std::vector<CStep> steps(nb);
    for (uint32_t b = 0; b < nb; b++) {
        const uint32_t e = w[1 + b], first = e & 0xffff, cnt = (e >> 16) & kStepCountMask;
        steps[b].flags = e & (kStepGeneric | kStepLeaf | kStepChain | kStepStore | (kStepRowsMask << kStepRowsShift));
        steps[b].ins.assign(ins + first, ins + first + cnt);
    }
    return steps;
}

}  // namespace

int lower_clusters(const Netlist& nl, const Partition& part, uint32_t C, uint32_t W, Lowered& low, ClusterPlan& plan,
                   std::string& err, bool wide_stores) {
    const size_t NP = part.procs.size();
    if (C < 1 || W < 1 || NP == 0) { err = "cluster lowering: bad geometry"; return SIM_ERR_BADARG; }
    const uint32_t G = C * W;                                   // processes per cluster
    const uint32_t n_groups = uint32_t((NP + G - 1) / G);
    plan = ClusterPlan();
    plan.C = C;
    plan.W = W;
    plan.grid = n_groups * C;

    // producer process of every register, and the registers each process reads
    std::vector<int32_t> proc_of_reg(nl.reg_w.size(), -1);
    for (size_t p = 0; p < NP; p++)
        for (int32_t f : part.procs[p])
            if (part.fibers[f].reg >= 0) proc_of_reg[part.fibers[f].reg] = int32_t(p);
    std::vector<std::vector<CStep>> steps(NP);
    std::vector<std::vector<uint32_t>> reads(NP);
    for (size_t p = 0; p < NP; p++) {
        steps[p] = read_steps(low, p);
        for (auto& st : steps[p])
            for (auto& d : st.ins)
                if (d.op == D_LDR) reads[p].push_back(d.imm);
    }

    // affinity between processes: register values passed either way
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> adj(NP);
    {
        std::vector<std::pair<uint32_t, uint32_t>> edges;
        for (size_t p = 0; p < NP; p++)
            for (uint32_t r : reads[p]) {
                int32_t q = proc_of_reg[r];
                if (q >= 0 && size_t(q) != p)
                    edges.push_back({uint32_t(std::min<size_t>(p, q)), uint32_t(std::max<size_t>(p, q))});
            }
        std::sort(edges.begin(), edges.end());
        for (size_t i = 0; i < edges.size();) {
            size_t j = i;
            while (j < edges.size() && edges[j] == edges[i]) j++;
            adj[edges[i].first].push_back({edges[i].second, uint32_t(j - i)});
            adj[edges[i].second].push_back({edges[i].first, uint32_t(j - i)});
            i = j;
        }
    }
    // placement: two streaming greedy passes (linear deterministic greedy:
    // each process joins the cluster holding most of its partners, discounted
    // by how full it is), one in breadth-first order of the communication
    // graph and one in process order; the better one is refined by swaps
    std::vector<uint64_t> weight(NP, 0);
    for (size_t p = 0; p < NP; p++)
        for (auto& e : adj[p]) weight[p] += e.second;
    auto local_weight = [&](const std::vector<int32_t>& grp) {
        uint64_t v = 0;
        for (size_t p = 0; p < NP; p++)
            for (auto& e : adj[p])
                if (grp[p] == grp[e.first]) v += e.second;
        return v / 2;
    };
    auto ldg = [&](const std::vector<uint32_t>& order) {
        std::vector<int32_t> grp(NP, -1);
        std::vector<uint32_t> size(n_groups, 0);
        std::vector<double> score(n_groups, 0.0);
        for (uint32_t p : order) {
            std::fill(score.begin(), score.end(), 0.0);
            for (auto& e : adj[p])
                if (grp[e.first] >= 0) score[grp[e.first]] += e.second;
            int32_t best = -1;
            double best_v = -1.0;
            for (uint32_t g = 0; g < n_groups; g++) {
                if (size[g] >= G) continue;
                double v = score[g] * (1.0 - double(size[g]) / G);
                if (v > best_v || (v == best_v && size[g] < size[best])) {
                    best = int32_t(g);
                    best_v = v;
                }
            }
            grp[p] = best;
            size[best]++;
        }
        return grp;
    };
    std::vector<uint32_t> bfs;
    {
        std::vector<uint8_t> seen(NP, 0);
        std::vector<uint32_t> by_weight(NP);
        std::iota(by_weight.begin(), by_weight.end(), 0u);
        std::stable_sort(by_weight.begin(), by_weight.end(), [&](uint32_t a, uint32_t b) { return weight[a] > weight[b]; });
        for (uint32_t root : by_weight) {
            if (seen[root]) continue;
            size_t head = bfs.size();
            bfs.push_back(root);
            seen[root] = 1;
            while (head < bfs.size()) {
                uint32_t p = bfs[head++];
                auto nb = adj[p];
                std::stable_sort(nb.begin(), nb.end(), [](auto& a, auto& b) { return a.second > b.second; });
                for (auto& e : nb)
                    if (!seen[e.first]) {
                        seen[e.first] = 1;
                        bfs.push_back(e.first);
                    }
            }
        }
    }
    std::vector<uint32_t> ident(NP);
    std::iota(ident.begin(), ident.end(), 0u);
    std::vector<int32_t> group = ldg(bfs);
    {
        std::vector<int32_t> g2 = ldg(ident);
        if (local_weight(g2) > local_weight(group)) group = g2;
    }
    // swap refinement: exchange two processes of different clusters when that
    // raises the weight kept inside clusters
    {
        auto gain_to = [&](uint32_t p, int32_t g) {   // partners of p in cluster g
            uint64_t v = 0;
            for (auto& e : adj[p])
                if (group[e.first] == g) v += e.second;
            return v;
        };
        for (int pass = 0; pass < 4; pass++) {
            bool moved = false;
            for (uint32_t p = 0; p < NP; p++) {
                if (adj[p].empty()) continue;
                // the cluster p is most connected to
                std::unordered_map<int32_t, uint64_t> w;
                for (auto& e : adj[p]) w[group[e.first]] += e.second;
                const int32_t gp = group[p];
                const uint64_t own = w.count(gp) ? w[gp] : 0;
                int32_t gb = gp;
                uint64_t wb = own;
                for (auto& [g, v] : w)
                    if (v > wb) { gb = g; wb = v; }
                if (gb == gp) continue;
                // the process q of gb whose move to p's cluster gains most
                int64_t best_gain = 0;
                int32_t best_q = -1;
                for (uint32_t q = 0; q < NP; q++) {
                    if (group[q] != gb) continue;
                    int64_t pq = 0;
                    for (auto& e : adj[p])
                        if (e.first == q) pq = e.second;
                    const int64_t gain = int64_t(wb) - int64_t(own) + int64_t(gain_to(q, gp)) - int64_t(gain_to(q, gb)) - 2 * pq;
                    if (gain > best_gain) { best_gain = gain; best_q = int32_t(q); }
                }
                if (best_q >= 0) {
                    group[best_q] = gp;
                    group[p] = gb;
                    moved = true;
                }
            }
            if (!moved) break;
        }
    }
    std::vector<std::vector<uint32_t>> members(n_groups);
    for (uint32_t p = 0; p < NP; p++) members[group[p]].push_back(p);
    plan.warp_proc.assign(size_t(plan.grid) * W, kNoProc);
    std::vector<uint32_t> cta_of(NP);
    for (uint32_t g = 0; g < n_groups; g++)
        for (size_t k = 0; k < members[g].size(); k++) {
            plan.warp_proc[size_t(g) * G + k] = members[g][k];
            cta_of[members[g][k]] = uint32_t((size_t(g) * G + k) / W);
        }

    // mirrors: per CTA, the registers its processes read from producers of
    // the same cluster (own CTA included)
    std::vector<std::vector<uint32_t>> mir(plan.grid);
    for (size_t p = 0; p < NP; p++) {
        const uint32_t c = cta_of[p];
        for (uint32_t r : reads[p]) {
            int32_t q = proc_of_reg[r];
            bool local = q >= 0 && cta_of[q] / C == c / C;
            if (q >= 0 && size_t(q) != p) (local ? plan.reads_local : plan.reads_remote)++;
            if (local) mir[c].push_back(r);
        }
    }
    std::vector<std::unordered_map<uint32_t, uint32_t>> mir_idx(plan.grid);
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> consumers(nl.reg_w.size());   // (CTA, entry)
    plan.mir_off.assign(plan.grid + 1, 0);
    for (uint32_t c = 0; c < plan.grid; c++) {
        auto& v = mir[c];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        plan.mir_off[c + 1] = plan.mir_off[c] + uint32_t(v.size());
        plan.mirror_words = std::max<uint32_t>(plan.mirror_words, uint32_t(v.size()));
        for (size_t i = 0; i < v.size(); i++) {
            mir_idx[c][v[i]] = uint32_t(i);
            consumers[v[i]].push_back({c, uint32_t(i)});
            plan.mir_reg.push_back(v[i]);
        }
    }
    if (plan.mirror_words > 0xffffff) { err = "cluster mirror too large"; return SIM_ERR_CAPACITY; }

    // rewrite: local reads from the mirror, mirror writes after the stores
    for (size_t p = 0; p < NP; p++) {
        const uint32_t c = cta_of[p];
        std::vector<DIns> stx;
        for (auto& st : steps[p])
            for (auto& d : st.ins) {
                if (d.op == D_LDR) {
                    auto it = mir_idx[c].find(d.imm);
                    if (it == mir_idx[c].end()) continue;
                    d.op = D_LDM;
                    d.c = 0;
                    d.b = uint16_t(it->second & 0xffff);
                    d.x = uint16_t(it->second >> 16);
                } else if (d.op == D_STR) {
                    for (auto& [cc, i] : consumers[d.imm]) {
                        DIns x{};
                        x.op = D_STX;
                        x.w = d.w;
                        x.a = d.a;
                        x.c = uint16_t(cc % C);
                        x.b = uint16_t(i & 0xffff);
                        x.x = uint16_t(i >> 16);
                        x.imm = d.imm;
                        stx.push_back(x);
                    }
                }
            }
        // without operator pairs: into the last store step while it has
        // room, then new store steps; with them: steps of 32
        const size_t width = wide_stores ? kLeafStepMax : 32;
        size_t k = 0;
        if (wide_stores && !steps[p].empty() && (steps[p].back().flags & kStepStore)) {
            auto& last = steps[p].back().ins;
            k = std::min(stx.size(), width - std::min(width, last.size()));
            last.insert(last.end(), stx.begin(), stx.begin() + k);
        }
        for (; k < stx.size(); k += width) {
            CStep st;
            st.flags = kStepGeneric | (wide_stores ? kStepStore : 0u);
            st.ins.assign(stx.begin() + k, stx.begin() + std::min(stx.size(), k + width));
            steps[p].push_back(std::move(st));
        }
    }

    // rebuild the bundle rows (32 instructions each: a wide leaf step takes
    // several) and the compact programs
    low.s_ins.clear();
    low.c_words.clear();
    low.max_bundles = 0;
    for (size_t p = 0; p < NP; p++) {
        low.s_off[p] = uint32_t(low.s_ins.size() / 32);
        for (const auto& st : steps[p]) {
            // a chain step reads as two rows: the first operators, then the second ones
            const size_t row = (st.flags & kStepChain) ? st.ins.size() / ((st.flags >> kStepRowsShift) & kStepRowsMask)
                                                       : 32;
            for (size_t k = 0; k < std::max<size_t>(1, st.ins.size()); k += row) {
                const size_t base = low.s_ins.size();
                low.s_ins.resize(base + 32, DIns{});
                const size_t n = std::min<size_t>(row, st.ins.size() - std::min(k, st.ins.size()));
                std::copy(st.ins.begin() + k, st.ins.begin() + k + n, low.s_ins.begin() + base);
            }
        }
        low.s_len[p] = uint32_t(low.s_ins.size() / 32) - low.s_off[p];
        low.c_off[p] = uint32_t(low.c_words.size());
        int rc = append_program(steps[p], low.c_words, err);
        if (rc) return rc;
        low.c_size[p] = uint32_t(low.c_words.size()) - low.c_off[p];
        low.max_bundles = std::max(low.max_bundles, low.c_words[low.c_off[p]]);
    }
    return SIM_OK;
}

}  // namespace rtl
