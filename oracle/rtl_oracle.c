/*
 * rtl_oracle.c -- plain, single-threaded CPU reference interpreter for
 * word-level RTL netlists in the `rtlnet 1` text format.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or table with the CUDA simulator; it has its own parser, its
 * own evaluator and its own stimulus and digest functions.
 *
 * What it computes (paper Sec. 3 and Sec. 3.2, "BSP RTL Simulation"):
 * cycle-accurate, zero-delay, full-cycle simulation.  Every register is split
 * into a read-only *current* value and a write-only *next* value; each cycle
 * the whole combinational graph is evaluated from the current values, then
 * every register takes its next value.  Partitioning into fibers/processes
 * (Sec. 5.1) must not change any value, so the reference is the sequential
 * definition: evaluate every node in topological order, then commit.
 *
 * Readings where the paper is silent (it works on Verilog through Verilator,
 * 2-state, Sec. 5):
 *   - values are unsigned, 1..64 bits, operands zero-extended; results are
 *     reduced modulo 2^w (add, sub, mul keep the low w bits);
 *   - shl/shr are logical with an unsigned amount; an amount >= 64 gives 0,
 *     otherwise the 64-bit shift is taken, then reduced to w bits;
 *   - eq/lt are unsigned compares of 1 bit; mux(s,a,b) = s != 0 ? a : b;
 *   - slice(a, lo) = (a >> lo) mod 2^w; concat(a, b) = a * 2^width(b) + b;
 *   - a memory read returns mem[addr mod depth] of the *current* memory;
 *     writes take effect at the clock edge, in ascending write-port order, so
 *     the highest-numbered port wins on an address conflict;
 *   - register next values are truncated or zero-extended to the register width.
 *
 * Clocks (paper Sec. 5, limitations: one top-level clock plus any number of
 * gated or divided clocks).  Our reading, in Verilog's event order:
 *   - `gate r e`: register r's clock is gated by node e; at an edge of its
 *     clock r takes its next value only if e is nonzero (e is evaluated
 *     together with r's next value);
 *   - `clock r d`: register r is clocked by the rising edge of the 1-bit
 *     register d (a divided clock).  d changes at its own clock edge, so the
 *     edge of r's clock comes after d's domain has committed: r's next value
 *     (and gate) are evaluated on the state *after* that commit, i.e. r
 *     samples the new values of the registers of earlier domains.
 *   One top-clock cycle therefore runs in phases: phase 0 evaluates every
 *   node and commits the top-clock registers and the memory writes; phase k
 *   re-evaluates every node on the state now and commits the registers whose
 *   clock register (of phase k-1) went from 0 at the start of the cycle to 1.
 *   Memory reads in the cone of a register on a divided clock are rejected
 *   (write ports are on the top clock).
 *
 * Stimulus: each input value is drawn from SplitMix64 (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), used as a
 * counter-based generator: output number n of a SplitMix64 stream seeded
 * with s is mix(s + n * gamma).  The per-instance key is output number
 * (inst + 1) of the stream seeded with `seed`; input k of cycle t is output
 * number (t * n_inputs + k + 1) of the stream seeded with the key, reduced to
 * the input width.
 *
 * Digest of a state: sum over registers r of mix(H(r) ^ reg[r]) plus sum over
 * memory words of mix(H(2^40 + m * 2^24 + a) ^ mem[m][a]), modulo 2^64, with
 * H(x) = x * gamma + 1 and mix the SplitMix64 output function.  It is
 * recomputed from scratch for every state.
 */
#define _POSIX_C_SOURCE 200809L
#include <ctype.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

enum {
    K_INPUT, K_REG, K_CONST, K_MEMRD,
    K_ADD, K_SUB, K_MUL, K_AND, K_OR, K_XOR, K_SHL, K_SHR, K_EQ, K_LT,
    K_MUX, K_SLICE, K_CONCAT, K_COUNT
};
static const char *KNAMES[K_COUNT] = {
    "input", "reg", "const", "memrd", "add", "sub", "mul", "and", "or", "xor",
    "shl", "shr", "eq", "lt", "mux", "slice", "concat"};

typedef struct {
    int kind;
    int width;
    int64_t arg[3];       /* node ids, or an index (input, reg, mem, slice lo) */
    uint64_t value;       /* const value */
} onode;

typedef struct {
    int n_in, n_reg, n_mem, n_node, n_wport;
    int *in_w;
    int *reg_w;
    uint64_t *reg_init;
    int64_t *reg_next;
    int64_t *reg_gate;    /* gate node of each register, or -1 */
    int64_t *reg_clk;     /* clock register of each register, or -1 (top clock) */
    int *reg_depth;       /* 0 on the top clock, 1 + depth of the clock register */
    int max_depth;
    int *mem_lg, *mem_w;
    uint64_t **mem_init;  /* per memory, depth words */
    onode *node;
    int64_t *wp_mem, *wp_en, *wp_addr, *wp_data;
    int64_t *order;       /* topological order of all nodes */
    /* The nodes copied into evaluation order: step j evaluates node order[j]
     * and its operands are named by their evaluation positions, so the value
     * array is indexed by position and the steps are read sequentially. */
    onode *step;
    int64_t *pos;         /* evaluation position of each node id */
} onet;

typedef struct {
    const onet *net;
    int n_mem;            /* copy of net->n_mem: freeing an instance never reads its net */
    uint64_t key;         /* stimulus key of this instance */
    uint64_t cycle;
    uint64_t *reg;        /* current register values */
    uint64_t *reg_nx;     /* scratch for next values */
    uint64_t *reg_start;  /* register values at the start of the cycle */
    uint64_t **mem;
    uint64_t *val;        /* node values of the cycle being evaluated */
    uint64_t *in_val;
    uint8_t *held;        /* input k is held at in_hold[k] */
    uint64_t *in_hold;
} osim;

/* ------------------------------------------------------------------------- */
/* Arithmetic helpers                                                         */
/* ------------------------------------------------------------------------- */
static uint64_t mask_of(int w) { return w >= 64 ? ~0ULL : ((1ULL << w) - 1ULL); }

uint64_t orc_mix64(uint64_t z)
{
    /* SplitMix64 output function (Steele, Lea, Flood 2014). */
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number n (n >= 1) of the SplitMix64 stream seeded with s. */
static uint64_t splitmix_nth(uint64_t s, uint64_t n) { return orc_mix64(s + n * GAMMA); }

uint64_t orc_instance_key(uint64_t seed, uint64_t inst) { return splitmix_nth(seed, inst + 1); }

uint64_t orc_stimulus(uint64_t seed, uint64_t inst, uint64_t t, uint32_t k, uint32_t n_in, int w)
{
    uint64_t key = orc_instance_key(seed, inst);
    return splitmix_nth(key, t * (uint64_t)n_in + k + 1) & mask_of(w);
}

/* One combinational operator (node semantics listed in the header). */
static inline uint64_t op_eval(int kind, int w, uint64_t a, uint64_t b, uint64_t c, int wb, int lo)
{
    uint64_t m = mask_of(w), r = 0;
    switch (kind) {
    case K_ADD: r = a + b; break;
    case K_SUB: r = a - b; break;
    case K_MUL: r = a * b; break;
    case K_AND: r = a & b; break;
    case K_OR:  r = a | b; break;
    case K_XOR: r = a ^ b; break;
    case K_SHL: r = b >= 64 ? 0 : a << b; break;
    case K_SHR: r = b >= 64 ? 0 : a >> b; break;
    case K_EQ:  r = a == b; break;
    case K_LT:  r = a < b; break;
    case K_MUX: r = a != 0 ? b : c; break;    /* here a is the select */
    case K_SLICE: r = lo >= 64 ? 0 : a >> lo; break;
    case K_CONCAT: r = wb >= 64 ? b : (a << wb) | b; break;
    default: r = 0;
    }
    return r & m;
}

uint64_t orc_op(int kind, int w, uint64_t a, uint64_t b, uint64_t c, int wb, int lo)
{
    return op_eval(kind, w, a, b, c, wb, lo);
}

static uint64_t hash_reg(uint64_t r) { return r * GAMMA + 1ULL; }

/* ------------------------------------------------------------------------- */
/* Parser                                                                     */
/* ------------------------------------------------------------------------- */

static int fail(char *err, size_t errlen, const char *fmt, ...)
{
    if (err && errlen) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, errlen, fmt, ap);
        va_end(ap);
    }
    return -1;
}

#define GROW(ptr, cnt, cap)                                                   \
    do {                                                                      \
        if ((size_t)(cnt) >= (cap)) {                                         \
            (cap) = (cap) ? (cap) * 2 : 64;                                   \
            void *np_ = realloc((ptr), sizeof(*(ptr)) * (size_t)(cap));       \
            if (!np_) return fail(err, errlen, "out of memory");              \
            (ptr) = np_;                                                      \
        }                                                                     \
    } while (0)

void orc_net_free(onet *n);

static int tokens(char *line, char **tok, int maxtok)
{
    int nt = 0;
    char *p = line;
    while (*p && nt < maxtok) {
        while (*p && isspace((unsigned char)*p)) p++;
        if (!*p || *p == '#') break;
        tok[nt++] = p;
        while (*p && !isspace((unsigned char)*p)) p++;
        if (*p) *p++ = 0;
    }
    return nt;
}

static int parse_u64(const char *s, uint64_t *out)
{
    char *end;
    if (!s || !*s || *s == '-') return -1;
    *out = strtoull(s, &end, 0);
    return *end ? -1 : 0;
}

static int parse_i64(const char *s, int64_t *out)
{
    uint64_t u;
    if (parse_u64(s, &u)) return -1;
    if (u > (uint64_t)INT64_MAX) return -1;
    *out = (int64_t)u;
    return 0;
}

static int parse_text(onet *n, char *text, char *err, size_t errlen)
{
    size_t cap_in = 0, cap_reg = 0, cap_mem = 0, cap_node = 0, cap_wp = 0;
    int64_t n_minit = 0;
    struct mi { int64_t m, a; uint64_t v; } *minit = NULL; size_t cap_mi = 0;
    char *tok[8];
    int line_no = 0, saw_header = 0, saw_end = 0;
    char *p = text;
    while (*p) {
        char *line = p;
        while (*p && *p != '\n') p++;
        if (*p) *p++ = 0;
        line_no++;
        int nt = tokens(line, tok, 8);
        if (nt == 0) continue;
        if (saw_end) return fail(err, errlen, "line %d: content after end", line_no);
        if (!saw_header) {
            if (nt != 2 || strcmp(tok[0], "rtlnet") || strcmp(tok[1], "1"))
                return fail(err, errlen, "line %d: expected 'rtlnet 1'", line_no);
            saw_header = 1;
            continue;
        }
        if (!strcmp(tok[0], "in")) {
            int64_t w;
            if (nt < 2 || parse_i64(tok[1], &w)) return fail(err, errlen, "line %d: bad in", line_no);
            GROW(n->in_w, n->n_in, cap_in);
            n->in_w[n->n_in++] = (int)w;
        } else if (!strcmp(tok[0], "reg")) {
            int64_t w; uint64_t init;
            if (nt < 3 || parse_i64(tok[1], &w) || parse_u64(tok[2], &init))
                return fail(err, errlen, "line %d: bad reg", line_no);
            if (n->n_reg >= (int)cap_reg) {
                size_t c = cap_reg;
                GROW(n->reg_w, n->n_reg, c);
                c = cap_reg; GROW(n->reg_init, n->n_reg, c);
                c = cap_reg; GROW(n->reg_next, n->n_reg, c);
                c = cap_reg; GROW(n->reg_gate, n->n_reg, c);
                c = cap_reg; GROW(n->reg_clk, n->n_reg, c);
                cap_reg = c;
            }
            n->reg_w[n->n_reg] = (int)w;
            n->reg_init[n->n_reg] = init;
            n->reg_next[n->n_reg] = -1;
            n->reg_gate[n->n_reg] = -1;
            n->reg_clk[n->n_reg] = -1;
            n->n_reg++;
        } else if (!strcmp(tok[0], "mem")) {
            int64_t lg, w;
            if (nt < 3 || parse_i64(tok[1], &lg) || parse_i64(tok[2], &w))
                return fail(err, errlen, "line %d: bad mem", line_no);
            if (n->n_mem >= (int)cap_mem) {
                size_t c = cap_mem;
                GROW(n->mem_lg, n->n_mem, c);
                c = cap_mem; GROW(n->mem_w, n->n_mem, c);
                cap_mem = c;
            }
            n->mem_lg[n->n_mem] = (int)lg;
            n->mem_w[n->n_mem] = (int)w;
            n->n_mem++;
        } else if (!strcmp(tok[0], "n")) {
            onode nd;
            int64_t w;
            memset(&nd, 0, sizeof nd);
            nd.arg[0] = nd.arg[1] = nd.arg[2] = -1;
            if (nt < 3 || parse_i64(tok[2], &w)) return fail(err, errlen, "line %d: bad node", line_no);
            nd.kind = -1;
            for (int k = 0; k < K_COUNT; k++)
                if (!strcmp(tok[1], KNAMES[k])) nd.kind = k;
            if (nd.kind < 0) return fail(err, errlen, "line %d: unknown op '%s'", line_no, tok[1]);
            nd.width = (int)w;
            int want = (nd.kind == K_MUX) ? 3 : (nd.kind == K_INPUT || nd.kind == K_REG || nd.kind == K_CONST) ? 1 : 2;
            if (nt != 3 + want) return fail(err, errlen, "line %d: op %s takes %d args", line_no, tok[1], want);
            if (nd.kind == K_CONST) {
                if (parse_u64(tok[3], &nd.value)) return fail(err, errlen, "line %d: bad const", line_no);
            } else {
                for (int k = 0; k < want; k++)
                    if (parse_i64(tok[3 + k], &nd.arg[k])) return fail(err, errlen, "line %d: bad arg", line_no);
            }
            GROW(n->node, n->n_node, cap_node);
            n->node[n->n_node++] = nd;
        } else if (!strcmp(tok[0], "next")) {
            int64_t r, x;
            if (nt != 3 || parse_i64(tok[1], &r) || parse_i64(tok[2], &x))
                return fail(err, errlen, "line %d: bad next", line_no);
            if (r < 0 || r >= n->n_reg) return fail(err, errlen, "line %d: next of unknown register", line_no);
            if (n->reg_next[r] >= 0) return fail(err, errlen, "line %d: register %lld has two next", line_no, (long long)r);
            n->reg_next[r] = x;
        } else if (!strcmp(tok[0], "gate") || !strcmp(tok[0], "clock")) {
            int64_t r, x;
            int is_gate = !strcmp(tok[0], "gate");
            if (nt != 3 || parse_i64(tok[1], &r) || parse_i64(tok[2], &x))
                return fail(err, errlen, "line %d: bad %s", line_no, tok[0]);
            if (r < 0 || r >= n->n_reg) return fail(err, errlen, "line %d: %s of unknown register", line_no, tok[0]);
            int64_t *slot = is_gate ? &n->reg_gate[r] : &n->reg_clk[r];
            if (*slot >= 0) return fail(err, errlen, "line %d: register %lld has two %s items", line_no, (long long)r, tok[0]);
            *slot = x;
        } else if (!strcmp(tok[0], "wport")) {
            int64_t v[4];
            if (nt != 5) return fail(err, errlen, "line %d: bad wport", line_no);
            for (int k = 0; k < 4; k++)
                if (parse_i64(tok[1 + k], &v[k])) return fail(err, errlen, "line %d: bad wport", line_no);
            if (n->n_wport >= (int)cap_wp) {
                size_t c = cap_wp;
                GROW(n->wp_mem, n->n_wport, c);
                c = cap_wp; GROW(n->wp_en, n->n_wport, c);
                c = cap_wp; GROW(n->wp_addr, n->n_wport, c);
                c = cap_wp; GROW(n->wp_data, n->n_wport, c);
                cap_wp = c;
            }
            n->wp_mem[n->n_wport] = v[0];
            n->wp_en[n->n_wport] = v[1];
            n->wp_addr[n->n_wport] = v[2];
            n->wp_data[n->n_wport] = v[3];
            n->n_wport++;
        } else if (!strcmp(tok[0], "minit")) {
            struct mi e;
            if (nt != 4 || parse_i64(tok[1], &e.m) || parse_i64(tok[2], &e.a) || parse_u64(tok[3], &e.v))
                return fail(err, errlen, "line %d: bad minit", line_no);
            GROW(minit, (size_t)n_minit, cap_mi);
            minit[n_minit++] = e;
        } else if (!strcmp(tok[0], "end")) {
            saw_end = 1;
        } else {
            return fail(err, errlen, "line %d: unknown item '%s'", line_no, tok[0]);
        }
    }
    if (!saw_header) { free(minit); return fail(err, errlen, "missing 'rtlnet 1' header"); }
    if (!saw_end) { free(minit); return fail(err, errlen, "missing 'end'"); }

    /* memory images */
    n->mem_init = calloc((size_t)n->n_mem + 1, sizeof(uint64_t *));
    for (int m = 0; m < n->n_mem; m++) {
        if (n->mem_lg[m] < 0 || n->mem_lg[m] > 24) { free(minit); return fail(err, errlen, "memory %d: log2 depth out of range", m); }
        if (n->mem_w[m] < 1 || n->mem_w[m] > 64) { free(minit); return fail(err, errlen, "memory %d: width out of range", m); }
        n->mem_init[m] = calloc((size_t)1 << n->mem_lg[m], sizeof(uint64_t));
    }
    for (int64_t i = 0; i < n_minit; i++) {
        if (minit[i].m < 0 || minit[i].m >= n->n_mem || minit[i].a < 0 || minit[i].a >= ((int64_t)1 << n->mem_lg[minit[i].m])) {
            free(minit);
            return fail(err, errlen, "minit out of range");
        }
        n->mem_init[minit[i].m][minit[i].a] = minit[i].v & mask_of(n->mem_w[minit[i].m]);
    }
    free(minit);
    return 0;
}

/* Which of arg[0..2] are node operands (bit k set) for a node kind. */
static int operand_bits(int kind)
{
    switch (kind) {
    case K_INPUT: case K_REG: case K_CONST: return 0;
    case K_MEMRD: return 2;        /* arg[0] is the memory, arg[1] the address */
    case K_SLICE: return 1;        /* arg[1] is the low bit index */
    case K_MUX: return 7;
    default: return 3;
    }
}

static int cmp_i64(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return a < b ? -1 : a > b;
}

/* Sort one level's node ids by (operator kind, id). */
static void sort_level_by_kind(const onet *n, int64_t *ids, int64_t cnt)
{
    int64_t start[K_COUNT + 1] = {0};
    qsort(ids, (size_t)cnt, sizeof(int64_t), cmp_i64);
    int64_t *tmp = malloc(sizeof(int64_t) * (size_t)(cnt + 1));
    for (int64_t i = 0; i < cnt; i++) start[n->node[ids[i]].kind + 1]++;
    for (int k = 0; k < K_COUNT; k++) start[k + 1] += start[k];
    for (int64_t i = 0; i < cnt; i++) tmp[start[n->node[ids[i]].kind]++] = ids[i];
    memcpy(ids, tmp, sizeof(int64_t) * (size_t)cnt);
    free(tmp);
}

/* Structural checks and topological order (Kahn's algorithm). */
static int check_and_order(onet *n, char *err, size_t errlen)
{
    int64_t N = n->n_node;
    for (int k = 0; k < n->n_in; k++)
        if (n->in_w[k] < 1 || n->in_w[k] > 64) return fail(err, errlen, "input %d: width out of range", k);
    for (int r = 0; r < n->n_reg; r++) {
        if (n->reg_w[r] < 1 || n->reg_w[r] > 64) return fail(err, errlen, "register %d: width out of range", r);
        if (n->reg_next[r] < 0 || n->reg_next[r] >= N) return fail(err, errlen, "register %d: missing or bad next", r);
        n->reg_init[r] &= mask_of(n->reg_w[r]);
        if (n->reg_gate[r] >= N) return fail(err, errlen, "register %d: bad gate node", r);
        if (n->reg_clk[r] >= 0) {
            int64_t d = n->reg_clk[r];
            if (d >= n->n_reg || d == r) return fail(err, errlen, "register %d: bad clock register", r);
            if (n->reg_w[d] != 1) return fail(err, errlen, "register %d: clock register must be 1 bit", r);
        }
    }
    /* depth of each register's clock: the length of its chain of clock registers */
    n->reg_depth = calloc((size_t)n->n_reg + 1, sizeof(int));
    n->max_depth = 0;
    for (int r = 0; r < n->n_reg; r++) {
        int depth = 0;
        for (int64_t q = n->reg_clk[r]; q >= 0; q = n->reg_clk[q])
            if (++depth > n->n_reg) return fail(err, errlen, "register %d: loop of clock registers", r);
        n->reg_depth[r] = depth;
        if (depth > n->max_depth) n->max_depth = depth;
    }
    for (int p = 0; p < n->n_wport; p++) {
        if (n->wp_mem[p] < 0 || n->wp_mem[p] >= n->n_mem) return fail(err, errlen, "wport %d: bad memory", p);
        if (n->wp_en[p] < 0 || n->wp_en[p] >= N || n->wp_addr[p] < 0 || n->wp_addr[p] >= N || n->wp_data[p] < 0 || n->wp_data[p] >= N)
            return fail(err, errlen, "wport %d: bad node", p);
    }
    int *indeg = calloc((size_t)N + 1, sizeof(int));
    for (int64_t i = 0; i < N; i++) {
        onode *d = &n->node[i];
        if (d->width < 1 || d->width > 64) { free(indeg); return fail(err, errlen, "node %lld: width out of range", (long long)i); }
        switch (d->kind) {
        case K_INPUT:
            if (d->arg[0] >= n->n_in || d->width != n->in_w[d->arg[0]]) { free(indeg); return fail(err, errlen, "node %lld: bad input", (long long)i); }
            break;
        case K_REG:
            if (d->arg[0] >= n->n_reg || d->width != n->reg_w[d->arg[0]]) { free(indeg); return fail(err, errlen, "node %lld: bad reg", (long long)i); }
            break;
        case K_CONST: d->value &= mask_of(d->width); break;
        case K_MEMRD:
            if (d->arg[0] >= n->n_mem || d->width != n->mem_w[d->arg[0]]) { free(indeg); return fail(err, errlen, "node %lld: bad memrd", (long long)i); }
            break;
        default: break;
        }
        for (int k = 0; k < 3; k++) {
            if (!(operand_bits(d->kind) >> k & 1)) continue;
            if (d->arg[k] < 0 || d->arg[k] >= N) { free(indeg); return fail(err, errlen, "node %lld: operand out of range", (long long)i); }
            indeg[i]++;
        }
        if (d->kind == K_SLICE && d->arg[1] + d->width > n->node[d->arg[0]].width) { free(indeg); return fail(err, errlen, "node %lld: bad slice", (long long)i); }
        if (d->kind == K_CONCAT && d->width != n->node[d->arg[0]].width + n->node[d->arg[1]].width) { free(indeg); return fail(err, errlen, "node %lld: bad concat", (long long)i); }
        if ((d->kind == K_EQ || d->kind == K_LT) && d->width != 1) { free(indeg); return fail(err, errlen, "node %lld: compare must be 1 bit", (long long)i); }
    }
    /* consumers of each node (CSR) */
    int64_t *cnt = calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t i = 0; i < N; i++)
        for (int k = 0; k < 3; k++)
            if (operand_bits(n->node[i].kind) >> k & 1) cnt[n->node[i].arg[k] + 1]++;
    for (int64_t i = 0; i < N; i++) cnt[i + 1] += cnt[i];
    int64_t *users = malloc(sizeof(int64_t) * (size_t)(cnt[N] + 1));
    int64_t *fillp = malloc(sizeof(int64_t) * (size_t)(N + 1));
    memcpy(fillp, cnt, sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; i++)
        for (int k = 0; k < 3; k++)
            if (operand_bits(n->node[i].kind) >> k & 1) users[fillp[n->node[i].arg[k]]++] = i;
    /* Kahn's algorithm by levels: level 0 holds the nodes without operands,
     * level L the nodes whose last operand became ready in level L-1.  Any
     * order of nodes inside one level is a topological order; sorting each
     * level by operator kind only makes the evaluation loop's branches
     * predictable. */
    n->order = malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < N; i++)
        if (indeg[i] == 0) n->order[tail++] = i;
    while (head < tail) {
        int64_t level_end = tail;
        sort_level_by_kind(n, n->order + head, level_end - head);
        for (; head < level_end; head++) {
            int64_t i = n->order[head];
            for (int64_t u = cnt[i]; u < cnt[i + 1]; u++)
                if (--indeg[users[u]] == 0) n->order[tail++] = users[u];
        }
    }
    free(indeg); free(cnt); free(users); free(fillp);
    if (tail != N) return fail(err, errlen, "combinational loop");
    /* no memory read in the cone of a register on a divided clock */
    if (n->max_depth > 0) {
        int64_t *seen = calloc((size_t)N + 1, sizeof(int64_t));
        int64_t *stack = malloc(sizeof(int64_t) * (size_t)(N + 1));
        for (int r = 0; r < n->n_reg; r++) {
            if (n->reg_depth[r] == 0) continue;
            int64_t sp = 0;
            stack[sp++] = n->reg_next[r];
            if (n->reg_gate[r] >= 0) stack[sp++] = n->reg_gate[r];
            while (sp > 0) {
                int64_t i = stack[--sp];
                if (seen[i] == r + 1) continue;
                seen[i] = r + 1;
                if (n->node[i].kind == K_MEMRD) {
                    free(seen); free(stack);
                    return fail(err, errlen, "register %d: memory read under a divided clock", r);
                }
                for (int k = 0; k < 3; k++)
                    if (operand_bits(n->node[i].kind) >> k & 1) stack[sp++] = n->node[i].arg[k];
            }
        }
        free(seen); free(stack);
    }
    n->pos = malloc(sizeof(int64_t) * (size_t)(N + 1));
    n->step = malloc(sizeof(onode) * (size_t)(N + 1));
    for (int64_t j = 0; j < N; j++) n->pos[n->order[j]] = j;
    for (int64_t j = 0; j < N; j++) {
        onode d = n->node[n->order[j]];
        for (int k = 0; k < 3; k++)
            if (operand_bits(d.kind) >> k & 1) d.arg[k] = n->pos[d.arg[k]];
        if (d.kind == K_CONCAT)           /* width of operand b, by its node id */
            d.value = (uint64_t)n->node[n->node[n->order[j]].arg[1]].width;
        n->step[j] = d;
    }
    return 0;
}

onet *orc_net_load_text(const char *text, size_t len, char *err, size_t errlen)
{
    onet *n = calloc(1, sizeof(onet));
    char *copy = malloc(len + 1);
    memcpy(copy, text, len);
    copy[len] = 0;
    if (parse_text(n, copy, err, errlen) || check_and_order(n, err, errlen)) {
        free(copy);
        orc_net_free(n);
        return NULL;
    }
    free(copy);
    return n;
}

onet *orc_net_load_file(const char *path, char *err, size_t errlen)
{
    FILE *f = fopen(path, "rb");
    if (!f) { fail(err, errlen, "cannot open %s", path); return NULL; }
    fseek(f, 0, SEEK_END);
    long sz = ftell(f);
    fseek(f, 0, SEEK_SET);
    char *buf = malloc((size_t)sz + 1);
    size_t got = fread(buf, 1, (size_t)sz, f);
    fclose(f);
    onet *n = orc_net_load_text(buf, got, err, errlen);
    free(buf);
    return n;
}

void orc_net_free(onet *n)
{
    if (!n) return;
    free(n->in_w); free(n->reg_w); free(n->reg_init); free(n->reg_next);
    free(n->reg_gate); free(n->reg_clk); free(n->reg_depth);
    if (n->mem_init)
        for (int m = 0; m < n->n_mem; m++) free(n->mem_init[m]);
    free(n->mem_init); free(n->mem_lg); free(n->mem_w);
    free(n->node); free(n->wp_mem); free(n->wp_en); free(n->wp_addr); free(n->wp_data);
    free(n->order); free(n->step); free(n->pos);
    free(n);
}

void orc_net_counts(const onet *n, int *out5)
{
    out5[0] = n->n_in; out5[1] = n->n_reg; out5[2] = n->n_mem; out5[3] = n->n_node; out5[4] = n->n_wport;
}

int orc_net_mem_lg(const onet *n, int m) { return n->mem_lg[m]; }

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
void orc_sim_reset(osim *s, uint64_t seed, uint64_t inst)
{
    const onet *n = s->net;
    s->key = orc_instance_key(seed, inst);
    s->cycle = 0;
    for (int r = 0; r < n->n_reg; r++) s->reg[r] = n->reg_init[r];
    for (int m = 0; m < n->n_mem; m++)
        memcpy(s->mem[m], n->mem_init[m], sizeof(uint64_t) << n->mem_lg[m]);
    memset(s->held, 0, (size_t)n->n_in + 1);
}

osim *orc_sim_new(const onet *n, uint64_t seed, uint64_t inst)
{
    osim *s = calloc(1, sizeof(osim));
    s->net = n;
    s->n_mem = n->n_mem;
    s->reg = calloc((size_t)n->n_reg + 1, sizeof(uint64_t));
    s->reg_nx = calloc((size_t)n->n_reg + 1, sizeof(uint64_t));
    s->reg_start = calloc((size_t)n->n_reg + 1, sizeof(uint64_t));
    s->mem = calloc((size_t)n->n_mem + 1, sizeof(uint64_t *));
    for (int m = 0; m < n->n_mem; m++) s->mem[m] = calloc((size_t)1 << n->mem_lg[m], sizeof(uint64_t));
    s->val = calloc((size_t)n->n_node + 1, sizeof(uint64_t));
    s->in_val = calloc((size_t)n->n_in + 1, sizeof(uint64_t));
    s->in_hold = calloc((size_t)n->n_in + 1, sizeof(uint64_t));
    s->held = calloc((size_t)n->n_in + 1, 1);
    orc_sim_reset(s, seed, inst);
    return s;
}

void orc_sim_free(osim *s)
{
    if (!s) return;
    for (int m = 0; m < s->n_mem; m++) free(s->mem[m]);
    free(s->mem); free(s->reg); free(s->reg_nx); free(s->reg_start); free(s->val); free(s->in_val);
    free(s->in_hold); free(s->held);
    free(s);
}

/* Digest of the current state, recomputed from every register and word. */
uint64_t orc_sim_digest(const osim *s)
{
    const onet *n = s->net;
    uint64_t d = 0;
    for (int r = 0; r < n->n_reg; r++) d += orc_mix64(hash_reg((uint64_t)r) ^ s->reg[r]);
    for (int m = 0; m < n->n_mem; m++) {
        uint64_t depth = 1ULL << n->mem_lg[m];
        for (uint64_t a = 0; a < depth; a++)
            d += orc_mix64(hash_reg((1ULL << 40) + ((uint64_t)m << 24) + a) ^ s->mem[m][a]);
    }
    return d;
}

/* Every node in topological order from the current state and the inputs of
 * this cycle; s->val[j] is the value of the node at evaluation position j. */
static void eval_nodes(osim *s)
{
    const onet *n = s->net;
    for (int64_t j = 0; j < n->n_node; j++) {
        const onode *d = &n->step[j];
        uint64_t v;
        switch (d->kind) {
        case K_INPUT: v = s->in_val[d->arg[0]]; break;
        case K_REG:   v = s->reg[d->arg[0]]; break;
        case K_CONST: v = d->value; break;
        case K_MEMRD: {
            uint64_t depth = 1ULL << n->mem_lg[d->arg[0]];
            v = s->mem[d->arg[0]][s->val[d->arg[1]] & (depth - 1)];
            break;
        }
        case K_SLICE:
            v = op_eval(K_SLICE, d->width, s->val[d->arg[0]], 0, 0, 0, (int)d->arg[1]);
            break;
        case K_CONCAT:   /* value holds the width of operand b */
            v = op_eval(K_CONCAT, d->width, s->val[d->arg[0]], s->val[d->arg[1]], 0, (int)d->value, 0);
            break;
        case K_MUX:
            v = op_eval(K_MUX, d->width, s->val[d->arg[0]], s->val[d->arg[1]], s->val[d->arg[2]], 0, 0);
            break;
        default:
            v = op_eval(d->kind, d->width, s->val[d->arg[0]], s->val[d->arg[1]], 0, 0, 0);
        }
        s->val[j] = v;
    }
}

/* Next value of register r from the node values just evaluated: its next
 * node resized to its width, or its current value when its gate is 0. */
static uint64_t reg_next_value(const osim *s, int r)
{
    const onet *n = s->net;
    if (n->reg_gate[r] >= 0 && s->val[n->pos[n->reg_gate[r]]] == 0) return s->reg[r];
    return s->val[n->pos[n->reg_next[r]]] & mask_of(n->reg_w[r]);
}

/* One simulated clock cycle: S_t -> S_{t+1} (paper Sec. 3.2). */
static void step_once(osim *s)
{
    const onet *n = s->net;
    /* (1) inputs of this cycle: held value, else the stimulus */
    for (int k = 0; k < n->n_in; k++)
        s->in_val[k] = s->held[k] ? (s->in_hold[k] & mask_of(n->in_w[k]))
                                  : (splitmix_nth(s->key, s->cycle * (uint64_t)n->n_in + (uint64_t)k + 1) & mask_of(n->in_w[k]));
    /* (2) every node from the current values only */
    eval_nodes(s);
    if (n->max_depth > 0) memcpy(s->reg_start, s->reg, sizeof(uint64_t) * (size_t)n->n_reg);
    /* (3) top-clock registers take their next values (resized), then commit */
    for (int r = 0; r < n->n_reg; r++)
        s->reg_nx[r] = n->reg_depth[r] == 0 ? reg_next_value(s, r) : s->reg[r];
    memcpy(s->reg, s->reg_nx, sizeof(uint64_t) * (size_t)n->n_reg);
    /* (4) memory writes in ascending port order (highest port wins) */
    for (int p = 0; p < n->n_wport; p++) {
        int m = (int)n->wp_mem[p];
        if (s->val[n->pos[n->wp_en[p]]] != 0) {
            uint64_t a = s->val[n->pos[n->wp_addr[p]]] & ((1ULL << n->mem_lg[m]) - 1);
            s->mem[m][a] = s->val[n->pos[n->wp_data[p]]] & mask_of(n->mem_w[m]);
        }
    }
    /* (5) divided clocks, one phase per depth: re-evaluate on the state after
     * the previous phase's commit; a register whose clock register rose
     * (0 at the start of the cycle, 1 now) takes its next value */
    for (int depth = 1; depth <= n->max_depth; depth++) {
        eval_nodes(s);
        for (int r = 0; r < n->n_reg; r++) {
            if (n->reg_depth[r] != depth) continue;
            int64_t d = n->reg_clk[r];
            int rose = s->reg_start[d] == 0 && s->reg[d] != 0;
            s->reg_nx[r] = rose ? reg_next_value(s, r) : s->reg[r];
        }
        for (int r = 0; r < n->n_reg; r++)
            if (n->reg_depth[r] == depth) s->reg[r] = s->reg_nx[r];
    }
    s->cycle++;
}

/* Run n cycles; digests[i] (if given) receives the digest of S_{cycle+i+1}. */
void orc_sim_run(osim *s, uint64_t ncycles, uint64_t *digests)
{
    for (uint64_t i = 0; i < ncycles; i++) {
        step_once(s);
        if (digests) digests[i] = orc_sim_digest(s);
    }
}

uint64_t orc_sim_cycle(const osim *s) { return s->cycle; }
void orc_sim_set_cycle(osim *s, uint64_t c) { s->cycle = c; }
uint64_t orc_sim_get_reg(const osim *s, int r) { return s->reg[r]; }
void orc_sim_set_reg(osim *s, int r, uint64_t v) { s->reg[r] = v & mask_of(s->net->reg_w[r]); }
void orc_sim_get_regs(const osim *s, uint64_t *out) { memcpy(out, s->reg, sizeof(uint64_t) * (size_t)s->net->n_reg); }
uint64_t orc_sim_get_mem(const osim *s, int m, uint64_t a) { return s->mem[m][a & ((1ULL << s->net->mem_lg[m]) - 1)]; }
void orc_sim_set_mem(osim *s, int m, uint64_t a, uint64_t v)
{
    s->mem[m][a & ((1ULL << s->net->mem_lg[m]) - 1)] = v & mask_of(s->net->mem_w[m]);
}
void orc_sim_hold_input(osim *s, int k, uint64_t v) { s->held[k] = 1; s->in_hold[k] = v; }
void orc_sim_release_input(osim *s, int k) { s->held[k] = 0; }
/* Value of node id i in the most recent cycle (for brute-force cross-checks). */
uint64_t orc_sim_node_value(const osim *s, int64_t i) { return s->val[s->net->pos[i]]; }

#ifdef ORACLE_MAIN
#include <time.h>
/* rtl_oracle <netlist> <seed> <inst> <cycles> : prints the final digest and timing. */
int main(int argc, char **argv)
{
    char err[256];
    if (argc < 5) { fprintf(stderr, "usage: %s net seed inst cycles\n", argv[0]); return 2; }
    onet *n = orc_net_load_file(argv[1], err, sizeof err);
    if (!n) { fprintf(stderr, "error: %s\n", err); return 1; }
    osim *s = orc_sim_new(n, strtoull(argv[2], 0, 0), strtoull(argv[3], 0, 0));
    struct timespec a, b;
    clock_gettime(CLOCK_MONOTONIC, &a);
    orc_sim_run(s, strtoull(argv[4], 0, 0), NULL);
    clock_gettime(CLOCK_MONOTONIC, &b);
    double dt = (double)(b.tv_sec - a.tv_sec) + 1e-9 * (double)(b.tv_nsec - a.tv_nsec);
    printf("{\"digest\": %llu, \"seconds\": %.6f}\n", (unsigned long long)orc_sim_digest(s), dt);
    orc_sim_free(s);
    orc_net_free(n);
    return 0;
}
#endif
