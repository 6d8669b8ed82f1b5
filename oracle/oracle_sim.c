/*
 * oracle_sim.c -- plain serial CPU reference for cycle-based RTL stuck-at fault
 * simulation. TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg call it; the product path never does.
 *
 * What it computes is the plain definition of the problem (Sec. II-B, "RTL Fault
 * Simulation"): inject ONE stuck-at fault, simulate the whole design cycle by cycle,
 * and detect the fault by comparing the faulty values of the primary outputs with the
 * good values obtained without faults. The paper's concurrent algorithm (good gate plus
 * bad gates per node, Sec. II-B) simulates many faulty machines together; it must reach
 * exactly this result, so the oracle is the one-machine-at-a-time definition written out,
 * with no event skipping, no sharing between faults and no reordering:
 *
 *   good run:  Q[r] = 0;  for t in 0..T-1:
 *                net[input i]  = stim[t][i] masked to its width
 *                net[reg r]    = Q[r]
 *                net[node n]   = op_n(operands) masked to width(n), in topological order
 *                gout[t][o]    = net[outputs[o]]
 *                Q[r]          = net[d_r] masked to width(r)     (global synchronization:
 *                                the non-blocking-assignment latch at the end of the cycle)
 *   fault (s, b, v): the same loop, but every time net[s] is produced (input read,
 *                register read or node evaluation) it is forced: bit b := v
 *                (the fault function applied at the injection node, Sec. IV-A, Table I).
 *                At the end of the combinational settle of cycle t, before the latch, the
 *                first output port o (lowest index) with net[outputs[o]] != gout[t][o]
 *                detects the fault: result (1, t, o) and the machine stops (fault
 *                dropping). After T cycles with no difference: (0, -1, -1).
 *
 * Other fault models through the same fault function (Sec. IV-A: a virtual faultyVal;
 * Sec. V-A: transient faults by overriding it):
 *   kind 2 (SEU, on a register) and kind 3 (SET, on an input or node net) flip bit b of
 *                the site in one cycle c only: a register's stored value flipped for cycle
 *                c is what its readers see in that cycle, and the latch at the end of c
 *                overwrites it, so both are "flip when t == c".
 *   port faults: site ids n_net + o name output port o, a virtual node between the
 *                port's net and the port (Sec. IV-A, Table I): the fault function applies
 *                to what port o observes, and to nothing else.
 *   no-drop mode (the paper's evaluation keeps every fault, Sec. V-A): the machine runs
 *                all T cycles; the result keeps the first detection and counts the cycles
 *                in which some port differs.
 *
 * Readings where the paper is silent (it works on Verilog through iverilog):
 *   2-valued logic (no X/Z); registers reset to 0; outputs sampled after the settle of
 *   cycle t and before the latch (a register-driven output shows Q_t); cycle index
 *   0-based; ties between ports go to the lowest port index; a stuck-at on a register
 *   forces the Q its readers see, while the register still stores its D value.
 *
 * Op semantics: operands are zero-extended to 64 bits, the op is computed in uint64 and
 * the result is masked to the node width. AND/OR/XOR bitwise; NOT ~a; ADD/SUB modulo
 * 2^64 (hence 2^w after masking); MUX2 a!=0 ? b : c; EQ a==b, LT a<b (unsigned, 1-bit);
 * SHL/SHR by the constant imm (imm >= 64 gives 0); SLICE a >> imm; CONCAT
 * (a << width(b)) | b; CONST imm.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_AND, O_OR, O_XOR, O_NOT, O_ADD, O_SUB, O_MUX2, O_EQ, O_LT, O_SHL, O_SHR,
       O_SLICE, O_CONCAT, O_CONST };

typedef struct {
    int32_t n_in, n_reg, n_node, n_out;
    const uint8_t *in_w;       /* [n_in]   */
    const uint8_t *reg_w;      /* [n_reg]  */
    const uint32_t *reg_d;     /* [n_reg]  net latched by each register */
    const uint8_t *op;         /* [n_node] */
    const uint8_t *w;          /* [n_node] */
    const uint32_t *a, *b, *c; /* [n_node] operand net ids */
    const uint64_t *imm;       /* [n_node] */
    const uint32_t *out;       /* [n_out]  net observed by each output port */
} oracle_design;

static uint64_t mask_of(unsigned w) { return w >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << w) - 1); }

static unsigned net_width(const oracle_design *d, uint32_t net)
{
    if (net < (uint32_t)d->n_in) return d->in_w[net];
    if (net < (uint32_t)(d->n_in + d->n_reg)) return d->reg_w[net - d->n_in];
    return d->w[net - d->n_in - d->n_reg];
}

/* Topological order of the nodes by Kahn's algorithm over node->node operand edges.
 * Returns 0, or -1 when the nodes form a combinational cycle. */
int oracle_topo_order(const oracle_design *d, int32_t *order)
{
    int32_t N = d->n_node, base = d->n_in + d->n_reg;
    int32_t *indeg = calloc((size_t)N + 1, sizeof(int32_t));
    int32_t *cnt = calloc((size_t)N + 1, sizeof(int32_t));
    int32_t *users = malloc(sizeof(int32_t) * (3 * (size_t)N + 1));
    int32_t *queue = malloc(sizeof(int32_t) * ((size_t)N + 1));
    int rc = 0;
    /* operands of node i that are nodes themselves */
    for (int32_t i = 0; i < N; i++) {
        uint32_t ops[3] = {d->a[i], d->b[i], d->c[i]};
        int nops = d->op[i] == O_CONST ? 0 : (d->op[i] == O_NOT || d->op[i] == O_SHL ||
                   d->op[i] == O_SHR || d->op[i] == O_SLICE) ? 1 : d->op[i] == O_MUX2 ? 3 : 2;
        for (int k = 0; k < nops; k++)
            if (ops[k] >= (uint32_t)base) { indeg[i]++; cnt[ops[k] - base]++; }
    }
    /* CSR of users */
    int32_t *start = calloc((size_t)N + 1, sizeof(int32_t));
    for (int32_t i = 0; i < N; i++) start[i + 1] = start[i] + cnt[i];
    memset(cnt, 0, sizeof(int32_t) * ((size_t)N + 1));
    for (int32_t i = 0; i < N; i++) {
        uint32_t ops[3] = {d->a[i], d->b[i], d->c[i]};
        int nops = d->op[i] == O_CONST ? 0 : (d->op[i] == O_NOT || d->op[i] == O_SHL ||
                   d->op[i] == O_SHR || d->op[i] == O_SLICE) ? 1 : d->op[i] == O_MUX2 ? 3 : 2;
        for (int k = 0; k < nops; k++)
            if (ops[k] >= (uint32_t)base) {
                int32_t p = ops[k] - base;
                users[start[p] + cnt[p]++] = i;
            }
    }
    int32_t head = 0, tail = 0, done = 0;
    for (int32_t i = 0; i < N; i++) if (indeg[i] == 0) queue[tail++] = i;
    while (head < tail) {
        int32_t n = queue[head++];
        order[done++] = n;
        for (int32_t k = start[n]; k < start[n + 1]; k++)
            if (--indeg[users[k]] == 0) queue[tail++] = users[k];
    }
    if (done != N) rc = -1;
    free(indeg); free(cnt); free(users); free(queue); free(start);
    return rc;
}

/* One node in evaluation (topological) order with its operands resolved once per call:
 * the op code, the net it drives, its operand nets (0 where the op reads fewer), its
 * constant, the mask of its width and, for CONCAT, the width of operand b. An op code
 * outside the op set gives 0. */
typedef struct {
    uint32_t op, out, a, b, c, wb;
    uint64_t imm, mask;
} oracle_step;

enum { O_NONE = 14 };

static int nops_of(unsigned op)
{
    return op == O_CONST ? 0 : (op == O_NOT || op == O_SHL || op == O_SHR || op == O_SLICE) ? 1
         : op == O_MUX2 ? 3 : op < O_NONE ? 2 : 0;
}

/* The nodes in a topological order as a list of steps. Returns a malloc'd array, or
 * NULL on a combinational cycle. */
static oracle_step *oracle_program(const oracle_design *d)
{
    int32_t N = d->n_node, base = d->n_in + d->n_reg;
    int32_t *order = malloc(sizeof(int32_t) * ((size_t)N + 1));
    if (oracle_topo_order(d, order) != 0) { free(order); return NULL; }
    oracle_step *prog = malloc(sizeof(oracle_step) * ((size_t)N + 1));
    for (int32_t k = 0; k < N; k++) {
        int32_t i = order[k];
        oracle_step *s = &prog[k];
        int nops = nops_of(d->op[i]);
        s->op = d->op[i] < O_NONE ? d->op[i] : O_NONE;
        s->out = (uint32_t)(base + i);
        s->a = nops >= 1 ? d->a[i] : 0;
        s->b = nops >= 2 ? d->b[i] : 0;
        s->c = nops >= 3 ? d->c[i] : 0;
        s->wb = s->op == O_CONCAT ? net_width(d, d->b[i]) : 0;
        s->imm = d->imm[i];
        s->mask = mask_of(d->w[i]);
    }
    free(order);
    return prog;
}

/* Evaluate one node from the current net values. Every op's value is computed and the
 * node's op code picks its own: a table instead of a branch per op, because the ops of
 * consecutive nodes are unrelated and a branch on them is mispredicted on most nodes. */
static uint64_t eval_step(const oracle_step *s, const uint64_t *net)
{
    uint64_t a = net[s->a], b = net[s->b], c = net[s->c], k = s->imm, r[O_NONE + 1];
    r[O_AND]    = a & b;
    r[O_OR]     = a | b;
    r[O_XOR]    = a ^ b;
    r[O_NOT]    = ~a;
    r[O_ADD]    = a + b;
    r[O_SUB]    = a - b;
    r[O_MUX2]   = (a != 0) ? b : c;
    r[O_EQ]     = (a == b) ? 1 : 0;
    r[O_LT]     = (a < b) ? 1 : 0;
    r[O_SHL]    = k >= 64 ? 0 : (a << k);
    r[O_SHR]    = k >= 64 ? 0 : (a >> k);
    r[O_SLICE]  = k >= 64 ? 0 : (a >> k);
    r[O_CONCAT] = (s->wb >= 64 ? 0 : (a << s->wb)) | b;
    r[O_CONST]  = k;
    r[O_NONE]   = 0;
    return r[s->op] & s->mask;
}

/* One machine over T cycles. With fault_net < 0 this is the good machine: it fills
 * gout[T][n_out]. Otherwise it compares against gout and returns the first detection
 * through *cycle and *port (both -1 if never detected) and the number of cycles with a
 * differing port through *mism. */
static void run_machine(const oracle_design *d, const oracle_step *prog, int32_t T,
                        const uint64_t *stim, uint64_t *gout_w, const uint64_t *gout_r,
                        uint64_t *trace_w,
                        int64_t fault_net, unsigned fault_bit, unsigned fault_val,
                        int64_t fault_cycle, int no_drop,
                        uint64_t *net, uint64_t *Q, int32_t *cycle, int32_t *port,
                        uint32_t *mism)
{
    int32_t I = d->n_in, R = d->n_reg, N = d->n_node, O = d->n_out;
    int64_t fault_port = fault_net - (int64_t)(I + R + N);   /* >= 0: a port fault */
    uint64_t m1 = 0, m0 = 0, mx = 0, fx;
    if (fault_net >= 0) {
        if (fault_val >= 2) mx = (uint64_t)1 << fault_bit;   /* SEU / SET: a flip */
        else if (fault_val) m1 = (uint64_t)1 << fault_bit;
        else           m0 = (uint64_t)1 << fault_bit;
    }
#define FAULTY(x) ((((x) & ~m0) | m1) ^ fx)
#define FORCE(netid) do { if ((int64_t)(netid) == fault_net) \
                              net[netid] = FAULTY(net[netid]); } while (0)
    for (int32_t r = 0; r < R; r++) Q[r] = 0;
    *cycle = -1; *port = -1; *mism = 0;
    for (int32_t t = 0; t < T; t++) {
        fx = (int64_t)t == fault_cycle ? mx : 0;   /* the flip acts in its own cycle only */
        for (int32_t i = 0; i < I; i++) {
            net[i] = stim[(size_t)t * I + i] & mask_of(d->in_w[i]);
            FORCE(i);
        }
        for (int32_t r = 0; r < R; r++) {
            net[I + r] = Q[r];
            FORCE(I + r);
        }
        for (int32_t k = 0; k < N; k++) {
            const oracle_step *st = &prog[k];
            net[st->out] = eval_step(st, net);
            FORCE(st->out);
        }
        if (trace_w) memcpy(trace_w + (size_t)t * (I + R + N), net, sizeof(uint64_t) * (I + R + N));
        if (fault_net < 0) {
            for (int32_t o = 0; o < O; o++) gout_w[(size_t)t * O + o] = net[d->out[o]];
        } else {
            int differs = 0;
            for (int32_t o = 0; o < O; o++) {
                uint64_t seen = net[d->out[o]];
                if ((int64_t)o == fault_port) seen = FAULTY(seen);   /* the port's virtual node */
                if (seen != gout_r[(size_t)t * O + o]) {
                    if (*cycle < 0) { *cycle = t; *port = o; }
                    differs = 1;
                    break;
                }
            }
            if (differs) {
                ++*mism;
                if (!no_drop) return;
            }
        }
        for (int32_t r = 0; r < R; r++) Q[r] = net[d->reg_d[r]] & mask_of(d->reg_w[r]);
    }
#undef FORCE
#undef FAULTY
}

static size_t n_nets(const oracle_design *d) { return (size_t)d->n_in + d->n_reg + d->n_node; }

/* Good machine: gout[T][n_out] and, when trace is non-null, every net's value in every
 * cycle, trace[T][n_in + n_reg + n_node]. Returns 0, or -1 on a combinational cycle. */
int oracle_good_run(const oracle_design *d, int32_t T, const uint64_t *stim, uint64_t *gout,
                    uint64_t *trace)
{
    oracle_step *prog = oracle_program(d);
    if (!prog) return -1;
    uint64_t *net = malloc(sizeof(uint64_t) * (n_nets(d) + 1));
    uint64_t *Q = malloc(sizeof(uint64_t) * ((size_t)d->n_reg + 1));
    int32_t cy, po;
    uint32_t mi;
    run_machine(d, prog, T, stim, gout, NULL, trace, -1, 0, 0, -1, 0, net, Q, &cy, &po, &mi);
    free(prog); free(net); free(Q);
    return 0;
}

/* Faulty machines, one after another, each compared against gout (from
 * oracle_good_run). Writes detected/cycle/port per fault. Returns 0 or -1. */
int oracle_fault_sim(const oracle_design *d, int32_t T, const uint64_t *stim,
                     const uint64_t *gout, int32_t F, const uint32_t *fnet,
                     const uint8_t *fbit, const uint8_t *fval,
                     uint8_t *detected, int32_t *cycle, int32_t *port)
{
    oracle_step *prog = oracle_program(d);
    if (!prog) return -1;
    uint64_t *net = malloc(sizeof(uint64_t) * (n_nets(d) + 1));
    uint64_t *Q = malloc(sizeof(uint64_t) * ((size_t)d->n_reg + 1));
    uint32_t mi;
    for (int32_t f = 0; f < F; f++) {
        run_machine(d, prog, T, stim, NULL, gout, NULL, (int64_t)fnet[f], fbit[f], fval[f],
                    -1, 0, net, Q, &cycle[f], &port[f], &mi);
        detected[f] = cycle[f] >= 0 ? 1 : 0;
    }
    free(prog); free(net); free(Q);
    return 0;
}

/* The same with a fault kind per fault (0 SA0, 1 SA1, 2 SEU, 3 SET; fcycle = the cycle
 * of a flip), port faults (site n_net + o) and the no-drop mode; mism[f] = cycles in
 * which some port differs (with dropping: 1 for a detected fault). Returns 0 or -1. */
int oracle_fault_sim_ex(const oracle_design *d, int32_t T, const uint64_t *stim,
                        const uint64_t *gout, int32_t F, const uint32_t *fnet,
                        const uint8_t *fbit, const uint8_t *fkind, const uint32_t *fcycle,
                        int32_t no_drop, uint8_t *detected, int32_t *cycle, int32_t *port,
                        uint32_t *mism)
{
    oracle_step *prog = oracle_program(d);
    if (!prog) return -1;
    uint64_t *net = malloc(sizeof(uint64_t) * (n_nets(d) + 1));
    uint64_t *Q = malloc(sizeof(uint64_t) * ((size_t)d->n_reg + 1));
    for (int32_t f = 0; f < F; f++) {
        int64_t fc = fkind[f] >= 2 ? (int64_t)fcycle[f] : -1;
        run_machine(d, prog, T, stim, NULL, gout, NULL, (int64_t)fnet[f], fbit[f], fkind[f],
                    fc, no_drop, net, Q, &cycle[f], &port[f], &mism[f]);
        detected[f] = cycle[f] >= 0 ? 1 : 0;
    }
    free(prog); free(net); free(Q);
    return 0;
}
