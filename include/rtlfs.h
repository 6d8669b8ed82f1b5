/*
 * rtlfs.h -- C ABI of librtlfs, a GB300 (sm_103a) cycle-based RTL stuck-at fault
 * simulator: the data-parallel hot path of RIROS (arXiv 2508.16376).
 *
 * Problem (Sec. II-B, "RTL Fault Simulation"): a design compiled into a graph of RTL
 * nodes (variables and word-level operators) and registers is simulated cycle by cycle
 * under a stimulus; registers take their next values at the end of every cycle (global
 * synchronization, the non-blocking-assignment latch). A stuck-at-0/1 fault forces one
 * bit of a wire, register or port (fault injection at the RTL node that produces the
 * value, Sec. IV-A / Table I); the fault is detected when a faulty output value differs
 * from the good one. The library returns, per fault, whether and when it is first
 * detected and on which output port; a detected fault is dropped from further cycles.
 *
 * Conventions shared by every call:
 *  - Every call returns an int status (RTLFS_OK or a negative RTLFS_E_* code); nothing
 *    throws or aborts across the ABI. rtlfs_last_error() gives a one-line reason.
 *  - Input arrays are host pointers, read during the call and copied (to device memory
 *    where needed); the caller keeps ownership and may free them on return.
 *  - Outputs are written into caller-allocated host buffers of the stated size.
 *  - A failed call leaves the context's previous state unchanged, except RTLFS_E_CUDA,
 *    after which the context should be destroyed.
 *  - One context per host thread; a context owns all of its device memory and streams.
 *  - Net id space of a design: [0, I) primary inputs, [I, I+R) register Q outputs,
 *    [I+R, I+R+N) node outputs (node i drives net I+R+i). Values are unsigned words of
 *    width 1..64 bits, held zero-extended in uint64; logic is 2-valued.
 */
#ifndef RTLFS_H
#define RTLFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define RTLFS_OK          0
#define RTLFS_E_ARG      -1   /* malformed argument: null pointer, id or size out of range */
#define RTLFS_E_CYCLE    -2   /* the nodes form a combinational cycle */
#define RTLFS_E_WIDTH    -3   /* a width is outside 1..64 or breaks an op's width rule */
#define RTLFS_E_NOMEM    -4   /* device or host allocation failed */
#define RTLFS_E_CUDA     -5   /* a CUDA call failed (destroy the context) */
#define RTLFS_E_TIMEOUT  -6   /* a per-fault work budget ran out (results flagged) */
#define RTLFS_E_STATE    -7   /* call out of order (e.g. run before stimulus/faults) */

/* ---- word-level ops ------------------------------------------------------------------
 * Operands are zero-extended to 64 bits, the op is computed in uint64 and the result is
 * masked to the node width w. a, b, c are operand net ids; imm is a constant.
 *   AND/OR/XOR  a op b            NOT   ~a
 *   ADD/SUB     a +/- b mod 2^w   MUX2  a != 0 ? b : c
 *   EQ/LT       a == b, a < b (unsigned); w must be 1
 *   SHL/SHR     a << imm, a >> imm (imm >= 64 gives 0)
 *   SLICE       a >> imm; requires imm + w <= width(a)
 *   CONCAT      (a << width(b)) | b; requires w == width(a) + width(b) <= 64
 *   CONST       imm (no operands)
 * These stand for the RTL operator nodes of the paper's graph (Sec. II-B, Fig. 2); the
 * paper's behavioral (VVP) nodes have no counterpart here. */
enum rtlfs_op {
    RTLFS_AND = 0, RTLFS_OR = 1, RTLFS_XOR = 2, RTLFS_NOT = 3, RTLFS_ADD = 4,
    RTLFS_SUB = 5, RTLFS_MUX2 = 6, RTLFS_EQ = 7, RTLFS_LT = 8, RTLFS_SHL = 9,
    RTLFS_SHR = 10, RTLFS_SLICE = 11, RTLFS_CONCAT = 12, RTLFS_CONST = 13
};

/* One operator node (24 bytes). Unused operand fields are ignored. */
typedef struct {
    uint8_t  op;        /* enum rtlfs_op */
    uint8_t  width;     /* result width, 1..64 */
    uint16_t reserved;  /* must be 0 */
    uint32_t a, b, c;   /* operand net ids */
    uint64_t imm;       /* shift amount, slice offset or constant */
} rtlfs_node;

/* One register (8 bytes): reset value 0; at the end of every cycle Q <- D masked to
 * width (the global synchronization of Sec. II-B). d_net may be any net. */
typedef struct {
    uint32_t d_net;
    uint8_t  width;     /* 1..64 */
    uint8_t  reserved[3];
} rtlfs_reg;

/* One stuck-at fault (8 bytes): bit `bit` of net `net` forced to `stuck` (0 or 1) every
 * time the net's value is produced -- input read, register read, node evaluation
 * (unified fault injection at the producing node, Sec. IV-A). A register fault forces
 * the Q its readers see; the register still stores its D value.
 * Port faults (Sec. IV-A, Table I: a port fault is injected into a virtual node inserted
 * for the port): net ids n_net + o, o < n_outputs, denote output port o -- a virtual node
 * between the port's net and the port, so the fault changes what port o observes and
 * nothing else (the net's other readers see its true value). An input port is its own
 * net (ids below n_inputs): a fault there reaches every reader of the input. */
typedef struct {
    uint32_t net;
    uint8_t  bit;       /* < width(net) */
    uint8_t  stuck;     /* 0 = stuck-at-0, 1 = stuck-at-1 */
    uint16_t reserved;
} rtlfs_fault;

/* Fault kinds of rtlfs_fault_ex (the fault function of Sec. IV-A, chosen per fault;
 * transient models, Sec. V-A). A flip inverts bit `bit` during cycle `cycle` only:
 *   SEU -- single-event upset of a register: the stored value of a register net has the
 *          bit flipped for cycle `cycle`; the latch at the end of that cycle overwrites it,
 *          so in a cycle-based model it acts as a one-cycle flip of the Q its readers see;
 *   SET -- single-event transient on a combinational net (an input, a node or an output
 *          port): the net's value is flipped during cycle `cycle`.
 * A flip always makes the site differ in its cycle; before it the machines are equal. */
#define RTLFS_FAULT_SA0  0
#define RTLFS_FAULT_SA1  1
#define RTLFS_FAULT_SEU  2   /* net must be a register (n_inputs <= net < n_inputs + n_regs) */
#define RTLFS_FAULT_SET  3   /* net must be an input, a node or an output port */

typedef struct {
    uint32_t net;       /* as in rtlfs_fault, port ids included */
    uint8_t  bit;       /* < width(net) */
    uint8_t  kind;      /* RTLFS_FAULT_* */
    uint16_t reserved;
    uint32_t cycle;     /* cycle of an SEU/SET (any value; >= n_cycles never acts) */
    uint32_t reserved2;
} rtlfs_fault_ex;

/* Per-fault result (12 bytes). Outputs are compared after the combinational settle of
 * cycle `cycle` (0-based), before the latch; `port` is the lowest differing output
 * index. Undetected: detected = 0, cycle = port = -1. detected = 255 marks a fault
 * whose work budget ran out (the run returns RTLFS_E_TIMEOUT). */
typedef struct {
    int32_t cycle;
    int32_t port;
    uint8_t detected;
    uint8_t reserved[3];
} rtlfs_result;

/* ---- run options ---------------------------------------------------------------------- */
#define RTLFS_SCHED_PLAIN      0   /* queue in fault-list order, no heavy pre-assignment */
#define RTLFS_SCHED_HEURISTIC  1   /* order by static cone size x toggle rate */
#define RTLFS_SCHED_MLP        2   /* order by the load predictor (falls back to heuristic
                                      when no weights are loaded) */

typedef struct {
    int32_t  scheduler;      /* RTLFS_SCHED_*; default HEURISTIC */
    int32_t  light_block;    /* threads per CTA of the light kernel (32..1024); 0 = auto */
    int32_t  heavy_block;    /* threads per CTA of the heavy kernel (32..1024); 0 = auto */
    int32_t  heavy_ctas;     /* resident heavy CTAs (scratch slots); 0 = auto */
    float    heavy_frac;     /* fraction of faults (highest predicted load) sent to the
                                heavy kernel from cycle 0; < 0 = auto */
    int32_t  use_graph;      /* 1 = capture the launch sequence in a CUDA graph and replay */
    uint64_t fault_budget;   /* max node evaluations per fault, 0 = unlimited */
    int32_t  light_cap;      /* light-lane capacity variant: 1 = 4 register diffs / 12 net
                                diffs / 12 pending nodes, 2 = 8/24/24, 3 = 8/48/48; 0 = auto */
    int32_t  window;         /* cycles per window: every live fault advances through the same
                                window of cycles, the good trace of the next window, the light
                                kernel and the heavy kernel overlap on three streams; 0 = each
                                fault runs its whole timeline in one light/heavy pass */
    int32_t  no_drop;        /* 1 = keep simulating a detected fault to the last cycle (the
                                paper's evaluation protocol, Sec. V-A): the result keeps the
                                first detection and rtlfs_mismatch_counts gives each fault's
                                number of cycles with a differing output */
    int32_t  stop_cycle;     /* windowed form, > 0: stop the campaign at this cycle (a multiple
                                of `window`, below the longest stimulus) and keep its state for
                                rtlfs_checkpoint_save; faults still being simulated report
                                detected = RTLFS_PENDING */
    int32_t  resume;         /* 1: continue the campaign from the checkpoint held by the context
                                (made by a stopped run or rtlfs_checkpoint_load); the other
                                options must match the stopped run's window, no_drop and
                                light_cap (RTLFS_E_ARG otherwise) */
    int32_t  heavy_form;     /* heavy kernel's record of differing nets: 0 = auto (the
                                exact one unless it costs resident CTAs), 1 = a shared-memory
                                bit per net, 2 = a small shared filter plus cycle stamps on
                                the values in global scratch (for designs whose per-net
                                bitmap would crowd shared memory), 3 = as 2 with the
                                per-node bitmap in global scratch too and a one-bit-per-word
                                summary in shared memory (for designs whose node bitmap
                                would crowd it; heavy_block 32 only) */
    int32_t  good_cluster;   /* good-trace form: 0 = auto (one CTA with the net values in
                                shared memory when the design fits, else the smallest
                                thread-block cluster whose CTAs hold them in distributed
                                shared memory, else one CTA over the global trace);
                                1 = one CTA; 2, 4, 8 or 16 = clusters of that many CTAs
                                (RTLFS_E_ARG when a design cannot run that way) */
    int32_t  good_staging;   /* one-CTA good trace: 0 = each thread prefetches its node
                                descriptors into registers two chunks ahead; 1 = a producer
                                warp stages them into a shared-memory ring with bulk
                                asynchronous copies (TMA) for the consumer threads. Same
                                results; RTLFS_E_CUDA if a staging wait runs out */
    int32_t  good_first;     /* windowed form: 1 = the good trace of every cycle (one launch
                                per design list), its transposition and the activation
                                bitplane run before the first faulty window, so the faulty
                                kernels never wait for the good trace; 0 = the good trace of
                                window w+1 overlaps the faulty kernels of window w. Ignored
                                by a run that stops at stop_cycle or resumes. Same results */
    int32_t  order_classes;  /* HEURISTIC / MLP schedule: 0 = the queue in descending score
                                order (4096 score buckets); 1, 2, 4, .. 64 = that many score
                                classes, highest first, each keeping the fault-list order (a
                                warp's light lanes then take faults of neighbouring sites);
                                RTLFS_E_ARG otherwise. Same results */
} rtlfs_run_opts;

/* Timing and counters of the last rtlfs_run (milliseconds from CUDA events). */
typedef struct {
    double   total_ms;       /* first launch to results on host */
    double   good_ms;        /* good-machine trace (all designs) */
    double   prep_ms;        /* features, predictor, queue order */
    double   faulty_ms;      /* light + heavy faulty-machine kernels */
    double   light_ms;       /* light kernel alone */
    double   heavy_ms;       /* promoted-fault heavy pass alone */
    uint64_t fault_cycles;   /* W = sum over faults of (cycle+1 if detected else T) */
    uint64_t node_evals;     /* sum of the per-fault propagation loads */
    uint64_t promoted;       /* light faults promoted to the heavy kernel */
    uint64_t heavy_initial;  /* faults assigned to the heavy kernel from cycle 0 */
    uint32_t n_launches;     /* kernels launched by the run */
    uint32_t heavy_form;     /* heavy kernel's record of differing nets in the run: 1 exact,
                                2 stamped, 3 stamped with the node bitmap in global scratch */
    uint64_t light_evals;         /* node evaluations done by the light kernel */
    uint64_t light_fault_cycles;  /* fault-cycles completed by the light kernel */
    uint64_t heavy_evals;         /* node evaluations done by the heavy kernel */
    uint64_t heavy_fault_cycles;  /* fault-cycles completed by the heavy kernel */
} rtlfs_stats;

typedef struct rtlfs_ctx rtlfs_ctx;   /* opaque */

/* Create a context on CUDA device `device`. *out receives the handle. Errors:
 * RTLFS_E_ARG (null out / bad device), RTLFS_E_CUDA. */
int rtlfs_create(rtlfs_ctx **out, int device);

/* Free every device and host resource of the context. Null is accepted. */
void rtlfs_destroy(rtlfs_ctx *ctx);

/* One-line description of the last error on this context ("" after success). */
const char *rtlfs_last_error(const rtlfs_ctx *ctx);

/* Load one design (Sec. II-B: the RTL graph; Sec. IV, Steps 1-4: compile, inject,
 * build the task graph): nodes[n_nodes], regs[n_regs], input_widths[n_inputs] (1..64),
 * output_nets[n_outputs] (port o observes net output_nets[o]). The library validates
 * ids and width rules, rejects combinational cycles (RTLFS_E_CYCLE; registers break
 * cycles), levelizes the nodes, builds fan-out and latch maps and uploads them. The new
 * design's id (0, 1, ... in load order) goes to *design_id. All designs of a context run
 * together in rtlfs_run. Errors: RTLFS_E_ARG, RTLFS_E_WIDTH, RTLFS_E_CYCLE, RTLFS_E_NOMEM. */
int rtlfs_load_design(rtlfs_ctx *ctx, const rtlfs_node *nodes, uint32_t n_nodes,
                      const rtlfs_reg *regs, uint32_t n_regs,
                      const uint8_t *input_widths, uint32_t n_inputs,
                      const uint32_t *output_nets, uint32_t n_outputs,
                      uint32_t *design_id);

/* Stimulus of a design: inputs[n_cycles][n_inputs] row-major; each value is masked to
 * its input's width on use. 1 <= n_cycles <= 2^21. Replaces an earlier stimulus. Errors:
 * RTLFS_E_ARG, RTLFS_E_NOMEM. */
int rtlfs_set_stimulus(rtlfs_ctx *ctx, uint32_t design_id, const uint64_t *inputs,
                       uint32_t n_cycles);

/* Fault list of a design: faults[n_faults] (n_faults may be 0). Each fault's bit must
 * be below its net's width (RTLFS_E_ARG otherwise). Duplicates are simulated
 * independently. Replaces an earlier list. Errors: RTLFS_E_ARG, RTLFS_E_NOMEM. */
int rtlfs_set_faults(rtlfs_ctx *ctx, uint32_t design_id, const rtlfs_fault *faults,
                     uint32_t n_faults);

/* Fault list of a design with per-fault kinds: stuck-at, SEU and SET faults (see
 * rtlfs_fault_ex). Validation as rtlfs_set_faults, plus: an SEU site must be a register,
 * an SET site must not be (its flip is an SEU). Replaces an earlier list. Errors:
 * RTLFS_E_ARG, RTLFS_E_NOMEM. */
int rtlfs_set_faults_ex(rtlfs_ctx *ctx, uint32_t design_id, const rtlfs_fault_ex *faults,
                        uint32_t n_faults);

/* Simulate every loaded design's fault list under its stimulus (the whole hot path: good
 * trace, load prediction and queue order, light and heavy faulty machines with output
 * compare, fault dropping and register latch). out_per_design[d] is a caller buffer of
 * n_faults(d) results in the design's fault-list order; out_load_per_design may be null
 * or hold per-design buffers (entries may be null) of n_faults(d) uint64 propagation
 * loads (node evaluations summed over the cycles the fault was simulated). opts may be
 * null (defaults). Results never depend on the options. Errors: RTLFS_E_STATE (a design
 * without stimulus), RTLFS_E_ARG, RTLFS_E_CUDA, RTLFS_E_TIMEOUT (fault_budget ran out;
 * the affected results carry detected = 255, the others are valid). */
int rtlfs_run(rtlfs_ctx *ctx, const rtlfs_run_opts *opts,
              rtlfs_result *const *out_per_design, uint64_t *const *out_load_per_design);

/* The plain GPU form: one thread per fault, one flat launch per design, no queue, no
 * heavy path, no prediction; same result contract as rtlfs_run. */
int rtlfs_run_plain(rtlfs_ctx *ctx, rtlfs_result *const *out_per_design);

/* Counters and timings of the last rtlfs_run / rtlfs_run_plain. */
int rtlfs_get_stats(const rtlfs_ctx *ctx, rtlfs_stats *out);

/* Checkpoint and resume at a window boundary (no counterpart in the paper, which runs a
 * campaign in one go). A run with stop_cycle = c leaves in the context everything the rest of
 * the campaign needs: each fault's result so far, load and mismatch count, the register
 * diffs of the faults still alive (light lanes and heavy CTAs alike), the campaign counters
 * and each design's good-trace row at cycle c-1 (the good machine restarts from it). These
 * calls move that state through a caller-owned buffer, e.g. to disk and into another
 * process. A resumed campaign reaches the same results, loads and mismatch counts as an
 * uninterrupted one.
 *   rtlfs_checkpoint_size: bytes the current checkpoint takes (RTLFS_E_STATE: none held).
 *   rtlfs_checkpoint_save: write it into buf[bytes] (RTLFS_E_ARG if bytes is too small).
 *   rtlfs_checkpoint_load: take a checkpoint into a context holding the same designs,
 *     stimuli and fault lists (RTLFS_E_ARG on a malformed buffer or a mismatch, including
 *     register-diff counts or register ids outside the bounds the kernels use); the next
 *     rtlfs_run with resume = 1 continues from it. */
#define RTLFS_PENDING 254   /* rtlfs_result.detected of a fault still alive at stop_cycle */
int rtlfs_checkpoint_size(rtlfs_ctx *ctx, uint64_t *bytes);
int rtlfs_checkpoint_save(rtlfs_ctx *ctx, void *buf, uint64_t bytes);
int rtlfs_checkpoint_load(rtlfs_ctx *ctx, const void *buf, uint64_t bytes);

/* After an rtlfs_run with no_drop = 1: for each fault of the design (in list order), the
 * number of cycles in which some output port differs from the good machine (n-detection
 * count; 0 = undetected). out[n_faults], caller-owned. RTLFS_E_STATE when the last run
 * dropped faults or the fault list changed since. */
int rtlfs_mismatch_counts(rtlfs_ctx *ctx, uint32_t design_id, uint32_t *out);

/* Test hooks: the good machine's outputs out[n_cycles][n_outputs], or every net's value
 * out[n_cycles][n_nets] in the caller's net numbering, as computed by the last run (or
 * by a good-trace-only run if none happened since the stimulus was set). */
int rtlfs_good_outputs(rtlfs_ctx *ctx, uint32_t design_id, uint64_t *out);
int rtlfs_good_trace(rtlfs_ctx *ctx, uint32_t design_id, uint64_t *out);

/* Design sizes after load: n_nets, number of topological levels, total fan-out edges. */
int rtlfs_design_info(const rtlfs_ctx *ctx, uint32_t design_id, uint32_t *n_nets,
                      uint32_t *n_levels, uint32_t *n_fanout_edges);

/* ---- load predictor ---------------------------------------------------------------------
 * The paper balances load with a runtime monitor that marks a node heavy when its share of
 * the run time passes a threshold (Sec. IV-C-2, Sec. V-A). Here a small MLP predicts each
 * fault's propagation load (node evaluations summed over the cycles it is simulated,
 * natural log of 1 + load) before the faulty kernels start; the prediction orders the work
 * queue and picks the faults that start in the heavy kernel (RTLFS_SCHED_MLP). It never
 * changes a result.
 *
 * Features (5 floats per fault, row-major [n][5]): static fan-out cone size (log2 of the
 * reconvergence-counting cone estimate, / 20, at most 1.5), topological level of the site
 * (0 for inputs/registers, else (level+1)/n_levels), register depth from the site to the
 * nearest output (min(depth,16)/16; 1 if no output is reachable), width of the site net
 * / 64, and the good-trace toggle rate of the site bit over the first P = min(T, 256)
 * cycles (changes between consecutive cycles / (P-1); 0 when P = 1). The prefix is the
 * same in every form of the campaign, so a windowed campaign orders its first window with
 * the features the predictor was trained on.
 *
 * Network: 5 -> 64 (ReLU) -> 64 (ReLU) -> 1, RTLFS_MLP_PARAMS parameters laid out as
 * W1[5][64], b1[64], W2[64][64], b2[64], w3[64], b3 (W[i][j] connects unit i of one layer
 * to unit j of the next). Parameters are BF16 (raw uint16 bit patterns); arithmetic
 * accumulates in FP32 on the CUDA cores. */
#define RTLFS_MLP_PARAMS 4609

/* Features of every fault of design_id into out[n_faults][5] (runs the good trace first if
 * needed). Errors: RTLFS_E_ARG, RTLFS_E_STATE, RTLFS_E_CUDA. */
int rtlfs_features(rtlfs_ctx *ctx, uint32_t design_id, float *out);

/* Load parameters w[RTLFS_MLP_PARAMS] (BF16 bit patterns); resets the optimizer state. */
int rtlfs_mlp_set_weights(rtlfs_ctx *ctx, const uint16_t *w);

/* Current parameters (BF16 bit patterns) into w[RTLFS_MLP_PARAMS]. RTLFS_E_STATE if none. */
int rtlfs_mlp_get_weights(rtlfs_ctx *ctx, uint16_t *w);

/* Predictions y[n] for features X[n][5]. RTLFS_E_STATE if no weights are loaded. */
int rtlfs_mlp_forward(rtlfs_ctx *ctx, const float *X, uint32_t n, float *y);

/* Mean squared error over n samples (*loss) and its gradient grad[RTLFS_MLP_PARAMS]
 * (FP32) with respect to every parameter, at the current BF16 parameters. */
int rtlfs_mlp_grad(rtlfs_ctx *ctx, const float *X, const float *t, uint32_t n, float *loss,
                   float *grad);

/* Adam training (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on n samples in the
 * given order, `batch` samples per step, for `epochs` passes; FP32 master parameters,
 * BF16 copies used by the forward pass. *final_loss (may be null) = mean squared error
 * accumulated over the last pass. */
int rtlfs_mlp_train(rtlfs_ctx *ctx, const float *X, const float *t, uint32_t n, uint32_t epochs,
                    uint32_t batch, float lr, float *final_loss);

/* ---- allocation-free fault simulation -------------------------------------------------
 * The paper has no counterpart to this call. It is for callers that cannot obtain device
 * memory from cudaMalloc at the point where they simulate: a host process whose device
 * memory is owned by another allocator (a framework's caching pool that has reserved the
 * GPU's memory, which this library cannot call into), and latency-critical paths where
 * the cost of an allocation, and the device-wide synchronisation cudaMalloc and cudaFree
 * can imply, are not acceptable. The call allocates nothing: no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * It simulates faults[n_faults] (device memory, rtlfs_fault records in the caller's net
 * numbering) of design design_id against that design's good trace, one thread per fault
 * (the plain GPU form), and writes results[n_faults] (device memory, rtlfs_result records)
 * with the same contract as rtlfs_run. Supported: stuck-at faults on input, register and
 * node nets. Output-port ids (n_net + o) are not supported by this call: such a fault gets
 * detected = 254 and the call returns RTLFS_E_ARG (rtlfs_run simulates them). The context
 * must already hold the design's current good trace (from rtlfs_run or rtlfs_good_outputs
 * after the last rtlfs_set_stimulus): RTLFS_E_STATE otherwise.
 *
 * Scratch: a file-scope device array of RTLFS_STATIC_SCRATCH_BYTES (64 MiB) inside the
 * library, held by every GPU that loads the library until the process exits. A design
 * needs 4 B per net once plus 12 B per net + 8 B per node + 24 B per register for every
 * simultaneously simulated fault (faults run in waves that fit); a design whose single
 * fault does not fit is rejected with RTLFS_E_ARG. Every call shares the array and leaves
 * its contents behind; the call clears what must start at zero. Calls whose work overlaps
 * on the GPU (other threads, other streams) race on the array: serialise them.
 *
 * What a call does: it copies the design's net-number map (4 B per net) from host memory
 * into the array, clears the wave's scratch, launches the kernel once per wave on `stream`
 * (a cudaStream_t; null = the legacy default stream), copies a 4-byte error word back to
 * the host and waits for `stream` before it returns. The first call on a device also looks
 * up the array's device address (cudaGetSymbolAddress) and keeps it; make that first call
 * before any stream capture. Returns RTLFS_E_ARG if a fault's net, bit or stuck value is
 * out of range (that fault's result carries detected = 254). */
int rtlfs_fault_sim_static(rtlfs_ctx *ctx, uint32_t design_id, const rtlfs_fault *faults,
                           uint32_t n_faults, rtlfs_result *results, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RTLFS_H */
