// rtlfs_internal.h -- device-side layouts shared by the host code and the kernels.
//
// Internal net numbering of a loaded design: [0, I) inputs, [I, I+R) register Qs,
// [I+R, I+R+N) nodes sorted by topological level (stable within a level), so that
// every operand of a node has a smaller id and each level is one contiguous id range.
// The caller's numbering is mapped at load time and restored on output.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rtlfs {

enum : uint32_t {
    OP_AND = 0, OP_OR, OP_XOR, OP_NOT, OP_ADD, OP_SUB, OP_MUX2, OP_EQ, OP_LT, OP_SHL,
    OP_SHR, OP_SLICE, OP_CONCAT, OP_CONST
};

constexpr uint32_t NO_PORT = 0xFFFFFFFFu;

// Threads of the good-trace CTA = maximum nodes per good-trace chunk.
constexpr uint32_t GOOD_BLOCK = 512;

// Node descriptor, 16 bytes: x/y/z = operand net ids (CONST: y:x = value), w = meta.
// meta bits: [0,4) op, [8,15) width 1..64, [16,24) k = shift amount, slice offset or
// width(b) for CONCAT, clamped to 64.
__host__ __device__ inline uint32_t meta_op(uint32_t m) { return m & 15u; }
__host__ __device__ inline uint32_t meta_w(uint32_t m) { return (m >> 8) & 127u; }
__host__ __device__ inline uint32_t meta_k(uint32_t m) { return (m >> 16) & 255u; }
__host__ __device__ inline uint32_t make_meta(uint32_t op, uint32_t w, uint32_t k) {
    return (op & 15u) | ((w & 127u) << 8) | ((k > 64u ? 64u : k) << 16);
}

// Per-net record, 16 bytes: x = first fan-out entry, y = end of fan-out entries,
// z = first latch entry (dreg_idx), w = (latch count, 255 = read dreg_off) << 24 | port,
// port = lowest output port observing the net (0xFFFFFF = none).
constexpr uint32_t NI_NO_PORT = 0xFFFFFFu;
__host__ __device__ inline uint32_t ni_port(uint32_t w) { return w & 0xFFFFFFu; }
__host__ __device__ inline uint32_t ni_nreg(uint32_t w) { return w >> 24; }

struct DevDesign {
    uint32_t I, R, N, O, n_net, n_levels, T, n_fo;
    uint32_t n_chunks;          // good-trace chunks (<= GOOD_BLOCK nodes each, never across levels)
    const uint4    *netinfo;    // [n_net]
    const uint2    *chunks;     // [n_chunks] {first node, end node | 1<<31 if last of its level}
    const uint4    *desc;       // [N]
    const uint32_t *lvl_start;  // [n_levels + 1] node-index range of each level
    const uint16_t *node_level; // [N]
    const uint8_t  *net_w;      // [n_net]
    const uint32_t *fo_off;     // [n_net + 1] fan-out CSR: consumer node indices
    const uint32_t *fo_idx;     // [n_fo]
    const uint16_t *fo_lvl;     // [n_fo] level of each consumer
    const uint32_t *dreg_off;   // [n_net + 1] registers latching each net
    const uint32_t *dreg_idx;   // [n_dreg]
    const uint32_t *dreg_rec;   // [n_dreg] register index | register width << 25
    const uint32_t *reg_d;      // [R] internal id of each register's D net
    const uint32_t *outport;    // [n_net] lowest output port observing the net, or NO_PORT
    const uint32_t *out_net;    // [O] internal id observed by each port
    const uint64_t *stim;       // [T][I]
    uint64_t *rows;             // [T][n_net] good trace, one row per cycle
    uint64_t *gcol;             // [n_net][T] good trace, one column per net
    // Cluster good trace (designs too large for one CTA's shared memory): the layout of
    // one CTA's value area and each CTA's descriptor, chunk and register lists.
    uint32_t cl_own;            // node values per CTA (words)
    uint32_t cl_rown;           // registers per CTA (words per bank)
    const uint4    *cl_desc;    // [C][cl_own] descriptors, operands as cluster locations
    const uint4    *cl_chunk;   // chunk lists {first slot, count | 1<<31 at a level's end, first node, 0}
    const uint32_t *cl_ch_off;  // [C + 1] chunk list of each CTA
    const uint4    *cl_reg;     // {register, D location, width, D net} by home CTA
    const uint32_t *cl_reg_off; // [C + 1] registers of each CTA (a contiguous index range)
};

// A net's location for the cluster good trace, 32 bits: the word in the holding CTA's
// value area (node values [0, own), register banks [own, own + 2 rown), inputs after
// them), the holder's rank in the cluster, and two flags: a register (add the bank of
// the cycle's parity) and an input (every CTA holds a copy: read the local one).
constexpr uint32_t CL_WORD = 0x00FFFFFFu;
constexpr uint32_t CL_RANK_SHIFT = 24;
constexpr uint32_t CL_REG = 1u << 28;
constexpr uint32_t CL_SELF = 1u << 29;
constexpr uint32_t CL_MAX = 16;   // largest cluster (non-portable size on sm_103a)

// All faults of all designs, concatenated in design order.
// Fault kinds (DevFaults.val): stuck-at 0, stuck-at 1, and a flip of the bit during one
// cycle (t0): a single-event upset on a register, a single-event transient on a net.
constexpr uint32_t FK_SA0 = 0, FK_SA1 = 1, FK_FLIP = 2;

struct DevFaults {
    uint32_t F;
    const uint32_t *site;       // internal net id (a port fault: the port's driver net)
    const uint8_t  *bit;
    const uint8_t  *val;        // kind: FK_SA0, FK_SA1, FK_FLIP
    const uint32_t *port;       // output port of a port fault, NO_PORT for a net fault
    const uint32_t *t0;         // cycle of an FK_FLIP fault
    uint32_t *mism;             // no-drop mode: cycles with a differing output per fault;
                                // null = drop each fault at its first detection
    const uint16_t *design;     // design index of each fault
    int32_t  *res_cycle;
    int32_t  *res_port;
    uint8_t  *res_det;
    uint64_t *load;             // node evaluations, summed over simulated cycles
    // Activation bitplane (optional, null = scan the good trace): bit (t mod 64) of
    // act[fault * act_stride + t / 64] is set when the site bit's good value at cycle t
    // differs from the stuck value, i.e. when the fault makes the machines differ by itself.
    const uint64_t *act;
    uint32_t act_stride;
};

// Light-lane capacities (per fault, per cycle): register diffs, net diffs, pending nodes.
// Three compiled variants, chosen per run (rtlfs_run_opts.light_cap 1..3).
constexpr int LIGHT_KR = 8;    // upper bound of every variant's register-diff capacity
constexpr int LIGHT_CAPS[3][3] = {{4, 12, 12}, {8, 24, 24}, {8, 48, 48}};

// A fault handed from the light kernel (or the scheduler) to the heavy kernel: resume at
// cycle t with `nreg` register diffs (reg index, faulty Q value).
struct HeavyItem {
    uint32_t fault;
    uint32_t t;
    uint32_t nreg;
    uint32_t reg_r[LIGHT_KR];
    uint64_t reg_v[LIGHT_KR];
};

struct Queues {
    const uint32_t *light_order;   // [n_light] global fault ids, in schedule order
    uint32_t n_light;
    unsigned long long *light_head;
    HeavyItem *heavy_items;        // [cap]
    uint32_t  *heavy_count;        // device counter of heavy items
    unsigned long long *heavy_head;
    uint32_t heavy_cap;
    unsigned long long *budget_hit; // faults whose work budget ran out
    uint64_t fault_budget;
    unsigned long long *counters;   // [0] node evaluations, [1] fault-cycles simulated
};

// Exact form of the heavy kernel: words of its net bitmap remembered for clearing; beyond
// this many the whole bitmap is cleared at the end of the cycle.
constexpr uint32_t HEAVY_DLIST = 128;
// Dirty nodes of one level a heavy CTA gathers into a list and splits over its threads;
// a level with more is walked word by word.
constexpr uint32_t HEAVY_NLIST = 256;
// Fan-out ranges a heavy CTA collects per level before marking consumers together; a
// range beyond this many is marked by the thread that kept the net.
constexpr uint32_t HEAVY_FRANGE = 64;
// Fan-out lists up to this long are marked by the thread that kept the net.
constexpr uint32_t HEAVY_INLINE_FANOUT = 16;

// Per-slot scratch of the heavy kernel (one slot per resident CTA).
// A heavy slot's faulty value of a net, valid in the cycle whose stamp it carries (a
// slot's stamps only grow, so nothing is cleared between cycles or faults).
struct __align__(16) HeavyVal {
    uint64_t v;
    uint32_t stamp;
    uint32_t pad;
};

struct HeavyScratch {
    HeavyVal *fval;      // [slots][max_net] faulty values of the nets that differ
    uint32_t *stamp;     // [slots] last stamp each slot used
    uint32_t *reg_r;     // [slots][2][max_reg]
    uint64_t *reg_v;     // [slots][2][max_reg]
    uint32_t *gbm;       // global-bitmap form: [slots][(max_node + 31) / 32] node bitmaps (zeroed)
    uint32_t max_net, max_reg, max_node, max_levels;
    // 1: the exact form -- a shared-memory bit per net marks the faulty values (8-byte values
    // at the start of each slot's array); 0: the stamped form (a small shared filter and
    // per-entry cycle stamps), chosen when the bitmap would cost resident CTAs
    uint32_t exact;
};

// ---- windowed campaign (cycles processed in windows [t0, t1) by every live fault) ------
// A heavy fault that reaches the end of a window carries its register diffs to the next
// window through a pool: pool_r/pool_v[off .. off+nreg).
struct HeavyCarry {
    uint32_t fault;
    uint32_t nreg;
    uint64_t off;
};

struct WinLight {
    const uint32_t *live_in;      // fault ids alive at t0
    uint32_t reverse;             // 1: take live_in back to front (survivor lists)
    const uint32_t *n_live_in;    // device count of live_in
    uint32_t *live_out;           // survivors at t1 (appended, order unspecified)
    uint32_t *n_live_out;
    unsigned long long *head;     // queue position in live_in (zero at run start)
    HeavyItem *prom;              // promotions: appended at *prom_total
    uint32_t *prom_total;
    uint32_t prom_cap;
    uint8_t *st_nreg;             // [F] register diffs carried between windows
    uint32_t *st_r;               // [LIGHT_KR][F]
    uint64_t *st_v;               // [LIGHT_KR][F]
    uint32_t F, t0, t1;
    unsigned long long *budget_hit;
    uint64_t fault_budget;
    unsigned long long *counters; // [0] evaluations, [1] fault-cycles
};

struct WinHeavy {
    const HeavyCarry *carry_in;   // heavy faults alive at t0
    const uint32_t *n_carry_in;
    const uint32_t *pool_r_in;
    const uint64_t *pool_v_in;
    HeavyCarry *carry_out;
    uint32_t *n_carry_out;
    uint32_t *pool_r_out;
    uint64_t *pool_v_out;
    unsigned long long *pool_top_out;
    uint64_t pool_cap;
    const HeavyItem *prom;        // this window's promotions: prom[*prom_begin .. *prom_end)
    const uint32_t *prom_begin;
    const uint32_t *prom_end;
    unsigned long long *head;
    uint32_t t0, t1;
    unsigned long long *budget_hit;
    uint64_t fault_budget;
    unsigned long long *counters;
    uint32_t *err;                // bit 1: pool overflow
};

// Launchers (rtlfs_kernels.cu). All enqueue on `stream` and return the launch status.
size_t good_smem_bytes(bool use_smem, uint32_t max_net, uint32_t max_reg, uint32_t max_chunks, bool staged);
// Good trace of cycles [t_begin, min(t_end, T)) of every listed design; t_begin > 0
// resumes from the trace row of cycle t_begin-1.
cudaError_t launch_good_trace(const DevDesign *d_designs, const uint32_t *design_list,
                              uint32_t n_list, uint32_t max_net, uint32_t max_reg,
                              uint32_t max_chunks, bool use_smem, bool staged, uint32_t *err,
                              cudaStream_t stream, uint32_t t_begin = 0,
                              uint32_t t_end = 0xFFFFFFFFu);
// Activation bitplane of every fault for cycles [t0, t1) (t0 a multiple of 64; t1 a
// multiple of 64 or the design's last cycle).
cudaError_t launch_activation(const DevDesign *d_designs, DevFaults f, uint64_t *act,
                              uint32_t t0, uint32_t t1, cudaStream_t stream);
// rows -> gcol for cycles [t0, t1) of all n_designs designs (one launch).
cudaError_t launch_transpose_window(const DevDesign *d_designs, uint32_t n_designs,
                                    uint32_t max_net, uint32_t t0, uint32_t t1,
                                    cudaStream_t stream);
cudaError_t launch_light_window(const DevDesign *d_designs, DevFaults f, WinLight w, int cap,
                                int block, int grid, cudaStream_t stream);
cudaError_t launch_heavy_window(const DevDesign *d_designs, DevFaults f, WinHeavy w,
                                HeavyScratch s, int block, int grid, cudaStream_t stream);
cudaError_t launch_transpose(uint64_t *gcol, const uint64_t *rows, uint32_t n_net, uint32_t T,
                             cudaStream_t stream);
// Shared memory of one cluster good-trace CTA for a design's layout.
size_t good_cluster_smem_bytes(uint32_t own, uint32_t rown, uint32_t n_inputs, uint32_t max_chunks);
// Clusters of C CTAs with `smem` bytes each that can be resident at once (0: none).
int good_cluster_max_active(uint32_t C, size_t smem);
// Good trace of the listed designs over cycles [t_begin, t_end), one cluster of C CTAs each.
// A launch that does not run in clusters of C CTAs does nothing and sets bit 2 of *err.
cudaError_t launch_good_cluster(const DevDesign *d_designs, const uint32_t *design_list,
                                uint32_t n_list, uint32_t C, size_t smem, uint32_t *err,
                                cudaStream_t stream, uint32_t t_begin, uint32_t t_end);
cudaError_t launch_light(const DevDesign *d_designs, DevFaults f, Queues q, int cap, int block,
                         int grid, cudaStream_t stream);
cudaError_t launch_heavy(const DevDesign *d_designs, DevFaults f, Queues q, HeavyScratch s,
                         int block, int grid, cudaStream_t stream);
// Dynamic shared memory of one heavy CTA (gbm: node bitmap in global scratch, a summary here).
size_t heavy_smem_bytes(uint32_t max_node, uint32_t max_levels, uint32_t max_net, bool exact, bool gbm);
cudaError_t launch_plain(const DevDesign *d_designs, uint32_t design, DevFaults f,
                         uint32_t first, uint32_t count, uint64_t *fval, uint32_t *stamp,
                         uint32_t *qstamp, uint32_t *heap, uint32_t *reg_r, uint64_t *reg_v,
                         uint32_t stride_net, uint32_t stride_node, uint32_t stride_reg,
                         cudaStream_t stream);
// Resident CTAs per SM of the light kernel (the windowed form's when `window`).
int light_max_blocks_per_sm(int cap, int block, bool window);
int heavy_max_blocks_per_sm(int block, size_t smem, bool exact, bool gbm);

}  // namespace rtlfs
