// rtlfs_host.cu -- host side of librtlfs: the C ABI declared in include/rtlfs.h.
//
// Load time (the paper's compile / inject / task-graph steps, Sec. IV Steps 1-4, here
// for a word-level op graph): validate, levelize, renumber nodes by level, build the
// fan-out CSR (successor updates of Algorithm 1), the register latch map and the output
// map, and upload them. Run time: good trace, schedule, light + heavy faulty kernels on
// two streams, results back to the caller.
#include "../../include/rtlfs.h"
#include "rtlfs_internal.h"
#include "rtlfs_sched.h"
#include "rtlfs_static.h"

#include <cuda_bf16.h>
#include <deque>
#include <memory>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace rtlfs;

namespace {

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t reserve(size_t count) {
        if (count <= n && p) return cudaSuccess;
        release();
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { p = nullptr; return e; }
        n = std::max<size_t>(count, 1);
        return cudaSuccess;
    }
    cudaError_t upload(const std::vector<T> &v) {
        cudaError_t e = reserve(v.size());
        if (e != cudaSuccess) return e;
        if (v.empty()) return cudaSuccess;
        return cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
};

struct Design {
    uint32_t I = 0, R = 0, N = 0, O = 0, n_net = 0, n_levels = 0, n_fo = 0;
    std::vector<uint32_t> ext2int, int2ext;
    std::vector<uint4> desc;
    std::vector<uint32_t> lvl_start;
    std::vector<uint16_t> node_level;
    std::vector<uint8_t> net_w;
    std::vector<uint32_t> fo_off, fo_idx, dreg_off, dreg_idx, dreg_rec, reg_d, outport, out_net;
    std::vector<uint4> netinfo;
    std::vector<uint2> chunks;
    std::vector<float> cone;          // static fan-out cone size estimate per net (log2 scale)
    std::vector<float> net_static;    // [n_net][4] cone, level, register depth, width (scaled)
    DBuf<float> d_net_static;
    DBuf<uint4> d_desc, d_netinfo;
    DBuf<uint2> d_chunks;
    DBuf<uint32_t> d_lvl_start, d_fo_off, d_fo_idx, d_dreg_off, d_dreg_idx, d_dreg_rec, d_reg_d,
        d_outport, d_out_net;
    DBuf<uint16_t> d_node_level, d_fo_lvl;
    std::vector<uint16_t> fo_lvl;
    DBuf<uint8_t> d_net_w;
    // stimulus and faults
    uint32_t T = 0;
    bool has_stim = false;
    DBuf<uint64_t> d_stim;
    std::vector<uint32_t> f_site;     // internal ids (a port fault: the port's driver net)
    std::vector<uint8_t> f_bit, f_val;   // f_val: fault kind FK_*
    std::vector<uint32_t> f_port, f_t0;  // output port of a port fault (NO_PORT); flip cycle
    // good trace
    DBuf<uint64_t> d_rows, d_gcol;
    bool trace_valid = false;
    // cluster good-trace plans, indexed by log2 of the cluster size (built on first use)
    struct ClusterPlan {
        uint32_t own = 0, rown = 0, max_ch = 0;
        size_t smem = 0;
        int usable = -1;   // clusters of this size can be resident (-1: not asked yet)
        DBuf<uint4> d_desc, d_chunk, d_reg;
        DBuf<uint32_t> d_ch_off, d_reg_off;
    };
    std::unique_ptr<ClusterPlan> plan[5];
};

}  // namespace

struct GoodLaunch {
    uint32_t n_smem = 0, n_glob = 0, max_net_s = 0, max_reg_s = 0, max_ch_s = 0, max_ch_g = 0;
    uint32_t n_cl[5] = {};        // designs on each cluster list (index log2 of the cluster size)
    size_t smem_cl[5] = {};       // shared memory per CTA of each cluster launch
};

struct rtlfs_ctx {
    int device = 0;
    GoodLaunch gl;
    // CUDA graph of the campaign's launch sequence, replayed while its key matches
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_key;
    uint32_t graph_launches = 0;
    cudaEvent_t ev_graph[2] = {};
    cudaEvent_t ev_gend = nullptr;   // end of the good-trace stream (timed inside a graph)
    // pinned scratch: [0..7] queue heads/counters, [8..9] heavy counts, [10..11] counter init
    unsigned long long *p_small = nullptr;
    int n_sm = 0;
    std::string err;
    std::vector<Design *> designs;
    cudaStream_t s_main = nullptr, s_heavy = nullptr, s_good = nullptr;
    // windowed campaign state
    DBuf<uint8_t> w_st_nreg;
    DBuf<uint32_t> w_st_r, w_live0, w_live1, w_cnt32, w_pool_r0, w_pool_r1;
    DBuf<uint64_t> w_st_v, w_pool_v0, w_pool_v1;
    DBuf<unsigned long long> w_cnt64;
    DBuf<uint64_t> d_act;              // activation bitplane [F][ceil(Tmax/64)]
    DBuf<HeavyCarry> w_carry0, w_carry1;
    uint64_t w_pool_cap = 0;
    cudaEvent_t ev_wg = nullptr, ev_wl = nullptr;
    // the good-trace launch lists of one span of cycles run side by side: the first on the
    // caller's stream, the others on these, joined back through the events
    cudaStream_t s_gaux[5] = {};
    cudaEvent_t ev_gfork = nullptr, ev_gjoin[5] = {};
    std::vector<cudaEvent_t> ev_win;   // [4][nw]: light start/end, heavy start/end
    cudaEvent_t ev[8] = {};
    DBuf<DevDesign> d_designs;
    DBuf<uint32_t> d_list_smem, d_list_glob, d_list_cl[5];
    uint32_t good_cluster = 0;         // good-trace mode of the next run (rtlfs_run_opts)
    uint32_t good_staging = 0;         // one-CTA good trace through the staged (TMA) ring
    bool faults_dirty = true;
    uint32_t F = 0;
    std::vector<uint32_t> f_first;    // first global fault id of each design
    DBuf<uint32_t> d_site, d_fport, d_ft0, d_mism;
    bool mism_valid = false;           // d_mism holds the counts of the last run (no-drop)
    DBuf<uint8_t> d_bit, d_val, d_det;
    DBuf<uint16_t> d_fdesign;
    DBuf<int32_t> d_cycle, d_port;
    DBuf<uint64_t> d_load;
    DBuf<uint32_t> d_order;
    DBuf<HeavyItem> d_init_items, d_prom_items;
    DBuf<uint32_t> d_counters;        // [0] init count, [1] prom count
    DBuf<uint32_t> d_err;             // bit 0: a good-trace staging wait ran out; bit 1: the heavy pool overflowed;
                                      // bit 2: a cluster good-trace launch ran without its clusters
    DBuf<unsigned long long> d_heads; // [0] light, [1] init heavy, [2] prom heavy, [3] budget,
                                      // [4..5] light evals/cycles, [6..7] heavy evals/cycles
    DBuf<HeavyVal> h_fval;
    DBuf<uint32_t> h_stamp;
    DBuf<uint32_t> h_regr;
    DBuf<uint64_t> h_regv;
    uint32_t heavy_slots = 0, heavy_grid = 0, hs_net = 0, hs_reg = 0, hs_node = 0, hs_lv = 0;
    bool heavy_exact = false;          // the heavy kernel's form for the current designs
    bool heavy_gbm = false;            // node bitmaps in global scratch (h_gbm)
    DBuf<uint32_t> h_gbm;
    bool stamps_stale = false;         // the exact form wrote values over stamp fields since
                                       // the scratch was last zeroed
    // scheduler state
    DBuf<const float *> d_static_ptrs;
    DBuf<float> d_X, d_heur, d_pred, d_mm;
    DBuf<uint32_t> d_hist;
    // load predictor: BF16 weights for inference, FP32 master + Adam moments for training
    bool has_weights = false;
    int adam_step = 0;
    DBuf<__nv_bfloat16> d_wb;
    DBuf<float> d_master, d_m, d_v, d_grad, d_loss, d_tx, d_ty;
    // pinned host staging of results
    int32_t *p_cycle = nullptr, *p_port = nullptr;
    uint8_t *p_det = nullptr;
    uint64_t *p_load = nullptr;
    size_t p_cap = 0;
    rtlfs_stats stats{};
    // campaign state at a window boundary (host copy), see rtlfs_checkpoint_*
    struct Checkpoint {
        bool valid = false;
        uint32_t window = 0;              // first window still to run
        uint32_t W = 0, F = 0, nodrop = 0;
        uint32_t lcap = 0;                // light capacity variant (its register-diff bound)
        std::vector<uint32_t> T, n_net;   // per design
        std::vector<uint8_t> det, st_nreg;
        std::vector<int32_t> cycle, port;
        std::vector<uint64_t> load, st_v, pool_v, heads, rows;
        std::vector<uint32_t> mism, live, st_r, pool_r;
        std::vector<HeavyCarry> carry;
    } ck;
};

namespace {

int fail(rtlfs_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CU(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RTLFS_E_NOMEM : RTLFS_E_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                          \
    } while (0)

inline int n_ops(uint32_t op) {
    return op == OP_CONST ? 0
         : (op == OP_NOT || op == OP_SHL || op == OP_SHR || op == OP_SLICE) ? 1
         : op == OP_MUX2 ? 3 : 2;
}

inline uint64_t host_mask(uint32_t w) { return w >= 64 ? ~0ull : ((1ull << w) - 1ull); }

int build_design(rtlfs_ctx *ctx, Design &D, const rtlfs_node *nodes, uint32_t N,
                 const rtlfs_reg *regs, uint32_t R, const uint8_t *in_w, uint32_t I,
                 const uint32_t *outs, uint32_t O) {
    const uint64_t n_net64 = (uint64_t)I + R + N;
    if (n_net64 == 0 || n_net64 >= (1ull << 31)) return fail(ctx, RTLFS_E_ARG, "bad net count");
    const uint32_t n_net = (uint32_t)n_net64, IR = I + R;
    std::vector<uint8_t> wext(n_net);
    for (uint32_t i = 0; i < I; ++i) {
        if (in_w[i] < 1 || in_w[i] > 64) return fail(ctx, RTLFS_E_WIDTH, "input %u width %u", i, in_w[i]);
        wext[i] = in_w[i];
    }
    for (uint32_t r = 0; r < R; ++r) {
        if (regs[r].width < 1 || regs[r].width > 64)
            return fail(ctx, RTLFS_E_WIDTH, "register %u width %u", r, regs[r].width);
        if (regs[r].d_net >= n_net) return fail(ctx, RTLFS_E_ARG, "register %u d_net out of range", r);
        wext[I + r] = regs[r].width;
    }
    for (uint32_t n = 0; n < N; ++n) {
        const rtlfs_node &x = nodes[n];
        if (x.op > OP_CONST) return fail(ctx, RTLFS_E_ARG, "node %u: bad op %u", n, x.op);
        if (x.width < 1 || x.width > 64) return fail(ctx, RTLFS_E_WIDTH, "node %u width %u", n, x.width);
        const uint32_t ops[3] = {x.a, x.b, x.c};
        for (int k = 0; k < n_ops(x.op); ++k)
            if (ops[k] >= n_net) return fail(ctx, RTLFS_E_ARG, "node %u operand %d out of range", n, k);
        wext[IR + n] = x.width;
    }
    for (uint32_t n = 0; n < N; ++n) {
        const rtlfs_node &x = nodes[n];
        if ((x.op == OP_EQ || x.op == OP_LT) && x.width != 1)
            return fail(ctx, RTLFS_E_WIDTH, "node %u: EQ/LT width must be 1", n);
        if (x.op == OP_SLICE && (uint64_t)x.imm + x.width > wext[x.a])
            return fail(ctx, RTLFS_E_WIDTH, "node %u: slice beyond operand width", n);
        if (x.op == OP_CONCAT && (uint32_t)wext[x.a] + wext[x.b] != x.width)
            return fail(ctx, RTLFS_E_WIDTH, "node %u: concat width mismatch", n);
    }
    for (uint32_t o = 0; o < O; ++o)
        if (outs[o] >= n_net) return fail(ctx, RTLFS_E_ARG, "output %u net out of range", o);
    if (O >= NI_NO_PORT) return fail(ctx, RTLFS_E_ARG, "too many output ports");

    // Levelize (Kahn over node->node operand edges); level 0 = no node operand.
    std::vector<uint32_t> indeg(N, 0), ucnt(N + 1, 0);
    for (uint32_t n = 0; n < N; ++n) {
        const uint32_t ops[3] = {nodes[n].a, nodes[n].b, nodes[n].c};
        for (int k = 0; k < n_ops(nodes[n].op); ++k)
            if (ops[k] >= IR) { ++indeg[n]; ++ucnt[ops[k] - IR + 1]; }
    }
    for (uint32_t n = 0; n < N; ++n) ucnt[n + 1] += ucnt[n];
    std::vector<uint32_t> users(ucnt[N]), fill(ucnt.begin(), ucnt.end() - 1);
    for (uint32_t n = 0; n < N; ++n) {
        const uint32_t ops[3] = {nodes[n].a, nodes[n].b, nodes[n].c};
        for (int k = 0; k < n_ops(nodes[n].op); ++k)
            if (ops[k] >= IR) users[fill[ops[k] - IR]++] = n;
    }
    std::vector<uint32_t> level(N, 0), queue;
    queue.reserve(N);
    for (uint32_t n = 0; n < N; ++n)
        if (indeg[n] == 0) queue.push_back(n);
    for (size_t h = 0; h < queue.size(); ++h) {
        const uint32_t n = queue[h];
        for (uint32_t e = ucnt[n]; e < ucnt[n + 1]; ++e) {
            const uint32_t u = users[e];
            level[u] = std::max(level[u], level[n] + 1);
            if (--indeg[u] == 0) queue.push_back(u);
        }
    }
    if (queue.size() != N) return fail(ctx, RTLFS_E_CYCLE, "combinational cycle among nodes");
    uint32_t NL = 0;
    for (uint32_t n = 0; n < N; ++n) NL = std::max(NL, level[n] + 1);
    if (N == 0) NL = 0;
    if (NL > 65535) return fail(ctx, RTLFS_E_ARG, "more than 65535 levels");

    // Renumber: nodes sorted by (level, op, index). Grouping a level's nodes by op keeps
    // the 32 nodes a warp evaluates together on one branch of the op switch.
    D.I = I; D.R = R; D.N = N; D.O = O; D.n_net = n_net; D.n_levels = NL;
    D.lvl_start.assign(NL + 1, 0);
    for (uint32_t n = 0; n < N; ++n) ++D.lvl_start[level[n] + 1];
    for (uint32_t l = 0; l < NL; ++l) D.lvl_start[l + 1] += D.lvl_start[l];
    std::vector<uint32_t> perm(N);
    for (uint32_t n = 0; n < N; ++n) perm[n] = n;
    std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) {
        return level[a] != level[b] ? level[a] < level[b] : nodes[a].op < nodes[b].op;
    });
    D.ext2int.resize(n_net);
    D.int2ext.resize(n_net);
    for (uint32_t i = 0; i < IR; ++i) D.ext2int[i] = D.int2ext[i] = i;
    D.node_level.resize(N);
    for (uint32_t k = 0; k < N; ++k) {
        const uint32_t n = perm[k];
        D.ext2int[IR + n] = IR + k;
        D.int2ext[IR + k] = IR + n;
        D.node_level[k] = (uint16_t)level[n];
    }
    D.net_w.resize(n_net);
    for (uint32_t e = 0; e < n_net; ++e) D.net_w[D.ext2int[e]] = wext[e];
    D.desc.resize(N);
    for (uint32_t n = 0; n < N; ++n) {
        const rtlfs_node &x = nodes[n];
        const uint32_t k = D.ext2int[IR + n] - IR;
        uint4 d;
        if (x.op == OP_CONST) {
            const uint64_t v = x.imm & host_mask(x.width);
            d.x = (uint32_t)v;
            d.y = (uint32_t)(v >> 32);
            d.z = 0;
        } else {
            const int no = n_ops(x.op);
            d.x = D.ext2int[x.a];
            d.y = no >= 2 ? D.ext2int[x.b] : 0;
            d.z = no >= 3 ? D.ext2int[x.c] : 0;
        }
        uint32_t kk = 0;
        if (x.op == OP_SHL || x.op == OP_SHR || x.op == OP_SLICE) kk = (uint32_t)std::min<uint64_t>(x.imm, 64);
        if (x.op == OP_CONCAT) kk = wext[x.b];
        d.w = make_meta(x.op, x.width, kk);
        D.desc[k] = d;
    }
    // Fan-out CSR over internal nets (each consumer once per distinct operand net).
    D.fo_off.assign(n_net + 1, 0);
    for (uint32_t k = 0; k < N; ++k) {
        const uint4 d = D.desc[k];
        const int no = n_ops(meta_op(d.w));
        const uint32_t ops[3] = {d.x, d.y, d.z};
        for (int j = 0; j < no; ++j) {
            bool dup = false;
            for (int i = 0; i < j; ++i) dup |= ops[i] == ops[j];
            if (!dup) ++D.fo_off[ops[j] + 1];
        }
    }
    for (uint32_t e = 0; e < n_net; ++e) D.fo_off[e + 1] += D.fo_off[e];
    D.n_fo = D.fo_off[n_net];
    D.fo_idx.resize(D.n_fo);
    {
        std::vector<uint32_t> f2(D.fo_off.begin(), D.fo_off.end() - 1);
        for (uint32_t k = 0; k < N; ++k) {
            const uint4 d = D.desc[k];
            const int no = n_ops(meta_op(d.w));
            const uint32_t ops[3] = {d.x, d.y, d.z};
            for (int j = 0; j < no; ++j) {
                bool dup = false;
                for (int i = 0; i < j; ++i) dup |= ops[i] == ops[j];
                if (!dup) D.fo_idx[f2[ops[j]]++] = k;
            }
        }
    }
    D.fo_lvl.resize(D.n_fo);
    for (uint32_t e = 0; e < D.n_fo; ++e) D.fo_lvl[e] = D.node_level[D.fo_idx[e]];
    // Latch map: registers whose D is each net.
    D.reg_d.resize(R);
    D.dreg_off.assign(n_net + 1, 0);
    for (uint32_t r = 0; r < R; ++r) {
        D.reg_d[r] = D.ext2int[regs[r].d_net];
        ++D.dreg_off[D.reg_d[r] + 1];
    }
    for (uint32_t e = 0; e < n_net; ++e) D.dreg_off[e + 1] += D.dreg_off[e];
    D.dreg_idx.resize(R);
    {
        std::vector<uint32_t> f2(D.dreg_off.begin(), D.dreg_off.end() - 1);
        for (uint32_t r = 0; r < R; ++r) D.dreg_idx[f2[D.reg_d[r]]++] = r;
    }
    if (R >= (1u << 25)) return fail(ctx, RTLFS_E_ARG, "more than 2^25 registers");
    D.dreg_rec.resize(R);
    for (uint32_t e = 0; e < R; ++e)
        D.dreg_rec[e] = D.dreg_idx[e] | ((uint32_t)wext[I + D.dreg_idx[e]] << 25);
    // Outputs.
    D.out_net.resize(O);
    D.outport.assign(n_net, NO_PORT);
    for (uint32_t o = 0; o < O; ++o) {
        const uint32_t net = D.ext2int[outs[o]];
        D.out_net[o] = net;
        D.outport[net] = std::min(D.outport[net], o);
    }
    // Per-net records and good-trace chunks.
    D.netinfo.resize(n_net);
    for (uint32_t e = 0; e < n_net; ++e) {
        const uint32_t nr = D.dreg_off[e + 1] - D.dreg_off[e];
        const uint32_t port = D.outport[e] == NO_PORT ? NI_NO_PORT : D.outport[e];
        D.netinfo[e] = make_uint4(D.fo_off[e], D.fo_off[e + 1], D.dreg_off[e],
                                  (std::min<uint32_t>(nr, 255u) << 24) | port);
    }
    D.chunks.clear();
    for (uint32_t l = 0; l < NL; ++l) {
        for (uint32_t lo = D.lvl_start[l]; lo < D.lvl_start[l + 1]; lo += GOOD_BLOCK) {
            const uint32_t hi = std::min(lo + GOOD_BLOCK, D.lvl_start[l + 1]);
            D.chunks.push_back(make_uint2(lo, hi | (hi == D.lvl_start[l + 1] ? 0x80000000u : 0u)));
        }
    }
    // Static fan-out cone estimate (reverse topological sum, capped): scheduling feature.
    D.cone.assign(n_net, 0.f);
    {
        std::vector<double> cs(n_net, 1.0);
        for (int64_t k = (int64_t)N - 1; k >= 0; --k) {
            const uint32_t net = IR + (uint32_t)k;
            double s = 1.0;
            for (uint32_t e = D.fo_off[net]; e < D.fo_off[net + 1]; ++e) s += cs[IR + D.fo_idx[e]];
            cs[net] = std::min(s, 1e9);
        }
        for (uint32_t net = 0; net < IR; ++net) {
            double s = 1.0;
            for (uint32_t e = D.fo_off[net]; e < D.fo_off[net + 1]; ++e) s += cs[IR + D.fo_idx[e]];
            cs[net] = std::min(s, 1e9);
        }
        for (uint32_t e = 0; e < n_net; ++e) D.cone[e] = (float)std::log2(cs[e]);
    }
    // Register depth to the outputs: fewest register stages on any path from the net to
    // an output port (0-1 breadth-first search backwards from the outputs).
    std::vector<uint32_t> depth(n_net, 0xFFFFFFFFu);
    {
        std::deque<uint32_t> dq;
        for (uint32_t o = 0; o < O; ++o)
            if (depth[D.out_net[o]] != 0) { depth[D.out_net[o]] = 0; dq.push_front(D.out_net[o]); }
        while (!dq.empty()) {
            const uint32_t y = dq.front();
            dq.pop_front();
            const uint32_t dy = depth[y];
            if (y >= IR) {
                const uint4 d = D.desc[y - IR];
                const int no = n_ops(meta_op(d.w));
                const uint32_t ops[3] = {d.x, d.y, d.z};
                for (int k = 0; k < no; ++k)
                    if (depth[ops[k]] > dy) { depth[ops[k]] = dy; dq.push_front(ops[k]); }
            } else if (y >= I) {
                const uint32_t x = D.reg_d[y - I];
                if (depth[x] > dy + 1) { depth[x] = dy + 1; dq.push_back(x); }
            }
        }
    }
    D.net_static.resize((size_t)n_net * 4);
    for (uint32_t e = 0; e < n_net; ++e) {
        float *ns = &D.net_static[(size_t)e * 4];
        ns[0] = std::min(D.cone[e] / 20.f, 1.5f);
        ns[1] = e < IR ? 0.f : (float)(D.node_level[e - IR] + 1) / (float)std::max<uint32_t>(NL, 1);
        ns[2] = (float)std::min<uint32_t>(depth[e], 16u) / 16.f;
        ns[3] = (float)D.net_w[e] / 64.f;
    }
    return RTLFS_OK;
}

int upload_design(rtlfs_ctx *ctx, Design &D) {
    CU(D.d_desc.upload(D.desc));
    CU(D.d_netinfo.upload(D.netinfo));
    CU(D.d_net_static.upload(D.net_static));
    CU(D.d_chunks.upload(D.chunks));
    CU(D.d_lvl_start.upload(D.lvl_start));
    CU(D.d_node_level.upload(D.node_level));
    CU(D.d_net_w.upload(D.net_w));
    CU(D.d_fo_off.upload(D.fo_off));
    CU(D.d_fo_idx.upload(D.fo_idx));
    CU(D.d_fo_lvl.upload(D.fo_lvl));
    CU(D.d_dreg_off.upload(D.dreg_off));
    CU(D.d_dreg_idx.upload(D.dreg_idx));
    CU(D.d_dreg_rec.upload(D.dreg_rec));
    CU(D.d_reg_d.upload(D.reg_d));
    CU(D.d_outport.upload(D.outport));
    CU(D.d_out_net.upload(D.out_net));
    return RTLFS_OK;
}

DevDesign dev_view(const Design &D) {
    DevDesign v{};
    v.I = D.I; v.R = D.R; v.N = D.N; v.O = D.O; v.n_net = D.n_net; v.n_levels = D.n_levels;
    v.T = D.T; v.n_fo = D.n_fo;
    v.n_chunks = (uint32_t)D.chunks.size();
    v.netinfo = D.d_netinfo.p; v.chunks = D.d_chunks.p;
    v.desc = D.d_desc.p; v.lvl_start = D.d_lvl_start.p; v.node_level = D.d_node_level.p;
    v.net_w = D.d_net_w.p; v.fo_off = D.d_fo_off.p; v.fo_idx = D.d_fo_idx.p; v.fo_lvl = D.d_fo_lvl.p;
    v.dreg_off = D.d_dreg_off.p; v.dreg_idx = D.d_dreg_idx.p; v.dreg_rec = D.d_dreg_rec.p; v.reg_d = D.d_reg_d.p;
    v.outport = D.d_outport.p; v.out_net = D.d_out_net.p; v.stim = D.d_stim.p;
    v.rows = D.d_rows.p; v.gcol = D.d_gcol.p;
    return v;
}

constexpr size_t SMEM_LIMIT = 227 * 1024;   // dynamic shared memory of one good-trace CTA

// Cluster plan of a design for clusters of C CTAs: every level's nodes split into C
// contiguous shares (CTA k owns its shares in level order, one value word per node),
// registers split into C contiguous index blocks (their home CTAs), every operand
// rewritten as the location of its value, and each CTA's chunk list (at least one chunk
// per level, so every CTA joins every level's barrier).
int build_cluster_plan(rtlfs_ctx *ctx, Design &D, uint32_t C, int lc) {
    auto P = std::make_unique<Design::ClusterPlan>();
    const uint32_t I = D.I, R = D.R, N = D.N, IR = I + R, NL = D.n_levels;
    std::vector<uint32_t> own(C, 0), node_rank(N), node_slot(N);
    std::vector<std::vector<uint4>> chunks(C);
    for (uint32_t l = 0; l < NL; ++l) {
        const uint32_t lo = D.lvl_start[l], n = D.lvl_start[l + 1] - lo;
        for (uint32_t k = 0; k < C; ++k) {
            const uint32_t a = lo + (uint32_t)((uint64_t)n * k / C);
            const uint32_t b = lo + (uint32_t)((uint64_t)n * (k + 1) / C);
            for (uint32_t x = a; x < b; ++x) { node_rank[x] = k; node_slot[x] = own[k] + (x - a); }
            if (a == b) chunks[k].push_back(make_uint4(own[k], 0x80000000u, a, 0));
            for (uint32_t x = a; x < b; x += GOOD_BLOCK) {
                const uint32_t m = std::min(GOOD_BLOCK, b - x);
                chunks[k].push_back(make_uint4(own[k] + (x - a), m | (x + m == b ? 0x80000000u : 0u), x, 0));
            }
            own[k] += b - a;
        }
    }
    std::vector<uint32_t> reg_off(C + 1), reg_home(R);
    for (uint32_t k = 0; k <= C; ++k) reg_off[k] = (uint32_t)((uint64_t)R * k / C);
    for (uint32_t k = 0; k < C; ++k)
        for (uint32_t r = reg_off[k]; r < reg_off[k + 1]; ++r) reg_home[r] = k;
    P->own = *std::max_element(own.begin(), own.end());
    P->rown = 0;
    for (uint32_t k = 0; k < C; ++k) P->rown = std::max(P->rown, reg_off[k + 1] - reg_off[k]);
    if ((uint64_t)P->own + 2ull * P->rown + I > CL_WORD) return fail(ctx, RTLFS_E_ARG, "design too large for a cluster plan");
    auto loc = [&](uint32_t net) -> uint32_t {
        if (net < I) return CL_SELF | (P->own + 2 * P->rown + net);
        if (net < IR) {
            const uint32_t r = net - I, k = reg_home[r];
            return CL_REG | (k << CL_RANK_SHIFT) | (P->own + r - reg_off[k]);
        }
        const uint32_t x = net - IR;
        return (node_rank[x] << CL_RANK_SHIFT) | node_slot[x];
    };
    std::vector<uint4> cdesc((size_t)C * P->own, make_uint4(0, 0, 0, 0));
    for (uint32_t x = 0; x < N; ++x) {
        uint4 d = D.desc[x];
        const int no = n_ops(meta_op(d.w));
        if (no >= 1) d.x = loc(d.x);
        if (no >= 2) d.y = loc(d.y);
        if (no >= 3) d.z = loc(d.z);
        cdesc[(size_t)node_rank[x] * P->own + node_slot[x]] = d;
    }
    std::vector<uint4> creg(R);
    for (uint32_t r = 0; r < R; ++r) creg[r] = make_uint4(r, loc(D.reg_d[r]), D.net_w[I + r], D.reg_d[r]);
    std::vector<uint4> call;
    std::vector<uint32_t> ch_off(C + 1, 0);
    P->max_ch = 0;
    for (uint32_t k = 0; k < C; ++k) {
        ch_off[k] = (uint32_t)call.size();
        call.insert(call.end(), chunks[k].begin(), chunks[k].end());
        P->max_ch = std::max<uint32_t>(P->max_ch, (uint32_t)chunks[k].size());
    }
    ch_off[C] = (uint32_t)call.size();
    P->smem = good_cluster_smem_bytes(P->own, P->rown, I, P->max_ch);
    CU(P->d_desc.upload(cdesc));
    CU(P->d_chunk.upload(call));
    CU(P->d_reg.upload(creg));
    CU(P->d_ch_off.upload(ch_off));
    CU(P->d_reg_off.upload(reg_off));
    D.plan[lc] = std::move(P);
    return RTLFS_OK;
}

// Whether clusters of C CTAs can run design D's good trace; builds the plan on first use.
int cluster_usable(rtlfs_ctx *ctx, Design &D, uint32_t C, int lc, bool *ok) {
    *ok = false;
    if (!D.plan[lc]) {
        int rc = build_cluster_plan(ctx, D, C, lc);
        if (rc != RTLFS_OK) return rc;
    }
    Design::ClusterPlan &P = *D.plan[lc];
    if (P.smem > SMEM_LIMIT) return RTLFS_OK;
    if ((uint64_t)D.T * P.max_ch >= (1ull << 32)) return RTLFS_OK;
    if (P.usable < 0) P.usable = good_cluster_max_active(C, P.smem) > 0 ? 1 : 0;
    *ok = P.usable == 1;
    return RTLFS_OK;
}

// Allocate traces, choose each design's good-trace form and upload the design table and
// the launch lists: one CTA with net values in shared memory when the design fits, else
// the smallest cluster whose CTAs hold the design in distributed shared memory, else one
// CTA with net values in the global trace. ctx->good_cluster overrides the choice:
// 1 = one CTA, 2..16 = clusters of that size.
int prepare_good(rtlfs_ctx *ctx) {
    std::vector<DevDesign> tab;
    std::vector<uint32_t> l_smem, l_glob, l_cl[5];
    GoodLaunch g{};
    const uint32_t force = ctx->good_cluster;
    for (size_t i = 0; i < ctx->designs.size(); ++i) {
        Design &D = *ctx->designs[i];
        const size_t cells = (size_t)D.n_net * D.T;
        CU(D.d_rows.reserve(cells));
        CU(D.d_gcol.reserve(cells));
        DevDesign v = dev_view(D);
        const uint32_t nch = (uint32_t)D.chunks.size();
        int lc = 0;   // log2 of the chosen cluster size; 0 = one CTA
        if (force >= 2) {
            lc = 1;
            while ((1u << lc) < force) ++lc;
            bool ok = false;
            int rc = cluster_usable(ctx, D, 1u << lc, lc, &ok);
            if (rc != RTLFS_OK) return rc;
            if (!ok) return fail(ctx, RTLFS_E_ARG, "design %zu cannot run its good trace on clusters of %u", i, 1u << lc);
        } else {
            // net values in shared memory when the design fits together with the designs
            // already on the shared-memory list (one launch covers the whole list)
            const uint32_t mn = std::max(g.max_net_s, D.n_net), mr = std::max(g.max_reg_s, D.R);
            const uint32_t mc = std::max(g.max_ch_s, nch);
            if (good_smem_bytes(true, mn, mr, mc, ctx->good_staging != 0) <= SMEM_LIMIT) {
                l_smem.push_back((uint32_t)i);
                g.max_net_s = mn; g.max_reg_s = mr; g.max_ch_s = mc;
            } else {
                if (force == 0) {
                    for (lc = 1; (1u << lc) <= CL_MAX; ++lc) {
                        bool ok = false;
                        int rc = cluster_usable(ctx, D, 1u << lc, lc, &ok);
                        if (rc != RTLFS_OK) return rc;
                        if (ok) break;
                    }
                    if ((1u << lc) > CL_MAX) lc = 0;
                }
                if (lc == 0) {
                    l_glob.push_back((uint32_t)i);
                    g.max_ch_g = std::max(g.max_ch_g, nch);
                }
            }
        }
        if (lc > 0) {
            const Design::ClusterPlan &P = *D.plan[lc];
            v.cl_own = P.own; v.cl_rown = P.rown;
            v.cl_desc = P.d_desc.p; v.cl_chunk = P.d_chunk.p; v.cl_ch_off = P.d_ch_off.p;
            v.cl_reg = P.d_reg.p; v.cl_reg_off = P.d_reg_off.p;
            l_cl[lc].push_back((uint32_t)i);
            g.smem_cl[lc] = std::max(g.smem_cl[lc], P.smem);
        }
        tab.push_back(v);
    }
    CU(ctx->d_designs.upload(tab));
    CU(ctx->d_list_smem.upload(l_smem));
    CU(ctx->d_list_glob.upload(l_glob));
    for (int lc = 1; lc < 5; ++lc) {
        CU(ctx->d_list_cl[lc].upload(l_cl[lc]));
        g.n_cl[lc] = (uint32_t)l_cl[lc].size();
    }
    if (good_smem_bytes(false, 0, 0, g.max_ch_g, ctx->good_staging != 0) > SMEM_LIMIT)
        return fail(ctx, RTLFS_E_ARG, "design has too many levels");
    CU(ctx->d_err.reserve(1));
    g.n_smem = (uint32_t)l_smem.size();
    g.n_glob = (uint32_t)l_glob.size();
    ctx->gl = g;
    return RTLFS_OK;
}

// Good-trace launches of cycles [t0, t1) for every list, ordered on `stream` (work enqueued
// on it later waits for all of them); *n counts them. The lists of different forms run
// concurrently: each design is a CTA or cluster of its own, independent of the others.
int launch_good_lists(rtlfs_ctx *ctx, cudaStream_t stream, uint32_t t0, uint32_t t1, uint32_t *n) {
    const GoodLaunch &g = ctx->gl;
    int k = 0;   // launches so far; the first goes on `stream`, the rest on s_gaux[k - 1]
    auto next_stream = [&](cudaStream_t *out) -> int {
        if (k == 0) {
            *out = stream;
        } else {
            if (k == 1) CU(cudaEventRecord(ctx->ev_gfork, stream));
            CU(cudaStreamWaitEvent(ctx->s_gaux[k - 1], ctx->ev_gfork, 0));
            *out = ctx->s_gaux[k - 1];
        }
        ++k;
        return RTLFS_OK;
    };
    cudaStream_t st = nullptr;
    if (g.n_smem) {
        if (int r = next_stream(&st)) return r;
        CU(launch_good_trace(ctx->d_designs.p, ctx->d_list_smem.p, g.n_smem, g.max_net_s, g.max_reg_s,
                             g.max_ch_s, true, ctx->good_staging != 0, ctx->d_err.p, st, t0, t1));
    }
    if (g.n_glob) {
        if (int r = next_stream(&st)) return r;
        CU(launch_good_trace(ctx->d_designs.p, ctx->d_list_glob.p, g.n_glob, 0, 0, g.max_ch_g, false,
                             ctx->good_staging != 0, ctx->d_err.p, st, t0, t1));
    }
    for (int lc = 1; lc < 5; ++lc) {
        if (!g.n_cl[lc]) continue;
        if (int r = next_stream(&st)) return r;
        CU(launch_good_cluster(ctx->d_designs.p, ctx->d_list_cl[lc].p, g.n_cl[lc], 1u << lc, g.smem_cl[lc], ctx->d_err.p,
                               st, t0, t1));
    }
    for (int j = 1; j < k; ++j) {   // join
        CU(cudaEventRecord(ctx->ev_gjoin[j - 1], ctx->s_gaux[j - 1]));
        CU(cudaStreamWaitEvent(stream, ctx->ev_gjoin[j - 1], 0));
    }
    *n += (uint32_t)k;
    return RTLFS_OK;
}

// Enqueue good trace + transposes on s_main (stream work only; prepare_good first).
int launch_good(rtlfs_ctx *ctx, uint32_t *n_launches = nullptr) {
    uint32_t n = 0;
    CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(uint32_t), ctx->s_main));
    int rc = launch_good_lists(ctx, ctx->s_main, 0, 0xFFFFFFFFu, &n);
    if (rc != RTLFS_OK) return rc;
    for (Design *D : ctx->designs) {
        CU(launch_transpose(D->d_gcol.p, D->d_rows.p, D->n_net, D->T, ctx->s_main));
        ++n;
    }
    if (n_launches) *n_launches += n;
    return RTLFS_OK;
}

int enqueue_good(rtlfs_ctx *ctx) {
    int rc = prepare_good(ctx);
    return rc != RTLFS_OK ? rc : launch_good(ctx);
}

int build_faults(rtlfs_ctx *ctx) {
    if (!ctx->faults_dirty) return RTLFS_OK;
    std::vector<uint32_t> site, port, t0;
    std::vector<uint8_t> bit, val;
    std::vector<uint16_t> des;
    ctx->f_first.clear();
    for (size_t i = 0; i < ctx->designs.size(); ++i) {
        Design &D = *ctx->designs[i];
        ctx->f_first.push_back((uint32_t)site.size());
        site.insert(site.end(), D.f_site.begin(), D.f_site.end());
        bit.insert(bit.end(), D.f_bit.begin(), D.f_bit.end());
        val.insert(val.end(), D.f_val.begin(), D.f_val.end());
        port.insert(port.end(), D.f_port.begin(), D.f_port.end());
        t0.insert(t0.end(), D.f_t0.begin(), D.f_t0.end());
        des.insert(des.end(), D.f_site.size(), (uint16_t)i);
    }
    ctx->f_first.push_back((uint32_t)site.size());
    ctx->F = (uint32_t)site.size();
    CU(ctx->d_site.upload(site));
    CU(ctx->d_bit.upload(bit));
    CU(ctx->d_val.upload(val));
    CU(ctx->d_fport.upload(port));
    CU(ctx->d_ft0.upload(t0));
    CU(ctx->d_mism.reserve(ctx->F));
    ctx->mism_valid = false;
    CU(ctx->d_fdesign.upload(des));
    CU(ctx->d_cycle.reserve(ctx->F));
    CU(ctx->d_port.reserve(ctx->F));
    CU(ctx->d_det.reserve(ctx->F));
    CU(ctx->d_load.reserve(ctx->F));
    CU(ctx->d_order.reserve(ctx->F));
    CU(ctx->d_prom_items.reserve(ctx->F));
    CU(ctx->d_init_items.reserve(ctx->F));
    if (ctx->p_cap < ctx->F || !ctx->p_cycle) {
        if (ctx->p_cycle) { cudaFreeHost(ctx->p_cycle); cudaFreeHost(ctx->p_port); cudaFreeHost(ctx->p_det); cudaFreeHost(ctx->p_load); }
        const size_t n = std::max<size_t>(ctx->F, 1);
        CU(cudaMallocHost(&ctx->p_cycle, n * sizeof(int32_t)));
        CU(cudaMallocHost(&ctx->p_port, n * sizeof(int32_t)));
        CU(cudaMallocHost(&ctx->p_det, n));
        CU(cudaMallocHost(&ctx->p_load, n * sizeof(uint64_t)));
        ctx->p_cap = n;
    }
    ctx->faults_dirty = false;
    return RTLFS_OK;
}

DevFaults dev_faults(rtlfs_ctx *ctx) {
    DevFaults f{};
    f.F = ctx->F;
    f.site = ctx->d_site.p; f.bit = ctx->d_bit.p; f.val = ctx->d_val.p; f.design = ctx->d_fdesign.p;
    f.port = ctx->d_fport.p; f.t0 = ctx->d_ft0.p;
    f.mism = nullptr;   // drop at first detection unless the run asks otherwise
    f.res_cycle = ctx->d_cycle.p; f.res_port = ctx->d_port.p; f.res_det = ctx->d_det.p;
    f.load = ctx->d_load.p;
    return f;
}

int ensure_heavy_scratch(rtlfs_ctx *ctx, int block, int want_slots, int form) {
    uint32_t mn = 1, mr = 1, mnode = 1, ml = 1;
    for (Design *D : ctx->designs) {
        mn = std::max(mn, D->n_net); mr = std::max(mr, D->R);
        mnode = std::max(mnode, D->N); ml = std::max(ml, D->n_levels);
    }
    // The exact form (a shared bit per net) unless that bitmap costs resident CTAs; the
    // global-bitmap form (node bitmap in global scratch, one warp per fault) when the node
    // bitmap in shared memory would halve the resident CTAs or worse: its marks and gathers
    // go through L2, which costs more per level than the occupancy it buys below that.
    if (form == 3 && block != 32) return fail(ctx, RTLFS_E_ARG, "heavy_form 3 needs heavy_block 32");
    const size_t smem_s = heavy_smem_bytes(mnode, ml, mn, false, false), smem_x = heavy_smem_bytes(mnode, ml, mn, true, false);
    const size_t smem_g = heavy_smem_bytes(mnode, ml, mn, false, true);
    const int per_sm_s = smem_s <= 220 * 1024 ? heavy_max_blocks_per_sm(block, smem_s, false, false) : 0;
    const int per_sm_x = smem_x <= 220 * 1024 ? heavy_max_blocks_per_sm(block, smem_x, true, false) : 0;
    const int per_sm_g = block == 32 && smem_g <= 220 * 1024 ? heavy_max_blocks_per_sm(block, smem_g, false, true) : 0;
    bool gbm = false, exact = false;
    if (form == 1) exact = per_sm_x > 0;
    else if (form == 3) gbm = true;
    else if (form == 0) {
        exact = per_sm_x >= per_sm_s;
        gbm = per_sm_g >= 2 * std::max(per_sm_x, per_sm_s);
        if (gbm) exact = false;
    }
    const int per_sm = gbm ? per_sm_g : exact ? per_sm_x : per_sm_s;
    if (per_sm < 1) return fail(ctx, RTLFS_E_ARG, "heavy kernel cannot be resident with block %d", block);
    ctx->heavy_exact = exact;
    ctx->heavy_gbm = gbm;
    if (exact) {
        ctx->stamps_stale = true;   // its 8-byte values overwrite stamp fields
    }
    int slots = want_slots > 0 ? want_slots : per_sm * ctx->n_sm;
    slots = std::min(slots, per_sm * ctx->n_sm);
    const bool grow = slots > (int)ctx->heavy_slots || mn > ctx->hs_net || mr > ctx->hs_reg;
    if (grow) {
        ctx->h_fval.release(); ctx->h_regr.release(); ctx->h_regv.release(); ctx->h_stamp.release();
        CU(ctx->h_fval.reserve((size_t)slots * mn));
        CU(ctx->h_stamp.reserve((size_t)slots));
        ctx->stamps_stale = true;   // fresh memory: zeroed below before a stamped run
        CU(ctx->h_regr.reserve((size_t)slots * 2 * mr));
        CU(ctx->h_regv.reserve((size_t)slots * 2 * mr));
        ctx->heavy_slots = slots; ctx->hs_net = mn; ctx->hs_reg = mr;
    }
    ctx->hs_node = mnode; ctx->hs_lv = ml;
    ctx->heavy_grid = (uint32_t)slots;
    if (gbm) {   // node bitmaps start zero and every fault leaves them zero
        const size_t need = (size_t)slots * ((mnode + 31) / 32);
        if (ctx->h_gbm.n < need) {
            ctx->h_gbm.release();
            CU(ctx->h_gbm.reserve(need));
            CU(cudaMemsetAsync(ctx->h_gbm.p, 0, ctx->h_gbm.n * sizeof(uint32_t), ctx->s_main));
        }
    }
    if (!exact && ctx->stamps_stale) {
        // stamp 0 is never current: zeroed entries and counters start every slot clean
        // (on the main stream, which every heavy launch of the campaign waits behind)
        CU(cudaMemsetAsync(ctx->h_fval.p, 0, ctx->h_fval.n * sizeof(HeavyVal), ctx->s_main));
        CU(cudaMemsetAsync(ctx->h_stamp.p, 0, ctx->h_stamp.n * sizeof(uint32_t), ctx->s_main));
        ctx->stamps_stale = false;
    }
    return RTLFS_OK;
}

HeavyScratch heavy_view(rtlfs_ctx *ctx) {
    HeavyScratch s{};
    s.fval = ctx->h_fval.p;
    s.stamp = ctx->h_stamp.p;
    s.reg_r = ctx->h_regr.p; s.reg_v = ctx->h_regv.p;
    s.max_net = ctx->hs_net; s.max_reg = ctx->hs_reg; s.max_node = ctx->hs_node;
    s.exact = ctx->heavy_exact ? 1u : 0u;
    s.gbm = ctx->heavy_gbm ? ctx->h_gbm.p : nullptr;
    s.max_levels = ctx->hs_lv;
    return s;
}

int ensure_sched_buffers(rtlfs_ctx *ctx) {
    std::vector<const float *> ptrs;
    for (Design *D : ctx->designs) ptrs.push_back(D->d_net_static.p);
    CU(ctx->d_static_ptrs.upload(ptrs));
    const size_t F = std::max<size_t>(ctx->F, 1);
    CU(ctx->d_X.reserve(F * MLP_IN));
    CU(ctx->d_heur.reserve(F));
    CU(ctx->d_pred.reserve(F));
    CU(ctx->d_mm.reserve(2));
    CU(ctx->d_hist.reserve(SORT_BUCKETS));
    return RTLFS_OK;
}

int ensure_mlp(rtlfs_ctx *ctx) {
    CU(ctx->d_wb.reserve(MLP_PARAMS));
    CU(ctx->d_master.reserve(MLP_PARAMS));
    CU(ctx->d_m.reserve(MLP_PARAMS));
    CU(ctx->d_v.reserve(MLP_PARAMS));
    CU(ctx->d_grad.reserve(MLP_PARAMS));
    CU(ctx->d_loss.reserve(1));
    return RTLFS_OK;
}

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        (void)cudaGetLastError();   // not sticky: keep it from reaching a later launch check
        return 0.f;
    }
    return ms;
}

}  // namespace

// ---- ABI ------------------------------------------------------------------------------

namespace {

// Validate one fault (caller numbering; ids n_net + o are output ports) and convert it to
// the device form. kind: RTLFS_FAULT_*.
int convert_fault(rtlfs_ctx *ctx, const Design &D, uint32_t i, uint32_t net, uint32_t bit, uint32_t kind,
                  uint32_t cycle, uint32_t *site, uint8_t *b, uint8_t *v, uint32_t *port, uint32_t *t0) {
    if (net >= D.n_net + D.O) return fail(ctx, RTLFS_E_ARG, "fault %u: net out of range", i);
    const bool is_port = net >= D.n_net;
    const uint32_t in = is_port ? D.out_net[net - D.n_net] : D.ext2int[net];
    if (bit >= D.net_w[in]) return fail(ctx, RTLFS_E_ARG, "fault %u: bit beyond net width", i);
    const bool is_reg = !is_port && in >= D.I && in < D.I + D.R;
    if (kind > RTLFS_FAULT_SET) return fail(ctx, RTLFS_E_ARG, "fault %u: unknown fault kind", i);
    if (kind == RTLFS_FAULT_SEU && !is_reg) return fail(ctx, RTLFS_E_ARG, "fault %u: an SEU site must be a register", i);
    if (kind == RTLFS_FAULT_SET && is_reg) return fail(ctx, RTLFS_E_ARG, "fault %u: a flip of a register is an SEU", i);
    *site = in;
    *b = (uint8_t)bit;
    *v = (uint8_t)(kind <= RTLFS_FAULT_SA1 ? kind : FK_FLIP);
    *port = is_port ? net - D.n_net : NO_PORT;
    *t0 = kind <= RTLFS_FAULT_SA1 ? 0u : cycle;
    return RTLFS_OK;
}

template <typename Get>
int set_faults_impl(rtlfs_ctx *ctx, uint32_t design_id, uint32_t n_faults, bool null_list, Get get) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size()) return fail(ctx, RTLFS_E_ARG, "bad design id");
    if (n_faults && null_list) return fail(ctx, RTLFS_E_ARG, "null faults");
    Design &D = *ctx->designs[design_id];
    std::vector<uint32_t> s(n_faults), port(n_faults), t0(n_faults);
    std::vector<uint8_t> b(n_faults), v(n_faults);
    for (uint32_t i = 0; i < n_faults; ++i) {
        uint32_t net, bit, kind, cycle;
        int rc = get(i, &net, &bit, &kind, &cycle);
        if (rc == RTLFS_OK) rc = convert_fault(ctx, D, i, net, bit, kind, cycle, &s[i], &b[i], &v[i], &port[i], &t0[i]);
        if (rc != RTLFS_OK) return rc;
    }
    D.f_site.swap(s); D.f_bit.swap(b); D.f_val.swap(v); D.f_port.swap(port); D.f_t0.swap(t0);
    ctx->faults_dirty = true;
    ctx->ck.valid = false;
    ctx->err.clear();
    return RTLFS_OK;
}

}  // namespace

namespace {

// Whether the context can continue the checkpoint: same fault count, designs, stimulus
// lengths, net counts, window, no-drop mode and light capacity (the light lanes' register
// diffs were bounded by it).
int checkpoint_matches(rtlfs_ctx *ctx, const rtlfs_ctx::Checkpoint &c, uint32_t W, bool nodrop, int lcap) {
    if (!c.valid) return fail(ctx, RTLFS_E_STATE, "no checkpoint to resume from");
    if (c.F != ctx->F || c.T.size() != ctx->designs.size())
        return fail(ctx, RTLFS_E_ARG, "checkpoint was taken on other fault lists or designs");
    for (size_t d = 0; d < ctx->designs.size(); ++d)
        if (c.T[d] != ctx->designs[d]->T || c.n_net[d] != ctx->designs[d]->n_net)
            return fail(ctx, RTLFS_E_ARG, "checkpoint design %zu differs from the context's", d);
    if (c.W != W) return fail(ctx, RTLFS_E_ARG, "resume needs the checkpoint's window (%u)", c.W);
    if (c.nodrop != (nodrop ? 1u : 0u)) return fail(ctx, RTLFS_E_ARG, "resume needs the checkpoint's no_drop mode");
    if (lcap >= 0 && c.lcap != (uint32_t)lcap)
        return fail(ctx, RTLFS_E_ARG, "resume needs the checkpoint's light_cap (%u)", c.lcap + 1);
    return RTLFS_OK;
}

// Copy the campaign state after window w_end - 1 to the host (after the stream has drained).
// pending[f] marks the faults still alive at the stop.
int take_checkpoint(rtlfs_ctx *ctx, uint32_t nw, uint32_t w_end, uint32_t W, bool nodrop, int lcap,
                    std::vector<uint8_t> *pending) {
    rtlfs_ctx::Checkpoint &c = ctx->ck;
    const uint32_t F = ctx->F, wl = w_end - 1;
    c = rtlfs_ctx::Checkpoint{};
    c.window = w_end; c.W = W; c.F = F; c.nodrop = nodrop ? 1u : 0u; c.lcap = (uint32_t)lcap;
    for (Design *D : ctx->designs) { c.T.push_back(D->T); c.n_net.push_back(D->n_net); }
    uint32_t n_live = 0, n_carry = 0;
    unsigned long long pool_top = 0;
    CU(cudaMemcpy(&n_live, ctx->w_cnt32.p + wl, 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&n_carry, ctx->w_cnt32.p + 2 * (size_t)nw + wl, 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&pool_top, ctx->w_cnt64.p + wl, 8, cudaMemcpyDeviceToHost));
    if (n_live > F || n_carry > F || pool_top > ctx->w_pool_cap) return fail(ctx, RTLFS_E_CUDA, "inconsistent campaign counters");
    auto get = [&](auto &v, const auto *src, size_t n) -> int {
        v.resize(n);
        if (n) CU(cudaMemcpy(v.data(), src, n * sizeof(v[0]), cudaMemcpyDeviceToHost));
        return RTLFS_OK;
    };
    int r = RTLFS_OK;
    if ((r = get(c.det, ctx->d_det.p, F)) || (r = get(c.cycle, ctx->d_cycle.p, F)) ||
        (r = get(c.port, ctx->d_port.p, F)) || (r = get(c.load, ctx->d_load.p, F)) ||
        (r = get(c.mism, ctx->d_mism.p, F)) || (r = get(c.st_nreg, ctx->w_st_nreg.p, F)) ||
        (r = get(c.st_r, ctx->w_st_r.p, (size_t)F * LIGHT_KR)) || (r = get(c.st_v, ctx->w_st_v.p, (size_t)F * LIGHT_KR)) ||
        (r = get(c.live, (wl & 1) ? ctx->w_live1.p : ctx->w_live0.p, n_live)) ||
        (r = get(c.carry, (wl & 1) ? ctx->w_carry1.p : ctx->w_carry0.p, n_carry)) ||
        (r = get(c.pool_r, (wl & 1) ? ctx->w_pool_r1.p : ctx->w_pool_r0.p, pool_top)) ||
        (r = get(c.pool_v, (wl & 1) ? ctx->w_pool_v1.p : ctx->w_pool_v0.p, pool_top)) ||
        (r = get(c.heads, ctx->d_heads.p, 8)))
        return r;
    // each design's good-trace row of the last cycle before the stop: the good machine's
    // registers restart from it
    const uint32_t cyc = w_end * W;
    for (Design *D : ctx->designs) {
        std::vector<uint64_t> row(D->n_net, 0);
        if (cyc <= D->T && D->n_net)
            CU(cudaMemcpy(row.data(), D->d_rows.p + (size_t)(cyc - 1) * D->n_net, (size_t)D->n_net * 8, cudaMemcpyDeviceToHost));
        c.rows.insert(c.rows.end(), row.begin(), row.end());
    }
    pending->assign(F, 0);
    for (uint32_t f : c.live) if (f < F) (*pending)[f] = 1;
    for (const HeavyCarry &h : c.carry) if (h.fault < F) (*pending)[h.fault] = 1;
    c.valid = true;
    return RTLFS_OK;
}

// Put the checkpoint's state where window w_begin reads it (stream work on s_main, before the
// first window's launches).
int restore_checkpoint(rtlfs_ctx *ctx, uint32_t nw, uint32_t w_begin, uint32_t *prom_total) {
    const rtlfs_ctx::Checkpoint &c = ctx->ck;
    const uint32_t F = ctx->F, wp = w_begin - 1;
    cudaStream_t s = ctx->s_main;
    auto put = [&](auto *dst, const auto &v) -> int {
        if (!v.empty()) CU(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, s));
        return RTLFS_OK;
    };
    int r = RTLFS_OK;
    if ((r = put(ctx->d_det.p, c.det)) || (r = put(ctx->d_cycle.p, c.cycle)) || (r = put(ctx->d_port.p, c.port)) ||
        (r = put(ctx->d_load.p, c.load)) || (r = put(ctx->d_mism.p, c.mism)) || (r = put(ctx->w_st_nreg.p, c.st_nreg)) ||
        (r = put(ctx->w_st_r.p, c.st_r)) || (r = put(ctx->w_st_v.p, c.st_v)) ||
        (r = put((w_begin & 1) ? ctx->w_live0.p : ctx->w_live1.p, c.live)) ||
        (r = put((w_begin & 1) ? ctx->w_carry0.p : ctx->w_carry1.p, c.carry)) ||
        (r = put((w_begin & 1) ? ctx->w_pool_r0.p : ctx->w_pool_r1.p, c.pool_r)) ||
        (r = put((w_begin & 1) ? ctx->w_pool_v0.p : ctx->w_pool_v1.p, c.pool_v)) ||
        (r = put(ctx->d_heads.p, c.heads)))
        return r;
    (void)F;
    // counts the first window reads: survivors, carries, and an empty promotion list
    uint32_t *cnt = reinterpret_cast<uint32_t *>(ctx->p_small + 13);
    cnt[0] = (uint32_t)c.live.size();
    cnt[1] = (uint32_t)c.carry.size();
    CU(cudaMemcpyAsync(ctx->w_cnt32.p + wp, cnt + 0, 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ctx->w_cnt32.p + 2 * (size_t)nw + wp, cnt + 1, 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(ctx->w_cnt32.p + nw + wp, 0, 4, s));
    CU(cudaMemsetAsync(prom_total, 0, 4, s));
    const uint32_t cyc = w_begin * c.W;
    size_t off = 0;
    for (size_t d = 0; d < ctx->designs.size(); ++d) {
        Design *D = ctx->designs[d];
        if (cyc <= D->T && D->n_net)
            CU(cudaMemcpyAsync(D->d_rows.p + (size_t)(cyc - 1) * D->n_net, c.rows.data() + off,
                               (size_t)D->n_net * 8, cudaMemcpyHostToDevice, s));
        off += D->n_net;
    }
    return RTLFS_OK;
}

// Checkpoint wire format: a header, per-design (T, n_net), then the arrays in a fixed order.
constexpr char CK_MAGIC[8] = {'R', 'T', 'L', 'F', 'S', 'C', 'K', '1'};
struct CkHeader {
    char magic[8];
    uint32_t n_designs, F, W, window, nodrop, n_live, n_carry, lcap;
    uint64_t pool_top, n_rows;
};

template <typename Fn>
void ck_fields(rtlfs_ctx::Checkpoint &c, Fn fn) {
    fn(c.T); fn(c.n_net); fn(c.det); fn(c.cycle); fn(c.port); fn(c.load); fn(c.mism); fn(c.st_nreg);
    fn(c.st_r); fn(c.st_v); fn(c.live); fn(c.carry); fn(c.pool_r); fn(c.pool_v); fn(c.heads); fn(c.rows);
}

}  // namespace

extern "C" {

int rtlfs_create(rtlfs_ctx **out, int device) {
    rtlfs_ctx *ctx = nullptr;
    if (!out) return RTLFS_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return RTLFS_E_ARG;
    ctx = new rtlfs_ctx();
    ctx->device = device;
    int rc = RTLFS_OK;
    auto init = [&]() -> int {
        CU(cudaSetDevice(device));
        CU(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device));
        CU(cudaStreamCreateWithFlags(&ctx->s_main, cudaStreamNonBlocking));
        CU(cudaStreamCreateWithFlags(&ctx->s_heavy, cudaStreamNonBlocking));
        // the good trace of the next window gates every fault of that window: its CTAs
        // take free SMs before pending light or heavy CTAs
        int lo_prio = 0, hi_prio = 0;
        CU(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
        CU(cudaStreamCreateWithPriority(&ctx->s_good, cudaStreamNonBlocking, hi_prio));
        for (auto &x : ctx->s_gaux) CU(cudaStreamCreateWithPriority(&x, cudaStreamNonBlocking, hi_prio));
        CU(cudaEventCreateWithFlags(&ctx->ev_gfork, cudaEventDisableTiming));
        for (auto &e : ctx->ev_gjoin) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&ctx->ev_wg, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&ctx->ev_wl, cudaEventDisableTiming));
        for (auto &e : ctx->ev) CU(cudaEventCreate(&e));
        for (auto &e : ctx->ev_graph) CU(cudaEventCreate(&e));
        CU(cudaEventCreate(&ctx->ev_gend));
        CU(ctx->d_counters.reserve(4));
        CU(ctx->d_heads.reserve(8));
        CU(cudaMallocHost(&ctx->p_small, 16 * sizeof(unsigned long long)));
        return RTLFS_OK;
    };
    rc = init();
    if (rc != RTLFS_OK) { rtlfs_destroy(ctx); return rc; }
    *out = ctx;
    return RTLFS_OK;
}

void rtlfs_destroy(rtlfs_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->s_main) cudaStreamSynchronize(ctx->s_main);
    if (ctx->s_heavy) cudaStreamSynchronize(ctx->s_heavy);
    for (Design *D : ctx->designs) delete D;
    ctx->designs.clear();
    for (auto &e : ctx->ev) if (e) cudaEventDestroy(e);
    for (auto &e : ctx->ev_graph) if (e) cudaEventDestroy(e);
    if (ctx->ev_gend) cudaEventDestroy(ctx->ev_gend);
    for (auto &e : ctx->ev_win) if (e) cudaEventDestroy(e);
    if (ctx->ev_wg) cudaEventDestroy(ctx->ev_wg);
    if (ctx->ev_wl) cudaEventDestroy(ctx->ev_wl);
    for (auto &x : ctx->s_gaux) if (x) { cudaStreamSynchronize(x); cudaStreamDestroy(x); }
    if (ctx->ev_gfork) cudaEventDestroy(ctx->ev_gfork);
    for (auto &e : ctx->ev_gjoin) if (e) cudaEventDestroy(e);
    if (ctx->s_good) { cudaStreamSynchronize(ctx->s_good); cudaStreamDestroy(ctx->s_good); }
    if (ctx->s_main) cudaStreamDestroy(ctx->s_main);
    if (ctx->s_heavy) cudaStreamDestroy(ctx->s_heavy);
    if (ctx->p_cycle) { cudaFreeHost(ctx->p_cycle); cudaFreeHost(ctx->p_port); cudaFreeHost(ctx->p_det); cudaFreeHost(ctx->p_load); }
    if (ctx->p_small) cudaFreeHost(ctx->p_small);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    delete ctx;
}

const char *rtlfs_last_error(const rtlfs_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int rtlfs_load_design(rtlfs_ctx *ctx, const rtlfs_node *nodes, uint32_t n_nodes,
                      const rtlfs_reg *regs, uint32_t n_regs, const uint8_t *input_widths,
                      uint32_t n_inputs, const uint32_t *output_nets, uint32_t n_outputs,
                      uint32_t *design_id) {
    if (!ctx) return RTLFS_E_ARG;
    if (!design_id || (n_nodes && !nodes) || (n_regs && !regs) || (n_inputs && !input_widths) ||
        (n_outputs && !output_nets))
        return fail(ctx, RTLFS_E_ARG, "null array with nonzero size");
    if (ctx->designs.size() >= 65535) return fail(ctx, RTLFS_E_ARG, "too many designs");
    CU(cudaSetDevice(ctx->device));
    Design *D = new Design();
    int rc = build_design(ctx, *D, nodes, n_nodes, regs, n_regs, input_widths, n_inputs,
                          output_nets, n_outputs);
    if (rc == RTLFS_OK) rc = upload_design(ctx, *D);
    if (rc != RTLFS_OK) { delete D; return rc; }
    *design_id = (uint32_t)ctx->designs.size();
    ctx->designs.push_back(D);
    ctx->faults_dirty = true;
    ctx->err.clear();
    return RTLFS_OK;
}

int rtlfs_set_stimulus(rtlfs_ctx *ctx, uint32_t design_id, const uint64_t *inputs, uint32_t n_cycles) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size()) return fail(ctx, RTLFS_E_ARG, "bad design id");
    Design &D = *ctx->designs[design_id];
    if (n_cycles < 1 || n_cycles > (1u << 21)) return fail(ctx, RTLFS_E_ARG, "n_cycles out of range (1..2^21)");
    if (D.I && !inputs) return fail(ctx, RTLFS_E_ARG, "null inputs");
    if ((size_t)D.n_net * n_cycles > (1ull << 36)) return fail(ctx, RTLFS_E_ARG, "trace too large");
    CU(cudaSetDevice(ctx->device));
    const size_t cells = (size_t)n_cycles * D.I;
    CU(D.d_stim.reserve(cells));
    if (cells) CU(cudaMemcpy(D.d_stim.p, inputs, cells * sizeof(uint64_t), cudaMemcpyHostToDevice));
    D.T = n_cycles;
    D.has_stim = true;
    D.trace_valid = false;
    ctx->ck.valid = false;
    ctx->err.clear();
    return RTLFS_OK;
}

int rtlfs_set_faults(rtlfs_ctx *ctx, uint32_t design_id, const rtlfs_fault *faults, uint32_t n_faults) {
    return set_faults_impl(ctx, design_id, n_faults, faults == nullptr,
                           [&](uint32_t i, uint32_t *net, uint32_t *bit, uint32_t *kind, uint32_t *cycle) {
                               const rtlfs_fault &x = faults[i];
                               if (x.stuck > 1) return fail(ctx, RTLFS_E_ARG, "fault %u: stuck value must be 0 or 1", i);
                               *net = x.net; *bit = x.bit; *kind = x.stuck; *cycle = 0;
                               return (int)RTLFS_OK;
                           });
}

int rtlfs_set_faults_ex(rtlfs_ctx *ctx, uint32_t design_id, const rtlfs_fault_ex *faults, uint32_t n_faults) {
    return set_faults_impl(ctx, design_id, n_faults, faults == nullptr,
                           [&](uint32_t i, uint32_t *net, uint32_t *bit, uint32_t *kind, uint32_t *cycle) {
                               const rtlfs_fault_ex &x = faults[i];
                               *net = x.net; *bit = x.bit; *kind = x.kind; *cycle = x.cycle;
                               return (int)RTLFS_OK;
                           });
}

int rtlfs_mismatch_counts(rtlfs_ctx *ctx, uint32_t design_id, uint32_t *out) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size()) return fail(ctx, RTLFS_E_ARG, "bad design id");
    if (!ctx->mism_valid || ctx->faults_dirty || ctx->f_first.size() != ctx->designs.size() + 1)
        return fail(ctx, RTLFS_E_STATE, "no no-drop run since the fault lists were set");
    const uint32_t first = ctx->f_first[design_id], n = ctx->f_first[design_id + 1] - first;
    if (n && !out) return fail(ctx, RTLFS_E_ARG, "null output");
    CU(cudaSetDevice(ctx->device));
    if (n) CU(cudaMemcpy(out, ctx->d_mism.p + first, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return RTLFS_OK;
}

static int run_good_only(rtlfs_ctx *ctx) {
    for (Design *D : ctx->designs)
        if (!D->has_stim) return fail(ctx, RTLFS_E_STATE, "a design has no stimulus");
    int rc = enqueue_good(ctx);
    if (rc != RTLFS_OK) return rc;
    uint32_t err = 0;
    CU(cudaMemcpyAsync(&err, ctx->d_err.p, sizeof(err), cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));
    if (err & 1u) return fail(ctx, RTLFS_E_CUDA, "good-trace staging did not complete (bounded wait ran out)");
    if (err & 4u) return fail(ctx, RTLFS_E_CUDA, "a cluster good-trace launch did not run in its clusters");
    for (Design *D : ctx->designs) D->trace_valid = true;
    return RTLFS_OK;
}

int rtlfs_run(rtlfs_ctx *ctx, const rtlfs_run_opts *opts_in, rtlfs_result *const *out,
              uint64_t *const *out_load) {
    if (!ctx) return RTLFS_E_ARG;
    if (ctx->designs.empty()) return fail(ctx, RTLFS_E_STATE, "no design loaded");
    if (!out) return fail(ctx, RTLFS_E_ARG, "null result array");
    for (Design *D : ctx->designs)
        if (!D->has_stim) return fail(ctx, RTLFS_E_STATE, "a design has no stimulus");
    rtlfs_run_opts o{};
    o.scheduler = RTLFS_SCHED_HEURISTIC;
    o.heavy_frac = -1.f;
    if (opts_in) o = *opts_in;
    const int lblock = o.light_block > 0 ? o.light_block : 128;
    const int lcap = o.light_cap > 0 ? o.light_cap - 1 : 1;
    if (lcap > 2) return fail(ctx, RTLFS_E_ARG, "light_cap must be 0..3");
    const int hblock = o.heavy_block > 0 ? o.heavy_block : 32;
    if (lblock < 32 || lblock > 256 || (lblock & 31)) return fail(ctx, RTLFS_E_ARG, "light_block must be a multiple of 32 in 32..256");
    if (hblock < 32 || hblock > 1024 || (hblock & 31)) return fail(ctx, RTLFS_E_ARG, "heavy_block must be a multiple of 32 in 32..1024");
    if (o.good_cluster < 0 || o.good_cluster > (int)CL_MAX || (o.good_cluster > 1 && (o.good_cluster & (o.good_cluster - 1))))
        return fail(ctx, RTLFS_E_ARG, "good_cluster must be 0, 1, 2, 4, 8 or 16");
    ctx->good_cluster = (uint32_t)o.good_cluster;
    if (o.good_staging < 0 || o.good_staging > 1) return fail(ctx, RTLFS_E_ARG, "good_staging must be 0 or 1");
    if (o.good_first < 0 || o.good_first > 1) return fail(ctx, RTLFS_E_ARG, "good_first must be 0 or 1");
    if (o.order_classes < 0 || o.order_classes > 64 || (o.order_classes & (o.order_classes - 1)))
        return fail(ctx, RTLFS_E_ARG, "order_classes must be 0 or a power of two up to 64");
    ctx->good_staging = (uint32_t)o.good_staging;
    CU(cudaSetDevice(ctx->device));
    const auto t_host0 = std::chrono::steady_clock::now();
    int rc = build_faults(ctx);
    if (rc != RTLFS_OK) return rc;
    const uint32_t F = ctx->F;

    // Schedule. PLAIN: fault-list order, nothing pre-assigned to the heavy kernel (order
    // uploaded from the host). HEURISTIC / MLP: computed on the device after the good
    // trace -- features, score (static cone x toggle rate, or the predictor), bucket sort
    // by descending score; the top heavy_frac of the faults start in the heavy kernel.
    const bool dev_sched = o.scheduler != RTLFS_SCHED_PLAIN && F > 0;
    const bool use_mlp = o.scheduler == RTLFS_SCHED_MLP && ctx->has_weights;
    const float hf = dev_sched ? (o.heavy_frac >= 0.f ? std::min(o.heavy_frac, 1.f) : 0.0f) : 0.f;
    const uint32_t n_heavy = (uint32_t)(hf * F);
    if (!dev_sched) {
        std::vector<uint32_t> order(F);
        for (uint32_t i = 0; i < F; ++i) order[i] = i;
        CU(ctx->d_order.upload(order));
    } else {
        rc = ensure_sched_buffers(ctx);
        if (rc != RTLFS_OK) return rc;
    }
    if (o.heavy_form < 0 || o.heavy_form > 3) return fail(ctx, RTLFS_E_ARG, "heavy_form must be 0, 1, 2 or 3");
    rc = ensure_heavy_scratch(ctx, hblock, o.heavy_ctas, o.heavy_form);
    if (rc != RTLFS_OK) return rc;
    rc = prepare_good(ctx);
    if (rc != RTLFS_OK) return rc;
    uint32_t *cinit = reinterpret_cast<uint32_t *>(ctx->p_small + 10);
    cinit[0] = n_heavy; cinit[1] = 0; cinit[2] = 0; cinit[3] = 0;
    const auto t_host1 = std::chrono::steady_clock::now();

    DevFaults f = dev_faults(ctx);
    const bool nodrop = o.no_drop != 0;
    if (nodrop) f.mism = ctx->d_mism.p;
    Queues ql{};
    ql.light_order = ctx->d_order.p + n_heavy;
    ql.n_light = F - n_heavy;
    ql.light_head = ctx->d_heads.p + 0;
    ql.heavy_items = ctx->d_prom_items.p;
    ql.heavy_count = ctx->d_counters.p + 1;
    ql.heavy_head = ctx->d_heads.p + 2;
    ql.heavy_cap = F;
    ql.budget_hit = ctx->d_heads.p + 3;
    ql.fault_budget = o.fault_budget;
    ql.counters = ctx->d_heads.p + 4;
    Queues qi = ql;
    qi.heavy_items = ctx->d_init_items.p;
    qi.heavy_count = ctx->d_counters.p + 0;
    qi.heavy_head = ctx->d_heads.p + 1;
    qi.counters = ctx->d_heads.p + 6;
    Queues qp = ql;
    qp.counters = ctx->d_heads.p + 6;
    const int per_sm = light_max_blocks_per_sm(lcap, lblock, o.window > 0);
    if (per_sm < 1) return fail(ctx, RTLFS_E_ARG, "light kernel cannot be resident");
    const int lgrid = (int)std::max<int64_t>(1, std::min<int64_t>((ql.n_light + lblock - 1) / lblock,
                                                                   (int64_t)per_sm * ctx->n_sm));
    const int hgrid = (int)ctx->heavy_grid;
    const int64_t lgrid_cap = (int64_t)per_sm * ctx->n_sm;
    HeavyScratch hs = heavy_view(ctx);
    cudaEvent_t *ev = ctx->ev;
    uint32_t launches = 0;

    // Windowed campaign: every live fault advances through the same window of cycles.
    uint32_t Tmax = 0, max_net = 0;
    for (Design *D : ctx->designs) { Tmax = std::max(Tmax, D->T); max_net = std::max(max_net, D->n_net); }
    const uint32_t W = o.window > 0 ? (uint32_t)o.window : 0;
    const uint32_t nw = W ? (Tmax + W - 1) / W : 0;
    if (W) {
        const size_t Fn = std::max<size_t>(F, 1);
        uint32_t mr = 1;
        for (Design *D : ctx->designs) mr = std::max(mr, D->R);
        CU(ctx->w_st_nreg.reserve(Fn));
        CU(ctx->w_st_r.reserve(Fn * LIGHT_KR));
        CU(ctx->w_st_v.reserve(Fn * LIGHT_KR));
        CU(ctx->w_live0.reserve(Fn));
        CU(ctx->w_live1.reserve(Fn));
        CU(ctx->w_carry0.reserve(Fn));
        CU(ctx->w_carry1.reserve(Fn));
        const uint64_t pool_cap = std::min<uint64_t>((uint64_t)Fn * mr, (uint64_t)16 << 20);
        CU(ctx->w_pool_r0.reserve(pool_cap));
        CU(ctx->w_pool_r1.reserve(pool_cap));
        CU(ctx->w_pool_v0.reserve(pool_cap));
        CU(ctx->w_pool_v1.reserve(pool_cap));
        ctx->w_pool_cap = pool_cap;
        CU(ctx->w_cnt32.reserve(3 * (size_t)nw + 4));   // n_live, prom_end, n_carry | prom_total, n_light, zero
        CU(ctx->w_cnt64.reserve(3 * (size_t)nw + 1));   // pool_top, light head, heavy head
        while (ctx->ev_win.size() < 4 * (size_t)nw) {
            cudaEvent_t e;
            CU(cudaEventCreate(&e));
            ctx->ev_win.push_back(e);
        }
        uint32_t *ci = reinterpret_cast<uint32_t *>(ctx->p_small + 10);
        ci[0] = n_heavy;        // prom_total starts after the initial heavy items
        ci[1] = F - n_heavy;    // faults in the first light window
        ci[2] = 0;
        ci[3] = 0;
    }
    // Checkpoint options: the campaign runs windows [w_begin, w_end).
    const bool stopping = o.stop_cycle > 0, resuming = o.resume != 0;
    if (o.stop_cycle < 0) return fail(ctx, RTLFS_E_ARG, "stop_cycle must not be negative");
    if ((stopping || resuming) && (!W || o.use_graph))
        return fail(ctx, RTLFS_E_ARG, "stop_cycle and resume need the windowed form without graph replay");
    if (stopping && ((uint32_t)o.stop_cycle % W != 0 || (uint32_t)o.stop_cycle >= Tmax))
        return fail(ctx, RTLFS_E_ARG, "stop_cycle must be a multiple of window below the longest stimulus");
    const uint32_t w_end = stopping ? (uint32_t)o.stop_cycle / W : nw;
    uint32_t w_begin = 0;
    if (resuming) {
        int rc2 = checkpoint_matches(ctx, ctx->ck, W, nodrop, lcap);
        if (rc2 != RTLFS_OK) return rc2;
        w_begin = ctx->ck.window;
        if (w_begin >= w_end) return fail(ctx, RTLFS_E_ARG, "stop_cycle is not after the checkpoint");
        if (ctx->ck.pool_r.size() > ctx->w_pool_cap) return fail(ctx, RTLFS_E_ARG, "checkpoint pool exceeds capacity");
    }
    // Per-window kernel times: plain event records, or, while the campaign is captured into
    // a graph, event-record nodes of the graph itself (external records), which keep their
    // timestamps on every replay.
    const bool timed_windows = W != 0;
    const bool good_first = W && o.good_first && !stopping && !resuming;
    auto rec_time = [&](cudaEvent_t e, cudaStream_t s) -> cudaError_t {
        return o.use_graph ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
    };
    // Activation bitplane: built after the good trace (per window when windows are whole
    // multiples of 64 cycles); otherwise the kernels scan the good trace.
    const bool use_act = F > 0 && (W == 0 || W % 64 == 0);
    const uint32_t act_stride = (Tmax + 63) / 64;
    if (use_act) {
        CU(ctx->d_act.reserve((size_t)F * act_stride));
        f.act = ctx->d_act.p;
        f.act_stride = act_stride;
    }

    // Windowed stream work (good trace on s_good, light on s_main, heavy on s_heavy).
    auto enqueue_windowed = [&]() -> int {
        launches = 0;
        uint32_t *c32 = ctx->w_cnt32.p;
        unsigned long long *c64 = ctx->w_cnt64.p;
        uint32_t *prom_total = c32 + 3 * nw, *n_light0 = c32 + 3 * nw + 1, *zero = c32 + 3 * nw + 2;
        CU(cudaEventRecord(ev[0], ctx->s_main));
        CU(cudaMemsetAsync(ctx->d_heads.p, 0, 8 * sizeof(unsigned long long), ctx->s_main));
        if (nodrop && F && !resuming) {   // results are written at first detection; the rest stay undetected
            CU(cudaMemsetAsync(ctx->d_mism.p, 0, (size_t)F * sizeof(uint32_t), ctx->s_main));
            CU(cudaMemsetAsync(ctx->d_det.p, 0, (size_t)F, ctx->s_main));
            CU(cudaMemsetAsync(ctx->d_cycle.p, 0xFF, (size_t)F * sizeof(int32_t), ctx->s_main));
            CU(cudaMemsetAsync(ctx->d_port.p, 0xFF, (size_t)F * sizeof(int32_t), ctx->s_main));
        }
        CU(cudaMemsetAsync(c32, 0, (3 * (size_t)nw + 4) * sizeof(uint32_t), ctx->s_main));
        CU(cudaMemsetAsync(c64, 0, (3 * (size_t)nw + 1) * sizeof(unsigned long long), ctx->s_main));
        CU(cudaMemcpyAsync(prom_total, ctx->p_small + 10, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->s_main));
        CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(uint32_t), ctx->s_main));
        if (F && !resuming) {
            CU(cudaMemsetAsync(ctx->d_load.p, 0, (size_t)F * sizeof(uint64_t), ctx->s_main));
            CU(cudaMemsetAsync(ctx->w_st_nreg.p, 0, F, ctx->s_main));
        }
        if (resuming) {
            int r4 = restore_checkpoint(ctx, nw, w_begin, prom_total);
            if (r4 != RTLFS_OK) return r4;
        }
        CU(cudaEventRecord(ctx->ev_wl, ctx->s_main));
        CU(cudaStreamWaitEvent(ctx->s_good, ctx->ev_wl, 0));
        CU(cudaStreamWaitEvent(ctx->s_heavy, ctx->ev_wl, 0));
        const uint32_t lblocks = (uint32_t)std::max<int64_t>(1, std::min<int64_t>(((int64_t)F + lblock - 1) / lblock,
                                                                                  (int64_t)lgrid_cap));
        // The scheduler of the first window reads the toggle rates of the first TOGGLE_CYCLES
        // cycles, so the good trace runs that far ahead before the first light kernel.
        const uint32_t w_sched = dev_sched && w_begin == 0 ? (std::min(TOGGLE_CYCLES, Tmax) + W - 1) / W : 0;
        uint32_t g_next = w_begin;   // next window whose good trace is to be enqueued
        if (good_first) {   // every cycle's good trace first: one launch per design list
            int r3 = launch_good_lists(ctx, ctx->s_good, 0, Tmax, &launches);
            if (r3 != RTLFS_OK) return r3;
            for (Design *D : ctx->designs) {
                CU(launch_transpose(D->d_gcol.p, D->d_rows.p, D->n_net, D->T, ctx->s_good));
                ++launches;
            }
            if (use_act) { CU(launch_activation(ctx->d_designs.p, f, ctx->d_act.p, 0, Tmax, ctx->s_good)); ++launches; }
            CU(cudaEventRecord(ev[1], ctx->s_good));
            g_next = nw;
        }
        for (uint32_t w = w_begin; w < w_end; ++w) {
            const uint32_t t0 = w * W, t1 = std::min(t0 + W, Tmax);
            // good trace of the window (and of the windows the scheduler needs)
            for (; g_next <= std::max(w, w_sched ? w_sched - 1 : 0u) && g_next < nw; ++g_next) {
                const uint32_t g0 = g_next * W, g1 = std::min(g0 + W, Tmax);
                int r3 = launch_good_lists(ctx, ctx->s_good, g0, g1, &launches);
                if (r3 != RTLFS_OK) return r3;
                CU(launch_transpose_window(ctx->d_designs.p, (uint32_t)ctx->designs.size(), max_net, g0, g1, ctx->s_good));
                ++launches;
                if (use_act) { CU(launch_activation(ctx->d_designs.p, f, ctx->d_act.p, g0, g1, ctx->s_good)); ++launches; }
                if (g_next == w_begin) CU(cudaEventRecord(ev[1], ctx->s_good));
            }
            CU(cudaEventRecord(ctx->ev_wg, ctx->s_good));
            // light kernel of the window (after the scheduler for the first one)
            CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_wg, 0));
            if (w == 0) {
                if (dev_sched) {
                    CU(launch_features(ctx->d_designs.p, f, ctx->d_static_ptrs.p, ctx->d_X.p, ctx->d_heur.p,
                                       ctx->s_main, TOGGLE_CYCLES));
                    const float *score = ctx->d_heur.p;
                    if (use_mlp) {
                        CU(launch_mlp_forward(ctx->d_wb.p, ctx->d_X.p, F, ctx->d_pred.p, ctx->s_main));
                        score = ctx->d_pred.p;
                        ++launches;
                    }
                    CU(launch_order(score, F, ctx->d_mm.p, ctx->d_hist.p, ctx->d_order.p, n_heavy,
                                    ctx->d_prom_items.p, ctx->s_main, (uint32_t)o.order_classes));
                    launches += 6 + (n_heavy ? 1 : 0);
                }
                CU(cudaEventRecord(ev[6], ctx->s_main));
            }
            WinLight wl{};
            wl.live_in = w == 0 ? ctx->d_order.p + n_heavy : (w & 1 ? ctx->w_live0.p : ctx->w_live1.p);
            wl.n_live_in = w == 0 ? n_light0 : c32 + (w - 1);
            wl.reverse = w > 0;
            wl.live_out = (w & 1) ? ctx->w_live1.p : ctx->w_live0.p;
            wl.n_live_out = c32 + w;
            wl.head = c64 + nw + w;
            wl.prom = ctx->d_prom_items.p;
            wl.prom_total = prom_total;
            wl.prom_cap = F;
            wl.st_nreg = ctx->w_st_nreg.p;
            wl.st_r = ctx->w_st_r.p;
            wl.st_v = ctx->w_st_v.p;
            wl.F = F;
            wl.t0 = t0;
            wl.t1 = t1;
            wl.budget_hit = ctx->d_heads.p + 3;
            wl.fault_budget = o.fault_budget;
            wl.counters = ctx->d_heads.p + 4;
            if (timed_windows) CU(rec_time(ctx->ev_win[0 * nw + w], ctx->s_main));
            if (F) { CU(launch_light_window(ctx->d_designs.p, f, wl, lcap, lblock, (int)lblocks, ctx->s_main)); ++launches; }
            if (timed_windows) CU(rec_time(ctx->ev_win[1 * nw + w], ctx->s_main));
            CU(cudaMemcpyAsync(c32 + nw + w, prom_total, sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->s_main));
            CU(cudaEventRecord(ctx->ev_wl, ctx->s_main));
            // heavy kernel of the window: carried heavy faults plus this window's promotions
            CU(cudaStreamWaitEvent(ctx->s_heavy, ctx->ev_wl, 0));
            WinHeavy wh{};
            wh.carry_in = (w & 1) ? ctx->w_carry0.p : ctx->w_carry1.p;
            wh.n_carry_in = w == 0 ? zero : c32 + 2 * nw + (w - 1);
            wh.pool_r_in = (w & 1) ? ctx->w_pool_r0.p : ctx->w_pool_r1.p;
            wh.pool_v_in = (w & 1) ? ctx->w_pool_v0.p : ctx->w_pool_v1.p;
            wh.carry_out = (w & 1) ? ctx->w_carry1.p : ctx->w_carry0.p;
            wh.n_carry_out = c32 + 2 * nw + w;
            wh.pool_r_out = (w & 1) ? ctx->w_pool_r1.p : ctx->w_pool_r0.p;
            wh.pool_v_out = (w & 1) ? ctx->w_pool_v1.p : ctx->w_pool_v0.p;
            wh.pool_top_out = c64 + w;
            wh.pool_cap = ctx->w_pool_cap;
            wh.prom = ctx->d_prom_items.p;
            wh.prom_begin = w == 0 ? zero : c32 + nw + (w - 1);
            wh.prom_end = c32 + nw + w;
            wh.head = c64 + 2 * nw + w;
            wh.t0 = t0;
            wh.t1 = t1;
            wh.budget_hit = ctx->d_heads.p + 3;
            wh.fault_budget = o.fault_budget;
            wh.counters = ctx->d_heads.p + 6;
            wh.err = ctx->d_err.p;
            if (timed_windows) CU(rec_time(ctx->ev_win[2 * nw + w], ctx->s_heavy));
            CU(launch_heavy_window(ctx->d_designs.p, f, wh, hs, hblock, hgrid, ctx->s_heavy));
            ++launches;
            if (timed_windows) CU(rec_time(ctx->ev_win[3 * nw + w], ctx->s_heavy));
        }
        CU(cudaEventRecord(ev[2], ctx->s_main));
        if (o.use_graph) CU(rec_time(ctx->ev_gend, ctx->s_good));
        CU(cudaEventRecord(ev[3], ctx->s_good));
        CU(cudaStreamWaitEvent(ctx->s_main, ev[3], 0));
        CU(cudaEventRecord(ev[4], ctx->s_heavy));
        CU(cudaStreamWaitEvent(ctx->s_main, ev[4], 0));
        if (F) {
            CU(cudaMemcpyAsync(ctx->p_cycle, ctx->d_cycle.p, (size_t)F * 4, cudaMemcpyDeviceToHost, ctx->s_main));
            CU(cudaMemcpyAsync(ctx->p_port, ctx->d_port.p, (size_t)F * 4, cudaMemcpyDeviceToHost, ctx->s_main));
            CU(cudaMemcpyAsync(ctx->p_det, ctx->d_det.p, (size_t)F, cudaMemcpyDeviceToHost, ctx->s_main));
            CU(cudaMemcpyAsync(ctx->p_load, ctx->d_load.p, (size_t)F * 8, cudaMemcpyDeviceToHost, ctx->s_main));
        }
        CU(cudaMemcpyAsync(ctx->p_small, ctx->d_heads.p, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->s_main));
        // counts reported as in the unwindowed form: [0] initial heavy, [1] promoted
        CU(cudaMemcpyAsync(ctx->p_small + 8, prom_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaMemcpyAsync(ctx->p_small + 12, ctx->d_err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaEventRecord(ev[5], ctx->s_main));
        return RTLFS_OK;
    };

    // The campaign's stream work: no allocation, no synchronous copy, so that it can be
    // captured into a CUDA graph and replayed.
    auto enqueue = [&]() -> int {
        launches = 0;
        CU(cudaEventRecord(ev[0], ctx->s_main));
        CU(cudaMemsetAsync(ctx->d_heads.p, 0, 8 * sizeof(unsigned long long), ctx->s_main));
        CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(uint32_t), ctx->s_main));
        if (nodrop && F) {   // results are written at first detection; the rest stay undetected
            CU(cudaMemsetAsync(ctx->d_mism.p, 0, (size_t)F * sizeof(uint32_t), ctx->s_main));
            CU(cudaMemsetAsync(ctx->d_det.p, 0, (size_t)F, ctx->s_main));
            CU(cudaMemsetAsync(ctx->d_cycle.p, 0xFF, (size_t)F * sizeof(int32_t), ctx->s_main));
            CU(cudaMemsetAsync(ctx->d_port.p, 0xFF, (size_t)F * sizeof(int32_t), ctx->s_main));
        }
        CU(cudaMemcpyAsync(ctx->d_counters.p, cinit, 4 * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->s_main));
        if (F) CU(cudaMemsetAsync(ctx->d_load.p, 0, (size_t)F * sizeof(uint64_t), ctx->s_main));
        int r2 = launch_good(ctx, &launches);
        if (r2 != RTLFS_OK) return r2;
        if (use_act) { CU(launch_activation(ctx->d_designs.p, f, ctx->d_act.p, 0, Tmax, ctx->s_main)); ++launches; }
        CU(cudaEventRecord(ev[1], ctx->s_main));
        if (dev_sched) {
            CU(launch_features(ctx->d_designs.p, f, ctx->d_static_ptrs.p, ctx->d_X.p, ctx->d_heur.p, ctx->s_main));
            const float *score = ctx->d_heur.p;
            if (use_mlp) {
                CU(launch_mlp_forward(ctx->d_wb.p, ctx->d_X.p, F, ctx->d_pred.p, ctx->s_main));
                score = ctx->d_pred.p;
                ++launches;
            }
            CU(launch_order(score, F, ctx->d_mm.p, ctx->d_hist.p, ctx->d_order.p, n_heavy,
                            ctx->d_init_items.p, ctx->s_main, (uint32_t)o.order_classes));
            launches += 6 + (n_heavy ? 1 : 0);
        }
        CU(cudaEventRecord(ev[6], ctx->s_main));
        if (ql.n_light) { CU(launch_light(ctx->d_designs.p, f, ql, lcap, lblock, lgrid, ctx->s_main)); ++launches; }
        CU(cudaEventRecord(ev[2], ctx->s_main));
        CU(cudaStreamWaitEvent(ctx->s_heavy, ev[6], 0));
        if (n_heavy) { CU(launch_heavy(ctx->d_designs.p, f, qi, hs, hblock, hgrid, ctx->s_heavy)); ++launches; }
        CU(cudaStreamWaitEvent(ctx->s_heavy, ev[2], 0));
        CU(cudaEventRecord(ev[3], ctx->s_heavy));
        CU(launch_heavy(ctx->d_designs.p, f, qp, hs, hblock, hgrid, ctx->s_heavy));
        ++launches;
        CU(cudaEventRecord(ev[4], ctx->s_heavy));
        CU(cudaStreamWaitEvent(ctx->s_main, ev[4], 0));
        if (F) {
            CU(cudaMemcpyAsync(ctx->p_cycle, ctx->d_cycle.p, (size_t)F * 4, cudaMemcpyDeviceToHost, ctx->s_main));
            CU(cudaMemcpyAsync(ctx->p_port, ctx->d_port.p, (size_t)F * 4, cudaMemcpyDeviceToHost, ctx->s_main));
            CU(cudaMemcpyAsync(ctx->p_det, ctx->d_det.p, (size_t)F, cudaMemcpyDeviceToHost, ctx->s_main));
            CU(cudaMemcpyAsync(ctx->p_load, ctx->d_load.p, (size_t)F * 8, cudaMemcpyDeviceToHost, ctx->s_main));
        }
        CU(cudaMemcpyAsync(ctx->p_small, ctx->d_heads.p, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaMemcpyAsync(ctx->p_small + 8, ctx->d_counters.p, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaMemcpyAsync(ctx->p_small + 12, ctx->d_err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaEventRecord(ev[5], ctx->s_main));
        return RTLFS_OK;
    };

    if (o.use_graph) {
        // Everything the captured work depends on by address or size.
        std::vector<uint64_t> key = {F, n_heavy, ql.n_light, (uint64_t)lcap, (uint64_t)lblock,
                                     (uint64_t)lgrid, (uint64_t)hblock, (uint64_t)hgrid,
                                     (uint64_t)dev_sched, (uint64_t)use_mlp, o.fault_budget, W,
                                     (uint64_t)nodrop, (uint64_t)good_first, (uint64_t)o.order_classes};
        const void *ptrs[] = {ctx->d_designs.p, ctx->d_list_smem.p, ctx->d_list_glob.p, ctx->d_order.p, ctx->d_err.p, ctx->h_gbm.p,
                              ctx->d_init_items.p, ctx->d_prom_items.p, ctx->d_heads.p, ctx->d_counters.p,
                              ctx->d_load.p, ctx->d_cycle.p, ctx->d_port.p, ctx->d_det.p, ctx->d_site.p,
                              ctx->d_bit.p, ctx->d_val.p, ctx->d_fdesign.p, ctx->p_cycle, ctx->p_port,
                              ctx->p_det, ctx->p_load, ctx->h_fval.p, ctx->h_stamp.p, ctx->h_regr.p, ctx->h_regv.p,
                              ctx->d_X.p, ctx->d_heur.p, ctx->d_pred.p, ctx->d_mm.p, ctx->d_hist.p,
                              ctx->d_wb.p, ctx->d_static_ptrs.p, ctx->w_st_nreg.p, ctx->w_st_r.p,
                              ctx->w_st_v.p, ctx->w_live0.p, ctx->w_live1.p, ctx->w_cnt32.p, ctx->w_cnt64.p,
                              ctx->w_carry0.p, ctx->w_carry1.p, ctx->w_pool_r0.p, ctx->w_pool_r1.p,
                              ctx->d_fport.p, ctx->d_ft0.p, ctx->d_mism.p,
                              ctx->w_pool_v0.p, ctx->w_pool_v1.p, ctx->d_act.p};
        for (const void *q : ptrs) key.push_back((uint64_t)(uintptr_t)q);
        const GoodLaunch &g = ctx->gl;
        key.insert(key.end(), {g.n_smem, g.n_glob, g.max_net_s, g.max_reg_s, g.max_ch_s, g.max_ch_g,
                               ctx->hs_net, ctx->hs_reg, ctx->hs_node, ctx->hs_lv, (uint64_t)ctx->heavy_exact, (uint64_t)ctx->heavy_gbm,
                               (uint64_t)ctx->good_staging});
        for (int lc = 1; lc < 5; ++lc)
            key.insert(key.end(), {(uint64_t)g.n_cl[lc], (uint64_t)g.smem_cl[lc],
                                   (uint64_t)(uintptr_t)ctx->d_list_cl[lc].p});
        for (Design *D : ctx->designs)
            key.insert(key.end(), {(uint64_t)(uintptr_t)D->d_rows.p, (uint64_t)(uintptr_t)D->d_gcol.p,
                                   D->n_net, D->T});
        if (!ctx->graph_exec || key != ctx->graph_key) {
            if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(ctx->s_main, cudaStreamCaptureModeRelaxed));
            int r2 = W ? enqueue_windowed() : enqueue();
            cudaError_t ec = cudaStreamEndCapture(ctx->s_main, &graph);
            if (r2 != RTLFS_OK) { if (graph) cudaGraphDestroy(graph); return r2; }
            CU(ec);
            cudaError_t ei = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            CU(ei);
            ctx->graph_key = key;
            ctx->graph_launches = launches;
        }
        launches = ctx->graph_launches;
        // events recorded inside a graph give no elapsed times: bracket the launch instead
        CU(cudaEventRecord(ctx->ev_graph[0], ctx->s_main));
        CU(cudaGraphLaunch(ctx->graph_exec, ctx->s_main));
        CU(cudaEventRecord(ctx->ev_graph[1], ctx->s_main));
    } else {
        rc = W ? enqueue_windowed() : enqueue();
        if (rc != RTLFS_OK) return rc;
    }
    CU(cudaStreamSynchronize(ctx->s_main));
    {
        const uint32_t kerr = *reinterpret_cast<const uint32_t *>(ctx->p_small + 12);
        if (kerr & 2u)
            return fail(ctx, RTLFS_E_NOMEM, "heavy register-diff pool overflowed; run with window = 0");
        if (kerr & 1u)
            return fail(ctx, RTLFS_E_CUDA, "good-trace staging did not complete (bounded wait ran out)");
        if (kerr & 4u)
            return fail(ctx, RTLFS_E_CUDA, "a cluster good-trace launch did not run in its clusters");
    }
    const unsigned long long *heads = ctx->p_small;
    const uint32_t *cnts = reinterpret_cast<const uint32_t *>(ctx->p_small + 8);
    for (Design *D : ctx->designs) D->trace_valid = !stopping && !resuming;
    ctx->mism_valid = nodrop && !stopping;
    std::vector<uint8_t> pending;
    if (stopping) {
        rc = take_checkpoint(ctx, nw, w_end, W, nodrop, lcap, &pending);
        if (rc != RTLFS_OK) return rc;
    } else {
        ctx->ck.valid = false;   // the campaign ran to its end
    }

    // Scatter results and counters.
    rtlfs_stats &st = ctx->stats;
    st = rtlfs_stats{};
    if (o.use_graph && W) {   // whole campaign, good-trace stream and each window kernel
        st.total_ms = ev_ms(ctx->ev_graph[0], ctx->ev_graph[1]);
        st.good_ms = ev_ms(ctx->ev_graph[0], ctx->ev_gend);
        st.prep_ms = std::chrono::duration<double, std::milli>(t_host1 - t_host0).count();
        for (uint32_t w = w_begin; w < w_end; ++w) {
            st.light_ms += ev_ms(ctx->ev_win[w], ctx->ev_win[nw + w]);
            st.heavy_ms += ev_ms(ctx->ev_win[2 * nw + w], ctx->ev_win[3 * nw + w]);
        }
    } else if (o.use_graph) {   // whole campaign only; per-phase times are not available
        st.total_ms = ev_ms(ctx->ev_graph[0], ctx->ev_graph[1]);
        st.prep_ms = std::chrono::duration<double, std::milli>(t_host1 - t_host0).count();
    } else if (W) {   // overlapped phases: each kernel's own summed duration
        st.total_ms = ev_ms(ev[0], ev[5]);
        st.good_ms = ev_ms(ev[0], ev[3]);
        st.prep_ms = std::chrono::duration<double, std::milli>(t_host1 - t_host0).count();
        for (uint32_t w = w_begin; w < w_end; ++w) {
            st.light_ms += ev_ms(ctx->ev_win[w], ctx->ev_win[nw + w]);
            st.heavy_ms += ev_ms(ctx->ev_win[2 * nw + w], ctx->ev_win[3 * nw + w]);
        }
        st.faulty_ms = ev_ms(ev[1], ev[4]);
    } else {
        st.total_ms = ev_ms(ev[0], ev[5]);
        st.good_ms = ev_ms(ev[0], ev[1]);
        st.prep_ms = ev_ms(ev[1], ev[6]) + std::chrono::duration<double, std::milli>(t_host1 - t_host0).count();
        st.faulty_ms = ev_ms(ev[6], ev[4]);
        st.light_ms = ev_ms(ev[6], ev[2]);
        st.heavy_ms = ev_ms(ev[3], ev[4]);
    }
    st.promoted = cnts[1];
    st.heavy_initial = cnts[0];
    if (W) {   // the windowed form reports the promotion list's total (initial + promoted)
        st.heavy_initial = resuming ? 0 : n_heavy;   // a resumed run's list holds promotions only
        st.promoted = cnts[0] - st.heavy_initial;
    }
    st.n_launches = launches;
    st.heavy_form = ctx->heavy_gbm ? 3u : ctx->heavy_exact ? 1u : 2u;
    st.light_evals = heads[4];
    st.light_fault_cycles = heads[5];
    st.heavy_evals = heads[6];
    st.heavy_fault_cycles = heads[7];
    for (size_t d = 0; d < ctx->designs.size(); ++d) {
        const Design &D = *ctx->designs[d];
        rtlfs_result *r = out[d];
        uint64_t *ld = out_load ? out_load[d] : nullptr;
        for (uint32_t i = ctx->f_first[d]; i < ctx->f_first[d + 1]; ++i) {
            const uint32_t k = i - ctx->f_first[d];
            const bool pend = !pending.empty() && pending[i];
            const uint8_t det = pend ? (uint8_t)RTLFS_PENDING : ctx->p_det[i];
            if (pend) { ctx->p_cycle[i] = -1; ctx->p_port[i] = -1; }
            if (r) {
                r[k].detected = det;
                r[k].cycle = ctx->p_cycle[i];
                r[k].port = ctx->p_port[i];
                r[k].reserved[0] = r[k].reserved[1] = r[k].reserved[2] = 0;
            }
            if (ld) ld[k] = ctx->p_load[i];
            st.node_evals += ctx->p_load[i];
            if (det == 1) st.fault_cycles += (uint64_t)ctx->p_cycle[i] + 1;
            else if (det == 0) st.fault_cycles += D.T;
        }
    }
    if (heads[3]) return fail(ctx, RTLFS_E_TIMEOUT, "%llu faults ran out of their work budget", heads[3]);
    ctx->err.clear();
    return RTLFS_OK;
}

int rtlfs_run_plain(rtlfs_ctx *ctx, rtlfs_result *const *out) {
    if (!ctx) return RTLFS_E_ARG;
    if (ctx->designs.empty()) return fail(ctx, RTLFS_E_STATE, "no design loaded");
    if (!out) return fail(ctx, RTLFS_E_ARG, "null result array");
    for (Design *D : ctx->designs)
        if (!D->has_stim) return fail(ctx, RTLFS_E_STATE, "a design has no stimulus");
    CU(cudaSetDevice(ctx->device));
    int rc = build_faults(ctx);
    if (rc != RTLFS_OK) return rc;
    cudaEvent_t *ev = ctx->ev;
    CU(cudaEventRecord(ev[0], ctx->s_main));
    rc = enqueue_good(ctx);
    if (rc != RTLFS_OK) return rc;
    CU(cudaEventRecord(ev[1], ctx->s_main));
    DevFaults f = dev_faults(ctx);
    ctx->mism_valid = false;
    uint32_t launches = 2 + (uint32_t)ctx->designs.size();
    // per-thread scratch, waves sized to a fixed memory budget
    const size_t budget = (size_t)8 << 30;
    DBuf<uint64_t> fval, regv;
    DBuf<uint32_t> stamp, qst, heap, regr;
    for (size_t d = 0; d < ctx->designs.size(); ++d) {
        Design &D = *ctx->designs[d];
        const uint32_t Fd = ctx->f_first[d + 1] - ctx->f_first[d];
        if (!Fd) continue;
        const size_t per = (size_t)D.n_net * 12 + (size_t)std::max<uint32_t>(D.N, 1) * 8 + (size_t)std::max<uint32_t>(D.R, 1) * 24;
        uint32_t wave = (uint32_t)std::max<size_t>(1, std::min<size_t>(Fd, budget / per));
        const uint32_t sn = D.n_net, snode = std::max<uint32_t>(D.N, 1), sreg = std::max<uint32_t>(D.R, 1);
        CU(fval.reserve((size_t)wave * sn));
        CU(stamp.reserve((size_t)wave * sn));
        CU(qst.reserve((size_t)wave * snode));
        CU(heap.reserve((size_t)wave * snode));
        CU(regr.reserve((size_t)wave * 2 * sreg));
        CU(regv.reserve((size_t)wave * 2 * sreg));
        for (uint32_t first = 0; first < Fd; first += wave) {
            const uint32_t cnt = std::min(wave, Fd - first);
            CU(cudaMemsetAsync(stamp.p, 0, (size_t)cnt * sn * 4, ctx->s_main));
            CU(cudaMemsetAsync(qst.p, 0, (size_t)cnt * snode * 4, ctx->s_main));
            CU(launch_plain(ctx->d_designs.p, (uint32_t)d, f, ctx->f_first[d] + first, cnt, fval.p,
                            stamp.p, qst.p, heap.p, regr.p, regv.p, sn, snode, sreg, ctx->s_main));
            ++launches;
        }
    }
    CU(cudaEventRecord(ev[4], ctx->s_main));
    const uint32_t F = ctx->F;
    if (F) {
        CU(cudaMemcpyAsync(ctx->p_cycle, ctx->d_cycle.p, (size_t)F * 4, cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaMemcpyAsync(ctx->p_port, ctx->d_port.p, (size_t)F * 4, cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaMemcpyAsync(ctx->p_det, ctx->d_det.p, (size_t)F, cudaMemcpyDeviceToHost, ctx->s_main));
        CU(cudaMemcpyAsync(ctx->p_load, ctx->d_load.p, (size_t)F * 8, cudaMemcpyDeviceToHost, ctx->s_main));
    }
    uint32_t gerr = 0;
    CU(cudaMemcpyAsync(&gerr, ctx->d_err.p, sizeof(gerr), cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaEventRecord(ev[5], ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));
    if (gerr & 1u) return fail(ctx, RTLFS_E_CUDA, "good-trace staging did not complete (bounded wait ran out)");
    if (gerr & 4u) return fail(ctx, RTLFS_E_CUDA, "a cluster good-trace launch did not run in its clusters");
    for (Design *D : ctx->designs) D->trace_valid = true;
    rtlfs_stats &st = ctx->stats;
    st = rtlfs_stats{};
    st.total_ms = ev_ms(ev[0], ev[5]);
    st.good_ms = ev_ms(ev[0], ev[1]);
    st.faulty_ms = ev_ms(ev[1], ev[4]);
    st.n_launches = launches;
    for (size_t d = 0; d < ctx->designs.size(); ++d) {
        const Design &D = *ctx->designs[d];
        for (uint32_t i = ctx->f_first[d]; i < ctx->f_first[d + 1]; ++i) {
            const uint32_t k = i - ctx->f_first[d];
            if (out[d]) {
                out[d][k].detected = ctx->p_det[i];
                out[d][k].cycle = ctx->p_cycle[i];
                out[d][k].port = ctx->p_port[i];
                out[d][k].reserved[0] = out[d][k].reserved[1] = out[d][k].reserved[2] = 0;
            }
            st.node_evals += ctx->p_load[i];
            st.fault_cycles += ctx->p_det[i] == 1 ? (uint64_t)ctx->p_cycle[i] + 1 : D.T;
        }
    }
    ctx->err.clear();
    return RTLFS_OK;
}

int rtlfs_get_stats(const rtlfs_ctx *ctx, rtlfs_stats *out) {
    if (!ctx || !out) return RTLFS_E_ARG;
    *out = ctx->stats;
    return RTLFS_OK;
}

int rtlfs_good_outputs(rtlfs_ctx *ctx, uint32_t design_id, uint64_t *out) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size() || !out) return fail(ctx, RTLFS_E_ARG, "bad design id or null out");
    Design &D = *ctx->designs[design_id];
    if (!D.has_stim) return fail(ctx, RTLFS_E_STATE, "design has no stimulus");
    CU(cudaSetDevice(ctx->device));
    if (!D.trace_valid) {
        int rc = run_good_only(ctx);
        if (rc != RTLFS_OK) return rc;
    }
    std::vector<uint64_t> col(D.T);
    for (uint32_t o = 0; o < D.O; ++o) {
        CU(cudaMemcpy(col.data(), D.d_gcol.p + (size_t)D.out_net[o] * D.T, (size_t)D.T * 8, cudaMemcpyDeviceToHost));
        for (uint32_t t = 0; t < D.T; ++t) out[(size_t)t * D.O + o] = col[t];
    }
    return RTLFS_OK;
}

int rtlfs_good_trace(rtlfs_ctx *ctx, uint32_t design_id, uint64_t *out) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size() || !out) return fail(ctx, RTLFS_E_ARG, "bad design id or null out");
    Design &D = *ctx->designs[design_id];
    if (!D.has_stim) return fail(ctx, RTLFS_E_STATE, "design has no stimulus");
    CU(cudaSetDevice(ctx->device));
    if (!D.trace_valid) {
        int rc = run_good_only(ctx);
        if (rc != RTLFS_OK) return rc;
    }
    std::vector<uint64_t> all((size_t)D.n_net * D.T);
    CU(cudaMemcpy(all.data(), D.d_gcol.p, all.size() * 8, cudaMemcpyDeviceToHost));
    for (uint32_t e = 0; e < D.n_net; ++e) {
        const uint64_t *col = all.data() + (size_t)D.ext2int[e] * D.T;
        for (uint32_t t = 0; t < D.T; ++t) out[(size_t)t * D.n_net + e] = col[t];
    }
    return RTLFS_OK;
}

int rtlfs_features(rtlfs_ctx *ctx, uint32_t design_id, float *out) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size() || !out) return fail(ctx, RTLFS_E_ARG, "bad design id or null out");
    CU(cudaSetDevice(ctx->device));
    int rc = build_faults(ctx);
    if (rc != RTLFS_OK) return rc;
    for (Design *D : ctx->designs)
        if (!D->trace_valid) { rc = run_good_only(ctx); if (rc != RTLFS_OK) return rc; break; }
    if (!ctx->F) return RTLFS_OK;
    rc = ensure_sched_buffers(ctx);
    if (rc != RTLFS_OK) return rc;
    CU(launch_features(ctx->d_designs.p, dev_faults(ctx), ctx->d_static_ptrs.p, ctx->d_X.p,
                       ctx->d_heur.p, ctx->s_main));
    const uint32_t a = ctx->f_first[design_id], b = ctx->f_first[design_id + 1];
    CU(cudaMemcpyAsync(out, ctx->d_X.p + (size_t)a * MLP_IN, (size_t)(b - a) * MLP_IN * sizeof(float),
                       cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));
    return RTLFS_OK;
}

int rtlfs_mlp_set_weights(rtlfs_ctx *ctx, const uint16_t *w) {
    if (!ctx) return RTLFS_E_ARG;
    if (!w) return fail(ctx, RTLFS_E_ARG, "null weights");
    CU(cudaSetDevice(ctx->device));
    int rc = ensure_mlp(ctx);
    if (rc != RTLFS_OK) return rc;
    std::vector<float> master(MLP_PARAMS);
    for (int i = 0; i < MLP_PARAMS; ++i) {
        const uint32_t bits = (uint32_t)w[i] << 16;
        std::memcpy(&master[i], &bits, 4);
    }
    CU(cudaMemcpy(ctx->d_wb.p, w, MLP_PARAMS * sizeof(uint16_t), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->d_master.p, master.data(), MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    CU(cudaMemset(ctx->d_m.p, 0, MLP_PARAMS * sizeof(float)));
    CU(cudaMemset(ctx->d_v.p, 0, MLP_PARAMS * sizeof(float)));
    CU(cudaMemset(ctx->d_grad.p, 0, MLP_PARAMS * sizeof(float)));
    ctx->adam_step = 0;
    ctx->has_weights = true;
    return RTLFS_OK;
}

int rtlfs_mlp_get_weights(rtlfs_ctx *ctx, uint16_t *w) {
    if (!ctx) return RTLFS_E_ARG;
    if (!w) return fail(ctx, RTLFS_E_ARG, "null weights");
    if (!ctx->has_weights) return fail(ctx, RTLFS_E_STATE, "no weights loaded");
    CU(cudaSetDevice(ctx->device));
    CU(cudaMemcpy(w, ctx->d_wb.p, MLP_PARAMS * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    return RTLFS_OK;
}

static int upload_samples(rtlfs_ctx *ctx, const float *X, const float *t, uint32_t n) {
    CU(ctx->d_tx.reserve((size_t)n * MLP_IN));
    CU(cudaMemcpy(ctx->d_tx.p, X, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice));
    if (t) {
        CU(ctx->d_ty.reserve(n));
        CU(cudaMemcpy(ctx->d_ty.p, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
    }
    return RTLFS_OK;
}

int rtlfs_mlp_forward(rtlfs_ctx *ctx, const float *X, uint32_t n, float *y) {
    if (!ctx) return RTLFS_E_ARG;
    if (!ctx->has_weights) return fail(ctx, RTLFS_E_STATE, "no weights loaded");
    if (n && (!X || !y)) return fail(ctx, RTLFS_E_ARG, "null array");
    if (!n) return RTLFS_OK;
    CU(cudaSetDevice(ctx->device));
    int rc = upload_samples(ctx, X, nullptr, n);
    if (rc != RTLFS_OK) return rc;
    CU(ctx->d_pred.reserve(n));
    CU(launch_mlp_forward(ctx->d_wb.p, ctx->d_tx.p, n, ctx->d_pred.p, ctx->s_main));
    CU(cudaMemcpyAsync(y, ctx->d_pred.p, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));
    return RTLFS_OK;
}

int rtlfs_mlp_grad(rtlfs_ctx *ctx, const float *X, const float *t, uint32_t n, float *loss,
                   float *grad) {
    if (!ctx) return RTLFS_E_ARG;
    if (!ctx->has_weights) return fail(ctx, RTLFS_E_STATE, "no weights loaded");
    if (!n || !X || !t || !loss || !grad) return fail(ctx, RTLFS_E_ARG, "null array or n = 0");
    CU(cudaSetDevice(ctx->device));
    int rc = upload_samples(ctx, X, t, n);
    if (rc != RTLFS_OK) return rc;
    CU(cudaMemsetAsync(ctx->d_grad.p, 0, MLP_PARAMS * sizeof(float), ctx->s_main));
    CU(cudaMemsetAsync(ctx->d_loss.p, 0, sizeof(float), ctx->s_main));
    CU(launch_mlp_grad(ctx->d_wb.p, ctx->d_tx.p, ctx->d_ty.p, n, ctx->d_grad.p, ctx->d_loss.p, ctx->s_main));
    float lsum = 0.f;
    CU(cudaMemcpyAsync(grad, ctx->d_grad.p, MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaMemcpyAsync(&lsum, ctx->d_loss.p, sizeof(float), cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));
    CU(cudaMemsetAsync(ctx->d_grad.p, 0, MLP_PARAMS * sizeof(float), ctx->s_main));
    *loss = lsum / (float)n;
    return RTLFS_OK;
}

int rtlfs_mlp_train(rtlfs_ctx *ctx, const float *X, const float *t, uint32_t n, uint32_t epochs,
                    uint32_t batch, float lr, float *final_loss) {
    if (!ctx) return RTLFS_E_ARG;
    if (!ctx->has_weights) return fail(ctx, RTLFS_E_STATE, "no weights loaded");
    if (!n || !X || !t || !batch || !(lr > 0.f)) return fail(ctx, RTLFS_E_ARG, "bad training arguments");
    CU(cudaSetDevice(ctx->device));
    int rc = upload_samples(ctx, X, t, n);
    if (rc != RTLFS_OK) return rc;
    float lsum = 0.f;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        CU(cudaMemsetAsync(ctx->d_loss.p, 0, sizeof(float), ctx->s_main));
        for (uint32_t s0 = 0; s0 < n; s0 += batch) {
            const uint32_t nb = std::min(batch, n - s0);
            CU(launch_mlp_grad(ctx->d_wb.p, ctx->d_tx.p + (size_t)s0 * MLP_IN, ctx->d_ty.p + s0, nb,
                               ctx->d_grad.p, ctx->d_loss.p, ctx->s_main));
            CU(launch_mlp_adam(ctx->d_master.p, ctx->d_wb.p, ctx->d_grad.p, ctx->d_m.p, ctx->d_v.p, lr,
                               0.9f, 0.999f, 1e-8f, ++ctx->adam_step, ctx->s_main));
        }
    }
    CU(cudaMemcpyAsync(&lsum, ctx->d_loss.p, sizeof(float), cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));
    if (final_loss) *final_loss = lsum / (float)n;
    return RTLFS_OK;
}

// Allocation-free variant of the plain form (see include/rtlfs.h): per-thread scratch in
// the library's static device array, faults and results in the caller's device buffers.
int rtlfs_fault_sim_static(rtlfs_ctx *ctx, uint32_t design_id, const rtlfs_fault *faults,
                           uint32_t n_faults, rtlfs_result *results, void *stream) {
    if (!ctx) return RTLFS_E_ARG;
    if (design_id >= ctx->designs.size()) return fail(ctx, RTLFS_E_ARG, "bad design id");
    if (n_faults && (!faults || !results)) return fail(ctx, RTLFS_E_ARG, "null faults or results");
    Design &D = *ctx->designs[design_id];
    if (!D.has_stim || !D.trace_valid)
        return fail(ctx, RTLFS_E_STATE, "the design's good trace is not current: call rtlfs_run or "
                                        "rtlfs_good_outputs after the last rtlfs_set_stimulus");
    if (!n_faults) return RTLFS_OK;
    CU(cudaSetDevice(ctx->device));
    void *arena_v = nullptr;
    CU(static_scratch_address(ctx->device, &arena_v));
    unsigned char *arena = (unsigned char *)arena_v;
    StaticLayout L{};
    L.sn = D.n_net;
    L.snode = std::max<uint32_t>(D.N, 1);
    L.sreg = std::max<uint32_t>(D.R, 1);
    L.per_thread = ((size_t)12 * L.sn + (size_t)8 * L.snode + (size_t)24 * L.sreg + 15) & ~(size_t)15;
    L.ext2int_off = 0;
    L.err_off = ((size_t)4 * D.n_net + 7) & ~(size_t)7;
    L.thread_off = (L.err_off + 8 + 255) & ~(size_t)255;
    if (L.thread_off + L.per_thread > STATIC_SCRATCH_BYTES)
        return fail(ctx, RTLFS_E_ARG, "design needs %zu bytes of scratch per fault; the static scratch "
                                      "holds %zu bytes", L.thread_off + L.per_thread,
                    (size_t)STATIC_SCRATCH_BYTES);
    const uint32_t wave = (uint32_t)std::min<size_t>(n_faults, (STATIC_SCRATCH_BYTES - L.thread_off) / L.per_thread);
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(arena + L.ext2int_off, D.ext2int.data(), (size_t)4 * D.n_net,
                       cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(arena + L.err_off, 0, 8, s));
    for (uint32_t first = 0; first < n_faults; first += wave) {
        const uint32_t cnt = std::min(wave, n_faults - first);
        // value stamps and queued stamps must start at zero for every thread of the wave
        CU(cudaMemsetAsync(arena + L.thread_off, 0, (size_t)cnt * L.per_thread, s));
        CU(launch_plain_static(ctx->d_designs.p, design_id, faults, results, first, cnt, arena, L, s));
    }
    uint32_t err = 0;
    CU(cudaMemcpyAsync(&err, arena + L.err_off, sizeof(err), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (err)
        return fail(ctx, RTLFS_E_ARG, "a fault's net, bit or stuck value is out of range (its result "
                                      "carries detected = 254)");
    ctx->err.clear();
    return RTLFS_OK;
}

int rtlfs_design_info(const rtlfs_ctx *ctx, uint32_t design_id, uint32_t *n_nets,
                      uint32_t *n_levels, uint32_t *n_fanout_edges) {
    if (!ctx || design_id >= ctx->designs.size()) return RTLFS_E_ARG;
    const Design &D = *ctx->designs[design_id];
    if (n_nets) *n_nets = D.n_net;
    if (n_levels) *n_levels = D.n_levels;
    if (n_fanout_edges) *n_fanout_edges = D.n_fo;
    return RTLFS_OK;
}


int rtlfs_checkpoint_size(rtlfs_ctx *ctx, uint64_t *bytes) {
    if (!ctx || !bytes) return RTLFS_E_ARG;
    if (!ctx->ck.valid) return fail(ctx, RTLFS_E_STATE, "no checkpoint held");
    uint64_t n = sizeof(CkHeader);
    ck_fields(ctx->ck, [&](auto &v) { n += v.size() * sizeof(v[0]); });
    *bytes = n;
    return RTLFS_OK;
}

int rtlfs_checkpoint_save(rtlfs_ctx *ctx, void *buf, uint64_t bytes) {
    uint64_t need = 0;
    int rc = rtlfs_checkpoint_size(ctx, &need);
    if (rc != RTLFS_OK) return rc;
    if (!buf || bytes < need) return fail(ctx, RTLFS_E_ARG, "checkpoint buffer too small (%llu bytes needed)", (unsigned long long)need);
    rtlfs_ctx::Checkpoint &c = ctx->ck;
    CkHeader h{};
    memcpy(h.magic, CK_MAGIC, 8);
    h.n_designs = (uint32_t)c.T.size(); h.F = c.F; h.W = c.W; h.window = c.window; h.nodrop = c.nodrop;
    h.lcap = c.lcap;
    h.n_live = (uint32_t)c.live.size(); h.n_carry = (uint32_t)c.carry.size();
    h.pool_top = c.pool_r.size(); h.n_rows = c.rows.size();
    unsigned char *p = static_cast<unsigned char *>(buf);
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    ck_fields(c, [&](auto &v) {
        if (!v.empty()) memcpy(p, v.data(), v.size() * sizeof(v[0]));
        p += v.size() * sizeof(v[0]);
    });
    ctx->err.clear();
    return RTLFS_OK;
}

int rtlfs_checkpoint_load(rtlfs_ctx *ctx, const void *buf, uint64_t bytes) {
    if (!ctx) return RTLFS_E_ARG;
    if (!buf || bytes < sizeof(CkHeader)) return fail(ctx, RTLFS_E_ARG, "checkpoint buffer too small");
    int rc = build_faults(ctx);
    if (rc != RTLFS_OK) return rc;
    CkHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, CK_MAGIC, 8) != 0) return fail(ctx, RTLFS_E_ARG, "not a checkpoint");
    const uint64_t F = h.F, nd = h.n_designs;
    if (h.W == 0 || h.window == 0 || h.n_live > F || h.n_carry > F || h.nodrop > 1 || nd > 65535 || h.lcap > 2)
        return fail(ctx, RTLFS_E_ARG, "malformed checkpoint header");
    // sizes the header implies, then the byte count must agree exactly
    rtlfs_ctx::Checkpoint c;
    c.T.resize(nd); c.n_net.resize(nd); c.det.resize(F); c.cycle.resize(F); c.port.resize(F);
    c.load.resize(F); c.mism.resize(F); c.st_nreg.resize(F); c.st_r.resize(F * LIGHT_KR);
    c.st_v.resize(F * LIGHT_KR); c.live.resize(h.n_live); c.carry.resize(h.n_carry);
    c.pool_r.resize(h.pool_top); c.pool_v.resize(h.pool_top); c.heads.resize(8); c.rows.resize(h.n_rows);
    uint64_t need = sizeof(CkHeader);
    ck_fields(c, [&](auto &v) { need += v.size() * sizeof(v[0]); });
    if (need != bytes) return fail(ctx, RTLFS_E_ARG, "checkpoint size does not match its header");
    const unsigned char *p = static_cast<const unsigned char *>(buf) + sizeof(CkHeader);
    ck_fields(c, [&](auto &v) {
        if (!v.empty()) memcpy(v.data(), p, v.size() * sizeof(v[0]));
        p += v.size() * sizeof(v[0]);
    });
    uint64_t rows = 0;
    for (uint32_t n : c.n_net) rows += n;
    if (rows != h.n_rows) return fail(ctx, RTLFS_E_ARG, "checkpoint rows do not match its designs");
    // everything the kernels index with: fault ids, register-diff counts within the bounds
    // the kernels were built for, register ids within the fault's design
    if (F != ctx->F || nd != ctx->designs.size())
        return fail(ctx, RTLFS_E_ARG, "checkpoint was taken on other fault lists or designs");
    std::vector<uint32_t> regs_of(F, 0);
    for (size_t d = 0; d < ctx->designs.size(); ++d)
        for (uint32_t f = ctx->f_first[d]; f < ctx->f_first[d + 1]; ++f) regs_of[f] = ctx->designs[d]->R;
    const uint32_t kr = (uint32_t)LIGHT_CAPS[h.lcap][0];
    for (uint32_t f : c.live) {
        if (f >= F || c.st_nreg[f] > kr) return fail(ctx, RTLFS_E_ARG, "checkpoint light fault out of range");
        for (uint32_t k = 0; k < c.st_nreg[f]; ++k)
            if (c.st_r[(size_t)k * F + f] >= regs_of[f]) return fail(ctx, RTLFS_E_ARG, "checkpoint register out of range");
    }
    for (const HeavyCarry &x : c.carry) {
        if (x.fault >= F || x.nreg > regs_of[x.fault] || x.off + x.nreg > h.pool_top)
            return fail(ctx, RTLFS_E_ARG, "checkpoint carry out of range");
        for (uint32_t k = 0; k < x.nreg; ++k)
            if (c.pool_r[x.off + k] >= regs_of[x.fault]) return fail(ctx, RTLFS_E_ARG, "checkpoint register out of range");
    }
    c.window = h.window; c.W = h.W; c.F = h.F; c.nodrop = h.nodrop; c.lcap = h.lcap; c.valid = true;
    rc = checkpoint_matches(ctx, c, c.W, c.nodrop != 0, -1);
    if (rc != RTLFS_OK) return rc;
    ctx->ck = std::move(c);
    ctx->err.clear();
    return RTLFS_OK;
}
}  // extern "C"
