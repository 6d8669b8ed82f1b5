// rtlfs_kernels.cu -- sm_103a kernels of the RTL stuck-at fault simulator.
//
// The method (Sec. II-B): the good machine is simulated once per cycle; each faulty
// machine is kept as its difference from the good one (the "bad gates" of concurrent
// fault simulation: a node carries a bad gate for a fault only where the fault's value
// differs from the good value), a node is evaluated for a fault only when one of its
// operands differs (the check step of Algorithm 1), the fault function forces the site
// bit (Sec. IV-A), outputs are compared with the good values, registers latch at the end
// of the cycle (global synchronization, Sec. II-B) and a detected fault is dropped.
//
// GPU form: the good machine is computed first for all cycles and stored (good trace),
// which makes every faulty machine independent of every other one across all cycles, so
// no global synchronization between faults is needed. Faults with small divergent cones
// run one lane per fault (the many low-load tasks, Sec. III / IV-C-1, balanced by a
// persistent queue the lanes take work from); faults with large cones run one CTA per
// fault, evaluating each topological level of the cone in parallel (the few high-load
// tasks split along their bad gates, Sec. IV-C-2). The register latch is folded into
// the cycle loop of each fault (no separate synchronization phase, Sec. IV-D).
#include "rtlfs_internal.h"

#include <cstdio>

namespace rtlfs {

__device__ __forceinline__ uint64_t wmask(uint32_t w) {
    return w >= 64 ? ~0ull : ((1ull << w) - 1ull);
}

__device__ __forceinline__ int n_operands(uint32_t op) {
    return op == OP_CONST ? 0
         : (op == OP_NOT || op == OP_SHL || op == OP_SHR || op == OP_SLICE) ? 1
         : op == OP_MUX2 ? 3 : 2;
}

// One word-level op on zero-extended operands, masked to the node width.
__device__ __forceinline__ uint64_t eval_op(uint4 d, uint64_t a, uint64_t b, uint64_t c) {
    const uint32_t m = d.w, k = meta_k(m);
    uint64_t r;
    switch (meta_op(m)) {
    case OP_AND:    r = a & b; break;
    case OP_OR:     r = a | b; break;
    case OP_XOR:    r = a ^ b; break;
    case OP_NOT:    r = ~a; break;
    case OP_ADD:    r = a + b; break;
    case OP_SUB:    r = a - b; break;
    case OP_MUX2:   r = a ? b : c; break;
    case OP_EQ:     r = (a == b) ? 1ull : 0ull; break;
    case OP_LT:     r = (a < b) ? 1ull : 0ull; break;
    case OP_SHL:    r = k >= 64 ? 0ull : (a << k); break;
    case OP_SHR:
    case OP_SLICE:  r = k >= 64 ? 0ull : (a >> k); break;
    case OP_CONCAT: r = (k >= 64 ? 0ull : (a << k)) | b; break;
    default:        r = ((uint64_t)d.y << 32) | d.x; break;   // CONST
    }
    return r & wmask(meta_w(m));
}

// Stuck-at fault function: force bit `bm` (a one-hot mask) to `sv`.
__device__ __forceinline__ uint64_t force_bit(uint64_t x, uint64_t bm, bool sv) {
    return sv ? (x | bm) : (x & ~bm);
}

// ===================================================================================
// Good-machine trace. One CTA per design walks the cycles; inside a cycle the nodes of
// one topological level are independent and are spread over the threads, with a
// barrier between levels. Net values of the current cycle live in shared memory when
// they fit (USE_SMEM) and are streamed to the row-major trace rows[t][net].
// ===================================================================================
template <bool USE_SMEM>
__global__ void __launch_bounds__(1024)
good_trace_kernel(const DevDesign *__restrict__ designs, const uint32_t *__restrict__ list,
                  uint32_t max_net) {
    extern __shared__ uint64_t gsm[];
    const DevDesign &D = designs[list[blockIdx.x]];
    const uint32_t I = D.I, R = D.R, IR = I + R, n_net = D.n_net, T = D.T, NL = D.n_levels;
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    uint64_t *val = gsm;                 // [max_net] when USE_SMEM
    uint64_t *qn = gsm + max_net;        // [max_reg] next register values when USE_SMEM
    for (uint32_t t = 0; t < T; ++t) {
        uint64_t *row = D.rows + (size_t)t * n_net;
        for (uint32_t i = tid; i < IR; i += B) {
            uint64_t v;
            if (i < I) v = D.stim[(size_t)t * I + i] & wmask(D.net_w[i]);
            else if (t == 0) v = 0ull;
            else if (USE_SMEM) v = qn[i - I];
            else v = (row - n_net)[D.reg_d[i - I]] & wmask(D.net_w[i]);   // previous row
            if (USE_SMEM) val[i] = v;
            row[i] = v;
        }
        __syncthreads();
        for (uint32_t L = 0; L < NL; ++L) {
            const uint32_t lo = D.lvl_start[L], hi = D.lvl_start[L + 1];
            for (uint32_t n = lo + tid; n < hi; n += B) {
                const uint4 d = D.desc[n];
                const uint32_t op = meta_op(d.w);
                const int no = n_operands(op);
                uint64_t a = 0, b = 0, c = 0;
                if (no >= 1) a = USE_SMEM ? val[d.x] : row[d.x];
                if (no >= 2) b = USE_SMEM ? val[d.y] : row[d.y];
                if (no >= 3) c = USE_SMEM ? val[d.z] : row[d.z];
                const uint64_t v = eval_op(d, a, b, c);
                if (USE_SMEM) val[IR + n] = v;
                row[IR + n] = v;
            }
            __syncthreads();
        }
        if (USE_SMEM) {
            for (uint32_t r = tid; r < R; r += B) qn[r] = val[D.reg_d[r]] & wmask(D.net_w[I + r]);
        }
        __syncthreads();
    }
}

// rows[T][n_net] -> gcol[n_net][T], 32x32 tiles through shared memory.
__global__ void transpose_kernel(uint64_t *__restrict__ gcol, const uint64_t *__restrict__ rows,
                                 uint32_t n_net, uint32_t T) {
    __shared__ uint64_t tile[32][33];
    const uint32_t n0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    const uint32_t tx = threadIdx.x, ty = threadIdx.y;
    for (uint32_t j = ty; j < 32; j += blockDim.y) {
        const uint32_t t = t0 + j, n = n0 + tx;
        if (t < T && n < n_net) tile[j][tx] = rows[(size_t)t * n_net + n];
    }
    __syncthreads();
    for (uint32_t j = ty; j < 32; j += blockDim.y) {
        const uint32_t n = n0 + j, t = t0 + tx;
        if (n < n_net && t < T) gcol[(size_t)n * T + t] = tile[tx][j];
    }
}

// ===================================================================================
// Light kernel: one lane per fault, persistent, lanes take faults from a global queue
// (atomic counter) as they finish -- dynamic balancing of the many low-load faults.
//
// Per fault and cycle the lane keeps, in its own slice of shared memory:
//   register diffs of the start of the cycle (reg, faulty Q) and of the next cycle,
//   the nets whose faulty value differs this cycle (net, value), sorted by net id,
//   a min-heap of node indices still to evaluate (topological order = index order).
// A cycle: seed the diff with the register diffs (and the forced site if it is an input
// or register), push the site node, then pop nodes in index order, evaluate each with
// faulty operands (diff value, else the good trace), force the site bit, keep the result
// if it differs from the good value and push its fan-out. The lowest output port among
// differing nets detects the fault; register diffs for the next cycle are collected as
// nets are kept (the latch, fused into the cycle). With no register diff left, only the
// site can make the machines differ again, so the lane skips to the next cycle where
// the site bit's good value differs from the stuck value. Any capacity overflow hands
// the fault, with its start-of-cycle state, to the heavy kernel.
// ===================================================================================
template <int KR, int KD, int KH>
__global__ void __launch_bounds__(256)
light_kernel(const DevDesign *__restrict__ designs, DevFaults f, Queues q) {
    extern __shared__ __align__(16) unsigned char lsm[];
    const uint32_t B = blockDim.x, tx = threadIdx.x;
    uint64_t *rv = reinterpret_cast<uint64_t *>(lsm);           // [2][KR][B]
    uint64_t *dv = rv + 2 * KR * B;                              // [KD][B]
    uint32_t *rr = reinterpret_cast<uint32_t *>(dv + KD * B);   // [2][KR][B]
    uint32_t *dn = rr + 2 * KR * B;                              // [KD][B]
    uint32_t *hp = dn + KD * B;                                  // [KH][B]
#define RV(bf, k) rv[((bf) * KR + (k)) * B + tx]
#define RR(bf, k) rr[((bf) * KR + (k)) * B + tx]
#define DV(k) dv[(k) * B + tx]
#define DN(k) dn[(k) * B + tx]
#define HP(k) hp[(k) * B + tx]

    for (;;) {
        const unsigned long long qi = atomicAdd(q.light_head, 1ull);
        if (qi >= q.n_light) break;
        const uint32_t fid = q.light_order[qi];
        const DevDesign &D = designs[f.design[fid]];
        const uint32_t I = D.I, IR = D.I + D.R, T = D.T;
        const uint64_t *__restrict__ gcol = D.gcol;
        const uint32_t site = f.site[fid];
        const uint32_t bit = f.bit[fid];
        const bool sv = f.val[fid] != 0;
        const uint64_t bm = 1ull << bit;
        const uint64_t *__restrict__ scol = gcol + (size_t)site * T;
        const uint32_t site_node = site >= IR ? site - IR : 0xFFFFFFFFu;

        uint32_t t = 0, nreg = 0, cur = 0;
        uint64_t load = 0;
        int status = 0;                 // 1 detected, 2 promoted, 3 budget
        int32_t det_cycle = -1, det_port = -1;

        for (;;) {
            if (nreg == 0) {
                // Skip quiescent cycles: nothing differs unless the site bit is activated.
                while (t < T) {
                    const uint64_t g = __ldg(scol + t);
                    if (((g >> bit) & 1ull) != (uint64_t)sv) break;
                    ++t;
                }
                if (t >= T) break;
            }
            const uint32_t nb = cur ^ 1u;
            uint32_t nd = 0, nh = 0, nreg_new = 0, minport = NO_PORT;
            uint64_t filter = 0;
            bool ovf = false;
            const uint64_t load_at_cycle_start = load;   // the heavy kernel redoes a promoted cycle

            auto heap_push = [&](uint32_t x) {
                if (nh >= (uint32_t)KH) { ovf = true; return; }
                uint32_t i = nh++;
                while (i > 0) {
                    const uint32_t p = (i - 1) >> 1;
                    const uint32_t hpv = HP(p);
                    if (hpv <= x) break;
                    HP(i) = hpv;
                    i = p;
                }
                HP(i) = x;
            };
            auto heap_pop = [&]() -> uint32_t {
                const uint32_t top = HP(0);
                const uint32_t x = HP(--nh);
                uint32_t i = 0;
                for (;;) {
                    uint32_t c = 2 * i + 1;
                    if (c >= nh) break;
                    uint32_t cv = HP(c);
                    if (c + 1 < nh) {
                        const uint32_t cv2 = HP(c + 1);
                        if (cv2 < cv) { cv = cv2; ++c; }
                    }
                    if (x <= cv) break;
                    HP(i) = cv;
                    i = c;
                }
                if (nh > 0) HP(i) = x;
                return top;
            };
            auto add_diff = [&](uint32_t net, uint64_t v, uint64_t g) {
                if (nd >= (uint32_t)KD) { ovf = true; return; }
                DN(nd) = net;
                DV(nd) = v;
                ++nd;
                filter |= 1ull << (net & 63u);
                const uint32_t p = __ldg(D.outport + net);
                minport = p < minport ? p : minport;
                const uint32_t e1 = __ldg(D.fo_off + net + 1);
                for (uint32_t e = __ldg(D.fo_off + net); e < e1; ++e) heap_push(__ldg(D.fo_idx + e));
                const uint32_t r1 = __ldg(D.dreg_off + net + 1);
                for (uint32_t e = __ldg(D.dreg_off + net); e < r1; ++e) {
                    const uint32_t r = __ldg(D.dreg_idx + e);
                    const uint64_t wm = wmask(__ldg(D.net_w + I + r));
                    const uint64_t qv = v & wm;
                    if (qv != (g & wm)) {
                        if (nreg_new >= (uint32_t)KR) { ovf = true; return; }
                        RR(nb, nreg_new) = r;
                        RV(nb, nreg_new) = qv;
                        ++nreg_new;
                    }
                }
            };
            auto lookup = [&](uint32_t x) -> uint64_t {
                if ((filter >> (x & 63u)) & 1ull) {
                    for (uint32_t k = 0; k < nd; ++k)
                        if (DN(k) == x) return DV(k);
                }
                return __ldg(gcol + (size_t)x * T + t);
            };

            bool site_seeded = false;
            for (uint32_t k = 0; k < nreg && !ovf; ++k) {
                const uint32_t net = I + RR(cur, k);
                uint64_t qv = RV(cur, k);
                if (net == site) { qv = force_bit(qv, bm, sv); site_seeded = true; }
                const uint64_t g = __ldg(gcol + (size_t)net * T + t);
                if (qv != g) add_diff(net, qv, g);
            }
            if (site < IR && !site_seeded && !ovf) {
                const uint64_t g = __ldg(scol + t);
                const uint64_t fv = force_bit(g, bm, sv);
                if (fv != g) add_diff(site, fv, g);
            }
            if (site_node != 0xFFFFFFFFu && !ovf) heap_push(site_node);
            uint32_t last = 0xFFFFFFFFu;
            while (nh > 0 && !ovf) {
                const uint32_t n = heap_pop();
                if (n == last) continue;
                last = n;
                const uint4 d = __ldg(D.desc + n);
                const uint32_t op = meta_op(d.w);
                const int no = n_operands(op);
                uint64_t a = 0, b = 0, c = 0;
                if (no >= 1) a = lookup(d.x);
                if (no >= 2) b = lookup(d.y);
                if (no >= 3) c = lookup(d.z);
                uint64_t v = eval_op(d, a, b, c);
                if (n == site_node) v = force_bit(v, bm, sv);
                ++load;
                const uint32_t net = IR + n;
                const uint64_t g = __ldg(gcol + (size_t)net * T + t);
                if (v != g) add_diff(net, v, g);
            }
            if (ovf) {
                const uint32_t p = atomicAdd(q.heavy_count, 1u);
                if (p < q.heavy_cap) {
                    HeavyItem &h = q.heavy_items[p];
                    h.fault = fid;
                    h.t = t;
                    h.nreg = nreg;
                    for (uint32_t k = 0; k < nreg; ++k) {
                        h.reg_r[k] = RR(cur, k);
                        h.reg_v[k] = RV(cur, k);
                    }
                }
                load = load_at_cycle_start;
                status = 2;
                break;
            }
            if (minport != NO_PORT) {
                det_cycle = (int32_t)t;
                det_port = (int32_t)minport;
                status = 1;
                break;
            }
            cur = nb;
            nreg = nreg_new;
            if (++t >= T) break;
            if (q.fault_budget && load > q.fault_budget) { status = 3; break; }
        }
        f.load[fid] = load;
        if (status != 2) {
            f.res_det[fid] = status == 1 ? 1 : status == 3 ? 255 : 0;
            f.res_cycle[fid] = det_cycle;
            f.res_port[fid] = det_port;
            if (status == 3) atomicAdd(q.budget_hit, 1ull);
        }
    }
#undef RV
#undef RR
#undef DV
#undef DN
#undef HP
}

// ===================================================================================
// Heavy kernel: one CTA per fault. The fault's faulty values live in per-slot scratch
// (value + cycle stamp per net, so nothing is cleared between cycles); a shared-memory
// bitmap over the node index space marks the nodes with a differing operand, and a
// per-level counter lets the CTA skip levels with nothing to do. Levels are processed
// in order, the dirty nodes of one level in parallel (the bad gates of the fault split
// over the threads), with one barrier per non-empty level.
// ===================================================================================
__global__ void __launch_bounds__(1024)
heavy_kernel(const DevDesign *__restrict__ designs, DevFaults f, Queues q, HeavyScratch S) {
    extern __shared__ __align__(16) uint32_t hsm[];
    const uint32_t nwords = (S.max_node + 31) / 32;
    uint32_t *bm = hsm;                  // [nwords] dirty bits
    uint32_t *cnt = bm + nwords;         // [max_levels] dirty nodes per level
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_t, s_nreg_new, s_minport, s_site_seeded;
    __shared__ unsigned long long s_load;
    const uint32_t tid = threadIdx.x, B = blockDim.x, slot = blockIdx.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    uint64_t *fval = S.fval + (size_t)slot * S.max_net;
    uint32_t *stamp = S.stamp + (size_t)slot * S.max_net;
    uint32_t *regR = S.reg_r + (size_t)slot * 2 * S.max_reg;
    uint64_t *regV = S.reg_v + (size_t)slot * 2 * S.max_reg;

    for (uint32_t i = tid; i < nwords; i += B) bm[i] = 0;
    for (uint32_t i = tid; i < S.max_levels; i += B) cnt[i] = 0;
    uint32_t epoch = S.epoch[slot];
    __syncthreads();

    for (;;) {
        if (tid == 0) s_item = atomicAdd(q.heavy_head, 1ull);
        __syncthreads();
        const unsigned long long idx = s_item;
        const uint32_t n_items = min(*((volatile uint32_t *)q.heavy_count), q.heavy_cap);
        if (idx >= n_items) break;
        const HeavyItem &it = q.heavy_items[idx];
        const uint32_t fid = it.fault;
        const DevDesign &D = designs[f.design[fid]];
        const uint32_t I = D.I, IR = D.I + D.R, T = D.T, NL = D.n_levels;
        const uint64_t *__restrict__ gcol = D.gcol;
        const uint32_t site = f.site[fid];
        const uint32_t bit = f.bit[fid];
        const bool sv = f.val[fid] != 0;
        const uint64_t bmask = 1ull << bit;
        const uint64_t *__restrict__ scol = gcol + (size_t)site * T;
        uint32_t t = it.t, nreg = it.nreg, cur = 0;
        for (uint32_t k = tid; k < nreg; k += B) {
            regR[k] = it.reg_r[k];
            regV[k] = it.reg_v[k];
        }
        if (tid == 0) s_load = 0;
        int status = 0;
        int32_t det_cycle = -1, det_port = -1;
        if (epoch > 0xFFFFF000u) {      // stamps about to wrap: clear and restart
            for (uint32_t i = tid; i < S.max_net; i += B) stamp[i] = 0;
            epoch = 0;
        }
        __syncthreads();

        for (;;) {
            if (nreg == 0) {
                if (warp == 0) {
                    uint32_t found = T;
                    for (uint32_t tt = t; tt < T; tt += 32) {
                        const uint32_t u = tt + lane;
                        bool act = false;
                        if (u < T) act = ((__ldg(scol + u) >> bit) & 1ull) != (uint64_t)sv;
                        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, act);
                        if (bal) { found = tt + __ffs(bal) - 1; break; }
                    }
                    if (lane == 0) s_t = found;
                }
                __syncthreads();
                t = s_t;
                if (t >= T) break;
            }
            ++epoch;
            const uint32_t nb = cur ^ 1u;
            if (tid == 0) { s_nreg_new = 0; s_minport = NO_PORT; s_site_seeded = 0; }
            __syncthreads();

            auto mark = [&](uint32_t net, uint64_t v, uint64_t g) {
                stamp[net] = epoch;
                fval[net] = v;
                const uint32_t p = __ldg(D.outport + net);
                if (p != NO_PORT) atomicMin(&s_minport, p);
                const uint32_t e1 = __ldg(D.fo_off + net + 1);
                for (uint32_t e = __ldg(D.fo_off + net); e < e1; ++e) {
                    const uint32_t c = __ldg(D.fo_idx + e);
                    const uint32_t b1 = 1u << (c & 31u);
                    const uint32_t old = atomicOr(&bm[c >> 5], b1);
                    if (!(old & b1)) atomicAdd(&cnt[__ldg(D.node_level + c)], 1u);
                }
                const uint32_t r1 = __ldg(D.dreg_off + net + 1);
                for (uint32_t e = __ldg(D.dreg_off + net); e < r1; ++e) {
                    const uint32_t r = __ldg(D.dreg_idx + e);
                    const uint64_t wm = wmask(__ldg(D.net_w + I + r));
                    const uint64_t qv = v & wm;
                    if (qv != (g & wm)) {
                        const uint32_t k = atomicAdd(&s_nreg_new, 1u);
                        regR[nb * S.max_reg + k] = r;
                        regV[nb * S.max_reg + k] = qv;
                    }
                }
            };
            auto lookup = [&](uint32_t x) -> uint64_t {
                if (stamp[x] == epoch) return fval[x];
                return __ldg(gcol + (size_t)x * T + t);
            };

            for (uint32_t k = tid; k < nreg; k += B) {
                const uint32_t net = I + regR[cur * S.max_reg + k];
                uint64_t qv = regV[cur * S.max_reg + k];
                if (net == site) { qv = force_bit(qv, bmask, sv); s_site_seeded = 1; }
                const uint64_t g = __ldg(gcol + (size_t)net * T + t);
                if (qv != g) mark(net, qv, g);
            }
            __syncthreads();
            if (tid == 0) {
                if (site < IR && !s_site_seeded) {
                    const uint64_t g = __ldg(scol + t);
                    const uint64_t fv = force_bit(g, bmask, sv);
                    if (fv != g) mark(site, fv, g);
                }
                if (site >= IR) {
                    const uint32_t c = site - IR;
                    const uint32_t b1 = 1u << (c & 31u);
                    const uint32_t old = atomicOr(&bm[c >> 5], b1);
                    if (!(old & b1)) atomicAdd(&cnt[__ldg(D.node_level + c)], 1u);
                }
            }
            __syncthreads();
            uint32_t my_load = 0;
            for (uint32_t L = 0; L < NL; ++L) {
                if (cnt[L] == 0) continue;
                const uint32_t lo = __ldg(D.lvl_start + L), hi = __ldg(D.lvl_start + L + 1);
                const uint32_t w0 = lo >> 5, w1 = (hi - 1) >> 5;
                for (uint32_t w = w0 + tid; w <= w1; w += B) {
                    uint32_t m = 0xFFFFFFFFu;
                    if (w == w0) m &= 0xFFFFFFFFu << (lo & 31u);
                    if (w == w1 && (hi & 31u)) m &= (1u << (hi & 31u)) - 1u;
                    if (!(bm[w] & m)) continue;
                    uint32_t bits = atomicAnd(&bm[w], ~m) & m;
                    while (bits) {
                        const uint32_t j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const uint32_t n = (w << 5) + j;
                        const uint4 d = __ldg(D.desc + n);
                        const uint32_t op = meta_op(d.w);
                        const int no = n_operands(op);
                        uint64_t a = 0, b = 0, c = 0;
                        if (no >= 1) a = lookup(d.x);
                        if (no >= 2) b = lookup(d.y);
                        if (no >= 3) c = lookup(d.z);
                        const uint32_t net = IR + n;
                        uint64_t v = eval_op(d, a, b, c);
                        if (net == site) v = force_bit(v, bmask, sv);
                        ++my_load;
                        const uint64_t g = __ldg(gcol + (size_t)net * T + t);
                        if (v != g) mark(net, v, g);
                    }
                }
                __syncthreads();
                if (tid == 0) cnt[L] = 0;
            }
            if (my_load) atomicAdd(&s_load, (unsigned long long)my_load);
            __syncthreads();
            if (s_minport != NO_PORT) {
                det_cycle = (int32_t)t;
                det_port = (int32_t)s_minport;
                status = 1;
                break;
            }
            nreg = s_nreg_new;
            cur = nb;
            if (++t >= T) break;
            if (q.fault_budget && (f.load[fid] + s_load) > q.fault_budget) { status = 3; break; }
            __syncthreads();
        }
        __syncthreads();
        if (tid == 0) {
            f.load[fid] += s_load;
            f.res_det[fid] = status == 1 ? 1 : status == 3 ? 255 : 0;
            f.res_cycle[fid] = det_cycle;
            f.res_port[fid] = det_port;
            if (status == 3) atomicAdd(q.budget_hit, 1ull);
        }
        __syncthreads();
    }
    if (tid == 0) S.epoch[slot] = epoch;
}

// ===================================================================================
// Plain GPU form: one thread per fault, one flat launch per design (and wave), no
// queue, no heavy path. Same sparse-diff method with unbounded per-thread state in
// global memory: value + stamp per net, a heap of pending nodes with a queued-stamp to
// avoid duplicates, and two register-diff lists.
// ===================================================================================
__global__ void __launch_bounds__(128)
plain_kernel(const DevDesign *__restrict__ designs, uint32_t design, DevFaults f,
             uint32_t first, uint32_t count, uint64_t *fval_all, uint32_t *stamp_all,
             uint32_t *qstamp_all, uint32_t *heap_all, uint32_t *regr_all, uint64_t *regv_all,
             uint32_t sn, uint32_t snode, uint32_t sreg) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= count) return;
    const uint32_t fid = first + tid;
    const DevDesign &D = designs[design];
    const uint32_t I = D.I, IR = D.I + D.R, T = D.T;
    const uint64_t *gcol = D.gcol;
    uint64_t *fval = fval_all + (size_t)tid * sn;
    uint32_t *stamp = stamp_all + (size_t)tid * sn;
    uint32_t *qst = qstamp_all + (size_t)tid * snode;
    uint32_t *hp = heap_all + (size_t)tid * snode;
    uint32_t *regr = regr_all + (size_t)tid * 2 * sreg;
    uint64_t *regv = regv_all + (size_t)tid * 2 * sreg;
    const uint32_t site = f.site[fid];
    const uint32_t bit = f.bit[fid];
    const bool sv = f.val[fid] != 0;
    const uint64_t bm = 1ull << bit;
    uint32_t nreg = 0, cur = 0, epoch = 0;
    uint64_t load = 0;
    int32_t det_cycle = -1, det_port = -1;
    int status = 0;
    for (uint32_t t = 0; t < T; ++t) {
        ++epoch;
        const uint32_t nb = cur ^ 1u;
        uint32_t nh = 0, nreg_new = 0, minport = NO_PORT;
        auto push = [&](uint32_t x) {
            if (qst[x] == epoch) return;
            qst[x] = epoch;
            uint32_t i = nh++;
            while (i > 0) {
                const uint32_t p = (i - 1) >> 1;
                if (hp[p] <= x) break;
                hp[i] = hp[p];
                i = p;
            }
            hp[i] = x;
        };
        auto pop = [&]() -> uint32_t {
            const uint32_t top = hp[0];
            const uint32_t x = hp[--nh];
            uint32_t i = 0;
            for (;;) {
                uint32_t c = 2 * i + 1;
                if (c >= nh) break;
                if (c + 1 < nh && hp[c + 1] < hp[c]) ++c;
                if (x <= hp[c]) break;
                hp[i] = hp[c];
                i = c;
            }
            if (nh > 0) hp[i] = x;
            return top;
        };
        auto keep = [&](uint32_t net, uint64_t v, uint64_t g) {
            stamp[net] = epoch;
            fval[net] = v;
            const uint32_t p = D.outport[net];
            minport = p < minport ? p : minport;
            for (uint32_t e = D.fo_off[net]; e < D.fo_off[net + 1]; ++e) push(D.fo_idx[e]);
            for (uint32_t e = D.dreg_off[net]; e < D.dreg_off[net + 1]; ++e) {
                const uint32_t r = D.dreg_idx[e];
                const uint64_t wm = wmask(D.net_w[I + r]);
                if ((v & wm) != (g & wm)) {
                    regr[nb * sreg + nreg_new] = r;
                    regv[nb * sreg + nreg_new] = v & wm;
                    ++nreg_new;
                }
            }
        };
        auto lookup = [&](uint32_t x) -> uint64_t {
            return stamp[x] == epoch ? fval[x] : gcol[(size_t)x * T + t];
        };
        bool site_seeded = false;
        for (uint32_t k = 0; k < nreg; ++k) {
            const uint32_t net = I + regr[cur * sreg + k];
            uint64_t qv = regv[cur * sreg + k];
            if (net == site) { qv = force_bit(qv, bm, sv); site_seeded = true; }
            const uint64_t g = gcol[(size_t)net * T + t];
            if (qv != g) keep(net, qv, g);
        }
        if (site < IR && !site_seeded) {
            const uint64_t g = gcol[(size_t)site * T + t];
            const uint64_t fv = force_bit(g, bm, sv);
            if (fv != g) keep(site, fv, g);
        }
        if (site >= IR) push(site - IR);
        while (nh > 0) {
            const uint32_t n = pop();
            const uint4 d = D.desc[n];
            const uint32_t op = meta_op(d.w);
            const int no = n_operands(op);
            uint64_t a = 0, b = 0, c = 0;
            if (no >= 1) a = lookup(d.x);
            if (no >= 2) b = lookup(d.y);
            if (no >= 3) c = lookup(d.z);
            const uint32_t net = IR + n;
            uint64_t v = eval_op(d, a, b, c);
            if (net == site) v = force_bit(v, bm, sv);
            ++load;
            const uint64_t g = gcol[(size_t)net * T + t];
            if (v != g) keep(net, v, g);
        }
        if (minport != NO_PORT) {
            det_cycle = (int32_t)t;
            det_port = (int32_t)minport;
            status = 1;
            break;
        }
        nreg = nreg_new;
        cur = nb;
    }
    f.load[fid] = load;
    f.res_det[fid] = status == 1 ? 1 : 0;
    f.res_cycle[fid] = det_cycle;
    f.res_port[fid] = det_port;
}

// ---- launchers -----------------------------------------------------------------------

cudaError_t launch_good_trace(const DevDesign *d_designs, const uint32_t *design_list,
                              uint32_t n_list, uint32_t max_net, uint32_t max_reg,
                              bool use_smem, cudaStream_t stream) {
    if (n_list == 0) return cudaSuccess;
    const size_t smem = use_smem ? ((size_t)max_net + (size_t)max_reg) * sizeof(uint64_t) : 0;
    cudaError_t e;
    if (use_smem) {
        e = cudaFuncSetAttribute(good_trace_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        good_trace_kernel<true><<<n_list, 1024, smem, stream>>>(d_designs, design_list, max_net);
    } else {
        e = cudaFuncSetAttribute(good_trace_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        good_trace_kernel<false><<<n_list, 1024, smem, stream>>>(d_designs, design_list, max_net);
    }
    return cudaGetLastError();
}

cudaError_t launch_transpose(uint64_t *gcol, const uint64_t *rows, uint32_t n_net, uint32_t T,
                             cudaStream_t stream) {
    dim3 grid((n_net + 31) / 32, (T + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, stream>>>(gcol, rows, n_net, T);
    return cudaGetLastError();
}

static size_t light_smem(int block) {
    return (size_t)block * ((2 * LIGHT_KR + LIGHT_KD) * sizeof(uint64_t) +
                            (2 * LIGHT_KR + LIGHT_KD + LIGHT_KH) * sizeof(uint32_t));
}

int light_max_blocks_per_sm(int block) {
    int n = 0;
    const size_t smem = light_smem(block);
    cudaFuncSetAttribute(light_kernel<LIGHT_KR, LIGHT_KD, LIGHT_KH>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, light_kernel<LIGHT_KR, LIGHT_KD, LIGHT_KH>,
                                                  block, smem);
    return n;
}

cudaError_t launch_light(const DevDesign *d_designs, DevFaults f, Queues q, int block, int grid,
                         cudaStream_t stream) {
    const size_t smem = light_smem(block);
    cudaError_t e = cudaFuncSetAttribute(light_kernel<LIGHT_KR, LIGHT_KD, LIGHT_KH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    light_kernel<LIGHT_KR, LIGHT_KD, LIGHT_KH><<<grid, block, smem, stream>>>(d_designs, f, q);
    return cudaGetLastError();
}

size_t heavy_smem_bytes(uint32_t max_node, uint32_t max_levels) {
    return ((size_t)(max_node + 31) / 32 + max_levels) * sizeof(uint32_t);
}

int heavy_max_blocks_per_sm(int block, size_t smem) {
    int n = 0;
    cudaFuncSetAttribute(heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, heavy_kernel, block, smem);
    return n;
}

cudaError_t launch_heavy(const DevDesign *d_designs, DevFaults f, Queues q, HeavyScratch s,
                         int block, int grid, cudaStream_t stream) {
    const size_t smem = heavy_smem_bytes(s.max_node, s.max_levels);
    cudaError_t e = cudaFuncSetAttribute(heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    heavy_kernel<<<grid, block, smem, stream>>>(d_designs, f, q, s);
    return cudaGetLastError();
}

cudaError_t launch_plain(const DevDesign *d_designs, uint32_t design, DevFaults f, uint32_t first,
                         uint32_t count, uint64_t *fval, uint32_t *stamp, uint32_t *qstamp,
                         uint32_t *heap, uint32_t *reg_r, uint64_t *reg_v, uint32_t stride_net,
                         uint32_t stride_node, uint32_t stride_reg, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    plain_kernel<<<(count + 127) / 128, 128, 0, stream>>>(d_designs, design, f, first, count, fval,
                                                          stamp, qstamp, heap, reg_r, reg_v,
                                                          stride_net, stride_node, stride_reg);
    return cudaGetLastError();
}

}  // namespace rtlfs
