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

#include <climits>
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

// The fault function at a fault's site (Sec. IV-A: applied wherever the site's value is
// produced; a virtual function in the paper, a switch on the kind here): stuck-at 0 or 1
// forces the bit in every cycle; a transient flip (an SEU on a register, an SET on an
// input or node net) inverts it during cycle t0 only. A port fault (port != NO_PORT) acts
// on what one output port observes of the site net and on nothing else.
struct FaultSite {
    uint32_t site, port, kind, t0;
    uint64_t bm;   // one-hot mask of the faulted bit
    __device__ __forceinline__ uint64_t apply(uint64_t v, uint32_t t) const {
        return kind == FK_SA0 ? (v & ~bm) : kind == FK_SA1 ? (v | bm) : (t == t0 ? v ^ bm : v);
    }
    // whether the fault function changes anything in cycle t (a stuck-at fault: always)
    __device__ __forceinline__ bool acts(uint32_t t) const { return kind != FK_FLIP || t == t0; }
};

__device__ __forceinline__ FaultSite load_fault(const DevFaults &f, uint32_t fid) {
    FaultSite s;
    s.site = f.site[fid];
    s.kind = f.val[fid];
    s.bm = 1ull << f.bit[fid];
    s.port = f.port ? f.port[fid] : NO_PORT;
    s.t0 = f.t0 ? f.t0[fid] : 0u;
    return s;
}

// ===================================================================================
// Good-machine trace. One CTA per design walks the cycles; inside a cycle the nodes of
// one topological level are independent and are spread over the threads, with a
// barrier between levels. The node list is cut into chunks of at most GOOD_BLOCK nodes
// that never straddle a level, so every thread owns at most one node per chunk. Each
// thread loads its node descriptors two chunks ahead of use (wrapping into the next
// cycle), so no evaluation waits on a global load. Net values of the current cycle live
// in shared memory when they fit (USE_SMEM) and are streamed to the row-major trace
// rows[t][net].
// ===================================================================================
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <bool USE_SMEM>
__global__ void __launch_bounds__(GOOD_BLOCK, 1)
good_trace_kernel(const DevDesign *__restrict__ designs, const uint32_t *__restrict__ list,
                  uint32_t max_net, uint32_t max_reg, uint32_t max_chunks, uint32_t t_begin, uint32_t t_end) {
    extern __shared__ __align__(128) uint64_t gsm[];
    const DevDesign &D = designs[list[blockIdx.x]];
    const uint32_t I = D.I, R = D.R, IR = I + R, n_net = D.n_net, NC = D.n_chunks;
    const uint32_t T = min(D.T, t_end);   // last cycle (exclusive) of this launch
    if (t_begin >= T) return;
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const size_t vwords = USE_SMEM ? (size_t)max_net + max_reg : 0;   // u64 words of values
    uint64_t *val = gsm;                                     // [max_net] when USE_SMEM
    uint64_t *qn = gsm + (USE_SMEM ? max_net : 0);           // [max_reg] when USE_SMEM
    uint2 *ch = reinterpret_cast<uint2 *>(gsm + vwords);     // [max_chunks]
    (void)max_chunks;
    for (uint32_t c = tid; c < NC; c += B) ch[c] = D.chunks[c];
    // this thread's input and its first two registers, kept in registers for every cycle
    const uint64_t in_mask = tid < I ? wmask(D.net_w[tid]) : 0ull;
    const uint32_t r0 = tid, r1 = tid + B;
    const uint32_t rd0 = r0 < R ? D.reg_d[r0] : 0, rd1 = r1 < R ? D.reg_d[r1] : 0;
    const uint64_t rm0 = r0 < R ? wmask(D.net_w[I + r0]) : 0, rm1 = r1 < R ? wmask(D.net_w[I + r1]) : 0;
    if (USE_SMEM && t_begin > 0) {   // resume: register values of t_begin from row t_begin-1
        const uint64_t *prev = D.rows + (size_t)(t_begin - 1) * n_net;
        for (uint32_t r = tid; r < R; r += B) qn[r] = prev[D.reg_d[r]] & wmask(D.net_w[I + r]);
    }
    __syncthreads();

    // Each thread prefetches its node descriptor two chunks ahead into registers (coalesced
    // loads from the L2-resident op graph, wrapping into the next cycle), so no evaluation
    // waits on a global load; chunks of one level are independent, so only a chunk that
    // ends a level is followed by a barrier.
    uint32_t cf = 0;                           // chunk of the next prefetch (wraps)
    auto prefetch = [&]() -> uint4 {
        if (NC == 0) return make_uint4(0u, 0u, 0u, 0u);   // a design without nodes
        const uint2 b = ch[cf];
        const uint32_t n = b.x + tid;
        cf = cf + 1 == NC ? 0 : cf + 1;
        return n < (b.y & 0x7FFFFFFFu) ? __ldg(D.desc + n) : make_uint4(0u, 0u, 0u, 0u);
    };
    uint4 dq0 = prefetch();
    uint4 dq1 = prefetch();
    uint64_t s_next = (tid < I) ? __ldg(D.stim + (size_t)t_begin * I + tid) : 0ull;

    for (uint32_t t = t_begin; t < T; ++t) {
        uint64_t *row = D.rows + (size_t)t * n_net;
        const uint64_t s_cur = s_next;
        if (tid < I && t + 1 < T) s_next = __ldg(D.stim + (size_t)(t + 1) * I + tid);
        for (uint32_t i = tid; i < IR; i += B) {
            uint64_t v;
            if (i < I) v = (i == tid ? s_cur : __ldg(D.stim + (size_t)t * I + i)) & (i == tid ? in_mask : wmask(D.net_w[i]));
            else if (t == 0) v = 0ull;
            else if (USE_SMEM) v = qn[i - I];
            else v = (row - n_net)[D.reg_d[i - I]] & wmask(D.net_w[i]);   // previous row
            if (USE_SMEM) val[i] = v;
            row[i] = v;
        }
        __syncthreads();
        for (uint32_t c = 0; c < NC; ++c) {
            const uint2 b = ch[c];
            const uint32_t n = b.x + tid;
            const uint4 d0 = dq0;
            dq0 = dq1;
            dq1 = prefetch();
            if (n < (b.y & 0x7FFFFFFFu)) {
                const uint32_t op = meta_op(d0.w);
                const int no = n_operands(op);
                uint64_t a = 0, bb = 0, cc = 0;
                if (no >= 1) a = USE_SMEM ? val[d0.x] : row[d0.x];
                if (no >= 2) bb = USE_SMEM ? val[d0.y] : row[d0.y];
                if (no >= 3) cc = USE_SMEM ? val[d0.z] : row[d0.z];
                const uint64_t v = eval_op(d0, a, bb, cc);
                if (USE_SMEM) val[IR + n] = v;
                row[IR + n] = v;
            }
            if (b.y & 0x80000000u) __syncthreads();   // the level's values are complete
        }
        if (USE_SMEM) {
            if (r0 < R) qn[r0] = val[rd0] & rm0;
            if (r1 < R) qn[r1] = val[rd1] & rm1;
            for (uint32_t r = tid + 2 * B; r < R; r += B) qn[r] = val[D.reg_d[r]] & wmask(D.net_w[I + r]);
        }
        __syncthreads();
    }
}

// Staged form of the single-CTA good trace: GOOD_BLOCK consumer threads plus one producer
// warp. The producer copies each chunk's descriptors into a ring of GOOD_NSTAGE shared
// buffers with bulk asynchronous copies (completion counted in bytes on the buffer's "full"
// mbarrier); each consumer warp arrives on the buffer's "empty" mbarrier once its lanes have
// read it, and the producer refills a buffer when every consumer warp has. Consumers
// synchronise among themselves (named barrier 1) only where a level ends and around the
// latch. Every wait is bounded: one that runs out sets a shared flag, after which no thread
// waits on the ring again; the kernel then runs to its end without evaluating, waits (again
// bounded) for copies still in flight, and reports through *err (bit 0).
// ===================================================================================
constexpr uint32_t GOOD_NSTAGE = 4;

__device__ __forceinline__ void tma_issue(uint64_t *mbar, void *dst, const void *src, uint32_t bytes) {
    const uint32_t mb = smem_u32(mbar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(mb) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    const uint32_t mb = smem_u32(mbar);
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mb), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" :: "n"(GOOD_BLOCK) : "memory");
}

template <bool USE_SMEM>
__global__ void __launch_bounds__(GOOD_BLOCK + 32, 1)
good_trace_staged_kernel(const DevDesign *__restrict__ designs, const uint32_t *__restrict__ list,
                         uint32_t max_net, uint32_t max_reg, uint32_t max_chunks, uint32_t *err,
                         uint32_t t_begin, uint32_t t_end) {
    extern __shared__ __align__(128) uint64_t gsm[];
    __shared__ __align__(8) uint64_t full[GOOD_NSTAGE], empty[GOOD_NSTAGE];
    __shared__ uint32_t s_fail;                      // a bounded wait ran out
    __shared__ unsigned long long s_issued;          // chunk instances the producer issued
    const DevDesign &D = designs[list[blockIdx.x]];
    const uint32_t I = D.I, R = D.R, IR = I + R, n_net = D.n_net, NC = D.n_chunks;
    const uint32_t T = min(D.T, t_end);
    if (t_begin >= T) return;   // the same for every thread of the CTA
    const uint32_t tid = threadIdx.x, B = GOOD_BLOCK;
    const size_t vwords = USE_SMEM ? (size_t)max_net + max_reg : 0;
    uint64_t *val = gsm;
    uint64_t *qn = gsm + (USE_SMEM ? max_net : 0);
    uint4 *stage = reinterpret_cast<uint4 *>(gsm + ((vwords + 1) & ~(size_t)1));   // [NSTAGE][GOOD_BLOCK]
    uint2 *ch = reinterpret_cast<uint2 *>(stage + GOOD_NSTAGE * GOOD_BLOCK);       // [max_chunks]
    (void)max_chunks;
    for (uint32_t c = tid; c < NC; c += blockDim.x) ch[c] = D.chunks[c];
    if (tid == 0) {
        s_fail = 0u;
        s_issued = 0ull;
        for (uint32_t b = 0; b < GOOD_NSTAGE; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(full + b)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(empty + b)), "n"(GOOD_BLOCK / 32) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bool consumer = tid < B;
    const uint64_t in_mask = consumer && tid < I ? wmask(D.net_w[tid]) : 0ull;
    const uint32_t r0 = tid, r1 = tid + B;
    const uint32_t rd0 = consumer && r0 < R ? D.reg_d[r0] : 0, rd1 = consumer && r1 < R ? D.reg_d[r1] : 0;
    const uint64_t rm0 = consumer && r0 < R ? wmask(D.net_w[I + r0]) : 0, rm1 = consumer && r1 < R ? wmask(D.net_w[I + r1]) : 0;
    if (USE_SMEM && consumer && t_begin > 0) {
        const uint64_t *prev = D.rows + (size_t)(t_begin - 1) * n_net;
        for (uint32_t r = tid; r < R; r += B) qn[r] = prev[D.reg_d[r]] & wmask(D.net_w[I + r]);
    }
    __syncthreads();
    const unsigned long long total = (unsigned long long)(T - t_begin) * NC;

    if (!consumer) {
        // producer: one lane walks the chunk instances of the launch, wrapping over the list
        if (tid == B) {
            uint32_t cf = 0;
            unsigned long long k = 0;
            for (; k < total; ++k) {
                const uint32_t b = (uint32_t)(k % GOOD_NSTAGE);
                if (k >= GOOD_NSTAGE &&
                    !mbar_wait(empty + b, (uint32_t)((k / GOOD_NSTAGE - 1) & 1ull))) {
                    atomicExch(&s_fail, 1u);
                    break;
                }
                if (*(volatile uint32_t *)&s_fail) break;
                const uint2 c = ch[cf];
                const uint32_t n = (c.y & 0x7FFFFFFFu) - c.x;   // >= 1: a chunk holds a node
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_issue(full + b, stage + b * GOOD_BLOCK, D.desc + c.x, n * 16u);
                cf = cf + 1 == NC ? 0 : cf + 1;
            }
            s_issued = k;
        }
    } else {
        const uint32_t lane = tid & 31u;
        uint32_t kb = 0, kp = 0;                 // buffer and phase parity of the current instance
        unsigned long long kc = 0;               // instances consumed
        uint64_t s_next = tid < I ? __ldg(D.stim + (size_t)t_begin * I + tid) : 0ull;
        for (uint32_t t = t_begin; t < T; ++t) {
            uint64_t *row = D.rows + (size_t)t * n_net;
            const uint64_t s_cur = s_next;
            if (tid < I && t + 1 < T) s_next = __ldg(D.stim + (size_t)(t + 1) * I + tid);
            for (uint32_t i = tid; i < IR; i += B) {
                uint64_t v;
                if (i < I) v = (i == tid ? s_cur : __ldg(D.stim + (size_t)t * I + i)) & (i == tid ? in_mask : wmask(D.net_w[i]));
                else if (t == 0) v = 0ull;
                else if (USE_SMEM) v = qn[i - I];
                else v = (row - n_net)[D.reg_d[i - I]] & wmask(D.net_w[i]);
                if (USE_SMEM) val[i] = v;
                row[i] = v;
            }
            consumers_sync();
            for (uint32_t c = 0; c < NC; ++c, ++kc) {
                const uint2 b = ch[c];
                const uint32_t n = b.x + tid;
                // every consumer waits for the instance's copy, node or not: a warp that
                // arrived on a buffer's "empty" barrier before its copy landed could run a
                // whole ring ahead and arrive twice in one phase
                const bool failed = *(volatile uint32_t *)&s_fail != 0u;
                bool ok = false;
                if (!failed) {
                    ok = mbar_wait(full + kb, kp);
                    if (!ok) atomicExch(&s_fail, 1u);
                }
                if (ok && n < (b.y & 0x7FFFFFFFu)) {
                    {
                        const uint4 d0 = stage[kb * GOOD_BLOCK + tid];
                        const uint32_t op = meta_op(d0.w);
                        const int no = n_operands(op);
                        uint64_t a = 0, bb = 0, cc = 0;
                        if (no >= 1) a = USE_SMEM ? val[d0.x] : row[d0.x];
                        if (no >= 2) bb = USE_SMEM ? val[d0.y] : row[d0.y];
                        if (no >= 3) cc = USE_SMEM ? val[d0.z] : row[d0.z];
                        const uint64_t v = eval_op(d0, a, bb, cc);
                        if (USE_SMEM) val[IR + n] = v;
                        row[IR + n] = v;
                    }
                }
                __syncwarp();   // this warp's lanes are done with the buffer
                if (lane == 0 && !failed)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(empty + kb)) : "memory");
                if (++kb == GOOD_NSTAGE) { kb = 0; kp ^= 1u; }
                if (b.y & 0x80000000u) consumers_sync();   // the level's values are complete
            }
            if (USE_SMEM) {
                if (r0 < R) qn[r0] = val[rd0] & rm0;
                if (r1 < R) qn[r1] = val[rd1] & rm1;
                for (uint32_t r = tid + 2 * B; r < R; r += B) qn[r] = val[D.reg_d[r]] & wmask(D.net_w[I + r]);
            }
            consumers_sync();
        }
        (void)kc;
    }
    __syncthreads();
    if (s_fail && tid == 0) {
        // report, and let copies still in flight land before the CTA's memory goes away: the
        // instances after the last one whose buffer was waited on completely (at most the
        // ring's depth)
        atomicOr(err, 1u);
        const unsigned long long issued = s_issued;
        const unsigned long long from = issued > GOOD_NSTAGE ? issued - GOOD_NSTAGE : 0ull;
        for (unsigned long long k = from; k < issued; ++k)
            mbar_wait(full + (uint32_t)(k % GOOD_NSTAGE), (uint32_t)((k / GOOD_NSTAGE) & 1ull));
    }
}

// ===================================================================================
// Good-machine trace of a design too large for one CTA's shared memory: one cluster of
// C CTAs (2..16) per design. Each CTA owns a contiguous share of every level's nodes and
// keeps their values of the current cycle in its own shared memory; a node reads each
// operand where it lives through distributed shared memory (mapa + ld.shared::cluster),
// its descriptor carrying the operand's location (CL_*). A register lives in its home
// CTA in two banks selected by the cycle's parity: the latch of cycle t fills bank
// (t+1)&1 while other registers' latches may still read Q_t from bank t&1 (a register
// fed by a register). Every CTA keeps its own copy of the inputs. A cluster barrier
// (release/acquire, so a level's values are visible cluster-wide) ends every level and
// the latch. Each CTA prefetches its own descriptor list three chunks ahead into
// registers (one more than the single-CTA kernel: a remote operand read and the cluster
// barrier make a level longer); a level in which a CTA owns no node is an empty chunk
// that only joins the barrier.
// ===================================================================================
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_ctas() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 64-bit load from the same shared-memory offset in CTA `rank` of this cluster.
__device__ __forceinline__ uint64_t dsm_load(uint32_t local_addr, uint32_t rank) {
    uint32_t ra;
    uint64_t v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local_addr), "r"(rank));
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(ra));
    return v;
}

__global__ void __launch_bounds__(GOOD_BLOCK, 1)
good_cluster_kernel(const DevDesign *__restrict__ designs, const uint32_t *__restrict__ list,
                    uint32_t C_launch, uint32_t *err, uint32_t t_begin, uint32_t t_end) {
    extern __shared__ __align__(128) uint64_t gsm[];
    const uint32_t rank = cluster_rank(), C = cluster_ctas();
    // The design list and every CTA's share assume clusters of C_launch CTAs: a launch that
    // did not get them (a tool replaying it without the cluster attribute) returns at once,
    // in every CTA before any cluster barrier, and flags the error.
    if (C != C_launch) {
        if (threadIdx.x == 0) atomicOr(err, 4u);
        return;
    }
    const DevDesign &D = designs[list[blockIdx.x / C]];
    const uint32_t I = D.I, IR = I + D.R, n_net = D.n_net;
    const uint32_t T = min(D.T, t_end);
    if (t_begin >= T) return;   // the same in every CTA of the cluster
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t own = D.cl_own, rown = D.cl_rown;
    const size_t vwords = (size_t)own + 2 * (size_t)rown + I;
    uint64_t *qv = gsm + own;            // [2][rown] register banks (node values [own] before)
    uint64_t *inv = qv + 2 * rown;       // [I] inputs
    const uint32_t c0 = D.cl_ch_off[rank], NC = D.cl_ch_off[rank + 1] - c0;
    uint4 *ch = reinterpret_cast<uint4 *>(gsm + ((vwords + 1) & ~(size_t)1));   // [NC]
    const uint4 *__restrict__ cdesc = D.cl_desc + (size_t)rank * own;
    const uint4 *__restrict__ creg = D.cl_reg + D.cl_reg_off[rank];
    const uint32_t NR = D.cl_reg_off[rank + 1] - D.cl_reg_off[rank];
    const uint32_t base = smem_u32(gsm);
    for (uint32_t c = tid; c < NC; c += B) ch[c] = D.cl_chunk[c0 + c];
    // registers entering t_begin: the reset value, or the latch of the previous window
    for (uint32_t j = tid; j < NR; j += B) {
        const uint4 g = creg[j];
        uint64_t q = 0ull;
        if (t_begin > 0) q = D.rows[(size_t)(t_begin - 1) * n_net + g.w] & wmask(g.z);
        qv[(t_begin & 1u) * rown + j] = q;
    }
    // all CTAs of the cluster are running and initialised before any remote read
    cluster_sync();

    uint32_t cf = 0;                             // chunk of the next prefetch (wraps)
    auto prefetch = [&]() -> uint4 {
        if (NC == 0) return make_uint4(0u, 0u, 0u, 0u);   // a design without nodes
        const uint4 b = ch[cf];
        cf = cf + 1 == NC ? 0 : cf + 1;
        return tid < (b.y & 0x7FFFFFFFu) ? __ldg(cdesc + b.x + tid) : make_uint4(0u, 0u, 0u, 0u);
    };
    uint4 dq0 = prefetch();
    uint4 dq1 = prefetch();
    uint4 dq2 = prefetch();

    for (uint32_t t = t_begin; t < T; ++t) {
        uint64_t *row = D.rows + (size_t)t * n_net;
        const uint32_t bank_off = (t & 1u) * rown;
        // inputs of cycle t into this CTA's copy; CTA 0 writes them to the trace
        for (uint32_t i = tid; i < I; i += B) {
            const uint64_t v = __ldg(D.stim + (size_t)t * I + i) & wmask(D.net_w[i]);
            inv[i] = v;
            if (rank == 0) row[i] = v;
        }
        // this CTA's registers (a contiguous index range): Q of cycle t to the trace
        for (uint32_t j = tid; j < NR; j += B) row[I + creg[j].x] = qv[bank_off + j];
        __syncthreads();
        auto fetch = [&](uint32_t e) -> uint64_t {
            const uint32_t w = (e & CL_WORD) + ((e & CL_REG) ? bank_off : 0u);
            const uint32_t r = (e & CL_SELF) ? rank : ((e >> CL_RANK_SHIFT) & 15u);
            return dsm_load(base + w * 8u, r);
        };
        for (uint32_t c = 0; c < NC; ++c) {
            const uint4 b = ch[c];
            const uint4 d0 = dq0;
            dq0 = dq1;
            dq1 = dq2;
            dq2 = prefetch();
            if (tid < (b.y & 0x7FFFFFFFu)) {
                const uint32_t op = meta_op(d0.w);
                const int no = n_operands(op);
                uint64_t a = 0, bb = 0, cc = 0;
                if (no >= 1) a = fetch(d0.x);
                if (no >= 2) bb = fetch(d0.y);
                if (no >= 3) cc = fetch(d0.z);
                const uint64_t v = eval_op(d0, a, bb, cc);
                gsm[b.x + tid] = v;
                row[IR + b.z + tid] = v;
            }
            if (b.y & 0x80000000u) cluster_sync();   // the level is complete cluster-wide
        }
        // latch: Q of cycle t+1 into the other bank
        for (uint32_t j = tid; j < NR; j += B) {
            const uint4 g = creg[j];
            qv[(rown - bank_off) + j] = fetch(g.y) & wmask(g.z);
        }
        cluster_sync();
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

// Window transpose: rows[t][net] -> gcol[net][t] for t in [t0, t1), every design (z).
__global__ void transpose_window_kernel(const DevDesign *__restrict__ designs, uint32_t t0, uint32_t t1) {
    __shared__ uint64_t tile[32][33];
    const DevDesign &D = designs[blockIdx.z];
    const uint32_t n_net = D.n_net, T = min(D.T, t1);
    const uint32_t n0 = blockIdx.x * 32, tb = t0 + blockIdx.y * 32;
    if (n0 >= n_net || tb >= T) return;
    const uint32_t tx = threadIdx.x, ty = threadIdx.y;
    for (uint32_t j = ty; j < 32; j += blockDim.y) {
        const uint32_t t = tb + j, n = n0 + tx;
        if (t < T && n < n_net) tile[j][tx] = D.rows[(size_t)t * n_net + n];
    }
    __syncthreads();
    for (uint32_t j = ty; j < 32; j += blockDim.y) {
        const uint32_t n = n0 + j, t = tb + tx;
        if (n < n_net && t < T) D.gcol[(size_t)n * D.T + t] = tile[tx][j];
    }
}

// Activation bitplane: one warp per fault reads 64 consecutive cycles of the site column
// (two coalesced 256-byte rows) and writes one 64-bit word per 64 cycles.
__global__ void activation_kernel(const DevDesign *__restrict__ designs, DevFaults f, uint64_t *act,
                                  uint32_t t0, uint32_t t1) {
    const uint32_t fid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (fid >= f.F) return;
    const DevDesign &D = designs[f.design[fid]];
    const uint32_t T = D.T, te = min(t1, T);
    const uint32_t site = f.site[fid], bit = f.bit[fid];
    const uint64_t sv = f.val[fid];   // a stuck-at fault acts where the bit differs from it
    const uint32_t tf = f.t0 ? f.t0[fid] : 0u;   // a flip acts in its own cycle only
    const uint64_t *col = D.gcol + (size_t)site * T;
    uint64_t *out = act + (size_t)fid * f.act_stride;
    for (uint32_t tw = t0; tw < te; tw += 64) {
        const uint32_t ta = tw + lane, tb = tw + 32 + lane;
        const bool a = ta < te && (sv == FK_FLIP ? ta == tf : ((__ldg(col + ta) >> bit) & 1ull) != sv);
        const bool b = tb < te && (sv == FK_FLIP ? tb == tf : ((__ldg(col + tb) >> bit) & 1ull) != sv);
        const uint32_t lo = __ballot_sync(0xFFFFFFFFu, a), hi = __ballot_sync(0xFFFFFFFFu, b);
        if (lane == 0) out[tw >> 6] = ((uint64_t)hi << 32) | lo;
    }
}

// First cycle in [t, tend) where the fault is active by itself, or tend.
__device__ __forceinline__ uint32_t next_active(const uint64_t *__restrict__ fact, uint32_t t, uint32_t tend) {
    while (t < tend) {
        const uint64_t w = __ldg(fact + (t >> 6)) >> (t & 63u);
        if (w) {
            const uint32_t a = t + (uint32_t)(__ffsll((long long)w) - 1);
            return a < tend ? a : tend;
        }
        t = (t | 63u) + 1;
    }
    return tend;
}

// ===================================================================================
// Heavy kernel: one CTA per fault (by default a single warp). Shared memory holds a bitmap
// over the nodes (dirty: some operand differs), the number of dirty nodes per level (so an
// empty level costs one shared read) and a ring of fan-out ranges to expand. Differing
// values live in per-slot global scratch beside the stamp of the cycle that wrote them: an
// operand read fetches that entry and the good value together and keeps the faulty one
// when its stamp is the current cycle's, so nothing needs clearing between cycles.
// Each level runs in up to three phases: (0) the level's dirty nodes are gathered from the
// bitmap into a shared list, so they split evenly over the threads however they cluster
// in the bitmap's words; (1) the threads evaluate them, and a kept net marks its consumers
// itself when it has few -- a list of at most HEAVY_PREFETCH is fetched beside the
// operands, so marking it waits on no further load -- or appends its fan-out range to the
// ring when it has many; (2) all threads mark the consumers of the long ranges together,
// so a control net with thousands of readers costs a few passes instead of one thread's
// loop. The two kernels below share this per-fault loop; they differ in where the faults
// come from and where a survivor's state goes.
// ===================================================================================
constexpr uint32_t HEAVY_PREFETCH = 4;
constexpr uint32_t HEAVY_FILTER = 4096;   // bits of the kept-net filter (stamped form)

// Shared scalars of one heavy CTA.
struct HeavyVars {
    unsigned long long load;   // node evaluations of the current fault
    uint32_t t;                // next active cycle, found by warp 0
    uint32_t nreg_new;         // register diffs latched this cycle
    uint32_t minport;          // lowest output port that differs this cycle
    uint32_t site_seeded;      // a register diff already covered the fault site
    uint32_t nd;               // exact form: words of the net bitmap to clear
    uint32_t nfr;              // fan-out ranges appended this cycle
    uint32_t nl;               // dirty nodes gathered for the current level
};

// Views of the heavy kernels' dynamic shared memory (heavy_smem_bytes sizes the same layout).
struct HeavySmem {
    uint32_t *bm;                 // [nwn] dirty nodes
    uint32_t *cnt;                // [max_levels] dirty nodes per level
    uint32_t *nlist;              // [HEAVY_NLIST] dirty nodes of the current level
    // stamped form: nets kept this cycle, by net id modulo HEAVY_FILTER (a clear bit: the
    // net holds its good value; a set bit: read the stamped entry)
    uint32_t *flt;                // [HEAVY_FILTER / 32]
    // exact form: a bit per net (differs this cycle) and the words to clear after it
    uint32_t *dbm;                // [nwd]
    uint32_t *dlist;              // [HEAVY_DLIST]
    uint2 *frange;                // [HEAVY_FRANGE] fan-out ranges (8-byte aligned)
    unsigned long long *lvm;      // [nlw] one bit per level that has dirty nodes
    // global-bitmap form: bm lives in the slot's global scratch and this shared summary has a
    // bit per bitmap word that may hold a mark this cycle (cleared at the cycle's end)
    uint32_t *top;                // [nwt]
    uint32_t nwd, nlw, nwt;
};

// Shared-memory words of the node record of one heavy CTA: the node bitmap itself, or, in
// the global-bitmap form, its one-bit-per-word summary.
__host__ __device__ inline size_t heavy_node_words(uint32_t max_node, bool gbm) {
    const size_t nwn = (size_t)(max_node + 31) / 32;
    return gbm ? (nwn + 31) / 32 : nwn;
}

template <bool EXACT, bool GBM = false>
__device__ __forceinline__ HeavySmem heavy_layout(uint32_t *hsm, const HeavyScratch &S, uint32_t slot = 0) {
    HeavySmem m;
    const uint32_t nwn = (S.max_node + 31) / 32;
    const size_t nodew = heavy_node_words(S.max_node, GBM);
    m.nwd = (S.max_net + 31) / 32;
    m.nlw = (S.max_levels + 63) / 64;
    m.nwt = GBM ? (uint32_t)nodew : 0u;
    m.bm = GBM ? S.gbm + (size_t)slot * nwn : hsm;
    m.top = GBM ? hsm : nullptr;
    m.cnt = hsm + nodew;
    m.nlist = m.cnt + S.max_levels;
    m.flt = m.nlist + HEAVY_NLIST;
    m.dbm = m.flt + (EXACT ? 0 : HEAVY_FILTER / 32);
    m.dlist = m.dbm + (EXACT ? m.nwd : 0);
    const size_t side = EXACT ? (size_t)m.nwd + HEAVY_DLIST : HEAVY_FILTER / 32;
    const size_t fr_words = (nodew + S.max_levels + HEAVY_NLIST + side + 1) & ~(size_t)1;
    m.frange = reinterpret_cast<uint2 *>(hsm + fr_words);
    m.lvm = reinterpret_cast<unsigned long long *>(m.frange + HEAVY_FRANGE);
    return m;
}

// Zero the bitmaps and counters once per CTA; every fault leaves them zero again (the
// global node bitmaps of the global-bitmap form are zeroed when allocated).
template <bool EXACT, bool GBM = false>
__device__ __forceinline__ void heavy_zero(const HeavySmem &m, const HeavyScratch &S, HeavyVars &V) {
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t nwn = (S.max_node + 31) / 32;
    if (GBM) {
        for (uint32_t i = tid; i < m.nwt; i += B) m.top[i] = 0;
    } else {
        for (uint32_t i = tid; i < nwn; i += B) m.bm[i] = 0;
    }
    for (uint32_t i = tid; i < S.max_levels; i += B) m.cnt[i] = 0;
    if (EXACT) {
        for (uint32_t i = tid; i < m.nwd; i += B) m.dbm[i] = 0;
    } else {
        for (uint32_t i = tid; i < HEAVY_FILTER / 32; i += B) m.flt[i] = 0;
    }
    for (uint32_t i = tid; i < m.nlw; i += B) m.lvm[i] = 0;
    if (tid == 0) { V.nfr = 0; V.nl = 0; V.load = 0; }
}

// Loads issued where they stand: volatile, so the compiler does not sink them into the
// branch that consumes them and they travel together with the operand loads.
__device__ __forceinline__ uint32_t ld_early_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_early_u16(const uint16_t *p) {
    unsigned short v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

// Outcome of one heavy fault's run.
struct HeavyRun {
    uint32_t t;        // in: first cycle; out: first cycle not completed (see status)
    uint32_t nreg;     // in: register diffs in half 0; out: in half `cur`
    uint32_t cur;      // out: the half of regR/regV that holds the live register diffs
    int status;        // 0 alive at tend, 1 detected at t, 3 over the load budget
    int32_t det_cycle, det_port;
    uint32_t mism;     // no-drop mode: cycles of this run with a differing output
};

// Simulate fault fid from cycle r.t until it is detected, exceeds the load budget or
// reaches tend. Cycles with no register diff and an inactive site are skipped without
// work. V.load accumulates the node evaluations; the caller zeroes it per fault. Every
// thread of the CTA calls this together and leaves the shared bitmaps zero.
template <bool EXACT>
__device__ __forceinline__ void heavy_run_fault(const DevDesign &D, const DevFaults &f, uint32_t fid,
                                                uint32_t tend, unsigned long long budget,
                                                const HeavySmem &sm, HeavyVars &V, HeavyVal *fval, uint32_t &stamp,
                                                uint32_t *regR, uint64_t *regV, uint32_t max_reg, uint32_t max_net,
                                                HeavyRun &r) {
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    const uint32_t I = D.I, IR = D.I + D.R, T = D.T, NL = D.n_levels;
    const uint64_t *__restrict__ gcol = D.gcol;
    const uint4 *__restrict__ netinfo = D.netinfo;
    const uint32_t *__restrict__ fo_idx = D.fo_idx;
    const uint16_t *__restrict__ fo_lvl = D.fo_lvl;
    const uint32_t *__restrict__ dreg_off = D.dreg_off;
    const uint32_t *__restrict__ dreg_rec = D.dreg_rec;
    const FaultSite fs = load_fault(f, fid);
    const uint32_t site = fs.site;
    const uint32_t bit = f.bit[fid];
    const uint64_t *__restrict__ scol = gcol + (size_t)site * T;
    uint32_t *const bm = sm.bm, *const cnt = sm.cnt;
    unsigned long long *const lvm = sm.lvm;
    const uint32_t nlw = sm.nlw;
    const bool nodrop = f.mism != nullptr;
    bool seen = nodrop && f.res_det[fid] == 1;   // no-drop: first detection already recorded
    uint32_t t = r.t, nreg = r.nreg, cur = 0, mism = 0;
    int status = 0;
    int32_t det_cycle = -1, det_port = -1;
    // A detection at cycle t on `port` (uniform across the CTA): stop (dropping), or
    // record the first one and count.
    auto detect = [&](uint32_t port) -> bool {
        if (!nodrop) {
            det_cycle = (int32_t)t;
            det_port = (int32_t)port;
            status = 1;
            return true;
        }
        if (!seen && tid == 0) {
            f.res_det[fid] = 1;
            f.res_cycle[fid] = (int32_t)t;
            f.res_port[fid] = (int32_t)port;
        }
        seen = true;
        ++mism;
        return false;
    };

    // Consumer node c (at level lv) becomes dirty.
    auto mark = [&](uint32_t c, uint32_t lv) {
        const uint32_t b1 = 1u << (c & 31u);
        const uint32_t o2 = atomicOr(&bm[c >> 5], b1);
        if (!(o2 & b1) && atomicAdd(&cnt[lv], 1u) == 0u) atomicOr(&lvm[lv >> 6], 1ull << (lv & 63u));
    };
    // The consumers of fan-out entries [e0, e1) with a stride: all threads share a long
    // range in expand(); one thread marks a short one.
    auto mark_range = [&](uint32_t e0, uint32_t e1, uint32_t first, uint32_t step) {
        for (uint32_t e = e0 + first; e < e1; e += step) mark(__ldg(fo_idx + e), __ldg(fo_lvl + e));
    };
    // Ranges live in a ring indexed by a per-cycle append counter V.nfr; fr_begin (the
    // same in every thread, advanced only after a barrier) is the first unexpanded one.
    uint32_t fr_begin = 0;
    auto expand = [&]() {   // call after a barrier
        const uint32_t end = V.nfr;
        const uint32_t n = min(end - fr_begin, HEAVY_FRANGE);
        for (uint32_t k = 0; k < n; ++k) {
            const uint2 fr = sm.frange[(fr_begin + k) % HEAVY_FRANGE];
            mark_range(fr.x, fr.y, tid, B);
        }
        fr_begin = end;
    };
    // A net that differs this cycle: its value, its flag, a detecting port, and the
    // registers it drives whose latched value differs too (into half nb).
    auto keep_value = [&](uint32_t net, uint64_t v, uint64_t g, uint4 ni, uint32_t nb) {
        if (EXACT) {
            reinterpret_cast<uint64_t *>(fval)[net] = v;
            if (!atomicOr(&sm.dbm[net >> 5], 1u << (net & 31u))) {   // first bit of the word
                const uint32_t k = atomicAdd(&V.nd, 1u);
                if (k < HEAVY_DLIST) sm.dlist[k] = net >> 5;
            }
        } else {
            reinterpret_cast<uint4 *>(fval)[net] = make_uint4((uint32_t)v, (uint32_t)(v >> 32), stamp, 0u);
            atomicOr(&sm.flt[(net / 32u) % (HEAVY_FILTER / 32u)], 1u << (net & 31u));
        }
        const uint32_t p = ni_port(ni.w);
        if (p != NI_NO_PORT) atomicMin(&V.minport, p);
        uint32_t nr = ni_nreg(ni.w);
        if (nr == 255u) nr = __ldg(dreg_off + net + 1) - ni.z;
        for (uint32_t e = ni.z; e < ni.z + nr; ++e) {
            const uint32_t rec = __ldg(dreg_rec + e);   // register | width << 25
            const uint64_t wm = wmask(rec >> 25);
            const uint64_t qv = v & wm;
            if (qv != (g & wm)) {
                const uint32_t k = atomicAdd(&V.nreg_new, 1u);
                regR[nb * max_reg + k] = rec & 0x1FFFFFFu;
                regV[nb * max_reg + k] = qv;
            }
        }
    };
    // Its consumers: a long list goes to the ring (marked here if the ring is full).
    auto keep_fanout = [&](uint4 ni) {
        if (ni.y - ni.x > HEAVY_INLINE_FANOUT) {
            const uint32_t k = atomicAdd(&V.nfr, 1u);
            if (k - fr_begin < HEAVY_FRANGE) sm.frange[k % HEAVY_FRANGE] = make_uint2(ni.x, ni.y);
            else mark_range(ni.x, ni.y, 0, 1);
        } else {
            mark_range(ni.x, ni.y, 0, 1);
        }
    };
    auto lookup = [&](uint32_t x) -> uint64_t {
        if (EXACT) {
            if ((sm.dbm[x >> 5] >> (x & 31u)) & 1u) return reinterpret_cast<const uint64_t *>(fval)[x];
        } else if ((sm.flt[(x / 32u) % (HEAVY_FILTER / 32u)] >> (x & 31u)) & 1u) {
            const uint4 e = reinterpret_cast<const uint4 *>(fval)[x];   // kept this cycle, or a
            if (e.z == stamp) return ((uint64_t)e.y << 32) | e.x;     // net sharing its bit
        }
        return __ldg(gcol + (size_t)x * T + t);
    };

    for (;;) {
        if (nreg == 0) {   // nothing latched: jump to the next cycle the fault acts by itself
            if (fs.kind == FK_FLIP) {
                t = t <= fs.t0 ? min(fs.t0, tend) : tend;
            } else {
                if (warp == 0 && f.act) {
                    if (lane == 0) V.t = next_active(f.act + (size_t)fid * f.act_stride, t, tend);
                } else if (warp == 0) {
                    uint32_t found = tend;
                    for (uint32_t tt = t; tt < tend; tt += 32) {
                        const uint32_t u = tt + lane;
                        bool act = false;
                        if (u < tend) act = ((__ldg(scol + u) >> bit) & 1ull) != (uint64_t)fs.kind;
                        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, act);
                        if (bal) { found = tt + __ffs(bal) - 1; break; }
                    }
                    if (lane == 0) V.t = found;
                }
                __syncthreads();
                t = V.t;
            }
            if (t >= tend) break;
            if (fs.port != NO_PORT) {
                // a port fault changes only what its port observes of the site net: the
                // machines differ exactly in the cycles the fault acts (virtual node evaluated)
                if (tid == 0) V.load += 1;
                if (detect(fs.port)) break;
                __syncthreads();
                if (++t >= tend) break;
                if (budget && (f.load[fid] + V.load) > budget) { status = 3; break; }
                continue;
            }
        }
        const uint32_t nb = cur ^ 1u;
        if (tid == 0) { V.nreg_new = 0; V.minport = NI_NO_PORT; V.site_seeded = 0; V.nd = 0; V.nfr = 0; }
        fr_begin = 0;
        if (!EXACT) {
            if (++stamp == 0u) {   // the slot's stamps wrapped: forget every old entry once
                for (uint32_t i = tid; i < max_net; i += B) fval[i].stamp = 0u;
                stamp = 1u;
            }
            for (uint32_t i = tid; i < HEAVY_FILTER / 32; i += B) sm.flt[i] = 0u;
        }
        __syncthreads();

        // registers that carry a difference into this cycle
        for (uint32_t k = tid; k < nreg; k += B) {
            const uint32_t net = I + regR[cur * max_reg + k];
            uint64_t qv = regV[cur * max_reg + k];
            const uint4 ni = __ldg(netinfo + net);
            const uint64_t g = __ldg(gcol + (size_t)net * T + t);
            if (net == site) { qv = fs.apply(qv, t); V.site_seeded = 1; }
            if (qv != g) { keep_value(net, qv, g, ni, nb); keep_fanout(ni); }
        }
        __syncthreads();
        if (tid == 0) {
            if (site < IR && !V.site_seeded) {   // input or register site
                const uint64_t g = __ldg(scol + t);
                const uint64_t fv = fs.apply(g, t);
                if (fv != g) {
                    const uint4 ni = __ldg(netinfo + site);
                    keep_value(site, fv, g, ni, nb);
                    keep_fanout(ni);
                }
            }
            if (site >= IR && fs.acts(t)) mark(site - IR, __ldg(D.node_level + site - IR));   // node site
        }
        __syncthreads();
        expand();
        __syncthreads();

        uint32_t my_load = 0;
        // Evaluate dirty node n; keep its value if it differs from the good machine.
        auto eval_node = [&](uint32_t n) {
            const uint32_t net = IR + n;
            const uint4 d = __ldg(D.desc + n);
            const uint4 ni = __ldg(netinfo + net);
            const uint64_t g = __ldg(gcol + (size_t)net * T + t);
            const uint32_t nf = ni.y - ni.x;
            uint32_t pc[HEAVY_PREFETCH], pl[HEAVY_PREFETCH];
#pragma unroll
            for (uint32_t k = 0; k < HEAVY_PREFETCH; ++k) {
                pc[k] = 0;
                pl[k] = 0;
                if (nf <= HEAVY_PREFETCH && k < nf) {
                    pc[k] = ld_early_u32(fo_idx + ni.x + k);
                    pl[k] = ld_early_u16(fo_lvl + ni.x + k);
                }
            }
            const uint32_t op = meta_op(d.w);
            const int no = n_operands(op);
            uint64_t a = 0, b = 0, c = 0;
            if (no >= 1) a = lookup(d.x);
            if (no >= 2) b = lookup(d.y);
            if (no >= 3) c = lookup(d.z);
            uint64_t v = eval_op(d, a, b, c);
            if (net == site) v = fs.apply(v, t);
            ++my_load;
            if (v != g) {
                keep_value(net, v, g, ni, nb);
                if (nf <= HEAVY_PREFETCH) {
#pragma unroll
                    for (uint32_t k = 0; k < HEAVY_PREFETCH; ++k)
                        if (k < nf) mark(pc[k], pl[k]);
                } else {
                    keep_fanout(ni);
                }
            }
        };

        for (uint32_t L = 0;;) {
            // next level with dirty nodes (bits are only ever set above the current level)
            uint32_t lw = L >> 6;
            unsigned long long m = lw < nlw ? lvm[lw] & (~0ull << (L & 63u)) : 0ull;
            while (!m && ++lw < nlw) m = lvm[lw];
            if (!m) break;
            L = (lw << 6) + (uint32_t)(__ffsll((long long)m) - 1);
            if (L >= NL) break;
            const uint32_t lo = __ldg(D.lvl_start + L), hi = __ldg(D.lvl_start + L + 1);
            const uint32_t w0 = lo >> 5, w1 = (hi - 1) >> 5;
            // every mark into level L was made at a lower level, behind a barrier: the
            // count is exact and the same in all threads
            const bool gather = cnt[L] <= HEAVY_NLIST;
            for (uint32_t w = w0 + tid; w <= w1; w += B) {
                uint32_t wm = 0xFFFFFFFFu;
                if (w == w0) wm &= 0xFFFFFFFFu << (lo & 31u);
                if (w == w1 && (hi & 31u)) wm &= (1u << (hi & 31u)) - 1u;
                if (!(bm[w] & wm)) continue;
                uint32_t bits = atomicAnd(&bm[w], ~wm) & wm;
                if (gather) {
                    uint32_t k = atomicAdd(&V.nl, (uint32_t)__popc(bits));
                    for (; bits; bits &= bits - 1, ++k)
                        if (k < HEAVY_NLIST) sm.nlist[k] = (w << 5) + (uint32_t)(__ffs(bits) - 1);
                } else {
                    for (; bits; bits &= bits - 1) eval_node((w << 5) + (uint32_t)(__ffs(bits) - 1));
                }
            }
            if (gather) {
                __syncthreads();
                const uint32_t nl = min(V.nl, HEAVY_NLIST);
                for (uint32_t i = tid; i < nl; i += B) eval_node(sm.nlist[i]);
            }
            __syncthreads();
            if (V.nfr != fr_begin) {   // uniform: read after the barrier
                expand();
                __syncthreads();
            }
            if (tid == 0) {
                cnt[L] = 0;
                atomicAnd(&lvm[L >> 6], ~(1ull << (L & 63u)));
                V.nl = 0;
            }
            __syncthreads();
            ++L;
        }
        if (my_load) atomicAdd(&V.load, (unsigned long long)my_load);
        __syncthreads();
        if (EXACT) {   // clear the net bitmap for the next cycle
            const uint32_t nd = V.nd;
            if (nd <= HEAVY_DLIST) {
                for (uint32_t k = tid; k < nd; k += B) sm.dbm[sm.dlist[k]] = 0;
            } else {
                for (uint32_t i = tid; i < sm.nwd; i += B) sm.dbm[i] = 0;
            }
        }
        if (V.minport != NI_NO_PORT && detect(V.minport)) break;
        nreg = V.nreg_new;
        cur = nb;
        if (++t >= tend) break;
        if (budget && (f.load[fid] + V.load) > budget) { status = 3; break; }
        __syncthreads();
    }
    r.t = t;
    r.nreg = nreg;
    r.cur = cur;
    r.status = status;
    r.det_cycle = det_cycle;
    r.det_port = det_port;
    r.mism = mism;
}

// One warp per fault (heavy_block = 32): the loop of heavy_run_fault with warp
// synchronisation in place of block barriers, the level's dirty nodes gathered by a warp
// prefix sum instead of shared atomics, the detecting port and the evaluation count kept
// per lane and reduced once per cycle, and the level bitmap cleared once per cycle. Same
// results and the same evaluation counts as heavy_run_fault.
template <bool EXACT, bool GBM>
__device__ __forceinline__ void heavy_run_fault_warp(const DevDesign &D, const DevFaults &f, uint32_t fid,
                                                     uint32_t tend, unsigned long long budget,
                                                     const HeavySmem &sm, HeavyVars &V, HeavyVal *fval, uint32_t &stamp,
                                                     uint32_t *regR, uint64_t *regV, uint32_t max_reg, uint32_t max_net,
                                                     HeavyRun &r) {
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t I = D.I, IR = D.I + D.R, T = D.T, NL = D.n_levels;
    const uint64_t *__restrict__ gcol = D.gcol;
    const uint4 *__restrict__ netinfo = D.netinfo;
    const uint32_t *__restrict__ fo_idx = D.fo_idx;
    const uint16_t *__restrict__ fo_lvl = D.fo_lvl;
    const uint32_t *__restrict__ dreg_off = D.dreg_off;
    const uint32_t *__restrict__ dreg_rec = D.dreg_rec;
    const FaultSite fs = load_fault(f, fid);
    const uint32_t site = fs.site;
    const uint32_t bit = f.bit[fid];
    const uint64_t *__restrict__ scol = gcol + (size_t)site * T;
    uint32_t *const bm = sm.bm, *const cnt = sm.cnt;
    unsigned long long *const lvm = sm.lvm;
    const uint32_t nlw = sm.nlw;
    const bool nodrop = f.mism != nullptr;
    bool seen = nodrop && f.res_det[fid] == 1;   // no-drop: first detection already recorded
    // evaluations this run may do before the fault's budget is exceeded (negative when it
    // already is; unlimited without a budget)
    const long long room = budget ? (long long)budget - (long long)f.load[fid] : LLONG_MAX;
    unsigned long long load = 0;                 // this run's evaluations (warp-uniform)
    uint32_t t = r.t, nreg = r.nreg, cur = 0, mism = 0;
    int status = 0;
    int32_t det_cycle = -1, det_port = -1;
    auto detect = [&](uint32_t port) -> bool {
        if (!nodrop) {
            det_cycle = (int32_t)t;
            det_port = (int32_t)port;
            status = 1;
            return true;
        }
        if (!seen && lane == 0) {
            f.res_det[fid] = 1;
            f.res_cycle[fid] = (int32_t)t;
            f.res_port[fid] = (int32_t)port;
        }
        seen = true;
        ++mism;
        return false;
    };
    auto mark = [&](uint32_t c, uint32_t lv) {
        const uint32_t b1 = 1u << (c & 31u);
        if (GBM) {
            // a reduction on the global word (no value back) and its summary bit; the level's
            // count may include a node marked twice, which only errs towards the scan path
            atomicOr(&bm[c >> 5], b1);
            atomicOr(&sm.top[c >> 10], 1u << ((c >> 5) & 31u));
            if (atomicAdd(&cnt[lv], 1u) == 0u) atomicOr(&lvm[lv >> 6], 1ull << (lv & 63u));
        } else {
            const uint32_t o2 = atomicOr(&bm[c >> 5], b1);
            if (!(o2 & b1) && atomicAdd(&cnt[lv], 1u) == 0u) atomicOr(&lvm[lv >> 6], 1ull << (lv & 63u));
        }
    };
    auto mark_range = [&](uint32_t e0, uint32_t e1, uint32_t first, uint32_t step) {
        for (uint32_t e = e0 + first; e < e1; e += step) mark(__ldg(fo_idx + e), __ldg(fo_lvl + e));
    };
    uint32_t fr_begin = 0;
    auto expand = [&]() {   // call after a warp sync
        const uint32_t end = V.nfr;
        const uint32_t n = min(end - fr_begin, HEAVY_FRANGE);
        for (uint32_t k = 0; k < n; ++k) {
            const uint2 fr = sm.frange[(fr_begin + k) % HEAVY_FRANGE];
            mark_range(fr.x, fr.y, lane, 32u);
        }
        fr_begin = end;
    };
    uint32_t pmin = NI_NO_PORT;   // this lane's lowest differing port in the cycle
    auto keep_value = [&](uint32_t net, uint64_t v, uint64_t g, uint4 ni, uint32_t nb) {
        if (EXACT) {
            reinterpret_cast<uint64_t *>(fval)[net] = v;
            if (!atomicOr(&sm.dbm[net >> 5], 1u << (net & 31u))) {   // first bit of the word
                const uint32_t k = atomicAdd(&V.nd, 1u);
                if (k < HEAVY_DLIST) sm.dlist[k] = net >> 5;
            }
        } else {
            reinterpret_cast<uint4 *>(fval)[net] = make_uint4((uint32_t)v, (uint32_t)(v >> 32), stamp, 0u);
            atomicOr(&sm.flt[(net / 32u) % (HEAVY_FILTER / 32u)], 1u << (net & 31u));
        }
        pmin = min(pmin, ni_port(ni.w));
        uint32_t nr = ni_nreg(ni.w);
        if (nr == 255u) nr = __ldg(dreg_off + net + 1) - ni.z;
        for (uint32_t e = ni.z; e < ni.z + nr; ++e) {
            const uint32_t rec = __ldg(dreg_rec + e);   // register | width << 25
            const uint64_t wm = wmask(rec >> 25);
            const uint64_t qv = v & wm;
            if (qv != (g & wm)) {
                const uint32_t k = atomicAdd(&V.nreg_new, 1u);
                regR[nb * max_reg + k] = rec & 0x1FFFFFFu;
                regV[nb * max_reg + k] = qv;
            }
        }
    };
    auto keep_fanout = [&](uint4 ni) {
        if (ni.y - ni.x > HEAVY_INLINE_FANOUT) {
            const uint32_t k = atomicAdd(&V.nfr, 1u);
            if (k - fr_begin < HEAVY_FRANGE) sm.frange[k % HEAVY_FRANGE] = make_uint2(ni.x, ni.y);
            else mark_range(ni.x, ni.y, 0, 1);
        } else {
            mark_range(ni.x, ni.y, 0, 1);
        }
    };
    auto lookup = [&](uint32_t x) -> uint64_t {
        if (EXACT) {
            if ((sm.dbm[x >> 5] >> (x & 31u)) & 1u) return reinterpret_cast<const uint64_t *>(fval)[x];
        } else if ((sm.flt[(x / 32u) % (HEAVY_FILTER / 32u)] >> (x & 31u)) & 1u) {
            const uint4 e = reinterpret_cast<const uint4 *>(fval)[x];   // kept this cycle, or a
            if (e.z == stamp) return ((uint64_t)e.y << 32) | e.x;     // net sharing its bit
        }
        return __ldg(gcol + (size_t)x * T + t);
    };

    for (;;) {
        if (nreg == 0) {   // nothing latched: jump to the next cycle the fault acts by itself
            if (fs.kind == FK_FLIP) {
                t = t <= fs.t0 ? min(fs.t0, tend) : tend;
            } else if (f.act) {
                const uint32_t tn = lane == 0 ? next_active(f.act + (size_t)fid * f.act_stride, t, tend) : 0u;
                t = __shfl_sync(FULL, tn, 0);
            } else {
                uint32_t found = tend;
                for (uint32_t tt = t; tt < tend; tt += 32) {
                    const uint32_t u = tt + lane;
                    const bool act = u < tend && ((__ldg(scol + u) >> bit) & 1ull) != (uint64_t)fs.kind;
                    const uint32_t bal = __ballot_sync(FULL, act);
                    if (bal) { found = tt + __ffs(bal) - 1; break; }
                }
                t = found;
            }
            if (t >= tend) break;
            if (fs.port != NO_PORT) {
                // a port fault changes only what its port observes of the site net
                ++load;
                if (detect(fs.port)) break;
                if (++t >= tend) break;
                if ((long long)load > room) { status = 3; break; }
                continue;
            }
        }
        const uint32_t nb = cur ^ 1u;
        if (lane == 0) { V.nreg_new = 0; V.nd = 0; V.nfr = 0; }
        fr_begin = 0;
        pmin = NI_NO_PORT;
        if (!EXACT) {
            if (++stamp == 0u) {   // the slot's stamps wrapped: forget every old entry once
                for (uint32_t i = lane; i < max_net; i += 32) fval[i].stamp = 0u;
                stamp = 1u;
            }
            for (uint32_t i = lane; i < HEAVY_FILTER / 32; i += 32) sm.flt[i] = 0u;
        }
        __syncwarp();

        // registers that carry a difference into this cycle
        bool seeded = false;
        for (uint32_t k = lane; k < nreg; k += 32) {
            const uint32_t net = I + regR[cur * max_reg + k];
            uint64_t qv = regV[cur * max_reg + k];
            const uint4 ni = __ldg(netinfo + net);
            const uint64_t g = __ldg(gcol + (size_t)net * T + t);
            if (net == site) { qv = fs.apply(qv, t); seeded = true; }
            if (qv != g) { keep_value(net, qv, g, ni, nb); keep_fanout(ni); }
        }
        const bool site_seeded = __any_sync(FULL, seeded);
        if (lane == 0) {
            if (site < IR && !site_seeded) {   // input or register site
                const uint64_t g = __ldg(scol + t);
                const uint64_t fv = fs.apply(g, t);
                if (fv != g) {
                    const uint4 ni = __ldg(netinfo + site);
                    keep_value(site, fv, g, ni, nb);
                    keep_fanout(ni);
                }
            }
            if (site >= IR && fs.acts(t)) mark(site - IR, __ldg(D.node_level + site - IR));   // node site
        }
        __syncwarp();
        expand();
        __syncwarp();

        uint32_t my_load = 0;
        auto eval_node = [&](uint32_t n) {
            const uint32_t net = IR + n;
            const uint4 d = __ldg(D.desc + n);
            const uint4 ni = __ldg(netinfo + net);
            const uint64_t g = __ldg(gcol + (size_t)net * T + t);
            const uint32_t nf = ni.y - ni.x;
            uint32_t pc[HEAVY_PREFETCH], pl[HEAVY_PREFETCH];
#pragma unroll
            for (uint32_t k = 0; k < HEAVY_PREFETCH; ++k) {
                pc[k] = 0;
                pl[k] = 0;
                if (nf <= HEAVY_PREFETCH && k < nf) {
                    pc[k] = ld_early_u32(fo_idx + ni.x + k);
                    pl[k] = ld_early_u16(fo_lvl + ni.x + k);
                }
            }
            const uint32_t op = meta_op(d.w);
            const int no = n_operands(op);
            uint64_t a = 0, b = 0, c = 0;
            if (no >= 1) a = lookup(d.x);
            if (no >= 2) b = lookup(d.y);
            if (no >= 3) c = lookup(d.z);
            uint64_t v = eval_op(d, a, b, c);
            if (net == site) v = fs.apply(v, t);
            ++my_load;
            if (v != g) {
                keep_value(net, v, g, ni, nb);
                if (nf <= HEAVY_PREFETCH) {
#pragma unroll
                    for (uint32_t k = 0; k < HEAVY_PREFETCH; ++k)
                        if (k < nf) mark(pc[k], pl[k]);
                } else {
                    keep_fanout(ni);
                }
            }
        };

        for (uint32_t L = 0;;) {
            // next level with dirty nodes: bits at or below a processed level are ignored
            // (marks only go to higher levels) and the whole bitmap is cleared per cycle
            uint32_t lw = L >> 6;
            unsigned long long m = lw < nlw ? lvm[lw] & (~0ull << (L & 63u)) : 0ull;
            while (!m && ++lw < nlw) m = lvm[lw];
            if (!m) break;
            L = (lw << 6) + (uint32_t)(__ffsll((long long)m) - 1);
            if (L >= NL) break;
            const uint32_t lo = __ldg(D.lvl_start + L), hi = __ldg(D.lvl_start + L + 1);
            const uint32_t w0 = lo >> 5, w1 = (hi - 1) >> 5;
            if (GBM) __threadfence_block();   // the warp's global marks are visible to its loads
            if (cnt[L] <= HEAVY_NLIST) {
                // gather: one bitmap word per lane, positions from a warp prefix sum; no
                // marks happen meanwhile, so each lane clears its word's level bits plainly
                uint32_t base = 0;
                for (uint32_t wb = w0; wb <= w1; wb += 32) {
                    const uint32_t w = wb + lane;
                    uint32_t bits = 0;
                    if (w <= w1) {
                        uint32_t wm = 0xFFFFFFFFu;
                        if (w == w0) wm &= 0xFFFFFFFFu << (lo & 31u);
                        if (w == w1 && (hi & 31u)) wm &= (1u << (hi & 31u)) - 1u;
                        if (GBM) {
                            if ((sm.top[w >> 5] >> (w & 31u)) & 1u) {   // the word may hold marks
                                const uint32_t word = __ldcg(bm + w);
                                bits = word & wm;
                                if (bits) __stcg(bm + w, word & ~wm);
                            }
                        } else {
                            const uint32_t word = bm[w];
                            bits = word & wm;
                            if (bits) bm[w] = word & ~wm;
                        }
                    }
                    const uint32_t cb = (uint32_t)__popc(bits);
                    uint32_t incl = cb;
#pragma unroll
                    for (uint32_t o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    uint32_t k = base + incl - cb;
                    for (; bits; bits &= bits - 1, ++k)
                        if (k < HEAVY_NLIST) sm.nlist[k] = (w << 5) + (uint32_t)(__ffs(bits) - 1);
                    base += __shfl_sync(FULL, incl, 31);
                }
                __syncwarp();
                const uint32_t nl = min(base, HEAVY_NLIST);
                for (uint32_t i = lane; i < nl; i += 32) eval_node(sm.nlist[i]);
            } else {
                for (uint32_t w = w0 + lane; w <= w1; w += 32) {
                    uint32_t wm = 0xFFFFFFFFu;
                    if (w == w0) wm &= 0xFFFFFFFFu << (lo & 31u);
                    if (w == w1 && (hi & 31u)) wm &= (1u << (hi & 31u)) - 1u;
                    if (GBM) {
                        // evaluations of this level may mark the next level's nodes in the same
                        // word meanwhile: clear this level's bits atomically
                        if (!((sm.top[w >> 5] >> (w & 31u)) & 1u)) continue;
                        if (!(__ldcg(bm + w) & wm)) continue;
                    } else if (!(bm[w] & wm)) {
                        continue;
                    }
                    uint32_t bits = atomicAnd(&bm[w], ~wm) & wm;
                    for (; bits; bits &= bits - 1) eval_node((w << 5) + (uint32_t)(__ffs(bits) - 1));
                }
            }
            __syncwarp();
            if (V.nfr != fr_begin) {   // uniform: read after the sync
                expand();
                __syncwarp();
            }
            if (lane == 0) cnt[L] = 0;
            ++L;
        }
        load += __reduce_add_sync(FULL, my_load);
        const uint32_t minport = __reduce_min_sync(FULL, pmin);
        __syncwarp();
        for (uint32_t i = lane; i < nlw; i += 32) lvm[i] = 0;
        if (GBM)   // every marked word was gathered and cleared; the summary bits may be stale
            for (uint32_t i = lane; i < sm.nwt; i += 32) sm.top[i] = 0;
        if (EXACT) {   // clear the net bitmap for the next cycle
            const uint32_t nd = V.nd;
            if (nd <= HEAVY_DLIST) {
                for (uint32_t k = lane; k < nd; k += 32) sm.dbm[sm.dlist[k]] = 0;
            } else {
                for (uint32_t i = lane; i < sm.nwd; i += 32) sm.dbm[i] = 0;
            }
        }
        if (minport != NI_NO_PORT && detect(minport)) break;
        nreg = V.nreg_new;
        cur = nb;
        if (++t >= tend) break;
        if ((long long)load > room) { status = 3; break; }
        __syncwarp();
    }
    __syncwarp();
    if (lane == 0) V.load = load;
    r.t = t;
    r.nreg = nreg;
    r.cur = cur;
    r.status = status;
    r.det_cycle = det_cycle;
    r.det_port = det_port;
    r.mism = mism;
}

// Barrier of a heavy CTA: one warp (heavy_block = 32) or several.
template <bool WARP>
__device__ __forceinline__ void hsync() {
    if (WARP) __syncwarp(); else __syncthreads();
}

template <bool WARP, bool EXACT, bool GBM = false>
__global__ void __launch_bounds__(WARP ? 32 : 1024, WARP ? 24 : 1)
heavy_kernel(const DevDesign *__restrict__ designs, DevFaults f, Queues q, HeavyScratch S) {
    extern __shared__ __align__(16) uint32_t hsm[];
    __shared__ HeavyVars V;
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_n_items;
    const uint32_t tid = threadIdx.x, B = blockDim.x, slot = blockIdx.x;
    const HeavySmem sm = heavy_layout<EXACT, GBM>(hsm, S, slot);
    HeavyVal *fval = S.fval + (size_t)slot * S.max_net;
    uint32_t *regR = S.reg_r + (size_t)slot * 2 * S.max_reg;
    uint64_t *regV = S.reg_v + (size_t)slot * 2 * S.max_reg;
    uint32_t stamp = EXACT ? 0u : S.stamp[slot];   // the same in every thread, advanced together
    heavy_zero<EXACT, GBM>(sm, S, V);
    hsync<WARP>();

    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(q.heavy_head, 1ull);
            s_n_items = min(*((volatile uint32_t *)q.heavy_count), q.heavy_cap);
        }
        hsync<WARP>();
        const unsigned long long idx = s_item;
        if (idx >= s_n_items) break;
        const HeavyItem &it = q.heavy_items[idx];
        const uint32_t fid = it.fault;
        const DevDesign &D = designs[f.design[fid]];
        for (uint32_t k = tid; k < it.nreg; k += B) {
            regR[k] = it.reg_r[k];
            regV[k] = it.reg_v[k];
        }
        if (tid == 0) V.load = 0;
        hsync<WARP>();
        HeavyRun r{it.t, it.nreg, 0, 0, -1, -1, 0};
        if (WARP) heavy_run_fault_warp<EXACT, GBM>(D, f, fid, D.T, q.fault_budget, sm, V, fval, stamp, regR, regV, S.max_reg, S.max_net, r);
        else heavy_run_fault<EXACT>(D, f, fid, D.T, q.fault_budget, sm, V, fval, stamp, regR, regV, S.max_reg, S.max_net, r);
        hsync<WARP>();
        if (tid == 0) {
            f.load[fid] += V.load;
            if (f.mism) f.mism[fid] += r.mism;
            if (!(r.status == 0 && f.mism)) {   // no-drop: a detection was recorded when it happened
                f.res_det[fid] = r.status == 1 ? 1 : r.status == 3 ? 255 : 0;
                f.res_cycle[fid] = r.det_cycle;
                f.res_port[fid] = r.det_port;
            }
            if (r.status == 3) atomicAdd(q.budget_hit, 1ull);
            atomicAdd(q.counters + 0, V.load);
            const uint32_t t_end = r.status == 1 ? r.t + 1 : min(r.t, D.T);
            atomicAdd(q.counters + 1, (unsigned long long)(t_end - it.t));
        }
        hsync<WARP>();
    }
    if (!EXACT && threadIdx.x == 0) S.stamp[slot] = stamp;   // the next launch continues from it
}

// Windowed heavy kernel: the heavy kernel over cycles [t0, t1) for the faults carried
// from the last window and those promoted in this one; survivors carry their register
// diffs to the next window through the pool.
// One-warp CTAs: 24 resident per SM at the 80 registers the exact and stamped forms take;
// the global-bitmap form (large designs, whose level steps wait on DRAM misses) is held to
// 64 registers (a few spilled bytes) so that 32 faults are in flight per SM.
template <bool WARP, bool EXACT, bool GBM = false>
__global__ void __launch_bounds__(WARP ? 32 : 1024, WARP ? (GBM ? 32 : 24) : 1)
heavy_window_kernel(const DevDesign *__restrict__ designs, DevFaults f, WinHeavy q, HeavyScratch S) {
    extern __shared__ __align__(16) uint32_t hsm[];
    __shared__ HeavyVars V;
    __shared__ unsigned long long s_item, s_off;
    const uint32_t tid = threadIdx.x, B = blockDim.x, slot = blockIdx.x;
    const HeavySmem sm = heavy_layout<EXACT, GBM>(hsm, S, slot);
    HeavyVal *fval = S.fval + (size_t)slot * S.max_net;
    uint32_t *regR = S.reg_r + (size_t)slot * 2 * S.max_reg;
    uint64_t *regV = S.reg_v + (size_t)slot * 2 * S.max_reg;
    uint32_t stamp = EXACT ? 0u : S.stamp[slot];   // the same in every thread, advanced together
    heavy_zero<EXACT, GBM>(sm, S, V);
    hsync<WARP>();

    // written before this launch by earlier work on the stream: the same in every thread
    const uint32_t n_carry = *q.n_carry_in, pb = *q.prom_begin, pe = *q.prom_end;
    const unsigned long long n_items = (unsigned long long)n_carry + (pe - pb);
    for (;;) {
        if (tid == 0) s_item = atomicAdd(q.head, 1ull);
        hsync<WARP>();
        const unsigned long long idx = s_item;
        if (idx >= n_items) break;
        const bool carried = idx < n_carry;
        // carried faults back to front: the slowest of the last window first
        const HeavyCarry cin = carried ? q.carry_in[n_carry - 1 - (uint32_t)idx] : HeavyCarry{0, 0, 0};
        const HeavyItem &it = q.prom[pb + (carried ? 0 : idx - n_carry)];
        const uint32_t fid = carried ? cin.fault : it.fault;
        const DevDesign &D = designs[f.design[fid]];
        const uint32_t tend = min(q.t1, D.T);   // this window ends at tend
        const uint32_t t_start = carried ? q.t0 : it.t;
        const uint32_t nreg0 = carried ? cin.nreg : it.nreg;
        for (uint32_t k = tid; k < nreg0; k += B) {
            regR[k] = carried ? q.pool_r_in[cin.off + k] : it.reg_r[k];
            regV[k] = carried ? q.pool_v_in[cin.off + k] : it.reg_v[k];
        }
        if (tid == 0) V.load = 0;
        hsync<WARP>();
        HeavyRun r{t_start, nreg0, 0, 0, -1, -1, 0};
        if (WARP) heavy_run_fault_warp<EXACT, GBM>(D, f, fid, tend, q.fault_budget, sm, V, fval, stamp, regR, regV, S.max_reg, S.max_net, r);
        else heavy_run_fault<EXACT>(D, f, fid, tend, q.fault_budget, sm, V, fval, stamp, regR, regV, S.max_reg, S.max_net, r);
        hsync<WARP>();
        const bool carry = r.status == 0 && tend < D.T;   // alive at the end of the window
        if (carry) {
            if (tid == 0) {
                const unsigned long long off = atomicAdd(q.pool_top_out, (unsigned long long)r.nreg);
                s_off = off + r.nreg <= q.pool_cap ? off : ~0ull;
                if (s_off == ~0ull) atomicOr(q.err, 2u);
            }
            hsync<WARP>();
            const unsigned long long off = s_off;
            if (off != ~0ull) {
                for (uint32_t k = tid; k < r.nreg; k += B) {
                    q.pool_r_out[off + k] = regR[r.cur * S.max_reg + k];
                    q.pool_v_out[off + k] = regV[r.cur * S.max_reg + k];
                }
                if (tid == 0) q.carry_out[atomicAdd(q.n_carry_out, 1u)] = HeavyCarry{fid, r.nreg, off};
            }
        }
        if (tid == 0) {
            f.load[fid] += V.load;
            if (f.mism) f.mism[fid] += r.mism;
            if (!carry && !(r.status == 0 && f.mism)) {
                f.res_det[fid] = r.status == 1 ? 1 : r.status == 3 ? 255 : 0;
                f.res_cycle[fid] = r.det_cycle;
                f.res_port[fid] = r.det_port;
            }
            if (r.status == 3) atomicAdd(q.budget_hit, 1ull);
            atomicAdd(q.counters + 0, V.load);
            const uint32_t t_end = r.status == 1 ? r.t + 1 : min(r.t, tend);
            atomicAdd(q.counters + 1, (unsigned long long)(t_end - t_start));
        }
        hsync<WARP>();
    }
    if (!EXACT && threadIdx.x == 0) S.stamp[slot] = stamp;   // the next launch continues from it
}

// ===================================================================================
// Light kernel: one lane per fault, persistent, lanes take faults from a global queue
// (atomic counter) as they finish -- dynamic balancing of the many low-load faults.
//
// Per fault and cycle the lane keeps, in its own slice of shared memory:
//   register diffs of the start of the cycle (reg, faulty Q) and of the next cycle,
//   the nets whose faulty value differs this cycle (net, value), in the order kept,
//   a min-heap of node indices still to evaluate (topological order = index order).
// A cycle: seed the diff with the register diffs (and the faulted site if it is an input
// or register), push the site node, then pop nodes in index order, evaluate each with
// faulty operands (diff value, else the good trace), apply the fault function at the
// site, keep the result if it differs from the good value and push its fan-out. The
// lowest output port among differing nets detects the fault; register diffs for the next
// cycle are collected as nets are kept (the latch, fused into the cycle). With no register
// diff left, only the fault itself can make the machines differ again, so the lane skips
// to the next cycle in which it acts. Any capacity overflow hands the fault, with its
// start-of-cycle state, to the heavy kernel. The two kernels below share this per-fault
// loop; they differ in where the faults come from and where a survivor's state goes.
// ===================================================================================

// Outcome of one light fault's run.
struct LightRun {
    uint32_t t;        // in: first cycle; out: first cycle not completed (see status)
    uint32_t nreg;     // in: register diffs in half 0; out: in half `cur`
    uint32_t cur;      // out: the half holding the live register diffs
    int status;        // 0 alive at tend, 1 detected at t, 2 promoted at t, 3 over budget
    int32_t det_cycle, det_port;
    uint64_t load;     // node evaluations of this run (a promoted cycle excluded)
    uint32_t mism;     // no-drop mode: cycles of this run with a differing output
};

// Where a light lane hands an overflowing fault.
struct Promote {
    HeavyItem *items;
    uint32_t *count;
    uint32_t cap;
};

template <int KR, int KD, int KH>
__device__ __forceinline__ void light_run_fault(const DevDesign &D, const DevFaults &f, uint32_t fid,
                                                uint32_t tend, uint64_t budget, uint64_t load_before,
                                                Promote prom, uint64_t *rv, uint64_t *dv, uint32_t *rr,
                                                uint32_t *dn, uint32_t *hp, LightRun &r) {
    const uint32_t B = blockDim.x, tx = threadIdx.x;
#define RV(bf, k) rv[((bf) * KR + (k)) * B + tx]
#define RR(bf, k) rr[((bf) * KR + (k)) * B + tx]
#define DV(k) dv[(k) * B + tx]
#define DN(k) dn[(k) * B + tx]
#define HP(k) hp[(k) * B + tx]
    const uint32_t I = D.I, IR = D.I + D.R, T = D.T;
    const uint64_t *__restrict__ gcol = D.gcol;
    const uint4 *__restrict__ netinfo = D.netinfo;
    const uint4 *__restrict__ desc = D.desc;
    const uint32_t *__restrict__ fo_idx = D.fo_idx;
    const uint32_t *__restrict__ dreg_off = D.dreg_off;
    const uint32_t *__restrict__ dreg_rec = D.dreg_rec;
    const FaultSite fs = load_fault(f, fid);
    const uint32_t site = fs.site;
    const uint64_t *__restrict__ scol = gcol + (size_t)site * T;
    const uint32_t site_node = site >= IR ? site - IR : 0xFFFFFFFFu;
    const bool nodrop = f.mism != nullptr;
    bool seen = nodrop && f.res_det[fid] == 1;   // no-drop: first detection already recorded

    uint32_t t = r.t, nreg = r.nreg, cur = 0, mism = 0;
    uint64_t load = 0;
    int status = 0;
    int32_t det_cycle = -1, det_port = -1;
    // A detection at cycle t on `port`: stop (dropping), or record the first one and count.
    auto detect = [&](uint32_t port) -> bool {
        if (!nodrop) {
            det_cycle = (int32_t)t;
            det_port = (int32_t)port;
            status = 1;
            return true;
        }
        if (!seen) {
            f.res_det[fid] = 1;
            f.res_cycle[fid] = (int32_t)t;
            f.res_port[fid] = (int32_t)port;
            seen = true;
        }
        ++mism;
        return false;
    };

    for (;;) {
        if (nreg == 0) {
            // Nothing latched: skip to the next cycle in which the fault acts by itself.
            // With the activation bitplane, 64 cycles per load; else four cycles per step.
            if (fs.kind == FK_FLIP) {
                t = t <= fs.t0 ? min(fs.t0, tend) : tend;
            } else if (f.act) {
                t = next_active(f.act + (size_t)fid * f.act_stride, t, tend);
            } else {
                const uint64_t want = fs.kind == FK_SA1 ? fs.bm : 0ull;   // quiescent: bit == stuck
                while (t + 4 <= tend) {
                    const uint64_t g0 = __ldg(scol + t), g1 = __ldg(scol + t + 1);
                    const uint64_t g2 = __ldg(scol + t + 2), g3 = __ldg(scol + t + 3);
                    if ((g0 & fs.bm) != want) break;
                    if ((g1 & fs.bm) != want) { t += 1; break; }
                    if ((g2 & fs.bm) != want) { t += 2; break; }
                    if ((g3 & fs.bm) != want) { t += 3; break; }
                    t += 4;
                }
                if (t + 4 > tend) {
                    while (t < tend && (__ldg(scol + t) & fs.bm) == want) ++t;
                }
            }
            if (t >= tend) break;
            if (fs.port != NO_PORT) {
                // a port fault changes only what its port observes of the site net: the
                // machines differ exactly in the cycles the fault acts (virtual node evaluated)
                ++load;
                if (detect(fs.port)) break;
                if (++t >= tend) break;
                if (budget && load_before + load > budget) { status = 3; break; }
                continue;
            }
        }
        const uint32_t nb = cur ^ 1u;
        uint32_t nd = 0, nh = 0, nreg_new = 0, minport = NI_NO_PORT;
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
        // Keep net (faulty v, good g, record ni): diff entry, detection, fan-out, latch.
        auto add_diff = [&](uint32_t net, uint64_t v, uint64_t g, uint4 ni) {
            if (nd >= (uint32_t)KD) { ovf = true; return; }
            DN(nd) = net;
            DV(nd) = v;
            ++nd;
            filter |= 1ull << (net & 63u);
            const uint32_t p = ni_port(ni.w);
            minport = p < minport ? p : minport;
            if (ni.y - ni.x > (uint32_t)KH) { ovf = true; return; }
            for (uint32_t e = ni.x; e < ni.y; e += 4) {
                // four independent loads in flight, then the pushes
                const uint32_t c0 = __ldg(fo_idx + e);
                const uint32_t c1 = e + 1 < ni.y ? __ldg(fo_idx + e + 1) : 0xFFFFFFFFu;
                const uint32_t c2 = e + 2 < ni.y ? __ldg(fo_idx + e + 2) : 0xFFFFFFFFu;
                const uint32_t c3 = e + 3 < ni.y ? __ldg(fo_idx + e + 3) : 0xFFFFFFFFu;
                heap_push(c0);
                if (c1 != 0xFFFFFFFFu) heap_push(c1);
                if (c2 != 0xFFFFFFFFu) heap_push(c2);
                if (c3 != 0xFFFFFFFFu) heap_push(c3);
            }
            uint32_t nr = ni_nreg(ni.w);
            if (nr) {
                if (nr == 255u) nr = __ldg(dreg_off + net + 1) - ni.z;
                for (uint32_t e = ni.z; e < ni.z + nr; ++e) {
                    const uint32_t rec = __ldg(dreg_rec + e);   // register | width << 25
                    const uint32_t rg = rec & 0x1FFFFFFu;
                    const uint64_t wm = wmask(rec >> 25);
                    const uint64_t qv = v & wm;
                    if (qv != (g & wm)) {
                        if (nreg_new >= (uint32_t)KR) { ovf = true; return; }
                        RR(nb, nreg_new) = rg;
                        RV(nb, nreg_new) = qv;
                        ++nreg_new;
                    }
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
            if (net == site) { qv = fs.apply(qv, t); site_seeded = true; }
            const uint64_t g = __ldg(gcol + (size_t)net * T + t);
            if (qv != g) add_diff(net, qv, g, __ldg(netinfo + net));
        }
        if (site < IR && !site_seeded && !ovf) {
            const uint64_t g = __ldg(scol + t);
            const uint64_t fv = fs.apply(g, t);
            if (fv != g) add_diff(site, fv, g, __ldg(netinfo + site));
        }
        if (site_node != 0xFFFFFFFFu && fs.acts(t) && !ovf) heap_push(site_node);
        uint32_t last = 0xFFFFFFFFu;
        while (nh > 0 && !ovf) {
            const uint32_t n = heap_pop();
            if (n == last) continue;
            last = n;
            const uint32_t net = IR + n;
            // independent loads first: descriptor, net record, good value
            const uint4 d = __ldg(desc + n);
            const uint4 ni = __ldg(netinfo + net);
            const uint64_t g = __ldg(gcol + (size_t)net * T + t);
            const uint32_t op = meta_op(d.w);
            const int no = n_operands(op);
            uint64_t a = 0, b = 0, c = 0;
            if (no >= 1) a = lookup(d.x);
            if (no >= 2) b = lookup(d.y);
            if (no >= 3) c = lookup(d.z);
            uint64_t v = eval_op(d, a, b, c);
            if (n == site_node) v = fs.apply(v, t);
            ++load;
            if (v != g) add_diff(net, v, g, ni);
        }
        if (ovf) {
            const uint32_t p = atomicAdd(prom.count, 1u);
            if (p < prom.cap) {
                HeavyItem &h = prom.items[p];
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
        if (minport != NI_NO_PORT && detect(minport)) break;
        cur = nb;
        nreg = nreg_new;
        if (++t >= tend) break;
        if (budget && load_before + load > budget) { status = 3; break; }
    }
    r.t = t;
    r.nreg = nreg;
    r.cur = cur;
    r.status = status;
    r.det_cycle = det_cycle;
    r.det_port = det_port;
    r.load = load;
    r.mism = mism;
}

// Carve a light CTA's dynamic shared memory: [2][KR][B] register values, [KD][B] diff
// values, [2][KR][B] register ids, [KD][B] diff nets, [KH][B] heap.
#define LIGHT_CARVE                                                     \
    extern __shared__ __align__(16) unsigned char lsm[];                \
    const uint32_t B = blockDim.x, tx = threadIdx.x;                    \
    uint64_t *rv = reinterpret_cast<uint64_t *>(lsm);                   \
    uint64_t *dv = rv + 2 * KR * B;                                     \
    uint32_t *rr = reinterpret_cast<uint32_t *>(dv + KD * B);           \
    uint32_t *dn = rr + 2 * KR * B;                                     \
    uint32_t *hp = dn + KD * B;

// Final result of a fault that stopped (detected, over budget, or at the design's last
// cycle); in no-drop mode a detection was recorded when it happened.
__device__ __forceinline__ void light_finish(const DevFaults &f, uint32_t fid, const LightRun &r,
                                             unsigned long long *budget_hit) {
    if (r.status == 0 && f.mism) return;
    f.res_det[fid] = r.status == 1 ? 1 : r.status == 3 ? 255 : 0;
    f.res_cycle[fid] = r.det_cycle;
    f.res_port[fid] = r.det_port;
    if (r.status == 3) atomicAdd(budget_hit, 1ull);
}

template <int KR, int KD, int KH>
__global__ void __launch_bounds__(256, 1)
light_kernel(const DevDesign *__restrict__ designs, DevFaults f, Queues q) {
    LIGHT_CARVE
    (void)tx;
    const Promote prom{q.heavy_items, q.heavy_count, q.heavy_cap};
    for (;;) {
        const unsigned long long qi = atomicAdd(q.light_head, 1ull);
        if (qi >= q.n_light) break;
        const uint32_t fid = q.light_order[qi];
        const DevDesign &D = designs[f.design[fid]];
        LightRun r{0, 0, 0, 0, -1, -1, 0, 0};
        light_run_fault<KR, KD, KH>(D, f, fid, D.T, q.fault_budget, 0, prom, rv, dv, rr, dn, hp, r);
        f.load[fid] = r.load;
        if (f.mism) f.mism[fid] += r.mism;
        if (r.status != 2) light_finish(f, fid, r, q.budget_hit);
        // t is the first cycle not completed (a detection cycle counts as simulated)
        atomicAdd(q.counters + 0, (unsigned long long)r.load);
        atomicAdd(q.counters + 1, (unsigned long long)(r.status == 1 ? r.t + 1 : r.t));
    }
}

// Windowed light kernel: the light kernel over cycles [t0, t1) of the live faults;
// survivors carry their register diffs to the next window.
template <int KR, int KD, int KH>
__global__ void __launch_bounds__(256, 1)
light_window_kernel(const DevDesign *__restrict__ designs, DevFaults f, WinLight q) {
    LIGHT_CARVE
    const Promote prom{q.prom, q.prom_total, q.prom_cap};
    const uint32_t n_live = *q.n_live_in;
    const uint32_t lane = tx & 31u;
    for (;;) {
        const unsigned long long qi = atomicAdd(q.head, 1ull);
        if (qi >= n_live) break;
        // Survivors were appended in the order they finished the last window, slowest last:
        // take them back to front so the slowest start first (longest processing time first).
        const uint32_t fid = q.live_in[q.reverse ? n_live - 1 - (uint32_t)qi : (uint32_t)qi];
        const DevDesign &D = designs[f.design[fid]];
        const uint32_t tend = min(q.t1, D.T);     // this window ends at tend
        LightRun r{q.t0, q.st_nreg[fid], 0, 0, -1, -1, 0, 0};
        for (uint32_t k = 0; k < r.nreg; ++k) {   // register diffs carried from the last window
            RR(0, k) = q.st_r[(size_t)k * q.F + fid];
            RV(0, k) = q.st_v[(size_t)k * q.F + fid];
        }
        const uint64_t load_before = f.load[fid];
        light_run_fault<KR, KD, KH>(D, f, fid, tend, q.fault_budget, load_before, prom, rv, dv, rr, dn, hp, r);
        f.load[fid] = load_before + r.load;
        if (f.mism) f.mism[fid] += r.mism;
        if (r.status == 1 || r.status == 3 || (r.status == 0 && tend == D.T)) {
            light_finish(f, fid, r, q.budget_hit);
        } else if (r.status == 0) {
            // alive at the end of the window: carry the register diffs, append to the
            // survivors (warp-aggregated: one atomic per group of lanes arriving together)
            q.st_nreg[fid] = (uint8_t)r.nreg;
            for (uint32_t k = 0; k < r.nreg; ++k) {
                q.st_r[(size_t)k * q.F + fid] = RR(r.cur, k);
                q.st_v[(size_t)k * q.F + fid] = RV(r.cur, k);
            }
            const unsigned m = __activemask();
            const int leader = __ffs(m) - 1;
            const unsigned rank = __popc(m & ((1u << lane) - 1u));
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(q.n_live_out, (uint32_t)__popc(m));
            base = __shfl_sync(m, base, leader);
            q.live_out[base + rank] = fid;
        }
        // t is the first cycle not completed (a detection cycle counts as simulated)
        atomicAdd(q.counters + 0, (unsigned long long)r.load);
        atomicAdd(q.counters + 1, (unsigned long long)((r.status == 1 ? r.t + 1 : r.t) - q.t0));
    }
}
#undef LIGHT_CARVE
#undef RV
#undef RR
#undef DV
#undef DN
#undef HP

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
    const FaultSite fs = load_fault(f, fid);
    const uint32_t site = fs.site;
    const bool nodrop = f.mism != nullptr;
    uint32_t nreg = 0, cur = 0, epoch = 0, mism = 0;
    uint64_t load = 0;
    int32_t det_cycle = -1, det_port = -1;
    for (uint32_t t = 0; t < T; ++t) {
        ++epoch;
        if (fs.port != NO_PORT) {
            // a port fault: the machines differ exactly where the fault changes what the
            // port observes of the (good) site net
            const uint64_t g = gcol[(size_t)site * T + t];
            if (fs.apply(g, t) == g) continue;
            ++load;
            if (det_cycle < 0) { det_cycle = (int32_t)t; det_port = (int32_t)fs.port; }
            ++mism;
            if (!nodrop) break;
            continue;
        }
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
            if (net == site) { qv = fs.apply(qv, t); site_seeded = true; }
            const uint64_t g = gcol[(size_t)net * T + t];
            if (qv != g) keep(net, qv, g);
        }
        if (site < IR && !site_seeded) {
            const uint64_t g = gcol[(size_t)site * T + t];
            const uint64_t fv = fs.apply(g, t);
            if (fv != g) keep(site, fv, g);
        }
        if (site >= IR && fs.acts(t)) push(site - IR);
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
            if (net == site) v = fs.apply(v, t);
            ++load;
            const uint64_t g = gcol[(size_t)net * T + t];
            if (v != g) keep(net, v, g);
        }
        if (minport != NO_PORT) {
            if (det_cycle < 0) { det_cycle = (int32_t)t; det_port = (int32_t)minport; }
            ++mism;
            if (!nodrop) break;
        }
        nreg = nreg_new;
        cur = nb;
    }
    f.load[fid] = load;
    if (nodrop) f.mism[fid] = mism;
    f.res_det[fid] = det_cycle >= 0 ? 1 : 0;
    f.res_cycle[fid] = det_cycle;
    f.res_port[fid] = det_port;
}

// ---- launchers -----------------------------------------------------------------------

size_t good_smem_bytes(bool use_smem, uint32_t max_net, uint32_t max_reg, uint32_t max_chunks, bool staged) {
    const size_t vwords = use_smem ? (size_t)max_net + max_reg : 0;
    if (staged)
        return ((vwords + 1) & ~(size_t)1) * sizeof(uint64_t) + (size_t)GOOD_NSTAGE * GOOD_BLOCK * 16 +
               (size_t)max_chunks * sizeof(uint2);
    return vwords * sizeof(uint64_t) + (size_t)max_chunks * sizeof(uint2);
}

cudaError_t launch_good_trace(const DevDesign *d_designs, const uint32_t *design_list,
                              uint32_t n_list, uint32_t max_net, uint32_t max_reg,
                              uint32_t max_chunks, bool use_smem, bool staged, uint32_t *err,
                              cudaStream_t stream, uint32_t t_begin, uint32_t t_end) {
    if (n_list == 0) return cudaSuccess;
    const size_t smem = good_smem_bytes(use_smem, max_net, max_reg, max_chunks, staged);
    cudaError_t e;
    if (staged) {
        const void *fn = use_smem ? (const void *)good_trace_staged_kernel<true> : (const void *)good_trace_staged_kernel<false>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (!use_smem) max_net = max_reg = 0;
        void *args[] = {(void *)&d_designs, (void *)&design_list, (void *)&max_net, (void *)&max_reg,
                        (void *)&max_chunks, (void *)&err, (void *)&t_begin, (void *)&t_end};
        return cudaLaunchKernel(fn, dim3(n_list), dim3(GOOD_BLOCK + 32), args, smem, stream);
    }
    if (use_smem) {
        e = cudaFuncSetAttribute(good_trace_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        good_trace_kernel<true><<<n_list, GOOD_BLOCK, smem, stream>>>(d_designs, design_list, max_net,
                                                                     max_reg, max_chunks,
                                                                     t_begin, t_end);
    } else {
        e = cudaFuncSetAttribute(good_trace_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        good_trace_kernel<false><<<n_list, GOOD_BLOCK, smem, stream>>>(d_designs, design_list, 0, 0,
                                                                      max_chunks, t_begin, t_end);
    }
    return cudaGetLastError();
}

size_t good_cluster_smem_bytes(uint32_t own, uint32_t rown, uint32_t n_inputs, uint32_t max_chunks) {
    const size_t vwords = (size_t)own + 2 * (size_t)rown + n_inputs;
    return ((vwords + 1) & ~(size_t)1) * sizeof(uint64_t) + (size_t)max_chunks * 16;
}

static cudaError_t good_cluster_attrs(uint32_t C, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(good_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(good_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

int good_cluster_max_active(uint32_t C, size_t smem) {
    if (good_cluster_attrs(C, smem) != cudaSuccess) { cudaGetLastError(); return 0; }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(GOOD_BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)good_cluster_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_good_cluster(const DevDesign *d_designs, const uint32_t *design_list,
                                uint32_t n_list, uint32_t C, size_t smem, uint32_t *err,
                                cudaStream_t stream, uint32_t t_begin, uint32_t t_end) {
    if (n_list == 0) return cudaSuccess;
    cudaError_t e = good_cluster_attrs(C, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(n_list * C);
    cfg.blockDim = dim3(GOOD_BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, good_cluster_kernel, d_designs, design_list, C, err, t_begin, t_end);
}

cudaError_t launch_transpose(uint64_t *gcol, const uint64_t *rows, uint32_t n_net, uint32_t T,
                             cudaStream_t stream) {
    dim3 grid((n_net + 31) / 32, (T + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, stream>>>(gcol, rows, n_net, T);
    return cudaGetLastError();
}

cudaError_t launch_activation(const DevDesign *d_designs, DevFaults f, uint64_t *act, uint32_t t0,
                              uint32_t t1, cudaStream_t stream) {
    if (!f.F || t1 <= t0) return cudaSuccess;
    activation_kernel<<<(f.F + 7) / 8, 256, 0, stream>>>(d_designs, f, act, t0, t1);
    return cudaGetLastError();
}

cudaError_t launch_transpose_window(const DevDesign *d_designs, uint32_t n_designs, uint32_t max_net,
                                    uint32_t t0, uint32_t t1, cudaStream_t stream) {
    if (!n_designs || t1 <= t0) return cudaSuccess;
    dim3 grid((max_net + 31) / 32, (t1 - t0 + 31) / 32, n_designs), block(32, 8);
    transpose_window_kernel<<<grid, block, 0, stream>>>(d_designs, t0, t1);
    return cudaGetLastError();
}

static size_t light_smem(int cap, int block) {
    const int KR = LIGHT_CAPS[cap][0], KD = LIGHT_CAPS[cap][1], KH = LIGHT_CAPS[cap][2];
    return (size_t)block * ((2 * KR + KD) * sizeof(uint64_t) + (2 * KR + KD + KH) * sizeof(uint32_t));
}

template <int C>
static void *light_fn() {
    return (void *)light_kernel<LIGHT_CAPS[C][0], LIGHT_CAPS[C][1], LIGHT_CAPS[C][2]>;
}

static void *light_kernel_ptr(int cap) {
    return cap == 0 ? light_fn<0>() : cap == 1 ? light_fn<1>() : light_fn<2>();
}

template <int C>
static void *light_window_fn() {
    return (void *)light_window_kernel<LIGHT_CAPS[C][0], LIGHT_CAPS[C][1], LIGHT_CAPS[C][2]>;
}

int light_max_blocks_per_sm(int cap, int block, bool window) {
    if (cap < 0 || cap > 2) return 0;
    int n = 0;
    const size_t smem = light_smem(cap, block);
    if (smem > 227 * 1024) return 0;
    void *fn = window ? (cap == 0 ? light_window_fn<0>() : cap == 1 ? light_window_fn<1>() : light_window_fn<2>())
                      : light_kernel_ptr(cap);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_light(const DevDesign *d_designs, DevFaults f, Queues q, int cap, int block,
                         int grid, cudaStream_t stream) {
    if (cap < 0 || cap > 2) return cudaErrorInvalidValue;
    const size_t smem = light_smem(cap, block);
    cudaError_t e = cudaFuncSetAttribute(light_kernel_ptr(cap),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&d_designs, (void *)&f, (void *)&q};
    return cudaLaunchKernel(light_kernel_ptr(cap), dim3(grid), dim3(block), args, smem, stream);
}

cudaError_t launch_light_window(const DevDesign *d_designs, DevFaults f, WinLight w, int cap,
                                int block, int grid, cudaStream_t stream) {
    if (cap < 0 || cap > 2) return cudaErrorInvalidValue;
    void *fn = cap == 0 ? light_window_fn<0>() : cap == 1 ? light_window_fn<1>() : light_window_fn<2>();
    const size_t smem = light_smem(cap, block);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&d_designs, (void *)&f, (void *)&w};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
}

size_t heavy_smem_bytes(uint32_t max_node, uint32_t max_levels, uint32_t max_net, bool exact, bool gbm) {
    const size_t side = exact ? (size_t)(max_net + 31) / 32 + HEAVY_DLIST : HEAVY_FILTER / 32;
    size_t words = heavy_node_words(max_node, gbm) + max_levels + HEAVY_NLIST + side;
    words = (words + 1) & ~(size_t)1;   // 8-byte alignment of the range list
    return words * sizeof(uint32_t) + HEAVY_FRANGE * sizeof(uint2) +
           (size_t)((max_levels + 63) / 64) * sizeof(unsigned long long);
}

static const void *heavy_fn(bool window, int block, bool exact, bool gbm = false) {
    if (gbm)   // one warp per fault, stamped net record
        return window ? (const void *)heavy_window_kernel<true, false, true> : (const void *)heavy_kernel<true, false, true>;
    if (window)
        return block == 32 ? (exact ? (const void *)heavy_window_kernel<true, true> : (const void *)heavy_window_kernel<true, false>)
                           : (exact ? (const void *)heavy_window_kernel<false, true> : (const void *)heavy_window_kernel<false, false>);
    return block == 32 ? (exact ? (const void *)heavy_kernel<true, true> : (const void *)heavy_kernel<true, false>)
                       : (exact ? (const void *)heavy_kernel<false, true> : (const void *)heavy_kernel<false, false>);
}

int heavy_max_blocks_per_sm(int block, size_t smem, bool exact, bool gbm) {
    int n = 0;
    const void *fn = heavy_fn(true, block, exact, gbm);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem);
    return n;
}

cudaError_t launch_heavy(const DevDesign *d_designs, DevFaults f, Queues q, HeavyScratch s,
                         int block, int grid, cudaStream_t stream) {
    const size_t smem = heavy_smem_bytes(s.max_node, s.max_levels, s.max_net, s.exact != 0, s.gbm != nullptr);
    const void *fn = heavy_fn(false, block, s.exact != 0, s.gbm != nullptr);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&d_designs, (void *)&f, (void *)&q, (void *)&s};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
}

cudaError_t launch_heavy_window(const DevDesign *d_designs, DevFaults f, WinHeavy w, HeavyScratch s,
                                int block, int grid, cudaStream_t stream) {
    const size_t smem = heavy_smem_bytes(s.max_node, s.max_levels, s.max_net, s.exact != 0, s.gbm != nullptr);
    const void *fn = heavy_fn(true, block, s.exact != 0, s.gbm != nullptr);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&d_designs, (void *)&f, (void *)&w, (void *)&s};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
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
