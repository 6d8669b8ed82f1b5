// rtlfs_static.cu -- allocation-free fault simulation: a variant of the plain
// one-thread-per-fault kernel whose per-thread scratch lives in one file-scope device
// array instead of memory obtained from cudaMalloc.
//
// Who needs it: callers that cannot obtain device memory from cudaMalloc where they run --
// a process whose device memory is owned by another allocator (a framework's caching pool
// that has reserved the GPU, which this library cannot call into), and latency-critical
// paths that cannot afford an allocation or the device-wide synchronisation cudaMalloc
// and cudaFree can imply. Such a caller passes its own device buffers for the faults and
// the results; the design and its good trace come from a context that was set up earlier.
//
// The array below is part of the library image: every GPU that loads the library keeps
// its 64 MiB until the process exits. Every call shares it, it keeps the contents the last
// call left, and two calls whose work overlaps on the GPU race on it.
#include "rtlfs_internal.h"
#include "rtlfs_static.h"

#include <mutex>

namespace rtlfs {

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Host side: the device address of g_static_scratch, looked up once per device. In host
// code the name g_static_scratch is only a host-side stand-in, not a device address.
cudaError_t static_scratch_address(int device, void **out) {
    static std::mutex mu;
    static void *addr[STATIC_MAX_DEVICES] = {};
    if (device < 0 || device >= STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        int prev = 0;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        e = cudaSetDevice(device);
        if (e != cudaSuccess) return e;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        addr[device] = p;
    }
    *out = addr[device];
    return cudaSuccess;
}

__device__ __forceinline__ uint64_t s_wmask(uint32_t w) {
    return w >= 64 ? ~0ull : ((1ull << w) - 1ull);
}

__device__ __forceinline__ int s_nops(uint32_t op) {
    return op == OP_CONST ? 0
         : (op == OP_NOT || op == OP_SHL || op == OP_SHR || op == OP_SLICE) ? 1
         : op == OP_MUX2 ? 3 : 2;
}

__device__ __forceinline__ uint64_t s_eval(uint4 d, uint64_t a, uint64_t b, uint64_t c) {
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
    default:        r = ((uint64_t)d.y << 32) | d.x; break;
    }
    return r & s_wmask(meta_w(m));
}

// One thread per fault of this wave; the wave's scratch is carved from the static array:
// [ext2int: n_net u32][error word][per thread: values u64, stamps u32, queued u32, heap u32,
// register diffs 2 x (u32 reg, u64 value)]. Stamps must be zero before the wave.
__global__ void __launch_bounds__(128)
plain_static_kernel(const DevDesign *__restrict__ designs, uint32_t design,
                    const StaticFault *__restrict__ faults, StaticResult *results,
                    uint32_t first, uint32_t count, unsigned char *arena, StaticLayout L) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= count) return;
    const uint32_t fi = first + tid;
    const DevDesign &D = designs[design];
    const uint32_t I = D.I, IR = D.I + D.R, T = D.T;
    const uint64_t *gcol = D.gcol;
    const uint32_t *ext2int = reinterpret_cast<const uint32_t *>(arena + L.ext2int_off);
    uint32_t *err = reinterpret_cast<uint32_t *>(arena + L.err_off);
    unsigned char *base = arena + L.thread_off + (size_t)tid * L.per_thread;
    uint64_t *fval = reinterpret_cast<uint64_t *>(base);
    uint64_t *regv = fval + L.sn;
    uint32_t *stamp = reinterpret_cast<uint32_t *>(regv + 2 * (size_t)L.sreg);
    uint32_t *qst = stamp + L.sn;
    uint32_t *hp = qst + L.snode;
    uint32_t *regr = hp + L.snode;

    const StaticFault fx = faults[fi];
    StaticResult out;
    out.cycle = -1;
    out.port = -1;
    out.detected = 0;
    out.reserved[0] = out.reserved[1] = out.reserved[2] = 0;
    if (fx.net >= D.n_net || fx.stuck > 1) {
        atomicOr(err, 1u);
        out.detected = 254;
        results[fi] = out;
        return;
    }
    const uint32_t site = ext2int[fx.net];
    if (fx.bit >= D.net_w[site]) {
        atomicOr(err, 1u);
        out.detected = 254;
        results[fi] = out;
        return;
    }
    const uint64_t bm = 1ull << fx.bit;
    const bool sv = fx.stuck != 0;
    auto force = [&](uint64_t x) { return sv ? (x | bm) : (x & ~bm); };
    uint32_t nreg = 0, cur = 0, epoch = 0;
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
                const uint64_t wm = s_wmask(D.net_w[I + r]);
                if ((v & wm) != (g & wm)) {
                    regr[nb * L.sreg + nreg_new] = r;
                    regv[nb * L.sreg + nreg_new] = v & wm;
                    ++nreg_new;
                }
            }
        };
        auto lookup = [&](uint32_t x) -> uint64_t {
            return stamp[x] == epoch ? fval[x] : gcol[(size_t)x * T + t];
        };
        bool site_seeded = false;
        for (uint32_t k = 0; k < nreg; ++k) {
            const uint32_t net = I + regr[cur * L.sreg + k];
            uint64_t qv = regv[cur * L.sreg + k];
            if (net == site) { qv = force(qv); site_seeded = true; }
            const uint64_t g = gcol[(size_t)net * T + t];
            if (qv != g) keep(net, qv, g);
        }
        if (site < IR && !site_seeded) {
            const uint64_t g = gcol[(size_t)site * T + t];
            const uint64_t fv = force(g);
            if (fv != g) keep(site, fv, g);
        }
        if (site >= IR) push(site - IR);
        while (nh > 0) {
            const uint32_t n = pop();
            const uint4 d = D.desc[n];
            const int no = s_nops(meta_op(d.w));
            uint64_t a = 0, b = 0, c = 0;
            if (no >= 1) a = lookup(d.x);
            if (no >= 2) b = lookup(d.y);
            if (no >= 3) c = lookup(d.z);
            const uint32_t net = IR + n;
            uint64_t v = s_eval(d, a, b, c);
            if (net == site) v = force(v);
            const uint64_t g = gcol[(size_t)net * T + t];
            if (v != g) keep(net, v, g);
        }
        if (minport != NO_PORT) {
            out.detected = 1;
            out.cycle = (int32_t)t;
            out.port = (int32_t)minport;
            break;
        }
        nreg = nreg_new;
        cur = nb;
    }
    results[fi] = out;
}

cudaError_t launch_plain_static(const DevDesign *d_designs, uint32_t design, const void *faults,
                                void *results, uint32_t first, uint32_t count, void *arena,
                                StaticLayout L, cudaStream_t stream) {
    if (!count) return cudaSuccess;
    plain_static_kernel<<<(count + 127) / 128, 128, 0, stream>>>(
        d_designs, design, (const StaticFault *)faults, (StaticResult *)results, first, count,
        (unsigned char *)arena, L);
    return cudaGetLastError();
}

}  // namespace rtlfs
