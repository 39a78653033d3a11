// Persistent serving kernel: the device-resident request loop of the
// continuous-batching service (the GPU side of the microservice Sec. 7
// proposes).
//
// The host publishes requests into a ring of host-mapped entries; the CTAs
// of one long-lived launch take work items (tickets) from a device counter
// and run each through the same per-item phases as the batch kernel
// (run_item), so a request's tile sums, and with the same reduction order
// its result, are bit-identical to qmccpw_greeks.  Every wait is bounded:
// a CTA whose ticket is not published within the idle limit leaves, and the
// host launches the kernel again when work arrives (the tickets held at
// exit are handed out first by that launch).  The protocol is described
// beside ServeRequest in qmccpw_internal.h.
#include <cuda_runtime.h>

#include <cstdint>

#include "fused_body.cuh"
#include "qmccpw_internal.h"

namespace qmccpw {
namespace {

static_assert(sizeof(ServeRequest) % 8 == 0, "ring entries are copied as 8-byte words");

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// loads of host-written words: system scope, not cached in L1
__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_sys(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint64_t *p, uint64_t v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }

// What thread 0 decided for the CTA's next step.
enum : int { kRunCached = 0, kRunLoad = 1, kLeave = 2 };

struct ServeShared {
    uint64_t ticket;   // the ticket held
    uint64_t seq;      // request to load (kRunLoad)
    int cmd;
    int last;          // this CTA finished a request's last item / is the last to leave
};

// Does request s start at or before ticket t?  An entry that no longer (or
// not consistently) holds s was reused, which the host does only after s and
// every request before it finished, so s lies before t's request: yes.
__device__ bool starts_at_or_before(const ServeParams &p, uint64_t s, uint64_t t) {
    const ServeRequest *e = p.ring + (s & (p.cap - 1));
    const uint64_t s1 = ld_acquire_sys(&e->seq);
    const uint64_t first = ld_relaxed_sys(&e->first_ticket);
    fence_acq_rel_sys();
    const uint64_t s2 = ld_relaxed_sys(&e->seq);
    if (s1 != s || s2 != s) return true;
    return first <= t;
}

// The request holding a published ticket: the last one in [oldest live,
// published) starting at or before it (binary search over the ring).
__device__ uint64_t find_request(const ServeParams &p, uint64_t t) {
    uint64_t lo = ld_acquire_sys(&p.ctl->oldest_live);
    uint64_t hi = ld_acquire_sys(&p.ctl->published_seq);
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (starts_at_or_before(p, mid, t)) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Thread 0: take a ticket (carried ones first), wait until it is published
// (bounded by the idle limit, a spin count and the stop word), and find its
// request.  On leaving, the held ticket is recorded for the next launch.
__device__ void claim(const ServeParams &p, const ServeRequest &cached, ServeShared &sh) {
    ServeState *st = p.st;
    const unsigned rc = *reinterpret_cast<volatile unsigned *>(&st->retry_count);
    uint64_t t = 0;
    bool have = false;
    if (*reinterpret_cast<volatile unsigned *>(&st->retry_next) < rc) {
        const unsigned i = atomicAdd(&st->retry_next, 1u);
        if (i < rc) {
            t = __ldcg(&st->retry[i]);
            have = true;
        }
    }
    if (!have) t = atomicAdd(&st->next_ticket, 1ull);
    sh.ticket = t;
    const uint64_t t0 = now_ns();
    const uint64_t max_spins = p.idle_ns / 16 + 4096;  // a second bound, should the timer stall
    unsigned sleep_ns = 32;
    for (uint64_t spin = 0;; ++spin) {
        if (t < ld_acquire_sys(&p.ctl->published_tickets)) break;
        if (ld_relaxed_sys(&p.ctl->stop) != 0u || now_ns() - t0 > p.idle_ns || spin > max_spins) {
            st->abandoned[blockIdx.x] = t;
            sh.cmd = kLeave;
            return;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 1024) sleep_ns *= 2;
    }
    if (cached.seq != ~0ull && t >= cached.first_ticket && t - cached.first_ticket < cached.items) {
        sh.cmd = kRunCached;  // the cached request is live (t is not done), so its copy is current
        return;
    }
    // the entry found must hold a request whose tickets contain t (checked
    // under the sequence lock); a few searches, then the launch ends with an
    // error rather than running an item of the wrong request
    for (int attempt = 0; attempt < 8; ++attempt) {
        const uint64_t s = find_request(p, t);
        const ServeRequest *e = p.ring + (s & (p.cap - 1));
        const uint64_t s1 = ld_acquire_sys(&e->seq);
        const uint64_t first = ld_relaxed_sys(&e->first_ticket);
        const uint64_t items = ld_relaxed_sys(&e->items);
        fence_acq_rel_sys();
        const uint64_t s2 = ld_relaxed_sys(&e->seq);
        if (s1 == s && s2 == s && t >= first && t - first < items) {
            sh.seq = s;
            sh.cmd = kRunLoad;
            return;
        }
    }
    st->abandoned[blockIdx.x] = t;
    atomicExch(&st->bad_ticket, 1u);  // the ring did not hold the ticket's request: reported as reason 4
    sh.cmd = kLeave;
}

// All threads: copy ring entry `seq` (live, so not rewritten) to shared memory.
__device__ void load_request(const ServeParams &p, uint64_t seq, ServeRequest &req) {
    const uint64_t *src = reinterpret_cast<const uint64_t *>(p.ring + (seq & (p.cap - 1)));
    uint64_t *dst = reinterpret_cast<uint64_t *>(&req);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(ServeRequest) / 8); i += blockDim.x)
        dst[i] = ld_relaxed_sys(src + i);
}

// All threads of the CTA that finished the request's last item: replicate
// estimates in tile order (reduce_replicate, as the batch reduction), the
// statistics, the results to the host-mapped output, then the flag.
__device__ void finish_request(const ServeParams &p, const ServeRequest &req, unsigned char *smem) {
    __threadfence();
    Neumaier(*part)[4] = reinterpret_cast<Neumaier(*)[4]>(smem);
    const ContractDev &c = req.c;
    const uint64_t tiles = static_cast<uint64_t>(c.tiles);
    double *per_rep = req.tile_sums + req.items * 4;
    for (int r = 0; r < c.R; ++r) {
        const double v = reduce_replicate(req.tile_sums + static_cast<uint64_t>(r) * tiles * 4, tiles, c.N, part);
        if (threadIdx.x < 4) per_rep[r * 4 + threadIdx.x] = v;
    }
    __syncthreads();
    double *out = req.out;
    for (int i = threadIdx.x; i < 4 * c.R; i += blockDim.x) out[i] = per_rep[i];
    if (threadIdx.x < 4) {
        double mean, se;
        replicate_stats(per_rep, c.R, threadIdx.x, mean, se);
        out[4 * c.R + threadIdx.x] = mean;
        out[4 * c.R + 4 + threadIdx.x] = se;
    }
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t slot = req.seq & (p.cap - 1);
        p.done_items[slot] = 0;  // the next request in this entry counts from zero
        __threadfence();
        st_release_sys(p.done + slot, req.seq + 1);
    }
}

// All threads of a leaving CTA.  The last CTA to leave hands the tickets
// held at exit, and the carried ones nobody took, to the next launch, in
// ticket order (oldest work first), and writes the exit record.
__device__ void leave(const ServeParams &p, ServeShared &sh, unsigned char *smem, size_t smem_bytes) {
    ServeState *st = p.st;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh.last = atomicAdd(&st->exited, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    const unsigned rc = *reinterpret_cast<volatile unsigned *>(&st->retry_count);
    const unsigned rn = min(*reinterpret_cast<volatile unsigned *>(&st->retry_next), rc);
    const unsigned total = gridDim.x + (rc - rn);
    uint32_t reason = ld_relaxed_sys(&p.ctl->stop) != 0u ? 2u : 1u;
    if (*reinterpret_cast<volatile unsigned *>(&st->bad_ticket) != 0u) reason = 4u;
    unsigned long long *list = reinterpret_cast<unsigned long long *>(smem);
    if (total > static_cast<unsigned>(kServeRetryCap) || total * sizeof(unsigned long long) > smem_bytes) {
        reason = 3u;  // cannot happen with a fixed grid (at most 2 x grid tickets are carried)
    } else {
        for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) list[i] = __ldcg(&st->abandoned[i]);
        for (unsigned i = threadIdx.x; i < rc - rn; i += blockDim.x) list[gridDim.x + i] = __ldcg(&st->retry[rn + i]);
        __syncthreads();
        // rank sort: the tickets are distinct
        for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
            const unsigned long long v = list[i];
            unsigned rank = 0;
            for (unsigned j = 0; j < total; ++j) rank += list[j] < v ? 1u : 0u;
            st->retry[rank] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->retry_count = reason == 3u ? 0u : total;
        st->retry_next = 0;
        st->exited = 0;
        st->bad_ticket = 0;
        ServeExit *e = p.exit_rec;
        e->launch = p.launch;
        e->reason = reason;
        e->next_ticket = st->next_ticket;
        e->carried = total;
        __threadfence_system();
    }
}

// One item of a request, a separate (not inlined) function per construction:
// each keeps the register allocation the batch kernel's inlined form gets,
// and the serving kernel stays small enough for the compiler.
template <typename T, int CONS>
__device__ __noinline__ void serve_item(const ContractDev &c, const ServeParams &p, uint32_t rep, uint64_t tile,
                                        double *tile_out, unsigned char *smem) {
    run_item<T, CONS>(c, p.sobol_table, p.sobol_shift, p.jstride, rep, tile, 0, nullptr, tile_out, smem);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) serve_kernel(const __grid_constant__ ServeParams p, uint32_t smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) ServeRequest req;
    __shared__ ServeShared sh;
    if (threadIdx.x == 0) req.seq = ~0ull;
    __syncthreads();
    while (true) {
        if (threadIdx.x == 0) claim(p, req, sh);
        __syncthreads();
        const int cmd = sh.cmd;
        if (cmd == kLeave) break;
        if (cmd == kRunLoad) {
            load_request(p, sh.seq, req);
            __syncthreads();
        }
        const ContractDev &c = req.c;
        const uint64_t local = sh.ticket - req.first_ticket;
        if (local >= req.items) {  // never expected: the entry was checked when found
            if (threadIdx.x == 0) {
                p.st->abandoned[blockIdx.x] = sh.ticket;
                atomicExch(&p.st->bad_ticket, 1u);
            }
            break;
        }
        const uint64_t tiles = static_cast<uint64_t>(c.tiles);
        const uint64_t r = local / tiles;
        const uint64_t tile = local - r * tiles;
        const uint32_t rep = static_cast<uint32_t>(r) + static_cast<uint32_t>(c.rep_first);
        double *tile_out = req.tile_sums + local * 4;
        switch (c.construction) {
            case QMCCPW_BB: serve_item<T, QMCCPW_BB>(c, p, rep, tile, tile_out, smem); break;
            case QMCCPW_STD: serve_item<T, QMCCPW_STD>(c, p, rep, tile, tile_out, smem); break;
            case QMCCPW_BB_LEAD: serve_item<T, QMCCPW_BB_LEAD>(c, p, rep, tile, tile_out, smem); break;
            case QMCCPW_PCA_LEAD: serve_item<T, QMCCPW_PCA_LEAD>(c, p, rep, tile, tile_out, smem); break;
            default: serve_item<T, QMCCPW_PCA>(c, p, rep, tile, tile_out, smem); break;
        }
        // the tile sums are written (run_item ends with a barrier); count the item
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0)
            sh.last = atomicAdd(p.done_items + (req.seq & (p.cap - 1)), 1ull) == req.items - 1;
        __syncthreads();
        if (sh.last) finish_request(p, req, smem);
    }
    leave(p, sh, smem, smem_bytes);
}

}  // namespace

int serve_prepare(int precision, size_t optin_bytes) {
    cudaFuncAttributes fa{};
    const void *f = precision == QMCCPW_FP64 ? reinterpret_cast<const void *>(serve_kernel<double>)
                                             : reinterpret_cast<const void *>(serve_kernel<float>);
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return static_cast<int>(e);
    return static_cast<int>(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(optin_bytes) - static_cast<int>(fa.sharedSizeBytes)));
}

int serve_occupancy(int precision, size_t smem_bytes, int *blocks_per_sm) {
    const void *f = precision == QMCCPW_FP64 ? reinterpret_cast<const void *>(serve_kernel<double>)
                                             : reinterpret_cast<const void *>(serve_kernel<float>);
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem_bytes));
}

int launch_serve(const ServeParams &p, int precision, size_t smem_bytes, int grid, void *stream) {
    if (grid < 1 || grid > kServeMaxGrid) return static_cast<int>(cudaErrorInvalidValue);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t sb = static_cast<uint32_t>(smem_bytes);
    if (precision == QMCCPW_FP64) serve_kernel<double><<<grid, kThreads, smem_bytes, s>>>(p, sb);
    else serve_kernel<float><<<grid, kThreads, smem_bytes, s>>>(p, sb);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace qmccpw
