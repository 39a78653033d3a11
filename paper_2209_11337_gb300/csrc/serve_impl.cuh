// Persistent serving kernel: the device-resident request loop of the
// continuous-batching service (the GPU side of the microservice Sec. 7
// proposes).  Included by serve_f32.cu and serve_f64.cu, one precision each.
//
// The host publishes requests into a ring of host-mapped entries.  The last
// CTA of the launch, the dispatcher, copies each newly published entry into
// a device ring and republishes it in device memory; the other CTAs, the
// workers, take work items (tickets) from a device counter and run each
// through the same per-item phases as the batch kernel (run_item), so a
// request's tile sums, and with the same reduction order its result, are
// bit-identical to qmccpw_greeks.  Workers read only device memory on the way
// to an item.  Every wait is bounded: a worker whose ticket is not published
// within the idle limit leaves, the dispatcher follows the last worker, and
// the host launches the kernel again when work arrives (the tickets held at
// exit are handed out first by that launch).  The protocol is described
// beside ServeRequest in qmccpw_internal.h.
#pragma once

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
// host-written words: system scope, not cached in L1
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
// device words shared by the CTAs of the launch: GPU scope
__device__ __forceinline__ uint64_t ld_acquire_gpu(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// What thread 0 decided for the CTA's next step.
enum : int { kRunCached = 0, kRunLoad = 1, kLeave = 2 };

struct ServeShared {
    uint64_t ticket;   // the ticket held
    uint64_t seq;      // request to load (kRunLoad)
    uint64_t from, to; // dispatcher: entries to copy
    int cmd;
    int last;          // this CTA finished a request's last item / is the last to leave
    int leave;         // dispatcher: leave now
};

// The device ring entry of request s, read consistently: false when the
// entry holds another request (reused after s finished) or was being written.
__device__ bool read_entry(const ServeParams &p, uint64_t s, uint64_t &first, uint64_t &items) {
    const ServeRequest *e = p.dev_ring + (s & (p.cap - 1));
    const uint64_t s1 = ld_acquire_gpu(&e->seq);
    first = ld_relaxed_gpu(&e->first_ticket);
    items = ld_relaxed_gpu(&e->items);
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    const uint64_t s2 = ld_relaxed_gpu(&e->seq);
    return s1 == s && s2 == s;
}

// The request holding a published ticket t: the last one in [oldest live,
// published) starting at or before it.  An entry that does not hold its
// request was reused, which the host does only after that request and every
// one before it finished, so it lies before t's request.  Forward probes
// from the request last run first (tickets are taken in order, so t's
// request is usually the next one), then a binary search.
__device__ uint64_t find_request(const ServeParams &p, uint64_t t, uint64_t hint) {
    uint64_t lo = ld_relaxed_gpu(&p.st->oldest_live);
    uint64_t hi = ld_acquire_gpu(&p.st->pub_seq);
    if (hint >= lo && hint < hi) {
        for (uint64_t s = hint; s < hi && s < hint + 4; ++s) {
            uint64_t first, items;
            if (!read_entry(p, s, first, items)) continue;
            if (t >= first && t - first < items) return s;
            if (first > t) break;
        }
    }
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        uint64_t first, items;
        if (!read_entry(p, mid, first, items) || first <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Worker thread 0: take a ticket (carried ones first), wait until it is
// published in device memory (bounded by the idle limit, a spin count and
// the stop word), and find its request.  On leaving, the held ticket is
// recorded for the next launch.
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
        if (t < ld_acquire_gpu(&st->pub_tickets)) break;
        if (ld_relaxed_gpu(&st->stop) != 0u || now_ns() - t0 > p.idle_ns || spin > max_spins) {
            st->abandoned[blockIdx.x] = t;
            sh.cmd = kLeave;
            return;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 512) sleep_ns *= 2;
    }
    if (cached.seq != ~0ull && t >= cached.first_ticket && t - cached.first_ticket < cached.items) {
        sh.cmd = kRunCached;  // the cached request is live (t is not done), so its copy is current
        return;
    }
    // the entry found must hold a request whose tickets contain t; a few
    // searches, then the launch ends with an error rather than running an
    // item of the wrong request
    const uint64_t hint = cached.seq != ~0ull ? cached.seq + 1 : 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        const uint64_t s = find_request(p, t, hint);
        uint64_t first, items;
        if (read_entry(p, s, first, items) && t >= first && t - first < items) {
            sh.seq = s;
            sh.cmd = kRunLoad;
            return;
        }
    }
    st->abandoned[blockIdx.x] = t;
    atomicExch(&st->bad_ticket, 1u);  // reported as exit reason 4
    sh.cmd = kLeave;
}

// All threads of a worker: copy device ring entry `seq` (live, so not being
// rewritten) to shared memory, past L1 (the entry's previous occupant may
// sit there).
__device__ void load_request(const ServeParams &p, uint64_t seq, ServeRequest &req) {
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(p.dev_ring + (seq & (p.cap - 1)));
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&req);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(ServeRequest) / 8); i += blockDim.x) dst[i] = __ldcg(src + i);
}

// All threads of the worker that finished the request's last item:
// replicate estimates in tile order (reduce_replicate, as the batch
// reduction), the statistics, the results to the host-mapped output, then
// the flag.
__device__ void finish_request(const ServeParams &p, const ServeRequest &req, unsigned char *smem) {
    __threadfence();
    Neumaier(*part)[4] = reinterpret_cast<Neumaier(*)[4]>(smem);
    const ContractDev &c = req.c;
    const uint64_t items = static_cast<uint64_t>(c.items);
    double *per_rep = req.tile_sums + req.items * 4;
    for (int r = 0; r < c.R; ++r) {
        const double v = reduce_replicate(req.tile_sums + static_cast<uint64_t>(r) * items * 4, items, c.N, part);
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

// All threads of the dispatcher CTA: mirror the host's publications into
// device memory until every worker has left or the stop word is set (or,
// as a last bound, a minute without a new request).
__device__ void dispatch(const ServeParams &p, ServeShared &sh) {
    ServeState *st = p.st;
    const unsigned workers = gridDim.x - 1;
    uint64_t last_news = now_ns();
    const uint64_t limit = p.idle_ns + 60000000000ull;
    while (true) {
        if (threadIdx.x == 0) {
            const uint64_t host_seq = ld_acquire_sys(&p.ctl->published_seq);
            const uint32_t stop = ld_relaxed_sys(&p.ctl->stop);
            sh.from = ld_relaxed_gpu(&st->pub_seq);  // only this CTA writes it
            sh.to = host_seq;
            if (sh.to - sh.from > p.cap) sh.to = sh.from;  // never expected: the host keeps cap entries live at most
            if (stop) *reinterpret_cast<volatile uint32_t *>(&st->stop) = 1u;
            sh.leave = stop != 0u || ld_relaxed_gpu(&st->exited) >= workers || now_ns() - last_news > limit;
        }
        __syncthreads();
        const uint64_t from = sh.from, to = sh.to;
        if (to > from) {
            // copy the new entries: the sequence word as ~0 while a copy is written
            for (uint64_t s = from; s < to; ++s) {
                ServeRequest *d = p.dev_ring + (s & (p.cap - 1));
                const uint64_t *src = reinterpret_cast<const uint64_t *>(p.ring + (s & (p.cap - 1)));
                if (threadIdx.x == 0) st_relaxed_gpu(&d->seq, ~0ull);
                __threadfence();
                __syncthreads();
                uint64_t *dw = reinterpret_cast<uint64_t *>(d);
                for (int i = 1 + threadIdx.x; i < static_cast<int>(sizeof(ServeRequest) / 8); i += blockDim.x)
                    dw[i] = ld_relaxed_sys(src + i);
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) st_release_gpu(&d->seq, s);
            }
            if (threadIdx.x == 0) {
                // tickets of the copied requests only (the host's ticket word may already cover later ones)
                const ServeRequest *lastd = p.dev_ring + ((to - 1) & (p.cap - 1));
                const uint64_t end = ld_relaxed_gpu(&lastd->first_ticket) + ld_relaxed_gpu(&lastd->items);
                st_relaxed_gpu(&st->oldest_live, ld_relaxed_sys(&p.ctl->oldest_live));
                st_release_gpu(&st->pub_seq, to);
                st_release_gpu(&st->pub_tickets, end);
            }
            last_news = now_ns();
        } else if (threadIdx.x == 0) {
            st_relaxed_gpu(&st->oldest_live, ld_relaxed_sys(&p.ctl->oldest_live));
        }
        __syncthreads();
        if (sh.leave) break;
        if (to == from && threadIdx.x == 0) __nanosleep(256);
        __syncthreads();
    }
}

// All threads of a leaving CTA.  The last CTA to leave hands the tickets
// held at exit, and the carried ones nobody took, to the next launch, in
// ticket order (oldest work first), and writes the exit record.
__device__ void leave(const ServeParams &p, ServeShared &sh, unsigned char *smem, size_t smem_bytes) {
    ServeState *st = p.st;
    const unsigned workers = gridDim.x - 1;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh.last = atomicAdd(&st->exited, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    const unsigned rc = *reinterpret_cast<volatile unsigned *>(&st->retry_count);
    const unsigned rn = min(*reinterpret_cast<volatile unsigned *>(&st->retry_next), rc);
    const unsigned total = workers + (rc - rn);
    uint32_t reason = ld_relaxed_sys(&p.ctl->stop) != 0u ? 2u : 1u;
    if (*reinterpret_cast<volatile unsigned *>(&st->bad_ticket) != 0u) reason = 4u;
    unsigned long long *list = reinterpret_cast<unsigned long long *>(smem);
    if (total > static_cast<unsigned>(kServeRetryCap) || total * sizeof(unsigned long long) > smem_bytes) {
        reason = 3u;  // cannot happen with a fixed grid (at most 2 x workers tickets are carried)
    } else {
        for (unsigned i = threadIdx.x; i < workers; i += blockDim.x) list[i] = __ldcg(&st->abandoned[i]);
        for (unsigned i = threadIdx.x; i < rc - rn; i += blockDim.x) list[workers + i] = __ldcg(&st->retry[rn + i]);
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

// One item of a request (its tiles [tile, tile_end), their sums added to
// item_acc), a separate (not inlined) function per construction: each keeps
// the register allocation the batch kernel's inlined form gets, and the
// serving kernel stays small enough for the compiler.
template <typename T, int CONS>
__device__ __noinline__ void serve_item(const ContractDev &c, const ServeParams &p, uint32_t rep, uint32_t tile,
                                        uint32_t tile_end, double *item_acc, unsigned char *smem) {
    for (; tile < tile_end; ++tile)  // tiles per replicate fit 32 bits
        run_item<T, CONS>(c, p.sobol_table, p.sobol_shift, p.jstride, rep, tile, 0, nullptr, item_acc, smem);
}

// Workers are CTAs 0 .. gridDim.x - 2; the last CTA dispatches.  WITH_PCA
// false leaves the PCA product out (the float form then fits three CTAs per
// SM; the host accepts no PCA request for it).
template <typename T, bool WITH_PCA>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4 && !WITH_PCA) ? 3 : 2)
    serve_kernel(const __grid_constant__ ServeParams p, uint32_t smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) ServeRequest req;
    __shared__ ServeShared sh;
    if (blockIdx.x == gridDim.x - 1) {
        dispatch(p, sh);
        leave(p, sh, smem, smem_bytes);
        return;
    }
    __shared__ double item_acc[8];
    item_acc_clear(item_acc);
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
        if (local >= req.items || (!WITH_PCA && c.construction == QMCCPW_PCA)) {  // never expected
            if (threadIdx.x == 0) {
                p.st->abandoned[blockIdx.x] = sh.ticket;
                atomicExch(&p.st->bad_ticket, 1u);
            }
            break;
        }
        const uint64_t items = static_cast<uint64_t>(c.items);
        const uint64_t r = local / items;
        uint64_t tile64, tile_end64;
        item_tiles(c, local - r * items, tile64, tile_end64);
        const uint32_t tile = static_cast<uint32_t>(tile64), tile_end = static_cast<uint32_t>(tile_end64);
        const uint32_t rep = static_cast<uint32_t>(r) + static_cast<uint32_t>(c.rep_first);
        switch (c.construction) {
            case QMCCPW_BB: serve_item<T, QMCCPW_BB>(c, p, rep, tile, tile_end, item_acc, smem); break;
            case QMCCPW_STD: serve_item<T, QMCCPW_STD>(c, p, rep, tile, tile_end, item_acc, smem); break;
            case QMCCPW_BB_LEAD: serve_item<T, QMCCPW_BB_LEAD>(c, p, rep, tile, tile_end, item_acc, smem); break;
            case QMCCPW_PCA_LEAD: serve_item<T, QMCCPW_PCA_LEAD>(c, p, rep, tile, tile_end, item_acc, smem); break;
            default:
                if constexpr (WITH_PCA) serve_item<T, QMCCPW_PCA>(c, p, rep, tile, tile_end, item_acc, smem);
                break;
        }
        item_flush<PointValue<T>>(req.tile_sums + local * 4, item_acc);
        // the item's sums are written (run_item ends with a barrier); count the item
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0)
            sh.last = atomicAdd(p.done_items + (req.seq & (p.cap - 1)), 1ull) == req.items - 1;
        __syncthreads();
        if (sh.last) finish_request(p, req, smem);
    }
    leave(p, sh, smem, smem_bytes);
}

template <typename K>
int serve_prepare_kernel(K kernel, size_t optin_bytes) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return static_cast<int>(e);
    return static_cast<int>(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(optin_bytes) - static_cast<int>(fa.sharedSizeBytes)));
}

template <typename K>
int serve_launch_kernel(K kernel, const ServeParams &p, size_t smem_bytes, int grid, void *stream) {
    if (grid < 2 || grid > kServeMaxGrid) return static_cast<int>(cudaErrorInvalidValue);
    kernel<<<grid, kThreads, smem_bytes, static_cast<cudaStream_t>(stream)>>>(p, static_cast<uint32_t>(smem_bytes));
    return static_cast<int>(cudaGetLastError());
}

}  // namespace
}  // namespace qmccpw
