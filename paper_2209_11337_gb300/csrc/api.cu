// C-ABI of libqmccpw (declared in include/qmccpw.h): plans, batches and
// diagnostics.  Host code only validates, builds per-d tables, lays out the
// work list and enqueues kernels; every step of the estimator runs on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qmccpw_internal.h"

using namespace qmccpw;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define QMC_CUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? QMCCPW_ERR_OOM : QMCCPW_ERR_CUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

#define QMC_TRY(expr)                     \
    do {                                  \
        int rc_ = (expr);                 \
        if (rc_ != QMCCPW_OK) return rc_; \
    } while (0)

// device buffer with RAII release
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    int alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&ptr, b);
        if (e != cudaSuccess) {
            ptr = nullptr;
            return fail(QMCCPW_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        bytes = b;
        return QMCCPW_OK;
    }
    // grow-only: keep the allocation when it is already large enough
    int ensure(size_t b) { return (ptr && bytes >= b) ? QMCCPW_OK : alloc(b); }
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// Device arrays of one batch: contract descriptors, work list and results.
struct BatchBuffers {
    DevBuf contracts, item_base, rep_owner, tile_sums, per_rep, stats, counters;
    void release() {
        for (DevBuf *d : {&contracts, &item_base, &rep_owner, &tile_sums, &per_rep, &stats, &counters}) d->release();
    }
};

// Tables that depend only on d (and T through dt): bridge schedule and PCA factor.
struct DTables {
    int n = 0;
    int n_levels = 0;
    DevBuf steps, w64, w32, level_start, pca64, pca32;
    DevBuf pca32lo;  // A^T - float(A^T): the leading-coordinate PCA carries the factor as hi + lo
    DevBuf slot_dim;  // the bridge dimension that drives each date (the inverse of the steps' node)
    DevBuf sub_start[3];  // bridge subtrees per thread of a point, G = 2, 4, 8 (bridge_phase)
    DevBuf lead64, lead32;  // loadings of the leading coordinate, dates 1..n: bridge (j/sqrt(n)) then PCA (first column)
    double lead_sum[2] = {0.0, 0.0};  // the sum of each form's loadings
    int32_t lead_increasing[2] = {0, 0};  // each form's loadings strictly increase with the date
    DevBuf tc[2];  // tensor-core split operands of Ahat (bf16, tf32; resident or streamed form by n), built on first use
};

bool is_tc(int precision) { return precision == QMCCPW_MIXED_TC_BF16X3 || precision == QMCCPW_MIXED_TC_TF32X3; }
constexpr int kSegments = 6;  // launch segments of a batch (segment_of)
// Kernel precision of one contract: a tensor-core precision applies to the PCA
// product only; bridge contracts under it run as MIXED.
int contract_precision(int precision, int construction) {
    return (is_tc(precision) && construction != QMCCPW_PCA) ? QMCCPW_MIXED : precision;
}
// tensor-core kernel of a PCA contract with n dimensions: resident (n <= 64)
// bf16 0 / tf32 1, streamed (n <= 256) bf16 2 / tf32 3
int tc_kind(int precision, int n) {
    const int base = precision == QMCCPW_MIXED_TC_BF16X3 ? 0 : 1;
    return n > pca_tc_max_n(base) ? base + 2 : base;
}
int tc_slot(int precision) { return precision == QMCCPW_MIXED_TC_BF16X3 ? 0 : 1; }
// launch segment of a contract (kernel precision kp): 0 bridge, 1 standard
// construction, 2 PCA on the streamed tensor-core kernel, 3 other PCA, 4 and
// 5 the leading-coordinate bridge and PCA; one grid per segment present, in
// this order
int segment_of(int kp, int construction, int n) {
    if (construction == QMCCPW_BB) return 0;
    if (construction == QMCCPW_STD) return 1;
    if (construction == QMCCPW_BB_LEAD) return 4;
    if (construction == QMCCPW_PCA_LEAD) return 5;
    return (is_tc(kp) && tc_kind(kp, n) >= 2) ? 2 : 3;
}
int segment_construction(int seg) {
    static const int cons[kSegments] = {QMCCPW_BB, QMCCPW_STD, QMCCPW_PCA, QMCCPW_PCA, QMCCPW_BB_LEAD, QMCCPW_PCA_LEAD};
    return cons[seg];
}
bool is_lead(int construction) { return construction == QMCCPW_BB_LEAD || construction == QMCCPW_PCA_LEAD; }

}  // namespace

struct QmcServer;

struct qmccpw_plan_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t seed = 0;
    int d_max = 0, r_max = 0, ndims = 0, jstride = 0;
    size_t workspace_bytes = 0;
    int sm_count = 0;
    DevBuf err;          // int: error status set by device code (bounded waits)
    DevBuf dir;          // unscrambled direction integers, ndims x 32
    DevBuf table;        // [r][b][j]
    DevBuf shift;        // [r][j]
    // unit-spacing bridge / PCA tables, keyed by d
    std::map<int, std::unique_ptr<DTables>> dtables;
    // grow-only buffers reused by the one-shot entry points
    BatchBuffers ws;
    // tile sizes chosen by qmccpw_autotune / qmccpw_tuning_set: (precision, construction, d) -> log2 P
    std::map<std::tuple<int, int, int>, int> tuned_tile;
    std::mutex mu;
    struct QmcServer *server = nullptr;  // continuous-batching service, when started
};

struct qmccpw_batch_s {
    qmccpw_plan_t plan = nullptr;
    int count = 0;
    int precision = 0;
    std::vector<ContractDev> host;   // contracts in launch order: bridge first, then PCA
    std::vector<int32_t> order;      // order[i] = caller's index of host[i]
    std::vector<int32_t> R;
    uint64_t items = 0, total_reps = 0;
    // launch segments (segment_of): items [seg_begin[k], seg_begin[k + 1])
    uint64_t seg_begin[kSegments + 1] = {};
    size_t smem[kSegments] = {};
    int grid[kSegments] = {};
    BatchBuffers own;          // used by prepared batches
    BatchBuffers *buf = &own;  // one-shot calls point this at the plan's workspace
    // replicate estimates copied after every launch to caller rows (qmccpw_batch_scatter_replicates)
    double *scatter_dst = nullptr;
    DevBuf scatter_rows;  // int64 destination row of each replicate slot
    // diagnostics
    double *point_out = nullptr;
    uint64_t point_k0 = 0;
    uint32_t rep_offset = 0;
    // fused-kernel timing: event pairs of the most recent launches
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<cudaEvent_t> ev_seg;  // kSegments per slot: the end of each launch segment
    int32_t timed = 0;  // launches recorded since the last read
    // CUDA-graph replay (qmccpw_batch_use_graph): the launch sequence captured
    // once on a private stream, then one graph launch per call
    bool use_graph = false;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    void drop_graph() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        graph_exec = nullptr;
    }
    // forget the previous contracts, keep the device buffers for reuse
    void reset_meta() {
        count = 0;
        host.clear();
        order.clear();
        R.clear();
        items = total_reps = 0;
        for (int k = 0; k <= kSegments; ++k) seg_begin[k] = 0;
        for (int k = 0; k < kSegments; ++k) {
            smem[k] = 0;
            grid[k] = 0;
        }
        point_out = nullptr;
        point_k0 = 0;
        rep_offset = 0;
    }
    ~qmccpw_batch_s() {
        for (auto e : ev_start) cudaEventDestroy(e);
        for (auto e : ev_stop) cudaEventDestroy(e);
        for (auto e : ev_seg) cudaEventDestroy(e);
        drop_graph();
        if (capture_stream) cudaStreamDestroy(capture_stream);
    }
};

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int validate_contract(const qmccpw_plan_s *p, const qmccpw_option &o, const qmccpw_market &m, uint64_t N,
                      int32_t R, int32_t construction, int32_t precision, bool diagnostic) {
    if (o.type < 0 || o.type > 3) return fail(QMCCPW_ERR_INVALID_ARG, "option.type out of range");
    if (o.d < 1 || o.d > p->d_max)
        return fail(QMCCPW_ERR_INVALID_ARG, "option.d " + std::to_string(o.d) + " outside 1..d_max=" +
                                                std::to_string(p->d_max));
    if (!finite_pos(o.K) || !finite_pos(o.T)) return fail(QMCCPW_ERR_INVALID_ARG, "K and T must be positive and finite");
    if (!finite_pos(m.S0) || !finite_pos(m.sigma) || !std::isfinite(m.r))
        return fail(QMCCPW_ERR_INVALID_ARG, "S0, sigma must be positive and finite, r finite");
    if (N < 1 || N > (1ull << 32)) return fail(QMCCPW_ERR_INVALID_ARG, "N must be in 1..2^32");
    if (!diagnostic && (R < 2 || R > p->r_max))
        return fail(QMCCPW_ERR_INVALID_ARG, "R " + std::to_string(R) + " outside 2..r_max=" + std::to_string(p->r_max));
    if (construction < QMCCPW_BB || construction > QMCCPW_PCA_LEAD)
        return fail(QMCCPW_ERR_INVALID_ARG, "construction out of range");
    if (is_lead(construction) && o.d + 1 > QMCCPW_D_LIMIT)
        return fail(QMCCPW_ERR_INVALID_ARG, "d too large for the full-path construction");
    if (precision < QMCCPW_FP64 || precision > QMCCPW_MIXED_TC_TF32X3)
        return fail(QMCCPW_ERR_INVALID_ARG, "precision out of range");
    if (is_tc(precision) && construction == QMCCPW_PCA) {
        const int kind = tc_kind(precision, o.d - 1);
        if (o.d - 1 > pca_tc_max_n(kind))
            return fail(QMCCPW_ERR_UNSUPPORTED,
                        "tensor-core PCA supports d <= " + std::to_string(pca_tc_max_n(kind) + 1));
    }
    return QMCCPW_OK;
}

// A public contract descriptor: its replicate range within the plan's
// randomisation, then the option, market and sizes.
int validate_qc(const qmccpw_plan_s *p, const qmccpw_contract &c, int32_t precision, bool diagnostic) {
    if (static_cast<uint64_t>(c.first_point) + c.N > (1ull << 32))
        return fail(QMCCPW_ERR_INVALID_ARG, "first_point + N must be <= 2^32");
    if (c.first_replicate < 0 || (!diagnostic && static_cast<int64_t>(c.first_replicate) + c.R > p->r_max))
        return fail(QMCCPW_ERR_INVALID_ARG, "replicates first_replicate .. first_replicate + R - 1 must lie in "
                                            "0..r_max-1 (r_max=" + std::to_string(p->r_max) + ")");
    return validate_contract(p, c.option, c.market, c.N, c.R, c.construction, precision, diagnostic);
}

// Bridge / PCA tables of d dates for unit spacing (dt = 1), built on first use
// and cached by the plan: with equal spacing both factors scale exactly as
// sqrt(dt), which the kernels apply, so one table set serves every maturity.
int get_dtables(qmccpw_plan_s *p, int d, double /*T*/, const DTables **out) {
    auto it = p->dtables.find(d);
    if (it != p->dtables.end()) {
        *out = it->second.get();
        return QMCCPW_OK;
    }
    auto t = std::make_unique<DTables>();
    const int n = d - 1;
    const double dt = 1.0;
    t->n = n;
    BridgePlan bp = bridge_plan(n, dt);
    t->n_levels = static_cast<int>(bp.level_start.size()) - 1;
    // float bridge coefficients are carried as hi + lo (hi = float(x), lo = float(x - hi)),
    // which keeps the path covariance exact to ~2^-48 at three extra FMAs per node
    // bridge: 8 floats per step (wl hi/lo, wr hi/lo, sd hi/lo, 2 pad) so a step is two aligned float4
    std::vector<float> w32(8 * bp.steps.size(), 0.0f);
    for (size_t b = 0; b < bp.steps.size(); ++b)
        for (int k = 0; k < 3; ++k) {
            const double x = bp.w[3 * b + k];
            w32[8 * b + 2 * k] = static_cast<float>(x);
            w32[8 * b + 2 * k + 1] = static_cast<float>(x - static_cast<double>(w32[8 * b + 2 * k]));
        }
    std::vector<double> A = n > 0 ? pca_factor(n, dt) : std::vector<double>();
    // float A^T, rows k, columns i padded to a multiple of 16 (the register block of the product)
    const int n_pad = (n + 15) & ~15;
    std::vector<float> A32(static_cast<size_t>(n) * n_pad, 0.0f), A32lo(A32.size(), 0.0f);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = A[static_cast<size_t>(i) * n + k];
            A32[static_cast<size_t>(k) * n_pad + i] = static_cast<float>(a);
            A32lo[static_cast<size_t>(k) * n_pad + i] = static_cast<float>(a - static_cast<double>(static_cast<float>(a)));
        }
    QMC_TRY(t->steps.alloc(sizeof(BridgeStep) * std::max<size_t>(1, bp.steps.size())));
    QMC_TRY(t->w64.alloc(sizeof(double) * std::max<size_t>(1, bp.w.size())));
    QMC_TRY(t->w32.alloc(sizeof(float) * std::max<size_t>(1, w32.size())));
    QMC_TRY(t->level_start.alloc(sizeof(int32_t) * bp.level_start.size()));
    std::vector<int32_t> slot_dim(static_cast<size_t>(n) + 1, -1);
    for (int j = 0; j < n; ++j) slot_dim[bp.steps[j].m] = j;
    QMC_TRY(t->slot_dim.alloc(sizeof(int32_t) * slot_dim.size()));
    QMC_CUDA(cudaMemcpy(t->slot_dim.ptr, slot_dim.data(), sizeof(int32_t) * slot_dim.size(), cudaMemcpyHostToDevice));
    // G threads per point: after the top levels that leave G intervals, the
    // nodes of each deeper level that fall in interval g (the number of top
    // split dates below the node's date) are a contiguous run; its start per
    // (level, g), G + 1 entries per level
    for (int gi = 0; gi < 3; ++gi) {
        const int G = 2 << gi, top = gi + 2;
        const int levels = t->n_levels;
        std::vector<int32_t> ss;
        std::vector<int> splits;
        for (int lvl = 1; lvl < std::min(top, levels); ++lvl)
            for (int b = bp.level_start[lvl]; b < bp.level_start[lvl + 1]; ++b) splits.push_back(bp.steps[b].m);
        for (int lvl = top; lvl < levels; ++lvl) {
            const int b0 = bp.level_start[lvl], b1 = bp.level_start[lvl + 1];
            for (int g = 0; g <= G; ++g) {
                int b = b0;
                while (b < b1) {
                    int sub = 0;
                    for (int m : splits) sub += m < bp.steps[b].m ? 1 : 0;
                    if (sub >= g) break;
                    ++b;
                }
                ss.push_back(g == G ? b1 : b);
            }
        }
        if (ss.empty()) ss.push_back(0);
        QMC_TRY(t->sub_start[gi].alloc(sizeof(int32_t) * ss.size()));
        QMC_CUDA(cudaMemcpy(t->sub_start[gi].ptr, ss.data(), sizeof(int32_t) * ss.size(), cudaMemcpyHostToDevice));
    }
    QMC_TRY(t->pca64.alloc(sizeof(double) * std::max<size_t>(1, A.size())));
    QMC_TRY(t->pca32.alloc(sizeof(float) * std::max<size_t>(1, A32.size())));
    QMC_TRY(t->pca32lo.alloc(sizeof(float) * std::max<size_t>(1, A32lo.size())));
    // the leading coordinate's loading when these n dates are a whole path: the bridge's
    // terminal value (W~(s_i) = (i/n) sqrt(n) z), then the first principal component
    const int nl = std::max(1, n);
    std::vector<double> lead(2 * static_cast<size_t>(nl), 0.0);
    for (int i = 1; i <= n; ++i) {
        lead[i - 1] = static_cast<double>(i) / std::sqrt(static_cast<double>(n));
        lead[nl + i - 1] = A[static_cast<size_t>(i - 1) * n];
    }
    for (int i = 0; i < n; ++i) {
        t->lead_sum[0] += lead[i];
        t->lead_sum[1] += lead[nl + i];
    }
    // strictly increasing by far more than a rounding (both forms are: i / sqrt(n), and
    // sin(i pi / (2n + 1)) for i <= n): then the lines steeper than date j's are the later dates'
    for (int f = 0; f < 2; ++f) {
        bool inc = true;
        for (int i = 1; i < n && inc; ++i)
            inc = lead[f * nl + i] - lead[f * nl + i - 1] > 1e-12 * std::fabs(lead[f * nl + i]);
        t->lead_increasing[f] = inc ? 1 : 0;
    }
    std::vector<float> lead32(2 * lead.size());  // float pairs (hi, lo)
    for (size_t i = 0; i < lead.size(); ++i) split_ff(lead[i], &lead32[2 * i]);
    QMC_TRY(t->lead64.alloc(sizeof(double) * lead.size()));
    QMC_TRY(t->lead32.alloc(sizeof(float) * lead32.size()));
    QMC_CUDA(cudaMemcpy(t->lead64.ptr, lead.data(), sizeof(double) * lead.size(), cudaMemcpyHostToDevice));
    QMC_CUDA(cudaMemcpy(t->lead32.ptr, lead32.data(), sizeof(float) * lead32.size(), cudaMemcpyHostToDevice));
    if (n > 0) {
        QMC_CUDA(cudaMemcpy(t->steps.ptr, bp.steps.data(), sizeof(BridgeStep) * bp.steps.size(), cudaMemcpyHostToDevice));
        QMC_CUDA(cudaMemcpy(t->w64.ptr, bp.w.data(), sizeof(double) * bp.w.size(), cudaMemcpyHostToDevice));
        QMC_CUDA(cudaMemcpy(t->w32.ptr, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice));
        QMC_CUDA(cudaMemcpy(t->pca64.ptr, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice));
        QMC_CUDA(cudaMemcpy(t->pca32.ptr, A32.data(), sizeof(float) * A32.size(), cudaMemcpyHostToDevice));
        QMC_CUDA(cudaMemcpy(t->pca32lo.ptr, A32lo.data(), sizeof(float) * A32lo.size(), cudaMemcpyHostToDevice));
    }
    QMC_CUDA(cudaMemcpy(t->level_start.ptr, bp.level_start.data(), sizeof(int32_t) * bp.level_start.size(),
                        cudaMemcpyHostToDevice));
    *out = t.get();
    p->dtables.emplace(d, std::move(t));
    return QMCCPW_OK;
}

// Shared-memory budget of the z/W tile of one CTA: 65 KiB lets three CTAs
// share an SM (228 KiB) with room for the static reduction scratch.
constexpr size_t kTileBudget = 66560;

int choose_tile_log2(int precision, int n, int construction = QMCCPW_BB) {
    const size_t elem = precision == QMCCPW_FP64 ? 8 : 4;
    const int row = tile_row_elems(construction, n);
    int lg = kMaxTileLog2;
    while (lg > 0 && (static_cast<size_t>(1u << lg) * row * elem) > kTileBudget) --lg;
    return lg;
}

// Gray-code run length of the Sobol' phase.  n >= 32: a warp takes items of
// one run x 32 dimensions (CUDA cores) or x 64 (tensor cores).  CUDA cores:
// the longest run of at most 32 points whose item count splits evenly over
// the 8 warps (or is at least 32), since each run starts with a walk over
// the bits of its first index (64-point runs were slower at d = 64: the
// unrolled run no longer fits the instruction cache as well).
// Tensor cores: 8 runs per tile (16 for n > 64).  Small n: (run, dim) items, at least two
// per thread.
int chunk_log2_for(int n, int tile_log2, bool tc) {
    const int P = 1 << tile_log2;
    int lg = tile_log2;
    if (n >= 32 && !tc) {
        const long per = (n + 31) >> 5;
        lg = std::min(tile_log2, 5);
        while (lg > 2) {
            const long items = static_cast<long>(P >> lg) * per;
            if (items % (kThreads / 32) == 0 || items >= 4L * (kThreads / 32)) break;
            --lg;
        }
    } else if (n >= 32) {
        // at least one run per warp per 64-dimension block: 8 warps (resident
        // kernel, n <= 64) or the streamed kernel's 15 producer warps
        const int warps = n > 64 ? 16 : kThreads / 32;
        while (lg > 2 && (P >> lg) < warps) --lg;
    } else {
        while (lg > 0 && static_cast<long>(n) * (P >> lg) < 2L * kThreads) --lg;
    }
    return lg;
}

// log2 of the points per tile of a contract: 128 on tensor cores, else the
// plan's tuned tile for (precision, construction, d) or the default
int contract_tile_log2(const qmccpw_plan_s *p, int precision, int construction, int d) {
    if (is_tc(precision)) return 7;
    auto tt = p->tuned_tile.find(std::make_tuple(precision == QMCCPW_FP64 ? 0 : 1, construction, d));
    return tt != p->tuned_tile.end() ? tt->second : choose_tile_log2(precision, d - 1, construction);
}

int build_contract(qmccpw_plan_s *p, const qmccpw_contract &in, int batch_precision, uint64_t item_base,
                   uint64_t rep_base, ContractDev *out) {
    const int precision = contract_precision(batch_precision, in.construction);
    const DTables *t = nullptr;
    // the leading-coordinate constructions build the whole path of the d dates: the tables of d + 1
    const bool lead = is_lead(in.construction);
    QMC_TRY(get_dtables(p, in.option.d + (lead ? 1 : 0), in.option.T, &t));
    ContractDev c{};
    c.type = in.option.type;
    c.d = in.option.d;
    c.n = in.option.d - 1;
    c.construction = in.construction;
    c.tile_log2 = contract_tile_log2(p, precision, in.construction, c.d);
    const int P = 1 << c.tile_log2;
    c.chunk_log2 = chunk_log2_for(c.n, c.tile_log2, is_tc(precision));
    c.R = in.R;
    c.rep_first = in.first_replicate;
    c.k_first = in.first_point;
    c.tiles = static_cast<int32_t>((in.N + P - 1) / P);
    set_item_grouping(c);
    c.groups = kThreads / P;
    c.n_levels = t->n_levels;
    c.row_stride = lead ? (c.n + 2) | 1 : (c.n + 1) | 1;
    // the register bridge (float, one thread per point, d = 16 or 64) and PCA read z by
    // dimension; the shared-memory bridge overwrites z with W~ in place at its date
    c.z_by_dim = (c.construction != QMCCPW_BB && c.construction != QMCCPW_BB_LEAD) ||
                         (c.construction == QMCCPW_BB && precision != QMCCPW_FP64 && c.groups == 1 &&
                          (c.n == 63 || c.n == 15))
                     ? 1 : 0;
    c.slot_shift = lead ? 1 : 0;
    if (lead) {
        const size_t off = c.construction == QMCCPW_PCA_LEAD ? static_cast<size_t>(std::max(1, c.d)) : 0;
        c.lead_a64 = t->lead64.as<double>() + off;
        c.lead_a32 = t->lead32.as<float>() + 2 * off;
        c.lead_amean = t->lead_sum[c.construction == QMCCPW_PCA_LEAD ? 1 : 0] / c.d;  // times sqrt(dt) below
        c.lead_increasing = t->lead_increasing[c.construction == QMCCPW_PCA_LEAD ? 1 : 0];
    }
    c.N = in.N;
    c.item_base = item_base;
    c.rep_base = rep_base;
    c.steps = t->steps.as<BridgeStep>();
    c.w64 = t->w64.as<double>();
    c.w32 = t->w32.as<float>();
    c.level_start = t->level_start.as<int32_t>();
    c.slot_dim = (c.construction == QMCCPW_BB && !c.z_by_dim) ? t->slot_dim.as<int32_t>() : nullptr;
    c.sub_start = nullptr;
    if (c.construction == QMCCPW_BB && !c.z_by_dim && c.groups >= 2 && c.groups <= 8)
        c.sub_start = t->sub_start[c.groups == 2 ? 0 : c.groups == 4 ? 1 : 2].as<int32_t>();
    c.pca64 = t->pca64.as<double>();
    c.pcaT32 = t->pca32.as<float>();
    c.pcaT32lo = t->pca32lo.as<float>();
    if (is_tc(precision)) {
        DTables *mt = const_cast<DTables *>(t);
        DevBuf &op = mt->tc[tc_slot(precision)];
        if (!op.ptr) {
            std::vector<unsigned char> bytes;
            pca_tc_operand(tc_kind(precision, c.n), c.n, pca_factor(c.n, 1.0), bytes);
            QMC_TRY(op.alloc(bytes.size()));
            QMC_CUDA(cudaMemcpy(op.ptr, bytes.data(), bytes.size(), cudaMemcpyHostToDevice));
        }
        c.tc_operand = op.ptr;
    }
    c.S0 = in.market.S0;
    c.K = in.option.K;
    c.T = in.option.T;
    c.r = in.market.r;
    c.sigma = in.market.sigma;
    contract_constants(c);
    if (lead) c.lead_amean *= c.sqrt_t1;
    *out = c;
    return QMCCPW_OK;
}

int batch_build(qmccpw_plan_s *p, const qmccpw_contract *cs, int32_t count, int32_t precision, bool diagnostic,
                qmccpw_batch_s *b, cudaStream_t stream = nullptr) {
    cudaStream_t st = stream ? stream : p->stream;
    if (count < 1) return fail(QMCCPW_ERR_INVALID_ARG, "count must be >= 1");
    for (int i = 0; i < count; ++i)
        QMC_TRY(validate_qc(p, cs[i], precision, diagnostic));
    QMC_CUDA(cudaSetDevice(p->device));
    b->plan = p;
    b->count = count;
    b->precision = precision;
    b->host.resize(count);
    b->R.resize(count);
    // launch order: by segment (bridge, standard, streamed tensor-core PCA,
    // other PCA); within each, larger d first (their items are the costliest,
    // and the dynamic schedule hands items out in order, so the tail of the
    // launch holds the cheap ones)
    b->order.clear();
    auto seg_of = [&](int i) {
        return segment_of(contract_precision(precision, cs[i].construction), cs[i].construction, cs[i].option.d - 1);
    };
    for (int seg = 0; seg < kSegments; ++seg) {
        const size_t first = b->order.size();
        for (int i = 0; i < count; ++i)
            if (seg_of(i) == seg) b->order.push_back(i);
        std::stable_sort(b->order.begin() + first, b->order.end(),
                         [&](int x, int y) { return cs[x].option.d > cs[y].option.d; });
    }
    uint64_t items = 0, reps = 0;
    std::vector<uint64_t> item_base(count), rep_owner;
    for (int k = 0; k < count; ++k) {
        const qmccpw_contract &in = cs[b->order[k]];
        QMC_TRY(build_contract(p, in, precision, items, reps, &b->host[k]));
        const ContractDev &c = b->host[k];
        item_base[k] = items;
        items += static_cast<uint64_t>(c.R) * c.items;
        const int kp = contract_precision(precision, in.construction);
        const int seg = segment_of(kp, in.construction, c.n);
        for (int g = seg + 1; g <= kSegments; ++g) b->seg_begin[g] = items;
        for (int r = 0; r < c.R; ++r) rep_owner.push_back(static_cast<uint64_t>(k));
        reps += c.R;
        b->R[k] = c.R;
        size_t &sm = b->smem[seg];
        sm = std::max(sm, is_tc(kp) ? pca_tc_smem_bytes(tc_kind(kp, c.n))
                                    : fused_smem_bytes(kp, in.construction, c.n, c.tile_log2));
    }
    b->items = items;
    b->total_reps = reps;
    const size_t scratch = items * 4 * sizeof(double);
    if (scratch > p->workspace_bytes)
        return fail(QMCCPW_ERR_OOM, "tile partial sums need " + std::to_string(scratch) +
                                        " bytes, more than the plan's workspace budget");
    BatchBuffers &B = *b->buf;
    QMC_TRY(B.contracts.ensure(sizeof(ContractDev) * count));
    QMC_TRY(B.item_base.ensure(sizeof(uint64_t) * count));
    QMC_TRY(B.rep_owner.ensure(sizeof(uint64_t) * reps));
    QMC_TRY(B.tile_sums.ensure(scratch));
    QMC_TRY(B.per_rep.ensure(sizeof(double) * 4 * reps));
    QMC_TRY(B.stats.ensure(sizeof(double) * 8 * count));
    QMC_TRY(B.counters.ensure(kSegments * sizeof(unsigned long long)));
    QMC_CUDA(cudaMemcpyAsync(B.contracts.ptr, b->host.data(), sizeof(ContractDev) * count, cudaMemcpyHostToDevice, st));
    QMC_CUDA(cudaMemcpyAsync(B.item_base.ptr, item_base.data(), sizeof(uint64_t) * count, cudaMemcpyHostToDevice, st));
    QMC_CUDA(cudaMemcpyAsync(B.rep_owner.ptr, rep_owner.data(), sizeof(uint64_t) * reps, cudaMemcpyHostToDevice, st));
    QMC_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
    for (int k = 0; k < kSegments; ++k) {
        const uint64_t range = b->seg_begin[k + 1] - b->seg_begin[k];
        if (range == 0) continue;
        int per_sm = 0;
        const int cons = segment_construction(k);
        const int kp = contract_precision(precision, cons);
        if (is_tc(kp))
            QMC_CUDA(static_cast<cudaError_t>(pca_tc_occupancy(tc_kind(kp, k == 2 ? 256 : 0), b->smem[k], &per_sm)));
        else
            QMC_CUDA(static_cast<cudaError_t>(fused_occupancy(kp, cons, b->smem[k], &per_sm)));
        if (per_sm < 1) return fail(QMCCPW_ERR_CUDA, "fused kernel does not fit on an SM");
        const uint64_t slots = static_cast<uint64_t>(per_sm) * p->sm_count;
        b->grid[k] = static_cast<int>(std::min<uint64_t>(range, slots));
    }
    return QMCCPW_OK;
}

int batch_enqueue(qmccpw_batch_s *b, cudaStream_t s, bool record_events = true) {
    qmccpw_plan_s *p = b->plan;
    const BatchBuffers &B = *b->buf;
    LaunchParams lp{};
    lp.contracts = B.contracts.as<ContractDev>();
    lp.count = b->count;
    lp.item_base = B.item_base.as<uint64_t>();
    lp.sobol_table = p->table.as<uint32_t>();
    lp.sobol_shift = p->shift.as<uint32_t>();
    lp.jstride = p->jstride;
    lp.rep_offset = b->rep_offset;
    lp.tile_sums = B.tile_sums.as<double>();
    lp.point_out = b->point_out;
    lp.point_k0 = b->point_k0;
    lp.error_flag = p->err.as<int>();
    const size_t cap = record_events ? b->ev_start.size() : 0;
    const size_t slot = cap ? static_cast<size_t>(b->timed) % cap : 0;
    if (cap) QMC_CUDA(cudaEventRecord(b->ev_start[slot], s));
    for (int k = 0; k < kSegments; ++k) {
        if (b->seg_begin[k + 1] > b->seg_begin[k]) {
            lp.item_begin = b->seg_begin[k];
            lp.item_end = b->seg_begin[k + 1];
            lp.work_counter = B.counters.as<unsigned long long>() + k;
            QMC_CUDA(cudaMemsetAsync(lp.work_counter, 0, sizeof(unsigned long long), s));
            const int cons = segment_construction(k);
            const int kp = contract_precision(b->precision, cons);
            if (is_tc(kp))
                QMC_CUDA(static_cast<cudaError_t>(
                    launch_pca_tc(lp, tc_kind(kp, k == 2 ? 256 : 0), b->smem[k], b->grid[k], s)));
            else
                QMC_CUDA(static_cast<cudaError_t>(launch_fused(lp, kp, cons, b->smem[k], b->grid[k], s)));
        }
        if (cap) QMC_CUDA(cudaEventRecord(b->ev_seg[slot * kSegments + k], s));
    }
    if (cap) {
        QMC_CUDA(cudaEventRecord(b->ev_stop[slot], s));
        ++b->timed;
    }
    if (!b->point_out)
        QMC_CUDA(static_cast<cudaError_t>(launch_reduce(B.contracts.as<ContractDev>(), b->count,
                                                        B.tile_sums.as<double>(), B.per_rep.as<double>(),
                                                        B.stats.as<double>(), b->total_reps,
                                                        B.rep_owner.as<uint64_t>(), s)));
    if (!b->point_out && b->scatter_dst)
        QMC_CUDA(static_cast<cudaError_t>(launch_scatter_replicates(
            B.per_rep.as<double>(), b->scatter_rows.as<int64_t>(), b->total_reps, b->scatter_dst, s)));
    return QMCCPW_OK;
}

int batch_collect(qmccpw_batch_s *b, qmccpw_result *out, cudaStream_t s) {
    const BatchBuffers &B = *b->buf;
    std::vector<double> stats(8 * static_cast<size_t>(b->count));
    std::vector<double> per(4 * b->total_reps);
    QMC_CUDA(cudaMemcpyAsync(stats.data(), B.stats.ptr, sizeof(double) * stats.size(), cudaMemcpyDeviceToHost, s));
    QMC_CUDA(cudaMemcpyAsync(per.data(), B.per_rep.ptr, sizeof(double) * per.size(), cudaMemcpyDeviceToHost, s));
    int flag = 0;
    QMC_CUDA(cudaMemcpyAsync(&flag, b->plan->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    QMC_CUDA(cudaStreamSynchronize(s));
    if (flag != 0) {
        QMC_CUDA(cudaMemsetAsync(b->plan->err.ptr, 0, sizeof(int), s));
        QMC_CUDA(cudaStreamSynchronize(s));
        return fail(flag, "a kernel's bounded wait expired; results of this call are invalid");
    }
    uint64_t rep = 0;
    for (int k = 0; k < b->count; ++k) {
        qmccpw_result &o = out[b->order[k]];
        std::memcpy(o.mean, &stats[8 * k], 4 * sizeof(double));
        std::memcpy(o.se, &stats[8 * k + 4], 4 * sizeof(double));
        if (o.per_replicate) std::memcpy(o.per_replicate, per.data() + 4 * rep, sizeof(double) * 4 * b->R[k]);
        rep += b->R[k];
    }
    return QMCCPW_OK;
}



}  // namespace

// ---------------------------------------------------------------------------
// Serving (qmccpw_server_*): the host side of the device-resident loop of
// serve.cu.  Requests are admitted in arrival order while their device
// scratch fits the arena and the ring has a free entry, written into the
// ring and published; a monitor thread collects finished requests (their
// completion flags in host-mapped memory), admits waiting ones, and launches
// the serving kernel again after it has left on its idle limit while work is
// published.  submit/poll/wait do the same steps themselves, so a request
// does not wait for the monitor's next turn.
// ---------------------------------------------------------------------------
// The serving kernel of a precision (serve_f32.cu, serve_f64.cu).
int qmccpw::launch_serve(const ServeParams &p, int precision, bool with_pca, size_t smem_bytes, int grid,
                         void *stream) {
    return precision == QMCCPW_FP64 ? serve_f64_launch(p, smem_bytes, grid, stream)
                                    : serve_f32_launch(p, with_pca, smem_bytes, grid, stream);
}
int qmccpw::serve_prepare(int precision, bool with_pca, size_t optin_bytes) {
    return precision == QMCCPW_FP64 ? serve_f64_prepare(optin_bytes) : serve_f32_prepare(with_pca, optin_bytes);
}
int qmccpw::serve_occupancy(int precision, bool with_pca, size_t smem_bytes, int *blocks_per_sm) {
    return precision == QMCCPW_FP64 ? serve_f64_occupancy(smem_bytes, blocks_per_sm)
                                    : serve_f32_occupancy(with_pca, smem_bytes, blocks_per_sm);
}

struct ServerResult {
    int status = QMCCPW_OK;
    double mean[4] = {0, 0, 0, 0}, se[4] = {0, 0, 0, 0};
    std::vector<double> per_rep;
};

// First-fit allocator over [0, size) (offsets in bytes, 256-byte granules).
struct ArenaAllocator {
    std::map<uint64_t, uint64_t> free_;  // offset -> length
    void init(uint64_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = (bytes + 255) & ~uint64_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const uint64_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = (bytes + 255) & ~uint64_t(255);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

struct PendingRequest {
    uint64_t ticket;
    qmccpw_contract in;
    ContractDev c;
    uint64_t items, bytes;
};

struct LiveRequest {
    uint64_t ticket, seq, slot, arena_off, bytes;
    int R;
    uint64_t point_dates;
};

template <typename T> bool host_alloc_mapped(T **host, T **dev, size_t count) {
    void *h = nullptr;
    if (cudaHostAlloc(&h, sizeof(T) * count, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) return false;
    std::memset(h, 0, sizeof(T) * count);
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        cudaFreeHost(h);
        return false;
    }
    *host = static_cast<T *>(h);
    *dev = static_cast<T *>(d);
    return true;
}

struct QmcServer {
    qmccpw_plan_s *plan = nullptr;
    qmccpw_server_desc desc{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<PendingRequest> pending;
    std::deque<LiveRequest> live;  // in request (seq) order
    std::unordered_map<uint64_t, ServerResult> results;
    std::unordered_map<uint64_t, bool> known;  // ticket -> submitted and not yet collected
    uint64_t next_ticket_id = 1;
    uint64_t next_seq = 0, next_first_ticket = 0;
    bool stopping = false;
    bool broken = false;  // a launch failed or ended inconsistently
    qmccpw_server_stats stats{};
    // ring and control words, host-mapped (h_ host view, d_ device view)
    uint64_t cap = 0, out_stride = 0;
    ServeRequest *h_ring = nullptr, *d_ring = nullptr;
    ServeControl *h_ctl = nullptr, *d_ctl = nullptr;
    uint64_t *h_done = nullptr, *d_done = nullptr;
    ServeExit *h_exit = nullptr, *d_exit = nullptr;
    double *h_out = nullptr, *d_out = nullptr;  // cap x out_stride doubles
    // device state, the device copy of the ring, and the tile-slot arena
    DevBuf state, dev_ring, arena_buf;
    bool with_pca = true;  // the serving kernel carries the PCA product
    ArenaAllocator arena;
    cudaStream_t stream = nullptr;
    cudaEvent_t exit_ev = nullptr;
    bool running = false;
    uint32_t launch_no = 0;
    size_t smem = 0;
    int grid = 0;
    std::thread monitor;

    uint64_t oldest_live() const { return live.empty() ? next_seq : live.front().seq; }

    // the kernel has left (stream work done): record why
    void check_exit() {
        if (!running) return;
        const cudaError_t q = cudaEventQuery(exit_ev);
        if (q == cudaErrorNotReady) return;
        running = false;
        if (q != cudaSuccess) {
            fail_live(QMCCPW_ERR_CUDA);
            return;
        }
        const uint32_t reason = __atomic_load_n(&h_exit->reason, __ATOMIC_ACQUIRE);
        if (reason == 1u) ++stats.idle_exits;
        // 3: carried tickets above capacity, 4: a ticket without its request (neither expected)
        if (reason == 3u || reason == 4u) fail_live(QMCCPW_ERR_CUDA);
    }

    void finish(const LiveRequest &lr, int status) {
        ServerResult r;
        r.status = status;
        if (status == QMCCPW_OK) {
            const double *o = h_out + lr.slot * out_stride;
            r.per_rep.assign(o, o + 4 * static_cast<size_t>(lr.R));
            std::memcpy(r.mean, o + 4 * lr.R, sizeof(r.mean));
            std::memcpy(r.se, o + 4 * lr.R + 4, sizeof(r.se));
            ++stats.completed;
            stats.point_dates += lr.point_dates;
        } else {
            ++stats.failed;
        }
        arena.release(lr.arena_off, lr.bytes);
        results[lr.ticket] = std::move(r);
    }

    // the device side failed: every request fails, and the server takes no more
    void fail_live(int status) {
        broken = true;
        for (const LiveRequest &lr : live) finish(lr, status);
        live.clear();
        for (const PendingRequest &pr : pending) {
            ServerResult r;
            r.status = status;
            results[pr.ticket] = std::move(r);
            ++stats.failed;
        }
        pending.clear();
        cv_done.notify_all();
    }

    // finished requests: flag == seq + 1
    void harvest() {
        bool any = false;
        for (auto it = live.begin(); it != live.end();) {
            if (__atomic_load_n(h_done + it->slot, __ATOMIC_ACQUIRE) == it->seq + 1) {
                finish(*it, QMCCPW_OK);
                it = live.erase(it);
                any = true;
            } else {
                ++it;
            }
        }
        if (any) {
            __atomic_store_n(&h_ctl->oldest_live, oldest_live(), __ATOMIC_RELEASE);
            cv_done.notify_all();
        }
    }

    void publish(PendingRequest &pr, uint64_t arena_off) {
        const uint64_t seq = next_seq++;
        const uint64_t slot = seq & (cap - 1);
        ServeRequest *e = h_ring + slot;
        __atomic_store_n(&e->seq, ~0ull, __ATOMIC_RELAXED);
        std::atomic_thread_fence(std::memory_order_release);
        e->first_ticket = next_first_ticket;
        e->items = pr.items;
        e->tile_sums = reinterpret_cast<double *>(arena_buf.as<unsigned char>() + arena_off);
        e->out = d_out + slot * out_stride;
        e->c = pr.c;
        __atomic_store_n(&e->seq, seq, __ATOMIC_RELEASE);
        next_first_ticket += pr.items;
        __atomic_store_n(&h_ctl->published_seq, seq + 1, __ATOMIC_RELEASE);
        __atomic_store_n(&h_ctl->published_tickets, next_first_ticket, __ATOMIC_RELEASE);
        LiveRequest lr;
        lr.ticket = pr.ticket;
        lr.seq = seq;
        lr.slot = slot;
        lr.arena_off = arena_off;
        lr.bytes = pr.bytes;
        lr.R = pr.in.R;
        lr.point_dates = pr.in.N * static_cast<uint64_t>(pr.in.R) * static_cast<uint64_t>(pr.in.option.d);
        live.push_back(lr);
    }

    // admission in arrival order: a free ring entry (the one of request
    // seq - cap finished, with every request before it) and arena space
    void admit() {
        while (!pending.empty() && next_seq - oldest_live() < cap &&
               static_cast<int64_t>(live.size()) < desc.max_inflight) {
            uint64_t off = 0;
            if (!arena.alloc(pending.front().bytes, &off)) break;
            publish(pending.front(), off);
            pending.pop_front();
        }
    }

    int launch() {
        ServeParams sp{};
        sp.ring = d_ring;
        sp.dev_ring = dev_ring.as<ServeRequest>();
        sp.cap = cap;
        sp.ctl = d_ctl;
        sp.done = d_done;
        sp.exit_rec = d_exit;
        sp.st = state.as<ServeState>();
        sp.done_items = reinterpret_cast<unsigned long long *>(state.as<unsigned char>() + sizeof(ServeState));
        sp.sobol_table = plan->table.as<uint32_t>();
        sp.sobol_shift = plan->shift.as<uint32_t>();
        sp.jstride = plan->jstride;
        sp.launch = ++launch_no;
        sp.idle_ns = static_cast<uint64_t>(desc.idle_limit_us) * 1000u;
        QMC_CUDA(static_cast<cudaError_t>(launch_serve(sp, desc.precision, with_pca, smem, grid, stream)));
        QMC_CUDA(cudaEventRecord(exit_ev, stream));
        running = true;
        ++stats.launches;
        return QMCCPW_OK;
    }

    // one turn of the host side (under mu): exit, finished requests,
    // admission, and a launch when published work has no kernel
    void step() {
        check_exit();
        if (broken) return;
        harvest();
        admit();
        if (!running && !live.empty()) {
            const int rc = launch();
            if (rc != QMCCPW_OK) fail_live(rc);
        }
    }

    void run() {
        cudaSetDevice(plan->device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            step();
            if (stopping && pending.empty() && live.empty()) break;
            const bool busy = !live.empty() || !pending.empty();
            cv_work.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::microseconds(2000));
        }
        // every request is finished: ask the kernel to leave and wait for it
        __atomic_store_n(&h_ctl->stop, 1u, __ATOMIC_RELEASE);
        lk.unlock();
        cudaStreamSynchronize(stream);
        lk.lock();
        check_exit();
    }

    int init(qmccpw_plan_s *p, const qmccpw_server_desc &d);

    ~QmcServer() {
        if (stream) {
            cudaStreamSynchronize(stream);
            cudaStreamDestroy(stream);
        }
        if (exit_ev) cudaEventDestroy(exit_ev);
        for (void *h : {static_cast<void *>(h_ring), static_cast<void *>(h_ctl), static_cast<void *>(h_done),
                        static_cast<void *>(h_exit), static_cast<void *>(h_out)})
            if (h) cudaFreeHost(h);
    }
};

namespace {

int fill_result(const ServerResult &r, qmccpw_result *out) {
    if (r.status != QMCCPW_OK) return fail(r.status, "the request failed on the device");
    std::memcpy(out->mean, r.mean, sizeof(r.mean));
    std::memcpy(out->se, r.se, sizeof(r.se));
    if (out->per_replicate) std::memcpy(out->per_replicate, r.per_rep.data(), sizeof(double) * r.per_rep.size());
    return QMCCPW_OK;
}

// Device scratch of one request: its tile slots and its replicate estimates.
uint64_t serve_bytes(uint64_t items, int R) { return (items + static_cast<uint64_t>(R)) * 32u; }

// Largest dynamic shared memory of any contract the plan accepts in this
// precision among the constructions of `mask`.
size_t serve_smem(const qmccpw_plan_s *p, int precision, int32_t mask) {
    size_t m = 0;
    for (int cons : {QMCCPW_BB, QMCCPW_STD, QMCCPW_PCA, QMCCPW_BB_LEAD, QMCCPW_PCA_LEAD})
        for (int d = 1; d <= p->d_max && (mask >> cons) & 1; ++d) {
            if (is_lead(cons) && d + 1 > QMCCPW_D_LIMIT) continue;
            m = std::max(m, fused_smem_bytes(precision, cons, d - 1, contract_tile_log2(p, precision, cons, d)));
        }
    return m;
}

}  // namespace

int QmcServer::init(qmccpw_plan_s *p, const qmccpw_server_desc &d) {
    plan = p;
    desc = d;
    if (desc.max_inflight == 0) desc.max_inflight = 1024;
    if (desc.idle_limit_us == 0) desc.idle_limit_us = 20000;
    if (desc.max_inflight_bytes == 0) desc.max_inflight_bytes = uint64_t(256) << 20;
    if (desc.constructions == 0) desc.constructions = 0x1F;  // every construction
    // ring entries: a power of two >= max_inflight, fewer when the host-mapped
    // results (R_max x 4 + 8 doubles per entry) would pass 256 MiB
    out_stride = 4u * static_cast<uint64_t>(plan->r_max) + 8u;
    cap = 1;
    while (cap < static_cast<uint64_t>(desc.max_inflight)) cap <<= 1;
    while (cap > 1 && cap * out_stride * sizeof(double) > (uint64_t(256) << 20)) cap >>= 1;
    if (static_cast<uint64_t>(desc.max_inflight) > cap) desc.max_inflight = static_cast<int32_t>(cap);
    QMC_CUDA(cudaSetDevice(plan->device));
    if (!host_alloc_mapped(&h_ring, &d_ring, cap) || !host_alloc_mapped(&h_ctl, &d_ctl, 1) ||
        !host_alloc_mapped(&h_done, &d_done, cap) || !host_alloc_mapped(&h_exit, &d_exit, 1) ||
        !host_alloc_mapped(&h_out, &d_out, cap * out_stride))
        return fail(QMCCPW_ERR_OOM, "cudaHostAlloc of the serving ring failed");
    for (uint64_t i = 0; i < cap; ++i) h_ring[i].seq = ~0ull;
    QMC_TRY(state.alloc(sizeof(ServeState) + sizeof(unsigned long long) * cap));
    QMC_TRY(dev_ring.alloc(sizeof(ServeRequest) * cap));
    QMC_TRY(arena_buf.alloc(desc.max_inflight_bytes));
    arena.init(desc.max_inflight_bytes);
    QMC_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    QMC_CUDA(cudaEventCreateWithFlags(&exit_ev, cudaEventDisableTiming));
    QMC_CUDA(cudaMemsetAsync(state.ptr, 0, state.bytes, stream));
    QMC_CUDA(cudaMemsetAsync(dev_ring.ptr, 0xFF, dev_ring.bytes, stream));  // every sequence word ~0
    QMC_CUDA(cudaStreamSynchronize(stream));
    with_pca = desc.precision == QMCCPW_FP64 || ((desc.constructions >> QMCCPW_PCA) & 1);
    smem = serve_smem(plan, desc.precision, desc.constructions);
    cudaDeviceProp prop{};
    QMC_CUDA(cudaGetDeviceProperties(&prop, plan->device));
    QMC_CUDA(static_cast<cudaError_t>(serve_prepare(desc.precision, with_pca, prop.sharedMemPerBlockOptin)));
    int per_sm = 0;
    QMC_CUDA(static_cast<cudaError_t>(serve_occupancy(desc.precision, with_pca, smem, &per_sm)));
    if (per_sm < 1) return fail(QMCCPW_ERR_CUDA, "the serving kernel does not fit on an SM");
    grid = std::min(kServeMaxGrid, per_sm * plan->sm_count);  // the workers and the dispatcher
    return QMCCPW_OK;
}

namespace {

// ---------------------------------------------------------------------------
// Allocation-free form (qmccpw_greeks_noalloc): every per-call device array
// lives in this file-scope array instead of cudaMalloc'd memory.  In host code
// the symbol is only a host-side stand-in; its device address is looked up
// once per device with cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
int noalloc_scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return fail(QMCCPW_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *ptr = nullptr;
        QMC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_addr[device] = static_cast<unsigned char *>(ptr);
    }
    *out = g_noalloc_addr[device];
    return QMCCPW_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

const char *qmccpw_last_error(void) { return g_last_error.c_str(); }

const char *qmccpw_version(void) { return "qmccpw 0.1 sm_103a"; }

int qmccpw_measure_pipe_peaks(int32_t device, qmccpw_pipe_peaks *out) {
    g_last_error.clear();
    if (!out || device < 0) return fail(QMCCPW_ERR_INVALID_ARG, "qmccpw_measure_pipe_peaks: NULL output or bad device");
    qmccpw_pipe_peaks r{};
    const int rc = measure_pipe_peaks(device, &r);
    if (rc < 0) return fail(QMCCPW_ERR_TIMEOUT, "qmccpw_measure_pipe_peaks: the wait for the tensor-core products expired");
    if (rc > 0)
        return fail(QMCCPW_ERR_CUDA, std::string("qmccpw_measure_pipe_peaks: ") +
                                         cudaGetErrorString(static_cast<cudaError_t>(rc)));
    *out = r;
    return QMCCPW_OK;
}

int qmccpw_plan(qmccpw_plan_t *out, const qmccpw_plan_desc *desc) {
    g_last_error.clear();
    if (!out || !desc) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (desc->d_max < 1 || desc->d_max > QMCCPW_D_LIMIT) return fail(QMCCPW_ERR_INVALID_ARG, "d_max out of range");
    if (desc->r_max < 2 || desc->r_max > QMCCPW_R_LIMIT) return fail(QMCCPW_ERR_INVALID_ARG, "r_max out of range");
    if (desc->reserved != 0) return fail(QMCCPW_ERR_INVALID_ARG, "reserved must be 0");
    auto p = std::make_unique<qmccpw_plan_s>();
    p->device = desc->device;
    QMC_CUDA(cudaSetDevice(p->device));
    QMC_CUDA(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));
    int smem_optin = 0;
    QMC_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    // allow every tile size up front (occupancy follows the bytes each launch asks for)
    for (int prec : {QMCCPW_FP64, QMCCPW_MIXED})
        QMC_CUDA(static_cast<cudaError_t>(fused_set_smem_limit(prec, static_cast<size_t>(smem_optin))));
    QMC_CUDA(static_cast<cudaError_t>(basket_prepare(static_cast<size_t>(smem_optin))));
    p->seed = desc->seed;
    p->d_max = desc->d_max;
    p->r_max = desc->r_max;
    p->ndims = std::max(1, desc->d_max - 1);
    p->jstride = (p->ndims + 31) & ~31;
    p->workspace_bytes = desc->workspace_bytes ? desc->workspace_bytes : (1ull << 30);
    if (desc->stream) {
        p->stream = static_cast<cudaStream_t>(desc->stream);
    } else {
        QMC_CUDA(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    for (int kind : {0, 1, 2, 3})
        QMC_CUDA(static_cast<cudaError_t>(pca_tc_prepare(kind, pca_tc_smem_bytes(kind))));
    QMC_TRY(p->err.alloc(sizeof(int)));
    QMC_CUDA(cudaMemset(p->err.ptr, 0, sizeof(int)));
    std::vector<uint32_t> v = direction_integers(p->ndims);
    QMC_TRY(p->dir.alloc(sizeof(uint32_t) * v.size()));
    QMC_TRY(p->table.alloc(sizeof(uint32_t) * 32u * p->jstride * static_cast<size_t>(p->r_max)));
    QMC_TRY(p->shift.alloc(sizeof(uint32_t) * p->jstride * static_cast<size_t>(p->r_max)));
    QMC_CUDA(cudaMemcpy(p->dir.ptr, v.data(), sizeof(uint32_t) * v.size(), cudaMemcpyHostToDevice));
    QMC_CUDA(cudaMemsetAsync(p->table.ptr, 0, p->table.bytes, p->stream));
    QMC_CUDA(cudaMemsetAsync(p->shift.ptr, 0, p->shift.bytes, p->stream));
    QMC_CUDA(static_cast<cudaError_t>(launch_scramble(p->seed, p->dir.as<uint32_t>(), p->ndims, p->jstride,
                                                      p->r_max, p->table.as<uint32_t>(), p->shift.as<uint32_t>(),
                                                      p->stream)));
    QMC_CUDA(cudaStreamSynchronize(p->stream));
    *out = p.release();
    return QMCCPW_OK;
}

int qmccpw_free(qmccpw_plan_t plan) {
    g_last_error.clear();
    if (!plan) return QMCCPW_OK;
    qmccpw_server_stop(plan);
    cudaSetDevice(plan->device);
    cudaStreamSynchronize(plan->stream);
    plan->dtables.clear();
    plan->ws.release();
    plan->dir.release();
    plan->table.release();
    plan->shift.release();
    if (plan->own_stream) cudaStreamDestroy(plan->stream);
    delete plan;
    return QMCCPW_OK;
}

int qmccpw_batch_create(qmccpw_plan_t plan, const qmccpw_contract *contracts, int32_t count, int32_t precision,
                        qmccpw_batch_t *out) {
    g_last_error.clear();
    if (!plan || !contracts || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lock(plan->mu);
    auto b = std::make_unique<qmccpw_batch_s>();
    QMC_TRY(batch_build(plan, contracts, count, precision, false, b.get()));
    *out = b.release();
    return QMCCPW_OK;
}

int qmccpw_batch_launch(qmccpw_batch_t batch, void *stream) {
    g_last_error.clear();
    if (!batch) return fail(QMCCPW_ERR_INVALID_ARG, "NULL batch");
    QMC_CUDA(cudaSetDevice(batch->plan->device));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : batch->plan->stream;
    if (!batch->use_graph) return batch_enqueue(batch, s);
    if (!batch->graph_exec) {
        if (!batch->capture_stream) QMC_CUDA(cudaStreamCreateWithFlags(&batch->capture_stream, cudaStreamNonBlocking));
        QMC_CUDA(cudaStreamBeginCapture(batch->capture_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = batch_enqueue(batch, batch->capture_stream, false);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(batch->capture_stream, &g);
        if (rc != QMCCPW_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        QMC_CUDA(ec);
        const cudaError_t ei = cudaGraphInstantiate(&batch->graph_exec, g, 0);
        cudaGraphDestroy(g);
        QMC_CUDA(ei);
    }
    const size_t cap = batch->ev_start.size();
    const size_t slot = cap ? static_cast<size_t>(batch->timed) % cap : 0;
    if (cap) QMC_CUDA(cudaEventRecord(batch->ev_start[slot], s));
    QMC_CUDA(cudaGraphLaunch(batch->graph_exec, s));
    if (cap) {
        QMC_CUDA(cudaEventRecord(batch->ev_stop[slot], s));
        ++batch->timed;
    }
    return QMCCPW_OK;
}

int qmccpw_batch_use_graph(qmccpw_batch_t batch, int32_t enable) {
    g_last_error.clear();
    if (!batch) return fail(QMCCPW_ERR_INVALID_ARG, "NULL batch");
    QMC_CUDA(cudaSetDevice(batch->plan->device));
    if (!enable) {
        QMC_CUDA(cudaDeviceSynchronize());
        batch->drop_graph();
    }
    batch->use_graph = enable != 0;
    return QMCCPW_OK;
}

int qmccpw_batch_scatter_replicates(qmccpw_batch_t batch, double *dst, const int64_t *first_row) {
    g_last_error.clear();
    if (!batch) return fail(QMCCPW_ERR_INVALID_ARG, "NULL batch");
    if (!dst) {
        batch->scatter_dst = nullptr;
        return QMCCPW_OK;
    }
    if (!first_row) return fail(QMCCPW_ERR_INVALID_ARG, "NULL first_row");
    std::vector<int64_t> rows(batch->total_reps);
    uint64_t slot = 0;
    for (int k = 0; k < batch->count; ++k) {
        const int64_t f = first_row[batch->order[k]];
        if (f < 0) return fail(QMCCPW_ERR_INVALID_ARG, "negative first_row");
        for (int r = 0; r < batch->R[k]; ++r) rows[slot++] = f + r;
    }
    QMC_CUDA(cudaSetDevice(batch->plan->device));
    QMC_CUDA(cudaDeviceSynchronize());  // no launch in flight reads the rows being replaced
    QMC_TRY(batch->scatter_rows.ensure(sizeof(int64_t) * rows.size()));
    QMC_CUDA(cudaMemcpy(batch->scatter_rows.ptr, rows.data(), sizeof(int64_t) * rows.size(), cudaMemcpyHostToDevice));
    batch->scatter_dst = dst;
    batch->drop_graph();  // a captured sequence would lack (or keep) the copy
    return QMCCPW_OK;
}

int qmccpw_replicate_stats(const double *per_replicate, const int64_t *first_row, const int32_t *R, int32_t count,
                           double *stats, void *stream) {
    g_last_error.clear();
    if (!per_replicate || !first_row || !R || !stats || count < 1)
        return fail(QMCCPW_ERR_INVALID_ARG, "qmccpw_replicate_stats: NULL array or count < 1");
    QMC_CUDA(static_cast<cudaError_t>(launch_gathered_stats(per_replicate, first_row, R, count, stats, stream)));
    return QMCCPW_OK;
}

int qmccpw_batch_results(qmccpw_batch_t batch, qmccpw_result *out) {
    g_last_error.clear();
    if (!batch || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    QMC_CUDA(cudaSetDevice(batch->plan->device));
    QMC_CUDA(cudaDeviceSynchronize());
    return batch_collect(batch, out, batch->plan->stream);
}

int qmccpw_batch_device_results(qmccpw_batch_t batch, const double **per_replicate, const double **stats) {
    g_last_error.clear();
    if (!batch) return fail(QMCCPW_ERR_INVALID_ARG, "NULL batch");
    if (per_replicate) *per_replicate = batch->buf->per_rep.as<double>();
    if (stats) *stats = batch->buf->stats.as<double>();
    return QMCCPW_OK;
}

int qmccpw_batch_launch_count(qmccpw_batch_t batch, int32_t *launches) {
    g_last_error.clear();
    if (!batch || !launches) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    // one grid per launch segment present, the per-replicate reduction, the statistics
    int n = 2;
    for (int k = 0; k < kSegments; ++k) n += batch->seg_begin[k + 1] > batch->seg_begin[k] ? 1 : 0;
    *launches = n;
    return QMCCPW_OK;
}

int qmccpw_batch_set_timing(qmccpw_batch_t batch, int32_t capacity) {
    g_last_error.clear();
    if (!batch || capacity < 0 || capacity > 4096) return fail(QMCCPW_ERR_INVALID_ARG, "bad batch or capacity");
    QMC_CUDA(cudaSetDevice(batch->plan->device));
    QMC_CUDA(cudaStreamSynchronize(batch->plan->stream));
    for (auto e : batch->ev_start) cudaEventDestroy(e);
    for (auto e : batch->ev_stop) cudaEventDestroy(e);
    for (auto e : batch->ev_seg) cudaEventDestroy(e);
    batch->ev_start.clear();
    batch->ev_stop.clear();
    batch->ev_seg.clear();
    batch->timed = 0;
    for (int i = 0; i < capacity; ++i) {
        cudaEvent_t a, b;
        QMC_CUDA(cudaEventCreate(&a));
        QMC_CUDA(cudaEventCreate(&b));
        batch->ev_start.push_back(a);
        batch->ev_stop.push_back(b);
        for (int k = 0; k < kSegments; ++k) {
            QMC_CUDA(cudaEventCreate(&a));
            batch->ev_seg.push_back(a);
        }
    }
    return QMCCPW_OK;
}

int qmccpw_batch_timing(qmccpw_batch_t batch, float *fused_ms, int32_t *launches) {
    g_last_error.clear();
    if (!batch || !fused_ms || !launches) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    const int cap = static_cast<int>(batch->ev_start.size());
    const int n = std::min(batch->timed, cap);
    float total = 0.0f;
    for (int i = 0; i < n; ++i) {
        QMC_CUDA(cudaEventSynchronize(batch->ev_stop[i]));
        float ms = 0.0f;
        QMC_CUDA(cudaEventElapsedTime(&ms, batch->ev_start[i], batch->ev_stop[i]));
        total += ms;
    }
    *fused_ms = total;
    *launches = n;
    batch->timed = 0;
    return QMCCPW_OK;
}

int qmccpw_batch_segment_timing(qmccpw_batch_t batch, float *segment_ms, int32_t *launches) {
    g_last_error.clear();
    if (!batch || !segment_ms || !launches) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    const int cap = static_cast<int>(batch->ev_start.size());
    const int n = std::min(batch->timed, cap);
    for (int k = 0; k < kSegments; ++k) segment_ms[k] = 0.0f;
    if (batch->use_graph) {  // a replay records no segment boundaries
        *launches = 0;
        return QMCCPW_OK;
    }
    for (int i = 0; i < n; ++i) {
        QMC_CUDA(cudaEventSynchronize(batch->ev_stop[i]));
        cudaEvent_t prev = batch->ev_start[i];
        for (int k = 0; k < kSegments; ++k) {
            float ms = 0.0f;
            QMC_CUDA(cudaEventElapsedTime(&ms, prev, batch->ev_seg[i * kSegments + k]));
            segment_ms[k] += ms;
            prev = batch->ev_seg[i * kSegments + k];
        }
    }
    *launches = n;
    return QMCCPW_OK;
}

int qmccpw_selftest_bounded_wait(int32_t device, int32_t limit_us, int32_t *kernel_status) {
    g_last_error.clear();
    if (!kernel_status || limit_us < 1 || limit_us > 1000000)
        return fail(QMCCPW_ERR_INVALID_ARG, "NULL status or limit outside 1..1e6 us");
    QMC_CUDA(cudaSetDevice(device));
    cudaStream_t st = nullptr;
    QMC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DevBuf flag;
    int rc = flag.alloc(sizeof(int));
    int host = -1;
    if (rc == QMCCPW_OK) {
        cudaError_t e = cudaMemsetAsync(flag.ptr, 0xff, sizeof(int), st);
        if (e == cudaSuccess)
            e = static_cast<cudaError_t>(launch_bounded_wait_probe(static_cast<uint64_t>(limit_us) * 1000u,
                                                                   flag.as<int>(), st));
        if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(QMCCPW_ERR_CUDA, cudaGetErrorString(e));
    }
    flag.release();
    cudaStreamDestroy(st);
    *kernel_status = host;
    return rc;
}

int qmccpw_batch_free(qmccpw_batch_t batch) {
    g_last_error.clear();
    if (!batch) return QMCCPW_OK;
    cudaSetDevice(batch->plan->device);
    cudaStreamSynchronize(batch->plan->stream);
    delete batch;
    return QMCCPW_OK;
}

int qmccpw_greeks_batch(qmccpw_plan_t plan, const qmccpw_contract *contracts, int32_t count, int32_t precision,
                        qmccpw_result *out) {
    g_last_error.clear();
    if (!plan || !contracts || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(plan->mu);
    qmccpw_batch_s b;
    b.buf = &plan->ws;
    QMC_TRY(batch_build(plan, contracts, count, precision, false, &b));
    QMC_TRY(batch_enqueue(&b, plan->stream));
    return batch_collect(&b, out, plan->stream);
}

int qmccpw_greeks(qmccpw_plan_t plan, const qmccpw_option *option, const qmccpw_market *market, uint64_t N,
                  int32_t R, int32_t construction, int32_t precision, qmccpw_result *out) {
    g_last_error.clear();
    if (!plan || !option || !market || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    qmccpw_contract c{};
    c.option = *option;
    c.market = *market;
    c.N = N;
    c.R = R;
    c.construction = construction;
    return qmccpw_greeks_batch(plan, &c, 1, precision, out);
}

int qmccpw_sobol_points(qmccpw_plan_t plan, uint32_t replicate, int32_t ndims, uint64_t k0, uint64_t count,
                        uint32_t *out) {
    g_last_error.clear();
    if (!plan || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    if (ndims < 1 || ndims > plan->ndims) return fail(QMCCPW_ERR_INVALID_ARG, "ndims outside 1..d_max-1");
    if (replicate >= static_cast<uint32_t>(plan->r_max)) return fail(QMCCPW_ERR_INVALID_ARG, "replicate >= r_max");
    if (count < 1 || count > (1ull << 20) || k0 + count > (1ull << 32))
        return fail(QMCCPW_ERR_INVALID_ARG, "count must be 1..2^20 and k0+count <= 2^32");
    std::lock_guard<std::mutex> lock(plan->mu);
    QMC_CUDA(cudaSetDevice(plan->device));
    DevBuf dout;
    QMC_TRY(dout.alloc(sizeof(uint32_t) * count * ndims));
    QMC_CUDA(static_cast<cudaError_t>(launch_sobol_dump(
        plan->table.as<uint32_t>() + static_cast<size_t>(replicate) * 32u * plan->jstride,
        plan->shift.as<uint32_t>() + static_cast<size_t>(replicate) * plan->jstride, plan->jstride, ndims, k0, count,
        dout.as<uint32_t>(), plan->stream)));
    QMC_CUDA(cudaStreamSynchronize(plan->stream));
    QMC_CUDA(cudaMemcpy(out, dout.ptr, sizeof(uint32_t) * count * ndims, cudaMemcpyDeviceToHost));
    return QMCCPW_OK;
}

int qmccpw_point_values(qmccpw_plan_t plan, const qmccpw_option *option, const qmccpw_market *market,
                        int32_t construction, int32_t precision, uint32_t replicate, uint64_t k0, uint64_t count,
                        double *out) {
    g_last_error.clear();
    if (!plan || !option || !market || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    if (replicate >= static_cast<uint32_t>(plan->r_max)) return fail(QMCCPW_ERR_INVALID_ARG, "replicate >= r_max");
    if (count < 1 || count > (1ull << 20) || k0 + count > (1ull << 32))
        return fail(QMCCPW_ERR_INVALID_ARG, "count must be 1..2^20 and k0+count <= 2^32");
    std::lock_guard<std::mutex> lock(plan->mu);
    qmccpw_contract c{};
    c.option = *option;
    c.market = *market;
    c.N = count;
    c.R = 1;
    c.construction = construction;
    qmccpw_batch_s b;
    b.buf = &plan->ws;
    QMC_TRY(batch_build(plan, &c, 1, precision, true, &b));
    DevBuf dout;
    QMC_TRY(dout.alloc(sizeof(double) * 4 * count));
    b.point_out = dout.as<double>();
    b.point_k0 = k0;
    b.rep_offset = replicate;
    QMC_TRY(batch_enqueue(&b, plan->stream));
    QMC_CUDA(cudaStreamSynchronize(plan->stream));
    QMC_CUDA(cudaMemcpy(out, dout.ptr, sizeof(double) * 4 * count, cudaMemcpyDeviceToHost));
    return QMCCPW_OK;
}


}  // extern "C"

namespace {

// Validate a basket and fill its kernel descriptor (everything but the
// device table of row slots, returned in slot_of_dim).
int basket_build(qmccpw_plan_s *p, const qmccpw_basket &bk, int precision, uint64_t N, BasketDev &b,
                 std::vector<int32_t> &slot_of_dim) {
    if (bk.reserved != 0) return fail(QMCCPW_ERR_INVALID_ARG, "qmccpw_basket.reserved must be 0");
    if (bk.type != QMCCPW_ARITH_ASIAN_CALL && bk.type != QMCCPW_BINARY_ASIAN)
        return fail(bk.type >= 0 && bk.type <= 3 ? QMCCPW_ERR_UNSUPPORTED : QMCCPW_ERR_INVALID_ARG,
                    "basket type: the arithmetic-Asian call or the binary on the basket average");
    if (precision != QMCCPW_FP64 && precision != QMCCPW_MIXED)
        return fail(precision >= 0 && precision <= QMCCPW_MIXED_TC_TF32X3 ? QMCCPW_ERR_UNSUPPORTED
                                                                          : QMCCPW_ERR_INVALID_ARG,
                    "basket precision: QMCCPW_FP64 or QMCCPW_MIXED");
    const int m = bk.m, d = bk.d;
    if (m < 1 || m > QMCCPW_ASSETS_MAX) return fail(QMCCPW_ERR_INVALID_ARG, "basket m outside 1..8");
    if (d < 1 || static_cast<int64_t>(m) * d > p->d_max)
        return fail(QMCCPW_ERR_INVALID_ARG, "basket needs 1 <= d and m * d <= d_max=" + std::to_string(p->d_max));
    if (!finite_pos(bk.K) || !finite_pos(bk.T) || !finite_pos(bk.S0) || !finite_pos(bk.sigma) || !std::isfinite(bk.r))
        return fail(QMCCPW_ERR_INVALID_ARG, "basket K, T, S0, sigma must be positive and finite, r finite");
    if (N < 1 || N > (1ull << 32)) return fail(QMCCPW_ERR_INVALID_ARG, "N must be in 1..2^32");
    if (!(bk.weight[0] > 0.0)) return fail(QMCCPW_ERR_INVALID_ARG, "basket weight[0] must be positive");
    for (int i = 0; i < m; ++i) {
        if (!std::isfinite(bk.weight[i]) || bk.weight[i] < 0.0 || !finite_pos(bk.spot[i]) || !finite_pos(bk.vol[i]))
            return fail(QMCCPW_ERR_INVALID_ARG, "basket weights >= 0, spots and vols > 0, all finite");
        if (bk.corr[i * m + i] != 1.0) return fail(QMCCPW_ERR_INVALID_ARG, "basket correlation diagonal must be 1");
        if (!(bk.corr[i] > 0.0))
            return fail(QMCCPW_ERR_INVALID_ARG, "every asset must be positively correlated with asset 1 (corr[i] > 0)");
        for (int k = 0; k < m; ++k)
            if (!(std::fabs(bk.corr[i * m + k]) <= 1.0) || bk.corr[i * m + k] != bk.corr[k * m + i])
                return fail(QMCCPW_ERR_INVALID_ARG, "basket correlation must be symmetric with entries in [-1, 1]");
    }
    double L[QMCCPW_ASSETS_MAX * QMCCPW_ASSETS_MAX];
    if (!cholesky_lower(m, bk.corr, L)) return fail(QMCCPW_ERR_INVALID_ARG, "basket correlation is not positive definite");
    const DTables *t = nullptr;
    QMC_TRY(get_dtables(p, d, bk.T, &t));
    const int n = d - 1;
    b = BasketDev{};
    b.type = bk.type;
    b.d = d;
    b.n = n;
    b.m = m;
    b.n_levels = t->n_levels;
    b.steps = t->steps.as<BridgeStep>();
    b.w64 = t->w64.as<double>();
    b.w32 = t->w32.as<float>();
    b.level_start = t->level_start.as<int32_t>();
    const double dt = bk.T / d, sdt = std::sqrt(dt);
    b.S0 = bk.S0;
    b.K = bk.K;
    b.disc = std::exp(-bk.r * bk.T);
    b.sqrt_dt = sdt;
    b.ln_K = std::log(bk.K);
    for (int i = 0; i < m; ++i) {
        const double sig = bk.vol[i] * bk.sigma, om = bk.r - 0.5 * sig * sig;
        for (int k = 0; k < m; ++k) {
            b.L[i * QMCCPW_ASSETS_MAX + k] = L[i * m + k];
            split_ff(L[i * m + k], b.Lf[i * QMCCPW_ASSETS_MAX + k]);
        }
        b.sig_sdt[i] = sig * sdt;
        b.om_dt[i] = om * dt;
        b.sig_dt[i] = sig * dt;
        b.f[i] = bk.weight[i] * bk.spot[i] * bk.S0 / d;
        b.l1[i] = L[i * m] * sdt;
        b.bcoef[i] = sig * b.l1[i];
        b.v[i] = bk.vol[i];
        b.ehalf[i] = std::exp(0.5 * b.bcoef[i] * b.bcoef[i]);
        split_ff(b.sig_sdt[i], b.ff_sig_sdt[i]);
        split_ff(b.om_dt[i], b.ff_om_dt[i]);
    }
    // the row: slot 0 = 0, factor k at date index s (1..n) in slot 1 + (s-1) m + k,
    // the first increment of factor k >= 1 in slot 1 + n m + k - 1
    const int nd = m * d - 1;
    slot_of_dim.assign(std::max(1, nd), 0);
    if (n > 0) {
        const BridgePlan bp = bridge_plan(n, 1.0);
        for (int j = 0; j < n * m; ++j) slot_of_dim[j] = 1 + (bp.steps[j / m].m - 1) * m + j % m;
    }
    for (int j = n * m; j < nd; ++j) slot_of_dim[j] = 1 + j;
    // tile: P points with P * row <= 65 KiB (two CTAs per SM and room for the rest), P in 16..256
    const size_t elem = precision == QMCCPW_FP64 ? 8 : 4;
    b.row_stride = (m * d) | 1;
    int lg = kMaxTileLog2;
    while (lg > 4 && (static_cast<size_t>(1u << lg) * b.row_stride * elem) > kTileBudget) --lg;
    b.tile_log2 = lg;
    b.groups = kThreads >> lg;
    b.chunk_log2 = chunk_log2_for(std::max(1, nd), lg, false);
    b.N = N;
    b.tiles = (N + (1u << lg) - 1) >> lg;
    return QMCCPW_OK;
}

size_t basket_smem_bytes(const BasketDev &b, int precision) {
    const size_t elem = precision == QMCCPW_FP64 ? 8 : 4;
    const size_t tile = (static_cast<size_t>(1) << b.tile_log2) * b.row_stride * elem;
    const size_t part = static_cast<size_t>(kThreads) * 3 * b.m * elem;  // the per-thread partial sums
    return std::max({tile, part, static_cast<size_t>(4 * kThreads * sizeof(double))});
}

// Run the basket over replicates rep_offset .. rep_offset + R - 1: per-replicate
// estimates and statistics into per_rep / stats (device), or with point_out
// (R = 1) every point's values.
int basket_run(qmccpw_plan_s *p, const qmccpw_basket &bk, int precision, uint64_t N, int R, uint32_t rep_offset,
               uint64_t point_k0, double *point_out, DevBuf &per_rep, DevBuf &stats) {
    BasketParams bp{};
    std::vector<int32_t> slots;
    QMC_TRY(basket_build(p, bk, precision, N, bp.b, slots));
    const uint64_t items = static_cast<uint64_t>(R) * bp.b.tiles;
    if (items * 4 * sizeof(double) > p->workspace_bytes)
        return fail(QMCCPW_ERR_OOM, "basket tile sums exceed the plan's workspace budget");
    QMC_CUDA(cudaSetDevice(p->device));
    DevBuf dslots, tile_sums, cdesc, owner;
    QMC_TRY(dslots.alloc(sizeof(int32_t) * slots.size()));
    QMC_CUDA(cudaMemcpyAsync(dslots.ptr, slots.data(), sizeof(int32_t) * slots.size(), cudaMemcpyHostToDevice,
                             p->stream));
    QMC_TRY(tile_sums.alloc(items * 4 * sizeof(double)));
    bp.b.slot_of_dim = dslots.as<int32_t>();
    bp.sobol_table = p->table.as<uint32_t>();
    bp.sobol_shift = p->shift.as<uint32_t>();
    bp.jstride = p->jstride;
    bp.rep_offset = rep_offset;
    bp.items = items;
    bp.tile_sums = tile_sums.as<double>();
    bp.point_out = point_out;
    bp.point_k0 = point_k0;
    const size_t smem = basket_smem_bytes(bp.b, precision);
    int per_sm = 0;
    QMC_CUDA(static_cast<cudaError_t>(basket_occupancy(precision, smem, &per_sm)));
    const uint64_t cap = static_cast<uint64_t>(std::max(1, per_sm)) * p->sm_count;
    const int grid = static_cast<int>(std::min<uint64_t>(items, cap));
    QMC_CUDA(static_cast<cudaError_t>(launch_basket(bp, precision, smem, grid, p->stream)));
    if (!point_out) {
        // reduction in tile order and the statistics, by the batch's kernels
        ContractDev c{};
        c.R = R;
        c.tiles = static_cast<int32_t>(bp.b.tiles);
        c.tpi = 1;  // the basket kernel writes one slot per tile
        c.items = c.tiles;
        c.N = N;
        c.item_base = 0;
        c.rep_base = 0;
        std::vector<uint64_t> rep_owner(static_cast<size_t>(R), 0);
        QMC_TRY(cdesc.alloc(sizeof(ContractDev)));
        QMC_TRY(owner.alloc(sizeof(uint64_t) * rep_owner.size()));
        QMC_TRY(per_rep.alloc(sizeof(double) * 4 * R));
        QMC_TRY(stats.alloc(sizeof(double) * 8));
        QMC_CUDA(cudaMemcpyAsync(cdesc.ptr, &c, sizeof(ContractDev), cudaMemcpyHostToDevice, p->stream));
        QMC_CUDA(cudaMemcpyAsync(owner.ptr, rep_owner.data(), sizeof(uint64_t) * rep_owner.size(),
                                 cudaMemcpyHostToDevice, p->stream));
        QMC_CUDA(static_cast<cudaError_t>(launch_reduce(cdesc.as<ContractDev>(), 1, tile_sums.as<double>(),
                                                        per_rep.as<double>(), stats.as<double>(),
                                                        static_cast<uint64_t>(R), owner.as<uint64_t>(), p->stream)));
    }
    // the host buffers above and the DevBufs live until the work is done
    QMC_CUDA(cudaStreamSynchronize(p->stream));
    return QMCCPW_OK;
}

}  // namespace

extern "C" {

int qmccpw_basket_greeks(qmccpw_plan_t plan, const qmccpw_basket *basket, uint64_t N, int32_t R,
                         int32_t precision, qmccpw_result *out) {
    g_last_error.clear();
    if (!plan || !basket || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    if (R < 2 || R > plan->r_max)
        return fail(QMCCPW_ERR_INVALID_ARG, "R " + std::to_string(R) + " outside 2..r_max=" + std::to_string(plan->r_max));
    std::lock_guard<std::mutex> lock(plan->mu);
    DevBuf per_rep, stats;
    QMC_TRY(basket_run(plan, *basket, precision, N, R, 0u, 0u, nullptr, per_rep, stats));
    double st[8];
    QMC_CUDA(cudaMemcpy(st, stats.ptr, sizeof(st), cudaMemcpyDeviceToHost));
    for (int g = 0; g < 4; ++g) {
        out->mean[g] = st[g];
        out->se[g] = st[4 + g];
    }
    if (out->per_replicate)
        QMC_CUDA(cudaMemcpy(out->per_replicate, per_rep.ptr, sizeof(double) * 4 * R, cudaMemcpyDeviceToHost));
    return QMCCPW_OK;
}

int qmccpw_basket_point_values(qmccpw_plan_t plan, const qmccpw_basket *basket, int32_t precision,
                               uint32_t replicate, uint64_t k0, uint64_t count, double *out) {
    g_last_error.clear();
    if (!plan || !basket || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    if (replicate >= static_cast<uint32_t>(plan->r_max)) return fail(QMCCPW_ERR_INVALID_ARG, "replicate >= r_max");
    if (count < 1 || count > (1ull << 20) || k0 + count > (1ull << 32))
        return fail(QMCCPW_ERR_INVALID_ARG, "count must be 1..2^20 and k0+count <= 2^32");
    std::lock_guard<std::mutex> lock(plan->mu);
    QMC_CUDA(cudaSetDevice(plan->device));
    DevBuf dout, per_rep, stats;
    QMC_TRY(dout.alloc(sizeof(double) * 4 * count));
    QMC_TRY(basket_run(plan, *basket, precision, count, 1, replicate, k0, dout.as<double>(), per_rep, stats));
    QMC_CUDA(cudaMemcpy(out, dout.ptr, sizeof(double) * 4 * count, cudaMemcpyDeviceToHost));
    return QMCCPW_OK;
}

int qmccpw_greeks_noalloc(qmccpw_plan_t plan, const qmccpw_option *option, const qmccpw_market *market, uint64_t N,
                          int32_t R, int32_t construction, int32_t precision, double *out, void *stream) {
    g_last_error.clear();
    if (!plan || !option || !market || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    QMC_TRY(validate_contract(plan, *option, *market, N, R, construction, precision, false));
    if (precision >= QMCCPW_MIXED_TC_BF16X3)
        return fail(QMCCPW_ERR_UNSUPPORTED, "the allocation-free entry point offers FP64 and MIXED only");
    if (is_lead(construction))
        return fail(QMCCPW_ERR_UNSUPPORTED, "the allocation-free entry point offers the bridge, PCA and standard constructions");
    std::lock_guard<std::mutex> lock(plan->mu);
    QMC_CUDA(cudaSetDevice(plan->device));
    unsigned char *scratch = nullptr;
    QMC_TRY(noalloc_scratch_address(plan->device, &scratch));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : plan->stream;

    // the contract and its bridge / PCA tables, built on the host
    const int d = option->d, n = d - 1;
    BridgePlan bp = bridge_plan(n, 1.0);  // unit spacing: the kernels scale by sqrt(dt)
    const int n_pad = (n + 15) & ~15;
    const bool pca = construction == QMCCPW_PCA;
    std::vector<double> A = (pca && n > 0) ? pca_factor(n, 1.0) : std::vector<double>();

    ContractDev c{};
    c.type = option->type;
    c.d = d;
    c.n = n;
    c.construction = construction;
    c.tile_log2 = choose_tile_log2(precision, n, construction);
    const int P = 1 << c.tile_log2;
    c.chunk_log2 = chunk_log2_for(n, c.tile_log2, false);
    c.R = R;
    c.tiles = static_cast<int32_t>((N + P - 1) / P);
    set_item_grouping(c);
    c.groups = kThreads / P;
    c.n_levels = static_cast<int>(bp.level_start.size()) - 1;
    c.row_stride = (n + 1) | 1;
    c.z_by_dim = (construction != QMCCPW_BB ||
                  (precision != QMCCPW_FP64 && c.groups == 1 && (n == 63 || n == 15))) ? 1 : 0;
    c.N = N;
    c.item_base = 0;
    c.rep_base = 0;
    const uint64_t items = static_cast<uint64_t>(R) * c.items;

    // layout of the scratch array (256-byte aligned pieces)
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align256(off + bytes); return at; };
    const size_t o_contract = take(sizeof(ContractDev));
    const size_t o_item_base = take(sizeof(uint64_t));
    const size_t o_rep_owner = take(sizeof(uint64_t) * R);
    const size_t o_steps = take(sizeof(BridgeStep) * bp.steps.size());
    const size_t o_w64 = take(sizeof(double) * bp.w.size());
    const size_t o_w32 = take(sizeof(float) * 8 * bp.steps.size());
    const size_t o_levels = take(sizeof(int32_t) * bp.level_start.size());
    const size_t o_pca64 = take(pca && precision == QMCCPW_FP64 ? sizeof(double) * A.size() : 0);
    const size_t o_pca32 = take(pca && precision != QMCCPW_FP64 ? sizeof(float) * n * n_pad : 0);
    const size_t staged = off;
    const size_t o_counter = take(sizeof(unsigned long long));
    const size_t o_tiles = take(sizeof(double) * 4 * items);
    if (off > kNoAllocScratchBytes)
        return fail(QMCCPW_ERR_OOM, "qmccpw_greeks_noalloc needs " + std::to_string(off) +
                                        " bytes of scratch; its fixed array holds " +
                                        std::to_string(kNoAllocScratchBytes) + " bytes (reduce N or R)");

    // stage the read-only part on the host, then one copy into the array
    std::vector<unsigned char> host(staged, 0);
    unsigned char *dev = scratch;
    c.steps = reinterpret_cast<const BridgeStep *>(dev + o_steps);
    c.w64 = reinterpret_cast<const double *>(dev + o_w64);
    c.w32 = reinterpret_cast<const float *>(dev + o_w32);
    c.level_start = reinterpret_cast<const int32_t *>(dev + o_levels);
    c.pca64 = reinterpret_cast<const double *>(dev + o_pca64);
    c.pcaT32 = reinterpret_cast<const float *>(dev + o_pca32);
    c.S0 = market->S0;
    c.K = option->K;
    c.T = option->T;
    c.r = market->r;
    c.sigma = market->sigma;
    contract_constants(c);
    std::memcpy(host.data() + o_contract, &c, sizeof(c));
    std::memset(host.data() + o_item_base, 0, sizeof(uint64_t));
    std::memset(host.data() + o_rep_owner, 0, sizeof(uint64_t) * R);  // every replicate belongs to contract 0
    if (!bp.steps.empty()) {
        std::memcpy(host.data() + o_steps, bp.steps.data(), sizeof(BridgeStep) * bp.steps.size());
        std::memcpy(host.data() + o_w64, bp.w.data(), sizeof(double) * bp.w.size());
        float *w32 = reinterpret_cast<float *>(host.data() + o_w32);
        for (size_t b = 0; b < bp.steps.size(); ++b)
            for (int k = 0; k < 3; ++k) {
                const double x = bp.w[3 * b + k];
                w32[8 * b + 2 * k] = static_cast<float>(x);
                w32[8 * b + 2 * k + 1] = static_cast<float>(x - static_cast<double>(w32[8 * b + 2 * k]));
            }
    }
    std::memcpy(host.data() + o_levels, bp.level_start.data(), sizeof(int32_t) * bp.level_start.size());
    if (pca && precision == QMCCPW_FP64 && !A.empty())
        std::memcpy(host.data() + o_pca64, A.data(), sizeof(double) * A.size());
    if (pca && precision != QMCCPW_FP64) {
        float *at = reinterpret_cast<float *>(host.data() + o_pca32);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) at[static_cast<size_t>(k) * n_pad + i] = static_cast<float>(A[static_cast<size_t>(i) * n + k]);
    }
    QMC_CUDA(cudaMemcpyAsync(dev, host.data(), staged, cudaMemcpyHostToDevice, s));

    int per_sm = 0;
    const size_t smem = fused_smem_bytes(precision, construction, n, c.tile_log2);
    QMC_CUDA(static_cast<cudaError_t>(fused_occupancy(precision, construction, smem, &per_sm)));
    if (per_sm < 1) return fail(QMCCPW_ERR_CUDA, "fused kernel does not fit on an SM");
    const int grid = static_cast<int>(std::min<uint64_t>(items, static_cast<uint64_t>(per_sm) * plan->sm_count));

    LaunchParams lp{};
    lp.contracts = reinterpret_cast<const ContractDev *>(dev + o_contract);
    lp.count = 1;
    lp.item_begin = 0;
    lp.item_end = items;
    lp.item_base = reinterpret_cast<const uint64_t *>(dev + o_item_base);
    lp.sobol_table = plan->table.as<uint32_t>();
    lp.sobol_shift = plan->shift.as<uint32_t>();
    lp.jstride = plan->jstride;
    lp.tile_sums = reinterpret_cast<double *>(dev + o_tiles);
    lp.work_counter = reinterpret_cast<unsigned long long *>(dev + o_counter);
    QMC_CUDA(cudaMemsetAsync(lp.work_counter, 0, sizeof(unsigned long long), s));
    QMC_CUDA(static_cast<cudaError_t>(launch_fused(lp, precision, construction, smem, grid, s)));
    QMC_CUDA(static_cast<cudaError_t>(launch_reduce(lp.contracts, 1, lp.tile_sums, out, out + 4 * static_cast<size_t>(R),
                                                    static_cast<uint64_t>(R),
                                                    reinterpret_cast<const uint64_t *>(dev + o_rep_owner), s)));
    return QMCCPW_OK;
}


int qmccpw_server_start(qmccpw_plan_t plan, const qmccpw_server_desc *desc) {
    g_last_error.clear();
    if (!plan || !desc) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    if (plan->server) return fail(QMCCPW_ERR_INVALID_ARG, "the plan already runs a server");
    if (desc->constructions < 0 || desc->constructions > 0x1F)
        return fail(QMCCPW_ERR_INVALID_ARG, "constructions: a mask of bits 0..4");
    if (desc->precision < QMCCPW_FP64 || desc->precision > QMCCPW_MIXED_TC_TF32X3)
        return fail(QMCCPW_ERR_INVALID_ARG, "precision out of range");
    if (is_tc(desc->precision))
        return fail(QMCCPW_ERR_UNSUPPORTED, "the serving loop runs the CUDA-core kernels: precision FP64 or MIXED");
    if (desc->max_inflight < 0 || desc->max_inflight > 4096)
        return fail(QMCCPW_ERR_INVALID_ARG, "max_inflight out of 0..4096");
    if (desc->idle_limit_us < 0 || desc->idle_limit_us > 10000000)
        return fail(QMCCPW_ERR_INVALID_ARG, "idle_limit_us out of 0..10^7");
    auto sv = std::make_unique<QmcServer>();
    QMC_TRY(sv->init(plan, *desc));
    QmcServer *raw = sv.get();
    sv->monitor = std::thread([raw] { raw->run(); });
    plan->server = sv.release();
    return QMCCPW_OK;
}

int qmccpw_submit(qmccpw_plan_t plan, const qmccpw_contract *contract, uint64_t *ticket) {
    g_last_error.clear();
    if (!plan || !contract || !ticket) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    QmcServer *sv = plan->server;
    if (!sv) return fail(QMCCPW_ERR_INVALID_ARG, "no server runs on this plan");
    QMC_TRY(validate_qc(plan, *contract, sv->desc.precision, false));
    if (!((sv->desc.constructions >> contract->construction) & 1))
        return fail(QMCCPW_ERR_UNSUPPORTED, "the server was started without this construction");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return fail(QMCCPW_ERR_INVALID_ARG, "the server is stopping");
    if (sv->broken) return fail(QMCCPW_ERR_CUDA, "the serving kernel failed; stop the server");
    PendingRequest pr;
    pr.in = *contract;
    QMC_TRY(build_contract(plan, *contract, sv->desc.precision, 0, 0, &pr.c));
    if (fused_smem_bytes(sv->desc.precision, contract->construction, pr.c.n, pr.c.tile_log2) > sv->smem)
        return fail(QMCCPW_ERR_UNSUPPORTED, "the request's tile needs more shared memory than the serving kernel has");
    pr.items = static_cast<uint64_t>(pr.c.R) * static_cast<uint64_t>(pr.c.items);
    pr.bytes = serve_bytes(pr.items, pr.c.R);
    if (((pr.bytes + 255) & ~uint64_t(255)) > sv->desc.max_inflight_bytes)
        return fail(QMCCPW_ERR_OOM, "the request needs more device scratch than max_inflight_bytes");
    pr.ticket = sv->next_ticket_id++;
    *ticket = pr.ticket;
    sv->known[pr.ticket] = true;
    sv->pending.push_back(pr);
    ++sv->stats.submitted;
    sv->step();  // publish now if it fits, launching the kernel if none runs
    sv->cv_work.notify_all();
    return QMCCPW_OK;
}

int qmccpw_poll(qmccpw_plan_t plan, uint64_t ticket, qmccpw_result *out) {
    g_last_error.clear();
    if (!plan || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    QmcServer *sv = plan->server;
    if (!sv) return fail(QMCCPW_ERR_INVALID_ARG, "no server runs on this plan");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->known.count(ticket)) return fail(QMCCPW_ERR_INVALID_ARG, "unknown or already collected ticket");
    sv->step();
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return QMCCPW_NOT_READY;
    const int rc = fill_result(it->second, out);
    sv->results.erase(it);
    sv->known.erase(ticket);
    return rc;
}

int qmccpw_wait(qmccpw_plan_t plan, uint64_t ticket, int32_t timeout_ms, qmccpw_result *out) {
    g_last_error.clear();
    if (!plan || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    QmcServer *sv = plan->server;
    if (!sv) return fail(QMCCPW_ERR_INVALID_ARG, "no server runs on this plan");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (!sv->known.count(ticket)) return fail(QMCCPW_ERR_INVALID_ARG, "unknown or already collected ticket");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (true) {
        sv->step();
        if (sv->results.count(ticket)) break;
        if (std::chrono::steady_clock::now() >= deadline) return fail(QMCCPW_ERR_TIMEOUT, "the request is not finished");
        sv->cv_done.wait_for(lk, std::chrono::microseconds(20));
    }
    auto it = sv->results.find(ticket);
    const int rc = fill_result(it->second, out);
    sv->results.erase(it);
    sv->known.erase(ticket);
    return rc;
}

int qmccpw_server_get_stats(qmccpw_plan_t plan, qmccpw_server_stats *out) {
    g_last_error.clear();
    if (!plan || !out) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    QmcServer *sv = plan->server;
    if (!sv) return fail(QMCCPW_ERR_INVALID_ARG, "no server runs on this plan");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->check_exit();
    *out = sv->stats;
    out->pending = sv->pending.size();
    out->inflight = sv->live.size();
    out->running = sv->running ? 1u : 0u;
    return QMCCPW_OK;
}

int qmccpw_server_stop(qmccpw_plan_t plan) {
    g_last_error.clear();
    if (!plan) return fail(QMCCPW_ERR_INVALID_ARG, "NULL plan");
    QmcServer *sv = plan->server;
    if (!sv) return QMCCPW_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
        sv->cv_work.notify_all();
    }
    sv->monitor.join();
    plan->server = nullptr;
    delete sv;
    return QMCCPW_OK;
}


int qmccpw_tuning_set(qmccpw_plan_t plan, int32_t precision, int32_t construction, int32_t d, int32_t points_per_tile) {
    g_last_error.clear();
    if (!plan) return fail(QMCCPW_ERR_INVALID_ARG, "NULL plan");
    if (precision != QMCCPW_FP64 && precision != QMCCPW_MIXED)
        return fail(QMCCPW_ERR_INVALID_ARG, "tuning applies to the FP64 and MIXED CUDA-core kernels");
    if (construction < QMCCPW_BB || construction > QMCCPW_PCA_LEAD) return fail(QMCCPW_ERR_INVALID_ARG, "construction");
    if (d < 1 || d > plan->d_max) return fail(QMCCPW_ERR_INVALID_ARG, "d outside the plan");
    std::lock_guard<std::mutex> lock(plan->mu);
    const auto key = std::make_tuple(precision == QMCCPW_FP64 ? 0 : 1, construction, d);
    if (points_per_tile == 0) {
        plan->tuned_tile.erase(key);
        return QMCCPW_OK;
    }
    int lg = 0;
    while (lg < kMaxTileLog2 && (1 << lg) < points_per_tile) ++lg;
    if ((1 << lg) != points_per_tile || points_per_tile < 32)
        return fail(QMCCPW_ERR_INVALID_ARG, "points_per_tile must be a power of two in 32..256");
    if (fused_smem_bytes(precision, construction, d - 1, lg) > 200u * 1024u)
        return fail(QMCCPW_ERR_INVALID_ARG, "tile too large for shared memory");
    plan->tuned_tile[key] = lg;
    return QMCCPW_OK;
}

int qmccpw_tuning_get(qmccpw_plan_t plan, int32_t precision, int32_t construction, int32_t d, int32_t *points_per_tile) {
    g_last_error.clear();
    if (!plan || !points_per_tile) return fail(QMCCPW_ERR_INVALID_ARG, "NULL argument");
    if (d < 1 || d > plan->d_max) return fail(QMCCPW_ERR_INVALID_ARG, "d outside the plan");
    std::lock_guard<std::mutex> lock(plan->mu);
    if (is_tc(precision)) {
        *points_per_tile = 128;
        return QMCCPW_OK;
    }
    auto it = plan->tuned_tile.find(std::make_tuple(precision == QMCCPW_FP64 ? 0 : 1, construction, d));
    *points_per_tile =
        1 << (it != plan->tuned_tile.end() ? it->second : choose_tile_log2(precision, d - 1, construction));
    return QMCCPW_OK;
}

int qmccpw_autotune(qmccpw_plan_t plan, const qmccpw_contract *sample, int32_t count, int32_t precision) {
    g_last_error.clear();
    if (!plan || !sample || count < 1) return fail(QMCCPW_ERR_INVALID_ARG, "NULL or empty sample");
    if (precision != QMCCPW_FP64 && precision != QMCCPW_MIXED)
        return fail(QMCCPW_ERR_INVALID_ARG, "tuning applies to the FP64 and MIXED CUDA-core kernels");
    std::lock_guard<std::mutex> lock(plan->mu);
    QMC_CUDA(cudaSetDevice(plan->device));
    cudaEvent_t e0, e1;
    QMC_CUDA(cudaEventCreate(&e0));
    QMC_CUDA(cudaEventCreate(&e1));
    int rc = QMCCPW_OK;
    std::map<std::pair<int, int>, bool> seen;
    for (int i = 0; i < count && rc == QMCCPW_OK; ++i) {
        const qmccpw_contract &src = sample[i];
        rc = validate_qc(plan, src, precision, false);
        if (rc != QMCCPW_OK) break;
        if (seen[std::make_pair(src.construction, src.option.d)]) continue;
        seen[std::make_pair(src.construction, src.option.d)] = true;
        const auto key = std::make_tuple(precision == QMCCPW_FP64 ? 0 : 1, src.construction, src.option.d);
        plan->tuned_tile.erase(key);
        const int base = choose_tile_log2(precision, src.option.d - 1, src.construction);
        // a workload of its own size: about 2^24 point-dates (2^21 in FP64)
        qmccpw_contract c = src;
        c.R = 4;
        c.first_replicate = 0;
        c.first_point = 0;
        const uint64_t target = precision == QMCCPW_FP64 ? (1ull << 21) : (1ull << 24);
        c.N = std::max<uint64_t>(1024, target / (4ull * static_cast<uint64_t>(c.option.d)));
        int best = base;
        float best_ms = 1e30f;
        for (int lg = std::min(kMaxTileLog2, base + 1); lg >= std::max(5, base - 2) && rc == QMCCPW_OK; --lg) {
            if (fused_smem_bytes(precision, c.construction, c.option.d - 1, lg) > 200u * 1024u) continue;
            plan->tuned_tile[key] = lg;
            qmccpw_batch_s b;
            b.buf = &plan->ws;
            rc = batch_build(plan, &c, 1, precision, false, &b);
            if (rc != QMCCPW_OK) break;
            float times[3];
            for (int rep = 0; rep < 4 && rc == QMCCPW_OK; ++rep) {
                if (rep > 0) cudaEventRecord(e0, plan->stream);
                rc = batch_enqueue(&b, plan->stream);
                if (rep > 0) {
                    cudaEventRecord(e1, plan->stream);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&times[rep - 1], e0, e1);
                }
            }
            if (rc != QMCCPW_OK) break;
            std::sort(times, times + 3);
            if (times[1] < best_ms) {
                best_ms = times[1];
                best = lg;
            }
        }
        plan->tuned_tile[key] = best;
    }
    cudaStreamSynchronize(plan->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
