// Internal declarations shared by the translation units of libqmccpw.
// Not part of the C-ABI (include/qmccpw.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qmccpw.h"

namespace qmccpw {

// ----------------------------------------------------------------------------
// Host tables (tables.cpp)
// ----------------------------------------------------------------------------

// SplitMix64 (Steele, Lea & Flood 2014), evaluated counter-style: the value
// for `counter` under `key` is output number counter+1 of the generator whose
// state starts at `key`.
uint64_t splitmix64_at(uint64_t key, uint64_t counter);

// Key of the stream that draws the initial direction integers.
constexpr uint64_t kDirectionKey = 0x2209113370D1CE5Dull;

// Direction integers v[j*32 + b] (b = 0..31 is the index bit) of Sobol'
// dimensions j = 0..ndims-1 (Sec. 2.2.2).
std::vector<uint32_t> direction_integers(int ndims);

// One step of the breadth-first Brownian bridge (Sec. 4.4) on s_i = i*dt:
// W[m] = wl*W[l] + wr*W[r] + sd*z, z being Sobol' dimension `step`.
struct BridgeStep {
    int32_t m, l, r, m_float_bits;  // the last field holds the bits of float(m)
};
struct BridgePlan {
    int n = 0;
    std::vector<BridgeStep> steps;       // n steps in consumption order
    std::vector<double> w;               // 3 per step: wl, wr, sd
    std::vector<int32_t> level_start;    // steps of level L are [level_start[L], level_start[L+1])
};
BridgePlan bridge_plan(int n, double dt);

// PCA factor A (n x n, row-major, A[i-1][k-1]) of Sigma_ik = dt*min(i,k).
std::vector<double> pca_factor(int n, double dt);

// ----------------------------------------------------------------------------
// Device-side descriptors (shared by api.cu and kernels.cu)
// ----------------------------------------------------------------------------

constexpr int kThreads = 256;            // threads per CTA of the fused kernel
constexpr int kMaxTileLog2 = 8;          // at most 256 points per tile

// Everything a CTA needs about its contract.  Built on the host, uploaded
// once per batch, read through the constant/L1 path.
struct ContractDev {
    int32_t type, d, n, construction;
    int32_t tile_log2;                   // P = 1 << tile_log2 points per tile
    int32_t chunk_log2;                  // Gray-code chunk length in the Sobol' phase
    int32_t R, tiles;                    // replicates, tiles per replicate
    int32_t tpi, items;                  // tiles per work item, work items per replicate (set_item_grouping)
    int32_t groups;                      // kThreads / P threads per point in the path phase
    int32_t n_levels;                    // bridge levels
    int32_t row_stride;                  // shared-memory row (point) stride in elements, odd
    int32_t z_by_dim;                    // 1: z of dimension j at column j+1+slot_shift; 0: at the date node j+slot_shift drives
    int32_t slot_shift;                  // 1 for the leading-coordinate constructions (dimension j drives node j+1), else 0
    int32_t lead_increasing;             // leading-coordinate constructions: the loadings strictly increase with the date
    int32_t rep_first;                   // randomisation index of the contract's replicate 0
    uint64_t N;
    uint64_t k_first;                    // Sobol' index of the contract's point 0
    uint64_t item_base;                  // first work item of this contract
    uint64_t rep_base;                   // first replicate slot of this contract (in per-replicate arrays)
    // per-d tables for unit spacing (device pointers); kernels scale by sqrt(dt)
    const BridgeStep *steps;
    const double *w64;                   // 3 per step: wl, wr, c (sd = c sqrt(dt))
    const float *w32;                    // (hi, lo) float pairs of wl, wr, sd + 2 pad: 8 per step
    const int32_t *level_start;
    const int32_t *slot_dim;             // shared-memory bridge (BB, z at its node): the dimension driving date m, m = 1..n; else null
    const int32_t *sub_start;            // shared-memory bridge with G = groups threads per point: per level below the top ones, G + 1 run starts of the threads' subtrees; else null
    const double *pca64;                 // n x n row-major
    const float *pcaT32;                 // A^T as float, [k][i], i padded to a multiple of 16 with zeros
    const float *pcaT32lo;               // A^T - float(A^T) in the same layout (leading-coordinate PCA)
    const void *tc_operand;              // tensor-core PCA: Ahat hi then lo, K-major core-matrix layout
    const double *lead_a64;              // leading-coordinate constructions: its loading on dates 1..d, unit spacing
    const float *lead_a32;               // the same as float pairs (hi, lo)
    // market-derived constants
    double S0, K, T, r, sigma;
    double dt;                           // t_1 = T/d: spacing of the separated dates
    double a;                            // sigma*sqrt(t_1)
    double omega;                        // r - sigma^2/2
    double psi0;                         // ln(K/S0) - omega*t_1 (switch point numerator before ln X^)
    double disc;                         // exp(-r T)
    double disc1;                        // exp(r (t_1 - T))
    double sqrt_t1;
    double inv_a;                        // 1/a
    double disc1_S0;                     // disc1 * S0
    double disc_K;                       // disc * K
    double k_bin_delta;                  // disc / (S0 a)
    double k_bin_gamma;                  // disc / (S0^2 a)
    double k_call_gamma;                 // disc K / (S0^2 a)
    double inv_sigma;
    double inv_d;                        // 1/d
    double ln_lead_c0;                   // ln(S0/d): leading-coordinate constructions
    double ln_S0;                        // ln S0 (the lookback under leading-coordinate conditioning)
    double ln_K;
    double lead_amean;                   // leading-coordinate constructions: mean over the dates of the loading times sqrt(dt)
    // constants of the float path as float hi + lo pairs (split_ff)
    // path: the exponent (sigma sqrt(dt)) w + (omega dt) node of the unit-spacing path w
    float ff_sig_sdt[2], ff_om_dt[2];
    float ff_sqrt_t1[2];                 // sqrt(dt)
    float ff_nsig_dt[2];                 // -sigma dt
    float ff_inv_d[2], ff_sdt_d[2];      // 1/d, sqrt(dt)/d
    float ff_nsigdt_d[2];                // -sigma dt / d
    float ff_sig_sdt_d[2];               // sigma sqrt(dt) / d (geometric mean)
    float ff_geo_l0[2], ff_geo_d0[2];    // omega dt S1 / d and -sigma dt S1 / d, S1 = n(n+1)/2
    // conditional step (1/sqrt(2 pi) folded into the density's constants)
    float ff_psi0[2], ff_inv_a[2], ff_inv_sigma[2], ff_a[2];
    float ff_disc1_S0[2], ff_disc_K[2], ff_disc1[2], ff_disc[2];
    float ff_kv_call[2];                 // disc K sqrt(t_1) / sqrt(2 pi)
    float ff_kg_call[2];                 // disc K / (S0^2 a sqrt(2 pi))
    float ff_kd_bin[2];                  // disc / (S0 a sqrt(2 pi))
    float ff_kg_bin[2];                  // disc / (S0^2 a sqrt(2 pi))
    float ff_kphi[2];                    // disc / sqrt(2 pi)
    // the leading-coordinate float path
    float ff_sig[2], ff_lnS0d[2], ff_lnK[2];
};

// A work item is a run of consecutive tiles of one replicate; its CTA adds
// the tiles' block sums (compensated, in tile order) and writes one 32-byte
// slot.  Large contracts take up to kMaxTilesPerItem tiles per item (one slot
// instead of 16: less scratch and fewer writes), while every replicate keeps
// at least kMinItemsPerRep items for the dynamic schedule to balance.  The
// grouping depends on the tiles per replicate only (not on R, the batch or
// the device), so a replicate's estimate is the same whichever call, batch,
// replicate range or server computes it.
constexpr int kMaxTilesPerItem = 16;
constexpr int kMinItemsPerRep = 256;
inline void set_item_grouping(ContractDev &c) {
    int tpi = 1;
    while (tpi < kMaxTilesPerItem && static_cast<int64_t>(tpi) * 2 * kMinItemsPerRep <= c.tiles) tpi *= 2;
    c.tpi = tpi;
    c.items = (c.tiles + tpi - 1) / tpi;
}

// hi + lo float pair of a double (hi = nearest float, lo = nearest float of the rest)
inline void split_ff(double x, float out[2]) {
    out[0] = static_cast<float>(x);
    out[1] = static_cast<float>(x - static_cast<double>(out[0]));
}

// Fill the derived constants of a contract from S0, K, T, r, sigma, d (host).
void contract_constants(ContractDev &c);

// Per-launch parameters of the fused kernel.
struct LaunchParams {
    const ContractDev *contracts;
    int32_t count;
    int32_t pad;
    uint64_t item_begin, item_end;       // work items [item_begin, item_end) of this launch
    const uint64_t *item_base;           // contract item bases, for the binary search
    const uint32_t *sobol_table;         // [rep][b][j] scrambled direction integers
    const uint32_t *sobol_shift;         // [rep][j]
    int32_t jstride;                     // j stride of the table rows
    uint32_t rep_offset;                 // added to every replicate index (diagnostics; 0 otherwise)
    double *tile_sums;                   // items x 4 partial sums (scratch)
    double *point_out;                   // optional per-point values, point x 4 (diagnostics)
    uint64_t point_k0;                   // index of the contract's point 0 (diagnostics; 0 otherwise)
    int *error_flag;                     // set to a qmccpw_status by a kernel whose bounded wait expired
    unsigned long long *work_counter;    // items handed out so far (zeroed before each launch)
};

// Launchers (kernels.cu).  Return the cudaError_t as int.
int launch_fused(const LaunchParams &p, int precision, int construction, size_t smem_bytes, int grid, void *stream);
int launch_reduce(const ContractDev *contracts, int32_t count, const double *tile_sums,
                  double *per_rep, double *stats, uint64_t total_reps, const uint64_t *rep_owner,
                  void *stream);
int launch_gathered_stats(const double *per_rep, const int64_t *first_row, const int32_t *R, int count,
                          double *stats, void *stream);
int launch_scatter_replicates(const double *per_rep, const int64_t *dst_row, uint64_t slots, double *dst,
                              void *stream);
int launch_scramble(uint64_t seed, const uint32_t *v, int ndims, int jstride, int reps,
                    uint32_t *table, uint32_t *shift, void *stream);
int launch_sobol_dump(const uint32_t *table, const uint32_t *shift, int jstride, int ndims,
                      uint64_t k0, uint64_t count, uint32_t *out, void *stream);
// dynamic shared memory of one CTA for a contract with n dims and 2^tile_log2 points
// Shared-memory elements per point of the fused kernel's tile: z / W~ in
// slots 0..n (odd stride); the leading-coordinate constructions build the
// whole path, slots 0..n+1, and the PCA one keeps its rest R in a second row.
inline int tile_row_elems(int construction, int n) {
    if (construction == QMCCPW_BB_LEAD) return (n + 2) | 1;
    if (construction == QMCCPW_PCA_LEAD) return 2 * ((n + 2) | 1);
    return (n + 1) | 1;
}
size_t fused_smem_bytes(int precision, int construction, int n, int tile_log2);
int fused_set_smem_limit(int precision, size_t optin_bytes);  // optin_bytes: the device's per-block opt-in maximum
int fused_occupancy(int precision, int construction, size_t smem_bytes, int *blocks_per_sm);

// ----------------------------------------------------------------------------
// Device-resident serving loop (serve_impl.cuh, serve_f32.cu, serve_f64.cu;
// host side in api.cu)
// ----------------------------------------------------------------------------
// The work items of every request, in publication order, are numbered by
// one global ticket sequence: request s owns tickets [first_ticket,
// first_ticket + items), item = replicate-major (replicate, tile) as in a
// batch.  The host writes a request into a ring of host-mapped entries, then
// publishes it by raising published_seq and published_tickets.  One CTA of
// the persistent kernel, the dispatcher, watches those host words, copies
// each new entry into a device-memory ring and republishes it in device
// memory; the other CTAs, the workers, touch host memory only to write
// results: they take tickets from a device counter, wait (bounded by
// %globaltimer) until their ticket is published on the device, run the item
// and count it; the worker that finishes a request's last item reduces it
// and raises the request's completion flag in host-mapped memory.  A worker
// that waits longer than the idle limit (or sees the stop word) records the
// ticket it holds and leaves, the dispatcher leaves after the last worker
// (or on the stop word), and the last CTA to leave carries every held ticket
// over to the next launch, which hands them out first, so no published item
// is lost when the kernel exits and the host launches it again.
constexpr int kServeMaxGrid = 1024;          // CTAs of one serving launch at most (workers + dispatcher)
constexpr int kServeRetryCap = 2 * kServeMaxGrid;

// One ring entry (host-mapped, and its copy in the device ring).  The host
// writes an entry before publication and while seq holds ~0, the
// dispatcher its copy likewise, so a reader that sees the same seq before
// and after reading knows the entry was not being rewritten.
struct ServeRequest {
    uint64_t seq;                            // request number
    uint64_t first_ticket, items;            // its tickets
    double *tile_sums;                       // device: items x 4 tile slots, then R x 4 replicate estimates
    double *out;                             // host-mapped: R x 4 replicate estimates, mean[4], se[4]
    ContractDev c;                           // rep_first set; item_base and rep_base unused
};

// Words the host writes (host-mapped).
struct ServeControl {
    uint64_t published_tickets;              // tickets below it belong to published requests
    uint64_t published_seq;                  // requests below it are in the ring
    uint64_t oldest_live;                    // requests below it are finished (their entries may be reused)
    uint32_t stop;                           // nonzero: every CTA leaves at its next wait
    uint32_t pad;
};

// Written by the last CTA of a launch (host-mapped).
struct ServeExit {
    uint32_t launch;                         // the launch's number
    uint32_t reason;                         // 1 idle limit, 2 stop word, 3 carried tickets above capacity,
                                             // 4 a ticket without a request in the ring
    uint64_t next_ticket;                    // first ticket never handed out
    uint32_t carried;                        // tickets carried to the next launch
    uint32_t pad;
};

// Device-memory state carried from one launch to the next (zeroed once).
struct ServeState {
    unsigned long long next_ticket;          // fresh tickets
    unsigned int retry_count;                // carried tickets of this launch, handed out first
    unsigned int retry_next;
    unsigned int exited;                     // CTAs of this launch that have left
    unsigned int bad_ticket;                 // nonzero: a CTA found no request for its ticket (exit reason 4)
    // the dispatcher's device copies of the host words
    uint64_t pub_tickets;                    // tickets below it are published in the device ring
    uint64_t pub_seq;                        // requests below it are in the device ring
    uint64_t oldest_live;
    uint32_t stop;
    uint32_t pad;
    unsigned long long retry[kServeRetryCap];
    unsigned long long abandoned[kServeMaxGrid];  // the ticket each worker held when it left
};

struct ServeParams {
    const ServeRequest *ring;                // host-mapped, cap entries
    ServeRequest *dev_ring;                  // device copies, cap entries
    uint64_t cap;                            // ring entries, a power of two
    const ServeControl *ctl;                 // host-mapped
    uint64_t *done;                          // host-mapped, per entry: seq + 1 once that request finished
    ServeExit *exit_rec;                     // host-mapped
    ServeState *st;                          // device
    unsigned long long *done_items;          // device, per entry: finished items of the request there
    const uint32_t *sobol_table;
    const uint32_t *sobol_shift;
    int32_t jstride;
    uint32_t launch;
    uint64_t idle_ns;                        // a worker leaves after waiting this long for a published ticket
};
// The serving kernels: precision FP64 or MIXED; with_pca false builds the
// MIXED kernel without the PCA product (three CTAs per SM instead of two).
// grid = workers + 1 (the last CTA is the dispatcher).
int launch_serve(const ServeParams &p, int precision, bool with_pca, size_t smem_bytes, int grid, void *stream);
int serve_prepare(int precision, bool with_pca, size_t optin_bytes);  // raise the dynamic shared-memory limit
int serve_occupancy(int precision, bool with_pca, size_t smem_bytes, int *blocks_per_sm);
int serve_f32_launch(const ServeParams &p, bool with_pca, size_t smem_bytes, int grid, void *stream);
int serve_f32_prepare(bool with_pca, size_t optin_bytes);
int serve_f32_occupancy(bool with_pca, size_t smem_bytes, int *blocks_per_sm);
int serve_f64_launch(const ServeParams &p, size_t smem_bytes, int grid, void *stream);
int serve_f64_prepare(size_t optin_bytes);
int serve_f64_occupancy(size_t smem_bytes, int *blocks_per_sm);

// Tensor-core PCA (pca_tc.cu).  kind 0: bf16 split (4 products), 1: tf32
// split (3 products), both n <= 64 with Ahat resident; kinds 2 (bf16) and 3
// (tf32): n <= 256, Ahat streamed in K-chunks.
size_t pca_tc_smem_bytes(int kind);
int launch_bounded_wait_probe(uint64_t limit_ns, int *status, void *stream);
int pca_tc_max_n(int kind);                          // largest n (dimensions) the kind supports
int pca_tc_prepare(int kind, size_t smem_bytes);     // raise the dynamic shared memory limit
int pca_tc_occupancy(int kind, size_t smem_bytes, int *blocks);
int launch_pca_tc(const LaunchParams &p, int kind, size_t smem_bytes, int grid, void *stream);
void pca_tc_operand(int kind, int n, const std::vector<double> &A_unit, std::vector<unsigned char> &out);

// ----------------------------------------------------------------------------
// Basket of m correlated assets (basket.cu; host side in api.cu)
// ----------------------------------------------------------------------------
// Lower Cholesky factor L of an m x m symmetric matrix C (row-major, m <= 8):
// false if C is not positive definite.
bool cholesky_lower(int m, const double *C, double *L);

// Everything the basket kernel reads about its contract: a kernel parameter
// (the constants reach the arithmetic as constant-bank operands).
struct BasketDev {
    int32_t type, d, n, m;
    int32_t tile_log2, chunk_log2, groups, row_stride;
    int32_t n_levels, pad0;
    uint64_t N, tiles;
    const BridgeStep *steps;             // unit-spacing bridge of the n nodes (shared with the single-asset tables)
    const double *w64;
    const float *w32;
    const int32_t *level_start;
    const int32_t *slot_of_dim;          // m d - 1 entries: the row slot Sobol' dimension j fills
    double S0, K, disc, sqrt_dt, ln_K;
    double L[QMCCPW_ASSETS_MAX * QMCCPW_ASSETS_MAX];  // Cholesky factor, [i*8 + k]
    double sig_sdt[QMCCPW_ASSETS_MAX];   // sigma_i sqrt(dt)
    double om_dt[QMCCPW_ASSETS_MAX];     // omega_i dt
    double sig_dt[QMCCPW_ASSETS_MAX];    // sigma_i dt
    double f[QMCCPW_ASSETS_MAX];         // w_i a_i S0 / d
    double bcoef[QMCCPW_ASSETS_MAX];     // b_i = sigma_i L_i1 sqrt(dt)
    double l1[QMCCPW_ASSETS_MAX];        // L_i1 sqrt(dt)
    double v[QMCCPW_ASSETS_MAX];         // relative volatility (d sigma_i / d sigma)
    double ehalf[QMCCPW_ASSETS_MAX];     // e^{b_i^2 / 2}
    float Lf[QMCCPW_ASSETS_MAX * QMCCPW_ASSETS_MAX][2];  // L as float pairs (hi, lo)
    float ff_sig_sdt[QMCCPW_ASSETS_MAX][2], ff_om_dt[QMCCPW_ASSETS_MAX][2];
};

struct BasketParams {
    BasketDev b;
    const uint32_t *sobol_table;         // [rep][b][j] scrambled direction integers
    const uint32_t *sobol_shift;         // [rep][j]
    int32_t jstride;
    uint32_t rep_offset;                 // randomisation index of replicate 0
    uint64_t items;                      // R x tiles work items, replicate-major
    double *tile_sums;                   // items x 4
    double *point_out;                   // optional per-point values (diagnostics)
    uint64_t point_k0;                   // index of point 0 (diagnostics; 0 otherwise)
};
int launch_basket(const BasketParams &p, int precision, size_t smem_bytes, int grid, void *stream);
int basket_prepare(size_t optin_bytes);
int basket_occupancy(int precision, size_t smem_bytes, int *blocks_per_sm);

// Pipe micro-benchmarks (peaks.cu): 0, a cudaError_t, or -QMCCPW_ERR_TIMEOUT.
int measure_pipe_peaks(int device, qmccpw_pipe_peaks *out);

}  // namespace qmccpw
