// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/nfl.h"

namespace nfl {

// Gather epilogues (Alg. 2 step 5 and its pieces); K(0) = 1 for the Gaussian.
enum Op { OP_W = 0, OP_A = 1, OP_LS = 2, OP_DEGREE = 3 };

// Per-node record in tile-sorted order: fractional offsets of n v~ - floor(n v~)
// on each axis and the box-local base cell packed 10 bits per axis.
struct __align__(16) PointF {
    float f[3];
    int32_t cell;
};
struct __align__(32) PointD {
    double f[3];
    int64_t cell;
};

// One unit of spread/gather work: a chunk of the nodes of one tile.
struct WorkItem {
    int32_t tile;
    int32_t start;
    int32_t count;
    int32_t pad;
};

constexpr int kMaxM = 12;
constexpr int kHostSlots = 3;   // device staging slots per direction for host-buffer products
constexpr int kBlockCols = 8;   // columns a block product takes through each stage in one launch
constexpr int kPolyCoef = 10;   // window polynomial degree 9
constexpr int kCheb = 8;        // Chebyshev basis of the dense-cell spread (degree 7)
constexpr int kDenseCell = 32;       // nodes per occupied cell from which a tile is spread by moments
constexpr int kGatherPiece = 8192;   // most nodes per slab piece of the moment interpolation

// Per-column buffers of block products (see Plan::blk).
struct BlockBuffers {
    void *grid = nullptr, *bufA = nullptr, *bufB = nullptr, *g = nullptr, *xsort = nullptr;
    double *xsorted = nullptr;
};

struct Plan {
    // problem
    int64_t n = 0;
    int d = 0, N = 0, m = 0, p = 0, prec = 0;
    int kernel = NFL_KERNEL_GAUSSIAN;
    bool bf16_taps = false;     // BF16W: window taps rounded to BF16 (prec is then FP32)
    double out_scale = 1.0;     // scaled fast sum -> caller's coordinates (multiquadrics: 1/rho, rho)
    double k0 = 1.0;            // K(0) in the caller's coordinates
    double sigma = 0, sigma_t = 0, rho = 1, eps_B = 0;
    double center[3] = {0, 0, 0};
    cudaStream_t stream = 0;
    // one-column products with dense tiles: the moment spread runs on `side`, forked
    // from and joined back into `stream`, so it fills the warp-slice spread's tail
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

    // oversampled grid and its active box
    int ngrid = 0;              // 2N
    int L[3] = {1, 1, 1};       // stored box extent per axis (<= ngrid)
    int wrap[3] = {0, 0, 0};    // 1 when the taps span more than ngrid on that axis
    int64_t t0[3] = {0, 0, 0};  // global index of box position 0 (information only)
    int64_t box_elems = 0;

    // tiles and work items
    int tile_edge = 0;          // cells per tile edge
    int ntile[3] = {1, 1, 1};
    int64_t tiles_total = 0, tiles_nonempty = 0;
    int64_t nitems = 0;
    WorkItem *items = nullptr;          // chunks of one tile (interpolation, other spreads)
    // warp-slice spread: runs of consecutive tiles along axis 2 of one row (pad = number
    // of tiles) or, for tiles with more than one chunk, single chunks (pad = 1)
    int64_t nsitems = 0;
    WorkItem *sitems = nullptr;
    int32_t *tile_start = nullptr;      // first sorted node of each tile; [tiles_total] = n
    std::vector<WorkItem> tile_items;   // host copy of the per-tile chunks, in tile order
    // per tile (3-D, nodes sorted by cell): the occupied cells, then the nodes of each of
    // the tile_edge slabs (cells of one axis-0 position); empty when not sorted by cell
    std::vector<int32_t> tile_cells;
    // one-column products with the dense-cell spread (moments_available): runs over the
    // sparse tiles for the warp spread, and the chunks of the dense tiles
    // the one-column spread and interpolation with dense cells: the warp-slice spread's
    // runs of sparse tiles, the tensor-core interpolation's chunks of sparse tiles and
    // the dense tiles' slab pieces (pad = the slab): at most dense_chunk nodes for the
    // moment spread, kGatherPiece for the moment interpolation (each piece forms or
    // expands its slab's moments once); each list largest first
    int64_t nsparse = 0, ngsparse = 0, nslab = 0, ngslab = 0;
    WorkItem *sparse_items = nullptr, *gsparse_items = nullptr, *slab_items = nullptr, *gslab_items = nullptr;
    int slide_tiles = 8;                // most tiles in one sliding run of the warp spread
    int chunk = 8192;                   // most nodes in one work item (tile chunk, sliding run)
    int dense_cell = kDenseCell;        // nodes per occupied cell from which a tile is dense
    int dense_chunk = 8192;             // most nodes in one slab piece of the moment spread
    int fft_cap = 512;                  // FFT passes: grid points per CTA

    // tile-sorted nodes
    void *pts = nullptr;        // PointF or PointD
    int32_t *perm = nullptr;    // sorted position -> input index
    double *dinv_sorted = nullptr;  // D_E^{-1/2} in sorted order
    void *xsort = nullptr;      // x~ of the current column in sorted order (spread type; 3-D cell kernels)
    double *xsorted = nullptr;  // z of the current column in sorted order: y = z + s f (interpolation epilogue)
    double *degree = nullptr;   // d_E in input order
    double min_deg = 0, max_deg = 0;
    bool degree_ok = false;

    // window phi(delta)/phi(0) = (m / s) sinh(b s) / sinh(b m), s = sqrt(m^2 - delta^2);
    // kb_inv_sinh_bm holds 1 / (1 - e^{-2 b m}) for the cancellation-free form
    double kb_b = 0, kb_inv_sinh_bm = 0;
    // FP32 window by taps: for tap j of a node at fractional offset f in [0, 1),
    // phi(f + m - 1 - j) / phi(0) = sum_k kb_poly[j][k] t^k, t = 2 f - 1, to
    // within FP32 rounding of the peak (Chebyshev interpolation in FP64).
    float kb_poly[2 * kMaxM][kPolyCoef] = {};
    // the same taps in the Chebyshev basis T_k(t), k < kCheb (interpolation at kCheb
    // Chebyshev points): phi(f + m - 1 - j) / phi(0) = sum_k kb_cheb[j][k] T_k(2 f - 1)
    float kb_cheb[2 * kMaxM][kCheb] = {};

    // FFT data
    int K[3] = {1, 1, 1};       // kept frequencies per axis (R2C axis N/2+1, others N+1)
    // one-column buffers: grid, bufA, bufB, g, xsort, xsorted (below); block products use
    // blk, the same buffers for block_cols columns (column strides box_elems, bufA_elems,
    // bufB_elems, box_elems and n), made on the first block product; column c's FP32C
    // scale sum |x~| at scratch[c]
    BlockBuffers blk;
    int block_cols = 1;                 // columns per block product (1: column by column)
    int l2_bytes = 0;
    int64_t bufA_elems = 0, bufB_elems = 0;
    void *grid = nullptr;       // spreading grid: float, double or int64 (FP32C)
    void *bufA = nullptr;       // complex FFT intermediates
    void *bufB = nullptr;
    void *g = nullptr;          // interpolation grid (real, FFT type)
    void *mult = nullptr;       // fused multiplier M_eff (real, FFT type)
    void *twiddle = nullptr;    // e^{-2 pi i q / ngrid}, q < ngrid/2 (complex, FFT type)
    double *scratch = nullptr;  // small device scalars (reductions, fixed-point scale)
    int *error_flag = nullptr;  // set by a kernel whose bounded wait ran out
    unsigned *work_counter = nullptr;   // next work item of [0] spread, [1] gather, [2] dense-cell spread,
                                        // [3] dense-cell gather (reset per column)
    int fault_kind = 0;         // fault test (nfl_plan_inject_fault): 1 = interpolation MMAs never issued
    int num_sms = 0;

    // host-buffer products (nfl_apply_host), made on first use: kHostSlots device
    // slots for x columns followed by kHostSlots for y columns, and two copy streams
    double *host_stage = nullptr;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_start = nullptr;
    cudaEvent_t ev_in[kHostSlots] = {}, ev_done[kHostSlots] = {}, ev_out[kHostSlots] = {};

    // several one-column products in one call: a second set of staging buffers and the
    // stream that stages column c + 1 while column c is transformed and interpolated
    // (made on the first such call)
    void *pipe_xsort = nullptr;
    double *pipe_xsorted = nullptr, *pipe_scratch = nullptr;
    cudaStream_t pipe_stream = nullptr;
    cudaEvent_t pipe_fork = nullptr, pipe_spread_done = nullptr, pipe_staged[2] = {};

    // stage timing: 5 events per timed column (before prep, spread, fft, gather, after)
    bool profile = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    std::vector<int> event_cols;        // columns covered by each timed product
};

// Precision-dependent element types.
inline bool fft_is_double(int prec) { return prec == NFL_PREC_FP64; }
inline bool points_are_double(int prec) { return prec == NFL_PREC_FP64; }

// launchers (stream-ordered, no host sync)
cudaError_t prepare_spread(Plan &P, int op, const double *x, int64_t ldx, int nc, bool ones, bool scale_dinv);
// the grid and work counters cleared for a product (the first half of prepare_spread)
cudaError_t clear_spread(Plan &P, int nc);
cudaError_t launch_spread(Plan &P, const double *x, int64_t col_off, bool ones, bool scale_dinv);
cudaError_t launch_fft(Plan &P, int nc = 1);
cudaError_t launch_gather(Plan &P, int op, const double *x, double *y);
cudaError_t launch_fixed_scale(Plan &P, const double *x, bool ones, bool scale_dinv);

// the whole Alg. 1 pipeline for one column: y = epilogue(W~ x)
nfl_status run_column(Plan &P, int op, const double *x, double *y);

// 3-D atomic-free spreading (spread3.cu): tile edge it needs for cut-off m (0: not available)
int column_tile_edge(int m);
cudaError_t launch_spread3_columns(Plan &P, const double *x, bool ones, bool scale_dinv);
cudaError_t stage_spread3_values(Plan &P, int op, const double *x, int64_t ldx, int nc, bool ones,
                                 bool scale_dinv);
bool spread_warp_available(const Plan &P);
cudaError_t launch_spread3_warp(Plan &P, int nc = 1);

// 3-D interpolation on the tensor cores (gather_tc.cu)
bool gather_tc_available(const Plan &P);
cudaError_t launch_gather_tc(Plan &P, int op, const double *x, double *y, int64_t ldy = 0, int nc = 1);

// streams of nfl_apply_batched: plans are spread over them, forked from and joined
// back to the caller's stream
constexpr int kBatchStreams = 16;
struct BatchStreams {
    bool ready = false;
    cudaStream_t s[kBatchStreams] = {};
    cudaEvent_t join[kBatchStreams] = {};
    cudaEvent_t fork = nullptr;
};
BatchStreams *batch_streams();

// A batch of plans whose products run with one launch per stage (batch.cu): every
// member is a 3-D FP32 / FP32C / BF16W plan of the same m and N on the warp-spread /
// tensor-core path; the batch owns contiguous staging, grid and FFT buffers for all
// members' columns and binds the caller's input and output blocks.
struct BatchPlanDev {
    const PointF *pts;
    const int32_t *perm;
    const double *dinv;
    const int32_t *tile_start;
    const WorkItem *items;        // gather chunks of the plan
    const WorkItem *sitems;       // warp-spread items of the plan
    const double *x;              // caller's input block, column c at x + c ldx
    double *y;                    // caller's output block, column c at y + c ldy
    int64_t ldx, ldy;
    float *xs;                    // staged x~, column c at xs + c n
    double *zd;                   // staged epilogue z, column c at zd + c n
    void *grid;                   // spreading grid, column c at grid + c box
    float *g;                     // interpolation grid, column c at g + c box
    double *abs_sum;              // FP32C scale sums, one per column
    int64_t n, box;
    int ntile[3], L[3], wrap[3];
    double k0, out_scale;
    int *error_flag;              // the member's device error flag
};
struct BatchItem {
    int32_t plan, item;
};
// One FFT pass over contiguous lines (fft.cu).
struct PassArgs {
    const void *in;
    void *out;
    int nA, nB;
    int64_t sA, sB;
    int Lin;
    unsigned lin_magic;   // ceil(2^32 / Lin): e / Lin = umulhi(e, lin_magic) for e < 2^22
    int64_t oC, oA;
    int Lout;
    int n, logn, N;
    int BB;
    const void *tw;       // e^{-2 pi i q / n}, q < n/2
    const void *M;        // fused multiplier, index ((b * nA) + a) * (N + 1) + (k + N/2)
    int real_in, real_out;
    const double *abs_sum;  // int64 fixed-point input: sum |x~| of the spread call, per column
    int64_t in_cstride, out_cstride;   // elements between the columns of a block (grid.z)
};

struct Batch {
    std::vector<Plan *> plans;
    int G = 0, op = 0, ncol = 1, m = 0, N = 0, prec = 0;
    bool bf16 = false;
    int num_sms = 0;
    BatchPlanDev *desc = nullptr;        // device, G entries
    BatchItem *sitems = nullptr, *gitems = nullptr;   // device: all spread / gather items, largest first
    int64_t nsitems = 0, ngitems = 0;
    int *stage_start = nullptr;          // device: first staging CTA of each plan, [G] = total
    int stage_ctas = 0;
    unsigned *counter = nullptr;         // device: [0] spread, [1] gather
    void *grid_all = nullptr;            // contiguous buffers of all members' columns
    size_t grid_bytes = 0;
    double *abs_all = nullptr;
    void *xs_all = nullptr, *zd_all = nullptr, *g_all = nullptr, *bufA_all = nullptr, *bufB_all = nullptr;
    PassArgs *pass_args[5] = {};         // device, G entries per FFT pass
    int *pass_start[5] = {};             // device: first CTA of each plan per pass, [G] = total
    int pass_ctas[5] = {};
    int fft_cap = 512;
    int *error_flag = nullptr;
    float poly[2 * kMaxM][kPolyCoef] = {};
    // stage timing: 5 events per timed run (before staging, spread, FFT, interpolation, after)
    bool profile = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    cudaStream_t last_stream = nullptr;
};
cudaError_t launch_stage_batch(Batch &B, cudaStream_t s);
cudaError_t launch_spread3_warp_batch(Batch &B, cudaStream_t s);
cudaError_t launch_fft_batch(Batch &B, cudaStream_t s);
cudaError_t launch_gather_tc_batch(Batch &B, cudaStream_t s);
// the five 3-D FFT passes of a plan over given buffers (column strides of the grids
// box, of bufA / bufB their sizes), with BB and the magic divisor set for cap
int fft_passes_3d(const Plan &P, const void *grid, void *bufA, void *bufB, void *g, int64_t sa, int64_t sb,
                  int cap, PassArgs *out, int nc, int *ctas);

// number of kernels one column launches
int kernels_per_column(const Plan &P);

// block products: nc <= block_cols columns through each stage in one launch (3-D
// warp spread + tensor-core gather only); the buffers hold block_cols columns
bool block_path_available(const Plan &P);
nfl_status ensure_columns(Plan &P, int nc);

// warp-spread work items from tile_items with runs of at most slide_tiles tiles
nfl_status rebuild_spread_items(Plan &P);
// re-split every tile into chunks of at most `chunk` nodes (host lists and device copies)
nfl_status rechunk_items(Plan &P, int chunk);

// the warp spread's work list built from tile_items (host)
std::vector<WorkItem> spread_item_list(const Plan &P);
// dense-cell spread (spread3_moments.cu): available for the plan, the split of the
// work lists into sliding runs over sparse tiles and the chunks of dense tiles (host),
// and the launch over the dense chunks (one column)
bool moments_available(const Plan &P);
struct ItemLists {
    std::vector<WorkItem> sparse, gsparse, slab, gslab;
};
ItemLists split_item_lists(const Plan &P);
cudaError_t launch_spread3_moments(Plan &P, cudaStream_t s);
cudaError_t launch_gather3_moments(Plan &P, int op, double *y, cudaStream_t s);
// `side` waits for the work queued on `stream` so far / `stream` waits for `side`
cudaError_t side_fork(Plan &P);
cudaError_t side_join(Plan &P);

}  // namespace nfl

#define NFL_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return _e;                    \
    } while (0)

#define NFL_STATUS_TRY(expr)                                                         \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess)                                                       \
            return _e == cudaErrorMemoryAllocation ? NFL_ERR_OUT_OF_MEMORY : NFL_ERR_CUDA; \
    } while (0)
