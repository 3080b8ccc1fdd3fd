// Internal types of libpc: host-side geometry of the product-convolution
// operator and the device-side descriptors its kernels consume.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <string>
#include <map>
#include <unordered_map>
#include <vector>

#include "pc.h"

namespace pc {

// ---------------------------------------------------------------------------
// Host geometry (Section 2.2 of the paper): box, leaves, sample points,
// cells(p_k), nbrs(k), bbox(U_k).  Coordinates use 3 slots; for 2D operators
// slot 2 is unused (extent 1, coordinate 0).
// ---------------------------------------------------------------------------
using I3 = std::array<int64_t, 3>;

struct Geometry {
    int d = 0;
    I3 shape{1, 1, 1};
    std::vector<I3> cell_lo, cell_hi;
    std::vector<I3> pts;                       // sample points, lexicographic
    std::vector<std::vector<int32_t>> points_of;  // per leaf: sample points in it (closed)
    std::vector<std::vector<int32_t>> cells_of;   // per point: leaves containing it
    std::vector<std::vector<int32_t>> nbrs;       // per point, ascending, includes itself
    std::vector<I3> bb_lo, bb_hi;              // bbox(U_k)
    int64_t bbox_elems(int k) const {
        int64_t n = 1;
        for (int a = 0; a < d; ++a) n *= bb_hi[k][a] - bb_lo[k][a] + 1;
        return n;
    }
};

// Validate the grid and build the geometry.  Returns PC_OK or PC_ERR_GRID /
// PC_ERR_ARG with a message in err.
pc_status build_geometry(const pc_box *box, const pc_grid *grid, Geometry &g, std::string &err);

// Harmonic weights (Section 2.4) on bbox(U_k), FP64, concatenated for k =
// 0..r-1; off[k] is the element offset of w_k.
pc_status build_weights(const Geometry &g, std::vector<double> &w, std::vector<int64_t> &off,
                        std::string &err);

// Extended impulse responses (Section 2.5) on the window [-R, R]^d, FP64,
// [r][(2R+1)^d].
void build_extension(const Geometry &g, int R, const double *phi, std::vector<double> &phiE);

// ---------------------------------------------------------------------------
// Device descriptors
// ---------------------------------------------------------------------------
// One unit of convolution work: an input tile of bbox(U_k) convolved with one
// sub-window of phi_k^E.  When 2R+1 is too wide for the FFT size, the window
// [-R, R]^d is cut into sub-windows with their own spectra; by linearity the
// sum over sub-windows is the full convolution.
struct Tile {
    int32_t patch;       // k
    int32_t spec;        // spectrum index (patch * nsub^d + sub-window)
    int32_t in_lo[3];    // input tile origin in Omega
    int32_t in_ext[3];   // input tile extents (<= T)
    int32_t out_lo[3];   // origin of the tile's linear-convolution output (may be < 0)
    int32_t kext[3];     // sub-window extents: output extent = in_ext + kext - 1
    int32_t w_ld[2];     // strides of the patch weight window: 2D {ext1, 1}; 3D {ext1*ext2, ext2}
    int64_t w_base;      // element offset of the weight at in_lo
};

// Cut of the kernel window [-R, R] (per axis) into nsub sub-windows of
// extent <= ws; sub-window s starts at -R + s * ws.
struct WindowSplit {
    int nsub = 1;
    int ws = 1;
};

struct Schedule {
    std::vector<Tile> tiles;                 // ordered by colour
    std::vector<int32_t> color_start;        // [n_colors + 1] into tiles
    std::vector<int32_t> dep_start;          // [n_tiles + 1]
    std::vector<int32_t> dep;                // tiles (indices into `tiles`) that must add first
};

// Split each bbox(U_k) into input tiles of extent <= T, colour the tiles so
// that tiles of one colour have disjoint output boxes (tile (+) [-R, R]^d,
// clipped to Omega) and disjoint input boxes, and list for every tile the
// overlapping tiles of lower colour.  Output pixels of the forward apply (and
// of the adjoint, which adds into the input boxes) then receive their
// contributions in colour order.
// With a non-empty `patches`, only those patches are tiled, and tile.spec
// numbers their spectra by position in the list (q * nsub^d + sub-window).
void build_schedule(const Geometry &g, int R, int T, const WindowSplit &ws, const std::vector<int64_t> &w_off,
                    Schedule &s, const std::vector<int32_t> &patches = {});

// One launch shape of an operator whose patches use different ones: its
// tiles are [tile_off, tile_off + n_tiles) of the operator's tile array (with
// the tiles' own colour classes and dependency lists, indices local to the
// part), its spectra start at spec_off complex values into the operator's
// spectra.  Each part is one launch of the patch kernel.
struct Part {
    int P = 0, T = 0;
    WindowSplit split;
    std::vector<int32_t> patches;    // the sample points k of the part, ascending
    int tile_off = 0, n_tiles = 0;
    int cs_off = 0, n_colors = 0;    // colour offsets at d_color_start + cs_off ([n_colors + 1])
    int ds_off = 0;                  // dependency starts at d_dep_start + ds_off ([n_tiles + 1])
    int dep_off = 0;                 // dependencies at d_dep + dep_off
    int64_t spec_off = 0, spec_stride = 0;
    void *d_tw = nullptr;            // W_P^j in compute precision (owned by the operator)
    int ctas = 0;
};

// Where the 2D adjoint kernel's store mode writes a tile's unweighted
// correlation block: element (b, row, col) of the tile's input box goes to
// store_base[off + b * ld_rhs + row * ld_row + col].
struct StoreDesc {
    int64_t off;
    int64_t ld_rhs;
    int32_t ld_row;
    int32_t pad_;
};

// Kernel parameter block shared by the 2D and 3D fused kernels.
struct ApplyParams {
    const void *x;
    void *y;
    int64_t ldx, ldy;
    int32_t nrhs, npairs;
    int32_t n[3];               // extents of the box y lives on (2D: n[2] = 1)
    int32_t R;
    int32_t nx[3];              // extents of the box x lives on (n for a whole-box apply; the source box S
                                // of a block apply); 2D: nx[2] = 1
    int32_t pad_nx_;
    const Tile *tiles;
    const int32_t *color_start;
    int32_t n_colors;
    const int32_t *dep_start;
    const int32_t *dep;
    uint32_t *done;             // [n_tiles][done_ld]
    int32_t done_ld;
    uint32_t epoch;
    int32_t *ctrl;              // [0..1] 64-bit work counter, [2] timeout flag
    const void *spec;           // spectra, per patch spec_stride complex values
    int64_t spec_stride;
    const void *w;              // weights (compute precision)
    const void *tw;             // W_P^k, k < P, compute precision complex
    int64_t total_items;
    // 2D adjoint only: when set, each tile's correlation flip(phi) * x over its
    // input box is stored unweighted (incremental estimator), not added to y
    const StoreDesc *store;
    void *store_base;
    // limit of each device-side wait of the apply, ns (0: 2 s); once one wait
    // gives up, the others of the launch give up at once
    int64_t wait_ns;
};

// One request on one operator inside a launch.
struct Segment {
    ApplyParams p;          // operator data, the request's x/y/nrhs, its ordering flags; p.total_items = its items
    int64_t item_begin;     // first launch-wide item index of the segment
    const uint32_t *ready;  // nullptr, or a word that equals ready_val once the segment's x is in place
    uint32_t ready_val;
    int32_t slot;           // completion slot in the host flag array, or -1
};

constexpr int kMaxSegments = 64;

// Device-resident descriptor of a launch that serves several requests.
// Items are claimed segment by segment, unless nrun > 0: then the launch's
// item order is the run table, runs of one (segment, colour) each in
// colour-major order across the segments (run i covers items
// [run_begin[i], run_begin[i + 1]) of segment run_segcol[2 i], colour
// run_segcol[2 i + 1], tile-major within the run as decode_item orders a
// colour), so that independent segments share every colour step.
struct LaunchDesc {
    int32_t nseg;
    int32_t nrun;
    int64_t total_items;
    const int64_t *run_begin;       // [nrun + 1]
    const int32_t *run_segcol;      // [nrun][2]
    Segment seg[kMaxSegments];
};

struct LaunchParams {
    const LaunchDesc *desc;         // nullptr: the single inline segment `one`
    Segment one;
    unsigned long long *counter;    // claim counter, zero at launch
    int32_t *status;                // [0] timeout flag
    uint32_t *seg_done;             // per-segment finished-item counters (descriptor launches)
    uint32_t *host_flags;           // mapped host memory: host_flags[slot] = 1 once a segment is complete
};

// Device data of the O(1) matrix entries (pc_entries.cu): box (2D: n[2] = 1),
// per pixel one leaf cell containing it, per cell its sample points (CSR),
// per patch bbox(U_k) origin/extents and weight offset, phi_k^E in FP64.
struct EntryData {
    int32_t d, R;
    int32_t n[3];
    const int32_t *cell_of;       // [N]
    const int32_t *cpts_start;    // [ncells + 1]
    const int32_t *cpts;          // sample points of each cell
    const int32_t *bb_lo;         // [r][3]
    const int32_t *bb_ext;        // [r][3] (axes beyond d: 1)
    const int64_t *w_off;         // [r]
    const double *phiE;           // [r][(2R+1)^d]
};

}  // namespace pc

struct pc_context {
    int device = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
    std::string last_error;
};

struct pc_operator {
    pc_context *ctx = nullptr;
    int d = 0;
    pc::I3 shape{1, 1, 1};
    int64_t N = 0;
    int R = 0, P = 0, T = 0, r = 0;
    pc::WindowSplit split;
    pc_precision prec = PC_FP32;
    int n_tiles = 0, n_colors = 0;
    size_t elem = 4;             // bytes of one real value
    // device memory
    void *d_spec = nullptr;
    size_t spec_bytes = 0;
    int64_t spec_stride = 0;
    void *d_w = nullptr;
    size_t w_bytes = 0;
    pc::Tile *d_tiles = nullptr;
    int32_t *d_color_start = nullptr;
    int32_t *d_dep_start = nullptr;
    int32_t *d_dep = nullptr;
    uint32_t *d_done = nullptr;
    int32_t done_cap = 0;
    int32_t *d_ctrl = nullptr;
    void *d_tw = nullptr;
    void *d_scratch = nullptr;   // 3D: per-CTA spectrum volumes (FP32) or per-item volumes of a chunk (BF16x3)
    int64_t scratch_items = 0;   // BF16x3 3D: items d_scratch holds
    void *d_tc_ops = nullptr;    // BF16x3 3D: DFT operand tiles for the tensor cores
    void *d_tc_ops_adj = nullptr;   // BF16x3 3D: the adjoint's (GEMM 1 over all 2 P columns)
    int tc_k1cap = 0;            // BF16x3 3D: K columns of the GEMM-1 operands
    // BF16x3 3D: per batch shape (pairs), the per-chunk item order of the tensor stage
    std::unordered_map<int32_t, int32_t *> tc_orders;
    // error estimator (Section 2.6): leaf cells [n][6] on the canonical box
    // (2D grids as (1, n0, n1)), per-cell sums, adjoint scratch
    int32_t *d_cells = nullptr;
    int32_t n_cells = 0;
    double *d_cell_sums = nullptr;
    void *d_est = nullptr;
    int64_t est_cap = 0;             // right-hand sides d_est holds
    // O(1) matrix entries (Section 3.1): device tables, one allocation
    void *d_entry_mem = nullptr;
    pc::EntryData entry{};
    // host-buffer applies: device staging (the whole batch's x and y for a
    // segmented launch, two chunk slots for the chunked pipeline), two copy
    // streams and the pipeline's events
    void *d_host_stage = nullptr;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t host_ev[7] = {};         // [0, 1] copied in, [2, 3] computed, [4, 5] copied out, [6] call start
    size_t host_stage_bytes = 0;
    // 2D host applies as one segmented launch: descriptor (pinned host and
    // device copies), per-segment finished-item counters, and in mapped host
    // memory per-segment ready words (host-written) and completion flags
    // (kernel-written); one event per segment's copy in
    pc::LaunchDesc *h_host_desc = nullptr, *d_host_desc = nullptr;
    uint32_t *d_host_seg_done = nullptr;
    uint32_t *h_host_ready = nullptr, *d_host_ready = nullptr;
    uint32_t *h_host_flags = nullptr, *d_host_flags = nullptr;
    std::vector<cudaEvent_t> host_in_ev;
    std::vector<cudaEvent_t> stage_ev;   // BF16x3 3D: [chunk][stage][begin, end] of the last apply
    int stage_chunks = 0;
    uint32_t epoch = 0;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;   // around the fused kernel of the last apply
    bool timed = false;
    int64_t wait_ns = 0;         // limit of each device-side wait of an apply (0: the kernels' default, 2 s)
    int ctas = 0, ctas_per_sm = 0;
    bool autotuned = false;      // launch shape chosen by timing candidates (pc_build_spectra, tune NULL)
    int tuned_candidates = 0;
    double tuned_ms = 0;
    int64_t launches_last = 0;
    size_t device_bytes = 0;
    double build_seconds = 0;
    // host copies of the schedule (plain path, block plans)
    std::vector<int32_t> color_start_h;
    std::vector<pc::Tile> tiles_h;
    std::vector<int32_t> dep_start_h, dep_h;
    // per sample point: coordinates, bbox(U_k) origin and extents (axes beyond d: 0 and 1),
    // and a 64-bit FNV-1a hash of phi_k^E's FP64 bytes (incremental estimator)
    std::vector<int32_t> pts_h, bb_lo_h, bb_ext_h;
    std::vector<uint64_t> phiE_hash;
    // plain-path scratch (lazily allocated)
    void *plain = nullptr;
    // launch shapes per patch group (2D, pc_tuning.per_patch): empty for an
    // operator with one shape, which its own fields describe
    std::vector<pc::Part> parts;
    void *d_big_scratch = nullptr;   // per-CTA 256^2 scratch fields of a part with P = 256
};

// Incremental randomized estimator (Algorithm 1): the probes Z and Y = A* Z
// (caller-owned, device), Y~ scratch, and per sample point (keyed by its
// coordinates) the unweighted correlations flip(phi_k^E) * Z on bbox(U_k),
// kept in an arena as [nsub^2][q][e0][e1] blocks between operators.
struct pc_estimator {
    struct Entry {
        int32_t bb_lo[2], bb_ext[2];
        uint64_t hash;           // of phi_k^E
        int32_t P, T, nsub;      // the tiling that produced the block
        int64_t off, len;        // elements in the arena
    };
    pc_context *ctx = nullptr;
    pc_precision prec = PC_FP32;
    size_t elem = 4;
    int64_t shape[2] = {0, 0};
    int64_t N = 0;
    int32_t q = 0;
    const void *z = nullptr, *y = nullptr;
    int64_t ldz = 0, ldy = 0;
    void *d_yt = nullptr;        // [q][N]
    void *arena = nullptr;
    std::map<std::pair<int32_t, int32_t>, Entry> cache;
    int64_t recomputed_total = 0;
};

// Block apply (Section 3.3): for each block of the plan, the operator's tiles
// that contribute to A~[T, S] (or (A~*)[T, S]), clipped and re-expressed in
// block coordinates; all blocks' tables concatenated, each block with its own
// ordering flags; one multi-segment launch runs up to kMaxSegments blocks.
struct pc_block_plan {
    struct Block {
        int64_t t_ext[3], s_ext[3];   // axes beyond d: 1
        int64_t nT, nS;
        int32_t tile_off, n_tiles, cs_off, n_colors, ds_off, dep_off, terms;
    };
    pc_operator *op = nullptr;
    bool adjoint = false;
    std::vector<Block> blocks;
    int n_tiles = 0, terms = 0;       // totals over the blocks
    pc::Tile *d_tiles = nullptr;
    int32_t *d_color_start = nullptr;
    int32_t *d_dep_start = nullptr;
    int32_t *d_dep = nullptr;
    uint32_t *d_done = nullptr;       // block b's flags at tile_off * done_cap
    int32_t done_cap = 0;
    int32_t *d_ctrl = nullptr;
    uint32_t epoch = 0;
    std::vector<int32_t> cs_h;        // host copy of the colour offsets
    // multi-block launches: per round of kMaxSegments blocks, a descriptor and
    // a run table (pinned host staging, then device); run_cap runs per round
    std::vector<pc::LaunchDesc *> h_desc;
    pc::LaunchDesc *d_desc = nullptr;
    std::vector<char *> h_runs;
    char *d_runs = nullptr;
    int32_t run_cap = 0;
    uint32_t *d_seg_done = nullptr;
    cudaEvent_t desc_ev = nullptr;    // after the last descriptor upload
    cudaStream_t last_stream = nullptr;
    bool launched = false;
};

namespace pc {
// kernels (pc_fft2d.cu, pc_spectra.cu, pc_plain.cu)
cudaError_t launch_zero(const ApplyParams &p, int64_t N, pc_precision prec, cudaStream_t s);
// adjoint = false: y = A~ x; true: y = A~* x (Eq. adjoint_random_z)
cudaError_t launch_fft2d(const ApplyParams &p, int P, pc_precision prec, int ctas, cudaStream_t s,
                         bool adjoint = false);
// multi-request launch (FP32, P = 128): y zero-fill + claim reset, then the fused kernel
// (fft2d_configure(128, PC_FP32, ...) must have been called; capturable)
// Multi-segment persistent launch of the 2D patch kernel (every segment's y
// zeroed and its flags cleared first): P = 128 FP32 for served requests;
// any 2D configuration (P, precision, direction) for chunked host applies.
cudaError_t launch_round(const LaunchDesc *d_desc, unsigned long long *counter, int32_t *status, uint32_t *seg_done,
                         uint32_t *host_flags, int ctas, size_t smem, cudaStream_t s, int P = 128,
                         pc_precision prec = PC_FP32, bool adjoint = false);
cudaError_t fft2d_configure(int P, pc_precision prec, int *ctas_per_sm, size_t *smem);
// 256 x 256 patch FFTs (pc_fft2d_big.cu), FP32, single launches: the three
// phases around a per-CTA scratch field of fft2d_big_scratch_bytes(1) bytes
cudaError_t fft2d_big_configure(int *ctas_per_sm);
size_t fft2d_big_scratch_bytes(int ctas);
cudaError_t launch_fft2d_big(const ApplyParams &p, int ctas, void *scratch, cudaStream_t s, bool adjoint);
constexpr int kBigFft = 256;
// d_psi: [nspec][W][W] FP64 windows placed at [0, W)^2; spectra [nspec][P/2+1][P]
cudaError_t build_spectra_2d(const double *d_psi, int nspec, int W, int P, pc_precision prec, void *d_spec,
                             const double2 *d_tw64, cudaStream_t s);
// 3D patch path (pc_fft3d.cu), FP32, P = 64.  The fused kernel runs clusters
// of CTAs, one scratch volume each: launch_fft3d takes the operator's whole
// CTA budget (not clamped to the item count) and a scratch of
// fft3d_scratch_bytes(that budget).
cudaError_t fft3d_configure(int *ctas_per_sm);
cudaError_t launch_fft3d(const ApplyParams &p, int ctas, void *scratch, cudaStream_t s, bool adjoint = false);
size_t fft3d_scratch_bytes(int ctas);
size_t fft3d_volume_bytes();   // one 64^3 complex FP32 volume
cudaError_t build_spectra_3d(const double *d_psi, int nspec, int W, int P, void *d_spec, const double2 *d_tw64,
                             cudaStream_t s);
// split 3D path: phase 1 and phase 3 over items [c0, c1), scratch volume of
// item i at scratch + (i - c0) * fft3d_volume_bytes().  Phase 3 keeps
// kPhase3Groups ordering flags per (tile, pair): done_ld >= npairs * groups.
constexpr int kPhase3Groups = 8;
// The fused 3D kernel runs clusters of CTAs (kCluster3dFwd for Ã, kCluster3dAdj
// for Ã*), each CTA adding one contiguous group of an item's output planes
// under its own ordering flag.
constexpr int kCluster3dFwd = 2;
constexpr int kCluster3dAdj = 1;
constexpr int kCluster3dMax = kCluster3dFwd > kCluster3dAdj ? kCluster3dFwd : kCluster3dAdj;
constexpr int kCluster3dMin = kCluster3dFwd < kCluster3dAdj ? kCluster3dFwd : kCluster3dAdj;
// ordering flags per (tile, pair) of an apply (either direction)
inline int flag_groups(int d, pc_precision prec) {
    return d == 3 ? (prec == PC_BF16X3 ? kPhase3Groups : kCluster3dMax) : 1;
}
cudaError_t launch_fft3d_phase1(const ApplyParams &p, int ctas, void *scratch, int64_t c0, int64_t c1,
                                cudaStream_t s, bool adjoint = false);
cudaError_t launch_fft3d_phase3(const ApplyParams &p, int ctas, const void *scratch, int64_t c0, int64_t c1,
                                cudaStream_t s, bool adjoint = false);
// tensor-core first-axis transform (pc_tc3d.cu), one CTA per SM.  Tiles of
// a BF16x3 operator are at most kTc3dMaxTile wide along the first axis, so
// GEMM 1 needs K <= kTc3dMaxK1 = 2 kTc3dMaxTile.
constexpr int64_t kTc3dChunkItems = 4096;
constexpr int kTc3dMaxTile = 48;
constexpr int kTc3dMaxK1 = 2 * kTc3dMaxTile;
int tc3d_k1cap(int tile);   // GEMM-1 K columns for tiles of extent <= tile
cudaError_t tc3d_build_operands(int k1cap, void **d_ops);
cudaError_t tc3d_configure();
// order: the items of every chunk [c0, c1) in tile-then-pair order (absolute
// item indices, entries c0 ... c1 - 1), then, at total_items + i, the tile
// of item order[i]
cudaError_t launch_tc3d_axis0(const ApplyParams &p, int ctas, void *scratch, const int32_t *order, int64_t c0,
                              int64_t c1, const void *ops, int k1cap, cudaStream_t s);
// the adjoint's tensor stage: ops_full = tc3d_build_operands(2 P) (GEMM 1
// over all first-axis planes)
cudaError_t launch_tc3d_axis0_adjoint(const ApplyParams &p, int ctas, void *scratch, const int32_t *order, int64_t c0,
                                      int64_t c1, const void *ops_full, cudaStream_t s);
pc_status plain_apply(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                      cudaStream_t s, std::string &err);
void plain_free(pc_operator *op);
// matrix entries (pc_entries.cu): out[i] = A~[rows[i], cols[i]] (flat indices), FP64
cudaError_t launch_entries(pc_precision prec, int64_t n, const int64_t *rows, const int64_t *cols, double *out,
                           const EntryData &e, const void *w, cudaStream_t s);
// grow the on-demand device buffers of an apply of nrhs vectors (pc_api.cpp)
pc_status prepare_batch(pc_operator *op, int32_t nrhs);
// The apply parameters of one part of a per_patch operator: `p` with the
// part's tiles, colour classes, dependency lists, ordering flags, spectra,
// twiddles and item count (pc_api.cpp).
ApplyParams part_params(const pc_operator *op, const Part &pt, const ApplyParams &p);
// Per-patch launch shape (pc_autotune.cpp): for each sample point k the FFT
// size and kernel-window split that the line-FFT work model prefers for
// bbox(U_k) (2D; P in {128, 256} for FP32, 64 for FP64); shape[k] = {P, nsub}.
// Tile extent of a window split ws at FFT size P: min(P - ws + 1, cap), cap
// = 2P/3 for the fused kernel's row staging, P for the 256^2 kernel.
inline int tile_cap(int P) { return P == kBigFft ? P : (2 * P) / 3; }
void choose_patch_shapes(const Geometry &g, int R, pc_precision prec, std::vector<std::array<int, 2>> &shape);
// autotuner (pc_autotune.cpp): pc_build_spectra with a NULL pc_tuning
pc_status autotune_build(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius,
                         const double *impulse, const double *weights, pc_precision prec, pc_operator **out);
// error estimator (pc_estimate.cu): out[c] = sum over cell c and q columns of (yt - y)^2, FP64
// incremental estimator (pc_incremental.cu): copy kept correlation blocks
// (copies[i] = {src, dst, len} in elements) and form
// yt[b][x] = sum_{k in points of cell_of[x]} w_k[x] * sum_s c_{k,s}[b][x - lo_k]
cudaError_t launch_block_copies(pc_precision prec, const int64_t *copies, int32_t n, const void *src, void *dst,
                                cudaStream_t s);
cudaError_t launch_corr_combine(pc_precision prec, const EntryData &e, const void *w, const void *c,
                                const int64_t *blk_off, int32_t nsub2, int32_t q, void *yt, int64_t N, cudaStream_t s);
cudaError_t launch_cell_sqdiff(pc_precision prec, const void *yt, int64_t ldyt, const void *y, int64_t ldy, int32_t q,
                               const int32_t *cells, int32_t ncells, int64_t n1, int64_t n2, double *out,
                               cudaStream_t s);
}  // namespace pc
