/*
 * pc.h - C ABI of the GB300 product-convolution library (libpc.so).
 *
 * The library applies the adaptive product-convolution approximation of
 * Alger, Rao, Myers, Bui-Thanh, Ghattas (arXiv 1805.06018):
 *
 *     y = A~ x = sum_{k=1}^{r} phi_k^E * (w_k . x)          (Section 2.1, Eq. conv_op_approx_main)
 *
 * on a box Omega = prod_i [0, shape_i - 1] in Z^d (d = 2 or 3), where
 *   - the sample points p_k are the corners of the leaf cells of a given grid
 *     (Section 2.2),
 *   - w_k are the harmonic partition-of-unity weights on the blocky
 *     neighbourhoods U_k (Section 2.4),
 *   - phi_k^E are the caller's impulse responses phi_k[z] = (A delta_{p_k})[z + p_k]
 *     (Eq. varphi_p_section2) extended with the neighbour average of Section 2.5
 *     (Eqs. vj_def, def_varphiE),
 *   - '*' is convolution with extension by zero (Eq. convolution_definition),
 *     evaluated with FFTs after zero padding (Section 3.2), patch by patch
 *     (the block translation of Section 3.3), output restricted to Omega.
 *
 * Conventions shared by every entry point:
 *   - Errors are returned as pc_status, never thrown and never abort().  The
 *     text of the last error of a context is available from pc_last_error().
 *   - Arrays are C order (last axis fastest).  A batch of vectors is
 *     [nrhs][n_1]...[n_d] with a stride (ld) between consecutive vectors.
 *   - "device" pointers are CUDA device memory of the context's device (the
 *     caller allocates them, e.g. with PyTorch); "host" pointers are ordinary
 *     host memory.  The library never frees caller memory.
 *   - Applies are asynchronous and stream ordered: they enqueue kernels on the
 *     caller's stream and return.  y is overwritten, not accumulated.  x and y
 *     must stay valid until the work on that stream has completed.  x and y
 *     must not overlap.  Applies of one operator must not run concurrently
 *     on the device (they share the operator's ordering flags); successive
 *     applies on one stream are fine.
 *   - pc_stream is a cudaStream_t passed as an opaque pointer (NULL = the
 *     legacy default stream).
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* libpc is built with hidden symbol visibility; these declarations are the
 * library's only exported symbols. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef enum {
    PC_OK = 0,
    PC_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, misaligned ld) */
    PC_ERR_GRID = 2,         /* leaf cells do not tile the box */
    PC_ERR_NOMEM = 3,        /* a host or device allocation failed */
    PC_ERR_BUDGET = 4,       /* a request does not fit the configured memory budget */
    PC_ERR_CUDA = 5,         /* a CUDA runtime call failed (message in pc_last_error) */
    PC_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    PC_ERR_NOT_READY = 7,    /* an asynchronous request has not finished */
    PC_ERR_UNSUPPORTED = 8   /* valid input outside what this build implements */
} pc_status;

typedef enum {
    PC_FP64 = 0,             /* FP64 data, FP64 FFTs (correctness configuration) */
    PC_FP32 = 1,             /* FP32 data, FP32 FFTs, spectra built in FP64 and rounded once */
    PC_BF16X3 = 2,           /* 3D operators: FP32 data and plane FFTs; the first-axis DFTs are
                                tensor-core GEMMs with split BF16 operands, a = a_hi + a_lo,
                                products a_lo b_hi + a_hi b_lo + a_hi b_hi accumulated in FP32 */
    PC_TF32X3 = 3            /* reserved (not built): split TF32 operands */
} pc_precision;

typedef void *pc_stream;     /* cudaStream_t */

/* Omega = prod_{i<ndim} [0, shape[i]-1]; ndim is 2 or 3, shape[i] >= 2. */
typedef struct {
    int32_t ndim;
    int64_t shape[3];
} pc_box;

/* Leaf cells of the binary tree of Section 2.2: num_cells closed integer
 * boxes, cells[(c*2 + 0)*ndim + i] = min point, cells[(c*2 + 1)*ndim + i] =
 * max point (host memory).  They must tile Omega, sharing facets: every
 * point of Omega lies in some cell, interiors are disjoint, and every cell has
 * max > min on each axis. */
typedef struct {
    int32_t num_cells;
    const int32_t *cells;
} pc_grid;

/* Launch-shape knobs of an operator.  pc_build_spectra with a NULL
 * pc_tuning autotunes them (times candidate shapes on the device and keeps
 * the fastest); in a non-NULL pc_tuning a field of 0 means "the library's
 * model choice" (no timing). */
typedef struct {
    int32_t fft_size;        /* padded FFT extent P per axis: 64, 128 (2D); 64 (3D) */
    int32_t tile;            /* input tile extent T <= min(P - W + 1, 2P/3), W the kernel
                                (sub-)window extent (2R+1 unless split) (0: that bound) */
    int32_t ctas_per_sm;     /* persistent CTAs per SM (0: occupancy limit) */
    int32_t wait_limit_us;   /* limit of every device-side wait of an apply (ordering flags,
                                copy completion, host-written ready words), microseconds
                                (0: 2 s).  A wait that runs out ends the launch early: every
                                other wait of the launch then gives up at once, the result is
                                invalid, and the apply's status query reports PC_ERR_TIMEOUT */
    int32_t window_split;    /* kernel sub-windows per axis: [-R, R] cut into window_split
                                pieces with their own spectra, an exact rewrite of the sum
                                (0: the count that minimises FFT work per input pixel) */
    int32_t per_patch;       /* 2D: 1 = each patch takes the FFT size (FP32: 128 or 256) and
                                window split that a model of the line-FFT work prefers for
                                its own bbox(U_k); the patches of each shape form a part,
                                applied by its own launch (fft_size, tile and window_split
                                are then ignored).  Such operators support the applies, the
                                host-buffer apply, serving (own apply on a slot), the estimator
                                and the entries; block plans, the incremental estimator
                                and the plain path refuse them (PC_ERR_UNSUPPORTED) */
    int32_t reserved[2];
} pc_tuning;

/* Read-only description of a built operator. */
typedef struct {
    int32_t ndim;
    int64_t shape[3];
    int32_t radius;          /* R: phi_k^E lives on [-R, R]^d */
    int32_t r;               /* number of sample points = number of convolutions */
    int32_t fft_size;        /* P */
    int32_t tile;            /* T */
    int32_t num_tiles;       /* work units per right-hand side pair */
    int32_t num_colors;      /* overlap-add order classes */
    int32_t precision;       /* pc_precision */
    int64_t spectra_bytes;   /* device bytes of the stored spectra */
    int64_t device_bytes;    /* all device bytes owned by the operator, including the
                                buffers its applies have grown so far */
    double build_seconds;    /* including the autotuner's candidates when it ran */
    int32_t window_split;    /* kernel sub-windows per axis */
    int32_t ctas_per_sm;     /* persistent CTAs per SM of the apply */
    int32_t autotuned;       /* 1 if the launch shape came from the autotuner */
    int32_t tuned_candidates;   /* candidate shapes the autotuner timed */
    double tuned_ms;         /* its time of the chosen shape per timed batch (ms) */
    int32_t num_parts;       /* launch shapes (parts) of a per_patch operator; 1 otherwise */
    int32_t reserved;
} pc_operator_info;

typedef struct pc_context pc_context;
typedef struct pc_operator pc_operator;
typedef struct pc_server pc_server;

/* Serving configuration (pc_serve_create). */
typedef struct {
    int64_t hbm_budget_bytes;   /* device bytes the server may hold for resident operators
                                   (counted while they have work in flight) plus request scratch */
    int32_t max_inflight;       /* requests admitted but not finished, <= 1024 */
    int32_t streams;            /* concurrent launch slots (1..4); launches on different slots overlap */
    int32_t max_requests_per_launch;   /* <= 64 */
    int32_t reserved[3];
} pc_serve_config;

/* Completion record of a served request (pc_serve_poll). Times are seconds
 * on the server's steady clock. */
typedef struct {
    double submit_s, launch_s, finish_s;
    int32_t nrhs;
    int32_t launch_requests;    /* requests that shared its launch */
    int32_t status;             /* pc_status of the request */
    int32_t reserved;
} pc_request_info;

/* Aggregate serving statistics since pc_serve_create. */
typedef struct {
    int64_t completed, rhs_completed, launches;
    double p50_latency_s, p99_latency_s, mean_latency_s;
    double busy_s;              /* first submit to last completion */
    double rhs_per_s;
    int64_t peak_bytes;         /* peak budgeted bytes */
} pc_serve_stats;

/* Create a library context bound to CUDA device `device`.  *ctx receives a
 * handle that the caller releases with pc_context_destroy.  Fails with
 * PC_ERR_CUDA if the device cannot be used and PC_ERR_UNSUPPORTED if it is
 * not compute capability 10.3. */
pc_status pc_context_create(int32_t device, pc_context **ctx);
pc_status pc_context_destroy(pc_context *ctx);

/* Text of the last error recorded in ctx (never NULL; "" when none).  With a
 * NULL ctx it returns the last error of a failed pc_context_create or of a
 * context-free call such as pc_sample_points.  Valid until the next call on
 * the same context. */
const char *pc_last_error(pc_context *ctx);

/* Sample points {p_k} = union of the corners of the leaf cells (Section 2.2),
 * in lexicographic order of their coordinates; that order defines k in every
 * other call.  *r receives their number; if points is not NULL it must hold
 * r*ndim int32 values (host) and receives them as [r][ndim].  Validates the
 * grid (PC_ERR_GRID). */
pc_status pc_sample_points(const pc_box *box, const pc_grid *grid, int32_t *r, int32_t *points);

/* Bounding boxes of the blocky neighbourhoods U_k (Section 2.2): lo and hi
 * receive [r][ndim] int32 (host); either may be NULL.  This is the layout of
 * caller-supplied weights in pc_build_spectra. */
pc_status pc_neighbourhood_boxes(const pc_box *box, const pc_grid *grid, int32_t *lo, int32_t *hi);

/* The harmonic partition-of-unity weights of Section 2.4 as the library
 * builds them (host computation, FP64, no GPU needed): on a leaf whose only
 * sample points are its corners the recursive Laplace construction gives the
 * multilinear hat; 2D leaves with hanging nodes solve the discrete Laplace
 * equation with piecewise-linear edge data; 3D leaves with hanging nodes
 * first solve it on each piece of their facets (a facet broken by finer
 * leaves across it is replaced by its intersections with their facets),
 * then in the interior.  *count receives the number of
 * values (sum over k of |bbox(U_k)|); if weights is not NULL it must hold
 * that many doubles and receives w_k on bbox(U_k), C order, k ascending
 * (zero outside U_k).  A 3D grid in which some facet piece has a corner that
 * is no sample point (the two sides of a facet split along different axes)
 * has no weights under Section 2.4's recursion: PC_ERR_GRID, as from
 * pc_build_spectra. */
pc_status pc_harmonic_weights(const pc_box *box, const pc_grid *grid, int64_t *count, double *weights);

/* The extended impulse responses phi_k^E of Section 2.5 (Eqs. vj_def,
 * def_varphiE) as the library builds them (host, FP64, no GPU needed):
 * impulse and impulse_ext are [r][(2R+1)^ndim] (layout of pc_build_spectra's
 * impulse argument).  Where p_k + z is outside Omega, phi_k^E[z] is the plain
 * average of the neighbours phi_j[z] (j in nbrs(k)) whose domain Omega - p_j
 * contains z, and 0 if there is none. */
pc_status pc_extend_impulse(const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                            double *impulse_ext);

/* Build an operator: weights, extended impulse responses and their padded
 * spectra (a one-time construction; spectra are computed in FP64 on the
 * device and stored in `prec`).
 *   radius   R >= 1: the operator is truncated so that phi_k vanishes
 *            outside [-R, R]^d (2R+1 <= fft_size - 1).
 *   impulse  host FP64 [r][(2R+1)^ndim]: phi_k[z] at window index z + R (C
 *            order over the window), k in sample-point order.  Values at
 *            z with p_k + z outside Omega are ignored (phi_k is only defined
 *            on Omega - p_k; Section 2.5 fills that region from neighbours).
 *   weights  NULL: the library builds the harmonic weights of Section 2.4
 *            (closed-form multilinear hats on cells without hanging nodes,
 *            discrete Laplace solves on cells with hanging nodes, 2D and 3D,
 *            as pc_harmonic_weights describes).
 *            Otherwise host FP64, w_k on bbox(U_k) (pc_neighbourhood_boxes),
 *            C order, concatenated for k = 0..r-1; entries outside U_k must
 *            be 0.
 *   prec     PC_FP64 (2D), PC_FP32, or PC_BF16X3 (3D only; the first-axis
 *            transform of each patch runs as split-BF16 tensor-core GEMMs,
 *            relative error of the result about 1e-5 against FP64).
 *   tune     NULL or knobs (see pc_tuning).
 * The operator owns its device memory until pc_operator_destroy.  The call
 * synchronises the device. */
pc_status pc_build_spectra(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius,
                           const double *impulse, const double *weights, pc_precision prec,
                           const pc_tuning *tune, pc_operator **op);

pc_status pc_operator_info_get(const pc_operator *op, pc_operator_info *info);

/* y = A~ x for one vector: x and y are device arrays of N = prod(shape)
 * elements of the operator's precision (float or double). */
pc_status pc_apply(pc_operator *op, const void *x, void *y, pc_stream stream);

/* Y[b] = A~ X[b] for b < nrhs: X[b] starts at x + b*ldx elements, Y[b] at
 * y + b*ldy elements (device), ldx, ldy >= N.  nrhs = 0 is a no-op. */
pc_status pc_apply_batched(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx,
                           void *y, int64_t ldy, pc_stream stream);

/* Adjoint apply: Y[b] = A~* X[b] for b < nrhs, where
 *   A~* x = sum_k w_k . (flip(phi_k^E) * x)          (Eq. adjoint_random_z;
 * real data, so the conjugates drop): the correlation of x with each
 * extended impulse response, weighted by w_k, summed over k.  This is the
 * operator the paper's a-posteriori error estimator applies to random
 * probes (Section 2.6).  Same arguments, layouts, stream semantics and
 * determinism as pc_apply_batched (y overwritten; each y element sums its
 * contributions in a fixed order).  PC_FP32 and PC_FP64 operators, 2D and
 * 3D, and PC_BF16X3 operators (the first-axis correlation as split-BF16
 * tensor-core GEMMs over all 2 P columns of the DFT, the conjugate spectrum
 * between them). */
pc_status pc_apply_adjoint_batched(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx,
                                   void *y, int64_t ldy, pc_stream stream);

/* Y[b] = A~ X[b] (adjoint = 0) or A~* X[b] (adjoint = 1) for b < nrhs with
 * x and y in HOST memory (X[b] at x + b*ldx, Y[b] at y + b*ldy elements,
 * ldx, ldy >= N, disjoint).  The batch moves in chunks of `chunk`
 * right-hand sides, rounded up to an even count so that the right-hand-side
 * pairs, and so every rounding, are those of one device apply of the whole
 * batch: the result is bitwise that of pc_apply_batched /
 * pc_apply_adjoint_batched.
 *   - 2D operators (chunk 0: about a quarter of the batch, at most 64
 *     chunks): the whole batch is staged on the device (2 * nrhs * N
 *     elements, kept by the operator) and computed by ONE persistent launch
 *     of the patch kernel.  Chunk i is copied in on an internal copy stream;
 *     when the calling thread sees that copy complete it sets the chunk's
 *     ready word in mapped host memory, which the kernel's CTAs wait for
 *     (bounded) before they take the chunk's work.  The kernel raises a
 *     completion flag in mapped host memory once the chunk's last result has
 *     landed, and the calling thread then copies the chunk out on a second
 *     copy stream.  The call therefore BLOCKS until the kernel has
 *     finished (at most 60 s after the work queued earlier on `stream`,
 *     else PC_ERR_TIMEOUT); the copies out of the last chunks may still be
 *     in flight when it returns.  Where launches block the calling thread
 *     (CUDA_LAUNCH_BLOCKING non-zero), and where the environment sets
 *     PC_HOST_PIPELINE=chunked (for tools that serialise launches, such as
 *     profilers), 2D operators take the chunked pipeline below instead,
 *     with the same chunks and the same bitwise result.
 *   - 3D operators (chunk 0: the whole batch, as their patch kernels gain
 *     little from smaller batches): chunk i is copied in, applied on
 *     `stream` and copied out
 *     through two device staging slots (4 * chunk * N elements), so that the
 *     copies of one chunk overlap the kernels of its neighbours; the call
 *     returns once everything is queued.
 * Stream-ordered: the copies start after the work already queued on
 * `stream`, and work queued on `stream` after the call starts once y is
 * complete.  x and y must stay valid until then and should be page-locked
 * (cudaHostAlloc or cudaHostRegister) for the copies to run asynchronously.
 * Calls on one operator must be serialised (one stream).  adjoint: 0 (A~)
 * or 1 (A~*), for every operator. */
pc_status pc_apply_host(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                        int32_t adjoint, int32_t chunk, pc_stream stream);

/* Matrix entries in O(1) each (Section 3.1, Eq. conv_matrix_entries):
 *   out[i] = A~[rows[i], cols[i]] = sum_{k : x in U_k} w_k[x] phi_k^E[y - x],
 * y = rows[i], x = cols[i] flat C-order indices into Omega.  Only the sample
 * points of a leaf cell containing x carry weight at x, so each entry visits
 * a handful of terms.  rows, cols: device int64 [n]; out: device double [n];
 * stream-ordered.  phi_k^E is kept in FP64, w_k in the operator's precision.
 * An index outside [0, N) yields NaN for that entry (no memory access).
 * These are the entries an H-matrix or CUR builder asks for (Section 3.4). */
pc_status pc_entries(pc_operator *op, int64_t n, const int64_t *rows, const int64_t *cols, double *out,
                     pc_stream stream);

/* ---------------------------------------------------------------------
 * Incremental estimator for the adaptive construction (Algorithm 1,
 * Section 2.8).  Y~ = A~* Z = sum_k w_k . c_k with the unweighted
 * correlations c_k = flip(phi_k^E) * Z on bbox(U_k) (Eq. adjoint_random_z).
 * c_k depends only on phi_k^E and bbox(U_k), so between the operators of
 * successive refinement passes it is recomputed only for sample points that
 * are new or whose extension changed (a new neighbour); the rest are kept.
 * --------------------------------------------------------------------- */
typedef struct pc_estimator pc_estimator;

/* q probes Z and Y = A* Z (device, [q][N] with strides ldz, ldy >= N, in
 * `prec`, PC_FP32 or PC_FP64) on the 2D box `box`; both stay owned by the
 * caller and must outlive the estimator.  Allocates Y~ scratch (q * N). */
pc_status pc_estimator_create(pc_context *ctx, const pc_box *box, pc_precision prec, int32_t q, const void *z,
                              int64_t ldz, const void *y, int64_t ldy, pc_estimator **est);

/* eta[C] = (1/sqrt(q)) ||Y~[C, .] - Y[C, .]|| for every leaf cell C of op
 * (Eq. randomized_estimator_ec), as pc_estimate_cell_errors, with Y~ formed
 * from the kept and the recomputed correlations: a sample point's block is
 * kept when its coordinates, bbox(U_k), patch tiling and phi_k^E (compared
 * by a 64-bit hash of its FP64 values) are unchanged.  *recomputed (if not
 * NULL) receives the number of points recomputed.  op must be a 2D operator
 * on the estimator's box in its precision; it is read only during the call.
 * Each output sums its terms in a fixed order (bitwise reproducible); the
 * result agrees with pc_estimate_cell_errors up to rounding (the two sum
 * the terms in different orders).  Synchronises `stream`. */
pc_status pc_estimator_update(pc_estimator *est, pc_operator *op, double *eta, int32_t *recomputed,
                              pc_stream stream);

pc_status pc_estimator_destroy(pc_estimator *est);

/* ---------------------------------------------------------------------
 * Refinement of the adaptive construction (Algorithm 1, Section 2.7), host
 * code on the leaf cells of pc_grid.  With pc_build_spectra and
 * pc_estimate_cell_errors (or pc_estimator_update) a C caller runs the whole
 * construction: build, estimate, pc_refine, repeat until eta_Omega <= tau.
 * impulse: phi_k of the current sample points, as for pc_build_spectra.
 * --------------------------------------------------------------------- */

/* One pass of Algorithm 1's refinement.  eta_Omega = sqrt(sum_C eta_C^2) /
 * y_rms (the overall estimator as a relative estimate: y_rms = ||Y||_F /
 * sqrt(q) of the caller's Y = A* Z; eta_c[C] from pc_estimate_cell_errors,
 * one per leaf in grid order).  If eta_Omega > tau, up to `batch` leaves are
 * split, largest eta_C first (ties: lower leaf index), each in its first
 * admissible direction of pc_split_directions (in 3D a direction is
 * admissible when pc_split_is_admissible says so, on the leaves as split so
 * far this pass; a leaf with none is passed over).  A split halves the leaf
 * at floor((c_min + c_max) / 2).  cells_out receives the new leaf list
 * (the unsplit leaves in their order, then each split leaf's two halves,
 * highest split leaf index first; layout as pc_grid.cells), room for
 * num_cells + batch leaves; *num_cells_out its length (num_cells when
 * eta_Omega <= tau or no leaf could be split).  batch = 1 is Algorithm 1 as
 * printed. */
pc_status pc_refine(const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                    const double *eta_c, double y_rms, double tau, int32_t batch, double *eta_omega,
                    int32_t *cells_out, int32_t *num_cells_out);

/* Subdivision directions of leaf `cell` (Section 2.7), best first: the axes
 * i with c_max^i - c_min^i > 2, ordered by || phi^{i+} - phi^{i-} ||, the
 * l2 norm over the window offsets z with c_mid + z in Omega of the
 * difference between the averages of phi_k^E (Eq. def_varphiE) over the
 * leaf's corners on its front and its back face along i; scores within a
 * relative 1e-9 of the best are a tie, won by the lowest axis.  dirs:
 * room for ndim entries; *ndirs the number written. */
pc_status pc_split_directions(const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                              int32_t cell, int32_t *dirs, int32_t *ndirs);

/* Whether halving leaf `cell` along `axis` keeps every facet piece of the
 * two halves (their facets' intersections of positive area with the facets
 * of the leaves across) with sample points at its corners, which the
 * recursive weights of Section 2.4 need; always 1 in 2D.  A 3D split that
 * breaks a facet crosswise gives 0.  PC_ERR_ARG if the leaf is thinner than
 * 2 along the axis. */
pc_status pc_split_is_admissible(const pc_box *box, const pc_grid *grid, int32_t cell, int32_t axis, int32_t *ok);

/* ---------------------------------------------------------------------
 * Block apply (Section 3.3).  For closed boxes T (targets) and S (sources)
 * inside Omega, and x_S extended by zero outside S:
 *   forward  y_T = A~[T, S] x_S
 *                = sum_{k : U_k meets S} (phi_k^E * (w_k . x_S))[T],
 *   adjoint  y_T = (A~*)[T, S] x_S
 *                = sum_{k : U_k meets T} w_k[T] . (flip(phi_k^E) * x_S)[T].
 * Each term is the paper's translated small convolution: a plan keeps the
 * operator's input tiles of bbox(U_k) that meet S (T for the adjoint) and
 * whose output box (tile (+) kernel sub-window) meets T (S), clips each to
 * S (T) and re-expresses it in the block's own coordinates.  The patch
 * spectra of the operator are reused as they are (the sub-window of
 * phi_k^E a tile convolves with does not depend on the tile's extent), so
 * a plan stores no spectra.  Work: one FFT convolution of the operator's
 * patch size per kept tile and pair of right-hand sides, i.e.
 * O(r_S P^d log P) per vector (r_T for the adjoint).  A plan fixes
 * (operator, T, S, direction); applying it repeatedly, as a Krylov or
 * randomized-SVD low-rank builder does (Section 3.4), needs no host work
 * beyond the launches.
 * --------------------------------------------------------------------- */
typedef struct pc_block_plan pc_block_plan;

/* t_lo, t_hi, s_lo, s_hi: host arrays of d int64 values (C axis order),
 * closed boxes with 0 <= lo <= hi < shape per axis, else PC_ERR_ARG.
 * adjoint: 0 (A~[T,S]) or 1 ((A~*)[T,S]).  PC_FP32 and PC_FP64 operators,
 * 2D and 3D; PC_BF16X3 operators return PC_ERR_UNSUPPORTED.  A 3D plan runs
 * on the operator's scratch volumes: its applies must not overlap
 * the operator's own applies or other 3D plans of the same operator (one
 * stream serialises them).  The plan allocates its device
 * tables (kept tiles, colour offsets, dependency lists, ordering flags,
 * control block); the call synchronises the device.  The operator must
 * outlive the plan.  *plan is NULL on failure. */
pc_status pc_block_plan_create(pc_operator *op, const int64_t *t_lo, const int64_t *t_hi, const int64_t *s_lo,
                               const int64_t *s_hi, int32_t adjoint, pc_block_plan **plan);

/* Y[b] = block X[b] for b < nrhs.  X[b] = x + b*ldx holds |S| values in C
 * order over S, Y[b] = y + b*ldy holds |T| values in C order over T (device,
 * operator precision, ldx >= |S|, ldy >= |T|, x and y disjoint).  y is
 * overwritten; every y element sums its contributions in a fixed order, so
 * the result is bitwise reproducible, and with S = T = Omega it is bitwise
 * that of pc_apply_batched (pc_apply_adjoint_batched).  Stream-ordered; the
 * first call with a larger batch grows the plan's ordering flags (and
 * synchronises the device).  Calls on one plan must be serialised (one
 * stream); different plans and the operator's own applies may overlap.
 * nrhs = 0 is a no-op.  PC_ERR_ARG for a plan of several blocks. */
pc_status pc_block_apply(pc_block_plan *plan, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                         pc_stream stream);

/* Several blocks of one operator and one direction in one plan: box bounds
 * as [nblocks][d] host arrays (block i at t_lo + i*d, ...).  Applying it runs
 * every block in one persistent launch (rounds of at most 64 blocks), each
 * block with its own tiles, colour order and ordering flags, so each block's
 * result is bitwise that of a single-block plan of that block; a low-rank
 * builder's many small blocks then fill the GPU together.  (3D plans run
 * their blocks one launch after another.) */
pc_status pc_block_plan_create_many(pc_operator *op, int32_t nblocks, const int64_t *t_lo, const int64_t *t_hi,
                                    const int64_t *s_lo, const int64_t *s_hi, int32_t adjoint, pc_block_plan **plan);

/* Y_i[b] = block_i X_i[b] for every block i of the plan and b < nrhs: x, y,
 * ldx, ldy are host arrays with one entry per block (device pointers and
 * strides as in pc_block_apply).  The blocks' y arrays must not overlap one
 * another.  Same stream semantics as pc_block_apply. */
pc_status pc_block_apply_many(pc_block_plan *plan, int32_t nrhs, const void *const *x, const int64_t *ldx,
                              void *const *y, const int64_t *ldy, pc_stream stream);

/* terms: sum over the blocks of the distinct k with a kept tile (at most
 * r_S, r_T for the adjoint, per block); tiles: kept tiles.  Either pointer
 * may be NULL. */
pc_status pc_block_plan_info(const pc_block_plan *plan, int32_t *terms, int32_t *tiles);

/* As pc_operator_check, for the plan's launches: synchronises the plan's
 * last stream; PC_ERR_TIMEOUT if a bounded wait gave up (flag cleared). */
pc_status pc_block_plan_check(pc_block_plan *plan);

pc_status pc_block_plan_destroy(pc_block_plan *plan);

/* Randomized a-posteriori error estimator (Section 2.6,
 * Eq. randomized_estimator_ec): for every leaf cell C of the operator's grid
 * (the cells passed to pc_build_spectra, in that order, as closed boxes),
 *   eta[C] = (1/sqrt(q)) || (A~* Z)[C, .] - Y[C, .] ||_F
 * where Z holds q probe vectors and Y = A* Z is supplied by the caller (the
 * paper's matrix-free access to A*).  With Z ~ N(0,1)^{N x q} this estimates
 * e_C = ||(A~ - A)[Omega, C]|| (Eq. relative_error).
 *   z, y   device, [q][N] with strides ldz, ldy >= N, operator precision.
 *   eta    host array of num_cells doubles, written before the call returns
 *          (the call synchronises `stream`).
 * The library applies A~* to z (as pc_apply_adjoint_batched, into scratch
 * that it allocates and keeps) and reduces each cell in FP64 in a fixed
 * order, so eta is bitwise reproducible.  Every operator, 2D and 3D (cells
 * as closed boxes); for PC_BF16X3 operators A~* z runs on the tensor-core
 * path. */
pc_status pc_estimate_cell_errors(pc_operator *op, int32_t q, const void *z, int64_t ldz, const void *y,
                                  int64_t ldy, double *eta, pc_stream stream);

/* Plain path for comparison: the same operator applied one vector at a time
 * through a gather kernel, a library FFT (cuFFT, 2D P x P or 3D P x P x P)
 * of each padded patch, a spectral product kernel, an inverse library FFT
 * and an output-stationary overlap-add kernel, all in FP32.  2D and 3D
 * operators with FP32 spectra (PC_FP32, and PC_BF16X3, whose spectra are
 * FP32); PC_FP64 gives PC_ERR_UNSUPPORTED.  Same arguments as
 * pc_apply_batched; it allocates its scratch on first use. */
pc_status pc_apply_plain(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx,
                         void *y, int64_t ldy, pc_stream stream);

/* Allocation-free variant of pc_apply_batched.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they apply the operator - for example a service that reserves all
 * of its GPU memory up front so that nothing on its request path can fail on
 * an out-of-memory error or wait for the device-wide synchronisation that a
 * cudaMalloc or cudaFree may imply, or code that runs where another allocator
 * owns the free device memory.  pc_apply_batched may allocate (it grows the
 * operator's ordering-flag buffer the first time a larger batch arrives);
 * this variant never calls cudaMalloc, cudaFree or any other allocating
 * routine.  Its scratch - one ordering flag per (tile, pair of right-hand
 * sides) plus a 64-byte control block - lives in a statically sized device
 * array of 1 MiB inside libpc that every GPU which loads the library holds
 * until the process exits.
 *   - Same arguments, layout and result as pc_apply_batched (y overwritten),
 *     for 2D operators; a 3D operator is refused with PC_ERR_UNSUPPORTED.
 *     The operator (spectra, weights, tiles) was allocated by
 *     pc_build_spectra; the caller owns x and y.
 *   - Limit: num_tiles * ceil(nrhs/2) <= 262128 (pc_operator_info gives
 *     num_tiles); larger batches fail with PC_ERR_ARG and a message, before
 *     anything is launched.  Split such batches.
 *   - The first call on a device sets the path up: it looks up the array's
 *     device address (cudaGetSymbolAddress with that device current), which
 *     also loads the library's module and with it the array, and loads this
 *     path's kernels; the result is cached.  A call with nrhs == 0 does this
 *     set-up and launches nothing: make such a call first, before the caller
 *     reserves its device memory and before any stream capture.
 *   - Every call, on every operator, shares the one array and it keeps the
 *     last call's contents; each call clears the part it uses before its
 *     kernel reads it.  Calls whose work overlaps on the GPU (different
 *     streams, or another thread) race on the array and give wrong results:
 *     serialise them, e.g. on one stream.
 *   - Device-side wait timeouts set a status word in the array, which
 *     pc_noalloc_check reads; the next call clears it.  The operator's own
 *     queries (pc_operator_check, pc_operator_kernel_time,
 *     pc_operator_launches) describe its last pc_apply* call and ignore the
 *     calls made here. */
pc_status pc_apply_batched_noalloc(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx,
                                   void *y, int64_t ldy, pc_stream stream);

/* Status of the last pc_apply_batched_noalloc call on ctx's device, which the
 * caller issued on `stream`: synchronises that stream, then returns
 * PC_ERR_TIMEOUT (and clears the word) if one of the call's device-side waits
 * ran out, else PC_OK.  Call it before the next allocation-free apply, which
 * clears the word.  Allocates nothing; the paper has no counterpart. */
pc_status pc_noalloc_check(pc_context *ctx, pc_stream stream);

/* ---------------------------------------------------------------------
 * Serving.  The paper's use of A~ is many applications to vectors that
 * arrive over time: preconditioner applications inside Krylov solves
 * (Section 5.2) and the random probes Y~ = A~* Z of the a-posteriori
 * estimator (Section 2.6, Algorithm 1).  A server keeps operators
 * resident, admits requests against a device-memory budget, and batches
 * the requests waiting at each moment - any operators, uneven right-hand
 * side counts - into one persistent launch of the fused kernel, replayed
 * from a CUDA graph captured at creation.  Launch slots run on separate
 * streams, so a new launch starts while earlier ones finish.  Each request
 * is computed exactly as pc_apply_batched would compute it alone.
 * 2D PC_FP32 operators with fft_size 128 are batched together as above.
 * Any other operator (2D with fft_size 64, PC_FP64 or per-patch shapes, 3D
 * PC_FP32 / PC_BF16X3) runs its requests on a launch slot through the
 * operator's own apply, one launch per such operator at a time: the request
 * at the head of the queue together with the requests on the same operator
 * and direction queued right behind it (at most 64 right-hand sides), whose
 * x blocks the server copies side by side into a staging buffer of the slot
 * (counted in the budget while the launch runs) and whose y blocks it copies
 * back.  Requests of different operators, and the batched launches, overlap
 * on the other slots.
 * --------------------------------------------------------------------- */

/* Create a server on ctx's device: a scheduler thread, `streams` launch
 * slots (each with its captured graph, a pinned launch descriptor, ordering
 * flags for up to 2^22 (tile, pair) units) and mapped completion flags. */
pc_status pc_serve_create(pc_context *ctx, const pc_serve_config *cfg, pc_server **srv);

/* pc_serve_submit flag: queue the adjoint Y = A~* X (Eq. adjoint_random_z)
 * instead; launches hold requests of one direction. */
#define PC_SERVE_ADJOINT 1u

/* Queue Y = A~ X for nrhs vectors: x and y are device arrays [nrhs][N] of
 * float (contiguous), owned by the caller and kept alive until pc_serve_poll
 * returns PC_OK for the ticket.  Returns at once with *ticket.  While an
 * operator has requests queued or running, the caller must not apply or
 * destroy it through other calls (the server's scheduler thread owns it;
 * for a 3D operator it grows the operator's ordering flags and scratch
 * before the launch, which may synchronise the device).  Errors:
 * PC_ERR_UNSUPPORTED for operators the server cannot launch, PC_ERR_BUDGET
 * if the operator and request alone exceed the budget, PC_ERR_ARG for bad
 * arguments.  flags: 0, or PC_SERVE_ADJOINT for Y = A~* X. */
pc_status pc_serve_submit(pc_server *srv, pc_operator *op, int32_t nrhs, const void *x, void *y, uint32_t flags,
                          uint64_t *ticket);

/* PC_ERR_NOT_READY while the request is queued or running; PC_OK (and
 * *info, if not NULL) once y holds the result - the record is then
 * released; PC_ERR_TIMEOUT / PC_ERR_CUDA if its launch failed; PC_ERR_ARG
 * for an unknown ticket. */
pc_status pc_serve_poll(pc_server *srv, uint64_t ticket, pc_request_info *info);

pc_status pc_serve_stats_get(pc_server *srv, pc_serve_stats *stats);

/* Waits for every admitted request, then stops the scheduler and frees the
 * server's resources.  Requests still queued are dropped. */
pc_status pc_serve_destroy(pc_server *srv);

/* Autotuner: enumerates the operator's launch shapes (FFT size P, kernel
 * sub-windows per axis, tile extent T, persistent CTAs per SM for 3D), ranks
 * them by a model of their line-FFT work, builds the best few and times a
 * batch of nrhs vectors on each with CUDA events on a private stream; a
 * candidate whose build, apply or device status fails is dropped.  Writes the
 * fastest into *best (*best_ms: its time per batch).  Same operator arguments
 * as pc_build_spectra, which runs the same search (nrhs = 32 in 2D, 8 in 3D)
 * when its pc_tuning is NULL and keeps the winning operator. */
pc_status pc_autotune(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                      const double *weights, pc_precision prec, int32_t nrhs, pc_tuning *best, double *best_ms);

/* Synchronise the operator's last stream and report device-side status:
 * PC_ERR_TIMEOUT if a bounded wait inside a kernel gave up since the last
 * call (the flag is then cleared), PC_ERR_CUDA on an asynchronous CUDA error. */
pc_status pc_operator_check(pc_operator *op);

/* Device time of the fused patch kernel of the operator's most recent
 * pc_apply / pc_apply_batched, in milliseconds, from CUDA events the library
 * records on the caller's stream just before and after that launch (the
 * zero-fill of y is outside the pair).  Waits for the end event.
 * PC_ERR_NOT_READY if no apply has been issued. */
pc_status pc_operator_kernel_time(pc_operator *op, float *ms);

/* Device time of one stage of the most recent apply of a 3D PC_BF16X3
 * operator, summed over its chunks of work items (milliseconds, CUDA events
 * on the caller's stream): stage 0 = input-plane 2D FFTs, 1 = tensor-core
 * first-axis DFT, spectral product and inverse DFT, 2 = inverse plane FFTs
 * and the ordered overlap-add.  Waits for the apply's end event.  The paper
 * has no counterpart (measurement helper).  PC_ERR_NOT_READY if the last
 * apply was not of that kind; PC_ERR_ARG if stage is not 0, 1 or 2. */
pc_status pc_operator_stage_time(pc_operator *op, int32_t stage, float *ms);

/* Counters of the operator's most recent apply (host): kernels launched. */
pc_status pc_operator_launches(const pc_operator *op, int64_t *kernels_last_apply);

pc_status pc_operator_destroy(pc_operator *op);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* PC_H */
