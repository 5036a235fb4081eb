/*
 * mf.h — C ABI of the GB300 grid max-flow / min-cut solver.
 *
 * The solver computes a maximum preflow and the minimum s-t cuts of a 2D or 3D
 * grid network by the parallel sweep of Augmented-path Region Discharge
 * (P-ARD): Algorithm 2 of Shekhovtsov & Hlavac, "A Distributed Mincut/Maxflow
 * Algorithm Combining Path Augmentation and Push-Relabel", with the region
 * discharge of Sec. 4.2 (Procedure ARD, Procedure Augment) and the
 * region-relabel and global-gap heuristics of Sec. 5.1.  Every region (a tile
 * of the grid) is discharged by one CUDA thread block per sweep; the flow and
 * label fusion of Algorithm 2 runs in a separate kernel.  Integer arithmetic
 * only (int32 capacities, int64 flow value); the results are exact.
 *
 * The problem (Sec. 2, Eq. 1): minimise over source sets S
 *     sum_{v not in S} cs(v) + sum_{v in S} ct(v) + sum_{u in S, w not in S} c(u,w)
 * where cs / ct are the source / sink link capacities of each grid vertex and
 * c(u,w) = c(w,u) >= 0 the capacity of the neighbour edge {u,w}.
 *
 * Conventions shared by every entry point:
 *   - vertex index v = (z*Y + y)*X + x (x fastest); n = X*Y*Z (Z = 1 in 2D);
 *   - connectivity 4 or 8 (2D) or 6 (3D) with the forward half-stencil
 *       4: h0 = (+1,0)   h1 = (0,+1)
 *       8: h0 = (+1,0)   h1 = (0,+1)   h2 = (+1,+1)   h3 = (-1,+1)
 *       6: h0 = (+1,0,0) h1 = (0,+1,0) h2 = (0,0,+1)
 *     and H = connectivity/2;
 *   - the synthetic networks of Sec. 7.1 join each node to the nodes at the
 *     displacements of the paper's list; MF_PAPER_STENCIL(c) (c = 8, 12, ...,
 *     28; ndim 2) takes its first c/2 entries as forward half-stencil
 *       h0 = (1,0) h1 = (0,1) h2 = (1,2) h3 = (2,1) h4 = (1,3) h5 = (3,1)
 *       h6 = (2,3) h7 = (3,2) h8 = (0,2) h9 = (2,0) h10 = (2,2) h11 = (3,3)
 *       h12 = (3,4) h13 = (4,2)
 *     (the list's first pair swapped so that c = 4 would be the 4-connected
 *     grid) with H = c/2; such grids are solved one by one on 32x32 tiles (or
 *     64x32 / 64x64 at c = 8) with
 *     the generic region discharge (kernel_variant 0 or 1 = ARD, 2 = PRD)
 *     and a global relabel of their own (opts.global_relabel_period), without
 *     warm start, region reduction, boundary relabel, batches or
 *     MF_STATE_HOST;
 *   - arc directions d = 0..2H-1: D(2h) = +h-th offset, D(2h+1) = -h-th
 *     offset; the reverse of d is d^1;
 *   - all arrays are dense int32 (or uint8) and row-major as above;
 *   - every call returns an mf_status; no C++ exception crosses the ABI;
 *     mf_last_error() gives a message for the last failing call on a handle;
 *   - input buffers stay owned by the caller and are copied; the handle owns
 *     all device memory it allocates; output buffers are caller-allocated;
 *   - "on_device" pointers are CUDA device pointers on the handle's device
 *     (e.g. the data_ptr() of a torch.cuda tensor); otherwise host pointers;
 *   - all work is ordered on the handle's stream; calls that return host data
 *     synchronise that stream.
 * The library has no CPU fallback: without a CUDA device mf_create_grid
 * fails with MF_ECUDA.
 */
#ifndef MF_H
#define MF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_grid mf_grid; /* opaque; owns all device memory of one instance */

/* connectivity code of the Sec. 7.1 synthetic stencil of connectivity c (see above) */
#define MF_PAPER_STENCIL(c) (100 + (c))

typedef enum {
    MF_OK = 0,
    MF_EINVAL = 1,       /* bad argument (dims, connectivity, tile, null pointer, negative capacity) */
    MF_ENOMEM = 2,       /* device or host allocation failed */
    MF_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error string) */
    MF_EOVERFLOW = 4,    /* capacities could overflow the int32 residual arithmetic */
    MF_ESWEEPLIMIT = 5,  /* opts.max_sweeps reached with active vertices left (state consistent) */
    MF_EROUNDLIMIT = 6,  /* a device-side loop hit its iteration cap (state consistent) */
    MF_ESTATE = 7        /* call out of order, e.g. mf_solve before mf_set_caps */
} mf_status;

/* Solver options.  mf_default_opts() fills the defaults. */
typedef struct {
    int32_t max_sweeps;            /* sweep cap; 0 = 2|B|^2+1 (the P-ARD bound, Sec. 4.4), clamped to 2^30 */
    int32_t partial_discharge;     /* 1: sweep s runs only ARD stages k <= s (Sec. 6.2); default 0 */
    int32_t global_gap;            /* 1: global gap heuristic after each sweep (Sec. 5.1); default 1 */
    int32_t global_relabel_period; /* P > 0: exact region-distance relabel after every P-th sweep (2D grids and
                                      3D grids with 32-wide tiles; Sec. 4.1 distance); 0 = off; default 4 */
    int32_t max_rounds;            /* cap on Augment rounds per stage inside one discharge; 0 = default 65536 */
    int32_t kernel_variant;        /* 0: bit-parallel 2D / 3D discharge where the tile allows (default); 1: generic kernel;
                                      2: Discharge = PRD (push-relabel region discharge of Sec. 3, exact region-relabel
                                      with unit arc lengths every round): the P-PRD algorithm on the same sweep loop,
                                      labels up to d_inf = n, global gap off, sweep cap 2n^2; for comparison */
    int32_t warm_start;            /* 1: start from the preflow of the last mf_warm_start instead of Init's zero flow */
    int32_t graph_loop;            /* 1: mf_solve runs the sweeps as one CUDA graph with a device-side while loop
                                      (per-phase times ms_discharge / ms_fuse are then not measured); default 0 */
    int32_t boundary_relabel_period; /* P > 0: boundary-relabel heuristic (Sec. 6.1) after every P-th sweep in
                                        which the global relabel does not run; any grid and tile; 0 = off (default) */
    int32_t global_relabel_first;  /* F > 0: the global relabel also runs after sweep F (where it is supported),
                                      besides every global_relabel_period-th sweep; 0 = off (default) */
    int32_t region_reduction;      /* 1: region reduction of Sec. 8 before Init (see mf_region_reduction): the
                                      strong source vertices are merged into s and the strong sink vertices into
                                      t, the sweeps run on the rest; flow value, S_min and S_max are those of the
                                      full network; not with warm_start; 0 = off (default) */
    int32_t reserved[5];
} mf_opts;

/* Statistics of the last mf_solve (all optional reading). */
typedef struct {
    int32_t sweeps;              /* sweeps of Algorithm 2 performed */
    int32_t boundary_size;       /* |B| of Sec. 4.1; d_inf = max(|B|, 1) */
    int64_t discharges;          /* region discharges performed (skipped regions not counted) */
    int64_t discharged_vertices; /* grid vertices inside the discharged regions, summed */
    int64_t stages;              /* ARD stages run, summed over discharges */
    int64_t rounds;              /* Augment rounds (BFS + layered push), summed */
    int64_t flow_value;          /* |f| (same as mf_flow_value) */
    int64_t launches;            /* CUDA kernels the solve launched */
    int32_t gaps;                /* sweeps in which the global gap raised labels */
    int32_t cut_passes;          /* passes of the cut-extraction closure */
    double ms_init, ms_sweeps, ms_cut, ms_total; /* device time per phase (CUDA events on the stream) */
    double ms_discharge;         /* device time of the discharge kernels alone, summed */
    double ms_fuse;              /* device time of fusion + gap + activity kernels, summed */
    int32_t global_relabels;     /* exact region-distance relabels run (opts.global_relabel_period) */
    int32_t relabel_levels;      /* BFS levels of those relabels, summed */
    int32_t projection_rounds;   /* rounds of the warm-start projection (0 for a cold start) */
    int32_t boundary_relabels;   /* boundary relabels applied (opts.boundary_relabel_period) */
    int32_t boundary_relabel_levels; /* levels of their searches over the auxiliary graph, summed */
    int32_t discharge_launches;  /* discharge launches timed in ms_discharge (single solve: one per sweep of the
                                    host loop; batch: persistent launches of this instance's kernel type) */
    int32_t reduced_vertices;    /* vertices merged into s or t by opts.region_reduction (0 without it) */
    int32_t reserved[1];
    double ms_relabel;           /* device time of the global and boundary relabels after sweeps (host-driven
                                    loops: CUDA events around each; a batch reports the whole batch's) */
} mf_stats;

/* Fill *opts with the defaults listed in mf_opts. */
void mf_default_opts(mf_opts *opts);

/*
 * Create a grid instance on the current CUDA device.
 *   ndim          2 or 3;
 *   dims          {X, Y, Z} (Z ignored and taken as 1 when ndim = 2), each >= 1;
 *   connectivity  4, 8 or MF_PAPER_STENCIL(c) for ndim = 2, 6 for ndim = 3;
 *   tile          region shape {tx, ty, tz}: the fixed partition of V into
 *                 regions R_k of Sec. 3 is the tiling of the grid by this
 *                 shape (edge tiles may be ragged).  Supported: 2D 64x64,
 *                 64x32, 32x32 and 32x16, 3D 32x16x8, 32x8x8, 32x8x4, 32x4x4 and
 *                 32x8x2 (bit-parallel discharge), 16x16x16 and 8x8x8; the
 *                 Sec. 7.1 stencils 32x32 (and 64x32, 64x64 at connectivity
 *                 8); NULL or {0,0,0} picks 32x32
 *                 (2D) / 32x8x4 (3D);
 *   cuda_stream   cudaStream_t to order all work on, or NULL for a stream
 *                 owned by the handle (non-blocking: device buffers that
 *                 other streams produce or consume must then be ordered by
 *                 the caller).  The default streams are given by their
 *                 handles cudaStreamLegacy / cudaStreamPerThread.
 * Allocates the device state (about (2H+6)*4 + 1 bytes per vertex plus a
 * second copy of the inputs).  On failure *out is NULL.
 */
mf_status mf_create_grid(mf_grid **out, int ndim, const int64_t dims[3], int connectivity,
                         const int32_t tile[3], void *cuda_stream);

/*
 * mf_create_grid with placement flags.  MF_STATE_HOST keeps the residual
 * planes, excess, labels, boundary outflows and the stored inputs (about
 * (3H+6)*4 bytes per vertex) in pinned host memory (the Grace memory of a
 * GB300 node): the kernels stage each region from there and write it back
 * over NVLink-C2C with plain loads and stores, the GPU keeps only the
 * per-region flags, counters, cut and relabel masks (a few bytes per
 * vertex).  This is the out-of-core mode of the sequential and streaming
 * variants (Sec. 4.3, Sec. 5.3: only the regions being discharged need to
 * be in fast memory); results are identical to device placement.
 * flags = 0 is mf_create_grid.  MF_EINVAL for unknown flags.
 */
#define MF_STATE_HOST 1
mf_status mf_create_grid_ex(mf_grid **out, int ndim, const int64_t dims[3], int connectivity,
                            const int32_t tile[3], void *cuda_stream, int flags);

/*
 * Set the capacities (Sec. 2: c : E -> N0, cs / ct the terminal links).
 *   cs, ct  int32[n], >= 0;
 *   nlink   int32[H][n]: nlink[h*n + v] = c(v, v + h-th forward offset)
 *           = c(v + offset, v); entries whose neighbour is outside the grid
 *           must be 0;
 *   on_device  0: host pointers, 1: device pointers; both are copied.
 * Errors: MF_EINVAL for negative capacities or nonzero links leaving the
 * grid; MF_EOVERFLOW if cs(v) plus the capacities of all edges at v could
 * exceed INT32_MAX, or if 2 c(u,w) could.
 */
mf_status mf_set_caps(mf_grid *g, const int32_t *cs, const int32_t *ct, const int32_t *nlink,
                      int on_device);

/*
 * mf_set_caps for count grids: the copies and validations of all grids are
 * enqueued first, then one wait per distinct stream; cs[i], ct[i], nlink[i]
 * as in mf_set_caps for grid i.  When every buffer is device, managed or
 * pinned host memory and the grids share one stream, a single kernel copies
 * all arrays (pinned host memory is read over the C2C link) and a single
 * kernel validates all grids.  The first grid that fails decides the
 * status (its message is also left on grids[0]); grids before it are set.
 */
mf_status mf_set_caps_batch(mf_grid *const *grids, int count, const int32_t *const *cs, const int32_t *const *ct,
                            const int32_t *const *nlink, int on_device);

/*
 * Solve: Init (Sec. 2: saturate every s-link; the part min(cs, ct) of each
 * vertex is sent s -> v -> t at once and counted in the flow value), then
 * sweeps of Algorithm 2 with Discharge = ARD until no vertex is active, then
 * the cut extraction.  opts may be NULL (defaults); stats may be NULL.
 * May be called again (it restarts from the stored capacities).
 * Errors: MF_ESTATE before mf_set_caps; MF_ESWEEPLIMIT / MF_EROUNDLIMIT when
 * a cap is hit (the preflow and labels stay valid; results are not final).
 */
mf_status mf_solve(mf_grid *g, const mf_opts *opts, mf_stats *stats);

/*
 * Step-wise form of mf_solve for inspection: mf_begin runs Init; each
 * mf_sweep runs one sweep of Algorithm 2 (discharge of every active region,
 * fusion, global gap) and returns the number of regions left active;
 * mf_finish extracts the cuts and the flow value.  mf_solve = begin, sweeps
 * until 0 active regions, finish.
 */
mf_status mf_begin(mf_grid *g, const mf_opts *opts);
mf_status mf_sweep(mf_grid *g, int32_t *active_regions);
mf_status mf_finish(mf_grid *g);

/*
 * Boundary-relabel heuristic of Sec. 6.1 on the current state (after mf_begin
 * or an mf_sweep; mf_solve runs it by itself with opts.boundary_relabel_period).
 * From the labels of the boundary vertices and the residual arcs between
 * regions alone it builds the section's auxiliary graph: one node per
 * (region, label) group, a length-0 arc from each group to the next higher
 * label of its region, a length-1 arc along each residual arc between regions.
 * The distance d' of a group to the label-0 groups is a valid lower bound on
 * the region distance, and every label becomes max(d, d').  A vertex inside a
 * region with label x > 0 takes the least d' of its region's groups with
 * label >= x (d_inf if none), so the labeling stays valid.  The gap histogram
 * and the region activity are rebuilt.
 *   info  int32[4] (nullable): [0] regions active afterwards, [1] levels of the
 *         search, [2] faces whose step list was shortened (their extra steps
 *         merged into one, which only weakens d'; 0 means d' is exact),
 *         [3] 1 if applied, 0 if the internal breakpoint pool overflowed (the
 *         labels are then unchanged).
 * Errors: MF_ESTATE before mf_begin; MF_ENOMEM / MF_ECUDA.
 */
mf_status mf_boundary_relabel(mf_grid *g, int32_t *info);

/*
 * Region reduction (Sec. 8, the Region Reduction algorithm) on the current
 * capacities, a preprocessing that decides vertices from one region's
 * network alone.  For every region R of the tiling by `tile`, the region
 * network G^R holds R with its terminal links, the boundary B^R (the
 * vertices outside R adjacent to R, without terminal links) and the edges
 * inside R and between R and B^R; from the zero flow it runs Augment(s,t),
 * splits B^R into B^S = {v : s -> v} and B^T = {v : v -> t}, runs
 * Augment(s,B^S) and Augment(B^T,t), and classifies each v of R in the final
 * residual network: s -> v strong source (on the source side of every
 * minimum cut of the whole network), v -> t strong sink (sink side of every
 * one), otherwise weak source if v does not reach B^R and weak sink if B^R
 * does not reach v (that side of some minimum cut).  One thread block per
 * region, the region network in shared memory.
 *   tile    region shape (NULL or zeros: the grid's tile if its network fits,
 *           else 32x32 in 2D and 32x8x4 in 3D); a region network has
 *           (tx+2)(ty+2)(tz+2) cells (tz+2 -> 1 in 2D) and needs
 *           ((connectivity+3)*4 + 3) bytes of shared memory per cell, at most
 *           232000 bytes;
 *   codes   uint8[n] (host or device per on_device): bit 1 strong source,
 *           bit 2 strong sink, bit 4 weak source, bit 8 weak sink;
 *   counts  int64[4] (nullable): strong sources, strong sinks, weak sources,
 *           weak sinks.
 * Errors: MF_ESTATE before mf_set_caps; MF_EINVAL if the tile's network does
 * not fit; MF_EROUNDLIMIT if an Augment of some region hit the round cap
 * (65536 rounds).
 */
mf_status mf_region_reduction(mf_grid *g, const int32_t tile[3], uint8_t *codes, int on_device, int64_t counts[4]);

/*
 * Batched solve: every grid of the array (each with capacities set, all on
 * one device) is solved at once.  Each sweep builds one work queue of the
 * active regions of all unfinished instances per kernel type (connectivity
 * and tile shape) and runs it with persistent thread blocks that pull
 * (instance, region) items; fusion, gap and activity run as one launch each
 * over the regions of the whole batch; an instance leaves the batch when it
 * has no active region.  All work is ordered on grids[0]'s stream.  Per
 * instance results are then read as after mf_solve (mf_get_cut,
 * mf_flow_value); stats (nullable) receives count entries (the ms_* fields
 * are those of the whole batch, except that without graph_loop ms_discharge
 * and discharge_launches are those of the persistent discharge launches of
 * the instance's kernel type, timed with CUDA events on the batch stream;
 * stats[0].launches also counts the launches shared by the whole batch, so
 * the launches of all entries add up to the batch's).  The global relabel (opts->
 * global_relabel_period) runs for every unfinished instance that supports it
 * after the same sweeps as in a single solve, so each instance takes the same
 * sweeps as alone.  With opts->warm_start = 1 each grid starts from its
 * projected preflow if mf_warm_start succeeded on it, and from Init
 * otherwise.  With opts->graph_loop = 1 the sweep loop of the batch is one
 * CUDA graph.  MF_ESWEEPLIMIT if instances are still active after
 * opts->max_sweeps sweeps (no cut is extracted; the grids stay usable and the
 * next solve starts again from Init).
 */
mf_status mf_solve_batch(mf_grid *const *grids, int count, const mf_opts *opts, mf_stats *stats);

/*
 * Minimum cut after a successful solve: out[v] = 1 if v is on the source side.
 *   which = 0: S_min, the closure of {v : e(v) > 0} under residual arcs
 *              (the minimal minimum-cut source set);
 *   which = 1: S_max = V minus {v : v -> t in G_f} (the cut (T-bar, T) of Sec. 2).
 * out is uint8[n] (host, or device when on_device = 1).
 */
mf_status mf_get_cut(mf_grid *g, uint8_t *out, int which, int on_device);

/*
 * mf_get_cut for count grids with one wait per distinct stream: out[i] is
 * uint8[n_i] for grid i; flows, if not NULL, int64[count] receives every
 * grid's flow value.  MF_ESTATE if a grid has no finished solve (nothing is
 * copied from that grid on); MF_EINVAL for NULL arrays or entries.
 */
mf_status mf_get_cuts_batch(mf_grid *const *grids, int count, int which, uint8_t *const *out, int on_device,
                            int64_t *flows);

/* |f| = sum of min(cs, ct) plus all flow the sweeps sent into t (int64). */
mf_status mf_flow_value(mf_grid *g, int64_t *out);

/*
 * Final (or current, after mf_sweep) residual network:
 *   res  int32[2H][n]: res[d*n + v] = residual capacity of the arc v -> v + D(d);
 *   tres int32[n]: residual of v -> t;  exc int32[n]: excess e_f(v).
 * Any of the three may be NULL.  Host or device buffers per on_device.
 */
mf_status mf_get_residual(mf_grid *g, int32_t *res, int32_t *tres, int32_t *exc, int on_device);

/* The residual network of the last solve (or of the current sweep): the
 * same as mf_get_residual(g, residual_out, NULL, NULL, 0): host int32[2H][n],
 * residual_out[d*n + v] = c_f(v -> v + D(d)).  NULL is a no-op. */
mf_status mf_get_flow(mf_grid *g, int32_t *residual_out);

/* Current labeling d (int32[n], values 0..d_inf) and d_inf. */
mf_status mf_get_labels(mf_grid *g, int32_t *lab, int32_t *d_inf, int on_device);

/*
 * Allocation-free cut extraction for 2D grids.  The paper has no counterpart:
 * this is a service for callers that must not allocate device memory at call
 * time, for example code that runs inside a framework owning all device
 * memory through its own pool with a fixed budget, or a latency-critical
 * loop where cudaMalloc (which may synchronise the device) is not allowed
 * after start-up.  It computes the same two cuts as mf_get_cut from a
 * residual network in the mf_get_residual layout:
 *   res, tres, exc  device pointers (int32[connectivity][n], int32[n], int32[n]),
 *                   typically the output of mf_get_residual(..., on_device = 1)
 *                   after a successful mf_solve;
 *   smin, smax      device outputs, uint8[n]: S_min (closure of {e > 0} under
 *                   residual arcs) and S_max (V minus {v -> t}), 1 = source side;
 *   dims            {X, Y}; connectivity 4 or 8; cuda_stream may be NULL.
 * All scratch lives in one file-scope device array of 8 MiB inside the
 * library (every GPU that loads the library holds it until the process
 * exits); nothing is allocated.  A grid needs
 *     256 + (connectivity + 2) * Y * ceil(X / 64) * 8
 * bytes of it, so the largest square grids are 2560 x 2560 at
 * 8-connectivity and 3328 x 3328 at 4-connectivity; larger grids are
 * rejected with MF_EINVAL.  Each call looks up the array's device address
 * for the current device.  All calls share the array: calls that overlap on
 * the GPU (other streams, other threads) race and must not be issued.  The
 * call synchronises cuda_stream (and reads a pass count back to the host)
 * before returning, so it cannot be used inside a stream capture.
 * Errors: MF_EINVAL (arguments, size), MF_ECUDA; message in
 * mf_last_error(NULL).
 */
mf_status mf_min_cut_2d_noalloc(const int64_t dims[2], int connectivity, const int32_t *res,
                                const int32_t *tres, const int32_t *exc, uint8_t *smin, uint8_t *smax,
                                void *cuda_stream);

/*
 * Learned warm start (2D grids; the paper is silent: the hook is the zero flow
 * of Init, Sec. 2).  Scale S = 100.
 *   mf_warm_features: x = device float[2+N][n]: cs/S, ct/S, then for arc
 *     directions d = 0..N-1 the capacity of the edge carried by arc d at v, /S.
 *   mf_warm_targets (after a finished solve): t = device float[N+2][n]: the
 *     flow out of v along arc d (d = 0..N-1), then, with m = min(cs, ct)
 *     routed straight through v by Init, cs - m - e(v) and ct - m - c_f(v,t);
 *     all /S.
 *   mf_warm_start: projects a prediction p (device float[N+2][n], target
 *     layout) to a valid preflow: edge flow f(v, v+h-th offset) = round(S p[2h][v])
 *     clamped to [-c, c]; sink flow round(S p[N+1][v]) clamped to
 *     [0, ct - min(cs,ct)]; every s-link saturated; then synchronous rounds in
 *     which each vertex with negative excess lowers its own outflows (sink
 *     first, then arcs 0..N-1) until no excess is negative.  The rounds are
 *     computed in phases over 32x32 tiles (a tile trims until none of its
 *     vertices has a deficit; phases repeat until no flow between tiles
 *     changes), which reaches the same preflow: any order of these trims
 *     ends at the least fixed point of a monotone map.  max_rounds <= 0 means
 *     4096 and caps the phases; *rounds (nullable) receives the phases run (0
 *     if the prediction already projected to a preflow).  The next
 *     mf_solve / mf_begin with opts.warm_start = 1 starts from this preflow;
 *     its labels are the exact region distances to t in the residual graph of
 *     that preflow (the global relabel, counted in stats.global_relabels) on
 *     2D grids with 32- or 64-wide tiles, else 0.  If no region is active
 *     after that relabel the solve makes no sweep.  MF_EROUNDLIMIT if the rounds run out: solve cold instead.
 * The results of a warm solve are the same exact flow value and cuts.
 */
mf_status mf_warm_features(mf_grid *g, float *x);
mf_status mf_warm_targets(mf_grid *g, float *t);
mf_status mf_warm_start(mf_grid *g, const float *pred, int32_t max_rounds, int32_t *rounds);
/* mf_warm_start for many grids with one wait: the projections are enqueued
 * on grids[0]'s stream.  preds[i] as in mf_warm_start, or NULL to leave grid
 * i cold; rounds (nullable, count entries) receives each grid's phases, or -1
 * where no preflow was reached (that grid then starts cold).  The next
 * mf_solve_batch with opts.warm_start = 1 starts every projected grid warm. */
mf_status mf_warm_start_batch(mf_grid *const *grids, int count, const float *const *preds, int32_t max_rounds,
                              int32_t *rounds);

/*
 * The network of the warm start: four 3x3 convolutions (zero padding),
 * C -> 32 -> 32 -> 32 -> C with ReLU after the first three, C = 6 (4-connected)
 * or 10 (8-connected).  FP32 master parameters, BF16 weights in every product,
 * FP32 accumulation.  Parameter vector: for layers l = 1..4 the weights
 * [C_out][C_in][3][3] then the biases [C_out].  Activations are device float
 * [N][C][H][W].  Training: forward, mf_cnn_mse (loss and dy), zero_grad,
 * backward (gradients of the parameters; needs the forward's input), Adam.
 * All work is ordered on cuda_stream (NULL: the legacy default stream); calls
 * that return host data (mse's loss, get_params/grads to host) synchronise it.
 */
typedef struct mf_cnn mf_cnn;
mf_status mf_cnn_create(mf_cnn **out, int in_ch, int out_ch, uint64_t seed, void *cuda_stream);
mf_status mf_cnn_destroy(mf_cnn *c);
const char *mf_cnn_last_error(const mf_cnn *c);
int64_t mf_cnn_num_params(const mf_cnn *c);
mf_status mf_cnn_get_params(mf_cnn *c, float *out, int on_device);
mf_status mf_cnn_set_params(mf_cnn *c, const float *in, int on_device);
mf_status mf_cnn_get_grads(mf_cnn *c, float *out, int on_device);
/* Load the parameters from a NumPy .npy file (little-endian float32 vector of
 * exactly mf_cnn_num_params entries, as written by the trainer); resets the
 * optimiser state.  MF_EINVAL with the reason in mf_cnn_last_error on a
 * missing file, another dtype or shape, or a truncated file. */
mf_status mf_load_model(mf_cnn *c, const char *path);
mf_status mf_cnn_forward(mf_cnn *c, const float *x, int N, int H, int W, float *y);
/* Inference only (no state kept for backward): the same network on the tensor
 * cores, with BF16 activations between layers (the input is rounded to BF16,
 * each hidden layer's ReLU output is stored as BF16), FP32 accumulation.
 * x and y as in mf_cnn_forward.  Holds two device buffers of N*H*W*32 BF16. */
mf_status mf_cnn_infer(mf_cnn *c, const float *x, int N, int H, int W, float *y);
mf_status mf_cnn_zero_grad(mf_cnn *c);
mf_status mf_cnn_backward(mf_cnn *c, const float *x, const float *dy);
mf_status mf_cnn_mse(mf_cnn *c, const float *y, const float *target, float *dy, int64_t count, double *loss);
mf_status mf_cnn_adam_step(mf_cnn *c, float lr, float beta1, float beta2, float eps);

/*
 * Optimality certificate of the last finished solve, computed on the device
 * from the original capacities: the preflow is feasible (0 <= r(v,w),
 * r(v,w) + r(w,v) = 2 c(v,w), 0 <= c_f(v,t) <= ct - min(cs,ct)), conserves
 * (e(v) = inflow - outflow >= 0 with every s-link saturated), and its flow
 * into t equals the capacity of the cut (S_min, V \ S_min) and the reported
 * flow value; by weak duality (Sec. 2) both are then optimal.
 *   cut_capacity (nullable)  capacity of (S_min, V \ S_min);
 *   violations   (nullable)  number of violated vertex / arc conditions;
 *   certified    (nullable)  1 iff violations = 0 and the three values agree.
 * MF_ESTATE without a finished solve.
 */
mf_status mf_certify(mf_grid *g, int64_t *cut_capacity, int64_t *violations, int32_t *certified);

/* Free the handle and all its device memory (NULL is a no-op). */
mf_status mf_destroy(mf_grid *g);

/* Message of the last failing call on g ("" if none; static text if g is NULL). */
const char *mf_last_error(const mf_grid *g);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */
