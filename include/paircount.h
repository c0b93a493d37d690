/*
 * paircount.h -- exact pair counting on one GB300 (sm_103a): grid and k-d tree.
 *
 * C ABI of the library built from paper_2301_12557_gb300/csrc.  Plain
 * pointers and sizes only.  Every pointer argument that carries catalogue
 * data or results may be HOST or DEVICE memory: the library asks the CUDA
 * driver which one it is and copies host data itself.  Edge arrays inside
 * pc_bins are always host memory.
 *
 * The operation (Zhao, "Fast Correlation Function Calculator", A&A 2023):
 *   Sect. 2.5  -- pair separation s = |x_j - x_i|, line-of-sight component
 *                 pi = |s.l|/|l|, sigma = sqrt(s^2 - pi^2), mu = pi/s, with
 *                 l = x_i + x_j (midpoint line of sight) or l = e_z;
 *   Sect. 3.2  -- monotone, continuous, zero-based bins, compared on squared
 *                 values (no square roots in the decision);
 *   Sect. 2.1  -- regular grid built in three passes (bounds, per-cell counts,
 *                 grouping) with points stored contiguously by cell;
 *   Sect. 3.1  -- auto counts visit each unordered pair once; periodic boxes
 *                 shift whole cells instead of wrapping each pair;
 *   Sect. 2.2, 3.1 -- the k-d tree (Alg. 1) and the dual-tree traversal
 *                 (Alg. 3) as a second space partition (pc_build_tree,
 *                 pc_count_tree);
 *   Sect. 3.2.4 -- the histogram-update micro-benchmark (pc_hist_s2).
 *
 * Exact semantics (identical to the FP64 definition the tests use):
 *   periodic canonical form  x <- x - L floor(x/L); if x<0 x+=L; if x>=L x-=L
 *   d = x_j - x_i per axis; periodic: d -= L if d > L/2, d += L if d < -L/2
 *   s2 = (dx*dx + dy*dy) + dz*dz in binary64 round-to-nearest, no FMA
 *   bin k of edges e[] iff e[k]^2 <= s2 < e[k+1]^2 (squares in binary64)
 *   (s, mu):   j = largest j < n_mu with pi2 >= (m[j]^2) * s2; m[0] = 0,
 *              m[n_mu] = 1 (mu = 1 goes to the last bin); s2 == 0 -> j = 0
 *   (sigma, pi): sigma2 = s2 - pi2 (clamped at 0); both axes half-open
 *   pi2 (LOS z) = dz*dz;  pi2 (midpoint) = (sl*sl)/ll with l = x_i + x_j,
 *              sl = (dx lx + dy ly) + dz lz, ll = (lx lx + ly ly) + lz lz
 *   auto: unordered pairs, no self-pairs; cross: all (i in g1, j in g2)
 *   weighted: sum of w_i * w_j per bin
 * Unweighted counts are bit-exact with that definition.  Weighted sums are
 * accumulated in binary64 (order-dependent rounding only).
 *
 * Per-device state: the library keeps count workspaces, captured graphs and
 * the allocation-free entry point's array address per device for the life of
 * the process; none of it survives a cudaDeviceReset, after which the library
 * must not be called on that device.
 */
#ifndef PAIRCOUNT_H
#define PAIRCOUNT_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  No call aborts or throws; details of the last failure on
 * the calling thread are available from pc_last_error(). */
typedef enum {
    PC_OK = 0,
    PC_EINVAL = -1,        /* invalid argument (message says which) */
    PC_ENOMEM = -2,        /* device or host allocation failed */
    PC_ECUDA = -3,         /* a CUDA runtime call failed */
    PC_EOVERFLOW = -4,     /* a size exceeds what the kernels index */
    PC_ETIMEOUT = -5,      /* a bounded device-side wait gave up */
    PC_EUNSUPPORTED = -6   /* valid request this build does not handle */
} pc_status;

typedef enum { PC_BIN_S = 0, PC_BIN_SMU = 1, PC_BIN_SIGPI = 2 } pc_mode;
typedef enum { PC_LOS_Z = 0, PC_LOS_MIDPOINT = 1 } pc_los;
typedef enum { PC_PREC_F32_RESCUE = 0, PC_PREC_F64 = 1 } pc_prec;

/* Domain.  periodic != 0: a box [0, L[a]) on every axis; coordinates are
 * folded into it (canonical form above).  periodic == 0: lo/hi give the grid
 * bounds when hi[a] > lo[a] on all three axes (all points must lie inside;
 * two grids used together in pc_count_cross must be built with the same
 * bounds), otherwise the bounds are the points' own bounding box. */
typedef struct {
    double L[3];
    int periodic;
    double lo[3];
    double hi[3];
} pc_box;

/* Histogram.  mode PC_BIN_S: n_a s bins, edges_a has n_a + 1 values.
 * PC_BIN_SMU: edges_a = s edges, edges_b = n_b + 1 mu edges from 0 to 1.
 * PC_BIN_SIGPI: edges_a = sigma edges, edges_b = pi edges.  Edges are
 * strictly increasing, finite and >= 0.  Output layout is row-major with the
 * first axis outermost: index = i_a * n_b + i_b (n_b = 1 for PC_BIN_S). */
typedef struct {
    int mode;               /* pc_mode */
    int los;                /* pc_los; midpoint needs a non-periodic box */
    int n_a;
    const double *edges_a;  /* host, n_a + 1 */
    int n_b;
    const double *edges_b;  /* host, n_b + 1 (ignored for PC_BIN_S) */
} pc_bins;

/* Tuning and execution options.  A NULL pc_opts pointer means all defaults
 * (every field 0). */
typedef struct {
    int prec;                    /* pc_prec: FP32 with FP64 rescue (0) or plain FP64 */
    double cell_size;            /* grid cell side; 0 = chosen by the cost model */
    int ipt;                     /* i-points per thread (2 or 4); 0 = auto */
    int priv;                    /* shared-histogram replication: 1 = one count copy per warp,
                                    2 = one shared copy, other values = automatic (up to 32
                                    lane copies, lane l updating copy l % k, when they fit
                                    16 KB: few bins then never collide within a warp) */
    long long rescue_capacity;   /* rescue-queue slots; 0 = auto; < 0 = none (all inline) */
    int use_graph;               /* pc_count_batch: replay a captured CUDA graph */
    int grid_ctas_per_sm;        /* persistent CTAs per SM; 0 = occupancy limit */
    int shard_index;             /* with shard_count > 1: count only the i-points of the */
    int shard_count;             /* cells (tree: list nodes) whose index % shard_count ==
                                    shard_index (multi-GPU shards; the int64 counts of all
                                    shards sum to the full count, and a shard is the same set
                                    of pairs whatever the precision or i-points per thread) */
} pc_opts;

/* Counters of the last count call (all optional). */
typedef struct {
    long long candidates;        /* pair separations evaluated by the kernel */
    long long rescued;           /* pairs re-evaluated in FP64 */
    long long rescue_inline;     /* of those, evaluated inline (queue full) */
    long long blocks;            /* i-blocks processed */
    double cell_size;            /* cell side used (first grid) */
    float ms_total;              /* device time of the call, milliseconds */
    float ms_pairs;              /* device time of the pair kernel alone */
    float ms_rescue;             /* device time of the rescue kernel */
    int launches;                /* kernels this call launched */
    long long pruned;            /* of the candidates, pairs the FP32 kernel decided out of
                                    range by one bounding-box test per point group */
    int prec;                    /* pc_prec that ran: PC_PREC_F64 also when FP32 was asked
                                    for but its error bound does not hold (midpoint line of
                                    sight with the observer too close to the points) */
    int wsum;                    /* weighted sums: 0 none; 1 binary64 products w_i w_j;
                                    2 exact products of binary32 significands accumulated
                                    as integers (evenly spaced bins, shared histograms, every
                                    weight a non-negative normal binary32 value or zero, each
                                    grid's weight exponents spanning at most 8 binades and
                                    the two grids' spans adding up to at most 12; truncation
                                    below 2^-34 relative), flushed in binary64; 3 the same
                                    for binary64 weights: the integer products of their
                                    binary32 roundings hi (conditions as for 2 on the his,
                                    which must reach 2^-78 where the weight is not a
                                    binary32 value) plus the binary32 terms hi_i lo_j +
                                    lo_i hi_j of their remainders lo = fl32(w - hi), rounded
                                    to the accumulators' unit (below 2^-34 relative) */
    long long tree_pairs;        /* pc_count_tree: list node pairs listed by the traversal */
    float ms_traverse;           /* pc_count_tree: device-and-host time of the traversal */
} pc_stats;

typedef struct pc_grid pc_grid;  /* opaque; owned by the library */

/* Build a grid: canonicalise (periodic) or bound (non-periodic) the points,
 * count points per cell, scan, and scatter them cell-sorted (SoA/AoS arrays
 * of FP32 cell-centre offsets and FP64 canonical coordinates) -- Sect. 2.1.
 *   xyz       n x 3 row-major binary64, host or device
 *   w         n weights (binary32 if w_is_f32 else binary64), or NULL
 *   r_max     largest separation the grid will serve (chooses the cell size
 *             when opt->cell_size == 0)
 *   stream    cudaStream_t (NULL = legacy default stream); all work is
 *             ordered on it and the call returns once the grid is built
 *   out       receives the new grid; release it with pc_free_grid
 * A periodic axis gets at least 2k + 1 cells for a stencil reach of k cells,
 * so that no two neighbour offsets reach the same cell; the cell side along
 * each axis is L[a] over its cell count (boxes may differ per axis).
 * Errors: PC_EINVAL (n < 0, NULL pointers, bad box, points outside given
 * bounds), PC_EOVERFLOW (n >= 2^31, or more than 2^26 cells -- e.g. a
 * periodic r_max within about 0.5 % of L/2, which the k-d tree path takes),
 * PC_ENOMEM, PC_ECUDA. */
pc_status pc_build_grid(const double *xyz, const void *w, int w_is_f32, long long n,
                        const pc_box *box, double r_max, const pc_opts *opt,
                        void *stream, pc_grid **out);

/* Release a grid (NULL is ignored). */
void pc_free_grid(pc_grid *g);

/* Number of points and cell side of a grid (either output may be NULL). */
pc_status pc_grid_info(const pc_grid *g, long long *n, double *cell_size);

/* Auto pair counts of one grid (unordered pairs, Sect. 3.1).
 *   counts    int64 [nbins], host or device; overwritten
 *   wcounts   binary64 [nbins] or NULL; weighted sums (the grid must carry
 *             weights)
 *   st        optional counters
 * Bins: see pc_bins.  Periodic boxes need the largest separation below L/2
 * (PC_EINVAL otherwise).  Returns after the results are written. */
pc_status pc_count_auto(const pc_grid *g, const pc_bins *b, const pc_opts *o, void *stream,
                        long long *counts, double *wcounts, pc_stats *st);

/* Cross pair counts: all (i in g1, j in g2) -- the data-random (DR) counts
 * of the estimators in Sect. 1, and any pair count of two catalogues (App. D:
 * the PAIR_COUNT sources, e.g. LR from catalogues L and R; DD, RR are auto
 * counts).  g1 and g2 must share box, bounds and cell size.
 *   counts    int64 [nbins], host or device; overwritten
 *   wcounts   binary64 [nbins] or NULL: sums of w_i w_j (both grids weighted)
 *   st        optional counters
 * Errors: PC_EINVAL (different boxes, bounds or cell sizes; bad bins),
 * PC_ENOMEM, PC_ECUDA.  Returns after the results are written. */
pc_status pc_count_cross(const pc_grid *g1, const pc_grid *g2, const pc_bins *b,
                         const pc_opts *o, void *stream, long long *counts, double *wcounts,
                         pc_stats *st);

/* Auto counts of m grids in one persistent launch (Sect. 4.2 task queue
 * analogue).  counts is m x nbins (row m), wcounts likewise or NULL.  All
 * grids must share box and cell size.  With o->use_graph the launch sequence
 * is captured once per (grids, bins) and replayed as a CUDA graph. */
pc_status pc_count_batch(const pc_grid *const *gs, int m, const pc_bins *b, const pc_opts *o,
                         void *stream, long long *counts, double *wcounts, pc_stats *st);

/* Auto pair counts like pc_count_auto, but the call allocates no device
 * memory (no cudaMalloc, cudaFree or allocating library routine): for
 * callers whose device memory is owned by another allocator, loops that must
 * not meet the implicit device synchronisation an allocation can trigger,
 * and processes running at their memory limit.  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 *   g         a grid from pc_build_grid, on the current device
 *   counts    int64 [nbins] (host or device), wcounts binary64 [nbins] or
 *             NULL; both written on return
 * All temporaries live in one fixed device array of about 12.3 MiB inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Its device address is looked up on the first call on each device
 * (a lookup that allocates nothing).  Like the library's
 * other per-device state (count workspaces, captured graphs), that address
 * does not survive a cudaDeviceReset of the device: do not call the library
 * on a device after resetting it.  Limits (PC_EOVERFLOW
 * beyond them): 16384 bins, 262144 grid cells, 524288 point blocks, 8192
 * stencil rows.  The array keeps the last call's contents and is cleared
 * where needed at the start of every call; calls are serialised by the
 * library and each returns only after its work has finished, and any two
 * such calls overlapping on the GPU (for instance from two processes sharing
 * one device context) would race on it. */
pc_status pc_count_auto_noalloc(const pc_grid *g, const pc_bins *b, const pc_opts *o,
                                void *stream, long long *counts, double *wcounts);

/* One configuration timed by pc_tune. */
typedef struct {
    double cell_size;   /* requested cell side */
    int ipt;            /* i-points per thread */
    int priv;           /* replication: 0 automatic, 1 one count copy per warp */
    float ms;           /* device time of the sampled pair and rescue kernels */
} pc_tune_trial;

/* Measured autotuner for the options of a count (the cost model of Appendix
 * B.1 gives the starting cell side).  Times the pair and rescue kernels on an
 * evenly spaced sample of the point blocks: 2 and 4 i-points per thread at
 * the model's cell side, then the better of those at cell sides in
 * quarter-octave steps from 0.7 to 2 times it (distinct grids only), then one
 * count copy per warp at the best, then (unless base fixes rescue_capacity)
 * the near-edge pairs evaluated inside the pair kernel (rescue_capacity -1)
 * instead of queued for the rescue kernel; writes the fastest options to
 * *out (base's other fields are kept).  pc_tune_trial of the last trial
 * carries the options it ran with.
 *   xyz, w, w_is_f32, n, box   the catalogue, as for pc_build_grid
 *   b                          the bins the counts will use
 *   base                       starting options (NULL = defaults); priv 1 or
 *                              2 there keeps the caller's replication
 *   trials                     optional host array of max_trials records;
 *                              *n_trials receives how many were written
 * Each trial runs on every S-th block, S chosen so that a trial takes about
 * 40 ms while every persistent CTA still gets two blocks or more.  Errors as
 * pc_build_grid and pc_count_auto; a cell side that needs too many cells is
 * skipped. */
pc_status pc_tune(const double *xyz, const void *w, int w_is_f32, long long n, const pc_box *box,
                  const pc_bins *b, const pc_opts *base, void *stream, pc_opts *out,
                  pc_tune_trial *trials, int max_trials, int *n_trials);

/* ---- k-d tree path (Sect. 2.2, Alg. 1; Sect. 3.1, Alg. 3) ---------------- */
typedef struct pc_tree pc_tree;  /* opaque; owned by the library */

/* Build the k-d tree of Alg. 1 on the GPU: the root holds all points; a node
 * of more than n_leaf points is split at the median along the axis of its
 * largest coordinate variance, the floor(n / 2) points of smallest coordinate
 * going to the left child, so the tree is balanced and all nodes of a level
 * hold the same share of the points to within one; every node keeps the
 * minimum bounding box (AABB) of its points.  Points are stored in tree order
 * (every node contiguous) as FP64 canonical coordinates and FP32 offsets from
 * the centre of their node at the list level: the level whose nodes the
 * traversal pairs and the pair kernel splits into balanced blocks of at most
 * 256 points.
 *   xyz, w, w_is_f32, n   as for pc_build_grid; n >= 1
 *   box                   periodic and L as for pc_build_grid (lo / hi are
 *                         not used: the tree bounds its own points)
 *   n_leaf                leaf capacity, 1..128
 *   list_cap              0: the list level is chosen among the levels whose
 *                         nodes hold 256..2048 points, for the fewest idle
 *                         lanes in the 256-point blocks; else a power of two
 *                         in [256, 65536]: the first level whose nodes hold at
 *                         most list_cap points
 *   stream                cudaStream_t; returns once the tree is built
 *   out                   the new tree; release it with pc_free_tree
 * Errors: PC_EINVAL (NULL pointers, n < 1, bad n_leaf or list_cap, bad box,
 * non-finite coordinates), PC_EOVERFLOW (n >= 2^31, more than 2^28 heap
 * slots), PC_ENOMEM, PC_ECUDA. */
pc_status pc_build_tree(const double *xyz, const void *w, int w_is_f32, long long n,
                        const pc_box *box, int n_leaf, int list_cap, void *stream,
                        pc_tree **out);

/* The k-d trees of m catalogues built together (Sect. 2.2, Alg. 1): one level
 * loop over all of them -- one pass of node statistics, one key pass and one
 * radix sort per level for every tree still being split -- instead of m
 * loops, for batches of many small catalogues (mocks).  Each tree is the one
 * pc_build_tree gives (the same node ranges, boxes and split axes, up to the
 * rounding of the node statistics on an exact variance tie) and is released
 * with pc_free_tree.
 *   xyz[k], w[k], n[k]    catalogue k as for pc_build_tree (host or device);
 *                         w NULL, or weights for every catalogue (all binary32
 *                         if w_is_f32, else all binary64)
 *   m                     number of catalogues, 1..65536
 *   box, n_leaf, list_cap as for pc_build_tree, shared by all trees
 *   stream                cudaStream_t; returns once every tree is built
 *   out                   m entries: out[k] receives catalogue k's tree (all
 *                         NULL on error)
 * Errors: PC_EINVAL (NULL pointers, m < 1, a catalogue without points,
 * weights for some catalogues only, bad n_leaf, list_cap or box, non-finite
 * coordinates), PC_EOVERFLOW (more than 2^31 points in all, more than 2^28
 * heap slots in one tree, m > 65536), PC_ENOMEM, PC_ECUDA. */
pc_status pc_build_tree_batch(const double *const *xyz, const void *const *w, int w_is_f32,
                              const long long *n, int m, const pc_box *box, int n_leaf,
                              int list_cap, void *stream, pc_tree **out);

/* Release a tree (NULL is ignored). */
void pc_free_tree(pc_tree *t);

/* Size of a tree (any output may be NULL): points, deepest level, list
 * level, heap slots 2^(depth + 1) - 1. */
pc_status pc_tree_info(const pc_tree *t, long long *n, int *depth, int *list_level,
                       long long *slots);

/* Copy the tree structure to HOST arrays (any may be NULL), heap order
 * (children of slot h: 2h + 1, 2h + 2):
 *   start, count  [slots] first tree position and points of each node;
 *                 count -1 marks an empty slot (below a leaf)
 *   axis          [slots] split axis, -1 for leaves and empty slots
 *   box           [6 slots] lo x, y, z, hi x, y, z of each node's points
 *   ord           [n] tree position -> input index */
pc_status pc_tree_export(const pc_tree *t, long long *start, long long *count, int *axis,
                         double *box, long long *ord);

/* Pair counts through the dual-tree traversal (Alg. 3): auto counts of t1
 * (t2 == NULL; unordered pairs) or cross counts of t1 x t2.  Node pairs
 * whose boxes lie farther apart than the largest separation (or, for s and
 * (s, mu) bins, all of whose pairs are closer than the first edge) are
 * dropped; the rest descend to pairs of list nodes, whose points are
 * evaluated by the same FP32 + binary64-rescue kernels as the grid path, so
 * the results follow the same exact definition.  Periodic boxes: every node
 * pair is taken under each periodic image of the second node.
 *   counts, wcounts, st   as for pc_count_auto (st adds tree_pairs, the list
 *                         node pairs, and ms_traverse; cell_size reports the
 *                         largest list node extent)
 *   o                     prec, ipt (2 or 4; blocks of at most 128 ipt points,
 *                         each list node split into equal blocks), priv,
 *                         rescue_capacity, grid_ctas_per_sm and the block
 *                         shards (shard_index of shard_count) apply
 * Errors: PC_EINVAL (trees of different boxes or devices, missing weights,
 * bad bins, a periodic separation of L/2 or more), PC_EUNSUPPORTED (plain
 * FP64 asked for, or forced by a midpoint line of sight too close to the
 * observer), PC_EOVERFLOW, PC_ENOMEM, PC_ECUDA. */
pc_status pc_count_tree(const pc_tree *t1, const pc_tree *t2, const pc_bins *b,
                        const pc_opts *o, void *stream, long long *counts, double *wcounts,
                        pc_stats *st);

/* Auto counts of m trees (all of one box and device) in one pair-kernel
 * launch: the tree path's counterpart of pc_count_batch.  Each tree is
 * traversed on its own (Alg. 3) and its list-node pairs appended to the
 * batch's lists; the persistent pair kernel then takes the blocks of all
 * trees from one work queue, each into its own histogram row.
 *   counts   int64 m x nbins (row k: tree k), host or device
 *   wcounts  binary64 m x nbins or NULL (every tree must carry weights)
 *   o, st    as for pc_count_tree
 * Errors as pc_count_tree. */
pc_status pc_count_tree_batch(const pc_tree *const *ts, int m, const pc_bins *b,
                              const pc_opts *o, void *stream, long long *counts,
                              double *wcounts, pc_stats *st);

/* Measured options of the k-d tree path for the auto count of a catalogue:
 * builds the tree (leaf capacity n_leaf) with the automatic list level and
 * with list nodes of at most 512, 1024, 2048 and 4096 points (distinct levels
 * only), times the pair and rescue kernels for 2 and 4 i-points per thread
 * on every S-th block (S as in pc_tune), and writes the fastest: out->ipt
 * (base's other fields kept) and *list_cap for pc_build_tree; the automatic
 * level with 2 i-points is kept unless another option is more than 3 %
 * faster.  A last trial (unless base fixes rescue_capacity) evaluates the
 * near-edge pairs inside the pair kernel (out->rescue_capacity -1 when
 * faster; its record has priv -1).  trials (cell_size holds the list_cap
 * tried, 0 = automatic) and n_trials as for pc_tune.
 * Errors as pc_build_tree and pc_count_tree. */
pc_status pc_tune_tree(const double *xyz, const void *w, int w_is_f32, long long n,
                       const pc_box *box, const pc_bins *b, int n_leaf, const pc_opts *base,
                       void *stream, pc_opts *out, int *list_cap, pc_tune_trial *trials,
                       int max_trials, int *n_trials);

/* ---- histogram-update micro-benchmark (Sect. 3.2.4) ---------------------- */
/* Histogram of n squared separations s2 (binary32, host or device), read
 * `repeat` times, on the edges e[0..nbins] with the pair definition's rule
 * (bin k iff e[k]^2 <= s2 < e[k+1]^2 in binary64; samples outside
 * [e[0]^2, e[nbins]^2) are not counted), by one update algorithm of Sect. 3.2:
 *   method 0  binary search over the squared edges (Sect. 3.2.1)
 *          1  reverse traversal from the last bin (Sect. 3.2.1)
 *          2  index mapping for linear bins, floor((sqrt(s2) - e0) / width),
 *             then a comparison with the neighbouring edges (Sect. 3.2.2)
 *          3  index mapping for logarithmic bins, on log2(s2) (Sect. 3.2.2;
 *             needs e[0] > 0), then the same correction
 *          4  hybrid index lookup table of table_size cells over the
 *             rescaled s2 (Sect. 3.2.3): each cell holds the range of bins
 *             its samples can reach, searched by reverse traversal
 * The table and the histogram live in shared memory (table_size <= 49152).
 *   counts   int64 [nbins], host or device: counts x repeat
 *   ms       optional: device time of the binning kernel
 * Errors: PC_EINVAL, PC_EOVERFLOW (over 2^31 samples per CTA),
 * PC_EUNSUPPORTED (table and histogram beyond shared memory), PC_ECUDA. */
pc_status pc_hist_s2(const float *s2, long long n, int repeat, const double *edges, int nbins,
                     int method, int table_size, void *stream, long long *counts, float *ms);

/* Measured arithmetic peak of the current device, for roofline fractions.
 * The paper has no counterpart (it benchmarks CPUs); this is measurement
 * infrastructure for the pair kernels' FP32 and FP64 pipes.
 *   kind      0: binary32 FFMA loop; 1: packed binary32 FFMA2 loop (two lanes
 *             per instruction); 2: binary64 DFMA loop
 *   iters     multiply-add steps per chain (0 = a default of ~50-150 ms)
 *   tflops    receives the rate, 10^12 flops per second (an FMA counts 2)
 *   ms        optional: the timed launch's duration
 * Every thread runs 8 independent FMA chains on a grid that fills every SM
 * to its thread limit; the launch is timed with CUDA events on `stream`
 * after one short untimed launch.  Allocates nothing; synchronises the
 * stream.  Errors: PC_EINVAL (bad kind or iters), PC_ECUDA. */
pc_status pc_fp_peak(int kind, long long iters, void *stream, double *tflops, float *ms);

/* Bounding box of n points (n x 3 binary64, host or device) -- the first of
 * the three grid-build passes of Sect. 2.1.  lo/hi are host arrays of 3. */
pc_status pc_aabb(const double *xyz, long long n, void *stream, double *lo, double *hi);

/* The stencil rows the grid path enumerates for cells of sides cell[3] and
 * largest separation r_max (Sect. 2.1; Sect. 3.1 duplicate removal when
 * half != 0).  Host-only: no device work.  Row k is rows[4k .. 4k + 3] =
 * {dy, dz, xlo, xhi}: the neighbour cells at offsets (dx, dy, dz) for dx in
 * [xlo, xhi].  A cell offset is in the full stencil when the smallest
 * distance between the two cells, max(|d| - 1, 0) x side per axis, is below
 * r_max.  The half stencil keeps exactly one of each pair of opposite
 * offsets (the own cell is the kernel's own-block pass and the offsets
 * (dx > 0, 0, 0)).  *n_rows receives the row count; PC_EOVERFLOW when it
 * exceeds max_rows. */
pc_status pc_stencil(const double cell[3], double r_max, int half, int max_rows, int *rows,
                     int *n_rows);

/* The FP32 path's error bands for a count (Sect. 2.5 quantities; how the
 * fast path stays exact is stated at the top of this header).  Host-only: no
 * device work.  For bins b on cells of sides cell[3] (the cell side, or for
 * the tree path the largest list-node extent), points within [lo, hi] per
 * axis, a periodic box of sides L[3] (L may be NULL when periodic == 0) and
 * rmin, a lower bound of the points' distance from the observer (midpoint
 * line of sight; 0 if unknown), out[0..18] receives:
 *   0 eps_a   band of s (s and (s, mu) bins) or of sigma ((sigma, pi) bins)
 *   1 eps_b   band of pi ((sigma, pi) bins)
 *   2 mu_A    the mu band is mu_A / s + mu_B ((s, mu) bins)
 *   3 mu_B
 *   4 rcut    FP32 candidate cut on the separation (largest separation plus
 *             twice the largest band)
 *   5 fp32_ok 1 when the FP32 path's bound holds (else counts run in FP64)
 *   6 lin     1 when the bins are found by a floor instead of tables
 *   7 r2cut   the FP32 cut the kernel compares s^2 against
 *   8..15     floor-based bins (when lin): t = s * invA + offA and bin =
 *             floor(t), not near an edge iff |frac(t) - 1/2| < thrA (offA
 *             carries +1 when the s range is tested, the bin then floor(t) -
 *             1); mu bins t_mu = mu * nB, not near iff |frac(t_mu) - 1/2| <
 *             cB - mA / s; then norange (1: e_0 = 0 and no range test) and
 *             log (1: logarithmic s edges, t from log2(s^2)):
 *             invA, offA, thrA, nB, mA, cB, norange, log (with log, t =
 *             log2(s^2) * invA + offA and the band is thrA - mS / s, mS in
 *             out[18])
 *   16..17    (sigma, pi) floor bins: t_pi = pi * invB, not near iff
 *             |frac(t_pi) - 1/2| < thrB (sigma as s, with offA = 0):
 *             invB, thrB
 *   18 mS     logarithmic s bins: the band's term in 1/s
 * A pair takes the fast path's bin only when its FP32 value lies at least
 * the band away from every edge; closer pairs are decided in binary64.
 * Errors: PC_EINVAL (NULL pointers, bad cell sides, bounds, box or bins). */
pc_status pc_fp32_bands(const pc_bins *b, const double cell[3], const double lo[3],
                        const double hi[3], const double L[3], int periodic, double rmin,
                        double out[19]);

/* The lookup tables the FP32 path stages for the same count as
 * pc_fp32_bands (host-only).  lut receives n_entries pairs {edge, bin
 * below} as binary32 (the bin as the float's bit pattern): per table T + 2
 * cells of width 1 / inv_w over the binned quantity, each holding the single
 * edge within the band of the cell (+inf: none; NaN: several, or the
 * sentinel cell T + 1, always rescued) and the bin just below it; a value v
 * takes cell min(floor(v inv_w), T + 1), bin = below + (v >= edge), and is
 * near an edge unless |v - edge| >= its band.  desc[0..6] = first entry, T
 * and inv_w of the first axis's table (s or sigma), the same for the second
 * (mu or pi), and mu's window (a mu band wider than it is always rescued).
 * *n_entries is set even when the tables do not fit max_entries
 * (PC_EOVERFLOW).  Errors as pc_fp32_bands. */
pc_status pc_fp32_tables(const pc_bins *b, const double cell[3], const double lo[3],
                         const double hi[3], const double L[3], int periodic, double rmin,
                         float *lut, int max_entries, int *n_entries, double desc[7]);

/* Cell side the cost model picks for n points in volume `volume` with
 * largest separation r_max (Appendix B.1: cost a N_pair + b N_node). */
double pc_suggest_cell_size(long long n, double volume, double r_max, int mode);

/* Number of kernels this library has launched since it was loaded (all
 * entry points, all threads).  Lets callers count device work per step. */
long long pc_launch_count(void);

/* Number of device (and pinned host) allocations this library has made since
 * it was loaded (all entry points, all threads): grids, trees, count
 * workspaces and temporaries.  Lets callers check that a call allocated
 * nothing (pc_count_auto_noalloc). */
long long pc_alloc_count(void);

/* Static description of a status code. */
const char *pc_strerror(pc_status s);

/* Detail message of the last failing call on this thread ("" if none). */
const char *pc_last_error(void);

/* Library version string. */
const char *pc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAIRCOUNT_H */
