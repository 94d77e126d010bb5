/* f2m.h -- C ABI of the GB300 (sm_103a) solver for the fractional 2-matching
 * (F2M) LP relaxation of the TSP by the gradient descent procedure (GDP) of
 * A. Antonov, "Gradient descent procedure for solving linear programming
 * relaxations of combinatorial optimization problems in parallel mode on extra
 * large scale" (arXiv 2011.08170).
 *
 * The problem (Section 4, "F2M"): given points p_v with integer coordinates and
 * an undirected candidate edge set E, minimise sum_e c_e x_e subject to
 * sum_{e in delta(v)} x_e = 2 for every node v and 0 <= x_e <= 1.  Costs are
 * TSPLIB EUC_2D lengths c_uv = floor(sqrt(dx^2 + dy^2) + 1/2) (the input of the
 * paper's program is TSPLIB 2-D coordinates, Section 5.1).  The optimum is
 * {0, 1/2, 1} valued (Section 4).
 *
 * The method (Sections 2-4): lambda_v is adjusted until the modified objective
 * z_e = c_e - lambda_u - lambda_v (Eq. 9) is "trivial": z_e < 0 on x_e = 1,
 * z_e = 0 on x_e = 1/2, z_e > 0 on x_e = 0 (rule (7)).  The gradient at v is
 * taken from the 2nd and 3rd shortest adjusted edges at v (Eq. 10), computed
 * for every node in parallel (Section 5.1).
 *
 * Numbers.  lambda and z are exact fixed-point integers in units of
 * 2^-frac_bits of a length unit.  One GDP sweep (Jacobi) sets, for every v,
 *   delta_v = trunc((z(2) + z(3)) / 2^damping_shift),  lambda_v += delta_v,
 * where z(2) <= z(3) are the 2nd and 3rd smallest z over the row of v.  The dual
 * bound reported is bound2 = 2 * LB = 4 * sum_v lambda_v + sum over directed
 * CSR entries of min(0, z_e), i.e. twice the Lagrangian bound
 * LB = 2 sum lambda + sum_e min(0, z_e), in units of 2^-frac_bits.  Every result
 * is bit-exact and independent of thread scheduling.
 *
 * A solve repeats: a GDP phase (to a fixed point, or max_iters sweeps); an
 * all-pairs pricing scan that adds every non-candidate edge with z < 0 (the
 * candidate graph may miss optimal edges, Section 5.3); primal x from the
 * signs of z (rule 7); where that x is infeasible (the degenerate stops of
 * Section 3, last paragraph) an exact min-cost-flow finisher on the host,
 * after which lambda has frac_bits + 1 bits.  It ends when a scan with the
 * final lambda finds nothing: x and lambda are then certified optimal for the
 * COMPLETE graph on the points.
 *
 * Conventions.
 *  - Pointers marked "host or device" may point to either; the library asks
 *    the driver which.  Work runs on the stream given at create time.
 *  - The library copies every input; the caller owns every output buffer.
 *  - No call exits or aborts.  Each returns a status; f2m_last_error(ctx)
 *    gives a message for the last failure on that context.
 *  - A context is not thread-safe: use one per host thread.
 *  - Indices in and out are the caller's numbering.
 */
#ifndef F2M_H
#define F2M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  F2M_OK = 0,
  F2M_ERR_INVALID_ARG = 1,      /* bad size, range, pointer or CSR */
  F2M_ERR_CUDA = 2,             /* a CUDA call failed */
  F2M_ERR_OOM = 3,              /* device or host allocation failed */
  F2M_ERR_NOT_CONVERGED = 4,    /* iteration or pricing-round cap reached */
  F2M_ERR_OVERFLOW = 5,         /* some |lambda| reached 2^29 (units 2^-F) */
  F2M_ERR_PRICING_OVERFLOW = 6, /* pair buffer too small (handled inside f2m_solve) */
  F2M_ERR_INFEASIBLE = 7,       /* no fractional 2-matching (b-matching) on the candidate graph */
  F2M_ERR_TIMEOUT = 8           /* a device-wide barrier wait ran past its budget */
} f2m_status;

typedef struct f2m_ctx f2m_ctx;   /* opaque, library-owned */

typedef struct {
  int32_t frac_bits;            /* F, fractional bits of lambda; 1..8; default 8 */
  int32_t damping_shift;        /* delta = trunc((z2+z3) / 2^shift); 1..8; default 2 */
  int64_t max_iters;            /* sweeps per GDP phase; default 128.  A phase ends at a
                                   fixed point or after max_iters sweeps; f2m_solve then goes
                                   on from the lambda reached (pricing, rule (7), finisher), so
                                   the certified optimum does not depend on it */
  int32_t max_pricing_rounds;   /* pricing scans per solve; default 64 */
  int32_t pricing;              /* 0 = solve on the candidate graph only, 1 = full scan of all
                                   n(n-1)/2 pairs (default), 2 = the same scan skipping tile pairs
                                   whose bounding boxes are too far apart to hold a pair with z < 0
                                   (same pairs found, same results) */
  int64_t pricing_cap;          /* initial pair-buffer capacity; default 1 << 20 */
  int64_t barrier_budget_cycles;/* spin budget of one device-wide barrier wait; default 4e9 */
  int32_t finisher;             /* 1 = exact finisher when rule (7) gives an infeasible x (default) */
  uint32_t flags;               /* F2M_FLAG_* bits; default 0 */
  int32_t gdp_lanes;            /* lanes per node in the tiled GDP kernel: 1 (one thread per node); 0 = auto */
  int32_t gdp_ctas_per_sm;      /* tiled GDP CTAs per SM: 1 (x1024 threads), 2 (x512); 0 = auto */
  int32_t batch_shape;          /* batched GDP kernel shape (threads, copy stages, CTAs per SM):
                                   -1 = picked by the autotuner (default), 0..4 = a fixed one */
  int32_t batch_graph;          /* 1 = replay each batched GDP phase from a captured CUDA graph
                                   (default), 0 = launch directly; same results */
} f2m_params;

/* f2m_params.flags: run GDP with the streaming kernel (CSR read from global
 * memory every sweep, caller node order) instead of the default shared-memory
 * tiled kernel (nodes renumbered along a Morton curve, each CTA's rows, own
 * lambda and halo held in shared memory).  Both give identical results. */
#define F2M_FLAG_STREAMING_GDP 1u

/* f2m_params.flags: run the shared-memory tiled GDP kernel with one sweep per
 * device-wide barrier instead of the default two (the default keeps each
 * CTA's halo rows and a second halo ring, computes the halo rows' sweep
 * redundantly, and meets the other CTAs once per two sweeps).  Identical
 * results either way. */
#define F2M_FLAG_ONE_SWEEP_GDP 2u

/* f2m_params.flags: class-by-class GDP sweeps (a Gauss-Seidel form of the
 * parallel update of Section 5.1; the paper does not describe it).  The graph
 * is coloured greedily -- each node takes the smallest colour not held by a
 * higher-priority neighbour, priority = larger degree, then larger
 * SplitMix64(v) (the generator's first output seeded with v), then smaller v --
 * and a sweep updates class 0, 1, ... in turn, every node of a class from the
 * current lambda of its neighbours, in place.  With damping_shift = 1 each
 * class update is exact block coordinate ascent and the bound never falls.
 * A node whose new value would reach 2^29 keeps its value and the phase stops
 * with OVERFLOW after that sweep.  The colouring is redone whenever the graph
 * changes.  Single-instance contexts; batches ignore the flag. */
#define F2M_FLAG_CLASS_SWEEPS 4u

/* f2m_params.flags (batches, with batch_shape -1): run batched GDP phases on
 * thread-block clusters instead of the default streaming batch kernels (the
 * union CSR streamed from HBM every sweep, one device-wide barrier per sweep):
 * every instance gets a cluster of 1-16 CTAs that holds its rows and lambda in
 * shared memory, with the hardware cluster barrier per sweep and neighbours'
 * lambda read through distributed shared memory.  A batch with an instance too
 * large for 16 CTAs (2048 nodes, 24,000 entries each) uses the streaming
 * kernels.  Same results either way. */
#define F2M_FLAG_BATCH_CLUSTERS 8u

/* f2m_params.flags: where the finisher's first phase (successive shortest
 * paths block by block, 2,048 nodes a block) runs.  By default (or with
 * F2M_FLAG_FINISHER_HOST) it runs on the host threads; F2M_FLAG_FINISHER_GPU
 * runs it on the GPU, one warp per block.  The same searches run in the same
 * order either way, so the results are identical; the searches are sequential
 * within a block, and one warp per block is slower than a host thread per
 * block at the sizes measured, so the host is the default. */
#define F2M_FLAG_FINISHER_HOST 16u
#define F2M_FLAG_FINISHER_GPU 32u

/* f2m_params.flags: run the full pricing scan (pricing = 1) with the
 * tensor-core filter (per 128 x 128 tile pair, quantised coordinates and radii
 * in a frame fitted to the pair; the test |D|^2 < (R_u + R_v)^2 as one exact
 * small-integer fp16 matrix product with an fp32 accumulator; candidates then
 * decided by the fp32 filter and exactly) instead of the default fp32 filter on
 * the CUDA cores.  The same pairs either way; at n = 100k the default is faster
 * (0.96 against 1.3 ms per scan on a GB300). */
#define F2M_FLAG_PRICING_TENSOR 64u

typedef struct {
  int64_t iterations;           /* GDP sweeps, all phases */
  int64_t phases;               /* GDP phases */
  int64_t pricing_rounds;       /* pricing scans */
  int64_t edges_added;          /* undirected edges added by pricing */
  int64_t finisher_calls;
  int64_t augmentations;        /* unit augmentations in the finisher */
  int64_t bound2;               /* 2*LB in units 2^-frac_bits */
  int64_t nnz;                  /* directed CSR entries after pricing */
  int32_t frac_bits;            /* of bound2 and lambda: F, or F+1 after the finisher */
  int32_t certified;            /* 0 none, 1 optimal on the candidate graph, 2 optimal on all pairs */
  int32_t status;               /* f2m_status of the solve */
  int32_t batch_shape;          /* batch totals: shape index of the batched GDP kernel; else -1 */
  int32_t batch_graph;          /* batch totals: 1 if the GDP phases ran from a captured graph */
  int32_t gdp_kernel;           /* GDP kernel of the last phase: F2M_GDP_KERNEL_* */
  double ms_gdp;                /* device time of the GDP phases */
  double ms_pricing;            /* device time of the pricing scans */
  double ms_merge;              /* device time of the CSR merges */
  double ms_extract;            /* device time of the sign extraction */
  double ms_finish;             /* host time of the finisher incl. copies */
  double ms_total;              /* host wall time of f2m_solve */
  /* the finisher's split (host clock): device preparation and copies to the
   * host, the three phases of successive shortest paths (blocks of 2,048
   * nodes on all host threads, blocks of 16,384, the rest per instance), and
   * the copies back with the scatter; augmentations per phase */
  double ms_finish_prep;
  double ms_finish_phase[3];
  double ms_finish_scatter;
  int64_t finish_aug_phase[3];
  int32_t finish_threads;       /* host threads the blocked phases used */
  int32_t finish_phase1_gpu;    /* 1 if the finisher's phase 1 ran on the GPU */
  int64_t pricing_pairs;        /* pairs the pricing scans evaluated: n(n-1)/2 a full scan (also
                                   the culled one, which skips pairs it proves positive), rows x n
                                   a certifying scan of the finisher's lambda (only the nodes
                                   whose lambda rose can make a pair negative) */
  int32_t certifying_scans;     /* scans of that second kind */
  int32_t pad_;
} f2m_info;

/* f2m_info.gdp_kernel values */
#define F2M_GDP_KERNEL_STREAMING 0     /* CSR read from global memory every sweep */
#define F2M_GDP_KERNEL_TILED 1         /* shared-memory tiles, one sweep per barrier */
#define F2M_GDP_KERNEL_TWO_SWEEP 2     /* shared-memory tiles, two sweeps per barrier */
#define F2M_GDP_KERNEL_TWO_SWEEP_PACKED 3  /* the same with 4-byte entries (larger tiles) */
#define F2M_GDP_KERNEL_CLASSES 4       /* class-by-class sweeps */
#define F2M_GDP_KERNEL_BATCH 5         /* batched, union CSR streamed */
#define F2M_GDP_KERNEL_BATCH_CLUSTERS 6  /* batched, one thread-block cluster per instance */
#define F2M_GDP_KERNEL_CUTS 7          /* node and subtour-cut duals, streaming */

/* Fills *p with the defaults above.  p must not be NULL. */
void f2m_default_params(f2m_params* p);

/* Creates a solver context for one instance (Section 4 F2M on a candidate graph;
 * Section 5.1 input: 2-D integer coordinates).
 *   xy       [n][2] int32, host or device; every coordinate in [0, 2^20).
 *   n        number of nodes, 4 <= n < 2^24.
 *   row_ptr  [n+1] int32, host or device; row_ptr[0] = 0, nondecreasing.
 *   col      [row_ptr[n]] int32, host or device; the candidate graph with both
 *            directions stored, each row sorted ascending, no self-loops, no
 *            duplicates, and every node of degree >= 3 (Eq. 10 needs a 3rd edge).
 *   params   NULL for defaults.
 *   stream   cudaStream_t (as void*) on which all work of this context runs;
 *            NULL = the legacy default stream.
 *   out      receives the context; on failure *out is NULL.
 * Computes the cost table (one exact integer cost per CSR entry) on the device.
 * lambda starts at 0.  Errors: INVALID_ARG (with the first violated rule in
 * f2m_last_error(NULL)), OOM, CUDA. */
f2m_status f2m_create(const int32_t* xy, int32_t n, const int32_t* row_ptr, const int32_t* col,
                      const f2m_params* params, void* stream, f2m_ctx** out);

/* Releases all memory of ctx.  NULL is ignored. */
void f2m_destroy(f2m_ctx* ctx);

/* Sets lambda (warm start, resume from a checkpoint).
 *   lambda  [n] int32, host or device, units 2^-frac_bits; |lambda| < 2^29.
 * Errors: INVALID_ARG (range), CUDA. */
f2m_status f2m_set_lambda(f2m_ctx* ctx, const int32_t* lambda, int32_t frac_bits);

/* Sets per-node degree requirements: the fractional b-matching LP
 * (sum of x over delta(v) = b_v, 0 <= x <= 1), the LP3 class of Section 3 with
 * binary coefficients and integral right sides (Eq. 8).  The GDP update then
 * takes the b_v-th and (b_v+1)-th smallest adjusted values of row v in place
 * of Eq. 10's 2nd and 3rd, the bound becomes 2*sum(b_v lambda_v) + sum over
 * directed entries of min(0, z), rule (7) extraction checks row sums 2 b_v, and
 * the finisher's supplies and demands are b_v.  Pricing is unchanged.
 *   b  [n] int32, host or device, copied; 1 <= b_v <= deg(v) - 1 for the
 *      graph held now (pricing only adds edges).  NULL restores b_v = 2.
 * Single-instance contexts only.  While b is set, GDP phases run on the
 * two-sweep shared-memory kernel (a sorted top-8 per row when every b_v < 8,
 * counting otherwise) or, where its tiles do not fit, the streaming kernel.
 * Errors: INVALID_ARG (range, with the first offending node in
 * f2m_last_error; the previous b stays), OOM, CUDA. */
f2m_status f2m_set_degrees(f2m_ctx* ctx, const int32_t* b);

/* The colouring of the current candidate graph used by F2M_FLAG_CLASS_SWEEPS
 * (computed now if the graph changed since the last one).
 *   color    [n] int32, host or device, written: the class of every node.
 *   ncolors  written: the number of classes.
 * Either pointer may be NULL.  Errors: INVALID_ARG (NULL ctx), OOM, CUDA. */
f2m_status f2m_get_colors(f2m_ctx* ctx, int32_t* color, int32_t* ncolors);

/* Full solve from the current lambda (see the header comment).  info may be
 * NULL.  Returns F2M_OK when certified (info->certified = 2 with pricing on, 1
 * with pricing off); NOT_CONVERGED when a cap ran out first (lambda and x
 * then hold the last state); OVERFLOW, INFEASIBLE, TIMEOUT, CUDA, OOM. */
f2m_status f2m_solve(f2m_ctx* ctx, f2m_info* info);

/* ---- the hot-path steps, one call each (Sections 4 and 5.1) --------------- */

/* One GDP phase (Eq. 9, Eq. 10, Jacobi): up to max_sweeps sweeps from the
 * current lambda (units 2^-F), stopping after the first sweep that changes no
 * lambda.  Runs as one persistent cooperative kernel with a device-wide
 * barrier per sweep.
 *   sweeps         out: sweeps run.
 *   trace_bound2   NULL or [trace_cap] int64 (host or device): bound2 at the
 *                  lambda each sweep started from.
 *   trace_changed  NULL or [trace_cap] int64: #nodes whose lambda changed.
 * Returns OK at a fixed point, NOT_CONVERGED at max_sweeps, OVERFLOW (lambda
 * left at the input of the overflowing sweep), TIMEOUT, CUDA. */
f2m_status f2m_gdp(f2m_ctx* ctx, int64_t max_sweeps, int64_t* sweeps, int64_t* trace_bound2,
                   int64_t* trace_changed, int64_t trace_cap);

/* Pricing scan: every pair u < v that is not a candidate edge and has
 * c_uv * 2^fb < lambda_u + lambda_v (z < 0), fb = the current frac_bits.
 *   count  out: number of such pairs (may exceed cap).
 *   pairs  NULL or [cap][2] int32 (host or device): the pairs, ascending
 *          (u, v) (caller numbering), when count <= cap.
 * The pairs are not added; see f2m_add_edges.  Errors: CUDA, OOM. */
f2m_status f2m_price(f2m_ctx* ctx, int64_t* count, int32_t* pairs, int64_t cap);

/* Adds undirected edges to the candidate graph (both directions, rows kept
 * sorted, pairs already present ignored) and their costs.
 *   pairs  [npairs][2] int32, host or device, u != v, both in [0, n).
 * Errors: INVALID_ARG, OOM, CUDA. */
f2m_status f2m_add_edges(f2m_ctx* ctx, const int32_t* pairs, int64_t npairs);

/* Primal from rule (7): x2_e = 2 if z_e < 0, 1 if z_e = 0, 0 if z_e > 0 (x in
 * half units), at the current lambda.
 *   x2   NULL or [nnz] uint8 (host or device), in the CSR order of f2m_get_x.
 *   bad  out: number of nodes whose row of x2 does not sum to 4. */
f2m_status f2m_extract(f2m_ctx* ctx, uint8_t* x2, int64_t* bad);

/* One GDP phase that allocates no memory, for callers that cannot allocate
 * device memory where they run it: cudaFree waits for the whole device, which a
 * caller driving other streams cannot afford; a framework that has reserved the
 * device memory for its own pool leaves nothing for cudaMalloc; a latency-bound
 * loop may forbid allocation once started.  The paper has no counterpart of
 * this entry point; it exists for those callers.
 * It runs the same sweeps as f2m_gdp (same results, bit for bit), but its
 * scratch (the second lambda buffer, the kernel's control block and the flags
 * of the input check) lives in a fixed file-scope device array of about 1 MiB
 * that every GPU loading this library holds until the process exits.  It calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *   row_ptr   [n+1] int32, device: the candidate CSR (rows as in f2m_create).
 *   ec        [nnz][2] int32, device: per CSR entry {column, cost c_e}.
 *   nnz       entries of ec; 3 n <= nnz < 2^31.
 *   n         4 <= n <= 262,144 (the size of the scratch array); larger n
 *             returns INVALID_ARG with the limit in errbuf.
 *   frac_bits, damping_shift   as in f2m_params (1..8).
 *   lambda    [n] int32, device, in/out: the start lambda, replaced by the
 *             result (units 2^-frac_bits).
 *   sweeps    host out: sweeps run.
 *   bound2    NULL or host out: bound2 at the lambda the last sweep started from.
 *   stream    cudaStream_t as void*, NULL = legacy default stream.
 *   errbuf    NULL or a caller buffer of errlen bytes for a message.
 * Before the sweeps a check kernel reads the inputs (row_ptr over [0, n],
 * ec over [0, nnz) only) and returns INVALID_ARG, with the first offending
 * node in errbuf, unless row_ptr runs from 0 to nnz without decreasing, every
 * column is in [0, n) and not its own row, every row has at least 3 entries,
 * every cost is in [0, 2^(29 - frac_bits)) and every |lambda| < 2^29 (so that
 * Eq. 9's z fits 32 bits).  Symmetry and the order of a row are not checked:
 * they change the answer, not the memory touched.
 * Every call looks up the array's device address on the current device, reuses
 * the same array and clears what must start at zero; calls that overlap on the
 * GPU (other streams or threads) race on it.  The call synchronizes `stream`
 * before it returns.
 * Returns OK, NOT_CONVERGED, OVERFLOW, TIMEOUT, INVALID_ARG, CUDA. */
f2m_status f2m_gdp_noalloc(const int32_t* row_ptr, const int32_t* ec, int64_t nnz, int32_t n,
                           int32_t frac_bits, int32_t damping_shift, int64_t max_sweeps,
                           int32_t* lambda, int64_t* sweeps, int64_t* bound2, void* stream,
                           char* errbuf, int64_t errlen);

/* ---- subtour-elimination cuts ------------------------------------------------
 * The paper's Discussion names F2M plus subtour elimination constraints as the
 * next relaxation for the method.  With cuts the LP is
 *   minimise c x  s.t.  x(delta(v)) = 2 for every node,  x(delta(S)) >= 2 for
 *   every cut S of the context's family,  0 <= x <= 1,
 * Section 2's LP3 with equalities (1) and inequalities (2), every constraint
 * of Section 3's class (8).  A cut dual mu_S >= 0 (Eq. 5) joins the modified
 * objective (Eq. 4): z_uv = c_uv 2^F - lambda_u - lambda_v - the mu_S of the
 * cuts that hold exactly one of u, v.  One Jacobi sweep sets every lambda_v as
 * before and every mu_S = max(0, mu_S + trunc((z(2) + z(3)) / 2^(shift + 2)))
 * with z(2) <= z(3) the 2nd and 3rd smallest z over delta(S) (a quarter of the
 * node step: many duals move a crossing edge at once); the bound becomes
 * bound2 = 4 sum lambda + 4 sum mu + sum over directed entries of min(0, z), a
 * lower bound on the LP with the cuts (on the complete graph once a pricing
 * scan with the same duals finds no pair).
 * The family is kept in up to 8 layers; layer l labels every node -1 or a cut
 * index s in [0, ncuts); the nodes labelled s form one cut (cuts of a layer
 * are disjoint).  While a context holds cuts, f2m_gdp, f2m_extract,
 * f2m_get_bound and f2m_price include them (GDP on a streaming kernel with
 * 64-bit z, f2m_info.gdp_kernel = F2M_GDP_KERNEL_CUTS); lambda stays in units
 * 2^-frac_bits.  f2m_solve refuses (its finisher solves F2M only) and
 * f2m_set_degrees refuses; single-instance contexts only. */

/* One cut layer from the x held now (the last solve's or extraction's): the
 * connected components of its support {e : x_e > 0}, numbered by their
 * smallest node; with m >= 3 components each is a cut, with m = 2 the one
 * without node 0 (delta(S) = delta(V \ S)), with m = 1 none; a component that
 * fewer than 3 candidate edges leave is left out (Section 3's gradient takes a
 * 3rd value).  The layer is not added (see f2m_add_cut_layer).
 *   comp   NULL or [n] int32 (host or device): the labels.
 *   ncuts  out: cuts in the layer (0: the support is connected).
 * Errors: INVALID_ARG, OOM, CUDA. */
f2m_status f2m_separate(f2m_ctx* ctx, int32_t* comp, int32_t* ncuts);

/* Adds a cut layer; its duals start at 0.
 *   comp   [n] int32 (host or device), copied: -1 or a cut index in [0, ncuts).
 *   ncuts  >= 1.
 * Every cut must have at least 3 candidate edges leaving it.  Errors:
 * INVALID_ARG (labels, a short cut, a 9th layer, b_v set, a batch; the context
 * is left as it was), OOM, CUDA. */
f2m_status f2m_add_cut_layer(f2m_ctx* ctx, const int32_t* comp, int32_t ncuts);

/* The cut duals, layer after layer (units 2^-frac_bits).
 *   count   in: capacity of mu; out: number of cuts.
 *   mu      NULL (query) or [count] int32, host or device.
 *   layers  NULL or out: number of layers. */
f2m_status f2m_get_cut_duals(f2m_ctx* ctx, int32_t* mu, int64_t* count, int32_t* layers);

typedef struct {
  int64_t iterations;           /* GDP sweeps, all stages */
  int64_t phases;               /* GDP phases */
  int64_t pricing_rounds;       /* pricing scans */
  int64_t edges_added;          /* undirected edges added by pricing */
  int64_t cuts;                 /* cuts added */
  int64_t bound2_f2m;           /* 2*LB after the first stage (no cuts), units 2^-frac_bits */
  int64_t bound2;               /* 2*LB at the end, units 2^-frac_bits */
  int32_t rounds;               /* separation rounds that added a layer */
  int32_t layers;               /* layers held at the end */
  int32_t frac_bits;
  int32_t certified;            /* 1: the last scan found no pair, so bound2 holds for the complete graph */
  int32_t status;
  int32_t pad;
  double ms_gdp, ms_pricing, ms_merge, ms_separate, ms_total;
} f2m_subtour_info;

/* GDP on F2M with subtour cuts added round by round.  A stage is: a GDP phase
 * (max_iters sweeps at most, or to a fixed point), then a pricing scan; while
 * the scan finds pairs they are added and another phase runs; the stage ends
 * with rule (7) x at the duals reached.  Stage 0 runs from the context's lambda
 * on the cuts it holds; each of the next `rounds` stages (0..8) first adds one
 * layer from f2m_separate on that x (it stops early when the support is
 * connected or 8 layers are held).  No finisher runs: the result is the
 * Lagrangian bound and the duals.  info may be NULL.
 * Errors: INVALID_ARG, OVERFLOW, TIMEOUT, NOT_CONVERGED (pricing rounds), OOM,
 * CUDA. */
f2m_status f2m_solve_subtour(f2m_ctx* ctx, int32_t rounds, f2m_subtour_info* info);

/* ---- batched solves: many independent instances in one context --------------- */

typedef struct f2m_batch f2m_batch;  /* opaque, library-owned */

/* Creates a batch of `count` instances, solved together: every device step of
 * f2m_solve_batch (one persistent GDP launch per phase, with instances that
 * reached their fixed point frozen, for max_iters sweeps at most; one pricing
 * scan over the pair tiles of the
 * instances that need one; one merge; one extraction; one finisher call) covers
 * all instances, and each instance's lambda, x and bound are those of its own
 * f2m_solve (the instances are kept apart as contiguous node ranges).
 *   n        [count] int32, HOST: nodes per instance, each >= 4, sum < 2^24.
 *   xy       [sum n][2] int32, host or device: the points, instance after instance.
 *   row_ptr  [sum (n_i + 1)] int32, host or device: each instance's own row_ptr
 *            (local, starting at 0), back to back.
 *   col      [sum nnz_i] int32, host or device: each instance's columns in its
 *            own numbering, back to back.  Rules per instance as in f2m_create.
 * Errors as f2m_create; the message is in f2m_last_error(NULL). */
f2m_status f2m_create_batch(int32_t count, const int32_t* n, const int32_t* xy,
                            const int32_t* row_ptr, const int32_t* col, const f2m_params* params,
                            void* stream, f2m_batch** out);

/* Solves every instance.  info: NULL or [count] (host) per-instance results
 * (augmentations = -1: counted for the batch only); total: NULL or the batch
 * totals (ms_* for the whole batch, iterations = sum of sweeps, frac_bits = -1).
 * Returns OK when every instance is certified. */
f2m_status f2m_solve_batch(f2m_batch* batch, f2m_info* info, f2m_info* total);

/* Results of instance i after f2m_solve_batch: lambda [n_i] in units
 * 2^-(*frac_bits); the instance's final candidate graph (local numbering) and
 * x in half units, as f2m_get_x.  Pointers host or device. */
f2m_status f2m_batch_get_lambda(f2m_batch* batch, int32_t i, int32_t* lambda, int32_t* frac_bits);
f2m_status f2m_batch_get_x(f2m_batch* batch, int32_t i, int64_t* nnz_inout, int32_t* row_ptr,
                           int32_t* col, uint8_t* x2);
const char* f2m_batch_last_error(const f2m_batch* batch);
void f2m_destroy_batch(f2m_batch* batch);

/* ---- candidate graph and learned warm start ------------------------------------ */

/* Reads a TSPLIB problem (the input of the GD program, Section 5.1) from text
 * in memory: keyword lines, then NODE_COORD_SECTION with one "id x y" line
 * per node (ids 1..DIMENSION, each once, any order), then optionally EOF.
 * EDGE_WEIGHT_TYPE must be EUC_2D and TYPE, if present, TSP; coordinates must
 * be integral (12, 12.0, 1.2e1) with a spread below 2^20 in x and in y.  Host
 * code only (no GPU).
 *   text, len    the file's bytes (not necessarily NUL-terminated).
 *   xy           [cap][2] int32, host, written with the points translated so
 *                that the smallest x and the smallest y are 0; NULL to query
 *                the size only.
 *   n_out        written: DIMENSION.
 *   translation  [2] int64, host, or NULL: the (x, y) that was subtracted.
 * Errors: INVALID_ARG, with the reason in f2m_tsplib_last_error(). */
f2m_status f2m_tsplib_parse(const char* text, int64_t len, int32_t* xy, int32_t cap, int32_t* n_out,
                            int64_t* translation);
/* The reason of the last f2m_tsplib_parse failure on this thread ("" if none). */
const char* f2m_tsplib_last_error(void);

/* k nearest neighbours of every point (the top-N nearest-neighbour candidate
 * graph of Section 5.3): the k other points with the smallest exact squared
 * distance dx^2 + dy^2 (int64), ties broken by smaller index; a copy of the
 * point (distance 0) counts, the point itself does not.
 *   xy      [n][2] int32, host or device; coordinates in [0, 2^20).
 *   n, k    1 <= k <= 32, n > k.
 *   nbr     [n][k] int32, host or device (caller-owned): row v lists v's
 *           neighbours nearest first.
 *   d2      NULL or [n][k] int64, host or device: their squared distances.
 *   stream  cudaStream_t as void*.
 * Errors: INVALID_ARG, OOM, CUDA (message in f2m_last_error(NULL)). */
f2m_status f2m_knn(const int32_t* xy, int32_t n, int32_t k, int32_t* nbr, int64_t* d2, void* stream);

/* The symmetrised k-NN candidate CSR that f2m_create takes: u ~ w when either
 * lists the other among its k nearest; rows sorted ascending.
 *   row_ptr  [n+1] int32, host or device.
 *   col      [2 n k] int32 (capacity), host or device; the first *nnz used.
 *   nnz      host out: entries written.
 * Errors: INVALID_ARG, OOM, CUDA. */
f2m_status f2m_knn_csr(const int32_t* xy, int32_t n, int32_t k, int32_t* row_ptr, int32_t* col,
                       int64_t* nnz, void* stream);

/* Features of the learned warm start: for node v the distances to its 16
 * nearest other points (as f2m_knn), ascending, divided by
 * s_v = max(1, their mean).
 *   feat   [n][16] float, host or device.   scale  [n] float: s_v.
 * Needs n > 16.  Errors: INVALID_ARG, OOM, CUDA. */
f2m_status f2m_features(const int32_t* xy, int32_t n, float* feat, float* scale, void* stream);

/* The warm-start network: 16 -> 128 -> 128 -> 1 with ReLU after both hidden
 * layers; it predicts lambda_v / s_v from the features of v.  The paper lets
 * the iteration start anywhere (Section 3); GDP from the predicted start is the
 * same exact method and certifies the same optimum.  Products run on the
 * tensor cores with bfloat16 inputs (features, W1, W2, the first hidden layer,
 * and in training the hidden-layer gradients, the second hidden layer and
 * dL/dy) and fp32 accumulation; master weights are fp32.
 * Parameter vector (float [F2M_MLP_NPARAMS]): W1 [128][16] (output-major),
 * b1 [128], W2 [128][128], b2 [128], w3 [128], b3. */
#define F2M_MLP_NPARAMS 18817
typedef struct f2m_mlp f2m_mlp;   /* opaque, library-owned */

/* params: [F2M_MLP_NPARAMS] float, host or device (copied).  All work of the
 * network runs on `stream`.  Errors: INVALID_ARG (NULL or a non-finite value),
 * OOM, CUDA (message in f2m_last_error(NULL)). */
f2m_status f2m_mlp_create(const float* params, void* stream, f2m_mlp** out);
void f2m_mlp_destroy(f2m_mlp* mlp);
/* Current fp32 parameters into out [F2M_MLP_NPARAMS] (host or device). */
f2m_status f2m_mlp_get_params(f2m_mlp* mlp, float* out);
const char* f2m_mlp_last_error(const f2m_mlp* mlp);

/* Network output y [count] for features [count][16] (both host or device). */
f2m_status f2m_mlp_forward(f2m_mlp* mlp, const float* feat, int64_t count, float* y);

/* Loss L = mean over the count samples of (y - target)^2 and its gradient with
 * respect to the parameters (grad [F2M_MLP_NPARAMS], loss: one float; host or
 * device).  One forward and backward pass, no update.  count >= 1. */
f2m_status f2m_mlp_grad(f2m_mlp* mlp, const float* feat, const float* target, int64_t count,
                        float* grad, float* loss);

typedef struct {
  int32_t epochs;        /* passes over the samples */
  int32_t batch;         /* samples per Adam step (>= 128) */
  float lr;              /* Adam step size of the first step */
  float lr_final_frac;   /* step size decays linearly to lr * lr_final_frac at the last step */
  float beta1, beta2, eps;
  uint64_t seed;         /* sample order: a fresh SplitMix64-keyed shuffle per epoch */
} f2m_train_params;

/* Trains the network in place with Adam (Kingma and Ba) on mean squared error:
 * each epoch shuffles the samples and takes ceil(count / batch) steps.
 *   feat [count][16], target [count]: host or device.
 *   epoch_loss  NULL or [epochs] float (host): mean loss of each epoch.
 * Adam's moments and step count carry over between calls. */
f2m_status f2m_mlp_train(f2m_mlp* mlp, const float* feat, const float* target, int64_t count,
                         const f2m_train_params* tp, float* epoch_loss);

/* Warm start of a context: features of its points, the network, and
 * lambda0_v = rint(2^F * s_v * y_v), clamped to |lambda0| <= 2^27, set as the
 * context's lambda (units 2^-F).  Runs on the context's stream.
 *   ms  NULL or out: device time of the features, network and rounding.
 * Errors: INVALID_ARG (n <= 16), OOM, CUDA, TIMEOUT. */
f2m_status f2m_warm_start(f2m_ctx* ctx, f2m_mlp* mlp, double* ms);

/* ---- results ----------------------------------------------------------------- */

/* lambda [n] int32 (host or device) in units 2^-(*frac_bits). */
f2m_status f2m_get_lambda(f2m_ctx* ctx, int32_t* lambda, int32_t* frac_bits);

/* bound2 = 2*LB at the current lambda, in units 2^-(*frac_bits). */
f2m_status f2m_get_bound(f2m_ctx* ctx, int64_t* bound2, int32_t* frac_bits);

/* The current candidate graph and x of the last solve (or extraction).
 *   nnz_inout  in: capacity of col/x2; out: entries needed.  Call with NULL
 *              arrays to query the size (it grows with pricing).
 *   row_ptr    NULL or [n+1] int32;  col  NULL or [nnz] int32;
 *   x2         NULL or [nnz] uint8 (0, 1, 2 = x of 0, 1/2, 1);
 *   cost       NULL or [nnz] int32: c_e of each entry.
 * All host or device.  INVALID_ARG if the capacity is too small. */
f2m_status f2m_get_x(f2m_ctx* ctx, int64_t* nnz_inout, int32_t* row_ptr, int32_t* col,
                     uint8_t* x2, int32_t* cost);

/* Number of kernel launches this library has made in this process (all
 * contexts, all threads).  A diagnostic with no counterpart in the paper. */
int64_t f2m_kernel_launches(void);

/* Checks, on the current device, the tensor-core arithmetic that the full
 * pricing scan's filter relies on (fp16 operands, fp32 accumulator, results
 * that must be exact integers): `rounds` products of 128 x 128 pairs of
 * operand rows drawn from `seed` within the ranges the filter produces, each
 * accumulator value compared with the exact integer product.  *checked: the
 * values compared; *mismatches: those that differ.  Runs on the legacy default
 * stream and synchronizes it.  A diagnostic with no counterpart in the paper.
 * Returns F2M_OK, F2M_ERR_INVALID_ARG (NULL output, rounds < 0), F2M_ERR_CUDA
 * or F2M_ERR_TIMEOUT (an mbarrier wait gave up). */
f2m_status f2m_pricing_mma_check(int64_t rounds, uint64_t seed, int64_t* checked, int64_t* mismatches);

/* Static text for a status code. */
const char* f2m_status_string(f2m_status s);

/* Message of the last failure on ctx (or of the last failed f2m_create when
 * ctx is NULL); "" if none.  Valid until the next call on the same context. */
const char* f2m_last_error(const f2m_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* F2M_H */
