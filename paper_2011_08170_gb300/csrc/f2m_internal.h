// Internal declarations of the f2m library (not part of the C ABI).
//
// Device data layout (one instance, n nodes, nnz directed CSR entries):
//   xy    int2[n]          point coordinates, each in [0, 2^20)
//   rp    int32[n+1]       CSR row offsets (both directions of every edge stored)
//   ec    int2[nnz]        per entry {col, cost}: 8 bytes streamed per entry
//   lam   int32[2][n]      lambda, Jacobi double buffer (units 2^-F)
//   lam2  int32[n]         lambda of the finisher (units 2^-(F+1))
//   x2    uint8[nnz]       primal x in half units
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace f2m {

constexpr int32_t kCoordLimit = 1 << 20;   // coordinates in [0, 2^20)
constexpr int64_t kLamLimit = 1LL << 29;   // |lambda| < 2^29 in units 2^-F
constexpr int kMaxCutLayers = 8;           // layers of subtour-elimination cuts (cuts.cu)

// Control block of the persistent GDP kernel (device memory, zeroed per phase).
struct GdpCtl {
  unsigned int bar_count;      // arrivals at the current barrier
  unsigned int bar_gen;        // barrier generation
  int status;                  // bit 0: lambda overflow, bit 1: barrier timeout
  int fixed_point;             // 1 if the last sweep changed no lambda
  long long slot_b2[3];        // per-sweep bound2 accumulators (ring of 3)
  unsigned long long slot_ch[3];  // per-sweep changed counts (ring of 3)
  long long sweeps;            // sweeps completed
  long long pad1;
  // ring of 4 per-sweep slots used by the tiled kernel (stop test lagged by two sweeps)
  long long q_b2[4];
  unsigned long long q_ch[4];
  int q_ovf[4];
};

constexpr int kGdpOverflow = 1;
constexpr int kGdpTimeout = 2;
constexpr int kGdpOddOverflow = 4;  // two-sweep kernel: the second sweep of a round overflowed

// Validation result written by the create-time check kernel.
struct CheckCtl {
  int flags;                   // bit set per violated rule
  int first_bad;               // smallest offending node (or entry)
};

enum CheckBits {
  kBadRowPtr = 1,
  kBadCol = 2,
  kUnsorted = 4,
  kSelfLoop = 8,
  kAsymmetric = 16,
  kLowDegree = 32,
  kBadCoord = 64,
  kBadPair = 128,
  kBadDegreeReq = 256,
};

// Device memory of this library (api.cu): a process-wide cache of freed
// blocks per device.  dev_free waits for the device (as cudaFree does) before
// the block can be handed out again; dev_free_synced is for a caller that has
// already waited for every use of the block.
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
void dev_free_synced(void* p);
// waits for the device once; while it lives, dev_free on this thread waits no more
struct DevSyncedScope {
  DevSyncedScope();
  ~DevSyncedScope();
};

// process-wide count of kernel launches made by this library (api.cu)
void count_launch();
void count_launches(long long k);  // k launches replayed from a captured graph

// ---- launchers (each enqueues on `st`) -------------------------------------

// validation of the input CSR and points; ctl must be zeroed (first_bad = INT_MAX)
cudaError_t launch_check(const int2* xy, const int32_t* rp, const int32_t* col, int32_t n,
                         int64_t nnz, CheckCtl* ctl, cudaStream_t st);
// coordinates in [0, 2^20) (flag kBadCoord); ctl zeroed with first_bad = INT_MAX
cudaError_t launch_check_points(const int2* xy, int32_t n, CheckCtl* ctl, cudaStream_t st);
// degree requirements 1 <= b_v <= deg(v) - 1 (flag kBadDegreeReq); the
// largest b_v into *bmax (zeroed by the caller)
cudaError_t launch_check_degrees(const int32_t* rp, const int32_t* bdeg, int32_t n, CheckCtl* ctl,
                                 unsigned long long* bmax, cudaStream_t st);
// ec[e] = {col[e], c(row(e), col[e])}
cudaError_t launch_build_ec(const int2* xy, const int32_t* rp, const int32_t* col, int32_t n,
                            int2* ec, cudaStream_t st);
// one persistent cooperative GDP phase; bdeg: degree requirements b_v in
// caller order (NULL: b_v = 2, the fractional 2-matching) -- likewise below
// (bmax: the largest b_v, which picks the selection method)
cudaError_t launch_gdp(const int32_t* rp, const int2* ec, const int32_t* bdeg, int32_t bmax,
                       int32_t* lam0, int32_t* lam1, int32_t n, int32_t F, int32_t shift,
                       int64_t max_sweeps, GdpCtl* ctl, long long* trace_b2,
                       unsigned long long* trace_ch, int64_t trace_cap, long long budget,
                       int num_sms, cudaStream_t st);
// bound2 at lam with fb fractional bits, into *out (zeroed by the launcher)
cudaError_t launch_bound(const int32_t* rp, const int2* ec, const int32_t* bdeg, const int32_t* lam,
                         int32_t n, int32_t fb, long long* out, cudaStream_t st);
// rule (7) extraction; *bad zeroed by the launcher
cudaError_t launch_extract(const int32_t* rp, const int2* ec, const int32_t* bdeg, const int32_t* lam,
                           int32_t n, int32_t fb, uint8_t* x2, unsigned long long* bad,
                           cudaStream_t st);
// lam_out = lam_in >> 1 (F+1 bits -> F bits, floor)
cudaError_t launch_halve(const int32_t* lam_in, int32_t* lam_out, int32_t n, cudaStream_t st);
// all-pairs pricing scan: pairs (u < v) outside the CSR with z < 0
// Tile pairs {i0, i1, j0, j1}: test i in [i0, i1) against j in [j0, j1), j > i.
constexpr int kPricingTile = 1024;  // i-points of a pricing tile pair (and the most j-points)
constexpr int kPricingJ = 512;      // j-points of a tile pair in the lists built for a scan
// pts[v] = {x, y, s, node perm[v]} (perm NULL: node v), s the filter radius of the node
cudaError_t launch_pricing_prep(const int2* xy, const int32_t* lam, const int32_t* perm, int32_t n, int32_t fb,
                                float4* pts, cudaStream_t st);
// bounding box {min x, min y, max x, max y} and largest s of each point range
cudaError_t launch_pricing_boxes(const float4* pts, const int2* ranges, int32_t nranges, float4* box, float* smax,
                                 cudaStream_t st);
// the scan over the tile pairs (positions in pts); count and pairs (nodes, u < v)
// tiles NULL: i-tiles of the ni points pts_i against j-tiles of all n points
// (inU flags the nodes of pts_i; ntiles = its tile count), else the list's
// tile pairs over pts (pts_i NULL)
cudaError_t launch_pricing_scan(const float4* pts, const int2* xy, const int32_t* lam, const int32_t* rp,
                                const int2* ec, int32_t n, int32_t fb, const int4* tiles, int32_t ntiles,
                                int2* pairs, int64_t cap, unsigned long long* count, unsigned int* tile_counter,
                                int num_sms, cudaStream_t st, const float4* pts_i = nullptr,
                                const uint8_t* inU = nullptr, int32_t ni = 0);
// nodes whose lambda rose above lam_ref << shift: flags, their points, their count
cudaError_t launch_pricing_raised(const int32_t* lam, const int32_t* lam_ref, int32_t n, int32_t shift,
                                  const float4* pts, uint8_t* inU, float4* pts_u, unsigned int* count,
                                  cudaStream_t st);
// the same scan on the tensor cores (pricing.cu): pts4[v] = {x, y, lambda, node
// perm[v]}; tiles {i0, i1, j0, j1} of at most kMmaTileI x kMmaTileJ positions
cudaError_t launch_pricing_mma_check(long long rounds, unsigned long long seed, unsigned long long* checked,
                                     unsigned long long* mismatches, int32_t* status, cudaStream_t st);
constexpr int kMmaTileI = 128;
constexpr int kMmaTileJ = 128;
cudaError_t launch_pricing_mma_prep(const int2* xy, const int32_t* lam, const int32_t* perm, int32_t n,
                                    int4* pts4, cudaStream_t st);
// ranges [nblocks]: the 128-point blocks; tblk [ntiles]: each tile pair's
// blocks {i-block, j-block, second j-block or -1}; box, lmax, frames: scratch;
// cand [cand_cap]: the filter's candidates (*ncand of them, more than
// cand_cap when the list overflowed: the scan is then incomplete)
cudaError_t launch_pricing_mma_scan(const int4* pts4, const int2* xy, const int32_t* lam, const int32_t* rp,
                                    const int2* ec, int32_t fb, const int4* tiles, const int4* tblk,
                                    int32_t ntiles, const int2* ranges, int32_t nblocks, int4* box, int32_t* lmax,
                                    int4* frames, int2* cand, int64_t cand_cap, unsigned long long* ncand,
                                    int2* pairs, int64_t cap, unsigned long long* count,
                                    unsigned int* tile_counter, int32_t* status, int num_sms, cudaStream_t st);
// CSR union with pairs; sizes: see graph.cu.  Returns the new nnz through *new_nnz_dev.
struct MergeBuffers {
  int32_t* deg;        // [n+1]
  int32_t* tmp_rp;     // [n+1]
  int32_t* tmp_col;    // [nnz + 2*npairs]
  int32_t* new_rp;     // [n+1]
  int32_t* block_sums; // scan scratch
  CheckCtl* ctl;
};
cudaError_t launch_merge_count(const int32_t* rp, const int2* pairs, int64_t npairs, int32_t n,
                               MergeBuffers& mb, cudaStream_t st);
cudaError_t launch_merge_fill(const int32_t* rp, const int2* ec, const int2* pairs, int64_t npairs,
                              int32_t n, MergeBuffers& mb, cudaStream_t st);
// ec_out: another array than ec_in (untouched rows are copied from ec_in)
cudaError_t launch_merge_finish(const int2* xy, const int32_t* rp, const int2* ec_in, int32_t n,
                                MergeBuffers& mb, int2* ec_out, cudaStream_t st);
// exclusive scan of in[0..m) into out[0..m], out[m] = total (m+1 outputs)
cudaError_t launch_scan(const int32_t* in, int32_t* out, int32_t m, int32_t* block_sums,
                        cudaStream_t st);
size_t scan_scratch_ints(int32_t m);
// split ec into col / cost arrays
cudaError_t launch_split_ec(const int2* ec, int64_t nnz, int32_t* col, int32_t* cost,
                            cudaStream_t st);

// ---- class-by-class GDP (gdp_classes.cu) ------------------------------------------
// greedy colouring of the caller-order CSR and the nodes grouped by class
struct ClassPlan {
  int32_t* color = nullptr;      // [n] colour of each node
  int32_t* order = nullptr;      // [n] nodes grouped by class
  int32_t* off = nullptr;        // [ncolors+1] class offsets into order
  unsigned int* ctl = nullptr;   // round counters
  int32_t cap = 0;
  int32_t ncolors = 0;
  int32_t rounds = 0;            // Jones-Plassmann rounds of the last colouring
  int64_t version = -1;          // GdpPlan::version of the graph coloured
  std::vector<int32_t> h_off;
};
cudaError_t color_classes(const int32_t* rp, const int2* ec, int32_t n, ClassPlan& cp,
                          cudaStream_t st);
void class_plan_free(ClassPlan& cp);
// one class-by-class phase, lambda updated in place (bdeg / bmax as launch_gdp)
cudaError_t launch_gdp_classes(const int32_t* rp, const int2* ec, const int32_t* bdeg, int32_t bmax,
                               int32_t* lam, const ClassPlan& cp, int32_t n, int32_t F,
                               int32_t shift, int64_t max_sweeps, GdpCtl* ctl, long long* trace_b2,
                               unsigned long long* trace_ch, int64_t trace_cap, long long budget,
                               int num_sms, cudaStream_t st);

// ---- shared-memory tiled GDP (gdp_tiled.cu) ----------------------------------------
// Spatial renumbering and per-CTA plan; see gdp_tiled.cu.
struct GdpPlan {
  int32_t n = 0;
  int64_t nnz = 0;               // entries of the internal CSR
  int64_t version = 0;           // bumped whenever the internal CSR is rebuilt
  bool valid = false;            // the tiled kernel can run this CSR
  int32_t B = 0, threads = 0;    // CTAs (one node range each) and threads per CTA
  int32_t maxO = 0, maxS = 0, maxH = 0;  // max own nodes, sliced entries, halo per CTA
  int32_t halo_total = 0;
  size_t smem = 0;               // dynamic shared memory per CTA
  int32_t* perm = nullptr;       // internal -> caller node
  int32_t* inv = nullptr;        // caller -> internal node
  int32_t* irp = nullptr;        // internal CSR offsets
  int2* iec = nullptr;           // internal {col, cost}
  int2* lec = nullptr;           // sliced {local index, cost * 2^F} per CTA
  int32_t* scount = nullptr;     // [B+1] sliced entries per CTA
  int32_t* soff = nullptr;       // [B+1] their offsets
  int32_t* order = nullptr;      // [n] node of each slot (degree-descending per CTA)
  int2* slc = nullptr;           // [n] per-CTA slice table {offset, depth}
  int32_t* part = nullptr;       // [B+1] node range of each CTA
  int32_t* hoff = nullptr;       // [B+1] halo offsets
  int32_t* hcount = nullptr;
  int32_t* halo = nullptr;       // halo node ids (internal)
  int32_t* tmp = nullptr;
  int32_t* stats = nullptr;
  int32_t* ilam[3] = {nullptr, nullptr, nullptr};  // lambda in internal order (ring of 3)
  uint64_t* keys = nullptr;
  uint64_t* keys2 = nullptr;
  int32_t* idx = nullptr;
  void* sort_tmp = nullptr;
  int32_t* scan_tmp = nullptr;
  int64_t irp_cap = 0, iec_cap = 0, lec_cap = 0, tmp_cap = 0, halo_cap = 0, scan_cap = 0;
  int64_t order_cap = 0, slc_cap = 0;
  int64_t cta_cap = 0;           // entries of part, hcount, scount, soff, hoff
  int64_t ilam_cap[3] = {0, 0, 0};
  // two-sweep form (gdp_tiled2.cu): H1 rows and the H2 ring per CTA
  bool valid2 = false;
  int32_t maxS2 = 0, maxSl2 = 0, maxL2 = 0, maxHH2 = 0;  // max sliced entries, slices, lambda slots, halo
  size_t smem2 = 0;
  int32_t* h2count = nullptr;    // [B+1] H2 per CTA
  int32_t* hhcount = nullptr;    // [B+1] H1 + H2 per CTA
  int32_t* s2count = nullptr;    // [B+1] sliced entries (own + H1 rows)
  int32_t* nslc = nullptr;       // [B+1] slices (own + H1)
  int32_t* hoff2 = nullptr;      // [B+1] offsets of the H1|H2 lists
  int32_t* soff2 = nullptr;      // [B+1] offsets of the sliced entries
  int32_t* sloff2 = nullptr;     // [B+1] slice offsets
  int32_t* halo2 = nullptr;      // H1 then H2 node ids per CTA
  int32_t* order2 = nullptr;     // local node of each slot
  int2* slc2 = nullptr;          // {offset, depth} per slice
  int2* lec2 = nullptr;          // sliced {local index, cost * 2^F}
  uint32_t* lec2p = nullptr;     // the same packed as cost << 13 | local index (packed2)
  int64_t lec2p_cap = 0;
  bool packed2 = false;          // the kernel reads lec2p (the 8-byte tiles do not fit)
  int32_t frac_bits2 = 8;        // F the entries were built with
  int32_t* tmp2 = nullptr;       // H2 lists during the build
  int32_t* stats2 = nullptr;
  int64_t cap2_small = 0, halo2_cap = 0, order2_cap = 0, slc2_cap = 0, lec2_cap = 0, tmp2_cap = 0;
};
cudaError_t sort_pairs_u64(void* temp, size_t& temp_bytes, const uint64_t* keys_in,
                           uint64_t* keys_out, const int32_t* vals_in, int32_t* vals_out,
                           int32_t count, int end_bit, cudaStream_t st);
// Morton renumbering inside each segment [seg_off[s], seg_off[s+1]) (segments stay contiguous)
cudaError_t plan_renumber(const int2* xy, int32_t n, const std::vector<int32_t>& seg_off, GdpPlan& p,
                          cudaStream_t st);
// internal CSR (always) and, if `tiles`, the per-CTA tiles of the shared-memory kernel
cudaError_t plan_build(const int32_t* rp, const int2* ec, int32_t n, int64_t nnz, int num_sms,
                       bool tiles, int32_t F, int32_t ctas_per_sm, GdpPlan& p, cudaStream_t st);
// the per-CTA tiles alone, for the internal CSR plan_build made last
cudaError_t plan_build_tiles(int num_sms, int32_t F, int32_t ctas_per_sm, GdpPlan& p, cudaStream_t st);
// dst[i] = src[perm[i]]  /  dst[perm[i]] = src[i]
cudaError_t gather_perm(const int32_t* src, const int32_t* perm, int32_t n, int32_t* dst,
                        cudaStream_t st);
cudaError_t scatter_perm(const int32_t* src, const int32_t* perm, int32_t n, int32_t* dst,
                         cudaStream_t st);
void plan_free(GdpPlan& p);
// gathers lam_in (caller order) into ilam[0], then one cooperative tiled launch
cudaError_t launch_gdp_tiled(GdpPlan& p, const int32_t* lam_in, int32_t shift, int64_t max_sweeps,
                             GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
                             int64_t trace_cap, long long budget, cudaStream_t st);
// two-sweep form on top of a valid one-sweep plan of 1024-thread CTAs (valid2 false if it does not fit)
cudaError_t plan_build2(GdpPlan& p, int32_t F, cudaStream_t st);
void plan2_free(GdpPlan& p);
// gathers lam_in into ilam[0], one cooperative launch; the result is in ilam[ctl->pad1].
// bint: degree requirements in internal order (NULL: b_v = 2), bmax their largest
cudaError_t launch_gdp_tiled2(GdpPlan& p, const int32_t* lam_in, int32_t shift, int64_t max_sweeps, GdpCtl* ctl,
                              long long* trace_b2, unsigned long long* trace_ch, int64_t trace_cap,
                              long long budget, const int32_t* bint, int32_t bmax, cudaStream_t st);
// lam_out (caller order) = ilam[which]
cudaError_t plan_scatter_lambda(const GdpPlan& p, int which, int32_t* lam_out, cudaStream_t st);

// ---- exact finisher (finisher_prep.cu on the device, finisher.cpp on the host) ---
// twin[e] for every internal entry; *missing (zeroed by the caller) counts
// entries without a reverse entry
cudaError_t fin_build_twin(const GdpPlan& p, int32_t* twin, unsigned long long* missing, cudaStream_t st);
// bdeg_caller: degree requirements in caller order (NULL: 2)
cudaError_t fin_prepare(const GdpPlan& p, const int32_t* lam_caller, const int32_t* bdeg_caller,
                        int32_t F, int32_t* lam_int, uint8_t* y, int32_t* exl, cudaStream_t st);
// x (half units, caller order) = y[e] + y[twin[e]] of the final flow; lambda
// at F+1 bits to caller order.  include (device, per segment; NULL = all): x
// of excluded segments is kept
cudaError_t fin_scatter(const GdpPlan& p, const int32_t* rp, const uint8_t* y_int,
                        const int32_t* twin, const int32_t* lam2_int, uint8_t* x_out,
                        int32_t* lam2_out, const int32_t* seg_off, int32_t nseg,
                        const uint8_t* include, cudaStream_t st);
// ---- batched GDP on thread-block clusters (gdp_cluster.cu) ------------------------
struct ClusterInst {
  int32_t node0;  // first internal node of the instance
  int32_t n;      // its nodes
  int32_t per;    // nodes per CTA (the last CTAs may hold fewer, or none)
  int32_t seg;    // instance id
};
struct ClusterOut {
  long long sweeps;
  int status;     // kGdpOverflow bit
  int fixed;      // 1 if the last sweep changed nothing
};
constexpr int kClusterNodes = 2048;      // most nodes one CTA holds
constexpr int kClusterEntries = 24000;   // most entries one CTA holds
size_t cluster_smem(int32_t emax, int32_t nmax);
// pk[e] = {owner rank << 16 | local index, cost << F} for the listed instances' entries
cudaError_t cluster_pack(const int32_t* irp, const int2* iec, const ClusterInst* d_insts, int32_t ninst,
                         int32_t F, int2* pk, cudaStream_t st);
// one cluster of C CTAs per listed instance; ilam (internal order) in and out; out zeroed
cudaError_t launch_gdp_cluster(int32_t C, int32_t threads, const int32_t* irp, const int2* pk,
                               const ClusterInst* d_insts, int32_t ninst, int32_t* ilam,
                               int32_t shift, int64_t max_sweeps, ClusterOut* out,
                               int32_t emax, int32_t nmax, cudaStream_t st);
// clusters of this shape that fit on the device at once (0: none)
int32_t cluster_max_smem_ok(int32_t C, int32_t threads, int32_t emax, int32_t nmax);

// ---- batched solver (batch_kernels.cu) --------------------------------------------
// Parameters of one launch of a batched GDP kernel, read from device memory so
// that a captured launch can be replayed with new values.
struct BatchChunk {
  int32_t ntiles;        // tiles in the list (those of the instances still active)
  int32_t pad;
  long long t_base;      // sweeps run by earlier launches of this phase
  long long max_sweeps;  // sweeps this launch may run
};
// tiles {first node, end node, segment, first entry} over the renumbered CSR
// with their end entries in tiles_e1; one cooperative launch of G CTAs of the
// given shape (see batch_kernels.cu); max_tiles sizes the per-CTA tile table
int batch_num_shapes();
// lambda of the buffer a batch GDP phase ended in, scattered to caller order
cudaError_t launch_batch_scatter_final(const int32_t* lam0, const int32_t* lam1, const GdpCtl* ctl,
                                       const int32_t* perm, int32_t n, int32_t* dst, cudaStream_t st);
int batch_shape_blocks(int shape, int mcap);  // CTAs per SM, 0 if the shape does not run
int batch_shape_tile(int shape, int* te, int* tn);  // tile entries and nodes of a shape
int batch_shape_units(int shape);  // tile owners per CTA: 1 (CTA form) or its warps (warp form)
cudaError_t launch_gdp_batch(int shape, const int32_t* irp, const int2* iec, const int4* tiles,
                             const int32_t* tiles_e1, const BatchChunk* chunk, int32_t max_tiles, int32_t G,
                             int32_t nseg, uint8_t* active, unsigned long long* seg_ch, long long* seg_sweeps,
                             int32_t* lam0, int32_t* lam1, int32_t F, int32_t shift, GdpCtl* ctl,
                             long long budget, cudaStream_t st);
cudaError_t launch_batch_extract_bound(const int32_t* rp, const int2* ec, const int32_t* lam,
                                       int32_t n, int32_t fb, const int32_t* seg_off, int32_t nseg,
                                       uint8_t* x2, long long* seg_b2, unsigned long long* seg_bad,
                                       const uint8_t* seg_write, cudaStream_t st);
cudaError_t launch_batch_union(const int32_t* rp_local, const int32_t* col_local,
                               const int32_t* seg_off, const int32_t* eoff, int32_t nseg, int32_t n,
                               int64_t nnz, int32_t* rp, int32_t* col, CheckCtl* ctl,
                               cudaStream_t st);
cudaError_t launch_batch_mask_surplus(int32_t* exl, const int32_t* seg_off, int32_t nseg,
                                      const uint8_t* include, int32_t n, cudaStream_t st);
// out[s] = rp[seg_off[s]], s = 0..nseg
cudaError_t launch_batch_seg_entry(const int32_t* rp, const int32_t* seg_off, int32_t nseg, int32_t* out,
                                   cudaStream_t st);
// results of the instances flagged in done (device mask) into the arenas, entries at eoff[s]
cudaError_t launch_batch_snapshot(const uint8_t* done, const int32_t* seg_off, int32_t nseg, const int32_t* rp,
                                  const int32_t* lam, const int2* ec, const uint8_t* x2, const long long* eoff,
                                  int32_t* res_lam, int32_t* res_rp, int2* res_ec, uint8_t* res_x2,
                                  cudaStream_t st);

struct FinisherWork;
FinisherWork* finisher_work_new();
// lets up to `threads` - 1 worker threads of the host finisher poll for a job
// that is about to come (a finisher call after some device work), so that the
// call does not wait for them to wake
void finisher_pool_wake(int32_t threads);
void finisher_work_reserve(FinisherWork* w, int32_t n);  // host work arrays for n nodes
void finisher_work_free(FinisherWork* w);
// Min-cost flow on the bipartite double cover, internal node order; see
// finisher.cpp.  y is the initial flow (updated to the optimal one), exl the
// left surpluses, lam2 receives pi(L) - pi(R) (F+1 bits).  Blocks and segments
// [seg_off[s], seg_off[s+1]) go to up to `threads` host threads; with include
// (per segment; NULL = all) the other segments are neither read nor written.
// Returns 0 ok, 7 infeasible, 5 overflow.
// time and augmentations of the finisher, summed over its calls
struct FinisherStats {
  double ms_prep = 0, ms_phase[3] = {0, 0, 0}, ms_scatter = 0;
  int64_t aug[3] = {0, 0, 0};
  int32_t threads = 0;
  int32_t phase1_gpu = 0;  // 1 if phase 1 ran on the GPU
};
// ext_pi / ext_ex (NULL: none): potentials [2n] and surpluses [2n] that phase
// 1 left when it ran on the GPU; the host then runs phases 2 and 3 only (the
// augmentations it reports are its own)
int host_finisher(int32_t n, const int32_t* irp, const int2* iec, const int32_t* twin, uint8_t* y,
                  const int32_t* exl, const int32_t* lam, int32_t F, int32_t* lam2,
                  const int32_t* seg_off, int32_t nseg, const uint8_t* include, int32_t threads,
                  int64_t* augmentations, FinisherWork* w, FinisherStats* stats, int64_t* ext_pi = nullptr,
                  int32_t* ext_ex = nullptr);
// the finisher's phase 1 on the GPU (finisher_gpu.cu): one warp per block
size_t fin_heap_item_bytes();
cudaError_t launch_fin_block_caps(const int2* blocks, int32_t nblocks, const int32_t* irp, long long* caps,
                                  cudaStream_t st);
cudaError_t launch_fin_blocks(int32_t n, const int2* blocks, int32_t nblocks, const int32_t* irp, const int2* iec,
                              const int32_t* twin, uint8_t* y, const int32_t* exl, const int32_t* lam, int32_t F,
                              long long* pi, long long* dist, int32_t* excess, int32_t* via, int32_t* pred,
                              uint32_t* reached, uint32_t* closed, void* heaps, const long long* heap_off,
                              int32_t* orders, long long* pushes, int32_t* status, long long budget,
                              cudaStream_t st);
constexpr int32_t kFinBlockNodes = 2048;  // nodes per block of the finisher's phase 1 (host and GPU)
// lam_out = 2 * lam_in (F bits -> F+1 bits)
cudaError_t launch_double(const int32_t* lam_in, int32_t* lam_out, int32_t n, cudaStream_t st);


// ---- k nearest neighbours and warm-start features (knn.cu) -------------------------
constexpr int kKnnMax = 32;    // largest k of the k-NN kernel
constexpr int kFeatures = 16;  // neighbour distances per node in the warm-start features
// exact k-NN lists (ties by index): nbr [n][k], d2 [n][k] (may be NULL); device pointers
cudaError_t knn_device(const int2* d_xy, int32_t n, int32_t k, int32_t* d_nbr, long long* d_d2,
                       cudaStream_t st);
// symmetrised k-NN CSR; d_col holds up to 2 n k entries; *nnz_out on the host (synchronises)
cudaError_t knn_csr_device(const int2* d_xy, int32_t n, int32_t k, int32_t* d_row_ptr, int32_t* d_col,
                           int64_t* nnz_out, cudaStream_t st);
// feat [n][16] = sorted 16-NN distances / s, s = max(1, their mean)
cudaError_t features_device(const int2* d_xy, int32_t n, float* d_feat, float* d_scale, cudaStream_t st);

// ---- warm-start network (mlp.cu) ----------------------------------------------------
// flat fp32 parameters: W1 [128][16], b1 [128], W2 [128][128], b2 [128], w3 [128], b3
constexpr int kOW1 = 0, kOb1 = 2048, kOW2 = 2176, kOb2 = 18560, kOw3 = 18688, kOb3 = 18816;
constexpr int kMlpParams = 18817;
constexpr int kImgW1Bytes = 128 * 16 * 2;   // bf16 operand image of W1
constexpr int kImgW2Bytes = 128 * 128 * 2;  // bf16 operand image of W2 (and of W2^T)
constexpr int kMlpImgBytes = kImgW1Bytes + 2 * kImgW2Bytes;
constexpr int kLambda0Limit = 1 << 27;      // |lambda0| clamp of the warm start
struct MlpAdam {
  float lr, beta1, beta2, eps, lr_final_frac;
  long long total_steps;  // linear decay of lr to lr * lr_final_frac over this many steps
  long long log_base;     // the loss of step t goes to loss_log[t - 1 - log_base]
};
cudaError_t mlp_pack(const float* master, uint8_t* img, cudaStream_t st);
int mlp_grid(int num_sms, long long count);
cudaError_t mlp_forward(const uint8_t* img, const float* master, const float* feat, long long count,
                        float* y, const float* scale, int32_t* lam, int32_t F, int num_sms, int* status,
                        cudaStream_t st);
cudaError_t mlp_train_launch(const uint8_t* img, const float* master, const float* feat, const float* target,
                             const int32_t* perm, long long s0, long long count, float two_over_b,
                             float* partial, int grid, long long* step_ctr, int* status, cudaStream_t st);
cudaError_t mlp_reduce_launch(const float* partial, int nparts, float* grad, float* master, float* m1,
                              float* m2, uint8_t* img, const long long* step_ctr, const MlpAdam& hp,
                              float* loss_log, cudaStream_t st);
cudaError_t mlp_perm_keys(uint64_t key, long long n, uint64_t* keys, int32_t* idx, cudaStream_t st);
}  // namespace f2m
