// Internal view of the f2m context, shared by the translation units that drive
// it (api.cu: one instance; batch.cu: many instances as one disjoint union).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/f2m.h"
#include "f2m_internal.h"

namespace f2m {
struct CutState;  // subtour-elimination cuts (cuts.cu)
}

struct f2m_ctx {
  // segments: contiguous node ranges that are separate instances (a batch);
  // one segment [0, n) for a single instance.  Pricing pairs stay inside a
  // segment; the tiled / batch GDP kernels freeze converged segments.
  std::vector<int32_t> seg_off{0};      // [nseg+1] node offsets
  std::vector<uint8_t> seg_scan;        // segments the next pricing scan covers (empty: all)
  std::vector<int64_t> seg_pairs;       // pairs per segment found by the last scan
  int32_t* d_seg_off = nullptr;         // device copy of seg_off (batches)
  uint8_t* d_fin_include = nullptr;     // per segment: the finisher may change it (NULL = all)
  int4* d_tiles = nullptr;              // pricing tile-pair list
  int64_t tiles_cap = 0;
  int64_t ntiles = 0;                   // tile pairs in d_tiles
  int tiles_kind = 0;                   // the list's form: 0 fp32 scan, 1 tensor-core scan
  bool tiles_valid = false;             // d_tiles holds the full scan's list for:
  std::vector<uint8_t> tiles_seg_scan;  //   these scanned segments
  std::vector<int32_t> tiles_seg_off;   //   of these segments
  int2* d_ranges = nullptr;             // culled pricing: point ranges of the tiles,
  float4* d_boxes = nullptr;            // their bounding boxes
  float* d_smax = nullptr;              // and largest filter radii
  int64_t ranges_cap = 0;

  int32_t n = 0;
  int64_t nnz = 0;
  int64_t ec_cap = 0;
  cudaStream_t st = nullptr;
  f2m_params p{};
  int num_sms = 0;
  int2* d_xy = nullptr;
  int32_t* d_rp = nullptr;
  int2* d_ec = nullptr;
  int2* d_ec_alt = nullptr;  // [ec_alt_cap] the merge writes here, then the two swap
  int64_t ec_alt_cap = 0;
  uint8_t* d_x2 = nullptr;
  int64_t x2_cap = 0;
  int32_t* d_lam[2] = {nullptr, nullptr};
  int32_t* d_lam2 = nullptr;
  int32_t* d_exl = nullptr;   // [n] the finisher's surpluses (its own: the plan's scratch
                              // still feeds a two-sweep plan built later)
  int32_t* d_b = nullptr;  // degree requirements b_v, caller order (NULL: b_v = 2)
  int32_t* d_b_int = nullptr;  // the same in the renumbered (internal) order
  int32_t b_max = 2;       // the largest b_v
  int32_t gdp_kernel = 0;  // F2M_GDP_KERNEL_* of the last GDP phase
  int cur = 0;          // d_lam[cur] holds lambda in units 2^-F
  int32_t fb_cur = 8;   // F, or F+1 while d_lam2 holds the current lambda
  f2m::GdpCtl* d_gdp = nullptr;
  long long* d_trace_b2 = nullptr;
  unsigned long long* d_trace_ch = nullptr;
  int64_t trace_cap = 0;
  float4* d_pts = nullptr;
  int4* d_pts4 = nullptr;       // tensor-core scan: {x, y, lambda, node} per renumbered position
  int32_t* d_pstat = nullptr;   // its status word
  int2* d_mranges = nullptr;    // its 128-point blocks (with the tile list: same segments)
  int4* d_mtblk = nullptr;      // blocks of each tile pair
  int4* d_mbox = nullptr;       // per block: bounding box, largest lambda (per scan)
  int32_t* d_mlmax = nullptr;
  int4* d_mframes = nullptr;    // per tile pair: the frame (per scan)
  int64_t mblocks = 0, mblocks_cap = 0, mtiles_cap = 0;
  int2* d_mcand = nullptr;      // the filter's candidates
  unsigned long long* d_mncand = nullptr;
  int64_t mcand_cap = 0;
  // the scan that certifies the finisher's lambda: a complete scan at lambda
  // lam_ref (units 2^-ref_fb) left every pair outside the CSR with z >= 0; if
  // the finisher is the only change of lambda since (lam_version counts every
  // change), a pair can turn negative only where lambda rose, so only those
  // nodes' rows are scanned
  int64_t lam_version = 0;      // bumped by every change of lambda
  int64_t ref_version = -1;     // lam_version of the scan that wrote d_lam_ref
  int64_t fin_src_version = -2; // lam_version before / after the last finisher call
  int64_t fin_dst_version = -3;
  int32_t ref_fb = 0;
  int32_t* d_lam_ref = nullptr; // [n] caller order
  uint8_t* d_raised = nullptr;  // [n] nodes whose lambda rose
  float4* d_pts_raised = nullptr;  // [n] their points
  unsigned int* d_nraised = nullptr;
  int64_t last_scan_rows = -1;  // rows of the last scan if it was a certifying one, else -1
  int64_t last_scan_pairs = 0;  // pairs the last scan evaluated
  int2* d_pairs = nullptr;
  int64_t pairs_cap = 0;
  int64_t npairs = 0;   // pairs held in d_pairs after the last scan
  unsigned long long* d_count = nullptr;
  unsigned int* d_tile = nullptr;
  int32_t* d_deg = nullptr;
  int32_t* d_tmp_rp = nullptr;
  int32_t* d_new_rp = nullptr;
  int32_t* d_block_sums = nullptr;
  int32_t* d_tmp_col = nullptr;
  int64_t tmp_col_cap = 0;
  int32_t* d_out_a = nullptr;  // split scratch for f2m_get_x
  int32_t* d_out_b = nullptr;
  int64_t out_cap = 0;
  f2m::CheckCtl* d_check = nullptr;
  long long* d_scalar = nullptr;
  unsigned long long* d_bad = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  f2m::GdpPlan plan;         // renumbering and tiles of the shared-memory GDP kernel
  bool plan1_pending = false;  // the one-sweep tiles are built at the next GDP phase
  bool plan2_pending = false;  // the two-sweep tiles are built at the next GDP phase
  f2m::ClassPlan classes;    // colour classes of the class-by-class GDP
  // exact finisher: device scratch, host work arrays; the h_ arrays point into
  // the process's one pinned host mirror while a finisher call holds it
  int32_t* d_twin = nullptr;
  uint8_t* d_fy = nullptr;
  int64_t fin_cap = 0;          // entries the device finisher buffers hold
  int64_t fin_version = -1;     // plan version the host mirror holds whole (while this context owns it)
  int64_t twin_version = -1;    // plan version of d_twin
  int32_t* h_irp = nullptr;
  int2* h_iec = nullptr;
  int32_t* h_twin = nullptr;
  uint8_t* h_y = nullptr;
  int32_t* h_exl = nullptr;
  int32_t* h_lam = nullptr;
  int32_t* h_lam2 = nullptr;
  f2m::FinisherWork* fin_work = nullptr;
  // the finisher's phase 1 on the GPU: node state of both copies, blocks, heaps
  long long* d_fpi = nullptr;
  long long* d_fdist = nullptr;
  int32_t* d_fex = nullptr;
  int32_t* d_fvia = nullptr;
  int32_t* d_fpred = nullptr;
  uint32_t* d_freach = nullptr;
  uint32_t* d_fclos = nullptr;
  int32_t* d_forder = nullptr;
  int32_t* d_fstat = nullptr;
  int2* d_fblk = nullptr;
  long long* d_fcaps = nullptr;
  long long* d_fheap_off = nullptr;
  long long* d_fpush = nullptr;
  uint8_t* d_fheap = nullptr;
  int64_t fblk_cap = 0, fheap_cap = 0;  // blocks, heap items
  int64_t* h_fpi = nullptr;             // pinned copies of the phase-1 state for the host
  int32_t* h_fex = nullptr;
  f2m::FinisherStats fin_stats;  // the finisher's split, summed since the solve began
  f2m::CutState* cuts = nullptr;  // layers of subtour-elimination cuts and their duals
  std::string err;
};

namespace f2m {

f2m_status fail(f2m_ctx* ctx, f2m_status s, const std::string& msg);
f2m_status cuda_fail(f2m_ctx* ctx, cudaError_t e, const char* what);

#define CK(ctx, call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, int64_t count) {
  *p = nullptr;
  size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
  return dev_malloc((void**)p, bytes);
}

template <typename T>
void dfree(T*& p) {
  if (p) dev_free((void*)p);
  p = nullptr;
}

// for a caller that has already waited for every use of the block
template <typename T>
void dfree_synced(T*& p) {
  if (p) dev_free_synced((void*)p);
  p = nullptr;
}

f2m_status check_params_internal(const f2m_params& p);
const int32_t* cur_lambda(f2m_ctx* c, int32_t* fb);
f2m_status gdp_phase(f2m_ctx* c, int64_t max_sweeps, int64_t* sweeps, bool want_trace,
                     int64_t trace_cap, double* ms);
// lam_override (device, [n], units 2^-fb): scan with it in place of lambda
f2m_status price_internal(f2m_ctx* c, double* ms, const int32_t* lam_override = nullptr);
f2m_status merge_internal(f2m_ctx* c, const int2* d_pairs, int64_t npairs, double* ms);
f2m_status extract_internal(f2m_ctx* c, int64_t* bad, double* ms);
f2m_status bound_internal(f2m_ctx* c, int64_t* b2);
// h_include (host, per segment; NULL = all): the segments the finisher works on
f2m_status finisher_internal(f2m_ctx* c, int64_t* aug, const uint8_t* h_include);
void copy_finisher_stats(const f2m_ctx* c, f2m_info* info);
// subtour-elimination cuts (cuts.cu)
void cut_state_free(CutState* s);
int64_t cut_count(const f2m_ctx* c);
f2m_status cut_gdp_phase(f2m_ctx* c, int64_t max_sweeps, int64_t* sweeps, long long* tb,
                         unsigned long long* tc, int64_t tcap, double* ms);
f2m_status cut_bound_extract(f2m_ctx* c, bool want_x, int64_t* b2, int64_t* bad);
f2m_status cut_price(f2m_ctx* c, double* ms);
// create a context for the graph, renumbering within segments when seg_off has
// more than one segment (seg_off[0] = 0, seg_off.back() = n)
f2m_status create_internal(const int32_t* xy, int32_t n, const int32_t* row_ptr, const int32_t* col,
                           const f2m_params* params, void* stream,
                           const std::vector<int32_t>& seg_off, f2m_ctx** out);

}  // namespace f2m
