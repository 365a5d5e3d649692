// internal.cuh -- state of an afmpb handle and the internal entry points shared by the
// translation units of the library (geometry, tree, near field, FMM, solver, C ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <exception>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/afmpb.h"

// Box centre and half width (32-byte aligned, one vector load).
struct __align__(32) dbl4 {
  double x, y, z, w;
};

namespace afmpb {

constexpr int kMaxOrder = 8;        // Chebyshev points per dimension, upper bound
constexpr int kMaxLevel = 20;       // deepest octree level
constexpr int kKeyBits = 21;        // Morton bits per dimension (63-bit keys)
constexpr int kNumOffsets = 316;    // M2L offsets: [-3,3]^3 minus [-1,1]^3
constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)
constexpr int kP2PThreads = 128;   // threads of a P2P block (one work unit of one target leaf at a time)
constexpr int kP2PResident = 6;    // P2P blocks kept resident per SM (<= 80 registers per thread)
constexpr int kP2PUnitsPerBlock = 3;   // P2P work units per resident block (sets the unit size; 2-3 best of 1-32)
constexpr double kP2PSkip = 0.9;    // P2P leaves out pairs closer than kP2PSkip * c * (rho_p + rho_t)

// Pair geometry of the P2P pass in FP32.  Positions are relative to the target's leaf
// centre; a source is shifted by the rounded difference of the two leaf centres.  Near-field
// setup calls the same functions to learn, bit for bit, which near pairs the P2P pass
// leaves out (those pairs then carry the whole near-rule value in the near CSR).  The
// _rn intrinsics keep the compiler from contracting the products into FMAs differently
// in the two kernels.
__device__ __forceinline__ float p2p_shift(float x, double src_centre, double tgt_centre) {
  return __fadd_rn(x, (float)(src_centre - tgt_centre));
}
__device__ __forceinline__ float p2p_r2(float dx, float dy, float dz) {
  return fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(dz, dz)));
}
// Scaled patch radius kP2PSkip * c * rho of one node; `scale` = (float)(kP2PSkip * c).
__device__ __forceinline__ float p2p_skip_radius(float scale, float rho) { return __fmul_rn(scale, rho); }
// True when the P2P pass evaluates the pair (squared distance r2, scaled radii sp and st).
__device__ __forceinline__ bool p2p_evaluates(float r2, float sp, float st) {
  const float R = __fadd_rn(sp, st);
  return r2 > __fmul_rn(R, R);
}

// Global -> shared copies with kCopyILP independent loads in flight per thread (a plain
// element loop issues each load only after the previous element's store).
constexpr int kCopyILP = 8;
__device__ __forceinline__ void copy_g2s(float *dst, const float *__restrict__ src, int n) {
  for (int e0 = threadIdx.x; e0 < n; e0 += blockDim.x * kCopyILP) {
    float v[kCopyILP];
#pragma unroll
    for (int u = 0; u < kCopyILP; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < n ? __ldg(src + e) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kCopyILP; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n) dst[e] = v[u];
    }
  }
}
// Same for 16-byte vectors (both pointers 16-byte aligned, n4 vectors).
__device__ __forceinline__ void copy_g2s4(float4 *dst, const float4 *__restrict__ src, int n4) {
  for (int e0 = threadIdx.x; e0 < n4; e0 += blockDim.x * kCopyILP) {
    float4 v[kCopyILP];
#pragma unroll
    for (int u = 0; u < kCopyILP; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < n4 ? __ldg(src + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kCopyILP; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n4) dst[e] = v[u];
    }
  }
}

// Error carried up the host call chain; every internal function returns one.
struct Err {
  afmpb_status code = AFMPB_OK;
  std::string msg;
  bool ok() const { return code == AFMPB_OK; }
};
inline Err make_err(afmpb_status c, const std::string &m) { return Err{c, m}; }

#define AFMPB_CUDA(call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return ::afmpb::make_err(AFMPB_ECUDA, std::string(#call) + ": " +               \
                                                cudaGetErrorString(e_));              \
  } while (0)

#define AFMPB_TRY(expr)                 \
  do {                                  \
    ::afmpb::Err e_ = (expr);           \
    if (!e_.ok()) return e_;            \
  } while (0)

// Makes the device's default memory pool keep freed memory for reuse (stream-ordered
// allocations of later handles then need no new device memory); once per device.
void keep_pool_memory();

// Device allocation registry owned by a handle.  With a stream set, memory comes from the
// device's stream-ordered pool (cudaMallocAsync / cudaFreeAsync on that stream): a free
// does not synchronise the device, so handles created and destroyed by one server slot do
// not stall the solves running on the others.
struct DeviceArena {
  std::vector<std::pair<void *, size_t>> blocks;
  size_t bytes = 0;
  size_t peak = 0;                 // high-water mark of bytes
  cudaStream_t stream = nullptr;   // stream the allocations and frees are ordered on
  template <class T>
  Err alloc(T **p, size_t count, const char *what) {
    *p = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = stream ? cudaMallocAsync(&q, count * sizeof(T), stream) : cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return make_err(AFMPB_ENOMEM, std::string("cudaMalloc ") + what + " (" +
                                        std::to_string(count * sizeof(T)) + " B): " +
                                        cudaGetErrorString(e));
    }
    blocks.push_back({q, count * sizeof(T)});
    bytes += count * sizeof(T);
    peak = std::max(peak, bytes);
    *p = static_cast<T *>(q);
    return Err{};
  }
  void release(void *p) {
    for (size_t i = 0; i < blocks.size(); ++i)
      if (blocks[i].first == p) {
        if (stream) cudaFreeAsync(p, stream);
        else cudaFree(p);
        bytes -= blocks[i].second;
        blocks.erase(blocks.begin() + i);
        return;
      }
  }
  void free_all() {
    for (auto &b : blocks) {
      if (stream) cudaFreeAsync(b.first, stream);
      else cudaFree(b.first);
    }
    blocks.clear();
    bytes = 0;
  }
};

// Host mirror of the octree shape (the device holds the arrays).
struct TreeShape {
  int nbox = 0, nleaf = 0, nlevel = 0;     // levels 0 .. nlevel-1
  std::vector<int> lvl_start;              // [nlevel + 1] box index ranges per level
  double c0[3] = {0, 0, 0};                // root centre
  double w0 = 1;                           // root half width (power of two)
  int64_t n_u = 0, n_v = 0, n_w = 0, n_x = 0, n_p2p_pairs = 0;
};

// Optional per-stage event marks (afmpb_profile_product); nullptr in normal launches.
struct StageTimer {
  cudaStream_t s = nullptr;
  std::vector<std::string> names;
  std::vector<cudaEvent_t> ends;
  std::vector<int> launches;
  void mark(const char *name, int nlaunch) {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    names.push_back(name);
    ends.push_back(e);
    launches.push_back(nlaunch);
  }
  ~StageTimer() {
    for (auto e : ends) cudaEventDestroy(e);
  }
};

// One M2L work group: all V-list pairs of one level and one offset.
struct M2LGroup {
  int level, offset, start, count;
};

// One tensor-core M2L work item: up to 128 pairs of one group.
struct TCItem {
  int group, start, count;
};

// One item of the target-stationary tensor-core M2L: a block of up to 128 target boxes
// [base, end) of one level, the runs [run0, run1) of its (offset, pairs) work and their
// entries [ent0, ent1), the kernel (0 Laplace, 1 Yukawa), its compressed table and rank,
// and the output scale.
struct __align__(16) TSItem {
  int base, end, run0, run1;
  int kt, table, rank;
  float scale;
  int ent0, ent1, req, pad1;    // the item's entries [ent0, ent1) (its runs are consecutive);
                                // req: the problem of a batched launch (0 otherwise)
};

// One problem of a batched P2P launch: the arrays and constants k_p2p takes, and a device
// flag (nullable) that stops its units when 0.
struct P2PReq {
  const int32_t *leaves;
  const int64_t *pptr;
  const int32_t *pidx, *bbeg, *bend;
  const dbl4 *center;
  const float4 *pos, *nrm;
  const float2 *xs;
  float4 *phi;
  const int *active;
  float inv_ebar, kappa, skip_scale;
};

// One problem of a batched target-stationary M2L launch: its runs, entries, compressed
// multipoles, tables and local expansions, and its stop flag.
struct TSReq {
  const int4 *runs;
  const uint64_t *ent;
  const void *Mc16, *tiles;
  float *Lc;
  const int *active;
};

}  // namespace afmpb

struct afmpb_t {
  // ---- parameters -------------------------------------------------------------------
  int64_t n = 0, nt = 0, natoms = 0;
  int device = 0;                  // CUDA device current at create time
  double eps_in = 1, eps_out = 1, kappa = 0, ebar = 1, alpha = 1, tol = 1e-6;
  int order = 6, ncoef = 216;
  afmpb_options opt{};
  std::string err;
  double ms_setup = 0;
  double ms_create[6] = {0, 0, 0, 0, 0, 0};

  // ---- streams / events --------------------------------------------------------------
  cudaStream_t stream = nullptr;   // handle stream (user's or own)
  bool own_stream = false;
  cudaStream_t side = nullptr;     // second stream: P2P beside the far-field chain
  cudaStream_t side2 = nullptr;    // third stream: P2L beside the upward pass and the M2L
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;

  afmpb::DeviceArena arena;

  // ---- mesh, caller order ------------------------------------------------------------
  double *d_xyz = nullptr;         // [3n]
  int32_t *d_tri = nullptr;        // [3nt]
  int64_t *d_inc_ptr = nullptr;    // [n+1] node -> incident triangles
  int32_t *d_inc_tri = nullptr;    // [3nt]
  double *d_tri_nrm = nullptr;     // [3nt] unit facet normals
  double *d_area64 = nullptr;      // [n]
  double *d_nrm64 = nullptr;       // [3n]
  double *d_rho64 = nullptr;       // [n]

  // ---- octree -----------------------------------------------------------------------
  afmpb::TreeShape shape;
  uint64_t *d_key = nullptr;       // [n] sorted Morton keys
  int32_t *d_perm = nullptr;       // [n] Morton position -> caller index
  int32_t *d_box_level = nullptr, *d_box_parent = nullptr, *d_box_child0 = nullptr,
          *d_box_nchild = nullptr, *d_box_begin = nullptr, *d_box_end = nullptr;
  int4 *d_box_anchor = nullptr;    // x, y, z cell coordinates at the box level, w = level
  dbl4 *d_box_center = nullptr; // centre, w = half width
  uint64_t *d_box_key = nullptr;   // Morton prefix at the box level
  double *d_box_rho = nullptr;     // largest patch radius inside the box
  int32_t *d_colleague = nullptr;  // [27 nbox]
  int32_t *d_leaves = nullptr;     // [nleaf] leaf box ids in Morton order
  int32_t *d_node_leaf = nullptr;  // [n] Morton position -> leaf box
  int32_t *d_leaf_index = nullptr; // [nbox] leaf box -> position in d_leaves, -1 otherwise
  // lists (CSR over boxes; u and w non-empty only for leaves)
  int64_t *d_u_ptr = nullptr, *d_v_ptr = nullptr, *d_w_ptr = nullptr, *d_x_ptr = nullptr;
  int32_t *d_u_idx = nullptr, *d_v_idx = nullptr, *d_w_idx = nullptr, *d_x_idx = nullptr;
  int64_t *d_p2p_ptr = nullptr;    // [nleaf+1] lists 1 + 3 per leaf (leaf order)
  int32_t *d_p2p_idx = nullptr;
  int4 *d_p2p_units = nullptr;     // [p2p_nunits] P2P work units (leaf, first and end entry of its
  int p2p_nunits = 0;              // source boxes in p2p_idx, -), most pairs first
  int p2p_resident = afmpb::kP2PResident;            // P2P blocks per SM (tile tuner)
  int p2p_units_per_block = afmpb::kP2PUnitsPerBlock;   // P2P unit size (tile tuner)
  int n_xbox = 0;                  // boxes whose list 4 goes to their local expansion (P2L)
  int32_t *d_xbox = nullptr;       // those boxes

  // ---- Morton-ordered node data -----------------------------------------------------
  float4 *d_pos = nullptr;         // position relative to the leaf centre, w = patch area
  float4 *d_nrm = nullptr;         // unit normal, w = patch radius rho

  // ---- near field -------------------------------------------------------------------
  int64_t nnz = 0;
  int64_t *d_near_ptr = nullptr;   // [n+1]
  int32_t *d_near_col = nullptr;   // [nnz] Morton positions
  float4 *d_near_coef = nullptr;   // [nnz] (dA, dB, dC, dD)
  uint8_t *d_near_full = nullptr;  // [nnz] 1 where the entry holds the whole near-rule value

  // ---- FMM --------------------------------------------------------------------------
  float *d_M = nullptr;            // [nbox][2][ncoef] multipole weights (Laplace, Yukawa)
  float *d_L = nullptr;            // [nbox][2][ncoef] local weights
  float *d_K_lap = nullptr;        // [316][ncoef][ncoef] unit-box Laplace M2L
  float *d_K_yuk = nullptr;        // [nlevel][316][ncoef][ncoef] Yukawa M2L per level
  std::vector<afmpb::M2LGroup> m2l_groups;
  afmpb::M2LGroup *d_m2l_groups = nullptr;
  int2 *d_m2l_pairs = nullptr;     // (target, source) boxes grouped by (level, offset)
  int64_t n_m2l_pairs = 0;
  int m2l_yuk_levels = 0;          // Yukawa M2L skipped on levels below this one
  bool laplace_only = false;       // no Yukawa translations at all (the Yukawa outputs are unused)
  // compressed M2L (m2l_rank > 0): bases Q per table (0 = Laplace on the unit box,
  // 1.. = Yukawa per level), translations C_o = Q^T K_o Q, compressed expansions
  int m2l_rank = 0;                // storage stride r (largest table rank, multiple of 16); 0 = full n^3
  std::vector<int> h_table_rank;   // each table's own rank (<= r; columns beyond it are zero)
  int *d_table_rank = nullptr;
  int m2l_ntables = 0;
  std::vector<int> h_level_table;  // level -> Yukawa table
  int *d_level_table = nullptr;
  float *d_Q = nullptr;            // [table][ncoef][r]
  float *d_QT = nullptr;           // [table][r][ncoef]
  float *d_C = nullptr;            // [table][316][r][r]
  float *d_Mc = nullptr;           // [nbox][2][r] compressed multipole vectors
  uint16_t *d_Mc16 = nullptr;      // [nbox][2][hi, lo][r] the same split into BF16 (precision 1)
  float *d_Lc = nullptr;           // [nbox][2][r] compressed local vectors
  int4 *d_m2l_chunks = nullptr;    // (first box, count, level) of the compress/expand CTAs
  int m2l_nchunks = 0;
  // tensor-core M2L (precision 1)
  int tc_items = 0;
  afmpb::TCItem *d_tc_items = nullptr;  // work items: (group, first pair, pair count)
  uint16_t *d_tc_tiles = nullptr;  // BF16 hi/lo translation tiles in the MMA operand layout
  int *d_tc_level_table = nullptr; // level -> Yukawa tile table
  int *d_tc_flag = nullptr;        // device alias of h_wait_flag (the kernels' error flag)
  int *h_wait_flag = nullptr;      // mapped pinned host int, set by a CTA whose bounded wait
                                   // expired; read (and cleared) by the host after the work
  // target-stationary tensor-core M2L (compressed ranks <= 112): list-2 entries sorted by
  // (target block, offset), their runs, and the work items
  int ts_nitems = 0;
  int ts_runs_per_item = 0;        // most runs per item (0: the default cut; tile tuner)
  std::vector<uint32_t> ts_rkey;   // host copy of the runs: (block, offset) key and entry count,
  std::vector<int32_t> ts_rcnt;    // to cut the items again
  afmpb::TSItem *d_ts_items = nullptr;
  // plane-wave M2L (options.m2l_method = 1): tables per (level, kernel), targets by direction
  std::vector<int> pw_set_of, pw_level_t0;
  int pw_pmax = 0, pw_maxlev = 0, pw_ntargets = 0;
  void *d_pw_sets = nullptr;
  int *d_pw_pnode = nullptr, *d_pw_pb = nullptr, *d_pw_perm = nullptr;
  float *d_pw_exs = nullptr, *d_pw_ext = nullptr, *d_pw_om = nullptr;
  float2 *d_pw_phx = nullptr, *d_pw_phy = nullptr, *d_pw_shift = nullptr, *d_pw_X = nullptr;
  int *d_pw_tbox = nullptr, *d_pw_dptr = nullptr, *d_pw_esrc = nullptr, *d_pw_eslot = nullptr;
  int4 *d_ts_runs = nullptr;       // (offset slot, first entry, end entry, -)
  uint64_t *d_ts_ent = nullptr;    // row in the block << 32 | source box
  uint16_t *d_ts_tiles = nullptr;  // C_o as BF16 hi/lo B-operand tiles [table][slot][2][R x R]

  // ---- leaf-capacity autotuner (AFMPB_LEAF_CAP_AUTO) --------------------------------
  bool autotuned = false;
  afmpb_autotune_report tune{};

  // ---- per-product work --------------------------------------------------------------
  float2 *d_xs = nullptr;          // [n] (f, h) Morton order
  float *d_ys = nullptr;           // [2n] y Morton order
  float4 *d_phi_far = nullptr;     // [n] (PhiL, dn PhiL, PhiY, dn PhiY) from L2P
  float4 *d_phi_near = nullptr;    // [n] same from P2P
  cudaGraphExec_t graph[8] = {};   // captured product (Morton-ordered d_xs -> d_ys), per parts mask
  cudaGraphExec_t graph_io[8] = {};          // the same with gather and scatter of caller buffers
  cudaGraph_t graph_io_tmpl[8] = {};         // templates of graph_io (their nodes are updated)
  cudaGraphNode_t io_gather[8] = {}, io_scatter[8] = {};
  const float *io_x[8] = {};                 // buffers the io graphs currently point at
  float *io_y[8] = {};
  cudaGraphExec_t graph_gm = nullptr;        // solver product: FP64 Krylov vector -> d_ys
  cudaGraph_t graph_gm_tmpl = nullptr;
  cudaGraphNode_t gm_to_xs = nullptr;
  const double *gm_src = nullptr;
  float *d_xhost_stage = nullptr, *d_yhost_stage = nullptr;   // afmpb_matvec_host staging
  float *d_prof_x = nullptr, *d_prof_y = nullptr;             // afmpb_profile_product buffers

  // ---- right-hand side, solution, atoms ---------------------------------------------
  double *d_atoms = nullptr;       // [3 natoms]
  double *d_q = nullptr;           // [natoms]
  double *d_b = nullptr;           // [2n] Morton order
  double bnorm = 0;
  double *d_sol = nullptr;         // [2n] Morton order
  bool solved = false;
  // GMRES work (allocated at first solve)
  int gm_m = 0;
  double *d_V = nullptr, *d_w = nullptr, *d_H = nullptr, *d_g = nullptr, *d_cs = nullptr,
         *d_sn = nullptr, *d_part = nullptr, *d_hcol = nullptr, *d_hcol2 = nullptr, *d_scal = nullptr;
  double *h_pinned = nullptr;
  int *d_gm_int = nullptr;         // [8] device step state: j, Arnoldi steps, second-pass flag, second passes,
                                   // running flag of a batched solve
  cudaGraphExec_t graph_cycle = nullptr;   // one GMRES cycle: a graph WHILE loop over Arnoldi steps
  int cycle_m = 0, cycle_orth = -1;        // restart length and orthogonalisation the cycle graph was built for
  // Laplace FMM over nodes and charges for the right-hand side and the energy (owned)
  afmpb_t *cf = nullptr;
};

namespace afmpb {

// geometry.cu
Err validate_mesh(const afmpb_mesh *mesh);
Err build_geometry(afmpb_t *h, const afmpb_mesh *mesh);
// tree.cu
Err build_tree(afmpb_t *h);
Err build_p2p_units(afmpb_t *h);       // P2P work units at h->p2p_units_per_block
// near.cu
Err build_near(afmpb_t *h);
// fmm.cu
Err build_fmm(afmpb_t *h);
// Parts of the far-field chain: the upward pass to the compressed expansions, the M2L,
// and the downward pass from the local expansions to d_phi_far.
constexpr int kFarUp = 1, kFarM2L = 2, kFarDown = 4, kFarAll = 7;
Err enqueue_far(afmpb_t *h, cudaStream_t s, StageTimer *tm = nullptr, int parts = kFarAll);   // P2M .. L2P
Err enqueue_p2p(afmpb_t *h, cudaStream_t s);          // P2P into d_phi_near
bool overlap_p2p(const afmpb_t *h);                   // P2P runs beside the far-field chain
// The P2P arguments of a handle, with a stop flag for batched launches.
P2PReq p2p_req_of(const afmpb_t *h, const int *active);
// One P2P launch over the units of several problems (unit.w names the problem); every
// problem's d_phi_near must be zeroed before it.
Err enqueue_p2p_batch(const P2PReq *d_reqs, const int4 *d_units, int nunits, int resident, cudaStream_t s);
// Combine flag beside the AFMPB_PART_* bits: the near correction was folded into the P2P
// sums by enqueue_near_fold (on the P2P branch, after P2P), which requires the far part.
constexpr int kNearFolded = 8;
Err enqueue_near_fold(afmpb_t *h, cudaStream_t s);   // near SpMV into phi_near, after P2P
Err enqueue_combine(afmpb_t *h, cudaStream_t s, int parts);
Err enqueue_m2l_tc(afmpb_t *h, cudaStream_t s);       // tensor-core M2L (precision 1)
Err build_m2l_tc(afmpb_t *h);
// m2l_ts.cu: the target-stationary tensor-core M2L
bool m2l_ts_applies(const afmpb_t *h);
Err build_m2l_ts(afmpb_t *h);
Err enqueue_m2l_ts(afmpb_t *h, cudaStream_t s);
// One target-stationary M2L launch over the items of several problems (TSItem.req names
// the problem); the items of stopped problems are compacted away first on the device.
Err enqueue_m2l_ts_batch(const TSReq *d_reqs, const TSItem *d_items, int nitems, TSItem *d_items_run, int *d_count,
                         int R, int *err_flag, cudaStream_t s);
Err cut_m2l_ts_items(afmpb_t *h);      // items from the stored runs at h->ts_runs_per_item
Err autotune_tiles(afmpb_t *h, afmpb_autotune_report *rep);   // autotune.cu: P2P and M2L tile shapes
void autotune_cache_tiles(const afmpb_t *h);
bool autotune_cached_tiles(afmpb_t *h);
// autotune.cu
Err autotune_leaf_cap(afmpb_t *h, afmpb_autotune_report *rep);
int autotune_cached_cap(int precision, int order, double kappa, int64_t n);   // 0 if none
// m2l_svd.cu: compressed translations; *compressed = false leaves the full ones in use
Err build_m2l_svd(afmpb_t *h, bool *compressed);
Err enqueue_m2l_svd(afmpb_t *h, cudaStream_t s, StageTimer *tm = nullptr, int parts = kFarAll);
// m2l_pw.cu: plane-wave M2L (d_M -> d_L, FP32) and its tables
Err build_m2l_pw(afmpb_t *h);
Err enqueue_m2l_pw(afmpb_t *h, cudaStream_t s);   // compress, translate, expand
Err alloc_wait_flag(afmpb_t *h);       // the mapped error flag of the bounded waits (once per handle)
// Waits for the handle's stream, then reports (and clears) the bounded-wait flag: *flag = 1
// when a wait of work queued on the handle expired since the last report.
Err read_tc_error(afmpb_t *h, int *flag);
Err selftest_bounded_wait(int spin_limit, int *expired);   // m2l_tc.cu             // 1 when a tensor-core wait expired
// solve.cu
Err build_rhs(afmpb_t *h);
Err enqueue_gather(afmpb_t *h, cudaStream_t s, const float *x_caller);
const void *gather_kernel();                           // k_gather, to find its graph node
const void *scatter_kernel();
const void *to_xs_kernel();
Err enqueue_to_xs(afmpb_t *h, cudaStream_t s, const double *v);   // FP64 Morton vector -> d_xs
Err product_from64(afmpb_t *h, cudaStream_t s, const double *v);  // d_ys = L v (one graph launch)
Err enqueue_scatter(afmpb_t *h, cudaStream_t s, float *y_caller);
Err run_solve(afmpb_t *h, afmpb_solve_info *info);
Err run_energy(afmpb_t *h, double *E);
// charge_fmm.cu
bool charge_fmm_wanted(const afmpb_t *h);
Err build_charge_fmm(afmpb_t *h);
Err charge_fmm_rhs(afmpb_t *h, double *b);       // b [2n], Morton order
Err charge_fmm_phi(afmpb_t *h, double *phi);     // reaction potential at the charges (with 1/(4 pi))
Err run_energy_noalloc(afmpb_t *h, double *E);      // static scratch, no allocation
// batch.cu: the merged work lists and descriptors of a batched solve, in stream-ordered
// device memory freed with the object
struct BatchLists {
  cudaStream_t stream = nullptr;
  std::vector<void *> bufs;
  P2PReq *d_p2p = nullptr;
  int **d_gms = nullptr;              // each problem's step state (gm[4]: running)
  int4 *d_units = nullptr;            // P2P units of all problems, by cost (unit.w = problem)
  int nunits = 0;
  TSReq *d_ts = nullptr;
  TSItem *d_items = nullptr, *d_items_run = nullptr;   // M2L items of all problems; the running ones
  int *d_count = nullptr;
  int nitems = 0;
  BatchLists() = default;
  BatchLists(const BatchLists &) = delete;
  BatchLists &operator=(const BatchLists &) = delete;
  ~BatchLists();
  Err alloc_bytes(void **p, size_t bytes, const char *what);
  template <class T>
  Err alloc(T **p, int64_t n, const char *what) {
    return alloc_bytes(reinterpret_cast<void **>(p), sizeof(T) * (size_t)(n > 0 ? n : 1), what);
  }
};
Err build_batch_lists(afmpb_t *const *hs, int k, bool fuse_m2l, BatchLists &L);
// solve.cu: lockstep GMRES of k handles (one graph launch per restart cycle for all)
Err run_solve_batch(afmpb_t *const *hs, int k, afmpb_solve_info *infos, afmpb_status *statuses);

// capi.cu
Err product_sorted(afmpb_t *h, cudaStream_t s, int parts);  // d_xs -> d_ys
Err enqueue_product_kernels(afmpb_t *h, cudaStream_t cap);   // d_xs -> d_ys on a capturing stream
Err recapture_products(afmpb_t *h);   // drop the captured product graphs and capture the full one again

// launch helpers
inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Host: f(part, begin, end) over [0, n) split into contiguous ranges, one per host thread
// (at most 16, and at most one per 4,096 items); returns the number of parts.  Part p
// covers [n p / parts, n (p + 1) / parts), so results written per part and concatenated
// in part order equal a sequential pass.
template <class F>
int host_parallel(int64_t n, F f) {
  const int parts = (int)std::max<int64_t>(
      1, std::min<int64_t>({16, (int64_t)std::max(1u, std::thread::hardware_concurrency()), n / 4096 + 1}));
  std::vector<std::thread> pool;
  for (int p = 1; p < parts; ++p) pool.emplace_back(f, p, n * p / parts, n * (p + 1) / parts);
  f(0, (int64_t)0, n / parts);
  for (auto &t : pool) t.join();
  return parts;
}

// The number of parts host_parallel will use for n items (to size per-part buffers).
inline int host_parts(int64_t n) {
  return (int)std::max<int64_t>(
      1, std::min<int64_t>({16, (int64_t)std::max(1u, std::thread::hardware_concurrency()), n / 4096 + 1}));
}
// Raise a kernel's dynamic shared-memory limit to at least `bytes` (the attribute is
// process-wide per kernel and per device, so it is only ever raised: a handle that needs
// less must not lower it under another handle's launch).
Err raise_smem_limit(const void *func, int bytes);

// The Err of the exception being handled; call only inside a catch block.  Host
// allocation and thread-creation failures are ENOMEM, anything else EINTERNAL.  The C
// entry points use it so that no C++ exception crosses the C boundary.
inline Err current_exception_err() {
  try {
    throw;
  } catch (const std::bad_alloc &) {
    return make_err(AFMPB_ENOMEM, "host memory allocation failed");
  } catch (const std::system_error &e) {
    return make_err(AFMPB_ENOMEM, std::string("host resources: ") + e.what());
  } catch (const std::exception &e) {
    return make_err(AFMPB_EINTERNAL, std::string("host exception: ") + e.what());
  } catch (...) {
    return make_err(AFMPB_EINTERNAL, "unknown host exception");
  }
}

inline Err check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return make_err(AFMPB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return Err{};
}

}  // namespace afmpb
