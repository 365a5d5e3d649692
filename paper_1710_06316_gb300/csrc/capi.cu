// capi.cu -- the C ABI declared in include/afmpb.h: handle lifecycle, the captured
// product graph, solve / energy entry points and the export calls used by tests.
//
// The product (one GMRES matvec, Sec. 2 step 3) is captured once per parts mask into a
// CUDA graph: the far-field chain (P2M, M2M per level, M2L, P2L, L2L per level, L2P) runs
// on the handle's capture stream while the point-to-point kernel runs beside it on a
// second stream; the combine kernel (near correction + Eq. 5 assembly) joins them.
// Replaying the graph replaces the paper's per-iteration DAG execution (Sec. 3.3:
// create the DAG once, execute it many times).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "internal.cuh"

using namespace afmpb;

namespace {

thread_local std::string g_err;

afmpb_status fail(afmpb_t *h, const Err &e) {
  if (h) h->err = e.msg;
  else g_err = e.msg;
  return e.code;
}

// Closes the try block that wraps the body of every C entry point: a host exception
// becomes a status (ENOMEM or EINTERNAL) with its message for afmpb_last_error.
#define AFMPB_CATCH(handle) \
  catch (...) {             \
    return fail((handle), current_exception_err()); \
  }

void destroy_handle(afmpb_t *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->cf) destroy_handle(h->cf);                   // shares h's stream, owns no stream
  for (auto &g : h->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto &g : h->graph_io)
    if (g) cudaGraphExecDestroy(g);
  for (auto &g : h->graph_io_tmpl)
    if (g) cudaGraphDestroy(g);
  if (h->graph_gm) cudaGraphExecDestroy(h->graph_gm);
  if (h->graph_gm_tmpl) cudaGraphDestroy(h->graph_gm_tmpl);
  if (h->graph_cycle) cudaGraphExecDestroy(h->graph_cycle);
  h->arena.free_all();
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->h_wait_flag) cudaFreeHost(h->h_wait_flag);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_t0) cudaEventDestroy(h->ev_t0);
  if (h->ev_t1) cudaEventDestroy(h->ev_t1);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->side2) cudaStreamDestroy(h->side2);
  if (h->ev_fork2) cudaEventDestroy(h->ev_fork2);
  if (h->ev_join2) cudaEventDestroy(h->ev_join2);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Captures the product for one parts mask.  With io == true the graph also holds the
// gather of the caller's x and the scatter into the caller's y (kernel nodes whose pointer
// arguments afmpb_matvec_parts updates in place for new buffers), so that a product is a
// single graph launch: a plain kernel launch right before the far-field graph cost ~0.3 ms
// of start-up on a 163,842-node product.
// P2P runs beside the far-field chain (fork onto the low-priority side stream) for meshes
// up to this size; above it the two run one after the other.  Measured products, mixed
// precision, overlapped vs serial: 164k nodes 0.65 vs 0.73 ms, 200k 1.11 vs 1.46 ms, 2.1M
// 13.9 vs 14.3 ms, 10.5M 69.3 vs 62.0 ms (there the concurrent form contends for L2 with
// working sets far above it).
constexpr int64_t kOverlapMaxNodes = 4000000;

Err capture_product(afmpb_t *h, int parts, bool io = false, const float *x = nullptr, float *y = nullptr) {
  // The far-field chain (a long sequence of short, latency-bound launches) is captured
  // from a high-priority stream and P2P from a low-priority one: the kernel nodes keep the
  // priorities, so the block scheduler feeds the chain first and P2P fills the rest.
  int lo = 0, hi = 0;
  AFMPB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  cudaStream_t cap = nullptr;
  AFMPB_CUDA(cudaStreamCreateWithPriority(&cap, cudaStreamNonBlocking, hi));
  struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamDestroy(s); } } sg{cap};
  AFMPB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  Err e;
  if (io) e = enqueue_gather(h, cap, x);
  int cparts = parts;
  if (e.ok() && (parts & AFMPB_PART_FAR)) {
    if (overlap_p2p(h)) {
      cudaEventRecord(h->ev_fork, cap);
      cudaStreamWaitEvent(h->side, h->ev_fork, 0);
      e = enqueue_p2p(h, h->side);
      if (e.ok() && (parts & AFMPB_PART_NEAR)) {   // the near SpMV beside the rest of the chain
        e = enqueue_near_fold(h, h->side);
        cparts |= kNearFolded;
      }
      cudaEventRecord(h->ev_join, h->side);
      if (e.ok()) e = enqueue_far(h, cap);
      cudaStreamWaitEvent(cap, h->ev_join, 0);
    } else {
      e = enqueue_p2p(h, cap);
      if (e.ok()) e = enqueue_far(h, cap);
    }
  }
  if (e.ok()) e = enqueue_combine(h, cap, cparts);
  if (e.ok() && io) e = enqueue_scatter(h, cap, y);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cap, &g);
  if (!e.ok()) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
  cudaGraphExec_t *exec = io ? &h->graph_io[parts] : &h->graph[parts];
  ce = cudaGraphInstantiate(exec, g, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(g);
    return make_err(AFMPB_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
  }
  if (!io) {
    cudaGraphDestroy(g);
    return Err{};
  }
  // keep the template graph: its gather and scatter nodes are updated per call
  h->graph_io_tmpl[parts] = g;
  size_t nn = 0;
  AFMPB_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  AFMPB_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    AFMPB_CUDA(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp{};
    AFMPB_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
    if (kp.func == gather_kernel()) h->io_gather[parts] = nd;
    if (kp.func == scatter_kernel()) h->io_scatter[parts] = nd;
  }
  if (!h->io_gather[parts] || !h->io_scatter[parts]) return make_err(AFMPB_ECUDA, "captured product: gather/scatter node missing");
  h->io_x[parts] = x;
  h->io_y[parts] = y;
  return Err{};
}

// The single-launch product on caller buffers (caller order in and out).
Err product_io(afmpb_t *h, int parts, const float *x, float *y) {
  if (!h->graph_io[parts]) {
    AFMPB_TRY(capture_product(h, parts, true, x, y));
  } else {
    if (x != h->io_x[parts]) {
      cudaKernelNodeParams kp{};
      AFMPB_CUDA(cudaGraphKernelNodeGetParams(h->io_gather[parts], &kp));
      int64_t n = h->n;
      const int32_t *perm = h->d_perm;
      float2 *xs = h->d_xs;
      void *args[] = {&n, &perm, (void *)&x, &xs};
      kp.kernelParams = args;
      kp.extra = nullptr;
      AFMPB_CUDA(cudaGraphExecKernelNodeSetParams(h->graph_io[parts], h->io_gather[parts], &kp));
      h->io_x[parts] = x;
    }
    if (y != h->io_y[parts]) {
      cudaKernelNodeParams kp{};
      AFMPB_CUDA(cudaGraphKernelNodeGetParams(h->io_scatter[parts], &kp));
      int64_t n = h->n;
      const int32_t *perm = h->d_perm;
      const float *ys = h->d_ys;
      void *args[] = {&n, &perm, (void *)&ys, (void *)&y};
      kp.kernelParams = args;
      kp.extra = nullptr;
      AFMPB_CUDA(cudaGraphExecKernelNodeSetParams(h->graph_io[parts], h->io_scatter[parts], &kp));
      h->io_y[parts] = y;
    }
  }
  AFMPB_CUDA(cudaGraphLaunch(h->graph_io[parts], h->stream));
  return Err{};
}

Err check_params(const afmpb_mesh *mesh, double eps_in, double eps_out, double kappa, int order, double tol,
                 const afmpb_options *o) {
  if (!mesh) return make_err(AFMPB_EINVAL, "mesh is NULL");
  if (!(eps_in > 0) || !(eps_out > 0) || !std::isfinite(eps_in) || !std::isfinite(eps_out))
    return make_err(AFMPB_EINVAL, "eps_in and eps_out must be positive and finite");
  if (!(kappa >= 0) || !std::isfinite(kappa)) return make_err(AFMPB_EINVAL, "kappa must be >= 0 and finite");
  if (order < 2 || order > kMaxOrder) return make_err(AFMPB_EINVAL, "fmm_order must be in [2, 8]");
  if (!(tol > 0) || !std::isfinite(tol)) return make_err(AFMPB_EINVAL, "tol must be positive");
  if (o) {
    if ((o->leaf_cap < 0 && o->leaf_cap != AFMPB_LEAF_CAP_AUTO) || (o->restart < 0 && o->restart != AFMPB_RESTART_NONE) ||
        o->max_restart < 0 || o->max_level < 0 || o->max_level > kMaxLevel)
      return make_err(AFMPB_EINVAL, "negative option or max_level above 20");
    if (o->orth != 0 && o->orth != AFMPB_ORTH_ONE_REDUCTION) return make_err(AFMPB_EINVAL, "orth must be 0 or 1");
    if (o->m2l_method != 0 && o->m2l_method != AFMPB_M2L_PLANE_WAVE)
      return make_err(AFMPB_EINVAL, "m2l_method must be 0 or 1");
    if (o->abs_tol < 0 || !(o->near_c >= 0)) return make_err(AFMPB_EINVAL, "abs_tol and near_c must be >= 0");
    if (o->precision != 0 && o->precision != 1) return make_err(AFMPB_EINVAL, "precision must be 0 or 1");
    if (o->restart > 4096) return make_err(AFMPB_EINVAL, "restart above 4096");
    if (o->charge_fmm < 0 || o->charge_fmm > 2) return make_err(AFMPB_EINVAL, "charge_fmm must be 0, 1 or 2");
  }
  return Err{};
}

Err create_impl(afmpb_t *h, const afmpb_mesh *mesh, const afmpb_charges *ch) {
  auto t0 = std::chrono::steady_clock::now();
  AFMPB_CUDA(cudaGetDevice(&h->device));
  AFMPB_TRY(alloc_wait_flag(h));
  if (h->opt.stream) {
    h->stream = (cudaStream_t)h->opt.stream;
  } else {
    AFMPB_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  keep_pool_memory();
  h->arena.stream = h->stream;
  {
    int lo = 0, hi = 0;
    AFMPB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    AFMPB_CUDA(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, lo));   // P2P: lowest
    AFMPB_CUDA(cudaStreamCreateWithPriority(&h->side2, cudaStreamNonBlocking, hi));  // P2L: with the chain
  }
  AFMPB_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  AFMPB_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  AFMPB_CUDA(cudaEventCreateWithFlags(&h->ev_fork2, cudaEventDisableTiming));
  AFMPB_CUDA(cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming));
  AFMPB_CUDA(cudaEventCreate(&h->ev_t0));
  AFMPB_CUDA(cudaEventCreate(&h->ev_t1));
  auto lap = [&](int i) {
    AFMPB_CUDA(cudaStreamSynchronize(h->stream));
    auto now = std::chrono::steady_clock::now();
    h->ms_create[i] = std::chrono::duration<double, std::milli>(now - t0).count();
    for (int k = 0; k < i; ++k) h->ms_create[i] -= h->ms_create[k];
    return Err{};
  };
  AFMPB_TRY(build_geometry(h, mesh));
  AFMPB_TRY(lap(0));
  AFMPB_TRY(build_tree(h));
  AFMPB_TRY(lap(1));
  AFMPB_TRY(build_near(h));
  AFMPB_TRY(lap(2));
  AFMPB_TRY(build_fmm(h));
  AFMPB_TRY(lap(3));
  auto &A = h->arena;
  AFMPB_TRY(A.alloc(&h->d_xs, h->n, "xs"));
  AFMPB_TRY(A.alloc(&h->d_ys, 2 * h->n, "ys"));
  AFMPB_TRY(A.alloc(&h->d_phi_far, h->n, "phi far"));
  AFMPB_TRY(A.alloc(&h->d_phi_near, h->n, "phi near"));
  AFMPB_CUDA(cudaMemsetAsync(h->d_xs, 0, sizeof(float2) * h->n, h->stream));
  if (ch && ch->n > 0) {
    h->natoms = ch->n;
    AFMPB_TRY(A.alloc(&h->d_atoms, 3 * ch->n, "atoms"));
    AFMPB_TRY(A.alloc(&h->d_q, ch->n, "charges"));
    AFMPB_CUDA(cudaMemcpyAsync(h->d_atoms, ch->xyz, sizeof(double) * 3 * ch->n, cudaMemcpyHostToDevice, h->stream));
    AFMPB_CUDA(cudaMemcpyAsync(h->d_q, ch->q, sizeof(double) * ch->n, cudaMemcpyHostToDevice, h->stream));
  }
  AFMPB_TRY(build_rhs(h));
  AFMPB_TRY(lap(4));
  AFMPB_TRY(capture_product(h, AFMPB_PART_ALL));
  AFMPB_TRY(lap(5));
  h->ms_setup = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return Err{};
}

}  // namespace

namespace afmpb {

bool overlap_p2p(const afmpb_t *h) { return h->n <= kOverlapMaxNodes; }
void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done.push_back(dev);
}

Err raise_smem_limit(const void *func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> limit;
  int dev = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int &cur = limit[{dev, func}];
  if (bytes <= cur) return Err{};
  AFMPB_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur = bytes;
  return Err{};
}

// The product for the solver: a graph that converts the FP64 Krylov vector v (Morton
// order) to the FP32 input itself, so that no separate launch precedes the graph.  The
// pointer argument of the conversion node is patched when v changes.
Err product_from64(afmpb_t *h, cudaStream_t s, const double *v) {
  if (!h->graph_gm) {
    int lo = 0, hi = 0;
    AFMPB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    cudaStream_t cap = nullptr;
    AFMPB_CUDA(cudaStreamCreateWithPriority(&cap, cudaStreamNonBlocking, hi));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamDestroy(s); } } sg{cap};
    AFMPB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    Err e = enqueue_to_xs(h, cap, v);
    if (e.ok()) e = enqueue_product_kernels(h, cap);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cap, &g);
    if (!e.ok() || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return e.ok() ? make_err(AFMPB_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce)) : e;
    }
    ce = cudaGraphInstantiate(&h->graph_gm, g, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(g);
      return make_err(AFMPB_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    }
    h->graph_gm_tmpl = g;
    size_t nn = 0;
    AFMPB_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    AFMPB_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      AFMPB_CUDA(cudaGraphNodeGetType(nd, &ty));
      if (ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp{};
      AFMPB_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
      if (kp.func == to_xs_kernel()) h->gm_to_xs = nd;
    }
    if (!h->gm_to_xs) return make_err(AFMPB_ECUDA, "captured solver product: conversion node missing");
    h->gm_src = v;
  } else if (v != h->gm_src) {
    cudaKernelNodeParams kp{};
    AFMPB_CUDA(cudaGraphKernelNodeGetParams(h->gm_to_xs, &kp));
    int64_t n = h->n;
    float2 *xs = h->d_xs;
    void *args[] = {&n, (void *)&v, &xs};
    kp.kernelParams = args;
    kp.extra = nullptr;
    AFMPB_CUDA(cudaGraphExecKernelNodeSetParams(h->graph_gm, h->gm_to_xs, &kp));
    h->gm_src = v;
  }
  AFMPB_CUDA(cudaGraphLaunch(h->graph_gm, s));
  return Err{};
}

// The product's kernels from d_xs to d_ys, enqueued on a capturing stream: P2P forked onto
// the low-priority side stream beside the far-field chain (up to kOverlapMaxNodes), then
// the combine.  Used by the GMRES cycle graph.
Err enqueue_product_kernels(afmpb_t *h, cudaStream_t cap) {
  Err e;
  int cparts = AFMPB_PART_ALL;
  if (overlap_p2p(h)) {
    cudaEventRecord(h->ev_fork, cap);
    cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    e = enqueue_p2p(h, h->side);
    if (e.ok()) {                                  // the near SpMV beside the rest of the chain
      e = enqueue_near_fold(h, h->side);
      cparts |= kNearFolded;
    }
    cudaEventRecord(h->ev_join, h->side);
    if (e.ok()) e = enqueue_far(h, cap);
    cudaStreamWaitEvent(cap, h->ev_join, 0);
  } else {
    e = enqueue_p2p(h, cap);
    if (e.ok()) e = enqueue_far(h, cap);
  }
  if (e.ok()) e = enqueue_combine(h, cap, cparts);
  return e;
}

// Launch shapes and work lists live in the captured graphs: after the tile tuner changes
// them, every graph is dropped (the solver's and the caller-buffer ones are captured again
// on their next use) and the full product is captured again.
Err recapture_products(afmpb_t *h) {
  AFMPB_CUDA(cudaStreamSynchronize(h->stream));
  for (int p = 0; p < 8; ++p) {
    if (h->graph[p]) cudaGraphExecDestroy(h->graph[p]);
    if (h->graph_io[p]) cudaGraphExecDestroy(h->graph_io[p]);
    if (h->graph_io_tmpl[p]) cudaGraphDestroy(h->graph_io_tmpl[p]);
    h->graph[p] = nullptr;
    h->graph_io[p] = nullptr;
    h->graph_io_tmpl[p] = nullptr;
    h->io_gather[p] = h->io_scatter[p] = nullptr;
    h->io_x[p] = nullptr;
    h->io_y[p] = nullptr;
  }
  if (h->graph_gm) cudaGraphExecDestroy(h->graph_gm);
  if (h->graph_gm_tmpl) cudaGraphDestroy(h->graph_gm_tmpl);
  h->graph_gm = nullptr;
  h->graph_gm_tmpl = nullptr;
  h->gm_to_xs = nullptr;
  h->gm_src = nullptr;
  if (h->graph_cycle) cudaGraphExecDestroy(h->graph_cycle);
  h->graph_cycle = nullptr;
  h->cycle_m = 0;
  return capture_product(h, AFMPB_PART_ALL);
}

Err product_sorted(afmpb_t *h, cudaStream_t s, int parts) {
  if (parts <= 0 || parts > AFMPB_PART_ALL) return make_err(AFMPB_EINVAL, "parts must be a non-empty AFMPB_PART_* mask");
  if (!h->graph[parts]) AFMPB_TRY(capture_product(h, parts));
  AFMPB_CUDA(cudaGraphLaunch(h->graph[parts], s));
  return Err{};
}
}  // namespace afmpb

namespace {

int default_leaf_cap(int precision) { return precision == 1 ? 80 : 192; }

Err build_handle(const afmpb_mesh *mesh, const afmpb_charges *charges, double eps_in, double eps_out, double kappa,
                 int fmm_order, double tol, const afmpb_options *options, int leaf_cap, afmpb_t **out) {
  afmpb_t *h = new (std::nothrow) afmpb_t();
  if (!h) return make_err(AFMPB_ENOMEM, "host allocation of the handle failed");
  h->n = mesh->n_nodes;
  h->nt = mesh->n_tris;
  h->eps_in = eps_in;
  h->eps_out = eps_out;
  h->kappa = kappa;
  h->ebar = eps_out / eps_in;
  h->alpha = 0.5 / h->ebar + 0.5;
  h->tol = tol;
  h->order = fmm_order;
  h->ncoef = fmm_order * fmm_order * fmm_order;
  if (options) h->opt = *options;
  h->opt.leaf_cap = leaf_cap;
  if (h->opt.restart == 0) h->opt.restart = 80;
  if (h->opt.max_restart == 0 && !(options && options->max_restart == 0 && options->restart != 0)) h->opt.max_restart = 5;
  if (h->opt.near_c == 0) h->opt.near_c = 2.0;
  if (h->opt.max_level == 0) h->opt.max_level = kMaxLevel;
  if (h->opt.m2l_tol == 0) h->opt.m2l_tol = 1e-5;
  Err e;
  try {
    e = create_impl(h, mesh, charges);
  } catch (...) {                                      // free what was built, then report
    e = current_exception_err();
  }
  if (!e.ok()) {
    destroy_handle(h);
    return e;
  }
  *out = h;
  return Err{};
}

}  // namespace

extern "C" {

afmpb_status afmpb_create(const afmpb_mesh *mesh, const afmpb_charges *charges, double eps_in, double eps_out,
                          double kappa, int fmm_order, double tol, const afmpb_options *options, afmpb_t **out) {
  try {
    if (!out) return fail(nullptr, make_err(AFMPB_EINVAL, "out is NULL"));
    *out = nullptr;
    Err e = check_params(mesh, eps_in, eps_out, kappa, fmm_order, tol, options);
    if (!e.ok()) return fail(nullptr, e);
    if (charges && charges->n > 0 && (!charges->xyz || !charges->q))
      return fail(nullptr, make_err(AFMPB_EINVAL, "charges->xyz and charges->q are required when charges->n > 0"));
    if (charges && charges->n < 0) return fail(nullptr, make_err(AFMPB_EINVAL, "charges->n < 0"));
    e = validate_mesh(mesh);
    if (!e.ok()) return fail(nullptr, e);
    const int prec = options ? options->precision : 0;
    const bool tune = options && options->leaf_cap == AFMPB_LEAF_CAP_AUTO;
    int cap = (options && options->leaf_cap > 0) ? options->leaf_cap : default_leaf_cap(prec);
    int cached = 0;
    if (tune) {
      cached = autotune_cached_cap(prec, fmm_order, kappa, mesh->n_nodes);
      if (cached) cap = cached;
    }
    afmpb_t *h = nullptr;
    e = build_handle(mesh, charges, eps_in, eps_out, kappa, fmm_order, tol, options, cap, &h);
    if (!e.ok()) return fail(nullptr, e);
    if (tune && !cached) {
      afmpb_autotune_report rep{};
      try {
        e = autotune_leaf_cap(h, &rep);
      } catch (...) {
        e = current_exception_err();
      }
      if (!e.ok()) {
        destroy_handle(h);
        return fail(nullptr, e);
      }
      if (rep.best_cap != cap && rep.predicted_best_ms < 0.97 * rep.predicted_start_ms) {
        destroy_handle(h);
        h = nullptr;
        e = build_handle(mesh, charges, eps_in, eps_out, kappa, fmm_order, tol, options, rep.best_cap, &h);
        if (!e.ok()) return fail(nullptr, e);
      }
      try {
        e = autotune_tiles(h, &rep);
      } catch (...) {
        e = current_exception_err();
      }
      if (!e.ok()) {
        destroy_handle(h);
        return fail(nullptr, e);
      }
      autotune_cache_tiles(h);
      h->autotuned = true;
      h->tune = rep;
    } else if (tune) {
      autotune_cached_tiles(h);            // the size class was tuned before: its tile shapes
    }
    *out = h;
    return AFMPB_OK;
  } AFMPB_CATCH(nullptr)
}

}  // extern "C"

namespace {
// A bounded device wait of earlier work on the handle expired (the flag is set without a
// synchronisation once that work has finished): report it once and clear it.
bool take_wait_expiry(afmpb_t *h) {
  if (!h->h_wait_flag) return false;
  volatile int *f = h->h_wait_flag;
  if (!*f) return false;
  *f = 0;
  return true;
}
const char *kExpiredEarlier =
    "a bounded device wait of an earlier product on this handle expired; its result is invalid "
    "(reported once; nothing was queued by this call)";
}  // namespace

extern "C" {

afmpb_status afmpb_matvec_parts(afmpb_t *h, const float *x, float *y, int parts) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    if (!x || !y) return fail(h, make_err(AFMPB_EINVAL, "x and y must be device pointers"));
    if (x == y) return fail(h, make_err(AFMPB_EINVAL, "x and y must not overlap"));
    if (parts <= 0 || parts > AFMPB_PART_ALL) return fail(h, make_err(AFMPB_EINVAL, "parts must be a non-empty AFMPB_PART_* mask"));
    if (take_wait_expiry(h)) return fail(h, make_err(AFMPB_ETIMEOUT, kExpiredEarlier));
    Err e = product_io(h, parts, x, y);
    return e.ok() ? AFMPB_OK : fail(h, e);
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_matvec(afmpb_t *h, const float *x, float *y) { return afmpb_matvec_parts(h, x, y, AFMPB_PART_ALL); }

afmpb_status afmpb_matvec_host(afmpb_t *h, const float *x, float *y) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    if (!x || !y) return fail(h, make_err(AFMPB_EINVAL, "x and y must be host pointers"));
    if (take_wait_expiry(h)) return fail(h, make_err(AFMPB_ETIMEOUT, kExpiredEarlier));
    const size_t bytes = sizeof(float) * 2 * h->n;
    Err e;
    if (!h->d_xhost_stage) {
      e = h->arena.alloc(&h->d_xhost_stage, 2 * h->n, "host stage x");
      if (e.ok()) e = h->arena.alloc(&h->d_yhost_stage, 2 * h->n, "host stage y");
      if (!e.ok()) return fail(h, e);
    }
    cudaError_t ce = cudaMemcpyAsync(h->d_xhost_stage, x, bytes, cudaMemcpyHostToDevice, h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, std::string("H2D: ") + cudaGetErrorString(ce)));
    e = product_io(h, AFMPB_PART_ALL, h->d_xhost_stage, h->d_yhost_stage);
    if (!e.ok()) return fail(h, e);
    ce = cudaMemcpyAsync(y, h->d_yhost_stage, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, std::string("D2H: ") + cudaGetErrorString(ce)));
    if (take_wait_expiry(h))
      return fail(h, make_err(AFMPB_ETIMEOUT, "a bounded device wait of this product expired; y is invalid"));
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_sync(afmpb_t *h) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    cudaError_t ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, std::string("stream: ") + cudaGetErrorString(ce)));
    if (take_wait_expiry(h))
      return fail(h, make_err(AFMPB_ETIMEOUT, "a bounded device wait of work queued on this handle expired; "
                                              "the products queued since the last report are invalid"));
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_inject_wait_expiry(afmpb_t *h) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    if (!h->h_wait_flag) return fail(h, make_err(AFMPB_ESTATE, "the handle has no wait flag"));
    cudaError_t ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, std::string("stream: ") + cudaGetErrorString(ce)));
    *(volatile int *)h->h_wait_flag = 1;
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_solve(afmpb_t *h, double *f, double *hh, afmpb_solve_info *info) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    if (h->natoms == 0) return fail(h, make_err(AFMPB_ESTATE, "the handle was created without charges"));
    if (take_wait_expiry(h)) return fail(h, make_err(AFMPB_ETIMEOUT, kExpiredEarlier));
    Err e = run_solve(h, info);
    if (!e.ok() && e.code != AFMPB_ENOCONV) return fail(h, e);
    if (f || hh) {
      std::vector<double> xs(2 * h->n);
      std::vector<int32_t> perm(h->n);
      cudaError_t ce = cudaMemcpyAsync(xs.data(), h->d_sol, sizeof(double) * 2 * h->n, cudaMemcpyDeviceToHost, h->stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(perm.data(), h->d_perm, sizeof(int32_t) * h->n, cudaMemcpyDeviceToHost, h->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
      if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, cudaGetErrorString(ce)));
      for (int64_t p = 0; p < h->n; ++p) {
        if (f) f[perm[p]] = xs[p];
        if (hh) hh[perm[p]] = xs[h->n + p];
      }
    }
    return e.ok() ? AFMPB_OK : fail(h, e);
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_solve_batch(afmpb_t *const *hs, int k, double *const *f, double *const *hh,
                               afmpb_solve_info *infos, afmpb_status *statuses) {
  afmpb_t *h0 = (hs && k > 0) ? hs[0] : nullptr;
  try {
    if (!hs || k < 1 || k > AFMPB_BATCH_MAX)
      return fail(nullptr, make_err(AFMPB_EINVAL, "a batch takes 1 to AFMPB_BATCH_MAX handles"));
    for (int i = 0; i < k; ++i) {
      if (!hs[i]) return fail(nullptr, make_err(AFMPB_EINVAL, "a handle of the batch is NULL"));
      if (hs[i]->natoms == 0)
        return fail(hs[i], make_err(AFMPB_ESTATE, "a handle of the batch was created without charges"));
      if (hs[i]->device != h0->device) return fail(hs[i], make_err(AFMPB_EINVAL, "the handles of a batch share one device"));
      for (int j = 0; j < i; ++j)
        if (hs[j] == hs[i]) return fail(hs[i], make_err(AFMPB_EINVAL, "a handle appears twice in the batch"));
    }
    for (int i = 0; i < k; ++i)
      if (take_wait_expiry(hs[i])) return fail(hs[i], make_err(AFMPB_ETIMEOUT, kExpiredEarlier));
    Err e = run_solve_batch(hs, k, infos, statuses);
    if (!e.ok() && e.code != AFMPB_ENOCONV) return fail(h0, e);
    for (int i = 0; i < k; ++i) {
      afmpb_t *h = hs[i];
      double *fi = f ? f[i] : nullptr, *hi = hh ? hh[i] : nullptr;
      if (!fi && !hi) continue;
      std::vector<double> xs(2 * h->n);
      std::vector<int32_t> perm(h->n);
      cudaError_t ce = cudaMemcpyAsync(xs.data(), h->d_sol, sizeof(double) * 2 * h->n, cudaMemcpyDeviceToHost, h->stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(perm.data(), h->d_perm, sizeof(int32_t) * h->n, cudaMemcpyDeviceToHost, h->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
      if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, cudaGetErrorString(ce)));
      for (int64_t p = 0; p < h->n; ++p) {
        if (fi) fi[perm[p]] = xs[p];
        if (hi) hi[perm[p]] = xs[h->n + p];
      }
    }
    return e.ok() ? AFMPB_OK : fail(h0, e);
  } AFMPB_CATCH(h0)
}

afmpb_status afmpb_energy(afmpb_t *h, double *E) {
  try {
    if (!h || !E) return fail(h, make_err(AFMPB_EINVAL, "handle and output are required"));
    Err e = run_energy(h, E);
    return e.ok() ? AFMPB_OK : fail(h, e);
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_energy_noalloc(afmpb_t *h, double *E) {
  try {
    if (!h || !E) return fail(h, make_err(AFMPB_EINVAL, "handle and output are required"));
    Err e = run_energy_noalloc(h, E);
    return e.ok() ? AFMPB_OK : fail(h, e);
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_rhs(afmpb_t *h, double *b) {
  try {
    if (!h || !b) return fail(h, make_err(AFMPB_EINVAL, "handle and output are required"));
    std::vector<double> bs(2 * h->n);
    std::vector<int32_t> perm(h->n);
    cudaError_t ce = cudaMemcpyAsync(bs.data(), h->d_b, sizeof(double) * 2 * h->n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(perm.data(), h->d_perm, sizeof(int32_t) * h->n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, cudaGetErrorString(ce)));
    for (int64_t p = 0; p < h->n; ++p) {
      b[perm[p]] = bs[p];
      b[h->n + perm[p]] = bs[h->n + p];
    }
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_get_geometry(afmpb_t *h, double *area, double *normals, double *rho) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    cudaError_t ce = cudaSuccess;
    if (area) ce = cudaMemcpyAsync(area, h->d_area64, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess && normals)
      ce = cudaMemcpyAsync(normals, h->d_nrm64, sizeof(double) * 3 * h->n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess && rho) ce = cudaMemcpyAsync(rho, h->d_rho64, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, cudaGetErrorString(ce)));
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_get_near(afmpb_t *h, int64_t *rowptr, int32_t *col, float *coef, uint8_t *whole) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    const int64_t n = h->n;
    std::vector<int64_t> ptr(n + 1);
    std::vector<int32_t> c(h->nnz), perm(n);
    std::vector<float4> cf(h->nnz);
    std::vector<uint8_t> fl(h->nnz);
    cudaError_t ce = cudaMemcpyAsync(ptr.data(), h->d_near_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(c.data(), h->d_near_col, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(cf.data(), h->d_near_coef, sizeof(float4) * h->nnz, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(fl.data(), h->d_near_full, h->nnz, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(perm.data(), h->d_perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, cudaGetErrorString(ce)));
    std::vector<int64_t> iperm(n);
    for (int64_t p = 0; p < n; ++p) iperm[perm[p]] = p;
    int64_t k = 0;
    if (rowptr) rowptr[0] = 0;
    for (int64_t o = 0; o < n; ++o) {
      const int64_t p = iperm[o];
      for (int64_t j = ptr[p]; j < ptr[p + 1]; ++j, ++k) {
        if (col) col[k] = perm[c[j]];
        if (whole) whole[k] = fl[j];
        if (coef) {
          coef[4 * k] = cf[j].x;
          coef[4 * k + 1] = cf[j].y;
          coef[4 * k + 2] = cf[j].z;
          coef[4 * k + 3] = cf[j].w;
        }
      }
      if (rowptr) rowptr[o + 1] = k;
    }
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_get_tree(afmpb_t *h, int32_t *box_level, int32_t *box_anchor, int32_t *box_range,
                            int32_t *box_parent, int32_t *perm, int64_t *u_ptr, int32_t *u_idx, int64_t *v_ptr,
                            int32_t *v_idx, int64_t *w_ptr, int32_t *w_idx, int64_t *x_ptr, int32_t *x_idx) {
  try {
    if (!h) return fail(nullptr, make_err(AFMPB_EINVAL, "handle is NULL"));
    const auto &T = h->shape;
    const int nb = T.nbox;
    cudaStream_t s = h->stream;
    cudaError_t ce = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (dst && ce == cudaSuccess && bytes) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    };
    cp(box_level, h->d_box_level, sizeof(int32_t) * nb);
    cp(box_parent, h->d_box_parent, sizeof(int32_t) * nb);
    cp(perm, h->d_perm, sizeof(int32_t) * h->n);
    cp(u_ptr, h->d_u_ptr, sizeof(int64_t) * (nb + 1));
    cp(u_idx, h->d_u_idx, sizeof(int32_t) * T.n_u);
    cp(v_ptr, h->d_v_ptr, sizeof(int64_t) * (nb + 1));
    cp(v_idx, h->d_v_idx, sizeof(int32_t) * T.n_v);
    cp(w_ptr, h->d_w_ptr, sizeof(int64_t) * (nb + 1));
    cp(w_idx, h->d_w_idx, sizeof(int32_t) * T.n_w);
    cp(x_ptr, h->d_x_ptr, sizeof(int64_t) * (nb + 1));
    cp(x_idx, h->d_x_idx, sizeof(int32_t) * T.n_x);
    std::vector<int4> anc;
    std::vector<int32_t> beg, end;
    if (box_anchor) {
      anc.resize(nb);
      cp(anc.data(), h->d_box_anchor, sizeof(int4) * nb);
    }
    if (box_range) {
      beg.resize(nb);
      end.resize(nb);
      cp(beg.data(), h->d_box_begin, sizeof(int32_t) * nb);
      cp(end.data(), h->d_box_end, sizeof(int32_t) * nb);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return fail(h, make_err(AFMPB_ECUDA, cudaGetErrorString(ce)));
    for (int b = 0; b < nb; ++b) {
      if (box_anchor) {
        box_anchor[3 * b] = anc[b].x;
        box_anchor[3 * b + 1] = anc[b].y;
        box_anchor[3 * b + 2] = anc[b].z;
      }
      if (box_range) {
        box_range[2 * b] = beg[b];
        box_range[2 * b + 1] = end[b];
      }
    }
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_get_info(const afmpb_t *h, afmpb_info *info) {
  try {
    if (!h || !info) return fail(nullptr, make_err(AFMPB_EINVAL, "handle and info are required"));
    std::memset(info, 0, sizeof(*info));
    const auto &T = h->shape;
    info->n_nodes = h->n;
    info->n_tris = h->nt;
    info->n_atoms = h->natoms;
    info->n_boxes = T.nbox;
    info->n_leaves = T.nleaf;
    info->n_levels = T.nlevel;
    info->nnz_near = h->nnz;
    info->n_list_u = T.n_u;
    info->n_list_v = T.n_v;
    info->n_list_w = T.n_w;
    info->n_list_x = T.n_x;
    info->n_p2p_pairs = T.n_p2p_pairs;
    info->n_m2l_pairs = h->n_m2l_pairs;
    info->order = h->order;
    info->precision = h->opt.precision;
    info->device_bytes = (int64_t)h->arena.bytes;
    for (int d = 0; d < 3; ++d) info->root_center[d] = T.c0[d];
    info->root_half_width = T.w0;
    for (int i = 0; i < 6; ++i) info->ms_create[i] = h->ms_create[i];
    info->device_bytes_peak = (int64_t)h->arena.peak;
    info->leaf_cap = h->opt.leaf_cap;
    info->autotuned = h->autotuned ? 1 : 0;
    info->m2l_rank = h->m2l_rank;
    info->m2l_tables = h->m2l_ntables;
    if (h->cf) {
      // the charge FMM is built after the handle's own setup scratch is released
      info->charge_fmm = 1;
      info->charge_fmm_boxes = h->cf->shape.nbox;
      info->device_bytes += (int64_t)h->cf->arena.bytes;
      info->device_bytes_peak = std::max(info->device_bytes_peak, (int64_t)(h->arena.bytes + h->cf->arena.peak));
    }
    return AFMPB_OK;
  } AFMPB_CATCH(nullptr)
}

afmpb_status afmpb_get_autotune(const afmpb_t *h, afmpb_autotune_report *r) {
  try {
    if (!h || !r) return AFMPB_EINVAL;
    if (!h->autotuned) return AFMPB_ESTATE;
    *r = h->tune;
    return AFMPB_OK;
  } AFMPB_CATCH(nullptr)
}

afmpb_status afmpb_profile_product(afmpb_t *h, int reps, void *flush, size_t flush_bytes, afmpb_profile *out) {
  try {
    if (!h || !out || reps <= 0) return fail(h, make_err(AFMPB_EINVAL, "handle, reps > 0 and out are required"));
    std::memset(out, 0, sizeof(*out));
    cudaStream_t s = h->stream;
    if (!h->d_prof_x) {
      Err e = h->arena.alloc(&h->d_prof_x, 2 * h->n, "profile x");
      if (e.ok()) e = h->arena.alloc(&h->d_prof_y, 2 * h->n, "profile y");
      if (!e.ok()) return fail(h, e);
    }
    // input: the last product result, in caller order (contents do not change timing)
    {
      Err e = enqueue_scatter(h, s, h->d_prof_x);
      if (!e.ok()) return fail(h, e);
    }
    std::vector<double> acc;
    std::vector<std::string> names;
    std::vector<int> launches;
    for (int r = 0; r < reps; ++r) {
      if (flush && flush_bytes) cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
      StageTimer tm;
      tm.s = s;
      cudaEvent_t start = nullptr;
      cudaEventCreate(&start);
      cudaEventRecord(start, s);
      Err e = enqueue_gather(h, s, h->d_prof_x);
      if (e.ok()) tm.mark("gather", 1);
      if (e.ok()) e = enqueue_far(h, s, &tm);
      if (e.ok()) e = enqueue_p2p(h, s);
      if (e.ok()) tm.mark("p2p", 1);
      if (e.ok()) e = enqueue_combine(h, s, AFMPB_PART_ALL);
      if (e.ok()) tm.mark("combine", 1);
      if (e.ok()) e = enqueue_scatter(h, s, h->d_prof_y);
      if (e.ok()) tm.mark("scatter", 1);
      cudaError_t ce = cudaStreamSynchronize(s);
      if (!e.ok() || ce != cudaSuccess) {
        cudaEventDestroy(start);
        return fail(h, e.ok() ? make_err(AFMPB_ECUDA, cudaGetErrorString(ce)) : e);
      }
      if (r == 0) {
        names = tm.names;
        launches = tm.launches;
        acc.assign(names.size(), 0.0);
      }
      cudaEvent_t prev = start;
      for (size_t i = 0; i < tm.ends.size() && i < acc.size(); ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, prev, tm.ends[i]);
        acc[i] += ms;
        prev = tm.ends[i];
      }
      cudaEventDestroy(start);
    }
    out->n_stages = (int)std::min<size_t>(names.size(), AFMPB_MAX_STAGES);
    int kernels = 0;
    for (int i = 0; i < out->n_stages; ++i) {
      std::strncpy(out->name[i], names[i].c_str(), 15);
      out->ms[i] = acc[i] / reps;
      out->launches[i] = launches[i];
      kernels += launches[i];
    }
    // the captured product (overlapped P2P) runs the near correction as a kernel of its own
    // on the P2P branch and an elementwise combine, where the stages above run one k_combine
    out->kernels_per_product = kernels + (overlap_p2p(h) ? 1 : 0);
    // graph replays (the path afmpb_matvec takes), same flush between repetitions
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double tot = 0.0;
    for (int r = 0; r < reps; ++r) {
      if (flush && flush_bytes) cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
      cudaEventRecord(a, s);
      Err e = product_sorted(h, s, AFMPB_PART_ALL);
      cudaEventRecord(b, s);
      if (!e.ok()) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return fail(h, e);
      }
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      tot += ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    out->ms_graph = tot / reps;
    return AFMPB_OK;
  } AFMPB_CATCH(h)
}

afmpb_status afmpb_destroy(afmpb_t *h) {
  try {
    destroy_handle(h);
    return AFMPB_OK;
  } AFMPB_CATCH(nullptr)
}

const char *afmpb_last_error(const afmpb_t *h) { return h ? h->err.c_str() : g_err.c_str(); }

size_t afmpb_estimate_bytes(int64_t n_nodes, int64_t n_atoms, int fmm_order, const afmpb_options *o) {
  if (n_nodes <= 0 || fmm_order < 2 || fmm_order > kMaxOrder) return 0;
  // the smallest candidate of the autotuner gives the most boxes
  const int cap = (o && o->leaf_cap > 0) ? o->leaf_cap
                  : (o && o->leaf_cap == AFMPB_LEAF_CAP_AUTO) ? 32 : ((o && o->precision == 1) ? 80 : 192);
  const int m = (o && o->restart > 0) ? o->restart : (o && o->restart == AFMPB_RESTART_NONE) ? AFMPB_RESTART_NONE_MAX : 80;
  const size_t n = (size_t)n_nodes, n3 = (size_t)fmm_order * fmm_order * fmm_order;
  const size_t nbox = 3 * (n / (size_t)std::max(cap / 2, 1) + 64);
  size_t b = 0;
  b += n * (3 * 8 + 8 + 3 * 8 + 8 + 2 * 16 + 8 + 4 + 4 + 2 * 16 + 8 + 2 * 4 + 4 * 16);   // nodes
  b += n * 3 * 16;                                          // near-field setup: hi/lo coordinates, normals
  b += 2 * n * (3 * 4 + 3 * 8 + 4 + 16);                    // triangles (+ FP32 facet normals at setup)
  const double c = (o && o->near_c > 0) ? o->near_c : 2.0;
  const size_t per_row = (size_t)std::ceil(80.0 * (c / 2.0) * (c / 2.0));             // isosurface meshes ~70
  b += n * per_row * (4 + 16 + 1) + 8 * (n + 1);                                        // near CSR
  b += nbox * (2 * 2 * n3 * 4 + 64 + 27 * 4 + 200 * 4 * 2);                             // boxes, lists
  b += 316 * n3 * n3 * 4 * 14;                                                          // M2L tables
  b += (size_t)(m + 1) * 2 * n * 8 + 8 * 2 * n * 8;                                     // GMRES
  b += (size_t)std::max<int64_t>(n_atoms, 0) * 32 * 2;
  const int cfm = o ? o->charge_fmm : 0;
  if (n_atoms > 0 && (cfm == 2 || (cfm == 0 && (double)n_nodes * (double)n_atoms > AFMPB_CHARGE_FMM_PAIRS))) {
    const size_t nu = n + (size_t)n_atoms;                                             // charge FMM
    const size_t nbu = 3 * (nu / (size_t)std::max(cap / 2, 1) + 64);
    b += nu * 160 + nbu * (2 * 2 * n3 * 4 + 64 + 27 * 4 + 200 * 4 * 2) + 316 * n3 * n3 * 4 * 14;
  }
  return b + (64u << 20);
}

const char *afmpb_version(void) { return "afmpb-gb300 0.1.0 (sm_103a)"; }

afmpb_status afmpb_selftest_bounded_wait(int spin_limit, int *expired) {
  try {
    if (!expired || spin_limit < 1 || spin_limit > (1 << 26))
      return fail(nullptr, make_err(AFMPB_EINVAL, "spin_limit must be in [1, 2^26] and expired non-NULL"));
    *expired = 0;
    Err e = selftest_bounded_wait(spin_limit, expired);
    return e.ok() ? AFMPB_OK : fail(nullptr, e);
  } AFMPB_CATCH(nullptr)
}

}  // extern "C"
