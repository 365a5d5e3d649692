// autotune.cu -- leaf-capacity and tile-shape autotuner (afmpb_options.leaf_cap =
// AFMPB_LEAF_CAP_AUTO).
//
// The leaf capacity s trades point-to-point work (list 1 and 3 pairs grow roughly like s)
// against far-field work (boxes and list-2 translations grow roughly like 1/s).  The tuner
//   1. calibrates the far field on the handle just built at a starting capacity s0: the
//      per-stage times of its product give the cost of one list-2 translation (the M2L
//      stage over its pair count) and of one box in the other tree passes (P2M, M2M, P2L,
//      L2L, L2P and the compressed-basis changes over the box count);
//   2. for every candidate s, builds only the octree and its lists over the same
//      geometry, and times the real P2P kernel on them;
//   3. predicts the product time  t(s) = t_P2P(s) + b * pairs_V(s) + c * boxes(s) + t_rest
//      and keeps the smallest.
// Then, on the handle at the chosen capacity, the tile shapes of the two heaviest kernels
// are picked by timing them: the P2P blocks kept resident per SM and the size of its work
// units, and the number of offsets per work item of the tensor-core M2L.
// The choices are cached per (precision, order, screened or not, log2 of the node count),
// so later handles of the same size class skip the tuning.
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace afmpb {

namespace {

constexpr int kCandidates[] = {32, 48, 64, 80, 96, 128, 160, 192, 256};

// Times the P2P kernel of a tree built at capacity `cap` over h's geometry.
Err time_candidate(afmpb_t *h, int cap, int reps, double *p2p_ms, int64_t *m2l_pairs, int *nbox) {
  afmpb_t *t = new (std::nothrow) afmpb_t();
  if (!t) return make_err(AFMPB_ENOMEM, "autotune: host allocation failed");
  struct Guard {
    afmpb_t *t;
    ~Guard() {
      if (t->stream) cudaStreamSynchronize(t->stream);
      t->arena.free_all();
      delete t;
    }
  } guard{t};
  // borrowed geometry (owned by h) and parameters
  t->n = h->n;
  t->nt = h->nt;
  t->order = h->order;
  t->ncoef = h->ncoef;
  t->kappa = h->kappa;
  t->ebar = h->ebar;
  t->opt = h->opt;
  t->opt.leaf_cap = cap;
  t->stream = h->stream;
  t->arena.stream = h->stream;
  t->d_xyz = h->d_xyz;
  t->d_rho64 = h->d_rho64;
  t->d_area64 = h->d_area64;
  t->d_nrm64 = h->d_nrm64;
  AFMPB_TRY(build_tree(t));
  AFMPB_TRY(t->arena.alloc(&t->d_xs, t->n, "autotune xs"));
  AFMPB_TRY(t->arena.alloc(&t->d_phi_near, t->n, "autotune phi"));
  AFMPB_CUDA(cudaMemsetAsync(t->d_xs, 0, sizeof(float2) * t->n, t->stream));
  AFMPB_TRY(enqueue_p2p(t, t->stream));                 // warm-up
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  AFMPB_CUDA(cudaEventCreate(&e0));
  AFMPB_CUDA(cudaEventCreate(&e1));
  Err err;
  cudaEventRecord(e0, t->stream);
  for (int r = 0; r < reps && err.ok(); ++r) err = enqueue_p2p(t, t->stream);
  cudaEventRecord(e1, t->stream);
  cudaError_t ce = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  AFMPB_TRY(err);
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(ce));
  *p2p_ms = ms / reps;
  *m2l_pairs = t->n_m2l_pairs;
  *nbox = t->shape.nbox;
  return Err{};
}

std::mutex g_cache_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_cache;
struct Tiles { int resident, units, runs; };
std::map<std::tuple<int, int, int, int, int>, Tiles> g_tile_cache;

// Mean time of `reps` launches of one stage on the handle's stream (after one warm-up).
template <class F>
Err time_stage(afmpb_t *h, int reps, F launch, double *ms) {
  AFMPB_TRY(launch());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  AFMPB_CUDA(cudaEventCreate(&e0));
  AFMPB_CUDA(cudaEventCreate(&e1));
  Err err;
  cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps && err.ok(); ++r) err = launch();
  cudaEventRecord(e1, h->stream);
  cudaError_t ce = cudaEventSynchronize(e1);
  float t = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  AFMPB_TRY(err);
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(ce));
  *ms = t / reps;
  return Err{};
}

std::tuple<int, int, int, int, int> cache_key(int precision, int order, double kappa, int64_t n) {
  int dev = 0;
  cudaGetDevice(&dev);
  return {dev, precision, order, kappa > 0 ? 1 : 0, (int)std::floor(std::log2((double)std::max<int64_t>(n, 1)))};
}

}  // namespace

// Tile shapes on the finished handle: P2P resident blocks per SM x work units per block,
// then the M2L offsets per item, each by timing the kernel itself.  The product graphs are
// captured again afterwards (they hold the launch shapes).
Err autotune_tiles(afmpb_t *h, afmpb_autotune_report *rep) {
  constexpr int kReps = 5;
  auto p2p = [&]() { return enqueue_p2p(h, h->stream); };
  double ms = 0, best_ms = 0;
  AFMPB_TRY(time_stage(h, kReps, p2p, &best_ms));
  rep->p2p_ms_default = best_ms;
  int best_r = h->p2p_resident, best_u = h->p2p_units_per_block;
  for (int u : {1, 2, 3, 4, 6}) {
    h->p2p_units_per_block = u;
    AFMPB_TRY(build_p2p_units(h));
    for (int r : {4, 5, 6}) {
      h->p2p_resident = r;
      AFMPB_TRY(time_stage(h, kReps, p2p, &ms));
      if (ms < best_ms) {
        best_ms = ms;
        best_r = r;
        best_u = u;
      }
    }
  }
  h->p2p_resident = best_r;
  h->p2p_units_per_block = best_u;
  AFMPB_TRY(build_p2p_units(h));
  rep->p2p_resident = best_r;
  rep->p2p_units_per_block = best_u;
  rep->p2p_ms_tuned = best_ms;
  if (m2l_ts_applies(h) && h->ts_nitems > 0) {
    auto m2l = [&]() { return enqueue_m2l_ts(h, h->stream); };
    AFMPB_TRY(time_stage(h, kReps, m2l, &best_ms));
    rep->m2l_ms_default = best_ms;
    int best_p = h->ts_runs_per_item;
    for (int per : {8, 16, 24, 32}) {
      h->ts_runs_per_item = per;
      AFMPB_TRY(cut_m2l_ts_items(h));
      AFMPB_TRY(time_stage(h, kReps, m2l, &ms));
      if (ms < best_ms) {
        best_ms = ms;
        best_p = per;
      }
    }
    h->ts_runs_per_item = best_p;
    AFMPB_TRY(cut_m2l_ts_items(h));
    rep->m2l_runs_per_item = best_p;
    rep->m2l_ms_tuned = best_ms;
  }
  return recapture_products(h);
}

void autotune_cache_tiles(const afmpb_t *h) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_tile_cache[cache_key(h->opt.precision, h->order, h->kappa, h->n)] =
      Tiles{h->p2p_resident, h->p2p_units_per_block, h->ts_runs_per_item};
}

// Applies the cached tile shapes of the handle's size class; false when there are none.
bool autotune_cached_tiles(afmpb_t *h) {
  Tiles t{};
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_tile_cache.find(cache_key(h->opt.precision, h->order, h->kappa, h->n));
    if (it == g_tile_cache.end()) return false;
    t = it->second;
  }
  h->p2p_resident = t.resident;
  h->p2p_units_per_block = t.units;
  h->ts_runs_per_item = t.runs;
  if (!build_p2p_units(h).ok()) return false;
  if (m2l_ts_applies(h) && h->ts_nitems > 0 && !cut_m2l_ts_items(h).ok()) return false;
  return recapture_products(h).ok();
}

int autotune_cached_cap(int precision, int order, double kappa, int64_t n) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_cache.find(cache_key(precision, order, kappa, n));
  return it == g_cache.end() ? 0 : it->second;
}

Err autotune_leaf_cap(afmpb_t *h, afmpb_autotune_report *rep) {
  const auto t0 = std::chrono::steady_clock::now();
  std::memset(rep, 0, sizeof(*rep));
  rep->start_cap = h->opt.leaf_cap;
  // 1. far-field calibration on the handle as built
  afmpb_profile prof{};
  if (afmpb_profile_product(h, 3, nullptr, 0, &prof) != AFMPB_OK) return make_err(AFMPB_ECUDA, "autotune: " + h->err);
  double m2l_ms = 0, box_ms = 0, p2p_ms = 0, rest_ms = 0;
  for (int i = 0; i < prof.n_stages; ++i) {
    const std::string nm = prof.name[i];
    if (nm == "m2l") m2l_ms += prof.ms[i];
    else if (nm == "p2m" || nm == "m2m" || nm == "p2l" || nm == "l2l" || nm == "l2p" || nm == "compress" ||
             nm == "expand")
      box_ms += prof.ms[i];
    else if (nm == "p2p") p2p_ms += prof.ms[i];
    else rest_ms += prof.ms[i];
  }
  const double b = h->n_m2l_pairs > 0 ? m2l_ms / (double)h->n_m2l_pairs : 0.0;
  const double c = h->shape.nbox > 0 ? box_ms / (double)h->shape.nbox : 0.0;
  rep->ms_per_m2l_pair = b;
  rep->ms_per_box = c;
  rep->ms_rest = rest_ms;
  // 2-3. candidates
  double best_t = 0;
  int best = h->opt.leaf_cap;
  for (int cap : kCandidates) {
    if (rep->n_candidates >= AFMPB_AUTOTUNE_MAX) break;
    if (cap >= h->n && cap != kCandidates[0]) break;   // one leaf already: larger caps are the same tree
    double tp = 0;
    int64_t pv = 0;
    int nb = 0;
    AFMPB_TRY(time_candidate(h, cap, 3, &tp, &pv, &nb));
    const double pred = tp + b * (double)pv + c * (double)nb + rest_ms;
    const int k = rep->n_candidates++;
    rep->cap[k] = cap;
    rep->p2p_ms[k] = tp;
    rep->predicted_ms[k] = pred;
    if (cap == rep->start_cap) rep->predicted_start_ms = pred;
    if (k == 0 || pred < best_t) {
      best_t = pred;
      best = cap;
    }
  }
  if (rep->predicted_start_ms == 0) rep->predicted_start_ms = p2p_ms + m2l_ms + box_ms + rest_ms;
  rep->best_cap = best;
  rep->predicted_best_ms = best_t;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[cache_key(h->opt.precision, h->order, h->kappa, h->n)] = best;
  }
  rep->ms_tuning = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return Err{};
}

}  // namespace afmpb
