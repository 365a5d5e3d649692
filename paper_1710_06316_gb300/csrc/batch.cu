// batch.cu -- the work lists of a batched (lockstep) solve of several problems.
//
// Each problem keeps its own handle: tree, operators, expansions and Krylov state.  What a
// batch adds is one P2P launch and one tensor-core M2L launch per Arnoldi step for all of
// them.  The P2P units of every problem are merged into one list, ordered by cost across
// problems (unit.w = problem), so the resident blocks deal out the union longest-first;
// the target-stationary M2L items are concatenated (TSItem.req = problem).  Per-problem
// descriptors give the kernels each problem's arrays and its stop flag (gm[4] of its
// step state), so a problem that has converged stops costing P2P and M2L work.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace afmpb {

namespace {

// Unit of problem `req` with its cost (targets x sources, the measure the units were cut by).
__global__ void k_batch_units(int n, const int4 *__restrict__ in, int req, P2PReq q, int4 *__restrict__ out,
                              uint64_t *__restrict__ cost) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 u = in[i];
  const int b = q.leaves[u.x];
  const int64_t nt = q.bend[b] - q.bbeg[b];
  int64_t ns = 0;
  for (int j = u.y; j < u.z; ++j) {
    const int c = q.pidx[j];
    ns += q.bend[c] - q.bbeg[c];
  }
  out[i] = make_int4(u.x, u.y, u.z, req);
  cost[i] = (uint64_t)(nt * ns);
}

__global__ void k_batch_items(int n, const TSItem *__restrict__ in, int req, TSItem *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TSItem it = in[i];
  it.req = req;
  out[i] = it;
}

}  // namespace

BatchLists::~BatchLists() {
  for (void *p : bufs) cudaFreeAsync(p, stream);
  if (!bufs.empty()) cudaStreamSynchronize(stream);
}

Err BatchLists::alloc_bytes(void **p, size_t bytes, const char *what) {
  *p = nullptr;
  const cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return make_err(e == cudaErrorMemoryAllocation ? AFMPB_ENOMEM : AFMPB_ECUDA,
                    std::string("device allocation failed (") + what + "): " + cudaGetErrorString(e));
  }
  bufs.push_back(*p);
  return Err{};
}

Err build_batch_lists(afmpb_t *const *hs, int k, bool fuse_m2l, BatchLists &L) {
  cudaStream_t s = L.stream;
  std::vector<P2PReq> p2p(k);
  std::vector<TSReq> ts(k);
  std::vector<int *> gms(k);
  int64_t nunits = 0, nitems = 0;
  for (int i = 0; i < k; ++i) {
    afmpb_t *h = hs[i];
    const int *act = h->d_gm_int + 4;
    p2p[i] = p2p_req_of(h, act);
    gms[i] = h->d_gm_int;
    nunits += h->p2p_nunits;
    if (fuse_m2l) {
      ts[i].runs = h->d_ts_runs;
      ts[i].ent = h->d_ts_ent;
      ts[i].Mc16 = h->d_Mc16;
      ts[i].tiles = h->d_ts_tiles;
      ts[i].Lc = h->d_Lc;
      ts[i].active = act;
      nitems += h->ts_nitems;
    }
  }
  if (nunits > INT32_MAX || nitems > INT32_MAX) return make_err(AFMPB_EINVAL, "batch work lists exceed 2^31 entries");
  AFMPB_TRY(L.alloc(&L.d_p2p, k, "batch p2p descriptors"));
  AFMPB_TRY(L.alloc(&L.d_gms, k, "batch step states"));
  AFMPB_CUDA(cudaMemcpyAsync(L.d_p2p, p2p.data(), sizeof(P2PReq) * k, cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(L.d_gms, gms.data(), sizeof(int *) * k, cudaMemcpyHostToDevice, s));

  // P2P: every problem's units with their costs, sorted by cost (descending) across problems
  L.nunits = (int)nunits;
  int4 *units = nullptr;
  uint64_t *cost = nullptr, *cost_sorted = nullptr;
  AFMPB_TRY(L.alloc(&units, nunits, "batch p2p units unsorted"));
  AFMPB_TRY(L.alloc(&cost, nunits, "batch p2p unit costs"));
  AFMPB_TRY(L.alloc(&cost_sorted, nunits, "batch p2p unit costs sorted"));
  AFMPB_TRY(L.alloc(&L.d_units, nunits, "batch p2p units"));
  int64_t off = 0;
  for (int i = 0; i < k; ++i) {
    const int n = hs[i]->p2p_nunits;
    if (n == 0) continue;
    k_batch_units<<<div_up(n, 128), 128, 0, s>>>(n, hs[i]->d_p2p_units, i, p2p[i], units + off, cost + off);
    AFMPB_TRY(check_launch("k_batch_units"));
    off += n;
  }
  if (nunits > 0) {
    size_t tmp_bytes = 0;
    AFMPB_CUDA(cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp_bytes, cost, cost_sorted, units, L.d_units,
                                                         (int)nunits, 0, 64, s));
    void *tmp = nullptr;
    AFMPB_TRY(L.alloc_bytes(&tmp, tmp_bytes, "batch p2p sort scratch"));
    AFMPB_CUDA(cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, cost, cost_sorted, units, L.d_units,
                                                         (int)nunits, 0, 64, s));
  }

  // M2L: the items of every problem, tagged with it
  L.nitems = (int)nitems;
  if (fuse_m2l) {
    AFMPB_TRY(L.alloc(&L.d_ts, k, "batch m2l descriptors"));
    AFMPB_CUDA(cudaMemcpyAsync(L.d_ts, ts.data(), sizeof(TSReq) * k, cudaMemcpyHostToDevice, s));
    AFMPB_TRY(L.alloc(&L.d_items, nitems, "batch m2l items"));
    AFMPB_TRY(L.alloc(&L.d_items_run, nitems, "batch m2l running items"));
    AFMPB_TRY(L.alloc(&L.d_count, 1, "batch m2l running count"));
    off = 0;
    for (int i = 0; i < k; ++i) {
      const int n = hs[i]->ts_nitems;
      if (n == 0) continue;
      k_batch_items<<<div_up(n, 128), 128, 0, s>>>(n, hs[i]->d_ts_items, i, L.d_items + off);
      AFMPB_TRY(check_launch("k_batch_items"));
      off += n;
    }
  }
  AFMPB_CUDA(cudaStreamSynchronize(s));
  return Err{};
}

}  // namespace afmpb
