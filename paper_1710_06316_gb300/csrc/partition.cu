// partition.cu -- the plan for one solve shared by several GPUs (host code only).
//
// The paper distributes one solve over many nodes (Sec. 3.3-3.4): the surface nodes, and
// with them the rows of the product and the entries of every Krylov vector, are split into
// ranges of the Morton order; each rank evaluates the rows of its nodes and needs from the
// other ranks
//   (a) the unknowns (f, h) of source nodes outside its range that its point-to-point pairs
//       (lists 1 and 3, and list 4 where it is summed directly or by P2L), and its near-field
//       rows read -- the halo, exchanged before every product (the near-field traffic that
//       dominates the paper's communication at scale, Sec. 5);
//   (b) the multipole expansions of list-2 source boxes it does not own, after the upward
//       pass; a box whose nodes lie on several ranks is shared: its expansion is the sum of
//       the ranks' partial expansions;
//   (c) the global sums of the Krylov inner products (one all-reduce per reduction).
// This file computes (a) and (b) from the octree and list arrays a handle exports
// (afmpb_get_tree, afmpb_get_near).  The split balances an estimate of each rank's work
// and cuts only between leaves, so that a leaf's targets stay on one rank.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "internal.cuh"

struct afmpb_plan_t {
  int nranks = 0;
  int64_t n_nodes = 0;
  std::vector<int64_t> cut;                        // [nranks + 1] node range boundaries
  std::vector<double> work;                        // [nranks]
  std::vector<std::vector<int64_t>> halo;          // per rank: sorted node positions read from others
  std::vector<std::vector<int32_t>> halo_owner;
  std::vector<std::vector<int64_t>> send;          // per rank: own nodes that others read, by destination
  std::vector<std::vector<int32_t>> send_dest;
  std::vector<std::vector<int32_t>> imports;       // per rank: list-2 source boxes it does not own
  std::vector<std::vector<int32_t>> import_owner;  // owner rank, or -1 for a shared box
  std::vector<std::vector<int32_t>> shared;        // per rank: shared boxes it contributes to
};

namespace {

using namespace afmpb;

int owner_of(const std::vector<int64_t> &cut, int64_t node) {
  return (int)(std::upper_bound(cut.begin(), cut.end(), node) - cut.begin()) - 1;
}

Err plan_impl(const afmpb_plan_input *in, int nranks, afmpb_plan_t *p) {
  const int64_t n = in->n_nodes, nb = in->n_boxes;
  p->nranks = nranks;
  p->n_nodes = n;
  auto lo = [&](int64_t b) { return (int64_t)in->box_range[2 * b]; };
  auto hi = [&](int64_t b) { return (int64_t)in->box_range[2 * b + 1]; };
  std::vector<char> is_leaf(nb, 1);
  for (int64_t b = 0; b < nb; ++b)
    if (in->box_parent[b] >= 0) is_leaf[in->box_parent[b]] = 0;
  // ---- work per leaf: its targets times the sources of lists 1, 3 and 4, plus its rows'
  //      near-field entries; leaves in Morton order of their node ranges
  std::vector<int64_t> leaves;
  for (int64_t b = 0; b < nb; ++b)
    if (is_leaf[b]) leaves.push_back(b);
  std::sort(leaves.begin(), leaves.end(), [&](int64_t a, int64_t c) { return lo(a) < lo(c); });
  std::vector<double> lw(leaves.size(), 0.0);
  for (size_t i = 0; i < leaves.size(); ++i) {
    const int64_t b = leaves[i], nt = hi(b) - lo(b);
    int64_t src = 0;
    for (int64_t j = in->u_ptr[b]; j < in->u_ptr[b + 1]; ++j) src += hi(in->u_idx[j]) - lo(in->u_idx[j]);
    for (int64_t j = in->w_ptr[b]; j < in->w_ptr[b + 1]; ++j) src += hi(in->w_idx[j]) - lo(in->w_idx[j]);
    for (int64_t a = b; a >= 0; a = in->box_parent[a])
      for (int64_t j = in->x_ptr[a]; j < in->x_ptr[a + 1]; ++j) src += hi(in->x_idx[j]) - lo(in->x_idx[j]);
    int64_t near = 0;
    if (in->near_ptr) near = in->near_ptr[hi(b)] - in->near_ptr[lo(b)];
    lw[i] = (double)nt * (double)src + (double)near;
  }
  // ---- the split: cumulative work cut at multiples of total / nranks, between leaves
  const double total = std::accumulate(lw.begin(), lw.end(), 0.0);
  p->cut.assign(nranks + 1, n);
  p->cut[0] = 0;
  p->work.assign(nranks, 0.0);
  {
    double acc = 0.0;
    int r = 0;
    for (size_t i = 0; i < leaves.size(); ++i) {
      // leaf i goes to the rank whose share its midpoint falls in (ranks stay ordered)
      const double mid = acc + 0.5 * lw[i];
      while (r + 1 < nranks && mid > total * (double)(r + 1) / nranks) p->cut[++r] = lo(leaves[i]);
      p->work[r] += lw[i];
      acc += lw[i];
    }
    for (int q = r + 1; q <= nranks; ++q) p->cut[q] = n;   // ranks left without leaves are empty
  }
  // ---- halo: source nodes outside the rank's range, from the point-to-point lists (and
  //      list 4, summed directly or by P2L at the rank's boxes) and the near-field rows
  p->halo.assign(nranks, {});
  p->halo_owner.assign(nranks, {});
  p->send.assign(nranks, {});
  p->send_dest.assign(nranks, {});
  p->imports.assign(nranks, {});
  p->import_owner.assign(nranks, {});
  p->shared.assign(nranks, {});
  std::vector<int64_t> stamp(n, -1);
  for (int r = 0; r < nranks; ++r) {
    const int64_t a = p->cut[r], e = p->cut[r + 1];
    std::vector<int64_t> &H = p->halo[r];
    auto add_range = [&](int64_t s0, int64_t s1) {
      for (int64_t t = s0; t < s1; ++t)
        if ((t < a || t >= e) && stamp[t] != r) {
          stamp[t] = r;
          H.push_back(t);
        }
    };
    for (size_t i = 0; i < leaves.size(); ++i) {
      const int64_t b = leaves[i];
      if (lo(b) < a || lo(b) >= e) continue;
      for (int64_t j = in->u_ptr[b]; j < in->u_ptr[b + 1]; ++j) add_range(lo(in->u_idx[j]), hi(in->u_idx[j]));
      for (int64_t j = in->w_ptr[b]; j < in->w_ptr[b + 1]; ++j) add_range(lo(in->w_idx[j]), hi(in->w_idx[j]));
    }
    // list 4: every box whose nodes touch the range (its own or an ancestor of its leaves)
    for (int64_t b = 0; b < nb; ++b) {
      if (hi(b) <= a || lo(b) >= e) continue;
      for (int64_t j = in->x_ptr[b]; j < in->x_ptr[b + 1]; ++j) add_range(lo(in->x_idx[j]), hi(in->x_idx[j]));
    }
    if (in->near_ptr)
      for (int64_t t = a; t < e; ++t)
        for (int64_t j = in->near_ptr[t]; j < in->near_ptr[t + 1]; ++j) add_range(in->near_col[j], in->near_col[j] + 1);
    std::sort(H.begin(), H.end());
    p->halo_owner[r].resize(H.size());
    for (size_t k = 0; k < H.size(); ++k) p->halo_owner[r][k] = owner_of(p->cut, H[k]);
    // ---- expansions: list-2 sources of the boxes whose nodes touch the range, unless the
    //      source lies inside the range; a source on several ranks is shared
    std::vector<int32_t> imp;
    for (int64_t b = 0; b < nb; ++b) {
      if (hi(b) <= a || lo(b) >= e) continue;
      if (hi(b) > lo(b) && (lo(b) < a || hi(b) > e)) p->shared[r].push_back((int32_t)b);
      for (int64_t j = in->v_ptr[b]; j < in->v_ptr[b + 1]; ++j) {
        const int32_t c = in->v_idx[j];
        if (lo(c) >= a && hi(c) <= e) continue;
        imp.push_back(c);
      }
    }
    std::sort(imp.begin(), imp.end());
    imp.erase(std::unique(imp.begin(), imp.end()), imp.end());
    p->imports[r] = imp;
    p->import_owner[r].resize(imp.size());
    for (size_t k = 0; k < imp.size(); ++k) {
      const int o0 = owner_of(p->cut, lo(imp[k])), o1 = owner_of(p->cut, hi(imp[k]) - 1);
      p->import_owner[r][k] = o0 == o1 ? o0 : -1;
    }
  }
  // ---- send lists: the transpose of the halos
  for (int r = 0; r < nranks; ++r)
    for (size_t k = 0; k < p->halo[r].size(); ++k) {
      const int o = p->halo_owner[r][k];
      p->send[o].push_back(p->halo[r][k]);
      p->send_dest[o].push_back(r);
    }
  for (int r = 0; r < nranks; ++r) {
    std::vector<size_t> ord(p->send[r].size());
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
      return p->send_dest[r][x] != p->send_dest[r][y] ? p->send_dest[r][x] < p->send_dest[r][y]
                                                      : p->send[r][x] < p->send[r][y];
    });
    std::vector<int64_t> s2(ord.size());
    std::vector<int32_t> d2(ord.size());
    for (size_t k = 0; k < ord.size(); ++k) {
      s2[k] = p->send[r][ord[k]];
      d2[k] = p->send_dest[r][ord[k]];
    }
    p->send[r] = std::move(s2);
    p->send_dest[r] = std::move(d2);
  }
  return Err{};
}

}  // namespace

extern "C" {

afmpb_status afmpb_plan_create(const afmpb_plan_input *in, int nranks, afmpb_plan_t **out) {
  try {
    if (!out) return AFMPB_EINVAL;
    *out = nullptr;
    if (!in || nranks < 1 || in->n_nodes < 1 || in->n_boxes < 1 || !in->box_range || !in->box_parent ||
        !in->u_ptr || !in->u_idx || !in->v_ptr || !in->v_idx || !in->w_ptr || !in->w_idx || !in->x_ptr ||
        !in->x_idx || (in->near_ptr && !in->near_col))
      return AFMPB_EINVAL;
    for (int64_t b = 0; b < in->n_boxes; ++b) {
      const int32_t l = in->box_range[2 * b], h = in->box_range[2 * b + 1], par = in->box_parent[b];
      if (l < 0 || h < l || h > in->n_nodes || par < -1 || par >= in->n_boxes) return AFMPB_EINVAL;
    }
    afmpb_plan_t *p = new (std::nothrow) afmpb_plan_t();
    if (!p) return AFMPB_ENOMEM;
    Err e = plan_impl(in, nranks, p);
    if (!e.ok()) {
      delete p;
      return e.code;
    }
    *out = p;
    return AFMPB_OK;
  } catch (...) {
    return current_exception_err().code;
  }
}

afmpb_status afmpb_plan_get_rank(const afmpb_plan_t *p, int rank, afmpb_plan_rank *info) {
  if (!p || !info || rank < 0 || rank >= p->nranks) return AFMPB_EINVAL;
  info->node_begin = p->cut[rank];
  info->node_end = p->cut[rank + 1];
  info->n_halo = (int64_t)p->halo[rank].size();
  info->n_send = (int64_t)p->send[rank].size();
  info->n_import_boxes = (int64_t)p->imports[rank].size();
  info->n_shared_boxes = (int64_t)p->shared[rank].size();
  info->work = p->work[rank];
  return AFMPB_OK;
}

afmpb_status afmpb_plan_get_halo(const afmpb_plan_t *p, int rank, int64_t *nodes, int32_t *owner) {
  if (!p || rank < 0 || rank >= p->nranks) return AFMPB_EINVAL;
  const auto &H = p->halo[rank];
  if (nodes) std::copy(H.begin(), H.end(), nodes);
  if (owner) std::copy(p->halo_owner[rank].begin(), p->halo_owner[rank].end(), owner);
  return AFMPB_OK;
}

afmpb_status afmpb_plan_get_send(const afmpb_plan_t *p, int rank, int64_t *nodes, int32_t *dest) {
  if (!p || rank < 0 || rank >= p->nranks) return AFMPB_EINVAL;
  if (nodes) std::copy(p->send[rank].begin(), p->send[rank].end(), nodes);
  if (dest) std::copy(p->send_dest[rank].begin(), p->send_dest[rank].end(), dest);
  return AFMPB_OK;
}

afmpb_status afmpb_plan_get_boxes(const afmpb_plan_t *p, int rank, int32_t *imports, int32_t *import_owner,
                                  int32_t *shared) {
  if (!p || rank < 0 || rank >= p->nranks) return AFMPB_EINVAL;
  if (imports) std::copy(p->imports[rank].begin(), p->imports[rank].end(), imports);
  if (import_owner) std::copy(p->import_owner[rank].begin(), p->import_owner[rank].end(), import_owner);
  if (shared) std::copy(p->shared[rank].begin(), p->shared[rank].end(), shared);
  return AFMPB_OK;
}

afmpb_status afmpb_plan_destroy(afmpb_plan_t *p) {
  delete p;
  return AFMPB_OK;
}

}  // extern "C"
