// tree.cu -- adaptive octree and the four interaction lists of the adaptive FMM.
//
// Nodes are sorted along a 63-bit Morton curve; a box is split while it holds more than
// leaf_cap nodes.  For every box the lists of Carrier, Greengard and Rokhlin are built
// (list 1 = U: adjacent leaves; list 2 = V: well-separated children of the parent's
// colleagues; list 3 = W: descendants of colleagues that are not adjacent but whose
// parent is; list 4 = X: the dual of W).  Following the paper's modified method
// (Sec. 3.2), list 3 is evaluated point to point like list 1, so the point-to-point
// source list of a leaf is U followed by W; list 4 is evaluated by source-to-local.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace afmpb {

__host__ __device__ inline uint64_t spread_bits3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffULL;
  x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}
__host__ __device__ inline uint64_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
  return (spread_bits3(ix) << 2) | (spread_bits3(iy) << 1) | spread_bits3(iz);
}

__global__ void k_morton(int64_t n, const double *__restrict__ xyz, double lox, double loy, double loz,
                         double inv_cell, uint64_t *__restrict__ key, int32_t *__restrict__ idx) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t top = (1u << kKeyBits) - 1;
  double c[3] = {(xyz[3 * v] - lox) * inv_cell, (xyz[3 * v + 1] - loy) * inv_cell, (xyz[3 * v + 2] - loz) * inv_cell};
  uint32_t q[3];
  for (int d = 0; d < 3; ++d) {
    double f = floor(c[d]);
    q[d] = f < 0 ? 0u : (f > (double)top ? top : (uint32_t)f);
  }
  key[v] = morton3(q[0], q[1], q[2]);
  idx[v] = (int32_t)v;
}

// Child boundaries of each splitting box at one level.
__global__ void k_split_count(int ls, int nl, int level, int leaf_cap, int max_level,
                              const uint64_t *__restrict__ key, const int32_t *__restrict__ bbeg,
                              const int32_t *__restrict__ bend, const uint64_t *__restrict__ bkey,
                              int32_t *__restrict__ bnd, int32_t *__restrict__ nch) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  int b = ls + i;
  int beg = bbeg[b], end = bend[b];
  if (end - beg <= leaf_cap || level >= max_level) {
    nch[i] = 0;
    return;
  }
  const int shift = 3 * (kKeyBits - (level + 1));
  const uint64_t base = bkey[b] << 3;
  int cnt = 0;
  bnd[9 * i] = beg;
  for (int o = 1; o < 8; ++o) {
    uint64_t target = base + o;
    int lo = beg, hi = end;   // first index with (key >> shift) >= target
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if ((key[mid] >> shift) < target) lo = mid + 1; else hi = mid;
    }
    bnd[9 * i + o] = lo;
  }
  bnd[9 * i + 8] = end;
  for (int o = 0; o < 8; ++o) cnt += bnd[9 * i + o + 1] > bnd[9 * i + o];
  nch[i] = cnt;
}

__global__ void k_split_write(int ls, int nl, int le, int level, const int32_t *__restrict__ bnd,
                              const int32_t *__restrict__ nch, const int32_t *__restrict__ off,
                              int32_t *blevel, int32_t *bparent, int32_t *bchild0, int32_t *bnchild,
                              int32_t *bbeg, int32_t *bend, int4 *banchor, uint64_t *bkey) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  int b = ls + i;
  if (nch[i] == 0) {
    bchild0[b] = -1;
    bnchild[b] = 0;
    return;
  }
  int c = le + off[i];
  bchild0[b] = c;
  bnchild[b] = nch[i];
  int4 a = banchor[b];
  uint64_t k = bkey[b] << 3;
  for (int o = 0; o < 8; ++o) {
    int s = bnd[9 * i + o], e = bnd[9 * i + o + 1];
    if (e <= s) continue;
    blevel[c] = level + 1;
    bparent[c] = b;
    bchild0[c] = -1;
    bnchild[c] = 0;
    bbeg[c] = s;
    bend[c] = e;
    banchor[c] = make_int4(2 * a.x + ((o >> 2) & 1), 2 * a.y + ((o >> 1) & 1), 2 * a.z + (o & 1), level + 1);
    bkey[c] = k + o;
    ++c;
  }
}

__global__ void k_box_geometry(int nbox, const int4 *__restrict__ anchor, double lox, double loy, double loz,
                               double w0, dbl4 *__restrict__ center) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int4 a = anchor[b];
  double w = ldexp(w0, -a.w);          // half width
  center[b] = dbl4{lox + (2.0 * a.x + 1.0) * w, loy + (2.0 * a.y + 1.0) * w, loz + (2.0 * a.z + 1.0) * w, w};
}

__global__ void k_colleagues(int nbox, const int4 *__restrict__ anchor, const uint64_t *__restrict__ bkey,
                             const int *__restrict__ lvl_start, int32_t *__restrict__ coll) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int4 a = anchor[b];
  int ls = lvl_start[a.w], le = lvl_start[a.w + 1];
  int lim = 1 << a.w;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        int slot = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);
        int x = a.x + dx, y = a.y + dy, z = a.z + dz;
        int found = -1;
        if (x >= 0 && y >= 0 && z >= 0 && x < lim && y < lim && z < lim) {
          uint64_t k = morton3(x, y, z);
          int lo = ls, hi = le;
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (bkey[mid] < k) lo = mid + 1; else hi = mid;
          }
          if (lo < le && bkey[lo] == k) found = lo;
        }
        coll[27 * b + slot] = found;
      }
}

// Closed boxes a and b touch or overlap.
__device__ __forceinline__ bool boxes_adjacent(int4 a, int4 b) {
  if (a.w > b.w) { int4 t = a; a = b; b = t; }
  int s = b.w - a.w;
  int lo, hi;
  lo = a.x << s; hi = (a.x + 1) << s; if (b.x + 1 < lo || b.x > hi) return false;
  lo = a.y << s; hi = (a.y + 1) << s; if (b.y + 1 < lo || b.y > hi) return false;
  lo = a.z << s; hi = (a.z + 1) << s; if (b.z + 1 < lo || b.z > hi) return false;
  return true;
}

constexpr int kStack = 8 * (kMaxLevel + 2);

// Lists 1 (same-level and finer part) and 3 for every leaf.  fill == false: count only.
__global__ void k_list_uw(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ coll,
                          const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                          const int4 *__restrict__ anchor, int64_t *__restrict__ ucnt,
                          int64_t *__restrict__ wcnt, const int64_t *__restrict__ uptr,
                          const int64_t *__restrict__ wptr, int32_t *__restrict__ uidx,
                          int32_t *__restrict__ widx, bool fill) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  int b = leaves[i];
  int4 ab = anchor[b];
  int64_t nu = 0, nw = 0;
  int64_t u0 = fill ? uptr[b] : 0, w0 = fill ? wptr[b] : 0;
  int stack[kStack];
  for (int ci = 0; ci < 27; ++ci) {
    int c = coll[27 * b + ci];
    if (c < 0) continue;
    if (c == b || nchild[c] == 0) {
      if (fill) uidx[u0 + nu] = c;
      ++nu;
      continue;
    }
    int sp = 0;
    for (int k = nchild[c] - 1; k >= 0; --k) stack[sp++] = child0[c] + k;
    while (sp > 0) {
      int d = stack[--sp];
      if (!boxes_adjacent(ab, anchor[d])) {
        if (fill) widx[w0 + nw] = d;
        ++nw;
      } else if (nchild[d] == 0) {
        if (fill) uidx[u0 + nu] = d;
        ++nu;
      } else {
        for (int k = nchild[d] - 1; k >= 0 && sp < kStack; --k) stack[sp++] = child0[d] + k;
      }
    }
  }
  if (!fill) {
    ucnt[b] = nu;
    wcnt[b] = nw;
  }
}

// List 2 for every box.
__global__ void k_list_v(int nbox, const int32_t *__restrict__ parent, const int32_t *__restrict__ coll,
                         const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                         const int4 *__restrict__ anchor, int64_t *__restrict__ vcnt,
                         const int64_t *__restrict__ vptr, int32_t *__restrict__ vidx, bool fill) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int p = parent[b];
  int64_t nv = 0, v0 = fill ? vptr[b] : 0;
  if (p >= 0) {
    int4 ab = anchor[b];
    for (int ci = 0; ci < 27; ++ci) {
      int c = coll[27 * p + ci];
      if (c < 0) continue;
      for (int k = 0; k < nchild[c]; ++k) {
        int d = child0[c] + k;
        int4 ad = anchor[d];
        if (abs(ad.x - ab.x) > 1 || abs(ad.y - ab.y) > 1 || abs(ad.z - ab.z) > 1) {
          if (fill) vidx[v0 + nv] = d;
          ++nv;
        }
      }
    }
  }
  if (!fill) vcnt[b] = nv;
}

__global__ void k_node_leaf(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ bbeg,
                            const int32_t *__restrict__ bend, int32_t *__restrict__ node_leaf) {
  int i = blockIdx.x;
  if (i >= nleaf) return;
  int b = leaves[i];
  for (int t = bbeg[b] + threadIdx.x; t < bend[b]; t += blockDim.x) node_leaf[t] = b;
}

// Morton-ordered node data: position relative to the leaf centre (exact box-centre
// differences keep FP32 relative to the leaf size), patch area; normal and patch radius.
__global__ void k_node_sorted(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ node_leaf,
                              const dbl4 *__restrict__ center, const double *__restrict__ xyz,
                              const double *__restrict__ area, const double *__restrict__ nrm,
                              const double *__restrict__ rho, float4 *__restrict__ pos, float4 *__restrict__ nr) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t o = perm[p];
  dbl4 c = center[node_leaf[p]];
  pos[p] = make_float4((float)(xyz[3 * o] - c.x), (float)(xyz[3 * o + 1] - c.y), (float)(xyz[3 * o + 2] - c.z),
                       (float)area[o]);
  nr[p] = make_float4((float)nrm[3 * o], (float)nrm[3 * o + 1], (float)nrm[3 * o + 2], (float)rho[o]);
}

__global__ void k_box_rho_leaf(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ bbeg,
                               const int32_t *__restrict__ bend, const int32_t *__restrict__ perm,
                               const double *__restrict__ rho, double *__restrict__ brho) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  int b = leaves[i];
  double r = 0.0;
  for (int t = bbeg[b]; t < bend[b]; ++t) r = fmax(r, rho[perm[t]]);
  brho[b] = r;
}

__global__ void k_box_rho_up(int ls, int nl, const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                             double *__restrict__ brho) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  int b = ls + i;
  if (nchild[b] == 0) return;
  double r = 0.0;
  for (int k = 0; k < nchild[b]; ++k) r = fmax(r, brho[child0[b] + k]);
  brho[b] = r;
}

namespace {

template <class T>
Err grow(afmpb_t *h, T **p, size_t used, size_t cap_new, const char *what) {
  T *q = nullptr;
  AFMPB_TRY(h->arena.alloc(&q, cap_new, what));
  if (*p && used) AFMPB_CUDA(cudaMemcpyAsync(q, *p, used * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
  if (*p) {
    AFMPB_CUDA(cudaStreamSynchronize(h->stream));
    h->arena.release(*p);
  }
  *p = q;
  return Err{};
}

template <class T>
Err to_host(std::vector<T> &v, const T *d, size_t count, cudaStream_t s) {
  v.resize(count);
  if (count) {
    cudaError_t e = cudaMemcpyAsync(v.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("D2H: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
  }
  return Err{};
}

template <class T>
Err to_device(afmpb_t *h, T **d, const std::vector<T> &v, const char *what) {
  AFMPB_TRY(h->arena.alloc(d, v.size(), what));
  if (!v.empty())
    AFMPB_CUDA(cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return Err{};
}

// exclusive scan of counts (host) into a CSR pointer array with a leading 0
std::vector<int64_t> csr_from_counts(const std::vector<int64_t> &cnt) {
  std::vector<int64_t> ptr(cnt.size() + 1, 0);
  for (size_t i = 0; i < cnt.size(); ++i) ptr[i + 1] = ptr[i] + cnt[i];
  return ptr;
}

}  // namespace

Err build_tree(afmpb_t *h) {
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  auto &A = h->arena;
  auto &T = h->shape;
  const int cap = h->opt.leaf_cap;
  const int maxL = h->opt.max_level;

  // ---- root cube: the tight bounding cube (a little padding so no node sits on the far
  //      face).  Node positions are stored relative to their leaf centre, so FP32 error
  //      scales with the leaf size, not with the root.
  std::vector<double> xyz(3 * n);
  AFMPB_CUDA(cudaMemcpyAsync(xyz.data(), h->d_xyz, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  {
    // per-part extents on the host cores, then the extent of the parts (min / max are
    // exact, so the result does not depend on the split)
    std::vector<double> part_ext(6 * (size_t)host_parts(n));
    const int parts = host_parallel(n, [&](int p, int64_t i0, int64_t i1) {
      double l[3] = {1e300, 1e300, 1e300}, u[3] = {-1e300, -1e300, -1e300};
      for (int64_t i = i0; i < i1; ++i)
        for (int d = 0; d < 3; ++d) {
          l[d] = std::min(l[d], xyz[3 * i + d]);
          u[d] = std::max(u[d], xyz[3 * i + d]);
        }
      for (int d = 0; d < 3; ++d) {
        part_ext[6 * p + d] = l[d];
        part_ext[6 * p + 3 + d] = u[d];
      }
    });
    for (int p = 0; p < parts; ++p)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], part_ext[6 * p + d]);
        hi[d] = std::max(hi[d], part_ext[6 * p + 3 + d]);
      }
  }
  double ext = 0;
  for (int d = 0; d < 3; ++d) {
    T.c0[d] = 0.5 * (lo[d] + hi[d]);
    ext = std::max(ext, 0.5 * (hi[d] - lo[d]));
  }
  double w0 = std::max(ext, 1e-6) * (1.0 + 1e-6);
  T.w0 = w0;
  const double lox = T.c0[0] - w0, loy = T.c0[1] - w0, loz = T.c0[2] - w0;

  // ---- Morton keys and a stable radix sort
  uint64_t *d_key_in = nullptr;
  int32_t *d_idx_in = nullptr;
  AFMPB_TRY(A.alloc(&d_key_in, n, "key_in"));
  AFMPB_TRY(A.alloc(&d_idx_in, n, "idx_in"));
  AFMPB_TRY(A.alloc(&h->d_key, n, "key"));
  AFMPB_TRY(A.alloc(&h->d_perm, n, "perm"));
  k_morton<<<div_up(n, 256), 256, 0, s>>>(n, h->d_xyz, lox, loy, loz, std::ldexp(1.0, kKeyBits) / (2.0 * w0),
                                          d_key_in, d_idx_in);
  AFMPB_TRY(check_launch("k_morton"));
  {
    size_t tmp_bytes = 0;
    AFMPB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, d_key_in, h->d_key, d_idx_in, h->d_perm,
                                               (int)n, 0, 3 * kKeyBits, s));
    uint8_t *tmp = nullptr;
    AFMPB_TRY(A.alloc(&tmp, tmp_bytes, "sort tmp"));
    AFMPB_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, d_key_in, h->d_key, d_idx_in, h->d_perm, (int)n,
                                               0, 3 * kKeyBits, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
    A.release(tmp);
  }
  A.release(d_key_in);
  A.release(d_idx_in);

  // ---- level-by-level adaptive split
  size_t capb = std::max<size_t>(1024, (size_t)(8 * (n / std::max(cap, 1) + 1)));
  int32_t *blevel = nullptr, *bparent = nullptr, *bchild0 = nullptr, *bnchild = nullptr, *bbeg = nullptr,
          *bend = nullptr;
  int4 *banchor = nullptr;
  uint64_t *bkey = nullptr;
  auto grow_all = [&](size_t used, size_t newcap) -> Err {
    AFMPB_TRY(grow(h, &blevel, used, newcap, "box_level"));
    AFMPB_TRY(grow(h, &bparent, used, newcap, "box_parent"));
    AFMPB_TRY(grow(h, &bchild0, used, newcap, "box_child0"));
    AFMPB_TRY(grow(h, &bnchild, used, newcap, "box_nchild"));
    AFMPB_TRY(grow(h, &bbeg, used, newcap, "box_begin"));
    AFMPB_TRY(grow(h, &bend, used, newcap, "box_end"));
    AFMPB_TRY(grow(h, &banchor, used, newcap, "box_anchor"));
    AFMPB_TRY(grow(h, &bkey, used, newcap, "box_key"));
    return Err{};
  };
  AFMPB_TRY(grow_all(0, capb));
  {
    int32_t zero = 0, minus1 = -1, nn = (int32_t)n;
    int4 a0 = make_int4(0, 0, 0, 0);
    uint64_t k0 = 0;
    AFMPB_CUDA(cudaMemcpyAsync(blevel, &zero, 4, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(bparent, &minus1, 4, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(bchild0, &minus1, 4, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(bnchild, &zero, 4, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(bbeg, &zero, 4, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(bend, &nn, 4, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(banchor, &a0, sizeof(int4), cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyAsync(bkey, &k0, 8, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
  }
  T.lvl_start = {0, 1};
  int32_t *d_bnd = nullptr, *d_nch = nullptr, *d_off = nullptr;
  size_t cap_lvl = 0;
  for (int level = 0;; ++level) {
    int ls = T.lvl_start[level], le = T.lvl_start[level + 1], nl = le - ls;
    if (level >= maxL || nl == 0) break;
    if ((size_t)nl > cap_lvl) {
      if (d_bnd) { A.release(d_bnd); A.release(d_nch); A.release(d_off); }
      cap_lvl = std::max<size_t>(2 * nl, 1024);
      AFMPB_TRY(A.alloc(&d_bnd, 9 * cap_lvl, "bnd"));
      AFMPB_TRY(A.alloc(&d_nch, cap_lvl, "nch"));
      AFMPB_TRY(A.alloc(&d_off, cap_lvl, "off"));
    }
    k_split_count<<<div_up(nl, 128), 128, 0, s>>>(ls, nl, level, cap, maxL, h->d_key, bbeg, bend, bkey, d_bnd,
                                                   d_nch);
    AFMPB_TRY(check_launch("k_split_count"));
    std::vector<int32_t> nch;
    AFMPB_TRY(to_host(nch, d_nch, nl, s));
    std::vector<int32_t> off(nl);
    int64_t total = 0;
    for (int i = 0; i < nl; ++i) { off[i] = (int32_t)total; total += nch[i]; }
    if (total == 0) break;
    if ((size_t)(le + total) > capb) {
      size_t nc = std::max<size_t>(2 * capb, (size_t)(le + total) + 1024);
      AFMPB_TRY(grow_all((size_t)le, nc));
      capb = nc;
    }
    AFMPB_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s));
    k_split_write<<<div_up(nl, 128), 128, 0, s>>>(ls, nl, le, level, d_bnd, d_nch, d_off, blevel, bparent, bchild0,
                                                   bnchild, bbeg, bend, banchor, bkey);
    AFMPB_TRY(check_launch("k_split_write"));
    T.lvl_start.push_back(le + (int)total);
  }
  if (d_bnd) { A.release(d_bnd); A.release(d_nch); A.release(d_off); }
  T.nlevel = (int)T.lvl_start.size() - 1;
  T.nbox = T.lvl_start.back();
  const int nbox = T.nbox;
  h->d_box_level = blevel; h->d_box_parent = bparent; h->d_box_child0 = bchild0; h->d_box_nchild = bnchild;
  h->d_box_begin = bbeg; h->d_box_end = bend; h->d_box_anchor = banchor; h->d_box_key = bkey;

  // ---- box geometry, leaves, colleagues
  AFMPB_TRY(A.alloc(&h->d_box_center, nbox, "box_center"));
  k_box_geometry<<<div_up(nbox, 256), 256, 0, s>>>(nbox, banchor, lox, loy, loz, w0, h->d_box_center);
  AFMPB_TRY(check_launch("k_box_geometry"));
  std::vector<int32_t> hn_child, hlevel, hparent, hbeg, hend;
  AFMPB_TRY(to_host(hn_child, bnchild, nbox, s));
  AFMPB_TRY(to_host(hlevel, blevel, nbox, s));
  std::vector<int32_t> leaves;
  for (int b = 0; b < nbox; ++b)
    if (hn_child[b] == 0) leaves.push_back(b);
  // leaves in Morton order of their node ranges
  AFMPB_TRY(to_host(hbeg, bbeg, nbox, s));
  std::sort(leaves.begin(), leaves.end(), [&](int a, int b) { return hbeg[a] < hbeg[b]; });
  T.nleaf = (int)leaves.size();
  AFMPB_TRY(to_device(h, &h->d_leaves, leaves, "leaves"));
  int *d_lvl_start = nullptr;
  AFMPB_TRY(to_device(h, &d_lvl_start, T.lvl_start, "lvl_start"));
  AFMPB_TRY(A.alloc(&h->d_colleague, 27 * (size_t)nbox, "colleague"));
  k_colleagues<<<div_up(nbox, 128), 128, 0, s>>>(nbox, banchor, bkey, d_lvl_start, h->d_colleague);
  AFMPB_TRY(check_launch("k_colleagues"));

  // ---- lists 1 (same level + finer) and 3 for leaves; list 2 for all boxes
  int64_t *d_cnt1 = nullptr, *d_cnt2 = nullptr;
  AFMPB_TRY(A.alloc(&d_cnt1, nbox, "cnt1"));
  AFMPB_TRY(A.alloc(&d_cnt2, nbox, "cnt2"));
  AFMPB_CUDA(cudaMemsetAsync(d_cnt1, 0, sizeof(int64_t) * nbox, s));
  AFMPB_CUDA(cudaMemsetAsync(d_cnt2, 0, sizeof(int64_t) * nbox, s));
  k_list_uw<<<div_up(T.nleaf, 64), 64, 0, s>>>(T.nleaf, h->d_leaves, h->d_colleague, bchild0, bnchild, banchor,
                                                d_cnt1, d_cnt2, nullptr, nullptr, nullptr, nullptr, false);
  AFMPB_TRY(check_launch("k_list_uw count"));
  std::vector<int64_t> ucnt, wcnt;
  AFMPB_TRY(to_host(ucnt, d_cnt1, nbox, s));
  AFMPB_TRY(to_host(wcnt, d_cnt2, nbox, s));
  std::vector<int64_t> u1ptr = csr_from_counts(ucnt), wptr = csr_from_counts(wcnt);
  int64_t *d_u1ptr = nullptr, *d_wptr = nullptr;
  int32_t *d_u1idx = nullptr;
  AFMPB_TRY(to_device(h, &d_u1ptr, u1ptr, "u1ptr"));
  AFMPB_TRY(to_device(h, &d_wptr, wptr, "wptr"));
  AFMPB_TRY(A.alloc(&d_u1idx, u1ptr.back(), "u1idx"));
  AFMPB_TRY(A.alloc(&h->d_w_idx, wptr.back(), "widx"));
  k_list_uw<<<div_up(T.nleaf, 64), 64, 0, s>>>(T.nleaf, h->d_leaves, h->d_colleague, bchild0, bnchild, banchor,
                                                nullptr, nullptr, d_u1ptr, d_wptr, d_u1idx, h->d_w_idx, true);
  AFMPB_TRY(check_launch("k_list_uw fill"));
  k_list_v<<<div_up(nbox, 128), 128, 0, s>>>(nbox, bparent, h->d_colleague, bchild0, bnchild, banchor, d_cnt1,
                                             nullptr, nullptr, false);
  AFMPB_TRY(check_launch("k_list_v count"));
  std::vector<int64_t> vcnt;
  AFMPB_TRY(to_host(vcnt, d_cnt1, nbox, s));
  std::vector<int64_t> vptr = csr_from_counts(vcnt);
  AFMPB_TRY(to_device(h, &h->d_v_ptr, vptr, "vptr"));
  AFMPB_TRY(A.alloc(&h->d_v_idx, vptr.back(), "vidx"));
  k_list_v<<<div_up(nbox, 128), 128, 0, s>>>(nbox, bparent, h->d_colleague, bchild0, bnchild, banchor, nullptr,
                                             h->d_v_ptr, h->d_v_idx, true);
  AFMPB_TRY(check_launch("k_list_v fill"));

  // ---- host: complete list 1 with its coarser half (transpose), list 4 = transpose of
  //      list 3, point-to-point list per leaf, M2L groups by (level, offset)
  std::vector<int32_t> u1idx, widx, vidx;
  AFMPB_TRY(to_host(u1idx, d_u1idx, u1ptr.back(), s));
  AFMPB_TRY(to_host(widx, h->d_w_idx, wptr.back(), s));
  AFMPB_TRY(to_host(vidx, h->d_v_idx, vptr.back(), s));
  A.release(d_u1idx);
  A.release(d_u1ptr);
  std::vector<std::vector<int32_t>> ucoarse(nbox), xl(nbox);
  for (int b = 0; b < nbox; ++b) {
    for (int64_t j = u1ptr[b]; j < u1ptr[b + 1]; ++j) {
      int c = u1idx[j];
      if (hlevel[c] > hlevel[b]) ucoarse[c].push_back(b);   // b is a coarser leaf adjacent to c
    }
    for (int64_t j = wptr[b]; j < wptr[b + 1]; ++j) xl[widx[j]].push_back(b);
  }
  std::vector<int64_t> uptr(nbox + 1, 0), xptr(nbox + 1, 0);
  for (int b = 0; b < nbox; ++b) {
    uptr[b + 1] = uptr[b] + (u1ptr[b + 1] - u1ptr[b]) + (int64_t)ucoarse[b].size();
    std::sort(xl[b].begin(), xl[b].end());
    xptr[b + 1] = xptr[b] + (int64_t)xl[b].size();
  }
  std::vector<int32_t> uidx(uptr.back()), xidx(xptr.back());
  for (int b = 0; b < nbox; ++b) {
    int64_t k = uptr[b];
    for (int64_t j = u1ptr[b]; j < u1ptr[b + 1]; ++j) uidx[k++] = u1idx[j];
    std::sort(ucoarse[b].begin(), ucoarse[b].end());
    for (int c : ucoarse[b]) uidx[k++] = c;
    std::copy(xl[b].begin(), xl[b].end(), xidx.begin() + xptr[b]);
  }
  AFMPB_TRY(to_device(h, &h->d_u_ptr, uptr, "uptr"));
  AFMPB_TRY(to_device(h, &h->d_u_idx, uidx, "uidx"));
  h->d_w_ptr = d_wptr;
  AFMPB_TRY(to_device(h, &h->d_x_ptr, xptr, "xptr"));
  AFMPB_TRY(to_device(h, &h->d_x_idx, xidx, "xidx"));
  // List 4 of a box is evaluated by P2P at the targets when the box holds no more nodes
  // than an expansion holds weights (n^3): the direct sum is then the cheaper route.
  // Otherwise it goes to the box's local expansion (P2L).  Either way each pair once.
  AFMPB_TRY(to_host(hend, bend, nbox, s));
  AFMPB_TRY(to_host(hparent, bparent, nbox, s));
  const int64_t x_direct_max = (int64_t)h->order * h->order * h->order;
  std::vector<char> x_direct(nbox, 0);
  h->h_xbox.clear();
  for (int b = 0; b < nbox; ++b) {
    if (xptr[b + 1] == xptr[b]) continue;
    if (hend[b] - hbeg[b] <= x_direct_max) x_direct[b] = 1;
    else h->h_xbox.push_back(b);
  }
  AFMPB_TRY(to_device(h, &h->d_xbox, h->h_xbox, "xbox"));

  // point-to-point source boxes per leaf: list 1, the leaves under each list-3 box
  // (node positions are stored relative to their own leaf, so P2P sources are leaves),
  // then the list-4 leaves of itself and its ancestors that are evaluated directly
  std::vector<int32_t> hchild0;
  AFMPB_TRY(to_host(hchild0, bchild0, nbox, s));
  std::vector<int64_t> pptr(T.nleaf + 1, 0);
  std::vector<int32_t> pidx;
  std::vector<double> cost(T.nleaf);
  int64_t pairs = 0;
  {
    // leaves in contiguous parts on the host threads, concatenated in order
    const int nparts = host_parts(T.nleaf);
    std::vector<std::vector<int32_t>> part(nparts);
    std::vector<int64_t> part_pairs(nparts, 0);
    host_parallel(T.nleaf, [&](int pt, int64_t i0, int64_t i1) {
      std::vector<int32_t> &px = part[pt];
      std::vector<int32_t> stack;
      int64_t pp = 0;
      for (int64_t i = i0; i < i1; ++i) {
        const int b = leaves[i];
        const int64_t nt_b = hend[b] - hbeg[b];
        const size_t start = px.size();
        int64_t src = 0;
        for (int64_t j = uptr[b]; j < uptr[b + 1]; ++j) { px.push_back(uidx[j]); src += hend[uidx[j]] - hbeg[uidx[j]]; }
        for (int a = b; a >= 0; a = hparent[a]) {
          if (!x_direct[a]) continue;
          for (int64_t j = xptr[a]; j < xptr[a + 1]; ++j) {
            px.push_back(xidx[j]);
            src += hend[xidx[j]] - hbeg[xidx[j]];
          }
        }
        for (int64_t j = wptr[b]; j < wptr[b + 1]; ++j) {
          stack.assign(1, widx[j]);
          while (!stack.empty()) {
            const int d = stack.back();
            stack.pop_back();
            if (hn_child[d] == 0) {
              px.push_back(d);
              src += hend[d] - hbeg[d];
            } else {
              for (int k = hn_child[d] - 1; k >= 0; --k) stack.push_back(hchild0[d] + k);
            }
          }
        }
        pptr[i + 1] = (int64_t)(px.size() - start);     // count; prefix-summed below
        // ascending source boxes: near-field setup looks a box up by binary search
        std::sort(px.begin() + start, px.end());
        pp += nt_b * src;
        // Relative time of the leaf's P2P block, for the longest-first order: tiles of up to
        // kP2PThreads targets, each thread slice walking its share of the sources, plus the
        // staging of every source per tile.  (A model of the two-targets-per-thread tiling
        // ordered the blocks worse: 0.335 vs 0.320 ms on the Kirkwood sphere.)
        const int64_t tile = std::max<int64_t>(1, std::min<int64_t>(nt_b, kP2PThreads));
        const int64_t slices = kP2PThreads / tile, ntiles = (nt_b + tile - 1) / tile;
        cost[i] = (double)ntiles * ((double)((src + slices - 1) / slices) + 0.25 * (double)src + 64.0);
      }
      part_pairs[pt] = pp;
    });
    for (int i = 0; i < T.nleaf; ++i) pptr[i + 1] += pptr[i];
    pidx.reserve(pptr[T.nleaf]);
    for (int pt = 0; pt < nparts; ++pt) {
      pidx.insert(pidx.end(), part[pt].begin(), part[pt].end());
      pairs += part_pairs[pt];
    }
  }
  AFMPB_TRY(to_device(h, &h->d_p2p_ptr, pptr, "p2p_ptr"));
  AFMPB_TRY(to_device(h, &h->d_p2p_idx, pidx, "p2p_idx"));
  {
    // Longest blocks first: the block scheduler then ends the launch on short blocks.
    std::vector<int32_t> order(T.nleaf);
    for (int i = 0; i < T.nleaf; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    AFMPB_TRY(to_device(h, &h->d_p2p_order, order, "p2p_order"));
  }
  T.n_u = (int64_t)uidx.size();
  T.n_v = (int64_t)vidx.size();
  T.n_w = (int64_t)widx.size();
  T.n_x = (int64_t)xidx.size();
  T.n_p2p_pairs = pairs - h->n;     // the diagonal t == p is skipped

  // M2L pairs grouped by (level, offset), each group's targets in box order: a counting
  // sort on the key level * 343 + offset code (stable, so target order is kept)
  {
    std::vector<int4> anc;
    AFMPB_TRY(to_host(anc, banchor, nbox, s));
    const int nkey = (T.nlevel + 1) * 343;
    const int64_t nv = vptr[nbox];
    std::vector<int32_t> key(nv);
    const int nparts = host_parts(nbox);
    std::vector<std::vector<int64_t>> pcount(nparts, std::vector<int64_t>(nkey, 0));
    host_parallel(nbox, [&](int pt, int64_t b0, int64_t b1) {
      std::vector<int64_t> &c = pcount[pt];
      for (int64_t b = b0; b < b1; ++b)
        for (int64_t j = vptr[b]; j < vptr[b + 1]; ++j) {
          const int cb = vidx[j];
          const int ox = anc[cb].x - anc[b].x, oy = anc[cb].y - anc[b].y, oz = anc[cb].z - anc[b].z;
          key[j] = anc[b].w * 343 + (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
          ++c[key[j]];
        }
    });
    // start of (key, part): keys in order, parts in box order within a key
    std::vector<int64_t> kcount(nkey + 1, 0);
    std::vector<std::vector<int64_t>> pstart(nparts, std::vector<int64_t>(nkey, 0));
    for (int k = 0; k < nkey; ++k) {
      int64_t run = kcount[k];
      for (int pt = 0; pt < nparts; ++pt) {
        pstart[pt][k] = run;
        run += pcount[pt][k];
      }
      kcount[k + 1] = run;
    }
    std::vector<int2> pairs_v(nv);
    host_parallel(nbox, [&](int pt, int64_t b0, int64_t b1) {
      std::vector<int64_t> &f = pstart[pt];
      for (int64_t b = b0; b < b1; ++b)
        for (int64_t j = vptr[b]; j < vptr[b + 1]; ++j) pairs_v[f[key[j]]++] = make_int2((int)b, vidx[j]);
    });
    h->m2l_groups.clear();
    for (int k = 0; k < nkey; ++k) {
      if (kcount[k + 1] == kcount[k]) continue;
      M2LGroup g;
      g.level = k / 343;
      g.offset = k % 343;               // raw code in [0, 343); mapped to a table slot in fmm.cu
      g.start = (int)kcount[k];
      g.count = (int)(kcount[k + 1] - kcount[k]);
      h->m2l_groups.push_back(g);
    }
    h->n_m2l_pairs = nv;
    AFMPB_TRY(to_device(h, &h->d_m2l_pairs, pairs_v, "m2l_pairs"));
  }

  // ---- Morton-ordered node arrays and box patch radii
  AFMPB_TRY(A.alloc(&h->d_node_leaf, n, "node_leaf"));
  k_node_leaf<<<T.nleaf, 128, 0, s>>>(T.nleaf, h->d_leaves, bbeg, bend, h->d_node_leaf);
  AFMPB_TRY(check_launch("k_node_leaf"));
  AFMPB_TRY(A.alloc(&h->d_pos, n, "pos"));
  AFMPB_TRY(A.alloc(&h->d_nrm, n, "nrm"));
  k_node_sorted<<<div_up(n, 256), 256, 0, s>>>(n, h->d_perm, h->d_node_leaf, h->d_box_center, h->d_xyz,
                                               h->d_area64, h->d_nrm64, h->d_rho64, h->d_pos, h->d_nrm);
  AFMPB_TRY(check_launch("k_node_sorted"));
  {
    std::vector<int32_t> leaf_index(nbox, -1);
    for (int i = 0; i < T.nleaf; ++i) leaf_index[leaves[i]] = i;
    AFMPB_TRY(to_device(h, &h->d_leaf_index, leaf_index, "leaf index"));
  }
  AFMPB_TRY(A.alloc(&h->d_box_rho, nbox, "box_rho"));
  k_box_rho_leaf<<<div_up(T.nleaf, 128), 128, 0, s>>>(T.nleaf, h->d_leaves, bbeg, bend, h->d_perm, h->d_rho64,
                                                      h->d_box_rho);
  AFMPB_TRY(check_launch("k_box_rho_leaf"));
  for (int level = T.nlevel - 2; level >= 0; --level) {
    int ls = T.lvl_start[level], nl = T.lvl_start[level + 1] - ls;
    k_box_rho_up<<<div_up(nl, 128), 128, 0, s>>>(ls, nl, bchild0, bnchild, h->d_box_rho);
    AFMPB_TRY(check_launch("k_box_rho_up"));
  }
  A.release(d_cnt1);
  A.release(d_cnt2);
  A.release(d_lvl_start);
  AFMPB_CUDA(cudaStreamSynchronize(s));
  return Err{};
}

}  // namespace afmpb
