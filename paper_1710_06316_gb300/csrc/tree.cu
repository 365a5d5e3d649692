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

// ---- device passes that turn the box arrays into lists (no host loop over boxes) ---------

// Extent of the node cloud: per-block minima and maxima, then one block folds the parts
// (min / max are exact, so the result does not depend on the partition).
constexpr int kExtThreads = 256;
__global__ void __launch_bounds__(kExtThreads) k_extent_part(int64_t n, const double *__restrict__ xyz,
                                                             double *__restrict__ part) {
  __shared__ double sh[6][kExtThreads];
  double l[3] = {1e300, 1e300, 1e300}, u[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const double v = xyz[3 * i + d];
      l[d] = fmin(l[d], v);
      u[d] = fmax(u[d], v);
    }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = l[d];
    sh[3 + d][threadIdx.x] = u[d];
  }
  __syncthreads();
  for (int s = kExtThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fmin(sh[d][threadIdx.x], sh[d][threadIdx.x + s]);
        sh[3 + d][threadIdx.x] = fmax(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kExtThreads) k_extent_final(int nblk, const double *__restrict__ part,
                                                               double *__restrict__ out) {
  __shared__ double sh[6][kExtThreads];
  double l[3] = {1e300, 1e300, 1e300}, u[3] = {-1e300, -1e300, -1e300};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      l[d] = fmin(l[d], part[6 * b + d]);
      u[d] = fmax(u[d], part[6 * b + 3 + d]);
    }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = l[d];
    sh[3 + d][threadIdx.x] = u[d];
  }
  __syncthreads();
  for (int s = kExtThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fmin(sh[d][threadIdx.x], sh[d][threadIdx.x + s]);
        sh[3 + d][threadIdx.x] = fmax(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_iota(int n, int32_t *__restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

// total[0] = off[nl - 1] + cnt[nl - 1] (the children of one level after the exclusive scan)
__global__ void k_level_total(int nl, const int32_t *__restrict__ off, const int32_t *__restrict__ cnt,
                              int64_t *__restrict__ total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) total[0] = nl > 0 ? (int64_t)off[nl - 1] + cnt[nl - 1] : 0;
}

__global__ void k_leaf_flags(int nbox, const int32_t *__restrict__ nchild, const int32_t *__restrict__ bbeg,
                             uint8_t *__restrict__ flag, int32_t *__restrict__ key) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  flag[b] = nchild[b] == 0;
  key[b] = bbeg[b];
}

__global__ void k_gather_i32(int n, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                             int32_t *__restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// Coarse half of list 1 and list 4, counted: a leaf b in list 1 of a finer leaf c puts c in
// b's list 1 as well (adjacency is symmetric); every box d in list 3 of a leaf b puts b in
// d's list 4 (the dual of list 3).
__global__ void k_dual_count(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ level,
                             const int64_t *__restrict__ u1ptr, const int32_t *__restrict__ u1idx,
                             const int64_t *__restrict__ wptr, const int32_t *__restrict__ widx,
                             int64_t *__restrict__ ucnt, int64_t *__restrict__ xcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  const int b = leaves[i];
  for (int64_t j = u1ptr[b]; j < u1ptr[b + 1]; ++j) {
    const int c = u1idx[j];
    if (level[c] > level[b]) atomicAdd((unsigned long long *)&ucnt[c], 1ull);
  }
  for (int64_t j = wptr[b]; j < wptr[b + 1]; ++j) atomicAdd((unsigned long long *)&xcnt[widx[j]], 1ull);
}

// own list-1 entries first (their order kept); cursors of the coarse part start behind them
__global__ void k_u_own(int nbox, const int64_t *__restrict__ u1ptr, const int32_t *__restrict__ u1idx,
                        const int64_t *__restrict__ uptr, int32_t *__restrict__ uidx, int64_t *__restrict__ seg_beg,
                        int64_t *__restrict__ cur) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const int64_t own = u1ptr[b + 1] - u1ptr[b];
  for (int64_t j = 0; j < own; ++j) uidx[uptr[b] + j] = u1idx[u1ptr[b] + j];
  seg_beg[b] = uptr[b] + own;
  cur[b] = uptr[b] + own;
}

__global__ void k_dual_fill(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ level,
                            const int64_t *__restrict__ u1ptr, const int32_t *__restrict__ u1idx,
                            const int64_t *__restrict__ wptr, const int32_t *__restrict__ widx,
                            int64_t *__restrict__ ucur, int32_t *__restrict__ uidx, int64_t *__restrict__ xcur,
                            int32_t *__restrict__ xidx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  const int b = leaves[i];
  for (int64_t j = u1ptr[b]; j < u1ptr[b + 1]; ++j) {
    const int c = u1idx[j];
    if (level[c] > level[b]) uidx[atomicAdd((unsigned long long *)&ucur[c], 1ull)] = b;
  }
  for (int64_t j = wptr[b]; j < wptr[b + 1]; ++j) {
    const int d = widx[j];
    xidx[atomicAdd((unsigned long long *)&xcur[d], 1ull)] = b;
  }
}

__global__ void k_copy_i64(int64_t n, const int64_t *__restrict__ src, int64_t *__restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

// whole list-1 row sizes: own entries (from the scanned pointers) + coarse entries; 0 at nbox
__global__ void k_u_rowsize(int nbox, const int64_t *__restrict__ u1ptr, const int64_t *__restrict__ coarse,
                            int64_t *__restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) out[b] = (u1ptr[b + 1] - u1ptr[b]) + coarse[b];
  else if (b == nbox) out[b] = 0;
}

// List 4 of a box goes point to point at the targets when the box holds no more nodes than
// an expansion holds weights (n^3): the direct sum is then the cheaper route; otherwise to
// the box's local expansion (P2L).
__global__ void k_x_route(int nbox, const int64_t *__restrict__ xptr, const int32_t *__restrict__ bbeg,
                          const int32_t *__restrict__ bend, int direct_max, uint8_t *__restrict__ direct,
                          uint8_t *__restrict__ p2l) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const bool has = xptr[b + 1] > xptr[b];
  const bool dir = has && bend[b] - bbeg[b] <= direct_max;
  direct[b] = dir;
  p2l[b] = has && !dir;
}

// Point-to-point source boxes of a leaf: list 1, the list-4 boxes of itself and its
// ancestors that are summed directly, and the leaves under each list-3 box (node positions
// are stored relative to their own leaf, so P2P sources are leaves).  fill == false counts
// boxes, source nodes, pairs and the block's relative cost (tiles of up to kP2PThreads
// targets, each thread slice walking its share of the sources, plus the staging of every
// source per tile, in quarter units).
__global__ void k_p2p_lists(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ bbeg,
                            const int32_t *__restrict__ bend, const int32_t *__restrict__ parent,
                            const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                            const int64_t *__restrict__ uptr, const int32_t *__restrict__ uidx,
                            const int64_t *__restrict__ xptr, const int32_t *__restrict__ xidx,
                            const uint8_t *__restrict__ x_direct, const int64_t *__restrict__ wptr,
                            const int32_t *__restrict__ widx, int64_t *__restrict__ cnt, int64_t *__restrict__ pairs,
                            uint64_t *__restrict__ cost, const int64_t *__restrict__ pptr, int32_t *__restrict__ pidx,
                            bool fill) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  const int b = leaves[i];
  int64_t k = fill ? pptr[i] : 0, nb = 0, src = 0;
  auto put = [&](int c) {
    if (fill) pidx[k + nb] = c;
    ++nb;
    src += bend[c] - bbeg[c];
  };
  for (int64_t j = uptr[b]; j < uptr[b + 1]; ++j) put(uidx[j]);
  for (int a = b; a >= 0; a = parent[a]) {
    if (!x_direct[a]) continue;
    for (int64_t j = xptr[a]; j < xptr[a + 1]; ++j) put(xidx[j]);
  }
  int stack[kStack];
  for (int64_t j = wptr[b]; j < wptr[b + 1]; ++j) {
    int sp = 0;
    stack[sp++] = widx[j];
    while (sp > 0) {
      const int d = stack[--sp];
      if (nchild[d] == 0) put(d);
      else
        for (int q = nchild[d] - 1; q >= 0 && sp < kStack; --q) stack[sp++] = child0[d] + q;
    }
  }
  if (fill) return;
  const int64_t nt = bend[b] - bbeg[b];
  cnt[i] = nb;
  pairs[i] = nt * src;
  const int64_t tile = max((int64_t)1, min(nt, (int64_t)kP2PThreads));
  const int64_t slices = kP2PThreads / tile, ntiles = (nt + tile - 1) / tile;
  cost[i] = (uint64_t)(ntiles * (4 * ((src + slices - 1) / slices) + src + 256));
}

// P2P work units: a leaf's source boxes cut into consecutive ranges of at most `budget`
// target-source pairs (a range holds at least one box), so that blocks of comparable cost
// can be dealt out statically.  fill == false counts the units of each leaf.
// unit = (leaf, first box entry, end box entry, pairs)
__global__ void k_p2p_units(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ bbeg,
                            const int32_t *__restrict__ bend, const int64_t *__restrict__ pptr,
                            const int32_t *__restrict__ pidx, int64_t budget, int64_t *__restrict__ cnt,
                            const int64_t *__restrict__ uptr, int4 *__restrict__ units, uint64_t *__restrict__ ucost,
                            bool fill) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  const int b = leaves[i];
  const int64_t nt = bend[b] - bbeg[b];
  int64_t k = fill ? uptr[i] : 0, nu = 0, acc = 0;
  int64_t start = pptr[i];
  for (int64_t j = pptr[i]; j < pptr[i + 1]; ++j) {
    const int c = pidx[j];
    const int64_t add = nt * (bend[c] - bbeg[c]);
    if (j > start && acc + add > budget) {
      if (fill) {
        units[k + nu] = make_int4(i, (int)start, (int)j, 0);
        ucost[k + nu] = (uint64_t)acc;
      }
      ++nu;
      start = j;
      acc = 0;
    }
    acc += add;
  }
  if (fill) {
    units[k + nu] = make_int4(i, (int)start, (int)pptr[i + 1], 0);
    ucost[k + nu] = (uint64_t)acc;
  }
  ++nu;
  if (!fill) cnt[i] = nu;
}

__global__ void k_gather_int4(int64_t n, const int32_t *__restrict__ idx, const int4 *__restrict__ src,
                              int4 *__restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// (level, offset) key and (target, source) pair of every list-2 entry, in box order
__global__ void k_m2l_keys(int nbox, const int64_t *__restrict__ vptr, const int32_t *__restrict__ vidx,
                           const int4 *__restrict__ anchor, uint32_t *__restrict__ key, uint64_t *__restrict__ pair) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const int4 ab = anchor[b];
  for (int64_t j = vptr[b]; j < vptr[b + 1]; ++j) {
    const int c = vidx[j];
    const int4 ac = anchor[c];
    key[j] = (uint32_t)(ab.w * 343 + (ac.x - ab.x + 3) * 49 + (ac.y - ab.y + 3) * 7 + (ac.z - ab.z + 3));
    pair[j] = ((uint64_t)(uint32_t)b << 32) | (uint32_t)c;
  }
}

__global__ void k_unpack_pairs(int64_t n, const uint64_t *__restrict__ pk, int2 *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_int2((int)(pk[i] >> 32), (int)(pk[i] & 0xffffffffu));
}

__global__ void k_leaf_index(int nleaf, const int32_t *__restrict__ leaves, int32_t *__restrict__ leaf_index) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nleaf) leaf_index[leaves[i]] = i;
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


}  // namespace

namespace {

// Runs one CUB device algorithm: the size query, scratch from the handle's arena, the
// call, and the scratch released once the stream has caught up.
template <class F>
Err cub_call(afmpb_t *h, const char *what, F f) {
  size_t bytes = 0;
  cudaError_t e = f(nullptr, bytes);
  if (e != cudaSuccess) return make_err(AFMPB_ECUDA, std::string(what) + " (size): " + cudaGetErrorString(e));
  uint8_t *tmp = nullptr;
  AFMPB_TRY(h->arena.alloc(&tmp, std::max<size_t>(bytes, 16), what));
  e = f(tmp, bytes);
  if (e != cudaSuccess) return make_err(AFMPB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  AFMPB_CUDA(cudaStreamSynchronize(h->stream));
  h->arena.release(tmp);
  return Err{};
}

template <class T>
Err read_one(T *out, const T *d, cudaStream_t s) {
  AFMPB_CUDA(cudaMemcpyAsync(out, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  return Err{};
}

// CSR pointers from per-row counts: cnt has rows + 1 entries with cnt[rows] = 0, ptr gets
// rows + 1 entries (exclusive scan); *total = ptr[rows].
Err csr_ptr(afmpb_t *h, const int64_t *cnt, int64_t rows, int64_t **ptr, int64_t *total, const char *what) {
  AFMPB_TRY(h->arena.alloc(ptr, rows + 1, what));
  int64_t *out = *ptr;
  AFMPB_TRY(cub_call(h, what, [&](void *t, size_t &bytes) {
    return cub::DeviceScan::ExclusiveSum(t, bytes, cnt, out, rows + 1, h->stream);
  }));
  return read_one(total, out + rows, h->stream);
}

// Sorts every row segment [beg[r], end[r]) of idx ascending, in place (rows of a few to a
// few hundred entries); entries outside the segments keep their place.
Err sort_rows(afmpb_t *h, int32_t *idx, int64_t nnz, const int64_t *beg, const int64_t *end, int64_t rows,
              const char *what) {
  if (nnz == 0 || rows == 0) return Err{};
  int32_t *tmp = nullptr;
  AFMPB_TRY(h->arena.alloc(&tmp, nnz, what));
  // entries outside every row segment are not written by the sort: start from a copy
  AFMPB_CUDA(cudaMemcpyAsync(tmp, idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, h->stream));
  AFMPB_TRY(cub_call(h, what, [&](void *t, size_t &bytes) {
    return cub::DeviceSegmentedSort::SortKeys(t, bytes, idx, tmp, nnz, rows, beg, end, h->stream);
  }));
  AFMPB_CUDA(cudaMemcpyAsync(idx, tmp, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, h->stream));
  AFMPB_CUDA(cudaStreamSynchronize(h->stream));
  h->arena.release(tmp);
  return Err{};
}

}  // namespace

// P2P work units over the handle's per-leaf source lists: a leaf's source boxes cut into
// consecutive ranges of at most `budget` pairs, about h->p2p_units_per_block units per
// resident block, longest first (a stable sort: equal costs keep leaf order).  Replaces
// earlier units; the tile tuner calls it again with other unit sizes.
Err build_p2p_units(afmpb_t *h) {
  auto &A = h->arena;
  cudaStream_t s = h->stream;
  const int nl = h->shape.nleaf;
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t pairs = h->shape.n_p2p_pairs + h->n;
  const int64_t budget =
      std::max<int64_t>(4096, pairs / ((int64_t)h->p2p_resident * sms * std::max(1, h->p2p_units_per_block)));
  int64_t *cnt = nullptr;
  AFMPB_TRY(A.alloc(&cnt, nl + 1, "p2p unit counts"));
  AFMPB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (nl + 1), s));
  k_p2p_units<<<div_up(nl, 128), 128, 0, s>>>(nl, h->d_leaves, h->d_box_begin, h->d_box_end, h->d_p2p_ptr,
                                              h->d_p2p_idx, budget, cnt, nullptr, nullptr, nullptr, false);
  AFMPB_TRY(check_launch("k_p2p_units count"));
  int64_t *d_uptr = nullptr, nunits = 0;
  AFMPB_TRY(csr_ptr(h, cnt, nl, &d_uptr, &nunits, "p2p unit ptr"));
  int4 *units = nullptr;
  uint64_t *ucost = nullptr, *ucost_sorted = nullptr;
  int32_t *uiota = nullptr, *uorder = nullptr;
  AFMPB_TRY(A.alloc(&units, nunits, "p2p units unsorted"));
  AFMPB_TRY(A.alloc(&ucost, nunits, "p2p unit cost"));
  AFMPB_TRY(A.alloc(&ucost_sorted, nunits, "p2p unit cost sorted"));
  AFMPB_TRY(A.alloc(&uiota, nunits, "p2p unit iota"));
  AFMPB_TRY(A.alloc(&uorder, nunits, "p2p unit order"));
  k_p2p_units<<<div_up(nl, 128), 128, 0, s>>>(nl, h->d_leaves, h->d_box_begin, h->d_box_end, h->d_p2p_ptr,
                                              h->d_p2p_idx, budget, nullptr, d_uptr, units, ucost, true);
  AFMPB_TRY(check_launch("k_p2p_units fill"));
  k_iota<<<div_up(nunits, 256), 256, 0, s>>>((int)nunits, uiota);
  AFMPB_TRY(check_launch("k_iota"));
  AFMPB_TRY(cub_call(h, "p2p unit order", [&](void *t, size_t &bytes) {
    return cub::DeviceRadixSort::SortPairsDescending(t, bytes, ucost, ucost_sorted, uiota, uorder, (int)nunits, 0, 64, s);
  }));
  if (h->d_p2p_units) A.release(h->d_p2p_units);
  AFMPB_TRY(A.alloc(&h->d_p2p_units, nunits, "p2p units"));
  k_gather_int4<<<div_up(nunits, 256), 256, 0, s>>>(nunits, uorder, units, h->d_p2p_units);
  AFMPB_TRY(check_launch("k_gather_int4"));
  h->p2p_nunits = (int)nunits;
  AFMPB_CUDA(cudaStreamSynchronize(s));
  for (void *q : {(void *)cnt, (void *)d_uptr, (void *)units, (void *)ucost, (void *)ucost_sorted, (void *)uiota,
                  (void *)uorder})
    A.release(q);
  return Err{};
}

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
  double lo[3], hi[3];
  {
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (n + kExtThreads - 1) / kExtThreads));
    double *d_part = nullptr, *d_ext = nullptr;
    AFMPB_TRY(A.alloc(&d_part, 6 * (size_t)nblk, "extent parts"));
    AFMPB_TRY(A.alloc(&d_ext, 6, "extent"));
    k_extent_part<<<nblk, kExtThreads, 0, s>>>(n, h->d_xyz, d_part);
    k_extent_final<<<1, kExtThreads, 0, s>>>(nblk, d_part, d_ext);
    AFMPB_TRY(check_launch("k_extent"));
    double ext6[6];
    AFMPB_CUDA(cudaMemcpyAsync(ext6, d_ext, sizeof(ext6), cudaMemcpyDeviceToHost, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
    A.release(d_part);
    A.release(d_ext);
    for (int d = 0; d < 3; ++d) {
      lo[d] = ext6[d];
      hi[d] = ext6[3 + d];
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
  AFMPB_TRY(cub_call(h, "morton sort", [&](void *t, size_t &bytes) {
    return cub::DeviceRadixSort::SortPairs(t, bytes, d_key_in, h->d_key, d_idx_in, h->d_perm, (int)n, 0,
                                           3 * kKeyBits, s);
  }));
  A.release(d_key_in);
  A.release(d_idx_in);

  // ---- level-by-level adaptive split (child offsets by a device scan; the host reads one
  //      count per level to size the box arrays)
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
  int64_t *d_total = nullptr;
  AFMPB_TRY(A.alloc(&d_total, 1, "level total"));
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
    AFMPB_TRY(cub_call(h, "level scan", [&](void *t, size_t &bytes) {
      return cub::DeviceScan::ExclusiveSum(t, bytes, d_nch, d_off, nl, s);
    }));
    k_level_total<<<1, 1, 0, s>>>(nl, d_off, d_nch, d_total);
    int64_t total = 0;
    AFMPB_TRY(read_one(&total, d_total, s));
    if (total == 0) break;
    if ((size_t)(le + total) > capb) {
      size_t nc = std::max<size_t>(2 * capb, (size_t)(le + total) + 1024);
      AFMPB_TRY(grow_all((size_t)le, nc));
      capb = nc;
    }
    k_split_write<<<div_up(nl, 128), 128, 0, s>>>(ls, nl, le, level, d_bnd, d_nch, d_off, blevel, bparent, bchild0,
                                                   bnchild, bbeg, bend, banchor, bkey);
    AFMPB_TRY(check_launch("k_split_write"));
    T.lvl_start.push_back(le + (int)total);
  }
  if (d_bnd) { A.release(d_bnd); A.release(d_nch); A.release(d_off); }
  A.release(d_total);
  T.nlevel = (int)T.lvl_start.size() - 1;
  T.nbox = T.lvl_start.back();
  const int nbox = T.nbox;
  h->d_box_level = blevel; h->d_box_parent = bparent; h->d_box_child0 = bchild0; h->d_box_nchild = bnchild;
  h->d_box_begin = bbeg; h->d_box_end = bend; h->d_box_anchor = banchor; h->d_box_key = bkey;

  // ---- box geometry; leaves (selected, then put in Morton order of their node ranges);
  //      colleagues
  AFMPB_TRY(A.alloc(&h->d_box_center, nbox, "box_center"));
  k_box_geometry<<<div_up(nbox, 256), 256, 0, s>>>(nbox, banchor, lox, loy, loz, w0, h->d_box_center);
  AFMPB_TRY(check_launch("k_box_geometry"));
  {
    uint8_t *flag = nullptr;
    int32_t *iota = nullptr, *sel = nullptr, *key = nullptr, *selkey = nullptr, *d_nsel = nullptr;
    AFMPB_TRY(A.alloc(&flag, nbox, "leaf flags"));
    AFMPB_TRY(A.alloc(&iota, nbox, "box iota"));
    AFMPB_TRY(A.alloc(&sel, nbox, "leaves unsorted"));
    AFMPB_TRY(A.alloc(&key, nbox, "leaf keys"));
    AFMPB_TRY(A.alloc(&selkey, nbox, "leaf keys selected"));
    AFMPB_TRY(A.alloc(&d_nsel, 1, "leaf count"));
    k_leaf_flags<<<div_up(nbox, 256), 256, 0, s>>>(nbox, bnchild, bbeg, flag, key);
    k_iota<<<div_up(nbox, 256), 256, 0, s>>>(nbox, iota);
    AFMPB_TRY(check_launch("k_leaf_flags"));
    AFMPB_TRY(cub_call(h, "leaf select", [&](void *t, size_t &bytes) {
      return cub::DeviceSelect::Flagged(t, bytes, iota, flag, sel, d_nsel, nbox, s);
    }));
    int32_t nleaf = 0;
    AFMPB_TRY(read_one(&nleaf, d_nsel, s));
    T.nleaf = nleaf;
    k_gather_i32<<<div_up(nleaf, 256), 256, 0, s>>>(nleaf, sel, key, selkey);
    AFMPB_TRY(check_launch("k_gather_i32"));
    AFMPB_TRY(A.alloc(&h->d_leaves, nleaf, "leaves"));
    int32_t *keys_out = key;                    // reused as the sorted-key output
    AFMPB_TRY(cub_call(h, "leaf sort", [&](void *t, size_t &bytes) {
      return cub::DeviceRadixSort::SortPairs(t, bytes, selkey, keys_out, sel, h->d_leaves, nleaf, 0, 32, s);
    }));
    for (void *q : {(void *)flag, (void *)iota, (void *)sel, (void *)key, (void *)selkey, (void *)d_nsel}) A.release(q);
  }
  int *d_lvl_start = nullptr;
  AFMPB_TRY(to_device(h, &d_lvl_start, T.lvl_start, "lvl_start"));
  AFMPB_TRY(A.alloc(&h->d_colleague, 27 * (size_t)nbox, "colleague"));
  k_colleagues<<<div_up(nbox, 128), 128, 0, s>>>(nbox, banchor, bkey, d_lvl_start, h->d_colleague);
  AFMPB_TRY(check_launch("k_colleagues"));

  // ---- lists 1 (same level + finer) and 3 for leaves; list 2 for all boxes
  int64_t *d_cnt1 = nullptr, *d_cnt2 = nullptr;
  AFMPB_TRY(A.alloc(&d_cnt1, nbox + 1, "cnt1"));
  AFMPB_TRY(A.alloc(&d_cnt2, nbox + 1, "cnt2"));
  AFMPB_CUDA(cudaMemsetAsync(d_cnt1, 0, sizeof(int64_t) * (nbox + 1), s));
  AFMPB_CUDA(cudaMemsetAsync(d_cnt2, 0, sizeof(int64_t) * (nbox + 1), s));
  k_list_uw<<<div_up(T.nleaf, 64), 64, 0, s>>>(T.nleaf, h->d_leaves, h->d_colleague, bchild0, bnchild, banchor,
                                                d_cnt1, d_cnt2, nullptr, nullptr, nullptr, nullptr, false);
  AFMPB_TRY(check_launch("k_list_uw count"));
  int64_t *d_u1ptr = nullptr, *d_wptr = nullptr;
  int64_t n_u1 = 0, n_w = 0;
  AFMPB_TRY(csr_ptr(h, d_cnt1, nbox, &d_u1ptr, &n_u1, "u1ptr"));
  AFMPB_TRY(csr_ptr(h, d_cnt2, nbox, &d_wptr, &n_w, "wptr"));
  int32_t *d_u1idx = nullptr;
  AFMPB_TRY(A.alloc(&d_u1idx, n_u1, "u1idx"));
  AFMPB_TRY(A.alloc(&h->d_w_idx, n_w, "widx"));
  k_list_uw<<<div_up(T.nleaf, 64), 64, 0, s>>>(T.nleaf, h->d_leaves, h->d_colleague, bchild0, bnchild, banchor,
                                                nullptr, nullptr, d_u1ptr, d_wptr, d_u1idx, h->d_w_idx, true);
  AFMPB_TRY(check_launch("k_list_uw fill"));
  h->d_w_ptr = d_wptr;
  AFMPB_CUDA(cudaMemsetAsync(d_cnt1, 0, sizeof(int64_t) * (nbox + 1), s));
  k_list_v<<<div_up(nbox, 128), 128, 0, s>>>(nbox, bparent, h->d_colleague, bchild0, bnchild, banchor, d_cnt1,
                                             nullptr, nullptr, false);
  AFMPB_TRY(check_launch("k_list_v count"));
  int64_t n_v = 0;
  AFMPB_TRY(csr_ptr(h, d_cnt1, nbox, &h->d_v_ptr, &n_v, "vptr"));
  AFMPB_TRY(A.alloc(&h->d_v_idx, n_v, "vidx"));
  k_list_v<<<div_up(nbox, 128), 128, 0, s>>>(nbox, bparent, h->d_colleague, bchild0, bnchild, banchor, nullptr,
                                             h->d_v_ptr, h->d_v_idx, true);
  AFMPB_TRY(check_launch("k_list_v fill"));

  // ---- list 1 completed with its coarser half, list 4 as the dual of list 3: counts,
  //      CSR pointers, fill by atomic cursors, then every row's dual part sorted ascending
  //      (the result does not depend on the order the cursors were taken in)
  AFMPB_CUDA(cudaMemsetAsync(d_cnt1, 0, sizeof(int64_t) * (nbox + 1), s));
  AFMPB_CUDA(cudaMemsetAsync(d_cnt2, 0, sizeof(int64_t) * (nbox + 1), s));
  k_dual_count<<<div_up(T.nleaf, 128), 128, 0, s>>>(T.nleaf, h->d_leaves, blevel, d_u1ptr, d_u1idx, d_wptr,
                                                    h->d_w_idx, d_cnt1, d_cnt2);
  AFMPB_TRY(check_launch("k_dual_count"));
  int64_t *d_uptr = nullptr, *d_xptr = nullptr;
  int64_t n_uall = 0, n_x = 0;
  {
    // u row sizes: own (from u1ptr) + coarse (d_cnt1)
    int64_t *d_ucount = nullptr;
    AFMPB_TRY(A.alloc(&d_ucount, nbox + 1, "u counts"));
    k_u_rowsize<<<div_up(nbox + 1, 256), 256, 0, s>>>(nbox, d_u1ptr, d_cnt1, d_ucount);
    AFMPB_TRY(check_launch("k_u_rowsize"));
    AFMPB_TRY(csr_ptr(h, d_ucount, nbox, &d_uptr, &n_uall, "uptr"));
    A.release(d_ucount);
  }
  AFMPB_TRY(csr_ptr(h, d_cnt2, nbox, &d_xptr, &n_x, "xptr"));
  h->d_u_ptr = d_uptr;
  h->d_x_ptr = d_xptr;
  AFMPB_TRY(A.alloc(&h->d_u_idx, n_uall, "uidx"));
  AFMPB_TRY(A.alloc(&h->d_x_idx, n_x, "xidx"));
  {
    int64_t *seg_beg = nullptr, *ucur = nullptr, *xcur = nullptr;
    AFMPB_TRY(A.alloc(&seg_beg, nbox, "u coarse begin"));
    AFMPB_TRY(A.alloc(&ucur, nbox, "u cursor"));
    AFMPB_TRY(A.alloc(&xcur, nbox, "x cursor"));
    k_u_own<<<div_up(nbox, 128), 128, 0, s>>>(nbox, d_u1ptr, d_u1idx, d_uptr, h->d_u_idx, seg_beg, ucur);
    k_copy_i64<<<div_up(nbox, 256), 256, 0, s>>>(nbox, d_xptr, xcur);
    AFMPB_TRY(check_launch("k_u_own"));
    k_dual_fill<<<div_up(T.nleaf, 128), 128, 0, s>>>(T.nleaf, h->d_leaves, blevel, d_u1ptr, d_u1idx, d_wptr,
                                                     h->d_w_idx, ucur, h->d_u_idx, xcur, h->d_x_idx);
    AFMPB_TRY(check_launch("k_dual_fill"));
    AFMPB_TRY(sort_rows(h, h->d_u_idx, n_uall, seg_beg, d_uptr + 1, nbox, "u coarse sort"));
    AFMPB_TRY(sort_rows(h, h->d_x_idx, n_x, d_xptr, d_xptr + 1, nbox, "x sort"));
    A.release(seg_beg);
    A.release(ucur);
    A.release(xcur);
  }
  A.release(d_u1idx);
  A.release(d_u1ptr);

  // ---- list 4 routes: direct at the targets for small boxes, else P2L
  uint8_t *d_xdirect = nullptr;
  AFMPB_TRY(A.alloc(&d_xdirect, nbox, "x direct"));
  {
    uint8_t *p2l = nullptr;
    int32_t *iota = nullptr, *d_nsel = nullptr;
    AFMPB_TRY(A.alloc(&p2l, nbox, "x p2l"));
    AFMPB_TRY(A.alloc(&iota, nbox, "box iota"));
    AFMPB_TRY(A.alloc(&d_nsel, 1, "x box count"));
    AFMPB_TRY(A.alloc(&h->d_xbox, nbox, "xbox"));
    k_x_route<<<div_up(nbox, 256), 256, 0, s>>>(nbox, d_xptr, bbeg, bend, h->order * h->order * h->order, d_xdirect,
                                                  p2l);
    k_iota<<<div_up(nbox, 256), 256, 0, s>>>(nbox, iota);
    AFMPB_TRY(check_launch("k_x_route"));
    AFMPB_TRY(cub_call(h, "x box select", [&](void *t, size_t &bytes) {
      return cub::DeviceSelect::Flagged(t, bytes, iota, p2l, h->d_xbox, d_nsel, nbox, s);
    }));
    AFMPB_TRY(read_one(&h->n_xbox, d_nsel, s));
    A.release(p2l);
    A.release(iota);
    A.release(d_nsel);
  }

  // ---- point-to-point source boxes per leaf (ascending: near-field setup looks a box up
  //      by binary search), the P2P pair count and the blocks' longest-first order
  {
    const int nl = T.nleaf;
    int64_t *cnt = nullptr, *pairs_l = nullptr, *d_pairs = nullptr;
    uint64_t *cost = nullptr, *cost_sorted = nullptr;
    int32_t *iota = nullptr;
    AFMPB_TRY(A.alloc(&cnt, nl + 1, "p2p counts"));
    AFMPB_TRY(A.alloc(&pairs_l, nl, "p2p pairs"));
    AFMPB_TRY(A.alloc(&d_pairs, 1, "p2p pair total"));
    AFMPB_TRY(A.alloc(&cost, nl, "p2p cost"));
    AFMPB_TRY(A.alloc(&cost_sorted, nl, "p2p cost sorted"));
    AFMPB_TRY(A.alloc(&iota, nl, "leaf iota"));
    AFMPB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (nl + 1), s));
    k_p2p_lists<<<div_up(nl, 64), 64, 0, s>>>(nl, h->d_leaves, bbeg, bend, bparent, bchild0, bnchild, d_uptr,
                                              h->d_u_idx, d_xptr, h->d_x_idx, d_xdirect, d_wptr, h->d_w_idx, cnt,
                                              pairs_l, cost, nullptr, nullptr, false);
    AFMPB_TRY(check_launch("k_p2p_lists count"));
    int64_t n_p = 0;
    AFMPB_TRY(csr_ptr(h, cnt, nl, &h->d_p2p_ptr, &n_p, "p2p_ptr"));
    AFMPB_TRY(A.alloc(&h->d_p2p_idx, n_p, "p2p_idx"));
    k_p2p_lists<<<div_up(nl, 64), 64, 0, s>>>(nl, h->d_leaves, bbeg, bend, bparent, bchild0, bnchild, d_uptr,
                                              h->d_u_idx, d_xptr, h->d_x_idx, d_xdirect, d_wptr, h->d_w_idx, nullptr,
                                              nullptr, nullptr, h->d_p2p_ptr, h->d_p2p_idx, true);
    AFMPB_TRY(check_launch("k_p2p_lists fill"));
    AFMPB_TRY(sort_rows(h, h->d_p2p_idx, n_p, h->d_p2p_ptr, h->d_p2p_ptr + 1, nl, "p2p sort"));
    AFMPB_TRY(cub_call(h, "p2p pairs", [&](void *t, size_t &bytes) {
      return cub::DeviceReduce::Sum(t, bytes, pairs_l, d_pairs, nl, s);
    }));
    int64_t pairs = 0;
    AFMPB_TRY(read_one(&pairs, d_pairs, s));
    T.n_p2p_pairs = pairs - h->n;     // the diagonal t == p is skipped
    AFMPB_TRY(build_p2p_units(h));
    for (void *q : {(void *)cnt, (void *)pairs_l, (void *)d_pairs, (void *)cost, (void *)cost_sorted, (void *)iota})
      A.release(q);
  }
  A.release(d_xdirect);
  T.n_u = n_uall;
  T.n_v = n_v;
  T.n_w = n_w;
  T.n_x = n_x;

  // ---- M2L pairs grouped by (level, offset), each group's targets in box order: a stable
  //      radix sort of the entries by key, then the runs of equal keys
  {
    const int nkey = (T.nlevel + 1) * 343;
    uint32_t *key = nullptr, *key_sorted = nullptr, *uniq = nullptr;
    uint64_t *pk = nullptr, *pk_sorted = nullptr;
    int32_t *runs = nullptr, *d_nruns = nullptr;
    const int64_t nv = std::max<int64_t>(n_v, 1);
    AFMPB_TRY(A.alloc(&key, nv, "m2l keys"));
    AFMPB_TRY(A.alloc(&key_sorted, nv, "m2l keys sorted"));
    AFMPB_TRY(A.alloc(&pk, nv, "m2l pairs packed"));
    AFMPB_TRY(A.alloc(&pk_sorted, nv, "m2l pairs sorted"));
    AFMPB_TRY(A.alloc(&uniq, nv, "m2l group keys"));
    AFMPB_TRY(A.alloc(&runs, nv, "m2l group sizes"));
    AFMPB_TRY(A.alloc(&d_nruns, 1, "m2l group count"));
    AFMPB_TRY(A.alloc(&h->d_m2l_pairs, nv, "m2l_pairs"));
    h->m2l_groups.clear();
    h->n_m2l_pairs = n_v;
    if (n_v > 0) {
      k_m2l_keys<<<div_up(nbox, 128), 128, 0, s>>>(nbox, h->d_v_ptr, h->d_v_idx, banchor, key, pk);
      AFMPB_TRY(check_launch("k_m2l_keys"));
      int bits = 1;
      while ((1 << bits) < nkey) ++bits;
      AFMPB_TRY(cub_call(h, "m2l key sort", [&](void *t, size_t &bytes) {
        return cub::DeviceRadixSort::SortPairs(t, bytes, key, key_sorted, pk, pk_sorted, n_v, 0, bits, s);
      }));
      AFMPB_TRY(cub_call(h, "m2l groups", [&](void *t, size_t &bytes) {
        return cub::DeviceRunLengthEncode::Encode(t, bytes, key_sorted, uniq, runs, d_nruns, n_v, s);
      }));
      k_unpack_pairs<<<div_up(n_v, 256), 256, 0, s>>>(n_v, pk_sorted, h->d_m2l_pairs);
      AFMPB_TRY(check_launch("k_unpack_pairs"));
      int32_t ng = 0;
      AFMPB_TRY(read_one(&ng, d_nruns, s));
      std::vector<uint32_t> gkey(ng);
      std::vector<int32_t> gcnt(ng);
      AFMPB_TRY(to_host(gkey, uniq, ng, s));
      AFMPB_TRY(to_host(gcnt, runs, ng, s));
      int start = 0;
      for (int g = 0; g < ng; ++g) {                    // one entry per (level, offset) group
        M2LGroup gr;
        gr.level = (int)(gkey[g] / 343);
        gr.offset = (int)(gkey[g] % 343);               // raw code in [0, 343); mapped to a table slot in fmm.cu
        gr.start = start;
        gr.count = gcnt[g];
        start += gcnt[g];
        h->m2l_groups.push_back(gr);
      }
    }
    for (void *q : {(void *)key, (void *)key_sorted, (void *)pk, (void *)pk_sorted, (void *)uniq, (void *)runs,
                    (void *)d_nruns})
      A.release(q);
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
  AFMPB_TRY(A.alloc(&h->d_leaf_index, nbox, "leaf index"));
  AFMPB_CUDA(cudaMemsetAsync(h->d_leaf_index, 0xff, sizeof(int32_t) * nbox, s));
  k_leaf_index<<<div_up(T.nleaf, 256), 256, 0, s>>>(T.nleaf, h->d_leaves, h->d_leaf_index);
  AFMPB_TRY(check_launch("k_leaf_index"));
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
