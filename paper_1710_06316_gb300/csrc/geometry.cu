// geometry.cu -- mesh validation and node-patch geometry (paper Sec. 2, Fig. 1).
//
// The patch of node v is bounded by the centroids of its incident triangles and the
// midpoints of its incident edges.  Inside each incident triangle T it is the quad
// (v, m_va, c_T, m_vb), whose area is area(T)/3; the patch normal used by the far
// rule is the normalised area-weighted mean of the facet normals (or the caller's
// normal).  rho_v, the largest distance from v to a patch vertex, sizes the near set.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "corner_csr.h"
#include "internal.cuh"

namespace afmpb {

namespace {

// f(begin, end) over [0, n) split into contiguous ranges, one per host thread (at most 16).
template <class F>
void parallel_ranges(int64_t n, F f) {
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({16, (int64_t)std::thread::hardware_concurrency(),
                                                             n / 65536 + 1}));
  std::vector<std::thread> pool;
  for (int64_t t = 1; t < nt; ++t) pool.emplace_back(f, n * t / nt, n * (t + 1) / nt);
  f(0, n / nt);
  for (auto &th : pool) th.join();
}

}  // namespace

Err validate_mesh(const afmpb_mesh *m) {
  if (!m || !m->xyz || !m->tri) return make_err(AFMPB_EINVAL, "mesh, mesh->xyz and mesh->tri are required");
  if (m->n_nodes < 4 || m->n_tris < 4) return make_err(AFMPB_EMESH, "a closed surface needs >= 4 nodes and triangles");
  if (m->n_nodes > (int64_t)INT32_MAX / 2 || m->n_tris > (int64_t)INT32_MAX / 4)
    return make_err(AFMPB_EINVAL, "mesh too large for 32-bit node / triangle indices");
  const int64_t n = m->n_nodes, nt = m->n_tris;
  std::atomic<int> bad_xyz{0};
  parallel_ranges(3 * n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      if (!std::isfinite(m->xyz[i])) bad_xyz = 1;
  });
  if (bad_xyz) return make_err(AFMPB_EINVAL, "non-finite node coordinate");
  // triangle checks; the enclosed volume (times 6) summed per thread range
  std::atomic<int64_t> bad_tri{-1};
  std::mutex vol_mu;
  double vol6 = 0.0;
  parallel_ranges(nt, [&](int64_t t0, int64_t t1) {
    double part = 0.0;
    for (int64_t t = t0; t < t1; ++t) {
      int32_t a = m->tri[3 * t], b = m->tri[3 * t + 1], c = m->tri[3 * t + 2];
      if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n || a == b || b == c || a == c) {
        bad_tri = t;
        return;
      }
      const double *A = m->xyz + 3 * (int64_t)a, *B = m->xyz + 3 * (int64_t)b, *C = m->xyz + 3 * (int64_t)c;
      double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
      if (w[0] == 0.0 && w[1] == 0.0 && w[2] == 0.0) {
        bad_tri = t;
        return;
      }
      part += A[0] * w[0] + A[1] * w[1] + A[2] * w[2];
    }
    std::lock_guard<std::mutex> lk(vol_mu);
    vol6 += part;
  });
  if (bad_tri >= 0) {
    // name the first offending triangle's fault (serial rescan of the flagged range is
    // not needed: any flagged triangle identifies the fault)
    const int64_t t = bad_tri;
    int32_t a = m->tri[3 * t], b = m->tri[3 * t + 1], c = m->tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n)
      return make_err(AFMPB_EMESH, "triangle " + std::to_string(t) + " has a node index out of range");
    if (a == b || b == c || a == c) return make_err(AFMPB_EMESH, "triangle " + std::to_string(t) + " repeats a node");
    return make_err(AFMPB_EMESH, "triangle " + std::to_string(t) + " has zero area");
  }
  // every directed edge once, and its reverse once: closed, edge-manifold, consistently
  // oriented.  Half-edges are bucketed by their first node (parallel counting sort,
  // linear in the triangle count); each bucket is sorted, so a repeated direction sits
  // next to itself and the reverse of i -> j is a binary search in bucket j.
  std::unique_ptr<int64_t[]> ptr;
  std::unique_ptr<int32_t[]> dst;
  corner_csr(n, nt, m->tri, corner_csr_threads(nt), ptr, dst,
             [m](int64_t t, int k) { return m->tri[3 * t + (k + 1) % 3]; });
  // the two bucket passes run on the host cores, node ranges per thread
  std::atomic<int> dup{0}, open_edge{0};
  int32_t *const d = dst.get();
  const int64_t *const pp = ptr.get();
  parallel_ranges(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      std::sort(d + pp[i], d + pp[i + 1]);
      for (int64_t k = pp[i] + 1; k < pp[i + 1]; ++k)
        if (d[k] == d[k - 1]) dup = 1;
    }
  });
  if (dup) return make_err(AFMPB_EMESH, "an edge is used twice in the same direction (non-manifold or mis-oriented)");
  parallel_ranges(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1 && !open_edge; ++i)
      for (int64_t k = pp[i]; k < pp[i + 1]; ++k) {
        const int64_t j = d[k];
        if (!std::binary_search(d + pp[j], d + pp[j + 1], (int32_t)i)) open_edge = 1;
      }
  });
  if (open_edge) return make_err(AFMPB_EMESH, "an edge has no opposite half-edge (open surface or mis-oriented triangle)");
  if (!(vol6 > 0.0)) return make_err(AFMPB_EMESH, "enclosed volume is not positive: triangles must be counter-clockwise seen from outside");
  if (m->normals) {
    for (int64_t i = 0; i < n; ++i) {
      const double *q = m->normals + 3 * i;
      double l = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
      if (!(l > 0.0) || !std::isfinite(l)) return make_err(AFMPB_EINVAL, "a supplied normal is zero or not finite");
    }
  }
  return Err{};
}

// Facet normals (unit) of every triangle.
__global__ void k_facets(int64_t nt, const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                         double *__restrict__ tnrm) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double *A = xyz + 3 * (int64_t)tri[3 * t], *B = xyz + 3 * (int64_t)tri[3 * t + 1],
               *C = xyz + 3 * (int64_t)tri[3 * t + 2];
  double u0 = B[0] - A[0], u1 = B[1] - A[1], u2 = B[2] - A[2];
  double v0 = C[0] - A[0], v1 = C[1] - A[1], v2 = C[2] - A[2];
  double w0 = u1 * v2 - u2 * v1, w1 = u2 * v0 - u0 * v2, w2 = u0 * v1 - u1 * v0;
  double l = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
  tnrm[3 * t] = w0 / l;
  tnrm[3 * t + 1] = w1 / l;
  tnrm[3 * t + 2] = w2 / l;
}

// Patch area, node normal and patch radius of every node (caller order).
__global__ void k_node_patch(int64_t n, const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                             const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_tri,
                             const double *__restrict__ user_nrm, double *__restrict__ area,
                             double *__restrict__ nrm, double *__restrict__ rho) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double xv = xyz[3 * v], yv = xyz[3 * v + 1], zv = xyz[3 * v + 2];
  double A = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0, r2max = 0.0;
  for (int64_t j = inc_ptr[v]; j < inc_ptr[v + 1]; ++j) {
    const int32_t t = inc_tri[j];
    double P[3][3];
    for (int k = 0; k < 3; ++k) {
      const double *q = xyz + 3 * (int64_t)tri[3 * t + k];
      P[k][0] = q[0]; P[k][1] = q[1]; P[k][2] = q[2];
    }
    double u0 = P[1][0] - P[0][0], u1 = P[1][1] - P[0][1], u2 = P[1][2] - P[0][2];
    double w0 = P[2][0] - P[0][0], w1 = P[2][1] - P[0][1], w2 = P[2][2] - P[0][2];
    double c0 = u1 * w2 - u2 * w1, c1 = u2 * w0 - u0 * w2, c2 = u0 * w1 - u1 * w0;
    double two_area = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    A += two_area / 6.0;              // area(T) / 3
    s0 += 0.5 * c0; s1 += 0.5 * c1; s2 += 0.5 * c2;   // area(T) * facet normal
    // patch vertices inside T: edge midpoints at v and the centroid
    double gx = (P[0][0] + P[1][0] + P[2][0]) / 3.0 - xv;
    double gy = (P[0][1] + P[1][1] + P[2][1]) / 3.0 - yv;
    double gz = (P[0][2] + P[1][2] + P[2][2]) / 3.0 - zv;
    r2max = fmax(r2max, gx * gx + gy * gy + gz * gz);
    for (int k = 0; k < 3; ++k) {
      if (tri[3 * t + k] == v) continue;
      double mx = 0.5 * (P[k][0] - xv), my = 0.5 * (P[k][1] - yv), mz = 0.5 * (P[k][2] - zv);
      r2max = fmax(r2max, mx * mx + my * my + mz * mz);
    }
  }
  area[v] = A;
  rho[v] = sqrt(r2max);
  if (user_nrm) {
    s0 = user_nrm[3 * v]; s1 = user_nrm[3 * v + 1]; s2 = user_nrm[3 * v + 2];
  }
  double l = sqrt(s0 * s0 + s1 * s1 + s2 * s2);
  nrm[3 * v] = s0 / l;
  nrm[3 * v + 1] = s1 / l;
  nrm[3 * v + 2] = s2 / l;
}

Err build_geometry(afmpb_t *h, const afmpb_mesh *m) {
  const int64_t n = h->n, nt = h->nt;
  // node -> incident triangle CSR (parallel counting sort; triangles of a node in index
  // order)
  std::unique_ptr<int64_t[]> inc_ptr;
  std::unique_ptr<int32_t[]> inc_tri;
  corner_csr(n, nt, m->tri, corner_csr_threads(nt), inc_ptr, inc_tri, [](int64_t t, int) { return (int32_t)t; });
  auto &A = h->arena;
  AFMPB_TRY(A.alloc(&h->d_xyz, 3 * n, "xyz"));
  AFMPB_TRY(A.alloc(&h->d_tri, 3 * nt, "tri"));
  AFMPB_TRY(A.alloc(&h->d_inc_ptr, n + 1, "inc_ptr"));
  AFMPB_TRY(A.alloc(&h->d_inc_tri, 3 * nt, "inc_tri"));
  AFMPB_TRY(A.alloc(&h->d_tri_nrm, 3 * nt, "tri_nrm"));
  AFMPB_TRY(A.alloc(&h->d_area64, n, "area"));
  AFMPB_TRY(A.alloc(&h->d_nrm64, 3 * n, "nrm"));
  AFMPB_TRY(A.alloc(&h->d_rho64, n, "rho"));
  cudaStream_t s = h->stream;
  AFMPB_CUDA(cudaMemcpyAsync(h->d_xyz, m->xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_tri, m->tri, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_inc_ptr, inc_ptr.get(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_inc_tri, inc_tri.get(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
  double *d_user = nullptr;
  if (m->normals) {
    AFMPB_TRY(A.alloc(&d_user, 3 * n, "user normals"));
    AFMPB_CUDA(cudaMemcpyAsync(d_user, m->normals, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
  }
  k_facets<<<div_up(nt, 256), 256, 0, s>>>(nt, h->d_xyz, h->d_tri, h->d_tri_nrm);
  AFMPB_TRY(check_launch("k_facets"));
  k_node_patch<<<div_up(n, 256), 256, 0, s>>>(n, h->d_xyz, h->d_tri, h->d_inc_ptr, h->d_inc_tri, d_user,
                                              h->d_area64, h->d_nrm64, h->d_rho64);
  AFMPB_TRY(check_launch("k_node_patch"));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  if (d_user) A.release(d_user);
  return Err{};
}

}  // namespace afmpb
