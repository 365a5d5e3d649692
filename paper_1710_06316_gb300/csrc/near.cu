// near.cu -- near-field patch coefficients (paper Sec. 2, Eq. 6 and the near/far rule
// after it; step 2 of the solution flow: computed once and saved).
//
// Near set of node p: t == p, or |x_p - x_t| < c (rho_p + rho_t).  The set is found by a
// pruned walk of the octree (box distance against c (rho_p + max rho in the box)), so it
// is exact and independent of the tree.  For each near pair the library stores the
// correction  X_near - X_far  (t != p) or the self-patch value X_pp, X in {A, B, C, D}:
// the far-field sums (FMM + P2P) use the point rule for every pair, and the correction
// turns the near pairs into the near rule.
//
// Near rule over each patch piece of t (two sub-triangles per incident triangle, facet
// normal as source normal): 7-point degree-5 Radon rule, split 1 -> 4 while the target
// is closer than 3 times the piece's longest edge to its centroid, at most 6 times.
// Self patch: the patch projected on the tangent plane of n_p, where the B and C
// integrands vanish and A, D are weakly singular; polar (Duffy) map about x_p with a
// 16 x 16 Gauss-Legendre rule.  All in FP64.
#include <cmath>

#include "internal.cuh"

namespace afmpb {

__constant__ double c_gl_x[16], c_gl_w[16];      // Gauss-Legendre on [0, 1]
__constant__ double c_rad_b[21], c_rad_w[7];     // Radon 7-point: barycentrics, weights

constexpr int kNearStack = 8 * (kMaxLevel + 2);
constexpr int kQuadDepth = 6;
constexpr double kRefine = 3.0;

struct KernelParams {
  double kappa, ebar;
};

// The four Eq. 6 integrands at one point: d = x_target - y_source, n0 target normal,
// ns source normal.
__device__ __forceinline__ void abcd_point(const KernelParams &kp, double dx, double dy, double dz,
                                           const double *n0, const double *ns, double o[4]) {
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2);
  double ndn = ns[0] * dx + ns[1] * dy + ns[2] * dz;
  double n0d = n0[0] * dx + n0[1] * dy + n0[2] * dz;
  double nn0 = ns[0] * n0[0] + ns[1] * n0[1] + ns[2] * n0[2];
  double G = kInv4Pi / r;
  double G3 = G / r2;
  double G5 = 3.0 * G3 / r2;
  double kr = kp.kappa * r;
  double e = exp(-kr);
  double g1 = (e * (1.0 + kr)) * G3;
  double g2 = (e * (1.0 + kr + kr * kr / 3.0)) * G5;
  o[0] = G - e * G;
  o[1] = ndn * G3 / kp.ebar - ndn * g1;
  o[2] = -n0d * G3 + n0d * g1 / kp.ebar;
  o[3] = ((nn0 * G3 - ndn * n0d * G5) - (nn0 * g1 - ndn * n0d * g2)) / kp.ebar;
}

// Adaptive Radon quadrature over triangle (v0, v1, v2), stackless walk of the 1 -> 4
// subdivision tree (path digits), accumulating into acc.
__device__ void quad_triangle(const KernelParams &kp, const double *x, const double *n0, const double *v0,
                              const double *v1, const double *v2, const double *ns, double acc[4]) {
  int dig[kQuadDepth + 1];
  int d = 0;
  dig[0] = 0;
  while (true) {
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) { a[k] = v0[k]; b[k] = v1[k]; c[k] = v2[k]; }
    for (int l = 1; l <= d; ++l) {
      double mab[3], mbc[3], mca[3];
      for (int k = 0; k < 3; ++k) {
        mab[k] = 0.5 * (a[k] + b[k]); mbc[k] = 0.5 * (b[k] + c[k]); mca[k] = 0.5 * (c[k] + a[k]);
      }
      switch (dig[l]) {
        case 0: for (int k = 0; k < 3; ++k) { b[k] = mab[k]; c[k] = mca[k]; } break;
        case 1: for (int k = 0; k < 3; ++k) { a[k] = mab[k]; c[k] = mbc[k]; } break;
        case 2: for (int k = 0; k < 3; ++k) { a[k] = mca[k]; b[k] = mbc[k]; } break;
        default: for (int k = 0; k < 3; ++k) { a[k] = mab[k]; b[k] = mbc[k]; c[k] = mca[k]; } break;
      }
    }
    double e01[3], e12[3], e20[3];
    for (int k = 0; k < 3; ++k) { e01[k] = b[k] - a[k]; e12[k] = c[k] - b[k]; e20[k] = a[k] - c[k]; }
    double l01 = sqrt(e01[0] * e01[0] + e01[1] * e01[1] + e01[2] * e01[2]);
    double l12 = sqrt(e12[0] * e12[0] + e12[1] * e12[1] + e12[2] * e12[2]);
    double l20 = sqrt(e20[0] * e20[0] + e20[1] * e20[1] + e20[2] * e20[2]);
    double diam = fmax(l01, fmax(l12, l20));
    double gx = (a[0] + b[0] + c[0]) / 3.0 - x[0], gy = (a[1] + b[1] + c[1]) / 3.0 - x[1],
           gz = (a[2] + b[2] + c[2]) / 3.0 - x[2];
    double dist = sqrt(gx * gx + gy * gy + gz * gz);
    if (d < kQuadDepth && dist < kRefine * diam) {
      ++d;
      dig[d] = 0;
      continue;
    }
    // e02 = c - a = -e20
    double cr0 = e01[1] * (-e20[2]) - e01[2] * (-e20[1]);
    double cr1 = e01[2] * (-e20[0]) - e01[0] * (-e20[2]);
    double cr2 = e01[0] * (-e20[1]) - e01[1] * (-e20[0]);
    double area = 0.5 * sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
    for (int q = 0; q < 7; ++q) {
      double y0 = c_rad_b[3 * q] * a[0] + c_rad_b[3 * q + 1] * b[0] + c_rad_b[3 * q + 2] * c[0];
      double y1 = c_rad_b[3 * q] * a[1] + c_rad_b[3 * q + 1] * b[1] + c_rad_b[3 * q + 2] * c[1];
      double y2 = c_rad_b[3 * q] * a[2] + c_rad_b[3 * q + 1] * b[2] + c_rad_b[3 * q + 2] * c[2];
      double o[4];
      abcd_point(kp, x[0] - y0, x[1] - y1, x[2] - y2, n0, ns, o);
      double w = area * c_rad_w[q];
      for (int k = 0; k < 4; ++k) acc[k] += w * o[k];
    }
    while (d > 0 && dig[d] == 3) --d;
    if (d == 0) break;
    ++dig[d];
  }
}

// Corner positions of triangle t rotated so that node v comes first.
__device__ __forceinline__ void tri_from(const double *xyz, const int32_t *tri, int32_t t, int64_t v, double P[3][3]) {
  int k0 = 0;
  for (int k = 0; k < 3; ++k)
    if (tri[3 * t + k] == v) k0 = k;
  for (int j = 0; j < 3; ++j) {
    const double *q = xyz + 3 * (int64_t)tri[3 * t + (k0 + j) % 3];
    P[j][0] = q[0]; P[j][1] = q[1]; P[j][2] = q[2];
  }
}

__device__ void near_rule(const KernelParams &kp, const double *xyz, const int32_t *tri, const int64_t *inc_ptr,
                          const int32_t *inc_tri, const double *tri_nrm, const double *xp, const double *np,
                          int64_t ot, double acc[4]) {
  for (int64_t j = inc_ptr[ot]; j < inc_ptr[ot + 1]; ++j) {
    int32_t T = inc_tri[j];
    double P[3][3];
    tri_from(xyz, tri, T, ot, P);
    double ma[3], mb[3], cen[3];
    for (int k = 0; k < 3; ++k) {
      ma[k] = 0.5 * (P[0][k] + P[1][k]);
      mb[k] = 0.5 * (P[0][k] + P[2][k]);
      cen[k] = (P[0][k] + P[1][k] + P[2][k]) / 3.0;
    }
    const double *ns = tri_nrm + 3 * (int64_t)T;
    quad_triangle(kp, xp, np, P[0], ma, cen, ns, acc);
    quad_triangle(kp, xp, np, P[0], cen, mb, ns, acc);
  }
}

__device__ void self_rule(const KernelParams &kp, const double *xyz, const int32_t *tri, const int64_t *inc_ptr,
                          const int32_t *inc_tri, int64_t op, const double *np, double o[4]) {
  const double *xp = xyz + 3 * op;
  double As = 0.0, Ds = 0.0;
  for (int64_t j = inc_ptr[op]; j < inc_ptr[op + 1]; ++j) {
    int32_t T = inc_tri[j];
    double P[3][3];
    tri_from(xyz, tri, T, op, P);
    double ma[3], mb[3], cen[3];
    for (int k = 0; k < 3; ++k) {
      ma[k] = 0.5 * (P[0][k] + P[1][k]);
      mb[k] = 0.5 * (P[0][k] + P[2][k]);
      cen[k] = (P[0][k] + P[1][k] + P[2][k]) / 3.0;
    }
    const double *far_pts[2][2] = {{ma, cen}, {cen, mb}};
    for (int q = 0; q < 2; ++q) {
      double e[2][3];
      for (int v = 0; v < 2; ++v) {
        double dv[3] = {far_pts[q][v][0] - xp[0], far_pts[q][v][1] - xp[1], far_pts[q][v][2] - xp[2]};
        double hgt = dv[0] * np[0] + dv[1] * np[1] + dv[2] * np[2];
        for (int k = 0; k < 3; ++k) e[v][k] = dv[k] - hgt * np[k];
      }
      double c0 = e[0][1] * e[1][2] - e[0][2] * e[1][1];
      double c1 = e[0][2] * e[1][0] - e[0][0] * e[1][2];
      double c2 = e[0][0] * e[1][1] - e[0][1] * e[1][0];
      double J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
      for (int it = 0; it < 16; ++it) {
        double tt = c_gl_x[it], wt = c_gl_w[it];
        double w0 = e[0][0] + tt * (e[1][0] - e[0][0]);
        double w1 = e[0][1] + tt * (e[1][1] - e[0][1]);
        double w2 = e[0][2] + tt * (e[1][2] - e[0][2]);
        double l = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
        for (int is = 0; is < 16; ++is) {
          double ss = c_gl_x[is], ws = c_gl_w[is];
          double xk = kp.kappa * ss * l;
          double fa = -expm1(-xk) * kInv4Pi / l;
          double num;
          if (xk < 0.05) {
            // 1 - e^{-x}(1 + x) = sum_{j>=2} (-1)^j (j - 1) x^j / j!
            double term = 0.5 * xk * xk, s = term;
            for (int jj = 3; jj < 12; ++jj) {
              term *= -xk * (double)(jj - 1) / ((double)jj * (double)(jj - 2));
              s += term;
            }
            num = s;
          } else {
            num = 1.0 - exp(-xk) * (1.0 + xk);
          }
          double fd = num * kInv4Pi / (ss * ss * l * l * l);
          As += J * wt * ws * fa;
          Ds += J * wt * ws * fd;
        }
      }
    }
  }
  o[0] = As;
  o[1] = 0.0;
  o[2] = 0.0;
  o[3] = Ds / kp.ebar;
}

// Near-set walk.  fill == false: count per row; else write the columns.
__global__ void k_near_search(int64_t n, double cnear, const int32_t *__restrict__ perm,
                              const double *__restrict__ xyz, const double *__restrict__ rho,
                              const dbl4 *__restrict__ center, const double *__restrict__ brho,
                              const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                              const int32_t *__restrict__ bbeg, const int32_t *__restrict__ bend,
                              int64_t *__restrict__ cnt, const int64_t *__restrict__ ptr,
                              int32_t *__restrict__ col, bool fill) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t op = perm[p];
  const double x0 = xyz[3 * op], x1 = xyz[3 * op + 1], x2 = xyz[3 * op + 2];
  const double rp = rho[op];
  int64_t k = 0, base = fill ? ptr[p] : 0;
  int stack[kNearStack];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    int b = stack[--sp];
    dbl4 c = center[b];
    double dx = fmax(fabs(x0 - c.x) - c.w, 0.0), dy = fmax(fabs(x1 - c.y) - c.w, 0.0),
           dz = fmax(fabs(x2 - c.z) - c.w, 0.0);
    double dbox = sqrt(dx * dx + dy * dy + dz * dz);
    if (dbox >= cnear * (rp + brho[b])) continue;
    if (nchild[b] == 0) {
      for (int t = bbeg[b]; t < bend[b]; ++t) {
        int64_t ot = perm[t];
        double ex = x0 - xyz[3 * ot], ey = x1 - xyz[3 * ot + 1], ez = x2 - xyz[3 * ot + 2];
        double dist = sqrt(ex * ex + ey * ey + ez * ez);
        if (t == p || dist < cnear * (rp + rho[ot])) {
          if (fill) col[base + k] = t;
          ++k;
        }
      }
    } else {
      for (int j = nchild[b] - 1; j >= 0 && sp < kNearStack; --j) stack[sp++] = child0[b] + j;
    }
  }
  if (!fill) cnt[p] = k;
}

// Coefficients, one warp per row.
__global__ void k_near_coef(int64_t n, KernelParams kp, const int32_t *__restrict__ perm,
                            const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                            const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_tri,
                            const double *__restrict__ tri_nrm, const double *__restrict__ area,
                            const double *__restrict__ nrm, const int64_t *__restrict__ ptr,
                            const int32_t *__restrict__ col, float4 *__restrict__ coef) {
  int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= n) return;
  int64_t op = perm[p];
  const double *xp = xyz + 3 * op;
  const double *np = nrm + 3 * op;
  for (int64_t j = ptr[p] + lane; j < ptr[p + 1]; j += 32) {
    int t = col[j];
    int64_t ot = perm[t];
    double o[4] = {0, 0, 0, 0};
    if (t == p) {
      self_rule(kp, xyz, tri, inc_ptr, inc_tri, op, np, o);
    } else {
      near_rule(kp, xyz, tri, inc_ptr, inc_tri, tri_nrm, xp, np, ot, o);
      double f[4];
      const double *xt = xyz + 3 * ot;
      abcd_point(kp, xp[0] - xt[0], xp[1] - xt[1], xp[2] - xt[2], np, nrm + 3 * ot, f);
      for (int k = 0; k < 4; ++k) o[k] -= area[ot] * f[k];
    }
    coef[j] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
  }
}

namespace {
void gauss_legendre_unit(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double step = p1 / dp;
      z -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = 0.5 * (z + 1.0);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}
}  // namespace

Err build_near(afmpb_t *h) {
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  auto &A = h->arena;
  {
    double gx[16], gw[16];
    gauss_legendre_unit(16, gx, gw);
    AFMPB_CUDA(cudaMemcpyToSymbolAsync(c_gl_x, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyToSymbolAsync(c_gl_w, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s));
    // Radon's 7-point rule (exact for degree 5): centroid and two orbits of three points
    const double r15 = std::sqrt(15.0);
    const double a1 = (6.0 - r15) / 21.0, a2 = (6.0 + r15) / 21.0;
    const double w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
    double b[21] = {1.0 / 3, 1.0 / 3, 1.0 / 3,
                    a1, a1, 1 - 2 * a1, a1, 1 - 2 * a1, a1, 1 - 2 * a1, a1, a1,
                    a2, a2, 1 - 2 * a2, a2, 1 - 2 * a2, a2, 1 - 2 * a2, a2, a2};
    double w[7] = {9.0 / 40, w1, w1, w1, w2, w2, w2};
    AFMPB_CUDA(cudaMemcpyToSymbolAsync(c_rad_b, b, sizeof(b), 0, cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaMemcpyToSymbolAsync(c_rad_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, s));
  }
  int64_t *d_cnt = nullptr;
  AFMPB_TRY(A.alloc(&d_cnt, n, "near cnt"));
  const double cnear = h->opt.near_c;
  k_near_search<<<div_up(n, 128), 128, 0, s>>>(n, cnear, h->d_perm, h->d_xyz, h->d_rho64, h->d_box_center,
                                               h->d_box_rho, h->d_box_child0, h->d_box_nchild, h->d_box_begin,
                                               h->d_box_end, d_cnt, nullptr, nullptr, false);
  AFMPB_TRY(check_launch("k_near_search count"));
  std::vector<int64_t> cnt(n), ptr(n + 1, 0);
  AFMPB_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; ++i) ptr[i + 1] = ptr[i] + cnt[i];
  h->nnz = ptr[n];
  AFMPB_TRY(A.alloc(&h->d_near_ptr, n + 1, "near ptr"));
  AFMPB_TRY(A.alloc(&h->d_near_col, h->nnz, "near col"));
  AFMPB_TRY(A.alloc(&h->d_near_coef, h->nnz, "near coef"));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_near_ptr, ptr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  k_near_search<<<div_up(n, 128), 128, 0, s>>>(n, cnear, h->d_perm, h->d_xyz, h->d_rho64, h->d_box_center,
                                               h->d_box_rho, h->d_box_child0, h->d_box_nchild, h->d_box_begin,
                                               h->d_box_end, nullptr, h->d_near_ptr, h->d_near_col, true);
  AFMPB_TRY(check_launch("k_near_search fill"));
  KernelParams kp{h->kappa, h->ebar};
  k_near_coef<<<div_up(n * 32, 128), 128, 0, s>>>(n, kp, h->d_perm, h->d_xyz, h->d_tri, h->d_inc_ptr, h->d_inc_tri,
                                                   h->d_tri_nrm, h->d_area64, h->d_nrm64, h->d_near_ptr,
                                                   h->d_near_col, h->d_near_coef);
  AFMPB_TRY(check_launch("k_near_coef"));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(d_cnt);
  return Err{};
}

}  // namespace afmpb
