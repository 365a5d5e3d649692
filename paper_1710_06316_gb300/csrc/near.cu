// near.cu -- near-field patch coefficients (paper Sec. 2, Eq. 6 and the near/far rule
// after it; step 2 of the solution flow: computed once and saved).
//
// Near set of node p: t == p, or |x_p - x_t| < c (rho_p + rho_t).  The set is found by a
// pruned walk of the octree (box distance against c (rho_p + max rho in the box)), so it
// is exact and independent of the tree; the membership test is done in FP64.  For each
// near pair the library stores the correction  X_near - X_far  (t != p) or the
// self-patch value X_pp, X in {A, B, C, D}: the far-field sums (FMM + P2P) use the point
// rule for every pair, and the correction turns the near pairs into the near rule.
//
// Near rule over each patch piece of t (two sub-triangles per incident triangle, facet
// normal as source normal): 7-point degree-5 Radon rule, split 1 -> 4 while the target
// is closer than 3 times the piece's longest edge to its centroid, at most 6 times.
// Self patch: the patch projected on the tangent plane of n_p, where the B and C
// integrands vanish and A, D are weakly singular; polar (Duffy) map about x_p with a
// 16 x 16 Gauss-Legendre rule.
//
// Precision: all geometry is first taken relative to the target x_p in FP64 (so no
// large-coordinate cancellation reaches the quadrature), then the quadrature runs in
// FP32 (the `Real` template parameter; GB300's FP32 rate is many times its FP64 rate).
#include <cmath>

#include <mutex>

#include "internal.cuh"

namespace afmpb {

__constant__ float c_gl_xf[16], c_gl_wf[16];     // Gauss-Legendre on [0, 1]
__constant__ float c_rad_bf[21], c_rad_wf[7];    // Radon 7-point: barycentrics, weights

constexpr int kNearStack = 8 * (kMaxLevel + 2);
constexpr int kQuadDepth = 6;

struct KernelParams {
  double kappa, ebar;
};

template <class Real>
struct V3 {
  Real x, y, z;
};

template <class Real>
__device__ __forceinline__ Real dot(const V3<Real> &a, const V3<Real> &b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// phi1(x) = 1 - e^{-x}(1 + x) and phi2(x) = 1 - e^{-x}(1 + x + x^2/3): the screened
// fractions of the Laplace 1/r^3 and 3/r^5 terms.  Below x = 0.5 they are summed from
// their power series (coefficients of x^j: (-1)^j (j-1) / j! and
// (-1)^(j+1) (j-1)(j-3) / (3 j!)), which avoids the cancellation of the direct forms.
template <class Real>
__device__ __forceinline__ void screened_fractions(Real x, Real &p1, Real &p2) {
  if (x < Real(0.5)) {
    Real t = x;            // x^j / j!
    Real s1 = 0, s2 = 0;
    for (int j = 2; j < 16; ++j) {
      t *= x / (Real)j;
      const Real sg = (j & 1) ? Real(-1) : Real(1);
      s1 += sg * (Real)(j - 1) * t;
      s2 -= sg * (Real)((j - 1) * (j - 3)) * t / Real(3);
    }
    p1 = s1;
    p2 = s2;
  } else {
    const Real e = exp(-x);
    p1 = Real(1) - e * (Real(1) + x);
    p2 = Real(1) - e * (Real(1) + x + x * x / Real(3));
  }
}

// The four Eq. 6 integrands at one point: d = x_target - y_source, n0 target normal,
// ns source normal.  The G - u differences of A and D are formed without cancellation
// (A through expm1, D through the screened fractions above).
template <class Real>
__device__ __forceinline__ void abcd_point(Real kappa, Real ebar, const V3<Real> &d, const V3<Real> &n0,
                                           const V3<Real> &ns, Real o[4]) {
  const Real r2 = dot(d, d);
  const Real r = sqrt(r2);
  const Real ndn = dot(ns, d), n0d = dot(n0, d), nn0 = dot(ns, n0);
  const Real G = Real(kInv4Pi) / r;
  const Real G3 = G / r2;
  const Real G5 = Real(3) * G3 / r2;
  const Real kr = kappa * r;
  const Real e = exp(-kr);
  const Real g1 = (e * (Real(1) + kr)) * G3;
  Real p1, p2;
  screened_fractions(kr, p1, p2);
  o[0] = -expm1(-kr) * G;                       // G - u
  o[1] = ndn * G3 / ebar - ndn * g1;
  o[2] = -n0d * G3 + n0d * g1 / ebar;
  o[3] = (nn0 * G3 * p1 - ndn * n0d * G5 * p2) / ebar;
}

// Adaptive Radon quadrature over triangle (v0, v1, v2) for a target at the origin,
// stackless walk of the 1 -> 4 subdivision tree (path digits), accumulating into acc.
template <class Real>
__device__ void quad_triangle(Real kappa, Real ebar, const V3<Real> &n0, const V3<Real> &v0, const V3<Real> &v1,
                              const V3<Real> &v2, const V3<Real> &ns, Real acc[4]) {
  int dig[kQuadDepth + 1];
  int d = 0;
  dig[0] = 0;
  while (true) {
    V3<Real> a = v0, b = v1, c = v2;
    for (int l = 1; l <= d; ++l) {
      const V3<Real> mab{Real(0.5) * (a.x + b.x), Real(0.5) * (a.y + b.y), Real(0.5) * (a.z + b.z)};
      const V3<Real> mbc{Real(0.5) * (b.x + c.x), Real(0.5) * (b.y + c.y), Real(0.5) * (b.z + c.z)};
      const V3<Real> mca{Real(0.5) * (c.x + a.x), Real(0.5) * (c.y + a.y), Real(0.5) * (c.z + a.z)};
      switch (dig[l]) {
        case 0: b = mab; c = mca; break;
        case 1: a = mab; c = mbc; break;
        case 2: a = mca; b = mbc; break;
        default: a = mab; b = mbc; c = mca; break;
      }
    }
    const V3<Real> e01{b.x - a.x, b.y - a.y, b.z - a.z}, e12{c.x - b.x, c.y - b.y, c.z - b.z},
        e02{c.x - a.x, c.y - a.y, c.z - a.z};
    const Real diam = sqrt(fmax(dot(e01, e01), fmax(dot(e12, e12), dot(e02, e02))));
    const V3<Real> g{(a.x + b.x + c.x) / Real(3), (a.y + b.y + c.y) / Real(3), (a.z + b.z + c.z) / Real(3)};
    if (d < kQuadDepth && sqrt(dot(g, g)) < Real(3) * diam) {
      ++d;
      dig[d] = 0;
      continue;
    }
    const V3<Real> cr{e01.y * e02.z - e01.z * e02.y, e01.z * e02.x - e01.x * e02.z, e01.x * e02.y - e01.y * e02.x};
    const Real area = Real(0.5) * sqrt(dot(cr, cr));
    for (int q = 0; q < 7; ++q) {
      const Real b0 = c_rad_bf[3 * q], b1 = c_rad_bf[3 * q + 1], b2 = c_rad_bf[3 * q + 2];
      const V3<Real> dq{-(b0 * a.x + b1 * b.x + b2 * c.x), -(b0 * a.y + b1 * b.y + b2 * c.y),
                        -(b0 * a.z + b1 * b.z + b2 * c.z)};
      Real o[4];
      abcd_point(kappa, ebar, dq, n0, ns, o);
      const Real w = area * c_rad_wf[q];
      for (int k = 0; k < 4; ++k) acc[k] += w * o[k];
    }
    while (d > 0 && dig[d] == 3) --d;
    if (d == 0) break;
    ++dig[d];
  }
}

// Corners of triangle t rotated so that node v comes first, relative to the point o
// (difference taken in FP64).
template <class Real>
__device__ __forceinline__ void tri_rel(const double *xyz, const int32_t *tri, int32_t t, int64_t v,
                                        const double *o, V3<Real> P[3]) {
  int k0 = 0;
  for (int k = 0; k < 3; ++k)
    if (tri[3 * t + k] == v) k0 = k;
  for (int j = 0; j < 3; ++j) {
    const double *q = xyz + 3 * (int64_t)tri[3 * t + (k0 + j) % 3];
    P[j] = V3<Real>{(Real)(q[0] - o[0]), (Real)(q[1] - o[1]), (Real)(q[2] - o[2])};
  }
}

template <class Real>
__device__ void near_rule(Real kappa, Real ebar, const double *xyz, const int32_t *tri, const int64_t *inc_ptr,
                          const int32_t *inc_tri, const double *tri_nrm, const double *xp, const V3<Real> &np,
                          int64_t ot, Real acc[4]) {
  for (int64_t j = inc_ptr[ot]; j < inc_ptr[ot + 1]; ++j) {
    const int32_t T = inc_tri[j];
    V3<Real> P[3];
    tri_rel(xyz, tri, T, ot, xp, P);
    const V3<Real> ma{Real(0.5) * (P[0].x + P[1].x), Real(0.5) * (P[0].y + P[1].y), Real(0.5) * (P[0].z + P[1].z)};
    const V3<Real> mb{Real(0.5) * (P[0].x + P[2].x), Real(0.5) * (P[0].y + P[2].y), Real(0.5) * (P[0].z + P[2].z)};
    const V3<Real> cen{(P[0].x + P[1].x + P[2].x) / Real(3), (P[0].y + P[1].y + P[2].y) / Real(3),
                       (P[0].z + P[1].z + P[2].z) / Real(3)};
    const double *tn = tri_nrm + 3 * (int64_t)T;
    const V3<Real> ns{(Real)tn[0], (Real)tn[1], (Real)tn[2]};
    quad_triangle(kappa, ebar, np, P[0], ma, cen, ns, acc);
    quad_triangle(kappa, ebar, np, P[0], cen, mb, ns, acc);
  }
}

template <class Real>
__device__ void self_rule(Real kappa, Real ebar, const double *xyz, const int32_t *tri, const int64_t *inc_ptr,
                          const int32_t *inc_tri, int64_t op, const V3<Real> &np, Real o[4]) {
  const double *xp = xyz + 3 * op;
  Real As = 0, Ds = 0;
  for (int64_t j = inc_ptr[op]; j < inc_ptr[op + 1]; ++j) {
    V3<Real> P[3];
    tri_rel(xyz, tri, inc_tri[j], op, xp, P);   // P[0] = 0 (the node itself)
    const V3<Real> ma{Real(0.5) * P[1].x, Real(0.5) * P[1].y, Real(0.5) * P[1].z};
    const V3<Real> mb{Real(0.5) * P[2].x, Real(0.5) * P[2].y, Real(0.5) * P[2].z};
    const V3<Real> cen{(P[1].x + P[2].x) / Real(3), (P[1].y + P[2].y) / Real(3), (P[1].z + P[2].z) / Real(3)};
    const V3<Real> far_pts[2][2] = {{ma, cen}, {cen, mb}};
    for (int q = 0; q < 2; ++q) {
      V3<Real> e[2];
      for (int v = 0; v < 2; ++v) {     // project on the tangent plane of n_p
        const V3<Real> dv = far_pts[q][v];
        const Real hgt = dot(dv, np);
        e[v] = V3<Real>{dv.x - hgt * np.x, dv.y - hgt * np.y, dv.z - hgt * np.z};
      }
      const V3<Real> cr{e[0].y * e[1].z - e[0].z * e[1].y, e[0].z * e[1].x - e[0].x * e[1].z,
                        e[0].x * e[1].y - e[0].y * e[1].x};
      const Real J = sqrt(dot(cr, cr));
      for (int it = 0; it < 16; ++it) {
        const Real tt = c_gl_xf[it], wt = c_gl_wf[it];
        const V3<Real> w{e[0].x + tt * (e[1].x - e[0].x), e[0].y + tt * (e[1].y - e[0].y),
                         e[0].z + tt * (e[1].z - e[0].z)};
        const Real l = sqrt(dot(w, w));
        for (int is = 0; is < 16; ++is) {
          const Real ss = c_gl_xf[is], ws = c_gl_wf[is];
          const Real xk = kappa * ss * l;
          const Real fa = -expm1(-xk) * Real(kInv4Pi) / l;
          Real num;
          if (xk < Real(0.5)) {
            // 1 - e^{-x}(1 + x) = sum_{j>=2} (-1)^j (j - 1) x^j / j!
            Real term = Real(0.5) * xk * xk, s = term;
            for (int jj = 3; jj < 14; ++jj) {
              term *= -xk * (Real)(jj - 1) / ((Real)jj * (Real)(jj - 2));
              s += term;
            }
            num = s;
          } else {
            num = Real(1) - exp(-xk) * (Real(1) + xk);
          }
          const Real fd = num * Real(kInv4Pi) / (ss * ss * l * l * l);
          As += J * wt * ws * fa;
          Ds += J * wt * ws * fd;
        }
      }
    }
  }
  o[0] = As;
  o[1] = 0;
  o[2] = 0;
  o[3] = Ds / ebar;
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

// What the P2P pass sees of a pair: its source lists and the FP32 node data.
struct P2PView {
  const int32_t *node_leaf, *leaf_index, *pidx;
  const int64_t *pptr;
  const dbl4 *center;
  const float4 *pos, *nrm;
  float skip_scale;
};

// Coefficients, one warp per row.  An entry is the near rule minus the point rule, except
// where the P2P pass leaves the pair out (the self entry among them): there it is the
// whole near-rule value and `full` is set.
template <class Real>
__global__ void __launch_bounds__(128) k_near_coef(int64_t n, KernelParams kp, const int32_t *__restrict__ perm,
                                                   const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                                                   const int64_t *__restrict__ inc_ptr,
                                                   const int32_t *__restrict__ inc_tri,
                                                   const double *__restrict__ tri_nrm, const double *__restrict__ area,
                                                   const double *__restrict__ nrm, const int64_t *__restrict__ ptr,
                                                   const int32_t *__restrict__ col, P2PView pv,
                                                   float4 *__restrict__ coef, uint8_t *__restrict__ full) {
  const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n) return;
  const int64_t op = perm[p];
  const double *xp = xyz + 3 * op;
  const V3<Real> np{(Real)nrm[3 * op], (Real)nrm[3 * op + 1], (Real)nrm[3 * op + 2]};
  const Real kappa = (Real)kp.kappa, ebar = (Real)kp.ebar;
  const int lp = pv.node_leaf[p];
  const dbl4 cp = pv.center[lp];
  const float4 xp32 = pv.pos[p];
  const float rsp = p2p_skip_radius(pv.skip_scale, pv.nrm[p].w);
  const int64_t l0 = pv.pptr[pv.leaf_index[lp]], l1 = pv.pptr[pv.leaf_index[lp] + 1];
  for (int64_t j = ptr[p] + lane; j < ptr[p + 1]; j += 32) {
    const int t = col[j];
    const int64_t ot = perm[t];
    Real o[4] = {0, 0, 0, 0};
    bool whole = true;
    if (t == p) {
      self_rule(kappa, ebar, xyz, tri, inc_ptr, inc_tri, op, np, o);
    } else {
      near_rule(kappa, ebar, xyz, tri, inc_ptr, inc_tri, tri_nrm, xp, np, ot, o);
      // Replay the P2P pass's FP32 distance test: when it evaluates this pair, the far
      // rule is already in the product and the entry is the correction.
      const int lt = pv.node_leaf[t];
      bool listed = false;
      for (int64_t k = l0; k < l1 && !listed; ++k) listed = pv.pidx[k] == lt;
      if (listed) {
        const dbl4 ct = pv.center[lt];
        const float4 y = pv.pos[t];
        const float dx = xp32.x - p2p_shift(y.x, ct.x, cp.x), dy = xp32.y - p2p_shift(y.y, ct.y, cp.y),
                    dz = xp32.z - p2p_shift(y.z, ct.z, cp.z);
        whole = !p2p_evaluates(p2p_r2(dx, dy, dz), rsp, p2p_skip_radius(pv.skip_scale, pv.nrm[t].w));
      } else {
        whole = false;                      // a far-field pair (M2L, P2L or L2P side)
      }
    }
    if (!whole) {
      const double *xt = xyz + 3 * ot;
      const V3<Real> d{(Real)(xp[0] - xt[0]), (Real)(xp[1] - xt[1]), (Real)(xp[2] - xt[2])};
      const V3<Real> nt{(Real)nrm[3 * ot], (Real)nrm[3 * ot + 1], (Real)nrm[3 * ot + 2]};
      Real f[4];
      abcd_point(kappa, ebar, d, np, nt, f);
      const Real at = (Real)area[ot];
      for (int k = 0; k < 4; ++k) o[k] -= at * f[k];
    }
    coef[j] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
    full[j] = whole ? 1 : 0;
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
// Quadrature constants (the same for every handle), uploaded once per device.
Err init_quadrature_tables() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return make_err(AFMPB_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return Err{};
  {
    double gx[16], gw[16];
    gauss_legendre_unit(16, gx, gw);
    float fx[16], fw[16];
    for (int i = 0; i < 16; ++i) { fx[i] = (float)gx[i]; fw[i] = (float)gw[i]; }
    AFMPB_CUDA(cudaMemcpyToSymbol(c_gl_xf, fx, sizeof(fx)));
    AFMPB_CUDA(cudaMemcpyToSymbol(c_gl_wf, fw, sizeof(fw)));
    // Radon's 7-point rule (exact for degree 5): centroid and two orbits of three points
    const double r15 = std::sqrt(15.0);
    const double a1 = (6.0 - r15) / 21.0, a2 = (6.0 + r15) / 21.0;
    const double w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
    const double b[21] = {1.0 / 3, 1.0 / 3, 1.0 / 3,
                          a1, a1, 1 - 2 * a1, a1, 1 - 2 * a1, a1, 1 - 2 * a1, a1, a1,
                          a2, a2, 1 - 2 * a2, a2, 1 - 2 * a2, a2, 1 - 2 * a2, a2, a2};
    const double w[7] = {9.0 / 40, w1, w1, w1, w2, w2, w2};
    float bf[21], wf[7];
    for (int i = 0; i < 21; ++i) bf[i] = (float)b[i];
    for (int i = 0; i < 7; ++i) wf[i] = (float)w[i];
    AFMPB_CUDA(cudaMemcpyToSymbol(c_rad_bf, bf, sizeof(bf)));
    AFMPB_CUDA(cudaMemcpyToSymbol(c_rad_wf, wf, sizeof(wf)));
  }
  done[dev] = true;
  return Err{};
}

}  // namespace

Err build_near(afmpb_t *h) {
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  auto &A = h->arena;
  AFMPB_TRY(init_quadrature_tables());
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
  AFMPB_TRY(A.alloc(&h->d_near_full, h->nnz, "near full"));
  const P2PView pv{h->d_node_leaf, h->d_leaf_index, h->d_p2p_idx, h->d_p2p_ptr, h->d_box_center,
                   h->d_pos,       h->d_nrm,        (float)(kP2PSkip * h->opt.near_c)};
  k_near_coef<float><<<div_up(n * 32, 128), 128, 0, s>>>(n, kp, h->d_perm, h->d_xyz, h->d_tri, h->d_inc_ptr,
                                                          h->d_inc_tri, h->d_tri_nrm, h->d_area64, h->d_nrm64,
                                                          h->d_near_ptr, h->d_near_col, pv, h->d_near_coef,
                                                          h->d_near_full);
  AFMPB_TRY(check_launch("k_near_coef"));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(d_cnt);
  return Err{};
}

}  // namespace afmpb
