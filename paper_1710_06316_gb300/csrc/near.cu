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
// Scheduling: self entries take one thread per node.  Off-diagonal entries are handed to
// lanes by a global counter, and each lane's adaptive walk is split into a cheap
// advance-to-next-leaf phase and a leaf-evaluation phase that the whole warp runs
// together (a lane per row with each lane walking its own tree left ~3 of 32 lanes busy).
//
// Precision: all geometry is first taken relative to the target x_p in FP64 (so no
// large-coordinate cancellation reaches the quadrature), then the quadrature runs in
// FP32 (the `Real` template parameter; GB300's FP32 rate is many times its FP64 rate).
#include <algorithm>
#include <cmath>

#include <mutex>

#include "internal.cuh"

namespace afmpb {

__constant__ float c_gl_xf[16], c_gl_wf[16];     // Gauss-Legendre on [0, 1]
__constant__ float c_gl_wi2f[16];                 // w_i / x_i^2 of the same rule
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

// phi0(x) = 1 - e^{-x}, phi1(x) = 1 - e^{-x}(1 + x) and phi2(x) = 1 - e^{-x}(1 + x + x^2/3):
// the screened fractions of the Laplace 1/r, 1/r^3 and 3/r^5 terms.  Below x = 0.5 they are
// summed from their Taylor series through x^10 (coefficients of x^j: (-1)^(j+1) / j!,
// (-1)^j (j-1) / j! and (-1)^(j+1) (j-1)(j-3) / (3 j!)) by Horner's rule with the
// coefficients as compile-time constants, which avoids the cancellation of the direct
// forms and every division; e = e^{-x} serves the direct forms above 0.5.
template <class Real, int N>
__device__ __forceinline__ Real horner(const Real (&c)[N], Real x) {
  Real s = c[N - 1];
#pragma unroll
  for (int j = N - 2; j >= 0; --j) s = s * x + c[j];
  return s;
}

template <class Real>
__device__ __forceinline__ void screened_fractions(Real x, Real e, Real &p0, Real &p1, Real &p2) {
  if (x < Real(0.5)) {
    constexpr Real c0[] = {Real(1),           Real(-1.0 / 2),      Real(1.0 / 6),       Real(-1.0 / 24),
                           Real(1.0 / 120),   Real(-1.0 / 720),    Real(1.0 / 5040),    Real(-1.0 / 40320),
                           Real(1.0 / 362880), Real(-1.0 / 3628800)};                  // x^1 .. x^10
    constexpr Real c1[] = {Real(1.0 / 2),     Real(-1.0 / 3),      Real(1.0 / 8),       Real(-1.0 / 30),
                           Real(1.0 / 144),   Real(-1.0 / 840),    Real(1.0 / 5760),    Real(-1.0 / 45360),
                           Real(1.0 / 403200)};                                          // x^2 .. x^10
    constexpr Real c2[] = {Real(1.0 / 6),     Real(0),             Real(-1.0 / 24),     Real(1.0 / 45),
                           Real(-1.0 / 144),  Real(1.0 / 630),     Real(-1.0 / 3456),   Real(1.0 / 22680),
                           Real(-1.0 / 172800)};                                         // x^2 .. x^10
    const Real x2 = x * x;
    p0 = x * horner(c0, x);
    p1 = x2 * horner(c1, x);
    p2 = x2 * horner(c2, x);
  } else {
    p0 = Real(1) - e;
    p1 = Real(1) - e * (Real(1) + x);
    p2 = Real(1) - e * (Real(1) + x + x * x * Real(1.0 / 3));
  }
}

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float exp_r(float x) { return __expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

// The four Eq. 6 integrands at one point: d = x_target - y_source, n0 target normal,
// ns source normal.  The G - u differences of A and D are formed without cancellation
// (through the screened fractions above).  No division: 1/r from rsqrt, 1/eps_bar given.
template <class Real>
__device__ __forceinline__ void abcd_point(Real kappa, Real inv_ebar, const V3<Real> &d, const V3<Real> &n0,
                                           const V3<Real> &ns, Real o[4]) {
  const Real r2 = dot(d, d);
  const Real ri = rsqrt_r(r2);
  const Real r = r2 * ri;
  const Real ri2 = ri * ri;
  const Real ndn = dot(ns, d), n0d = dot(n0, d), nn0 = dot(ns, n0);
  const Real G = Real(kInv4Pi) * ri;
  const Real G3 = G * ri2;
  const Real G5 = Real(3) * G3 * ri2;
  const Real kr = kappa * r;
  const Real e = exp_r(-kr);
  const Real g1 = (e * (Real(1) + kr)) * G3;
  Real p0, p1, p2;
  screened_fractions(kr, e, p0, p1, p2);
  o[0] = p0 * G;                                 // G - u
  o[1] = ndn * (G3 * inv_ebar - g1);
  o[2] = n0d * (g1 * inv_ebar - G3);
  o[3] = (nn0 * G3 * p1 - ndn * n0d * G5 * p2) * inv_ebar;
}

// FP32 geometry for the quadrature (caller order): each coordinate x split into
// hi = fl32(x) and lo = fl32(x - hi), so that a difference of two points formed as
// (hi_a - hi_b) + (lo_a - lo_b) carries the same ~1e-7 relative error as the FP64
// difference rounded to FP32, without FP64 arithmetic; normals with the patch area,
// facet normals.
struct GeomF32 {
  const float4 *hi, *lo;      // [n] position split, w unused
  const float4 *nrm_area;     // [n] node normal, w = patch area
  const float4 *tri_nrm;      // [nt] unit facet normal
};

__global__ void k_geom_f32(int64_t n, int64_t nt, const double *__restrict__ xyz, const double *__restrict__ nrm,
                           const double *__restrict__ area, const double *__restrict__ tri_nrm,
                           float4 *__restrict__ hi, float4 *__restrict__ lo, float4 *__restrict__ nrm_area,
                           float4 *__restrict__ tnrm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
      h[d] = (float)xyz[3 * i + d];
      l[d] = (float)(xyz[3 * i + d] - (double)h[d]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], 0.f);
    lo[i] = make_float4(l[0], l[1], l[2], 0.f);
    nrm_area[i] = make_float4((float)nrm[3 * i], (float)nrm[3 * i + 1], (float)nrm[3 * i + 2], (float)area[i]);
  }
  if (i < nt) tnrm[i] = make_float4((float)tri_nrm[3 * i], (float)tri_nrm[3 * i + 1], (float)tri_nrm[3 * i + 2], 0.f);
}

__device__ __forceinline__ V3<float> diff_f32(const GeomF32 &g, int64_t a, const float4 &ho, const float4 &lo) {
  const float4 ha = g.hi[a], la = g.lo[a];
  return V3<float>{(ha.x - ho.x) + (la.x - lo.x), (ha.y - ho.y) + (la.y - lo.y), (ha.z - ho.z) + (la.z - lo.z)};
}

// Corners of triangle t rotated so that node v comes first, relative to node o.
__device__ __forceinline__ void tri_rel_f32(const GeomF32 &g, const int32_t *tri, int32_t t, int64_t v, int64_t o,
                                            V3<float> P[3]) {
  int k0 = 0;
  for (int k = 0; k < 3; ++k)
    if (tri[3 * t + k] == v) k0 = k;
  const float4 ho = g.hi[o], lo = g.lo[o];
  for (int j = 0; j < 3; ++j) P[j] = diff_f32(g, tri[3 * t + (k0 + j) % 3], ho, lo);
}

template <class Real>
__device__ void self_rule(Real kappa, Real inv_ebar, const GeomF32 &gf, const int32_t *tri, const int64_t *inc_ptr,
                          const int32_t *inc_tri, int64_t op, const V3<Real> &np, Real o[4]) {
  Real As = 0, Ds = 0;
  for (int64_t j = inc_ptr[op]; j < inc_ptr[op + 1]; ++j) {
    V3<Real> P[3];
    tri_rel_f32(gf, tri, inc_tri[j], op, op, P);   // P[0] = 0 (the node itself)
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
        const Real l2 = dot(w, w);
        const Real il = rsqrt_r(l2), l = l2 * il;
        const Real ca = J * wt * Real(kInv4Pi) * il;             // A: (1 - e^{-x}) / l
        const Real cd = ca * il * il;                             // D: phi1(x) / (s^2 l^3)
        Real sa = 0, sd = 0;
        for (int is = 0; is < 16; ++is) {
          const Real xk = kappa * c_gl_xf[is] * l;
          Real p0, p1, p2;
          screened_fractions(xk, exp_r(-xk), p0, p1, p2);
          sa += c_gl_wf[is] * p0;
          sd += c_gl_wi2f[is] * p1;
        }
        As += ca * sa;
        Ds += cd * sd;
      }
    }
  }
  o[0] = As;
  o[1] = 0;
  o[2] = 0;
  o[3] = Ds * inv_ebar;
}

// Near-set walk.  fill == false: count per row; else write the columns.
__global__ void k_near_search(int64_t n, double cnear, const int32_t *__restrict__ perm,
                              const double *__restrict__ xyz, const double *__restrict__ rho,
                              const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
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
    // box pruning: compared squared (a box at the boundary is kept, never wrongly dropped:
    // the squared test errs by a few ulps and a kept box is only searched)
    const double bR = cnear * (rp + brho[b]);
    if (dx * dx + dy * dy + dz * dz >= bR * bR * (1.0 + 1e-12)) continue;
    if (nchild[b] == 0) {
      // FP32 pre-test on the leaf-relative positions.  The FP32 distance carries an
      // absolute error below 2^-22 (|o| + |q|) per component (|o|, |q|: the offsets it is
      // formed from), so d^2 is off by less than 5e-7 R S + 1e-6 R^2 near the boundary
      // (S = sum of the |o| and |q| components); the FP64 test decides inside twice that.
      const float ox = (float)(x0 - c.x), oy = (float)(x1 - c.y), oz = (float)(x2 - c.z);
      const float so = fabsf(ox) + fabsf(oy) + fabsf(oz);
      const float frp = (float)(cnear * rp), fc = (float)cnear;
      for (int t = bbeg[b]; t < bend[b]; ++t) {
        const float4 q = pos[t];
        const float fx = ox - q.x, fy = oy - q.y, fz = oz - q.z;
        const float fd2 = fx * fx + fy * fy + fz * fz;
        const float fR = fmaf(fc, nrm[t].w, frp);
        const float fR2 = fR * fR;
        const float S = so + fabsf(q.x) + fabsf(q.y) + fabsf(q.z);
        const float margin = 1e-6f * fR * S + 1e-5f * fR2;
        bool in;
        if (fd2 < fR2 - margin) {
          in = true;
        } else if (fd2 > fR2 + margin) {
          in = false;
        } else {
          int64_t ot = perm[t];
          double ex = x0 - xyz[3 * ot], ey = x1 - xyz[3 * ot + 1], ez = x2 - xyz[3 * ot + 2];
          const double d2 = ex * ex + ey * ey + ez * ez;
          const double R = cnear * (rp + rho[ot]);
          // dist < R decided on squares, and with the square root (the defining test)
          // only inside the few-ulp band where the two could disagree
          in = d2 < R * R * (1.0 - 1e-12);
          if (!in && d2 < R * R * (1.0 + 1e-12)) in = sqrt(d2) < R;
        }
        if (t == p || in) {
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

// Self entries (t == p): one thread per node; the fixed 16 x 16 rule keeps the lanes
// of a warp together.  Columns of a row are in ascending Morton order.
__global__ void __launch_bounds__(128) k_near_self(int64_t n, KernelParams kp, const int32_t *__restrict__ perm,
                                                   GeomF32 gf, const int32_t *__restrict__ tri,
                                                   const int64_t *__restrict__ inc_ptr,
                                                   const int32_t *__restrict__ inc_tri,
                                                   const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                                   float4 *__restrict__ coef, uint8_t *__restrict__ full) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t lo = ptr[p], hi = ptr[p + 1] - 1;
  while (lo < hi) {                           // the diagonal entry
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < p) lo = mid + 1; else hi = mid;
  }
  const int64_t op = perm[p];
  const float4 na = gf.nrm_area[op];
  const V3<float> np{na.x, na.y, na.z};
  float o[4] = {0, 0, 0, 0};
  self_rule((float)kp.kappa, (float)(1.0 / kp.ebar), gf, tri, inc_ptr, inc_tri, op, np, o);
  coef[lo] = make_float4(o[0], o[1], o[2], o[3]);
  full[lo] = 1;
}

// What the P2P pass sees of a pair: its source lists (ascending per leaf) and the FP32
// node data.
struct P2PView {
  const int32_t *node_leaf, *leaf_index, *pidx;
  const int64_t *pptr;
  const dbl4 *center;
  const float4 *pos, *nrm;
  float skip_scale;
};

// Replays the P2P pass's FP32 distance test for target p and source t: true when the
// pass leaves the pair out (then the entry holds the whole near-rule value).
__device__ __forceinline__ bool p2p_leaves_out(const P2PView &pv, int p, int t) {
  const int lp = pv.node_leaf[p], lt = pv.node_leaf[t];
  const int li = pv.leaf_index[lp];
  int64_t lo = pv.pptr[li], hi = pv.pptr[li + 1];
  while (lo < hi) {                           // is leaf lt a P2P source of leaf lp?
    const int64_t mid = (lo + hi) >> 1;
    if (pv.pidx[mid] < lt) lo = mid + 1; else hi = mid;
  }
  if (lo == pv.pptr[li + 1] || pv.pidx[lo] != lt) return false;   // far-field pair
  const dbl4 cp = pv.center[lp], ct = pv.center[lt];
  const float4 xp = pv.pos[p], y = pv.pos[t];
  const float dx = xp.x - p2p_shift(y.x, ct.x, cp.x), dy = xp.y - p2p_shift(y.y, ct.y, cp.y),
              dz = xp.z - p2p_shift(y.z, ct.z, cp.z);
  return !p2p_evaluates(p2p_r2(dx, dy, dz), p2p_skip_radius(pv.skip_scale, pv.nrm[p].w),
                        p2p_skip_radius(pv.skip_scale, pv.nrm[t].w));
}

// Off-diagonal entries (t != p).  An entry is the near rule minus the point rule, except
// where the P2P pass leaves the pair out: there it is the whole near-rule value and `full`
// is set.  Lanes take entries from a global counter.  For its entry a lane walks the
// adaptive subdivision tree of every patch piece of t (the same rule and order as a
// recursive walk: pieces by incident triangle, depth first), but the walk is split in two
// phases per step so that the warp stays together where the work is: every lane first
// advances its own walk to its next leaf sub-triangle (cheap, divergent), then all lanes
// evaluate their leaves' 7 quadrature points at once.  The path of the walk is kept as
// 2-bit digits in a register.
__global__ void __launch_bounds__(128) k_near_pairs(int64_t nnz, const int32_t *__restrict__ row,
                                                    unsigned long long *__restrict__ counter, KernelParams kp,
                                                    const int32_t *__restrict__ perm, GeomF32 gf,
                                                    const int32_t *__restrict__ tri,
                                                    const int64_t *__restrict__ inc_ptr,
                                                    const int32_t *__restrict__ inc_tri,
                                                    const int32_t *__restrict__ col,
                                                    P2PView pv, float4 *__restrict__ coef,
                                                    uint8_t *__restrict__ full) {
  const float kappa = (float)kp.kappa, inv_ebar = (float)(1.0 / kp.ebar);
  bool done = false, in_pair = false, in_piece = false, have = false, whole = false;
  int64_t e = 0, tj = 0, tend = 0, op = 0, ot = 0;
  int half = 0, d = 0;
  uint32_t path = 0;                          // digit of level l in bits 2(l-1) .. 2l-1
  V3<float> np{0, 0, 0}, ns{0, 0, 0}, R0{0, 0, 0}, R1{0, 0, 0}, R2{0, 0, 0};
  V3<float> la{0, 0, 0}, lb{0, 0, 0}, lc{0, 0, 0};
  float larea = 0.f, acc[4] = {0, 0, 0, 0};
  while (true) {
    // phase 1: advance to the next leaf (or the next entry)
    while (!have && !done) {
      if (!in_pair) {
        e = (int64_t)atomicAdd(counter, 1ULL);
        if (e >= nnz) {
          done = true;
          break;
        }
        const int p = row[e], t = col[e];
        if (t == p) continue;                 // diagonal: k_near_self
        op = perm[p];
        ot = perm[t];
        {
          const float4 na = gf.nrm_area[op];
          np = V3<float>{na.x, na.y, na.z};
        }
        whole = p2p_leaves_out(pv, p, t);
        tj = inc_ptr[ot];
        tend = inc_ptr[ot + 1];
        half = 0;
        in_piece = false;
        acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
        in_pair = true;
      }
      if (!in_piece) {
        if (tj >= tend) {                     // entry finished
          float o[4] = {acc[0], acc[1], acc[2], acc[3]};
          if (!whole) {
            const V3<float> dd = diff_f32(gf, op, gf.hi[ot], gf.lo[ot]);
            const float4 na = gf.nrm_area[ot];
            const V3<float> nt{na.x, na.y, na.z};
            float f[4];
            abcd_point(kappa, inv_ebar, dd, np, nt, f);
            const float at = na.w;
            for (int k = 0; k < 4; ++k) o[k] -= at * f[k];
          }
          coef[e] = make_float4(o[0], o[1], o[2], o[3]);
          full[e] = whole ? 1 : 0;
          in_pair = false;
          continue;
        }
        const int32_t T = inc_tri[tj];
        V3<float> P[3];
        tri_rel_f32(gf, tri, T, ot, op, P);
        const V3<float> ma{0.5f * (P[0].x + P[1].x), 0.5f * (P[0].y + P[1].y), 0.5f * (P[0].z + P[1].z)};
        const V3<float> mb{0.5f * (P[0].x + P[2].x), 0.5f * (P[0].y + P[2].y), 0.5f * (P[0].z + P[2].z)};
        const float third = 1.0f / 3.0f;
        const V3<float> cen{(P[0].x + P[1].x + P[2].x) * third, (P[0].y + P[1].y + P[2].y) * third,
                            (P[0].z + P[1].z + P[2].z) * third};
        {
          const float4 tn = gf.tri_nrm[T];
          ns = V3<float>{tn.x, tn.y, tn.z};
        }
        R0 = P[0];
        R1 = half == 0 ? ma : cen;
        R2 = half == 0 ? cen : mb;
        d = 0;
        path = 0;
        in_piece = true;
      }
      // the node at (d, path)
      V3<float> a = R0, b = R1, c = R2;
      for (int l = 1; l <= d; ++l) {
        const V3<float> mab{0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z)};
        const V3<float> mbc{0.5f * (b.x + c.x), 0.5f * (b.y + c.y), 0.5f * (b.z + c.z)};
        const V3<float> mca{0.5f * (c.x + a.x), 0.5f * (c.y + a.y), 0.5f * (c.z + a.z)};
        switch ((path >> (2 * (l - 1))) & 3u) {
          case 0: b = mab; c = mca; break;
          case 1: a = mab; c = mbc; break;
          case 2: a = mca; b = mbc; break;
          default: a = mab; b = mbc; c = mca; break;
        }
      }
      const V3<float> e01{b.x - a.x, b.y - a.y, b.z - a.z}, e12{c.x - b.x, c.y - b.y, c.z - b.z},
          e02{c.x - a.x, c.y - a.y, c.z - a.z};
      // split while |centroid| < 3 x the longest edge (compared squared)
      const float diam2 = fmaxf(dot(e01, e01), fmaxf(dot(e12, e12), dot(e02, e02)));
      const float third = 1.0f / 3.0f;
      const V3<float> g{(a.x + b.x + c.x) * third, (a.y + b.y + c.y) * third, (a.z + b.z + c.z) * third};
      if (d < kQuadDepth && dot(g, g) < 9.0f * diam2) {
        ++d;                                  // first child (its digit is 0)
        continue;
      }
      const V3<float> cr{e01.y * e02.z - e01.z * e02.y, e01.z * e02.x - e01.x * e02.z, e01.x * e02.y - e01.y * e02.x};
      la = a;
      lb = b;
      lc = c;
      larea = 0.5f * sqrtf(dot(cr, cr));
      have = true;
      // next node of the walk: the next sibling, climbing past last children
      while (d > 0 && ((path >> (2 * (d - 1))) & 3u) == 3u) {
        path &= ~(3u << (2 * (d - 1)));
        --d;
      }
      if (d > 0) {
        path += 1u << (2 * (d - 1));
      } else {
        in_piece = false;                     // piece done: the other half, or the next triangle
        if (half == 0) {
          half = 1;
        } else {
          half = 0;
          ++tj;
        }
      }
    }
    if (__all_sync(0xffffffffu, !have)) break; // every lane has run out of entries
    // phase 2: the lanes' leaves together
    if (have) {
      for (int q = 0; q < 7; ++q) {
        const float b0 = c_rad_bf[3 * q], b1 = c_rad_bf[3 * q + 1], b2 = c_rad_bf[3 * q + 2];
        const V3<float> dq{-(b0 * la.x + b1 * lb.x + b2 * lc.x), -(b0 * la.y + b1 * lb.y + b2 * lc.y),
                           -(b0 * la.z + b1 * lb.z + b2 * lc.z)};
        float o[4];
        abcd_point(kappa, inv_ebar, dq, np, ns, o);
        const float w = larea * c_rad_wf[q];
        for (int k = 0; k < 4; ++k) acc[k] += w * o[k];
      }
      have = false;
    }
  }
}

__global__ void k_near_rows(int64_t n, const int64_t *__restrict__ ptr, int32_t *__restrict__ row) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  for (int64_t j = ptr[p]; j < ptr[p + 1]; ++j) row[j] = (int32_t)p;
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
    float fwi2[16];
    for (int i = 0; i < 16; ++i) fwi2[i] = (float)(gw[i] / (gx[i] * gx[i]));
    AFMPB_CUDA(cudaMemcpyToSymbol(c_gl_wi2f, fwi2, sizeof(fwi2)));
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
  k_near_search<<<div_up(n, 128), 128, 0, s>>>(n, cnear, h->d_perm, h->d_xyz, h->d_rho64, h->d_pos, h->d_nrm,
                                               h->d_box_center, h->d_box_rho, h->d_box_child0, h->d_box_nchild,
                                               h->d_box_begin, h->d_box_end, d_cnt, nullptr, nullptr, false);
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
  k_near_search<<<div_up(n, 128), 128, 0, s>>>(n, cnear, h->d_perm, h->d_xyz, h->d_rho64, h->d_pos, h->d_nrm,
                                               h->d_box_center, h->d_box_rho, h->d_box_child0, h->d_box_nchild,
                                               h->d_box_begin, h->d_box_end, nullptr, h->d_near_ptr, h->d_near_col,
                                               true);
  AFMPB_TRY(check_launch("k_near_search fill"));
  KernelParams kp{h->kappa, h->ebar};
  AFMPB_TRY(A.alloc(&h->d_near_full, h->nnz, "near full"));
  float4 *g_hi = nullptr, *g_lo = nullptr, *g_na = nullptr, *g_tn = nullptr;
  AFMPB_TRY(A.alloc(&g_hi, n, "near geometry hi"));
  AFMPB_TRY(A.alloc(&g_lo, n, "near geometry lo"));
  AFMPB_TRY(A.alloc(&g_na, n, "near normals"));
  AFMPB_TRY(A.alloc(&g_tn, h->nt, "near facet normals"));
  k_geom_f32<<<div_up(std::max<int64_t>(n, h->nt), 256), 256, 0, s>>>(n, h->nt, h->d_xyz, h->d_nrm64, h->d_area64,
                                                                      h->d_tri_nrm, g_hi, g_lo, g_na, g_tn);
  AFMPB_TRY(check_launch("k_geom_f32"));
  const GeomF32 gf{g_hi, g_lo, g_na, g_tn};
  k_near_self<<<div_up(n, 128), 128, 0, s>>>(n, kp, h->d_perm, gf, h->d_tri, h->d_inc_ptr, h->d_inc_tri,
                                              h->d_near_ptr, h->d_near_col, h->d_near_coef, h->d_near_full);
  AFMPB_TRY(check_launch("k_near_self"));
  int32_t *d_row = nullptr;
  unsigned long long *d_counter = nullptr;
  AFMPB_TRY(A.alloc(&d_row, h->nnz, "near rows"));
  AFMPB_TRY(A.alloc(&d_counter, 1, "near counter"));
  AFMPB_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s));
  k_near_rows<<<div_up(n, 256), 256, 0, s>>>(n, h->d_near_ptr, d_row);
  AFMPB_TRY(check_launch("k_near_rows"));
  const P2PView pv{h->d_node_leaf, h->d_leaf_index, h->d_p2p_idx, h->d_p2p_ptr, h->d_box_center,
                   h->d_pos,       h->d_nrm,        (float)(kP2PSkip * h->opt.near_c)};
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = div_up(h->nnz, 128);   // lanes take entries dynamically; cap the grid
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
  k_near_pairs<<<grid, 128, 0, s>>>(h->nnz, d_row, d_counter, kp, h->d_perm, gf, h->d_tri, h->d_inc_ptr,
                                    h->d_inc_tri, h->d_near_col, pv, h->d_near_coef, h->d_near_full);
  AFMPB_TRY(check_launch("k_near_pairs"));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(g_tn);
  A.release(g_na);
  A.release(g_lo);
  A.release(g_hi);
  A.release(d_counter);
  A.release(d_row);
  A.release(d_cnt);
  return Err{};
}

}  // namespace afmpb
