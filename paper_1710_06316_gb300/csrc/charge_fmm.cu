// charge_fmm.cu -- the charge-surface sums of the right-hand side and of the energy by a
// Laplace FMM over one octree that holds both the surface nodes and the charges.
//
// Both sums are point sums of the Laplace kernel between two point sets:
//   right-hand side of Eq. 5 (charges -> nodes):
//       b_p = (1/eps_out) [ sum_k q_k G(x_p, r_k) ;  sum_k q_k dG/dn_p(x_p, r_k) ]
//   energy (nodes -> charges):
//       phi(r_k) = sum_t a_t [ eps_bar h_t G(r_k, x_t) - f_t dG/dn_t(r_k, x_t) ]
// Summed directly they cost (charges x nodes) pair terms, 1.2e13 for a capsid-sized system
// (1.2M atoms, 10M nodes): seconds each even on the GPU.  Here the library runs its own
// FMM (the same octree build, Chebyshev expansions, compressed M2L and P2P kernels as the
// product, all in FP32) over the union of the two sets.  Every point is both a source
// and a target; the input weights decide which points act as sources:
//   * charges enter as points of unit area with h = q, f = 0 and no normal;
//   * nodes enter with their patch area a_t and normal n_t.
// The product's Laplace output at a target is then sum_t a_t [h_t G - (1/eps_bar) f_t dG/dn_t]
// and its normal derivative at the target (zero for charges, which have no normal):
//   * with charge weights only (nodes f = h = 0): the two rows of b times eps_out;
//   * with the surface solution on the nodes (charges 0): phi(r_k) / eps_bar.
// No pair is skipped: both sums use the point rule everywhere (the product's near-field
// correction and its skip radius do not apply).  Only the Laplace half is translated (no
// Yukawa M2L tables or translations); the P2P, P2M and L2P kernels still form the Yukawa
// half, which is left unused.
//
// Accuracy.  These sums cancel strongly: with charges of both signs the potential at a
// node is ~20x smaller than the sum of its terms' magnitudes, so the FMM's error relative
// to the result is that much larger than the product's.  The charge FMM therefore runs at
// order 8 (Chebyshev interpolation error ~rho^-8 instead of ~rho^-6 for list-2 pairs,
// rho ~ 5.8) with translations compressed at 1e-7: on a 3,000-charge sphere order 6 gave
// 3.7e-5 relative error in the right-hand side, order 8 gives ~1e-5.  The sums run once
// per solve, so the extra cost is paid once.  Both passes run on the handle's stream.
#include <algorithm>

#include "internal.cuh"

namespace afmpb {

namespace {

constexpr int kChargeFmmOrder = 8;
constexpr double kChargeFmmTol = 1e-7;
constexpr int kChargeFmmMinLeaf = 128;   // order 8 expansions hold 512 weights

// Union points: [0, n) = the nodes in Morton order of the handle, [n, n + natoms) = charges.
__global__ void k_cf_points(int64_t n, int64_t natoms, const int32_t *__restrict__ perm,
                            const double *__restrict__ xyz, const double *__restrict__ area,
                            const double *__restrict__ nrm, const double *__restrict__ atoms,
                            double *__restrict__ uxyz, double *__restrict__ uarea, double *__restrict__ unrm,
                            double *__restrict__ urho) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n + natoms) return;
  if (i < n) {
    const int64_t o = perm[i];
    for (int d = 0; d < 3; ++d) {
      uxyz[3 * i + d] = xyz[3 * o + d];
      unrm[3 * i + d] = nrm[3 * o + d];
    }
    uarea[i] = area[o];
  } else {
    const int64_t k = i - n;
    for (int d = 0; d < 3; ++d) {
      uxyz[3 * i + d] = atoms[3 * k + d];
      unrm[3 * i + d] = 0.0;
    }
    uarea[i] = 1.0;
  }
  urho[i] = 0.0;
}

// Source weights in the union's Morton order: charges (sol == nullptr) or the surface
// solution [f; h] (Morton order of the handle).
__global__ void k_cf_load(int64_t nu, int64_t n, const int32_t *__restrict__ uperm, const double *__restrict__ q,
                          const double *__restrict__ sol, float2 *__restrict__ xs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nu) return;
  const int64_t u = uperm[i];
  float2 w = make_float2(0.f, 0.f);
  if (sol) {
    if (u < n) w = make_float2((float)sol[u], (float)sol[n + u]);
  } else if (u >= n) {
    w = make_float2(0.f, (float)q[u - n]);
  }
  xs[i] = w;
}

__global__ void k_cf_rhs_out(int64_t nu, int64_t n, const int32_t *__restrict__ uperm,
                             const float4 *__restrict__ pfar, const float4 *__restrict__ pnear, double scale,
                             double *__restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nu) return;
  const int64_t u = uperm[i];
  if (u >= n) return;
  const float4 a = pfar[i], c = pnear[i];
  b[u] = scale * ((double)a.x + (double)c.x);
  b[n + u] = scale * ((double)a.y + (double)c.y);
}

__global__ void k_cf_phi_out(int64_t nu, int64_t n, const int32_t *__restrict__ uperm,
                             const float4 *__restrict__ pfar, const float4 *__restrict__ pnear, double ebar,
                             double *__restrict__ phi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nu) return;
  const int64_t u = uperm[i];
  if (u < n) return;
  phi[u - n] = ebar * ((double)pfar[i].x + (double)pnear[i].x);
}

// One pass of the union FMM on the handle's stream: far field, then P2P.
Err run_union(afmpb_t *u, cudaStream_t s) {
  AFMPB_TRY(enqueue_far(u, s));
  AFMPB_TRY(enqueue_p2p(u, s));
  return Err{};
}

Err check_union_tc(afmpb_t *u) {
  if (u->opt.precision != 1) return Err{};
  int flag = 0;
  AFMPB_TRY(read_tc_error(u, &flag));
  if (flag) return make_err(AFMPB_ETIMEOUT, "a tensor-core M2L wait expired in the charge FMM");
  return Err{};
}

}  // namespace

bool charge_fmm_wanted(const afmpb_t *h) {
  if (h->natoms == 0) return false;
  if (h->opt.charge_fmm == 1) return false;
  if (h->opt.charge_fmm == 2) return true;
  return (double)h->n * (double)h->natoms > AFMPB_CHARGE_FMM_PAIRS;
}

Err build_charge_fmm(afmpb_t *h) {
  afmpb_t *u = new (std::nothrow) afmpb_t();
  if (!u) return make_err(AFMPB_ENOMEM, "charge FMM: host allocation failed");
  h->cf = u;                                        // owned by h from here on
  u->n = h->n + h->natoms;
  u->nt = 0;
  u->order = std::max(h->order, kChargeFmmOrder);
  u->ncoef = u->order * u->order * u->order;
  u->laplace_only = true;
  u->kappa = h->kappa;
  u->eps_in = h->eps_in;
  u->eps_out = h->eps_out;
  u->ebar = h->ebar;
  u->alpha = h->alpha;
  u->opt = h->opt;
  u->opt.near_c = 0.0;                              // P2P skip radius 0: every pair counts
  u->opt.precision = 0;                             // FP32 M2L (order 8 may stay uncompressed)
  u->opt.leaf_cap = std::max(h->opt.leaf_cap, kChargeFmmMinLeaf);
  if (u->opt.m2l_tol > 0) u->opt.m2l_tol = std::min(u->opt.m2l_tol, kChargeFmmTol);
  u->opt.stream = nullptr;
  u->stream = h->stream;
  u->arena.stream = h->stream;
  u->own_stream = false;
  const int64_t nu = u->n;
  cudaStream_t s = h->stream;
  auto &A = u->arena;
  AFMPB_TRY(A.alloc(&u->d_xyz, 3 * nu, "charge fmm xyz"));
  AFMPB_TRY(A.alloc(&u->d_area64, nu, "charge fmm area"));
  AFMPB_TRY(A.alloc(&u->d_nrm64, 3 * nu, "charge fmm normals"));
  AFMPB_TRY(A.alloc(&u->d_rho64, nu, "charge fmm rho"));
  k_cf_points<<<div_up(nu, 256), 256, 0, s>>>(h->n, h->natoms, h->d_perm, h->d_xyz, h->d_area64, h->d_nrm64,
                                               h->d_atoms, u->d_xyz, u->d_area64, u->d_nrm64, u->d_rho64);
  AFMPB_TRY(check_launch("k_cf_points"));
  AFMPB_TRY(build_tree(u));
  AFMPB_TRY(build_fmm(u));
  // the FP64 point arrays were only needed to build the tree and the sorted points
  A.release(u->d_xyz);
  A.release(u->d_area64);
  A.release(u->d_nrm64);
  A.release(u->d_rho64);
  u->d_xyz = u->d_area64 = u->d_nrm64 = u->d_rho64 = nullptr;
  AFMPB_TRY(A.alloc(&u->d_xs, nu, "charge fmm weights"));
  AFMPB_TRY(A.alloc(&u->d_phi_far, nu, "charge fmm far"));
  AFMPB_TRY(A.alloc(&u->d_phi_near, nu, "charge fmm near"));
  return Err{};
}

Err charge_fmm_rhs(afmpb_t *h, double *b) {
  afmpb_t *u = h->cf;
  cudaStream_t s = h->stream;
  const int64_t nu = u->n;
  k_cf_load<<<div_up(nu, 256), 256, 0, s>>>(nu, h->n, u->d_perm, h->d_q, nullptr, u->d_xs);
  AFMPB_TRY(check_launch("k_cf_load charges"));
  AFMPB_TRY(run_union(u, s));
  k_cf_rhs_out<<<div_up(nu, 256), 256, 0, s>>>(nu, h->n, u->d_perm, u->d_phi_far, u->d_phi_near,
                                                1.0 / h->eps_out, b);
  AFMPB_TRY(check_launch("k_cf_rhs_out"));
  return check_union_tc(u);
}

Err charge_fmm_phi(afmpb_t *h, double *phi) {
  afmpb_t *u = h->cf;
  cudaStream_t s = h->stream;
  const int64_t nu = u->n;
  k_cf_load<<<div_up(nu, 256), 256, 0, s>>>(nu, h->n, u->d_perm, nullptr, h->d_sol, u->d_xs);
  AFMPB_TRY(check_launch("k_cf_load solution"));
  AFMPB_TRY(run_union(u, s));
  k_cf_phi_out<<<div_up(nu, 256), 256, 0, s>>>(nu, h->n, u->d_perm, u->d_phi_far, u->d_phi_near, h->ebar, phi);
  AFMPB_TRY(check_launch("k_cf_phi_out"));
  return check_union_tc(u);
}

}  // namespace afmpb
