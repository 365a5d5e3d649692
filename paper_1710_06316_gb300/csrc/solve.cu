// solve.cu -- right-hand side (Eq. 5), restarted GMRES on the device (Sec. 3.4, Eq. 7)
// and the polar solvation energy.
//
// GMRES keeps its FP64 Krylov basis resident in device memory in the octree's Morton
// order, next to the node data (the paper stores each basis component with its node,
// Sec. 3.4, and feeds the newest basis vector straight to the product).  Each Arnoldi
// step runs the FP32 product, then classical Gram-Schmidt applied twice (two batched
// sets of inner products instead of one global reduction per inner product), the
// Givens update on the device, and reads back one residual estimate for the stop test
// |g_{j+1}| <= eps_rel ||b||_2 + eps_abs (Eq. 7).  All reductions use a fixed
// partition and a fixed summation order, so results are reproducible.
#include <chrono>
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace afmpb {

// ---- permutations between caller order and Morton order -------------------------------
__global__ void k_gather(int64_t n, const int32_t *__restrict__ perm, const float *__restrict__ x,
                         float2 *__restrict__ xs) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t o = perm[p];
  xs[p] = make_float2(x[o], x[n + o]);
}

__global__ void k_scatter(int64_t n, const int32_t *__restrict__ perm, const float *__restrict__ ys,
                          float *__restrict__ y) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t o = perm[p];
  y[o] = ys[p];
  y[n + o] = ys[n + p];
}

Err enqueue_gather(afmpb_t *h, cudaStream_t s, const float *x) {
  k_gather<<<div_up(h->n, 256), 256, 0, s>>>(h->n, h->d_perm, x, h->d_xs);
  return check_launch("k_gather");
}

const void *gather_kernel() { return (const void *)k_gather; }
const void *scatter_kernel() { return (const void *)k_scatter; }

Err enqueue_scatter(afmpb_t *h, cudaStream_t s, float *y) {
  k_scatter<<<div_up(h->n, 256), 256, 0, s>>>(h->n, h->d_perm, h->d_ys, y);
  return check_launch("k_scatter");
}

// ---- right-hand side: b = (1/eps_out) [sum_k q_k G(x_p, r_k); sum_k q_k dG/dn0(x_p, r_k)]
// (Eq. 5; the second row is the normal derivative at the target, as Eq. 3 states).
__global__ void __launch_bounds__(128) k_rhs(const int32_t *__restrict__ leaves, const int32_t *__restrict__ bbeg,
                                             const int32_t *__restrict__ bend, const dbl4 *__restrict__ center,
                                             const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                                             int64_t natoms, const double *__restrict__ atoms,
                                             const double *__restrict__ q, double scale, int64_t n,
                                             double *__restrict__ b) {
  constexpr int CH = 256;
  __shared__ float4 sa[CH];
  const int leaf = leaves[blockIdx.x];
  const dbl4 c = center[leaf];
  for (int t0 = bbeg[leaf]; t0 < bend[leaf]; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    const bool act = t < bend[leaf];
    const float4 xp = act ? pos[t] : make_float4(0, 0, 0, 0);
    const float4 np = act ? nrm[t] : make_float4(0, 0, 0, 0);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k0 = 0; k0 < natoms; k0 += CH) {
      const int cnt = (int)min((int64_t)CH, natoms - k0);
      __syncthreads();
      for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const double *a = atoms + 3 * (k0 + k);
        sa[k] = make_float4((float)(a[0] - c.x), (float)(a[1] - c.y), (float)(a[2] - c.z), (float)q[k0 + k]);
      }
      __syncthreads();
      if (act) {
        float p1 = 0.f, p2 = 0.f;
        for (int k = 0; k < cnt; ++k) {
          const float4 a = sa[k];
          const float dx = xp.x - a.x, dy = xp.y - a.y, dz = xp.z - a.z;
          const float ri = rsqrtf(dx * dx + dy * dy + dz * dz);
          p1 = fmaf(a.w, ri, p1);
          p2 = fmaf(-a.w * (np.x * dx + np.y * dy + np.z * dz), ri * ri * ri, p2);
        }
        s1 += (double)p1;
        s2 += (double)p2;
      }
    }
    if (act) {
      b[t] = scale * s1;
      b[n + t] = scale * s2;
    }
  }
}

// ---- FP64 vector kernels ---------------------------------------------------------------
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;   // valid in thread 0
}

// part[blk * stride + i] = sum over the block's chunk of V_i . w, i in [0, nv)
__global__ void __launch_bounds__(kRedThreads) k_multidot(int64_t len, int nv, const double *__restrict__ V,
                                                          int64_t ldv, const double *__restrict__ w,
                                                          double *__restrict__ part, int stride) {
  __shared__ double sh[32];
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(len, lo + chunk);
  for (int i = 0; i < nv; ++i) {
    const double *v = V + (int64_t)i * ldv;
    double s = 0.0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) s = fma(v[k], w[k], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * stride + i] = s;
  }
}

// out[i] = sum_blk part[blk * stride + i] (fixed order); mode 1: out[i] += that, mode 2: sqrt
__global__ void k_reduce_parts(int nblk, int nv, const double *__restrict__ part, int stride,
                               double *__restrict__ out, int mode) {
  __shared__ double sh[32];
  const int i = blockIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(int64_t)b * stride + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    if (mode == 0) out[i] = s;
    else if (mode == 1) out[i] += s;
    else out[i] = sqrt(s);
  }
}

// v = w / nrm (nrm on the device); also writes the FP32 (f, h) product input
__global__ void k_normalize(int64_t n, const double *__restrict__ w, const double *__restrict__ nrm,
                            double *__restrict__ v, float2 *__restrict__ xs) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double inv = 1.0 / nrm[0];
  const double a = w[p] * inv, b = w[n + p] * inv;
  v[p] = a;
  v[n + p] = b;
  if (xs) xs[p] = make_float2((float)a, (float)b);
}

__global__ void k_to_xs(int64_t n, const double *__restrict__ v, float2 *__restrict__ xs) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  xs[p] = make_float2((float)v[p], (float)v[n + p]);
}

const void *to_xs_kernel() { return (const void *)k_to_xs; }
Err enqueue_to_xs(afmpb_t *h, cudaStream_t s, const double *v) {
  k_to_xs<<<div_up(h->n, 256), 256, 0, s>>>(h->n, v, h->d_xs);
  return check_launch("k_to_xs");
}

// w = ys (FP32 -> FP64), optionally w = b - ys; returns at once when guard is set and
// *guard == 0 (a stopped problem of a batch)
__global__ void k_from_ys(int64_t len, const float *__restrict__ ys, const double *__restrict__ b,
                          double *__restrict__ w, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= len) return;
  w[k] = b ? b[k] - (double)ys[k] : (double)ys[k];
}

__global__ void k_set_beta(double *__restrict__ g, int m, const double *__restrict__ beta) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta[0];
  }
}

// ---- energy: phi_reac(r_k) = sum_t a_t [eps_bar h_t G(r_k, x_t) - f_t dG/dn_t(r_k, x_t)]
__global__ void __launch_bounds__(128) k_energy_part(int nleaf, int leaves_per_blk, const int32_t *__restrict__ leaves,
                                                     const int32_t *__restrict__ bbeg, const int32_t *__restrict__ bend,
                                                     const dbl4 *__restrict__ center, const float4 *__restrict__ pos,
                                                     const float4 *__restrict__ nrm, const double *__restrict__ sol,
                                                     int64_t n, double ebar, int64_t natoms,
                                                     const double *__restrict__ atoms, double *__restrict__ part) {
  constexpr int CH = 128;
  __shared__ float4 sp[CH], sn[CH];
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = k < natoms;
  double acc = 0.0;
  const int l0 = blockIdx.y * leaves_per_blk, l1 = min(nleaf, l0 + leaves_per_blk);
  for (int li = l0; li < l1; ++li) {
    const int leaf = leaves[li];
    const dbl4 c = center[leaf];
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (act) {
      ax = (float)(atoms[3 * k] - c.x);
      ay = (float)(atoms[3 * k + 1] - c.y);
      az = (float)(atoms[3 * k + 2] - c.z);
    }
    for (int t0 = bbeg[leaf]; t0 < bend[leaf]; t0 += CH) {
      const int cnt = min(CH, bend[leaf] - t0);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const float4 p = pos[t0 + e], q = nrm[t0 + e];
        const double f = sol[t0 + e], hh = sol[n + t0 + e];
        sp[e] = make_float4(p.x, p.y, p.z, (float)(p.w * ebar * hh));
        sn[e] = make_float4(q.x, q.y, q.z, (float)(p.w * f));
      }
      __syncthreads();
      if (act) {
        float s = 0.f;
        for (int e = 0; e < cnt; ++e) {
          const float4 p = sp[e], q = sn[e];
          const float dx = ax - p.x, dy = ay - p.y, dz = az - p.z;
          const float ri = rsqrtf(dx * dx + dy * dy + dz * dz);
          s = fmaf(p.w, ri, s);
          s = fmaf(-q.w * (q.x * dx + q.y * dy + q.z * dz), ri * ri * ri, s);
        }
        acc += (double)s;
      }
    }
  }
  if (act) part[(int64_t)blockIdx.y * natoms + k] = acc * kInv4Pi;
}

__global__ void k_energy_final(int nparts, int64_t natoms, const double *__restrict__ part,
                               const double *__restrict__ q, double scale, double *__restrict__ phi,
                               double *__restrict__ E) {
  __shared__ double sh[32];
  double e = 0.0;
  for (int64_t k = threadIdx.x; k < natoms; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * natoms + k];
    phi[k] = s;
    e += 0.5 * q[k] * s;
  }
  e = block_sum(e, sh);
  if (threadIdx.x == 0) E[0] = e * scale;
}

// ---- host ---------------------------------------------------------------------------------
Err build_rhs(afmpb_t *h) {
  const int64_t n = h->n;
  AFMPB_TRY(h->arena.alloc(&h->d_b, 2 * n, "rhs"));
  if (h->natoms == 0) {
    AFMPB_CUDA(cudaMemsetAsync(h->d_b, 0, sizeof(double) * 2 * n, h->stream));
    return Err{};
  }
  if (charge_fmm_wanted(h)) {
    AFMPB_TRY(build_charge_fmm(h));
    return charge_fmm_rhs(h, h->d_b);
  }
  k_rhs<<<h->shape.nleaf, 128, 0, h->stream>>>(h->d_leaves, h->d_box_begin, h->d_box_end, h->d_box_center, h->d_pos,
                                                h->d_nrm, h->natoms, h->d_atoms, h->d_q, kInv4Pi / h->eps_out, n,
                                                h->d_b);
  AFMPB_TRY(check_launch("k_rhs"));
  return Err{};
}

namespace {

int red_blocks(int64_t len) { return (int)std::max<int64_t>(1, std::min<int64_t>(1184, (len + 2047) / 2048)); }

// out[0..nv) = V_i . w (FP64, deterministic)
Err multidot(afmpb_t *h, int64_t len, int nv, const double *V, int64_t ldv, const double *w, double *out, int mode) {
  const int nb = red_blocks(len);
  const int stride = h->gm_m + 2;
  k_multidot<<<nb, kRedThreads, 0, h->stream>>>(len, nv, V, ldv, w, h->d_part, stride);
  AFMPB_TRY(check_launch("k_multidot"));
  k_reduce_parts<<<nv, 256, 0, h->stream>>>(nb, nv, h->d_part, stride, out, mode);
  return check_launch("k_reduce_parts");
}

Err norm2(afmpb_t *h, int64_t len, const double *w, double *out) { return multidot(h, len, 1, w, 0, w, out, 2); }

}  // namespace

// ---- the Arnoldi step as step-indexed kernels --------------------------------------------
// One captured Arnoldi step serves every step of a cycle: the kernels read the step index
// j from device memory (gm[0]) instead of taking it as a launch parameter, and the last
// kernel of the step advances j and sets the condition of the graph WHILE loop that runs
// the steps.  gm[1] counts the steps, gm[2] is the second-pass flag of the one-reduction
// form (the guarded kernels return at once while it is 0) and gm[3] counts second passes.
// Reorthogonalise when ||w - V h|| < kReorthTol ||w||: the test the FP64 reference GMRES
// applies to its second Gram-Schmidt pass.
constexpr double kReorthTol = 1e-3;

__global__ void k_to_xs_j(int64_t n, const double *__restrict__ V, int64_t n2, const int *__restrict__ gm,
                          float2 *__restrict__ xs, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double *v = V + (int64_t)gm[0] * n2;
  xs[p] = make_float2((float)v[p], (float)v[n + p]);
}

// part[blk * stride + i] = block's share of V_i . w for i < j + 1, and of w . w at i = j + 1
// when self_dot == 1 (self_dot == 2: w . w alone, at i = 0); returns at once when guard is
// set and *guard == 0.
__global__ void __launch_bounds__(kRedThreads) k_multidot_j(int64_t len, const int *__restrict__ gm,
                                                            const double *__restrict__ V, int64_t ldv,
                                                            const double *__restrict__ w, double *__restrict__ part,
                                                            int stride, int self_dot, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double sh[32];
  const int nv = self_dot == 2 ? 0 : gm[0] + 1;        // 2: w . w alone, at index 0
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(len, lo + chunk);
  for (int i = 0; i < nv + (self_dot ? 1 : 0); ++i) {
    const double *v = i < nv ? V + (int64_t)i * ldv : w;
    double s = 0.0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) s = fma(v[k], w[k], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * stride + i] = s;
  }
}

// out[i] = sum_blk part[blk * stride + i] for i < j + 1 + extra (fixed order)
__global__ void k_reduce_parts_j(int nblk, const int *__restrict__ gm, int extra, const double *__restrict__ part,
                                 int stride, double *__restrict__ out, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double sh[32];
  const int i = blockIdx.x;
  if (i >= gm[0] + 1 + extra) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(int64_t)b * stride + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[i] = s;
}

// w -= sum_{i <= j} c_i V_i
__global__ void k_sub_combo_j(int64_t len, const int *__restrict__ gm, const double *__restrict__ V, int64_t ldv,
                              const double *__restrict__ c, double *__restrict__ w, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  const int nv = gm[0] + 1;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nv; ++i) s = fma(c[i], V[(int64_t)i * ldv + k], s);
    w[k] -= s;
  }
}

__global__ void k_add_small_j(const int *__restrict__ gm, const double *__restrict__ a, double *__restrict__ b,
                              const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  for (int i = threadIdx.x; i < gm[0] + 1; i += blockDim.x) b[i] += a[i];
}

// hcol[j + 1] = sqrt(sum_blk part[blk * stride])  (the norm of w after the last pass)
__global__ void k_norm_to_j(int nblk, const double *__restrict__ part, int stride, const int *__restrict__ gm,
                            double *__restrict__ hcol, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(int64_t)b * stride];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) hcol[gm[0] + 1] = sqrt(s);
}

// One-reduction form: hcol[0..j] = V^T w and hcol[j+1] = ||w||^2 from the fused reduction.
// ||w - V h||^2 = ||w||^2 - ||h||^2 (Pythagoras, V orthonormal); below kReorthTol^2 ||w||^2
// the difference has lost its digits and the orthogonality is in doubt: flag a second pass.
__global__ void k_pythagoras_j(int *__restrict__ gm, double *__restrict__ hcol, const int *__restrict__ guard) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (guard && *guard == 0) return;
  const int j = gm[0];
  const double wsq = hcol[j + 1];
  double hsq = 0.0;
  for (int i = 0; i <= j; ++i) hsq = fma(hcol[i], hcol[i], hsq);
  const double rest = wsq - hsq;
  if (rest > kReorthTol * kReorthTol * wsq) {
    hcol[j + 1] = sqrt(rest);
    gm[2] = 0;
  } else {
    gm[2] = 1;
    gm[3] += 1;
  }
}

// V_{j+1} = w / hcol[j+1]
__global__ void k_normalize_j(int64_t n, const double *__restrict__ w, const double *__restrict__ hcol,
                              const int *__restrict__ gm, double *__restrict__ V, int64_t n2,
                              const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int j = gm[0];
  const double inv = 1.0 / hcol[j + 1];
  double *v = V + (int64_t)(j + 1) * n2;
  v[p] = w[p] * inv;
  v[n + p] = w[n + p] * inv;
}

// Givens update of Hessenberg column j: the new column from hcol, the earlier rotations
// applied, a new rotation zeroing its subdiagonal, the residual estimate |g[j + 1]|.
__device__ __forceinline__ void givens_update(int j, int m, const double *__restrict__ hcol, double *__restrict__ H,
                                              double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                                              double *__restrict__ res) {
  double *col = H + (int64_t)j * (m + 1);
  for (int i = 0; i <= j + 1; ++i) col[i] = hcol[i];
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j], b = col[j + 1];
  const double den = hypot(a, b);
  cs[j] = den > 0 ? a / den : 1.0;
  sn[j] = den > 0 ? b / den : 0.0;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  res[0] = fabs(g[j + 1]);
}

// (as k_givens, j from the device)
__global__ void k_givens_j(const int *__restrict__ gm, int m, const double *__restrict__ hcol, double *__restrict__ H,
                           double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                           double *__restrict__ res, const int *__restrict__ guard) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (guard && *guard == 0) return;
  givens_update(gm[0], m, hcol, H, cs, sn, g, res);
}

// End of a step: j += 1; continue the WHILE loop while the Givens residual estimate is
// above the tolerance of Eq. 7 and the basis has room.
__global__ void k_step_end(int *__restrict__ gm, int m, const double *__restrict__ res, const double *__restrict__ tol,
                           cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = gm[0] + 1;
  gm[0] = j;
  gm[1] += 1;
  const double r = res[0];
  const bool go = j < m && r > tol[0];      // a NaN residual stops as well
  cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// back substitution H(0:k,0:k) y = g(0:k), k = gm[0] steps of the cycle, y over g
__global__ void k_backsolve_j(const int *__restrict__ gm, int m, const double *__restrict__ H, double *__restrict__ g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = gm[0];
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(int64_t)c * (m + 1) + i] * g[c];
    g[i] = s / H[(int64_t)i * (m + 1) + i];
  }
}

// x += sum_{i < k} y_i V_i, k = gm[0]
__global__ void k_update_x(int64_t len, const int *__restrict__ gm, const double *__restrict__ V, int64_t ldv,
                           const double *__restrict__ y, double *__restrict__ x) {
  const int k = gm[0];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(y[i], V[(int64_t)i * ldv + p], s);
    x[p] += s;
  }
}

__global__ void k_cycle_start(int *__restrict__ gm) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    gm[0] = 0;
    gm[2] = 0;
  }
}

// ---- the default Arnoldi step (classical Gram-Schmidt twice) in four kernels ----------------
// Each reduction is folded by the block that finishes last (an atomic ticket in gm[5..7]):
// it sums every block's partial in block order, one warp per coefficient with a fixed
// shuffle tree, so the result does not depend on which block ends last.  The three
// passes over the basis are: w = y with the dots V^T w; w -= V h1 with the dots V^T w;
// w -= V h2 with ||w||^2.  The third pass's last block also applies the Givens update and
// the stop test of Eq. 7; the fourth kernel normalises V_{j+1} and writes it, in FP32, as
// the next product's input.
__device__ __forceinline__ bool last_block_of(int *ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

__device__ __forceinline__ void fold_parts(int nb, int cnt, const double *part, int stride, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < cnt; i += nw) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(part + (int64_t)b * stride + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
  }
}

// w = ys (FP32 -> FP64); h1 = V_{0..j}^T w
__global__ void __launch_bounds__(kRedThreads) k_gs_first(int64_t len, int *__restrict__ gm, const double *__restrict__ V,
                                                          int64_t ldv, const float *__restrict__ ys,
                                                          double *__restrict__ w, double *__restrict__ part, int stride,
                                                          double *__restrict__ hcol, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double sh[32];
  const int nv = gm[0] + 1;
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(len, lo + chunk);
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) w[k] = (double)ys[k];
  for (int i = 0; i < nv; ++i) {
    const double *v = V + (int64_t)i * ldv;
    double a = 0.0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) a = fma(v[k], w[k], a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * stride + i] = a;
  }
  if (last_block_of(gm + 5)) {
    fold_parts(gridDim.x, nv, part, stride, hcol);
    if (threadIdx.x == 0) gm[5] = 0;
  }
}

// w -= V h1; h2 = V^T w; h1 += h2
__global__ void __launch_bounds__(kRedThreads) k_gs_second(int64_t len, int *__restrict__ gm, const double *__restrict__ V,
                                                           int64_t ldv, double *__restrict__ w, double *__restrict__ part,
                                                           int stride, double *__restrict__ hcol, double *__restrict__ hcol2,
                                                           const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double sh[32];
  const int nv = gm[0] + 1;
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(len, lo + chunk);
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(hcol[i], V[(int64_t)i * ldv + k], a);
    w[k] -= a;
  }
  for (int i = 0; i < nv; ++i) {
    const double *v = V + (int64_t)i * ldv;
    double a = 0.0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) a = fma(v[k], w[k], a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * stride + i] = a;
  }
  if (last_block_of(gm + 6)) {
    fold_parts(gridDim.x, nv, part, stride, hcol2);
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hcol[i] += hcol2[i];
    if (threadIdx.x == 0) gm[6] = 0;
  }
}

// w -= V h2; ||w||; Givens update; j += 1 and the stop test (batch: the problem's running
// flag, else the condition of the graph's WHILE loop)
__global__ void __launch_bounds__(kRedThreads) k_gs_norm(int64_t len, int *__restrict__ gm, int m,
                                                         const double *__restrict__ V, int64_t ldv, double *__restrict__ w,
                                                         double *__restrict__ part, int stride, double *__restrict__ hcol,
                                                         const double *__restrict__ hcol2, double *__restrict__ H,
                                                         double *__restrict__ cs, double *__restrict__ sn,
                                                         double *__restrict__ g, double *__restrict__ res,
                                                         const double *__restrict__ tol, int batch,
                                                         cudaGraphConditionalHandle loop, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double sh[32];
  const int j = gm[0], nv = j + 1;
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(len, lo + chunk);
  double q = 0.0;
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(hcol2[i], V[(int64_t)i * ldv + k], a);
    const double x = w[k] - a;
    w[k] = x;
    q = fma(x, x, q);
  }
  q = block_sum(q, sh);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * stride] = q;
  if (last_block_of(gm + 7)) {
    __shared__ double s_nrm;
    fold_parts(gridDim.x, 1, part, stride, &s_nrm);
    __syncthreads();
    if (threadIdx.x == 0) {
      gm[7] = 0;
      hcol[j + 1] = sqrt(s_nrm);
      givens_update(j, m, hcol, H, cs, sn, g, res);
      gm[0] = j + 1;
      gm[1] += 1;
      const bool go = j + 1 < m && res[0] > tol[0];      // a NaN residual stops as well
      if (batch) {
        if (!go) {
          gm[4] = 0;
          gm[2] = 0;
        }
      } else {
        cudaGraphSetConditional(loop, go ? 1u : 0u);
      }
    }
  }
}

// V_{j+1} = w / ||w|| (j + 1 = gm[0] after the step end) and its FP32 copy for the next product
__global__ void k_gs_normalize(int64_t n, const int *__restrict__ gm, const double *__restrict__ w,
                               const double *__restrict__ hcol, double *__restrict__ V, int64_t n2,
                               float2 *__restrict__ xs, const int *__restrict__ guard) {
  if (guard && *guard == 0) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int j = gm[0];
  const double inv = 1.0 / hcol[j];
  double *v = V + (int64_t)j * n2;
  const double a = w[p] * inv, b = w[n + p] * inv;
  v[p] = a;
  v[n + p] = b;
  xs[p] = make_float2((float)a, (float)b);
}

__global__ void k_step_end_b(int *__restrict__ gm, int m, const double *__restrict__ res,
                             const double *__restrict__ tol);

namespace {

// Krylov dimension of the no-restart mode: the largest whose basis fits in half of the
// free device memory, at most AFMPB_RESTART_NONE_MAX.
Err restart_length(afmpb_t *h, int *m) {
  if (h->opt.restart != AFMPB_RESTART_NONE) {
    *m = h->opt.restart;
    return Err{};
  }
  if (h->gm_m > 0 && h->d_V) {                 // keep the basis of an earlier solve
    *m = h->gm_m;
    return Err{};
  }
  size_t free_b = 0, total_b = 0;
  AFMPB_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t per = sizeof(double) * 2 * (size_t)h->n;
  const size_t fit = free_b / 2 / per;
  *m = (int)std::max<size_t>(2, std::min<size_t>(AFMPB_RESTART_NONE_MAX, fit > 1 ? fit - 1 : 1));
  return Err{};
}

// The Arnoldi step around the product: V_j to the FP32 product input, then (after the
// product) orthogonalisation, normalisation and the Givens update.  `act` (nullable) is a
// batch problem's running flag: every kernel returns at once while it is 0.
Err enqueue_step_head(afmpb_t *h, cudaStream_t cap, const int *act) {
  if (h->opt.orth == 0) return Err{};     // the previous step (or the cycle start) wrote xs
  const int64_t n = h->n, n2 = 2 * n;
  k_to_xs_j<<<div_up(n, 256), 256, 0, cap>>>(n, h->d_V, n2, h->d_gm_int, h->d_xs, act);
  return check_launch("k_to_xs_j");
}

// The product input V_j in FP32 at a cycle start (the fused step writes it for the next
// step itself).
Err enqueue_cycle_xs(afmpb_t *h, cudaStream_t s, const int *act) {
  if (h->opt.orth != 0) return Err{};
  const int64_t n = h->n, n2 = 2 * n;
  k_to_xs_j<<<div_up(n, 256), 256, 0, s>>>(n, h->d_V, n2, h->d_gm_int, h->d_xs, act);
  return check_launch("k_to_xs_j (cycle start)");
}

Err enqueue_step_tail(afmpb_t *h, int m, cudaStream_t cap, const int *act, bool batch, cudaGraphConditionalHandle loop) {
  const int64_t n = h->n, n2 = 2 * n;
  const int orth = h->opt.orth;
  if (orth == 0) {
    const int nb = red_blocks(n2), stride = m + 2;
    int *gm = h->d_gm_int;
    k_gs_first<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_ys, h->d_w, h->d_part, stride, h->d_hcol, act);
    k_gs_second<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, h->d_hcol, h->d_hcol2, act);
    k_gs_norm<<<nb, kRedThreads, 0, cap>>>(n2, gm, m, h->d_V, n2, h->d_w, h->d_part, stride, h->d_hcol, h->d_hcol2,
                                           h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_scal + 2, h->d_scal + 4,
                                           batch ? 1 : 0, loop, act);
    k_gs_normalize<<<div_up(n, 256), 256, 0, cap>>>(n, gm, h->d_w, h->d_hcol, h->d_V, n2, h->d_xs, act);
    return check_launch("arnoldi step (fused)");
  }
  const int *gm = h->d_gm_int;
  int *gmw = h->d_gm_int;
  const int *guard = gm + 2;              // second-pass flag: 0 whenever the problem is stopped
  const int *first = act;                 // the first pass runs while the problem runs
  const int nb = red_blocks(n2), stride = m + 2;
  const int nb_el = div_up(n, 256), nb_el2 = div_up(n2, 256);
  const int nb_comb = std::min(nb_el2, 4 * 1184);
  k_from_ys<<<nb_el2, 256, 0, cap>>>(n2, h->d_ys, nullptr, h->d_w, act);
  if (orth == 0) {      // classical Gram-Schmidt twice, then the norm: three reductions
    k_multidot_j<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, 0, first);
    k_reduce_parts_j<<<m + 1, 256, 0, cap>>>(nb, gm, 0, h->d_part, stride, h->d_hcol, first);
    k_sub_combo_j<<<nb_comb, 256, 0, cap>>>(n2, gm, h->d_V, n2, h->d_hcol, h->d_w, first);
    k_multidot_j<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, 0, first);
    k_reduce_parts_j<<<m + 1, 256, 0, cap>>>(nb, gm, 0, h->d_part, stride, h->d_hcol2, first);
    k_sub_combo_j<<<nb_comb, 256, 0, cap>>>(n2, gm, h->d_V, n2, h->d_hcol2, h->d_w, first);
    k_add_small_j<<<1, 128, 0, cap>>>(gm, h->d_hcol2, h->d_hcol, first);
    if (act) k_multidot_j<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, 2, act);
    else k_multidot<<<nb, kRedThreads, 0, cap>>>(n2, 1, h->d_w, 0, h->d_w, h->d_part, stride);
    k_norm_to_j<<<1, 256, 0, cap>>>(nb, h->d_part, stride, gm, h->d_hcol, first);
  } else {              // one fused reduction; a guarded second pass on loss of orthogonality
    k_multidot_j<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, 1, first);
    k_reduce_parts_j<<<m + 2, 256, 0, cap>>>(nb, gm, 1, h->d_part, stride, h->d_hcol, first);
    k_sub_combo_j<<<nb_comb, 256, 0, cap>>>(n2, gm, h->d_V, n2, h->d_hcol, h->d_w, first);
    k_pythagoras_j<<<1, 1, 0, cap>>>(gmw, h->d_hcol, act);
    k_multidot_j<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, 0, guard);
    k_reduce_parts_j<<<m + 1, 256, 0, cap>>>(nb, gm, 0, h->d_part, stride, h->d_hcol2, guard);
    k_sub_combo_j<<<nb_comb, 256, 0, cap>>>(n2, gm, h->d_V, n2, h->d_hcol2, h->d_w, guard);
    k_add_small_j<<<1, 128, 0, cap>>>(gm, h->d_hcol2, h->d_hcol, guard);
    k_multidot_j<<<nb, kRedThreads, 0, cap>>>(n2, gm, h->d_V, n2, h->d_w, h->d_part, stride, 2, guard);
    k_norm_to_j<<<1, 256, 0, cap>>>(nb, h->d_part, stride, gm, h->d_hcol, guard);
  }
  k_normalize_j<<<nb_el, 256, 0, cap>>>(n, h->d_w, h->d_hcol, gm, h->d_V, n2, act);
  k_givens_j<<<1, 1, 0, cap>>>(gm, m, h->d_hcol, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_scal + 2, act);
  if (batch) k_step_end_b<<<1, 1, 0, cap>>>(gmw, m, h->d_scal + 2, h->d_scal + 4);
  else k_step_end<<<1, 1, 0, cap>>>(gmw, m, h->d_scal + 2, h->d_scal + 4, loop);
  return check_launch("arnoldi step");
}

// The cycle graph: a WHILE node whose body is one Arnoldi step (the FP32 product of V_j,
// orthogonalisation, normalisation, Givens update, stop test).
Err build_cycle_graph(afmpb_t *h, int m) {
  const int orth = h->opt.orth;
  if (h->graph_cycle) {
    cudaGraphExecDestroy(h->graph_cycle);
    h->graph_cycle = nullptr;
  }
  cudaGraph_t g = nullptr;
  AFMPB_CUDA(cudaGraphCreate(&g, 0));
  struct GraphGuard { cudaGraph_t g; ~GraphGuard() { if (g) cudaGraphDestroy(g); } } gg{g};
  cudaGraphConditionalHandle loop;
  AFMPB_CUDA(cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  AFMPB_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  int lo = 0, hi = 0;
  AFMPB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  cudaStream_t cap = nullptr;
  AFMPB_CUDA(cudaStreamCreateWithPriority(&cap, cudaStreamNonBlocking, hi));
  struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamDestroy(s); } } sg{cap};
  AFMPB_CUDA(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  Err e = enqueue_step_head(h, cap, nullptr);
  if (e.ok()) e = enqueue_product_kernels(h, cap);
  if (e.ok()) e = enqueue_step_tail(h, m, cap, nullptr, false, loop);
  cudaGraph_t out = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cap, &out);
  if (!e.ok()) return e;
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("cudaStreamEndCapture (cycle): ") + cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&h->graph_cycle, g, 0);
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("cudaGraphInstantiate (cycle): ") + cudaGetErrorString(ce));
  h->cycle_m = m;
  h->cycle_orth = orth;
  return Err{};
}

// The Krylov basis, Hessenberg matrix, work vectors and step state of an m-step cycle
// (kept from an earlier solve of the same m).
Err prepare_gmres(afmpb_t *h, int m) {
  const int64_t n2 = 2 * h->n;
  auto &A = h->arena;
  if (h->gm_m != m || !h->d_V) {
    if (h->d_V) {
      for (void *p : {(void *)h->d_V, (void *)h->d_w, (void *)h->d_H, (void *)h->d_g, (void *)h->d_cs,
                      (void *)h->d_sn, (void *)h->d_part, (void *)h->d_hcol, (void *)h->d_hcol2, (void *)h->d_scal})
        A.release(p);
    }
    h->gm_m = m;
    AFMPB_TRY(A.alloc(&h->d_V, (size_t)(m + 1) * n2, "gmres basis"));
    AFMPB_TRY(A.alloc(&h->d_w, n2, "gmres w"));
    AFMPB_TRY(A.alloc(&h->d_H, (size_t)(m + 1) * m, "gmres H"));
    AFMPB_TRY(A.alloc(&h->d_g, m + 2, "gmres g"));
    AFMPB_TRY(A.alloc(&h->d_cs, m + 1, "gmres cs"));
    AFMPB_TRY(A.alloc(&h->d_sn, m + 1, "gmres sn"));
    AFMPB_TRY(A.alloc(&h->d_part, (size_t)1184 * (m + 2), "gmres partials"));
    AFMPB_TRY(A.alloc(&h->d_hcol, m + 2, "gmres hcol"));
    AFMPB_TRY(A.alloc(&h->d_hcol2, m + 2, "gmres hcol2"));
    AFMPB_TRY(A.alloc(&h->d_scal, 8, "gmres scalars"));
    if (!h->d_gm_int) AFMPB_TRY(A.alloc(&h->d_gm_int, 8, "gmres step state"));
    if (!h->h_pinned) AFMPB_CUDA(cudaMallocHost(&h->h_pinned, 8 * sizeof(double)));
  }
  if (!h->d_sol) AFMPB_TRY(A.alloc(&h->d_sol, n2, "solution"));
  return Err{};
}

}  // namespace

Err run_solve(afmpb_t *h, afmpb_solve_info *info) {
  const int64_t n = h->n, n2 = 2 * n;
  int m = 0;
  AFMPB_TRY(restart_length(h, &m));
  const int max_restart = h->opt.max_restart;
  cudaStream_t s = h->stream;
  AFMPB_TRY(prepare_gmres(h, m));
  if (!h->graph_cycle || h->cycle_m != m || h->cycle_orth != h->opt.orth) AFMPB_TRY(build_cycle_graph(h, m));
  double *x = h->d_sol;
  volatile double *hp = h->h_pinned;
  const int nb_el = div_up(n, 256), nb_el2 = div_up(n2, 256);
  const int nb_comb = std::min(nb_el2, 4 * 1184);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  AFMPB_CUDA(cudaEventCreate(&e0));
  AFMPB_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } guard{e0, e1};
  AFMPB_CUDA(cudaEventRecord(h->ev_t0, s));
  auto read_scalar = [&](const double *d, int slot) -> Err {
    AFMPB_CUDA(cudaMemcpyAsync((double *)hp + slot, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
    return Err{};
  };
  int h_gm[4] = {0, 0, 0, 0};

  AFMPB_TRY(norm2(h, n2, h->d_b, h->d_scal + 0));
  AFMPB_TRY(read_scalar(h->d_scal + 0, 0));
  const double bnorm = hp[0];
  h->bnorm = bnorm;
  const double tol = h->tol * bnorm + h->opt.abs_tol;
  hp[4] = tol;
  AFMPB_CUDA(cudaMemcpyAsync(h->d_scal + 4, (const double *)hp + 4, sizeof(double), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemsetAsync(h->d_gm_int, 0, 8 * sizeof(int), s));
  AFMPB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n2, s));
  int restarts = 0, products = 0;
  bool converged = false;
  double res = bnorm;
  for (int cycle = 0; cycle <= max_restart && !converged; ++cycle) {
    if (cycle == 0) {   // x0 = 0: r = b
      AFMPB_CUDA(cudaMemcpyAsync(h->d_w, h->d_b, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
    } else {
      ++restarts;
      ++products;
      AFMPB_TRY(product_from64(h, s, x));
      k_from_ys<<<nb_el2, 256, 0, s>>>(n2, h->d_ys, h->d_b, h->d_w, nullptr);
      AFMPB_TRY(check_launch("residual"));
    }
    AFMPB_TRY(norm2(h, n2, h->d_w, h->d_scal + 1));
    AFMPB_TRY(read_scalar(h->d_scal + 1, 1));
    res = hp[1];
    if (!(res > tol)) {
      converged = !std::isnan(res);
      break;
    }
    k_normalize<<<nb_el, 256, 0, s>>>(n, h->d_w, h->d_scal + 1, h->d_V, nullptr);
    k_set_beta<<<1, 1, 0, s>>>(h->d_g, m, h->d_scal + 1);
    k_cycle_start<<<1, 1, 0, s>>>(h->d_gm_int);
    AFMPB_TRY(check_launch("gmres start"));
    AFMPB_TRY(enqueue_cycle_xs(h, s, nullptr));
    // the Arnoldi steps of the cycle: one graph launch, no host synchronisation inside
    AFMPB_CUDA(cudaGraphLaunch(h->graph_cycle, s));
    // x += V y, H y = g
    k_backsolve_j<<<1, 1, 0, s>>>(h->d_gm_int, m, h->d_H, h->d_g);
    k_update_x<<<nb_comb, 256, 0, s>>>(n2, h->d_gm_int, h->d_V, n2, h->d_g, x);
    AFMPB_TRY(check_launch("gmres update"));
    AFMPB_CUDA(cudaMemcpyAsync(h_gm, h->d_gm_int, sizeof(h_gm), cudaMemcpyDeviceToHost, s));
    AFMPB_TRY(read_scalar(h->d_scal + 2, 2));
    res = hp[2];
    products += h_gm[0];
    if (!(res > tol)) converged = !std::isnan(res);
  }
  // true residual with one more product (its CUDA-event time stands for every product)
  AFMPB_CUDA(cudaEventRecord(e0, s));
  AFMPB_TRY(product_from64(h, s, x));
  AFMPB_CUDA(cudaEventRecord(e1, s));
  ++products;
  k_from_ys<<<nb_el2, 256, 0, s>>>(n2, h->d_ys, h->d_b, h->d_w, nullptr);
  AFMPB_TRY(norm2(h, n2, h->d_w, h->d_scal + 3));
  AFMPB_TRY(read_scalar(h->d_scal + 3, 3));
  float ms_one = 0.f;
  AFMPB_CUDA(cudaEventElapsedTime(&ms_one, e0, e1));
  AFMPB_CUDA(cudaEventRecord(h->ev_t1, s));
  AFMPB_CUDA(cudaEventSynchronize(h->ev_t1));
  float ms_all = 0.f;
  AFMPB_CUDA(cudaEventElapsedTime(&ms_all, h->ev_t0, h->ev_t1));
  h->solved = true;
  {
    int flag = 0;
    AFMPB_TRY(read_tc_error(h, &flag));
    if (flag) return make_err(AFMPB_ETIMEOUT, "a bounded device wait expired during the solve; the products are not valid");
  }
  if (info) {
    info->iters = h_gm[1];
    info->restarts = restarts;
    info->res_est = res;
    info->res_true = bnorm > 0 ? hp[3] / bnorm : hp[3];
    info->bnorm = bnorm;
    info->ms_setup = h->ms_setup;
    info->ms_matvec_total = ms_one * products;
    info->ms_gmres = ms_all;
    info->nnz_near = h->nnz;
    info->n_boxes = h->shape.nbox;
    info->krylov_dim = m;
    info->second_passes = h->opt.orth == 0 ? h_gm[1] : h_gm[3];
  }
  if (!converged) return make_err(AFMPB_ENOCONV, "GMRES did not reach the tolerance within max_restart cycles");
  return Err{};
}

// ---- batched solve: several problems' GMRES in lockstep ----------------------------------
// Each problem keeps its own Krylov state; one graph launch runs a restart cycle of all of
// them.  Its WHILE body is one Arnoldi step of every running problem with one P2P launch
// and one tensor-core M2L launch over all their work, the rest of each product and each
// orthogonalisation on a branch of its own.  gm[4] says whether a problem runs in the
// cycle: it is set at the cycle start, cleared when its Givens residual meets the
// tolerance or its basis is full, and every kernel of a stopped problem returns at once;
// the loop ends when no problem runs.

__global__ void k_cycle_start_b(int *__restrict__ gm, int run) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    gm[0] = 0;
    gm[2] = 0;
    gm[4] = run;
  }
}

// End of a running problem's step: j += 1; it stops (and its second-pass flag is cleared,
// so that no guarded kernel of it runs) when the residual estimate meets the tolerance or
// the basis has no room.
__global__ void k_step_end_b(int *__restrict__ gm, int m, const double *__restrict__ res,
                             const double *__restrict__ tol) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || gm[4] == 0) return;
  const int j = gm[0] + 1;
  gm[0] = j;
  gm[1] += 1;
  const double r = res[0];
  if (!(j < m && r > tol[0])) {
    gm[4] = 0;
    gm[2] = 0;
  }
}

__global__ void k_batch_go(int k, int *const *__restrict__ gms, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned any = 0;
  for (int i = 0; i < k; ++i) any |= gms[i][4] != 0 ? 1u : 0u;
  cudaGraphSetConditional(loop, any);
}

namespace {

// Fused M2L needs every problem on the target-stationary kernel with one compressed rank.
bool batch_fuses_m2l(afmpb_t *const *hs, int k) {
  for (int i = 0; i < k; ++i)
    if (!m2l_ts_applies(hs[i]) || hs[i]->m2l_rank != hs[0]->m2l_rank || hs[i]->m2l_groups.empty() ||
        hs[i]->opt.m2l_method != 0)
      return false;
  return true;
}

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  ~BatchGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto e : events) cudaEventDestroy(e);
    for (auto s : streams) cudaStreamDestroy(s);
  }
  Err stream(cudaStream_t *s, int prio) {
    AFMPB_CUDA(cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, prio));
    streams.push_back(*s);
    return Err{};
  }
  Err event(cudaEvent_t *e) {
    AFMPB_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    events.push_back(*e);
    return Err{};
  }
};

Err build_batch_graph(afmpb_t *const *hs, int k, const int *ms, bool fuse_m2l, const BatchLists &L, BatchGraph &G) {
  cudaGraph_t g = nullptr;
  AFMPB_CUDA(cudaGraphCreate(&g, 0));
  struct GraphGuard { cudaGraph_t g; ~GraphGuard() { if (g) cudaGraphDestroy(g); } } gg{g};
  cudaGraphConditionalHandle loop;
  AFMPB_CUDA(cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  AFMPB_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  int lo = 0, hi = 0;
  AFMPB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  cudaStream_t cap = nullptr, sp = nullptr, sm = nullptr;
  AFMPB_TRY(G.stream(&cap, hi));
  AFMPB_TRY(G.stream(&sp, lo));            // P2P fills the SMs the far-field chains leave free
  AFMPB_TRY(G.stream(&sm, hi));
  std::vector<cudaStream_t> si(k);
  std::vector<cudaEvent_t> ev_a(k), ev_b(k), ev_e(k);
  cudaEvent_t ev_fork = nullptr, ev_p = nullptr, ev_m = nullptr;
  AFMPB_TRY(G.event(&ev_fork));
  AFMPB_TRY(G.event(&ev_p));
  AFMPB_TRY(G.event(&ev_m));
  for (int i = 0; i < k; ++i) {
    AFMPB_TRY(G.stream(&si[i], hi));
    AFMPB_TRY(G.event(&ev_a[i]));
    AFMPB_TRY(G.event(&ev_b[i]));
    AFMPB_TRY(G.event(&ev_e[i]));
  }
  AFMPB_CUDA(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  Err e;
  auto step = [&]() -> Err {
    AFMPB_CUDA(cudaEventRecord(ev_fork, cap));
    for (int i = 0; i < k; ++i) {
      afmpb_t *h = hs[i];
      const int *act = h->d_gm_int + 4;
      AFMPB_CUDA(cudaStreamWaitEvent(si[i], ev_fork, 0));
      AFMPB_TRY(enqueue_step_head(h, si[i], act));
      AFMPB_CUDA(cudaMemsetAsync(h->d_phi_near, 0, sizeof(float4) * h->n, si[i]));
      AFMPB_CUDA(cudaEventRecord(ev_a[i], si[i]));
      AFMPB_TRY(enqueue_far(h, si[i], nullptr, fuse_m2l ? kFarUp : kFarUp | kFarM2L));
      AFMPB_CUDA(cudaEventRecord(ev_b[i], si[i]));
    }
    for (int i = 0; i < k; ++i) AFMPB_CUDA(cudaStreamWaitEvent(sp, ev_a[i], 0));
    AFMPB_TRY(enqueue_p2p_batch(L.d_p2p, L.d_units, L.nunits, kP2PResident, sp));
    AFMPB_CUDA(cudaEventRecord(ev_p, sp));
    if (fuse_m2l) {
      for (int i = 0; i < k; ++i) AFMPB_CUDA(cudaStreamWaitEvent(sm, ev_b[i], 0));
      AFMPB_TRY(enqueue_m2l_ts_batch(L.d_ts, L.d_items, L.nitems, L.d_items_run, L.d_count, hs[0]->m2l_rank,
                                     hs[0]->d_tc_flag, sm));
      AFMPB_CUDA(cudaEventRecord(ev_m, sm));
    }
    for (int i = 0; i < k; ++i) {
      afmpb_t *h = hs[i];
      const int *act = h->d_gm_int + 4;
      if (fuse_m2l) AFMPB_CUDA(cudaStreamWaitEvent(si[i], ev_m, 0));
      AFMPB_TRY(enqueue_far(h, si[i], nullptr, kFarDown));
      AFMPB_CUDA(cudaStreamWaitEvent(si[i], ev_p, 0));
      AFMPB_TRY(enqueue_combine(h, si[i], AFMPB_PART_ALL));
      AFMPB_TRY(enqueue_step_tail(h, ms[i], si[i], act, true, loop));
      AFMPB_CUDA(cudaEventRecord(ev_e[i], si[i]));
      AFMPB_CUDA(cudaStreamWaitEvent(cap, ev_e[i], 0));
    }
    k_batch_go<<<1, 1, 0, cap>>>(k, L.d_gms, loop);
    return check_launch("k_batch_go");
  };
  e = step();
  cudaGraph_t out = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cap, &out);
  if (!e.ok()) return e;
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("cudaStreamEndCapture (batch): ") + cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&G.exec, g, 0);
  if (ce != cudaSuccess) return make_err(AFMPB_ECUDA, std::string("cudaGraphInstantiate (batch): ") + cudaGetErrorString(ce));
  return Err{};
}

}  // namespace

Err run_solve_batch(afmpb_t *const *hs, int k, afmpb_solve_info *infos, afmpb_status *statuses) {
  std::vector<int> ms(k);
  for (int i = 0; i < k; ++i) {
    AFMPB_TRY(restart_length(hs[i], &ms[i]));
    AFMPB_TRY(prepare_gmres(hs[i], ms[i]));
    AFMPB_CUDA(cudaStreamSynchronize(hs[i]->stream));
  }
  const bool fuse_m2l = batch_fuses_m2l(hs, k);
  BatchGraph G;
  cudaStream_t bs = nullptr;
  {
    int lo = 0, hi = 0;
    AFMPB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    AFMPB_TRY(G.stream(&bs, hi));
  }
  BatchLists L;
  L.stream = bs;
  AFMPB_TRY(build_batch_lists(hs, k, fuse_m2l, L));
  AFMPB_TRY(build_batch_graph(hs, k, ms.data(), fuse_m2l, L, G));

  struct State {
    double bnorm = 0, tol = 0, res = 0;
    int restarts = 0, products = 0, cycles = 0;
    bool running = true, converged = false;
    int gm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  };
  std::vector<State> st(k);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  AFMPB_CUDA(cudaEventCreate(&t0));
  AFMPB_CUDA(cudaEventCreate(&t1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{t0, t1};
  AFMPB_CUDA(cudaEventRecord(t0, bs));
  AFMPB_CUDA(cudaStreamSynchronize(bs));
  auto read_scalar = [&](afmpb_t *h, const double *d, int slot) -> Err {
    AFMPB_CUDA(cudaMemcpyAsync((double *)h->h_pinned + slot, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    AFMPB_CUDA(cudaStreamSynchronize(h->stream));
    return Err{};
  };
  for (int i = 0; i < k; ++i) {
    afmpb_t *h = hs[i];
    const int64_t n2 = 2 * h->n;
    AFMPB_TRY(norm2(h, n2, h->d_b, h->d_scal + 0));
    AFMPB_TRY(read_scalar(h, h->d_scal + 0, 0));
    st[i].bnorm = h->h_pinned[0];
    h->bnorm = st[i].bnorm;
    st[i].tol = h->tol * st[i].bnorm + h->opt.abs_tol;
    st[i].res = st[i].bnorm;
    h->h_pinned[4] = st[i].tol;
    AFMPB_CUDA(cudaMemcpyAsync(h->d_scal + 4, (const double *)h->h_pinned + 4, sizeof(double), cudaMemcpyHostToDevice,
                               h->stream));
    AFMPB_CUDA(cudaMemsetAsync(h->d_gm_int, 0, 8 * sizeof(int), h->stream));
    AFMPB_CUDA(cudaMemsetAsync(h->d_sol, 0, sizeof(double) * n2, h->stream));
  }
  for (;;) {
    // each running problem: residual of its current x, and the start of its next cycle
    int nrun = 0;
    for (int i = 0; i < k; ++i) {
      afmpb_t *h = hs[i];
      State &S = st[i];
      const int64_t n = h->n, n2 = 2 * n;
      if (S.running && S.cycles > h->opt.max_restart) S.running = false;
      if (S.running) {
        if (S.cycles == 0) {
          AFMPB_CUDA(cudaMemcpyAsync(h->d_w, h->d_b, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
        } else {
          ++S.restarts;
          ++S.products;
          AFMPB_TRY(product_from64(h, h->stream, h->d_sol));
          k_from_ys<<<div_up(n2, 256), 256, 0, h->stream>>>(n2, h->d_ys, h->d_b, h->d_w, nullptr);
          AFMPB_TRY(check_launch("residual"));
        }
        AFMPB_TRY(norm2(h, n2, h->d_w, h->d_scal + 1));
        AFMPB_TRY(read_scalar(h, h->d_scal + 1, 1));
        S.res = h->h_pinned[1];
        if (!(S.res > S.tol)) {
          S.converged = !std::isnan(S.res);
          S.running = false;
        }
      }
      if (S.running) {
        k_normalize<<<div_up(n, 256), 256, 0, h->stream>>>(n, h->d_w, h->d_scal + 1, h->d_V, nullptr);
        k_set_beta<<<1, 1, 0, h->stream>>>(h->d_g, ms[i], h->d_scal + 1);
        ++nrun;
      }
      k_cycle_start_b<<<1, 1, 0, h->stream>>>(h->d_gm_int, S.running ? 1 : 0);
      AFMPB_TRY(check_launch("batch cycle start"));
      if (S.running) AFMPB_TRY(enqueue_cycle_xs(h, h->stream, nullptr));
      AFMPB_CUDA(cudaStreamSynchronize(h->stream));
    }
    if (nrun == 0) break;
    // the Arnoldi steps of every running problem: one graph launch
    AFMPB_CUDA(cudaGraphLaunch(G.exec, bs));
    AFMPB_CUDA(cudaStreamSynchronize(bs));
    for (int i = 0; i < k; ++i) {
      afmpb_t *h = hs[i];
      State &S = st[i];
      if (!S.running) continue;
      const int64_t n2 = 2 * h->n;
      k_backsolve_j<<<1, 1, 0, h->stream>>>(h->d_gm_int, ms[i], h->d_H, h->d_g);
      k_update_x<<<std::min(div_up(n2, 256), 4 * 1184), 256, 0, h->stream>>>(n2, h->d_gm_int, h->d_V, n2, h->d_g,
                                                                              h->d_sol);
      AFMPB_TRY(check_launch("batch gmres update"));
      AFMPB_CUDA(cudaMemcpyAsync(S.gm, h->d_gm_int, sizeof(S.gm), cudaMemcpyDeviceToHost, h->stream));
      AFMPB_TRY(read_scalar(h, h->d_scal + 2, 2));
      S.res = h->h_pinned[2];
      S.products += S.gm[0];
      ++S.cycles;
      if (!(S.res > S.tol)) {
        S.converged = !std::isnan(S.res);
        S.running = false;
      }
    }
  }
  AFMPB_CUDA(cudaEventRecord(t1, bs));
  AFMPB_CUDA(cudaEventSynchronize(t1));
  float ms_all = 0.f;
  AFMPB_CUDA(cudaEventElapsedTime(&ms_all, t0, t1));
  Err first_fail;
  for (int i = 0; i < k; ++i) {
    afmpb_t *h = hs[i];
    State &S = st[i];
    const int64_t n2 = 2 * h->n;
    // true residual with one more product (its CUDA-event time stands for every product)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    AFMPB_CUDA(cudaEventCreate(&e0));
    AFMPB_CUDA(cudaEventCreate(&e1));
    EvGuard g2{e0, e1};
    AFMPB_CUDA(cudaEventRecord(e0, h->stream));
    AFMPB_TRY(product_from64(h, h->stream, h->d_sol));
    AFMPB_CUDA(cudaEventRecord(e1, h->stream));
    ++S.products;
    k_from_ys<<<div_up(n2, 256), 256, 0, h->stream>>>(n2, h->d_ys, h->d_b, h->d_w, nullptr);
    AFMPB_TRY(norm2(h, n2, h->d_w, h->d_scal + 3));
    AFMPB_TRY(read_scalar(h, h->d_scal + 3, 3));
    float ms_one = 0.f;
    AFMPB_CUDA(cudaEventElapsedTime(&ms_one, e0, e1));
    h->solved = true;
    int flag = 0;
    AFMPB_TRY(read_tc_error(h, &flag));
    if (infos) {
      afmpb_solve_info &I = infos[i];
      I.iters = S.gm[1];
      I.restarts = S.restarts;
      I.res_est = S.res;
      I.res_true = S.bnorm > 0 ? h->h_pinned[3] / S.bnorm : h->h_pinned[3];
      I.bnorm = S.bnorm;
      I.ms_setup = h->ms_setup;
      I.ms_matvec_total = ms_one * S.products;
      I.ms_gmres = ms_all;
      I.nnz_near = h->nnz;
      I.n_boxes = h->shape.nbox;
      I.krylov_dim = ms[i];
      I.second_passes = h->opt.orth == 0 ? S.gm[1] : S.gm[3];
    }
    if (statuses) statuses[i] = flag ? AFMPB_ETIMEOUT : S.converged ? AFMPB_OK : AFMPB_ENOCONV;
    if (first_fail.ok() && flag)
      first_fail = make_err(AFMPB_ETIMEOUT, "a bounded device wait expired during the batched solve; its products are not valid");
    if (first_fail.ok() && !S.converged)
      first_fail = make_err(AFMPB_ENOCONV, "GMRES did not reach the tolerance within max_restart cycles for a problem of the batch");
  }
  return first_fail;
}

Err run_energy(afmpb_t *h, double *E) {
  if (!h->solved || !h->d_sol) return make_err(AFMPB_ESTATE, "afmpb_energy needs a prior afmpb_solve");
  if (h->natoms == 0) return make_err(AFMPB_ESTATE, "the handle has no charges");
  const int nleaf = h->shape.nleaf;
  const int nparts = h->cf ? 1 : std::min(nleaf, 64);
  const int lpb = div_up(nleaf, nparts);
  const int nparts_used = h->cf ? 1 : div_up(nleaf, lpb);
  double *d_part = nullptr, *d_phi = nullptr, *d_E = nullptr;
  auto &A = h->arena;
  AFMPB_TRY(A.alloc(&d_part, (size_t)nparts_used * h->natoms, "energy partials"));
  AFMPB_TRY(A.alloc(&d_phi, h->natoms, "phi reac"));
  AFMPB_TRY(A.alloc(&d_E, 1, "energy"));
  if (h->cf) {
    AFMPB_TRY(charge_fmm_phi(h, d_part));
  } else {
    dim3 grid(div_up(h->natoms, 128), nparts_used);
    k_energy_part<<<grid, 128, 0, h->stream>>>(nleaf, lpb, h->d_leaves, h->d_box_begin, h->d_box_end,
                                                h->d_box_center, h->d_pos, h->d_nrm, h->d_sol, h->n, h->ebar,
                                                h->natoms, h->d_atoms, d_part);
    AFMPB_TRY(check_launch("k_energy_part"));
  }
  const double K_c = 332.0636;   // kcal A / (mol e^2)
  k_energy_final<<<1, 256, 0, h->stream>>>(nparts_used, h->natoms, d_part, h->d_q, 4.0 * kPi * K_c, d_phi, d_E);
  AFMPB_TRY(check_launch("k_energy_final"));
  AFMPB_CUDA(cudaMemcpyAsync(E, d_E, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  AFMPB_CUDA(cudaStreamSynchronize(h->stream));
  A.release(d_part);
  A.release(d_phi);
  A.release(d_E);
  return Err{};
}

// ---- allocation-free energy ---------------------------------------------------------------
// The partial sums, reaction potentials and the energy of afmpb_energy_noalloc live in
// this static device array instead of buffers allocated per call.  In host code the
// symbol is only a stand-in: its device address is looked up once per device with
// cudaGetSymbolAddress and cached.
constexpr int kNoAllocParts = 16;
constexpr int kNoAllocMaxAtoms = AFMPB_NOALLOC_MAX_ATOMS;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocParts * kNoAllocMaxAtoms + kNoAllocMaxAtoms + 1];

namespace {
constexpr int kMaxDevices = 64;
double *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;
}  // namespace

Err run_energy_noalloc(afmpb_t *h, double *E) {
  if (!h->solved || !h->d_sol) return make_err(AFMPB_ESTATE, "afmpb_energy_noalloc needs a prior afmpb_solve");
  if (h->natoms == 0) return make_err(AFMPB_ESTATE, "the handle has no charges");
  if (h->natoms > kNoAllocMaxAtoms)
    return make_err(AFMPB_EINVAL, "afmpb_energy_noalloc handles at most AFMPB_NOALLOC_MAX_ATOMS (" +
                                      std::to_string(kNoAllocMaxAtoms) + ") charges; the handle has " +
                                      std::to_string(h->natoms));
  int dev = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return make_err(AFMPB_EINVAL, "device ordinal out of range");
  // the scratch address is per device: the handle's kernels must run where it is looked up
  if (dev != h->device)
    return make_err(AFMPB_EINVAL, "the current device (" + std::to_string(dev) + ") is not the handle's device (" +
                                      std::to_string(h->device) + "); make it current first");
  // One scratch array per device: calls on different handles of the same device take
  // turns (the lock is held until the result has been copied back).
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    AFMPB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  double *base = g_noalloc_ptr[dev];
  double *d_part = base;                                    // [parts][natoms], fully rewritten
  double *d_phi = base + (size_t)kNoAllocParts * kNoAllocMaxAtoms;
  double *d_E = d_phi + kNoAllocMaxAtoms;
  const int nleaf = h->shape.nleaf;
  const int nparts = h->cf ? 1 : std::min(nleaf, kNoAllocParts);
  const int lpb = div_up(nleaf, nparts);
  const int nparts_used = h->cf ? 1 : div_up(nleaf, lpb);
  if (h->cf) {
    AFMPB_TRY(charge_fmm_phi(h, d_part));          // the charge FMM's buffers exist already
  } else {
    dim3 grid(div_up(h->natoms, 128), nparts_used);
    k_energy_part<<<grid, 128, 0, h->stream>>>(nleaf, lpb, h->d_leaves, h->d_box_begin, h->d_box_end,
                                                h->d_box_center, h->d_pos, h->d_nrm, h->d_sol, h->n, h->ebar,
                                                h->natoms, h->d_atoms, d_part);
    AFMPB_TRY(check_launch("k_energy_part (no alloc)"));
  }
  const double K_c = 332.0636;   // kcal A / (mol e^2)
  k_energy_final<<<1, 256, 0, h->stream>>>(nparts_used, h->natoms, d_part, h->d_q, 4.0 * kPi * K_c, d_phi, d_E);
  AFMPB_TRY(check_launch("k_energy_final (no alloc)"));
  AFMPB_CUDA(cudaMemcpyAsync(E, d_E, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  AFMPB_CUDA(cudaStreamSynchronize(h->stream));
  return Err{};
}

}  // namespace afmpb
