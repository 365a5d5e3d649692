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

// w -= sum_i c_i V_i   (c on the device)
__global__ void k_sub_combo(int64_t len, int nv, const double *__restrict__ V, int64_t ldv,
                            const double *__restrict__ c, double sign, double *__restrict__ w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nv; ++i) s = fma(c[i], V[(int64_t)i * ldv + k], s);
    w[k] += sign * s;
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

// w = ys (FP32 -> FP64), optionally w = b - ys
__global__ void k_from_ys(int64_t len, const float *__restrict__ ys, const double *__restrict__ b,
                          double *__restrict__ w) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= len) return;
  w[k] = b ? b[k] - (double)ys[k] : (double)ys[k];
}

// Givens update of Hessenberg column j (hcol[0..j+1]); H column-major (m+1) x m.
__global__ void k_givens(int j, int m, const double *__restrict__ hcol, double *__restrict__ H,
                         double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                         double *__restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
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

// back substitution H(0:k,0:k) y = g(0:k), y written over g
__global__ void k_backsolve(int k, int m, const double *__restrict__ H, double *__restrict__ g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(int64_t)c * (m + 1) + i] * g[c];
    g[i] = s / H[(int64_t)i * (m + 1) + i];
  }
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

__global__ void k_add_small(int k, const double *__restrict__ a, double *__restrict__ b) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) b[i] += a[i];
}

Err run_solve(afmpb_t *h, afmpb_solve_info *info) {
  const int64_t n = h->n, n2 = 2 * n;
  const int m = h->opt.restart, max_restart = h->opt.max_restart;
  cudaStream_t s = h->stream;
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
    if (!h->h_pinned) AFMPB_CUDA(cudaMallocHost(&h->h_pinned, 8 * sizeof(double)));
  }
  if (!h->d_sol) AFMPB_TRY(A.alloc(&h->d_sol, n2, "solution"));
  double *x = h->d_sol;
  volatile double *hp = h->h_pinned;
  const int nb_el = div_up(n, 256), nb_el2 = div_up(n2, 256);
  const int nb_comb = std::min(nb_el2, 4 * 1184);
  double ms_mv = 0.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  AFMPB_CUDA(cudaEventCreate(&e0));
  AFMPB_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } guard{e0, e1};
  AFMPB_CUDA(cudaEventRecord(h->ev_t0, s));
  auto timed_product = [&](const double *v) -> Err {   // d_ys = L v (one graph launch)
    AFMPB_CUDA(cudaEventRecord(e0, s));
    AFMPB_TRY(product_from64(h, s, v));
    AFMPB_CUDA(cudaEventRecord(e1, s));
    return Err{};
  };
  auto read_scalar = [&](const double *d, int slot) -> Err {
    AFMPB_CUDA(cudaMemcpyAsync((double *)hp + slot, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
    return Err{};
  };
  auto add_mv_time = [&]() -> Err {
    float t = 0.f;
    AFMPB_CUDA(cudaEventElapsedTime(&t, e0, e1));
    ms_mv += t;
    return Err{};
  };

  AFMPB_TRY(norm2(h, n2, h->d_b, h->d_scal + 0));
  AFMPB_TRY(read_scalar(h->d_scal + 0, 0));
  const double bnorm = hp[0];
  h->bnorm = bnorm;
  const double tol = h->tol * bnorm + h->opt.abs_tol;
  AFMPB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n2, s));
  int iters = 0, restarts = 0;
  bool converged = false;
  double res = bnorm;
  for (int cycle = 0; cycle <= max_restart && !converged; ++cycle) {
    if (cycle == 0) {   // x0 = 0: r = b
      AFMPB_CUDA(cudaMemcpyAsync(h->d_w, h->d_b, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
    } else {
      ++restarts;
      AFMPB_TRY(timed_product(x));
      k_from_ys<<<nb_el2, 256, 0, s>>>(n2, h->d_ys, h->d_b, h->d_w);
      AFMPB_TRY(check_launch("residual"));
    }
    AFMPB_TRY(norm2(h, n2, h->d_w, h->d_scal + 1));
    AFMPB_TRY(read_scalar(h->d_scal + 1, 1));
    if (cycle > 0) AFMPB_TRY(add_mv_time());
    res = hp[1];
    if (!(res > tol)) {
      converged = !std::isnan(res);
      break;
    }
    k_normalize<<<nb_el, 256, 0, s>>>(n, h->d_w, h->d_scal + 1, h->d_V, nullptr);
    k_set_beta<<<1, 1, 0, s>>>(h->d_g, m, h->d_scal + 1);
    AFMPB_TRY(check_launch("gmres start"));
    int k = 0;
    for (int j = 0; j < m; ++j) {
      AFMPB_TRY(timed_product(h->d_V + (size_t)j * n2));
      k_from_ys<<<nb_el2, 256, 0, s>>>(n2, h->d_ys, nullptr, h->d_w);
      // classical Gram-Schmidt applied twice
      AFMPB_TRY(multidot(h, n2, j + 1, h->d_V, n2, h->d_w, h->d_hcol, 0));
      k_sub_combo<<<nb_comb, 256, 0, s>>>(n2, j + 1, h->d_V, n2, h->d_hcol, -1.0, h->d_w);
      AFMPB_TRY(multidot(h, n2, j + 1, h->d_V, n2, h->d_w, h->d_hcol2, 0));
      k_sub_combo<<<nb_comb, 256, 0, s>>>(n2, j + 1, h->d_V, n2, h->d_hcol2, -1.0, h->d_w);
      k_add_small<<<1, 128, 0, s>>>(j + 1, h->d_hcol2, h->d_hcol);
      AFMPB_TRY(norm2(h, n2, h->d_w, h->d_hcol + j + 1));
      k_normalize<<<nb_el, 256, 0, s>>>(n, h->d_w, h->d_hcol + j + 1, h->d_V + (size_t)(j + 1) * n2, nullptr);
      k_givens<<<1, 1, 0, s>>>(j, m, h->d_hcol, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_scal + 2);
      AFMPB_TRY(check_launch("arnoldi"));
      AFMPB_TRY(read_scalar(h->d_scal + 2, 2));
      AFMPB_TRY(add_mv_time());
      res = hp[2];
      ++iters;
      k = j + 1;
      if (!(res > tol)) {
        converged = !std::isnan(res);
        break;
      }
    }
    // x += V y, H y = g
    k_backsolve<<<1, 1, 0, s>>>(k, m, h->d_H, h->d_g);
    k_sub_combo<<<nb_comb, 256, 0, s>>>(n2, k, h->d_V, n2, h->d_g, 1.0, x);
    AFMPB_TRY(check_launch("gmres update"));
  }
  // true residual with one more product
  AFMPB_TRY(timed_product(x));
  k_from_ys<<<nb_el2, 256, 0, s>>>(n2, h->d_ys, h->d_b, h->d_w);
  AFMPB_TRY(norm2(h, n2, h->d_w, h->d_scal + 3));
  AFMPB_TRY(read_scalar(h->d_scal + 3, 3));
  AFMPB_TRY(add_mv_time());
  AFMPB_CUDA(cudaEventRecord(h->ev_t1, s));
  AFMPB_CUDA(cudaEventSynchronize(h->ev_t1));
  float ms_all = 0.f;
  AFMPB_CUDA(cudaEventElapsedTime(&ms_all, h->ev_t0, h->ev_t1));
  h->solved = true;
  if (h->opt.precision == 1) {
    int flag = 0;
    AFMPB_TRY(read_tc_error(h, &flag));
    if (flag) return make_err(AFMPB_ETIMEOUT, "a tensor-core M2L wait expired; the products are not valid");
  }
  if (info) {
    info->iters = iters;
    info->restarts = restarts;
    info->res_est = res;
    info->res_true = bnorm > 0 ? hp[3] / bnorm : hp[3];
    info->bnorm = bnorm;
    info->ms_setup = h->ms_setup;
    info->ms_matvec_total = ms_mv;
    info->ms_gmres = ms_all;
    info->nnz_near = h->nnz;
    info->n_boxes = h->shape.nbox;
  }
  if (!converged) return make_err(AFMPB_ENOCONV, "GMRES did not reach the tolerance within max_restart cycles");
  return Err{};
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
