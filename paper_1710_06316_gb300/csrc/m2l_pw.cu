// m2l_pw.cu -- plane-wave (exponential) M2L: the alternative to the dense translations.
//
// The list-2 interaction of a target box T with a source box S of the same level (width
// w, centres at least two widths apart along some axis) goes through plane waves, the
// exponential expansions of FMM97 that the paper's FMM (DASHMM) uses.  In box units, with
// the separation axis a turned to +z' (direction d: the axis and its sign), every
// target-source pair has z' in [1, 4] and transverse distance rho <= 4 sqrt(2), and
//
//   exp(-k r) / r ~= sum_j w_j exp(-(k + t_j) z') (2 / M_j) Re sum_{l < M_j/2}
//                     exp(i s_j (x' cos a_l + y' sin a_l)),   s_j = sqrt(t_j^2 + 2 k t_j),
//
// with k = kappa w (0 for the Laplace kernel) and the quadrature of pw_quadrature.h (an
// absolute error below 1e-6 of 1/r).  The expansions here are the Chebyshev ones of the
// rest of the FMM (equivalent densities M at the n^3 points of the source box, potentials
// L at those of the target box), so the three steps are
//   M2X  X_d(S)[p]  = sum_m M_S[m] exp(u_j (s c_{m,a} - 1/2)) exp(-i s_j (c_{m,b} cos a_l + c_{m,c} sin a_l))
//   X2X  Y_d(T)[p]  = sum_{S in list 2 of T, direction d} X_d(S)[p] exp(-u_j (|D_a| - 1)) exp(i s_j (D_b cos a_l + D_c sin a_l))
//   X2L  L_T[i]    += scale Re sum_p (2 w_j / M_j) Y_d(T)[p] exp(-u_j (s c_{i,a} + 1/2)) exp(i s_j (c_{i,b} cos a_l + c_{i,c} sin a_l))
// for plane wave p = (j, l), u_j = k + t_j, D = c_T - c_S in box units, c the Chebyshev
// points scaled to [-1/2, 1/2], (b, c) the transverse axes, and scale = 1 / (4 pi w) (the
// kernel 1/(4 pi r) of the dense tables in real units).  Every factor is at most 1.  The
// six directions share one base frame: the Chebyshev grid maps onto itself under axis
// permutations and sign flips, so direction d reads M and writes L through an index map.
// M2X and X2L are applied one tensor axis at a time (the z' exponential, then the two
// transverse phases), O(P n^2 + K n^3) per box and direction for P plane waves and K
// t-nodes, instead of O(P n^3).
#include <cmath>

#include "internal.cuh"
#include "pw_quadrature.h"

namespace afmpb {

namespace {

constexpr int kPwThreads = 256;
constexpr int kPwMaxNodes = 48;      // t-nodes of one band (the generated quadratures have <= 40)

struct PwSetDev {
  int K, P;        // t-nodes, plane waves kept
  int k0, p0;      // offsets into the node and plane-wave arrays
  int64_t sh0;     // offset into the translation table (kNumOffsets x P complex)
  float scale;     // 1 / (4 pi w)
};

// One base-frame pass of M2X for box b, kernel kt, all six directions.
template <int N>
__global__ void __launch_bounds__(kPwThreads) k_pw_m2x(int ls, int set0, int set1, const PwSetDev *__restrict__ sets,
                                                       const float *__restrict__ ex_src, const int *__restrict__ pnode,
                                                       const float2 *__restrict__ phx, const float2 *__restrict__ phy,
                                                       const int *__restrict__ perm, int pmax,
                                                       const float *__restrict__ M, float2 *__restrict__ X) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int kt = blockIdx.y;
  const int q = kt == 0 ? set0 : set1;
  if (q < 0) return;
  const PwSetDev S = sets[q];
  const int b = ls + (int)blockIdx.x;
  __shared__ float Ms[N3];
  __shared__ float St[kPwMaxNodes * N2];
  for (int m = threadIdx.x; m < N3; m += blockDim.x) Ms[m] = M[((size_t)b * 2 + kt) * N3 + m];
  for (int d = 0; d < 6; ++d) {
    __syncthreads();
    // St[j][i1][i2] = sum_i3 exp(u_j (c_i3 - 1/2)) M[perm_d(i1, i2, i3)]
    for (int e = threadIdx.x; e < S.K * N2; e += blockDim.x) {
      const int j = e / N2, i12 = e % N2;
      const float *ex = ex_src + (size_t)(S.k0 + j) * N;
      const int *pm = perm + d * N3 + i12 * N;
      float acc = 0.0f;
#pragma unroll
      for (int i3 = 0; i3 < N; ++i3) acc = fmaf(ex[i3], Ms[pm[i3]], acc);
      St[e] = acc;
    }
    __syncthreads();
    float2 *Xd = X + (((size_t)b * 2 + kt) * 6 + d) * pmax;
    for (int p = threadIdx.x; p < S.P; p += blockDim.x) {
      const int j = pnode[S.p0 + p];
      const float2 *ax = phx + (size_t)(S.p0 + p) * N, *ay = phy + (size_t)(S.p0 + p) * N;
      const float *st = St + j * N2;
      float cr = 0.0f, ci = 0.0f;
#pragma unroll
      for (int i2 = 0; i2 < N; ++i2) {
        float ir = 0.0f, ii = 0.0f;
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1) {
          const float v = st[i1 * N + i2];
          ir = fmaf(ax[i1].x, v, ir);
          ii = fmaf(ax[i1].y, v, ii);
        }
        const float2 y = ay[i2];
        cr = fmaf(y.x, ir, fmaf(-y.y, ii, cr));
        ci = fmaf(y.x, ii, fmaf(y.y, ir, ci));
      }
      Xd[p] = make_float2(cr, ci);
    }
  }
}

// X2X + X2L for one target box and kernel: for each direction the translated sum of its
// list-2 sources' plane waves, then the potentials at the target's Chebyshev points.
template <int N>
__global__ void __launch_bounds__(kPwThreads) k_pw_x2l(int t0, int set0, int set1, const int *__restrict__ tbox,
                                                       const int *__restrict__ dptr, const int *__restrict__ esrc,
                                                       const int *__restrict__ eslot, const PwSetDev *__restrict__ sets,
                                                       const float *__restrict__ ex_tgt,
                                                       const int *__restrict__ pb, const float *__restrict__ om,
                                                       const float2 *__restrict__ phx, const float2 *__restrict__ phy,
                                                       const float2 *__restrict__ shift, const int *__restrict__ perm,
                                                       int pmax, const float2 *__restrict__ X, float *__restrict__ L) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int kt = blockIdx.y;
  const int q = kt == 0 ? set0 : set1;
  if (q < 0) return;
  const PwSetDev S = sets[q];
  const int ti = t0 + (int)blockIdx.x;
  const int T = tbox[ti];
  extern __shared__ float2 Y[];                      // [pmax]
  __shared__ float G[kPwMaxNodes * N2];
  __shared__ float Ls[N3];
  for (int m = threadIdx.x; m < N3; m += blockDim.x) Ls[m] = 0.0f;
  for (int d = 0; d < 6; ++d) {
    const int e0 = dptr[ti * 7 + d], e1 = dptr[ti * 7 + d + 1];
    if (e0 == e1) continue;                          // uniform
    __syncthreads();
    for (int p = threadIdx.x; p < S.P; p += blockDim.x) {
      float yr = 0.0f, yi = 0.0f;
      for (int e = e0; e < e1; ++e) {
        const float2 x = X[(((size_t)esrc[e] * 2 + kt) * 6 + d) * pmax + p];
        const float2 sh = shift[S.sh0 + (int64_t)eslot[e] * S.P + p];
        yr = fmaf(sh.x, x.x, fmaf(-sh.y, x.y, yr));
        yi = fmaf(sh.x, x.y, fmaf(sh.y, x.x, yi));
      }
      const float w = om[S.p0 + p];
      Y[p] = make_float2(w * yr, w * yi);
    }
    __syncthreads();
    // G[j][i1][i2] = Re sum_{p of node j} Y[p] exp(i s (c_i1 cos a + c_i2 sin a))
    for (int e = threadIdx.x; e < S.K * N2; e += blockDim.x) {
      const int j = e / N2, i1 = (e / N) % N, i2 = e % N;
      const int pa = pb[S.k0 + j] - S.p0, p1 = pb[S.k0 + j + 1] - S.p0;   // node j's waves in the set
      float acc = 0.0f;
      for (int p = pa; p < p1; ++p) {
        const float2 a = phx[(size_t)(S.p0 + p) * N + i1], c = phy[(size_t)(S.p0 + p) * N + i2];
        // conj(a) conj(c) = conj(a c); Re(Y conj(a c)) = Y.x (a c).x + Y.y (a c).y
        const float ar = a.x * c.x - a.y * c.y, ai = a.x * c.y + a.y * c.x;
        acc = fmaf(Y[p].x, ar, fmaf(Y[p].y, ai, acc));
      }
      G[e] = acc;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < N3; m += blockDim.x) {
      const int i12 = m / N, i3 = m % N;
      float acc = 0.0f;
      for (int j = 0; j < S.K; ++j) acc = fmaf(ex_tgt[(size_t)(S.k0 + j) * N + i3], G[j * N2 + i12], acc);
      Ls[perm[d * N3 + m]] += acc;                   // a permutation: no two threads share a slot
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < N3; m += blockDim.x) L[((size_t)T * 2 + kt) * N3 + m] += S.scale * Ls[m];
}

}  // namespace

// Tables of every (level, kernel) that has list-2 work, the target lists by direction, and
// the plane-wave buffer.
Err build_m2l_pw(afmpb_t *h) {
  const int N = h->order, N3 = N * N * N;
  auto &A = h->arena;
  cudaStream_t s = h->stream;
  const auto &T = h->shape;
  if (h->m2l_groups.empty()) return Err{};
  std::vector<double> c(N);
  for (int m = 0; m < N; ++m) c[m] = 0.5 * std::cos((2.0 * m + 1.0) * M_PI / (2.0 * N));
  // offsets of the table slots (source - target, in box widths), as the dense tables order them
  std::vector<int3> offs;
  for (int ox = -3; ox <= 3; ++ox)
    for (int oy = -3; oy <= 3; ++oy)
      for (int oz = -3; oz <= 3; ++oz) {
        if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
        offs.push_back(make_int3(ox, oy, oz));
      }
  // direction of a slot: axis of the separation (z, then y, then x) and its sign, with
  // D = target - source; the transverse axes (b, c) per axis a
  auto dir_of = [&](const int3 &o, int *axis, int *sgn, int *Da, int *Db, int *Dc) {
    const int D[3] = {-o.x, -o.y, -o.z};
    const int a = std::abs(D[2]) >= 2 ? 2 : std::abs(D[1]) >= 2 ? 1 : 0;
    const int b = a == 2 ? 0 : a == 1 ? 2 : 1, cc = a == 2 ? 1 : a == 1 ? 0 : 2;
    *axis = a;
    *sgn = D[a] > 0 ? 1 : -1;
    *Da = std::abs(D[a]);
    *Db = D[b];
    *Dc = D[cc];
    return 2 * a + (D[a] > 0 ? 0 : 1);
  };
  // index maps: base point (i1, i2, i3) of direction d -> original point
  std::vector<int> perm(6 * N3);
  for (int d = 0; d < 6; ++d) {
    const int a = d / 2, sg = (d % 2) ? -1 : 1;
    const int b = a == 2 ? 0 : a == 1 ? 2 : 1, cc = a == 2 ? 1 : a == 1 ? 0 : 2;
    for (int i1 = 0; i1 < N; ++i1)
      for (int i2 = 0; i2 < N; ++i2)
        for (int i3 = 0; i3 < N; ++i3) {
          int idx[3];
          idx[b] = i1;
          idx[cc] = i2;
          idx[a] = sg > 0 ? i3 : N - 1 - i3;
          perm[d * N3 + (i1 * N + i2) * N + i3] = (idx[0] * N + idx[1]) * N + idx[2];
        }
  }
  int maxlev = 0;
  for (const auto &g : h->m2l_groups) maxlev = std::max(maxlev, g.level + 1);
  std::vector<int> set_of(2 * maxlev, -1);
  std::vector<PwSetDev> sets;
  std::vector<int> pnode, pbv;
  std::vector<float> ex_src, ex_tgt, om;
  std::vector<float2> phx, phy, shift;
  int kcount = 0, pcount = 0, pmax = 0;
  int64_t shcount = 0;
  std::vector<char> has_level(maxlev, 0);
  for (const auto &g : h->m2l_groups) has_level[g.level] = 1;
  for (int l = 0; l < maxlev; ++l) {
    if (!has_level[l]) continue;
    const double whalf = std::ldexp(T.w0, -l), width = 2.0 * whalf;
    for (int kt = 0; kt < 2; ++kt) {
      if (kt == 1 && (l < h->m2l_yuk_levels || h->laplace_only)) continue;
      const double kp = kt == 0 ? 0.0 : h->kappa * width;
      int band = 0;
      if (kt == 1) {
        band = -1;
        for (int bb = 1; bb < kPwBands; ++bb)
          if (kp <= kPwBandHi[bb] && band < 0) band = bb;
        if (band < 0) continue;                      // screened: exp(-k z) <= exp(-16) of 1/r
      }
      PwSetDev S{};
      S.k0 = kcount;
      S.p0 = pcount;
      S.sh0 = shcount;
      S.scale = (float)(kInv4Pi / width);
      S.K = kPwOff[band + 1] - kPwOff[band];
      std::vector<double> ax, ay;
      for (int j = 0; j < S.K; ++j) {
        const double t = kPwT[kPwOff[band] + j], wq = kPwW[kPwOff[band] + j];
        const int Mj = kPwM[kPwOff[band] + j];
        const double u = kp + t, sj = std::sqrt(t * t + 2.0 * kp * t);
        pbv.push_back(pcount + (int)ax.size());        // first wave of node j (absolute)
        for (int n = 0; n < N; ++n) {
          ex_src.push_back((float)std::exp(u * (c[n] - 0.5)));
          ex_tgt.push_back((float)std::exp(-u * (c[n] + 0.5)));
        }
        for (int l2 = 0; l2 < Mj / 2; ++l2) {
          const double al = 2.0 * M_PI * (l2 + 0.5) / Mj;
          ax.push_back(sj * std::cos(al));
          ay.push_back(sj * std::sin(al));
          pnode.push_back(j);
          om.push_back((float)(2.0 * wq / Mj));
          for (int n = 0; n < N; ++n) {
            phx.push_back(make_float2((float)std::cos(ax.back() * c[n]), (float)-std::sin(ax.back() * c[n])));
            phy.push_back(make_float2((float)std::cos(ay.back() * c[n]), (float)-std::sin(ay.back() * c[n])));
          }
        }
      }
      S.P = (int)ax.size();
      if (S.K > kPwMaxNodes) return make_err(AFMPB_EINTERNAL, "plane-wave quadrature larger than the kernel's node buffer");
      // translation table: per slot the diagonal shift of its direction's waves
      for (size_t o = 0; o < offs.size(); ++o) {
        int axis, sg, Da, Db, Dc;
        dir_of(offs[o], &axis, &sg, &Da, &Db, &Dc);
        size_t p = 0;
        for (int j = 0; j < S.K; ++j) {
          const double t = kPwT[kPwOff[band] + j];
          const double u = kp + t;
          const int Mj = kPwM[kPwOff[band] + j];
          const double dec = std::exp(-u * (Da - 1));
          for (int l2 = 0; l2 < Mj / 2; ++l2, ++p) {
            const double ph = ax[p] * Db + ay[p] * Dc;
            shift.push_back(make_float2((float)(dec * std::cos(ph)), (float)(dec * std::sin(ph))));
          }
        }
      }
      kcount += S.K;
      pcount += S.P;
      shcount += (int64_t)offs.size() * S.P;
      pmax = std::max(pmax, S.P);
      set_of[2 * l + kt] = (int)sets.size();
      sets.push_back(S);
    }
  }
  pbv.push_back(pcount);          // pb[k0 + j] .. pb[k0 + j + 1]: the waves of node j (absolute)
  // list 2 by target: (source, slot) entries grouped by direction
  const size_t np = (size_t)h->n_m2l_pairs;
  std::vector<int2> pairs(np);
  if (np) AFMPB_CUDA(cudaMemcpyAsync(pairs.data(), h->d_m2l_pairs, sizeof(int2) * np, cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  std::vector<int> dir_slot(offs.size());
  for (size_t o = 0; o < offs.size(); ++o) {
    int axis, sg, Da, Db, Dc;
    dir_slot[o] = dir_of(offs[o], &axis, &sg, &Da, &Db, &Dc);
  }
  struct Ent { int tgt, dir, src, slot; };
  std::vector<Ent> ents;
  ents.reserve(np);
  for (const auto &g : h->m2l_groups)
    for (int i = 0; i < g.count; ++i) {
      const int2 pr = pairs[g.start + i];
      ents.push_back({pr.x, dir_slot[g.offset], pr.y, g.offset});
    }
  std::sort(ents.begin(), ents.end(), [](const Ent &a, const Ent &b) {
    return a.tgt != b.tgt ? a.tgt < b.tgt : a.dir != b.dir ? a.dir < b.dir : a.src < b.src;
  });
  std::vector<int> tbox, dptr, esrc(ents.size()), eslot(ents.size());
  h->pw_level_t0.assign(maxlev + 1, 0);
  for (size_t e = 0; e < ents.size();) {
    size_t f = e;
    while (f < ents.size() && ents[f].tgt == ents[e].tgt) ++f;
    tbox.push_back(ents[e].tgt);
    size_t g = e;
    for (int d = 0; d < 6; ++d) {
      dptr.push_back((int)g);
      while (g < f && ents[g].dir == d) ++g;
    }
    dptr.push_back((int)f);
    for (size_t k = e; k < f; ++k) {
      esrc[k] = ents[k].src;
      eslot[k] = ents[k].slot;
    }
    e = f;
  }
  // targets are in box order, so each level's targets are one range [t0[l], t0[l + 1])
  for (int l = 0; l <= maxlev; ++l)
    h->pw_level_t0[l] = (int)(std::lower_bound(tbox.begin(), tbox.end(), T.lvl_start[l]) - tbox.begin());
  h->pw_set_of = set_of;
  h->pw_pmax = pmax;
  h->pw_maxlev = maxlev;
  h->pw_ntargets = (int)tbox.size();
  auto up = [&](auto **d, const auto &v, const char *what) -> Err {
    AFMPB_TRY(A.alloc(d, std::max<size_t>(1, v.size()), what));
    if (!v.empty()) AFMPB_CUDA(cudaMemcpyAsync(*d, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice, s));
    return Err{};
  };
  PwSetDev *d_sets = nullptr;
  AFMPB_TRY(up(&d_sets, sets, "pw sets"));
  h->d_pw_sets = d_sets;
  AFMPB_TRY(up(&h->d_pw_pnode, pnode, "pw wave nodes"));
  AFMPB_TRY(up(&h->d_pw_pb, pbv, "pw node ranges"));
  AFMPB_TRY(up(&h->d_pw_exs, ex_src, "pw source decays"));
  AFMPB_TRY(up(&h->d_pw_ext, ex_tgt, "pw target decays"));
  AFMPB_TRY(up(&h->d_pw_om, om, "pw weights"));
  AFMPB_TRY(up(&h->d_pw_phx, phx, "pw x phases"));
  AFMPB_TRY(up(&h->d_pw_phy, phy, "pw y phases"));
  AFMPB_TRY(up(&h->d_pw_shift, shift, "pw translations"));
  AFMPB_TRY(up(&h->d_pw_perm, perm, "pw index maps"));
  AFMPB_TRY(up(&h->d_pw_tbox, tbox, "pw targets"));
  AFMPB_TRY(up(&h->d_pw_dptr, dptr, "pw direction ranges"));
  AFMPB_TRY(up(&h->d_pw_esrc, esrc, "pw sources"));
  AFMPB_TRY(up(&h->d_pw_eslot, eslot, "pw slots"));
  AFMPB_TRY(A.alloc(&h->d_pw_X, (size_t)T.nbox * 2 * 6 * std::max(1, pmax), "pw plane waves"));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  const size_t smem = sizeof(float2) * (size_t)pmax;
  switch (N) {
#define AFMPB_PW_SMEM(n) case n: AFMPB_TRY(raise_smem_limit((const void *)k_pw_x2l<n>, (int)smem)); break;
    AFMPB_PW_SMEM(2) AFMPB_PW_SMEM(3) AFMPB_PW_SMEM(4) AFMPB_PW_SMEM(5) AFMPB_PW_SMEM(6) AFMPB_PW_SMEM(7)
    AFMPB_PW_SMEM(8)
#undef AFMPB_PW_SMEM
    default: return make_err(AFMPB_EINVAL, "fmm_order must be in [2, 8]");
  }
  return Err{};
}

namespace {
template <int N>
Err launch_pw(afmpb_t *h, cudaStream_t s) {
  const auto &T = h->shape;
  const auto *sets = reinterpret_cast<const PwSetDev *>(h->d_pw_sets);
  for (int l = 0; l < h->pw_maxlev; ++l) {
    const int s0 = h->pw_set_of[2 * l], s1 = h->pw_set_of[2 * l + 1];
    if (s0 < 0 && s1 < 0) continue;
    const int ls = T.lvl_start[l], nl = T.lvl_start[l + 1] - ls;
    k_pw_m2x<N><<<dim3((unsigned)nl, 2), kPwThreads, 0, s>>>(ls, s0, s1, sets, h->d_pw_exs, h->d_pw_pnode, h->d_pw_phx,
                                                             h->d_pw_phy, h->d_pw_perm, h->pw_pmax, h->d_M, h->d_pw_X);
    AFMPB_TRY(check_launch("k_pw_m2x"));
  }
  for (int l = 0; l < h->pw_maxlev; ++l) {
    const int s0 = h->pw_set_of[2 * l], s1 = h->pw_set_of[2 * l + 1];
    const int t0 = h->pw_level_t0[l], t1 = h->pw_level_t0[l + 1];
    if ((s0 < 0 && s1 < 0) || t1 <= t0) continue;
    k_pw_x2l<N><<<dim3((unsigned)(t1 - t0), 2), kPwThreads, sizeof(float2) * h->pw_pmax, s>>>(
        t0, s0, s1, h->d_pw_tbox, h->d_pw_dptr, h->d_pw_esrc, h->d_pw_eslot, sets, h->d_pw_ext,
        h->d_pw_pb, h->d_pw_om, h->d_pw_phx, h->d_pw_phy, h->d_pw_shift, h->d_pw_perm, h->pw_pmax, h->d_pw_X, h->d_L);
    AFMPB_TRY(check_launch("k_pw_x2l"));
  }
  return Err{};
}
}  // namespace

Err enqueue_m2l_pw(afmpb_t *h, cudaStream_t s) {
  switch (h->order) {
    case 2: return launch_pw<2>(h, s);
    case 3: return launch_pw<3>(h, s);
    case 4: return launch_pw<4>(h, s);
    case 5: return launch_pw<5>(h, s);
    case 6: return launch_pw<6>(h, s);
    case 7: return launch_pw<7>(h, s);
    case 8: return launch_pw<8>(h, s);
    default: return make_err(AFMPB_EINVAL, "fmm_order must be in [2, 8]");
  }
}

}  // namespace afmpb
