// fmm.cu -- far-field sums of the node-patch operator: adaptive FMM + point-to-point.
//
// For x = [f; h] every source node t carries a charge c_t = a_t h_t and a dipole
// strength g_t = -a_t f_t along its normal n_t (Eq. 6 with the far rule: integrand
// constant on the patch).  With G = 1/(4 pi r), u = exp(-kappa r)/(4 pi r) and the
// dipole entering as d . grad_y, the four far sums of the solution flow (Sec. 2,
// step 3b: single- and double-layer Laplace and Yukawa) are
//     PhiL(p) = sum_t c_t G + (g_t / eps_bar) n_t . grad_y G
//     PhiY(p) = sum_t c_t u + g_t n_t . grad_y u
// and their target normal derivatives n_p . grad_x.  They are evaluated together in one
// tree pass (the "ViewSet" idea of Sec. 3.1): every box carries one Laplace and one
// Yukawa expansion.
//
// Expansions: tensor-product Chebyshev interpolation of the kernel on each box
// (n = order points per dimension, n^3 weights per box and kernel).  The same
// weights serve the single and the double layer (Sec. 3.2 notes the two share their
// expansion form): the dipole enters P2M through the gradient of the interpolating
// polynomial, and the normal derivative leaves L2P the same way.  M2L is a dense
// n^3 x n^3 kernel matrix per (level, offset); the paper's FMM97 plane-wave M2L is
// replaced by these dense translations, which are contractions suited to the GPU.
//
// Lists: 1 and 3 by P2P (Sec. 3.2 modified method), 2 by M2L, 4 by P2L (S_to_L).
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace afmpb {

// Per-order tables (index = order n), written once per device before the first handle
// uses them, so that handles of different orders can run side by side.
__constant__ float c_cheb[kMaxOrder + 1][kMaxOrder * kMaxOrder];     // Cm[m][k] = w_k T_k(x_m)
__constant__ float c_m2m[kMaxOrder + 1][2 * kMaxOrder * kMaxOrder];  // S2[c][m][m']
__constant__ float c_nodes[kMaxOrder + 1][kMaxOrder];                // Chebyshev points on [-1, 1]

// s_m(x) and s_m'(x) for the n interpolation polynomials.
template <int N>
__device__ __forceinline__ void cheb_basis(float x, float s[N], float ds[N]) {
  float T[N], dT[N];
  T[0] = 1.0f;
  dT[0] = 0.0f;
  if (N > 1) {
    T[1] = x;
    dT[1] = 1.0f;
  }
#pragma unroll
  for (int k = 2; k < N; ++k) {
    T[k] = 2.0f * x * T[k - 1] - T[k - 2];
    dT[k] = 2.0f * T[k - 1] + 2.0f * x * dT[k - 1] - dT[k - 2];
  }
#pragma unroll
  for (int m = 0; m < N; ++m) {
    float a = 0.0f, b = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      a = fmaf(c_cheb[N][m * kMaxOrder + k], T[k], a);
      b = fmaf(c_cheb[N][m * kMaxOrder + k], dT[k], b);
    }
    s[m] = a;
    ds[m] = b;
  }
}

// ------------------------------------------------------------------------------------
// P2M: leaf sources -> Laplace and Yukawa multipole weights.
// ------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_p2m(int nleaf, const int32_t *__restrict__ leaves,
                                            const int32_t *__restrict__ bbeg, const int32_t *__restrict__ bend,
                                            const dbl4 *__restrict__ center, const float4 *__restrict__ pos,
                                            const float4 *__restrict__ nrm, const float2 *__restrict__ xs,
                                            float inv_ebar, float *__restrict__ M) {
  // Four leaves per CTA, a group of 64 threads each (synchronised by its own named
  // barrier); thread (j, k) of a group holds the N weights (i, j, k) of both sums, so a
  // node's y-z factors are formed once and applied along the whole x axis:
  //   A[ijk] += c Sx[i] (Sy[j] Sz[k]),  B[ijk] += dSx[i] (g_x Sy Sz) + Sx[i] (g_y dSy Sz + g_z Sy dSz)
  // (one leaf per 64-thread CTA ran P2M faster alone but held up P2P beside it: the
  // product took 0.565 against 0.532 ms on the 163,842-node sphere)
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int CH = 64;
  static_assert(N2 <= 64, "one thread per (j, k)");
  __shared__ float sxa[4][CH][2 * N];   // Sx, dSx
  __shared__ float syza[4][CH][4 * N];  // Sy, dSy, Sz, dSz
  __shared__ float4 swa[4][CH];         // c, g nx / w, g ny / w, g nz / w
  const int grp = threadIdx.x >> 6, gt = threadIdx.x & 63;
  const int li = blockIdx.x * 4 + grp;
  if (li >= nleaf) return;                              // whole groups only (named barriers below)
  float (*sx)[2 * N] = sxa[grp];
  float (*syz)[4 * N] = syza[grp];
  float4 *sw = swa[grp];
  const int b = leaves[li];
  const int beg = bbeg[b], end = bend[b];
  const float invw = (float)(1.0 / center[b].w);
  const bool act = gt < N2;
  const int j = act ? gt / N : 0, k = act ? gt % N : 0;
  float A[N], B[N];
#pragma unroll
  for (int i = 0; i < N; ++i) A[i] = B[i] = 0.0f;
  for (int c0 = beg; c0 < end; c0 += CH) {
    const int cnt = min(CH, end - c0);
    if (gt < cnt) {
      const int t = gt;
      const float4 p = pos[c0 + t], q = nrm[c0 + t];
      const float2 fh = xs[c0 + t];
      float s[N], ds[N];
      cheb_basis<N>(p.x * invw, s, ds);
#pragma unroll
      for (int m = 0; m < N; ++m) { sx[t][m] = s[m]; sx[t][N + m] = ds[m]; }
      cheb_basis<N>(p.y * invw, s, ds);
#pragma unroll
      for (int m = 0; m < N; ++m) { syz[t][m] = s[m]; syz[t][N + m] = ds[m]; }
      cheb_basis<N>(p.z * invw, s, ds);
#pragma unroll
      for (int m = 0; m < N; ++m) { syz[t][2 * N + m] = s[m]; syz[t][3 * N + m] = ds[m]; }
      const float g = -p.w * fh.x * invw;
      sw[t] = make_float4(p.w * fh.y, g * q.x, g * q.y, g * q.z);
    }
    asm volatile("bar.sync %0, 64;" ::"r"(grp + 1) : "memory");
    if (act) {
      for (int t = 0; t < cnt; ++t) {
        const float sy = syz[t][j], dsy = syz[t][N + j], sz = syz[t][2 * N + k], dsz = syz[t][3 * N + k];
        const float4 w = sw[t];
        const float yz = sy * sz;
        const float pa = w.x * yz, pb = w.y * yz, pq = fmaf(w.z, dsy * sz, w.w * (sy * dsz));
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float x = sx[t][i], dx = sx[t][N + i];
          A[i] = fmaf(pa, x, A[i]);
          B[i] = fmaf(pb, dx, fmaf(pq, x, B[i]));
        }
      }
    }
    asm volatile("bar.sync %0, 64;" ::"r"(grp + 1) : "memory");
  }
  if (act) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int m = (i * N + j) * N + k;
      M[(size_t)b * 2 * N3 + m] = fmaf(B[i], inv_ebar, A[i]);
      M[(size_t)b * 2 * N3 + N3 + m] = A[i] + B[i];
    }
  }
}

// Apply the separable 1-D operator S2[c] along the three axes of a box of weights.
// transpose == false: out[i,j,k] = sum S[cx][i][i'] S[cy][j][j'] S[cz][k][k'] in[i',j',k']
// transpose == true : out[i',j',k'] = sum S[cx][i][i'] ... in[i,j,k]
// The operators come from shared memory (sS[c][row][q], staged by stage_m2m_ops): a
// thread's row depends on its output point, and constant-memory reads that differ across
// a warp are serialised.
template <int N>
__device__ __forceinline__ void stage_m2m_ops(float *sS) {
  for (int e = threadIdx.x; e < 2 * N * N; e += blockDim.x) {
    const int c = e / (N * N), r = (e / N) % N, q = e % N;
    sS[e] = c_m2m[N][c * kMaxOrder * kMaxOrder + r * kMaxOrder + q];
  }
}

template <int N>
__device__ __forceinline__ float apply_axis(const float *in, const float *sS, int m, int axis, int c, bool transpose) {
  const int i = m / (N * N), j = (m / N) % N, k = m % N;
  const float *S = sS + c * N * N;
  float acc = 0.0f;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    int src;
    int row = axis == 0 ? i : (axis == 1 ? j : k);
    float w = transpose ? S[q * N + row] : S[row * N + q];
    if (axis == 0) src = q * N * N + j * N + k;
    else if (axis == 1) src = i * N * N + q * N + k;
    else src = i * N * N + j * N + q;
    acc = fmaf(w, in[src], acc);
  }
  return acc;
}

// M2M: every parent of one level sums its children's translated multipoles.
template <int N>
__global__ void k_m2m(int ls, const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                      const int4 *__restrict__ anchor, float *__restrict__ M) {
  constexpr int N3 = N * N * N;
  __shared__ float s0[2 * N3], s1[2 * N3], sS[2 * N * N];
  const int b = ls + blockIdx.x;
  const int nc = nchild[b];
  if (nc == 0) return;
  stage_m2m_ops<N>(sS);
  const int e = threadIdx.x;               // (kernel, m)
  const bool act = e < 2 * N3;
  const int kt = e / N3, m = e % N3;
  float acc = 0.0f;
  for (int q = 0; q < nc; ++q) {
    const int c = child0[b] + q;
    const int4 a = anchor[c];
    if (act) s0[e] = M[(size_t)c * 2 * N3 + e];
    __syncthreads();
    float v = act ? apply_axis<N>(s0 + kt * N3, sS, m, 2, a.z & 1, false) : 0.0f;
    __syncthreads();
    if (act) s1[e] = v;
    __syncthreads();
    v = act ? apply_axis<N>(s1 + kt * N3, sS, m, 1, a.y & 1, false) : 0.0f;
    __syncthreads();
    if (act) s0[e] = v;
    __syncthreads();
    v = act ? apply_axis<N>(s0 + kt * N3, sS, m, 0, a.x & 1, false) : 0.0f;
    acc += v;
    __syncthreads();
  }
  if (act) M[(size_t)b * 2 * N3 + e] = acc;
}

// L2L: every box of one level adds its parent's local expansion, re-interpolated.
template <int N>
__global__ void k_l2l(int ls, const int32_t *__restrict__ parent, const int4 *__restrict__ anchor,
                      float *__restrict__ L) {
  constexpr int N3 = N * N * N;
  __shared__ float s0[2 * N3], s1[2 * N3], sS[2 * N * N];
  const int b = ls + blockIdx.x;
  const int p = parent[b];
  stage_m2m_ops<N>(sS);
  const int4 a = anchor[b];
  const int e = threadIdx.x;
  const bool act = e < 2 * N3;
  const int kt = e / N3, m = e % N3;
  if (act) s0[e] = L[(size_t)p * 2 * N3 + e];
  __syncthreads();
  float v = act ? apply_axis<N>(s0 + kt * N3, sS, m, 0, a.x & 1, true) : 0.0f;
  __syncthreads();
  if (act) s1[e] = v;
  __syncthreads();
  v = act ? apply_axis<N>(s1 + kt * N3, sS, m, 1, a.y & 1, true) : 0.0f;
  __syncthreads();
  if (act) s0[e] = v;
  __syncthreads();
  v = act ? apply_axis<N>(s0 + kt * N3, sS, m, 2, a.z & 1, true) : 0.0f;
  if (act) L[(size_t)b * 2 * N3 + e] += v;
}

// ------------------------------------------------------------------------------------
// M2L (FP32, CUDA cores).  One CTA per (row tile of 64 target weights, (level, offset)
// group, kernel); the 64 x n^3 slice of the translation matrix stays in shared memory
// while the group's pairs stream through in chunks of 32.  Results are added with
// atomics (several offsets feed the same target box).
// ------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_m2l(const M2LGroup *__restrict__ groups, const int2 *__restrict__ pairs,
                                             const float *__restrict__ Klap, const float *__restrict__ Kyuk,
                                             const dbl4 *__restrict__ center, int yuk_min_level,
                                             const float *__restrict__ M, float *__restrict__ L) {
  constexpr int N3 = N * N * N;
  constexpr int RT = 64, PC = 32, LD = N3 + 1;
  extern __shared__ float smem[];
  float *Ks = smem;                 // [RT][LD]
  float *Ms = smem + RT * LD;       // [N3][PC]
  const M2LGroup g = groups[blockIdx.y];
  const int kt = blockIdx.z;
  if (kt == 1 && g.level < yuk_min_level) return;
  const int r0 = blockIdx.x * RT;
  const int rows = min(RT, N3 - r0);
  const size_t N6 = (size_t)N3 * N3;
  const float *K = kt == 0 ? Klap + (size_t)g.offset * N6 : Kyuk + ((size_t)g.level * kNumOffsets + g.offset) * N6;
  for (int e = threadIdx.x; e < RT * N3; e += blockDim.x) {
    int r = e / N3, c = e % N3;
    Ks[r * LD + c] = r < rows ? K[(size_t)(r0 + r) * N3 + c] : 0.0f;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pc = 0; pc < g.count; pc += PC) {
    const int cnt = min(PC, g.count - pc);
    __syncthreads();
    for (int e = threadIdx.x; e < N3 * PC; e += blockDim.x) {
      int p = e / N3, k = e % N3;
      float v = 0.0f;
      if (p < cnt) v = M[((size_t)pairs[g.start + pc + p].y * 2 + kt) * N3 + k];
      Ms[k * PC + p] = v;
    }
    __syncthreads();
    float acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    const float *k0 = Ks + lane * LD, *k1 = Ks + (lane + 32) * LD;
#pragma unroll 4
    for (int k = 0; k < N3; ++k) {
      const float a0 = k0[k], a1 = k1[k];
      const float4 mv = *reinterpret_cast<const float4 *>(Ms + k * PC + warp * 4);
      acc[0][0] = fmaf(a0, mv.x, acc[0][0]); acc[0][1] = fmaf(a0, mv.y, acc[0][1]);
      acc[0][2] = fmaf(a0, mv.z, acc[0][2]); acc[0][3] = fmaf(a0, mv.w, acc[0][3]);
      acc[1][0] = fmaf(a1, mv.x, acc[1][0]); acc[1][1] = fmaf(a1, mv.y, acc[1][1]);
      acc[1][2] = fmaf(a1, mv.z, acc[1][2]); acc[1][3] = fmaf(a1, mv.w, acc[1][3]);
    }
    const float scale = kt == 0 ? (float)(1.0 / center[pairs[g.start].x].w) : 1.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = warp * 4 + q;
      if (p >= cnt) continue;
      const int tb = pairs[g.start + pc + p].x;
      float *dst = L + ((size_t)tb * 2 + kt) * N3 + r0;
      if (lane < rows) atomicAdd(dst + lane, acc[0][q] * scale);
      if (lane + 32 < rows) atomicAdd(dst + lane + 32, acc[1][q] * scale);
    }
  }
}

// M2L matrices: Laplace for a unit box (scaled by 1/w when used), Yukawa per level.
__global__ void k_m2l_table(int N, int nslots, const int3 *__restrict__ offs, double kw, double invw,
                            float *__restrict__ out) {
  const int N3 = N * N * N;
  const int64_t tot = (int64_t)nslots * N3 * N3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int slot = (int)(e / ((int64_t)N3 * N3));
    int rem = (int)(e % ((int64_t)N3 * N3));
    int mt = rem / N3, ms = rem % N3;
    int3 o = offs[slot];
    const float *nd = c_nodes[N];
    double tx = nd[mt / (N * N)], ty = nd[(mt / N) % N], tz = nd[mt % N];
    double sx = 2.0 * o.x + nd[ms / (N * N)], sy = 2.0 * o.y + nd[(ms / N) % N], sz = 2.0 * o.z + nd[ms % N];
    double r = sqrt((tx - sx) * (tx - sx) + (ty - sy) * (ty - sy) + (tz - sz) * (tz - sz));
    double v = kInv4Pi / r;
    if (kw >= 0.0) v = exp(-kw * r) * v * invw;
    out[e] = (float)v;
  }
}

// ------------------------------------------------------------------------------------
// P2L: list-4 sources straight into a box's local weights.
// ------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_p2l(const int32_t *__restrict__ xbox, const int64_t *__restrict__ xptr,
                                             const int32_t *__restrict__ xidx, const int32_t *__restrict__ bbeg,
                                             const int32_t *__restrict__ bend, const dbl4 *__restrict__ center,
                                             const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                                             const float2 *__restrict__ xs, float inv_ebar, float kappa,
                                             float *__restrict__ L) {
  constexpr int N3 = N * N * N;
  constexpr int CH = 128;
  __shared__ float4 sp[CH], sn[CH];
  const int b = xbox[blockIdx.x];
  const dbl4 cb = center[b];
  const float w = (float)cb.w;
  float accL[(N3 + 255) / 256], accY[(N3 + 255) / 256];
  float px[(N3 + 255) / 256], py[(N3 + 255) / 256], pz[(N3 + 255) / 256];
#pragma unroll
  for (int r = 0; r < (N3 + 255) / 256; ++r) {
    accL[r] = accY[r] = 0.0f;
    int m = threadIdx.x + 256 * r;
    if (m < N3) {
      px[r] = w * c_nodes[N][m / (N * N)];
      py[r] = w * c_nodes[N][(m / N) % N];
      pz[r] = w * c_nodes[N][m % N];
    }
  }
  for (int64_t j = xptr[b]; j < xptr[b + 1]; ++j) {
    const int c = xidx[j];
    const dbl4 cc = center[c];
    const float ox = (float)(cc.x - cb.x), oy = (float)(cc.y - cb.y), oz = (float)(cc.z - cb.z);
    for (int s0 = bbeg[c]; s0 < bend[c]; s0 += CH) {
      const int cnt = min(CH, bend[c] - s0);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        float4 p = pos[s0 + t], q = nrm[s0 + t];
        float2 fh = xs[s0 + t];
        sp[t] = make_float4(p.x + ox, p.y + oy, p.z + oz, p.w * fh.y);
        sn[t] = make_float4(q.x, q.y, q.z, -p.w * fh.x);
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < (N3 + 255) / 256; ++r) {
        if (threadIdx.x + 256 * r >= N3) continue;
        float aL = accL[r], aY = accY[r];
        for (int t = 0; t < cnt; ++t) {
          const float4 y = sp[t], q = sn[t];
          const float dx = px[r] - y.x, dy = py[r] - y.y, dz = pz[r] - y.z;
          const float r2 = dx * dx + dy * dy + dz * dz;
          const float ri = rsqrtf(r2);
          const float rr = r2 * ri;
          const float G = ri, G3 = ri * ri * ri;
          const float ndt = q.x * dx + q.y * dy + q.z * dz;
          const float e = __expf(-kappa * rr);
          const float g1 = e * (1.0f + kappa * rr) * G3;
          aL += y.w * G + q.w * inv_ebar * ndt * G3;
          aY += y.w * e * G + q.w * ndt * g1;
        }
        accL[r] = aL;
        accY[r] = aY;
      }
    }
  }
  const float s = (float)kInv4Pi;
#pragma unroll
  for (int r = 0; r < (N3 + 255) / 256; ++r) {
    int m = threadIdx.x + 256 * r;
    if (m < N3) {
      L[(size_t)b * 2 * N3 + m] += s * accL[r];
      L[(size_t)b * 2 * N3 + N3 + m] += s * accY[r];
    }
  }
}

// ------------------------------------------------------------------------------------
// L2P: evaluate both local expansions and their normal derivatives at leaf targets.
// ------------------------------------------------------------------------------------
constexpr int kL2PThreads = 64;   // leaves hold ~cap/3 nodes on surfaces

template <int N>
__global__ void __launch_bounds__(kL2PThreads, 12) k_l2p(const int32_t *__restrict__ leaves, const int32_t *__restrict__ bbeg,
                                             const int32_t *__restrict__ bend, const dbl4 *__restrict__ center,
                                             const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                                             const float *__restrict__ L, float4 *__restrict__ phi) {
  constexpr int N3 = N * N * N;
  __shared__ float sL[2 * N3];
  const int b = leaves[blockIdx.x];
  for (int e = threadIdx.x; e < 2 * N3; e += blockDim.x) sL[e] = L[(size_t)b * 2 * N3 + e];
  __syncthreads();
  const float invw = (float)(1.0 / center[b].w);
  for (int t = bbeg[b] + threadIdx.x; t < bend[b]; t += blockDim.x) {
    const float4 p = pos[t], q = nrm[t];
    float sx[N], dsx[N], sy[N], dsy[N], sz[N], dsz[N];
    cheb_basis<N>(p.x * invw, sx, dsx);
    cheb_basis<N>(p.y * invw, sy, dsy);
    cheb_basis<N>(p.z * invw, sz, dsz);
    float out[4];
#pragma unroll 1
    for (int kt = 0; kt < 2; ++kt) {
      const float *Lk = sL + kt * N3;
      float phi0 = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float a = 0.f, bj = 0.f, cj = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          float u = 0.f, du = 0.f;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const float l = Lk[(i * N + j) * N + k];
            u = fmaf(l, sz[k], u);
            du = fmaf(l, dsz[k], du);
          }
          a = fmaf(u, sy[j], a);
          bj = fmaf(u, dsy[j], bj);
          cj = fmaf(du, sy[j], cj);
        }
        phi0 = fmaf(a, sx[i], phi0);
        gx = fmaf(a, dsx[i], gx);
        gy = fmaf(bj, sx[i], gy);
        gz = fmaf(cj, sx[i], gz);
      }
      const float dn = (q.x * gx + q.y * gy + q.z * gz) * invw;
      if (kt == 0) { out[0] = phi0; out[1] = dn; } else { out[2] = phi0; out[3] = dn; }
    }
    phi[t] = make_float4(out[0], out[1], out[2], out[3]);
  }
}

// ------------------------------------------------------------------------------------
// P2P (lists 1 and 3): point (far-rule) sums over t != p, both kernels, both outputs.
// ------------------------------------------------------------------------------------
constexpr int kP2PChunk = 768;      // sources staged in shared memory at a time (8 CTAs/SM)
constexpr int kP2PPairs = kP2PChunk / 2;
constexpr int kP2PBoxes = 64;       // source boxes described in shared memory at a time
constexpr int kP2PRegBlocks = kP2PResident;

// Far-rule sums of one source at one target, without the 1/(4 pi):
//   PhiL += c/r + (g/eps_bar) (n.d)/r^3
//   dn PhiL += -c (n0.d)/r^3 + (g/eps_bar) [(n0.n)/r^3 - 3 (n.d)(n0.d)/r^5]
//   PhiY += c e/r + g (n.d) e1/r^3,           e = exp(-kr), e1 = e (1 + kr)
//   dn PhiY += e1 [g (n0.n) - c (n0.d)]/r^3 - 3 g e2 (n.d)(n0.d)/r^5,  e2 = e (1 + kr + (kr)^2/3)
// with d = x_target - y_source.  g enters only through the vector g n.
//
// The sums run on packed FP32 pairs (sm_100 FFMA2 / FADD2 / FMUL2): each thread takes
// its target against two sources per instruction, lane 0 an even and lane 1 an odd
// source of the staged chunk.  The target's coordinates, normal and skip radius sit in
// both lanes for the whole loop; the staging stores every source component already
// paired with its neighbour's, so no instruction of the loop packs or broadcasts.
// Every packed operation rounds each lane as its scalar counterpart does, so the
// distance and skip test below are the scalar p2p_r2 / p2p_evaluates, bit for bit.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// 2^x on the special-function unit (PTX ex2.approx); e^-kr = 2^(-kr log2 e).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) on the special-function unit, flushing subnormal inputs (PTX rsqrt.approx.ftz):
// P2P evaluates it only for r^2 above the squared skip radius (~1e-2 A^2), far from the
// subnormal range, so the flush changes nothing there and saves the subnormal handling
// that rsqrtf carries.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct P2PTarget {
  float2 x, y, z;        // position in the target leaf's frame, both lanes
  float2 nx, ny, nz;     // unit normal n0
  float2 rs;             // scaled skip radius
};

// sources: a = (-x0, -x1, -y0, -y1), b = (-z0, -z1, c0, c1), c = (gnx0, gnx1, gny0, gny1),
// d = (gnz0, gnz1, skip0, skip1); positions in the target leaf's frame.
__device__ __forceinline__ void p2p_pair2(const P2PTarget &t, const float4 &a, const float4 &b, const float4 &c,
                                          const float4 &d, float2 inv_e, float2 kappa, float2 &sL, float2 &nD,
                                          float2 &sY, float2 &dY) {
  const float2 dx = __fadd2_rn(t.x, make_float2(a.x, a.y));
  const float2 dy = __fadd2_rn(t.y, make_float2(a.z, a.w));
  const float2 dz = __fadd2_rn(t.z, make_float2(b.x, b.y));
  const float2 cc = make_float2(b.z, b.w);
  const float2 gx = make_float2(c.x, c.y), gy = make_float2(c.z, c.w), gz = make_float2(d.x, d.y);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));   // p2p_r2
  const float2 R = __fadd2_rn(t.rs, make_float2(d.z, d.w));                        // p2p_evaluates
  const float2 RR = __fmul2_rn(R, R);
  // Pairs inside the skip radius (t == p among them) contribute nothing here: the near
  // CSR carries their whole near-rule value.
  const float2 ri = make_float2(r2.x > RR.x ? rsqrt_approx(r2.x) : 0.0f, r2.y > RR.y ? rsqrt_approx(r2.y) : 0.0f);
  const float2 ri2 = __fmul2_rn(ri, ri);
  const float2 G3 = __fmul2_rn(ri, ri2);
  const float2 gnd = __ffma2_rn(gx, dx, __ffma2_rn(gy, dy, __fmul2_rn(gz, dz)));      // g n.d
  const float2 npd = __ffma2_rn(t.nx, dx, __ffma2_rn(t.ny, dy, __fmul2_rn(t.nz, dz)));  // n0.d
  const float2 gnn = __ffma2_rn(t.nx, gx, __ffma2_rn(t.ny, gy, __fmul2_rn(t.nz, gz)));  // g n0.n
  const float2 kr = __fmul2_rn(kappa, __fmul2_rn(r2, ri));
  const float2 arg = __fmul2_rn(kr, dup2(-1.4426950408889634f));
  const float2 ex = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
  const float2 e1 = __ffma2_rn(ex, kr, ex);
  const float2 e2 = __ffma2_rn(__fmul2_rn(ex, kr), __fmul2_rn(kr, dup2(1.0f / 3.0f)), e1);
  const float2 cri = __fmul2_rn(cc, ri);
  const float2 A = __fmul2_rn(gnd, G3);
  const float2 B = __fmul2_rn(gnn, G3);
  const float2 npdG3 = __fmul2_rn(npd, G3);
  const float2 Tn = __fmul2_rn(__fmul2_rn(__fmul2_rn(A, dup2(-3.0f)), npd), ri2);     // -T
  sL = __fadd2_rn(sL, __ffma2_rn(inv_e, A, cri));
  // nD accumulates -dn PhiL = c (n0.d)/r^3 - (1/eps_bar)(B - T)
  nD = __ffma2_rn(make_float2(-inv_e.x, -inv_e.y), __fadd2_rn(B, Tn), __ffma2_rn(cc, npdG3, nD));
  sY = __ffma2_rn(ex, cri, __ffma2_rn(e1, A, sY));
  // negated operands instead of products with -1 (measured: P2P 0.256 -> 0.2515 ms on the
  // 163,842-node sphere)
  const float2 BmC = __ffma2_rn(make_float2(-cc.x, -cc.y), npdG3, B);               // B - c (n0.d)/r^3
  dY = __ffma2_rn(e1, BmC, __ffma2_rn(e2, Tn, dY));
}

// A unit that covers its leaf's whole source list stores; a part of a split leaf adds.
__device__ __forceinline__ void store_or_add(float4 *p, float4 v, bool whole) {
  if (whole) *p = v;
  else asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// A P2P argument: the kernel's own, or (batched) the unit's problem's, read from shared
// memory where it is used so that no pointer stays live across the loops.
#define P2P_ARG(name) (kBatch ? s_req.name : name##_1)

// The body of the P2P kernels: with kBatch the work units of several problems share one
// launch, unit.w naming the problem whose arrays (reqs[unit.w], copied to shared memory
// per unit) it reads, and units of a problem whose *active flag is 0 are skipped.
template <bool kBatch>
__device__ __forceinline__ void p2p_body(int nunits, const int4 *__restrict__ units, const int32_t *__restrict__ leaves_1,
                                         const int64_t *__restrict__ pptr_1, const int32_t *__restrict__ pidx_1,
                                         const int32_t *__restrict__ bbeg_1, const int32_t *__restrict__ bend_1,
                                         const dbl4 *__restrict__ center_1, const float4 *__restrict__ pos_1,
                                         const float4 *__restrict__ nrm_1, const float2 *__restrict__ xs_1,
                                         float inv_ebar_1, float kappa_1, float skip_scale_1, float4 *__restrict__ phi_1,
                                         const P2PReq *__restrict__ reqs) {
  static_assert(2 * kP2PThreads <= kP2PPairs, "the reduction reuses the staging buffer");
  __shared__ float4 sa[kP2PPairs], sb[kP2PPairs], sc[kP2PPairs], sd[kP2PPairs];
  __shared__ int s_beg[kP2PBoxes], s_pre[kP2PBoxes + 1];
  __shared__ float s_off[kP2PBoxes][3];
  __shared__ __align__(8) P2PReq s_req;
  float4 *red = sa;
  // The resident blocks walk the cost-ordered work units in boustrophedon order: in round
  // k block b takes unit k G + b for even k and k G + G - 1 - b for odd k (G blocks), so
  // the block that drew the costliest unit of one round draws the cheapest of the next.  A
  // unit is one leaf's targets against a range of its source boxes; leaves with more pairs
  // than the unit budget are split, and their units add into the (zeroed) output.
  const int G = gridDim.x;
  for (int k = 0; k * G < nunits; ++k) {
  const int li = k * G + ((k & 1) ? (G - 1 - (int)blockIdx.x) : (int)blockIdx.x);
  if (li >= nunits) continue;
  if (k > 0) __syncthreads();                           // the previous unit's reduction read red
  const int4 unit = units[li];
  if constexpr (kBatch) {
    static_assert(sizeof(P2PReq) % 8 == 0, "copied as 8-byte words");
    if (threadIdx.x < sizeof(P2PReq) / 8)
      reinterpret_cast<uint64_t *>(&s_req)[threadIdx.x] = reinterpret_cast<const uint64_t *>(reqs + unit.w)[threadIdx.x];
    __syncthreads();
    if (s_req.active && *s_req.active == 0) continue;  // uniform: the problem has stopped
  }
  const float2 inv_e = dup2(kBatch ? s_req.inv_ebar : inv_ebar_1), kap = dup2(kBatch ? s_req.kappa : kappa_1);
  const int leaf = unit.x;
  const int b = P2P_ARG(leaves)[leaf];
  const dbl4 cb = P2P_ARG(center)[b];
  const int tb = P2P_ARG(bbeg)[b], te = P2P_ARG(bend)[b];
  // each thread takes two targets, t and t + tile, against the same sources
  const int tile = min((te - tb + 1) / 2, kP2PThreads);
  const int slices = kP2PThreads / tile;
  const int ti = threadIdx.x % tile, si = threadIdx.x / tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t l0 = unit.y, l1 = unit.z;               // this unit's source boxes
  const bool whole = l0 == P2P_ARG(pptr)[leaf] && l1 == P2P_ARG(pptr)[leaf + 1];
  for (int t0 = tb; t0 < te; t0 += 2 * tile) {
    const int t = t0 + ti, t2 = t + tile;
    const bool act = si < slices && t < te;
    const bool act2 = act && t2 < te;
    P2PTarget tg, tg2;
    {
      const float4 xp = act ? P2P_ARG(pos)[t] : make_float4(0, 0, 0, 0);
      const float4 np = act ? P2P_ARG(nrm)[t] : make_float4(0, 0, 0, 0);
      tg.x = dup2(xp.x); tg.y = dup2(xp.y); tg.z = dup2(xp.z);
      tg.nx = dup2(np.x); tg.ny = dup2(np.y); tg.nz = dup2(np.z);
      tg.rs = dup2(p2p_skip_radius(P2P_ARG(skip_scale), np.w));
      // a missing second target repeats the first (its sums are not stored)
      const float4 xq = act2 ? P2P_ARG(pos)[t2] : xp;
      const float4 nq = act2 ? P2P_ARG(nrm)[t2] : np;
      tg2.x = dup2(xq.x); tg2.y = dup2(xq.y); tg2.z = dup2(xq.z);
      tg2.nx = dup2(nq.x); tg2.ny = dup2(nq.y); tg2.nz = dup2(nq.z);
      tg2.rs = dup2(p2p_skip_radius(P2P_ARG(skip_scale), nq.w));
    }
    float2 sL = dup2(0.f), nD = dup2(0.f), sY = dup2(0.f), dY = dup2(0.f);
    float2 sL2 = dup2(0.f), nD2 = dup2(0.f), sY2 = dup2(0.f), dY2 = dup2(0.f);
    for (int64_t g0 = l0; g0 < l1; g0 += kP2PBoxes) {
      const int nb = (int)min((int64_t)kP2PBoxes, l1 - g0);
      __syncthreads();
      int mycnt = 0;
      if (threadIdx.x < nb) {
        const int c = P2P_ARG(pidx)[g0 + threadIdx.x];
        const dbl4 cc = P2P_ARG(center)[c];
        s_beg[threadIdx.x] = P2P_ARG(bbeg)[c];
        mycnt = P2P_ARG(bend)[c] - P2P_ARG(bbeg)[c];
        s_off[threadIdx.x][0] = (float)(cc.x - cb.x);
        s_off[threadIdx.x][1] = (float)(cc.y - cb.y);
        s_off[threadIdx.x][2] = (float)(cc.z - cb.z);
      }
      if (warp < 2) {                       // inclusive scan of the (<= 64) box sizes
        int v = mycnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        s_pre[threadIdx.x + 1] = v;         // per-warp partial; fixed up below
      }
      __syncthreads();
      if (threadIdx.x >= 32 && threadIdx.x < 64) s_pre[threadIdx.x + 1] += s_pre[32];
      if (threadIdx.x == 0) s_pre[0] = 0;
      __syncthreads();
      const int total = s_pre[nb];
      for (int c0 = 0; c0 < total; c0 += kP2PChunk) {
        const int cnt = min(kP2PChunk, total - c0);
        const int npairs = (cnt + 1) >> 1;
        if (c0 > 0) __syncthreads();
        for (int e = threadIdx.x; e < 2 * npairs; e += kP2PThreads) {
          float px = 0.f, py = 0.f, pz = 0.f, cw = 0.f, gx = 0.f, gy = 0.f, gz = 0.f, rs = 3.0e18f;
          if (e < cnt) {                    // the odd slot past the end stays a never-evaluated pad
            const int j = c0 + e;
            int lo = 0, hi = nb;            // last box with s_pre[box] <= j
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (s_pre[mid] <= j) lo = mid; else hi = mid;
            }
            const int sidx = s_beg[lo] + (j - s_pre[lo]);
            const float4 p = P2P_ARG(pos)[sidx], q = P2P_ARG(nrm)[sidx];
            const float2 fh = P2P_ARG(xs)[sidx];
            px = __fadd_rn(p.x, s_off[lo][0]);
            py = __fadd_rn(p.y, s_off[lo][1]);
            pz = __fadd_rn(p.z, s_off[lo][2]);
            cw = p.w * fh.y;
            const float g = -p.w * fh.x;
            gx = g * q.x; gy = g * q.y; gz = g * q.z;
            rs = p2p_skip_radius(P2P_ARG(skip_scale), q.w);
          }
          const int pr = e >> 1, ln = e & 1;
          float *fa = reinterpret_cast<float *>(sa + pr), *fb = reinterpret_cast<float *>(sb + pr);
          float *fc = reinterpret_cast<float *>(sc + pr), *fd = reinterpret_cast<float *>(sd + pr);
          fa[ln] = -px; fa[2 + ln] = -py;
          fb[ln] = -pz; fb[2 + ln] = cw;
          fc[ln] = gx; fc[2 + ln] = gy;
          fd[ln] = gz; fd[2 + ln] = rs;
        }
        __syncthreads();
        if (act) {
          for (int e = si; e < npairs; e += slices) {
            const float4 qa = sa[e], qb = sb[e], qc = sc[e], qd = sd[e];
            p2p_pair2(tg, qa, qb, qc, qd, inv_e, kap, sL, nD, sY, dY);
            p2p_pair2(tg2, qa, qb, qc, qd, inv_e, kap, sL2, nD2, sY2, dY2);
          }
        }
      }
    }
    __syncthreads();
    red[threadIdx.x] = make_float4(sL.x + sL.y, -(nD.x + nD.y), sY.x + sY.y, dY.x + dY.y);
    red[kP2PThreads + threadIdx.x] = make_float4(sL2.x + sL2.y, -(nD2.x + nD2.y), sY2.x + sY2.y, dY2.x + dY2.y);
    __syncthreads();
    if (si == 0 && t < te) {
      const float s = (float)kInv4Pi;
      float4 a = red[ti];
      for (int k = 1; k < slices; ++k) {
        const float4 v = red[k * tile + ti];
        a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
      }
      store_or_add(P2P_ARG(phi) + t, make_float4(s * a.x, s * a.y, s * a.z, s * a.w), whole);
      if (t2 < te) {
        float4 c = red[kP2PThreads + ti];
        for (int k = 1; k < slices; ++k) {
          const float4 v = red[kP2PThreads + k * tile + ti];
          c.x += v.x; c.y += v.y; c.z += v.z; c.w += v.w;
        }
        store_or_add(P2P_ARG(phi) + t2, make_float4(s * c.x, s * c.y, s * c.z, s * c.w), whole);
      }
    }
  }
  }
}

__global__ void __launch_bounds__(kP2PThreads, kP2PRegBlocks) k_p2p(int nunits, const int4 *__restrict__ units,
                                                      const int32_t *__restrict__ leaves,
                                                      const int64_t *__restrict__ pptr,
                                                      const int32_t *__restrict__ pidx,
                                                      const int32_t *__restrict__ bbeg,
                                                      const int32_t *__restrict__ bend,
                                                      const dbl4 *__restrict__ center,
                                                      const float4 *__restrict__ pos,
                                                      const float4 *__restrict__ nrm,
                                                      const float2 *__restrict__ xs, float inv_ebar,
                                                      float kappa, float skip_scale,
                                                      float4 *__restrict__ phi) {
  p2p_body<false>(nunits, units, leaves, pptr, pidx, bbeg, bend, center, pos, nrm, xs, inv_ebar, kappa, skip_scale,
                  phi, nullptr);
}

// P2P of several problems in one launch: the units of all of them, cost-ordered together.
__global__ void __launch_bounds__(kP2PThreads, kP2PRegBlocks) k_p2p_batch(int nunits, const int4 *__restrict__ units,
                                                                          const P2PReq *__restrict__ reqs) {
  p2p_body<true>(nunits, units, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f,
                 0.f, 0.f, nullptr, reqs);
}

// ------------------------------------------------------------------------------------
// Combine (Eq. 5): y1 = alpha f - PhiL + PhiY + sum_near (dB f - dA h)
//                  y2 = alpha h - dn PhiL + dn PhiY / eps_bar + sum_near (dD f - dC h)
// Eight lanes per row walk the near-field CSR.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_combine(int64_t n, int parts, float alpha, float inv_ebar,
                                                 const float2 *__restrict__ xs, const float4 *__restrict__ pfar,
                                                 const float4 *__restrict__ pnear, const int64_t *__restrict__ nptr,
                                                 const int32_t *__restrict__ ncol, const float4 *__restrict__ ncoef,
                                                 float *__restrict__ ys) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = gid >> 3;
  const int sub = threadIdx.x & 7;
  const bool row = p < n;           // every lane stays for the shuffles below
  float a1 = 0.f, a2 = 0.f;
  if (row && (parts & AFMPB_PART_NEAR)) {
    for (int64_t j = nptr[p] + sub; j < nptr[p + 1]; j += 8) {
      const float4 c = ncoef[j];
      const float2 x = xs[ncol[j]];
      a1 = fmaf(c.y, x.x, fmaf(-c.x, x.y, a1));
      a2 = fmaf(c.w, x.x, fmaf(-c.z, x.y, a2));
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    a1 += __shfl_xor_sync(0xffffffffu, a1, o, 8);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o, 8);
  }
  if (row && sub == 0) {
    const float2 x = xs[p];
    if (parts & AFMPB_PART_DIAG) {
      a1 += alpha * x.x;
      a2 += alpha * x.y;
    }
    if (parts & AFMPB_PART_FAR) {
      const float4 u = pfar[p], v = pnear[p];
      a1 += -(u.x + v.x) + (u.z + v.z);
      a2 += -(u.y + v.y) + (u.w + v.w) * inv_ebar;
    }
    ys[p] = a1;
    ys[n + p] = a2;
  }
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
namespace {

double cheb_s(int n, int m, double x) {   // s_m(x) in double (host tables)
  double xm = std::cos((2.0 * m + 1.0) * kPi / (2.0 * n));
  double v = 1.0 / n;
  for (int k = 1; k < n; ++k) v += 2.0 / n * std::cos(k * std::acos(xm)) * std::cos(k * std::acos(std::max(-1.0, std::min(1.0, x))));
  return v;
}

// Chebyshev tables of every order, uploaded once per device (host double -> float).
Err init_cheb_tables() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return make_err(AFMPB_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return Err{};
  static float cheb[kMaxOrder + 1][kMaxOrder * kMaxOrder], nodes[kMaxOrder + 1][kMaxOrder],
      m2m[kMaxOrder + 1][2 * kMaxOrder * kMaxOrder];
  for (int n = 2; n <= kMaxOrder; ++n) {
    for (int m = 0; m < n; ++m) {
      nodes[n][m] = (float)std::cos((2.0 * m + 1.0) * kPi / (2.0 * n));
      for (int k = 0; k < n; ++k)
        cheb[n][m * kMaxOrder + k] = (float)((k == 0 ? 1.0 : 2.0) / n * std::cos(k * (2.0 * m + 1.0) * kPi / (2.0 * n)));
    }
    for (int c = 0; c < 2; ++c)
      for (int m = 0; m < n; ++m)
        for (int mp = 0; mp < n; ++mp) {
          const double xmp = std::cos((2.0 * mp + 1.0) * kPi / (2.0 * n));
          const double xi = (c == 0 ? -0.5 : 0.5) + 0.5 * xmp;
          m2m[n][c * kMaxOrder * kMaxOrder + m * kMaxOrder + mp] = (float)cheb_s(n, m, xi);
        }
  }
  AFMPB_CUDA(cudaMemcpyToSymbol(c_cheb, cheb, sizeof(cheb)));
  AFMPB_CUDA(cudaMemcpyToSymbol(c_nodes, nodes, sizeof(nodes)));
  AFMPB_CUDA(cudaMemcpyToSymbol(c_m2m, m2m, sizeof(m2m)));
  done[dev] = true;
  return Err{};
}

template <int N>
Err launch_far(afmpb_t *h, cudaStream_t s, StageTimer *tm, int parts) {
  constexpr int N3 = N * N * N;
  const auto &T = h->shape;
  const float inv_ebar = (float)(1.0 / h->ebar);
  const int mthreads = ((2 * N3 + 31) / 32) * 32;
  const bool plane_wave = h->opt.m2l_method == AFMPB_M2L_PLANE_WAVE;
  const bool compressed = !h->m2l_groups.empty() && h->m2l_rank > 0 && !plane_wave;
  // P2L adds into L, which the compressed M2L does not touch (it writes Lc; the expansion
  // adds Lc into L afterwards): in a whole product it runs on a branch of its own from the
  // zeroed L to just before the expansion, beside the upward pass and the M2L.
  const bool p2l_beside = compressed && parts == kFarAll && !tm && h->side2 && h->n_xbox > 0;
  auto launch_p2l = [&](cudaStream_t st) -> Err {
    k_p2l<N><<<(unsigned)h->n_xbox, 256, 0, st>>>(h->d_xbox, h->d_x_ptr, h->d_x_idx, h->d_box_begin, h->d_box_end,
                                                  h->d_box_center, h->d_pos, h->d_nrm, h->d_xs, inv_ebar,
                                                  (float)h->kappa, h->d_L);
    return check_launch("k_p2l");
  };
  if (parts & kFarUp) {
  AFMPB_CUDA(cudaMemsetAsync(h->d_L, 0, sizeof(float) * (size_t)T.nbox * 2 * N3, s));
  if (p2l_beside) {
    AFMPB_CUDA(cudaEventRecord(h->ev_fork2, s));
    AFMPB_CUDA(cudaStreamWaitEvent(h->side2, h->ev_fork2, 0));
    AFMPB_TRY(launch_p2l(h->side2));
    AFMPB_CUDA(cudaEventRecord(h->ev_join2, h->side2));
  }
  k_p2m<N><<<(T.nleaf + 3) / 4, 256, 0, s>>>(T.nleaf, h->d_leaves, h->d_box_begin, h->d_box_end, h->d_box_center, h->d_pos,
                                   h->d_nrm, h->d_xs, inv_ebar, h->d_M);
  AFMPB_TRY(check_launch("k_p2m"));
  if (tm) tm->mark("p2m", 1);
  for (int level = T.nlevel - 2; level >= 2; --level) {
    int ls = T.lvl_start[level], nl = T.lvl_start[level + 1] - ls;
    k_m2m<N><<<nl, mthreads, 0, s>>>(ls, h->d_box_child0, h->d_box_nchild, h->d_box_anchor, h->d_M);
    AFMPB_TRY(check_launch("k_m2m"));
  }
  if (tm) tm->mark("m2m", std::max(0, T.nlevel - 3));
  }
  if (compressed && p2l_beside) {
    AFMPB_TRY(enqueue_m2l_svd(h, s, tm, kFarUp | kFarM2L));
    AFMPB_CUDA(cudaStreamWaitEvent(s, h->ev_join2, 0));
    AFMPB_TRY(enqueue_m2l_svd(h, s, tm, kFarDown));
  } else if (compressed) {
    AFMPB_TRY(enqueue_m2l_svd(h, s, tm, parts));  // marks compress, m2l, expand itself
  } else if (!h->m2l_groups.empty() && (parts & kFarM2L)) {
    if (plane_wave) {
      AFMPB_TRY(enqueue_m2l_pw(h, s));
    } else if (h->opt.precision == 1) {
      AFMPB_TRY(enqueue_m2l_tc(h, s));
    } else {
      constexpr int RT = 64, PC = 32;
      const size_t smem = sizeof(float) * (RT * (N3 + 1) + N3 * PC);
      dim3 grid((N3 + RT - 1) / RT, (unsigned)h->m2l_groups.size(), 2);
      k_m2l<N><<<grid, 256, smem, s>>>(h->d_m2l_groups, h->d_m2l_pairs, h->d_K_lap, h->d_K_yuk, h->d_box_center,
                                       h->m2l_yuk_levels, h->d_M, h->d_L);
      AFMPB_TRY(check_launch("k_m2l"));
    }
  }
  if (tm && !compressed) tm->mark("m2l", h->m2l_groups.empty() ? 0 : 1);
  if (!(parts & kFarDown)) return Err{};
  if (h->n_xbox > 0 && !p2l_beside) AFMPB_TRY(launch_p2l(s));
  if (tm) tm->mark("p2l", h->n_xbox > 0 ? 1 : 0);
  for (int level = 3; level < T.nlevel; ++level) {
    int ls = T.lvl_start[level], nl = T.lvl_start[level + 1] - ls;
    k_l2l<N><<<nl, mthreads, 0, s>>>(ls, h->d_box_parent, h->d_box_anchor, h->d_L);
    AFMPB_TRY(check_launch("k_l2l"));
  }
  if (tm) tm->mark("l2l", std::max(0, T.nlevel - 3));
  k_l2p<N><<<T.nleaf, kL2PThreads, 0, s>>>(h->d_leaves, h->d_box_begin, h->d_box_end, h->d_box_center, h->d_pos, h->d_nrm,
                                   h->d_L, h->d_phi_far);
  AFMPB_TRY(check_launch("k_l2p"));
  if (tm) tm->mark("l2p", 1);
  return Err{};
}

template <int N>
Err set_m2l_smem() {
  constexpr int N3 = N * N * N;
  const size_t smem = sizeof(float) * (64 * (N3 + 1) + N3 * 32);
  AFMPB_TRY(raise_smem_limit((const void *)k_m2l<N>, (int)smem));
  return Err{};
}

}  // namespace

Err enqueue_far(afmpb_t *h, cudaStream_t s, StageTimer *tm, int parts) {
  switch (h->order) {
    case 2: return launch_far<2>(h, s, tm, parts);
    case 3: return launch_far<3>(h, s, tm, parts);
    case 4: return launch_far<4>(h, s, tm, parts);
    case 5: return launch_far<5>(h, s, tm, parts);
    case 6: return launch_far<6>(h, s, tm, parts);
    case 7: return launch_far<7>(h, s, tm, parts);
    case 8: return launch_far<8>(h, s, tm, parts);
    default: return make_err(AFMPB_EINVAL, "fmm_order must be in [2, 8]");
  }
}

Err enqueue_p2p(afmpb_t *h, cudaStream_t s) {
  // Beside the far-field chain, six resident blocks per SM walk the units while the
  // chain's kernels run at a higher stream priority (measured best among four to six, and
  // against one block per unit: 0.565 against 0.595 ms for the 163,842-node product).
  // Alone (meshes above the overlap limit) one block per unit lets the block scheduler
  // hand the cost-ordered units out as blocks finish, which balances better than the
  // static deal (0.226 against 0.256 ms for the same sphere's P2P timed alone).
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = overlap_p2p(h) ? std::max(1, std::min(h->p2p_nunits, std::min(h->p2p_resident, kP2PRegBlocks) * sms))
                                  : std::max(1, h->p2p_nunits);
  AFMPB_CUDA(cudaMemsetAsync(h->d_phi_near, 0, sizeof(float4) * h->n, s));   // split leaves add into it
  k_p2p<<<grid, kP2PThreads, 0, s>>>(h->p2p_nunits, h->d_p2p_units, h->d_leaves, h->d_p2p_ptr, h->d_p2p_idx, h->d_box_begin,
                                                  h->d_box_end, h->d_box_center, h->d_pos, h->d_nrm, h->d_xs,
                                                  (float)(1.0 / h->ebar), (float)h->kappa,
                                                  (float)(kP2PSkip * h->opt.near_c), h->d_phi_near);
  return check_launch("k_p2p");
}

P2PReq p2p_req_of(const afmpb_t *h, const int *active) {
  P2PReq q{};
  q.leaves = h->d_leaves;
  q.pptr = h->d_p2p_ptr;
  q.pidx = h->d_p2p_idx;
  q.bbeg = h->d_box_begin;
  q.bend = h->d_box_end;
  q.center = h->d_box_center;
  q.pos = h->d_pos;
  q.nrm = h->d_nrm;
  q.xs = h->d_xs;
  q.phi = h->d_phi_near;
  q.active = active;
  q.inv_ebar = (float)(1.0 / h->ebar);
  q.kappa = (float)h->kappa;
  q.skip_scale = (float)(kP2PSkip * h->opt.near_c);
  return q;
}

Err enqueue_p2p_batch(const P2PReq *d_reqs, const int4 *d_units, int nunits, int resident, cudaStream_t s) {
  if (nunits == 0) return Err{};
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, std::min(nunits, std::min(resident, kP2PRegBlocks) * sms));
  k_p2p_batch<<<grid, kP2PThreads, 0, s>>>(nunits, d_units, d_reqs);
  return check_launch("k_p2p_batch");
}

// The near-field correction of Eq. 5 folded into the P2P sums, on the P2P branch right
// after P2P, so that it overlaps the rest of the far-field chain instead of following it:
//   PhiL <- PhiL - sum_near (dB f - dA h),   dn PhiL <- dn PhiL - sum_near (dD f - dC h)
// (the combine subtracts PhiL and dn PhiL, so the correction enters with its own sign).
// Eight lanes per row walk the near-field CSR, as in k_combine.
__global__ void __launch_bounds__(256) k_near_fold(int64_t n, const float2 *__restrict__ xs,
                                                   const int64_t *__restrict__ nptr, const int32_t *__restrict__ ncol,
                                                   const float4 *__restrict__ ncoef, float4 *__restrict__ pnear) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = gid >> 3;
  const int sub = threadIdx.x & 7;
  const bool row = p < n;           // every lane stays for the shuffles below
  float a1 = 0.f, a2 = 0.f;
  if (row) {
    for (int64_t j = nptr[p] + sub; j < nptr[p + 1]; j += 8) {
      const float4 c = ncoef[j];
      const float2 x = xs[ncol[j]];
      a1 = fmaf(c.y, x.x, fmaf(-c.x, x.y, a1));
      a2 = fmaf(c.w, x.x, fmaf(-c.z, x.y, a2));
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    a1 += __shfl_xor_sync(0xffffffffu, a1, o, 8);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o, 8);
  }
  if (row && sub == 0) {
    float4 v = pnear[p];
    v.x -= a1;
    v.y -= a2;
    pnear[p] = v;
  }
}

// Eq. 5 assembly when the near correction is already in the P2P sums: one thread per row.
__global__ void __launch_bounds__(256) k_combine_folded(int64_t n, int parts, float alpha, float inv_ebar,
                                                        const float2 *__restrict__ xs, const float4 *__restrict__ pfar,
                                                        const float4 *__restrict__ pnear, float *__restrict__ ys) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  float a1 = 0.f, a2 = 0.f;
  if (parts & AFMPB_PART_DIAG) {
    const float2 x = xs[p];
    a1 = alpha * x.x;
    a2 = alpha * x.y;
  }
  const float4 u = pfar[p], v = pnear[p];
  a1 += -(u.x + v.x) + (u.z + v.z);
  a2 += -(u.y + v.y) + (u.w + v.w) * inv_ebar;
  ys[p] = a1;
  ys[n + p] = a2;
}

Err enqueue_near_fold(afmpb_t *h, cudaStream_t s) {
  if (h->n == 0) return Err{};
  k_near_fold<<<div_up(h->n * 8, 256), 256, 0, s>>>(h->n, h->d_xs, h->d_near_ptr, h->d_near_col, h->d_near_coef,
                                                     h->d_phi_near);
  return check_launch("k_near_fold");
}

Err enqueue_combine(afmpb_t *h, cudaStream_t s, int parts) {
  if (parts & kNearFolded) {          // near correction already in the P2P sums (with the far part)
    if (h->n == 0) return Err{};
    k_combine_folded<<<div_up(h->n, 256), 256, 0, s>>>(h->n, parts, (float)h->alpha, (float)(1.0 / h->ebar), h->d_xs,
                                                        h->d_phi_far, h->d_phi_near, h->d_ys);
    return check_launch("k_combine_folded");
  }
  k_combine<<<div_up(h->n * 8, 256), 256, 0, s>>>(h->n, parts, (float)h->alpha, (float)(1.0 / h->ebar), h->d_xs,
                                                   h->d_phi_far, h->d_phi_near, h->d_near_ptr, h->d_near_col,
                                                   h->d_near_coef, h->d_ys);
  return check_launch("k_combine");
}

Err build_fmm(afmpb_t *h) {
  const int n = h->order;
  const int N3 = n * n * n;
  cudaStream_t s = h->stream;
  auto &A = h->arena;
  const auto &T = h->shape;
  AFMPB_TRY(init_cheb_tables());
  // offset slots: [-3,3]^3 minus [-1,1]^3
  std::vector<int> code_to_slot(343, -1);
  std::vector<int3> offs;
  for (int ox = -3; ox <= 3; ++ox)
    for (int oy = -3; oy <= 3; ++oy)
      for (int oz = -3; oz <= 3; ++oz) {
        if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
        code_to_slot[(ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)] = (int)offs.size();
        offs.push_back(make_int3(ox, oy, oz));
      }
  int3 *d_offs = nullptr;
  AFMPB_TRY(A.alloc(&d_offs, offs.size(), "m2l offsets"));
  AFMPB_CUDA(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int3) * offs.size(), cudaMemcpyHostToDevice, s));
  for (auto &g : h->m2l_groups) g.offset = code_to_slot[g.offset];
  if (!h->m2l_groups.empty()) {
    AFMPB_TRY(A.alloc(&h->d_m2l_groups, h->m2l_groups.size(), "m2l groups"));
    AFMPB_CUDA(cudaMemcpyAsync(h->d_m2l_groups, h->m2l_groups.data(), sizeof(M2LGroup) * h->m2l_groups.size(),
                               cudaMemcpyHostToDevice, s));
  }
  // Yukawa M2L is skipped on coarse levels where the screened kernel across the one-box
  // gap of a list-2 pair (distance >= 2 w) is below e^-40 of its unscreened value.
  int maxlev = 0;
  for (auto &g : h->m2l_groups) maxlev = std::max(maxlev, g.level + 1);
  h->m2l_yuk_levels = 0;
  while (h->m2l_yuk_levels < maxlev && h->kappa * 2.0 * std::ldexp(T.w0, -h->m2l_yuk_levels) > 40.0)
    ++h->m2l_yuk_levels;
  if (h->laplace_only) h->m2l_yuk_levels = maxlev;
  bool compressed = false;
  AFMPB_TRY(build_m2l_svd(h, &compressed));
  if (compressed) {
    A.release(d_offs);
    AFMPB_TRY(A.alloc(&h->d_M, (size_t)T.nbox * 2 * N3, "M"));
    AFMPB_TRY(A.alloc(&h->d_L, (size_t)T.nbox * 2 * N3, "L"));
    AFMPB_CUDA(cudaMemsetAsync(h->d_M, 0, sizeof(float) * (size_t)T.nbox * 2 * N3, s));
    if (h->opt.precision == 1) AFMPB_TRY(build_m2l_tc(h));
    if (h->opt.m2l_method == AFMPB_M2L_PLANE_WAVE) AFMPB_TRY(build_m2l_pw(h));
    return Err{};
  }
  const size_t N6 = (size_t)N3 * N3;
  AFMPB_TRY(A.alloc(&h->d_K_lap, kNumOffsets * N6, "K laplace"));
  AFMPB_TRY(A.alloc(&h->d_K_yuk, h->laplace_only ? 1 : (size_t)std::max(maxlev, 1) * kNumOffsets * N6, "K yukawa"));
  k_m2l_table<<<1024, 256, 0, s>>>(n, kNumOffsets, d_offs, -1.0, 1.0, h->d_K_lap);
  AFMPB_TRY(check_launch("k_m2l_table lap"));
  for (int l = std::max(2, h->m2l_yuk_levels); l < maxlev; ++l) {
    double w = std::ldexp(T.w0, -l);
    k_m2l_table<<<1024, 256, 0, s>>>(n, kNumOffsets, d_offs, h->kappa * w, 1.0 / w,
                                     h->d_K_yuk + (size_t)l * kNumOffsets * N6);
    AFMPB_TRY(check_launch("k_m2l_table yuk"));
  }
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(d_offs);
  AFMPB_TRY(A.alloc(&h->d_M, (size_t)T.nbox * 2 * N3, "M"));
  AFMPB_TRY(A.alloc(&h->d_L, (size_t)T.nbox * 2 * N3, "L"));
  AFMPB_CUDA(cudaMemsetAsync(h->d_M, 0, sizeof(float) * (size_t)T.nbox * 2 * N3, s));
  switch (n) {
    case 2: AFMPB_TRY(set_m2l_smem<2>()); break;
    case 3: AFMPB_TRY(set_m2l_smem<3>()); break;
    case 4: AFMPB_TRY(set_m2l_smem<4>()); break;
    case 5: AFMPB_TRY(set_m2l_smem<5>()); break;
    case 6: AFMPB_TRY(set_m2l_smem<6>()); break;
    case 7: AFMPB_TRY(set_m2l_smem<7>()); break;
    case 8: AFMPB_TRY(set_m2l_smem<8>()); break;
    default: return make_err(AFMPB_EINVAL, "fmm_order must be in [2, 8]");
  }
  if (h->opt.precision == 1) AFMPB_TRY(build_m2l_tc(h));
  if (h->opt.m2l_method == AFMPB_M2L_PLANE_WAVE) AFMPB_TRY(build_m2l_pw(h));
  return Err{};
}

}  // namespace afmpb
