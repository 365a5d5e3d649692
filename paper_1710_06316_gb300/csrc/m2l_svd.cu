// m2l_svd.cu -- compressed list-2 translations (M2L).
//
// The 316 translation matrices K_o of one kernel and level (n^3 x n^3, Chebyshev points
// of a target box against those of the box at offset o) share one numerically low-rank
// row space and one column space: with Q the leading eigenvectors of the Gram matrix
// sum_o K_o K_o^T, C_o = Q^T K_o Q (r x r) stands for K_o, and
//     L += K_o M   becomes   L += Q (C_o (Q^T M)).
// Because the offset set is symmetric and the kernels are radial, K_{-o} = K_o^T, so the
// same Q spans the column space (sum_o K_o^T K_o is the same Gram matrix).
// The product compresses every multipole vector once (Mc = Q^T M), translates r-vectors,
// and expands every local vector once (L += Q Lc): the translation work falls by
// (n^3 / r)^2.  r is the number of singular values of the stacked operators above
// m2l_tol times the largest, rounded up to a multiple of 16 and shared by all tables.
//
// Setup (FP64 on the GPU, eigenproblems on the host): per table, the FP64 matrices K_o,
// the Gram matrix, its eigen-decomposition, then C_o = Q^T (K_o Q).
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <thread>

#include "internal.cuh"
#include "symeig.h"

namespace afmpb {

namespace {

constexpr int kGramTile = 32;       // Gram matrix tile (32 x 32 per CTA)
constexpr int kRowsPerCta = 8;      // rows of T = K_o Q (and of C) per CTA
constexpr int kChunkBoxes = 16;     // boxes per compress / expand CTA (a multiple of 4; 16 against 32:
                                    // expand 32 -> 27 us on the 163,842-node sphere)
constexpr int kMaxN3 = kMaxOrder * kMaxOrder * kMaxOrder;
constexpr int kMaxRank = 192;       // largest compressed size (M2L staging in shared memory)

struct NodesD {
  double x[kMaxOrder];
};

// K_o(i, k): kernel between point i of the unit target box and point k of the source box
// at offset o (centres 2 o apart).  kw < 0: Laplace 1/(4 pi r); else Yukawa
// exp(-kw r)/(4 pi r) times invw (the box half width w enters as kw = kappa w).
__device__ __forceinline__ double m2l_entry(const NodesD &nd, int N, int3 o, int i, int k, double kw, double invw) {
  const double tx = nd.x[i / (N * N)], ty = nd.x[(i / N) % N], tz = nd.x[i % N];
  const double sx = 2.0 * o.x + nd.x[k / (N * N)], sy = 2.0 * o.y + nd.x[(k / N) % N],
               sz = 2.0 * o.z + nd.x[k % N];
  const double r = sqrt((tx - sx) * (tx - sx) + (ty - sy) * (ty - sy) + (tz - sz) * (tz - sz));
  double v = kInv4Pi / r;
  if (kw >= 0.0) v = exp(-kw * r) * v * invw;
  return v;
}

__global__ void k_table_f64(int N, int noffs, const int3 *__restrict__ offs, NodesD nd, double kw, double invw,
                            double *__restrict__ K) {
  const int N3 = N * N * N;
  const int64_t tot = (int64_t)noffs * N3 * N3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(e / ((int64_t)N3 * N3));
    const int rem = (int)(e % ((int64_t)N3 * N3));
    K[e] = m2l_entry(nd, N, offs[o], rem / N3, rem % N3, kw, invw);
  }
}

// The same table in FP32 (for C_o = Q^T K_o Q, which the products use in FP32 and BF16).
__global__ void k_table_f32(int N, int noffs, const int3 *__restrict__ offs, NodesD nd, double kw, double invw,
                            float *__restrict__ K) {
  const int N3 = N * N * N;
  const int64_t tot = (int64_t)noffs * N3 * N3;
  const float fkw = (float)kw, finvw = (float)invw, c = (float)kInv4Pi;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(e / ((int64_t)N3 * N3));
    const int rem = (int)(e % ((int64_t)N3 * N3));
    const int i = rem / N3, k = rem % N3;
    const int3 of = offs[o];
    const float dx = (float)(nd.x[i / (N * N)] - 2.0 * of.x - nd.x[k / (N * N)]);
    const float dy = (float)(nd.x[(i / N) % N] - 2.0 * of.y - nd.x[(k / N) % N]);
    const float dz = (float)(nd.x[i % N] - 2.0 * of.z - nd.x[k % N]);
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    float v = c / r;
    if (fkw >= 0.0f) v = expf(-fkw * r) * v * finvw;
    K[e] = v;
  }
}

// H_r = K_r K_r^T for one offset per orbit of the cube's symmetry group (blockIdx.z = r).
__global__ void __launch_bounds__(256) k_gram_rep(int N3, const double *__restrict__ K, double *__restrict__ H) {
  __shared__ double Ki[kGramTile][kGramTile + 1], Kj[kGramTile][kGramTile + 1];
  const int i0 = blockIdx.x * kGramTile, j0 = blockIdx.y * kGramTile;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2] = {{0, 0}, {0, 0}};
  const double *Ko = K + (size_t)blockIdx.z * N3 * N3;
  for (int k0 = 0; k0 < N3; k0 += kGramTile) {
    __syncthreads();
    for (int e = threadIdx.x; e < kGramTile * kGramTile; e += blockDim.x) {
      const int r = e / kGramTile, c = e % kGramTile, k = k0 + c;
      Ki[r][c] = (i0 + r < N3 && k < N3) ? Ko[(size_t)(i0 + r) * N3 + k] : 0.0;
      Kj[r][c] = (j0 + r < N3 && k < N3) ? Ko[(size_t)(j0 + r) * N3 + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < kGramTile; ++c) {
      const double a0 = Ki[ty][c], a1 = Ki[ty + 16][c], b0 = Kj[tx][c], b1 = Kj[tx + 16][c];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
  }
  double *Hr = H + (size_t)blockIdx.z * N3 * N3;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < N3 && j < N3) Hr[(size_t)i * N3 + j] = acc[a][b];
    }
}

// Gram = sum over all offsets of K_o K_o^T, from the orbit representatives: an offset g.o
// of the orbit of r has K_{g.o} = P_g K_r P_g^T (the kernel depends on |x - y| only and the
// Chebyshev grid is symmetric), so the orbit contributes (|orbit| / 48) sum_g P_g H_r P_g^T,
// entry (i, j) of which is H_r(perm_g(i), perm_g(j)) summed over the 48 elements g.
__global__ void k_gram_sym(int N3, int nrep, const double *__restrict__ H, const double *__restrict__ wrep,
                           const int32_t *__restrict__ perm, double *__restrict__ gram) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)N3 * N3) return;
  const int i = (int)(e / N3), j = (int)(e % N3);
  double sum = 0.0;
  for (int r = 0; r < nrep; ++r) {
    const double *Hr = H + (size_t)r * N3 * N3;
    double t = 0.0;
    for (int g = 0; g < 48; ++g) t += Hr[(size_t)perm[g * N3 + i] * N3 + perm[g * N3 + j]];
    sum += wrep[r] * t;
  }
  gram[e] = sum;
}

// T[o][i][b] = sum_k K_o(i, k) Q(k, b)        (Q: [N3][R]; FP32: the operators C_o are used
// in FP32 and BF16 by the products, while the basis Q itself comes from the FP64 Gram matrix)
__global__ void __launch_bounds__(128) k_kq(int N3, int R, const float *__restrict__ K, const float *__restrict__ Q,
                                            float *__restrict__ T) {
  __shared__ float Ks[kRowsPerCta][kMaxN3];
  const int o = blockIdx.x, i0 = blockIdx.y * kRowsPerCta;
  const int rows = min(kRowsPerCta, N3 - i0);
  for (int e = threadIdx.x; e < kRowsPerCta * N3; e += blockDim.x) {
    const int r = e / N3, k = e % N3;
    Ks[r][k] = r < rows ? K[((size_t)o * N3 + i0 + r) * N3 + k] : 0.0f;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < R; b += blockDim.x) {
    float acc[kRowsPerCta] = {};
    for (int k = 0; k < N3; ++k) {
      const float q = Q[(size_t)k * R + b];
#pragma unroll
      for (int r = 0; r < kRowsPerCta; ++r) acc[r] = fmaf(Ks[r][k], q, acc[r]);
    }
    for (int r = 0; r < rows; ++r) T[((size_t)o * N3 + i0 + r) * R + b] = acc[r];
  }
}

// C[o][a][b] = sum_i Q(i, a) T[o][i][b], stored FP32
__global__ void __launch_bounds__(128) k_qtt(int N3, int R, const float *__restrict__ Q, const float *__restrict__ T,
                                             float *__restrict__ C) {
  __shared__ float Qs[kRowsPerCta][kMaxN3];
  const int o = blockIdx.x, a0 = blockIdx.y * kRowsPerCta;
  const int rows = min(kRowsPerCta, R - a0);
  for (int e = threadIdx.x; e < kRowsPerCta * N3; e += blockDim.x) {
    const int r = e / N3, i = e % N3;
    Qs[r][i] = r < rows ? Q[(size_t)i * R + a0 + r] : 0.0f;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < R; b += blockDim.x) {
    float acc[kRowsPerCta] = {};
    for (int i = 0; i < N3; ++i) {
      const float t = T[((size_t)o * N3 + i) * R + b];
#pragma unroll
      for (int r = 0; r < kRowsPerCta; ++r) acc[r] = fmaf(Qs[r][i], t, acc[r]);
    }
    for (int r = 0; r < rows; ++r) C[((size_t)o * R + a0 + r) * R + b] = acc[r];
  }
}

// Asynchronous global -> shared copies (cp.async); src_bytes = 0 writes zeros.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Per-box basis change for one chunk of up to kChunkBoxes boxes of one level:
//     Y[b][kt][c] (+)= sum_k A_table[k][c] X[b][kt][k]
// compress: A = Q (K = n^3, ncol = r), X = M, Y = Mc;  expand: A = Q^T (K = r,
// ncol = n^3), X = Lc, Y = L (accumulated).  The chunk's X vectors (X[k][box]) and slabs
// of kSlabRows rows of A reach shared memory by cp.async in a kStages-deep pipeline, so
// the copy of slab s + 2 overlaps the products of slab s (a K of one or two slabs gets
// one or two buffers: the expand of r = 64 fits three CTAs per SM instead of two).  A thread owns 4 boxes x 4
// columns per tile (two 16-byte shared loads per 16 FMAs) and up to TILES tiles; ncol is
// a multiple of 4.
constexpr int kSlabRows = 32;
constexpr int kStages = 3;
// buffers the pipeline needs for K rows: slab s + 2 is issued while slab s is used
__host__ __device__ __forceinline__ int basis_stages(int K) {
  const int nslab = (K + kSlabRows - 1) / kSlabRows;
  return nslab < kStages ? (nslab > 0 ? nslab : 1) : kStages;
}
template <int TILES, bool ACCUM>
__global__ void __launch_bounds__(256) k_box_basis(int K, int ncol, const int4 *__restrict__ chunks,
                                                   const int *__restrict__ level_table,
                                                   const int *__restrict__ table_rank, int yuk_min,
                                                   const float *__restrict__ A, const float *__restrict__ X,
                                                   float *__restrict__ Y, __nv_bfloat16 *__restrict__ Y16) {
  extern __shared__ __align__(16) float sm[];
  float *Xs = sm;                                      // [K][kChunkBoxes]
  float *As = sm + (size_t)K * kChunkBoxes;            // [kStages][kSlabRows][ncol]
  const int4 ch = chunks[blockIdx.x];                  // first box, count, level
  const int kt = blockIdx.y;
  if (kt == 1 && ch.z < yuk_min) return;               // no Yukawa translations on this level
  const int table = kt == 0 ? 0 : level_table[ch.z];
  const float *At = A + (size_t)table * K * ncol;
  // the table's own rank bounds the output columns (compress) or the contraction (expand)
  const int Keff = ACCUM ? table_rank[table] : K;
  const int ceff = ACCUM ? ncol : table_rank[table];
  const int slab_elems = kSlabRows * ncol;
  const int nslab = (Keff + kSlabRows - 1) / kSlabRows;
  const int nst = basis_stages(K);                     // slab buffers (fewer when K has fewer slabs)
  // X: the box index runs fastest so that the shared stores hit distinct banks
  for (int e = threadIdx.x; e < Keff * kChunkBoxes; e += blockDim.x) {
    const int j = e % kChunkBoxes, k = e / kChunkBoxes;
    const bool v = j < ch.y;
    cp_async4(Xs + e, v ? X + ((size_t)(ch.x + j) * 2 + kt) * K + k : X, v);
  }
  // a thread's 16-byte groups of a slab: (row, group) from threadIdx.x, advanced by
  // blockDim.x groups with a carry (no division in the copy loop)
  const int c4n = ceff / 4;
  const int c4d = max(c4n, 1);
  const int r_first = c4n > 0 ? (int)threadIdx.x / c4d : kSlabRows, c_first = (int)threadIdx.x % c4d;
  const int r_step = (int)blockDim.x / c4d, c_step = (int)blockDim.x % c4d;
  auto issue_slab = [&](int sl) {
    if (sl < nslab) {
      float *dst = As + (size_t)(sl % nst) * slab_elems;
      const int k0 = sl * kSlabRows;
      const int rows = min(kSlabRows, Keff - k0);
      const float *src = At + (size_t)k0 * ncol;
      for (int r = r_first, c = c_first; r < kSlabRows;) {   // 16-byte groups used
        const bool v = r < rows;
        cp_async16(dst + r * ncol + 4 * c, v ? src + (size_t)r * ncol + 4 * c : At, v);
        r += r_step;
        c += c_step;
        if (c >= c4n) { c -= c4n; ++r; }
      }
    }
    cp_async_commit();                                 // empty groups keep the count
  };
  issue_slab(0);                                       // commits X together with slab 0
  issue_slab(1);
  const int ncol4 = ceff / 4;
  const int ntiles = (kChunkBoxes / 4) * ncol4;
  float acc[TILES][4][4] = {};
  for (int sl = 0; sl < nslab; ++sl) {
    cp_async_wait_1();                                 // X and slab sl have landed
    __syncthreads();
    issue_slab(sl + 2);                                // its buffer held slab sl - 1
    const float *as = As + (size_t)(sl % nst) * slab_elems;
    const int k0 = sl * kSlabRows, rows = min(kSlabRows, Keff - k0);
#pragma unroll
    for (int t = 0; t < TILES; ++t) {
      const int tile = threadIdx.x + t * blockDim.x;
      if (tile >= ntiles) continue;
      const int c0 = (tile % ncol4) * 4, b0 = (tile / ncol4) * 4;
#pragma unroll 4
      for (int kk = 0; kk < rows; ++kk) {
        const float4 a = *reinterpret_cast<const float4 *>(as + (size_t)kk * ncol + c0);
        const float4 x = *reinterpret_cast<const float4 *>(Xs + (size_t)(k0 + kk) * kChunkBoxes + b0);
        const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[t][i][j] = fmaf(xv[i], av[j], acc[t][i][j]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < TILES; ++t) {
    const int tile = threadIdx.x + t * blockDim.x;
    if (tile >= ntiles) continue;
    const int c4 = tile % ncol4, b0 = (tile / ncol4) * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (b0 + i >= ch.y) continue;
      float4 *y = reinterpret_cast<float4 *>(Y + ((size_t)(ch.x + b0 + i) * 2 + kt) * ncol) + c4;
      float4 v = make_float4(acc[t][i][0], acc[t][i][1], acc[t][i][2], acc[t][i][3]);
      if (ACCUM) {
        const float4 o = *y;
        v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
      }
      *y = v;
      if (!ACCUM && Y16) {   // the same vector split into BF16 hi / lo for the tensor-core M2L
        const float w[4] = {v.x, v.y, v.z, v.w};
        __align__(8) __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          hi[j] = __float2bfloat16_rn(w[j]);
          lo[j] = __float2bfloat16_rn(w[j] - __bfloat162float(hi[j]));
        }
        __nv_bfloat16 *y16 = Y16 + ((size_t)(ch.x + b0 + i) * 2 + kt) * 2 * ncol + 4 * c4;
        *reinterpret_cast<uint2 *>(y16) = *reinterpret_cast<const uint2 *>(hi);
        *reinterpret_cast<uint2 *>(y16 + ncol) = *reinterpret_cast<const uint2 *>(lo);
      }
    }
  }
}

int basis_tiles(int ncol) { return ((kChunkBoxes / 4) * (ncol / 4) + 255) / 256; }
size_t basis_smem(int K, int ncol) {
  return sizeof(float) * ((size_t)K * kChunkBoxes + (size_t)basis_stages(K) * kSlabRows * ncol);
}

template <bool ACCUM>
Err launch_box_basis(cudaStream_t s, dim3 grid, int K, int ncol, const int4 *chunks, const int *level_table,
                     const int *table_rank, int yuk_min, const float *A, const float *X, float *Y,
                     __nv_bfloat16 *Y16 = nullptr) {
  const size_t smem = basis_smem(K, ncol);
  const int nthr = std::min(256, (((kChunkBoxes / 4) * (ncol / 4) + 31) / 32) * 32);   // threads with a tile
  switch (basis_tiles(ncol)) {
    case 1: k_box_basis<1, ACCUM><<<grid, nthr, smem, s>>>(K, ncol, chunks, level_table, table_rank, yuk_min, A, X, Y, Y16); break;
    case 2: k_box_basis<2, ACCUM><<<grid, 256, smem, s>>>(K, ncol, chunks, level_table, table_rank, yuk_min, A, X, Y, Y16); break;
    case 3: k_box_basis<3, ACCUM><<<grid, 256, smem, s>>>(K, ncol, chunks, level_table, table_rank, yuk_min, A, X, Y, Y16); break;
    default: k_box_basis<4, ACCUM><<<grid, 256, smem, s>>>(K, ncol, chunks, level_table, table_rank, yuk_min, A, X, Y, Y16); break;
  }
  return check_launch(ACCUM ? "k_box_basis expand" : "k_box_basis compress");
}

template <bool ACCUM>
Err set_box_basis_smem(int K, int ncol) {
  const int smem = (int)basis_smem(K, ncol);
  switch (basis_tiles(ncol)) {
    case 1: AFMPB_TRY(raise_smem_limit((const void *)k_box_basis<1, ACCUM>, smem)); break;
    case 2: AFMPB_TRY(raise_smem_limit((const void *)k_box_basis<2, ACCUM>, smem)); break;
    case 3: AFMPB_TRY(raise_smem_limit((const void *)k_box_basis<3, ACCUM>, smem)); break;
    default: AFMPB_TRY(raise_smem_limit((const void *)k_box_basis<4, ACCUM>, smem)); break;
  }
  return Err{};
}

// Compressed M2L on the CUDA cores: one CTA per ((level, offset) group, kernel); the
// R x R operator stays in shared memory while the group's pairs stream through in chunks
// of 32 (a warp owns 4 pairs, a lane RPL rows).  Results are added with atomics.
template <int RPL>
__global__ void __launch_bounds__(256) k_m2l_c(int Rs, const M2LGroup *__restrict__ groups,
                                               const int2 *__restrict__ pairs, const float *__restrict__ C,
                                               const int *__restrict__ level_table,
                                               const int *__restrict__ table_rank, const dbl4 *__restrict__ center,
                                               int yuk_min, const float *__restrict__ Mc, float *__restrict__ Lc) {
  extern __shared__ float smem[];
  const int LD = Rs + 1;
  float *Cs = smem;                 // [Rs][LD], the table's R x R block used
  float *Ms = smem + Rs * LD;       // [R][32]
  const M2LGroup g = groups[blockIdx.x];
  const int kt = blockIdx.y;
  if (kt == 1 && g.level < yuk_min) return;
  const int table = kt == 0 ? 0 : level_table[g.level];
  const int R = table_rank[table];            // this table's rank (stride Rs in memory)
  const float *Cg = C + ((size_t)table * kNumOffsets + g.offset) * Rs * Rs;
  for (int e0 = threadIdx.x; e0 < R * R; e0 += blockDim.x * kCopyILP) {
    float v[kCopyILP];
#pragma unroll
    for (int u = 0; u < kCopyILP; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < R * R ? __ldg(Cg + (size_t)(e / R) * Rs + e % R) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kCopyILP; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < R * R) Cs[(e / R) * LD + e % R] = v[u];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float scale = kt == 0 ? (float)(1.0 / center[pairs[g.start].x].w) : 1.0f;
  __shared__ int s_src[32], s_tgt[32];
  for (int pc = 0; pc < g.count; pc += 32) {
    const int cnt = min(32, g.count - pc);
    __syncthreads();
    if (threadIdx.x < 32) {
      const int2 pr = threadIdx.x < cnt ? pairs[g.start + pc + threadIdx.x] : make_int2(0, 0);
      s_tgt[threadIdx.x] = pr.x;
      s_src[threadIdx.x] = pr.y;
    }
    __syncthreads();
    for (int e0 = threadIdx.x; e0 < R * 32; e0 += blockDim.x * kCopyILP) {
      float v[kCopyILP];
#pragma unroll
      for (int u = 0; u < kCopyILP; ++u) {
        const int e = e0 + u * (int)blockDim.x, p = e / R, k = e % R;
        v[u] = (e < R * 32 && p < cnt) ? __ldg(Mc + ((size_t)s_src[p] * 2 + kt) * Rs + k) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < kCopyILP; ++u) {
        const int e = e0 + u * (int)blockDim.x, p = e / R, k = e % R;
        if (e < R * 32) Ms[k * 32 + p] = v[u];
      }
    }
    __syncthreads();
    float acc[RPL][4] = {};
#pragma unroll 2
    for (int k = 0; k < R; ++k) {
      const float4 mv = *reinterpret_cast<const float4 *>(Ms + k * 32 + warp * 4);
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int row = lane + 32 * r;
        const float a = row < R ? Cs[row * LD + k] : 0.0f;
        acc[r][0] = fmaf(a, mv.x, acc[r][0]);
        acc[r][1] = fmaf(a, mv.y, acc[r][1]);
        acc[r][2] = fmaf(a, mv.z, acc[r][2]);
        acc[r][3] = fmaf(a, mv.w, acc[r][3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = warp * 4 + q;
      if (p >= cnt) continue;
      float *dst = Lc + ((size_t)s_tgt[p] * 2 + kt) * Rs;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int row = lane + 32 * r;
        if (row < R) atomicAdd(dst + row, acc[r][q] * scale);
      }
    }
  }
}

template <int RPL>
Err launch_m2l_c(afmpb_t *h, cudaStream_t s) {
  const int R = h->m2l_rank;
  const size_t smem = sizeof(float) * ((size_t)R * (R + 1) + (size_t)R * 32);
  dim3 grid((unsigned)h->m2l_groups.size(), 2);
  k_m2l_c<RPL><<<grid, 256, smem, s>>>(R, h->d_m2l_groups, h->d_m2l_pairs, h->d_C, h->d_level_table,
                                       h->d_table_rank, h->d_box_center, h->m2l_yuk_levels, h->d_Mc, h->d_Lc);
  return check_launch("k_m2l_c");
}

template <int RPL>
Err set_m2l_c_smem(int R) {
  const size_t smem = sizeof(float) * ((size_t)R * (R + 1) + (size_t)R * 32);
  AFMPB_TRY(raise_smem_limit((const void *)k_m2l_c<RPL>, (int)smem));
  return Err{};
}

}  // namespace

Err build_m2l_svd(afmpb_t *h, bool *compressed) {
  *compressed = false;
  const double tol = h->opt.m2l_tol;
  const int n = h->order, N3 = n * n * n;
  // the basis kernels move 16-byte vectors of n^3 weights: orders 2, 4, 6, 8
  if (tol < 0.0 || h->m2l_groups.empty() || N3 % 4 != 0) return Err{};
  cudaStream_t s = h->stream;
  auto &A = h->arena;
  const auto &T = h->shape;
  // tables: 0 = Laplace on the unit box, then Yukawa per level that translates
  int maxlev = 0;
  for (auto &g : h->m2l_groups) maxlev = std::max(maxlev, g.level + 1);
  std::vector<double> tab_kw(1, -1.0), tab_invw(1, 1.0);
  std::vector<int> level_table(std::max(maxlev, 1), 0);
  for (int l = std::max(2, h->m2l_yuk_levels); l < maxlev; ++l) {
    const double w = std::ldexp(T.w0, -l);
    level_table[l] = (int)tab_kw.size();
    tab_kw.push_back(h->kappa * w);
    tab_invw.push_back(1.0 / w);
  }
  const int ntab = (int)tab_kw.size();
  NodesD nd{};
  for (int m = 0; m < n; ++m) nd.x[m] = (double)(float)std::cos((2.0 * m + 1.0) * kPi / (2.0 * n));
  std::vector<int3> offs;
  for (int ox = -3; ox <= 3; ++ox)
    for (int oy = -3; oy <= 3; ++oy)
      for (int oz = -3; oz <= 3; ++oz)
        if (std::abs(ox) > 1 || std::abs(oy) > 1 || std::abs(oz) > 1) offs.push_back(make_int3(ox, oy, oz));
  // The cube's 48 symmetries g (axis permutation sg, signs sn): offsets fall into 16
  // orbits; for each g, perm_g maps Chebyshev point i to the point at g applied to it.
  std::vector<std::array<int, 6>> group;
  {
    const int perms3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (auto &pm : perms3)
      for (int sg = 0; sg < 8; ++sg)
        group.push_back({pm[0], pm[1], pm[2], (sg & 1) ? -1 : 1, (sg & 2) ? -1 : 1, (sg & 4) ? -1 : 1});
  }
  auto act = [&](const std::array<int, 6> &g, const int v[3], int out[3]) {
    for (int d = 0; d < 3; ++d) out[d] = g[3 + d] * v[g[d]];
  };
  std::vector<int32_t> perm((size_t)48 * N3);
  for (int gi = 0; gi < 48; ++gi)
    for (int i = 0; i < N3; ++i) {
      const int idx[3] = {i / (n * n), (i / n) % n, i % n};
      int out[3];
      for (int d = 0; d < 3; ++d) {
        const int src = idx[group[gi][d]];
        out[d] = group[gi][3 + d] > 0 ? src : n - 1 - src;   // node n-1-m is -node m
      }
      perm[(size_t)gi * N3 + i] = (out[0] * n + out[1]) * n + out[2];
    }
  std::vector<int3> reps;
  std::vector<double> wrep;
  {
    std::vector<char> seen(343, 0);
    for (const int3 &o : offs) {
      const int code = (o.x + 3) * 49 + (o.y + 3) * 7 + (o.z + 3);
      if (seen[code]) continue;
      int orbit = 0;
      const int v[3] = {o.x, o.y, o.z};
      for (auto &g : group) {
        int w[3];
        act(g, v, w);
        const int c = (w[0] + 3) * 49 + (w[1] + 3) * 7 + (w[2] + 3);
        if (!seen[c]) {
          seen[c] = 1;
          ++orbit;
        }
      }
      reps.push_back(o);
      wrep.push_back((double)orbit / 48.0);
    }
  }
  const int nrep = (int)reps.size();
  int3 *d_offs = nullptr, *d_reps = nullptr;
  double *d_K = nullptr, *d_gram = nullptr, *d_H = nullptr, *d_wrep = nullptr;
  int32_t *d_perm = nullptr;
  AFMPB_TRY(A.alloc(&d_offs, offs.size(), "svd offsets"));
  AFMPB_TRY(A.alloc(&d_reps, reps.size(), "svd orbit offsets"));
  AFMPB_TRY(A.alloc(&d_wrep, wrep.size(), "svd orbit weights"));
  AFMPB_TRY(A.alloc(&d_perm, perm.size(), "svd point permutations"));
  AFMPB_TRY(A.alloc(&d_H, (size_t)nrep * N3 * N3, "svd orbit grams"));
  AFMPB_TRY(A.alloc(&d_K, (size_t)kNumOffsets * N3 * N3, "svd K64"));
  AFMPB_TRY(A.alloc(&d_gram, (size_t)N3 * N3, "svd gram"));
  AFMPB_CUDA(cudaMemcpyAsync(d_reps, reps.data(), sizeof(int3) * reps.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(d_wrep, wrep.data(), sizeof(double) * wrep.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int3) * offs.size(), cudaMemcpyHostToDevice, s));
  // Gram matrices and their eigen-decompositions
  std::vector<std::vector<double>> gram(ntab, std::vector<double>((size_t)N3 * N3));
  const dim3 ggrid((N3 + kGramTile - 1) / kGramTile, (N3 + kGramTile - 1) / kGramTile, nrep);
  for (int t = 0; t < ntab; ++t) {
    k_table_f64<<<256, 256, 0, s>>>(n, nrep, d_reps, nd, tab_kw[t], tab_invw[t], d_K);
    AFMPB_TRY(check_launch("k_table_f64 orbits"));
    k_gram_rep<<<ggrid, 256, 0, s>>>(N3, d_K, d_H);
    AFMPB_TRY(check_launch("k_gram_rep"));
    k_gram_sym<<<div_up((int64_t)N3 * N3, 256), 256, 0, s>>>(N3, nrep, d_H, d_wrep, d_perm, d_gram);
    AFMPB_TRY(check_launch("k_gram_sym"));
    AFMPB_CUDA(cudaMemcpyAsync(gram[t].data(), d_gram, sizeof(double) * N3 * N3, cudaMemcpyDeviceToHost, s));
  }
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(d_H);
  A.release(d_perm);
  A.release(d_wrep);
  A.release(d_reps);
  std::vector<std::vector<double>> lam(ntab, std::vector<double>(N3)), zt(ntab, std::vector<double>((size_t)N3 * N3));
  std::vector<int> rc(ntab, 0);
  {
    std::vector<std::thread> pool;
    for (int t = 0; t < ntab; ++t)
      pool.emplace_back([&, t] { rc[t] = sym_eig_desc(N3, gram[t].data(), lam[t].data(), zt[t].data()); });
    for (auto &th : pool) th.join();
  }
  int rmax = 1;
  std::vector<int> rank(ntab);
  for (int t = 0; t < ntab; ++t)
    if (rc[t] != 0) return make_err(AFMPB_EINTERNAL, "M2L compression: eigensolver did not converge");
  for (int t = 0; t < ntab; ++t) {
    // Singular values of the stacked operators are the square roots of the eigenvalues.
    // The cut is relative to the larger of the table's own largest singular value and
    // the Laplace table's at the same level (sigma_0(Laplace) / w): the Yukawa and
    // Laplace far fields enter each row of Eq. 5 with O(1) weights, so a translation
    // error counts against the Laplace scale.  On strongly screened levels (kappa w of
    // several units on large molecules) the screened kernel is orders of magnitude
    // smaller and needs far fewer vectors than a cut relative to itself would keep.
    const double ref = std::max(std::sqrt(std::max(lam[t][0], 0.0)), std::sqrt(std::max(lam[0][0], 0.0)) * tab_invw[t]);
    int r = 0;
    while (r < N3 && lam[t][r] > 0.0 && std::sqrt(lam[t][r]) > tol * ref) ++r;
    rank[t] = std::min(N3, std::max(16, (r + 15) / 16 * 16));   // own rank, a multiple of 16
    rmax = std::max(rmax, rank[t]);
  }
  const int R = rmax;                  // storage stride; table t uses its first rank[t] columns
  if (R > kMaxRank || R >= N3) {       // no gain: keep the full translations
    A.release(d_gram);
    A.release(d_K);
    A.release(d_offs);
    return Err{};
  }
  h->m2l_rank = R;
  h->m2l_ntables = ntab;
  h->h_level_table = level_table;
  h->h_table_rank = rank;
  AFMPB_TRY(A.alloc(&h->d_table_rank, rank.size(), "svd table ranks"));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_table_rank, rank.data(), sizeof(int) * rank.size(), cudaMemcpyHostToDevice, s));
  AFMPB_TRY(A.alloc(&h->d_level_table, level_table.size(), "svd level table"));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_level_table, level_table.data(), sizeof(int) * level_table.size(),
                             cudaMemcpyHostToDevice, s));
  // bases Q (FP32, from the FP64 eigenvectors) and C_o = Q^T K_o Q (FP32)
  AFMPB_TRY(A.alloc(&h->d_Q, (size_t)ntab * N3 * R, "svd Q"));
  AFMPB_TRY(A.alloc(&h->d_QT, (size_t)ntab * R * N3, "svd QT"));
  AFMPB_TRY(A.alloc(&h->d_C, (size_t)ntab * kNumOffsets * R * R, "svd C"));
  float *d_Kf = reinterpret_cast<float *>(d_K), *d_T = nullptr;   // the FP64 table buffer is free now
  AFMPB_TRY(A.alloc(&d_T, (size_t)kNumOffsets * N3 * R, "svd T"));
  std::vector<float> qf((size_t)ntab * N3 * R), qtf((size_t)ntab * R * N3);
  for (int t = 0; t < ntab; ++t)
    for (int i = 0; i < N3; ++i)
      for (int a = 0; a < R; ++a) {
        const double v = a < rank[t] ? zt[t][(size_t)a * N3 + i] : 0.0;   // zero beyond the rank
        qf[((size_t)t * N3 + i) * R + a] = (float)v;
        qtf[((size_t)t * R + a) * N3 + i] = (float)v;
      }
  AFMPB_CUDA(cudaMemcpyAsync(h->d_Q, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_QT, qtf.data(), sizeof(float) * qtf.size(), cudaMemcpyHostToDevice, s));
  for (int t = 0; t < ntab; ++t) {
    const float *Qt = h->d_Q + (size_t)t * N3 * R;
    k_table_f32<<<1024, 256, 0, s>>>(n, kNumOffsets, d_offs, nd, tab_kw[t], tab_invw[t], d_Kf);
    AFMPB_TRY(check_launch("k_table_f32"));
    k_kq<<<dim3(kNumOffsets, (N3 + kRowsPerCta - 1) / kRowsPerCta), 128, 0, s>>>(N3, R, d_Kf, Qt, d_T);
    AFMPB_TRY(check_launch("k_kq"));
    k_qtt<<<dim3(kNumOffsets, (R + kRowsPerCta - 1) / kRowsPerCta), 128, 0, s>>>(
        N3, R, Qt, d_T, h->d_C + (size_t)t * kNumOffsets * R * R);
    AFMPB_TRY(check_launch("k_qtt"));
  }
  // compress / expand work: chunks of up to kChunkBoxes boxes of one level, on the levels
  // that have list-2 pairs
  std::vector<int4> chunks;
  for (int l = 2; l < std::min(T.nlevel, maxlev); ++l)
    for (int b = T.lvl_start[l]; b < T.lvl_start[l + 1]; b += kChunkBoxes)
      chunks.push_back(make_int4(b, std::min(kChunkBoxes, T.lvl_start[l + 1] - b), l, 0));
  h->m2l_nchunks = (int)chunks.size();
  AFMPB_TRY(A.alloc(&h->d_m2l_chunks, std::max<size_t>(1, chunks.size()), "svd chunks"));
  if (!chunks.empty())
    AFMPB_CUDA(cudaMemcpyAsync(h->d_m2l_chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, s));
  AFMPB_TRY(A.alloc(&h->d_Mc, (size_t)T.nbox * 2 * R, "Mc"));
  if (h->opt.precision == 1) {                     // BF16 hi / lo copy for the tensor-core M2L
    AFMPB_TRY(A.alloc(&h->d_Mc16, (size_t)T.nbox * 2 * 2 * R, "Mc bf16"));
    AFMPB_CUDA(cudaMemsetAsync(h->d_Mc16, 0, sizeof(uint16_t) * (size_t)T.nbox * 2 * 2 * R, s));
  }
  AFMPB_TRY(A.alloc(&h->d_Lc, (size_t)T.nbox * 2 * R, "Lc"));
  AFMPB_CUDA(cudaMemsetAsync(h->d_Mc, 0, sizeof(float) * (size_t)T.nbox * 2 * R, s));
  AFMPB_TRY(set_box_basis_smem<false>(N3, R));
  AFMPB_TRY(set_box_basis_smem<true>(R, N3));
  const int rpl = (R + 31) / 32;
  switch (rpl) {
    case 1: AFMPB_TRY(set_m2l_c_smem<1>(R)); break;
    case 2: AFMPB_TRY(set_m2l_c_smem<2>(R)); break;
    case 3: AFMPB_TRY(set_m2l_c_smem<3>(R)); break;
    case 4: AFMPB_TRY(set_m2l_c_smem<4>(R)); break;
    case 5: AFMPB_TRY(set_m2l_c_smem<5>(R)); break;
    default: AFMPB_TRY(set_m2l_c_smem<6>(R)); break;
  }
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(d_T);
  A.release(d_gram);
  A.release(d_K);
  A.release(d_offs);
  *compressed = true;
  return Err{};
}

Err enqueue_m2l_svd(afmpb_t *h, cudaStream_t s, StageTimer *tm, int parts) {
  const int R = h->m2l_rank, N3 = h->ncoef;
  const auto &T = h->shape;
  if (parts & kFarUp) AFMPB_CUDA(cudaMemsetAsync(h->d_Lc, 0, sizeof(float) * (size_t)T.nbox * 2 * R, s));
  if (h->m2l_nchunks == 0) return Err{};
  const dim3 cgrid((unsigned)h->m2l_nchunks, 2);
  if (parts & kFarUp) {
    AFMPB_TRY(launch_box_basis<false>(s, cgrid, N3, R, h->d_m2l_chunks, h->d_level_table, h->d_table_rank,
                                       h->m2l_yuk_levels, h->d_Q, h->d_M, h->d_Mc,
                                       reinterpret_cast<__nv_bfloat16 *>(h->d_Mc16)));
    if (tm) tm->mark("compress", 1);             // Lc memset (not a kernel) + basis change
  }
  if (!(parts & kFarM2L)) {
  } else if (h->opt.precision == 1) {
    AFMPB_TRY(enqueue_m2l_tc(h, s));
  } else {
    switch ((R + 31) / 32) {
      case 1: AFMPB_TRY(launch_m2l_c<1>(h, s)); break;
      case 2: AFMPB_TRY(launch_m2l_c<2>(h, s)); break;
      case 3: AFMPB_TRY(launch_m2l_c<3>(h, s)); break;
      case 4: AFMPB_TRY(launch_m2l_c<4>(h, s)); break;
      case 5: AFMPB_TRY(launch_m2l_c<5>(h, s)); break;
      default: AFMPB_TRY(launch_m2l_c<6>(h, s)); break;
    }
  }
  if (tm && (parts & kFarM2L)) tm->mark("m2l", 1);
  if (!(parts & kFarDown)) return Err{};
  AFMPB_TRY(launch_box_basis<true>(s, cgrid, R, N3, h->d_m2l_chunks, h->d_level_table, h->d_table_rank,
                                   h->m2l_yuk_levels, h->d_QT, h->d_Lc, h->d_L));
  if (tm) tm->mark("expand", 1);
  return Err{};
}

}  // namespace afmpb
