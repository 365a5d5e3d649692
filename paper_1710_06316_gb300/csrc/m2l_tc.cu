// m2l_tc.cu -- list-2 translations (M2L) on the 5th-generation tensor cores
// (precision mode 1).
//
// Each (level, offset) group of list-2 pairs is a dense product
//      L[:, targets] += K_o (R x R) * M[:, sources]          (Laplace and Yukawa)
// with R = n^3 (full translations) or the compressed size r (K_o = C_o, M and L the
// compressed vectors Mc and Lc).  A CTA takes one 128-row slice of K_o (A operand) and
// up to 112 pairs (B operand, the gathered source vectors) and runs tcgen05.mma
// (kind::f16: BF16 inputs, FP32 accumulation in tensor memory).  FP32 accuracy is kept by splitting every value into
// BF16 high and low parts, x = hi + lo, and summing hi*hi + hi*lo + lo*hi.
//
// The contraction (R <= 224 after padding to 16) runs in halves of 112 so that a CTA needs
// ~105 KB of shared memory and two CTAs share an SM, overlapping one CTA's loads with the
// other's MMAs.  The A halves (pre-converted at setup into the MMA operand layout) arrive
// by bulk asynchronous copy (the TMA engine, completion counted on an mbarrier) while the
// 256 threads gather and split the B half.  One thread issues the MMAs and commits them
// to a second mbarrier; the accumulator is read with tcgen05.ld and added into the target
// local expansions.
//
// Operand layout in shared memory: canonical K-major without swizzle -- 8 x 16-byte core
// matrices (8 rows x 8 BF16), rows strided by 128 B, K strided by rows/8 * 128 B.
// Every mbarrier wait is bounded: on expiry the kernel records an error flag, waits once
// more (bounded) for its own operations, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace afmpb {

constexpr int kTcRows = 128;                   // MMA M
constexpr int kTcPairs = 112;                  // MMA N upper bound (pairs per CTA)
constexpr int kTcKHalf = 112;                  // K per half (7 MMA k-steps of 16)
constexpr int kTcK = 2 * kTcKHalf;             // largest contraction: 224 >= n^3 for order <= 6
constexpr int kTcAElems = kTcRows * kTcKHalf;  // 14,336 BF16 per A half-tile (hi or lo)
constexpr int kTcBElems = kTcPairs * kTcKHalf; // 12,544 BF16 per B half-tile
constexpr int kTcThreads = 256;
constexpr int kTcTmemCols = 128;



// Translation matrices -> BF16 hi/lo half-tiles in the operand layout.
// out: [table][slot][row tile][k half][hi, lo][kTcAElems].  Sources: compressed tables
// C [table][slot][R][R] when C is given, else Klap / Kyuk [level][slot] (R = n^3).
__global__ void k_tc_tables(int N3, int ntables, int nslots, const float *__restrict__ Klap,
                            const float *__restrict__ Kyuk, const float *__restrict__ C,
                            const int *__restrict__ table_level, __nv_bfloat16 *__restrict__ out) {
  const int rtiles = (N3 + kTcRows - 1) / kTcRows;
  const int64_t total = (int64_t)ntables * nslots * rtiles * 2 * kTcAElems;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int within = (int)(e % kTcAElems);
    int64_t t = e / kTcAElems;
    const int kh = (int)(t % 2);
    t /= 2;
    const int rt = (int)(t % rtiles);
    t /= rtiles;
    const int slot = (int)(t % nslots);
    const int table = (int)(t / nslots);
    const int row = within / kTcKHalf, kk = within % kTcKHalf;
    const int r = rt * kTcRows + row, k = kh * kTcKHalf + kk;
    float v = 0.0f;
    if (r < N3 && k < N3) {
      const float *K = C ? C + ((size_t)table * nslots + slot) * N3 * N3
                         : table == 0 ? Klap + (size_t)slot * N3 * N3
                                      : Kyuk + ((size_t)table_level[table] * kNumOffsets + slot) * N3 * N3;
      v = K[(size_t)r * N3 + k];
    }
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    const int64_t base = ((((int64_t)table * nslots + slot) * rtiles + rt) * 2 + kh) * 2 * kTcAElems;
    const uint32_t off = canon_off(row, kk, kTcRows) >> 1;
    out[base + off] = hi;
    out[base + kTcAElems + off] = lo;
  }
}

__global__ void __launch_bounds__(kTcThreads, 2) k_m2l_tc(int N3, const TCItem *__restrict__ items,
                                                          const M2LGroup *__restrict__ groups,
                                                          const int2 *__restrict__ pairs,
                                                          const __nv_bfloat16 *__restrict__ tiles,
                                                          const int *__restrict__ level_table, int nslots,
                                                          int yuk_min_level, const dbl4 *__restrict__ center,
                                                          const float *__restrict__ M, float *__restrict__ L,
                                                          int *__restrict__ err_flag,
                                                          const int *__restrict__ table_rank) {
  extern __shared__ __align__(128) uint8_t smem[];
  __nv_bfloat16 *a_hi = reinterpret_cast<__nv_bfloat16 *>(smem);
  __nv_bfloat16 *a_lo = a_hi + kTcAElems;
  __nv_bfloat16 *b_hi = a_lo + kTcAElems;
  __nv_bfloat16 *b_lo = b_hi + kTcBElems;
  __shared__ __align__(8) uint64_t mbar_load, mbar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int s_src[kTcPairs], s_tgt[kTcPairs];

  const TCItem it = items[blockIdx.x];
  const M2LGroup g = groups[it.group];
  const int rt = blockIdx.y;
  const int kt = blockIdx.z;
  const int rtiles = (N3 + kTcRows - 1) / kTcRows;
  if (kt == 1 && g.level < yuk_min_level) return;       // screened away (uniform per CTA)
  const int table = kt == 0 ? 0 : level_table[g.level];
  // compressed tables: the table's own rank bounds rows and contraction (N3 is the stride)
  const int Rt = table_rank ? table_rank[table] : N3;
  if (rt * kTcRows >= Rt) return;                       // no rows of this tile (uniform)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cnt = it.count;
  const int npad = (cnt + 15) & ~15;
  const uint32_t mb_load = cvta_smem(&mbar_load), mb_mma = cvta_smem(&mbar_mma);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cvta_smem(&tmem_base)),
                 "r"(kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_load));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_mma));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (threadIdx.x < kTcPairs) {
    const bool v = threadIdx.x < cnt;
    const int2 pr = v ? pairs[g.start + it.start + threadIdx.x] : make_int2(-1, -1);
    s_src[threadIdx.x] = pr.y;
    s_tgt[threadIdx.x] = pr.x;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  bool ok = true;
  const int nkh = (Rt + kTcKHalf - 1) / kTcKHalf;     // contraction halves (1 or 2)
  int issued = 0;                                      // MMA commits made on mb_mma
  int loads = 0;                                       // A-operand copies started on mb_load

  for (int kh = 0; kh < nkh && ok; ++kh) {
    ++loads;
    // A half: two bulk copies (hi, lo) tracked by mb_load
    if (threadIdx.x == 0) {
      const int64_t base = ((((int64_t)table * nslots + g.offset) * rtiles + rt) * 2 + kh) * 2 * kTcAElems;
      const __nv_bfloat16 *src = tiles + base;
      const uint32_t bytes = 2 * kTcAElems * 2;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb_load), "r"(bytes));
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              cvta_smem(a_hi)),
          "l"(src), "r"((uint32_t)(kTcAElems * 2)), "r"(mb_load)
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              cvta_smem(a_lo)),
          "l"(src + kTcAElems), "r"((uint32_t)(kTcAElems * 2)), "r"(mb_load)
          : "memory");
    }
    // B half: gathered source multipoles, split into hi / lo (rows = pairs).  Each thread
    // first issues all of its loads (up to kU units of 8 values), then converts and stores.
    constexpr int kG = kTcKHalf / 8;    // 14 groups of 8 along K
    constexpr int kU = (kTcPairs * kG + kTcThreads - 1) / kTcThreads;
    float4 u[kU][2];
#pragma unroll
    for (int i = 0; i < kU; ++i) {
      const int e = threadIdx.x + i * kTcThreads;
      const int p = e / kG, k8 = e % kG;
      const int k0 = kh * kTcKHalf + k8 * 8;
      u[i][0] = u[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < kTcPairs * kG && p < cnt && k0 < Rt) {
        const float *m = M + ((size_t)s_src[p] * 2 + kt) * N3 + k0;
        if (k0 + 8 <= Rt) {
          u[i][0] = __ldg(reinterpret_cast<const float4 *>(m));
          u[i][1] = __ldg(reinterpret_cast<const float4 *>(m + 4));
        } else {
          float v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = (k0 + q < Rt) ? m[q] : 0.0f;
          u[i][0] = make_float4(v[0], v[1], v[2], v[3]);
          u[i][1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kU; ++i) {
      const int e = threadIdx.x + i * kTcThreads;
      if (e >= kTcPairs * kG) continue;
      const int p = e / kG, k8 = e % kG;
      const float v[8] = {u[i][0].x, u[i][0].y, u[i][0].z, u[i][0].w, u[i][1].x, u[i][1].y, u[i][1].z, u[i][1].w};
      __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) split_bf16(v[q], hi[q], lo[q]);
      const uint32_t off = canon_off(p, k8 * 8, kTcPairs);
      *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(b_hi) + off) = *reinterpret_cast<const uint4 *>(hi);
      *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(b_lo) + off) = *reinterpret_cast<const uint4 *>(lo);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    ok = __syncthreads_and(mbar_wait(mb_load, (uint32_t)kh));   // block-uniform
    if (ok && threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t idesc = instr_desc(kTcRows, npad);
      const uint32_t lbo_a = (kTcRows / 8) * 128, lbo_b = (kTcPairs / 8) * 128, sbo = 128;
      const uint32_t sa_hi = cvta_smem(a_hi), sa_lo = cvta_smem(a_lo);
      const uint32_t sb_hi = cvta_smem(b_hi), sb_lo = cvta_smem(b_lo);
      const int ksteps = (min(kTcKHalf, Rt - kh * kTcKHalf) + 15) / 16;
      for (int s = 0; s < ksteps; ++s) {
        const uint32_t ka = 2 * s * lbo_a, kb = 2 * s * lbo_b;
        const uint64_t dah = smem_desc(sa_hi + ka, lbo_a, sbo), dal = smem_desc(sa_lo + ka, lbo_a, sbo);
        const uint64_t dbh = smem_desc(sb_hi + kb, lbo_b, sbo), dbl = smem_desc(sb_lo + kb, lbo_b, sbo);
        const uint32_t acc0 = (kh > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb_mma));
    }
    if (ok) ++issued;                                  // block-uniform
    // the MMAs must finish reading A and B before the next half overwrites them
    ok = __syncthreads_and(ok && mbar_wait(mb_mma, (uint32_t)kh));
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (lane == 0) atomicExch(err_flag, 1);      // the handle's flag: set when a bounded wait expired
    // bounded: let the last issued MMA group (they complete in order) drain before the
    // tensor memory is freed
    if (issued > 0) mbar_wait(mb_mma, (uint32_t)((issued - 1) & 1));
    if (loads > 0) mbar_wait(mb_load, (uint32_t)((loads - 1) & 1));    // and the last bulk copy
  } else {
    // epilogue: warps w and w+4 read accumulator rows 32 (w % 4) .. + 31 (one row per lane)
    // and split the columns; the tile is transposed through shared memory (the A buffer,
    // free once the MMAs completed) so that every thread adds 4 consecutive rows of one
    // pair with a single 16-byte vector atomic.
    float *tile = reinterpret_cast<float *>(smem);       // [pair][128 rows]
    const int quarter = warp & 3, half = warp >> 2;
    const int lrow = quarter * 32 + lane;
    for (int c0 = half * 16; c0 < npad; c0 += 32) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int q = 0; q < 16; ++q) tile[(c0 + q) * kTcRows + lrow] = __uint_as_float(r[q]);
    }
    __syncthreads();
    const float scale = kt == 0 ? (float)(1.0 / center[s_tgt[0]].w) : 1.0f;
    const int rows_valid = min(kTcRows, Rt - rt * kTcRows);   // a multiple of 4
    for (int e = threadIdx.x; e < cnt * (kTcRows / 4); e += kTcThreads) {
      const int p = e / (kTcRows / 4), g4 = (e % (kTcRows / 4)) * 4;
      if (g4 >= rows_valid) continue;
      float4 v = *reinterpret_cast<const float4 *>(tile + p * kTcRows + g4);
      v.x *= scale; v.y *= scale; v.z *= scale; v.w *= scale;
      atomicAdd(reinterpret_cast<float4 *>(L + ((size_t)s_tgt[p] * 2 + kt) * N3 + rt * kTcRows + g4), v);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

namespace {
constexpr int kTcSmem = (2 * kTcAElems + 2 * kTcBElems) * 2;
}

Err build_m2l_tc(afmpb_t *h) {
  // R: compressed size (a multiple of 16) or n^3
  const int N3 = h->m2l_rank > 0 ? h->m2l_rank : h->ncoef;
  // the epilogue adds 4 consecutive weights with one 16-byte atomic: R must be a
  // multiple of 4 and fit the 224-wide contraction
  if (N3 > kTcK || N3 % 4 != 0)
    return make_err(AFMPB_EINVAL, "precision 1 (tensor-core M2L) supports fmm_order 2, 4 or 6, "
                                  "or a compressed rank <= 224");
  // compressed ranks <= 112: the target-stationary kernel (m2l_ts.cu) takes the whole M2L
  if (m2l_ts_applies(h)) return build_m2l_ts(h);
  auto &A = h->arena;
  cudaStream_t s = h->stream;
  // work items: chunks of <= 112 pairs per (level, offset) group
  std::vector<TCItem> items;
  int maxlev = 0;
  for (size_t gi = 0; gi < h->m2l_groups.size(); ++gi) {
    const auto &g = h->m2l_groups[gi];
    maxlev = std::max(maxlev, g.level + 1);
    for (int st = 0; st < g.count; st += kTcPairs) items.push_back(TCItem{(int)gi, st, std::min(kTcPairs, g.count - st)});
  }
  h->tc_items = (int)items.size();
  if (items.empty()) return Err{};
  // tables: 0 = Laplace (unit box), 1.. = Yukawa per level that needs it
  std::vector<int> level_table(std::max(maxlev, 1), 0), table_level(1, 0);
  for (int l = std::max(2, h->m2l_yuk_levels); l < maxlev; ++l) {
    level_table[l] = (int)table_level.size();
    table_level.push_back(l);
  }
  const int ntables = (int)table_level.size();
  const int rtiles = (N3 + kTcRows - 1) / kTcRows;
  const size_t elems = (size_t)ntables * kNumOffsets * rtiles * 2 * 2 * kTcAElems;
  AFMPB_TRY(A.alloc(&h->d_tc_tiles, elems, "tensor-core M2L tiles"));
  int *d_table_level = nullptr;
  AFMPB_TRY(A.alloc(&d_table_level, table_level.size(), "table level"));
  AFMPB_TRY(A.alloc(&h->d_tc_level_table, level_table.size(), "level table"));
  AFMPB_TRY(A.alloc(&h->d_tc_items, items.size(), "tc items"));
  AFMPB_TRY(alloc_wait_flag(h));
  AFMPB_CUDA(cudaMemcpyAsync(d_table_level, table_level.data(), sizeof(int) * table_level.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_tc_level_table, level_table.data(), sizeof(int) * level_table.size(),
                             cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(h->d_tc_items, items.data(), sizeof(TCItem) * items.size(), cudaMemcpyHostToDevice, s));
  k_tc_tables<<<2048, 256, 0, s>>>(N3, ntables, kNumOffsets, h->d_K_lap, h->d_K_yuk,
                                   h->m2l_rank > 0 ? h->d_C : nullptr, d_table_level,
                                   reinterpret_cast<__nv_bfloat16 *>(h->d_tc_tiles));
  AFMPB_TRY(check_launch("k_tc_tables"));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  A.release(d_table_level);
  AFMPB_TRY(raise_smem_limit((const void *)k_m2l_tc, kTcSmem));
  return Err{};
}

Err enqueue_m2l_tc(afmpb_t *h, cudaStream_t s) {
  if (m2l_ts_applies(h)) return enqueue_m2l_ts(h, s);
  if (h->tc_items == 0) return Err{};
  const bool comp = h->m2l_rank > 0;
  const int N3 = comp ? h->m2l_rank : h->ncoef;
  dim3 grid((unsigned)h->tc_items, (N3 + kTcRows - 1) / kTcRows, 2);
  k_m2l_tc<<<grid, kTcThreads, kTcSmem, s>>>(N3, h->d_tc_items, h->d_m2l_groups, h->d_m2l_pairs,
                                             reinterpret_cast<const __nv_bfloat16 *>(h->d_tc_tiles),
                                             h->d_tc_level_table, kNumOffsets, h->m2l_yuk_levels,
                                             h->d_box_center, comp ? h->d_Mc : h->d_M, comp ? h->d_Lc : h->d_L,
                                             h->d_tc_flag, comp ? h->d_table_rank : nullptr);
  return check_launch("k_m2l_tc");
}

// The bounded wait run on purpose: an mbarrier expecting one arrival that never comes.
__global__ void k_wait_selftest(uint32_t limit, int *flag) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t mb = cvta_smem(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
  asm volatile("fence.mbarrier_init.release.cluster;");
  if (!mbar_wait(mb, 0, limit)) atomicExch(flag, 1);
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb));
}

Err selftest_bounded_wait(int spin_limit, int *expired) {
  cudaStream_t s = nullptr;
  AFMPB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct Guard {
    cudaStream_t s;
    int *d = nullptr;
    ~Guard() {
      if (d) cudaFree(d);
      cudaStreamDestroy(s);
    }
  } g{s};
  AFMPB_CUDA(cudaMalloc(&g.d, sizeof(int)));
  AFMPB_CUDA(cudaMemsetAsync(g.d, 0, sizeof(int), s));
  k_wait_selftest<<<1, 1, 0, s>>>((uint32_t)spin_limit, g.d);
  AFMPB_TRY(check_launch("k_wait_selftest"));
  AFMPB_CUDA(cudaMemcpyAsync(expired, g.d, sizeof(int), cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  return Err{};
}

// The flag lives in mapped pinned host memory: kernels write it through its device alias
// only when a wait expires, and the host reads it without a copy once the work is done.
Err alloc_wait_flag(afmpb_t *h) {
  if (h->h_wait_flag) return Err{};
  void *p = nullptr;
  cudaError_t e = cudaHostAlloc(&p, sizeof(int), cudaHostAllocMapped);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return make_err(AFMPB_ENOMEM, std::string("cudaHostAlloc (wait flag): ") + cudaGetErrorString(e));
  }
  h->h_wait_flag = static_cast<int *>(p);
  *h->h_wait_flag = 0;
  void *d = nullptr;
  AFMPB_CUDA(cudaHostGetDevicePointer(&d, p, 0));
  h->d_tc_flag = static_cast<int *>(d);
  return Err{};
}

Err read_tc_error(afmpb_t *h, int *flag) {
  *flag = 0;
  if (!h->h_wait_flag) return Err{};
  AFMPB_CUDA(cudaStreamSynchronize(h->stream));
  volatile int *f = h->h_wait_flag;
  if (*f) {
    *flag = 1;
    *f = 0;
  }
  return Err{};
}

}  // namespace afmpb
