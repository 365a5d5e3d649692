// m2l_ts.cu -- compressed list-2 translations accumulated per target box on the 5th-
// generation tensor cores (precision mode 1, compressed ranks <= 112).
//
// The M2L of a level sums, for every target box b,   Lc[b] += sum_o C_o Mc[src(b, o)]
// over the offsets o of its list 2 (paper Sec. 3: the V-list translations of the FMM).
// Here a work item is a block of 128 consecutive target boxes of one level and one kernel
// (Laplace or Yukawa) with a range of its offsets (each offset's pairs form one run).  For each offset the source vectors of
// the targets that have a source there are gathered into the rows of the A operand (absent
// targets get zero rows), the translation C_o is the B operand, and
//      D[target, :] += A[target, :] C_o^T            (M = 128 targets, N = K = r)
// accumulates in tensor memory across all the offsets of the item (tcgen05.mma kind::f16,
// BF16 hi/lo split into hi*hi + hi*lo + lo*hi, FP32 accumulation).  The accumulator is
// read once per item and added into the targets' compressed local vectors: one write per
// target and item instead of one per translated pair.
//
// Warp roles (288 threads): warps 0-3 gather the A operand of the next offset (16-byte
// cp.async, zero fill for absent rows) while one thread brings C_o by bulk asynchronous
// copy; warp 8 issues the MMAs; warps 4-7 read the accumulator (tcgen05.ld, one target
// per lane) and add it into Lc.  Two operand stages and two accumulators let the gather of
// offset k + 1, the MMAs of offset k and the epilogue of the previous item overlap.  Every
// mbarrier wait is bounded: on expiry the CTA records the handle's error flag, lets its
// own MMAs drain (bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cub/cub.cuh>

#include <algorithm>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace afmpb {

constexpr int kTsRows = 128;                   // target boxes per block (MMA M, TMEM lanes)
constexpr int kTsThreads = 288;                // 4 gather warps, 4 epilogue warps, 1 MMA warp
constexpr int kTsMaxR = 112;                   // largest compressed rank this kernel takes
constexpr int kTsItemRuns = 32;                // most runs (offsets) in one item
constexpr int kTsItemEnt = 512;                // most entries (translated pairs) in one item

// B operand tiles: C_o split into BF16 hi / lo in the canonical K-major layout with R rows.
// out: [table][slot][hi, lo][R x R]
__global__ void k_ts_tables(int R, int ntables, const float *__restrict__ C, __nv_bfloat16 *__restrict__ out) {
  const int64_t per = (int64_t)R * R;
  const int64_t total = (int64_t)ntables * kNumOffsets * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = e / per;
    const int within = (int)(e % per);
    const int n = within / R, k = within % R;          // C_o[n][k]: output n, input k
    __nv_bfloat16 hi, lo;
    split_bf16(C[e], hi, lo);
    const uint32_t off = canon_off(n, k, R) >> 1;
    out[tile * 2 * per + off] = hi;
    out[tile * 2 * per + per + off] = lo;
  }
}

// (block, offset) key and (row, source) entry of every list-2 pair: key = global block *
// kNumOffsets + offset slot, entry = row << 32 | source box.
__global__ void k_ts_keys(const M2LGroup *__restrict__ groups, const int2 *__restrict__ pairs,
                          const int *__restrict__ lvl_start, const int *__restrict__ blk_start,
                          uint32_t *__restrict__ key, uint64_t *__restrict__ ent) {
  const M2LGroup g = groups[blockIdx.x];
  for (int j = threadIdx.x; j < g.count; j += blockDim.x) {
    const int2 pr = pairs[g.start + j];
    const int rel = pr.x - lvl_start[g.level];
    const int blk = blk_start[g.level] + rel / kTsRows;
    key[g.start + j] = (uint32_t)blk * kNumOffsets + (uint32_t)g.offset;
    ent[g.start + j] = ((uint64_t)(uint32_t)(rel % kTsRows) << 32) | (uint32_t)pr.y;
  }
}

__device__ __forceinline__ void ts_producer_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ bool ts_producer_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// With kBatch the items of several problems share the launch: item.req names the problem
// whose runs, entries, multipoles, tables and local expansions (reqs[item.req]) it uses,
// and the item count is read from *d_nitems (a list compacted to the running problems).
template <int NS, bool kBatch>
__global__ void __launch_bounds__(kTsThreads) k_m2l_ts(int R, int nitems_arg, const TSItem *__restrict__ items,
                                                      const int4 *__restrict__ runs_1,
                                                      const uint64_t *__restrict__ ent_1,
                                                      const __nv_bfloat16 *__restrict__ Mc16_1,
                                                      const __nv_bfloat16 *__restrict__ tiles_1,
                                                      float *__restrict__ Lc_1, int *__restrict__ err_flag,
                                                      const int *__restrict__ d_nitems,
                                                      const TSReq *__restrict__ reqs) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int nitems = kBatch ? *d_nitems : nitems_arg;
  auto runs_of = [&](const TSItem &it) -> const int4 * { return kBatch ? reqs[it.req].runs : runs_1; };
  auto ent_of = [&](const TSItem &it) -> const uint64_t * { return kBatch ? reqs[it.req].ent : ent_1; };
  auto mc_of = [&](const TSItem &it) -> const __nv_bfloat16 * {
    return kBatch ? reinterpret_cast<const __nv_bfloat16 *>(reqs[it.req].Mc16) : Mc16_1;
  };
  auto tiles_of = [&](const TSItem &it) -> const __nv_bfloat16 * {
    return kBatch ? reinterpret_cast<const __nv_bfloat16 *>(reqs[it.req].tiles) : tiles_1;
  };
  auto lc_of = [&](const TSItem &it) -> float * { return kBatch ? reqs[it.req].Lc : Lc_1; };
  // stage s: A hi, A lo (kTsRows x R each), B hi, B lo (R x R each)
  const uint32_t a_bytes = (uint32_t)(kTsRows * R * 2), b_bytes = (uint32_t)(R * R * 2);
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  const uint32_t s_base = cvta_smem(smem);
  __shared__ __align__(8) uint64_t bar_full[NS], bar_empty[NS], bar_accf[2], bar_acce[2];
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t s_old[NS][4], s_new[NS][4];        // rows present in each stage: last run, run being staged
  __shared__ __align__(16) int4 s_runs[2][kTsItemRuns];   // the runs and entries of two items, brought
  __shared__ __align__(16) uint64_t s_ent[2][kTsItemEnt + 2];   // in by bulk copy one item ahead
  __shared__ __align__(8) uint64_t bar_item[2];
  __shared__ int s_last;                                 // runs whose MMAs were committed (failure drain)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nitems + (int)gridDim.x - 1) / (int)gridDim.x;
  const int i0 = (int)blockIdx.x * per, i1 = min(nitems, i0 + per);
  if (i0 >= i1) return;                                  // uniform per CTA
  uint32_t mb_full[NS], mb_empty[NS], mb_accf[2], mb_acce[2];
  for (int b = 0; b < NS; ++b) {
    mb_full[b] = cvta_smem(&bar_full[b]);
    mb_empty[b] = cvta_smem(&bar_empty[b]);
  }
  for (int b = 0; b < 2; ++b) {
    mb_accf[b] = cvta_smem(&bar_accf[b]);
    mb_acce[b] = cvta_smem(&bar_acce[b]);
  }
  // two accumulators of R FP32 columns each, rounded up to a power of two >= 32
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(2 * R)) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cvta_smem(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < NS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_full[b]));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_empty[b]));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_accf[b]));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(mb_acce[b]));   // one arrival per epilogue warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cvta_smem(&bar_item[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_last = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  bool failed = false;

  if (warp < 4) {
    // ---- gather: the A operand of run k + 1 is staged while run k's MMAs are issued -----
    // Each run has at most one entry per target row (a target has one source per offset),
    // so producer thread t copies the row of the run's t-th entry.  A stage keeps the rows
    // of its last run: a 128-bit mask per stage records them, and a row that was present
    // and is not now is cleared, so rows that stay absent cost nothing.  The runs and
    // entries of an item are brought into shared memory by bulk copy one item ahead.
    const uint32_t mb_item[2] = {cvta_smem(&bar_item[0]), cvta_smem(&bar_item[1])};
    auto load_item = [&](int k, int b) {                 // thread 0: item k's runs and entries -> buffer b
      const TSItem it = items[k];
      const uint32_t rb = (uint32_t)(it.run1 - it.run0) * 16;
      const int a0 = it.ent0 & ~1;                       // 16-byte aligned start (entries are 8 bytes)
      const uint32_t eb = (uint32_t)(((it.ent1 - a0) + 1) & ~1) * 8;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the buffer done
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb_item[b]), "r"(rb + eb) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       cvta_smem(&s_runs[b][0])),
                   "l"(runs_of(it) + it.run0), "r"(rb), "r"(mb_item[b])
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       cvta_smem(&s_ent[b][0])),
                   "l"(ent_of(it) + a0), "r"(eb), "r"(mb_item[b])
                   : "memory");
    };
    int issued = -1, waited = -1;                        // item positions loaded / waited for (thread 0 issues)
    if (threadIdx.x == 0) {
      load_item(i0, 0);
      issued = 0;
      if (i0 + 1 < i1) {
        load_item(i0 + 1, 1);
        issued = 1;
      }
    }
    // cursor over this CTA's runs
    int c_it = i0, c_k = 0;                              // item, its position among this CTA's items
    TSItem c_item = items[i0];
    int c_r = c_item.run0;
    if (!ts_producer_all(mbar_wait(mb_item[0], 0))) failed = true;
    waited = 0;
    auto stage_run = [&](int s) {                        // stage run (c_item, c_r) into stage s
      const int b = c_k & 1;
      const int4 run = s_runs[b][c_r - c_item.run0];     // (offset slot, first entry, end entry, -)
      const uint32_t st = s_base + (uint32_t)s * stage_bytes;
      if (threadIdx.x == 0) {
        // C_o of the item's table: hi and lo tiles, counted on the stage's full barrier
        const __nv_bfloat16 *src = tiles_of(c_item) + ((size_t)c_item.table * kNumOffsets + run.x) * 2 * R * R;
        asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(mb_full[s]), "r"(2 * b_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                st + 2 * a_bytes),
            "l"(src), "r"(b_bytes), "r"(mb_full[s])
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                st + 2 * a_bytes + b_bytes),
            "l"(src + R * R), "r"(b_bytes), "r"(mb_full[s])
            : "memory");
      }
      const int e = run.y + (int)threadIdx.x;
      const bool have = e < run.z;
      const uint64_t v = have ? s_ent[b][(c_item.ent0 & 1) + (e - c_item.ent0)] : 0ull;
      const int prow = (int)(v >> 32), psrc = (int)(uint32_t)v;
      if (have) atomicOr(&s_new[s][prow >> 5], 1u << (prow & 31));
      ts_producer_sync();
      const int row = threadIdx.x;
      const bool was = (s_old[s][row >> 5] >> (row & 31)) & 1u;
      const bool now = (s_new[s][row >> 5] >> (row & 31)) & 1u;
      if (have) {
        const int kg = c_item.rank / 8;                  // 16-byte groups along K that the MMAs read
        const __nv_bfloat16 *g = mc_of(c_item) + ((size_t)psrc * 2 + c_item.kt) * 2 * R;
        for (int k8 = 0; k8 < kg; ++k8) {
          const uint32_t off = canon_off(prow, k8 * 8, kTsRows);
          cp_async16_zfill(st + off, g + k8 * 8, true);
          cp_async16_zfill(st + a_bytes + off, g + R + k8 * 8, true);
        }
      }
      if (was && !now) {
        for (int k8 = 0; k8 < R / 8; ++k8) {
          const uint32_t off = canon_off(row, k8 * 8, kTsRows);
          asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(st + off), "r"(0u) : "memory");
          asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(st + a_bytes + off), "r"(0u) : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      ts_producer_sync();                                // every thread has read the masks and its entry
      if (threadIdx.x < 4) {
        s_old[s][threadIdx.x] = s_new[s][threadIdx.x];
        s_new[s][threadIdx.x] = 0u;
      }
    };
    auto advance = [&]() -> bool {                       // next run of this CTA; false at the end
      if (++c_r < c_item.run1) return true;
      // item c_k is fully staged: its buffer takes item c_k + 2
      if (threadIdx.x == 0 && c_it + 2 < i1) {
        load_item(c_it + 2, c_k & 1);
        issued = c_k + 2;
      }
      if (++c_it >= i1) return false;
      ++c_k;
      c_item = items[c_it];
      c_r = c_item.run0;
      if (!ts_producer_all(mbar_wait(mb_item[c_k & 1], (uint32_t)((c_k >> 1) & 1)))) failed = true;
      waited = c_k;
      return !failed;
    };
    // the stages start all zero (no row present)
    if (threadIdx.x < 4 * NS) {
      (&s_old[0][0])[threadIdx.x] = 0u;
      (&s_new[0][0])[threadIdx.x] = 0u;
    }
    for (uint32_t o = threadIdx.x * 16; o < NS * stage_bytes; o += 128 * 16)
      asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(s_base + o), "r"(0u) : "memory");
    ts_producer_sync();
    if (!failed) {
      // runs are staged up to NS - 1 ahead of the MMAs: run `use` is announced as soon as
      // its copies have landed, then run use + NS - 1 is staged into the stage that run
      // use - 1 read
      int staged = 0;
      bool more = true;
      for (; staged < NS - 1 && more; ++staged) {
        stage_run(staged % NS);
        more = advance();
      }
      for (int use = 0; !failed; ++use) {
        const int s = use % NS;
        if (more) asm volatile("cp.async.wait_group %0;" ::"n"(NS - 2) : "memory");   // run `use` has landed
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ts_producer_sync();
        if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb_full[s]) : "memory");
        if (more) {
          const int s1 = staged % NS;
          bool ok = true;
          if (staged >= NS) ok = mbar_wait(mb_empty[s1], (uint32_t)(((staged / NS) - 1) & 1));   // its last MMAs done
          if (!ts_producer_all(ok)) {
            failed = true;
            break;
          }
          stage_run(s1);
          ++staged;
          more = advance();
        }
        if (use + 1 >= staged) break;                    // every staged run is announced, none is left
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (threadIdx.x == 0)                                // after a failure: let issued item copies land (bounded)
      for (int k = waited + 1; k <= issued; ++k) mbar_wait(mb_item[k & 1], (uint32_t)((k >> 1) & 1));
  } else if (warp == 8) {
    // ---- MMA issue (one thread) ----------------------------------------------------------
    if (lane == 0) {
      int use = 0, committed = 0;
      const uint32_t lbo_a = (kTsRows / 8) * 128, lbo_b = (uint32_t)(R / 8) * 128, sbo = 128;
      for (int it = i0, k = 0; it < i1 && !failed; ++it, ++k) {
        const TSItem item = items[it];
        const int a = k & 1;
        if (k >= 2 && !mbar_wait(mb_acce[a], (uint32_t)(((k >> 1) - 1) & 1))) {   // epilogue of item k - 2 read it
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t acc = tmem + (uint32_t)(a * R);
        const uint32_t idesc = instr_desc(kTsRows, R);
        for (int r = item.run0; r < item.run1; ++r, ++use) {
          const int s = use % NS;
          if (!mbar_wait(mb_full[s], (uint32_t)((use / NS) & 1))) {
            failed = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t st = s_base + (uint32_t)s * stage_bytes;
          const uint32_t sa_hi = st, sa_lo = st + a_bytes, sb_hi = st + 2 * a_bytes, sb_lo = sb_hi + b_bytes;
          for (int q = 0; q < item.rank / 16; ++q) {
            const uint32_t ka = 2 * q * lbo_a, kb = 2 * q * lbo_b;
            const uint64_t dah = smem_desc(sa_hi + ka, lbo_a, sbo), dal = smem_desc(sa_lo + ka, lbo_a, sbo);
            const uint64_t dbh = smem_desc(sb_hi + kb, lbo_b, sbo), dbl = smem_desc(sb_lo + kb, lbo_b, sbo);
            const uint32_t first = (r == item.run0 && q == 0) ? 0u : 1u;      // 0: overwrite the accumulator
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                "l"(dah), "l"(dbh), "r"(idesc), "r"(first));
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
          }
          // the stage is free once these MMAs have read it
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mb_empty[s]));
          committed = use + 1;
        }
        if (failed) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            mb_accf[a]));
      }
      s_last = committed;
    }
    failed = __shfl_sync(0xffffffffu, failed, 0);
  } else {
    // ---- epilogue: one target box per lane ------------------------------------------------
    const int ew = warp - 4;
    const int row = 32 * ew + lane;
    for (int it = i0, k = 0; it < i1; ++it, ++k) {
      const TSItem item = items[it];
      const int a = k & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(mb_accf[a], (uint32_t)((k >> 1) & 1)));
      if (!ok) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int box = item.base + row;
      const bool valid = box < item.end;
      float *out = lc_of(item) + ((size_t)(valid ? box : 0) * 2 + item.kt) * R;
      for (int c0 = 0; c0 < item.rank; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(a * R + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (valid) {
          const float sc = item.scale;
#pragma unroll
          for (int q = 0; q < 16; q += 4)
            red_add_v4(out + c0 + q, __uint_as_float(v[q]) * sc, __uint_as_float(v[q + 1]) * sc,
                       __uint_as_float(v[q + 2]) * sc, __uint_as_float(v[q + 3]) * sc);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb_acce[a]) : "memory");
    }
  }
  if (failed && lane == 0) atomicExch(err_flag, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x == 0) {
    // bounded: the last committed MMA group has read its stage before the memory goes
    const int last = s_last;
    if (last > 0) mbar_wait(mb_empty[(last - 1) % NS], (uint32_t)(((last - 1) / NS) & 1));
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

namespace {
int ts_stage_bytes(int R) { return 2 * kTsRows * R * 2 + 2 * R * R * 2; }   // A hi, lo + B hi, lo
// Two operand stages, two CTAs per SM (R <= 64): measured on the 163,842-node sphere,
// 120 us against 188 us with four stages on one CTA per SM
int ts_stages(int) { return 2; }
int ts_smem_bytes(int R) { return ts_stages(R) * ts_stage_bytes(R); }
}  // namespace

bool m2l_ts_applies(const afmpb_t *h) { return h->m2l_rank > 0 && h->m2l_rank <= kTsMaxR && h->d_Mc16; }

// Work of the kernel: the list-2 entries re-sorted by (target block, offset) on the device,
// the runs of equal keys, and items of at most `per_item` runs of one block and one kernel.
Err build_m2l_ts(afmpb_t *h) {
  const std::vector<int> &level_table = h->h_level_table;
  const int R = h->m2l_rank;
  auto &A = h->arena;
  cudaStream_t s = h->stream;
  const auto &T = h->shape;
  const int64_t np = h->n_m2l_pairs;
  h->ts_nitems = 0;
  if (np == 0 || h->m2l_groups.empty()) return Err{};
  // global block index of each level's first block of kTsRows boxes
  std::vector<int> blk_start(T.nlevel + 1, 0);
  for (int l = 0; l < T.nlevel; ++l)
    blk_start[l + 1] = blk_start[l] + (T.lvl_start[l + 1] - T.lvl_start[l] + kTsRows - 1) / kTsRows;
  int *d_lvl = nullptr, *d_blk = nullptr;
  uint32_t *key = nullptr, *key_sorted = nullptr, *uniq = nullptr;
  uint64_t *ent = nullptr;
  int32_t *cnt = nullptr, *d_nruns = nullptr;
  AFMPB_TRY(A.alloc(&d_lvl, T.lvl_start.size(), "ts level start"));
  AFMPB_TRY(A.alloc(&d_blk, blk_start.size(), "ts block start"));
  AFMPB_TRY(A.alloc(&key, np, "ts keys"));
  AFMPB_TRY(A.alloc(&key_sorted, np, "ts keys sorted"));
  AFMPB_TRY(A.alloc(&ent, np, "ts entries unsorted"));
  AFMPB_TRY(A.alloc(&h->d_ts_ent, np + 2, "ts entries"));   // +2: 16-byte rounded item copies
  AFMPB_TRY(A.alloc(&uniq, np, "ts run keys"));
  AFMPB_TRY(A.alloc(&cnt, np, "ts run sizes"));
  AFMPB_TRY(A.alloc(&d_nruns, 1, "ts run count"));
  AFMPB_CUDA(cudaMemcpyAsync(d_lvl, T.lvl_start.data(), sizeof(int) * T.lvl_start.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaMemcpyAsync(d_blk, blk_start.data(), sizeof(int) * blk_start.size(), cudaMemcpyHostToDevice, s));
  k_ts_keys<<<(unsigned)h->m2l_groups.size(), 256, 0, s>>>(h->d_m2l_groups, h->d_m2l_pairs, d_lvl, d_blk, key, ent);
  AFMPB_TRY(check_launch("k_ts_keys"));
  int bits = 1;
  while (((uint64_t)1 << bits) < (uint64_t)blk_start.back() * kNumOffsets) ++bits;
  {
    size_t bytes = 0;
    AFMPB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, key, key_sorted, ent, h->d_ts_ent, np, 0, bits, s));
    uint8_t *tmp = nullptr;
    AFMPB_TRY(A.alloc(&tmp, std::max<size_t>(bytes, 16), "ts sort scratch"));
    AFMPB_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, key, key_sorted, ent, h->d_ts_ent, np, 0, bits, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
    A.release(tmp);
    bytes = 0;
    AFMPB_CUDA(cub::DeviceRunLengthEncode::Encode(nullptr, bytes, key_sorted, uniq, cnt, d_nruns, np, s));
    AFMPB_TRY(A.alloc(&tmp, std::max<size_t>(bytes, 16), "ts encode scratch"));
    AFMPB_CUDA(cub::DeviceRunLengthEncode::Encode(tmp, bytes, key_sorted, uniq, cnt, d_nruns, np, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
    A.release(tmp);
  }
  int32_t nruns = 0;
  AFMPB_CUDA(cudaMemcpyAsync(&nruns, d_nruns, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  std::vector<uint32_t> rkey(nruns);
  std::vector<int32_t> rcnt(nruns);
  AFMPB_CUDA(cudaMemcpyAsync(rkey.data(), uniq, sizeof(uint32_t) * nruns, cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaMemcpyAsync(rcnt.data(), cnt, sizeof(int32_t) * nruns, cudaMemcpyDeviceToHost, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  for (void *q : {(void *)d_lvl, (void *)d_blk, (void *)key, (void *)key_sorted, (void *)ent, (void *)uniq,
                  (void *)cnt, (void *)d_nruns})
    A.release(q);
  h->ts_rkey = std::move(rkey);
  h->ts_rcnt = std::move(rcnt);
  {
    // runs (offset slot, first entry, end entry)
    std::vector<int4> runs(nruns);
    int64_t e0 = 0;
    for (int r = 0; r < nruns; ++r) {
      runs[r] = make_int4((int)(h->ts_rkey[r] % kNumOffsets), (int)e0, (int)(e0 + h->ts_rcnt[r]), 0);
      e0 += h->ts_rcnt[r];
    }
    AFMPB_TRY(A.alloc(&h->d_ts_runs, std::max<size_t>(1, runs.size()), "ts runs"));
    AFMPB_CUDA(cudaMemcpyAsync(h->d_ts_runs, runs.data(), sizeof(int4) * runs.size(), cudaMemcpyHostToDevice, s));
    AFMPB_CUDA(cudaStreamSynchronize(s));
  }
  AFMPB_TRY(cut_m2l_ts_items(h));
  // B tiles from the compressed FP32 tables
  const size_t elems = (size_t)h->m2l_ntables * kNumOffsets * 2 * R * R;
  AFMPB_TRY(A.alloc(&h->d_ts_tiles, elems, "ts translation tiles"));
  k_ts_tables<<<2048, 256, 0, s>>>(R, h->m2l_ntables, h->d_C, reinterpret_cast<__nv_bfloat16 *>(h->d_ts_tiles));
  AFMPB_TRY(check_launch("k_ts_tables"));
  AFMPB_TRY(alloc_wait_flag(h));
  if (ts_stages(R) == 4) {
    AFMPB_TRY(raise_smem_limit((const void *)k_m2l_ts<4, false>, ts_smem_bytes(R)));
    AFMPB_TRY(raise_smem_limit((const void *)k_m2l_ts<4, true>, ts_smem_bytes(R)));
  } else {
    AFMPB_TRY(raise_smem_limit((const void *)k_m2l_ts<2, false>, ts_smem_bytes(R)));
    AFMPB_TRY(raise_smem_limit((const void *)k_m2l_ts<2, true>, ts_smem_bytes(R)));
  }
  AFMPB_CUDA(cudaStreamSynchronize(s));
  return Err{};
}

// Items over the stored runs: consecutive runs of one target block and one kernel, at most
// h->ts_runs_per_item runs (0: about four items per SM, at most kTsItemRuns) and kTsItemEnt
// entries each.  Replaces earlier items; the tile tuner calls it with other sizes.
Err cut_m2l_ts_items(afmpb_t *h) {
  auto &A = h->arena;
  cudaStream_t s = h->stream;
  const auto &T = h->shape;
  const std::vector<uint32_t> &rkey = h->ts_rkey;
  const std::vector<int32_t> &rcnt = h->ts_rcnt;
  const int nruns = (int)rkey.size();
  const std::vector<int> &level_table = h->h_level_table;
  std::vector<int> blk_start(T.nlevel + 1, 0);
  for (int l = 0; l < T.nlevel; ++l)
    blk_start[l + 1] = blk_start[l] + (T.lvl_start[l + 1] - T.lvl_start[l] + kTsRows - 1) / kTsRows;
  std::vector<int64_t> rstart(nruns + 1, 0);
  for (int r = 0; r < nruns; ++r) rstart[r + 1] = rstart[r] + rcnt[r];
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_item = h->ts_runs_per_item > 0 ? std::min(kTsItemRuns, h->ts_runs_per_item)
                                                : std::min(kTsItemRuns, std::max(8, nruns / std::max(1, 4 * sms)));
  std::vector<TSItem> items;
  auto level_of_block = [&](int blk) {
    int l = 0;
    while (l + 1 < (int)blk_start.size() && blk_start[l + 1] <= blk) ++l;
    return l;
  };
  for (int kt = 0; kt < 2; ++kt) {
    for (int r = 0; r < nruns;) {
      const int blk = (int)(rkey[r] / kNumOffsets);
      int rend = r;
      while (rend < nruns && (int)(rkey[rend] / kNumOffsets) == blk) ++rend;
      const int l = level_of_block(blk);
      const bool use = kt == 0 || (l >= h->m2l_yuk_levels && !h->laplace_only);
      if (use) {
        const int table = kt == 0 ? 0 : level_table[l];
        const int base = T.lvl_start[l] + (blk - blk_start[l]) * kTsRows;
        const int end = std::min(base + kTsRows, T.lvl_start[l + 1]);
        // consecutive runs of the block, at most per_item runs and kTsItemEnt entries each
        for (int q0 = r; q0 < rend;) {
          int q1 = q0, ne = 0;
          while (q1 < rend && q1 - q0 < per_item && ne + rcnt[q1] <= kTsItemEnt) ne += rcnt[q1++];
          TSItem it{};
          it.base = base;
          it.end = end;
          it.run0 = q0;
          it.run1 = q1;
          it.ent0 = (int)rstart[q0];
          it.ent1 = (int)rstart[q1];
          it.kt = kt;
          it.table = table;
          it.rank = h->h_table_rank[table];
          // Laplace tables are for the unit box: scale by 1 / w of the level
          it.scale = kt == 0 ? (float)(1.0 / std::ldexp(T.w0, -l)) : 1.0f;
          items.push_back(it);
          q0 = q1;
        }
      }
      r = rend;
    }
  }
  h->ts_nitems = (int)items.size();
  if (h->d_ts_items) A.release(h->d_ts_items);
  AFMPB_TRY(A.alloc(&h->d_ts_items, std::max<size_t>(1, items.size()), "ts items"));
  if (!items.empty())
    AFMPB_CUDA(cudaMemcpyAsync(h->d_ts_items, items.data(), sizeof(TSItem) * items.size(), cudaMemcpyHostToDevice, s));
  AFMPB_CUDA(cudaStreamSynchronize(s));
  return Err{};
}

Err enqueue_m2l_ts(afmpb_t *h, cudaStream_t s) {
  if (h->ts_nitems == 0) return Err{};
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int R = h->m2l_rank;
  const int per_sm = std::max(1, std::min(2, (227 * 1024) / (ts_smem_bytes(R) + 12 * 1024)));
  const unsigned grid = (unsigned)std::min(h->ts_nitems, per_sm * sms);
  const auto *mc = reinterpret_cast<const __nv_bfloat16 *>(h->d_Mc16);
  const auto *tl = reinterpret_cast<const __nv_bfloat16 *>(h->d_ts_tiles);
  if (ts_stages(R) == 4)
    k_m2l_ts<4, false><<<grid, kTsThreads, ts_smem_bytes(R), s>>>(R, h->ts_nitems, h->d_ts_items, h->d_ts_runs,
                                                                  h->d_ts_ent, mc, tl, h->d_Lc, h->d_tc_flag,
                                                                  nullptr, nullptr);
  else
    k_m2l_ts<2, false><<<grid, kTsThreads, ts_smem_bytes(R), s>>>(R, h->ts_nitems, h->d_ts_items, h->d_ts_runs,
                                                                  h->d_ts_ent, mc, tl, h->d_Lc, h->d_tc_flag,
                                                                  nullptr, nullptr);
  return check_launch("k_m2l_ts");
}

// The items of the running problems of a batch, in their order: one block scans the
// flags 1024 items at a time.
__global__ void __launch_bounds__(1024) k_ts_compact(int n, const TSItem *__restrict__ in, const TSReq *__restrict__ reqs,
                                                     TSItem *__restrict__ out, int *__restrict__ count) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += 1024) {
    const int i = c0 + (int)threadIdx.x;
    TSItem it{};
    int keep = 0;
    if (i < n) {
      it = in[i];
      const int *a = reqs[it.req].active;
      keep = (a == nullptr || *a != 0) ? 1 : 0;
    }
    int v = keep;                                        // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      s_warp[lane] = w;                                  // inclusive over warps
    }
    __syncthreads();
    const int before = s_base + (warp > 0 ? s_warp[warp - 1] : 0) + v - keep;
    if (keep) out[before] = it;
    __syncthreads();
    if (threadIdx.x == 0) s_base += s_warp[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = s_base;
}

Err enqueue_m2l_ts_batch(const TSReq *d_reqs, const TSItem *d_items, int nitems, TSItem *d_items_run, int *d_count,
                         int R, int *err_flag, cudaStream_t s) {
  if (nitems == 0) return Err{};
  int dev = 0, sms = 0;
  AFMPB_CUDA(cudaGetDevice(&dev));
  AFMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  k_ts_compact<<<1, 1024, 0, s>>>(nitems, d_items, d_reqs, d_items_run, d_count);
  AFMPB_TRY(check_launch("k_ts_compact"));
  const int per_sm = std::max(1, std::min(2, (227 * 1024) / (ts_smem_bytes(R) + 12 * 1024)));
  const unsigned grid = (unsigned)std::min(nitems, per_sm * sms);
  if (ts_stages(R) == 4)
    k_m2l_ts<4, true><<<grid, kTsThreads, ts_smem_bytes(R), s>>>(R, 0, d_items_run, nullptr, nullptr, nullptr,
                                                                 nullptr, nullptr, err_flag, d_count, d_reqs);
  else
    k_m2l_ts<2, true><<<grid, kTsThreads, ts_smem_bytes(R), s>>>(R, 0, d_items_run, nullptr, nullptr, nullptr,
                                                                 nullptr, nullptr, err_flag, d_count, d_reqs);
  return check_launch("k_m2l_ts batch");
}

}  // namespace afmpb
