// corner_csr.h -- node -> triangle-corner buckets of a triangle list, built on the host
// cores.  Plain C++ (no CUDA): shared by the mesh check and the geometry setup, and
// compiled on its own by the host tests.
#pragma once

#include <algorithm>
#include <cstdint>
#include <memory>
#include <thread>
#include <vector>

namespace afmpb {

// Host threads for a pass over nt triangles: at most 16, one per 65,536 triangles.
inline int corner_csr_threads(int64_t nt) {
  const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
  return (int)std::max<int64_t>(1, std::min<int64_t>({16, hw, nt / 65536 + 1}));
}

// Buckets the 3 nt corners of the triangle list tri[nt][3] by their node.  For node v,
// out[ptr[v] .. ptr[v + 1]) holds value(t, k) for every corner k of a triangle t that
// sits at v, in increasing t, then k: the order of one serial pass over the list.  Every
// node index must lie in [0, n).  ptr (n + 1 entries) and out (3 nt entries) are
// allocated here without initialisation: the threads that fill them touch their pages
// first, so the page faults of these large arrays are taken in parallel as well.
//
// A stable parallel counting sort in two levels.  Nodes are grouped in blocks of
// kBlock consecutive indices.  (1) Each thread takes a contiguous range of triangles and
// counts its corners per block; a prefix over (block, thread) gives every thread its own
// slot range inside each block's bucket.  (2) Each thread copies its corners, as (node,
// value) pairs in triangle order, into those slots: a bucket holds its corners in
// increasing t.  (3) Blocks are then split among the threads, and each block is counting-
// sorted by node in cache (kBlock counters), which keeps the triangle order inside a node.
// The result does not depend on the thread count.
template <class V>
void corner_csr(int64_t n, int64_t nt, const int32_t *tri, int threads, std::unique_ptr<int64_t[]> &ptr,
                std::unique_ptr<int32_t[]> &out, V value) {
  constexpr int64_t kBlock = 4096;
  const int64_t nb = (n + kBlock - 1) / kBlock;
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(threads, std::max<int64_t>(nt, 1)));
  ptr.reset(new int64_t[n + 1]);
  out.reset(new int32_t[3 * nt]);
  if (n == 0) {
    ptr[0] = 0;
    return;
  }
  auto run = [T](auto f) {
    std::vector<std::thread> pool;
    for (int p = 1; p < T; ++p) pool.emplace_back(f, p);
    f(0);
    for (auto &th : pool) th.join();
  };
  // (1) corner counts per (thread, block)
  std::vector<int64_t> slot((size_t)T * nb, 0);   // then: first slot of thread p in block b
  run([&](int p) {
    int64_t *c = slot.data() + (size_t)p * nb;
    for (int64_t e = 3 * (nt * p / T); e < 3 * (nt * (p + 1) / T); ++e) ++c[tri[e] / kBlock];
  });
  std::vector<int64_t> bstart(nb + 1, 0);
  {
    int64_t s = 0;
    for (int64_t b = 0; b < nb; ++b) {
      bstart[b] = s;
      for (int p = 0; p < T; ++p) {
        const int64_t c = slot[(size_t)p * nb + b];
        slot[(size_t)p * nb + b] = s;
        s += c;
      }
    }
    bstart[nb] = s;
  }
  // (2) (node, value) pairs into the block buckets, each thread in triangle order
  std::unique_ptr<int32_t[]> node(new int32_t[3 * nt]), val(new int32_t[3 * nt]);
  run([&](int p) {
    int64_t *cur = slot.data() + (size_t)p * nb;
    for (int64_t t = nt * p / T; t < nt * (p + 1) / T; ++t)
      for (int k = 0; k < 3; ++k) {
        const int32_t v = tri[3 * t + k];
        const int64_t i = cur[v / kBlock]++;
        node[i] = v;
        val[i] = value(t, k);
      }
  });
  // (3) stable counting sort of each block by node
  run([&](int p) {
    std::vector<int64_t> cnt(kBlock + 1);
    for (int64_t b = nb * p / T; b < nb * (p + 1) / T; ++b) {
      const int64_t v0 = b * kBlock, nv = std::min(kBlock, n - v0);
      std::fill(cnt.begin(), cnt.begin() + nv + 1, 0);
      for (int64_t i = bstart[b]; i < bstart[b + 1]; ++i) ++cnt[node[i] - v0 + 1];
      cnt[0] = bstart[b];
      for (int64_t j = 0; j < nv; ++j) cnt[j + 1] += cnt[j];
      for (int64_t j = 0; j < nv; ++j) ptr[v0 + j] = cnt[j];
      if (b == nb - 1) ptr[n] = cnt[nv];
      for (int64_t i = bstart[b]; i < bstart[b + 1]; ++i) out[cnt[node[i] - v0]++] = val[i];
    }
  });
}

}  // namespace afmpb
