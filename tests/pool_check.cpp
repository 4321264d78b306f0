// Host test of the serving pool allocator (csrc/pool.h) against a brute-force
// model: a map of granules, each free or owned by one live block.  Random
// alloc/release sequences check, after every operation, that
//  - a successful alloc returns the lowest offset that starts a run of free
//    granules long enough (first fit in address order), granule-aligned and
//    inside the budget, and an alloc fails exactly when no such run exists;
//  - the free list equals the maximal free runs of the model (coalesced,
//    address-ordered) and used() equals the owned granules;
// and that releasing everything leaves one free block of the whole budget.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "pool.h"

using irk::PoolAllocator;

static int fail(const char* what, long long a, long long b) {
  std::printf("FAIL %s %lld %lld\n", what, a, b);
  return 1;
}

int main() {
  const size_t G = PoolAllocator::kGranule;
  std::mt19937_64 rng(12345);
  long long checked = 0;
  for (int trial = 0; trial < 40; ++trial) {
    const size_t ngran = 8 + rng() % 200;
    const size_t budget = ngran * G + rng() % G;  // ragged budget: rounded down
    PoolAllocator pool;
    pool.init(budget);
    if (pool.size() != ngran * G) return fail("size", (long long)pool.size(), (long long)(ngran * G));
    std::vector<int> owner(ngran, 0);  // 0 = free, else block id
    struct Live { size_t off, bytes, gran; int id; };
    std::vector<Live> live;
    int next_id = 1;
    for (int op = 0; op < 400; ++op) {
      const bool do_alloc = live.empty() || (rng() % 100) < 55;
      if (do_alloc) {
        const size_t bytes = 1 + rng() % (G * (1 + ngran / 4));
        const size_t need = (bytes + G - 1) / G;
        // model: lowest start of a free run of length >= need
        long long want = -1;
        for (size_t g = 0; g < ngran && want < 0;) {
          if (owner[g] != 0) { ++g; continue; }
          size_t e = g;
          while (e < ngran && owner[e] == 0) ++e;
          if (e - g >= need) want = (long long)g;
          g = e;
        }
        size_t off = 0;
        const bool ok = pool.alloc(bytes, &off);
        if (ok != (want >= 0)) return fail("alloc success", ok, want);
        if (ok) {
          if (off % G) return fail("alignment", (long long)off, 0);
          if ((long long)(off / G) != want) return fail("first fit", (long long)(off / G), want);
          if (off + need * G > pool.size()) return fail("inside budget", (long long)off, (long long)need);
          for (size_t g = off / G; g < off / G + need; ++g) owner[g] = next_id;
          live.push_back({off, bytes, need, next_id++});
        }
      } else {
        const size_t k = rng() % live.size();
        const Live b = live[k];
        live.erase(live.begin() + k);
        pool.release(b.off, b.bytes);
        for (size_t g = b.off / G; g < b.off / G + b.gran; ++g) {
          if (owner[g] != b.id) return fail("ownership", (long long)g, owner[g]);
          owner[g] = 0;
        }
      }
      // free list == maximal free runs of the model; used == owned granules
      std::vector<std::pair<size_t, size_t>> runs;
      size_t owned = 0;
      for (size_t g = 0; g < ngran;) {
        if (owner[g] != 0) { ++owned; ++g; continue; }
        size_t e = g;
        while (e < ngran && owner[e] == 0) ++e;
        runs.push_back({g * G, (e - g) * G});
        g = e;
      }
      const auto& fl = pool.free_blocks();
      if (fl.size() != runs.size()) return fail("free blocks", (long long)fl.size(), (long long)runs.size());
      size_t i = 0;
      for (const auto& kv : fl) {
        if (kv.first != runs[i].first || kv.second != runs[i].second)
          return fail("free run", (long long)kv.first, (long long)runs[i].first);
        ++i;
      }
      if (pool.used() != owned * G) return fail("used", (long long)pool.used(), (long long)(owned * G));
      if (pool.peak() < pool.used()) return fail("peak", (long long)pool.peak(), (long long)pool.used());
      ++checked;
    }
    for (const Live& b : live) pool.release(b.off, b.bytes);
    const auto& fl = pool.free_blocks();
    if (fl.size() != 1 || fl.begin()->first != 0 || fl.begin()->second != pool.size() || pool.used() != 0)
      return fail("all released", (long long)fl.size(), (long long)pool.used());
  }
  // a budget below one granule manages nothing; every alloc fails
  PoolAllocator tiny;
  tiny.init(G - 1);
  size_t off = 0;
  if (tiny.size() != 0 || tiny.alloc(1, &off)) return fail("tiny budget", (long long)tiny.size(), 0);
  std::printf("ok %lld states checked\n", checked);
  return 0;
}
