// Randomised check of rplu::Arena (csrc/arena.h) against a brute-force byte map:
// blocks never overlap, stay inside the region and are aligned; freeing
// everything restores one free block; alloc fails only when no free run fits.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "arena.h"

int main() {
  const int64_t size = 1 << 20;
  rplu::Arena a(size);
  std::vector<char> used(size / rplu::Arena::kAlign, 0);
  struct B { int64_t off, bytes; };
  std::vector<B> live;
  std::mt19937_64 rng(7);
  for (int it = 0; it < 200000; ++it) {
    if (live.empty() || rng() % 3) {
      const int64_t bytes = 1 + (int64_t)(rng() % 20000);
      const int64_t off = a.alloc(bytes);
      const int64_t units = rplu::Arena::round_up(bytes) / rplu::Arena::kAlign;
      if (off < 0) {
        // no free run of `units` may exist
        int64_t run = 0, best = 0;
        for (char u : used) { run = u ? 0 : run + 1; best = run > best ? run : best; }
        if (best >= units) { printf("FAIL alloc refused with a fitting run\n"); return 1; }
        continue;
      }
      if (off % rplu::Arena::kAlign || off + units * rplu::Arena::kAlign > size) { printf("FAIL bounds\n"); return 1; }
      for (int64_t u = off / rplu::Arena::kAlign; u < off / rplu::Arena::kAlign + units; ++u) {
        if (used[u]) { printf("FAIL overlap\n"); return 1; }
        used[u] = 1;
      }
      live.push_back({off, bytes});
    } else {
      const size_t k = rng() % live.size();
      const B b = live[k];
      live[k] = live.back();
      live.pop_back();
      a.release(b.off, b.bytes);
      const int64_t units = rplu::Arena::round_up(b.bytes) / rplu::Arena::kAlign;
      for (int64_t u = b.off / rplu::Arena::kAlign; u < b.off / rplu::Arena::kAlign + units; ++u) used[u] = 0;
    }
    int64_t inuse = 0;
    if (it % 1000 == 0) {
      for (char u : used) inuse += u;
      if (inuse * rplu::Arena::kAlign != a.used()) { printf("FAIL used accounting\n"); return 1; }
    }
  }
  for (const B& b : live) a.release(b.off, b.bytes);
  if (a.used() != 0 || a.free_blocks() != 1 || a.largest_free() != size) { printf("FAIL final state\n"); return 1; }
  printf("ok\n");
  return 0;
}
