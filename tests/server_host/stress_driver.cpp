// Stress driver for the serving loop against the host-only stand-in (fake_device.cpp), meant
// to run under ThreadSanitizer: several client threads open sessions, feed them, finalize some
// and close them (often before the worker has admitted them), re-open the same shapes at once,
// and wait for every request. Exits 0 when every request completed with SPCA_OK and each
// finalized result matched its session's own rows.
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <thread>
#include <vector>

#include "spca.h"
#include "spca_server.h"

extern "C" void fake_set_delays(int64_t create_us, int64_t update_us, int64_t finalize_us);
extern "C" int64_t fake_live_sessions(void);

namespace {

const uint64_t kGold = 0x9E3779B97F4A7C15ull;

uint64_t digest_of(const std::vector<std::vector<float>>& blocks) {
  uint64_t h = 1469598103934665603ull;
  for (const auto& b : blocks)
    for (float f : b) {
      uint32_t w;
      std::memcpy(&w, &f, 4);
      h ^= w;
      h *= 1099511628211ull;
    }
  return h;
}

double unit(uint64_t x) { return static_cast<double>(x >> 11) * (1.0 / 9007199254740992.0); }

std::atomic<int> g_failures{0};

void client(spca_server* sv, int idx, int iters) {
  std::mt19937_64 rng(1234 + idx);
  const int64_t n = 16;
  const int k = 3, p = 1;
  std::vector<std::vector<float>> keep;   // rows stay valid until their requests complete
  std::vector<uint64_t> tickets;
  keep.reserve(static_cast<size_t>(iters) * 2);
  for (int it = 0; it < iters; ++it) {
    const uint64_t seed = 100000ull * idx + it;
    int32_t id = -1;
    if (spca_server_open(sv, n, k, p, seed, &id) != SPCA_OK) {
      g_failures++;
      return;
    }
    std::vector<std::vector<float>> mine;
    const int nblocks = 1 + static_cast<int>(rng() % 3);
    for (int b = 0; b < nblocks; ++b) {
      const int64_t m = 1 + static_cast<int64_t>(rng() % 6);
      std::vector<float> rows(static_cast<size_t>(m * n));
      for (float& x : rows) x = static_cast<float>(static_cast<int64_t>(rng() % 2001) - 1000) / 64.0f;
      keep.push_back(rows);
      mine.push_back(rows);
      uint64_t t = 0;
      if (spca_server_update(sv, id, keep.back().data(), m, n, &t) != SPCA_OK) g_failures++;
      tickets.push_back(t);
    }
    if (it % 4 == 3) {
      std::vector<double> sig(k), V(static_cast<size_t>(n * k));
      uint64_t t = 0;
      if (spca_server_finalize(sv, id, sig.data(), V.data(), &t) != SPCA_OK || spca_server_wait(sv, t, 30.0) != SPCA_OK) {
        g_failures++;
      } else {
        const uint64_t h = digest_of(mine);
        for (int i = 0; i < k; ++i)
          if (sig[static_cast<size_t>(i)] != unit((h ^ seed) + static_cast<uint64_t>(i) * kGold)) g_failures++;
      }
    }
    spca_server_close(sv, id);
  }
  for (uint64_t t : tickets)
    if (spca_server_wait(sv, t, 30.0) != SPCA_OK) g_failures++;
}

}  // namespace

int main() {
  fake_set_delays(800, 20, 100);
  spca_server_options opt;
  spca_server_default_options(&opt);
  spca_server* sv = nullptr;
  if (spca_server_create(&opt, &sv) != SPCA_OK) return 2;
  std::vector<std::thread> th;
  for (int i = 0; i < 4; ++i) th.emplace_back(client, sv, i, 40);
  for (auto& t : th) t.join();
  spca_server_stats st;
  spca_server_get_stats(sv, &st);
  spca_server_destroy(sv);
  std::printf("failures %d created %lld from_pool %lld live_sessions %lld\n", g_failures.load(),
              static_cast<long long>(st.sessions_created), static_cast<long long>(st.admissions_from_pool),
              static_cast<long long>(fake_live_sessions()));
  return (g_failures.load() == 0 && fake_live_sessions() == 0) ? 0 : 1;
}
