// Seeded synthetic CSR generator: meshes and R-MAT graphs.
//
// Input side only: this file draws graphs and builds CSR arrays. It holds no
// traversal arithmetic (levels, distances, labels) and is shared by the CUDA
// path and the CPU oracle only through the arrays it writes.
//
// All randomness is counter-based (SplitMix64 mixing keyed by seed, stream,
// index), so results are identical for any thread count and on any host.
#include "../../include/irgl_gen.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <thread>
#include <unordered_set>
#include <vector>

namespace {

// SplitMix64 output mixing (Vigna, public domain definition).
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ULL;

inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t index) {
  uint64_t key = mix64(mix64(seed + kGolden) ^ (stream * 0xd1b54a32d192ed03ULL + 0x632be59bd9b4e019ULL));
  return mix64(key + (index + 1) * kGolden);
}

// Stream ids (one per independent decision family).
enum : uint64_t {
  kStreamPerm = 1,
  kStreamWeight = 2,
  kStreamDelete = 3,
  kStreamExtraVertex = 4,
  kStreamExtraOffset = 5,
  kStreamRmatLevel = 1000,  // + level/2
};

inline int32_t weight_of(uint64_t seed, uint32_t u, uint32_t v) {
  return 1 + static_cast<int32_t>(draw(seed, kStreamWeight, (static_cast<uint64_t>(u) << 32) | v) % 100u);
}

int hw_threads(int n) {
  if (n > 0) return n;
  unsigned h = std::thread::hardware_concurrency();
  return h == 0 ? 4 : static_cast<int>(std::min(h, 64u));
}

template <class F>
void parallel_for(uint64_t n, int nthreads, F&& f) {
  nthreads = std::max(1, std::min<int>(nthreads, static_cast<int>((n + 65535) / 65536)));
  if (nthreads <= 1) { f(0, n); return; }
  std::vector<std::thread> ts;
  uint64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t lo = std::min<uint64_t>(n, t * chunk), hi = std::min<uint64_t>(n, lo + chunk);
    ts.emplace_back([&f, lo, hi] { f(lo, hi); });
  }
  for (auto& t : ts) t.join();
}

// Indices of the k smallest keys draw(seed, stream, i), i < n (ties by index), ascending by index.
std::vector<uint64_t> k_smallest(uint64_t n, uint64_t k, uint64_t seed, uint64_t stream) {
  std::vector<uint64_t> out;
  if (k == 0 || n == 0) return out;
  k = std::min(k, n);
  std::vector<std::pair<uint64_t, uint64_t>> keys(n);
  for (uint64_t i = 0; i < n; ++i) keys[i] = {draw(seed, stream, i), i};
  std::nth_element(keys.begin(), keys.begin() + (k - 1), keys.end());
  out.reserve(k);
  for (uint64_t i = 0; i < k; ++i) out.push_back(keys[i].second);
  std::sort(out.begin(), out.end());
  return out;
}

}  // namespace

extern "C" uint64_t irglgen_draw(uint64_t seed, uint64_t stream, uint64_t index) {
  return draw(seed, stream, index);
}

extern "C" int64_t irglgen_mesh(uint32_t rows, uint32_t cols, uint64_t seed, double del_frac,
                                double extra_frac, uint32_t radius, uint32_t* row_ptr, uint32_t* col,
                                int32_t* w, uint64_t cap) {
  if (rows == 0 || cols == 0 || !row_ptr || !col) return -1;
  if (del_frac < 0 || del_frac > 1 || extra_frac < 0 || extra_frac > 1) return -1;
  const uint64_t n = static_cast<uint64_t>(rows) * cols;
  if (n >= 0xFFFFFFFFull) return -1;
  try {
    // Undirected grid edge e: horizontal (r,c)-(r,c+1) at e = r*(cols-1)+c,
    // vertical (r,c)-(r+1,c) at e = H + r*cols + c.
    const uint64_t H = static_cast<uint64_t>(rows) * (cols - 1);
    const uint64_t E = H + static_cast<uint64_t>(rows - 1) * cols;
    std::vector<uint8_t> deleted(E, 0);
    const uint64_t k_del = static_cast<uint64_t>(std::llround(del_frac * static_cast<double>(E)));
    for (uint64_t e : k_smallest(E, k_del, seed, kStreamDelete)) deleted[e] = 1;

    auto h_edge = [&](uint32_t r, uint32_t c) { return static_cast<uint64_t>(r) * (cols - 1) + c; };
    auto v_edge = [&](uint32_t r, uint32_t c) { return H + static_cast<uint64_t>(r) * cols + c; };
    // Is the grid edge between neighbouring cells a and b present?
    auto grid_present = [&](uint32_t r0, uint32_t c0, uint32_t r1, uint32_t c1) -> bool {
      if (r0 == r1) return !deleted[h_edge(r0, std::min(c0, c1))];
      return !deleted[v_edge(std::min(r0, r1), c0)];
    };

    // Extra edges.
    std::vector<std::pair<int32_t, int32_t>> offsets;
    for (int32_t dr = -static_cast<int32_t>(radius); dr <= static_cast<int32_t>(radius); ++dr)
      for (int32_t dc = -static_cast<int32_t>(radius); dc <= static_cast<int32_t>(radius); ++dc)
        if ((dr != 0 || dc != 0) && std::abs(dr) + std::abs(dc) <= static_cast<int32_t>(radius))
          offsets.emplace_back(dr, dc);
    const uint64_t k_extra = static_cast<uint64_t>(std::llround(extra_frac * static_cast<double>(n)));
    std::vector<std::pair<uint32_t, uint32_t>> extra;  // (min, max)
    if (k_extra > 0 && !offsets.empty()) {
      std::unordered_set<uint64_t> have;
      for (uint64_t v : k_smallest(n, k_extra, seed, kStreamExtraVertex)) {
        const uint32_t r = static_cast<uint32_t>(v / cols), c = static_cast<uint32_t>(v % cols);
        for (uint64_t t = 0; t < 4096; ++t) {
          const auto& o = offsets[draw(seed, kStreamExtraOffset, v * 4096 + t) % offsets.size()];
          const int64_t r2 = static_cast<int64_t>(r) + o.first, c2 = static_cast<int64_t>(c) + o.second;
          if (r2 < 0 || c2 < 0 || r2 >= rows || c2 >= cols) continue;
          const uint32_t u2 = static_cast<uint32_t>(r2 * cols + c2);
          const uint32_t lo = std::min<uint32_t>(static_cast<uint32_t>(v), u2);
          const uint32_t hi = std::max<uint32_t>(static_cast<uint32_t>(v), u2);
          const uint64_t key = (static_cast<uint64_t>(lo) << 32) | hi;
          if (have.count(key)) continue;
          if (std::abs(o.first) + std::abs(o.second) == 1 &&
              grid_present(r, c, static_cast<uint32_t>(r2), static_cast<uint32_t>(c2)))
            continue;
          have.insert(key);
          extra.emplace_back(lo, hi);
          break;
        }
      }
    }

    // Degrees.
    std::vector<uint32_t> deg(n, 0);
    for (uint32_t r = 0; r < rows; ++r)
      for (uint32_t c = 0; c < cols; ++c) {
        uint32_t d = 0;
        if (r > 0 && grid_present(r - 1, c, r, c)) ++d;
        if (c > 0 && grid_present(r, c - 1, r, c)) ++d;
        if (c + 1 < cols && grid_present(r, c, r, c + 1)) ++d;
        if (r + 1 < rows && grid_present(r, c, r + 1, c)) ++d;
        deg[static_cast<uint64_t>(r) * cols + c] = d;
      }
    for (auto& e : extra) { ++deg[e.first]; ++deg[e.second]; }
    uint64_t m = 0;
    row_ptr[0] = 0;
    for (uint64_t v = 0; v < n; ++v) {
      m += deg[v];
      if (m > 0xFFFFFFFFull) return -1;
      row_ptr[v + 1] = static_cast<uint32_t>(m);
    }
    if (m > cap) return -2;

    // Fill rows: grid neighbours in increasing id order, then extras, then sort.
    std::vector<uint32_t> fill(n, 0);
    for (uint32_t r = 0; r < rows; ++r)
      for (uint32_t c = 0; c < cols; ++c) {
        const uint64_t v = static_cast<uint64_t>(r) * cols + c;
        uint32_t* out = col + row_ptr[v];
        uint32_t k = 0;
        if (r > 0 && grid_present(r - 1, c, r, c)) out[k++] = static_cast<uint32_t>(v - cols);
        if (c > 0 && grid_present(r, c - 1, r, c)) out[k++] = static_cast<uint32_t>(v - 1);
        if (c + 1 < cols && grid_present(r, c, r, c + 1)) out[k++] = static_cast<uint32_t>(v + 1);
        if (r + 1 < rows && grid_present(r, c, r + 1, c)) out[k++] = static_cast<uint32_t>(v + cols);
        fill[v] = k;
      }
    for (auto& e : extra) {
      col[row_ptr[e.first] + fill[e.first]++] = e.second;
      col[row_ptr[e.second] + fill[e.second]++] = e.first;
    }
    if (!extra.empty()) {
      std::vector<uint8_t> touched(n, 0);
      for (auto& e : extra) touched[e.first] = touched[e.second] = 1;
      for (uint64_t v = 0; v < n; ++v)
        if (touched[v]) std::sort(col + row_ptr[v], col + row_ptr[v + 1]);
    }
    if (w) {
      for (uint64_t v = 0; v < n; ++v)
        for (uint32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
          const uint32_t u2 = col[e];
          w[e] = weight_of(seed, std::min<uint32_t>(static_cast<uint32_t>(v), u2),
                           std::max<uint32_t>(static_cast<uint32_t>(v), u2));
        }
    }
    return static_cast<int64_t>(m);
  } catch (const std::bad_alloc&) {
    return -3;
  }
}

extern "C" int64_t irglgen_rmat(uint32_t scale, uint32_t ef, double a, double b, double c, uint64_t seed,
                                int nthreads, uint32_t* row_ptr, uint32_t* col, int32_t* w, uint64_t cap) {
  if (scale == 0 || scale > 31 || ef == 0 || !row_ptr || !col) return -1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
  const uint64_t n = 1ull << scale;
  const uint64_t S = static_cast<uint64_t>(ef) * n;
  if (S > 0xFFFFFFFFull) return -1;
  nthreads = hw_threads(nthreads);
  try {
    // Seeded vertex permutation (Fisher-Yates driven by counter draws).
    std::vector<uint32_t> perm(n);
    for (uint64_t i = 0; i < n; ++i) perm[i] = static_cast<uint32_t>(i);
    for (uint64_t i = n - 1; i > 0; --i) {
      const uint64_t j = draw(seed, kStreamPerm, i) % (i + 1);
      std::swap(perm[i], perm[j]);
    }
    // Quadrant thresholds on a 32-bit uniform.
    const double two32 = 4294967296.0;
    auto thr = [&](double p) -> uint64_t { return static_cast<uint64_t>(std::floor(std::min(1.0, p) * two32)); };
    const uint64_t t_a = thr(a), t_ab = thr(a + b), t_abc = thr(a + b + c);

    std::vector<uint32_t> s_src(S), s_dst(S);
    parallel_for(S, nthreads, [&](uint64_t lo, uint64_t hi) {
      for (uint64_t i = lo; i < hi; ++i) {
        uint32_t u = 0, v = 0;
        uint64_t r64 = 0;
        for (uint32_t l = 0; l < scale; ++l) {
          if ((l & 1) == 0) r64 = draw(seed, kStreamRmatLevel + l / 2, i);
          const uint64_t r = (l & 1) ? (r64 >> 32) : (r64 & 0xFFFFFFFFull);
          uint32_t q = r < t_a ? 0u : (r < t_ab ? 1u : (r < t_abc ? 2u : 3u));
          u = (u << 1) | (q >> 1);
          v = (v << 1) | (q & 1u);
        }
        s_src[i] = perm[u];
        s_dst[i] = perm[v];
      }
    });
    perm.clear();
    perm.shrink_to_fit();

    // Count out-degrees (self-loops dropped), scatter, then sort+dedup rows.
    std::vector<std::atomic<uint32_t>> cnt(n);
    for (uint64_t v = 0; v < n; ++v) cnt[v].store(0, std::memory_order_relaxed);
    parallel_for(S, nthreads, [&](uint64_t lo, uint64_t hi) {
      for (uint64_t i = lo; i < hi; ++i)
        if (s_src[i] != s_dst[i]) cnt[s_src[i]].fetch_add(1, std::memory_order_relaxed);
    });
    std::vector<uint64_t> off(n + 1, 0);
    for (uint64_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v].load(std::memory_order_relaxed);
    const uint64_t S2 = off[n];
    for (uint64_t v = 0; v < n; ++v) cnt[v].store(0, std::memory_order_relaxed);
    std::vector<uint32_t> tmp(S2);
    parallel_for(S, nthreads, [&](uint64_t lo, uint64_t hi) {
      for (uint64_t i = lo; i < hi; ++i) {
        const uint32_t u = s_src[i], v = s_dst[i];
        if (u == v) continue;
        const uint32_t p = cnt[u].fetch_add(1, std::memory_order_relaxed);
        tmp[off[u] + p] = v;
      }
    });
    s_src.clear(); s_src.shrink_to_fit();
    s_dst.clear(); s_dst.shrink_to_fit();
    std::vector<uint32_t> ndeg(n, 0);
    parallel_for(n, nthreads, [&](uint64_t lo, uint64_t hi) {
      for (uint64_t v = lo; v < hi; ++v) {
        uint32_t* b = tmp.data() + off[v];
        uint32_t* e = tmp.data() + off[v + 1];
        std::sort(b, e);
        ndeg[v] = static_cast<uint32_t>(std::unique(b, e) - b);
      }
    });
    uint64_t m = 0;
    row_ptr[0] = 0;
    for (uint64_t v = 0; v < n; ++v) {
      m += ndeg[v];
      row_ptr[v + 1] = static_cast<uint32_t>(m);
    }
    if (m > cap) return -2;
    parallel_for(n, nthreads, [&](uint64_t lo, uint64_t hi) {
      for (uint64_t v = lo; v < hi; ++v) {
        std::memcpy(col + row_ptr[v], tmp.data() + off[v], sizeof(uint32_t) * ndeg[v]);
        if (w)
          for (uint32_t k = 0; k < ndeg[v]; ++k)
            w[row_ptr[v] + k] = weight_of(seed, static_cast<uint32_t>(v), tmp[off[v] + k]);
      }
    });
    return static_cast<int64_t>(m);
  } catch (const std::bad_alloc&) {
    return -3;
  }
}
