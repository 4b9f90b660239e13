// bank_model.h - row strides of the row-pass shared-memory buffers, chosen
// by a model of the shared-memory banks (host code).
//
// A row block keeps, per row, an FFT scratch row and a staging row.  Several
// rows share a warp when a row has fewer than 32 threads, and the cooperative
// mixed I/O gives one warp min(rpc, 32) rows at once, so the distance between
// consecutive rows decides how a warp's accesses fall on the 32 banks.  The
// model counts, for every warp instruction of a block, the 128-byte
// wavefronts it needs: the largest number of the warp's accesses that land on
// one element slot modulo E = 128 B / sizeof(complex).  It follows the index
// formulas of fft.cuh (Stockham passes, padded by one complex per 16) and of
// the cooperative I/O in kernels.cuh (thread t serves row t % rpc and modes
// t / rpc + i blockDim / rpc).  For each launch shape the planner takes the
// smallest stride >= the row's length among the E candidates with the fewest
// wavefronts in all.
#pragma once

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace sbi {
namespace bank {

inline int pad16(int i) { return i + (i >> 4); }

struct Geometry {
  int n;        // complex length of a row (packed real FFT: nx / 2)
  int R;        // elements per thread
  int TPR;      // threads per row
  int rpc;      // rows per block
  int W;        // kept modes per row
  int E;        // element slots per 128-B wavefront
};

// Addresses (within one row) of every shared-memory instruction of a
// Stockham transform of length N by N/R threads: each entry maps the thread
// index j to an element index.  The last entry is the consumer's read of the
// natural-order result.  shuffled: the transform hands its last pass the data
// by warp shuffles and ends in registers (fft.cuh, kShuffleFft), so only the
// first pass's scatter and gather touch shared memory.
inline void stockham_pattern(int N, int R, std::vector<std::vector<int>>& ins, bool shuffled = false) {
  const int T = N / R;
  int Ls = 1;
  auto push = [&](auto f) {
    std::vector<int> a(T);
    for (int j = 0; j < T; ++j) a[j] = f(j);
    ins.push_back(a);
  };
  if (N == 1) return;
  if (shuffled) {
    for (int r = 0; r < R; ++r) push([&](int j) { return pad16(j * R) + pad16(r); });
    for (int r = 0; r < R; ++r) push([&](int j) { return pad16(j) + pad16(r * T); });
    return;
  }
  while (true) {
    if (N / Ls >= R) {
      for (int r = 0; r < R; ++r)
        push([&](int j) { const int k = j & (Ls - 1); return pad16((j - k) * R) + pad16(k) + pad16(r * Ls); });
      if (Ls * R < N) {
        for (int r = 0; r < R; ++r) push([&](int j) { return pad16(j) + pad16(r * T); });
        Ls *= R;
        continue;
      }
      break;
    }
    const int RP = N / Ls, Q = R / RP;
    for (int q = 0; q < Q; ++q)
      for (int m = 0; m < RP; ++m)
        push([&](int j) { return pad16(j) + pad16(q * T) + pad16(m * Ls); });
    break;
  }
  for (int r = 0; r < R; ++r) push([&](int j) { return pad16(j) + pad16(r * T); });
}

inline int wavefronts(const std::vector<int>& addr, int E) {
  std::vector<int> cnt(E, 0);
  int mx = 0;
  for (int a : addr) mx = std::max(mx, ++cnt[((a % E) + E) % E]);
  return mx;
}

// Wavefronts of the per-row (FFT) instructions over all warps of a block;
// shuffled: see stockham_pattern, plus the writes of the kept modes to the
// row (element k = j + r TPR < W, r2c_regs in kernels.cuh).
inline long long fft_cost(const Geometry& g, int S, bool shuffled = false) {
  std::vector<std::vector<int>> ins;
  stockham_pattern(g.n, g.R, ins, shuffled);
  if (shuffled) {
    for (int r = 0; r < g.R && r * g.TPR < g.W; ++r) {
      std::vector<int> a(g.TPR);
      for (int j = 0; j < g.TPR; ++j) a[j] = j + r * g.TPR < g.W ? j + r * g.TPR : -1;
      ins.push_back(a);
    }
  }
  const int threads = g.rpc * g.TPR;
  long long tot = 0;
  for (int w = 0; w * 32 < threads; ++w) {
    for (const auto& f : ins) {
      std::vector<int> addr;
      for (int t = 32 * w; t < std::min(threads, 32 * w + 32); ++t) {
        const int row = t / g.TPR, j = t % g.TPR;
        if (f[j] >= 0) addr.push_back(row * S + f[j]);
      }
      if (!addr.empty()) tot += wavefronts(addr, g.E);
    }
  }
  return tot;
}

// Wavefronts of the cooperative I/O over a block: `f(rl, k)` is the element a
// thread serving row rl and mode k < W touches (nothing when it returns < 0).
template <class F>
long long coop_cost(const Geometry& g, F f) {
  const int threads = g.rpc * g.TPR, kstep = threads / g.rpc;
  long long tot = 0;
  for (int w = 0; w * 32 < threads; ++w) {
    for (int it = 0; it * kstep < g.W; ++it) {
      std::vector<int> addr;
      for (int t = 32 * w; t < std::min(threads, 32 * w + 32); ++t) {
        const int rl = t % g.rpc, k = t / g.rpc + it * kstep;
        if (k >= g.W) continue;
        const int a = f(rl, k);
        if (a >= 0) addr.push_back(a);
      }
      if (!addr.empty()) tot += wavefronts(addr, g.E);
    }
  }
  return tot;
}

// Reads of a staged row by the row's own threads in the packed inverse real
// FFT (c2r_input): elements k and n - k (when < W) for k = j + r TPR.
inline long long c2r_cost(const Geometry& g, int S) {
  const int threads = g.rpc * g.TPR;
  long long tot = 0;
  for (int w = 0; w * 32 < threads; ++w) {
    for (int r = 0; r < g.R; ++r) {
      std::vector<int> a1, a2;
      for (int t = 32 * w; t < std::min(threads, 32 * w + 32); ++t) {
        const int row = t / g.TPR, j = t % g.TPR, k = j + r * g.TPR, kk = g.n - k;
        if (k < g.W) a1.push_back(row * S + k);
        if (k > 0 && kk < g.W) a2.push_back(row * S + kk);
      }
      if (!a1.empty()) tot += wavefronts(a1, g.E);
      if (!a2.empty()) tot += wavefronts(a2, g.E);
    }
  }
  return tot;
}

inline int best_stride(int len, int E, const std::function<long long(int)>& cost) {
  int best = len;
  long long bc = -1;
  for (int S = len; S < len + E; ++S) {
    const long long c = cost(S);
    if (bc < 0 || c < bc) {
      bc = c;
      best = S;
    }
  }
  return best;
}

// Strides of a row pass (k_row): the FFT scratch (FFT + the forward output's
// cooperative reads of k and n - k) and the staging rows (the cooperative
// copies in + the packed inverse's reads).  rk = true: the RK stage pass,
// which stages into the scratch rows themselves.
struct RowStrides {
  int fbs, sws;
};

// shuffled: the row transforms end in registers (kShuffleFft); the forward
// outputs are then written per row and read back by the cooperative store
// one element each (no Z[k], Z[n-k] pair).  fb_min: the least FFT scratch
// row (the split transforms of fft.cuh need a little more than the padded
// length).  Rows of 32 threads or more never share a warp, so for them the
// transform's own accesses cost the same at every stride and only the
// cooperative copies decide.
inline RowStrides choose(int n, int R, int TPR, int rpc, int W, int elem_bytes, bool rk, bool shuffled,
                         int fb_min = 0) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int, int, bool, bool, int>, RowStrides> cache;
  const auto key = std::make_tuple(n, R, TPR, rpc, W, elem_bytes, rk, shuffled, fb_min);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const Geometry g{n, R, TPR, rpc, W, 128 / elem_bytes};
  const int fb_len = std::max(n + (n >> 4) + 1, fb_min);
  auto io_reads = [&](int S) {
    if (shuffled) return coop_cost(g, [&](int rl, int k) { return rl * S + k; });
    return coop_cost(g, [&](int rl, int k) { return rl * S + pad16(k); }) +
           coop_cost(g, [&](int rl, int k) { return rl * S + pad16((n - k) & (n - 1)); });
  };
  auto staging = [&](int S) {
    return coop_cost(g, [&](int rl, int k) { return rl * S + k; }) + c2r_cost(g, S);
  };
  RowStrides out{};
  if (rk) {
    out.fbs = best_stride(fb_len, g.E,
                          [&](int S) { return fft_cost(g, S, shuffled) + io_reads(S) + staging(S); });
    out.sws = 0;
  } else {
    out.fbs = best_stride(fb_len, g.E, [&](int S) { return fft_cost(g, S, shuffled) + io_reads(S); });
    out.sws = best_stride(std::max(W, 1), g.E, staging);
  }
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = out;
  return out;
}

}  // namespace bank
}  // namespace sbi
