// Host side of the codec: domain validation, the decode table (Sec. 3.3), the
// trainer of the prebuilt per-domain structures (Sec. 3.2.1, Sec. 3.3, Fig. 4)
// and the sequential single-pass encoder (Sec. 4.1, Alg. 1) that produces the
// streams the GPU decodes.  Plain C++17 on the CPU; no CUDA.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <thread>
#include <vector>

#include "fptc.h"
#include "fptc_codec.h"
#include "host_util.h"

namespace fptc {

namespace {
thread_local std::string g_error;
}

void set_error(const char *fmt, ...) noexcept {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  try {
    g_error = buf;
  } catch (...) {  // no memory for the text: keep the status, drop the message
    g_error.clear();
  }
}

void clear_error() noexcept { g_error.clear(); }

namespace {

// Cosine table of Eq. 1: cosv[k * N + n] = cos(pi (2n + 1) k / 2N).
std::vector<double> cos_table(uint32_t N, uint32_t E) {
  std::vector<double> t((size_t)N * E);
  for (uint32_t k = 0; k < E; ++k)
    for (uint32_t n = 0; n < N; ++n) t[(size_t)k * N + n] = std::cos(M_PI * (2.0 * n + 1.0) * k / (2.0 * N));
  return t;
}

// Eq. 1 of one zero-padded window, first E bins.
void forward_window(const float *x, uint64_t avail, uint32_t N, uint32_t E, const std::vector<double> &cosv,
                    double *C) {
  double xw[128];
  for (uint32_t n = 0; n < N; ++n) xw[n] = n < avail ? (double)x[n] : 0.0;
  for (uint32_t k = 0; k < E; ++k) {
    const double *row = cosv.data() + (size_t)k * N;
    double acc = 0.0;
    for (uint32_t n = 0; n < N; ++n) acc += xw[n] * row[n];
    C[k] = acc * (2.0 / N);
  }
}

struct Quantizer {
  double A0, A1, mu, alpha, log1pmu;
  uint32_t B1, B2;
  explicit Quantizer(const fptc_domain &d)
      : A0(d.scale[0]), A1(d.scale[1]), mu(d.mu), alpha(d.alpha1), log1pmu(std::log1p(d.mu)), B1(d.B1), B2(d.B2) {}

  // Eq. 2 with the level map 128 + round(127 q) / 128 - round(128 q)
  uint8_t zone0(double c) const {
    if (!(A0 > 1e-30) || std::isnan(c)) return 128;
    const double a = std::min(std::fabs(c), A0);
    const double q = std::log1p(mu * (a / A0)) / log1pmu;
    long v = c >= 0.0 ? 128 + (long)std::floor(127.0 * q + 0.5) : 128 - (long)std::floor(128.0 * q + 0.5);
    return (uint8_t)std::clamp(v, 0L, 255L);
  }
  // Eq. 3, |c| clamped to A1
  uint8_t zone1(double c) const {
    if (!(A1 > 1e-30) || std::isnan(c)) return 128;
    const double d1 = alpha * A1;
    const double m = std::min(std::fabs(c), A1);
    if (m <= d1) return 128;
    const double r = (m - d1) / (A1 - d1);
    long v = c > 0 ? 129 + (long)std::floor(r * 126.0 + 0.5) : 127 - (long)std::floor(r * 127.0 + 0.5);
    return (uint8_t)std::clamp(v, 0L, 255L);
  }
  uint8_t level(uint32_t k, double c) const { return k < B1 ? zone0(c) : (k < B2 ? zone1(c) : (uint8_t)128); }
};

// Length-limited optimal code lengths by package-merge (Larmore-Hirschberg).
// Every item carries the multiset of leaves it contains (counts per symbol);
// the code length of a symbol is its count over the cheapest 2n - 2 items of
// the final merged list.
bool package_merge(const uint64_t *freq, uint32_t lmax, uint8_t *len) {
  struct Item {
    uint64_t w;
    std::vector<uint16_t> cnt;  // per used symbol
  };
  std::vector<uint32_t> used;
  for (uint32_t s = 0; s < 256; ++s) {
    len[s] = 0;
    if (freq[s]) used.push_back(s);
  }
  const size_t n = used.size();
  if (n == 0) return true;
  if (n == 1) {
    len[used[0]] = 1;
    return true;
  }
  if (lmax < 16 && (size_t(1) << lmax) < n) return false;
  std::stable_sort(used.begin(), used.end(), [&](uint32_t a, uint32_t b) { return freq[a] < freq[b]; });
  std::vector<Item> leaves(n);
  for (size_t i = 0; i < n; ++i) {
    leaves[i].w = freq[used[i]];
    leaves[i].cnt.assign(n, 0);
    leaves[i].cnt[i] = 1;
  }
  std::vector<Item> cur = leaves;
  for (uint32_t level = 1; level < lmax; ++level) {
    std::vector<Item> pk;
    for (size_t i = 0; i + 1 < cur.size(); i += 2) {
      Item it;
      it.w = cur[i].w + cur[i + 1].w;
      it.cnt.resize(n);
      for (size_t j = 0; j < n; ++j) it.cnt[j] = (uint16_t)(cur[i].cnt[j] + cur[i + 1].cnt[j]);
      pk.push_back(std::move(it));
    }
    std::vector<Item> merged;
    merged.reserve(n + pk.size());
    size_t a = 0, b = 0;
    while (a < n || b < pk.size()) {
      if (b >= pk.size() || (a < n && leaves[a].w <= pk[b].w))
        merged.push_back(leaves[a++]);
      else
        merged.push_back(std::move(pk[b++]));
    }
    cur.swap(merged);
  }
  if (cur.size() < 2 * n - 2) return false;
  std::vector<uint32_t> total(n, 0);
  for (size_t i = 0; i < 2 * n - 2; ++i)
    for (size_t j = 0; j < n; ++j) total[j] += cur[i].cnt[j];
  for (size_t j = 0; j < n; ++j) len[used[j]] = (uint8_t)total[j];
  return true;
}

}  // namespace

// Total order of the non-NaN doubles as unsigned keys.
static uint64_t order_key(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return (u >> 63) ? ~u : u | 0x8000000000000000ull;
}
static double from_key(uint64_t k) {
  const uint64_t u = (k >> 63) ? k & 0x7fffffffffffffffull : ~k;
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}

void host_zone_bounds(const fptc_domain &d, uint32_t zone, double *bounds) {
  const Quantizer qz(d);
  auto level = [&](double c) -> uint32_t { return zone == 0 ? qz.zone0(c) : qz.zone1(c); };
  const double ninf = -std::numeric_limits<double>::infinity(), pinf = std::numeric_limits<double>::infinity();
  for (uint32_t L = 1; L <= 255; ++L) {
    if (level(ninf) >= L) {
      bounds[L - 1] = ninf;
    } else if (level(pinf) < L) {
      bounds[L - 1] = std::numeric_limits<double>::quiet_NaN();  // no double: never <= c
    } else {  // level(lo) < L <= level(hi): the smallest such key by bisection
      uint64_t lo = order_key(ninf), hi = order_key(pinf);
      while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (level(from_key(mid)) >= L)
          hi = mid;
        else
          lo = mid;
      }
      bounds[L - 1] = from_key(hi);
    }
  }
}

}  // namespace fptc

using namespace fptc;

extern "C" {

const char *fptc_last_error_message(void) { return g_error.c_str(); }

fptc_status fptc_validate_domain(const fptc_domain *d) {
  return guarded([&]() -> fptc_status {
    if (!d) {
      set_error("domain is NULL");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (d->N < 4 || d->N > 128) {
      set_error("N = %u outside [4, 128]", d->N);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (d->E < 1 || d->E > d->N) {
      set_error("E = %u outside [1, N]", d->E);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (d->B1 > d->B2 || d->B2 > d->E) {
      set_error("zone boundaries need 0 <= B1 <= B2 <= E (B1 = %u, B2 = %u)", d->B1, d->B2);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (!(d->mu > 0.0) || !std::isfinite(d->mu)) {
      set_error("mu must be positive");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (!(d->alpha1 >= 0.0 && d->alpha1 <= 1.0)) {
      set_error("alpha1 must lie in [0, 1]");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    for (int z = 0; z < 3; ++z) {
      if (!std::isfinite(d->scale[z]) || d->scale[z] < 0.0) {
        set_error("scale[%d] must be finite and >= 0", z);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
    }
    if (d->lmax < 1 || d->lmax > 16) {
      set_error("lmax = %u outside [1, 16]", d->lmax);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    uint64_t kraft = 0;
    int coded = 0;
    for (int s = 0; s < 256; ++s) {
      if (d->code_len[s] > d->lmax) {
        set_error("code length %u of level %d exceeds lmax %u", d->code_len[s], s, d->lmax);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
      if (d->code_len[s]) {
        kraft += uint64_t(1) << (d->lmax - d->code_len[s]);
        ++coded;
      }
    }
    if (coded == 0) {
      set_error("no level has a code");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (kraft > (uint64_t(1) << d->lmax)) {
      set_error("code lengths break the Kraft inequality");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    return FPTC_OK;
  });
}

fptc_status fptc_canonical_codes(const fptc_domain *d, uint32_t *codes) {
  return guarded([&]() -> fptc_status {
    fptc_status st = fptc_validate_domain(d);
    if (st != FPTC_OK) return st;
    uint32_t count[17] = {0};
    for (int s = 0; s < 256; ++s) count[d->code_len[s]]++;
    count[0] = 0;
    uint32_t first[17] = {0};
    uint32_t c = 0;
    for (uint32_t l = 1; l <= 16; ++l) {
      c = (c + count[l - 1]) << 1;
      first[l] = c;
    }
    for (int s = 0; s < 256; ++s) codes[s] = d->code_len[s] ? first[d->code_len[s]]++ : 0u;
    return FPTC_OK;
  });
}

fptc_status fptc_build_decode_table(const fptc_domain *d, uint16_t *table) {
  return guarded([&]() -> fptc_status {
    uint32_t codes[256];
    fptc_status st = fptc_canonical_codes(d, codes);
    if (st != FPTC_OK) return st;
    const uint32_t L = d->lmax;
    std::memset(table, 0, sizeof(uint16_t) << L);
    for (int s = 0; s < 256; ++s) {
      const uint32_t l = d->code_len[s];
      if (!l) continue;
      const uint32_t lo = codes[s] << (L - l), hi = (codes[s] + 1) << (L - l);
      for (uint32_t p = lo; p < hi; ++p) table[p] = (uint16_t)(s | (l << 8));
    }
    return FPTC_OK;
  });
}

fptc_status fptc_zone_bounds(const fptc_domain *d, uint32_t zone, double *bounds) {
  return guarded([&]() -> fptc_status {
    clear_error();
    if (!d || !bounds || zone > 1) {
      set_error("need a domain, zone 0 or 1 and room for 255 bounds");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    const fptc_status st = fptc_validate_domain(d);
    if (st != FPTC_OK) return st;
    host_zone_bounds(*d, zone, bounds);
    return FPTC_OK;
  });
}

uint64_t fptc_word_capacity(const fptc_domain *d, uint64_t S) {
  if (!d || d->N == 0 || d->lmax == 0) return 0;
  const uint64_t L = (S + d->N - 1) / d->N * d->E;
  const uint64_t per = std::max<uint64_t>(1, (65 - d->lmax + d->lmax - 1) / d->lmax);
  return L / per + 2;
}

fptc_status fptc_train_domain(const float *x, const uint64_t *offsets, const uint64_t *lengths, uint64_t n_signals,
                              double percentile, fptc_domain *d) {
  return guarded([&]() -> fptc_status {
    clear_error();
    if (!d || (n_signals && (!x || !offsets || !lengths))) {
      set_error("NULL argument");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (!(percentile > 0.0 && percentile <= 100.0)) {
      set_error("percentile must lie in (0, 100]");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    // validate the shape parameters with a placeholder complete code
    fptc_domain probe = *d;
    for (int s = 0; s < 256; ++s) probe.code_len[s] = 8;
    probe.scale[0] = probe.scale[1] = probe.scale[2] = 0.0;
    if (d->lmax < 8) probe.lmax = 8;
    fptc_status st = fptc_validate_domain(&probe);
    if (st != FPTC_OK) return st;
    if (d->lmax < 8) {
      set_error("lmax must be >= 8 to code 256 levels");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    const uint32_t N = d->N, E = d->E;
    const auto cosv = cos_table(N, E);
    std::vector<double> coef;
    for (uint64_t i = 0; i < n_signals; ++i) {
      const uint64_t S = lengths[i];
      const uint64_t W = (S + N - 1) / N;
      const size_t base = coef.size();
      coef.resize(base + W * E);
      for (uint64_t w = 0; w < W; ++w)
        forward_window(x + offsets[i] + w * N, S - w * N, N, E, cosv, coef.data() + base + w * E);
    }
    const uint64_t rows = coef.size() / E;
    for (int z = 0; z < 2; ++z) {
      const uint32_t k0 = z == 0 ? 0 : d->B1, k1 = z == 0 ? d->B1 : d->B2;
      std::vector<double> v;
      v.reserve(rows * (k1 - k0));
      for (uint64_t r = 0; r < rows; ++r)
        for (uint32_t k = k0; k < k1; ++k) v.push_back(std::fabs(coef[r * E + k]));
      double A = 0.0;
      if (!v.empty()) {
        long rank = (long)std::ceil(percentile / 100.0 * (double)v.size() - 1e-9);
        size_t idx = (size_t)std::clamp(rank - 1, 0L, (long)v.size() - 1);
        std::nth_element(v.begin(), v.begin() + idx, v.end());
        A = v[idx];
      }
      d->scale[z] = A;
    }
    d->scale[2] = 0.0;
    const Quantizer qz(*d);
    uint64_t hist[256];
    for (int s = 0; s < 256; ++s) hist[s] = 1;
    for (uint64_t r = 0; r < rows; ++r)
      for (uint32_t k = 0; k < E; ++k) hist[qz.level(k, coef[r * E + k])]++;
    if (!package_merge(hist, d->lmax, d->code_len)) {
      set_error("package-merge failed");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    return FPTC_OK;
  });
}

fptc_status fptc_encode_stream(const fptc_domain *d, const float *x, uint64_t S, uint64_t *words, uint8_t *symlen,
                               uint64_t capacity, uint64_t *n_words, uint8_t *levels) {
  return guarded([&]() -> fptc_status {
    uint32_t codes[256];
    fptc_status st = fptc_canonical_codes(d, codes);
    if (st != FPTC_OK) return st;
    if ((S && !x) || !n_words || (capacity && (!words || !symlen))) {
      set_error("NULL argument");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    const uint32_t N = d->N, E = d->E;
    const auto cosv = cos_table(N, E);
    const Quantizer qz(*d);
    const uint64_t W = (S + N - 1) / N;
    double C[128];
    uint64_t w_out = 0, buf = 0;
    uint32_t bits = 0, count = 0;
    for (uint64_t w = 0; w < W; ++w) {
      forward_window(x + w * N, S - w * N, N, E, cosv, C);
      for (uint32_t k = 0; k < E; ++k) {
        const uint8_t lv = qz.level(k, C[k]);
        if (levels) levels[w * E + k] = lv;
        const uint32_t cl = d->code_len[lv];
        if (!cl) {
          set_error("level %u has no code", lv);
          return FPTC_ERR_INVALID_ARGUMENT;
        }
        if (bits + cl > 64) {  // close the word; the codeword goes to the next one
          if (w_out >= capacity) {
            set_error("word capacity exceeded");
            return FPTC_ERR_INVALID_ARGUMENT;
          }
          words[w_out] = buf;
          symlen[w_out] = (uint8_t)count;
          ++w_out;
          buf = 0;
          bits = 0;
          count = 0;
        }
        buf |= (uint64_t)codes[lv] << (64 - bits - cl);
        bits += cl;
        ++count;
      }
    }
    if (count) {
      if (w_out >= capacity) {
        set_error("word capacity exceeded");
        return FPTC_ERR_INVALID_ARGUMENT;
      }
      words[w_out] = buf;
      symlen[w_out] = (uint8_t)count;
      ++w_out;
    }
    *n_words = w_out;
    return FPTC_OK;
  });
}

fptc_status fptc_encode_batch(const fptc_domain *domains, uint32_t n_domains, const float *x,
                              const uint64_t *x_offsets, const uint64_t *lengths, const uint32_t *domain_idx,
                              uint64_t n, uint64_t *words, uint8_t *symlen, const uint64_t *capacity_offsets,
                              uint64_t *n_words, int n_threads) {
  return guarded([&]() -> fptc_status {
    clear_error();
    for (uint64_t i = 0; i < n; ++i) {
      if (domain_idx[i] >= n_domains) {
        set_error("signal %llu: domain out of range", (unsigned long long)i);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
    }
    unsigned hw = std::thread::hardware_concurrency();
    const unsigned nt = n_threads > 0 ? (unsigned)n_threads : (hw ? hw : 1u);
    std::atomic<uint64_t> next{0};
    std::atomic<int> failed{0};
    auto work = [&]() {
      for (;;) {
        const uint64_t i = next.fetch_add(1);
        if (i >= n || failed.load()) return;
        const fptc_domain &d = domains[domain_idx[i]];
        const uint64_t cap = fptc_word_capacity(&d, lengths[i]);
        if (fptc_encode_stream(&d, x + x_offsets[i], lengths[i], words + capacity_offsets[i],
                               symlen + capacity_offsets[i], cap, &n_words[i], nullptr) != FPTC_OK)
          failed.store(1);
      }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    if (failed.load()) {
      set_error("encoding failed");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    return FPTC_OK;
  });
}

}  // extern "C"
