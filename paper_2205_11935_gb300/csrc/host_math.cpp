// Host-side mathematics of the ctl library: prime chains and roots, the SplitMix64
// streams that key generation and encryption draw from, the FP64 canonical-embedding
// encoder (Sec. 3.1 "SIMD Encoding") and the CRT used when decrypting.
#include <cmath>
#include <cstring>
#include <algorithm>
#include "ctl_internal.h"

namespace ctl {

typedef unsigned __int128 u128;

u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 h_powmod(u64 a, u64 e, u64 q) {
  u64 acc = 1 % q, base = a % q;
  for (; e; e >>= 1) {
    if (e & 1) acc = h_mulmod(acc, base, q);
    base = h_mulmod(base, base, q);
  }
  return acc;
}
u64 h_invmod(u64 a, u64 q) { return h_powmod(a, q - 2, q); }
u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
u64 h_mont(u64 x, u64 q) { return (u64)(((u128)(x % q) << 64) % q); }
u64 h_neg_inv64(u64 q) {
  // Newton iteration for q^-1 mod 2^64 (q odd): x <- x * (2 - q x) doubles the bits.
  u64 x = q;  // correct to 3 bits for odd q
  for (int i = 0; i < 6; i++) x *= 2 - q * x;
  return x;
}
uint32_t h_bitrev(uint32_t x, uint32_t logn) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < logn; i++, x >>= 1) r = (r << 1) | (x & 1u);
  return r;
}

// Miller-Rabin with the first twelve prime bases: deterministic below 3.3 * 10^24.
static bool probable_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 b : bases)
    if (n % b == 0) return n == b;
  u64 d = n - 1;
  unsigned r = 0;
  while (!(d & 1)) d >>= 1, r++;
  for (u64 b : bases) {
    u64 x = h_powmod(b, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (unsigned i = 1; i < r && witness; i++) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

// Prime chain rule: for each size b in order, the largest prime q < 2^b with
// q = 1 mod max(2N, 2^15) not chosen before.
bool plan_primes(uint32_t N, const std::vector<uint32_t>& bits, std::vector<u64>& out) {
  const u64 step = std::max<u64>(2ull * N, 1ull << 15);
  out.clear();
  for (uint32_t b : bits) {
    if (b < 20 || b > 61) return false;
    const u64 hi = 1ull << b;
    if (hi <= 2 * step) return false;
    u64 cand = hi - step + 1;
    bool ok = false;
    while (cand > step) {
      if (std::find(out.begin(), out.end(), cand) == out.end() && probable_prime(cand)) {
        out.push_back(cand);
        ok = true;
        break;
      }
      cand -= step;
    }
    if (!ok) return false;
  }
  return true;
}

// The smallest primitive 2N-th root of unity modulo q.
u64 min_primitive_2n_root(u64 q, uint32_t N) {
  const u64 ord = 2ull * N, cof = (q - 1) / ord;
  u64 root = 0;
  for (u64 g = 2;; g++) {
    u64 c = h_powmod(g, cof, q);
    if (h_powmod(c, N, q) == q - 1) {
      root = c;
      break;
    }
  }
  // all primitive 2N-th roots are root^k, k odd
  const u64 sq = h_mulmod(root, root, q);
  u64 best = root, cur = root;
  for (u64 k = 3; k < ord; k += 2) {
    cur = h_mulmod(cur, sq, q);
    best = std::min(best, cur);
  }
  return best;
}

// ---------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): state += 0x9E3779B97F4A7C15, output the
// finaliser of the state.  Stream (seed, id) starts from state
// mix(seed ^ mix(id + gamma)).
// ---------------------------------------------------------------------------------
static inline u64 splitmix_finalise(u64 z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
static const u64 kGoldenGamma = 0x9E3779B97F4A7C15ull;
SplitMixStream::SplitMixStream(u64 seed, u64 stream)
    : key(splitmix_finalise(seed ^ splitmix_finalise(stream + kGoldenGamma))), ctr(0) {}
u64 SplitMixStream::next() {
  ++ctr;
  return splitmix_finalise(key + ctr * kGoldenGamma);
}
u64 stream_id_secret() { return 1ull << 56; }
u64 stream_id_key_a(u64 key_id, u64 digit, u64 limb) { return (2ull << 56) | (key_id << 24) | (digit << 12) | limb; }
u64 stream_id_key_e(u64 key_id, u64 digit) { return (3ull << 56) | (key_id << 24) | (digit << 12); }
u64 stream_id_enc_a(u64 limb) { return (4ull << 56) | limb; }
u64 stream_id_enc_e() { return 5ull << 56; }

void draw_uniform(SplitMixStream& st, u64 q, uint32_t N, u64* out) {
  unsigned bits = 64 - __builtin_clzll(q);
  const u64 mask = bits == 64 ? ~0ull : ((1ull << bits) - 1);
  uint32_t n = 0;
  while (n < N) {
    const u64 w = st.next() & mask;
    if (w < q) out[n++] = w;
  }
}
void draw_ternary(SplitMixStream& st, uint32_t N, i64* out) {
  static const i64 map3[3] = {0, 1, -1};
  uint32_t n = 0;
  while (n < N) {
    const u64 w = st.next() & 3ull;
    if (w != 3) out[n++] = map3[w];
  }
}
void draw_cbd21(SplitMixStream& st, uint32_t N, i64* out) {
  const u64 m21 = (1ull << 21) - 1;
  for (uint32_t n = 0; n < N; n++) {
    const u64 w = st.next();
    out[n] = (i64)__builtin_popcountll(w & m21) - (i64)__builtin_popcountll((w >> 21) & m21);
  }
}

// ---------------------------------------------------------------------------------
// Encoder.  Slots j < N/2 live at the odd powers zeta^(5^j) and their conjugates at
// zeta^(-5^j), zeta = exp(i pi / N).  With omega = zeta^2, evaluating m at zeta^(2i+1)
// is a length-N DFT of the twisted vector m_k zeta^k, so both directions are one FFT.
// ---------------------------------------------------------------------------------
void Encoder::init(uint32_t n) {
  N = n;
  const uint32_t half = N / 2;
  slot_pos.resize(half);
  conj_pos.resize(half);
  u64 e = 1;
  for (uint32_t j = 0; j < half; j++) {
    slot_pos[j] = (uint32_t)((e - 1) / 2);
    conj_pos[j] = (uint32_t)((2ull * N - e - 1) / 2);
    e = (e * 5) % (2ull * N);
  }
  cs.resize(N);
  sn.resize(N);
  zc.resize(N);
  zs.resize(N);
  for (uint32_t k = 0; k < N; k++) {
    cs[k] = std::cos(2.0 * M_PI * (double)k / (double)N);
    sn[k] = std::sin(2.0 * M_PI * (double)k / (double)N);
    zc[k] = std::cos(M_PI * (double)k / (double)N);
    zs[k] = std::sin(M_PI * (double)k / (double)N);
  }
}

// In-place radix-2 DFT: X_i = sum_k x_k omega^(+-ik), omega = exp(2 pi i / N).
void Encoder::fft(std::vector<double>& re, std::vector<double>& im, bool inverse) const {
  const uint32_t n = N;
  uint32_t logn = 0;
  while ((1u << logn) < n) logn++;
  for (uint32_t i = 0; i < n; i++) {
    uint32_t j = h_bitrev(i, logn);
    if (j > i) {
      std::swap(re[i], re[j]);
      std::swap(im[i], im[j]);
    }
  }
  for (uint32_t len = 2; len <= n; len <<= 1) {
    const uint32_t half = len / 2, stride = n / len;
    for (uint32_t s = 0; s < n; s += len) {
      for (uint32_t k = 0; k < half; k++) {
        const double wr = cs[k * stride], wi = inverse ? -sn[k * stride] : sn[k * stride];
        const double ur = re[s + k], ui = im[s + k];
        const double xr = re[s + k + half], xi = im[s + k + half];
        const double vr = xr * wr - xi * wi, vi = xr * wi + xi * wr;
        re[s + k] = ur + vr;
        im[s + k] = ui + vi;
        re[s + k + half] = ur - vr;
        im[s + k + half] = ui - vi;
      }
    }
  }
}

bool Encoder::encode(const double* z, size_t nz, double scale, i64* m) const {
  std::vector<double> re(N, 0.0), im(N, 0.0);
  for (size_t j = 0; j < nz; j++) {
    re[slot_pos[j]] = z[j];
    re[conj_pos[j]] = z[j];  // real slots: the conjugate value is the same real number
  }
  // m_k = (1/N) zeta^-k sum_i Z_i omega^(-ik)
  fft(re, im, true);
  bool ok = true;
  for (uint32_t k = 0; k < N; k++) {
    const double v = (re[k] * zc[k] + im[k] * zs[k]) / (double)N * scale;  // Re(zeta^-k * X_k)
    if (!(std::fabs(v) < 4.0e18)) {
      ok = false;
      m[k] = 0;
      continue;
    }
    m[k] = (i64)std::llround(v);
  }
  return ok;
}

bool Encoder::encode_rns(const double* z, size_t nz, double scale, const u64* moduli, uint32_t lvl,
                         u64* out) const {
  std::vector<double> re(N, 0.0), im(N, 0.0);
  for (size_t j = 0; j < nz; j++) {
    re[slot_pos[j]] = z[j];
    re[conj_pos[j]] = z[j];
  }
  fft(re, im, true);
  for (uint32_t k = 0; k < N; k++) {
    const double v = (re[k] * zc[k] + im[k] * zs[k]) / (double)N * scale;
    if (!std::isfinite(v) || std::fabs(v) > 1e300) return false;
    const double r = std::fabs(v) < 4503599627370496.0 ? (double)std::llround(v) : v;  // integral from 2^52
    const double a = std::fabs(r);
    int e = 0;
    const double mant = std::frexp(a, &e);  // a = mant * 2^e, mant in [0.5, 1)
    u64 M = (u64)std::ldexp(mant, 53);      // a = M * 2^(e - 53), M < 2^53
    e -= 53;
    if (e < 0) {
      M >>= -e;  // a is an integer, so the shifted-out bits are zero
      e = 0;
    }
    for (uint32_t i = 0; i < lvl; i++) {
      const u64 q = moduli[i];
      u64 res = h_mulmod(M % q, h_powmod(2, (u64)e, q), q);
      if (r < 0 && res) res = q - res;
      out[(size_t)i * N + k] = res;
    }
  }
  return true;
}

void Encoder::decode(const double* m, size_t nz, double scale, double* z) const {
  std::vector<double> re(N), im(N);
  for (uint32_t k = 0; k < N; k++) {
    re[k] = m[k] * zc[k];
    im[k] = m[k] * zs[k];
  }
  fft(re, im, false);
  for (size_t j = 0; j < nz; j++) z[j] = re[slot_pos[j]] / scale;
}

// ---------------------------------------------------------------------------------
// Centred CRT (Garner's mixed radix) with exact multiword accumulation.
// ---------------------------------------------------------------------------------
namespace {
struct Words {
  std::vector<u64> w;
  explicit Words(size_t n) : w(n, 0) {}
  void mul_add(u64 m, u64 a) {  // this = this * m + a
    u128 carry = a;
    for (auto& x : w) {
      u128 t = (u128)x * m + carry;
      x = (u64)t;
      carry = t >> 64;
    }
  }
  int cmp(const Words& o) const {
    for (size_t i = w.size(); i-- > 0;)
      if (w[i] != o.w[i]) return w[i] < o.w[i] ? -1 : 1;
    return 0;
  }
  void sub_from(const Words& big) {  // this = big - this
    u64 borrow = 0;
    for (size_t i = 0; i < w.size(); i++) {
      u128 d = (u128)big.w[i] - w[i] - borrow;
      w[i] = (u64)d;
      borrow = (u64)(d >> 127);
    }
  }
  double to_double() const {
    double r = 0;
    for (size_t i = w.size(); i-- > 0;) r = r * 18446744073709551616.0 + (double)w[i];
    return r;
  }
};
}  // namespace

void crt_centred_to_double(const u64* res, size_t stride, uint32_t lvl, const u64* primes, size_t N, double* out) {
  const size_t nw = lvl + 1;
  // Garner coefficients: inv[i][j] = q_j^-1 mod q_i (j < i)
  std::vector<u64> inv(lvl * lvl, 0);
  for (uint32_t i = 0; i < lvl; i++)
    for (uint32_t j = 0; j < i; j++) inv[i * lvl + j] = h_invmod(primes[j] % primes[i], primes[i]);
  Words Q(nw), half(nw);
  Q.w[0] = 1;
  for (uint32_t i = 0; i < lvl; i++) Q.mul_add(primes[i], 0);
  // half = floor(Q/2)
  u64 carry = 0;
  for (size_t i = nw; i-- > 0;) {
    half.w[i] = (Q.w[i] >> 1) | (carry << 63);
    carry = Q.w[i] & 1;
  }
  std::vector<u64> v(lvl);
  for (size_t k = 0; k < N; k++) {
    for (uint32_t i = 0; i < lvl; i++) {
      const u64 qi = primes[i];
      u64 x = res[i * stride + k] % qi;
      for (uint32_t j = 0; j < i; j++) {
        u64 d = (x + qi - v[j] % qi) % qi;
        x = h_mulmod(d, inv[i * lvl + j], qi);
      }
      v[i] = x;
    }
    Words X(nw);
    for (uint32_t i = lvl; i-- > 0;) X.mul_add(primes[i], v[i]);  // Horner on the mixed radix
    if (X.cmp(half) > 0) {
      X.sub_from(Q);
      out[k] = -X.to_double();
    } else {
      out[k] = X.to_double();
    }
  }
}

}  // namespace ctl
