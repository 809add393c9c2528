// CKKS oracle for the CryptoTL server-side evaluation (TEST INFRASTRUCTURE).
//
// This file is the plain, slow, obviously-correct CPU statement of every integer map
// that the GPU library computes.  Only the test-suite, the package smoke check and the
// benchmark's CPU-baseline leg may load it; the product path never does.  It shares no
// code with the CUDA library: primes, roots, the pseudo-random generator, encoding,
// key generation, products, base conversion and rescaling are all written here again.
//
// Representation: polynomials in Z_q[X]/(X^N+1) are kept in COEFFICIENT form, one
// residue vector per prime ("limb"), limb-major: poly[limb][coef].  Ciphertexts are
// [2][limbs][N].  Products are schoolbook negacyclic convolutions; CRT, fast base
// conversion and rescaling use an explicit big-integer type.
//
// Method (CryptoTL, Sec. 3.1): CKKS with SIMD slot encoding, rescaling after each
// multiplication, rotations, the baby-step giant-step diagonal mat-vec of Eq. (bsgs)
// and a square activation.  Where the paper leaves a detail open (prime choice, root
// choice, sampling, key-switching variant, rounding) this file fixes one reading; each
// is stated at the function that implements it.
//
// Parity unpinned: none of the functions below is unpinned; the pins live in tests/.
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <vector>
#include <map>
#include <algorithm>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------------
// Word arithmetic modulo a prime q < 2^62 (plain 128-bit products and remainders).
// ---------------------------------------------------------------------------------
static inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static inline u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }
static u64 powmod(u64 a, u64 e, u64 q) {
  u64 r = 1 % q; a %= q;
  while (e) { if (e & 1) r = mulmod(r, a, q); a = mulmod(a, a, q); e >>= 1; }
  return r;
}
static inline u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }  // q prime
static inline u64 from_signed(i64 v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 a = (u64)(-(v + 1)) + 1;  // |v| without overflow at INT64_MIN
  u64 m = a % q;
  return m ? q - m : 0;
}

// ---------------------------------------------------------------------------------
// Fixed-width unsigned big integer (little-endian 64-bit words), enough for 20 primes.
// ---------------------------------------------------------------------------------
struct Big {
  static const int W = 22;
  u64 w[W];
  Big() { memset(w, 0, sizeof(w)); }
  explicit Big(u64 v) { memset(w, 0, sizeof(w)); w[0] = v; }
  bool is_zero() const { for (int i = 0; i < W; i++) if (w[i]) return false; return true; }
};
static int big_cmp(const Big& a, const Big& b) {
  for (int i = Big::W - 1; i >= 0; i--) { if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1; }
  return 0;
}
static void big_add(Big& a, const Big& b) {  // a += b
  u64 c = 0;
  for (int i = 0; i < Big::W; i++) { u128 s = (u128)a.w[i] + b.w[i] + c; a.w[i] = (u64)s; c = (u64)(s >> 64); }
}
static void big_sub(Big& a, const Big& b) {  // a -= b, requires a >= b
  u64 br = 0;
  for (int i = 0; i < Big::W; i++) {
    u128 d = (u128)a.w[i] - b.w[i] - br;
    a.w[i] = (u64)d; br = (u64)(d >> 64) ? 1 : 0;
  }
}
static void big_add_u64(Big& a, u64 v) { Big b(v); big_add(a, b); }
static Big big_mul_u64(const Big& a, u64 m) {
  Big r; u64 c = 0;
  for (int i = 0; i < Big::W; i++) { u128 p = (u128)a.w[i] * m + c; r.w[i] = (u64)p; c = (u64)(p >> 64); }
  return r;
}
static u64 big_mod_u64(const Big& a, u64 q) {
  u128 r = 0;
  for (int i = Big::W - 1; i >= 0; i--) r = ((r << 64) | a.w[i]) % q;
  return (u64)r;
}
static Big big_div_u64(const Big& a, u64 q, u64* rem) {
  Big r; u128 cur = 0;
  for (int i = Big::W - 1; i >= 0; i--) { cur = (cur << 64) | a.w[i]; r.w[i] = (u64)(cur / q); cur %= q; }
  if (rem) *rem = (u64)cur;
  return r;
}
static double big_to_double(const Big& a) {
  double r = 0.0;
  for (int i = Big::W - 1; i >= 0; i--) r = r * 18446744073709551616.0 + (double)a.w[i];
  return r;
}
static Big big_product(const std::vector<u64>& ps) {
  Big r(1);
  for (u64 p : ps) r = big_mul_u64(r, p);
  return r;
}

// ---------------------------------------------------------------------------------
// Primes and roots.
// ---------------------------------------------------------------------------------
// Deterministic Miller-Rabin for 64-bit integers with the first twelve primes as
// bases (sufficient for all n < 3.3e24, Sorenson & Webster 2015).
static bool is_prime_u64(u64 n) {
  if (n < 2) return false;
  static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 p : small) { if (n % p == 0) return n == p; }
  u64 d = n - 1; int s = 0;
  while ((d & 1) == 0) { d >>= 1; s++; }
  for (u64 a : small) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; r++) { x = mulmod(x, x, n); if (x == n - 1) { comp = false; break; } }
    if (comp) return false;
  }
  return true;
}

// Reading of the prime choice (the paper fixes only the bit sizes, Sec. 3.1
// "Multiplicative Depth" and Tab. 1): for each requested size b, in chain order
// (data primes q_0.. first, special primes after), take the largest prime q < 2^b with
// q = 1 mod M, M = max(2N, 32768), that has not been taken already.  The common
// M = 2^15 lets rings of degree up to 16384 share one chain.
static bool gen_primes(uint32_t N, const std::vector<uint32_t>& bits, std::vector<u64>& out) {
  u64 M = std::max<u64>(2ull * N, 32768ull);
  out.clear();
  for (uint32_t b : bits) {
    if (b < 20 || b > 61) return false;
    u64 top = 1ull << b;
    if (top <= 2 * M) return false;
    bool found = false;
    for (u64 q = top - M + 1; q > M; q -= M) {
      if (std::find(out.begin(), out.end(), q) != out.end()) continue;
      if (is_prime_u64(q)) { out.push_back(q); found = true; break; }
    }
    if (!found) return false;
  }
  return true;
}

// Reading of the root choice: psi is the smallest primitive 2N-th root of unity mod q.
// A candidate x^((q-1)/2N) is a primitive 2N-th root exactly when its N-th power is -1.
static u64 find_psi(u64 q, uint32_t N) {
  u64 e = (q - 1) / (2ull * N);
  u64 psi0 = 0;
  for (u64 x = 2; x < q; x++) {
    u64 w = powmod(x, e, q);
    if (powmod(w, N, q) == q - 1) { psi0 = w; break; }
  }
  u64 best = psi0, w2 = mulmod(psi0, psi0, q), cur = psi0;
  for (u64 k = 3; k < 2ull * N; k += 2) { cur = mulmod(cur, w2, q); if (cur < best) best = cur; }
  return best;
}

static uint32_t bitrev(uint32_t x, uint32_t logn) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < logn; i++) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

// ---------------------------------------------------------------------------------
// Counter-based generator: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), whose state
// advances by the golden gamma and whose output is the published 64-bit finaliser.
// A stream (seed, stream id) starts at state K = mix(seed XOR mix(stream + gamma));
// its i-th word (i = 0, 1, ...) is mix(K + (i+1) * gamma).
// ---------------------------------------------------------------------------------
static const u64 GAMMA = 0x9E3779B97F4A7C15ull;
static inline u64 sm_mix(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
struct Stream {
  u64 key, ctr;
  Stream(u64 seed, u64 stream) : key(sm_mix(seed ^ sm_mix(stream + GAMMA))), ctr(0) {}
  u64 next() { ctr++; return sm_mix(key + ctr * GAMMA); }
};
// Stream identifiers (tag in the top byte).
static u64 sid_secret() { return 1ull << 56; }
static u64 sid_key_a(u64 key_id, u64 digit, u64 limb) { return (2ull << 56) | (key_id << 24) | (digit << 12) | limb; }
static u64 sid_key_e(u64 key_id, u64 digit) { return (3ull << 56) | (key_id << 24) | (digit << 12); }
static u64 sid_enc_a(u64 limb) { return (4ull << 56) | limb; }
static u64 sid_enc_e() { return 5ull << 56; }

static uint32_t bitlen(u64 v) { uint32_t b = 0; while (v) { b++; v >>= 1; } return b; }
// Uniform residue mod q: take the low bitlen(q) bits of successive words, reject >= q.
static void sample_uniform(Stream& st, u64 q, uint32_t N, u64* out) {
  u64 mask = (bitlen(q) >= 64) ? ~0ull : ((1ull << bitlen(q)) - 1);
  for (uint32_t i = 0; i < N;) { u64 w = st.next() & mask; if (w < q) out[i++] = w; }
}
// Ternary secret: low two bits of successive words, 3 rejected; 0 -> 0, 1 -> 1, 2 -> -1.
static void sample_ternary(Stream& st, uint32_t N, i64* out) {
  for (uint32_t i = 0; i < N;) {
    u64 w = st.next() & 3;
    if (w == 3) continue;
    out[i++] = (w == 0) ? 0 : (w == 1 ? 1 : -1);
  }
}
// Error: centred binomial with k = 21, one word per coefficient:
// popcount(bits 0..20) - popcount(bits 21..41).
static void sample_cbd21(Stream& st, uint32_t N, i64* out) {
  for (uint32_t i = 0; i < N; i++) {
    u64 w = st.next();
    out[i] = (i64)__builtin_popcountll(w & 0x1FFFFFull) - (i64)__builtin_popcountll((w >> 21) & 0x1FFFFFull);
  }
}

// ---------------------------------------------------------------------------------
// Polynomial arithmetic per limb (coefficient form).
// ---------------------------------------------------------------------------------
// Negacyclic schoolbook product: c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j mod q.
static void negacyclic_mul(const u64* a, const u64* b, u64* c, uint32_t N, u64 q) {
#pragma omp parallel for schedule(static) if (N >= 512)
  for (int64_t k = 0; k < (int64_t)N; k++) {
    u128 pos = 0, neg = 0;
    int cnt = 0;
    u64 p = 0, n = 0;
    for (int64_t i = 0; i <= k; i++) {
      pos += (u128)a[i] * b[k - i];
      if (++cnt == 32) { pos %= q; cnt = 0; }
    }
    p = (u64)(pos % q);
    cnt = 0;
    for (int64_t i = k + 1; i < (int64_t)N; i++) {
      neg += (u128)a[i] * b[N + k - i];
      if (++cnt == 32) { neg %= q; cnt = 0; }
    }
    n = (u64)(neg % q);
    c[k] = submod(p, n, q);
  }
}
// Automorphism sigma_g: X^i -> X^(i*g mod 2N), with X^N = -1.
static void automorphism(const u64* a, u64* out, uint32_t N, u64 g, u64 q) {
  u64 twoN = 2ull * N;
  for (uint32_t i = 0; i < N; i++) {
    u64 e = ((u64)i * g) % twoN;
    if (e < N) out[e] = a[i];
    else out[e - N] = (a[i] == 0) ? 0 : q - a[i];
  }
}

// ---------------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------------
struct orc_ctx {
  uint32_t N, logN, L, K, alpha, beta;
  double scale;
  std::vector<u64> mods;  // L data primes then K special primes
  std::vector<u64> psi;
  Big P;                  // product of special primes
};

struct orc_keys {
  const orc_ctx* ctx;
  std::vector<i64> s;                 // ternary secret
  // key_id -> [beta][2][L+K][N]; key_id 0 is the relinearisation key, odd g the
  // Galois key for X -> X^g.
  std::map<u64, std::vector<u64>> evk;
};

static u64 gal_elt(const orc_ctx* c, int64_t r) {
  int64_t n = c->N / 2;
  int64_t rr = ((r % n) + n) % n;
  return powmod(5, (u64)rr, 2ull * c->N);
}

extern "C" {

orc_ctx* orc_ctx_create(uint32_t N, const uint32_t* qbits, uint32_t nq, const uint32_t* pbits,
                        uint32_t np, uint32_t dnum, double scale) {
  if (N < 8 || (N & (N - 1)) || N > 65536 || nq == 0 || np == 0 || dnum == 0 || dnum > nq) return nullptr;
  orc_ctx* c = new orc_ctx();
  c->N = N; c->logN = 0; while ((1u << c->logN) < N) c->logN++;
  c->L = nq; c->K = np;
  c->alpha = (nq + dnum - 1) / dnum;
  c->beta = (nq + c->alpha - 1) / c->alpha;
  c->scale = scale;
  std::vector<uint32_t> bits(qbits, qbits + nq);
  bits.insert(bits.end(), pbits, pbits + np);
  if (!gen_primes(N, bits, c->mods)) { delete c; return nullptr; }
  for (u64 q : c->mods) c->psi.push_back(find_psi(q, N));
  c->P = big_product(std::vector<u64>(c->mods.begin() + nq, c->mods.end()));
  return c;
}
void orc_ctx_destroy(orc_ctx* c) { delete c; }
int orc_ctx_moduli(const orc_ctx* c, u64* out) { for (size_t i = 0; i < c->mods.size(); i++) out[i] = c->mods[i]; return (int)c->mods.size(); }
int orc_ctx_psi(const orc_ctx* c, u64* out) { for (size_t i = 0; i < c->psi.size(); i++) out[i] = c->psi[i]; return (int)c->psi.size(); }
uint32_t orc_ctx_alpha(const orc_ctx* c) { return c->alpha; }
uint32_t orc_ctx_beta(const orc_ctx* c) { return c->beta; }
int orc_primes(uint32_t N, const uint32_t* bits, uint32_t n, u64* out) {
  std::vector<u64> ps;
  if (!gen_primes(N, std::vector<uint32_t>(bits, bits + n), ps)) return -1;
  for (uint32_t i = 0; i < n; i++) out[i] = ps[i];
  return 0;
}
u64 orc_psi(u64 q, uint32_t N) { return find_psi(q, N); }
int orc_is_prime(u64 n) { return is_prime_u64(n) ? 1 : 0; }

u64 orc_prng_word(u64 seed, u64 stream, u64 i) {
  Stream st(seed, stream);
  u64 w = 0;
  for (u64 k = 0; k <= i; k++) w = st.next();
  return w;
}
void orc_sample(u64 seed, u64 stream, int kind, u64 q, uint32_t N, i64* out) {
  Stream st(seed, stream);
  if (kind == 0) { std::vector<u64> tmp(N); sample_uniform(st, q, N, tmp.data()); for (uint32_t i = 0; i < N; i++) out[i] = (i64)tmp[i]; }
  else if (kind == 1) sample_ternary(st, N, out);
  else sample_cbd21(st, N, out);
}

// NTT form by definition: a_hat[k] = sum_i a[i] * psi^((2*bitrev(k)+1)*i) mod q.
int orc_ntt_direct(const orc_ctx* c, uint32_t pi, const u64* a, u64* out) {
  u64 q = c->mods[pi], psi = c->psi[pi];
  uint32_t N = c->N;
#pragma omp parallel for schedule(static) if (N >= 256)
  for (int64_t k = 0; k < (int64_t)N; k++) {
    u64 root = powmod(psi, 2ull * bitrev((uint32_t)k, c->logN) + 1, q);
    u64 acc = 0, pw = 1;
    for (uint32_t i = 0; i < N; i++) { acc = addmod(acc, mulmod(a[i], pw, q), q); pw = mulmod(pw, root, q); }
    out[k] = acc;
  }
  return 0;
}
// Inverse by definition: a[i] = N^-1 * sum_k a_hat[k] * psi^(-(2*bitrev(k)+1)*i).
int orc_intt_direct(const orc_ctx* c, uint32_t pi, const u64* ahat, u64* out) {
  u64 q = c->mods[pi], psi_inv = invmod(c->psi[pi], q), ninv = invmod(c->N, q);
  uint32_t N = c->N;
#pragma omp parallel for schedule(static) if (N >= 256)
  for (int64_t i = 0; i < (int64_t)N; i++) {
    u64 acc = 0;
    for (uint32_t k = 0; k < N; k++) {
      u64 e = ((2ull * bitrev(k, c->logN) + 1) * (u64)i) % (2ull * N);
      acc = addmod(acc, mulmod(ahat[k], powmod(psi_inv, e, q), q), q);
    }
    out[i] = mulmod(acc, ninv, q);
  }
  return 0;
}
int orc_negacyclic_mul(const orc_ctx* c, uint32_t pi, const u64* a, const u64* b, u64* out) {
  negacyclic_mul(a, b, out, c->N, c->mods[pi]);
  return 0;
}
int orc_automorphism(const orc_ctx* c, uint32_t pi, u64 g, const u64* a, u64* out) {
  automorphism(a, out, c->N, g, c->mods[pi]);
  return 0;
}
u64 orc_galois_element(const orc_ctx* c, int64_t r) { return gal_elt(c, r); }

// ---------------------------------------------------------------------------------
// Encoding (Sec. 3.1 "SIMD Encoding"): slot j sits at the root zeta^(5^j), zeta =
// exp(i*pi/N), j < N/2.  For real slot values the inverse embedding is
//   m_k = round(scale * (2/N) * sum_j z_j * cos(pi * (5^j * k mod 2N) / N)),
// rounding half away from zero.  Decoding evaluates m at zeta^(5^j) and divides by the
// scale (real part returned).
// ---------------------------------------------------------------------------------
int orc_encode(const orc_ctx* c, const double* z, uint32_t nz, double scale, i64* m) {
  uint32_t N = c->N, n = N / 2;
  if (nz > n) return -1;
  u64 twoN = 2ull * N;
  std::vector<double> costab(twoN);
  for (u64 e = 0; e < twoN; e++) costab[e] = cos(M_PI * (double)e / (double)N);
  std::vector<u64> rot(nz);
  u64 r = 1;
  for (uint32_t j = 0; j < nz; j++) { rot[j] = r; r = (r * 5) % twoN; }
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t k = 0; k < (int64_t)N; k++) {
    double acc = 0.0;
    for (uint32_t j = 0; j < nz; j++) acc += z[j] * costab[(rot[j] * (u64)k) % twoN];
    double v = scale * (2.0 / (double)N) * acc;
    if (!(fabs(v) < 4.0e18)) { bad++; m[k] = 0; continue; }
    m[k] = (i64)llround(v);
  }
  return bad ? -2 : 0;
}
int orc_decode(const orc_ctx* c, const double* m, double scale, uint32_t nz, double* z) {
  uint32_t N = c->N, n = N / 2;
  if (nz > n) return -1;
  u64 twoN = 2ull * N;
  std::vector<double> costab(twoN);
  for (u64 e = 0; e < twoN; e++) costab[e] = cos(M_PI * (double)e / (double)N);
  std::vector<u64> rot(nz);
  u64 r = 1;
  for (uint32_t j = 0; j < nz; j++) { rot[j] = r; r = (r * 5) % twoN; }
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)nz; j++) {
    double acc = 0.0;
    for (uint32_t k = 0; k < N; k++) acc += m[k] * costab[(rot[j] * (u64)k) % twoN];
    z[j] = acc / scale;
  }
  return 0;
}

// ---------------------------------------------------------------------------------
// Keys.  s is ternary.  A key-switching key from s' to s has, for each digit d (alpha
// consecutive data primes starting at q_0, the last digit possibly shorter), over all
// L+K primes:  evk_d = ( -a_d*s + e_d + P*[Qhat_d]*s' , a_d ),  where [Qhat_d] is the
// CRT idempotent of digit d, i.e. P*[Qhat_d] = P mod q_i on the primes of digit d and 0
// on every other prime.  s' = s^2 for relinearisation; s' = sigma_g(s) for rotation.
// ---------------------------------------------------------------------------------
static void gen_ksk(const orc_ctx* c, orc_keys* k, u64 seed, u64 key_id, const std::vector<i64>& sprime) {
  uint32_t N = c->N, LK = c->L + c->K;
  std::vector<u64> out((size_t)c->beta * 2 * LK * N);
  std::vector<i64> e(N);
  std::vector<u64> a(N), sres(N), spres(N), as(N);
  for (uint32_t d = 0; d < c->beta; d++) {
    Stream se(seed, sid_key_e(key_id, d));
    sample_cbd21(se, N, e.data());
    uint32_t d0 = d * c->alpha, d1 = std::min(d0 + c->alpha, c->L);
    for (uint32_t i = 0; i < LK; i++) {
      u64 q = c->mods[i];
      Stream sa(seed, sid_key_a(key_id, d, i));
      sample_uniform(sa, q, N, a.data());
      for (uint32_t j = 0; j < N; j++) { sres[j] = from_signed(k->s[j], q); spres[j] = from_signed(sprime[j], q); }
      negacyclic_mul(a.data(), sres.data(), as.data(), N, q);
      u64 gadget = (i >= d0 && i < d1) ? big_mod_u64(c->P, q) : 0;
      u64* b0 = &out[(((size_t)d * 2 + 0) * LK + i) * N];
      u64* b1 = &out[(((size_t)d * 2 + 1) * LK + i) * N];
      for (uint32_t j = 0; j < N; j++) {
        u64 v = submod(from_signed(e[j], q), as[j], q);
        v = addmod(v, mulmod(gadget, spres[j], q), q);
        b0[j] = v;
        b1[j] = a[j];
      }
    }
  }
  k->evk[key_id] = std::move(out);
}

orc_keys* orc_keygen(const orc_ctx* c, const int32_t* rots, uint32_t nrot, u64 seed) {
  uint32_t N = c->N;
  orc_keys* k = new orc_keys();
  k->ctx = c;
  k->s.resize(N);
  Stream ss(seed, sid_secret());
  sample_ternary(ss, N, k->s.data());
  // s^2 over the integers (negacyclic), coefficients bounded by N.
  std::vector<i64> s2(N, 0);
  for (uint32_t i = 0; i < N; i++) {
    if (!k->s[i]) continue;
    for (uint32_t j = 0; j < N; j++) {
      i64 p = k->s[i] * k->s[j];
      uint32_t e = i + j;
      if (e < N) s2[e] += p; else s2[e - N] -= p;
    }
  }
  gen_ksk(c, k, seed, 0, s2);
  for (uint32_t r = 0; r < nrot; r++) {
    u64 g = gal_elt(c, rots[r]);
    if (g == 1 || k->evk.count(g)) continue;
    std::vector<i64> sg(N);
    for (uint32_t i = 0; i < N; i++) {
      u64 e = ((u64)i * g) % (2ull * N);
      if (e < N) sg[e] = k->s[i]; else sg[e - N] = -k->s[i];
    }
    gen_ksk(c, k, seed, g, sg);
  }
  return k;
}
void orc_keys_destroy(orc_keys* k) { delete k; }
int orc_keys_secret(const orc_keys* k, i64* s) { for (size_t i = 0; i < k->s.size(); i++) s[i] = k->s[i]; return 0; }
int orc_keys_has(const orc_keys* k, u64 key_id) { return k->evk.count(key_id) ? 1 : 0; }
// Exports the key [beta][2][L+K][N] (coefficient form).
int orc_keys_export(const orc_keys* k, u64 key_id, u64* out) {
  auto it = k->evk.find(key_id);
  if (it == k->evk.end()) return -1;
  memcpy(out, it->second.data(), it->second.size() * sizeof(u64));
  return 0;
}

// ---------------------------------------------------------------------------------
// Encryption with the secret key at the top level (the C->S message of Sec. 5.1 is one
// ring element plus a seed): ct = ( [-a*s + m + e]_Q , a ).
// ---------------------------------------------------------------------------------
int orc_encrypt(const orc_ctx* c, const orc_keys* k, const i64* m, u64 seed, u64* ct) {
  uint32_t N = c->N, L = c->L;
  std::vector<i64> e(N);
  Stream se(seed, sid_enc_e());
  sample_cbd21(se, N, e.data());
  std::vector<u64> a(N), sres(N), as(N);
  for (uint32_t i = 0; i < L; i++) {
    u64 q = c->mods[i];
    Stream sa(seed, sid_enc_a(i));
    sample_uniform(sa, q, N, a.data());
    for (uint32_t j = 0; j < N; j++) sres[j] = from_signed(k->s[j], q);
    negacyclic_mul(a.data(), sres.data(), as.data(), N, q);
    u64* c0 = ct + (size_t)i * N;
    u64* c1 = ct + ((size_t)L + i) * N;
    for (uint32_t j = 0; j < N; j++) {
      c0[j] = addmod(submod(from_signed(m[j], q), as[j], q), from_signed(e[j], q), q);
      c1[j] = a[j];
    }
  }
  return 0;
}

// CRT of residues over the first `lvl` data primes into [0, Q).
static Big crt(const orc_ctx* c, const u64* res, uint32_t lvl, const Big& Q,
               const std::vector<Big>& Qhat, const std::vector<u64>& Qhat_inv) {
  Big acc;
  for (uint32_t i = 0; i < lvl; i++) {
    u64 t = mulmod(res[i], Qhat_inv[i], c->mods[i]);
    big_add(acc, big_mul_u64(Qhat[i], t));
  }
  while (big_cmp(acc, Q) >= 0) big_sub(acc, Q);
  return acc;
}
static void crt_tables(const orc_ctx* c, uint32_t lvl, Big& Q, std::vector<Big>& Qhat, std::vector<u64>& Qhat_inv) {
  std::vector<u64> ps(c->mods.begin(), c->mods.begin() + lvl);
  Q = big_product(ps);
  Qhat.assign(lvl, Big());
  Qhat_inv.assign(lvl, 0);
  for (uint32_t i = 0; i < lvl; i++) {
    u64 r;
    Qhat[i] = big_div_u64(Q, c->mods[i], &r);
    Qhat_inv[i] = invmod(big_mod_u64(Qhat[i], c->mods[i]), c->mods[i]);
  }
}

// Decryption: m' = [c0 + c1*s]_{Q_lvl}, returned as centred values in double.
int orc_decrypt(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, double* out) {
  uint32_t N = c->N;
  if (lvl == 0 || lvl > c->L) return -1;
  std::vector<u64> res((size_t)lvl * N), sres(N), prod(N);
  for (uint32_t i = 0; i < lvl; i++) {
    u64 q = c->mods[i];
    for (uint32_t j = 0; j < N; j++) sres[j] = from_signed(k->s[j], q);
    negacyclic_mul(ct + ((size_t)lvl + i) * N, sres.data(), prod.data(), N, q);
    for (uint32_t j = 0; j < N; j++) res[(size_t)i * N + j] = addmod(ct[(size_t)i * N + j], prod[j], q);
  }
  Big Q; std::vector<Big> Qhat; std::vector<u64> Qinv;
  crt_tables(c, lvl, Q, Qhat, Qinv);
  Big half = big_div_u64(Q, 2, nullptr);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)N; j++) {
    std::vector<u64> r(lvl);
    for (uint32_t i = 0; i < lvl; i++) r[i] = res[(size_t)i * N + j];
    Big v = crt(c, r.data(), lvl, Q, Qhat, Qinv);
    if (big_cmp(v, half) > 0) { Big t = Q; big_sub(t, v); out[j] = -big_to_double(t); }
    else out[j] = big_to_double(v);
  }
  return 0;
}

// ---------------------------------------------------------------------------------
// Ciphertext-level operations.  A ciphertext at level `lvl` holds the first lvl data
// primes: [2][lvl][N].
// ---------------------------------------------------------------------------------
int orc_add(const orc_ctx* c, const u64* a, const u64* b, uint32_t lvl, u64* out) {
  uint32_t N = c->N;
  for (uint32_t p = 0; p < 2; p++)
    for (uint32_t i = 0; i < lvl; i++)
      for (uint32_t j = 0; j < N; j++) {
        size_t o = ((size_t)p * lvl + i) * N + j;
        out[o] = addmod(a[o], b[o], c->mods[i]);
      }
  return 0;
}
// Plaintext-ciphertext product: (c0*p, c1*p) for an integer plaintext polynomial p.
int orc_mul_plain(const orc_ctx* c, const u64* ct, uint32_t lvl, const i64* pt, u64* out) {
  uint32_t N = c->N;
  std::vector<u64> pr(N);
  for (uint32_t i = 0; i < lvl; i++) {
    u64 q = c->mods[i];
    for (uint32_t j = 0; j < N; j++) pr[j] = from_signed(pt[j], q);
    for (uint32_t p = 0; p < 2; p++)
      negacyclic_mul(ct + ((size_t)p * lvl + i) * N, pr.data(), out + ((size_t)p * lvl + i) * N, N, q);
  }
  return 0;
}
int orc_add_plain(const orc_ctx* c, const u64* ct, uint32_t lvl, const i64* pt, u64* out) {
  uint32_t N = c->N;
  memcpy(out, ct, sizeof(u64) * 2 * lvl * N);
  for (uint32_t i = 0; i < lvl; i++)
    for (uint32_t j = 0; j < N; j++) out[(size_t)i * N + j] = addmod(ct[(size_t)i * N + j], from_signed(pt[j], c->mods[i]), c->mods[i]);
  return 0;
}

// Rescale (Sec. 3.1: rescaling is a rounding division by the last prime): for each
// coefficient, with C the CRT value in [0, Q_lvl) and q the last prime,
//   C' = floor((C + floor(q/2)) / q), reduced modulo the remaining primes.
int orc_rescale(const orc_ctx* c, const u64* ct, uint32_t lvl, u64* out) {
  uint32_t N = c->N;
  if (lvl < 2) return -1;
  Big Q; std::vector<Big> Qhat; std::vector<u64> Qinv;
  crt_tables(c, lvl, Q, Qhat, Qinv);
  u64 ql = c->mods[lvl - 1];
  for (uint32_t p = 0; p < 2; p++) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)N; j++) {
      std::vector<u64> r(lvl);
      for (uint32_t i = 0; i < lvl; i++) r[i] = ct[((size_t)p * lvl + i) * N + j];
      Big v = crt(c, r.data(), lvl, Q, Qhat, Qinv);
      big_add_u64(v, ql / 2);
      Big qt = big_div_u64(v, ql, nullptr);
      for (uint32_t i = 0; i + 1 < lvl; i++) out[((size_t)p * (lvl - 1) + i) * N + j] = big_mod_u64(qt, c->mods[i]);
    }
  }
  return 0;
}

// ModUp of digit d of a coefficient-form polynomial at level lvl (fast base conversion,
// no exact correction): with D the digit's live primes, Q_d their product and
// Qhat_j = Q_d / q_j, the integer  y = sum_{j in D} [a_j * Qhat_j^-1]_{q_j} * Qhat_j
// (= a + u*Q_d with 0 <= u < |D|) is reduced modulo every live data prime and every
// special prime.  Output basis order: data primes 0..lvl-1, then special primes.
int orc_modup(const orc_ctx* c, const u64* poly, uint32_t lvl, uint32_t d, u64* out, u64* u_out) {
  uint32_t N = c->N, K = c->K;
  uint32_t d0 = d * c->alpha, d1 = std::min(d0 + c->alpha, lvl);
  if (d0 >= lvl) return -1;
  std::vector<u64> dig(c->mods.begin() + d0, c->mods.begin() + d1);
  Big Qd = big_product(dig);
  std::vector<Big> Qhat(dig.size());
  std::vector<u64> Qhat_inv(dig.size());
  for (size_t j = 0; j < dig.size(); j++) {
    Qhat[j] = big_div_u64(Qd, dig[j], nullptr);
    Qhat_inv[j] = invmod(big_mod_u64(Qhat[j], dig[j]), dig[j]);
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)N; k++) {
    Big y;
    for (size_t j = 0; j < dig.size(); j++) {
      u64 t = mulmod(poly[(size_t)(d0 + j) * N + k], Qhat_inv[j], dig[j]);
      big_add(y, big_mul_u64(Qhat[j], t));
    }
    for (uint32_t i = 0; i < lvl; i++) out[(size_t)i * N + k] = big_mod_u64(y, c->mods[i]);
    for (uint32_t i = 0; i < K; i++) out[(size_t)(lvl + i) * N + k] = big_mod_u64(y, c->mods[c->L + i]);
    if (u_out) {
      u64 u = 0;
      while (big_cmp(y, Qd) >= 0) { big_sub(y, Qd); u++; }
      u_out[k] = u;
    }
  }
  return 0;
}

// ModDown of an extended polynomial [lvl+K][N] (data primes then special primes):
// y_P = sum_j [c_{p_j} * Phat_j^-1]_{p_j} * Phat_j (fast conversion of the special part,
// no rounding offset), out_i = (c_i - y_P) * P^-1 mod q_i.
int orc_moddown(const orc_ctx* c, const u64* ext, uint32_t lvl, u64* out) {
  uint32_t N = c->N, K = c->K, L = c->L;
  std::vector<u64> sp(c->mods.begin() + L, c->mods.end());
  std::vector<Big> Phat(K);
  std::vector<u64> Phat_inv(K), Pinv(lvl);
  for (uint32_t j = 0; j < K; j++) {
    Phat[j] = big_div_u64(c->P, sp[j], nullptr);
    Phat_inv[j] = invmod(big_mod_u64(Phat[j], sp[j]), sp[j]);
  }
  for (uint32_t i = 0; i < lvl; i++) Pinv[i] = invmod(big_mod_u64(c->P, c->mods[i]), c->mods[i]);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)N; k++) {
    Big y;
    for (uint32_t j = 0; j < K; j++) {
      u64 t = mulmod(ext[(size_t)(lvl + j) * N + k], Phat_inv[j], sp[j]);
      big_add(y, big_mul_u64(Phat[j], t));
    }
    for (uint32_t i = 0; i < lvl; i++) {
      u64 q = c->mods[i];
      out[(size_t)i * N + k] = mulmod(submod(ext[(size_t)i * N + k], big_mod_u64(y, q), q), Pinv[i], q);
    }
  }
  return 0;
}

// The key product of hybrid key switching, kept in the extended basis (before ModDown):
// acc[t] = sum_d sigma_g(ModUp_d(x)) * evk_d[t], [2][lvl+K][N].
static int ks_ext(const orc_ctx* c, const orc_keys* k, u64 key_id, const u64* x, uint32_t lvl, u64 g,
                  std::vector<u64>& acc0, std::vector<u64>& acc1) {
  auto it = k->evk.find(key_id);
  if (it == k->evk.end()) return -2;
  uint32_t N = c->N, K = c->K, L = c->L, LK = L + K, E = lvl + K;
  uint32_t nd = (lvl + c->alpha - 1) / c->alpha;
  std::vector<u64> ext((size_t)E * N), tmp(N), prod(N);
  acc0.assign((size_t)E * N, 0);
  acc1.assign((size_t)E * N, 0);
  for (uint32_t d = 0; d < nd; d++) {
    orc_modup(c, x, lvl, d, ext.data(), nullptr);
    for (uint32_t i = 0; i < E; i++) {
      uint32_t gi = i < lvl ? i : L + (i - lvl);
      u64 q = c->mods[gi];
      u64* e = &ext[(size_t)i * N];
      if (g != 1) { automorphism(e, tmp.data(), N, g, q); memcpy(e, tmp.data(), N * sizeof(u64)); }
      const u64* k0 = &it->second[(((size_t)d * 2 + 0) * LK + gi) * N];
      const u64* k1 = &it->second[(((size_t)d * 2 + 1) * LK + gi) * N];
      negacyclic_mul(e, k0, prod.data(), N, q);
      for (uint32_t j = 0; j < N; j++) acc0[(size_t)i * N + j] = addmod(acc0[(size_t)i * N + j], prod[j], q);
      negacyclic_mul(e, k1, prod.data(), N, q);
      for (uint32_t j = 0; j < N; j++) acc1[(size_t)i * N + j] = addmod(acc1[(size_t)i * N + j], prod[j], q);
    }
  }
  return 0;
}

// Hybrid key switching of a coefficient-form polynomial x at level lvl with key key_id:
// for every live digit d, ext_d = ModUp_d(x); if g != 1 each ext_d is first mapped by
// sigma_g; then acc_t = sum_d ext_d * evk_d[t] over the live data primes and the special
// primes, and the result is (ModDown(acc_0), ModDown(acc_1)).  Key limbs of primes that
// are no longer live are not used.
int orc_keyswitch(const orc_ctx* c, const orc_keys* k, u64 key_id, const u64* x, uint32_t lvl, u64 g, u64* out) {
  std::vector<u64> acc0, acc1;
  int rc = ks_ext(c, k, key_id, x, lvl, g, acc0, acc1);
  if (rc) return rc;
  orc_moddown(c, acc0.data(), lvl, out);
  orc_moddown(c, acc1.data(), lvl, out + (size_t)lvl * c->N);
  return 0;
}

// Rotation to the left by r slots (Sec. 3.1, rot_j): g = 5^(r mod N/2) mod 2N.  The
// order is fixed as ModUp(c1) -> sigma_g on the digits -> key product -> ModDown, and
// the result is (sigma_g(c0) + ks_0, ks_1).  r = 0 mod N/2 returns the input.
int orc_rotate(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, int64_t r, u64* out) {
  uint32_t N = c->N;
  u64 g = gal_elt(c, r);
  if (g == 1) { memcpy(out, ct, sizeof(u64) * 2 * lvl * N); return 0; }
  std::vector<u64> ks((size_t)2 * lvl * N), a(N);
  int rc = orc_keyswitch(c, k, g, ct + (size_t)lvl * N, lvl, g, ks.data());
  if (rc) return rc;
  for (uint32_t i = 0; i < lvl; i++) {
    u64 q = c->mods[i];
    automorphism(ct + (size_t)i * N, a.data(), N, g, q);
    for (uint32_t j = 0; j < N; j++) {
      out[(size_t)i * N + j] = addmod(a[j], ks[(size_t)i * N + j], q);
      out[((size_t)lvl + i) * N + j] = ks[((size_t)lvl + i) * N + j];
    }
  }
  return 0;
}

// Relinearisation of (d0, d1, d2) [3][lvl][N]: (d0 + ks_0, d1 + ks_1), ks = KS_rlk(d2).
int orc_relin(const orc_ctx* c, const orc_keys* k, const u64* d, uint32_t lvl, u64* out) {
  uint32_t N = c->N;
  std::vector<u64> ks((size_t)2 * lvl * N);
  int rc = orc_keyswitch(c, k, 0, d + (size_t)2 * lvl * N, lvl, 1, ks.data());
  if (rc) return rc;
  for (uint32_t p = 0; p < 2; p++)
    for (uint32_t i = 0; i < lvl; i++)
      for (uint32_t j = 0; j < N; j++) {
        size_t o = ((size_t)p * lvl + i) * N + j;
        out[o] = addmod(d[o], ks[o], c->mods[i]);
      }
  return 0;
}

// Square activation: tensor (c0^2, 2*c0*c1, c1^2), relinearise, rescale.
int orc_square(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, u64* out) {
  uint32_t N = c->N;
  if (lvl < 2) return -1;
  std::vector<u64> d((size_t)3 * lvl * N), t(N), r((size_t)2 * lvl * N);
  for (uint32_t i = 0; i < lvl; i++) {
    u64 q = c->mods[i];
    const u64* c0 = ct + (size_t)i * N;
    const u64* c1 = ct + ((size_t)lvl + i) * N;
    negacyclic_mul(c0, c0, &d[(size_t)i * N], N, q);
    negacyclic_mul(c0, c1, t.data(), N, q);
    for (uint32_t j = 0; j < N; j++) d[((size_t)lvl + i) * N + j] = addmod(t[j], t[j], q);
    negacyclic_mul(c1, c1, &d[((size_t)2 * lvl + i) * N], N, q);
  }
  int rc = orc_relin(c, k, d.data(), lvl, r.data());
  if (rc) return rc;
  return orc_rescale(c, r.data(), lvl, out);
}

// Baby-step giant-step sizes (Eq. bsgs): t is the next power of two >= max(m, n) (the
// paper pads non-square matrices with zeros) and t = t1 * t2 with t1 = 2^ceil(log2(t)/2).
uint32_t orc_bsgs_t(uint32_t m, uint32_t n) { uint32_t t = 1; while (t < m || t < n) t <<= 1; return t; }
uint32_t orc_bsgs_t1(uint32_t t) { uint32_t lg = 0; while ((1u << lg) < t) lg++; return 1u << ((lg + 1) / 2); }
// The split of the lazy-ModDown form (orc_dense_lazy): there a baby step is one key
// product and a giant step a whole key switch (about four baby steps), so
// t1 = min(t, 2^ceil(log2(4t)/2)), which minimises (t1 - 1) + 4 (t2 - 1).
uint32_t orc_bsgs_t1_lazy(uint32_t t) {
  uint32_t lg = 0;
  while ((1u << lg) < t) lg++;
  uint32_t t1 = 1u << ((lg + 3) / 2);
  return t1 < t ? t1 : t;
}

// Diagonal plaintexts of a dense layer W (m x n, row-major) for Eq. (bsgs):
// diag_i[r] = W[r][(r+i) mod t] (zero outside W), diag'_i = rot_{-floor(i/t1)*t1}(diag_i)
// with diag_i placed in slots [0, t) of the full slot vector, encoded at `scale`.
// t1 = 0 takes orc_bsgs_t1(t).  With `windows` = p > 1 (Sec. 3.1 "Multiple
// Predictions": p inputs per ciphertext, each in its own window of 2t slots), the
// pattern of slots [0, 2t) is repeated at slots [2t w, 2t (w+1)) for w < p.
int orc_encode_diagonals_w(const orc_ctx* c, const double* W, uint32_t m, uint32_t n, uint32_t t1, double scale,
                           uint32_t windows, i64* pts) {
  uint32_t t = orc_bsgs_t(m, n), ns = c->N / 2;
  if (!t1) t1 = orc_bsgs_t1(t);
  if (windows == 0 || 2 * t * windows > ns) return -1;
  std::vector<double> v(ns);
  for (uint32_t i = 0; i < t; i++) {
    std::fill(v.begin(), v.end(), 0.0);
    uint32_t sh = (i / t1) * t1;
    for (uint32_t w = 0; w < windows; w++)
      for (uint32_t r = 0; r < t; r++) {
        uint32_t col = (r + i) % t;
        double x = (r < m && col < n) ? W[(size_t)r * n + col] : 0.0;
        v[2 * t * w + r + sh] = x;
      }
    int rc = orc_encode(c, v.data(), ns, scale, pts + (size_t)i * c->N);
    if (rc) return rc;
  }
  return 0;
}
int orc_encode_diagonals(const orc_ctx* c, const double* W, uint32_t m, uint32_t n, uint32_t t1, double scale,
                         i64* pts) {
  return orc_encode_diagonals_w(c, W, m, n, t1, scale, 1, pts);
}

// Dense layer by Eq. (bsgs) on an input laid out as [x, x] over 2t slots, as the plain
// composition of whole rotations (each one ModUp -> sigma_g -> key product -> ModDown,
// the baby steps sharing one ModUp):
//   out = sum_k rot_{k t1}( sum_j diag'_{k t1 + j} o rot_j(ct) ),
// inner sums in increasing j, outer in increasing k, then an optional plaintext bias
// (added to c0) and a rescale.  counters[0..2] receive the rotations, plaintext
// products and additions performed (t1+t2-2, t, t-1).
int orc_dense(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, const i64* pts, uint32_t t,
              const i64* bias, u64* out, u64* counters) {
  uint32_t N = c->N, t1 = orc_bsgs_t1(t), t2 = t / t1;
  size_t csz = (size_t)2 * lvl * N;
  std::vector<u64> baby((size_t)t1 * csz), inner(csz), prod(csz), acc(csz), rot(csz);
  u64 nrot = 0, nmul = 0, nadd = 0;
  for (uint32_t j = 0; j < t1; j++) {
    int rc = orc_rotate(c, k, ct, lvl, j, &baby[(size_t)j * csz]);
    if (rc) return rc;
    if (j) nrot++;
  }
  for (uint32_t kk = 0; kk < t2; kk++) {
    for (uint32_t j = 0; j < t1; j++) {
      orc_mul_plain(c, &baby[(size_t)j * csz], lvl, pts + (size_t)(kk * t1 + j) * N, prod.data());
      nmul++;
      if (j == 0) inner = prod; else { orc_add(c, inner.data(), prod.data(), lvl, inner.data()); nadd++; }
    }
    if (kk) { int rc = orc_rotate(c, k, inner.data(), lvl, (int64_t)kk * t1, rot.data()); if (rc) return rc; nrot++; inner = rot; }
    if (kk == 0) acc = inner; else { orc_add(c, acc.data(), inner.data(), lvl, acc.data()); nadd++; }
  }
  if (bias) orc_add_plain(c, acc.data(), lvl, bias, acc.data());
  if (counters) { counters[0] = nrot; counters[1] = nmul; counters[2] = nadd; }
  return orc_rescale(c, acc.data(), lvl, out);
}

// Dense layer by Eq. (bsgs) with every ModDown of the baby and giant steps postponed
// (an alternative to orc_dense, not bit-identical to it: the rotations are key switches
// kept in the extended basis Q*P, and the division by P happens once per giant step
// and once at the end).  With E = lvl + K limbs (data primes, then special primes),
// P the special modulus and t1 = orc_bsgs_t1_lazy(t):
//   B_0 = (P*c0, P*c1) (zero on the special limbs),
//   B_j = (P*sigma_j(c0) + a_0, a_1), (a_0, a_1) = key product of c1 for rot_j, j >= 1,
//   I_k = sum_j diag'_{k t1 + j} o B_j over all E limbs (diagonals reduced mod every prime),
//   S   = I_0 + sum_{k >= 1} ( sigma_{k t1}(I_k.0) + b_0, b_1 ),
//         (b_0, b_1) = key product of ModDown(I_k.1) for rot_{k t1},
//   out = rescale( (ModDown(S.0), ModDown(S.1)) [+ bias on c0] ).
// The sums run in increasing j and k.  counters as for orc_dense.
int orc_dense_lazy(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, const i64* pts, uint32_t t,
                   const i64* bias, u64* out, u64* counters) {
  uint32_t N = c->N, K = c->K, L = c->L, E = lvl + K, t1 = orc_bsgs_t1_lazy(t), t2 = t / t1;
  auto prime = [&](uint32_t i) { return c->mods[i < lvl ? i : L + (i - lvl)]; };
  const size_t ew = (size_t)E * N;  // one polynomial in the extended basis
  std::vector<u64> B((size_t)t1 * 2 * ew, 0), S(2 * ew), Ik(2 * ew), pr(N), prod(N), tmp(N), c1d((size_t)lvl * N);
  std::vector<u64> a0, a1;
  u64 nrot = 0, nmul = 0, nadd = 0;
  std::vector<u64> Pq(lvl);
  for (uint32_t i = 0; i < lvl; i++) Pq[i] = big_mod_u64(c->P, c->mods[i]);
  // baby steps in the extended basis
  for (uint32_t j = 0; j < t1; j++) {
    u64* Bj = &B[(size_t)j * 2 * ew];
    u64 g = gal_elt(c, j);
    if (g != 1) {
      int rc = ks_ext(c, k, g, ct + (size_t)lvl * N, lvl, g, a0, a1);
      if (rc) return rc;
      std::copy(a0.begin(), a0.end(), Bj);
      std::copy(a1.begin(), a1.end(), Bj + ew);
      nrot++;
    }
    for (uint32_t i = 0; i < lvl; i++) {
      u64 q = c->mods[i];
      for (uint32_t p = 0; p < 2; p++) {
        const u64* src = ct + ((size_t)p * lvl + i) * N;
        if (g != 1 && p == 0) { automorphism(src, tmp.data(), N, g, q); src = tmp.data(); }
        if (g != 1 && p == 1) continue;  // the key product carries the whole c1 part
        u64* d = Bj + (size_t)p * ew + (size_t)i * N;
        for (uint32_t x = 0; x < N; x++) d[x] = addmod(d[x], mulmod(src[x], Pq[i], q), q);
      }
    }
  }
  // inner sums and giant steps
  for (uint32_t kk = 0; kk < t2; kk++) {
    std::fill(Ik.begin(), Ik.end(), 0);
    for (uint32_t j = 0; j < t1; j++) {
      const i64* pt = pts + (size_t)(kk * t1 + j) * N;
      for (uint32_t i = 0; i < E; i++) {
        u64 q = prime(i);
        for (uint32_t x = 0; x < N; x++) pr[x] = from_signed(pt[x], q);
        for (uint32_t p = 0; p < 2; p++) {
          negacyclic_mul(&B[(size_t)j * 2 * ew + (size_t)p * ew + (size_t)i * N], pr.data(), prod.data(), N, q);
          u64* d = &Ik[(size_t)p * ew + (size_t)i * N];
          for (uint32_t x = 0; x < N; x++) d[x] = addmod(d[x], prod[x], q);
        }
      }
      nmul++;
      if (j) nadd++;
    }
    if (kk == 0) { S = Ik; continue; }
    u64 g = gal_elt(c, (int64_t)kk * t1);
    orc_moddown(c, &Ik[ew], lvl, c1d.data());
    int rc = ks_ext(c, k, g, c1d.data(), lvl, g, a0, a1);
    if (rc) return rc;
    nrot++;
    nadd++;
    for (uint32_t i = 0; i < E; i++) {
      u64 q = prime(i);
      automorphism(&Ik[(size_t)i * N], tmp.data(), N, g, q);
      for (uint32_t x = 0; x < N; x++) {
        size_t o = (size_t)i * N + x;
        S[o] = addmod(S[o], addmod(tmp[x], a0[o], q), q);
        S[ew + o] = addmod(S[ew + o], a1[o], q);
      }
    }
  }
  std::vector<u64> acc((size_t)2 * lvl * N);
  orc_moddown(c, S.data(), lvl, acc.data());
  orc_moddown(c, S.data() + ew, lvl, acc.data() + (size_t)lvl * N);
  if (bias) orc_add_plain(c, acc.data(), lvl, bias, acc.data());
  if (counters) { counters[0] = nrot; counters[1] = nmul; counters[2] = nadd; }
  return orc_rescale(c, acc.data(), lvl, out);
}

// Rectangular diagonal form of a dense layer.  Sec. 3.1 ("Dense-Layer") pads a non-square
// matrix with zeros to a square one; this reading pads only the short side.  For W (m x n,
// row-major) with tm = pow2 >= m below tn = pow2 >= n, the tm diagonals of length tn are
//   rd_i[r] = W[r mod tm][(r + i) mod tn]   (zero outside W),  r < tn,  i < tm,
// so that z = sum_i rd_i o rot_i(x), on the [x, x] input layout over 2 tn slots, holds in
// slot r < tn the partial sum over the columns (r + i) mod tn of row r mod tm, and
// y[j] = sum_{k < tn/tm} z[j + k tm].  They are placed as in Eq. (bsgs):
// rd'_i = rot_{-floor(i/t1) t1}(rd_i) with rd_i in slots [0, tn) and t1 = orc_bsgs_t1(tm).
// lazy = 1 places them for the lazy-ModDown form's split t1 = orc_bsgs_t1_lazy(tm).
int orc_encode_diagonals_rect_ex(const orc_ctx* c, const double* W, uint32_t m, uint32_t n, double scale, int lazy,
                                 i64* pts) {
  const uint32_t tm = orc_bsgs_t(m, 1), tn = orc_bsgs_t(n, 1), ns = c->N / 2;
  if (tm >= tn || 2 * tn > ns) return -1;
  const uint32_t t1 = lazy ? orc_bsgs_t1_lazy(tm) : orc_bsgs_t1(tm);
  std::vector<double> v(ns);
  for (uint32_t i = 0; i < tm; i++) {
    std::fill(v.begin(), v.end(), 0.0);
    const uint32_t sh = (i / t1) * t1;
    for (uint32_t r = 0; r < tn; r++) {
      const uint32_t row = r % tm, col = (r + i) % tn;
      v[r + sh] = (row < m && col < n) ? W[(size_t)row * n + col] : 0.0;
    }
    int rc = orc_encode(c, v.data(), ns, scale, pts + (size_t)i * c->N);
    if (rc) return rc;
  }
  return 0;
}
int orc_encode_diagonals_rect(const orc_ctx* c, const double* W, uint32_t m, uint32_t n, double scale, i64* pts) {
  return orc_encode_diagonals_rect_ex(c, W, m, n, scale, 0, pts);
}

// Rectangular dense layer on the [x, x] layout over 2 tn slots, with the tm plaintexts of
// orc_encode_diagonals_rect:
//   z' = rescale( sum_k rot_{k t1}( sum_j rd'_{k t1 + j} o rot_j(ct) ) [+ bias] )
// (the composed form of orc_dense over tm diagonals), then for fold >= 1 the sum over the
// tn/tm blocks of z':
//   S = z';  S = S + rot_s(S)  for s = tn/2, tn/4, ..., tm,
// which leaves y[j] in slot j < tm, and for fold = 2 also  S = S + rot_{-tm}(z'),  which
// puts y[j] in slot tm + j as well: the [y, y] layout a following layer of width tm
// reads (the replicate of Sec. 3.1 "Multiple Predictions" taken into the fold).  Other
// slots hold partial sums.  counters: rotations t1+t2-2 + log2(tn/tm) (+1), products tm,
// additions tm-1 + log2(tn/tm) (+1).
// With lazy = 1, z' is the lazy-ModDown form of Eq. (bsgs) over the tm diagonals
// (orc_dense_lazy, diagonals placed for its split) and the fold is the same.
int orc_dense_rect_ex(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, const i64* pts, uint32_t tm,
                      uint32_t tn, const i64* bias, int fold, int lazy, u64* out, u64* counters) {
  if (tm == 0 || tm >= tn || (tm & (tm - 1)) || (tn & (tn - 1)) || fold < 0 || fold > 2 || lvl < 2) return -1;
  const uint32_t lo = lvl - 1;
  const size_t csz = (size_t)2 * lo * c->N;
  std::vector<u64> z(csz), r(csz);
  u64 cnt[3] = {0, 0, 0};
  int rc = lazy ? orc_dense_lazy(c, k, ct, lvl, pts, tm, bias, z.data(), cnt)
                : orc_dense(c, k, ct, lvl, pts, tm, bias, z.data(), cnt);
  if (rc) return rc;
  std::vector<u64> S = z;
  if (fold >= 1) {
    for (uint32_t s = tn / 2; s >= tm; s /= 2) {
      rc = orc_rotate(c, k, S.data(), lo, (int64_t)s, r.data());
      if (rc) return rc;
      orc_add(c, S.data(), r.data(), lo, S.data());
      cnt[0]++;
      cnt[2]++;
    }
    if (fold == 2) {
      rc = orc_rotate(c, k, z.data(), lo, -(int64_t)tm, r.data());
      if (rc) return rc;
      orc_add(c, S.data(), r.data(), lo, S.data());
      cnt[0]++;
      cnt[2]++;
    }
  }
  std::copy(S.begin(), S.end(), out);
  if (counters) { counters[0] = cnt[0]; counters[1] = cnt[1]; counters[2] = cnt[2]; }
  return 0;
}
int orc_dense_rect(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, const i64* pts, uint32_t tm,
                   uint32_t tn, const i64* bias, int fold, u64* out, u64* counters) {
  return orc_dense_rect_ex(c, k, ct, lvl, pts, tm, tn, bias, fold, 0, out, counters);
}

// Replicate: y + rot_{-t}(y), which turns a vector held in slots [0, t) into [y, y].
int orc_replicate(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, uint32_t t, u64* out) {
  std::vector<u64> r((size_t)2 * lvl * c->N);
  int rc = orc_rotate(c, k, ct, lvl, -(int64_t)t, r.data());
  if (rc) return rc;
  return orc_add(c, ct, r.data(), lvl, out);
}

// ---------------------------------------------------------------------------------
// The other layers of the paper's frozen network (Sec. 3.1: "1D Convolutions",
// "Average Pool", "ReLU") and the ciphertext operations they are composed of.
// ---------------------------------------------------------------------------------

// Tensor product of two ciphertexts at the same level: (a0*b0, a0*b1 + a1*b0, a1*b1),
// [3][lvl][N], each a negacyclic schoolbook product per prime.
int orc_tensor(const orc_ctx* c, const u64* a, const u64* b, uint32_t lvl, u64* d) {
  uint32_t N = c->N;
  std::vector<u64> t(N), u(N);
  for (uint32_t i = 0; i < lvl; i++) {
    u64 q = c->mods[i];
    const u64* a0 = a + (size_t)i * N;
    const u64* a1 = a + ((size_t)lvl + i) * N;
    const u64* b0 = b + (size_t)i * N;
    const u64* b1 = b + ((size_t)lvl + i) * N;
    negacyclic_mul(a0, b0, d + (size_t)i * N, N, q);
    negacyclic_mul(a0, b1, t.data(), N, q);
    negacyclic_mul(a1, b0, u.data(), N, q);
    for (uint32_t j = 0; j < N; j++) d[((size_t)lvl + i) * N + j] = addmod(t[j], u[j], q);
    negacyclic_mul(a1, b1, d + ((size_t)2 * lvl + i) * N, N, q);
  }
  return 0;
}

// Ciphertext-ciphertext product (HMult): tensor, relinearise with the s^2 -> s key,
// rescale.  The output scale is scale_a * scale_b / q_{lvl-1}.
int orc_mul(const orc_ctx* c, const orc_keys* k, const u64* a, const u64* b, uint32_t lvl, u64* out) {
  if (lvl < 2) return -1;
  std::vector<u64> d((size_t)3 * lvl * c->N), r((size_t)2 * lvl * c->N);
  orc_tensor(c, a, b, lvl, d.data());
  int rc = orc_relin(c, k, d.data(), lvl, r.data());
  if (rc) return rc;
  return orc_rescale(c, r.data(), lvl, out);
}

// Product with an integer constant C: (C*c0, C*c1) mod every prime.  The constant
// polynomial C decodes to the value C/scale in every slot.
int orc_mul_const(const orc_ctx* c, const u64* ct, uint32_t lvl, i64 C, u64* out) {
  uint32_t N = c->N;
  for (uint32_t p = 0; p < 2; p++)
    for (uint32_t i = 0; i < lvl; i++) {
      u64 q = c->mods[i], cq = from_signed(C, q);
      for (uint32_t j = 0; j < N; j++) {
        size_t o = ((size_t)p * lvl + i) * N + j;
        out[o] = mulmod(ct[o], cq, q);
      }
    }
  return 0;
}

// Sum with an integer constant C in every slot: C is added to the constant coefficient
// of c0 (the plaintext (C, 0, ..., 0)).
int orc_add_const(const orc_ctx* c, const u64* ct, uint32_t lvl, i64 C, u64* out) {
  uint32_t N = c->N;
  memcpy(out, ct, sizeof(u64) * 2 * lvl * N);
  for (uint32_t i = 0; i < lvl; i++) out[(size_t)i * N] = addmod(ct[(size_t)i * N], from_signed(C, c->mods[i]), c->mods[i]);
  return 0;
}

// Level drop: keeps the first `to` limbs of both polynomials, i.e. reduces the
// ciphertext modulo Q_to with no division (the scale is unchanged).
int orc_drop_level(const orc_ctx* c, const u64* ct, uint32_t lvl, uint32_t to, u64* out) {
  uint32_t N = c->N;
  if (to == 0 || to > lvl) return -1;
  for (uint32_t p = 0; p < 2; p++)
    memcpy(out + (size_t)p * to * N, ct + (size_t)p * lvl * N, sizeof(u64) * to * N);
  return 0;
}

// Integer constants of the degree-3 polynomial evaluation below, from the FP64 scale
// bookkeeping (q_a = q_{lvl-1}, q_b = q_{lvl-2}, S = in_scale):
//   S2 = S*S/q_a,  Sw = S2*S/q_b,
//   C3 = round(a3*q_a), C2 = round(a2*S), C1 = round(a1*((Sw*q_a)/S)), C0 = round(a0*Sw),
// rounding half away from zero.  consts[4] = {C0, C1, C2, C3}; *out_scale = Sw.
int orc_poly3_consts(const orc_ctx* c, uint32_t lvl, double in_scale, const double* a, i64* consts,
                     double* out_scale) {
  if (lvl < 3 || lvl > c->L) return -1;
  double qa = (double)c->mods[lvl - 1], qb = (double)c->mods[lvl - 2];
  double S2 = in_scale * in_scale / qa;
  double Sw = S2 * in_scale / qb;
  consts[3] = (i64)llround(a[3] * qa);
  consts[2] = (i64)llround(a[2] * in_scale);
  consts[1] = (i64)llround(a[1] * (Sw * qa / in_scale));
  consts[0] = (i64)llround(a[0] * Sw);
  if (out_scale) *out_scale = Sw;
  return 0;
}

// Degree-3 polynomial a3 z^3 + a2 z^2 + a1 z + a0 at multiplicative depth 2 (Sec. 3.1,
// "ReLU": the paper's ReLU approximation is such a polynomial).  Reading (the paper
// fixes only the polynomial): with z at level lvl and scale S, constants as in
// orc_poly3_consts,
//   z2 = square(z)                                (level lvl-1, scale S2)
//   v  = rescale(C3 * z) + C2                     (level lvl-1, scale S)
//   w  = HMult(z2, v) (tensor, relin, rescale)    (level lvl-2, scale Sw)
//   l  = drop_{lvl-2}(rescale(C1 * z))            (level lvl-2, scale Sw)
//   out = (w + l) + C0                            (level lvl-2, scale Sw)
// so that out decodes to z^2 (a3 z + a2) + a1 z + a0.
int orc_poly3(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, double in_scale, const double* a,
              u64* out, double* out_scale) {
  i64 C[4];
  int rc = orc_poly3_consts(c, lvl, in_scale, a, C, out_scale);
  if (rc) return rc;
  uint32_t N = c->N;
  size_t w1 = (size_t)2 * (lvl - 1) * N, w2 = (size_t)2 * (lvl - 2) * N;
  std::vector<u64> z2(w1), t((size_t)2 * lvl * N), v(w1), w(w2), l1(w1), l(w2);
  if ((rc = orc_square(c, k, ct, lvl, z2.data()))) return rc;
  orc_mul_const(c, ct, lvl, C[3], t.data());
  orc_rescale(c, t.data(), lvl, v.data());
  orc_add_const(c, v.data(), lvl - 1, C[2], v.data());
  if ((rc = orc_mul(c, k, z2.data(), v.data(), lvl - 1, w.data()))) return rc;
  orc_mul_const(c, ct, lvl, C[1], t.data());
  orc_rescale(c, t.data(), lvl, l1.data());
  orc_drop_level(c, l1.data(), lvl - 1, lvl - 2, l.data());
  orc_add(c, w.data(), l.data(), lvl - 2, out);
  return orc_add_const(c, out, lvl - 2, C[0], out);
}

// Average pooling with stride 1 and size f (Sec. 3.1 "Average Pool"): the sum of
// rot_{-i}(x) over i = 0..f-1 (the printed bound "i = 0..f" disagrees with the stated
// f-1 rotations; read as f terms), in increasing i, times the constant
// Cf = round(q_{lvl-1}/f) (the value 1/f at scale q_{lvl-1}), then rescale; the output
// keeps the input scale.  counters[0..2]: rotations, constant products, additions.
int orc_avgpool(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, uint32_t f, u64* out,
                u64* counters) {
  if (lvl < 2 || f == 0) return -1;
  uint32_t N = c->N;
  size_t w = (size_t)2 * lvl * N;
  std::vector<u64> s(ct, ct + w), r(w);
  u64 nrot = 0, nadd = 0;
  for (uint32_t i = 1; i < f; i++) {
    int rc = orc_rotate(c, k, ct, lvl, -(int64_t)i, r.data());
    if (rc) return rc;
    nrot++;
    orc_add(c, s.data(), r.data(), lvl, s.data());
    nadd++;
  }
  i64 Cf = (i64)llround((double)c->mods[lvl - 1] / (double)f);
  orc_mul_const(c, s.data(), lvl, Cf, s.data());
  if (counters) { counters[0] = nrot; counters[1] = 1; counters[2] = nadd; }
  return orc_rescale(c, s.data(), lvl, out);
}

// Plaintexts of the packed single-input single-output 1D convolution (Sec. 3.1 "1D
// Convolutions", after GAZELLE): filter w[f], input of length n held as [x, x] at block
// stride t (slots [0, n) and [t, t+n)).  pt_i has w[i] in the slots s < 2t with
// (s mod t) < n and 0 elsewhere, encoded at `scale`; with `windows` = p > 1 the pattern
// repeats in each window of 2t slots (s < 2t p).
int orc_encode_conv_w(const orc_ctx* c, const double* w, uint32_t f, uint32_t n, uint32_t t, double scale,
                      uint32_t windows, i64* pts) {
  uint32_t ns = c->N / 2;
  if (f == 0 || n == 0 || n > t || windows == 0 || 2 * t * windows > ns) return -1;
  std::vector<double> v(ns);
  for (uint32_t i = 0; i < f; i++) {
    for (uint32_t s = 0; s < ns; s++) v[s] = (s < 2 * t * windows && (s % t) < n) ? w[i] : 0.0;
    int rc = orc_encode(c, v.data(), ns, scale, pts + (size_t)i * c->N);
    if (rc) return rc;
  }
  return 0;
}
int orc_encode_conv(const orc_ctx* c, const double* w, uint32_t f, uint32_t n, uint32_t t, double scale, i64* pts) {
  return orc_encode_conv_w(c, w, f, n, t, scale, 1, pts);
}

// 1D convolution with "same" zero padding: out = sum_{i=0}^{f-1} pt_i o rot_{i-h}(x),
// h = floor((f-1)/2), in increasing i (rot_0 = x), then an optional plaintext bias (on
// c0) and a rescale.  Slot s of the output holds sum_i w[i] x[s+i-h].  counters[0..2]:
// rotations (f-1), plaintext products (f), additions (f-1).
int orc_conv1d(const orc_ctx* c, const orc_keys* k, const u64* ct, uint32_t lvl, const i64* pts, uint32_t f,
               const i64* bias, u64* out, u64* counters) {
  if (lvl < 2 || f == 0) return -1;
  uint32_t N = c->N;
  int64_t h = (int64_t)(f - 1) / 2;
  size_t w = (size_t)2 * lvl * N;
  std::vector<u64> acc(w), r(w), prod(w);
  u64 nrot = 0, nmul = 0, nadd = 0;
  for (uint32_t i = 0; i < f; i++) {
    int64_t o = (int64_t)i - h;
    const u64* src = ct;
    if (o != 0) {
      int rc = orc_rotate(c, k, ct, lvl, o, r.data());
      if (rc) return rc;
      nrot++;
      src = r.data();
    }
    orc_mul_plain(c, src, lvl, pts + (size_t)i * N, prod.data());
    nmul++;
    if (i == 0) acc = prod; else { orc_add(c, acc.data(), prod.data(), lvl, acc.data()); nadd++; }
  }
  if (bias) orc_add_plain(c, acc.data(), lvl, bias, acc.data());
  if (counters) { counters[0] = nrot; counters[1] = nmul; counters[2] = nadd; }
  return orc_rescale(c, acc.data(), lvl, out);
}

}  // extern "C"
