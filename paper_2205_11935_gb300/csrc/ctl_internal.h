// Internal declarations of the ctl library (not part of the C-ABI).
#pragma once
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <map>
#include <mutex>
#include <atomic>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ctl.h"

namespace ctl {

typedef unsigned long long u64;
typedef long long i64;

// ---------------------------------------------------------------------------------
// Per-prime constants, device resident.
// ---------------------------------------------------------------------------------
struct DPrime {
  u64 q;        // the prime
  u64 qinv;     // q^-1 mod 2^64 (Montgomery, positive form)
  u64 r2;       // 2^128 mod q: mulmod_mont(x, r2) = x * 2^64 mod q
  u64 rmod;     // 2^64 mod q: mulmod_mont(x, rmod) = x mod q for any 64-bit x
  u64 ninv, ninv_sh;  // N^-1 mod q and its Shoup companion
  u64 iw1, iw1_sh;    // (psi^-1)^{bitrev(1)} * N^-1: the folded last inverse twiddle
  u64 split;          // kSplitW when q < 2^54 (operands split into kSplitW-bit halves), else 0
  u64 bar;            // floor(2^64 / q) when 2^32 < q (reduce_wide), else 0
};

// Split form of a residue v < 2^54 for the split-half products of the key product and the
// baby-step giant-step sums: (v >> kSplitW) << 32 | (v & (2^kSplitW - 1)).  One width for
// every such prime keeps the shifts compile-time constants; the halves stay below 2^27, so
// a product of two halves is below 2^54 and a Karatsuba middle term below 2^56, leaving
// room for sums of up to 32 terms in 64 bits.
constexpr int kSplitW = 27;

// Fast base conversion from a set of source primes S to target primes:
//   y_i = sum_{j in S} [x_j * Shat_j^-1]_{s_j} * (Shat_j mod t_i)  mod t_i.
// The source limbs arrive with the factor Shat_j^-1 already applied (it is folded into the
// inverse NTT that precedes every conversion), so a conversion is a sum of products with
// the constants Shat_j mod t_i, taken in Shoup form.
struct ConvTab {
  int ns;               // |S|
  int nt;               // number of target positions
  const u64* c;         // [ns][nt] Shat_j mod t_i
  const u64* c_sh;      // [ns][nt] floor(c * 2^64 / t_i)
};

// Rescale constants for dropping the last prime of a level-lvl ciphertext.
struct RescaleTab {
  const u64* inv;     // [lvl-1] q_last^-1 mod q_i
  const u64* inv_sh;  // [lvl-1]
  const u64* hmod;    // [lvl-1] floor(q_last/2) mod q_i
  u64 qlast, h;
};

// Keys and Galois elements of the rotations served by one key-switching launch, passed
// by value as a kernel parameter (no host-to-device copy on the hot path).
#define CTL_MAX_ROT 64
struct RotList {
  int n;
  const u64* key[CTL_MAX_ROT];  // device key [beta][2][L+K][N] (Montgomery, NTT form)
  u64 g[CTL_MAX_ROT];           // Galois element (1 = no automorphism)
  u64 ginv[CTL_MAX_ROT];        // g^-1 mod 2N (filled by the key-product launcher)
};

// Last-stage constants of an inverse NTT that also multiplies its output by a per-prime
// factor c (c * N^-1 and c * (psi^-1)^bitrev(1) * N^-1 with Shoup companions): folding
// the factor Shat_j^-1 of a base conversion into the transform that precedes it.
struct InvScale {
  u64 ninv, ninv_sh, iw1, iw1_sh;
};

// ModDown constants (special primes P -> data primes).
struct ModDownTab {
  ConvTab conv;       // S = special primes, targets = data primes 0..L-1
  const u64* pinv;    // [L] P^-1 mod q_i
  const u64* pinv_sh; // [L]
  const u64* pmod;    // [L] P mod q_i
  const u64* pmod_sh; // [L]
};

// ---------------------------------------------------------------------------------
// Host-side mathematics (host_math.cpp).
// ---------------------------------------------------------------------------------
bool plan_primes(uint32_t N, const std::vector<uint32_t>& bits, std::vector<u64>& out);
u64 min_primitive_2n_root(u64 q, uint32_t N);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_invmod(u64 a, u64 q);
u64 h_shoup(u64 w, u64 q);        // floor(w * 2^64 / q)
u64 h_mont(u64 x, u64 q);         // x * 2^64 mod q
u64 h_neg_inv64(u64 q);           // q^-1 mod 2^64
uint32_t h_bitrev(uint32_t x, uint32_t logn);

// SplitMix64 streams and the samplers of the key/encryption randomness.
struct SplitMixStream {
  u64 key, ctr;
  SplitMixStream(u64 seed, u64 stream);
  u64 next();
};
u64 stream_id_secret();
u64 stream_id_key_a(u64 key_id, u64 digit, u64 limb);
u64 stream_id_key_e(u64 key_id, u64 digit);
u64 stream_id_enc_a(u64 limb);
u64 stream_id_enc_e();
void draw_uniform(SplitMixStream& st, u64 q, uint32_t N, u64* out);
void draw_ternary(SplitMixStream& st, uint32_t N, i64* out);
void draw_cbd21(SplitMixStream& st, uint32_t N, i64* out);

// FP64 canonical-embedding encoder (radix-2 complex FFT).
struct Encoder {
  uint32_t N = 0;
  std::vector<uint32_t> slot_pos;   // odd-power index (e-1)/2 of slot j, e = 5^j mod 2N
  std::vector<uint32_t> conj_pos;   // index of the conjugate root -5^j
  std::vector<double> cs, sn;       // cos/sin(2*pi*k/N)
  std::vector<double> zc, zs;       // cos/sin(pi*k/N): the twist zeta^k
  void init(uint32_t n);
  // m_k = round(scale * (2/N) * Re sum_j z_j zeta^(-5^j k)); returns false on overflow.
  bool encode(const double* z, size_t nz, double scale, i64* m) const;
  // The same coefficients for any scale (up to 2^1000), as residues modulo the lvl primes
  // moduli[0..lvl): out[i][k] = round(m_k) mod q_i, rounding half away from zero (a value
  // of 2^53 or more is already an integer in FP64 and is reduced exactly).
  bool encode_rns(const double* z, size_t nz, double scale, const u64* moduli, uint32_t lvl, u64* out) const;
  // z_j = Re( sum_k m_k zeta^(5^j k) ) / scale for j < nz.
  void decode(const double* m, size_t nz, double scale, double* z) const;
 private:
  void fft(std::vector<double>& re, std::vector<double>& im, bool inverse) const;
};

// Centred CRT of residues over the first lvl primes, returned as double.
void crt_centred_to_double(const u64* res, size_t stride, uint32_t lvl, const u64* primes, size_t N, double* out);

// ---------------------------------------------------------------------------------
// Launch statistics (kernel launches and per-class device time).
// ---------------------------------------------------------------------------------
enum KernelClass {
  KC_NTT_FWD = 0, KC_NTT_INV, KC_MODUP, KC_KEYIP, KC_MODDOWN, KC_RESCALE, KC_BSGS, KC_ELEM, KC_COUNT
};
extern const char* kKernelClassName[KC_COUNT];

struct Timing {
  bool enabled = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> pool;
  double ms[KC_COUNT] = {0};
  uint64_t launches[KC_COUNT] = {0};
  double work[KC_COUNT] = {0};   // algorithmic units (modmul or MAC) attributed to the class
  double bytes[KC_COUNT] = {0};  // algorithmic HBM bytes (each operand read once, each result written once)
};

}  // namespace ctl

// ---------------------------------------------------------------------------------
// Opaque handles of the C-ABI.
// ---------------------------------------------------------------------------------
namespace ctl {
struct ClientTabs;
}  // namespace ctl

struct ctl_context {
  uint32_t N = 0, logN = 0, L = 0, K = 0, alpha = 1, beta = 1;
  double scale = 0;
  uint64_t seed = 0;
  std::vector<ctl::u64> moduli;   // L data primes then K special primes
  int device = 0, sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ctl_alloc_fn alloc_fn = nullptr;
  ctl_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  // device tables
  ctl::DPrime* d_primes = nullptr;
  ctl::u64* d_tw2 = nullptr;     // [L+K][N][2] forward twiddles (psi^{bitrev(i)}, Shoup companion)
  ctl::u64* d_itw2 = nullptr;    // [L+K][N][2] inverse twiddles ((psi^-1)^{bitrev(i)}, Shoup companion)
  ctl::u64* d_tables = nullptr;  // conversion / rescale constants
  std::vector<ctl::ConvTab> modup_tabs;      // index (lvl-1)*beta + d
  std::vector<ctl::RescaleTab> rescale_tabs; // index lvl (valid for lvl >= 2)
  ctl::ModDownTab moddown;
  ctl::InvScale* d_md_scale = nullptr;  // [L+K]: factor Phat_j^-1 on the special primes
  ctl::InvScale* d_mu_scale = nullptr;  // [L][L+K]: level lvl's factor Qhat_i^-1 on data prime i
  std::vector<ctl::DPrime> h_primes;
  ctl::Encoder enc;
  ctl::Timing timing;
  std::atomic<uint64_t> launch_count{0};
  uint64_t op_rot = 0, op_ptmul = 0, op_add = 0, op_relin = 0, op_rescale = 0;
  int ntt_shape_fwd = CTL_NTT_SHAPE_R32, ntt_shape_inv = CTL_NTT_SHAPE_R32;  // ctl_set_ntt_shape / autotune
  int dense_mode = CTL_DENSE_COMPOSED;          // ctl_set_dense_mode
  int bsgs_chunk = 32, bsgs_karatsuba = 1;      // ctl_set_bsgs_shape (measured fastest)
  uint64_t ks_budget = 16ull << 30;              // ctl_set_keyswitch_budget
  uint32_t windows = 1;                          // ctl_set_windows: prediction windows per ciphertext
  const ctl_context* parent = nullptr;  // clones share the parent's device tables
  ctl::ClientTabs* client = nullptr;    // GPU encoder / sampler / CRT tables (client.cu)
};

namespace ctl {
inline size_t ct_words(const ctl_context* c, uint32_t lvl, uint32_t count) { return (size_t)count * 2 * lvl * c->N; }
}  // namespace ctl

struct ctl_keys {
  ctl_context* ctx = nullptr;
  std::vector<ctl::i64> s;               // ternary secret (host)
  ctl::u64* d_s = nullptr;               // [L+K][N] NTT form, plain residues
  // key_id -> device key [beta][2][L+K][N], NTT form, Montgomery form
  std::map<ctl::u64, ctl::u64*> evk;
  size_t key_bytes = 0;
};

struct ctl_ct {
  ctl_context* ctx = nullptr;
  ctl::u64* d = nullptr;    // [count][2][level][N], NTT form
  uint32_t level = 0;       // live data primes
  uint32_t count = 1;       // ciphertexts in this batch
  double scale = 0;
  size_t bytes = 0;
};

namespace ctl {

// NVTX range over a scope (one per model layer and per key switch), for profilers that
// attach to the process (ncu --nvtx); without a tool the push and pop are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// ---------------------------------------------------------------------------------
// Memory and error helpers (ctl_api.cu).
// ---------------------------------------------------------------------------------
void* dev_alloc(ctl_context* c, size_t bytes);
void dev_free(ctl_context* c, void* p);

// Device buffer of `words` 64-bit words from the context's allocator, released
// (stream-ordered) at scope exit.
struct DBuf {
  ctl_context* c = nullptr;
  u64* p = nullptr;
  DBuf() = default;
  DBuf(ctl_context* cc, size_t words) : c(cc) { p = (u64*)dev_alloc(cc, words * sizeof(u64)); }
  ~DBuf() {
    if (p) dev_free(c, p);
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  u64* release() {
    u64* r = p;
    p = nullptr;
    return r;
  }
};
#define CHECK_ALLOC(buf)                     \
  do {                                       \
    if (!(buf).p) {                          \
      set_error("device allocation failed"); \
      return CTL_ENOMEM;                     \
    }                                        \
  } while (0)
// A new ciphertext handle [count][2][lvl][N] at `scale` (null when allocation fails).
ctl_ct* new_ct(ctl_context* c, uint32_t lvl, uint32_t count, double scale);
inline size_t ct_words(const ctl_context* c, uint32_t lvl, uint32_t count);
// The client tables (client.cu): created with the context for N <= 16384.
struct ClientTabs;
int client_tables_create(ctl_context* c);
void client_tables_destroy(ctl_context* c);
// Batch encryption of integer plaintexts m [count][N] (device) with the device sampler, and
// decryption to centred coefficient values [count][N] (device doubles) (client.cu).
int encrypt_coeffs_dev(ctl_context* c, const ctl_keys* k, const i64* m_dev, uint32_t count, const u64* seeds,
                       ctl_ct** out);
int decrypt_coeffs_dev(ctl_context* c, const ctl_keys* k, const ctl_ct* ct, double* m_dev);
void set_error(const char* fmt, ...);
int cuda_check(cudaError_t e, const char* what);
inline int last_cuda(const char* what) { return cuda_check(cudaGetLastError(), what); }
void timing_begin(ctl_context* c, int cls, cudaEvent_t* ev);
void timing_end(ctl_context* c, int cls, cudaEvent_t ev, double work, double bytes = 0.0);

inline uint32_t prime_of_limb(uint32_t l, uint32_t lvl, uint32_t L) { return l < lvl ? l : L + (l - lvl); }

// ---------------------------------------------------------------------------------
// Kernel launchers (ntt.cu, ntt_modup.cu, ntt_moddown.cu, ntt_giant.cu, kernels.cu).  All operate on the context stream.
// Layout conventions: a "poly" is [limbs][N]; polys are spaced by poly_stride words.
// A limb l of a poly of a level-lvl object maps to prime prime_of_limb(l, lvl, L).
// ---------------------------------------------------------------------------------
// In-place forward / inverse NTT of limbs [limb_lo, limb_hi) of n_polys polys.
void launch_ntt_fwd(ctl_context* c, u64* data, size_t poly_stride, int n_polys, int limb_lo, int limb_hi, int lvl);
void launch_ntt_inv(ctl_context* c, u64* data, size_t poly_stride, int n_polys, int limb_lo, int limb_hi, int lvl);
// Inverse NTT of limb lvl-1 of each poly, writing r = [x + floor(q/2)]_q (coefficient form)
// to r_out[p][N].
void launch_intt_rescale_last(ctl_context* c, const u64* in, size_t poly_stride, int n_polys, int lvl, u64* r_out);
// Rescale combine: out[p][i] = (in[p][i] - NTT_i((r - h) mod q_i)) * q_last^-1 for i < lvl-1.
void launch_rescale_ntt(ctl_context* c, const u64* r, const u64* in, size_t in_stride, u64* out, size_t out_stride,
                        int n_polys, int lvl);
// ModUp of c1 (coefficient form src_coef, NTT form src_ntt; polys spaced by src_stride)
// into ext[b][d][E][N] (NTT form), E = lvl + K, for all live digits d.  Limbs whose prime
// has a split width w are stored split, (v >> w) << 32 | (v & (2^w - 1)), for the key product.
void launch_modup_ntt(ctl_context* c, const u64* src_coef, size_t coef_stride, const u64* src_ntt, size_t src_stride,
                      int nb, int lvl, u64* ext);
// Key inner products with automorphism: for rotation r (g[r], key[r]) and batch b:
//   acc[r][b][t][i][k] = sum_d ext_r[b][d][i][perm_g(k)] * key_r[d][t][prime(i)][k],
// ext_r = ext + r * ext_r_stride (0 when the ModUp is shared by all rotations).
// With add_pc0 set, output poly t = 0 on the data limbs also gets sigma_g(P * c0), with the
// data limbs of P * c0 for input b at add_pc0 + b*add_b (NTT form, [lvl][N], residues in
// [0, q_i), as launch_scale_to_ext writes them): the baby step of a rotation kept in the
// extended basis.
void launch_key_ip(ctl_context* c, const u64* ext, size_t ext_r_stride, int nb, int lvl, const RotList& rl, u64* acc,
                   const u64* add_pc0 = nullptr, size_t add_b = 0);
// Key inner products of nr = rl.n rotations summed into S in the extended basis:
//   S[b][0] += sum_r ( ip_r[b][0] + sigma_{g_r}(add[r][b]) ),  S[b][1] += sum_r ip_r[b][1],
// ext_r = ext + r*ext_r_stride ([nb][nd][E][N] each), add[r][b] = add + r*add_r + b*add_b
// ([E][N]), S[b] = S + b*s_b ([2][E][N]).
void launch_key_ip_acc(ctl_context* c, const u64* ext, size_t ext_r_stride, int nb, int lvl, const RotList& rl,
                       const u64* add, size_t add_r, size_t add_b, u64* S, size_t s_b);
// Extended-basis image of a batch: out[b][t] ([E][N]) = P * in[b][t] on the data limbs,
// 0 on the special limbs; in [nb][2][lvl][N].
void launch_scale_to_ext(ctl_context* c, const u64* in, u64* out, int nb, int lvl);
// ModDown after the special limbs of acc [nr][nb][2][E][N] were inverse-transformed in
// place: out[p][i] = (acc[p][i] - NTT_i(conv_i(acc[p][specials]))) * P^-1 (+ addend),
// out [nr][nb][2][lvl][N].  Addend of output (r, b, t): addend + r*add_r + b*add_b + t*add_p
// read through sigma_{g_r}; t = 1 gets one only if add_both.  With accum (nr = 1 only),
// out += result instead of out = result.
void launch_moddown_ntt(ctl_context* c, const u64* acc, int nr, int nb, int lvl, u64* out, const u64* addend,
                        size_t add_r, size_t add_b, size_t add_p, bool add_both, const RotList& rl,
                        bool accum = false);
// Sum of the ModDowns of nr key-switching results (the giant steps of a dense layer),
// without one NTT per result: the ModDown of acc_r is (acc_r - NTT(conv_r)) * P^-1 on the
// data limbs, with conv_r the base conversion of its special limbs, and the NTT is
// linear, so the sum over r needs sum_r acc_r (NTT form) and sum_r conv_r (coefficient
// form) only.  Accumulates over the nr results of acc [nr][nb][2][E][N] (special limbs
// inverse-transformed in place, conversion factors folded in):
//   D[b][t][l] += sum_r acc_r[b][t][l],  C[b][t][l] += sum_r conv_r[b][t][l],
//   A[b][l] += sum_r sigma_{g_r}(addend_r[b])[l] (addend of rotation r at addend + r*add_r
//   + b*add_b), all [nb][2 or 1][lvl][N]; first: D, C, A are set instead of added to.
void launch_giant_accum(ctl_context* c, const u64* acc, int nr, int nb, int lvl, const RotList& rl,
                        const u64* addend, size_t add_r, size_t add_b, u64* D, u64* C, u64* A, bool first);
// out[b][t] += (D[b][t] - NTT(C[b][t])) * P^-1 + (t == 0 ? A[b] : 0) for the sums above.
void launch_giant_moddown(ctl_context* c, const u64* D, const u64* C, const u64* A, int nb, int lvl, u64* out);
// ModDown of n_polys extended polys spaced by acc_stride (special limbs already
// inverse-transformed in place, as above) into out + p*out_stride ([lvl][N]), no addend.
void launch_moddown_polys(ctl_context* c, const u64* acc, size_t acc_stride, int n_polys, int lvl, u64* out,
                          size_t out_stride);
// Out-of-place inverse NTT; with scl, limb output of prime pi is also multiplied by the
// factor folded into scl[pi].
void launch_ntt_inv_oop(ctl_context* c, const u64* src, size_t src_stride, u64* dst, size_t dst_stride, int n_polys,
                        int limb_lo, int limb_hi, int lvl, const InvScale* scl = nullptr);

// Elementwise (kernels.cu).
void launch_add(ctl_context* c, const u64* a, const u64* b, u64* out, int n_polys, int lvl, size_t stride_a,
                size_t stride_b, size_t stride_o);
void launch_sub(ctl_context* c, const u64* a, const u64* b, u64* out, int n_polys, int lvl, size_t stride_a,
                size_t stride_b, size_t stride_o);
// out = ct * pt_mont (pt in Montgomery form, [lvl_pt][N], same for every poly).
void launch_mul_plain(ctl_context* c, const u64* ct, const u64* pt, u64* out, int n_polys, int lvl,
                      size_t stride_ct, size_t stride_o);
// out = ct + pt on poly 0 of each ciphertext.
void launch_add_plain(ctl_context* c, u64* ct, const u64* pt, int n_ct, int lvl, size_t ct_stride);
// (a0,a1) -> (a0^2, 2 a0 a1, a1^2) for each of nb ciphertexts; d layout [nb][3][lvl][N].
void launch_tensor_square(ctl_context* c, const u64* ct, u64* d, int nb, int lvl);
// Montgomery form conversion of limbs (to: x*R, from: x*R^-1).
void launch_to_mont(ctl_context* c, u64* data, int n_polys, int limbs, int lvl, size_t stride, bool to);
// Signed integer polynomial -> residues [limbs][N] with limb prime map (lvl, L).
void launch_from_signed(ctl_context* c, const i64* src, u64* dst, int n_polys, int limbs, int lvl, size_t src_stride,
                        size_t dst_stride);
// Key assembly: b = -a*s + e + gadget_i * s' (NTT form), then Montgomery form of b and a.
void launch_keygen_combine(ctl_context* c, u64* key, const u64* s_ntt, const u64* e_ntt, const u64* sp_ntt, int beta,
                           int alpha, const u64* pmod);
// Encryption: c0 = -a*s + m + e at each limb; inputs NTT form; c1 = a already in place.
void launch_encrypt_combine(ctl_context* c, u64* ct, const u64* s_ntt, const u64* me_ntt, int lvl);
// Decryption: out = c0 + c1 * s (NTT form) for nb ciphertexts -> out [nb][lvl][N].
void launch_decrypt_mul(ctl_context* c, const u64* ct, const u64* s_ntt, u64* out, int nb, int lvl);
// Automorphism of a whole object in the NTT domain.
void launch_automorph(ctl_context* c, const u64* in, u64* out, int n_polys, int limbs, int lvl, size_t stride, u64 g);
// Baby-step giant-step inner sums over polys of `limbs` limbs (prime map (lvl, L)):
//   inner[k][b][p][i] = sum_j diag[k*t1+j][i] * baby[j][b][p][i]   (diag in Montgomery form)
// wino: the diagonal pair terms of launch_bsgs_wino_diag ([t2][limbs][N]) for the
// Winograd form of the Karatsuba shape (t1 >= 2).
void launch_bsgs_inner(ctl_context* c, const u64* baby, const u64* diag, size_t diag_stride, const u64* wino,
                       u64* inner, int t1, int t2, int nb, int limbs, int lvl);
void launch_bsgs_wino_diag(ctl_context* c, const u64* diag, size_t diag_stride, u64* wino, int t1, int t2, int limbs,
                           int lvl);
// Re-pack Montgomery-form plaintext limbs [cnt][limbs][N] (prime map (lvl, L)) for the
// split product: on limbs whose prime has split width w > 0,
// v -> (v >> w) << 32 | (v & (2^w - 1)).
void launch_split_limbs(ctl_context* c, u64* data, int cnt, int limbs, int lvl);

// Kernels of the other layers of the paper's network (kernels.cu).
// Per-limb constants passed by value: m[i] a multiplier in Montgomery form
// (m_plain * 2^64 mod q_i), a[i] an addend residue.  Levels above kMaxConstLimbs are
// refused by the callers.
constexpr int kMaxConstLimbs = 64;
struct LimbConsts {
  u64 m[kMaxConstLimbs];
  u64 a[kMaxConstLimbs];
};
// (a, b) -> (a0 b0, a0 b1 + a1 b0, a1 b1) for nb ciphertext pairs; d [nb][3][lvl][N].
void launch_tensor2(ctl_context* c, const u64* a, const u64* b, u64* d, int nb, int lvl);
// out[pp] = in[pp] * m (if has_m) + add[pp] (if add non-null) + (pp even ? a : 0), for
// n_polys polys (two per ciphertext, poly 0 first) spaced by s_in / s_add / s_out words.
void launch_affine(ctl_context* c, const u64* in, size_t s_in, const u64* add, size_t s_add, u64* out, size_t s_out,
                   const LimbConsts& K, bool has_m, int n_polys, int lvl);
// out = (x + sum_{r < nr} rots[r]) * m, x and out [nb][2][lvl][N], rots [nr][nb][2][lvl][N].
void launch_sum_scale(ctl_context* c, const u64* x, const u64* rots, int nr, u64* out, const LimbConsts& K, int nb,
                      int lvl);
// out = sum_{i < f} rots[i] o pts[i] (pts [f][lvl][N], Montgomery form), in increasing i.
void launch_pt_mac(ctl_context* c, const u64* rots, const u64* pts, int f, u64* out, int nb, int lvl);

}  // namespace ctl
