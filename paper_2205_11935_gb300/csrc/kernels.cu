// Element-wise kernels of the CKKS server path (NTT domain), the key-switching inner
// product and the baby-step giant-step inner sums of Eq. (bsgs).
//
// All products are exact: Montgomery reduction of 128-bit accumulators against
// operands stored in Montgomery form (keys, diagonal plaintexts), so a lazy sum of
// several 64x64-bit products costs one reduction.
#include <algorithm>

#include "ctl_internal.h"
#include "modarith.cuh"

namespace ctl {

__device__ __forceinline__ uint32_t brv_k(uint32_t x, int logn) { return __brev(x) >> (32 - logn); }
__device__ __forceinline__ uint32_t auto_src_k(uint32_t k, u64 g, int logN) {
  uint32_t e = 2u * brv_k(k, logN) + 1u;
  uint32_t e2 = (uint32_t)(((u64)e * g) & ((2ull << logN) - 1));
  return brv_k((e2 - 1u) >> 1, logN);
}

static const int kThreads = 256;

static int elem_grid(ctl_context* c, size_t total) {
  size_t g = (total + kThreads - 1) / kThreads;
  size_t cap = (size_t)c->sm_count * 16;
  return (int)(g < cap ? g : cap);
}

// A launch with its algorithmic work (modmul or MAC units) and HBM bytes for the
// per-class rooflines; CTL_LAUNCH counts no bytes.
#define CTL_LAUNCH_C(cls, work, bytes, grid, ...) \
  do {                                            \
    cudaEvent_t ev__;                             \
    timing_begin(c, cls, &ev__);                  \
    __VA_ARGS__;                                  \
    c->launch_count++;                            \
    timing_end(c, cls, ev__, work, bytes);        \
  } while (0)
#define CTL_LAUNCH(cls, work, grid, ...) CTL_LAUNCH_C(cls, work, 0.0, grid, __VA_ARGS__)

// ---------------------------------------------------------------------------------
// add / sub over n_polys polys of lvl limbs (limb i -> prime i).
// ---------------------------------------------------------------------------------
template <bool SUB>
__global__ void k_addsub(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ o,
                         const DPrime* __restrict__ pr, int logN, int lvl, size_t total, size_t sa, size_t sb,
                         size_t so) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / (lvl * N), r = idx % (lvl * N);
    const int i = (int)(r >> logN);
    const u64 q = pr[i].q;
    const u64 x = a[p * sa + r], y = b[p * sb + r];
    o[p * so + r] = SUB ? submod(x, y, q) : addmod(x, y, q);
  }
}

void launch_add(ctl_context* c, const u64* a, const u64* b, u64* out, int n_polys, int lvl, size_t sa, size_t sb,
                size_t so) {
  size_t total = (size_t)n_polys * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g, (k_addsub<false><<<g, kThreads, 0, c->stream>>>(a, b, out, c->d_primes, (int)c->logN, lvl,
                                                                          total, sa, sb, so)));
}
void launch_sub(ctl_context* c, const u64* a, const u64* b, u64* out, int n_polys, int lvl, size_t sa, size_t sb,
                size_t so) {
  size_t total = (size_t)n_polys * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g, (k_addsub<true><<<g, kThreads, 0, c->stream>>>(a, b, out, c->d_primes, (int)c->logN, lvl,
                                                                         total, sa, sb, so)));
}

// ---------------------------------------------------------------------------------
// Plaintext product (pt in Montgomery form, NTT domain) and plaintext addition.
// ---------------------------------------------------------------------------------
__global__ void k_mul_plain(const u64* __restrict__ ct, const u64* __restrict__ pt, u64* __restrict__ o,
                            const DPrime* __restrict__ pr, int logN, int lvl, size_t total, size_t sc, size_t so) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / (lvl * N), r = idx % (lvl * N);
    const int i = (int)(r >> logN);
    o[p * so + r] = mulmod_mont(ct[p * sc + r], pt[r], pr[i].q, pr[i].qinv);
  }
}
void launch_mul_plain(ctl_context* c, const u64* ct, const u64* pt, u64* out, int n_polys, int lvl, size_t sc,
                      size_t so) {
  size_t total = (size_t)n_polys * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, (double)total, g,
             (k_mul_plain<<<g, kThreads, 0, c->stream>>>(ct, pt, out, c->d_primes, (int)c->logN, lvl, total, sc, so)));
}

__global__ void k_add_plain(u64* ct, const u64* __restrict__ pt, const DPrime* __restrict__ pr, int logN, int lvl,
                            size_t total, size_t sc) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx / (lvl * N), r = idx % (lvl * N);
    const int i = (int)(r >> logN);
    ct[b * sc + r] = addmod(ct[b * sc + r], pt[r], pr[i].q);
  }
}
void launch_add_plain(ctl_context* c, u64* ct, const u64* pt, int n_ct, int lvl, size_t ct_stride) {
  size_t total = (size_t)n_ct * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_add_plain<<<g, kThreads, 0, c->stream>>>(ct, pt, c->d_primes, (int)c->logN, lvl, total, ct_stride)));
}

// ---------------------------------------------------------------------------------
// Tensor of a ciphertext with itself: (c0^2, 2 c0 c1, c1^2).
// ---------------------------------------------------------------------------------
__global__ void k_tensor_sq(const u64* __restrict__ ct, u64* __restrict__ d, const DPrime* __restrict__ pr, int logN,
                            int lvl, size_t total) {
  const size_t N = (size_t)1 << logN;
  const size_t LN = (size_t)lvl * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx / LN, r = idx % LN;
    const int i = (int)(r >> logN);
    const DPrime P = pr[i];
    const u64 a0 = ct[b * 2 * LN + r], a1 = ct[b * 2 * LN + LN + r];
    const u64 a0m = mulmod_mont(a0, P.r2, P.q, P.qinv);  // a0 * R
    const u64 a1m = mulmod_mont(a1, P.r2, P.q, P.qinv);  // a1 * R
    const u64 x01 = mulmod_mont(a1, a0m, P.q, P.qinv);
    d[b * 3 * LN + r] = mulmod_mont(a0, a0m, P.q, P.qinv);
    d[b * 3 * LN + LN + r] = addmod(x01, x01, P.q);
    d[b * 3 * LN + 2 * LN + r] = mulmod_mont(a1, a1m, P.q, P.qinv);
  }
}
void launch_tensor_square(ctl_context* c, const u64* ct, u64* d, int nb, int lvl) {
  size_t total = (size_t)nb * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 5.0 * total, g,
             (k_tensor_sq<<<g, kThreads, 0, c->stream>>>(ct, d, c->d_primes, (int)c->logN, lvl, total)));
}

// ---------------------------------------------------------------------------------
// Montgomery form conversion and signed-integer import.
// ---------------------------------------------------------------------------------
__global__ void k_mont(u64* data, const DPrime* __restrict__ pr, int logN, int limbs, int lvl, int L, size_t total,
                       size_t stride, bool to) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / (limbs * N), r = idx % (limbs * N);
    const int l = (int)(r >> logN);
    const int pi = l < lvl ? l : L + (l - lvl);
    const DPrime P = pr[pi];
    u64& v = data[p * stride + r];
    v = to ? mulmod_mont(v, P.r2, P.q, P.qinv) : redc(0, v, P.q, P.qinv);
  }
}
void launch_to_mont(ctl_context* c, u64* data, int n_polys, int limbs, int lvl, size_t stride, bool to) {
  size_t total = (size_t)n_polys * limbs * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_mont<<<g, kThreads, 0, c->stream>>>(data, c->d_primes, (int)c->logN, limbs, lvl, (int)c->L, total,
                                                    stride, to)));
}

__global__ void k_from_signed(const i64* __restrict__ src, u64* __restrict__ dst, const DPrime* __restrict__ pr,
                              int logN, int limbs, int lvl, int L, size_t total, size_t ss, size_t ds) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / (limbs * N), r = idx % (limbs * N);
    const int l = (int)(r >> logN);
    const size_t k = r & (N - 1);
    const int pi = l < lvl ? l : L + (l - lvl);
    const DPrime P = pr[pi];
    const i64 v = src[p * ss + k];
    const u64 a = v >= 0 ? (u64)v : (u64)(-(v + 1)) + 1ull;
    const u64 m = mulmod_mont(a, P.rmod, P.q, P.qinv);  // a mod q
    dst[p * ds + r] = v >= 0 ? m : negmod(m, P.q);
  }
}
void launch_from_signed(ctl_context* c, const i64* src, u64* dst, int n_polys, int limbs, int lvl, size_t ss,
                        size_t ds) {
  size_t total = (size_t)n_polys * limbs * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_from_signed<<<g, kThreads, 0, c->stream>>>(src, dst, c->d_primes, (int)c->logN, limbs, lvl, (int)c->L,
                                                           total, ss, ds)));
}

// ---------------------------------------------------------------------------------
// Key generation: key [beta][2][LK][N] holds a in poly 1 (NTT form) on entry; e_ntt is
// [beta][LK][N]; sp_ntt [LK][N] is s'; pmod[i] = P mod q_i.  Writes
//   b = -a*s + e + [i in digit d] * (P mod q_i) * s'   and converts b and a to Montgomery form.
// ---------------------------------------------------------------------------------
__global__ void k_keygen(u64* key, const u64* __restrict__ s, const u64* __restrict__ e, const u64* __restrict__ sp,
                         const u64* __restrict__ pmod, const DPrime* __restrict__ pr, int logN, int LK, int L,
                         int alpha, size_t total) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t d = idx / (LK * N), r = idx % (LK * N);
    const int i = (int)(r >> logN);
    const DPrime P = pr[i];
    u64* b0 = key + (d * 2) * LK * N + r;
    u64* b1 = key + (d * 2 + 1) * LK * N + r;
    const u64 a = *b1;
    const u64 as = mulmod_plain(a, s[r], P.q, P.qinv, P.r2);
    u64 v = submod(e[d * LK * N + r], as, P.q);
    const bool in_digit = (i < L) && (i >= (int)d * alpha) && (i < ((int)d + 1) * alpha);
    if (in_digit) v = addmod(v, mulmod_plain(pmod[i], sp[r], P.q, P.qinv, P.r2), P.q);
    *b0 = mulmod_mont(v, P.r2, P.q, P.qinv);
    *b1 = mulmod_mont(a, P.r2, P.q, P.qinv);
  }
}
void launch_keygen_combine(ctl_context* c, u64* key, const u64* s_ntt, const u64* e_ntt, const u64* sp_ntt, int beta,
                           int alpha, const u64* pmod) {
  const int LK = (int)(c->L + c->K);
  size_t total = (size_t)beta * LK * c->N;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_keygen<<<g, kThreads, 0, c->stream>>>(key, s_ntt, e_ntt, sp_ntt, pmod, c->d_primes, (int)c->logN,
                                                      LK, (int)c->L, alpha, total)));
}

// ---------------------------------------------------------------------------------
// Encryption / decryption arithmetic.
// ---------------------------------------------------------------------------------
__global__ void k_encrypt(u64* ct, const u64* __restrict__ s, const u64* __restrict__ me,
                          const DPrime* __restrict__ pr, int logN, int lvl, size_t total) {
  const size_t N = (size_t)1 << logN;
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < total; r += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(r >> logN);
    const DPrime P = pr[i];
    const u64 a = ct[(size_t)lvl * N + r];
    ct[r] = submod(me[r], mulmod_plain(a, s[r], P.q, P.qinv, P.r2), P.q);
  }
}
void launch_encrypt_combine(ctl_context* c, u64* ct, const u64* s_ntt, const u64* me_ntt, int lvl) {
  size_t total = (size_t)lvl * c->N;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_encrypt<<<g, kThreads, 0, c->stream>>>(ct, s_ntt, me_ntt, c->d_primes, (int)c->logN, lvl, total)));
}

__global__ void k_decrypt(const u64* __restrict__ ct, const u64* __restrict__ s, u64* __restrict__ out,
                          const DPrime* __restrict__ pr, int logN, int lvl, size_t total) {
  const size_t N = (size_t)1 << logN;
  const size_t LN = (size_t)lvl * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx / LN, r = idx % LN;
    const int i = (int)(r >> logN);
    const DPrime P = pr[i];
    out[idx] = addmod(ct[b * 2 * LN + r], mulmod_plain(ct[b * 2 * LN + LN + r], s[r], P.q, P.qinv, P.r2), P.q);
  }
}
void launch_decrypt_mul(ctl_context* c, const u64* ct, const u64* s_ntt, u64* out, int nb, int lvl) {
  size_t total = (size_t)nb * lvl * c->N;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_decrypt<<<g, kThreads, 0, c->stream>>>(ct, s_ntt, out, c->d_primes, (int)c->logN, lvl, total)));
}

// ---------------------------------------------------------------------------------
// Automorphism sigma_g of whole polys in the NTT domain (a gather).
// ---------------------------------------------------------------------------------
__global__ void k_automorph(const u64* __restrict__ in, u64* __restrict__ out, int logN, int limbs, size_t total,
                            size_t stride, u64 g) {
  const size_t N = (size_t)1 << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / (limbs * N), r = idx % (limbs * N);
    const size_t l = r >> logN, k = r & (N - 1);
    out[p * stride + r] = in[p * stride + l * N + auto_src_k((uint32_t)k, g, logN)];
  }
}
void launch_automorph(ctl_context* c, const u64* in, u64* out, int n_polys, int limbs, int, size_t stride, u64 g) {
  size_t total = (size_t)n_polys * limbs * c->N;
  int gr = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, gr,
             (k_automorph<<<gr, kThreads, 0, c->stream>>>(in, out, (int)c->logN, limbs, total, stride, g)));
}

// ---------------------------------------------------------------------------------
// Key-switching inner product with the automorphism folded into the gather.
//   acc[r][b][t][i][k] = sum_{d < nd} ext[b][d][i][src_g(k)] * key_r[d][t][prime(i)][k]
// Key values are in Montgomery form, so one REDC yields the plain residue.  The 128-bit
// sum of nd products stays below q * 2^64 when nd * q < 2^64 (REDC precondition); the
// CHECK variant reduces the high word on the way for larger digit counts.
// ---------------------------------------------------------------------------------
// One thread per (limb i, coefficient k) of rotation r = blockIdx.y keeps the 2*nd key
// values in registers and sweeps the batch, so each key value leaves HBM once per
// launch.  The automorphism gather stays inside an aligned 32-element block for the 32
// consecutive k of a warp (bit-reversed order), so it touches as many sectors as a
// coalesced load.  On limbs whose prime is below 2^54 the products use kSplitW-bit halves
// (the ModUp stores its digits split; three 32x32->64 multiply-adds per product, no
// carries); otherwise 64x64->128 products with the high word kept below q.
__device__ __forceinline__ u64 split_of(u64 v) { return ((v >> kSplitW) << 32) | (v & ((1ull << kSplitW) - 1)); }
// REDC of S = a00 + a01 * 2^W + a11 * 2^(2W) (W = kSplitW), a 128-bit value below q * 2^64.
__device__ __forceinline__ u64 split_redc(u64 a00, u64 a01, u64 a11, u64 q, u64 qinv) {
  constexpr int W = kSplitW;
  u64 lo = a00, hi = 0;
  const u64 t_lo = a01 << W, t_hi = a01 >> (64 - W);
  lo += t_lo;
  hi += t_hi + (lo < t_lo);
  const u64 u_lo = a11 << (2 * W), u_hi = a11 >> (64 - 2 * W);
  lo += u_lo;
  hi += u_hi + (lo < u_lo);
  return redc(hi, lo, q, qinv);
}

// Karatsuba multiply-adds of a split operand x = x1 * 2^32 + x0 with two split constants
// (k0 = k01:k00 and k1 = k11:k10, middle operands ks0 = k00 + k01, ks1 = k10 + k11):
//   a00 += x0 k00, a11 += x1 k01, am += (x0 + x1) ks0, and the same into c* for k1.
// Six 32x32->64 multiply-adds and one add, written out so that no other instruction
// enters the product chain.
__device__ __forceinline__ void kara_mac2(u64& a00, u64& a11, u64& am, u64& c00, u64& c11, u64& cm, u64 x,
                                          uint32_t k00, uint32_t k01, uint32_t ks0, uint32_t k10, uint32_t k11,
                                          uint32_t ks1) {
  asm("{\n\t"
      ".reg .u32 x0, x1, xs;\n\t"
      "mov.b64 {x0, x1}, %6;\n\t"
      "add.u32 xs, x0, x1;\n\t"
      "mad.wide.u32 %0, x0, %7, %0;\n\t"
      "mad.wide.u32 %1, x1, %8, %1;\n\t"
      "mad.wide.u32 %2, xs, %9, %2;\n\t"
      "mad.wide.u32 %3, x0, %10, %3;\n\t"
      "mad.wide.u32 %4, x1, %11, %4;\n\t"
      "mad.wide.u32 %5, xs, %12, %5;\n\t"
      "}"
      : "+l"(a00), "+l"(a11), "+l"(am), "+l"(c00), "+l"(c11), "+l"(cm)
      : "l"(x), "r"(k00), "r"(k01), "r"(ks0), "r"(k10), "r"(k11), "r"(ks1));
}

// Karatsuba multiply-add of two split operands x = x1:x0 and d = d1:d0 (32-bit halves):
//   a00 += x0 d0, a11 += x1 d1, am += (x0 + x1)(d0 + d1).
__device__ __forceinline__ void kara_mac1(u64& a00, u64& a11, u64& am, u64 x, u64 d) {
  asm("{\n\t"
      ".reg .u32 x0, x1, xs, d0, d1, ds;\n\t"
      "mov.b64 {x0, x1}, %3;\n\t"
      "mov.b64 {d0, d1}, %4;\n\t"
      "add.u32 xs, x0, x1;\n\t"
      "add.u32 ds, d0, d1;\n\t"
      "mad.wide.u32 %0, x0, d0, %0;\n\t"
      "mad.wide.u32 %1, x1, d1, %1;\n\t"
      "mad.wide.u32 %2, xs, ds, %2;\n\t"
      "}"
      : "+l"(a00), "+l"(a11), "+l"(am)
      : "l"(x), "l"(d));
}

// Key values of one (limb, coefficient) for the nd digits of one rotation, in split form
// where the limb's prime is below 2^54 (sp).  ND is the digit count, or an upper bound
// of it (nd <= ND) for the largest counts.
template <int ND>
struct KeyRegs {
  u64 k0[ND], k1[ND];
  uint32_t s0[ND], s1[ND];  // split key halves summed (Karatsuba middle operands)
  __device__ __forceinline__ void load(const u64* key, int nd, int pi, int LK, size_t N, uint32_t k, bool sp) {
#pragma unroll
    for (int d = 0; d < ND; d++) {
      k0[d] = d < nd ? key[(((size_t)d * 2) * LK + pi) * N + k] : 0;
      k1[d] = d < nd ? key[(((size_t)d * 2 + 1) * LK + pi) * N + k] : 0;
      if (sp) {
        k0[d] = split_of(k0[d]);
        k1[d] = split_of(k1[d]);
        s0[d] = (uint32_t)k0[d] + (uint32_t)(k0[d] >> 32);
        s1[d] = (uint32_t)k1[d] + (uint32_t)(k1[d] >> 32);
      }
    }
  }
  // The nd digit values of one ciphertext (issued together, before any arithmetic).
  __device__ __forceinline__ static void fetch(const u64* eb, size_t EN, int nd, u64 (&xv)[ND]) {
#pragma unroll
    for (int d = 0; d < ND; d++) xv[d] = d < nd ? eb[(size_t)d * EN] : 0;
  }
  // (r0, r1) = sum_d xv[d] * (k0[d], k1[d]) mod q, plain residues.  On split limbs the
  // digit values arrive split and each product takes three 32x32->64 multiply-adds
  // (Karatsuba: the middle term is (x0 + x1)(k0 + k1) - x0 k0 - x1 k1; every sum stays
  // below nd * 2^(2W+2) <= 2^60 for nd <= 16, W = 27).
  __device__ __forceinline__ void ip(const u64 (&xv)[ND], int nd, bool sp, const DPrime& P, u64& r0,
                                     u64& r1) const {
    if (sp) {
      u64 a00 = 0, am = 0, a11 = 0, c00 = 0, cm = 0, c11 = 0;
#pragma unroll
      for (int d = 0; d < ND; d++) {
        if (d < nd)
          kara_mac2(a00, a11, am, c00, c11, cm, xv[d], (uint32_t)k0[d], (uint32_t)(k0[d] >> 32), s0[d],
                    (uint32_t)k1[d], (uint32_t)(k1[d] >> 32), s1[d]);
      }
      r0 = split_redc(a00, am - a00 - a11, a11, P.q, P.qinv);
      r1 = split_redc(c00, cm - c00 - c11, c11, P.q, P.qinv);
    } else if constexpr (ND <= 8) {
      // at most 8 products below q^2 < 2^124: the 128-bit sums cannot overflow and their
      // high words stay below 2^63, reduced once before REDC (same residue as reducing
      // after every product)
      u64 lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
      for (int d = 0; d < ND; d++) {
        if (d < nd) {
          const u64 x = xv[d];
          mac(lo0, hi0, x, k0[d]);
          mac(lo1, hi1, x, k1[d]);
        }
      }
      r0 = redc(reduce_wide(hi0, P.q, P.bar), lo0, P.q, P.qinv);
      r1 = redc(reduce_wide(hi1, P.q, P.bar), lo1, P.q, P.qinv);
    } else {
      u64 lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
      for (int d = 0; d < ND; d++) {
        if (d < nd) {
          const u64 x = xv[d];
          mac(lo0, hi0, x, k0[d]);
          mac(lo1, hi1, x, k1[d]);
          if (hi0 >= P.q) hi0 -= P.q;
          if (hi1 >= P.q) hi1 -= P.q;
        }
      }
      r0 = redc(hi0, lo0, P.q, P.qinv);
      r1 = redc(hi1, lo1, P.q, P.qinv);
    }
  }
};

// ND: the digit count when EXACT, else an upper bound of the run-time count nd_arg.
template <int ND, bool EXACT>
__device__ __forceinline__ void key_ip_body(const u64* __restrict__ ext, size_t ext_r, const RotList& rl,
                                            u64* __restrict__ acc, const u64* __restrict__ add_pc0, size_t add_b,
                                            const DPrime* __restrict__ pr, int logN, int nb, int nd_arg, int E,
                                            int lvl, int L, int LK) {
  const int nd = EXACT ? ND : nd_arg;
  const size_t N = (size_t)1 << logN;
  const size_t EN = (size_t)E << logN;
  // src_major (one ModUp shared by all rotations): the rotations run fastest over the
  // grid and a thread owns a SOURCE element s, writing destination k = sigma_g^-1(s), so
  // consecutive blocks read the same digits (from L2).  Otherwise a thread owns a
  // destination element k and gathers its source s = sigma_g(k).
  const bool src_major = ext_r == 0;
  const int r = src_major ? blockIdx.x : blockIdx.y;
  const size_t idx = (src_major ? blockIdx.y : blockIdx.x) * (size_t)blockDim.x + threadIdx.x;
  if (idx >= EN) return;
  const int i = (int)(idx >> logN);
  const uint32_t e = (uint32_t)(idx & (N - 1));
  const int pi = i < lvl ? i : L + (i - lvl);
  const DPrime P = pr[pi];
  const bool sp = P.split != 0;
  const u64 g = rl.g[r];
  const uint32_t k = (g == 1 || !src_major) ? e : auto_src_k(e, rl.ginv[r], logN);
  const uint32_t ks = (g == 1 || src_major) ? e : auto_src_k(e, g, logN);
  KeyRegs<ND> kr;
  kr.load(rl.key[r], nd, pi, LK, N, k, sp);
  // baby step in the extended basis: + sigma_g(P * c0) on the data limbs (the product taken
  // once per layer, not once per rotation)
  const bool with_c0 = add_pc0 != nullptr && i < lvl;
  const u64* c0 = with_c0 ? add_pc0 + ((size_t)i << logN) + ks : nullptr;
  // running pointers (ciphertext b: digits at ex + d*EN, outputs at o and o + EN): the
  // loop advances them by constant strides instead of recomputing 64-bit offsets
  const u64* ex = ext + (size_t)r * ext_r + ((size_t)i << logN) + ks;
  u64* o = acc + (size_t)r * 2 * nb * EN + ((size_t)i << logN) + k;
  const size_t xstep = (size_t)nd * EN, ostep = 2 * EN;
  // two ciphertexts per iteration: all their loads are issued before the arithmetic
  int b = 0;
  for (; b + 1 < nb; b += 2) {
    u64 xa[ND], xb[ND];
    KeyRegs<ND>::fetch(ex, EN, nd, xa);
    KeyRegs<ND>::fetch(ex + xstep, EN, nd, xb);
    ex += 2 * xstep;
    u64 ca = 0, cb = 0;
    if (with_c0) {
      ca = c0[0];
      cb = c0[add_b];
      c0 += 2 * add_b;
    }
    u64 r0, r1, s0, s1;
    kr.ip(xa, nd, sp, P, r0, r1);
    kr.ip(xb, nd, sp, P, s0, s1);
    if (with_c0) {
      r0 = addmod(r0, ca, P.q);
      s0 = addmod(s0, cb, P.q);
    }
    o[0] = r0;
    o[EN] = r1;
    o[ostep] = s0;
    o[ostep + EN] = s1;
    o += 2 * ostep;
  }
  if (b < nb) {
    u64 xa[ND];
    KeyRegs<ND>::fetch(ex, EN, nd, xa);
    u64 r0, r1;
    kr.ip(xa, nd, sp, P, r0, r1);
    if (with_c0) r0 = addmod(r0, c0[0], P.q);
    o[0] = r0;
    o[EN] = r1;
  }
}
// Up to four digits the key product fits 80 registers and runs three blocks per SM
// (measured faster than two blocks at 98 registers: it is issue-bound, and more resident
// warps cover the dependent multiply-add chains); the larger digit counts keep their
// registers (they would spill at 80).
template <int ND, bool EXACT>
__global__ void __launch_bounds__(256, 3) k_key_ip(const u64* __restrict__ ext, size_t ext_r,
                                                   const __grid_constant__ RotList rl, u64* __restrict__ acc,
                                                   const u64* __restrict__ add_pc0, size_t add_b,
                                                   const DPrime* __restrict__ pr, int logN, int nb, int nd_arg,
                                                   int E, int lvl, int L, int LK) {
  key_ip_body<ND, EXACT>(ext, ext_r, rl, acc, add_pc0, add_b, pr, logN, nb, nd_arg, E, lvl, L, LK);
}
template <int ND, bool EXACT>
__global__ void __launch_bounds__(256) k_key_ip_wide(const u64* __restrict__ ext, size_t ext_r,
                                                     const __grid_constant__ RotList rl, u64* __restrict__ acc,
                                                     const u64* __restrict__ add_pc0, size_t add_b,
                                                     const DPrime* __restrict__ pr, int logN, int nb, int nd_arg,
                                                     int E, int lvl, int L, int LK) {
  key_ip_body<ND, EXACT>(ext, ext_r, rl, acc, add_pc0, add_b, pr, logN, nb, nd_arg, E, lvl, L, LK);
}

// g^-1 mod 2N for odd g (2N a power of two): Newton iteration on the 2-adic inverse.
static u64 inv_mod_2n(u64 g, u64 two_n) {
  u64 x = g;  // correct to 3 bits for odd g
  for (int it = 0; it < 6; it++) x *= 2 - g * x;
  return x & (two_n - 1);
}

void launch_key_ip(ctl_context* c, const u64* ext, size_t ext_r, int nb, int lvl, const RotList& rl_in, u64* acc,
                   const u64* add_pc0, size_t add_b) {
  RotList rl = rl_in;
  for (int r = 0; r < rl.n; r++) rl.ginv[r] = inv_mod_2n(rl.g[r], 2ull * c->N);
  const int nrot = rl.n;
  const int nd = (lvl + (int)c->alpha - 1) / (int)c->alpha;
  const int E = lvl + (int)c->K;
  const int LK = (int)(c->L + c->K);
  const size_t EN = (size_t)E * c->N;
  const unsigned eblocks = (unsigned)((EN + 255) / 256);
  dim3 grid = ext_r == 0 ? dim3((unsigned)nrot, eblocks) : dim3(eblocks, (unsigned)nrot);
  double work = 2.0 * nd * EN * nb * nrot;
  // bytes: the extended digits once (shared by the rotations when hoisted), each rotation's
  // key once, the two accumulator polys written, and the P * c0 addend read when given
  const double bytes = 8.0 * (double)EN * ((ext_r == 0 ? 1.0 : nrot) * nb * nd + 2.0 * nd * nrot + 2.0 * nrot * nb +
                                           (add_pc0 ? (double)nrot * nb * lvl / E : 0.0));
#define CTL_KEYIP_CASE(KERN, NDV, EX)                                                                          \
  CTL_LAUNCH_C(KC_KEYIP, work, bytes, grid,                                                                    \
             (KERN<NDV, EX><<<grid, 256, 0, c->stream>>>(ext, ext_r, rl, acc, add_pc0, add_b, c->d_primes,      \
                                                         (int)c->logN, nb, nd, E, lvl, (int)c->L, LK)))
  switch (nd) {
    case 1: CTL_KEYIP_CASE(k_key_ip, 1, true); break;
    case 2: CTL_KEYIP_CASE(k_key_ip, 2, true); break;
    case 3: CTL_KEYIP_CASE(k_key_ip, 3, true); break;
    case 4: CTL_KEYIP_CASE(k_key_ip, 4, true); break;
    default:
      if (nd <= 8) CTL_KEYIP_CASE(k_key_ip_wide, 8, false);
      else CTL_KEYIP_CASE(k_key_ip_wide, 16, false);
  }
#undef CTL_KEYIP_CASE
}

// Giant steps in the extended basis: one thread per (limb i, coefficient k) sweeps the
// rotations r (their key values in registers, one rotation at a time) and, for each,
// the ciphertexts b of its block's share of the batch, adding the key product and the
// rotated poly-0 term into the running sum S.  Every element of S has one owner thread,
// so no two threads update it.
template <int ND>
__global__ void __launch_bounds__(256) k_key_ip_acc(const u64* __restrict__ ext, size_t ext_r,
                                                    const __grid_constant__ RotList rl, const u64* __restrict__ add,
                                                    size_t add_r, size_t add_b, u64* __restrict__ S, size_t s_b,
                                                    const DPrime* __restrict__ pr, int logN, int nb, int b_per,
                                                    int nd, int E, int lvl, int L, int LK) {
  const size_t N = (size_t)1 << logN;
  const size_t EN = (size_t)E << logN;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= EN) return;
  const int b0 = blockIdx.y * b_per, b1 = min(nb, b0 + b_per);
  const int i = (int)(idx >> logN);
  const uint32_t k = (uint32_t)(idx & (N - 1));
  const int pi = i < lvl ? i : L + (i - lvl);
  const DPrime P = pr[pi];
  const bool sp = P.split != 0;
  for (int r = 0; r < rl.n; r++) {
    const u64 g = rl.g[r];
    const uint32_t ks = g == 1 ? k : auto_src_k(k, g, logN);
    KeyRegs<ND> kr;
    kr.load(rl.key[r], nd, pi, LK, N, k, sp);
    const u64* ex = ext + (size_t)r * ext_r + ((size_t)i << logN) + ks;
    const u64* ad = add + (size_t)r * add_r + ((size_t)i << logN) + ks;
    // two ciphertexts per iteration: all their loads are issued before the arithmetic
    int b = b0;
    for (; b + 1 < b1; b += 2) {
      u64 xa[ND], xb[ND];
      KeyRegs<ND>::fetch(ex + (size_t)b * nd * EN, EN, nd, xa);
      KeyRegs<ND>::fetch(ex + (size_t)(b + 1) * nd * EN, EN, nd, xb);
      u64* sa = S + (size_t)b * s_b + idx;
      u64* sb = S + (size_t)(b + 1) * s_b + idx;
      const u64 aa = ad[(size_t)b * add_b], ab = ad[(size_t)(b + 1) * add_b];
      const u64 sa0 = sa[0], sa1 = sa[EN], sb0 = sb[0], sb1 = sb[EN];
      u64 r0, r1, q0, q1;
      kr.ip(xa, nd, sp, P, r0, r1);
      kr.ip(xb, nd, sp, P, q0, q1);
      sa[0] = addmod(sa0, addmod(r0, aa, P.q), P.q);
      sa[EN] = addmod(sa1, r1, P.q);
      sb[0] = addmod(sb0, addmod(q0, ab, P.q), P.q);
      sb[EN] = addmod(sb1, q1, P.q);
    }
    if (b < b1) {
      u64 xa[ND];
      KeyRegs<ND>::fetch(ex + (size_t)b * nd * EN, EN, nd, xa);
      u64 r0, r1;
      kr.ip(xa, nd, sp, P, r0, r1);
      u64* sa = S + (size_t)b * s_b + idx;
      sa[0] = addmod(sa[0], addmod(r0, ad[(size_t)b * add_b], P.q), P.q);
      sa[EN] = addmod(sa[EN], r1, P.q);
    }
  }
}
void launch_key_ip_acc(ctl_context* c, const u64* ext, size_t ext_r, int nb, int lvl, const RotList& rl,
                       const u64* add, size_t add_r, size_t add_b, u64* S, size_t s_b) {
  const int nd = (lvl + (int)c->alpha - 1) / (int)c->alpha;
  const int E = lvl + (int)c->K;
  const int LK = (int)(c->L + c->K);
  const size_t EN = (size_t)E * c->N;
  const unsigned gx = (unsigned)((EN + 255) / 256);
  // split the batch over blockIdx.y in shares of at most 16 ciphertexts: a block's sums
  // (256 elements x 16 ciphertexts x 2 polys, 64 KB) are re-read once per rotation, and the
  // shares of all resident blocks (tens of MB) stay in L2 between those passes (measured
  // faster than shares of 8 and than two shares of the whole batch)
  const int splits = std::max(1, (nb + 15) / 16);
  const int b_per = (nb + splits - 1) / splits;
  dim3 grid(gx, (unsigned)((nb + b_per - 1) / b_per));
  double work = 2.0 * nd * EN * nb * rl.n;
  // bytes: the digits of every rotation's input, the keys, the poly-0 addend of every
  // rotation, and the sums S (two polys) read and written once
  const double bytes = 8.0 * (double)EN * ((double)rl.n * nb * nd + 2.0 * nd * rl.n + (double)rl.n * nb +
                                           4.0 * nb);
#define CTL_KEYIPA_CASE(NDV)                                                                                     \
  CTL_LAUNCH_C(KC_KEYIP, work, bytes, grid,                                                                      \
             (k_key_ip_acc<NDV><<<grid, 256, 0, c->stream>>>(ext, ext_r, rl, add, add_r, add_b, S, s_b,           \
                                                             c->d_primes, (int)c->logN, nb, b_per, nd, E, lvl,    \
                                                             (int)c->L, LK)))
  if (nd <= 1) CTL_KEYIPA_CASE(1);
  else if (nd <= 2) CTL_KEYIPA_CASE(2);
  else if (nd <= 4) CTL_KEYIPA_CASE(4);
  else if (nd <= 8) CTL_KEYIPA_CASE(8);
  else CTL_KEYIPA_CASE(16);
#undef CTL_KEYIPA_CASE
}

// Extended-basis image P * x of a batch: data limbs times (P mod q_i), special limbs 0.
__global__ void k_scale_ext(const u64* __restrict__ in, u64* __restrict__ out, const u64* __restrict__ pmod,
                            const u64* __restrict__ pmod_sh, const DPrime* __restrict__ pr, int logN, int lvl, int E,
                            size_t total) {
  const size_t EN = (size_t)E << logN, LN = (size_t)lvl << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / EN, r = idx % EN;
    const int i = (int)(r >> logN);
    out[idx] = i < lvl ? shoup(in[p * LN + r], __ldg(pmod + i), __ldg(pmod_sh + i), pr[i].q) : 0;
  }
}
void launch_scale_to_ext(ctl_context* c, const u64* in, u64* out, int nb, int lvl) {
  const int E = lvl + (int)c->K;
  size_t total = (size_t)nb * 2 * E * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_scale_ext<<<g, kThreads, 0, c->stream>>>(in, out, c->moddown.pmod, c->moddown.pmod_sh, c->d_primes,
                                                         (int)c->logN, lvl, E, total)));
}

// ---------------------------------------------------------------------------------
// Baby-step giant-step inner sums (Eq. bsgs):
//   inner[k][b][p][i][c] = sum_{j < t1} diag[k*t1 + j][i][c] * baby[j][b][p][i][c]
// A block covers 32 coefficients of one limb for 8 (ciphertext, poly) pairs (one warp
// each).  For every giant step k the block stages the t1 x 32 diagonal values in shared
// memory once for its 8 warps (and the grid runs the pairs fastest so other blocks find
// the same tile in L2); each thread keeps its t1 baby-step values in registers.
// Products are exact: on limbs whose prime is below 2^54 both operands are in split form
// (kSplitW-bit halves) and the t1 products go into three 64-bit sums with plain
// 32x32->64 multiply-adds (no carries: t1 * 2^56 < 2^64), combined once into a 128-bit value;
// otherwise full 64x64->128 products are summed.  One Montgomery reduction per output
// (diagonals are in Montgomery form; t1 * q < 2^64 keeps the REDC precondition).
// ---------------------------------------------------------------------------------
__global__ void k_split(u64* data, const DPrime* __restrict__ pr, int logN, int limbs, int lvl, int L,
                        size_t total) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((idx >> logN) % limbs);
    if (!pr[i < lvl ? i : L + (i - lvl)].split) continue;
    data[idx] = split_of(data[idx]);
  }
}
void launch_split_limbs(ctl_context* c, u64* data, int cnt, int limbs, int lvl) {
  size_t total = (size_t)cnt * limbs * c->N;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_split<<<g, kThreads, 0, c->stream>>>(data, c->d_primes, (int)c->logN, limbs, lvl, (int)c->L, total)));
}

// 16-byte global -> shared copy that completes asynchronously (L2 only), and its group
// fences: the next giant step's diagonal tile is in flight while the current one is used.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The baby steps are taken in chunks of T1 = min(t1, 32) (registers); a chunk after the
// first adds its partial sums to the ones the same thread stored for the chunk before
// (that value is requested before the chunk's products, so its latency is covered).
// A block has one warp per (ciphertext, poly) pair, up to 8.
template <int T1, bool KARA>
__global__ void __launch_bounds__(256) k_bsgs(const u64* __restrict__ baby, const u64* __restrict__ diag,
                                              size_t diag_stride, const u64* __restrict__ wino,
                                              u64* __restrict__ inner, const DPrime* __restrict__ pr, int logN,
                                              int t1, int t2, int nb, int limbs, int lvl, int L) {
  __shared__ __align__(16) u64 Ds[2][T1][32];
  const size_t LN = (size_t)limbs << logN;
  const size_t chunk = blockIdx.y + (size_t)blockIdx.z * gridDim.y;
  if (chunk >= (LN >> 5)) return;  // whole block
  const int bp_count = nb * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bp = blockIdx.x * (blockDim.x >> 5) + warp;
  const size_t c0 = chunk * 32;  // first coefficient index in [0, limbs*N)
  const size_t cidx = c0 + lane;
  const int i = (int)(c0 >> logN);
  const DPrime P = pr[i < lvl ? i : L + (i - lvl)];
  const bool sp = P.split != 0;
  const bool active = bp < bp_count;
  const size_t bstride = (size_t)bp_count * LN;  // stride between baby steps j
  const int n_chunks = t1 / T1;
  // step s = (chunk jc, giant step k): diag[k*t1 + jc*T1 + j][c0 .. c0+32), j < T1 -> Ds[buf]
  auto stage = [&](int s_, int buf) {
    const int jc = s_ / t2, k = s_ % t2;
    const u64* dk = diag + (size_t)(k * t1 + jc * T1) * diag_stride + c0;
    for (int e = threadIdx.x; e < T1 * 16; e += blockDim.x) {
      const int row = e >> 4, col = (e & 15) * 2;
      cp_async16(&Ds[buf][row][col], dk + (size_t)row * diag_stride + col);
    }
    cp_async_commit();
  };
  stage(0, 0);
  u64 x[T1];
  u64 Y = 0;  // Winograd form: REDC(sum_i x_{2i} x_{2i+1}) of this chunk
  constexpr bool kWino = KARA && T1 >= 2;
  const int n_steps = n_chunks * t2;
  const u64* xb = baby + (size_t)bp * LN + cidx;
  u64* ob = inner + (size_t)bp * LN + cidx;
  for (int s_ = 0; s_ < n_steps; s_++) {
    const int jc = s_ / t2, k = s_ % t2;
    if (k == 0) {  // this chunk's baby-step values, in split form
#pragma unroll
      for (int j = 0; j < T1; j++) x[j] = active ? xb[(size_t)(jc * T1 + j) * bstride] : 0;
      if (sp) {
#pragma unroll
        for (int j = 0; j < T1; j++) x[j] = split_of(x[j]);
        if constexpr (kWino) {
          u64 y00 = 0, y11 = 0, ym = 0;
#pragma unroll
          for (int j = 0; j < T1; j += 2) kara_mac1(y00, y11, ym, x[j], x[j + 1]);
          Y = split_redc(y00, ym - y00 - y11, y11, P.q, P.qinv);
        }
      }
    }
    u64* o = ob + (size_t)k * bstride;
    const u64 prev = (active && jc > 0) ? *o : 0;
    // Winograd form: the diagonal pair term of giant step k (subtracted once, in chunk 0)
    const u64 ek = (kWino && sp && active && jc == 0) ? __ldg(wino + (size_t)k * LN + cidx) : 0;
    cp_async_wait_all();  // tile s has landed (the only group in flight)
    __syncthreads();      // ... for every thread, and every warp is done with tile s-1
    if (s_ + 1 < n_steps) stage(s_ + 1, (s_ + 1) & 1);
    const u64(*D)[32] = Ds[s_ & 1];
    u64 res;
    if (sp) {
      u64 a00 = 0, a11 = 0, m;
      if constexpr (kWino) {
        // Winograd's inner product: sum_j x_j d_j = sum_i (x_{2i} + d_{2i+1})(x_{2i+1} + d_{2i})
        // - sum_i x_{2i} x_{2i+1} - sum_i d_{2i} d_{2i+1}: T1/2 products, each a Karatsuba
        // product of split sums (halves below 2^28, so the packed 64-bit add carries
        // nothing across halves); am < (T1/2) * 2^58 <= 2^62, and the 128-bit total
        // sum (x + d)(x' + d') < 16 (2q)^2 stays below q * 2^64 (REDC precondition)
        u64 am = 0;
#pragma unroll
        for (int j = 0; j < T1; j += 2) kara_mac1(a00, a11, am, x[j] + D[j + 1][lane], x[j + 1] + D[j][lane]);
        m = am - a00 - a11;
      } else if constexpr (KARA) {
        // three multiply-adds per product: middle term (x0 + x1)(d0 + d1) - x0 d0 - x1 d1;
        // am < T1 * 2^56 <= 2^61
        u64 am = 0;
#pragma unroll
        for (int j = 0; j < T1; j++) kara_mac1(a00, a11, am, x[j], D[j][lane]);
        m = am - a00 - a11;
      } else {
        // two accumulators for the middle term keep the dependent chains short
        u64 a01 = 0, a10 = 0;
#pragma unroll
        for (int j = 0; j < T1; j++) {
          const u64 d = D[j][lane];
          const uint32_t d0 = (uint32_t)d, d1 = (uint32_t)(d >> 32);
          const uint32_t x0 = (uint32_t)x[j], x1 = (uint32_t)(x[j] >> 32);
          a00 += (u64)x0 * d0;
          a01 += (u64)x0 * d1;
          a10 += (u64)x1 * d0;
          a11 += (u64)x1 * d1;
        }
        m = a01 + a10;
      }
      // S = a11 * 2^(2W) + m * 2^W + a00 (W = kSplitW); m < 2^62
      res = split_redc(a00, m, a11, P.q, P.qinv);
      if constexpr (kWino) res = submod(submod(res, Y, P.q), ek, P.q);
    } else if (P.q < (1ull << 61)) {
      // at most 32 products below q^2 < 2^122: no overflow, the high word stays below 2^63
      // and is reduced once before REDC (the same residue as reducing after every product)
      u64 lo = 0, hi = 0;
#pragma unroll
      for (int j = 0; j < T1; j++) mac(lo, hi, x[j], D[j][lane]);
      res = redc(reduce_wide(hi, P.q, P.bar), lo, P.q, P.qinv);
    } else {
      u64 lo = 0, hi = 0;
#pragma unroll
      for (int j = 0; j < T1; j++) {
        mac(lo, hi, x[j], D[j][lane]);
        if (hi >= P.q) hi -= P.q;
      }
      res = redc(hi, lo, P.q, P.qinv);
    }
    if (active) *o = jc == 0 ? res : addmod(prev, res, P.q);
  }
}

// Diagonal pair terms of Winograd's inner product, once per dense layer:
//   wino[k][i][c] = REDC( sum_{j even, j + 1 < t1} diag[k t1 + j][i][c] * diag[k t1 + j + 1][i][c] )
// (the diagonals are in Montgomery form, so this is the plain sum of d_j d_{j+1} times
// 2^64 mod q; the accumulated high word is kept below q by subtracting q * 2^64).
__global__ void k_wino_diag(const u64* __restrict__ diag, size_t diag_stride, u64* __restrict__ wino,
                            const DPrime* __restrict__ pr, int logN, int t1, int limbs, int lvl, int L,
                            size_t total) {
  const size_t LN = (size_t)limbs << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t k = idx / LN, r = idx % LN;
    const int i = (int)(r >> logN);
    const DPrime P = pr[i < lvl ? i : L + (i - lvl)];
    const u64 mask = (1ull << kSplitW) - 1;
    u64 lo = 0, hi = 0;
    for (int j = 0; j + 1 < t1; j += 2) {
      u64 a = diag[(k * t1 + j) * diag_stride + r], b = diag[(k * t1 + j + 1) * diag_stride + r];
      if (P.split) {  // stored split: back to the plain residue
        a = ((a >> 32) << kSplitW) | (a & mask);
        b = ((b >> 32) << kSplitW) | (b & mask);
      }
      mac(lo, hi, a, b);
      if (hi >= P.q) hi -= P.q;
    }
    wino[idx] = redc(hi, lo, P.q, P.qinv);
  }
}
void launch_bsgs_wino_diag(ctl_context* c, const u64* diag, size_t diag_stride, u64* wino, int t1, int t2, int limbs,
                           int lvl) {
  const size_t total = (size_t)t2 * limbs * c->N;
  const int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 0, g,
             (k_wino_diag<<<g, kThreads, 0, c->stream>>>(diag, diag_stride, wino, c->d_primes, (int)c->logN, t1,
                                                          limbs, lvl, (int)c->L, total)));
}

void launch_bsgs_inner(ctl_context* c, const u64* baby, const u64* diag, size_t diag_stride, const u64* wino,
                       u64* inner, int t1, int t2, int nb, int limbs, int lvl) {
  const size_t LN = (size_t)limbs * c->N;
  const size_t chunks = LN / 32;
  const unsigned gy = (unsigned)std::min<size_t>(chunks, 65535);
  const int wpb = std::min(8, nb * 2);  // warps (ciphertext polys) per block
  dim3 grid((unsigned)((nb * 2 + wpb - 1) / wpb), gy, (unsigned)((chunks + gy - 1) / gy));
  double work = (double)t1 * t2 * nb * 2 * LN;
  // bytes: the t1 baby steps and the t diagonals (plus the t2 Winograd pair terms) read
  // once, the t2 inner sums written once
  const double bytes = 8.0 * (double)LN * ((double)t1 * nb * 2 + (double)t1 * t2 + t2 + (double)t2 * nb * 2);
  const bool kara = c->bsgs_karatsuba != 0;
#define CTL_BSGS_CASE(TT)                                                                                      \
  case TT:                                                                                                     \
    if (kara)                                                                                                  \
      CTL_LAUNCH_C(KC_BSGS, work, bytes, grid,                                                                 \
                 (k_bsgs<TT, true><<<grid, 32 * wpb, 0, c->stream>>>(baby, diag, diag_stride, wino,      \
                                                                     inner, c->d_primes, (int)c->logN, t1, t2, nb,   \
                                                                     limbs, lvl, (int)c->L)));                \
    else                                                                                                       \
      CTL_LAUNCH_C(KC_BSGS, work, bytes, grid,                                                                 \
                 (k_bsgs<TT, false><<<grid, 32 * wpb, 0, c->stream>>>(baby, diag, diag_stride, wino,    \
                                                                      inner, c->d_primes, (int)c->logN, t1, t2, nb,  \
                                                                      limbs, lvl, (int)c->L)));               \
    break;
  // T1 = min(t1, chunk cap); t1 and the cap are powers of two, so T1 divides t1
  const int cap = c->bsgs_chunk == 16 ? 16 : 32;
  int T1 = 1;
  while (T1 < t1 && T1 < cap) T1 <<= 1;
  switch (T1) {
    CTL_BSGS_CASE(1)
    CTL_BSGS_CASE(2)
    CTL_BSGS_CASE(4)
    CTL_BSGS_CASE(8)
    CTL_BSGS_CASE(16)
    default:
      CTL_BSGS_CASE(32)
  }
#undef CTL_BSGS_CASE
}

// ---------------------------------------------------------------------------------
// Kernels of the other layers of the paper's frozen network (Sec. 3.1: ReLU
// approximation, average pooling, 1D convolution).  All are element-wise over the
// NTT domain and bound by HBM traffic.
// ---------------------------------------------------------------------------------
// Tensor of two ciphertexts: (a0 b0, a0 b1 + a1 b0, a1 b1); d [nb][3][lvl][N].
__global__ void k_tensor2(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ d,
                          const DPrime* __restrict__ pr, int logN, int lvl, size_t total) {
  const size_t N = (size_t)1 << logN;
  const size_t LN = (size_t)lvl * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t j = idx / LN, r = idx % LN;
    const int i = (int)(r >> logN);
    const DPrime P = pr[i];
    const u64 a0 = a[j * 2 * LN + r], a1 = a[j * 2 * LN + LN + r];
    const u64 b0m = mulmod_mont(b[j * 2 * LN + r], P.r2, P.q, P.qinv);       // b0 * R
    const u64 b1m = mulmod_mont(b[j * 2 * LN + LN + r], P.r2, P.q, P.qinv);  // b1 * R
    d[j * 3 * LN + r] = mulmod_mont(a0, b0m, P.q, P.qinv);
    d[j * 3 * LN + LN + r] = addmod(mulmod_mont(a0, b1m, P.q, P.qinv), mulmod_mont(a1, b0m, P.q, P.qinv), P.q);
    d[j * 3 * LN + 2 * LN + r] = mulmod_mont(a1, b1m, P.q, P.qinv);
  }
}
void launch_tensor2(ctl_context* c, const u64* a, const u64* b, u64* d, int nb, int lvl) {
  size_t total = (size_t)nb * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, 6.0 * total, g,
             (k_tensor2<<<g, kThreads, 0, c->stream>>>(a, b, d, c->d_primes, (int)c->logN, lvl, total)));
}

// out[pp] = in[pp] * m_i (if has_m) + add[pp] (if add) + (pp even ? a_i : 0), for the
// polys pp = 0..n_polys-1 (two per ciphertext), limb i -> prime i.
__global__ void k_affine(const u64* in, size_t s_in, const u64* add, size_t s_add, u64* out, size_t s_out,
                         const __grid_constant__ LimbConsts K, bool has_m, const DPrime* __restrict__ pr, int logN,
                         int lvl, size_t total) {
  const size_t N = (size_t)1 << logN;
  const size_t LN = (size_t)lvl * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t pp = idx / LN, r = idx % LN;
    const int i = (int)(r >> logN);
    const u64 q = pr[i].q;
    u64 v = in[pp * s_in + r];
    if (has_m) v = mulmod_mont(v, K.m[i], q, pr[i].qinv);
    if (add) v = addmod(v, add[pp * s_add + r], q);
    if (!(pp & 1)) v = addmod(v, K.a[i], q);
    out[pp * s_out + r] = v;
  }
}
void launch_affine(ctl_context* c, const u64* in, size_t s_in, const u64* add, size_t s_add, u64* out, size_t s_out,
                   const LimbConsts& K, bool has_m, int n_polys, int lvl) {
  size_t total = (size_t)n_polys * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, has_m ? (double)total : 0.0, g,
             (k_affine<<<g, kThreads, 0, c->stream>>>(in, s_in, add, s_add, out, s_out, K, has_m, c->d_primes,
                                                     (int)c->logN, lvl, total)));
}

// out[j] = (x[j] + sum_{r < nr} rots[r][j]) * m_i over nb ciphertexts [nb][2][lvl][N];
// rots [nr][nb][2][lvl][N].
__global__ void k_sum_scale(const u64* __restrict__ x, const u64* __restrict__ rots, int nr, u64* __restrict__ out,
                            const __grid_constant__ LimbConsts K, const DPrime* __restrict__ pr, int logN, int lvl,
                            size_t total) {
  const size_t N = (size_t)1 << logN;
  const size_t LN = (size_t)lvl * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((idx % LN) >> logN);
    const u64 q = pr[i].q;
    u64 s = x[idx];
    for (int r = 0; r < nr; r++) s = addmod(s, rots[(size_t)r * total + idx], q);
    out[idx] = mulmod_mont(s, K.m[i], q, pr[i].qinv);
  }
}
void launch_sum_scale(ctl_context* c, const u64* x, const u64* rots, int nr, u64* out, const LimbConsts& K, int nb,
                      int lvl) {
  size_t total = (size_t)nb * 2 * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, (double)total, g,
             (k_sum_scale<<<g, kThreads, 0, c->stream>>>(x, rots, nr, out, K, c->d_primes, (int)c->logN, lvl,
                                                        total)));
}

// out[j] = sum_{i < f} rots[i][j] o pts[i] over nb ciphertexts [nb][2][lvl][N]; rots
// [f][nb][2][lvl][N]; pts [f][lvl][N] in Montgomery form; sums in increasing i.
__global__ void k_pt_mac(const u64* __restrict__ rots, const u64* __restrict__ pts, int f, u64* __restrict__ out,
                         const DPrime* __restrict__ pr, int logN, int lvl, size_t total) {
  const size_t N = (size_t)1 << logN;
  const size_t LN = (size_t)lvl * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t r = idx % LN;
    const int i = (int)(r >> logN);
    const u64 q = pr[i].q, qinv = pr[i].qinv;
    u64 s = mulmod_mont(rots[idx], pts[r], q, qinv);
    for (int k = 1; k < f; k++) s = addmod(s, mulmod_mont(rots[(size_t)k * total + idx], pts[(size_t)k * LN + r], q, qinv), q);
    out[idx] = s;
  }
}
void launch_pt_mac(ctl_context* c, const u64* rots, const u64* pts, int f, u64* out, int nb, int lvl) {
  size_t total = (size_t)nb * 2 * lvl * c->N;
  if (!total) return;
  int g = elem_grid(c, total);
  CTL_LAUNCH(KC_ELEM, (double)f * total, g,
             (k_pt_mac<<<g, kThreads, 0, c->stream>>>(rots, pts, f, out, c->d_primes, (int)c->logN, lvl, total)));
}

}  // namespace ctl
