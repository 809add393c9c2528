// Exact 64-bit modular arithmetic for word-size primes q < 2^62 on sm_103a.
//
// CKKS keeps every ring element as residues modulo word-size primes (RNS); all of the
// server-side evaluation (Sec. 3.1 of CryptoTL: rescaling, rotations, plaintext and
// ciphertext products) reduces to the operations below.  There is no floating point:
// every result is the exact residue.
//
//  * shoup_lazy / shoup: product with a constant w known ahead of time (NTT twiddles,
//    base-conversion constants), using w' = floor(w * 2^64 / q) (V. Shoup).  The lazy
//    form returns a value in [0, 2q) for any 64-bit x.
//  * redc: Montgomery reduction of a 128-bit T = hi*2^64 + lo with hi < q, returning
//    T * 2^-64 mod q in [0, q) (P. Montgomery, 1985), with the positive inverse
//    qinv = q^-1 mod 2^64.  Operands stored "in Montgomery form" (times 2^64 mod q)
//    make redc(a * b_mont) the plain residue a*b mod q.
//  * mac: 64x64 -> 128-bit multiply-accumulate, the unit of the lazy inner products.
#pragma once
#include <cstdint>

namespace ctl {

typedef unsigned long long u64;

__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 wsh, u64 q) {
  u64 qh = __umul64hi(x, wsh);
  return x * w - qh * q;
}
// Shoup product with the quotient estimated from three of the four 32x32-bit partial
// products of x * wsh (the low x low one dropped): the estimate e is at most 3 below
// floor(x * w / q) (the dropped terms and truncated halves sum to less than 3 * 2^32 over
// 2^32, Shoup's own estimate is at most 1 low), so the result lies in [0, 4q) for any
// 64-bit x.  On sm_103 the high-half and wide 32-bit products are the slow integer
// operations; this takes five of them and four low products, with the subtraction
// x * w - e * q folded into the multiply-adds as x * w + e * (2^64 - q) mod 2^64.
__device__ __forceinline__ u64 shoup_small(u64 x, u64 w, u64 wsh, u64 q) {
  const u64 nq = 0ull - q;
  u64 r;
  asm("{\n\t"
      ".reg .u32 x0, x1, s0, s1, w0, w1, n0, n1, t, l, h, e0, e1, r0, r1;\n\t"
      ".reg .u64 a, e;\n\t"
      "mov.b64 {x0, x1}, %1;\n\t"
      "mov.b64 {w0, w1}, %2;\n\t"
      "mov.b64 {s0, s1}, %3;\n\t"
      "mov.b64 {n0, n1}, %4;\n\t"
      "mul.hi.u32 t, x0, s1;\n\t"          // e = x1*s1 + hi(x0*s1) + hi(x1*s0)
      "mad.hi.cc.u32 l, x1, s0, t;\n\t"
      "addc.u32 h, 0, 0;\n\t"
      "mov.b64 a, {l, h};\n\t"
      "mad.wide.u32 e, x1, s1, a;\n\t"
      "mov.b64 {e0, e1}, e;\n\t"
      "mul.wide.u32 a, x0, w0;\n\t"        // r = x*w + e*(2^64 - q) mod 2^64
      "mad.wide.u32 a, e0, n0, a;\n\t"
      "mov.b64 {r0, r1}, a;\n\t"
      "mad.lo.u32 r1, x0, w1, r1;\n\t"
      "mad.lo.u32 r1, x1, w0, r1;\n\t"
      "mad.lo.u32 r1, e0, n1, r1;\n\t"
      "mad.lo.u32 r1, e1, n0, r1;\n\t"
      "mov.b64 %0, {r0, r1};\n\t"
      "}"
      : "=l"(r)
      : "l"(x), "l"(w), "l"(wsh), "l"(nq));
  return r;
}
__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 wsh, u64 q) {
  u64 r = shoup_lazy(x, w, wsh, q);
  return r >= q ? r - q : r;
}
__device__ __forceinline__ u64 redc(u64 hi, u64 lo, u64 q, u64 qinv) {
  u64 m = lo * qinv;
  u64 t = __umul64hi(m, q);
  return hi >= t ? hi - t : hi - t + q;
}
__device__ __forceinline__ void mac(u64& lo, u64& hi, u64 a, u64 b) {
  u64 pl = a * b, ph = __umul64hi(a, b);
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(pl), "l"(ph));
}
// a * b mod q for bmont = b * 2^64 mod q and any 64-bit a.
__device__ __forceinline__ u64 mulmod_mont(u64 a, u64 bmont, u64 q, u64 qinv) {
  return redc(__umul64hi(a, bmont), a * bmont, q, qinv);
}
// a * b mod q for two plain residues (a, b < q): two reductions, the second by R^2.
__device__ __forceinline__ u64 mulmod_plain(u64 a, u64 b, u64 q, u64 qinv, u64 r2) {
  u64 t = redc(__umul64hi(a, b), a * b, q, qinv);  // a*b*R^-1
  return mulmod_mont(t, r2, q, qinv);                // * R^2 * R^-1
}
__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ u64 negmod(u64 a, u64 q) { return a ? q - a : 0; }
// Reduction of a value in [0, 4q) to [0, q).
__device__ __forceinline__ u64 reduce4(u64 a, u64 q) {
  if (a >= 2 * q) a -= 2 * q;
  return a >= q ? a - q : a;
}
// Reduction of any a < 2^63 to [0, q) for 2^32 < q, with bar = floor(2^64 / q) < 2^32:
// the quotient estimate floor((a >> 32) * bar / 2^32) is at most 2 below floor(a / q)
// (truncating a to its high word loses < 2^32 / q <= 1, truncating 2^64 / q to bar loses
// < (a >> 32) / 2^32 < 1/2, the final floor < 1), so a - estimate * q lies in [0, 3q).
__device__ __forceinline__ u64 reduce_wide(u64 a, u64 q, u64 bar) {
  const uint32_t e = (uint32_t)(((u64)(uint32_t)(a >> 32) * (uint32_t)bar) >> 32);
  u64 r = a - (u64)e * q;
  if (r >= 2 * q) r -= 2 * q;
  return r >= q ? r - q : r;
}

}  // namespace ctl
