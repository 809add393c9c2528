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

}  // namespace ctl
