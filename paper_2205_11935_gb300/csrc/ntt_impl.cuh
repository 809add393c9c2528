// Negacyclic NTT / inverse NTT over word-size primes, with fused key-switching and
// rescaling prologues/epilogues.
//
// Definition (the NTT form of a in Z_q[X]/(X^N+1)):  a_hat[k] = a(psi^(2*bitrev(k)+1)),
// psi the smallest primitive 2N-th root of unity mod q; outputs in bit-reversed order.
// Forward: Cooley-Tukey butterflies with the psi powers merged (twiddle of stage m,
// group i: psi^bitrev(m+i)); inverse: Gentleman-Sande butterflies with
// (psi^-1)^bitrev(m+i) and N^-1 folded into the last stage.  Values stay lazily reduced
// (Harvey): forward butterflies keep [0, 4q), inverse [0, 2q); q < 2^62 (primes below
// 2^56 take a path with fewer reductions, described at ct_bfly).  Twiddles are
// stored as interleaved (w, floor(w * 2^64 / q)) pairs and read with one 16-byte load.
//
// GPU mapping.  For N in {4096, 8192, 16384} one CTA of N/32 threads owns a limb and
// each thread keeps 32 elements in registers through three passes of 5, 5 and
// log2(N)-10 stages; two shared-memory transposes (padded by one word in 16) connect
// them.  The forward transform reads its input straight from global memory into
// registers (thread t takes elements t + k*N/32: coalesced), the inverse writes its
// output the same way.  Stage indices are compile-time, so only the block index of a
// sub-transform is computed at run time.  Other N use a generic shared-memory kernel.
//
// CKKS (Sec. 3.1 of CryptoTL) needs these transforms around every key switch
// (rotations, relinearisation) and every rescale; the functors below fuse the fast base
// conversions of ModUp/ModDown and the rescale arithmetic into the element loads and
// stores, so each converted limb makes one trip through HBM.
//
// This header holds the device code and the launch helpers; the host launchers are split over
// ntt.cu (plain and rescaling transforms), ntt_modup.cu, ntt_moddown.cu and ntt_giant.cu, so
// that their template instances compile in parallel.
#pragma once
#include "ctl_internal.h"
#include "modarith.cuh"

namespace ctl {

__device__ __forceinline__ int pidx(int j) { return j + (j >> 4); }

__device__ __forceinline__ uint32_t brv_dev(uint32_t x, int logn) { return __brev(x) >> (32 - logn); }

// Index k' with new[k] = old[k'] for sigma_g in the bit-reversed NTT domain:
// exponent e_k = 2*bitrev(k)+1 maps to g*e_k mod 2N = e_{k'}.
__device__ __forceinline__ uint32_t auto_src(uint32_t k, u64 g, int logN) {
  uint32_t e = 2u * brv_dev(k, logN) + 1u;
  uint32_t e2 = (uint32_t)(((u64)e * g) & ((2ull << logN) - 1));
  return brv_dev((e2 - 1u) >> 1, logN);
}

// The same index with 32-bit arithmetic, for g < 2N <= 2^17 (e * g < 2^32).
__device__ __forceinline__ uint32_t auto_src32(uint32_t k, uint32_t g, int logN) {
  const uint32_t e = 2u * brv_dev(k, logN) + 1u;
  return brv_dev((((e * g) & ((2u << logN) - 1)) - 1u) >> 1, logN);
}

// Load of an element that this thread alone reads and then overwrites: no memory clobber,
// so the compiler may issue it ahead of stores to other elements (it cannot prove on its
// own that those stores do not alias it).
__device__ __forceinline__ u64 ld_own(const u64* p) {
  u64 v;
  asm("ld.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// Asynchronous bulk prefetch of a contiguous global range into L2 (one instruction, no
// registers); the range is 16-byte aligned and a multiple of 16 bytes (whole limbs).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  const unsigned long long g = (unsigned long long)__cvta_generic_to_global(p);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(bytes) : "memory");
}

// Harvey butterflies.  Forward: X is brought below 2q, outputs stay below 4q.  With
// SMALL (2^32 < q < 2^56) X is left as it is and the twiddle product is shoup_small
// (below 4q): each stage adds less than 4q to the bound, so an input below q leaves the
// 14 stages of N = 16384 below 57q, and the store reduces once.
template <bool SMALL = false>
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, const ulonglong2 w, u64 q) {
  u64 X = x;
  if constexpr (!SMALL) {
    const u64 q2 = 2 * q;
    if (X >= q2) X -= q2;
    const u64 T = shoup_lazy(y, w.x, w.y, q);
    x = X + T;
    y = X - T + q2;
  } else {
    // keeps the butterflies in program order: left free, the scheduler interleaves enough
    // of them to run out of registers
    asm volatile("" : "+l"(X));
    const u64 T = shoup_small(y, w.x, w.y, q);
    x = X + T;
    y = X - T + 4 * q;
  }
}
// Inverse: inputs below 2q, outputs below 2q (the sum reduced once).
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, const ulonglong2 w, u64 q) {
  const u64 q2 = 2 * q;
  const u64 U = x, V = y;
  u64 S = U + V;
  if (S >= q2) S -= q2;
  x = S;
  y = shoup_lazy(U - V + q2, w.x, w.y, q);
}
// Inverse without reduction of the sum (q * 2^logN < 2^63): V is below the multiple
// C >= 2q of q that bounds this stage's inputs, the sum below 2C (the next stage's
// bound), the difference path below 4q after its shoup_small product.
__device__ __forceinline__ void gs_bfly_s(u64& x, u64& y, const ulonglong2 w, u64 q, u64 C) {
  const u64 U = x, V = y;
  x = U + V;
  y = shoup_small(U - V + C, w.x, w.y, q);
}

// LOGR stages of a radix-2^LOGR sub-transform held in registers x[0..2^LOGR), for the
// stages S0..S0+LOGR-1 and block index b at stage S0.
template <int S0, int LOGR, bool SMALL = false>
__device__ __forceinline__ void fwd_regs(u64* x, int b, const ulonglong2* __restrict__ tw, u64 q) {
  constexpr int R = 1 << LOGR;
#pragma unroll
  for (int u = 0; u < LOGR; u++) {
    const int h = R >> (u + 1);
    const ulonglong2* tu = tw + (1 << (S0 + u)) + (b << u);
#pragma unroll
    for (int k = 0; k < R; k++) {
      if (k & h) continue;
      ct_bfly<SMALL>(x[k], x[k + h], __ldg(tu + (k >> (LOGR - u))), q);
    }
  }
}
// The last-stage constants of an inverse transform (N^-1 and the folded last twiddle).
struct InvLast {
  u64 ninv, ninv_sh, iw1, iw1_sh;
};

// Inverse stages S0+LOGR-1 .. S0.  With SMALL (q * 2^LOGN < 2^63) the inputs of stage s
// are below C_s = q * 2^(LOGN - s) (2q at the first stage, doubling per stage) and no sum
// is reduced; the last stage's two products bring both outputs below 4q (below 2q on the
// general path).
template <int S0, int LOGR, class PL, bool SMALL = false, int LOGN = 0>
__device__ __forceinline__ void inv_regs(u64* x, int b, const ulonglong2* __restrict__ tw, u64 q, const PL& P) {
  constexpr int R = 1 << LOGR;
#pragma unroll
  for (int u = LOGR - 1; u >= 0; u--) {
    const int h = R >> (u + 1);
    const ulonglong2* tu = tw + (1 << (S0 + u)) + (b << u);
    const u64 C = SMALL ? q << (LOGN - (S0 + u)) : 2 * q;
#pragma unroll
    for (int k = 0; k < R; k++) {
      if (k & h) continue;
      if (S0 + u == 0) {  // last stage: fold N^-1
        const u64 U = x[k], V = x[k + h];
        if constexpr (SMALL) {
          x[k] = shoup_small(U + V, P.ninv, P.ninv_sh, q);
          x[k + h] = shoup_small(U - V + C, P.iw1, P.iw1_sh, q);
        } else {
          x[k] = shoup_lazy(U + V, P.ninv, P.ninv_sh, q);
          x[k + h] = shoup_lazy(U - V + C, P.iw1, P.iw1_sh, q);
        }
      } else if constexpr (SMALL) {
        gs_bfly_s(x[k], x[k + h], __ldg(tu + (k >> (LOGR - u))), q, C);
      } else {
        gs_bfly(x[k], x[k + h], __ldg(tu + (k >> (LOGR - u))), q);
      }
    }
  }
}

// Which path a limb's transform takes (the same answer for every thread of a block).
__device__ __forceinline__ bool fwd_small(const DPrime& P) { return P.bar != 0 && P.q < (1ull << 56); }
__device__ __forceinline__ bool inv_small(u64 q, int logN) { return q < (1ull << (63 - logN)); }

// ---------------------------------------------------------------------------------
// Element functors.  A functor is a constant kernel parameter (__grid_constant__, so
// its tables are read in place); its per-item state lives in a small State struct.
// begin(st, p, l, pi, ...) binds item (poly p, limb l, prime pi) and returns false if
// the item is complete already (the same answer for the whole block); get(st, j)
// yields input element j (reduced, < q); put<SMALL>(st, j, v) consumes output element j
// given lazily reduced: below 4q, or below 64q with SMALL (the forward transform's
// small-prime path, q < 2^56).
// ---------------------------------------------------------------------------------
struct ProLoad {
  // inputs parked in shared memory first as well: with all loads of a thread in flight
  // in registers, the forward transform runs out of registers
  static constexpr bool kStage = true;
  const u64* src;
  size_t poly_stride;
  struct State {
    const u64* g;
  };
  __device__ bool begin(State& st, int p, int l, int, const DPrime*, int logN) const {
    st.g = src + (size_t)p * poly_stride + ((size_t)l << logN);
    return true;
  }
  __device__ u64 get(const State& st, int j) const { return st.g[j]; }
  template <int G>
  __device__ void getg(const State& st, int k0, int stride, u64 (&y)[G]) const {
#pragma unroll
    for (int g = 0; g < G; g++) y[g] = st.g[k0 + g * stride];
  }
  __device__ void prefetch_src(int p, int l, int, int logN) const {
    l2_prefetch(src + (size_t)p * poly_stride + ((size_t)l << logN), 8u << logN);
  }
};

// Full reduction of an output element: below 4q, or below 64q on the small-prime path.
template <bool SMALL>
__device__ __forceinline__ u64 reduce_out(u64 v, u64 q, u64 bar) {
  if constexpr (SMALL) return reduce_wide(v, q, bar);
  else return reduce4(v, q);
}

struct EpiStore {
  u64* dst;
  size_t poly_stride;
  struct State {
    u64* o;
    u64 q, bar;
  };
  __device__ void begin(State& st, int p, int l, int pi, const DPrime* pr, int logN) const {
    st.o = dst + (size_t)p * poly_stride + ((size_t)l << logN);
    st.q = pr[pi].q;
    st.bar = pr[pi].bar;
  }
  template <bool SMALL = false>
  __device__ void put(const State& st, int j, u64 v) const { st.o[j] = reduce_out<SMALL>(v, st.q, st.bar); }
  template <bool SMALL, int G>
  __device__ void putg(const State& st, int j0, int stride, const u64 (&v)[G]) const {
#pragma unroll
    for (int g = 0; g < G; g++) put<SMALL>(st, j0 + g * stride, v[g]);
  }
  __device__ void prefetch(const State&, int) const {}
};

// Store of ModUp digits for the key product: on limbs whose prime is below 2^54 the
// residue is stored in split form (kSplitW-bit halves in the two words), the operand form
// of the split-half multiply-adds, so the key product does not split it once per rotation.
struct EpiStoreSplit {
  u64* dst;
  size_t poly_stride;
  struct State {
    u64* o;
    u64 q, bar;
    bool sp;
  };
  __device__ void begin(State& st, int p, int l, int pi, const DPrime* pr, int logN) const {
    st.o = dst + (size_t)p * poly_stride + ((size_t)l << logN);
    st.q = pr[pi].q;
    st.bar = pr[pi].bar;
    st.sp = pr[pi].split != 0;
  }
  template <bool SMALL = false>
  __device__ void put(const State& st, int j, u64 v) const {
    const u64 r = reduce_out<SMALL>(v, st.q, st.bar);
    st.o[j] = st.sp ? ((r >> kSplitW) << 32) | (r & ((1ull << kSplitW) - 1)) : r;
  }
  template <bool SMALL, int G>
  __device__ void putg(const State& st, int j0, int stride, const u64 (&v)[G]) const {
#pragma unroll
    for (int g = 0; g < G; g++) put<SMALL>(st, j0 + g * stride, v[g]);
  }
  __device__ void prefetch(const State&, int) const {}
};

// Fast base conversion of one element: y = sum_j v_j * (Shat_j mod t) mod t over the
// ns <= NS source limbs, v_j = [x_j * Shat_j^-1]_{s_j} as stored by the inverse NTT that
// precedes the conversion; exact residue in [0, t).  Each product is a shoup_small (below
// 4t, for any source value) and the running sum stays below 4t (t < 2^61).
template <int NS>
struct ConvState {
  int ns;
  const u64* srcs[NS];
  u64 c[NS], c_sh[NS];
  u64 t;
  __device__ void bind(const ConvTab& T, int tpos, const u64* base, size_t limb0, int logN, u64 tq) {
    ns = T.ns;
#pragma unroll
    for (int j = 0; j < NS; j++) {
      const int jj = j < ns ? j : 0;
      srcs[j] = base + ((limb0 + jj) << logN);
      c[j] = __ldg(T.c + (size_t)jj * T.nt + tpos);
      c_sh[j] = __ldg(T.c_sh + (size_t)jj * T.nt + tpos);
    }
    t = tq;
  }
  // The source limbs are read-only in the launch (non-coherent loads, free to be issued
  // ahead of the kernel's shared-memory stores).
  __device__ u64 eval(int k) const {
    u64 s = 0;
#pragma unroll
    for (int j = 0; j < NS; j++)
      if (j < ns) {
        s += shoup_small(__ldg(srcs[j] + k), c[j], c_sh[j], t);
        if (s >= 4 * t) s -= 4 * t;
      }
    return reduce4(s, t);
  }
  // G elements k0 + g*stride: all G * ns source loads are issued before any product.
  template <int G>
  __device__ void evalg(int k0, int stride, u64 (&y)[G]) const {
    u64 v[NS][G];
#pragma unroll
    for (int j = 0; j < NS; j++)
#pragma unroll
      for (int g = 0; g < G; g++) v[j][g] = j < ns ? __ldg(srcs[j] + k0 + g * stride) : 0;
#pragma unroll
    for (int g = 0; g < G; g++) {
      u64 s = 0;
#pragma unroll
      for (int j = 0; j < NS; j++)
        if (j < ns) {
          s += shoup_small(v[j][g], c[j], c_sh[j], t);
          if (s >= 4 * t) s -= 4 * t;
        }
      y[g] = reduce4(s, t);
    }
  }
};

#define CTL_MAX_DIGITS 16
template <int NS>
struct ProModUp {
  static constexpr bool kStage = true;
  const u64* coef;   // c1 coefficient form, input b's limbs at coef + b*coef_stride
  size_t coef_stride;
  const u64* ntt;    // c1 NTT form, input b's limbs at ntt + b*stride
  size_t stride;
  u64* ext;          // [nb][nd][E][N]
  int nd, E, lvl, alpha;
  ConvTab tabs[CTL_MAX_DIGITS];
  typedef ConvState<NS> State;
  __device__ bool begin(State& st, int p, int l, int pi, const DPrime* pr, int logN) const {
    const int b = p / nd, d = p % nd;
    const int d0 = d * alpha, d1 = min(d0 + alpha, lvl);
    const int N = 1 << logN;
    if (l >= d0 && l < d1) {  // the digit's own primes: y = x mod q_l, already in NTT form
      const u64* g = ntt + (size_t)b * stride + ((size_t)l << logN);
      u64* o = ext + (((size_t)p * E + l) << logN);
      const bool sp = pr[pi].split != 0;  // stored split, as EpiStoreSplit does
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const u64 v = g[k];
        o[k] = sp ? ((v >> kSplitW) << 32) | (v & ((1ull << kSplitW) - 1)) : v;
      }
      return false;
    }
    st.bind(tabs[d], l, coef + (size_t)b * coef_stride, (size_t)d0, logN, pr[pi].q);
    return true;
  }
  __device__ void prefetch_src(int p, int l, int, int logN) const {
    const int b = p / nd, d = p % nd;
    const int d0 = d * alpha, d1 = min(d0 + alpha, lvl);
    if (l >= d0 && l < d1) {
      l2_prefetch(ntt + (size_t)b * stride + ((size_t)l << logN), 8u << logN);
    } else {
      for (int j = d0; j < d1; j++) l2_prefetch(coef + (size_t)b * coef_stride + ((size_t)j << logN), 8u << logN);
    }
  }
  __device__ u64 get(const State& st, int j) const { return st.eval(j); }
  template <int G>
  __device__ void getg(const State& st, int k0, int stride, u64 (&y)[G]) const {
    st.template evalg<G>(k0, stride, y);
  }
};

template <int NS>
struct ProModDown {
  static constexpr bool kStage = true;
  const u64* acc;    // [np][E][N], special limbs (positions lvl..lvl+K-1) in coefficient form
  size_t acc_stride;
  int lvl;
  ConvTab tab;       // sources: special primes; target position = data limb index
  typedef ConvState<NS> State;
  __device__ bool begin(State& st, int p, int l, int pi, const DPrime* pr, int logN) const {
    st.bind(tab, l, acc + (size_t)p * acc_stride, (size_t)lvl, logN, pr[pi].q);
    return true;
  }
  __device__ void prefetch_src(int p, int, int, int logN) const {
    for (int j = 0; j < tab.ns; j++) l2_prefetch(acc + (size_t)p * acc_stride + ((size_t)(lvl + j) << logN), 8u << logN);
  }
  __device__ u64 get(const State& st, int j) const { return st.eval(j); }
  template <int G>
  __device__ void getg(const State& st, int k0, int stride, u64 (&y)[G]) const {
    st.template evalg<G>(k0, stride, y);
  }
};

struct EpiModDown {
  const u64* acc;
  size_t acc_stride;
  u64* out;
  size_t out_stride;
  const u64* pinv;
  const u64* pinv_sh;
  // Optional addend for output poly p = (r*nb + b)*2 + t: addend + r*add_r + b*add_b + t*add_p,
  // read through sigma_{g_r}; t = 1 only if add_both.
  const u64* addend;
  size_t add_r, add_b, add_p;
  int add_both;
  int nb;
  int accum;  // 1: out += result (each output element is written by one item of the launch)
  u64 g[CTL_MAX_ROT];
  struct State {
    const u64* a;
    u64* o;
    const u64* ad;
    u64 gg, q, pv, pvs;
    int lg;
  };
  __device__ void begin(State& st, int p, int l, int pi, const DPrime* pr, int logN) const {
    st.q = pr[pi].q;
    st.pv = __ldg(pinv + l);
    st.pvs = __ldg(pinv_sh + l);
    st.a = acc + (size_t)p * acc_stride + ((size_t)l << logN);
    st.o = out + (size_t)p * out_stride + ((size_t)l << logN);
    st.ad = nullptr;
    st.gg = 1;
    st.lg = logN;
    const int t = p & 1;
    if (addend && (t == 0 || add_both)) {
      const int rb = p >> 1, r = rb / nb, b = rb % nb;
      st.ad = addend + (size_t)r * add_r + (size_t)b * add_b + (size_t)t * add_p + ((size_t)l << logN);
      st.gg = g[r];
    }
  }
  __device__ void prefetch(const State& st, int logN) const {
    l2_prefetch(st.a, 8u << logN);
    if (st.ad) l2_prefetch(st.ad, 8u << logN);
    if (accum) l2_prefetch(st.o, 8u << logN);
  }
  // (acc - v) P^-1: the Shoup product takes acc + c*q - v for the bound c*q of v (4q, or
  // 64q with SMALL).  G elements j0 + g*stride at a time: every load of the group (acc
  // and the addend read-only in the launch, the running sum read by its owner only) is
  // issued before the first store, so the group's loads are in flight together.
  template <bool SMALL, int G>
  __device__ void putg(const State& st, int j0, int stride, const u64 (&v)[G]) const {
    const u64 cq = SMALL ? 64 * st.q : 4 * st.q;
    u64 a[G], ad[G], ac[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
      const uint32_t j = (uint32_t)(j0 + g * stride);
      a[g] = __ldg(st.a + j);
      ad[g] = st.ad ? __ldg(st.ad + (st.gg == 1 ? j : auto_src32(j, (uint32_t)st.gg, st.lg))) : 0;
      ac[g] = accum ? ld_own(st.o + j) : 0;
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
      u64 r = shoup_small(a[g] + cq - v[g], st.pv, st.pvs, st.q);  // below 4q
      r = reduce4(r, st.q);
      r = addmod(addmod(r, ad[g], st.q), ac[g], st.q);
      st.o[j0 + g * stride] = r;
    }
  }
};

struct EpiRescaleLast {   // inverse NTT of the last limb -> r = [x + h]_q_last
  u64* r_out;
  u64 h;
  struct State {
    u64* o;
    u64 q;
  };
  __device__ void begin(State& st, int p, int, int pi, const DPrime* pr, int logN) const {
    st.o = r_out + ((size_t)p << logN);
    st.q = pr[pi].q;
  }
  __device__ void put(const State& st, int j, u64 v) const { st.o[j] = addmod(reduce4(v, st.q), h, st.q); }
  __device__ void prefetch(const State&, int) const {}
};

struct ProRescale {       // (r - h) mod q_i in coefficient form
  static constexpr bool kStage = true;
  const u64* r;
  u64 h;
  struct State {
    const u64* g;
    u64 q, qinv, rm;
  };
  __device__ bool begin(State& st, int p, int, int pi, const DPrime* pr, int logN) const {
    st.g = r + ((size_t)p << logN);
    st.q = pr[pi].q;
    st.qinv = pr[pi].qinv;
    st.rm = pr[pi].rmod;
    return true;
  }
  __device__ void prefetch_src(int p, int, int, int logN) const { l2_prefetch(r + ((size_t)p << logN), 8u << logN); }
  __device__ u64 get(const State& st, int j) const {
    const u64 v = st.g[j];
    return v >= h ? mulmod_mont(v - h, st.rm, st.q, st.qinv) : negmod(mulmod_mont(h - v, st.rm, st.q, st.qinv), st.q);
  }
  template <int G>
  __device__ void getg(const State& st, int k0, int stride, u64 (&y)[G]) const {
    u64 v[G];
#pragma unroll
    for (int g = 0; g < G; g++) v[g] = st.g[k0 + g * stride];
#pragma unroll
    for (int g = 0; g < G; g++)
      y[g] = v[g] >= h ? mulmod_mont(v[g] - h, st.rm, st.q, st.qinv)
                       : negmod(mulmod_mont(h - v[g], st.rm, st.q, st.qinv), st.q);
  }
};

struct EpiRescale {       // out_i = (in_i - x) * q_last^-1
  const u64* in;
  size_t in_stride;
  u64* out;
  size_t out_stride;
  const u64* inv;
  const u64* inv_sh;
  struct State {
    const u64* a;
    u64* o;
    u64 q, w, ws;
  };
  __device__ void begin(State& st, int p, int l, int pi, const DPrime* pr, int logN) const {
    st.q = pr[pi].q;
    st.w = __ldg(inv + l);
    st.ws = __ldg(inv_sh + l);
    st.a = in + (size_t)p * in_stride + ((size_t)l << logN);
    st.o = out + (size_t)p * out_stride + ((size_t)l << logN);
  }
  // (in - v) q_last^-1 through one Shoup product of in + c*q - v (c*q the bound of v); the
  // input is read-only in the launch, so a group's loads go ahead of its stores
  template <bool SMALL, int G>
  __device__ void putg(const State& st, int j0, int stride, const u64 (&v)[G]) const {
    const u64 cq = SMALL ? 64 * st.q : 4 * st.q;
    u64 a[G];
#pragma unroll
    for (int g = 0; g < G; g++) a[g] = __ldg(st.a + j0 + g * stride);
#pragma unroll
    for (int g = 0; g < G; g++) st.o[j0 + g * stride] = reduce4(shoup_small(a[g] + cq - v[g], st.w, st.ws, st.q), st.q);
  }
  __device__ void prefetch(const State& st, int logN) const { l2_prefetch(st.a, 8u << logN); }
};

// ---------------------------------------------------------------------------------
// Register-resident kernels, N = 2^LOGN in {4096, 8192, 16384}: N/32 threads.
// Each limb's transform takes the small-prime path (no reductions inside the stages,
// one at the store) or the general one; the branch is the same for the whole block.
// ---------------------------------------------------------------------------------
// Forward stages and the epilogue of one item, inputs x[k] = element t + T*k.
template <int LOGN, bool SMALL, class Epi>
__device__ __forceinline__ void fwd32_body(u64* x, u64* smem, int t, const ulonglong2* __restrict__ W, u64 q,
                                           const Epi& epi, int p, int l, int pi, const DPrime* __restrict__ primes) {
  constexpr int N = 1 << LOGN, T = N / 32, RC = LOGN - 10, R = 1 << RC;
  // stages 0..4: sub-transform on elements t + T*k, block index 0
  fwd_regs<0, 5, SMALL>(x, 0, W, q);
#pragma unroll
  for (int k = 0; k < 32; k++) smem[pidx(t + T * k)] = x[k];
  __syncthreads();
  {  // stages 5..9
    const int b = t >> RC, o = t & (R - 1);
    const int base = (b << (LOGN - 5)) + o;
#pragma unroll
    for (int k = 0; k < 32; k++) x[k] = smem[pidx(base + (k << RC))];
    fwd_regs<5, 5, SMALL>(x, b, W, q);
#pragma unroll
    for (int k = 0; k < 32; k++) smem[pidx(base + (k << RC))] = x[k];
  }
  __syncthreads();
  // stages 10..LOGN-1: 32/R contiguous sub-transforms of R elements per thread
#pragma unroll
  for (int i = 0; i < 32 / R; i++) {
    const int b = t + T * i;
#pragma unroll
    for (int k = 0; k < R; k++) x[i * R + k] = smem[pidx(b * R + k)];
  }
#pragma unroll
  for (int i = 0; i < 32 / R; i++) fwd_regs<10, RC, SMALL>(x + i * R, t + T * i, W, q);
#pragma unroll
  for (int i = 0; i < 32 / R; i++) {
    const int b = t + T * i;
#pragma unroll
    for (int k = 0; k < R; k++) smem[pidx(b * R + k)] = x[i * R + k];
  }
  __syncthreads();
  typename Epi::State es;
  epi.begin(es, p, l, pi, primes, LOGN);
#pragma unroll 2
  for (int k0 = 0; k0 < 32; k0 += 4) {
    u64 v[4];
#pragma unroll
    for (int g = 0; g < 4; g++) v[g] = smem[pidx(t + T * (k0 + g))];
    epi.template putg<SMALL, 4>(es, t + T * k0, T, v);
  }
}

template <int LOGN, class Pro, class Epi>
__global__ void __launch_bounds__((1 << LOGN) / 32, 16384 / (1 << LOGN))
k_nttf_reg(const __grid_constant__ Pro pro, const __grid_constant__ Epi epi, const DPrime* __restrict__ primes,
           const ulonglong2* __restrict__ tw, int n_items, int lr, int limb_lo, int lvl, int L) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ u64 smem[];
  const int t = threadIdx.x;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    typename Pro::State ps;
    if (!pro.begin(ps, p, l, pi, primes, LOGN)) continue;
    if (threadIdx.x == 0) {  // L2 prefetch: this item's epilogue reads, the next item's sources
      typename Epi::State es;  // bound again after the transform (not live through it)
      epi.begin(es, p, l, pi, primes, LOGN);
      epi.prefetch(es, LOGN);
      const int nx = item + gridDim.x;
      if (nx < n_items) {
        const int p2 = nx / lr, l2 = limb_lo + nx % lr;
        pro.prefetch_src(p2, l2, l2 < lvl ? l2 : L + (l2 - lvl), LOGN);
      }
    }
    const DPrime& P = primes[pi];
    const u64 q = P.q;
    const ulonglong2* W = tw + ((size_t)pi << LOGN);
    u64 x[32];
    if constexpr (Pro::kStage) {
      // arithmetic-heavy prologue: each thread parks its own 32 inputs in shared memory
      // first (no barrier needed), so several loads are in flight while x[] is not live
#pragma unroll 4
      for (int k = 0; k < 32; k++) smem[pidx(t + T * k)] = pro.get(ps, t + T * k);
#pragma unroll
      for (int k = 0; k < 32; k++) x[k] = smem[pidx(t + T * k)];
    } else {
#pragma unroll
      for (int k = 0; k < 32; k++) x[k] = pro.get(ps, t + T * k);
    }
    if (fwd_small(P))
      fwd32_body<LOGN, true>(x, smem, t, W, q, epi, p, l, pi, primes);
    else
      fwd32_body<LOGN, false>(x, smem, t, W, q, epi, p, l, pi, primes);
    __syncthreads();
  }
}

// Inverse stages of one item from shared memory (its inputs stored there), outputs to
// the epilogue (below 4q).
template <int LOGN, bool SMALL, class Epi>
__device__ __forceinline__ void inv32_body(u64* x, u64* smem, int t, const ulonglong2* __restrict__ W, u64 q,
                                           const DPrime& P, const Epi& epi, int p, int l, int pi,
                                           const DPrime* __restrict__ primes) {
  constexpr int N = 1 << LOGN, T = N / 32, RC = LOGN - 10, R = 1 << RC;
  // stages LOGN-1..10 on contiguous sub-transforms
#pragma unroll
  for (int i = 0; i < 32 / R; i++) {
    const int b = t + T * i;
#pragma unroll
    for (int k = 0; k < R; k++) x[i * R + k] = smem[pidx(b * R + k)];
  }
#pragma unroll
  for (int i = 0; i < 32 / R; i++) inv_regs<10, RC, DPrime, SMALL, LOGN>(x + i * R, t + T * i, W, q, P);
#pragma unroll
  for (int i = 0; i < 32 / R; i++) {
    const int b = t + T * i;
#pragma unroll
    for (int k = 0; k < R; k++) smem[pidx(b * R + k)] = x[i * R + k];
  }
  __syncthreads();
  {  // stages 9..5
    const int b = t >> RC, o = t & (R - 1);
    const int base = (b << (LOGN - 5)) + o;
#pragma unroll
    for (int k = 0; k < 32; k++) x[k] = smem[pidx(base + (k << RC))];
    inv_regs<5, 5, DPrime, SMALL, LOGN>(x, b, W, q, P);
#pragma unroll
    for (int k = 0; k < 32; k++) smem[pidx(base + (k << RC))] = x[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 32; k++) x[k] = smem[pidx(t + T * k)];
  // stages 4..0 (N^-1 folded into stage 0), outputs straight to global
  inv_regs<0, 5, DPrime, SMALL, LOGN>(x, 0, W, q, P);
  typename Epi::State es;
  epi.begin(es, p, l, pi, primes, LOGN);
#pragma unroll
  for (int k = 0; k < 32; k++) epi.put(es, t + T * k, x[k]);
}

template <int LOGN, class Pro, class Epi>
__global__ void __launch_bounds__((1 << LOGN) / 32, 16384 / (1 << LOGN))
k_ntti_reg(const __grid_constant__ Pro pro, const __grid_constant__ Epi epi, const DPrime* __restrict__ primes,
           const ulonglong2* __restrict__ tw, int n_items, int lr, int limb_lo, int lvl, int L,
           const InvScale* __restrict__ scl) {
  constexpr int N = 1 << LOGN, T = N / 32;
  extern __shared__ u64 smem[];
  const int t = threadIdx.x;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    typename Pro::State ps;
    if (!pro.begin(ps, p, l, pi, primes, LOGN)) continue;
    if (threadIdx.x == 0) {  // L2 prefetch: this item's epilogue reads, the next item's sources
      typename Epi::State es;  // bound again after the transform (not live through it)
      epi.begin(es, p, l, pi, primes, LOGN);
      epi.prefetch(es, LOGN);
      const int nx = item + gridDim.x;
      if (nx < n_items) {
        const int p2 = nx / lr, l2 = limb_lo + nx % lr;
        pro.prefetch_src(p2, l2, l2 < lvl ? l2 : L + (l2 - lvl), LOGN);
      }
    }
    DPrime P = primes[pi];
    if (scl) {  // output also multiplied by the factor folded into scl[pi]
      const InvScale f = scl[pi];
      P.ninv = f.ninv;
      P.ninv_sh = f.ninv_sh;
      P.iw1 = f.iw1;
      P.iw1_sh = f.iw1_sh;
    }
    const u64 q = P.q;
    const ulonglong2* W = tw + ((size_t)pi << LOGN);
    u64 x[32];
#pragma unroll 8
    for (int k = 0; k < 32; k++) smem[pidx(t + T * k)] = pro.get(ps, t + T * k);
    __syncthreads();
    if (inv_small(q, LOGN))
      inv32_body<LOGN, true>(x, smem, t, W, q, P, epi, p, l, pi, primes);
    else
      inv32_body<LOGN, false>(x, smem, t, W, q, P, epi, p, l, pi, primes);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Generic shared-memory kernels (any N = 2^logN, 16 <= N <= 16384).
// ---------------------------------------------------------------------------------
template <int LOGR>
__device__ __forceinline__ void fwd_pass(u64* s, int logN, int s0, const ulonglong2* __restrict__ tw, u64 q) {
  constexpr int R = 1 << LOGR;
  const int nsub = 1 << (logN - LOGR);
  const int log_tl = logN - s0 - LOGR;
  for (int p = threadIdx.x; p < nsub; p += blockDim.x) {
    const int b = p >> log_tl;
    const int o = p & ((1 << log_tl) - 1);
    const int base = (b << (logN - s0)) + o;
    u64 x[R];
#pragma unroll
    for (int k = 0; k < R; k++) x[k] = s[pidx(base + (k << log_tl))];
#pragma unroll
    for (int u = 0; u < LOGR; u++) {
      const int h = R >> (u + 1);
#pragma unroll
      for (int k = 0; k < R; k++) {
        if (k & h) continue;
        ct_bfly(x[k], x[k + h], __ldg(tw + (1 << (s0 + u)) + (b << u) + (k >> (LOGR - u))), q);
      }
    }
#pragma unroll
    for (int k = 0; k < R; k++) s[pidx(base + (k << log_tl))] = x[k];
  }
}

template <int LOGR>
__device__ __forceinline__ void inv_pass(u64* s, int logN, int s_lo, const ulonglong2* __restrict__ tw, u64 q,
                                         const DPrime& P) {
  constexpr int R = 1 << LOGR;
  const int nsub = 1 << (logN - LOGR);
  const int log_tl = logN - s_lo - LOGR;
  for (int p = threadIdx.x; p < nsub; p += blockDim.x) {
    const int b = p >> log_tl;
    const int o = p & ((1 << log_tl) - 1);
    const int base = (b << (logN - s_lo)) + o;
    u64 x[R];
#pragma unroll
    for (int k = 0; k < R; k++) x[k] = s[pidx(base + (k << log_tl))];
#pragma unroll
    for (int u = LOGR - 1; u >= 0; u--) {
      const int h = R >> (u + 1);
      const bool last = (s_lo + u) == 0;
#pragma unroll
      for (int k = 0; k < R; k++) {
        if (k & h) continue;
        if (last) {
          const u64 U = x[k], V = x[k + h];
          x[k] = shoup_lazy(U + V, P.ninv, P.ninv_sh, q);
          x[k + h] = shoup_lazy(U - V + 2 * q, P.iw1, P.iw1_sh, q);
        } else {
          gs_bfly(x[k], x[k + h], __ldg(tw + (1 << (s_lo + u)) + (b << u) + (k >> (LOGR - u))), q);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < R; k++) s[pidx(base + (k << log_tl))] = x[k];
  }
}

// Pass plan: ceil(logN/4) passes, the first ones one stage larger when uneven.
__device__ __forceinline__ int pass_bits(int logN, int i) {
  const int np = (logN + 3) / 4;
  const int base = logN / np, extra = logN % np;
  return base + (i < extra ? 1 : 0);
}

template <class Pro, class Epi>
__global__ void __launch_bounds__(512) k_nttf_gen(const __grid_constant__ Pro pro, const __grid_constant__ Epi epi,
                                                  const DPrime* __restrict__ primes,
                                                  const ulonglong2* __restrict__ tw, int logN, int n_items, int lr,
                                                  int limb_lo, int lvl, int L) {
  extern __shared__ u64 smem[];
  const int N = 1 << logN;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    typename Pro::State ps;
    if (!pro.begin(ps, p, l, pi, primes, logN)) continue;
    typename Epi::State es;
    epi.begin(es, p, l, pi, primes, logN);
    for (int k = threadIdx.x; k < N; k += blockDim.x) smem[pidx(k)] = pro.get(ps, k);
    __syncthreads();
    const ulonglong2* W = tw + ((size_t)pi << logN);
    const u64 q = primes[pi].q;
    const int np = (logN + 3) / 4;
    int s0 = 0;
    for (int i = 0; i < np; i++) {
      const int r = pass_bits(logN, i);
      switch (r) {
        case 4: fwd_pass<4>(smem, logN, s0, W, q); break;
        case 3: fwd_pass<3>(smem, logN, s0, W, q); break;
        case 2: fwd_pass<2>(smem, logN, s0, W, q); break;
        default: fwd_pass<1>(smem, logN, s0, W, q); break;
      }
      __syncthreads();
      s0 += r;
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const u64 v[1] = {smem[pidx(k)]};
      epi.template putg<false, 1>(es, k, 0, v);
    }
    __syncthreads();
  }
}

template <class Pro, class Epi>
__global__ void __launch_bounds__(512) k_ntti_gen(const __grid_constant__ Pro pro, const __grid_constant__ Epi epi,
                                                  const DPrime* __restrict__ primes,
                                                  const ulonglong2* __restrict__ tw, int logN, int n_items, int lr,
                                                  int limb_lo, int lvl, int L, const InvScale* __restrict__ scl) {
  extern __shared__ u64 smem[];
  const int N = 1 << logN;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    typename Pro::State ps;
    if (!pro.begin(ps, p, l, pi, primes, logN)) continue;
    typename Epi::State es;
    epi.begin(es, p, l, pi, primes, logN);
    for (int k = threadIdx.x; k < N; k += blockDim.x) smem[pidx(k)] = pro.get(ps, k);
    __syncthreads();
    DPrime P = primes[pi];
    if (scl) {  // output also multiplied by the factor folded into scl[pi]
      const InvScale f = scl[pi];
      P.ninv = f.ninv;
      P.ninv_sh = f.ninv_sh;
      P.iw1 = f.iw1;
      P.iw1_sh = f.iw1_sh;
    }
    const ulonglong2* W = tw + ((size_t)pi << logN);
    const int np = (logN + 3) / 4;
    int top = logN;
    for (int i = 0; i < np; i++) {
      const int r = pass_bits(logN, i);
      const int s_lo = top - r;
      switch (r) {
        case 4: inv_pass<4>(smem, logN, s_lo, W, P.q, P); break;
        case 3: inv_pass<3>(smem, logN, s_lo, W, P.q, P); break;
        case 2: inv_pass<2>(smem, logN, s_lo, W, P.q, P); break;
        default: inv_pass<1>(smem, logN, s_lo, W, P.q, P); break;
      }
      __syncthreads();
      top = s_lo;
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) epi.put(es, k, smem[pidx(k)]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Register-resident kernels with 16 elements per thread (N/16 threads, 4-stage passes):
// half the registers per thread of the kernels above, so twice as many warps resident
// per SM to cover memory latency, at the price of one more shared-memory transpose.
// ---------------------------------------------------------------------------------
// Pass of stages [S0, S0 + LOGR) on sub-transforms of 2^LOGR elements, 16 / 2^LOGR per
// thread: sub-transform u = t + T*i is block b = u / D (block index at stage S0), offset
// o = u % D, elements b * (N >> S0) + o + k * D with D = N >> (S0 + LOGR).
template <int LOGN, int S0, int LOGR>
struct Pass16 {
  static constexpr int N = 1 << LOGN, T = N / 16, R = 1 << LOGR, NS = 16 / R, D = N >> (S0 + LOGR);
  __device__ __forceinline__ static int blk(int t, int i) { return (t + T * i) / D; }
  __device__ __forceinline__ static int pos(int t, int i, int k) {
    const int u = t + T * i;
    return (u / D) * (N >> S0) + (u % D) + k * D;
  }
  // pidx(pos(t, i, k)) = pidx(pos(t, i, 0)) + OFF(k) with OFF(k) = k*D + (k*D >> 4): the
  // first element of a sub-transform is o (mod D*R) with o < D, and D*R is a multiple of
  // 16 or the whole sub-transform stays inside one 16-element group.  So a sub-transform
  // needs one address register and compile-time offsets.
  __device__ __forceinline__ static constexpr int OFF(int k) { return k * D + ((k * D) >> 4); }
  __device__ __forceinline__ static void load(u64* x, const u64* smem, int t) {
#pragma unroll
    for (int i = 0; i < NS; i++) {
      const u64* s = smem + pidx(pos(t, i, 0));
#pragma unroll
      for (int k = 0; k < R; k++) x[i * R + k] = s[OFF(k)];
    }
  }
  __device__ __forceinline__ static void store(const u64* x, u64* smem, int t) {
#pragma unroll
    for (int i = 0; i < NS; i++) {
      u64* s = smem + pidx(pos(t, i, 0));
#pragma unroll
      for (int k = 0; k < R; k++) s[OFF(k)] = x[i * R + k];
    }
  }
  template <bool SMALL>
  __device__ __forceinline__ static void fwd(u64* x, int t, const ulonglong2* W, u64 q) {
#pragma unroll
    for (int i = 0; i < NS; i++) fwd_regs<S0, LOGR, SMALL>(x + i * R, blk(t, i), W, q);
  }
  template <bool SMALL>
  __device__ __forceinline__ static void inv(u64* x, int t, const ulonglong2* W, u64 q, const InvLast& P) {
#pragma unroll
    for (int i = 0; i < NS; i++) inv_regs<S0, LOGR, InvLast, SMALL, LOGN>(x + i * R, blk(t, i), W, q, P);
  }
};

// The last pass (stages S0 .. LOGN-1, sub-transforms of R = 2^LOGR consecutive elements)
// with warp w owning the 512 consecutive elements 512w .. 512w+511 and lane j its
// sub-transforms 512w/R + 32i + j (i < 16/R): consecutive lanes take consecutive
// sub-transforms (coalesced twiddles, conflict-free padded addresses), and the pass
// before it (stages 8..11, blocks of N/256 elements shared by N/4096 threads) wrote the
// warp's 512 elements from the same warp, so a warp barrier orders the exchange.
template <int LOGN, int S0, int LOGR>
struct PassLast16 {
  static_assert(S0 + LOGR == LOGN, "the last pass ends at stage LOGN");
  static constexpr int R = 1 << LOGR, NS = 16 / R, UW = 512 / R;
  __device__ __forceinline__ static int sub(int t, int i) { return (t >> 5) * UW + 32 * i + (t & 31); }
  __device__ __forceinline__ static void load(u64* x, const u64* smem, int t) {
#pragma unroll
    for (int i = 0; i < NS; i++) {
      const u64* s = smem + pidx(sub(t, i) * R);
#pragma unroll
      for (int k = 0; k < R; k++) x[i * R + k] = s[k];
    }
  }
  __device__ __forceinline__ static void store(const u64* x, u64* smem, int t) {
#pragma unroll
    for (int i = 0; i < NS; i++) {
      u64* s = smem + pidx(sub(t, i) * R);
#pragma unroll
      for (int k = 0; k < R; k++) s[k] = x[i * R + k];
    }
  }
  template <bool SMALL>
  __device__ __forceinline__ static void fwd(u64* x, int t, const ulonglong2* W, u64 q) {
#pragma unroll
    for (int i = 0; i < NS; i++) fwd_regs<S0, LOGR, SMALL>(x + i * R, sub(t, i), W, q);
  }
  template <bool SMALL>
  __device__ __forceinline__ static void inv(u64* x, int t, const ulonglong2* W, u64 q, const InvLast& P) {
#pragma unroll
    for (int i = 0; i < NS; i++) inv_regs<S0, LOGR, InvLast, SMALL, LOGN>(x + i * R, sub(t, i), W, q, P);
  }
};

// Barrier of the aligned group of G threads that exchange data between the second and
// third passes (G = N / 256: the threads of one block of N/16 elements at stage 4).  A
// warp barrier when the group fits a warp; otherwise named barriers 1..8 over groups of
// max(G, T/8) threads (T = N/16 threads; barrier 0 is the block's).
template <int LOGN>
__device__ __forceinline__ void pass12_sync(int t) {
  constexpr int N = 1 << LOGN, T = N / 16, G0 = N / 256, G = G0 > T / 8 ? G0 : T / 8;
  if constexpr (G0 <= 32) {
    __syncwarp();
  } else {
    static_assert(T / G <= 8 && G % 32 == 0, "at most 8 named groups of whole warps");
    asm volatile("bar.sync %0, %1;" ::"r"(1 + t / G), "n"(G) : "memory");
  }
}

// Forward passes and the epilogue of one item (16 elements per thread).
template <int LOGN, bool SMALL, class Epi>
__device__ __forceinline__ void fwd16_body(u64* x, u64* smem, int t, const ulonglong2* __restrict__ W, u64 q,
                                           const Epi& epi, int p, int l, int pi, const DPrime* __restrict__ primes) {
  constexpr int N = 1 << LOGN, T = N / 16, R3 = LOGN - 12;
  typedef Pass16<LOGN, 0, 4> P0;
  typedef Pass16<LOGN, 4, 4> P1;
  // Exchanges: all threads after the first pass, groups of N/256 threads after the second,
  // a warp after the third; the epilogue reads element t + T*k, so all threads again.
  P0::template fwd<SMALL>(x, t, W, q);
  P0::store(x, smem, t);
  __syncthreads();
  P1::load(x, smem, t);
  P1::template fwd<SMALL>(x, t, W, q);
  P1::store(x, smem, t);
  pass12_sync<LOGN>(t);
  if constexpr (R3 > 0) {
    typedef Pass16<LOGN, 8, 4> P2;
    typedef PassLast16<LOGN, 12, R3> P3;
    P2::load(x, smem, t);
    P2::template fwd<SMALL>(x, t, W, q);
    P2::store(x, smem, t);
    __syncwarp();
    P3::load(x, smem, t);
    P3::template fwd<SMALL>(x, t, W, q);
    P3::store(x, smem, t);
  } else {  // N = 4096: the third pass is the last
    typedef PassLast16<LOGN, 8, 4> P2;
    P2::load(x, smem, t);
    P2::template fwd<SMALL>(x, t, W, q);
    P2::store(x, smem, t);
  }
  __syncthreads();
  typename Epi::State es;
  epi.begin(es, p, l, pi, primes, LOGN);
#pragma unroll 2
  for (int k0 = 0; k0 < 16; k0 += 4) {
    u64 v[4];
#pragma unroll
    for (int g = 0; g < 4; g++) v[g] = smem[pidx(t + T * (k0 + g))];
    epi.template putg<SMALL, 4>(es, t + T * k0, T, v);
  }
}

template <int LOGN, class Pro, class Epi>
__global__ void __launch_bounds__((1 << LOGN) / 16, 16384 / (1 << LOGN))
k_nttf_r16(const __grid_constant__ Pro pro, const __grid_constant__ Epi epi, const DPrime* __restrict__ primes,
           const ulonglong2* __restrict__ tw, int n_items, int lr, int limb_lo, int lvl, int L) {
  static_assert(LOGN >= 12 && LOGN <= 14, "16-element kernels cover N = 4096 .. 16384");
  constexpr int N = 1 << LOGN, T = N / 16;
  extern __shared__ u64 smem[];
  const int t = threadIdx.x;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    typename Pro::State ps;
    if (!pro.begin(ps, p, l, pi, primes, LOGN)) continue;
    if (threadIdx.x == 0) {  // L2 prefetch: this item's epilogue reads, the next item's sources
      typename Epi::State es;  // bound again after the transform (not live through it)
      epi.begin(es, p, l, pi, primes, LOGN);
      epi.prefetch(es, LOGN);
      const int nx = item + gridDim.x;
      if (nx < n_items) {
        const int p2 = nx / lr, l2 = limb_lo + nx % lr;
        pro.prefetch_src(p2, l2, l2 < lvl ? l2 : L + (l2 - lvl), LOGN);
      }
    }
    const DPrime& P = primes[pi];
    const u64 q = P.q;
    const ulonglong2* W = tw + ((size_t)pi << LOGN);
    u64 x[16];
    if constexpr (Pro::kStage) {
      // groups of four elements, every source load of a group in flight together
#pragma unroll 1
      for (int k0 = 0; k0 < 16; k0 += 4) {
        u64 y[4];
        pro.template getg<4>(ps, t + T * k0, T, y);
#pragma unroll
        for (int g = 0; g < 4; g++) smem[pidx(t + T * (k0 + g))] = y[g];
      }
#pragma unroll
      for (int k = 0; k < 16; k++) x[k] = smem[pidx(t + T * k)];
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) x[k] = pro.get(ps, t + T * k);
    }
    if (fwd_small(P))
      fwd16_body<LOGN, true>(x, smem, t, W, q, epi, p, l, pi, primes);
    else
      fwd16_body<LOGN, false>(x, smem, t, W, q, epi, p, l, pi, primes);
    // No barrier before the next item: from the epilogue up to the next item's first
    // barrier a thread reads and writes only its own slots (elements t + T*k), and every
    // other thread's reads of them ended before the barrier that precedes the epilogue.
  }
}

// Inverse passes of one item from shared memory, outputs (below 4q) to the epilogue.
template <int LOGN, bool SMALL, class Epi>
__device__ __forceinline__ void inv16_body(u64* x, u64* smem, int t, const ulonglong2* __restrict__ W, u64 q,
                                           const InvLast& P, const Epi& epi, int p, int l, int pi,
                                           const DPrime* __restrict__ primes) {
  constexpr int N = 1 << LOGN, T = N / 16, R3 = LOGN - 12;
  typedef Pass16<LOGN, 0, 4> P0;
  typedef Pass16<LOGN, 4, 4> P1;
  // Exchanges (the caller's barrier precedes the first pass): a warp after the first pass,
  // groups of N/256 threads before the second to last, all threads before the last.
  if constexpr (R3 > 0) {
    typedef PassLast16<LOGN, 12, R3> P3;
    typedef Pass16<LOGN, 8, 4> P2;
    P3::load(x, smem, t);
    P3::template inv<SMALL>(x, t, W, q, P);
    P3::store(x, smem, t);
    __syncwarp();
    P2::load(x, smem, t);
    P2::template inv<SMALL>(x, t, W, q, P);
    P2::store(x, smem, t);
  } else {  // N = 4096: the first pass is stages 11..8
    typedef PassLast16<LOGN, 8, 4> P2;
    P2::load(x, smem, t);
    P2::template inv<SMALL>(x, t, W, q, P);
    P2::store(x, smem, t);
  }
  pass12_sync<LOGN>(t);
  P1::load(x, smem, t);
  P1::template inv<SMALL>(x, t, W, q, P);
  P1::store(x, smem, t);
  __syncthreads();
  P0::load(x, smem, t);
  // stages 3..0 (N^-1 folded into stage 0), outputs straight to global
  P0::template inv<SMALL>(x, t, W, q, P);
  typename Epi::State es;
  epi.begin(es, p, l, pi, primes, LOGN);
#pragma unroll
  for (int k = 0; k < 16; k++) epi.put(es, t + T * k, x[k]);
}

template <int LOGN, class Pro, class Epi>
__global__ void __launch_bounds__((1 << LOGN) / 16, 16384 / (1 << LOGN))
k_ntti_r16(const __grid_constant__ Pro pro, const __grid_constant__ Epi epi, const DPrime* __restrict__ primes,
           const ulonglong2* __restrict__ tw, int n_items, int lr, int limb_lo, int lvl, int L,
           const InvScale* __restrict__ scl) {
  static_assert(LOGN >= 12 && LOGN <= 14, "16-element kernels cover N = 4096 .. 16384");
  constexpr int N = 1 << LOGN, T = N / 16;
  extern __shared__ u64 smem[];
  const int t = threadIdx.x;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    typename Pro::State ps;
    if (!pro.begin(ps, p, l, pi, primes, LOGN)) continue;
    if (threadIdx.x == 0) {  // L2 prefetch: this item's epilogue reads, the next item's sources
      typename Epi::State es;  // bound again after the transform (not live through it)
      epi.begin(es, p, l, pi, primes, LOGN);
      epi.prefetch(es, LOGN);
      const int nx = item + gridDim.x;
      if (nx < n_items) {
        const int p2 = nx / lr, l2 = limb_lo + nx % lr;
        pro.prefetch_src(p2, l2, l2 < lvl ? l2 : L + (l2 - lvl), LOGN);
      }
    }
    const u64 q = primes[pi].q;
    InvLast P;
    if (scl) {  // output also multiplied by the factor folded into scl[pi]
      const InvScale f = scl[pi];
      P = InvLast{f.ninv, f.ninv_sh, f.iw1, f.iw1_sh};
    } else {
      P = InvLast{primes[pi].ninv, primes[pi].ninv_sh, primes[pi].iw1, primes[pi].iw1_sh};
    }
    const ulonglong2* W = tw + ((size_t)pi << LOGN);
    u64 x[16];
#pragma unroll 8
    for (int k = 0; k < 16; k++) smem[pidx(t + T * k)] = pro.get(ps, t + T * k);
    __syncthreads();
    if (inv_small(q, LOGN))
      inv16_body<LOGN, true>(x, smem, t, W, q, P, epi, p, l, pi, primes);
    else
      inv16_body<LOGN, false>(x, smem, t, W, q, P, epi, p, l, pi, primes);
    // No barrier before the next item: after the last barrier of the transform a thread
    // reads only its own slots (elements t + T*k), the ones its next prologue writes.
  }
}

// ---------------------------------------------------------------------------------
// Launch helpers.
// ---------------------------------------------------------------------------------
static inline size_t ntt_smem(int N) { return (size_t)(N + N / 16) * sizeof(u64); }

template <class K>
static int grid_for(ctl_context* c, K kern, int threads, size_t smem, int items) {
  static std::map<std::pair<const void*, size_t>, int> cache;
  static std::mutex mu;
  int per_sm;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair((const void*)kern, smem);
    auto it = cache.find(key);
    if (it == cache.end()) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
      if (per_sm < 1) per_sm = 1;
      cache[key] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  int g = c->sm_count * per_sm;
  return items < g ? items : g;
}

template <bool INV, int LOGN, class Pro, class Epi>
static void launch_reg(ctl_context* c, const Pro& pro, const Epi& epi, int items, int lr, int limb_lo, int lvl,
                       const InvScale* scl) {
  const size_t sm = ntt_smem(1 << LOGN);
  const ulonglong2* tw = (const ulonglong2*)(INV ? c->d_itw2 : c->d_tw2);
  if ((INV ? c->ntt_shape_inv : c->ntt_shape_fwd) == CTL_NTT_SHAPE_R16) {
    const int th = (1 << LOGN) / 16;
    if constexpr (INV) {
      auto kern = k_ntti_r16<LOGN, Pro, Epi>;
      const int grid = grid_for(c, kern, th, sm, items);
      kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, tw, items, lr, limb_lo, lvl, (int)c->L, scl);
    } else {
      auto kern = k_nttf_r16<LOGN, Pro, Epi>;
      const int grid = grid_for(c, kern, th, sm, items);
      kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, tw, items, lr, limb_lo, lvl, (int)c->L);
    }
    return;
  }
  const int th = (1 << LOGN) / 32;
  if constexpr (INV) {
    auto kern = k_ntti_reg<LOGN, Pro, Epi>;
    const int grid = grid_for(c, kern, th, sm, items);
    kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, tw, items, lr, limb_lo, lvl, (int)c->L, scl);
  } else {
    auto kern = k_nttf_reg<LOGN, Pro, Epi>;
    const int grid = grid_for(c, kern, th, sm, items);
    kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, tw, items, lr, limb_lo, lvl, (int)c->L);
  }
}

// Algorithmic cost of one launch: modular multiplications and HBM bytes (every operand
// read once and every result written once), accumulated per kernel class for the
// rooflines.
struct Cost {
  double work, bytes;
};

template <bool INV, class Pro, class Epi>
static void run_ntt(ctl_context* c, int cls, const Pro& pro, const Epi& epi, int n_polys, int limb_lo, int limb_hi,
                    int lvl, Cost cost, const InvScale* scl = nullptr) {
  const int lr = limb_hi - limb_lo;
  const int items = n_polys * lr;
  if (items <= 0) return;
  cudaEvent_t ev;
  timing_begin(c, cls, &ev);
  switch (c->logN) {
    case 12: launch_reg<INV, 12>(c, pro, epi, items, lr, limb_lo, lvl, scl); break;
    case 13: launch_reg<INV, 13>(c, pro, epi, items, lr, limb_lo, lvl, scl); break;
    case 14: launch_reg<INV, 14>(c, pro, epi, items, lr, limb_lo, lvl, scl); break;
    default: {
      const int N = (int)c->N;
      int th = N / 16;
      th = th < 32 ? 32 : (th > 512 ? 512 : th);
      const size_t sm = ntt_smem(N);
      const ulonglong2* tw = (const ulonglong2*)(INV ? c->d_itw2 : c->d_tw2);
      if constexpr (INV) {
        auto kern = k_ntti_gen<Pro, Epi>;
        const int grid = grid_for(c, kern, th, sm, items);
        kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, tw, (int)c->logN, items, lr, limb_lo, lvl,
                                          (int)c->L, scl);
      } else {
        auto kern = k_nttf_gen<Pro, Epi>;
        const int grid = grid_for(c, kern, th, sm, items);
        kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, tw, (int)c->logN, items, lr, limb_lo, lvl,
                                          (int)c->L);
      }
    }
  }
  c->launch_count++;
  timing_end(c, cls, ev, cost.work, cost.bytes);
}

static inline double butterflies(const ctl_context* c) { return 0.5 * c->N * c->logN; }
// A plain limb transform of `limbs` limbs: butterflies (plus one product per coefficient
// when a scale is folded in), one limb read and one written each.
static inline Cost limb_cost(const ctl_context* c, double limbs, bool scaled = false) {
  const double N = (double)c->N;
  return {limbs * (butterflies(c) + (scaled ? N : 0.0)), limbs * 16.0 * N};
}

}  // namespace ctl
