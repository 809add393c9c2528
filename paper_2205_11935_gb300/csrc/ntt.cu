// Negacyclic NTT / inverse NTT over word-size primes, with fused key-switching and
// rescaling prologues/epilogues.
//
// Definition (the NTT form of a in Z_q[X]/(X^N+1)):  a_hat[k] = a(psi^(2*bitrev(k)+1)),
// psi the smallest primitive 2N-th root of unity mod q; outputs in bit-reversed order.
// Forward: Cooley-Tukey butterflies with the psi powers merged (twiddle table
// tw[i] = psi^bitrev(i)); inverse: Gentleman-Sande butterflies with (psi^-1)^bitrev(i)
// and N^-1 folded into the last stage.  Values stay lazily reduced (Harvey): forward
// butterflies keep [0, 4q), inverse [0, 2q); q < 2^62.
//
// GPU mapping: one CTA owns one limb (N <= 16384 words, 128 KiB) in shared memory,
// padded by one word every 16 to spread the strided accesses over the banks.  Stages
// are grouped into passes of up to four (radix-16 sub-transforms held in registers);
// each pass is one shared-memory round trip.  CTAs loop over the limbs of a batch.
//
// CKKS (Sec. 3.1 of CryptoTL) needs these transforms around every key switch
// (rotations, relinearisation) and every rescale; the functors below fuse the fast base
// conversions of ModUp/ModDown and the rescale arithmetic into the load/store phases so
// that each converted limb makes one trip through HBM.
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

template <int LOGR>
__device__ __forceinline__ void fwd_pass(u64* s, int logN, int s0, const u64* __restrict__ tw,
                                         const u64* __restrict__ tws, u64 q) {
  constexpr int R = 1 << LOGR;
  const int nsub = 1 << (logN - LOGR);
  const int log_tl = logN - s0 - LOGR;
  const u64 q2 = 2 * q;
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
        const int widx = (1 << (s0 + u)) + (b << u) + (k >> (LOGR - u));
        const u64 w = __ldg(tw + widx), wsh = __ldg(tws + widx);
        u64 X = x[k];
        if (X >= q2) X -= q2;
        const u64 T = shoup_lazy(x[k + h], w, wsh, q);
        x[k] = X + T;
        x[k + h] = X - T + q2;
      }
    }
#pragma unroll
    for (int k = 0; k < R; k++) s[pidx(base + (k << log_tl))] = x[k];
  }
}

template <int LOGR>
__device__ __forceinline__ void inv_pass(u64* s, int logN, int s_lo, const u64* __restrict__ tw,
                                         const u64* __restrict__ tws, u64 q, const DPrime& P) {
  constexpr int R = 1 << LOGR;
  const int nsub = 1 << (logN - LOGR);
  const int log_tl = logN - s_lo - LOGR;
  const u64 q2 = 2 * q;
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
        const u64 U = x[k], V = x[k + h];
        if (last) {
          x[k] = shoup_lazy(U + V, P.ninv, P.ninv_sh, q);
          x[k + h] = shoup_lazy(U - V + q2, P.iw1, P.iw1_sh, q);
        } else {
          const int widx = (1 << (s_lo + u)) + (b << u) + (k >> (LOGR - u));
          const u64 w = __ldg(tw + widx), wsh = __ldg(tws + widx);
          u64 S = U + V;
          if (S >= q2) S -= q2;
          x[k] = S;
          x[k + h] = shoup_lazy(U - V + q2, w, wsh, q);
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

__device__ __forceinline__ void ntt_fwd_core(u64* s, int logN, const u64* tw, const u64* tws, u64 q) {
  const int np = (logN + 3) / 4;
  int s0 = 0;
  for (int i = 0; i < np; i++) {
    const int r = pass_bits(logN, i);
    switch (r) {
      case 4: fwd_pass<4>(s, logN, s0, tw, tws, q); break;
      case 3: fwd_pass<3>(s, logN, s0, tw, tws, q); break;
      case 2: fwd_pass<2>(s, logN, s0, tw, tws, q); break;
      default: fwd_pass<1>(s, logN, s0, tw, tws, q); break;
    }
    __syncthreads();
    s0 += r;
  }
}

__device__ __forceinline__ void ntt_inv_core(u64* s, int logN, const u64* tw, const u64* tws, u64 q, const DPrime& P) {
  const int np = (logN + 3) / 4;
  int top = logN;
  for (int i = 0; i < np; i++) {
    const int r = pass_bits(logN, i);
    const int s_lo = top - r;
    switch (r) {
      case 4: inv_pass<4>(s, logN, s_lo, tw, tws, q, P); break;
      case 3: inv_pass<3>(s, logN, s_lo, tw, tws, q, P); break;
      case 2: inv_pass<2>(s, logN, s_lo, tw, tws, q, P); break;
      default: inv_pass<1>(s, logN, s_lo, tw, tws, q, P); break;
    }
    __syncthreads();
    top = s_lo;
  }
}

// ---------------------------------------------------------------------------------
// Load / store functors.  load() fills s[pidx(k)], k < N, and returns true, or handles
// the item itself and returns false (uniformly for the block).
// ---------------------------------------------------------------------------------
struct ProLoad {
  const u64* src;
  size_t poly_stride;
  __device__ bool load(u64* s, int p, int l, int, const DPrime*, int N) const {
    const u64* g = src + (size_t)p * poly_stride + (size_t)l * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) s[pidx(k)] = g[k];
    return true;
  }
};

struct EpiStore {
  u64* dst;
  size_t poly_stride;
  __device__ void store(const u64* s, int p, int l, int pi, const DPrime* pr, int N) const {
    const u64 q = pr[pi].q;
    u64* g = dst + (size_t)p * poly_stride + (size_t)l * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) g[k] = reduce4(s[pidx(k)], q);
  }
};

// Fast base conversion of one coefficient: y = sum_j [x_j * Shat_j^-1]_{s_j} * Shat_j
// mod t (the constant Shat_j mod t held in Montgomery form), exact residue in [0, t).
__device__ __forceinline__ u64 conv_coef(const ConvTab& T, int tpos, const u64* const* srcs, int k, u64 t,
                                         u64 tinv) {
  u64 lo = 0, hi = 0;
  for (int j = 0; j < T.ns; j++) {
    const u64 sj = __ldg(T.sq + j);
    const u64 v = shoup(srcs[j][k], __ldg(T.sinv + j), __ldg(T.sinv_sh + j), sj);
    mac(lo, hi, v, __ldg(T.cmont + (size_t)j * T.nt + tpos));
  }
  return redc(hi, lo, t, tinv);
}

#define CTL_MAX_DIGITS 16
struct ProModUp {
  const u64* coef;   // c1 coefficient form, input b's limbs at coef + b*coef_stride
  size_t coef_stride;
  const u64* ntt;    // c1 NTT form, input b's limbs at ntt + b*stride
  size_t stride;
  u64* ext;          // [nb][nd][E][N]
  int nd, E, lvl, alpha;
  ConvTab tabs[CTL_MAX_DIGITS];
  __device__ bool load(u64* s, int p, int l, int pi, const DPrime* pr, int N) const {
    const int b = p / nd, d = p % nd;
    const int d0 = d * alpha, d1 = min(d0 + alpha, lvl);
    if (l >= d0 && l < d1) {  // the digit's own primes: y = x mod q_l, already in NTT form
      const u64* g = ntt + (size_t)b * stride + (size_t)l * N;
      u64* o = ext + ((size_t)p * E + l) * N;
      for (int k = threadIdx.x; k < N; k += blockDim.x) o[k] = g[k];
      return false;
    }
    const u64* srcs[8];
    const ConvTab& T = tabs[d];
    for (int j = 0; j < T.ns; j++) srcs[j] = coef + (size_t)b * coef_stride + (size_t)(d0 + j) * N;
    const u64 t = pr[pi].q, tinv = pr[pi].qinv;
    for (int k = threadIdx.x; k < N; k += blockDim.x) s[pidx(k)] = conv_coef(T, l, srcs, k, t, tinv);
    return true;
  }
};

struct ProModDown {
  const u64* acc;    // [np][E][N], special limbs (positions lvl..lvl+K-1) in coefficient form
  size_t acc_stride;
  int lvl;
  ConvTab tab;       // sources: special primes; target position = data limb index
  __device__ bool load(u64* s, int p, int l, int pi, const DPrime* pr, int N) const {
    const u64* srcs[8];
    for (int j = 0; j < tab.ns; j++) srcs[j] = acc + (size_t)p * acc_stride + (size_t)(lvl + j) * N;
    const u64 t = pr[pi].q, tinv = pr[pi].qinv;
    for (int k = threadIdx.x; k < N; k += blockDim.x) s[pidx(k)] = conv_coef(tab, l, srcs, k, t, tinv);
    return true;
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
  u64 g[CTL_MAX_ROT];
  int nb;
  int logN;
  __device__ void store(const u64* s, int p, int l, int pi, const DPrime* pr, int N) const {
    const u64 q = pr[pi].q;
    const u64 pv = __ldg(pinv + l), pvs = __ldg(pinv_sh + l);
    const u64* a = acc + (size_t)p * acc_stride + (size_t)l * N;
    u64* o = out + (size_t)p * out_stride + (size_t)l * N;
    const u64* ad = nullptr;
    u64 g = 1;
    const int t = p & 1;
    if (addend && (t == 0 || add_both)) {
      const int rb = p >> 1, r = rb / nb, b = rb % nb;
      ad = addend + (size_t)r * add_r + (size_t)b * add_b + (size_t)t * add_p + (size_t)l * N;
      g = this->g[r];
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const u64 x = reduce4(s[pidx(k)], q);
      u64 v = shoup(submod(a[k], x, q), pv, pvs, q);
      if (ad) v = addmod(v, ad[g == 1 ? k : auto_src(k, g, logN)], q);
      o[k] = v;
    }
  }
};

struct EpiRescaleLast {   // inverse NTT of the last limb -> r = [x + h]_q_last
  u64* r_out;
  u64 h;
  __device__ void store(const u64* s, int p, int, int pi, const DPrime* pr, int N) const {
    const u64 q = pr[pi].q;
    u64* o = r_out + (size_t)p * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) o[k] = addmod(reduce4(s[pidx(k)], q), h, q);
  }
};

struct ProRescale {       // (r - h) mod q_i in coefficient form
  const u64* r;
  u64 h;
  __device__ bool load(u64* s, int p, int, int pi, const DPrime* pr, int N) const {
    const u64 q = pr[pi].q, qinv = pr[pi].qinv, rm = pr[pi].rmod;
    const u64* g = r + (size_t)p * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const u64 v = g[k];
      s[pidx(k)] = v >= h ? mulmod_mont(v - h, rm, q, qinv) : negmod(mulmod_mont(h - v, rm, q, qinv), q);
    }
    return true;
  }
};

struct EpiRescale {       // out_i = (in_i - x) * q_last^-1
  const u64* in;
  size_t in_stride;
  u64* out;
  size_t out_stride;
  const u64* inv;
  const u64* inv_sh;
  __device__ void store(const u64* s, int p, int l, int pi, const DPrime* pr, int N) const {
    const u64 q = pr[pi].q;
    const u64 w = __ldg(inv + l), ws = __ldg(inv_sh + l);
    const u64* a = in + (size_t)p * in_stride + (size_t)l * N;
    u64* o = out + (size_t)p * out_stride + (size_t)l * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) o[k] = shoup(submod(a[k], reduce4(s[pidx(k)], q), q), w, ws, q);
  }
};

// ---------------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------------
template <class Pro, class Epi>
__global__ void __launch_bounds__(512) k_ntt_fwd(Pro pro, Epi epi, const DPrime* __restrict__ primes,
                                                 const u64* __restrict__ tw, const u64* __restrict__ tws, int logN,
                                                 int n_items, int lr, int limb_lo, int lvl, int L) {
  extern __shared__ u64 smem[];
  const int N = 1 << logN;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    if (!pro.load(smem, p, l, pi, primes, N)) continue;
    __syncthreads();
    ntt_fwd_core(smem, logN, tw + (size_t)pi * N, tws + (size_t)pi * N, primes[pi].q);
    epi.store(smem, p, l, pi, primes, N);
    __syncthreads();
  }
}

template <class Pro, class Epi>
__global__ void __launch_bounds__(512) k_ntt_inv(Pro pro, Epi epi, const DPrime* __restrict__ primes,
                                                 const u64* __restrict__ tw, const u64* __restrict__ tws, int logN,
                                                 int n_items, int lr, int limb_lo, int lvl, int L) {
  extern __shared__ u64 smem[];
  const int N = 1 << logN;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int p = item / lr, l = limb_lo + item % lr;
    const int pi = l < lvl ? l : L + (l - lvl);
    if (!pro.load(smem, p, l, pi, primes, N)) continue;
    __syncthreads();
    const DPrime P = primes[pi];
    ntt_inv_core(smem, logN, tw + (size_t)pi * N, tws + (size_t)pi * N, P.q, P);
    epi.store(smem, p, l, pi, primes, N);
    __syncthreads();
  }
}

static int ntt_threads(int N) {
  int t = N / 16;
  if (t < 32) t = 32;
  if (t > 512) t = 512;
  return t;
}
static size_t ntt_smem(int N) { return (size_t)(N + N / 16) * sizeof(u64); }

template <class K>
static int grid_for(ctl_context* c, K kern, int threads, size_t smem, int items) {
  static thread_local std::map<std::pair<const void*, size_t>, int> cache;
  auto key = std::make_pair((const void*)kern, smem);
  auto it = cache.find(key);
  int per_sm;
  if (it == cache.end()) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) per_sm = 1;
    cache[key] = per_sm;
  } else {
    per_sm = it->second;
  }
  int g = c->sm_count * per_sm;
  return items < g ? items : g;
}

template <class Pro, class Epi>
static void run_fwd(ctl_context* c, int cls, const Pro& pro, const Epi& epi, int n_polys, int limb_lo, int limb_hi,
                    int lvl, double work_per_limb) {
  const int lr = limb_hi - limb_lo;
  const int items = n_polys * lr;
  if (items <= 0) return;
  const int N = (int)c->N, th = ntt_threads(N);
  const size_t sm = ntt_smem(N);
  auto kern = k_ntt_fwd<Pro, Epi>;
  const int grid = grid_for(c, kern, th, sm, items);
  cudaEvent_t ev;
  timing_begin(c, cls, &ev);
  kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, c->d_tw, c->d_tw_sh, (int)c->logN, items, lr, limb_lo, lvl,
                                    (int)c->L);
  c->launch_count++;
  timing_end(c, cls, ev, work_per_limb * items);
}

template <class Pro, class Epi>
static void run_inv(ctl_context* c, int cls, const Pro& pro, const Epi& epi, int n_polys, int limb_lo, int limb_hi,
                    int lvl, double work_per_limb) {
  const int lr = limb_hi - limb_lo;
  const int items = n_polys * lr;
  if (items <= 0) return;
  const int N = (int)c->N, th = ntt_threads(N);
  const size_t sm = ntt_smem(N);
  auto kern = k_ntt_inv<Pro, Epi>;
  const int grid = grid_for(c, kern, th, sm, items);
  cudaEvent_t ev;
  timing_begin(c, cls, &ev);
  kern<<<grid, th, sm, c->stream>>>(pro, epi, c->d_primes, c->d_itw, c->d_itw_sh, (int)c->logN, items, lr, limb_lo,
                                    lvl, (int)c->L);
  c->launch_count++;
  timing_end(c, cls, ev, work_per_limb * items);
}

static double butterflies(const ctl_context* c) { return 0.5 * c->N * c->logN; }

void launch_ntt_fwd(ctl_context* c, u64* data, size_t poly_stride, int n_polys, int limb_lo, int limb_hi, int lvl) {
  run_fwd(c, KC_NTT_FWD, ProLoad{data, poly_stride}, EpiStore{data, poly_stride}, n_polys, limb_lo, limb_hi, lvl,
          butterflies(c));
}

void launch_ntt_inv(ctl_context* c, u64* data, size_t poly_stride, int n_polys, int limb_lo, int limb_hi, int lvl) {
  run_inv(c, KC_NTT_INV, ProLoad{data, poly_stride}, EpiStore{data, poly_stride}, n_polys, limb_lo, limb_hi, lvl,
          butterflies(c));
}

void launch_intt_rescale_last(ctl_context* c, const u64* in, size_t poly_stride, int n_polys, int lvl, u64* r_out) {
  const RescaleTab& R = c->rescale_tabs[lvl];
  // limb lvl-1 of poly p is read at in + p*poly_stride + (lvl-1)*N; the store functor
  // writes r_out[p].
  run_inv(c, KC_RESCALE, ProLoad{in, poly_stride}, EpiRescaleLast{r_out, R.h}, n_polys, lvl - 1, lvl, lvl,
          butterflies(c));
}

void launch_rescale_ntt(ctl_context* c, const u64* r, const u64* in, size_t in_stride, u64* out, size_t out_stride,
                        int n_polys, int lvl) {
  const RescaleTab& R = c->rescale_tabs[lvl];
  run_fwd(c, KC_RESCALE, ProRescale{r, R.h}, EpiRescale{in, in_stride, out, out_stride, R.inv, R.inv_sh}, n_polys, 0,
          lvl - 1, lvl, butterflies(c) + 2.0 * c->N);
}

void launch_modup_ntt(ctl_context* c, const u64* src_coef, size_t coef_stride, const u64* src_ntt, size_t src_stride,
                      int nb, int lvl, u64* ext) {
  const int nd = (lvl + (int)c->alpha - 1) / (int)c->alpha;
  const int E = lvl + (int)c->K;
  ProModUp pro;
  pro.coef = src_coef;
  pro.coef_stride = coef_stride;
  pro.ntt = src_ntt;
  pro.stride = src_stride;
  pro.ext = ext;
  pro.nd = nd;
  pro.E = E;
  pro.lvl = lvl;
  pro.alpha = (int)c->alpha;
  for (int d = 0; d < nd && d < CTL_MAX_DIGITS; d++) pro.tabs[d] = c->modup_tabs[(size_t)(lvl - 1) * c->beta + d];
  run_fwd(c, KC_MODUP, pro, EpiStore{ext, (size_t)E * c->N}, nb * nd, 0, E, lvl,
          butterflies(c) + (double)c->alpha * 2.0 * c->N);
}

void launch_moddown_ntt(ctl_context* c, const u64* acc, int nr, int nb, int lvl, u64* out, const u64* addend,
                        size_t add_r, size_t add_b, size_t add_p, bool add_both, const RotList& rl) {
  const int E = lvl + (int)c->K;
  ProModDown pro{acc, (size_t)E * c->N, lvl, c->moddown.conv};
  EpiModDown epi;
  epi.acc = acc;
  epi.acc_stride = (size_t)E * c->N;
  epi.out = out;
  epi.out_stride = (size_t)lvl * c->N;
  epi.pinv = c->moddown.pinv;
  epi.pinv_sh = c->moddown.pinv_sh;
  epi.addend = addend;
  epi.add_r = add_r;
  epi.add_b = add_b;
  epi.add_p = add_p;
  epi.add_both = add_both ? 1 : 0;
  for (int r = 0; r < CTL_MAX_ROT; r++) epi.g[r] = r < rl.n ? rl.g[r] : 1;
  epi.nb = nb;
  epi.logN = (int)c->logN;
  run_fwd(c, KC_MODDOWN, pro, epi, nr * nb * 2, 0, lvl, lvl, butterflies(c) + (double)(c->K * 2 + 1) * c->N);
}

void launch_ntt_inv_oop(ctl_context* c, const u64* src, size_t src_stride, u64* dst, size_t dst_stride, int n_polys,
                        int limb_lo, int limb_hi, int lvl) {
  // limb l of poly p: read at src + p*src_stride + l*N, written at dst + p*dst_stride + l*N
  run_inv(c, KC_NTT_INV, ProLoad{src, src_stride}, EpiStore{dst, dst_stride}, n_polys, limb_lo, limb_hi, lvl,
          butterflies(c));
}

}  // namespace ctl
