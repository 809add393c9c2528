// C-ABI of the ctl library: contexts, keys, ciphertexts and the homomorphic operations
// of CryptoTL's server step (ClassifyHE, Fig. alg:cryptotl; layers of Sec. 3.1).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <algorithm>
#include <memory>
#include <tuple>
#include <mutex>
#include <new>
#include <array>

#include "ctl_internal.h"
#include "modarith.cuh"

using namespace ctl;

// =====================================================================================
// Errors, memory, timing
// =====================================================================================
static thread_local std::string g_last_error;

namespace ctl {
const char* kKernelClassName[KC_COUNT] = {"ntt_fwd", "ntt_inv", "modup_ntt", "key_ip",
                                          "moddown_ntt", "rescale", "bsgs_inner", "elementwise"};

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}
int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CTL_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CTL_ENOMEM : CTL_ECUDA;
}
void* dev_alloc(ctl_context* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(bytes, (void*)c->stream, c->alloc_user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}
void dev_free(ctl_context* c, void* p) {
  if (!p) return;
  if (c->free_fn) c->free_fn(p, (void*)c->stream, c->alloc_user);
  else cudaFreeAsync(p, c->stream);
}
void timing_begin(ctl_context* c, int, cudaEvent_t* ev) {
  *ev = nullptr;
  if (!c->timing.enabled) return;
  cudaEvent_t e;
  if (!c->timing.pool.empty()) {
    e = c->timing.pool.back();
    c->timing.pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  cudaEventRecord(e, c->stream);
  *ev = e;
}
void timing_end(ctl_context* c, int cls, cudaEvent_t ev, double work, double bytes) {
  if (!c->timing.enabled || !ev) return;
  cudaEvent_t e;
  if (!c->timing.pool.empty()) {
    e = c->timing.pool.back();
    c->timing.pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  cudaEventRecord(e, c->stream);
  c->timing.pending.push_back({cls, {ev, e}});
  c->timing.launches[cls]++;
  c->timing.work[cls] += work;
  c->timing.bytes[cls] += bytes;
}
}  // namespace ctl

namespace {

#define CHECK_ARG(cond, msg)      \
  do {                            \
    if (!(cond)) {                \
      set_error("%s", msg);       \
      return CTL_EINVAL;          \
    }                             \
  } while (0)


}  // namespace

ctl_ct* ctl::new_ct(ctl_context* c, uint32_t lvl, uint32_t count, double scale) {
  ctl_ct* ct = new (std::nothrow) ctl_ct();
  if (!ct) return nullptr;
  ct->ctx = c;
  ct->level = lvl;
  ct->count = count;
  ct->scale = scale;
  ct->bytes = ct_words(c, lvl, count) * sizeof(u64);
  ct->d = (u64*)dev_alloc(c, ct->bytes);
  if (!ct->d) {
    delete ct;
    return nullptr;
  }
  return ct;
}

namespace {

// Scale agreement up to FP64 rounding of the bookkeeping.
bool same_scale(double a, double b) { return std::fabs(a - b) <= 1e-9 * std::max(std::fabs(a), std::fabs(b)); }

}  // namespace

// =====================================================================================
// Context
// =====================================================================================
extern "C" const char* ctl_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* ctl_version(void) { return "ctl 0.1 (sm_103a)"; }

extern "C" int ctl_plan_primes(uint32_t N, const uint32_t* bits, uint32_t n, uint64_t* out) {
  if (!bits || !out || n == 0) {
    set_error("ctl_plan_primes: null argument");
    return CTL_EINVAL;
  }
  std::vector<u64> ps;
  if (N < 16 || (N & (N - 1)) || !plan_primes(N, std::vector<uint32_t>(bits, bits + n), ps)) {
    set_error("ctl_plan_primes: invalid N or bit sizes");
    return CTL_EINVAL;
  }
  for (uint32_t i = 0; i < n; i++) out[i] = ps[i];
  return CTL_OK;
}

static int build_tables(ctl_context* c) {
  const uint32_t N = c->N, L = c->L, K = c->K, LK = L + K;
  const std::vector<u64>& m = c->moduli;
  // per-prime constants and twiddles
  // interleaved (w, w') pairs: tw2[(i*N + k)*2 + {0,1}]
  std::vector<u64> tw2((size_t)LK * N * 2), itw2((size_t)LK * N * 2);
  c->h_primes.resize(LK);
  for (uint32_t i = 0; i < LK; i++) {
    const u64 q = m[i];
    const u64 psi = min_primitive_2n_root(q, N), psi_inv = h_invmod(psi, q);
    for (uint32_t k = 0; k < N; k++) {
      const uint32_t e = h_bitrev(k, c->logN);
      const u64 w = h_powmod(psi, e, q), wi = h_powmod(psi_inv, e, q);
      tw2[((size_t)i * N + k) * 2] = w;
      tw2[((size_t)i * N + k) * 2 + 1] = h_shoup(w, q);
      itw2[((size_t)i * N + k) * 2] = wi;
      itw2[((size_t)i * N + k) * 2 + 1] = h_shoup(wi, q);
    }
    DPrime& P = c->h_primes[i];
    P.q = q;
    P.qinv = h_neg_inv64(q);
    P.rmod = h_mont(1, q);
    P.r2 = h_mulmod(P.rmod, P.rmod, q);
    P.ninv = h_invmod(N % q, q);
    P.ninv_sh = h_shoup(P.ninv, q);
    P.iw1 = h_mulmod(itw2[((size_t)i * N + 1) * 2], P.ninv, q);
    P.iw1_sh = h_shoup(P.iw1, q);
    const unsigned bits = 64 - __builtin_clzll(q);
    P.split = bits <= 54 ? kSplitW : 0;
    P.bar = q > (1ull << 32) ? (u64)((((unsigned __int128)1) << 64) / q) : 0;
  }
  // conversion tables, packed into one host vector then copied to the device
  std::vector<u64> tab;
  struct Pending {
    size_t c, c_sh;
    int ns, nt;
  };
  std::vector<Pending> modup_p;
  auto add_conv = [&](const std::vector<uint32_t>& src, const std::vector<uint32_t>& tgt) {
    Pending pd;
    pd.ns = (int)src.size();
    pd.nt = (int)tgt.size();
    pd.c = tab.size();
    for (uint32_t sj : src) {
      for (uint32_t ti : tgt) {
        const u64 qt = m[ti];
        u64 prod = 1 % qt;
        for (uint32_t so : src)
          if (so != sj) prod = h_mulmod(prod, m[so] % qt, qt);
        tab.push_back(prod);
      }
    }
    pd.c_sh = tab.size();
    for (int j = 0; j < pd.ns; j++)
      for (int i = 0; i < pd.nt; i++) tab.push_back(h_shoup(tab[pd.c + (size_t)j * pd.nt + i], m[tgt[i]]));
    return pd;
  };
  for (uint32_t lvl = 1; lvl <= L; lvl++) {
    for (uint32_t d = 0; d < c->beta; d++) {
      std::vector<uint32_t> src, tgt;
      for (uint32_t j = d * c->alpha; j < std::min((d + 1) * c->alpha, lvl); j++) src.push_back(j);
      for (uint32_t i = 0; i < lvl + K; i++) tgt.push_back(prime_of_limb(i, lvl, L));
      if (src.empty()) src.push_back(0);  // unused digit slot
      modup_p.push_back(add_conv(src, tgt));
    }
  }
  std::vector<uint32_t> sp, dp;
  for (uint32_t j = 0; j < K; j++) sp.push_back(L + j);
  for (uint32_t i = 0; i < L; i++) dp.push_back(i);
  Pending md = add_conv(sp, dp);
  const size_t pinv_off = tab.size();
  for (uint32_t i = 0; i < L; i++) {
    u64 P = 1;
    for (uint32_t j = 0; j < K; j++) P = h_mulmod(P, m[L + j] % m[i], m[i]);
    tab.push_back(h_invmod(P, m[i]));
  }
  const size_t pinvsh_off = tab.size();
  for (uint32_t i = 0; i < L; i++) tab.push_back(h_shoup(tab[pinv_off + i], m[i]));
  const size_t pmod_off = tab.size();
  for (uint32_t i = 0; i < L; i++) {
    u64 P = 1;
    for (uint32_t j = 0; j < K; j++) P = h_mulmod(P, m[L + j] % m[i], m[i]);
    tab.push_back(P);
  }
  const size_t pmodsh_off = tab.size();
  for (uint32_t i = 0; i < L; i++) tab.push_back(h_shoup(tab[pmod_off + i], m[i]));
  std::vector<size_t> rs_off(L + 1, 0);
  for (uint32_t lvl = 2; lvl <= L; lvl++) {
    const u64 ql = m[lvl - 1];
    rs_off[lvl] = tab.size();
    for (uint32_t i = 0; i + 1 < lvl; i++) tab.push_back(h_invmod(ql % m[i], m[i]));
    for (uint32_t i = 0; i + 1 < lvl; i++) tab.push_back(h_shoup(tab[rs_off[lvl] + i], m[i]));
    for (uint32_t i = 0; i + 1 < lvl; i++) tab.push_back((ql / 2) % m[i]);
  }
  // device copies
  const size_t twb = (size_t)LK * N * sizeof(u64);
  int rc;
  if ((rc = cuda_check(cudaMalloc(&c->d_primes, LK * sizeof(DPrime)), "cudaMalloc primes"))) return rc;
  if ((rc = cuda_check(cudaMalloc(&c->d_tw2, 4 * twb), "cudaMalloc twiddles"))) return rc;
  c->d_itw2 = c->d_tw2 + (size_t)LK * N * 2;
  if ((rc = cuda_check(cudaMalloc(&c->d_tables, tab.size() * sizeof(u64)), "cudaMalloc tables"))) return rc;
  cudaMemcpy(c->d_primes, c->h_primes.data(), LK * sizeof(DPrime), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_tw2, tw2.data(), 2 * twb, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_itw2, itw2.data(), 2 * twb, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_tables, tab.data(), tab.size() * sizeof(u64), cudaMemcpyHostToDevice);
  auto mk = [&](const Pending& p) {
    ConvTab t;
    t.ns = p.ns;
    t.nt = p.nt;
    t.c = c->d_tables + p.c;
    t.c_sh = c->d_tables + p.c_sh;
    return t;
  };
  for (auto& p : modup_p) c->modup_tabs.push_back(mk(p));
  c->moddown.conv = mk(md);
  c->moddown.pinv = c->d_tables + pinv_off;
  c->moddown.pinv_sh = c->d_tables + pinvsh_off;
  c->moddown.pmod = c->d_tables + pmod_off;
  c->moddown.pmod_sh = c->d_tables + pmodsh_off;
  c->rescale_tabs.assign(L + 1, RescaleTab{});
  for (uint32_t lvl = 2; lvl <= L; lvl++) {
    RescaleTab& R = c->rescale_tabs[lvl];
    R.inv = c->d_tables + rs_off[lvl];
    R.inv_sh = R.inv + (lvl - 1);
    R.hmod = R.inv_sh + (lvl - 1);
    R.qlast = m[lvl - 1];
    R.h = m[lvl - 1] / 2;
  }
  // Inverse-NTT last-stage constants with a conversion factor folded in:
  //   ModDown: factor Phat_j^-1 mod p_j on special prime j;
  //   ModUp at level lvl: factor Qhat_i^-1 mod q_i for data prime i of its (live) digit.
  auto fold = [&](uint32_t pi, u64 f) {
    const DPrime& P = c->h_primes[pi];
    const u64 q = P.q;
    InvScale s;
    s.ninv = h_mulmod(f % q, P.ninv, q);
    s.ninv_sh = h_shoup(s.ninv, q);
    s.iw1 = h_mulmod(f % q, P.iw1, q);
    s.iw1_sh = h_shoup(s.iw1, q);
    return s;
  };
  std::vector<InvScale> mds(LK), mu((size_t)L * LK);
  for (uint32_t pi = 0; pi < LK; pi++) mds[pi] = fold(pi, 1);
  for (uint32_t j = 0; j < K; j++) {
    const u64 pj = m[L + j];
    u64 prod = 1;
    for (uint32_t o = 0; o < K; o++)
      if (o != j) prod = h_mulmod(prod, m[L + o] % pj, pj);
    mds[L + j] = fold(L + j, h_invmod(prod, pj));
  }
  for (uint32_t lvl = 1; lvl <= L; lvl++) {
    InvScale* row = &mu[(size_t)(lvl - 1) * LK];
    for (uint32_t pi = 0; pi < LK; pi++) row[pi] = fold(pi, 1);
    for (uint32_t i = 0; i < lvl; i++) {
      const uint32_t d0 = (i / c->alpha) * c->alpha, d1 = std::min(d0 + c->alpha, lvl);
      u64 prod = 1;
      for (uint32_t o = d0; o < d1; o++)
        if (o != i) prod = h_mulmod(prod, m[o] % m[i], m[i]);
      row[i] = fold(i, h_invmod(prod, m[i]));
    }
  }
  if ((rc = cuda_check(cudaMalloc(&c->d_md_scale, (mds.size() + mu.size()) * sizeof(InvScale)), "cudaMalloc scale")))
    return rc;
  c->d_mu_scale = c->d_md_scale + mds.size();
  cudaMemcpy(c->d_md_scale, mds.data(), mds.size() * sizeof(InvScale), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_mu_scale, mu.data(), mu.size() * sizeof(InvScale), cudaMemcpyHostToDevice);
  return cuda_check(cudaGetLastError(), "table upload");
}

extern "C" int ctl_context_create(ctl_context** out, uint32_t N, const uint32_t* q_bits, uint32_t n_q,
                                  const uint32_t* p_bits, uint32_t n_p, uint32_t dnum, double scale, uint64_t seed) {
  if (!out || !q_bits || !p_bits) {
    set_error("ctl_context_create: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (N < 16 || N > 16384 || (N & (N - 1)) || n_q == 0 || n_p == 0 || n_p > 8 || dnum == 0 || dnum > n_q ||
      !(scale > 1.0)) {
    set_error("ctl_context_create: invalid parameters (N=%u n_q=%u n_p=%u dnum=%u)", N, n_q, n_p, dnum);
    return CTL_EINVAL;
  }
  std::unique_ptr<ctl_context> c(new ctl_context());
  c->N = N;
  while ((1u << c->logN) < N) c->logN++;
  c->L = n_q;
  c->K = n_p;
  c->alpha = (n_q + dnum - 1) / dnum;
  c->beta = (n_q + c->alpha - 1) / c->alpha;
  if (c->alpha > 8 || c->beta > 16) {
    set_error("ctl_context_create: digit shape alpha=%u beta=%u unsupported", c->alpha, c->beta);
    return CTL_ENOTSUP;
  }
  c->scale = scale;
  c->seed = seed;
  std::vector<uint32_t> bits(q_bits, q_bits + n_q);
  bits.insert(bits.end(), p_bits, p_bits + n_p);
  if (!plan_primes(N, bits, c->moduli)) {
    set_error("ctl_context_create: no prime chain for these bit sizes");
    return CTL_EINVAL;
  }
  int rc;
  if ((rc = cuda_check(cudaGetDevice(&c->device), "cudaGetDevice"))) return rc;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if ((rc = cuda_check(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream"))) return rc;
  c->own_stream = true;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  c->enc.init(N);
  if ((rc = build_tables(c.get()))) return rc;
  if ((rc = client_tables_create(c.get()))) return rc;
  if ((rc = ctl_autotune_ntt(c.get(), 0, nullptr, nullptr)) && rc != CTL_ENOMEM) return rc;
  *out = c.release();
  return CTL_OK;
}

extern "C" void ctl_context_destroy(ctl_context* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& pe : c->timing.pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (auto e : c->timing.pool) cudaEventDestroy(e);
  if (!c->parent) {  // clones share the parent's tables
    client_tables_destroy(c);
    cudaFree(c->d_primes);
    cudaFree(c->d_tw2);
    cudaFree(c->d_tables);
    cudaFree(c->d_md_scale);
  }
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

// A context with the same parameters and device tables as `c` and its own stream, so
// that work for one parameter set can run on several streams at once.  Keys and models
// made with `c` may be used with the clone.  Destroy clones before `c`.
extern "C" int ctl_context_clone(const ctl_context* c, ctl_context** out) {
  if (!c || !out) {
    set_error("ctl_context_clone: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<ctl_context> k(new ctl_context());
  k->N = c->N;
  k->logN = c->logN;
  k->L = c->L;
  k->K = c->K;
  k->alpha = c->alpha;
  k->beta = c->beta;
  k->scale = c->scale;
  k->seed = c->seed;
  k->moduli = c->moduli;
  k->device = c->device;
  k->sm_count = c->sm_count;
  k->alloc_fn = c->alloc_fn;
  k->free_fn = c->free_fn;
  k->alloc_user = c->alloc_user;
  k->d_primes = c->d_primes;
  k->d_tw2 = c->d_tw2;
  k->d_itw2 = c->d_itw2;
  k->d_tables = c->d_tables;
  k->modup_tabs = c->modup_tabs;
  k->rescale_tabs = c->rescale_tabs;
  k->moddown = c->moddown;
  k->d_md_scale = c->d_md_scale;
  k->d_mu_scale = c->d_mu_scale;
  k->client = c->client;
  k->h_primes = c->h_primes;
  k->enc = c->enc;
  k->dense_mode = c->dense_mode;
  k->ntt_shape_fwd = c->ntt_shape_fwd;
  k->ntt_shape_inv = c->ntt_shape_inv;
  k->bsgs_chunk = c->bsgs_chunk;
  k->bsgs_karatsuba = c->bsgs_karatsuba;
  k->ks_budget = c->ks_budget;
  k->windows = c->windows;
  k->parent = c->parent ? c->parent : c;
  if (int rc = cuda_check(cudaStreamCreateWithFlags(&k->stream, cudaStreamNonBlocking), "stream")) return rc;
  k->own_stream = true;
  *out = k.release();
  return CTL_OK;
}

extern "C" int ctl_context_info(const ctl_context* c, uint64_t* moduli, uint32_t* n_q, uint32_t* n_p,
                                uint32_t* alpha) {
  if (!c) {
    set_error("ctl_context_info: null context");
    return CTL_EINVAL;
  }
  if (moduli)
    for (size_t i = 0; i < c->moduli.size(); i++) moduli[i] = c->moduli[i];
  if (n_q) *n_q = c->L;
  if (n_p) *n_p = c->K;
  if (alpha) *alpha = c->alpha;
  return CTL_OK;
}

extern "C" int ctl_set_stream(ctl_context* c, void* stream) {
  if (!c) {
    set_error("ctl_set_stream: null context");
    return CTL_EINVAL;
  }
  if (stream) {
    // the caller's stream: the library stops owning one (its own is finished and
    // destroyed first, so earlier work stays ordered before later work)
    if (c->own_stream) {
      cudaStreamSynchronize(c->stream);
      cudaStreamDestroy(c->stream);
    }
    c->stream = (cudaStream_t)stream;
    c->own_stream = false;
  } else {
    cudaStream_t s;
    if (int rc = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream")) return rc;
    if (c->own_stream) cudaStreamDestroy(c->stream);
    c->stream = s;
    c->own_stream = true;
    return CTL_OK;
  }
  return CTL_OK;
}

extern "C" int ctl_set_allocator(ctl_context* c, ctl_alloc_fn a, ctl_free_fn f, void* user) {
  if (!c || (!a) != (!f)) {
    set_error("ctl_set_allocator: need both hooks or neither");
    return CTL_EINVAL;
  }
  c->alloc_fn = a;
  c->free_fn = f;
  c->alloc_user = user;
  return CTL_OK;
}

extern "C" int ctl_set_dense_mode(ctl_context* c, int mode) {
  if (!c || mode < CTL_DENSE_COMPOSED || mode > CTL_DENSE_RECT_LAZY) {
    set_error("ctl_set_dense_mode: invalid argument");
    return CTL_EINVAL;
  }
  c->dense_mode = mode;
  return CTL_OK;
}

extern "C" int ctl_set_ntt_shape(ctl_context* c, int fwd_shape, int inv_shape) {
  auto ok = [](int v) { return v == CTL_NTT_SHAPE_AUTO || v == CTL_NTT_SHAPE_R32 || v == CTL_NTT_SHAPE_R16; };
  if (!c || !ok(fwd_shape) || !ok(inv_shape)) {
    set_error("ctl_set_ntt_shape: invalid argument");
    return CTL_EINVAL;
  }
  if (fwd_shape != CTL_NTT_SHAPE_AUTO) c->ntt_shape_fwd = fwd_shape;
  if (inv_shape != CTL_NTT_SHAPE_AUTO) c->ntt_shape_inv = inv_shape;
  return CTL_OK;
}

extern "C" int ctl_set_bsgs_shape(ctl_context* c, int chunk, int karatsuba) {
  if (!c || (chunk != 16 && chunk != 32) || (karatsuba != 0 && karatsuba != 1)) {
    set_error("ctl_set_bsgs_shape: invalid argument");
    return CTL_EINVAL;
  }
  c->bsgs_chunk = chunk;
  c->bsgs_karatsuba = karatsuba;
  return CTL_OK;
}

extern "C" int ctl_set_windows(ctl_context* c, uint32_t p) {
  if (!c || p == 0 || p > c->N / 4) {
    set_error("ctl_set_windows: p must be in [1, N/4]");
    return CTL_EINVAL;
  }
  c->windows = p;
  return CTL_OK;
}

extern "C" int ctl_set_keyswitch_budget(ctl_context* c, uint64_t bytes) {
  if (!c || bytes == 0) {
    set_error("ctl_set_keyswitch_budget: invalid argument");
    return CTL_EINVAL;
  }
  c->ks_budget = bytes;
  return CTL_OK;
}

extern "C" int ctl_get_ntt_shape(const ctl_context* c, int* fwd_shape, int* inv_shape) {
  if (!c) {
    set_error("ctl_get_ntt_shape: null context");
    return CTL_EINVAL;
  }
  if (fwd_shape) *fwd_shape = c->ntt_shape_fwd;
  if (inv_shape) *inv_shape = c->ntt_shape_inv;
  return CTL_OK;
}

// Times plain forward and inverse transforms of both register shapes on zero-filled
// scratch limbs (a valid residue for every prime) and keeps the faster shape per
// direction.  The launches are not counted in the context's statistics.
extern "C" int ctl_autotune_ntt(ctl_context* c, uint32_t batch_limbs, int* fwd_shape, int* inv_shape) {
  if (!c) {
    set_error("ctl_autotune_ntt: null context");
    return CTL_EINVAL;
  }
  auto report = [&]() {
    if (fwd_shape) *fwd_shape = c->ntt_shape_fwd;
    if (inv_shape) *inv_shape = c->ntt_shape_inv;
    return CTL_OK;
  };
  if (c->logN < 12 || c->logN > 14) return report();  // one kernel shape only
  const uint32_t LK = c->L + c->K;
  if (batch_limbs == 0) batch_limbs = 8u * (uint32_t)c->sm_count;
  const int n_polys = (int)std::max<uint32_t>(1, batch_limbs / LK);
  DBuf buf(c, (size_t)n_polys * LK * c->N);
  if (!buf.p) {
    set_error("ctl_autotune_ntt: scratch allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemsetAsync(buf.p, 0, (size_t)n_polys * LK * c->N * sizeof(u64), c->stream);
  const uint64_t launches0 = c->launch_count.load();
  const bool timing0 = c->timing.enabled;
  c->timing.enabled = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_it = [&](bool inv, int shape) {
    (inv ? c->ntt_shape_inv : c->ntt_shape_fwd) = shape;
    auto run = [&]() {
      if (inv)
        launch_ntt_inv(c, buf.p, (size_t)LK * c->N, n_polys, 0, (int)LK, (int)c->L);
      else
        launch_ntt_fwd(c, buf.p, (size_t)LK * c->N, n_polys, 0, (int)LK, (int)c->L);
    };
    run();  // warm-up (and occupancy query)
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 3; r++) run();
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  for (int inv = 0; inv < 2; inv++) {
    const float t32 = time_it(inv, CTL_NTT_SHAPE_R32);
    const float t16 = time_it(inv, CTL_NTT_SHAPE_R16);
    (inv ? c->ntt_shape_inv : c->ntt_shape_fwd) = t16 < t32 ? CTL_NTT_SHAPE_R16 : CTL_NTT_SHAPE_R32;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing.enabled = timing0;
  c->launch_count = launches0;
  if (int rc = last_cuda("ctl_autotune_ntt")) return rc;
  return report();
}

extern "C" int ctl_synchronize(ctl_context* c) {
  if (!c) return CTL_EINVAL;
  return cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
}

extern "C" uint64_t ctl_galois_element(const ctl_context* c, int64_t r) {
  const int64_t n = c->N / 2;
  const int64_t rr = ((r % n) + n) % n;
  return h_powmod(5, (u64)rr, 2ull * c->N);
}

// =====================================================================================
// Keys
// =====================================================================================
namespace {

// Pointwise product of two plain NTT-form polys over all L+K primes (s * s).
__global__ void k_pointwise_sq(const u64* __restrict__ a, u64* __restrict__ o, const DPrime* __restrict__ pr,
                               int logN, size_t total) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const DPrime P = pr[idx >> logN];
    o[idx] = mulmod_plain(a[idx], a[idx], P.q, P.qinv, P.r2);
  }
}

int gen_key(ctl_context* c, ctl_keys* k, u64 seed, u64 key_id, const u64* sp_ntt) {
  const uint32_t N = c->N, L = c->L, LK = c->L + c->K, beta = c->beta;
  const size_t kw = (size_t)beta * 2 * LK * N;
  std::vector<u64> host(kw, 0);
  std::vector<i64> e((size_t)beta * N);
  for (uint32_t d = 0; d < beta; d++) {
    SplitMixStream se(seed, stream_id_key_e(key_id, d));
    draw_cbd21(se, N, &e[(size_t)d * N]);
    for (uint32_t i = 0; i < LK; i++) {
      SplitMixStream sa(seed, stream_id_key_a(key_id, d, i));
      draw_uniform(sa, c->moduli[i], N, &host[(((size_t)d * 2 + 1) * LK + i) * N]);
    }
  }
  DBuf key(c, kw), ed(c, (size_t)beta * N), e_res(c, (size_t)beta * LK * N), pmod(c, LK);
  if (!key.p || !ed.p || !e_res.p || !pmod.p) {
    set_error("keygen: device allocation failed");
    return CTL_ENOMEM;
  }
  std::vector<u64> pm(LK, 0);
  for (uint32_t i = 0; i < L; i++) {
    u64 P = 1;
    for (uint32_t j = 0; j < c->K; j++) P = h_mulmod(P, c->moduli[L + j] % c->moduli[i], c->moduli[i]);
    pm[i] = P;
  }
  cudaMemcpyAsync(key.p, host.data(), kw * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(ed.p, e.data(), e.size() * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(pmod.p, pm.data(), LK * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  // a -> NTT (poly 1 of every digit), e -> residues -> NTT
  launch_ntt_fwd(c, key.p + (size_t)LK * N, (size_t)2 * LK * N, (int)beta, 0, (int)LK, (int)L);
  launch_from_signed(c, (const i64*)ed.p, e_res.p, (int)beta, (int)LK, (int)L, N, (size_t)LK * N);
  launch_ntt_fwd(c, e_res.p, (size_t)LK * N, (int)beta, 0, (int)LK, (int)L);
  launch_keygen_combine(c, key.p, k->d_s, e_res.p, sp_ntt, (int)beta, (int)c->alpha, pmod.p);
  if (int rc = last_cuda("keygen")) return rc;
  // keep host vectors alive until the copies are done
  if (int rc = cuda_check(cudaStreamSynchronize(c->stream), "keygen sync")) return rc;
  k->evk[key_id] = key.release();
  k->key_bytes += kw * sizeof(u64);
  return CTL_OK;
}

}  // namespace

extern "C" int ctl_keygen(ctl_context* c, const int32_t* rot, uint32_t n_rot, uint64_t seed, ctl_keys** out) {
  if (!c || !out || (n_rot && !rot)) {
    set_error("ctl_keygen: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  const uint32_t N = c->N, LK = c->L + c->K;
  std::unique_ptr<ctl_keys> k(new ctl_keys());
  k->ctx = c;
  k->s.resize(N);
  SplitMixStream ss(seed, stream_id_secret());
  draw_ternary(ss, N, k->s.data());
  DBuf sraw(c, N), sq(c, (size_t)LK * N), sg(c, (size_t)LK * N);
  k->d_s = (u64*)dev_alloc(c, (size_t)LK * N * sizeof(u64));
  if (!sraw.p || !sq.p || !sg.p || !k->d_s) {
    set_error("keygen: device allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(sraw.p, k->s.data(), N * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  launch_from_signed(c, (const i64*)sraw.p, k->d_s, 1, (int)LK, (int)c->L, N, (size_t)LK * N);
  launch_ntt_fwd(c, k->d_s, (size_t)LK * N, 1, 0, (int)LK, (int)c->L);
  {
    size_t total = (size_t)LK * N;
    k_pointwise_sq<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(k->d_s, sq.p, c->d_primes, (int)c->logN,
                                                                           total);
    c->launch_count++;
  }
  int rc = gen_key(c, k.get(), seed, 0, sq.p);
  if (rc) return rc;
  for (uint32_t i = 0; i < n_rot; i++) {
    const u64 g = ctl_galois_element(c, rot[i]);
    if (g == 1 || k->evk.count(g)) continue;
    launch_automorph(c, k->d_s, sg.p, 1, (int)LK, (int)c->L, (size_t)LK * N, g);
    if ((rc = gen_key(c, k.get(), seed, g, sg.p))) {
      for (auto& kv : k->evk) dev_free(c, kv.second);
      return rc;
    }
  }
  if ((rc = cuda_check(cudaStreamSynchronize(c->stream), "keygen"))) return rc;
  *out = k.release();
  return CTL_OK;
}

extern "C" void ctl_keys_destroy(ctl_keys* k) {
  if (!k) return;
  ctl_context* c = k->ctx;
  cudaStreamSynchronize(c->stream);
  for (auto& kv : k->evk) dev_free(c, kv.second);
  dev_free(c, k->d_s);
  cudaStreamSynchronize(c->stream);
  delete k;
}

extern "C" int ctl_keys_create(ctl_context* c, ctl_keys** out) {
  if (!c || !out) {
    set_error("ctl_keys_create: null argument");
    return CTL_EINVAL;
  }
  ctl_keys* k = new (std::nothrow) ctl_keys();
  if (!k) {
    set_error("ctl_keys_create: allocation failed");
    return CTL_ENOMEM;
  }
  k->ctx = c;
  *out = k;
  return CTL_OK;
}

extern "C" int ctl_keys_import(ctl_keys* k, uint64_t key_id, const uint64_t* coeffs, size_t n_words) {
  if (!k || !coeffs) {
    set_error("ctl_keys_import: null argument");
    return CTL_EINVAL;
  }
  ctl_context* c = k->ctx;
  const uint32_t N = c->N, LK = c->L + c->K;
  const size_t kw = (size_t)c->beta * 2 * LK * N;
  if (n_words != kw) {
    set_error("ctl_keys_import: %zu words given, a key has %zu", n_words, kw);
    return CTL_EINVAL;
  }
  if (key_id != 0 && (!(key_id & 1) || key_id >= 2ull * N)) {
    set_error("ctl_keys_import: key id %llu is neither 0 nor an odd Galois element below 2N",
              (unsigned long long)key_id);
    return CTL_EINVAL;
  }
  for (size_t j = 0; j < (size_t)c->beta * 2; j++)
    for (uint32_t i = 0; i < LK; i++)
      for (uint32_t x = 0; x < N; x++)
        if (coeffs[(j * LK + i) * N + x] >= c->moduli[i]) {
          set_error("ctl_keys_import: residue out of range (limb %u)", i);
          return CTL_EINVAL;
        }
  DBuf key(c, kw);
  CHECK_ALLOC(key);
  cudaMemcpyAsync(key.p, coeffs, kw * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  launch_ntt_fwd(c, key.p, (size_t)LK * N, (int)(2 * c->beta), 0, (int)LK, (int)c->L);
  launch_to_mont(c, key.p, (int)(2 * c->beta), (int)LK, (int)c->L, (size_t)LK * N, true);
  if (int rc = cuda_check(cudaStreamSynchronize(c->stream), "key import")) return rc;
  auto it = k->evk.find(key_id);
  if (it != k->evk.end()) {
    dev_free(c, it->second);
    k->key_bytes -= kw * sizeof(u64);
  }
  k->evk[key_id] = key.release();
  k->key_bytes += kw * sizeof(u64);
  return CTL_OK;
}

extern "C" int ctl_keys_export(const ctl_keys* k, uint64_t key_id, uint64_t* out, size_t cap) {
  if (!k || !out) {
    set_error("ctl_keys_export: null argument");
    return CTL_EINVAL;
  }
  ctl_context* c = k->ctx;
  auto it = k->evk.find(key_id);
  if (it == k->evk.end()) {
    set_error("ctl_keys_export: no key %llu", (unsigned long long)key_id);
    return CTL_EKEY;
  }
  const uint32_t N = c->N, LK = c->L + c->K;
  const size_t kw = (size_t)c->beta * 2 * LK * N;
  if (cap < kw) {
    set_error("ctl_keys_export: capacity %zu < %zu", cap, kw);
    return CTL_EINVAL;
  }
  DBuf tmp(c, kw);
  CHECK_ALLOC(tmp);
  cudaMemcpyAsync(tmp.p, it->second, kw * sizeof(u64), cudaMemcpyDeviceToDevice, c->stream);
  launch_to_mont(c, tmp.p, (int)(2 * c->beta), (int)LK, (int)c->L, (size_t)LK * N, false);
  launch_ntt_inv(c, tmp.p, (size_t)LK * N, (int)(2 * c->beta), 0, (int)LK, (int)c->L);
  cudaMemcpyAsync(out, tmp.p, kw * sizeof(u64), cudaMemcpyDeviceToHost, c->stream);
  return cuda_check(cudaStreamSynchronize(c->stream), "key export");
}

// =====================================================================================
// Encoding, encryption, decryption
// =====================================================================================
extern "C" int ctl_encode(ctl_context* c, const double* x, size_t n, double scale, int64_t* m) {
  if (!c || !m || (n && !x) || n > c->N / 2 || !(scale > 0)) {
    set_error("ctl_encode: invalid argument");
    return CTL_EINVAL;
  }
  if (!c->enc.encode(x, n, scale, (i64*)m)) {
    set_error("ctl_encode: coefficient overflow (scale too large)");
    return CTL_EINVAL;
  }
  return CTL_OK;
}

extern "C" int ctl_decode(ctl_context* c, const double* m, size_t n, double scale, double* y) {
  if (!c || !m || !y || n > c->N / 2) {
    set_error("ctl_decode: invalid argument");
    return CTL_EINVAL;
  }
  c->enc.decode(m, n, scale, y);
  return CTL_OK;
}

extern "C" int ctl_encrypt_coeffs(ctl_context* c, const ctl_keys* k, const int64_t* m, uint64_t seed, ctl_ct** out) {
  if (!c || !k || !m || !out) {
    set_error("ctl_encrypt_coeffs: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (!k->d_s) {
    set_error("ctl_encrypt_coeffs: this key set holds no secret key (imported evaluation keys)");
    return CTL_EKEY;
  }
  const uint32_t N = c->N, L = c->L;
  if (c->client) {  // the device sampler (client.cu): the same streams, drawn on the GPU
    DBuf md(c, N);
    CHECK_ALLOC(md);
    cudaMemcpyAsync(md.p, m, N * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
    return encrypt_coeffs_dev(c, k, (const i64*)md.p, 1, (const u64*)&seed, out);
  }
  std::vector<u64> a((size_t)L * N);
  for (uint32_t i = 0; i < L; i++) {
    SplitMixStream sa(seed, stream_id_enc_a(i));
    draw_uniform(sa, c->moduli[i], N, &a[(size_t)i * N]);
  }
  std::vector<i64> me(N);
  SplitMixStream se(seed, stream_id_enc_e());
  draw_cbd21(se, N, me.data());
  for (uint32_t j = 0; j < N; j++) {
    if (m[j] > (int64_t)4e18 || m[j] < -(int64_t)4e18) {
      set_error("ctl_encrypt_coeffs: coefficient out of range");
      return CTL_EINVAL;
    }
    me[j] += m[j];
  }
  ctl_ct* ct = new_ct(c, L, 1, c->scale);
  DBuf raw(c, N), mer(c, (size_t)L * N);
  if (!ct || !raw.p || !mer.p) {
    if (ct) ctl_ct_destroy(ct);
    set_error("ctl_encrypt: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(ct->d + (size_t)L * N, a.data(), a.size() * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(raw.p, me.data(), N * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  launch_ntt_fwd(c, ct->d + (size_t)L * N, (size_t)L * N, 1, 0, (int)L, (int)L);
  launch_from_signed(c, (const i64*)raw.p, mer.p, 1, (int)L, (int)L, N, (size_t)L * N);
  launch_ntt_fwd(c, mer.p, (size_t)L * N, 1, 0, (int)L, (int)L);
  launch_encrypt_combine(c, ct->d, k->d_s, mer.p, (int)L);
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "encrypt");
  if (rc) {
    ctl_ct_destroy(ct);
    return rc;
  }
  *out = ct;
  return CTL_OK;
}

extern "C" int ctl_encrypt(ctl_context* c, const ctl_keys* k, const double* x, size_t n, uint64_t seed, ctl_ct** out) {
  if (!c || !k || !out || (n && !x) || n > c->N / 2) {
    set_error("ctl_encrypt: invalid argument");
    return CTL_EINVAL;
  }
  std::vector<i64> m(c->N);
  if (!c->enc.encode(x, n, c->scale, m.data())) {
    set_error("ctl_encrypt: coefficient overflow");
    return CTL_EINVAL;
  }
  return ctl_encrypt_coeffs(c, k, (const int64_t*)m.data(), seed, out);
}

extern "C" int ctl_decrypt_coeffs(ctl_context* c, const ctl_keys* k, const ctl_ct* ct, double* m) {
  if (!c || !k || !ct || !m) {
    set_error("ctl_decrypt_coeffs: null argument");
    return CTL_EINVAL;
  }
  if (!k->d_s) {
    set_error("ctl_decrypt_coeffs: this key set holds no secret key (imported evaluation keys)");
    return CTL_EKEY;
  }
  const uint32_t N = c->N, lvl = ct->level;
  if (c->client) {  // the centred CRT on the device (client.cu); ct's first ciphertext
    DBuf md(c, (size_t)ct->count * N);
    CHECK_ALLOC(md);
    if (int rc = decrypt_coeffs_dev(c, k, ct, (double*)md.p)) return rc;
    cudaMemcpyAsync(m, md.p, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    return cuda_check(cudaStreamSynchronize(c->stream), "decrypt");
  }
  DBuf t(c, (size_t)lvl * N);
  CHECK_ALLOC(t);
  launch_decrypt_mul(c, ct->d, k->d_s, t.p, 1, (int)lvl);
  launch_ntt_inv(c, t.p, (size_t)lvl * N, 1, 0, (int)lvl, (int)lvl);
  std::vector<u64> h((size_t)lvl * N);
  cudaMemcpyAsync(h.data(), t.p, h.size() * sizeof(u64), cudaMemcpyDeviceToHost, c->stream);
  if (int rc = cuda_check(cudaStreamSynchronize(c->stream), "decrypt")) return rc;
  crt_centred_to_double(h.data(), N, lvl, c->moduli.data(), N, m);
  return CTL_OK;
}

extern "C" int ctl_decrypt(ctl_context* c, const ctl_keys* k, const ctl_ct* ct, double* y, size_t n) {
  if (!c || !k || !ct || !y || n > c->N / 2) {
    set_error("ctl_decrypt: invalid argument");
    return CTL_EINVAL;
  }
  std::vector<double> m(c->N);
  if (int rc = ctl_decrypt_coeffs(c, k, ct, m.data())) return rc;
  c->enc.decode(m.data(), n, ct->scale, y);
  return CTL_OK;
}

// =====================================================================================
// Ciphertext handles
// =====================================================================================
static int import_common(ctl_context* c, const uint64_t* src, bool dev, uint32_t count, uint32_t level, double scale,
                         ctl_ct** out) {
  if (!c || !src || !out || count == 0 || level == 0 || level > c->L || !(scale > 0)) {
    set_error("ctl_ct_import: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  ctl_ct* ct = new_ct(c, level, count, scale);
  if (!ct) {
    set_error("ctl_ct_import: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(ct->d, src, ct->bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  launch_ntt_fwd(c, ct->d, (size_t)level * c->N, (int)(2 * count), 0, (int)level, (int)level);
  if (int rc = last_cuda("import")) {
    ctl_ct_destroy(ct);
    return rc;
  }
  *out = ct;
  return CTL_OK;
}
extern "C" int ctl_ct_import(ctl_context* c, const uint64_t* coeffs, uint32_t count, uint32_t level, double scale,
                             ctl_ct** out) {
  return import_common(c, coeffs, false, count, level, scale, out);
}
extern "C" int ctl_ct_import_dev(ctl_context* c, const uint64_t* coeffs, uint32_t count, uint32_t level, double scale,
                                 ctl_ct** out) {
  return import_common(c, coeffs, true, count, level, scale, out);
}

static int export_common(const ctl_ct* ct, uint64_t* dst, size_t cap, bool dev) {
  if (!ct || !dst) {
    set_error("ctl_ct_export: null argument");
    return CTL_EINVAL;
  }
  ctl_context* c = ct->ctx;
  const size_t w = ct_words(c, ct->level, ct->count);
  if (cap < w) {
    set_error("ctl_ct_export: capacity %zu < %zu", cap, w);
    return CTL_EINVAL;
  }
  if (dev) {
    launch_ntt_inv_oop(c, ct->d, (size_t)ct->level * c->N, (u64*)dst, (size_t)ct->level * c->N, (int)(2 * ct->count),
                       0, (int)ct->level, (int)ct->level);
    return last_cuda("export");
  }
  DBuf t(c, w);
  CHECK_ALLOC(t);
  launch_ntt_inv_oop(c, ct->d, (size_t)ct->level * c->N, t.p, (size_t)ct->level * c->N, (int)(2 * ct->count), 0,
                     (int)ct->level, (int)ct->level);
  cudaMemcpyAsync(dst, t.p, w * sizeof(u64), cudaMemcpyDeviceToHost, c->stream);
  return cuda_check(cudaStreamSynchronize(c->stream), "export");
}
extern "C" int ctl_ct_export(const ctl_ct* ct, uint64_t* coeffs, size_t cap) { return export_common(ct, coeffs, cap, false); }
extern "C" int ctl_ct_export_dev(const ctl_ct* ct, uint64_t* coeffs, size_t cap) {
  return export_common(ct, coeffs, cap, true);
}

extern "C" int ctl_ct_info(const ctl_ct* ct, uint32_t* level, uint32_t* count, double* scale) {
  if (!ct) {
    set_error("ctl_ct_info: null ciphertext");
    return CTL_EINVAL;
  }
  if (level) *level = ct->level;
  if (count) *count = ct->count;
  if (scale) *scale = ct->scale;
  return CTL_OK;
}

extern "C" int ctl_ct_concat(ctl_context* c, const ctl_ct* const* cts, size_t n, ctl_ct** out) {
  if (!c || !cts || !out || n == 0) {
    set_error("ctl_ct_concat: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  uint32_t total = 0;
  for (size_t i = 0; i < n; i++) {
    if (!cts[i] || cts[i]->level != cts[0]->level) {
      set_error("ctl_ct_concat: level mismatch");
      return CTL_ELEVEL;
    }
    if (!same_scale(cts[i]->scale, cts[0]->scale)) {
      set_error("ctl_ct_concat: scale mismatch");
      return CTL_ESCALE;
    }
    total += cts[i]->count;
  }
  ctl_ct* o = new_ct(c, cts[0]->level, total, cts[0]->scale);
  if (!o) {
    set_error("ctl_ct_concat: allocation failed");
    return CTL_ENOMEM;
  }
  size_t off = 0;
  for (size_t i = 0; i < n; i++) {
    cudaMemcpyAsync((char*)o->d + off, cts[i]->d, cts[i]->bytes, cudaMemcpyDeviceToDevice, c->stream);
    off += cts[i]->bytes;
  }
  *out = o;
  return last_cuda("concat");
}

extern "C" int ctl_ct_slice(const ctl_ct* b, uint32_t i, ctl_ct** out) {
  if (!b || !out || i >= b->count) {
    set_error("ctl_ct_slice: invalid argument");
    return CTL_EINVAL;
  }
  ctl_context* c = b->ctx;
  ctl_ct* o = new_ct(c, b->level, 1, b->scale);
  if (!o) {
    set_error("ctl_ct_slice: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(o->d, (const char*)b->d + (size_t)i * o->bytes, o->bytes, cudaMemcpyDeviceToDevice, c->stream);
  *out = o;
  return last_cuda("slice");
}

extern "C" void ctl_ct_destroy(ctl_ct* ct) {
  if (!ct) return;
  dev_free(ct->ctx, ct->d);
  delete ct;
}

// =====================================================================================
// Key switching core (hybrid: ModUp -> [sigma_g] -> key product -> ModDown)
// =====================================================================================
namespace {

// Key switch of the polys x_{r,b} (NTT form, level lvl; x_{r,b} = x + r*x_r + b*x_b with
// x_r either 0 (one input shared by all rotations: hoisting) or nb*x_b) with the key and
// Galois element of rotation r.  out [nr][nb][2][lvl][N].  The addend (nullable) is
// added through sigma_g as described at launch_moddown_ntt.
// With giant (the giant steps of a dense layer), the nr results are not formed: their
// sum is accumulated as the three partial sums of launch_giant_accum (giant->first: the
// first chunk), and launch_giant_moddown later adds it into the layer's output.
struct GiantSums {
  u64* D = nullptr;
  u64* C = nullptr;
  u64* A = nullptr;
  bool first = true;
};
int keyswitch(ctl_context* c, int nr, int nb, int lvl, const u64* x, size_t x_r, size_t x_b,
              const std::vector<const u64*>& keys, const std::vector<u64>& gs, const u64* addend, size_t add_r,
              size_t add_b, size_t add_p, bool add_both, u64* out, const GiantSums* giant = nullptr) {
  const uint32_t N = c->N;
  const int nd = (lvl + (int)c->alpha - 1) / (int)c->alpha;
  const int E = lvl + (int)c->K;
  const bool hoisted = (x_r == 0);
  const int n_in = hoisted ? nb : nr * nb;
  NvtxRange range(giant ? "keyswitch (giant steps)" : hoisted ? "keyswitch (hoisted)" : "keyswitch");
  if (nr > CTL_MAX_ROT) {
    set_error("keyswitch: at most %d rotations per launch", CTL_MAX_ROT);
    return CTL_EINVAL;
  }
  DBuf xc(c, (size_t)n_in * lvl * N), ext(c, (size_t)n_in * nd * E * N), acc(c, (size_t)nr * nb * 2 * E * N);
  if (!xc.p || !ext.p || !acc.p) {
    set_error("keyswitch: device allocation failed");
    return CTL_ENOMEM;
  }
  RotList rl;
  rl.n = nr;
  for (int r = 0; r < CTL_MAX_ROT; r++) {
    rl.key[r] = r < nr ? keys[r] : nullptr;
    rl.g[r] = r < nr ? gs[r] : 1;
  }
  // 1. coefficient form of the inputs
  // (the digit factors Qhat_i^-1 of the ModUp conversion are folded into this transform)
  launch_ntt_inv_oop(c, x, x_b, xc.p, (size_t)lvl * N, n_in, 0, lvl, lvl,
                     c->d_mu_scale + (size_t)(lvl - 1) * (c->L + c->K));
  // 2. ModUp + NTT of every digit
  launch_modup_ntt(c, xc.p, (size_t)lvl * N, x, x_b, n_in, lvl, ext.p);
  // 3. key inner products (automorphism folded into the gather)
  launch_key_ip(c, ext.p, hoisted ? 0 : (size_t)nb * nd * E * N, nb, lvl, rl, acc.p);
  // 4. ModDown: special limbs to coefficient form, then conversion + NTT + combine
  // (the factors Phat_j^-1 of the ModDown conversion are folded into this transform)
  launch_ntt_inv_oop(c, acc.p, (size_t)E * N, acc.p, (size_t)E * N, nr * nb * 2, lvl, E, lvl, c->d_md_scale);
  if (!giant) {
    launch_moddown_ntt(c, acc.p, nr, nb, lvl, out, addend, add_r, add_b, add_p, add_both, rl);
  } else {
    // sums of the nr ModDowns: data limbs and conversions summed over the rotations
    // (no transform per rotation); the addend (poly 0 only) is summed through sigma_g
    launch_giant_accum(c, acc.p, nr, nb, lvl, rl, addend, add_r, add_b, giant->D, giant->C, giant->A,
                       giant->first);
  }
  return last_cuda("keyswitch");
}

// Rotations of one ciphertext batch by several amounts (hoisted), chunked to bound memory.
int rotate_many(ctl_context* c, const ctl_keys* k, const u64* in, int nb, int lvl, const std::vector<int64_t>& rots,
                u64* out /*[nr][nb][2][lvl][N]*/) {
  const uint32_t N = c->N;
  const size_t ctw = (size_t)2 * lvl * N;
  std::vector<const u64*> keys;
  std::vector<u64> gs;
  std::vector<int> idx;
  for (size_t r = 0; r < rots.size(); r++) {
    const u64 g = ctl_galois_element(c, rots[r]);
    if (g == 1) {
      cudaMemcpyAsync(out + r * nb * ctw, in, nb * ctw * sizeof(u64), cudaMemcpyDeviceToDevice, c->stream);
      continue;
    }
    auto it = k->evk.find(g);
    if (it == k->evk.end()) {
      set_error("missing Galois key for rotation %lld", (long long)rots[r]);
      return CTL_EKEY;
    }
    keys.push_back(it->second);
    gs.push_back(g);
    idx.push_back((int)r);
  }
  if (keys.empty()) return last_cuda("rotate");
  // chunk so that the accumulators stay within the key-switching budget
  const int E = lvl + (int)c->K;
  const size_t acc_per_rot = (size_t)nb * 2 * E * N * sizeof(u64);
  int chunk = (int)std::max<size_t>(1, (size_t)c->ks_budget / std::max<size_t>(acc_per_rot, 1));
  chunk = std::min(chunk, CTL_MAX_ROT);
  for (size_t s = 0; s < keys.size();) {
    // consecutive output slots only (idx contiguous runs)
    size_t e = s + 1;
    while (e < keys.size() && (int)(e - s) < chunk && idx[e] == idx[e - 1] + 1) e++;
    std::vector<const u64*> kk(keys.begin() + s, keys.begin() + e);
    std::vector<u64> gg(gs.begin() + s, gs.begin() + e);
    int rc = keyswitch(c, (int)(e - s), nb, lvl, in + (size_t)lvl * N, 0, ctw, kk, gg, in, 0, ctw, 0, false,
                       out + (size_t)idx[s] * nb * ctw);
    if (rc) return rc;
    c->op_rot += (e - s) * nb;
    s = e;
  }
  return CTL_OK;
}

int rescale_into(ctl_context* c, const u64* in, int nb, int lvl, u64* out) {
  const uint32_t N = c->N;
  DBuf r(c, (size_t)nb * 2 * N);
  CHECK_ALLOC(r);
  launch_intt_rescale_last(c, in, (size_t)lvl * N, nb * 2, lvl, r.p);
  launch_rescale_ntt(c, r.p, in, (size_t)lvl * N, out, (size_t)(lvl - 1) * N, nb * 2, lvl);
  c->op_rescale += nb;
  return last_cuda("rescale");
}

}  // namespace

// =====================================================================================
// Homomorphic operations
// =====================================================================================
extern "C" int ctl_rotate(ctl_context* c, const ctl_keys* k, const ctl_ct* in, int32_t r, ctl_ct** out) {
  if (!c || !k || !in || !out) {
    set_error("ctl_rotate: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  ctl_ct* o = new_ct(c, in->level, in->count, in->scale);
  if (!o) {
    set_error("ctl_rotate: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = rotate_many(c, k, in->d, (int)in->count, (int)in->level, {r}, o->d);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

extern "C" int ctl_rescale(ctl_context* c, const ctl_ct* in, ctl_ct** out) {
  if (!c || !in || !out) {
    set_error("ctl_rescale: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (in->level < 2) {
    set_error("ctl_rescale: no level left");
    return CTL_ELEVEL;
  }
  ctl_ct* o = new_ct(c, in->level - 1, in->count, in->scale / (double)c->moduli[in->level - 1]);
  if (!o) {
    set_error("ctl_rescale: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = rescale_into(c, in->d, (int)in->count, (int)in->level, o->d);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

namespace {
int square_into(ctl_context* c, const ctl_keys* k, const u64* in, int nb, int lvl, u64* out) {
  const uint32_t N = c->N;
  auto it = k->evk.find(0);
  if (it == k->evk.end()) {
    set_error("missing relinearisation key");
    return CTL_EKEY;
  }
  const size_t LN = (size_t)lvl * N;
  DBuf d(c, (size_t)nb * 3 * LN), r(c, (size_t)nb * 2 * LN);
  if (!d.p || !r.p) {
    set_error("square: allocation failed");
    return CTL_ENOMEM;
  }
  launch_tensor_square(c, in, d.p, nb, lvl);
  int rc = keyswitch(c, 1, nb, lvl, d.p + 2 * LN, 0, 3 * LN, {it->second}, {1}, d.p, 0, 3 * LN, LN, true, r.p);
  if (rc) return rc;
  c->op_relin += nb;
  return rescale_into(c, r.p, nb, lvl, out);
}
}  // namespace

extern "C" int ctl_eval_square(ctl_context* c, const ctl_keys* k, const ctl_ct* in, ctl_ct** out) {
  if (!c || !k || !in || !out) {
    set_error("ctl_eval_square: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (in->level < 2) {
    set_error("ctl_eval_square: no level left");
    return CTL_ELEVEL;
  }
  const double q = (double)c->moduli[in->level - 1];
  ctl_ct* o = new_ct(c, in->level - 1, in->count, in->scale * in->scale / q);
  if (!o) {
    set_error("ctl_eval_square: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = square_into(c, k, in->d, (int)in->count, (int)in->level, o->d);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

extern "C" int ctl_add(ctl_context* c, const ctl_ct* a, const ctl_ct* b, ctl_ct** out) {
  if (!c || !a || !b || !out) {
    set_error("ctl_add: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (a->level != b->level || a->count != b->count) {
    set_error("ctl_add: shape mismatch");
    return CTL_ELEVEL;
  }
  if (!same_scale(a->scale, b->scale)) {
    set_error("ctl_add: scale mismatch");
    return CTL_ESCALE;
  }
  ctl_ct* o = new_ct(c, a->level, a->count, a->scale);
  if (!o) {
    set_error("ctl_add: allocation failed");
    return CTL_ENOMEM;
  }
  const size_t LN = (size_t)a->level * c->N;
  launch_add(c, a->d, b->d, o->d, (int)(2 * a->count), (int)a->level, LN, LN, LN);
  c->op_add += a->count;
  *out = o;
  return last_cuda("add");
}

// =====================================================================================
// Dense layer (Eq. bsgs) with pre-encoded diagonals
// =====================================================================================
struct DenseLayer {
  uint32_t m = 0, n = 0, t = 0, t1 = 0, t2 = 0, lvl = 0;
  bool lazy = false;     // lazy-ModDown form (CTL_DENSE_LAZY_MODDOWN) instead of composed rotations
  // rectangular form (CTL_DENSE_RECT, t = tm < tn): t diagonals of length tn, then the fold
  // over the tn/t blocks after the rescale (fold 1), and the [y, y] layout at stride t (fold 2)
  bool rect = false;
  uint32_t tn = 0;
  int fold = 0;
  double pt_scale = 0, in_scale = 0, out_scale = 0;
  u64* diag = nullptr;   // [t][limbs][N] NTT + Montgomery form (split); limbs = lvl (+K if lazy)
  u64* wino = nullptr;   // [t2][limbs][N] diagonal pair terms of the Winograd inner sums
  u64* bias = nullptr;   // [lvl][N] NTT form (plain residues) or null
};

namespace {

uint32_t bsgs_t(uint32_t m, uint32_t n) {
  uint32_t t = 1;
  while (t < m || t < n) t <<= 1;
  return t;
}
// t = t1 * t2 with t1 = 2^ceil(log2(t)/2).  The lazy-ModDown form takes
// t1 = min(t, 2^ceil(log2(4t)/2)) instead: there a giant step (ModDown of c1, ModUp, key
// product) costs about four baby steps (a key product in the extended basis), and this
// split minimises (t1 - 1) + 4 (t2 - 1).
uint32_t bsgs_t1(uint32_t t, bool lazy) {
  uint32_t lg = 0;
  while ((1u << lg) < t) lg++;
  if (!lazy) return 1u << ((lg + 1) / 2);
  const uint32_t t1 = 1u << ((lg + 3) / 2);
  return t1 < t ? t1 : t;
}

// Upload integer coefficient plaintexts [cnt][N] as NTT-form residues over `limbs`
// limbs of level lvl (limbs = lvl + K: the extended basis, special primes last).
int upload_plaintexts(ctl_context* c, const i64* coeffs, uint32_t cnt, uint32_t lvl, uint32_t limbs, bool mont,
                      u64** out) {
  const uint32_t N = c->N;
  DBuf raw(c, (size_t)cnt * N);
  u64* d = (u64*)dev_alloc(c, (size_t)cnt * limbs * N * sizeof(u64));
  if (!raw.p || !d) {
    if (d) dev_free(c, d);
    set_error("plaintext upload: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(raw.p, coeffs, (size_t)cnt * N * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  launch_from_signed(c, (const i64*)raw.p, d, (int)cnt, (int)limbs, (int)lvl, N, (size_t)limbs * N);
  launch_ntt_fwd(c, d, (size_t)limbs * N, (int)cnt, 0, (int)limbs, (int)lvl);
  if (mont) launch_to_mont(c, d, (int)cnt, (int)limbs, (int)lvl, (size_t)limbs * N, true);
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "plaintext upload");
  if (rc) {
    dev_free(c, d);
    return rc;
  }
  *out = d;
  return CTL_OK;
}

// Upload plaintext residues [lvl][N] (coefficient form, limb i modulo q_i) as NTT-form
// residues: the plaintexts whose scale is too large for 64-bit coefficients.
int upload_residues(ctl_context* c, const u64* res, uint32_t lvl, u64** out) {
  u64* d = (u64*)dev_alloc(c, (size_t)lvl * c->N * sizeof(u64));
  if (!d) {
    set_error("plaintext upload: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(d, res, (size_t)lvl * c->N * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  launch_ntt_fwd(c, d, (size_t)lvl * c->N, 1, 0, (int)lvl, (int)lvl);
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "plaintext upload");
  if (rc) {
    dev_free(c, d);
    return rc;
  }
  *out = d;
  return CTL_OK;
}

// Diagonals of W for Eq. (bsgs): diag_i[r] = W[r][(r+i) mod t] (zero padded),
// diag'_i = rot_{-floor(i/t1)*t1}(diag_i), i.e. diag_i placed at slots [k*t1, k*t1 + t).
// With c->windows = p > 1 (Sec. 3.1 "Multiple Predictions") the pattern of slots [0, 2t)
// repeats in every window [2t w, 2t (w+1)), w < p.
int encode_diagonals(ctl_context* c, const double* W, uint32_t m, uint32_t n, uint32_t t1, double scale,
                     std::vector<i64>& pts) {
  const uint32_t t = bsgs_t(m, n), ns = c->N / 2;
  pts.assign((size_t)t * c->N, 0);
  std::vector<double> v(ns);
  for (uint32_t i = 0; i < t; i++) {
    std::fill(v.begin(), v.end(), 0.0);
    const uint32_t sh = (i / t1) * t1;
    for (uint32_t w = 0; w < c->windows; w++)
      for (uint32_t r = 0; r < t; r++) {
        const uint32_t col = (r + i) % t;
        v[2 * t * w + r + sh] = (r < m && col < n) ? W[(size_t)r * n + col] : 0.0;
      }
    if (!c->enc.encode(v.data(), ns, scale, &pts[(size_t)i * c->N])) {
      set_error("dense: diagonal encoding overflow");
      return CTL_EINVAL;
    }
  }
  return CTL_OK;
}

// Rectangular diagonals of W (m x n, tm = pow2 >= m below tn = pow2 >= n):
// rd_i[r] = W[r mod tm][(r + i) mod tn] for r < tn, i < tm, placed as rd'_i =
// rot_{-floor(i/t1) t1}(rd_i) with rd_i in slots [0, tn); pts [tm][N].
int encode_diagonals_rect(ctl_context* c, const double* W, uint32_t m, uint32_t n, uint32_t tm, uint32_t tn,
                          uint32_t t1, double scale, std::vector<i64>& pts) {
  const uint32_t ns = c->N / 2;
  pts.assign((size_t)tm * c->N, 0);
  std::vector<double> v(ns);
  for (uint32_t i = 0; i < tm; i++) {
    std::fill(v.begin(), v.end(), 0.0);
    const uint32_t sh = (i / t1) * t1;
    for (uint32_t r = 0; r < tn; r++) {
      const uint32_t row = r % tm, col = (r + i) % tn;
      v[r + sh] = (row < m && col < n) ? W[(size_t)row * n + col] : 0.0;
    }
    if (!c->enc.encode(v.data(), ns, scale, &pts[(size_t)i * c->N])) {
      set_error("dense: diagonal encoding overflow");
      return CTL_EINVAL;
    }
  }
  return CTL_OK;
}

// The rectangular form's shape: tm < tn, both powers of two, one window, 2 tn <= N/2.
struct RectSpec {
  uint32_t tn = 0;
  int fold = 0;
};

int dense_prepare(ctl_context* c, DenseLayer& D, const double* W, const double* bias, const int64_t* pts_in,
                  const int64_t* bias_in, uint32_t m, uint32_t n, uint32_t t_given, uint32_t lvl, double in_scale,
                  double pt_scale, const RectSpec* rs = nullptr) {
  D.m = m;
  D.n = n;
  D.t = pts_in ? t_given : (rs ? bsgs_t(m, 1) : bsgs_t(m, n));
  D.rect = rs != nullptr;
  if (rs) {
    D.tn = rs->tn;
    D.fold = rs->fold;
    if (c->windows != 1 || D.t >= D.tn || (D.tn & (D.tn - 1)) || 2 * D.tn > c->N / 2 || rs->fold < 0 ||
        rs->fold > 2) {
      set_error("dense (rectangular): needs tm < tn (powers of two), 2 tn <= N/2 and one window");
      return CTL_EINVAL;
    }
  }
  D.lazy = c->dense_mode == CTL_DENSE_LAZY_MODDOWN || c->dense_mode == CTL_DENSE_RECT_LAZY;
  D.t1 = bsgs_t1(D.t, D.lazy);
  D.t2 = D.t / D.t1;
  D.lvl = lvl;
  D.in_scale = in_scale;
  if (lvl < 2) {
    set_error("dense: needs two live primes");
    return CTL_ELEVEL;
  }
  if (2 * D.t * c->windows > c->N / 2 || D.t == 0 || (D.t & (D.t - 1))) {
    set_error("dense: t=%u does not fit N/2 slots with the [x, x] layout in %u windows", D.t, c->windows);
    return CTL_EINVAL;
  }
  const double ql = (double)c->moduli[lvl - 1];
  // diagonals at q_last * Delta / scale_in: the rescaled output carries Delta again
  D.pt_scale = pt_scale > 0 ? pt_scale : ql * (c->scale / in_scale);
  D.out_scale = pt_scale > 0 ? in_scale * pt_scale / ql : c->scale;
  std::vector<i64> enc;
  const i64* src = (const i64*)pts_in;
  if (!src) {
    if (int rc = D.rect ? encode_diagonals_rect(c, W, m, n, D.t, D.tn, D.t1, D.pt_scale, enc)
                        : encode_diagonals(c, W, m, n, D.t1, D.pt_scale, enc))
      return rc;
    src = enc.data();
  }
  const uint32_t limbs = D.lazy ? lvl + c->K : lvl;
  if (int rc = upload_plaintexts(c, src, D.t, lvl, limbs, true, &D.diag)) return rc;
  launch_split_limbs(c, D.diag, (int)D.t, (int)limbs, (int)lvl);
  {
    DBuf w(c, (size_t)D.t2 * limbs * c->N);
    if (!w.p) {
      set_error("dense: allocation failed (diagonal pair terms)");
      return CTL_ENOMEM;
    }
    launch_bsgs_wino_diag(c, D.diag, (size_t)limbs * c->N, w.p, (int)D.t1, (int)D.t2, (int)limbs, (int)lvl);
    D.wino = w.release();
  }
  if (bias_in) {
    if (int rc = upload_plaintexts(c, (const i64*)bias_in, 1, lvl, lvl, false, &D.bias)) return rc;
  } else if (bias) {
    // the bias joins the products before the rescale, at their scale in_scale * pt_scale
    // (far above 2^63): encoded straight to residues
    std::vector<double> v(c->N / 2, 0.0);
    for (uint32_t w = 0; w < c->windows; w++)
      for (uint32_t r = 0; r < m; r++) v[2 * D.t * w + r] = bias[r];
    std::vector<u64> res((size_t)lvl * c->N);
    if (!c->enc.encode_rns(v.data(), v.size(), in_scale * D.pt_scale, c->moduli.data(), lvl, res.data())) {
      set_error("dense: bias encoding overflow");
      return CTL_EINVAL;
    }
    if (int rc = upload_residues(c, res.data(), lvl, &D.bias)) return rc;
  }
  return CTL_OK;
}

void dense_release(ctl_context* c, DenseLayer& D) {
  dev_free(c, D.diag);
  dev_free(c, D.wino);
  dev_free(c, D.bias);
  D.diag = D.wino = D.bias = nullptr;
}

// Galois keys of the rotations r0, r0 + step, ... (n of them) as a RotList.
int rot_list(ctl_context* c, const ctl_keys* k, int64_t r0, int64_t step, int n, RotList& rl) {
  if (n > CTL_MAX_ROT) {
    set_error("at most %d rotations per launch", CTL_MAX_ROT);
    return CTL_EINVAL;
  }
  rl.n = n;
  for (int r = 0; r < CTL_MAX_ROT; r++) {
    rl.key[r] = nullptr;
    rl.g[r] = 1;
  }
  for (int r = 0; r < n; r++) {
    const int64_t amt = r0 + step * r;
    const u64 g = ctl_galois_element(c, amt);
    auto it = k->evk.find(g);
    if (it == k->evk.end()) {
      set_error("dense: missing Galois key for rotation %lld", (long long)amt);
      return CTL_EKEY;
    }
    rl.key[r] = it->second;
    rl.g[r] = g;
  }
  return CTL_OK;
}

// Dense layer by Eq. (bsgs), lazy-ModDown form, every ModDown postponed (E = lvl + K limbs):
//   baby[0] = P * in, baby[j] = (P * sigma_j(c0) + ip_j.0, ip_j.1)   (one shared ModUp of c1),
//   inner[k] = sum_j diag'_{k t1 + j} o baby[j]                        (all E limbs),
//   S = inner[0] + sum_{k >= 1} (sigma_{k t1}(inner[k].0) + ip'_k.0, ip'_k.1),
//       ip'_k = key product of ModDown(inner[k].1) for rot_{k t1},
//   out = rescale( ModDown(S) [+ bias] ),  batch nb.
int rect_fold(ctl_context* c, const ctl_keys* k, const DenseLayer& D, u64* S, int nb, int lv);

int dense_apply_lazy(ctl_context* c, const ctl_keys* k, const DenseLayer& D, const u64* in, int nb, u64* out) {
  const uint32_t N = c->N, lvl = D.lvl, t1 = D.t1, t2 = D.t2;
  const int E = (int)lvl + (int)c->K;
  const int nd = ((int)lvl + (int)c->alpha - 1) / (int)c->alpha;
  const size_t EN = (size_t)E * N, LN = (size_t)lvl * N, ctw = 2 * LN, xw = 2 * EN * nb;
  const InvScale* mu = c->d_mu_scale + (size_t)(lvl - 1) * (c->L + c->K);
  DBuf baby(c, xw * t1), inner(c, xw * t2);
  if (!baby.p || !inner.p) {
    set_error("dense: allocation failed (batch %d)", nb);
    return CTL_ENOMEM;
  }
  // baby steps in the extended basis
  launch_scale_to_ext(c, in, baby.p, nb, (int)lvl);
  if (t1 > 1) {
    DBuf xc(c, (size_t)nb * LN), ext(c, (size_t)nb * nd * EN);
    CHECK_ALLOC(xc);
    CHECK_ALLOC(ext);
    launch_ntt_inv_oop(c, in + LN, ctw, xc.p, LN, nb, 0, (int)lvl, (int)lvl, mu);
    launch_modup_ntt(c, xc.p, LN, in + LN, ctw, nb, (int)lvl, ext.p);
    for (uint32_t j0 = 1; j0 < t1; j0 += CTL_MAX_ROT) {
      const int n = (int)std::min<uint32_t>(t1 - j0, CTL_MAX_ROT);
      RotList rl;
      if (int rc = rot_list(c, k, j0, 1, n, rl)) return rc;
      // addend: P * c0 of each input, poly 0 of baby step 0 (stride 2 E N per input)
      launch_key_ip(c, ext.p, 0, nb, (int)lvl, rl, baby.p + (size_t)j0 * xw, baby.p, 2 * EN);
    }
    c->op_rot += (uint64_t)(t1 - 1) * nb;
  }
  // inner sums for all giant steps
  launch_bsgs_inner(c, baby.p, D.diag, EN, D.wino, inner.p, (int)t1, (int)t2, nb, E, (int)lvl);
  c->op_ptmul += (uint64_t)D.t * nb;
  c->op_add += (uint64_t)(D.t - 1) * nb;
  dev_free(c, baby.release());
  // giant steps accumulated into S = inner[0], chunked by rotations
  if (t2 > 1) {
    const size_t per = (size_t)nb * N * sizeof(u64) * (2 * (size_t)lvl + (size_t)nd * E);
    const int chunk = (int)std::min<size_t>(
        std::min<size_t>(CTL_MAX_ROT, t2 - 1), std::max<size_t>(1, (size_t)c->ks_budget / std::max<size_t>(per, 1)));
    DBuf x1(c, (size_t)chunk * nb * LN), xc(c, (size_t)chunk * nb * LN), ext(c, (size_t)chunk * nb * nd * EN);
    if (!x1.p || !xc.p || !ext.p) {
      set_error("dense: allocation failed (batch %d)", nb);
      return CTL_ENOMEM;
    }
    for (uint32_t k0 = 1; k0 < t2; k0 += chunk) {
      const int nr = (int)std::min<uint32_t>(t2 - k0, (uint32_t)chunk);
      RotList rl;
      if (int rc = rot_list(c, k, (int64_t)k0 * t1, t1, nr, rl)) return rc;
      u64* Ik = inner.p + (size_t)k0 * xw;
      // ModDown of the c1 parts (special limbs to coefficient form in place first)
      launch_ntt_inv_oop(c, Ik + EN, 2 * EN, Ik + EN, 2 * EN, nr * nb, (int)lvl, E, (int)lvl, c->d_md_scale);
      launch_moddown_polys(c, Ik + EN, 2 * EN, nr * nb, (int)lvl, x1.p, LN);
      // key products of the rotations, kept in the extended basis and summed into S
      launch_ntt_inv_oop(c, x1.p, LN, xc.p, LN, nr * nb, 0, (int)lvl, (int)lvl, mu);
      launch_modup_ntt(c, xc.p, LN, x1.p, LN, nr * nb, (int)lvl, ext.p);
      launch_key_ip_acc(c, ext.p, (size_t)nb * nd * EN, nb, (int)lvl, rl, Ik, xw, 2 * EN, inner.p, 2 * EN);
      c->op_rot += (uint64_t)nr * nb;
    }
  }
  // one ModDown of both polys of S, then bias and rescale
  DBuf acc(c, (size_t)nb * ctw);
  CHECK_ALLOC(acc);
  launch_ntt_inv_oop(c, inner.p, EN, inner.p, EN, 2 * nb, (int)lvl, E, (int)lvl, c->d_md_scale);
  launch_moddown_polys(c, inner.p, EN, 2 * nb, (int)lvl, acc.p, LN);
  if (D.bias) launch_add_plain(c, acc.p, D.bias, nb, (int)lvl, ctw);
  int rc = rescale_into(c, acc.p, nb, (int)lvl, out);
  if (rc || !D.rect || D.fold == 0) return rc;
  return rect_fold(c, k, D, out, nb, (int)lvl - 1);
}

// The fold of the rectangular form on the rescaled partial sums z' (level lv, batch nb,
// in place in S = z'):  S = S + rot_s(S) for s = tn/2, tn/4, ..., tm, leaving y in slots
// [0, tm); with fold 2 also S = S + rot_{-tm}(z'), the [y, y] layout at stride tm.  The
// first fold rotation and rot_{-tm}(z') rotate the same ciphertext and share one ModUp.
int rect_fold(ctl_context* c, const ctl_keys* k, const DenseLayer& D, u64* S, int nb, int lv) {
  const size_t LN = (size_t)lv * c->N, bw = (size_t)nb * 2 * LN;
  std::vector<int64_t> first = {(int64_t)(D.tn / 2)};
  if (D.fold == 2) first.push_back(-(int64_t)D.t);
  DBuf tmp(c, bw * first.size());
  CHECK_ALLOC(tmp);
  if (int rc = rotate_many(c, k, S, nb, lv, first, tmp.p)) return rc;
  launch_add(c, S, tmp.p, S, nb * 2, lv, LN, LN, LN);
  c->op_add += nb;
  for (uint32_t sh = D.tn / 4; sh >= D.t; sh /= 2) {
    if (int rc = rotate_many(c, k, S, nb, lv, {(int64_t)sh}, tmp.p)) return rc;
    launch_add(c, S, tmp.p, S, nb * 2, lv, LN, LN, LN);
    c->op_add += nb;
  }
  if (D.fold == 2) {
    launch_add(c, S, tmp.p + bw, S, nb * 2, lv, LN, LN, LN);
    c->op_add += nb;
  }
  return last_cuda("dense fold");
}

// Dense layer by Eq. (bsgs) as the composition of whole rotations, batch nb:
//   out = rescale( sum_k rot_{k t1}( sum_j diag'_{k t1 + j} o rot_j(in) ) [+ bias] ),
// the baby steps sharing one ModUp (hoisted), each rotation ending with its ModDown.
int dense_apply_composed(ctl_context* c, const ctl_keys* k, const DenseLayer& D, const u64* in, int nb, u64* out) {
  const uint32_t N = c->N, lvl = D.lvl, t1 = D.t1, t2 = D.t2;
  const size_t LN = (size_t)lvl * N, ctw = 2 * LN, bw = ctw * nb;
  DBuf baby(c, bw * t1), inner(c, bw * t2);
  if (!baby.p || !inner.p) {
    set_error("dense: allocation failed (batch %d)", nb);
    return CTL_ENOMEM;
  }
  // baby steps rot_j(in), j = 0..t1-1 (hoisted: one ModUp shared by all)
  std::vector<int64_t> rots;
  for (uint32_t j = 0; j < t1; j++) rots.push_back(j);
  if (int rc = rotate_many(c, k, in, nb, (int)lvl, rots, baby.p)) return rc;
  // inner sums for all giant steps
  launch_bsgs_inner(c, baby.p, D.diag, LN, D.wino, inner.p, (int)t1, (int)t2, nb, (int)lvl, (int)lvl);
  c->op_ptmul += (uint64_t)D.t * nb;
  c->op_add += (uint64_t)(D.t - 1) * nb;
  dev_free(c, baby.release());
  // giant steps: acc = inner[0] + sum_{k >= 1} rot_{k t1}(inner[k]), chunked, each rotation
  // with its own input; acc is the k = 0 slice of inner.  Each rotation is a whole key
  // switch (its own ModUp, key product and ModDown), but the sum of their ModDowns takes
  // one transform per output limb: the data limbs and the conversions of the rotations
  // are summed first (exact, the transform being linear), then transformed once.  The
  // rotations go in chunks whose key-switching temporaries stay within the budget.
  u64* acc = inner.p;
  if (t2 > 1) {
    const int E = (int)lvl + (int)c->K;
    const int nd = ((int)lvl + (int)c->alpha - 1) / (int)c->alpha;
    const size_t per = (size_t)nb * N * sizeof(u64) * ((size_t)2 * E + (size_t)nd * E + (size_t)lvl);
    const int chunk = (int)std::min<size_t>(
        std::min<size_t>(CTL_MAX_ROT, t2 - 1), std::max<size_t>(1, (size_t)c->ks_budget / std::max<size_t>(per, 1)));
    DBuf gD(c, bw), gC(c, bw), gA(c, bw / 2);
    if (!gD.p || !gC.p || !gA.p) {
      set_error("dense: allocation failed (giant-step sums, batch %d)", nb);
      return CTL_ENOMEM;
    }
    GiantSums gs_sums;
    gs_sums.D = gD.p;
    gs_sums.C = gC.p;
    gs_sums.A = gA.p;
    for (uint32_t k0 = 1; k0 < t2; k0 += chunk) {
      const int nr = (int)std::min<uint32_t>(t2 - k0, (uint32_t)chunk);
      RotList rl;
      if (int rc = rot_list(c, k, (int64_t)k0 * t1, t1, nr, rl)) return rc;
      std::vector<const u64*> keys(rl.key, rl.key + nr);
      std::vector<u64> gs(rl.g, rl.g + nr);
      const u64* src = inner.p + (size_t)k0 * bw;
      gs_sums.first = (k0 == 1);
      int rc = keyswitch(c, nr, nb, (int)lvl, src + LN, bw, ctw, keys, gs, src, bw, ctw, 0, false, acc, &gs_sums);
      if (rc) return rc;
      c->op_rot += (uint64_t)nr * nb;
    }
    launch_giant_moddown(c, gD.p, gC.p, gA.p, nb, (int)lvl, acc);
  }
  if (D.bias) launch_add_plain(c, acc, D.bias, nb, (int)lvl, ctw);
  int rc = rescale_into(c, acc, nb, (int)lvl, out);
  if (rc || !D.rect || D.fold == 0) return rc;
  return rect_fold(c, k, D, out, nb, (int)lvl - 1);
}

int dense_apply(ctl_context* c, const ctl_keys* k, const DenseLayer& D, const u64* in, int nb, u64* out) {
  return D.lazy ? dense_apply_lazy(c, k, D, in, nb, out) : dense_apply_composed(c, k, D, in, nb, out);
}

}  // namespace

static int dense_common(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const double* W, const double* bias,
                        const int64_t* pts, const int64_t* bias_c, uint32_t m, uint32_t n, uint32_t t, double pt_scale,
                        ctl_ct** out, const RectSpec* rs = nullptr) {
  if (!c || !k || !in || !out) {
    set_error("dense: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  DenseLayer D;
  int rc = dense_prepare(c, D, W, bias, pts, bias_c, m, n, t, in->level, in->scale, pt_scale, rs);
  if (rc) {
    dense_release(c, D);
    return rc;
  }
  ctl_ct* o = new_ct(c, in->level - 1, in->count, D.out_scale);
  if (!o) {
    dense_release(c, D);
    set_error("dense: allocation failed");
    return CTL_ENOMEM;
  }
  rc = dense_apply(c, k, D, in->d, (int)in->count, o->d);
  dense_release(c, D);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

extern "C" int ctl_eval_dense(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const double* W, uint32_t m,
                              uint32_t n, const double* bias, ctl_ct** out) {
  if (!W || m == 0 || n == 0) {
    set_error("ctl_eval_dense: invalid weights");
    return CTL_EINVAL;
  }
  // CTL_DENSE_RECT: the rectangular form (fold 1) when the padded output side is shorter
  const uint32_t tm = bsgs_t(m, 1), tn = bsgs_t(n, 1);
  if (c && (c->dense_mode == CTL_DENSE_RECT || c->dense_mode == CTL_DENSE_RECT_LAZY) && tm < tn && c->windows == 1) {
    RectSpec rs{tn, 1};
    return dense_common(c, k, in, W, bias, nullptr, nullptr, m, n, 0, 0.0, out, &rs);
  }
  return dense_common(c, k, in, W, bias, nullptr, nullptr, m, n, 0, 0.0, out);
}

extern "C" int ctl_eval_dense_rect(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const double* W, uint32_t m,
                                   uint32_t n, const double* bias, int fold, ctl_ct** out) {
  if (!W || m == 0 || n == 0) {
    set_error("ctl_eval_dense_rect: invalid weights");
    return CTL_EINVAL;
  }
  RectSpec rs{bsgs_t(n, 1), fold};
  return dense_common(c, k, in, W, bias, nullptr, nullptr, m, n, 0, 0.0, out, &rs);
}

extern "C" int ctl_eval_dense_rect_coeffs(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const int64_t* pts,
                                          uint32_t tm, uint32_t tn, const int64_t* bias, double pt_scale, int fold,
                                          ctl_ct** out) {
  if (!pts || tm == 0 || (tm & (tm - 1)) || !(pt_scale > 0)) {
    set_error("ctl_eval_dense_rect_coeffs: invalid plaintexts");
    return CTL_EINVAL;
  }
  RectSpec rs{tn, fold};
  return dense_common(c, k, in, nullptr, nullptr, pts, bias, tm, tn, tm, pt_scale, out, &rs);
}

extern "C" int ctl_eval_dense_coeffs(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const int64_t* pts,
                                     uint32_t t, const int64_t* bias, double pt_scale, ctl_ct** out) {
  if (!pts || t == 0 || !(pt_scale > 0)) {
    set_error("ctl_eval_dense_coeffs: invalid plaintexts");
    return CTL_EINVAL;
  }
  return dense_common(c, k, in, nullptr, nullptr, pts, bias, t, t, t, pt_scale, out);
}

extern "C" int ctl_replicate(ctl_context* c, const ctl_keys* k, const ctl_ct* in, uint32_t t, ctl_ct** out) {
  if (!c || !k || !in || !out) {
    set_error("ctl_replicate: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  ctl_ct* o = new_ct(c, in->level, in->count, in->scale);
  if (!o) {
    set_error("ctl_replicate: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = rotate_many(c, k, in->d, (int)in->count, (int)in->level, {-(int64_t)t}, o->d);
  if (!rc) {
    const size_t LN = (size_t)in->level * c->N;
    launch_add(c, o->d, in->d, o->d, (int)(2 * in->count), (int)in->level, LN, LN, LN);
    c->op_add += in->count;
    rc = last_cuda("replicate");
  }
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

extern "C" int ctl_mul_plain_coeffs(ctl_context* c, const ctl_ct* in, const int64_t* pt, double pt_scale,
                                    ctl_ct** out) {
  if (!c || !in || !pt || !out || !(pt_scale > 0)) {
    set_error("ctl_mul_plain_coeffs: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  u64* d = nullptr;
  int rc = upload_plaintexts(c, (const i64*)pt, 1, in->level, in->level, true, &d);
  if (rc) return rc;
  ctl_ct* o = new_ct(c, in->level, in->count, in->scale * pt_scale);
  if (!o) {
    dev_free(c, d);
    set_error("ctl_mul_plain_coeffs: allocation failed");
    return CTL_ENOMEM;
  }
  const size_t LN = (size_t)in->level * c->N;
  launch_mul_plain(c, in->d, d, o->d, (int)(2 * in->count), (int)in->level, LN, LN);
  c->op_ptmul += in->count;
  dev_free(c, d);
  *out = o;
  return last_cuda("mul_plain");
}

// =====================================================================================
// The other layers of the paper's frozen network (Sec. 3.1): the ciphertext product,
// constant products and sums, level drop, the degree-3 ReLU approximation, average
// pooling and the packed 1D convolution.
// =====================================================================================
namespace {
inline u64 h_from_signed(i64 v, u64 q) {
  const u64 a = (u64)(v < 0 ? -(v + 1) : v) % q;  // |v| or |v|-1 without overflow
  if (v >= 0) return a;
  const u64 m = (a + 1) % q;  // |v| mod q
  return m ? q - m : 0;
}

// Per-limb constants for launch_affine / launch_sum_scale over the first lvl primes.
int limb_consts(ctl_context* c, int lvl, bool has_m, i64 mul, i64 add, LimbConsts& K) {
  if (lvl > kMaxConstLimbs) {
    set_error("level %d above the %d limbs of constant-operand kernels", lvl, kMaxConstLimbs);
    return CTL_ENOTSUP;
  }
  for (int i = 0; i < kMaxConstLimbs; i++) K.m[i] = K.a[i] = 0;
  for (int i = 0; i < lvl; i++) {
    const u64 q = c->moduli[i];
    K.m[i] = has_m ? h_mont(h_from_signed(mul, q), q) : 0;
    K.a[i] = h_from_signed(add, q);
  }
  return CTL_OK;
}

// round(v), half away from zero, if it fits a 64-bit integer.
bool to_i64(double v, i64* out) {
  if (!(std::fabs(v) < 9.0e18)) return false;
  *out = (i64)std::llround(v);
  return true;
}

// HMult of two batches at level lvl: tensor, relinearisation, rescale.
int mul_into(ctl_context* c, const ctl_keys* k, const u64* a, const u64* b, int nb, int lvl, u64* out) {
  const uint32_t N = c->N;
  auto it = k->evk.find(0);
  if (it == k->evk.end()) {
    set_error("missing relinearisation key");
    return CTL_EKEY;
  }
  const size_t LN = (size_t)lvl * N;
  DBuf d(c, (size_t)nb * 3 * LN), r(c, (size_t)nb * 2 * LN);
  if (!d.p || !r.p) {
    set_error("mul: allocation failed");
    return CTL_ENOMEM;
  }
  launch_tensor2(c, a, b, d.p, nb, lvl);
  int rc = keyswitch(c, 1, nb, lvl, d.p + 2 * LN, 0, 3 * LN, {it->second}, {1}, d.p, 0, 3 * LN, LN, true, r.p);
  if (rc) return rc;
  c->op_relin += nb;
  return rescale_into(c, r.p, nb, lvl, out);
}

// Constants of the degree-3 polynomial at level lvl (q_a = q_{lvl-1}, q_b = q_{lvl-2}):
// S2 = S*S/q_a, Sw = S2*S/q_b, C3 = round(a3*q_a), C2 = round(a2*S),
// C1 = round(a1*((Sw*q_a)/S)), C0 = round(a0*Sw), rounding half away from zero.
int poly3_consts(ctl_context* c, int lvl, double S, const double* a, i64 C[4], double* Sw_out) {
  if (lvl < 3) {
    set_error("poly3: needs three live primes (depth 2)");
    return CTL_ELEVEL;
  }
  const double qa = (double)c->moduli[lvl - 1], qb = (double)c->moduli[lvl - 2];
  const double S2 = S * S / qa;
  const double Sw = S2 * S / qb;
  if (!to_i64(a[3] * qa, &C[3]) || !to_i64(a[2] * S, &C[2]) || !to_i64(a[1] * (Sw * qa / S), &C[1]) ||
      !to_i64(a[0] * Sw, &C[0])) {
    set_error("poly3: a coefficient does not fit a 64-bit constant at this scale");
    return CTL_EINVAL;
  }
  *Sw_out = Sw;
  return CTL_OK;
}

// a3 z^3 + a2 z^2 + a1 z + a0 at depth 2:
//   z2 = square(z); v = rescale(C3 z) + C2; w = HMult(z2, v); l = drop(rescale(C1 z));
//   out = w + l + C0 (level lvl-2, scale Sw).
int poly3_into(ctl_context* c, const ctl_keys* k, const u64* in, int nb, int lvl, double S, const double* a, u64* out,
               double* out_scale) {
  const uint32_t N = c->N;
  i64 C[4];
  double Sw;
  if (int rc = poly3_consts(c, lvl, S, a, C, &Sw)) return rc;
  LimbConsts K3, K2, K1, K0;
  if (int rc = limb_consts(c, lvl, true, C[3], 0, K3)) return rc;
  limb_consts(c, lvl, false, 0, C[2], K2);
  limb_consts(c, lvl, true, C[1], 0, K1);
  limb_consts(c, lvl, false, 0, C[0], K0);
  const size_t L0 = (size_t)lvl * N, L1 = (size_t)(lvl - 1) * N, L2 = (size_t)(lvl - 2) * N;
  DBuf z2(c, (size_t)nb * 2 * L1), t(c, (size_t)nb * 2 * L0), v(c, (size_t)nb * 2 * L1), w(c, (size_t)nb * 2 * L2);
  if (!z2.p || !t.p || !v.p || !w.p) {
    set_error("poly3: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = square_into(c, k, in, nb, lvl, z2.p);
  if (rc) return rc;
  launch_affine(c, in, L0, nullptr, 0, t.p, L0, K3, true, 2 * nb, lvl);
  if ((rc = rescale_into(c, t.p, nb, lvl, v.p))) return rc;
  launch_affine(c, v.p, L1, nullptr, 0, v.p, L1, K2, false, 2 * nb, lvl - 1);
  if ((rc = mul_into(c, k, z2.p, v.p, nb, lvl - 1, w.p))) return rc;
  launch_affine(c, in, L0, nullptr, 0, t.p, L0, K1, true, 2 * nb, lvl);
  if ((rc = rescale_into(c, t.p, nb, lvl, v.p))) return rc;  // l at level lvl-1, read on lvl-2 limbs
  launch_affine(c, w.p, L2, v.p, L1, out, L2, K0, false, 2 * nb, lvl - 2);
  c->op_ptmul += 2 * nb;
  c->op_add += 2 * nb;
  *out_scale = Sw;
  return last_cuda("poly3");
}

// Average pool of size f: (sum_{i<f} rot_{-i}(x)) * round(q_{lvl-1}/f), rescaled.
int avgpool_into(ctl_context* c, const ctl_keys* k, const u64* in, int nb, int lvl, uint32_t f, u64* out) {
  if (lvl < 2 || f == 0 || f > (uint32_t)c->N / 2) {
    set_error("avgpool: invalid size or no level left");
    return f == 0 || f > (uint32_t)c->N / 2 ? CTL_EINVAL : CTL_ELEVEL;
  }
  const size_t cw = ct_words(c, lvl, nb);
  i64 Cf;
  to_i64((double)c->moduli[lvl - 1] / (double)f, &Cf);
  LimbConsts K;
  if (int rc = limb_consts(c, lvl, true, Cf, 0, K)) return rc;
  DBuf rots(c, (size_t)(f > 1 ? f - 1 : 1) * cw), s(c, cw);
  if (!rots.p || !s.p) {
    set_error("avgpool: allocation failed");
    return CTL_ENOMEM;
  }
  std::vector<int64_t> r;
  for (uint32_t i = 1; i < f; i++) r.push_back(-(int64_t)i);
  if (!r.empty())
    if (int rc = rotate_many(c, k, in, nb, lvl, r, rots.p)) return rc;
  launch_sum_scale(c, in, rots.p, (int)f - 1, s.p, K, nb, lvl);
  c->op_add += (f - 1) * nb;
  c->op_ptmul += nb;
  return rescale_into(c, s.p, nb, lvl, out);
}
}  // namespace

// Packed single-input single-output 1D convolution layer (Sec. 3.1 "1D Convolutions").
struct ConvLayer {
  uint32_t f = 0, n = 0, t = 0, lvl = 0;
  double pt_scale = 0, in_scale = 0, out_scale = 0;
  u64* pts = nullptr;   // [f][lvl][N], NTT + Montgomery form
  u64* bias = nullptr;  // [lvl][N], NTT form, or null
};

namespace {
// Plaintexts of the convolution: pt_i has w[i] in the slots s < 2t with (s mod t) < n.
int conv_prepare(ctl_context* c, ConvLayer& V, const double* w, const double* bias, const int64_t* pts_in,
                 const int64_t* bias_in, uint32_t f, uint32_t n, uint32_t t, uint32_t lvl, double in_scale,
                 double pt_scale) {
  V.f = f;
  V.n = n;
  V.t = t;
  V.lvl = lvl;
  V.in_scale = in_scale;
  if (lvl < 2) {
    set_error("conv1d: needs two live primes");
    return CTL_ELEVEL;
  }
  if (f == 0 || f > (uint32_t)c->N / 2 || (!pts_in && (n == 0 || n > t || 2 * t * c->windows > c->N / 2))) {
    set_error("conv1d: invalid shape (f=%u n=%u t=%u)", f, n, t);
    return CTL_EINVAL;
  }
  const double ql = (double)c->moduli[lvl - 1];
  V.pt_scale = pt_scale > 0 ? pt_scale : ql * (c->scale / in_scale);
  V.out_scale = pt_scale > 0 ? in_scale * pt_scale / ql : c->scale;
  std::vector<i64> enc;
  const i64* src = (const i64*)pts_in;
  if (!src) {
    const uint32_t ns = c->N / 2;
    enc.assign((size_t)f * c->N, 0);
    std::vector<double> v(ns);
    for (uint32_t i = 0; i < f; i++) {
      for (uint32_t s = 0; s < ns; s++) v[s] = (s < 2 * t * c->windows && (s % t) < n) ? w[i] : 0.0;
      if (!c->enc.encode(v.data(), ns, V.pt_scale, &enc[(size_t)i * c->N])) {
        set_error("conv1d: plaintext encoding overflow");
        return CTL_EINVAL;
      }
    }
    src = enc.data();
  }
  if (int rc = upload_plaintexts(c, src, f, lvl, lvl, true, &V.pts)) return rc;
  if (bias_in) {
    if (int rc = upload_plaintexts(c, (const i64*)bias_in, 1, lvl, lvl, false, &V.bias)) return rc;
  } else if (bias) {
    // added before the rescale, at the products' scale in_scale * pt_scale: residues
    std::vector<double> v(c->N / 2, 0.0);
    for (uint32_t w = 0; w < c->windows; w++)
      for (uint32_t s = 0; s < n; s++) v[2 * t * w + s] = v[2 * t * w + t + s] = bias[s];
    std::vector<u64> res((size_t)lvl * c->N);
    if (!c->enc.encode_rns(v.data(), v.size(), in_scale * V.pt_scale, c->moduli.data(), lvl, res.data())) {
      set_error("conv1d: bias encoding overflow");
      return CTL_EINVAL;
    }
    if (int rc = upload_residues(c, res.data(), lvl, &V.bias)) return rc;
  }
  return CTL_OK;
}

void conv_release(ctl_context* c, ConvLayer& V) {
  dev_free(c, V.pts);
  dev_free(c, V.bias);
  V.pts = V.bias = nullptr;
}

// out = rescale(sum_{i<f} pt_i o rot_{i-h}(x) [+ bias]), h = (f-1)/2; the rotations share
// one ModUp (hoisted) and each is bit-identical to ctl_rotate.
int conv_apply(ctl_context* c, const ctl_keys* k, const ConvLayer& V, const u64* in, int nb, u64* out) {
  const int lvl = (int)V.lvl;
  const size_t cw = ct_words(c, lvl, nb);
  DBuf rots(c, (size_t)V.f * cw), acc(c, cw);
  if (!rots.p || !acc.p) {
    set_error("conv1d: allocation failed");
    return CTL_ENOMEM;
  }
  const int64_t h = ((int64_t)V.f - 1) / 2;
  std::vector<int64_t> r;
  for (uint32_t i = 0; i < V.f; i++) r.push_back((int64_t)i - h);
  if (int rc = rotate_many(c, k, in, nb, lvl, r, rots.p)) return rc;
  launch_pt_mac(c, rots.p, V.pts, (int)V.f, acc.p, nb, lvl);
  c->op_ptmul += (uint64_t)V.f * nb;
  c->op_add += (uint64_t)(V.f - 1) * nb;
  if (V.bias) launch_add_plain(c, acc.p, V.bias, nb, lvl, (size_t)2 * lvl * c->N);
  return rescale_into(c, acc.p, nb, lvl, out);
}
}  // namespace

extern "C" int ctl_eval_mul(ctl_context* c, const ctl_keys* k, const ctl_ct* a, const ctl_ct* b, ctl_ct** out) {
  if (!c || !k || !a || !b || !out) {
    set_error("ctl_eval_mul: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (a->level != b->level || a->count != b->count) {
    set_error("ctl_eval_mul: shape mismatch");
    return CTL_ELEVEL;
  }
  if (a->level < 2) {
    set_error("ctl_eval_mul: no level left");
    return CTL_ELEVEL;
  }
  ctl_ct* o = new_ct(c, a->level - 1, a->count, a->scale * b->scale / (double)c->moduli[a->level - 1]);
  if (!o) {
    set_error("ctl_eval_mul: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = mul_into(c, k, a->d, b->d, (int)a->count, (int)a->level, o->d);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

static int affine_common(ctl_context* c, const ctl_ct* in, bool has_m, int64_t mul, int64_t add, double out_scale,
                         ctl_ct** out) {
  if (!c || !in || !out) {
    set_error("constant operation: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  LimbConsts K;
  if (int rc = limb_consts(c, (int)in->level, has_m, mul, add, K)) return rc;
  ctl_ct* o = new_ct(c, in->level, in->count, out_scale);
  if (!o) {
    set_error("constant operation: allocation failed");
    return CTL_ENOMEM;
  }
  const size_t LN = (size_t)in->level * c->N;
  launch_affine(c, in->d, LN, nullptr, 0, o->d, LN, K, has_m, (int)(2 * in->count), (int)in->level);
  *out = o;
  return last_cuda("constant operation");
}

extern "C" int ctl_mul_const(ctl_context* c, const ctl_ct* in, int64_t cst, double c_scale, ctl_ct** out) {
  if (!(c_scale > 0)) {
    set_error("ctl_mul_const: invalid constant scale");
    return CTL_EINVAL;
  }
  if (!in) {
    set_error("ctl_mul_const: null argument");
    return CTL_EINVAL;
  }
  int rc = affine_common(c, in, true, cst, 0, in->scale * c_scale, out);
  if (!rc) c->op_ptmul += in->count;
  return rc;
}

extern "C" int ctl_add_const(ctl_context* c, const ctl_ct* in, int64_t cst, ctl_ct** out) {
  if (!in) {
    set_error("ctl_add_const: null argument");
    return CTL_EINVAL;
  }
  return affine_common(c, in, false, 0, cst, in->scale, out);
}

extern "C" int ctl_drop_level(ctl_context* c, const ctl_ct* in, uint32_t level, ctl_ct** out) {
  if (!c || !in || !out) {
    set_error("ctl_drop_level: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (level == 0 || level > in->level) {
    set_error("ctl_drop_level: level %u not in [1, %u]", level, in->level);
    return CTL_ELEVEL;
  }
  ctl_ct* o = new_ct(c, level, in->count, in->scale);
  if (!o) {
    set_error("ctl_drop_level: allocation failed");
    return CTL_ENOMEM;
  }
  const size_t N = c->N;
  cudaMemcpy2DAsync(o->d, (size_t)level * N * sizeof(u64), in->d, (size_t)in->level * N * sizeof(u64),
                    (size_t)level * N * sizeof(u64), (size_t)2 * in->count, cudaMemcpyDeviceToDevice, c->stream);
  *out = o;
  return last_cuda("drop_level");
}

extern "C" int ctl_eval_poly3(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const double* a, ctl_ct** out) {
  if (!c || !k || !in || !a || !out) {
    set_error("ctl_eval_poly3: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  i64 C[4];
  double Sw;
  if (int rc = poly3_consts(c, (int)in->level, in->scale, a, C, &Sw)) return rc;
  ctl_ct* o = new_ct(c, in->level - 2, in->count, Sw);
  if (!o) {
    set_error("ctl_eval_poly3: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = poly3_into(c, k, in->d, (int)in->count, (int)in->level, in->scale, a, o->d, &Sw);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

extern "C" int ctl_eval_avgpool(ctl_context* c, const ctl_keys* k, const ctl_ct* in, uint32_t f, ctl_ct** out) {
  if (!c || !k || !in || !out) {
    set_error("ctl_eval_avgpool: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (in->level < 2) {
    set_error("ctl_eval_avgpool: no level left");
    return CTL_ELEVEL;
  }
  ctl_ct* o = new_ct(c, in->level - 1, in->count, in->scale);
  if (!o) {
    set_error("ctl_eval_avgpool: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = avgpool_into(c, k, in->d, (int)in->count, (int)in->level, f, o->d);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

static int conv_common(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const double* w, const double* bias,
                       const int64_t* pts, const int64_t* bias_c, uint32_t f, uint32_t n, uint32_t t, double pt_scale,
                       ctl_ct** out) {
  if (!c || !k || !in || !out) {
    set_error("conv1d: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  ConvLayer V;
  int rc = conv_prepare(c, V, w, bias, pts, bias_c, f, n, t, in->level, in->scale, pt_scale);
  if (rc) {
    conv_release(c, V);
    return rc;
  }
  ctl_ct* o = new_ct(c, in->level - 1, in->count, V.out_scale);
  if (!o) {
    conv_release(c, V);
    set_error("conv1d: allocation failed");
    return CTL_ENOMEM;
  }
  rc = conv_apply(c, k, V, in->d, (int)in->count, o->d);
  conv_release(c, V);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

extern "C" int ctl_eval_conv1d(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const double* w, uint32_t f,
                               uint32_t n, uint32_t t, const double* bias, ctl_ct** out) {
  if (!w) {
    set_error("ctl_eval_conv1d: null filter");
    return CTL_EINVAL;
  }
  return conv_common(c, k, in, w, bias, nullptr, nullptr, f, n, t, 0.0, out);
}

extern "C" int ctl_eval_conv1d_coeffs(ctl_context* c, const ctl_keys* k, const ctl_ct* in, const int64_t* pts,
                                      uint32_t f, const int64_t* bias, double pt_scale, ctl_ct** out) {
  if (!pts || !(pt_scale > 0)) {
    set_error("ctl_eval_conv1d_coeffs: invalid plaintexts");
    return CTL_EINVAL;
  }
  return conv_common(c, k, in, nullptr, nullptr, pts, bias, f, 0, 0, pt_scale, out);
}

extern "C" int ctl_ntt_dev(ctl_context* c, const uint64_t* in, uint64_t* out, uint32_t n_polys, uint32_t limbs,
                           int inverse) {
  if (!c || !in || !out || limbs == 0 || limbs > c->L + c->K || n_polys == 0) {
    set_error("ctl_ntt_dev: invalid argument");
    return CTL_EINVAL;
  }
  const size_t stride = (size_t)limbs * c->N;
  // prime of limb l is l: the (lvl = L, L = L) limb map is the identity on the chain
  if (inverse) {
    launch_ntt_inv_oop(c, (const u64*)in, stride, (u64*)out, stride, (int)n_polys, 0, (int)limbs, (int)c->L);
  } else {
    if (in != out) cudaMemcpyAsync(out, in, n_polys * stride * sizeof(u64), cudaMemcpyDeviceToDevice, c->stream);
    launch_ntt_fwd(c, (u64*)out, stride, (int)n_polys, 0, (int)limbs, (int)c->L);
  }
  return last_cuda("ntt");
}

// =====================================================================================
// Models (the frozen server layers M_S)
// =====================================================================================
struct LayerPlan {
  int kind = 0;
  DenseLayer dense;
  ConvLayer conv;
  double poly[4] = {0, 0, 0, 0};  // poly3: a0..a3
  uint32_t pool_f = 0;            // avgpool: size f
  uint32_t rep_t = 0;
  bool skip = false;              // a replicate already done by the preceding rectangular fold
  uint32_t in_level = 0;
  double in_scale = 0, out_scale = 0;
};
// A captured forward: the whole layer sequence of a model for one (context, keys, batch
// size), reading a fixed staging input and writing a fixed staging output.
// Batches from this size on are captured as two concurrent halves (ctl_model_forward_graph).
static constexpr uint32_t kGraphSplitMin = 8;  // measured: a loss at 2, even at 4, gains from 8 on
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  ctl::u64* in_buf = nullptr;
  ctl::u64* out_buf = nullptr;
  ctl_context* twin = nullptr;  // clone whose stream runs the second half of a split batch
  uint32_t nb1 = 0;             // ciphertexts in the first half (all of them if not split)
  uint64_t kernels = 0;
  uint64_t ops[5] = {0, 0, 0, 0, 0};
};
struct ctl_model {
  ctl_context* ctx = nullptr;
  std::vector<LayerPlan> layers;
  uint32_t in_level = 0, out_level = 0;
  double in_scale = 0, out_scale = 0;
  std::vector<int32_t> rotations;
  uint64_t bytes = 0;
  std::mutex graph_mu;
  std::map<std::tuple<const ctl_context*, const ctl_keys*, uint32_t>, GraphEntry> graphs;
};

extern "C" int ctl_model_create(ctl_context* c, const ctl_layer* layers, uint32_t n_layers, uint32_t in_level,
                                double in_scale, ctl_model** out) {
  if (!c || !layers || !out || n_layers == 0 || in_level == 0 || in_level > c->L || !(in_scale > 0)) {
    set_error("ctl_model_create: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<ctl_model> M(new ctl_model());
  M->ctx = c;
  M->in_level = in_level;
  M->in_scale = in_scale;
  uint32_t lvl = in_level;
  double sc = in_scale;
  std::vector<int32_t> rots;
  auto fail = [&](int rc) {
    for (auto& L : M->layers) {
      dense_release(c, L.dense);
      conv_release(c, L.conv);
    }
    return rc;
  };
  std::vector<bool> skip(n_layers, false);
  for (uint32_t i = 0; i < n_layers; i++) {
    const ctl_layer& ly = layers[i];
    LayerPlan P;
    P.kind = ly.kind;
    P.in_level = lvl;
    P.in_scale = sc;
    if (skip[i]) {  // the replicate the preceding rectangular dense layer's fold produced
      P.skip = true;
      P.rep_t = ly.rep_t;
      P.out_scale = sc;
      M->layers.push_back(P);
      continue;
    }
    if (ly.kind == CTL_LAYER_DENSE) {
      if (ly.m == 0 || ly.n == 0 || (!ly.W && !ly.pt_coeffs)) {
        set_error("ctl_model_create: dense layer %u needs W or coefficients", i);
        return fail(CTL_EINVAL);
      }
      // CTL_DENSE_RECT: a layer whose padded output side tm is below its input side tn
      // takes the rectangular form; when the next layers are [square,] replicate(tm), the
      // fold also forms the [y, y] layout and that replicate is not run again
      const uint32_t tm = bsgs_t(ly.m, 1), tn = bsgs_t(ly.n, 1);
      RectSpec rs{tn, 1};
      // (injected coefficients are then the tm rectangular diagonals)
      const bool rect = (c->dense_mode == CTL_DENSE_RECT || c->dense_mode == CTL_DENSE_RECT_LAZY) && tm < tn &&
                        c->windows == 1;
      if (rect) {
        uint32_t j = i + 1;
        if (j < n_layers && layers[j].kind == CTL_LAYER_SQUARE) j++;
        if (j < n_layers && layers[j].kind == CTL_LAYER_REPLICATE && layers[j].rep_t == tm) {
          rs.fold = 2;
          skip[j] = true;
        }
      }
      const uint32_t t = rect ? tm : bsgs_t(ly.m, ly.n);
      if (int rc = dense_prepare(c, P.dense, ly.W, ly.bias, ly.pt_coeffs, nullptr, ly.m, ly.n, t, lvl, sc, 0.0,
                                 rect ? &rs : nullptr)) {
        M->layers.push_back(P);
        return fail(rc);
      }
      M->bytes += (uint64_t)(P.dense.t + P.dense.t2) * (P.dense.lazy ? lvl + c->K : lvl) * c->N * 8;
      for (uint32_t j = 1; j < P.dense.t1; j++) rots.push_back((int32_t)j);
      for (uint32_t k = 1; k < P.dense.t2; k++) rots.push_back((int32_t)(k * P.dense.t1));
      if (P.dense.rect) {
        for (uint32_t sh = P.dense.tn / 2; sh >= P.dense.t; sh /= 2) rots.push_back((int32_t)sh);
        if (P.dense.fold == 2) rots.push_back(-(int32_t)P.dense.t);
      }
      sc = P.dense.out_scale;
      lvl--;
    } else if (ly.kind == CTL_LAYER_SQUARE) {
      if (lvl < 2) {
        set_error("ctl_model_create: no level left for square layer %u", i);
        return fail(CTL_ELEVEL);
      }
      sc = sc * sc / (double)c->moduli[lvl - 1];
      lvl--;
    } else if (ly.kind == CTL_LAYER_REPLICATE) {
      if (ly.rep_t == 0 || 2 * ly.rep_t > c->N / 2) {
        set_error("ctl_model_create: invalid replicate shift");
        return fail(CTL_EINVAL);
      }
      P.rep_t = ly.rep_t;
      rots.push_back(-(int32_t)ly.rep_t);
    } else if (ly.kind == CTL_LAYER_CONV1D) {
      if (ly.m == 0 || (!ly.W && !ly.pt_coeffs)) {
        set_error("ctl_model_create: conv1d layer %u needs a filter or coefficients", i);
        return fail(CTL_EINVAL);
      }
      if (int rc = conv_prepare(c, P.conv, ly.W, ly.bias, ly.pt_coeffs, nullptr, ly.m, ly.n, ly.rep_t, lvl, sc,
                                0.0)) {
        M->layers.push_back(P);
        return fail(rc);
      }
      M->bytes += (uint64_t)P.conv.f * lvl * c->N * 8;
      const int32_t h = ((int32_t)ly.m - 1) / 2;
      for (int32_t j = 0; j < (int32_t)ly.m; j++)
        if (j != h) rots.push_back(j - h);
      sc = P.conv.out_scale;
      lvl--;
    } else if (ly.kind == CTL_LAYER_POLY3) {
      if (!ly.W) {
        set_error("ctl_model_create: poly3 layer %u needs its four coefficients in W", i);
        return fail(CTL_EINVAL);
      }
      i64 C[4];
      double Sw;
      if (int rc = poly3_consts(c, (int)lvl, sc, ly.W, C, &Sw)) return fail(rc);
      for (int j = 0; j < 4; j++) P.poly[j] = ly.W[j];
      sc = Sw;
      lvl -= 2;
    } else if (ly.kind == CTL_LAYER_AVGPOOL) {
      if (ly.m == 0 || ly.m > c->N / 2 || lvl < 2) {
        set_error("ctl_model_create: avgpool layer %u: invalid size or no level left", i);
        return fail(lvl < 2 ? CTL_ELEVEL : CTL_EINVAL);
      }
      P.pool_f = ly.m;
      for (uint32_t j = 1; j < ly.m; j++) rots.push_back(-(int32_t)j);
      lvl--;
    } else {
      set_error("ctl_model_create: unknown layer kind %d", ly.kind);
      return fail(CTL_EINVAL);
    }
    P.out_scale = sc;
    M->layers.push_back(P);
  }
  std::sort(rots.begin(), rots.end());
  rots.erase(std::unique(rots.begin(), rots.end()), rots.end());
  M->rotations = rots;
  M->out_level = lvl;
  M->out_scale = sc;
  *out = M.release();
  return CTL_OK;
}

extern "C" void ctl_model_destroy(ctl_model* M) {
  if (!M) return;
  for (auto& kv : M->graphs) {
    ctl_context* gc = const_cast<ctl_context*>(std::get<0>(kv.first));
    cudaStreamSynchronize(gc->stream);
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    dev_free(gc, kv.second.in_buf);
    dev_free(gc, kv.second.out_buf);
    cudaStreamSynchronize(gc->stream);
    if (kv.second.twin) ctl_context_destroy(kv.second.twin);
  }
  for (auto& L : M->layers) {
    dense_release(M->ctx, L.dense);
    conv_release(M->ctx, L.conv);
  }
  cudaStreamSynchronize(M->ctx->stream);
  delete M;
}

extern "C" int ctl_model_rotations(const ctl_model* M, int32_t* rot, uint32_t cap, uint32_t* n_rot) {
  if (!M || !n_rot) {
    set_error("ctl_model_rotations: null argument");
    return CTL_EINVAL;
  }
  *n_rot = (uint32_t)M->rotations.size();
  if (rot)
    for (uint32_t i = 0; i < cap && i < M->rotations.size(); i++) rot[i] = M->rotations[i];
  return CTL_OK;
}

extern "C" int ctl_model_info(const ctl_model* M, uint32_t* out_level, double* out_scale, uint64_t* bytes) {
  if (!M) {
    set_error("ctl_model_info: null model");
    return CTL_EINVAL;
  }
  if (out_level) *out_level = M->out_level;
  if (out_scale) *out_scale = M->out_scale;
  if (bytes) *bytes = M->bytes;
  return CTL_OK;
}

// Runs the layers of M on nb ciphertexts at `in` (level M->in_level), writing the
// output ciphertexts to `out` (level M->out_level).
static int model_run(ctl_context* c, const ctl_model* M, const ctl_keys* k, const u64* in, int nb, u64* out) {
  const uint32_t N = c->N;
  DBuf a(c, ct_words(c, M->in_level, nb)), b(c, ct_words(c, M->in_level, nb));
  if (!a.p || !b.p) {
    set_error("ctl_model_forward: allocation failed");
    return CTL_ENOMEM;
  }
  const u64* cur = in;
  u64* bufs[2] = {a.p, b.p};
  int w = 0;
  uint32_t lvl = M->in_level;
  static const char* kLayerName[] = {"?", "dense", "square", "replicate", "conv1d", "poly3", "avgpool"};
  for (const LayerPlan& P : M->layers) {
    if (P.skip) continue;
    u64* dst = bufs[w];
    int rc = CTL_OK;
    NvtxRange range(P.kind >= 1 && P.kind <= 6 ? kLayerName[P.kind] : kLayerName[0]);
    if (P.kind == CTL_LAYER_DENSE) {
      rc = dense_apply(c, k, P.dense, cur, nb, dst);
      lvl--;
    } else if (P.kind == CTL_LAYER_SQUARE) {
      rc = square_into(c, k, cur, nb, (int)lvl, dst);
      lvl--;
    } else if (P.kind == CTL_LAYER_CONV1D) {
      rc = conv_apply(c, k, P.conv, cur, nb, dst);
      lvl--;
    } else if (P.kind == CTL_LAYER_POLY3) {
      double sw;
      rc = poly3_into(c, k, cur, nb, (int)lvl, P.in_scale, P.poly, dst, &sw);
      lvl -= 2;
    } else if (P.kind == CTL_LAYER_AVGPOOL) {
      rc = avgpool_into(c, k, cur, nb, (int)lvl, P.pool_f, dst);
      lvl--;
    } else {
      rc = rotate_many(c, k, cur, nb, (int)lvl, {-(int64_t)P.rep_t}, dst);
      if (!rc) {
        const size_t LN = (size_t)lvl * N;
        launch_add(c, dst, cur, dst, nb * 2, (int)lvl, LN, LN, LN);
        c->op_add += nb;
      }
    }
    if (rc) return rc;
    cur = dst;
    w ^= 1;
  }
  cudaMemcpyAsync(out, cur, ct_words(c, lvl, nb) * sizeof(u64), cudaMemcpyDeviceToDevice, c->stream);
  return last_cuda("model forward");
}

static int forward_check(ctl_context* c, const ctl_model* M, const ctl_keys* k, const ctl_ct* in, ctl_ct** out) {
  if (!c || !M || !k || !in || !out) {
    set_error("ctl_model_forward: null argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (in->level != M->in_level) {
    set_error("ctl_model_forward: input level %u, model expects %u", in->level, M->in_level);
    return CTL_ELEVEL;
  }
  if (!same_scale(in->scale, M->in_scale)) {
    set_error("ctl_model_forward: input scale mismatch");
    return CTL_ESCALE;
  }
  if (c->N != M->ctx->N || c->moduli != M->ctx->moduli) {
    set_error("ctl_model_forward: context parameters differ from the model's");
    return CTL_EINVAL;
  }
  return CTL_OK;
}

extern "C" int ctl_model_forward(ctl_context* c, const ctl_model* M, const ctl_keys* k, const ctl_ct* in,
                                 ctl_ct** out) {
  if (int rc = forward_check(c, M, k, in, out)) return rc;
  ctl_ct* o = new_ct(c, M->out_level, in->count, M->out_scale);
  if (!o) {
    set_error("ctl_model_forward: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = model_run(c, M, k, in->d, (int)in->count, o->d);
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  *out = o;
  return CTL_OK;
}

// Same result as ctl_model_forward, replaying a CUDA graph of the whole forward that is
// captured on the first call for this (context, keys, batch size).
extern "C" int ctl_model_forward_graph(ctl_context* c, const ctl_model* M, const ctl_keys* k, const ctl_ct* in,
                                       ctl_ct** out) {
  if (int rc = forward_check(c, M, k, in, out)) return rc;
  if (c->alloc_fn) {
    set_error("ctl_model_forward_graph: graphs need the library's stream-ordered pool");
    return CTL_ENOTSUP;
  }
  ctl_model* Mm = const_cast<ctl_model*>(M);
  std::lock_guard<std::mutex> lk(Mm->graph_mu);
  const uint32_t nb = in->count;
  auto key = std::make_tuple((const ctl_context*)c, k, nb);
  auto it = Mm->graphs.find(key);
  if (it == Mm->graphs.end()) {
    GraphEntry G;
    G.in_buf = (u64*)dev_alloc(c, ct_words(c, M->in_level, nb) * sizeof(u64));
    G.out_buf = (u64*)dev_alloc(c, ct_words(c, M->out_level, nb) * sizeof(u64));
    if (!G.in_buf || !G.out_buf) {
      dev_free(c, G.in_buf);
      dev_free(c, G.out_buf);
      set_error("ctl_model_forward_graph: allocation failed");
      return CTL_ENOMEM;
    }
    cudaMemsetAsync(G.in_buf, 0, ct_words(c, M->in_level, nb) * sizeof(u64), c->stream);
    // A batch of kGraphSplitMin ciphertexts or more is captured as two halves on concurrent
    // branches, the second on a clone's stream: the ciphertexts are independent, so the
    // result is the same, and each launch's last wave overlaps the other half's work.
    G.nb1 = nb >= kGraphSplitMin ? nb / 2 : nb;
    const uint32_t nb2 = nb - G.nb1;
    u64* in2 = G.in_buf + ct_words(c, M->in_level, G.nb1);
    u64* out2 = G.out_buf + ct_words(c, M->out_level, G.nb1);
    auto release = [&]() {
      cudaStreamSynchronize(c->stream);
      if (G.twin) ctl_context_destroy(G.twin);
      dev_free(c, G.in_buf);
      dev_free(c, G.out_buf);
    };
    int rc = CTL_OK;
    if (nb2) {
      rc = ctl_context_clone(c, &G.twin);
      if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream), "graph staging");
    }
    // one eager run (per half) settles every launch configuration before capture
    if (!rc) rc = model_run(c, M, k, G.in_buf, (int)G.nb1, G.out_buf);
    if (!rc && nb2) rc = model_run(G.twin, M, k, in2, (int)nb2, out2);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream), "graph warm-up");
    if (!rc && nb2) rc = cuda_check(cudaStreamSynchronize(G.twin->stream), "graph warm-up");
    if (rc) {
      release();
      return rc;
    }
    const bool timing = c->timing.enabled;
    c->timing.enabled = false;
    const uint64_t l0 = c->launch_count.load(), t0 = nb2 ? G.twin->launch_count.load() : 0;
    const uint64_t o0[5] = {c->op_rot, c->op_ptmul, c->op_add, c->op_relin, c->op_rescale};
    ctl_context* tw = nb2 ? G.twin : c;  // the second half's counters (c's own when not split)
    const uint64_t p0[5] = {tw->op_rot, tw->op_ptmul, tw->op_add, tw->op_relin, tw->op_rescale};
    cudaGraph_t graph = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (nb2) {
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    }
    rc = cuda_check(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) {
      if (nb2) {
        cudaEventRecord(fork, c->stream);
        cudaStreamWaitEvent(G.twin->stream, fork, 0);
      }
      int rr = model_run(c, M, k, G.in_buf, (int)G.nb1, G.out_buf);
      if (nb2) {
        if (!rr) rr = model_run(G.twin, M, k, in2, (int)nb2, out2);
        cudaEventRecord(join, G.twin->stream);
        cudaStreamWaitEvent(c->stream, join, 0);
      }
      const int re = cuda_check(cudaStreamEndCapture(c->stream, &graph), "end capture");
      rc = rr ? rr : re;
    }
    if (!rc) rc = cuda_check(cudaGraphInstantiate(&G.exec, graph, 0), "graph instantiate");
    if (graph) cudaGraphDestroy(graph);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    c->timing.enabled = timing;
    G.kernels = c->launch_count.load() - l0;
    const uint64_t o1[5] = {c->op_rot, c->op_ptmul, c->op_add, c->op_relin, c->op_rescale};
    for (int i = 0; i < 5; i++) G.ops[i] = o1[i] - o0[i];
    if (nb2) {  // the second half's launches and operations, counted by its clone
      const uint64_t p1[5] = {tw->op_rot, tw->op_ptmul, tw->op_add, tw->op_relin, tw->op_rescale};
      for (int i = 0; i < 5; i++) G.ops[i] += p1[i] - p0[i];
      G.kernels += tw->launch_count.load() - t0;
    }
    c->launch_count = l0;
    c->op_rot = o0[0];
    c->op_ptmul = o0[1];
    c->op_add = o0[2];
    c->op_relin = o0[3];
    c->op_rescale = o0[4];
    if (rc) {
      cudaGetLastError();
      release();
      return rc;
    }
    it = Mm->graphs.emplace(key, G).first;
  }
  GraphEntry& G = it->second;
  ctl_ct* o = new_ct(c, M->out_level, nb, M->out_scale);
  if (!o) {
    set_error("ctl_model_forward_graph: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(G.in_buf, in->d, in->bytes, cudaMemcpyDeviceToDevice, c->stream);
  int rc = cuda_check(cudaGraphLaunch(G.exec, c->stream), "graph launch");
  cudaMemcpyAsync(o->d, G.out_buf, o->bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (!rc) rc = last_cuda("graph forward");
  if (rc) {
    ctl_ct_destroy(o);
    return rc;
  }
  c->launch_count += G.kernels;
  c->op_rot += G.ops[0];
  c->op_ptmul += G.ops[1];
  c->op_add += G.ops[2];
  c->op_relin += G.ops[3];
  c->op_rescale += G.ops[4];
  *out = o;
  return CTL_OK;
}

// =====================================================================================
// Several groups of ciphertexts (each with its own context, model and keys: mixed ring
// degrees, levels and layer shapes) as one CUDA graph
// =====================================================================================
struct ctl_multi {
  std::vector<ctl_context*> ctx;
  std::vector<const ctl_model*> model;
  std::vector<const ctl_keys*> keys;
  std::vector<uint32_t> count;
  std::vector<u64*> in_buf, out_buf;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
};

static void multi_release(ctl_multi* m) {
  if (!m) return;
  if (m->exec) {
    cudaStreamSynchronize(m->ctx[0]->stream);
    cudaGraphExecDestroy(m->exec);
  }
  for (size_t i = 0; i < m->ctx.size(); i++) {
    if (i < m->in_buf.size()) dev_free(m->ctx[i], m->in_buf[i]);
    if (i < m->out_buf.size()) dev_free(m->ctx[i], m->out_buf[i]);
    cudaStreamSynchronize(m->ctx[i]->stream);
  }
  delete m;
}

// Captures the n groups' forwards as branches of one graph: the first context's stream
// forks to every group's stream (an event), each group's layer sequence is captured on its
// own stream (stream-ordered temporaries become graph memory nodes), and the branches join
// back.  Groups on distinct streams (e.g. context clones) run concurrently when replayed.
extern "C" int ctl_multi_create(uint32_t n, ctl_context* const* ctxs, const ctl_model* const* models,
                                const ctl_keys* const* keys, const uint32_t* counts, ctl_multi** out) {
  if (!n || !ctxs || !models || !keys || !counts || !out) {
    set_error("ctl_multi_create: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<ctl_multi> m(new ctl_multi());
  for (uint32_t i = 0; i < n; i++) {
    ctl_context* c = ctxs[i];
    const ctl_model* M = models[i];
    if (!c || !M || !keys[i] || !counts[i] || c->alloc_fn || c->N != M->ctx->N || c->moduli != M->ctx->moduli ||
        c->device != ctxs[0]->device) {
      set_error("ctl_multi_create: group %u: null handle, zero count, a caller allocator, a model of other "
                "parameters or another device", i);
      return CTL_EINVAL;
    }
    m->ctx.push_back(c);
    m->model.push_back(M);
    m->keys.push_back(keys[i]);
    m->count.push_back(counts[i]);
  }
  for (uint32_t i = 0; i < n; i++) {
    ctl_context* c = ctxs[i];
    const ctl_model* M = models[i];
    u64* a = (u64*)dev_alloc(c, ct_words(c, M->in_level, counts[i]) * sizeof(u64));
    u64* b = (u64*)dev_alloc(c, ct_words(c, M->out_level, counts[i]) * sizeof(u64));
    m->in_buf.push_back(a);
    m->out_buf.push_back(b);
    if (!a || !b) {
      set_error("ctl_multi_create: allocation failed");
      multi_release(m.release());
      return CTL_ENOMEM;
    }
    cudaMemsetAsync(a, 0, ct_words(c, M->in_level, counts[i]) * sizeof(u64), c->stream);
    // one eager run per group settles every launch configuration before the capture
    int rc = model_run(c, M, keys[i], a, (int)counts[i], b);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream), "multi warm-up");
    if (rc) {
      multi_release(m.release());
      return rc;
    }
  }
  std::vector<bool> timing(n);
  std::vector<uint64_t> l0(n);
  std::vector<std::array<uint64_t, 5>> o0(n);
  for (uint32_t i = 0; i < n; i++) {
    ctl_context* c = ctxs[i];
    timing[i] = c->timing.enabled;
    c->timing.enabled = false;
    l0[i] = c->launch_count.load();
    o0[i] = {c->op_rot, c->op_ptmul, c->op_add, c->op_relin, c->op_rescale};
  }
  cudaStream_t s0 = ctxs[0]->stream;
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  for (auto& e : ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  cudaGraph_t graph = nullptr;
  int rc = cuda_check(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (!rc) {
    int rr = CTL_OK;
    cudaEventRecord(ev[n], s0);
    for (uint32_t i = 0; i < n && !rr; i++) {
      ctl_context* c = ctxs[i];
      if (c->stream != s0) cudaStreamWaitEvent(c->stream, ev[n], 0);
      rr = model_run(c, models[i], keys[i], m->in_buf[i], (int)counts[i], m->out_buf[i]);
      if (c->stream != s0) {
        cudaEventRecord(ev[i], c->stream);
        cudaStreamWaitEvent(s0, ev[i], 0);
      }
    }
    const int re = cuda_check(cudaStreamEndCapture(s0, &graph), "end capture");
    rc = rr ? rr : re;
  }
  if (!rc) rc = cuda_check(cudaGraphInstantiate(&m->exec, graph, 0), "graph instantiate");
  if (graph) cudaGraphDestroy(graph);
  for (auto& e : ev) cudaEventDestroy(e);
  for (uint32_t i = 0; i < n; i++) {
    ctl_context* c = ctxs[i];
    c->timing.enabled = timing[i];
    m->kernels += c->launch_count.load() - l0[i];
    c->launch_count = l0[i];
    c->op_rot = o0[i][0];
    c->op_ptmul = o0[i][1];
    c->op_add = o0[i][2];
    c->op_relin = o0[i][3];
    c->op_rescale = o0[i][4];
  }
  if (rc) {
    cudaGetLastError();
    multi_release(m.release());
    return rc;
  }
  *out = m.release();
  return CTL_OK;
}

// One graph launch for all groups: inputs copied into the staging buffers, the graph
// replayed on the first context's stream, outputs copied out; every group's context
// stream then waits for that work, so later calls on the outputs are ordered after it.
extern "C" int ctl_multi_forward(ctl_multi* m, const ctl_ct* const* in, ctl_ct** out) {
  if (!m || !in || !out) {
    set_error("ctl_multi_forward: null argument");
    return CTL_EINVAL;
  }
  const size_t n = m->ctx.size();
  for (size_t i = 0; i < n; i++) {
    out[i] = nullptr;
    const ctl_model* M = m->model[i];
    if (!in[i] || in[i]->count != m->count[i] || in[i]->level != M->in_level ||
        !same_scale(in[i]->scale, M->in_scale) || in[i]->ctx->N != m->ctx[i]->N) {
      set_error("ctl_multi_forward: input %zu does not match its group (count, level, scale or ring)", i);
      return CTL_EINVAL;
    }
  }
  cudaStream_t s0 = m->ctx[0]->stream;
  cudaEvent_t e;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  for (size_t i = 0; i < n; i++) {  // inputs made on the group's stream come first
    if (m->ctx[i]->stream != s0) {
      cudaEventRecord(e, m->ctx[i]->stream);
      cudaStreamWaitEvent(s0, e, 0);
    }
    cudaMemcpyAsync(m->in_buf[i], in[i]->d, in[i]->bytes, cudaMemcpyDeviceToDevice, s0);
  }
  int rc = cuda_check(cudaGraphLaunch(m->exec, s0), "graph launch");
  for (size_t i = 0; i < n && !rc; i++) {
    ctl_context* c = m->ctx[i];
    ctl_ct* o = new_ct(c, m->model[i]->out_level, m->count[i], m->model[i]->out_scale);
    if (!o) {
      set_error("ctl_multi_forward: allocation failed");
      rc = CTL_ENOMEM;
      break;
    }
    cudaMemcpyAsync(o->d, m->out_buf[i], o->bytes, cudaMemcpyDeviceToDevice, s0);
    out[i] = o;
  }
  cudaEventRecord(e, s0);
  for (size_t i = 0; i < n; i++)
    if (m->ctx[i]->stream != s0) cudaStreamWaitEvent(m->ctx[i]->stream, e, 0);
  cudaEventDestroy(e);
  if (!rc) rc = last_cuda("multi forward");
  if (rc) {
    for (size_t i = 0; i < n; i++) {
      if (out[i]) ctl_ct_destroy(out[i]);
      out[i] = nullptr;
    }
    return rc;
  }
  m->ctx[0]->launch_count += m->kernels;
  return CTL_OK;
}

extern "C" void ctl_multi_destroy(ctl_multi* m) { multi_release(m); }

// =====================================================================================
// Statistics
// =====================================================================================
extern "C" int ctl_stats_reset(ctl_context* c) {
  if (!c) return CTL_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (auto& pe : c->timing.pending) {
    c->timing.pool.push_back(pe.second.first);
    c->timing.pool.push_back(pe.second.second);
  }
  c->timing.pending.clear();
  for (int i = 0; i < KC_COUNT; i++) {
    c->timing.ms[i] = 0;
    c->timing.launches[i] = 0;
    c->timing.work[i] = 0;
    c->timing.bytes[i] = 0;
  }
  c->launch_count = 0;
  c->op_rot = c->op_ptmul = c->op_add = c->op_relin = c->op_rescale = 0;
  return CTL_OK;
}
extern "C" int ctl_stats_enable_timing(ctl_context* c, int enable) {
  if (!c) return CTL_EINVAL;
  c->timing.enabled = enable != 0;
  return CTL_OK;
}
extern "C" uint64_t ctl_stats_launches(const ctl_context* c) { return c ? c->launch_count.load() : 0; }
extern "C" int ctl_stats_ops(const ctl_context* c, uint64_t* o) {
  if (!c || !o) return CTL_EINVAL;
  o[0] = c->op_rot;
  o[1] = c->op_ptmul;
  o[2] = c->op_add;
  o[3] = c->op_relin;
  o[4] = c->op_rescale;
  return CTL_OK;
}
extern "C" int ctl_stats_kernel_classes(void) { return KC_COUNT; }
extern "C" const char* ctl_stats_class_name(int i) { return (i >= 0 && i < KC_COUNT) ? kKernelClassName[i] : ""; }
extern "C" int ctl_stats_kernels(ctl_context* c, double* ms, uint64_t* launches, double* work) {
  if (!c) return CTL_EINVAL;
  if (int rc = cuda_check(cudaStreamSynchronize(c->stream), "stats")) return rc;
  for (auto& pe : c->timing.pending) {
    float t = 0;
    cudaEventElapsedTime(&t, pe.second.first, pe.second.second);
    c->timing.ms[pe.first] += t;
    c->timing.pool.push_back(pe.second.first);
    c->timing.pool.push_back(pe.second.second);
  }
  c->timing.pending.clear();
  for (int i = 0; i < KC_COUNT; i++) {
    if (ms) ms[i] = c->timing.ms[i];
    if (launches) launches[i] = c->timing.launches[i];
    if (work) work[i] = c->timing.work[i];
  }
  return CTL_OK;
}

extern "C" int ctl_stats_kernel_bytes(const ctl_context* c, double* bytes) {
  if (!c || !bytes) return CTL_EINVAL;
  for (int i = 0; i < KC_COUNT; i++) bytes[i] = c->timing.bytes[i];
  return CTL_OK;
}
