// The client's side of CryptoTL's protocol (Fig. alg:cryptotl: HE.Enc before the query,
// HE.Dec after it) on the GPU, for batches of queries: SIMD encoding and decoding
// (Sec. 3.1 "SIMD Encoding") as FP64 FFTs in shared memory, the encryption randomness
// drawn on the device from the same counter-based streams as the host, and the centred
// CRT of decryption.
//
// Encoding.  Slot j lives at the root zeta^(e_j), zeta = exp(i pi / N), e_j = 5^j mod 2N.
// Every e_j is 1 mod 4, so with w_k = m_k + i m_(k+N/2) (k < N/2) and zeta^(N/2 e_j) = i,
//   m(zeta^(e_j)) = sum_(k < N/2) (w_k zeta^k) Omega^(p_j k),  Omega = zeta^4,  p_j = (e_j - 1) / 4,
// a length-N/2 DFT whose outputs p_j run over [0, N/2) once.  Encoding inverts it (the real
// m with m(zeta^(e_j)) = scale * z_j is unique), decoding applies it.  One CTA transforms one
// polynomial with all N/2 complex values in shared memory (N <= 16384: 128 KB).
//
// Sampling.  A stream (seed, id) yields words finalise(key + c * gamma), c = 1, 2, ... (the
// SplitMix64 generator the host and the oracle use).  Uniform residues take the words whose
// low bits (masked to the prime's bit length) fall below q, in order: a CTA scans a block
// of words at a time and places the accepted ones by a prefix count, which gives the same
// residues as the sequential draw.  Errors take one word per coefficient.
#include <cmath>
#include <vector>

#include "ctl_internal.h"
#include "modarith.cuh"

namespace ctl {

// Device tables of the client's transforms and CRT, one allocation per context (shared by
// its clones).
struct ClientTabs {
  double2* tw = nullptr;     // [N/4] Omega^k = exp(2 pi i k / (N/2))
  double2* twist = nullptr;  // [N/2] zeta^k = exp(pi i k / N)
  uint32_t* pos = nullptr;   // [N/2] p_j = (e_j - 1) / 4
  u64* garner = nullptr;     // [L][L] q_j^-1 mod q_i (j < i)
  u64* qwords = nullptr;     // [L+1][L+1]: words of Q_l = q_0 ... q_(l-1) at row l
  u64* halfwords = nullptr;  // [L+1][L+1]: words of floor(Q_l / 2)
  int err_off = 0;
  int* err = nullptr;        // error flags of the sampling and encoding kernels
  void* block = nullptr;
};

namespace {

constexpr u64 kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kMaxClientLogN = 14;

__device__ __forceinline__ u64 sm_finalise(u64 z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
__device__ __forceinline__ u64 stream_key(u64 seed, u64 id) { return sm_finalise(seed ^ sm_finalise(id + kGamma)); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Radix-2 decimation-in-time transform of the M = 2^logM values in shared memory, input in
// bit-reversed order, output in natural order: X_p = sum_k x_k Omega^(+-pk).
template <bool INV>
__device__ void fft_smem(double2* x, const double2* __restrict__ tw, int logM) {
  const int M = 1 << logM;
  for (int s = 1; s <= logM; s++) {
    const int half = 1 << (s - 1), stride = M >> s;
    for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
      const int k = b & (half - 1);
      const int i0 = ((b >> (s - 1)) << s) + k, i1 = i0 + half;
      double2 w = __ldg(tw + (size_t)k * stride);
      if (INV) w.y = -w.y;
      const double2 u = x[i0], v = cmul(x[i1], w);
      x[i0] = make_double2(u.x + v.x, u.y + v.y);
      x[i1] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ uint32_t brv(uint32_t x, int bits) { return __brev(x) >> (32 - bits); }

// m_k = round(scale * Re(w_k)), m_(k+M) = round(scale * Im(w_k)), w = zeta^-k y_k,
// y = (2/N) * inverse DFT of the slot values placed at p_j.
__global__ void k_encode(const double* __restrict__ z, size_t nz, size_t z_stride, double scale, i64* __restrict__ m,
                         const double2* __restrict__ tw, const double2* __restrict__ twist,
                         const uint32_t* __restrict__ pos, int logN, int* __restrict__ err) {
  extern __shared__ double2 x[];
  const int logM = logN - 1, M = 1 << logM, N = 1 << logN;
  const size_t b = blockIdx.x;
  for (int p = threadIdx.x; p < M; p += blockDim.x) x[p] = make_double2(0.0, 0.0);
  __syncthreads();
  for (size_t j = threadIdx.x; j < nz; j += blockDim.x) x[brv(__ldg(pos + j), logM)].x = z[b * z_stride + j];
  __syncthreads();
  fft_smem<true>(x, tw, logM);
  const double f = 2.0 / (double)N * scale;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double2 t = __ldg(twist + k);
    const double2 y = x[k];
    const double re = (y.x * t.x + y.y * t.y) * f, im = (y.y * t.x - y.x * t.y) * f;  // y * conj(zeta^k)
    if (!(fabs(re) < 4.0e18) || !(fabs(im) < 4.0e18)) {
      atomicExch(err, 1);
      m[b * N + k] = 0;
      m[b * N + k + M] = 0;
      continue;
    }
    m[b * N + k] = (i64)llround(re);
    m[b * N + k + M] = (i64)llround(im);
  }
}

// z_j = Re(DFT(y)[p_j]) / scale, y_k = (m_k + i m_(k+M)) zeta^k.
__global__ void k_decode(const double* __restrict__ m, size_t nz, size_t z_stride, double inv_scale,
                         double* __restrict__ z, const double2* __restrict__ tw, const double2* __restrict__ twist,
                         const uint32_t* __restrict__ pos, int logN) {
  extern __shared__ double2 x[];
  const int logM = logN - 1, M = 1 << logM, N = 1 << logN;
  const size_t b = blockIdx.x;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double2 w = make_double2(m[b * N + k], m[b * N + k + M]);
    x[brv(k, logM)] = cmul(w, __ldg(twist + k));
  }
  __syncthreads();
  fft_smem<false>(x, tw, logM);
  for (size_t j = threadIdx.x; j < nz; j += blockDim.x) z[b * z_stride + j] = x[__ldg(pos + j)].x * inv_scale;
}

// Uniform residues below q[l] from stream (seed_b, enc_a(l)): one CTA per (ciphertext b,
// limb l), blockDim a multiple of 32 (<= 1024).  Words are masked to the bit length of q
// and kept when below q, in stream order.  An iteration limit (never reached: every word
// is kept with probability above 1/2) ends the loop with an error flag.
__global__ void k_sample_uniform(const u64* __restrict__ seeds, const DPrime* __restrict__ pr, int L, int logN,
                                 u64* __restrict__ out, size_t ct_stride, int* __restrict__ err) {
  __shared__ uint32_t warp_cnt[32];
  const int b = blockIdx.x / L, l = blockIdx.x % L;
  const u64 q = pr[l].q;
  const int bits = 64 - __clzll((long long)q);
  const u64 mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
  const u64 key = stream_key(seeds[b], (4ull << 56) | (u64)l);
  const uint32_t N = 1u << logN;
  u64* o = out + (size_t)b * ct_stride + ((size_t)l << logN);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint32_t filled = 0;
  u64 base = 0;
  const int max_iter = 64 * (int)((N + blockDim.x - 1) / blockDim.x) + 64;
  for (int it = 0; it < max_iter && filled < N; it++) {
    const u64 w = sm_finalise(key + (base + threadIdx.x + 1) * kGamma) & mask;
    const bool acc = w < q;
    const uint32_t ball = __ballot_sync(0xffffffffu, acc);
    if (lane == 0) warp_cnt[warp] = __popc(ball);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int v = 0; v < nwarps; v++) {
      const uint32_t cv = warp_cnt[v];
      if (v < warp) before += cv;
      total += cv;
    }
    const uint32_t at = filled + before + __popc(ball & ((1u << lane) - 1));
    if (acc && at < N) o[at] = w;
    filled += total;
    base += blockDim.x;
    __syncthreads();  // warp_cnt is rewritten next iteration
  }
  if (threadIdx.x == 0 && filled < N) atomicExch(err, 2);
}

// m + e for the ciphertexts of a batch: e from stream (seed_b, enc_e), one word per
// coefficient (centred binomial, k = 21), added to the encoded coefficients m [count][N].
__global__ void k_add_cbd21(const u64* __restrict__ seeds, const i64* __restrict__ m, i64* __restrict__ me,
                            int logN, size_t total, int* __restrict__ err) {
  const u64 m21 = (1ull << 21) - 1;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx >> logN, k = idx & (((size_t)1 << logN) - 1);
    const u64 w = sm_finalise(stream_key(seeds[b], 5ull << 56) + (u64)(k + 1) * kGamma);
    const i64 e = (i64)__popcll(w & m21) - (i64)__popcll((w >> 21) & m21);
    const i64 v = m[idx];
    if (v > (i64)4000000000000000000ll || v < -(i64)4000000000000000000ll) {
      atomicExch(err, 1);
      me[idx] = 0;
    } else {
      me[idx] = v + e;
    }
  }
}

// c0 = (m + e) - a * s for a batch: ct [count][2][L][N] with c1 = a (NTT form), me [count][L][N].
__global__ void k_encrypt_batch(u64* __restrict__ ct, const u64* __restrict__ s, const u64* __restrict__ me,
                                const DPrime* __restrict__ pr, int logN, int L, size_t total) {
  const size_t LN = (size_t)L << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx / LN, r = idx % LN;
    const DPrime P = pr[r >> logN];
    const u64 a = ct[b * 2 * LN + LN + r];
    ct[b * 2 * LN + r] = submod(me[idx], mulmod_plain(a, s[r], P.q, P.qinv, P.r2), P.q);
  }
}

// Centred CRT of coefficient-form residues [count][lvl][N] to doubles [count][N] (Garner's
// mixed radix, then Horner over lvl + 1 64-bit words, the value above Q/2 taken negative).
__global__ void k_crt_centred(const u64* __restrict__ res, int lvl, int logN, size_t total,
                              const DPrime* __restrict__ pr, const u64* __restrict__ garner, int Lg,
                              const u64* __restrict__ Qw, const u64* __restrict__ Hw, double* __restrict__ out) {
  constexpr int kMaxW = 17;
  const int nw = lvl + 1;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx >> logN, k = idx & (((size_t)1 << logN) - 1);
    u64 v[kMaxW - 1];
    for (int i = 0; i < lvl; i++) {
      const DPrime P = pr[i];
      u64 x = res[(b * lvl + i) << logN | k];
      x = mulmod_mont(x, P.rmod, P.q, P.qinv);  // below q_i
      for (int j = 0; j < i; j++) {
        const u64 vj = mulmod_mont(v[j], P.rmod, P.q, P.qinv);
        x = mulmod_plain(submod(x, vj, P.q), garner[(size_t)i * Lg + j], P.q, P.qinv, P.r2);
      }
      v[i] = x;
    }
    u64 X[kMaxW];
    for (int w = 0; w < nw; w++) X[w] = 0;
    for (int i = lvl - 1; i >= 0; i--) {  // X = X * q_i + v_i
      const u64 qi = pr[i].q;
      u64 carry = v[i];
      for (int w = 0; w < nw; w++) {
        const u64 lo = X[w] * qi, hi = __umul64hi(X[w], qi);
        const u64 s = lo + carry;
        carry = hi + (s < lo ? 1 : 0);
        X[w] = s;
      }
    }
    int cmp = 0;
    for (int w = nw - 1; w >= 0 && cmp == 0; w--)
      if (X[w] != Hw[w]) cmp = X[w] > Hw[w] ? 1 : -1;
    const bool neg = cmp > 0;
    if (neg) {  // X = Q - X
      u64 borrow = 0;
      for (int w = 0; w < nw; w++) {
        const u64 a = Qw[w], bb = X[w];
        const u64 d = a - bb - borrow;
        borrow = (a < bb || (a == bb && borrow)) ? 1 : 0;
        X[w] = d;
      }
    }
    double r = 0;
    for (int w = nw - 1; w >= 0; w--) r = r * 18446744073709551616.0 + (double)X[w];
    out[idx] = neg ? -r : r;
  }
}

}  // namespace
}  // namespace ctl

namespace ctl {

int client_tables_create(ctl_context* c) {
  // the host paths cover other rings and chains longer than the CRT kernel's 16 primes
  if (c->logN > kMaxClientLogN || c->logN < 2 || c->L > 16) return CTL_OK;
  const uint32_t N = c->N, M = N / 2, L = c->L;
  std::vector<double2> tw(M / 2), twist(M);
  for (uint32_t k = 0; k < M / 2; k++) tw[k] = make_double2(c->enc.cs[2 * k], c->enc.sn[2 * k]);
  for (uint32_t k = 0; k < M; k++) twist[k] = make_double2(c->enc.zc[k], c->enc.zs[k]);
  std::vector<uint32_t> pos(M);
  for (uint32_t j = 0; j < M; j++) pos[j] = c->enc.slot_pos[j] / 2;
  std::vector<u64> garner((size_t)L * L, 0), qw((size_t)(L + 1) * (L + 1), 0), hw((size_t)(L + 1) * (L + 1), 0);
  for (uint32_t i = 0; i < L; i++)
    for (uint32_t j = 0; j < i; j++) garner[(size_t)i * L + j] = h_invmod(c->moduli[j] % c->moduli[i], c->moduli[i]);
  for (uint32_t l = 1; l <= L; l++) {
    u64* Q = &qw[(size_t)l * (L + 1)];
    Q[0] = 1;
    for (uint32_t i = 0; i < l; i++) {  // Q = Q * q_i
      unsigned __int128 carry = 0;
      for (uint32_t w = 0; w <= L; w++) {
        const unsigned __int128 t = (unsigned __int128)Q[w] * c->moduli[i] + carry;
        Q[w] = (u64)t;
        carry = t >> 64;
      }
    }
    u64* H = &hw[(size_t)l * (L + 1)];
    u64 cy = 0;
    for (uint32_t w = L + 1; w-- > 0;) {
      H[w] = (Q[w] >> 1) | (cy << 63);
      cy = Q[w] & 1;
    }
  }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_tw = 0, o_twist = o_tw + al(tw.size() * sizeof(double2));
  const size_t o_pos = o_twist + al(twist.size() * sizeof(double2));
  const size_t o_g = o_pos + al(pos.size() * sizeof(uint32_t));
  const size_t o_q = o_g + al(garner.size() * sizeof(u64) + 8);
  const size_t o_h = o_q + al(qw.size() * sizeof(u64));
  const size_t o_e = o_h + al(hw.size() * sizeof(u64));
  const size_t bytes = o_e + 256;
  char* blk = nullptr;
  if (cudaMalloc(&blk, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("client tables: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpy(blk + o_tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice);
  cudaMemcpy(blk + o_twist, twist.data(), twist.size() * sizeof(double2), cudaMemcpyHostToDevice);
  cudaMemcpy(blk + o_pos, pos.data(), pos.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(blk + o_g, garner.data(), garner.size() * sizeof(u64), cudaMemcpyHostToDevice);
  cudaMemcpy(blk + o_q, qw.data(), qw.size() * sizeof(u64), cudaMemcpyHostToDevice);
  cudaMemcpy(blk + o_h, hw.data(), hw.size() * sizeof(u64), cudaMemcpyHostToDevice);
  cudaMemset(blk + o_e, 0, 256);
  ClientTabs* T = new ClientTabs();
  T->block = blk;
  T->tw = (double2*)(blk + o_tw);
  T->twist = (double2*)(blk + o_twist);
  T->pos = (uint32_t*)(blk + o_pos);
  T->garner = (u64*)(blk + o_g);
  T->qwords = (u64*)(blk + o_q);
  T->halfwords = (u64*)(blk + o_h);
  T->err = (int*)(blk + o_e);
  c->client = T;
  return cuda_check(cudaGetLastError(), "client tables");
}

void client_tables_destroy(ctl_context* c) {
  if (!c->client) return;
  cudaFree(c->client->block);
  delete c->client;
  c->client = nullptr;
}

namespace {

int need_client(const ctl_context* c, const char* who) {
  if (!c->client) {
    set_error("%s: the GPU client transforms need 4 <= N <= 16384 and at most 16 data primes", who);
    return CTL_EINVAL;
  }
  return CTL_OK;
}

// Reads and clears the context's device error flags (synchronises the stream).
int client_errors(ctl_context* c, const char* who) {
  int flag = 0;
  cudaMemcpyAsync(&flag, c->client->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (int rc = cuda_check(cudaStreamSynchronize(c->stream), who)) return rc;
  if (flag) {
    cudaMemsetAsync(c->client->err, 0, sizeof(int), c->stream);
    set_error(flag == 1 ? "%s: coefficient out of range (scale too large)" : "%s: sampler ran out of words", who);
    return CTL_EINVAL;
  }
  return CTL_OK;
}

size_t fft_smem_bytes(const ctl_context* c) { return (size_t)(c->N / 2) * sizeof(double2); }

void launch_encode(ctl_context* c, const double* z, size_t nz, uint32_t count, double scale, i64* m) {
  const size_t sm = fft_smem_bytes(c);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  k_encode<<<count, 512, sm, c->stream>>>(z, nz, nz, scale, m, c->client->tw, c->client->twist, c->client->pos,
                                          (int)c->logN, c->client->err);
  c->launch_count++;
}

void launch_decode(ctl_context* c, const double* m, size_t nz, uint32_t count, double scale, double* z) {
  const size_t sm = fft_smem_bytes(c);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  k_decode<<<count, 512, sm, c->stream>>>(m, nz, nz, 1.0 / scale, z, c->client->tw, c->client->twist,
                                          c->client->pos, (int)c->logN);
  c->launch_count++;
}

int grid_of(const ctl_context* c, size_t total) {
  size_t g = (total + 255) / 256, cap = (size_t)c->sm_count * 16;
  return (int)(g < cap ? g : cap);
}

}  // namespace

// Encryption of count integer plaintexts m [count][N] (device) under the secret key:
// c1 = a (uniform, stream (seed_b, enc_a(limb))), c0 = m + e - a s (e centred binomial,
// stream (seed_b, enc_e)), at the top level; the same streams as the host and the oracle.
int encrypt_coeffs_dev(ctl_context* c, const ctl_keys* k, const i64* m_dev, uint32_t count, const u64* seeds,
                       ctl_ct** out) {
  const uint32_t N = c->N, L = c->L;
  const size_t LN = (size_t)L * N;
  ctl_ct* ct = new_ct(c, L, count, c->scale);
  DBuf sd(c, count), me(c, (size_t)count * N), mer(c, (size_t)count * LN);
  if (!ct || !sd.p || !me.p || !mer.p) {
    if (ct) ctl_ct_destroy(ct);
    set_error("ctl_encrypt: allocation failed");
    return CTL_ENOMEM;
  }
  cudaMemcpyAsync(sd.p, seeds, count * sizeof(u64), cudaMemcpyHostToDevice, c->stream);
  k_sample_uniform<<<count * L, 1024, 0, c->stream>>>(sd.p, c->d_primes, (int)L, (int)c->logN, ct->d + LN, 2 * LN,
                                                      c->client->err);
  const size_t tot = (size_t)count * N;
  k_add_cbd21<<<grid_of(c, tot), 256, 0, c->stream>>>(sd.p, m_dev, (i64*)me.p, (int)c->logN, tot, c->client->err);
  c->launch_count += 2;
  launch_ntt_fwd(c, ct->d + LN, 2 * LN, (int)count, 0, (int)L, (int)L);
  launch_from_signed(c, (const i64*)me.p, mer.p, (int)count, (int)L, (int)L, N, LN);
  launch_ntt_fwd(c, mer.p, LN, (int)count, 0, (int)L, (int)L);
  const size_t tl = (size_t)count * LN;
  k_encrypt_batch<<<grid_of(c, tl), 256, 0, c->stream>>>(ct->d, k->d_s, mer.p, c->d_primes, (int)c->logN, (int)L,
                                                          tl);
  c->launch_count++;
  if (int rc = client_errors(c, "ctl_encrypt")) {
    ctl_ct_destroy(ct);
    return rc;
  }
  *out = ct;
  return CTL_OK;
}

// Decryption to centred coefficient values [count][N] (device doubles).
int decrypt_coeffs_dev(ctl_context* c, const ctl_keys* k, const ctl_ct* ct, double* m_dev) {
  const uint32_t N = c->N, lvl = ct->level, L = c->L;
  DBuf t(c, (size_t)ct->count * lvl * N);
  CHECK_ALLOC(t);
  launch_decrypt_mul(c, ct->d, k->d_s, t.p, (int)ct->count, (int)lvl);
  launch_ntt_inv(c, t.p, (size_t)lvl * N, (int)ct->count, 0, (int)lvl, (int)lvl);
  const size_t tot = (size_t)ct->count * N;
  k_crt_centred<<<grid_of(c, tot), 256, 0, c->stream>>>(t.p, (int)lvl, (int)c->logN, tot, c->d_primes,
                                                         c->client->garner, (int)L,
                                                         c->client->qwords + (size_t)lvl * (L + 1),
                                                         c->client->halfwords + (size_t)lvl * (L + 1), m_dev);
  c->launch_count++;
  return last_cuda("decrypt");
}

}  // namespace ctl

using namespace ctl;

extern "C" int ctl_encode_dev(ctl_context* c, const double* z_dev, size_t nz, uint32_t count, double scale,
                              int64_t* m_dev) {
  if (!c || !m_dev || (nz && !z_dev) || !count || nz > c->N / 2 || !(scale > 0)) {
    set_error("ctl_encode_dev: invalid argument");
    return CTL_EINVAL;
  }
  if (int rc = need_client(c, "ctl_encode_dev")) return rc;
  launch_encode(c, z_dev, nz, count, scale, (i64*)m_dev);
  return client_errors(c, "ctl_encode_dev");
}

extern "C" int ctl_decode_dev(ctl_context* c, const double* m_dev, uint32_t count, size_t nz, double scale,
                              double* z_dev) {
  if (!c || !m_dev || !z_dev || !count || nz > c->N / 2 || !(scale > 0)) {
    set_error("ctl_decode_dev: invalid argument");
    return CTL_EINVAL;
  }
  if (int rc = need_client(c, "ctl_decode_dev")) return rc;
  launch_decode(c, m_dev, nz, count, scale, z_dev);
  return last_cuda("ctl_decode_dev");
}

extern "C" int ctl_encrypt_coeffs_dev(ctl_context* c, const ctl_keys* k, const int64_t* m_dev, uint32_t count,
                                      const uint64_t* seeds, ctl_ct** out) {
  if (!c || !k || !m_dev || !seeds || !count || !out) {
    set_error("ctl_encrypt_coeffs_dev: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (!k->d_s) {
    set_error("ctl_encrypt_coeffs_dev: this key set holds no secret key (imported evaluation keys)");
    return CTL_EKEY;
  }
  if (int rc = need_client(c, "ctl_encrypt_coeffs_dev")) return rc;
  return encrypt_coeffs_dev(c, k, (const i64*)m_dev, count, (const u64*)seeds, out);
}

extern "C" int ctl_encrypt_dev(ctl_context* c, const ctl_keys* k, const double* z_dev, size_t nz, uint32_t count,
                               const uint64_t* seeds, ctl_ct** out) {
  if (!c || !k || (nz && !z_dev) || !seeds || !count || !out || nz > c->N / 2) {
    set_error("ctl_encrypt_dev: invalid argument");
    return CTL_EINVAL;
  }
  *out = nullptr;
  if (!k->d_s) {
    set_error("ctl_encrypt_dev: this key set holds no secret key (imported evaluation keys)");
    return CTL_EKEY;
  }
  if (int rc = need_client(c, "ctl_encrypt_dev")) return rc;
  DBuf m(c, (size_t)count * c->N);
  CHECK_ALLOC(m);
  launch_encode(c, z_dev, nz, count, c->scale, (i64*)m.p);
  return encrypt_coeffs_dev(c, k, (const i64*)m.p, count, (const u64*)seeds, out);
}

extern "C" int ctl_decrypt_coeffs_dev(ctl_context* c, const ctl_keys* k, const ctl_ct* ct, double* m_dev) {
  if (!c || !k || !ct || !m_dev) {
    set_error("ctl_decrypt_coeffs_dev: null argument");
    return CTL_EINVAL;
  }
  if (!k->d_s) {
    set_error("ctl_decrypt_coeffs_dev: this key set holds no secret key (imported evaluation keys)");
    return CTL_EKEY;
  }
  if (int rc = need_client(c, "ctl_decrypt_coeffs_dev")) return rc;
  return decrypt_coeffs_dev(c, k, ct, m_dev);
}

extern "C" int ctl_decrypt_dev(ctl_context* c, const ctl_keys* k, const ctl_ct* ct, size_t nz, double* z_dev) {
  if (!c || !k || !ct || !z_dev || nz > c->N / 2) {
    set_error("ctl_decrypt_dev: invalid argument");
    return CTL_EINVAL;
  }
  if (!k->d_s) {
    set_error("ctl_decrypt_dev: this key set holds no secret key (imported evaluation keys)");
    return CTL_EKEY;
  }
  if (int rc = need_client(c, "ctl_decrypt_dev")) return rc;
  DBuf m(c, (size_t)ct->count * c->N);
  CHECK_ALLOC(m);
  if (int rc = decrypt_coeffs_dev(c, k, ct, (double*)m.p)) return rc;
  launch_decode(c, (const double*)m.p, nz, ct->count, ct->scale, z_dev);
  return last_cuda("ctl_decrypt_dev");
}
