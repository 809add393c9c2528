// Giant-step sums of ModDowns and their final transform (kernels in ntt_impl.cuh and below).
#include "ntt_impl.cuh"

namespace ctl {

// ---------------------------------------------------------------------------------
// Giant-step sums of ModDowns (see launch_giant_accum in ctl_internal.h).  A thread owns
// coefficient k of (ciphertext b, poly t) for a group of up to LG data limbs and sweeps
// the nr results, RPI at a time: per result it reads the K special-limb values once and
// converts them to every limb of its group.
// ---------------------------------------------------------------------------------
template <int K, int LG, int RPI>
__global__ void __launch_bounds__(256, 4) k_giant_accum(const u64* __restrict__ acc, int nr, int nb, int lvl, int E,
                                                        int logN, const __grid_constant__ RotList rl,
                                                        const u64* __restrict__ addend, size_t add_r, size_t add_b,
                                                        u64* __restrict__ D, u64* __restrict__ C,
                                                        u64* __restrict__ A, int first,
                                                        const __grid_constant__ ConvTab tab,
                                                        const DPrime* __restrict__ pr) {
  const int N = 1 << logN;
  const int ngroups = (lvl + LG - 1) / LG;
  const size_t total = (size_t)nb * 2 * ngroups * N;
  const size_t EN = (size_t)E << logN, LN = (size_t)lvl << logN;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(idx & (N - 1));
    const size_t rest = idx >> logN;
    const int grp = (int)(rest % ngroups);
    const int bt = (int)(rest / ngroups), b = bt >> 1, t = bt & 1;
    const int l0 = grp * LG;
    const int ng = min(LG, lvl - l0);
    u64 q[LG], cc[K][LG], cs[K][LG], d[LG], cv[LG], a[LG];
#pragma unroll
    for (int g = 0; g < LG; g++) {
      const int l = g < ng ? l0 + g : l0;
      q[g] = pr[l].q;
#pragma unroll
      for (int j = 0; j < K; j++) {
        cc[j][g] = __ldg(tab.c + (size_t)j * tab.nt + l);
        cs[j][g] = __ldg(tab.c_sh + (size_t)j * tab.nt + l);
      }
      d[g] = cv[g] = a[g] = 0;
    }
    const bool with_a = t == 0 && addend != nullptr;
    // one rotation's contribution from its loaded values
    auto add_rot = [&](const u64 (&sv)[K], const u64 (&dv)[LG], const u64 (&av)[LG]) {
#pragma unroll
      for (int g = 0; g < LG; g++) {
        if (g >= ng) break;
        d[g] = addmod(d[g], dv[g], q[g]);
        u64 s = 0;
#pragma unroll
        for (int j = 0; j < K; j++) {
          s += shoup_small(sv[j], cc[j][g], cs[j][g], q[g]);
          if (s >= 4 * q[g]) s -= 4 * q[g];
        }
        cv[g] = addmod(cv[g], reduce4(s, q[g]), q[g]);
        if (with_a) a[g] = addmod(a[g], av[g], q[g]);
      }
    };
    auto load_rot = [&](int r, u64 (&sv)[K], u64 (&dv)[LG], u64 (&av)[LG]) {
      const u64* base = acc + ((size_t)r * nb * 2 + bt) * EN + k;
#pragma unroll
      for (int j = 0; j < K; j++) sv[j] = __ldg(base + ((size_t)(lvl + j) << logN));
      const uint32_t src = rl.g[r] == 1 ? k : auto_src32(k, (uint32_t)rl.g[r], logN);
      const u64* ad = with_a ? addend + r * add_r + b * add_b + src : nullptr;
#pragma unroll
      for (int g = 0; g < LG; g++) {
        const int l = g < ng ? l0 + g : l0;
        dv[g] = __ldg(base + ((size_t)l << logN));
        av[g] = with_a ? __ldg(ad + ((size_t)l << logN)) : 0;
      }
    };
    // RPI rotations per iteration: all their loads in flight before the arithmetic
    int r = 0;
    for (; r + RPI - 1 < nr; r += RPI) {
      u64 sv[RPI][K], dv[RPI][LG], av[RPI][LG];
#pragma unroll
      for (int u = 0; u < RPI; u++) load_rot(r + u, sv[u], dv[u], av[u]);
#pragma unroll
      for (int u = 0; u < RPI; u++) add_rot(sv[u], dv[u], av[u]);
    }
    for (; r < nr; r++) {
      u64 s0[K], d0[LG], a0[LG];
      load_rot(r, s0, d0, a0);
      add_rot(s0, d0, a0);
    }
#pragma unroll
    for (int g = 0; g < LG; g++) {
      if (g >= ng) break;
      const int l = l0 + g;
      const size_t o = (size_t)bt * LN + ((size_t)l << logN) + k;
      D[o] = first ? d[g] : addmod(D[o], d[g], q[g]);
      C[o] = first ? cv[g] : addmod(C[o], cv[g], q[g]);
      if (t == 0) {
        const size_t oa = (size_t)b * LN + ((size_t)l << logN) + k;
        A[oa] = first ? a[g] : addmod(A[oa], a[g], q[g]);
      }
    }
  }
}

void launch_giant_accum(ctl_context* c, const u64* acc, int nr, int nb, int lvl, const RotList& rl,
                        const u64* addend, size_t add_r, size_t add_b, u64* D, u64* C, u64* A, bool first) {
  // One limb per thread and two rotations' loads in flight, at 63 registers (four blocks of
  // 256 per SM): the sums are bound by global-memory latency, so more resident warps beat
  // fewer re-reads of the special limbs (which L2 serves); measured on the batched forward
  // against two or four limbs per thread and three or four rotations per iteration.
  constexpr int LG = 1, RPI = 2;
  const int ngroups = (lvl + LG - 1) / LG;
  const size_t total = (size_t)nb * 2 * ngroups * c->N;
  if (!total || nr <= 0) return;
  size_t g = (total + 255) / 256;
  const size_t cap = (size_t)c->sm_count * 16;
  const int grid = (int)(g < cap ? g : cap);
  const int E = lvl + (int)c->K;
  const double work = (double)nr * nb * 2 * lvl * c->N * c->K;
  // per rotation: the data and special limbs of both polys and the addend (poly 0) read once;
  // the three sums read (unless first) and written once per launch
  const double Nd = (double)c->N;
  const double bytes = 8.0 * Nd * ((double)nr * nb * (2.0 * (lvl + c->K) + (addend ? lvl : 0)) +
                                   (first ? 1.0 : 2.0) * nb * 5.0 * lvl);
  cudaEvent_t ev;
  timing_begin(c, KC_MODDOWN, &ev);
  switch (c->K) {
#define CTL_GIANT_CASE(KK)                                                                                        \
  case KK:                                                                                                        \
    k_giant_accum<KK, LG, RPI><<<grid, 256, 0, c->stream>>>(acc, nr, nb, lvl, E, (int)c->logN, rl, addend,       \
                                                            add_r, add_b, D, C, A, first ? 1 : 0,                 \
                                                            c->moddown.conv, c->d_primes);                        \
    break;
    CTL_GIANT_CASE(1)
    CTL_GIANT_CASE(2)
    CTL_GIANT_CASE(3)
    CTL_GIANT_CASE(4)
#undef CTL_GIANT_CASE
    default:
      set_error("giant-step ModDown: at most 4 special primes");
      break;
  }
  c->launch_count++;
  timing_end(c, KC_MODDOWN, ev, work, bytes);
}

void launch_giant_moddown(ctl_context* c, const u64* D, const u64* C, const u64* A, int nb, int lvl, u64* out) {
  const size_t LN = (size_t)lvl * c->N;
  EpiModDown epi;
  epi.acc = D;
  epi.acc_stride = LN;
  epi.out = out;
  epi.out_stride = LN;
  epi.pinv = c->moddown.pinv;
  epi.pinv_sh = c->moddown.pinv_sh;
  epi.addend = A;
  epi.add_r = 0;
  epi.add_b = LN;
  epi.add_p = 0;
  epi.add_both = 0;
  epi.nb = nb;
  epi.accum = 1;
  for (int r = 0; r < CTL_MAX_ROT; r++) epi.g[r] = 1;
  // per output limb: the transform of the summed conversions and the P^-1 product; bytes:
  // the sums C and D and the addend sum A (poly 0) read, the output read and written
  const double N = (double)c->N, limbs = 2.0 * nb * lvl;
  run_ntt<false>(c, KC_MODDOWN, ProLoad{C, LN}, epi, nb * 2, 0, lvl, lvl,
                 Cost{limbs * (butterflies(c) + N), 8.0 * N * (limbs * 4.0 + nb * lvl)});
}

}  // namespace ctl
