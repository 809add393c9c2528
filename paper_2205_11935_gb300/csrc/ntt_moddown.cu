// Host launchers of ModDown: the conversion from the special primes fused into the forward
// transforms of the data limbs, P^-1 and the optional addend in the epilogue (kernels in
// ntt_impl.cuh).
#include "ntt_impl.cuh"

namespace ctl {

template <int NS>
static void moddown_ns(ctl_context* c, const u64* acc, size_t acc_stride, int n_polys, int lvl, u64* out,
                       size_t out_stride, const u64* addend, size_t add_r, size_t add_b, size_t add_p, bool add_both,
                       int nb, const RotList* rl, bool accum) {
  ProModDown<NS> pro;
  pro.acc = acc;
  pro.acc_stride = acc_stride;
  pro.lvl = lvl;
  pro.tab = c->moddown.conv;
  EpiModDown epi;
  epi.acc = acc;
  epi.acc_stride = acc_stride;
  epi.out = out;
  epi.out_stride = out_stride;
  epi.pinv = c->moddown.pinv;
  epi.pinv_sh = c->moddown.pinv_sh;
  epi.addend = addend;
  epi.add_r = add_r;
  epi.add_b = add_b;
  epi.add_p = add_p;
  epi.add_both = add_both ? 1 : 0;
  epi.nb = nb;
  epi.accum = accum ? 1 : 0;
  for (int r = 0; r < CTL_MAX_ROT; r++) epi.g[r] = (rl && r < rl->n) ? rl->g[r] : 1;
  // per output limb: the transform, one product per special limb (conversion) and the P^-1
  // product.  Bytes: the K special limbs once per poly; per output limb its accumulator
  // limb read, the result written, and the addend (and the output, when accumulating) read.
  const double N = (double)c->N;
  const double add_polys = addend ? (add_both ? n_polys : n_polys / 2.0) : 0.0;
  const double bytes = 8.0 * N * ((double)n_polys * c->K + (double)lvl * (2.0 * n_polys + add_polys +
                                                                          (accum ? n_polys : 0.0)));
  run_ntt<false>(c, KC_MODDOWN, pro, epi, n_polys, 0, lvl, lvl,
                 Cost{(double)n_polys * lvl * (butterflies(c) + (double)(c->K + 1) * N), bytes});
}

template <class... A>
static void moddown_dispatch(ctl_context* c, A... a) {
  switch (c->K) {
    case 1: moddown_ns<1>(c, a...); break;
    case 2: moddown_ns<2>(c, a...); break;
    case 3:
    case 4: moddown_ns<4>(c, a...); break;
    default: moddown_ns<8>(c, a...); break;
  }
}

void launch_moddown_ntt(ctl_context* c, const u64* acc, int nr, int nb, int lvl, u64* out, const u64* addend,
                        size_t add_r, size_t add_b, size_t add_p, bool add_both, const RotList& rl, bool accum) {
  const size_t EN = (size_t)(lvl + (int)c->K) * c->N;
  moddown_dispatch(c, acc, EN, nr * nb * 2, lvl, out, (size_t)lvl * c->N, addend, add_r, add_b, add_p, add_both, nb,
                   &rl, accum);
}

void launch_moddown_polys(ctl_context* c, const u64* acc, size_t acc_stride, int n_polys, int lvl, u64* out,
                          size_t out_stride) {
  moddown_dispatch(c, acc, acc_stride, n_polys, lvl, out, out_stride, (const u64*)nullptr, (size_t)0, (size_t)0,
                   (size_t)0, false, 1, (const RotList*)nullptr, false);
}

}  // namespace ctl
