// Host launcher of ModUp: the fast base conversion of each digit fused into the forward
// transforms of its extended limbs (kernels in ntt_impl.cuh).
#include "ntt_impl.cuh"

namespace ctl {

template <int NS>
static void modup_ns(ctl_context* c, const u64* src_coef, size_t coef_stride, const u64* src_ntt, size_t src_stride,
                     int nb, int lvl, u64* ext) {
  const int nd = (lvl + (int)c->alpha - 1) / (int)c->alpha;
  const int E = lvl + (int)c->K;
  ProModUp<NS> pro;
  pro.coef = src_coef;
  pro.coef_stride = coef_stride;
  pro.ntt = src_ntt;
  pro.stride = src_stride;
  pro.ext = ext;
  pro.nd = nd;
  pro.E = E;
  pro.lvl = lvl;
  pro.alpha = (int)c->alpha;
  for (int d = 0; d < CTL_MAX_DIGITS; d++)
    pro.tabs[d] = d < nd ? c->modup_tabs[(size_t)(lvl - 1) * c->beta + d] : ConvTab{};
  // Algorithmic work: only the E - |d| converted limbs of digit d are credited, each with
  // its transform and one product per source limb of the digit (the digit's own limbs are
  // copies; the per-source factors [a_j q_hat_j^-1] belong to the preceding inverse
  // transform).  Bytes: the digit's coefficient-form and NTT-form limbs read once, the E
  // extended limbs written once.
  double work = 0, bytes = 0;
  const double N = (double)c->N;
  for (int d = 0; d < nd; d++) {
    const int dl = std::min((int)c->alpha, lvl - d * (int)c->alpha);
    work += (double)(E - dl) * (butterflies(c) + dl * N);
    bytes += 8.0 * N * (2.0 * dl + E);
  }
  run_ntt<false>(c, KC_MODUP, pro, EpiStoreSplit{ext, (size_t)E * c->N}, nb * nd, 0, E, lvl,
                 Cost{nb * work, nb * bytes});
}

void launch_modup_ntt(ctl_context* c, const u64* src_coef, size_t coef_stride, const u64* src_ntt, size_t src_stride,
                      int nb, int lvl, u64* ext) {
  switch (c->alpha) {
    case 1: modup_ns<1>(c, src_coef, coef_stride, src_ntt, src_stride, nb, lvl, ext); break;
    case 2: modup_ns<2>(c, src_coef, coef_stride, src_ntt, src_stride, nb, lvl, ext); break;
    case 3:
    case 4: modup_ns<4>(c, src_coef, coef_stride, src_ntt, src_stride, nb, lvl, ext); break;
    default: modup_ns<8>(c, src_coef, coef_stride, src_ntt, src_stride, nb, lvl, ext); break;
  }
}

}  // namespace ctl
