// Host launchers of the plain and rescaling transforms (kernels in ntt_impl.cuh).
#include "ntt_impl.cuh"

namespace ctl {

void launch_ntt_fwd(ctl_context* c, u64* data, size_t poly_stride, int n_polys, int limb_lo, int limb_hi, int lvl) {
  run_ntt<false>(c, KC_NTT_FWD, ProLoad{data, poly_stride}, EpiStore{data, poly_stride}, n_polys,
                 limb_lo, limb_hi, lvl, limb_cost(c, (double)n_polys * (limb_hi - limb_lo)));
}

void launch_ntt_inv(ctl_context* c, u64* data, size_t poly_stride, int n_polys, int limb_lo, int limb_hi, int lvl) {
  run_ntt<true>(c, KC_NTT_INV, ProLoad{data, poly_stride}, EpiStore{data, poly_stride}, n_polys,
                limb_lo, limb_hi, lvl, limb_cost(c, (double)n_polys * (limb_hi - limb_lo)));
}

void launch_ntt_inv_oop(ctl_context* c, const u64* src, size_t src_stride, u64* dst, size_t dst_stride, int n_polys,
                        int limb_lo, int limb_hi, int lvl, const InvScale* scl) {
  // limb l of poly p: read at src + p*src_stride + l*N, written at dst + p*dst_stride + l*N
  run_ntt<true>(c, KC_NTT_INV, ProLoad{src, src_stride}, EpiStore{dst, dst_stride}, n_polys, limb_lo, limb_hi, lvl,
                limb_cost(c, (double)n_polys * (limb_hi - limb_lo), scl != nullptr), scl);
}

void launch_intt_rescale_last(ctl_context* c, const u64* in, size_t poly_stride, int n_polys, int lvl, u64* r_out) {
  const RescaleTab& R = c->rescale_tabs[lvl];
  // limb lvl-1 of poly p is read at in + p*poly_stride + (lvl-1)*N; r_out[p] is written.
  run_ntt<true>(c, KC_RESCALE, ProLoad{in, poly_stride}, EpiRescaleLast{r_out, R.h}, n_polys,
                lvl - 1, lvl, lvl, limb_cost(c, (double)n_polys));
}

void launch_rescale_ntt(ctl_context* c, const u64* r, const u64* in, size_t in_stride, u64* out, size_t out_stride,
                        int n_polys, int lvl) {
  const RescaleTab& R = c->rescale_tabs[lvl];
  ProRescale pro{r, R.h};
  EpiRescale epi{in, in_stride, out, out_stride, R.inv, R.inv_sh};
  // per output limb: the transform of the last limb's residue r, then (c_i - r) q_l^-1 (two
  // products); bytes: r once per poly, each input limb read and each output limb written
  const double N = (double)c->N, outl = (double)n_polys * (lvl - 1);
  run_ntt<false>(c, KC_RESCALE, pro, epi, n_polys, 0, lvl - 1, lvl,
                 Cost{outl * (butterflies(c) + 2.0 * N), 8.0 * N * (n_polys + 2.0 * outl)});
}

}  // namespace ctl
