// Ciphertext serialisation for the client <-> server messages of CryptoTL (Sec. 5.1: the
// client sends a ciphertext of log2(q) * N bits, the server answers with log2(q_0) * 2N
// bits).  Host-only: works on coefficient-form arrays as ctl_ct_export writes them, so a
// client or a server can size and pack messages without a GPU.
//
// Format (little-endian):
//   bytes 0..3   'C' 'T' 'L' '1'
//   bytes 4..7   N
//   bytes 8..9   level (live data primes)
//   byte  10     stored polynomials (1 = c0 only, seeded; 2 = c0 and c1)
//   byte  11     flags (bit 0: seeded, c1 is regenerated from the seed)
//   bytes 12..15 zero
//   bytes 16..23 seed (seeded messages only)
//   then, per stored polynomial and per limb i < level, the N residues packed LSB-first
//   at w_i = bit length of q_i bits each, every limb padded to a whole byte.
#include <cstring>

#include "ctl_internal.h"

using namespace ctl;

namespace {
constexpr size_t kHeader = 16;

uint32_t bitlen(u64 v) {
  uint32_t b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

size_t limb_bytes(u64 q, uint32_t N) { return ((size_t)bitlen(q) * N + 7) / 8; }

bool valid(uint32_t N, const uint64_t* moduli, uint32_t level) {
  return moduli && level > 0 && level <= 0xFFFF && N >= 2 && (N & (N - 1)) == 0;
}

void put32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
uint32_t get32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
}  // namespace

extern "C" size_t ctl_serialized_size(uint32_t N, const uint64_t* moduli, uint32_t level, int seeded) {
  if (!valid(N, moduli, level)) return 0;
  size_t s = kHeader + (seeded ? 8 : 0);
  for (uint32_t i = 0; i < level; i++) s += (seeded ? 1 : 2) * limb_bytes(moduli[i], N);
  return s;
}

extern "C" int ctl_serialize(uint32_t N, const uint64_t* moduli, uint32_t level, const uint64_t* coeffs, int seeded,
                             uint64_t seed, uint8_t* out, size_t cap, size_t* size) {
  if (!valid(N, moduli, level) || !coeffs || !out) {
    set_error("ctl_serialize: invalid argument");
    return CTL_EINVAL;
  }
  const size_t need = ctl_serialized_size(N, moduli, level, seeded);
  if (cap < need) {
    set_error("ctl_serialize: %zu bytes needed, %zu given", need, cap);
    return CTL_EINVAL;
  }
  const uint32_t np = seeded ? 1 : 2;
  for (uint32_t p = 0; p < np; p++)
    for (uint32_t i = 0; i < level; i++)
      for (uint32_t k = 0; k < N; k++)
        if (coeffs[((size_t)p * level + i) * N + k] >= moduli[i]) {
          set_error("ctl_serialize: residue not reduced (poly %u, limb %u)", p, i);
          return CTL_EINVAL;
        }
  memset(out, 0, need);
  out[0] = 'C';
  out[1] = 'T';
  out[2] = 'L';
  out[3] = '1';
  put32(out + 4, N);
  out[8] = (uint8_t)(level & 0xFF);
  out[9] = (uint8_t)(level >> 8);
  out[10] = (uint8_t)np;
  out[11] = seeded ? 1 : 0;
  size_t pos = kHeader;
  if (seeded) {
    for (int b = 0; b < 8; b++) out[pos + b] = (uint8_t)(seed >> (8 * b));
    pos += 8;
  }
  for (uint32_t p = 0; p < np; p++)
    for (uint32_t i = 0; i < level; i++) {
      const uint32_t w = bitlen(moduli[i]);
      const uint64_t* src = coeffs + ((size_t)p * level + i) * N;
      // LSB-first bit stream: residues enter a 128-bit window, whole bytes leave it
      unsigned __int128 acc = 0;
      uint32_t nbits = 0;
      size_t o = pos;
      for (uint32_t k = 0; k < N; k++) {
        acc |= (unsigned __int128)src[k] << nbits;
        nbits += w;
        while (nbits >= 8) {
          out[o++] = (uint8_t)acc;
          acc >>= 8;
          nbits -= 8;
        }
      }
      if (nbits) out[o] = (uint8_t)acc;
      pos += limb_bytes(moduli[i], N);
    }
  if (size) *size = need;
  return CTL_OK;
}

extern "C" int ctl_deserialize(const uint8_t* in, size_t size, uint32_t N, const uint64_t* moduli, uint32_t max_level,
                               uint64_t* coeffs, size_t cap, uint32_t* level) {
  if (!in || !moduli || !coeffs || size < kHeader) {
    set_error("ctl_deserialize: invalid argument");
    return CTL_EINVAL;
  }
  if (in[0] != 'C' || in[1] != 'T' || in[2] != 'L' || in[3] != '1' || get32(in + 4) != N) {
    set_error("ctl_deserialize: not a ciphertext message for N = %u", N);
    return CTL_EINVAL;
  }
  const uint32_t lvl = (uint32_t)in[8] | ((uint32_t)in[9] << 8);
  const uint32_t np = in[10];
  const bool seeded = (in[11] & 1) != 0;
  if (lvl == 0 || lvl > max_level || np != (seeded ? 1u : 2u) || (in[11] & ~1u) ||
      size != ctl_serialized_size(N, moduli, lvl, seeded ? 1 : 0)) {
    set_error("ctl_deserialize: malformed header or size");
    return CTL_EINVAL;
  }
  if (cap < (size_t)2 * lvl * N) {
    set_error("ctl_deserialize: output needs %zu words", (size_t)2 * lvl * N);
    return CTL_EINVAL;
  }
  size_t pos = kHeader;
  u64 seed = 0;
  if (seeded) {
    for (int b = 0; b < 8; b++) seed |= (u64)in[pos + b] << (8 * b);
    pos += 8;
  }
  for (uint32_t p = 0; p < np; p++)
    for (uint32_t i = 0; i < lvl; i++) {
      const uint32_t w = bitlen(moduli[i]);
      const u64 mask = w == 64 ? ~0ull : (1ull << w) - 1;
      uint64_t* dst = coeffs + ((size_t)p * lvl + i) * N;
      unsigned __int128 acc = 0;
      uint32_t nbits = 0;
      size_t o = pos;
      for (uint32_t k = 0; k < N; k++) {
        while (nbits < w) {
          acc |= (unsigned __int128)in[o++] << nbits;
          nbits += 8;
        }
        const u64 v = (u64)acc & mask;
        acc >>= w;
        nbits -= w;
        if (v >= moduli[i]) {
          set_error("ctl_deserialize: residue out of range (poly %u, limb %u)", p, i);
          return CTL_EINVAL;
        }
        dst[k] = v;
      }
      pos += limb_bytes(moduli[i], N);
    }
  if (seeded) {
    // c1 = a of the encryption with this seed: uniform residues from the stream of each limb
    for (uint32_t i = 0; i < lvl; i++) {
      SplitMixStream sa(seed, stream_id_enc_a(i));
      draw_uniform(sa, moduli[i], N, (u64*)(coeffs + ((size_t)lvl + i) * N));
    }
  }
  if (level) *level = lvl;
  return CTL_OK;
}

// Host-only encoding straight to residues (the path a plaintext takes when its scale is
// beyond 64-bit coefficients, such as a bias added before a rescale).
extern "C" int ctl_encode_residues(uint32_t N, const uint64_t* moduli, uint32_t lvl, const double* x, size_t n,
                                   double scale, uint64_t* out) {
  if (!moduli || !out || (n && !x) || N < 16 || N > 16384 || (N & (N - 1)) || n > N / 2 || lvl == 0 ||
      !(scale > 0)) {
    set_error("ctl_encode_residues: invalid argument");
    return CTL_EINVAL;
  }
  Encoder e;
  e.init(N);
  if (!e.encode_rns(x, n, scale, (const u64*)moduli, lvl, (u64*)out)) {
    set_error("ctl_encode_residues: value out of range");
    return CTL_EINVAL;
  }
  return CTL_OK;
}
