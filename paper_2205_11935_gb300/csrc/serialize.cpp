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

// One limb of N residues, LSB-first at w bits each through a 128-bit window; out holds
// limb_bytes(q, N) zeroed bytes.
void pack_limb(const u64* src, uint32_t N, uint32_t w, uint8_t* out) {
  unsigned __int128 acc = 0;
  uint32_t nbits = 0;
  size_t o = 0;
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
}
// The inverse; false if a residue is not below q.
bool unpack_limb(const uint8_t* in, uint32_t N, uint32_t w, u64 q, u64* dst) {
  const u64 mask = w == 64 ? ~0ull : (1ull << w) - 1;
  unsigned __int128 acc = 0;
  uint32_t nbits = 0;
  size_t o = 0;
  for (uint32_t k = 0; k < N; k++) {
    while (nbits < w) {
      acc |= (unsigned __int128)in[o++] << nbits;
      nbits += 8;
    }
    const u64 v = (u64)acc & mask;
    acc >>= w;
    nbits -= w;
    if (v >= q) return false;
    dst[k] = v;
  }
  return true;
}
void put64(uint8_t* p, u64 v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
u64 get64(const uint8_t* p) {
  u64 v = 0;
  for (int i = 0; i < 8; i++) v |= (u64)p[i] << (8 * i);
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
      pack_limb((const u64*)(coeffs + ((size_t)p * level + i) * N), N, bitlen(moduli[i]), out + pos);
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
      if (!unpack_limb(in + pos, N, bitlen(moduli[i]), moduli[i], (u64*)(coeffs + ((size_t)p * lvl + i) * N))) {
        set_error("ctl_deserialize: residue out of range (poly %u, limb %u)", p, i);
        return CTL_EINVAL;
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

// ---------------------------------------------------------------------------------
// Key-switching key messages (the evaluation keys a client sends to the server).  Format:
//   bytes 0..3 'C' 'T' 'L' 'K', 4..7 N, 8..9 limbs (data then special primes), 10 digits
//   (beta), 11 flags (bit 0: seeded), 12..19 key id, 20..27 key seed (seeded only), then
//   per digit d the limbs of b_d and, unless seeded, of a_d, packed as ciphertext limbs.
// A seeded message omits every a_d: it is the uniform polynomial of the key generation's
// streams (seed, key id, digit, limb), drawn again on receipt.
// ---------------------------------------------------------------------------------
namespace {
constexpr size_t kKeyHeader = 20;
}

extern "C" size_t ctl_key_message_size(uint32_t N, const uint64_t* moduli, uint32_t limbs, uint32_t beta,
                                       int seeded) {
  if (!valid(N, moduli, limbs) || beta == 0 || beta > 255) return 0;
  size_t s = kKeyHeader + (seeded ? 8 : 0), per = 0;
  for (uint32_t i = 0; i < limbs; i++) per += limb_bytes(moduli[i], N);
  return s + (size_t)beta * (seeded ? 1 : 2) * per;
}

extern "C" int ctl_serialize_key(uint32_t N, const uint64_t* moduli, uint32_t limbs, uint32_t beta, uint64_t key_id,
                                 const uint64_t* coeffs, int seeded, uint64_t seed, uint8_t* out, size_t cap,
                                 size_t* size) {
  const size_t need = ctl_key_message_size(N, moduli, limbs, beta, seeded);
  if (!need || !coeffs || !out) {
    set_error("ctl_serialize_key: invalid argument");
    return CTL_EINVAL;
  }
  if (cap < need) {
    set_error("ctl_serialize_key: %zu bytes needed, %zu given", need, cap);
    return CTL_EINVAL;
  }
  for (size_t j = 0; j < (size_t)beta * 2; j++)
    for (uint32_t i = 0; i < limbs; i++)
      for (uint32_t k = 0; k < N; k++)
        if (coeffs[(j * limbs + i) * N + k] >= moduli[i]) {
          set_error("ctl_serialize_key: residue not reduced (limb %u)", i);
          return CTL_EINVAL;
        }
  memset(out, 0, need);
  out[0] = 'C';
  out[1] = 'T';
  out[2] = 'L';
  out[3] = 'K';
  put32(out + 4, N);
  out[8] = (uint8_t)(limbs & 0xFF);
  out[9] = (uint8_t)(limbs >> 8);
  out[10] = (uint8_t)beta;
  out[11] = seeded ? 1 : 0;
  put64(out + 12, key_id);
  size_t pos = kKeyHeader;
  if (seeded) {
    put64(out + pos, seed);
    pos += 8;
  }
  for (uint32_t d = 0; d < beta; d++)
    for (uint32_t p = 0; p < (seeded ? 1u : 2u); p++)
      for (uint32_t i = 0; i < limbs; i++) {
        pack_limb((const u64*)(coeffs + (((size_t)d * 2 + p) * limbs + i) * N), N, bitlen(moduli[i]), out + pos);
        pos += limb_bytes(moduli[i], N);
      }
  if (size) *size = need;
  return CTL_OK;
}

extern "C" int ctl_deserialize_key(const uint8_t* in, size_t size, uint32_t N, const uint64_t* moduli,
                                   uint32_t limbs, uint32_t beta, uint64_t* coeffs, size_t cap,
                                   uint64_t* key_id) {
  if (!in || !moduli || !coeffs || size < kKeyHeader) {
    set_error("ctl_deserialize_key: invalid argument");
    return CTL_EINVAL;
  }
  const bool seeded = (in[11] & 1) != 0;
  if (in[0] != 'C' || in[1] != 'T' || in[2] != 'L' || in[3] != 'K' || get32(in + 4) != N ||
      ((uint32_t)in[8] | ((uint32_t)in[9] << 8)) != limbs || in[10] != beta || (in[11] & ~1u) ||
      size != ctl_key_message_size(N, moduli, limbs, beta, seeded ? 1 : 0)) {
    set_error("ctl_deserialize_key: not a key message for these parameters");
    return CTL_EINVAL;
  }
  if (cap < (size_t)beta * 2 * limbs * N) {
    set_error("ctl_deserialize_key: output needs %zu words", (size_t)beta * 2 * limbs * N);
    return CTL_EINVAL;
  }
  const u64 kid = get64(in + 12);
  size_t pos = kKeyHeader;
  u64 seed = 0;
  if (seeded) {
    seed = get64(in + pos);
    pos += 8;
  }
  for (uint32_t d = 0; d < beta; d++)
    for (uint32_t p = 0; p < (seeded ? 1u : 2u); p++)
      for (uint32_t i = 0; i < limbs; i++) {
        if (!unpack_limb(in + pos, N, bitlen(moduli[i]), moduli[i],
                         (u64*)(coeffs + (((size_t)d * 2 + p) * limbs + i) * N))) {
          set_error("ctl_deserialize_key: residue out of range (digit %u, limb %u)", d, i);
          return CTL_EINVAL;
        }
        pos += limb_bytes(moduli[i], N);
      }
  if (seeded)
    for (uint32_t d = 0; d < beta; d++)
      for (uint32_t i = 0; i < limbs; i++) {
        SplitMixStream sa(seed, stream_id_key_a(kid, d, i));
        draw_uniform(sa, moduli[i], N, (u64*)(coeffs + (((size_t)d * 2 + 1) * limbs + i) * N));
      }
  if (key_id) *key_id = kid;
  return CTL_OK;
}
