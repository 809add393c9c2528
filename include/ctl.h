/*
 * ctl.h -- C-ABI of the GB300 CKKS server path of CryptoTL (arXiv 2205.11935).
 *
 * CryptoTL's protocol (Fig. "alg:cryptotl", Sec. 3) has a client encrypt its input,
 * a server evaluate its frozen layers on the ciphertext ("ClassifyHE"), and the client
 * decrypt the resulting features.  This library is the server side, on one GPU:
 * CKKS with RNS limbs, hybrid key switching, the baby-step giant-step diagonal mat-vec
 * of Eq. (bsgs), the square activation and rescaling (Sec. 3.1).  The client calls
 * (keygen, encrypt, decrypt) are provided so that a test or a caller can close the loop.
 *
 * Conventions for every function:
 *  - Return value: CTL_OK (0) or a negative CTL_E* code; the message of the last error
 *    of the calling thread is available from ctl_last_error().  No C++ exception
 *    crosses this interface.  On error, output handles are left untouched (NULL).
 *  - Ownership: handles are created by the library and released by the matching
 *    *_destroy.  Input arrays are owned by the caller and are read (copied) before the
 *    call returns.  Output arrays are written before the call returns.
 *  - Pointers: every array argument is a HOST pointer unless its name ends in _dev.
 *  - Streams: all GPU work of a context runs on its stream (ctl_set_stream); calls that
 *    return host data synchronise that stream first.  Contexts and keys are immutable
 *    after creation and may be shared; a ciphertext must not be used by two concurrent
 *    calls.
 *  - Layout: a ciphertext at level l (l live data primes q_0..q_{l-1}) is a pair of
 *    ring elements, stored limb-major as [2][l][N] 64-bit residues.  Exported and
 *    imported ciphertexts are in coefficient form; on the device they are kept in the
 *    NTT (evaluation) form.  A batch of B ciphertexts is [B][2][l][N].
 *  - Parameters: the ring degree N is a power of two in [16, 16384]; prime sizes are
 *    20..61 bits; every prime is the largest unused prime q < 2^b with q = 1 mod
 *    max(2N, 32768) (so that N = 8192 and N = 16384 share primes).
 */
#ifndef CTL_H
#define CTL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CTL_OK 0
#define CTL_EINVAL (-1)   /* invalid argument (sizes, N, primes, NULL handle)        */
#define CTL_ELEVEL (-2)   /* no level left to rescale / level mismatch              */
#define CTL_ESCALE (-3)   /* scale mismatch between operands                        */
#define CTL_EKEY (-4)     /* a needed Galois or relinearisation key is missing      */
#define CTL_ENOMEM (-5)   /* device or host allocation failed                       */
#define CTL_ECUDA (-6)    /* a CUDA runtime call failed                              */
#define CTL_ETIMEOUT (-7) /* a bounded device or host wait expired                   */
#define CTL_EBUSY (-8)    /* admission refused (memory budget or queue full)        */
#define CTL_ENOTSUP (-9)  /* unsupported parameter combination                       */

typedef struct ctl_context ctl_context;
typedef struct ctl_keys ctl_keys;
typedef struct ctl_ct ctl_ct;
typedef struct ctl_model ctl_model;
typedef struct ctl_server ctl_server;
typedef struct ctl_multi ctl_multi;

/* Device allocator hooks: alloc(bytes, stream, user) returns device memory ordered on
 * `stream`; free(ptr, stream, user) releases it.  NULL hooks select the library's
 * stream-ordered pool (cudaMallocAsync). */
typedef void* (*ctl_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*ctl_free_fn)(void* ptr, void* stream, void* user);

/* Thread-local message of the last error, or "" if none. */
const char* ctl_last_error(void);
/* Library version string. */
const char* ctl_version(void);

/* Host only (no GPU needed): the primes the library would choose for `n` bit sizes at
 * ring degree N, written to out[n].  Same rule as ctl_context_create. */
int ctl_plan_primes(uint32_t N, const uint32_t* bits, uint32_t n, uint64_t* out);

/* ---------------------------------------------------------------------------------
 * Context: CKKS parameters (Sec. 3.1, "The CKKS HE scheme"; the modulus chain of the
 * "Multiplicative Depth" paragraph).  q_bits[n_q] is the data chain, q_0 first (the
 * last prime is the first to be dropped by rescaling); p_bits[n_p] are the special
 * primes of key switching.  dnum (1..n_q) is the number of key-switching digits at the
 * top level; each digit holds alpha = ceil(n_q/dnum) consecutive data primes.  scale is
 * the nominal encoding scale Delta.  seed is reserved for context-level randomness.
 * Builds device twiddle and base-conversion tables on the current CUDA device.
 * Errors: CTL_EINVAL (bad N or bit sizes), CTL_ECUDA, CTL_ENOMEM.
 * ------------------------------------------------------------------------------- */
int ctl_context_create(ctl_context** out, uint32_t N, const uint32_t* q_bits, uint32_t n_q, const uint32_t* p_bits,
                       uint32_t n_p, uint32_t dnum, double scale, uint64_t seed);
void ctl_context_destroy(ctl_context* ctx);
/* Writes the n_q + n_p primes (data chain then special primes) to moduli (nullable) and
 * the counts to the other (nullable) outputs. */
int ctl_context_info(const ctl_context* ctx, uint64_t* moduli, uint32_t* n_q, uint32_t* n_p, uint32_t* alpha);
/* Makes the context issue its work on `stream` (a cudaStream_t owned by the caller, which
 * must outlive the context's use of it; the library never destroys it), or, with NULL, on a
 * new stream of the library's own.  Work already queued on the previous stream is finished
 * first. */
int ctl_set_stream(ctl_context* ctx, void* stream);
int ctl_set_allocator(ctl_context* ctx, ctl_alloc_fn alloc_fn, ctl_free_fn free_fn, void* user);
/* Blocks until the context stream is idle. */
int ctl_synchronize(ctl_context* ctx);
/* How later dense layers (ctl_eval_dense*, ctl_model_create) evaluate Eq. (bsgs):
 *   CTL_DENSE_COMPOSED (default): the composition of whole rotations, each ending with
 *     its ModDown, the baby steps sharing one ModUp; t1 = 2^ceil(log2(t)/2).  Bit-identical
 *     to composing ctl_rotate, ctl_mul_plain_coeffs, ctl_add and ctl_rescale.
 *   CTL_DENSE_LAZY_MODDOWN: rotations kept in the extended basis Q*P, ModDown once per
 *     giant step (on c1) and once at the end; t1 = min(t, 2^ceil(log2(4t)/2)).  A
 *     different ciphertext of the same values (lower noise), not bit-identical to the
 *     default; needs the Galois keys of its own split.
 *   CTL_DENSE_RECT: the composed form, except that a layer whose padded output side
 *     tm = 2^ceil(log2 m) is below its input side tn = 2^ceil(log2 n) takes the
 *     rectangular form of ctl_eval_dense_rect (tm diagonals instead of tn, plus a
 *     log2(tn/tm)-rotation fold).  In a model, when such a layer is followed by
 *     [square,] replicate(tm), the fold also forms the [y, y] layout (fold 2) and that
 *     replicate is not run again.  Layers with tm >= tn are as in the composed form.
 *   CTL_DENSE_RECT_LAZY: as CTL_DENSE_RECT with Eq. (bsgs) of every layer (rectangular or
 *     not) in the lazy-ModDown form and its split; the fold is the same.
 * The paper fixes neither choice (Sec. 3.1 only fixes t = t1 * t2 and the hoisting).  A
 * model keeps the mode it was created with.  Errors: CTL_EINVAL (unknown mode). */
/* Register-resident NTT shapes for N = 4096 .. 16384 (other N use one shared-memory
 * kernel): R32 = N/32 threads with 32 elements each in three passes (5 + 5 + log2N-10
 * stages); R16 = N/16 threads with 16 elements each in 4-stage passes (twice the warps
 * per SM, one more shared-memory transpose).  Both compute the same exact transform.
 * ctl_set_ntt_shape sets the forward and inverse shapes of a context (CTL_NTT_SHAPE_AUTO
 * keeps the current one); ctl_autotune_ntt times both shapes on scratch limbs of the
 * context (plain forward and inverse transforms over batch_limbs limbs) and keeps the
 * faster per direction, writing the choices to the nullable outputs.  Contexts run the
 * autotuner once at creation.  Errors: CTL_EINVAL, CTL_ENOMEM, CTL_ECUDA. */
#define CTL_NTT_SHAPE_AUTO (-1)
#define CTL_NTT_SHAPE_R32 0
#define CTL_NTT_SHAPE_R16 1
int ctl_set_ntt_shape(ctl_context* ctx, int fwd_shape, int inv_shape);
int ctl_get_ntt_shape(const ctl_context* ctx, int* fwd_shape, int* inv_shape);
int ctl_autotune_ntt(ctl_context* ctx, uint32_t batch_limbs, int* fwd_shape, int* inv_shape);
/* Shape of the baby-step giant-step inner-sum kernel: baby-step values held per thread
 * (chunk 16 or 32; larger t1 is summed in chunks) and the split products with four or
 * three (karatsuba = 1) 32x32->64 multiply-adds.  Results are identical for every
 * shape.  Errors: CTL_EINVAL. */
int ctl_set_bsgs_shape(ctl_context* ctx, int chunk, int karatsuba);
/* Device-memory cap (bytes) of the key-switching temporaries of one launch group: the
 * rotations of a dense layer's baby and giant steps are key-switched in chunks whose
 * temporaries (coefficient-form inputs, ModUp digits, key-product results) stay within
 * it, at least one rotation per chunk.  Default 16 GiB.  Results are identical for every
 * cap (giant-step sums are carried across chunks).  Errors: CTL_EINVAL (null context or
 * zero bytes). */
int ctl_set_keyswitch_budget(ctl_context* ctx, uint64_t bytes);
/* Prediction windows (Sec. 3.1 "Multiple Predictions": p = floor(#slots / (2 #neurons))
 * inputs share one ciphertext).  Dense and conv1d layers created afterwards (and the
 * direct ctl_eval_dense / ctl_eval_conv1d calls) encode their plaintexts for p windows:
 * the pattern of slots [0, 2t) is repeated in every window [2t w, 2t (w+1)), w < p, so
 * each window of 2t slots is evaluated as an independent input ([x_w, x_w] at block
 * stride t inside its window) and its output sits at the start of the window.  The
 * rotations and the other layers are unchanged.  Default 1.  A layer whose 2 t p exceeds
 * N/2 fails with CTL_EINVAL.  Injected coefficient plaintexts are used as given.
 * Errors: CTL_EINVAL (p = 0 or p > N/4). */
int ctl_set_windows(ctl_context* ctx, uint32_t p);
#define CTL_DENSE_COMPOSED 0
#define CTL_DENSE_LAZY_MODDOWN 1
#define CTL_DENSE_RECT 2
#define CTL_DENSE_RECT_LAZY 3
int ctl_set_dense_mode(ctl_context* ctx, int mode);

/* ---------------------------------------------------------------------------------
 * Keys (Fig. alg:cryptotl: the client's key pair; Sec. 3.1 rotations need Galois keys).
 * Samples the ternary secret, the relinearisation key (s^2 -> s) and one Galois key
 * (sigma_{5^r}(s) -> s) per distinct rotation r of rotations[n_rot] (r < 0 allowed,
 * r = 0 mod N/2 needs none), all from SplitMix64 streams of `seed`.  Keys live on the
 * device.  Errors: CTL_EINVAL, CTL_ENOMEM, CTL_ECUDA.
 * ------------------------------------------------------------------------------- */
int ctl_keygen(ctl_context* ctx, const int32_t* rotations, uint32_t n_rot, uint64_t seed, ctl_keys** out);
void ctl_keys_destroy(ctl_keys* keys);
/* Exports key `key_id` (0 = relinearisation, odd g = Galois key of X -> X^g) as
 * [beta][2][n_q+n_p][N] coefficient-form residues into out (cap words).
 * Errors: CTL_EKEY (no such key), CTL_EINVAL (cap too small). */
int ctl_keys_export(const ctl_keys* keys, uint64_t key_id, uint64_t* out, size_t cap);
/* Evaluation keys received from a client (Fig. alg:cryptotl: the server holds the
 * client's public evaluation keys, never its secret).  ctl_keys_create makes an empty key
 * set with no secret: ctl_encrypt* and ctl_decrypt* on it fail with CTL_EKEY.
 * ctl_keys_import adds (or replaces) key key_id (0 = relinearisation, an odd Galois
 * element g < 2N = the key of X -> X^g) from the coefficient-form residues
 * coeffs[beta][2][n_q+n_p][N] that ctl_keys_export writes (n_words must equal that
 * size).  The import synchronises the context stream.  Errors: CTL_EINVAL (size, key id,
 * a residue >= its prime), CTL_ENOMEM, CTL_ECUDA. */
int ctl_keys_create(ctl_context* ctx, ctl_keys** out);
int ctl_keys_import(ctl_keys* keys, uint64_t key_id, const uint64_t* coeffs, size_t n_words);
/* Galois element 5^(r mod N/2) mod 2N of a left rotation by r. */
uint64_t ctl_galois_element(const ctl_context* ctx, int64_t r);

/* ---------------------------------------------------------------------------------
 * Client side (Fig. alg:cryptotl: HE.Enc, HE.Dec; Sec. 3.1 "SIMD Encoding").
 * ctl_encode: slot values x[n] (n <= N/2) -> integer coefficients m[N] at `scale`
 *   (host FP64 canonical embedding, round half away from zero).
 * ctl_encrypt: encodes x at the nominal scale and encrypts at the top level with the
 *   secret key: ct = (-a*s + m + e, a), a and e drawn from streams of `seed`.
 * ctl_encrypt_coeffs: the same from given integer coefficients m[N] (where the device client
 *   path applies, the randomness is drawn on the device, as ctl_encrypt_coeffs_dev does).
 * ctl_decrypt: decrypts and decodes the first n slots into y[n] (synchronises).
 * ctl_decrypt_coeffs: the centred coefficients of c0 + c1*s as doubles, m[N] (the CRT runs
 *   on the device where the device client path applies).
 * ------------------------------------------------------------------------------- */
int ctl_encode(ctl_context* ctx, const double* x, size_t n, double scale, int64_t* m);
int ctl_decode(ctl_context* ctx, const double* m, size_t n, double scale, double* y);
int ctl_encrypt(ctl_context* ctx, const ctl_keys* keys, const double* x, size_t n, uint64_t seed, ctl_ct** out);
int ctl_encrypt_coeffs(ctl_context* ctx, const ctl_keys* keys, const int64_t* m, uint64_t seed, ctl_ct** out);
int ctl_decrypt(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* ct, double* y, size_t n);
int ctl_decrypt_coeffs(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* ct, double* m);

/* Client side on the device, for batches of queries (N <= 16384 and at most 16 data primes;
 * CTL_EINVAL otherwise).
 * All pointers named *_dev are device memory owned by the caller; seeds is a host array.
 * ctl_encode_dev: count slot vectors z_dev[count][nz] -> integer coefficients
 *   m_dev[count][N] at `scale`: the canonical embedding of Sec. 3.1 computed as one
 *   length-N/2 FP64 FFT per vector (slot j at zeta^(5^j), zeta = exp(i pi / N)), rounded
 *   half away from zero.  Agrees with ctl_encode within one unit per coefficient (two FP64
 *   evaluation orders).  Synchronises; CTL_EINVAL if a coefficient leaves +-4e18.
 * ctl_decode_dev: m_dev[count][N] (doubles) -> z_dev[count][nz], the real parts of the
 *   slots divided by scale.  Asynchronous on the context stream.
 * ctl_encrypt_coeffs_dev: encrypts m_dev[count][N] at the top level, ciphertext b with
 *   seeds[b]: the uniform a and the centred binomial e are drawn on the device from the
 *   same counter-based streams as ctl_encrypt_coeffs, so each ciphertext equals
 *   ctl_encrypt_coeffs(m_b, seeds[b]) bit for bit.  Synchronises.
 * ctl_encrypt_dev: ctl_encode_dev at the nominal scale, then ctl_encrypt_coeffs_dev.
 * ctl_decrypt_coeffs_dev: the centred coefficients of c0 + c1*s of every ciphertext of ct
 *   as doubles, m_dev[count][N] (Garner's mixed radix on the device).  Asynchronous.
 * ctl_decrypt_dev: ctl_decrypt_coeffs_dev, then ctl_decode_dev at ct's scale into
 *   z_dev[count][nz].  Asynchronous.
 * Errors: CTL_EINVAL, CTL_EKEY (a key set without the secret), CTL_ENOMEM, CTL_ECUDA. */
int ctl_encode_dev(ctl_context* ctx, const double* z_dev, size_t nz, uint32_t count, double scale, int64_t* m_dev);
int ctl_decode_dev(ctl_context* ctx, const double* m_dev, uint32_t count, size_t nz, double scale, double* z_dev);
int ctl_encrypt_coeffs_dev(ctl_context* ctx, const ctl_keys* keys, const int64_t* m_dev, uint32_t count,
                           const uint64_t* seeds, ctl_ct** out);
int ctl_encrypt_dev(ctl_context* ctx, const ctl_keys* keys, const double* z_dev, size_t nz, uint32_t count,
                    const uint64_t* seeds, ctl_ct** out);
int ctl_decrypt_coeffs_dev(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* ct, double* m_dev);
int ctl_decrypt_dev(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* ct, size_t nz, double* z_dev);

/* ---------------------------------------------------------------------------------
 * Ciphertext handles.  ctl_ct_import copies count ciphertexts [count][2][level][N]
 * (coefficient form) from host memory to the device; ctl_ct_export writes them back
 * (synchronises).  ctl_ct_import_dev / export_dev do the same from/to device memory
 * (the caller's pointer, ordered on the context stream).
 * ------------------------------------------------------------------------------- */
int ctl_ct_import(ctl_context* ctx, const uint64_t* coeffs, uint32_t count, uint32_t level, double scale,
                  ctl_ct** out);
int ctl_ct_export(const ctl_ct* ct, uint64_t* coeffs, size_t cap);
int ctl_ct_import_dev(ctl_context* ctx, const uint64_t* coeffs_dev, uint32_t count, uint32_t level, double scale,
                      ctl_ct** out);
int ctl_ct_export_dev(const ctl_ct* ct, uint64_t* coeffs_dev, size_t cap);
int ctl_ct_info(const ctl_ct* ct, uint32_t* level, uint32_t* count, double* scale);
/* Concatenates cts[n] (same level and scale) into one batch; ctl_ct_slice copies
 * ciphertext i of a batch out. */
int ctl_ct_concat(ctl_context* ctx, const ctl_ct* const* cts, size_t n, ctl_ct** out);
int ctl_ct_slice(const ctl_ct* batch, uint32_t i, ctl_ct** out);
void ctl_ct_destroy(ctl_ct* ct);

/* ---------------------------------------------------------------------------------
 * Messages (Sec. 5.1: the client sends a ciphertext of log2(q) * N bits, the server
 * answers with one of log2(q_0) * 2N bits).  Host only, no GPU needed: these work on
 * coefficient-form arrays [2][level][N] as ctl_ct_export writes them and the primes of
 * the chain (ctl_plan_primes / ctl_context_info).  A message is a 16-byte header
 * ("CTL1", N, level, stored polys, flags), for seeded messages the 8-byte encryption
 * seed, then every stored limb i packed LSB-first at bitlen(q_i) bits per residue, each
 * limb padded to a byte.  seeded != 0 stores c0 only: valid for a fresh ctl_encrypt
 * result, whose c1 is the uniform polynomial drawn from the seed, which ctl_deserialize
 * draws again (the C->S message is then one ring element, as in Sec. 5.1).
 * ctl_serialized_size: message bytes (0 for invalid arguments).
 * ctl_serialize: writes the message to out[cap] and its size to *size (nullable).
 *   Errors: CTL_EINVAL (cap too small, a residue >= its prime, bad arguments).
 * ctl_deserialize: reads a message of exactly `size` bytes for ring degree N and primes
 *   moduli[>= level] into coeffs[2][level][N] (cap words) and its level (<= max_level) to
 *   *level.  Errors: CTL_EINVAL (malformed header, size, residue out of range).
 * ------------------------------------------------------------------------------- */
size_t ctl_serialized_size(uint32_t N, const uint64_t* moduli, uint32_t level, int seeded);
/* Key-switching key messages (the evaluation keys a client sends; host only): a key
 * [beta][2][limbs][N] in the coefficient form of ctl_keys_export (limbs = n_q + n_p, primes
 * moduli[limbs], data then special) is packed like ciphertext limbs after a 20-byte header
 * ("CTLK", N, limbs, beta, flags, key id).  seeded != 0 stores only the b part of every
 * digit plus the key-generation seed: the a parts are the uniform polynomials of the
 * streams (seed, key id, digit, limb), which ctl_deserialize_key draws again.  The
 * message of a key made by ctl_keygen(..., seed) with that seed is half the size.
 * Errors: CTL_EINVAL (capacity, parameters, a residue >= its prime, malformed message). */
size_t ctl_key_message_size(uint32_t N, const uint64_t* moduli, uint32_t limbs, uint32_t beta, int seeded);
int ctl_serialize_key(uint32_t N, const uint64_t* moduli, uint32_t limbs, uint32_t beta, uint64_t key_id,
                      const uint64_t* coeffs, int seeded, uint64_t seed, uint8_t* out, size_t cap, size_t* size);
int ctl_deserialize_key(const uint8_t* in, size_t size, uint32_t N, const uint64_t* moduli, uint32_t limbs,
                        uint32_t beta, uint64_t* coeffs, size_t cap, uint64_t* key_id);
/* Host only: slot values x[n] encoded at `scale` (any magnitude up to ~2^1000) straight to
 * residues out[lvl][N] modulo moduli[0..lvl): round(m_k) mod q_i with m_k as ctl_encode
 * defines it (half away from zero).  This is how dense and conv1d layers encode their
 * biases, which join the products before the rescale at scale in_scale * pt_scale.
 * Errors: CTL_EINVAL. */
int ctl_encode_residues(uint32_t N, const uint64_t* moduli, uint32_t lvl, const double* x, size_t n, double scale,
                        uint64_t* out);
int ctl_serialize(uint32_t N, const uint64_t* moduli, uint32_t level, const uint64_t* coeffs, int seeded,
                  uint64_t seed, uint8_t* out, size_t cap, size_t* size);
int ctl_deserialize(const uint8_t* in, size_t size, uint32_t N, const uint64_t* moduli, uint32_t max_level,
                    uint64_t* coeffs, size_t cap, uint32_t* level);

/* ---------------------------------------------------------------------------------
 * Homomorphic operations (Sec. 3.1).  Each accepts a batch (count >= 1) and returns a
 * new handle; the input is not modified.
 * ctl_rotate: left rotation of the slots by r (rot_r of Eq. bsgs).  Hybrid key
 *   switching: ModUp(c1) -> sigma_g -> key product -> ModDown; (sigma_g(c0) + ks0, ks1).
 *   Errors: CTL_EKEY if the Galois key of r is missing.
 * ctl_rescale: divides by the last prime with rounding ("rescaling ... is equivalent to
 *   rounding", Sec. 3.1).  Errors: CTL_ELEVEL at level 1.
 * ctl_eval_square: HMult(ct, ct) + relinearisation + rescale (the square activation;
 *   ciphertext products are the costliest operation, Sec. 5.1).  Scale becomes
 *   scale^2 / q_last.
 * ctl_eval_dense: y = W x for W (m x n, row-major FP64) by Eq. (bsgs): t = next power of
 *   two >= max(m, n) (zero padding), t2 = t/t1; t1+t2-2 rotations, t plaintext products,
 *   depth 1.  The split t1 depends on the dense mode (ctl_set_dense_mode):
 *     CTL_DENSE_COMPOSED (default): t1 = 2^ceil(log2(t)/2);
 *     CTL_DENSE_LAZY_MODDOWN:       t1 = min(t, 2^ceil(log2(4t)/2)).
 *   Either way the layer needs the Galois keys of 1..t1-1 and k*t1 (k = 1..t2-1) for
 *   that mode's t1 (ctl_model_rotations lists them).  In CTL_DENSE_RECT and
 *   CTL_DENSE_RECT_LAZY a layer with 2^ceil(log2 m) < 2^ceil(log2 n) is evaluated as
 *   ctl_eval_dense_rect with fold 1 (its keys and output layout are that call's); other
 *   layers as in CTL_DENSE_COMPOSED and CTL_DENSE_LAZY_MODDOWN respectively.  The input must hold [x, x] in slots
 *   [0, 2t); the output holds y in slots [0, m) and zeros elsewhere.  The diagonals are
 *   encoded at scale q_last * Delta / scale_in, so the output carries Delta again.
 *   bias (nullable, m values) is added before the rescale.
 *   Errors: CTL_EINVAL (2t > N/2), CTL_EKEY, CTL_ELEVEL.
 * ctl_eval_dense_coeffs: the same with the t diagonal plaintexts given as integer
 *   coefficients pts[t][N] (and bias as coefficients, nullable); the scale bookkeeping
 *   uses pt_scale.  Lets a caller inject exactly encoded plaintexts.
 * ctl_replicate: y + rot_{-t}(y): turns y in slots [0, t) into [y, y] (the layout the
 *   next dense layer needs, Sec. 3.1 "Multiple Predictions").
 * ------------------------------------------------------------------------------- */
int ctl_rotate(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, int32_t r, ctl_ct** out);
int ctl_rescale(ctl_context* ctx, const ctl_ct* in, ctl_ct** out);
int ctl_eval_square(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, ctl_ct** out);
int ctl_eval_dense(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const double* W, uint32_t m, uint32_t n,
                   const double* bias, ctl_ct** out);
int ctl_eval_dense_coeffs(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const int64_t* pts, uint32_t t,
                          const int64_t* bias, double pt_scale, ctl_ct** out);
int ctl_replicate(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, uint32_t t, ctl_ct** out);
/* Rectangular form of a dense layer (Sec. 3.1 "Dense-Layer" pads a non-square matrix with
 * zeros; this form pads only the short side).  For W (m x n) with tm = 2^ceil(log2 m)
 * below tn = 2^ceil(log2 n), on the [x, x] layout over 2 tn slots:
 *   rd_i[r] = W[r mod tm][(r + i) mod tn], r < tn, i < tm (zero outside W);
 *   z' = rescale( sum_k rot_{k t1}( sum_j rd'_{k t1 + j} o rot_j(x) ) [+ bias] ),
 *        rd'_i = rot_{-floor(i/t1) t1}(rd_i), t1 = 2^ceil(log2(tm)/2), t2 = tm / t1;
 *   fold >= 1: S = z'; S = S + rot_s(S) for s = tn/2, tn/4, ..., tm  -> y in slots [0, m);
 *   fold == 2: S = S + rot_{-tm}(z')                                  -> y also in [tm, tm + m).
 * Other slots of the output hold partial sums (not zeros).  Work: tm plaintext products
 * and t1 + t2 - 2 + log2(tn/tm) (+1) rotations, against tn products and about 2 sqrt(tn)
 * rotations for the square padding.  Needs the Galois keys of 1..t1-1, k*t1, the fold
 * shifts tn/2 .. tm and (fold 2) -tm.  bias (m values) is added before the rescale.
 * In the lazy-ModDown modes the sums of Eq. (bsgs) take that form and its split t1 =
 * min(tm, 2^ceil(log2(4 tm)/2)); the fold is the same.
 * Errors: CTL_EINVAL (tm >= tn, 2 tn > N/2, windows > 1), CTL_EKEY, CTL_ELEVEL.
 * ctl_eval_dense_rect_coeffs: the same with the tm plaintexts given as integer
 * coefficients pts[tm][N] (and bias as coefficients, nullable) at pt_scale. */
int ctl_eval_dense_rect(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const double* W, uint32_t m,
                        uint32_t n, const double* bias, int fold, ctl_ct** out);
int ctl_eval_dense_rect_coeffs(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const int64_t* pts,
                               uint32_t tm, uint32_t tn, const int64_t* bias, double pt_scale, int fold, ctl_ct** out);
int ctl_add(ctl_context* ctx, const ctl_ct* a, const ctl_ct* b, ctl_ct** out);
int ctl_mul_plain_coeffs(ctl_context* ctx, const ctl_ct* in, const int64_t* pt, double pt_scale, ctl_ct** out);

/* ---------------------------------------------------------------------------------
 * The other layers of the paper's frozen server network (Sec. 3.1 "1D Convolutions",
 * "Average Pool", "ReLU"; Sec. 4.1: Conv1D f = 9 -> Dense 768 + approximated ReLU ->
 * AveragePooling 3 -> Dense 766) and the operations they are built from.  Batches as
 * above; the input is not modified; on error *out is NULL.
 * ctl_eval_mul: HMult of two ciphertexts (same level and count): tensor product,
 *   relinearisation (s^2 -> s key), rescale.  Scale becomes scale_a * scale_b / q_last.
 *   ctl_eval_mul(a, a) equals ctl_eval_square(a) bit for bit.  Errors: CTL_ELEVEL
 *   (shapes differ or level < 2), CTL_EKEY.
 * ctl_mul_const: (C*c0, C*c1) for the integer constant C (the slot value C / c_scale in
 *   every slot); scale becomes scale * c_scale; no rescale.
 * ctl_add_const: adds the integer constant C to every slot (the plaintext (C, 0, .., 0)
 *   on c0); the slot value C / scale.  Scale unchanged.
 * ctl_drop_level: keeps the first `level` primes (reduction modulo Q_level, no division;
 *   scale unchanged).  Errors: CTL_ELEVEL (level 0 or above the input's).
 * ctl_eval_poly3: a[3] z^3 + a[2] z^2 + a[1] z + a[0] (a = a0..a3; the paper's ReLU
 *   approximation is such a polynomial) at multiplicative depth 2.  With q_a, q_b the
 *   last two primes and S the input scale: S2 = S*S/q_a, Sw = S2*S/q_b, integer
 *   constants C3 = round(a3 q_a), C2 = round(a2 S), C1 = round(a1 (Sw q_a)/S),
 *   C0 = round(a0 Sw) (half away from zero), and
 *     out = HMult(square(z), rescale(C3 z) + C2) + drop(rescale(C1 z)) + C0,
 *   level - 2, scale Sw.  Errors: CTL_ELEVEL (level < 3), CTL_EINVAL (a constant above
 *   2^63), CTL_EKEY.
 * ctl_eval_avgpool: stride-1 average pool of size f, (1/f) sum_{i=0}^{f-1} rot_{-i}(x):
 *   f-1 rotations (one shared ModUp), the sum times round(q_last / f), rescale.  Output
 *   slot s holds the mean of input slots s-f+1..s; scale unchanged.  Needs the Galois
 *   keys of -1..-(f-1).  Errors: CTL_ELEVEL, CTL_EINVAL (f = 0 or f > N/2), CTL_EKEY.
 * ctl_eval_conv1d: packed single-input single-output convolution with filter w[f] and
 *   "same" zero padding on an input of length n held as [x, x] at block stride t (slots
 *   [0, n) and [t, t+n), zeros elsewhere; n + (f-1)/2 <= t keeps the padding):
 *   out = sum_{i<f} pt_i o rot_{i-h}(x) (+ bias), h = (f-1)/2, then rescale, with pt_i
 *   holding w[i] in the slots s < 2t with (s mod t) < n, encoded at q_last * Delta / scale
 *   (the output carries Delta).  Output slot s < n holds sum_i w[i] x[s+i-h], repeated at
 *   t + s.  f plaintext products, f-1 rotations (hoisted), depth 1.  bias (nullable) has
 *   n values.  Needs the Galois keys of i-h, i != h.  Errors: CTL_EINVAL (shape),
 *   CTL_ELEVEL, CTL_EKEY.
 * ctl_eval_conv1d_coeffs: the same with the f plaintexts given as integer coefficients
 *   pts[f][N] (and bias as coefficients, nullable) at pt_scale.
 * ------------------------------------------------------------------------------- */
int ctl_eval_mul(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* a, const ctl_ct* b, ctl_ct** out);
int ctl_mul_const(ctl_context* ctx, const ctl_ct* in, int64_t c, double c_scale, ctl_ct** out);
int ctl_add_const(ctl_context* ctx, const ctl_ct* in, int64_t c, ctl_ct** out);
int ctl_drop_level(ctl_context* ctx, const ctl_ct* in, uint32_t level, ctl_ct** out);
int ctl_eval_poly3(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const double* a, ctl_ct** out);
int ctl_eval_avgpool(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, uint32_t f, ctl_ct** out);
int ctl_eval_conv1d(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const double* w, uint32_t f, uint32_t n,
                    uint32_t t, const double* bias, ctl_ct** out);
int ctl_eval_conv1d_coeffs(ctl_context* ctx, const ctl_keys* keys, const ctl_ct* in, const int64_t* pts, uint32_t f,
                           const int64_t* bias, double pt_scale, ctl_ct** out);

/* ---------------------------------------------------------------------------------
 * Transform access.  ctl_ntt_dev computes, for n_polys polys of `limbs` limbs each
 * ([n_polys][limbs][N] words, limb l taken modulo prime l of the chain q_0..q_{n_q-1},
 * p_0..), the negacyclic NTT a_hat[k] = a(psi^(2*bitrev(k)+1)) (psi the smallest
 * primitive 2N-th root of unity; bit-reversed order) or, with inverse != 0, its inverse.
 * in_dev and out_dev are device pointers (they may be equal); inputs must be reduced.
 * Ordered on the context stream; does not synchronise.
 * Errors: CTL_EINVAL (limbs > n_q + n_p, null pointer).
 * ------------------------------------------------------------------------------- */
int ctl_ntt_dev(ctl_context* ctx, const uint64_t* in_dev, uint64_t* out_dev, uint32_t n_polys, uint32_t limbs,
                int inverse);

/* ---------------------------------------------------------------------------------
 * Rescale with no device allocation (no counterpart in the paper: a deployment aid).
 * For callers that must not allocate device memory while they run -- a host framework
 * that already owns the device's memory through its own arena, or a latency-critical
 * serving thread where an allocation could stall or fail mid-request.  Same arithmetic
 * as ctl_rescale, on the caller's device buffers: in_dev holds `count` ciphertexts
 * [count][2][level][N] in NTT form (as ctl_ntt_dev produces them, limb l modulo q_l),
 * out_dev receives [count][2][level-1][N], also NTT form.  The only scratch space used
 * is a fixed array compiled into the library (ctl_rescale_static_capacity_words()
 * 64-bit words = 4 MiB, held on every GPU that loads the library until the process
 * exits); count * 2 * N must not exceed it (else CTL_EINVAL, with the limit in
 * ctl_last_error()).  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before any
 * stream capture.  All calls share the one array: calls whose GPU work overlaps (on
 * different streams or contexts of the same device) race and corrupt each other;
 * order them on one stream.  Nothing in the array needs to start at zero.  Work is
 * ordered on the context stream; the call does not synchronise.  Keep kernel timing
 * (ctl_stats_enable_timing) off around it: timing records CUDA events from a pool.
 * Errors: CTL_EINVAL, CTL_ELEVEL (level < 2), CTL_ECUDA.
 * ------------------------------------------------------------------------------- */
int ctl_rescale_static_dev(ctl_context* ctx, const uint64_t* in_dev, uint64_t* out_dev, uint32_t count,
                           uint32_t level);
size_t ctl_rescale_static_capacity_words(void);

/* ---------------------------------------------------------------------------------
 * Models: the frozen server layers of Fig. alg:cryptotl (M_S), encoded once.
 * A layer is CTL_LAYER_DENSE (W m x n, optional bias, optional injected coefficients
 * pt_coeffs[t][N]), CTL_LAYER_SQUARE, CTL_LAYER_REPLICATE (t = rep_t),
 * CTL_LAYER_CONV1D (filter W[m], f = m, input length n, block stride t = rep_t, optional
 * bias[n], optional injected pt_coeffs[f][N]; as ctl_eval_conv1d), CTL_LAYER_POLY3 (W =
 * the four coefficients a0..a3; as ctl_eval_poly3, two levels) or CTL_LAYER_AVGPOOL
 * (size f = m; as ctl_eval_avgpool).  The model is
 * built for ciphertexts entering at in_level with scale in_scale; the diagonals of each
 * dense layer are encoded at the level and scale that layer will see.
 * ctl_model_forward runs ClassifyHE on a batch of ciphertexts under one key set.
 * ctl_model_rotations lists the rotations the model needs (for ctl_keygen).
 * ------------------------------------------------------------------------------- */
#define CTL_LAYER_DENSE 1
#define CTL_LAYER_SQUARE 2
#define CTL_LAYER_REPLICATE 3
#define CTL_LAYER_CONV1D 4
#define CTL_LAYER_POLY3 5
#define CTL_LAYER_AVGPOOL 6
typedef struct ctl_layer {
  int32_t kind;
  uint32_t m, n;              /* dense: output and input dimensions                 */
  const double* W;            /* dense: m x n row-major (nullable if pt_coeffs);
                                 conv1d: filter[m]; poly3: a0..a3                  */
  const double* bias;         /* dense: m values or NULL                            */
  const int64_t* pt_coeffs;   /* dense: injected diagonal coefficients [t][N] or NULL */
  uint32_t rep_t;             /* replicate: shift t                                 */
} ctl_layer;

int ctl_model_create(ctl_context* ctx, const ctl_layer* layers, uint32_t n_layers, uint32_t in_level, double in_scale,
                     ctl_model** out);
void ctl_model_destroy(ctl_model* model);
/* Writes up to cap distinct rotation amounts to rot and their number to *n_rot. */
int ctl_model_rotations(const ctl_model* model, int32_t* rot, uint32_t cap, uint32_t* n_rot);
int ctl_model_forward(ctl_context* ctx, const ctl_model* model, const ctl_keys* keys, const ctl_ct* in, ctl_ct** out);
/* The same forward, bit for bit, replayed from a CUDA graph.  The first call for a given
 * (ctx, keys, batch size) runs the forward once eagerly, then captures the whole layer
 * sequence (kernels, stream-ordered temporary allocations, copies) into a graph with
 * fixed staging buffers; later calls copy the input into the staging buffer, replay the
 * graph and copy the result out, with one launch instead of several hundred.  Calls
 * for the same (ctx, model) must not overlap.  A batch of 8 ciphertexts or more is
 * captured as two halves on concurrent branches of the graph, the second half on the
 * stream of a context clone that the graph keeps (same result: the ciphertexts of a batch
 * are independent; the halves' launches overlap on the device, and their temporaries are
 * live at the same time).  Needs the library's own allocator (CTL_ENOTSUP after
 * ctl_set_allocator).  Graph memory and the clone are released by ctl_model_destroy,
 * which must come before ctl_context_destroy of ctx. */
int ctl_model_forward_graph(ctl_context* ctx, const ctl_model* model, const ctl_keys* keys, const ctl_ct* in,
                            ctl_ct** out);
/* Several groups of queries in one launch (configuration 4's uneven batch: mixed ring
 * degrees, depths and layer shapes; each query is one ClassifyHE call of Fig. alg:cryptotl).
 * Group i has its own context ctxs[i] (ring, primes, stream), model models[i], keys keys[i]
 * and a batch of counts[i] ciphertexts.  ctl_multi_create runs each group once eagerly on
 * zero inputs, then captures all groups' forwards as branches of ONE CUDA graph: the first
 * context's stream forks to every group's stream, each branch is that group's whole layer
 * sequence, and the branches join back; groups on distinct streams (e.g. context clones,
 * one per group) run concurrently when the graph is replayed.  ctl_multi_forward takes one
 * input batch per group (matching count, level and scale), launches the graph once on
 * ctxs[0]'s stream and returns one output per group; every group's stream is ordered after
 * that work.  Each output equals ctl_model_forward of its group alone, bit for bit.  The
 * contexts, models and keys must outlive the handle; ctl_multi_destroy releases the graph
 * and its staging buffers.  Needs the library's own allocator.  Errors: CTL_EINVAL,
 * CTL_ENOMEM, CTL_ECUDA (and the errors of the groups' forwards at creation). */
int ctl_multi_create(uint32_t n, ctl_context* const* ctxs, const ctl_model* const* models, const ctl_keys* const* keys,
                     const uint32_t* counts, ctl_multi** out);
int ctl_multi_forward(ctl_multi* multi, const ctl_ct* const* in, ctl_ct** out);
void ctl_multi_destroy(ctl_multi* multi);

/* Output level and scale of the model. */
int ctl_model_info(const ctl_model* model, uint32_t* out_level, double* out_scale, uint64_t* bytes);

/* ---------------------------------------------------------------------------------
 * Context clones: same parameters and device tables, own stream.  Keys and models made
 * with the original may be used with a clone, so one parameter set can run on several
 * streams at once.  Destroy clones (ctl_context_destroy) before the original.
 * ------------------------------------------------------------------------------- */
int ctl_context_clone(const ctl_context* ctx, ctl_context** out);

/* ---------------------------------------------------------------------------------
 * Serving (Fig. alg:cryptotl: each client query is one ClassifyHE call).  A server has
 * lanes (context + model, added before start) and clients (key set bound to a lane, kept
 * resident).  ctl_server_submit copies one ciphertext (coefficient form, [2][L][N] at
 * the lane's top level) and returns a request id, or CTL_EBUSY when max_queue requests
 * wait.  n_workers threads, each with its own stream per lane, repeatedly take the oldest
 * request, batch it with up to max_batch-1 other queued requests of the same client,
 * admit the batch when its device-memory estimate fits under mem_budget_bytes (a batch
 * of one always runs when nothing else is in flight), and run import -> forward ->
 * export.  So requests arriving while others run are admitted as memory frees up, and
 * different clients' batches overlap on the device.  ctl_server_poll returns CTL_OK
 * with the result ([2][out_level][N]) and the request's latency (submit to completion),
 * CTL_EBUSY while pending, or the negative code the request failed with (the server keeps
 * serving).  ctl_server_wait blocks up to timeout_ms (then CTL_ETIMEOUT).
 * ctl_server_stats: counts6 = submitted, completed, rejected, failed, batches, batched
 * ciphertexts; latency percentiles in ms over completed requests.
 * ------------------------------------------------------------------------------- */
int ctl_server_create(ctl_server** out, uint64_t mem_budget_bytes, uint32_t n_workers, uint32_t max_batch,
                      uint32_t max_queue);
int ctl_server_add_lane(ctl_server* srv, ctl_context* ctx, const ctl_model* model, uint32_t* lane);
int ctl_server_add_client(ctl_server* srv, uint32_t lane, const ctl_keys* keys, uint32_t* client);
int ctl_server_io_words(const ctl_server* srv, uint32_t client, size_t* in_words, size_t* out_words);
int ctl_server_start(ctl_server* srv);
int ctl_server_submit(ctl_server* srv, uint32_t client, const uint64_t* ct_coeffs, uint64_t* request);
int ctl_server_poll(ctl_server* srv, uint64_t request, uint64_t* out, size_t cap, double* latency_ms);
int ctl_server_wait(ctl_server* srv, uint64_t request, uint32_t timeout_ms, uint64_t* out, size_t cap,
                    double* latency_ms);
int ctl_server_stats(ctl_server* srv, uint64_t* counts6, double* p50_ms, double* p99_ms);
/* Memory admission of the server: the device-memory estimate per in-flight ciphertext of
 * the client's lane (a batch of n reserves n times it, and is admitted only while the
 * reservations of running batches plus its own stay within mem_budget_bytes; a batch of
 * one runs even above the budget when nothing else runs), the highest total reservation
 * so far, and how often a worker found requests queued but had to wait for memory. */
int ctl_server_admission(ctl_server* srv, uint32_t client, uint64_t* bytes_per_ct, uint64_t* peak_reserved,
                         uint64_t* deferred);
/* Stops the workers (queued requests are dropped) and releases the server. */
void ctl_server_destroy(ctl_server* srv);

/* Microbenchmark of the integer work units the roofline counts, on the current device:
 * writes units per clock per SM (at the device's maximum SM clock) of kind 0 = 64-bit
 * Shoup modular multiplication, 1 = Harvey butterfly, 2 = three-high-half Shoup product,
 * 3 = split-half multiply-accumulate (four 32x32->64 multiply-adds).  Synchronous; tens of
 * milliseconds.  Errors: CTL_EINVAL, CTL_ENOMEM, CTL_ECUDA. */
int ctl_microbench_unit_rate(int kind, double* per_clk_sm);

/* Evaluates one of the kernels' modular-arithmetic primitives (the word-size residue
 * arithmetic of Sec. 3.1's RNS representation) on n host values x, on the current
 * device, writing n results to host out.  Synchronous; allocates 16n bytes of device
 * memory for the call.  kind:
 *   0 shoup(x, w, wsh, q)      = x*w mod q in [0, q) for any 64-bit x, wsh = floor(w 2^64 / q);
 *   1 shoup_lazy(x, w, wsh, q) = x*w mod q plus 0 or q, in [0, 2q);
 *   2 shoup_small(x, w, wsh, q): x*w mod q plus a multiple of q, in [0, 4q);
 *   3 reduce_wide(x, q, aux)   = x mod q for x < 2^63, 2^32 < q, aux = floor(2^64 / q);
 *   4 mulmod_mont(x, w, q, aux) = x * w * 2^-64 mod q for any 64-bit x, w < q,
 *                                 aux = q^-1 mod 2^64;
 *   5 reduce4(x, q)            = x mod q for x < 4q.
 * Errors: CTL_EINVAL, CTL_ENOMEM, CTL_ECUDA. */
int ctl_modarith_eval(int kind, const uint64_t* x, size_t n, uint64_t w, uint64_t wsh, uint64_t q, uint64_t aux,
                      uint64_t* out);

/* ---------------------------------------------------------------------------------
 * Statistics: kernel launches since the last reset, homomorphic operation counters
 * (rotations, plaintext products, additions, relinearisations, rescales), and, when
 * timing is enabled, per-kernel-class device milliseconds and launch counts measured
 * with CUDA events on the context stream.  Class names: ctl_stats_class_name(i).
 * ------------------------------------------------------------------------------- */
int ctl_stats_reset(ctl_context* ctx);
int ctl_stats_enable_timing(ctl_context* ctx, int enable);
uint64_t ctl_stats_launches(const ctl_context* ctx);
int ctl_stats_ops(const ctl_context* ctx, uint64_t* ops5);
int ctl_stats_kernel_classes(void);
const char* ctl_stats_class_name(int i);
/* Collects pending event timings (synchronises) and writes ms[i], launches[i] and the
 * algorithmic modular multiplications work[i] of each class i. */
int ctl_stats_kernels(ctl_context* ctx, double* ms, uint64_t* launches, double* work);
/* Writes bytes[i], the algorithmic HBM bytes of class i since the last reset (every
 * operand of a launch read once and every result written once), for the HBM side of the
 * per-class rooflines.  Counted while timing is enabled, like work[i]. */
int ctl_stats_kernel_bytes(const ctl_context* ctx, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* CTL_H */
