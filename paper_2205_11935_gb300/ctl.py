"""ctypes binding of the ctl C-ABI (include/ctl.h): argument marshalling only.

Every ``ctl_*`` function of the header is available under the same name on the
loaded library (``lib()``); the small classes below only convert numpy arrays and
raise ``CtlError`` on negative return codes.  All homomorphic work runs in the CUDA
library; nothing here computes on ciphertexts.  If the compiled library is missing the
import fails loudly (there is no CPU fallback).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libctl.so")

CTL_LAYER_DENSE, CTL_LAYER_SQUARE, CTL_LAYER_REPLICATE = 1, 2, 3
CTL_LAYER_CONV1D, CTL_LAYER_POLY3, CTL_LAYER_AVGPOOL = 4, 5, 6
ERRORS = {-1: "EINVAL", -2: "ELEVEL", -3: "ESCALE", -4: "EKEY", -5: "ENOMEM", -6: "ECUDA", -7: "ETIMEOUT",
          -8: "EBUSY", -9: "ENOTSUP"}


class CtlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Layer(C.Structure):
    _fields_ = [("kind", C.c_int32), ("m", C.c_uint32), ("n", C.c_uint32), ("W", C.POINTER(C.c_double)),
                ("bias", C.POINTER(C.c_double)), ("pt_coeffs", C.POINTER(C.c_int64)), ("rep_t", C.c_uint32)]


_vp = C.c_void_p
_pp = C.POINTER(C.c_void_p)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)
_sz = C.c_size_t

SIGNATURES = {
    "ctl_last_error": (C.c_char_p, []),
    "ctl_version": (C.c_char_p, []),
    "ctl_plan_primes": (C.c_int, [C.c_uint32, _u32p, C.c_uint32, _u64p]),
    "ctl_context_create": (C.c_int, [_pp, C.c_uint32, _u32p, C.c_uint32, _u32p, C.c_uint32, C.c_uint32, C.c_double,
                                     C.c_uint64]),
    "ctl_context_destroy": (None, [_vp]),
    "ctl_context_info": (C.c_int, [_vp, _u64p, _u32p, _u32p, _u32p]),
    "ctl_set_stream": (C.c_int, [_vp, _vp]),
    "ctl_set_allocator": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ctl_set_dense_mode": (C.c_int, [_vp, C.c_int]),
    "ctl_set_ntt_shape": (C.c_int, [_vp, C.c_int, C.c_int]),
    "ctl_get_ntt_shape": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ctl_set_bsgs_shape": (C.c_int, [_vp, C.c_int, C.c_int]),
    "ctl_set_keyswitch_budget": (C.c_int, [_vp, C.c_uint64]),
    "ctl_set_windows": (C.c_int, [_vp, C.c_uint32]),
    "ctl_autotune_ntt": (C.c_int, [_vp, C.c_uint32, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ctl_synchronize": (C.c_int, [_vp]),
    "ctl_keygen": (C.c_int, [_vp, _i32p, C.c_uint32, C.c_uint64, _pp]),
    "ctl_keys_destroy": (None, [_vp]),
    "ctl_keys_export": (C.c_int, [_vp, C.c_uint64, _u64p, _sz]),
    "ctl_keys_create": (C.c_int, [_vp, _pp]),
    "ctl_keys_import": (C.c_int, [_vp, C.c_uint64, _u64p, _sz]),
    "ctl_galois_element": (C.c_uint64, [_vp, C.c_int64]),
    "ctl_encode": (C.c_int, [_vp, _dp, _sz, C.c_double, _i64p]),
    "ctl_decode": (C.c_int, [_vp, _dp, _sz, C.c_double, _dp]),
    "ctl_encrypt": (C.c_int, [_vp, _vp, _dp, _sz, C.c_uint64, _pp]),
    "ctl_encrypt_coeffs": (C.c_int, [_vp, _vp, _i64p, C.c_uint64, _pp]),
    "ctl_decrypt": (C.c_int, [_vp, _vp, _vp, _dp, _sz]),
    "ctl_decrypt_coeffs": (C.c_int, [_vp, _vp, _vp, _dp]),
    "ctl_ct_import": (C.c_int, [_vp, _u64p, C.c_uint32, C.c_uint32, C.c_double, _pp]),
    "ctl_ct_export": (C.c_int, [_vp, _u64p, _sz]),
    "ctl_ct_import_dev": (C.c_int, [_vp, _vp, C.c_uint32, C.c_uint32, C.c_double, _pp]),
    "ctl_ct_export_dev": (C.c_int, [_vp, _vp, _sz]),
    "ctl_ct_info": (C.c_int, [_vp, _u32p, _u32p, _dp]),
    "ctl_ct_concat": (C.c_int, [_vp, _pp, _sz, _pp]),
    "ctl_ct_slice": (C.c_int, [_vp, C.c_uint32, _pp]),
    "ctl_ct_destroy": (None, [_vp]),
    "ctl_rotate": (C.c_int, [_vp, _vp, _vp, C.c_int32, _pp]),
    "ctl_rescale": (C.c_int, [_vp, _vp, _pp]),
    "ctl_eval_square": (C.c_int, [_vp, _vp, _vp, _pp]),
    "ctl_eval_dense": (C.c_int, [_vp, _vp, _vp, _dp, C.c_uint32, C.c_uint32, _dp, _pp]),
    "ctl_eval_dense_coeffs": (C.c_int, [_vp, _vp, _vp, _i64p, C.c_uint32, _i64p, C.c_double, _pp]),
    "ctl_eval_dense_rect": (C.c_int, [_vp, _vp, _vp, _dp, C.c_uint32, C.c_uint32, _dp, C.c_int, _pp]),
    "ctl_eval_dense_rect_coeffs": (C.c_int, [_vp, _vp, _vp, _i64p, C.c_uint32, C.c_uint32, _i64p, C.c_double,
                                             C.c_int, _pp]),
    "ctl_replicate": (C.c_int, [_vp, _vp, _vp, C.c_uint32, _pp]),
    "ctl_add": (C.c_int, [_vp, _vp, _vp, _pp]),
    "ctl_mul_plain_coeffs": (C.c_int, [_vp, _vp, _i64p, C.c_double, _pp]),
    "ctl_eval_mul": (C.c_int, [_vp, _vp, _vp, _vp, _pp]),
    "ctl_mul_const": (C.c_int, [_vp, _vp, C.c_int64, C.c_double, _pp]),
    "ctl_add_const": (C.c_int, [_vp, _vp, C.c_int64, _pp]),
    "ctl_drop_level": (C.c_int, [_vp, _vp, C.c_uint32, _pp]),
    "ctl_eval_poly3": (C.c_int, [_vp, _vp, _vp, _dp, _pp]),
    "ctl_eval_avgpool": (C.c_int, [_vp, _vp, _vp, C.c_uint32, _pp]),
    "ctl_eval_conv1d": (C.c_int, [_vp, _vp, _vp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, _dp, _pp]),
    "ctl_eval_conv1d_coeffs": (C.c_int, [_vp, _vp, _vp, _i64p, C.c_uint32, _i64p, C.c_double, _pp]),
    "ctl_ntt_dev": (C.c_int, [_vp, _vp, _vp, C.c_uint32, C.c_uint32, C.c_int]),
    "ctl_serialized_size": (C.c_size_t, [C.c_uint32, _u64p, C.c_uint32, C.c_int]),
    "ctl_encode_residues": (C.c_int, [C.c_uint32, _u64p, C.c_uint32, _dp, _sz, C.c_double, _u64p]),
    "ctl_key_message_size": (C.c_size_t, [C.c_uint32, _u64p, C.c_uint32, C.c_uint32, C.c_int]),
    "ctl_serialize_key": (C.c_int, [C.c_uint32, _u64p, C.c_uint32, C.c_uint32, C.c_uint64, _u64p, C.c_int,
                                    C.c_uint64, C.POINTER(C.c_uint8), _sz, C.POINTER(C.c_size_t)]),
    "ctl_deserialize_key": (C.c_int, [C.POINTER(C.c_uint8), _sz, C.c_uint32, _u64p, C.c_uint32, C.c_uint32, _u64p,
                                      _sz, _u64p]),
    "ctl_serialize": (C.c_int, [C.c_uint32, _u64p, C.c_uint32, _u64p, C.c_int, C.c_uint64, C.POINTER(C.c_uint8),
                                _sz, C.POINTER(C.c_size_t)]),
    "ctl_deserialize": (C.c_int, [C.POINTER(C.c_uint8), _sz, C.c_uint32, _u64p, C.c_uint32, _u64p, _sz, _u32p]),
    "ctl_rescale_static_dev": (C.c_int, [_vp, _vp, _vp, C.c_uint32, C.c_uint32]),
    "ctl_rescale_static_capacity_words": (C.c_size_t, []),
    "ctl_model_create": (C.c_int, [_vp, C.POINTER(Layer), C.c_uint32, C.c_uint32, C.c_double, _pp]),
    "ctl_model_destroy": (None, [_vp]),
    "ctl_model_rotations": (C.c_int, [_vp, _i32p, C.c_uint32, _u32p]),
    "ctl_model_forward": (C.c_int, [_vp, _vp, _vp, _vp, _pp]),
    "ctl_model_forward_graph": (C.c_int, [_vp, _vp, _vp, _vp, _pp]),
    "ctl_model_info": (C.c_int, [_vp, _u32p, _dp, _u64p]),
    "ctl_multi_create": (C.c_int, [C.c_uint32, _pp, _pp, _pp, _u32p, _pp]),
    "ctl_multi_forward": (C.c_int, [_vp, _pp, _pp]),
    "ctl_multi_destroy": (None, [_vp]),
    "ctl_context_clone": (C.c_int, [_vp, _pp]),
    "ctl_server_create": (C.c_int, [_pp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]),
    "ctl_server_add_lane": (C.c_int, [_vp, _vp, _vp, _u32p]),
    "ctl_server_add_client": (C.c_int, [_vp, C.c_uint32, _vp, _u32p]),
    "ctl_server_io_words": (C.c_int, [_vp, C.c_uint32, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "ctl_server_start": (C.c_int, [_vp]),
    "ctl_server_submit": (C.c_int, [_vp, C.c_uint32, _u64p, _u64p]),
    "ctl_server_poll": (C.c_int, [_vp, C.c_uint64, _u64p, _sz, _dp]),
    "ctl_server_wait": (C.c_int, [_vp, C.c_uint64, C.c_uint32, _u64p, _sz, _dp]),
    "ctl_server_stats": (C.c_int, [_vp, _u64p, _dp, _dp]),
    "ctl_server_admission": (C.c_int, [_vp, C.c_uint32, _u64p, _u64p, _u64p]),
    "ctl_server_destroy": (None, [_vp]),
    "ctl_microbench_unit_rate": (C.c_int, [C.c_int, _dp]),
    "ctl_encode_dev": (C.c_int, [_vp, _vp, _sz, C.c_uint32, C.c_double, _vp]),
    "ctl_decode_dev": (C.c_int, [_vp, _vp, C.c_uint32, _sz, C.c_double, _vp]),
    "ctl_encrypt_coeffs_dev": (C.c_int, [_vp, _vp, _vp, C.c_uint32, _u64p, _pp]),
    "ctl_encrypt_dev": (C.c_int, [_vp, _vp, _vp, _sz, C.c_uint32, _u64p, _pp]),
    "ctl_decrypt_coeffs_dev": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ctl_decrypt_dev": (C.c_int, [_vp, _vp, _vp, _sz, _vp]),
    "ctl_modarith_eval": (C.c_int, [C.c_int, _u64p, _sz, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, _u64p]),
    "ctl_stats_reset": (C.c_int, [_vp]),
    "ctl_stats_enable_timing": (C.c_int, [_vp, C.c_int]),
    "ctl_stats_launches": (C.c_uint64, [_vp]),
    "ctl_stats_ops": (C.c_int, [_vp, _u64p]),
    "ctl_stats_kernel_classes": (C.c_int, []),
    "ctl_stats_class_name": (C.c_char_p, [C.c_int]),
    "ctl_stats_kernels": (C.c_int, [_vp, _dp, _u64p, _dp]),
    "ctl_stats_kernel_bytes": (C.c_int, [_vp, _dp]),
}

_LIB = None


def lib():
    """Load libctl.so (built by ``paper_2205_11935_gb300.build``); raises if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2205_11935_gb300/build.py)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc):
    if rc != 0:
        raise CtlError(rc, lib().ctl_last_error().decode())


def _p(a, t):
    return a.ctypes.data_as(t)


def microbench_unit_rate(kind):
    """Units per clock per SM of kind 0 = Shoup modmul, 1 = Harvey butterfly, 2 = three-high-half
    Shoup product, 3 = split-half multiply-accumulate (ctl_microbench_unit_rate)."""
    v = C.c_double()
    _check(lib().ctl_microbench_unit_rate(int(kind), C.byref(v)))
    return v.value


def modarith_eval(kind, x, q, w=0, wsh=0, aux=0):
    """One modular-arithmetic primitive of the kernels evaluated on the device over the
    values x (ctl_modarith_eval); returns a uint64 array."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros_like(x)
    _check(lib().ctl_modarith_eval(int(kind), _p(x, _u64p), x.size, int(w), int(wsh), int(q), int(aux),
                                   _p(out, _u64p)))
    return out


def plan_primes(N, bits):
    b = np.asarray(bits, dtype=np.uint32)
    out = np.zeros(len(b), dtype=np.uint64)
    _check(lib().ctl_plan_primes(N, _p(b, _u32p), len(b), _p(out, _u64p)))
    return [int(x) for x in out]


def serialize(N, moduli, coeffs, seed=None):
    """Message bytes of a coefficient-form ciphertext [2][level][N]; with seed, the seeded
    form (c0 and the seed; valid for a fresh encryption with that seed)."""
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    a = np.ascontiguousarray(coeffs, dtype=np.uint64)
    level = a.shape[-2]
    seeded = 0 if seed is None else 1
    n = lib().ctl_serialized_size(N, _p(m, _u64p), level, seeded)
    out = np.zeros(n, dtype=np.uint8)
    size = C.c_size_t()
    _check(lib().ctl_serialize(N, _p(m, _u64p), level, _p(a, _u64p), seeded, 0 if seed is None else int(seed),
                               _p(out, C.POINTER(C.c_uint8)), n, C.byref(size)))
    return out.tobytes()


def encode_residues(N, moduli, x, scale):
    """Slot values encoded at any scale, as residues [len(moduli)][N] (host only)."""
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((len(m), N), dtype=np.uint64)
    _check(lib().ctl_encode_residues(N, _p(m, _u64p), len(m), _p(x, _dp), len(x), float(scale), _p(out, _u64p)))
    return out


def serialize_key(N, moduli, key_id, coeffs, seed=None):
    """Message bytes of a key [beta][2][limbs][N] (coefficient form, as Keys.export returns);
    with seed (the ctl_keygen seed), the seeded form that omits the a parts."""
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    a = np.ascontiguousarray(coeffs, dtype=np.uint64)
    beta, _, limbs, _ = a.shape
    seeded = 0 if seed is None else 1
    n = lib().ctl_key_message_size(N, _p(m, _u64p), limbs, beta, seeded)
    out = np.zeros(n, dtype=np.uint8)
    _check(lib().ctl_serialize_key(N, _p(m, _u64p), limbs, beta, int(key_id), _p(a, _u64p), seeded,
                                   0 if seed is None else int(seed), _p(out, C.POINTER(C.c_uint8)), n, None))
    return out.tobytes()


def deserialize_key(msg, N, moduli, beta):
    """(key id, key [beta][2][limbs][N]) of a key message."""
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    b = np.frombuffer(bytes(msg), dtype=np.uint8).copy()
    out = np.zeros((beta, 2, len(m), N), dtype=np.uint64)
    kid = C.c_uint64()
    _check(lib().ctl_deserialize_key(_p(b, C.POINTER(C.c_uint8)), len(b), N, _p(m, _u64p), len(m), beta,
                                     _p(out, _u64p), out.size, C.byref(kid)))
    return kid.value, out


def deserialize(msg, N, moduli):
    """Coefficient-form ciphertext [2][level][N] of a message."""
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    b = np.frombuffer(bytes(msg), dtype=np.uint8).copy()
    out = np.zeros(2 * len(m) * N, dtype=np.uint64)
    lvl = C.c_uint32()
    _check(lib().ctl_deserialize(_p(b, C.POINTER(C.c_uint8)), len(b), N, _p(m, _u64p), len(m), _p(out, _u64p),
                                 out.size, C.byref(lvl)))
    return out[:2 * lvl.value * N].reshape(2, lvl.value, N)


class Context:
    def __init__(self, N, q_bits, p_bits, dnum=None, scale=2.0 ** 40, seed=0, stream=None):
        L = lib()
        qb = np.asarray(q_bits, dtype=np.uint32)
        pb = np.asarray(p_bits, dtype=np.uint32)
        dnum = len(qb) if dnum is None else dnum
        h = C.c_void_p()
        _check(L.ctl_context_create(C.byref(h), N, _p(qb, _u32p), len(qb), _p(pb, _u32p), len(pb), dnum, scale, seed))
        self.h = h
        self.N, self.L, self.K, self.scale = N, len(qb), len(pb), scale
        mods = np.zeros(self.L + self.K, dtype=np.uint64)
        a = C.c_uint32()
        _check(L.ctl_context_info(h, _p(mods, _u64p), None, None, C.byref(a)))
        self.moduli = [int(x) for x in mods]
        self.alpha = a.value
        self.beta = (self.L + self.alpha - 1) // self.alpha
        if stream is not None:
            self.set_stream(stream)

    DENSE_COMPOSED = 0
    DENSE_LAZY_MODDOWN = 1
    DENSE_RECT = 2
    DENSE_RECT_LAZY = 3

    def set_dense_mode(self, mode):
        """Dense layers created afterwards: DENSE_COMPOSED (default), DENSE_LAZY_MODDOWN or
        DENSE_RECT (rectangular form for layers whose output side is the shorter)."""
        _check(lib().ctl_set_dense_mode(self.h, int(mode)))

    NTT_R32 = 0
    NTT_R16 = 1

    def set_ntt_shape(self, fwd=-1, inv=-1):
        """Register NTT shapes (NTT_R32 / NTT_R16; -1 keeps the current one)."""
        _check(lib().ctl_set_ntt_shape(self.h, int(fwd), int(inv)))

    def set_bsgs_shape(self, chunk=32, karatsuba=1):
        _check(lib().ctl_set_bsgs_shape(self.h, int(chunk), int(karatsuba)))

    def set_windows(self, p):
        """Prediction windows of 2t slots per ciphertext for layers created afterwards."""
        _check(lib().ctl_set_windows(self.h, int(p)))

    def set_keyswitch_budget(self, nbytes):
        _check(lib().ctl_set_keyswitch_budget(self.h, int(nbytes)))

    def ntt_shape(self):
        f, i = C.c_int(), C.c_int()
        _check(lib().ctl_get_ntt_shape(self.h, C.byref(f), C.byref(i)))
        return f.value, i.value

    def autotune_ntt(self, batch_limbs=0):
        """Re-times both NTT shapes and keeps the faster per direction; returns (fwd, inv)."""
        f, i = C.c_int(), C.c_int()
        _check(lib().ctl_autotune_ntt(self.h, batch_limbs, C.byref(f), C.byref(i)))
        return f.value, i.value

    def set_stream(self, stream_ptr):
        _check(lib().ctl_set_stream(self.h, C.c_void_p(stream_ptr)))

    def clone(self, stream_ptr=None):
        """ctl_context_clone: same parameters and device tables, own stream (close the
        clone before the original)."""
        h = C.c_void_p()
        _check(lib().ctl_context_clone(self.h, C.byref(h)))
        c = object.__new__(Context)
        c.h = h
        c.N, c.L, c.K, c.scale = self.N, self.L, self.K, self.scale
        c.moduli, c.alpha, c.beta = self.moduli, self.alpha, self.beta
        if stream_ptr is not None:
            c.set_stream(stream_ptr)
        return c

    def synchronize(self):
        _check(lib().ctl_synchronize(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().ctl_context_destroy(self.h)
            self.h = None

    def galois_element(self, r):
        return int(lib().ctl_galois_element(self.h, r))

    def keygen(self, rotations=(), seed=3):
        r = np.asarray(list(rotations), dtype=np.int32)
        h = C.c_void_p()
        _check(lib().ctl_keygen(self.h, _p(r, _i32p), len(r), seed, C.byref(h)))
        return Keys(self, h)

    def keys_create(self):
        """An empty key set (no secret) for evaluation keys received from a client."""
        h = C.c_void_p()
        _check(lib().ctl_keys_create(self.h, C.byref(h)))
        return Keys(self, h)

    def encode(self, x, scale=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        m = np.zeros(self.N, dtype=np.int64)
        _check(lib().ctl_encode(self.h, _p(x, _dp), len(x), self.scale if scale is None else scale, _p(m, _i64p)))
        return m

    def decode(self, m, n, scale=None):
        m = np.ascontiguousarray(m, dtype=np.float64)
        y = np.zeros(n, dtype=np.float64)
        _check(lib().ctl_decode(self.h, _p(m, _dp), n, self.scale if scale is None else scale, _p(y, _dp)))
        return y

    def encrypt(self, keys, x, seed):
        x = np.ascontiguousarray(x, dtype=np.float64)
        h = C.c_void_p()
        _check(lib().ctl_encrypt(self.h, keys.h, _p(x, _dp), len(x), seed, C.byref(h)))
        return Ciphertext(self, h)

    def encrypt_coeffs(self, keys, m, seed):
        m = np.ascontiguousarray(m, dtype=np.int64)
        h = C.c_void_p()
        _check(lib().ctl_encrypt_coeffs(self.h, keys.h, _p(m, _i64p), seed, C.byref(h)))
        return Ciphertext(self, h)

    def decrypt(self, keys, ct, n):
        y = np.zeros(n, dtype=np.float64)
        _check(lib().ctl_decrypt(self.h, keys.h, ct.h, _p(y, _dp), n))
        return y

    def decrypt_coeffs(self, keys, ct):
        m = np.zeros(self.N, dtype=np.float64)
        _check(lib().ctl_decrypt_coeffs(self.h, keys.h, ct.h, _p(m, _dp)))
        return m

    # --- the client side on the device (pointers are device addresses, e.g. data_ptr()) ---
    def encode_dev(self, z_ptr, nz, count, m_ptr, scale=None):
        _check(lib().ctl_encode_dev(self.h, C.c_void_p(z_ptr), nz, count, self.scale if scale is None else scale,
                                    C.c_void_p(m_ptr)))

    def decode_dev(self, m_ptr, count, nz, z_ptr, scale=None):
        _check(lib().ctl_decode_dev(self.h, C.c_void_p(m_ptr), count, nz, self.scale if scale is None else scale,
                                    C.c_void_p(z_ptr)))

    def encrypt_coeffs_dev(self, keys, m_ptr, count, seeds):
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        h = C.c_void_p()
        _check(lib().ctl_encrypt_coeffs_dev(self.h, keys.h, C.c_void_p(m_ptr), count, _p(sd, _u64p), C.byref(h)))
        return Ciphertext(self, h)

    def encrypt_dev(self, keys, z_ptr, nz, count, seeds):
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        h = C.c_void_p()
        _check(lib().ctl_encrypt_dev(self.h, keys.h, C.c_void_p(z_ptr), nz, count, _p(sd, _u64p), C.byref(h)))
        return Ciphertext(self, h)

    def decrypt_coeffs_dev(self, keys, ct, m_ptr):
        _check(lib().ctl_decrypt_coeffs_dev(self.h, keys.h, ct.h, C.c_void_p(m_ptr)))

    def decrypt_dev(self, keys, ct, nz, z_ptr):
        _check(lib().ctl_decrypt_dev(self.h, keys.h, ct.h, nz, C.c_void_p(z_ptr)))

    def ct_import(self, coeffs, scale):
        a = np.ascontiguousarray(coeffs, dtype=np.uint64)
        if a.ndim == 3:
            a = a[None]
        count, _, level, _ = a.shape
        h = C.c_void_p()
        _check(lib().ctl_ct_import(self.h, _p(a, _u64p), count, level, scale, C.byref(h)))
        return Ciphertext(self, h)

    def concat(self, cts):
        arr = (C.c_void_p * len(cts))(*[c.h.value for c in cts])
        h = C.c_void_p()
        _check(lib().ctl_ct_concat(self.h, C.cast(arr, _pp), len(cts), C.byref(h)))
        return Ciphertext(self, h)

    # --- operations -------------------------------------------------------------
    def _op(self, fn, *args):
        h = C.c_void_p()
        _check(fn(*args, C.byref(h)))
        return Ciphertext(self, h)

    def rotate(self, keys, ct, r):
        return self._op(lib().ctl_rotate, self.h, keys.h, ct.h, r)

    def rescale(self, ct):
        return self._op(lib().ctl_rescale, self.h, ct.h)

    def square(self, keys, ct):
        return self._op(lib().ctl_eval_square, self.h, keys.h, ct.h)

    def dense(self, keys, ct, W, bias=None):
        W = np.ascontiguousarray(W, dtype=np.float64)
        m, n = W.shape
        bp = _p(np.ascontiguousarray(bias, dtype=np.float64), _dp) if bias is not None else None
        return self._op(lib().ctl_eval_dense, self.h, keys.h, ct.h, _p(W, _dp), m, n, bp)

    def dense_coeffs(self, keys, ct, pts, pt_scale, bias=None):
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        bp = _p(np.ascontiguousarray(bias, dtype=np.int64), _i64p) if bias is not None else None
        return self._op(lib().ctl_eval_dense_coeffs, self.h, keys.h, ct.h, _p(pts, _i64p), pts.shape[0], bp,
                        pt_scale)

    def replicate(self, keys, ct, t):
        return self._op(lib().ctl_replicate, self.h, keys.h, ct.h, t)

    def dense_rect(self, keys, ct, W, bias=None, fold=2):
        W = np.ascontiguousarray(W, dtype=np.float64)
        m, n = W.shape
        bp = _p(np.ascontiguousarray(bias, dtype=np.float64), _dp) if bias is not None else None
        return self._op(lib().ctl_eval_dense_rect, self.h, keys.h, ct.h, _p(W, _dp), m, n, bp, int(fold))

    def dense_rect_coeffs(self, keys, ct, pts, tn, pt_scale, bias=None, fold=2):
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        bp = _p(np.ascontiguousarray(bias, dtype=np.int64), _i64p) if bias is not None else None
        return self._op(lib().ctl_eval_dense_rect_coeffs, self.h, keys.h, ct.h, _p(pts, _i64p), pts.shape[0], int(tn),
                        bp, pt_scale, int(fold))

    def add(self, a, b):
        return self._op(lib().ctl_add, self.h, a.h, b.h)

    def mul_plain_coeffs(self, ct, pt, pt_scale):
        pt = np.ascontiguousarray(pt, dtype=np.int64)
        return self._op(lib().ctl_mul_plain_coeffs, self.h, ct.h, _p(pt, _i64p), pt_scale)

    def mul(self, keys, a, b):
        """HMult of two ciphertexts: tensor, relinearisation, rescale."""
        return self._op(lib().ctl_eval_mul, self.h, keys.h, a.h, b.h)

    def mul_const(self, ct, c, c_scale):
        return self._op(lib().ctl_mul_const, self.h, ct.h, int(c), float(c_scale))

    def add_const(self, ct, c):
        return self._op(lib().ctl_add_const, self.h, ct.h, int(c))

    def drop_level(self, ct, level):
        return self._op(lib().ctl_drop_level, self.h, ct.h, level)

    def poly3(self, keys, ct, a):
        """a[3] z^3 + a[2] z^2 + a[1] z + a[0] (a = a0..a3) at depth 2."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        return self._op(lib().ctl_eval_poly3, self.h, keys.h, ct.h, _p(a, _dp))

    def avgpool(self, keys, ct, f):
        return self._op(lib().ctl_eval_avgpool, self.h, keys.h, ct.h, f)

    def conv1d(self, keys, ct, w, n, t, bias=None):
        w = np.ascontiguousarray(w, dtype=np.float64)
        bp = _p(np.ascontiguousarray(bias, dtype=np.float64), _dp) if bias is not None else None
        return self._op(lib().ctl_eval_conv1d, self.h, keys.h, ct.h, _p(w, _dp), len(w), n, t, bp)

    def conv1d_coeffs(self, keys, ct, pts, pt_scale, bias=None):
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        bp = _p(np.ascontiguousarray(bias, dtype=np.int64), _i64p) if bias is not None else None
        return self._op(lib().ctl_eval_conv1d_coeffs, self.h, keys.h, ct.h, _p(pts, _i64p), pts.shape[0], bp,
                        pt_scale)

    def ntt_dev(self, in_ptr, out_ptr, n_polys, limbs, inverse=False):
        _check(lib().ctl_ntt_dev(self.h, C.c_void_p(in_ptr), C.c_void_p(out_ptr), n_polys, limbs, 1 if inverse else 0))

    # --- statistics -------------------------------------------------------------
    def stats_reset(self):
        _check(lib().ctl_stats_reset(self.h))

    def stats_enable_timing(self, on=True):
        _check(lib().ctl_stats_enable_timing(self.h, 1 if on else 0))

    def stats_launches(self):
        return int(lib().ctl_stats_launches(self.h))

    def stats_ops(self):
        o = np.zeros(5, dtype=np.uint64)
        _check(lib().ctl_stats_ops(self.h, _p(o, _u64p)))
        return dict(zip(["rotations", "ptmul", "add", "relin", "rescale"], [int(x) for x in o]))

    def stats_kernels(self):
        n = lib().ctl_stats_kernel_classes()
        ms = np.zeros(n)
        la = np.zeros(n, dtype=np.uint64)
        wk = np.zeros(n)
        by = np.zeros(n)
        _check(lib().ctl_stats_kernels(self.h, _p(ms, _dp), _p(la, _u64p), _p(wk, _dp)))
        _check(lib().ctl_stats_kernel_bytes(self.h, _p(by, _dp)))
        return {lib().ctl_stats_class_name(i).decode(): {"ms": float(ms[i]), "launches": int(la[i]),
                                                           "modmul": float(wk[i]), "bytes": float(by[i])}
                for i in range(n)}


class Keys:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def export(self, key_id):
        c = self.ctx
        out = np.zeros((c.beta, 2, c.L + c.K, c.N), dtype=np.uint64)
        _check(lib().ctl_keys_export(self.h, key_id, _p(out, _u64p), out.size))
        return out

    def import_key(self, key_id, coeffs):
        a = np.ascontiguousarray(coeffs, dtype=np.uint64)
        _check(lib().ctl_keys_import(self.h, int(key_id), _p(a, _u64p), a.size))

    def close(self):
        # a handle outlives nothing: once its context is destroyed, the context took its
        # device memory with it and the handle must not be released again
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            lib().ctl_keys_destroy(self.h)
        self.h = None


class Ciphertext:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def info(self):
        lvl, cnt, sc = C.c_uint32(), C.c_uint32(), C.c_double()
        _check(lib().ctl_ct_info(self.h, C.byref(lvl), C.byref(cnt), C.byref(sc)))
        return lvl.value, cnt.value, sc.value

    @property
    def level(self):
        return self.info()[0]

    @property
    def count(self):
        return self.info()[1]

    @property
    def scale(self):
        return self.info()[2]

    def export(self):
        lvl, cnt, _ = self.info()
        out = np.zeros((cnt, 2, lvl, self.ctx.N), dtype=np.uint64)
        _check(lib().ctl_ct_export(self.h, _p(out, _u64p), out.size))
        return out

    def slice(self, i):
        h = C.c_void_p()
        _check(lib().ctl_ct_slice(self.h, i, C.byref(h)))
        return Ciphertext(self.ctx, h)

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            lib().ctl_ct_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """Frozen server layers: list of ("dense", W[, bias][, pt_coeffs]), ("square",), ("replicate", t),
    ("conv1d", w, n, t[, bias][, pt_coeffs]), ("poly3", a0..a3), ("avgpool", f)."""

    def __init__(self, ctx, layers, in_level=None, in_scale=None):
        self.ctx = ctx
        self._keep = []
        arr = (Layer * len(layers))()
        for i, ly in enumerate(layers):
            kind = ly[0]
            if kind == "dense":
                W = np.ascontiguousarray(ly[1], dtype=np.float64)
                self._keep.append(W)
                arr[i].kind = CTL_LAYER_DENSE
                arr[i].m, arr[i].n = W.shape
                arr[i].W = _p(W, _dp)
                if len(ly) > 2 and ly[2] is not None:
                    b = np.ascontiguousarray(ly[2], dtype=np.float64)
                    self._keep.append(b)
                    arr[i].bias = _p(b, _dp)
                if len(ly) > 3 and ly[3] is not None:
                    pc = np.ascontiguousarray(ly[3], dtype=np.int64)
                    self._keep.append(pc)
                    arr[i].pt_coeffs = _p(pc, _i64p)
            elif kind == "square":
                arr[i].kind = CTL_LAYER_SQUARE
            elif kind == "replicate":
                arr[i].kind = CTL_LAYER_REPLICATE
                arr[i].rep_t = ly[1]
            elif kind == "conv1d":
                w = np.ascontiguousarray(ly[1], dtype=np.float64)
                self._keep.append(w)
                arr[i].kind = CTL_LAYER_CONV1D
                arr[i].m, arr[i].n, arr[i].rep_t = len(w), ly[2], ly[3]
                arr[i].W = _p(w, _dp)
                if len(ly) > 4 and ly[4] is not None:
                    b = np.ascontiguousarray(ly[4], dtype=np.float64)
                    self._keep.append(b)
                    arr[i].bias = _p(b, _dp)
                if len(ly) > 5 and ly[5] is not None:
                    pc = np.ascontiguousarray(ly[5], dtype=np.int64)
                    self._keep.append(pc)
                    arr[i].pt_coeffs = _p(pc, _i64p)
            elif kind == "poly3":
                a = np.ascontiguousarray(ly[1], dtype=np.float64)
                if a.shape != (4,):
                    raise ValueError("poly3 takes the four coefficients a0..a3")
                self._keep.append(a)
                arr[i].kind = CTL_LAYER_POLY3
                arr[i].W = _p(a, _dp)
            elif kind == "avgpool":
                arr[i].kind = CTL_LAYER_AVGPOOL
                arr[i].m = ly[1]
            else:
                raise ValueError(kind)
        h = C.c_void_p()
        _check(lib().ctl_model_create(ctx.h, arr, len(layers), ctx.L if in_level is None else in_level,
                                      ctx.scale if in_scale is None else in_scale, C.byref(h)))
        self.h = h
        self._keep = []

    def rotations(self):
        n = C.c_uint32()
        _check(lib().ctl_model_rotations(self.h, None, 0, C.byref(n)))
        r = np.zeros(n.value, dtype=np.int32)
        _check(lib().ctl_model_rotations(self.h, _p(r, _i32p), n.value, C.byref(n)))
        return [int(x) for x in r]

    def info(self):
        lvl, sc, by = C.c_uint32(), C.c_double(), C.c_uint64()
        _check(lib().ctl_model_info(self.h, C.byref(lvl), C.byref(sc), C.byref(by)))
        return lvl.value, sc.value, by.value

    def forward(self, keys, ct, graph=False, ctx=None):
        ctx = self.ctx if ctx is None else ctx
        h = C.c_void_p()
        fn = lib().ctl_model_forward_graph if graph else lib().ctl_model_forward
        _check(fn(ctx.h, self.h, keys.h, ct.h, C.byref(h)))
        return Ciphertext(ctx, h)

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            lib().ctl_model_destroy(self.h)
        self.h = None


class Multi:
    """Groups of (context, model, keys, batch size) forwarded by one CUDA graph launch
    (ctl_multi_*); outputs are bit-identical to each group's own forward."""

    def __init__(self, groups):
        n = len(groups)
        self.groups = list(groups)
        ctxs = (C.c_void_p * n)(*[g[0].h for g in groups])
        models = (C.c_void_p * n)(*[g[1].h for g in groups])
        keys = (C.c_void_p * n)(*[g[2].h for g in groups])
        counts = np.ascontiguousarray([g[3] for g in groups], dtype=np.uint32)
        h = C.c_void_p()
        _check(lib().ctl_multi_create(n, C.cast(ctxs, _pp), C.cast(models, _pp), C.cast(keys, _pp),
                                      _p(counts, _u32p), C.byref(h)))
        self.h = h

    def forward(self, cts):
        n = len(self.groups)
        ins = (C.c_void_p * n)(*[c.h for c in cts])
        outs = (C.c_void_p * n)()
        _check(lib().ctl_multi_forward(self.h, C.cast(ins, _pp), C.cast(outs, _pp)))
        return [Ciphertext(self.groups[i][0], C.c_void_p(outs[i])) for i in range(n)]

    def close(self):
        if self.h:
            lib().ctl_multi_destroy(self.h)
            self.h = None


class Server:
    """Continuous-batching request loop (ctl_server_*): lanes = (context, model), clients = keys."""

    def __init__(self, mem_budget_bytes, n_workers=4, max_batch=64, max_queue=4096):
        h = C.c_void_p()
        _check(lib().ctl_server_create(C.byref(h), int(mem_budget_bytes), n_workers, max_batch, max_queue))
        self.h = h
        self._keep = []

    def add_lane(self, ctx, model):
        lane = C.c_uint32()
        _check(lib().ctl_server_add_lane(self.h, ctx.h, model.h, C.byref(lane)))
        self._keep += [ctx, model]
        return lane.value

    def add_client(self, lane, keys):
        cl = C.c_uint32()
        _check(lib().ctl_server_add_client(self.h, lane, keys.h, C.byref(cl)))
        self._keep.append(keys)
        return cl.value

    def admission(self, client):
        """(bytes per in-flight ciphertext of the client's lane, highest total reservation,
        number of waits for memory) (ctl_server_admission)."""
        b, pk, d = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().ctl_server_admission(self.h, client, C.byref(b), C.byref(pk), C.byref(d)))
        return b.value, pk.value, d.value

    def io_words(self, client):
        i, o = C.c_size_t(), C.c_size_t()
        _check(lib().ctl_server_io_words(self.h, client, C.byref(i), C.byref(o)))
        return i.value, o.value

    def start(self):
        _check(lib().ctl_server_start(self.h))

    def submit(self, client, coeffs):
        """Returns a request id, or None if the queue is full (CTL_EBUSY)."""
        a = np.ascontiguousarray(coeffs, dtype=np.uint64)
        rid = C.c_uint64()
        rc = lib().ctl_server_submit(self.h, client, _p(a, _u64p), C.byref(rid))
        if rc == -8:
            return None
        _check(rc)
        return rid.value

    def wait(self, rid, out_words, timeout_ms=600000):
        out = np.zeros(out_words, dtype=np.uint64)
        lat = C.c_double()
        _check(lib().ctl_server_wait(self.h, rid, timeout_ms, _p(out, _u64p), out.size, C.byref(lat)))
        return out, lat.value

    def poll(self, rid, out_words):
        """(result, latency_ms) when done, None while pending; raises on failure."""
        out = np.zeros(out_words, dtype=np.uint64)
        lat = C.c_double()
        rc = lib().ctl_server_poll(self.h, rid, _p(out, _u64p), out.size, C.byref(lat))
        if rc == -8:
            return None
        _check(rc)
        return out, lat.value

    def stats(self):
        c6 = np.zeros(6, dtype=np.uint64)
        p50, p99 = C.c_double(), C.c_double()
        _check(lib().ctl_server_stats(self.h, _p(c6, _u64p), C.byref(p50), C.byref(p99)))
        names = ["submitted", "completed", "rejected", "failed", "batches", "batched_cts"]
        d = dict(zip(names, [int(x) for x in c6]))
        d.update(p50_ms=p50.value, p99_ms=p99.value)
        return d

    def close(self):
        if getattr(self, "h", None):
            lib().ctl_server_destroy(self.h)
            self.h = None
