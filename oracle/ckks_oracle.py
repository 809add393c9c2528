"""ctypes wrapper of the C++ CKKS oracle (test infrastructure only).

Every function maps one-to-one to a function of ``ckks_oracle.cpp``; arrays are numpy.
Ciphertexts are coefficient-form residues shaped ``[2, level, N]`` (uint64), where
``level`` is the number of live data primes.
"""
import ctypes as C
import numpy as np

from .build import build as build_oracle

_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)
_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = C.CDLL(build_oracle())
        vp = C.c_void_p
        sig = {
            "orc_ctx_create": (vp, [C.c_uint32, _u32p, C.c_uint32, _u32p, C.c_uint32, C.c_uint32, C.c_double]),
            "orc_ctx_destroy": (None, [vp]),
            "orc_ctx_moduli": (C.c_int, [vp, _u64p]),
            "orc_ctx_psi": (C.c_int, [vp, _u64p]),
            "orc_ctx_alpha": (C.c_uint32, [vp]),
            "orc_ctx_beta": (C.c_uint32, [vp]),
            "orc_primes": (C.c_int, [C.c_uint32, _u32p, C.c_uint32, _u64p]),
            "orc_psi": (C.c_uint64, [C.c_uint64, C.c_uint32]),
            "orc_is_prime": (C.c_int, [C.c_uint64]),
            "orc_prng_word": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
            "orc_sample": (None, [C.c_uint64, C.c_uint64, C.c_int, C.c_uint64, C.c_uint32, _i64p]),
            "orc_ntt_direct": (C.c_int, [vp, C.c_uint32, _u64p, _u64p]),
            "orc_intt_direct": (C.c_int, [vp, C.c_uint32, _u64p, _u64p]),
            "orc_negacyclic_mul": (C.c_int, [vp, C.c_uint32, _u64p, _u64p, _u64p]),
            "orc_automorphism": (C.c_int, [vp, C.c_uint32, C.c_uint64, _u64p, _u64p]),
            "orc_galois_element": (C.c_uint64, [vp, C.c_int64]),
            "orc_encode": (C.c_int, [vp, _dp, C.c_uint32, C.c_double, _i64p]),
            "orc_decode": (C.c_int, [vp, _dp, C.c_double, C.c_uint32, _dp]),
            "orc_keygen": (vp, [vp, _i32p, C.c_uint32, C.c_uint64]),
            "orc_keys_destroy": (None, [vp]),
            "orc_keys_secret": (C.c_int, [vp, _i64p]),
            "orc_keys_has": (C.c_int, [vp, C.c_uint64]),
            "orc_keys_export": (C.c_int, [vp, C.c_uint64, _u64p]),
            "orc_encrypt": (C.c_int, [vp, vp, _i64p, C.c_uint64, _u64p]),
            "orc_decrypt": (C.c_int, [vp, vp, _u64p, C.c_uint32, _dp]),
            "orc_add": (C.c_int, [vp, _u64p, _u64p, C.c_uint32, _u64p]),
            "orc_mul_plain": (C.c_int, [vp, _u64p, C.c_uint32, _i64p, _u64p]),
            "orc_add_plain": (C.c_int, [vp, _u64p, C.c_uint32, _i64p, _u64p]),
            "orc_rescale": (C.c_int, [vp, _u64p, C.c_uint32, _u64p]),
            "orc_modup": (C.c_int, [vp, _u64p, C.c_uint32, C.c_uint32, _u64p, _u64p]),
            "orc_moddown": (C.c_int, [vp, _u64p, C.c_uint32, _u64p]),
            "orc_keyswitch": (C.c_int, [vp, vp, C.c_uint64, _u64p, C.c_uint32, C.c_uint64, _u64p]),
            "orc_rotate": (C.c_int, [vp, vp, _u64p, C.c_uint32, C.c_int64, _u64p]),
            "orc_relin": (C.c_int, [vp, vp, _u64p, C.c_uint32, _u64p]),
            "orc_square": (C.c_int, [vp, vp, _u64p, C.c_uint32, _u64p]),
            "orc_bsgs_t": (C.c_uint32, [C.c_uint32, C.c_uint32]),
            "orc_bsgs_t1": (C.c_uint32, [C.c_uint32]),
            "orc_bsgs_t1_lazy": (C.c_uint32, [C.c_uint32]),
            "orc_encode_diagonals": (C.c_int, [vp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double, _i64p]),
            "orc_encode_diagonals_w": (C.c_int, [vp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double,
                                                 C.c_uint32, _i64p]),
            "orc_encode_conv_w": (C.c_int, [vp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double, C.c_uint32,
                                            _i64p]),
            "orc_dense": (C.c_int, [vp, vp, _u64p, C.c_uint32, _i64p, C.c_uint32, _i64p, _u64p, _u64p]),
            "orc_dense_lazy": (C.c_int, [vp, vp, _u64p, C.c_uint32, _i64p, C.c_uint32, _i64p, _u64p, _u64p]),
            "orc_replicate": (C.c_int, [vp, vp, _u64p, C.c_uint32, C.c_uint32, _u64p]),
            "orc_encode_diagonals_rect": (C.c_int, [vp, _dp, C.c_uint32, C.c_uint32, C.c_double, _i64p]),
            "orc_encode_diagonals_rect_ex": (C.c_int, [vp, _dp, C.c_uint32, C.c_uint32, C.c_double, C.c_int,
                                                       _i64p]),
            "orc_dense_rect_ex": (C.c_int, [vp, vp, _u64p, C.c_uint32, _i64p, C.c_uint32, C.c_uint32, _i64p, C.c_int,
                                            C.c_int, _u64p, _u64p]),
            "orc_dense_rect": (C.c_int, [vp, vp, _u64p, C.c_uint32, _i64p, C.c_uint32, C.c_uint32, _i64p, C.c_int,
                                         _u64p, _u64p]),
            "orc_tensor": (C.c_int, [vp, _u64p, _u64p, C.c_uint32, _u64p]),
            "orc_mul": (C.c_int, [vp, vp, _u64p, _u64p, C.c_uint32, _u64p]),
            "orc_mul_const": (C.c_int, [vp, _u64p, C.c_uint32, C.c_int64, _u64p]),
            "orc_add_const": (C.c_int, [vp, _u64p, C.c_uint32, C.c_int64, _u64p]),
            "orc_drop_level": (C.c_int, [vp, _u64p, C.c_uint32, C.c_uint32, _u64p]),
            "orc_poly3_consts": (C.c_int, [vp, C.c_uint32, C.c_double, _dp, _i64p, _dp]),
            "orc_poly3": (C.c_int, [vp, vp, _u64p, C.c_uint32, C.c_double, _dp, _u64p, _dp]),
            "orc_avgpool": (C.c_int, [vp, vp, _u64p, C.c_uint32, C.c_uint32, _u64p, _u64p]),
            "orc_encode_conv": (C.c_int, [vp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double, _i64p]),
            "orc_conv1d": (C.c_int, [vp, vp, _u64p, C.c_uint32, _i64p, C.c_uint32, _i64p, _u64p, _u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(t)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _chk(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def primes(N, bits):
    b = np.asarray(bits, dtype=np.uint32)
    out = np.zeros(len(b), dtype=np.uint64)
    _chk(_lib().orc_primes(N, _p(b, _u32p), len(b), _p(out, _u64p)), "primes")
    return [int(x) for x in out]


def psi(q, N):
    return int(_lib().orc_psi(q, N))


def is_prime(n):
    return bool(_lib().orc_is_prime(n))


def prng_word(seed, stream, i):
    return int(_lib().orc_prng_word(seed, stream, i))


def sample(seed, stream, kind, q, N):
    """kind 0 = uniform mod q, 1 = ternary, 2 = centred binomial (k = 21)."""
    out = np.zeros(N, dtype=np.int64)
    _lib().orc_sample(seed, stream, kind, q, N, _p(out, _i64p))
    return out


class Oracle:
    """One CKKS parameter set: ring degree N, data primes, special primes, digits."""

    def __init__(self, N, q_bits, p_bits, dnum=None, scale=2.0 ** 40):
        self.lib = _lib()
        qb = np.asarray(q_bits, dtype=np.uint32)
        pb = np.asarray(p_bits, dtype=np.uint32)
        dnum = len(qb) if dnum is None else dnum
        self.h = self.lib.orc_ctx_create(N, _p(qb, _u32p), len(qb), _p(pb, _u32p), len(pb), dnum, scale)
        if not self.h:
            raise ValueError("invalid oracle parameters")
        self.N, self.L, self.K, self.scale = N, len(qb), len(pb), scale
        m = np.zeros(self.L + self.K, dtype=np.uint64)
        self.lib.orc_ctx_moduli(self.h, _p(m, _u64p))
        self.moduli = [int(x) for x in m]
        ps = np.zeros(self.L + self.K, dtype=np.uint64)
        self.lib.orc_ctx_psi(self.h, _p(ps, _u64p))
        self.psis = [int(x) for x in ps]
        self.alpha = int(self.lib.orc_ctx_alpha(self.h))
        self.beta = int(self.lib.orc_ctx_beta(self.h))
        self.keys = None

    def __del__(self):
        try:
            if self.keys:
                self.lib.orc_keys_destroy(self.keys)
            if self.h:
                self.lib.orc_ctx_destroy(self.h)
        except Exception:
            pass

    # --- rings -------------------------------------------------------------------
    def ntt_direct(self, pi, a):
        a = _u64(a); out = np.zeros(self.N, dtype=np.uint64)
        _chk(self.lib.orc_ntt_direct(self.h, pi, _p(a, _u64p), _p(out, _u64p)), "ntt")
        return out

    def intt_direct(self, pi, a):
        a = _u64(a); out = np.zeros(self.N, dtype=np.uint64)
        _chk(self.lib.orc_intt_direct(self.h, pi, _p(a, _u64p), _p(out, _u64p)), "intt")
        return out

    def polymul(self, pi, a, b):
        a = _u64(a); b = _u64(b); out = np.zeros(self.N, dtype=np.uint64)
        _chk(self.lib.orc_negacyclic_mul(self.h, pi, _p(a, _u64p), _p(b, _u64p), _p(out, _u64p)), "mul")
        return out

    def automorphism(self, pi, g, a):
        a = _u64(a); out = np.zeros(self.N, dtype=np.uint64)
        _chk(self.lib.orc_automorphism(self.h, pi, g, _p(a, _u64p), _p(out, _u64p)), "auto")
        return out

    def galois_element(self, r):
        return int(self.lib.orc_galois_element(self.h, r))

    # --- encoding ----------------------------------------------------------------
    def encode(self, z, scale=None):
        z = np.ascontiguousarray(z, dtype=np.float64)
        out = np.zeros(self.N, dtype=np.int64)
        _chk(self.lib.orc_encode(self.h, _p(z, _dp), len(z), self.scale if scale is None else scale, _p(out, _i64p)), "encode")
        return out

    def decode(self, m, nz, scale=None):
        m = np.ascontiguousarray(m, dtype=np.float64)
        out = np.zeros(nz, dtype=np.float64)
        _chk(self.lib.orc_decode(self.h, _p(m, _dp), self.scale if scale is None else scale, nz, _p(out, _dp)), "decode")
        return out

    # --- keys --------------------------------------------------------------------
    def keygen(self, rotations=(), seed=3):
        r = np.asarray(list(rotations), dtype=np.int32)
        if self.keys:
            self.lib.orc_keys_destroy(self.keys)
        self.keys = self.lib.orc_keygen(self.h, _p(r, _i32p), len(r), seed)
        return self.keys

    def secret(self):
        s = np.zeros(self.N, dtype=np.int64)
        self.lib.orc_keys_secret(self.keys, _p(s, _i64p))
        return s

    def key_export(self, key_id):
        out = np.zeros((self.beta, 2, self.L + self.K, self.N), dtype=np.uint64)
        _chk(self.lib.orc_keys_export(self.keys, key_id, _p(out, _u64p)), "key export")
        return out

    # --- ciphertexts -------------------------------------------------------------
    def encrypt(self, m, seed):
        m = _i64(m); ct = np.zeros((2, self.L, self.N), dtype=np.uint64)
        _chk(self.lib.orc_encrypt(self.h, self.keys, _p(m, _i64p), seed, _p(ct, _u64p)), "encrypt")
        return ct

    def decrypt(self, ct):
        ct = _u64(ct); lvl = ct.shape[1]
        out = np.zeros(self.N, dtype=np.float64)
        _chk(self.lib.orc_decrypt(self.h, self.keys, _p(ct, _u64p), lvl, _p(out, _dp)), "decrypt")
        return out

    def add(self, a, b):
        a = _u64(a); b = _u64(b); out = np.zeros_like(a)
        _chk(self.lib.orc_add(self.h, _p(a, _u64p), _p(b, _u64p), a.shape[1], _p(out, _u64p)), "add")
        return out

    def mul_plain(self, ct, pt):
        ct = _u64(ct); pt = _i64(pt); out = np.zeros_like(ct)
        _chk(self.lib.orc_mul_plain(self.h, _p(ct, _u64p), ct.shape[1], _p(pt, _i64p), _p(out, _u64p)), "mul_plain")
        return out

    def add_plain(self, ct, pt):
        ct = _u64(ct); pt = _i64(pt); out = np.zeros_like(ct)
        _chk(self.lib.orc_add_plain(self.h, _p(ct, _u64p), ct.shape[1], _p(pt, _i64p), _p(out, _u64p)), "add_plain")
        return out

    def rescale(self, ct):
        ct = _u64(ct); lvl = ct.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        _chk(self.lib.orc_rescale(self.h, _p(ct, _u64p), lvl, _p(out, _u64p)), "rescale")
        return out

    def modup(self, poly, digit):
        poly = _u64(poly); lvl = poly.shape[0]
        out = np.zeros((lvl + self.K, self.N), dtype=np.uint64)
        u = np.zeros(self.N, dtype=np.uint64)
        _chk(self.lib.orc_modup(self.h, _p(poly, _u64p), lvl, digit, _p(out, _u64p), _p(u, _u64p)), "modup")
        return out, u

    def moddown(self, ext):
        ext = _u64(ext); lvl = ext.shape[0] - self.K
        out = np.zeros((lvl, self.N), dtype=np.uint64)
        _chk(self.lib.orc_moddown(self.h, _p(ext, _u64p), lvl, _p(out, _u64p)), "moddown")
        return out

    def keyswitch(self, key_id, poly, g=1):
        poly = _u64(poly); lvl = poly.shape[0]
        out = np.zeros((2, lvl, self.N), dtype=np.uint64)
        _chk(self.lib.orc_keyswitch(self.h, self.keys, key_id, _p(poly, _u64p), lvl, g, _p(out, _u64p)), "keyswitch")
        return out

    def rotate(self, ct, r):
        ct = _u64(ct); out = np.zeros_like(ct)
        _chk(self.lib.orc_rotate(self.h, self.keys, _p(ct, _u64p), ct.shape[1], r, _p(out, _u64p)), "rotate")
        return out

    def relin(self, d):
        d = _u64(d); lvl = d.shape[1]
        out = np.zeros((2, lvl, self.N), dtype=np.uint64)
        _chk(self.lib.orc_relin(self.h, self.keys, _p(d, _u64p), lvl, _p(out, _u64p)), "relin")
        return out

    def square(self, ct):
        ct = _u64(ct); lvl = ct.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        _chk(self.lib.orc_square(self.h, self.keys, _p(ct, _u64p), lvl, _p(out, _u64p)), "square")
        return out

    @staticmethod
    def bsgs_t(m, n):
        return int(_lib().orc_bsgs_t(m, n))

    @staticmethod
    def bsgs_t1(t, lazy=False):
        return int(_lib().orc_bsgs_t1_lazy(t) if lazy else _lib().orc_bsgs_t1(t))

    @classmethod
    def bsgs_rotations(cls, m, n, lazy=False):
        """Galois rotations a dense layer m x n needs: 1..t1-1 and k*t1 for k = 1..t2-1."""
        t = cls.bsgs_t(m, n)
        t1 = cls.bsgs_t1(t, lazy)
        return list(range(1, t1)) + [k * t1 for k in range(1, t // t1)]

    def encode_diagonals(self, W, scale, lazy=False, windows=1):
        """Diagonal plaintexts of Eq. (bsgs); windows = p repeats them in p windows of 2t
        slots (Sec. 3.1, Multiple Predictions)."""
        W = np.ascontiguousarray(W, dtype=np.float64)
        m, n = W.shape
        t = self.bsgs_t(m, n)
        out = np.zeros((t, self.N), dtype=np.int64)
        _chk(self.lib.orc_encode_diagonals_w(self.h, _p(W, _dp), m, n, self.bsgs_t1(t, lazy), scale, windows,
                                             _p(out, _i64p)), "encode_diagonals")
        return out

    def dense(self, ct, pts, bias=None, lazy=False):
        """Dense layer by Eq. (bsgs) as the composition of whole rotations; lazy=True takes
        the lazy-ModDown form instead (its own split and diagonals; decodes to the same
        values within the noise)."""
        ct = _u64(ct); pts = _i64(pts); lvl = ct.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        cnt = np.zeros(3, dtype=np.uint64)
        bp = _p(_i64(bias), _i64p) if bias is not None else None
        fn = self.lib.orc_dense_lazy if lazy else self.lib.orc_dense
        _chk(fn(self.h, self.keys, _p(ct, _u64p), lvl, _p(pts, _i64p), pts.shape[0], bp,
                _p(out, _u64p), _p(cnt, _u64p)), "dense")
        return out, [int(x) for x in cnt]

    def encode_diagonals_rect(self, W, scale, lazy=False):
        """The tm rectangular diagonals of a dense layer m x n with tm < tn (powers of two
        >= m and >= n), placed as in Eq. (bsgs) with t1 = bsgs_t1(tm, lazy)."""
        W = np.ascontiguousarray(W, dtype=np.float64)
        m, n = W.shape
        tm = self.bsgs_t(m, 1)
        out = np.zeros((tm, self.N), dtype=np.int64)
        _chk(self.lib.orc_encode_diagonals_rect_ex(self.h, _p(W, _dp), m, n, scale, int(lazy), _p(out, _i64p)),
             "encode_rect")
        return out

    def dense_rect(self, ct, pts, tn, bias=None, fold=2, lazy=False):
        """Rectangular dense layer: Eq. (bsgs) over the tm = len(pts) diagonals (composed, or
        the lazy-ModDown form with lazy=True), the rescale, then fold = 1: the sum over the
        tn/tm blocks (y in slots [0, tm)), fold = 2: and the [y, y] layout at block stride
        tm; fold = 0: no fold."""
        ct = _u64(ct); pts = _i64(pts); lvl = ct.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        cnt = np.zeros(3, dtype=np.uint64)
        bp = _p(_i64(bias), _i64p) if bias is not None else None
        _chk(self.lib.orc_dense_rect_ex(self.h, self.keys, _p(ct, _u64p), lvl, _p(pts, _i64p), pts.shape[0], tn, bp,
                                        fold, int(lazy), _p(out, _u64p), _p(cnt, _u64p)), "dense_rect")
        return out, [int(x) for x in cnt]

    @classmethod
    def rect_rotations(cls, m, n, fold=2, lazy=False):
        """Galois rotations of the rectangular form: the Eq. (bsgs) split of tm, the fold
        shifts tn/2 .. tm and, fold = 2, -tm."""
        tm, tn = cls.bsgs_t(m, 1), cls.bsgs_t(n, 1)
        t1 = cls.bsgs_t1(tm, lazy)
        rots = list(range(1, t1)) + [k * t1 for k in range(1, tm // t1)]
        if fold >= 1:
            s = tn // 2
            while s >= tm:
                rots.append(s)
                s //= 2
        if fold == 2:
            rots.append(-tm)
        return rots

    def replicate(self, ct, t):
        ct = _u64(ct); out = np.zeros_like(ct)
        _chk(self.lib.orc_replicate(self.h, self.keys, _p(ct, _u64p), ct.shape[1], t, _p(out, _u64p)), "replicate")
        return out

    # --- the other layers of the paper's frozen network (Sec. 3.1) ---------------
    def tensor(self, a, b):
        a = _u64(a); b = _u64(b); lvl = a.shape[1]
        out = np.zeros((3, lvl, self.N), dtype=np.uint64)
        _chk(self.lib.orc_tensor(self.h, _p(a, _u64p), _p(b, _u64p), lvl, _p(out, _u64p)), "tensor")
        return out

    def mul(self, a, b):
        """HMult of two ciphertexts at the same level: tensor, relinearise, rescale."""
        a = _u64(a); b = _u64(b); lvl = a.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        _chk(self.lib.orc_mul(self.h, self.keys, _p(a, _u64p), _p(b, _u64p), lvl, _p(out, _u64p)), "mul")
        return out

    def mul_const(self, ct, c):
        ct = _u64(ct); out = np.zeros_like(ct)
        _chk(self.lib.orc_mul_const(self.h, _p(ct, _u64p), ct.shape[1], int(c), _p(out, _u64p)), "mul_const")
        return out

    def add_const(self, ct, c):
        ct = _u64(ct); out = np.zeros_like(ct)
        _chk(self.lib.orc_add_const(self.h, _p(ct, _u64p), ct.shape[1], int(c), _p(out, _u64p)), "add_const")
        return out

    def drop_level(self, ct, to):
        ct = _u64(ct); out = np.zeros((2, to, self.N), dtype=np.uint64)
        _chk(self.lib.orc_drop_level(self.h, _p(ct, _u64p), ct.shape[1], to, _p(out, _u64p)), "drop_level")
        return out

    def poly3_consts(self, lvl, in_scale, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        C = np.zeros(4, dtype=np.int64)
        out_scale = np.zeros(1)
        _chk(self.lib.orc_poly3_consts(self.h, lvl, in_scale, _p(a, _dp), _p(C, _i64p), _p(out_scale, _dp)),
             "poly3_consts")
        return [int(x) for x in C], float(out_scale[0])

    def poly3(self, ct, in_scale, a):
        """a[3] z^3 + a[2] z^2 + a[1] z + a[0] at depth 2; returns (ct, out_scale)."""
        ct = _u64(ct); lvl = ct.shape[1]
        a = np.ascontiguousarray(a, dtype=np.float64)
        out = np.zeros((2, lvl - 2, self.N), dtype=np.uint64)
        sc = np.zeros(1)
        _chk(self.lib.orc_poly3(self.h, self.keys, _p(ct, _u64p), lvl, in_scale, _p(a, _dp), _p(out, _u64p),
                                _p(sc, _dp)), "poly3")
        return out, float(sc[0])

    def avgpool(self, ct, f):
        ct = _u64(ct); lvl = ct.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        cnt = np.zeros(3, dtype=np.uint64)
        _chk(self.lib.orc_avgpool(self.h, self.keys, _p(ct, _u64p), lvl, f, _p(out, _u64p), _p(cnt, _u64p)),
             "avgpool")
        return out, [int(x) for x in cnt]

    def encode_conv(self, w, n, t, scale, windows=1):
        w = np.ascontiguousarray(w, dtype=np.float64)
        out = np.zeros((len(w), self.N), dtype=np.int64)
        _chk(self.lib.orc_encode_conv_w(self.h, _p(w, _dp), len(w), n, t, scale, windows, _p(out, _i64p)),
             "encode_conv")
        return out

    def conv1d(self, ct, pts, bias=None):
        ct = _u64(ct); pts = _i64(pts); lvl = ct.shape[1]
        out = np.zeros((2, lvl - 1, self.N), dtype=np.uint64)
        cnt = np.zeros(3, dtype=np.uint64)
        bp = _p(_i64(bias), _i64p) if bias is not None else None
        _chk(self.lib.orc_conv1d(self.h, self.keys, _p(ct, _u64p), lvl, _p(pts, _i64p), pts.shape[0], bp,
                                 _p(out, _u64p), _p(cnt, _u64p)), "conv1d")
        return out, [int(x) for x in cnt]

    # --- composite helpers (scale bookkeeping of the oracle's reading) -----------
    def dense_scale(self, lvl, in_scale=None):
        """Plaintext scale of a dense layer applied at level lvl to an input at in_scale
        (default Delta): q_{lvl-1} * Delta / in_scale, so that the rescaled output carries
        the nominal scale Delta again."""
        return float(self.moduli[lvl - 1]) * (self.scale / (self.scale if in_scale is None else in_scale))

    def square_scale(self, lvl, in_scale):
        return in_scale * in_scale / float(self.moduli[lvl - 1])
