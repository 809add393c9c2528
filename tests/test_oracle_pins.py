"""Pins of the CKKS oracle against things other than itself (CPU only).

Each test checks an oracle function against a published value, a closed form, an
invariant, an independent library routine (sympy, Python big integers, numpy FP64) or
brute force on tiny inputs.  The oracle follows Sec. 3.1 of the CryptoTL paper (CKKS,
SIMD encoding, rescaling, rotations, Eq. (bsgs)).
"""
import json
import os

import numpy as np
import pytest
import sympy
from sympy.ntheory.modular import crt as sympy_crt

from oracle import ckks_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def brv(k, logn):
    return int(format(k, f"0{logn}b")[::-1], 2) if logn else 0


def py_negacyclic(a, b, q):
    """Linear convolution by numpy on Python ints, then the X^N = -1 fold."""
    N = len(a)
    full = np.convolve(np.array([int(x) for x in a], dtype=object), np.array([int(x) for x in b], dtype=object))
    full = list(full) + [0] * (2 * N - len(full))
    return [int((full[k] - full[k + N]) % q) for k in range(N)]


def crt_int(res, mods):
    return int(sympy_crt([int(m) for m in mods], [int(r) for r in res])[0])


def centred(v, Q):
    v %= Q
    return v - Q if v > Q // 2 else v


# ----------------------------------------------------------------------------- PRNG
def test_splitmix64_published_vector():
    # A stream whose key is 0 reproduces the raw SplitMix64 sequence from state 0:
    # key = mix(seed ^ mix(stream + gamma)) = 0 when seed = mix(stream + gamma).
    # mix(0 + gamma) is the first published word, so seed = vals[0] gives key 0 for stream 0.
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = [O.prng_word(vals[0], 0, i) for i in range(len(vals))]
    assert got == vals


def test_sampling_distributions():
    N = 1 << 14
    q = (1 << 40) - (1 << 15) + 1
    u = O.sample(7, 123, 0, q, N)
    assert u.min() >= 0 and int(u.max()) < q
    assert abs(u.astype(np.float64).mean() / q - 0.5) < 0.02
    t = O.sample(7, 124, 1, 0, N)
    assert set(np.unique(t).tolist()) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs((t == v).mean() - 1 / 3) < 0.02
    e = O.sample(7, 125, 2, 0, N)
    assert np.abs(e).max() <= 21
    assert abs(e.mean()) < 0.1 and abs(e.var() - 10.5) < 0.6  # centred binomial k=21: var 21/2


def test_centred_binomial_is_k21_exactly():
    # The error distribution is a difference of two sums of 21 fair bits: P(e = v) =
    # C(42, 21 + v) / 2^42, variance 21/2.  At 2^18 samples the variance is known to about
    # +-0.03 (one standard deviation), so k = 20 (variance 10) or k = 22 (11) fails the
    # +-0.15 window; the chi-square statistic against the exact k = 21 law (43 cells, tail
    # cells merged) rejects the neighbouring k as well.
    from math import comb
    e = np.concatenate([O.sample(11, 900 + s, 2, 0, 1 << 16) for s in range(4)])
    n = len(e)
    assert abs(e.var() - 10.5) < 0.15
    pmf = {v: comb(42, 21 + v) / 2.0 ** 42 for v in range(-21, 22)}
    cells = [v for v in range(-21, 22) if pmf[v] * n >= 5]
    lo, hi = min(cells), max(cells)
    obs = [np.sum(e <= lo)] + [np.sum(e == v) for v in range(lo + 1, hi)] + [np.sum(e >= hi)]
    exp = [sum(pmf[v] for v in range(-21, lo + 1)) * n] + [pmf[v] * n for v in range(lo + 1, hi)] + \
          [sum(pmf[v] for v in range(hi, 22)) * n]
    chi2 = sum((o - x) ** 2 / x for o, x in zip(obs, exp))
    # dof = cells - 1 (about 25); 80 is far in the tail of that chi-square law, while k = 20
    # or k = 22 gives a statistic in the thousands at this sample size.
    assert chi2 < 80, chi2


# ----------------------------------------------------------------------------- primes
@pytest.mark.parametrize("N,bits", [(4096, [50, 40, 40, 60]), (8192, [60, 40, 40, 40, 60]),
                                    (16384, [45] * 8 + [60, 60])])
def test_primes_are_largest_ntt_friendly(N, bits):
    ps = O.primes(N, bits)
    M = max(2 * N, 32768)
    assert len(set(ps)) == len(ps)
    for i, (q, b) in enumerate(zip(ps, bits)):
        assert sympy.isprime(q)
        assert q < (1 << b) and q % M == 1
        # no unused prime of the same form lies between q and 2^b
        c = (1 << b) - M + 1
        while c > q:
            assert c in ps[:i] or not sympy.isprime(c)
            c -= M


def test_paper_modulus_budget_reading():
    # Sec. 3.1: depth 6 needs 8 primes, 6 close to Delta plus two wider ones; Tab. 1 gives
    # log2 q = 218 (Delta = 2^25) and 420 (Delta = 2^50).  Reading: the two wide primes have
    # log2(Delta) + gamma bits with gamma the pre-comma bits (60 - log2 Delta in SEAL).
    g = json.load(open(os.path.join(GOLD, "paper_params.json")))
    assert g["n_primes"] == 8 and g["depth"] == 6
    for ps in g["param_sets"]:
        d = ps["log2_delta"]
        wide = (ps["log2_q"] - g["n_primes_near_delta"] * d) // 2
        assert g["n_primes_near_delta"] * d + 2 * wide == ps["log2_q"]
        primes = O.primes(ps["N"], [wide] + [d] * 6 + [wide])
        assert sum(int(p).bit_length() for p in primes) == ps["log2_q"]


def test_paper_predictions_per_ciphertext():
    # Sec. 3.1 "Multiple Predictions": p = floor(#slots / (2 * #neurons)), Tab. 1 column p.
    g = json.load(open(os.path.join(GOLD, "paper_params.json")))
    for ps in g["param_sets"]:
        assert (ps["N"] // 2) // (2 * g["largest_dense_neurons"]) == ps["p"]


# ----------------------------------------------------------------------------- roots / NTT
@pytest.mark.parametrize("N", [16, 64])
def test_psi_is_smallest_primitive_root(N):
    q = O.primes(N, [40])[0]
    psi = O.psi(q, N)
    assert pow(psi, N, q) == q - 1
    g = sympy.primitive_root(q)
    base = pow(g, (q - 1) // (2 * N), q)
    roots = [pow(base, k, q) for k in range(1, 2 * N, 2)]
    assert psi == min(roots)


@pytest.mark.parametrize("N", [16, 64, 256])
def test_ntt_convolution_theorem(N):
    o = O.Oracle(N, [40, 40], [50])
    rng = np.random.default_rng(N)
    for pi, q in enumerate(o.moduli[:2]):
        a = rng.integers(0, q, N, dtype=np.uint64)
        b = rng.integers(0, q, N, dtype=np.uint64)
        A, B = o.ntt_direct(pi, a), o.ntt_direct(pi, b)
        prod = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
        assert [int(v) for v in o.intt_direct(pi, prod)] == py_negacyclic(a, b, q)
        assert [int(v) for v in o.intt_direct(pi, A)] == [int(v) for v in a]


@pytest.mark.parametrize("N", [16, 128])
def test_ntt_of_monomial_is_bitreversed_points(N):
    # NTT(X)[k] is the k-th evaluation point psi^(2*brv(k)+1), NTT(1) is all ones.
    o = O.Oracle(N, [40], [50])
    q, psi = o.moduli[0], o.psis[0]
    logn = N.bit_length() - 1
    x = np.zeros(N, dtype=np.uint64); x[1] = 1
    assert [int(v) for v in o.ntt_direct(0, x)] == [pow(psi, 2 * brv(k, logn) + 1, q) for k in range(N)]
    one = np.zeros(N, dtype=np.uint64); one[0] = 1
    assert all(int(v) == 1 for v in o.ntt_direct(0, one))


@pytest.mark.parametrize("N", [16, 64, 512])
def test_negacyclic_mul_bruteforce(N):
    o = O.Oracle(N, [61], [50])
    q = o.moduli[0]
    rng = np.random.default_rng(1)
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    assert [int(v) for v in o.polymul(0, a, b)] == py_negacyclic(a, b, q)


def test_automorphism_homomorphism_and_composition():
    N = 64
    o = O.Oracle(N, [40], [50])
    q = o.moduli[0]
    rng = np.random.default_rng(2)
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    g, h = 5, 2 * N - 1
    sa = o.automorphism(0, g, a)
    # ring homomorphism: sigma(a*b) = sigma(a)*sigma(b)
    assert np.array_equal(o.automorphism(0, g, o.polymul(0, a, b)), o.polymul(0, sa, o.automorphism(0, g, b)))
    # composition: sigma_g(sigma_h(a)) = sigma_{gh}(a)
    assert np.array_equal(o.automorphism(0, g, o.automorphism(0, h, a)), o.automorphism(0, (g * h) % (2 * N), a))
    # closed form on the monomial X: sigma_g(X) = X^g
    x = np.zeros(N, dtype=np.uint64); x[1] = 1
    exp = np.zeros(N, dtype=np.uint64); exp[g] = 1
    assert np.array_equal(o.automorphism(0, g, x), exp)


# ----------------------------------------------------------------------------- encoding
def test_encode_constant_closed_form():
    o = O.Oracle(256, [50], [60])
    for c in (0.5, -0.25, 0.123456789):
        m = o.encode(np.full(128, c), 2.0 ** 40)
        assert m[0] == round(c * 2 ** 40) and not m[1:].any()


def test_encode_decode_roundtrip_and_ring_structure():
    N = 256
    o = O.Oracle(N, [50], [60])
    rng = np.random.default_rng(3)
    z1, z2 = rng.uniform(-1, 1, N // 2), rng.uniform(-1, 1, N // 2)
    D = 2.0 ** 30
    m1, m2 = o.encode(z1, D), o.encode(z2, D)
    assert np.max(np.abs(o.decode(m1.astype(np.float64), N // 2, D) - z1)) < 1e-7
    # the canonical embedding turns the negacyclic product into the slot-wise product
    full = np.convolve(m1.astype(object), m2.astype(object))
    full = list(full) + [0] * (2 * N - len(full))
    prod = np.array([float(full[k] - full[k + N]) for k in range(N)])
    assert np.max(np.abs(o.decode(prod, N // 2, D * D) - z1 * z2)) < 1e-6
    # X -> X^5 rotates the slots left by one (slot j sits at zeta^(5^j))
    rot = np.zeros(N)
    for i in range(N):
        e = (5 * i) % (2 * N)
        if e < N:
            rot[e] += m1[i]
        else:
            rot[e - N] -= m1[i]
    assert np.max(np.abs(o.decode(rot, N // 2, D) - np.roll(z1, -1))) < 1e-7


# ----------------------------------------------------------------------------- keys / enc
def small_ctx(N=64, q_bits=(50, 40, 40), p_bits=(60,), dnum=None, rots=(1, 2, -4)):
    o = O.Oracle(N, list(q_bits), list(p_bits), dnum=dnum, scale=2.0 ** 40)
    o.keygen(rots, seed=3)
    return o


def test_encrypt_structure_and_decrypt():
    o = small_ctx()
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, o.N // 2)
    m = o.encode(z)
    ct = o.encrypt(m, 4)
    s = o.secret()
    assert set(np.unique(s).tolist()) <= {-1, 0, 1}
    # c0 + c1*s - m is the encryption noise, bounded by the binomial support (21)
    for i, q in enumerate(o.moduli[: o.L]):
        cs = py_negacyclic(ct[1, i], [int(v) % q for v in s], q)
        e = [centred(int(ct[0, i, k]) + cs[k] - int(m[k]), q) for k in range(o.N)]
        assert max(abs(v) for v in e) <= 21
    d = o.decrypt(ct)
    assert np.max(np.abs(d - m)) <= 21
    assert np.max(np.abs(o.decode(d, o.N // 2) - z)) < 1e-8


@pytest.mark.parametrize("dnum", [3, 2])
def test_keyswitch_key_structure(dnum):
    o = small_ctx(N=16, q_bits=(50, 40, 40), p_bits=(60,), dnum=dnum, rots=(1,))
    s = [int(v) for v in o.secret()]
    N, L, K = o.N, o.L, o.K
    P = o.moduli[L]
    s2 = [0] * N
    for i in range(N):
        for j in range(N):
            e = i + j
            if e < N:
                s2[e] += s[i] * s[j]
            else:
                s2[e - N] -= s[i] * s[j]
    g = o.galois_element(1)
    sg = [0] * N
    for i in range(N):
        e = (i * g) % (2 * N)
        if e < N:
            sg[e] += s[i]
        else:
            sg[e - N] -= s[i]
    for key_id, sp in ((0, s2), (g, sg)):
        evk = o.key_export(key_id)
        for d in range(o.beta):
            errs = []
            for i, q in enumerate(o.moduli):
                in_digit = d * o.alpha <= i < min((d + 1) * o.alpha, L)
                b1s = py_negacyclic(evk[d, 1, i], [v % q for v in s], q)
                gad = (P % q) if in_digit else 0
                errs.append([centred(int(evk[d, 0, i, k]) + b1s[k] - gad * sp[k], q) for k in range(N)])
            # the same small error polynomial on every prime, bounded by 21
            assert all(e == errs[0] for e in errs)
            assert max(abs(v) for v in errs[0]) <= 21


# ----------------------------------------------------------------------------- base conversion
@pytest.mark.parametrize("dnum", [3, 2, 1])
def test_modup_invariants(dnum):
    o = O.Oracle(32, [50, 40, 40], [60, 58], dnum=dnum)
    rng = np.random.default_rng(5)
    lvl = 3
    poly = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.moduli[:lvl]])
    basis = o.moduli[:lvl] + o.moduli[o.L:]
    for d in range((lvl + o.alpha - 1) // o.alpha):
        ext, u = o.modup(poly, d)
        dig = list(range(d * o.alpha, min((d + 1) * o.alpha, lvl)))
        Qd = 1
        for j in dig:
            Qd *= o.moduli[j]
        for k in range(o.N):
            a = crt_int([poly[j, k] for j in dig], [o.moduli[j] for j in dig])
            Y = crt_int(ext[:, k], basis)
            # Y = a + u*Q_d with 0 <= u < |digit|
            assert (Y - a) % Qd == 0
            uu = (Y - a) // Qd
            assert 0 <= uu < len(dig) and uu == int(u[k])


@pytest.mark.parametrize("dnum", [3, 2, 1])
@pytest.mark.parametrize("pbits", [[60], [60, 58]])
def test_modup_is_the_fast_conversion_elementwise(dnum, pbits):
    # The fixed ModUp variant (fast base conversion, no correction): for digit d with primes
    # q_j, q_hat_j = Q_d / q_j, every other prime p of Q_l u P receives
    #   y mod p,  y = sum_j [a_j * q_hat_j^-1]_{q_j} * q_hat_j   (a Python integer),
    # and the digit's own primes receive a_j unchanged.  An exact conversion (y = a) or
    # any other correction differs from this on most coefficients.
    o = O.Oracle(32, [50, 40, 40], pbits, dnum=dnum)
    rng = np.random.default_rng(50 + dnum + 10 * len(pbits))
    lvl = 3
    poly = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.moduli[:lvl]])
    basis = o.moduli[:lvl] + o.moduli[o.L:]
    for d in range((lvl + o.alpha - 1) // o.alpha):
        ext, _ = o.modup(poly, d)
        dig = list(range(d * o.alpha, min((d + 1) * o.alpha, lvl)))
        qs = [o.moduli[j] for j in dig]
        Qd = 1
        for q in qs:
            Qd *= q
        hats = [Qd // q for q in qs]
        invs = [pow(h % q, -1, q) for h, q in zip(hats, qs)]
        n_differ_from_exact = 0
        for k in range(o.N):
            y = sum(((int(poly[j, k]) * iv) % q) * h for j, q, h, iv in zip(dig, qs, hats, invs))
            a = y % Qd  # the digit value itself (CRT), what an exact conversion would carry
            for i, p in enumerate(basis):
                want = int(poly[i, k]) if i in dig else y % p
                assert int(ext[i, k]) == want, (d, i, k)
            n_differ_from_exact += y != a
        if len(dig) > 1:
            assert n_differ_from_exact > 0  # the inputs exercise the u > 0 case


@pytest.mark.parametrize("lvl", [3, 2])
@pytest.mark.parametrize("pbits", [[60], [60, 58]])
def test_moddown_is_the_fast_conversion_elementwise(pbits, lvl):
    # The fixed ModDown variant (no rounding offset): with P = prod p_j, P_hat_j = P / p_j,
    #   out_i = (c_i - sum_j [c_{p_j} * P_hat_j^-1]_{p_j} * P_hat_j) * P^-1  mod q_i.
    # Adding floor(P/2) first (the rounding variant) changes about half of the outputs.
    o = O.Oracle(32, [50, 40, 40], pbits)
    rng = np.random.default_rng(60 + lvl + 10 * len(pbits))
    ps = o.moduli[o.L:]
    basis = o.moduli[:lvl] + ps
    ext = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in basis])
    out = o.moddown(ext)
    P = 1
    for p in ps:
        P *= p
    hats = [P // p for p in ps]
    invs = [pow(h % p, -1, p) for h, p in zip(hats, ps)]
    for k in range(o.N):
        yP = sum(((int(ext[lvl + j, k]) * iv) % p) * h for j, (p, h, iv) in enumerate(zip(ps, hats, invs)))
        for i in range(lvl):
            q = o.moduli[i]
            assert int(out[i, k]) == ((int(ext[i, k]) - yP) * pow(P % q, -1, q)) % q, (i, k)


@pytest.mark.parametrize("pbits", [[60], [60, 58]])
def test_moddown_invariant(pbits):
    o = O.Oracle(32, [50, 40, 40], pbits)
    rng = np.random.default_rng(6)
    lvl = 3
    basis = o.moduli[:lvl] + o.moduli[o.L:]
    ext = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in basis])
    out = o.moddown(ext)
    Q = int(np.prod([sympy.Integer(q) for q in o.moduli[:lvl]]))
    P = int(np.prod([sympy.Integer(q) for q in o.moduli[o.L:]]))
    for k in range(o.N):
        C = crt_int(ext[:, k], basis)
        R = crt_int(out[:, k], o.moduli[:lvl])
        yP = (C - P * R) % Q
        # y_P is a representative of C mod P within [0, K*P)
        assert yP % P == C % P and yP < len(pbits) * P


def test_rescale_exact_rounding_and_inverse():
    o = O.Oracle(32, [50, 40, 40], [60])
    rng = np.random.default_rng(7)
    lvl = 3
    ct = np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.moduli[:lvl]]) for _ in range(2)])
    out = o.rescale(ct)
    ql = o.moduli[lvl - 1]
    for p in range(2):
        for k in range(o.N):
            C = crt_int(ct[p, :, k], o.moduli[:lvl])
            Cp = (C + ql // 2) // ql  # round half up (q odd: no ties)
            assert [int(out[p, i, k]) for i in range(lvl - 1)] == [Cp % q for q in o.moduli[: lvl - 1]]
    # rescale(q_l * c) = c
    low = np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.moduli[: lvl - 1]]) for _ in range(2)])
    lift = np.zeros_like(ct)
    for p in range(2):
        for k in range(o.N):
            C = crt_int(low[p, :, k], o.moduli[: lvl - 1]) * ql
            for i in range(lvl):
                lift[p, i, k] = C % o.moduli[i]
    assert np.array_equal(o.rescale(lift), low)


# ----------------------------------------------------------------------------- homomorphic ops
@pytest.mark.parametrize("dnum,pbits", [(3, (60,)), (2, (60, 60))])
def test_keyswitch_semantics(dnum, pbits):
    # P must exceed the digit modulus (one 60-bit prime per 50/40-bit digit, two for two)
    o = small_ctx(N=64, dnum=dnum, p_bits=pbits)
    s = [int(v) for v in o.secret()]
    rng = np.random.default_rng(8)
    lvl = 3
    x = np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.moduli[:lvl]])
    ks = o.keyswitch(0, x)
    # KS_{s^2 -> s}(x) decrypts to x * s^2 up to a small error
    for i, q in enumerate(o.moduli[:lvl]):
        sq = [v % q for v in s]
        s2 = py_negacyclic(sq, sq, q)
        lhs = py_negacyclic(ks[1, i], sq, q)
        want = py_negacyclic(x[i], s2, q)
        err = [centred(int(ks[0, i, k]) + lhs[k] - want[k], q) for k in range(o.N)]
        assert max(abs(v) for v in err) < 2 ** 20


@pytest.mark.parametrize("r", [1, 2, -4])
def test_rotation_is_slot_roll(r):
    o = small_ctx(N=128)
    rng = np.random.default_rng(9)
    z = rng.uniform(-1, 1, o.N // 2)
    ct = o.encrypt(o.encode(z), 11)
    out = o.rotate(ct, r)
    assert np.max(np.abs(o.decode(o.decrypt(out), o.N // 2) - np.roll(z, -r))) < 1e-6


def test_square_matches_fp64():
    o = small_ctx(N=128)
    rng = np.random.default_rng(10)
    z = rng.uniform(-1, 1, o.N // 2)
    ct = o.encrypt(o.encode(z), 12)
    sq = o.square(ct)
    sc = o.square_scale(3, o.scale)
    assert sq.shape[1] == 2
    assert np.max(np.abs(o.decode(o.decrypt(sq), o.N // 2, sc) - z * z)) < 1e-6


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("m,n", [(8, 16), (16, 16), (5, 12)])
def test_dense_bsgs_matches_fp64_and_op_counts(m, n, lazy):
    N = 128
    t = O.Oracle.bsgs_t(m, n)
    t1 = O.Oracle.bsgs_t1(t, lazy)
    t2 = t // t1
    o = small_ctx(N=N, rots=O.Oracle.bsgs_rotations(m, n, lazy))
    rng = np.random.default_rng(m * 100 + n)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(N // 2)
    slots[:n] = x
    slots[t:t + n] = x  # [x, x] over 2t slots (Sec. 3.1, Multiple Predictions: 2 * #neurons)
    ct = o.encrypt(o.encode(slots), 13)
    lvl = 3
    pts = o.encode_diagonals(W, o.dense_scale(lvl), lazy)
    out, cnt = o.dense(ct, pts, lazy=lazy)
    # Sec. 3.1: t1 + t2 - 2 rotations, t plaintext products, t - 1 additions
    assert cnt == [t1 + t2 - 2, t, t - 1]
    y = o.decode(o.decrypt(out), N // 2)  # input at Delta: the output is at Delta too
    assert np.max(np.abs(y[:m] - W @ x)) < 1e-6
    assert np.max(np.abs(y[m:])) < 1e-6  # outputs outside [0, m) stay zero


def test_bsgs_splits():
    # t = t1 * t2 (Eq. bsgs).  Default split t1 = 2^ceil(log2(t)/2); the lazy form's split
    # is the power of two minimising (t1 - 1) + 4 (t2 - 1), ties to the larger t1, found
    # here by brute force.
    for lg in range(0, 13):
        t = 1 << lg
        assert O.Oracle.bsgs_t1(t) == 1 << ((lg + 1) // 2)
        best = min(((1 << a) for a in range(lg + 1)), key=lambda a: ((a - 1) + 4 * (t // a - 1), -a))
        assert O.Oracle.bsgs_t1(t, lazy=True) == best, t


def test_dense_is_composition_of_rotations():
    """With one ModUp shared by the baby steps, the dense layer is bit-identical to the
    composition of whole rotations, products, sums and a rescale in the order of Eq. (bsgs)."""
    N, m, n = 128, 16, 16
    t = 16
    t1, t2 = O.Oracle.bsgs_t1(t), t // O.Oracle.bsgs_t1(t)
    o = small_ctx(N=N, rots=O.Oracle.bsgs_rotations(m, n))
    rng = np.random.default_rng(23)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(N // 2); slots[:n] = x; slots[t:t + n] = x
    ct = o.encrypt(o.encode(slots), 24)
    pts = o.encode_diagonals(W, o.dense_scale(3))
    baby = [o.rotate(ct, j) for j in range(t1)]
    acc = None
    for k in range(t2):
        inner = None
        for j in range(t1):
            term = o.mul_plain(baby[j], pts[k * t1 + j])
            inner = term if inner is None else o.add(inner, term)
        rot = o.rotate(inner, k * t1)
        acc = rot if acc is None else o.add(acc, rot)
    assert np.array_equal(o.dense(ct, pts)[0], o.rescale(acc))


def test_dense_equals_direct_diagonal_method():
    # The diagonal method without baby-step/giant-step (t rotations) decodes to the same.
    N, m, n = 128, 8, 8
    t = 8
    o = small_ctx(N=N, rots=list(range(1, 8)))
    rng = np.random.default_rng(14)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(N // 2); slots[:n] = x; slots[t:t + n] = x
    ct = o.encrypt(o.encode(slots), 15)
    sc = o.dense_scale(3)
    acc = None
    for i in range(t):
        diag = np.zeros(N // 2)
        diag[:t] = [W[r, (r + i) % t] for r in range(t)]
        term = o.mul_plain(o.rotate(ct, i), o.encode(diag, sc))
        acc = term if acc is None else o.add(acc, term)
    direct = o.decode(o.decrypt(o.rescale(acc)), N // 2)
    pts = o.encode_diagonals(W, sc)
    bsgs = o.decode(o.decrypt(o.dense(ct, pts)[0]), N // 2)
    assert np.max(np.abs(direct - bsgs)) < 1e-6


@pytest.mark.parametrize("m,n,pb", [(16, 16, [60]), (32, 32, [50, 50]), (4, 8, [60])])
def test_dense_lazy_moddown_equals_composed_rotations(m, n, pb):
    """The lazy-ModDown form and the composition of whole rotations encrypt the same
    layer output: decoded values agree far inside the noise bound; and with only
    diagonal 0 non-zero (no rotation at all) both reduce to rescale(diag o ct) exactly
    (ModDown(P * x) = x)."""
    N = 128
    o = O.Oracle(N, [60, 40, 40, 40], pb, scale=2.0 ** 40)
    o.keygen(sorted(set(O.Oracle.bsgs_rotations(m, n) + O.Oracle.bsgs_rotations(m, n, True))), seed=3)
    t = O.Oracle.bsgs_t(m, n)
    rng = np.random.default_rng(m + 7 * n)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(N // 2); slots[:n] = x; slots[t:t + n] = x
    ct = o.encrypt(o.encode(slots), 21)
    pl = o.encode_diagonals(W, o.dense_scale(4), lazy=True)
    pc = o.encode_diagonals(W, o.dense_scale(4))
    lazy, c1 = o.dense(ct, pl, lazy=True)
    comp, c2 = o.dense(ct, pc)
    y1 = o.decode(o.decrypt(lazy), N // 2)
    y2 = o.decode(o.decrypt(comp), N // 2)
    assert np.max(np.abs(y1 - y2)) < 1e-7
    assert np.max(np.abs(y1[:m] - W @ x)) < 1e-6
    # only diagonal 0 non-zero: no key switch takes part in the result
    pz = np.zeros_like(pl); pz[0] = pl[0]
    a, _ = o.dense(ct, pz, lazy=True)
    b, _ = o.dense(ct, pz)
    assert np.array_equal(a, b)
    assert np.array_equal(a, o.rescale(o.mul_plain(ct, pl[0])))


def test_replicate():
    o = small_ctx(N=128, rots=(-16,))
    rng = np.random.default_rng(16)
    y = rng.uniform(-1, 1, 16)
    slots = np.zeros(64); slots[:16] = y
    ct = o.encrypt(o.encode(slots), 17)
    out = o.decode(o.decrypt(o.replicate(ct, 16)), 64)
    assert np.max(np.abs(out[:16] - y)) < 1e-7 and np.max(np.abs(out[16:32] - y)) < 1e-7
    assert np.max(np.abs(out[32:])) < 1e-7


def test_small_network_matches_fp64():
    """dense(16->8) -> x^2 -> replicate -> dense(8->4), the layer pattern of the paper's
    frozen stack with the square activation, decoded within 1e-4 of FP64."""
    N = 256
    r1 = O.Oracle.bsgs_rotations(8, 16)
    r2 = O.Oracle.bsgs_rotations(4, 8) + [-8]
    o = O.Oracle(N, [60, 40, 40, 40], [60], scale=2.0 ** 40)
    o.keygen(sorted(set(r1 + r2)), seed=3)
    rng = np.random.default_rng(18)
    W1 = rng.normal(0, 1 / 4, (8, 16)); W2 = rng.normal(0, 1 / np.sqrt(8), (4, 8))
    x = rng.uniform(-1, 1, 16)
    slots = np.zeros(N // 2); slots[:16] = x; slots[16:32] = x
    ct = o.encrypt(o.encode(slots), 19)
    sc = o.scale  # a dense layer restores Delta, the square squares it over q_last
    h = o.dense(ct, o.encode_diagonals(W1, o.dense_scale(4, sc)))[0]
    sc = o.scale
    h = o.square(h); sc = o.square_scale(3, sc)
    h = o.replicate(h, 8)
    h = o.dense(h, o.encode_diagonals(W2, o.dense_scale(2, sc)))[0]
    sc = o.scale
    y = o.decode(o.decrypt(h), 4, sc)
    ref = W2 @ (W1 @ x) ** 2
    assert np.max(np.abs(y - ref)) < 1e-4
