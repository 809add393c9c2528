"""Host-side ciphertext messages (no GPU): round trips, the sizes Sec. 5.1 states
(client -> server: log2(q) * N bits; server -> client: log2(q_0) * 2N bits) against the
paper's Tab. 1, and the seeded form against the oracle's own encryption."""
import json
import os

import numpy as np
import pytest

from oracle import ckks_oracle as O
from paper_2205_11935_gb300 import ctl

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = {"CryptoTL_p1": (8192, [34] + [25] * 6, [34]), "CryptoTL_p2": (16384, [60] + [50] * 6, [60])}


def table1():
    with open(os.path.join(GOLD, "paper_params.json")) as f:
        return {p["name"]: p for p in json.load(f)["param_sets"]}


def rand_ct(N, moduli, level, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in moduli[:level]]) for _ in range(2)])


@pytest.mark.parametrize("name", list(PAPER))
def test_round_trip_and_sizes_against_table1(name):
    N, qb, pb = PAPER[name]
    moduli = ctl.plan_primes(N, qb + pb)
    L = len(qb)
    ct = rand_ct(N, moduli, L, 1)
    msg = ctl.serialize(N, moduli[:L], ct)
    assert np.array_equal(ctl.deserialize(msg, N, moduli[:L]), ct)
    tab = table1()[name]
    bits = [int(q).bit_length() for q in moduli]
    # server -> client: q_0 only after the six rescales, both polys (Sec. 5.1 formula)
    out = rand_ct(N, moduli, 1, 2)
    s2c = ctl.serialize(N, moduli[:1], out)
    assert len(s2c) == 16 + bits[0] * 2 * N // 8
    assert len(s2c) <= tab["s2c_kB"] * 1000
    # client -> server: the seeded fresh ciphertext is one ring element; its size is at
    # most log2(q) * N bits with q the whole modulus of Tab. 1 (data and special primes)
    c2s = len(ctl.serialize(N, moduli[:L], ct, seed=7))
    assert c2s == 16 + 8 + sum(bits[:L]) * N // 8
    assert c2s <= tab["log2_q"] * N // 8 + 24 and c2s <= tab["c2s_kB"] * 1000
    assert sum(bits) == tab["log2_q"]  # the chain's bit lengths add up to Tab. 1's log2 q


def test_seeded_message_regenerates_the_oracles_c1():
    N, qb, pb = 256, [60, 40, 40], [60]
    o = O.Oracle(N, qb, pb, scale=2.0 ** 40)
    o.keygen([], seed=3)
    z = np.random.default_rng(3).uniform(-1, 1, N // 2)
    ct = o.encrypt(o.encode(z), 1234)
    msg = ctl.serialize(N, o.moduli[:3], ct, seed=1234)
    back = ctl.deserialize(msg, N, o.moduli[:3])
    assert np.array_equal(back, ct)
    assert len(msg) < len(ctl.serialize(N, o.moduli[:3], ct))


def test_malformed_messages_are_refused():
    N = 64
    moduli = ctl.plan_primes(N, [50, 40])
    ct = rand_ct(N, moduli, 2, 5)
    msg = bytearray(ctl.serialize(N, moduli, ct))
    for bad in (bytes(msg[:-1]), b"XTL1" + bytes(msg[4:]), bytes(msg) + b"\0"):
        with pytest.raises(ctl.CtlError):
            ctl.deserialize(bad, N, moduli)
    with pytest.raises(ctl.CtlError):
        ctl.deserialize(bytes(msg), 2 * N, moduli)
    # a residue at or above its prime is refused on both sides
    big = ct.copy()
    big[0, 0, 0] = moduli[0]
    with pytest.raises(ctl.CtlError):
        ctl.serialize(N, moduli, big)
    # a message of a deeper level than the caller accepts
    with pytest.raises(ctl.CtlError):
        ctl.deserialize(bytes(msg), N, moduli[:1])


@pytest.mark.parametrize("log_scale", [30, 80, 100])
def test_encode_residues_matches_the_oracle_encoding(log_scale):
    """Residue encoding at scales beyond 64-bit coefficients (a bias before a rescale):
    the CRT value of the residues, divided by 2^(s-30), is the oracle's 2^30 encoding
    within one unit plus the FP64 rounding of the large product."""
    from sympy.ntheory.modular import crt

    N = 256
    moduli = ctl.plan_primes(N, [60, 50, 50, 50])
    o = O.Oracle(N, [60, 50, 50, 50], [60], scale=2.0 ** 30)
    z = np.random.default_rng(4).uniform(-1, 1, N // 2)
    res = ctl.encode_residues(N, moduli, z, 2.0 ** log_scale)
    ref = o.encode(z, 2.0 ** 30)
    Q = 1
    for q in moduli:
        Q *= q
    shift = 2 ** (log_scale - 30)
    for k in range(0, N, 7):
        v = int(crt(moduli, [int(r[k]) for r in res])[0])
        v = v - Q if v > Q // 2 else v
        assert abs(v / shift - int(ref[k])) <= 1 + abs(int(ref[k])) * 2.0 ** -50
    if log_scale == 30:  # within 64 bits: the same rounding as the 64-bit encoder, mod q
        for i, q in enumerate(moduli):
            assert np.array_equal(res[i], (ref.astype(object) % q).astype(np.uint64))


@pytest.mark.parametrize("seeded", [False, True])
def test_key_messages_round_trip_and_seeded_form_regenerates_the_oracles_keys(seeded):
    """The seeded key message carries only the b parts; the receiver draws the a parts
    again from the key-generation streams.  Pinned against the oracle's own key
    generation (an independent implementation of the generator and the stream ids)."""
    N, qb, pb, dnum = 256, [45, 45, 45, 45], [60, 60], 2
    o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    o.keygen([1, -4], seed=11)
    for r in (None, 1, -4):
        kid = 0 if r is None else o.galois_element(r)
        key = o.key_export(kid)
        msg = ctl.serialize_key(N, o.moduli, kid, key, seed=11 if seeded else None)
        got_id, back = ctl.deserialize_key(msg, N, o.moduli, o.beta)
        assert got_id == kid and np.array_equal(back, key)
    full = ctl.serialize_key(N, o.moduli, 0, o.key_export(0))
    half = ctl.serialize_key(N, o.moduli, 0, o.key_export(0), seed=11)
    assert len(half) - 8 - 20 == (len(full) - 20) // 2


def test_key_message_sizes_for_the_batched_parameters():
    # N = 16384, 8 x 45-bit + 2 x 60-bit primes, 4 digits: 4 x 2 x 983,040 bytes, or half seeded
    N = 16384
    moduli = ctl.plan_primes(N, [45] * 8 + [60, 60])
    m = np.asarray(moduli, dtype=np.uint64)
    import ctypes as C
    size = ctl.lib().ctl_key_message_size(N, m.ctypes.data_as(C.POINTER(C.c_uint64)), 10, 4, 0)
    seeded = ctl.lib().ctl_key_message_size(N, m.ctypes.data_as(C.POINTER(C.c_uint64)), 10, 4, 1)
    per = (8 * 45 + 2 * 60) * N // 8
    assert size == 20 + 8 * per and seeded == 28 + 4 * per


def test_malformed_key_messages_are_refused():
    N = 64
    moduli = ctl.plan_primes(N, [50, 40, 60])
    rng = np.random.default_rng(6)
    key = np.stack([np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in moduli])
                              for _ in range(2)]) for _ in range(2)])
    msg = ctl.serialize_key(N, moduli, 5, key)
    assert np.array_equal(ctl.deserialize_key(msg, N, moduli, 2)[1], key)
    for bad in (msg[:-1], b"CTL1" + msg[4:], msg + b"\0"):
        with pytest.raises(ctl.CtlError):
            ctl.deserialize_key(bad, N, moduli, 2)
    with pytest.raises(ctl.CtlError):
        ctl.deserialize_key(msg, N, moduli, 3)  # another digit count
    big = key.copy()
    big[1, 0, 2, 7] = moduli[2]
    with pytest.raises(ctl.CtlError):
        ctl.serialize_key(N, moduli, 5, big)
