"""Pins of the oracle's other layers of the paper's frozen network (CPU only): the
ciphertext product, constant products and sums, level drop, the degree-3 ReLU
approximation, average pooling and the packed 1D convolution (Sec. 3.1), and the
paper's whole frozen stack (Sec. 4.1) with its stated depth of 6.

Each is checked against something other than the oracle: brute-force big-integer
products, the constant-polynomial closed form, numpy's correlation, FP64 plaintext
evaluation, and the operation counts the paper states.
"""
import numpy as np
import pytest

from oracle import ckks_oracle as O
from tests import netref


def py_negacyclic(a, b, q):
    N = len(a)
    full = np.convolve(np.array([int(x) for x in a], dtype=object), np.array([int(x) for x in b], dtype=object))
    full = list(full) + [0] * (2 * N - len(full))
    return [int((full[k] - full[k + N]) % q) for k in range(N)]


def ctx(N=128, q_bits=(50, 40, 40, 40), p_bits=(60,), rots=(1, 2, -1, -2), dnum=None, scale=2.0 ** 40):
    o = O.Oracle(N, list(q_bits), list(p_bits), dnum=dnum, scale=scale)
    o.keygen(rots, seed=3)
    return o


def enc(o, z, seed):
    return o.encrypt(o.encode(z), seed)


def dec(o, ct, scale, n=None):
    return o.decode(o.decrypt(ct), o.N // 2 if n is None else n, scale)


def test_tensor_bruteforce():
    o = ctx(N=16)
    rng = np.random.default_rng(1)
    a = np.stack([np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in o.moduli[:2]]) for _ in range(2)])
    b = np.stack([np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in o.moduli[:2]]) for _ in range(2)])
    d = o.tensor(a, b)
    for i in range(2):
        q = o.moduli[i]
        assert list(map(int, d[0, i])) == py_negacyclic(a[0, i], b[0, i], q)
        cross = [(u + v) % q for u, v in zip(py_negacyclic(a[0, i], b[1, i], q), py_negacyclic(a[1, i], b[0, i], q))]
        assert list(map(int, d[1, i])) == cross
        assert list(map(int, d[2, i])) == py_negacyclic(a[1, i], b[1, i], q)


def test_mul_of_two_ciphertexts_matches_fp64_and_square():
    o = ctx()
    rng = np.random.default_rng(2)
    za, zb = rng.uniform(-1, 1, 64), rng.uniform(-1, 1, 64)
    a, b = enc(o, za, 5), enc(o, zb, 6)
    out = o.mul(a, b)
    assert out.shape[1] == 3
    sc = o.scale * o.scale / o.moduli[3]
    assert np.max(np.abs(dec(o, out, sc) - za * zb)) < 1e-6
    # HMult(a, a) is the square activation, bit for bit
    assert np.array_equal(o.mul(a, a), o.square(a))


def test_mul_const_and_add_const_are_constant_plaintexts():
    o = ctx()
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, 64)
    ct = enc(o, z, 7)
    for C in (12345, -98765, 2 ** 40 + 3, 0):
        pt = np.zeros(o.N, dtype=np.int64)
        pt[0] = C  # the closed form of a constant slot vector's encoding
        assert np.array_equal(o.mul_const(ct, C), o.mul_plain(ct, pt))
        assert np.array_equal(o.add_const(ct, C), o.add_plain(ct, pt))
    C = int(round(-0.75 * o.moduli[3]))
    y = dec(o, o.rescale(o.mul_const(ct, C)), o.scale)
    assert np.max(np.abs(y - (-0.75) * z)) < 1e-6
    y = dec(o, o.add_const(ct, int(round(0.3 * o.scale))), o.scale)
    assert np.max(np.abs(y - (z + 0.3))) < 1e-6


def test_drop_level_keeps_values():
    o = ctx()
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, 64)
    ct = enc(o, z, 8)
    d = o.drop_level(ct, 2)
    assert d.shape == (2, 2, o.N)
    assert np.array_equal(d[:, :2], ct[:, :2])
    assert np.max(np.abs(dec(o, d, o.scale) - z)) < 1e-6


@pytest.mark.parametrize("which", ["paper", 0, 1, 2, 3])
def test_poly3_matches_fp64(which):
    """The paper's ReLU approximation, and each monomial alone (a dropped or misplaced
    term fails one of them); depth 2."""
    o = ctx(q_bits=(60, 40, 40, 40, 40))
    a = netref.relu_coeffs() if which == "paper" else [1.0 if i == which else 0.0 for i in range(4)]
    rng = np.random.default_rng(5)
    z = rng.uniform(-4, 4, 64)
    ct = enc(o, z, 9)
    out, sc = o.poly3(ct, o.scale, a)
    assert out.shape[1] == 3  # two levels consumed
    C, sc2 = o.poly3_consts(5, o.scale, a)
    assert sc2 == sc
    assert np.max(np.abs(dec(o, out, sc) - netref.poly3(a, z))) < 1e-6


def test_paper_relu_coefficients_approximate_relu():
    # the golden coefficients (Sec. 3.1) approximate max(z, 0) on the inputs the paper's
    # network sees; a sign or order slip in reading them breaks this
    a = netref.relu_coeffs()
    z = np.linspace(-3, 7, 101)
    assert np.max(np.abs(netref.poly3(a, z) - np.maximum(z, 0))) < 0.6
    assert abs(netref.poly3(a, 4.0) - 4.0) < 0.1


@pytest.mark.parametrize("f", [2, 3, 4])
def test_avgpool_matches_fp64_and_counts(f):
    o = ctx(rots=[-i for i in range(1, f)])
    rng = np.random.default_rng(6)
    z = rng.uniform(-1, 1, 64)
    ct = enc(o, z, 10)
    out, cnt = o.avgpool(ct, f)
    # Sec. 3.1: f-1 rotations, one plaintext (constant) product; f-1 additions here
    # (the paper counts f, with the bias-free sum read as f terms)
    assert cnt == [f - 1, 1, f - 1]
    want = sum(np.roll(z, i) for i in range(f)) / f  # rot_{-i} moves slot s to s + i
    assert np.max(np.abs(dec(o, out, o.scale) - want)) < 1e-6


@pytest.mark.parametrize("f,n,t", [(3, 10, 16), (9, 20, 32), (5, 28, 32)])
def test_conv1d_matches_numpy_and_counts(f, n, t):
    h = (f - 1) // 2
    o = ctx(rots=[i - h for i in range(f) if i != h])
    rng = np.random.default_rng(f * 10 + n)
    x = rng.uniform(-1, 1, n)
    w = rng.normal(0, 1 / np.sqrt(f), f)
    ct = enc(o, netref.replicated_slots(x, t, o.N // 2), 11)
    pts = o.encode_conv(w, n, t, o.dense_scale(4))
    out, cnt = o.conv1d(ct, pts)
    assert cnt == [f - 1, f, f - 1]  # Sec. 3.1: f products, f-1 rotations
    y = dec(o, out, o.scale)
    want = np.correlate(x, w, "same")
    if n + h <= t:  # the zero padding of the block holds the "same" boundary
        assert np.max(np.abs(y[:n] - want)) < 1e-6
        assert np.max(np.abs(y[t:t + n] - want)) < 1e-6
    assert np.max(np.abs(y[n:t])) < 1e-6 and np.max(np.abs(y[t + n:])) < 1e-6


def paper_net_oracle(o, ct, w, W1, W2s, a, n, t):
    """The paper's frozen stack on the oracle: conv(f) -> dense -> replicate ->
    ReLU_approx -> avgpool(3) -> dense; returns (ct, scale, level trace)."""
    lv = [ct.shape[1]]
    sc = o.scale
    h = o.conv1d(ct, o.encode_conv(w, n, t, o.dense_scale(ct.shape[1], sc)))[0]; lv.append(h.shape[1])
    h = o.dense(h, o.encode_diagonals(W1, o.dense_scale(h.shape[1], sc)))[0]; lv.append(h.shape[1])
    h = o.replicate(h, t)
    h, sc = o.poly3(h, sc, a); lv.append(h.shape[1])
    h = o.avgpool(h, 3)[0]; lv.append(h.shape[1])
    h = o.dense(h, o.encode_diagonals(W2s, o.dense_scale(h.shape[1], sc)))[0]; lv.append(h.shape[1])
    return h, o.scale, lv


def paper_net_rotations(n, m2, f, t):
    h = (f - 1) // 2
    r = [i - h for i in range(f) if i != h]
    r += O.Oracle.bsgs_rotations(n, n) + [-t, -1, -2] + O.Oracle.bsgs_rotations(m2, n)
    return sorted(set(r))


@pytest.mark.parametrize("q_bits,p_bits,log_scale,tol", [
    ((60, 40, 40, 40, 40, 40, 40), (60,), 40, 1e-4),
    ((34, 25, 25, 25, 25, 25, 25), (34,), 25, 1e-3),  # CryptoTL_p1's prime sizes (Tab. 1)
])
def test_paper_network_depth_6_matches_fp64(q_bits, p_bits, log_scale, tol):
    """Sec. 3.1 "Multiplicative Depth": the frozen network has depth 6, so 7 data primes
    leave one (q_0) at the output.  Scaled to n = 24 inputs (t = 32) at N = 256."""
    N, n, f = 256, 24, 9
    t = O.Oracle.bsgs_t(n, n)
    w, W1, W2, W2s = netref.paper_net_weights(n, f=f)
    m2 = W2.shape[0]
    o = ctx(N=N, q_bits=q_bits, p_bits=p_bits, rots=paper_net_rotations(n, m2, f, t), scale=2.0 ** log_scale)
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, n)
    a = netref.relu_coeffs()
    ct = enc(o, netref.replicated_slots(x, t, N // 2), 12)
    out, sc, lv = paper_net_oracle(o, ct, w, W1, W2s, a, n, t)
    assert lv == [7, 6, 5, 3, 2, 1]  # conv 1, dense 1, ReLU 2, pool 1, dense 1
    y = dec(o, out, sc, m2)
    assert np.max(np.abs(y - netref.paper_net_fp64(x, w, W1, W2, a))) < tol


def test_paper_predictions_per_ciphertext_windows():
    """Sec. 3.1 "Multiple Predictions": p = floor(#slots / (2 #neurons)) inputs share one
    ciphertext, each in its own window of 2t slots; every window's output equals the
    FP64 network of its own input.  N = 512 (256 slots), n = 24 (t = 32): p = 4."""
    N, n, f = 512, 24, 9
    t = O.Oracle.bsgs_t(n, n)
    p = (N // 2) // (2 * t)
    assert p == 4
    w, W1, W2, W2s = netref.paper_net_weights(n, f=f)
    m2 = W2.shape[0]
    o = ctx(N=N, q_bits=(60, 40, 40, 40, 40, 40, 40), p_bits=(60,), rots=paper_net_rotations(n, m2, f, t))
    rng = np.random.default_rng(8)
    xs = rng.uniform(-1, 1, (p, n))
    slots = np.zeros(N // 2)
    for k in range(p):
        slots[2 * t * k:2 * t * (k + 1)] = netref.replicated_slots(xs[k], t, 2 * t)
    a = netref.relu_coeffs()
    h = enc(o, slots, 13)
    sc = o.scale
    h = o.conv1d(h, o.encode_conv(w, n, t, o.dense_scale(7, sc), windows=p))[0]
    h = o.dense(h, o.encode_diagonals(W1, o.dense_scale(6, sc), windows=p))[0]
    h = o.replicate(h, t)
    h, sc = o.poly3(h, sc, a)
    h = o.avgpool(h, 3)[0]
    h = o.dense(h, o.encode_diagonals(W2s, o.dense_scale(2, sc), windows=p))[0]
    y = dec(o, h, o.scale)
    for k in range(p):
        assert np.max(np.abs(y[2 * t * k:2 * t * k + m2] - netref.paper_net_fp64(xs[k], w, W1, W2, a))) < 1e-4
    # windows = 1 reproduces the single-window encoding
    assert np.array_equal(o.encode_diagonals(W1, 2.0 ** 30), o.encode_diagonals(W1, 2.0 ** 30, windows=1))


def test_degenerate_cases():
    """Average pooling of size 1 is the identity at one level less (the constant q_last
    at scale q_last, then an exact division); the zero polynomial gives zero; a 1-tap
    convolution is a plaintext product."""
    o = ctx()
    rng = np.random.default_rng(20)
    z = rng.uniform(-1, 1, 64)
    ct = enc(o, z, 21)
    out, cnt = o.avgpool(ct, 1)
    assert cnt == [0, 1, 0]
    assert np.array_equal(out, o.drop_level(ct, 3))
    zero, sc = o.poly3(ct, o.scale, [0.0, 0.0, 0.0, 0.0])
    assert np.max(np.abs(dec(o, zero, sc))) < 1e-6
    pts = o.encode_conv([0.5], 10, 16, o.dense_scale(4))
    c1, cnt = o.conv1d(ct, pts)
    assert cnt == [0, 1, 0]
    assert np.array_equal(c1, o.rescale(o.mul_plain(ct, pts[0])))


def rect_model(W, x, tn, ns, fold):
    """FP64 slot vector of the rectangular dense form (its definition written out): the
    partial sums z[r] = sum_i rd_i[r] x~[r + i] over the tm diagonals of length tn, then the
    fold S = z; S += rot_s(S) for s = tn/2 .. tm; (fold = 2) S += rot_{-tm}(z)."""
    m, n = W.shape
    tm = 1
    while tm < m:
        tm <<= 1
    xt = np.zeros(ns)
    xt[:n] = x
    xt[tn:tn + n] = x
    z = np.zeros(ns)
    for r in range(tn):
        for i in range(tm):
            row, col = r % tm, (r + i) % tn
            if row < m and col < n:
                z[r] += W[row, col] * xt[r + i]
    S = z.copy()
    if fold >= 1:
        s = tn // 2
        while s >= tm:
            S = S + np.roll(S, -s)  # rot_s moves slot r + s to slot r
            s //= 2
    if fold == 2:
        S = S + np.roll(z, tm)
    return z, S


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("m,n", [(4, 16), (3, 12), (8, 32), (2, 64)])
@pytest.mark.parametrize("fold", [0, 1, 2])
def test_dense_rect_matches_its_fp64_definition(m, n, fold, lazy):
    # Rectangular diagonals (tm < tn): every slot of the decoded output against the FP64
    # partial sums and fold of the definition; after the fold, W x sits in slots [0, m)
    # (and [tm, tm + m) with fold = 2), as the dense layer of Sec. 3.1 computes.  lazy:
    # the BSGS part in the lazy-ModDown form (its own split), the same fold.
    rots = O.Oracle.rect_rotations(m, n, fold, lazy)
    o = ctx(N=256, rots=rots)
    rng = np.random.default_rng(m * 100 + n)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    tm, tn = O.Oracle.bsgs_t(m, 1), O.Oracle.bsgs_t(n, 1)
    ct = enc(o, netref.replicated_slots(x, tn, o.N // 2), 12)
    pts = o.encode_diagonals_rect(W, o.dense_scale(4), lazy)
    assert pts.shape == (tm, o.N)
    out, cnt = o.dense_rect(ct, pts, tn, fold=fold, lazy=lazy)
    t1 = O.Oracle.bsgs_t1(tm, lazy)
    folds = (tn // tm).bit_length() - 1 if fold >= 1 else 0
    extra = folds + (1 if fold == 2 else 0)
    assert cnt == [(t1 - 1) + (tm // t1 - 1) + extra, tm, tm - 1 + extra]
    assert len(set(rots)) == (t1 - 1) + (tm // t1 - 1) + extra
    y = dec(o, out, o.scale)
    _, S = rect_model(W, x, tn, o.N // 2, fold)
    assert np.max(np.abs(y - S)) < 1e-6
    if fold >= 1:
        assert np.max(np.abs(y[:m] - W @ x)) < 1e-6
    if fold == 2:
        assert np.max(np.abs(y[tm:tm + m] - W @ x)) < 1e-6


def test_dense_rect_rejects_square_shapes():
    o = ctx(N=256, rots=[1])
    with pytest.raises(RuntimeError):
        o.encode_diagonals_rect(np.ones((16, 16)), o.dense_scale(4))


def test_keyswitch_noise_matches_its_derivation():
    # The CryptoTL_p1 tolerances rest on netref.keyswitch_slot_sigma: the decoded error
    # that one key switch adds at scale 2^25 (N = 256, the paper's p1 prime sizes).  The
    # measured deviation of rot_1's slot errors must agree with it within a factor of 2.
    o = ctx(N=256, q_bits=[34] + [25] * 6, p_bits=[34], rots=[1], dnum=7, scale=2.0 ** 25)
    sd = netref.keyswitch_slot_sigma(256, [34] + [25] * 6, [34], 25)
    errs = []
    rng = np.random.default_rng(25)
    for t in range(4):
        z = rng.uniform(-1, 1, 128)
        ct = enc(o, z, 40 + t)
        errs.append(dec(o, o.rotate(ct, 1), 2.0 ** 25) - np.roll(z, -1))
    got = float(np.std(np.concatenate(errs)))
    assert 0.5 * sd < got < 2.0 * sd, (got, sd)
