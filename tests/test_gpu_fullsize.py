"""Bit-exact parity at the batched workload's full parameters (N = 16384, 8 x 45-bit
primes, 2 x 60-bit special primes, dnum = 4), for the operations the oracle computes in
seconds at that size: key generation, encryption, a rotation, a rescale and the square
activation, alone and inside a batch (the launch shape the benchmark times)."""
import numpy as np
import pytest

from oracle import ckks_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402


def test_cfg3_parameters_full_size_bit_exact():
    N, qb, pb, dnum = 16384, [45] * 8, [60, 60], 4
    o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    o.keygen([1], seed=3)
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    k = g.keygen([1], seed=3)
    assert g.moduli == o.moduli
    for kid in (0, g.galois_element(1)):
        assert np.array_equal(k.export(kid), o.key_export(kid))
    z = np.random.default_rng(130).uniform(-1, 1, N // 2)
    m = o.encode(z)
    ct_o = o.encrypt(m, 5)
    assert np.array_equal(g.encrypt_coeffs(k, m, 5).export()[0], ct_o)
    ct = g.ct_import(ct_o, 2.0 ** 40)
    rot = o.rotate(ct_o, 1)
    assert np.array_equal(g.rotate(k, ct, 1).export()[0], rot)
    assert np.array_equal(g.rescale(ct).export()[0], o.rescale(ct_o))
    sq = o.square(ct_o)
    assert np.array_equal(g.square(k, ct).export()[0], sq)
    # inside a batch of 8 different ciphertexts, member 5 is ct
    others = [o.encrypt(o.encode(np.full(N // 2, 0.1 * i)), 40 + i) for i in range(8)]
    others[5] = ct_o
    b = g.ct_import(np.stack(others), 2.0 ** 40)
    assert np.array_equal(g.rotate(k, b, 1).export()[5], rot)
    assert np.array_equal(g.square(k, b).export()[5], sq)


# ----------------------------------------------------------------------------- modular arithmetic
def _edge_inputs(q, rng, wide=True):
    top = (1 << 64) if wide else (1 << 63)
    vals = [0, 1, q - 1, q, q + 1, 2 * q - 1, 2 * q, 4 * q - 1, (1 << 32) - 1, 1 << 32, (1 << 63) - 1]
    if wide:
        vals += [1 << 63, (1 << 64) - 1, (1 << 64) - q]
    vals = [v for v in vals if 0 <= v < top]
    vals += [int(v) for v in rng.integers(0, top, 4000, dtype=np.uint64 if wide else np.int64)]
    return np.array(vals, dtype=np.uint64)


@pytest.mark.parametrize("bits", [34, 45, 50, 60, 61])
def test_modarith_primitives_exact(bits):
    """The kernels' Shoup, three-high-half Shoup, wide-reduction and Montgomery primitives
    against exact integer arithmetic (Python integers stand in for unsigned __int128) on
    edge and random 64-bit inputs, for primes of the sizes the parameter sets use."""
    q = O.primes(16384, [bits])[0]
    rng = np.random.default_rng(bits)
    xs = _edge_inputs(q, rng)
    xi = [int(v) for v in xs]
    for w in (1, 2, q - 1, int(rng.integers(0, q)), int(rng.integers(0, q))):
        wsh = (w << 64) // q
        r0 = ctl.modarith_eval(0, xs, q, w, wsh)
        r1 = ctl.modarith_eval(1, xs, q, w, wsh)
        r2 = ctl.modarith_eval(2, xs, q, w, wsh)
        for x, a, b, c in zip(xi, r0, r1, r2):
            exact = (x * w) % q
            assert int(a) == exact, ("shoup", x, w)
            assert int(b) % q == exact and int(b) < 2 * q, ("shoup_lazy", x, w)
            assert int(c) % q == exact and int(c) < 4 * q, ("shoup_small", x, w)
        bmont = w  # any w < q: mulmod_mont returns x * w * 2^-64 mod q
        r4 = ctl.modarith_eval(4, xs, q, bmont, 0, aux=pow(q, -1, 1 << 64))
        rinv = pow(1 << 64, -1, q)
        for x, a in zip(xi, r4):
            assert int(a) == (x * bmont * rinv) % q, ("mulmod_mont", x, w)
    # reduce_wide: any x < 2^63 (primes above 2^32)
    if q > (1 << 32):
        xw = _edge_inputs(q, rng, wide=False)
        r3 = ctl.modarith_eval(3, xw, q, aux=(1 << 64) // q)
        for x, a in zip(xw, r3):
            assert int(a) == int(x) % q, ("reduce_wide", int(x))
    x4 = np.array([0, 1, q - 1, q, 2 * q - 1, 2 * q, 3 * q + 5, 4 * q - 1] +
                  [int(v) for v in rng.integers(0, 4 * q, 2000, dtype=np.uint64)], dtype=np.uint64)
    r5 = ctl.modarith_eval(5, x4, q)
    assert all(int(a) == int(x) % q for x, a in zip(x4, r5))


# ----------------------------------------------------------------------------- NTT extremes
def _brv(k, logn):
    return int(format(k, f"0{logn}b")[::-1], 2)


@pytest.mark.parametrize("shape", [0, 1])
def test_ntt_16384_all_q_minus_1(shape):
    """Every coefficient q - 1 on every limb, the largest values the small-prime path (45-bit
    primes, no reduction inside the stages) and the general path (60/61-bit) receive.  The
    NTT of the constant polynomial c * sum_i X^i has the closed form c * (1 - w^N) / (1 - w)
    = 2c / (1 - w) at w = psi^(2 brv(k) + 1) (w^N = -1), checked on every output, and one
    limb against the oracle's direct evaluation; the inverse gives the input back."""
    N, logn = 16384, 14
    qb = [45, 45, 60, 61]
    o = O.Oracle(N, qb, [60])
    g = ctl.Context(N, qb, [60])
    g.set_ntt_shape(shape, shape)
    L = len(qb)
    a = np.stack([np.full(N, q - 1, dtype=np.uint64) for q in o.moduli[:L]])[None]
    x = to_dev(a)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    g.ntt_dev(x.data_ptr(), y.data_ptr(), 1, L)
    g.synchronize()
    got = from_dev(y, a.shape)
    for i in range(L):
        q, psi = o.moduli[i], o.psis[i]
        for k in range(N):
            w = pow(psi, 2 * _brv(k, logn) + 1, q)
            want = ((q - 1) * 2 * pow((1 - w) % q, -1, q)) % q
            assert int(got[0, i, k]) == want, (i, k)
    assert np.array_equal(got[0, 0], o.ntt_direct(0, a[0, 0]))
    z = torch.empty_like(x)
    g.ntt_dev(y.data_ptr(), z.data_ptr(), 1, L, inverse=True)
    g.synchronize()
    assert np.array_equal(from_dev(z, a.shape), a)
    g.close()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def from_dev(t, shape):
    return t.cpu().numpy().view(np.uint64).reshape(shape)


# ----------------------------------------------------------------------------- dense at full size
_FULL = {}


def _full_pair(rots):
    """Oracle and library at the batched workload's parameters with the keys of rots."""
    N, qb, pb, dnum = 16384, [45] * 8, [60, 60], 4
    key = tuple(sorted(rots))
    if key not in _FULL:
        o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
        o.keygen(list(key), seed=3)
        g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
        k = g.keygen(list(key), seed=3)
        _FULL.clear()
        _FULL[key] = (o, g, k)
    return _FULL[key]


@pytest.mark.parametrize("budget", [0, 1])
def test_dense_64_full_size_bit_exact(budget):
    """Eq. (bsgs) at N = 16384 with 45-bit primes, two 60-bit special primes, dnum = 4: a
    64 x 64 layer (t1 = t2 = 8: 7 hoisted baby steps, 7 giant steps through the summed
    giant-step ModDown) bit-exact against the oracle, alone and as member 1 of a batch of
    3.  budget = 1 caps the key-switching temporaries at one rotation per chunk, so the
    giant-step sums run over seven chunks (first chunk and accumulating chunks)."""
    m = n = 64
    rots = O.Oracle.bsgs_rotations(m, n)
    o, g, k = _full_pair(rots)
    N = 16384
    rng = np.random.default_rng(640)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    t = O.Oracle.bsgs_t(m, n)
    cts = []
    for i in range(3):
        x = rng.uniform(-1, 1, n)
        slots = np.zeros(N // 2)
        slots[:n] = x
        slots[t:t + n] = x
        cts.append(o.encrypt(o.encode(slots), 700 + i))
    lvl = 8
    sc = o.dense_scale(lvl)
    pts = o.encode_diagonals(W, sc)
    if budget:
        g.set_keyswitch_budget(1)
    try:
        exp = _cached_dense(o, cts[1], pts)
        assert np.array_equal(g.dense_coeffs(k, g.ct_import(cts[1], 2.0 ** 40), pts, sc).export()[0], exp)
        out = g.dense_coeffs(k, g.ct_import(np.stack(cts), 2.0 ** 40), pts, sc).export()
        assert np.array_equal(out[1], exp)
    finally:
        g.set_keyswitch_budget(16 << 30)


_DENSE_EXP = {}


def _cached_dense(o, ct, pts):
    key = (ct.tobytes()[:64], pts.tobytes()[:64])
    if key not in _DENSE_EXP:
        _DENSE_EXP[key] = o.dense(ct, pts)[0]
    return _DENSE_EXP[key]


def test_dense_rect_full_size_bit_exact():
    """The rectangular form at N = 16384 with the batched workload's primes: a 16 x 64 layer
    (tm = 16, tn = 64: 6 BSGS rotations, a fold of two and the [y, y] rotation), bit-exact
    against the oracle alone and as member 2 of a batch of 3."""
    m, n = 16, 64
    rots = O.Oracle.rect_rotations(m, n, 2)
    o, g, k = _full_pair(rots)
    N = 16384
    rng = np.random.default_rng(1664)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    cts = []
    for i in range(3):
        x = rng.uniform(-1, 1, n)
        slots = np.zeros(N // 2)
        slots[:n] = x
        slots[n:2 * n] = x
        cts.append(o.encrypt(o.encode(slots), 800 + i))
    sc = o.dense_scale(8)
    pts = o.encode_diagonals_rect(W, sc)
    exp = o.dense_rect(cts[2], pts, n, fold=2)[0]
    assert np.array_equal(g.dense_rect_coeffs(k, g.ct_import(cts[2], 2.0 ** 40), pts, n, sc, fold=2).export()[0], exp)
    out = g.dense_rect_coeffs(k, g.ct_import(np.stack(cts), 2.0 ** 40), pts, n, sc, fold=2).export()
    assert np.array_equal(out[2], exp)


def test_dense_rect_lazy_full_size_bit_exact():
    """The batched benchmark's dense form (rectangular, lazy-ModDown sums) at N = 16384: a
    16 x 64 layer with fold 2 bit-exact against the oracle, as member 0 of a batch of 2."""
    m, n = 16, 64
    rots = O.Oracle.rect_rotations(m, n, 2, lazy=True)
    o, g, k = _full_pair(rots)
    N = 16384
    rng = np.random.default_rng(1665)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    cts = []
    for i in range(2):
        x = rng.uniform(-1, 1, n)
        slots = np.zeros(N // 2)
        slots[:n] = x
        slots[n:2 * n] = x
        cts.append(o.encrypt(o.encode(slots), 900 + i))
    sc = o.dense_scale(8)
    pts = o.encode_diagonals_rect(W, sc, lazy=True)
    exp = o.dense_rect(cts[0], pts, n, fold=2, lazy=True)[0]
    g.set_dense_mode(g.DENSE_RECT_LAZY)
    try:
        out = g.dense_rect_coeffs(k, g.ct_import(np.stack(cts), 2.0 ** 40), pts, n, sc, fold=2).export()
    finally:
        g.set_dense_mode(g.DENSE_COMPOSED)
    assert np.array_equal(out[0], exp)
