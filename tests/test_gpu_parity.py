"""GPU parity: the CUDA path (through the C-ABI) against the CKKS oracle.

Integer outputs (NTT limbs, keys, ciphertexts) must be bit-exact; decoded values must be
within 1e-4 max-abs of the FP64 plaintext computation (at scale 2^40).  Bit-exact tests
inject the oracle's integer plaintexts (two FP64 encoders may round a coefficient
differently), and the GPU's own encoder is checked against the oracle's within one unit.
"""
import numpy as np
import pytest

from oracle import ckks_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402

TOL = 1e-4

# (N, q_bits, p_bits, dnum): cfg1-like (alpha 1), cfg3-like (alpha 2, two special primes),
# cfg2-like (60-bit q0)
PARAMS = {
    "a1": (64, [50, 40, 40], [60], 3),
    "a2": (256, [45, 45, 45, 45], [60, 60], 2),
    "c2": (1024, [60, 40, 40, 40], [60], 4),
}
ROTS = [1, 2, 3, 5, 7, -4, -8, 12]


class Pair:
    def __init__(self, name, rots=ROTS, seed=3):
        N, qb, pb, dnum = PARAMS[name]
        self.o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
        self.o.keygen(rots, seed=seed)
        self.g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
        self.k = self.g.keygen(rots, seed=seed)
        self.N = N

    def fresh(self, seed=11, z=None):
        rng = np.random.default_rng(seed)
        if z is None:
            z = rng.uniform(-1, 1, self.N // 2)
        m = self.o.encode(z)
        return z, self.o.encrypt(m, seed)


_cache = {}


def pair(name):
    if name not in _cache:
        _cache[name] = Pair(name)
    return _cache[name]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def from_dev(t, shape):
    return t.cpu().numpy().view(np.uint64).reshape(shape)


# ----------------------------------------------------------------------------- NTT
@pytest.mark.parametrize("N,shape", [(16, 0), (32, 0), (64, 0), (256, 0), (1024, 0), (4096, 0), (4096, 1),
                                     (8192, 0), (8192, 1)])
def test_ntt_matches_definition(N, shape):
    o = O.Oracle(N, [50, 40, 61], [60])
    g = ctl.Context(N, [50, 40, 61], [60])
    g.set_ntt_shape(shape, shape)  # both register shapes (N = 4096 .. 16384)
    rng = np.random.default_rng(N)
    limbs = 4
    a = np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in o.moduli[:limbs]])[None]
    a[0, 0, :3] = 0
    a[0, 1, :3] = np.uint64(o.moduli[1] - 1)  # edge values
    x = to_dev(a)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    g.ntt_dev(x.data_ptr(), y.data_ptr(), 1, limbs)
    g.synchronize()
    got = from_dev(y, a.shape)
    check = range(limbs) if N <= 1024 else ([0, 3] if N <= 4096 else [2])
    for i in check:
        assert np.array_equal(got[0, i], o.ntt_direct(i, a[0, i])), f"limb {i}"
    z = torch.empty_like(x)
    g.ntt_dev(y.data_ptr(), z.data_ptr(), 1, limbs, inverse=True)
    g.synchronize()
    assert np.array_equal(from_dev(z, a.shape), a)
    g.close()


@pytest.mark.parametrize("N", [4096, 8192])
def test_ntt_many_limbs_per_block(N):
    """Thousands of limbs at N = 4096 and 8192, several per CTA (the 16-element kernels go on
    to a CTA's next limb without a block-wide barrier): both register shapes give the same
    transform of every limb, the inverse returns the input, and sampled limbs, among them the
    last, equal the oracle's direct evaluation."""
    o = O.Oracle(N, [50, 40, 61], [60])
    g = ctl.Context(N, [50, 40, 61], [60])
    limbs, polys = 3, (1200 if N == 4096 else 600)
    rng = np.random.default_rng(N + 7)
    a = np.empty((polys, limbs, N), dtype=np.uint64)
    for i in range(limbs):
        a[:, i] = rng.integers(0, o.moduli[i], (polys, N), dtype=np.uint64)
    a[-1, 1, :5] = np.uint64(o.moduli[1] - 1)  # edge values in the last limb of a CTA's run
    x = to_dev(a)
    fwd = {}
    for shape in (0, 1):
        g.set_ntt_shape(shape, shape)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        torch.cuda.synchronize()
        g.ntt_dev(x.data_ptr(), y.data_ptr(), polys, limbs)
        g.ntt_dev(y.data_ptr(), z.data_ptr(), polys, limbs, inverse=True)
        g.synchronize()
        assert torch.equal(z, x), f"shape {shape}: inverse of forward"
        fwd[shape] = y
    assert torch.equal(fwd[0], fwd[1])
    for p, i in ((polys - 1, 1), (polys // 2, 0), (1, 2)):
        got = from_dev(fwd[1][p, i].contiguous(), (N,))
        assert np.array_equal(got, o.ntt_direct(i, a[p, i])), f"poly {p}, limb {i}"
    g.close()


@pytest.mark.parametrize("shape", [0, 1])
def test_ntt_16384_convolution_and_batch(shape):
    """N = 16384 (the batched workload's ring): NTT-domain product equals the schoolbook
    negacyclic product; a batch of polys transforms like each alone (both NTT shapes)."""
    N = 16384
    o = O.Oracle(N, [45, 45], [60])
    g = ctl.Context(N, [45, 45], [60])
    g.set_ntt_shape(shape, shape)
    rng = np.random.default_rng(5)
    q = o.moduli[0]
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    ab = np.zeros((3, 3, N), dtype=np.uint64)  # 3 polys x 3 limbs
    for p in range(3):
        for i in range(3):
            ab[p, i] = rng.integers(0, g.moduli[i], N, dtype=np.uint64)
    ab[0, 0], ab[1, 0] = a, b
    x = to_dev(ab)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    g.ntt_dev(x.data_ptr(), y.data_ptr(), 3, 3)
    g.synchronize()
    Y = from_dev(y, ab.shape)
    prod = np.array([(int(u) * int(v)) % q for u, v in zip(Y[0, 0], Y[1, 0])], dtype=np.uint64)
    pd = to_dev(prod[None, None])
    out = torch.empty_like(pd)
    torch.cuda.synchronize()
    g.ntt_dev(pd.data_ptr(), out.data_ptr(), 1, 1, inverse=True)
    g.synchronize()
    assert np.array_equal(from_dev(out, (N,)), o.polymul(0, a, b))
    # each poly of the batch alone
    for p in (1, 2):
        x1 = to_dev(ab[p:p + 1])
        y1 = torch.empty_like(x1)
        torch.cuda.synchronize()
        g.ntt_dev(x1.data_ptr(), y1.data_ptr(), 1, 3)
        g.synchronize()
        assert np.array_equal(from_dev(y1, (1, 3, N))[0], Y[p])
    g.close()


# ----------------------------------------------------------------------------- keys / encryption
@pytest.mark.parametrize("name", list(PARAMS))
def test_primes_and_keys_bit_exact(name):
    P = pair(name)
    assert P.g.moduli == P.o.moduli
    for r in (None, 1, -4):
        kid = 0 if r is None else P.o.galois_element(r)
        assert np.array_equal(P.k.export(kid), P.o.key_export(kid)), f"key {kid}"


@pytest.mark.parametrize("name", list(PARAMS))
def test_encrypt_decrypt_bit_exact(name):
    P = pair(name)
    z, ct_o = P.fresh(21)
    m = P.o.encode(z)
    ct = P.g.encrypt_coeffs(P.k, m, 21)
    assert np.array_equal(ct.export()[0], ct_o)
    assert np.array_equal(P.g.decrypt_coeffs(P.k, ct), P.o.decrypt(ct_o))
    assert np.max(np.abs(P.g.decrypt(P.k, ct, P.N // 2) - z)) < TOL


@pytest.mark.parametrize("name", list(PARAMS))
def test_encoder_within_one_unit(name):
    P = pair(name)
    rng = np.random.default_rng(22)
    for scale in (2.0 ** 40, 2.0 ** 50):
        z = rng.uniform(-1, 1, P.N // 2)
        d = np.abs(P.g.encode(z, scale) - P.o.encode(z, scale))
        assert d.max() <= 1
    z = rng.uniform(-1, 1, P.N // 2)
    m = P.o.encode(z).astype(np.float64)
    assert np.max(np.abs(P.g.decode(m, P.N // 2) - P.o.decode(m, P.N // 2))) < 1e-9


# ----------------------------------------------------------------------------- operations
@pytest.mark.parametrize("name", list(PARAMS))
@pytest.mark.parametrize("r", [1, 3, -4, 12, 0])
def test_rotate_bit_exact(name, r):
    P = pair(name)
    z, ct_o = P.fresh(30)
    ct = P.g.ct_import(ct_o, 2.0 ** 40)
    out = P.g.rotate(P.k, ct, r)
    assert np.array_equal(out.export()[0], P.o.rotate(ct_o, r))


@pytest.mark.parametrize("name", list(PARAMS))
def test_rotate_batch_and_lower_level(name):
    P = pair(name)
    cts = [P.fresh(40 + i)[1] for i in range(3)]
    low = [P.o.rescale(c) for c in cts]
    b = P.g.ct_import(np.stack(low), 2.0 ** 40 / P.o.moduli[len(P.o.moduli) - P.o.K - 1])
    out = P.g.rotate(P.k, b, 5).export()
    for i in range(3):
        assert np.array_equal(out[i], P.o.rotate(low[i], 5))


@pytest.mark.parametrize("name", list(PARAMS))
def test_rescale_bit_exact(name):
    P = pair(name)
    _, ct_o = P.fresh(50)
    ct = P.g.ct_import(ct_o, 2.0 ** 40)
    r1 = P.g.rescale(ct)
    e1 = P.o.rescale(ct_o)
    assert np.array_equal(r1.export()[0], e1)
    r2 = P.g.rescale(r1)
    assert np.array_equal(r2.export()[0], P.o.rescale(e1))


@pytest.mark.parametrize("name", list(PARAMS))
def test_square_bit_exact_and_fp64(name):
    P = pair(name)
    z, ct_o = P.fresh(60)
    ct = P.g.ct_import(ct_o, 2.0 ** 40)
    sq = P.g.square(P.k, ct)
    exp = P.o.square(ct_o)
    assert np.array_equal(sq.export()[0], exp)
    assert np.max(np.abs(P.g.decrypt(P.k, sq, P.N // 2) - z * z)) < TOL


@pytest.mark.parametrize("name", list(PARAMS))
def test_mul_plain_and_add(name):
    P = pair(name)
    z, ct_o = P.fresh(65)
    pt = P.o.encode(np.linspace(-1, 1, P.N // 2), 2.0 ** 30)
    ct = P.g.ct_import(ct_o, 2.0 ** 40)
    assert np.array_equal(P.g.mul_plain_coeffs(ct, pt, 2.0 ** 30).export()[0], P.o.mul_plain(ct_o, pt))
    assert np.array_equal(P.g.add(ct, ct).export()[0], P.o.add(ct_o, ct_o))


def dense_case(P, m, n, seed):
    rng = np.random.default_rng(seed)
    t = O.Oracle.bsgs_t(m, n)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(P.N // 2)
    slots[:n] = x
    slots[t:t + n] = x
    z, ct_o = P.fresh(seed, z=slots)
    return W, x, t, ct_o


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("name,m,n", [("a1", 8, 16), ("a1", 5, 12), ("a2", 16, 16), ("c2", 32, 64), ("c2", 3, 1),
                                      ("c2", 128, 128)])
def test_dense_bit_exact_injected_and_fp64(name, m, n, lazy):
    P = pair(name)
    rots = sorted(set(O.Oracle.bsgs_rotations(m, n, lazy)))
    o = O.Oracle(P.N, *PARAMS[name][1:3], dnum=PARAMS[name][3], scale=2.0 ** 40)
    o.keygen(rots, seed=3)
    g = P.g
    k = g.keygen(rots, seed=3)
    W, x, t, ct_o = dense_case(P, m, n, 70 + m)
    lvl = ct_o.shape[1]
    sc = o.dense_scale(lvl)
    pts = o.encode_diagonals(W, sc, lazy)
    exp, cnt = o.dense(ct_o, pts, lazy=lazy)
    ct = g.ct_import(ct_o, 2.0 ** 40)
    g.set_dense_mode(g.DENSE_LAZY_MODDOWN if lazy else g.DENSE_COMPOSED)
    try:
        g.stats_reset()
        out = g.dense_coeffs(k, ct, pts, sc)
        ops = g.stats_ops()
        assert np.array_equal(out.export()[0], exp)
        assert ops["rotations"] == cnt[0] and ops["ptmul"] == cnt[1] and ops["add"] == cnt[2]
        # the library's own diagonal encoding: decoded within tolerance of FP64, output at Delta
        out2 = g.dense(k, ct, W)
        assert out2.info()[2] == 2.0 ** 40
        y = g.decrypt(k, out2, P.N // 2)
        assert np.max(np.abs(y[:m] - W @ x)) < TOL
        assert np.max(np.abs(y[m:])) < TOL
    finally:
        g.set_dense_mode(g.DENSE_COMPOSED)
    k.close()


def test_dense_mode_argument():
    P = pair("a1")
    with pytest.raises(ctl.CtlError):
        P.g.set_dense_mode(7)


@pytest.mark.parametrize("name", list(PARAMS))
def test_replicate_bit_exact(name):
    P = pair(name)
    _, ct_o = P.fresh(80)
    ct = P.g.ct_import(ct_o, 2.0 ** 40)
    assert np.array_equal(P.g.replicate(P.k, ct, 8).export()[0], P.o.replicate(ct_o, 8))


# ----------------------------------------------------------------------------- networks
def network_case(N, q_bits, p_bits, dnum, dims, seed=90, sizes_only=False):
    """dense(d0->d1) -> x^2 -> replicate -> dense(d1->d2) ... with FP64 reference."""
    rng = np.random.default_rng(seed)
    Ws = [rng.normal(0, 1 / np.sqrt(dims[i]), (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    x = rng.uniform(-1, 1, dims[0])
    layers = []
    ref = x.copy()
    for i, W in enumerate(Ws):
        layers.append(("dense", W))
        ref = W @ ref
        if i + 1 < len(Ws):
            layers.append(("square",))
            ref = ref * ref
            t_next = O.Oracle.bsgs_t(Ws[i + 1].shape[0], Ws[i + 1].shape[1])
            layers.append(("replicate", t_next))
    t0 = O.Oracle.bsgs_t(Ws[0].shape[0], Ws[0].shape[1])
    slots = np.zeros(N // 2)
    slots[:dims[0]] = x
    slots[t0:t0 + dims[0]] = x
    return layers, slots, ref


def oracle_forward(o, ct, layers, lazy=False):
    sc = o.scale  # a dense layer restores Delta, a square squares the scale over q_last
    for ly in layers:
        lvl = ct.shape[1]
        if ly[0] == "dense":
            ct = o.dense(ct, o.encode_diagonals(ly[1], o.dense_scale(lvl, sc), lazy), lazy=lazy)[0]
            sc = o.scale
        elif ly[0] == "square":
            ct = o.square(ct)
            sc = o.square_scale(lvl, sc)
        else:
            ct = o.replicate(ct, ly[1])
    return ct, sc


def inject(o, layers, lazy=False):
    """Same layers with the oracle's diagonal coefficients attached."""
    out, sc, lvl = [], o.scale, o.L
    for ly in layers:
        if ly[0] == "dense":
            out.append(("dense", ly[1], None, o.encode_diagonals(ly[1], o.dense_scale(lvl, sc), lazy)))
            sc = o.scale
            lvl -= 1
        elif ly[0] == "square":
            out.append(ly)
            sc = o.square_scale(lvl, sc)
            lvl -= 1
        else:
            out.append(ly)
    return out


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("N,qb,pb,dnum,dims", [
    (256, [60, 40, 40, 40], [60], 4, [16, 8, 4]),
    (512, [45, 45, 45, 45, 45, 45], [60, 60], 3, [32, 16, 16, 8]),
])
def test_network_bit_exact_and_fp64(N, qb, pb, dnum, dims, lazy):
    layers, slots, ref = network_case(N, qb, pb, dnum, dims)
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    if lazy:
        g.set_dense_mode(g.DENSE_LAZY_MODDOWN)
    o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    model = ctl.Model(g, inject(o, layers, lazy))
    rots = model.rotations()
    o.keygen(rots, seed=3)
    k = g.keygen(rots, seed=3)
    ct_o = o.encrypt(o.encode(slots), 4)
    exp, sc = oracle_forward(o, ct_o, layers, lazy)
    out = model.forward(k, g.ct_import(ct_o, 2.0 ** 40))
    assert np.array_equal(out.export()[0], exp)
    y = g.decrypt(k, out, len(ref))
    assert np.max(np.abs(y - ref)) < TOL
    # the model with the library's own encoding
    model2 = ctl.Model(g, layers)
    y2 = g.decrypt(k, model2.forward(k, g.encrypt(k, slots, 4)), len(ref))
    assert np.max(np.abs(y2 - ref)) < TOL


@pytest.mark.parametrize("lazy,shape", [(False, 0), (False, 1), (True, 0)])
def test_cfg1_full_size_bit_exact(lazy, shape):
    """N = 4096, q {50,40,40} + 60-bit special prime, dense 64->32 then x^2 (single query),
    with both register NTT shapes."""
    N, qb, pb = 4096, [50, 40, 40], [60]
    rng = np.random.default_rng(1)
    W = rng.normal(0, 1 / 8, (32, 64))
    x = rng.uniform(-1, 1, 64)
    slots = np.zeros(N // 2)
    slots[:64] = x
    slots[64:128] = x
    layers = [("dense", W), ("square",)]
    g = ctl.Context(N, qb, pb, scale=2.0 ** 40)
    g.set_ntt_shape(shape, shape)
    if lazy:
        g.set_dense_mode(g.DENSE_LAZY_MODDOWN)
    o = O.Oracle(N, qb, pb, scale=2.0 ** 40)
    model = ctl.Model(g, inject(o, layers, lazy))
    rots = model.rotations()
    o.keygen(rots, seed=3)
    k = g.keygen(rots, seed=3)
    ct_o = o.encrypt(o.encode(slots), 4)
    exp, _ = oracle_forward(o, ct_o, layers, lazy)
    out = model.forward(k, g.ct_import(ct_o, 2.0 ** 40))
    assert np.array_equal(out.export()[0], exp)
    assert np.max(np.abs(g.decrypt(k, out, 32) - (W @ x) ** 2)) < TOL


def test_batch_equals_single():
    N, qb, pb = 1024, [60, 40, 40, 40], [60]
    layers, slots, ref = network_case(N, qb, pb, 4, [32, 16, 8])
    g = ctl.Context(N, qb, pb, scale=2.0 ** 40)
    model = ctl.Model(g, layers)
    k = g.keygen(model.rotations(), seed=3)
    rng = np.random.default_rng(7)
    singles = []
    for i in range(4):
        s = slots.copy() if i == 0 else np.concatenate([rng.uniform(-1, 1, 64), np.zeros(N // 2 - 64)])
        singles.append(g.encrypt(k, s, 100 + i))
    batch = g.concat(singles)
    outb = model.forward(k, batch).export()
    for i, s in enumerate(singles):
        assert np.array_equal(model.forward(k, s).export()[0], outb[i])


def test_error_codes():
    P = pair("a1")
    _, ct_o = P.fresh(99)
    ct = P.g.ct_import(ct_o, 2.0 ** 40)
    with pytest.raises(ctl.CtlError) as e:
        P.g.rotate(P.k, ct, 9)  # no key for 9
    assert e.value.code == -4
    low = P.g.rescale(P.g.rescale(ct))
    with pytest.raises(ctl.CtlError) as e:
        P.g.rescale(low)
    assert e.value.code == -2
    other = P.g.ct_import(ct_o, 2.0 ** 39)
    with pytest.raises(ctl.CtlError) as e:
        P.g.add(ct, other)
    assert e.value.code == -3
    with pytest.raises(ctl.CtlError) as e:
        ctl.Context(100, [40], [60])
    assert e.value.code == -1


@pytest.mark.parametrize("lazy", [False, True])
def test_ntt_shapes_agree_on_a_16384_network(lazy):
    """Both register NTT shapes (and so every fused ModUp / ModDown / rescale kernel of
    each) give the same ciphertext bits on the batched workload's ring and chain shape."""
    N, qb, pb, dnum = 16384, [45] * 5, [60, 60], 3
    layers, slots, ref = network_case(N, qb, pb, dnum, [64, 32, 16])
    outs = []
    for shape in (0, 1):
        g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
        g.set_ntt_shape(shape, shape)
        if lazy:
            g.set_dense_mode(g.DENSE_LAZY_MODDOWN)
        model = ctl.Model(g, layers)
        k = g.keygen(model.rotations(), seed=3)
        ct = g.concat([g.encrypt(k, slots, 4), g.encrypt(k, slots, 5)])
        out = model.forward(k, ct)
        outs.append(out.export())
        y = g.decrypt(k, out.slice(0), len(ref))
        assert np.max(np.abs(y - ref)) < TOL
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("chunk,kara", [(32, 0), (32, 1), (16, 0), (16, 1)])
def test_bsgs_shapes_bit_exact(chunk, kara):
    """Every shape of the inner-sum kernel (baby steps held per thread, three or four
    multiply-adds per split product) gives the oracle's dense layer, with t1 = 64 > chunk."""
    P = pair("c2")
    m = n = 256  # t = 256: t1 = 16 (default split) and 32 (lazy split)
    for lazy in (False, True):
        rots = sorted(set(O.Oracle.bsgs_rotations(m, n, lazy)))
        o = O.Oracle(P.N, *PARAMS["c2"][1:3], dnum=PARAMS["c2"][3], scale=2.0 ** 40)
        o.keygen(rots, seed=3)
        k = P.g.keygen(rots, seed=3)
        W, x, t, ct_o = dense_case(P, m, n, 91)
        sc = o.dense_scale(ct_o.shape[1])
        pts = o.encode_diagonals(W, sc, lazy)
        exp, _ = o.dense(ct_o, pts, lazy=lazy)
        P.g.set_bsgs_shape(chunk, kara)
        P.g.set_dense_mode(P.g.DENSE_LAZY_MODDOWN if lazy else P.g.DENSE_COMPOSED)
        try:
            out = P.g.dense_coeffs(k, P.g.ct_import(ct_o, 2.0 ** 40), pts, sc)
            assert np.array_equal(out.export()[0], exp)
        finally:
            P.g.set_bsgs_shape(32, 1)
            P.g.set_dense_mode(P.g.DENSE_COMPOSED)
        k.close()


@pytest.mark.parametrize("lazy", [False, True])
def test_keyswitch_chunks_bit_exact(lazy):
    """A key-switching budget of one byte forces one rotation per chunk: the baby steps
    and the giant-step sums (carried across chunks) give the oracle's dense layer, the
    same bits as the default single chunk, for a batch of two ciphertexts."""
    P = pair("c2")
    m = n = 256  # t = 256: 15 giant-step rotations in the default split
    rots = sorted(set(O.Oracle.bsgs_rotations(m, n, lazy)))
    o = O.Oracle(P.N, *PARAMS["c2"][1:3], dnum=PARAMS["c2"][3], scale=2.0 ** 40)
    o.keygen(rots, seed=3)
    k = P.g.keygen(rots, seed=3)
    W, x, t, ct_o = dense_case(P, m, n, 93)
    _, ct_o2 = P.fresh(94, z=None)
    sc = o.dense_scale(ct_o.shape[1])
    pts = o.encode_diagonals(W, sc, lazy)
    exp = [o.dense(c, pts, lazy=lazy)[0] for c in (ct_o, ct_o2)]
    P.g.set_dense_mode(P.g.DENSE_LAZY_MODDOWN if lazy else P.g.DENSE_COMPOSED)
    try:
        outs = []
        for budget in (1 << 34, 1):
            P.g.set_keyswitch_budget(budget)
            batch = P.g.concat([P.g.ct_import(ct_o, 2.0 ** 40), P.g.ct_import(ct_o2, 2.0 ** 40)])
            outs.append(P.g.dense_coeffs(k, batch, pts, sc).export())
        for got in outs:
            assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
    finally:
        P.g.set_keyswitch_budget(16 << 30)
        P.g.set_dense_mode(P.g.DENSE_COMPOSED)
    k.close()
    with pytest.raises(ctl.CtlError):
        P.g.set_keyswitch_budget(0)


def _fp64_forward(Ws, x, square_last):
    h = x
    for i, W in enumerate(Ws):
        h = W @ h
        if i + 1 < len(Ws) or square_last:
            h = h * h
    return h


@pytest.mark.parametrize("name,N,qb,pb,dnum,dims,B,mode", [
    ("cfg2", 8192, [60, 40, 40, 40], [60], 4, [512, 128, 64], 2, 0),
    ("cfg3", 16384, [45] * 8, [60, 60], 4, [1024, 256, 256, 64], 8, 0),
    ("cfg3", 16384, [45] * 8, [60, 60], 4, [1024, 256, 256, 64], 8, 3),
])
def test_full_size_networks_properties(name, N, qb, pb, dnum, dims, B, mode):
    """The single-query (N = 8192) and batched (N = 16384) networks at their full sizes,
    in the launch configuration bench.py times (mode 3: CTL_DENSE_RECT_LAZY, the batched
    benchmark's form): every decoded output within 1e-4 of the FP64 network, each
    ciphertext of the batch bit-identical to its forward alone, the CUDA-graph replay
    bit-identical to the eager forward, and two runs identical."""
    rng = np.random.default_rng(1)
    Ws = [rng.normal(0, 1 / np.sqrt(dims[i]), (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    layers = []
    for i, W in enumerate(Ws):
        layers.append(("dense", W))
        if i + 1 < len(Ws):
            layers += [("square",), ("replicate", O.Oracle.bsgs_t(*Ws[i + 1].shape))]
    t0 = O.Oracle.bsgs_t(*Ws[0].shape)
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    g.set_dense_mode(mode)
    model = ctl.Model(g, layers)
    k = g.keygen(model.rotations(), seed=3)
    xs, cts = [], []
    for i in range(B):
        x = rng.uniform(-1, 1, dims[0])
        s = np.zeros(N // 2)
        s[:dims[0]] = x
        s[t0:t0 + dims[0]] = x
        xs.append(x)
        cts.append(g.encrypt(k, s, 4 + i))
    batch = g.concat(cts)
    out = model.forward(k, batch)
    got = out.export()
    for i in range(B):
        y = g.decrypt(k, out.slice(i), dims[-1])
        assert np.max(np.abs(y - _fp64_forward(Ws, xs[i], False))) < TOL
    for i in (0, B - 1):
        assert np.array_equal(model.forward(k, cts[i]).export()[0], got[i])
    assert np.array_equal(model.forward(k, batch, graph=True).export(), got)
    assert np.array_equal(model.forward(k, batch).export(), got)


# ----------------------------------------------------------------------------- rectangular form
def rect_case(P, m, n, seed):
    rng = np.random.default_rng(seed)
    tn = O.Oracle.bsgs_t(n, 1)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(P.N // 2)
    slots[:n] = x
    slots[tn:tn + n] = x
    _, ct_o = P.fresh(seed, z=slots)
    return W, x, tn, ct_o


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("fold", [0, 1, 2])
@pytest.mark.parametrize("name,m,n", [("a1", 4, 16), ("a2", 8, 64), ("a2", 3, 40), ("c2", 32, 128), ("c2", 1, 64)])
def test_dense_rect_bit_exact_and_fp64(name, m, n, fold, lazy):
    """The rectangular form (tm < tn) against the oracle's, bit-exact, with its operation
    counts, in the composed and the lazy-ModDown forms; the library's own encoding decodes
    to W x in slots [0, m) (and [tm, tm + m) with fold 2)."""
    P = pair(name)
    rots = sorted(set(O.Oracle.rect_rotations(m, n, fold, lazy)))
    o = O.Oracle(P.N, *PARAMS[name][1:3], dnum=PARAMS[name][3], scale=2.0 ** 40)
    o.keygen(rots, seed=3)
    g = P.g
    k = g.keygen(rots, seed=3)
    W, x, tn, ct_o = rect_case(P, m, n, 170 + m)
    tm = O.Oracle.bsgs_t(m, 1)
    sc = o.dense_scale(ct_o.shape[1])
    pts = o.encode_diagonals_rect(W, sc, lazy)
    exp, cnt = o.dense_rect(ct_o, pts, tn, fold=fold, lazy=lazy)
    ct = g.ct_import(ct_o, 2.0 ** 40)
    g.set_dense_mode(g.DENSE_RECT_LAZY if lazy else g.DENSE_RECT)
    try:
        g.stats_reset()
        out = g.dense_rect_coeffs(k, ct, pts, tn, sc, fold=fold)
        ops = g.stats_ops()
        assert np.array_equal(out.export()[0], exp)
        assert ops["rotations"] == cnt[0] and ops["ptmul"] == cnt[1] and ops["add"] == cnt[2]
        if fold:
            y = g.decrypt(k, g.dense_rect(k, ct, W, fold=fold), P.N // 2)
            assert np.max(np.abs(y[:m] - W @ x)) < TOL
            if fold == 2:
                assert np.max(np.abs(y[tm:tm + m] - W @ x)) < TOL
    finally:
        g.set_dense_mode(g.DENSE_COMPOSED)
    k.close()


def test_dense_rect_arguments():
    P = pair("a2")
    W = np.ones((16, 16))
    ct = P.g.ct_import(P.fresh(5)[1], 2.0 ** 40)
    with pytest.raises(ctl.CtlError):
        P.g.dense_rect(P.k, ct, W)  # tm = tn: not rectangular
    with pytest.raises(ctl.CtlError):
        P.g.dense_rect(P.k, ct, np.ones((4, 128)))  # 2 tn > N/2


def oracle_forward_rect(o, ct, layers, lazy=False):
    """The oracle's forward under the rectangular mode: a dense layer with tm < tn takes
    the rectangular form, with fold 2 (and the next replicate(tm) not run) when
    [square,] replicate(tm) follows it; lazy: every Eq. (bsgs) in the lazy-ModDown form."""
    sc, skip = o.scale, set()
    for i, ly in enumerate(layers):
        lvl = ct.shape[1]
        if i in skip:
            continue
        if ly[0] == "dense":
            m, n = ly[1].shape
            tm, tn = O.Oracle.bsgs_t(m, 1), O.Oracle.bsgs_t(n, 1)
            if tm < tn:
                j = i + 1
                if j < len(layers) and layers[j][0] == "square":
                    j += 1
                fold = 1
                if j < len(layers) and layers[j][0] == "replicate" and layers[j][1] == tm:
                    fold = 2
                    skip.add(j)
                pts = o.encode_diagonals_rect(ly[1], o.dense_scale(lvl, sc), lazy)
                ct = o.dense_rect(ct, pts, tn, fold=fold, lazy=lazy)[0]
            else:
                ct = o.dense(ct, o.encode_diagonals(ly[1], o.dense_scale(lvl, sc), lazy), lazy=lazy)[0]
            sc = o.scale
        elif ly[0] == "square":
            ct = o.square(ct)
            sc = o.square_scale(lvl, sc)
        else:
            ct = o.replicate(ct, ly[1])
    return ct, sc


def inject_rect(o, layers, lazy=False):
    out, sc, lvl = [], o.scale, o.L
    for ly in layers:
        if ly[0] == "dense":
            m, n = ly[1].shape
            rect = O.Oracle.bsgs_t(m, 1) < O.Oracle.bsgs_t(n, 1)
            pts = (o.encode_diagonals_rect(ly[1], o.dense_scale(lvl, sc), lazy) if rect
                   else o.encode_diagonals(ly[1], o.dense_scale(lvl, sc), lazy))
            out.append(("dense", ly[1], None, pts))
            sc = o.scale
            lvl -= 1
        elif ly[0] == "square":
            out.append(ly)
            sc = o.square_scale(lvl, sc)
            lvl -= 1
        else:
            out.append(ly)
    return out


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("N,qb,pb,dnum,dims", [
    (256, [60, 40, 40, 40], [60], 4, [16, 8, 4]),
    (512, [45, 45, 45, 45, 45, 45], [60, 60], 3, [64, 16, 16, 4]),
])
def test_network_rect_bit_exact_and_fp64(N, qb, pb, dnum, dims, lazy):
    """A model under CTL_DENSE_RECT (the batched network's shape: shrinking layers take the
    rectangular form, the first one's fold forms the next layer's [y, y]) against the
    oracle's composition of the same layers, bit-exact, and FP64 within the tolerance."""
    layers, slots, ref = network_case(N, qb, pb, dnum, dims)
    t0 = O.Oracle.bsgs_t(dims[0], 1)
    slots = np.zeros(N // 2)
    x = network_case(N, qb, pb, dnum, dims)[1][:dims[0]]
    slots[:dims[0]] = x
    slots[t0:t0 + dims[0]] = x
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    g.set_dense_mode(g.DENSE_RECT_LAZY if lazy else g.DENSE_RECT)
    o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    model = ctl.Model(g, inject_rect(o, layers, lazy))
    rots = model.rotations()
    o.keygen(rots, seed=3)
    k = g.keygen(rots, seed=3)
    ct_o = o.encrypt(o.encode(slots), 4)
    exp, sc = oracle_forward_rect(o, ct_o, layers, lazy)
    out = model.forward(k, g.ct_import(ct_o, 2.0 ** 40))
    assert np.array_equal(out.export()[0], exp)
    assert np.array_equal(model.forward(k, g.ct_import(ct_o, 2.0 ** 40), graph=True).export()[0], exp)
    y = g.decrypt(k, out, len(ref))
    assert np.max(np.abs(y - ref)) < TOL
    model2 = ctl.Model(g, layers)  # the library's own encoding
    y2 = g.decrypt(k, model2.forward(k, g.encrypt(k, slots, 4)), len(ref))
    assert np.max(np.abs(y2 - ref)) < TOL


@pytest.mark.parametrize("seed", range(6))
def test_dense_random_shapes_all_forms_bit_exact(seed):
    """Random layer shapes (square, shrinking, growing, non-powers of two) in each dense form,
    bit-exact against the oracle's function for that form: composed (Eq. bsgs with square
    padding), lazy-ModDown, and, for shrinking layers, the rectangular form composed and
    lazy with a random fold."""
    rng = np.random.default_rng(900 + seed)
    name = ["a2", "c2"][seed % 2]
    P = pair(name)
    half = P.N // 2
    lim = half // 2
    m = int(rng.integers(1, lim + 1))
    n = int(rng.integers(1, lim + 1))
    tm, tn = O.Oracle.bsgs_t(m, 1), O.Oracle.bsgs_t(n, 1)
    t = O.Oracle.bsgs_t(m, n)
    W = rng.normal(0, 1 / np.sqrt(n), (m, n))
    x = rng.uniform(-1, 1, n)
    slots = np.zeros(half)
    slots[:n] = x
    slots[t:t + n] = x
    _, ct_o = P.fresh(950 + seed, z=slots)
    lvl = ct_o.shape[1]
    o = O.Oracle(P.N, *PARAMS[name][1:3], dnum=PARAMS[name][3], scale=2.0 ** 40)
    g = P.g
    forms = [("composed", False, None), ("lazy", True, None)]
    if tm < tn:
        forms += [("rect", False, int(rng.integers(0, 3))), ("rect_lazy", True, int(rng.integers(0, 3)))]
    for form, lazy, fold in forms:
        if fold is None:
            rots = O.Oracle.bsgs_rotations(m, n, lazy)
        else:
            rots = O.Oracle.rect_rotations(m, n, fold, lazy)
        rots = sorted(set(rots))
        o.keygen(rots, seed=3)
        k = g.keygen(rots, seed=3)
        sc = o.dense_scale(lvl)
        ct = g.ct_import(ct_o, 2.0 ** 40)
        try:
            if fold is None:
                g.set_dense_mode(g.DENSE_LAZY_MODDOWN if lazy else g.DENSE_COMPOSED)
                pts = o.encode_diagonals(W, sc, lazy)
                exp = o.dense(ct_o, pts, lazy=lazy)[0]
                got = g.dense_coeffs(k, ct, pts, sc).export()[0]
            else:
                g.set_dense_mode(g.DENSE_RECT_LAZY if lazy else g.DENSE_RECT)
                pts = o.encode_diagonals_rect(W, sc, lazy)
                # the rectangular input layout: [x, x] at stride tn
                s2 = np.zeros(half)
                s2[:n] = x
                s2[tn:tn + n] = x
                ct2_o = o.encrypt(o.encode(s2), 970 + seed)
                exp = o.dense_rect(ct2_o, pts, tn, fold=fold, lazy=lazy)[0]
                got = g.dense_rect_coeffs(k, g.ct_import(ct2_o, 2.0 ** 40), pts, tn, sc, fold=fold).export()[0]
            assert np.array_equal(got, exp), (form, m, n, fold)
        finally:
            g.set_dense_mode(g.DENSE_COMPOSED)
        k.close()


@pytest.mark.parametrize("lazy", [False, True])
def test_dense_rect_with_bias(lazy):
    """The rectangular form with a bias (added before the rescale, so the fold carries it
    into both halves of the [y, y] layout): bit-exact against the oracle with an injected
    integer bias, and W x + b within the tolerance with the library's own encodings."""
    P = pair("c2")
    m, n = 24, 100
    rots = sorted(set(O.Oracle.rect_rotations(m, n, 2, lazy)))
    o = O.Oracle(P.N, *PARAMS["c2"][1:3], dnum=PARAMS["c2"][3], scale=2.0 ** 40)
    o.keygen(rots, seed=3)
    g = P.g
    k = g.keygen(rots, seed=3)
    W, x, tn, ct_o = rect_case(P, m, n, 333)
    tm = O.Oracle.bsgs_t(m, 1)
    sc = o.dense_scale(ct_o.shape[1])
    pts = o.encode_diagonals_rect(W, sc, lazy)
    bias_c = np.random.default_rng(4).integers(-2 ** 40, 2 ** 40, P.N, dtype=np.int64)
    exp = o.dense_rect(ct_o, pts, tn, bias=bias_c, fold=2, lazy=lazy)[0]
    ct = g.ct_import(ct_o, 2.0 ** 40)
    g.set_dense_mode(g.DENSE_RECT_LAZY if lazy else g.DENSE_RECT)
    try:
        got = g.dense_rect_coeffs(k, ct, pts, tn, sc, bias=bias_c, fold=2).export()[0]
        assert np.array_equal(got, exp)
        b = np.random.default_rng(5).uniform(-0.5, 0.5, m)
        y = g.decrypt(k, g.dense_rect(k, ct, W, bias=b, fold=2), P.N // 2)
        assert np.max(np.abs(y[:m] - (W @ x + b))) < TOL
        assert np.max(np.abs(y[tm:tm + m] - (W @ x + b))) < TOL
    finally:
        g.set_dense_mode(g.DENSE_COMPOSED)
    k.close()
