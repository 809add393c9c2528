"""GPU parity of the other layers of the paper's frozen network (Sec. 3.1: the ReLU
approximation, average pooling, the packed 1D convolution; Sec. 4.1: the whole stack)
through the C-ABI, against the CKKS oracle.

Ciphertexts must be bit-exact with the oracle's on the same keys and randomness (the
oracle's integer plaintexts are injected where an FP64 encoder is involved); decoded
values must be within 1e-4 of FP64 at scale 2^40 (and 2^50).  At CryptoTL_p1's scale
2^25 the bound follows from the key-switching noise (netref.keyswitch_error_bound): one
key switch at the input scale leaves a slot error of deviation
sqrt(N/2) * sqrt(N * 10.5 * sum_d q_d^2 / (3 P^2)) / 2^25 (1.0e-5 at N = 256, 3.2e-4 at
N = 8192, with the 34-bit q0 digit over the 34-bit P dominating), the frozen stack carries
about five such errors to an output at the input scale (convolution, first dense layer's
baby steps, replicate, pool, last dense layer's baby steps), and the maximum over the
outputs stays within sqrt(2 ln n) + 2 deviations: 1.0e-4 at N = 256, 4.2e-3 at N = 8192
with 1532 outputs.
"""
import numpy as np
import pytest

from oracle import ckks_oracle as O
from tests import netref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402

TOL = 1e-4
P1_BITS = ([34] + [25] * 6, [34])  # CryptoTL_p1: digit (data prime) sizes, special prime
TOL_P1 = netref.keyswitch_error_bound(256, *P1_BITS, 25, n_ks=5, n_outputs=128)
TOL_P1_FULL = netref.keyswitch_error_bound(8192, *P1_BITS, 25, n_ks=5, n_outputs=2 * 766)

# (N, q_bits, p_bits, dnum, log2 scale)
PARAMS = {
    "b4": (256, [60, 40, 40, 40, 40], [60], 5, 40),              # alpha 1, five digits
    "b2": (512, [45, 45, 45, 45, 45], [60, 60], 3, 40),          # alpha 2, two special primes
    "p1": (256, [34, 25, 25, 25, 25, 25, 25], [34], 7, 25),      # CryptoTL_p1's prime sizes
}
ROTS = [1, 2, 3, -1, -2, -3, 4, -4]


class Pair:
    def __init__(self, name, rots=ROTS):
        N, qb, pb, dnum, ls = PARAMS[name]
        self.scale = 2.0 ** ls
        self.o = O.Oracle(N, qb, pb, dnum=dnum, scale=self.scale)
        self.o.keygen(rots, seed=3)
        self.g = ctl.Context(N, qb, pb, dnum=dnum, scale=self.scale)
        self.k = self.g.keygen(rots, seed=3)
        self.N = N

    def fresh(self, seed, z=None, lo=-1.0, hi=1.0):
        rng = np.random.default_rng(seed)
        if z is None:
            z = rng.uniform(lo, hi, self.N // 2)
        return z, self.o.encrypt(self.o.encode(z), seed)


_cache = {}


def pair(name):
    if name not in _cache:
        _cache[name] = Pair(name)
    return _cache[name]


def tol(name):
    return TOL_P1 if name == "p1" else TOL


@pytest.mark.parametrize("name", list(PARAMS))
def test_mul_bit_exact_and_fp64(name):
    P = pair(name)
    za, a_o = P.fresh(101)
    zb, b_o = P.fresh(102)
    a, b = P.g.ct_import(a_o, P.scale), P.g.ct_import(b_o, P.scale)
    out = P.g.mul(P.k, a, b)
    assert np.array_equal(out.export()[0], P.o.mul(a_o, b_o))
    assert np.max(np.abs(P.g.decrypt(P.k, out, P.N // 2) - za * zb)) < tol(name)
    # HMult(a, a) is the square activation, bit for bit
    assert np.array_equal(P.g.mul(P.k, a, a).export()[0], P.g.square(P.k, a).export()[0])


@pytest.mark.parametrize("name", list(PARAMS))
def test_constant_ops_and_level_drop_bit_exact(name):
    P = pair(name)
    z, ct_o = P.fresh(103)
    ct = P.g.ct_import(ct_o, P.scale)
    for C in (123456789, -987654321, 0, 2 ** 45 + 7):
        assert np.array_equal(P.g.mul_const(ct, C, 1.0).export()[0], P.o.mul_const(ct_o, C))
        assert np.array_equal(P.g.add_const(ct, C).export()[0], P.o.add_const(ct_o, C))
    lvl = ct_o.shape[1]
    d = P.g.drop_level(ct, lvl - 2)
    assert d.info()[0] == lvl - 2
    assert np.array_equal(d.export()[0], P.o.drop_level(ct_o, lvl - 2))
    with pytest.raises(ctl.CtlError):
        P.g.drop_level(ct, lvl + 1)


@pytest.mark.parametrize("name", list(PARAMS))
@pytest.mark.parametrize("which", ["paper", 3, 1])
def test_poly3_bit_exact_and_fp64(name, which):
    P = pair(name)
    a = netref.relu_coeffs() if which == "paper" else [0.5 if i == which else 0.0 for i in range(4)]
    z, ct_o = P.fresh(104, lo=-3.0, hi=3.0)
    exp, sc = P.o.poly3(ct_o, P.scale, a)
    ct = P.g.ct_import(ct_o, P.scale)
    out = P.g.poly3(P.k, ct, a)
    lvl, cnt, gsc = out.info()
    assert lvl == ct_o.shape[1] - 2 and gsc == sc
    assert np.array_equal(out.export()[0], exp)
    assert np.max(np.abs(P.g.decrypt(P.k, out, P.N // 2) - netref.poly3(a, z))) < 3 * tol(name)


@pytest.mark.parametrize("name", list(PARAMS))
@pytest.mark.parametrize("f", [2, 3, 4])
def test_avgpool_bit_exact_and_fp64(name, f):
    P = pair(name)
    z, ct_o = P.fresh(105 + f)
    exp, cnt = P.o.avgpool(ct_o, f)
    ct = P.g.ct_import(ct_o, P.scale)
    P.g.stats_reset()
    out = P.g.avgpool(P.k, ct, f)
    ops = P.g.stats_ops()
    assert np.array_equal(out.export()[0], exp)
    assert ops["rotations"] == cnt[0] and ops["ptmul"] == cnt[1] and ops["add"] == cnt[2]
    want = sum(np.roll(z, i) for i in range(f)) / f
    assert np.max(np.abs(P.g.decrypt(P.k, out, P.N // 2) - want)) < tol(name)


@pytest.mark.parametrize("name", list(PARAMS))
@pytest.mark.parametrize("f,n,t", [(3, 10, 16), (9, 20, 32), (1, 8, 8)])
def test_conv1d_bit_exact_injected_and_fp64(name, f, n, t):
    P = pair(name)
    rng = np.random.default_rng(106 + f)
    x = rng.uniform(-1, 1, n)
    w = rng.normal(0, 1 / np.sqrt(f), f)
    z, ct_o = P.fresh(107, z=netref.replicated_slots(x, t, P.N // 2))
    lvl = ct_o.shape[1]
    sc = P.o.dense_scale(lvl)
    pts = P.o.encode_conv(w, n, t, sc)
    exp, cnt = P.o.conv1d(ct_o, pts)
    ct = P.g.ct_import(ct_o, P.scale)
    P.g.stats_reset()
    out = P.g.conv1d_coeffs(P.k, ct, pts, sc)
    ops = P.g.stats_ops()
    assert np.array_equal(out.export()[0], exp)
    assert ops["rotations"] == cnt[0] and ops["ptmul"] == cnt[1] and ops["add"] == cnt[2]
    # the library's own plaintext encoding: decoded within tolerance of numpy's correlation
    out2 = P.g.conv1d(P.k, ct, w, n, t)
    assert out2.info()[2] == P.scale
    y = P.g.decrypt(P.k, out2, P.N // 2)
    want = np.correlate(x, w, "same")
    assert np.max(np.abs(y[:n] - want)) < tol(name) and np.max(np.abs(y[t:t + n] - want)) < tol(name)
    if n < t:
        assert np.max(np.abs(y[n:t])) < tol(name)


# ----------------------------------------------------------------------------- the paper's stack
def paper_layers(o, n, t, w, W1, W2s, a, lvl, scale, inject=True):
    """conv(f) -> dense n->n -> replicate -> ReLU_approx -> avgpool(3) -> dense (Sec. 4.1),
    with the oracle's plaintexts injected (inject) so that the GPU result is bit-exact."""
    sc = scale
    conv_pts = o.encode_conv(w, n, t, o.dense_scale(lvl, sc)) if inject else None
    d1 = o.encode_diagonals(W1, o.dense_scale(lvl - 1, sc)) if inject else None
    sw = o.poly3_consts(lvl - 2, sc, a)[1]
    d2 = o.encode_diagonals(W2s, o.dense_scale(lvl - 5, sw)) if inject else None
    return [("conv1d", w, n, t, None, conv_pts), ("dense", W1, None, d1), ("replicate", t), ("poly3", a),
            ("avgpool", 3), ("dense", W2s, None, d2)]


def paper_rotations(n, m2, f, t):
    h = (f - 1) // 2
    r = [i - h for i in range(f) if i != h]
    r += O.Oracle.bsgs_rotations(n, n) + [-t, -1, -2] + O.Oracle.bsgs_rotations(m2, n)
    return sorted(set(r))


def oracle_paper_net(o, ct, layers):
    for ly in layers:
        if ly[0] == "conv1d":
            ct = o.conv1d(ct, ly[5])[0]
        elif ly[0] == "dense":
            ct = o.dense(ct, ly[3])[0]
        elif ly[0] == "replicate":
            ct = o.replicate(ct, ly[1])
        elif ly[0] == "poly3":
            ct = o.poly3(ct, o.scale, ly[1])[0]
        elif ly[0] == "avgpool":
            ct = o.avgpool(ct, ly[1])[0]
    return ct


@pytest.mark.parametrize("name", ["b4p", "p1"])
def test_paper_network_bit_exact_and_fp64(name):
    """The whole frozen stack (depth 6) at N = 256, n = 24: bit-exact against the oracle,
    batch members equal to their single forward, graph replay equal to the eager forward."""
    N, n, f = 256, 24, 9
    qb, pb, ls = ([60] + [40] * 6, [60], 40) if name == "b4p" else ([34] + [25] * 6, [34], 25)
    scale = 2.0 ** ls
    t = O.Oracle.bsgs_t(n, n)
    w, W1, W2, W2s = netref.paper_net_weights(n, f=f)
    m2 = W2.shape[0]
    rots = paper_rotations(n, m2, f, t)
    o = O.Oracle(N, qb, pb, dnum=7, scale=scale)
    o.keygen(rots, seed=3)
    g = ctl.Context(N, qb, pb, dnum=7, scale=scale)
    k = g.keygen(rots, seed=3)
    a = netref.relu_coeffs()
    layers = paper_layers(o, n, t, w, W1, W2s, a, 7, scale)
    model = ctl.Model(g, layers)
    assert sorted(model.rotations()) == rots
    assert model.info()[0] == 1  # depth 6: seven data primes leave q_0
    xs = np.random.default_rng(108).uniform(-1, 1, (3, n))
    cts_o = [o.encrypt(o.encode(netref.replicated_slots(x, t, N // 2)), 200 + i) for i, x in enumerate(xs)]
    exp = oracle_paper_net(o, cts_o[0], layers)
    out = model.forward(k, g.ct_import(cts_o[0], scale))
    assert np.array_equal(out.export()[0], exp)
    y = g.decrypt(k, out, m2)
    assert np.max(np.abs(y - netref.paper_net_fp64(xs[0], w, W1, W2, a))) < (TOL_P1 if name == "p1" else TOL)
    batch = g.ct_import(np.stack(cts_o), scale)
    ob = model.forward(k, batch).export()
    og = model.forward(k, batch, graph=True).export()
    assert np.array_equal(ob[0], exp) and np.array_equal(og, ob)
    for i in (1, 2):
        assert np.array_equal(ob[i], model.forward(k, g.ct_import(cts_o[i], scale)).export()[0])
    # the library's own encodings: decoded within tolerance
    model2 = ctl.Model(g, paper_layers(o, n, t, w, W1, W2s, a, 7, scale, inject=False))
    y2 = g.decrypt(k, model2.forward(k, g.ct_import(cts_o[1], scale)), m2)
    assert np.max(np.abs(y2 - netref.paper_net_fp64(xs[1], w, W1, W2, a))) < (TOL_P1 if name == "p1" else TOL)
    model.close()
    model2.close()


@pytest.mark.parametrize("name,N,qb,pb,ls,tol_", [
    ("CryptoTL_p1", 8192, [34] + [25] * 6, [34], 25, TOL_P1_FULL),
    ("CryptoTL_p2", 16384, [60] + [50] * 6, [60], 50, TOL),
])
def test_paper_network_full_size(name, N, qb, pb, ls, tol_):
    """The paper's stack at its own parameter sets (Tab. 1) and sizes (Sec. 4.1: 768
    inputs, Dense 768, AvgPool 3, Dense 766), in the bench's launch configuration: decoded
    within tolerance of FP64; batch members equal to single forwards; graph replay equal."""
    n, f = 768, 9
    scale = 2.0 ** ls
    t = O.Oracle.bsgs_t(n, n)
    w, W1, W2, W2s = netref.paper_net_weights(n, f=f)
    m2 = W2.shape[0]
    g = ctl.Context(N, qb, pb, dnum=7, scale=scale)
    a = netref.relu_coeffs()
    model = ctl.Model(g, [("conv1d", w, n, t), ("dense", W1), ("replicate", t), ("poly3", a), ("avgpool", 3),
                          ("dense", W2s)])
    k = g.keygen(model.rotations(), seed=3)
    xs = np.random.default_rng(109).uniform(-1, 1, (2, n))
    cts = [g.encrypt(k, netref.replicated_slots(x, t, N // 2), 300 + i) for i, x in enumerate(xs)]
    batch = g.concat(cts)
    out = model.forward(k, batch)
    assert out.info()[0] == 1
    for i in range(2):
        y = g.decrypt(k, out.slice(i), m2)
        err = np.max(np.abs(y - netref.paper_net_fp64(xs[i], w, W1, W2, a)))
        print(f"{name}: max decoded error vs FP64 {err:.3e}")
        assert err < tol_, (name, err)
    single = model.forward(k, cts[1], graph=True).export()[0]
    assert np.array_equal(single, out.export()[1])
    model.close()


def test_paper_network_prediction_windows_bit_exact():
    """Sec. 3.1 "Multiple Predictions": p = 4 inputs in one ciphertext (N = 512, n = 24,
    t = 32), plaintexts encoded for 4 windows: bit-exact against the oracle with injected
    plaintexts, and every window within 1e-4 of its own FP64 network with the library's
    own encodings (ctl_set_windows)."""
    N, n, f = 512, 24, 9
    qb, pb, scale = [60] + [40] * 6, [60], 2.0 ** 40
    t = O.Oracle.bsgs_t(n, n)
    p = (N // 2) // (2 * t)
    w, W1, W2, W2s = netref.paper_net_weights(n, f=f)
    m2 = W2.shape[0]
    rots = paper_rotations(n, m2, f, t)
    o = O.Oracle(N, qb, pb, dnum=7, scale=scale)
    o.keygen(rots, seed=3)
    g = ctl.Context(N, qb, pb, dnum=7, scale=scale)
    k = g.keygen(rots, seed=3)
    a = netref.relu_coeffs()
    xs = np.random.default_rng(110).uniform(-1, 1, (p, n))
    slots = np.zeros(N // 2)
    for j in range(p):
        slots[2 * t * j:2 * t * (j + 1)] = netref.replicated_slots(xs[j], t, 2 * t)
    ct_o = o.encrypt(o.encode(slots), 400)
    sw = o.poly3_consts(5, scale, a)[1]
    layers = [("conv1d", w, n, t, None, o.encode_conv(w, n, t, o.dense_scale(7), windows=p)),
              ("dense", W1, None, o.encode_diagonals(W1, o.dense_scale(6), windows=p)), ("replicate", t),
              ("poly3", a), ("avgpool", 3), ("dense", W2s, None, o.encode_diagonals(W2s, o.dense_scale(2, sw),
                                                                                    windows=p))]
    exp = oracle_paper_net(o, ct_o, layers)
    model = ctl.Model(g, layers)
    out = model.forward(k, g.ct_import(ct_o, scale))
    assert np.array_equal(out.export()[0], exp)
    g.set_windows(p)
    model2 = ctl.Model(g, [("conv1d", w, n, t), ("dense", W1), ("replicate", t), ("poly3", a), ("avgpool", 3),
                           ("dense", W2s)])
    y = g.decrypt(k, model2.forward(k, g.ct_import(ct_o, scale)), N // 2)
    for j in range(p):
        assert np.max(np.abs(y[2 * t * j:2 * t * j + m2] - netref.paper_net_fp64(xs[j], w, W1, W2, a))) < TOL
    with pytest.raises(ctl.CtlError):
        g.set_windows(0)
    g.set_windows(p + 1)  # 2 t (p+1) > N/2: a layer for this t no longer fits
    with pytest.raises(ctl.CtlError):
        ctl.Model(g, [("dense", W1)])
    model.close()
    model2.close()


def test_biases_windows_and_lazy_dense_in_the_paper_stack():
    """Biases of conv1d and dense layers (library encodings, replicated per window), the
    lazy-ModDown dense form inside the paper's stack, and direct calls equal to the
    model's layers: decoded within 1e-4 of FP64 per window."""
    N, n, f = 512, 24, 9
    qb, pb, scale = [60] + [40] * 6, [60], 2.0 ** 40
    t = O.Oracle.bsgs_t(n, n)
    p = (N // 2) // (2 * t)
    w, W1, W2, W2s = netref.paper_net_weights(n, f=f)
    m2 = W2.shape[0]
    rng = np.random.default_rng(111)
    bc, b1, b2 = rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, m2)
    a = netref.relu_coeffs()

    def ref(x):
        h = netref.conv_same(x, w) + bc
        z = W1 @ h + b1
        r = netref.poly3(a, z)
        return W2 @ netref.avgpool_valid(r, 3) + b2

    xs = rng.uniform(-1, 1, (p, n))
    slots = np.zeros(N // 2)
    for j in range(p):
        slots[2 * t * j:2 * t * (j + 1)] = netref.replicated_slots(xs[j], t, 2 * t)
    for lazy in (False, True):
        g = ctl.Context(N, qb, pb, dnum=7, scale=scale)
        g.set_windows(p)
        g.set_dense_mode(g.DENSE_LAZY_MODDOWN if lazy else g.DENSE_COMPOSED)
        layers = [("conv1d", w, n, t, bc), ("dense", W1, b1), ("replicate", t), ("poly3", a), ("avgpool", 3),
                  ("dense", W2s, b2)]
        model = ctl.Model(g, layers)
        k = g.keygen(model.rotations(), seed=3)
        ct = g.encrypt(k, slots, 500)
        out = model.forward(k, ct)
        y = g.decrypt(k, out, N // 2)
        for j in range(p):
            assert np.max(np.abs(y[2 * t * j:2 * t * j + m2] - ref(xs[j]))) < TOL, (lazy, j)
        # the same layers as direct calls give the same ciphertext
        h = g.conv1d(k, ct, w, n, t, bias=bc)
        h = g.dense(k, h, W1, bias=b1)
        h = g.replicate(k, h, t)
        h = g.poly3(k, h, a)
        h = g.avgpool(k, h, 3)
        h = g.dense(k, h, W2s, bias=b2)
        assert np.array_equal(h.export(), out.export())
        model.close()


def test_layer_error_codes():
    """Refusals of the new calls: each fails with its documented code and leaves the
    context usable."""
    P = pair("b4")
    g, k = P.g, P.k
    z, ct_o = P.fresh(112)
    ct = g.ct_import(ct_o, P.scale)
    low = g.drop_level(ct, 2)

    def code(fn, *a):
        with pytest.raises(ctl.CtlError) as e:
            fn(*a)
        return e.value.code

    assert code(g.mul, k, ct, low) == -2                  # levels differ
    assert code(g.poly3, k, low, [0, 1, 0, 0]) == -2      # depth 2 needs three primes
    assert code(g.poly3, k, ct, [0, 0, 0, 1e30]) == -1    # a constant beyond 2^63
    assert code(g.avgpool, k, ct, 0) == -1
    assert code(g.avgpool, k, ct, P.N) == -1
    assert code(g.conv1d, k, ct, [1.0, 2.0, 3.0], 40, 32) == -1   # n > t
    assert code(g.conv1d, k, ct, [1.0], 8, P.N) == -1             # 2t beyond the slots
    assert code(g.drop_level, ct, 0) == -2
    assert code(g.mul_const, ct, 3, 0.0) == -1
    assert code(g.avgpool, k, g.drop_level(ct, 1), 2) == -2       # no level left
    assert code(g.rotate, k, ct, 9) == -4                          # no Galois key for 9
    with pytest.raises(ctl.CtlError) as e:
        ctl.Model(g, [("poly3", [0, 1, 0, 0])], in_level=2)
    assert e.value.code == -2
    # the context still works
    out = g.poly3(k, ct, [0.1, 0.2, 0.3, 0.0])
    assert out.info()[0] == ct_o.shape[1] - 2
