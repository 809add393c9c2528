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
