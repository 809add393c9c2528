"""The protocol's split of keys (Fig. alg:cryptotl): the client generates its keys and
sends the evaluation keys; the server, holding no secret, imports them and evaluates.
The served result must be bit-identical to an evaluation with the client's own key set,
and the imported set must refuse to encrypt or decrypt."""
import numpy as np
import pytest

from oracle import ckks_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402


def test_imported_evaluation_keys_serve_bit_identical_results():
    N, qb, pb = 1024, [60, 40, 40, 40], [60]
    rng = np.random.default_rng(120)
    W1, W2 = rng.normal(0, 0.25, (16, 32)), rng.normal(0, 0.25, (8, 16))
    layers = [("dense", W1), ("square",), ("replicate", 16), ("dense", W2)]
    client = ctl.Context(N, qb, pb, scale=2.0 ** 40)
    server = ctl.Context(N, qb, pb, scale=2.0 ** 40)
    m_client = ctl.Model(client, layers)
    m_server = ctl.Model(server, layers)
    rots = m_client.rotations()
    assert rots == m_server.rotations()
    keys = client.keygen(rots, seed=3)
    # the client sends the relinearisation key and one Galois key per rotation
    evk = server.keys_create()
    ids = [0] + sorted({client.galois_element(r) for r in rots})
    for kid in ids:
        evk.import_key(kid, keys.export(kid))
        assert np.array_equal(evk.export(kid), keys.export(kid))
    x = rng.uniform(-1, 1, 32)
    slots = np.zeros(N // 2)
    slots[:32] = x
    slots[32:64] = x
    ct = client.encrypt(keys, slots, 7)
    msg = ctl.serialize(N, client.moduli[:4], ct.export()[0], seed=7)  # C -> S: c0 and the seed
    ct_s = server.ct_import(ctl.deserialize(msg, N, server.moduli[:4]), 2.0 ** 40)
    out_s = m_server.forward(evk, ct_s).export()[0]
    out_c = m_client.forward(keys, ct).export()[0]
    assert np.array_equal(out_s, out_c)
    y = client.decrypt(keys, client.ct_import(out_s, m_client.info()[1]), 8)
    assert np.max(np.abs(y - W2 @ (W1 @ x) ** 2)) < 1e-4
    # the server's key set holds no secret
    with pytest.raises(ctl.CtlError) as e:
        server.decrypt(evk, ct_s, 4)
    assert e.value.code == -4
    with pytest.raises(ctl.CtlError):
        server.encrypt(evk, slots, 9)
    # a key the server was not sent
    with pytest.raises(ctl.CtlError) as e:
        server.rotate(evk, ct_s, 9)
    assert e.value.code == -4


def test_malformed_key_imports_are_refused():
    N = 256
    c = ctl.Context(N, [50, 40], [60], scale=2.0 ** 40)
    k = c.keygen([1], seed=3)
    evk = c.keys_create()
    good = k.export(0)
    with pytest.raises(ctl.CtlError):
        evk.import_key(0, good[:1])  # wrong size
    with pytest.raises(ctl.CtlError):
        evk.import_key(6, good)  # even: not a Galois element
    bad = good.copy()
    bad[0, 0, 1, 3] = O.primes(N, [50, 40, 60])[1]  # a residue equal to its prime
    with pytest.raises(ctl.CtlError):
        evk.import_key(0, bad)
    evk.import_key(0, good)
