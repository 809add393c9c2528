"""GPU checks of the client's side on the device (Fig. alg:cryptotl: HE.Enc, HE.Dec;
Sec. 3.1 "SIMD Encoding"): the FFT encoder against the oracle's direct evaluation of the
canonical embedding (within one unit per coefficient), the FFT decoder against the
oracle's decoder, encryption with the randomness drawn on the device bit-exact against
the oracle's sequential streams, and decryption's centred CRT equal to the oracle's."""
import numpy as np
import pytest

from oracle import ckks_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402

PARAMS = {
    64: ([50, 40, 40], [60], 3),
    1024: ([60, 40, 40, 40], [60], 4),
    4096: ([50, 40, 40], [60], 3),
    16384: ([45] * 8, [60, 60], 4),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N", [64, 1024, 4096, 16384])
def test_encode_and_decode_on_the_device(N):
    qb, pb, dnum = PARAMS[N]
    o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    rng = np.random.default_rng(N)
    count = 1 if N == 16384 else 3
    for nz in (N // 2, N // 2 - 3):
        z = rng.uniform(-1, 1, (count, nz))
        m = torch.empty((count, N), dtype=torch.int64, device="cuda")
        zd = dev(z)
        torch.cuda.synchronize()
        g.encode_dev(zd.data_ptr(), nz, count, m.data_ptr())
        got = m.cpu().numpy()
        for b in range(count):
            assert np.max(np.abs(got[b] - o.encode(z[b]))) <= 1
    # decoding: the oracle's decoder on the same integer coefficients
    mi = np.stack([o.encode(rng.uniform(-1, 1, N // 2)) for _ in range(count)]).astype(np.float64)
    md = dev(mi)
    zo = torch.empty((count, N // 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g.decode_dev(md.data_ptr(), count, N // 2, zo.data_ptr())
    g.synchronize()
    zz = zo.cpu().numpy()
    for b in range(count):
        assert np.max(np.abs(zz[b] - o.decode(mi[b], N // 2))) < 1e-9
    with pytest.raises(ctl.CtlError):
        g.encode_dev(zd.data_ptr(), N // 2 + 1, 1, m.data_ptr())
    g.close()


@pytest.mark.parametrize("N", [64, 1024, 16384])
def test_encrypt_and_decrypt_on_the_device_bit_exact(N):
    """Each ciphertext of a batch encrypted with the device sampler equals the oracle's
    encryption of the same integer plaintext with the same seed; the device CRT of
    decryption gives the oracle's centred coefficients, and the whole client round trip
    (encode, encrypt, decrypt, decode on the device) returns the slots."""
    qb, pb, dnum = PARAMS[N]
    o = O.Oracle(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    o.keygen([], seed=3)
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    k = g.keygen([], seed=3)
    rng = np.random.default_rng(N + 1)
    count = 3
    z = rng.uniform(-1, 1, (count, N // 2))
    m = np.stack([o.encode(z[b]) for b in range(count)])
    seeds = [11 + 7 * b for b in range(count)]
    md = dev(m)
    torch.cuda.synchronize()
    ct = g.encrypt_coeffs_dev(k, md.data_ptr(), count, seeds)
    got = ct.export()
    exp = [o.encrypt(m[b], seeds[b]) for b in range(count)]
    for b in range(count):
        assert np.array_equal(got[b], exp[b]), f"ciphertext {b}"
    co = torch.empty((count, N), dtype=torch.float64, device="cuda")
    g.decrypt_coeffs_dev(k, ct, co.data_ptr())
    g.synchronize()
    cc = co.cpu().numpy()
    for b in range(count):
        assert np.array_equal(cc[b], o.decrypt(exp[b])), f"decryption {b}"
    zd = dev(z)
    torch.cuda.synchronize()
    ct2 = g.encrypt_dev(k, zd.data_ptr(), N // 2, count, seeds)
    zo = torch.empty((count, N // 2), dtype=torch.float64, device="cuda")
    g.decrypt_dev(k, ct2, N // 2, zo.data_ptr())
    g.synchronize()
    assert np.max(np.abs(zo.cpu().numpy() - z)) < 1e-6
    k.close()
    g.close()


def test_client_round_trip_through_a_model():
    """Encode and encrypt a batch on the device, run a model, decrypt and decode on the
    device: the outputs match the FP64 network within 1e-4."""
    N, qb, pb, dnum = 4096, [50, 40, 40], [60], 3
    rng = np.random.default_rng(3)
    W = rng.normal(0, 1 / 8, (32, 64))
    g = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    model = ctl.Model(g, [("dense", W), ("square",)])
    k = g.keygen(model.rotations(), seed=3)
    count = 4
    x = rng.uniform(-1, 1, (count, 64))
    slots = np.zeros((count, 128))
    slots[:, :64] = x
    slots[:, 64:] = x
    zd = dev(slots)
    torch.cuda.synchronize()
    ct = g.encrypt_dev(k, zd.data_ptr(), 128, count, list(range(40, 40 + count)))
    out = model.forward(k, ct)
    y = torch.empty((count, 32), dtype=torch.float64, device="cuda")
    g.decrypt_dev(k, out, 32, y.data_ptr())
    g.synchronize()
    assert np.max(np.abs(y.cpu().numpy() - (x @ W.T) ** 2)) < 1e-4
