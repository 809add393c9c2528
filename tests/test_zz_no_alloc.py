"""GPU check of ctl_rescale_static_dev, the rescale entry point that allocates nothing.

It serves callers that may not allocate device memory while running (a framework that
owns the device through its own arena, a latency-bound serving thread); its scratch is
a fixed array inside the library.  Through the C-ABI, its output must equal the
ordinary allocating ctl_rescale on the same ciphertexts, and the oracle's rescale
(the rounding division by the last prime, computed with big integers on the CPU), for
two calls in a row (the shared array keeps the previous call's contents, which must not
leak into the next).  This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import ckks_oracle as O  # noqa: E402
from paper_2205_11935_gb300 import ctl  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("N,qb,pb,count", [(4096, [50, 40, 40], [60], 3), (16384, [45] * 8, [60, 60], 4)])
def test_static_rescale_matches_allocating_rescale(N, qb, pb, count):
    g = ctl.Context(N, qb, pb, dnum=len(qb) // 2 or 1, scale=2.0 ** 40)
    o = O.Oracle(N, qb, pb, dnum=len(qb) // 2 or 1, scale=2.0 ** 40)
    assert o.moduli == g.moduli
    k = g.keygen([], seed=3)
    L = len(qb)
    lib = ctl.lib()
    cap = int(lib.ctl_rescale_static_capacity_words())
    assert cap >= count * 2 * N
    rng = np.random.default_rng(N + count)
    for call in range(2):  # two calls in a row on the same scratch array
        xs = rng.uniform(-1, 1, (count, N // 2))
        cts = [g.encrypt(k, xs[i], 100 * call + i) for i in range(count)]
        batch = g.concat(cts)
        ref = g.rescale(batch).export()  # allocating path, coefficient form
        coeffs = batch.export()  # [count][2][L][N] coefficient form
        x = _dev(coeffs)
        torch.cuda.synchronize()
        g.ntt_dev(x.data_ptr(), x.data_ptr(), 2 * count, L)  # to NTT form
        out = torch.zeros((count, 2, L - 1, N), dtype=torch.int64, device="cuda")
        rc = lib.ctl_rescale_static_dev(g.h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), count, L)
        assert rc == 0, lib.ctl_last_error().decode()
        g.ntt_dev(out.data_ptr(), out.data_ptr(), 2 * count, L - 1, inverse=True)
        g.synchronize()
        got = out.cpu().numpy().view(np.uint64).reshape(count, 2, L - 1, N)
        assert np.array_equal(got, ref), f"call {call}: differs from ctl_rescale"
        for i in range(count):
            assert np.array_equal(got[i], o.rescale(coeffs[i])), f"call {call}: differs from the oracle"
    # sizes beyond the fixed scratch are refused with a clear message
    too_many = cap // (2 * N) + 1
    rc = lib.ctl_rescale_static_dev(g.h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), too_many, L)
    assert rc == -1 and b"fixed limit" in lib.ctl_last_error()
    for h in cts + [batch, k]:
        h.close()
    g.close()
