"""Streams handed to a context stay the caller's: destroying the context (or a clone that
worked on the caller's stream) leaves the stream usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402


def test_callers_stream_outlives_the_context_and_its_clone():
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    c = ctl.Context(64, [50, 40], [60], scale=2.0 ** 40)
    c.set_stream(s1.cuda_stream)
    k = c.keygen([1], seed=3)
    x = np.linspace(-1, 1, 32)
    ct = c.encrypt(k, x, 5)
    clone = c.clone(s2.cuda_stream)
    r = clone.rotate(k, ct, 1)  # the clone works on s2 with the original's keys
    clone.synchronize()
    y = c.decrypt(k, r, 32)
    assert np.max(np.abs(y - np.roll(x, -1))) < 1e-6
    r.close()
    clone.close()
    with torch.cuda.stream(s2):
        t = torch.full((8,), 2.0, device="cuda") * 3
    s2.synchronize()
    assert float(t.sum()) == 48.0
    ct.close()
    k.close()
    c.close()
    with torch.cuda.stream(s1):
        t = torch.full((8,), 1.0, device="cuda") + 1
    s1.synchronize()
    assert float(t.sum()) == 16.0
