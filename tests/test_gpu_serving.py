"""GPU checks of the batching and serving layer: CUDA-graph forwards and the
continuous-batching server return exactly what a plain single-query forward returns
(the integer path is deterministic, so 'the same' means bit-identical), a failing
client's requests fail while the server keeps serving, a full queue is refused, and
batches are admitted by the memory budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2205_11935_gb300 import ctl  # noqa: E402


def bsgs_t(m, n):
    t = 1
    while t < m or t < n:
        t <<= 1
    return t


def make_lane(N, qb, pb, dnum, dims, seed):
    rng = np.random.default_rng(seed)
    Ws = [rng.normal(0, 1 / np.sqrt(dims[i]), (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    layers = []
    for i, W in enumerate(Ws):
        layers.append(("dense", W))
        if i + 1 < len(Ws):
            layers += [("square",), ("replicate", bsgs_t(*Ws[i + 1].shape))]
    ctx = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
    model = ctl.Model(ctx, layers)
    return ctx, model, Ws


def query(ctx, keys, n_in, t0, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, n_in)
    slots = np.zeros(ctx.N // 2)
    slots[:n_in] = x
    slots[t0:t0 + n_in] = x
    return ctx.encrypt(keys, slots, seed)


@pytest.mark.parametrize("N,qb,pb,dnum,dims,B", [(4096, [50, 40, 40], [60], 3, [64, 32], 1),
                                                 (8192, [60, 40, 40, 40], [60], 4, [128, 64, 32], 3),
                                                 (4096, [50, 40, 40], [60], 3, [64, 32], 67)])
def test_graph_forward_equals_eager(N, qb, pb, dnum, dims, B):
    """The graph forward equals the eager one bit for bit, and each replay counts the same
    operations; B = 67 takes the capture as two concurrent halves (33 + 34 ciphertexts)."""
    ctx, model, _ = make_lane(N, qb, pb, dnum, dims, 1)
    keys = ctx.keygen(model.rotations(), seed=3)
    t0 = bsgs_t(dims[1], dims[0])
    batch = ctx.concat([query(ctx, keys, dims[0], t0, 10 + i) for i in range(B)])
    ctx.stats_reset()
    eager = model.forward(keys, batch).export()
    ops = ctx.stats_ops()
    for i in range(3):  # first call captures, later calls replay
        ctx.stats_reset()
        g = model.forward(keys, batch, graph=True).export()
        assert np.array_equal(g, eager)
        if i:
            assert ctx.stats_ops() == ops
    assert ctx.stats_launches() > 0 and ctx.stats_ops()["rotations"] > 0


def test_server_results_identical_alone_and_in_the_mix():
    lanes = [(4096, [50, 40, 40], [60], 3, [64, 32]), (8192, [60, 40, 40, 40], [60], 4, [128, 64, 32])]
    srv = ctl.Server(mem_budget_bytes=8 << 30, n_workers=3, max_batch=4, max_queue=1000)
    made = []
    for li, (N, qb, pb, dnum, dims) in enumerate(lanes):
        ctx, model, _ = make_lane(N, qb, pb, dnum, dims, 1 + li)
        lane = srv.add_lane(ctx, model)
        for c in range(3):
            keys = ctx.keygen(model.rotations(), seed=30 + 3 * li + c)
            made.append((srv.add_client(lane, keys), ctx, model, keys, dims, bsgs_t(dims[1], dims[0])))
    srv.start()
    rng = np.random.default_rng(7)
    jobs = []
    for i in range(40):  # a mixed burst over both lanes and all six clients
        cl, ctx, model, keys, dims, t0 = made[rng.integers(len(made))]
        ct = query(ctx, keys, dims[0], t0, 1000 + i)
        coeffs = ct.export()[0]
        alone = model.forward(keys, ct).export()[0]
        rid = srv.submit(cl, coeffs)
        assert rid is not None
        jobs.append((rid, alone, srv.io_words(cl)[1]))
    for rid, alone, ow in jobs:
        got, lat = srv.wait(rid, ow)
        assert np.array_equal(got.reshape(alone.shape), alone)
        assert lat > 0
    st = srv.stats()
    assert st["completed"] == 40 and st["failed"] == 0 and st["batches"] <= 40
    srv.close()


def test_server_failure_and_full_queue():
    ctx, model, _ = make_lane(4096, [50, 40, 40], [60], 3, [64, 32], 5)
    good = ctx.keygen(model.rotations(), seed=3)
    bad = ctx.keygen([1], seed=4)  # lacks most of the model's rotation keys
    srv = ctl.Server(mem_budget_bytes=4 << 30, n_workers=1, max_batch=1, max_queue=2)
    lane = srv.add_lane(ctx, model)
    cg, cb = srv.add_client(lane, good), srv.add_client(lane, bad)
    srv.start()
    ow = srv.io_words(cg)[1]
    ct = query(ctx, good, 64, 64, 9)
    coeffs = ct.export()[0]
    rb = srv.submit(cb, coeffs)
    with pytest.raises(ctl.CtlError) as e:
        srv.wait(rb, ow)
    assert e.value.code == -4  # missing Galois key: the request fails ...
    rg = srv.submit(cg, coeffs)
    got, _ = srv.wait(rg, ow)  # ... and the server keeps serving
    assert np.array_equal(got.reshape(2, -1, ctx.N), model.forward(good, ct).export()[0])
    ids = [srv.submit(cg, coeffs) for _ in range(50)]  # a burst beyond max_queue is refused
    assert any(i is None for i in ids)
    for i in ids:
        if i is not None:
            srv.wait(i, ow)
    assert srv.stats()["rejected"] > 0
    srv.close()


def test_server_admits_by_memory_budget():
    """A budget that holds one in-flight ciphertext's estimate but not two: every batch
    shrinks to one request, workers wait while another batch holds the memory (the total
    reservation never exceeds the budget), and every request still completes, bit-identical
    to the same query run alone."""
    ctx, model, _ = make_lane(4096, [50, 40, 40], [60], 3, [64, 32], 6)
    keys = ctx.keygen(model.rotations(), seed=3)
    probe = ctl.Server(mem_budget_bytes=1 << 40, n_workers=1, max_batch=1, max_queue=4)
    cl0 = probe.add_client(probe.add_lane(ctx, model), keys)
    bpc = probe.admission(cl0)[0]
    probe.close()
    assert bpc > 0
    budget = bpc + bpc // 2
    srv = ctl.Server(mem_budget_bytes=budget, n_workers=3, max_batch=4, max_queue=100)
    cl = srv.add_client(srv.add_lane(ctx, model), keys)
    ow = srv.io_words(cl)[1]
    cts = [query(ctx, keys, 64, 64, 500 + i) for i in range(12)]
    alone = [model.forward(keys, c).export()[0] for c in cts]
    coeffs = [c.export()[0] for c in cts]
    srv.start()
    ids = [srv.submit(cl, x) for x in coeffs]  # a burst: requests queue behind the running one
    assert all(i is not None for i in ids)
    for rid, want in zip(ids, alone):
        got, _ = srv.wait(rid, ow)
        assert np.array_equal(got.reshape(want.shape), want)
    st = srv.stats()
    b, peak, deferred = srv.admission(cl)
    assert b == bpc
    assert st["completed"] == 12 and st["failed"] == 0
    assert st["batches"] == 12  # groups of up to 4 shrank to 1 to fit the budget
    assert peak <= budget  # never two batches' reservations at once
    assert deferred > 0  # idle workers waited for memory while requests were queued
    srv.close()


def test_multi_graph_equals_each_groups_forward():
    """Configuration 4's one-launch form: three groups with different ring degrees, depths,
    dense forms and batch sizes captured as branches of one CUDA graph; every output equals
    its group's own forward bit for bit, on two calls with different inputs, and a second
    context clone per group runs its branch on its own stream."""
    specs = [  # (N, q, p, dnum, dims, dense mode, batch)
        (8192, [60, 40, 40], [60], 3, [256, 64], 0, 2),
        (16384, [60, 40, 40, 40, 40], [60, 60], 3, [512, 128, 64], 3, 3),
        (8192, [60, 40, 40, 40, 40], [60], 5, [128, 128, 128], 2, 1),
    ]
    groups, made = [], []
    for gi, (N, qb, pb, dnum, dims, mode, B) in enumerate(specs):
        rng = np.random.default_rng(gi)
        Ws = [rng.normal(0, 1 / np.sqrt(dims[i]), (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
        layers = []
        for i, W in enumerate(Ws):
            layers.append(("dense", W))
            layers.append(("square",))
            if i + 1 < len(Ws):
                layers.append(("replicate", bsgs_t(*Ws[i + 1].shape)))
        ctx = ctl.Context(N, qb, pb, dnum=dnum, scale=2.0 ** 40)
        ctx.set_dense_mode(mode)
        model = ctl.Model(ctx, layers)
        keys = ctx.keygen(model.rotations(), seed=10 + gi)
        clone = ctx.clone()
        groups.append((clone, model, keys, B))
        made.append((ctx, model, keys, dims, B, bsgs_t(Ws[0].shape[0], Ws[0].shape[1])))
    multi = ctl.Multi(groups)
    for call in range(2):
        ins, exp = [], []
        for gi, (ctx, model, keys, dims, B, t0) in enumerate(made):
            batch = ctx.concat([query(ctx, keys, dims[0], t0, 100 * call + 10 * gi + b) for b in range(B)])
            ins.append(batch)
            exp.append(model.forward(keys, batch).export())
        outs = multi.forward(ins)
        for gi in range(len(made)):
            assert np.array_equal(outs[gi].export(), exp[gi]), f"call {call}, group {gi}"
    # an input that does not match its group (batch size) is refused, nothing launched
    ctx0, _, keys0, dims0, B0, t00 = made[0]
    wrong = ctx0.concat([query(ctx0, keys0, dims0[0], t00, 7 + b) for b in range(B0 + 1)])
    with pytest.raises(ctl.CtlError):
        multi.forward([wrong] + ins[1:])
    multi.close()
    for clone, _, _, _ in groups:
        clone.close()
