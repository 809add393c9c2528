"""Benchmark: encrypted forwards per second of CryptoTL's server step (ClassifyHE).

Workload (default "batched"): 256 CKKS ciphertexts at N = 16384 (8 x 45-bit data
primes, 2 x 60-bit special primes, dnum = 4, scale 2^40) under one client's keys,
through the frozen layers dense 1024->256, x^2, dense 256->256, x^2, dense 256->64
(Sec. 3.1 layer algorithms; diagonal mat-vec of Eq. (bsgs) with hoisted baby steps).
Synthetic data: inputs ~U[-1,1], weights ~N(0, 1/fan_in), fixed seeds.

One JSON line on rank 0:
  value    forwards/s with the input batch resident in HBM (CUDA events on the library's
           stream, max over ranks);
  e2e      forwards/s through the C-ABI with host buffers: import (H2D) + forward +
           export (D2H) of every step inside the timed region;
  roofline the dominant kernel class against the integer-multiply (IMAD) peak
           (152 SMs x 64 IMAD/clk x clock), counted in 64-bit Shoup modular
           multiplications at their measured IMAD cost;
  cpu_baseline the CKKS oracle on the host cores, on a bounded sample (one rotation,
           one plaintext product and one rescale at the top level), extrapolated by the
           forward's operation counts.
``--impl reference`` times that oracle leg alone on this workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT = 152
IMAD_PER_CLK_SM = 64          # 32-bit integer multiply-add lanes per SM per clock (issue slots)
MAX_SM_MHZ = 2070.0
MAC_CLASSES = ("key_ip", "bsgs_inner")  # kernel classes whose work unit is a split-half MAC
HBM_FALLBACK_GBS = 6800.0     # copy bandwidth of an earlier GB300 measurement, if none is given
# DRAM traffic over algorithmic bytes per kernel class: the dram__bytes_read.sum +
# dram__bytes_write.sum of every launch of one forward of the batched network in its
# benchmark form (CTL_DENSE_RECT_LAZY) at batch 16, over the algorithmic bytes the library
# counts for the same launches.  A full-size launch's traffic is taken as this ratio times
# its algorithmic bytes; ratios below 1 are L2 hits at batch 16, so this is a lower
# estimate at batch 256.  A class missing here was not captured for the current kernels.
TRAFFIC_RATIO = {"modup_ntt": 0.833, "moddown_ntt": 0.759, "key_ip": 0.802, "bsgs_inner": 0.987,
                 "ntt_inv": 0.631, "rescale": 0.571}


def hbm_peak_gbs():
    """The measured copy bandwidth of the GB300s, else the fallback (says which)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"

WORKLOADS = {
    "batched": dict(N=16384, q=[45] * 8, p=[60, 60], dnum=4, batch=256, dims=[1024, 256, 256, 64],
                    dense_form="rect_lazy",
                    desc="256 ciphertexts, N=16384, 8x45-bit q + 2x60-bit p, dnum=4, scale 2^40; "
                         "dense 1024->256, x^2, dense 256->256, x^2, dense 256->64"),
    "single8192": dict(N=8192, q=[60, 40, 40, 40], p=[60], dnum=4, batch=1, dims=[512, 128, 64],
                       desc="1 ciphertext, N=8192, q {60,40,40,40} + 60-bit p, scale 2^40; "
                            "dense 512->128, x^2, dense 128->64"),
    "single4096": dict(N=4096, q=[50, 40, 40], p=[60], dnum=3, batch=1, dims=[64, 32], square_last=True,
                       desc="1 ciphertext, N=4096, q {50,40,40} + 60-bit p, scale 2^40; dense 64->32, x^2"),
    # the paper's own frozen network (Sec. 4.1) at its parameter sets (Tab. 1)
    "paper_p1": dict(N=8192, q=[34] + [25] * 6, p=[34], dnum=7, batch=1, dims=[768, 768, 766], net="paper",
                     scale=2.0 ** 25,
                     desc="CryptoTL_p1: N=8192, q {34, 6x25} + 34-bit p (218 bits), scale 2^25; conv1d f=9 on 768 "
                          "inputs, dense 768->768, ReLU approx (deg 3), avgpool 3, dense ->766; 1 ciphertext"),
    "paper_p2": dict(N=16384, q=[60] + [50] * 6, p=[60], dnum=7, batch=1, dims=[768, 768, 766], net="paper",
                     scale=2.0 ** 50,
                     desc="CryptoTL_p2: N=16384, q {60, 6x50} + 60-bit p (420 bits), scale 2^50; conv1d f=9 on 768 "
                          "inputs, dense 768->768, ReLU approx (deg 3), avgpool 3, dense ->766; 1 ciphertext"),
}
# t_S of one forward on one notebook CPU thread with SEAL + AVX-512 (Tab. 1), for context
PAPER_T_S = {"paper_p1": 1.08, "paper_p2": 2.56}
# ReLU approximation of Sec. 3.1 (a3 z^3 + a2 z^2 + a1 z + a0), as a0..a3
RELU_APPROX = [0.49383, 0.59259, 0.092593, -0.0061728]


# dense-layer forms (ctl_set_dense_mode): square padding or the rectangular form for shrinking
# layers, each with Eq. (bsgs) composed of whole rotations or in the lazy-ModDown form
DENSE_FORMS = {"square": "DENSE_COMPOSED", "lazy": "DENSE_LAZY_MODDOWN", "rect": "DENSE_RECT",
               "rect_lazy": "DENSE_RECT_LAZY"}
DENSE_FORM_DESC = {
    "square": "ctl_set_dense_mode(CTL_DENSE_COMPOSED): every dense layer padded to a square t x t matrix, "
              "t = 2^ceil(log2 max(m, n)), t1 = 2^ceil(log2(t)/2), whole rotations",
    "lazy": "ctl_set_dense_mode(CTL_DENSE_LAZY_MODDOWN): square padding, rotations kept in the extended basis, "
            "ModDown once per giant step and once per layer, t1 = min(t, 2^ceil(log2(4t)/2))",
    "rect": "ctl_set_dense_mode(CTL_DENSE_RECT): shrinking layers with tm diagonals of length tn and a "
            "log2(tn/tm)-rotation fold, whole rotations",
    "rect_lazy": "ctl_set_dense_mode(CTL_DENSE_RECT_LAZY): the rectangular form for shrinking layers, every "
                 "Eq. (bsgs) in the lazy-ModDown form and its split"}


def bsgs_t(m, n):
    t = 1
    while t < m or t < n:
        t <<= 1
    return t


def layers_for(dims, square_last):
    rng = np.random.default_rng(1)
    Ws = [rng.normal(0, 1 / np.sqrt(dims[i]), (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    layers = []
    for i, W in enumerate(Ws):
        layers.append(("dense", W))
        if i + 1 < len(Ws):
            layers.append(("square",))
            layers.append(("replicate", bsgs_t(*Ws[i + 1].shape)))
        elif square_last:
            layers.append(("square",))
    return layers, Ws


def paper_layers_for(n, f=9, pool=3):
    """The paper's frozen network (Sec. 4.1) on n inputs held as [x, x] at block stride t:
    conv1d(f) -> dense n->n -> replicate -> ReLU approx -> avgpool(pool) -> dense to
    n-pool+1 outputs.  Synthetic weights: filter ~N(0, 1/f), dense ~N(0, 1/fan_in).  The
    valid pooled value k sits in slot k+pool-1, so the last matrix is applied with its
    columns moved right by pool-1."""
    rng = np.random.default_rng(1)
    t = bsgs_t(n, n)
    w = rng.normal(0, 1 / np.sqrt(f), f)
    W1 = rng.normal(0, 1 / np.sqrt(n), (n, n))
    W2 = rng.normal(0, 1 / np.sqrt(n - pool + 1), (n - pool + 1, n - pool + 1))
    W2s = np.zeros((n - pool + 1, n))
    W2s[:, pool - 1:] = W2
    layers = [("conv1d", w, n, t), ("dense", W1), ("replicate", t), ("poly3", RELU_APPROX), ("avgpool", pool),
              ("dense", W2s)]
    return layers, (w, W1, W2, pool)


def paper_fp64(weights, x):
    w, W1, W2, pool = weights
    h = np.correlate(x, w, "same")
    z = W1 @ h
    a = RELU_APPROX
    r = ((a[3] * z + a[2]) * z + a[1]) * z + a[0]
    p = np.array([np.mean(r[k:k + pool]) for k in range(len(r) - pool + 1)])
    return W2 @ p


def inputs_for(N, dims, B, t0, windows=1):
    """B ciphertexts of `windows` inputs each, input j of a ciphertext as [x, x] at block
    stride t0 in slots [2 t0 j, 2 t0 (j+1)); returns xs [B][windows][n] and the slots."""
    rng = np.random.default_rng(2)
    xs = rng.uniform(-1, 1, (B, windows, dims[0]))
    slots = np.zeros((B, N // 2))
    for j in range(windows):
        slots[:, 2 * t0 * j:2 * t0 * j + dims[0]] = xs[:, j]
        slots[:, 2 * t0 * j + t0:2 * t0 * j + t0 + dims[0]] = xs[:, j]
    return xs, slots


def fp64_forward(Ws, x, square_last):
    h = x
    for i, W in enumerate(Ws):
        h = W @ h
        if i + 1 < len(Ws) or square_last:
            h = h * h
    return h


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = []
        mx = MAX_SM_MHZ
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = float(s[1])
                for n, v in zip(names, s[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def op_plan(wl):
    """(key switches, plaintext products, rescales, level) per step of the forward, in the
    oracle's terms: a key switch is a rotation or a relinearisation, a ciphertext product's
    tensor counts as 1.5 (square) or 2 (two operands) plaintext products."""
    L = len(wl["q"])
    plan, lvl = [], L

    form = wl.get("dense_form", "square")
    lazy = form in ("lazy", "rect_lazy")

    def split(t):
        lg = t.bit_length() - 1
        if lazy:  # the lazy-ModDown form's split, min(t, 2^ceil(log2(4t)/2))
            t1 = min(t, 1 << ((lg + 3) // 2))
        else:  # the composed form's split, 2^ceil(log2(t)/2)
            t1 = 1 << ((lg + 1) // 2)
        return t1, t // t1

    if wl.get("net") == "paper":
        n, t = wl["dims"][0], bsgs_t(wl["dims"][0], wl["dims"][0])
        t1, t2 = split(t)
        plan.append((8, 9, 1, lvl)); lvl -= 1                     # conv1d f=9
        plan.append((t1 + t2 - 2, t, 1, lvl)); lvl -= 1           # dense
        plan.append((1, 0, 0, lvl))                               # replicate
        plan.append((1, 1.5, 3, lvl)); plan.append((1, 2, 1, lvl - 1)); lvl -= 2  # ReLU approx
        plan.append((2, 0, 1, lvl)); lvl -= 1                     # avgpool 3
        plan.append((t1 + t2 - 2, t, 1, lvl))                     # dense
        return plan
    dims = wl["dims"]
    rect = form in ("rect", "rect_lazy")
    for i in range(len(dims) - 1):
        tm, tn = bsgs_t(dims[i + 1], 1), bsgs_t(dims[i], 1)
        last = i + 1 == len(dims) - 1
        if rect and tm < tn:
            # rectangular form: Eq. (bsgs) over tm diagonals, then the fold after the rescale
            # (log2(tn/tm) rotations, one more when it also forms the next layer's [y, y])
            t1, t2 = split(tm)
            fuse = not last and bsgs_t(dims[i + 2], dims[i + 1]) == tm
            plan.append((t1 + t2 - 2, tm, 1, lvl))
            plan.append(((tn // tm).bit_length() - 1 + (1 if fuse else 0), 0, 0, lvl - 1))
        else:
            t = bsgs_t(dims[i + 1], dims[i])
            t1, t2 = split(t)
            plan.append((t1 + t2 - 2, t, 1, lvl))
            fuse = False
        lvl -= 1
        if not last or wl.get("square_last", False):
            plan.append((1, 1.5, 1, lvl))  # square: 3 products, relinearisation, rescale
            lvl -= 1
            if not last and not fuse:
                plan.append((1, 0, 0, lvl))  # replicate
    return plan


class OracleSample:
    """A bounded sample of the workload on the oracle (the plain C++ CKKS implementation),
    timed on the host cores.  set-up (keys, plaintexts) is not timed; step() runs one sample
    and returns its seconds; `fraction` is the share of one encrypted forward a sample does.

    Rings of N <= 4096 (the dense/square networks): a sample is one whole forward
    (fraction 1), with its decoded error against FP64.  Larger rings: a sample is one
    rotation, one plaintext product and one rescale at the workload's top level; the
    forward is that many samples as its operation counts say (key switches weighted by
    their digits x limbs relative to the top level, products and rescales by their limbs),
    with the weights taken from the timed sample itself."""

    def __init__(self, wl, whole=None):
        from oracle import ckks_oracle as O

        self.wl = wl
        self.cores = os.cpu_count()
        N, q = wl["N"], wl["q"]
        self.whole = (N <= 4096 and wl.get("net") != "paper") if whole is None else whole
        self.o = O.Oracle(N, q, wl["p"], dnum=wl["dnum"], scale=wl.get("scale", 2.0 ** 40))
        o = self.o
        if self.whole:
            square_last = wl.get("square_last", False)
            layers, self.Ws = layers_for(wl["dims"], square_last)
            form = wl.get("dense_form", "square")
            rect, lazy = form in ("rect", "rect_lazy"), form in ("lazy", "rect_lazy")
            rots, skip = set(), set()
            for ly in layers:
                if ly[0] == "replicate":
                    rots.add(-ly[1])
            lvl, sc, self.plan = len(q), o.scale, []
            for i, ly in enumerate(layers):  # plaintexts at the level and scale each layer sees
                if i in skip:
                    continue
                if ly[0] == "dense":
                    m, n = ly[1].shape
                    tm, tn = bsgs_t(m, 1), bsgs_t(n, 1)
                    if rect and tm < tn:  # the rectangular form, as the library's CTL_DENSE_RECT
                        j = i + 1 + (1 if i + 1 < len(layers) and layers[i + 1][0] == "square" else 0)
                        fold = 2 if j < len(layers) and layers[j] == ("replicate", tm) else 1
                        if fold == 2:
                            skip.add(j)
                        rots |= set(O.Oracle.rect_rotations(m, n, fold, lazy))
                        self.plan.append(("rect", o.encode_diagonals_rect(ly[1], o.dense_scale(lvl, sc), lazy), tn,
                                          fold))
                    else:
                        rots |= set(O.Oracle.bsgs_rotations(m, n, lazy))
                        self.plan.append(("dense", o.encode_diagonals(ly[1], o.dense_scale(lvl, sc), lazy)))
                    sc, lvl = o.scale, lvl - 1
                elif ly[0] == "square":
                    self.plan.append(("square",))
                    sc, lvl = o.square_scale(lvl, sc), lvl - 1
                else:
                    self.plan.append(ly)
            o.keygen(sorted(rots), seed=3)
            self.lazy = lazy
            self.out_scale = sc
            t0 = bsgs_t(*self.Ws[0].shape)
            self.xs, slots = inputs_for(N, wl["dims"], 1, t0)
            self.ct = o.encrypt(o.encode(slots[0]), 4)
            self.fraction = 1.0
            self.err = None
        else:
            o.keygen([1], seed=3)
            rng = np.random.default_rng(9)
            L = len(q)
            self.ct = np.stack([np.stack([rng.integers(0, m, N, dtype=np.uint64) for m in o.moduli[:L]])
                                for _ in range(2)])
            self.pt = rng.integers(-2 ** 20, 2 ** 20, N, dtype=np.int64)
            self.fraction = None
            self.parts = None

    def step(self):
        o = self.o
        t0 = time.perf_counter()
        if self.whole:
            h = self.ct
            for st in self.plan:
                if st[0] == "dense":
                    h = o.dense(h, st[1], lazy=self.lazy)[0]
                elif st[0] == "rect":
                    h = o.dense_rect(h, st[1], st[2], fold=st[3], lazy=self.lazy)[0]
                elif st[0] == "square":
                    h = o.square(h)
                else:
                    h = o.replicate(h, st[1])
            secs = time.perf_counter() - t0
            if self.err is None:
                sq = self.wl.get("square_last", False)
                y = o.decode(o.decrypt(h), self.wl["dims"][-1], self.out_scale)
                self.err = float(np.max(np.abs(y - fp64_forward(self.Ws, self.xs[0, 0], sq))))
            return secs
        o.rotate(self.ct, 1)
        t1 = time.perf_counter()
        o.mul_plain(self.ct, self.pt)
        t2 = time.perf_counter()
        o.rescale(self.ct)
        t3 = time.perf_counter()
        self.parts = (t1 - t0, t2 - t1, t3 - t2)
        self.fraction = (t3 - t0) / self.forward_seconds(*self.parts)
        return t3 - t0

    def forward_seconds(self, t_rot, t_pt, t_rs):
        """One forward from the operation counts, each operation at its level."""
        wl = self.wl
        L, K = len(wl["q"]), len(wl["p"])
        alpha = (L + wl["dnum"] - 1) // wl["dnum"]

        def ks_scale(lv):
            return (((lv + alpha - 1) // alpha) * (lv + K)) / (((L + alpha - 1) // alpha) * (L + K))

        return sum(ks * t_rot * ks_scale(lv) + npt * t_pt * lv / L + nrs * t_rs * lv / L
                   for ks, npt, nrs, lv in op_plan(wl))

    def describe(self):
        if self.whole:
            return (f"one whole forward per step on the oracle ({self.cores} host threads), N={self.wl['N']}; "
                    f"decoded error {self.err:.1e} against FP64")
        t_rot, t_pt, t_rs = self.parts
        return (f"oracle on {self.cores} host threads, per step: 1 rotation ({t_rot:.2f} s), 1 plaintext product "
                f"({t_pt:.2f} s) and 1 rescale ({t_rs:.3f} s) at N={self.wl['N']}, level {len(self.wl['q'])}; "
                f"a step is {self.fraction:.2e} of a forward by the forward's operation and limb counts "
                f"(forwards/s extrapolated from the timed steps)")


def cpu_oracle_sample(wl, steps=1):
    """The oracle's forwards/s on the host cores from `steps` timed samples (see
    OracleSample); returns (forwards/s, description, cores, per-step seconds)."""
    smp = OracleSample(wl)
    secs = [smp.step() for _ in range(steps)]
    t = statistics.median(secs)
    return smp.fraction / t, smp.describe(), smp.cores, secs


def shared_config(wl, world, **extra):
    """The `config` object both arms print for the same workload."""
    cfg = {"workload": wl["desc"], "batch_per_gpu": wl["batch"], "N": wl["N"],
           "parallelism": f"replicas x{world}", "dense_form": wl.get("dense_form", "square"),
           "l2": "inputs larger than L2 (working set of tens of GB per step)"}
    cfg.update(extra)
    return cfg


def run_reference(args, wl, rank, world):
    """The oracle as the reference arm: W untimed and K timed steps, each one bounded
    sample of the workload (OracleSample) on rank 0's host cores; other ranks do no work."""
    if rank != 0:
        return
    smp = OracleSample(wl)
    for _ in range(args.warmup):
        smp.step()
    t_start = time.perf_counter()
    secs = [smp.step() for _ in range(args.steps)]
    total = time.perf_counter() - t_start
    value = smp.fraction * len(secs) / total
    line = {"impl": "reference", "metric": "encrypted forwards/sec (batched)", "value": value,
            "unit": "forwards/s", "n_gpus": args.gpus, "steps": len(secs), "warmup": args.warmup,
            "ms_per_step": total * 1e3 / len(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": shared_config(wl, world),
            "cpu_baseline": {"value": value, "unit": "forwards/s", "cores": smp.cores, "kind": "oracle",
                             "sample": smp.describe()},
            "e2e": {"value": value, "unit": "forwards/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SHAPES = {  # the three query shapes of the serving mix (configurations 1-3)
    "cfg1": dict(N=4096, q=[50, 40, 40], p=[60], dnum=3, dims=[64, 32], square_last=True),
    "cfg2": dict(N=8192, q=[60, 40, 40, 40], p=[60], dnum=4, dims=[512, 128, 64], square_last=False),
    "cfg3": dict(N=16384, q=[45] * 8, p=[60, 60], dnum=4, dims=[1024, 256, 256, 64], square_last=False),
}


def _slots(N, n_in, t0, x):
    s = np.zeros(N // 2)
    s[:n_in] = x
    s[t0:t0 + n_in] = x
    return s


def run_serving(args, ctl):
    """Configuration 5: Poisson arrivals from 64 clients, each with its own keys resident
    in HBM and a query shape drawn uniformly from configurations 1-3; continuous batching
    with memory admission; p50/p99 latency (submit to result on the host) and throughput
    per arrival rate."""
    rng = np.random.default_rng(5)
    lanes = {}
    srv = ctl.Server(mem_budget_bytes=int(args.mem_budget_gb * 2 ** 30), n_workers=args.workers,
                     max_batch=args.max_batch, max_queue=100000)
    for name, sh in SHAPES.items():
        layers, Ws = layers_for(sh["dims"], sh["square_last"])
        ctx = ctl.Context(sh["N"], sh["q"], sh["p"], dnum=sh["dnum"], scale=2.0 ** 40)
        model = ctl.Model(ctx, layers)
        lanes[name] = (ctx, model, srv.add_lane(ctx, model), bsgs_t(Ws[0].shape[0], Ws[0].shape[1]))
    clients = []
    for c in range(args.clients):
        name = list(SHAPES)[rng.integers(3)]
        ctx, model, lane, t0 = lanes[name]
        keys = ctx.keygen(model.rotations(), seed=1000 + c)
        cid = srv.add_client(lane, keys)
        pool = []
        for i in range(4):  # a few distinct ciphertexts per client, resubmitted
            x = rng.uniform(-1, 1, SHAPES[name]["dims"][0])
            pool.append(ctx.encrypt(keys, _slots(ctx.N, len(x), t0, x), 4 + 100 * c + i).export()[0])
        clients.append((cid, name, pool, srv.io_words(cid)[1]))
    srv.start()
    points = []
    for lam in args.rates:
        before = srv.stats()
        t_end = time.perf_counter() + args.seconds
        t_next = time.perf_counter()
        ids = []
        while True:
            t_next += rng.exponential(1.0 / lam)
            if t_next > t_end:
                break
            d = t_next - time.perf_counter()
            if d > 0:
                time.sleep(d)
            cid, name, pool, ow = clients[rng.integers(len(clients))]
            rid = srv.submit(cid, pool[rng.integers(len(pool))])
            if rid is not None:
                ids.append((rid, ow))
        t0 = time.perf_counter()
        lats = []
        for rid, ow in ids:
            _, lat = srv.wait(rid, ow, timeout_ms=600000)
            lats.append(lat)
        wall = (t_end - (t_end - args.seconds)) + (time.perf_counter() - t0)
        after = srv.stats()
        lats.sort()
        points.append({"rate_req_s": lam, "completed": len(lats),
                       "throughput_fwd_s": len(lats) / wall if wall > 0 else 0.0,
                       "p50_ms": float(np.percentile(lats, 50)) if lats else None,
                       "p99_ms": float(np.percentile(lats, 99)) if lats else None,
                       "rejected": after["rejected"] - before["rejected"],
                       "batches": after["batches"] - before["batches"]})
    srv.close()
    return points


def run_uneven(args, ctl):
    """Configuration 4: 1024 queries with N in {8192, 16384}, depth 2..6 and input
    dimension in {128, 256, 512, 1024}, uniformly.  Chain q0 = 60 bits plus d primes of
    40 bits; one 60-bit special prime at N = 8192, two (alpha = 2) at N = 16384.  Network:
    alternating dense (in -> 128, 128 -> 128, the last -> 64) and x^2, d levels in all.
    Grouped execution (queries of one shape batched, groups overlapped by the server's
    workers) against one launch sequence per ciphertext."""
    rng = np.random.default_rng(4)
    shapes = {}
    for Nn in (8192, 16384):
        for d in range(2, 7):
            q = [60] + [40] * d
            p = [60] if Nn == 8192 else [60, 60]
            dnum = len(q) if Nn == 8192 else (len(q) + 1) // 2
            ctx = ctl.Context(Nn, q, p, dnum=dnum, scale=2.0 ** 40)
            ctx.set_dense_mode(getattr(ctx, DENSE_FORMS[args.dense_form or "rect_lazy"]))
            shapes[(Nn, d)] = {"ctx": ctx, "models": {}}
    queries = [((int(rng.choice([8192, 16384])), int(rng.integers(2, 7))), int(rng.choice([128, 256, 512, 1024])))
               for _ in range(args.queries)]
    srv = ctl.Server(mem_budget_bytes=int(args.mem_budget_gb * 2 ** 30), n_workers=args.workers,
                     max_batch=args.max_batch, max_queue=100000)
    clients = {}
    for (key, dim) in sorted(set(queries)):
        Nn, d = key
        sh = shapes[key]
        ctx = sh["ctx"]
        w = np.random.default_rng(dim + d)
        layers, dims_now, ops = [], dim, 0
        while ops < d:
            out = 64 if ops + 2 >= d else 128
            if ops > 0:
                layers.append(("replicate", bsgs_t(out, dims_now)))
            layers.append(("dense", w.normal(0, 1 / np.sqrt(dims_now), (out, dims_now))))
            dims_now, ops = out, ops + 1
            if ops < d:
                layers.append(("square",))
                ops += 1
        model = ctl.Model(ctx, layers)
        sh["models"][dim] = model
        sh["rots"] = sh.get("rots", set()) | set(model.rotations())  # one key set per context
    for key, sh in shapes.items():
        sh["keys"] = sh["ctx"].keygen(sorted(sh.get("rots", set())), seed=77)
    cts = []
    for i, (key, dim) in enumerate(queries):
        sh = shapes[key]
        ctx = sh["ctx"]
        t0 = bsgs_t(128 if key[1] > 2 else 64, dim)
        x = rng.uniform(-1, 1, dim)
        cts.append(ctx.encrypt(sh["keys"], _slots(ctx.N, dim, t0, x), 9000 + i))
    lanes = {}
    for key, sh in shapes.items():
        for dim, model in sh["models"].items():
            lane = srv.add_lane(sh["ctx"], model)
            lanes[(key, dim)] = srv.add_client(lane, sh["keys"])
    srv.start()
    coeffs = [ct.export()[0] for ct in cts]
    # grouped: submit everything, the server batches per shape and overlaps groups
    t0 = time.perf_counter()
    ids = [(srv.submit(lanes[q], coeffs[i]), srv.io_words(lanes[q])[1]) for i, q in enumerate(queries)]
    for rid, ow in ids:
        srv.wait(rid, ow, timeout_ms=600000)
    grouped = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    # one forward per ciphertext, in submission order
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (key, dim) in enumerate(queries):
        sh = shapes[key]
        o = sh["models"][dim].forward(sh["keys"], cts[i])
        o.close()
    for sh in shapes.values():
        sh["ctx"].synchronize()
    single = time.perf_counter() - t0
    # one CUDA graph for the whole uneven batch: each shape group (its queries batched) is a
    # branch of the graph on its own context clone's stream (ctl_multi_*), one launch per batch
    groups, ins, members = [], [], []
    for (key, dim) in sorted(set(queries)):
        sh = shapes[key]
        idx = [i for i, q in enumerate(queries) if q == (key, dim)]
        clone = sh["ctx"].clone()
        groups.append((clone, sh["models"][dim], sh["keys"], len(idx)))
        ins.append(sh["ctx"].concat([cts[i] for i in idx]))
        members.append(idx)
    multi = ctl.Multi(groups)
    outs = multi.forward(ins)  # check against each query's own forward on a sample
    same = True
    for g in range(0, len(groups), max(1, len(groups) // 8)):
        key, dim = queries[members[g][0]]
        sh = shapes[key]
        alone = sh["models"][dim].forward(sh["keys"], cts[members[g][0]]).export()[0]
        same = same and bool(np.array_equal(outs[g].export()[0], alone))
    for o in outs:
        o.close()
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        for o in multi.forward(ins):
            o.close()
    for clone, _, _, _ in groups:
        clone.synchronize()
    one = (time.perf_counter() - t0) / reps
    multi.close()
    for clone, _, _, _ in groups:
        clone.close()
    return {"queries": len(queries), "shapes": len(set(queries)), "grouped_fwd_s": len(queries) / grouped,
            "per_ct_fwd_s": len(queries) / single, "speedup": single / grouped, "server_batches": st["batches"],
            "one_graph_fwd_s": len(queries) / one, "one_graph_vs_per_ct": single / one,
            "one_graph_bit_identical_to_single": same,
            "one_graph_desc": "all shape groups as branches of one CUDA graph (ctl_multi_forward), one launch per "
                              "batch of 1024 queries, device-resident inputs"}


def single_query_point(ctl, torch, name, steps):
    """One query per forward through the replayed CUDA graph: forwards/s and p50/p99 of the
    per-forward device time (CUDA events on the library's stream), inputs resident."""
    wl = WORKLOADS[name]
    layers, Ws = layers_for(wl["dims"], wl.get("square_last", False))
    t0 = bsgs_t(Ws[0].shape[0], Ws[0].shape[1])
    stream = torch.cuda.Stream()
    ctx = ctl.Context(wl["N"], wl["q"], wl["p"], dnum=wl["dnum"], scale=2.0 ** 40)
    ctx.set_stream(stream.cuda_stream)
    ctx.set_dense_mode(getattr(ctx, DENSE_FORMS[wl.get("dense_form", "square")]))
    model = ctl.Model(ctx, layers)
    keys = ctx.keygen(model.rotations(), seed=3)
    xs, slots = inputs_for(wl["N"], wl["dims"], 1, t0)
    ct = ctx.encrypt(keys, slots[0], 4)
    o = model.forward(keys, ct, graph=True)
    y = ctx.decrypt(keys, o, wl["dims"][-1])
    err = float(np.max(np.abs(y - fp64_forward(Ws, xs[0, 0], wl.get("square_last", False)))))
    o.close()
    for _ in range(10):
        model.forward(keys, ct, graph=True).close()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        model.forward(keys, ct, graph=True).close()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
    total = ev[0].elapsed_time(ev[-1])
    # end to end through the C-ABI: the query imported from host memory (coefficient form, as
    # the client sends it), the graph forward, the result exported to host memory, each step
    coeffs = ct.export()[0]
    lat = []
    for i in range(steps):
        t0 = time.perf_counter()
        ci = ctx.ct_import(coeffs, 2.0 ** 40)
        co = model.forward(keys, ci, graph=True)
        co.export()
        lat.append((time.perf_counter() - t0) * 1e3)
        ci.close()
        co.close()
    lat.sort()
    res = {"desc": wl["desc"].replace("256 ciphertexts", "1 ciphertext"), "value": steps / (total / 1e3),
           "unit": "forwards/s", "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
           "steps": steps, "cuda_graph": True, "max_abs_err_vs_fp64": err,
           "e2e": {"value": steps / (sum(lat) / 1e3), "unit": "forwards/s", "p50_ms": float(np.percentile(lat, 50)),
                   "p99_ms": float(np.percentile(lat, 99)),
                   "desc": "host coefficients in, graph forward, host coefficients out, per query (wall clock)"}}
    ct.close()
    model.close()
    keys.close()
    ctx.close()
    return res


def client_round_trip_point(ctl, torch, ctx, model, keys, slots, m_out, steps):
    """The whole protocol for a batch, client side on the device too: the slot vectors
    copied from pinned host memory, encoded and encrypted on the GPU (ctl_encrypt_dev), the
    forward (graph), decrypted and decoded on the GPU (ctl_decrypt_dev), and the outputs
    copied back to pinned host memory, every step."""
    B, nz = slots.shape
    host_in = torch.from_numpy(np.ascontiguousarray(slots)).pin_memory()
    host_out = torch.empty((B, m_out), dtype=torch.float64).pin_memory()
    z_dev = torch.empty((B, nz), dtype=torch.float64, device="cuda")
    y_dev = torch.empty((B, m_out), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def one(step):
        z_dev.copy_(host_in, non_blocking=True)
        stream.synchronize()
        ct = ctx.encrypt_dev(keys, z_dev.data_ptr(), nz, B, [1000003 * step + b for b in range(B)])
        out = model.forward(keys, ct, graph=True)
        ctx.decrypt_dev(keys, out, m_out, y_dev.data_ptr())
        ctx.synchronize()
        host_out.copy_(y_dev, non_blocking=True)
        torch.cuda.synchronize()
        ct.close()
        out.close()

    one(0)
    t0 = time.perf_counter()
    for s in range(steps):
        one(s + 1)
    secs = time.perf_counter() - t0
    return {"value": B * steps / secs, "unit": "forwards/s", "steps": steps, "batch": B,
            "h2d_bytes_per_step": int(host_in.numel() * 8), "d2h_bytes_per_step": int(host_out.numel() * 8),
            "desc": "host FP64 slots -> device encode + encrypt (ctl_encrypt_dev) -> forward (graph) -> device "
                    "decrypt + decode (ctl_decrypt_dev) -> host FP64 outputs, every step (wall clock)"}


def serving_point(ctl, rate, seconds, n_clients):
    """One arrival rate of configuration 5 (see run_serving), fewer clients and seconds."""
    ns = argparse.Namespace(mem_budget_gb=160.0, workers=4, max_batch=64, clients=n_clients, rates=[rate],
                            seconds=seconds)
    pt = run_serving(ns, ctl)[0]
    pt.update({"clients": n_clients, "seconds": seconds, "unit": "forwards/s",
               "desc": "Poisson arrivals, query shapes of configurations 1-3, per-client keys resident, "
                       "continuous batching with memory admission; latency = submit to result on the host"})
    return pt


def max_over_ranks(x, dist):
    """The slowest rank's time: every rank runs its own replica on its own GPU (the
    queries are independent, so there is no data-path collective), and the job's time is
    the maximum over ranks.  NCCL reduces a device tensor, gloo a host one."""
    if not dist:
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, batch, steps, seconds):
    """Whole-job forwards per second: world replicas of `batch` ciphertexts per step."""
    return world * batch * steps / seconds


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (default 5; 500 for single-query workloads, so that the clock sampler sees "
                         "the timed region)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=list(WORKLOADS) + ["serving", "uneven"])
    ap.add_argument("--batch", type=int, default=0, help="override the batch size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--graph", type=int, default=1, help="1 (default): replay a CUDA graph of the forward; 0: eager")
    ap.add_argument("--class-steps", type=int, default=2,
                    help="eager forwards timed per kernel class after the timed steps (roofline breakdown)")
    ap.add_argument("--rates", type=float, nargs="+", default=[50, 100, 200, 500, 1000, 2000])
    ap.add_argument("--seconds", type=float, default=5.0, help="serving: load duration per arrival rate")
    ap.add_argument("--clients", type=int, default=64)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--mem-budget-gb", type=float, default=160.0)
    ap.add_argument("--queries", type=int, default=1024)
    ap.add_argument("--ntt-shape", default="auto", choices=["auto", "r32", "r16"],
                    help="register NTT shape (default: the context's autotuned choice)")
    ap.add_argument("--bsgs-shape", default="", help="chunk,karatsuba for the BSGS kernel (default: library's)")
    ap.add_argument("--profile-forward", action="store_true",
                    help="run one eager forward inside cudaProfilerStart/Stop and print its per-class "
                         "algorithmic work and bytes (for an ncu capture of exactly that forward)")
    ap.add_argument("--dense-form", default="", choices=[""] + list(DENSE_FORMS),
                    help="square / lazy / rect / rect_lazy (ctl_set_dense_mode); default: the workload's "
                         "(rect_lazy for the batched network, square otherwise)")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the single-query and serving points measured beside the batched value")
    ap.add_argument("--single-steps", type=int, default=300, help="timed single-query forwards per point")
    ap.add_argument("--serve-rate", type=float, default=500.0, help="arrival rate of the serving point (req/s)")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--serve-clients", type=int, default=16)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the extra measurement of the lazy-ModDown dense form")
    args = ap.parse_args()
    if args.workload in ("serving", "uneven"):
        import torch

        import __graft_entry__

        __graft_entry__.build()
        from paper_2205_11935_gb300 import ctl

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        res = run_serving(args, ctl) if args.workload == "serving" else run_uneven(args, ctl)
        print(json.dumps({"workload": args.workload, "result": res}), flush=True)
        return
    wl = dict(WORKLOADS[args.workload])
    if args.batch:
        wl["batch"] = args.batch
    if args.dense_form:
        wl["dense_form"] = args.dense_form
    if not args.steps:
        args.steps = 500 if wl["batch"] == 1 else 5

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    # one rank per node compiles (the object files are shared); the others wait for it
    if local == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    if local != 0:
        __graft_entry__.build()  # up to date by now: returns at once
    from paper_2205_11935_gb300 import ctl

    N, B = wl["N"], wl["batch"]
    scale = wl.get("scale", 2.0 ** 40)
    square_last = wl.get("square_last", False)
    if wl.get("net") == "paper":
        layers, pw = paper_layers_for(wl["dims"][0])
        t0 = bsgs_t(wl["dims"][0], wl["dims"][0])

        def reference(x):
            return paper_fp64(pw, x)
    else:
        layers, Ws = layers_for(wl["dims"], square_last)
        t0 = bsgs_t(Ws[0].shape[0], Ws[0].shape[1])

        def reference(x):
            return fp64_forward(Ws, x, square_last)
    stream = torch.cuda.Stream()
    ctx = ctl.Context(N, wl["q"], wl["p"], dnum=wl["dnum"], scale=scale)
    ctx.set_stream(stream.cuda_stream)
    # Sec. 3.1 "Multiple Predictions": the paper's network packs p = floor(#slots / 2t)
    # inputs per ciphertext (one window of 2t slots each)
    windows = (N // 2) // (2 * t0) if wl.get("net") == "paper" else 1
    dense_form = args.dense_form or wl.get("dense_form", "square")
    wl["dense_form"] = dense_form
    ctx.set_dense_mode(getattr(ctx, DENSE_FORMS[dense_form]))
    ctx.set_windows(windows)
    if args.ntt_shape != "auto":
        sh = ctx.NTT_R16 if args.ntt_shape == "r16" else ctx.NTT_R32
        ctx.set_ntt_shape(sh, sh)
    if args.bsgs_shape:
        ctx.set_bsgs_shape(*[int(v) for v in args.bsgs_shape.split(",")])
    shape_names = {ctx.NTT_R32: "r32", ctx.NTT_R16: "r16"}
    ntt_shape = dict(zip(("fwd", "inv"), (shape_names.get(v, str(v)) for v in ctx.ntt_shape())))
    model = ctl.Model(ctx, layers)
    keys = ctx.keygen(model.rotations(), seed=3)
    xs, slots = inputs_for(N, wl["dims"], B, t0, windows)
    cts = [ctx.encrypt(keys, slots[i], 4 + i) for i in range(B)]
    batch = ctx.concat(cts)
    for c in cts:
        c.close()
    out_level, out_scale, model_bytes = model.info()

    # correctness of the measured configuration: decoded outputs vs FP64 on a sample
    out = model.forward(keys, batch)
    check_idx = sorted({0, B // 2, B - 1})
    max_err = 0.0
    m_out = wl["dims"][-1]
    for i in check_idx:
        yi = ctx.decrypt(keys, out.slice(i), 2 * t0 * (windows - 1) + m_out)
        for j in range(windows):
            max_err = max(max_err, float(np.max(np.abs(yi[2 * t0 * j:2 * t0 * j + m_out] - reference(xs[i, j])))))
    out.close()

    if args.profile_forward:
        # one eager forward between cudaProfilerStart/Stop (for ncu --profile-from-start off),
        # with the library's per-class algorithmic work and bytes of the same launches
        model.forward(keys, batch).close()
        torch.cuda.synchronize()
        ctx.stats_reset()
        ctx.stats_enable_timing(True)
        torch.cuda.profiler.start()
        model.forward(keys, batch).close()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        kern = {k: v for k, v in ctx.stats_kernels().items() if v["launches"]}
        print(json.dumps({"profile_forward": wl["desc"], "batch": B, "launches": ctx.stats_launches(),
                          "classes": kern}), flush=True)
        return

    # the forward replays one captured CUDA graph by default (all launches of the network,
    # captured once per batch size); --graph 0 times eager launches instead
    use_graph = args.graph != 0

    def step():
        o = model.forward(keys, batch, graph=use_graph)
        o.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: device-resident inputs, no per-launch events
    ctx.stats_reset()
    ctx.stats_enable_timing(False)
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for s in range(args.steps):
        step()
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    launches = ctx.stats_launches()
    ops = ctx.stats_ops()
    total_ms = max_over_ranks(total_ms, dist)
    value = replica_throughput(world, B, args.steps, total_ms / 1e3)

    # per-kernel-class device time in a separate pass: eager forwards of the same kernels
    # with CUDA events around every launch on the library's stream (untimed for `value`)
    ctx.stats_reset()
    ctx.stats_enable_timing(True)
    class_steps = max(1, min(args.steps, args.class_steps))
    for _ in range(class_steps):
        o = model.forward(keys, batch)
        o.close()
    kern = ctx.stats_kernels()
    ctx.stats_enable_timing(False)
    class_ms_per_step = sum(v["ms"] for v in kern.values()) / class_steps
    timing_source = (f"CUDA events around every launch of {class_steps} eager forwards run after the timed "
                     f"steps (the timed steps replay the graph without events)")

    # end to end through host buffers
    e2e = None
    if not args.no_e2e:
        host_in = batch.export()  # coefficient form, as a client would send it
        pinned_in = torch.from_numpy(host_in.view(np.int64)).pin_memory()
        h2d = host_in.nbytes
        out_words = B * 2 * out_level * N
        pinned_out = torch.empty(out_words, dtype=torch.int64).pin_memory()
        import ctypes as C

        # two streams: step i+1's upload (H2D copy and transform, on a context clone's
        # stream) and step i's download (D2H copy) overlap step i's forward; every step
        # still uploads its inputs and reads its result back inside the timed region
        io_stream = torch.cuda.Stream()
        ctx_io = ctx.clone(io_stream.cuda_stream)
        out_dev = [torch.empty(out_words, dtype=torch.int64, device="cuda") for _ in range(2)]
        pinned_outs = [pinned_out, torch.empty(out_words, dtype=torch.int64).pin_memory()]

        def e2e_run(steps):
            ci, ev_in, d2h = [None] * steps, [None] * steps, [None] * steps

            def upload(i):
                h = C.c_void_p()
                ctl._check(ctl.lib().ctl_ct_import(ctx_io.h, C.cast(pinned_in.data_ptr(), ctl._u64p), B,
                                                   len(wl["q"]), scale, C.byref(h)))
                ci[i] = ctl.Ciphertext(ctx_io, h)
                ev_in[i] = torch.cuda.Event()
                ev_in[i].record(io_stream)

            upload(0)
            for i in range(steps):
                stream.wait_event(ev_in[i])
                co = model.forward(keys, ci[i], graph=use_graph)
                if i + 1 < steps:
                    upload(i + 1)
                if i >= 2:
                    stream.wait_event(d2h[i - 2])  # staging buffer i % 2 has been read back
                ctl._check(ctl.lib().ctl_ct_export_dev(co.h, C.c_void_p(out_dev[i % 2].data_ptr()), out_words))
                done = torch.cuda.Event()
                done.record(stream)
                io_stream.wait_event(done)
                with torch.cuda.stream(io_stream):
                    pinned_outs[i % 2].copy_(out_dev[i % 2], non_blocking=True)
                d2h[i] = torch.cuda.Event()
                d2h[i].record(io_stream)
                co.close()
                ci[i].close()  # freed on the upload stream, after the forward (waited above)
            torch.cuda.synchronize()

        e2e_run(1)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t_start = time.perf_counter()
        e2e_run(args.steps)
        e2e_s = time.perf_counter() - t_start
        ctx_io.close()
        e2e_s = max_over_ranks(e2e_s, dist)
        e2e = {"value": replica_throughput(world, B, args.steps, e2e_s), "unit": "forwards/s",
               "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(out_words * 8)}

    # the same workload with the dense layers in the lazy-ModDown form (a different, equally
    # valid ciphertext; its own BSGS split and Galois keys): reported beside, not as, the value
    variants = None
    if not args.no_variants and world == 1:
        # the same workload with the dense layers in the other forms (different, equally valid
        # ciphertexts with their own Galois keys): reported beside, not as, the value
        forms = {name: (getattr(ctx, DENSE_FORMS[name]), DENSE_FORM_DESC[name]) for name in DENSE_FORMS
                 if name != dense_form}
        variants = {}
        for name, (mode, desc) in forms.items():
            ctx.set_dense_mode(mode)
            model_l = ctl.Model(ctx, layers)
            keys_l = ctx.keygen(model_l.rotations(), seed=3)  # same secret (same seed)
            o = model_l.forward(keys_l, batch)
            err_l = 0.0
            for i in check_idx:
                yi = ctx.decrypt(keys_l, o.slice(i), 2 * t0 * (windows - 1) + m_out)
                for j in range(windows):
                    err_l = max(err_l, float(np.max(np.abs(yi[2 * t0 * j:2 * t0 * j + m_out] - reference(xs[i, j])))))
            o.close()
            for _ in range(2):
                model_l.forward(keys_l, batch).close()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                model_l.forward(keys_l, batch).close()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_l = e0.elapsed_time(e1)
            variants[name] = {
                "value": B * args.steps / (ms_l / 1e3), "unit": "forwards/s", "ms_per_step": ms_l / args.steps,
                "max_abs_err_vs_fp64": err_l, "rotation_keys": len(model_l.rotations()), "cuda_graph": False,
                "desc": desc}
            model_l.close()
            keys_l.close()
        ctx.set_dense_mode(getattr(ctx, DENSE_FORMS[dense_form]))

    # rooflines per kernel class.  Work units: Shoup modmuls for the transform classes and
    # split-half MACs for the key product and BSGS sums; each unit's peak is this GPU's rate
    # measured now by the unit-rate microbenchmark (ctl_microbench_unit_rate) at the maximum
    # SM clock; the HBM side takes the class's algorithmic bytes against the measured copy
    # bandwidth.  A class's roofline time is max(bytes / HBM, work / unit peak) and its
    # fraction that time over the measured one.
    ub = {name: ctl.microbench_unit_rate(kind) for kind, name in
          enumerate(("shoup_modmul", "harvey_butterfly", "shoup_three_half", "split_mac"))}
    clk = MAX_SM_MHZ * 1e6
    peak_modmul = SM_COUNT * clk * ub["shoup_modmul"]
    peak_mac = SM_COUNT * clk * ub["split_mac"]
    imad_slots = SM_COUNT * IMAD_PER_CLK_SM * clk
    hbm_gbs, hbm_src = hbm_peak_gbs()
    classes = {k: v for k, v in kern.items() if v["launches"]}

    def unit_peak(k):
        return ("Gmac/s", peak_mac) if k in MAC_CLASSES else ("Gmodmul/s", peak_modmul)

    per_class = {}
    for k, v in classes.items():
        secs = v["ms"] / 1e3
        u, pk = unit_peak(k)
        t_alu = v["modmul"] / pk
        t_hbm = v["bytes"] / (hbm_gbs * 1e9)
        per_class[k] = {
            "ms_per_step": v["ms"] / class_steps, "launches_per_step": v["launches"] / class_steps,
            "share": v["ms"] / max(sum(x["ms"] for x in classes.values()), 1e-9),
            "work_rate": v["modmul"] / secs / 1e9 if secs else 0.0, "work_unit": u, "work_peak": pk / 1e9,
            "alu_frac": t_alu / secs if secs else 0.0,
            "hbm_gbs": v["bytes"] / secs / 1e9 if secs else 0.0, "hbm_frac": t_hbm / secs if secs else 0.0,
            "bound": "hbm" if t_hbm > t_alu else "alu",
            "frac": max(t_alu, t_hbm) / secs if secs else 0.0,
            "algorithmic_bytes_per_step": v["bytes"] / class_steps,
            "traffic_over_algorithmic": TRAFFIC_RATIO.get(k)}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d, pc = classes[dom], per_class[dom]
    n_launch = max(d["launches"], 1)
    avg_s = d["ms"] / 1e3 / n_launch
    if pc["bound"] == "hbm":
        achieved, peak, unit = d["bytes"] / n_launch / avg_s / 1e9, hbm_gbs, "GB/s"
        peak_basis = f"HBM copy bandwidth, {hbm_src}"
    else:
        u, pk = unit_peak(dom)
        achieved, peak, unit = d["modmul"] / n_launch / avg_s / 1e9, pk / 1e9, u
        peak_basis = (f"{SM_COUNT} SMs x {MAX_SM_MHZ:.0f} MHz x "
                      f"{ub['split_mac' if dom in MAC_CLASSES else 'shoup_modmul']:.3f} units/clk/SM measured "
                      f"now (ctl_microbench_unit_rate)")
    ratio = TRAFFIC_RATIO.get(dom)
    roofline = {"bound": pc["bound"], "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "peak_basis": peak_basis,
                "traffic": ratio * d["bytes"] / n_launch if ratio else None,
                "traffic_basis": ("ncu dram bytes over algorithmic bytes of this class at batch 16, times the "
                                  "algorithmic bytes of an average launch" if ratio else None),
                "algorithmic_bytes_per_launch": d["bytes"] / n_launch,
                "hbm_peak_gbs": hbm_gbs, "hbm_frac": pc["hbm_frac"], "alu_frac": pc["alu_frac"],
                "avg_launch_ms": d["ms"] / n_launch, "classes": per_class,
                "unit_rates_per_clk_sm": ub,
                "imad_slot_peak": {"per_s": imad_slots,
                                   "slots_per_shoup_modmul": IMAD_PER_CLK_SM / ub["shoup_modmul"],
                                   "slots_per_split_mac": IMAD_PER_CLK_SM / ub["split_mac"]},
                "eager_ms_per_step": class_ms_per_step,
                "timing": timing_source}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        fwd_s, desc, cores, _ = cpu_oracle_sample(wl)
        cpu = {"value": fwd_s, "unit": "forwards/s", "cores": cores, "kind": "oracle", "sample": desc}

    # the other configurations, measured in the same run: single queries under the graph
    # (configurations 1 and 2, and the batched network one query at a time), one short
    # serving point (configuration 5), the client round trip and the uneven batch
    # (configuration 4)
    others = None
    if rank == 0 and world == 1 and args.workload == "batched" and not args.no_others:
        others = {name: single_query_point(ctl, torch, name, args.single_steps)
                  for name in ("single4096", "single8192", "batched")}
        others["batched"]["desc"] = "the batched network, one query per forward (batch 1)"
        if not args.no_cpu_baseline:  # the oracle on the host cores for configurations 1 and 2
            for name in ("single4096", "single8192"):
                fwd_s, desc, cores, _ = cpu_oracle_sample(WORKLOADS[name])
                others[name]["cpu_baseline"] = {"value": fwd_s, "unit": "forwards/s", "cores": cores,
                                                "kind": "oracle", "sample": desc}
        others["serving"] = serving_point(ctl, args.serve_rate, args.serve_seconds, args.serve_clients)
        others["client_round_trip"] = client_round_trip_point(ctl, torch, ctx, model, keys, slots, m_out, 3)
        un = run_uneven(argparse.Namespace(queries=1024, workers=4, max_batch=64, mem_budget_gb=160.0,
                                           dense_form=""), ctl)
        un.update({"unit": "forwards/s", "desc": "configuration 4: 1024 queries, N in {8192, 16384}, depth 2-6, "
                   "input 128-1024, each shape group a branch of one CUDA graph (ctl_multi_forward)"})
        others["uneven"] = un

    if rank == 0:
        lat = sorted(step_ms)
        line = {"metric": "encrypted forwards/sec (batched)", "value": value, "unit": "forwards/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": shared_config(wl, world),
                "run": {"cuda_graph": bool(use_graph), "ntt_shape": ntt_shape, "max_abs_err_vs_fp64": max_err},
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "per": f"batch of {B}"},
                "ops_per_step": {k: v / args.steps for k, v in ops.items()},
                "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": int(launches), "variants": variants, "other_workloads": others}
        if args.workload in PAPER_T_S:
            ts, pp = PAPER_T_S[args.workload], {"paper_p1": 2, "paper_p2": 5}[args.workload]
            line["predictions_per_ciphertext"] = windows
            line["predictions_per_s"] = value * windows
            line["paper_context"] = {
                "t_S_s": ts, "predictions_per_forward": pp, "predictions_per_s": pp / ts,
                "note": "Tab. 1: SEAL 4.0 + HEXL (AVX-512) on one i7-1165G7 thread; context only (other "
                        "hardware; the paper packs 768-wide windows, here windows of 2t = 2048 slots)"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
