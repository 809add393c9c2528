"""Seeded synthetic weights and FP64 plaintext references for the paper's frozen
server network (Sec. 4.1: Conv1D with filter size 9, Dense 768 with the approximated
ReLU, AveragePooling of size 3, Dense 766), scaled by the input length n.

The weights stand in for the trained server model, which is not available: the
filter ~N(0, 1/f), dense weights ~N(0, 1/fan_in).  Nothing here computes on
ciphertexts; both the oracle tests and the GPU tests take their weights and their
expected plaintext values from this module.
"""
import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def relu_coeffs():
    """(a0, a1, a2, a3) of the paper's degree-3 ReLU approximation (Sec. 3.1, "ReLU")."""
    with open(os.path.join(GOLD, "paper_params.json")) as f:
        a3, a2, a1, a0 = json.load(f)["relu_approx_coeffs_deg3_to_0"]
    return [a0, a1, a2, a3]


def poly3(a, z):
    return ((a[3] * z + a[2]) * z + a[1]) * z + a[0]


def conv_same(x, w):
    """out[j] = sum_i w[i] x[j + i - h], h = (f-1)//2, zero outside [0, n)."""
    n, f = len(x), len(w)
    h = (f - 1) // 2
    out = np.zeros(n)
    for j in range(n):
        for i in range(f):
            k = j + i - h
            if 0 <= k < n:
                out[j] += w[i] * x[k]
    return out


def avgpool_valid(r, f):
    """Stride-1 average pool of size f over the valid windows: length n - f + 1."""
    n = len(r)
    return np.array([np.mean(r[k:k + f]) for k in range(n - f + 1)])


def paper_net_weights(n, m2=None, f=9, pool=3, seed=1):
    """Weights of conv(f) -> dense n->n -> ReLU_approx -> avgpool(pool) -> dense (n-pool+1)->m2.
    Returns (w, W1, W2, W2s) where W2s is W2 with its columns moved right by pool-1, the
    form the slot algorithm applies (the valid pooled value k sits in slot k + pool - 1)."""
    rng = np.random.default_rng(seed)
    m2 = n - pool + 1 if m2 is None else m2
    w = rng.normal(0, 1 / np.sqrt(f), f)
    W1 = rng.normal(0, 1 / np.sqrt(n), (n, n))
    W2 = rng.normal(0, 1 / np.sqrt(n - pool + 1), (m2, n - pool + 1))
    W2s = np.zeros((m2, n))
    W2s[:, pool - 1:] = W2
    return w, W1, W2, W2s


def paper_net_fp64(x, w, W1, W2, a, pool=3):
    h = conv_same(x, w)
    z = W1 @ h
    r = poly3(a, z)
    p = avgpool_valid(r, pool)
    return W2 @ p


def replicated_slots(x, t, n_slots):
    """[x, x] at block stride t (Sec. 3.1, Multiple Predictions: 2 * #neurons slots)."""
    s = np.zeros(n_slots)
    s[:len(x)] = x
    s[t:t + len(x)] = x
    return s


def keyswitch_slot_sigma(N, digit_bits, p_bits, log_scale, var_e=10.5):
    """Standard deviation of one slot's decoded error after one hybrid key switch of a
    ciphertext at scale 2^log_scale.  The key product adds sum_d ModUp_d(c1) * e_d: each
    coefficient of ModUp_d is uniform below q_d (second moment q_d^2 / 3), each error
    coefficient has variance var_e (centred binomial k = 21: 21/2), and a negacyclic
    product sums N such terms, so a coefficient's variance is N var_e sum_d q_d^2 / 3 before
    ModDown divides it by P.  A slot is a sum of N coefficients times unit-modulus roots,
    so its real part has sqrt(N/2) times the coefficient's deviation; decoding divides by
    the scale.  (The ModDown rounding and the encryption noise are far smaller at the
    parameter sets used here.)"""
    P2 = float(2 ** (2 * sum(p_bits)))
    s = sum(float(2 ** (2 * b)) for b in digit_bits) / P2
    coef_sd = (N * var_e * s / 3.0) ** 0.5
    return coef_sd * (N / 2) ** 0.5 / 2.0 ** log_scale


def keyswitch_error_bound(N, digit_bits, p_bits, log_scale, n_ks, n_outputs, k=None):
    """Max-abs bound over n_outputs slots for an output that accumulates n_ks independent
    key-switch errors at the input scale (unit-norm weight rows carry each through): a
    Gaussian tail at k standard deviations, k = sqrt(2 ln(n_outputs)) + 2 by default."""
    import math

    if k is None:
        k = math.sqrt(2.0 * math.log(max(n_outputs, 2))) + 2.0
    return k * math.sqrt(n_ks) * keyswitch_slot_sigma(N, digit_bits, p_bits, log_scale)
