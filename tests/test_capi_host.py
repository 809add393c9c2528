"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol that
include/ctl.h declares, and its host-only prime planner agrees with the oracle."""
import os
import re

import pytest

from oracle import ckks_oracle as O
from paper_2205_11935_gb300 import ctl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ctl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(ctl_[a-z0-9_]+)\s*\(", src))
    names -= {"ctl_alloc_fn", "ctl_free_fn"}
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = ctl.lib()
    names = declared_functions()
    assert len(names) > 40
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding covers the same set
    assert set(names) <= set(ctl.SIGNATURES), sorted(set(names) - set(ctl.SIGNATURES))


def test_version_and_error_string():
    L = ctl.lib()
    assert b"sm_103a" in L.ctl_version()
    with pytest.raises(ctl.CtlError) as e:
        ctl.plan_primes(100, [40])  # N not a power of two
    assert e.value.code == -1


@pytest.mark.parametrize("N,bits", [(64, [50, 40, 40, 60]), (4096, [50, 40, 40, 60]), (8192, [60, 40, 40, 40, 60]),
                                    (16384, [45] * 8 + [60, 60]), (8192, [34] + [25] * 6 + [34])])
def test_prime_planner_matches_oracle(N, bits):
    assert ctl.plan_primes(N, bits) == O.primes(N, bits)


def test_prime_planner_rejects_out_of_range_bits():
    with pytest.raises(ctl.CtlError):
        ctl.plan_primes(4096, [62])
    with pytest.raises(ctl.CtlError):
        ctl.plan_primes(4096, [19])
