"""The library's host rule from d_lambda to (l, s, lambda0) against the
oracle's statement of Section 3 / Lemma 2.1 (no GPU work: the rule is host
code in the C-ABI library)."""

import numpy as np
import pytest

pytest.importorskip("torch")

from oracle import effdim


@pytest.fixture(scope="module")
def rule():
    try:
        from paper_2405_05865_gb300.api import params_from_effdim
    except ImportError as e:
        pytest.skip(f"library not built: {e}")
    return params_from_effdim


@pytest.mark.parametrize("d,n,lam", [(0.0, 16, 1.0), (0.3, 64, 1e-2), (7.5, 100, 1e-3), (181.49, 1024, 1e-3),
                                     (323.0, 2048, 1e-2), (511.9999, 4096, 1e-2), (512.0, 4096, 1e-2),
                                     (2029.2, 16384, 1e-2), (600.0, 2000, 1e-2), (3000.0, 8192, 5e-1),
                                     (300.0, 1000, 1e-2), (600.0, 1000, 1e-2), (1500.0, 1000, 1e-2)])
def test_rule_matches_oracle(rule, d, n, lam):
    got = rule(d, n, lam)
    want = effdim.params_from_effdim(d, n, lam)
    for key in ("l", "s", "capped", "direct"):
        assert got[key] == want[key], key
    assert got["lambda0"] == want["lambda0"]
    assert got["d_lambda"] == d and got["d_std_err"] == 0.0


def test_rule_rejects_bad_arguments(rule):
    from paper_2405_05865_gb300 import MspError
    for args in ((-1.0, 64, 1e-2), (float("nan"), 64, 1e-2), (1.0, 8, 1e-2), (1.0, 64, 0.0)):
        with pytest.raises(MspError):
            rule(*args)
