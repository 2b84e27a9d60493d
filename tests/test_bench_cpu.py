"""bench.py's host-side contract, checked without a GPU: the defaults (one
GPU, at least three warm-up steps), the whole-job rate and the FLOP counts
the TFLOP/s figure uses (2 n^3 / 3 for the factorization plus the product
with the multiplier)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _args(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_defaults_follow_the_contract():
    a = _args()
    assert a.gpus == 1 and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 1
    assert a.n == 16384 and a.prec == "sliced" and a.kind == "gaussian"


@pytest.mark.parametrize("kind,ag", [("gaussian", lambda n: 2.0 * n ** 3), ("sparse", lambda n: 8.0 * n * n)])
def test_flop_counts(kind, ag):
    a = _args("--kind", kind, "--n", "1024")
    fact, got = bench.flops_per_solve(a)
    assert fact == pytest.approx(2.0 * 1024 ** 3 / 3.0)
    assert got == pytest.approx(ag(1024))


def test_job_rate_counts_every_rank():
    assert bench.job_rate(4, 8, 2000.0) == pytest.approx(16.0)
    assert bench.reduce_max(3.0, 1, "cpu") == 3.0
