"""CPU checks of the numbers bench.py derives without a GPU: the algorithmic work per
Montgomery product and per exponentiation (the roofline numerator), tied to the half
products the oracle's method models count, and the rule that a recorded DRAM-traffic
figure is reported only for the sources it was captured on."""
import importlib.util
import json
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _alg6_high_half(n):
    N = si.random_odd_moduli(si.stream(0, "test", "other", 900 + n), 1, 32 * n)
    Np, _, _ = oracle.ctx(N)
    T = np.zeros(2 * n, np.uint32)
    T[0] = 3
    return oracle.montred_alg6(T, N[0], Np[0])["pp"]


@pytest.mark.parametrize("n", [1, 2, 5, 32, 64, 128])
def test_imad_counts_match_the_oracles_half_products(bench, n):
    """One 32-bit multiply-add per half product (lo or hi). Truncated: T (2n^2 for a product,
    n^2 + n for a square: doubled cross products plus the diagonal), q (the low half, n^2) and
    the high half of qN as counted by the Alg. 6 model. Classical: the whole q*N (2n^2)."""
    c = bench.imad_counts(n)
    high = _alg6_high_half(n)
    assert c["mul_trunc"] == 2 * n * n + n * n + high
    assert c["sqr_trunc"] == (n * n + n) + n * n + high
    assert c["mul_full"] == 2 * n * n + n * n + 2 * n * n
    assert c["sqr_full"] == (n * n + n) + n * n + 2 * n * n


def test_headline_work_per_exponentiation(bench):
    """2048 bits, w = 5, 2048-bit exponents: 410 windows of 5 squarings and a product, the
    31 products of the table (to-Montgomery included) and the product with 1."""
    c = bench.imad_counts(64)
    assert bench.modexp_imad(2048, 2048, 5) == 2050 * c["sqr_trunc"] + 442 * c["mul_trunc"] == 32_879_812
    assert bench.modexp_imad(2048, 2048, 5, "full") == 2050 * c["sqr_full"] + 442 * c["mul_full"]


def test_traffic_record_only_for_its_sources(bench, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["k_modexp_2048_w5"]
    monkeypatch.setattr(bench, "sources_digest", lambda: rec["sources_digest"])
    got = bench.recorded_traffic("k_modexp_2048_w5", rec["instances"] // 2)
    assert got == pytest.approx(rec["dram_bytes_per_launch"] / 2)
    monkeypatch.setattr(bench, "sources_digest", lambda: "0" * 16)
    assert bench.recorded_traffic("k_modexp_2048_w5", rec["instances"]) is None
    assert bench.recorded_traffic("no_such_kernel", 1) is None


def test_sources_digest_covers_the_kernel_sources(bench, tmp_path, monkeypatch):
    """The digest is that of the CUDA sources and headers: a copy digests the same, and changing
    one header of the copy (a comment is enough) changes it, so a stale traffic figure drops out."""
    import shutil
    shutil.copytree(os.path.join(ROOT, "paper_2410_18129_gb300", "csrc"), tmp_path / "paper_2410_18129_gb300" / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), tmp_path / "include")
    d0 = bench.sources_digest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.sources_digest() == d0
    with open(tmp_path / "paper_2410_18129_gb300" / "csrc" / "mp_group.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.sources_digest() != d0
