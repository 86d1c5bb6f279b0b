"""Pins for the oracle's random-number and Q16 contract (no GPU).

* Philox4x32-10 is checked against PyTorch's ATen ``philox_engine`` header, an
  independent implementation of the same published generator (Salmon et al.,
  SC'11), compiled here from its readable source.
* The walk draw's key/counter layout is checked through the same engine.
* Q16 alpha values are checked against exact values of 65536/p and the
  rejection rules.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch_include():
    try:
        import torch
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) else None


@pytest.fixture(scope="module")
def aten_kat(tmp_path_factory):
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("ATen PhiloxRNGEngine.h or g++ not available")
    exe = str(tmp_path_factory.mktemp("kat") / "kat")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, os.path.join(HERE, "aten_philox_kat.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("ATen Philox header did not compile: " + r.stderr[-400:])

    def run(rows):
        inp = "\n".join(" ".join(str(int(x)) for x in row) for row in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return [tuple(int(x) for x in line.split()) for line in out.strip().splitlines()]

    return run


def test_philox_matches_aten(aten_kat):
    rng = np.random.default_rng(12345)
    rows = [(0, 0, 0, 0, 0, 0), (1, 0, 0, 0, 0, 0), (0, 0, 0, 0, 1, 0), (0xFFFFFFFF,) * 6]
    rows += [tuple(int(x) for x in rng.integers(0, 2**32, size=6, dtype=np.uint64)) for _ in range(300)]
    want = aten_kat(rows)
    for row, w in zip(rows, want):
        got = oracle.philox4x32_10(row[:4], row[4:])
        assert tuple(int(x) for x in got) == w, row


def test_draw_layout_matches_aten(aten_kat):
    """u = out[1]<<32 | out[0] with counter (k, lo(w), hi(w), 0) and key (lo(seed), hi(seed))."""
    rng = np.random.default_rng(7)
    cases = [(1, 0, 0), (1, 5, 79), (2**40 + 3, 2**33 + 17, 3)]
    cases += [(int(rng.integers(0, 2**63)), int(rng.integers(0, 2**40)), int(rng.integers(0, 80)))
              for _ in range(100)]
    rows = [(k, w & 0xFFFFFFFF, w >> 32, 0, s & 0xFFFFFFFF, s >> 32) for s, w, k in cases]
    want = aten_kat(rows)
    for (s, w, k), o in zip(cases, want):
        assert oracle.draw(s, w, k) == (o[1] << 32) | o[0]


def test_philox_distinct_streams():
    # different walk ids / steps give different draws (no accidental key reuse)
    draws = {oracle.draw(1, w, k) for w in range(200) for k in range(20)}
    assert len(draws) == 200 * 20


@pytest.mark.parametrize(
    "p,expect",
    [(1.0, 65536), (0.5, 131072), (2.0, 32768), (0.25, 262144), (4.0, 16384), (3.0, 21845),
     (0.3, 218453), (1 / 3, 196608), (0.7, 93623), (65536.0, 1), (2.0**-8, 2**24)],
)
def test_alpha_q16_values(p, expect):
    # 65536/p rounded to nearest: exact rational values checked by hand
    a_p, a_q = oracle.alpha_q16(p, p)
    assert a_p == expect and a_q == expect


def test_alpha_q16_matches_rounded_quotient():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        p = float(np.exp(rng.uniform(np.log(0.01), np.log(100.0))))
        q = float(np.exp(rng.uniform(np.log(0.01), np.log(100.0))))
        a_p, a_q = oracle.alpha_q16(p, q)
        # Python's round() is round-half-even on the same IEEE double quotient
        assert a_p == round(65536.0 / p) and a_q == round(65536.0 / q)


@pytest.mark.parametrize("p,q", [(0.0, 1.0), (1.0, -1.0), (float("nan"), 1.0), (1.0, float("inf")),
                                 (131072.0 * 2, 1.0), (1.0, 2.0**-9)])
def test_alpha_q16_rejects(p, q):
    with pytest.raises(ValueError):
        oracle.alpha_q16(p, q)
