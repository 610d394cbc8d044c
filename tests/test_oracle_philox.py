"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. SC'11)
and of its Box-Muller normals.

The bit pattern is checked against an independent library implementation
(Triton's `tl.philox`, run by Triton's CPU interpreter in a subprocess); the
normals are checked statistically.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def k(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor([[x - (1 << 32) if x >= (1 << 31) else x for x in row] for row in ctrs],
                     dtype=torch.int32)
    out = torch.zeros_like(c)
    k[(1,)](c, out, seed, c.shape[0])
    res.append([[v & 0xFFFFFFFF for v in row] for row in out.tolist()])
print(json.dumps(res))
"""


def test_philox_matches_triton_library(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    cases = []
    for seed in [0, 1, 0xFFFFFFFF, 20250611, 0x123456789ABCDEF0, (1 << 64) - 1]:
        ctrs = rng.integers(0, 1 << 32, size=(16, 4), dtype=np.uint64).tolist()
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        cases.append([int(seed), [[int(v) for v in row] for row in ctrs]])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), outs in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
        for ctr, want in zip(ctrs, outs):
            assert orc.philox4x32_10(ctr, key) == want, (seed, ctr)


def test_philox_words_are_uniform(orc):
    # 4 * 20000 words: chi-square of the top byte, and of the low byte.
    words = np.array([orc.philox4x32_10([i, 3, 5, 7], [11, 13]) for i in range(20000)],
                     dtype=np.uint64).reshape(-1)
    for shift in (24, 0):
        h = np.bincount(((words >> shift) & 0xFF).astype(np.int64), minlength=256)
        chi2, p = stats.chisquare(h)
        assert p > 1e-4, (shift, p)


def test_normals_moments_and_ks(orc):
    n = np.array([orc.normals3(20250611, 5, 0, c, s) for c in range(4000) for s in range(5)])
    for axis in range(3):
        v = n[:, axis]
        assert abs(v.mean()) < 5 * (1 / np.sqrt(v.size))
        assert abs(v.var() - 1.0) < 5 * np.sqrt(2.0 / v.size)
        assert abs(stats.kurtosis(v)) < 5 * np.sqrt(24.0 / v.size)
        assert stats.kstest(v, "norm").pvalue > 1e-4
    # the three components are uncorrelated
    c = np.corrcoef(n.T)
    assert np.all(np.abs(c - np.eye(3)) < 5 / np.sqrt(n.shape[0]))


def test_streams_are_distinct_per_purpose_event_carrier_step(orc):
    base = orc.normals3(1, 2, 0, 3, 4)
    assert orc.normals3(1, 2, 1, 3, 4) != base   # purpose
    assert orc.normals3(1, 9, 0, 3, 4) != base   # event
    assert orc.normals3(1, 2, 0, 8, 4) != base   # carrier
    assert orc.normals3(1, 2, 0, 3, 5) != base   # step
    assert orc.normals3(2, 2, 0, 3, 4) != base   # seed
    assert orc.normals3(1, 2, 0, 3, 4) == base   # deterministic


def test_uniform_mapping_is_symmetric_open_and_fp32_exact(orc):
    # u(w) = ((w >> 9) + 1/2) 2^-23: the complement word maps to 1 - u exactly,
    # both ends stay inside (0, 1), and every value is an odd multiple of
    # 2^-24, so FP32 and FP64 hold it exactly (the device draws the same u)
    rng = np.random.default_rng(3)
    words = list(rng.integers(0, 1 << 32, 2000, dtype=np.uint64)) + [0, 1, 511, 512,
                                                                      0xFFFFFFFF, 0x80000000]
    for w in words:
        w = int(w)
        u, v = orc.uniform(w), orc.uniform(w ^ 0xFFFFFFFF)
        assert 0.0 < u < 1.0
        assert u + v == 1.0
        k = u * (1 << 24)
        assert k == int(k) and int(k) % 2 == 1
        assert float(np.float32(u)) == u
    assert orc.uniform(0) == 2.0 ** -24 and orc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # 512 consecutive words share one value (the low 9 bits are dropped)
    assert orc.uniform(512 * 77) == orc.uniform(512 * 77 + 511) != orc.uniform(512 * 78)


def test_stream_layout_keeps_large_event_ids_and_purposes_apart(orc):
    # event ids use both counter words; the purpose sits above bit 28 of the
    # high word, so events below 2^60 never share a stream with another
    # purpose of another event
    for hi_bits in (24, 26, 27):
        ev = 1 << (32 + hi_bits)
        for purpose in (1, 2, 3, 4):
            assert orc.normals3(7, ev, 0, 5, 6) != orc.normals3(7, 0, purpose, 5, 6)
            assert orc.normals3(7, ev * purpose, 0, 5, 6) != orc.normals3(7, 0, purpose, 5, 6)
    assert orc.normals3(7, (1 << 60) - 1, 0, 5, 6) != orc.normals3(7, (1 << 60) - 1, 1, 5, 6)
