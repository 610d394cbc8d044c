"""The allocation-free field entry point (cts_field_noalloc), for callers
that cannot allocate device memory and hand in their own buffers, checked
against the FP64 oracle's field on the same FP32 positions.  Several calls
in a row: the fixed scratch array must be left ready for the next call; the
largest accepted input (131 072 carriers) fills every tile of that array."""
import numpy as np
import pytest

import oracle
import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5    # the field tolerance of the parity tests
EPS = 1e-6    # the Plummer length the entry point is given
MAX_N = 131_072


def _abs_sum(xyz, rows, eps=EPS):
    """k_C sum_j |term_ij| at the given rows: the conditioning of the field sum."""
    kc = oracle.coulomb_k()
    x = xyz.astype(np.float64)
    out = np.zeros(len(rows))
    for q, i in enumerate(rows):
        d = x[i] - x
        r2 = (d * d).sum(axis=1) + eps * eps
        t = np.sqrt(r2 - eps * eps) / r2 ** 1.5
        t[i] = 0.0
        out[q] = kc * t.sum()
    return out


def _oracle_field(xyz, nh, rows=None):
    sign = np.ones(xyz.shape[0], dtype=np.int8)
    sign[nh:] = -1
    return oracle.field(xyz.astype(np.float64), sign=sign, eps=EPS, rows=rows)


def _compare(got, ref, xyz, rows):
    S = _abs_sum(xyz, rows)
    err = np.linalg.norm(got - ref, axis=1)
    mag = np.linalg.norm(ref, axis=1)
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
    assert (err / np.maximum(mag, 1e-3 * S)).max() <= TOL


def _call(torch, xyz, nh, ne, softening=EPS):
    d = torch.from_numpy(np.ascontiguousarray(xyz.T)).cuda()   # caller-owned buffers
    out = torch.empty(3 * xyz.shape[0], dtype=torch.float32, device="cuda")
    rc = cts.cts_field_noalloc(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), nh, ne,
                               11.7, softening, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert rc == cts.SIM_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(3, -1).T.astype(np.float64)


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cts.load()
    oracle.build()
    return torch


def test_noalloc_field_matches_the_oracle_on_consecutive_calls():
    torch = _torch()
    rng = np.random.default_rng(21)
    h = rng.standard_normal((2000, 3)) * 2.0
    e = rng.standard_normal((1500, 3)) * 2.0 + np.array([0.3, 0.0, 2.0])
    small_h = rng.standard_normal((120, 3))
    small_e = rng.standard_normal((80, 3)) + np.array([0.5, 0.0, 0.0])
    cases = [(np.concatenate([h, e]).astype(np.float32), 2000, 1500),
             (W.random_cloud(5525, 0.83, seed=4).astype(np.float32), 5525, 0),
             (np.concatenate([small_h, small_e]).astype(np.float32), 120, 80)]
    cases.append(cases[0])  # the first input again, after a larger and a smaller call
    for xyz, nh, ne in cases:
        got = _call(torch, xyz, nh, ne)
        ref = _oracle_field(xyz, nh)
        _compare(got, ref, xyz, np.arange(xyz.shape[0]))


def test_noalloc_field_at_its_largest_input():
    # 131 072 carriers (every tile of the fixed array, the last one full),
    # twice in a row; sampled rows against the oracle, spread over the first,
    # a middle and the last tile and over both species
    torch = _torch()
    nh, ne = 100_000, MAX_N - 100_000
    xyz = np.concatenate([W.random_cloud(nh, 4.0, seed=8),
                          W.random_cloud(ne, 4.0, center=(1.0, 0.0, 3.0), seed=9)])
    xyz = xyz.astype(np.float32)
    rows = np.unique(np.concatenate([np.arange(0, 64), np.arange(65_500, 65_560),
                                     np.arange(nh - 32, nh + 32),
                                     np.arange(MAX_N - 64, MAX_N),
                                     np.random.default_rng(3).integers(0, MAX_N, 200)]))
    ref = _oracle_field(xyz, nh, rows=rows)
    for _ in range(2):
        got = _call(torch, xyz, nh, ne)
        _compare(got[rows], ref, xyz, rows)


def test_noalloc_rejects_inputs_beyond_its_fixed_scratch():
    _torch()
    assert cts.cts_field_noalloc(None, None, None, MAX_N, 1, 11.7, EPS, None) == \
        cts.SIM_ENOMEM_BUDGET
    assert cts.cts_field_noalloc(None, None, None, 0, 0, 11.7, EPS, None) == cts.SIM_OK
    for bad in (float("inf"), float("nan"), -1.0):
        assert cts.cts_field_noalloc(None, None, None, 10, 0, 11.7, bad, None) == cts.SIM_EINVAL
