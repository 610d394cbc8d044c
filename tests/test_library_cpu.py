"""CPU-side checks of the C-ABI library: it loads without a GPU, exports every
symbol the public headers declare, validates parameters before touching a
device, and its host scheduling logic (unit planner, arena allocator, drift
time estimate) is correct.  No kernel is launched here."""
import glob
import math
import os
import re

import numpy as np
import pytest

import paper_2506_09712_gb300 as cts
from paper_2506_09712_gb300 import build as cts_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cts_build.build()
    return cts.load()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|double|const\s+char\s*\*)\s+(\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert {"sim_init", "sim_submit", "sim_poll", "sim_destroy", "cts_plan_units"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(cts.EXPORTED)


def test_checked_build_loads_and_reports_itself(lib):
    # the bounds-checked build (-DCTS_BOUNDS_CHECK) exports the same ABI and
    # says which build it is; the default build compiles no checks
    import ctypes as C
    path = cts_build.build(checked=True)
    assert path.endswith("libcts_checked.so") and os.path.exists(path)
    checked = C.CDLL(path)
    for name in _declared_symbols():
        assert hasattr(checked, name), name
    assert checked.sim_build_flags() == cts.SIM_BUILD_BOUNDS_CHECK
    assert lib.sim_build_flags() == 0


def test_strerror_names_every_code(lib):
    for code in range(-9, 1):
        assert cts.strerror(code) != "unknown status"
    assert cts.strerror(-99) == "unknown status"


def _good():
    s = cts.make_sensor(dict(thickness_um=320.0, bias_V=150.0, depletion_V=60.0, dt_ps=10.0))
    f = cts.make_field()
    m = cts.make_mobility(dict(mu0_h=480.0, vsat_h=0.95e7, beta_h=1.2))
    return s, f, m


@pytest.mark.parametrize("field,value", [
    ("thickness_um", 0.0), ("dt_ps", -1.0), ("temperature_K", 0.0), ("grid_n", 0),
    ("species", 2), ("max_steps", 0), ("bias_V", 10.0), ("pitch_um", float("nan")),
])
def test_init_rejects_bad_sensor(lib, field, value):
    s, f, m = _good()
    setattr(s, field, value)
    rc, h = cts.sim_init(s, f, m, None)
    assert rc == cts.SIM_EINVAL and not h.value


def test_init_rejects_bad_mobility(lib):
    s, f, m = _good()
    m.beta_h = 0.0
    assert cts.sim_init(s, f, m, None)[0] == cts.SIM_EINVAL
    s, f, m = _good()
    s.species = cts.CTS_BOTH          # electrons need their own parameters
    assert cts.sim_init(s, f, m, None)[0] == cts.SIM_EINVAL


def test_init_without_device_reports_enodev(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s, f, m = _good()
    rc, h = cts.sim_init(s, f, m, None)
    assert rc == cts.SIM_ENODEV and not h.value


def test_kernel_hooks_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cts.SimError) as e:
        cts.sim_debug_philox([[0, 0, 0, 0]], [[0, 0]])
    assert e.value.code == cts.SIM_ENODEV
    with pytest.raises(cts.SimError) as e:
        cts.sim_debug_fma_peak(0)
    assert e.value.code == cts.SIM_ENODEV


def _check_cover(units, n_h, n_e):
    """Every ordered pair (i, j) of a slot is covered exactly once: per slot and
    species the i-tiles partition the carriers, and per i-tile the j ranges
    partition the slot's concatenated source list."""
    tiles = {}
    for (slot, spec, i0, ni, j0, j1, split, nsplit, iblock, pbase) in units:
        tiles.setdefault((slot, spec, i0, ni), []).append((j0, j1))
    per_species = {}
    for (slot, spec, i0, ni), js in tiles.items():
        js.sort()
        n = n_h[slot] + n_e[slot]
        assert js[0][0] == 0 and js[-1][1] == n, (slot, js)
        for (a0, a1), (b0, b1) in zip(js, js[1:]):
            assert a1 == b0 and a0 < a1
        per_species.setdefault((slot, spec), []).append((i0, i0 + ni))
    for slot in range(len(n_h)):
        if n_h[slot] <= 0:
            continue
        for spec, cnt in ((0, n_h[slot]), (1, n_e[slot])):
            iv = sorted(per_species.get((slot, spec), []))
            if cnt == 0:
                assert not iv
                continue
            assert iv[0][0] == 0 and iv[-1][1] == cnt
            for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
                assert a1 == b0
    return True


@pytest.mark.parametrize("n_h,n_e,tile,grid", [
    ([5525] * 64, [0] * 64, 512, 912),
    ([5525] * 16, [0] * 16, 512, 912),
    ([5525], [0], 512, 456),
    ([829, 0, 1381, 6906, 3], [0, 0, 0, 0, 0], 512, 456),
    ([3000, 17], [3000, 5], 256, 300),
    ([55250] * 2, [55250] * 2, 512, 912),
    ([1], [0], 512, 456),
])
def test_planner_covers_every_pair_once_and_balances(lib, n_h, n_e, tile, grid):
    rc, units, begin, pfl = cts.cts_plan_units(n_h, n_e, tile, grid)
    assert rc == 0
    assert _check_cover(units, n_h, n_e)
    assert all(n_h[u[0]] > 0 for u in units)          # idle slots get no units
    # CTA ranges: monotone, cover all units
    assert begin[0] == 0 and begin[-1] == len(units) and np.all(np.diff(begin) >= 0)
    # j boundaries of split segments are multiples of 4 (16-byte aligned copies)
    n_of = {s: n_h[s] + n_e[s] for s in range(len(n_h))}
    for u in units:
        assert u[4] % 4 == 0 and (u[5] % 4 == 0 or u[5] == n_of[u[0]])
    # equal shares: every working CTA gets the same pair count within 4 tiles' j step
    cost = units[:, 3] * (units[:, 5] - units[:, 4])
    per_cta = np.array([cost[begin[g]:begin[g + 1]].sum() for g in range(grid)])
    busy = per_cta[per_cta > 0]
    total = sum((n_h[s] + n_e[s]) ** 2 for s in range(len(n_h)) if n_h[s] > 0)
    assert per_cta.sum() == total
    if len(busy) > 1:
        assert busy.max() - busy.min() <= 2 * 4 * tile + 1, (busy.min(), busy.max())
    # split tiles: consistent metadata, disjoint partial regions inside pfl
    blocks = {}
    for u in units:
        if u[7] > 1:
            blocks.setdefault(u[8], []).append(u)
    ends = []
    for b, us in blocks.items():
        assert sorted(x[6] for x in us) == list(range(us[0][7]))
        assert len({(x[0], x[1], x[2], x[9]) for x in us}) == 1
        ends.append((us[0][9], us[0][9] + 3 * tile))
    ends.sort()
    for (a0, a1), (b0, b1) in zip(ends, ends[1:]):
        assert a1 <= b0
    if ends:
        assert ends[-1][1] <= pfl


def test_planner_small_work_uses_fewer_ctas(lib):
    # 829^2 pairs: shares of >= 65536 pairs -> at most 10 CTAs get work
    rc, units, begin, _ = cts.cts_plan_units([829], [0], 512, 456)
    busy = np.count_nonzero(np.diff(begin))
    assert rc == 0 and 1 <= busy <= 10
    # no splitting allowed: whole tiles, dealt longest first
    rc, units, begin, pfl = cts.cts_plan_units([5525], [0], 512, 456, allow_split=0)
    assert rc == 0 and pfl == 0 and units.shape[0] == 11 and np.all(units[:, 7] == 1)


def test_planner_respects_budgets(lib):
    # every piece of a split tile takes 3 * tile_i partial sums: a budget of
    # 40 such regions splits a few of the 44 tiles and runs the rest whole
    cap = 3 * 512 * 40
    rc, units, begin, pfl = cts.cts_plan_units([5525] * 4, [0] * 4, 512, 456, partial_cap=cap)
    split_tiles = {tuple(u[:3]) for u in units if u[7] > 1}
    assert rc == 0 and pfl <= cap and 0 < len(split_tiles) < 44
    assert _check_cover(units, [5525] * 4, [0] * 4)
    # a budget smaller than two regions splits nothing
    rc, units, begin, pfl = cts.cts_plan_units([5525] * 4, [0] * 4, 512, 456,
                                               partial_cap=3 * 512)
    assert rc == 0 and pfl == 0 and np.all(units[:, 7] == 1)
    assert _check_cover(units, [5525] * 4, [0] * 4)
    rc, _, _, _ = cts.cts_plan_units([5525] * 64, [0] * 64, 512, 456, max_units=100)
    assert rc == -2


def test_arena_first_fit_and_coalescing(lib):
    # allocate 3 blocks, free the middle, reuse it; free all, whole capacity again
    ops = [100, 200, 300, -2, 150, -1, -3, -5, 1000]
    rc, res = cts.cts_arena_replay(1024, ops)
    assert rc == 0
    a, b, c = res[0], res[1], res[2]
    assert (a, b, c) == (0, 128, 352)            # rounded to multiples of 32
    assert res[4] == 128                         # the freed middle block is reused
    assert res[8] == 0                           # everything coalesced
    rc, res = cts.cts_arena_replay(256, [200, 100])
    assert res[1] == -1                          # no room


def test_estimate_steps_matches_eq9(lib):
    # beta = 1: Eq. 9 closed form, t = (1/(mu0 k)) ln(E(0)/E(z0)) + z0 / vsat.
    H, Vb, Vd, mu0, vsat = 320.0, 150.0, 60.0, 480.0, 0.95e7
    for depth in (10.0, 120.0, 300.0):
        z0 = H - depth
        E = lambda z: (Vb - Vd) / H + 2 * Vd * (H - z) / H ** 2
        t = 1 / (mu0 * 0.1 * 2 * Vd / H ** 2) * math.log(E(0) / E(z0)) + z0 / (vsat * 1e-5)
        est = cts.cts_estimate_steps(H, Vb, Vd, mu0, vsat, 1.0, 10.0, depth)
        assert est == pytest.approx(t / 0.01, rel=1e-4)


@pytest.mark.parametrize("n_h,n_e", [([5525] * 64, [0] * 64), ([5525] * 3, [0] * 3),
                                     ([3000, 900], [2000, 10]), ([829], [0])])
def test_guided_dynamic_plan(lib, n_h, n_e):
    # allow_split = 2: one queue of pieces, largest first, shrinking at the end
    rc, units, begin, pfl = cts.cts_plan_units(n_h, n_e, 512, 608, allow_split=2)
    assert rc == 0
    assert _check_cover(units, n_h, n_e)
    assert begin[-1] == len(units) and np.all(begin[:-1] == 0)
    cost = units[:, 3] * (units[:, 5] - units[:, 4])
    assert np.all(np.diff(cost) <= 0)
    # the smallest pieces are much smaller than the largest when there is enough work
    if cost.sum() > 608 * 512 * 4096:
        assert cost[-1] * 8 <= cost[0]


@pytest.mark.parametrize("n_h,n_e", [([5525] * 64, [0] * 64), ([5525] * 3, [0] * 3),
                                     ([3000, 0, 900], [2000, 0, 10]), ([829], [0])])
def test_slot_major_plan_for_multi_step_launches(lib, n_h, n_e):
    # allow_split = 3: the same pieces, slot by slot, shrinking within each slot,
    # so that a queue replayed over several steps finishes a slot's step well
    # before the slot's next step comes up
    rc, units, begin, pfl = cts.cts_plan_units(n_h, n_e, 512, 608, allow_split=3)
    assert rc == 0
    assert _check_cover(units, n_h, n_e)
    assert begin[-1] == len(units) and np.all(begin[:-1] == 0)
    slots = units[:, 0]
    assert np.all(np.diff(slots) >= 0)                # slot-major
    cost = units[:, 3] * (units[:, 5] - units[:, 4])
    for s in np.unique(slots):
        c = cost[slots == s]
        assert np.all(np.diff(c) <= 0)                # largest first within the slot
    # one slot: the same pieces as the single-step guided queue
    if len(n_h) == 1:
        rc2, units2, _, _ = cts.cts_plan_units(n_h, n_e, 512, 608, allow_split=2)
        assert np.array_equal(units, units2)


def test_fano_pairs_match_the_oracle():
    # the library's host draw and the oracle's are separate implementations of
    # the same counter-based stream and normal approximation
    import oracle
    for e in (3.0, 8.0, 17.5, 25.0):
        for k in range(0, 3000, 7):
            assert cts.cts_fano_pairs(20250611, k, e, 0.13) == oracle.fano_pairs(20250611, k, e, 0.13)
        assert cts.cts_fano_pairs(1, 2, e, 0.0) == oracle.n_pairs(e)
    with pytest.raises(ValueError):
        cts.cts_fano_pairs(1, 2, -1.0, 0.13)


def test_readout_rejects_bad_arguments_before_the_device(lib):
    import numpy as np
    with pytest.raises(cts.SimError) as e:
        cts.sim_readout(np.zeros((1, 33, 33), np.int32), [1], [0], 20.0)
    assert e.value.code == cts.SIM_EINVAL
    with pytest.raises(cts.SimError) as e:
        cts.sim_readout(np.zeros((1, 9, 9), np.int32), [1], [0], 20.0, n_bins=10, spec_bin_keV=0.0)
    assert e.value.code == cts.SIM_EINVAL


def test_spherical_model_needs_holes_only(lib):
    import workloads as W
    p = W.preset("track_200keV_320um")
    with pytest.raises(cts.SimError) as e:
        cts.Simulator(p["sensor"], p["mobility"], field=W.field_switches(spherical=1))
    assert e.value.code == cts.SIM_EINVAL
    p = W.preset("batch_20keV_320um")
    with pytest.raises(cts.SimError) as e:
        cts.Simulator(p["sensor"], p["mobility"], field=dict(W.field_switches(), spherical=2))
    assert e.value.code == cts.SIM_EINVAL


def test_ggd_fits_match_the_oracle():
    import numpy as np
    import oracle
    x = oracle.ggd_samples(9, 2, 30000, 4.1, 2.6)
    a, b = cts.cts_fit_ggd(x)
    oa, ob = oracle.fit_ggd(x)
    assert a == pytest.approx(oa, rel=1e-8) and b == pytest.approx(ob, rel=1e-8)
    with pytest.raises(ValueError):
        cts.cts_fit_ggd(np.zeros(5))
    # Eq. 10: weighted linear least squares
    rng = np.random.default_rng(4)
    t = np.linspace(0.1, 15.0, 40)
    pa = [1.0, 1.8, 0.2, -0.004]
    y = oracle.alpha_of_t(pa, t) + 0.01 * rng.standard_normal(t.size)
    w = rng.uniform(0.5, 2.0, t.size)
    assert np.allclose(cts.cts_fit_alpha_t(t, y, w), oracle.fit_alpha_of_t(t, y, w), atol=1e-9)
    # Eq. 11: noise-free data give back the parameters; on noisy data the
    # library's Levenberg-Marquardt and scipy's solver agree
    pb = [0.35, 1.5, 0.6, 1.1, -0.7]
    start = [0.3, 1.3, 0.5, 0.9, -0.5]
    assert np.allclose(cts.cts_fit_beta_t(t, oracle.beta_of_t(pb, t), start), pb,
                       rtol=1e-5, atol=1e-7)
    yb = oracle.beta_of_t(pb, t) + 0.005 * rng.standard_normal(t.size)
    q = cts.cts_fit_beta_t(t, yb, start)
    qo = oracle.fit_beta_of_t(t, yb, start)
    cost = lambda p: ((yb - oracle.beta_of_t(p, t)) ** 2).sum()
    assert cost(q) == pytest.approx(cost(qo), rel=1e-4)
    # with per-point sigma both minimise the weighted cost, and the weighted
    # optimum differs from the unweighted one
    sg = np.where(t < 6.0, 0.002, 0.02)
    ys = oracle.beta_of_t(pb, t) + sg * rng.standard_normal(t.size)
    qs = cts.cts_fit_beta_t(t, ys, start, sg)
    qso = oracle.fit_beta_of_t(t, ys, start, sg)
    wcost = lambda p: (((ys - oracle.beta_of_t(p, t)) / sg) ** 2).sum()
    assert wcost(qs) == pytest.approx(wcost(qso), rel=1e-4)
    q_unw = cts.cts_fit_beta_t(t, ys, start)
    assert wcost(qs) < wcost(q_unw) * (1 - 1e-3)
    # from the unweighted optimum every step toward the weighted one raises
    # the unweighted cost: only a fit that accepts steps by the weighted cost
    # gets there
    q2 = cts.cts_fit_beta_t(t, ys, q_unw, sg)
    assert wcost(q2) == pytest.approx(wcost(qso), rel=1e-4)
    for tt in (0.5, 3.0, 12.0):
        a1, b1 = cts.cts_ggd_params_at(pa, pb, tt)
        assert a1 == pytest.approx(float(oracle.alpha_of_t(pa, tt)), rel=1e-14)
        assert b1 == pytest.approx(float(oracle.beta_of_t(pb, tt)), rel=1e-14)


def test_generate_checks_arguments_before_the_device(lib):
    ev = dict(seed=1, event_id=0, n_pairs=10, x_um=0.0, y_um=0.0, alpha=2.0, beta=2.5)
    with pytest.raises(cts.SimError) as e:
        cts.sim_generate([dict(ev, beta=50.0)], 25.0, 9)
    assert e.value.code == cts.SIM_EINVAL
    with pytest.raises(cts.SimError) as e:
        cts.sim_generate([ev], 25.0, 40)
    assert e.value.code == cts.SIM_EINVAL
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(cts.SimError) as e:
            cts.sim_generate([ev], 25.0, 9)
        assert e.value.code == cts.SIM_ENODEV


@pytest.mark.parametrize("table", [[1.0], [1.0, -0.5], [1.0, float("nan")], [0.0, 1.0]])
def test_bad_drift_tables_are_rejected(lib, table):
    import workloads as W
    p = W.preset("plain_3keV_100um")
    with pytest.raises(cts.SimError) as e:
        cts.Simulator(dict(p["sensor"], drift_table_Vum=table), p["mobility"])
    assert e.value.code == cts.SIM_EINVAL


@pytest.mark.parametrize("flags,grid_n", [(-1, 9), (4, 9), (7, 9),
                                          (cts.SIM_INDUCED_PIXELS, 2),
                                          (cts.SIM_INDUCED_TOTAL | cts.SIM_INDUCED_PIXELS, 1)])
def test_induced_recording_flags_are_checked_before_the_device(lib, flags, grid_n):
    # unknown flags, and a 3 x 3 pixel window that does not fit the grid
    import workloads as W
    p = W.preset("plain_3keV_100um")
    with pytest.raises(cts.SimError) as e:
        cts.Simulator(dict(p["sensor"], grid_n=grid_n), p["mobility"], keep_induced=flags)
    assert e.value.code == cts.SIM_EINVAL


def test_pixel_signal_buffers_follow_the_option(lib):
    # the result arrays the binding hands to the library: 9 per step
    r = cts.Results(2, 5, 0, 7, induced_px=True)
    assert r.induced_px.shape == (2, 7, 3, 3)
    assert bool(r.arr[1].induced_px) and r.arr[1].induced_capacity == 7
    r = cts.Results(2, 5, 0, 7)
    assert r.induced_px is None and not r.arr[0].induced_px


def test_host_model_entry_points_reject_bad_input(lib):
    import ctypes as C
    import numpy as np
    L = cts.load()
    d = C.POINTER(C.c_double)
    one = np.ones(3)
    # too few points, null outputs
    assert L.cts_fit_ggd(one.ctypes.data_as(d), 1, None, None) == -1
    assert L.cts_fit_alpha_t(one.ctypes.data_as(d), one.ctypes.data_as(d), None, 3,
                             np.zeros(4).ctypes.data_as(d)) == -1
    assert L.cts_fit_beta_t(one.ctypes.data_as(d), one.ctypes.data_as(d), None, 3,
                            np.zeros(5).ctypes.data_as(d)) == -1
    # parameters that make alpha non-positive, and a negative drift time
    with pytest.raises(ValueError):
        cts.cts_ggd_params_at([-1.0, 0, 0, 0], [0, 0, 1, 0, 0], 1.0)
    with pytest.raises(ValueError):
        cts.cts_ggd_params_at([1.0, 0, 0, 0], [0, 0, 1, 0, 0], -1.0)
    # the launch log needs a handle
    n = C.c_int32(0)
    assert L.sim_debug_launch_log(None, None, 0, C.byref(n)) == cts.SIM_EINVAL
    assert L.sim_debug_fma_peak(-1, 1, None) == cts.SIM_EINVAL


def test_public_struct_layouts_match_the_binding(tmp_path):
    # the ctypes mirrors of include/cts.h must agree field by field
    import ctypes as C
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"sim_sensor_t": cts.sim_sensor_t, "sim_field_t": cts.sim_field_t,
               "sim_mobility_t": cts.sim_mobility_t, "sim_options_t": cts.sim_options_t,
               "sim_event_t": cts.sim_event_t, "sim_result_t": cts.sim_result_t,
               "sim_stats_t": cts.sim_stats_t, "sim_readout_params_t": cts.sim_readout_params_t,
               "sim_cluster_t": cts.sim_cluster_t, "sim_gen_event_t": cts.sim_gen_event_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cts.h"', "int main(void) {"]
    for name, py in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            parts = ln.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for name, py in structs.items():
        assert got[(name, "size")] == C.sizeof(py), name
        for f, _ in py._fields_:
            assert got[(name, f)] == getattr(py, f).offset, (name, f)


def test_autotune_cache_file_roundtrip(tmp_path):
    import ctypes as C
    import numpy as np
    L = cts.load()
    path = str(tmp_path / "table.txt").encode()
    mins = np.array([0, 1000, 50000], dtype=np.int64)
    vars_ = np.array([2, 1, 4], dtype=np.int32)
    p64, p32 = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
    assert L.cts_variant_table_save(path, b"GPU X", 11, mins.ctypes.data_as(p64),
                                    vars_.ctypes.data_as(p32), 3) == 0
    m2, v2, n = np.zeros(8, np.int64), np.zeros(8, np.int32), C.c_int32(0)
    assert L.cts_variant_table_load(path, b"GPU X", 11, m2.ctypes.data_as(p64),
                                    v2.ctypes.data_as(p32), 8, C.byref(n)) == 0
    assert n.value == 3 and np.array_equal(m2[:3], mins) and np.array_equal(v2[:3], vars_)
    # another device or another set of variants: not used
    assert L.cts_variant_table_load(path, b"GPU Y", 11, m2.ctypes.data_as(p64),
                                    v2.ctypes.data_as(p32), 8, C.byref(n)) == -4 and n.value == 0
    assert L.cts_variant_table_load(path, b"GPU X", 12, m2.ctypes.data_as(p64),
                                    v2.ctypes.data_as(p32), 8, C.byref(n)) == -4
    # too small a buffer, a missing file, a damaged file
    assert L.cts_variant_table_load(path, b"GPU X", 11, m2.ctypes.data_as(p64),
                                    v2.ctypes.data_as(p32), 2, C.byref(n)) == -2
    assert L.cts_variant_table_load(str(tmp_path / "none").encode(), b"GPU X", 11,
                                    m2.ctypes.data_as(p64), v2.ctypes.data_as(p32), 8,
                                    C.byref(n)) == -3
    bad = tmp_path / "bad.txt"
    bad.write_text("cts-variant-table 1\nGPU X\n11 2\n0 3\n5 99\n")
    assert L.cts_variant_table_load(str(bad).encode(), b"GPU X", 11, m2.ctypes.data_as(p64),
                                    v2.ctypes.data_as(p32), 8, C.byref(n)) == -2


@pytest.mark.parametrize("mode", [2, 3])
def test_dynamic_plans_keep_partial_sums_inside_their_buffer(lib, mode):
    # every piece of a split tile owns its 3 * tile_i region of the FP64
    # partial-sum buffer (pbase + 3 * tile_i * piece); a plan must never place
    # one beyond the buffer it is given, and regions never overlap
    tile = 512
    for cap in (0, 3 * tile, 3 * tile * 5, 3 * tile * 40, 3 * tile * 400):
        rc, units, begin, pfl = cts.cts_plan_units([5525] * 16, [0] * 16, tile, 608,
                                                   allow_split=mode, partial_cap=cap)
        assert rc == 0 and pfl <= cap
        assert _check_cover(units, [5525] * 16, [0] * 16)
        split = units[units[:, 7] > 1]
        regions = {}
        used = np.zeros(max(cap, 1), dtype=int)
        for u in split:
            lo = u[9] + 3 * tile * u[6]
            assert 0 <= u[9] and 0 <= u[6] < u[7] and lo + 3 * tile <= cap
            used[lo:lo + 3 * tile] += 1
            regions.setdefault((u[0], u[1], u[2]), set()).add((u[8], u[9], u[7]))
        assert used.max() <= 1
        # one (combine counter, base, pieces) per tile, different tiles never share one
        assert all(len(v) == 1 for v in regions.values())
        owners = [next(iter(v)) for v in regions.values()]
        assert len({o[1] for o in owners}) == len(owners) == len({o[0] for o in owners})
        if cap >= 3 * tile * 400:
            assert len(split) > 0


def test_whole_tile_plan_is_balanced_longest_first(lib):
    # allow_split = 0 deals whole tiles, longest first, to the least loaded
    # CTA: no CTA ends above the mean load plus one tile (list scheduling)
    n_h, n_e, tile, grid = [5525, 829, 3000, 1381, 2210, 4834], [0] * 6, 512, 8
    rc, units, begin, pfl = cts.cts_plan_units(n_h, n_e, tile, grid, allow_split=0)
    assert rc == 0 and pfl == 0 and np.all(units[:, 7] == 1)
    assert _check_cover(units, n_h, n_e)
    cost = units[:, 3] * (units[:, 5] - units[:, 4])
    load = np.array([cost[begin[g]:begin[g + 1]].sum() for g in range(grid)])
    assert load.max() <= cost.sum() / grid + cost.max()
    assert np.count_nonzero(load) == grid
