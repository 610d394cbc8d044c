"""Python binding of the GB300 charge-transport library (include/cts.h).

Brute-force drift-diffusion-repulsion Monte Carlo of Xie et al., arXiv
2506.09712 (Sec. 2.1, Algorithm 1), run by hand-written sm_103a kernels in
``_build/libcts.so``.  This module only marshals arguments through ctypes: the
functions keep the C names (``sim_init``, ``sim_submit``, ``sim_poll`` ...),
and ``Simulator`` wraps a handle for convenience.  There is no fallback: if
the library is missing or no sm_103 device is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CTS_CHECKED=1 selects the bounds-checked build (build.build(checked=True))
CHECKED = os.environ.get("CTS_CHECKED", "") == "1"
LIB_PATH = (os.path.join(_HERE, "_build_checked", "libcts_checked.so") if CHECKED
            else os.path.join(_HERE, "_build", "libcts.so"))

SIM_OK, SIM_EINVAL, SIM_ENOMEM_BUDGET, SIM_EAGAIN, SIM_ETIMEOUT = 0, -1, -2, -3, -4
SIM_ECUDA, SIM_EMAXSTEPS, SIM_ENUMERIC, SIM_ESTATE, SIM_ENODEV = -5, -6, -7, -8, -9
CTS_HOLES, CTS_BOTH = 1, 3
CTS_MOB_CT, CTS_MOB_CONST = 0, 1
CTS_PHOTON, CTS_TRACK, CTS_EXPLICIT = 0, 1, 2
CTS_MODE_PLAIN, CTS_MODE_BATCHED, CTS_MODE_SERVE = 0, 1, 2
SIM_INDUCED_TOTAL, SIM_INDUCED_PIXELS = 1, 2   # options.keep_induced flags
SIM_BUILD_BOUNDS_CHECK = 1                       # sim_build_flags()


class sim_sensor_t(C.Structure):
    _fields_ = [("thickness_um", C.c_double), ("bias_V", C.c_double),
                ("depletion_V", C.c_double), ("temperature_K", C.c_double),
                ("eps_r", C.c_double), ("pitch_um", C.c_double), ("dt_ps", C.c_double),
                ("softening_um", C.c_double), ("max_steps", C.c_int64),
                ("grid_n", C.c_int32), ("species", C.c_int32),
                ("drift_table_Vum", C.POINTER(C.c_double)), ("drift_table_n", C.c_int32)]


class sim_field_t(C.Structure):
    _fields_ = [("repulsion", C.c_int32), ("drift", C.c_int32), ("diffusion", C.c_int32),
                ("spherical", C.c_int32)]


class sim_mobility_t(C.Structure):
    _fields_ = [("model", C.c_int32), ("reserved", C.c_int32),
                ("mu0_h", C.c_double), ("vsat_h", C.c_double), ("beta_h", C.c_double),
                ("mu0_e", C.c_double), ("vsat_e", C.c_double), ("beta_e", C.c_double)]


class sim_options_t(C.Structure):
    _fields_ = [("mode", C.c_int32), ("device", C.c_int32), ("max_slots", C.c_int32),
                ("chunk_steps", C.c_int32), ("max_carriers", C.c_int64),
                ("hbm_budget_bytes", C.c_int64), ("queue_capacity", C.c_int32),
                ("variant", C.c_int32), ("disable_graphs", C.c_int32),
                ("keep_final_xy", C.c_int32), ("time_launches", C.c_int32),
                ("keep_induced", C.c_int32), ("step_launches", C.c_int32),
                ("stream", C.c_void_p), ("autotune_cache", C.c_char_p),
                ("sph_cluster", C.c_int32), ("reserved", C.c_int32)]


class sim_readout_params_t(C.Structure):
    _fields_ = [("grid_n", C.c_int32), ("n_bins", C.c_int32), ("ev_per_pair", C.c_double),
                ("noise_keV", C.c_double), ("beam_keV", C.c_double), ("window_keV", C.c_double),
                ("veto_factor", C.c_double), ("spec_lo_keV", C.c_double),
                ("spec_bin_keV", C.c_double)]


class sim_cluster_t(C.Structure):
    _fields_ = [("accepted", C.c_int32), ("vetoed", C.c_int32), ("cx", C.c_int32),
                ("cy", C.c_int32), ("e_cluster", C.c_double), ("e", C.c_double * 9)]


class sim_gen_event_t(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("event_id", C.c_uint64), ("n_pairs", C.c_int32),
                ("reserved", C.c_int32), ("x_um", C.c_double), ("y_um", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double)]


class sim_event_t(C.Structure):
    _fields_ = [("event_id", C.c_uint64), ("seed", C.c_uint64), ("kind", C.c_int32),
                ("n_pairs", C.c_int32), ("energy_keV", C.c_double), ("depth_um", C.c_double),
                ("x_um", C.c_double), ("y_um", C.c_double), ("sigma_um", C.c_double),
                ("track_len_um", C.c_double), ("theta_deg", C.c_double),
                ("phi_deg", C.c_double), ("explicit_xyz", C.POINTER(C.c_double)),
                ("explicit_sign", C.POINTER(C.c_int8))]


class sim_result_t(C.Structure):
    _fields_ = [("event_id", C.c_uint64), ("status", C.c_int32), ("n_carriers", C.c_int32),
                ("n_steps", C.c_int64), ("n_collected", C.c_int64), ("n_outside", C.c_int64),
                ("n_lost", C.c_int64), ("interactions", C.c_int64),
                ("t_submit_ns", C.c_double), ("t_start_ns", C.c_double),
                ("t_done_ns", C.c_double), ("pixels", C.POINTER(C.c_int32)),
                ("final_xy", C.POINTER(C.c_double)), ("retire_step", C.POINTER(C.c_int32)),
                ("capacity", C.c_int64), ("induced_e", C.POINTER(C.c_double)),
                ("induced_capacity", C.c_int64), ("induced_px", C.POINTER(C.c_double))]


class sim_stats_t(C.Structure):
    _fields_ = [("events_done", C.c_int64), ("interactions", C.c_int64),
                ("steps_launched", C.c_int64), ("kernel_launches", C.c_int64),
                ("chunks", C.c_int64), ("queue_depth", C.c_int64), ("rejected", C.c_int64),
                ("sm_count", C.c_int32), ("variant", C.c_int32), ("device_ms", C.c_double),
                ("step_kernel_ms", C.c_double), ("step_kernel_launches", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
                ("symmetric", C.c_int32), ("sph_cluster", C.c_int32)]


class cts_unit_t(C.Structure):
    _fields_ = [(n, C.c_int32) for n in
                ("slot", "spec", "i0", "ni", "j0", "j1", "split", "nsplit", "iblock", "pbase")]


# Every symbol that include/cts.h and include/cts_host.h declare.
EXPORTED = ["sim_init", "sim_submit", "sim_poll", "sim_run", "sim_stage", "sim_execute",
            "sim_collect", "sim_get_stats", "sim_destroy", "sim_strerror", "sim_debug_field",
            "sim_debug_bin", "sim_debug_philox", "sim_debug_normals", "sim_debug_trajectory",
            "sim_debug_inject", "sim_debug_step", "sim_debug_trace_step", "sim_debug_time_step", "sim_debug_launch_log",
            "sim_debug_fma_peak", "sim_build_flags", "sim_readout", "cts_fano_pairs", "sim_generate",
            "cts_fit_ggd", "cts_fit_alpha_t", "cts_fit_beta_t", "cts_ggd_params_at",
            "cts_variant_table_save", "cts_variant_table_load",
            "sim_set_variants",
            "sim_get_variants", "sim_autotune", "sim_reset", "cts_field_noalloc", "cts_plan_units", "cts_plan_sym",
            "cts_arena_replay",
            "cts_estimate_steps"]

_lib = None


class SimError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else strerror(code))


def load(build_if_missing: bool = True):
    """Load libcts.so (building it in-tree first if needed).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) and build_if_missing:
        from . import build as _b
        _b.build(checked=CHECKED)
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH}")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    i32, i64, u32, u64, d = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    sig = {
        "sim_init": [P(sim_sensor_t), P(sim_field_t), P(sim_mobility_t), P(sim_options_t),
                     P(C.c_void_p)],
        "sim_submit": [C.c_void_p, P(sim_event_t), C.c_int, P(C.c_int)],
        "sim_poll": [C.c_void_p, P(sim_result_t), C.c_int, P(C.c_int), C.c_int],
        "sim_run": [C.c_void_p, P(sim_event_t), C.c_int, P(sim_result_t)],
        "sim_stage": [C.c_void_p, P(sim_event_t), C.c_int],
        "sim_execute": [C.c_void_p],
        "sim_collect": [C.c_void_p, P(sim_result_t), C.c_int, P(C.c_int)],
        "sim_get_stats": [C.c_void_p, P(sim_stats_t)],
        "sim_destroy": [C.c_void_p],
        "sim_strerror": [C.c_int],
        "sim_debug_field": [C.c_void_p, P(C.c_float), P(C.c_float), P(C.c_float), i32, i32,
                            P(d)],
        "sim_debug_bin": [C.c_void_p, P(d), P(d), i64, P(i32), P(i64)],
        "sim_debug_philox": [P(u32), P(u32), i64, P(u32), P(u32)],
        "sim_debug_normals": [P(u64), i64, P(d)],
        "sim_debug_trajectory": [C.c_void_p, P(sim_event_t), i64, P(d), P(C.c_int8), i64,
                                 P(i64)],
        "sim_debug_step": [C.c_void_p, u64, u64, i32, P(d), P(C.c_int8), P(d), P(C.c_int8)],
        "sim_debug_inject": [C.c_void_p, C.c_int],
        "sim_debug_trace_step": [C.c_void_p, P(u64), i32, P(i32)],
        "sim_debug_time_step": [C.c_void_p, i32, i32, P(d)],
        "sim_debug_launch_log": [C.c_void_p, P(d), i32, P(i32)],
        "sim_debug_fma_peak": [i32, i32, P(d)],
        "sim_build_flags": [],
        "sim_readout": [P(sim_readout_params_t), P(i32), P(u64), P(u64), i32, i32, P(d),
                        P(sim_cluster_t), P(i64)],
        "cts_fano_pairs": [u64, u64, d, d, P(i32)],
        "sim_generate": [P(sim_gen_event_t), i32, d, i32, i32, P(i32), P(i64)],
        "cts_fit_ggd": [P(d), i64, P(d), P(d)],
        "cts_fit_alpha_t": [P(d), P(d), P(d), i32, P(d)],
        "cts_fit_beta_t": [P(d), P(d), P(d), i32, P(d)],
        "cts_ggd_params_at": [P(d), P(d), d, P(d), P(d)],
        "cts_variant_table_save": [C.c_char_p, C.c_char_p, i32, P(i64), P(i32), i32],
        "cts_variant_table_load": [C.c_char_p, C.c_char_p, i32, P(i64), P(i32), i32, P(i32)],
        "sim_set_variants": [C.c_void_p, P(i64), P(i32), i32],
        "sim_reset": [C.c_void_p],
        "sim_get_variants": [C.c_void_p, P(i64), P(i32), i32, P(i32)],
        "sim_autotune": [C.c_void_p, P(sim_event_t), i32, i32, P(i32)],
        "cts_field_noalloc": [C.c_void_p, C.c_void_p, C.c_void_p, i32, i32, d, d, C.c_void_p,
                              C.c_void_p],
        "cts_plan_units": [P(i32), P(i32), i32, i32, i32, i32, i32, i64, P(cts_unit_t), P(i32),
                           P(i32), P(i64)],
        "cts_plan_sym": [P(i32), P(i32), i32, i32, C.c_void_p, P(i32), C.c_void_p, i32, P(i32),
                         P(i32), i64, P(i64)],
        "cts_arena_replay": [i64, P(i64), i32, P(i64)],
        "cts_estimate_steps": [d, d, d, d, d, d, d, d],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.sim_strerror.restype = C.c_char_p
    lib.cts_estimate_steps.restype = C.c_double
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().sim_strerror(int(code)).decode()


def _check(rc, what):
    if rc != SIM_OK:
        raise SimError(rc, what)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


# ----------------------------------------------------------------------------
# Same-name thin wrappers (argument marshalling only)
# ----------------------------------------------------------------------------
def sim_init(sensor: sim_sensor_t, field: sim_field_t, mobility: sim_mobility_t,
             options: sim_options_t | None = None):
    h = C.c_void_p()
    rc = load().sim_init(C.byref(sensor), C.byref(field), C.byref(mobility),
                         C.byref(options) if options is not None else None, C.byref(h))
    return rc, h


def sim_submit(h, events, n=None):
    n = len(events) if n is None else n
    acc = C.c_int(0)
    rc = load().sim_submit(h, events, n, C.byref(acc))
    return rc, acc.value


def sim_poll(h, results, max_out, timeout_ms):
    n = C.c_int(0)
    rc = load().sim_poll(h, results, max_out, C.byref(n), timeout_ms)
    return rc, n.value


def sim_run(h, events, n, results):
    return load().sim_run(h, events, n, results)


def sim_stage(h, events, n):
    return load().sim_stage(h, events, n)


def sim_execute(h):
    return load().sim_execute(h)


def sim_collect(h, results, max_out):
    n = C.c_int(0)
    rc = load().sim_collect(h, results, max_out, C.byref(n))
    return rc, n.value


def sim_get_stats(h):
    st = sim_stats_t()
    _check(load().sim_get_stats(h, C.byref(st)), "sim_get_stats")
    return st


def sim_destroy(h):
    return load().sim_destroy(h)


def sim_strerror(code):
    return strerror(code)


def sim_debug_field(h, xyz, n_h, n_e=0):
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    x = np.ascontiguousarray(xyz[:, 0]); y = np.ascontiguousarray(xyz[:, 1])
    z = np.ascontiguousarray(xyz[:, 2])
    out = np.zeros((xyz.shape[0], 3), dtype=np.float64)
    rc = load().sim_debug_field(h, _ptr(x, C.c_float), _ptr(y, C.c_float), _ptr(z, C.c_float),
                                int(n_h), int(n_e), _ptr(out, C.c_double))
    _check(rc, "sim_debug_field")
    return out


def sim_debug_bin(h, x, y, grid_n):
    x = np.ascontiguousarray(x, dtype=np.float64); y = np.ascontiguousarray(y, dtype=np.float64)
    pix = np.zeros(grid_n * grid_n, dtype=np.int32)
    out = C.c_int64(0)
    _check(load().sim_debug_bin(h, _ptr(x, C.c_double), _ptr(y, C.c_double), x.size,
                                _ptr(pix, C.c_int32), C.byref(out)), "sim_debug_bin")
    return pix.reshape(grid_n, grid_n), out.value


def sim_debug_philox(ctr, key, with_curand=False):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    n = ctr.shape[0]
    out = np.zeros((n, 4), dtype=np.uint32)
    cur = np.zeros((n, 4), dtype=np.uint32) if with_curand else None
    _check(load().sim_debug_philox(_ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32), n,
                                   _ptr(out, C.c_uint32), _ptr(cur, C.c_uint32)),
           "sim_debug_philox")
    return (out, cur) if with_curand else out


def sim_debug_normals(tuples):
    t = np.ascontiguousarray(tuples, dtype=np.uint64).reshape(-1, 5)
    out = np.zeros((t.shape[0], 3), dtype=np.float64)
    _check(load().sim_debug_normals(_ptr(t, C.c_uint64), t.shape[0], _ptr(out, C.c_double)),
           "sim_debug_normals")
    return out


def sim_debug_trajectory(h, event: sim_event_t, n_steps, n_carriers):
    pos = np.zeros((max(n_carriers, 1), 3), dtype=np.float64)
    st = np.zeros(max(n_carriers, 1), dtype=np.int8)
    done = C.c_int64(0)
    rc = load().sim_debug_trajectory(h, C.byref(event), int(n_steps), _ptr(pos, C.c_double),
                                     _ptr(st, C.c_int8), pos.shape[0], C.byref(done))
    _check(rc, "sim_debug_trajectory")
    return pos[:n_carriers], st[:n_carriers], done.value


def sim_debug_step(h, seed, event_id, xyz, sign=None):
    """One step through the step kernel from FP64 positions xyz (n x 3, all
    active carriers 0..n-1 of event (seed, event_id) at its step 0); returns
    (positions, states) after the step."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    sg = None if sign is None else np.ascontiguousarray(sign, dtype=np.int8)
    out = np.zeros((n, 3), dtype=np.float64)
    st = np.zeros(n, dtype=np.int8)
    _check(load().sim_debug_step(h, int(seed), int(event_id), n, _ptr(xyz, C.c_double),
                                 _ptr(sg, C.c_int8), _ptr(out, C.c_double), _ptr(st, C.c_int8)),
           "sim_debug_step")
    return out, st


def sim_debug_inject(h, fault):
    return load().sim_debug_inject(h, int(fault))


def cts_fano_pairs(seed, event_id, energy_keV, fano=0.13):
    """Carrier pairs of one photon with Fano statistics (goes into n_pairs)."""
    n = C.c_int32(0)
    rc = load().cts_fano_pairs(int(seed), int(event_id), float(energy_keV), float(fano),
                               C.byref(n))
    if rc != 0:
        raise ValueError("cts_fano_pairs: bad arguments")
    return n.value


# numpy record layout of sim_gen_event_t (56 bytes)
GEN_EVENT_DTYPE = np.dtype([("seed", "<u8"), ("event_id", "<u8"), ("n_pairs", "<i4"),
                            ("reserved", "<i4"), ("x_um", "<f8"), ("y_um", "<f8"),
                            ("alpha", "<f8"), ("beta", "<f8")])


def gen_events(seed, event_id, n_pairs, x_um, y_um, alpha, beta):
    """A GEN_EVENT_DTYPE record array from per-event columns (or scalars)."""
    cols = [np.asarray(c) for c in (seed, event_id, n_pairs, x_um, y_um, alpha, beta)]
    n = max(c.size for c in cols)
    rec = np.zeros(n, dtype=GEN_EVENT_DTYPE)
    for name, c in zip(("seed", "event_id", "n_pairs", "x_um", "y_um", "alpha", "beta"), cols):
        rec[name] = np.broadcast_to(c, (n,))
    return rec


def sim_generate(events, pitch_um, grid_n, device=0):
    """Fast generation on the GPU from a GEN_EVENT_DTYPE record array or dicts
    with seed, event_id, n_pairs, x_um, y_um, alpha, beta: pixel counts
    (n_ev x g x g) and off-grid counts."""
    if isinstance(events, np.ndarray) and events.dtype == GEN_EVENT_DTYPE:
        rec = np.ascontiguousarray(events)
    else:
        ev = list(events)
        rec = gen_events(*[[e[k] for e in ev] for k in
                           ("seed", "event_id", "n_pairs", "x_um", "y_um", "alpha", "beta")]) \
            if ev else np.zeros(0, dtype=GEN_EVENT_DTYPE)
    n = rec.size
    pix = np.zeros((n, grid_n, grid_n), np.int32)
    out = np.zeros(max(n, 1), np.int64)
    buf = rec if n else np.zeros(1, dtype=GEN_EVENT_DTYPE)
    _check(load().sim_generate(buf.ctypes.data_as(C.POINTER(sim_gen_event_t)), n,
                               float(pitch_um), int(grid_n), int(device),
                               _ptr(pix, C.c_int32), _ptr(out, C.c_int64)), "sim_generate")
    return pix, out[:n]


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def cts_fit_ggd(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    a, b = C.c_double(0.0), C.c_double(0.0)
    if load().cts_fit_ggd(_dptr(x), x.size, C.byref(a), C.byref(b)) != 0:
        raise ValueError("cts_fit_ggd: need two or more finite, not all zero samples")
    return a.value, b.value


def cts_fit_alpha_t(t, alpha, w=None):
    t = np.ascontiguousarray(t, dtype=np.float64)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    p = np.zeros(4)
    if load().cts_fit_alpha_t(_dptr(t), _dptr(al), _dptr(wv) if wv is not None else None,
                              t.size, _dptr(p)) != 0:
        raise ValueError("cts_fit_alpha_t failed")
    return p


def cts_fit_beta_t(t, beta, p0, sigma=None):
    t = np.ascontiguousarray(t, dtype=np.float64)
    be = np.ascontiguousarray(beta, dtype=np.float64)
    sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    p = np.array(p0, dtype=np.float64)
    if load().cts_fit_beta_t(_dptr(t), _dptr(be), _dptr(sg) if sg is not None else None,
                             t.size, _dptr(p)) != 0:
        raise ValueError("cts_fit_beta_t failed")
    return p


def cts_ggd_params_at(p_alpha, p_beta, t):
    pa = np.ascontiguousarray(p_alpha, dtype=np.float64)
    pb = np.ascontiguousarray(p_beta, dtype=np.float64)
    a, b = C.c_double(0.0), C.c_double(0.0)
    rc = load().cts_ggd_params_at(_dptr(pa), _dptr(pb), float(t), C.byref(a), C.byref(b))
    if rc != 0:
        raise ValueError("cts_ggd_params_at: bad input or non-positive parameters")
    return a.value, b.value


READOUT_DEFAULTS = dict(ev_per_pair=3.62, noise_keV=0.13, window_keV=1.0, veto_factor=3.0,
                        spec_lo_keV=0.0, spec_bin_keV=0.1)


def sim_readout(counts, seeds, event_ids, beam_keV, n_bins=0, device=0, want_pixels=False,
                **kw):
    """Detector readout of pixel-count maps (n_ev x g x g) on the GPU: noisy
    pixel energies, the 3 x 3 cluster around the largest pixel, the pile-up
    veto, the energy window and the single-pixel spectrum.  Returns a dict
    like the oracle's readout: e (if want_pixels), cluster, cx, cy,
    e_cluster, accepted, vetoed, spectrum."""
    prm_d = dict(READOUT_DEFAULTS, **kw)
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    n_ev, g = counts.shape[0], counts.shape[1]
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    ids = np.ascontiguousarray(event_ids, dtype=np.uint64)
    prm = sim_readout_params_t(grid_n=g, n_bins=int(n_bins), beam_keV=float(beam_keV),
                               **{k: float(v) for k, v in prm_d.items()})
    cl = (sim_cluster_t * max(n_ev, 1))()
    spec = np.zeros(max(int(n_bins), 1), np.int64)
    pix = np.zeros((n_ev, g, g)) if want_pixels else None
    _check(load().sim_readout(C.byref(prm), _ptr(counts, C.c_int32), _ptr(seeds, C.c_uint64),
                              _ptr(ids, C.c_uint64), n_ev, int(device),
                              _ptr(pix, C.c_double) if want_pixels else None, cl,
                              _ptr(spec, C.c_int64) if n_bins > 0 else None), "sim_readout")
    raw = np.frombuffer(cl, dtype=np.uint8, count=96 * n_ev).reshape(n_ev, 96)
    ints = raw[:, :16].copy().view(np.int32).reshape(n_ev, 4)
    dbl = raw[:, 16:].copy().view(np.float64).reshape(n_ev, 10)
    out = dict(cluster=dbl[:, 1:], e_cluster=dbl[:, 0], accepted=ints[:, 0], vetoed=ints[:, 1],
               cx=ints[:, 2], cy=ints[:, 3], spectrum=spec[:int(n_bins)])
    if want_pixels:
        out["e"] = pix
    return out


def sim_build_flags() -> int:
    """SIM_BUILD_BOUNDS_CHECK when the loaded library is the checked build."""
    return load().sim_build_flags()


def sim_debug_fma_peak(device=0, packed=True):
    """Measured FP32 FMA throughput (flops/s) of FMA chains on `device`."""
    v = C.c_double(0.0)
    _check(load().sim_debug_fma_peak(int(device), 1 if packed else 0, C.byref(v)),
           "sim_debug_fma_peak")
    return v.value


def sim_debug_launch_log(h, cap=1 << 20):
    """Per-launch (kernel ms, carrier pairs covered, events running, 1 if the
    symmetric kernel ran) rows of the step kernel since the last call (handle
    made with time_launches)."""
    out = np.zeros((cap, 4), dtype=np.float64)
    n = C.c_int32(0)
    _check(load().sim_debug_launch_log(h, out.ctypes.data_as(C.POINTER(C.c_double)), int(cap),
                                       C.byref(n)), "sim_debug_launch_log")
    return out[:n.value].copy()


def sim_debug_time_step(h, variant=0, reps=3):
    """Mean launch time (ms) of the pair kernel on the staged events."""
    ms = C.c_double(0.0)
    _check(load().sim_debug_time_step(h, int(variant), int(reps), C.byref(ms)),
           "sim_debug_time_step")
    return ms.value


def sim_set_variants(h, min_pairs, variants):
    mp = np.ascontiguousarray(min_pairs, dtype=np.int64)
    vs = np.ascontiguousarray(variants, dtype=np.int32)
    _check(load().sim_set_variants(h, _ptr(mp, C.c_int64), _ptr(vs, C.c_int32), mp.size),
           "sim_set_variants")


def sim_reset(h):
    _check(load().sim_reset(h), "sim_reset")


def sim_get_variants(h, cap=64):
    mp = np.zeros(cap, dtype=np.int64)
    vs = np.zeros(cap, dtype=np.int32)
    n = C.c_int32(0)
    _check(load().sim_get_variants(h, _ptr(mp, C.c_int64), _ptr(vs, C.c_int32), cap,
                                   C.byref(n)), "sim_get_variants")
    return [(int(mp[q]), int(vs[q])) for q in range(min(n.value, cap))]


def sim_autotune(h, events, n, reps=3):
    nb = C.c_int32(0)
    _check(load().sim_autotune(h, events, int(n), int(reps), C.byref(nb)), "sim_autotune")
    return nb.value


def sim_debug_trace_step(h, max_ctas=8192):
    """Per-CTA (smid, t_start_ns, t_end_ns, pairs, units, ns_prologue, ns_loop,
    ns_epilogue) of one field-only step."""
    out = np.zeros((max_ctas, 8), dtype=np.uint64)
    n = C.c_int32(0)
    _check(load().sim_debug_trace_step(h, _ptr(out, C.c_uint64), max_ctas, C.byref(n)),
           "sim_debug_trace_step")
    return out[:n.value]


def cts_field_noalloc(dev_x, dev_y, dev_z, n_h, n_e, eps_r, softening_um, dev_E, stream=None):
    """Allocation-free field: device pointers (ints) in and out; returns the status code."""
    return load().cts_field_noalloc(dev_x, dev_y, dev_z, int(n_h), int(n_e), float(eps_r),
                                    float(softening_um), dev_E, stream)


def cts_plan_units(n_h, n_e, tile_i, grid, allow_split=1, max_units=65536,
                   partial_cap=1 << 26):
    """Returns (rc, units[n, 10], cta_begin[grid + 1], partial_floats)."""
    n_h = np.ascontiguousarray(n_h, dtype=np.int32); n_e = np.ascontiguousarray(n_e, dtype=np.int32)
    out = (cts_unit_t * max_units)()
    begin = np.zeros(grid + 1, dtype=np.int32)
    n = C.c_int32(0)
    pf = C.c_int64(0)
    rc = load().cts_plan_units(_ptr(n_h, C.c_int32), _ptr(n_e, C.c_int32), n_h.size, tile_i,
                               grid, allow_split, max_units, partial_cap, out, C.byref(n),
                               _ptr(begin, C.c_int32), C.byref(pf))
    if rc != 0:
        return rc, None, None, 0
    raw = np.frombuffer(out, dtype=np.int32, count=n.value * 10).reshape(-1, 10)
    return rc, raw.astype(np.int64), begin, pf.value


SYM_UNIT_FIELDS = ("slot", "spec_i", "spec_j", "ib0", "ib1", "jt0", "jt1", "p_i", "p_j", "duty",
                   "kind", "npair")
SYM_TILE_FIELDS = ("slot", "spec", "tile", "n", "lptr", "lcnt")


def cts_plan_sym(n_h, n_e, max_units=65536):
    """The symmetric kernel's plan of one step: (rc, units[n, 12], tiles[m, 6],
    lists[L], n_partials); columns as SYM_UNIT_FIELDS and SYM_TILE_FIELDS."""
    n_h = np.ascontiguousarray(n_h, dtype=np.int32); n_e = np.ascontiguousarray(n_e, dtype=np.int32)
    per_slot = [(max(a, 0) + 63) // 64 + (max(b, 0) + 63) // 64 for a, b in zip(n_h, n_e)]
    tiles_cap = int(sum(per_slot)) + 1
    units = np.zeros((max_units, len(SYM_UNIT_FIELDS)), dtype=np.int32)
    tiles = np.zeros((tiles_cap, 6), dtype=np.int32)
    # a tile's list holds at most one I and one J partial per unit of its slot
    lists_cap = max(1, int(sum(t * (2 * t + 16) for t in per_slot)))
    lists = np.zeros(lists_cap, dtype=np.int32)
    nu, nt, npart = C.c_int32(0), C.c_int32(0), C.c_int64(0)
    rc = load().cts_plan_sym(_ptr(n_h, C.c_int32), _ptr(n_e, C.c_int32), n_h.size, max_units,
                             units.ctypes.data, C.byref(nu), tiles.ctypes.data, tiles_cap,
                             C.byref(nt), _ptr(lists, C.c_int32), lists_cap, C.byref(npart))
    if rc != 0:
        return rc, None, None, None, 0
    return (rc, units[:nu.value].astype(np.int64), tiles[:nt.value].astype(np.int64),
            lists[:int(tiles[:nt.value, 5].sum())].copy(), npart.value)


def cts_arena_replay(capacity, ops):
    ops = np.ascontiguousarray(ops, dtype=np.int64)
    res = np.zeros(ops.size, dtype=np.int64)
    rc = load().cts_arena_replay(int(capacity), _ptr(ops, C.c_int64), ops.size, _ptr(res, C.c_int64))
    return rc, res


def cts_estimate_steps(thickness_um, bias_V, depletion_V, mu0, vsat, beta, dt_ps, depth_um):
    return load().cts_estimate_steps(thickness_um, bias_V, depletion_V, mu0, vsat, beta, dt_ps,
                                     depth_um)


# ----------------------------------------------------------------------------
# Convenience layer: presets (dicts) -> structs, and a handle object
# ----------------------------------------------------------------------------
def make_sensor(d: dict) -> sim_sensor_t:
    s = sim_sensor_t()
    s.thickness_um = d["thickness_um"]; s.bias_V = d["bias_V"]; s.depletion_V = d["depletion_V"]
    s.temperature_K = d.get("temperature_K", 293.0); s.eps_r = d.get("eps_r", 11.7)
    s.pitch_um = d.get("pitch_um", 25.0); s.dt_ps = d["dt_ps"]
    s.softening_um = d.get("softening_um", 1e-6); s.max_steps = d.get("max_steps", 200_000)
    s.grid_n = d.get("grid_n", 9); s.species = d.get("species", CTS_HOLES)
    tab = d.get("drift_table_Vum")
    if tab is not None:
        tab = np.ascontiguousarray(tab, dtype=np.float64)
        s._drift_table = tab            # kept alive until sim_init has copied it
        s.drift_table_Vum = tab.ctypes.data_as(C.POINTER(C.c_double))
        s.drift_table_n = tab.size
    return s


def make_field(d: dict | None = None) -> sim_field_t:
    d = d or {}
    return sim_field_t(d.get("repulsion", 1), d.get("drift", 1), d.get("diffusion", 1),
                       d.get("spherical", 0))


def make_mobility(d: dict) -> sim_mobility_t:
    m = sim_mobility_t()
    m.model = d.get("model", CTS_MOB_CT)
    m.mu0_h, m.vsat_h, m.beta_h = d["mu0_h"], d["vsat_h"], d["beta_h"]
    m.mu0_e, m.vsat_e, m.beta_e = d.get("mu0_e", 0.0), d.get("vsat_e", 0.0), d.get("beta_e", 0.0)
    return m


def make_options(mode=CTS_MODE_BATCHED, **kw) -> sim_options_t:
    o = sim_options_t()
    o.mode = mode
    for k, v in kw.items():
        if k == "autotune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def make_events(events: list[dict]):
    """Array of sim_event_t from dicts (explicit positions are kept alive on it)."""
    arr = (sim_event_t * max(len(events), 1))()
    keep = []
    for k, ev in enumerate(events):
        e = arr[k]
        e.event_id = ev.get("event_id", k); e.seed = ev.get("seed", 0)
        e.kind = ev.get("kind", CTS_PHOTON); e.n_pairs = ev.get("n_pairs", 0)
        e.energy_keV = ev.get("energy_keV", 0.0); e.depth_um = ev.get("depth_um", 0.0)
        e.x_um = ev.get("x_um", 0.0); e.y_um = ev.get("y_um", 0.0)
        e.sigma_um = ev.get("sigma_um", -1.0); e.track_len_um = ev.get("track_len_um", 0.0)
        e.theta_deg = ev.get("theta_deg", 0.0); e.phi_deg = ev.get("phi_deg", 0.0)
        if e.kind == CTS_EXPLICIT:
            xyz = np.ascontiguousarray(ev["explicit_xyz"], dtype=np.float64).reshape(-1)
            keep.append(xyz)
            e.explicit_xyz = _ptr(xyz, C.c_double)
            e.n_pairs = xyz.size // 3
            if ev.get("explicit_sign") is not None:
                sg = np.ascontiguousarray(ev["explicit_sign"], dtype=np.int8)
                keep.append(sg)
                e.explicit_sign = _ptr(sg, C.c_int8)
    arr._keep = keep
    return arr


class Results:
    """Caller-owned result buffers for n events."""

    def __init__(self, n: int, grid_n: int, capacity: int = 0, induced_capacity: int = 0,
                 induced_px: bool = False):
        self.n, self.grid_n, self.capacity = n, grid_n, capacity
        self.induced_capacity = induced_capacity
        self.has_px = bool(induced_px and induced_capacity)
        self.induced = np.zeros((max(n, 1), max(induced_capacity, 1)), dtype=np.float64)
        self.induced_px = (np.zeros((max(n, 1), induced_capacity, 3, 3), dtype=np.float64)
                           if self.has_px else None)
        self.pixels = np.zeros((max(n, 1), grid_n, grid_n), dtype=np.int32)
        self.final_xy = np.zeros((max(n, 1), max(capacity, 1), 2), dtype=np.float64)
        self.retire_step = np.zeros((max(n, 1), max(capacity, 1)), dtype=np.int32)
        self.arr = (sim_result_t * max(n, 1))()
        for k in range(max(n, 1)):
            r = self.arr[k]
            r.pixels = _ptr(self.pixels[k], C.c_int32)
            if capacity:
                r.final_xy = _ptr(self.final_xy[k], C.c_double)
                r.retire_step = _ptr(self.retire_step[k], C.c_int32)
                r.capacity = capacity
            if induced_capacity:
                r.induced_e = _ptr(self.induced[k], C.c_double)
                r.induced_capacity = induced_capacity
            if self.has_px:
                r.induced_px = _ptr(self.induced_px[k], C.c_double)

    def record(self, k: int) -> dict:
        r = self.arr[k]
        return dict(event_id=r.event_id, status=r.status, n_carriers=r.n_carriers,
                    n_steps=r.n_steps, n_collected=r.n_collected, n_outside=r.n_outside,
                    n_lost=r.n_lost, interactions=r.interactions, t_submit_ns=r.t_submit_ns,
                    t_start_ns=r.t_start_ns, t_done_ns=r.t_done_ns,
                    pixels=self.pixels[k].copy(),
                    final_xy=self.final_xy[k, :r.n_carriers].copy() if self.capacity else None,
                    retire_step=self.retire_step[k, :r.n_carriers].copy() if self.capacity else None,
                    induced=(self.induced[k, :min(r.n_steps, self.induced_capacity)].copy()
                             if self.induced_capacity else None),
                    induced_px=(self.induced_px[k, :min(r.n_steps, self.induced_capacity)].copy()
                                if self.has_px else None))


class Simulator:
    """A library handle built from preset dictionaries (see ``workloads``)."""

    def __init__(self, sensor: dict, mobility: dict, field: dict | None = None,
                 mode=CTS_MODE_BATCHED, **options):
        self.sensor_d = dict(sensor)
        self.grid_n = int(sensor.get("grid_n", 9))
        self._sensor = make_sensor(sensor)
        self._field = make_field(field)
        self._mob = make_mobility(mobility)
        self._opt = make_options(mode, **options)
        self._px = bool(self._opt.keep_induced & SIM_INDUCED_PIXELS)
        rc, self.h = sim_init(self._sensor, self._field, self._mob, self._opt)
        _check(rc, "sim_init")

    def close(self):
        if self.h:
            sim_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, events: list[dict], keep_xy_capacity: int = 0,
            induced_capacity: int = 0) -> list[dict]:
        evs = make_events(events)
        res = Results(len(events), self.grid_n, keep_xy_capacity, induced_capacity, self._px)
        _check(sim_run(self.h, evs, len(events), res.arr), "sim_run")
        return [res.record(k) for k in range(len(events))]

    def stage(self, events: list[dict]):
        self._staged = make_events(events)
        _check(sim_stage(self.h, self._staged, len(events)), "sim_stage")

    def execute(self):
        _check(sim_execute(self.h), "sim_execute")

    def collect(self, n: int, keep_xy_capacity: int = 0, induced_capacity: int = 0) -> list[dict]:
        res = Results(n, self.grid_n, keep_xy_capacity, induced_capacity, self._px)
        rc, got = sim_collect(self.h, res.arr, n)
        _check(rc, "sim_collect")
        return [res.record(k) for k in range(got)]

    def submit(self, events: list[dict]) -> tuple[int, int]:
        evs = make_events(events)
        return sim_submit(self.h, evs, len(events))

    def poll(self, max_out: int, timeout_ms: int, keep_xy_capacity: int = 0,
             induced_capacity: int = 0) -> list[dict]:
        res = Results(max_out, self.grid_n, keep_xy_capacity, induced_capacity, self._px)
        rc, n = sim_poll(self.h, res.arr, max_out, timeout_ms)
        if rc == SIM_ETIMEOUT:
            return []
        _check(rc, "sim_poll")
        return [res.record(k) for k in range(n)]

    def stats(self) -> dict:
        st = sim_get_stats(self.h)
        return {f: getattr(st, f) for f, _ in sim_stats_t._fields_}

    def field(self, xyz, n_h, n_e=0):
        return sim_debug_field(self.h, xyz, n_h, n_e)

    def bin(self, x, y):
        return sim_debug_bin(self.h, x, y, self.grid_n)

    def trajectory(self, event: dict, n_steps: int):
        evs = make_events([event])
        n = event.get("n_carriers")
        if n is None:
            raise ValueError("trajectory needs event['n_carriers']")
        return sim_debug_trajectory(self.h, evs[0], n_steps, n)

    def inject(self, fault: int):
        return sim_debug_inject(self.h, fault)

    def set_variants(self, table):
        """table: [(min_pairs, variant)] ascending; [] restores the fixed variant."""
        sim_set_variants(self.h, [t[0] for t in table], [t[1] for t in table])

    def reset(self):
        sim_reset(self.h)

    def autotune(self, events: list[dict], reps: int = 3):
        """Measure every kernel variant on batches of these events and install
        the fastest per amount of resident pair work; returns the table."""
        evs = make_events(events)
        sim_autotune(self.h, evs, len(events), reps)
        return sim_get_variants(self.h)

    def variants(self):
        return sim_get_variants(self.h)
