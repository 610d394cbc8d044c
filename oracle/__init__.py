"""FP64 CPU oracle of the brute-force charge-transport Monte Carlo (arXiv 2506.09712).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product (the CUDA library and its
binding) never imports this package, and this package never imports the
product.  The arithmetic lives in ``cts_oracle.c`` (plain C, FP64, OpenMP);
this module only marshals arguments through ctypes.

Parameter dictionaries use the same field names as the workload presets in
``workloads``: sensor geometry and bias, field switches, mobility parameters.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cts_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libcts_oracle.so")

PHOTON, TRACK, EXPLICIT = 0, 1, 2
HOLES, BOTH = 1, 3
MOB_CT, MOB_CONST = 0, 1
ACTIVE, COLLECTED, RETIRED = 0, 1, 2
OK, EMAXSTEPS = 0, -6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) into _build/."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [
        ("thickness_um", C.c_double), ("bias_V", C.c_double), ("depletion_V", C.c_double),
        ("temperature_K", C.c_double), ("eps_r", C.c_double), ("pitch_um", C.c_double),
        ("grid_n", C.c_int32), ("dt_ps", C.c_double), ("max_steps", C.c_int64),
        ("species", C.c_int32), ("softening_um", C.c_double),
        ("repulsion", C.c_int32), ("drift", C.c_int32), ("diffusion", C.c_int32),
        ("mob_model", C.c_int32),
        ("mu0_h", C.c_double), ("vsat_h", C.c_double), ("beta_h", C.c_double),
        ("mu0_e", C.c_double), ("vsat_e", C.c_double), ("beta_e", C.c_double),
        ("spherical", C.c_int32),
        ("drift_table", C.POINTER(C.c_double)), ("drift_table_n", C.c_int32),
    ]


class _Event(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("event_id", C.c_uint64), ("kind", C.c_int32),
        ("energy_keV", C.c_double), ("n_pairs", C.c_int32), ("depth_um", C.c_double),
        ("x_um", C.c_double), ("y_um", C.c_double), ("sigma_um", C.c_double),
        ("track_len_um", C.c_double), ("theta_deg", C.c_double), ("phi_deg", C.c_double),
        ("explicit_xyz", C.POINTER(C.c_double)), ("explicit_sign", C.POINTER(C.c_int8)),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("n_steps", C.c_int64), ("n_collected", C.c_int64),
        ("n_outside", C.c_int64), ("n_lost", C.c_int64), ("interactions", C.c_int64),
        ("pixels", C.POINTER(C.c_int32)), ("final_x", C.POINTER(C.c_double)),
        ("final_y", C.POINTER(C.c_double)), ("retire_step", C.POINTER(C.c_int32)),
        ("pos_out", C.POINTER(C.c_double)), ("state_out", C.POINTER(C.c_int8)),
        ("sign_out", C.POINTER(C.c_int8)),
        ("induced", C.POINTER(C.c_double)), ("induced_capacity", C.c_int64),
        ("induced_px", C.POINTER(C.c_double)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, i32, u32, u64 = C.c_double, C.c_int64, C.c_int32, C.c_uint32, C.c_uint64
        P = C.POINTER
        _lib.or_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        _lib.or_normals3.argtypes = [u64, u64, u32, u32, u32, P(d)]
        _lib.or_coulomb_k.argtypes = [d]; _lib.or_coulomb_k.restype = d
        _lib.or_thermal_voltage.argtypes = [d]; _lib.or_thermal_voltage.restype = d
        _lib.or_n_pairs.argtypes = [d]; _lib.or_n_pairs.restype = i32
        _lib.or_sigma_um.argtypes = [d]; _lib.or_sigma_um.restype = d
        _lib.or_drift_field.argtypes = [P(_Params), d]; _lib.or_drift_field.restype = d
        _lib.or_mobility.argtypes = [P(_Params), C.c_int, d]; _lib.or_mobility.restype = d
        _lib.or_field_rows.argtypes = [i64, P(d), P(d), P(d), P(C.c_int8), P(C.c_int8),
                                       P(i64), i64, d, d, C.c_int, P(d), P(d), P(d)]
        _lib.or_field.argtypes = [i64, P(d), P(d), P(d), P(C.c_int8), P(C.c_int8), d, d,
                                  C.c_int, P(d), P(d), P(d)]
        _lib.or_pixel_of.argtypes = [P(_Params), d, d, P(i32), P(i32)]
        _lib.or_pixel_of.restype = C.c_int
        _lib.or_bin.argtypes = [P(_Params), i64, P(d), P(d), P(i32), P(i64)]
        _lib.or_event_carriers.argtypes = [P(_Params), P(_Event)]
        _lib.or_event_carriers.restype = i64
        _lib.or_init_event.argtypes = [P(_Params), P(_Event), P(d), P(d), P(d), P(C.c_int8)]
        _lib.or_run_event.argtypes = [P(_Params), P(_Event), P(_Result), C.c_int]
        _lib.or_run_event.restype = C.c_int
        _lib.or_run_events.argtypes = [P(_Params), P(_Event), i64, P(_Result)]
        _lib.or_max_threads.restype = C.c_int
        _lib.or_fano_pairs.argtypes = [u64, u64, d, d]; _lib.or_fano_pairs.restype = i32
        _lib.or_ggd_pdf.argtypes = [d, d, d]; _lib.or_ggd_pdf.restype = d
        _lib.or_fit_ggd.argtypes = [P(d), i64, P(d), P(d)]; _lib.or_fit_ggd.restype = C.c_int
        _lib.or_ggd_sample.argtypes = [u64, u64, u32, u32, d, d]; _lib.or_ggd_sample.restype = d
        _lib.or_generate_event.argtypes = [u64, u64, i32, d, d, d, d, d, i32, P(i32), P(i64)]
        _lib.or_field_spherical.argtypes = [i64, P(i64), P(d), P(d), P(d), d, P(d), P(d), P(d)]
        _lib.or_readout_event.argtypes = [P(i32), i32, u64, u64, d, d, d, d, d, P(d), P(d),
                                          P(i32), P(i32), P(d), P(i32)]
        _lib.or_readout_event.restype = C.c_int
        _lib.or_spectrum_add.argtypes = [P(d), i32, d, d, i32, P(i64)]
        _lib.or_uniform.argtypes = [u32]
        _lib.or_uniform.restype = d
        _lib.or_rect_solid_angle.argtypes = [d, d, d, d, d, d, d]
        _lib.or_rect_solid_angle.restype = d
        _lib.or_weighting_potential.argtypes = [d, d, d, d, d, d, d, d, i32]
        _lib.or_weighting_potential.restype = d
        _lib.or_window_potentials.argtypes = [P(_Params), d, d, d, P(d)]
        _lib.or_step.argtypes = [P(_Params), u64, u64, i64, i64, P(d), P(d), P(d),
                                 P(C.c_int8), P(C.c_int8), C.c_int]
        _lib.or_step.restype = i64
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------
def make_params(sensor: dict, field: dict | None = None, mobility: dict | None = None) -> _Params:
    """Build the oracle's parameter block from preset dictionaries."""
    field = field or {}
    mobility = mobility or {}
    p = _Params()
    p.thickness_um = sensor["thickness_um"]
    p.bias_V = sensor["bias_V"]
    p.depletion_V = sensor["depletion_V"]
    p.temperature_K = sensor.get("temperature_K", 293.0)
    p.eps_r = sensor.get("eps_r", 11.7)
    p.pitch_um = sensor.get("pitch_um", 25.0)
    p.grid_n = sensor.get("grid_n", 9)
    p.dt_ps = sensor["dt_ps"]
    p.max_steps = sensor.get("max_steps", 1_000_000)
    p.species = sensor.get("species", HOLES)
    p.softening_um = sensor.get("oracle_softening_um", 0.0)
    p.repulsion = field.get("repulsion", 1)
    p.drift = field.get("drift", 1)
    p.diffusion = field.get("diffusion", 1)
    p.mob_model = mobility.get("model", MOB_CT)
    p.mu0_h = mobility["mu0_h"]
    p.vsat_h = mobility["vsat_h"]
    p.beta_h = mobility["beta_h"]
    p.mu0_e = mobility.get("mu0_e", 0.0)
    p.vsat_e = mobility.get("vsat_e", 1.0)
    p.beta_e = mobility.get("beta_e", 1.0)
    p.spherical = field.get("spherical", 0)
    tab = sensor.get("drift_table_Vum")
    if tab is not None:
        tab = np.ascontiguousarray(tab, dtype=np.float64)
        p._drift_table = tab            # kept alive with the parameters
        p.drift_table = tab.ctypes.data_as(C.POINTER(C.c_double))
        p.drift_table_n = tab.size
    return p


def make_event(ev: dict, keep: list) -> _Event:
    e = _Event()
    e.seed = ev.get("seed", 0)
    e.event_id = ev.get("event_id", 0)
    e.kind = ev.get("kind", PHOTON)
    e.energy_keV = ev.get("energy_keV", 0.0)
    e.n_pairs = ev.get("n_pairs", 0)
    e.depth_um = ev.get("depth_um", 0.0)
    e.x_um = ev.get("x_um", 0.0)
    e.y_um = ev.get("y_um", 0.0)
    e.sigma_um = ev.get("sigma_um", -1.0)
    e.track_len_um = ev.get("track_len_um", 0.0)
    e.theta_deg = ev.get("theta_deg", 0.0)
    e.phi_deg = ev.get("phi_deg", 0.0)
    if e.kind == EXPLICIT:
        xyz = np.ascontiguousarray(ev["explicit_xyz"], dtype=np.float64).reshape(-1)
        keep.append(xyz)
        e.explicit_xyz = _ptr(xyz, C.c_double)
        e.n_pairs = xyz.size // 3
        if ev.get("explicit_sign") is not None:
            sg = np.ascontiguousarray(ev["explicit_sign"], dtype=np.int8)
            keep.append(sg)
            e.explicit_sign = _ptr(sg, C.c_int8)
    return e


# ----------------------------------------------------------------------------
# Small exported pieces (pinned individually by the tests)
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(word: int) -> float:
    """The uniform in (0, 1) that a 32-bit Philox word maps to."""
    return lib().or_uniform(int(word) & 0xFFFFFFFF)


def normals3(seed, event_id, purpose, carrier, step):
    o = (C.c_double * 3)()
    lib().or_normals3(seed, event_id, purpose, carrier, step, o)
    return [o[0], o[1], o[2]]


def coulomb_k(eps_r=11.7):
    return lib().or_coulomb_k(eps_r)


def thermal_voltage(T):
    return lib().or_thermal_voltage(T)


def n_pairs(energy_keV):
    return lib().or_n_pairs(energy_keV)


def field_spherical(xyz, kc=None):
    """FP64 repulsion field of the simplified spherical model (Eq. 7) on the
    holes at xyz (n x 3): k_C Q(<r) (r_i - c) / r^3, c the mean position."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    x, y, z = (np.ascontiguousarray(xyz[:, k]) for k in range(3))
    rows = np.arange(n, dtype=np.int64)
    ex, ey, ez = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().or_field_spherical(n, _ptr(rows, C.c_int64), _ptr(x, C.c_double), _ptr(y, C.c_double),
                             _ptr(z, C.c_double), coulomb_k() if kc is None else kc,
                             _ptr(ex, C.c_double), _ptr(ey, C.c_double), _ptr(ez, C.c_double))
    return np.stack([ex, ey, ez], axis=1)


def ggd_pdf(x, alpha, beta):
    """Eq. 8, the generalised Gaussian density on the whole line."""
    return lib().or_ggd_pdf(float(x), float(alpha), float(beta))


def fit_ggd(x):
    """Maximum-likelihood (alpha, beta) of Eq. 8 for samples centred at 0."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    a, b = C.c_double(0.0), C.c_double(0.0)
    if lib().or_fit_ggd(_ptr(x, C.c_double), x.size, C.byref(a), C.byref(b)) != 0:
        raise ValueError("fit_ggd needs at least two non-zero samples")
    return a.value, b.value


def ggd_samples(seed, event_id, n, alpha, beta, axis=0):
    """The generator's GGD variates of carriers 0 .. n-1 on one axis."""
    L = lib()
    return np.array([L.or_ggd_sample(int(seed), int(event_id), c, axis, float(alpha),
                                     float(beta)) for c in range(n)])


def generate(events, pitch_um, grid_n):
    """Fast event generation (Sec. 4.2) from per-event dicts with seed,
    event_id, n_pairs, x_um, y_um, alpha, beta: pixel counts (n_ev x g x g)
    and carriers outside the grid."""
    L = lib()
    pix = np.zeros((len(events), grid_n, grid_n), np.int32)
    out = np.zeros(len(events), np.int64)
    for k, e in enumerate(events):
        o = C.c_int64(0)
        L.or_generate_event(int(e["seed"]), int(e["event_id"]), int(e["n_pairs"]),
                            float(e["x_um"]), float(e["y_um"]), float(e["alpha"]),
                            float(e["beta"]), float(pitch_um), int(grid_n),
                            _ptr(pix[k], C.c_int32), C.byref(o))
        out[k] = o.value
    return pix, out


def alpha_of_t(p, t):
    """Eq. 10: alpha(t) = p0 + p1 sqrt(t) + p2 t + p3 t^2."""
    t = np.asarray(t, dtype=np.float64)
    return p[0] + p[1] * np.sqrt(t) + p[2] * t + p[3] * t * t


def beta_of_t(p, t):
    """Eq. 11 as read here: beta(t) = 2 + p0 max(t - p1, 0)^p2 + p3 exp(p4 t)."""
    t = np.asarray(t, dtype=np.float64)
    return 2.0 + p[0] * np.maximum(t - p[1], 0.0) ** p[2] + p[3] * np.exp(p[4] * t)


def fit_alpha_of_t(t, alpha, w=None):
    """Weighted linear least squares of Eq. 10 (numpy's solver)."""
    t = np.asarray(t, dtype=np.float64)
    A = np.stack([np.ones_like(t), np.sqrt(t), t, t * t], axis=1)
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    return np.linalg.lstsq(A * w[:, None], np.asarray(alpha) * w, rcond=None)[0]


def fit_beta_of_t(t, beta, p0, sigma=None):
    """Least squares of Eq. 11 from the starting point p0 (scipy's solver)."""
    from scipy import optimize
    return optimize.curve_fit(lambda tt, *q: beta_of_t(q, tt), np.asarray(t, float),
                              np.asarray(beta, float), p0=list(p0), sigma=sigma,
                              maxfev=20000)[0]


def fano_pairs(seed, event_id, energy_keV, fano=0.13):
    """Carrier pairs of one photon with Fano fluctuations (Sec. 4.2)."""
    return lib().or_fano_pairs(int(seed), int(event_id), float(energy_keV), float(fano))


# Readout parameters of the detector (Sec. 4.1 selection, Sec. 4.2 noise).
READOUT_DEFAULTS = dict(ev_per_pair=3.62, noise_keV=0.13, window_keV=1.0, veto_factor=3.0,
                        spec_lo_keV=0.0, spec_bin_keV=0.1)


def readout(counts, seeds, event_ids, beam_keV, n_bins, **kw):
    """Readout of events' pixel counts (n_ev x grid_n x grid_n): noisy pixel
    energies, 3 x 3 cluster around the largest pixel, pile-up veto, energy
    window and the single-pixel spectrum of the accepted clusters.  Returns a
    dict of arrays: e (keV maps), cluster (n_ev x 9), cx, cy, e_cluster,
    accepted, vetoed, spectrum (n_bins)."""
    prm = dict(READOUT_DEFAULTS, **kw)
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    n_ev, g = counts.shape[0], counts.shape[1]
    out = dict(e=np.zeros((n_ev, g, g)), cluster=np.zeros((n_ev, 9)),
               cx=np.zeros(n_ev, np.int32), cy=np.zeros(n_ev, np.int32),
               e_cluster=np.zeros(n_ev), accepted=np.zeros(n_ev, np.int32),
               vetoed=np.zeros(n_ev, np.int32), spectrum=np.zeros(n_bins, np.int64))
    L = lib()
    for k in range(n_ev):
        e = np.zeros(g * g); cl = np.zeros(9)
        cx, cy, v = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        ec = C.c_double(0.0)
        acc = L.or_readout_event(_ptr(counts[k], C.c_int32), g, int(seeds[k]), int(event_ids[k]),
                                 prm["ev_per_pair"], prm["noise_keV"], float(beam_keV),
                                 prm["window_keV"], prm["veto_factor"], _ptr(e, C.c_double),
                                 _ptr(cl, C.c_double), C.byref(cx), C.byref(cy), C.byref(ec),
                                 C.byref(v))
        L.or_spectrum_add(_ptr(cl, C.c_double), acc, prm["spec_lo_keV"], prm["spec_bin_keV"],
                          n_bins, _ptr(out["spectrum"], C.c_int64))
        out["e"][k] = e.reshape(g, g); out["cluster"][k] = cl
        out["cx"][k], out["cy"][k], out["e_cluster"][k] = cx.value, cy.value, ec.value
        out["accepted"][k], out["vetoed"][k] = acc, v.value
    return out


def sigma_um(energy_keV):
    return lib().or_sigma_um(energy_keV)


def drift_field(params: _Params, z):
    return lib().or_drift_field(C.byref(params), z)


def mobility(params: _Params, sign, E):
    return lib().or_mobility(C.byref(params), int(sign), E)


def field(xyz, sign=None, active=None, kc=None, eps=0.0, rows=None, parallel=True):
    """FP64 repulsion field (Eq. 4 read as a field) at `rows` (default: all)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    x = np.ascontiguousarray(xyz[:, 0]); y = np.ascontiguousarray(xyz[:, 1])
    z = np.ascontiguousarray(xyz[:, 2])
    sg = None if sign is None else np.ascontiguousarray(sign, dtype=np.int8)
    ac = None if active is None else np.ascontiguousarray(active, dtype=np.int8)
    if kc is None:
        kc = coulomb_k()
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    ex = np.zeros(rows.size); ey = np.zeros(rows.size); ez = np.zeros(rows.size)
    lib().or_field_rows(n, _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(z, C.c_double),
                        _ptr(sg, C.c_int8), _ptr(ac, C.c_int8), _ptr(rows, C.c_int64),
                        rows.size, kc, eps, 1 if parallel else 0,
                        _ptr(ex, C.c_double), _ptr(ey, C.c_double), _ptr(ez, C.c_double))
    return np.stack([ex, ey, ez], axis=1)


def pixel_of(params: _Params, x, y):
    ix = C.c_int32(); iy = C.c_int32()
    ok = lib().or_pixel_of(C.byref(params), x, y, C.byref(ix), C.byref(iy))
    return (ix.value, iy.value) if ok else None


def bin_positions(params: _Params, x, y):
    x = np.ascontiguousarray(x, dtype=np.float64); y = np.ascontiguousarray(y, dtype=np.float64)
    pix = np.zeros(params.grid_n * params.grid_n, dtype=np.int32)
    out = C.c_int64(0)
    lib().or_bin(C.byref(params), x.size, _ptr(x, C.c_double), _ptr(y, C.c_double),
                 _ptr(pix, C.c_int32), C.byref(out))
    return pix.reshape(params.grid_n, params.grid_n), out.value


def init_event(params: _Params, ev: dict):
    keep = []
    e = make_event(ev, keep)
    n = lib().or_event_carriers(C.byref(params), C.byref(e))
    x = np.zeros(n); y = np.zeros(n); z = np.zeros(n); s = np.zeros(n, dtype=np.int8)
    lib().or_init_event(C.byref(params), C.byref(e), _ptr(x, C.c_double), _ptr(y, C.c_double),
                        _ptr(z, C.c_double), _ptr(s, C.c_int8))
    return np.stack([x, y, z], axis=1), s


# ----------------------------------------------------------------------------
# Whole events (Algorithm 1)
# ----------------------------------------------------------------------------
@dataclass
class EventResult:
    status: int
    n_steps: int
    n_collected: int
    n_outside: int
    n_lost: int
    interactions: int
    pixels: np.ndarray
    final_xy: np.ndarray
    retire_step: np.ndarray
    pos: np.ndarray
    state: np.ndarray
    sign: np.ndarray
    induced: np.ndarray = None    # charge on the collecting surface after each step (e)
    induced_px: np.ndarray = None  # (steps, 3, 3): charge on the 3 x 3 centre pixels (e)


INDUCED_CAPACITY = 20000   # steps of the induced-charge record the oracle keeps


def _alloc_result(params, n, induced_px=False):
    cap = int(min(params.max_steps, INDUCED_CAPACITY)) or 1
    bufs = dict(induced=np.zeros(cap), induced_px=np.zeros(9 * cap) if induced_px else None,
                pixels=np.zeros(params.grid_n * params.grid_n, dtype=np.int32),
                fx=np.zeros(max(n, 1)), fy=np.zeros(max(n, 1)),
                rs=np.zeros(max(n, 1), dtype=np.int32), pos=np.zeros(3 * max(n, 1)),
                st=np.zeros(max(n, 1), dtype=np.int8), sg=np.zeros(max(n, 1), dtype=np.int8))
    r = _Result()
    r.pixels = _ptr(bufs["pixels"], C.c_int32)
    r.final_x = _ptr(bufs["fx"], C.c_double)
    r.final_y = _ptr(bufs["fy"], C.c_double)
    r.retire_step = _ptr(bufs["rs"], C.c_int32)
    r.pos_out = _ptr(bufs["pos"], C.c_double)
    r.state_out = _ptr(bufs["st"], C.c_int8)
    r.sign_out = _ptr(bufs["sg"], C.c_int8)
    r.induced = _ptr(bufs["induced"], C.c_double)
    r.induced_capacity = bufs["induced"].size
    r.induced_px = _ptr(bufs["induced_px"], C.c_double)
    return r, bufs


def _wrap(params, r, bufs, n):
    return EventResult(
        status=r.status, n_steps=r.n_steps, n_collected=r.n_collected, n_outside=r.n_outside,
        n_lost=r.n_lost, interactions=r.interactions,
        pixels=bufs["pixels"].reshape(params.grid_n, params.grid_n).copy(),
        final_xy=np.stack([bufs["fx"][:n], bufs["fy"][:n]], axis=1),
        retire_step=bufs["rs"][:n].copy(), pos=bufs["pos"][:3 * n].reshape(n, 3).copy(),
        state=bufs["st"][:n].copy(), sign=bufs["sg"][:n].copy(),
        induced=bufs["induced"][:min(r.n_steps, bufs["induced"].size)].copy(),
        induced_px=(None if bufs["induced_px"] is None else
                    bufs["induced_px"].reshape(-1, 3, 3)[:min(r.n_steps, r.induced_capacity)]
                    .copy()))


def run_events(params: _Params, events: list[dict], induced_px: bool = False) -> list[EventResult]:
    """Run independent events (OpenMP across events when there are several).
    induced_px: also record the charge induced on the 3 x 3 pixels around the
    grid's centre pixel after every step (pixel weighting potentials)."""
    keep = []
    evs = (_Event * max(len(events), 1))()
    for k, ev in enumerate(events):
        evs[k] = make_event(ev, keep)
    results = (_Result * max(len(events), 1))()
    sizes, bufl = [], []
    for k in range(len(events)):
        n = lib().or_event_carriers(C.byref(params), C.byref(evs[k]))
        r, b = _alloc_result(params, n, induced_px)
        results[k] = r
        sizes.append(n); bufl.append(b)
    if len(events) == 1:
        lib().or_run_event(C.byref(params), C.byref(evs[0]), C.byref(results[0]), 1)
    elif events:
        lib().or_run_events(C.byref(params), evs, len(events), results)
    return [_wrap(params, results[k], bufl[k], sizes[k]) for k in range(len(events))]


def run_event(params: _Params, ev: dict, induced_px: bool = False) -> EventResult:
    return run_events(params, [ev], induced_px)[0]


def step(params: _Params, seed: int, event_id: int, step_index: int, pos, sign, state):
    """One time step of Algorithm 1 from the given FP64 positions (n x 3),
    signs and states (carriers laid out as init_event does): the repulsion
    field from these positions, the moves with the diffusion normals of step
    `step_index`, then the boundaries.  Returns (new positions, new states)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    x = np.ascontiguousarray(pos[:, 0]); y = np.ascontiguousarray(pos[:, 1])
    z = np.ascontiguousarray(pos[:, 2])
    sg = np.ascontiguousarray(sign, dtype=np.int8)
    st = np.array(state, dtype=np.int8)
    lib().or_step(C.byref(params), int(seed), int(event_id), int(step_index), n,
                  _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(z, C.c_double),
                  _ptr(sg, C.c_int8), _ptr(st, C.c_int8), 1)
    return np.stack([x, y, z], axis=1), st


WEIGHT_PAIRS = 32   # image pairs the oracle sums before the two-term tail


def rect_solid_angle(x, y, zeta, rect) -> float:
    """Half-space potential (solid angle / 2 pi, signed like zeta) of the
    rectangle rect = (x1, x2, y1, y2) on the plane zeta = 0 seen from (x, y, zeta)."""
    return lib().or_rect_solid_angle(float(x), float(y), float(zeta), *map(float, rect))


def weighting_potential(x, y, z, rect, thickness_um, n_pairs: int = WEIGHT_PAIRS) -> float:
    """Weighting potential of the pixel rect = (x1, x2, y1, y2) on the
    collecting surface z = 0 of a sensor of thickness H, at (x, y, z)."""
    return lib().or_weighting_potential(float(x), float(y), float(z), *map(float, rect),
                                        float(thickness_um), int(n_pairs))


def window_potentials(params: _Params, x, y, z) -> np.ndarray:
    """Weighting potentials (3 x 3, [row][col]) of the pixels around the grid's
    centre pixel at (x, y, z), as the transport run records them."""
    out = np.zeros(9)
    lib().or_window_potentials(C.byref(params), float(x), float(y), float(z), _ptr(out, C.c_double))
    return out.reshape(3, 3)


def max_threads() -> int:
    return lib().or_max_threads()


def count_interactions(retire_step: np.ndarray, n_steps: int) -> int:
    """Sum over steps of N_act (N_act - 1), from per-carrier retire steps."""
    rs = np.asarray(retire_step, dtype=np.int64)
    total = 0
    for k in range(n_steps):
        a = int(np.count_nonzero((rs == -2) | (rs >= k)))
        total += a * (a - 1)
    return total

