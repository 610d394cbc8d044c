"""Seeded synthetic workloads shaped like the paper's (arXiv 2506.09712) simulation sets.

This module is the one piece shared by the FP64 oracle and the CUDA path: it
produces *inputs* only -- sensor presets, event descriptors (seed, id,
energy, absorption depth, entry point) and arrival times -- and holds none of
the transport arithmetic.  The paper's measured data and the silicon X-ray
attenuation tables are not available, so depths are drawn from a truncated
exponential whose attenuation length follows the power law
``lambda(E) = 69.6 um * (E / 8 keV)^2.9`` (an approximation for silicon above
the K edge, stated as an assumption of the synthetic workload).

Presets (sizes from the paper's sensors and energies, Sec. 2 and Sec. 4):

  plain_3keV_100um      8 photons of 3 keV (N = 829), 100 um / 50 V / Vd 20 V,
                        dt 50 ps, 5x5 pixels, sigma 0.5 um
  batch_20keV_320um     64 photons of 20 keV (N = 5525), 320 um / 150 V /
                        Vd 60 V, dt 10 ps, 9x9 pixels
  uneven_5_25keV_450um  10^4 photons, E ~ U(5, 25) keV, 450 um / 200 V /
                        Vd 118.7 V, dt 10 ps, 9x9 pixels
  serve_mix_320um       Poisson arrivals at 2 kHz; 60 % 8 keV, 30 % 17.5 keV,
                        10 % 25 keV; 320 um / 150 V / Vd 60 V, dt 10 ps
  track_200keV_320um    16 straight 150 um electron tracks, 55 250 pairs, both
                        carrier species, 320 um / 200 V / Vd 60 V, dt 5 ps,
                        17x17 pixels
  mip_50um              10 minimum-ionising tracks perpendicular through a
                        50 um sensor (Vd 20 V, 50 V), 80 pairs/um (4000),
                        lateral sigma 1 nm, both species, dt 5 ps; electrons
                        are the collected species (see MIP_MOBILITY)

Each preset also exists as a JSON config under ``configs/`` (``python -m
workloads`` rewrites them); an edited copy can be passed wherever a preset
name is accepted.
"""
from __future__ import annotations

import copy
import json
import os

import numpy as np

MASTER_SEED = 20250611

PHOTON, TRACK, EXPLICIT = 0, 1, 2
HOLES, BOTH = 1, 3
MOB_CT, MOB_CONST = 0, 1

# Caughey-Thomas / Jacoboni-Canali-form hole parameters used for every preset.
HOLE_MOBILITY = dict(model=MOB_CT, mu0_h=480.0, vsat_h=0.95e7, beta_h=1.2)
# Electron parameters (only the two-species track preset uses them): the
# Jacoboni-Canali temperature laws evaluated at 293 K; recalled values.
ELECTRON_MOBILITY = dict(mu0_e=1610.0, vsat_e=1.09e7, beta_e=1.095)


def attenuation_length_um(energy_keV: float) -> float:
    """Synthetic-workload attenuation length of silicon (see module docstring)."""
    return 69.6 * (energy_keV / 8.0) ** 2.9


def _sensor(thickness, bias, vdep, dt_ps, grid_n, species=HOLES):
    return dict(thickness_um=float(thickness), bias_V=float(bias), depletion_V=float(vdep),
                temperature_K=293.0, eps_r=11.7, pitch_um=25.0, grid_n=int(grid_n),
                dt_ps=float(dt_ps), max_steps=200_000, species=species,
                softening_um=1e-6)


# The MIP study collects electrons.  Flipping every charge and the drift field
# leaves the equations of motion unchanged, so the collected species (the
# library's "holes", collected at z = 0) takes the electron parameters and
# the other species (drifting to the back) the hole parameters.
MIP_MOBILITY = dict(model=MOB_CT, mu0_h=ELECTRON_MOBILITY["mu0_e"],
                    vsat_h=ELECTRON_MOBILITY["vsat_e"], beta_h=ELECTRON_MOBILITY["beta_e"],
                    mu0_e=HOLE_MOBILITY["mu0_h"], vsat_e=HOLE_MOBILITY["vsat_h"],
                    beta_e=HOLE_MOBILITY["beta_h"])

PRESETS = {
    "plain_3keV_100um": dict(
        sensor=_sensor(100, 50, 20, 50, 5), mobility=dict(HOLE_MOBILITY),
        n_events=8, energies=[(3.0, 1.0)], sigma_um=0.5),
    "batch_20keV_320um": dict(
        sensor=_sensor(320, 150, 60, 10, 9), mobility=dict(HOLE_MOBILITY),
        n_events=64, energies=[(20.0, 1.0)], sigma_um=-1.0),
    "uneven_5_25keV_450um": dict(
        sensor=_sensor(450, 200, 60.0 * (450.0 / 320.0) ** 2, 10, 9),
        mobility=dict(HOLE_MOBILITY), n_events=10_000, energy_uniform=(5.0, 25.0),
        sigma_um=-1.0),
    "serve_mix_320um": dict(
        sensor=_sensor(320, 150, 60, 10, 9), mobility=dict(HOLE_MOBILITY),
        n_events=2000, energies=[(8.0, 0.6), (17.5, 0.3), (25.0, 0.1)], sigma_um=-1.0,
        rate_hz=2000.0),
    "mip_50um": dict(
        sensor=_sensor(50, 50, 20, 5, 9, species=BOTH), mobility=dict(MIP_MOBILITY),
        n_events=10, track=True, n_pairs=4000, track_len_um=50.0, theta_max_deg=0.0,
        sigma_um=0.001),
    "track_200keV_320um": dict(
        sensor=_sensor(320, 200, 60, 5, 17, species=BOTH),
        mobility=dict(HOLE_MOBILITY, **ELECTRON_MOBILITY), n_events=16, track=True,
        n_pairs=55_250, track_len_um=150.0, theta_max_deg=60.0, sigma_um=0.5),
}


CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")

# JSON workload configs: the preset's dictionary as it is (sensor, mobility,
# event recipe).  Exactly one event recipe: energies (a list of [keV, weight]),
# energy_uniform ([lo, hi] keV) or track (with n_pairs, track_len_um,
# theta_max_deg).
_SENSOR_KEYS = {"thickness_um", "bias_V", "depletion_V", "temperature_K", "eps_r", "pitch_um",
                "grid_n", "dt_ps", "max_steps", "species", "softening_um"}
_OPTIONAL_KEYS = {"rate_hz", "name"}


def _check_config(cfg: dict) -> dict:
    if not isinstance(cfg, dict):
        raise ValueError("a workload config is a JSON object")
    for key in ("sensor", "mobility", "n_events", "sigma_um"):
        if key not in cfg:
            raise ValueError(f"workload config lacks {key!r}")
    missing = _SENSOR_KEYS - set(cfg["sensor"])
    if missing:
        raise ValueError(f"sensor lacks {sorted(missing)}")
    recipes = [k for k in ("energies", "energy_uniform", "track") if k in cfg]
    if len(recipes) != 1:
        raise ValueError("give exactly one of energies, energy_uniform, track")
    known = {"sensor", "mobility", "n_events", "sigma_um", "energies", "energy_uniform", "track",
             "n_pairs", "track_len_um", "theta_max_deg"} | _OPTIONAL_KEYS
    extra = set(cfg) - known
    if extra:
        raise ValueError(f"unknown workload config keys {sorted(extra)}")
    if "track" in cfg:
        for key in ("n_pairs", "track_len_um", "theta_max_deg"):
            if key not in cfg:
                raise ValueError(f"a track workload needs {key!r}")
    if int(cfg["n_events"]) < 0:
        raise ValueError("n_events must be >= 0")
    out = copy.deepcopy(cfg)
    if "energies" in out:
        out["energies"] = [tuple(map(float, e)) for e in out["energies"]]
    if "energy_uniform" in out:
        out["energy_uniform"] = tuple(map(float, out["energy_uniform"]))
    return out


def save_config(name: str, path: str) -> None:
    """Write a preset as a JSON workload config."""
    cfg = dict(copy.deepcopy(PRESETS[name]), name=name)
    with open(path, "w") as fh:
        json.dump(cfg, fh, indent=1, sort_keys=True)
        fh.write("\n")


def load_config(path: str) -> dict:
    """Read and check a JSON workload config (the shape of a preset)."""
    with open(path) as fh:
        return _check_config(json.load(fh))


def _resolve(workload) -> dict:
    if isinstance(workload, dict):
        return _check_config(workload)
    if isinstance(workload, str) and workload.endswith(".json"):
        return load_config(workload)
    return PRESETS[workload]


def preset(name) -> dict:
    """A deep copy of a preset (sensor, mobility and event-generation recipe);
    `name` may also be a config dictionary or the path of a JSON config."""
    return copy.deepcopy(_resolve(name))


def field_switches(repulsion=1, drift=1, diffusion=1, spherical=0) -> dict:
    """Transport-term switches; spherical = 1 selects the simplified spherical
    repulsion model instead of the pairwise field."""
    return dict(repulsion=int(repulsion), drift=int(drift), diffusion=int(diffusion),
                spherical=int(spherical))


def sample_depths(rng: np.random.Generator, energy_keV, thickness_um: float) -> np.ndarray:
    """Absorption depth below the entrance surface: exponential, truncated to [0, H)."""
    e = np.atleast_1d(np.asarray(energy_keV, dtype=np.float64))
    lam = attenuation_length_um(e)
    u = rng.random(e.shape)
    return -lam * np.log1p(-u * (-np.expm1(-thickness_um / lam)))


def make_events(name, n: int | None = None, seed: int = MASTER_SEED,
                first_id: int = 0) -> list[dict]:
    """Event descriptors for a preset, a config dictionary or the path of a
    JSON config (deterministic in `seed` and the ids)."""
    p = _resolve(name)
    s = p["sensor"]
    n = p["n_events"] if n is None else int(n)
    rng = np.random.default_rng([seed, first_id, 0x5EED])
    pitch = s["pitch_um"]
    events = []
    if p.get("track"):
        theta = rng.uniform(0.0, p["theta_max_deg"], n)
        phi = rng.uniform(0.0, 360.0, n)
        xy = rng.uniform(-0.5 * pitch, 0.5 * pitch, (n, 2))
        for k in range(n):
            events.append(dict(seed=seed, event_id=first_id + k, kind=TRACK,
                               energy_keV=200.0, n_pairs=p["n_pairs"], depth_um=0.0,
                               x_um=float(xy[k, 0]), y_um=float(xy[k, 1]),
                               sigma_um=p["sigma_um"], track_len_um=p["track_len_um"],
                               theta_deg=float(theta[k]), phi_deg=float(phi[k])))
        return events
    if "energy_uniform" in p:
        lo, hi = p["energy_uniform"]
        energies = rng.uniform(lo, hi, n)
    else:
        vals = np.array([e for e, _ in p["energies"]])
        probs = np.array([w for _, w in p["energies"]])
        energies = vals[rng.choice(len(vals), size=n, p=probs / probs.sum())]
    depths = sample_depths(rng, energies, s["thickness_um"])
    xy = rng.uniform(-0.5 * pitch, 0.5 * pitch, (n, 2))
    for k in range(n):
        events.append(dict(seed=seed, event_id=first_id + k, kind=PHOTON,
                           energy_keV=float(energies[k]), n_pairs=0,
                           depth_um=float(depths[k]), x_um=float(xy[k, 0]),
                           y_um=float(xy[k, 1]), sigma_um=float(p["sigma_um"])))
    return events


def poisson_arrivals(rate_hz: float, n: int, seed: int = MASTER_SEED) -> np.ndarray:
    """Arrival times in seconds of a Poisson process of the given mean rate."""
    rng = np.random.default_rng([seed, 0xA77])
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


def explicit_event(xyz, sign=None, seed: int = MASTER_SEED, event_id: int = 0) -> dict:
    """An event whose initial carrier positions are given directly."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    ev = dict(seed=seed, event_id=event_id, kind=EXPLICIT, explicit_xyz=xyz,
              n_pairs=int(xyz.shape[0]))
    if sign is not None:
        ev["explicit_sign"] = np.ascontiguousarray(sign, dtype=np.int8)
    return ev


def random_cloud(n: int, sigma_um: float, center=(0.0, 0.0, 0.0), seed: int = 1) -> np.ndarray:
    """A seeded isotropic Gaussian point set (test input for the field kernels)."""
    rng = np.random.default_rng([seed, n, 0xC10D])
    return np.asarray(center) + sigma_um * rng.standard_normal((n, 3))
