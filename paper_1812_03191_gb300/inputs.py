"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's.

This module holds parameter sets and random-number draws only: no step of the
solver's arithmetic.  Both sides receive the same dicts and arrays from here.

Workloads (all synthetic; the paper uses no dataset):
  * ``single_mesh``   -- one 32^3 level on [-4,4]^3, Mach 0.5 wind along -x,
                         GM=0.01, softening 2 cells, chi=1, L=0 (Sec. 3.4 set-up,
                         transposed to a full box with upstream injection).
  * ``nested``        -- 3 levels of 64^3 on [-8,8]^3, ratio 2, Mach 0.5, GM=0.01,
                         chi=1, luminosity L_c = 4 pi GM rho0 chi / gamma (Eq. 49)
                         deposited as a Gaussian of sigma = softening = 2 finest cells.
  * ``precision``     -- 5 levels of 128^3 on [-16,16]^3, Mach 1.2, same physics.
  * ``batched``       -- 64 independent runs (seed 1812031910): levels uniform in 2..4,
                         per-run mesh from {32,48,64,96}^3, Mach log-uniform in
                         [0.1,3], chi log-uniform in [0.3,3], GM=0.01, L = 0 or L_c(chi)
                         with probability 1/2, coarse box [-8,8]^3.
  * ``requests``      -- the serving stream (seed 1812031911): Poisson arrivals, levels
                         2..6, mesh from {48,64,96,128}^3, Mach uniform in [0.05,4],
                         chi log-uniform in [0.3,3], L on/off.
"""
from __future__ import annotations

import math

import numpy as np

# boundary types (same numbering on both sides of the boundary)
BC_PERIODIC, BC_OUTFLOW, BC_INFLOW, BC_REFLECT = 0, 1, 2, 3

DEFAULT_G = 8      # ghost layers: twice the reach of one level step (measured: 4)
DEFAULT_BAND = 5   # CommMean band in coarse cells (smallest band with exact results)


def base_params(**over) -> dict:
    p = dict(
        gamma=5.0 / 3.0, rho0=1.0, cs=1.0, mach=0.5, flow_dir=(-1.0, 0.0, 0.0),
        GM=0.01, eps=0.5, chi=1.0, L=0.0, lum_sigma=0.0,
        cfl=0.44, cfl_diff=0.44, dt_fixed=0.0, xi_mode=0,
        bc=(BC_OUTFLOW, BC_INFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW),
        diff_face_rho=0, hydro_on=1, band=DEFAULT_BAND, av_c2=0.0,
    )
    p.update(over)
    return p


def critical_luminosity(GM, rho0, chi, gamma):
    """L_c of Eq. 49 (used only to choose the luminosity of a workload)."""
    return 4.0 * math.pi * GM * rho0 * chi / gamma


def wind_bcs(flow_dir):
    """Injection on the upstream face, outflow elsewhere."""
    bc = [BC_OUTFLOW] * 6
    ax = int(np.argmax(np.abs(flow_dir)))
    bc[2 * ax + (1 if flow_dir[ax] < 0 else 0)] = BC_INFLOW
    return tuple(bc)


def single_mesh():
    return dict(
        name="single_mesh_32^3_fp64",
        n_levels=1, n=32, lo=(-4.0,) * 3, hi=(4.0,) * 3, G=DEFAULT_G, steps=20,
        params=base_params(eps=0.5),
    )


def nested(n=64, n_levels=3, half=8.0, mach=0.5, steps=1000):
    dx_f = 2 * half / n / 2 ** (n_levels - 1)
    eps = 2 * dx_f
    p = base_params(mach=mach, eps=eps, lum_sigma=eps,
                    L=critical_luminosity(0.01, 1.0, 1.0, 5.0 / 3.0))
    return dict(
        name=f"nested_{n_levels}x{n}^3_fp64",
        n_levels=n_levels, n=n, lo=(-half,) * 3, hi=(half,) * 3, G=DEFAULT_G, steps=steps,
        params=p,
    )


def precision(n=128, n_levels=5, half=16.0):
    cfg = nested(n=n, n_levels=n_levels, half=half, mach=1.2, steps=50)
    cfg["name"] = f"precision_{n_levels}x{n}^3"
    return cfg


def quadrant(n=32, n_levels=6, half=8.0, mach=3.0, quarter=False, **over):
    """The set-up of Sec. 3.4 on its quadrant domain: flow along +z, the perturber
    at the corner vertex of x, y >= 0; every level spans [0, l 2^-k]^2 x
    [-l 2^-k, l 2^-k] with n/2 x n/2 x n cells.  The planes x = 0 and y = 0 are
    mirror planes (the run stands for the whole domain, whose force it reports);
    the outer x and y faces reflect too, and both z faces hold the background.
    quarter=True: the low-Mach hierarchy of Sec. 4.1.1, a ground of n x n x 2n cells
    over [0, l]^2 x [-l, l] and levels of n/2 x n/2 x n, the first over a quarter of
    the ground's extent (n0 in the returned dict)."""
    p = base_params(gamma=1.4, mach=mach, flow_dir=(0.0, 0.0, 1.0), eps=0.0,
                    bc=(BC_REFLECT,) * 4 + (BC_INFLOW,) * 2)
    p.update(over)
    nf = (n // 2, n // 2, n)
    n0 = (n, n, 2 * n) if quarter else nf
    return dict(
        name=f"quadrant_{n_levels}x{n // 2}x{n // 2}x{n}" + ("_quarter" if quarter else ""),
        n_levels=n_levels, n=nf, n0=n0, lo=(0.0, 0.0, -half), hi=(half,) * 3,
        G=DEFAULT_G, params=p,
    )


def smooth_perturbation(shape, seed, amp, n_modes=4):
    """Sum of a few random low-wavenumber periodic modes (shape = (nz, ny, nx))."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                          indexing="ij")
    out = np.zeros(shape)
    for _ in range(n_modes):
        kx, ky, kz = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        out += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * x + ky * y + kz * z) + ph)
    return amp * out / n_modes


def random_state(n, n_levels, seed, amp=1e-2):
    """Per-level multiplicative/additive perturbations of (rho, e, vx, vy, vz)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_levels):
        out.append([rng.standard_normal((n, n, n)) * amp for _ in range(5)])
    return out


def _run_params(rng, mach, chi, lum_on, n, n_levels, half):
    dx_f = 2 * half / n / 2 ** (n_levels - 1)
    eps = 2 * dx_f
    L = critical_luminosity(0.01, 1.0, chi, 5.0 / 3.0) if lum_on else 0.0
    return base_params(mach=mach, chi=chi, GM=0.01, eps=eps, L=L,
                       lum_sigma=eps if lum_on else 0.0)


def batched(n_runs=64, seed=1812031910, half=8.0, sizes=(32, 48, 64, 96), levels=(2, 3, 4)):
    """Independent runs of the batched form (see the module docstring)."""
    rng = np.random.default_rng(seed)
    runs = []
    for _ in range(n_runs):
        nl = int(rng.choice(levels))
        n = int(rng.choice(sizes))
        mach = float(np.exp(rng.uniform(np.log(0.1), np.log(3.0))))
        chi = float(np.exp(rng.uniform(np.log(0.3), np.log(3.0))))
        lum_on = bool(rng.random() < 0.5)
        runs.append(dict(n_levels=nl, n=n, lo=(-half,) * 3, hi=(half,) * 3, G=DEFAULT_G,
                         params=_run_params(rng, mach, chi, lum_on, n, nl, half)))
    return runs


def requests(n_req, rate, seed=1812031911, half=8.0, sizes=(48, 64, 96, 128),
             levels=(2, 3, 4, 5, 6)):
    """Serving stream: (arrival time, run spec) with Poisson arrivals of `rate` per s."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_req):
        t += float(rng.exponential(1.0 / rate))
        nl = int(rng.choice(levels))
        n = int(rng.choice(sizes))
        mach = float(rng.uniform(0.05, 4.0))
        chi = float(np.exp(rng.uniform(np.log(0.3), np.log(3.0))))
        lum_on = bool(rng.random() < 0.5)
        out.append((t, dict(n_levels=nl, n=n, lo=(-half,) * 3, hi=(half,) * 3, G=DEFAULT_G,
                            params=_run_params(rng, mach, chi, lum_on, n, nl, half))))
    return out
