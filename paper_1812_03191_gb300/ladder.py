"""Heating-force differencing over a ladder of nested levels (Sec. 4.1, Eq. 5, Eq. 24).

The heating force is the difference between the force on a luminous perturber and
on a cold one in otherwise identical runs (Eq. 5).  For every level count of the
ladder a hot run (luminosity L) and a cold run (L = 0) are admitted to one pool and
stepped together with the same fixed time step, so their force histories share
their time points; the heating force is their difference along the perturber's
motion.  Adding a level halves the finest cell: in the supersonic regime the
heating force then grows by (gamma - 1) GM L ln 2 / (chi V^2) (Eq. 24, from the
logarithm of Eq. 13), independent of the level count.

Set-up (Sec. 4 and 4.1): gamma = 1.4, rho0 = c_s = 1, GM = 1e-3, chi = 0.1,
L = 2e-4, no softening, the energy L dt split over the eight cells around the
perturber's vertex, a coarse box [-l, l]^3 with l = 100 lambda and
lambda = chi / (gamma V) (Eq. 7), n = 32 cells per level and axis, so that 6 levels
reach the paper's finest cell of 25/128 lambda, run to 100 tau with
tau = chi / (gamma^2 V^2) (Eq. 9).  quadrant=True runs the paper's own 16 x 16 x 32
quadrant meshes over [0, l]^2 x [-l, l] with mirror planes x = 0 and y = 0 and the
flow along +z (the same cells, a quarter of the work).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import binding
from . import inputs as I


def lam(chi, gamma, V):
    """cut-off length of the hot plume (Eq. 7)"""
    return chi / (gamma * V)


def tau(chi, gamma, V):
    """settling time of the heating force (Eq. 9)"""
    return chi / (gamma * gamma * V * V)


def eq24_increment(gamma, GM, L, chi, V):
    """growth of the supersonic heating force when the resolution doubles (Eq. 24)"""
    return (gamma - 1.0) * GM * L * math.log(2.0) / (chi * V * V)


def eq8_force(gamma, GM, L, chi, cs=1.0):
    """low-Mach heating force M a_{0,L,chi} of the linear steady state (Eq. 8)"""
    return gamma * (gamma - 1.0) * GM * L / (2.0 * chi * cs * cs)


def h_fraction(rp):
    """share of the low-Mach heating force from within r' = r / 2 lambda (Eq. 23)"""
    return (1.0 - 2.0 * rp - math.exp(-2.0 * rp)) / (2.0 * rp * rp) + 1.0


def fixed_dt(n_levels, n, half, params, safety=0.8):
    """coarse step from the Courant and diffusion limits of every level (Eq. 55 with
    xi = 2), for the background flow, times a safety factor for the perturbation"""
    V = params["mach"] * params["cs"]
    best = math.inf
    for l in range(n_levels):
        dx = 2.0 * half / n / 2**l
        lim = params["cfl"] * dx / (params["cs"] + V)
        if params["chi"] > 0:
            lim = min(lim, params["cfl_diff"] * dx * dx / (6.0 * params["chi"]))
        best = min(best, lim * 2**l)
    return safety * best


def setup(mach=3.0, chi=0.1, GM=1e-3, L=2e-4, gamma=1.4, n=32, box_lambdas=100.0,
          quadrant=False):
    """parameter dicts of the hot and cold runs and the coarse half-width; with
    quadrant=True the flow is along +z and the planes x = 0, y = 0 are mirror planes
    (the paper's n/2 x n/2 x n quadrant meshes, Sec. 3.4)"""
    half = box_lambdas * lam(chi, gamma, mach)
    base = I.base_params(gamma=gamma, rho0=1.0, cs=1.0, mach=mach, GM=GM, eps=0.0, chi=chi,
                         L=0.0, lum_sigma=0.0)
    if quadrant:
        base = I.quadrant(n=n, n_levels=1, half=half, mach=mach, gamma=gamma, GM=GM, eps=0.0,
                          chi=chi, L=0.0, lum_sigma=0.0)["params"]
    hot = dict(base, L=L)
    cold = dict(base, L=0.0)
    return hot, cold, half


def geometry(n, half, quadrant):
    """cells per axis and box of every level: a full box of n^3, or the quadrant's
    n/2 x n/2 x n over [0, l]^2 x [-l, l] (the same cells)"""
    if quadrant:
        return (n // 2, n // 2, n), (0.0, 0.0, -half), (half,) * 3
    return (n, n, n), (-half,) * 3, (half,) * 3


def low_mach(mach=0.1, n_levels=6, chi=0.1, GM=1e-3, L=2e-4, gamma=1.4, n=32,
             t_end_taus=100.0, precision=binding.DF_FP32_STATE, sample_every=8,
             quadrant=False):
    """One hot/cold pair at low Mach (Sec. 4.1.1): the heating force against Eq. 8
    times the share h(r'_max) - h(r'_min) of Eq. 23 that the box (r'_max = l / 2
    lambda) and the finest cell (r'_min = dx / 2 lambda) can hold."""
    out = run(levels=(n_levels,), mach=mach, chi=chi, GM=GM, L=L, gamma=gamma, n=n,
              t_end_taus=t_end_taus, precision=precision, sample_every=sample_every,
              quadrant=quadrant)
    lam_ = lam(chi, gamma, mach)
    r = out["runs"][n_levels]
    rp_min = r["finest_dx"] / (2.0 * lam_)
    rp_max = out["half"] / (2.0 * lam_)
    share = h_fraction(rp_max) - h_fraction(rp_min)
    out["eq8_force"] = eq8_force(gamma, GM, L, chi)
    out["eq23_share"] = share
    out["expected"] = out["eq8_force"] * share
    out["ratio"] = r["final"] / out["expected"]
    return out


def pairs(levels, pa, pb, half, n=32, t_end=1.0, precision=binding.DF_FP32_STATE,
          sample_every=8, budget=32 << 30, quadrant=False):
    """Runs with parameters pa and pb for every level count, one pool, the same fixed
    coarse step per level count (from pa's limits); the history of F_a - F_b along
    the motion and its final value (mean over the last tenth of the run)."""
    nn, lo, hi = geometry(n, half, quadrant)
    pool = binding.Pool(budget, precision=precision)
    runs = {}
    for nl in levels:
        dt = fixed_dt(nl, n, half, pa)
        sa = pool.admit(nl, nn, lo, hi, I.DEFAULT_G, dict(pa, dt_fixed=dt))
        sb = pool.admit(nl, nn, lo, hi, I.DEFAULT_G, dict(pb, dt_fixed=dt))
        if sa is None or sb is None:
            raise RuntimeError("the runs do not fit the pool budget")
        runs[nl] = dict(slots=(sa, sb), dt=dt, steps=0, t=[], F=[], done=False)
    d = np.asarray(pa["flow_dir"], dtype=float)
    d = d / np.linalg.norm(d)
    t0 = time.perf_counter()
    cell_updates = 0
    while not all(p["done"] for p in runs.values()):
        pool.step(sample_every)
        q = pool.query()
        for nl, p in runs.items():
            if p["done"]:
                continue
            sa, sb = p["slots"]
            p["steps"] += sample_every
            cell_updates += 2 * sample_every * nn[0] * nn[1] * nn[2] * (2**nl - 1)
            if q[sa, 5] != 0 or q[sb, 5] != 0:
                raise RuntimeError(f"{nl} levels: unhealthy state")
            if q[sa, 3] != q[sb, 3]:
                raise RuntimeError("paired runs out of step")
            Fa = -float(np.dot(q[sa, :3], d))
            Fb = -float(np.dot(q[sb, :3], d))
            p["t"].append(float(q[sa, 3]))
            p["F"].append(Fa - Fb)
            if q[sa, 3] >= t_end:
                p["done"] = True
                pool.release(sa)
                pool.release(sb)
    wall = time.perf_counter() - t0
    pool.close()
    out = dict(levels=list(levels), t_end=t_end, half=half, wall_s=wall,
               cell_updates=cell_updates, runs={})
    for nl, p in runs.items():
        t = np.array(p["t"])
        F = np.array(p["F"])
        tail = t >= 0.9 * t[-1]
        out["runs"][nl] = dict(dt=p["dt"], steps=p["steps"], t=t.tolist(), F=F.tolist(),
                               final=float(F[tail].mean()),
                               finest_dx=2.0 * half / n / 2**(nl - 1))
    return out


def run(levels=(4, 5, 6, 7), mach=3.0, chi=0.1, GM=1e-3, L=2e-4, gamma=1.4, n=32,
        t_end_taus=100.0, precision=binding.DF_FP32_STATE, sample_every=4,
        budget=32 << 30, quadrant=False):
    """Heating force (hot minus cold run, Eq. 5) for every level count, stepped to
    t_end = t_end_taus * tau, with the increments between successive level counts
    and the Eq. 24 prediction."""
    hot, cold, half = setup(mach, chi, GM, L, gamma, n, quadrant=quadrant)
    out = pairs(levels, hot, cold, half, n=n, t_end=t_end_taus * tau(chi, gamma, mach),
                precision=precision, sample_every=sample_every, budget=budget,
                quadrant=quadrant)
    out["predicted_increment"] = eq24_increment(gamma, GM, L, chi, mach)
    for r in out["runs"].values():
        r["F_heating"] = r.pop("F")
    final = {nl: r["final"] for nl, r in out["runs"].items()}
    out["increments"] = {f"{a}->{b}": final[b] - final[a] for a, b in zip(levels, levels[1:])}
    return out


def cold_thermal(mach=0.1, n_levels=6, chi=0.1, GM=1e-3, gamma=1.4, n=32, t_end_taus=100.0,
                 precision=binding.DF_FP32_STATE, sample_every=8, quadrant=False):
    """Cold thermal force (Sec. 4.2): a cold perturber with thermal diffusion minus the
    same in an adiabatic gas, at low Mach, against -(gamma - 1)/2 F0 (Eq. 48, Eq. 50,
    Eq. 51) times the Eq. 23 share of the box (the perturbation is that of a heat sink
    of luminosity -L_c, Eq. 49).  quadrant=True: the paper's quadrant meshes and
    boundaries (Sec. 3.4), as in `setup`."""
    _, cold, half = setup(mach, chi, GM, 0.0, gamma, n, quadrant=quadrant)
    adiabatic = dict(cold, chi=0.0)
    out = pairs((n_levels,), cold, adiabatic, half, n=n,
                t_end=t_end_taus * tau(chi, gamma, mach), precision=precision,
                sample_every=sample_every, quadrant=quadrant)
    lam_ = lam(chi, gamma, mach)
    r = out["runs"][n_levels]
    share = h_fraction(half / (2.0 * lam_)) - h_fraction(r["finest_dx"] / (2.0 * lam_))
    F0 = 4.0 * math.pi * GM * GM
    out["eq51_force"] = -(gamma - 1.0) / 2.0 * F0
    out["eq23_share"] = share
    out["expected"] = out["eq51_force"] * share
    out["ratio"] = r["final"] / out["expected"]
    return out


def paper_cold_thermal(mach=0.1, n_levels=10, chi=0.1, GM=1e-3, gamma=1.4, n=64,
                       box_lambdas=3200.0, t_end_taus=100.0,
                       precision=binding.DF_FP32_STATE, sample_every=8):
    """Cold thermal force (Sec. 4.2) in the paper's own geometry for it: the quadrant
    domain with mirror planes x = 0 and y = 0, a ground of n x n x 2n cells and
    levels of n/2 x n/2 x n, the first over a quarter of the ground (Sec. 4.1.1),
    l = box_lambdas lambda.  A cold perturber with diffusion minus the same in an
    adiabatic gas, both stepped with the same fixed coarse step to t_end_taus tau,
    against -(gamma - 1)/2 F0 (Eq. 51) times the Eq. 23 share of the box and the
    finest cell.  The two runs are contexts, stepped alternately."""
    lam_ = lam(chi, gamma, mach)
    half = box_lambdas * lam_
    q = I.quadrant(n=n, n_levels=n_levels, half=half, mach=mach, quarter=True, GM=GM,
                   chi=chi, L=0.0, gamma=gamma)
    cold = q["params"]
    adiabatic = dict(cold, chi=0.0)
    dt = fixed_dt(n_levels, 2 * n, half, cold)  # the ground's cell is half / n
    sims = [binding.Sim(n_levels, q["n"], q["lo"], q["hi"], q["G"], dict(p, dt_fixed=dt),
                        precision=precision, n0=q["n0"]) for p in (cold, adiabatic)]
    d = np.asarray(cold["flow_dir"], dtype=float)
    t_end = t_end_taus * tau(chi, gamma, mach)
    ts, F = [], []
    t0 = time.perf_counter()
    t = 0.0
    steps = 0
    while t < t_end:
        for s in sims:
            s.step(sample_every)
        steps += sample_every
        fa, fb = (-float(np.dot(s.force()[0], d)) for s in sims)
        t = sims[0].status()[0]
        if sims[0].status()[2] or sims[1].status()[2]:
            raise RuntimeError("unhealthy state")
        ts.append(t)
        F.append(fa - fb)
    wall = time.perf_counter() - t0
    for s in sims:
        s.close()
    ts, F = np.array(ts), np.array(F)
    finest_dx = half / n / 2 ** (n_levels - 1)
    share = h_fraction(half / (2.0 * lam_)) - h_fraction(finest_dx / (2.0 * lam_))
    F0 = 4.0 * math.pi * GM * GM
    final = float(F[ts >= 0.9 * ts[-1]].mean())
    expected = -(gamma - 1.0) / 2.0 * F0 * share
    return dict(mach=mach, n_levels=n_levels, half=half, dt=dt, steps=steps, t=ts.tolist(),
                F=F.tolist(), final=final, finest_dx=finest_dx, eq23_share=share,
                eq51_force=-(gamma - 1.0) / 2.0 * F0, expected=expected,
                ratio=final / expected, wall_s=wall)

