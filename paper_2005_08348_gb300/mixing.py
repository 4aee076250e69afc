"""Mixing of a two-type bilayer measured as in arXiv:2005.08348 Sec. 4.

The observable is the highest peak of the in-plane g(r) of one lipid type's
head beads (``mdas_head_rdf``), followed against force evaluations from a
phase-separated start and fitted with a + b exp(-x / tau).  Three samplers
follow the protocols of Sec. 3:

- plain MD;
- MC-MD: one exchange trial after every 2000 MD steps, 2001 force
  evaluations per attempt;
- MDAS: 2000 MD steps, then an alchemical trajectory of 1000 steps with
  lambda changed every 10 steps (100 lambda values), 3000 force evaluations
  per attempt.

Force evaluations are counted as the paper counts them: MD and alchemical
steps, one per MC trial.  The bilayer is a synthetic stand-in (seeded bead
parameters, not Martini's), so the rates are this model's and not the
paper's DPPC/DPPS numbers.

Run on a GPU:  python -m paper_2005_08348_gb300.mixing [--evals N] [--every N] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import mdas, synth

MD_BETWEEN = 2000            # MD steps between two exchange attempts
AT_LAMBDAS, AT_STEPS = 100, 10   # MDAS: lambda values, MD steps per value


def bilayer(nx: int = 20, ny: int = 20, seed: int = 1006) -> synth.Membrane:
    """2 nx ny lipids (800 by default), two types 1:1 in stripes along x, 5 nm of water."""
    return synth.membrane(nx, ny, n_lipid_types=2, fracs=[0.5, 0.5], water_thickness=5.0, seed=seed,
                          layout="separated")


def g_of_r(counts, n_heads, box, r_max):
    """g(r) from head-pair counts: per leaflet [2, n_bins] and over both
    leaflets [n_bins], each count over the pairs an ideal 2D gas of the same
    heads would put in that annulus; r at the bin centres."""
    counts = np.asarray(counts, np.float64)
    nb = counts.shape[1]
    dr = r_max / nb
    k = np.arange(nb, dtype=np.float64)
    shell = math.pi * ((k + 1) ** 2 - k ** 2) * dr * dr / (box[0] * box[1])
    pairs = np.array([0.5 * n * (n - 1) for n in n_heads], np.float64)
    ideal = pairs[:, None] * shell[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(ideal > 0, counts / np.where(ideal > 0, ideal, 1.0), 0.0)
        tot = ideal.sum(0)
        both = np.where(tot > 0, counts.sum(0) / np.where(tot > 0, tot, 1.0), 0.0)
    return (k + 0.5) * dr, g, both


def max_g(system, lipid_type=1, head_k=1, r_max=3.0, n_bins=20) -> float:
    c, nh = system.head_rdf(lipid_type, head_k, r_max, n_bins)
    return float(g_of_r(c, nh, system.box()[0], r_max)[2].max())   # the current box (pressure coupling)


def exp_fit(x, y):
    """Least-squares y = a + b exp(-x / tau); None when the fit fails."""
    from scipy.optimize import curve_fit
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if len(x) < 4:
        return None
    f = lambda t, a, b, tau: a + b * np.exp(-t / tau)
    try:
        p, _ = curve_fit(f, x, y, p0=(y[-1], y[0] - y[-1], max(x[-1] / 3.0, 1.0)), maxfev=20000)
    except Exception:
        return None
    a, b, tau = (float(v) for v in p)
    if not (tau > 0 and math.isfinite(tau)):
        return None
    return dict(a=a, b=b, tau=tau)


def exp_fit_plateau(x, y, a):
    """Least-squares y = a + b exp(-x / tau) with the plateau a given."""
    from scipy.optimize import curve_fit
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    f = lambda t, b, tau: a + b * np.exp(-t / tau)
    try:
        p, _ = curve_fit(f, x, y, p0=(max(y[0] - a, 1e-3), max(x[-1] / 3.0, 1.0)), maxfev=20000)
    except Exception:
        return None
    b, tau = (float(v) for v in p)
    return dict(a=float(a), b=b, tau=tau) if tau > 0 and math.isfinite(tau) else None


def speedups(res: dict) -> dict:
    """tau(MD) / tau(method), from free fits and from fits sharing the mixed
    plateau (the mean plateau of the exchange samplers' free fits), which
    stays defined when MD has not come near it within the sampled window."""
    out = {}
    free = {k: (res[k]["fit"] or {}).get("tau") for k in res}
    out["free_fit"] = {k: free["md"] / free[k] if free["md"] and free[k] else None for k in ("mcmd", "mdas")}
    pl = [res[k]["fit"]["a"] for k in ("mcmd", "mdas") if res[k]["fit"]]
    if pl:
        a = float(np.mean(pl))
        t = {k: (exp_fit_plateau(res[k]["force_evaluations"], res[k]["max_g"], a) or {}).get("tau") for k in res}
        out["common_plateau"] = dict(plateau=a, tau=t, speedup={k: t["md"] / t[k] if t["md"] and t[k] else None
                                                               for k in ("mcmd", "mdas")})
    return out


def run(kind: str, m, evals: int, every: int, melt: int = 20000, precision: str = "fp32") -> dict:
    """One sampler until `evals` force evaluations, max g(r) of type-1 head
    beads at least every `every` evaluations.  The start is the membrane's
    lattice melted by `melt` MD steps with the types fixed (not counted): the
    stripes stay, the lattice order goes."""
    s = mdas.System(m, precision=precision)
    s.md_steps(melt, swap_every=0)
    xs, ys = [0], [max_g(s)]
    done, nxt = 0, every
    t0 = time.perf_counter()
    while done < evals:
        if kind == "md":
            s.md_steps(MD_BETWEEN, swap_every=0)
            done += MD_BETWEEN
        elif kind == "mcmd":
            s.md_steps(MD_BETWEEN, swap_every=MD_BETWEEN)
            done += MD_BETWEEN + 1
        elif kind == "mdas":
            s.md_steps(MD_BETWEEN, swap_every=0)
            s.alchemical_move(1, AT_LAMBDAS, AT_STEPS)
            done += MD_BETWEEN + AT_LAMBDAS * AT_STEPS
        else:
            raise ValueError(kind)
        if done >= nxt:
            xs.append(done)
            ys.append(max_g(s))
            nxt += every
    c = s.counters()
    out = dict(kind=kind, force_evaluations=xs, max_g=ys, fit=exp_fit(xs, ys), seconds=time.perf_counter() - t0)
    if kind == "mcmd":
        out.update(attempts=c["trials"], accepted=c["accepted"], null=c["null_trials"])
    if kind == "mdas":
        out.update(attempts=c["moves"], accepted=c["moves_accepted"])
    s.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--evals", type=int, default=2_000_000)
    ap.add_argument("--every", type=int, default=40_000)
    ap.add_argument("--melt", type=int, default=20_000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    m = bilayer()
    res = {k: run(k, m, a.evals, a.every, a.melt) for k in ("md", "mcmd", "mdas")}
    speed = speedups(res)
    summary = dict(workload=f"{m.n_lipids} lipids, 2 types 1:1 in stripes, {m.n_beads} beads",
                   observable="max g(r) of type-1 head beads (second head bead), in-plane, both leaflets, "
                              "0.15 nm bins to 3 nm", melt_md_steps=a.melt,
                   speedup_vs_md=speed, runs=res)
    line = json.dumps(summary)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")
    print(line)


if __name__ == "__main__":
    main()
