"""Seeded synthetic membranes shaped like the paper's Martini bilayers.

This module only places beads and draws seeded parameters; it holds none of
the sampling method's arithmetic (no energies, forces, integrator or
acceptance rule).  Both the CUDA library and the CPU oracle consume what it
returns, so the two sides always start from identical inputs.

Geometry (the paper's DPPC/DPPS bilayer, Sec. 3 and Fig. 1, reduced to a
same-topology coarse-grained lipid):

* every lipid is a straight rod of 12 beads (2 head, 2 linker, 8 tail) spaced
  by the bond length b0 = 0.47 nm, on a square grid of 0.8 nm (0.64 nm^2 per
  lipid);
* the two leaflets interdigitate: the lower leaflet's grid is offset by
  (0.4, 0.4) nm and its rods sit one bead spacing lower, so the slab is
  12 * 0.47 = 5.64 nm thick and opposite rods are >= 0.566 nm apart;
* water beads sit on a jittered cubic lattice at 8.3 beads/nm^3 in the slab
  between the periodic images of the bilayer, 0.25 nm from the head layers;
  the box height is derived from the water count.

Positions are encoded as unsigned 32-bit fractions of the box edge
(x = u * L / 2^32); `quantize` is that encoding, shared by both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# bead-type indices of the seeded 10-type table
BT_QP, BT_QN, BT_P0, BT_NA, BT_C1, BT_C3, BT_W = 0, 1, 2, 3, 4, 5, 6
N_BEAD_TYPES = 10
BEADS_PER_LIPID = 12
BOND_LENGTH = 0.47
GRID = 0.8
GAP = 0.25
WATER_DENSITY = 8.3
BOLTZMANN = 0.0083144626  # kJ/(mol K)

# lipid type -> bead type of each of the 12 beads (head0, head1, 2 linkers, 8 tails).
# L0 is PC-like (charged head pair +1/-1), L1 differs from L0 only in the first
# head bead (neutral P0, the PC<->PS one-bead change of Fig. 1), L2 differs
# from L0 only in its 8 tail beads.
LIPID_BEAD_TYPES = np.array(
    [
        [BT_QP, BT_QN, BT_NA, BT_NA] + [BT_C1] * 8,
        [BT_P0, BT_QN, BT_NA, BT_NA] + [BT_C1] * 8,
        [BT_QP, BT_QN, BT_NA, BT_NA] + [BT_C3] * 8,
    ],
    dtype=np.int32,
)
CHARGES = np.array([+1.0, -1.0, 0, 0, 0, 0, 0, 0, 0, 0], dtype=np.float64)
BONDS = np.array([[k, k + 1] for k in range(11)], dtype=np.int32)
ANGLES = np.array([[k, k + 1, k + 2] for k in range(10)], dtype=np.int32)


@dataclass
class Membrane:
    """A synthetic system; every array is a plain numpy array."""

    box: np.ndarray                 # [3] float64, nm
    pos: np.ndarray                 # [N,3] float64, nm, in [0, L)
    pos_u: np.ndarray               # [N,3] uint32 fixed-point fractions of the box
    vel: np.ndarray                 # [N,3] float64, nm/ps
    lipid_first_bead: np.ndarray    # [n_lipids] int32
    lipid_type: np.ndarray          # [n_lipids] int32
    lipid_bead_type: np.ndarray     # [n_lipid_types, 12] int32
    water_bead_type: int
    eps: np.ndarray                 # [10,10] float64 kJ/mol, symmetric
    sigma: np.ndarray               # [10,10] float64 nm
    charge: np.ndarray              # [10] float64 e
    bonds: np.ndarray               # [11,2] int32 local bead indices
    angles: np.ndarray              # [10,3] int32 local bead indices
    kb: float = 1250.0
    b0: float = 0.47
    ktheta: float = 25.0
    theta0_deg: float = 180.0
    rc: float = 1.1
    eps_r: float = 15.0
    eps_rf: float = 0.0             # 0 means infinity
    temperature: float = 310.0
    dt: float = 0.02
    tau_t: float = 1.0
    mass: float = 72.0
    seed: int = 0
    system_id: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_beads(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_lipids(self) -> int:
        return int(self.lipid_first_bead.shape[0])

    @property
    def kT(self) -> float:
        return BOLTZMANN * self.temperature


def quantize(pos: np.ndarray, box: np.ndarray) -> np.ndarray:
    """x -> u = floor(x / L * 2^32) mod 2^32 (the state's position encoding)."""
    frac = np.asarray(pos, np.float64) / np.asarray(box, np.float64)[None, :]
    k = np.floor(frac * 4294967296.0).astype(np.int64)
    return np.mod(k, 1 << 32).astype(np.uint32)


def dequantize(pos_u: np.ndarray, box: np.ndarray) -> np.ndarray:
    return pos_u.astype(np.float64) * (np.asarray(box, np.float64)[None, :] / 4294967296.0)


def eps_table(seed: int, lo: float = 2.0, hi: float = 5.6) -> np.ndarray:
    """Symmetric 10x10 pair-well table, each unordered pair uniform in [lo, hi]."""
    rng = np.random.default_rng(seed + 7919)
    e = rng.uniform(lo, hi, size=(N_BEAD_TYPES, N_BEAD_TYPES))
    return np.triu(e) + np.triu(e, 1).T


def _type_counts(n: int, fracs) -> list[int]:
    counts = [int(round(f * n)) for f in fracs]
    counts[-1] = n - sum(counts[:-1])
    return counts


def membrane(nx: int, ny: int | None = None, n_lipid_types: int = 2, fracs=None,
             n_water: int | None = None, water_thickness: float | None = None,
             seed: int = 1001, system_id: int = 0, n_lipids: int | None = None,
             temperature: float = 310.0, jitter: float = 0.02, layout: str = "random") -> Membrane:
    """Build a bilayer of nx*ny grid sites per leaflet (n_lipids/2 filled per leaflet).

    layout "random": lipid types shuffled by seed; "separated": in each leaflet
    the types fill stripes along x in order (a phase-separated start)."""
    ny = nx if ny is None else ny
    fracs = fracs if fracs is not None else [1.0 / n_lipid_types] * n_lipid_types
    per_leaflet = nx * ny if n_lipids is None else n_lipids // 2
    assert per_leaflet <= nx * ny
    rng = np.random.default_rng(seed)
    lx, ly = nx * GRID, ny * GRID
    slab = BEADS_PER_LIPID * BOND_LENGTH
    if n_water is None:
        n_water = int(round(WATER_DENSITY * lx * ly * (water_thickness or 5.0)))
    # water lattice: in-plane counts from the lattice constant, layer count from n_water
    a = WATER_DENSITY ** (-1.0 / 3.0)
    nwx, nwy = max(1, round(lx / a)), max(1, round(ly / a))
    nwz = max(1, round(n_water / (nwx * nwy)))
    tw = nwx * nwy * nwz / (WATER_DENSITY * lx * ly)
    lz = slab + 2 * GAP + tw
    box = np.array([lx, ly, lz])

    pos = []
    first = []
    zb = GAP
    for leaf in range(2):
        sites = [(i, j) for j in range(ny) for i in range(nx)][:per_leaflet]
        for (i, j) in sites:
            first.append(len(pos))
            if leaf == 0:   # upper leaflet: heads up, grid at cell centres
                x0, y0 = (i + 0.5) * GRID, (j + 0.5) * GRID
                for k in range(BEADS_PER_LIPID):
                    pos.append((x0, y0, zb + (12 - k) * BOND_LENGTH))
            else:           # lower leaflet: heads down, grid offset by half a cell
                x0, y0 = i * GRID, j * GRID
                for k in range(BEADS_PER_LIPID):
                    pos.append((x0, y0, zb + k * BOND_LENGTH))
    n_lip = len(first)
    dz = tw / nwz
    z0 = zb + slab + GAP
    for kz in range(nwz):
        for jy in range(nwy):
            for ix in range(nwx):
                pos.append(((ix + 0.5) * lx / nwx, (jy + 0.5) * ly / nwy, z0 + (kz + 0.5) * dz))
    pos = np.array(pos, dtype=np.float64)
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    pos = np.mod(pos, box[None, :])
    pos_u = quantize(pos, box)

    counts = _type_counts(n_lip, fracs)
    lt = np.concatenate([np.full(c, t, np.int32) for t, c in enumerate(counts)])
    rng.shuffle(lt)
    if layout == "separated":
        # per leaflet, lipids ordered by grid column x then row: types in that order
        per = _type_counts(per_leaflet, fracs)
        tl = np.concatenate([np.full(c, t, np.int32) for t, c in enumerate(per)])
        sites = [(i, j) for j in range(ny) for i in range(nx)][:per_leaflet]
        order = sorted(range(per_leaflet), key=lambda q: (sites[q][0], sites[q][1]))
        for leaf in range(2):
            for rank, q in enumerate(order):
                lt[leaf * per_leaflet + q] = tl[rank]
    elif layout != "random":
        raise ValueError(f"layout {layout!r}")
    kT = BOLTZMANN * temperature
    vel = rng.normal(0.0, math.sqrt(kT / 72.0), size=pos.shape)
    return Membrane(
        box=box, pos=pos, pos_u=pos_u, vel=vel,
        lipid_first_bead=np.array(first, np.int32), lipid_type=lt.astype(np.int32),
        lipid_bead_type=LIPID_BEAD_TYPES[:n_lipid_types].copy(), water_bead_type=BT_W,
        eps=eps_table(seed), sigma=np.full((N_BEAD_TYPES, N_BEAD_TYPES), 0.47),
        charge=CHARGES.copy(), bonds=BONDS.copy(), angles=ANGLES.copy(),
        temperature=temperature, seed=seed, system_id=system_id,
        meta=dict(nx=nx, ny=ny, n_water=int(pos.shape[0] - n_lip * 12), water_layers=nwz),
    )


# ---- the workloads: bilayers of 128, 1152 and 4608 lipids, replica sets, served patches ----

def mcmd_small(seed: int = 1001) -> Membrane:
    """128 lipids (8x8 per leaflet), 2 types 50/50, ~1700 water; FP64 MC-MD."""
    return membrane(8, n_lipid_types=2, fracs=[0.5, 0.5], n_water=1700, seed=seed)


def mcmd_large(seed: int = 1002) -> Membrane:
    """1152 lipids (24x24 per leaflet), 3 types 40/40/20, ~20k water."""
    return membrane(24, n_lipid_types=3, fracs=[0.4, 0.4, 0.2], n_water=20000, seed=seed)


def mdas_patch(seed: int = 1003) -> Membrane:
    """4608 lipids (48x48 per leaflet), 3 types, ~85k water (~140k beads)."""
    return membrane(48, n_lipid_types=3, fracs=[0.4, 0.4, 0.2], n_water=85000, seed=seed)


def patch(n_lipids: int, n_types: int, seed: int, system_id: int = 0) -> Membrane:
    """A bilayer of n_lipids (even) on a near-square grid with a 5 nm water slab."""
    m = n_lipids // 2
    nx = math.ceil(math.sqrt(m))
    ny = math.ceil(m / nx)
    fr = [1.0 / n_types] * n_types
    return membrane(nx, ny, n_lipid_types=n_types, fracs=fr, water_thickness=5.0,
                    seed=seed, system_id=system_id, n_lipids=2 * m)


def replica_set(n_replicas: int = 64, lo: int = 128, hi: int = 2048, seed: int = 1004):
    """Independent bilayers with lipid counts uniform in [lo, hi] (even), 2-3 types."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_replicas):
        n = int(rng.integers(lo, hi + 1)) // 2 * 2
        nt = int(rng.integers(2, 4))
        out.append(patch(n, nt, seed=seed * 1000 + r, system_id=r))
    return out


def tiny(n_side: int = 2, n_water: int = 40, seed: int = 5, n_lipid_types: int = 2,
         nx: int | None = None, ny: int | None = None) -> Membrane:
    """A very small bilayer for brute-force checks (box edge >= 3 rc)."""
    nx = nx or max(n_side, 5)
    ny = ny or nx
    return membrane(nx, ny, n_lipid_types=n_lipid_types, n_water=n_water, seed=seed,
                    n_lipids=2 * n_side * n_side)
