"""Small hand-made systems for the tests (bead placement only)."""
import numpy as np

from paper_2005_08348_gb300 import synth


def beads(points, types, box=(4.0, 4.0, 4.0), eps=None, charge=None, eps_rf=0.0):
    """Free beads (one-bead 'lipids') at the given points with the given bead types."""
    pts = np.asarray(points, np.float64)
    n = pts.shape[0]
    box = np.asarray(box, np.float64)
    pos = np.mod(pts, box[None, :])
    tbl = synth.eps_table(3) if eps is None else np.asarray(eps, np.float64)
    ch = synth.CHARGES.copy() if charge is None else np.asarray(charge, np.float64)
    nbt = tbl.shape[0]
    return synth.Membrane(
        box=box, pos=pos, pos_u=synth.quantize(pos, box), vel=np.zeros_like(pos),
        lipid_first_bead=np.arange(n, dtype=np.int32),
        lipid_type=np.asarray(types, np.int32),
        lipid_bead_type=np.arange(nbt, dtype=np.int32).reshape(nbt, 1),
        water_bead_type=synth.BT_W, eps=tbl, sigma=np.full((nbt, nbt), 0.47), charge=ch,
        bonds=np.zeros((0, 2), np.int32), angles=np.zeros((0, 3), np.int32), eps_rf=eps_rf,
    )


def with_types(m, lipid_types):
    m.lipid_type = np.asarray(lipid_types, np.int32)
    return m


def pair_distances(pos, box):
    d = pos[:, None, :] - pos[None, :, :]
    d -= box[None, None, :] * np.round(d / box[None, None, :])
    r = np.sqrt((d * d).sum(-1))
    iu = np.triu_indices(pos.shape[0], 1)
    return r[iu]
