"""The seeded synthetic workloads have the sizes, boxes, type mixes and
conditions the design notes state, and the same seed gives the same bits."""
import numpy as np
import pytest

from paper_2005_08348_gb300 import synth


@pytest.mark.parametrize("make,lipids,beads,box,types", [
    (synth.mcmd_small, 128, 3226, (6.4, 6.4, 11.111), (64, 64)),
    (synth.mcmd_large, 1152, 33597, (19.2, 19.2, 12.602), (461, 461, 230)),
    (synth.mdas_patch, 4608, 140472, (38.4, 38.4, 13.099), (1843, 1843, 922)),
])
def test_workload_shapes(make, lipids, beads, box, types):
    m = make()
    assert (m.n_lipids, m.n_beads) == (lipids, beads)
    assert np.allclose(m.box, box, atol=5e-4)
    assert tuple(np.bincount(m.lipid_type)) == types
    assert m.temperature == 310.0 and m.dt == 0.02 and m.rc == 1.1 and m.eps_r == 15.0
    # 0.64 nm^2 per lipid on each leaflet's square grid
    assert m.box[0] * m.box[1] / (lipids / 2) == pytest.approx(0.64)
    # every bead inside the box, fixed point consistent with nm
    assert np.all((m.pos >= 0) & (m.pos < m.box[None, :]))
    assert np.allclose(m.pos_u.astype(np.float64) * (m.box / 2 ** 32)[None, :], m.pos, atol=1e-8)


def test_workloads_are_seeded():
    a, b, c = synth.mcmd_small(), synth.mcmd_small(), synth.mcmd_small(seed=1009)
    assert np.array_equal(a.pos_u, b.pos_u) and np.array_equal(a.vel, b.vel)
    assert np.array_equal(a.lipid_type, b.lipid_type)
    assert not np.array_equal(a.vel, c.vel)


def test_replica_set_sizes():
    reps = synth.replica_set()
    assert len(reps) == 64
    n = np.array([r.n_lipids for r in reps])
    assert np.all((n >= 128) & (n <= 2048) & (n % 2 == 0))
    assert sum(r.n_beads for r in reps) == 1787976
    assert [r.system_id for r in reps] == list(range(64))
