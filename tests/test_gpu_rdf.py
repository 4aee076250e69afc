"""The mixing observable of Sec. 4 (in-plane head-bead pair distribution per
leaflet): the GPU's integer pair counts equal the oracle's exactly, on the
bench workloads after MD with exchanges, for every lipid type and several
binnings up to half the box."""
import numpy as np
import pytest

import oracle
from paper_2005_08348_gb300 import mdas, mixing, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["small", "large", "patch"])
def test_head_rdf_counts_match_oracle(which):
    m = {"small": synth.mcmd_small, "large": synth.mcmd_large, "patch": synth.mdas_patch}[which]()
    s = mdas.System(m, precision="fp32")
    s.md_steps(40, swap_every=2)
    st = s.get_state()
    o = oracle.Oracle(m)
    half = 0.5 * min(m.box[0], m.box[1])
    for lt in range(m.lipid_bead_type.shape[0]):
        for head_k, r_max, n_bins in ((1, 3.0, 60), (0, half, 1024), (1, 1.0, 7)):
            c, nh = s.head_rdf(lt, head_k, r_max, n_bins)
            co, nho = o.head_rdf(st["pos_u"], st["ltype"], lt, head_k, r_max, n_bins)
            assert np.array_equal(nh, nho)
            assert np.array_equal(c, co), (lt, head_k, r_max, n_bins)
    assert c.sum() > 0


def test_head_rdf_separated_start_and_bad_arguments():
    m = mixing.bilayer(nx=10, ny=20)
    s = mdas.System(m, precision="fp32")
    c, nh = s.head_rdf(1, 1, 3.0, 60)
    co, nho = oracle.Oracle(m).head_rdf(m.pos_u, m.lipid_type, 1, 1, 3.0, 60)
    assert np.array_equal(c, co) and list(nh) == [100, 100]     # 10 x 20 sites per leaflet
    r, g, g2 = mixing.g_of_r(c, nh, m.box, 3.0)
    assert g2.max() > 1.5          # a stripe of one type: strongly enriched neighbours
    for bad in (dict(lipid_type=7), dict(head_k=11), dict(n_bins=0), dict(n_bins=2000), dict(r_max=100.0)):
        kw = dict(lipid_type=1, head_k=1, r_max=3.0, n_bins=60)
        kw.update(bad)
        with pytest.raises(mdas.MdasError):
            s.head_rdf(**kw)
