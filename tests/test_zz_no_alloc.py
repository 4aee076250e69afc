"""mdas_forces_noalloc: one force evaluation that allocates nothing.

It serves callers that cannot allocate device memory while they run (a fixed
memory budget handed over by a host application, a framework that owns the
device heap, a real-time loop that must not meet cudaMalloc's implicit
synchronisation).  Its forces must equal those of the regular entry point,
mdas_forces, within the force tolerance, on consecutive calls that reuse the
shared scratch array.
"""
import numpy as np
import pytest

from paper_2005_08348_gb300 import mdas, synth

pytestmark = pytest.mark.gpu

F_TOL = 1e-5


def force_err(F, Fo):
    frms = np.sqrt((Fo * Fo).sum(1).mean())
    return (np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_forces_equal_regular_forces_on_two_calls(prec):
    import torch
    m = synth.mcmd_small()
    s = mdas.System(m, precision=prec)
    f_out = torch.empty(m.n_beads * 3, dtype=torch.float64, device="cuda")
    for call in range(2):
        s.md_steps(7, swap_every=7 if call else 0)          # a different state on each call
        st = s.get_state()
        F_ref = s.forces()
        pos = torch.from_numpy(st["pos_u"].reshape(-1).view(np.int32).copy()).cuda()
        lt = torch.from_numpy(st["ltype"].astype(np.int32)).cuda()
        f_out.fill_(np.nan)
        torch.cuda.synchronize()
        mdas.forces_noalloc(s, pos.data_ptr(), lt.data_ptr(), f_out.data_ptr())
        F = f_out.cpu().numpy().reshape(-1, 3)
        assert np.isfinite(F).all()
        assert force_err(F, F_ref) < F_TOL, (call, force_err(F, F_ref))


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    m = synth.mcmd_large()                                   # 33,597 beads > 16,384
    s = mdas.System(m)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(mdas.MdasError) as e:
        mdas.forces_noalloc(s, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
    assert e.value.status == 1


def test_noalloc_forces_after_pressure_coupling_use_the_current_box():
    """Positions are fractions of the box: after box updates (Sec. 3 pressure
    coupling) the allocation-free call must read them in the current box, as
    mdas_forces does, not in the box the system was created with."""
    import torch
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp64", pcouple=dict(nstpcouple=5, tau_p=1.0))
    s.md_steps(20)
    box, _, _ = s.box()
    assert np.abs(box - m.box).max() > 1e-4 * m.box.max()
    st = s.get_state()
    F_ref = s.forces()
    pos = torch.from_numpy(st["pos_u"].reshape(-1).view(np.int32).copy()).cuda()
    lt = torch.from_numpy(st["ltype"].astype(np.int32)).cuda()
    f_out = torch.full((m.n_beads * 3,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    mdas.forces_noalloc(s, pos.data_ptr(), lt.data_ptr(), f_out.data_ptr())
    F = f_out.cpu().numpy().reshape(-1, 3)
    assert force_err(F, F_ref) < F_TOL, force_err(F, F_ref)
