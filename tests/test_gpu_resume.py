"""Checkpoint and resume: a run continued from a saved state repeats the
uninterrupted run bit for bit.

Every random number of the method is drawn from Philox at counters carried in
the state (MD steps, trials, moves, AT steps), the state holds the exact
fixed-point positions, and get_state also returns the positions the pair list
was built at and the kinetic energy the thermostat reads next; a fresh system
given all of it sums the same pairs in the same order."""
import numpy as np
import pytest

from paper_2005_08348_gb300 import mdas, synth

pytestmark = pytest.mark.gpu


def same(a, b):
    for k in ("pos_u", "vel", "ltype", "step", "trial", "move", "at_step"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec,persistent", [("fp32", True), ("fp32", False), ("fp64", True)])
def test_md_with_trials_resumes_exactly(prec, persistent):
    m = synth.mcmd_small()
    a = mdas.System(m, precision=prec)
    a.set_persistent(persistent)
    a.md_steps(40, swap_every=4)
    saved = a.get_state()
    assert saved["list_ref"] is not None and saved["ke"] is not None
    a.md_steps(60, swap_every=4)
    b = mdas.System(m, precision=prec)
    b.set_persistent(persistent)
    b.resume(saved)
    b.md_steps(60, swap_every=4)
    same(a.get_state(), b.get_state())
    ea, eb = a.energy(), b.energy()
    assert ea["total"] == eb["total"]
    # the continuation saw list rebuilds of its own
    assert b.counters()["list_builds"] >= 2


def test_resume_across_exchange_batches_and_mdas_moves():
    m = synth.mcmd_small()
    a = mdas.System(m, precision="fp32")

    def rest(s):
        s.swap_trials(64)
        r = s.alchemical_move(2, 4, 3)
        s.md_steps(30, swap_every=3)
        return r

    a.md_steps(21, swap_every=3)
    a.swap_trials(32)
    saved = a.get_state()
    ra = rest(a)
    b = mdas.System(m, precision="fp32")
    b.resume(saved)
    rb = rest(b)
    assert ra["w"] == rb["w"] and ra["accepted"] == rb["accepted"]
    assert np.array_equal(ra["pairs"], rb["pairs"])
    same(a.get_state(), b.get_state())


def test_resume_right_after_a_rejected_or_accepted_move():
    """After an MDAS move the velocities may be the snapshot's (rejection) and
    the list stale: get_state says so and the resumed run rebuilds the same
    way the uninterrupted one does."""
    m = synth.mcmd_small()
    a = mdas.System(m, precision="fp32")
    a.md_steps(10, swap_every=0)
    a.alchemical_move(2, 3, 2)
    saved = a.get_state()
    a.md_steps(25, swap_every=5)
    b = mdas.System(m, precision="fp32")
    b.resume(saved)
    b.md_steps(25, swap_every=5)
    same(a.get_state(), b.get_state())


def test_list_ref_far_from_the_positions_is_refused():
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp32")
    s.md_steps(5, swap_every=0)
    st = s.get_state()
    ref = st["list_ref"].copy()
    ref[7, 0] += np.uint32(1 << 28)          # 1/16 of the box edge away
    with pytest.raises(mdas.MdasError):
        s.set_state(pos_u=st["pos_u"], vel=st["vel"], ltype=st["ltype"], step=st["step"], list_ref=ref)
    # the plain restore (no list_ref) still works and the system runs on
    s.set_state(pos_u=st["pos_u"], vel=st["vel"], ltype=st["ltype"], step=st["step"])
    s.md_steps(5, swap_every=0)
    assert s.counters()["md_steps"] == 10


def test_expired_wait_is_reported_and_the_run_resumes():
    """Failure detection without a fault: a grid-barrier wait of the MD kernel
    runs out (an arrival that never comes), the host reads MDAS_ERR_TIMEOUT,
    the system refuses dynamics until a state is installed, and the context
    stays usable: the resumed run equals one that never stalled."""
    m = synth.mcmd_small()
    a = mdas.System(m, precision="fp32")
    a.md_steps(12, swap_every=3)
    with pytest.raises(mdas.MdasError) as e:
        a.wait_timeout_probe()
    assert e.value.status == 5
    with pytest.raises(mdas.MdasError):
        a.md_steps(1)
    a.resume(a.get_state())
    a.md_steps(24, swap_every=3)
    b = mdas.System(m, precision="fp32")
    b.md_steps(12, swap_every=3)
    b.md_steps(24, swap_every=3)
    same(a.get_state(), b.get_state())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_packed_state_round_trip(prec):
    """mdas_get_state_packed / mdas_set_state_packed: the library's own layout
    holds the same state as get_state; installing it continues exactly as
    set_state with the same arrays (both rebuild the pair list); meta words
    follow the lipid types; a bad lipid type is refused before any copy."""
    torch = pytest.importorskip("torch")
    m = synth.mcmd_small()
    a = mdas.System(m, precision=prec)
    a.md_steps(30, swap_every=2)
    pos4, vel4, lt = a.get_state_packed()
    st = a.get_state()
    assert np.array_equal(pos4[:, :3], st["pos_u"])
    assert np.array_equal(vel4[:, :3].astype(np.float64), st["vel"])
    assert np.array_equal(lt, st["ltype"])
    bpl = synth.BEADS_PER_LIPID
    lip_beads = m.n_lipids * bpl
    bt = pos4[:lip_beads, 3] & 15
    assert np.array_equal(bt, m.lipid_bead_type[np.repeat(lt, bpl), np.tile(np.arange(bpl), m.n_lipids)])
    assert np.all(pos4[lip_beads:, 3] & 15 == m.water_bead_type)
    # a new lipid-type assignment travels with the packed state
    lt2 = lt.copy()
    lt2[:4] = (lt2[:4] + 1) % 2
    b, c = mdas.System(m, precision=prec), mdas.System(m, precision=prec)
    p4 = pos4.copy()
    p4[:, 3] = 0                                          # meta words are rebuilt from the types
    b.set_state_packed(p4, vel4, lt2)
    c.set_state(pos_u=st["pos_u"], vel=st["vel"], ltype=lt2)
    for s in (b, c):
        s.md_steps(40, swap_every=1)
    same(b.get_state(), c.get_state())
    assert b.energy()["total"] == c.energy()["total"]
    # pinned torch tensors as the host arrays
    tp = torch.empty((m.n_beads, 4), dtype=torch.int32).pin_memory()
    tv = torch.empty((m.n_beads, 4), dtype=torch.float64 if prec == "fp64" else torch.float32).pin_memory()
    tl = torch.empty(m.n_lipids, dtype=torch.int32).pin_memory()
    b.get_state_packed(tp, tv, tl)
    sb = b.get_state()
    assert np.array_equal(tp.numpy()[:, :3].view(np.uint32), sb["pos_u"])
    assert np.array_equal(tl.numpy(), sb["ltype"])
    bad = lt.copy()
    bad[0] = 99
    with pytest.raises(mdas.MdasError) as e:
        b.set_state_packed(p4, vel4, bad)
    assert e.value.status == 1
    same(b.get_state(), sb)                               # nothing was installed
