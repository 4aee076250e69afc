"""Semi-isotropic Parrinello-Rahman pressure coupling (Sec. 3) against the
oracle: the pressure tensor, box velocity and box of every update, the trial
decisions and the states of an FP64 trajectory; the first update in FP32;
the same bits from every launch mode and call split; exact resume; the guard
that stops a box below what the cell grids allow."""
import numpy as np
import pytest

import oracle
from paper_2005_08348_gb300 import mdas, synth

pytestmark = pytest.mark.gpu

PC = dict(p_ref=1.0, tau_p=12.0, compressibility=3e-4, nstpcouple=5, box_margin=0.05)
DE_TOL = 1e-4


def _baro(pc=PC):
    return oracle.barostat(p_ref=pc["p_ref"], tau_p=pc["tau_p"], beta=pc["compressibility"], nst=pc["nstpcouple"])


def _dx_nm(a, b, box):
    d = np.abs((a.astype(np.int64) - b.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
    return float((d * (np.asarray(box) / 2 ** 32)[None, :]).max())


def test_fp64_npt_trajectory_matches_oracle():
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp64", pcouple=PC)
    o = oracle.Oracle(m)
    so = o.state()
    b = _baro()
    rec_o = []
    for _ in range(6):                       # six coupling intervals, a trial after each
        s.md_steps(5, swap_every=5)
        rec_o += o.md_steps_npt(so, b, 5, swap_every=5)
        box, bv, P = s.box()
        assert np.allclose(P, list(b.P), rtol=1e-7, atol=1e-6), (P, list(b.P))
        assert np.allclose(bv, list(b.boxv), rtol=1e-7, atol=1e-12), (bv, list(b.boxv))
        assert np.allclose(box, o.box, rtol=1e-10, atol=0), (box, o.box)
    assert abs(box[0] / m.box[0] - 1) > 1e-3            # the box did move
    rec = s.trial_log(0, 6)
    for g, r in zip(rec, rec_o):
        assert (g["a"], g["b"], bool(g["null"]), bool(g["accepted"])) == (r["a"], r["b"], r["null"], r["accepted"])
        if not r["null"]:
            assert abs(g["dE"] - r["dE"]) < DE_TOL
    st = s.get_state()
    assert np.array_equal(st["ltype"], so["ltype"])
    assert _dx_nm(st["pos_u"], so["pos_u"], box) < 1e-6
    assert np.allclose(st["box"], box) and np.allclose(st["box_velocity"], bv)
    e = s.energy()
    to, _ = o.energy(so["pos_u"], ltype=so["ltype"], forces=False)
    assert e["potential"] == pytest.approx(to["total"], rel=1e-7)


def test_fp32_first_update_matches_oracle():
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp32", pcouple=PC)
    o = oracle.Oracle(m)
    so = o.state()
    b = _baro()
    s.md_steps(5, swap_every=0)
    o.md_steps_npt(so, b, 5)
    box, bv, P = s.box()
    # FP32 forces (max relative error ~5e-6) and the FP32 step's virial sums
    assert np.allclose(P, list(b.P), rtol=0, atol=1.0), (P, list(b.P))
    assert np.allclose(box, o.box, rtol=1e-8, atol=0)


def test_npt_with_an_mdas_move_matches_oracle():
    """The alchemical trajectory runs at the box it starts with; constant-
    pressure MD resumes after it."""
    m = synth.mcmd_small(seed=2025)
    s = mdas.System(m, precision="fp64", pcouple=PC)
    o = oracle.Oracle(m)
    so = o.state()
    b = _baro()
    s.md_steps(5)
    o.md_steps_npt(so, b, 5)
    res = s.alchemical_move(4, 3, 2)
    ro = o.mdas_move(so, 4, 3, 2)
    assert np.array_equal(res["pairs"], ro["pairs"])
    assert abs(res["w"] - ro["w"]) < DE_TOL and res["accepted"] == ro["accepted"]
    s.md_steps(10)
    o.md_steps_npt(so, b, 10)
    box, bv, P = s.box()
    assert np.allclose(P, list(b.P), rtol=1e-7, atol=1e-6)
    assert np.allclose(box, o.box, rtol=1e-10, atol=0)
    st = s.get_state()
    assert np.array_equal(st["ltype"], so["ltype"])
    assert _dx_nm(st["pos_u"], so["pos_u"], box) < 1e-6


def test_launch_modes_and_call_splits_agree():
    m = synth.mcmd_small()
    runs = []
    for persistent, calls in ((True, [30]), (False, [30]), (True, [7, 23]), (False, [12, 18])):
        s = mdas.System(m, precision="fp32", pcouple=PC)
        s.set_persistent(persistent)
        for n in calls:
            s.md_steps(n, swap_every=1)
        runs.append((s.get_state(), s.box()))
    st0, b0 = runs[0]
    for st, bx in runs[1:]:
        for k in ("pos_u", "vel", "ltype", "box", "box_velocity"):
            assert np.array_equal(st[k], st0[k]), k
        assert np.array_equal(bx[2], b0[2])


def test_npt_resumes_exactly():
    m = synth.mcmd_small()
    a = mdas.System(m, precision="fp32", pcouple=PC)
    a.md_steps(12, swap_every=3)
    saved = a.get_state()
    a.md_steps(18, swap_every=3)
    b = mdas.System(m, precision="fp32", pcouple=PC)
    b.resume(saved)
    b.md_steps(18, swap_every=3)
    sa, sb = a.get_state(), b.get_state()
    for k in ("pos_u", "vel", "ltype", "box", "box_velocity", "step", "trial"):
        assert np.array_equal(sa[k], sb[k]), k


def test_box_below_the_grid_minimum_stops_the_system():
    """A reference pressure far above the system's drives the box down past
    its margin in one update: the update is refused (box unchanged), the
    call reports an unstable state and dynamics wait for a new state."""
    m = synth.mcmd_small()
    pc = dict(PC, p_ref=5e4, tau_p=0.5)
    s = mdas.System(m, precision="fp32", pcouple=pc)
    st = s.get_state()
    with pytest.raises(mdas.MdasError) as e:
        s.md_steps(5)
    assert e.value.status == 4
    assert np.array_equal(s.box()[0], m.box)
    with pytest.raises(mdas.MdasError):
        s.md_steps(1)
    s.set_state(pos_u=st["pos_u"], vel=st["vel"], ltype=st["ltype"])
    s.md_steps(3)


def test_constant_volume_systems_report_no_pressure_and_keep_the_box():
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp32")
    s.md_steps(20)
    box, bv, P = s.box()
    assert np.array_equal(box, m.box) and not bv.any() and not P.any()


def test_fp64_shrinking_box_matches_oracle():
    """A reference pressure above the system's shrinks the box by several
    percent in 20 steps: the pair list, built at a larger box, keeps every
    pair within the cutoff (its displacement bound shrinks with the box), so
    the trajectory still follows the oracle's, which has no list."""
    m = synth.mcmd_small()
    pc = dict(PC, p_ref=4000.0, tau_p=2.0, box_margin=0.2)
    s = mdas.System(m, precision="fp64", pcouple=pc)
    o = oracle.Oracle(m)
    so = o.state()
    b = _baro(pc)
    lo = np.array(m.box, float)
    for _ in range(4):
        s.md_steps(5, swap_every=5)
        o.md_steps_npt(so, b, 5, swap_every=5)
        box, bv, P = s.box()
        assert np.allclose(P, list(b.P), rtol=1e-7, atol=1e-6), (P, list(b.P))
        assert np.allclose(box, o.box, rtol=1e-10, atol=0)
        lo = np.minimum(lo, box)
    assert np.all(lo < 0.95 * m.box)
    st = s.get_state()
    assert np.array_equal(st["ltype"], so["ltype"])
    assert _dx_nm(st["pos_u"], so["pos_u"], box) < 1e-6


def test_batches_mix_coupled_and_constant_volume_systems():
    """In one batch a pressure-coupled system and a constant-volume one each
    get the bits of their solo runs; coupled systems at different coupling
    phases are refused."""
    m1, m2 = synth.mcmd_small(), synth.mcmd_small(seed=1009)
    a = mdas.System(m1, precision="fp32", pcouple=PC)
    b = mdas.System(m2, precision="fp32")
    mdas.batch_run([a, b], 17, 0)
    a2 = mdas.System(m1, precision="fp32", pcouple=PC)
    a2.md_steps(17)
    b2 = mdas.System(m2, precision="fp32")
    b2.md_steps(17)
    for x, y in ((a, a2), (b, b2)):
        sx, sy = x.get_state(), y.get_state()
        for k in ("pos_u", "vel", "box", "box_velocity"):
            assert np.array_equal(sx[k], sy[k]), k
    assert not np.array_equal(a.get_state()["box"], m1.box)
    c = mdas.System(m1, precision="fp32", pcouple=PC)
    c.md_steps(3)
    with pytest.raises(mdas.MdasError) as e:
        mdas.batch_run([a, c], 5, 0)
    assert e.value.status == 1
