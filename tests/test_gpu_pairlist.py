"""Pair list of the MD step (a Verlet list with a skin, rebuilt when a bead
has moved half the skin): its rebuilds must not change the physics.

The forces of an MD step are the cutoff sums of Sec. 3 whatever the skin, so
trajectories with different skins (different rebuild schedules, different
summation grouping) agree to rounding; graph replays (conditional rebuild
nodes) and plain launches give the same bits."""
import numpy as np
import pytest

from paper_2005_08348_gb300 import mdas, synth
import oracle

pytestmark = pytest.mark.gpu


def test_rebuilds_happen_and_are_counted():
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp32")
    s.md_steps(200, swap_every=0)
    c = s.counters()
    assert c["md_steps"] == 200
    assert 2 <= c["list_builds"] < 200, c["list_builds"]
    # a tiny skin forces a rebuild nearly every step
    t = mdas.System(m, precision="fp32", list_skin=0.004)
    t.md_steps(20, swap_every=0)
    assert t.counters()["list_builds"] >= 10


def test_skin_does_not_change_the_trajectory_fp64():
    m = synth.mcmd_small()
    out = []
    for skin in (0.01, 0.3):
        s = mdas.System(m, precision="fp64", list_skin=skin)
        s.md_steps(30, swap_every=5)
        out.append(s.get_state())
    a, b = out
    assert np.array_equal(a["ltype"], b["ltype"])
    d = (a["pos_u"].astype(np.int64) - b["pos_u"].astype(np.int64) + 2**31) % 2**32 - 2**31
    assert np.abs(d).max() <= 64, np.abs(d).max()


@pytest.mark.parametrize("lanes", [4, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_persistent_and_separate_launches_agree(prec, lanes):
    """The persistent kernel and the separate kernels give the same bits, with
    trials, in one call or split over several (both step shapes)."""
    m = synth.mcmd_small()
    runs = []
    for persistent, calls in ((True, [36]), (False, [9, 9, 9, 9]), (True, [12, 24])):
        s = mdas.System(m, precision=prec)
        s.set_list_lanes(lanes)
        s.set_persistent(persistent)
        for n in calls:
            s.md_steps(n, swap_every=3)
        runs.append((s.get_state(), s.counters()))
    st0, c0 = runs[0]
    assert c0["list_builds"] >= 3 and c0["trials"] == 12
    for st, c in runs[1:]:
        assert np.array_equal(st["pos_u"], st0["pos_u"])
        assert np.array_equal(st["vel"], st0["vel"])
        assert np.array_equal(st["ltype"], st0["ltype"])
        assert (c["list_builds"], c["accepted"], c["md_steps"]) == (c0["list_builds"], c0["accepted"], c0["md_steps"])


def test_one_step_after_rebuild_matches_oracle_fp64():
    # a state far from the list's build positions (set by set_state) is rebuilt
    m = synth.mcmd_small()
    s = mdas.System(m, precision="fp64")
    s.md_steps(10, swap_every=0)
    st = s.get_state()
    rng = np.random.default_rng(5)
    shift = rng.integers(-2 ** 25, 2 ** 25, size=(m.n_beads, 3))
    pos_u = ((st["pos_u"].astype(np.int64) + shift) % 2 ** 32).astype(np.uint32)
    s.set_state(pos_u=pos_u, vel=st["vel"], ltype=st["ltype"], step=st["step"], trial=st["trial"])
    s.md_steps(1, swap_every=0)
    got = s.get_state()
    o = oracle.Oracle(m)
    so = o.state(pos_u=pos_u, vel=st["vel"], ltype=st["ltype"], step=st["step"])
    o.md_steps(so, 1)
    d = (got["pos_u"].astype(np.int64) - so["pos_u"].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    assert np.abs(d).max() <= 1, np.abs(d).max()
    assert np.abs(got["vel"] - so["vel"]).max() < 1e-10


@pytest.mark.parametrize("lanes", [4, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("which", ["small", "large"])
def test_step_kernel_forces_match_oracle(prec, which, lanes):
    """The MD step's own forces: from rest without a thermostat one step gives
    v = F dt / m exactly up to one rounding, so F = v m / dt is compared with
    the oracle's forces at the force tolerance."""
    m = synth.mcmd_small() if which == "small" else synth.mcmd_large()
    s = mdas.System(m, precision=prec, tau_t=0.0)
    s.set_list_lanes(lanes)
    s.md_steps(5, swap_every=0)                    # a state the list was built for earlier
    st = s.get_state()
    s.set_state(pos_u=st["pos_u"], vel=np.zeros_like(st["vel"]), ltype=st["ltype"], step=st["step"])
    s.md_steps(8, swap_every=0)                    # moves the beads, keeps the list when it can
    st = s.get_state()
    s.set_state(pos_u=st["pos_u"], vel=np.zeros_like(st["vel"]), ltype=st["ltype"], step=st["step"])
    s.md_steps(1, swap_every=0)
    F = s.get_state()["vel"] * (m.mass / m.dt)
    _, Fo = oracle.Oracle(m).energy(st["pos_u"], ltype=st["ltype"])
    frms = np.sqrt((Fo * Fo).sum(1).mean())
    err = (np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max()
    assert err < (1e-10 if prec == "fp64" else 1e-5), err


def test_tune_list_skin_times_every_candidate():
    """The autotuner creates, times and destroys one batch per candidate skin
    and leaves the caller's systems alone."""
    ms = synth.replica_set(3, lo=128, hi=256, seed=11)
    keep = mdas.System(ms[0], precision="fp32")
    keep.md_steps(5, swap_every=0)
    before = keep.get_state()
    best, us = mdas.tune_list_skin(ms, skins=(0.1, 0.3), md_steps=20, swap_trials=4, rounds=2)
    assert best in (0.1, 0.3) and set(us) == {0.1, 0.3}
    assert all(np.isfinite(v) and v > 0 for v in us.values())
    assert us[best] == min(us.values())
    after = keep.get_state()
    assert np.array_equal(before["pos_u"], after["pos_u"])
    # a system made with the tuned skin runs like any other
    s = mdas.System(ms[0], precision="fp32", list_skin=best)
    s.md_steps(10, swap_every=5)
    assert s.counters()["md_steps"] == 10
    with pytest.raises(mdas.MdasError):
        mdas.tune_list_skin(ms[:1], skins=(0.3, 0.0), md_steps=10)


@pytest.mark.parametrize("lanes", [4, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_trials_beside_the_next_step_match_separate_launches(prec, lanes):
    """In the persistent kernel each exchange trial runs beside the next MD
    step; the items it can change wait for its decision and, after an accepted
    exchange, sum their forces again.  The result is the bits of trials run
    strictly after their step (separate launches)."""
    m = synth.mcmd_small()
    runs = []
    for persistent in (True, False):
        s = mdas.System(m, precision=prec, temperature=450.0)
        s.set_list_lanes(lanes)
        s.set_persistent(persistent)
        s.md_steps(150, swap_every=1)
        s.md_steps(7, swap_every=2)
        runs.append((s.get_state(), s.counters()))
    (a, ca), (b, cb) = runs
    assert ca["accepted"] >= 3 and ca["item_redos"] > 0, ca
    assert cb["item_redos"] == 0
    assert np.array_equal(a["pos_u"], b["pos_u"])
    assert np.array_equal(a["vel"], b["vel"])
    assert np.array_equal(a["ltype"], b["ltype"])
    for key in ("md_steps", "force_evals", "trials", "null_trials", "accepted", "list_builds"):
        assert ca[key] == cb[key], key


def test_trials_across_segment_boundaries():
    """Trial intervals that do not divide the 511-step segments (and one
    longer than a segment): the same trials and bits as separate launches."""
    m = synth.mcmd_small()
    runs = []
    for persistent in (True, False):
        s = mdas.System(m, precision="fp32")
        s.set_persistent(persistent)
        s.md_steps(1200, swap_every=10)
        s.md_steps(4100, swap_every=2000)
        runs.append((s.get_state(), s.counters()))
    (a, ca), (b, cb) = runs
    assert ca["trials"] == 120 + 2 == cb["trials"]
    assert np.array_equal(a["pos_u"], b["pos_u"]) and np.array_equal(a["ltype"], b["ltype"])
    assert ca["accepted"] == cb["accepted"]


@pytest.mark.parametrize("lanes", [4, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_alchemical_trajectory_in_one_run_matches_separate_launches(prec, lanes):
    """The MDAS trajectory (lambda advanced and each block's work term added
    inside the MD run) gives the same work, decision and bits in the
    persistent kernel as with separate launches."""
    m = synth.mcmd_small(seed=2024)
    out = []
    for persistent in (True, False):
        s = mdas.System(m, precision=prec)
        s.set_list_lanes(lanes)
        s.set_persistent(persistent)
        s.md_steps(10, swap_every=0)
        res = [s.alchemical_move(4, 6, 3) for _ in range(2)]
        out.append((res, s.get_state()))
    (ra, sa), (rb, sb) = out
    for x, y in zip(ra, rb):
        assert x["w"] == y["w"] and x["accepted"] == y["accepted"]
    assert np.array_equal(sa["pos_u"], sb["pos_u"]) and np.array_equal(sa["vel"], sb["vel"])


@pytest.mark.parametrize("lanes", [4, 2])
def test_tune_batch_times_skins_and_layouts_with_the_same_bits(lanes):
    """The batch tuner times every (skin, layout, wave, lanes) candidate; the
    layouts of a batch (partitioned, lockstep) and its waves give the same
    bits, for either step shape."""
    ms = synth.replica_set(6, lo=600, hi=2048, seed=12)
    if lanes == 4:
        best, part, wave, lane, us = mdas.tune_batch(ms, skins=(0.25, 0.3), waves=(0, 60_000), lanes=(2, 4),
                                                     md_steps=20, swap_trials=8, rounds=1)
        assert set(us) == {(sk, p, w, n) for sk in (0.25, 0.3) for p in (False, True) for w in (0, 60_000)
                           for n in (2, 4)}
        assert us[(best, part, wave, lane)] == min(us.values())
    out = []
    for layout, wv in ((True, 0), (False, 0), (True, 60_000)):
        sy = [mdas.System(m) for m in ms]
        for s in sy:
            s.set_list_lanes(lanes)
            s.set_partitioned(layout)
            s.set_batch_wave(wv)
        mdas.batch_run(sy, 15, 10)
        mdas.batch_run(sy, 15, 10)
        out.append([s.get_state() for s in sy])
    for runs in zip(*out):
        a = runs[0]
        for b in runs[1:]:
            assert np.array_equal(a["pos_u"], b["pos_u"]) and np.array_equal(a["vel"], b["vel"])
            assert np.array_equal(a["ltype"], b["ltype"]) and a["trial"] == b["trial"]


def test_list_lanes_switch_and_refusals():
    """A system may change its step shape between MD calls (its pair list is
    built again for the new shape); the systems of a batch must agree, and
    only 2 or 4 list columns per bead exist."""
    m = synth.mcmd_small()
    a = mdas.System(m)
    a.md_steps(10, swap_every=2)
    b0 = a.counters()["list_builds"]
    a.set_list_lanes(2)
    a.md_steps(10, swap_every=2)
    c = a.counters()
    assert c["md_steps"] == 20 and c["trials"] == 10 and c["list_builds"] > b0
    st = a.get_state()
    to, _ = oracle.Oracle(m).energy(st["pos_u"], ltype=st["ltype"], forces=False)
    assert abs(a.energy()["potential"] - to["total"]) <= 1e-9 * abs(to["total"])
    with pytest.raises(mdas.MdasError) as err:
        a.set_list_lanes(3)
    assert err.value.status == 1
    b = mdas.System(m)
    with pytest.raises(mdas.MdasError) as err:
        mdas.batch_run([a, b], 5, 0)
    assert err.value.status == 1
    b.set_list_lanes(2)
    mdas.batch_run([a, b], 5, 0)
    assert a.counters()["md_steps"] == 25 and b.counters()["md_steps"] == 5
    # the batch of these two systems follows a later change of shape (and its agreement check too)
    a.set_list_lanes(4)
    with pytest.raises(mdas.MdasError) as err:
        mdas.batch_run([a, b], 5, 0)
    assert err.value.status == 1
    b.set_list_lanes(4)
    mdas.batch_run([a, b], 5, 0)
    assert a.counters()["md_steps"] == 30 and b.counters()["md_steps"] == 10
