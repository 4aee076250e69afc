"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances (stated for the hot path): forces max relative 1e-5 (normalised by
max(|F_i|, F_rms)), energy relative 1e-9, dE and work absolute 1e-4 kJ/mol,
integer state (cell lists, lipid types, trial proposals) bit-exact; an
accept/reject decision may differ only when |dE + kT ln u| < 1e-4.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_08348_gb300 import mdas, synth

pytestmark = pytest.mark.gpu

F_TOL, E_TOL, DE_TOL = 1e-5, 1e-9, 1e-4


def force_err(F, Fo):
    frms = np.sqrt((Fo * Fo).sum(1).mean())
    return (np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max()


@pytest.fixture(scope="module")
def small():
    return synth.mcmd_small()


@pytest.fixture(scope="module")
def large():
    return synth.mcmd_large()


def test_philox_bit_equal_to_oracle():
    out = mdas.philox(0, 0, 0, 0, 0, 1)
    assert [int(x) for x in out[0]] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    rng = np.random.default_rng(0)
    for _ in range(4):
        k0, k1, c1, c2, c3 = [int(x) for x in rng.integers(0, 2 ** 32, 5, dtype=np.uint64)]
        g = mdas.philox(k0, k1, c1, c2, c3, 257)
        for i in (0, 1, 100, 256):
            assert [int(x) for x in g[i]] == oracle.philox([i, c1, c2, c3], [k0, k1])


def test_positions_enter_bit_exact(small):
    s = mdas.System(small)
    assert np.array_equal(s.get_state()["pos_u"], small.pos_u)


@pytest.mark.parametrize("which", ["small", "large"])
def test_cell_list_bit_exact(which, small, large):
    m = small if which == "small" else large
    s = mdas.System(m)
    s.md_steps(7)
    st = s.get_state()
    ids, start, nc = s.cell_list()
    o = oracle.Oracle(m)
    assert nc == o.cell_dims()
    _, srt, st_o = o.cell_list(st["pos_u"])
    assert np.array_equal(ids, srt) and np.array_equal(start, st_o)


@pytest.mark.parametrize("which,prec", [("small", "fp64"), ("small", "fp32"), ("large", "fp32")])
def test_forces_match_oracle(which, prec, small, large):
    m = small if which == "small" else large
    s = mdas.System(m, precision=prec)
    s.md_steps(5)
    st = s.get_state()
    F = s.forces()
    _, Fo = oracle.Oracle(m).energy(st["pos_u"], ltype=st["ltype"])
    err = force_err(F, Fo)
    assert err < (1e-10 if prec == "fp64" else F_TOL), err


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_energy_matches_oracle(prec, small):
    s = mdas.System(small, precision=prec)
    s.md_steps(3)
    st = s.get_state()
    e = s.energy()
    to, _ = oracle.Oracle(small).energy(st["pos_u"], ltype=st["ltype"], forces=False)
    assert e["pairs"] == to["pairs"]
    for k in ("lj", "rf", "bond", "angle"):
        assert abs(e[k] - to[k]) <= E_TOL * abs(to["total"]), (k, e[k], to[k])
    assert e["potential"] == pytest.approx(to["total"], rel=E_TOL)
    ke = 0.5 * 72.0 * (st["vel"] ** 2).sum()
    assert e["kinetic"] == pytest.approx(ke, rel=1e-12)


def test_delta_energy_matches_oracle(large):
    s = mdas.System(large)
    st = s.get_state()
    o = oracle.Oracle(large)
    lt = st["ltype"]
    rng = np.random.default_rng(1)
    n = 0
    while n < 12:
        a, b = rng.integers(0, large.n_lipids, 2)
        if lt[a] == lt[b]:
            continue
        d_gpu = s.delta_energy([a, b], [lt[b], lt[a]])
        d_or = o.swap_dE(st["pos_u"], lt, a, b)
        assert abs(d_gpu - d_or) < DE_TOL, (a, b, d_gpu, d_or)
        n += 1


@pytest.mark.parametrize("path", ["speculative", "sequential"])
@pytest.mark.parametrize("which", ["small", "large"])
def test_batched_trials_equal_sequential_oracle(which, path, small, large):
    """mdas_swap_trials evaluates trials in speculative rounds or one after
    another from the pair lists; either outcome must equal the oracle's
    one-after-another processing (Sec. 2, Eq. 1)."""
    m = small if which == "small" else large
    s = mdas.System(m, temperature=600.0)
    s.set_trial_path(path)
    st0 = s.get_state()
    stats, rec = s.swap_trials(256)
    o = oracle.Oracle(m, temperature=600.0)
    lt_o, rec_o = o.swap_trials(st0["pos_u"], st0["ltype"], st0["trial"], 256)
    ties = 0
    for g, r in zip(rec, rec_o):
        assert (g["a"], g["b"], bool(g["null"])) == (r["a"], r["b"], r["null"])
        assert g["u"] == r["u"]
        if r["null"]:
            continue
        assert abs(g["dE"] - r["dE"]) < DE_TOL
        if abs(r["dE"] + o.kT * math.log(r["u"])) < DE_TOL:
            ties += 1
        else:
            assert bool(g["accepted"]) == r["accepted"]
    assert ties == 0
    st1 = s.get_state()
    assert np.array_equal(st1["ltype"], lt_o)
    assert np.array_equal(st1["pos_u"], st0["pos_u"])
    assert stats["accepted"] > 0 and stats["trials"] == 256
    assert np.array_equal(np.bincount(st1["ltype"]), np.bincount(st0["ltype"]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_step_map(prec, small):
    """Oracle step applied to the GPU state at step n vs the GPU state at n+1."""
    s = mdas.System(small, precision=prec)
    s.md_steps(10)
    st = s.get_state()
    s.md_steps(1)
    st1 = s.get_state()
    o = oracle.Oracle(small)
    so = o.state(pos_u=st["pos_u"], vel=st["vel"], ltype=st["ltype"], step=st["step"])
    o.md_steps(so, 1)
    dpos = np.abs((st1["pos_u"].astype(np.int64) - so["pos_u"].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
    dv = np.abs(st1["vel"] - so["vel"]).max()
    if prec == "fp64":
        assert dpos.max() <= 1 and dv < 1e-10, (dpos.max(), dv)
    else:
        assert dpos.max() <= 256 and dv < 2e-5, (dpos.max(), dv)


@pytest.mark.parametrize("lanes", [4, 2])
def test_fp64_trajectory_with_trials(small, lanes):
    """200 steps at 20 fs with a trial every 10 steps, FP64 (the 128-lipid MC-MD
    workload), both step shapes: trial decisions identical, states close at
    the end."""
    s = mdas.System(small, precision="fp64")
    s.set_list_lanes(lanes)
    s.md_steps(200, swap_every=10)
    st = s.get_state()
    rec = s.trial_log(0, 20)
    o = oracle.Oracle(small)
    so = o.state()
    rec_o = o.md_steps(so, 200, swap_every=10)
    for g, r in zip(rec, rec_o):
        assert (g["a"], g["b"], bool(g["null"]), bool(g["accepted"])) == (r["a"], r["b"], r["null"], r["accepted"])
        if not r["null"]:
            assert abs(g["dE"] - r["dE"]) < DE_TOL
    assert np.array_equal(st["ltype"], so["ltype"])
    dx = np.abs((st["pos_u"].astype(np.int64) - so["pos_u"].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
    dx_nm = (dx * (small.box / 2 ** 32)[None, :]).max()
    assert dx_nm < 1e-6, dx_nm
    e = s.energy()
    to, _ = o.energy(so["pos_u"], ltype=so["ltype"], forces=False)
    assert e["potential"] == pytest.approx(to["total"], rel=1e-7)


def test_mdas_single_step_equals_exchange(large):
    """Sec. 2: delta-lambda = 1, M = 0 is the MC exchange: w equals dE."""
    s = mdas.System(large)
    st = s.get_state()
    lt = st["ltype"]
    a = 0
    b = int(np.nonzero(lt != lt[a])[0][0])
    d = oracle.Oracle(large).swap_dE(st["pos_u"], lt, a, b)
    res = s.alchemical_move(1, 1, 0, pairs=[[a, b]])
    assert abs(res["w"] - d) < DE_TOL
    assert res["accepted"] == (res["w"] + s.kT * math.log(res["u"]) <= 0)
    st1 = s.get_state()
    assert np.array_equal(st1["pos_u"], st["pos_u"])
    if res["accepted"]:
        assert st1["ltype"][a] == lt[b] and st1["ltype"][b] == lt[a]
    else:
        assert np.array_equal(st1["ltype"], lt)


@pytest.mark.parametrize("K,M", [(3, 2), (4, 0)])
def test_mdas_move_matches_oracle(K, M):
    m = synth.mcmd_small(seed=2024)
    s = mdas.System(m, precision="fp64")
    o = oracle.Oracle(m)
    so = o.state()
    for _ in range(3):
        res = s.alchemical_move(8, K, M)
        ro = o.mdas_move(so, 8, K, M)
        assert np.array_equal(res["pairs"], ro["pairs"])
        assert abs(res["w"] - ro["w"]) < DE_TOL, (res["w"], ro["w"])
        assert res["u"] == ro["u"] and res["accepted"] == ro["accepted"]
        st = s.get_state()
        assert np.array_equal(st["ltype"], so["ltype"])
        dx = np.abs((st["pos_u"].astype(np.int64) - so["pos_u"].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
        assert dx.max() <= 2
        assert st["move"] == so["move"] and st["at_step"] == so["at_step"]


def test_lambda_forces_linear(small):
    """U(l) = (1-l) U_A + l U_B: delta energy of the B types equals U_B - U_A."""
    s = mdas.System(small, precision="fp64")
    st = s.get_state()
    lt = st["ltype"].copy()
    lipids = np.arange(6)
    newt = 1 - lt[:6]
    d = s.delta_energy(lipids, newt)
    o = oracle.Oracle(small)
    ltB = lt.copy()
    ltB[:6] = newt
    eA = o.energy(st["pos_u"], ltype=lt, forces=False)[0]["total"]
    eB = o.energy(st["pos_u"], ltype=ltB, forces=False)[0]["total"]
    assert abs(d - (eB - eA)) < DE_TOL


def test_deterministic_rerun(large):
    out = []
    for _ in range(2):
        s = mdas.System(large)
        s.md_steps(30, swap_every=3)
        st = s.get_state()
        out.append((st["pos_u"].tobytes(), st["vel"].tobytes(), st["ltype"].tobytes()))
        s.close()
    assert out[0] == out[1]


@pytest.mark.parametrize("lanes,path", [(4, "speculative"), (2, "speculative"), (4, "sequential")])
def test_batch_equals_solo(lanes, path):
    ms = [synth.patch(n, 2 + (n % 2), seed=50 + n, system_id=k) for k, n in enumerate([130, 258, 400])]
    solo = []
    for m in ms:
        s = mdas.System(m)
        s.set_list_lanes(lanes)
        s.set_trial_path(path)
        s.md_steps(12)
        s.swap_trials(20, log=False)
        st = s.get_state()
        solo.append(st)
        s.close()
    sy = [mdas.System(m) for m in ms]
    for s in sy:
        s.set_list_lanes(lanes)
        s.set_trial_path(path)
    mdas.batch_run(sy, 12, 20)
    for s, st in zip(sy, solo):
        b = s.get_state()
        assert np.array_equal(b["pos_u"], st["pos_u"])
        assert np.array_equal(b["vel"], st["vel"])
        assert np.array_equal(b["ltype"], st["ltype"])


def test_water_only_and_ragged_sizes():
    m = synth.membrane(5, n_lipid_types=1, n_water=333, seed=9, n_lipids=0)
    s = mdas.System(m)
    s.md_steps(5)
    st = s.get_state()
    F = s.forces()
    _, Fo = oracle.Oracle(m).energy(st["pos_u"], ltype=st["ltype"])
    assert force_err(F, Fo) < F_TOL
    stats, _ = s.swap_trials(4)
    assert stats["trials"] == 0


def test_nonfinite_state_is_reported_not_trapped(small):
    s = mdas.System(small)
    st = s.get_state()
    v = st["vel"].copy()
    v[5, 1] = np.nan
    s.set_state(pos_u=st["pos_u"], vel=v, ltype=st["ltype"])
    with pytest.raises(mdas.MdasError) as e:
        s.md_steps(2)
    assert e.value.status == 4
    with pytest.raises(mdas.MdasError):
        s.md_steps(1)
    s.set_state(pos_u=st["pos_u"], vel=st["vel"], ltype=st["ltype"])
    s.md_steps(2)


def test_nve_drift_within_twice_the_oracles(small):
    """NVE (no thermostat), 1000 steps of 10 fs on the 128-lipid bilayer from
    the same start: the total energy of the FP32 GPU trajectory strays from
    its start and drifts (slope of a linear fit over the run) no more than
    twice as much as the FP64 oracle's over the same steps; no secular
    blow-up."""
    dt, n, every = 0.01, 1000, 50
    s = mdas.System(small, precision="fp32", tau_t=0.0, dt=dt)
    o = oracle.Oracle(small, tau_t=0.0, dt=dt)
    so = o.state()

    def e_or():
        u = o.energy(so["pos_u"], ltype=so["ltype"], forces=False)[0]["total"]
        return u + 0.5 * small.mass * (so["vel"] ** 2).sum()

    eg, eo = [s.energy()["total"]], [e_or()]
    for _ in range(n // every):
        s.md_steps(every)
        eg.append(s.energy()["total"])
        o.md_steps(so, every)
        eo.append(e_or())

    def stray_and_drift(e):
        e = np.asarray(e)
        t = np.arange(len(e)) * every
        return np.abs(e - e[0]).max(), abs(np.polyfit(t, e, 1)[0]) * n

    sg, dg = stray_and_drift(eg)
    so_, do_ = stray_and_drift(eo)
    assert abs(eg[0] - eo[0]) < 1e-6 * abs(eo[0])
    assert sg <= 2.0 * so_, (sg, so_, eg, eo)
    assert dg <= 2.0 * max(do_, so_), (dg, do_, so_)


def test_mdas_move_full_size_matches_oracle():
    """The MDAS workload at full size: 4608-lipid bilayer (~140k beads), a move
    of 8 pairs (16 lipids) over 10 lambda steps of 5 MD steps each, FP64."""
    m = synth.mdas_patch()
    s = mdas.System(m, precision="fp64")
    o = oracle.Oracle(m)
    so = o.state()
    res = s.alchemical_move(8, 10, 5)
    ro = o.mdas_move(so, 8, 10, 5)
    assert np.array_equal(res["pairs"], ro["pairs"])
    assert abs(res["w"] - ro["w"]) < DE_TOL, (res["w"], ro["w"])
    assert res["u"] == ro["u"] and res["accepted"] == ro["accepted"]
    st = s.get_state()
    assert np.array_equal(st["ltype"], so["ltype"])
    dx = np.abs((st["pos_u"].astype(np.int64) - so["pos_u"].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
    assert dx.max() <= 4, dx.max()
    assert st["move"] == so["move"] and st["at_step"] == so["at_step"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_device_views_read_the_state_without_copies(prec, small):
    """mdas_device_ptrs: torch tensors over the library's own arrays hold the
    state get_state copies out, and follow the next call without a copy."""
    s = mdas.System(small, precision=prec)
    s.md_steps(7, swap_every=7)
    v = s.device_views()
    st = s.get_state()
    pos = v["pos"].cpu().numpy().view(np.uint32)
    assert np.array_equal(pos[:, :3], st["pos_u"])
    o = oracle.Oracle(small)
    assert np.array_equal(pos[:, 3] & 15, o.bead_types(st["ltype"]))
    assert np.array_equal(v["vel"].cpu().numpy()[:, :3].astype(np.float64), st["vel"])
    assert np.array_equal(v["ltype"].cpu().numpy(), st["ltype"])
    assert np.array_equal(v["box"], small.box)
    s.md_steps(3)
    assert np.array_equal(v["pos"].cpu().numpy().view(np.uint32)[:, :3], s.get_state()["pos_u"])
    assert v["pos"].data_ptr() == s.device_views()["pos"].data_ptr()
