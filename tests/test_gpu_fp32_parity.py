"""CUDA path vs the FP64 oracle at the precision the benchmarks run: FP32 pair
arithmetic (positions in fixed point, FP64 energy changes and work sums).

- MDAS moves (Sec. 2, Eqs. 2-3) in FP32, laid open block by block
  (mdas_alchemical_move_trace): every lambda block's work equals the oracle's
  U_{lambda_k}(x_k) - U_{lambda_k-1}(x_k) on the GPU's own x_k within 1e-4
  kJ/mol, and the FP32 step forces at intermediate lambda equal the oracle's
  forces of U(lambda) within 1e-5 (linear and soft-core paths, on the
  128-lipid bilayer and on the full 4608-lipid MDAS workload).
- The in-MD exchange trials of the 1152-lipid MC-MD workload (one trial after
  every MD step, FP32), replayed on the oracle: the same proposals, dE within
  1e-4 kJ/mol on the GPU's pre-trial state, the same decisions except within
  1e-4 of the Metropolis boundary (counted), the same types.
- FP64 energies of the 1152-lipid workload; batches of replicas of 128-2048
  lipids equal to their solo runs, with one replica's batched trials in
  lockstep with the oracle.
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


def _types_AB(o, ltype, pairs):
    ltB = np.array(ltype, np.int32).copy()
    for a, b in pairs:
        ltB[a], ltB[b] = ltype[b], ltype[a]
    return o.bead_types(ltype), o.bead_types(ltB)


@pytest.mark.parametrize("soft", [0.0, 0.05])
def test_traced_move_gives_the_bits_of_the_move(soft):
    """Laying the trajectory open block by block changes nothing: the same
    work, decision and final state as the single-run move (FP32)."""
    m = synth.mcmd_small(seed=2024)
    out = []
    for traced in (False, True):
        s = mdas.System(m, precision="fp32")
        if soft:
            s.set_soft_core(soft)
        s.md_steps(10)
        res = [s.alchemical_move_trace(4, 5, 3) if traced else s.alchemical_move(4, 5, 3) for _ in range(2)]
        out.append((res, s.get_state()))
    (ra, sa), (rb, sb) = out
    for x, y in zip(ra, rb):
        assert x["w"] == y["w"] and x["accepted"] == y["accepted"]
        assert np.array_equal(x["pairs"], y["pairs"])
    assert np.array_equal(sa["pos_u"], sb["pos_u"]) and np.array_equal(sa["vel"], sb["vel"])
    assert np.array_equal(sa["ltype"], sb["ltype"])
    w = rb[0]
    assert w["w"] == pytest.approx(w["w_blocks"].sum(), abs=1e-9)


def _block_work_parity(m, soft, n_pairs, K, M):
    s = mdas.System(m, precision="fp32")
    o = oracle.Oracle(m, soft_core=soft)
    if soft:
        s.set_soft_core(soft)
    s.md_steps(5)
    st = s.get_state()
    res = s.alchemical_move_trace(n_pairs, K, M, velocities=False)
    btA, btB = _types_AB(o, st["ltype"], res["pairs"])
    assert (btA != btB).any()
    worst = 0.0
    for k in range(K):
        dw = o.work_increment(res["pos_blocks"][k], btA, btB, k / K, (k + 1) / K)
        worst = max(worst, abs(res["w_blocks"][k] - dw))
    assert worst < DE_TOL, worst
    assert res["w"] == pytest.approx(res["w_blocks"].sum(), abs=1e-9)
    return res


@pytest.mark.parametrize("soft", [0.0, 0.05])
def test_fp32_block_work_matches_oracle_small(soft):
    _block_work_parity(synth.mcmd_small(seed=2024), soft, 8, 6, 3)


@pytest.mark.parametrize("soft", [0.0, 0.05])
def test_fp32_block_work_matches_oracle_full_size(soft):
    """The MDAS workload as benchmarked: 4608 lipids (~140k beads), 8 pairs,
    10 lambda steps of 5 MD steps, FP32 pair arithmetic, FP64 work."""
    _block_work_parity(synth.mdas_patch(), soft, 8, 10, 5)


def _lambda_force_parity(m, soft, n_pairs, K, blocks):
    """From rest without a thermostat, with one MD step per lambda block, block
    b's step gives v_{b+1} = v_b + F_{lambda_b}(x_b) dt / m: the FP32 step
    forces of U(lambda_b) at intermediate lambda, compared with the oracle's."""
    s = mdas.System(m, precision="fp32", tau_t=0.0)
    o = oracle.Oracle(m, soft_core=soft)
    if soft:
        s.set_soft_core(soft)
    s.md_steps(5)
    st = s.get_state()
    s.set_state(pos_u=st["pos_u"], vel=np.zeros_like(st["vel"]), ltype=st["ltype"], step=st["step"],
                trial=st["trial"], move=st["move"], at_step=st["at_step"])
    res = s.alchemical_move_trace(n_pairs, K, 1)
    btA, btB = _types_AB(o, st["ltype"], res["pairs"])
    worst = 0.0
    for b in blocks:
        assert 1 <= b < K
        F = (res["vel_blocks"][b] - res["vel_blocks"][b - 1]) * (m.mass / m.dt)
        _, Fo = o.energy(res["pos_blocks"][b - 1], btA=btA, btB=btB, lam=b / K)
        worst = max(worst, force_err(F, Fo))
    assert worst < F_TOL, worst


@pytest.mark.parametrize("soft", [0.0, 0.05])
def test_fp32_lambda_step_forces_match_oracle_small(soft):
    _lambda_force_parity(synth.mcmd_small(seed=2024), soft, 8, 4, [1, 2, 3])


def test_fp32_lambda_step_forces_match_oracle_full_size():
    _lambda_force_parity(synth.mdas_patch(), 0.0, 8, 4, [2])


def test_fp32_in_md_trials_replay_on_the_oracle():
    """The 1152-lipid MC-MD workload as benchmarked (FP32, one exchange trial
    after every MD step, the trial running beside the next step in the
    persistent kernel).  The run split at every trial gives the same bits;
    each trial's dE, recomputed by the oracle on the GPU's pre-trial state,
    agrees within 1e-4 kJ/mol and so does the decision, except within 1e-4
    of the Metropolis boundary (counted)."""
    m = synth.mcmd_large()
    n = 60
    a = mdas.System(m, precision="fp32")
    a.md_steps(n, swap_every=1)
    rec = a.trial_log(0, n)
    fa = a.get_state()
    b = mdas.System(m, precision="fp32")
    pre = []
    lt_prev = b.get_state()["ltype"]
    for _ in range(n):
        b.md_steps(1, swap_every=1)
        st = b.get_state()
        pre.append((st["pos_u"], lt_prev))
        lt_prev = st["ltype"]
    fb = b.get_state()
    assert np.array_equal(fa["pos_u"], fb["pos_u"]) and np.array_equal(fa["ltype"], fb["ltype"])
    assert np.array_equal(rec, b.trial_log(0, n))
    o = oracle.Oracle(m)
    ties = accepted = 0
    for r, (pu, lt) in zip(rec, pre):
        pa, pb, u = o.swap_proposal(int(r["index"]))
        assert (int(r["a"]), int(r["b"]), float(r["u"])) == (pa, pb, u)
        null = pa == pb or lt[pa] == lt[pb]
        assert bool(r["null"]) == null
        nxt = lt.copy()
        if not null:
            d = o.swap_dE(pu, lt, pa, pb)
            assert abs(float(r["dE"]) - d) < DE_TOL, (r, d)
            if abs(d + o.kT * math.log(u)) < DE_TOL:
                ties += 1
            else:
                assert bool(r["accepted"]) == (d + o.kT * math.log(u) <= 0)
            if r["accepted"]:
                nxt[pa], nxt[pb] = lt[pb], lt[pa]
                accepted += 1
    assert accepted > 0
    assert ties == 0
    # the types follow the records
    for (pu, lt), (pu2, lt2), r in zip(pre[:-1], pre[1:], rec[:-1]):
        exp = lt.copy()
        if r["accepted"]:
            exp[r["a"]], exp[r["b"]] = lt[r["b"]], lt[r["a"]]
        assert np.array_equal(exp, lt2)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_energy_matches_oracle_large(prec):
    m = synth.mcmd_large()
    s = mdas.System(m, precision=prec)
    s.md_steps(3)
    st = s.get_state()
    e = s.energy()
    to, _ = oracle.Oracle(m).energy(st["pos_u"], ltype=st["ltype"], forces=False)
    assert e["pairs"] == to["pairs"]
    for k in ("lj", "rf", "bond", "angle"):
        assert abs(e[k] - to[k]) <= E_TOL * abs(to["total"]), (k, e[k], to[k])
    assert e["potential"] == pytest.approx(to["total"], rel=E_TOL)


def test_batch_of_replicas_128_to_2048_lipids():
    """Eight replicas spanning the batched workload's sizes (128-2048 lipids,
    2 and 3 types) advance in one batch exactly as they do alone (FP32 bits),
    and one replica's batched exchange trials match the oracle's sequential
    trials on its post-MD state."""
    sizes = [128, 300, 512, 800, 1100, 1400, 1700, 2048]
    ms = [synth.patch(n, 2 + (k % 2), seed=70 + k, system_id=k) for k, n in enumerate(sizes)]
    solo = []
    for m in ms:
        s = mdas.System(m)
        s.md_steps(12)
        s.swap_trials(24, log=False)
        s.md_steps(7)
        s.swap_trials(16, log=False)
        solo.append(s.get_state())
        s.close()
    sy = [mdas.System(m) for m in ms]
    mdas.batch_run(sy, 12, 0)
    x = 2                                         # the 512-lipid replica
    post_md = sy[x].get_state()
    mdas.batch_run(sy, 0, 24)
    mid = sy[x].get_state()
    mdas.batch_run(sy, 7, 16)                     # a second round: the trial counters must have kept step
    for s, st in zip(sy, solo):
        g = s.get_state()
        assert np.array_equal(g["pos_u"], st["pos_u"])
        assert np.array_equal(g["vel"], st["vel"])
        assert np.array_equal(g["ltype"], st["ltype"])
        assert (g["step"], g["trial"]) == (st["step"], st["trial"])
    o = oracle.Oracle(ms[x])
    lt_o, rec_o = o.swap_trials(post_md["pos_u"], post_md["ltype"], post_md["trial"], 24)
    rec = sy[x].trial_log(post_md["trial"], 24)
    ties = 0
    for g, r in zip(rec, rec_o):
        assert (int(g["a"]), int(g["b"]), bool(g["null"]), float(g["u"])) == (r["a"], r["b"], r["null"], r["u"])
        if r["null"]:
            continue
        assert abs(float(g["dE"]) - r["dE"]) < DE_TOL
        if abs(r["dE"] + o.kT * math.log(r["u"])) < DE_TOL:
            ties += 1
        else:
            assert bool(g["accepted"]) == r["accepted"]
    assert ties == 0
    assert np.array_equal(mid["ltype"], lt_o)
