"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks a fact that does not come from the oracle itself: published
known-answer vectors, closed forms at special points, limits, invariants,
brute force, finite differences and exact enumeration.  A dropped term, a
wrong sign or a transposed index in oracle.c fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2005_08348_gb300 import synth
from tests._systems import beads, pair_distances

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIG = 0.47
RC = 1.1
F_COUL = 138.935458


def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors (SC'11)."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert oracle.philox(v[:4], v[4:6]) == v[6:10]
        n += 1
    assert n == 3


def _two(r, ta, tb, **kw):
    m = beads([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]], [ta, tb], box=(5.0, 5.0, 5.0), **kw)
    return m, oracle.Oracle(m)


def _u(r, ta, tb, **kw):
    m, o = _two(r, ta, tb, **kw)
    t, F = o.energy(m.pos_u, cells=False)
    return t, F, m


def test_lj_minimum_and_depth():
    """Neutral pair: the force vanishes at 2^(1/6) sigma and the well depth
    below the cutoff value is eps (Sec. 3: LJ with potential shift)."""
    ta, tb = synth.BT_C1, synth.BT_C3
    rmin = 2 ** (1 / 6) * SIG
    t, F, m = _u(rmin, ta, tb)
    eps = m.eps[ta, tb]
    # position quantisation moves r by < 1e-9 nm: the force there is < 1e-6
    assert abs(F[0, 0]) < 1e-5
    # a golden-section search on the oracle's own energies lands on 2^(1/6) sigma
    a, b = 0.50, 0.56
    g = (math.sqrt(5) - 1) / 2
    for _ in range(60):
        c, d = b - g * (b - a), a + g * (b - a)
        if _u(c, ta, tb)[0]["lj"] < _u(d, ta, tb)[0]["lj"]:
            b = d
        else:
            a = c
    assert abs(0.5 * (a + b) - rmin) < 2e-6
    # depth: u(rmin) - u(rc-) equals -eps plus the unshifted tail at rc, which
    # for sigma/rc = 0.4273 is +0.02419 eps
    s6 = (SIG / RC) ** 6
    u_rc = _u(RC * (1 - 1e-12), ta, tb)[0]["lj"]
    assert abs(u_rc) < 1e-9
    assert t["lj"] == pytest.approx(-eps * (1 - 4 * (s6 - s6 * s6)), rel=1e-9)
    assert 4 * (s6 - s6 * s6) == pytest.approx(0.024190, abs=2e-6)
    assert t["rf"] == 0.0 and t["pairs"] == 1


def test_lj_repulsive_wall_sign():
    """Inside sigma the LJ force pushes the beads apart; past rmin it pulls."""
    _, F, _ = _u(0.42, synth.BT_C1, synth.BT_C1)
    assert F[0, 0] < 0 < F[1, 0]          # bead 0 is at smaller x
    _, F, _ = _u(0.8, synth.BT_C1, synth.BT_C1)
    assert F[0, 0] > 0 > F[1, 0]


def test_reaction_field_limits():
    """RF (eps_r = 15, eps_rf = infinity): Coulomb at short range, zero energy
    and zero force at the cutoff (conducting boundary)."""
    zero = np.zeros((10, 10))
    # Coulomb limit: u r -> f q1 q2 / eps_r for r -> 0
    r = 1e-3
    t, F, _ = _u(r, synth.BT_QP, synth.BT_QN, eps=zero)
    assert t["rf"] * r == pytest.approx(-F_COUL / 15.0, rel=2e-3)
    assert t["lj"] == 0.0
    # attraction of opposite charges
    assert F[0, 0] > 0
    # zero energy and force at rc
    t, F, _ = _u(RC * (1 - 1e-9), synth.BT_QP, synth.BT_QN, eps=zero)
    assert abs(t["rf"]) < 1e-7
    assert abs(F[0, 0]) < 1e-6
    # with eps_rf = eps_r the RF correction vanishes: plain Coulomb shifted to 0 at rc
    t, F, m = _u(0.5, synth.BT_QP, synth.BT_QP, eps=zero, eps_rf=15.0)
    x = synth.dequantize(m.pos_u, m.box)
    r = x[1, 0] - x[0, 0]                       # the quantised separation
    assert t["rf"] == pytest.approx(F_COUL / 15.0 * (1 / r - 1 / RC), rel=1e-12)
    assert F[1, 0] == pytest.approx(F_COUL / 15.0 / r ** 2, rel=1e-12)


def test_cutoff():
    """Every type pair's LJ+RF energy reaches zero at rc and is zero beyond."""
    for ta in range(7):
        for tb in range(7):
            t, _, _ = _u(RC * (1 - 1e-11), ta, tb)
            assert abs(t["total"]) < 1e-8
            t, F, _ = _u(RC * (1 + 1e-6), ta, tb)
            assert t["total"] == 0.0 and not F.any() and t["pairs"] == 0


def test_net_force_zero():
    m = synth.tiny(seed=11)
    o = oracle.Oracle(m)
    _, F = o.energy(m.pos_u)
    frms = np.sqrt((F * F).sum(1).mean())
    assert np.abs(F.sum(0)).max() <= 1e-12 * frms * m.n_beads


@pytest.mark.parametrize("lam", [0.0, 0.37, 1.0])
def test_forces_match_energy_gradient(lam):
    """Central finite differences of U(lambda) match F = -grad U (1e-6 rel)."""
    m = synth.tiny(seed=21)
    o = oracle.Oracle(m)
    ltB = m.lipid_type.copy()
    ltB[0], ltB[1] = m.lipid_type[1], m.lipid_type[0]
    ltB[2], ltB[3] = 1 - ltB[2], 1 - ltB[3]
    btA, btB = o.bead_types(m.lipid_type), o.bead_types(ltB)
    r = pair_distances(synth.dequantize(m.pos_u, m.box), m.box)
    assert np.abs(r - RC).min() > 2e-5          # no pair straddles the cutoff under +-h (h ~ 1e-6)
    _, F = o.energy(m.pos_u, btA=btA, btB=btB, lam=lam)
    rng = np.random.default_rng(3)
    k = 1 << 10                                  # h = k L / 2^32 ~ 1e-6 nm
    worst = 0.0
    frms = np.sqrt((F * F).sum(1).mean())
    for i in rng.choice(m.n_beads, 30, replace=False):
        for d in range(3):
            h = k * m.box[d] / 2 ** 32
            p, q = m.pos_u.copy(), m.pos_u.copy()
            p[i, d] += np.uint32(k)
            q[i, d] -= np.uint32(k)
            up = o.energy(p, btA=btA, btB=btB, lam=lam, forces=False)[0]["total"]
            um = o.energy(q, btA=btA, btB=btB, lam=lam, forces=False)[0]["total"]
            fd = -(up - um) / (2 * h)
            worst = max(worst, abs(fd - F[i, d]) / max(abs(F[i, d]), frms))
    assert worst < 1e-6


def test_bonded_rest_state_and_restoring():
    """A straight rod at bond length b0 has zero bond and angle energy; a
    stretched bond pulls back and a bent angle pushes back toward 180 deg."""
    m = synth.membrane(3, n_lipid_types=1, n_water=0, seed=2, n_lipids=2, jitter=0.0)
    o = oracle.Oracle(m)
    t, _ = o.energy(m.pos_u)
    assert t["bond"] < 1e-9 and t["angle"] < 1e-12
    p = m.pos_u.copy()
    p[0, 2] += np.uint32(int(0.05 / m.box[2] * 2 ** 32))    # stretch bond 0-1 (bead 0 is the top)
    t, F = o.energy(p)
    assert t["bond"] == pytest.approx(0.5 * 1250 * 0.05 ** 2, rel=1e-6)
    assert F[0, 2] < 0
    p = m.pos_u.copy()
    p[1, 0] += np.uint32(int(0.1 / m.box[0] * 2 ** 32))     # bend bead 1 sideways
    t, F = o.energy(p)
    assert t["angle"] > 0 and F[1, 0] < 0


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_cell_list_sum_equals_brute_force(seed):
    m = synth.tiny(n_side=2, n_water=60, seed=seed)
    assert min(m.box) >= 3 * RC and m.n_beads <= 200
    o = oracle.Oracle(m)
    tb, Fb = o.energy(m.pos_u, cells=False)
    tc, Fc = o.energy(m.pos_u, cells=True)
    assert tb["pairs"] == tc["pairs"]
    assert tc["total"] == pytest.approx(tb["total"], rel=1e-12)
    assert np.abs(Fb - Fc).max() <= 1e-12 * np.abs(Fb).max()


def test_cell_list_is_stable_counting_sort():
    m = synth.mcmd_small()
    o = oracle.Oracle(m)
    nc = o.cell_dims()
    cell_of, srt, start = o.cell_list(m.pos_u)
    c = (m.pos_u.astype(np.uint64) * np.array(nc, np.uint64)) >> np.uint64(32)
    cid = (c[:, 2] * nc[1] + c[:, 1]) * nc[0] + c[:, 0]
    assert np.array_equal(cid.astype(np.int32), cell_of)
    assert np.array_equal(np.lexsort((np.arange(m.n_beads), cid)), srt)
    assert np.array_equal(np.searchsorted(np.sort(cid), np.arange(len(start)), "left"), start)


def test_swap_dE_equals_difference_of_full_energies():
    for m in (synth.tiny(seed=41, n_lipid_types=2), synth.tiny(seed=42, n_lipid_types=3)):
        o = oracle.Oracle(m)
        lt = m.lipid_type
        U = abs(o.energy(m.pos_u, forces=False)[0]["total"])
        n = 0
        for a in range(m.n_lipids):
            for b in range(a + 1, m.n_lipids):
                if lt[a] == lt[b]:
                    continue
                d1 = o.swap_dE(m.pos_u, lt, a, b)
                d2 = o.swap_dE_full(m.pos_u, lt, a, b)
                assert d1 == pytest.approx(d2, abs=1e-9 * U)
                n += 1
        assert n > 0


def test_swaps_keep_coordinates_and_composition():
    """Sec. 2: an exchange changes potential parameters only; composition is
    conserved by exchanging a pair."""
    m = synth.mcmd_small()
    o = oracle.Oracle(m, temperature=3000.0)
    before = m.pos_u.copy()
    lt, recs = o.swap_trials(m.pos_u, m.lipid_type, 0, 200)
    assert np.array_equal(before, m.pos_u)
    assert np.array_equal(np.bincount(lt, minlength=3), np.bincount(m.lipid_type, minlength=3))
    assert any(r["accepted"] for r in recs) and any(r["null"] for r in recs)
    for r in recs:
        assert r["null"] == (r["a"] == r["b"] or r["null"])


def test_metropolis_rule():
    """Eq. 1: a non-null trial is accepted iff u <= exp(-dE/kT)."""
    m = synth.tiny(seed=43)
    o = oracle.Oracle(m, temperature=2000.0)
    lt, recs = o.swap_trials(m.pos_u, m.lipid_type, 0, 400)
    seen = set()
    for r in recs:
        if r["null"]:
            assert not r["accepted"]
            continue
        seen.add(r["accepted"])
        assert r["accepted"] == (r["u"] <= math.exp(-r["dE"] / o.kT))
    assert seen == {True, False}


def test_mdas_single_step_is_mc_exchange():
    """Sec. 2: MDAS with delta-lambda = 1 and M = 0 is one MC exchange: the
    work equals the swap dE and the decision is the Metropolis one."""
    m = synth.tiny(seed=44)
    o = oracle.Oracle(m)
    st = o.state()
    lt = m.lipid_type
    a, b = [(a, b) for a in range(m.n_lipids) for b in range(m.n_lipids) if lt[a] != lt[b]][0]
    res = o.mdas_move(st, 1, 1, 0, pairs=[[a, b]])
    assert res["w"] == pytest.approx(o.swap_dE(m.pos_u, lt, a, b), abs=1e-9)
    assert res["accepted"] == (res["w"] + o.kT * math.log(res["u"]) <= 0)
    assert np.array_equal(st["pos_u"], m.pos_u)


@pytest.mark.parametrize("K", [1, 4, 10])
def test_mdas_work_without_dynamics_is_the_exchange_energy(K):
    """With M = 0 the coordinates stay put, so Eq. 2 telescopes to
    U_B(x0) - U_A(x0) for any number of lambda steps."""
    m = synth.tiny(seed=45, n_lipid_types=3)
    o = oracle.Oracle(m)
    lt = m.lipid_type
    pairs = o.mdas_pairs(lt, 0, 2)
    assert len(pairs) == 2
    ltB = lt.copy()
    for a, b in pairs:
        ltB[a], ltB[b] = lt[b], lt[a]
    dU = o.energy(m.pos_u, ltype=ltB, forces=False)[0]["total"] - o.energy(m.pos_u, ltype=lt, forces=False)[0]["total"]
    st = o.state()
    res = o.mdas_move(st, 2, K, 0)
    assert np.array_equal(res["pairs"], pairs)
    assert res["w"] == pytest.approx(dU, abs=1e-9 * abs(dU) + 1e-9)


def _free_flight_system():
    """Three one-bead lipids, no charges, no bonds.  Only bead types 1 and 2
    interact (eps 3 kJ/mol).  Lipid a (type 0) flies at 2.5 nm/ps towards the
    resting probe X (type 2), from 1.3 nm; lipid b (type 1) rests 1.6 nm from
    X.  In state A nothing is within rc of a partner it interacts with, so
    every bead moves in a straight line.  Exchanging a and b makes a interact
    with X."""
    eps = np.zeros((10, 10))
    eps[1, 2] = eps[2, 1] = 3.0
    m = beads([[0.7, 2.0, 2.0], [2.0, 3.6, 2.0], [2.0, 2.0, 2.0]], [0, 1, 2], box=(4.0, 4.0, 4.0), eps=eps,
              charge=np.zeros(10))
    m.vel = np.zeros((3, 3))
    m.vel[0, 0] = 2.5
    return m


def test_mdas_work_is_taken_after_each_block():
    """Eq. 2 with dynamics (M > 0): the work of a lambda step is
    U_{lam_k}(x_k) - U_{lam_k-1}(x_k) at the coordinates x_k reached *after*
    the block's M steps.  In free flight (thermostat off, no force in state
    A) x_1 = x_0 + M rint(v dt 2^32 / L) exactly.  After 8 steps a is 0.9 nm
    from X, inside rc, so w is the shifted Lennard-Jones energy there; at
    x_0 it was 1.3 nm away, so taking the work before the block would give
    exactly 0."""
    m = _free_flight_system()
    o = oracle.Oracle(m, tau_t=0.0)
    M = 8
    q = m.dt * 2 ** 32 / m.box[0]
    x1 = m.pos_u.astype(np.int64)
    x1[0, 0] = (x1[0, 0] + M * int(np.rint(2.5 * q))) % 2 ** 32
    x1 = x1.astype(np.uint32)
    st = o.state()
    res = o.mdas_move(st, 1, 1, M, pairs=[[0, 1]], cells=False)
    btA, btB = o.bead_types([0, 1, 2]), o.bead_types([1, 0, 2])
    uA1 = o.energy(x1, btA=btA, cells=False, forces=False)[0]["total"]
    uB1 = o.energy(x1, btA=btB, cells=False, forces=False)[0]["total"]
    uA0 = o.energy(m.pos_u, btA=btA, cells=False, forces=False)[0]["total"]
    uB0 = o.energy(m.pos_u, btA=btB, cells=False, forces=False)[0]["total"]
    assert uA1 == 0.0 and uA0 == 0.0 and uB0 == 0.0
    r = float((int(x1[2, 0]) - int(x1[0, 0])) * (m.box[0] / 2 ** 32))
    assert 0.85 < r < 0.95
    lj = lambda x: 4 * 3.0 * ((SIG / x) ** 12 - (SIG / x) ** 6)
    assert res["w"] == pytest.approx(lj(r) - lj(RC), rel=1e-12)
    assert res["w"] == pytest.approx(uB1 - uA1, abs=1e-12)
    assert res["w"] < -0.1                               # the before-the-block reading gives uB0 - uA0 = 0
    assert res["accepted"]                                # w < 0
    assert np.array_equal(st["pos_u"], x1)
    assert st["at_step"] == M


@pytest.mark.parametrize("nf", [3, 4, 7])
def test_bussi_fast_coupling_draws_the_canonical_kinetic_energy(nf):
    """Bussi et al. (2007) at tau_T -> 0 (c = exp(-dt / tau_T) = 0): the new
    kinetic energy is drawn from the canonical distribution of Nf degrees of
    freedom itself, K_new = (K_t / Nf) chi2(Nf), because R1^2 and the
    chi2(Nf - 1) variate together make Nf squared normals.  A chi2(Nf) in
    place of chi2(Nf - 1) gives chi2(Nf + 1), which the test rejects."""
    from scipy.stats import chi2, kstest
    o = oracle.Oracle(synth.tiny(), tau_t=1e-5, dt=0.02)
    kt, K = 7.5, 3.0
    x = np.array([o.bussi_alpha(K, nf, kt, 0, i) ** 2 * K * nf / kt for i in range(20000)])
    assert kstest(x, chi2(nf).cdf).pvalue > 1e-3
    assert kstest(x, chi2(nf + 1).cdf).pvalue < 1e-6


def test_bussi_kinetic_energy_variance():
    """Bussi et al. (2007): with s = (1 - c) K_t / Nf the new kinetic energy is
    c K + 2 sqrt(c K s) R1 + s chi2(Nf), so its mean is c K + (1 - c) K_t and
    its variance 2 Nf s^2 + 4 c K s.  A wrong R1 coefficient or a dropped
    cross term moves the variance far outside the bound."""
    o = oracle.Oracle(synth.tiny(), tau_t=0.1, dt=0.02)
    c = math.exp(-0.02 / 0.1)
    nf, kt, K = 60, 30.0, 20.0
    n = 40000
    kn = np.array([o.bussi_alpha(K, nf, kt, 0, i) ** 2 * K for i in range(n)])
    s = (1 - c) * kt / nf
    mean, var = c * K + (1 - c) * kt, 2 * nf * s * s + 4 * c * K * s
    assert abs(kn.mean() - mean) < 4 * math.sqrt(var / n)
    assert abs(kn.var() / var - 1) < 0.05, (kn.var(), var)


@pytest.mark.parametrize("soft", [0.0, 0.05])
def test_work_increment_equals_difference_of_full_energies(soft):
    """The work of one lambda step summed over the pairs with a changing bead
    equals the difference of the two full energies U_{l1} - U_{l0}, for two
    exchanged pairs of a three-type bilayer, linear and soft-core paths."""
    m = synth.tiny(seed=49, n_lipid_types=3)
    o = oracle.Oracle(m, soft_core=soft)
    lt = m.lipid_type
    pairs = o.mdas_pairs(lt, 0, 2)
    assert len(pairs) == 2
    ltB = lt.copy()
    for a, b in pairs:
        ltB[a], ltB[b] = lt[b], lt[a]
    btA, btB = o.bead_types(lt), o.bead_types(ltB)
    assert (btA != btB).sum() >= 2
    for l0, l1 in [(0.0, 0.25), (0.4, 0.7), (0.9, 1.0)]:
        full = (o.energy(m.pos_u, btA=btA, btB=btB, lam=l1, cells=False, forces=False)[0]["total"] -
                o.energy(m.pos_u, btA=btA, btB=btB, lam=l0, cells=False, forces=False)[0]["total"])
        got = o.work_increment(m.pos_u, btA, btB, l0, l1)
        assert got == pytest.approx(full, abs=1e-9 * max(1.0, abs(full)))
        assert abs(got) > 1e-3


def test_lambda_path_is_linear():
    """U(lambda) = (1 - lambda) U_A + lambda U_B (Sec. 2): forces are linear too."""
    m = synth.tiny(seed=46)
    o = oracle.Oracle(m)
    ltB = m.lipid_type.copy()
    ltB[:2] = ltB[1::-1]
    btA, btB = o.bead_types(m.lipid_type), o.bead_types(ltB)
    t0, F0 = o.energy(m.pos_u, btA=btA)
    t1, F1 = o.energy(m.pos_u, btA=btB)
    for lam in (0.25, 0.6):
        tl, Fl = o.energy(m.pos_u, btA=btA, btB=btB, lam=lam)
        assert tl["total"] == pytest.approx((1 - lam) * t0["total"] + lam * t1["total"], rel=1e-12)
        assert np.abs(Fl - ((1 - lam) * F0 + lam * F1)).max() < 1e-9 * np.abs(F0).max()


def test_mdas_reject_restores_state_and_accept_keeps_types():
    m = synth.tiny(seed=47)
    o = oracle.Oracle(m)
    outcomes = set()
    st = o.state()
    for _ in range(12):
        x0, v0, lt0 = st["pos_u"].copy(), st["vel"].copy(), st["ltype"].copy()
        res = o.mdas_move(st, 2, 3, 2)
        outcomes.add(res["accepted"])
        if res["accepted"]:
            exp = lt0.copy()
            for a, b in res["pairs"]:
                exp[a], exp[b] = lt0[b], lt0[a]
            assert np.array_equal(st["ltype"], exp)
            assert not np.array_equal(st["pos_u"], x0)
        else:
            assert np.array_equal(st["pos_u"], x0) and np.array_equal(st["vel"], v0)
            assert np.array_equal(st["ltype"], lt0)
        # MD between moves so later proposals see new states
        o.md_steps(st, 2)
    assert st["move"] == 12


def test_detailed_balance_exact_enumeration():
    """Swaps only, frozen coordinates, 2 + 2 lipids of two types: the six
    occupancies are visited with Boltzmann weights exp(-U/kT)."""
    from itertools import combinations
    from scipy.stats import chisquare
    m = synth.membrane(5, n_lipid_types=2, n_water=30, seed=48, n_lipids=4)   # 2 per leaflet
    m.lipid_type = np.array([0, 0, 1, 1], np.int32)
    o = oracle.Oracle(m, temperature=100.0)     # kT ~ the spread of the six energies
    states = [tuple(1 if i in c else 0 for i in range(4)) for c in combinations(range(4), 2)]
    U = np.array([o.energy(m.pos_u, ltype=np.array(s, np.int32), forces=False)[0]["total"] for s in states])
    w = np.exp(-(U - U.min()) / o.kT)
    p = w / w.sum()
    assert p.min() > 0.05 and p.max() / p.min() > 2.0
    lt = m.lipid_type.copy()
    counts = np.zeros(6)
    n_steps = 30000
    lt, recs = o.swap_trials(m.pos_u, lt, 0, 0)
    t = 0
    chunk = 1000
    while t < n_steps:
        lt_cur = lt
        lt, recs = o.swap_trials(m.pos_u, lt_cur, t, chunk)
        # replay the chunk to record the state after every trial
        cur = lt_cur.copy()
        for r in recs:
            if r["accepted"]:
                cur[r["a"]], cur[r["b"]] = cur[r["b"]], cur[r["a"]]
            counts[states.index(tuple(int(x) for x in cur))] += 1
        assert np.array_equal(cur, lt)
        t += chunk
    _, pval = chisquare(counts, p * counts.sum())
    # consecutive states are correlated; thin the effective sample size by 4
    _, pthin = chisquare(counts / 4, p * counts.sum() / 4)
    assert pthin > 1e-3, (counts / counts.sum(), p, pval)


def test_chi2_and_gaussian_moments():
    m = synth.tiny()
    o = oracle.Oracle(m)
    for k in (2, 9, 300):
        x = np.array([o.chi2(k, i, 7) for i in range(4000)])
        assert abs(x.mean() - k) < 4 * math.sqrt(2 * k / 4000)
        assert abs(x.var() / (2 * k) - 1) < 0.12
    us = np.array([oracle.uniform53(*oracle.philox([i, 1, 2, 3], [5, 6])[:2]) for i in range(20000)])
    assert us.min() > 0 and us.max() <= 1 and abs(us.mean() - 0.5) < 0.01


def test_bussi_kinetic_energy_distribution():
    """The rescaled kinetic energy has mean c K + (1 - c) K_t (Bussi et al. 2007)."""
    m = synth.tiny()
    o = oracle.Oracle(m, tau_t=0.1, dt=0.02)
    c = math.exp(-0.02 / 0.1)
    nf, kt, K = 60, 30.0, 20.0
    kn = np.array([o.bussi_alpha(K, nf, kt, 0, i) ** 2 * K for i in range(6000)])
    assert abs(kn.mean() - (c * K + (1 - c) * kt)) < 4 * kn.std() / math.sqrt(len(kn))
    assert o.bussi_alpha(K, nf, kt, 0, 0) == o.bussi_alpha(K, nf, kt, 0, 0)
    o2 = oracle.Oracle(m, tau_t=0.0)
    assert o2.bussi_alpha(K, nf, kt, 0, 0) == 1.0


def test_nve_energy_error_scales_as_dt_squared():
    """Leapfrog without thermostat: the fluctuation of U + <K> (K averaged over
    the two half steps) shrinks about 4x when dt halves, with no drift."""
    m = synth.tiny(n_side=2, n_water=50, seed=49)

    def fluct(dt, n):
        o = oracle.Oracle(m, tau_t=0.0, dt=dt)
        st = o.state()
        E = []
        for _ in range(n):
            U = o.energy(st["pos_u"], ltype=st["ltype"], forces=False)[0]["total"]
            k0 = 0.5 * 72 * (st["vel"] ** 2).sum()
            o.md_steps(st, 1)
            k1 = 0.5 * 72 * (st["vel"] ** 2).sum()
            E.append(U + 0.5 * (k0 + k1))
        E = np.array(E)
        return E.std(), abs(E[-n // 4:].mean() - E[: n // 4].mean())

    s1, d1 = fluct(0.01, 200)
    s2, d2 = fluct(0.005, 400)
    assert 2.8 < s1 / s2 < 5.5, (s1, s2)
    assert d1 < 5 * s1


# ---------------------------------------------------------------- head-bead g(r)
def _lattice_pairs(a, nside, dr, n_bins):
    """Unordered pairs per bin on a periodic square lattice of N = nside^2
    heads (spacing a): every lattice vector v within the minimum image gives
    N / 2 pairs at |v| (counting integer vectors, no positions involved)."""
    vec = np.zeros(n_bins, np.int64)
    for p in range(-nside, nside + 1):
        for q in range(-nside, nside + 1):
            if (p, q) == (0, 0) or 2 * abs(p) >= nside or 2 * abs(q) >= nside:
                continue
            r = math.hypot(p, q) * a
            if r < n_bins * dr:
                vec[int(r // dr)] += 1
    return vec * (nside * nside) // 2


def test_head_rdf_square_lattice_closed_form():
    """Heads on the two leaflets' perfect square lattices (spacing 0.8 nm,
    offset by half a cell between leaflets): the counts per bin are the
    lattice's shells, with no pair across the leaflets."""
    m = synth.membrane(8, n_lipid_types=1, fracs=[1.0], n_water=40, jitter=0.0, seed=3)
    o = oracle.Oracle(m)
    r_max, n_bins = 3.1, 40
    counts, nh = o.head_rdf(m.pos_u, np.zeros(m.n_lipids, np.int32), 0, 1, r_max, n_bins)
    assert list(nh) == [64, 64]
    exp = _lattice_pairs(0.8, 8, r_max / n_bins, n_bins)
    assert np.array_equal(counts[0], exp) and np.array_equal(counts[1], exp)


def test_head_rdf_checkerboard_types():
    """A checkerboard of two types: the type-0 heads form a square lattice of
    spacing 0.8 * sqrt(2) rotated by 45 degrees (vectors (1,1), (1,-1)), half
    the sites; type 1 the same by symmetry; a type with no lipid gives zeros."""
    m = synth.membrane(8, n_lipid_types=2, fracs=[0.5, 0.5], n_water=40, jitter=0.0, seed=3)
    o = oracle.Oracle(m)
    lt = np.zeros(m.n_lipids, np.int32)
    for leaf in range(2):
        for j in range(8):
            for i in range(8):
                lt[leaf * 64 + j * 8 + i] = (i + j) % 2
    r_max, n_bins = 3.1, 40
    dr = r_max / n_bins
    # vectors p (1,1) + q (1,-1) of the sublattice, within the minimum image of the 8x8 box
    exp = np.zeros(n_bins, np.int64)
    for vx in range(-3, 4):
        for vy in range(-3, 4):
            if (vx, vy) == (0, 0) or (vx + vy) % 2:
                continue
            r = math.hypot(vx, vy) * 0.8
            if r < r_max:
                exp[int(r // dr)] += 1
    exp = exp * 32 // 2
    for t in (0, 1):
        counts, nh = o.head_rdf(m.pos_u, lt, t, 1, r_max, n_bins)
        assert list(nh) == [32, 32]
        assert np.array_equal(counts[0], exp) and np.array_equal(counts[1], exp)
    counts, nh = o.head_rdf(m.pos_u, lt, 5, 1, r_max, n_bins)
    assert counts.sum() == 0 and list(nh) == [0, 0]


def test_g_of_r_normalisation_uniform_and_separated_layout():
    """The g(r) normalisation: heads at uniform random positions give g = 1
    within counting noise (the ideal 2D gas it divides by); the separated
    layout puts each type in one stripe per leaflet."""
    from paper_2005_08348_gb300 import mixing
    rng = np.random.default_rng(4)
    box = np.array([20.0, 20.0, 10.0])
    n = 4000
    r_max, nb = 4.0, 20
    counts = np.zeros((2, nb), np.int64)
    for leaf in range(2):
        p = rng.uniform(0, 20.0, size=(n, 2))
        for i in range(n):
            d = p[i + 1:] - p[i]
            d -= 20.0 * np.round(d / 20.0)
            r = np.sqrt((d * d).sum(1))
            counts[leaf] += np.bincount((r[r < r_max] / (r_max / nb)).astype(int), minlength=nb)[:nb]
    r, g, both = mixing.g_of_r(counts, [n, n], box, r_max)
    assert np.all(np.abs(both[2:] - 1.0) < 0.05), both
    m = mixing.bilayer(nx=10, ny=20)
    lt = m.lipid_type.reshape(2, 200)
    col = np.arange(200) % 10                      # grid column (x) of each site of a leaflet
    for leaf in range(2):
        assert np.array_equal(lt[leaf], (col >= 5).astype(np.int32))


def test_mutation_semi_grand_weights_with_equal_types():
    """Two lipid types with the same beads: every mutation has dE = 0 exactly,
    so the chain gives each lipid type 1 with probability e^(dmu/kT) / (1 +
    e^(dmu/kT)), the semi-grand weight (here 3/4); chemical-potential gaps of
    +-1e6 kJ/mol force acceptance and rejection."""
    m = synth.tiny(n_side=4)
    m.lipid_bead_type[1] = m.lipid_bead_type[0]
    o = oracle.Oracle(m)
    mu = [0.0, o.kT * math.log(3.0)]
    n = 6000
    recs, lt = o.mutation_trials(m.pos_u, m.lipid_type, 0, n, mu)
    assert all(r["dE"] == 0.0 and not r["null"] for r in recs)
    cur = np.array(m.lipid_type, np.int32)
    frac = []
    for r in recs:
        if r["accepted"]:
            cur[r["a"]] = r["b"]
        frac.append(cur.mean())
    f = float(np.mean(frac[n // 3:]))
    assert abs(f - 0.75) < 0.04, f
    assert np.array_equal(cur, lt)
    up, _ = o.mutation_trials(m.pos_u, np.zeros(m.n_lipids, np.int32), 0, 50, [0.0, 1e6])
    assert all(r["accepted"] and r["b"] == 1 for r in up[:1])
    down, lt2 = o.mutation_trials(m.pos_u, np.zeros(m.n_lipids, np.int32), 0, 50, [0.0, -1e6])
    assert not any(r["accepted"] for r in down) and lt2.sum() == 0


def test_leaflets_and_interleaflet_pairs():
    """The leaflet rule on the generator's bilayer (upper leaflet first) and
    on a box too thin for a head-to-tail minimum image; pairs of an exchange
    between the leaflets (Sec. 4) are disjoint, across the leaflets and of
    different types."""
    for m in (synth.mcmd_small(), synth.membrane(6, n_lipid_types=2, n_water=10, seed=9)):
        o = oracle.Oracle(m)
        leaf = o.leaflets(m.pos_u)
        half = m.n_lipids // 2
        assert np.array_equal(leaf, np.repeat([0, 1], half))
        for move in range(3):
            pairs = o.interleaflet_pairs(m.pos_u, m.lipid_type, move, 5)
            assert len(pairs) == 5 and len(set(pairs.ravel())) == 10
            assert all(leaf[a] == 0 and leaf[b] == 1 and m.lipid_type[a] != m.lipid_type[b] for a, b in pairs)


def test_interleaflet_proposal_is_uniform():
    """One pair per move: every (leaflet-0 lipid, leaflet-1 lipid) pair of
    different types is proposed equally often (chi-squared), and no other
    pair ever is."""
    from scipy.stats import chisquare
    m = synth.membrane(3, n_lipid_types=2, n_water=10, seed=12)       # 9 lipids per leaflet
    o = oracle.Oracle(m)
    leaf, lt = o.leaflets(m.pos_u), m.lipid_type
    valid = [(a, b) for a in range(m.n_lipids) for b in range(m.n_lipids)
             if leaf[a] == 0 and leaf[b] == 1 and lt[a] != lt[b]]
    assert len(valid) >= 10
    counts = dict.fromkeys(valid, 0)
    n = 40 * len(valid)
    for move in range(n):
        (a, b), = o.interleaflet_pairs(m.pos_u, lt, move, 1)
        counts[(int(a), int(b))] += 1
    assert sum(counts.values()) == n
    assert chisquare(list(counts.values())).pvalue > 1e-3


# ---------------------------------------------------------------- soft-core alchemical path
def _sc_system():
    m = synth.tiny(seed=21)
    ltB = m.lipid_type.copy()
    ltB[0], ltB[1] = m.lipid_type[1], m.lipid_type[0]
    ltB[2], ltB[3] = 1 - ltB[2], 1 - ltB[3]
    return m, ltB


@pytest.mark.parametrize("lam", [0.25, 0.6])
def test_soft_core_forces_match_energy_gradient(lam):
    """Eq. 4 path (delta 0.05 nm^2): central finite differences of U(lambda)
    match F = -grad U (1e-6 rel), pairs with a changed bead included."""
    m, ltB = _sc_system()
    o = oracle.Oracle(m, soft_core=0.05)
    btA, btB = o.bead_types(m.lipid_type), o.bead_types(ltB)
    _, F = o.energy(m.pos_u, btA=btA, btB=btB, lam=lam)
    rng = np.random.default_rng(5)
    k = 1 << 10
    worst = 0.0
    frms = np.sqrt((F * F).sum(1).mean())
    changed = np.flatnonzero(btA != btB)
    for i in list(changed) + list(rng.choice(m.n_beads, 12, replace=False)):
        for d in range(3):
            h = k * m.box[d] / 2 ** 32
            p, q = m.pos_u.copy(), m.pos_u.copy()
            p[i, d] += np.uint32(k)
            q[i, d] -= np.uint32(k)
            up = o.energy(p, btA=btA, btB=btB, lam=lam, forces=False)[0]["total"]
            um = o.energy(q, btA=btA, btB=btB, lam=lam, forces=False)[0]["total"]
            worst = max(worst, abs(-(up - um) / (2 * h) - F[i, d]) / max(abs(F[i, d]), frms))
    assert worst < 1e-6


def test_soft_core_end_states_and_vanishing_delta():
    """At lambda 0 and 1 the soft-core path is the A and B energy; it differs
    in between; as delta -> 0 it becomes the linear path (1-l) U_A + l U_B."""
    m, ltB = _sc_system()
    lin, sc, tiny = oracle.Oracle(m), oracle.Oracle(m, soft_core=0.05), oracle.Oracle(m, soft_core=1e-12)
    btA, btB = lin.bead_types(m.lipid_type), lin.bead_types(ltB)
    e = lambda o, l: o.energy(m.pos_u, btA=btA, btB=btB, lam=l, forces=False)[0]["total"]
    eA = lin.energy(m.pos_u, btA=btA, forces=False)[0]["total"]
    eB = lin.energy(m.pos_u, btA=btB, forces=False)[0]["total"]
    assert abs(e(sc, 0.0) - eA) <= 1e-9 * abs(eA)
    assert abs(e(sc, 1.0) - eB) <= 1e-9 * abs(eB)
    for l in (0.3, 0.7):
        assert abs(e(tiny, l) - ((1 - l) * eA + l * eB)) <= 1e-9 * abs(eA)
        assert abs(e(sc, l) - e(lin, l)) > 1e-6


# ---- semi-isotropic Parrinello-Rahman pressure coupling (Sec. 3) ----------

@pytest.mark.parametrize("seed", [31, 32])
def test_virial_is_half_the_box_derivative_of_the_energy(seed):
    """Xi_a = 1/2 dU/d ln L_a at fixed fractional coordinates: central
    differences of the energy under a stretch of one box edge (pairs, bonds
    and angles all move with the box)."""
    m = synth.tiny(n_side=3, n_water=120, seed=seed)
    O = oracle.Oracle(m)
    P, K, Xi = O.pressure(m.pos_u, m.vel)
    L0 = O.box
    # small enough that no pair crosses the cutoff within +-h (the shifted
    # Lennard-Jones force does not vanish there)
    r = pair_distances(m.pos_u.astype(np.float64) * (L0 / 2.0 ** 32), L0)
    h = min(1e-6, 0.3 * float(np.min(np.abs(r / m.rc - 1.0))))
    assert h > 1e-9
    for a in range(3):
        u = []
        for sgn in (1, -1):
            L = L0.copy()
            L[a] *= 1 + sgn * h
            O.box = L
            u.append(O.energy(m.pos_u, forces=False)[0]["total"])
        O.box = L0
        dudlnL = (u[0] - u[1]) / (math.log(1 + h) - math.log(1 - h))
        tol = 1e-6 * (abs(Xi[a]) + 10.0) + 1e-15 * abs(u[0]) / h
        assert abs(dudlnL - 2 * Xi[a]) <= tol, (a, h, dudlnL, 2 * Xi[a])


def test_virial_of_a_stretched_bond_and_a_bent_angle():
    """One lipid alone (no partners in range): the virial is that of its
    bonds and angles only, and still matches the box derivative."""
    m = synth.tiny(n_side=1, n_water=0, seed=33)
    keep = m.lipid_first_bead[:1]
    n = 12
    m.pos_u = m.pos_u[:n].copy()
    m.pos = m.pos[:n].copy()
    m.vel = m.vel[:n].copy()
    m.lipid_first_bead = keep.copy()
    m.lipid_type = m.lipid_type[:1].copy()
    # stretch the lipid along x and tilt it so every bond and angle is strained
    m.pos_u[:, 0] += (np.arange(n, dtype=np.uint32) * np.uint32(1 << 22))
    m.pos_u[:, 2] += (np.arange(n, dtype=np.uint32) ** 2 * np.uint32(1 << 20))
    O = oracle.Oracle(m)
    _, _, Xi = O.pressure(m.pos_u, np.zeros_like(m.vel))
    L0 = O.box
    h = 1e-6
    for a in range(3):
        u = []
        for sgn in (1, -1):
            L = L0.copy()
            L[a] *= 1 + sgn * h
            O.box = L
            u.append(O.energy(m.pos_u, forces=False, cells=False)[0]["total"])
        O.box = L0
        d = (u[0] - u[1]) / (math.log(1 + h) - math.log(1 - h))
        assert abs(d - 2 * Xi[a]) <= 1e-6 * (abs(Xi[a]) + 1.0), (a, d, 2 * Xi[a])
    assert np.abs(Xi).max() > 1.0


def test_ideal_gas_pressure_in_bar():
    """No interactions: P = n k_B T with SI constants, the velocities chosen so
    that every axis holds 1/2 N k T exactly."""
    m = synth.tiny(n_side=3, n_water=120, seed=34)
    m.eps = np.zeros_like(m.eps)
    m.charge = np.zeros_like(m.charge)
    O = oracle.Oracle(m, kb=0.0, ktheta=0.0)
    T = 310.0
    R = 1.380649e-23 * 6.02214076e23 * 1e-3          # kJ / mol / K
    v0 = math.sqrt(R * T / m.mass)                   # nm/ps
    rng = np.random.default_rng(3)
    vel = v0 * rng.choice([-1.0, 1.0], size=(m.n_beads, 3))
    P, K, Xi = O.pressure(m.pos_u, vel)
    assert np.all(Xi == 0.0)
    V = float(np.prod(O.box)) * 1e-27                 # m^3
    expect = m.n_beads / V * 1.380649e-23 * T / 1e5   # bar
    assert np.allclose(P, expect, rtol=1e-9, atol=0.0), (P, expect)


def _box_period(axis_set, tau_p, beta=4.5e-5, L0=10.0, amp=1e-4, p_ref=1.0):
    """Period of the box coupled to a linear equation of state
    P = p_ref - (V - V0) / (beta V0) (only the edges in axis_set move)."""
    nst, dt = 1, tau_p / 4000.0
    b = oracle.barostat(p_ref=p_ref, tau_p=tau_p, beta=beta, nst=nst)
    box = np.full(3, L0)
    for a in axis_set:
        box[a] = L0 * (1 + amp)
    V0 = L0 ** 3
    t, last, ups = 0.0, box[axis_set[0]] - L0, []
    for k in range(40000):
        V = float(np.prod(box))
        p = p_ref - (V - V0) / (beta * V0)
        P = [p if a in axis_set else p_ref for a in range(3)]
        box = oracle.pr_box_update(dt, box, b, P)
        t += nst * dt
        x = box[axis_set[0]] - L0
        if last < 0 <= x:
            ups.append(t - dt * x / (x - last))
        last = x
        if len(ups) == 3:
            break
    assert len(ups) == 3
    return (ups[2] - ups[0]) / 2, b


def test_pr_box_oscillation_periods():
    """Linearised: the normal edge alone oscillates with period sqrt(3) tau_p
    in a cubic box, the two lateral edges together with sqrt(3/2) tau_p (the
    barostat mass W^-1 = 4 pi^2 beta / (3 tau_p^2 L_max)); an isotropic box
    would give tau_p itself."""
    tau = 4.0
    Tz, _ = _box_period([2], tau)
    assert abs(Tz / (math.sqrt(3.0) * tau) - 1) < 2e-3, Tz
    Txy, _ = _box_period([0, 1], tau)
    assert abs(Txy / (math.sqrt(1.5) * tau) - 1) < 2e-3, Txy


def test_pr_box_direction_and_rest():
    """The box grows under an excess pressure, shrinks under a deficit, stays
    at rest at p_ref; x and y see their mean pressure."""
    b = oracle.barostat(p_ref=1.0, tau_p=12.0, beta=3e-4, nst=10)
    box = oracle.pr_box_update(0.02, [8.0, 8.0, 10.0], b, [1.0, 1.0, 1.0])
    assert np.all(box == [8.0, 8.0, 10.0]) and np.all(np.array(b.boxv) == 0)
    box = oracle.pr_box_update(0.02, [8.0, 8.0, 10.0], b, [101.0, -99.0, 51.0])
    assert box[0] == box[1] == 8.0 and box[2] > 10.0 and b.M[2] > 0
    b2 = oracle.barostat(p_ref=1.0, tau_p=12.0, beta=3e-4, nst=10)
    box = oracle.pr_box_update(0.02, [8.0, 8.0, 10.0], b2, [-50.0, -50.0, 1.0])
    assert box[0] < 8.0 and box[0] == box[1] and box[2] == 10.0
    assert np.isclose(b2.M[0], b2.boxv[0] / box[0])


def test_npt_velocity_coupling_closed_form():
    """No forces, no thermostat, a box velocity held fixed (no update within
    the run): v_n = (1 - dt M_a)^n v_0 per axis."""
    m = synth.tiny(n_side=3, n_water=120, seed=35)
    m.eps = np.zeros_like(m.eps)
    m.charge = np.zeros_like(m.charge)
    O = oracle.Oracle(m, kb=0.0, ktheta=0.0, tau_t=0.0)
    b = oracle.barostat(nst=1000)
    M = [0.01, 0.02, -0.03]
    for a in range(3):
        b.M[a] = M[a]
    st = O.state()
    v0 = st["vel"].copy()
    O.md_steps_npt(st, b, 7)
    for a in range(3):
        assert np.allclose(st["vel"][:, a], v0[:, a] * (1 - m.dt * M[a]) ** 7, rtol=1e-13, atol=0)


def test_npt_without_coupling_is_plain_md():
    """beta = 0 (no box motion): the constant-pressure driver gives the same
    bits as plain MD, trials included."""
    m = synth.mcmd_small()
    O = oracle.Oracle(m)
    a, b = O.state(), O.state()
    ra = O.md_steps(a, 6, swap_every=3)
    bar = oracle.barostat(beta=0.0, nst=2)
    rb = O.md_steps_npt(b, bar, 6, swap_every=3)
    assert ra == rb
    assert np.array_equal(a["pos_u"], b["pos_u"]) and np.array_equal(a["vel"], b["vel"])
    assert np.all(O.box == m.box)


def test_npt_pressure_is_that_of_the_step_forces_and_new_velocities():
    """The pressure a box update uses is or_pressure (pinned above) taken at
    the positions the step started from and the box before the update, with
    the velocities the step produced."""
    m = synth.tiny(n_side=3, n_water=120, seed=36)
    O = oracle.Oracle(m)
    st = O.state()
    x0, L0 = st["pos_u"].copy(), O.box
    b = oracle.barostat(nst=1)
    O.md_steps_npt(st, b, 1)
    L1 = O.box
    assert not np.array_equal(L1, L0)
    O.box = L0
    P, _, _ = O.pressure(x0, st["vel"])
    O.box = L1
    assert np.allclose(list(b.P), P, rtol=1e-12, atol=1e-9), (list(b.P), P)
