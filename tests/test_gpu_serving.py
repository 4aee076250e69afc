"""Serving loop (mdas_server_*): continuous batching of MD, swap and MDAS jobs
on device-resident patches.  Each job's result must be the same alone and in
the mix, admission must respect the slot count and the memory budget."""
import numpy as np
import pytest

from paper_2005_08348_gb300 import mdas, synth

pytestmark = pytest.mark.gpu

GB = 1 << 30


def patches():
    return [synth.patch(n, 2 + k % 2, seed=300 + k, system_id=k) for k, n in enumerate([130, 200, 256, 310, 180, 420])]


def jobs(ps):
    kinds = [(mdas.JOB_MD, 60), (mdas.JOB_SWAPS, 64), (mdas.JOB_MDAS, 0), (mdas.JOB_SWAPS, 64),
             (mdas.JOB_MD, 35), (mdas.JOB_MDAS, 0)]
    return [(p, k, n) for p, (k, n) in zip(ps, kinds)]


def run(server, js, stagger):
    """Submit the jobs (two per round when staggered, else all at once) and
    run rounds until every job is done; results in submission order."""
    ids = []
    pending = list(js)
    res = {}
    for _ in range(10000):
        for _ in range(2 if stagger else len(pending)):
            if pending:
                p, k, n = pending.pop(0)
                ids.append(server.submit(p, k, n=n, n_pairs=2, n_lambda=3, md_per_lambda=2))
        active, queued = server.run(1)
        for r in server.results():
            res[r["job_id"]] = r
        if not pending and active == 0 and queued == 0:
            break
    return [res[i] for i in ids]


def test_results_same_alone_and_in_the_mix():
    ps = patches()
    js = jobs(ps)
    mix = run(mdas.Server(4 * GB, max_active=3, md_quantum=10, keep_state_hash=True), js, stagger=True)
    for (p, k, n), r in zip(js, mix):
        alone = run(mdas.Server(4 * GB, max_active=1, md_quantum=25, keep_state_hash=True), [(p, k, n)], stagger=False)[0]
        assert r["state_hash"] == alone["state_hash"], (k, n)
        for key in ("md_steps", "trials", "accepted", "w", "move_accepted"):
            assert r[key] == alone[key], key
    kinds = [r["kind"] for r in mix]
    assert sorted(set(kinds)) == [0, 1, 2]
    assert all(r["t_done"] >= r["t_admit"] >= r["t_submit"] for r in mix)
    md = [r for r in mix if r["kind"] == mdas.JOB_MD]
    assert [r["md_steps"] for r in md] == [60, 35]
    sw = [r for r in mix if r["kind"] == mdas.JOB_SWAPS]
    assert all(r["trials"] == 64 for r in sw)


def test_admission_by_slots_and_memory():
    ps = patches()
    sv = mdas.Server(4 * GB, max_active=2, md_quantum=5)
    for p in ps:
        sv.submit(p, mdas.JOB_MD, n=20)
    seen = []
    for _ in range(1000):
        a, q = sv.run(1)
        seen.append(a)
        if a == 0 and q == 0:
            break
    assert max(seen) <= 2 and len(sv.results()) == len(ps)
    # a budget that holds any one of three systems but no two admits them one by one
    fp = sorted(mdas.footprint(p) for p in ps[:3])
    budget = fp[0] + fp[1] - 1
    assert budget >= fp[2]
    sv = mdas.Server(budget, max_active=8, md_quantum=5)
    for p in ps[:3]:
        sv.submit(p, mdas.JOB_MD, n=10)
    a, q = sv.run(1)
    assert a == 1 and q == 2
    with pytest.raises(mdas.MdasError) as e:
        mdas.Server(mdas.footprint(ps[0]) // 2, max_active=2).submit(ps[0], mdas.JOB_MD, n=5)
    assert e.value.status == 2


def test_mdas_jobs_run_as_one_batched_move():
    """MDAS jobs that are active together run as one batched move (one launch
    per phase for all of them); each result equals the job run alone."""
    ps = patches()[:4]
    js = [(p, mdas.JOB_MDAS, 0) for p in ps]
    sv = mdas.Server(4 * GB, max_active=4, md_quantum=10, keep_state_hash=True)
    ids = [sv.submit(p, k, n=n, n_pairs=2, n_lambda=3, md_per_lambda=2) for p, k, n in js]
    assert sv.run(1) == (0, 0)                           # all four done in one round
    res = {r["job_id"]: r for r in sv.results()}
    mix = [res[i] for i in ids]
    for (p, k, n), r in zip(js, mix):
        alone = run(mdas.Server(4 * GB, max_active=1, md_quantum=25, keep_state_hash=True), [(p, k, n)],
                    stagger=False)[0]
        assert r["state_hash"] == alone["state_hash"]
        assert (r["w"], r["move_accepted"], r["md_steps"]) == (alone["w"], alone["move_accepted"], alone["md_steps"])


def test_resident_patches_carry_state_between_jobs():
    """Resident patches (mdas_server_add_patch / submit_to): each patch's jobs
    run one after another in submission order on its device-resident state,
    patches run together; every patch ends in the state of the same job
    sequence run alone through the one-system calls."""
    ps = patches()[:3]
    seq = [(mdas.JOB_MD, 30), (mdas.JOB_SWAPS, 40), (mdas.JOB_MD, 15), (mdas.JOB_MDAS, 0)]
    sv = mdas.Server(4 * GB, max_active=8, md_quantum=10)
    pids = [sv.add_patch(p) for p in ps]
    for kind, n in seq:                                    # interleaved over the patches
        for pid in pids:
            sv.submit_to(pid, kind, n=n, n_pairs=2, n_lambda=3, md_per_lambda=2)
    done = []
    for _ in range(1000):
        a, q = sv.run(1)
        done += sv.results()
        if a == 0 and q == 0:
            break
    assert len(done) == len(seq) * len(ps)
    assert sorted(r["md_steps"] for r in done if r["kind"] == mdas.JOB_MD) == sorted([30, 15] * 3)
    for p, pid in zip(ps, pids):
        s = mdas.System(p)
        for kind, n in seq:
            if kind == mdas.JOB_MD:
                s.md_steps(n)
            elif kind == mdas.JOB_SWAPS:
                s.swap_trials(n, log=False)
            else:
                s.alchemical_move(2, 3, 2)
        ref = s.get_state()
        got = sv.patch_state(pid, p.n_beads, p.n_lipids)
        assert np.array_equal(got["pos_u"], ref["pos_u"])
        assert np.array_equal(got["vel"], ref["vel"])
        assert np.array_equal(got["ltype"], ref["ltype"])
        assert (got["trial"], got["move"]) == (ref["trial"], ref["move"])


def test_resident_patch_admission_and_removal():
    ps = patches()[:2]
    f0, f1 = mdas.footprint(ps[0]), mdas.footprint(ps[1])
    sv = mdas.Server(max(f0, f1) + min(f0, f1) // 2, max_active=4)   # either patch alone, not both
    pid = sv.add_patch(ps[0])
    with pytest.raises(mdas.MdasError) as e:             # no room left for a second patch
        sv.add_patch(ps[1])
    assert e.value.status == 2
    sv.submit_to(pid, mdas.JOB_MD, n=5)
    with pytest.raises(mdas.MdasError) as e:             # a queued job holds the patch
        sv.remove_patch(pid)
    assert e.value.status == 6
    while sv.run(1) != (0, 0):
        pass
    sv.remove_patch(pid)
    pid2 = sv.add_patch(ps[1])                            # its memory is back
    with pytest.raises(mdas.MdasError):
        sv.submit_to(pid, mdas.JOB_MD, n=5)               # removed
    sv.remove_patch(pid2)


def test_largest_patch_same_alone_and_in_the_mix():
    """Jobs on a patch at the served workload's largest size (16384 lipids,
    ~413k beads) beside small ones: MD and MDAS results on it, and the small
    jobs' results, are the same alone and in the mix."""
    big = synth.patch(16384, 3, seed=777, system_id=40)
    small = patches()[:2]
    js = [(big, mdas.JOB_MD, 30), (small[0], mdas.JOB_SWAPS, 64), (small[1], mdas.JOB_MD, 25), (big, mdas.JOB_MDAS, 0)]
    mix = run(mdas.Server(16 * GB, max_active=4, md_quantum=10, keep_state_hash=True), js, stagger=True)
    for (p, k, n), r in zip(js, mix):
        alone = run(mdas.Server(16 * GB, max_active=1, md_quantum=25, keep_state_hash=True), [(p, k, n)],
                    stagger=False)[0]
        assert r["state_hash"] == alone["state_hash"], (k, n)
        for key in ("md_steps", "trials", "accepted", "w", "move_accepted"):
            assert r[key] == alone[key], key
