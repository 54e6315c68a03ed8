"""Per-level cluster sizes of the rounding launches (tnlbm_clusters,
tnlbm_set_clusters, tnlbm_tune_clusters and their batch forms).

The tuner runs one step eagerly without its final copy, so it must leave the
populations, the step count and the discarded weight exactly as they were.
A cluster size changes only how the CTAs of a job share its FP64 centre SVD:
a tuned step agrees with the untuned one to round-off in FP64 and to FP32
storage in the mixed mode (the gates of the cluster-vs-single-CTA test), and a
batch stepped with some sizes equals its members stepped alone with the same
sizes bit for bit."""
import numpy as np
import pytest

import synth
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_07615_gb300 import tnlbm as T
    return T


def porous16(prec, seed=1, chi=24):
    """16^3 sphere pack, products formed exactly (Kronecker bonds up to
    chi^2), so each level holds several large centre SVDs."""
    return dict(tau=0.7, periodic=(1, 1, 1), solid=synth.sphere_pack(4, 3.0, 0.3, seed), chi_mask=16,
                eps_mask=1e-10, force=(1e-5, 0, 0), chi_max=chi, eps=1e-8, precision=prec, hadamard=1,
                modes=synth.fourier_modes(7, 3 + seed, kmax=2, amp_rho=1e-3, amp_u=1e-3))


def flat(pops):
    return np.concatenate([c.ravel() for cs in pops for c in cs])


@pytest.mark.parametrize("prec,gate", [(0, 1e-10), (3, 1e-4)])
def test_tuning_keeps_the_state_and_keeps_a_fastest_size(tl, prec, gate):
    kw = porous16(prec)
    sim = tl.Sim(4, **kw)
    sim.step(1)
    p0, st0 = flat(sim.get_populations()), sim.stats()
    sizes0, jobs = sim.clusters()
    assert len(sizes0) == len(jobs) and any(jobs)
    res = sim.tune_clusters(reps=1)
    p1, st1 = flat(sim.get_populations()), sim.stats()
    assert np.array_equal(p0, p1)
    assert st1["steps"] == st0["steps"] and st1["discarded2"] == st0["discarded2"] and st1["status"] == 0
    assert res["jobs"] == jobs and not res["cached"]
    for l, (P, J, t) in enumerate(zip(res["sizes"], jobs, res["ms"])):
        if J == 0:
            assert P == 0 and t == {}
            continue
        assert P in t and sizes0[l] in t, (l, P, t)
        assert t[P] <= 1.02 * min(t.values()) * (1 + 1e-9), (l, P, t)
        if P != sizes0[l]:
            assert t[P] * 1.02 < t[sizes0[l]], (l, P, t)
    assert sim.clusters()[0] == res["sizes"]
    print("prec %d tuned sizes %s (occupancy rule %s), jobs %s" % (prec, res["sizes"], sizes0, jobs))
    # the tuned graph steps on from the same state as an untuned simulation
    ref = tl.Sim(4, **kw)
    ref.step(3)
    sim.step(2)
    a, b = sim.macroscopic(), ref.macroscopic()
    assert sim.stats()["steps"] == 3
    err = rel_l2(a[1], b[1])
    print("tuned vs untuned rel-L2(u) = %.3e" % err)
    assert err <= gate
    sim.close()
    ref.close()


def test_set_clusters_checks_its_sizes(tl):
    sim = tl.Sim(4, **porous16(3))
    sizes, jobs = sim.clusters()
    n = len(sizes)
    with pytest.raises(tl.nat.TnlbmError):
        sim.set_clusters([1] * (n + 1))
    for bad in (0, 17):
        with pytest.raises(tl.nat.TnlbmError):
            sim.set_clusters([bad] * n)
    assert sim.clusters()[0] == sizes               # a refused call changes nothing
    ones = [1 if j else 0 for j in jobs]
    sim.set_clusters(ones)
    assert sim.clusters()[0] == ones
    sim.step(1)
    assert sim.stats()["status"] == 0 and sim.stats()["max_cluster"] == 1
    sim.close()
    f32 = tl.Sim(4, **porous16(1))
    sizes, jobs = f32.clusters()
    assert set(sizes) <= {0, 1}
    with pytest.raises(tl.nat.TnlbmError):
        f32.set_clusters([2 if j else 0 for j in jobs])
    res = f32.tune_clusters(reps=1)                 # FP32 jobs run one CTA each: nothing to time
    assert all(t == {} for t in res["ms"]) and res["sizes"] == sizes
    f32.close()


def test_batch_tuning_and_members_alone_with_the_same_sizes(tl, tmp_path):
    cfgs = [dict(n_per_axis=4, **porous16(3, seed=1, chi=24)), dict(n_per_axis=4, **porous16(3, seed=2, chi=16))]
    b = tl.Batch(cfgs)
    b.step(1)
    before = [flat(s.get_populations()) for s in b.sims]
    cache = str(tmp_path / "clusters.json")
    res = b.tune_clusters(reps=1, cache=cache)
    assert not res["cached"]
    assert all(np.array_equal(p, flat(s.get_populations())) for p, s in zip(before, b.sims))
    assert all(s.stats()["steps"] == 1 for s in b.sims)
    again = b.tune_clusters(cache=cache)            # the stored choice, applied without timing
    assert again["cached"] and again["sizes"] == res["sizes"] and b.clusters()[0] == res["sizes"]
    b.step(2)
    got = [s.macroscopic() for s in b.sims]
    for i, kw in enumerate(cfgs):
        kw = dict(kw)
        n = kw.pop("n_per_axis")
        alone = tl.Sim(n, **kw)
        own, jobs = alone.clusters()
        alone.set_clusters([res["sizes"][l] if jobs[l] else 0 for l in range(len(own))])
        alone.step(3)
        rho, u = alone.macroscopic()
        alone.close()
        print("member %d: max |du| = %.3e" % (i, float(np.abs(u - got[i][1]).max())))
        assert np.array_equal(rho, got[i][0]) and np.array_equal(u, got[i][1]), i
    b.close()


def test_tuning_keeps_to_max_cluster(tl):
    """tnlbm_config.max_cluster caps every size the tuner times and keeps
    (BF16 mode: its centre SVDs are the mixed mode's FP64 cluster SVDs)."""
    sim = tl.Sim(4, max_cluster=4, **porous16(4))
    sim.step(1)
    res = sim.tune_clusters(reps=1)
    assert all(P <= 4 for P in res["sizes"]) and any(P > 0 for P in res["sizes"])
    assert all(max(t) <= 4 for t in res["ms"] if t)
    sim.step(1)
    assert sim.stats()["status"] == 0 and sim.stats()["max_cluster"] <= 4
    sim.close()
