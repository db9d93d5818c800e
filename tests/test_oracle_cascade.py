"""Pins of the oracle's full cascade (every product stepped again from the next step on).

What fixes a cascade independently of the code that runs it:
- energy: with no pusher the fields do no work, and each event splits its parent's energy
  exactly (Sec. 3: the photon takes xi gamma, the lepton keeps (1 - xi) gamma; Eq. again_pp:
  the pair shares sum to the photon's energy), so the energy of the alive particles is the
  primaries' initial energy at the end of any cascade;
- bookkeeping: every product record is one created particle, with the species and member
  of the record, a parent that existed before it, and an id of its own;
- independence: a particle's evolution depends on its id, the step and its field only, so
  the primary of a cascade evolves as in a run without children, and a created particle
  evolves as a primary of its own that starts at the step after its creation.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W


def _workload(n, nsteps, seed, a0=150.0, gamma0=1e4):
    d = W.config2(n=n, seed=seed, dtype=np.float64, a0=a0, gamma0=gamma0)
    E = np.zeros((n, nsteps, 6))
    for j in range(nsteps):
        (_, ey, _), (_, _, bz) = W.plane_wave_fields(d["k0"], d["amp0"], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"], d["py"], d["pz"]], 1).astype(np.float64)
    return d, p, E


def make_cascade(oracle, n=48, nsteps=60):
    d, p, E = _workload(n, nsteps, seed=5)
    r = oracle.mc_cascade(p, d["tau"], np.arange(n, dtype=np.uint64), d["flags"], np.zeros(n, np.uint8), E,
                          rho=W.RHO, dt=W.DT, seed=17, nsteps=nsteps)
    return dict(n=n, nsteps=nsteps, d=d, p=p, E=E, r=r, seed=17)


@pytest.fixture(scope="module")
def cascade(oracle):
    return make_cascade(oracle)


def _energy(p, species):
    p2 = (p * p).sum(axis=1)
    return np.where(species == W.SP_PHOTON, np.sqrt(p2), np.sqrt(1.0 + p2))


def test_cascade_reaches_the_second_generation(cascade):
    q = cascade["r"]["particles"]
    ids = set(q["id"].tolist())
    assert (q["species"] == W.SP_PHOTON).sum() > 100
    assert (q["member"] > 0).sum() >= 4                    # pairs from emitted photons
    # particles whose parent is itself a created particle (grandchildren and deeper)
    assert sum(int(pid) in ids for pid in q["parent_id"]) >= 4


def test_cascade_conserves_energy(cascade):
    r, p0 = cascade["r"], cascade["p"]
    q = r["particles"]
    e0 = _energy(p0, np.zeros(len(p0), np.uint8)).sum()
    prim_alive = (r["flags"] & 1).astype(bool)
    kid_alive = (q["flags"] & 1).astype(bool)
    # created leptons without momentum would leave the step with energy 1; there are none here
    assert not ((q["species"] != W.SP_PHOTON) & ~kid_alive).any()
    e1 = _energy(r["p"][prim_alive], np.zeros(prim_alive.sum(), np.uint8)).sum() + \
        _energy(q["p"][kid_alive], q["species"][kid_alive]).sum()
    assert abs(e1 - e0) <= 1e-12 * e0, (e1, e0)
    # converted photons are the only dead created particles, and each left a pair
    dead = ~kid_alive
    assert (q["species"][dead] == W.SP_PHOTON).all()
    assert dead.sum() == (q["member"] == 1).sum() == (q["member"] == 2).sum()


def test_cascade_bookkeeping(cascade, oracle):
    r, n, nsteps, seed = cascade["r"], cascade["n"], cascade["nsteps"], cascade["seed"]
    q, prod = r["particles"], r["products"]
    assert len(q) == len(prod) == r["n_events"].sum() + (q["member"] == 2).sum()
    # the same (parent, step, member) triples, with the record's species
    key = lambda a: sorted(zip(a["parent_id"].tolist(), a["step"].tolist(), a["member"].tolist(),
                               a["species"].tolist()))
    assert key(q) == key(prod)
    ids = q["id"]
    assert len(np.unique(ids)) == len(ids) and bool((ids >> np.uint64(63)).all())
    born = {int(i): int(s) for i, s in zip(ids, q["step"])}
    for k in range(len(q)):
        pid = int(q["parent_id"][k])
        if pid < n:                                      # a primary: any step of the run
            assert q["root"][k] == pid
        else:                                            # a created particle: stepped from born + 1
            assert q["step"][k] >= born[pid] + 1
        assert 0 <= q["step"][k] < nsteps
        assert int(ids[k]) == oracle.child_id(seed, pid, 0, int(q["step"][k]), int(q["member"][k]))


def test_child_ids_are_philox_words(oracle):
    # bit 63 over the first two words of the counter (parent lo, parent hi, step, 0x100 | tag << 2 | member)
    parent, step = 0x0123456789ABCDEF, 77
    for tag in range(4):
        for member in range(3):
            w = oracle.philox(np.array([parent], np.uint64), step, 0x100 | (tag << 2) | member, 42)[0]
            want = (1 << 63) | ((int(w[1]) & 0x7FFFFFFF) << 32) | int(w[0])
            assert oracle.child_id(42, parent, tag, step, member) == want
    assert len({oracle.child_id(42, parent, t, step, m) for t in range(4) for m in range(3)}) == 12


def test_cascade_primaries_evolve_as_without_children(cascade, oracle):
    c = cascade
    n, d = c["n"], c["d"]
    plain = oracle.mc_run(c["p"], d["tau"], np.arange(n, dtype=np.uint64), d["flags"], np.zeros(n, np.uint8),
                          c["E"], rho=W.RHO, dt=W.DT, seed=c["seed"], nsteps=c["nsteps"])
    r = c["r"]
    assert np.array_equal(plain["p"], r["p"]) and np.array_equal(plain["tau"], r["tau"])
    assert np.array_equal(plain["flags"], r["flags"])
    mine = r["products"][r["products"]["parent_id"] < n]
    key = lambda a: sorted(zip(a["parent_id"].tolist(), a["step"].tolist(), a["member"].tolist(),
                               map(tuple, a["p"].tolist())))
    assert key(plain["products"]) == key(mine)


def test_created_particles_evolve_as_primaries_of_their_own(cascade, oracle):
    """Each particle created at step s, restarted as a primary (its id, tag 0, its creation
    momentum, no optical depth) at step s + 1 in its lineage's field, ends as in the cascade."""
    c = cascade
    q, prod, nsteps = c["r"]["particles"], c["r"]["products"], c["nsteps"]
    # creation momentum of each created particle: its product record
    rec = {(int(a), int(s), int(m)): np.array(pp) for a, s, m, pp in
           zip(prod["parent_id"], prod["step"], prod["member"], prod["p"])}
    checked = 0
    for s in np.unique(q["step"]):
        sel = np.nonzero((q["step"] == s) & (q["step"] < nsteps - 1))[0]
        if len(sel) == 0:
            continue
        k = len(sel)
        p = np.stack([rec[(int(q["parent_id"][i]), int(s), int(q["member"][i]))] for i in sel])
        alive = (np.abs(p).sum(axis=1) > 0).astype(np.uint8)
        fl = alive | 2                                   # alive | just created
        E = c["E"][q["root"][sel], s + 1:, :]
        out = oracle.mc_run(p, -np.ones(k), q["id"][sel], fl, q["species"][sel], E, rho=W.RHO, dt=W.DT,
                            seed=c["seed"], step0=int(s) + 1, nsteps=nsteps - int(s) - 1)
        assert np.array_equal(out["p"], q["p"][sel]), s
        assert np.array_equal(out["tau"], q["tau"][sel]), s
        assert np.array_equal(out["flags"], q["flags"][sel]), s
        checked += k
    assert checked > 100
