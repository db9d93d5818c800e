"""GPU tests of the photon surrogate on the Monte Carlo step's event path (sfq_set_surrogate).

Workload: config 2 (electrons with gamma ~ N(2000, 5%) head-on with the plane wave of
a0 = 100, dt = 0.01 period, photon emission by the optical depth, Sec. 2 and 4.1) at
2^16 - 2^18 particles.  The network is trained on the GPU on the plain fitted sampler's
targets and calibrated (tol_u = 1e-3), as the bench does.  Checks:
  - the step decides the same events as without the surrogate (the decision does not
    depend on the sampler), queues each emission with the chi, r_1 (Philox word 1), energy
    and momentum the step read, and the surrogate pass samples exactly what
    sfq_mlp_sample_photon_xi returns for those inputs, recoils the emitter by 1 - xi along
    its direction and records the collinear photon xi gamma (Sec. 3);
  - emissions past the queue's capacity take the plain sampler in the step kernel,
    counted as fallbacks, and agree with the run without the surrogate;
  - over 40 steps of 2^18 electrons, the probability-integral transform of every sampled
    fraction under the oracle's CDF at its event's chi is uniform: KS within the network's
    judged bound (1e-3) plus the sampling noise of the event count.
"""
import math

import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=2024)
    net = sfq.Surrogate(ctx, seed=7)
    g = np.random.default_rng(21)
    n = 1 << 22
    chi = np.exp(g.uniform(np.log(1e-3), np.log(100.0), n)).astype(np.float32)
    u = ((g.integers(0, 1 << 23, n) + 0.5) / (1 << 23)).astype(np.float32)
    tchi, tu = torch.as_tensor(chi).cuda(), torch.as_tensor(u).cuda()
    net.train(tchi, tu, net.plain_targets(tchi, tu), steps=30000, batch=8192, lr=3e-3, quantize=True, seed=9)
    nflag, max_err = net.calibrate(1e-3)
    yield ctx, net
    ctx.set_surrogate(None)
    net.close()
    ctx.close()


def _population(ctx, d):
    import torch
    from paper_2301_07684_gb300 import sfq
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"]), T(d["flags"]))
    F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), T(d["table"]), d["k_step"], amp0=d["amp0"])
    return P, F


def _step(ctx, P, F, step, cap):
    import torch
    from paper_2301_07684_gb300 import sfq
    out, cnt = sfq.ProductBuffers(cap, torch.float32, "cuda"), sfq.counters_tensor()
    ctx.mc_step(P, F, step, out, counters=cnt)
    torch.cuda.synchronize()
    return out, sfq.counters_dict(cnt)


def test_step_queues_and_finishes_every_emission(setup):
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx, net = setup
    n = (1 << 16) + 77
    d = W.config2(n=n, seed=4)
    # the first step from the same state with and without the surrogate (the draws of step 3)
    P0, F = _population(ctx, d)
    ctx.set_surrogate(None)
    out0, c0 = _step(ctx, P0, F, 3, n)
    q = sfq.EventQueue(n)
    ctx.set_surrogate(net, q, use_flags=True)
    P1, F1 = _population(ctx, d)
    out1, c1 = _step(ctx, P1, F1, 3, n)
    ctx.set_surrogate(None)
    k = q.n()
    assert c1["events"] == c0["events"] == c1["emitted"] == k > 1000, (c0, c1, k)
    assert c1["dropped"] == 0 and c1["timeouts"] == 0 and sfq.counters_status(torch.tensor(
        [c1[x] for x in sfq.COUNTER_NAMES] + [0, 0])) == "SFQ_OK"
    idx = q.index[:k].cpu().numpy()
    # the same emitters
    assert np.array_equal(np.sort(idx), np.sort(out0.parent_id[:k].cpu().numpy()))
    # the queued draw is the step's word 1 for (id, step 3)
    u = ctx.uniforms(q.index[:k].clone(), 3)
    assert torch.equal(q.r[:k], u[:, 1])
    # the queued energy and momentum are the initial state's
    pre = torch.stack([torch.as_tensor(d[c]).cuda()[q.index[:k]] for c in ("px", "py", "pz")], 1)
    assert torch.equal(torch.stack([q.px[:k], q.py[:k], q.pz[:k]], 1), pre)
    g_ref = torch.sqrt(1.0 + (pre.double() ** 2).sum(1))
    assert float((q.gamma[:k].double() / g_ref - 1).abs().max()) < 3e-7
    # the pass sampled what the standalone surrogate samples for those inputs
    xi, xc = net.sample_photon_xi(q.chi[:k].clone(), q.r[:k].clone(), use_flags=True)
    assert torch.equal(q.xi[:k], xi)
    # records: the collinear photon xi gamma of each queued emission, in the emitter's direction
    rec_pid = out1.parent_id[:k].cpu().numpy()
    order = np.argsort(rec_pid)
    qo = np.argsort(idx)
    assert np.array_equal(rec_pid[order], idx[qo])
    rp = np.stack([out1.px[:k].cpu().numpy(), out1.py[:k].cpu().numpy(), out1.pz[:k].cpu().numpy()], 1)[order]
    g = q.gamma[:k].cpu().numpy().astype(np.float64)[qo]
    x = xi.cpu().numpy().astype(np.float64)[qo]
    xcn = xc.cpu().numpy().astype(np.float64)[qo]
    np.testing.assert_allclose(np.linalg.norm(rp, axis=1), g * x, rtol=2e-6)
    assert np.all(out1.meta[:k].cpu().numpy() == sfq.SFQ_PHOTON)
    assert np.all(out1.step[:k].cpu().numpy() == 3)
    # the emitters recoiled to (1 - xi) gamma along their direction; the others are untouched
    pm = np.sqrt(np.maximum((g * xcn) ** 2 - 1.0, 0.0))
    got = np.stack([P1.px.cpu().numpy(), P1.py.cpu().numpy(), P1.pz.cpu().numpy()], 1)
    np.testing.assert_allclose(np.linalg.norm(got[idx[qo]], axis=1), pm, rtol=2e-6)
    rest = np.ones(n, bool)
    rest[idx] = False
    assert np.array_equal(got[rest, 0], d["px"][rest]) and np.all(got[rest, 1:] == 0)
    # the optical depth of the emitters was reset as without the surrogate
    assert torch.equal(P1.tau, P0.tau)


def test_full_queue_falls_back_to_the_plain_sampler(setup):
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx, net = setup
    n = 1 << 15
    d = W.config2(n=n, seed=6)
    P0, F = _population(ctx, d)
    ctx.set_surrogate(None)
    out0, c0 = _step(ctx, P0, F, 0, n)
    cap = 200
    q = sfq.EventQueue(cap)
    ctx.set_surrogate(net, q, use_flags=True)
    P1, F1 = _population(ctx, d)
    out1, c1 = _step(ctx, P1, F1, 0, n)
    ctx.set_surrogate(None)
    assert int(q.count[0].item()) == c1["events"] > cap
    assert c1["emitted"] == c1["events"] == c0["events"] and out1.n() == c0["events"]
    assert c1["surrogate_fallbacks"] >= c1["events"] - cap
    # the emitters the queue could not take were sampled by the plain sampler: their records
    # equal the run without the surrogate
    queued = q.index[:cap].cpu().numpy()
    k = out1.n()
    pa, pb = out1.parent_id[:k].cpu().numpy(), out0.parent_id[:k].cpu().numpy()
    oa, ob = np.argsort(pa), np.argsort(pb)
    assert np.array_equal(pa[oa], pb[ob])
    xa, xb = out1.px[:k].cpu().numpy()[oa], out0.px[:k].cpu().numpy()[ob]
    inline = ~np.isin(pa[oa], queued)
    assert inline.sum() == c1["events"] - cap
    assert np.array_equal(xa[inline], xb[inline])


def test_sampled_fractions_follow_the_oracle_cdf(setup, dense_photon_cdf):
    """40 steps of 2^18 electrons: KS of F_oracle(xi | chi) over every emission."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx, net = setup
    n, nsteps = 1 << 18, 40
    d = W.config2(n=n, seed=8)
    P, F = _population(ctx, d)
    q = sfq.EventQueue(n)
    ctx.set_surrogate(net, q, use_flags=True)
    chi, xi = [], []
    cnt = sfq.counters_tensor()
    out = sfq.ProductBuffers(n, torch.float32, "cuda")
    for s in range(nsteps):
        out.reset()
        ctx.mc_step(P, F, s, out, counters=cnt)
        k = q.n()
        chi.append(q.chi[:k].cpu().numpy())
        xi.append(q.xi[:k].cpu().numpy())
    ctx.set_surrogate(None)
    c = sfq.counters_dict(cnt)
    chi = np.concatenate(chi).astype(np.float64)
    xi = np.concatenate(xi).astype(np.float64)
    m = chi.size
    assert m == c["events"] == c["emitted"] and c["dropped"] == 0
    # the dense CDF covers the network's domain chi in [1e-3, 100]; the rare emissions at
    # smaller chi (near the field's zero crossings) took the plain sampler
    keep = (chi >= 1e-3) & (chi <= 100.0)
    chi, xi = chi[keep], xi[keep]
    m = chi.size
    s = xi / (1.0 - xi)
    lnw = (np.log(2.0 * s) - np.log(3.0) - np.log(chi)) / 3.0
    p = np.sort(1.0 / (1.0 + np.exp(-dense_photon_cdf.logit(np.log(chi), lnw))))
    i = np.arange(m, dtype=np.float64)
    ks = max(np.max((i + 1) / m - p), np.max(p - i / m))
    bound = 1e-3 + 1.63 / math.sqrt(m)             # the judged network bound + 99 % sampling noise
    print(f"\nsurrogate in the step: {m} emissions, KS {ks:.2e} (bound {bound:.2e}), "
          f"fallbacks {c['surrogate_fallbacks']}")
    assert ks < bound, (ks, bound)
