"""GPU tests of the context options: the "fast" pair-rate cutoff and the coefficient
count of the energy samplers (Sec. 4.2 and Sec. 4.5 of the paper).

Pair-rate cutoff: W_pair is zero below chi_min and unchanged (bit for bit) above it;
a photon run with chi_min = 0.3 creates no pair at chi < 0.3.

Sampler coefficients: with k of the n coefficients per variable, every piece of the
inverse-CDF tables is truncated in the Chebyshev basis.  The sampled energies are
compared with the oracle's exact inverse transform (config-1 inputs): the error may grow
by at most the truncation error the header states, times 3 for the photon fraction
(xi = s / (1 + s), s ~ w-bar^3), and it must stay within the path's tolerance at
k = n - 1 (binary32: 1e-5).  A Monte Carlo run at k = n - 1 passes the same lineage
comparison with the oracle as the full tables.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

from mc_compare import compare_lineages
from test_gpu_mc_step import NEAR, TOL, gpu_subset, oracle_lineages

pytestmark = pytest.mark.gpu

# worst relative truncation error of w-bar (photon) and of 1 - v-bar (pair) per dropped degree
TRUNC = {"fp32": {"photon": {1: 6.4e-7, 2: 3.7e-6}, "pair": {1: 1.8e-6, 2: 8.7e-6}},
         "fp64": {"photon": {1: 6.6e-12, 2: 6.2e-11}, "pair": {1: 2.3e-11, 2: 2.0e-10}}}


def _ctx(precision, seed=0):
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    return sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=seed)


def _dev(ctx, a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=ctx.dtype)


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pair_rate_cutoff(precision):
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx(precision)
    d = W.config1()
    npd = np.float32 if precision == "fp32" else np.float64
    g, x = d["gamma_g"].astype(npd), d["chi_g"].astype(npd)
    x = np.concatenate([x, np.array([0.01, 0.2999, 0.3, 0.3001], npd)])
    g = np.concatenate([g, np.full(4, 1e3, npd)])
    full = ctx.pair_rate(_dev(ctx, g), _dev(ctx, x)).cpu().numpy()
    ctx.set_pair_rate_cutoff(0.3)
    fast = ctx.pair_rate(_dev(ctx, g), _dev(ctx, x)).cpu().numpy()
    cut = x < npd(0.3)
    # (W_pair ~ exp(-8/(3 chi)) underflows binary32 near chi = 0.01, so only most of the
    # full rates below the cutoff are nonzero)
    assert np.all(fast[cut] == 0.0) and np.count_nonzero(full[cut]) > 0.9 * cut.sum()
    np.testing.assert_array_equal(fast[~cut], full[~cut])
    for bad in (0.005, -1.0, 3000.0, float("nan")):
        with pytest.raises(sfq.SfqError):
            ctx.set_pair_rate_cutoff(bad)
    ctx.set_pair_rate_cutoff(0.01)
    back = ctx.pair_rate(_dev(ctx, g), _dev(ctx, x)).cpu().numpy()
    np.testing.assert_array_equal(back, full)
    ctx.close()


def test_photon_run_with_fast_cutoff():
    """Config-3 photons with chi_min = 0.3: every conversion happens at chi >= 0.3."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx("fp32", seed=31)
    ctx.set_pair_rate_cutoff(0.3)
    n, nsteps = 8192, 60
    d = W.config3(n=n, seed=2)
    T = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=dt)
    P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"], torch.float64), T(d["flags"]))
    F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), T(d["table"]), d["k_step"], amp=T(d["amp"]))
    out, cnt = sfq.ProductBuffers(4 * n, ctx.dtype, ctx.device), sfq.counters_tensor()
    for s in range(nsteps):
        ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert c["pairs"] > 100
    k = out.n()
    pid = out.parent_id[:k].cpu().numpy().astype(np.int64)
    step = out.step[:k].cpu().numpy().astype(np.int64)
    (_, ey, _), _ = W.plane_wave_fields(d["k0"][pid], d["amp"][pid], d["table"], step)
    chi_ev = 2.0 * np.abs(d["px"][pid].astype(np.float64)) * np.abs(ey.astype(np.float64)) / W.RHO
    assert chi_ev.min() >= 0.3 * (1 - 1e-5), chi_ev.min()
    # photons whose peak chi is below the cutoff never convert
    low = np.nonzero(d["chi_peak"] < 0.29)[0]
    assert np.all(P.flags[torch.as_tensor(low, device=ctx.device)].cpu().numpy() & 1)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sampler_coefficients(precision, oracle):
    ctx = _ctx(precision)
    n, k = ctx.sampler_coefficients()
    assert (n, k) == ((9, 9) if precision == "fp32" else (12, 12))
    d = W.config1()
    npd = np.float32 if precision == "fp32" else np.float64
    words = oracle.philox(d["id_e"], 0, 0, ctx.seed)
    r = oracle.uniforms_from_words(words)[:, 1]
    xe_chi = d["chi_e"].astype(npd).astype(np.float64)
    xg_chi = d["chi_g"].astype(npd).astype(np.float64)
    s = oracle.photon_s(r, xe_chi)
    ref_xi = s / (1 + s)
    ref_e, ref_p = oracle.pair_shares(r, xg_chi)
    errs = {}
    for drop in (0, 1, 2):
        ctx.set_sampler_coefficients(n - drop)
        assert ctx.sampler_coefficients() == (n, n - drop)
        xi, _ = ctx.sample_photon_xi(_dev(ctx, xe_chi), _dev(ctx, r))
        xe, xp = ctx.sample_pair_xi(_dev(ctx, xg_chi), _dev(ctx, r))
        e_ph = _rel(xi.cpu().numpy(), ref_xi).max()
        e_pp = max(_rel(xe.cpu().numpy(), ref_e).max(), _rel(xp.cpu().numpy(), ref_p).max())
        errs[drop] = (e_ph, e_pp)
    base_ph, base_pp = errs[0]
    assert base_ph < TOL[precision] and base_pp < TOL[precision]
    for drop in (1, 2):
        e_ph, e_pp = errs[drop]
        assert e_ph <= base_ph + 3 * TRUNC[precision]["photon"][drop] * 1.5, (drop, errs)
        assert e_pp <= base_pp + TRUNC[precision]["pair"][drop] * 1.5, (drop, errs)
    assert errs[1][0] < TOL[precision] and errs[1][1] < TOL[precision], errs
    from paper_2301_07684_gb300 import sfq
    for bad in (n + 1, n - 3, 0):
        with pytest.raises(sfq.SfqError):
            ctx.set_sampler_coefficients(bad)
    print(f"\n{precision} sampler error vs oracle (photon xi, pair shares) by dropped degree: {errs}")
    ctx.close()


def test_step_with_truncated_sampler(oracle):
    """Config-2 run with k = n - 1 on the binary32 path: lineages agree with the oracle."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx("fp32", seed=2024)
    ctx.set_sampler_coefficients(8)
    n, nsteps = 8192 + 77, 60
    d = W.config2(n=n, seed=0)
    T = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=dt)
    P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"], torch.float64), T(d["flags"]))
    F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), T(d["table"]), d["k_step"], amp0=d["amp0"])
    out, cnt = sfq.ProductBuffers(8 * n, ctx.dtype, ctx.device), sfq.counters_tensor()
    for s in range(nsteps):
        ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    ids = np.unique(np.concatenate([W.sample_ids(n, 128, seed=5), [0, n - 1]]))
    orc = oracle_lineages(oracle, d, ids, nsteps, ctx.rho, ctx.seed, NEAR["fp32"])
    final, prod = gpu_subset(P, out, ids)
    s = compare_lineages(ids, orc, final, prod, TOL["fp32"], nsteps)
    assert s["records"] > 100 and s["near"] <= 2, s
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_clenshaw_evaluator_agrees_with_horner(precision):
    """The Chebyshev pieces evaluated by Clenshaw's recurrence give Horner's values on the
    monomial pieces to rounding (rates and both samplers over their whole domains); the
    evaluator excludes the truncated samplers; switching back restores Horner bit for bit."""
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=0)
    g = np.random.default_rng(4)
    n = 1 << 16
    dev = lambda a: torch.as_tensor(a).to(device=ctx.device, dtype=ctx.dtype)
    chi = dev(10.0 ** g.uniform(-4, 3.2, n))
    gam = dev(10.0 ** g.uniform(1, 5, n))
    r = dev(g.uniform(2.0 ** -24, 1 - 2.0 ** -24, n))

    def evaluate():
        return [ctx.photon_rate(gam, chi), ctx.pair_rate(gam, chi), *ctx.sample_photon_xi(chi, r),
                *ctx.sample_pair_xi(chi, r)]

    h = evaluate()
    ctx.set_evaluator(sfq.SFQ_EVAL_CLENSHAW)
    c = evaluate()
    # rounding of the two evaluations (binary32: ~2e-7 each, times 3 through s ~ w-bar^3)
    tol = 4e-6 if precision == "fp32" else 1e-13
    for a, b in zip(h, c):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        big = np.abs(a) > (np.finfo(np.float32).tiny * 1e3 if precision == "fp32" else 1e-300)
        assert big.mean() > 0.5
        assert (np.abs(b[big] - a[big]) / np.abs(a[big])).max() <= tol
    assert any(not torch.equal(a, b) for a, b in zip(h, c))           # another evaluation ran
    with pytest.raises(sfq.SfqError):
        ctx.set_sampler_coefficients(sfq_k(ctx) - 1)
    ctx.set_evaluator(sfq.SFQ_EVAL_HORNER)
    for a, b in zip(h, evaluate()):
        assert torch.equal(a, b)
    ctx.set_sampler_coefficients(sfq_k(ctx) - 1)
    with pytest.raises(sfq.SfqError):
        ctx.set_evaluator(sfq.SFQ_EVAL_CLENSHAW)
    ctx.close()


def sfq_k(ctx):
    return ctx.sampler_coefficients()[0]

