"""GPU parity of the rate and sampling entry points against the FP64 oracle.

Workload: config 1 (4096 electrons with gamma log-uniform in [10, 1e4] and chi
log-uniform in [1e-3, 10]; 4096 photons with chi log-uniform in [0.1, 100] and
gamma log-uniform in [1e2, 1e5]; one energy sample per particle from Philox,
seed 0, step 0), plus edge cases: chi = 0, piece boundaries, the ends of the
fitted ranges, r at the ends of the uniform grid.
Tolerances: 1e-5 relative on the binary32 path, 1e-10 on the binary64 path; the
Philox words are compared bit for bit.  Every test runs with both evaluators of the
fitted tables: Horner on the monomial pieces and Clenshaw on the same pieces in the
Chebyshev basis (sfq_set_evaluator).
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", params=["fp32", "fp64", "fp32/clenshaw", "fp64/clenshaw"])
def ctx(request):
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    precision, _, evaluator = request.param.partition("/")
    c = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=0)
    if evaluator:
        c.set_evaluator(sfq.SFQ_EVAL_CLENSHAW)
    c.name = precision
    yield c
    c.close()


def _dev(ctx, a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=ctx.dtype)


def _cast(ctx, a):
    """The values the device sees, as float64 for the oracle."""
    return np.asarray(a, dtype=np.float32 if ctx.name == "fp32" else np.float64).astype(np.float64)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def test_prefactor_matches_oracle(ctx, oracle):
    rho = oracle.rho_from_ref_len(W.REF_LEN)
    assert ctx.rho == pytest.approx(rho, rel=1e-15)
    assert ctx.pref == pytest.approx(oracle.rate_prefactor(rho), rel=1e-15)


def test_photon_rate_config1(ctx, oracle):
    d = W.config1()
    g, x = _cast(ctx, d["gamma_e"]), _cast(ctx, d["chi_e"])
    gpu = ctx.photon_rate(_dev(ctx, g), _dev(ctx, x)).cpu().numpy()
    ref = oracle.photon_rate(g, x, oracle.rate_prefactor(ctx.rho))
    assert _rel(gpu, ref).max() < TOL[ctx.name]


def test_pair_rate_config1(ctx, oracle):
    d = W.config1()
    g, x = _cast(ctx, d["gamma_g"]), _cast(ctx, d["chi_g"])
    gpu = ctx.pair_rate(_dev(ctx, g), _dev(ctx, x)).cpu().numpy()
    ref = oracle.pair_rate(g, x, oracle.rate_prefactor(ctx.rho))
    assert _rel(gpu, ref).max() < TOL[ctx.name]


def _edge_chis(lo_exp, hi_exp, extra):
    v = [extra]
    for e in range(lo_exp, hi_exp + 1):
        b = 2.0 ** e
        v += [b, b * (1 - 2 ** -20), b * (1 + 2 ** -20), 1.5 * b, 1.25 * b, 1.75 * b]
    return np.concatenate([np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in v])


def test_photon_rate_whole_range(ctx, oracle):
    chis = _edge_chis(-12, 19, [0.0, 1e-9, 1e-6, 2000.0])
    chis = _cast(ctx, chis)
    g = np.full_like(chis, 1000.0)
    gpu = ctx.photon_rate(_dev(ctx, g), _dev(ctx, chis)).cpu().numpy()
    ref = oracle.photon_rate(g, chis, oracle.rate_prefactor(ctx.rho))
    nz = ref > 0
    assert np.all(gpu[~nz] == 0)
    assert _rel(gpu[nz], ref[nz]).max() < TOL[ctx.name]


def test_pair_rate_whole_range(ctx, oracle):
    chis = _cast(ctx, _edge_chis(-7, 19, [0.0, 0.0099, 0.01, 0.0100001, 0.24, 2000.0]))
    g = np.full_like(chis, 1000.0)
    gpu = ctx.pair_rate(_dev(ctx, g), _dev(ctx, chis)).cpu().numpy()
    ref = oracle.pair_rate(g, chis, oracle.rate_prefactor(ctx.rho))
    zero = ref == 0
    assert np.all(gpu[zero] == 0)
    # binary32 cannot hold rates below its normal range; compare those absolutely
    tiny = np.finfo(np.float32).tiny if ctx.name == "fp32" else 0.0
    big = (~zero) & (ref > tiny / TOL[ctx.name])
    assert _rel(gpu[big], ref[big]).max() < TOL[ctx.name]
    small = (~zero) & ~big
    assert np.all(np.abs(gpu[small] - ref[small]) <= 2 * tiny)


def test_uniforms_bit_exact(ctx, oracle):
    import torch
    ids = torch.arange(4096, dtype=torch.int64, device=ctx.device) * 7919 + 3
    u = ctx.uniforms(ids, step=11, tag=2).cpu().numpy()
    words = oracle.philox(ids.cpu().numpy().astype(np.uint64), 11, 2, ctx.seed)
    ref = oracle.uniforms_from_words(words)
    np.testing.assert_array_equal(u.astype(np.float64), ref)


def _oracle_r(oracle, ids, seed):
    return oracle.uniforms_from_words(oracle.philox(ids, 0, 0, seed))[:, 1]


def test_photon_xi_config1(ctx, oracle):
    d = W.config1()
    x = _cast(ctx, d["chi_e"])
    r = _oracle_r(oracle, d["id_e"], ctx.seed)            # word 1 of Philox(seed 0, id, step 0)
    xi, xic = ctx.sample_photon_xi(_dev(ctx, x), _dev(ctx, r))
    s = oracle.photon_s(r, x)
    assert _rel(xi.cpu().numpy(), s / (1 + s)).max() < TOL[ctx.name]
    assert _rel(xic.cpu().numpy(), 1 / (1 + s)).max() < TOL[ctx.name]


def test_pair_xi_config1(ctx, oracle):
    d = W.config1()
    x = _cast(ctx, d["chi_g"])
    r = _oracle_r(oracle, d["id_g"], ctx.seed)
    xe, xp = ctx.sample_pair_xi(_dev(ctx, x), _dev(ctx, r))
    re, rp = oracle.pair_shares(r, x)
    assert _rel(xe.cpu().numpy(), re).max() < TOL[ctx.name]
    assert _rel(xp.cpu().numpy(), rp).max() < TOL[ctx.name]


def _edge_r():
    r = [2.0 ** -24, 3 * 2.0 ** -24, 0.5 - 2.0 ** -24, 0.5 + 2.0 ** -24, 1 - 2.0 ** -24, 1 - 3 * 2.0 ** -24]
    for e in range(-23, -1):
        r += [2.0 ** e + 2.0 ** -24, 2.0 ** e - 2.0 ** -24, 1 - 2.0 ** e + 2.0 ** -24, 1 - 2.0 ** e - 2.0 ** -24]
    return np.array(sorted(set(r)))


def test_photon_xi_edges(ctx, oracle):
    r = _edge_r()
    chis = np.array([0.0, 1e-7, 2.0 ** -10, 2.0 ** -10 * (1 - 2 ** -20), 0.3, 1.0, 7.5, 2000.0, 4095.0])
    R, X = np.meshgrid(r, chis)
    R, X = _cast(ctx, R.ravel()), _cast(ctx, X.ravel())
    xi, xic = ctx.sample_photon_xi(_dev(ctx, X), _dev(ctx, R))
    s = oracle.photon_s(R, X)
    ok = s > 0
    assert np.all(xi.cpu().numpy()[~ok] == 0)
    assert _rel(xi.cpu().numpy()[ok], (s / (1 + s))[ok]).max() < TOL[ctx.name]
    assert _rel(xic.cpu().numpy(), 1 / (1 + s)).max() < TOL[ctx.name]


def test_pair_xi_edges(ctx, oracle):
    r = _edge_r()
    chis = np.array([0.01, 0.0123, 2.0 ** -6, 0.3, 1.0, 7.5, 2000.0, 4095.0])
    R, X = np.meshgrid(r, chis)
    R, X = _cast(ctx, R.ravel()), _cast(ctx, X.ravel())
    xe, xp = ctx.sample_pair_xi(_dev(ctx, X), _dev(ctx, R))
    re, rp = oracle.pair_shares(R, X)
    assert _rel(xe.cpu().numpy(), re).max() < TOL[ctx.name]
    assert _rel(xp.cpu().numpy(), rp).max() < TOL[ctx.name]


def test_empty_and_ragged_sizes(ctx):
    import torch
    e = torch.empty(0, dtype=ctx.dtype, device=ctx.device)
    assert ctx.photon_rate(e, e).numel() == 0
    for n in (1, 3, 255, 257, 1023, 1025):
        g = torch.full((n,), 100.0, dtype=ctx.dtype, device=ctx.device)
        x = torch.full((n,), 0.5, dtype=ctx.dtype, device=ctx.device)
        r = ctx.photon_rate(g, x)
        assert torch.all(r == r[0]).item() and r[0].item() > 0


def test_counters_count_out_of_range(ctx):
    import torch
    from paper_2301_07684_gb300 import sfq
    cnt = sfq.counters_tensor()
    g = torch.full((4,), 100.0, dtype=ctx.dtype, device=ctx.device)
    x = torch.tensor([0.5, 2.0 ** 21, float("nan"), 1.0], dtype=ctx.dtype, device=ctx.device)
    out = ctx.photon_rate(g, x, counters=cnt)
    d = sfq.counters_dict(cnt)
    assert d["out_of_range"] == 1 and d["nan_input"] == 1
    assert out[2].item() == 0.0


def test_argument_errors(ctx):
    import torch
    from paper_2301_07684_gb300 import sfq
    g = torch.full((8,), 100.0, dtype=ctx.dtype, device=ctx.device)
    with pytest.raises(sfq.SfqError):
        ctx.photon_rate(g[1:], g[1:])        # misaligned by one element
