"""GPU parity of the Boris push (sfq_push) against the oracle's push.

Workload: a config-2 population (electrons, gamma ~ N(2000, 5%)) with positrons and photons
mixed in, in random structure-of-arrays fields of the wave's strength (|E|, |B| ~ 100) and
in the plane wave; 16384 + 77 particles (several blocks and a ragged tail), dt = 0.01
periods.  Tolerance: |u_gpu - u_oracle| <= 2e-6 |u| (binary32) and 1e-13 |u| (binary64),
component by component; photons and dead particles bit for bit unchanged.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {"fp32": 2e-6, "fp64": 1e-13}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("field_mode", ["soa", "pw"])
def test_push_matches_oracle(oracle, precision, field_mode):
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=1)
    npd = np.float32 if precision == "fp32" else np.float64
    n = 16384 + 77
    d = W.config2(n=n, seed=9, dtype=npd)
    g = np.random.default_rng(4)
    flags = d["flags"].copy()
    sp = g.integers(0, 3, n)
    flags = (1 | (sp << 2)).astype(np.uint8)
    flags[::97] &= np.uint8(0xFE)                      # some dead particles
    u0 = np.stack([d["px"], d["py"], d["pz"]], 1).astype(npd)
    u0[:, 1] = g.normal(0.0, 30.0, n).astype(npd)      # momenta off the axis
    T = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=dt)
    P = sfq.ParticleBuffers(T(u0[:, 0]), T(u0[:, 1]), T(u0[:, 2]), T(d["tau"], torch.float64), T(flags))
    step = 5
    if field_mode == "soa":
        E = g.normal(0.0, 100.0, (n, 3)).astype(npd)
        B = g.normal(0.0, 100.0, (n, 3)).astype(npd)
        F = sfq.FieldSource.soa(*(T(E[:, k]) for k in range(3)), *(T(B[:, k]) for k in range(3)))
    else:
        F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), T(d["table"]), d["k_step"], amp0=d["amp0"])
        (ex, ey, ez), (bx, by, bz) = W.plane_wave_fields(d["k0"], d["amp0"], d["table"], step)
        E = np.stack([ex, ey, ez], 1).astype(npd)
        B = np.stack([bx, by, bz], 1).astype(npd)
    ctx.push(P, F, step, W.DT)
    torch.cuda.synchronize()
    gpu = np.stack([P.px.cpu().numpy(), P.py.cpu().numpy(), P.pz.cpu().numpy()], 1).astype(np.float64)
    q = np.where(sp == 0, -1.0, np.where(sp == 1, 1.0, 0.0))
    q[(flags & 1) == 0] = 0.0
    ref = oracle.boris_push(u0.astype(np.float64), E.astype(np.float64), B.astype(np.float64), q, W.DT)
    mag = np.linalg.norm(u0.astype(np.float64), axis=1)[:, None]
    moved = q != 0.0
    err = np.abs(gpu[moved] - ref[moved]) / mag[moved]
    assert err.max() < TOL[precision], err.max()
    np.testing.assert_array_equal(gpu[~moved], u0[~moved].astype(np.float64))
    from paper_2301_07684_gb300.sfq import SfqError
    with pytest.raises(SfqError):
        ctx.push(P, F, step, -1.0)
    ctx.close()
