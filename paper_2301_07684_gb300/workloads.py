"""Seeded synthetic inputs (laser-beam-shaped workloads).

Inputs only: this module holds none of the method's arithmetic (no chi, no rates,
no sampling).  Both the CUDA path and the test oracle are fed from it.

Workloads (normalised units: times 1/omega_r, fields E_r = m c omega_r/|e|,
momenta m c; the laser has wavelength 0.8 um and omega_r = 2 pi c / lambda):
  config 1  rates and one energy sample: 4096 electrons with gamma log-uniform in
            [10, 1e4], p along +x, E_y chosen so that chi is log-uniform in
            [1e-3, 10], B = 0; 4096 photons with chi log-uniform in [0.1, 100] and
            gamma log-uniform in [1e2, 1e5].
  config 2  2^24 electrons, gamma ~ Normal(2000, 5%), p along -x, in a linearly
            polarised plane wave along +x with a0 = 100: E_y = B_z = a0 cos(phi),
            per-particle phase uniform in [0, 2 pi), 200 steps of 0.01 laser period.
  config 3  2^24 photons with peak chi log-uniform in [0.1, 100] and gamma
            log-uniform in [1e2, 1e5], p along -x, each in a plane wave whose
            amplitude gives that peak chi; 100 steps.
  config 4  64 beams with particle counts log-uniform in [1e3, 4e6], one species
            each (uniform over e-, e+, photon), a0 uniform in [10, 300], gamma0
            log-uniform in [200, 1e4]; 500 steps.
The phase of a particle moving at -c through the wave advances by 2 omega_r dt per
step; it is kept as an integer index into a cosine table of K = 6400 entries
(k_step = 128 per step for dt = 0.01 periods), so that host and device form the
same field values (one rounded product amp * cos).
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA_C = 3.8615926796e-13          # reduced Compton length [m], CODATA 2018
WAVELENGTH = 0.8e-6
REF_LEN = WAVELENGTH / (2 * math.pi)  # lambda_r = lambda / 2 pi
RHO = REF_LEN / LAMBDA_C              # critical field in units of E_r
DT = 0.01 * 2 * math.pi               # 0.01 laser period in 1/omega_r
K_TABLE = 6400
K_STEP = 128                          # 2 omega_r dt / (2 pi / K_TABLE)

SP_ELECTRON, SP_POSITRON, SP_PHOTON = 0, 1, 2
ALIVE = 1
SPECIES_SHIFT = 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def log_uniform(g, lo, hi, n):
    return np.exp(g.uniform(math.log(lo), math.log(hi), n))


def cos_table(dtype=np.float32, K=K_TABLE):
    return np.cos(2 * np.pi * np.arange(K) / K).astype(dtype)


def plane_wave_fields(k0, amp, table, step, k_step=K_STEP):
    """(E, B) of the wave at integer phase index k0 + step*k_step (host reference of the
    device's plane-wave field source; the product amp*cos is formed in table's dtype)."""
    K = table.shape[0]
    idx = (k0.astype(np.int64) + (step * k_step) % K) % K
    f = (np.asarray(amp, dtype=table.dtype) * table[idx]).astype(table.dtype)
    z = np.zeros_like(f)
    return (z, f, z), (z, z, f)


def flags_for(species, n):
    return np.full(n, ALIVE | (species << SPECIES_SHIFT), dtype=np.uint8)


def config1(seed=0, n=4096, dtype=np.float64):
    g = rng(seed)
    ge = log_uniform(g, 10.0, 1e4, n)
    chi_e = log_uniform(g, 1e-3, 10.0, n)
    ey = chi_e * RHO / ge                           # E_y such that gamma |E_y| / F_cr = chi
    gg = log_uniform(g, 1e2, 1e5, n)
    chi_g = log_uniform(g, 0.1, 100.0, n)
    return dict(gamma_e=ge.astype(dtype), chi_e=chi_e.astype(dtype), ey_e=ey.astype(dtype),
                gamma_g=gg.astype(dtype), chi_g=chi_g.astype(dtype),
                id_e=np.arange(n, dtype=np.uint64), id_g=np.arange(n, 2 * n, dtype=np.uint64))


def config2(n=1 << 24, seed=0, dtype=np.float32, a0=100.0, gamma0=2000.0, spread=0.05):
    g = rng(seed)
    gam = g.normal(gamma0, spread * gamma0, n)
    pm = np.sqrt(gam * gam - 1.0)
    k0 = g.integers(0, K_TABLE, n, dtype=np.uint32)
    return dict(px=(-pm).astype(dtype), py=np.zeros(n, dtype), pz=np.zeros(n, dtype),
                tau=np.full(n, -1.0), flags=flags_for(SP_ELECTRON, n), k0=k0,
                amp0=float(np.asarray(a0, dtype=dtype)), table=cos_table(dtype), k_step=K_STEP,
                dt=DT, rho=RHO, nsteps=200)


def config3(n=1 << 24, seed=0, dtype=np.float32):
    g = rng(seed)
    chi_peak = log_uniform(g, 0.1, 100.0, n)
    gam = log_uniform(g, 1e2, 1e5, n)
    k0 = g.integers(0, K_TABLE, n, dtype=np.uint32)
    amp = chi_peak * RHO / (2.0 * gam)              # head-on photon: chi = 2 gamma a |cos| / rho
    return dict(px=(-gam).astype(dtype), py=np.zeros(n, dtype), pz=np.zeros(n, dtype),
                tau=np.full(n, -1.0), flags=flags_for(SP_PHOTON, n), k0=k0, amp=amp.astype(dtype),
                table=cos_table(dtype), k_step=K_STEP, dt=DT, rho=RHO, nsteps=100, chi_peak=chi_peak)


def config4(seed=0, dtype=np.float32, nbeams=64, scale=1.0):
    g = rng(seed)
    counts = np.maximum(1, np.round(log_uniform(g, 1e3, 4e6, nbeams) * scale)).astype(np.int64)
    species = g.integers(0, 3, nbeams)
    a0 = g.uniform(10.0, 300.0, nbeams)
    gamma0 = log_uniform(g, 200.0, 1e4, nbeams)
    n = int(counts.sum())
    beam = np.repeat(np.arange(nbeams), counts)
    gam = gamma0[beam] * (1.0 + 0.05 * g.standard_normal(n))
    sp = species[beam]
    pm = np.where(sp == SP_PHOTON, gam, np.sqrt(np.maximum(gam * gam - 1.0, 0.0)))
    k0 = g.integers(0, K_TABLE, n, dtype=np.uint32)
    flags = (ALIVE | (sp << SPECIES_SHIFT)).astype(np.uint8)
    return dict(px=(-pm).astype(dtype), py=np.zeros(n, dtype), pz=np.zeros(n, dtype), tau=np.full(n, -1.0),
                flags=flags, k0=k0, amp=a0[beam].astype(dtype), table=cos_table(dtype), k_step=K_STEP,
                dt=DT, rho=RHO, nsteps=500, counts=counts, species=species, a0=a0, gamma0=gamma0)


def sample_ids(n, k, seed=1):
    """k distinct particle indices of n, chosen by a seeded generator (for oracle subsets)."""
    g = rng(seed)
    return np.sort(g.choice(n, size=min(k, n), replace=False))
