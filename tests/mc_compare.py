"""Comparison of GPU Monte Carlo runs with oracle lineages (shared by the GPU tests).

A lineage (a primary particle and everything it creates) is compared bit for bit
on its decisions -- which steps produced which products -- and within an error
budget on momenta and optical depth, up to its first decision that the oracle
flags as near threshold (|tau_d| <= 1e-6 tau0 for the optical depth); later
records of such a lineage are excluded and counted.  Momentum components are
compared relative to the momentum's magnitude.

The budget follows from the stated tolerance `tol` of the rates and of the sampled
fractions xi and 1 - xi (1e-5 binary32, 1e-10 binary64; Eq. pe_rate_3, Eq. again):
  - an event multiplies the emitter's energy by 1 - xi and gives the photon xi gamma,
    so each event adds at most tol to the relative error of the energies it produces;
  - an emitter that carries a relative error e samples its next xi at chi ~ gamma that
    is off by e, and the fraction moves with chi at most in proportion
    (d ln xi / d ln chi <= 1), so the product of its next event carries up to 2 e + tol;
  - hence an emitter with k earlier events (a lepton created by a pair conversion
    counts its creation as one) produces a record within tol (1 + 2 k) and holds a
    momentum within tol (1 + 2 k);
  - the optical depth consumed since the last reset is a sum of rates R dt, each within
    tol + e of the oracle's (R ~ W~_rad(chi) chi / gamma and |d ln W~_rad / d ln chi| <= 1),
    and never exceeds the drawn tau0 = -ln u <= 24 ln 2 (u >= 2^-24), so the final tau_d
    is within 24 ln 2 tol (1 + 2 K) after K events.
"""
import math

import numpy as np

TAU0_MAX = 24 * math.log(2.0)         # the largest -ln u of the uniform map (u >= 2^-24)


def budget(tol, k):
    """Relative error budget of an energy produced after k earlier events in its chain."""
    return tol * (1 + 2 * k)


def _rel(a, b):
    return np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / np.maximum(np.abs(b), 1e-300)


def compare_lineages(ids, orc, gpu_final, gpu_prod, tol, nsteps, step0=0, check_final=True):
    """ids: primary ids checked; orc: oracle.mc_run result for those ids (same order);
    gpu_final: dict with px, py, pz, tau, flags for the same ids;
    gpu_prod: dict of numpy arrays (px, py, pz, parent_id, step, meta) of records whose
    parent is one of the ids.  Returns a summary dict; raises AssertionError on a mismatch."""
    summary = dict(lineages=len(ids), near=0, records=0, excluded_records=0, events=int(orc["n_events"].sum()))
    first_near = orc["first_near_step"]
    # oracle products per parent
    op = orc["products"]
    o_key = {}
    for k in range(len(op)):
        o_key.setdefault(int(op["parent_id"][k]), []).append(k)
    g_key = {}
    for k in range(len(gpu_prod["parent_id"])):
        g_key.setdefault(int(gpu_prod["parent_id"][k]), []).append(k)
    for j, pid in enumerate(ids):
        pid = int(pid)
        cut = first_near[j] if first_near[j] >= 0 else step0 + nsteps
        if first_near[j] >= 0:
            summary["near"] += 1
        ok = [k for k in o_key.get(pid, []) if op["step"][k] < cut]
        gk = [k for k in g_key.get(pid, []) if gpu_prod["step"][k] < cut]
        summary["excluded_records"] += len(o_key.get(pid, [])) - len(ok)

        def okey(k):
            return (int(op["step"][k]), int(op["member"][k]), int(op["parent_tag"][k]))

        def gkey(k):
            m = int(gpu_prod["meta"][k])
            return (int(gpu_prod["step"][k]), (m >> 2) & 3, (m >> 4) & 3)

        ok.sort(key=okey)
        gk.sort(key=gkey)
        assert [okey(k) for k in ok] == [gkey(k) for k in gk], \
            f"lineage {pid}: oracle records {[okey(k) for k in ok]} vs gpu {[gkey(k) for k in gk]}"
        # earlier events of each emitter (parent tag 0: the primary; 1, 2: the leptons of its
        # conversion, whose creation counts as one) before each record, in step order
        seen = {}
        for ko, kg in zip(ok, gk):
            step, member, ptag = okey(ko)
            if member == 0:
                k = seen.get(ptag, 1 if ptag else 0)
                seen[ptag] = k + 1
            else:
                k = seen.get(0, 0)                   # the converting photon: its own events (none)
            b = budget(tol, k)
            summary["max_budget_k"] = max(summary.get("max_budget_k", 0), k)
            # components within the budget relative to the vector's magnitude (a component
            # near zero, e.g. a transverse momentum crossing zero, carries only rounding)
            pmag = float(np.linalg.norm(op["p"][ko]))
            for c, name in enumerate(("px", "py", "pz")):
                ov, gv = op["p"][ko][c], gpu_prod[name][kg]
                if ov == 0.0:
                    assert abs(gv) <= tol * 1e-6 * max(1.0, np.abs(op["p"][ko]).max()), (pid, name, gv)
                else:
                    assert abs(float(gv) - float(ov)) < b * max(abs(float(ov)), pmag), (pid, name, gv, ov, k)
        summary["records"] += len(ok)
        if first_near[j] < 0 and check_final:
            # final state of the primary after its K events
            K = seen.get(0, 0)
            b = budget(tol, K)
            assert bool(gpu_final["flags"][j] & 1) == bool(orc["flags"][j] & 1), pid
            pmag = float(np.linalg.norm(orc["p"][j]))
            for c, name in enumerate(("px", "py", "pz")):
                ov, gv = orc["p"][j][c], gpu_final[name][j]
                if ov == 0.0:
                    assert abs(gv) <= 1e-30 + tol * 1e-6, (pid, name)
                else:
                    assert abs(float(gv) - float(ov)) < b * max(abs(float(ov)), pmag), (pid, name, gv, ov, K)
            if orc["flags"][j] & 1:
                assert abs(gpu_final["tau"][j] - orc["tau"][j]) <= TAU0_MAX * b, \
                    (pid, gpu_final["tau"][j], orc["tau"][j], K)
    return summary
