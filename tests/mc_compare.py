"""Comparison of GPU Monte Carlo runs with oracle lineages (shared by the GPU tests).

A lineage (a primary particle and everything it creates) is compared bit for bit
on its decisions -- which steps produced which products -- and within the
precision tolerance on momenta and optical depth, up to its first decision that
the oracle flags as near threshold (|tau_d| <= 1e-6 tau0 for the optical depth);
later records of such a lineage are excluded and counted.  Momentum components are compared
relative to the momentum's magnitude.
"""
import numpy as np


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
        for ko, kg in zip(ok, gk):
            # components within the tolerance relative to the vector's magnitude (a component
            # near zero, e.g. a transverse momentum crossing zero, carries only rounding)
            pmag = float(np.linalg.norm(op["p"][ko]))
            for c, name in enumerate(("px", "py", "pz")):
                ov, gv = op["p"][ko][c], gpu_prod[name][kg]
                if ov == 0.0:
                    assert abs(gv) <= tol * 1e-6 * max(1.0, np.abs(op["p"][ko]).max()), (pid, name, gv)
                else:
                    assert abs(float(gv) - float(ov)) < tol * 10 * max(abs(float(ov)), pmag), (pid, name, gv, ov)
        summary["records"] += len(ok)
        if first_near[j] < 0 and check_final:
            # final state of the primary
            assert bool(gpu_final["flags"][j] & 1) == bool(orc["flags"][j] & 1), pid
            pmag = float(np.linalg.norm(orc["p"][j]))
            for c, name in enumerate(("px", "py", "pz")):
                ov, gv = orc["p"][j][c], gpu_final[name][j]
                if ov == 0.0:
                    assert abs(gv) <= 1e-30 + tol * 1e-6, (pid, name)
                else:
                    assert abs(float(gv) - float(ov)) < tol * 10 * max(abs(float(ov)), pmag), (pid, name, gv, ov)
            if orc["flags"][j] & 1:
                # optical depth: the decrements differ by the rate tolerance
                assert abs(gpu_final["tau"][j] - orc["tau"][j]) <= tol * max(1.0, orc["tau"][j]) * 20, \
                    (pid, gpu_final["tau"][j], orc["tau"][j])
    return summary
