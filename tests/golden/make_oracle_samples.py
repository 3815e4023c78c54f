"""Write a golden fixture of the FP64 oracle's converged solution of one
workload: cycle count, final relative residual, residual history (every 50
cycles), the solution norm and the solution at seeded sample points.

Calls only the oracle (oracle/) and the seeded input generators; nothing from
the CUDA path.  Usage:
    python tests/golden/make_oracle_samples.py ecs_const  [out.json]
    python tests/golden/make_oracle_samples.py layered    [out.json]
    python tests/golden/make_oracle_samples.py --divergence layered
    python tests/golden/make_oracle_samples.py --gmres bump
    python tests/golden/make_oracle_samples.py --gmres ionization 4   (k0 = 4)
    python tests/golden/make_oracle_samples.py --gmres-history layered 512 12
    python tests/golden/make_oracle_samples.py --fgmres-gmres layered 512 12
"""

import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1211_4752_gb300 import workloads  # noqa: E402


def divergence(w, out):
    """Residual history of the oracle's cycle loop on a workload where the
    weighted-Jacobi cycle diverges (Sec. 3.2): rho_k until rho > 1e3."""
    H = oracle.build_hierarchy(w["n"], w["dim"], w["k2"], layers=w["layers"])
    f = w["rhs"][0]
    u = np.zeros_like(f)
    nf = np.linalg.norm(f)
    hist = []
    while len(hist) < 200:
        u = oracle.vcycle(H, 0, u, f)
        rho = float(np.linalg.norm(f - oracle.apply_operator(H.levels[0], u)) / nf)
        hist.append(rho)
        if not (rho <= 1e3):
            break
    data = dict(workload=w["name"], n=w["n"], dim=w["dim"], layers=w["layers"],
                diverged_at_cycle=len(hist), history=hist,
                note="FP64 oracle, V(1,1) weighted Jacobi 0.8, u0 = 0; rho_k after cycle k")
    out.write_text(json.dumps(data))
    print(out, len(hist), hist[-1])


def gmres_history(w, out, cycles=400):
    """rho_k of the oracle's GMRES(3)-smoothed cycle loop for a fixed number of
    cycles, with no stop test (the loop stagnates or diverges on the thin-layer
    layered medium; this records its course)."""
    H = oracle.build_hierarchy(w["n"], w["dim"], w["k2"], layers=w["layers"], smoother="gmres")
    f = w["rhs"][0]
    u = np.zeros_like(f)
    nf = np.linalg.norm(f)
    hist = []
    for _ in range(cycles):
        u = oracle.vcycle(H, 0, u, f)
        hist.append(float(np.linalg.norm(f - oracle.apply_operator(H.levels[0], u)) / nf))
    data = dict(workload=w["name"], n=w["n"], dim=w["dim"], layers=w["layers"], history=hist,
                note="FP64 oracle, V(1,1) GMRES(3) smoothing, u0 = 0; rho_k after cycle k")
    out.write_text(json.dumps(data))
    print(out, len(hist), hist[-1])


def fgmres_gmres(w, out, m=32):
    """FGMRES(m) right-preconditioned by one GMRES(3)-smoothed V-cycle per
    iteration (the use of the cycle in Table 3), to 1e-6: iterations, the
    residual at each restart and the solution at seeded sample points."""
    t0 = time.time()
    H = oracle.build_hierarchy(w["n"], w["dim"], w["k2"], layers=w["layers"], smoother="gmres")
    f = w["rhs"][0]
    res = oracle.fgmres(H, f, tol=1e-6, m=m, max_iter=5000)
    u = res.u
    rng = np.random.default_rng(1234)
    N = w["n"] - 1
    idx = [tuple(int(v) for v in rng.integers(0, N, size=w["dim"])) for _ in range(512)]
    vals = [[float(u[i].real), float(u[i].imag)] for i in idx]
    data = dict(workload=w["name"], n=w["n"], dim=w["dim"], layers=w["layers"], tol=1e-6,
                restart=m, iterations=res.cycles, restart_history=[float(x) for x in res.history],
                u_norm=float(np.linalg.norm(u)), sample_index=idx, sample_value=vals,
                seconds=time.time() - t0,
                note="FP64 oracle, FGMRES(%d) with one V(1,1) GMRES(3)-smoothed cycle per "
                     "iteration as right preconditioner, u0 = 0" % m)
    out.write_text(json.dumps(data))
    print(out, res.cycles, res.history[-1], data["seconds"])


def main():
    which = sys.argv[1]
    if which in ("--gmres-history", "--fgmres-gmres"):
        w = getattr(workloads, sys.argv[2])(*[int(a) for a in sys.argv[3:]])
        if which == "--gmres-history":
            gmres_history(w, Path(__file__).with_name(w["name"] + "_gmres_history.json"))
        else:
            fgmres_gmres(w, Path(__file__).with_name(w["name"] + "_fgmres32_gmres.json"))
        return
    if which == "--divergence":
        w = getattr(workloads, sys.argv[2])()
        divergence(w, Path(__file__).with_name(w["name"] + "_divergence.json"))
        return
    smoother = "jacobi"
    if which == "--gmres":      # GMRES(3) smoothing (Sec. 3.2)
        smoother = "gmres"
        which = sys.argv[2]
    extra = [int(a) for a in sys.argv[3 if smoother == "gmres" else 2:] if a.isdigit()]
    w = getattr(workloads, which)(*extra)
    suffix = "_gmres" if smoother == "gmres" else ""
    out = Path(__file__).with_name(w["name"] + suffix + ".json")
    t0 = time.time()
    H = oracle.build_hierarchy(w["n"], w["dim"], w["k2"], layers=w["layers"], smoother=smoother)
    f = w["rhs"][0]
    res = oracle.solve(H, f, tol=1e-6, max_cycles=20000)
    u = res.u
    rng = np.random.default_rng(1234)
    N = w["n"] - 1
    idx = [tuple(int(v) for v in rng.integers(0, N, size=w["dim"])) for _ in range(512)]
    src = tuple(int(v) for v in np.argwhere(f != 0)[0])
    for d in range(-3, 4):
        idx.append(tuple(min(max(s + d, 0), N - 1) for s in src))
    vals = [[float(u[i].real), float(u[i].imag)] for i in idx]
    data = dict(workload=w["name"], n=w["n"], dim=w["dim"], layers=w["layers"],
                tol=1e-6, cycles=res.cycles, rel_residual=res.history[-1],
                history_every50=res.history[::50], u_norm=float(np.linalg.norm(u)),
                u_maxabs=float(np.abs(u).max()), sample_index=idx,
                sample_value=vals, seconds=time.time() - t0,
                smoother=smoother,
                note="FP64 oracle, V(1,1) cycles (" + ("GMRES(3)" if smoother == "gmres" else
                     "weighted Jacobi 0.8") + "), CSL shifts theta_l = l (pi/6)/log2(n), "
                     "coarsest 3^dim interior, u0 = 0")
    out.write_text(json.dumps(data))
    print(out, res.cycles, res.history[-1], data["seconds"])


if __name__ == "__main__":
    main()
