"""Profiling entry: one step (or one rates call) of the fine-mesh drag workload.

``python -m paper_2109_08547_gb300.profile_step step --nk 80 --nq 40`` runs two untimed
steps, then one step, and writes ``<out>/step_window.txt`` with the number of kernel
launches before that step and the number inside it (the ``-s`` and ``-c`` of an ncu launch
list).  ``rates --nk 40 --nq 20`` builds the meshes once and runs one transition-rate call,
a small case for a full capture of one kernel.  Every step goes through the C-ABI library.
"""
import argparse
import dataclasses
import json
import os

from . import binding as B
from . import synthetic as S


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("mode", choices=["step", "rates"])
    p.add_argument("--nk", type=int, default=80)
    p.add_argument("--nq", type=int, default=40)
    p.add_argument("--precision", default="fp64-sliced", choices=sorted(B.PRECISIONS))
    p.add_argument("--solve", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--delta", default="gauss", choices=["gauss", "tetra"])
    p.add_argument("--warm", type=int, default=2)
    p.add_argument("--device-loop", type=int, default=1, choices=[0, 1],
                   help="1: the solve as one graph launch with device-driven loops (the bench default)")
    p.add_argument("--out", default=".", help="directory of step_window.txt")
    a = p.parse_args(argv)
    wl = S.workload_cscl8(a.nk, a.nq)
    wl = dataclasses.replace(wl, delta=a.delta)
    prec = B.PRECISIONS[a.precision]
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        if a.mode == "rates":
            B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
            r = B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, prec,
                                           delta=wl.delta)
            print(json.dumps({"rates_ms": r["ms"], "stage_a_ms": r["ms_stage_a"], "pairs": r["n_pairs"]}))
            return
        kw = dict(level="dragged", precision=prec, solve_precision=a.solve, accel=0, tol=1e-8,
                  device_loop=bool(a.device_loop))
        for _ in range(a.warm):
            B.run_path(ctx, wl, **kw)
        l0 = B.kernel_launches()
        r = B.run_path(ctx, wl, **kw)
        n = B.kernel_launches() - l0
        os.makedirs(a.out, exist_ok=True)
        with open(os.path.join(a.out, "step_window.txt"), "w") as f:
            f.write(f"{l0} {n}\n")
        print(json.dumps({"launches_before": l0, "step_launches": n, "mesh_ms": r.mesh["ms"],
                          "rates_ms": r.rates["ms"], "solve_ms": r.solve["ms"],
                          "outer": r.solve["outer_iters"]}))


if __name__ == "__main__":
    main()
