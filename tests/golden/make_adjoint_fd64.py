"""Writes tests/golden/adjoint_pack128_T2000_fd64.txt with the FP64 oracle
only: central finite differences of the smooth saturation J = mean over
fluid nodes of (1 - phi)/2 after T = 2000 steps of the gradient workload
(workloads.adjoint_pack(): 128^3 periodic sphere pack, porosity 0.25,
Scheme-II theta = 40 deg (Eqs. 32-33), body force g_x = 5e-6 (Eq. 36)),
with respect to theta (per degree; h = 0.5 and 1 deg) and g_x (h = 5, 10
and 20 % of g_x). These are the finite differences the hand-written
adjoint is compared with; their spread over h shows how far they have
converged.

Run from the repository root:  python tests/golden/make_adjoint_fd64.py
(11 forward runs of 2000 steps over 0.52 M fluid nodes; about 10 minutes
per run on 8 cores)."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2407_10914_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                   "adjoint_pack128_T2000_fd64.txt")
T = 2000
H_THETA = (0.5, 1.0)
H_GX = (0.05, 0.1, 0.2)


def main():
    O.build()
    case = W.adjoint_pack(steps=T)

    def J(**over):
        p = dict(case.params)
        p.update(over)
        o = O.Oracle(case.lattice, case.solid, case.periodic)
        o.set_params(**p)
        o.init_state(case.phi0)
        o.step(T)
        return o.reduce(O.SW_SMOOTH)

    t0 = time.time()
    th0, g0 = case.params["theta_deg"], case.params["g"][0]
    lines = ["# FP64 oracle, workloads.adjoint_pack() (128^3 pack, Scheme-II "
             "theta 40, g_x 5e-6), J = smooth S_w after 2000 steps.",
             "# quantity h value"]
    lines.append(f"J 0 {J():.17e}")
    for h in H_THETA:
        d = (J(theta_deg=th0 + h) - J(theta_deg=th0 - h)) / (2 * h)
        lines.append(f"dJ_dtheta_per_deg {h} {d:.17e}")
    for f in H_GX:
        hg = f * g0
        d = (J(g=(g0 + hg, 0.0, 0.0)) - J(g=(g0 - hg, 0.0, 0.0))) / (2 * hg)
        lines.append(f"dJ_dgx {f} {d:.17e}")
    lines.append(f"# {time.time() - t0:.0f} s on {O.max_threads()} threads")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
