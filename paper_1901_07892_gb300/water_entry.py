"""Water entry of a horizontal cylinder (Sec. 8.5): the stability contrast
between the consistent mass/momentum transport (Sec. 4.2.2) and the
non-conservative, inconsistent formulation (Sec. 4.2.3), and the slamming
coefficient C_s = F.e_z / (rho_l R V^2) per unit length (Sec. 8.5's C_s
equation) against the penetration depth P_d = V (t - t_impact) / R.

Run:  python -m paper_1901_07892_gb300.water_entry [--form both|consistent|nonconservative]
      [--cells-per-radius 22] [--pd-end 1.0] [--precision mixed|fp64]

Set-up (Sec. 8.5): radius R = 0.055, a tank about 40 R x 24 R with water in
the lower half, the cylinder's centre at (20 R, 14 R), i.e. 2 R above the
still water, so that its bottom touches the surface at t_impact = R / V;
density rho_s = rho_l, every degree of
freedom locked and the body driven down at V = 1, gravity from rho^flow
(Sec. 5), n_cells = 2, no-slip walls, dt = 0.02 h.  Run as a slab four cells
thick along the cylinder's axis with free-slip walls there (every field is
uniform along y), on one uniform grid of the paper's finest spacing
(22 cells per radius; the paper uses two AMR levels): the extents are rounded
to 896 x 512 cells at h = 1/400 so that the multigrid coarsens.
Reported per formulation: whether the run stayed finite, max |u| / V over
the run (a stable entry stays of order one), and C_s at a few penetration
depths.
"""
import argparse
import json
import math
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from paper_1901_07892_gb300 import inputs  # noqa: E402

R, V = 0.055, 1.0


def build(cells_per_radius):
    h = R / cells_per_radius
    nx = int(round(40 * R / h / 64)) * 64
    nz = int(round(24 * R / h / 64)) * 64
    ny = 4
    lx, lz = nx * h, nz * h
    depth = 0.5 * lz
    c = inputs.Case(nx=nx, ny=ny, nz=nz, lx=lx, ly=ny * h, lz=lz, bc=(-1.0, -1.0, 1.0, 1.0, -1.0, -1.0),
                    dt=0.02 * h, gravity_mode="flow", rho_s=1000.0)
    x, y, z = c.cell_xyz()
    c.phi = np.broadcast_to(z - depth, (nz, ny, nx)).copy()
    center = (0.5 * lx, 0.5 * c.ly, depth + 2.0 * R)
    half = 0.5 * c.ly
    c.psi = np.broadcast_to(inputs.cylinder_distance((x, y, z), center, R, half), (nz, ny, nx)).copy()
    c.markers, c.dV = inputs.cylinder_lattice(center, R, half, c.h)
    c.lock = (True,) * 6
    c.extra["cylinder"] = (R, half)
    return c, depth


def run(form, cells_per_radius, pd_end, precision, every=20):
    from paper_1901_07892_gb300 import wsi
    c, depth = build(cells_per_radius)
    tf = wsi.FORM_CONSISTENT if form == "consistent" else wsi.FORM_NONCONSERVATIVE
    ctx = wsi.Context.from_case(c, precision=precision, restart=30, transport_form=tf)
    ctx.set_case(c, U_pres=(0.0, 0.0, -V))
    t_impact = R / V
    nsteps = int(math.ceil((t_impact + pd_end * R / V) / c.dt))
    L = c.ly
    rows, umax_max, finite = [], 0.0, True
    for n in range(nsteps):
        try:
            st = ctx.step(c.dt, rtol=1e-8, max_iters=300)
        except wsi.WsiError as e:
            finite = False
            rows.append({"step": n + 1, "error": str(e)})
            break
        t = (n + 1) * c.dt
        umax_max = max(umax_max, st.umax)
        if not (math.isfinite(st.umax) and st.umax < 1e3 * V):
            finite = False
            rows.append({"step": n + 1, "umax": st.umax})
            break
        if (n + 1) % every == 0 or n + 1 == nsteps:
            rows.append({"t": t, "Pd": V * (t - t_impact) / R, "Cs": st.F_lm[2] / (c.rho_l * R * V * V * L),
                         "umax_over_V": st.umax / V, "fgmres": list(st.iters[:2])})
    ctx.close()
    return {"form": form, "grid": [c.nx, c.ny, c.nz], "h": c.lx / c.nx, "dt": c.dt, "steps_run": n + 1,
            "stayed_finite": finite, "max_umax_over_V": umax_max / V, "samples": rows}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--form", default="both", choices=["both", "consistent", "nonconservative"])
    ap.add_argument("--cells-per-radius", type=float, default=22.0)
    ap.add_argument("--pd-end", type=float, default=1.0)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    a = ap.parse_args(argv)
    from paper_1901_07892_gb300 import wsi
    prec = wsi.PREC_MIXED if a.precision == "mixed" else wsi.PREC_FP64
    forms = ["consistent", "nonconservative"] if a.form == "both" else [a.form]
    for f in forms:
        r = run(f, a.cells_per_radius, a.pd_end, prec)
        keep = [s for s in r["samples"] if "Pd" in s and s["Pd"] >= 0.0]
        print(json.dumps({k: v for k, v in r.items() if k != "samples"}), flush=True)
        for s in keep[:: max(1, len(keep) // 12)] + (r["samples"][-1:] if not r["stayed_finite"] else []):
            print("  " + json.dumps(s), flush=True)


if __name__ == "__main__":
    main()
