"""Second-order Stokes waves in the numerical wave tank (Sec. 7.2, the table
of wave cases A, B, C): the elevation at a probe 2.87 wavelengths down the
tank against the analytic second-order surface, at three resolutions.

Run:  python -m paper_1901_07892_gb300.wave_validation [--case A] [--nx 512,1024,2048]
      [--t-end 20] [--limiter xsppm7|cui] [--precision mixed|fp64]
      [--generator inlet|zone] [--lid open|wall]

Set-up per case (depth d, height H, period T, wavelength lambda from the
dispersion relation): a 68 d x 1.3 d tank (water depth d, air above), run as
a slab four cells thick in y with free-slip y walls (every field is uniform
along y), no-slip x and z walls; one cell of interface smearing (n_cells =
1); the wave generated by the Dirichlet inlet at the left wall with an open
top (the paper's set-up, the defaults), or by a relaxation zone one
wavelength long under a closed lid (--generator zone --lid wall); damped
over the last 10 d; time step dt = 100 / (57 nx) as in Sec. 7.2.  The elevation eta = z - d - phi is
read in the probe column at the cell nearest the interface and averaged over
y.  Reported per resolution: the error in the largest elevation over the
window after the wave front has passed (the paper's measure) and the
maximum pointwise error over that window, and the convergence rates between
successive resolutions.  The paper reports rates of 1.23 and 1.17 for
case A with its own inlet, grids and limiter: context, not a target.
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

G = 9.81
# Sec. 7.2, table of wave cases: depth, H/d, T / sqrt(d/g)
CASES = {"A": (0.4, 0.05, 9.8995), "B": (0.4, 0.10, 9.8995), "C": (2.35, 0.05, 4.0825)}


def wavenumber(omega, d, tol=1e-15):
    k = omega * omega / G
    for _ in range(100):
        f = G * k * math.tanh(k * d) - omega * omega
        df = G * math.tanh(k * d) + G * k * d / math.cosh(k * d) ** 2
        dk = f / df
        k -= dk
        if abs(dk) < tol * k:
            break
    return k


def analytic_eta(x, t, H, T, d):
    """Second-order Stokes surface elevation (Sec. 7.1)."""
    w = 2 * math.pi / T
    k = wavenumber(w, d)
    lam = 2 * math.pi / k
    th = k * x - w * t
    c2 = math.pi * H * H / (8 * lam) * math.cosh(k * d) * (2 + math.cosh(2 * k * d)) / math.sinh(k * d) ** 3
    return 0.5 * H * np.cos(th) + c2 * np.cos(2 * th)


def build(case, nx, generator="inlet", lid="open"):
    d, hr, tr = CASES[case]
    H, T = hr * d, tr * math.sqrt(d / G)
    lam = 2 * math.pi / wavenumber(2 * math.pi / T, d)
    nz = nx // 8
    lx, lz = 68 * d, 1.3 * d
    hz = lz / nz
    ny = 4
    c = inputs.Case(nx=nx, ny=ny, nz=nz, lx=lx, ly=ny * hz, lz=lz, bc=(-1.0, -1.0, 1.0, 1.0, -1.0, -1.0),
                    dt=100.0 / (57.0 * nx))
    c.n_cells = 1.0
    c.rho_s = c.rho_l
    c.open_top = lid == "open"
    x, y, z = c.cell_xyz()
    c.phi = np.broadcast_to(z - d, (nz, ny, nx)).copy()
    c.psi = np.ones((nz, ny, nx))
    waves = dict(H=H, T=T, depth=d, x_gen=lam if generator == "zone" else 0.0, x_damp=lx - 10 * d,
                 inlet=generator == "inlet")
    return c, waves, dict(d=d, H=H, T=T, lam=lam, probe=2.87 * lam)


def run(case, nx, t_end, precision, limiter, generator="inlet", lid="open", every=2):
    import torch
    from paper_1901_07892_gb300 import wsi
    c, waves, p = build(case, nx, generator, lid)
    ctx = wsi.Context.from_case(c, precision=precision, restart=20, ls_limiter=limiter)
    ctx.set_case(c, with_body=False)
    ctx.set_waves(**waves)
    hz = c.lz / c.nz
    ip = int(p["probe"] / (c.lx / c.nx))
    zc = (np.arange(c.nz) + 0.5) * hz
    phi = torch.empty(c.nx * c.ny * c.nz, dtype=torch.float64, device="cuda")
    ts, etas = [], []
    nsteps = int(round(t_end / c.dt))
    iters = []
    for n in range(nsteps):
        st = ctx.step(c.dt, rtol=1e-8, max_iters=200)
        iters.append(st.iters[0] + st.iters[1])
        if (n + 1) % every == 0:
            phi = ctx.get_field(wsi.F_PHI, like=phi)
            col = phi.view(c.nz, c.ny, c.nx)[:, :, ip].cpu().numpy()   # (nz, ny)
            e = []
            for jy in range(c.ny):
                kk = int(np.argmin(np.abs(col[:, jy])))
                e.append(zc[kk] - p["d"] - col[kk, jy])
            ts.append((n + 1) * c.dt)
            etas.append(float(np.mean(e)))
    ctx.close()
    x_probe = (ip + 0.5) * c.lx / c.nx
    return np.array(ts), np.array(etas), x_probe, p, float(np.mean(iters))


def errors(ts, etas, x_probe, p, t_end):
    # the front moves at the group velocity; leave it two periods to pass
    d, T = p["d"], p["T"]
    k = 2 * math.pi / p["lam"]
    cg = 0.5 * (1 + 2 * k * d / math.sinh(2 * k * d)) * p["lam"] / T
    t0 = (x_probe - p["lam"]) / cg + 2 * T
    win = (ts >= t0) & (ts <= t_end)
    ex = analytic_eta(x_probe, ts[win], p["H"], T, d)
    return {"window": [t0, t_end], "max_elevation_error": abs(etas[win].max() - ex.max()),
            "max_pointwise_error": float(np.abs(etas[win] - ex).max()), "H": p["H"],
            "analytic_max": float(ex.max()), "numerical_max": float(etas[win].max())}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="A", choices=list(CASES))
    ap.add_argument("--nx", default="512,1024,2048")
    ap.add_argument("--t-end", type=float, default=20.0)
    ap.add_argument("--limiter", default="xsppm7", choices=["xsppm7", "cui"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--generator", default="inlet", choices=["inlet", "zone"])
    ap.add_argument("--lid", default="open", choices=["open", "wall"])
    a = ap.parse_args(argv)
    from paper_1901_07892_gb300 import wsi
    lim = wsi.LIMIT_XSPPM7 if a.limiter == "xsppm7" else wsi.LIMIT_CUI
    prec = wsi.PREC_MIXED if a.precision == "mixed" else wsi.PREC_FP64
    rows = []
    for nx in [int(v) for v in a.nx.split(",")]:
        ts, etas, xp, p, its = run(a.case, nx, a.t_end, prec, lim, a.generator, a.lid)
        r = errors(ts, etas, xp, p, a.t_end)
        r.update(nx=nx, nz=nx // 8, dt=100.0 / (57.0 * nx), mean_fgmres_iters_per_step=its)
        rows.append(r)
        print(json.dumps(r), flush=True)
    rates = []
    for r0, r1 in zip(rows, rows[1:]):
        rates.append({"grids": [r0["nx"], r1["nx"]],
                      "rate_max_elevation": math.log2(r0["max_elevation_error"] / r1["max_elevation_error"])
                      if r1["max_elevation_error"] > 0 else None,
                      "rate_pointwise": math.log2(r0["max_pointwise_error"] / r1["max_pointwise_error"])})
    print(json.dumps({"case": a.case, "limiter": a.limiter, "precision": a.precision, "generator": a.generator,
                      "lid": a.lid, "rates": rates,
                      "paper_rates_case_A_context": [1.23, 1.17]}), flush=True)


if __name__ == "__main__":
    main()
