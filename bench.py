"""Throughput of the implicit Stokes time step on GB300.

One "step" is one full time step of the method (Sec. 4.2): level-set
advection, materials, SSP-RK3 consistent transport, two implicit Stokes
solves (FGMRES + projection preconditioner + pressure multigrid) to a
relative residual of 1e-8, and the DLM rigidity projection with the marker
update.  Workload (default): a 256^3 three-phase tank over the unit cube,
water depth 0.6 perturbed by 8 seeded Fourier modes (amplitude <= 0.05),
density ratio 1000:1.2, locked 0.2 x 0.2 x 0.1 box (one marker per half
cell) centred on the surface, dt = 5e-4; the surface sloshes, so every solve
iterates.  Metric: cell-steps/s = cells x steps / time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wsi|reference]
       [--precision mixed|fp64] [--n 256] [--roofline-kernel stokes|rbgs_p|...|reinit]
       [--workload tank|cylinder|wave] [--form consistent|nonconservative] [--reinit K]
--form nonconservative integrates the paper's non-conservative, inconsistent
formulation instead (Sec. 4.2.3); --reinit K reinitialises phi with K
pseudo-time steps at the end of every step (Sec. 4.1).  Both change the
workload's name in the JSON line; the defaults are the headline workload.
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method needs no exchange between replicas here): weak scaling.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1901_07892_gb300 import inputs  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# float64 FMA rate derived from the unit counts (152 SMs x 2 FP64 FMA/clk/SM x
# 2 flop x 2.07 GHz); used only when the measurement (wsi_fma_peak) fails
FP64_PEAK_DERIVED_GFLOPS = 152 * 2 * 2 * 2.07
# DRAM bytes per cell of one launch, measured with ncu at 128^3 (dram__bytes_read.sum +
# dram__bytes_write.sum, profiles/k_stokes_df_tank128.md) for the current kernel revision;
# scaled by the cells of the workload (empty while no capture of the current revision exists)
TRAFFIC_PER_CELL = {("stokes", "mixed"): (200.392192e6 + 46.134528e6) / 128 ** 3}
KCLASS = {"stokes": 0, "rbgs_p": 1, "rbgs_v": 2, "transport": 3, "mdot": 4, "maxpy": 5, "restrict": 6,
          "prolong": 7, "reinit": 8}


def kernel_model(name, nx, ny, nz, prec_bytes):
    """Algorithmic bytes and flops per launch of a kernel class (each array
    touched once; coefficient arrays included)."""
    N = nx * ny * nz
    F = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)
    E = (nx + 1) * (ny + 1) * nz + (nx + 1) * ny * (nz + 1) + nx * (ny + 1) * (nz + 1)
    if name == "stokes":
        # read u,v,w,p, rho_face, mu_cc, mu_edges; write 4 outputs: 8 bytes each
        # (float64, or the (hi, lo) float32 pairs of the double-float matvec)
        byts = 8 * (F + N + F + N + E + F + N)
        flops = 44 * F + 8 * N
        # float64 arithmetic is bound by the float64 pipe; the double-float
        # matvec of the mixed path is reported against HBM
        return byts, flops, ("alu" if prec_bytes == 8 else "hbm")
    if name == "rbgs_p":
        # one colour: read x (all), b (half), 3 beta face arrays; write x (half)
        byts = prec_bytes * (N + N // 2 + F + N // 2)
        return byts, 14 * N // 2, "hbm"
    if name == "rbgs_v":
        byts = prec_bytes * (F + F // 2 + F + N + E + F // 2)
        return byts, 50 * F // 2, "hbm"
    if name == "transport":
        # launches differ (density only, or with the velocity): the library
        # sums each launch's algorithmic bytes (wsi_ktimer_bytes): per
        # component the transported density, the three velocity arrays of the
        # advective velocities, the transported velocity (convective term)
        # and the result, in the storage type
        return None, None, "hbm"
    if name in ("mdot", "maxpy"):
        # launches differ in the number of basis vectors: the library sums
        # each launch's algorithmic bytes (wsi_ktimer_bytes)
        return None, None, "hbm"
    if name == "reinit":
        # first stage: read phi and the one-byte sign/crossing code, write
        # phi*; second stage: also read phi^m (phi~ itself is read only next
        # to the interface); the average of the two per launch
        return (5 * prec_bytes + 2) * N // 2, 90 * N, "hbm"
    raise ValueError(name)


def sample_clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                              "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def sample_clocks_stop(h, path, gpu_index):
    p, f = h
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
            "samples": len(sm)}


def build_case(n, workload="tank"):
    """tank: n^3 sloshing tank with a locked box (rho_s = densest fluid,
    gravity from rho^flow, Sec. 5).  cylinder: the largest configuration's
    wave tank, (2n) x n x n cells over 8 x 2 x 2 m, water depth 1 m, a
    free-floating cylinder (radius 0.15 m, length 1.6 m, rho_s = 500, free in
    surge, heave and pitch) under a regular wave (H 0.1 m, T 1.2 s) generated
    over x in [0, 1] and damped over [7, 8]."""
    if workload == "wave":
        # the wave tank: (n) x (n/2) x (n/2) cells over 4 x 1 x 1 m, depth 0.5 m,
        # second-order Stokes wave H 0.05 m, T 1 s, locked trapezoidal bar
        c = inputs.wave_tank(nx=n, ny=n // 2, nz=n // 2, dt=0.01)
        c.extra["waves"] = dict(c.extra["wave"])
        return c
    if workload == "cylinder":
        c = inputs.tank_cylinder(nxyz=(2 * n, n, n), lxyz=(8.0, 2.0, 2.0), depth=1.0, radius=0.15, length=1.6,
                                 dt=2.5e-3)
        c.extra["waves"] = dict(H=0.1, T=1.2, depth=1.0, x_gen=1.0, x_damp=7.0)
        return c
    c = inputs.tank3d(n=n, seed=7, dt=5e-4)
    c.rho_s = c.rho_l  # locked body: rho_s = densest fluid, gravity from rho^flow (Sec. 5)
    return c


def workload_name(args):
    name = _base_workload_name(args)
    if getattr(args, "form", "consistent") == "nonconservative":
        name += ", non-conservative momentum form"
    return name + (", phi reinitialised (%d pseudo-time steps)" % args.reinit if args.reinit else "")


def _base_workload_name(args):
    if args.workload == "wave":
        return ("wave%d: %dx%dx%d wave tank 4x1x1 m, second-order Stokes wave H 0.05 m T 1 s, locked trapezoidal "
                "bar, 2 Stokes solves per step to rtol %.0e" % (args.n, args.n, args.n // 2, args.n // 2, args.rtol))
    if args.workload == "cylinder":
        return ("cylinder%d: %dx%dx%d wave tank 8x2x2 m, regular wave H 0.1 m T 1.2 s, free-floating cylinder "
                "(r 0.15 m, L 1.6 m, rho_s 500), 2 Stokes solves per step to rtol %.0e"
                % (args.n, 2 * args.n, args.n, args.n, args.rtol))
    return ("tank%d: %d^3 three-phase tank, 8-mode seeded surface, locked box, 2 Stokes solves per step to rtol %.0e"
            % (args.n, args.n, args.rtol))


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the whole job takes as long as its
    slowest replica); x itself when not distributed."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, cells, steps, seconds):
    """Whole-job cell-steps/s: every replica advances its own grid."""
    return world * cells * steps / seconds


def learned_comparison(args, stream):
    """Pressure solves D(beta G) x = y to 1e-8 at args.n^3 (the projection
    sub-problem): learned initial guess + float32 V-cycles vs plain float32
    V-cycles vs plain float64 V-cycles, all with float64 residuals.  The
    guess network (16/32/64 channels) works on a 32^3 multigrid level: level
    2 of the (n/2)^3 training tanks, level 3 of the n^3 evaluation tanks.  It
    is trained on the GPU on pairs the plain solver generates: a seeded random
    right-hand side y on a training tank and its solution x from the plain
    float32 cycles (to 1e-8).  Evaluation tanks use unseen seeds; y is a
    seeded random cell field with its mean removed."""
    import torch
    from paper_1901_07892_gb300 import wsi
    n_tr = args.n // 2
    lg_tr, lg_ev = 2, 3
    nc = n_tr >> lg_tr
    net = wsi.UNet(nc, nc, nc, 16, 32, 64, seed=11)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    tanks = 4
    per = max(1, args.learned_train // tanks)
    losses = []
    t0 = time.perf_counter()
    for s in range(tanks):
        c = inputs.tank3d(n=n_tr, seed=100 + s, with_body=False)
        plain = wsi.Context.from_case(c, precision=wsi.PREC_MIXED, stream=stream.cuda_stream)
        plain.set_case(c, with_body=False)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED, stream=stream.cuda_stream)
        ctx.set_case(c, with_body=False)
        wsi.attach_unet_guess(ctx, net, lg_tr)
        for k in range(per):
            y = torch.rand(ctx.ncell, dtype=torch.float64, device="cuda", generator=gen) * 2.0 - 1.0
            y -= y.mean()
            x, _ = wsi.pressure_solve(plain, y, rtol=1e-8, max_cycles=100)
            losses.append(wsi.unet_train_guess(ctx, y, x, 1e-3 if k < 0.7 * per else 3e-4))
        plain.close()
        ctx.close()
    train_s = time.perf_counter() - t0
    rows = []
    for s in (10 ** 6, 10 ** 6 + 1):
        c = inputs.tank3d(n=args.n, seed=s, with_body=False)
        y = torch.from_numpy(inputs.random_cells(c.phi.shape, s).ravel()).cuda()
        y -= y.mean()
        row = {"seed": s}
        for name, prec, guess in (("learned_fp32", wsi.PREC_MIXED, True), ("plain_fp32", wsi.PREC_MIXED, False),
                                  ("plain_fp64", wsi.PREC_FP64, False)):
            ctx = wsi.Context.from_case(c, precision=prec, stream=stream.cuda_stream)
            ctx.set_case(c, with_body=False)
            if guess:
                wsi.attach_unet_guess(ctx, net, lg_ev)
            wsi.pressure_solve(ctx, y.clone(), rtol=args.rtol, max_cycles=200)  # warm-up (set-up, caches)
            x, st = wsi.pressure_solve(ctx, y.clone(), rtol=args.rtol, max_cycles=200)
            row[name] = {"ms": st.ms, "cycles": st.iters, "rel_residual": st.rel_residual,
                         "guess_kept": st.guess}
            ctx.close()
        rows.append(row)
    net.close()
    mean = lambda k: float(np.mean([r[k]["ms"] for r in rows]))
    return {"what": "pressure solve to rtol %.0e at %d^3 (float64 residuals), time to tolerance; learned: initial "
                    "guess from the network on the 32^3 level" % (args.rtol, args.n),
            "train": {"pairs": len(losses), "seconds": train_s, "tank": "%d^3" % n_tr,
                      "loss_first50": float(np.mean(losses[:50])), "loss_last50": float(np.mean(losses[-50:]))},
            "solves": rows, "ms_learned_fp32": mean("learned_fp32"), "ms_plain_fp32": mean("plain_fp32"),
            "ms_plain_fp64": mean("plain_fp64"),
            "speedup_learned_fp32_over_plain_fp64": mean("plain_fp64") / mean("learned_fp32"),
            "speedup_learned_fp32_over_plain_fp32": mean("plain_fp32") / mean("learned_fp32")}


def oracle_sample_step(n_sample=12, workload="tank", reinit_iters=0, form="consistent"):
    """One oracle step of the same recipe at a small size (host cores):
    n_sample^3 for the tank, (2 n_sample) x n_sample x n_sample for the
    cylinder tank, n_sample x n_sample/2 x n_sample/2 for the wave tank (the
    last two without the wave zones)."""
    from oracle.grid import Grid
    from oracle import step as ost
    c = build_case(n_sample, workload)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    if workload == "cylinder":
        pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_s, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                       gravity_mode="full")
        body = ost.Body(c.markers, c.dV, list(c.lock), cylinder=c.extra["cylinder"])
    elif workload == "wave":
        pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_s, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                       gravity_mode="flow")
        body = ost.Body(c.markers, c.dV, [True] * 6)
    else:
        pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_s, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                       gravity_mode="flow")
        body = ost.Body(c.markers, c.dV, [True] * 6, half=c.box_half)
    s = ost.State(g, pr, c.phi, c.psi, body)
    t0 = time.perf_counter()
    ost.step(s, c.dt, reinit_iters=reinit_iters, form=form)
    dt = time.perf_counter() - t0
    return g.n_cells, dt


def other_configs(args, stream):
    """The other configurations of the workload list, timed the same way
    (CUDA events on the library's stream after 3 warm-up steps), each from
    a fresh context: the 128^3 hydrostatic tank (50 steps, solves/s and the
    spurious velocity left), the 256x128x128 wave tank (200 steps mixed, 20
    plain float64) and the largest, 512x256x256 wave tank with the free
    cylinder (10 steps mixed, 5 plain float64: a sample of its 500)."""
    import torch
    from paper_1901_07892_gb300 import wsi

    def run(c, prec, steps, waves=None, rho_s=None):
        ctx = wsi.Context.from_case(c, precision=prec, restart=20, stream=stream.cuda_stream)
        if rho_s is not None:
            ctx.set_case(c, rho_s=rho_s)
        else:
            ctx.set_case(c)
        if waves:
            ctx.set_waves(**waves)
        for _ in range(3):
            ctx.step(c.dt, rtol=args.rtol, max_iters=200)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        its = []
        for _ in range(steps):
            st = ctx.step(c.dt, rtol=args.rtol, max_iters=200)
            its.append([st.iters[0], st.iters[1]])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        cells = c.nx * c.ny * c.nz
        out = {"steps": steps, "ms_per_step": ms / steps, "cell_steps_per_s": cells * steps / (ms * 1e-3),
               "solves_per_s": 2 * steps / (ms * 1e-3), "fgmres_iters": its, "umax": st.umax}
        ctx.close()
        return out

    res = {}
    c = inputs.tank3d(n=128, seed=None, dt=5e-4)
    res["hydrostatic128"] = {"what": "128^3 tank, flat surface z = 0.6, locked 0.2x0.2x0.1 box, rho^flow g, "
                                     "u0 = 0, dt 5e-4, rtol %.0e" % args.rtol,
                             "mixed": run(c, wsi.PREC_MIXED, 50, rho_s=c.rho_l),
                             "plain_fp64": run(c, wsi.PREC_FP64, 50, rho_s=c.rho_l)}
    c = build_case(256, "wave")
    w = c.extra["waves"]
    res["wave256x128x128"] = {"what": "wave tank 4x1x1 m, depth 0.5, Stokes wave H 0.05 T 1, locked bar, dt 0.01",
                              "mixed": run(c, wsi.PREC_MIXED, 200, waves=w),
                              "plain_fp64": run(c, wsi.PREC_FP64, 20, waves=w)}
    c = build_case(256, "cylinder")
    w = c.extra["waves"]
    res["cylinder512x256x256"] = {"what": "wave tank 8x2x2 m, depth 1, regular wave H 0.1 T 1.2, free cylinder "
                                          "r 0.15 L 1.6 rho_s 500, dt 2.5e-3 (a 10-step sample of 500)",
                                  "mixed": run(c, wsi.PREC_MIXED, 10, waves=w),
                                  "plain_fp64": run(c, wsi.PREC_FP64, 5, waves=w)}
    for v in res.values():
        v["speedup_mixed_over_fp64"] = v["plain_fp64"]["ms_per_step"] / v["mixed"]["ms_per_step"]
    return res


def oracle_matvec_rate(c):
    """The oracle's Stokes matvec on the full-size workload (materials
    excluded), single-threaded numpy: cell-applies/s, beside the GPU's
    dominant kernel on the same grid."""
    from oracle.grid import Grid
    from oracle.materials import Materials
    from oracle import operators as ops
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    m = Materials(g, c.phi, c.psi, c.rho_l, c.rho_g, c.rho_s, c.mu_l, c.mu_g, c.mu_s, c.n_cells)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(sum(g.n_faces(d) for d in range(3)) + g.n_cells)
    t0 = time.perf_counter()
    ops.stokes_apply(g, m, m.rho_face, c.dt, c.theta, x)
    dt = time.perf_counter() - t0
    return {"value": g.n_cells / dt, "unit": "cell-applies/s", "cores": 1, "seconds": dt,
            "sample": "one oracle Stokes matvec at %dx%dx%d (float64 numpy)" % (c.nx, c.ny, c.nz)}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_sample = {"tank": 12, "cylinder": 8, "wave": 16}[args.workload]
    times = []
    cells = 0
    for i in range(args.warmup + args.steps):
        cells, dt = oracle_sample_step(n_sample, args.workload, args.reinit, args.form)
        if i >= args.warmup:
            times.append(dt)
    T = float(np.sum(times))
    value = cells * len(times) / T
    sample = "one oracle step (materials, transport, exact sparse-LU Stokes solves, DLM) of the same %s " \
             "recipe at %s per step; numpy/scipy, single-threaded" % (
                 args.workload, {"tank": "%d^3" % n_sample, "cylinder": "%dx%dx%d" % (2 * n_sample, n_sample, n_sample),
                                 "wave": "%dx%dx%d" % (n_sample, n_sample // 2, n_sample // 2)}[args.workload])
    line = {"impl": "reference", "metric": "cell-steps/s", "value": value, "unit": "cell-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args), "sample": sample},
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wsi", choices=["wsi", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--roofline-kernel", default="stokes", choices=list(KCLASS))
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned pressure-solve comparison")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (hydrostatic 128^3, wave tank, largest cylinder tank)")
    ap.add_argument("--visc-sweeps", type=int, default=2, help="viscous red-black sweeps per preconditioner apply")
    ap.add_argument("--form", default="consistent", choices=["consistent", "nonconservative"],
                    help="momentum formulation: consistent mass/momentum transport (default) or the "
                         "non-conservative one with the level-set density")
    ap.add_argument("--reinit", type=int, default=0,
                    help="pseudo-time steps of the level-set reinitialisation at the end of every step")
    ap.add_argument("--mg", default="2,2", help="pressure V-cycle pre,post smoothing sweeps (or degrees)")
    ap.add_argument("--smoother", default="rbgs", choices=["rbgs", "chebyshev"],
                    help="pressure multigrid smoother")
    ap.add_argument("--learned-train", type=int, default=1200, help="training samples for the learned comparison")
    ap.add_argument("--workload", default="tank", choices=["tank", "cylinder", "wave"],
                    help="tank: n^3 sloshing tank (default); cylinder: (2n) x n x n wave tank with a free cylinder; "
                         "wave: n x n/2 x n/2 wave tank with a submerged bar")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_1901_07892_gb300 import wsi
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    c = build_case(args.n, args.workload)
    cells = c.nx * c.ny * c.nz
    prec = wsi.PREC_MIXED if args.precision == "mixed" else wsi.PREC_FP64

    def make_ctx(p):
        pre, post = (int(v) for v in args.mg.split(","))
        ctx = wsi.Context.from_case(c, precision=p, restart=20, stream=stream.cuda_stream, mg_pre=pre, mg_post=post,
                                    visc_sweeps=args.visc_sweeps, reinit_iters=args.reinit,
                                    mg_smoother=(wsi.SMOOTH_CHEBYSHEV if args.smoother == "chebyshev"
                                                 else wsi.SMOOTH_RBGS),
                                    transport_form=(wsi.FORM_NONCONSERVATIVE if args.form == "nonconservative"
                                                    else wsi.FORM_CONSISTENT))
        if args.workload in ("cylinder", "wave"):
            ctx.set_case(c)
            ctx.set_waves(**c.extra["waves"])
        else:
            ctx.set_case(c, rho_s=c.rho_l)
        return ctx

    def timed_steps(ctx, k):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        its = []
        for _ in range(k):
            st = ctx.step(c.dt, rtol=args.rtol, max_iters=200)
            its.append([st.iters[0], st.iters[1]])
        ev1.record(stream)
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        return ms, its

    # measured float64 FMA rate of this GPU (denominator of the "alu" roofline)
    try:
        fp64_peak, fp64_peak_note = wsi.fma_peak(True, stream.cuda_stream), "measured (wsi_fma_peak)"
    except Exception as e:  # noqa: BLE001
        fp64_peak, fp64_peak_note = FP64_PEAK_DERIVED_GFLOPS, "derived: 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz (%s)" % e

    ctx = make_ctx(prec)
    for _ in range(args.warmup):
        ctx.step(c.dt, rtol=args.rtol, max_iters=200)
    clk_path = os.path.join(tempfile.gettempdir(), "wsi_clocks_%d_rank%d.csv" % (os.getpid(), rank))
    clk = sample_clocks_start(clk_path)
    kname = args.roofline_kernel
    wsi.ktimer_enable(KCLASS[kname])
    l0 = wsi.launch_count()
    ms, its = timed_steps(ctx, args.steps)
    l1 = wsi.launch_count()
    kt_ms, kt_n = wsi.ktimer_read()
    kt_bytes = wsi.ktimer_bytes()
    wsi.ktimer_enable(-1)
    clocks = sample_clocks_stop(clk, clk_path, torch.cuda.current_device())
    value = job_throughput(world, cells, args.steps, ms * 1e-3)

    # roofline of the chosen kernel: algorithmic work per launch / measured duration
    pb = 4 if prec == wsi.PREC_MIXED else 8
    byts, flops, bound = kernel_model(kname, c.nx, c.ny, c.nz, pb)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    roof = None
    if byts is None and kt_n > 0:
        byts = kt_bytes / kt_n  # average algorithmic bytes per launch
    if kt_n > 0:
        dur = kt_ms / kt_n * 1e-3
        if bound == "alu":
            roof = {"bound": "alu", "achieved": flops / dur / 1e12, "peak": fp64_peak / 1e3,
                    "unit": "TFLOP/s", "frac": flops / dur / 1e9 / fp64_peak,
                    "traffic": None, "kernel": kname, "launches": kt_n, "avg_us": dur * 1e6,
                    "algorithmic_bytes_per_launch": byts, "flops_per_launch": flops,
                    "peak_note": "float64 FMA rate " + fp64_peak_note}
        else:
            hb = peaks.get("hbm_gbs", 6800.0)
            tpc = TRAFFIC_PER_CELL.get((kname, args.precision))
            roof = {"bound": "hbm", "achieved": byts / dur / 1e9, "peak": hb, "unit": "GB/s",
                    "frac": byts / dur / 1e9 / hb, "traffic": tpc * cells if tpc else None, "kernel": kname,
                    "launches": kt_n,
                    "avg_us": dur * 1e6, "algorithmic_bytes_per_launch": byts,
                    "peak_note": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}

    # end to end through the C ABI with host buffers: upload the state from
    # pinned host memory, step, read the new velocity and pressure back
    hv = torch.empty(ctx.nvel, dtype=torch.float64).pin_memory()
    hvo = torch.empty(ctx.nvel, dtype=torch.float64).pin_memory()
    hphi = torch.empty(ctx.ncell, dtype=torch.float64).pin_memory()
    hpsi = torch.empty(ctx.ncell, dtype=torch.float64).pin_memory()
    hp = torch.empty(ctx.ncell, dtype=torch.float64).pin_memory()
    for arr, f in ((hv, wsi.F_VEL), (hvo, wsi.F_VEL_OLD), (hphi, wsi.F_PHI), (hpsi, wsi.F_PSI)):
        ctx.L.wsi_get_field(ctx._h, f, wsi._ptr(arr))
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for arr, f in ((hv, wsi.F_VEL), (hvo, wsi.F_VEL_OLD), (hphi, wsi.F_PHI), (hpsi, wsi.F_PSI)):
            ctx.L.wsi_set_field(ctx._h, f, wsi._ptr(arr))
        ctx.step(c.dt, rtol=args.rtol, max_iters=200)
        ctx.L.wsi_get_field(ctx._h, wsi.F_VEL, wsi._ptr(hv))
        ctx.L.wsi_get_field(ctx._h, wsi.F_P, wsi._ptr(hp))
        ctx.L.wsi_get_field(ctx._h, wsi.F_VEL_OLD, wsi._ptr(hvo))
        ctx.L.wsi_get_field(ctx._h, wsi.F_PHI, wsi._ptr(hphi))
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    h2d = 8 * (2 * ctx.nvel + 2 * ctx.ncell)
    d2h = 8 * (2 * ctx.nvel + 2 * ctx.ncell)
    e2e = {"value": job_throughput(world, cells, args.steps, e2e_s), "unit": "cell-steps/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}
    ctx.close()

    compare = None
    if not args.no_compare and prec == wsi.PREC_MIXED:
        ctx64 = make_ctx(wsi.PREC_FP64)
        for _ in range(args.warmup):
            ctx64.step(c.dt, rtol=args.rtol, max_iters=200)
        ms64, its64 = timed_steps(ctx64, args.steps)
        compare = {"plain_fp64": {"value": world * cells * args.steps / (ms64 * 1e-3), "unit": "cell-steps/s",
                                  "ms_per_step": ms64 / args.steps, "fgmres_iters": its64},
                   "speedup_mixed_over_fp64": ms64 / ms}
        ctx64.close()

    configs = None
    if not args.no_configs and rank == 0 and args.workload == "tank" and args.n == 256:
        configs = other_configs(args, stream)

    learned = None
    if not args.no_learned and rank == 0 and args.workload == "tank":
        learned = learned_comparison(args, stream)

    cpu = None
    if rank == 0 and not args.no_cpu:
        n_s, t_s = oracle_sample_step({"tank": 12, "cylinder": 8, "wave": 16}[args.workload], args.workload,
                                      args.reinit, args.form)
        cpu = {"value": n_s / t_s, "unit": "cell-steps/s", "cores": 1, "host_cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "one oracle time step (exact sparse-LU solves) of the same %s recipe at %s; "
                         "numpy/scipy single-threaded on the GPU host"
                         % (args.workload, {"tank": "12^3", "cylinder": "16x8x8 without wave zones",
                                            "wave": "16x8x8 without wave zones"}[args.workload])}
        if args.workload == "tank" and args.roofline_kernel == "stokes":
            cpu["full_size_matvec"] = oracle_matvec_rate(c)
    if rank == 0:
        line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "solves_per_s": world * 2 * args.steps / (ms * 1e-3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 outer / f32 preconditioner" if prec == wsi.PREC_MIXED else "f64",
                "data": "synthetic",
                "config": {"workload": workload_name(args),
                           "cells": cells, "precision": args.precision, "l2": "inputs larger than L2 (no flush)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "mg_pre_post": args.mg, "mg_smoother": args.smoother, "visc_sweeps": args.visc_sweeps,
                           "fgmres_iters": its, "reinit_iters": args.reinit, "form": args.form},
                "gpu_launches": int(l1 - l0), "roofline": roof, "fp64_fma_peak_tflops": fp64_peak / 1e3, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "compare": compare, "configs": configs, "learned": learned}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
