#!/usr/bin/env python
"""Throughput of the PolyPIC transfer step on one GB300.

Workload: the fluid dam break on a 128^3 grid (the 64 x 128 x 64-cell corner
block inside the 2-cell wall margin, 62 x 124 x 62 cells at 8 particles per
cell: 3,813,248 particles), 27
modes per velocity component, FP32 coefficients, dt = 5e-4, gravity -9.81,
zero initial velocity.  A step is one pass of the whole transfer path through
the C ABI: stable cell sort, P2G, grid update, G2P with advection; the
particle state ping-pongs between two buffers (G2P writes it in sorted order).

Printed (rank 0, one JSON line): whole-job M particle-steps/s over the timed
steps, the per-phase split, the roofline of the dominant call, the variants
(APIC = 4-mode truncation, BF16 and FP16 per-particle-scaled coefficients),
an end-to-end figure with host buffers, the clocks seen while timing, and the
FP64 CPU oracle timed on a bounded sample on the host.

--impl reference times that oracle alone (the only reference available: the
paper's own code is a CPU simulator that is not available here).
--gpus N (under torchrun) runs N independent replicas, one per GPU: the
transfers are not sharded, so no collective is involved.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PolyPIC P2G+G2P M particle-steps/s vs plain FP32 form; % HBM roofline"
UNIT = "M particle-steps/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128, help="grid cells per axis (default 128)")
    ap.add_argument("--preroll", type=int, default=200,
                    help="dam-break steps with pressure projection run (untimed) before the "
                         "timed steps, so that they start from the sustained state")
    ap.add_argument("--variants",
                    default="graph,fused,apic4,apic4_gradw,apic4_affine,affine27,bf16,f16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--e2e-lanes", type=int, default=3,
                    help="streams (each with its own device buffers) the e2e steps rotate over")
    ap.add_argument("--large-steps", type=int, default=100,
                    help="steps of the 256^3 fluid + fabric row per coefficient format")
    ap.add_argument("--rows", default="coupled,fabric,update,projection,adjoint,large",
                    help="the other rows of the path, each timed on its own workload")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(torch, ms_local: float, units_per_rank: int, steps: int, world: int,
                   device) -> tuple:
    """Whole-job throughput of N independent replicas: the slowest rank's time
    (max over ranks, an all_reduce on the process group when world > 1) and
    the units all ranks processed per second over it, in millions."""
    ms = ms_local
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world * steps / (ms * 1e-3) / 1e6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- workload

# DRAM bytes (read + write) per particle of one k_p2g_tiles<27, FP32> launch,
# from a full ncu capture on the 96^3 dam break (1,557,376 particles: 537.2 MB
# read, 13.8 MB written); P2G traffic grows in proportion to the particles, so
# it scales to the 128^3 launch.  It must go back to None whenever the kernel
# changes after that capture.
P2G_TILES_DRAM_BYTES_PER_PARTICLE = (537.27232e6 + 13.886464e6) / 1557376


def block_cells(n: int):
    """Cells per axis of the dam break's seeded block: [0, n/2) x [0, n) x
    [0, n/2) clipped to the 2-cell margin at every wall."""
    half = min(n // 2, n - 2) - 2
    return (half, n - 4, half)


def workload_name(n: int, P: int, preroll: int) -> str:
    """The `config.workload` text of the headline line."""
    d = "x".join(str(c) for c in block_cells(n))
    return (f"dam_break_{n}^3: the {n // 2}x{n}x{n // 2}-cell corner block inside the 2-cell "
            f"wall margin ({d} cells), 8 particles/cell ({P} particles), 27 modes, FP32 "
            f"coefficients, dt 5e-4, timed after {preroll} steps with pressure projection")


def algorithmic_bytes(R: int, fmt: str):
    """Per particle-step bytes of the P2G and G2P calls.  P2G reads x, m and
    c; G2P reads x and writes x and c; the grid term (P2G writes of m and mv,
    G2P reads of v~ on 3 face grids: 36 B per cell at 8 particles per cell) is
    split 24/12 between them."""
    cbytes = 12 * R if fmt == "f32" else 6 * R + 4
    p2g = 16 + cbytes + 24 / 8
    g2p = 24 + cbytes + 12 / 8
    return p2g, g2p


def launches_per_step() -> int:
    """Kernels of ours per polypic_step (one phase, no projection): keys with
    arrival ranks, the 3-kernel count scan, the scatter, the per-cell order,
    the crowded-cell pass (exits at once when no cell holds more than 64
    particles), P2G tiles + the tile reduction with the grid update fused in,
    G2P."""
    return 1 + 3 + 1 + 1 + 1 + 2 + 1


def make_state(pp, ctx, scene, device):
    f = scene.fluid
    a = pp.upload_particles(ctx, f.x, f.mass, None, device=device)
    b = ctx.new_particles(a.count, device=device)
    return a, b


# FP32 FMAs of the sum-factorised contractions per particle-step at 27 modes:
# P2G 81 + 81 + 108 per component (the padded 4 x 3 x 3 footprint), G2P's fit
# 729 (27 modes x 3 components x 3 stages of 3); stencil weights, decisions
# and addressing are not counted.
FMA_PER_PARTICLE_STEP_27 = 3 * (81 + 81 + 108) + 729


def alu_ceiling(torch, device, P, ph, clocks):
    """The plain-ALU view of P2G + G2P: the counted FMAs per particle-step
    over their time, against SMs x 128 FP32 lanes x 2 flop x the SM clock."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or clocks.get("sm_mhz") or 2070.0
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    flops = 2.0 * FMA_PER_PARTICLE_STEP_27 * P
    achieved = flops / ((ph[1] + ph[3]) * 1e-3) / 1e12
    return {"unit": "TFLOP/s (FP32)", "peak": round(peak, 1), "achieved": round(achieved, 2),
            "frac": round(achieved / peak, 4), "flop_per_particle_step": 2 * FMA_PER_PARTICLE_STEP_27,
            "note": "counted contraction FMAs only (no weights, decisions or addressing)"}


def preroll(pp, torch, scene, steps, device):
    """The dam break run `steps` steps from rest WITH the pressure projection
    (multigrid-preconditioned CG, FP64 reductions), FP32 coefficients, 27
    modes: the sustained state every timed figure starts from (the particles
    have fallen and spread, and cells hold uneven counts)."""
    ctx = pp.Context(scene.n, scene.dx, 27)
    a, b = make_state(pp, ctx, scene, device)
    g = ctx.new_grid(device=device)
    ws = ctx.workspace(a.count, device=device)
    prj = pp.UpdateSettings(dt=scene.dt, project=True, pcg_maxiter=2000)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for _ in range(steps):
        pp.polypic_step(ctx, a, b, g, prj, ws, stream=stream)
        a, b = b, a
    torch.cuda.synchronize()
    st = pp.polypic_check_device_status(ctx)
    if st != 0:
        raise RuntimeError(f"device status {pp.STATUS_NAMES.get(st)} during the pre-roll")
    out = {"x": a.x.clone(), "mass": a.mass.clone(), "coeff": a.coeff.clone(),
           "vel": [v.clone() for v in g.vel], "steps": steps,
           "seconds": round(time.perf_counter() - t0, 2),
           "stability": state_stats(pp, torch, a, scene.dt, scene.dx, steps)}
    del ctx, a, b, g, ws
    torch.cuda.empty_cache()
    return out


def state_from(pp, ctx, pre, device):
    """(src, dst) particle states of context ctx at the pre-rolled positions:
    the pre-rolled FP32 27-mode coefficients as they are, or, for another mode
    count, format or variant, the coefficients G2P fits (dt = 0, positions
    unchanged) from the pre-rolled grid velocity."""
    src = pp.upload_particles(ctx, pre["x"], pre["mass"], None, device=device)
    dst = ctx.new_particles(src.count, device=device)
    if ctx.num_modes == 27 and ctx.coeff_format == "f32" and not ctx.variant:
        src.coeff.copy_(pre["coeff"])
        return src, dst
    ws = ctx.workspace(src.count, device=device)
    g = ctx.new_grid(device=device)
    for a in range(3):
        g.vel[a].copy_(pre["vel"][a])
    pp.polypic_sort(ctx, src, ws)
    pp.polypic_g2p(ctx, g, src, dst, 0.0, ws)
    del ws, g
    return dst, src


def round_efficiency(cell_start) -> float:
    """Particles over 32 x the fullest cell, summed over the 32-key blocks:
    the share of lane rounds a one-lane-per-cell P2G would keep busy (a
    property of the state; the library's schedule balances it)."""
    cs = cell_start.cpu().numpy().view(np.uint32).astype(np.int64)
    cnt = np.diff(cs).reshape(-1, 32)
    mx = cnt.max(axis=1)
    live = mx > 0
    return round(float(cnt.sum() / max(1, (32 * mx[live]).sum())), 4)


def state_stats(pp, torch, ps, dt, dx, steps_run):
    """Stability of a state (reported, not gated: the paper found 27 fluid
    modes unstable in coupled runs): the particle velocity c_p0 (decoded for
    16-bit codes), its largest magnitude, the CFL number max |v| dt / dx, the
    kinetic energy per particle and whether every coefficient is finite."""
    c = ps.coeff.float()
    if ps.scale is not None and ps.coeff.dtype != torch.float32:
        v = c[:, 0, :, 0] * ps.scale[None, :]      # mode 0: the low half of word 0
    else:
        v = c[:, 0, :]
    speed = torch.sqrt((v.double() ** 2).sum(dim=0))
    vmax = float(speed.max().item()) if speed.numel() else 0.0
    ke = float((0.5 * ps.mass.double() * speed ** 2).mean().item()) if speed.numel() else 0.0
    return {"steps_run": steps_run, "max_speed_m_s": round(vmax, 4),
            "cfl": round(vmax * dt / dx, 4), "kinetic_energy_per_particle_j": ke,
            "finite": bool(torch.isfinite(c).all().item())}


def run_variant(pp, torch, scene, pre, R, fmt, steps, warmup, device, **ctx_opts):
    """Times `steps` calls of polypic_step (the whole path, as a user runs it)
    from the pre-rolled state, then `steps` steps made of the individual calls
    (sort, P2G, grid update, G2P) with events between them for the per-phase
    split.  ctx_opts: the context's map_affine / apic_grad_w variants."""
    ctx = pp.Context(scene.n, scene.dx, R, coeff_format=fmt, **ctx_opts)
    src, dst = state_from(pp, ctx, pre, device)
    g = ctx.new_grid(device=device)
    ws = ctx.workspace(src.count, device=device)
    prm = pp.UpdateSettings(dt=scene.dt)
    stream = torch.cuda.current_stream()

    def phases(s, d, ev):
        pp.polypic_sort(ctx, s, ws, stream)
        ev[0].record(stream)
        pp.polypic_p2g_mapped(ctx, s, g, scene.dt, ws, stream)
        ev[1].record(stream)
        pp.polypic_grid_update(ctx, g, prm, stream=stream)
        ev[2].record(stream)
        pp.polypic_g2p(ctx, g, s, d, scene.dt, ws, stream)
        ev[3].record(stream)

    for _ in range(warmup):
        pp.polypic_step(ctx, src, dst, g, prm, ws, stream=stream)
        src, dst = dst, src
    torch.cuda.synchronize()
    st = pp.polypic_check_device_status(ctx)
    if st != 0:
        raise RuntimeError(f"device status {pp.STATUS_NAMES.get(st)} during warm-up")
    E = lambda: torch.cuda.Event(enable_timing=True)
    start, end = E(), E()
    start.record(stream)
    for _ in range(steps):
        pp.polypic_step(ctx, src, dst, g, prm, ws, stream=stream)
        src, dst = dst, src
    end.record(stream)
    torch.cuda.synchronize()
    total_ms = start.elapsed_time(end)

    evs = [[E(), E(), E(), E()] for _ in range(steps)]
    starts = [E() for _ in range(steps)]
    for k in range(steps):
        starts[k].record(stream)
        phases(src, dst, evs[k])
        src, dst = dst, src
    torch.cuda.synchronize()
    ph = np.zeros(4)
    for k in range(steps):
        ph[0] += starts[k].elapsed_time(evs[k][0])
        ph[1] += evs[k][0].elapsed_time(evs[k][1])
        ph[2] += evs[k][1].elapsed_time(evs[k][2])
        ph[3] += evs[k][2].elapsed_time(evs[k][3])
    st = pp.polypic_check_device_status(ctx)
    return {"ctx": ctx, "count": src.count, "total_ms": total_ms,
            "phase_ms": (ph / steps).tolist(), "status": pp.STATUS_NAMES.get(st),
            "round_efficiency": round_efficiency(src.cell_start),
            "stability": state_stats(pp, torch, src, scene.dt, scene.dx,
                                     pre["steps"] + warmup + 2 * steps)}


class L2Flush:
    """Writes a 256 MB buffer (twice the 129 MB L2) before each timed call of
    a workload whose data would otherwise stay in L2 between calls."""

    def __init__(self, torch, device):
        self.buf = torch.empty(64 << 20, dtype=torch.float32, device=device)

    def __call__(self):
        self.buf.fill_(1.0)


def time_calls(torch, fn, iters, flush, stream):
    """Median device time (ms) of `iters` calls of fn, each bracketed by CUDA
    events on `stream` after an L2 flush (not timed)."""
    E = lambda: torch.cuda.Event(enable_timing=True)
    evs = []
    for _ in range(iters):
        flush()
        a, b = E(), E()
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in evs]))


def face_nodes(n):
    return sum((n[0] + (a == 0)) * (n[1] + (a == 1)) * (n[2] + (a == 2)) for a in range(3))


def run_rows(pp, torch, scenes, device, hbm, which, iters=10, warmup=3, large_steps=100):
    """The rows of the path outside the headline step, each on the workload
    it is defined on: the coupled fluid + fabric step (splash scene, 128^3),
    the grid update and the pressure projection (dam break, 128^3), and the
    three adjoints (random-velocity half box, 64^3, 27 modes).  Each figure is
    the median of `iters` calls with L2 flushed before each."""
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch, device)
    rows = {}

    def gbs(nbytes, ms):
        v = nbytes / (ms * 1e-3) / 1e9
        return {"achieved_gbs": round(v, 1), "frac_of_peak": round(v / hbm, 4),
                "algorithmic_bytes": int(nbytes)}

    if "coupled" in which:
        sc = scenes.splash_scene(n=128, R_fluid=27, R_solid=27)
        ctx = pp.Context(sc.n, sc.dx, 27)
        fi = pp.upload_particles(ctx, sc.fluid.x, sc.fluid.mass, sc.fluid.coeff, device=device)
        si = pp.upload_particles(ctx, sc.solid.x, sc.solid.mass, None,
                                 mass_abs=sc.solid.mass_abs, device=device)
        fo = ctx.new_particles(fi.count, device=device)
        so = ctx.new_particles(si.count, solid=True, device=device)
        gf, gs = ctx.new_grid(device=device), ctx.new_grid(device=device)
        ws = ctx.workspace(fi.count, si.count, device=device)
        prm = pp.UpdateSettings(dt=sc.dt, drag_k=5.0)
        st = {"f": (fi, fo), "s": (si, so)}

        def step():
            (a, b), (c, d) = st["f"], st["s"]
            pp.polypic_step(ctx, a, b, gf, prm, ws, solid_in=c, solid_out=d, gs=gs,
                            stream=stream)
            st["f"], st["s"] = (b, a), (d, c)
        for _ in range(warmup):
            step()
        ms = time_calls(torch, step, iters, flush, stream)
        npart = fi.count + si.count
        p2g_b, g2p_b = algorithmic_bytes(27, "f32")
        nbytes = fi.count * (p2g_b + g2p_b) + si.count * (p2g_b + 4 + g2p_b + 4)
        rows["A2_coupled_step"] = {
            "workload": f"splash 128^3: fluid sphere {fi.count} + sheet {si.count} particles, "
                        "27 modes FP32, drag K 5", "ms": round(ms, 4),
            "value": round(npart / (ms * 1e-3) / 1e6, 1), "unit": UNIT,
            **gbs(nbytes, ms),
            "bytes_note": "P2G+G2P algorithmic bytes of both phases over the whole step "
                          "(sort, two P2G, drag update, two G2P)",
            "status": pp.STATUS_NAMES.get(pp.polypic_check_device_status(ctx))}
        del ctx, fi, si, fo, so, gf, gs, ws

    if "fabric" in which:
        # the same splash with the fabric and absorption stand-ins in the step
        sc = scenes.splash_scene(n=128, R_fluid=27, R_solid=27)
        m = int(sc.meta.get("sheet_vertices", 256 * 256) ** 0.5 + 0.5)
        h = 0.8 / (m - 1)
        ctx = pp.Context(sc.n, sc.dx, 27)
        fi = pp.upload_particles(ctx, sc.fluid.x, sc.fluid.mass, sc.fluid.coeff, device=device)
        si = pp.upload_particles(ctx, sc.solid.x, sc.solid.mass, None, mass_abs=sc.solid.mass_abs,
                                 device=device, ids=np.arange(sc.solid.n))
        fo = ctx.new_particles(fi.count, device=device)
        so = ctx.new_particles(si.count, solid=True, device=device, ids=True)
        gf, gs = ctx.new_grid(device=device), ctx.new_grid(device=device)
        ws = ctx.workspace(fi.count, si.count, device=device)
        prm = pp.UpdateSettings(dt=sc.dt, drag_k=5.0)
        fab = pp.FabricSettings(verts_per_side=m, rest_length=h, k_stretch=20.0, k_shear=8.0,
                                k_bend=2.0, damping=1e-4, absorb_rate=5.0, absorb_capacity=2.0,
                                absorb_max_fraction=0.2)
        st = {"f": (fi, fo), "s": (si, so)}

        def cstep():
            (a, b), (c, d) = st["f"], st["s"]
            pp.polypic_step_coupled(ctx, a, b, c, d, gf, gs, prm, fab, ws, stream=stream)
            st["f"], st["s"] = (b, a), (d, c)

        def total_mass():
            (a, _), (c, _) = st["f"], st["s"]
            return float(a.mass.double().sum().item() + c.mass_abs.double().sum().item())
        # 150 untimed steps first: the sphere (2 m/s, 5 cells above the sheet)
        # reaches the sheet, so the timed steps absorb and stretch it
        for _ in range(150 + warmup):
            cstep()
        m0 = total_mass()
        ms = time_calls(torch, cstep, iters, flush, stream)
        for _ in range(40):
            cstep()
        torch.cuda.synchronize()
        m1 = total_mass()
        (a, _), (c, _) = st["f"], st["s"]
        ms_forces = time_calls(torch, lambda: pp.polypic_fabric_forces(ctx, c, fab, 0.0, ws,
                                                                       stream=stream),
                               iters, flush, stream)
        pp.polypic_sort(ctx, a, ws, stream)
        pp.polypic_sort(ctx, c, ws, stream)
        ms_absorb = time_calls(torch, lambda: pp.polypic_absorb(ctx, a, c, fab, sc.dt,
                                                                stream=stream),
                               iters, flush, stream)
        rows["f3_fabric_step"] = {
            "workload": f"splash 128^3 with the stand-ins: fluid sphere {fi.count} + sheet "
                        f"{si.count} particles ({m}^2 lattice, springs k 20/8/2 N/m, damping "
                        "1e-4 kg/s; absorption rate 5/s, capacity 2, at most 20% of a cell's "
                        "fluid per step), 27 modes FP32, drag K 5",
            "ms": round(ms, 4), "value": round((fi.count + si.count) / (ms * 1e-3) / 1e6, 1),
            "unit": UNIT, "ms_fabric_forces": round(ms_forces, 4),
            "ms_absorb": round(ms_absorb, 4),
            "mass_drift_rel": abs(m1 - m0) / m0, "absorbed_kg": float(c.mass_abs.double().sum()),
            "stability": state_stats(pp, torch, c, sc.dt, sc.dx, 150 + warmup + iters + 40),
            "status": pp.STATUS_NAMES.get(pp.polypic_check_device_status(ctx))}
        del ctx, fi, si, fo, so, gf, gs, ws

    if "update" in which or "projection" in which:
        sc = scenes.dam_break_scene(n=128, R=27)
        ctx = pp.Context(sc.n, sc.dx, 27)
        a = pp.upload_particles(ctx, sc.fluid.x, sc.fluid.mass, None, device=device)
        b = ctx.new_particles(a.count, device=device)
        g = ctx.new_grid(device=device)
        ws = ctx.workspace(a.count, device=device)
        prm = pp.UpdateSettings(dt=sc.dt)
        for _ in range(10):
            pp.polypic_step(ctx, a, b, g, prm, ws, stream=stream)
            a, b = b, a
        pp.polypic_sort(ctx, a, ws, stream)
        pp.polypic_p2g(ctx, a, g, ws, stream)
        upd = lambda: pp.polypic_grid_update(ctx, g, prm, stream=stream)
        for _ in range(warmup):
            upd()
        ms_u = time_calls(torch, upd, iters, flush, stream)
        nodes = face_nodes(sc.n)
        if "update" in which:
            rows["A3_grid_update"] = {
                "workload": "dam break 128^3 after 10 steps, 3 face grids", "ms": round(ms_u, 4),
                "face_nodes": nodes, **gbs(12 * nodes, ms_u),
                "bytes_note": "12 B per face node: m and mv read, v written"}
        if "projection" in which:
            prj = pp.UpdateSettings(dt=sc.dt, project=True, pcg_maxiter=2000)
            pr = lambda: pp.polypic_grid_update(ctx, g, prj, fluid_particles=a, ws=ws,
                                                stream=stream)
            pr()
            ms_p = time_calls(torch, pr, 3, flush, stream)
            rows["A4_projection"] = {
                "workload": "dam break 128^3 after 10 steps: about 476,656 fluid cells (the "
                            "62x124x62-cell block), multigrid-preconditioned CG to rtol 1e-6, "
                            "at most 2000 iterations",
                "ms_update_and_projection": round(ms_p, 3),
                "ms_projection": round(ms_p - ms_u, 3),
                "note": "not in the headline step; the host reads the residual every 8 "
                        "iterations",
                "status": pp.STATUS_NAMES.get(pp.polypic_check_device_status(ctx))}
        del ctx, a, b, g, ws

    if "adjoint" in which:
        R = 27
        sc = scenes.random_velocity_scene(n=64, R=R, seed=0, sigma_v=0.3, dt=1e-3)
        ctx = pp.Context(sc.n, sc.dx, R)
        p0 = pp.upload_particles(ctx, sc.fluid.x, sc.fluid.mass, sc.fluid.coeff, device=device)
        ws = ctx.workspace(p0.count, device=device)
        g = ctx.new_grid(device=device)
        prm = pp.UpdateSettings(dt=sc.dt)
        # one forward step first: a rollout's saved states are in the slot
        # order of the previous step's sort, as here
        ps = ctx.new_particles(p0.count, device=device)
        pp.polypic_step(ctx, p0, ps, g, prm, ws, stream=stream)
        del p0
        pp.polypic_sort(ctx, ps, ws, stream)
        pp.polypic_p2g(ctx, ps, g, ws, stream)
        pp.polypic_grid_update(ctx, g, prm, stream=stream)
        gen = torch.Generator(device=device).manual_seed(1)
        bar_out = ctx.new_particles(ps.count, device=device)
        bar_out.coeff.normal_(generator=gen)
        bar_out.x.normal_(generator=gen)
        bar_grid, bar_mid = ctx.new_grid(device=device), ctx.new_grid(device=device)
        bar_in = ctx.new_particles(ps.count, device=device)
        calls = {
            "g2p_adjoint": lambda: pp.polypic_g2p_adjoint(ctx, g, ps, sc.dt, bar_out, bar_grid,
                                                          bar_in, ws, stream=stream),
            "grid_update_adjoint": lambda: pp.polypic_grid_update_adjoint(
                ctx, g, prm, bar_grid, bar_mid, stream=stream),
            "p2g_adjoint": lambda: pp.polypic_p2g_adjoint(ctx, ps, bar_mid, bar_in, ws,
                                                          accumulate=True, stream=stream),
        }
        P, cells, nodes = ps.count, int(np.prod(sc.n)), face_nodes(sc.n)
        nbytes = {
            "g2p_adjoint": P * (12 + 24 + 12 * R + 12) + 2 * 4 * nodes,
            "grid_update_adjoint": 20 * nodes,
            "p2g_adjoint": P * (12 + 4 + 12 * R + 12 * R + 24) + 8 * nodes,
        }
        out = {"workload": f"random-velocity half box 64^3: {P} particles, 27 modes FP32, "
                           "state after one forward step"}
        tot = 0.0
        for name, fn in calls.items():
            for _ in range(warmup):
                fn()
            ms = time_calls(torch, fn, iters, flush, stream)
            tot += ms
            out[name] = {"ms": round(ms, 4), **gbs(nbytes[name], ms)}
        out["ms_adjoint_step"] = round(tot, 4)
        out["value"] = round(P / (tot * 1e-3) / 1e6, 1)
        out["unit"] = "M particle-steps/s (adjoint of one transfer step)"
        out["bytes_note"] = ("g2p_adjoint: x, bar c, bar x in, bar x out, v and bar v; "
                             "p2g_adjoint: x, m, c, bar c, bar x (read-modify-write), bar grid")
        out["status"] = pp.STATUS_NAMES.get(pp.polypic_check_device_status(ctx))
        rows["A8_adjoints"] = out
        del ctx, ps, ws, g, bar_out, bar_grid, bar_mid, bar_in
    if "large" in which:
        rows["cfg_large_fluid_fabric_256"] = run_large(pp, torch, scenes, device,
                                                       steps=large_steps, timed=10, hbm=hbm)
    del flush
    torch.cuda.empty_cache()
    return rows


def field_on_grid(torch, scene, ctx, device):
    """The large scene's vortical field sampled at the face positions of the
    three face grids (device tensors in the library's grid layout)."""
    out = []
    dx = scene.dx
    for a in range(3):
        d = ctx.grid_dims(a)
        off = [0.0 if b == a else 0.5 for b in range(3)]
        ax = [(torch.arange(d[b], device=device, dtype=torch.float64) + off[b]) * dx
              for b in range(3)]
        zz, yy, xx = torch.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        v = torch.zeros_like(xx)
        for k, amp, ph in scene.meta["field"]:
            v += float(amp[a]) * torch.sin(2 * np.pi * (float(k[0]) * xx + float(k[1]) * yy
                                                          + float(k[2]) * zz) + ph)
        out.append(v.float().contiguous())
        del xx, yy, zz, v
    return out


def run_large(pp, torch, scenes, device, steps, timed, hbm=None):
    """Large fluid + fabric at 256^3: ~64M fluid particles (the lower half-box
    at 8 per cell, a vortical initial field) and a 1024^2-vertex sheet (3.1M
    vertex and element particles), 27 modes, dt 2.5e-4, FP32 coefficients
    against BF16 and FP16 per-particle-scaled codes.  Each format fits its
    initial modes from the same grid field, then runs `steps` steps of both
    phases with the pressure projection (FP64 reductions) and drag; the last
    `timed` steps are made of the individual calls with CUDA events, and the
    transfer time per step (the sorts, P2Gs and G2Ps of both phases; the grid
    update and projection are reported apart) gives the throughput.  The 16-bit
    forms' grid momentum is compared, on the first P2G, with the FP32 form's
    (itself within 1e-5 of the FP64 oracle at smaller sizes)."""
    sc = scenes.large_scene()
    f, sol = sc.fluid, sc.solid
    timed = max(1, min(timed, steps))
    stream = torch.cuda.current_stream()
    E = lambda: torch.cuda.Event(enable_timing=True)
    out = {"workload": f"256^3 half box, {f.n} fluid particles (8/cell, vortical field of 4 "
                       f"solenoidal modes, 0.5 m/s) + {sol.n} sheet particles "
                       f"(1024^2 vertices at y = 0.75), 27 modes, dt 2.5e-4, drag K 5, "
                       f"projection every step", "steps": steps, "timed_steps": timed}
    ref_mom = None
    for fmt in ("f32", "bf16", "f16"):
        ctx = pp.Context(sc.n, sc.dx, 27, coeff_format=fmt)
        vel = field_on_grid(torch, sc, ctx, device)
        g0 = ctx.new_grid(device=device)
        for a in range(3):
            g0.vel[a].copy_(vel[a])
        del vel
        ws = ctx.workspace(f.n, sol.n, device=device)
        fa = pp.upload_particles(ctx, f.x, f.mass, None, device=device)
        fb = ctx.new_particles(f.n, device=device)
        sa = pp.upload_particles(ctx, sol.x, sol.mass, None, mass_abs=sol.mass_abs, device=device)
        sb = ctx.new_particles(sol.n, solid=True, device=device)
        pp.polypic_sort(ctx, fa, ws)
        pp.polypic_g2p(ctx, g0, fa, fb, 0.0, ws)
        pp.polypic_sort(ctx, sa, ws)
        pp.polypic_g2p(ctx, g0, sa, sb, 0.0, ws)
        fa, fb, sa, sb = fb, fa, sb, sa
        gf, gs = g0, ctx.new_grid(device=device)
        # first P2G: the grid-momentum error of the 16-bit forms against FP32
        pp.polypic_sort(ctx, fa, ws)
        pp.polypic_p2g(ctx, fa, gf, ws)
        torch.cuda.synchronize()
        if fmt == "f32":
            ref_mom = [m.clone() for m in gf.mom]
            err = None
        else:
            num = sum(float(((gf.mom[a].double() - ref_mom[a].double()) ** 2).sum()) for a in range(3))
            den = sum(float((ref_mom[a].double() ** 2).sum()) for a in range(3))
            mx = max(float((gf.mom[a] - ref_mom[a]).abs().max()) for a in range(3))
            mref = max(float(ref_mom[a].abs().max()) for a in range(3))
            err = {"norm_rel": num ** 0.5 / den ** 0.5, "max_rel": mx / mref}
        prm = pp.UpdateSettings(dt=sc.dt, project=True, drag_k=5.0, pcg_maxiter=2000)
        t_tr, t_upd = 0.0, 0.0
        for k in range(steps):
            ev = [E() for _ in range(8)]
            ev[0].record(stream)
            pp.polypic_sort(ctx, fa, ws, stream)
            pp.polypic_p2g(ctx, fa, gf, ws, stream)
            ev[1].record(stream)
            pp.polypic_sort(ctx, sa, ws, stream)
            pp.polypic_p2g(ctx, sa, gs, ws, stream)
            ev[2].record(stream)
            pp.polypic_grid_update(ctx, gf, prm, solid=gs, fluid_particles=fa, ws=ws,
                                   stream=stream)
            ev[3].record(stream)
            pp.polypic_g2p(ctx, gf, fa, fb, sc.dt, ws, stream)
            ev[4].record(stream)
            pp.polypic_g2p(ctx, gs, sa, sb, sc.dt, ws, stream)
            ev[5].record(stream)
            fa, fb, sa, sb = fb, fa, sb, sa
            if k >= steps - timed:
                torch.cuda.synchronize()
                t_tr += (ev[0].elapsed_time(ev[1]) + ev[1].elapsed_time(ev[2])
                         + ev[3].elapsed_time(ev[4]) + ev[4].elapsed_time(ev[5]))
                t_upd += ev[2].elapsed_time(ev[3])
        torch.cuda.synchronize()
        st = pp.polypic_check_device_status(ctx)
        ms = t_tr / timed
        pb, gb = algorithmic_bytes(27, fmt)
        nbytes = f.n * (pb + gb) + sol.n * (pb + 4 + gb + 4)   # + m_abs read and written
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[fmt] = {"ms_transfers_per_step": round(ms, 3),
                    "ms_update_and_projection_per_step": round(t_upd / timed, 3),
                    "value": round((f.n + sol.n) / (ms * 1e-3) / 1e6, 1), "unit": UNIT,
                    "achieved_gbs": round(gbs, 1),
                    "frac_of_peak": round(gbs / hbm, 4) if hbm else None,
                    "bytes_note": "P2G + G2P algorithmic bytes of both phases over the "
                                  "transfer time (the sorts included)",
                    "grid_momentum_error_vs_f32": err,
                    "stability": state_stats(pp, torch, fa, sc.dt, sc.dx, steps),
                    "status": pp.STATUS_NAMES.get(st)}
        del ctx, fa, fb, sa, sb, gf, gs, g0, ws
        torch.cuda.empty_cache()
    for fmt in ("bf16", "f16"):
        out[fmt]["speedup_vs_f32"] = round(out["f32"]["ms_transfers_per_step"]
                                           / out[fmt]["ms_transfers_per_step"], 3)
    del ref_mom
    torch.cuda.empty_cache()
    return out


def run_graph(pp, torch, scene, pre, R, steps, warmup, device):
    """polypic_step replayed from CUDA graphs: the two ping-pong steps (a -> b,
    b -> a) are each captured once (the step makes no host synchronisation
    without the projection) and replayed `steps` times, which removes the
    launch gaps between its kernels."""
    ctx = pp.Context(scene.n, scene.dx, R)
    a, b = state_from(pp, ctx, pre, device)
    g = ctx.new_grid(device=device)
    ws = ctx.workspace(a.count, device=device)
    prm = pp.UpdateSettings(dt=scene.dt)
    for _ in range(warmup):                   # also configures the kernels before capture
        pp.polypic_step(ctx, a, b, g, prm, ws, stream=torch.cuda.current_stream())
        a, b = b, a
    torch.cuda.synchronize()
    graphs = []
    for src, dst in ((a, b), (b, a)):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            pp.polypic_step(ctx, src, dst, g, prm, ws, stream=torch.cuda.current_stream())
        graphs.append(gr)
    for k in range(2):
        graphs[k % 2].replay()
    torch.cuda.synchronize()
    E = lambda: torch.cuda.Event(enable_timing=True)
    s0, s1 = E(), E()
    s0.record()
    for k in range(steps):
        graphs[k % 2].replay()
    s1.record()
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1)
    st = pp.polypic_check_device_status(ctx)
    return {"value": a.count * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
            "status": pp.STATUS_NAMES.get(st)}


def run_fused(pp, torch, scene, pre, steps, warmup, device):
    """The fused transfer on the same workload: each step sorts, runs
    polypic_g2p2g (G2P of step n with the P2G of step n + 1, the movers
    through a spill phase) and the grid update, so a step's work is the same
    as polypic_step's (one sort, one P2G, one update, one G2P per particle)
    with the staying particles' coefficients kept out of HBM.  The timed
    loop starts from the pre-rolled state's P2G and update; the per-phase
    split comes from a second loop with events between the calls."""
    ctx = pp.Context(scene.n, scene.dx, 27)
    a, b = state_from(pp, ctx, pre, device)
    ws = ctx.workspace(a.count, device=device)
    spill = ctx.new_particles(a.count // 2, device=device)
    prm = pp.UpdateSettings(dt=scene.dt)
    stream = torch.cuda.current_stream()
    gf, gn = ctx.new_grid(device=device), ctx.new_grid(device=device)
    pp.polypic_sort(ctx, a, ws, stream)
    pp.polypic_p2g(ctx, a, gf, ws, stream)
    pp.polypic_grid_update(ctx, gf, prm, stream=stream)
    st = {"a": a, "b": b, "g": gf, "n": gn}

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        pp.polypic_g2p2g(ctx, st["g"], st["a"], st["b"], spill, st["n"], scene.dt, ws, stream)
        if ev is not None:
            ev[1].record(stream)
        pp.polypic_grid_update(ctx, st["n"], prm, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        pp.polypic_sort(ctx, st["b"], ws, stream)
        if ev is not None:
            ev[3].record(stream)
        st["a"], st["b"], st["g"], st["n"] = st["b"], st["a"], st["n"], st["g"]
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    E = lambda: torch.cuda.Event(enable_timing=True)
    s0, s1 = E(), E()
    s0.record(stream)
    for _ in range(steps):
        step()
    s1.record(stream)
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / steps
    evs = [[E() for _ in range(4)] for _ in range(steps)]
    for k in range(steps):
        step(evs[k])
    torch.cuda.synchronize()
    ph = np.zeros(3)
    for e in evs:
        ph += [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
    ph /= steps
    # share of particles that changed cell in the last step (state a's slots
    # against the new positions of the same particles)
    old, new = st["b"], st["a"]        # the last step's input (its slot order) and output
    inv = np.float32(1.0 / scene.dx)
    k_old = torch.floor(old.x[:, old.perm.long()] * inv)
    k_new = torch.floor(new.x * inv)
    moved = float((k_old != k_new).any(dim=0).float().mean().item())
    return {"ms_per_step": ms, "value": a.count / (ms * 1e-3) / 1e6,
            "phase_ms": {"g2p2g": round(ph[0], 4), "grid_update": round(ph[1], 4),
                         "sort": round(ph[2], 4)},
            "movers_share": round(moved, 4),
            "status": pp.STATUS_NAMES.get(pp.polypic_check_device_status(ctx))}


def run_e2e(pp, torch, scene, pre, R, steps, device, lanes=2):
    """Through the C ABI with host buffers: every step copies the particle
    state in from pinned host memory, runs polypic_step, and copies the new
    state back out.  Steps alternate between `lanes` streams, each with its
    own device buffers, grid and workspace, so that one step's results stream
    back while the next step's inputs stream in and compute; every step still
    moves its full input and output across the host link inside the timed
    region."""
    ctx = pp.Context(scene.n, scene.dx, R)
    P = int(pre["x"].shape[1])
    prm = pp.UpdateSettings(dt=scene.dt)
    h_x = pre["x"].cpu().pin_memory()
    h_m = pre["mass"].cpu().pin_memory()
    h_c = pre["coeff"].cpu().pin_memory()
    L = []
    for _ in range(lanes):
        L.append({"s": torch.cuda.Stream(device=device),
                  "in": ctx.new_particles(P, device=device),
                  "out": ctx.new_particles(P, device=device),
                  "g": ctx.new_grid(device=device), "ws": ctx.workspace(P, device=device),
                  "xo": torch.empty((3, P), dtype=torch.float32).pin_memory(),
                  "co": torch.empty((3, R, P), dtype=torch.float32).pin_memory()})
    h2d = (h_x.numel() + h_m.numel() + h_c.numel()) * 4
    d2h = (L[0]["xo"].numel() + L[0]["co"].numel()) * 4

    def step(lane):
        with torch.cuda.stream(lane["s"]):
            lane["in"].x.copy_(h_x, non_blocking=True)
            lane["in"].mass.copy_(h_m, non_blocking=True)
            lane["in"].coeff.copy_(h_c, non_blocking=True)
            pp.polypic_step(ctx, lane["in"], lane["out"], lane["g"], prm, lane["ws"],
                            stream=lane["s"])
            lane["xo"].copy_(lane["out"].x, non_blocking=True)
            lane["co"].copy_(lane["out"].coeff, non_blocking=True)

    for lane in L:
        step(lane)
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(main)
    for lane in L:
        lane["s"].wait_event(a)
    for k in range(steps):
        step(L[k % lanes])
    for lane in L:
        main.wait_stream(lane["s"])
    b.record(main)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    st = pp.polypic_check_device_status(ctx)
    return {"value": P / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "streams": lanes, "status": pp.STATUS_NAMES.get(st)}


def cpu_baseline(scene, R, target_s=12.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same
    workload: the first S particles of the scene on the full grid, one step
    each (P2G, grid update, G2P); S grows until a run takes a few seconds.
    Timed on all host cores (OpenMP: G2P split by particle, P2G on private
    grids summed in thread order) and on one thread."""
    import oracle
    f = scene.fluid
    cores = os.cpu_count() or 1

    def timed(threads, S0):
        oracle.set_threads(threads)
        S = S0
        try:
            while True:
                x = f.x[:, :S]
                m = f.mass[:S]
                c = np.zeros((3, R, S))
                t0 = time.perf_counter()
                oracle.step(x, m, c, scene.n, scene.dx, scene.dt)
                el = time.perf_counter() - t0
                if el > target_s / 4 or S >= f.n:
                    return S, el
                S = min(f.n, int(S * max(2.0, (target_s / 4) / max(el, 1e-3))))
        finally:
            oracle.set_threads(1)

    S1, e1 = timed(1, 2000)
    Sn, en = timed(cores, 4000 * cores)
    return {"value": Sn / en / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{Sn} of {f.n} particles of the initial dam break, one full step "
                      f"(P2G, grid update, G2P) on the {scene.n[0]}^3 grid, FP64, "
                      f"{cores} OpenMP threads", "seconds": round(en, 3),
            "single_thread": {"value": S1 / e1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": f"{S1} particles, one step", "seconds": round(e1, 3)}}


# ---------------------------------------------------------------- arms

def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2308_01060_gb300 import scenes
    import oracle
    oracle.build()
    scene = scenes.dam_break_scene(n=args.n, R=27)
    f = scene.fluid
    cores = os.cpu_count() or 1
    S = min(10000 * cores, f.n)
    x = f.x[:, :S]
    m = f.mass[:S]
    c = np.zeros((3, 27, S))
    oracle.set_threads(cores)
    try:
        for _ in range(max(args.warmup, 0)):
            oracle.step(x, m, c, scene.n, scene.dx, scene.dt)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c_new, x_new, _ = oracle.step(x, m, c, scene.n, scene.dx, scene.dt)
            x, c = x_new, c_new
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    value = S * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dam_break_{args.n}^3, 27 modes, dt 5e-4",
                       "sample_particles_per_step": S},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{S} of {f.n} particles of the initial dam break per "
                                       f"step on the full grid, {cores} OpenMP threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def our_arm(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    from paper_2308_01060_gb300 import polypic as pp
    from paper_2308_01060_gb300 import scenes
    pp.load_library()

    scene = scenes.dam_break_scene(n=args.n, R=27)
    P = scene.fluid.n
    hbm, peak_kind = peaks()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # the sustained state: the dam break stepped with projection (untimed)
    pre = preroll(pp, torch, scene, args.preroll, device)

    # headline: 27 modes, FP32 coefficients
    barrier()
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    sampler.start()
    t_wall = time.perf_counter()
    main = run_variant(pp, torch, scene, pre, 27, "f32", args.steps, args.warmup, device)
    barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    ms, value = job_throughput(torch, main["total_ms"], P, args.steps, world, device)
    ms_step = ms / args.steps

    p2g_b, g2p_b = algorithmic_bytes(27, "f32")
    ph = main["phase_ms"]
    p2g_gbs = P * p2g_b / (ph[1] * 1e-3) / 1e9
    g2p_gbs = P * g2p_b / (ph[3] * 1e-3) / 1e9
    pair_gbs = P * (p2g_b + g2p_b) / ((ph[1] + ph[3]) * 1e-3) / 1e9
    dominant = "p2g" if ph[1] >= ph[3] else "g2p"
    dom_gbs = p2g_gbs if dominant == "p2g" else g2p_gbs
    roofline = {
        "bound": "hbm", "achieved": round(dom_gbs, 1), "peak": hbm, "unit": "GB/s",
        "frac": round(dom_gbs / hbm, 4),
        "traffic": (round(P * P2G_TILES_DRAM_BYTES_PER_PARTICLE / 1e9, 4)
                    if dominant == "p2g" and P2G_TILES_DRAM_BYTES_PER_PARTICLE else None),
        "traffic_unit": "GB per launch (k_p2g_tiles only, scaled from a 96^3 capture)",
        "kernel": "polypic_p2g call (k_p2g_tiles + k_p2g_reduce)" if dominant == "p2g"
        else "polypic_g2p (k_g2p_tiles)",
        "algorithmic_bytes_per_particle": p2g_b if dominant == "p2g" else g2p_b,
        "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
        else "fallback 6800 GB/s",
        "alu_ceiling": alu_ceiling(torch, device, P, ph, clocks),
    }

    variants = {}
    variant_defs = {
        "apic4": (4, "f32", {}),
        "apic4_gradw": (4, "f32", {"apic_grad_w": True}),     # Eq 10 in G2P
        "apic4_affine": (4, "f32", {"map_affine": True}),     # Eq 12 in P2G
        "affine27": (27, "f32", {"map_affine": True}),        # Eq 12, per-node modes
        "bf16": (27, "bf16", {}),
        "f16": (27, "f16", {}),
    }
    for v in [s for s in args.variants.split(",") if s]:
        if v == "fused":
            r = run_fused(pp, torch, scene, pre, args.steps, args.warmup, device)
            variants[v] = {"modes": 27, "coeff_format": "f32",
                           "note": "sort + polypic_g2p2g + grid update per step: the new "
                                   "coefficients of particles that stay in their cell never "
                                   "reach HBM; movers go through a spill phase (one host read "
                                   "of their count per step)",
                           **r, "speedup_vs_f32_step": round(ms_step / r["ms_per_step"], 3)}
            continue
        if v == "graph":
            r = run_graph(pp, torch, scene, pre, 27, args.steps, args.warmup, device)
            variants[v] = {"modes": 27, "coeff_format": "f32",
                           "note": "the same polypic_step calls, replayed from two CUDA graphs",
                           **r, "speedup_vs_f32_step": round(ms_step / r["ms_per_step"], 3)}
            continue
        R, fmt, opts = variant_defs[v]
        r = run_variant(pp, torch, scene, pre, R, fmt, args.steps, args.warmup, device, **opts)
        pb, gb = algorithmic_bytes(R, fmt)
        vph = r["phase_ms"]
        variants[v] = {
            "modes": R, "coeff_format": fmt, **({"options": opts} if opts else {}),
            "value": P * args.steps / (r["total_ms"] * 1e-3) / 1e6,
            "ms_per_step": r["total_ms"] / args.steps,
            "phase_ms": [round(x, 4) for x in vph],
            "p2g_g2p_gbs": round(P * (pb + gb) / ((vph[1] + vph[3]) * 1e-3) / 1e9, 1),
            "speedup_vs_f32_step": round(ms_step / (r["total_ms"] / args.steps), 3),
            "speedup_vs_f32_p2g_g2p": round((ph[1] + ph[3]) / (vph[1] + vph[3]), 3),
            "stability": r["stability"],
            "status": r["status"],
        }
        del r

    rows = run_rows(pp, torch, scenes, device, hbm, [r for r in args.rows.split(",") if r],
                    large_steps=args.large_steps) if args.rows else {}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(pp, torch, scene, pre, 27, args.e2e_steps, device, lanes=args.e2e_lanes)
        e2e["ms_per_step"], e2e["value"] = job_throughput(torch, e2e["ms_per_step"], P, 1, world,
                                                          device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene, 27)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": workload_name(args.n, P, args.preroll),
                "preroll": {"steps": args.preroll, "seconds": pre["seconds"],
                            "stability": pre["stability"]},
                "round_efficiency": main["round_efficiency"],
                "particles_per_gpu": P, "grid": list(scene.n), "modes": 27,
                "step": "polypic_step: sort + P2G (grid update fused) + G2P/advect",
                "l2": f"inputs larger than L2 ({P * (16 + 324) / 1e9:.2f} GB of particle state "
                      f"read per step vs 129 MB L2); no flush",
                "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            },
            "phase_ms": {"sort": round(ph[0], 4), "p2g": round(ph[1], 4),
                         "grid_update": round(ph[2], 4), "g2p": round(ph[3], 4),
                         "note": "separate calls, timed after the headline loop"},
            "p2g_g2p_only": {"value": round(P * world / ((ph[1] + ph[3]) * 1e-3) / 1e6, 3),
                             "unit": UNIT, "gbs": round(pair_gbs, 1),
                             "frac_of_peak": round(pair_gbs / hbm, 4)},
            "roofline": roofline,
            "variants": variants,
            "rows": rows,
            "e2e": e2e,
            "gpu_launches": launches_per_step() * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "device_status": main["status"],
            "stability": main["stability"],
            "wall_s_headline": round(wall, 2),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
