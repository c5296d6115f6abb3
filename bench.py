"""Benchmark of the envelope-tracking FEMPIC particle step on GB300.

Workload: unit cube as 48^3 hexes x 6 Kuhn tets (663,552 tets), 10M electrons
at 5 eV (uniform, Maxwellian), TE101 cavity envelope at 10 kV/m, dt = 0.5 ns;
synthetic inputs generated from fixed seeds.  One step = gather + carrier +
push + track + deposit for every particle (fempic_push_step) and the deposit
finalize (fempic_deposit).  The FP32-mixed form is the headline value; the
FP64 form is measured side by side.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own 10M particles: a z-slab, i.e. a
contiguous tet range, of a uniform load of N x 10M (weak scaling).  Each
step's edge deposit dG is finalized per rank, all-reduced, and added to every
rank's G_cum.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+track+deposit), FP32-mixed vs FP64, % HBM peak"
DATA_DESC = {
    "cube48": "synthetic (seeded): Kuhn cube mesh, TE101 envelope DoFs, uniform Maxwellian electrons",
    "jittered64": "synthetic (seeded): jittered Kuhn cube mesh, random windowed complex DoFs, beam + plasma electrons",
    "large96": "synthetic (seeded, generated in chunks): Kuhn cube mesh, random windowed complex DoFs, "
               "Maxwellian electrons and ions",
}
WORKLOAD_DESC = {
    "cube48": "cube48_10M_te101: 48^3x6 Kuhn cube (663,552 tets), 10M electrons at 5 eV, TE101 10 kV/m, dt 0.5 ns",
    "jittered64": "jittered64_50M: 64^3x6 cube with interior nodes jittered +-20% (1,572,864 tets), 5M 10 keV "
                  "electron beam along z + 45M 5 eV plasma with 1+0.5cos(2 pi x) density, random windowed DoFs, "
                  "dt 0.5 ns",
    "large96": "large96_400M: 96^3x6 Kuhn cube (5,308,416 tets), 200M electrons + 200M ions (1836 m_e) at 2 eV, "
               "random windowed DoFs, dt 0.5 ns",
}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal, for context next to the measured copy peak
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "push_mixed_cube48_10M.txt")
FP64_SUMMARY = os.path.join(ROOT, "profiles", "fp64_ops_cube48_4M.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2208_12795_gb300", "csrc", f)
                  for f in ("fempic_env.cu", "fempic_internal.h")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--particles", type=int, default=10_000_000)
    ap.add_argument("--sort-every", type=int, default=4)
    ap.add_argument("--no-fp64", action="store_true", help="skip the side-by-side FP64 form")
    ap.add_argument("--no-q24", action="store_true", help="skip the 24-bit mixed variant")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-particles", type=int, default=1_000_000)
    ap.add_argument("--cpu-steps", type=int, default=30)
    ap.add_argument("--no-cpu-parallel", action="store_true", help="skip the all-cores oracle baseline")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the gradient-window measurement")
    ap.add_argument("--no-levels3", action="store_true", help="skip the three-level envelope measurement")
    ap.add_argument("--no-downshift", action="store_true", help="skip the downshifted-integrator measurement")
    ap.add_argument("--no-errors", action="store_true", help="skip the per-quantity error report against the oracle")
    ap.add_argument("--no-large", action="store_true", help="skip the 50M jittered and 400M two-species legs")
    ap.add_argument("--large-steps", type=int, default=None,
                    help="steps of the large legs (default: the workloads' own, 50 for jittered64, 20 for large96)")
    ap.add_argument("--workload", choices=("cube48", "jittered64", "large96"), default="cube48",
                    help="cube48: 48^3x6 cube, 10M e- (headline); jittered64: 64^3x6 jittered cube, 50M "
                         "(10 keV beam + cosine plasma), random DoFs; large96: 96^3x6 cube, 400M e- + ions")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def bytes_alg_per_step(n_p, counts, form):
    """Algorithmic bytes of one step: particle state read + written, mesh
    tables (4 node, 4 neighbour, 6 edge, 4 face ids per tet), node
    coordinates, complex DoFs and the dG write."""
    s_p = 52 if form == "fp64" else 40
    s_dof = 16 if form == "fp64" else 8
    nn, ne, nf, nt = counts
    return n_p * 2 * s_p + 72 * nt + 24 * nn + (s_dof + 8) * ne + s_dof * nf


def bytes_reverse_window(n_p, counts, form, steps, every, stash, recompute_steps):
    """Algorithmic bytes of a window's reverse sweep: the recomputed forward
    steps; per step in stash mode a copy of the new state (read + write), or
    in recompute mode the two state copies that seed each step's pair; per
    adjoint step the state before it (positions, velocities, tet), the
    velocities and status after it, the adjoint state read and written, and
    the per-tet and DoF gradient terms; per segment the checkpoint copy and
    the adjoint unpermute (adjoint read + written, permutation read)."""
    nn, ne, nf, nt = counts
    s_state = 53 if form == "fp64" else 41
    s_adj = 48 if form == "fp64" else 36
    before = 52 if form == "fp64" else 40
    after = (24 if form == "fp64" else 12) + 1
    segs = -(-steps // every)
    per_step_mesh = 72 * nt + 4 * 80 * nt + 32 * (ne + nf)
    b = recompute_steps * bytes_alg_per_step(n_p, counts, form)
    b += steps * n_p * 2 * s_state * (1 if stash else 2)
    b += steps * (n_p * (before + after + 2 * s_adj) + per_step_mesh)
    b += segs * n_p * (2 * s_state + 2 * s_adj + 4)
    return b


def bytes_alg_per_step_downshift(n_p, counts, form="fp64"):
    """Algorithmic bytes of one downshifted step: the particle state and the
    history the rule needs (v^{n-1..n-3}: 9 values; the complex E~ and B~
    samples of levels n-1 and n-2: 24 values; f64 in the FP64 form, 264 B,
    f32 in the mixed forms, 132 B), each read and written, plus the mesh and
    DoF terms of the step."""
    nn, ne, nf, nt = counts
    s_p, s_h, s_dof = (52, 264, 16) if form == "fp64" else (40, 132, 8)
    return n_p * 2 * (s_p + s_h) + 72 * nt + 24 * nn + (s_dof + 8) * ne + s_dof * nf


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _profile_value(key, path=PROFILE_SUMMARY):
    """A per-particle figure from a committed ncu summary; None when absent
    or when the kernel source changed since the capture."""
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    try:
        if kv.get("kernel_source_sha") != kernel_source_hash():
            return None
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic(n_p):
    """DRAM bytes per launch of the mixed push group, scaled to n_p particles."""
    v = _profile_value("dram_bytes_per_particle")
    return None if v is None else v * n_p


def issue_roofline(n_p, t_launch_s, sm_mhz):
    """Issue-slot roofline of the staged common path k_push_mixed_tma: its
    warp instructions per launch (ncu count per particle, scaled to n_p) over
    the launch time, against 4 warp instructions per clock on each of the
    GPU's SMs at the sampled SM clock."""
    ipp = _profile_value("tma_warp_instructions_per_particle")
    if ipp is None or t_launch_s <= 0:
        return None
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * sm_mhz * 1e6
    achieved = ipp * n_p / t_launch_s
    return {"kernel": "k_push_mixed_tma", "bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak, "warp_instructions_per_launch": ipp * n_p,
            "avg_launch_ms": t_launch_s * 1e3,
            "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz (median SM clock sampled in the timed region)"}


def fp64_roofline(n_p, t_launch_s, rate):
    """FP64-pipe roofline of the FP64 form's push group (k_push_fp64 +
    k_cross_fp64): FP64 lane operations per launch (ncu count per particle,
    scaled to n_p) over the launch time, against the FP64 FMA rate measured
    in this run."""
    opp = _profile_value("fp64_lane_ops_per_particle", FP64_SUMMARY)
    if opp is None or t_launch_s <= 0 or not rate:
        return None
    achieved = opp * n_p / t_launch_s
    return {"kernel": "k_push_fp64 + k_cross_fp64", "bound": "fp64", "achieved": achieved, "peak": rate,
            "unit": "FP64 lane-ops/s", "frac": achieved / rate, "fp64_lane_ops_per_particle": opp,
            "peak_source": "fempic_measure_fp64_rate: independent FMA chains on every SM, this run"}


def large_leg(kind, steps, warmup, sort_every):
    """Forward step of the 64^3 jittered beam + plasma load (50M) or of the
    96^3 two-species load (400M), contract mixed form, particles drawn on the
    device; timed with CUDA events like the headline."""
    import torch
    from paper_2208_12795_gb300 import inputs as I
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    if kind == "jittered64":
        wl = I.workload_jittered64(n_particles=2)
        cols, table = I.device_beam_plasma(50_000_000, I.SEED_BASE + 30)
    else:
        wl = I.workload_large96(n_particles=2)
        cols, table = I.device_two_species(400_000_000, I.SEED_BASE + 50, vdtype=torch.float32)
    n = int(cols[0].numel())
    vel = [c.to(torch.float32) for c in cols[3:]]
    st = ParticleState(cols[0], cols[1], cols[2], vel[0], vel[1], vel[2], *table, track_crossings=False)
    del cols
    env = FempicEnv.from_mesh(wl.mesh, precision=1)
    env.locate(st)
    scratch = st.empty_like()
    env.sort(st, scratch)
    e = torch.from_numpy(wl.e_tilde).to(torch.complex64).cuda()
    b = torch.from_numpy(wl.b_tilde).to(torch.complex64).cuda()

    def step(k):
        t = k * wl.dt
        env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt)
        if sort_every > 0 and (k + 1) % sort_every == 0:
            env.sort(st, scratch)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    st0 = env.stats()
    env.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for k in range(warmup, warmup + steps):
        step(k)
    ev1.record()
    torch.cuda.synchronize()
    env.profile(False)
    ms = ev0.elapsed_time(ev1)
    prof = env.profile_read()
    st1 = env.stats()
    counts = (env.n_nodes, env.n_edges, env.n_faces, env.n_tets)
    b_alg = bytes_alg_per_step(n, counts, "mixed")
    peak = measured_peaks()[0]
    push = prof["push"]
    t_push = push["ms"] / max(push["launches"], 1) / 1e3
    out = {"workload": WORKLOAD_DESC[kind] + " (particles drawn on the device)", "form": "mixed",
           "value": n * steps / (ms / 1e3), "unit": "particle-steps/s", "steps": steps, "warmup": warmup,
           "ms_per_step": ms / steps, "algorithmic_bytes_per_step": b_alg,
           "hbm_frac_step": b_alg / (ms / steps / 1e3) / 1e9 / peak,
           "hbm_frac_push": b_alg / t_push / 1e9 / peak,
           "crossings_per_particle_step": (st1["crossings"] - st0["crossings"]) / (n * steps),
           "kernel_ms_per_step": {k: v["ms"] / steps for k, v in prof.items() if v["launches"]},
           "sort_every": sort_every}
    env.close()
    del st, scratch
    torch.cuda.empty_cache()
    return out


def config2_errors(wl, n_sub, steps):
    """Per-quantity error of the GPU forms against the FP64 oracle on the 48^3
    cube workload: the first n_sub particles for `steps` steps, same seeded
    inputs on both sides."""
    import torch
    from oracle.oracle import OracleMesh, OracleState, push_step as oracle_push
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    P = wl.particles.subset(n_sub)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    tet0, _ = om.locate(P.x, P.y, P.z)
    ost = OracleState(P, tet0)
    oG = np.zeros(om.n_edges)
    t0 = time.perf_counter()
    for k in range(steps):
        oracle_push(om, ost, wl.e_tilde, wl.b_tilde, wl.amp(k * wl.dt), wl.omega0, k * wl.dt, wl.dt, oG)
    t_or = time.perf_counter() - t0
    en = None
    res = {"workload": f"cube48 TE101 10 kV/m, first {n_sub} of the 10M electrons, {steps} steps "
                       f"(dt 0.5 ns, ramp sigma 20 ns)",
           "note": "positions in m (absolute), velocities relative; G_cum relative to max |G_cum|; a particle "
                   "whose FP32 trajectory passes within rounding of a face can take the other tet and then "
                   "sample other fields, which sets the max of the mixed forms",
           "oracle_s": t_or, "oracle_crossings_per_particle": float(ost.n_cross.mean())}
    for name, prec in (("fp64", 0), ("mixed", 1), ("mixed_q24", 2)):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        st = ParticleState.from_host(P, prec)
        env.locate(st)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
        rho0 = env.nodal_charge(st)
        for k in range(steps):
            t = k * wl.dt
            env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
            env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
        rho1 = env.nodal_charge(st).cpu().numpy()
        rho0 = rho0.cpu().numpy()
        g = st.to_numpy()
        Gg = G.cpu().numpy()
        if en is None:
            en = env.query()["edge_nodes"]
        div = np.zeros(env.n_nodes)
        np.add.at(div, en[:, 1], Gg)
        np.subtract.at(div, en[:, 0], Gg)
        er = np.sqrt((g["x"] - ost.x) ** 2 + (g["y"] - ost.y) ** 2 + (g["z"] - ost.z) ** 2)
        vr = np.sqrt(ost.vx ** 2 + ost.vy ** 2 + ost.vz ** 2)
        ev = np.sqrt((g["vx"] - ost.vx) ** 2 + (g["vy"] - ost.vy) ** 2 + (g["vz"] - ost.vz) ** 2) / vr
        gerr = np.abs(Gg - oG) / np.abs(oG).max()
        res[name] = {"r_err_max_m": float(er.max()), "r_err_p999_m": float(np.quantile(er, 0.999)),
                     "r_err_p99_m": float(np.quantile(er, 0.99)), "r_err_median_m": float(np.median(er)),
                     "v_rel_err_max": float(ev.max()), "v_rel_err_p999": float(np.quantile(ev, 0.999)),
                     "v_rel_err_p99": float(np.quantile(ev, 0.99)), "v_rel_err_median": float(np.median(ev)),
                     "tet_agreement": float((g["tet"] == ost.tet).mean()),
                     "particles_on_another_tet": int((g["tet"] != ost.tet).sum()),
                     "crossing_count_agreement": float((g["n_cross"] == ost.n_cross).mean()),
                     "G_cum_err_rel_max": float(gerr.max()), "G_cum_err_rel_p99": float(np.quantile(gerr, 0.99)),
                     "conservation_residual_rel": float(np.abs(div - (rho1 - rho0)).max() / np.abs(rho1).max())}
        env.close()
    return res


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_2208_12795_gb300 import build, inputs as I, shard
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    n_p = args.particles
    big_host = None
    if args.workload == "cube48":
        wl = I.te101_cavity(48, n_p, 5.0, 1e4, 100, 2 + 100 * rank, name="cube48_10M_te101")
        if world > 1:   # this rank's z-slab (a contiguous tet range) of the world x n_p global load
            wl = dataclasses.replace(wl, particles=shard.slab_load(wl.particles, rank, world))
    elif args.workload == "jittered64":
        n_p = args.particles if args.particles != 10_000_000 else 50_000_000
        wl = I.workload_jittered64(n_p)
        args.no_fp64 = True
    else:
        n_p = args.particles if args.particles != 10_000_000 else 400_000_000
        big_host = I.large96_species(n_p)
        wl = I.workload_large96(n_particles=2)          # mesh, DoFs, dt; particles streamed below
        args.no_fp64 = True
        args.no_cpu = True
    mesh = wl.mesh
    stream = torch.cuda.current_stream()

    def particle_state(prec):
        if big_host is None:
            return ParticleState.from_host(wl.particles, prec, track_crossings=False)
        sb, q, m, w, temp = big_host
        vdt = torch.float64 if prec == 0 else torch.float32
        arrs = [torch.empty(n_p, dtype=torch.float64, device="cuda") for _ in range(3)] + \
               [torch.empty(n_p, dtype=vdt, device="cuda") for _ in range(3)]
        chunk = 20_000_000
        for s in range(len(q)):
            for c0 in range(int(sb[s]), int(sb[s + 1]), chunk):
                c1 = min(int(sb[s + 1]), c0 + chunk)
                cols = I.maxwellian_chunk(I.SEED_BASE + 5 + 1000 * s, c0 // chunk, c1 - c0, temp, m[s])
                for a, col in zip(arrs, cols):
                    a[c0:c1].copy_(torch.from_numpy(np.ascontiguousarray(col)))
        return ParticleState(*arrs, sb, q, m, w, track_crossings=False)

    def timed_form(form):
        prec = {"mixed": 1, "mixed_q24": 2, "fp64": 0}[form]
        env = FempicEnv.from_mesh(mesh, precision=prec)
        st = particle_state(prec)
        env.locate(st)
        scratch = st.empty_like()
        env.sort(st, scratch)                 # initial tet-sorted layout (untimed)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        sharded = shard.ShardedDeposit(env) if world > 1 else None
        counts = (env.n_nodes, env.n_edges, env.n_faces, env.n_tets)

        def step(n):
            t = n * wl.dt
            env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
            if sharded is not None:   # local dG, all-reduced, added to every rank's G_cum
                sharded(wl.omega0, t + wl.dt)
            else:
                env.deposit(wl.omega0, t + wl.dt)
            if args.sort_every > 0 and (n + 1) % args.sort_every == 0:
                env.sort(st, scratch)

        for n in range(args.warmup):
            step(n)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.2)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        env.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for n in range(args.warmup, args.warmup + args.steps):
            step(n)
        ev1.record(stream)
        torch.cuda.synchronize()
        env.profile(False)
        if world > 1:
            dist.barrier()
        ck = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        prof = env.profile_read()
        stats = env.stats()
        res = dict(ms=ms, prof=prof, stats=stats, counts=counts, clocks=ck, env=env, st=st, e=e, b=b,
                   scratch=scratch)
        return res

    out = {}
    mixed = timed_form("mixed")
    out["mixed"] = mixed
    if not args.no_q24:
        q = timed_form("mixed_q24")
        out["mixed_q24"] = q
        q["env"].close()
        del q["st"], q["scratch"]
    if not args.no_fp64:
        f64 = timed_form("fp64")
        out["fp64"] = f64
        f64["env"].close()

    # e2e through the public API with host buffers: per step, the envelope
    # DoFs arrive from pinned host memory (the field solver's output) and the
    # step's edge deposit dG goes back to pinned host memory.  The copies run
    # on a copy stream into double buffers, ordered by events: step n+1's DoFs
    # come in while step n computes, and step n's dG goes out while step n+1
    # computes; every step's copies are inside the timed region.
    env, st = mixed["env"], mixed["st"]
    e_host = [torch.from_numpy(wl.e_tilde).to(torch.complex64).pin_memory() for _ in range(2)]
    b_host = [torch.from_numpy(wl.b_tilde).to(torch.complex64).pin_memory() for _ in range(2)]
    e_dev = [torch.empty_like(e_host[0], device="cuda") for _ in range(2)]
    b_dev = [torch.empty_like(b_host[0], device="cuda") for _ in range(2)]
    dG_dev = [torch.zeros(env.n_edges, dtype=torch.float64, device="cuda") for _ in range(2)]
    dG_host = [torch.zeros(env.n_edges, dtype=torch.float64).pin_memory() for _ in range(2)]
    h2d = e_host[0].numel() * 8 + b_host[0].numel() * 8
    d2h = dG_host[0].numel() * 8
    k0 = args.warmup + args.steps
    comp = torch.cuda.current_stream()
    copy_s = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    in_ready, in_free = [ev(), ev()], [ev(), ev()]
    out_ready, out_free = [ev(), ev()], [ev(), ev()]
    for k in range(2):
        in_free[k].record(comp)
        out_free[k].record(comp)

    def stage_in(n):
        k = n & 1
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(in_free[k])
            e_dev[k].copy_(e_host[k], non_blocking=True)
            b_dev[k].copy_(b_host[k], non_blocking=True)
            in_ready[k].record(copy_s)

    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    stage_in(k0)
    for n in range(k0, k0 + args.steps):
        t = n * wl.dt
        k = n & 1
        if n + 1 < k0 + args.steps:
            stage_in(n + 1)
        comp.wait_event(in_ready[k])
        env.push_step(st, e_dev[k], b_dev[k], wl.amp(t), wl.omega0, t, wl.dt)
        in_free[k].record(comp)
        comp.wait_event(out_free[k])
        if world > 1:
            env.deposit_local(dG_dev[k])
            dist.all_reduce(dG_dev[k])
            env.accumulate(wl.omega0, t + wl.dt, dG_dev[k])
        else:
            env.deposit(wl.omega0, t + wl.dt, dG_out=dG_dev[k])
        out_ready[k].record(comp)
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(out_ready[k])
            dG_host[k].copy_(dG_dev[k], non_blocking=True)
            out_free[k].record(copy_s)
        if args.sort_every > 0 and (n + 1) % args.sort_every == 0:
            env.sort(st, mixed["scratch"])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    mixed["e2e_s"] = e2e_s
    mixed["h2d"], mixed["d2h"] = h2d, d2h

    # The same step with the envelope interpolated in time from three DoF
    # levels (t_{n-1}, t_n, t_{n+1}, a field step of 21 fine steps), device
    # resident: only the per-tet field construction reads the extra levels.
    lv3 = None
    if not args.no_levels3:
        from paper_2208_12795_gb300 import capi
        e0 = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b0 = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        e_lv = [e0 * s for s in (0.98, 1.0, 1.02)]
        b_lv = [b0 * s for s in (0.98, 1.0, 1.02)]
        k1 = k0 + args.steps
        mid = (k1 + args.steps // 2) * wl.dt
        tau = (mid - 21 * wl.dt, mid, mid + 21 * wl.dt)

        def step3(n):
            t = n * wl.dt
            env.push_step3(st, e_lv, b_lv, capi.fempic_lagrange3(tau, t), wl.amp(t), wl.omega0, t, wl.dt)
            if world > 1:
                env.deposit_local(dG_dev)
                dist.all_reduce(dG_dev)
                env.accumulate(wl.omega0, t + wl.dt, dG_dev)
            else:
                env.deposit(wl.omega0, t + wl.dt)
            if args.sort_every > 0 and (n + 1) % args.sort_every == 0:
                env.sort(st, mixed["scratch"])

        for n in range(k1, k1 + 3):
            step3(n)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        env.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for n in range(k1 + 3, k1 + 3 + args.steps):
            step3(n)
        ev1.record(stream)
        torch.cuda.synchronize()
        env.profile(False)
        ms3 = ev0.elapsed_time(ev1)
        if world > 1:
            tt = torch.tensor([ms3], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms3 = float(tt.item())
        pr3 = env.profile_read()
        lv3 = {"value": n_p * world * args.steps / (ms3 / 1e3), "unit": "particle-steps/s",
               "ms_per_step": ms3 / args.steps, "field_ms_per_step": pr3["field"]["ms"] / args.steps,
               "field_ms_per_step_one_level": mixed["prof"]["field"]["ms"] / args.steps,
               "what": "fempic_push_step3: envelope interpolated from 3 DoF levels with second-order "
                       "Lagrange weights at each fine step (field step = 21 fine steps)"}
    mixed["levels3"] = lv3
    env.close()

    # The downshifted integrator (Sec. III-D: M/L velocity rule, AB4
    # positions) on the FP64 form and on the contract mixed form, device
    # resident, after the other legs; the set is re-sorted on its cadence with
    # the history planes carried through the same permutation (Downshift.sort).
    def downshift_leg(prec):
        env_d = FempicEnv.from_mesh(mesh, precision=prec)
        st_d = particle_state(prec)
        env_d.locate(st_d)
        env_d.sort(st_d, st_d.empty_like())
        ds = Downshift(env_d, st_d.n)
        scratch_d = st_d.empty_like()
        # a re-sort also gathers the 33 history planes, against a step of
        # several ms: every 4x the push step's cadence
        ds_sort = 4 * args.sort_every
        e_d = torch.from_numpy(wl.e_tilde).to(env_d.dof_dtype).cuda()
        b_d = torch.from_numpy(wl.b_tilde).to(env_d.dof_dtype).cuda()
        dG_d = torch.zeros(env_d.n_edges, dtype=torch.float64, device="cuda")

        def step_ds(n):
            t = n * wl.dt
            ds.step(st_d, e_d, b_d, wl.amp(t), wl.omega0, t, wl.dt)
            if world > 1:
                env_d.deposit_local(dG_d)
                dist.all_reduce(dG_d)
                env_d.accumulate(wl.omega0, t + wl.dt, dG_d)
            else:
                env_d.deposit(wl.omega0, t + wl.dt)
            if ds_sort > 0 and (n + 1) % ds_sort == 0:
                ds.sort(st_d, scratch_d)

        for n in range(max(3, args.warmup)):
            step_ds(n)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        env_d.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for n in range(max(3, args.warmup), max(3, args.warmup) + args.steps):
            step_ds(n)
        ev1.record(stream)
        torch.cuda.synchronize()
        env_d.profile(False)
        ms_d = ev0.elapsed_time(ev1)
        if world > 1:
            tt = torch.tensor([ms_d], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms_d = float(tt.item())
        pr = env_d.profile_read()
        env_ms = pr["field"]["ms"] + pr["push"]["ms"]
        sort_ms = pr["sort"]["ms"]
        counts_d = (env_d.n_nodes, env_d.n_edges, env_d.n_faces, env_d.n_tets)
        form = "fp64" if prec == 0 else "mixed"
        b_ds = bytes_alg_per_step_downshift(n_p, counts_d, form)
        t_step = ms_d / args.steps / 1e3
        rec = {
            "value": n_p * world * args.steps / (ms_d / 1e3), "unit": "particle-steps/s",
            "ms_per_step": ms_d / args.steps,
            "env_step_ms_per_step": env_ms / args.steps,
            "downshift_kernels_ms_per_step": (ms_d - env_ms - sort_ms - pr["finalize"]["ms"]) / args.steps,
            "sort_ms_per_step": sort_ms / args.steps,
            "sort_every": ds_sort,
            "algorithmic_bytes_per_step": b_ds,
            "hbm_frac_of_step": b_ds / t_step / 1e9 / measured_peaks()[0],
            "what": f"fempic_push_step_downshift ({'FP64' if prec == 0 else 'contract mixed form: FP32 rule, samples and history'}): "
                    "envelope samples + M/L velocity rule + AB4 (k_ds_pre), the env's step under a zero field "
                    "for tracking/deposit, wall mirrors of the history (k_ds_post); re-sorted with the history "
                    "carried along (sort_ms_per_step: the particle sort; the plane gather is in the step time)"}
        ds.close()
        env_d.close()
        del st_d, ds, scratch_d
        return rec

    if not args.no_downshift and args.workload == "cube48":
        out["downshift"] = downshift_leg(0)
        out["downshift_mixed"] = downshift_leg(1)

    adj = None if (args.no_adjoint or args.workload != "cube48") else adjoint_window(rank)
    if args.workload == "cube48" and not args.no_errors:
        out["errors"] = config2_errors(wl, 100_000, 100)
    if args.workload == "cube48" and not args.no_large and world == 1:
        own = {"jittered64": 50, "large96": 20}
        out["large"] = {k: large_leg(k, args.large_steps or own[k], 2, args.sort_every) for k in own}
        if not args.no_adjoint:
            out["large_adjoint"] = large_adjoint_leg(args.large_steps or own["large96"])
    from paper_2208_12795_gb300 import capi as _capi
    out["fp64_rate"] = _capi.fempic_measure_fp64_rate(torch.cuda.current_stream().cuda_stream)
    if rank == 0:
        cpu = None if (args.no_cpu or world > 1) else cpu_baseline(wl, args.cpu_particles, args.cpu_steps)
        if cpu is not None and args.workload == "cube48" and not args.no_cpu_parallel:
            cpu["all_cores"] = cpu_baseline_parallel(wl, 4 * args.cpu_particles, args.cpu_steps)
        report(args, world, n_p, out, cpu, adj)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def adjoint_window(rank):
    """Gradient of the kinetic energy after K = 50 steps on the 48^3 cube with
    4M electrons at 5 eV, checkpoints every 10 (the differentiation
    workload): forward with checkpoints, then the reverse sweep (segment
    recompute + adjoint steps), both forms, timed with CUDA events."""
    import torch
    from paper_2208_12795_gb300 import adjoint as A, inputs as I
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    wl = I.workload_adjoint48()
    res = {}
    for form, prec in (("mixed", 1), ("fp64", 0)):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        counts = (env.n_nodes, env.n_edges, env.n_faces, env.n_tets)
        st0 = ParticleState.from_host(wl.particles, prec, track_crossings=False)
        env.locate(st0)
        sc = st0.empty_like()
        env.sort(st0, sc)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        sch = A.Schedule(wl.amp, wl.omega0, wl.dt, wl.steps, 10)
        A.kinetic_energy_and_grad(env, st0, e, b, A.Schedule(wl.amp, wl.omega0, wl.dt, 4, 2))   # warm-up
        torch.cuda.synchronize()
        env.profile(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        final, ckpts = A.forward_checkpointed(env, st0, e, b, sch)
        ev[1].record()
        vdt = torch.float64 if prec == 0 else torch.float32
        adj = A.AdjointState(st0.n, vdt)
        A.kinetic_energy(env, final, seed=adj)
        A.reverse_sweep(env, ckpts, e, b, sch, adj)
        ev[2].record()
        torch.cuda.synchronize()
        t_fwd, t_rev = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
        prof = env.profile_read()
        env.profile(False)
        units = st0.n * sch.steps
        res[form] = {"forward_particle_steps_per_s": units / t_fwd,
                     "reverse_particle_steps_per_s": units / t_rev,
                     "gradient_window_s": t_fwd + t_rev,
                     "kernel_ms": {k: v["ms"] for k, v in prof.items() if v["launches"]}}
        env.close()
    return {"workload": "cube48_4M_adjoint: 48^3x6 cube, 4M electrons at 5 eV, TE101 10 kV/m, K=50, "
                        "checkpoint every 10; loss = kinetic energy after K steps",
            "unit": "particle-steps/s", "particles": wl.particles.n, "counts": counts, "steps": wl.steps,
            "every": 10, **res}


def large_adjoint_leg(steps):
    """Gradient window on the 96^3 two-species load (400M particles, contract
    mixed form): kinetic energy after `steps` steps, gradients with respect
    to the DoFs and the initial phase space.  adjoint.plan_window picks the
    checkpoint interval and the reverse mode for 85% of the device memory
    free once the load is resident; the plan's predicted peak is reported
    beside the allocator's measured one."""
    import torch
    from paper_2208_12795_gb300 import adjoint as A, inputs as I
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    wl = I.workload_large96(n_particles=2)
    cols, table = I.device_two_species(400_000_000, I.SEED_BASE + 50, vdtype=torch.float32)
    n = int(cols[0].numel())
    vel = [c.to(torch.float32) for c in cols[3:]]
    st0 = ParticleState(cols[0], cols[1], cols[2], vel[0], vel[1], vel[2], *table, track_crossings=False)
    del cols, vel
    env = FempicEnv.from_mesh(wl.mesh, precision=1)
    counts = (env.n_nodes, env.n_edges, env.n_faces, env.n_tets)
    env.locate(st0)
    sc = st0.empty_like()
    env.sort(st0, sc)
    del sc
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    S, Ab = A.state_nbytes(st0), n * (3 * 8 + 3 * 4)
    plan = A.plan_window(n, steps, S, Ab, int(0.85 * free))
    A.kinetic_energy_and_grad(env, st0, e, b, A.Schedule(wl.amp, wl.omega0, wl.dt, 2, 1))   # warm-up
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    sch = A.Schedule(wl.amp, wl.omega0, wl.dt, steps, plan.every, stash=plan.stash)
    env.profile(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    final, ckpts = A.forward_checkpointed(env, st0, e, b, sch)
    ev[1].record()
    adj = A.AdjointState(n, torch.float32)
    A.kinetic_energy(env, final, seed=adj)
    del final
    A.reverse_sweep(env, ckpts, e, b, sch, adj)
    ev[2].record()
    torch.cuda.synchronize()
    prof = env.profile_read()
    env.profile(False)
    peak_meas = torch.cuda.max_memory_allocated() - base
    t_fwd, t_rev = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    hbm = measured_peaks()[0]
    fb = bytes_alg_per_step(n, counts, "mixed")
    rb = bytes_reverse_window(n, counts, "mixed", steps, plan.every, plan.stash, plan.recompute_steps)
    out = {"workload": WORKLOAD_DESC["large96"] + f" (particles drawn on the device); loss = kinetic energy "
                       f"after K={steps} steps",
           "form": "mixed", "unit": "particle-steps/s", "particles": n, "steps": steps,
           "forward_particle_steps_per_s": n * steps / t_fwd,
           "reverse_particle_steps_per_s": n * steps / t_rev,
           "gradient_window_s": t_fwd + t_rev,
           "hbm_frac_forward": fb * steps / t_fwd / 1e9 / hbm,
           "hbm_frac_reverse": rb / t_rev / 1e9 / hbm,
           "bytes_per_particle_step_forward": fb / n,
           "bytes_per_particle_step_reverse": rb / (n * steps),
           "memory_plan": {"every": plan.every, "stash": plan.stash, "recompute_steps": plan.recompute_steps,
                           "budget_gb": 0.85 * free / 1e9, "predicted_peak_gb": plan.peak_bytes / 1e9,
                           "measured_peak_gb": peak_meas / 1e9, "state_gb": S / 1e9, "adjoint_gb": Ab / 1e9},
           "kernel_ms": {k: v["ms"] for k, v in prof.items() if v["launches"]}}
    env.close()
    del st0, ckpts, adj
    torch.cuda.empty_cache()
    return out


def cpu_baseline(wl, n_sample, steps):
    """The FP64 oracle as it stands, single thread, on the first n_sample
    particles of the same workload."""
    from oracle.oracle import OracleMesh, OracleState, push_step as oracle_push
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles.subset(n_sample)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    t0 = time.perf_counter()
    for n in range(steps):
        oracle_push(om, st, wl.e_tilde, wl.b_tilde, wl.amp(n * wl.dt), wl.omega0, n * wl.dt, wl.dt, G)
    el = time.perf_counter() - t0
    return {"value": n_sample * steps / el, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_sample} of the 10M particles, {steps} steps, FP64 C oracle, 1 thread "
                      f"({el:.1f} s)"}


_BARRIER = None


def _init_worker(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_chunk(job):
    """Worker of the parallel CPU baseline: the oracle as it stands on one
    slice of the particles; all workers start their step loops together (a
    barrier after the set-up); returns the wall-clock interval of the loop."""
    nodes, tets, lo, hi, cols, sb, q, m, w, e, b, amps, omega0, dt = job
    from oracle.oracle import OracleMesh, OracleState, push_step as oracle_push
    from paper_2208_12795_gb300.inputs import Particles
    om = OracleMesh(nodes, tets, lo, hi)
    P = Particles(*cols, sb, q, m, w)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    _BARRIER.wait(timeout=900)
    t0 = time.time()
    for n, a in enumerate(amps):
        oracle_push(om, st, e, b, a, omega0, n * dt, dt, G)
    return t0, time.time()


def cpu_baseline_parallel(wl, n_sample, steps):
    """The FP64 oracle as it stands, one process per host core (spawned), each
    on its slice of the first n_sample particles; the rate is all processes'
    particle-steps over the wall-clock span of their step loops."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    P = wl.particles
    amps = [wl.amp(n * wl.dt) for n in range(steps)]
    bounds = np.linspace(0, n_sample, cores + 1).astype(np.int64)
    jobs = []
    for c in range(cores):
        a, z = int(bounds[c]), int(bounds[c + 1])
        cols = [np.ascontiguousarray(x[a:z]) for x in (P.x, P.y, P.z, P.vx, P.vy, P.vz)]
        jobs.append((wl.mesh.nodes, wl.mesh.tets, wl.mesh.lo, wl.mesh.hi, cols, np.array([0, z - a], np.int64),
                     P.q, P.m, P.w, wl.e_tilde, wl.b_tilde, amps, wl.omega0, wl.dt))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    with ctx.Pool(cores, initializer=_init_worker, initargs=(barrier,)) as pool:
        spans = pool.map(_oracle_chunk, jobs, chunksize=1)
    el = max(t1 for _, t1 in spans) - min(t0 for t0, _ in spans)
    return {"value": n_sample * steps / el, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample} of the 10M particles in {cores} slices, {steps} steps, FP64 C oracle, "
                      f"one spawned process per core ({el:.1f} s span of the step loops)"}


def report(args, world, n_p, out, cpu, adj=None):
    peak, peak_src = measured_peaks()
    m = out["mixed"]
    K = args.steps
    total = n_p * world * K
    value = total / (m["ms"] / 1e3)
    push = m["prof"]["push"]
    t_push = push["ms"] / max(push["launches"], 1) / 1e3
    b_alg = bytes_alg_per_step(n_p, m["counts"], "mixed")
    achieved = b_alg / t_push / 1e9
    launches = sum(v["kernels"] for v in m["prof"].values())
    traffic = profiled_traffic(n_p)
    rec = {
        "metric": METRIC,
        "value": value,
        "unit": "particle-steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": m["ms"] / K,
        "value_without_sort": total / ((m["ms"] - m["prof"]["sort"]["ms"]) / 1e3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64 mixed (FP32 gather/carrier/Boris; FP64 positions; FP64-accurate exit parameter, "
                 "crossing barycentrics and deposit; FP64 edge accumulation)",
        "data": DATA_DESC[args.workload],
        "config": {
            "workload": WORKLOAD_DESC[args.workload],
            "form": "mixed",
            "particles_per_gpu": n_p,
            "n_tets": m["counts"][3],
            "sort_every": 4 * args.sort_every,
            "l2": f"inputs larger than L2 (particle SoA {n_p * 41 / 1e6:.0f} MB per GPU per step)",
            "parallelism": f"particles sharded by tet range over {world} GPUs, dG all-reduced" if world > 1 else "1 GPU",
        },
        "roofline": {
            "kernel": "push step group: k_push_mixed_tma (+ k_push_mixed ragged tail) + k_cross_df",
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "peak_source": f"{peak_src} copy bandwidth",
            "algorithmic_bytes_per_launch": b_alg,
            "avg_launch_ms": t_push * 1e3,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "frac_step": b_alg / (m["ms"] / K / 1e3) / 1e9 / peak,
            "frac_step_note": "whole step (field, push group, finalize, sort amortised) on the same "
                              "algorithmic bytes",
        },
        "e2e": {"value": total / m["e2e_s"], "unit": "particle-steps/s",
                "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"]},
        "roofline_issue": issue_roofline(
            n_p, (push["ms"] - m["prof"]["cross"]["ms"]) / max(push["launches"], 1) / 1e3,
            float(m["clocks"].get("sm_mhz") or 2070.0)),
        "gpu_launches": launches,
        "kernel_ms": {k: v["ms"] for k, v in m["prof"].items() if v["launches"]},
        "kernel_ms_note": "summed CUDA-event time over the timed steps per library call; 'cross' "
                          "(k_cross_df, or k_cross_q24 in the 24-bit variant) is part of 'push'",
        "crossings_per_particle_step": m["stats"]["crossings"] / max(1, n_p * (K + args.warmup)),
        "clocks": m["clocks"],
    }
    if "fp64" in out:
        f = out["fp64"]
        fp = f["prof"]["push"]
        tf = fp["ms"] / max(fp["launches"], 1) / 1e3
        bf = bytes_alg_per_step(n_p, f["counts"], "fp64")
        rec["fp64_form"] = {"value": total / (f["ms"] / 1e3), "ms_per_step": f["ms"] / K,
                            "push_avg_launch_ms": tf * 1e3, "hbm_frac": bf / tf / 1e9 / peak,
                            "roofline_fp64": fp64_roofline(n_p, tf, out.get("fp64_rate")),
                            "clocks": f["clocks"]}
    if "mixed_q24" in out:
        q = out["mixed_q24"]
        qp = q["prof"]["push"]
        tq = qp["ms"] / max(qp["launches"], 1) / 1e3
        rec["mixed_q24"] = {"value": total / (q["ms"] / 1e3), "ms_per_step": q["ms"] / K,
                            "push_avg_launch_ms": tq * 1e3, "hbm_frac_push": b_alg / tq / 1e9 / peak,
                            "hbm_frac_step": b_alg / (q["ms"] / K / 1e3) / 1e9 / peak,
                            "kernel_ms": {k: v["ms"] for k, v in q["prof"].items() if v["launches"]},
                            "what": "FEMPIC_MIXED_Q24: tracking and deposit on 24-bit integer barycentrics "
                                    "(exit parameter FP32, deposit exact in int64 at 2^-24 of a tet)"}
    if m.get("levels3") is not None:
        rec["levels3"] = m["levels3"]
    if "downshift" in out:
        rec["downshift"] = out["downshift"]
    if "downshift_mixed" in out:
        rec["downshift_mixed"] = out["downshift_mixed"]
    if adj is not None:
        # HBM fractions of the gradient window: forward steps on the forward
        # algorithmic bytes, the reverse sweep on bytes_reverse_window
        counts = adj.get("counts", (0, 0, 0, 0))
        n_adj = adj.get("particles", 0)
        for form in ("mixed", "fp64"):
            r = adj.get(form)
            if not r or not n_adj:
                continue
            K = adj["steps"]
            fb = bytes_alg_per_step(n_adj, counts, form) / n_adj
            rb = bytes_reverse_window(n_adj, counts, form, K, adj["every"], True, K) / (n_adj * K)
            r["bytes_per_particle_step_forward"] = fb
            r["bytes_per_particle_step_reverse"] = rb
            r["hbm_frac_forward"] = r["forward_particle_steps_per_s"] * fb / 1e9 / peak
            r["hbm_frac_reverse"] = r["reverse_particle_steps_per_s"] * rb / 1e9 / peak
        rec["adjoint"] = adj
    if "errors" in out:
        rec["mixed_error_vs_oracle"] = out["errors"]
    if "large" in out:
        rec["large_forward"] = out["large"]
    if "large_adjoint" in out:
        rec["large_adjoint"] = out["large_adjoint"]
    if out.get("fp64_rate"):
        rec["fp64_rate_lane_ops_per_s"] = out["fp64_rate"]
    if cpu is not None:
        rec["cpu_baseline"] = cpu
    print(json.dumps(rec), flush=True)


# --------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle timed as it stands on the host cores: each step is one
    oracle step over a bounded sample of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.oracle import OracleMesh, OracleState, push_step as oracle_push
    from paper_2208_12795_gb300 import inputs as I
    n_s = 20_000
    wl = I.te101_cavity(48, n_s, 5.0, 1e4, 100, 2, name="cube48_10M_te101")
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    for n in range(args.warmup):
        oracle_push(om, st, wl.e_tilde, wl.b_tilde, wl.amp(n * wl.dt), wl.omega0, n * wl.dt, wl.dt, G)
    t0 = time.perf_counter()
    for n in range(args.warmup, args.warmup + args.steps):
        oracle_push(om, st, wl.e_tilde, wl.b_tilde, wl.amp(n * wl.dt), wl.omega0, n * wl.dt, wl.dt, G)
    el = time.perf_counter() - t0
    value = n_s * args.steps / el
    sample = f"{n_s} particles of the same workload per step, FP64 C oracle, 1 thread"
    rec = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded)",
           "config": {"workload": "cube48_10M_te101: 48^3x6 Kuhn cube (663,552 tets), 5 eV electrons, "
                                  "TE101 10 kV/m, dt 0.5 ns", "form": "oracle", "sample": sample},
           "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
