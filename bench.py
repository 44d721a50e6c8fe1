#!/usr/bin/env python
"""QED particle-steps/s of the spin/polarization-resolved SF-QED step on one GB300.

Workload (config 2): 1e6 electrons, gamma ~ N(2e4, 5%), transverse and longitudinal rms
1 um, spins uniform on the sphere, head-on with a circularly polarised paraxial Gaussian
pulse (a0 = 100, w0 = 3 um, 10-cycle sin^2 envelope); NCS + NBW + VB + T-BMT with photon
and pair compaction every step; dt = T0/200.  The beam starts 150 steps before its centre
meets the pulse centre at the focus; those 150 steps run untimed (they populate photons
and pairs), then W warm-up steps, then K timed steps.  A "step" is one qed_step over all
live e-, e+ and photons; the metric counts every live particle of every step.

Timing: CUDA events on the library's stream around each step, L2 flushed (256 MB write)
before every timed step; per-kernel durations from the library's timing hook; clocks
sampled with nvidia-smi during the timed loop.  The mixed path (headline) and the plain
FP64 path run the same workload.  e2e: the host-buffer entry point (qed_step_host) with
pinned host arrays, copies included.  cpu_baseline / --impl reference: the FP64 oracle
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QED particle-steps/s: mixed vs FP64 GPU at matched spectra; HBM % of peak"
PRE_STEPS = 150
T_SHIFT = 8.5 * math.pi


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def c2_workload(n, seed):
    import workloads
    wl = workloads.c2(n=n, seed=seed)
    wl["e"]["z"] = wl["e"]["z"] + T_SHIFT
    wl["t0"] = T_SHIFT
    wl["step0"] = int(round(T_SHIFT / wl["dt"]))
    return wl


# algorithmic bytes per particle-step (state that must be read and written)
#   photon pass: read x,y,z + k + xi + theta + id, write x,y,z + xi + theta
#   lepton pass: read x,y,z + p + S + id, write x,y,z + p + S
BYTES = {
    "mixed": {"lep": 104, "ph": 100, "ncs_birth": 68, "nbw_birth": 120},
    "f64": {"lep": 152, "ph": 144, "ncs_birth": 104, "nbw_birth": 176},
}

# DRAM bytes per unit (dram__bytes_read.sum + dram__bytes_write.sum of one launch divided
# by the particles it processed) from the ncu traffic capture of the streaming passes kept
# under profiles/; scaled to a launch by its particle count.  Must be re-captured whenever
# either streaming kernel changes.
TRAFFIC_PER_UNIT = {"k_photon": 85.74, "k_lepton": 63.92}


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed loop runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.out = os.path.join("/tmp", f"qed_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.out):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 8:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def replica_seed(rank):
    """seed of the 1e6-electron workload on a rank: replicas are independent collisions"""
    return 2 + rank


def aggregate(torch, dist, device, ms, parts):
    """whole-job timing over replicas: the slowest rank's time and every rank's particle-steps
    (identity without a process group)"""
    if dist is None:
        return ms, parts
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([parts], device=device, dtype=torch.float64)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def run_gpu_path(q, torch, wl, prec, steps, warmup, flush, flags, kernel_steps, pre=PRE_STEPS, caps=None,
                 before=None):
    """Pre-run, warm up, time `steps` steps (the headline), then `kernel_steps` more steps
    with the library's per-kernel timing on (kernels serialised, event records and a sync
    inside every step, so they are kept out of the headline loop)."""
    n = len(wl["e"]["id"])
    caps = caps or {"cap_e": n + 4_000_000, "cap_p": 4_000_000, "cap_ph": 40 * n}
    sim = q.Simulation(wl, prec=prec, **caps)
    stream = torch.cuda.current_stream()
    sim.run(pre, flags)
    if before is not None:
        before(sim)
    sim.run(warmup, flags)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(nsteps):
        tot_ms, parts, lep, ph, ncs_b, nbw_b = 0.0, 0, 0, 0, 0, 0
        for _ in range(nsteps):
            ne, npos, nph = sim.e.count(), sim.pos.count(), sim.ph.count()
            parts += ne + npos + nph
            lep += ne + npos
            ph += nph
            flush.zero_()
            s0 = sim.stats.clone()
            ev0.record(stream)
            q.qed_step(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, sim.fields, sim.t, sim.dt,
                       sim.seed, sim.step_no, flags, sim.stats.data_ptr())
            ev1.record(stream)
            ev1.synchronize()
            tot_ms += ev0.elapsed_time(ev1)
            d = (sim.stats - s0).cpu().numpy()
            ncs_b += int(d[0] + d[1])
            nbw_b += int(d[2])
            sim.t += sim.dt
            sim.step_no += 1
        return {"ms": tot_ms, "particles": parts, "lep_units": lep, "ph_units": ph, "ncs_births": ncs_b,
                "nbw_births": nbw_b}

    info = timed(steps)
    info["status"] = sim.status()
    info["final_counts"] = (sim.e.count(), sim.pos.count(), sim.ph.count())
    q.qed_set_timing(sim.ctx, True)
    q.qed_get_timing(sim.ctx)
    kinfo = timed(kernel_steps)
    kms, ksteps = q.qed_get_timing(sim.ctx)
    q.qed_set_timing(sim.ctx, False)
    kinfo.update({"kernel_ms": kms, "kernel_steps": ksteps})
    info["kern"] = kinfo
    return sim, info


C3_N, C3_PRE = 30_000_000, 20
C3_GRID_BYTES = 6 * 4096 * 2048 * 4   # the six FP32 Yee components


def run_c3(q, torch, steps, warmup, flush, f64_steps, kernel_steps):
    """Grid-gathered fields: 3e7 electrons (gamma0 = 4000, tile-sorted) in a 4096 x 2048
    FP32 Yee snapshot of an a0 = 150 pulse reflected off a dense slab, TSC gather, NCS + NBW
    with spins; dt = T0/64.  C3_PRE untimed steps populate photons, then the same timing as
    the headline (L2 flushed before every step; the grid alone is 201 MB > L2)."""
    import workloads
    wl = workloads.c3(n=C3_N, seed=3)
    flags = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
    caps = {"cap_e": C3_N + 4_000_000, "cap_p": 4_000_000, "cap_ph": 60_000_000}
    out = {"workload": "c3_grid_4096x2048_yee_tsc_a150_g4000", "electrons": C3_N, "pre_steps": C3_PRE,
           "unit": "particle-steps/s"}
    b = BYTES["mixed"]
    for name, prec, nsteps in (("mixed", q.QED_PREC_MIXED, steps), ("f64", q.QED_PREC_F64, f64_steps)):
        if nsteps <= 0:
            continue
        sim, info = run_gpu_path(q, torch, wl, prec, nsteps, warmup, flush, flags,
                                 kernel_steps if name == "mixed" else 0, pre=C3_PRE, caps=caps)
        v = info["particles"] / (info["ms"] * 1e-3)
        r = {"value": v, "ms_per_step": info["ms"] / nsteps, "steps": nsteps, "status": info["status"],
             "counts_after": info["final_counts"]}
        kn = info["kern"]
        if name == "mixed" and kn["kernel_steps"]:
            ks = kn["kernel_steps"]
            k_ph_ms, k_lep_ms, k_ev_ms = kn["kernel_ms"]
            lep_bytes = kn["lep_units"] * b["lep"] + kn["ncs_births"] * b["ncs_birth"] + ks * C3_GRID_BYTES
            ph_bytes = kn["ph_units"] * b["ph"] + kn["nbw_births"] * b["nbw_birth"]
            r["kernels"] = {"steps": ks, "k_lepton_ms": k_lep_ms / ks, "k_photon_ms": k_ph_ms / ks,
                            "event_kernels_ms": k_ev_ms / ks,
                            "k_lepton_GBs": lep_bytes / (k_lep_ms * 1e-3) / 1e9 if k_lep_ms else None,
                            "k_photon_GBs": ph_bytes / (k_ph_ms * 1e-3) / 1e9 if k_ph_ms else None,
                            "leptons_per_launch": kn["lep_units"] / ks, "photons_per_launch": kn["ph_units"] / ks,
                            "bytes_note": "k_lepton counts 104 B per lepton plus the whole 201 MB grid once"}
        out[name] = r
        sim.close()
    if "mixed" in out and "f64" in out:
        out["speedup_mixed"] = out["mixed"]["value"] / out["f64"]["value"]
    # the same electrons sorted by cell on the device (qed_sort_cells, what a PIC code does
    # every few steps): the grid gather's loads of a warp then share cache lines
    if steps > 0:
        sort_ms = []
        sim, info = run_gpu_path(q, torch, wl, q.QED_PREC_MIXED, steps, warmup, flush, flags, kernel_steps,
                                 pre=C3_PRE, caps=caps, before=lambda s: sort_ms.append(timed_sort(q, torch, s)))
        kn = info["kern"]
        ks = max(kn["kernel_steps"], 1)
        resort = timed_sort(q, torch, sim)   # steady state: after the timed steps' drift, scratch in place
        ms_s = info["ms"] / steps
        out["mixed_cell_sorted"] = {"value": info["particles"] / (info["ms"] * 1e-3),
                                    "ms_per_step": ms_s, "steps": steps, "status": info["status"],
                                    "k_lepton_ms": kn["kernel_ms"][1] / ks, "k_photon_ms": kn["kernel_ms"][0] / ks,
                                    "sort_ms": resort, "sort_first_call_ms": sort_ms[0],
                                    "sorting_every_20_steps_ms_per_step": ms_s + resort / 20.0,
                                    "note": "electrons sorted by qed_sort_cells after the untimed steps (first call: "
                                            "with its scratch allocation); sort_ms re-sorts after the timed steps"}
        if "mixed" in out:
            out["mixed_cell_sorted"]["sorting_every_20_steps_wins"] = \
                ms_s + resort / 20.0 < out["mixed"]["ms_per_step"]
        sim.close()
    return out


def timed_sort(q, torch, sim):
    """qed_sort_cells of the electrons, timed with CUDA events (ms)."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    q.qed_sort_cells(sim.ctx, sim.e.handle, sim.fields)
    ev1.record()
    ev1.synchronize()
    return ev0.elapsed_time(ev1)


def run_pic(q, torch, steps, warmup):
    """Self-consistent PIC around the step: the 3e7-electron grid workload (4096 x 2048
    cells, fields evolved by the Yee solver from the reflected-pulse snapshot, bounded
    grid) with Esirkepov deposition of every lepton move, NCS + NBW + VB + T-BMT, mixed
    path.  Per step: FDTD_B(dt/2), qed_step(... | QED_F_DEPOSIT), FDTD_B(dt/2), FDTD_E(dt).
    Macro-particle weight 0.01 (about 1 n_c).  The field solver's own rate is timed apart:
    132 B per cell and step (two B halves of 36 B, one E update of 60 B incl. J)."""
    import numpy as np
    import workloads
    wl = workloads.c3(n=C3_N, seed=3)
    g = wl["grid"]
    ny, nx = g["Ey"].shape
    wl["e"]["w"] = np.full(C3_N, 0.01)
    flags = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
    sim = q.PicSimulation(wl, nx, ny, g["dx"], g["dy"], periodic=0,
                          fields={k: g[k] for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}, prec=q.QED_PREC_MIXED,
                          cap_e=C3_N + 4_000_000, cap_p=4_000_000, cap_ph=60_000_000)
    sim.run(C3_PRE + warmup, flags)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_run():
        p0 = int(sim.stats[6].item())
        ev0.record()
        sim.run(steps, flags)
        ev1.record()
        ev1.synchronize()
        return ev0.elapsed_time(ev1), int(sim.stats[6].item()) - p0

    ms, parts = timed_run()
    # then the run continued after sorting the electrons by cell (a PIC code sorts every few
    # steps): a tile's 256 electrons then cover a few rows of cells, so its deposition window
    # and the global atomics that flush it shrink
    sort_first = timed_sort(q, torch, sim)
    ms_s, parts_s = timed_run()
    sort_ms = timed_sort(q, torch, sim)   # steady state: after the drift of the timed steps
    reps = 20
    ev0.record()
    for _ in range(reps):
        q.qed_fdtd_advance(sim.g, q.QED_FDTD_B, 0.5 * sim.dt)
        q.qed_fdtd_advance(sim.g, q.QED_FDTD_B, 0.5 * sim.dt)
        q.qed_fdtd_advance(sim.g, q.QED_FDTD_E, sim.dt)
    ev1.record()
    ev1.synchronize()
    fd_ms = ev0.elapsed_time(ev1) / reps
    out = {"workload": "c3 grid 4096x2048 + Yee solver + Esirkepov deposition, 3e7 electrons",
           "value": parts / (ms * 1e-3), "unit": "particle-steps/s", "ms_per_step": ms / steps, "steps": steps,
           "fdtd_ms_per_step": fd_ms, "fdtd_GBs": 132.0 * nx * ny / (fd_ms * 1e-3) / 1e9,
           "counts_after": (sim.e.count(), sim.pos.count(), sim.ph.count()), "status": sim.status(),
           "cell_sorted": {"value": parts_s / (ms_s * 1e-3), "ms_per_step": ms_s / steps, "steps": steps,
                           "sort_ms": sort_ms, "sort_first_call_ms": sort_first,
                           "sorting_every_20_steps_ms_per_step": ms_s / steps + sort_ms / 20.0,
                           "sorting_every_20_steps_wins": ms_s / steps + sort_ms / 20.0 < ms / steps,
                           "note": "the same run continued after one qed_sort_cells of the electrons (first call: "
                                   "with its scratch allocation); sort_ms re-sorts after those steps"}}
    sim.close()
    return out


def run_rr(q, torch, steps, warmup, flush, kernel_steps):
    """Radiative pusher (deterministic radiation reaction instead of the NCS Monte Carlo):
    the 1e6-electron focused-pulse workload with the quantum-corrected LL force and the
    radiative T-BMT (QED_F_MLL | QED_F_MBMT | QED_F_SPIN), mixed and FP64 paths; only
    electrons stream (104 B / 152 B per particle-step)."""
    flags = q.QED_F_MLL | q.QED_F_MBMT | q.QED_F_SPIN
    n = 1_000_000
    caps = {"cap_e": n, "cap_p": 16, "cap_ph": 16}
    out = {"workload": "c2_focused_cp_a100_g2e4, 1e6 electrons, MLL + radiative T-BMT", "unit": "particle-steps/s"}
    for name, prec, nst, bpp in (("mixed", q.QED_PREC_MIXED, steps, 104), ("f64", q.QED_PREC_F64, steps, 152)):
        sim, info = run_gpu_path(q, torch, c2_workload(n, 2), prec, nst, warmup, flush, flags, kernel_steps,
                                 caps=caps)
        kn = info["kern"]
        ks = max(kn["kernel_steps"], 1)
        k_lep_ms = kn["kernel_ms"][1]
        out[name] = {"value": info["particles"] / (info["ms"] * 1e-3), "ms_per_step": info["ms"] / nst,
                     "k_lepton_ms": k_lep_ms / ks,
                     "k_lepton_GBs": kn["lep_units"] * bpp / (k_lep_ms * 1e-3) / 1e9 if k_lep_ms else None,
                     "status": info["status"]}
        sim.close()
    out["speedup_mixed"] = out["mixed"]["value"] / out["f64"]["value"]
    return out


def run_matter(q, torch, steps, warmup, flush, pre=40, f64_steps=10):
    """Bremsstrahlung and Bethe-Heitler pairs in matter (Sec. III E): 1e6 electrons of
    1 GeV entering 5 mm of gold, no field, c dt = 5 um (the paper's Geant4 comparison
    geometry); `pre` untimed steps populate photons and pairs, then the timing of the
    headline (L2 flushed before every step).  Mixed and FP64 paths."""
    import workloads
    n = 1_000_000
    wl = workloads.slab(n=n, seed=5)
    flags = q.QED_F_BREMS | q.QED_F_BH
    caps = {"cap_e": 3 * n, "cap_p": 2 * n, "cap_ph": 8 * n}
    out = {"workload": wl["name"], "unit": "particle-steps/s", "pre_steps": pre, "medium": wl["medium"]}
    for name, prec, nst in (("mixed", q.QED_PREC_MIXED, steps), ("f64", q.QED_PREC_F64, f64_steps)):
        if nst <= 0:
            continue
        sim, info = run_gpu_path(q, torch, wl, prec, nst, warmup, flush, flags, 0, pre=pre, caps=caps)
        c = sim.counters()
        out[name] = {"value": info["particles"] / (info["ms"] * 1e-3), "ms_per_step": info["ms"] / nst,
                     "steps": nst, "status": info["status"], "counts_after": info["final_counts"],
                     "brems": c["n_brems_e"] + c["n_brems_p"], "pairs": c["n_bh"]}
        sim.close()
    if "mixed" in out and "f64" in out:
        out["speedup_mixed"] = out["mixed"]["value"] / out["f64"]["value"]
    return out


C4_PRE = 150   # the ensembles start 150 steps before the beam centres reach the focus


def c4_workload(seed=4):
    """64 independent collisions of uneven size (10^U(3,6) particles each), a0, gamma0,
    polarisation and spin states varying, every fourth a gamma beam, each moved like the
    1e6-electron workload so that its collision falls in the timed window."""
    import workloads
    wls = workloads.c4(n_ens=64, seed=seed)
    for wl in wls:
        for sp in ("e", "ph"):
            if len(wl[sp]["id"]):
                wl[sp]["z"] = wl[sp]["z"] + T_SHIFT
        wl["t0"] = T_SHIFT
        wl["step0"] = int(round(T_SHIFT / wl["dt"]))
    return wls


def run_c4(q, torch, steps, warmup, tune_steps=2, f64_steps=10):
    """Batched ensembles: CUDA-graph replay of one batched step after the autotuner picked
    the launch shape.  For comparison the same ensembles, advanced to the same step on a
    second copy (runs are deterministic), step one by one with qed_step over the same
    segment of the trajectory; and an FP64 batch of the same ensembles, advanced to the
    same step, over f64_steps steps of that segment.  Streamed bytes: the mean live e-, e+
    and photons of the timed window (start and end) times 104 / 100 B per particle-step."""
    wls = c4_workload()
    caps = []
    for wl in wls:
        n = len(wl["e"]["id"]) + len(wl["ph"]["id"])
        caps.append({"cap_e": n + n // 2 + 4096, "cap_p": n // 2 + 4096, "cap_ph": 24 * n + 4096})
    flags = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
    n0 = sum(len(w["e"]["id"]) + len(w["ph"]["id"]) for w in wls)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def processed(b):
        return int(torch.stack([s.stats for s in b.sims]).sum(0)[6].item())

    def live(b):
        lep = sum(s.e.count() + s.pos.count() for s in b.sims)
        return lep, sum(s.ph.count() for s in b.sims)

    b = q.Batch(wls, prec=q.QED_PREC_MIXED, flags=flags, caps=caps)
    b.run(C4_PRE)
    cfg, tune_rate = q.qed_batch_tune(b.b, tune_steps)
    b.run(warmup)
    torch.cuda.synchronize()
    done = b.clocks()[0][1] - wls[0]["step0"]
    p0 = processed(b)
    l0, g0 = live(b)
    ev0.record()
    b.run(steps)
    ev1.record()
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    value = (processed(b) - p0) / (ms * 1e-3)
    l1, g1 = live(b)
    gbs = 0.5 * ((l0 + l1) * BYTES["mixed"]["lep"] + (g0 + g1) * BYTES["mixed"]["ph"]) * steps / (ms * 1e-3) / 1e9
    status = q.qed_read_status(b.ctx)
    b.close()
    # FP64 batch of the same ensembles over the start of the same segment
    f64 = None
    if f64_steps > 0:
        b = q.Batch(c4_workload(), prec=q.QED_PREC_F64, flags=flags, caps=caps)
        b.run(done)
        torch.cuda.synchronize()
        p0 = processed(b)
        ev0.record()
        b.run(f64_steps)
        ev1.record()
        ev1.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        f64 = {"value": (processed(b) - p0) / (ms64 * 1e-3), "ms_per_step": ms64 / f64_steps, "steps": f64_steps}
        b.close()
    # second copy, advanced to the same step, then one qed_step per ensemble per step
    b = q.Batch(c4_workload(), prec=q.QED_PREC_MIXED, flags=flags, caps=caps)
    b.run(done)
    for k, (t, st) in enumerate(b.clocks()):
        b.sims[k].t, b.sims[k].step_no = t, st
    torch.cuda.synchronize()
    p0 = processed(b)
    ev0.record()
    for _ in range(steps):
        for s in b.sims:
            s.run(1, flags)
    ev1.record()
    ev1.synchronize()
    ms_seq = ev0.elapsed_time(ev1)
    seq_value = (processed(b) - p0) / (ms_seq * 1e-3)
    b.close()
    return {"workload": "c4_64_ensembles_loguniform_1e3_1e6", "value": value, "unit": "particle-steps/s",
            "ensembles": len(wls), "particles_at_start": n0, "steps_before_timing": done, "steps": steps,
            "ms_per_step": ms / steps, "launch": "cuda_graph", "tuned_config": cfg, "tune_best_rate": tune_rate,
            "sequential_qed_step": {"value": seq_value, "ms_per_step": ms_seq / steps,
                                    "note": "same ensembles, same steps, 64 qed_step calls per step"},
            "batched_over_sequential": value / seq_value, "status": status,
            "step_GBs_approx": gbs, "step_hbm_frac_approx": gbs / _peaks()[0], "step_frac": gbs / _peaks()[0],
            "f64": f64, "speedup_mixed_over_f64": value / f64["value"] if f64 else None,
            "l2": "not flushed: every step streams > 1 GB of particle state (L2 is 129 MB)"}


def _photon_spectrum(q, sp, nbins=48):
    """photon dN/d(ln omega) and <xi> in the (x, y) detection basis, via qed_diag"""
    import numpy as np
    d = q.diag(sp, q.diag_spec(q.QED_DIAG_SPECTRUM, nbins, 1, 1.0, 3e4))
    b = d["bins"][0]
    return b[:, 0], b[:, 1:4] / np.maximum(b[:, :1], 1e-300), b[:, 4]


C5_BATCH = 1024   # Adam steps, not samples, set the fit: 1e8 rows at 1024 take ~10 s


def run_c5(q, torch, steps, n_train=100_000_000):
    """Learned sampler: training on table-sampled rows, its ln u error against the table
    sampler on held-out rows, the tensor-core evaluation rate, then the 1e6-electron
    workload stepped with it and with the table path (same seeds): throughput of both and
    the photon spectrum / polarisation of the learned run as pulls against the table run
    (the comparison with the oracle is in the GPU tests)."""
    import numpy as np
    ctx = q.qed_init_tables()
    torch.cuda.synchronize()
    t0 = time.time()
    q.qed_mlp_train(ctx, n_train, C5_BATCH, seed=5)
    train_s = time.time() - t0
    rng = np.random.default_rng(77)
    nr = 1_000_000
    rows = np.stack([rng.uniform(math.log(1e-3), math.log(10.0), nr), rng.uniform(-1, 1, nr),
                     rng.uniform(1e-7, 1 - 1e-7, nr)], 1).astype(np.float32)
    x = torch.as_tensor(rows, device="cuda")
    y_m = torch.empty(nr, device="cuda")
    y_t = torch.empty(nr, device="cuda")
    q.qed_mlp_target(ctx, x.data_ptr(), y_t.data_ptr(), nr)
    q.qed_mlp_eval(ctx, x.data_ptr(), y_m.data_ptr(), nr)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(10):
        q.qed_mlp_eval(ctx, x.data_ptr(), y_m.data_ptr(), nr)
    ev1.record()
    ev1.synchronize()
    eval_rate = 10 * nr / (ev0.elapsed_time(ev1) * 1e-3)
    err = (y_m - y_t).abs().cpu().numpy()
    # the 1e6-electron workload with each sampler
    flags = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
    n = 1_000_000
    res = {}
    for name, extra in (("table", 0), ("learned", q.QED_F_MLP)):
        sctx = q.qed_ctx_share(ctx)
        sim = q.Simulation(c2_workload(n, 2), prec=q.QED_PREC_MIXED, ctx=sctx, cap_e=n + 4_000_000,
                           cap_p=4_000_000, cap_ph=40 * n)
        sim.run(PRE_STEPS, flags | extra)
        torch.cuda.synchronize()
        p0 = int(sim.stats[6].item())
        ev0.record()
        sim.run(steps, flags | extra)
        ev1.record()
        ev1.synchronize()
        rate = (int(sim.stats[6].item()) - p0) / (ev0.elapsed_time(ev1) * 1e-3)
        h, xi, cnt = _photon_spectrum(q, sim.ph)
        res[name] = {"rate": rate, "h": h, "xi": xi, "cnt": cnt, "status": sim.status(),
                     "counts": (sim.e.count(), sim.pos.count(), sim.ph.count())}
        sim.close()
        q.qed_destroy(sctx)
    q.qed_destroy(ctx)
    ht, hm = res["table"]["h"], res["learned"]["h"]
    ok = (ht > 100) & (hm > 100)
    pull_h = (hm - ht)[ok] / np.sqrt(hm + ht)[ok]
    rel_h = np.abs(hm - ht)[ok] / ht[ok]
    sig_xi = np.sqrt(1.0 / ht[ok] + 1.0 / hm[ok])
    pull_xi = (res["learned"]["xi"][ok] - res["table"]["xi"][ok]) / sig_xi[:, None]
    return {"train": {"samples": n_train, "batch": C5_BATCH, "seconds": train_s},
            "ln_u_error_vs_table": {"rows": nr, "median": float(np.median(err)),
                                    "p99": float(np.quantile(err, 0.99)), "max": float(err.max())},
            "eval_rows_per_s": eval_rate,
            "workload": "c2_focused_cp_a100_g2e4, 1e6 electrons", "steps": steps,
            "rate_learned": res["learned"]["rate"], "rate_table": res["table"]["rate"],
            "counts_learned": res["learned"]["counts"], "counts_table": res["table"]["counts"],
            "photon_spectrum_pull_vs_table": {"bins": int(ok.sum()), "rms": float(np.sqrt(np.mean(pull_h ** 2))),
                                              "max_abs": float(np.abs(pull_h).max()),
                                              "max_rel_diff": float(rel_h.max()), "median_rel_diff": float(np.median(rel_h)),
                                              "note": "same seeds: the two runs are correlated, pulls use independent errors"},
            "stokes_pull_vs_table": {"rms": [float(v) for v in np.sqrt(np.mean(pull_xi ** 2, 0))],
                                     "max_abs": [float(v) for v in np.abs(pull_xi).max(0)]},
            "status": [res["table"]["status"], res["learned"]["status"]]}


def run_diag(q, torch, sim, reps=5):
    """End-of-run observables on the final state: photon spectrum with the Stokes parameters
    in the (x, y) detection basis, electron spectrum with the mean spin (mixed layout reads
    k, xi, theta, w = 32 B per photon and p, S, w = 28 B per electron)."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, sp, bytes_per in (("photon_spectrum", sim.ph, 32), ("electron_spectrum", sim.e, 28)):
        spec = q.diag_spec(q.QED_DIAG_SPECTRUM, 256, 1, 1.0, 3e4)
        buf = torch.zeros(5 * 257 + 2, dtype=torch.float64, device="cuda")
        q.qed_diag(sim.ctx, sp.handle, spec, buf.data_ptr())
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            q.qed_diag(sim.ctx, sp.handle, spec, buf.data_ptr())
        ev1.record()
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        n = sp.count()
        out[name] = {"ms": ms, "particles": n, "GBs": n * bytes_per / (ms * 1e-3) / 1e9}
    return out


def run_e2e(q, torch, sim, prec, steps, flags):
    """Host-resident particles: every step copies the live state in and out (pinned)."""
    import ctypes as C
    rt = torch.float64 if prec == q.QED_PREC_F64 else torch.float32
    hosts, keep = [], []
    for sp in (sim.e, sim.pos, sim.ph):
        soa = q.qed_soa()
        d = {}
        for k, v in sp.t.items():
            h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
            h.copy_(v)
            d[k] = h
            setattr(soa, k, h.data_ptr())
        hosts.append(soa)
        keep.append(d)
    counts = [sim.e.count(), sim.pos.count(), sim.ph.count()]
    esz = 8 if prec == q.QED_PREC_F64 else 4
    per = {0: 24 + 7 * esz + 8, 1: 24 + 7 * esz + 8, 2: 24 + 8 * esz + 8}

    def host_step(counts):
        out = q.qed_step_host(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, hosts[0], hosts[1],
                              hosts[2], counts, sim.fields, sim.t, sim.dt, sim.seed, sim.step_no, flags)
        sim.t += sim.dt
        sim.step_no += 1
        return out

    for _ in range(2):   # untimed warm-up through the same call
        counts = host_step(counts)
    tot_p = h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        tot_p += sum(counts)
        h2d += sum(per[k] * counts[k] for k in range(3))
        counts = host_step(counts)
        d2h += sum(per[k] * counts[k] for k in range(3))
    el = time.perf_counter() - t0
    out = {"value": tot_p / el, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d // steps,
           "d2h_bytes_per_step": d2h // steps, "steps": steps, "particles": tot_p, "seconds": el}
    out["copy_bound"] = copy_bound(torch, h2d / steps, d2h / steps, tot_p / steps)
    return out


def copy_bound(torch, h2d, d2h, particles):
    """What the host-buffer step could reach if it were only its copies: one plain pinned
    host->device and device->host copy of up to 1 GiB each, timed with CUDA events, and the
    particle-steps/s of a step that moves h2d + d2h bytes at those rates."""
    nb = int(min(max(h2d, d2h), 1 << 30)) // 16 * 16
    if nb <= 0:
        return None
    h = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nb, dtype=torch.uint8, device="cuda")
    rates = {}
    for name, dst, src in (("h2d_GBs", d, h), ("d2h_GBs", h, d)):
        dst.copy_(src, non_blocking=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        ev1.record()
        ev1.synchronize()
        rates[name] = 3 * nb / (ev0.elapsed_time(ev1) * 1e-3) / 1e9
    t = h2d / (rates["h2d_GBs"] * 1e9) + d2h / (rates["d2h_GBs"] * 1e9)
    del h, d
    return dict(rates, bytes_timed=nb, value=particles / t, unit="particle-steps/s", scope="one GPU")


def oracle_sample(n_e, steps_timed, warmup=0, seed=2, threads=None, log_tol=None):
    """The oracle on a bounded sample of the same workload: the untimed steps on every host
    core, then `steps_timed` steps timed on all `threads` cores (default: every core the
    process may use) and the same steps again, from a copy of the same state, on one core
    (the two runs are identical step for step).  Returns both rates and the all-core run's
    final state, with its near-tie log when log_tol is given."""
    import oracle
    o = oracle.Oracle()
    nt = o.set_threads(threads or len(os.sched_getaffinity(0)))
    if log_tol is not None:
        o.set_near_tol(log_tol)
    wl = c2_workload(n_e, seed)
    s = oracle.Sim(o, wl)
    flags = oracle.F_NCS | oracle.F_NBW | oracle.F_VB | oracle.F_SPIN
    s.run(PRE_STEPS + warmup, flags)
    snap = dict(s.state(), t0=s.t, step0=s.step_no, field=wl["field"], dt=wl["dt"], seed=wl["seed"])
    snap["next_id"] = snap.pop("next_id")

    def timed(sim):
        tot = 0
        t0 = time.perf_counter()
        for _ in range(steps_timed):
            tot += sim.e.n + sim.pos.n + sim.ph.n
            sim.run(1, flags)
        return tot, time.perf_counter() - t0

    tot, el = timed(s)
    out = {"threads": nt, "value": tot / el, "particle_steps": tot, "seconds": el, "state": s.state(),
           "steps": PRE_STEPS + warmup + steps_timed}
    if log_tol is not None:
        out["near"] = o.near_log()
        o.set_near_tol(1e-6)
    o.set_threads(1)
    s1 = oracle.Sim(o, snap, cap_e=s.e.cap, cap_p=s.pos.cap, cap_ph=s.ph.cap)
    tot1, el1 = timed(s1)
    out["single"] = {"threads": 1, "value": tot1 / el1, "particle_steps": tot1, "seconds": el1}
    return out


def accuracy(q, torch, orc_run, n_e, seed=2):
    """Error of the mixed path against the FP64 oracle on the oracle's sample of the headline
    workload (the cpu_baseline run: same electrons, same seed, same steps), and against the
    FP64 GPU path on the same inputs:
      per particle -- primary electrons after all the steps: largest relative momentum error
        and largest spin-component error of the mixed path, excluding electrons with a
        logged near-tie decision (the draw within 1e-4 relative of its threshold at some
        step), which are counted; the FP64 GPU path over every particle;
      observables -- photon weight per ln-energy bin, mean Stokes parameters in the (x, y)
        detection basis, pair yield, mean positron spin: value of each path and pull
        (difference over the Poisson / binomial error of one run; same seeds, so the runs
        are correlated and the pulls are small by construction)."""
    import numpy as np
    from oracle import diag as odiag
    wl = c2_workload(n_e, seed)
    flags = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
    steps = orc_run["steps"]
    nbins, lo, hi = 8, 10.0, 3.0e4
    spec = q.diag_spec(q.QED_DIAG_SPECTRUM, nbins, 1, lo, hi, ref=(1.0, 0.0, 0.0))
    runs = {}
    for name, prec in (("mixed", q.QED_PREC_MIXED), ("f64_gpu", q.QED_PREC_F64)):
        sim = q.Simulation(wl, prec=prec, cap_e=4 * n_e + 100_000, cap_p=2 * n_e + 100_000, cap_ph=80 * n_e)
        sim.run(steps, flags)
        st = sim.state()
        d = q.diag(sim.ph, spec)
        runs[name] = (st, d["bins"][0], d["total"], sim.status())
        sim.close()
    ost = orc_run["state"]
    od = odiag.diag(ost["ph"], odiag.SPECTRUM, nbins, 1, lo, hi, ref=(1.0, 0.0, 0.0), photon=True)
    runs["oracle"] = (ost, od["bins"][0], od["total"], 0)

    def by_id(d):
        o = np.argsort(d["id"], kind="stable")
        return {k: v[o] for k, v in d.items()}

    def errs(g, o, ids=None):
        g, o = by_id(g), by_id(o)
        if ids is not None:
            g = {k: v[np.isin(g["id"], ids)] for k, v in g.items()}
            o = {k: v[np.isin(o["id"], ids)] for k, v in o.items()}
        assert np.array_equal(g["id"], o["id"])
        pg, po = (np.stack([d["px"], d["py"], d["pz"]], 1) for d in (g, o))
        dp = np.linalg.norm(pg - po, axis=1) / np.maximum(np.linalg.norm(po, axis=1), 1.0)
        ds = np.abs(np.stack([g[k] - o[k] for k in ("s1", "s2", "s3")], 1)).max(1)
        return g["id"], dp, ds

    prim = np.asarray(wl["e"]["id"], dtype=np.uint64)
    ids, dp, ds = errs(runs["mixed"][0]["e"], ost["e"], prim)
    nid, _, _, nm = orc_run["near"]
    near = set(nid[nm < 1e-4].tolist())
    has_near = np.array([int(i) in near for i in ids], dtype=bool)
    bad = (dp > 2e-5) | (ds > 2e-5)
    ex = bad & has_near          # differ, with a decision within 1e-4 of its threshold
    per = {"electrons": int(len(ids)), "exempted_near_ties": int(ex.sum()),
           "beyond_2e-5_without_near_tie": int((bad & ~has_near).sum()),
           "max_rel_dp": float(dp[~ex].max()), "max_dS": float(ds[~ex].max()),
           "median_rel_dp": float(np.median(dp[~ex])), "median_dS": float(np.median(ds[~ex])),
           "rule": "an electron may exceed 2e-5 only if the oracle logged one of its decisions within "
                   "1e-4 relative of its threshold; maxima are over all other electrons"}
    f64 = {}
    same_ids = all(np.array_equal(np.sort(runs["f64_gpu"][0][sp]["id"]), np.sort(ost[sp]["id"]))
                   for sp in ("e", "pos", "ph"))
    if same_ids:
        f64 = {"ids_identical": True}
        for sp in ("e", "pos", "ph"):
            _, a, b = errs(runs["f64_gpu"][0][sp], ost[sp])
            f64[sp] = {"max_rel_dp": float(a.max()) if len(a) else 0.0, "max_dS": float(b.max()) if len(b) else 0.0}
    else:
        f64 = {"ids_identical": False}

    def obs(run):
        st, bins, tot, _ = run
        pos = st["pos"]
        s = np.stack([pos["s1"], pos["s2"], pos["s3"]], 1)
        return {"spec": bins[:, 0], "xi": tot[1:4] / max(tot[0], 1e-300), "n_ph": float(tot[0]),
                "pairs": float(len(pos["id"])), "pos_S": s.mean(0) if len(s) else np.zeros(3), "n_pos": len(s)}

    O = {k: obs(v) for k, v in runs.items()}

    def compare(a, b):
        A, B = O[a], O[b]
        sp_sig = np.sqrt(np.maximum(A["spec"] + B["spec"], 1.0))
        use = (A["spec"] > 100) & (B["spec"] > 100)
        xi_sig = np.sqrt((1 - np.minimum(A["xi"] ** 2, 1)) / max(A["n_ph"], 1) +
                         (1 - np.minimum(B["xi"] ** 2, 1)) / max(B["n_ph"], 1))
        pr_sig = math.sqrt(A["pairs"] + B["pairs"]) or 1.0
        ps_sig = np.sqrt((1 - np.minimum(A["pos_S"] ** 2, 1)) / max(A["n_pos"], 1) +
                         (1 - np.minimum(B["pos_S"] ** 2, 1)) / max(B["n_pos"], 1))
        return {"photon_spectrum_pull_max": float(np.abs((A["spec"] - B["spec"])[use] / sp_sig[use]).max()),
                "photon_spectrum_rel_diff_max": float(np.abs((A["spec"] - B["spec"])[use] / B["spec"][use]).max()),
                "stokes_xi": [float(v) for v in A["xi"]], "stokes_xi_ref": [float(v) for v in B["xi"]],
                "stokes_pull": [float(v) for v in (A["xi"] - B["xi"]) / xi_sig],
                "pairs": A["pairs"], "pairs_ref": B["pairs"], "pair_pull": (A["pairs"] - B["pairs"]) / pr_sig,
                "positron_S": [float(v) for v in A["pos_S"]], "positron_S_ref": [float(v) for v in B["pos_S"]],
                "positron_S_pull": [float(v) for v in (A["pos_S"] - B["pos_S"]) / ps_sig]}

    return {"workload": f"c2_focused_cp_a100_g2e4, the oracle sample: {n_e} electrons, {steps} steps",
            "per_particle_mixed_vs_oracle": per, "per_particle_f64_gpu_vs_oracle": f64,
            "observables_mixed_vs_oracle": compare("mixed", "oracle"),
            "observables_mixed_vs_f64_gpu": compare("mixed", "f64_gpu"),
            "status": [runs["mixed"][3], runs["f64_gpu"][3]],
            "note": "same inputs and Philox streams on all three; pulls use the error of independent runs"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-sample", type=int, default=20_000)
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--c5-steps", type=int, default=50,
                    help="timed steps of the learned-sampler leg (0: skip)")
    ap.add_argument("--c4-steps", type=int, default=100,
                    help="timed steps of the 64-ensemble batch (0: skip)")
    ap.add_argument("--c3-steps", type=int, default=50,
                    help="timed steps of the 3e7-electron grid workload (0: skip)")
    ap.add_argument("--c3-f64-steps", type=int, default=10,
                    help="timed steps of the grid workload on the FP64 path (0: skip)")
    ap.add_argument("--pic-steps", type=int, default=20,
                    help="timed steps of the self-consistent PIC leg (0: skip)")
    ap.add_argument("--rr-steps", type=int, default=50,
                    help="timed steps of the radiative-pusher leg (0: skip)")
    ap.add_argument("--matter-steps", type=int, default=50,
                    help="timed steps of the bremsstrahlung / Bethe-Heitler leg (0: skip)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy block (mixed path vs the oracle sample and the FP64 GPU path)")
    ap.add_argument("--kernel-steps", type=int, default=20,
                    help="steps after the timed ones with per-kernel timing (roofline)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        r = oracle_sample(args.cpu_sample, args.steps, args.warmup)
        v, el, ncores = r["value"], r["seconds"], r["threads"]
        line = {"metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": "c2_focused_cp_a100_g2e4", "electrons": args.cpu_sample,
                           "pre_steps": PRE_STEPS, "processes": "NCS+NBW+VB+T-BMT"},
                "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": ncores, "kind": "oracle",
                                 "sample": f"{args.cpu_sample} electrons of the same beam recipe, "
                                           f"{args.steps} steps after {PRE_STEPS + args.warmup} untimed",
                                 "single_core": {"value": r["single"]["value"], "cores": 1}},
                "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    import paper_2306_11288_gb300 as q

    if world > 1:
        # replicas: the headline and e2e on every rank; the single-GPU side legs only at N = 1
        args.c3_steps = args.c4_steps = args.c5_steps = args.rr_steps = args.pic_steps = args.matter_steps = 0
        args.no_f64 = True
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        q.build()
    if dist is not None:
        dist.barrier()
    flags = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    wl = c2_workload(args.n, seed=replica_seed(rank))

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        sim, info = run_gpu_path(q, torch, wl, q.QED_PREC_MIXED, args.steps, args.warmup, flush, flags,
                                 args.kernel_steps)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    f64 = None
    if not args.no_f64:
        sim64, f64 = run_gpu_path(q, torch, c2_workload(args.n, seed=replica_seed(rank)), q.QED_PREC_F64, args.steps,
                                  args.warmup, flush, flags, min(args.kernel_steps, args.steps))
        sim64.close()
    diag = run_diag(q, torch, sim)
    c3 = (run_c3(q, torch, args.c3_steps, args.warmup, flush, args.c3_f64_steps, min(args.kernel_steps, 10))
          if args.c3_steps > 0 else None)
    rr = run_rr(q, torch, args.rr_steps, args.warmup, flush, min(args.kernel_steps, 10)) if args.rr_steps > 0 else None
    pic = run_pic(q, torch, args.pic_steps, args.warmup) if args.pic_steps > 0 else None
    matter = run_matter(q, torch, args.matter_steps, args.warmup, flush) if args.matter_steps > 0 else None
    c4 = run_c4(q, torch, args.c4_steps, args.warmup) if args.c4_steps > 0 else None
    c5 = run_c5(q, torch, args.c5_steps) if args.c5_steps > 0 else None
    e2e = run_e2e(q, torch, sim, q.QED_PREC_MIXED, args.e2e_steps, flags)

    ms, parts = aggregate(torch, dist, "cuda", info["ms"], info["particles"])
    e2e_ms, e2e_parts = aggregate(torch, dist, "cuda", 1e3 * e2e["seconds"], e2e["particles"])
    e2e["value"] = e2e_parts / (e2e_ms * 1e-3)
    for k in ("h2d_bytes_per_step", "d2h_bytes_per_step"):   # whole job: every rank's copies
        e2e[k] = int(aggregate(torch, dist, "cuda", 0.0, e2e[k])[1])
    if rank != 0:
        sim.close()
        dist.destroy_process_group()
        return 0

    peak, peak_kind = _peaks()
    b = BYTES["mixed"]
    kn = info["kern"]
    k_ph_ms, k_lep_ms, k_ev_ms = kn["kernel_ms"]
    ks = max(kn["kernel_steps"], 1)
    lep_bytes = kn["lep_units"] * b["lep"] + kn["ncs_births"] * b["ncs_birth"]
    ph_bytes = kn["ph_units"] * b["ph"] + kn["nbw_births"] * b["nbw_birth"]
    dom = "k_photon" if k_ph_ms >= k_lep_ms else "k_lepton"
    dom_bytes, dom_ms = (ph_bytes, k_ph_ms) if dom == "k_photon" else (lep_bytes, k_lep_ms)
    dom_units = kn["ph_units"] if dom == "k_photon" else kn["lep_units"]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    value = parts / (ms * 1e-3)
    # the whole step: algorithmic bytes of every pass and birth over the timed steps
    step_gbs = (info["ph_units"] * b["ph"] + info["lep_units"] * b["lep"] + info["ncs_births"] * b["ncs_birth"] +
                info["nbw_births"] * b["nbw_birth"]) / (ms * 1e-3) / 1e9
    cpu = oracle_sample(max(args.cpu_sample, 1), 20, 0, log_tol=1e-3)
    acc = accuracy(q, torch, cpu, max(args.cpu_sample, 1)) if not args.no_accuracy else None
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64-islands",
        "data": "synthetic",
        "config": {"workload": "c2_focused_cp_a100_g2e4", "electrons_per_gpu": args.n,
                   "processes": "NCS+NBW+VB+T-BMT, compaction every step", "pre_steps": PRE_STEPS,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} (copy)",
                     "traffic": TRAFFIC_PER_UNIT[dom] * dom_units / ks if TRAFFIC_PER_UNIT else None,
                     "bytes_per_launch": dom_bytes / ks, "avg_launch_ms": dom_ms / ks,
                     "launches_timed": ks, "units_per_launch": dom_units / ks,
                     "step_frac": step_gbs / peak,
                     "step_frac_note": "whole step (all passes, births, event kernels) at its algorithmic "
                                       "bytes over ms_per_step, against the same peak"},
        "kernels": {"steps": ks, "k_photon_ms": k_ph_ms / ks, "k_lepton_ms": k_lep_ms / ks,
                    "event_kernels_ms": k_ev_ms / ks, "step_ms_serialised": kn["ms"] / ks,
                    "k_photon_GBs": ph_bytes / (k_ph_ms * 1e-3) / 1e9 if k_ph_ms else None,
                    "k_lepton_GBs": lep_bytes / (k_lep_ms * 1e-3) / 1e9 if k_lep_ms else None,
                    "photons_per_launch": kn["ph_units"] / ks, "leptons_per_launch": kn["lep_units"] / ks},
        "step_GBs": step_gbs,
        "cpu_baseline": {"value": cpu["value"], "unit": "particle-steps/s", "cores": cpu["threads"], "kind": "oracle",
                         "sample": f"{args.cpu_sample} electrons of the same beam recipe, 20 steps after "
                                   f"{PRE_STEPS} untimed (untimed steps on every core)",
                         "single_core": {"value": cpu["single"]["value"], "cores": 1}},
        "accuracy": acc,
        "e2e": e2e,
        "diag": diag,
        "c3": c3,
        "c4": c4,
        "radiative_pusher": rr,
        "pic": pic,
        "matter": matter,
        "c5": c5,
        "gpu_launches": 4 * args.steps,   # headline loop; per step: photon, lepton, scans, events
        "clocks": clk.summary(),
        "counts_after": {"e": info["final_counts"][0], "pos": info["final_counts"][1],
                         "ph": info["final_counts"][2]},
        "status": info["status"],
    }
    if f64 is not None:
        v64 = f64["particles"] / (f64["ms"] * 1e-3)
        k64 = f64["kern"]
        ks64 = max(k64["kernel_steps"], 1)
        line["f64"] = {"value": v64, "ms_per_step": f64["ms"] / args.steps, "speedup_mixed": value / v64,
                       "k_photon_ms": k64["kernel_ms"][0] / ks64, "k_lepton_ms": k64["kernel_ms"][1] / ks64,
                       "event_kernels_ms": k64["kernel_ms"][2] / ks64}
    print(json.dumps(line))
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
