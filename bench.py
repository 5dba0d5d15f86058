#!/usr/bin/env python
"""Benchmark: daughter atom-steps/s of the TTCF daughter ensemble on GB300.

Workload (bulk WCA, Example 1 state point; the 16384-daughter configuration):
N = 2048 atoms, rho = 0.8442, T = 0.722, dt = 0.0025; 4096 mother states
(64 independent mothers x 64 states 200 steps apart after 20000
thermalisation steps), x4 mappings = 16384 daughters of 1000 steps.  The
shear rates 1e-1 ... 1e-7 reuse the same mothers.  One benchmark step = one
full pass of the hot path over the 16384-daughter batch at one shear rate:
spawn (mapping, Omega(0), B(0)), the persistent daughter launch and the
on-device reduction of <Omega(0)B(s)>, its integral and the direct average;
successive steps take the rates in turn (1e-1, 1e-2, ..., 1e-7, 1e-1, ...).
Inputs are synthetic and seeded.

value  = sum over daughters of N * steps / device time of the steps, inputs
         resident in HBM (mothers made on the GPU before timing);
e2e    = the same through the C ABI with host buffers: mothers copied from
         pinned host memory and the viscosity read back inside the timed
         region.

The last stdout line is the compact result (one JSON object of < 2 KB).
The long sections (confined channel, uneven batch, planar elongational
flow, control variate, precision floor, Green-Kubo, momentum kicks, mapping
study, plain GPU arm, oracle parity sample) are printed before it, one JSON
line each, or written to the file given by --sections-out.

Launch:  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs the same per-GPU workload on its own mothers
(weak scaling); the only exchange is a final merge of the per-sample
ensemble statistics.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import shutil
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

RATES = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7]
HEADLINE_RATES = (1e-1, 1e-3, 1e-7)
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (sm_103)
N_SM = 152
SM_MAX_MHZ = 2070.0
FLOPS_PER_PAIR = 36.0            # one unique WCA pair with virial (Newton 3)
FLOPS_PER_PAIR_LJ = 25.0         # one unique LJ-c_ij pair of the confined system (no virial)
# DRAM bytes of the dominant kernels from one ncu capture each (small cases,
# profiles/*.md), scaled to a launch by the units it processes:
# daughter_kernel reads its mothers (per daughter) and writes the series (per
# sample); conf_kernel streams its per-CTA scratch (per atom-step).
BULK_READ_PER_DAUGHTER = 31.3e3
BULK_WRITE_PER_SAMPLE = 10.9
CONF_BYTES_PER_ATOM_STEP = 399.0
CONF_RATES = [1e-1, 1e-3, 1e-5, 1e-7]
UNEVEN_SIZES = (256, 864, 4000)
UNEVEN_RATES = [1e-2, 1e-3, 1e-4, 1e-5, 1e-6]
PROBE_SRC = os.path.join(HERE, "paper_2312_02990_gb300", "microbench", "alu_rates.cu")


def fp32_peak_tflops(mhz=SM_MAX_MHZ):
    return N_SM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=7)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n-atoms", type=int, default=2048)
    p.add_argument("--mothers", type=int, default=64)
    p.add_argument("--states", type=int, default=64)
    p.add_argument("--daughter-steps", type=int, default=1000)
    p.add_argument("--n-eq", type=int, default=20000)
    p.add_argument("--spacing", type=int, default=200)
    p.add_argument("--sections-out", default=None,
                   help="write the long sections to this JSON file instead of stdout lines")
    p.add_argument("--no-sections", action="store_true", help="headline only (with the CPU baseline)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-groups", type=int, default=16,
                   help="mother groups of the oracle sample (CPU baseline and parity per rate)")
    p.add_argument("--oracle-eq", type=int, default=2000)
    p.add_argument("--no-cv", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--cv-train-groups", type=int, default=16384)
    p.add_argument("--cv-eval-groups", type=int, default=4096)
    p.add_argument("--cv-aux", type=int, default=16384)
    p.add_argument("--cv-steps", type=int, default=500)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-confined", action="store_true")
    p.add_argument("--no-uneven", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-floor", action="store_true", help="skip the precision-floor sweep")
    p.add_argument("--no-gk", action="store_true", help="skip the Green-Kubo cross-check")
    p.add_argument("--no-kick", action="store_true", help="skip the momentum-kick mothers section")
    p.add_argument("--no-mapstudy", action="store_true", help="skip the mapping-set / Eq. 4 study")
    p.add_argument("--no-probe", action="store_true", help="skip the FP32 throughput probe")
    p.add_argument("--no-elong", action="store_true", help="skip the planar elongational flow section")
    p.add_argument("--elong-chains", type=int, default=256,
                   help="independent N=256 mother chains of the elongational section")
    p.add_argument("--elong-states", type=int, default=16, help="mother states per chain")
    p.add_argument("--only", default=None,
                   help="run one section alone and print its JSON (confined, uneven, cv, floor, "
                        "gk, kick, mapstudy, probe, elong)")
    p.add_argument("--conf-chains", type=int, default=64, help="independent confined mother chains")
    p.add_argument("--conf-states", type=int, default=4, help="mother states per chain")
    p.add_argument("--conf-eq", type=int, default=4000)
    p.add_argument("--conf-spacing", type=int, default=200)
    p.add_argument("--conf-steps", type=int, default=2000)
    p.add_argument("--conf-eq-steps", type=int, default=20000,
                   help="steps of the zero-shear chains of the equilibrium friction estimate")
    p.add_argument("--uneven-chains", type=int, default=64)
    p.add_argument("--uneven-states", type=int, default=4)
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "power_w_median": float(np.median(power)) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


class Sections:
    """The long sections: one JSON line each on stdout (before the compact
    result line), or collected into one JSON file."""

    def __init__(self, path):
        self.path = path
        self.all = {}

    def emit(self, name, d):
        self.all[name] = d
        if self.path is None:
            print(json.dumps({"section": name, **d}), flush=True)

    def close(self):
        if self.path is not None:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            with open(self.path, "w") as f:
                json.dump(self.all, f, indent=1)


# --------------------------------------------------------------- GB300 --
def make_mothers(T, args, rank, N, L, n_mothers=None, n_states=None, seed_off=0, n_eq=None):
    """Equilibrium mothers on the GPU (untimed set-up): [G, 6, N], [G]."""
    from paper_2312_02990_gb300 import inputs
    nm = n_mothers or args.mothers
    init = np.stack([inputs.initial_state(N, inputs.BASE_SEED + 1000 * rank + seed_off + k)
                     for k in range(nm)])
    cfg = T.config_default()
    cfg.precision = T.TTCF_MIXED
    with T.Context(cfg) as c:
        ms, al = c.sample_mothers(init, L, n_eq=args.n_eq if n_eq is None else n_eq,
                                  n_states=n_states or args.states, spacing=args.spacing)
    return ms.reshape(-1, 6, N), al.reshape(-1)


def bench_config(T, args, precision=None):
    cfg = T.config_default()
    cfg.precision = T.TTCF_MIXED if precision is None else precision
    cfg.n_steps = args.daughter_steps
    if args.tuned:   # launch variant and skin chosen by the autotuner (set-up)
        cfg.kernel_variant, cfg.skin, cfg.cell_frac = args.tuned
    return cfg


def one_step(T, args, L, rate, mothers, alpha, want_response=False):
    """One pass of the hot path over the batch at one shear rate, through
    the C ABI: create, spawn (device or host inputs), run, read back the
    viscosity (and the response)."""
    c = T.Context(bench_config(T, args))
    bid = c.spawn_daughters(mothers, alpha, float(rate), box=L)
    c.run()
    v = c.viscosity(bid)
    r = None
    if want_response:   # for the multi-rank merge (with <Omega(0)> for the Eq. 4 form)
        r = c.response(bid)
        r["omega_mean"], r["n_valid"] = c.omega_mean(bid)
    stats = c.get_stats()
    c.close()
    return v, r, stats


def bench_gb300(args):
    import torch

    from paper_2312_02990_gb300 import inputs
    from paper_2312_02990_gb300 import ttcf as T

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        T.load(build_if_missing=True)
    if world > 1:   # the other ranks load the library rank 0 built
        torch.distributed.barrier()
        T.load(build_if_missing=False)
    N = args.n_atoms
    L = inputs.bulk_box(N)
    sec = Sections(args.sections_out)

    t0 = time.time()
    ms, al = make_mothers(T, args, rank, N, L)
    t_mothers = time.time() - t0
    G = ms.shape[0]
    D = 4 * G
    atom_steps = float(D) * N * args.daughter_steps     # per benchmark step
    ms_dev = torch.from_numpy(ms).cuda()
    al_dev = torch.from_numpy(al).cuda()
    # the autotuner times every launch variant, Verlet skin and list-cell
    # width on a sample of these mothers (untimed set-up); the runs use it
    args.tuned = None
    if not args.no_autotune:
        cfg = T.config_default()
        cfg.precision, cfg.n_steps = T.TTCF_MIXED, args.daughter_steps
        with T.Context(cfg) as c:
            v, sk, fr, _ = c.autotune(ms[:min(G, 152)], L, shear_rate=1e-3, n_steps=200)
        args.tuned = (v, sk, fr)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    st = torch.cuda.current_stream()
    for k in range(args.warmup):
        one_step(T, args, L, RATES[k % len(RATES)], ms_dev, al_dev)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    kernel_ms, spawn_ms, pairs, rebuilds, launches = [], [], [], [], 0
    per_rate = {}
    for k in range(args.steps):
        g = RATES[k % len(RATES)]
        v, r, s = one_step(T, args, L, g, ms_dev, al_dev, want_response=world > 1)
        per_rate[g] = (v, r)
        kernel_ms.append(s["ms_run"])
        spawn_ms.append(s["ms_spawn"])
        pairs.append(s["pairs_interacting"])
        rebuilds.append(s["rebuilds"])
        launches += s["launches"] + 1            # + the spawn kernel
    ev1.record(st)
    barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    if world > 1:
        tt = torch.tensor([ms_total], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(tt.item())
    ms_step = ms_total / args.steps
    value = atom_steps * world / (ms_step * 1e-3)

    # end to end through the C ABI with host buffers (pinned): the mothers
    # go host -> device and the viscosity device -> host in every step
    e2e = None
    if not args.no_e2e:
        pin_ms = torch.from_numpy(ms).pin_memory()
        pin_al = torch.from_numpy(al).pin_memory()
        host = (pin_ms.numpy(), pin_al.numpy())
        one_step(T, args, L, RATES[0], *host)
        barrier()
        t1 = time.perf_counter()
        for k in range(args.steps):
            one_step(T, args, L, RATES[k % len(RATES)], *host)
        barrier()
        e2e_s = (time.perf_counter() - t1) / args.steps
        if world > 1:
            tt = torch.tensor([e2e_s], device="cuda")
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(tt.item())
        S = args.daughter_steps + 1
        e2e = {"value": atom_steps * world / e2e_s, "unit": "atom-steps/s",
               "h2d_bytes_per_step": int(ms.nbytes + al.nbytes + G * 8),
               # viscosity (9 x S doubles of the reduction) + per-daughter status/counters
               "d2h_bytes_per_step": int(9 * S * 8 + D * 16)}

    # the dominant kernel: the persistent daughter launch of one step
    k_ms = float(np.mean(kernel_ms))
    flops = float(np.mean(pairs)) / 2.0 * FLOPS_PER_PAIR
    achieved = flops / (k_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    traffic = D * (BULK_READ_PER_DAUGHTER + BULK_WRITE_PER_SAMPLE * (args.daughter_steps + 1))
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 5), "traffic": traffic,
                "kernel": "daughter_kernel", "kernel_ms": round(k_ms, 2),
                "spawn_ms": round(float(np.mean(spawn_ms)), 2),
                "peak_src": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz"}
    # the one exchange of the weak-scaled job: per-rate ensemble statistics
    # merged over ranks (each rank's groups are independent)
    eta = {}
    for g in RATES:
        if g not in per_rate:
            continue
        v, r = per_rate[g]
        if world > 1:
            from paper_2312_02990_gb300 import merge
            m = merge.merge_ranks(r, r["n_valid"], r["omega_mean"])
            eta[g] = (float(-m["ttcf"][-1] / g), float(m["ttcf_se"][-1] / g),
                      float(-m["dav"][-1] / g), float(m["dav_se"][-1] / g))
        else:
            eta[g] = (float(v["eta_ttcf"][-1]), float(v["eta_ttcf_se"][-1]),
                      float(v["eta_dav"][-1]), float(v["eta_dav_se"][-1]))
    sec.emit("viscosity_t_end", {f"{g:.0e}": {"eta_ttcf": e[0], "eta_ttcf_se": e[1], "eta_dav": e[2],
                                              "eta_dav_se": e[3]} for g, e in eta.items()})

    summary = {}
    # the oracle on a bounded sample: CPU baseline and per-rate parity
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = guarded("oracle", lambda: oracle_leg(T, args, N, L))
        if isinstance(res, tuple):
            cpu, chk = res
            summary["oracle_err"] = {k: [round(x["d_eta_over_se"], 4), float(f"{x['b_rel_max']:.2e}")]
                                     for k, x in chk["rates"].items()}
        else:
            chk = res
        sec.emit("oracle_check", chk)
    if rank == 0 and not args.no_sections:
        run_sections(T, torch, args, sec, summary, N, L, ms_dev, al_dev, eta, ms_step)
    sec.close()

    line = {
        "metric": "daughter atom-steps/s", "value": value, "unit": "atom-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "precision": "MIXED: FP32 pair forces, float-pair state, FP64 Omega/B/accumulation",
        "data": "synthetic (seeded FCC + Maxwell, GPU-thermalised mothers)",
        "config": {"workload": f"bulk WCA N={N}, {G} mother states x 4 mappings = {D} daughters x "
                               f"{args.daughter_steps} steps per step, one shear rate per step cycling "
                               "1e-1..1e-7",
                   "autotuned": None if not args.tuned else [args.tuned[0], args.tuned[1],
                                                             round(args.tuned[2], 4)],
                   "l2": "inputs larger than L2 (mothers 403 MB, series 131 MB per step)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons")},
        "eta_t_end": {f"{g:.0e}": [round(eta[g][0], 4), round(eta[g][1], 4)] for g in HEADLINE_RATES
                      if g in eta},
        "pairs_per_atom_step": round(float(np.mean(pairs)) / atom_steps, 4),
        **summary,
    }
    if rank == 0:
        out = json.dumps(line)
        if len(out) > 2000:   # keep the last line short: drop the extras first
            for k in ("pairs_per_atom_step", "cv", "uneven", "confined"):
                line.pop(k, None)
                out = json.dumps(line)
                if len(out) <= 2000:
                    break
        print(out, flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def guarded(name, fn):
    """Run one section; a failure is reported in its place and does not
    stop the benchmark (the result line is still printed)."""
    try:
        return fn()
    except Exception as e:   # noqa: BLE001 -- reported in the section's JSON
        return {"error": f"{type(e).__name__}: {e}"[:500], "section_failed": name}


def run_sections(T, torch, args, sec, summary, N, L, ms_dev, al_dev, eta, ms_step):
    """The long sections (rank 0), each emitted as it finishes; a compact
    digest of each goes into the result line."""
    try:
        _run_sections(T, torch, args, sec, summary, N, L, ms_dev, al_dev, eta, ms_step)
    except Exception as e:   # noqa: BLE001 -- the result line must still be printed
        summary["sections_error"] = f"{type(e).__name__}: {e}"[:200]


def _run_sections(T, torch, args, sec, summary, N, L, ms_dev, al_dev, eta, ms_step):
    if not args.no_plain:
        p = guarded("plain", lambda: plain_section(T, torch, args, N, L, ms_dev, al_dev))
        g = p.get("rate")
        if g in eta and "efficiency_plain_per_gpu_second" in p:   # efficiency 1/(Var(eta) T_GPU) of the benchmark step at that rate
            e_new = 1.0 / (eta[g][1] ** 2 * ms_step * 1e-3)
            p["efficiency_new_per_gpu_second"] = e_new
            p["efficiency_ratio_new_vs_plain"] = e_new / p["efficiency_plain_per_gpu_second"]
            summary["var_eff_vs_plain"] = round(p["efficiency_ratio_new_vs_plain"], 2)
        sec.emit("plain_gpu_ttcf", p)
    if not args.no_uneven:
        u = guarded("uneven", lambda: uneven_section(T, torch, args))
        if "value" in u:
            summary["uneven"] = {"value": float(f"{u['value']:.4g}"), "frac": round(u["roofline"]["frac"], 4),
                                 "daughters": u["daughters"]}
        sec.emit("uneven_batch", u)
    if not args.no_confined:
        c = guarded("confined", lambda: confined_section(T, torch, args))
        if "value" in c:
            summary["confined"] = {"value": float(f"{c['value']:.4g}"), "frac": round(c["roofline"]["frac"], 4),
                                   "daughters": c["daughters"]}
        sec.emit("confined", c)
    if not args.no_elong:
        el = guarded("elong", lambda: elong_section(T, torch, args))
        if "value" in el:
            summary["elong"] = {"value": float(f"{el['value']:.4g}"), "frac": round(el["roofline"]["frac"], 4),
                                "eta1_t_end": {k: [round(v[0], 3), round(v[1], 3)]
                                               for k, v in el["eta1_t_end"].items()},
                                "eta_shear_t_end": [round(x, 3) for x in el["eta_shear_t_end"]]}
        sec.emit("elongational", el)
    if not args.no_cv:
        cv = guarded("cv", lambda: cv_section(T, torch, args))
        if "variance_gain" in cv:
            summary["cv"] = {"gain": round(cv["variance_gain"], 3),
                             "eff": round(cv["efficiency_gain_cv_vs_same_kernels"], 3)}
        sec.emit("control_variate", cv)
    if not args.no_probe:
        pr = guarded("probe", probe_section)
        if pr.get("ffma_tflops_at_max_clock"):
            summary["fp32_probe_tflops"] = round(pr["ffma_tflops_at_max_clock"], 2)
        sec.emit("fp32_probe", pr)
    if not args.no_floor:
        sec.emit("precision_floor", guarded("floor", lambda: precision_floor_section(T, torch, args)))
    if not args.no_gk:
        sec.emit("green_kubo", guarded("gk", lambda: green_kubo_section(T, torch, args, N, L)))
    if not args.no_kick:
        sec.emit("kick_mothers", guarded("kick", lambda: kick_section(T, torch, args, N, L)))
    if not args.no_mapstudy:
        sec.emit("mapping_study", guarded("mapstudy", lambda: mapping_study_section(T, torch, args)))


def plain_section(T, torch, args, N, L, ms_dev, al_dev, n_groups=152, rate=1e-3):
    """Plain GPU TTCF: the same kernels in FP64 mode, one non-persistent
    launch per MD step (chunked runs of one step: state saved and reloaded,
    list rebuilt), no graph, no control variate, on n_groups of the
    benchmark's mother states at one rate.  Its own variance and time give
    its efficiency 1/(Var(eta_TTCF(t_end)) T_GPU), which does not depend on
    the number of groups (Var ~ 1/G, T ~ G)."""
    cfg = T.config_default()
    cfg.precision, cfg.n_steps, cfg.use_graph = T.TTCF_FP64, args.daughter_steps, 0
    with T.Context(cfg) as c:
        bid = c.spawn_daughters(ms_dev[:n_groups], al_dev[:n_groups], rate, box=L)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.daughter_steps):
            c.run(1)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        v = c.viscosity(bid)
    se = float(v["eta_ttcf_se"][-1])
    return {"rate": rate, "groups": n_groups, "daughter_steps": args.daughter_steps, "seconds": el,
            "atom_steps_per_s": 4 * n_groups * N * args.daughter_steps / el,
            "eta_ttcf": float(v["eta_ttcf"][-1]), "eta_ttcf_se": se,
            "efficiency_plain_per_gpu_second": 1.0 / (se * se * el),
            "definition": "FP64 mode, one non-persistent launch per MD step, no graph, no control variate"}


def uneven_section(T, torch, args):
    """The uneven batch: bulk WCA systems of N = 256, 864 and 4000 with
    shear rates 1e-2 ... 1e-6, 256 mother states per N (64 GPU mother chains
    x 4 states) x 4 mappings per (N, rate) cell = 15360 daughters of 1000
    steps in one graph-captured run (one persistent launch per size class
    on forked streams), launch shapes autotuned per N; MIXED."""
    from paper_2312_02990_gb300 import inputs
    moth = {}
    t0 = time.perf_counter()
    for N in UNEVEN_SIZES:
        L = inputs.bulk_box(N)
        moth[N] = make_mothers(T, args, 0, N, L, n_mothers=args.uneven_chains,
                               n_states=args.uneven_states, seed_off=30000 + N, n_eq=4000)
    t_moth = time.perf_counter() - t0
    cfg = T.config_default()
    cfg.precision, cfg.n_steps, cfg.use_graph = T.TTCF_MIXED, args.daughter_steps, 1
    with T.Context(cfg) as c:
        tuned = {}
        for N in UNEVEN_SIZES:
            ms = moth[N][0]
            tuned[N] = c.autotune(ms[:min(len(ms), 152)], inputs.bulk_box(N), shear_rate=1e-3, n_steps=100)[:3]
        dev = {N: (torch.from_numpy(moth[N][0]).cuda(), torch.from_numpy(moth[N][1]).cuda())
               for N in UNEVEN_SIZES}
        ids = {(N, g): c.spawn_daughters(*dev[N], g, box=inputs.bulk_box(N))
               for N in UNEVEN_SIZES for g in UNEVEN_RATES}
        c.run()
        st = c.get_stats()
        eta = {f"N{N}_{g:.0e}": float(c.viscosity(b)["eta_ttcf"][-1]) for (N, g), b in ids.items()}
        bad = int(sum(np.count_nonzero(c.group_status(b, len(moth[N][0]))) for (N, g), b in ids.items()))
    D = sum(4 * len(moth[N][0]) * len(UNEVEN_RATES) for N in UNEVEN_SIZES)
    atom_steps = sum(4 * len(moth[N][0]) * len(UNEVEN_RATES) * N for N in UNEVEN_SIZES) * args.daughter_steps
    k_ms = st["ms_run"]
    flops = st["pairs_interacting"] / 2.0 * FLOPS_PER_PAIR
    achieved = flops / (k_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    return {"value": atom_steps / (k_ms * 1e-3), "unit": "atom-steps/s", "daughters": D,
            "workload": f"bulk WCA N = {list(UNEVEN_SIZES)} x rates {UNEVEN_RATES}, "
                        f"{args.uneven_chains * args.uneven_states} mother states x 4 mappings per cell, "
                        f"{args.daughter_steps} steps, one graph-captured run, MIXED",
            "kernel_ms": k_ms, "launches": st["launches"],
            "autotuned": {str(N): [t[0], t[1], round(t[2], 4)] for N, t in tuned.items()},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": "daughter_kernel (3 size classes)"},
            "pairs_per_atom_step": st["pairs_interacting"] / atom_steps,
            "flagged_groups": bad, "mother_setup_s": t_moth, "eta_ttcf_t_end": eta}


ELONG_RATES = [1e-1, 1e-3, 1e-5]


def elong_section(T, torch, args):
    """Planar elongational flow (grad u = diag(eps, 0, -eps), deforming box)
    on the N=256 system: elong_chains x elong_states GPU mother states x the
    four mappings {identity, p -> -p, x <-> z, both} x daughter_steps steps
    at each rate of ELONG_RATES (one batch per rate, one run, MIXED); the
    same mothers sheared at 1e-3 give the shear viscosity, which the
    elongational viscosity eta_1 = -<P_xx - P_zz>/(4 eps) equals in the
    linear regime (an isotropic fluid: P_xx - P_zz is the shear stress of
    axes turned by 45 degrees)."""
    from paper_2312_02990_gb300 import inputs
    N = 256
    L = inputs.bulk_box(N)
    t0 = time.perf_counter()
    ms, al = make_mothers(T, args, 0, N, L, n_mothers=args.elong_chains, n_states=args.elong_states,
                          seed_off=50000, n_eq=4000)
    t_moth = time.perf_counter() - t0
    msd, ald = torch.from_numpy(ms).cuda(), torch.from_numpy(al).cuda()
    G = len(ms)
    cfg = T.config_default()
    cfg.system, cfg.precision = T.TTCF_BULK_WCA_ELONG, T.TTCF_MIXED
    cfg.n_steps, cfg.mapping_mask = args.daughter_steps, 0x30003
    with T.Context(cfg) as c:
        ids = {g: c.spawn_daughters(msd, ald, g, box=L) for g in ELONG_RATES}
        c.run()
        st = c.get_stats()
        eta = {}
        for g, b in ids.items():
            v = c.viscosity(b)
            eta[f"{g:.0e}"] = [float(v["eta_ttcf"][-1]), float(v["eta_ttcf_se"][-1]),
                               float(v["eta_dav"][-1]), float(v["eta_dav_se"][-1])]
        bad = int(sum(np.count_nonzero(c.group_status(b, G)) for b in ids.values()))
    scfg = T.config_default()
    scfg.precision, scfg.n_steps = T.TTCF_MIXED, args.daughter_steps
    with T.Context(scfg) as c:
        b = c.spawn_daughters(msd, ald, 1e-3, box=L)
        c.run()
        vs = c.viscosity(b)
    D = 4 * G * len(ELONG_RATES)
    atom_steps = D * N * args.daughter_steps
    k_ms = st["ms_run"]
    achieved = st["pairs_interacting"] / 2.0 * FLOPS_PER_PAIR / (k_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    return {"value": atom_steps / (k_ms * 1e-3), "unit": "atom-steps/s", "daughters": D,
            "workload": f"bulk WCA N = {N}, planar elongation at rates {ELONG_RATES}, {G} mother states "
                        f"x 4 mappings per rate, {args.daughter_steps} steps, one run, MIXED",
            "kernel_ms": k_ms, "launches": st["launches"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": "elong_kernel"},
            "pairs_per_atom_step": st["pairs_interacting"] / atom_steps,
            "eta1_t_end": {k: v[:2] for k, v in eta.items()},
            "eta1_dav_t_end": {k: v[2:] for k, v in eta.items()},
            "eta_shear_t_end": [float(vs["eta_ttcf"][-1]), float(vs["eta_ttcf_se"][-1])],
            "flagged_groups": bad, "mother_setup_s": t_moth}


def cv_section(T, torch, args):
    """Learned control variate on the N=256 system: train on 16384 groups
    (65536 daughters) at gamma = 1e-3, evaluate at gamma = 1e-6 on 4096
    disjoint groups with 65536 independent auxiliary mother states."""
    from paper_2312_02990_gb300 import inputs
    N = 256
    L = inputs.bulk_box(N)
    n_tr, n_ev, n_aux = args.cv_train_groups, args.cv_eval_groups, args.cv_aux
    total = n_tr + n_ev + n_aux
    n_moth = 64
    per = (total + n_moth - 1) // n_moth
    cfg = T.config_default()
    cfg.precision, cfg.n_steps = T.TTCF_MIXED, args.cv_steps
    t0 = time.perf_counter()
    with T.Context(cfg) as c:
        init = np.stack([inputs.initial_state(N, inputs.BASE_SEED + 50000 + k) for k in range(n_moth)])
        ms, al = c.sample_mothers(init, L, n_eq=args.n_eq, n_states=per, spacing=args.spacing)
    t_moth = time.perf_counter() - t0
    order = np.arange(n_moth * per).reshape(n_moth, per).T.ravel()
    ms, al = ms.reshape(-1, 6, N)[order], al.reshape(-1)[order]
    tr, ev = slice(0, n_tr), slice(n_tr, n_tr + n_ev)
    aux = slice(n_tr + n_ev, total)
    with T.Context(cfg) as c:
        bt = c.spawn_daughters(ms[tr], al[tr], 1e-3, box=L)
        be = c.spawn_daughters(ms[ev], al[ev], 1e-6, box=L)
        torch.cuda.synchronize()
        t = time.perf_counter()
        c.run()
        torch.cuda.synchronize()
        t_run = time.perf_counter() - t
        t = time.perf_counter()
        loss = c.cv_train(bt)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t
        # the auxiliary states are device-resident like the evaluation
        # daughters' mothers after their spawn (untimed copy)
        ms_aux = torch.from_numpy(np.ascontiguousarray(ms[aux])).cuda()
        al_aux = torch.from_numpy(np.ascontiguousarray(al[aux])).cuda()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = c.cv_apply(be, ms_aux, al_aux)
        torch.cuda.synchronize()
        t_apply = time.perf_counter() - t
    t_eval_run = t_run * n_ev / (n_tr + n_ev)
    # efficiency 1/(Var * T_GPU) of the evaluation estimate, with and without
    # the network's training time amortised into it
    e_plain = 1.0 / (r["se_plain"] ** 2 * t_eval_run)
    e_cv = 1.0 / (r["se_cv"] ** 2 * (t_eval_run + t_apply))
    e_cv_train = 1.0 / (r["se_cv"] ** 2 * (t_eval_run + t_apply + t_train))
    return {"eta_plain": r["eta_plain"], "se_plain": r["se_plain"], "eta_cv": r["eta_cv"],
            "se_cv": r["se_cv"], "c": r["c"], "variance_gain": r["gain"],
            "efficiency_gain_cv_vs_same_kernels": e_cv / e_plain,
            "efficiency_gain_cv_with_training": e_cv_train / e_plain,
            "train_loss_first_last": [float(loss[0]), float(loss[-1])],
            "groups": {"train": n_tr, "eval": n_ev, "aux": n_aux}, "daughter_steps": args.cv_steps,
            "seconds": {"mothers": t_moth, "run": t_run, "eval_run": t_eval_run, "train": t_train,
                        "apply": t_apply}}


def green_kubo_section(T, torch, args, N, L):
    """Zero-field cross-check of the TTCF viscosity: the Green-Kubo integral
    (V/T) int <P_xy(0)P_xy(t)> dt over 152 GPU mother chains of the same
    system (4000 thermalisation steps, then 20000 recorded steps), at the
    TTCF daughters' t_end; standard error over chains."""
    from paper_2312_02990_gb300 import inputs
    chains, n_eq, n, lag = 152, 4000, 20000, args.daughter_steps
    init = np.stack([inputs.initial_state(N, inputs.BASE_SEED + 70000 + k) for k in range(chains)])
    t0 = time.perf_counter()
    with T.Context(T.config_default()) as c:
        r = c.mother_acf(init, L, n_eq=n_eq, n_steps=n, max_lag=lag, want_series=True)
    el = time.perf_counter() - t0
    B = r["series"]
    V, dt, Tt = float(np.prod(L)), 0.0025, 0.722
    per = []
    for g in range(chains):   # each chain's own estimate, for the spread
        b = B[g]
        acf = np.array([np.mean(b[:n - k] * b[k:]) for k in range(0, lag + 1, 10)])
        per.append(V / Tt * float(np.sum(0.5 * (acf[1:] + acf[:-1])) * 10 * dt))
    return {"eta_gk_t_end": float(r["eta_gk"][-1]), "eta_gk_se": float(np.std(per, ddof=1) / np.sqrt(chains)),
            "t_end": lag * dt, "chains": chains, "steps_per_chain": n, "seconds": el}


def mapping_study_section(T, torch, args):
    """Mapping sets against the Eq. 4 correction: TTCF viscosity of the
    N=256 system at t = 2.5 from the same 256 mother states with the four
    mappings of Eq. 3 (<Omega(0)> = 0 in every group), identity plus
    x-reflection (cancels Omega(0) too), identity plus time reversal (does
    not: Omega(0) is even under p -> -p) and identity alone; each with the
    plain TTCF integrand and the Eq. 4 form <Omega(0)B(s)> -
    <Omega(0)><B(s)>; then the larger sets the paper lists after Eq. 3
    (component mirrors: Eq. 3 with z -> -z, all 16 mirror combinations, and
    all 32 with the x <-> z exchange), first with <B(0)> from the data (the library's
    estimator: the mappings make it exactly 0), then with <B(0)> set to its
    equilibrium value 0 (the integral alone; standard errors over mother
    groups from the daughters' series).  The cost-normalised error is
    SE x sqrt(daughters) (one daughter trajectory's worth of work)."""
    from paper_2312_02990_gb300 import inputs
    N, n_steps = 256, 1000
    L = inputs.bulk_box(N)
    rates = [1e-2, 1e-4, 1e-6]
    sets = {"eq3_all4": 0xF, "id_xrefl": 0x5, "id_trev": 0x3, "id_only": 0x1,
            # the further choices listed after Eq. 3: Eq. 3 with the z-mirror
            # (8 codes), every component mirror (16), and with the x <-> z
            # exchange (32); each set is closed under the x-reflection
            "eq3_zmirror8": 0x0F0F, "mirrors16": 0xFFFF, "mirrors_swap32": 0xFFFFFFFF}
    cfg = T.config_default()
    cfg.precision = T.TTCF_MIXED
    init = np.stack([inputs.initial_state(N, inputs.BASE_SEED + 91000 + k) for k in range(64)])
    with T.Context(cfg) as c:
        ms, al = c.sample_mothers(init, L, n_eq=4000, n_states=4, spacing=200)
    ms, al = ms.reshape(-1, 6, N), al.reshape(-1)
    G = ms.shape[0]
    out = {}
    for sname, mask in sets.items():
        cfg = T.config_default()
        cfg.precision, cfg.n_steps, cfg.mapping_mask = T.TTCF_MIXED, n_steps, mask
        M = bin(mask).count("1")
        res = {}
        with T.Context(cfg) as c:
            ids = [c.spawn_daughters(ms, al, g, box=L) for g in rates]
            c.run()
            for g, b in zip(rates, ids):
                B, om = c.daughter_series(b, G * M)
                row = {"daughters": G * M, "omega0_mean_over_sd": float(abs(om.mean()) / om.std())}
                for est, corr in (("plain", False), ("eq4", True)):
                    r = c.response(b, corrected=corr)
                    eta, se = -r["ttcf"][-1] / g, r["ttcf_se"][-1] / g
                    row[est] = {"eta": float(eta), "se": float(se),
                                "se_per_daughter": float(se * np.sqrt(G * M))}
                # the integral alone (<B(0)> = 0 imposed), per mother group
                dt = cfg.dt * cfg.sample_every
                I = dt * (0.5 * (B[:, 0] + B[:, -1]) + B[:, 1:-1].sum(axis=1))
                for est, corr in (("plain_b0_zero", False), ("eq4_b0_zero", True)):
                    x = om * I
                    if corr:
                        x = x - om.mean() * I.mean()
                    eg = -x.reshape(G, M).mean(axis=1) / g
                    se = float(eg.std(ddof=1) / np.sqrt(G))
                    row[est] = {"eta": float(eg.mean()), "se": se, "se_per_daughter": se * np.sqrt(G * M)}
                res[f"{g:.0e}"] = row
        out[sname] = res
    return {"workload": f"bulk WCA N=256, {G} mother states, {n_steps} steps (t = 2.5), MIXED",
            "results": out}


def kick_section(T, torch, args, N, L):
    """Further mother states from one thermalised state by small momentum
    kicks (ttcf_kick_states): device time of 152 kicked copies of one
    thermalised N=2048 state (kick 1e-6 sqrt(T), device buffers), and the
    number of steps after which the copies, run as GPU mother chains,
    spread in P_xy like independent equilibrium samples (90 % of the
    equilibrium spread, 20-step running mean)."""
    from paper_2312_02990_gb300 import inputs
    copies, kick, n_run = 152, 1e-6, 6000
    cfg = T.config_default()
    cfg.precision = T.TTCF_MIXED
    with T.Context(cfg) as c:
        st, _ = c.sample_mothers(inputs.initial_state(N, inputs.BASE_SEED + 90000), L, n_eq=4000,
                                 n_states=1, spacing=1)
        st = np.asarray(st).reshape(6, N)
        dev = torch.from_numpy(st).cuda()
        c.kick_states(dev, copies, kick, 1)            # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        cp = c.kick_states(dev, copies, kick, inputs.BASE_SEED)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = c.mother_acf(cp.cpu().numpy(), L, n_eq=0, n_steps=n_run, max_lag=10, want_series=True)
    ser = r["series"]
    eq = float(ser[:, -2000:].std())
    spread = np.convolve(ser.std(axis=0), np.ones(20) / 20, mode="valid")
    above = np.nonzero(spread >= 0.9 * eq)[0]
    return {"copies": copies, "kick": kick, "n_atoms": N, "kick_ms": ms,
            "bytes_written": copies * 6 * N * 8, "write_GB_per_s": copies * 6 * N * 8 / (ms * 1e-3) / 1e9,
            "decorrelation_steps": int(above[0]) if above.size else None,
            "decorrelation_time": float(above[0] * 0.0025) if above.size else None,
            "spread_at_start": float(spread[0] / eq), "thermalisation_steps_of_the_source": 4000,
            "note": "IEEE-double kernel (log, sin, cos per kick): bound by the FP64 pipe, not by HBM"}


def precision_floor_section(T, torch, args):
    """Signal, noise and precision floor across the shear rate (Eqs. 13-17):
    the N=256 system at every decade from 1e-1 to 1e-15, MIXED and FP64, on
    the same 256 mother states (64 GPU mother chains x 4 states), 4
    mappings, 4000 steps, read at t = 1.25 (transient: the four mapped
    daughters of a mother are still correlated, so the direct average's
    noise is still small) and t = 10 (past the chaotic decorrelation, the
    steady state the paper's analysis assumes).  Per rate and time:
    <P_xy> by TTCF and by direct average (DAV) with their standard errors
    over mother groups, the signal-to-noise ratios |<P_xy>|/SE,
    sigma(Omega(0)) over daughters, the standard error of the integrand
    <Omega(0) P_xy(t)>, the viscosities; and the log-log slopes against the
    rate over the linear regime (rate <= 1e-3) of sigma(Omega(0)), the
    integrand's SE and the SEs of <P_xy> by TTCF and DAV, which the paper's
    analysis (steady state) predicts as 1, 1, 1 and 0: SNR_TTCF flat and
    SNR_DAV proportional to the rate."""
    from paper_2312_02990_gb300 import inputs
    N, n_steps = 256, 4000
    L = inputs.bulk_box(N)
    rates = [10.0 ** -k for k in range(1, 16)]
    times = {"t1.25": 500, "t10": 4000}
    cfg = T.config_default()
    cfg.precision = T.TTCF_MIXED
    init = np.stack([inputs.initial_state(N, inputs.BASE_SEED + 90000 + k) for k in range(64)])
    with T.Context(cfg) as c:
        ms, al = c.sample_mothers(init, L, n_eq=4000, n_states=4, spacing=200)
    ms, al = ms.reshape(-1, 6, N), al.reshape(-1)
    D = 4 * ms.shape[0]
    out, slopes = {}, {}
    t0 = time.perf_counter()
    for name, prec in (("mixed", T.TTCF_MIXED), ("fp64", T.TTCF_FP64)):
        cfg = T.config_default()
        cfg.precision, cfg.n_steps = prec, n_steps
        with T.Context(cfg) as c:
            ids = [c.spawn_daughters(ms, al, g, box=L) for g in rates]
            c.run()
            res = {tk: {} for tk in times}
            for g, b in zip(rates, ids):
                v = c.viscosity(b)
                r = c.response(b)
                _, om = c.daughter_series(b, D)
                for tk, s in times.items():
                    res[tk][f"{g:.0e}"] = {
                        "eta_ttcf": float(v["eta_ttcf"][s]), "eta_ttcf_se": float(v["eta_ttcf_se"][s]),
                        "eta_dav": float(v["eta_dav"][s]), "eta_dav_se": float(v["eta_dav_se"][s]),
                        "pxy_ttcf": float(r["ttcf"][s]), "pxy_ttcf_se": float(r["ttcf_se"][s]),
                        "pxy_dav": float(r["dav"][s]), "pxy_dav_se": float(r["dav_se"][s]),
                        "snr_ttcf": float(abs(r["ttcf"][s]) / r["ttcf_se"][s]),
                        "snr_dav": float(abs(r["dav"][s]) / r["dav_se"][s]),
                        "sigma_omega0": float(np.std(om)), "integrand_se": float(r["corr_se"][s])}
            out[name] = res
        lin = [g for g in rates if g <= 1e-3]
        lg = np.log10(lin)
        slopes[name] = {}
        for tk in times:
            def slope(key):
                y = np.array([res[tk][f"{g:.0e}"][key] for g in lin])
                return float(np.polyfit(lg, np.log10(y), 1)[0]) if np.all(y > 0) else None
            slopes[name][tk] = {k: slope(k) for k in ("sigma_omega0", "integrand_se", "pxy_ttcf_se", "pxy_dav_se")}
    return {"workload": f"bulk WCA N=256, {ms.shape[0]} mother states x 4 mappings, {n_steps} steps, "
                        "read at t = 1.25 and t = 10, rates 1e-1 ... 1e-15",
            "snr": "|<P_xy(t)>| / its standard error over mother groups",
            "seconds": time.perf_counter() - t0,
            "slopes_rate_le_1e-3": slopes, "results": out}


def confined_section(T, torch, args):
    """Confined channel of Example 2 (6048 fluid + 4200 tethered wall atoms,
    dt = 0.005): GPU-thermalised mothers (lattices at rest; 64 chains x 4
    states = 256 mother states), then every mother x 4 mappings x 4 shear
    rates 1e-1 ... 1e-7 = 4096 daughters of conf_steps steps in one
    persistent launch.  Reports daughter atom-steps/s of that launch, the
    wall-stress responses and the slip velocity and friction coefficient of
    Eq. 12 at t_end (TTCF and direct average)."""
    from paper_2312_02990_gb300 import inputs
    sysd = inputs.confined_system()
    N, box = sysd["state"].shape[1], sysd["box"]
    cfg = T.config_default()
    cfg.system, cfg.precision = T.TTCF_CONFINED_LJ, T.TTCF_MIXED
    cfg.dt, cfg.T, cfg.tau_T = 0.005, 1.0, 0.25
    cfg.n_steps, cfg.sample_every = args.conf_steps, 10
    rng = np.random.default_rng(inputs.BASE_SEED + 777)
    init = np.repeat(sysd["state"][None], args.conf_chains, axis=0)
    # independent chains: fresh Maxwell momenta per chain (same temperature)
    init[:, 3:] = rng.standard_normal((args.conf_chains, 3, N))
    for t in (0, 1, 2):
        sel = sysd["types"] == t
        init[:, 3:, sel] -= init[:, 3:, sel].mean(axis=2, keepdims=True)
    t0 = time.perf_counter()
    with T.Context(cfg) as c:
        ms, al, cs = c.sample_mothers_confined(init, sysd["types"], sysd["lattice"], box,
                                               n_eq=args.conf_eq, n_states=args.conf_states,
                                               spacing=args.conf_spacing, allow_numeric=True)
    t_moth = time.perf_counter() - t0
    # a chain in which a fluid atom entered a wall is dropped
    keep = cs == 0
    ms, al = ms[keep].reshape(-1, 6, N), al[keep].reshape(-1)
    G = ms.shape[0]
    with T.Context(cfg) as c:
        ids = [c.spawn_confined(ms, sysd["types"], sysd["lattice"], box, al, g) for g in CONF_RATES]
        # a group whose daughter fails (e.g. a fluid atom pushed through a
        # wall at the highest rate) is excluded from the averages and counted
        c.run(allow_numeric=True)
        st = c.get_stats()
        resp = {}
        for g, b in zip(CONF_RATES, ids):
            gs = c.group_status(b, G)
            top = c.response_obs(b, 1)
            bot = c.response_obs(b, 0)
            fr = [c.friction(b, w) for w in (0, 1)]
            resp[f"{g:.0e}"] = {"slip_top_ttcf": float(fr[1]["slip_ttcf"][-1]),
                                "slip_top_dav": float(fr[1]["slip_dav"][-1]),
                                "xi_top_ttcf": float(fr[1]["xi_ttcf"][-1]),
                                "xi_top_dav": float(fr[1]["xi_dav"][-1]),
                                "xi_bottom_ttcf": float(fr[0]["xi_ttcf"][-1]),
                                "wall_stress_top_ttcf": float(top["ttcf"][-1]),
                                "wall_stress_top_ttcf_se": float(top["ttcf_se"][-1]),
                                "wall_stress_top_dav": float(top["dav"][-1]),
                                "wall_stress_top_dav_se": float(top["dav_se"][-1]),
                                "wall_stress_bottom_ttcf": float(bot["ttcf"][-1]),
                                "wall_stress_bottom_ttcf_se": float(bot["ttcf_se"][-1]),
                                "excluded_groups": int(np.count_nonzero(gs)),
                                "status_flags": int(np.bitwise_or.reduce(gs))}
    # the equilibrium friction coefficient xi_0 (Eq. 12 by the equilibrium
    # method): the same mother states run at zero shear with one mapping are
    # equilibrium trajectories; slip/force correlations over t = 10 (every
    # 5th step), Maxwell fit of the friction kernel
    eq_cfg = T.config_default()
    eq_cfg.system, eq_cfg.precision = T.TTCF_CONFINED_LJ, T.TTCF_MIXED
    eq_cfg.dt, eq_cfg.T, eq_cfg.tau_T = 0.005, 1.0, 0.25
    eq_cfg.n_steps, eq_cfg.sample_every, eq_cfg.mapping_mask = args.conf_eq_steps, 5, 1
    n_eq_ch = min(G, 152)
    t0 = time.perf_counter()
    with T.Context(eq_cfg) as c:
        bid = c.spawn_confined(ms[:n_eq_ch], sysd["types"], sysd["lattice"], box, al[:n_eq_ch], 0.0)
        c.run(allow_numeric=True)
        lag = min(400, args.conf_eq_steps // 5 - 1)
        svals = np.linspace(0.05, 1.0, 20)
        eq = [c.friction_equilibrium(bid, w, lag, svals) for w in (0, 1)]
    t_eq = time.perf_counter() - t0
    friction_eq = {"xi0_bottom": float(eq[0]["xi0"]), "xi0_top": float(eq[1]["xi0"]),
                   "tau_m": [float(eq[0]["tau_m"]), float(eq[1]["tau_m"])],
                   "xi_ratio_unfitted": [float(eq[0]["xi_ratio"]), float(eq[1]["xi_ratio"])],
                   "chains": n_eq_ch, "steps": args.conf_eq_steps, "max_lag_time": lag * 5 * 0.005,
                   "laplace_s": [0.05, 1.0, 20], "seconds": t_eq}
    D = 4 * G * len(CONF_RATES)
    atom_steps = float(D) * N * args.conf_steps
    k_ms = st["ms_run"]
    flops = st["pairs_interacting"] / 2.0 * FLOPS_PER_PAIR_LJ
    achieved = flops / (k_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    return {"value": atom_steps / (k_ms * 1e-3), "unit": "atom-steps/s", "daughters": D,
            "workload": f"confined LJ channel N={N} ({sysd['n_fluid']} fluid + {sysd['n_wall']} wall), "
                        f"{G} mother states x 4 mappings x {len(CONF_RATES)} shear rates = {D} daughters "
                        f"x {args.conf_steps} steps (dt 0.005), MIXED",
            "kernel_ms": k_ms,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": "conf_kernel",
                         "traffic": CONF_BYTES_PER_ATOM_STEP * atom_steps,
                         "algorithmic": "unique interacting pairs x 25 FP32 flops"},
            "pairs_per_atom_step": st["pairs_interacting"] / atom_steps,
            "rebuilds_per_daughter_step": st["rebuilds"] / (D * args.conf_steps),
            "mother_setup_s": t_moth, "mother_chains_dropped": int(np.count_nonzero(~keep)),
            "friction_equilibrium": friction_eq, "responses_t_end": resp}


def probe_section():
    """FP32 throughput measured on this GPU by the instruction-rate probe
    (FFMA chains, clock64 per SM and CUDA events): a measured companion to
    the derived FP32 peak of the roofline."""
    cc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(PROBE_SRC) or not os.path.exists(cc):
        return {"error": "probe source or nvcc missing"}
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "alu_rates")
        r = subprocess.run([cc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, PROBE_SRC],
                           capture_output=True, text=True)
        if r.returncode != 0:
            return {"error": "probe build failed"}
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    out = {"raw": [ln for ln in r.stdout.splitlines() if ln.strip()][:20]}
    for ln in r.stdout.splitlines():
        m = re.match(r"(FFMA f32|FFMA2 \(2 FMA per instr\)|DFMA f64)\s+thread-ops/clk/SM=\s*([\d.]+).*"
                     r"Gop/s=\s*([\d.]+).*MHz~(\d+)", ln)
        if m:
            key = {"FFMA f32": "ffma", "DFMA f64": "dfma"}.get(m.group(1), "ffma2")
            out[f"{key}_per_clk_sm"] = float(m.group(2))
            out[f"{key}_gops"] = float(m.group(3))
            out[f"{key}_mhz"] = float(m.group(4))
    if "ffma_per_clk_sm" in out:
        out["ffma_tflops_at_max_clock"] = out["ffma_per_clk_sm"] * 2 * N_SM * SM_MAX_MHZ * 1e6 / 1e12
    return out


# -------------------------------------------------------------- oracle --
def oracle_mothers(N, n_groups, n_eq, threads, seed_off=0):
    """Oracle-thermalised mother states (one chain each, untimed)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_2312_02990_gb300 import inputs
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))

    def one(k):
        return oracle.mother(b, inputs.initial_state(N, inputs.BASE_SEED + 7 * k + seed_off), n_eq=n_eq,
                             n_states=1, spacing=1)

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, range(n_groups)))
    return b, np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


def oracle_leg(T, args, N, L):
    """The FP64 CPU oracle on a bounded sample of the benchmark workload:
    oracle-made mothers x 4 mappings x 1000 steps at the rates 1e-1, 1e-3
    and 1e-7 (timed: the CPU baseline), then the GPU on the same inputs in
    the benchmark's launch configuration, and the error of each GPU result
    against the oracle (per rate: TTCF viscosity at t_end in units of the
    sample's standard error, and the largest relative B(s) difference)."""
    import oracle
    threads = os.cpu_count() or 1
    Go, n = args.oracle_groups, args.daughter_steps
    rates = list(HEADLINE_RATES)
    b, ms, al = oracle_mothers(N, Go, args.oracle_eq, threads)
    msr = np.ascontiguousarray(np.concatenate([ms] * len(rates)))
    alr = np.concatenate([al] * len(rates))
    gm = np.repeat(rates, Go)
    t = time.perf_counter()
    Bo, Omo = oracle.daughters(b, msr, alr, gm, n, n_threads=threads)
    el = time.perf_counter() - t
    D = 4 * Go * len(rates)
    cpu = {"value": D * N * n / el, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
           "sample": f"{D} daughters x {n} steps, N={N}, rates 1e-1/1e-3/1e-7 ({el:.1f} s)"}
    with T.Context(bench_config(T, args)) as c:
        ids = [c.spawn_daughters(ms, al, g, box=L) for g in rates]
        c.run()
        gpu = [(c.daughter_series(bid, 4 * Go), c.viscosity(bid)) for bid in ids]
    out = {}
    for k, (g, ((B, Om), v)) in enumerate(zip(rates, gpu)):
        sl = slice(4 * Go * k, 4 * Go * (k + 1))
        ro = oracle.viscosity(oracle.responses(Bo[sl], Omo[sl], 4, b.dt), g)
        d = abs(float(v["eta_ttcf"][-1]) - float(ro["eta_ttcf"][-1]))
        se = float(ro["eta_ttcf_se"][-1])
        out[f"{g:.0e}"] = {"eta_gpu": float(v["eta_ttcf"][-1]), "eta_oracle": float(ro["eta_ttcf"][-1]),
                           "eta_se_sample": se, "d_eta": d, "d_eta_over_se": d / se,
                           "b_rel_max": float(np.abs(B - Bo[sl]).max() / np.abs(Bo[sl]).max()),
                           "omega_rel_max": float(np.abs(Om - Omo[sl]).max() / np.abs(Omo[sl]).max())}
    chk = {"groups": Go, "daughters_per_rate": 4 * Go, "steps": n, "mother_eq_steps": args.oracle_eq,
           "note": "same oracle-made inputs on both sides; GPU in the benchmark's launch configuration",
           "rates": out}
    return cpu, chk


def bench_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host
    cores, on a bounded sample of the same workload per step (rates in
    turn, as in the GPU arm)."""
    rank, world, local = dist_info()
    if rank != 0:
        return
    import oracle
    N = args.n_atoms
    threads = os.cpu_count() or 1
    groups = max(1, threads // 4)
    steps = 200
    b, ms, al = oracle_mothers(N, groups, 600, threads, seed_off=5)
    vals = []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        oracle.daughters(b, ms, al, RATES[k % len(RATES)], steps, n_threads=threads)
        el = time.perf_counter() - t
        if k >= args.warmup:
            vals.append(el)
    el = float(np.mean(vals))
    v = 4 * groups * N * steps / el
    line = {"impl": "reference", "metric": "daughter atom-steps/s", "value": v,
            "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded FCC + Maxwell, oracle-thermalised mothers)",
            "config": {"workload": f"bulk WCA N={N}, 4096 mother states x 4 mappings = 16384 daughters x "
                                   f"{args.daughter_steps} steps per step, one shear rate per step cycling "
                                   "1e-1..1e-7"},
            "cpu_baseline": {"value": v, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"bounded sample per step: {4 * groups} daughters x {steps} steps"},
            "e2e": {"value": v, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        bench_reference(args)
    elif args.only:
        import torch

        from paper_2312_02990_gb300 import inputs
        from paper_2312_02990_gb300 import ttcf as T
        T.load(build_if_missing=True)
        args.tuned = None
        N = args.n_atoms
        L = inputs.bulk_box(N)
        fn = {"confined": lambda: confined_section(T, torch, args),
              "uneven": lambda: uneven_section(T, torch, args),
              "cv": lambda: cv_section(T, torch, args),
              "floor": lambda: precision_floor_section(T, torch, args),
              "gk": lambda: green_kubo_section(T, torch, args, N, L),
              "kick": lambda: kick_section(T, torch, args, N, L),
              "mapstudy": lambda: mapping_study_section(T, torch, args),
              "probe": probe_section,
              "elong": lambda: elong_section(T, torch, args)}[args.only]
        print(json.dumps(fn()))
    else:
        bench_gb300(args)


if __name__ == "__main__":
    main()
