"""Benchmark of the phasor-PIC hot path on B300.

A step is one RF period of one argon ICP cell: N_RF = 400 PIC steps (field
reconstruction, fused gather/Boris/MCC/deposit kernel, ionisation append,
Poisson refinement, turn charges and harmonic accumulation, counting sorts)
plus the period end (two plasma-only Helmholtz solves, back-emf, displacement
currents, powers, controller, network solve, relaxation, field composition).
The metric is particle-steps per second: live macroparticles pushed, summed
over all PIC steps, divided by the device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cell60]
  python bench.py --impl reference ...    # the FP64 CPU oracle on host cores

Under torchrun (N > 1) every rank advances its own independent cell (seed
offset by rank; cells share nothing), the timing is the max over ranks and
`value` is the particle-steps of all ranks divided by that time.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and time-to-stationary-state vs plain FP64 PIC, 1 B300"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = 52      # read cell,dr,dz,vr,vt,vz,uid (28 B) + write 6 x 4 B


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cell60")
    ap.add_argument("--cpu-steps", type=int, default=1, help="PIC steps of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(ms, psteps, dist):
    """Whole-job timing: the max of the per-rank device times and the sum of
    the particle-steps of all ranks (CPU tensors, any backend)."""
    import torch
    if dist is None:
        return ms, float(psteps)
    t = torch.tensor([ms], dtype=torch.float64)
    p = torch.tensor([float(psteps)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0]), float(p[0])


def workload_desc(cfg, name):
    return ("%s: %dx%d cells over r<=%.2f m, z<=%.2f m, %d macroparticles/species, %d turns, Ar %.0f mTorr, "
            "dt=T/%d%s" % (name, cfg.nr, cfg.nz, cfg.r_max, cfg.z_max, cfg.n_init, len(cfg.turn_r),
                           cfg.pressure_pa / 133.322368 * 1e3, round(1 / (cfg.freq * cfg.dt)),
                           (", controller target %.0f W" % cfg.p_target) if cfg.power_control else ""))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
                for k, n in enumerate(names):
                    if s[5 + k].lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline inputs
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def push_kernel_hash():
    src = open(os.path.join(ROOT, "paper_2609_15043_b300", "csrc", "pp_particles.cu"), "rb").read()
    return hashlib.sha1(src).hexdigest()[:12]


def profiled_traffic(workload):
    """DRAM bytes per push-kernel launch from the committed ncu summary, valid
    only while the kernel source is unchanged (hash recorded in the summary)."""
    path = os.path.join(ROOT, "profiles", "push_kernel_%s.md" % workload)
    try:
        txt = open(path).read()
    except OSError:
        return None
    h = re.search(r"kernel_source_sha1:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not t or h.group(1) != push_kernel_hash():
        return None
    return float(t.group(1))


# ---------------------------------------------------------------- CPU oracle
def make_oracle(cfg):
    from oracle.cell import OracleCell
    from paper_2609_15043_b300 import workloads
    w = workloads.macro_weight(cfg)
    oc = OracleCell(cfg, [w, w])
    for sp in (0, 1):
        p = workloads.population(cfg, sp)
        oc.set_particles(sp, p["cell"].astype(np.int64), p["dr"].astype(np.float64), p["dz"].astype(np.float64),
                         p["vr"].astype(np.float64), p["vt"].astype(np.float64), p["vz"].astype(np.float64),
                         p["uid"])
    oc.prime(np.float64)
    return oc


def time_oracle(oc, steps):
    """Times `steps` FP64 oracle PIC steps; returns (seconds, particle-steps)."""
    t0 = time.perf_counter()
    pushed = 0
    for _ in range(steps):
        pushed += oc.step(np.float64)["stats"]["pushed"]
    return time.perf_counter() - t0, pushed


def cpu_baseline(cfg, args):
    oc = make_oracle(cfg)
    dt, pushed = time_oracle(oc, args.cpu_steps)
    return {"value": pushed / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d PIC step(s) of the full workload (%d particle-steps, %.1f s), FP64 numpy/scipy "
                      "oracle, single thread; host has %d cores" % (args.cpu_steps, pushed, dt, os.cpu_count())}


def run_reference(args, cfg, ws, rank):
    """The reference arm is the oracle itself on the host cores: each bench
    step is `--cpu-steps` oracle PIC steps of the same workload (a bounded
    sample; a whole RF period would take hours)."""
    if rank != 0:
        return
    oc = make_oracle(cfg)
    for _ in range(min(args.warmup, 1)):
        time_oracle(oc, 1)
    total_t, total_p = 0.0, 0
    for _ in range(args.steps):
        dt, pushed = time_oracle(oc, args.cpu_steps)
        total_t += dt
        total_p += pushed
    value = total_p / total_t
    sample = ("%d x %d PIC step(s) of the full workload after %d warm-up step(s), FP64 numpy/scipy oracle, "
              "single thread; host has %d cores" % (args.steps, args.cpu_steps, min(args.warmup, 1),
                                                    os.cpu_count()))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(cfg, args.workload),
                       "step": "%d oracle PIC step(s) per bench step" % args.cpu_steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_ours(args, cfg, ws, rank, local):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the product path has no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        # timing reductions run on CPU tensors: gloo for them, no data-path collective
        dist.init_process_group("gloo")
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = cfg.replace(seed=cfg.seed + rank)
    cell = pp.Cell(cfg)
    for sp in (0, 1):
        cell.set_particles(sp, workloads.population(cfg, sp))
    stream = torch.cuda.default_stream()
    sh = stream.cuda_stream
    cell.prime(sh)
    for _ in range(args.warmup):
        cell.advance_period(1, sh)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed region: K periods, inputs resident in HBM
    c0 = cell.counters()
    l0 = pp.launch_count()
    cell.set_profiling(True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        cell.advance_period(1, sh)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    phases = cell.phase_times()
    cell.set_profiling(False)
    launches = pp.launch_count() - l0
    c1 = cell.counters()
    psteps = c1["particle_steps"] - c0["particle_steps"]
    ms_all, ps_all = reduce_over_ranks(ms, psteps, dist)
    value = ps_all / (ms_all / 1e3)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        barrier()
        c2 = cell.counters()
        x, vg = cell.circuit_state()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            cell.set_circuit_state(x, vg)            # host -> device: 16(2N+1) + 8 B
            cell.advance_period(1, sh)
            rec = cell.turn_phasors(sh)              # device -> host: the period record
            x, vg = rec["x_next"], rec["vg_next"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        c3 = cell.counters()
        n = len(cfg.turn_r)
        e2e = {"value": (c3["particle_steps"] - c2["particle_steps"]) / dt, "unit": UNIT,
               "h2d_bytes_per_step": 16 * (2 * n + 1) + 8,
               "d2h_bytes_per_step": pp.C.sizeof(pp.PPRecord) + 4}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    push_ms, push_n = phases["push"]
    per_launch_particles = psteps / max(push_n, 1)
    achieved = BYTES_PER_PARTICLE_STEP * per_launch_particles / (push_ms / push_n / 1e3) / 1e9
    traffic = profiled_traffic(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 particles, f64 fields/circuit",
        "data": "synthetic",
        "config": {"workload": workload_desc(cfg, args.workload),
                   "step": "one RF period: %d PIC steps + period end" % cell.n_rf,
                   "l2": "inputs larger than L2 (%.0f MB of particle state)" % (
                       2 * cfg.n_init * 28 / 1e6),
                   "parallelism": "independent cell per GPU" if ws > 1 else "1 cell",
                   "time_to_stationary": None},
        "roofline": {"bound": "hbm", "kernel": "push_kernel", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "measured" if peaks else "fallback",
                     "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
                     "avg_launch_ms": push_ms / max(push_n, 1)},
        "phase_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args)
    print(json.dumps(line), flush=True)
    cell.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_env()
    from paper_2609_15043_b300 import workloads
    cfg = workloads.WORKLOADS[args.workload]()
    if args.impl == "reference":
        run_reference(args, cfg, ws, rank)
    else:
        run_ours(args, cfg, ws, rank, local)


if __name__ == "__main__":
    main()
