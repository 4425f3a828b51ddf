"""Benchmark: DoF-steps/s of the DG acoustic solver on a GB300.

Workload (one GPU): unit cube split into 32^3 curved hexahedra, degree k = 5
(28,311,552 DoF counting p, v_x, v_y, v_z), variable rho and c, reflecting
walls, Gaussian pressure pulse, FP64.  One bench step advances one state by
one LSRK(5,4) time step and another by one ADER time step (order k+1 = 6,
degree reduction every second derivative) at the same dt (Cr = 0.1), so a
step processes 2 x 28.3M DoF-steps and runs every kernel of the hot path.

Timing: W untimed warm-up steps, then K steps of each method (one stepper
call per method, as a solve runs) bracketed by a barrier and a device
synchronisation, timed with CUDA events on the launching stream; the max over
ranks is reported.  The state (226 MB) and geometry (1.8 GB) are
larger than L2, so no flush is needed between steps.  Per-kernel device time
comes from the library's own event profiling on the same stream.

e2e: every step, per method, dg_solve_host copies the state from pinned host
memory to the device, advances one step and copies it back (also reported:
K steps per dg_solve_host call).

--impl reference: the FP64 CPU oracle on a bounded sample of the same recipe
(4^3 elements), one LSRK and one ADER step per bench step, single thread.

Multi-GPU (torchrun, N > 1): every rank runs its own replica of the
workload; value = DoF-steps of all ranks / max time over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF-steps/s at fixed L2 error (ADER/LSRK, FP32/FP64); served p99 latency"
UNIT = "DoF-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Derived FP pipe peaks of a GB300 (152 SMs, 2070 MHz maximum SM clock):
# FP64: 2 FMA/clk/SM (the nominal 1.25 TFLOP/s) -> 152 * 2 * 2 * 2.07e9;
# FP32: 128 FMA/clk/SM -> 152 * 128 * 2 * 2.07e9.
FP64_PEAK = 152 * 2 * 2 * 2.07e9
FP32_PEAK = 152 * 128 * 2 * 2.07e9
HBM_FALLBACK = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--size", type=int, default=32, help="elements per axis")
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--tiling", default="", help="elements per block 'op,tck' instead of autotuning")
    ap.add_argument("--basis", default="g", choices=["g", "gl"],
                    help="state inside the steppers: g = Gauss-point values (default), gl = the paper's storage")
    ap.add_argument("--pred", default="auto", choices=["auto", "lines", "columns"],
                    help="predictor kernel for Gauss-point states (dg_set_predictor_kernel)")
    ap.add_argument("--workload", default="curved_pulse",
                    choices=["curved_pulse", "plane_wave", "batched", "served", "reduction",
                             "time_to_accuracy", "time_to_accuracy_2d", "basis_change"])
    ap.add_argument("--lam", type=float, default=20.0, help="served: arrivals per second")
    ap.add_argument("--duration", type=float, default=10.0, help="served: arrival window, seconds")
    ap.add_argument("--nrange", default="8,24", help="served: elements per axis, min,max")
    ap.add_argument("--srange", default="100,400", help="served: ADER steps per request, min,max")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--active-dof", type=float, default=3e8,
                    help="served: admit while active solves hold fewer DoFs than this (0 = budget only)")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--autotune", default="", help="autotune table (JSON) to apply to every solver")
    ap.add_argument("--accuracy", type=int, default=0,
                    help="instead of timing: run this many steps of each method in FP32 and FP64 "
                         "and report the relative l2 differences and errors against the exact plane wave")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32, batched and served forms measured beside the headline")
    ap.add_argument("--batch-steps", type=int, default=500,
                    help="batched form: ADER steps of every instance (500 in the configured workload)")
    ap.add_argument("--cpu-steps", type=int, default=0,
                    help="steps of the oracle's sample (default: 20 on the 4^3 curved pulse, 2 on larger samples)")
    ap.add_argument("--cpu-size", type=int, default=0,
                    help="elements per axis of the oracle's sample (default 4 curved pulse, 16 plane wave)")
    ap.add_argument("--kset", default="1,4,7", help="time_to_accuracy: degrees")
    ap.add_argument("--t-end", type=float, default=1.0, help="time_to_accuracy: end time")
    return ap.parse_args()


def workload(N, k, name="curved_pulse"):
    import synth
    if name == "plane_wave":
        return synth.configs.plane_wave(N=N, k=k)
    return synth.configs.curved_pulse(N=N, k=k, nsteps=200)


def workload_desc(N, k, prec, name="curved_pulse"):
    dof = 4 * (k + 1) ** 3 * N ** 3
    if name == "plane_wave":
        return (f"plane_wave: periodic unit cube, {N}^3 affine hexahedra, k={k} ({dof} DoF), rho=c=1, "
                f"p=cos(4 pi (x+y+z) - w t), Cr=0.1; bench step = 1 LSRK(5,4) step + 1 ADER(order "
                f"{k + 1}, reduction every 2nd derivative) step, {prec.upper()}")
    return (f"curved_pulse: unit cube, {N}^3 curved hexahedra (x_i += 0.05 prod sin 2 pi x_j), "
            f"k={k} ({dof} DoF), c=1+0.5 sin2pix cos2piy, rho=1+0.3 cos2piz, walls, Gaussian "
            f"pulse sigma=0.05 (seed 2), Cr=0.1; bench step = 1 LSRK(5,4) step + 1 ADER(order {k + 1}, "
            f"reduction every 2nd derivative) step, {prec.upper()}")


# ------------------------------------------------------------------ ranks
def reduce_max(x, world, device):
    """Max of a float over all ranks of the default process group."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ms_max, world):
    """Whole-job throughput: every rank's units over the slowest rank's time
    (replicas: each rank runs the same workload)."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.proc, self.path = dev, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import synth, oracle
cfg = (synth.configs.plane_wave(N={n}, k={k}) if {workload!r} == "plane_wave"
       else synth.configs.curved_pulse(N={n}, k={k}))
o = oracle.Oracle(cfg["mesh"], {k}, cfg["rho"], cfg["c"], 1.0)
U1 = cfg["U0"].copy(); U2 = cfg["U0"].copy()
for _ in range({warm}):
    U1 = o.lsrk(U1, cfg["dt"], 1); U2 = o.ader(U2, cfg["dt"], 1, 2)
while time.time() < {t_start}:
    time.sleep(0.01)
times = []
w0 = time.time()
for _ in range({steps}):
    t0 = time.perf_counter()
    U1 = o.lsrk(U1, cfg["dt"], 1); U2 = o.ader(U2, cfg["dt"], 1, 2)
    times.append(time.perf_counter() - t0)
print(json.dumps({{"times": times, "dof": int(U1.size), "w0": w0, "w1": time.time()}}))
"""


def run_oracle(n, k, warm, steps, workload="curved_pulse", procs=1, start_delay=0.0):
    """The oracle as it stands, one LSRK and one ADER step per timed step,
    on ``procs`` host cores at once: that many independent single-threaded
    copies of the same sample, started together (each waits for a common
    wall-clock start after its set-up).  Returns (DoF-steps/s of all copies
    over the span from the first start to the last end, that span, details)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t_start = time.time() + start_delay if procs > 1 else 0.0
    code = CPU_SNIPPET.format(root=ROOT, n=n, k=k, warm=warm, steps=steps, workload=workload, t_start=t_start)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    outs = []
    for p in ps:
        so, se = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle run failed: " + se[-2000:])
        outs.append(json.loads(so.strip().splitlines()[-1]))
    if procs == 1:
        total = sum(outs[0]["times"])
    else:
        total = max(o["w1"] for o in outs) - min(o["w0"] for o in outs)
    work = sum(2 * o["dof"] * len(o["times"]) for o in outs)
    return work / total, total, {"procs": procs, "per_copy_seconds": [sum(o["times"]) for o in outs]}


def cpu_sample_desc(n, k, steps, workload="curved_pulse", procs=1):
    who = ("numpy, 1 thread" if procs == 1 else
           f"numpy, {procs} single-threaded copies of the sample running at once, one per host core")
    return (f"FP64 oracle (dense element matrices, {who}) on the {n}^3-element instance of "
            f"the same {workload} recipe (k={k}, {4 * (k + 1) ** 3 * n ** 3} DoF): {steps} steps of 1 LSRK + "
            f"1 ADER step, oracle set-up excluded")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(n, k, steps, workload):
    """The oracle on every host core, with the single-thread figure beside it."""
    cores = host_cores()
    v1, t1, _ = run_oracle(n, k, 1, steps, workload)
    vp, tp, det = run_oracle(n, k, 1, steps, workload, procs=cores, start_delay=15.0 + 0.2 * cores)
    return {"value": vp, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": cpu_sample_desc(n, k, steps, workload, cores), "seconds": tp,
            "single_thread": {"value": v1, "cores": 1, "seconds": t1,
                              "sample": cpu_sample_desc(n, k, steps, workload)},
            "per_copy_seconds": det["per_copy_seconds"]}


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = 4
    cores = host_cores()
    value, total, det = run_oracle(n, args.k, args.warmup, args.steps, procs=cores, start_delay=15.0 + 0.2 * cores)
    sample = cpu_sample_desc(n, args.k, args.steps, procs=cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_desc(args.size, args.k, "fp64"),
                                        "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ shared timing
def make_solver(args, cfg, prec, dgw, basis=None, pred=None, tiling=None):
    """A solver on cfg in the bench's configuration: state basis, predictor
    form, and elements per block autotuned for this workload (results do not
    depend on the tiling)."""
    from paper_1805_03981_gb300 import autotune
    basis = args.basis if basis is None else basis
    pred = args.pred if pred is None else pred
    tiling = args.tiling if tiling is None else tiling
    s = dgw.Solver(cfg["mesh"], cfg["k"], prec, cfg["alpha"], cfg["rho"], cfg["c"])
    s.set_basis(dgw.BASIS_G if basis == "g" else dgw.BASIS_GL)
    s.set_predictor_kernel({"auto": dgw.PRED_AUTO, "lines": dgw.PRED_LINES, "columns": dgw.PRED_COLUMNS}[pred])
    if tiling:
        s.set_tiling(*(int(x) for x in tiling.split(",")))
    else:
        for kind in (dgw.KIND_LSRK, dgw.KIND_TCK):
            s.tune(kind, autotune.CANDIDATES, reps=2)
    return s


def predictor_label(pred, basis, prec, affine):
    """The predictor kernel a stepper runs (dg_set_predictor_kernel)."""
    if pred == "lines" or basis == "gl" or (pred == "auto" and prec == "fp64"):
        return "lines"
    if pred == "auto" and prec == "fp32" and affine:
        return "interleaved columns"
    return "columns"


def time_steps(args, s, cfg, dgw, torch, barrier, local, steps=None, warmup=None):
    """W untimed steps, then K steps of each method (one stepper call per
    method, as a solve runs; with the Gauss basis a call changes basis once
    on entry and once on exit), timed with CUDA events on the launching
    stream, with the library's per-kernel event profile and the clocks
    sampled meanwhile."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    dt = cfg["dt"]
    U_l = s.to_device(cfg["U0"])
    U_a = s.to_device(cfg["U0"])
    stream = torch.cuda.current_stream()
    s.step_lsrk(U_l, dt, warmup)
    s.step_ader(U_a, dt, warmup, 2)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    s.profile(True)
    s.profile_read(reset=True)
    launches0 = s.launch_count()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step_lsrk(U_l, dt, steps)
    s.step_ader(U_a, dt, steps, 2)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = s.launch_count() - launches0
    prof = s.profile_read(reset=True)
    s.profile(False)
    clk = clocks.stop()
    dof = 4 * (cfg["k"] + 1) ** 3 * cfg["mesh"]["n_elem"]
    t_lsrk = prof["lsrk_stage"][0]
    t_ader = prof["ader_update"][0] + prof["tck"][0]
    per_method = {"lsrk": dof * steps / (t_lsrk * 1e-3) if t_lsrk else None,
                  "ader": dof * steps / (t_ader * 1e-3) if t_ader else None}
    return {"ms": ms, "prof": prof, "launches": launches, "clocks": clk, "per_method": per_method,
            "U_l": U_l, "U_a": U_a, "steps": steps, "warmup": warmup}


_PROBE = {}


def _probe_peak(dgw, prec):
    """FMA-pipe TFLOP/s of this GPU, measured once per precision."""
    if prec not in _PROBE:
        try:
            _PROBE[prec] = dgw.probe_fma_peak(prec, 4096 if prec == dgw.DG_FP64 else 65536)
        except Exception:
            _PROBE[prec] = None
    return _PROBE[prec]


def roofline(args, s, prof, N, k, prec, dgw, tiling, workload_name, basis):
    """Roofline of the dominant kernel: algorithmic flops (FP64 pipe, or FP32
    pipe when the arithmetic intensity puts it above the HBM roof) or bytes
    per launch over its average launch time from the event profile."""
    from paper_1805_03981_gb300 import opcount, traffic
    rsize = 8 if prec == dgw.DG_FP64 else 4
    dom = max(prof, key=lambda kk: prof[kk][0])
    tot_ms, nlaunch = prof[dom]
    avg_s = tot_ms * 1e-3 / max(nlaunch, 1)
    E = N ** 3
    nonwall = 1.0 if workload_name == "plane_wave" else 1.0 - 1.0 / N
    aff = s.is_affine()
    flops = opcount.flops_per_element(dom, k + 1, 2, nonwall, basis, aff) * E
    byts = opcount.bytes_per_element(dom, k + 1, rsize, 2, affine=aff and (basis == "g" or dom == "tck")) * E
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs")
    if prec == dgw.DG_FP64:
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": FP64_PEAK / 1e12,
                "unit": "TFLOP/s", "peak_source": "derived FP64 pipe: 152 SM x 2 FMA/clk x 2 x 2.07 GHz"}
    else:
        ai = flops / byts
        peak_hbm = (hbm or HBM_FALLBACK) * 1e9
        if ai * peak_hbm > FP32_PEAK:
            roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": FP32_PEAK / 1e12,
                    "unit": "TFLOP/s", "peak_source": "derived FP32 pipe: 152 SM x 128 FMA/clk x 2 x 2.07 GHz"}
        else:
            roof = {"bound": "hbm", "achieved": byts / avg_s / 1e9, "peak": hbm or HBM_FALLBACK,
                    "unit": "GB/s", "peak_source": "measured" if hbm else "fallback"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if roof["bound"] == "alu":
        # the same pipe measured on this GPU by an FMA probe (dg_probe_fma_peak),
        # beside the derived nominal peak
        probe = _probe_peak(dgw, prec)
        roof["probe_peak"] = probe
        roof["frac_of_probe"] = roof["achieved"] / probe if probe else None
    roof["kernel"] = dom
    # DRAM bytes per launch from the ncu table, when it was taken on these
    # sources and this launch configuration (else null)
    roof["traffic"] = traffic.lookup(workload_name, "fp64" if prec == dgw.DG_FP64 else "fp32", N, k, basis,
                                     tiling, dom)
    roof["traffic_source"] = ("profiles/dram_traffic.txt (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
                              if roof["traffic"] is not None else
                              "none recorded for these sources and this launch configuration")
    roof["per_launch_ms"] = avg_s * 1e3
    roof["algorithmic_flops_per_launch"] = flops
    roof["algorithmic_bytes_per_launch"] = byts
    return roof


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def precision_form(args, dgw, torch, barrier, local, N=64, k=4):
    """The precision form on its own workload: the plane wave on the 64^3
    periodic affine mesh at k = 4, FP32 operator and state with FP64
    geometry set-up; timed like the headline (W + K steps of each method),
    then the final states compared with the FP64 path after the same steps
    and with the exact solution at the nodes."""
    cfg = workload(N, k, "plane_wave")
    s = make_solver(args, cfg, dgw.DG_FP32, dgw, basis="g", pred="auto", tiling="")
    tiling = s.tiling()
    m = time_steps(args, s, cfg, dgw, torch, barrier, local)
    dof = 4 * (k + 1) ** 3 * N ** 3
    out = {"workload": workload_desc(N, k, "fp32", "plane_wave"), "dtype": "f32",
           "value": 2 * dof * m["steps"] / (m["ms"] * 1e-3), "unit": UNIT, "ms_per_step": m["ms"] / m["steps"],
           "per_method_dofs_per_s": m["per_method"],
           "kernel_ms": {kk: {"total_ms": v[0], "launches": v[1]} for kk, v in m["prof"].items() if v[1]},
           "roofline": roofline(args, s, m["prof"], N, k, dgw.DG_FP32, dgw, tiling, "plane_wave", "g"),
           "tiling_elements_per_block": {"operator": tiling[0], "tck": tiling[1]},
           "predictor_kernel": predictor_label("auto", "g", "fp32", s.is_affine()),
           "gpu_launches": m["launches"], "clocks": m["clocks"]}
    nst = m["steps"] + m["warmup"]
    u32 = {"lsrk": m["U_l"].double().cpu().numpy(), "ader": m["U_a"].double().cpu().numpy()}
    s.close()
    del m
    s64 = make_solver(args, cfg, dgw.DG_FP64, dgw, basis="g", pred="auto", tiling="5,5")
    exact = np.transpose(cfg["exact"](cfg["xnodes"], nst * cfg["dt"]), (0, 2, 1))
    acc = {"steps": nst}
    for method in ("lsrk", "ader"):
        U = s64.to_device(cfg["U0"])
        if method == "lsrk":
            s64.step_lsrk(U, cfg["dt"], nst)
        else:
            s64.step_ader(U, cfg["dt"], nst, 2)
        torch.cuda.synchronize()
        u64 = U.cpu().numpy()
        del U
        acc[method] = {"fp32_vs_fp64_rel_l2": _rel(u32[method], u64),
                       "fp32_vs_exact_nodal_rel_l2": _rel(u32[method], exact),
                       "fp64_vs_exact_nodal_rel_l2": _rel(u64, exact)}
    s64.close()
    out["accuracy_after_timed_steps"] = acc
    return out


def measure_forms(args, dgw, torch, barrier, local):
    """The precision, batched and served forms, each measured in this run
    beside the FP64 headline."""
    forms = {}
    t0 = time.perf_counter()
    forms["precision_fp32"] = precision_form(args, dgw, torch, barrier, local)
    forms["precision_fp32"]["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    forms["batched_fp32"] = batched_measure(args, dgw, torch, steps=args.batch_steps)
    forms["batched_fp32"]["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    forms["served_fp32"] = served_measure(args, dgw, torch)
    forms["served_fp32"]["wall_s"] = time.perf_counter() - t0
    return forms


# ------------------------------------------------------------------ precision study
def accuracy_study(args, cfg, dgw, torch):
    """FP32 vs FP64 on the GPU after ``args.accuracy`` steps of each method,
    and both against the exact solution at the nodes (plane wave)."""
    k, steps = cfg["k"], args.accuracy
    out = {"workload": workload_desc(args.size, k, "fp32/fp64", args.workload), "steps": steps,
           "dt": cfg["dt"]}
    exact = None
    if cfg.get("exact") is not None:
        exact = np.transpose(cfg["exact"](cfg["xnodes"], steps * cfg["dt"]), (0, 2, 1))
    for method in ("lsrk", "ader"):
        res = {}
        for prec in (dgw.DG_FP64, dgw.DG_FP32):
            s = dgw.Solver(cfg["mesh"], k, prec, cfg["alpha"], cfg["rho"], cfg["c"])
            U = s.to_device(cfg["U0"])
            t0 = time.perf_counter()
            if method == "lsrk":
                s.step_lsrk(U, cfg["dt"], steps)
            else:
                s.step_ader(U, cfg["dt"], steps, 2)
            torch.cuda.synchronize()
            res[prec] = (U.double().cpu().numpy(), time.perf_counter() - t0)
            s.close()
        u64, u32 = res[dgw.DG_FP64][0], res[dgw.DG_FP32][0]
        r = {"fp32_vs_fp64_rel_l2": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)),
             "seconds_fp64": res[dgw.DG_FP64][1], "seconds_fp32": res[dgw.DG_FP32][1]}
        if exact is not None:
            r["fp64_vs_exact_nodal_rel_l2"] = float(np.linalg.norm(u64 - exact) / np.linalg.norm(exact))
            r["fp32_vs_exact_nodal_rel_l2"] = float(np.linalg.norm(u32 - exact) / np.linalg.norm(exact))
        out[method] = r
    print(json.dumps({"accuracy": out}))
    return 0


# ------------------------------------------------------------------ batched form
def _gen_one(seed):
    import synth
    c = synth.configs.random_instance(seed, nsteps=500)
    c.pop("xnodes", None)
    c["mesh"].pop("deform", None)
    return c


def generate_instances(seeds, workers=None):
    """Seeded instances built in a process pool started with 'spawn' (safe
    after CUDA is initialised in this process)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_one, seeds, chunksize=4))


def _l2_pressure_error(U, xnodes, exact, t, k):
    """Relative continuous L2 error of the pressure against exact(x, t) on a
    mesh of equal affine elements (constant det J cancels in the ratio):
    GL nodal values and node positions are interpolated to (k+3)-point Gauss
    points per direction (tensor Lagrange interpolation)."""
    from numpy.polynomial import legendre as leg
    n, m = k + 1, k + 3
    xq, wq = leg.leggauss(m)
    xgl = np.concatenate(([-1.0], np.sort(np.real(leg.legroots(leg.legder([0] * (n - 1) + [1])))), [1.0])) \
        if n > 2 else np.array([-1.0, 1.0])
    L = np.ones((m, n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (xq - xgl[b]) / (xgl[a] - xgl[b])
    E = U.shape[0]
    p = U[:, 0].reshape(E, n, n, n)                       # [e][z][y][x]
    ph = np.einsum("qa,rb,sc,ecba->esrq", L, L, L, p).reshape(E, -1)
    X = xnodes.reshape(E, n, n, n, 3)
    Xq = np.einsum("qa,rb,sc,ecbai->esrqi", L, L, L, X).reshape(E, -1, 3)
    w = np.einsum("a,b,c->cba", wq, wq, wq).reshape(-1)
    pe = exact(Xq, t)[..., 0]
    return float(np.sqrt(np.sum(w * (ph - pe) ** 2) / np.sum(w * pe ** 2)))


def time_to_accuracy_bench(args, dgw, torch):
    """Accuracy against GPU time (Sec. 4.5, Fig. solv-acc-RK-vs-ADER, in 3D):
    the standing wave on periodic Cartesian meshes of growing size, degrees
    k = 1, 4, 7, LSRK(5,4), the paper's LSRK5(9), ADER and HDG-ADER (order
    k+1, reduction every 2nd derivative), at Cr = 0.1 and at 0.9 times each method's critical Courant
    number (measured on the GPU first), to t_end = 1; relative L2 pressure
    error at t_end against the device time of the solve."""
    import synth
    from paper_1805_03981_gb300 import crit_courant
    prec = dgw.DG_FP64 if args.prec == "fp64" else dgw.DG_FP32
    sizes = {1: (4, 8, 16, 32, 64), 2: (4, 8, 16, 32), 3: (4, 8, 16, 24, 32), 4: (2, 4, 8, 16, 24),
             5: (2, 4, 8, 16, 20), 6: (2, 4, 8, 12, 16), 7: (2, 4, 8, 12, 16)}
    t_end = args.t_end
    rows, crit = [], {}
    methods = ("lsrk", "lsrk59", "ader", "hdg_ader")
    for k in (int(x) for x in args.kset.split(",")):
        for method in methods:
            crit[(k, method)] = crit_courant.critical(k, method)
        for N in sizes[k]:
            cfg = synth.configs.standing_wave(N=N, k=k)
            s = dgw.Solver(cfg["mesh"], k, prec, cfg["alpha"], cfg["rho"], cfg["c"])
            s.set_basis(dgw.BASIS_G if args.basis == "g" else dgw.BASIS_GL)
            dof = 4 * (k + 1) ** 3 * N ** 3
            for method in methods:
                s.set_lsrk_scheme(dgw.LSRK59 if method == "lsrk59" else dgw.LSRK_CK54)
                for label, cr in (("0.1", 0.1), ("0.9crit", 0.9 * crit[(k, method)])):
                    dt_max = synth.configs.dt_from_courant(cr, cfg["mesh"]["h"], 1.0, k)
                    steps = int(np.ceil(t_end / dt_max))
                    dt = t_end / steps
                    U = s.to_device(cfg["U0"])
                    torch.cuda.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record()
                    if method in ("lsrk", "lsrk59"):
                        s.step_lsrk(U, dt, steps)
                    elif method == "hdg_ader":
                        s.step_hdg_ader(U, dt, steps, 2)
                    else:
                        s.step_ader(U, dt, steps, 2)
                    ev1.record()
                    torch.cuda.synchronize()
                    sec = ev0.elapsed_time(ev1) * 1e-3
                    err = _l2_pressure_error(U.double().cpu().numpy(), cfg["xnodes"], cfg["exact"], t_end, k)
                    rows.append({"k": k, "N": N, "dof": dof, "method": method, "cr": label,
                                 "cr_value": cr, "steps": steps, "gpu_seconds": sec, "l2_p": err,
                                 "dofs_per_s": dof * steps / sec})
            s.close()
    out = {"time_to_accuracy": {
        "workload": "standing wave p = cos 2pi x cos 2pi y cos 2pi z cos wt on periodic Cartesian N^3 meshes, "
                    "rho = c = 1, upwind, t_end = %g, %s, state basis %s" % (t_end, args.prec.upper(), args.basis),
        "crit_courant": {"%d/%s" % kk: v for kk, v in crit.items()}, "rows": rows}}
    print(json.dumps(out))
    return 0


def _l2_pressure_error_2d(U, xnodes, exact, t, k):
    """The 2D counterpart of _l2_pressure_error (equal affine elements)."""
    from numpy.polynomial import legendre as leg
    n, m = k + 1, k + 3
    xq, wq = leg.leggauss(m)
    xgl = np.concatenate(([-1.0], np.sort(np.real(leg.legroots(leg.legder([0] * (n - 1) + [1])))), [1.0])) \
        if n > 2 else np.array([-1.0, 1.0])
    L = np.ones((m, n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (xq - xgl[b]) / (xgl[a] - xgl[b])
    E = U.shape[0]
    ph = np.einsum("qa,rb,eba->erq", L, L, U[:, 0].reshape(E, n, n)).reshape(E, -1)
    Xq = np.einsum("qa,rb,ebai->erqi", L, L, xnodes.reshape(E, n, n, 2)).reshape(E, -1, 2)
    w = np.einsum("a,b->ba", wq, wq).reshape(-1)
    pe = exact(Xq, t)[..., 0]
    return float(np.sqrt(np.sum(w * (ph - pe) ** 2) / np.sum(w * pe ** 2)))


def time_to_accuracy_2d_bench(args, dgw, torch):
    """The paper's time-versus-accuracy study in its own 2D setting (Sec. 4.7,
    Fig. solv-acc-RK-vs-ADER): a seven-mode standing field on the periodic
    unit square (stand-in for the paper's membrane), rho = c = 1, k = 1, 4,
    7, LSRK(5,4) and ADER at Cr = 0.1 and at 0.9 of each method's critical
    Courant number (measured on the GPU in 2D first), to t_end; relative L2
    pressure error against the device time of the solve."""
    from synth import mesh2d
    from paper_1805_03981_gb300 import crit_courant
    prec = dgw.DG_FP64 if args.prec == "fp64" else dgw.DG_FP32
    sizes = {1: (8, 16, 32, 64, 128, 256, 512), 4: (4, 8, 16, 32, 64, 128), 7: (4, 8, 16, 32, 64)}
    t_end = args.t_end
    rows, crit = [], {}
    for k in (int(x) for x in args.kset.split(",")):
        for method in ("lsrk", "ader"):
            crit[(k, method)] = crit_courant.critical(k, method, dim=2)
        for N in sizes[k]:
            cfg = mesh2d.standing_wave_config_2d(N=N, k=k, exact=mesh2d.membrane_modes_2d)
            s = dgw.Solver2D(cfg["mesh"], k, prec, 1.0, cfg["rho"], cfg["c"])
            dof = 3 * (k + 1) ** 2 * N * N
            for method in ("lsrk", "ader"):
                for label, cr in (("0.1", 0.1), ("0.9crit", 0.9 * crit[(k, method)])):
                    steps = int(np.ceil(t_end / (cr * cfg["mesh"]["h"] / k ** 1.5)))
                    dt = t_end / steps
                    U = s.to_device(cfg["U0"])
                    torch.cuda.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record()
                    if method == "lsrk":
                        s.step_lsrk(U, dt, steps)
                    else:
                        s.step_ader(U, dt, steps, 2)
                    ev1.record()
                    torch.cuda.synchronize()
                    sec = ev0.elapsed_time(ev1) * 1e-3
                    err = _l2_pressure_error_2d(U.double().cpu().numpy(), cfg["xnodes"], cfg["exact"], t_end, k)
                    rows.append({"k": k, "N": N, "dof": dof, "method": method, "cr": label, "cr_value": cr,
                                 "steps": steps, "gpu_seconds": sec, "l2_p": err, "dofs_per_s": dof * steps / sec})
            s.close()
    print(json.dumps({"time_to_accuracy_2d": {
        "workload": "seven-mode standing field on the periodic unit square (N^2 quadrilaterals), rho = c = 1, "
                    "upwind, t_end = %g, %s" % (t_end, args.prec.upper()),
        "crit_courant_2d": {"%d/%s" % kk: v for kk, v in crit.items()}, "rows": rows}}))
    return 0


def reduction_bench(args, dgw, torch):
    """Degree reduction in the predictor every 0, 1, 2 or 3 derivatives
    (Sec. 3.3, Fig. reduc-comp) for k = 1..7 on the curved-pulse recipe at
    about 28M DoF per k: the op-count model of the predictor relative to no
    reduction, next to its measured device time per launch relative to no
    reduction (ADER steps in the chosen storage basis and precision)."""
    from paper_1805_03981_gb300 import opcount
    prec = dgw.DG_FP64 if args.prec == "fp64" else dgw.DG_FP32
    rows = []
    for k in range(1, 8):
        n = k + 1
        N = max(4, round((28.3e6 / (4 * n ** 3)) ** (1.0 / 3.0)))
        cfg = workload(N, k)
        s = dgw.Solver(cfg["mesh"], k, prec, cfg["alpha"], cfg["rho"], cfg["c"])
        s.set_basis(dgw.BASIS_G if args.basis == "g" else dgw.BASIS_GL)
        base = None
        for red in (0, 1, 2, 3):
            U = s.to_device(cfg["U0"])
            s.step_ader(U, cfg["dt"], args.warmup, red)
            torch.cuda.synchronize()
            s.profile(True)
            s.profile_read(reset=True)
            s.step_ader(U, cfg["dt"], args.steps, red)
            torch.cuda.synchronize()
            ms, nl = s.profile_read(reset=True)["tck"]
            s.profile(False)
            per = ms / max(nl, 1)
            flops = opcount.tck_flops(n, red, args.basis, s.is_affine()) * N ** 3
            if red == 0:
                base = (per, flops)
            rows.append({"k": k, "N": N, "reduce_every": red, "tck_ms_per_launch": per,
                         "time_rel_to_none": per / base[0], "model_flops_rel_to_none": flops / base[1],
                         "tflops": flops / (per * 1e-3) / 1e12})
        s.close()
    out = {"reduction": {"workload": "curved_pulse recipe at ~28M DoF per k, ADER predictor, reduce_every 0/1/2/3, "
                                     + args.prec.upper() + ", state basis " + args.basis,
                         "steps": args.steps, "rows": rows}}
    print(json.dumps(out))
    return 0


def basis_change_bench(args, dgw, torch):
    """What the basis change (Sec. 3.2) and the degree reduction (Sec. 3.3)
    save, measured: for k = 1..7 on the curved-pulse recipe at about 28M DoF
    per k, device time per ADER step (predictor + update) with
      alg1:   GL states, the predictor without the basis change (Alg. 1),
              no reduction;
      alg2:   GL states, the predictor with the on-the-fly basis change
              (Alg. 2), no reduction;
      alg2_3: Gauss-point states, Alg. 2 with reduction every 2nd
              derivative (the bench default);
    and per LSRK(5,4) step (Gauss-point states), next to the op-count models
    of the three predictors.  The measured counterpart of the paper's
    Fig. comp-opcounts-RK-ADER, which shows counts only."""
    from paper_1805_03981_gb300 import opcount
    prec = dgw.DG_FP64 if args.prec == "fp64" else dgw.DG_FP32
    rows = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn(args.warmup)
        torch.cuda.synchronize()
        ev0.record()
        fn(args.steps)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / args.steps

    for k in range(1, 8):
        n = k + 1
        N = max(4, round((28.3e6 / (4 * n ** 3)) ** (1.0 / 3.0)))
        cfg = workload(N, k)
        dof = 4 * n ** 3 * N ** 3
        s = dgw.Solver(cfg["mesh"], k, prec, cfg["alpha"], cfg["rho"], cfg["c"])
        aff = s.is_affine()
        row = {"k": k, "N": N, "dof": dof}
        U = s.to_device(cfg["U0"])
        for name, basis, pred, red in (("alg1", dgw.BASIS_GL, dgw.PRED_GL_PROJECTION, 0),
                                       ("alg2", dgw.BASIS_GL, dgw.PRED_AUTO, 0),
                                       ("alg2_3", dgw.BASIS_G, dgw.PRED_AUTO, 2)):
            s.set_basis(basis)
            s.set_predictor_kernel(pred)
            ms = timed(lambda m: s.step_ader(U, cfg["dt"], m, red))
            row[name + "_ms_per_step"] = ms
            row[name + "_ns_per_dof_step"] = ms * 1e6 / dof
        s.set_basis(dgw.BASIS_G)
        s.set_predictor_kernel(dgw.PRED_AUTO)
        ms = timed(lambda m: s.step_lsrk(U, cfg["dt"], m))
        row["lsrk_ms_per_step"] = ms
        row["lsrk_ns_per_dof_step"] = ms * 1e6 / dof
        row["model_tck_flops_per_elem"] = {"alg1": opcount.tck_flops_alg1(n, aff),
                                           "alg2": opcount.tck_flops(n, 0, "gl", aff),
                                           "alg2_3": opcount.tck_flops(n, 2, "g", aff)}
        rows.append(row)
        s.close()
    out = {"basis_change": {"workload": "curved_pulse recipe at ~28M DoF per k, " + args.prec.upper()
                                        + "; device time per ADER step with the three predictors and per LSRK(5,4) step",
                            "steps": args.steps, "rows": rows}}
    print(json.dumps(out))
    return 0


def batched_measure(args, dgw, torch, steps=None, fp64_every=8):
    """256 independent seeded solves (N ~ U{4..24} elements per axis, k ~
    U{2..7}, random smooth rho and c in [0.55, 1.95], curving <= 0.05, walls,
    Gaussian pulses), FP32 ADER (order k+1, reduction every 2nd derivative).
    Times the batched persistent form (8 warm-up steps, then ``steps``)
    against the same solves run one at a time in FP32, and in FP64 on every
    ``fp64_every``-th instance, which also gives each of those instances'
    relative l2 difference between the batched FP32 result and FP64 after
    the same steps."""
    from paper_1805_03981_gb300 import autotune
    table = autotune.load(args.autotune) if args.autotune else None
    n = args.instances
    steps = args.steps if steps is None else steps
    warm = 8
    t_gen = time.perf_counter()
    cfgs = generate_instances([4 * 10 ** 6 + i for i in range(n)])
    dof = [4 * (c["k"] + 1) ** 3 * c["mesh"]["n_elem"] for c in cfgs]
    total = sum(dof)
    t_gen = time.perf_counter() - t_gen
    out = {"workload": f"batched: {n} instances, N~U{{4..24}}^3 curved hexahedra, k~U{{2..7}}, seeded rho/c/pulses, "
                       f"ADER order k+1", "total_dof": total, "steps": steps, "warmup": warm,
           "state_basis": args.basis, "dtype": "f32",
           "k_histogram": {str(k): sum(1 for c in cfgs if c["k"] == k) for k in range(2, 8)}}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    t_setup = time.perf_counter()
    solvers = [dgw.Solver(c["mesh"], c["k"], dgw.DG_FP32, 1.0, c["rho"], c["c"]) for c in cfgs]
    for sv in solvers:
        sv.set_basis(dgw.BASIS_G if args.basis == "g" else dgw.BASIS_GL)
        if table:
            autotune.apply(sv, table)
    states = [sv.to_device(c["U0"]) for sv, c in zip(solvers, cfgs)]
    out["setup_s"] = time.perf_counter() - t_setup
    out["host_generation_s"] = t_gen
    b = dgw.Batch(solvers, states, [c["dt"] for c in cfgs])
    b.set_basis(dgw.BASIS_G if args.basis == "g" else dgw.BASIS_GL, convert_each_call=True)
    b.step_ader(warm, 2)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step_ader(steps, 2)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    out["value"] = total * steps / (ms * 1e-3)
    out["unit"] = UNIT
    out["batched_fp32"] = {"dofs_per_s": out["value"], "ms_per_step": ms / steps, "info": b.info()}
    sample = list(range(0, n, fp64_every))
    final32 = {i: states[i].double().cpu().numpy() for i in sample}
    # one solve at a time, FP32, same steps
    for sv, c, U in zip(solvers, cfgs, states):
        sv.step_ader(U, c["dt"], 2, 2)
    torch.cuda.synchronize()
    ev0.record(stream)
    for sv, c, U in zip(solvers, cfgs, states):
        sv.step_ader(U, c["dt"], steps, 2)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms1 = ev0.elapsed_time(ev1)
    out["one_at_a_time_fp32"] = {"dofs_per_s": total * steps / (ms1 * 1e-3), "ms_per_step": ms1 / steps}
    b.close()
    for sv in solvers:
        sv.close()
    del states
    # one solve at a time, FP64, on the sampled instances (contexts created
    # and freed one by one): warm + steps steps from the same initial state
    ms64, dof64, errs = 0.0, 0, []
    for i in sample:
        c = cfgs[i]
        sv = dgw.Solver(c["mesh"], c["k"], dgw.DG_FP64, 1.0, c["rho"], c["c"])
        sv.set_basis(dgw.BASIS_G if args.basis == "g" else dgw.BASIS_GL)
        U = sv.to_device(c["U0"])
        sv.step_ader(U, c["dt"], warm, 2)
        torch.cuda.synchronize()
        ev0.record(stream)
        sv.step_ader(U, c["dt"], steps, 2)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 += ev0.elapsed_time(ev1)
        dof64 += dof[i]
        errs.append(_rel(final32[i], U.cpu().numpy()))
        sv.close()
    out["one_at_a_time_fp64"] = {"dofs_per_s": dof64 * steps / (ms64 * 1e-3), "ms_per_step_sample": ms64 / steps,
                                 "instances_timed": len(sample)}
    out["fp32_vs_fp64_rel_l2"] = {"max": max(errs), "median": float(np.median(errs)), "instances": len(errs),
                                  "steps": warm + steps}
    out["speedup_batched_fp32_vs_fp64_one_at_a_time"] = (out["batched_fp32"]["dofs_per_s"]
                                                          / out["one_at_a_time_fp64"]["dofs_per_s"])
    out["speedup_batched_vs_one_at_a_time_fp32"] = (out["batched_fp32"]["dofs_per_s"]
                                                     / out["one_at_a_time_fp32"]["dofs_per_s"])
    return out


def batched_bench(args, dgw, torch):
    print(json.dumps({"batched": batched_measure(args, dgw, torch)}))
    return 0


# ------------------------------------------------------------------ served form
def _gen_request(spec):
    import synth
    seed, N, k, steps = spec
    c = synth.configs.random_instance(seed, N=N, k=k, nsteps=steps, curved=False)
    c.pop("xnodes", None)
    c["mesh"].pop("deform", None)
    c["U0"] = c["U0"].astype(np.float32)
    return c


def served_measure(args, dgw, torch):
    """Poisson stream of FP32 ADER solves (seed 5): cube meshes with N ~
    U{nmin..nmax} elements per axis, k ~ U{3,5,7}, seeded coefficient fields
    and pulses, U{smin..smax} steps at Cr = 0.1, against an HBM budget.
    Arrivals are replayed in real time; latency = completion - arrival.
    Beside it, the FP64 one-at-a-time form: one completed request per degree
    is solved again in FP64, which gives the FP64 service rates of the
    modelled FIFO queue and the relative l2 difference of the served FP32
    result from FP64 at the same steps."""
    import concurrent.futures as cf
    import multiprocessing as mp
    rng = np.random.default_rng(5)
    nmin, nmax = (int(x) for x in args.nrange.split(","))
    smin, smax = (int(x) for x in args.srange.split(","))
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / args.lam)
        if t >= args.duration:
            break
        arrivals.append(t)
    specs = [(5 * 10 ** 6 + i, int(rng.integers(nmin, nmax + 1)), int(rng.choice([3, 5, 7])),
              int(rng.integers(smin, smax + 1))) for i in range(len(arrivals))]
    t_gen = time.perf_counter()
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        reqs = list(ex.map(_gen_request, specs, chunksize=2))
    t_gen = time.perf_counter() - t_gen
    dofs = np.array([4 * (c["k"] + 1) ** 3 * c["mesh"]["n_elem"] for c in reqs], float)
    work = dofs * np.array([c["nsteps"] for c in reqs])
    srv = dgw.Server(int(args.budget_gb * (1 << 30)), prec=dgw.DG_FP32, chunk_steps=16,
                     max_active_dof=args.active_dof)
    # warm the library (tables, kernels) outside the measured stream
    w = _gen_request((1, 4, 3, 2))
    srv.poll(srv.submit(w["mesh"], 3, w["rho"], w["c"], w["U0"], w["dt"], 2), timeout_ms=60000)
    t0 = time.perf_counter()
    pending, done = {}, {}
    for i, (ta, c) in enumerate(zip(arrivals, reqs)):
        while True:
            now = time.perf_counter() - t0
            if now >= ta:
                break
            for tk in list(pending):
                r = srv.poll(tk)
                if r is not None:
                    done[pending.pop(tk)] = r
            time.sleep(min(0.002, max(0.0, ta - now)))
        pending[srv.submit(c["mesh"], c["k"], c["rho"], c["c"], c["U0"], c["dt"], c["nsteps"])] = i
    backlog_at_end = len(pending)
    cap = args.duration * 4 + 60
    while pending and time.perf_counter() - t0 < cap:
        for tk in list(pending):
            r = srv.poll(tk, timeout_ms=1)
            if r is not None:
                done[pending.pop(tk)] = r
    st = srv.stats()
    srv.close()
    lat = np.array([done[i]["t_done"] - done[i]["t_submit"] for i in sorted(done)])
    t_first = min(done[i]["t_submit"] for i in done)
    t_last = max(done[i]["t_done"] for i in done)
    completed_work = float(sum(work[i] for i in done))
    out = {"workload": f"served: Poisson lambda={args.lam}/s for {args.duration} s ({len(reqs)} requests), "
                       f"N~U{{{nmin}..{nmax}}}^3 affine hexahedra, k~U{{3,5,7}}, steps~U{{{smin}..{smax}}}, "
                       f"FP32 ADER, budget {args.budget_gb} GB, active-DoF cap {args.active_dof:g}",
           "requests": len(reqs), "completed": len(done), "censored": len(pending),
           "offered_dofs_per_s": float(work.sum() / args.duration),
           "throughput_dofs_per_s": completed_work / (t_last - t_first),
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "max": float(lat.max()), "p99_is_lower_bound": bool(pending)},
           "backlog_at_end_of_arrivals": backlog_at_end, "host_generation_s": t_gen,
           "server": {k: st[k] for k in ("peak_active", "rounds", "batches_built", "hbm_peak", "busy_s")}}
    # FP64 one-at-a-time, modelled: measured FP64 ADER rate per degree on one
    # completed request each (its whole solve), replayed through a
    # single-server FIFO over the same arrivals
    rate64, diff64, setup32 = {}, {}, {}
    for k in (3, 5, 7):
        cands = [j for j in sorted(done) if reqs[j]["k"] == k] or [j for j, c in enumerate(reqs) if c["k"] == k]
        if not cands:
            continue
        i = cands[0]
        c = reqs[i]
        # what an admission pays before its first step: the FP32 context's
        # set-up (validation, upload, FP64 geometry kernels)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        s32 = dgw.Solver(c["mesh"], k, dgw.DG_FP32, 1.0, c["rho"], c["c"])
        torch.cuda.synchronize()
        setup32[k] = {"seconds": time.perf_counter() - ta, "elements": int(c["mesh"]["n_elem"])}
        s32.close()
        s = dgw.Solver(c["mesh"], k, dgw.DG_FP64, 1.0, c["rho"], c["c"])
        s.set_basis(dgw.BASIS_G)
        U = s.to_device(c["U0"].astype(np.float64))
        torch.cuda.synchronize()
        ta = time.perf_counter()
        s.step_ader(U, c["dt"], c["nsteps"], 2)
        torch.cuda.synchronize()
        rate64[k] = dofs[i] * c["nsteps"] / (time.perf_counter() - ta)
        if i in done:
            diff64[k] = _rel(done[i]["out"].astype(np.float64), U.cpu().numpy())
        s.close()
    free_at, lat64 = 0.0, []
    for ta, c, wk in zip(arrivals, reqs, work):
        start = max(ta, free_at)
        free_at = start + wk / rate64[c["k"]]
        lat64.append(free_at - ta)
    lat64 = np.array(lat64)
    out["fp64_one_at_a_time_modelled"] = {
        "rate_dofs_per_s_by_k": rate64, "throughput_dofs_per_s": float(work.sum() / (free_at - arrivals[0])),
        "latency_s": {"p50": float(np.percentile(lat64, 50)), "p99": float(np.percentile(lat64, 99))},
        "note": "modelled: measured FP64 service rates replayed through a single-server FIFO queue"}
    out["fp32_vs_fp64_rel_l2_by_k"] = diff64
    out["context_setup_by_k"] = setup32
    out["value"] = out["throughput_dofs_per_s"]
    out["unit"] = UNIT
    out["dtype"] = "f32"
    return out


def served_bench(args, dgw, torch):
    print(json.dumps({"served": served_measure(args, dgw, torch)}))
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import torch.distributed as dist
    import paper_1805_03981_gb300 as dgw
    from paper_1805_03981_gb300 import opcount, traffic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(x, world, "cuda")

    prec = dgw.DG_FP64 if args.prec == "fp64" else dgw.DG_FP32
    if args.workload == "batched":
        return batched_bench(args, dgw, torch)
    if args.workload == "served":
        return served_bench(args, dgw, torch)
    if args.workload == "reduction":
        return reduction_bench(args, dgw, torch)
    if args.workload == "time_to_accuracy":
        return time_to_accuracy_bench(args, dgw, torch)
    if args.workload == "time_to_accuracy_2d":
        return time_to_accuracy_2d_bench(args, dgw, torch)
    if args.workload == "basis_change":
        return basis_change_bench(args, dgw, torch)
    N, k = args.size, args.k
    cfg = workload(N, k, args.workload)
    if args.accuracy:
        return accuracy_study(args, cfg, dgw, torch)
    s = make_solver(args, cfg, prec, dgw)
    tiling = s.tiling()
    dof = 4 * (k + 1) ** 3 * N ** 3
    dt = cfg["dt"]
    m = time_steps(args, s, cfg, dgw, torch, barrier, local)
    ms_max = max_over_ranks(m["ms"])
    value = job_value(2 * dof * args.steps, ms_max, world)
    prof, launches, clk, per_method = m["prof"], m["launches"], m["clocks"], m["per_method"]
    roof = roofline(args, s, prof, N, k, prec, dgw, tiling, args.workload, args.basis)

    # e2e through the C ABI with host buffers (pinned), copies inside the timing
    Uh = torch.from_numpy(np.ascontiguousarray(cfg["U0"])).to(s.dtype).pin_memory()
    out_l = torch.empty_like(Uh).pin_memory()
    out_a = torch.empty_like(Uh).pin_memory()
    in_l, in_a = Uh.clone().pin_memory(), Uh.clone().pin_memory()
    s.solve_host(0, in_l, out_l, dt, 1)
    s.solve_host(1, in_a, out_a, dt, 1, 2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):         # every step: state in from the host, one step, state out
        s.solve_host(0, in_l, out_l, dt, 1)
        s.solve_host(1, in_a, out_a, dt, 1, 2)
        in_l, out_l = out_l, in_l
        in_a, out_a = out_a, in_a
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    t0 = time.perf_counter()
    s.solve_host(0, in_l, out_l, dt, args.steps)
    s.solve_host(1, in_a, out_a, dt, args.steps, 2)
    barrier()
    solve_s = max_over_ranks(time.perf_counter() - t0)
    state_bytes = s.info()["state_bytes"]
    e2e = {"value": world * 2 * dof * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 2 * state_bytes, "d2h_bytes_per_step": 2 * state_bytes,
           "note": "each step, per method: dg_solve_host copies the state in from pinned host memory, "
                   "advances one step and copies it back",
           "k_steps_per_call_value": world * 2 * dof * args.steps / solve_s}
    device_mb = s.device_bytes() >> 20
    m_affine = s.is_affine()
    s.close()
    del m

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in ("curved_pulse", "plane_wave"):
        try:
            n_cpu = args.cpu_size or (4 if args.workload == "curved_pulse" else 16)
            st_cpu = args.cpu_steps or (20 if n_cpu <= 4 else 2)
            cpu = cpu_baseline(n_cpu, k, st_cpu, args.workload)
        except Exception as exc:  # the GPU number stands without it
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(exc)[:200]}

    forms = None
    if world == 1 and not args.no_forms and args.workload == "curved_pulse" and args.size == 32 and args.k == 5:
        forms = measure_forms(args, dgw, torch, barrier, local)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == dgw.DG_FP64 else "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(N, k, args.prec, args.workload), "elements": N ** 3, "k": k, "dof": dof,
                       "state_basis_inside_steppers": "Gauss points (G)" if args.basis == "g" else "Gauss-Lobatto (GL)",
                       "tiling_elements_per_block": {"operator": tiling[0], "tck": tiling[1]},
                       "predictor_kernel": predictor_label(args.pred, args.basis, args.prec, m_affine),
                       "affine_compact_kernels": m_affine,
                       "l2": "inputs larger than L2 (state %d MB, %d MB device-resident incl. geometry), no flush"
                       % (state_bytes >> 20, device_mb),
                       "parallelism": "replicas" if world > 1 else "single"},
            "per_method_dofs_per_s": per_method,
            "kernel_ms": {kk: {"total_ms": v[0], "launches": v[1]} for kk, v in prof.items() if v[1]},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
        }
        if forms is not None:
            line["forms"] = forms
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
