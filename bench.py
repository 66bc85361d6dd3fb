"""Benchmark of the fused D2Q9 relative-velocity step on GB300.

Headline workload: D2Q9 FP32, 4096 x 4096 periodic, Taylor-Green vortex u0 = 0.04,
rho0 = 1, s = (0,0,0,1.4,1.8,1.8,1.2,1.2,1.4) (s_nu = 1.8), prescribed relative velocity
u~(x,t) = 0.03 (cos 2 pi y/L, sin 2 pi x/L) cos(2 pi t / 1000). One bench step is one
time step (pull transport + relaxation in the moving frame), one kernel launch. The
0.6 GB state (1.2 GB moved per step) is larger than L2, so no flush is needed between
steps.

``python bench.py [--gpus N] [--steps K] [--warmup W]`` prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on the host cores instead (same metric).
With N > 1 (torchrun) every rank advances its own replica of the lattice (weak scaling;
the step has no exchange across replicas). ``--decomp slab`` instead splits one lattice of
N stacked Taylor-Green cells into slabs, one per rank, with a halo exchange per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and fraction of HBM roofline, relative-velocity step vs plain MRT"
L = 4096
S_RATES = [0, 0, 0, 1.4, 1.8, 1.8, 1.2, 1.2, 1.4]
UT_AMP, UT_PERIOD = 0.03, 1000.0
BYTES_PER_NODE = {"fp32": 72, "fp16": 36, "bf16": 36}
WORKLOAD = ("D2Q9 relative-velocity step, FP32, 4096x4096 periodic, Taylor-Green u0=0.04, "
            "s_nu=1.8, prescribed u~ = 0.03 (cos 2pi y/L, sin 2pi x/L) cos(2pi t/1000)")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "d2q9_step_tg4096_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1312_3297_gb300", "csrc", f)
                  for f in ("d2q9.cuh", "d2q9_kernels.cu", "pull.cuh", "f32x2.cuh")]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary, if the
    kernel sources are unchanged since it was taken; else None."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256_16") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the GPU is busy."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="lbmrv_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 5.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def mark(self) -> int:
        try:
            with open(self.path) as fh:
                return sum(1 for _ in fh)
        except OSError:
            return 0

    def stop(self):
        if self.proc is not None:
            time.sleep(0.06)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, first_line: int, last_line: int):
        rows = []
        try:
            with open(self.path) as fh:
                lines = fh.read().splitlines()
        except OSError:
            lines = []
        sel = lines[first_line:last_line + 1] or lines[-3:]
        for ln in sel:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        power = []
        for r in rows:
            try:
                power.append(float(r[3].split()[0]))
            except (ValueError, IndexError):
                pass
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "power_w": round(statistics.median(power), 1) if power else None,
                "samples": len(rows)}


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device) -> float:
    """The slowest rank's value: an all-reduce MAX over the default process group (the
    value itself when no group is initialised or it has one rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput of `world` replicas, each advancing `nodes_per_rank` nodes by
    `steps` steps, timed by the slowest rank (weak scaling)."""
    return world * nodes_per_rank * steps / (ms_max * 1e-3) / 1e6


def default_width(lattice: str, storage: str, nx: int) -> int:
    """Nodes per thread of the automatically chosen step kernel (the library's rule)."""
    widest = 4 if storage == "fp32" else 8
    while widest > 1 and nx % widest:
        widest //= 2
    return widest


def kernel_label(lattice: str, storage: str, nx: int, mode: str, scheme: str = "rv",
                 width: int = 0) -> str:
    """Name of the step kernel the library launches for this configuration."""
    nv = width or default_width(lattice, storage, nx)
    if lattice == "d2q9":
        name = "k_step_vec" if scheme == "rv" else "k_step_vec, Geier basis"
    elif storage == "fp32":
        name = "k_step3"
    else:
        name = {8: "k_step3_pipe", 4: "k_step3_pipe_pairs"}.get(nv, "k_step3")
    return f"{name}<{storage},{nv},{mode}>"


# ------------------------------------------------------------------ GPU arm
def time_steps(sim, steps: int, torch):
    """Device time (ms) of `steps` fused steps on the handle's stream, CUDA events."""
    st = sim.stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    sim.step(steps)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b)


def stored_base_field(torch, size):
    """The prescribed field's base (cos 2 pi y/L, sin 2 pi x/L), held as a device array."""
    k = 2 * 3.141592653589793 / size
    i = torch.arange(size, dtype=torch.float64, device="cuda")
    ux = torch.cos(k * i)[:, None].expand(size, size)
    uy = torch.sin(k * i)[None, :].expand(size, size)
    return torch.stack([ux, uy]).to(torch.float32).contiguous()


def make_sim(torch, D2Q9, inp, storage, mode, size, fields, u_ref=None, stored_field=False):
    sim = D2Q9(size, size, S_RATES, mode=mode, storage=storage, u_ref=u_ref)
    if mode == "prescribed":
        sim.set_utilde(stored_base_field(torch, size) if stored_field else None, UT_AMP,
                       UT_PERIOD)
    rho, ux, uy = (torch.as_tensor(fields[k], dtype=torch.float32) for k in ("rho", "ux", "uy"))
    sim.init_equilibrium(rho, ux, uy)
    return sim


def side_measure(torch, D2Q9, inp, storage, mode, size, fields, steps, peak, u_ref=None,
                 stored_field=False):
    sim = make_sim(torch, D2Q9, inp, storage, mode, size, fields, u_ref=u_ref,
                   stored_field=stored_field)
    sim.step(3)
    ms = time_steps(sim, steps, torch)
    sim.close()
    n = size * size
    per = ms / steps
    bpn = BYTES_PER_NODE[storage] + (8 if stored_field else 0)  # + the field's two floats
    gbs = bpn * n / (per * 1e-3) / 1e9
    return {"mlups": round(n / (per * 1e-3) / 1e6, 1), "ms_per_step": round(per, 5),
            "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}


class SlabRun:
    """The slab driver behind the interface the timed loop uses (step, stream, conserved,
    close)."""

    def __init__(self, slab):
        self.slab = slab
        self.stream = slab.sim.stream

    def step(self, n=1):
        self.slab.step(n)

    def conserved(self, allow_nonfinite=False):
        c = self.slab.conserved3()
        return [c[0], c[1], c[2], c[4]]

    def close(self):
        self.slab.close()


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import lbm_inputs as inp
    from paper_1312_3297_gb300 import D2Q9, binding

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load()
    peak, peak_kind = measured_peaks()
    size = args.size
    if args.lattice == "d3q19":
        from paper_1312_3297_gb300 import D3Q19

        n = size ** 3
        d3 = inp.taylor_green_3d(size, size, size, u0=0.04)
        sim = D3Q19(size, size, size, [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3,
                    mode="fluid" if args.mode == "prescribed" else args.mode, storage=args.storage)
        if args.width:
            sim.set_kernel_width(args.width)
        sim.init_equilibrium(torch.as_tensor(d3["rho"], dtype=torch.float32),
                             *(torch.as_tensor(c, dtype=torch.float32) for c in d3["u"]))
        del d3
    elif args.decomp == "slab":
        # weak scaling on one lattice of size x (size * world) rows, one slab per rank: N
        # Taylor-Green cells stacked in y, each rank owning one cell's rows; every step
        # exchanges the slab faces with the neighbouring ranks
        from paper_1312_3297_gb300.slab import Slab

        n = size * size
        fields = inp.taylor_green(size, size, u0=0.04)
        slab = Slab(D2Q9, (size, size * world), S_RATES, rank=rank, world=world,
                    mode=args.mode, storage=args.storage)
        if args.mode == "prescribed":
            slab.sim.set_utilde(None, UT_AMP, UT_PERIOD)
        slab.init_equilibrium(*(torch.as_tensor(fields[k], dtype=torch.float32)
                                for k in ("rho", "ux", "uy")))
        sim = SlabRun(slab)
    else:
        n = size * size
        fields = inp.taylor_green(size, size, u0=0.04)
        if args.scheme == "cascaded":
            from paper_1312_3297_gb300 import D2Q9Cascaded as scheme
        else:
            scheme = D2Q9
        sim = make_sim(torch, scheme, inp, args.storage, args.mode, size, fields)
        if args.width:
            sim.set_kernel_width(args.width)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
        first = clocks.mark()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms = time_steps(sim, args.steps, torch)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall_ms = (time.perf_counter() - t_wall) * 1e3
    if clocks:
        last = clocks.mark()
        clocks.stop()
        clock_info = clocks.summary(first, last)
    ms = max_over_ranks(ms, torch.device("cuda", local))
    # The K timed steps can be a few milliseconds; repeats of at least 100 ms each, taken
    # after the timed region, show how stable the per-step time is.
    repeats = None
    if rank == 0 and not args.no_extras:
        k_rep = max(args.steps, int(100.0 / max(ms / args.steps, 1e-3)) + 1)
        runs = [time_steps(sim, k_rep, torch) / k_rep for _ in range(5)]
        repeats = {"steps_per_run": k_rep, "ms_per_step_runs": [round(r, 5) for r in runs],
                   "ms_per_step_median": round(statistics.median(runs), 5)}
    finite = sim.conserved(allow_nonfinite=True)
    sim.close()
    per_step_ms = ms / args.steps
    mlups = job_mlups(n, world, args.steps, ms)
    e2e = None
    if not args.no_e2e and size == L and args.storage == "fp32" and args.mode == "prescribed" \
            and args.lattice == "d2q9" and args.decomp == "replicas" and args.scheme == "rv":
        # every rank runs its replica end to end; the job's figure takes the slowest rank
        if world > 1:
            dist.barrier()
        e2e = e2e_measure(torch, D2Q9, inp, fields, args.steps)
        worst = max_over_ranks(e2e.pop("seconds"), torch.device("cuda", local))
        e2e["value"] = round(job_mlups(n, world, args.steps, worst * 1e3), 1)
        e2e["runs_rank0"] = e2e.pop("runs")
    bpn = BYTES_PER_NODE[args.storage] * (19 / 9 if args.lattice == "d3q19" else 1)
    achieved = bpn * n / (per_step_ms * 1e-3) / 1e9
    headline = (size == L and args.storage == "fp32" and args.mode == "prescribed"
                and args.lattice == "d2q9" and args.decomp == "replicas"
                and args.scheme == "rv" and not args.width)
    out = None
    if rank == 0:
        extras = {}
        if not args.no_extras and world == 1 and headline:
            k = max(50, min(args.steps, 300))
            extras["plain_mrt_u0"] = side_measure(torch, D2Q9, inp, "fp32", "zero", L, fields,
                                                  k, peak)
            extras["relative_u_fluid"] = side_measure(torch, D2Q9, inp, "fp32", "fluid", L,
                                                      fields, k, peak)
            extras["relative_u_prescribed"] = {
                "mlups": round(n / (per_step_ms * 1e-3) / 1e6, 1),
                "ms_per_step": round(per_step_ms, 5), "gbs": round(achieved, 1),
                "frac": round(achieved / peak, 4)}
            # the same u~(x, t) read from a stored base field: 80 B/node
            extras["relative_u_prescribed_stored_field"] = side_measure(
                torch, D2Q9, inp, "fp32", "prescribed", L, fields, k, peak, stored_field=True)
            # perturbed uniform flow U = (0.05, 0.02); 16-bit storage relative to the
            # library's automatic reference (the mean flow of the initial fields), the
            # default form, which meets the 2e-3 velocity bar on this workload
            big = inp.perturbed_uniform(8192, 8192, seed=0)
            for st in ("fp16", "bf16"):
                extras[f"precision_{st}_8192"] = side_measure(torch, D2Q9, inp, st, "fluid",
                                                              8192, big, k, peak)
            extras["fp32_fluid_8192"] = side_measure(torch, D2Q9, inp, "fp32", "fluid", 8192,
                                                     big, k, peak)
            extras["cascaded_geier_16bit_8192"] = cascaded16_measure(torch, big, k, peak)
            del big
            extras["cascaded_geier_fluid"] = cascaded_measure(torch, inp, fields, k, peak)
            extras["conserved_sums_4096"] = sums_measure(torch, D2Q9, inp, fields)
            extras["slab_one_rank_4096"] = slab_measure(torch, D2Q9, inp, fields, k, peak,
                                                        per_step_ms)
            extras["adjoint_1024"] = adjoint_measure(torch, D2Q9, inp, peak)
            extras["adjoint_4096"] = adjoint_step_measure(torch, D2Q9, inp, peak, 4096, 60)
            extras["adjoint_16bit_1024"] = {
                st: adjoint_step_measure(torch, D2Q9, inp, peak, 1024, 1000, st)
                for st in ("fp16", "bf16")}
            extras["adjoint_16bit_4096"] = adjoint_step_measure(torch, D2Q9, inp, peak, 4096,
                                                                60, "fp16")
            extras["d3q19_256"] = d3q19_measure(torch, inp, k, peak)
        cpu = cpu_baseline_measure() if (world == 1 and not args.no_cpu) else None
        out = {
            "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_step_ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "fp32" else f"{args.storage} storage, f32 math",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if headline else
                       f"{args.lattice}{' cascaded' if args.scheme == 'cascaded' else ''} "
                       f"{args.storage} side {size} Taylor-Green, u~ mode {args.mode}",
                       "nodes": n, "bytes_per_node_step": round(bpn, 1),
                       "l2": f"state {bpn / 2 * n / 1e9:.2f} GB > 129 MB L2; no flush needed",
                       "parallelism": f"{args.decomp} x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": recorded_traffic() if headline else None,
                         "peak_kind": peak_kind,
                         "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                         "kernel": kernel_label(args.lattice, args.storage, size, args.mode,
                                                args.scheme, args.width)},
            "clocks": clock_info,
            "e2e": e2e,
            # one step kernel per step and rank; a slab adds its pack and unpack kernels
            "gpu_launches": args.steps * world * (3 if args.decomp == "slab" else 1),
            "cpu_baseline": cpu,
            "modes": extras,
            "wall_ms_timed_region": round(wall_ms, 2),
            "repeats": repeats,
            "ms_per_step_x_sm_mhz": (round(per_step_ms * clock_info["sm_mhz"], 2)
                                     if clocks and clock_info.get("sm_mhz") else None),
            "nonfinite_nodes": finite[3],
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def slab_measure(torch, D2Q9, inp, fields, steps, peak, ref_ms):
    """The headline workload through the slab driver with one slab (its own neighbour): each
    step packs the two faces' crossing populations into the halo buffers, unpacks them into
    the halo rows and runs the fused step on 4096 + 2 rows; the cost of the decomposition's
    machinery against the plain step (ref_ms per step)."""
    from paper_1312_3297_gb300.slab import Slab

    sl = Slab(D2Q9, (L, L), S_RATES, mode="prescribed")
    sl.sim.set_utilde(None, UT_AMP, UT_PERIOD)
    sl.init_equilibrium(*(torch.as_tensor(fields[k], dtype=torch.float32)
                          for k in ("rho", "ux", "uy")))
    sl.step(3)
    st = sl.sim.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    sl.step(steps)
    b.record(st)
    b.synchronize()
    per = a.elapsed_time(b) / steps
    sl.close()
    n = L * L
    return {"ms_per_step": round(per, 5), "mlups": round(n / (per * 1e-3) / 1e6, 1),
            "frac": round(72 * n / (per * 1e-3) / 1e9 / peak, 4),
            "over_plain_step": round(per / ref_ms, 4),
            "kernels_per_step": "1 pack (both faces, straight into the other face's halo "
                                "buffer) + 1 unpack + 1 step"}


def sums_measure(torch, D2Q9, inp, fields, reps: int = 30):
    """One step followed by the FP64 conserved sums of its result, synchronously: with the
    sums fused into the step kernel (lbmrv_step_conserved) and with the separate reduction
    pass over the stored state (lbmrv_step + lbmrv_conserved3). Wall clock per check, host
    calls and the read-back included (the kernels' own times: `--case sums` under ncu)."""
    sim = make_sim(torch, D2Q9, inp, "fp32", "prescribed", L, fields)
    sim.step(3)
    out = {}
    for name, check in (("fused", lambda: sim.step_conserved(1)),
                        ("separate", lambda: (sim.step(1), sim.conserved3()))):
        check()
        torch.cuda.synchronize()
        runs = []
        for _ in range(reps):
            t0 = time.perf_counter()
            check()
            runs.append((time.perf_counter() - t0) * 1e3)
        out[f"{name}_ms"] = round(statistics.median(runs), 4)
    sim.close()
    out["saved_ms"] = round(out["separate_ms"] - out["fused_ms"], 4)
    return out


def sums_arm(args):
    """The conserved-sum checks alone (profiling captures): on D2Q9 4096^2 (FP32, FP16;
    prescribed u~) and D3Q19 256^3 (FP32, FP16; u~ = q/rho), three plain steps, then
    `args.steps` rounds of a fused check (lbmrv_step_conserved) and a separate one
    (lbmrv_step + lbmrv_conserved3). Prints the median wall clock per check as one JSON
    line; ncu's launch list of this command gives the kernels' times."""
    import torch

    import lbm_inputs as inp
    from paper_1312_3297_gb300 import D2Q9, D3Q19, binding

    binding.load()
    out = {}
    fields = inp.taylor_green(L, L, u0=0.04)
    d3 = inp.taylor_green_3d(256, 256, 256, u0=0.04)
    s3 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3
    for lattice in ("d2q9", "d3q19"):
        for st in ("fp32", "fp16"):
            if lattice == "d2q9":
                sim = make_sim(torch, D2Q9, inp, st, "prescribed", L, fields)
            else:
                sim = D3Q19(256, 256, 256, s3, mode="fluid", storage=st)
                sim.init_equilibrium(torch.as_tensor(d3["rho"], dtype=torch.float32),
                                     *(torch.as_tensor(c, dtype=torch.float32)
                                       for c in d3["u"]))
            sim.step(3)
            fused, separate = [], []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                sim.step_conserved(1)
                fused.append((time.perf_counter() - t0) * 1e3)
                t0 = time.perf_counter()
                sim.step(1)
                sim.conserved3()
                separate.append((time.perf_counter() - t0) * 1e3)
            sim.close()
            out[f"{lattice}_{st}"] = {"fused_ms": round(statistics.median(fused), 4),
                                      "separate_ms": round(statistics.median(separate), 4)}
    print(json.dumps({"case": "sums", "checks": args.steps, **out}), flush=True)


def cascaded_measure(torch, inp, fields, steps, peak):
    """Geier's cascaded scheme (D2Q9, Geier basis, product equilibrium, u~ = q/rho) on the
    same 4096^2 Taylor-Green workload, FP32."""
    from paper_1312_3297_gb300 import D2Q9Cascaded

    sim = D2Q9Cascaded(L, L, [0, 0, 0, 1.3, 1.8, 1.8, 1.5, 1.5, 1.2], mode="fluid")
    sim.init_equilibrium(*(torch.as_tensor(fields[k], dtype=torch.float32)
                           for k in ("rho", "ux", "uy")))
    sim.step(3)
    per = time_steps(sim, steps, torch) / steps
    sim.close()
    n = L * L
    gbs = 72 * n / (per * 1e-3) / 1e9
    return {"mlups": round(n / (per * 1e-3) / 1e6, 1), "ms_per_step": round(per, 5),
            "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}


def cascaded16_measure(torch, big, steps, peak):
    """Geier's cascaded scheme in FP16 and BF16 storage on the 8192^2 perturbed uniform flow
    (automatic reference), 36 B per node and step."""
    from paper_1312_3297_gb300 import D2Q9Cascaded

    out = {}
    n = 8192 * 8192
    for st in ("fp16", "bf16"):
        sim = D2Q9Cascaded(8192, 8192, S_RATES, mode="fluid", storage=st)
        sim.init_equilibrium(*(torch.as_tensor(big[k], dtype=torch.float32)
                               for k in ("rho", "ux", "uy")))
        sim.step(3)
        per = time_steps(sim, steps, torch) / steps
        sim.close()
        gbs = 36 * n / (per * 1e-3) / 1e9
        out[st] = {"mlups": round(n / (per * 1e-3) / 1e6, 1), "ms_per_step": round(per, 5),
                   "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    return out


def d3q19_measure(torch, inp, steps, peak):
    """D3Q19 FP32, 256^3 3D Taylor-Green vortex u0 = 0.04, s_nu = 1.7, u~ = q/rho: 152 B per
    node and step (19 populations read + written)."""
    from paper_1312_3297_gb300 import D3Q19

    L3 = 256
    n = L3 ** 3
    d = inp.taylor_green_3d(L3, L3, L3, u0=0.04)
    s3 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3
    out = {}
    for storage, bpn in (("fp32", 152), ("fp16", 76), ("bf16", 76)):
        sim = D3Q19(L3, L3, L3, s3, mode="fluid", storage=storage)
        sim.init_equilibrium(torch.as_tensor(d["rho"], dtype=torch.float32),
                             *(torch.as_tensor(c, dtype=torch.float32) for c in d["u"]))
        sim.step(3)
        per = time_steps(sim, steps, torch) / steps
        sim.close()
        gbs = bpn * n / (per * 1e-3) / 1e9
        out[storage] = {"mlups": round(n / (per * 1e-3) / 1e6, 1), "ms_per_step": round(per, 5),
                        "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    return out


def adjoint_measure(torch, D2Q9, inp, peak, n_steps: int = 2000):
    """Adjoint workload: 1024^2 noisy shear wave, prescribed u~, kinetic-energy loss,
    2000 steps with sqrt(N) = 45 checkpoints. Reports the forward step, the adjoint step
    alone (checkpoint every state on a 1000-step window: no recompute), and the whole
    gradient (checkpointed forward + recompute + reverse sweep + equilibrium adjoint)."""
    size = 1024
    n = size * size
    d = inp.noisy_shear_wave(size, size, seed=0)
    sim = D2Q9(size, size, S_RATES, mode="prescribed")
    sim.set_utilde(None, UT_AMP, UT_PERIOD)
    rho = torch.as_tensor(d["rho"], dtype=torch.float32, device="cuda")
    u = torch.stack([torch.as_tensor(d[k], dtype=torch.float32, device="cuda")
                     for k in ("ux", "uy")])
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    st = sim.stream
    # forward step alone
    sim.init_equilibrium(rho, u[0], u[1])
    sim.step(5)
    fwd_ms = time_steps(sim, 1000, torch) / 1000
    # adjoint step alone: every state checkpointed, so the sweep has no recompute
    w = 1000  # every state checkpointed: 1000 x 37.7 MB; per-call fixed work amortised
    ws = sim.adjoint_workspace(w, 1)
    sim.init_equilibrium(rho, u[0], u[1])
    sim.forward_checkpointed(w, 1, ws)
    _, dlds = sim.kinetic_energy(grad=True)
    sim.adjoint(w, 1, ws, dlds)  # warm
    a, b = ev(), ev()
    a.record(st)
    sim.adjoint(w, 1, ws, dlds)
    b.record(st)
    b.synchronize()
    adj_ms = a.elapsed_time(b) / w
    del ws
    # whole gradient, sqrt(N) checkpoints
    seg = 45
    ws = sim.adjoint_workspace(n_steps, seg)
    torch.cuda.synchronize()
    e0, e1, e2, e3 = ev(), ev(), ev(), ev()
    e0.record(st)
    sim.init_equilibrium(rho, u[0], u[1])
    sim.forward_checkpointed(n_steps, seg, ws)
    e1.record(st)
    ke, dlds = sim.kinetic_energy(grad=True)
    e2.record(st)
    d0, ds, da, _ = sim.adjoint(n_steps, seg, ws, dlds)
    sim.equilibrium_vjp(rho, u, d0)
    e3.record(st)
    e3.synchronize()
    ws_gb = ws.numel() / 1e9
    del ws
    # the same gradient with every state stored (no recomputation), when HBM holds them all
    all_states = None
    from paper_1312_3297_gb300 import binding

    need = binding.lbmrv_adjoint_workspace_bytes(sim.h, n_steps, 1)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if 0 < need < 0.8 * free:
        ws = sim.adjoint_workspace(n_steps, 1)
        torch.cuda.synchronize()
        f0, f1 = ev(), ev()
        f0.record(st)
        sim.init_equilibrium(rho, u[0], u[1])
        sim.forward_checkpointed(n_steps, 1, ws)
        _, dlds1 = sim.kinetic_energy(grad=True)
        d1, ds1, da1, _ = sim.adjoint(n_steps, 1, ws, dlds1)
        sim.equilibrium_vjp(rho, u, d1)
        f1.record(st)
        f1.synchronize()
        all_states = {"workspace_gb": round(ws.numel() / 1e9, 2),
                      "gradient_ms": round(f0.elapsed_time(f1), 2),
                      "gradient_over_forward_run": round(f0.elapsed_time(f1) /
                                                         (fwd_ms * n_steps), 3),
                      "dL_dsnu_same_as_sqrtN": bool(ds1[4] + ds1[5] == ds[4] + ds[5])}
        del ws
    sim.close()
    return {"workload": f"1024^2 noisy shear wave, prescribed u~, KE loss, {n_steps} steps, seg 45",
            "forward_ms_per_step": round(fwd_ms, 5),
            "adjoint_ms_per_step": round(adj_ms, 5),
            "adjoint_over_forward": round(adj_ms / fwd_ms, 3),
            "adjoint_gbs": round(108 * n / (adj_ms * 1e-3) / 1e9, 1),
            "adjoint_frac": round(108 * n / (adj_ms * 1e-3) / 1e9 / peak, 4),
            "checkpointed_forward_ms": round(e0.elapsed_time(e1), 2),
            "reverse_sweep_ms": round(e2.elapsed_time(e3), 2),
            "gradient_over_forward_run": round(e0.elapsed_time(e3) / (fwd_ms * n_steps), 3),
            "workspace_gb": round(ws_gb, 2), "loss": ke, "dL_dsnu": ds[4] + ds[5],
            "dL_dA": da, "every_state_stored": all_states}


def adjoint_step_measure(torch, D2Q9, inp, peak, size: int, window: int, storage="fp32"):
    """The adjoint step alone at size^2 (every state of a `window`-step run checkpointed, so
    the sweep has no recompute), beside the forward step on the same lattice and storage:
    ms per step, algorithmic GB/s (S_{k-1} read in the storage type, mu_{k+1} read and mu_k
    written in FP32: 108 B/node, 90 B/node with 16-bit states) and its fraction of the
    measured copy bandwidth."""
    n = size * size
    d = inp.noisy_shear_wave(size, size, seed=0)
    sim = D2Q9(size, size, S_RATES, mode="prescribed", storage=storage)
    sim.set_utilde(None, UT_AMP, UT_PERIOD)
    rho = torch.as_tensor(d["rho"], dtype=torch.float32, device="cuda")
    u = torch.stack([torch.as_tensor(d[k], dtype=torch.float32, device="cuda")
                     for k in ("ux", "uy")])
    st = sim.stream
    sim.init_equilibrium(rho, u[0], u[1])
    sim.step(5)
    fwd_ms = time_steps(sim, window, torch) / window
    ws = sim.adjoint_workspace(window, 1)
    sim.init_equilibrium(rho, u[0], u[1])
    sim.forward_checkpointed(window, 1, ws)
    _, dlds = sim.kinetic_energy(grad=True)
    sim.adjoint(window, 1, ws, dlds)  # warm
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    sim.adjoint(window, 1, ws, dlds)
    b.record(st)
    b.synchronize()
    adj_ms = a.elapsed_time(b) / window
    del ws
    sim.close()
    torch.cuda.empty_cache()
    gbs = (BYTES_PER_NODE[storage] // 2 + 72) * n / (adj_ms * 1e-3) / 1e9
    return {"storage": storage,
            "forward_ms_per_step": round(fwd_ms, 5), "adjoint_ms_per_step": round(adj_ms, 5),
            "adjoint_over_forward": round(adj_ms / fwd_ms, 3), "adjoint_gbs": round(gbs, 1),
            "adjoint_frac": round(gbs / peak, 4)}


def adjoint_arm(args):
    """The adjoint workload alone (one GPU): its JSON dict on one line."""
    import torch

    import lbm_inputs as inp
    from paper_1312_3297_gb300 import D2Q9, binding

    binding.load()
    peak, _ = measured_peaks()
    print(json.dumps(adjoint_measure(torch, D2Q9, inp, peak, n_steps=args.adjoint_steps)),
          flush=True)


def e2e_measure(torch, D2Q9, inp, fields, steps):
    """Through the public API with host buffers: pinned host fields -> device,
    equilibrium, `steps` steps, moments back to pinned host memory."""
    n = L * L
    rho_h = torch.as_tensor(fields["rho"], dtype=torch.float32).reshape(-1).pin_memory()
    u_h = torch.stack([torch.as_tensor(fields["ux"], dtype=torch.float32),
                       torch.as_tensor(fields["uy"], dtype=torch.float32)]).reshape(2, -1)
    u_h = u_h.pin_memory()
    rho_o = torch.empty((L, L), dtype=torch.float32, pin_memory=True)
    u_o = torch.empty((2, L, L), dtype=torch.float32, pin_memory=True)
    sim = D2Q9(L, L, S_RATES, mode="prescribed", storage="fp32")
    sim.set_utilde(None, UT_AMP, UT_PERIOD)
    sim.init_equilibrium_host(rho_h, u_h)
    sim.step(3)
    sim.moments_host(rho_o, u_o)
    torch.cuda.synchronize()
    runs = []
    for _ in range(3):
        t0 = time.perf_counter()
        sim.init_equilibrium_host(rho_h, u_h)
        sim.step(steps)
        sim.moments_host(rho_o, u_o)  # synchronous
        runs.append(n * steps / (time.perf_counter() - t0) / 1e6)
    sim.close()
    med = statistics.median(runs)
    return {"value": round(med, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": round(12 * n / steps, 1),
            "d2h_bytes_per_step": round(12 * n / steps, 1),
            "unit_of_work": f"one {steps}-step run from host rho,u to host rho,u "
                            "(median of 3 runs)",
            "runs": [round(r, 1) for r in runs],
            "seconds": n * steps / (med * 1e6)}


# ------------------------------------------------------------------ CPU oracle
class OracleBand:
    """The FP64 definition oracle (per-node M(u~) and LU solve) advancing a 4096-wide
    periodic band of `rows` rows of the Taylor-Green workload (prescribed u~ evaluated
    at the band's global coordinates), with `threads` OpenMP threads."""

    def __init__(self, rows: int, threads: int, method=None, mode=None):
        import numpy as np

        import oracle

        self.oracle, self.np = oracle, np
        self.rows, self.threads, self.t = rows, threads, 1
        x = np.arange(L, dtype=np.float64)[None, :]
        y = np.arange(rows, dtype=np.float64)[:, None]
        k = 2 * np.pi / L
        ux = -0.04 * np.cos(k * x) * np.sin(k * y)
        uy = 0.04 * np.sin(k * x) * np.cos(k * y)
        rho = 1.0 + 3.0 * (-0.04 ** 2 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)))
        self.f = oracle.init_equilibrium(rho, ux, uy, 1.0)
        self.work = np.empty_like(self.f)
        self.ut0 = np.stack([np.cos(k * y) * np.ones((1, L)), np.sin(k * x) * np.ones((rows, 1))])
        self.s = np.array(S_RATES, float)
        self.method = oracle.METHOD_DEFINITION if method is None else method
        self.mode = oracle.MODE_PRESCRIBED if mode is None else mode

    def step(self) -> float:
        t0 = time.perf_counter()
        self.oracle.run_inplace(self.f, self.work, 1.0, self.s, self.mode, 1,
                                t0=self.t, method=self.method, ut0=self.ut0,
                                amp=UT_AMP, period=UT_PERIOD, nthreads=self.threads)
        self.t += 1
        return time.perf_counter() - t0


def _oracle_threads():
    import oracle

    oracle.build()
    return (os.cpu_count() or 1) if oracle.openmp_enabled() else 1


def _calibrated_rows(threads: int, seconds_per_step: float, **kw) -> int:
    probe = OracleBand(16, threads, **kw)
    probe.step()
    rate = 16 * L / probe.step()  # nodes per second
    return int(max(1, min(L, seconds_per_step * rate / L)))


def _band_mlups(threads: int, seconds: float, **kw):
    """Oracle MLUPS on a band sized for `seconds` of work; when the whole lattice takes
    less, whole-lattice steps are repeated until `seconds` have passed."""
    rows = _calibrated_rows(threads, seconds, **kw)
    band = OracleBand(rows, threads, **kw)
    dt, steps = 0.0, 0
    while steps == 0 or dt < 0.8 * seconds:
        dt += band.step()
        steps += 1
    return rows * L * steps / dt / 1e6, (rows, steps), dt


def cpu_baseline_measure(target_s: float = 12.0):
    """The FP64 definition oracle on all host cores (the reported baseline), plus two
    context rows: the same oracle on one core, and the fixed-moment MRT oracle (u~ = 0)
    on all cores."""
    import oracle

    threads = _oracle_threads()
    value, (rows, steps), dt = _band_mlups(threads, target_s)
    one, _, _ = _band_mlups(1, 3.0)
    mrt, (mrt_rows, mrt_steps), _ = _band_mlups(threads, 3.0, method=oracle.METHOD_MRT,
                                                mode=oracle.MODE_ZERO)
    return {"value": round(value, 3), "unit": "MLUPS", "cores": threads,
            "kind": "oracle",
            "sample": (f"{steps} time step(s) of a {L}x{rows} periodic band of the 4096^2 "
                       f"Taylor-Green workload, prescribed u~, FP64 definition oracle "
                       f"(per-node M(u~) and LU solve), {dt:.1f} s"),
            "single_core_mlups": round(one, 3),
            "plain_mrt_oracle_mlups": round(mrt, 3),
            "plain_mrt_sample": (f"{mrt_steps} step(s) of a {L}x{mrt_rows} band, fixed-moment "
                                 f"MRT oracle, u~ = 0, all cores")}


def reference_arm(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    threads = _oracle_threads()
    rows = _calibrated_rows(threads, 120.0 / (args.steps + args.warmup))
    band = OracleBand(rows, threads)
    for _ in range(args.warmup):
        band.step()
    total = sum(band.step() for _ in range(args.steps))
    per = total / args.steps
    value = rows * L / per / 1e6
    sample = (f"each step: one time step of a {L}x{rows} periodic band of the 4096^2 "
              f"Taylor-Green workload, FP64 definition oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_rows": rows},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--size", type=int, default=L,
                    help="lattice side (a smaller case for profiling captures)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="population storage of the timed run (profiling captures)")
    ap.add_argument("--mode", default="prescribed", choices=["zero", "fluid", "prescribed"],
                    help="relative velocity of the timed run (profiling captures)")
    ap.add_argument("--lattice", default="d2q9", choices=["d2q9", "d3q19"],
                    help="lattice of the timed run (d3q19: --size is the cube side)")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="N > 1: independent replicas (default), or one lattice of N stacked "
                         "Taylor-Green cells split into slabs with a halo exchange per step")
    ap.add_argument("--width", type=int, default=0,
                    help="nodes per thread of the step kernel (0: the library's choice; "
                         "profiling captures)")
    ap.add_argument("--scheme", default="rv", choices=["rv", "cascaded"],
                    help="D2Q9 relaxation of the timed run: the relative-velocity scheme's "
                         "orthogonal basis (rv) or Geier's cascaded basis (profiling captures)")
    ap.add_argument("--case", default="step", choices=["step", "adjoint", "sums"],
                    help="adjoint: only the adjoint workload's timings; sums: only the "
                         "conserved-sum checks (profiling captures)")
    ap.add_argument("--adjoint-steps", type=int, default=2000,
                    help="time steps of the adjoint workload's whole-gradient run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.case == "adjoint":
        adjoint_arm(args)
    elif args.case == "sums":
        sums_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
