"""Throughput benchmark: env-steps/s of one TaCauchy env-step (implicit IPC
step + per-tet Cauchy stress + pressure map) on GelSight-Mini-like pads.

Workload (synthetic, seeded): graded 18x24x4 mm pad of ~60k tets, E = 0.3 MPa,
nu = 0.45, bottom fixed, pressed by a seeded sphere / cylinder / filleted box
to depth U[0.2, 1.0] mm with slip U[0, 0.5] mm over 20 dynamic steps at
dt = 1/60 s (then released along the same path), 240x320 pressure map, FP32
element/barrier/PCG arithmetic with FP64 reductions.  One bench step = every
env on this GPU advances by one env-step; value = env-steps/s over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--envs B] [--impl ours|reference]

Rank 0 prints one JSON line.  --impl reference times the FP64 CPU oracle
(oracle/) on the host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s (step+stress+pressure map) served vs plain GPU form; p50/p99 latency"
UNIT = "env-steps/s"
WORKLOAD = ("gelsight-like graded pad 18x24x4 mm, ~60k tets, sphere/cylinder/box indenter, "
            "20 dynamic steps dt=1/60 s, 240x320 map, FP32 mixed")

# DRAM traffic per launch unit from the committed ncu captures (profiles/),
# keyed by kernel; valid only while the kernel's source file is unchanged.
NCU_TRAFFIC = {}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


def pcg_iteration_bytes(info):
    """Algorithmic bytes of one PCG iteration of one env (FP32): element SpMV
    (tet ids 16, Dm^-1 36, volume 4, H9 180 read, 12 slot values 48 written, p
    read once per vertex), contact SpMV (per primitive: ids, packed block,
    result), per-vertex gather of the slots (CSR offset, incidence id and 3
    values per incidence; q written), the update (dx, r read+write; p, q,
    M^-1 read; z written) and the direction update (z, p read; p written)."""
    nt, nv = info["nt"], info["nv"]
    nvc, nec, nfc = info["nvc"], info["nec"], info["nfc"]
    deg = 4.0 * nt / nv
    spmv = nt * (16 + 36 + 4 + 180 + 48) + 12 * nv
    contact = nvc * (4 + 24 + 12 + 12) + nec * (8 + 84 + 24 + 24) + nfc * (12 + 180 + 36 + 36)
    gather = nv * (4 + deg * (4 + 12) + 12 + 12 + 1)
    update = nv * (24 + 24 + 12 + 12 + 24 + 12)
    pupdate = nv * (12 + 24)
    return spmv + contact + gather + update + pupdate


# algorithmic bytes per launch of the kernels of one env (FP32 mixed mode)
def algorithmic_bytes(name, info, pcg_iters_per_launch=None):
    nt, nv = info["nt"], info["nv"]
    deg = 4.0 * nt / nv  # tet incidences per vertex
    if name == "k_pcg_persistent":
        return pcg_iteration_bytes(info) * pcg_iters_per_launch if pcg_iters_per_launch else None
    table = {
        # idx 16 + Dm^-1 36 + vol 4 + H9 180 (read) + 12 outputs 48 (write); p read once per vertex
        "k_spmv_elem": nt * (16 + 36 + 4 + 180 + 48) + 12 * nv,
        # idx 16 + Dm^-1 36 + vol 4 (read) + H9 180 + 36 slots 144 (write); u read once per vertex
        "k_elem_hess": nt * (16 + 36 + 4 + 180 + 144) + 12 * nv,
        "k_elem_energy": nt * (16 + 36 + 4) + 12 * nv,
        # CSR offsets + incidence ids + 12 slot values per incidence; p read, q write
        "k_pcg_q": nv * (4 + deg * (4 + 12) + 12 + 12 + 1),
        # dx, r (read+write), p, q, Minv (read), z (write)
        "k_pcg_update": nv * (24 + 24 + 12 + 12 + 24 + 12),
        "k_pcg_p": nv * (12 + 24),
        # CSR + 36 slot values per incidence; g and Minv written
        "k_assemble": nv * (4 + deg * (4 + 36) + 12 + 24 + 1),
        "k_stress": nt * (16 + 36 + 24) + 12 * nv,
        "k_axpy": nv * 36,
    }
    return table.get(name)


KERNEL_SRC = {"k_pcg_persistent": "solver.cu", "k_spmv_elem": "solver.cu", "k_pcg_q": "solver.cu", "k_pcg_update": "solver.cu",
              "k_pcg_p": "solver.cu", "k_assemble": "solver.cu", "k_elem_hess": "elem.cu",
              "k_elem_energy": "elem.cu", "k_stress": "elem.cu", "k_axpy": "solver.cu"}


def src_sha(fname):
    p = os.path.join(ROOT, "paper_2606_20426_gb300", "csrc", fname)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names[1:], parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


def make_envs(B, rank):
    from synth import meshes, workloads
    mesh = meshes.graded_pad()
    envs = []
    for b in range(B):
        e = workloads.gelsight_env(1000 * rank + b, mesh=mesh)
        # load 20 steps, then unload along the same path (cycled)
        e["bench_poses"] = e["poses"] + e["poses"][-2::-1] + [e["start_pose"]]
        envs.append(e)
    return envs


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2606_20426_gb300 import Env

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    B = args.envs
    cfgs = make_envs(B, rank)
    with torch.cuda.stream(stream):
        envs = [Env(c, precision="fp32", stream=stream) for c in cfgs]
    infos = [e.info for e in envs]
    sig = [torch.empty((6, i["nt"]), dtype=torch.float32, device=dev) for i in infos]
    maps = [torch.empty((i["H"], i["W"]), dtype=torch.float32, device=dev) for i in infos]
    masks = [torch.empty((i["H"], i["W"]), dtype=torch.uint8, device=dev) for i in infos]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    cursor = [0] * B

    def env_step(b, host=None):
        e, c = envs[b], cfgs[b]
        pose = c["bench_poses"][cursor[b] % len(c["bench_poses"])]
        cursor[b] += 1
        e.step(pose)
        e.stress(sig[b])
        e.pressure_map(maps[b], masks[b])
        if host is not None:
            host[0][b].copy_(sig[b], non_blocking=True)
            host[1][b].copy_(maps[b], non_blocking=True)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            for b in range(B):
                env_step(b)
        barrier()
        # ---------------- timed region (device time, L2 flushed between steps)
        lat = []
        total_ms = 0.0
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(B)]
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.fill_(float(k))
                torch.cuda.synchronize(dev)
                for b in range(B):
                    ev[b][0].record(stream)
                    env_step(b)
                    ev[b][1].record(stream)
                torch.cuda.synchronize(dev)
                step_ms = sum(a.elapsed_time(z) for a, z in ev)
                lat += [a.elapsed_time(z) for a, z in ev]
                total_ms += step_ms
        barrier()
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        clocks = clk.summary()
        value = world * B * args.steps / (total_ms / 1e3)
        # ---------------- end-to-end through the API with host buffers
        host = ([torch.empty((6, i["nt"]), dtype=torch.float32).pin_memory() for i in infos],
                [torch.empty((i["H"], i["W"]), dtype=torch.float32).pin_memory() for i in infos])
        e2e_steps = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for b in range(B):
                env_step(b, host)
            torch.cuda.synchronize(dev)
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_value = world * B * e2e_steps / e2e_s
        d2h = sum(4 * 6 * i["nt"] + 4 * i["H"] * i["W"] for i in infos)
        h2d = B * 96  # the target pose (12 doubles) per env-step
        # ---------------- per-kernel times of a profiled repeat of the timed steps
        pcg0 = sum(e.get_info()["pcg_iters"] for e in envs)
        for e in envs:
            e.profile(True)
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            for b in range(B):
                env_step(b)
        torch.cuda.synchronize(dev)
        pcg_profiled = sum(e.get_info()["pcg_iters"] for e in envs) - pcg0
        prof = {}
        for e in envs:
            for name, (ms, n) in e.kernel_times().items():
                a, c = prof.get(name, (0.0, 0))
                prof[name] = (a + ms, c + n)
            e.profile(False)
    launches = sum(n for _, n in prof.values())
    top = sorted(prof.items(), key=lambda kv: -kv[1][0])
    roof = None
    peak, peak_kind = peaks()
    for name, (ms, n) in top:
        it_per_launch = pcg_profiled / n if name == "k_pcg_persistent" and n else None
        per = [algorithmic_bytes(name, i, it_per_launch) for i in infos]
        if per[0] is None or n == 0:
            continue
        # launches spread evenly over the B envs of this rank
        bytes_per_launch = sum(per) / len(per)
        achieved = bytes_per_launch / (ms / n / 1e3) / 1e9
        tr = NCU_TRAFFIC.get(name)
        traffic = None
        if tr and tr["sha"] == src_sha(KERNEL_SRC[name]):
            traffic = tr["bytes_per_unit"] * (sum(i["nt"] for i in infos) / len(infos))
        roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "units_per_launch": (round(it_per_launch, 2) if it_per_launch else None),
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "bytes_per_launch": int(bytes_per_launch), "avg_launch_us": ms / n * 1e3,
                "share_of_kernel_time": round(ms / sum(v[0] for v in prof.values()), 4)}
        break
    tot_ms = sum(v[0] for v in prof.values())
    kernel_table = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot_ms, 4)}
                    for k, v in top[:12]}
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "envs_per_gpu": B, "form": "plain (one env per launch sequence)",
                   "l2": "flushed between timed steps (256 MB write)", "tets_per_env": infos[0]["nt"],
                   "verts_per_env": infos[0]["nv"]},
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3)},
        "clocks": clocks,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches // max(1, args.steps) * args.steps),
        "roofline": roof,
        "kernels": kernel_table,
        "solver": {"newton_per_env_step": sum(e.get_info()["newton_iters"] for e in envs) /
                   max(1, sum(e.get_info()["steps"] for e in envs)),
                   "pcg_per_env_step": sum(e.get_info()["pcg_iters"] for e in envs) /
                   max(1, sum(e.get_info()["steps"] for e in envs))},
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(out["solver"]["newton_per_env_step"], args.cpu_seconds)
    for e in envs:
        e.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
from synth import workloads
from oracle.sim import Scene
budget = {budget}
env = workloads.gelsight_env(0)
t0 = time.perf_counter(); sc = Scene(env); t_setup = time.perf_counter() - t0
Y0 = sc.indenter(sc.pose); Y1 = sc.indenter(env["poses"][0])
frac, _ = sc.ccd_alpha(sc.x, 0 * sc.x, Y0, Y1)
s = 1.0 if frac >= 1 else frac
Ys = (1 - s) * Y0 + s * Y1
x = sc.x.copy(); xt = x + sc.h * sc.v
its = 0; t0 = time.perf_counter()
import numpy as np
import scipy.sparse.linalg as spla
fr = np.repeat(sc.free, 3)
while time.perf_counter() - t0 < budget or its == 0:
    E, g, H = sc.gradient_hessian(x, Ys, xt)
    g[~sc.free] = 0
    p = np.zeros(3 * sc.nv); p[fr] = spla.spsolve(H[fr][:, fr].tocsc(), -g.ravel()[fr]); p = p.reshape(-1, 3)
    a, cand = sc.ccd_alpha(x, p, Ys)
    for _ in range(61):
        if sc.energy(x + a * p, Ys, cand, xt) <= E: break
        a *= 0.5
    x = x + a * p; its += 1
t_newton = (time.perf_counter() - t0) / its
t0 = time.perf_counter(); sig = sc.stress(x); m = sc.pressure_map(x=x); t_ext = time.perf_counter() - t0
print(json.dumps(dict(t_newton=t_newton, iters=its, t_extract=t_ext, t_setup=t_setup, nt=sc.nt)))
"""


def cpu_baseline(newton_per_env_step, budget):
    """The oracle, single-threaded, on a bounded sample: Newton iterations of
    the first substep of one GelSight-like env for ~budget seconds, plus one
    stress + pressure-map extraction; env-steps/s = 1 / (t_newton x Newton
    iterations per env-step + t_extract), with the iteration count per
    env-step taken from the timed run (same solver settings)."""
    envv = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, budget=float(budget))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=envv, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per_env_step = d["t_newton"] * newton_per_env_step + d["t_extract"]
    return {"value": round(1.0 / per_env_step, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{d['iters']} oracle Newton iterations ({d['t_newton']:.2f} s each) of the first substep of "
                       f"one {d['nt']}-tet env + one stress/pressure-map extraction ({d['t_extract']:.2f} s), "
                       f"scaled by {newton_per_env_step:.1f} Newton iterations per env-step")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.perf_counter()
    samples = []
    newton_per_env_step = args.ref_newton_per_step
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(newton_per_env_step, max(2.0, args.cpu_seconds / max(1, args.steps)))
        if k >= args.warmup:
            samples.append(cb)
    vals = [s["value"] for s in samples if s.get("value")]
    value = statistics.mean(vals) if vals else None
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": (1e3 / value) if value else None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "envs_per_gpu": 1, "form": "FP64 CPU oracle, single thread"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": samples[-1].get("sample") if samples else None},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--envs", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-newton-per-step", type=float, default=40.0,
                    help="Newton iterations per env-step used to scale the reference arm's sample")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
