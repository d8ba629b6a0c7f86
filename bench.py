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
    """Algorithmic bytes of one PCG iteration of one env (FP32): the BSR
    product q = A p (per 3x3 block 36 B of values + 4 B column id; row offsets
    4 B and p 12 B read, q 12 B written per vertex), the vector update (dx, r
    read + write 48 B; p, q 24 B and M^-1 24 B read; z 12 B written) and the
    direction update (z, p read 24 B; p written 12 B)."""
    nv, nnzb = info["nv"], info["nnzb"]
    spmv = nnzb * 40 + nv * (4 + 12 + 12)
    update = nv * (48 + 24 + 24 + 12)
    pupdate = nv * 36
    return spmv + update + pupdate


# algorithmic bytes per launch of the per-env kernels (FP32 mixed mode)
def algorithmic_bytes(name, info):
    nt, nv, nfc, nvc = info["nt"], info["nv"], info["nfc"], info["nvc"]
    npix = info["H"] * info["W"]
    table = {
        # tet ids 16 + Dm^-1 36 + sigma 24 written; displacement read once per vertex
        "k_stress": nt * (16 + 36 + 24) + 12 * nv,
        # parent 4 + tet ids 16 + Dm^-1 36 + face ids 12 + (p, A) 8 written + the
        # parent's fourth vertex 12; contact vertices: displacement 12 + rest
        # position 24 (FP64)
        "k_traction": nfc * (4 + 16 + 36 + 12 + 8 + 12) + nvc * 36,
        # CSR offsets 8 per vertex, incidence ids 4 x ~3 per face, (p, A) 8 per
        # face, vertex value 4 written
        "k_vertex_avg": nvc * (8 + 4) + nfc * (12 + 8),
        # covering face 4 + weights 12 + value 4 + mask 1 per pixel; face slots
        # and vertex values once
        "k_splat": npix * 21 + nfc * 12 + nvc * 4,
    }
    return table.get(name)


KERNEL_SRC = {"k_pcg_batched": "solver.cu", "k_stress": "elem.cu", "k_traction": "extract.cu",
              "k_vertex_avg": "extract.cu", "k_splat": "extract.cu"}


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


def _kernel_table(prof):
    tot = sum(v[0] for v in prof.values()) or 1.0
    top = sorted(prof.items(), key=lambda kv: -kv[1][0])
    return top, {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot, 4)} for k, v in top[:14]}


def _roofline(top, infos, pcg_iters_by_env, peak, peak_kind):
    """Roofline of the dominant kernel whose algorithmic bytes are known.
    k_pcg_batched: one launch runs every env of the phase for its own number of
    iterations, so bytes = sum over envs of (bytes per iteration x iterations)
    over the profiled region, divided by the kernel's total time there."""
    tot = sum(v[0] for _, v in top) or 1.0
    for name, (ms, n) in top:
        if n == 0:
            continue
        if name == "k_pcg_batched":
            total_bytes = sum(pcg_iteration_bytes(i) * it for i, it in zip(infos, pcg_iters_by_env))
            units = sum(pcg_iters_by_env) / n
        else:
            per = [algorithmic_bytes(name, i) for i in infos]
            if per[0] is None:
                continue
            total_bytes = sum(per) / len(per) * n  # per-env launches spread evenly over the envs
            units = None
        bytes_per_launch = total_bytes / n
        achieved = bytes_per_launch / (ms / n / 1e3) / 1e9
        tr = NCU_TRAFFIC.get(name)
        traffic = None
        if tr and tr["sha"] == src_sha(KERNEL_SRC[name]):
            traffic = tr["bytes_per_launch"]
        return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "bytes_per_launch": int(bytes_per_launch),
                "avg_launch_us": round(ms / n * 1e3, 2), "units_per_launch": (round(units, 2) if units else None),
                "share_of_kernel_time": round(ms / tot, 4)}
    return None


def _extraction_fracs(prof, infos, peak):
    out = {}
    for name in ("k_stress", "k_traction", "k_vertex_avg", "k_splat"):
        if name not in prof or prof[name][1] == 0:
            continue
        ms, n = prof[name]
        b = sum(algorithmic_bytes(name, i) for i in infos) / len(infos)
        out[name] = {"avg_launch_us": round(ms / n * 1e3, 2), "bytes_per_launch": int(b),
                     "frac": round(b / (ms / n / 1e3) / 1e9 / peak, 4)}
    return out


def stress_sweep(dev, stream, peak, sizes=(100_000, 1_000_000, 10_000_000), reps=10):
    """tc_stress_from_F over nt random SPD-perturbed F (||F - I|| <= 0.3):
    60 algorithmic bytes per tet (F read 36, sigma written 24)."""
    import torch
    from paper_2606_20426_gb300 import stress_from_F
    from synth.workloads import random_deformation_gradients
    res = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for nt in sizes:
        F = torch.from_numpy(random_deformation_gradients(7, nt).reshape(nt, 9).astype("float32")).to(dev)
        out = torch.empty((6, nt), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(3):
                stress_from_F(F, 0.3e6, 0.45, out=out, stream=stream)
            ts = []
            for r in range(reps):
                flush.fill_(float(r))
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                stress_from_F(F, 0.3e6, 0.45, out=out, stream=stream)
                z.record(stream)
                z.synchronize()
                ts.append(a.elapsed_time(z))
        ms = statistics.median(ts)
        gbs = 60.0 * nt / (ms / 1e3) / 1e9
        res[str(nt)] = {"us": round(ms * 1e3, 2), "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)}
        del F, out
    return res


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2606_20426_gb300 import Env, step_batch

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
        served = [Env(c, precision="fp32", stream=stream) for c in cfgs]
        plain = [Env(c, precision="fp32", stream=stream) for c in cfgs] if args.plain else []
    infos = [e.info for e in served]
    sig = [torch.empty((6, i["nt"]), dtype=torch.float32, device=dev) for i in infos]
    maps = [torch.empty((i["H"], i["W"]), dtype=torch.float32, device=dev) for i in infos]
    masks = [torch.empty((i["H"], i["W"]), dtype=torch.uint8, device=dev) for i in infos]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    cur = {"served": 0, "plain": [0] * B}

    def pose_of(b, k):
        c = cfgs[b]["bench_poses"]
        return c[k % len(c)]

    def extract(envs, host=None):
        for b, e in enumerate(envs):
            e.stress(sig[b])
            e.pressure_map(maps[b], masks[b])
            if host is not None:
                host[0][b].copy_(sig[b], non_blocking=True)
                host[1][b].copy_(maps[b], non_blocking=True)

    def served_step(host=None):
        k = cur["served"]
        cur["served"] += 1
        codes = step_batch(served, [pose_of(b, k) for b in range(B)])
        if any(codes):
            raise RuntimeError(f"tc_step_batch statuses {codes}")
        extract(served, host)

    def plain_step(b, host=None):
        k = cur["plain"][b]
        cur["plain"][b] += 1
        plain[b].step(pose_of(b, k))
        plain[b].stress(sig[b])
        plain[b].pressure_map(maps[b], masks[b])
        if host is not None:
            host[0][b].copy_(sig[b], non_blocking=True)
            host[1][b].copy_(maps[b], non_blocking=True)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            served_step()
            for b in range(len(plain)):
                plain_step(b)
        barrier()
        # ------------- timed region, served form: one batched call per step
        lat, total_ms = [], 0.0
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.fill_(float(k))
                torch.cuda.synchronize(dev)
                ev[0].record(stream)
                served_step()
                ev[1].record(stream)
                torch.cuda.synchronize(dev)
                ms = ev[0].elapsed_time(ev[1])
                total_ms += ms
                lat += [ms] * B  # every env's result is ready when the batch returns
        barrier()
        total_ms = max_over_ranks(total_ms)
        clocks = clk.summary()
        value = world * B * args.steps / (total_ms / 1e3)
        # ------------- plain form: one env per launch sequence, same requests
        plain_out = None
        if plain:
            plat, ptotal = [], 0.0
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(B)]
            for k in range(args.steps):
                flush.fill_(float(k))
                torch.cuda.synchronize(dev)
                for b in range(B):
                    evs[b][0].record(stream)
                    plain_step(b)
                    evs[b][1].record(stream)
                torch.cuda.synchronize(dev)
                plat += [a.elapsed_time(z) for a, z in evs]
                ptotal += sum(a.elapsed_time(z) for a, z in evs)
            barrier()
            ptotal = max_over_ranks(ptotal)
            plain_out = {"value": round(world * B * args.steps / (ptotal / 1e3), 3), "unit": UNIT,
                         "ms_per_step": round(ptotal / args.steps, 3),
                         "latency_ms": {"p50": round(float(np.percentile(plat, 50)), 3),
                                        "p99": round(float(np.percentile(plat, 99)), 3)},
                         "form": "plain: tc_step + tc_stress + tc_pressure_map per env, one env after another"}
        # ------------- end to end through the API with pinned host buffers
        host = ([torch.empty((6, i["nt"]), dtype=torch.float32).pin_memory() for i in infos],
                [torch.empty((i["H"], i["W"]), dtype=torch.float32).pin_memory() for i in infos])
        e2e_steps = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            served_step(host)
            torch.cuda.synchronize(dev)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        e2e_value = world * B * e2e_steps / e2e_s
        d2h = sum(4 * 6 * i["nt"] + 4 * i["H"] * i["W"] for i in infos)
        h2d = B * 96  # the target pose (12 doubles) per env-step
        # ------------- per-kernel times of a profiled repeat of the served steps
        pcg0 = [e.get_info()["pcg_iters"] for e in served]
        for e in served:
            e.profile(True)
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            served_step()
        torch.cuda.synchronize(dev)
        pcg_by_env = [e.get_info()["pcg_iters"] - p0 for e, p0 in zip(served, pcg0)]
        prof = {}
        for e in served:
            for name, (ms, n) in e.kernel_times().items():
                a, c = prof.get(name, (0.0, 0))
                prof[name] = (a + ms, c + n)
            e.profile(False)
    launches = sum(n for _, n in prof.values())
    peak, peak_kind = peaks()
    top, kernel_table = _kernel_table(prof)
    roof = _roofline(top, infos, pcg_by_env, peak, peak_kind)
    steps_done = max(1, sum(e.get_info()["steps"] for e in served))
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "envs_per_gpu": B,
                   "form": "batched: one tc_step_batch over all envs (one launch per Newton phase), "
                           "then tc_stress + tc_pressure_map per env",
                   "l2": "flushed between timed steps (256 MB write)",
                   "tets_per_env": [i["nt"] for i in infos][:4], "verts_per_env": [i["nv"] for i in infos][:4]},
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3)},
        "plain": plain_out,
        "clocks": clocks,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roof,
        "extraction": _extraction_fracs(prof, infos, peak),
        "kernels": kernel_table,
        "solver": {"newton_per_env_step": sum(e.get_info()["newton_iters"] for e in served) / steps_done,
                   "pcg_per_env_step": sum(e.get_info()["pcg_iters"] for e in served) / steps_done},
    }
    for e in served + plain:
        e.close()
    if args.sweep:
        out["stress_sweep"] = stress_sweep(dev, stream, peak)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(out["solver"]["newton_per_env_step"], args.cpu_seconds)
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
    ap.add_argument("--envs", type=int, default=8)
    ap.add_argument("--plain", type=int, default=1, help="also time the plain one-env-per-launch form")
    ap.add_argument("--sweep", type=int, default=1, help="also run the tc_stress_from_F size sweep")
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
