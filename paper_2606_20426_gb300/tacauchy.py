"""Python binding of the C ABI in include/tacauchy.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
(paper_2606_20426_gb300/libtacauchy.so).  PyTorch supplies device memory
(its caching allocator backs every env allocation) and streams; outputs are
torch CUDA tensors.  There is no CPU fallback: importing works without a GPU
(for builds and symbol checks), but every call that computes needs the
library and a CUDA device and raises otherwise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtacauchy.so")

TC_FP64, TC_FP32_MIXED = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid mesh", 3: "initial penetration", 4: "newton maxiter",
          5: "pcg maxiter", 6: "line search", 7: "non-finite", 8: "cuda error", 9: "out of memory",
          10: "admission", 11: "timeout", 12: "capacity"}

# every symbol include/tacauchy.h declares
EXPORTS = ["tc_create_scene", "tc_step", "tc_step_batch", "tc_stress", "tc_traction", "tc_pressure_map", "tc_contact_force",
           "tc_surface_faces", "tc_boundary_faces", "tc_pixel_table", "tc_get_positions", "tc_set_positions",
           "tc_env_info", "tc_destroy", "tc_status_str", "tc_stress_from_F", "tc_profile_enable",
           "tc_profile_read", "tc_pressure_map_noalloc", "tc_server_create", "tc_submit", "tc_poll", "tc_wait",
           "tc_server_info", "tc_server_stream", "tc_server_destroy", "tc_pcg_shape", "tc_autotune_pcg",
           "tc_energy_gradient", "tc_extract_batch", "tc_vertex_forces", "tc_force_pressure_map",
           "tc_depth_map"]


class TcError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")


class Mesh(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("nv", ctypes.c_int32), ("tets", ctypes.c_void_p), ("nt", ctypes.c_int32)]


class Material(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("density", ctypes.c_double),
                ("per_tet_E_nu", ctypes.c_void_p), ("model", ctypes.c_int32)]


# material laws (tc_material.model)
MODELS = {"snh": 0, "snh_log": 1}


class SceneOpts(ctypes.Structure):
    _fields_ = [("dhat", ctypes.c_double), ("kappa", ctypes.c_double), ("dt", ctypes.c_double),
                ("newton_rtol", ctypes.c_double), ("newton_max", ctypes.c_int32), ("pcg_max", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("contact_axis", ctypes.c_int32),
                ("friction_mu", ctypes.c_double), ("friction_eps_v", ctypes.c_double)]


class TriMesh(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("nv", ctypes.c_int32), ("F", ctypes.c_void_p), ("nf", ctypes.c_int32)]


class Pose(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class Grid(ctypes.Structure):
    _fields_ = [("axis_u", ctypes.c_int32), ("axis_v", ctypes.c_int32), ("origin", ctypes.c_double * 2),
                ("pixel", ctypes.c_double * 2), ("H", ctypes.c_int32), ("W", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_double), ("launches", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("rounds", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("queued", ctypes.c_int32), ("inflight", ctypes.c_int32), ("peak_inflight", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("workers", ctypes.c_int32), ("inflight_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("evictions", ctypes.c_int64), ("known_envs", ctypes.c_int32)]


class PcgTune(ctypes.Structure):
    _fields_ = [("cluster_ctas", ctypes.c_int32), ("threads", ctypes.c_int32), ("coresident", ctypes.c_int32),
                ("us_per_env_iter", ctypes.c_double), ("env_iters", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32), ("nf", ctypes.c_int32), ("nfc", ctypes.c_int32),
                ("nec", ctypes.c_int32), ("nvc", ctypes.c_int32), ("ind_nv", ctypes.c_int32),
                ("ind_nf", ctypes.c_int32), ("ind_ne", ctypes.c_int32), ("H", ctypes.c_int32),
                ("W", ctypes.c_int32), ("newton_iters", ctypes.c_int64), ("pcg_iters", ctypes.c_int64),
                ("substeps", ctypes.c_int64), ("steps", ctypes.c_int64), ("line_search_halvings", ctypes.c_int64),
                ("kappa", ctypes.c_double), ("device_bytes", ctypes.c_size_t), ("nnzb", ctypes.c_int64),
                ("pcg_capped", ctypes.c_int64), ("working_bytes", ctypes.c_size_t),
                ("working_resident", ctypes.c_int32)]


_lib = None


def load():
    """Load libtacauchy.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2606_20426_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    sig = {
        "tc_create_scene": [ctypes.POINTER(Mesh), ctypes.POINTER(Material), P, ctypes.c_int32,
                            ctypes.POINTER(TriMesh), ctypes.POINTER(Pose), ctypes.POINTER(SceneOpts),
                            ctypes.POINTER(Grid), ctypes.POINTER(Allocator), P, ctypes.POINTER(P)],
        "tc_step": [P, ctypes.POINTER(Pose)],
        "tc_step_batch": [ctypes.POINTER(P), ctypes.c_int32, ctypes.POINTER(Pose), ctypes.POINTER(ctypes.c_int32)],
        "tc_stress": [P, P],
        "tc_traction": [P, P, P, P],
        "tc_pressure_map": [P, ctypes.POINTER(Grid), P, P],
        "tc_extract_batch": [ctypes.POINTER(P), ctypes.c_int32, ctypes.POINTER(P), ctypes.POINTER(P),
                             ctypes.POINTER(P)],
        "tc_contact_force": [P, P],
        "tc_vertex_forces": [P, P, P, P, P],
        "tc_depth_map": [P, ctypes.POINTER(Grid), P, P],
        "tc_force_pressure_map": [P, ctypes.POINTER(Grid), P, P],
        "tc_energy_gradient": [P, P, P],
        "tc_surface_faces": [P, P, P],
        "tc_boundary_faces": [P, P, P],
        "tc_pixel_table": [P, P, P],
        "tc_get_positions": [P, P],
        "tc_set_positions": [P, P],
        "tc_env_info": [P, ctypes.POINTER(Info)],
        "tc_stress_from_F": [P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, P, P],
        "tc_profile_enable": [P, ctypes.c_int32],
        "tc_profile_read": [P, ctypes.POINTER(KernelTime), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
        "tc_pressure_map_noalloc": [P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, ctypes.c_int32, P, P,
                                    ctypes.c_int32, P, P, ctypes.c_int32, P, P, P],
        "tc_server_create": [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(P)],
        "tc_server_stream": [P, ctypes.c_int32, ctypes.POINTER(P)],
        "tc_submit": [P, P, ctypes.POINTER(Pose), P, P, P, ctypes.POINTER(ctypes.c_uint64)],
        "tc_poll": [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(Result)],
        "tc_wait": [P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(Result)],
        "tc_server_info": [P, ctypes.POINTER(ServerStats)],
        "tc_pcg_shape": [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
        "tc_autotune_pcg": [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(PcgTune),
                            ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    lib.tc_destroy.argtypes = [P]
    lib.tc_destroy.restype = None
    lib.tc_server_destroy.argtypes = [P]
    lib.tc_server_destroy.restype = None
    lib.tc_status_str.argtypes = [ctypes.c_int32]
    lib.tc_status_str.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code, where):
    if code != 0:
        raise TcError(code, where)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("tacauchy needs a CUDA device")
    return torch


def make_pose(p):
    """dict(R=(3,3), t=(3,)) or Pose -> Pose."""
    if isinstance(p, Pose):
        return p
    out = Pose()
    R = np.asarray(p["R"], dtype=np.float64).reshape(9)
    t = np.asarray(p["t"], dtype=np.float64).reshape(3)
    for k in range(9):
        out.R[k] = R[k]
    for k in range(3):
        out.t[k] = t[k]
    return out


def make_grid(g):
    """dict(axis_u, axis_v, origin, pixel, H, W) -> Grid."""
    return Grid(int(g["axis_u"]), int(g["axis_v"]), (ctypes.c_double * 2)(*[float(v) for v in g["origin"]]),
                (ctypes.c_double * 2)(*[float(v) for v in g["pixel"]]), int(g["H"]), int(g["W"]))


class _TorchAllocator:
    """tc_allocator backed by the PyTorch caching allocator."""

    def __init__(self, torch):
        self.torch = torch

        def alloc(ctx, nbytes, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:
                return None

        def release(ctx, ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc = ALLOC_FN(alloc)
        self._release = RELEASE_FN(release)
        self.struct = Allocator(self._alloc, self._release, None)


class Env:
    """One simulated sensor: gel pad + rigid indenter + pixel grid."""

    def __init__(self, env, precision=None, stream=None, torch_allocator=True, allocator=None):
        """allocator: an object whose `.struct` is an Allocator (tc_allocator)
        to use instead of the PyTorch caching allocator."""
        torch = _torch()
        lib = load()
        self.torch, self.lib = torch, lib
        X = np.ascontiguousarray(env["X"], dtype=np.float64)
        T = np.ascontiguousarray(env["tets"], dtype=np.int32)
        fixed = np.ascontiguousarray(env["fixed"], dtype=np.int32)
        V = np.ascontiguousarray(env["ind_V"], dtype=np.float64)
        F = np.ascontiguousarray(env["ind_F"], dtype=np.int32)
        self._keep = (X, T, fixed, V, F)
        m, o = env["material"], env["opts"]
        prec = precision if precision is not None else o.get("precision", "fp64")
        if isinstance(prec, str):
            prec = TC_FP64 if prec == "fp64" else TC_FP32_MIXED
        self.precision = prec
        mesh = Mesh(X.ctypes.data, X.shape[0], T.ctypes.data, T.shape[0])
        per_tet = None
        if m.get("per_tet") is not None:
            per_tet = np.ascontiguousarray(m["per_tet"], dtype=np.float64).reshape(-1, 2)
        self._keep = self._keep + (per_tet,)
        law = m.get("model", "snh")
        if law not in MODELS:
            raise ValueError(f"unknown material law {law!r}")
        mat = Material(m["E"], m["nu"], m["density"], per_tet.ctypes.data if per_tet is not None else None,
                       MODELS[law])
        opts = SceneOpts(o["dhat"], o.get("kappa", 0.0), o.get("dt", 0.0), o.get("newton_rtol", 1e-6),
                         o.get("newton_max", 1024), o.get("pcg_max", 1000), prec, o.get("contact_axis", -1),
                         o.get("friction_mu", 0.0), o.get("friction_eps_v", 0.01))
        ind = TriMesh(V.ctypes.data, V.shape[0], F.ctypes.data, F.shape[0])
        g = env.get("grid")
        grid = make_grid(g) if g is not None else None
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if allocator is not None:
            self._allocator = allocator
        else:
            self._allocator = _TorchAllocator(torch) if torch_allocator else None
        handle = ctypes.c_void_p()
        pose = make_pose(env["start_pose"])
        code = lib.tc_create_scene(ctypes.byref(mesh), ctypes.byref(mat), fixed.ctypes.data, len(fixed),
                                   ctypes.byref(ind), ctypes.byref(pose), ctypes.byref(opts),
                                   ctypes.byref(grid) if grid is not None else None,
                                   ctypes.byref(self._allocator.struct) if self._allocator else None,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
        _check(code, "tc_create_scene")
        self.h = handle
        self.info = self.get_info()

    # ------------------------------------------------------------- calls
    def get_info(self):
        inf = Info()
        _check(self.lib.tc_env_info(self.h, ctypes.byref(inf)), "tc_env_info")
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def step(self, pose):
        p = make_pose(pose)
        _check(self.lib.tc_step(self.h, ctypes.byref(p)), "tc_step")

    def stress(self, out=None):
        """(6, nt) float32 CUDA tensor: xx, yy, zz, xy, yz, zx."""
        nt = self.info["nt"]
        if out is None:
            out = self.torch.empty((6, nt), dtype=self.torch.float32, device="cuda")
        _check(self.lib.tc_stress(self.h, ctypes.c_void_p(out.data_ptr())), "tc_stress")
        return out

    def traction(self):
        n = self.info["nfc"]
        t = self.torch.empty((3, n), dtype=self.torch.float32, device="cuda")
        p = self.torch.empty((n,), dtype=self.torch.float32, device="cuda")
        tt = self.torch.empty((3, n), dtype=self.torch.float32, device="cuda")
        _check(self.lib.tc_traction(self.h, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                    ctypes.c_void_p(tt.data_ptr())), "tc_traction")
        return t, p, tt

    def pressure_map(self, out=None, mask=None, want_mask=True, grid=None):
        """(H, W) float32 map and uint8 mask on `grid` (a dict like the env's
        "grid" entry), or on the grid given at create time when None."""
        if grid is None:
            H, W = self.info["H"], self.info["W"]
            g = None
        else:
            H, W = int(grid["H"]), int(grid["W"])
            g = make_grid(grid)
        if out is None:
            out = self.torch.empty((H, W), dtype=self.torch.float32, device="cuda")
        if mask is None and want_mask:
            mask = self.torch.empty((H, W), dtype=self.torch.uint8, device="cuda")
        _check(self.lib.tc_pressure_map(self.h, ctypes.byref(g) if g is not None else None,
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(mask.data_ptr()) if mask is not None else None),
               "tc_pressure_map")
        return out, mask

    def energy_gradient(self):
        """(E, g): the incremental potential at the current state and its
        gradient (nv, 3) with fixed vertices zeroed."""
        E = ctypes.c_double()
        g = np.empty((self.info["nv"], 3), dtype=np.float64)
        _check(self.lib.tc_energy_gradient(self.h, ctypes.byref(E), g.ctypes.data), "tc_energy_gradient")
        return E.value, g

    def vertex_forces(self):
        """Algorithm 2 per contact vertex: (f, f_n, f_tau) as (3, nvc) and p
        (nvc,) float32 CUDA tensors."""
        n = self.info["nvc"]
        t = [self.torch.empty((3, n), dtype=self.torch.float32, device="cuda") for _ in range(3)]
        p = self.torch.empty((n,), dtype=self.torch.float32, device="cuda")
        _check(self.lib.tc_vertex_forces(self.h, *[ctypes.c_void_p(x.data_ptr()) for x in t],
                                         ctypes.c_void_p(p.data_ptr())), "tc_vertex_forces")
        return t[0], t[1], t[2], p

    def force_pressure_map(self, grid=None, out=None, mask=None):
        """(H, W) map of the contact-force pressure |f_k| / A_k and its mask."""
        g = make_grid(grid) if grid is not None else None
        H, W = (int(grid["H"]), int(grid["W"])) if grid is not None else (self.info["H"], self.info["W"])
        if out is None:
            out = self.torch.empty((H, W), dtype=self.torch.float32, device="cuda")
        if mask is None:
            mask = self.torch.empty((H, W), dtype=self.torch.uint8, device="cuda")
        _check(self.lib.tc_force_pressure_map(self.h, ctypes.byref(g) if g is not None else None,
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr())),
               "tc_force_pressure_map")
        return out, mask

    def depth_map(self, grid=None, out=None, mask=None):
        """(H, W) float32 height of the deformed contact surface seen from the
        contact side, and its coverage mask (tc_depth_map)."""
        g = make_grid(grid) if grid is not None else None
        H, W = (int(grid["H"]), int(grid["W"])) if grid is not None else (self.info["H"], self.info["W"])
        if out is None:
            out = self.torch.empty((H, W), dtype=self.torch.float32, device="cuda")
        if mask is None:
            mask = self.torch.empty((H, W), dtype=self.torch.uint8, device="cuda")
        _check(self.lib.tc_depth_map(self.h, ctypes.byref(g) if g is not None else None,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr())),
               "tc_depth_map")
        return out, mask

    def contact_force(self):
        f = np.zeros(3)
        _check(self.lib.tc_contact_force(self.h, f.ctypes.data), "tc_contact_force")
        return f

    def surface_faces(self):
        n = self.info["nfc"]
        f = np.zeros((n, 3), dtype=np.int32)
        p = np.zeros(n, dtype=np.int32)
        _check(self.lib.tc_surface_faces(self.h, f.ctypes.data, p.ctypes.data), "tc_surface_faces")
        return f, p

    def boundary_faces(self):
        n = self.info["nf"]
        f = np.zeros((n, 3), dtype=np.int32)
        p = np.zeros(n, dtype=np.int32)
        _check(self.lib.tc_boundary_faces(self.h, f.ctypes.data, p.ctypes.data), "tc_boundary_faces")
        return f, p

    def pixel_table(self):
        n = self.info["H"] * self.info["W"]
        f = np.zeros(n, dtype=np.int32)
        w = np.zeros((n, 3), dtype=np.float32)
        _check(self.lib.tc_pixel_table(self.h, f.ctypes.data, w.ctypes.data), "tc_pixel_table")
        return f, w

    def positions(self):
        x = np.zeros((self.info["nv"], 3))
        _check(self.lib.tc_get_positions(self.h, x.ctypes.data), "tc_get_positions")
        return x

    def set_positions(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        _check(self.lib.tc_set_positions(self.h, x.ctypes.data), "tc_set_positions")

    def profile(self, on=True):
        """Enable (and clear) or disable per-kernel timing."""
        _check(self.lib.tc_profile_enable(self.h, 1 if on else 0), "tc_profile_enable")

    def kernel_times(self):
        """{kernel name: (total ms, launches)} since profiling was enabled."""
        buf = (KernelTime * 64)()
        n = ctypes.c_int32()
        _check(self.lib.tc_profile_read(self.h, buf, 64, ctypes.byref(n)), "tc_profile_read")
        return {buf[i].name.decode(): (buf[i].ms, buf[i].launches) for i in range(min(n.value, 64))}

    def close(self):
        if getattr(self, "h", None):
            self.lib.tc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _result(r):
    return {"status": int(r.status), "queue_us": r.queue_us, "latency_us": r.latency_us, "rounds": int(r.rounds)}


class Server:
    """Continuous-batching step server (tc_server_*): submit() queues one step
    of an env and returns a ticket; wait()/poll() collect the result."""

    TIMEOUT = 11

    def __init__(self, hbm_budget_bytes, max_slots, workers=0):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.tc_server_create(int(hbm_budget_bytes), int(max_slots), int(workers), ctypes.byref(h)),
               "tc_server_create")
        self.h = h

    def submit(self, env, pose, sigma=None, map=None, mask=None):
        """Queue a step of `env` toward `pose`; sigma (6, nt), map (H, W) and
        mask (H, W) are optional CUDA tensors written when the step is done."""
        p = make_pose(pose)
        t = ctypes.c_uint64()
        _check(self.lib.tc_submit(self.h, env.h, ctypes.byref(p), _ptr(sigma), _ptr(map), _ptr(mask),
                                  ctypes.byref(t)), "tc_submit")
        return t.value

    def poll(self, ticket):
        done = ctypes.c_int32()
        r = Result()
        _check(self.lib.tc_poll(self.h, ticket, ctypes.byref(done), ctypes.byref(r)), "tc_poll")
        return _result(r) if done.value else None

    def wait(self, ticket, timeout_s=60.0):
        """The request's result dict, or None if it is not done in time."""
        r = Result()
        code = self.lib.tc_wait(self.h, ticket, int(timeout_s * 1e6), ctypes.byref(r))
        if code == self.TIMEOUT:
            return None
        _check(code, "tc_wait")
        return _result(r)

    def info(self):
        st = ServerStats()
        _check(self.lib.tc_server_info(self.h, ctypes.byref(st)), "tc_server_info")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def streams(self):
        """The workers' CUDA streams as torch streams (for events)."""
        torch = _torch()
        out = []
        for w in range(self.info()["workers"]):
            p = ctypes.c_void_p()
            _check(self.lib.tc_server_stream(self.h, w, ctypes.byref(p)), "tc_server_stream")
            out.append(torch.cuda.ExternalStream(p.value))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.tc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcg_shape(precision, cluster_ctas, threads):
    """Select the PCG launch shape (process-wide for the precision)."""
    prec = TC_FP64 if precision in ("fp64", TC_FP64) else TC_FP32_MIXED
    _check(load().tc_pcg_shape(prec, int(cluster_ctas), int(threads)), "tc_pcg_shape")


def autotune_pcg(envs, mode="latency"):
    """Time the envs' PCG solves under every launch shape, keep the fastest;
    mode "latency": each env's solve alone, "throughput": one launch over all.
    Returns one dict per shape tried."""
    envs = list(envs)
    lib = load()
    handles = (ctypes.c_void_p * len(envs))(*[e.h for e in envs])
    res = (PcgTune * 8)()
    n = ctypes.c_int32()
    m = 1 if mode == "throughput" else 0
    _check(lib.tc_autotune_pcg(handles, len(envs), m, res, 8, ctypes.byref(n)), "tc_autotune_pcg")
    return [{k: getattr(res[i], k) for k, _ in PcgTune._fields_} for i in range(min(n.value, 8))]


def step_batch(envs, poses, raise_on_error=False):
    """One step of each env in `envs` toward the matching pose, all Newton
    phases launched once over the whole batch (tc_step_batch).  Returns the
    list of per-env status codes; with raise_on_error the first non-zero one
    raises TcError."""
    envs = list(envs)
    poses = list(poses)
    if len(envs) != len(poses):
        raise ValueError("one pose per env")
    n = len(envs)
    lib = load()
    handles = (ctypes.c_void_p * max(n, 1))(*[e.h for e in envs])
    targets = (Pose * max(n, 1))(*[make_pose(p) for p in poses])
    statuses = (ctypes.c_int32 * max(n, 1))()
    _check(lib.tc_step_batch(handles, n, targets, statuses), "tc_step_batch")
    out = [int(statuses[i]) for i in range(n)]
    if raise_on_error:
        for code in out:
            _check(code, "tc_step_batch")
    return out


def extract_batch(envs, sigmas=None, maps=None, masks=None):
    """Stress (6, nt) and pressure map / mask (H, W) of every env in one
    launch (tc_extract_batch).  sigmas, maps, masks: lists of CUDA tensors (or
    None entries), one per env, or None to skip that output for all."""
    envs = list(envs)
    n = len(envs)
    lib = load()
    handles = (ctypes.c_void_p * max(n, 1))(*[e.h for e in envs])

    def ptrs(ts):
        if ts is None:
            return None
        return (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() if t is not None else None for t in ts])
    _check(lib.tc_extract_batch(handles, n, ptrs(sigmas), ptrs(maps), ptrs(masks)), "tc_extract_batch")


def stress_from_F(F, E, nu, out=None, stream=None):
    """sigma (6, n) from a CUDA float32 tensor F of shape (n, 9) or (n, 3, 3)."""
    torch = _torch()
    lib = load()
    n = F.shape[0]
    if out is None:
        out = torch.empty((6, n), dtype=torch.float32, device=F.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.tc_stress_from_F(ctypes.c_void_p(F.data_ptr()), n, E, nu, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(s.cuda_stream)), "tc_stress_from_F")
    return out


def pressure_map_noalloc(x, sigma, cfaces, cparent, cface_slot, cv_face_off, cv_face_idx, pix_face, pix_w, out,
                         mask=None, stream=None):
    """Pressure map from caller-owned CUDA tensors, with no device allocation
    inside the library (see tc_pressure_map_noalloc in include/tacauchy.h).
    x (3, nv) float32, sigma (6, nt) float32, cfaces / cface_slot (3, nfc)
    int32, cparent (nfc,) int32, cv_face_off (nvc+1,) int32, cv_face_idx int32,
    pix_face (npix,) int32, pix_w (3, npix) float32, out (npix,) float32,
    mask (npix,) uint8 or None."""
    torch = _torch()
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(lib.tc_pressure_map_noalloc(vp(x), x.shape[1], vp(sigma), sigma.shape[1], vp(cfaces), vp(cparent),
                                       vp(cface_slot), cfaces.shape[1], vp(cv_face_off), vp(cv_face_idx),
                                       cv_face_off.shape[0] - 1, vp(pix_face), vp(pix_w), pix_face.shape[0],
                                       vp(out), vp(mask), ctypes.c_void_p(s.cuda_stream)),
           "tc_pressure_map_noalloc")
    return out
